"""Block sharding of one field (oracle): axis-0 slabs refactored
independently, planned together for a whole-field target.

Pins:
* slabs partition axis 0 (contiguous, sizes differ by at most one);
* one block: the global plan is the block's own plan, for error-bound and
  PSNR targets alike;
* several blocks: the assembled retrieval meets the whole-field target on
  the data (max error within rel * R of the whole field; PSNR of the
  whole field at least the target), and the PSNR plan's summed bound is
  within its budget;
* the PSNR budget is spent where it buys most: a block that is exactly
  zero (every plane free of error at b = 0) gets no planes while the rest
  share the budget.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import shard
from synth import grf

SCH = oracle.Scheme(mode="eb", interp="level", degree="cubic", decomp_axis=2)


def test_slabs_partition_axis0():
    X = np.zeros((23, 4, 4), np.float32)
    for k in (1, 2, 3, 5, 23):
        sl = shard.split(X, k)
        assert sl[0][0] == 0 and sl[-1][1] == 23
        assert all(a[1] == b[0] for a, b in zip(sl, sl[1:]))
        sizes = [b - a for a, b in sl]
        assert max(sizes) - min(sizes) <= 1 and len(sl) == k


@pytest.mark.parametrize("t", [oracle.Target("rel", 1e-3), oracle.Target("psnr", 70.0)])
def test_one_block_is_the_plain_plan(t):
    X = grf((18, 22, 26), 401, np.float32)
    hs, sl = shard.refactor_blocks(X, SCH, 1)
    pls, bound, ok = shard.plan_global(hs, t)
    one = oracle.plan(hs[0], t)
    assert pls[0]["b"] == one["b"] and ok == one["satisfied"]


@pytest.mark.parametrize("k", [2, 3])
@pytest.mark.parametrize("t", [oracle.Target("rel", 1e-2), oracle.Target("rel", 1e-4),
                               oracle.Target("psnr", 50.0), oracle.Target("psnr", 80.0)])
def test_blocks_meet_the_whole_field_target(k, t):
    X = grf((24, 20, 28), 402, np.float32)
    hs, sl = shard.refactor_blocks(X, SCH, k)
    pls, bound, ok = shard.plan_global(hs, t)
    assert ok
    Y = shard.retrieve_blocks(hs, sl, pls, X.shape, X.dtype)
    R = float(X.max()) - float(X.min())
    assert R == shard.field_range(hs)
    d = Y.astype(np.float64) - X.astype(np.float64)
    if t.kind == "rel":
        assert float(np.abs(d).max()) <= t.value * R
    else:
        budget = X.size * (R / 10 ** (t.value / 20)) ** 2
        assert bound <= budget
        mse = float(np.mean(d * d))
        assert mse == 0 or 20 * math.log10(R / math.sqrt(mse)) >= t.value


def test_psnr_budget_skips_a_zero_block():
    X = grf((24, 20, 28), 403, np.float32)
    X[:12] = 0.0
    hs, sl = shard.refactor_blocks(X, SCH, 2)
    pls, bound, ok = shard.plan_global(hs, oracle.Target("psnr", 60.0))
    assert ok and sum(pls[0]["b"]) == 0 and sum(pls[1]["b"]) > 0
