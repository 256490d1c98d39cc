"""Incremental invocation of the retrieval interpreter (oracle).

Progressive retrieval re-uses the planes it already fetched (Sec. III-A,
the refinement of an earlier retrieval): a tighter target is planned from
the earlier plan, never drops a plane, and pays only for the planes it
adds.  Checked on small fields of both interpolation families, for
error-bound and PSNR sessions of tightening targets:

* each plan contains the previous one, stream by stream;
* a satisfied plan's retrieval meets the target on the data itself (max
  error for error bounds, PSNR for PSNR targets), and its bound holds;
* from an empty plan the interpreter gives exactly the one-shot plan, and
  from the one-shot plan of the same target it adds nothing;
* the bytes added over a session sum to the final plan's bytes.
"""
import math

import numpy as np
import pytest

import oracle
from synth import grf

SCHEMES = [
    oracle.Scheme(mode="eb", interp="level", degree="cubic", decomp_axis=2),
    oracle.Scheme(mode="psnr", interp="region", degree="cubic", decomp_axis=0),
]


@pytest.fixture(scope="module", params=range(len(SCHEMES)))
def handle(request):
    X = grf((17, 22, 26), 301 + request.param, np.float32)
    return X, oracle.refactor(X, SCHEMES[request.param])


def _check(X, h, pl, t):
    x, _ = oracle.retrieve(h, pl)
    R = h["meta"]["R"]
    d = x.astype(np.float64) - X.astype(np.float64)
    if t.kind == "rel":
        err = float(np.abs(d).max())
        assert err <= pl["bound"] and err <= t.value * R, (t.value, err, pl["bound"])
    else:
        mse = float(np.mean(d * d))
        assert mse == 0 or 20 * math.log10(R / math.sqrt(mse)) >= t.value


@pytest.mark.parametrize("kind,values", [("rel", (1e-2, 1e-3, 1e-4, 1e-5)), ("psnr", (40.0, 60.0, 80.0, 100.0))])
def test_session_plans_grow_and_meet_their_targets(handle, kind, values):
    X, h = handle
    prev, spent = None, 0
    tabs = [s["tab"] for s in h["streams"]]
    for v in values:
        t = oracle.Target(kind, v)
        pl = oracle.plan(h, t, have=prev)
        if prev is not None:
            assert all(a >= b for a, b in zip(pl["b"], prev["b"])), (v, pl["b"], prev["b"])
            spent += pl["bytes"] - prev["bytes"]
        else:
            spent = pl["bytes"]
        assert pl["bytes"] == sum(tab["bytes"][bi] for tab, bi in zip(tabs, pl["b"]))
        if pl["satisfied"]:
            _check(X, h, pl, t)
        prev = pl
    assert spent == prev["bytes"]


@pytest.mark.parametrize("t", [oracle.Target("rel", 1e-3), oracle.Target("psnr", 70.0)])
def test_empty_and_complete_starting_plans(handle, t):
    X, h = handle
    one = oracle.plan(h, t)
    zero = oracle.plan(h, t, have=[0] * len(one["b"]))
    assert zero["b"] == one["b"] and zero["bound"] == one["bound"]
    again = oracle.plan(h, t, have=one)
    assert again["b"] == one["b"] and again["bytes"] == one["bytes"]


def test_a_looser_target_after_a_tight_one_adds_nothing(handle):
    X, h = handle
    tight = oracle.plan(h, oracle.Target("rel", 1e-5))
    loose = oracle.plan(h, oracle.Target("rel", 1e-2), have=tight)
    assert loose["b"] == tight["b"]
