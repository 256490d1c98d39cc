"""Every level schedule against the oracle.

The autotuner picks, per level grid, the general tile kernel or the plane-
marching kernel with one of several plane chunks, or with TMA-staged
inputs (-2; -3 on 16 x 64 columns for FP32; register prefetch where the TMA
form does not apply); all of them must compute identical values.  The autotune test checks only the schedule that won, so
here each candidate is pinned in turn (pcr_autotune_set) for level 0 (FP32)
and level 1 (fixed point), in both directions, and the refactored streams
and the retrieved field are compared with the oracle bit for bit.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CHOICES = (0, 8, 16, 32, 64, -1, -2, -3)


def test_every_pinned_schedule_matches_the_oracle():
    import oracle
    import paper_2609_04573_b300 as pcr
    from synth import grf
    from _compare import oracle_scheme, compare_streams
    X = grf((37, 45, 260), 171, np.float32)
    sch = pcr.Scheme(interp="level", degree="cubic", decomp_axis=2)
    h_or = oracle.refactor(X, oracle_scheme(sch, 3))
    pl_or = oracle.plan(h_or, oracle.Target("rel", 1e-4))
    x_or, _ = oracle.retrieve(h_or, pl_or)
    x = torch.from_numpy(X).cuda()
    m0 = X.shape
    m1 = tuple((n - 1) // 2 + 1 for n in X.shape)
    keys = [(0, r, 3, 0) + m0 for r in (0, 1)] + [(2, r, 3, 0) + m1 for r in (0, 1)]
    pcr.autotune(False)
    pcr.autotune_table(reset=True)
    try:
        for c in CHOICES:
            for k in keys:
                pcr.autotune_pin(k, c)
            h = pcr.refactor(x, sch)
            compare_streams(h, h_or)
            out, pl = h.retrieve(pcr.Target("rel", 1e-4))
            assert pl.planes == pl_or["b"], c
            assert np.array_equal(out.cpu().numpy(), x_or), c
            table = pcr.autotune_table()
            assert all(table[k][0] == c for k in keys), (c, table)
            assert pcr.device_status() == 0
    finally:
        pcr.autotune_table(reset=True)


def test_pin_rejects_unknown_choices():
    import paper_2609_04573_b300 as pcr
    with pytest.raises(pcr.PcrError):
        pcr.autotune_pin((0, 0, 3, 0, 8, 8, 8), 7)
    with pytest.raises(pcr.PcrError):
        pcr.autotune_pin((5, 0, 3, 0, 8, 8, 8), -1)
    pcr.autotune_table(reset=True)
