"""Incremental invocation of the interpreter on the GPU path against the
oracle: progressive sessions of tightening error-bound and PSNR targets
(pcr_plan_more through Progressive.refine) give the oracle's incremental
plans and, retrieved, the oracle's fields bit for bit; the bytes a session
adds sum to its final plan's bytes; a malformed starting plan is refused.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("sch_kw,kind,values", [
    (dict(mode="eb", interp="level", degree="cubic", decomp_axis=2), "rel", (1e-2, 1e-3, 1e-4, 1e-5)),
    (dict(mode="psnr", interp="region", degree="cubic", decomp_axis=0), "psnr", (40.0, 60.0, 80.0, 100.0)),
    (dict(mode="eb", interp="level", degree="cubic", decomp_axis=2), "psnr", (50.0, 70.0, 90.0)),
])
def test_progressive_session_matches_the_oracle(sch_kw, kind, values):
    import oracle
    import paper_2609_04573_b300 as pcr
    from synth import grf
    from _compare import oracle_scheme
    X = grf((33, 41, 58), 311, np.float32)
    sch = pcr.Scheme(**sch_kw)
    h = pcr.refactor(torch.from_numpy(X).cuda(), sch)
    h_or = oracle.refactor(X, oracle_scheme(sch, 3))
    sess = pcr.Progressive(h)
    prev_or = None
    for v in values:
        out, pl, added = sess.refine(pcr.Target(kind, v))
        pl_or = oracle.plan(h_or, oracle.Target(kind, v), have=prev_or)
        assert pl.planes == pl_or["b"], v
        assert pl.bytes == pl_or["bytes"]
        x_or, _ = oracle.retrieve(h_or, pl_or)
        assert np.array_equal(out.cpu().numpy(), x_or), v
        prev_or = pl_or
    assert sess.fetched == sess.plan.bytes


def test_malformed_starting_plan_is_refused():
    import paper_2609_04573_b300 as pcr
    from synth import grf
    X = grf((20, 24, 28), 312, np.float32)
    h = pcr.refactor(torch.from_numpy(X).cuda(), pcr.Scheme(interp="level", degree="cubic", decomp_axis=2))
    bad = h.plan_from_planes([0] * (h.nstreams - 1))
    with pytest.raises(pcr.PcrError):
        h.plan(pcr.Target("rel", 1e-3), have=bad)
    over = h.plan_from_planes([99] * h.nstreams)
    with pytest.raises(pcr.PcrError):
        h.plan(pcr.Target("rel", 1e-3), have=over)
