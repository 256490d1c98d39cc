"""Best-first search interpreter (pcr_plan_search) against the oracle's
(oracle.bounds.best_first), on handles refactored on the GPU:

* the same planes, bytes, bound and search statistics (expansions, proof,
  greedy bytes) for error-bound and PSNR targets, per-level with
  decomposition and per-region, under a small expansion budget (the two
  searches must expand the same states in the same order) and on a small
  field where the search runs to its proof;
* from fetched planes (incremental invocation) likewise;
* the searched plan never costs more than the greedy plan, retrieves
  within its target, and equals the oracle's retrieval of the same plan.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SCHEMES = [
    (dict(mode="eb", interp="level", degree="cubic", decomp_axis=2), "rel", (1e-2, 1e-4)),
    (dict(mode="psnr", interp="region", degree="cubic", decomp_axis=0), "psnr", (40.0, 80.0)),
    (dict(mode="eb", interp="level", degree="cubic", decomp_axis=2), "psnr", (50.0,)),
    (dict(mode="eb", interp="region", degree="linear"), "rel", (1e-3,)),
]


def _pair(shape, seed, sch_kw):
    import oracle
    import paper_2609_04573_b300 as pcr
    from synth import grf
    from _compare import oracle_scheme
    X = grf(shape, seed, np.float32)
    sch = pcr.Scheme(**sch_kw)
    h = pcr.refactor(torch.from_numpy(X).cuda(), sch)
    return X, h, oracle.refactor(X, oracle_scheme(sch, len(shape)))


def _same(pl, info, pl_or):
    assert pl.planes == pl_or["b"]
    assert pl.bytes == pl_or["bytes"]
    assert pl.bound == pl_or["bound"]
    s = pl_or["search"]
    assert (info["expanded"], info["optimal"], info["greedy_bytes"]) == (s["expanded"], s["optimal"], s["greedy_bytes"])


@pytest.mark.parametrize("sch_kw,kind,values", SCHEMES)
def test_search_matches_the_oracle(sch_kw, kind, values):
    import oracle
    import paper_2609_04573_b300 as pcr
    X, h, h_or = _pair((33, 41, 58), 411, sch_kw)
    for v in values:
        t = pcr.Target(kind, v)
        pl, info = h.plan_search(t, max_nodes=300)
        pl_or = oracle.plan(h_or, oracle.Target(kind, v), search=300)
        _same(pl, info, pl_or)
        g = h.plan(t)
        assert pl.bytes <= g.bytes and info["greedy_bytes"] == g.bytes
        out, _ = h.retrieve(pl)
        x_or, _ = oracle.retrieve(h_or, pl_or)
        assert np.array_equal(out.cpu().numpy(), x_or)
        if kind == "rel":
            err = np.abs(out.cpu().numpy().astype(np.float64) - X).max()
            assert err <= v * (X.max() - X.min())


def test_search_to_its_proof_and_from_fetched_planes():
    import oracle
    import paper_2609_04573_b300 as pcr
    X, h, h_or = _pair((12, 10, 9), 5, dict(mode="explicit", interp="region", degree="cubic", nlevels=2, nplanes=10))
    for kind, v in (("rel", 1e-1), ("psnr", 40.0), ("rel", 3e-2)):
        pl, info = h.plan_search(pcr.Target(kind, v), max_nodes=10 ** 6)
        pl_or = oracle.plan(h_or, oracle.Target(kind, v), search=10 ** 6)
        _same(pl, info, pl_or)
        assert info["optimal"]
    first = h.plan(pcr.Target("rel", 1e-1))
    first_or = oracle.plan(h_or, oracle.Target("rel", 1e-1))
    pl, info = h.plan_search(pcr.Target("rel", 1e-2), max_nodes=10 ** 6, have=first)
    pl_or = oracle.plan(h_or, oracle.Target("rel", 1e-2), have=first_or, search=10 ** 6)
    _same(pl, info, pl_or)
    assert all(a >= b for a, b in zip(pl.planes, first.planes))


def test_search_arguments():
    import paper_2609_04573_b300 as pcr
    X, h, _ = _pair((20, 24, 28), 7, dict(mode="eb", interp="level", degree="cubic", decomp_axis=2))
    with pytest.raises(pcr.PcrError):
        h.plan_search(pcr.Target("rel", 1e-3), max_nodes=-1)
    bad = h.plan_from_planes([0] * (h.nstreams - 1))
    with pytest.raises(pcr.PcrError):
        h.plan_search(pcr.Target("rel", 1e-3), have=bad)
    pl, info = h.plan_search(pcr.Target("rel", 1e-30), allow_unsat=True)
    assert not pl.satisfied and pl.planes == h.plan(pcr.Target("rel", 1e-30), allow_unsat=True).planes
