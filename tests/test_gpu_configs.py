"""The workload configurations as parity cases (CUDA path vs oracle, bit for
bit), at the sizes the oracle finishes in seconds.

* Plain method: the 64^3 FP32 sum of 8 Gaussians plus noise, per-level
  linear, 32 planes, retrievals at relative 1e-2, 1e-4, 1e-6 and with every
  plane.
* Precision variant (climate-like zonal bands x lognormal noise, reduced to
  32x48x96): refactored in FP64 with FP64 tables, retrievals down to 1e-9;
  the same field cast to FP32 and refactored in FP32, its error stated
  against the FP64 field (cast error + retrieval error).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _parity(X, sch, targets):
    import oracle
    import paper_2609_04573_b300 as pcr
    from _compare import oracle_scheme, compare_streams
    h_or = oracle.refactor(X, oracle_scheme(sch, X.ndim))
    h = pcr.refactor(torch.from_numpy(X).cuda(), sch)
    compare_streams(h, h_or)
    R = h_or["meta"]["R"]
    outs = {}
    for kind, v in targets:
        t = oracle.Target(kind, v)
        pl_or = oracle.plan(h_or, t)
        pl = h.plan(pcr.Target(kind, v), allow_unsat=True)
        assert pl.planes == pl_or["b"] and pl.bound == pl_or["bound"]
        x_or, _ = oracle.retrieve(h_or, pl_or)
        out, _ = h.retrieve(pl)
        got = out.cpu().numpy()
        assert np.array_equal(got, x_or), (kind, v)
        if pl.satisfied and kind in ("rel", "abs"):
            lim = v * R if kind == "rel" else v
            assert np.abs(got.astype(np.float64) - X.astype(np.float64)).max() <= lim
        outs[(kind, v)] = (got, pl)
    return h, outs, R


def test_plain_method_gaussians_64():
    import paper_2609_04573_b300 as pcr
    from synth import config_field
    X = config_field("c1_gaussians_64")
    assert X.shape == (64, 64, 64) and X.dtype == np.float32
    sch = pcr.Scheme(interp="level", degree="linear", nplanes=32)
    h, outs, R = _parity(X, sch, [("rel", 1e-2), ("rel", 1e-4), ("rel", 1e-6), ("abs", 0.0)])
    got, pl = outs[("abs", 0.0)]       # every plane
    assert all(b == h.stream_info(i)["nplanes"] for i, b in enumerate(pl.planes))
    assert np.abs(got.astype(np.float64) - X).max() <= pl.bound


def test_precision_variant_fp64_and_fp32_cast():
    import paper_2609_04573_b300 as pcr
    from synth import climate
    X64 = climate((32, 48, 96), 3, np.float64)
    sch = pcr.Scheme(interp="level", degree="cubic", decomp_axis=2)
    tg = [("rel", 10.0 ** -k) for k in range(3, 10)]
    _, outs64, R = _parity(X64, sch, tg)
    X32 = X64.astype(np.float32)
    cast = np.abs(X32.astype(np.float64) - X64).max()
    _, outs32, _ = _parity(X32, sch, tg[:4])
    for (kind, v), (got, pl) in outs32.items():
        if pl.satisfied:   # error against the FP64 field: cast error + retrieval error
            assert np.abs(got.astype(np.float64) - X64).max() <= cast + v * R * (1 + 1e-6)
    for (kind, v), (got, pl) in outs64.items():
        assert pl.satisfied, v


def test_precision_variant_fp64_larger():
    """The FP64 climate-like field at 64x96x128 (786 K points): streams,
    plans and retrieved fields bit-exact against the oracle at relative
    bounds 1e-3..1e-9; each retrieval's error measured against the FP64
    field stays within its bound."""
    import paper_2609_04573_b300 as pcr
    from synth import climate
    X64 = climate((64, 96, 128), 3, np.float64)
    sch = pcr.Scheme(interp="level", degree="cubic", decomp_axis=2)
    tg = [("rel", 10.0 ** -k) for k in range(3, 10)]
    _, outs64, R = _parity(X64, sch, tg)
    for (kind, v), (got, pl) in outs64.items():
        assert pl.satisfied, v
        assert np.abs(got - X64).max() <= v * R


def test_batch_shape_classes_match_the_oracle():
    """One field of each batched shape class (3-D slabs, 3-D elongated, 2-D),
    reduced to sizes the oracle finishes in seconds, through the batched
    refactor and the graph-captured batch: streams and tables bit-exact
    against the oracle, and a retrieval equal to the oracle's."""
    import oracle
    import paper_2609_04573_b300 as pcr
    from synth import grf
    from _compare import oracle_scheme, compare_streams
    shapes = [(25, 125, 125), (16, 64, 256), (450, 900)]
    Xs = [grf(s, 1000 + i, np.float32) for i, s in enumerate(shapes)]
    xs = [torch.from_numpy(X).cuda() for X in Xs]
    schs = [pcr.Scheme(interp="level", degree="cubic", decomp_axis=2 if X.ndim == 3 else -1) for X in Xs]
    hb = pcr.refactor_batch(xs, schs)
    g = pcr.RefactorGraph(xs, schs)
    g.run()
    for X, s, h1, h2 in zip(Xs, schs, hb, g.handles):
        h_or = oracle.refactor(X, oracle_scheme(s, X.ndim))
        compare_streams(h1, h_or)
        compare_streams(h2, h_or)
        pl_or = oracle.plan(h_or, oracle.Target("rel", 1e-4))
        x_or, _ = oracle.retrieve(h_or, pl_or)
        for h in (h1, h2):
            out, info = h.retrieve(pcr.Target("rel", 1e-4))
            assert info.planes == pl_or["b"]
            assert np.array_equal(out.cpu().numpy(), x_or)
