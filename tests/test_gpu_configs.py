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
