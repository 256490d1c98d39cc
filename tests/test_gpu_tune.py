"""Target-driven sampled tuning on the GPU (Sec. VI-A): the library's tuner
samples the same blocks, refactors them with every candidate on the GPU,
plans every tolerance with the library's interpreter and must cast exactly
the oracle tuner's votes (same byte counts) and pick its scheme; a refactor
asking for the tuner (PCR_INTERP_AUTO) equals the refactor with the chosen
scheme."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _to_oracle(s, ndim):
    from oracle.pipeline import Scheme as OS
    order = s.order
    if order is not None and ndim == 2:
        order = tuple(a + 1 for a in order)
    return OS(mode=s.mode, interp=s.interp, degree=s.degree, order=order if s.interp == "region" else None,
              decomp_axis=s.decomp_axis, encoding=s.encoding)


def _anisotropic(n=48, seed=4):
    rng = np.random.default_rng(seed)
    i0, i1, i2 = np.meshgrid(*[np.arange(n)] * 3, indexing="ij")
    g = np.sin(i0 / 7.0) * np.cos(i1 / 9.0) + 0.5 * np.sin((i0 + i1) / 11.0)
    h = rng.standard_normal(n)[None, None, :]
    return (g * (1.0 + 0.5 * h) + 0.2 * np.sin(i2 / 5.0)).astype(np.float32)


@pytest.mark.parametrize("case", ["aniso_eb", "grf2d_psnr", "grf_eb_sample"])
def test_tuner_votes_equal_the_oracle(case):
    import paper_2609_04573_b300 as pcr
    from oracle import tune as tn
    from synth import grf
    if case == "aniso_eb":
        X, mode, frac, edge = _anisotropic(), "eb", 1.0, 48
    elif case == "grf2d_psnr":
        X, mode, frac, edge = grf((200, 300), 91, np.float32), "psnr", 0.05, 32
    else:
        X, mode, frac, edge = grf((128, 128, 128), 92, np.float32), "eb", 0.01, 48
    win, info = pcr.tune(torch.from_numpy(X).cuda(), mode, fraction=frac, edge=edge)
    origins, b = tn.sample_blocks(X.shape, frac, edge)
    assert info["nblocks"] == len(origins) and info["block"] == b
    cands = [_to_oracle(c, X.ndim) for c in info["candidates"]]
    assert cands == tn.candidates(mode, X.ndim)
    w_or, votes, table = tn.tune(X, mode, fraction=frac, edge=edge, cands=cands)
    assert info["bytes"] == table
    assert info["votes"] == votes
    assert _to_oracle(win, X.ndim) == w_or
    if case == "aniso_eb":
        assert win.decomp_axis == 2          # slices normal to the rough axis


def test_auto_refactor_equals_the_tuned_scheme():
    import paper_2609_04573_b300 as pcr
    from _compare import compare_streams
    import oracle
    X = _anisotropic(40, 6)
    x = torch.from_numpy(X).cuda()
    win, _ = pcr.tune(x, "eb")
    h = pcr.refactor(x, pcr.Scheme(mode="eb", interp="auto"))
    got = h.scheme()
    assert (got.interp, got.order, got.decomp_axis, got.encoding) == (win.interp, win.order, win.decomp_axis,
                                                                      win.encoding)
    compare_streams(h, oracle.refactor(X, _to_oracle(got, 3)))
