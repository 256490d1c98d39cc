"""CUDA path vs CPU oracle, element by element, on seeded inputs that span
several 4096-element segments, ragged row tails and the degenerate cases.

Bars: quantised integers, bitplanes, sign sub-streams and integer
table sums bit-exact; coefficients equal because both sides evaluate the same
expression trees in the same precision; every retrieval within its bound.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import Target as OTarget  # noqa: E402
from synth import grf, gaussians  # noqa: E402

from _compare import oracle_scheme, compare_streams, psnr  # noqa: E402


def _pcr():
    import paper_2609_04573_b300 as pcr
    return pcr


CASES = [
    # (shape, dtype, scheme kwargs)
    ((33, 45, 67), np.float32, dict(interp="level", degree="linear")),
    ((33, 45, 67), np.float32, dict(interp="level", degree="cubic", decomp_axis=2)),
    ((29, 38, 70), np.float32, dict(mode="psnr", interp="region", degree="cubic", decomp_axis=0)),
    ((31, 36, 41), np.float32, dict(interp="region", degree="linear", order=(2, 0, 1), decomp_axis=1)),
    ((17, 20, 33), np.float64, dict(interp="level", degree="cubic", decomp_axis=2)),
    ((17, 21, 35), np.float64, dict(mode="psnr", interp="region", degree="cubic")),
    ((130, 257), np.float32, dict(interp="level", degree="cubic")),
    ((97, 130), np.float64, dict(mode="psnr", interp="region", degree="linear", order=(1, 0))),
    ((9, 9, 9), np.float32, dict(mode="psnr", interp="level", degree="cubic", encoding="generic")),
    ((2, 3, 2), np.float32, dict(interp="level", degree="linear")),
    ((5, 5, 5), np.float32, dict(interp="region", degree="cubic", nlevels=1)),
    ((12, 10, 9), np.float32, dict(interp="level", degree="cubic", nplanes=6, nlevels=3)),
    # rows of whole 16-byte vectors: level 0 runs the plane-marching kernel
    # (ragged column tiles along both in-plane axes, several plane chunks)
    ((37, 45, 260), np.float32, dict(interp="level", degree="cubic", decomp_axis=2)),
    ((36, 33, 132), np.float32, dict(interp="level", degree="linear")),
    ((18, 20, 66), np.float64, dict(interp="level", degree="cubic", decomp_axis=1)),
    ((24, 17, 40), np.float32, dict(mode="psnr", interp="level", degree="cubic")),
    # B not a multiple of 4 with whole 4096-value segments: plane rows of
    # later streams start off 16-byte boundaries
    ((40, 52, 70), np.float32, dict(interp="level", degree="cubic", decomp_axis=2, nplanes=6)),
    # per-region in pass order (0, 1, 2) on rows of whole 16-byte vectors:
    # the plane-marching kernel with original / reconstructed sources
    ((36, 40, 68), np.float32, dict(interp="region", degree="cubic", decomp_axis=2)),
    ((34, 30, 64), np.float32, dict(mode="psnr", interp="region", degree="linear")),
    ((20, 24, 34), np.float64, dict(interp="region", degree="cubic")),
]


def _field(shape, dtype, seed):
    return grf(shape, seed, dtype) if len(shape) == 3 and min(shape) > 4 else \
        gaussians(shape, seed, dtype=np.float64).astype(dtype)


@pytest.mark.parametrize("ci", range(len(CASES)))
def test_refactor_retrieve_parity(ci):
    pcr = _pcr()
    shape, dtype, kw = CASES[ci]
    X = _field(shape, dtype, 100 + ci)
    sch = pcr.Scheme(**kw)
    h_or = oracle.refactor(X, oracle_scheme(sch, X.ndim))
    xt = torch.from_numpy(X).cuda()
    h = pcr.refactor(xt, sch)
    torch.cuda.synchronize()
    xmin, xmax, G = h.field_stats()
    assert (xmin, xmax, G) == (h_or["meta"]["xmin"], h_or["meta"]["xmax"], h_or["meta"]["G"])
    compare_streams(h, h_or)
    if h_or["M0"] is not None:
        init, segs = h_or["M0"]
        assert h.max_ordering() == [init] + [s[2] for s in segs]
    R = h_or["meta"]["R"]
    targets = [OTarget("rel", v) for v in (1e-1, 1e-3, 1e-5, 1e-7)] + \
              [OTarget("psnr", v) for v in (40.0, 80.0, 120.0)]
    for t in targets:
        pl_or = oracle.plan(h_or, t)
        pl = h.plan(pcr.Target(t.kind, t.value), allow_unsat=True)
        assert pl.planes == pl_or["b"], (t, pl.planes, pl_or["b"])
        assert pl.bound == pl_or["bound"] and pl.satisfied == pl_or["satisfied"]
        assert pl.bytes == pl_or["bytes"]
        x_or, _ = oracle.retrieve(h_or, pl_or)
        out, _ = h.retrieve(pl)
        got = out.cpu().numpy()
        assert np.array_equal(got, x_or), f"retrieval differs for {t}"
        if pl.satisfied:
            err = np.abs(got.astype(np.float64) - X.astype(np.float64)).max()
            if t.kind == "rel":
                assert err <= t.value * R
            else:
                assert psnr(got, X, R) >= t.value


@pytest.mark.parametrize("kind,enc,B", [(0, 1, 32), (0, 2, 32), (1, 1, 64), (1, 2, 64),
                                        (2, 1, 32), (2, 2, 32), (2, 1, 64), (2, 2, 64), (0, 1, 7)])
def test_encode_oracle_coefficients_bit_exact(kind, enc, B):
    """pcr_debug_encode fed the oracle's values: planes, signs, counts and
    pair counts are bit-exact (value kinds: f32, f64, fixed point)."""
    pcr = _pcr()
    from oracle import bitplane as bp
    rng = np.random.default_rng(kind * 10 + enc + B)
    n = 3 * 4096 + 96
    if kind == 0:
        v = (rng.standard_normal(n) * np.exp(rng.uniform(-10, 0, n))).astype(np.float32)
    elif kind == 1:
        v = rng.standard_normal(n) * np.exp(rng.uniform(-20, 0, n))
    else:
        v = rng.integers(-(1 << 44), 1 << 44, size=n).astype(np.int64)
    v[::9] = 0
    encname = "generic" if enc == 1 else "negabinary"
    e = bp.encode(v, kind == 2, B, encname, True)
    got = pcr.debug_encode(torch.from_numpy(v).cuda(), kind, B, enc, True)
    assert np.array_equal(got["planes"], e["planes"])
    assert list(got["plane_nz"]) == e["plane_nz"]
    if enc == 1:
        assert np.array_equal(got["sign_counts"].astype(np.int64), e["sign_counts"])
        for g in range(got["sign_counts"].shape[0]):
            want = np.concatenate(e["signs"][g])
            assert np.array_equal(got["signs"][g, :want.size], want)
    C = e["pairs"]
    for a in range(B):
        for b in range(a, B):
            assert int(got["pairs"][a, b]) == int(C[a, b])


@pytest.mark.parametrize("enc,B,lg", [(1, 32, -120), (2, 32, -120), (1, 7, -130), (2, 4, 126),
                                      (1, 1, 126), (1, 32, 126), (2, 32, 0)])
def test_encode_f32_without_pairs_bit_exact(enc, B, lg):
    """FP32 streams without pair tables (the persistent encoder): planes,
    signs and counts bit-exact, down to subnormal values (scaling 2^k with
    k > 127) and up to near the largest float (k at or below -126 for small
    B), over whole segments and a ragged last one."""
    pcr = _pcr()
    from oracle import bitplane as bp
    rng = np.random.default_rng(1000 + enc * 100 + B + lg)
    n = 5 * 4096 + 160
    v = rng.standard_normal(n) * np.exp(rng.uniform(-12, 0, n)) * 2.0 ** lg
    v = np.clip(v, -3.0e38, 3.0e38).astype(np.float32)
    v[::7] = 0
    v[4096:8192] = 0                          # a segment with no significant value
    encname = "generic" if enc == 1 else "negabinary"
    e = bp.encode(v, False, B, encname, False)
    got = pcr.debug_encode(torch.from_numpy(v).cuda(), 0, B, enc, False)
    assert np.array_equal(got["planes"], e["planes"])
    assert list(got["plane_nz"]) == e["plane_nz"]
    if enc == 1:
        assert np.array_equal(got["sign_counts"].astype(np.int64), e["sign_counts"])
        for g in range(got["sign_counts"].shape[0]):
            want = np.concatenate(e["signs"][g])
            assert np.array_equal(got["signs"][g, :want.size], want)


@pytest.mark.parametrize("lg,kw", [(-120, dict(interp="level", degree="cubic", decomp_axis=2)),
                                   (-120, dict(mode="psnr", interp="level", degree="cubic")),
                                   (100, dict(interp="level", degree="cubic", decomp_axis=2))])
def test_extreme_magnitude_fields_parity(lg, kw):
    """Fields of tiny (subnormal coefficients) and huge magnitude: streams,
    plans and retrievals equal the oracle's (quantisation scale 2^k outside
    the normal range on one side, dequantisation on the other)."""
    pcr = _pcr()
    X = (grf((33, 40, 64), 77, np.float64) * 2.0 ** lg).astype(np.float32)
    sch = pcr.Scheme(**kw)
    h_or = oracle.refactor(X, oracle_scheme(sch, X.ndim))
    h = pcr.refactor(torch.from_numpy(X).cuda(), sch)
    torch.cuda.synchronize()
    compare_streams(h, h_or)
    targets = [OTarget("rel", v) for v in (1e-2, 1e-5)] + [OTarget("psnr", v) for v in (60.0,)]
    for t in targets:
        pl_or = oracle.plan(h_or, t)
        pl = h.plan(pcr.Target(t.kind, t.value), allow_unsat=True)
        assert pl.planes == pl_or["b"] and pl.bound == pl_or["bound"]
        x_or, _ = oracle.retrieve(h_or, pl_or)
        out, _ = h.retrieve(pl)
        assert np.array_equal(out.cpu().numpy(), x_or), f"retrieval differs for {t}"


def test_serialize_round_trip():
    pcr = _pcr()
    X = grf((20, 24, 33), 7, np.float32)
    h = pcr.refactor(torch.from_numpy(X).cuda(), pcr.Scheme(interp="level", degree="cubic", decomp_axis=2))
    blob = h.serialize()
    h2 = pcr.deserialize(blob)
    t = pcr.Target("rel", 1e-4)
    a, pa = h.retrieve(t)
    b, pb = h2.retrieve(t)
    assert pa.planes == pb.planes
    assert torch.equal(a, b)
    bad = bytearray(blob)
    bad[-5] ^= 0xFF
    with pytest.raises(pcr.PcrError):
        pcr.deserialize(bytes(bad))
    with pytest.raises(pcr.PcrError):
        pcr.deserialize(blob[:-9])


def test_unsatisfiable_and_invalid_args():
    pcr = _pcr()
    X = grf((17, 17, 17), 8, np.float32)
    h = pcr.refactor(torch.from_numpy(X).cuda(), pcr.Scheme(degree="cubic"))
    with pytest.raises(pcr.Unsatisfiable):
        h.plan(pcr.Target("rel", 1e-12))
    pl = h.plan(pcr.Target("rel", 1e-12), allow_unsat=True)
    assert not pl.satisfied and pl.planes and max(pl.planes) > 0
    bad = torch.full((8, 8, 8), float("nan"), device="cuda")
    with pytest.raises(pcr.PcrError):
        pcr.refactor(bad)
    with pytest.raises(ValueError):
        pcr.refactor(torch.zeros(4, 4, 4, dtype=torch.float16, device="cuda"))
    with pytest.raises(pcr.PcrError):
        pcr.refactor(torch.zeros(1, 4, 4, device="cuda"))
