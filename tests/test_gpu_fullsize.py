"""Parity at the full size of the bench's workload: the 512^3 FP32
turbulence-like field, per-level cubic interpolation, decomposition with
slices normal to the fastest axis, generic planes, B = 32 -- the
configuration and launch shapes bench.py times.  The oracle cannot refactor
the whole field in test time, so:

* sampled outputs: a level-0 coefficient depends on the field within 3
  points per axis (the cubic per-level passes) and its decomposed value on
  coefficients within 4 more points in the slice, so the oracle's level-0
  prediction and decomposition run on 64^3 windows whose origins are
  multiples of 8 (region and sub-level parities as in the whole field).
  Every level-0 element lying at least 8 points inside its window (or at a
  field edge) must carry, in the library's plane words, exactly the code
  the oracle's quantisation gives its value with the stream's exponent
  (the stream maximum is appended to the oracle's input so its E is the
  stream's).  Windows: the 8 field corners and 4 interior positions.
* properties that hold at any size: every retrieval within its bound for
  relative targets 1e-1..1e-7 and PSNR 40..120 dB, payload bytes never
  shrinking as the target tightens, and all planes within the all-planes
  bound.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 512


@pytest.fixture(scope="module")
def refactored():
    import paper_2609_04573_b300 as pcr
    from synth.device import grf_torch
    x = grf_torch((N, N, N), 2)
    sch = pcr.Scheme(mode="eb", interp="level", degree="cubic", decomp_axis=2)
    h = pcr.refactor(x, sch)
    torch.cuda.synchronize()
    return x, sch, h


def _codes(planes, e, B):
    w, b = e >> 5, (e & 31).astype(np.uint32)
    q = np.zeros(e.shape, np.uint64)
    for k in range(B):
        q |= ((planes[k, w] >> b) & 1).astype(np.uint64) << np.uint64(B - 1 - k)
    return q


def test_sampled_level0_codes_equal_the_oracle(refactored):
    import oracle.bitplane as bp
    from oracle.geometry import build_geometry, auto_levels, region_lattice, decomp_axes
    from oracle.interp import predict_level, level_points_mask, decompose
    x, sch, h = refactored
    X = x.cpu().numpy()
    shape3 = X.shape
    order = (0, 1, 2)
    geo = build_geometry(shape3, auto_levels(shape3), "level", order, 2)
    assert len(geo.streams) == h.nstreams
    lvl0 = [i for i, s in enumerate(geo.streams) if s.level == 0 and not s.is_int]
    assert lvl0 and all(geo.streams[i].sub > 0 for i in lvl0)
    gpu = {}
    for i in lvl0:
        info = h.stream_info(i)
        assert (info["level"], info["sub"]) == (0, geo.streams[i].sub)
        gpu[i] = (h.stream_copy(i)[0], info["nplanes"], np.float32(info["vmax"]))
    rng = np.random.default_rng(5)
    origins = [(a, b, c) for a in (0, N - 64) for b in (0, N - 64) for c in (0, N - 64)]
    origins += [tuple(int(v) * 8 for v in rng.integers(1, (N - 64) // 8, 3)) for _ in range(4)]
    checked = 0
    for o in origins:
        e = tuple(min(N, oa + 64) for oa in o)
        Xw = X[o[0]:e[0], o[1]:e[1], o[2]:e[2]]
        W = predict_level(Xw, order, "level", sch.degree)
        C = np.where(level_points_mask(Xw.shape, order), Xw - W, 0).astype(np.float32)
        D = np.zeros_like(C)
        for r in (1, 2, 3):
            sl = region_lattice(Xw.shape, 0, order, r).slices()
            D[sl] = decompose(C[sl].copy(), decomp_axes(2))
        lo = [oa if oa == 0 else oa + 8 for oa in o]
        hi = [ea if ea == N else ea - 8 for ea in e]
        for i in lvl0:
            planes, B, vmax = gpu[i]
            base = 0
            for lat in geo.streams[i].lattices:
                ks = []
                for a in range(3):
                    st, sp, cnt = lat.start[a], lat.step[a], lat.count[a]
                    k0 = max(0, -(-(lo[a] - st) // sp))
                    k1 = min(cnt - 1, (hi[a] - 1 - st) // sp)
                    ks.append(np.arange(k0, k1 + 1) if k1 >= k0 else np.zeros(0, np.int64))
                if all(len(k) for k in ks):
                    K0, K1, K2 = np.meshgrid(*ks, indexing="ij")
                    g = [lat.start[a] + lat.step[a] * K for a, K in enumerate((K0, K1, K2))]
                    vals = D[g[0] - o[0], g[1] - o[1], g[2] - o[2]].ravel()
                    elem = (base + (K0 * lat.count[1] + K1) * lat.row_pad + K2).ravel()
                    want = bp.quantize(np.append(vals, vmax), False, B, bp.GENERIC)["q"][:-1]
                    got = _codes(planes, elem, B)
                    bad = np.nonzero(got != want.astype(np.uint64))[0]
                    assert bad.size == 0, (o, i, int(elem[bad[0]]), int(got[bad[0]]), int(want[bad[0]]))
                    checked += vals.size
                base += lat.n_pad
    assert checked > 500_000


def test_full_size_retrievals_within_bound(refactored):
    import paper_2609_04573_b300 as pcr
    x, sch, h = refactored
    xmin, xmax, _ = h.field_stats()
    R = xmax - xmin
    xd = x.double()
    prev = -1
    for v in (1e-1, 1e-2, 1e-3, 1e-4, 1e-5, 1e-6, 1e-7):
        pl = h.plan(pcr.Target("rel", v), allow_unsat=True)
        assert pl.bytes >= prev
        prev = pl.bytes
        if pl.satisfied:
            out, _ = h.retrieve(pl)
            err = (out.double() - xd).abs().max().item()
            assert err <= v * R, (v, err)
            assert err <= pl.bound
    prev = -1
    for db in (40.0, 60.0, 80.0, 100.0, 120.0):
        pl = h.plan(pcr.Target("psnr", db), allow_unsat=True)
        assert pl.bytes >= prev
        prev = pl.bytes
        if pl.satisfied:
            out, _ = h.retrieve(pl)
            mse = ((out.double() - xd) ** 2).mean().item()
            assert mse == 0 or 20 * np.log10(R / np.sqrt(mse)) >= db, (db, mse)
    pl = h.plan(pcr.Target("abs", 0.0), allow_unsat=True)
    out, _ = h.retrieve(pl)
    assert (out.double() - xd).abs().max().item() <= pl.bound
