"""Pins of the CPU oracle against facts the paper and the mathematics fix.

None of these re-types the oracle's own formula: each checks a closed form, a
different construction of the same quantity, an invariant or brute force.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import Scheme, Target, bitplane as bp, bounds as bd, interp as ip
from oracle.geometry import (auto_levels, build_geometry, region_lattice,
                             coarse_lattice, WORD)
from oracle.pipeline import to_fixed, from_fixed, fixed_scale
from synth import grf, gaussians, polynomial

GOLDEN = __file__.replace("test_oracle_pins.py", "golden")


# ---------------------------------------------------------------- geometry
def test_levels_partition_every_point():
    """Sec. IV: levels are disjoint and together hold every point once."""
    for shape in [(1, 17, 33), (9, 8, 13), (17, 17, 17), (5, 6, 7)]:
        for interp, order in [("level", None), ("region", (2, 0, 1))]:
            act = tuple(a for a in range(3) if shape[a] > 1)
            o = order if (order and len(act) == 3) else act
            if interp == "level":
                o = act
            L = auto_levels(shape)
            g = build_geometry(shape, L, interp, o, -1)
            hits = np.zeros(shape, dtype=int)
            for s in g.streams:
                for lat in s.lattices:
                    hits[lat.slices()] += 1
            assert (hits == 1).all()


def test_region3_shape_matches_fig4():
    """Fig. 4: region 3 of the finest level of a 500^3 field is 500x500x250."""
    lat = region_lattice((500, 500, 500), 0, (0, 1, 2), 3)
    assert lat.count == (500, 500, 250)
    assert region_lattice((500, 500, 500), 0, (0, 1, 2), 1).count == (250, 250, 250)


def test_region_count_3L_minus_2_plus_1():
    """Sec. V-C: per-region interpolation yields 3(L-1)+1 regions."""
    for L in (2, 3, 5):
        g = build_geometry((33, 33, 33), L, "region", (0, 1, 2), -1)
        assert len(g.streams) == 3 * (L - 1) + 1
    g = build_geometry((33, 33, 33), 4, "region", (0, 1, 2), 2)
    # each decomposed region splits into three (Sec. V-C)
    assert len(g.streams) == 3 * (4 - 1) + 1 + 2 * 3


def test_decomposition_sublevels_partition_region():
    g = build_geometry((12, 19, 23), 3, "level", (0, 1, 2), 2)
    hits = np.zeros((12, 19, 23), dtype=int)
    for s in g.streams:
        if s.level == 0:
            for lat in s.lattices:
                hits[lat.slices()] += 1
    lvl0 = np.ones((12, 19, 23), bool)
    lvl0[::2, ::2, ::2] = False
    assert (hits[lvl0] == 1).all() and (hits[~lvl0] == 0).all()


def test_rows_padded_to_words():
    g = build_geometry((10, 11, 37), 3, "level", (0, 1, 2), -1)
    for s in g.streams:
        assert s.n_pad % WORD == 0 and s.n_pad >= s.n_real


# ---------------------------------------------------------- interpolation
def _direct_multilinear(G):
    """Sec. IV: edge, face and cube centres are the means of 2, 4 and 8
    coarse corners -- computed here directly from corners with Fractions."""
    out = {}
    m = G.shape
    for idx in itertools.product(*[range(k) for k in m]):
        if all(i % 2 == 0 for i in idx):
            continue
        corners = []
        for a in itertools.product(*[((i - 1, i + 1) if i % 2 else (i,)) for i in idx]):
            corners.append(Fraction(int(G[a])))
        out[idx] = sum(corners) / len(corners)
    return out


def test_per_level_linear_equals_2_4_8_means():
    """Sec. VI-C: sequential per-axis passes reading predictions equal the
    direct edge / face / cube means of the coarse corners."""
    rng = np.random.default_rng(7)
    G = rng.integers(-64, 64, size=(5, 7, 9)).astype(np.float64)
    W = ip.predict_level(G, (0, 1, 2), "level", "linear")
    for idx, val in _direct_multilinear(G).items():
        assert Fraction(W[idx]) == val, idx


def test_golden_linear_cube():
    """tests/golden/linear_centres.txt: hand-computed 3x3x3 example of the
    2 / 4 / 8-point means (Sec. IV, Fig. 2 top row)."""
    rows = [l.split() for l in open(f"{GOLDEN}/linear_centres.txt")
            if l.strip() and not l.startswith("#")]
    G = np.zeros((3, 3, 3))
    want = {}
    for r in rows:
        i, j, k, v = int(r[1]), int(r[2]), int(r[3]), float(r[4])
        if r[0] == "corner":
            G[i, j, k] = v
        else:
            want[(i, j, k)] = v
    W = ip.predict_level(G, (0, 1, 2), "level", "linear")
    for idx, v in want.items():
        assert W[idx] == v, idx


@pytest.mark.parametrize("interp", ["level", "region"])
def test_polynomial_reproduction_float(interp):
    """Cubic rules reproduce quadratics everywhere and cubics in the
    interior; linear rules reproduce affine fields (n = 2^k + 1 so no line
    ends in a one-sided constant rule)."""
    n = 17
    for degree, pdeg, tol in [("linear", 1, 1e-12), ("cubic", 2, 1e-11)]:
        X = polynomial((n, n, n), 3, pdeg)
        W = ip.predict_level(X, (0, 1, 2), interp, degree)
        assert np.abs(X - W).max() < tol
    # a full cubic is reproduced at points whose every pass used the 4-point rule
    X = polynomial((n, n, n), 4, 3)
    W = ip.predict_level(X, (0, 1, 2), interp, "cubic")
    inner = (slice(4, n - 4),) * 3
    assert np.abs(X - W)[inner].max() < 1e-11


def test_polynomial_reproduction_fixed_point():
    """Exact integer passes: floors lose less than one quantum per pass."""
    n = 17
    X = polynomial((n, n, n), 5, 2)
    G, h = fixed_scale(float(np.abs(X).max()))
    Xi = to_fixed(X, G)
    for degree in ("linear", "cubic"):
        src = Xi if degree == "cubic" else to_fixed(polynomial((n, n, n), 6, 1), G)
        W = ip.predict_level(src[::2, ::2, ::2].copy(), (0, 1, 2), "level", degree)
        C = src[::2, ::2, ::2] - W
        assert np.abs(C).max() <= 8 + 2  # conversion floor + three pass floors


def test_per_region_uses_originals():
    """Sec. IV: per-region predicts region 2 from *original* region-1 values."""
    rng = np.random.default_rng(3)
    X = rng.standard_normal((9, 9, 9))
    W = ip.predict_level(X, (0, 1, 2), "region", "linear")
    # a region-2 point (i0 odd, i1 odd, i2 even)
    i0, i1, i2 = 3, 5, 4
    assert W[i0, i1, i2] == (X[i0, i1 - 1, i2] + X[i0, i1 + 1, i2]) * 0.5
    Wl = ip.predict_level(X, (0, 1, 2), "level", "linear")
    assert Wl[i0, i1, i2] != W[i0, i1, i2]


def test_lebesgue_constants():
    """Lam = max row sum of |weights| of every 1-D rule."""
    for degree, lam in (("linear", 1.0), ("cubic", 1.25)):
        for m in (3, 5, 6, 9, 33):
            P = bd.pass_matrix(m, degree)
            assert np.abs(P).sum(axis=1).max() <= lam + 1e-15
            assert abs(P.sum(axis=1) - 1).max() < 1e-15   # constants reproduced


def test_rowsum_upper_bounds_spectral_norm():
    for degree in ("linear", "cubic"):
        for m in (5, 8, 17, 64):
            P = bd.pass_matrix(m, degree)
            s = np.linalg.norm(P, 2) ** 2
            assert s <= bd.rowsum_ptp(m, degree) + 1e-12


# ----------------------------------------------------------- decomposition
@pytest.mark.parametrize("shape,axis", [((9, 13, 7), 2), ((16, 11, 10), 0), ((6, 9, 17), 1)])
def test_decompose_recompose_identity(shape, axis):
    """Alg. 2 inverts Alg. 1's coefficient decomposition exactly (values on a
    dyadic grid so every operation is exact)."""
    rng = np.random.default_rng(11)
    A = rng.integers(-1000, 1000, size=shape).astype(np.float64)
    uv = tuple(a for a in range(3) if a != axis)
    D = ip.decompose(A, uv)
    assert (D[tuple(slice(0, None, 4) if a in uv else slice(None) for a in range(3))]
            == A[tuple(slice(0, None, 4) if a in uv else slice(None) for a in range(3))]).all()
    R = ip.recompose(D, uv)
    assert (R == A).all()


def test_decomposition_annihilates_affine_slices():
    """Linear per-level sub-levels predict affine slices exactly."""
    u = np.arange(13)[:, None, None]
    v = np.arange(17)[None, :, None]
    w = np.arange(5)[None, None, :]
    A = (3.0 * u - 2.0 * v + 0.5 * w + 7.0) * np.ones((13, 17, 5))
    D = ip.decompose(A, (0, 1))
    s1 = np.zeros(A.shape, bool)
    s1[::4, ::4, :] = True
    # every S2/S3 point whose stencil stayed inside the slice is exact
    inner = np.zeros(A.shape, bool)
    inner[:12, :16, :] = True
    assert np.abs(D[~s1 & inner]).max() == 0


# ------------------------------------------------------------- bitplanes
def test_negabinary_golden_digits():
    """Base -2 digits (textbook): 2 = 110, 3 = 111, 6 = 11010, -1 = 11,
    -2 = 10 (tests/golden/negabinary.txt)."""
    for line in open(f"{GOLDEN}/negabinary.txt"):
        if not line.strip() or line.startswith("#"):
            continue
        val, digits = line.split()
        nb = bp._to_negabinary(np.array([int(val)], dtype=np.int64), 32)
        assert format(int(nb[0]), "b") == digits
        assert int(bp.from_negabinary(nb, 32)[0]) == int(val)


@pytest.mark.parametrize("B", [32, 64])
def test_negabinary_round_trip(B):
    rng = np.random.default_rng(5)
    lim = 1 << (B - 3)
    s = rng.integers(-lim + 1, lim, size=20000, dtype=np.int64)
    nb = bp._to_negabinary(s, B)
    assert (bp.from_negabinary(nb, B) == s).all()
    # every digit value sum(d_i (-2)^i) equals the decoded value
    d = [int(x) for x in format(int(nb[0]), "b")[::-1]]
    assert sum(di * (-2) ** i for i, di in enumerate(d)) == int(s[0])


def test_negabinary_dropped_digit_bound_is_tight():
    for k in range(1, 12):
        vals = [sum(d * (-2) ** i for i, d in enumerate(ds))
                for ds in itertools.product((0, 1), repeat=k)]
        assert max(abs(v) for v in vals) == bd.nb_dropped_max(k)


def test_pack_words_layout():
    """Plane word w bit j = element 32 w + j (LSB first)."""
    bits = np.zeros(64, bool)
    bits[[0, 5, 31, 33]] = True
    w = bp.pack_words(bits)
    assert list(w) == [(1 << 0) | (1 << 5) | (1 << 31), 1 << 1]


@pytest.mark.parametrize("enc", ["generic", "negabinary"])
@pytest.mark.parametrize("is_int", [False, True])
def test_all_planes_round_trip_and_table_bounds(enc, is_int):
    """Integers round-trip with all planes; every table entry bounds the
    actual error of that many planes; maxerr is monotone from b >= 1."""
    rng = np.random.default_rng(9)
    n = 4096 + 64
    if is_int:
        vals = rng.integers(-(1 << 41), 1 << 41, size=n).astype(np.int64)
        vals[::7] = 0
    else:
        vals = (rng.standard_normal(n) * np.exp(rng.uniform(-12, 0, n))).astype(np.float32)
        vals[::5] = 0
    B = 32
    h = 2.0 ** -30
    e = bp.encode(vals, is_int, B, enc, True)
    nbytes = bp.stream_bytes(e, B, n // 32)
    tab = bd.stream_tables(e, n, is_int, B, enc, h, True, nbytes)
    v64 = vals.astype(np.float64) * (h if is_int else 1.0)
    for b in range(B + 1):
        dec = bp.decode(e, n, is_int, B, enc, b, np.dtype(np.float32))
        d64 = dec.astype(np.float64) * (h if is_int else 1.0)
        err = np.abs(v64 - d64)
        assert err.max() <= tab["maxerr"][b] * (1 + 1e-15)
        assert (err ** 2).sum() <= tab["sq"][b] * (1 + 1e-12)
        if b >= 2:
            assert tab["maxerr"][b] < tab["maxerr"][b - 1]
    if is_int and enc == "generic":
        dec = bp.decode(e, n, is_int, B, enc, B, None)
        sh = e["quant"]["sh"]
        assert (dec == np.sign(vals) * ((np.abs(vals) >> sh) << sh)).all()
    if enc == "generic" and not is_int:
        # closed form of Sec. V-C: 2^(E-b) for b >= 1
        E = math.frexp(float(np.abs(vals).max()))[1]
        assert tab["maxerr"][3] == 2.0 ** (E - 3)


def test_sign_substreams_hold_first_significant_bit_signs():
    vals = np.array([0.0, -0.75, 0.4, -0.1, 0.3] + [0.0] * 27, dtype=np.float32)
    e = bp.encode(vals, False, 32, "generic", False)
    # E = 0 (max 0.75): q = floor(|v| 2^32); MSB planes: 0.75 -> 0, 0.4 -> 1,
    # 0.3 -> 1, 0.1 -> 3
    cnt = e["sign_counts"][0]
    assert cnt[0] == 1 and cnt[1] == 2 and cnt[3] == 1 and cnt.sum() == 4
    assert bp.unpack_words(e["signs"][0][0], 1)[0]            # -0.75
    assert list(bp.unpack_words(e["signs"][0][1], 2)) == [False, False]
    assert bp.unpack_words(e["signs"][0][3], 1)[0]            # -0.1


def test_pair_count_tables_equal_direct_sums():
    """Exact integer sqerr tables: pair counts give sum (r_b + 1)^2 exactly."""
    rng = np.random.default_rng(2)
    vals = rng.integers(-(1 << 20), 1 << 20, size=256).astype(np.int64)
    for enc in ("generic", "negabinary"):
        e = bp.encode(vals, True, 32, enc, True)
        q = e["quant"]["q"].astype(object)
        C = e["pairs"]
        for b in (0, 5, 17, 31, 32):
            k = 32 - b
            if enc == "generic":
                direct = sum(((int(x) & ((1 << k) - 1))) ** 2 for x in q)
                s2 = sum(C[j, jj] << (62 - j - jj) for j in range(b, 32) for jj in range(b, 32))
            else:
                def low(x):
                    return sum(((int(x) >> i) & 1) * (-2) ** i for i in range(k))
                direct = sum(low(x) ** 2 for x in q)
                s2 = sum((-1) ** (j + jj) * (C[j, jj] << (62 - j - jj))
                         for j in range(b, 32) for jj in range(b, 32))
            assert s2 == direct


# ---------------------------------------------------------- fixed point
def test_fixed_point_conversion_round_trip():
    X = grf((9, 10, 11), 4, np.float32)
    G, h = fixed_scale(float(np.abs(X).max()))
    assert (from_fixed(to_fixed(X, G), G, np.dtype(np.float32)) == X).all()


def test_int64_to_float32_single_rounding():
    """x' = float(x_int) h must round once: a value that double rounding via
    float64 would send the other way."""
    v = (1 << 60) + (1 << 36) + 1          # just above a float32 tie
    f = from_fixed(np.array([v], np.int64), 40, np.dtype(np.float32))[0]
    exact = Fraction(v)
    cands = [np.float32(2.0 ** 60), np.nextafter(np.float32(2.0 ** 60), np.float32(np.inf))]
    best = min(cands, key=lambda c: abs(Fraction(float(c)) - exact))
    assert f == best


# --------------------------------------------------- bounds: brute force
def _all_plane_vectors(B, n, limit=None, seed=0):
    if limit is None:
        yield from itertools.product(range(B + 1), repeat=n)
    else:
        rng = np.random.default_rng(seed)
        for _ in range(limit):
            yield tuple(int(x) for x in rng.integers(0, B + 1, size=n))


@pytest.mark.parametrize("shape,scheme,limit", [
    ((8, 8, 8), Scheme(interp="level", degree="linear", nlevels=3, nplanes=6), None),
    ((9, 9, 9), Scheme(interp="level", degree="cubic", nlevels=3, nplanes=6), None),
    ((1, 8, 8), Scheme(interp="level", degree="cubic", nlevels=3, nplanes=6), None),
    ((8, 8, 8), Scheme(mode="psnr", interp="region", degree="cubic", nlevels=3, nplanes=6), 400),
    ((9, 9, 9), Scheme(mode="psnr", interp="level", degree="cubic", decomp_axis=2, nlevels=3,
                       nplanes=6), 400),
    ((9, 9, 9), Scheme(interp="region", degree="linear", order=(1, 2, 0), decomp_axis=0,
                       nlevels=3, nplanes=6), 400),
])
@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_bruteforce_bounds_hold(shape, scheme, limit, dtype):
    """Every plane-count vector (or a seeded sample): the actual max error and
    the actual sum of squared errors stay within the composed bounds."""
    X = gaussians(shape, 13, dtype=np.float64).astype(dtype)
    if shape[0] == 1:
        X = X.reshape(shape[1:])
    h = oracle.refactor(X, scheme)
    comp = h["comp"]
    tabs = [s["tab"] for s in h["streams"]]
    ns = len(tabs)
    X64 = X.astype(np.float64)
    for bvec in _all_plane_vectors(6, ns, limit):
        xr, _ = oracle.retrieve(h, dict(b=list(bvec), bound=0, satisfied=True, bytes=0, kind="abs"))
        err = np.abs(xr.astype(np.float64) - X64)
        em = [t["maxerr"][b] for t, b in zip(tabs, bvec)]
        sq = [t["sq"][b] for t, b in zip(tabs, bvec)]
        assert err.max() <= comp.linf(em), bvec
        assert (err ** 2).sum() <= comp.l2(sq, em), bvec


# ------------------------------------------------------ invariant sweeps
SCHEMES = [
    Scheme(interp="level", degree="linear"),
    Scheme(interp="level", degree="cubic"),
    Scheme(interp="level", degree="cubic", decomp_axis=2),
    Scheme(mode="psnr", interp="region", degree="cubic", decomp_axis=2),
    Scheme(mode="psnr", interp="region", degree="linear", order=(2, 1, 0), decomp_axis=1),
    Scheme(interp="region", degree="cubic", order=(1, 0, 2), encoding="negabinary"),
]


@pytest.mark.parametrize("si", range(len(SCHEMES)))
def test_invariant_sweep(si):
    """Random shapes 2..40 per axis, both dtypes, targets 1e-1 .. 1e-9 and
    PSNR 30 .. 140: a satisfied plan never exceeds its target; an unsatisfied
    one is refused only when even all planes cannot meet it."""
    rng = np.random.default_rng(100 + si)
    sch = SCHEMES[si]
    for trial in range(4):
        nd = 3 if trial % 2 == 0 else 2
        shape = tuple(int(x) for x in rng.integers(2, 41, size=nd))
        dt = np.float32 if trial < 2 else np.float64
        X = grf(shape, 50 + trial, dt) * float(rng.uniform(0.01, 100))
        X = X.astype(dt)
        s2 = Scheme(**{**sch.__dict__})
        if nd == 2 or min(shape) < 3:
            s2.decomp_axis = -1
            if s2.order is not None:
                s2.order = None
        h = oracle.refactor(X, s2)
        R = h["meta"]["R"]
        X64 = X.astype(np.float64)
        for v in (1e-1, 1e-3, 1e-5, 1e-7, 1e-9):
            xr, pl = oracle.retrieve(h, Target("rel", v))
            err = np.abs(xr.astype(np.float64) - X64).max()
            if pl["satisfied"]:
                assert err <= v * R
            else:
                allb = dict(b=[len(t["tab"]["maxerr"]) - 1 for t in h["streams"]])
                em = [t["tab"]["maxerr"][-1] for t in h["streams"]]
                assert h["comp"].linf(em) > v * R
        for p in (30.0, 80.0, 140.0):
            xr, pl = oracle.retrieve(h, Target("psnr", p))
            mse = np.mean((xr.astype(np.float64) - X64) ** 2)
            if pl["satisfied"] and R > 0:
                assert mse == 0 or 20 * math.log10(R / math.sqrt(mse)) >= p


def test_greedy_is_feasible_and_monotone_in_target():
    X = grf((33, 33, 33), 21, np.float32)
    h = oracle.refactor(X, Scheme(interp="level", degree="cubic", decomp_axis=2))
    prev = 0
    for v in (1e-1, 1e-2, 1e-3, 1e-4, 1e-5):
        pl = oracle.plan(h, Target("rel", v))
        assert pl["satisfied"] and pl["bound"] <= v * h["meta"]["R"]
        assert pl["bytes"] >= prev
        prev = pl["bytes"]


def test_max_ordering_segments_descend_and_merge_equal_steps():
    """Sec. V-C: segments sorted by descending cumulative error; steps with
    equal error merge (so no two consecutive segments repeat a region error)."""
    X = grf((33, 33, 33), 22, np.float32)
    h = oracle.refactor(X, Scheme(interp="level", degree="cubic", decomp_axis=2))
    init, segs = h["M0"]
    errs = [init] + [s[2] for s in segs]
    assert all(a >= b for a, b in zip(errs, errs[1:]))
    assert errs[-1] < errs[0]
    # all planes of all 9 streams are assigned exactly once overall
    final = {}
    for upd, _, _ in segs:
        for i, nb in upd:
            assert nb > final.get(i, 0)
            final[i] = nb


def test_psnr_plan_meets_definition():
    """Sec. III-A: PSNR = 20 log10((max x - min x) / RMSE).  The planner's SSE
    bound for a PSNR target must imply that PSNR by the definition, and the
    retrieved field's PSNR, computed here from the definition in FP64, must
    reach it."""
    X = grf((24, 20, 28), 23, np.float32)
    X64 = X.astype(np.float64)
    h = oracle.refactor(X, Scheme(mode="psnr", interp="region", degree="cubic"))
    R = float(X64.max() - X64.min())
    for p in (40.0, 70.0, 100.0):
        xr, pl = oracle.retrieve(h, Target("psnr", p))
        assert pl["satisfied"]
        sse = float(np.sum((xr.astype(np.float64) - X64) ** 2))
        assert sse <= pl["bound"]
        assert 20 * math.log10(R / math.sqrt(pl["bound"] / X.size)) >= p
        assert 20 * math.log10(R / math.sqrt(sse / X.size)) >= p


def _golden_streams():
    streams, cur = [], None
    for line in open(f"{GOLDEN}/stream_bytes.txt"):
        f = line.split()
        if not f or f[0].startswith("#"):
            continue
        if f[0] == "stream":
            cur = dict(enc=f[1], B=int(f[2]), n=int(f[3]), vals={})
            streams.append(cur)
        elif f[0] == "value":
            cur["vals"][int(f[1])] = int(f[2])
        elif f[0] == "range":            # elements lo .. hi-1 all hold one value
            for i in range(int(f[1]), int(f[2])):
                cur["vals"][i] = int(f[3])
        elif f[0] == "expect":
            cur["expect"] = [int(x) for x in f[1:]]
    return streams


def test_stream_bytes_hand_counted():
    """bytes(b) equals hand-counted tables (tests/golden/stream_bytes.txt):
    zero planes are free, sign words of planes < b only, counted per sign
    segment; negabinary XOR can make a digit plane free."""
    for st in _golden_streams():
        vals = np.zeros(st["n"], dtype=np.int64)
        for i, v in st["vals"].items():
            vals[i] = v
        enc = bp.encode(vals, True, st["B"], st["enc"], False)
        assert bp.stream_bytes(enc, st["B"], st["n"] // WORD) == st["expect"]


def test_fp64_all_planes_near_lossless():
    """Every plane of an FP64 refactor gives the field back to within 1e-14
    of its range (the paper's near-lossless full retrieval; the fixed point
    of levels >= 1 keeps 48 fraction bits for FP64 fields, so the only
    losses are its floor and FP64 rounding at level 0), and an FP32 field to
    within a few units in the last place."""
    for shape, sch in [((24, 28, 32), Scheme(interp="level", degree="cubic", decomp_axis=2)),
                       ((26, 31, 29), Scheme(mode="psnr", interp="region", degree="cubic")),
                       ((1, 60, 70), Scheme(interp="level", degree="linear"))]:
        X = grf(shape, 77, np.float64)
        X = X[0] if shape[0] == 1 else X
        h = oracle.refactor(X, sch)
        assert h["meta"]["F"] == 48
        B = h["meta"]["B"]
        xr, _ = oracle.retrieve(h, dict(b=[B] * len(h["streams"])))
        R = h["meta"]["R"]
        assert np.abs(xr - X).max() <= 1e-14 * R
        X32 = X.astype(np.float32)
        h32 = oracle.refactor(X32, sch)
        xr32, _ = oracle.retrieve(h32, dict(b=[32] * len(h32["streams"])))
        assert np.abs(xr32.astype(np.float64) - X32).max() <= 8 * 2.0 ** -24 * np.abs(X32).max()
