"""Pins of the oracle's level-0 rounding allowance rho_0 against exact
arithmetic.

The bound composition (Sec. III-A error bound, Sec. V-C error maps) splits the
error of a reconstructed level-0 point into the exact propagation of the
coarser grid's error through the interpolant, the exact propagation of the
coefficient truncation (through the inverse decomposition, Sec. V-B), and the
rounding of the floating-point evaluation, which rho_0 must bound.  Here that
rounding part is computed exactly with rationals from the oracle's own
intermediate values:

  per-level   R = (x - x') - P(x_c - x'_c) - dc
  per-region  R_r = (x - x') - P_r((x - x') at the sources) - dc

with P the interpolant in exact arithmetic (the 4-point / 3-point Lagrange,
2-point mean and constant rules of Sec. IV, here with rational weights),
x'_c the reconstructed coarse values the retrieval actually used, and dc the
exact propagation of the coefficient error c - c_hat (decomposed regions:
the exact inverse decomposition of d - d_hat).  The pin: max |R| <= rho_0,
and rho_0 is no more than a stated factor above max |R| on random smooth
fields (the allowance is a worst case; random roundings partly cancel).

The per-rule constants kappa behind rho_0 are pinned separately: each 1-D
rule's floating-point evaluation differs from its exact value by at most
kappa u V on inputs bounded by V, and random inputs come within a factor 3.
"""
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import Scheme, Target, interp as ip
from oracle.geometry import region_lattice, decomp_axes
from synth import grf

# rho_0 may exceed the exact rounding error by at most these factors here:
# with every plane the retrieval's coarse values are almost the refactor's,
# so the two predictions round almost alike and their errors largely cancel;
# with truncated plans they round independently
LOOSE_ALL_PLANES = 256.0
LOOSE_TRUNCATED = 32.0

W_CUBIC = (Fraction(-1, 16), Fraction(9, 16), Fraction(9, 16), Fraction(-1, 16))
W_LEFT = (Fraction(3, 8), Fraction(6, 8), Fraction(-1, 8))      # j-1, j+1, j+3
W_RIGHT = (Fraction(-1, 8), Fraction(6, 8), Fraction(3, 8))     # j-3, j-1, j+1


def _q(a):
    """Exact rationals of a float array."""
    out = np.empty(a.shape, dtype=object)
    flat, src = out.reshape(-1), np.asarray(a, dtype=np.float64).reshape(-1)
    for i, v in enumerate(src):
        flat[i] = Fraction(float(v))
    return out


def _line_exact(A, ax, degree):
    """Exact predictions at the odd indices along ``ax`` from the even ones."""
    m = A.shape[ax]
    shp = list(A.shape)
    shp[ax] = m // 2
    out = np.empty(shp, dtype=object)

    def at(j):
        return np.take(A, j, axis=ax)

    for t, j in enumerate(range(1, m, 2)):
        p1, m3, p3 = j + 1 < m, j - 3 >= 0, j + 3 < m
        if degree == "cubic" and p1 and m3 and p3:
            v = sum((w * at(k) for w, k in zip(W_CUBIC, (j - 3, j - 1, j + 1, j + 3))), start=0 * at(j - 1))
        elif degree == "cubic" and p1 and p3:
            v = sum((w * at(k) for w, k in zip(W_LEFT, (j - 1, j + 1, j + 3))), start=0 * at(j - 1))
        elif degree == "cubic" and p1 and m3:
            v = sum((w * at(k) for w, k in zip(W_RIGHT, (j - 3, j - 1, j + 1))), start=0 * at(j - 1))
        elif p1:
            v = Fraction(1, 2) * (at(j - 1) + at(j + 1))
        else:
            v = at(j - 1)
        idx = [slice(None)] * A.ndim
        idx[ax] = t
        out[tuple(idx)] = v
    return out


def _src(ndim, order, r):
    sl = [slice(None)] * ndim
    for b in order[r + 1:]:
        sl[b] = slice(0, None, 2)
    return sl


def _dst(ndim, order, r):
    sl = _src(ndim, order, r)
    sl[order[r]] = slice(1, None, 2)
    return tuple(sl)


def _tensor_exact(G, order, degree):
    """Exact per-level interpolant of the even-grid values of G at every level
    point (sequential passes reading predictions)."""
    W = G.copy()
    for r, a in enumerate(order):
        W[_dst(G.ndim, order, r)] = _line_exact(W[tuple(_src(G.ndim, order, r))], a, degree)
    return W


def _recompose_exact(D, uv):
    """Exact inverse decomposition of a region's compact array (linear maps)."""
    R = D.copy()
    sl = [slice(None)] * 3
    for ax in uv:
        sl[ax] = slice(0, None, 2)
    for view in (R[tuple(sl)], R):
        W = _tensor_exact(view, uv, "linear")
        for r in range(len(uv)):
            d = _dst(3, uv, r)
            view[d] = W[d] + view[d]
    return R


def _rounding_part(h, tr_r, pl, X):
    """max |R| over the level-0 points (see module docstring) and rho_0."""
    tr_q = {}
    xr, _ = oracle.retrieve(h, pl, trace=tr_q)
    hh = h
    meta = hh["meta"]
    shape3, order = meta["shape3"], meta["order"]
    x = _q(X.reshape(shape3))
    xp = _q(xr.reshape(shape3))
    err = x - xp
    # exact propagation of the coefficient error
    dc = _q(tr_r["c"]) - _q(tr_q["c_hat"])
    if meta["decomp_axis"] >= 0:
        uv = decomp_axes(meta["decomp_axis"])
        dd = _q(tr_r["d"]) - _q(tr_q["d_hat"])
        for r in range(1, len(order) + 1):
            sl = region_lattice(shape3, 0, order, r).slices()
            dc[sl] = _recompose_exact(dd[sl].copy(), uv)
    R = np.zeros(shape3, dtype=object)
    if meta["interp"] == "level":
        E = err.copy()
        lvl = ip.level_points_mask(shape3, order)
        E[lvl] = 0                      # coarse errors only
        P = _tensor_exact(E, order, meta["degree"])
        R[lvl] = (err - P - dc)[lvl]
    else:
        for r, a in enumerate(order):
            d = _dst(3, order, r)
            P = _line_exact(err[tuple(_src(3, order, r))], a, meta["degree"])
            R[d] = err[d] - P - dc[d]
    worst = max(abs(v) for v in R.reshape(-1))
    comp = hh["comp"]
    errs = [s["tab"]["maxerr"][b] for s, b in zip(hh["streams"], pl["b"])]
    E1, e0 = comp._e1_and_e0(errs)
    return float(worst), comp.rho0(E1, e0)


CASES = [
    ((17, 18, 20), Scheme(interp="level", degree="cubic", nlevels=3), np.float32),
    ((17, 18, 20), Scheme(interp="level", degree="cubic", decomp_axis=2, nlevels=3), np.float32),
    ((16, 19, 21), Scheme(interp="level", degree="linear", decomp_axis=0, nlevels=3), np.float32),
    ((18, 17, 19), Scheme(mode="psnr", interp="region", degree="cubic", decomp_axis=2, nlevels=3),
     np.float32),
    ((17, 18, 20), Scheme(interp="region", degree="cubic", order=(2, 0, 1), nlevels=3), np.float32),
    ((17, 18, 20), Scheme(interp="level", degree="cubic", decomp_axis=1, nlevels=3), np.float64),
    ((1, 40, 44), Scheme(interp="level", degree="cubic", nlevels=3), np.float32),
]


@pytest.mark.parametrize("shape,scheme,dtype", CASES)
def test_rho0_bounds_exact_rounding(shape, scheme, dtype):
    X = grf(shape, 41, dtype)
    X = X[0] if shape[0] == 1 else X
    tr_r = {}
    h = oracle.refactor(X, scheme, trace=tr_r)
    R = h["meta"]["R"]
    B = h["meta"]["B"]
    plans = [dict(b=[B] * len(h["streams"]))]          # all planes
    for v in (1e-3, 1e-5):
        plans.append(oracle.plan(h, Target("rel", v)))
    for pl in plans:
        worst, rho = _rounding_part(h, tr_r, pl, X)
        assert worst <= rho
        assert worst > 0
        loose = LOOSE_ALL_PLANES if "satisfied" not in pl else LOOSE_TRUNCATED
        assert rho <= loose * worst, (rho, worst)
    assert R > 0


def _ulp_max(dt):
    return 2.0 ** (-24 if dt == np.float32 else -53)


@pytest.mark.parametrize("dt", [np.float32, np.float64])
def test_rule_rounding_constants(dt):
    """Each 1-D rule's evaluation error <= kappa u V (V = max |input|), and
    random inputs reach more than a third of it: cubic 2.75, edges 2.875,
    linear 1."""
    rng = np.random.default_rng(3)
    n = 1 << 14
    u = _ulp_max(dt)
    f = ip._F(np.dtype(dt))
    V = 1.0
    # full-mantissa inputs in [-V, V] (uniform draws sit on a fixed-point grid)
    a, b, c, d = (np.sin(rng.uniform(0.0, 1e4, n)).astype(dt) * dt(V) for _ in range(4))
    a[: n // 4] = np.abs(a[: n // 4])     # some lines of one sign: large sums
    b[: n // 4] = np.abs(b[: n // 4])
    c[: n // 4] = -np.abs(c[: n // 4])
    d[: n // 4] = -np.abs(d[: n // 4])
    A, Bq, Cq, D = (_q(v) for v in (a, b, c, d))
    cases = {
        "cubic": (f.cubic(a, b, c, d), W_CUBIC[0] * A + W_CUBIC[1] * Bq + W_CUBIC[2] * Cq + W_CUBIC[3] * D, 2.75),
        "left": (f.left(a, b, c), W_LEFT[0] * A + W_LEFT[1] * Bq + W_LEFT[2] * Cq, 2.875),
        "right": (f.right(a, b, c), W_RIGHT[0] * A + W_RIGHT[1] * Bq + W_RIGHT[2] * Cq, 2.875),
        "linear": (f.lin(a, b), Fraction(1, 2) * (A + Bq), 1.0),
    }
    for name, (got, exact, kappa) in cases.items():
        e = max(abs(Fraction(float(g)) - x) for g, x in zip(got, exact))
        assert e <= Fraction(kappa) * Fraction(u) * Fraction(V), name
        assert e >= Fraction(kappa) * Fraction(u) * Fraction(V) / 3, (name, float(e / Fraction(u)))
