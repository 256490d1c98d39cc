"""Interpolation, coefficient decomposition and their inverses (oracle).

Test infrastructure only.

Sec. IV: both schemes visit a level's regions one axis at a time ("fastest
direction interpolation", Sec. VI-C): region r is predicted by a 1-D rule
along pass axis pi(r) from the points that are even along that axis.
* per-level (PMGARD-style): those source points hold *predictions* for points
  of earlier regions, which makes the result the tensor-product interpolant of
  the coarser grid (edge / face / cube centres = means of 2 / 4 / 8 corners in
  the linear case, Sec. IV);
* per-region (SZ3 / IPComp-style): the sources are the *original* values
  (Sec. IV: "using the original data values rather than the quantized ones").
Reconstruction (Alg. 2) runs the same passes on reconstructed values; in the
per-region scheme each region reads the reconstructed earlier regions.

1-D rules at an odd index j of a line of m points (index unit = the level
stride); the paper says "cubic" (Alg. 1/2) without boundary handling; the
readings here are 4-point Lagrange in the interior, the 3-point Lagrange rule
at either edge, the 2-point mean when only j-1, j+1 exist, and j-1 when j+1 is
outside the line:
  cubic     (9 (a[j-1] + a[j+1]) - (a[j-3] + a[j+3])) / 16
  left      (3 a[j-1] + 6 a[j+1] - a[j+3]) / 8
  right     (6 a[j-1] + 3 a[j+1] - a[j-3]) / 8
  linear    (a[j-1] + a[j+1]) / 2
  constant  a[j-1]
Floating point evaluates exactly the expression trees in ``_F`` (left to right,
no fused multiply-add); fixed point evaluates the integer numerator and floors
the division by a power of two (arithmetic right shift).  The floating-point
trees are written to round little: with inputs bounded by V and unit
roundoff u, the cubic rule as mean + correction,
  s1 = a[j-1] + a[j+1],  s2 = a[j-3] + a[j+3],  s1 / 2 + (s1 - s2) / 16,
rounds s1 (weight 9/16, |s1| <= 2V), s2 (1/16, 2V), s1 - s2 (1/16, 4V) and the
sum (|result| <= 1.25 V): at most 2.75 u V; the edge rule as
  0.75 a[j+1] + (0.375 a[j-1] - 0.125 a[j+3])
rounds 0.75 a (0.75 V), 0.375 a (0.375 V), the difference (0.5 V) and the sum
(1.25 V): 2.875 u V; the linear rule rounds a + b once: u V.
"""
import numpy as np

LINEAR, CUBIC = "linear", "cubic"


class _F:
    """Floating-point rules in the field dtype."""

    def __init__(self, dt):
        self.dt = dt
        self.c = {k: dt.type(v) for k, v in
                  dict(h=0.5, e=0.125, s=0.0625, q3=0.375, q6=0.75).items()}

    def lin(self, a, b):
        return (a + b) * self.c["h"]

    def cubic(self, m3, m1, p1, p3):
        s1 = m1 + p1
        s2 = m3 + p3
        return s1 * self.c["h"] + (s1 - s2) * self.c["s"]

    def left(self, m1, p1, p3):
        return p1 * self.c["q6"] + (m1 * self.c["q3"] - p3 * self.c["e"])

    def right(self, m3, m1, p1):
        return m1 * self.c["q6"] + (p1 * self.c["q3"] - m3 * self.c["e"])


class _I:
    """Fixed-point rules on int64 (exact numerators, floored shifts)."""

    def lin(self, a, b):
        return (a + b) >> 1

    def cubic(self, m3, m1, p1, p3):
        return (9 * (m1 + p1) - (m3 + p3)) >> 4

    def left(self, m1, p1, p3):
        return (3 * m1 + 6 * p1 - p3) >> 3

    def right(self, m3, m1, p1):
        return (6 * m1 + 3 * p1 - m3) >> 3


def _ops(arr):
    if arr.dtype == np.int64:
        return _I()
    return _F(arr.dtype)


def predict_line(A, ax, degree):
    """Predictions for every odd index along ``ax`` of ``A`` from its even
    indices.  Returns an array whose ``ax`` extent is m // 2."""
    m = A.shape[ax]
    ops = _ops(A)
    out_shape = list(A.shape)
    out_shape[ax] = m // 2
    out = np.empty(out_shape, dtype=A.dtype)

    def at(j):
        return np.take(A, j, axis=ax)

    for t, j in enumerate(range(1, m, 2)):
        p1, m3, p3 = j + 1 < m, j - 3 >= 0, j + 3 < m
        if degree == CUBIC and p1 and m3 and p3:
            val = ops.cubic(at(j - 3), at(j - 1), at(j + 1), at(j + 3))
        elif degree == CUBIC and p1 and p3:
            val = ops.left(at(j - 1), at(j + 1), at(j + 3))
        elif degree == CUBIC and p1 and m3:
            val = ops.right(at(j - 3), at(j - 1), at(j + 1))
        elif p1:
            val = ops.lin(at(j - 1), at(j + 1))
        else:
            val = at(j - 1)
        idx = [slice(None)] * A.ndim
        idx[ax] = t
        out[tuple(idx)] = val
    return out


def _src_index(ndim, order, r):
    """Region r (0-based) of a pass: full along order[r], even along later
    pass axes, everything along earlier ones."""
    sl = [slice(None)] * ndim
    for b in order[r + 1:]:
        sl[b] = slice(0, None, 2)
    return sl


def _dst_index(ndim, order, r):
    sl = _src_index(ndim, order, r)
    sl[order[r]] = slice(1, None, 2)
    return tuple(sl)


def predict_level(G, order, interp, degree):
    """Refactor-side predictions on one level's s-grid array ``G`` (coarse
    points at even indices along every axis of ``order``).  Returns W with the
    prediction at every level point and G at the coarse points."""
    W = G.copy()
    for r, a in enumerate(order):
        src = tuple(_src_index(G.ndim, order, r))
        base = W[src] if interp == "level" else G[src]
        W[_dst_index(G.ndim, order, r)] = predict_line(base, a, degree)
    return W


def reconstruct_level(G, order, interp, degree):
    """In place: coarse points of ``G`` hold reconstructed values, level
    points hold decoded coefficients; on return level points hold
    x' = P(reconstructed) + c_hat (Alg. 2)."""
    if interp == "level":
        W = G.copy()
        for r, a in enumerate(order):
            src = tuple(_src_index(G.ndim, order, r))
            W[_dst_index(G.ndim, order, r)] = predict_line(W[src], a, degree)
        for r in range(len(order)):
            dst = _dst_index(G.ndim, order, r)
            G[dst] = W[dst] + G[dst]
    else:
        for r, a in enumerate(order):
            src = tuple(_src_index(G.ndim, order, r))
            dst = _dst_index(G.ndim, order, r)
            G[dst] = predict_line(G[src], a, degree) + G[dst]
    return G


def level_points_mask(shape, order):
    """Boolean mask of level points (odd along some axis of ``order``)."""
    mask = np.zeros(shape, dtype=bool)
    for r in range(len(order)):
        mask[_dst_index(len(shape), order, r)] = True
    return mask


# --------------------------------------------------------------------------
# Coefficient decomposition (Sec. V-B, Alg. 1 lines for LinearInterpolate /
# ExtractLevel; inverse in Alg. 2).  Each region's compact coefficient array is
# a stack of 2-D slices normal to the decomposition axis.  A 3-level 2-D
# per-level *linear* hierarchy is applied to every slice: S1 = 4-grid (raw),
# S2 predicted from S1 on the 2-grid, S3 predicted from the 2-grid.  Both
# predictions use the original coefficients (Alg. 1 computes Pi_1 and Pi_2 on
# the undecomposed slice S).
# --------------------------------------------------------------------------

def decompose(A, uv):
    """Return D (same shape as A): S1 entries = A, S2 / S3 entries = A - W."""
    D = A.copy()
    # stride-1 sub-level (S3): predict from the 2-grid of originals
    W1 = predict_level(A, uv, "level", LINEAR)
    m1 = level_points_mask(A.shape, uv)
    D[m1] = A[m1] - W1[m1]
    # stride-2 sub-level (S2): predict from the 4-grid, on the 2-grid view
    sl = [slice(None)] * 3
    for ax in uv:
        sl[ax] = slice(0, None, 2)
    sl = tuple(sl)
    V2 = A[sl]
    W2 = predict_level(V2, uv, "level", LINEAR)
    m2 = level_points_mask(V2.shape, uv)
    D2 = D[sl]                      # view into D
    D2[m2] = V2[m2] - W2[m2]
    return D


def recompose(Dhat, uv):
    """Inverse of ``decompose`` on decoded values (Alg. 2): S1 raw, then S2 on
    the 2-grid view, then S3 on the full grid."""
    R = Dhat.copy()
    sl = [slice(None)] * 3
    for ax in uv:
        sl[ax] = slice(0, None, 2)
    V2 = R[tuple(sl)]               # view
    reconstruct_level(V2, uv, "level", LINEAR)
    reconstruct_level(R, uv, "level", LINEAR)
    return R
