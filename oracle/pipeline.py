"""End-to-end refactor (Alg. 1) and retrieve (Alg. 2) -- oracle.

Test infrastructure only.

Arithmetic (a reading; the paper runs FP64 data in FP64): level 0 and its
coefficient decomposition run in the field's dtype; levels >= 1 (at most 1/8
of the points, but their errors are amplified by up to Lam^(d l) on the way to
level 0) run in exact 64-bit fixed point with quantum h = 2^(G - F), where
max|x| < 2^G and F = fix_bits(dtype, L): 40 for FP32 fields (far below FP32
resolution), for FP64 fields 48, or 56 - L for deep hierarchies so that
every reconstruction numerator keeps int64 headroom (values up to
4.2 (Lam^d)^L 2^F, numerators up to 20 times that).  The fixed-point value of
x is floor(x / h).
"""
import math
from dataclasses import dataclass
from typing import Optional, Tuple

import numpy as np

from . import bitplane as bp
from . import bounds as bd
from .geometry import (active_axes, auto_levels, max_levels, build_geometry, count_from,
                       decomp_axes, region_lattice, coarse_lattice)
from .interp import (decompose, level_points_mask, predict_level, recompose,
                     reconstruct_level)

FIX_BITS_F32 = 40


def fix_bits(dtag, L):
    """Fraction bits F of the fixed point of levels >= 1."""
    return FIX_BITS_F32 if dtag == "f32" else min(48, 56 - L)


@dataclass
class Scheme:
    mode: str = "eb"             # "eb" | "psnr" | "explicit" (both tables, generic default)
    interp: str = "level"        # "level" | "region"
    degree: str = "cubic"        # "linear" | "cubic"
    order: Optional[Tuple[int, ...]] = None   # per-region pass order
    decomp_axis: int = -1        # slice normal of the coefficient decomposition
    encoding: Optional[str] = None  # "generic" | "negabinary" (default by mode)
    nlevels: int = 0
    nplanes: int = 0


@dataclass
class Target:
    kind: str                    # "abs" | "rel" | "psnr"
    value: float


def shape3_of(shape):
    return (1,) + tuple(shape) if len(shape) == 2 else tuple(shape)


def fixed_scale(M, F=FIX_BITS_F32):
    G = math.frexp(M)[1] if M > 0 else 0
    return G, math.ldexp(1.0, G - F)


def to_fixed(X, G, F=FIX_BITS_F32):
    """floor(x 2^(F - G)), exactly (FP64 product of an exact power of two;
    for FP64 inputs with F - G large enough to leave the FP64 range of exact
    integers the product is still exact: scaling by 2^k never rounds)."""
    return np.floor(np.ldexp(X.astype(np.float64), F - G)).astype(np.int64)


def from_fixed(xi, G, dtype, F=FIX_BITS_F32):
    return (xi.astype(dtype) * dtype.type(math.ldexp(1.0, G - F))).astype(dtype)


def _grid(shape3, s):
    return tuple(slice(0, None, s) if shape3[a] > 1 else slice(None) for a in range(3))


def _stream_values(stream, src):
    parts = []
    for lat in stream.lattices:
        if lat.empty():
            continue
        a = src[lat.slices()]
        pad = lat.row_pad - a.shape[2]
        if pad:
            a = np.concatenate([a, np.zeros(a.shape[:2] + (pad,), a.dtype)], axis=2)
        parts.append(a.reshape(-1))
    if not parts:
        return np.zeros(0, dtype=src.dtype)
    return np.concatenate(parts)


def _scatter(stream, vals, dst):
    off = 0
    for lat in stream.lattices:
        if lat.empty():
            continue
        c0, c1, c2 = lat.count
        a = vals[off:off + lat.n_pad].reshape(c0, c1, lat.row_pad)[:, :, :c2]
        dst[lat.slices()] = a
        off += lat.n_pad


def refactor(X, scheme=Scheme(), trace=None):
    """Alg. 1.  ``trace`` (a dict, optional) receives the level-0 coefficient
    array ``c`` and the decomposed values ``d`` (for tests)."""
    X = np.asarray(X)
    assert X.ndim in (2, 3) and min(X.shape) >= 2
    dt = X.dtype
    dtag = {np.dtype(np.float32): "f32", np.dtype(np.float64): "f64"}[dt]
    shape3 = shape3_of(X.shape)
    X3 = X.reshape(shape3)
    act = active_axes(shape3)
    B = scheme.nplanes or (32 if dtag == "f32" else 64)
    L = scheme.nlevels or auto_levels(shape3)
    assert 1 <= L <= max_levels(shape3)
    order = tuple(scheme.order) if (scheme.order and scheme.interp == "region") else act
    encoding = scheme.encoding or ("negabinary" if scheme.mode == "psnr" else "generic")
    exact_sq = scheme.mode != "eb"       # exact integer squared-error tables
    dax = scheme.decomp_axis if (len(act) == 3 and L >= 2) else -1
    geo = build_geometry(shape3, L, scheme.interp, order, dax)

    # a1: field statistics (Sec. III-A: PSNR uses max - min)
    xmin, xmax = float(X3.min()), float(X3.max())
    M = max(abs(xmin), abs(xmax))
    F = fix_bits(dtag, L)
    G, h = fixed_scale(M, F)

    Ci = np.zeros(shape3, dtype=np.int64)
    Cf = np.zeros(shape3, dtype=dt)
    Df = np.zeros(shape3, dtype=dt)
    if L == 1:
        Cf[...] = X3
    else:
        Xi = to_fixed(X3, G, F)
        cl = coarse_lattice(shape3, L).slices()
        Ci[cl] = Xi[cl]
        for level in range(1, L - 1):                      # Alg. 1, l = 1..L-2
            sl = _grid(shape3, 1 << level)
            Gs = Xi[sl].copy()
            W = predict_level(Gs, order, scheme.interp, scheme.degree)
            mask = level_points_mask(Gs.shape, order)
            view = Ci[sl]
            view[mask] = (Gs - W)[mask]
        W = predict_level(X3, order, scheme.interp, scheme.degree)   # level 0
        mask = level_points_mask(shape3, order)
        Cf[mask] = (X3 - W)[mask]
        if dax >= 0:                                        # Alg. 1 CoeffDecom
            uv = decomp_axes(dax)
            for r in range(1, len(order) + 1):
                sl = region_lattice(shape3, 0, order, r).slices()
                Df[sl] = decompose(Cf[sl].copy(), uv)

    if trace is not None:
        trace["c"], trace["d"] = Cf.copy(), Df.copy()
    streams = []
    for s in geo.streams:
        src = Ci if s.is_int else (Df if s.sub > 0 else Cf)
        vals = _stream_values(s, src)
        enc = bp.encode(vals, s.is_int, B, encoding, exact_sq)
        nbytes = bp.stream_bytes(enc, B, s.words)
        tab = bd.stream_tables(enc, s.n_real, s.is_int, B, encoding, h, exact_sq, nbytes)
        streams.append(dict(level=s.level, region=s.region, sub=s.sub,
                            n_real=s.n_real, n_pad=s.n_pad, is_int=s.is_int,
                            enc=enc, tab=tab, geo=s))

    # C0c: max |c| over the level-0 coefficients; Dm: max |value| of the
    # decomposition's predicted sub-levels (S2, S3); C0: max over both
    C0c = M if L == 1 else float(np.abs(Cf[level_points_mask(shape3, order)]).max())
    Dm = 0.0
    for s in streams:
        if s["level"] == 0 and not s["is_int"] and s["sub"] >= 2:
            Dm = max(Dm, s["enc"]["quant"]["vmax"])
    C0 = C0c
    for s in streams:
        if s["level"] == 0 and not s["is_int"]:
            C0 = max(C0, s["enc"]["quant"]["vmax"])
    meta = dict(L=L, d=len(order), degree=scheme.degree, interp=scheme.interp,
                dtype=dtag, h=h, G=G, F=F, M=M, C0=C0, C0c=C0c, Dm=Dm, R=xmax - xmin, xmin=xmin,
                xmax=xmax, n=X3.size, B=B, encoding=encoding, order=order,
                decomp_axis=dax, shape3=shape3, shape=X.shape, mode=scheme.mode)
    _add_factors(meta, geo)
    comp = bd.Composer(meta, streams)
    M0 = None
    if scheme.interp == "level" and dax >= 0:
        by_r = {}
        for i in comp.by_level[0]:
            by_r.setdefault(streams[i]["region"], []).append(i)
        M0 = bd.max_ordering(by_r, [s["tab"] for s in streams])
    return dict(meta=meta, geo=geo, streams=streams, comp=comp, M0=M0, dtype=dt)


def _add_factors(meta, geo):
    shape3, L, order = meta["shape3"], meta["L"], meta["order"]
    lvl_cnt = {l: 0 for l in range(L)}
    reg_cnt = {}
    for s in geo.streams:
        lvl_cnt[s.level] += s.n_real
        reg_cnt[(s.level, s.region)] = reg_cnt.get((s.level, s.region), 0) + s.n_real
    meta["level_counts"] = lvl_cnt
    meta["region_counts"] = reg_cnt
    lf, rf = {}, {}
    for level in range(L - 1):
        s = 1 << level
        prod = 1.0
        for a in order:
            prod *= 1.0 + bd.rowsum_ptp(count_from(shape3[a], 0, s), meta["degree"])
        lf[level] = math.sqrt(prod - 1.0)
        for r, a in enumerate(order, start=1):
            rf[(level, r)] = math.sqrt(bd.rowsum_ptp(count_from(shape3[a], 0, s), meta["degree"]))
    meta["level_factor"], meta["region_factor"] = lf, rf
    df = {}
    if meta["decomp_axis"] >= 0:
        uv = decomp_axes(meta["decomp_axis"])
        for r in range(1, len(order) + 1):
            lat = region_lattice(shape3, 0, order, r)
            p2, p3 = 1.0, 1.0
            for ax in uv:
                c = lat.count[ax]
                p3 *= 1.0 + bd.rowsum_ptp(c, "linear")
                p2 *= 1.0 + bd.rowsum_ptp(count_from(c, 0, 2), "linear")
            df[r] = (math.sqrt(p2 - 1.0), math.sqrt(p3 - 1.0))
    meta["decomp_factors"] = df


def plan(handle, target, have=None, search=None):
    """Retrieval interpreter: planes per stream for a target.  ``have``: a
    plan whose planes are already fetched (incremental invocation, see
    bounds.greedy); the result contains it.  ``search``: None for the
    greedy, else the expansion budget of the best-first search
    (bounds.best_first; its statistics under "search")."""
    meta = handle["meta"]
    tabs = [s["tab"] for s in handle["streams"]]
    comp = handle["comp"]
    hb = have["b"] if isinstance(have, dict) else have
    if target.kind in ("abs", "rel"):
        goal, kind = target.value * (meta["R"] if target.kind == "rel" else 1.0), "linf"
    else:
        ratio = meta["R"] / (10.0 ** (target.value / 20.0))
        goal, kind = meta["n"] * ratio * ratio, "l2"
    info = None
    if search is None:
        b, bound, ok = bd.greedy(comp, tabs, goal, kind, hb)
    else:
        b, bound, ok, info = bd.best_first(comp, tabs, goal, kind, hb, search)
    total = sum(t["bytes"][bi] for t, bi in zip(tabs, b))
    out = dict(b=b, bound=bound, satisfied=ok, bytes=total, kind=target.kind)
    if info is not None:
        out["search"] = info
    return out


def retrieve(handle, target_or_plan, trace=None):
    """Alg. 2: decode the planned planes, recompose level 0, reconstruct
    coarse -> fine.  Returns (x', plan).  ``trace`` (a dict, optional)
    receives the decoded level-0 coefficients ``c_hat`` (recomposed) and
    decoded sub-level values ``d_hat`` (for tests)."""
    pl = target_or_plan if isinstance(target_or_plan, dict) else plan(handle, target_or_plan)
    meta = handle["meta"]
    dt = handle["dtype"]
    shape3, L, order = meta["shape3"], meta["L"], meta["order"]
    B, enc_kind = meta["B"], meta["encoding"]
    Ci = np.zeros(shape3, dtype=np.int64)
    Cf = np.zeros(shape3, dtype=dt)
    Df = np.zeros(shape3, dtype=dt)
    for s, b in zip(handle["streams"], pl["b"]):
        vals = bp.decode(s["enc"], s["n_pad"], s["is_int"], B, enc_kind, b, dt)
        dst = Ci if s["is_int"] else (Df if s["sub"] > 0 else Cf)
        _scatter(s["geo"], vals, dst)
    if L == 1:
        return Cf.reshape(meta["shape"]), pl
    if meta["decomp_axis"] >= 0:
        uv = decomp_axes(meta["decomp_axis"])
        for r in range(1, len(order) + 1):
            sl = region_lattice(shape3, 0, order, r).slices()
            Cf[sl] = recompose(Df[sl].copy(), uv)
    if trace is not None:
        trace["c_hat"], trace["d_hat"] = Cf.copy(), Df.copy()
    Xi = np.zeros(shape3, dtype=np.int64)
    cl = coarse_lattice(shape3, L).slices()
    Xi[cl] = Ci[cl]
    for level in range(L - 2, 0, -1):
        sl = _grid(shape3, 1 << level)
        Gs = Xi[sl]
        mask = level_points_mask(Gs.shape, order)
        Gs[mask] = Ci[sl][mask]
        reconstruct_level(Gs, order, meta["interp"], meta["degree"])
    Xr = np.zeros(shape3, dtype=dt)
    g2 = _grid(shape3, 2)
    Xr[g2] = from_fixed(Xi[g2], meta["G"], dt, meta["F"])
    mask = level_points_mask(shape3, order)
    Xr[mask] = Cf[mask]
    reconstruct_level(Xr, order, meta["interp"], meta["degree"])
    return Xr.reshape(meta["shape"]), pl
