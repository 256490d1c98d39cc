"""Error tables, bound composition, max ordering and the retrieval planner
(oracle).  Test infrastructure only.

Sec. III-A: error-bound mode minimises the retrieved size S_tau subject to
max|x - x'| <= tau; PSNR = 20 log10((max x - min x) / RMSE).  Sec. V-C: a
level's maximum coefficient gives a bitplane -> absolute error map; with
coefficient decomposition, the level's error is the maximum over regions, and
"max ordering" merges the per-region loading orders by descending cumulative
error, merging steps with equal error, into segments with an error list M_0.
Sec. VI-B: the interpreter picks how many bitplanes to retrieve.

Readings (the paper gives estimates; these bounds are guarantees):
* L-infinity: per-level E_l = Lam^d E_{l+1} + e_l + rho_l; per-region
  F_r = Lam max(E_{l+1}, F_1..F_{r-1}) + e_{l,r} + rho_l, E_l = max(E_{l+1}, F_r);
  Lam = 1.25 (cubic: sum of |weights| of every boundary rule) or 1 (linear).
  A decomposed region's coefficient error is e_1 + e_2 + e_3 (the bilinear
  per-level predictions have unit weight sum).
* L2 (PSNR): ||P e||_2 <= sqrt(||P^T P||_inf) ||e||_2 per 1-D pass, with the
  row sum computed exactly for every line length; tensor passes multiply.
* Rounding at level 0 (field dtype, unit roundoff u): the coarse values
  enter as the fixed-point reconstruction rounded once to the field dtype
  (error <= u Y, added to the incoming error); every level-0 point then
  carries rho_0 = G u (Pr + Y + Cr) + s, with
  Y = M + Lam^d (E_1 + sum e_0) bounding |x'| and the retrieval's inputs;
  Pr the rounding of the prediction in refactoring and in retrieval: one
  pass (per-region) rounds at most kappa (M + Y); per-level pass k rounds at
  most kappa V_k, which the later d - k passes multiply by Lam^(d-k), where
  pass 1 reads coarse values (V_1 = M, retrieval Y) and pass k >= 2 also
  earlier passes' predictions, each bounded by Lam^(k-1) times that and also
  by M + C0c (1 + 2u) (a prediction W at a level-0 point satisfies
  |W| <= |x| + |c| / (1 - u)), retrieval Y + C0c (1 + 2u);
  Y the final addition; Cr the coefficient side, with C0c = max |c| over
  level 0 and Dm = max |value| of the decomposition's sub-levels S2, S3:
  c = x - P rounded once (C0c), negabinary dequantisation (C0c); with
  decomposition, per sub-level S2 its forward difference (Dm), the two
  linear predictions (2 C0c) and the addition (C0c), and S3 its forward
  difference (Dm), the two 2-pass bilinear predictions (4 C0c), the
  addition (C0c) and the S2 points it reads: Cr = 9 C0c + 2 Dm generic,
  10 C0c + 4 Dm negabinary (dequantisation of S1, S2, S3); s the subnormal
  floor; G = 1.0001 the second-order terms.  kappa = worst rounding of one 1-D rule per unit input:
  2.875 cubic (2.75 inside, 2.875 at the edges, see interp._F), 1 linear.
  Fixed-point levels lose < one quantum per floor.
* Greedy planner: take the step with the largest bound decrease per byte
  until the bound meets the target (the paper uses greedy for PMGARD and a DP
  / best-first search for its own modes; greedy is this build's reading).
"""
import math

import numpy as np

LAMBDA = {"linear": 1.0, "cubic": 1.25}
KAPPA = {"linear": 1.0, "cubic": 2.875}
U_W = {"f32": 2.0 ** -24, "f64": 2.0 ** -53}
# 256 times the largest absolute rounding error of a subnormal result
SUBNORMAL = {"f32": 2.0 ** -142, "f64": 2.0 ** -1067}
MARGIN = 1.000000001
ROUND2 = 1.0001      # second-order rounding terms (n u < 1e-4 for the chains here)


def _up(x):
    """float(x) rounded up (x: python int or float)."""
    f = float(x)
    if isinstance(x, int) and int(f) < x:
        f = math.nextafter(f, math.inf)
    return f


# --------------------------------------------------------------------------
# per-stream tables
# --------------------------------------------------------------------------

def nb_dropped_max(k):
    """Largest |value| of k negabinary digits: floor((2^(k+1) - 1) / 3)."""
    return ((1 << (k + 1)) - 1) // 3


def stream_tables(enc, n_real, is_int, B, encoding, h, psnr_mode, bytes_b):
    """maxerr[b], sq[b] (rigorous upper bounds) and bytes[b], b = 0..B."""
    qd = enc["quant"]
    if is_int:
        vmax_abs = _up(qd["vmax"]) * h
        unit = math.ldexp(h, qd["sh"] + (3 if encoding == "negabinary" else 0))
    else:
        vmax_abs = qd["vmax"]
        unit = math.ldexp(1.0, qd["E"] - B + (3 if encoding == "negabinary" else 0))
    zero = qd["vmax"] == 0
    maxerr = [0.0] * (B + 1)
    sq = [0.0] * (B + 1)
    for b in range(B + 1):
        if zero:
            continue
        if b == 0:
            maxerr[b] = vmax_abs
        elif encoding == "generic":
            maxerr[b] = math.ldexp(unit, B - b)
        else:
            maxerr[b] = _up(nb_dropped_max(B - b) + 1) * unit
    if zero:
        return dict(maxerr=maxerr, sq=sq, bytes=bytes_b, unit=unit)
    if psnr_mode:
        C = enc["pairs"]
        for b in range(B + 1):
            s2 = 0
            s1 = 0
            for j in range(b, B):
                for jj in range(b, B):
                    w = 2 * B - 2 - j - jj
                    if encoding == "generic":
                        s2 += C[j, jj] << w
                    else:
                        s2 += (-1) ** (j + jj) * (C[j, jj] << w)
                if encoding == "generic":
                    s1 += C[j, j] << (B - 1 - j)
            if encoding != "generic":
                s1 = math.isqrt(n_real * s2)
                if s1 * s1 < n_real * s2:
                    s1 += 1
            total = s2 + 2 * s1 + n_real
            sq[b] = _up(total) * unit * unit
    else:
        for b in range(B + 1):
            sq[b] = n_real * maxerr[b] * maxerr[b]
    return dict(maxerr=maxerr, sq=sq, bytes=bytes_b, unit=unit)


# --------------------------------------------------------------------------
# spectral factors of the 1-D upsampling operators (L2 composition)
# --------------------------------------------------------------------------

def pass_matrix(m, degree):
    """P: (m//2) x ceil(m/2) weights mapping even-index values of a line of m
    points to its odd indices (same boundary rules as interp.predict_line)."""
    mc = (m + 1) // 2
    P = np.zeros((m // 2, mc))
    for t, j in enumerate(range(1, m, 2)):
        p1, m3, p3 = j + 1 < m, j - 3 >= 0, j + 3 < m
        if degree == "cubic" and p1 and m3 and p3:
            w = {j - 3: -1 / 16, j - 1: 9 / 16, j + 1: 9 / 16, j + 3: -1 / 16}
        elif degree == "cubic" and p1 and p3:
            w = {j - 1: 3 / 8, j + 1: 6 / 8, j + 3: -1 / 8}
        elif degree == "cubic" and p1 and m3:
            w = {j - 3: -1 / 8, j - 1: 6 / 8, j + 1: 3 / 8}
        elif p1:
            w = {j - 1: 0.5, j + 1: 0.5}
        else:
            w = {j - 1: 1.0}
        for src, val in w.items():
            P[t, src // 2] += val
    return P


_RS_CACHE = {}


def rowsum_ptp(m, degree):
    """||P^T P||_inf (exact in float64: weights are dyadic)."""
    key = (m, degree)
    if key not in _RS_CACHE:
        P = pass_matrix(m, degree)
        _RS_CACHE[key] = float(np.abs(P.T @ P).sum(axis=1).max()) if P.size else 0.0
    return _RS_CACHE[key]


# --------------------------------------------------------------------------
# composition
# --------------------------------------------------------------------------

class Composer:
    """Bound composition for one refactored field (see module docstring)."""

    def __init__(self, meta, streams):
        self.m = meta
        self.st = streams      # list of dict(level, region, sub, n_real, ...)
        self.L = meta["L"]
        self.d = meta["d"]
        self.lam = LAMBDA[meta["degree"]]
        self.uw = U_W[meta["dtype"]]
        self.h = meta["h"]
        self.M = meta["M"]
        self.C0 = meta["C0"]
        kap = KAPPA[meta["degree"]]
        lam_d1 = 1.0
        for _ in range(self.d - 1):
            lam_d1 *= self.lam
        self.lam_d = lam_d1 * self.lam
        self.rho_fix = (2.0 * self.d * lam_d1 + 2.0) * self.h
        neg = 1.0 if meta["encoding"] == "negabinary" else 0.0
        self.C0c = meta["C0c"]
        if meta["decomp_axis"] >= 0:
            self.cr = (9.0 + neg) * self.C0c + (2.0 + 2.0 * neg) * meta["Dm"]
        else:
            self.cr = (1.0 + neg) * self.C0c
        self.sub = SUBNORMAL[meta["dtype"]]
        self.kap = kap
        # stream groups
        self.by_level = {}
        for i, s in enumerate(streams):
            self.by_level.setdefault(s["level"], []).append(i)

    # ---- L-infinity -------------------------------------------------------
    def _mag(self, E1, e0sum):
        """Y: bound on |x'| and on the inputs of the retrieval's level-0
        prediction."""
        return self.M + self.lam_d * (E1 + e0sum)

    def _pred_rounding(self, Y):
        """Pr: rounding of the level-0 prediction, refactoring + retrieval."""
        M, lam, d = self.M, self.lam, self.d
        if self.m["interp"] != "level":
            return self.kap * (M + Y)
        cap = self.C0c * (1.0 + 2.0 * self.uw)
        acc = 0.0
        lk = 1.0                       # Lam^(k-1)
        for k in range(d):
            vr = M if k == 0 else min(lk * M, M + cap)
            vt = Y if k == 0 else min(lk * Y, Y + cap)
            prop = 1.0                 # Lam^(d-k), later passes
            for _ in range(d - 1 - k):
                prop *= lam
            acc += prop * (vr + vt)
            lk *= lam
        return self.kap * acc

    def rho0(self, E1, e0sum):
        if self.L == 1:
            return MARGIN * 1.01 * self.uw * self.C0
        Y = self._mag(E1, e0sum)
        return ROUND2 * self.uw * (self._pred_rounding(Y) + Y + self.cr) + self.sub

    def conv(self, E1, e0sum):
        """Rounding of the fixed-point coarse values to the field dtype."""
        return ROUND2 * self.uw * self._mag(E1, e0sum)

    def region_errors(self, level, err):
        """e_{l,r} per region (sum of sub-streams); region 0 = whole level."""
        out = {}
        for i in self.by_level[level]:
            r = self.st[i]["region"]
            out[r] = out.get(r, 0.0) + err[i]
        return out

    def linf(self, err):
        """Composed bound E_0 from per-stream errors ``err``."""
        L = self.L
        E = err[self.by_level[L - 1][0]] + (self.h if L - 1 >= 1 else 0.0)
        if L == 1:
            return (E + self.rho0(0.0, 0.0)) * MARGIN
        for level in range(L - 2, -1, -1):
            reg = self.region_errors(level, err)
            if level == 0:
                rho = self.rho0(E, sum(reg.values()))
                E = E + self.conv(E, sum(reg.values()))
            else:
                rho = self.rho_fix
            if self.m["interp"] == "level":
                e = max(reg.values())
                E = self.lam_d * E + e + rho
            else:
                F = []
                for r in sorted(reg):
                    base = E
                    for f in F:
                        base = max(base, f)
                    F.append(self.lam * base + reg[r] + rho)
                for f in F:
                    E = max(E, f)
        return E * MARGIN

    # ---- L2 ---------------------------------------------------------------
    def _e1_and_e0(self, err):
        """E_1 (composed bound of level 1) and the sum of level-0 region
        errors: the magnitude terms of the level-0 rounding allowance."""
        L = self.L
        if L == 1:
            return 0.0, 0.0
        E = err[self.by_level[L - 1][0]] + (self.h if L - 1 >= 1 else 0.0)
        for level in range(L - 2, 0, -1):
            reg = self.region_errors(level, err)
            if self.m["interp"] == "level":
                E = self.lam_d * E + max(reg.values()) + self.rho_fix
            else:
                F = []
                for r in sorted(reg):
                    base = E
                    for f in F:
                        base = max(base, f)
                    F.append(self.lam * base + reg[r] + self.rho_fix)
                for f in F:
                    E = max(E, f)
        return E, sum(self.region_errors(0, err).values())

    def l2(self, sq, err):
        """Upper bound on the sum of squared errors (per-stream sq, and the
        per-stream max errors of the same plan for the rounding terms)."""
        m = self.m
        L = self.L
        cnt = m["level_counts"]
        N = math.sqrt(sq[self.by_level[L - 1][0]])
        if L == 1:
            N += self.rho0(0.0, 0.0) * math.sqrt(cnt[0])
            return (N * N) * MARGIN
        N += self.h * math.sqrt(cnt[L - 1])
        E1, e0 = self._e1_and_e0(err)
        for level in range(L - 2, -1, -1):
            rho = self.rho0(E1, e0) if level == 0 else self.rho_fix
            if level == 0:
                N = N + self.conv(E1, e0) * math.sqrt(m["n"] - cnt[0])
            groups = {}
            for i in self.by_level[level]:
                s = self.st[i]
                groups.setdefault(s["region"], []).append((s["sub"], i))
            cnorm = {}
            for r, items in groups.items():
                items.sort()
                if items[0][0] == 0:
                    cnorm[r] = math.sqrt(sq[items[0][1]])
                else:
                    a2, a3 = m["decomp_factors"][r]
                    n1 = math.sqrt(sq[items[0][1]])
                    n2 = math.sqrt(sq[items[1][1]]) + a2 * n1
                    n3 = math.sqrt(sq[items[2][1]]) + a3 * math.sqrt(n1 * n1 + n2 * n2)
                    cnorm[r] = math.sqrt(n1 * n1 + n2 * n2 + n3 * n3)
            if m["interp"] == "level":
                c = 0.0
                for r in sorted(cnorm):
                    c += cnorm[r] * cnorm[r]
                t = m["level_factor"][level] * N + math.sqrt(c) + rho * math.sqrt(cnt[level])
                N = math.sqrt(N * N + t * t)
            else:
                T = N * N
                for r in sorted(cnorm):
                    t = (m["region_factor"][(level, r)] * math.sqrt(T) + cnorm[r]
                         + rho * math.sqrt(m["region_counts"][(level, r)]))
                    T += t * t
                N = math.sqrt(T)
        return (N * N) * MARGIN


# --------------------------------------------------------------------------
# staircases, max ordering and the greedy planner
# --------------------------------------------------------------------------

def useful_steps(vals, bytes_b):
    """Plane counts that strictly lower ``vals`` (from b = 0), with their byte
    increments: [(b, vals[b], bytes[b] - bytes[prev])]."""
    out = []
    b = 0
    B = len(vals) - 1
    while True:
        nb = b + 1
        while nb <= B and not vals[nb] < vals[b]:
            nb += 1
        if nb > B:
            return out
        out.append((nb, vals[nb], bytes_b[nb] - bytes_b[b]))
        b = nb


def _region_sequence(ids, tabs):
    """Greedy loading order inside one decomposed region: repeatedly add the
    next useful plane step of the sub-stream with the largest decrease of
    e_1 + e_2 + e_3 per byte (ties: lower sub-level)."""
    b = {i: 0 for i in ids}
    steps = {i: useful_steps(tabs[i]["maxerr"], tabs[i]["bytes"]) for i in ids}
    pos = {i: 0 for i in ids}

    def total():
        t = 0.0
        for i in ids:
            t = t + tabs[i]["maxerr"][b[i]]
        return t

    cur = total()
    seq = []
    while True:
        best = None
        for i in ids:
            if pos[i] >= len(steps[i]):
                continue
            nb, val, db = steps[i][pos[i]]
            de = tabs[i]["maxerr"][b[i]] - val
            ratio = math.inf if db == 0 else de / db
            if best is None or ratio > best[0]:
                best = (ratio, i, nb, db)
        if best is None:
            return seq
        _, i, nb, db = best
        b[i] = nb
        pos[i] += 1
        cur = total()
        seq.append((cur, [(i, nb)], db))


def max_ordering(level_ids_by_region, tabs):
    """Sec. V-C max ordering: merge the per-region loading orders by
    descending cumulative error; steps with equal error merge into one
    segment.  Returns (initial level error, [(updates, bytes, level error)])."""
    allsteps = []
    cur = {}
    for r, ids in sorted(level_ids_by_region.items()):
        t = 0.0
        for i in ids:
            t = t + tabs[i]["maxerr"][0]
        cur[r] = t
        for k, (e, upd, db) in enumerate(_region_sequence(ids, tabs)):
            allsteps.append((e, r, k, upd, db))
    allsteps.sort(key=lambda s: (-s[0], s[1], s[2]))
    init = max(cur.values())
    segs = []
    i = 0
    while i < len(allsteps):
        j = i
        upd, db = [], 0
        while j < len(allsteps) and allsteps[j][0] == allsteps[i][0]:
            e, r, k, u, d = allsteps[j]
            upd += u
            db += d
            cur[r] = e
            j += 1
        segs.append((upd, db, max(cur.values())))
        i = j
    return init, segs


class Unit:
    def __init__(self, ids, steps, weight):
        self.ids = ids          # stream indices
        self.steps = steps      # [(updates [(stream, b)], dbytes, unit value)]
        self.weight = weight


def _compress(init, segs):
    """Merge segments that do not lower the unit value into the next one."""
    out = []
    upd, db, prev = [], 0, init
    for u, d, v in segs:
        upd = upd + u
        db += d
        if v < prev:
            out.append((upd, db, v))
            upd, db, prev = [], 0, v
    return out


def build_units(comp, tabs, kind):
    """Planning units.  kind 'linf': per-level levels (max-ordered at a
    decomposed level 0) or per-region streams; kind 'l2': every stream."""
    units = []
    d = comp.d
    for level in range(comp.L - 1, -1, -1):
        ids = comp.by_level[level]
        w = float(2 ** (d * level))
        if kind == "linf" and comp.m["interp"] == "level" and len(ids) > 1:
            by_r = {}
            for i in ids:
                by_r.setdefault(comp.st[i]["region"], []).append(i)
            init, segs = max_ordering(by_r, tabs)
            units.append(Unit(ids, _compress(init, segs), w))
        else:
            key = "maxerr" if kind == "linf" else "sq"
            for i in ids:
                st = [([(i, nb)], db, v) for nb, v, db in useful_steps(tabs[i][key], tabs[i]["bytes"])]
                units.append(Unit([i], st, w))
    return units


def greedy(comp, tabs, target, kind, have=None):
    """Greedy interpreter: returns (planes per stream, bound, satisfied).

    ``have`` (incremental invocation, the progressive retrieval of Sec. III-A
    reusing fetched planes): planes already fetched per stream.  The plan
    starts there and never drops a plane; a step costs only the bytes of the
    planes it adds beyond what is fetched, and steps whose planes are all
    fetched are passed over.  Without ``have`` every step costs its
    staircase increment (the same number when nothing is fetched)."""
    n = len(tabs)
    b = list(have) if have is not None else [0] * n
    units = build_units(comp, tabs, kind)
    pos = [0] * len(units)
    if have is not None:
        for ui, u in enumerate(units):
            while pos[ui] < len(u.steps) and all(nb <= b[i] for i, nb in u.steps[pos[ui]][0]):
                pos[ui] += 1

    def step_cost(upd, db, bb):
        if have is None:
            return db
        top = {}
        for i, nb in upd:
            top[i] = max(top.get(i, 0), nb)
        return sum(tabs[i]["bytes"][max(nb, bb[i])] - tabs[i]["bytes"][bb[i]] for i, nb in top.items())

    def evaluate(bb):
        err = [tabs[i]["maxerr"][bb[i]] for i in range(n)]
        if kind == "linf":
            return comp.linf(err)
        sq = [tabs[i]["sq"][bb[i]] for i in range(n)]
        return comp.l2(sq, err)

    def unit_value(u, bb):
        key = "maxerr" if kind == "linf" else "sq"
        if len(u.ids) == 1:
            return tabs[u.ids[0]][key][bb[u.ids[0]]]
        reg = {}
        for i in u.ids:
            r = comp.st[i]["region"]
            reg[r] = reg.get(r, 0.0) + tabs[i]["maxerr"][bb[i]]
        return max(reg.values())

    bound = evaluate(b)
    while bound > target:
        best = None
        fallback = None
        for ui, u in enumerate(units):
            if pos[ui] >= len(u.steps):
                continue
            upd, db, _ = u.steps[pos[ui]]
            db = step_cost(upd, db, b)
            trial = list(b)
            for i, nb in upd:
                trial[i] = nb if have is None else max(trial[i], nb)
            nbnd = evaluate(trial)
            gain = bound - nbnd
            ratio = math.inf if db == 0 else gain / db
            if gain > 0 or db == 0:
                if best is None or ratio > best[0]:
                    best = (ratio, ui, trial, nbnd)
            own = (unit_value(u, b) - unit_value(u, trial)) * u.weight
            fr = math.inf if db == 0 else own / db
            if fallback is None or fr > fallback[0]:
                fallback = (fr, ui, trial, nbnd)
        if best is None:
            best = fallback
        if best is None:
            return b, bound, False
        _, ui, b, bound = best
        pos[ui] += 1
    return b, bound, True


# --------------------------------------------------------------------------
# best-first search interpreter
# --------------------------------------------------------------------------

SEARCH_NODES = 4096     # default expansion budget of the search


def unit_planes(units, n, have=None):
    """Per unit u and position p (its first p steps taken): the plane count
    of each of its streams, {stream: planes}, starting from ``have`` (or
    zero) the way the greedy applies steps."""
    out = []
    for u in units:
        cur = {i: (have[i] if have is not None else 0) for i in u.ids}
        seq = [dict(cur)]
        for upd, _, _ in u.steps:
            for i, nb in upd:
                cur[i] = nb if have is None else max(cur[i], nb)
            seq.append(dict(cur))
        out.append(seq)
    return out


def best_first(comp, tabs, target, kind, have=None, max_nodes=SEARCH_NODES):
    """Best-first search for the smallest retrieval meeting the bound
    (Sec. VI-B: per-level + decomposition uses a best-first search with
    pruning and incremental invocation; per-region a dynamic program -- both
    aim at the fewest bytes whose bound meets the target).  Reading: one
    search for every mode, over the greedy's planning units; a state is the
    number of steps taken in each unit (positions), its cost the bytes it
    adds to ``have`` (or to nothing); the bound is monotone in every unit.

    * lower positions: unit u needs at least q_u steps, the fewest for which
      the bound meets the target with every other unit complete;
    * incumbent: the greedy plan, at its positions (per unit the last
      position with the greedy's planes), improved by local moves until none
      applies: for each unit in turn, drop its last step while that is
      cheaper and meets the target; then for each ordered pair of units
      (a, b), move one step from a to b when that is cheaper and meets the
      target;
    * uniform-cost order from q over a tree that reaches every state once
      (a state only advances units at or after the one its parent
      advanced); key (cost, push order); a child that meets the target
      becomes the incumbent when cheaper; children costing at least the
      incumbent are cut; the search stops when the cheapest open state
      costs at least the incumbent (the incumbent is then the minimum) or
      after ``max_nodes`` expansions (the best plan found so far).

    Returns (planes, bound, satisfied, info) with info = dict(expanded,
    optimal, greedy_bytes) (greedy_bytes counted like the cost)."""
    import heapq

    n = len(tabs)
    bg, bound_g, ok = greedy(comp, tabs, target, kind, have)
    base = list(have) if have is not None else [0] * n

    def added(bb):
        return sum(tabs[i]["bytes"][bb[i]] - tabs[i]["bytes"][base[i]] for i in range(n))

    info = dict(expanded=0, optimal=False, greedy_bytes=added(bg))
    if not ok:
        return bg, bound_g, False, info
    units = build_units(comp, tabs, kind)
    U = len(units)
    pls = unit_planes(units, n, have)
    S = [len(u.steps) for u in units]
    cost = [[sum(tabs[i]["bytes"][pl[i]] - tabs[i]["bytes"][base[i]] for i in pl) for pl in seq] for seq in pls]
    start = [0] * U
    if have is not None:
        for ui, u in enumerate(units):
            while start[ui] < S[ui] and all(nb <= base[i] for i, nb in u.steps[start[ui]][0]):
                start[ui] += 1

    def planes_of(pos):
        bb = list(base)
        for ui in range(U):
            for i, v in pls[ui][pos[ui]].items():
                bb[i] = v
        return bb

    def bound_of(pos):
        bb = planes_of(pos)
        err = [tabs[i]["maxerr"][bb[i]] for i in range(n)]
        if kind == "linf":
            return comp.linf(err)
        return comp.l2([tabs[i]["sq"][bb[i]] for i in range(n)], err)

    q = []
    for ui in range(U):
        pos = list(S)
        p = start[ui]
        while True:
            pos[ui] = p
            if p == S[ui] or bound_of(pos) <= target:
                break
            p += 1
        q.append(p)

    # the greedy's positions, then local moves
    pos = []
    for ui in range(U):
        p = 0
        for k in range(S[ui] + 1):
            if all(bg[i] == v for i, v in pls[ui][k].items()):
                p = k
        pos.append(p)
    c_best, best_bound = info["greedy_bytes"], bound_g
    changed = True
    while changed:
        changed = False
        for a in range(U):
            while pos[a] > max(start[a], q[a]):
                t = list(pos)
                t[a] -= 1
                ct = c_best - cost[a][pos[a]] + cost[a][t[a]]
                if ct >= c_best:
                    break
                v = bound_of(t)
                if v > target:
                    break
                pos, c_best, best_bound, changed = t, ct, v, True
        for a in range(U):
            for b2 in range(U):
                if b2 == a or pos[a] <= max(start[a], q[a]) or pos[b2] >= S[b2]:
                    continue
                t = list(pos)
                t[a] -= 1
                t[b2] += 1
                ct = c_best - cost[a][pos[a]] + cost[a][t[a]] - cost[b2][pos[b2]] + cost[b2][t[b2]]
                if ct >= c_best:
                    continue
                v = bound_of(t)
                if v <= target:
                    pos, c_best, best_bound, changed = t, ct, v, True
    best_b = planes_of(pos)

    c0 = sum(cost[ui][q[ui]] for ui in range(U))
    if c0 >= c_best:
        info["optimal"] = True
        return best_b, best_bound, True, info
    v = bound_of(q)
    if v <= target:
        info["optimal"] = True
        return planes_of(q), v, True, info
    heap = [(c0, 0, tuple(q), 0)]
    seq = 1
    while heap:
        c, _, pos, lu = heapq.heappop(heap)
        if c >= c_best:
            break
        if info["expanded"] >= max_nodes:
            return best_b, best_bound, True, info
        info["expanded"] += 1
        for ui in range(lu, U):
            p = pos[ui]
            if p >= S[ui]:
                continue
            nc = c + cost[ui][p + 1] - cost[ui][p]
            if nc >= c_best:
                continue
            child = pos[:ui] + (p + 1,) + pos[ui + 1:]
            v = bound_of(child)
            if v <= target:
                best_b, best_bound, c_best = planes_of(child), v, nc
            else:
                heapq.heappush(heap, (nc, seq, child, ui))
                seq += 1
    info["optimal"] = True
    return best_b, best_bound, True, info
