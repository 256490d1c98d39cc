"""Block sharding of one field (oracle).  Test infrastructure only.

Sec. VII's scaling experiment refactors fixed blocks of a field
independently, one block per core, and retrieves the field from them.
Here a field is split along axis 0 into contiguous slabs, each refactored
as a field of its own (no halo: blocks do not read each other), and a
target for the whole field is planned over all blocks' tables together:

* error bounds (abs, rel): relative targets use the whole field's range;
  every block is planned for the same absolute tolerance with its own
  interpreter (the field's max error is its blocks' largest), so the plan
  of a block does not depend on the others;
* PSNR: one budget of squared errors for the whole field, N (R 10^(-p/20))^2
  (N points, R the field's range), spent by one greedy over the planning
  units of every block: each step is the one with the largest decrease of
  its own block's L2 bound per byte (strictly larger wins, so ties go to
  the earlier block and, within it, the earlier unit), until the blocks'
  bounds sum to at most the budget; when no step lowers a bound, the step
  with the largest decrease of its own stream's squared-error table entry
  (times the unit's weight) per byte, as the one-field interpreter does.
  With one block this is the block's own interpreter.

Readings (the paper states no more): slabs of ceil or floor of n0 / k
planes, the first n0 mod k of them one plane thicker; blocks refactored
with the whole field's scheme.
"""
import math

import numpy as np

from . import bounds as bd
from .pipeline import plan, refactor, retrieve, Target


def split(X, k):
    """Contiguous axis-0 slabs of X: list of (start, stop)."""
    n0 = X.shape[0]
    if not 1 <= k <= n0:
        raise ValueError("need 1 <= k <= n0")
    out, a = [], 0
    for i in range(k):
        t = n0 // k + (1 if i < n0 % k else 0)
        out.append((a, a + t))
        a += t
    return out


def refactor_blocks(X, scheme, k):
    """One oracle handle per slab; returns (handles, slabs)."""
    sl = split(X, k)
    return [refactor(np.ascontiguousarray(X[a:b]), scheme) for a, b in sl], sl


def field_range(hs):
    return max(h["meta"]["xmax"] for h in hs) - min(h["meta"]["xmin"] for h in hs)


def _greedy_l2_global(hs, budget):
    """The PSNR greedy over every block's units (see module docstring)."""
    tabs = [[s["tab"] for s in h["streams"]] for h in hs]
    comps = [h["comp"] for h in hs]
    units = [bd.build_units(c, t, "l2") for c, t in zip(comps, tabs)]
    b = [[0] * len(t) for t in tabs]
    pos = [[0] * len(u) for u in units]

    def bound_of(k, bb):
        t = tabs[k]
        err = [t[i]["maxerr"][bb[i]] for i in range(len(t))]
        sq = [t[i]["sq"][bb[i]] for i in range(len(t))]
        return comps[k].l2(sq, err)

    E = [bound_of(k, b[k]) for k in range(len(hs))]
    total = sum(E)
    while total > budget:
        best = fallback = None
        for k in range(len(hs)):
            for ui, u in enumerate(units[k]):
                if pos[k][ui] >= len(u.steps):
                    continue
                upd, db, _ = u.steps[pos[k][ui]]
                trial = list(b[k])
                for i, nb in upd:
                    trial[i] = nb
                nE = bound_of(k, trial)
                gain = E[k] - nE
                ratio = math.inf if db == 0 else gain / db
                if gain > 0 or db == 0:
                    if best is None or ratio > best[0]:
                        best = (ratio, k, ui, trial, nE)
                i0 = u.ids[0]
                own = (tabs[k][i0]["sq"][b[k][i0]] - tabs[k][i0]["sq"][trial[i0]]) * u.weight
                fr = math.inf if db == 0 else own / db
                if fallback is None or fr > fallback[0]:
                    fallback = (fr, k, ui, trial, nE)
        if best is None:
            best = fallback
        if best is None:
            return b, total, False
        _, k, ui, trial, nE = best
        b[k] = trial
        pos[k][ui] += 1
        total = total - E[k] + nE
        E[k] = nE
    return b, total, True


def plan_global(hs, target):
    """Plans of every block for a whole-field target: (plans, bound,
    satisfied); bound = max error bound (abs/rel) or the summed squared-
    error bound (PSNR)."""
    R = field_range(hs)
    if target.kind in ("abs", "rel"):
        tau = target.value * (R if target.kind == "rel" else 1.0)
        pls = [plan(h, Target("abs", tau)) for h in hs]
        return pls, max(p["bound"] for p in pls), all(p["satisfied"] for p in pls)
    N = sum(h["meta"]["n"] for h in hs)
    ratio = R / (10.0 ** (target.value / 20.0))
    b, total, ok = _greedy_l2_global(hs, N * ratio * ratio)
    pls = []
    for h, bb in zip(hs, b):
        tabs = [s["tab"] for s in h["streams"]]
        pls.append(dict(b=bb, bound=None, satisfied=ok, bytes=sum(t["bytes"][i] for t, i in zip(tabs, bb)),
                        kind="psnr"))
    return pls, total, ok


def retrieve_blocks(hs, slabs, pls, shape, dtype):
    """The whole field from its blocks' retrievals."""
    out = np.zeros(shape, dtype)
    for h, (a, b), p in zip(hs, slabs, pls):
        out[a:b], _ = retrieve(h, p)
    return out
