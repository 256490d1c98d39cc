"""Target-driven sampled tuning (oracle).  Test infrastructure only.

Sec. VI-A: sample 1 % of the field uniformly, evaluate the retrieval
efficiency of every candidate configuration at 9 tolerances (1e-3, 5e-4,
1e-4, ..., 1e-7) and vote: at each tolerance the configuration that needs the
fewest bytes gets one vote; the configuration with the most votes wins.
Candidates (tuning table of Sec. VI-A): error-bound mode -- per-level or
per-region interpolation (6 pass orders in 3-D), coefficient decomposition
off or along one of the 3 axes, generic planes; PSNR mode -- per-region only,
the same decomposition options, negabinary + XOR planes.  Cubic interpolation
throughout (the paper's choice, Sec. IV).

Readings (the paper gives no more detail):
* "uniformly sample 1 %": whole blocks of b^D points (b = min(64, n) per axis;
  interpolation needs neighbours, so single points would not do), centred on
  a regular k_0 x .. x k_(D-1) grid; the counts grow one axis at a time (the
  axis with the most points per block slot first) while the blocks stay
  within `fraction` of the field, at least one block.  Each block is
  refactored as a field of its own.
* tolerances are relative to the whole field's range R.  Error-bound mode:
  every block planned for max |x - x'| <= tau R.  PSNR mode: for
  RMSE <= tau R, i.e. PSNR >= -20 log10(tau), every block planned for a sum
  of squared errors <= n_block (tau R)^2.
* a configuration that cannot meet a tolerance in some block takes no part
  in that tolerance's vote; equal byte counts go to the earlier candidate; a
  tie of votes goes to the earlier candidate.
"""
import itertools

import numpy as np

from . import bounds as bd
from .pipeline import Scheme, refactor

TOLERANCES = (1e-3, 5e-4, 1e-4, 5e-5, 1e-5, 5e-6, 1e-6, 5e-7, 1e-7)


def candidates(mode, ndim):
    """Candidate schemes in the order ties are broken (pass orders in the
    oracle's axes: a 2-D field is its 3-D view 1 x n0 x n1, axes 1 and 2)."""
    axes = tuple(range(ndim)) if ndim == 3 else (1, 2)
    orders = list(itertools.permutations(axes))
    decomps = (-1, 0, 1, 2) if ndim == 3 else (-1,)
    out = []
    if mode == "eb":
        interps = [("level", None)] + [("region", o) for o in orders]
        enc = "generic"
    else:
        interps = [("region", o) for o in orders]
        enc = "negabinary"
    for interp, order in interps:
        for dax in decomps:
            out.append(Scheme(mode=mode, interp=interp, degree="cubic", order=order, decomp_axis=dax,
                              encoding=enc))
    return out


def sample_blocks(shape, fraction=0.01, edge=64):
    """Block origins and edges of the uniform sample (see module docstring)."""
    D = len(shape)
    b = [min(edge, n) for n in shape]
    N = int(np.prod(shape))
    per = int(np.prod(b))
    k = [1] * D
    while True:
        ratios = [shape[d] / (k[d] + 1) for d in range(D)]
        best = None
        for d in range(D):
            if (k[d] + 1) * b[d] <= shape[d] and (best is None or ratios[d] > ratios[best]):
                best = d
        if best is None:
            break
        trial = list(k)
        trial[best] += 1
        if int(np.prod(trial)) * per > fraction * N:
            break
        k = trial
    origins = []
    for idx in itertools.product(*[range(kd) for kd in k]):
        o = []
        for d in range(D):
            c = ((2 * idx[d] + 1) * shape[d]) // (2 * k[d])      # slot centre
            o.append(min(max(c - b[d] // 2, 0), shape[d] - b[d]))
        origins.append(tuple(o))
    return origins, tuple(b)


def block_bytes(h, tau_abs, psnr):
    """Bytes one refactored block needs to meet the tolerance, or None."""
    tabs = [s["tab"] for s in h["streams"]]
    if psnr:
        b, bound, ok = bd.greedy(h["comp"], tabs, h["meta"]["n"] * tau_abs * tau_abs, "l2")
    else:
        b, bound, ok = bd.greedy(h["comp"], tabs, tau_abs, "linf")
    if not ok:
        return None
    return sum(t["bytes"][bi] for t, bi in zip(tabs, b))


def tune(X, mode="eb", fraction=0.01, edge=64, cands=None, tolerances=TOLERANCES):
    """Returns (winning scheme, votes per candidate, bytes[candidate][tol])."""
    X = np.asarray(X)
    R = float(X.max()) - float(X.min())
    cands = cands if cands is not None else candidates(mode, X.ndim)
    origins, b = sample_blocks(X.shape, fraction, edge)
    blocks = [X[tuple(slice(o, o + e) for o, e in zip(org, b))] for org in origins]
    table = []
    for sch in cands:
        hs = [refactor(blk, sch) for blk in blocks]
        row = []
        for tau in tolerances:
            tot = 0
            for h in hs:
                nb = block_bytes(h, tau * R, mode == "psnr")
                if nb is None:
                    tot = None
                    break
                tot += nb
            row.append(tot)
        table.append(row)
    votes = [0] * len(cands)
    for t in range(len(tolerances)):
        best = None
        for c in range(len(cands)):
            v = table[c][t]
            if v is not None and (best is None or v < table[best][t]):
                best = c
        if best is not None:
            votes[best] += 1
    win = 0
    for c in range(len(cands)):
        if votes[c] > votes[win]:
            win = c
    return cands[win], votes, table
