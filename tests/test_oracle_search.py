"""Best-first search interpreter (oracle.bounds.best_first): pins.

* Brute force: on fields small enough to enumerate every combination of
  planning-unit positions, the search's plan costs exactly the fewest bytes
  of any combination whose composed bound meets the target (per-level with
  and without decomposition, per-region; L-infinity and L2 targets), and
  it says it proved that.
* With fetched planes (incremental invocation): the plan contains them and
  its added bytes equal the brute-force minimum over combinations that
  contain them.
* Never worse than the greedy, strictly better somewhere on these fields.
* A zero budget returns the greedy plan or a plan at the lower positions;
  an unsatisfiable target returns the greedy's all-planes answer.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import bounds as bd
from synth import grf

CASES = [((17, 17), 3, 12, "level", -1), ((9, 9, 9), 2, 10, "level", 0), ((12, 10, 9), 2, 10, "region", -1)]


def _handle(shape, L, B, interp, dax):
    X = grf(shape, 5, np.float32)
    return oracle.refactor(X, oracle.Scheme(mode="explicit", interp=interp, nlevels=L, nplanes=B, decomp_axis=dax))


def _brute(comp, tabs, goal, kind, have=None):
    """Fewest added bytes over every combination of unit positions (None
    when none meets the goal)."""
    n = len(tabs)
    units = bd.build_units(comp, tabs, kind)
    pls = bd.unit_planes(units, n, have)
    base = list(have) if have is not None else [0] * n
    best = None
    for pos in itertools.product(*[range(len(u.steps) + 1) for u in units]):
        b = list(base)
        for ui, p in enumerate(pos):
            for i, v in pls[ui][p].items():
                b[i] = v
        cost = sum(tabs[i]["bytes"][b[i]] - tabs[i]["bytes"][base[i]] for i in range(n))
        if best is not None and cost >= best:
            continue
        err = [tabs[i]["maxerr"][b[i]] for i in range(n)]
        v = comp.linf(err) if kind == "linf" else comp.l2([tabs[i]["sq"][b[i]] for i in range(n)], err)
        if v <= goal:
            best = cost
    return best


def _goal(h, kind, t):
    R = h["meta"]["R"]
    return t * R if kind == "linf" else h["meta"]["n"] * (t * R) ** 2


def _kinds(shape, interp):
    return ["linf"] if (len(shape) == 3 and interp == "level") else ["linf", "l2"]


@pytest.mark.parametrize("case", CASES)
def test_search_equals_brute_force(case):
    h = _handle(*case)
    tabs = [s["tab"] for s in h["streams"]]
    comp = h["comp"]
    improved = 0
    for kind in _kinds(case[0], case[3]):
        for t in (1e-1, 3e-2, 1e-2, 3e-3):
            goal = _goal(h, kind, t)
            want = _brute(comp, tabs, goal, kind)
            b, bound, ok, info = bd.best_first(comp, tabs, goal, kind, None, 10 ** 6)
            cost = sum(tabs[i]["bytes"][b[i]] for i in range(len(tabs)))
            if want is None:
                assert not ok
                continue
            assert ok and info["optimal"] and cost == want and bound <= goal
            err = [tabs[i]["maxerr"][b[i]] for i in range(len(tabs))]
            again = comp.linf(err) if kind == "linf" else comp.l2([tabs[i]["sq"][b[i]] for i in range(len(tabs))], err)
            assert again == bound
            assert cost <= info["greedy_bytes"]
            improved += cost < info["greedy_bytes"]
    assert improved >= 1


def test_search_from_fetched_planes():
    h = _handle((17, 17), 3, 12, "level", -1)
    tabs = [s["tab"] for s in h["streams"]]
    comp = h["comp"]
    for kind in ("linf", "l2"):
        first, _, _ = bd.greedy(comp, tabs, _goal(h, kind, 1e-1), kind)
        goal = _goal(h, kind, 1e-2)
        want = _brute(comp, tabs, goal, kind, first)
        b, bound, ok, info = bd.best_first(comp, tabs, goal, kind, first, 10 ** 6)
        assert ok and info["optimal"] and bound <= goal
        assert all(x >= y for x, y in zip(b, first))
        added = sum(tabs[i]["bytes"][b[i]] - tabs[i]["bytes"][first[i]] for i in range(len(tabs)))
        assert added == want <= info["greedy_bytes"]


def test_zero_budget_and_unsatisfiable():
    h = _handle((12, 10, 9), 2, 10, "region", -1)
    tabs = [s["tab"] for s in h["streams"]]
    comp = h["comp"]
    goal = _goal(h, "l2", 1e-1)
    gb, gbound, gok = bd.greedy(comp, tabs, goal, "l2")
    b, bound, ok, info = bd.best_first(comp, tabs, goal, "l2", None, 0)
    assert ok and bound <= goal and info["expanded"] == 0
    assert sum(tabs[i]["bytes"][b[i]] for i in range(len(tabs))) <= info["greedy_bytes"]
    goal = _goal(h, "linf", 1e-9)
    gb, gbound, gok = bd.greedy(comp, tabs, goal, "linf")
    b, bound, ok, info = bd.best_first(comp, tabs, goal, "linf", None, 100)
    assert not gok and not ok and b == gb and bound == gbound


def test_plan_entry_point():
    h = _handle((17, 17), 3, 12, "level", -1)
    g = oracle.plan(h, oracle.Target("rel", 3e-2))
    s = oracle.plan(h, oracle.Target("rel", 3e-2), search=10 ** 5)
    assert s["satisfied"] and s["bytes"] <= g["bytes"] and s["search"]["optimal"]
    assert "search" not in g
