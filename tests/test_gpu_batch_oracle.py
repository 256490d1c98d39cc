"""Batched refactor against the oracle, and the size of its captured graph.

The batched forms run the refactor stage by stage across all fields of the
batch (statistics, level-0 prediction, fixed-point copy, coarsest level,
fixed-point levels, decomposition, row padding, encode), each stage in as
few launches as the batched kernels' parameter blocks allow.

* Fields: two of each shape class of the 96-field batch workload at reduced
  size (3-D 100x500x500 -> 20x52x64, 3-D 64x256x1024 -> 16x32x128, 2-D
  1800x3600 -> 90x180; the 3-D ones take the batched plane-marching and
  TMA-decomposition kernels), one ragged 3-D field (21x45x70: the general
  tile and decomposition kernels) and one FP64 field.
* Every handle from refactor_batch, from RefactorGraph's creation and from a
  graph run on refilled inputs equals oracle.refactor of its field stream
  for stream (planes, signs, counts, tables).
* The captured graph holds tens of kernels whatever the batch size: 3x the
  fields add at most a few launches (stages whose items outgrow one
  parameter block), not 3x the kernels.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _fields(seed):
    from synth import grf
    shapes = [(20, 52, 64), (20, 52, 64), (16, 32, 128), (16, 32, 128), (90, 180), (90, 180), (21, 45, 70)]
    xs = [grf(s, seed + i, np.float32) for i, s in enumerate(shapes)]
    xs.append(grf((18, 30, 40), seed + 50, np.float64))
    return xs


def _schemes(Xs):
    import paper_2609_04573_b300 as pcr
    return [pcr.Scheme(interp="level", degree="cubic", decomp_axis=2 if X.ndim == 3 else -1) for X in Xs]


def _check_all(hs, Xs, schs):
    import oracle
    from _compare import oracle_scheme, compare_streams
    for h, X, s in zip(hs, Xs, schs):
        compare_streams(h, oracle.refactor(X, oracle_scheme(s, X.ndim)))


def test_refactor_batch_equals_the_oracle():
    import paper_2609_04573_b300 as pcr
    Xs = _fields(301)
    schs = _schemes(Xs)
    hs = pcr.refactor_batch([torch.from_numpy(X).cuda() for X in Xs], schs)
    _check_all(hs, Xs, schs)


def test_refactor_graph_equals_the_oracle_and_stays_small():
    import paper_2609_04573_b300 as pcr
    Xs = _fields(401)
    schs = _schemes(Xs)
    xs = [torch.from_numpy(X).cuda() for X in Xs]
    g = pcr.RefactorGraph(xs, schs)
    _check_all(g.handles, Xs, schs)
    Ys = _fields(501)
    for x, Y in zip(xs, Ys):
        x.copy_(torch.from_numpy(Y))
    g.run()
    _check_all(g.handles, Ys, schs)
    k1 = g.info()["kernels"]
    # the same classes three times over
    Zs = _fields(601) + _fields(701) + _fields(801)
    g3 = pcr.RefactorGraph([torch.from_numpy(Z).cuda() for Z in Zs], _schemes(Zs))
    k3 = g3.info()["kernels"]
    assert k1 <= 40 and k3 <= k1 + 6, (k1, k3)
