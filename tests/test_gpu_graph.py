"""Batched refactor captured in one CUDA graph, and the level autotuner.

* pcr_refactor_graph: the handles after creation, and after every run on
  refilled inputs, refactor byte-for-byte like pcr_refactor of the same data
  (uneven 3-D and 2-D shapes, the plane-marching and the general levels);
  repeated runs on the same data give the same streams (sign slot tails are
  cleared in the graph); retrievals from graph handles equal single ones.
* Autotuner: with tuning on, a field whose levels have several schedules
  still matches the oracle bit for bit, and the table records every tuned
  (kind, direction, degree, grid) with a valid choice.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _same(ha, hb):
    assert ha.nstreams == hb.nstreams
    assert ha.field_stats() == hb.field_stats()
    for i in range(ha.nstreams):
        for u, v in zip(ha.stream_copy(i), hb.stream_copy(i)):
            assert np.array_equal(u, v), i
        assert ha.tables(i) == hb.tables(i)


def _fields(seed):
    from synth import grf
    return [grf((36, 44, 72), seed, np.float32), grf((96, 130), seed + 1, np.float32),
            grf((20, 33, 65), seed + 2, np.float32), grf((40, 40, 64), seed + 3, np.float32)]


def test_graph_handles_equal_single_refactors_across_runs():
    import paper_2609_04573_b300 as pcr
    xs = [torch.from_numpy(x).cuda() for x in _fields(51)]
    sch = [pcr.Scheme(interp="level", degree="cubic", decomp_axis=2 if x.dim() == 3 else -1) for x in xs]
    g = pcr.RefactorGraph(xs, sch)
    info = g.info()
    assert info["kernels"] > 0 and info["nodes"] >= info["kernels"] and info["arena_bytes"] > 0
    for x, s, hg in zip(xs, sch, g.handles):
        _same(hg, pcr.refactor(x, s))
    for seed in (61, 71):   # refill the captured inputs in place, run the graph
        for x, new in zip(xs, _fields(seed)):
            x.copy_(torch.from_numpy(new))
        g.run()
        for x, s, hg in zip(xs, sch, g.handles):
            _same(hg, pcr.refactor(x, s))
    g.run()                 # same data again: same streams
    for x, s, hg in zip(xs, sch, g.handles):
        _same(hg, pcr.refactor(x, s))
        t = pcr.Target("rel", 1e-3)
        out_g, pl_g = hg.retrieve(t)
        hs = pcr.refactor(x, s)
        out_s, pl_s = hs.retrieve(t)
        assert pl_g.planes == pl_s.planes
        assert torch.equal(out_g, out_s)


def test_autotuned_levels_match_the_oracle():
    import oracle
    import paper_2609_04573_b300 as pcr
    from synth import grf
    from _compare import oracle_scheme, compare_streams
    X = grf((37, 45, 260), 131, np.float32)
    sch = pcr.Scheme(interp="level", degree="cubic", decomp_axis=2)
    pcr.autotune_table(reset=True)
    pcr.autotune(True)
    try:
        h = pcr.refactor(torch.from_numpy(X).cuda(), sch)
        out, pl = h.retrieve(pcr.Target("rel", 1e-4))
    finally:
        pcr.autotune(False)
    table = pcr.autotune_table(reset=True)
    h_or = oracle.refactor(X, oracle_scheme(sch, 3))
    compare_streams(h, h_or)
    pl_or = oracle.plan(h_or, oracle.Target("rel", 1e-4))
    assert pl.planes == pl_or["b"]
    x_or, _ = oracle.retrieve(h_or, pl_or)
    assert np.array_equal(out.cpu().numpy(), x_or)
    # level 0 (f32) and level 1 (fixed point), refactor and retrieval
    kinds = {(k[0], k[1]) for k in table}
    assert {(0, 0), (0, 1), (2, 0), (2, 1)} <= kinds, table
    for (choice, ms) in table.values():
        assert choice in (0, 8, 16, 32, 64, -1, -2, -3) and ms >= 0
