"""Batched and served forms: every result equals the single-call result.

* pcr_refactor_batch: each field of a batch (uneven shapes, 2-D and 3-D)
  refactors byte-for-byte like its own pcr_refactor.
* Server (continuous batching, memory admission, two streams): every
  request's field equals the one a single retrieval of the same request
  returns, whatever the mix it was batched with, and served results (whole
  fields and boxes) equal the oracle's retrieval.
"""
import random
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _fields():
    from synth import grf
    return [grf((36, 44, 70), 41, np.float32), grf((96, 130), 42, np.float32),
            grf((20, 33, 65), 43, np.float32), grf((64, 64, 64), 44, np.float32)]


def test_refactor_batch_equals_single():
    import paper_2609_04573_b300 as pcr
    xs = [torch.from_numpy(x).cuda() for x in _fields()]
    sch = pcr.Scheme(interp="level", degree="cubic", decomp_axis=2)
    batch = pcr.refactor_batch(xs, sch)
    for x, hb in zip(xs, batch):
        hs = pcr.refactor(x, sch)
        assert hb.nstreams == hs.nstreams
        assert hb.field_stats() == hs.field_stats()
        for i in range(hs.nstreams):
            a, b = hb.stream_copy(i), hs.stream_copy(i)
            for u, v in zip(a, b):
                assert np.array_equal(u, v), i
            assert hb.tables(i) == hs.tables(i)


def test_server_results_equal_single_retrievals():
    import paper_2609_04573_b300 as pcr
    from paper_2609_04573_b300.serve import Server
    rng = random.Random(7)
    xs = [torch.from_numpy(x).cuda() for x in _fields()]
    hs = [pcr.refactor(x, pcr.Scheme(interp="level", degree="cubic", decomp_axis=2 if x.dim() == 3 else -1))
          for x in xs[:2]]
    hs += [pcr.refactor(x, pcr.Scheme(mode="psnr", interp="region", degree="cubic")) for x in xs[2:]]
    reqs = []
    for _ in range(40):
        f = rng.randrange(len(hs))
        if rng.random() < 0.5:
            t = pcr.Target("rel", 10.0 ** -rng.randint(2, 5))
        else:
            t = pcr.Target("psnr", float(rng.choice([40, 60, 80, 100])))
        box = None
        if rng.random() < 0.3:
            box = tuple((0, s // 2) for s in hs[f].shape)
        reqs.append((f, t, box))
    want = []
    for f, t, box in reqs:
        out, _ = hs[f].retrieve(hs[f].plan(t, allow_unsat=True))
        want.append(out[tuple(slice(lo, hi) for lo, hi in box)] if box else out)
    torch.cuda.synchronize()
    budget = 3 * max(h.retrieve_scratch_bytes() + h.out_bytes for h in hs)
    srv = Server(hs, mem_budget=budget, max_batch=4, streams=2, start=False)
    live = [srv.submit(f, t, box) for f, t, box in reqs[:8]]   # queued before the worker runs
    srv.start()
    for f, t, box in reqs[8:]:
        live.append(srv.submit(f, t, box))
        time.sleep(rng.random() * 0.002)
    got = [r.future.result(timeout=60) for r in live]
    srv.close()
    for g, w in zip(got, want):
        assert torch.equal(g, w)
    assert srv.batches < len(reqs)          # some groups held several requests
    assert all(r.latency > 0 for r in live)
    assert srv.mem_in_use == 0


def test_served_results_match_the_oracle():
    import oracle
    import paper_2609_04573_b300 as pcr
    from paper_2609_04573_b300.serve import Server
    from _compare import oracle_scheme
    Xs = _fields()[:3]
    schs = [pcr.Scheme(interp="level", degree="cubic", decomp_axis=2 if X.ndim == 3 else -1) for X in Xs[:2]]
    schs.append(pcr.Scheme(mode="psnr", interp="region", degree="cubic", decomp_axis=0))
    hs = [pcr.refactor(torch.from_numpy(X).cuda(), s) for X, s in zip(Xs, schs)]
    hos = [oracle.refactor(X, oracle_scheme(s, X.ndim)) for X, s in zip(Xs, schs)]
    reqs = [(0, pcr.Target("rel", 1e-3), None), (1, pcr.Target("psnr", 70.0), None),
            (2, pcr.Target("psnr", 90.0), ((3, 17), (5, 30), (10, 65))),
            (0, pcr.Target("rel", 1e-5), ((0, 18), (20, 44), (33, 70))), (2, pcr.Target("rel", 1e-4), None),
            (1, pcr.Target("rel", 1e-2), ((40, 96), (0, 64)))]
    budget = 3 * max(h.retrieve_scratch_bytes() + h.out_bytes for h in hs)
    srv = Server(hs, mem_budget=budget, max_batch=4, streams=2, start=False)
    live = [srv.submit(f, t, box) for f, t, box in reqs]
    srv.start()
    got = [r.future.result(timeout=60) for r in live]
    srv.close()
    for (f, t, box), g in zip(reqs, got):
        pl_or = oracle.plan(hos[f], oracle.Target(t.kind, t.value))
        x_or, _ = oracle.retrieve(hos[f], pl_or)
        if box:
            x_or = x_or[tuple(slice(lo, hi) for lo, hi in box)]
        assert np.array_equal(g.cpu().numpy(), x_or), (f, t, box)
