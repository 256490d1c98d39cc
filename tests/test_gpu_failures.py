"""Failure paths, injected on the host (no GPU fault is ever provoked).

* Out of device memory: a pcr_allocator that returns NULL at its k-th call,
  for every k below the number of calls a successful run makes, in the
  single, batched and graph-captured refactors and in a retrieval.  Every
  such call reports PCR_ERR_OOM with a message, hands back every block it
  did obtain (once the call returns, the allocator's live blocks are those
  it held before), and the library stays usable: the same call with a
  working allocator afterwards gives the handle / field of a run that never
  failed.
* Cancellation: served requests cancelled before the worker starts never
  run (their futures stay cancelled, no memory stays charged), the others
  complete and equal single retrievals.
"""
import random

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


class FaultyAllocator:
    """A pcr_allocator over torch's caching allocator that returns NULL at
    call number `fail_at` (None: never) and tracks the blocks it handed out."""

    def __init__(self, pcr, fail_at=None):
        self.calls = 0
        self.fail_at = fail_at
        self.live = set()
        self.stray_frees = 0   # frees of blocks this allocator never handed out

        def alloc(ctx, nbytes, stream):
            k = self.calls
            self.calls += 1
            if self.fail_at is not None and k == self.fail_at:
                return None
            p = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)
            self.live.add(p)
            return p

        def free(ctx, ptr, stream):
            if ptr:
                if ptr not in self.live:
                    self.stray_frees += 1
                    return
                self.live.discard(ptr)
                torch.cuda.caching_allocator_delete(ptr)

        self._cbs = (pcr._ALLOC_FN(alloc), pcr._FREE_FN(free))
        self.c = pcr._Allocator(None, *self._cbs)


def _same(ha, hb):
    assert ha.nstreams == hb.nstreams
    assert ha.field_stats() == hb.field_stats()
    for i in range(ha.nstreams):
        for u, v in zip(ha.stream_copy(i), hb.stream_copy(i)):
            assert np.array_equal(u, v), i
        assert ha.tables(i) == hb.tables(i)


def _expect_oom(pcr, fn):
    with pytest.raises(pcr.PcrError) as ei:
        fn()
    assert ei.value.status == pcr.ERR_OOM and "allocation failed" in str(ei.value), str(ei.value)


def _sweep(pcr, run, check):
    """run(allocator) with a failure at every call of a successful run."""
    ok = FaultyAllocator(pcr)
    ref = run(ok)
    n = ok.calls
    assert n >= 1
    for k in range(n):
        a = FaultyAllocator(pcr, fail_at=k)
        _expect_oom(pcr, lambda: run(a))
        torch.cuda.synchronize()
        assert not a.live and not a.stray_frees, (k, len(a.live), a.stray_frees)
    again = FaultyAllocator(pcr)
    check(ref, run(again))
    return n


def _fields():
    from synth import grf
    return [grf((21, 34, 48), 901, np.float32), grf((40, 66), 902, np.float32), grf((18, 20, 24), 903, np.float64)]


def test_refactor_out_of_memory_at_every_allocation():
    import paper_2609_04573_b300 as pcr
    X = _fields()[0]
    x = torch.from_numpy(X).cuda()
    sch = pcr.Scheme(interp="level", degree="cubic", decomp_axis=2)
    n = _sweep(pcr, lambda a: pcr.refactor(x, sch, allocator=a), _same)
    assert n >= 2   # the handle's block and the call's scratch


def test_batched_refactor_out_of_memory_at_every_allocation():
    import paper_2609_04573_b300 as pcr
    xs = [torch.from_numpy(X).cuda() for X in _fields()]
    schs = [pcr.Scheme(interp="level", degree="cubic", decomp_axis=2 if x.dim() == 3 else -1) for x in xs]

    def check(ra, rb):
        for ha, hb in zip(ra, rb):
            _same(ha, hb)
    n = _sweep(pcr, lambda a: pcr.refactor_batch(xs, schs, allocator=a), check)
    assert n >= len(xs) + 1


def test_graph_creation_out_of_memory_at_every_allocation():
    import paper_2609_04573_b300 as pcr
    xs = [torch.from_numpy(X).cuda() for X in _fields()[:2]]
    schs = [pcr.Scheme(interp="level", degree="cubic", decomp_axis=2 if x.dim() == 3 else -1) for x in xs]

    def check(ga, gb):
        gb.run()
        for ha, hb in zip(ga.handles, gb.handles):
            _same(ha, hb)
    n = _sweep(pcr, lambda a: pcr.RefactorGraph(xs, schs, allocator=a), check)
    assert n >= 3


def test_retrieval_out_of_memory_at_every_allocation():
    import paper_2609_04573_b300 as pcr
    X = _fields()[0]
    x = torch.from_numpy(X).cuda()
    sch = pcr.Scheme(interp="level", degree="cubic", decomp_axis=2)
    a = FaultyAllocator(pcr)
    h = pcr.refactor(x, sch, allocator=a)
    plan = h.plan(pcr.Target("rel", 1e-4))
    want, _ = h.retrieve(plan)
    torch.cuda.synchronize()
    held = set(a.live)           # the handle's own block
    start = a.calls
    h.retrieve(plan)
    torch.cuda.synchronize()
    n = a.calls - start
    assert n >= 1
    for k in range(n):
        a.fail_at = a.calls + k
        _expect_oom(pcr, lambda: h.retrieve(plan))
        torch.cuda.synchronize()
        assert a.live == held and not a.stray_frees, k
    a.fail_at = None
    got, _ = h.retrieve(plan)
    assert torch.equal(got, want)


def test_cancelled_requests_never_run():
    import paper_2609_04573_b300 as pcr
    from paper_2609_04573_b300.serve import Server
    rng = random.Random(17)
    Xs = _fields()[:2]
    hs = [pcr.refactor(torch.from_numpy(X).cuda(), pcr.Scheme(interp="level", degree="cubic",
                                                                decomp_axis=2 if X.ndim == 3 else -1))
          for X in Xs]
    reqs = [(rng.randrange(2), pcr.Target("rel", 10.0 ** -rng.randint(2, 5))) for _ in range(12)]
    srv = Server(hs, mem_budget=1 << 34, max_batch=4, streams=2, start=False)
    live = [srv.submit(f, t) for f, t in reqs]
    drop = set(range(0, 12, 3))
    for i in drop:
        assert live[i].cancel()
    srv.start()
    for i, r in enumerate(live):
        if i in drop:
            continue
        got = r.future.result(timeout=60)
        f, t = reqs[i]
        want, _ = hs[f].retrieve(hs[f].plan(t, allow_unsat=True))
        assert torch.equal(got, want)
    srv.close()
    assert srv.cancelled == len(drop)
    assert all(live[i].future.cancelled() for i in drop)
    assert srv.mem_in_use == 0
