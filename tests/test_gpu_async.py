"""Asynchronous refactor (pcr_refactor_begin / pcr_refactor_end): the handle
equals pcr_refactor's, with several jobs in flight on one stream and with
the pipelined loop (the next field's refactor enqueued before the current
one is planned and retrieved)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _same(ha, hb):
    assert ha.nstreams == hb.nstreams
    assert ha.field_stats() == hb.field_stats()
    for i in range(hb.nstreams):
        for u, v in zip(ha.stream_copy(i), hb.stream_copy(i)):
            assert np.array_equal(u, v), i
        assert ha.tables(i) == hb.tables(i)


def _fields():
    from synth import grf
    return [torch.from_numpy(grf((36, 44, 70), 51 + k, np.float32)).cuda() for k in range(3)]


def test_async_equals_sync():
    import paper_2609_04573_b300 as pcr
    xs = _fields()
    schemes = [pcr.Scheme(interp="level", degree="cubic", decomp_axis=2),
               pcr.Scheme(mode="psnr", interp="region", degree="cubic"),
               pcr.Scheme(interp="level", degree="linear")]
    jobs = [pcr.refactor_async(x, s) for x, s in zip(xs, schemes)]   # all in flight
    hs = [j.result() for j in jobs]
    for x, s, h in zip(xs, schemes, hs):
        _same(h, pcr.refactor(x, s))


def test_pipelined_loop_retrievals_equal_sync():
    import paper_2609_04573_b300 as pcr
    xs = _fields()
    sch = pcr.Scheme(interp="level", degree="cubic", decomp_axis=2)
    tg = pcr.Target("rel", 1e-4)
    want = []
    for x in xs:
        h = pcr.refactor(x, sch)
        want.append(h.retrieve(h.plan(tg))[0].clone())
    torch.cuda.synchronize()
    got = []
    job = pcr.refactor_async(xs[0], sch)
    for k in range(len(xs)):
        nxt = pcr.refactor_async(xs[k + 1], sch) if k + 1 < len(xs) else None
        h = job.result()
        out, _ = h.retrieve(h.plan(tg))
        got.append(out)
        job = nxt
    torch.cuda.synchronize()
    for g, w in zip(got, want):
        assert torch.equal(g, w)


def test_abandoned_job_and_consumed_job():
    import paper_2609_04573_b300 as pcr
    x = _fields()[0]
    j = pcr.refactor_async(x, pcr.Scheme())
    del j                                     # waits for its work, releases everything
    j = pcr.refactor_async(x, pcr.Scheme())
    j.result()
    with pytest.raises(RuntimeError):
        j.result()
    torch.cuda.synchronize()
