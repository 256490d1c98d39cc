"""The one-call boundary: pcr_retrieve(handle, target) -> field with its
retrieval info, batched retrieval by target, the tables of every stream and
the explicit scheme mode, each compared with the oracle (Sec. III-A problem
statement: retrieve the smallest stream prefix meeting a target)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _setup(sch, shape=(34, 41, 66), seed=51):
    import oracle
    import paper_2609_04573_b300 as pcr
    from synth import grf
    from _compare import oracle_scheme
    X = grf(shape, seed, np.float32)
    h = pcr.refactor(torch.from_numpy(X).cuda(), sch)
    h_or = oracle.refactor(X, oracle_scheme(sch, X.ndim))
    return pcr, oracle, X, h, h_or


def test_one_call_retrieve_matches_oracle():
    import paper_2609_04573_b300 as pcr
    pcr_, oracle, X, h, h_or = _setup(pcr.Scheme(interp="level", degree="cubic", decomp_axis=2))
    for kind, v in (("rel", 1e-2), ("rel", 1e-5), ("psnr", 60.0)):
        out, info = h.retrieve(pcr.Target(kind, v), gpu_time=True)
        pl_or = oracle.plan(h_or, oracle.Target(kind, v))
        assert info.planes == pl_or["b"] and info.bytes == pl_or["bytes"] and info.satisfied
        assert info.bound == pl_or["bound"]
        assert info.bits_per_value == 8.0 * pl_or["bytes"] / X.size
        assert info.gpu_ms > 0 and info.plan_ms >= 0 and info.enqueue_ms >= 0
        x_or, _ = oracle.retrieve(h_or, pl_or)
        assert np.array_equal(out.cpu().numpy(), x_or)


def test_one_call_box_target_is_the_crop():
    import paper_2609_04573_b300 as pcr
    pcr_, oracle, X, h, h_or = _setup(pcr.Scheme(interp="region", degree="cubic", decomp_axis=0))
    box = ((5, 29), (0, 17), (33, 66))
    full, info_f = h.retrieve(pcr.Target("rel", 1e-4))
    part, info_b = h.retrieve(pcr.Target("rel", 1e-4, box=box))
    assert info_b.planes == info_f.planes
    assert torch.equal(part, full[5:29, 0:17, 33:66])
    pl_or = oracle.plan(h_or, oracle.Target("rel", 1e-4))
    x_or, _ = oracle.retrieve(h_or, pl_or)
    assert np.array_equal(part.cpu().numpy(), x_or[5:29, 0:17, 33:66])


def test_batch_by_target_equals_single_calls():
    import paper_2609_04573_b300 as pcr
    from synth import grf
    xs = [torch.from_numpy(grf(s, 60 + i, np.float32)).cuda()
          for i, s in enumerate([(20, 30, 40), (33, 17, 65), (1, 70, 90)])]
    xs[2] = xs[2][0].contiguous()
    hs = [pcr.refactor(x, pcr.Scheme(interp="level", degree="cubic", decomp_axis=2 if x.dim() == 3 else -1))
          for x in xs]
    targets = [pcr.Target("rel", 1e-3), pcr.Target("psnr", 80.0), pcr.Target("abs", 1e-4)]
    outs = [torch.empty_like(x) for x in xs]
    infos = pcr.retrieve_batch_targets(hs, targets, outs)
    for h, t, o, inf in zip(hs, targets, outs, infos):
        want, wi = h.retrieve(t)
        assert inf.planes == wi.planes and inf.bytes == wi.bytes
        assert torch.equal(o, want)


def test_get_tables_equal_oracle_tables():
    import paper_2609_04573_b300 as pcr
    pcr_, oracle, X, h, h_or = _setup(pcr.Scheme(mode="psnr", interp="region", degree="cubic", decomp_axis=2))
    t = h.get_tables()
    assert len(t["exponent"]) == len(h_or["streams"])
    for i, s in enumerate(h_or["streams"]):
        tab = s["tab"]
        assert list(t["maxerr"][i]) == list(tab["maxerr"])
        assert list(t["sq"][i]) == list(tab["sq"])
        assert [int(b) for b in t["bytes"][i]] == list(tab["bytes"])
        q = s["enc"]["quant"]
        assert t["exponent"][i] == (q["e"] if s["is_int"] else q["E"])


def test_explicit_mode_serves_both_target_kinds():
    import paper_2609_04573_b300 as pcr
    from _compare import compare_streams
    pcr_, oracle, X, h, h_or = _setup(pcr.Scheme(mode="explicit", interp="level", degree="cubic",
                                                 decomp_axis=1))
    compare_streams(h, h_or)
    for kind, v in (("rel", 1e-4), ("psnr", 90.0)):
        out, info = h.retrieve(pcr.Target(kind, v))
        pl_or = oracle.plan(h_or, oracle.Target(kind, v))
        assert info.planes == pl_or["b"]
        x_or, _ = oracle.retrieve(h_or, pl_or)
        assert np.array_equal(out.cpu().numpy(), x_or)


def test_unsatisfiable_target_fills_info_and_enqueues_nothing():
    import ctypes as C
    import paper_2609_04573_b300 as pcr
    pcr_, oracle, X, h, h_or = _setup(pcr.Scheme(interp="level", degree="cubic"))
    out = torch.full(X.shape, 7.0, device="cuda")
    info = pcr._Info()
    st = pcr._lib.pcr_retrieve(h._p, C.byref(pcr.Target("rel", 1e-9).c()), C.c_void_p(out.data_ptr()),
                               C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(info))
    torch.cuda.synchronize()
    assert st == pcr.ERR_UNSAT and info.satisfied == 0 and info.bound > 0
    assert info.nstreams == h.nstreams and all(info.planes[i] == 32 for i in range(h.nstreams))
    assert bool((out == 7.0).all())
