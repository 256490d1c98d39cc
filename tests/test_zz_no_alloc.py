"""pcr_retrieve_static: retrieval that allocates no device memory.

Some callers cannot allocate device memory: applications whose own pool or
arena owns the whole GPU, hosts that forbid libraries to allocate for them,
and latency-bound loops where cudaMalloc / cudaFree would synchronise the
device.  These tests call the allocation-free entry point through the C ABI
and check that it returns exactly what pcr_retrieve returns, on two calls in a
row (the second reuses the shared array after the first), for FP32 and FP64
handles, for a handle whose retrieval work list is kept on the device and for
one from pcr_deserialize (work list uploaded by every call), while neither
the handle's allocator nor torch's caching allocator sees a single
allocation.  A field too large for the fixed array is refused with a clear
error.  The file name sorts last so that a stop-at-first-failure run has
already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


class CountingAllocator:
    """A pcr_allocator that counts its calls and takes memory from torch."""

    def __init__(self, pcr):
        self.allocs = 0
        self.frees = 0

        def alloc(ctx, nbytes, stream):
            self.allocs += 1
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)

        def free(ctx, ptr, stream):
            self.frees += 1
            if ptr:
                torch.cuda.caching_allocator_delete(ptr)

        self._cbs = (pcr._ALLOC_FN(alloc), pcr._FREE_FN(free))
        self.c = pcr._Allocator(None, *self._cbs)


def _refactor(pcr, x, scheme, allocator):
    dims = (C.c_int64 * x.dim())(*x.shape)
    out = C.c_void_p()
    st = pcr._lib.pcr_refactor(C.c_void_p(x.data_ptr()), x.dim(), dims, pcr._DT[x.dtype],
                               C.byref(scheme.c(x.dim())), C.byref(allocator.c),
                               C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(out))
    pcr._check(st)
    return pcr.Handle(out.value, x.shape, x.dtype, x.device)


def _deserialize(pcr, data, allocator):
    buf = C.create_string_buffer(data, len(data))
    out = C.c_void_p()
    pcr._check(pcr._lib.pcr_deserialize(buf, len(data), C.byref(allocator.c),
                                        C.c_void_p(torch.cuda.current_stream().cuda_stream), C.byref(out)))
    return out.value


def _torch_allocs():
    return torch.cuda.memory_stats().get("allocation.all.allocated", 0)


def _check_static(pcr, h, allocator, targets):
    for tgt in targets:
        plan = h.plan(tgt)
        want, _ = h.retrieve(plan)
        outs = [torch.full_like(want, float("nan")) for _ in range(2)]
        torch.cuda.synchronize()
        n_lib, n_torch = allocator.allocs, _torch_allocs()
        for out in outs:             # two calls in a row on the shared array
            st = pcr._lib.pcr_retrieve_static(h._p, C.byref(plan._c), C.c_void_p(out.data_ptr()),
                                              C.c_void_p(torch.cuda.current_stream().cuda_stream))
            pcr._check(st)
        torch.cuda.synchronize()
        assert allocator.allocs == n_lib, "the handle's allocator was called"
        assert _torch_allocs() == n_torch, "torch's allocator was called"
        for out in outs:
            assert torch.equal(out, want)


def test_static_retrieve_matches_retrieve_twice():
    import paper_2609_04573_b300 as pcr
    from synth import grf
    X = grf((40, 52, 70), 31, np.float32)
    al = CountingAllocator(pcr)
    for sch in (pcr.Scheme(interp="level", degree="cubic", decomp_axis=2),
                pcr.Scheme(mode="psnr", interp="region", degree="cubic")):
        h = _refactor(pcr, torch.from_numpy(X).cuda(), sch, al)
        _check_static(pcr, h, al, (pcr.Target("rel", 1e-3), pcr.Target("psnr", 70.0)))


def test_static_retrieve_fp64_and_deserialized_handle():
    import paper_2609_04573_b300 as pcr
    from synth import grf
    X = grf((36, 44, 50), 33, np.float64)
    al = CountingAllocator(pcr)
    h = _refactor(pcr, torch.from_numpy(X).cuda(), pcr.Scheme(interp="level", degree="cubic", decomp_axis=1), al)
    targets = (pcr.Target("rel", 1e-6), pcr.Target("rel", 1e-9))
    _check_static(pcr, h, al, targets)
    # a deserialized handle keeps no retrieval work list: every call uploads it
    ptr = _deserialize(pcr, h.serialize(), al)
    h2 = pcr.Handle(ptr, h.shape, h.dtype, h.device)
    _check_static(pcr, h2, al, targets)


def test_static_retrieve_refuses_oversized_fields():
    import paper_2609_04573_b300 as pcr
    from synth import grf
    X = grf((160, 160, 160), 32, np.float32)
    h = pcr.refactor(torch.from_numpy(X).cuda(), pcr.Scheme(interp="level", degree="cubic", decomp_axis=2))
    plan = h.plan(pcr.Target("rel", 1e-2))
    out = torch.zeros_like(torch.from_numpy(X).cuda())
    with pytest.raises(pcr.PcrError) as ei:
        h.retrieve_static(plan, out)
    assert "static array holds" in str(ei.value)
