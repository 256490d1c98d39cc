"""pcr_retrieve_static: retrieval with no device allocation.

Some callers cannot allocate device memory (work enqueued during CUDA graph
capture, applications whose own arena owns the GPU, latency-bound loops where
cudaMalloc would synchronise the device).  This checks, through the C ABI,
that the allocation-free entry point returns exactly what pcr_retrieve
returns, on two calls in a row (the second reuses the shared array after the
first), and that a field too large for the fixed array is refused with a
clear error.  The file name sorts last so a stop-at-first-failure run has
already run every other test.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_static_retrieve_matches_retrieve_twice():
    import paper_2609_04573_b300 as pcr
    from synth import grf
    X = grf((40, 52, 70), 31, np.float32)
    for sch in (pcr.Scheme(interp="level", degree="cubic", decomp_axis=2),
                pcr.Scheme(mode="psnr", interp="region", degree="cubic")):
        h = pcr.refactor(torch.from_numpy(X).cuda(), sch)
        for tgt in (pcr.Target("rel", 1e-3), pcr.Target("psnr", 70.0)):
            plan = h.plan(tgt)
            want, _ = h.retrieve(plan)
            for _ in range(2):
                out = torch.full_like(want, float("nan"))
                h.retrieve_static(plan, out)
                torch.cuda.synchronize()
                assert torch.equal(out, want)


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
