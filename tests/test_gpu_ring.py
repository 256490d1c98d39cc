"""Level-0 retrieval's coarse ring at the plane edges, CUDA path vs oracle.

The marching retrieval takes the coarse points (the 2-grid) from the
fixed-point copy: by one tensor copy per even plane where the 2-grid's rows
are 16-byte multiples, by register loads otherwise, and by register loads
for each plane chunk's first three ring planes.  These cases put the last
ring plane of a chunk on, just inside and just past the field's end (plane
counts 5 .. 19, even and odd, one chunk and several), in FP32 and FP64, per
level and per region.  Every retrieved value must equal the oracle's
(Alg. 2), and no bounded device wait may give up.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import oracle  # noqa: E402
from oracle import Target as OTarget  # noqa: E402
from synth import grf  # noqa: E402

from _compare import oracle_scheme  # noqa: E402

SCHEMES = [
    dict(interp="level", degree="cubic", decomp_axis=2),
    dict(interp="region", degree="cubic"),
    dict(interp="level", degree="linear"),
]

CASES = [
    # FP32: 2-grid rows of m2 / 2 words, always 16-byte multiples (m2 % 4 == 0)
    ((5, 24, 64), np.float32),
    ((6, 20, 36), np.float32),
    ((9, 18, 40), np.float32),
    ((10, 34, 68), np.float32),
    ((19, 16, 128), np.float32),
    # FP64: 20-word rows take the tensor copy, 21-word rows the register loads
    ((12, 20, 40), np.float64),
    ((11, 22, 42), np.float64),
]


@pytest.mark.parametrize("si", range(len(SCHEMES)))
@pytest.mark.parametrize("ci", range(len(CASES)))
def test_ring_edges(ci, si):
    import paper_2609_04573_b300 as pcr
    shape, dtype = CASES[ci]
    X = grf(shape, 700 + 10 * ci + si, dtype)
    sch = pcr.Scheme(**SCHEMES[si])
    h_or = oracle.refactor(X, oracle_scheme(sch, X.ndim))
    h = pcr.refactor(torch.from_numpy(X).cuda(), sch)
    torch.cuda.synchronize()
    for t in (OTarget("rel", 1e-2), OTarget("rel", 1e-5)):
        pl_or = oracle.plan(h_or, t)
        pl = h.plan(pcr.Target(t.kind, t.value), allow_unsat=True)
        assert pl.planes == pl_or["b"], t
        x_or, _ = oracle.retrieve(h_or, pl_or)
        out, _ = h.retrieve(pl)
        assert np.array_equal(out.cpu().numpy(), x_or), f"{shape} {SCHEMES[si]} {t}"
    assert pcr.device_status() == 0
