"""Box retrieval (pcr_retrieve_box): the box of a field retrieved alone is,
value for value, the same box of the whole-field retrieval with the same
plan -- boxes at corners, edges and inside, odd and even origins, one point
wide and the whole field; per-level cubic with decomposition (the
plane-marching and block-recompose launches restricted to the box), per-level
linear, per-region cubic, FP64, 2-D, and a shape whose level 0 runs the
general tile kernel."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CASES = [
    ((70, 66, 132), np.float32, dict(interp="level", degree="cubic", decomp_axis=2)),
    ((40, 52, 67), np.float32, dict(interp="level", degree="cubic", decomp_axis=2)),
    ((36, 33, 132), np.float32, dict(interp="level", degree="linear")),
    ((31, 36, 41), np.float32, dict(interp="region", degree="cubic", order=(2, 0, 1), decomp_axis=1)),
    ((36, 40, 68), np.float32, dict(interp="region", degree="cubic", decomp_axis=2)),
    ((34, 40, 66), np.float64, dict(interp="level", degree="cubic", decomp_axis=2)),
    ((130, 257), np.float32, dict(interp="level", degree="cubic")),
]


def _boxes(shape, rng):
    out = [tuple((0, n) for n in shape), tuple((0, 1) for _ in shape),
           tuple((n - 1, n) for n in shape), tuple((0, min(n, 17)) for n in shape),
           tuple((max(0, n - 23), n) for n in shape)]
    for _ in range(6):
        box = []
        for n in shape:
            a = int(rng.integers(0, n - 1))
            box.append((a, int(rng.integers(a + 1, min(n, a + 40) + 1))))
        out.append(tuple(box))
    return out


@pytest.mark.parametrize("ci", range(len(CASES)))
def test_box_equals_the_box_of_the_full_retrieval(ci):
    import paper_2609_04573_b300 as pcr
    from synth import grf
    shape, dtype, kw = CASES[ci]
    x = torch.from_numpy(grf(shape, 300 + ci, dtype)).cuda()
    h = pcr.refactor(x, pcr.Scheme(**kw))
    rng = np.random.default_rng(ci)
    for t in (pcr.Target("rel", 1e-2), pcr.Target("rel", 1e-5)):
        pl = h.plan(t, allow_unsat=True)
        full, _ = h.retrieve(pl)
        for box in _boxes(shape, rng):
            got, _ = h.retrieve_box(pl, box)
            want = full[tuple(slice(a, b) for a, b in box)]
            assert torch.equal(got, want), (box, t.value)
