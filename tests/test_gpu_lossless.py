"""Lossless coding of plane words on the GPU against the oracle.

* One segment at a time (pcr_debug_pack): header and payload words equal
  oracle.lossless.encode_segment's for every density, ragged lengths and
  the all-zero and all-one extremes.
* Whole handles: the packed byte tables equal the oracle's (each stream's
  planes coded per segment with oracle.lossless.pack_stream, plus the sign
  words), for both encodings.
* Containers with coded planes: pcr_deserialize restores the handle (same
  planes, tables and retrieved field) and the container is smaller than
  the raw one; a flipped byte is refused.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _words(bits):
    return (bits.reshape(-1, 32).astype(np.uint64) << np.arange(32, dtype=np.uint64)).sum(1).astype(np.uint32)


@pytest.mark.parametrize("density", [0.0, 1 / 4096, 1 / 700, 1 / 64, 1 / 9, 1 / 3, 0.5, 1.0])
@pytest.mark.parametrize("nwords", [128, 77, 1])
def test_segment_code_equals_the_oracle(density, nwords):
    import paper_2609_04573_b300 as pcr
    from oracle import lossless as ll
    rng = np.random.default_rng(int(density * 1e5) + 7 * nwords)
    w = _words(rng.random(nwords * 32) < density)
    d = torch.from_numpy(w.view(np.int32)).cuda()
    hdr = C.c_uint32()
    pay = (C.c_uint32 * 128)()
    npay = C.c_int()
    pcr._check(pcr._lib.pcr_debug_pack(C.c_void_p(d.data_ptr()), nwords, C.byref(hdr), pay, C.byref(npay)))
    h_or, p_or = ll.encode_segment(w)
    assert hdr.value == h_or
    assert npay.value == p_or.size and list(pay[:npay.value]) == [int(v) for v in p_or]


@pytest.mark.parametrize("sch_kw", [dict(mode="eb", interp="level", degree="cubic", decomp_axis=2),
                                    dict(mode="psnr", interp="region", degree="cubic", decomp_axis=0)])
def test_packed_tables_equal_the_oracle(sch_kw):
    import oracle
    import paper_2609_04573_b300 as pcr
    from oracle import lossless as ll
    from synth import grf
    from _compare import oracle_scheme
    X = grf((33, 40, 70), 611, np.float32)
    sch = pcr.Scheme(**sch_kw)
    h = pcr.refactor(torch.from_numpy(X).cuda(), sch)
    h_or = oracle.refactor(X, oracle_scheme(sch, 3))
    got = h.packed_tables()
    for i, s in enumerate(h_or["streams"]):
        enc, raw = s["enc"], s["tab"]["bytes"]
        words = enc["planes"].shape[1]
        _, _, sizes = ll.pack_stream(enc["planes"], enc["plane_nz"])
        # the raw table with each plane's raw words replaced by its coded size
        want, swap = [0], 0
        for k in range(len(sizes)):
            swap += int(sizes[k]) - (4 * words if enc["plane_nz"][k] else 0)
            want.append(int(raw[k + 1]) + swap)
        assert got[i] == want, i


def test_packed_container_round_trip_and_corruption():
    import paper_2609_04573_b300 as pcr
    from synth import grf
    X = grf((40, 48, 64), 612, np.float32)
    h = pcr.refactor(torch.from_numpy(X).cuda(), pcr.Scheme(interp="level", degree="cubic", decomp_axis=2))
    raw, packed = h.serialize(), h.serialize_packed()
    assert len(packed) < len(raw)
    h2 = pcr.deserialize(packed)
    for i in range(h.nstreams):
        for u, v in zip(h.stream_copy(i), h2.stream_copy(i)):
            assert np.array_equal(u, v), i
        assert h.tables(i) == h2.tables(i)
    for t in (pcr.Target("rel", 1e-2), pcr.Target("rel", 1e-5), pcr.Target("psnr", 70.0)):
        a, _ = h.retrieve(t)
        b, _ = h2.retrieve(t)
        assert torch.equal(a, b)
    assert h2.packed_tables() == h.packed_tables()
    bad = bytearray(packed)
    bad[len(bad) // 2] ^= 0x10
    with pytest.raises(pcr.PcrError):
        pcr.deserialize(bytes(bad))
