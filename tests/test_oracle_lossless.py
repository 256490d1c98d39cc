"""Lossless coding of plane words (oracle.lossless): pins.

* A hand-coded example: ones at bits 0 and 3 of a 4096-bit segment give
  m = 2, k = 10 (the largest k with 2 * 2^k <= 4094), gaps 0 and 2, and the
  22-bit code 0 0000000000 | 0 0000000010, whose only one sits at bit 20 of
  the first payload word; header 1 | 10 << 2 | 2 << 6 | 1 << 19 (one
  payload word).
* Round trip on sparse, dense and ragged segments of every density.
* The Rice code length equals the sum over gaps of (g >> k) + 1 + k,
  counted here from the gaps directly.
* Dense random words fall back to RAW with the words themselves.
* The k rule: m 2^k <= n - m < m 2^(k+1) (or k = 15, or k = 0 when n - m < m).
* Zero planes of a stream cost nothing; packed bytes add up per segment.
"""
import numpy as np
import pytest

from oracle import lossless as ll


def test_hand_coded_example():
    w = np.zeros(128, np.uint32)
    w[0] = 0b1001
    h, p = ll.encode_segment(w)
    assert h == 1 | (10 << 2) | (2 << 6) | (1 << 19)
    assert p.size == 1 and int(p[0]) == 1 << 20
    assert np.array_equal(ll.decode(h, p, 128), w)


@pytest.mark.parametrize("density", [0.0, 1 / 4096, 1 / 512, 1 / 64, 1 / 16, 1 / 4, 0.5, 0.9, 1.0])
@pytest.mark.parametrize("nwords", [128, 37, 1])
def test_round_trip(density, nwords):
    rng = np.random.default_rng(int(density * 1e6) + nwords)
    bits = rng.random(nwords * 32) < density
    w = (bits.reshape(-1, 32).astype(np.uint64) << np.arange(32, dtype=np.uint64)).sum(1).astype(np.uint32)
    h, p = ll.encode_segment(w)
    assert np.array_equal(ll.decode(h, p, nwords), w)
    m = int(bits.sum())
    assert (h >> 6) & 0x1FFF == m if m else h == ll.ZERO
    assert h >> 19 == p.size
    if h & 3 == ll.RICE:
        k = (h >> 2) & 15
        pos = np.flatnonzero(bits)
        gaps = np.diff(np.concatenate([[-1], pos])) - 1
        nbits = int(sum((int(g) >> k) + 1 + k for g in gaps))
        assert nbits < nwords * 32 and p.size == -(-nbits // 32)
    if h & 3 == ll.RAW:
        assert np.array_equal(p, w)


def test_dense_words_are_stored_raw():
    rng = np.random.default_rng(3)
    w = rng.integers(0, 2 ** 32, 128, dtype=np.uint64).astype(np.uint32)
    h, p = ll.encode_segment(w)
    assert h & 3 == ll.RAW and np.array_equal(p, w)


@pytest.mark.parametrize("n", [32, 4096])
def test_k_rule(n):
    for m in range(1, n + 1, max(1, n // 97)):
        k = ll.rice_k(m, n)
        if n - m < m:
            assert k == 0
        else:
            assert m << k <= n - m
            assert k == 15 or (m << (k + 1)) > n - m


def test_stream_packing_sizes():
    rng = np.random.default_rng(9)
    B, words = 6, 300          # 3 segments, the last ragged
    planes = np.zeros((B, words), np.uint32)
    for k in (1, 3, 4):
        bits = rng.random(words * 32) < [0, 0.002, 0, 0.05, 0.5, 0][k]
        planes[k] = (bits.reshape(-1, 32).astype(np.uint64) << np.arange(32, dtype=np.uint64)).sum(1)
    nz = [int(np.count_nonzero(planes[k])) for k in range(B)]
    heads, pays, sizes = ll.pack_stream(planes, nz)
    for k in range(B):
        if not nz[k]:
            assert sizes[k] == 0
            continue
        tot = 0
        for g in range(3):
            n = min(128, words - 128 * g)
            assert np.array_equal(ll.decode(int(heads[k, g]), pays[(k, g)], n), planes[k, 128 * g:128 * g + n])
            tot += 4 + 4 * pays[(k, g)].size
        assert sizes[k] == tot
    t = ll.packed_bytes_table(sizes)
    assert t[0] == 0 and t[-1] == sizes.sum() and np.all(np.diff(t) >= 0)
    assert sizes[1] < 4 * words and sizes[3] < 4 * words     # sparse planes shrink
