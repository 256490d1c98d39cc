"""Lossless coding of plane words (oracle).  Test infrastructure only.

The paper follows bitplane encoding with lossless compression of the planes
(Sec. V opening) and its bitrates include it.  Reading (the paper does not
fix a coder): each (stream, plane, 4096-value segment) -- a string of 4096
bits, bit e of plane word j being value 32 j + e -- is coded on its own:

* m = number of ones.  m = 0: ZERO, nothing stored.
* else Rice coding of the zero runs before each one: with the ones at
  positions q_1 < .. < q_m and q_0 = -1, the gaps g_i = q_i - q_(i-1) - 1
  are written in order, each as (g >> k) one-bits, a zero-bit, then the k
  low bits of g, most significant first; the zeros after the last one are
  implied by m.  k is the largest integer with m 2^k <= 4096 - m (0 when
  4096 - m < m), at most 15.
* when that code is not shorter than the 4096 raw bits (or the segment is
  shorter than 4096 values and the code not shorter than its raw bits):
  RAW, the plane words themselves.

Stored per segment and plane: one header word (mode in bits 0-1: 0 ZERO,
1 RICE, 2 RAW; k in bits 2-5; m in bits 6-18; payload words in bits 19-27)
and the payload: RICE the code bits packed least significant bit first
into ceil(bits / 32) words, RAW the segment's plane words.  A plane with no nonzero word in the whole
stream is not stored (as in the raw byte tables); its packed size is 0.
Packed bytes of a plane: the sum over its segments of 4 (header) + 4 x
payload words.
"""
import numpy as np

SEG_BITS = 4096
ZERO, RICE, RAW = 0, 1, 2


def rice_k(m, nbits=SEG_BITS):
    k = 0
    while k < 15 and (m << (k + 1)) <= nbits - m:
        k += 1
    return k


def _bits_of(words):
    """Bit string (numpy bool array) of plane words, bit e of word j at 32 j + e."""
    w = np.asarray(words, dtype=np.uint32)
    return ((w[:, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(bool).ravel()


def _words_of(bits):
    b = np.asarray(bits, dtype=np.uint32).reshape(-1, 32)
    return (b << np.arange(32, dtype=np.uint32)).sum(axis=1).astype(np.uint32)


def encode_segment(words):
    """(header, payload words) of one plane of one segment."""
    words = np.asarray(words, dtype=np.uint32)
    bits = _bits_of(words)
    n = bits.size
    ones = np.flatnonzero(bits)
    m = int(ones.size)
    if m == 0:
        return ZERO, np.zeros(0, np.uint32)
    k = rice_k(m, n)
    code = []
    prev = -1
    for q in ones:
        g = int(q) - prev - 1
        code.extend([1] * (g >> k))
        code.append(0)
        code.extend((g >> (k - 1 - t)) & 1 for t in range(k))
        prev = int(q)
    if len(code) >= n:
        return RAW | (k << 2) | (m << 6) | (words.size << 19), words.copy()
    pad = (-len(code)) % 32
    payload = _words_of(np.array(code + [0] * pad, dtype=np.uint32))
    return RICE | (k << 2) | (m << 6) | (payload.size << 19), payload


def _decode_rice(bits, k, m, n):
    out = np.zeros(n, dtype=bool)
    t, prev = 0, -1
    for _ in range(m):
        q = 0
        while bits[t]:
            q += 1
            t += 1
        t += 1
        low = 0
        for _ in range(k):
            low = (low << 1) | int(bits[t])
            t += 1
        prev = prev + 1 + (q << k | low)
        out[prev] = True
    return out


def decode(header, payload, nwords):
    """Plane words of one segment from its header and payload."""
    mode, k, m = header & 3, (header >> 2) & 15, (header >> 6) & 0x1FFF
    if mode == ZERO:
        return np.zeros(nwords, np.uint32)
    if mode == RAW:
        return np.asarray(payload, np.uint32)[:nwords].copy()
    return _words_of(_decode_rice(_bits_of(payload), k, m, nwords * 32))


def pack_stream(planes, nz):
    """Packed form of one stream: planes [B][words] (words a multiple of
    32 values each), nz[k] = nonzero words of plane k.  Returns (headers
    [B][nseg], payloads {(k, seg): words}, packed bytes per plane [B])."""
    B, words = planes.shape
    nseg = -(-words // (SEG_BITS // 32))
    heads = np.zeros((B, nseg), np.uint32)
    pays = {}
    sizes = np.zeros(B, np.int64)
    for k in range(B):
        if not nz[k]:
            continue
        for g in range(nseg):
            w = planes[k, g * 128:(g + 1) * 128]
            h, p = encode_segment(w)
            heads[k, g] = h
            pays[(k, g)] = p
            sizes[k] += 4 + 4 * p.size
    return heads, pays, sizes


def packed_bytes_table(sizes):
    """Cumulative packed plane bytes: entry b = planes 0 .. b-1."""
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
