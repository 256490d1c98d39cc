"""Quantisation, bitplanes, sign sub-streams and error statistics (oracle).

Test infrastructure only.

Sec. V-C / PMGARD: a stream's coefficients are scaled by the exponent of
their maximum (stored as metadata), which gives a one-to-one map from the
number of retrieved bitplanes to an absolute error bound.  Encodings (Sec.
VI-A tuning table): generic sign-magnitude bitplanes (error-bound mode) and
negabinary digits with XOR between consecutive planes (PSNR mode).

Definitions used (B planes, plane k holds bit B-1-k, k = 0 is the MSB):
* float streams (level 0, field dtype): E = frexp exponent of m = max|v|
  (m = f 2^E, 0.5 <= f < 1).
  generic     q = floor(|v| 2^(B-E)),                  unit u = 2^(E-B)
  negabinary  s = trunc(v 2^(B-3-E)),                  unit u = 2^(E-B+3)
* fixed-point streams (levels >= 1, int64 value c in quanta h): e = bit
  length of max|c|; sh = max(0, e - B) (generic) or max(0, e - B + 3)
  (negabinary); q = |c| >> sh, s = sign(c) (|c| >> sh); u = 2^sh h.
* negabinary digits nb = (s + M) xor M mod 2^B, M = 0b1010..10; the stored
  plane k is nb-plane k xor nb-plane k-1 (k >= 1).  |s| < 2^(B-3) keeps the
  top digit zero, so every partial decode fits in int64.
* plane k, word w holds elements 32w .. 32w+31, bit j = element 32w+j.
* generic sign sub-streams: per segment of SEG_ELEMS elements and per plane
  k, the signs of the elements whose most significant set bit is plane k, in
  element order, packed like plane words (Sec. VI-C emits the sign with the
  first set bit; here those bits are gathered per plane).
"""
import numpy as np

from .geometry import SEG_ELEMS, WORD

GENERIC, NEGABINARY = "generic", "negabinary"


def nb_mask(B):
    return int("10" * (B // 2), 2)


def _udt(B):
    return np.uint32 if B == 32 else np.uint64


def quantize(vals, is_int, B, encoding):
    """Returns dict(q=unsigned B-bit codes (generic q / negabinary nb digits),
    neg=bool signs (generic), vmax, scale) for a 1-D stream."""
    ut = _udt(B)
    if is_int:
        a = np.abs(vals)
        vmax = int(a.max()) if a.size else 0
        e = vmax.bit_length()
        if encoding == GENERIC:
            sh = max(0, e - B)
            q = (a >> sh).astype(ut)
            return dict(q=q, neg=vals < 0, vmax=vmax, e=e, sh=sh)
        sh = max(0, e - (B - 3))
        s = np.sign(vals) * (a >> sh)
        return dict(q=_to_negabinary(s.astype(np.int64), B), vmax=vmax, e=e, sh=sh)
    a = np.abs(vals)
    vmax = float(a.max()) if a.size else 0.0
    E = int(np.frexp(vmax)[1]) if vmax > 0 else 0
    if encoding == GENERIC:
        q = np.floor(np.ldexp(a, B - E)).astype(ut)
        return dict(q=q, neg=vals < 0, vmax=vmax, E=E)
    s = np.trunc(np.ldexp(vals, B - 3 - E)).astype(np.int64)
    return dict(q=_to_negabinary(s, B), vmax=vmax, E=E)


def _to_negabinary(s, B):
    M = nb_mask(B)
    if B == 32:
        return (((s + M) & 0xFFFFFFFF) ^ M).astype(np.uint32)
    su = s.astype(np.uint64)  # two's complement wrap
    return (su + np.uint64(M)) ^ np.uint64(M)


def from_negabinary(nb, B):
    """Signed value of negabinary digits (int64)."""
    M = nb_mask(B)
    if B == 32:
        return (nb.astype(np.int64) ^ M) - M
    x = (nb ^ np.uint64(M)) - np.uint64(M)
    return x.view(np.int64)


def digit_planes(q, B):
    """Bool matrix [B, n]: row k = bit B-1-k."""
    ut = q.dtype.type
    return np.stack([((q >> ut(B - 1 - k)) & ut(1)).astype(bool) for k in range(B)])


def pack_words(bits):
    """Bool vector (length multiple of 32) -> uint32 words, LSB = first."""
    by = np.packbits(bits.astype(np.uint8), bitorder="little")
    return by.view("<u4").astype(np.uint32)


def unpack_words(words, n):
    by = np.asarray(words, dtype="<u4").view(np.uint8)
    return np.unpackbits(by, bitorder="little")[:n].astype(bool)


def msb_plane(q, B):
    """Plane index of the most significant set bit (B for q == 0)."""
    p = np.full(q.shape, B, dtype=np.int64)
    ut = q.dtype.type
    for k in range(B - 1, -1, -1):
        p[((q >> ut(B - 1 - k)) & ut(1)) == 1] = k
    return p


def encode(vals, is_int, B, encoding, want_pairs):
    """Full encoding of one stream (1-D padded values)."""
    n = vals.size
    assert n % WORD == 0
    qd = quantize(vals, is_int, B, encoding)
    digits = digit_planes(qd["q"], B)
    stored = digits.copy()
    if encoding == NEGABINARY:
        stored[1:] ^= digits[:-1]
    planes = np.stack([pack_words(stored[k]) for k in range(B)]) if n else \
        np.zeros((B, 0), np.uint32)
    out = dict(quant=qd, planes=planes,
               plane_nz=[int(np.count_nonzero(planes[k])) for k in range(B)])
    if encoding == GENERIC:
        p = msb_plane(qd["q"], B)
        nseg = -(-n // SEG_ELEMS)
        counts = np.zeros((nseg, B), dtype=np.int64)
        signs = []
        for g in range(nseg):
            lo, hi = g * SEG_ELEMS, min(n, (g + 1) * SEG_ELEMS)
            seg_words = []
            for k in range(B):
                sel = qd["neg"][lo:hi][p[lo:hi] == k]
                counts[g, k] = sel.size
                padded = np.zeros(-(-sel.size // WORD) * WORD, dtype=bool)
                padded[:sel.size] = sel
                seg_words.append(pack_words(padded))
            signs.append(seg_words)
        out["sign_counts"] = counts
        out["signs"] = signs
    if want_pairs:
        wd = [pack_words(digits[k]) for k in range(B)]
        C = np.zeros((B, B), dtype=object)
        for j in range(B):
            for jj in range(j, B):
                C[j, jj] = int(np.bitwise_count(wd[j] & wd[jj]).sum())
                C[jj, j] = C[j, jj]
        out["pairs"] = C
    return out


def decode(enc, n, is_int, B, encoding, b, dtype):
    """Values from the first b stored planes (zero-fill below)."""
    planes = enc["planes"]
    qd = enc["quant"]
    ut = _udt(B)
    digits = np.zeros((B, n), dtype=bool)
    for k in range(b):
        digits[k] = unpack_words(planes[k], n)
    if encoding == NEGABINARY:
        for k in range(1, b):
            digits[k] ^= digits[k - 1]
    code = np.zeros(n, dtype=ut)
    for k in range(b):
        code |= digits[k].astype(ut) << ut(B - 1 - k)
    if encoding == GENERIC:
        neg = np.zeros(n, dtype=bool)
        p = msb_plane(code, B)
        for g, seg in enumerate(enc["signs"]):
            lo, hi = g * SEG_ELEMS, min(n, (g + 1) * SEG_ELEMS)
            pg = p[lo:hi]
            for k in range(min(b, B)):
                idx = np.nonzero(pg == k)[0]
                if idx.size:
                    bits = unpack_words(seg[k], idx.size)
                    neg[lo + idx] = bits
        if is_int:
            mag = code.astype(np.int64) << qd["sh"]
            return np.where(neg, -mag, mag)
        mag = np.ldexp(code.astype(dtype), qd["E"] - B).astype(dtype)
        return np.where(neg, -mag, mag)
    val = from_negabinary(code, B)
    if is_int:
        return val << qd["sh"]
    return np.ldexp(val.astype(dtype), qd["E"] - B + 3).astype(dtype)


def stream_bytes(enc, B, words):
    """bytes(b) for b = 0..B: plane words (all-zero planes cost nothing)
    plus, for the generic encoding, the sign words of planes < b."""
    out = [0] * (B + 1)
    acc = 0
    for k in range(B):
        if enc["plane_nz"][k]:
            acc += 4 * words
        if "sign_counts" in enc:
            acc += 4 * int(np.sum(-(-enc["sign_counts"][:, k] // WORD)))
        out[k + 1] = acc
    return out
