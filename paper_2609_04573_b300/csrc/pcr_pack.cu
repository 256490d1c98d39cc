// Lossless coding of plane words (Sec. V: bitplane encoding followed by
// lossless compression).  Each plane of each 4096-value segment of a stream
// (a string of at most 4096 bits, bit e of plane word j being value
// 32 j + e) is coded on its own:
//   m = number of ones; m = 0: ZERO (header only);
//   else the Rice code of the zero runs before each one -- gaps g_i =
//   q_i - q_(i-1) - 1 (q_0 = -1) as (g >> k) one-bits, a zero-bit and the k
//   low bits of g, most significant first; the zeros after the last one are
//   implied by m -- with k the largest value <= 15 such that m 2^k <= n - m
//   (n the segment's bits; 0 when n - m < m): RICE, the code packed least
//   significant bit first into 32-bit words;
//   or, when that code is not shorter than the n raw bits: RAW, the words.
// Header word: mode (bits 0-1: 0 ZERO, 1 RICE, 2 RAW), k (bits 2-5),
// m (bits 6-18), payload words (bits 19-27).  One thread per (stream, plane, segment) task: sizes
// first (the host turns them into payload offsets), then the payloads; and
// the inverse, payloads back into plane words.
#include <cuda_runtime.h>

#include <cstdint>

#include "pcr_internal.h"

namespace pcr {

constexpr uint32_t kPackZero = 0, kPackRice = 1, kPackRaw = 2;

__device__ __forceinline__ int rice_k_of(int m, int n) {
  int k = 0;
  while (k < 15 && (m << (k + 1)) <= n - m) k++;
  return k;
}

// header and payload words of one plane of one segment (nw words at w)
__device__ void pack_size(const uint32_t* __restrict__ w, int nw, uint32_t& header, uint32_t& pwords) {
  const int n = nw * 32;
  int m = 0;
  for (int j = 0; j < nw; j++) m += __popc(w[j]);
  if (m == 0) {
    header = kPackZero;
    pwords = 0;
    return;
  }
  const int k = rice_k_of(m, n);
  // code bits: m (1 + k) + sum of (g >> k), stopped once it reaches n
  int64_t bits = (int64_t)m * (1 + k);
  int prev = -1;
  for (int j = 0; j < nw && bits < n; j++) {
    uint32_t x = w[j];
    while (x) {
      const int b = __ffs(x) - 1;
      x &= x - 1;
      const int q = 32 * j + b;
      bits += (q - prev - 1) >> k;
      prev = q;
    }
  }
  if (bits >= n) {
    pwords = (uint32_t)nw;
    header = kPackRaw | ((uint32_t)k << 2) | ((uint32_t)m << 6) | (pwords << 19);
  } else {
    pwords = (uint32_t)((bits + 31) / 32);
    header = kPackRice | ((uint32_t)k << 2) | ((uint32_t)m << 6) | (pwords << 19);
  }
}


__global__ void k_pack_sizes(const PackTask* __restrict__ tasks, int ntasks, uint32_t* __restrict__ headers,
                             uint32_t* __restrict__ pwords) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntasks) return;
  const PackTask tk = tasks[t];
  const int64_t w0 = (int64_t)tk.seg * kSegWords;
  const int nw = (int)min((int64_t)kSegWords, tk.words - w0);
  pack_size(tk.plane + w0, nw, headers[t], pwords[t]);
}

// payload of one task at out (pwords words, header from k_pack_sizes)
__global__ void k_pack_write(const PackTask* __restrict__ tasks, int ntasks, const uint32_t* __restrict__ headers,
                             const uint64_t* __restrict__ offsets, uint32_t* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntasks) return;
  const PackTask tk = tasks[t];
  const int64_t w0 = (int64_t)tk.seg * kSegWords;
  const int nw = (int)min((int64_t)kSegWords, tk.words - w0);
  const uint32_t* w = tk.plane + w0;
  uint32_t* o = out + offsets[t];
  const uint32_t h = headers[t];
  const uint32_t mode = h & 3;
  if (mode == kPackZero) return;
  if (mode == kPackRaw) {
    for (int j = 0; j < nw; j++) o[j] = w[j];
    return;
  }
  const int k = (h >> 2) & 15;
  uint32_t acc = 0;
  int fill = 0;   // bits in acc
  int64_t ow = 0;
  auto put = [&](uint32_t bit) {
    acc |= bit << fill;
    if (++fill == 32) {
      o[ow++] = acc;
      acc = 0;
      fill = 0;
    }
  };
  int prev = -1;
  for (int j = 0; j < nw; j++) {
    uint32_t x = w[j];
    while (x) {
      const int b = __ffs(x) - 1;
      x &= x - 1;
      const int q = 32 * j + b;
      const int g = q - prev - 1;
      prev = q;
      for (int u = g >> k; u > 0; u--) put(1u);
      put(0u);
      for (int i = k - 1; i >= 0; i--) put(((uint32_t)g >> i) & 1u);
    }
  }
  if (fill) o[ow] = acc;
}

// plane words of one task from its header and payload (ZERO: zeros)
__global__ void k_unpack(const PackTask* __restrict__ tasks, int ntasks, const uint32_t* __restrict__ headers,
                         const uint64_t* __restrict__ offsets, const uint32_t* __restrict__ in, int* err) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntasks) return;
  const PackTask tk = tasks[t];
  const int64_t w0 = (int64_t)tk.seg * kSegWords;
  const int nw = (int)min((int64_t)kSegWords, tk.words - w0);
  uint32_t* w = tk.plane + w0;
  const uint32_t* p = in + offsets[t];
  const uint32_t h = headers[t];
  const uint32_t mode = h & 3;
  if (mode == kPackZero) {
    for (int j = 0; j < nw; j++) w[j] = 0u;
    return;
  }
  if (mode == kPackRaw) {
    for (int j = 0; j < nw; j++) w[j] = p[j];
    return;
  }
  const int k = (h >> 2) & 15, m = (int)((h >> 6) & 0x1FFF);
  const int n = nw * 32;
  for (int j = 0; j < nw; j++) w[j] = 0u;
  // the payload is read within its word count (header, checked by the host
  // against the segment); a code that runs past it or sets a bit beyond
  // the segment is corrupt: flagged, nothing written past it
  const int64_t lim = (int64_t)(h >> 19) * 32;
  int64_t bitpos = 0;
  auto get = [&]() -> uint32_t {
    const uint32_t v = (p[bitpos >> 5] >> (bitpos & 31)) & 1u;
    bitpos++;
    return v;
  };
  int prev = -1;
  for (int i = 0; i < m; i++) {
    int g = 0;
    while (bitpos < lim && get()) g += 1 << k;
    for (int u = k - 1; u >= 0 && bitpos < lim; u--) g |= (int)get() << u;
    const int q = prev + 1 + g;
    if (bitpos > lim || q >= n || q < 0) {
      atomicExch(err, 1);
      return;
    }
    w[q >> 5] |= 1u << (q & 31);
    prev = q;
  }
}

void launch_pack_sizes(const PackTask* tasks, int ntasks, uint32_t* headers, uint32_t* pwords, cudaStream_t s) {
  if (ntasks <= 0) return;
  count_launch();
  k_pack_sizes<<<(ntasks + 127) / 128, 128, 0, s>>>(tasks, ntasks, headers, pwords);
}

void launch_pack_write(const PackTask* tasks, int ntasks, const uint32_t* headers, const uint64_t* offsets,
                       uint32_t* out, cudaStream_t s) {
  if (ntasks <= 0) return;
  count_launch();
  k_pack_write<<<(ntasks + 127) / 128, 128, 0, s>>>(tasks, ntasks, headers, offsets, out);
}

void launch_unpack(const PackTask* tasks, int ntasks, const uint32_t* headers, const uint64_t* offsets,
                   const uint32_t* in, int* err, cudaStream_t s) {
  if (ntasks <= 0) return;
  count_launch();
  k_unpack<<<(ntasks + 127) / 128, 128, 0, s>>>(tasks, ntasks, headers, offsets, in, err);
}

}  // namespace pcr
