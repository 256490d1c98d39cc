// Tiled interpolation and coefficient-decomposition kernels (sm_103a).
//
// One CTA owns a box of one level's grid, stages the box plus a halo in
// shared memory with coalesced row loads along the fastest axis, and runs
// the level's region passes there (Sec. VI-C "fastest direction
// interpolation": region r is predicted along its pass axis from the points
// that are even along it).  Every prediction is evaluated once per tile, so
// the per-level tensor interpolant costs about one 1-D rule per point.
//
// The same kernel serves the four directions of the method:
//   refactor, per-level  : c = x - W, shared memory keeps predictions W
//   refactor, per-region : c = x - W, W from original values only
//   retrieve, per-level  : x' = W + c_hat, W from reconstructed coarse values
//   retrieve, per-region : x' = W + c_hat, earlier regions reconstructed in
//                          the tile (halo points recomputed, not exchanged)
// Arithmetic: the rules of pcr_kernels.cu (identical expression trees).
#include <cuda_runtime.h>
#include <algorithm>
#include <atomic>
#include <mutex>
#include <map>
#include <cstdint>
#include <type_traits>
#include <vector>

#include <cuda.h>
#include <cudaTypedefs.h>

#include "pcr_internal.h"

namespace pcr {

#define FULLMASK 0xFFFFFFFFu

// minimum / maximum / finiteness of whole fields (pcr_kernels.cu)
void launch_minmax_multi(int vk, const void* const* xs, const int64_t* ns, FieldStats* const* sts, int n,
                         cudaStream_t s);

// 1-D interpolation rules, same expressions as the codec file's (rounding:
// cubic <= 2.75 u V, edges <= 2.875 u V, mean <= u V for inputs bounded by V)
template <typename T> struct TAr;
template <> struct TAr<float> {
  __device__ static float lin(float a, float b) { return __fmul_rn(__fadd_rn(a, b), 0.5f); }
  __device__ static float cub(float m3, float m1, float p1, float p3) {
    const float s1 = __fadd_rn(m1, p1);   // mean + correction: s1 / 2 + (s1 - s2) / 16
    return __fadd_rn(__fmul_rn(s1, 0.5f), __fmul_rn(__fsub_rn(s1, __fadd_rn(m3, p3)), 0.0625f));
  }
  __device__ static float lft(float m1, float p1, float p3) {
    return __fadd_rn(__fmul_rn(p1, 0.75f), __fsub_rn(__fmul_rn(m1, 0.375f), __fmul_rn(p3, 0.125f)));
  }
  __device__ static float rgt(float m3, float m1, float p1) {
    return __fadd_rn(__fmul_rn(m1, 0.75f), __fsub_rn(__fmul_rn(p1, 0.375f), __fmul_rn(m3, 0.125f)));
  }
  __device__ static float add(float a, float b) { return __fadd_rn(a, b); }
  __device__ static float sub(float a, float b) { return __fsub_rn(a, b); }
  __device__ static unsigned long long mag(float v) { return __float_as_uint(fabsf(v)); }
};
template <> struct TAr<double> {
  __device__ static double lin(double a, double b) { return __dmul_rn(__dadd_rn(a, b), 0.5); }
  __device__ static double cub(double m3, double m1, double p1, double p3) {
    const double s1 = __dadd_rn(m1, p1);
    return __dadd_rn(__dmul_rn(s1, 0.5), __dmul_rn(__dsub_rn(s1, __dadd_rn(m3, p3)), 0.0625));
  }
  __device__ static double lft(double m1, double p1, double p3) {
    return __dadd_rn(__dmul_rn(p1, 0.75), __dsub_rn(__dmul_rn(m1, 0.375), __dmul_rn(p3, 0.125)));
  }
  __device__ static double rgt(double m3, double m1, double p1) {
    return __dadd_rn(__dmul_rn(m1, 0.75), __dsub_rn(__dmul_rn(p1, 0.375), __dmul_rn(m3, 0.125)));
  }
  __device__ static double add(double a, double b) { return __dadd_rn(a, b); }
  __device__ static double sub(double a, double b) { return __dsub_rn(a, b); }
  __device__ static unsigned long long mag(double v) { return (unsigned long long)__double_as_longlong(fabs(v)); }
};
template <> struct TAr<int64_t> {
  __device__ static int64_t lin(int64_t a, int64_t b) { return (a + b) >> 1; }
  __device__ static int64_t cub(int64_t m3, int64_t m1, int64_t p1, int64_t p3) { return (9 * (m1 + p1) - (m3 + p3)) >> 4; }
  __device__ static int64_t lft(int64_t m1, int64_t p1, int64_t p3) { return (3 * m1 + 6 * p1 - p3) >> 3; }
  __device__ static int64_t rgt(int64_t m3, int64_t m1, int64_t p1) { return (6 * m1 + 3 * p1 - m3) >> 3; }
  __device__ static int64_t add(int64_t a, int64_t b) { return a + b; }
  __device__ static int64_t sub(int64_t a, int64_t b) { return a - b; }
  __device__ static unsigned long long mag(int64_t v) { return (unsigned long long)(v < 0 ? -v : v); }
};

// one 1-D rule at odd index j of a line of m points; at(k) reads index k
template <typename T, class F>
__device__ __forceinline__ T rule(int j, int m, int degree, const F& at) {
  const bool p1 = j + 1 < m;
  if (degree == 3) {
    const bool m3 = j >= 3, p3 = j + 3 < m;
    if (p1 && m3 && p3) return TAr<T>::cub(at(j - 3), at(j - 1), at(j + 1), at(j + 3));
    if (p1 && p3) return TAr<T>::lft(at(j - 1), at(j + 1), at(j + 3));
    if (p1 && m3) return TAr<T>::rgt(at(j - 3), at(j - 1), at(j + 1));
  }
  if (p1) return TAr<T>::lin(at(j - 1), at(j + 1));
  return at(j - 1);
}

__device__ __forceinline__ unsigned long long wmax(unsigned long long v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(FULLMASK, v, o);
    v = t > v ? t : v;
  }
  return v;
}

__device__ __forceinline__ void push_max(unsigned long long* slot, unsigned long long v, int bytes) {
  v = wmax(v);
  if ((threadIdx.x & 31) == 0 && v && slot) {
    if (bytes == 4) atomicMax((unsigned int*)slot, (unsigned int)v);
    else atomicMax(slot, v);
  }
}

// warp maximum of |values| given as bit patterns of A, merged into a slot
// holding the bits of a non-negative double
template <typename A>
__device__ __forceinline__ void push_max_double(unsigned long long* slot, unsigned long long v) {
  v = wmax(v);
  if ((threadIdx.x & 31) == 0 && v && slot) {
    const double d = sizeof(A) == 4 ? (double)__uint_as_float((unsigned)v) : __longlong_as_double((long long)v);
    atomicMax(slot, (unsigned long long)__double_as_longlong(d));
  }
}

// ---------------------------------------------------------------------------
// interpolation tile kernel
// ---------------------------------------------------------------------------
// asynchronous global -> shared copies (zero-filled when !valid)
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(sa), "l"(gmem), "r"(valid ? 4 : 0));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem, bool valid) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(sa), "l"(gmem), "r"(valid ? 8 : 0));
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::);
  asm volatile("cp.async.wait_group 0;\n" ::);
}
// One region pass of one staged tile along compile-time axis AX.
// Range: odd along AX inside the tile; even along later pass axes (with the
// halo when `halo`); the tile along earlier axes.  Shared-memory neighbours
// along AX are at compile-time offsets; interior lines skip the boundary
// checks of the 1-D rule.
template <typename A, int AX, int T0, int T1, int T2, int H0, int H, int S1, int S2>
__device__ __forceinline__ void tile_pass(const TileArgs& a, A* __restrict__ S, const TileRegion& R, int b0, int b1,
                                          int b2, int o0, int o1, int o2, bool later0, bool later1, bool later2,
                                          bool halo, bool per_level, bool retrieve, A* __restrict__ dst) {
  constexpr int DEG = H == 3 ? 3 : 1;
  constexpr int SSTEP = AX == 0 ? S1 * S2 : (AX == 1 ? S2 : 1);
  const int m[3] = {(int)a.m[0], (int)a.m[1], (int)a.m[2]};
  const int b[3] = {b0, b1, b2};
  const int Tt[3] = {T0, T1, T2};
  const int Hh[3] = {H0, H, H};
  const bool later[3] = {later0, later1, later2};
  int lo[3], n[3], st[3];
#pragma unroll
  for (int k = 0; k < 3; k++) {
    int l, hi;
    if (k == AX) {
      l = b[k] + 1;
      hi = min(b[k] + Tt[k], m[k]);
      st[k] = 2;
    } else if (later[k]) {
      l = (halo ? max(b[k] - Hh[k], 0) : b[k]);
      l = (l + 1) & ~1;
      hi = halo ? min(b[k] + Tt[k] + Hh[k], m[k]) : min(b[k] + Tt[k], m[k]);
      st[k] = 2;
    } else {
      l = b[k];
      hi = min(b[k] + Tt[k], m[k]);
      st[k] = 1;
    }
    lo[k] = l;
    n[k] = hi > l ? (hi - l + st[k] - 1) / st[k] : 0;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int sh0 = R.step[0] == 2, sh1 = R.step[1] == 2, sh2 = R.step[2] == 2;
  const int rs0 = (int)R.start[0], rs1 = (int)R.start[1], rs2 = (int)R.start[2];
  // streams hold fewer than 2^31 elements, so staging offsets fit in 32 bits
  const int rc1 = (int)R.count[1], rpad = (int)R.row_pad, rbase = (int)R.base;
  A* __restrict__ stg = reinterpret_cast<A*>(R.stage);
  const int mlen = m[AX];
  const int rows = n[0] * n[1];
  const unsigned inv = n[1] ? ((1u << 20) + n[1] - 1) / n[1] : 0;   // row / n1 without a division
  float fmx = 0.0f;
  unsigned long long imx = 0;
  const int total = rows * n[2];
  const unsigned inv2 = n[2] ? ((1u << 20) + n[2] - 1) / n[2] : 0;   // idx / n2 (idx < 2^14)
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int row = (int)(((unsigned)idx * inv2) >> 20), i2 = idx - row * n[2];
    const int i0 = (int)(((unsigned)row * inv) >> 20), i1 = row - i0 * n[1];
    const int q0 = lo[0] + st[0] * i0, q1 = lo[1] + st[1] * i1, q2 = lo[2] + st[2] * i2;
    const int sp = ((q0 - o0) * S1 + (q1 - o1)) * S2 + (q2 - o2);
    A W;
    const int jj = AX == 0 ? q0 : (AX == 1 ? q1 : q2);
    if (DEG == 3 && jj >= 3 && jj + 3 < mlen) {
      W = TAr<A>::cub(S[sp - 3 * SSTEP], S[sp - SSTEP], S[sp + SSTEP], S[sp + 3 * SSTEP]);
    } else {
      auto at = [&](int k) -> A { return S[sp + (k - jj) * SSTEP]; };
      W = rule<A>(jj, mlen, DEG, at);
    }
    const bool in_tile = q0 >= b0 && q0 < b0 + T0 && q1 >= b1 && q1 < b1 + T1 && q2 >= b2 && q2 < b2 + T2;
    const int si = rbase + (((q0 - rs0) >> sh0) * rc1 + ((q1 - rs1) >> sh1)) * rpad + ((q2 - rs2) >> sh2);
    if (!retrieve) {
      if (in_tile) {
        const A c = TAr<A>::sub(S[sp], W);
        stg[si] = c;
        if constexpr (std::is_same<A, float>::value) fmx = fmaxf(fmx, fabsf(c));
        else {
          const unsigned long long mg = TAr<A>::mag(c);
          imx = mg > imx ? mg : imx;
        }
      }
      if (per_level) S[sp] = W;
    } else {
      const int64_t di = (int64_t)q0 * a.stride[0] + (int64_t)q1 * a.stride[1] + (int64_t)q2 * a.stride[2];
      if (per_level) {
        S[sp] = W;
        if (in_tile) dst[di] = TAr<A>::add(W, stg[si]);
      } else {
        const A xv = TAr<A>::add(W, stg[si]);
        S[sp] = xv;
        if (in_tile) dst[di] = xv;
      }
    }
  }
  (void)lane;
  (void)warp;
  (void)nwarp;
  if (!retrieve) {
    if constexpr (std::is_same<A, float>::value) imx = __float_as_uint(fmx);
    if (R.vmax_double) push_max_double<A>(R.vmax, imx);
    else push_max(R.vmax, imx, sizeof(A));
  }
}

template <typename A, int T0, int T1, int T2, int H0, int H>
__device__ __forceinline__ void tile_interp_body(const TileArgs& a, unsigned bid) {
  // the x extent of the staged box starts 4 points (not H) before the tile so
  // that, for float fields whose rows are 16-byte multiples, every staged row
  // is loaded with aligned 16-byte vectors
  constexpr int XL = 4;
  constexpr int S1 = T1 + 2 * H, S2 = T2 + 8;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  A* S = reinterpret_cast<A*>(smem_raw);

  const unsigned nt2 = (unsigned)a.ntiles[2], nt1 = (unsigned)a.ntiles[1];
  const int b2 = (int)(bid % nt2 + a.tlo[2]) * T2;
  bid /= nt2;
  const int b1 = (int)(bid % nt1 + a.tlo[1]) * T1;
  const int b0 = (int)(bid / nt1 + a.tlo[0]) * T0;
  const int o0 = b0 - H0, o1 = b1 - H, o2 = b2 - XL;
  const A* __restrict__ src = reinterpret_cast<const A*>(a.src);
  A* __restrict__ dst = reinterpret_cast<A*>(a.dst);
  {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int m0 = (int)a.m[0], m1 = (int)a.m[1], m2 = (int)a.m[2];
    const int64_t st2 = a.stride[2];
    // 16-byte vectors: float rows of unit x-stride, 16-byte aligned row starts
    const bool vec = sizeof(A) == 4 && st2 == 1 && (a.stride[1] % 4) == 0 && (a.stride[0] % 4) == 0 &&
                     ((uintptr_t)src % 16) == 0;
    // rows needed along an axis: the tile, plus the halo points that are
    // even (every 1-D rule reads points even along its axis)
    constexpr int HL0 = H0 == 0 ? 0 : H0 / 2, HR0 = H0 == 0 ? 0 : (H0 + 1) / 2;
    constexpr int HL = H / 2, HR = (H + 1) / 2;
    constexpr int R0 = T0 + HL0 + HR0, R1 = T1 + HL + HR;
    auto rowpos = [](int c, int b, int T, int hl) -> int {   // compact row -> coordinate
      if (c < hl) return b - 2 * (hl - c);
      if (c < hl + T) return b + (c - hl);
      return b + T + 2 * (c - hl - T);
    };
    if (vec) {
      constexpr int NV = S2 / 4;
      for (int idx = threadIdx.x; idx < R0 * R1 * NV; idx += blockDim.x) {
        const int rr = idx / NV, v = idx - rr * NV;
        const int c0 = rr / R1, c1 = rr - c0 * R1;
        const int q0 = rowpos(c0, b0, T0, HL0), q1 = rowpos(c1, b1, T1, HL);
        const bool rok = q0 >= 0 && q0 < m0 && q1 >= 0 && q1 < m1;
        const float* rp = reinterpret_cast<const float*>(src) + (rok ? (int64_t)q0 * a.stride[0] + (int64_t)q1 * a.stride[1] : 0);
        float* d = reinterpret_cast<float*>(S) + ((q0 - o0) * S1 + (q1 - o1)) * S2 + 4 * v;
        const int x = o2 + 4 * v;
        if (rok && x >= 0 && x + 3 < m2) {
          cp_async16(d, rp + x);
        } else {
#pragma unroll
          for (int e = 0; e < 4; e++) {
            const bool ok = rok && x + e >= 0 && x + e < m2;
            cp_async4(d + e, ok ? (const void*)(rp + x + e) : (const void*)src, ok);
          }
        }
      }
    } else {
      for (int idx = threadIdx.x; idx < R0 * R1 * S2; idx += blockDim.x) {
        const int rr = idx / S2, i2 = idx - rr * S2;
        const int c0 = rr / R1, c1 = rr - c0 * R1;
        const int q0 = rowpos(c0, b0, T0, HL0), q1 = rowpos(c1, b1, T1, HL);
        const int q2 = o2 + i2;
        const bool ok = q0 >= 0 && q0 < m0 && q1 >= 0 && q1 < m1 && q2 >= 0 && q2 < m2;
        A* d = S + ((q0 - o0) * S1 + (q1 - o1)) * S2 + i2;
        const A* g = ok ? src + (int64_t)q0 * a.stride[0] + (int64_t)q1 * a.stride[1] + (int64_t)q2 * st2 : src;
        if (sizeof(A) == 4) cp_async4(d, g, ok);
        else cp_async8(d, g, ok);
      }
    }
    (void)lane;
    (void)warp;
    (void)nwarp;
  }
  cp_async_wait_all();
  __syncthreads();

  const bool per_level = a.interp == 0;
  const bool retrieve = a.retrieve != 0;
  const bool halo = retrieve || per_level;
  for (int r = 0; r < a.d; r++) {
    const int ax = r == 0 ? a.order[0] : (r == 1 ? a.order[1] : a.order[2]);
    bool l0 = false, l1 = false, l2 = false;
    for (int k = r + 1; k < a.d; k++) {
      const int bx = k == 1 ? a.order[1] : a.order[2];
      l0 |= bx == 0;
      l1 |= bx == 1;
      l2 |= bx == 2;
    }
    const TileRegion R = r == 0 ? a.reg[0] : (r == 1 ? a.reg[1] : a.reg[2]);
    if (ax == 0)
      tile_pass<A, 0, T0, T1, T2, H0, H, S1, S2>(a, S, R, b0, b1, b2, o0, o1, o2, l0, l1, l2, halo, per_level,
                                                 retrieve, dst);
    else if (ax == 1)
      tile_pass<A, 1, T0, T1, T2, H0, H, S1, S2>(a, S, R, b0, b1, b2, o0, o1, o2, l0, l1, l2, halo, per_level,
                                                 retrieve, dst);
    else
      tile_pass<A, 2, T0, T1, T2, H0, H, S1, S2>(a, S, R, b0, b1, b2, o0, o1, o2, l0, l1, l2, halo, per_level,
                                                 retrieve, dst);
    __syncthreads();
  }
}

template <typename A, int T0, int T1, int T2, int H0, int H>
__global__ void __launch_bounds__(256) k_tile_interp(TileArgs a) {
  tile_interp_body<A, T0, T1, T2, H0, H>(a, blockIdx.x);
}

// Several independent level grids (the levels >= 1 of a refactor, or of
// several fields) in one launch: the tiles of args[i] are blocks
// first[i] .. first[i + 1] - 1.
template <typename A, int T0, int T1, int T2, int H0, int H>
__global__ void __launch_bounds__(256) k_tile_interp_multi(const __grid_constant__ TileBatch b) {
  const int i = batch_find(b.first, b.n);
  tile_interp_body<A, T0, T1, T2, H0, H>(b.args[i], blockIdx.x - (unsigned)b.first[i]);
}

// ---------------------------------------------------------------------------
// coefficient decomposition tile kernel (Sec. V-B, Alg. 1 / Alg. 2)
// ---------------------------------------------------------------------------
// Works on one region's compact array (dims cnt, row-major) with slices
// normal to axis N; in-slice axes U < V.  The tile covers T[k] compact points
// per axis plus one extra point at the high end of each in-slice axis (the
// next 4-grid line), so every prediction is local.  Sub-level slots:
// 0 S1 (4-grid), 1 S2a (u = 2 mod 4, v = 0 mod 4), 2 S2b (u even, v = 2 mod
// 4), 3 S3a (u odd, v even), 4 S3b (v odd).
template <int N> struct Axes;
template <> struct Axes<0> { static constexpr int U = 1, V = 2; };
template <> struct Axes<1> { static constexpr int U = 0, V = 2; };
template <> struct Axes<2> { static constexpr int U = 0, V = 1; };

__device__ __forceinline__ int slot_of(int ku, int kv) {
  if (((ku | kv) & 3) == 0) return 0;
  if (((ku | kv) & 1) == 0) return (kv & 3) == 0 ? 1 : 2;
  return (kv & 1) == 0 ? 3 : 4;
}

// log2 of the sub-lattice steps along (u, v) and starts, per slot
__device__ __forceinline__ void slot_geom(int sl, int& su, int& lu, int& sv, int& lv) {
  switch (sl) {
    case 0: su = 0; lu = 2; sv = 0; lv = 2; break;
    case 1: su = 2; lu = 2; sv = 0; lv = 2; break;
    case 2: su = 0; lu = 1; sv = 2; lv = 2; break;
    case 3: su = 1; lu = 1; sv = 0; lv = 1; break;
    default: su = 0; lu = 0; sv = 1; lv = 1; break;
  }
}

template <typename A, int N, int T0, int T1, int T2>
__global__ void __launch_bounds__(256) k_tile_decomp(DecompArgs a) {
  constexpr int U = Axes<N>::U, V = Axes<N>::V;
  constexpr int S0 = T0 + (N != 0), S1 = T1 + (N != 1), S2 = T2 + (N != 2);
  constexpr int TS[3] = {T0, T1, T2};
  extern __shared__ __align__(16) unsigned char smem_raw[];
  A* S = reinterpret_cast<A*>(smem_raw);
  int64_t bid = blockIdx.x;
  const int tb2 = (int)((bid % a.ntiles[2]) * T2);
  bid /= a.ntiles[2];
  const int tb1 = (int)((bid % a.ntiles[1]) * T1);
  const int tb0 = (int)((bid / a.ntiles[1]) * T0);
  const int cnt0 = (int)a.cnt[0], cnt1 = (int)a.cnt[1], cnt2 = (int)a.cnt[2];
  const int cu = (int)a.cnt[U], cv = (int)a.cnt[V];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  A* __restrict__ comp = reinterpret_cast<A*>(a.comp);
  (void)TS;

  auto pick = [](int k0, int k1, int k2, int ax) { return ax == 0 ? k0 : (ax == 1 ? k1 : k2); };
  auto stage_index = [&](int sl, int k0, int k1, int k2) -> int64_t {
    int su, lu, sv, lv;
    slot_geom(sl, su, lu, sv, lv);
    const DecompSub& sb = a.subs[sl];
    int l[3] = {k0, k1, k2};
    l[U] = (pick(k0, k1, k2, U) - su) >> lu;
    l[V] = (pick(k0, k1, k2, V) - sv) >> lv;
    return sb.base + ((int64_t)l[0] * sb.count[1] + l[1]) * sb.row_pad + l[2];
  };
  auto sidx = [&](int k0, int k1, int k2) { return ((k0 - tb0) * S1 + (k1 - tb1)) * S2 + (k2 - tb2); };
  constexpr int dU = U == 0 ? S1 * S2 : (U == 1 ? S2 : 1);
  constexpr int dV = V == 0 ? S1 * S2 : (V == 1 ? S2 : 1);

  for (int row = warp; row < S0 * S1; row += nwarp) {
    const int k0 = tb0 + row / S1, k1 = tb1 + row % S1;
#pragma unroll 2
    for (int i2 = lane; i2 < S2; i2 += 32) {
      const int k2 = tb2 + i2;
      A val = A(0);
      if (k0 < cnt0 && k1 < cnt1 && k2 < cnt2) {
        if (!a.retrieve) {
          val = comp[((int64_t)k0 * cnt1 + k1) * cnt2 + k2];
        } else {
          const int sl = slot_of(pick(k0, k1, k2, U), pick(k0, k1, k2, V));
          val = reinterpret_cast<const A*>(a.subs[sl].stage)[stage_index(sl, k0, k1, k2)];
        }
      }
      S[row * S2 + i2] = val;
    }
  }
  __syncthreads();

  // per-level linear prediction (Alg. 1 Pi_2: t = 2 from the 4-grid;
  // Pi_1: t = 1 from the 2-grid); the v pass reads u-pass predictions
  auto predict = [&](int sp, int ku, int kv, int t) -> A {
    auto pass_u = [&](int p) -> A {
      if (ku + t < cu) return TAr<A>::lin(S[p - t * dU], S[p + t * dU]);
      return S[p - t * dU];
    };
    if ((kv & (2 * t - 1)) == 0) return pass_u(sp);
    const bool u_coarse = (ku & (2 * t - 1)) == 0;
    auto src = [&](int p) -> A { return u_coarse ? S[p] : pass_u(p); };
    if (kv + t < cv) return TAr<A>::lin(src(sp - t * dV), src(sp + t * dV));
    return src(sp - t * dV);
  };

  if (!a.retrieve) {
    unsigned long long m0 = 0, m1 = 0, m2 = 0, m3 = 0, m4 = 0, cm = 0;
    for (int row = warp; row < T0 * T1; row += nwarp) {
      const int k0 = tb0 + row / T1, k1 = tb1 + row % T1;
      if (k0 >= cnt0 || k1 >= cnt1) continue;
      for (int i2 = lane; i2 < T2; i2 += 32) {
        const int k2 = tb2 + i2;
        if (k2 >= cnt2) continue;
        const int ku = pick(k0, k1, k2, U), kv = pick(k0, k1, k2, V);
        const int sl = slot_of(ku, kv);
        const int sp = sidx(k0, k1, k2);
        const A c = S[sp];
        const unsigned long long cg = TAr<A>::mag(c);
        cm = cg > cm ? cg : cm;
        const A dv = sl == 0 ? c : TAr<A>::sub(c, predict(sp, ku, kv, sl <= 2 ? 2 : 1));
        reinterpret_cast<A*>(a.subs[sl].stage)[stage_index(sl, k0, k1, k2)] = dv;
        const unsigned long long mg = TAr<A>::mag(dv);
        if (sl == 0) m0 = mg > m0 ? mg : m0;
        else if (sl == 1) m1 = mg > m1 ? mg : m1;
        else if (sl == 2) m2 = mg > m2 ? mg : m2;
        else if (sl == 3) m3 = mg > m3 ? mg : m3;
        else m4 = mg > m4 ? mg : m4;
      }
    }
    push_max(a.subs[0].vmax, m0, sizeof(A));
    push_max(a.subs[1].vmax, m1, sizeof(A));
    push_max(a.subs[2].vmax, m2, sizeof(A));
    push_max(a.subs[3].vmax, m3, sizeof(A));
    push_max(a.subs[4].vmax, m4, sizeof(A));
    push_max_double<A>(a.c0, cm);
    return;
  }
  // recompose: S1 as decoded; S2 (tile + high halo) from S1; then S3 (tile)
  for (int row = warp; row < S0 * S1; row += nwarp) {
    const int k0 = tb0 + row / S1, k1 = tb1 + row % S1;
    if (k0 >= cnt0 || k1 >= cnt1) continue;
    for (int i2 = lane; i2 < S2; i2 += 32) {
      const int k2 = tb2 + i2;
      if (k2 >= cnt2) continue;
      const int ku = pick(k0, k1, k2, U), kv = pick(k0, k1, k2, V);
      const int sl = slot_of(ku, kv);
      if (sl != 1 && sl != 2) continue;
      const int sp = row * S2 + i2;
      S[sp] = TAr<A>::add(predict(sp, ku, kv, 2), S[sp]);
    }
  }
  __syncthreads();
  for (int row = warp; row < T0 * T1; row += nwarp) {
    const int k0 = tb0 + row / T1, k1 = tb1 + row % T1;
    if (k0 >= cnt0 || k1 >= cnt1) continue;
    for (int i2 = lane; i2 < T2; i2 += 32) {
      const int k2 = tb2 + i2;
      if (k2 >= cnt2) continue;
      const int ku = pick(k0, k1, k2, U), kv = pick(k0, k1, k2, V);
      const int sp = sidx(k0, k1, k2);
      A r = S[sp];
      if (slot_of(ku, kv) >= 3) r = TAr<A>::add(predict(sp, ku, kv, 1), r);
      comp[((int64_t)k0 * cnt1 + k1) * cnt2 + k2] = r;
    }
  }
}

// Slices normal to the fastest axis (N = 2, in-slice axes u = 0, v = 1).
// One thread owns the 4 x 4 block (4a.., 4b..) of in-slice points for one
// vector of VEC consecutive points along the normal axis, and holds the
// block's 5 x 5 neighbourhood (the next 4-grid lines included) in registers.
// Within a block the sub-level of point (du, dv) and its prediction rule are
// compile-time constants; the lines shared with the next blocks are read
// again by those blocks (from L2).  Loads and stores are VEC-wide along the
// contiguous normal axis.
template <typename A, int VEC> struct VecT { A v[VEC]; };
template <typename A, int VEC>
__device__ __forceinline__ void vld(VecT<A, VEC>& d, const A* p) {
  if constexpr (VEC * sizeof(A) == 16) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(p));
    static_assert(sizeof(VecT<A, VEC>) == 16, "vector size");
    d = *reinterpret_cast<const VecT<A, VEC>*>(&t);
  } else if constexpr (VEC * sizeof(A) == 8) {
    const float2 t = __ldg(reinterpret_cast<const float2*>(p));
    d = *reinterpret_cast<const VecT<A, VEC>*>(&t);
  } else {
#pragma unroll
    for (int e = 0; e < VEC; e++) d.v[e] = p[e];
  }
}
template <typename A, int VEC>
__device__ __forceinline__ void vst(A* p, const VecT<A, VEC>& d) {
  if constexpr (VEC * sizeof(A) == 16) {
    *reinterpret_cast<float4*>(p) = *reinterpret_cast<const float4*>(&d);
  } else if constexpr (VEC * sizeof(A) == 8) {
    *reinterpret_cast<float2*>(p) = *reinterpret_cast<const float2*>(&d);
  } else {
#pragma unroll
    for (int e = 0; e < VEC; e++) p[e] = d.v[e];
  }
}

// sub-level slot of in-block offsets (du, dv) (both taken mod 4)
__host__ __device__ constexpr int blk_slot(int du, int dv) {
  return ((du | dv) & 3) == 0 ? 0 : (((du | dv) & 1) == 0 ? ((dv & 3) == 0 ? 1 : 2) : ((dv & 1) == 0 ? 3 : 4));
}
__host__ __device__ constexpr int blk_su(int sl) { return sl == 1 ? 2 : (sl == 3 ? 1 : 0); }
__host__ __device__ constexpr int blk_lu(int sl) { return sl <= 1 ? 2 : (sl <= 3 ? 1 : 0); }
__host__ __device__ constexpr int blk_sv(int sl) { return sl == 2 ? 2 : (sl == 4 ? 1 : 0); }
__host__ __device__ constexpr int blk_lv(int sl) { return sl <= 2 ? 2 : 1; }

template <typename A, int VEC>
__global__ void __launch_bounds__(128) k_decomp_blk(DecompArgs a) {
  using V = VecT<A, VEC>;
  const unsigned nvec = (unsigned)a.ntiles[2], nbb = (unsigned)a.ntiles[1], nab = (unsigned)a.ntiles[0];
  const unsigned item = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned iv = item % nvec + (unsigned)a.tlo[2], rest = item / nvec;
  const unsigned bb = rest % nbb + (unsigned)a.tlo[1], ab = rest / nbb + (unsigned)a.tlo[0];
  const bool live = rest / nbb < nab;
  const int cu = (int)a.cnt[0], cv = (int)a.cnt[1];
  const int64_t cw = a.cnt[2];
  const int u0 = 4 * (int)ab, v0 = 4 * (int)bb;
  const int64_t k2 = (int64_t)iv * VEC;
  A* __restrict__ comp = reinterpret_cast<A*>(a.comp);
  bool vu[5], vv[5];
#pragma unroll
  for (int d = 0; d < 5; d++) {
    vu[d] = live && u0 + d < cu;
    vv[d] = live && v0 + d < cv;
  }
  // row of slot sl holding in-block offsets (du, dv), this thread's vector
  auto srow = [&](int sl, int du, int dv) -> A* {
    const DecompSub& sb = a.subs[sl];
    const int64_t ui = ((int64_t)ab << (2 - blk_lu(sl))) + ((du - blk_su(sl)) >> blk_lu(sl));
    const int64_t vi = ((int64_t)bb << (2 - blk_lv(sl))) + ((dv - blk_sv(sl)) >> blk_lv(sl));
    return reinterpret_cast<A*>(sb.stage) + sb.base + (ui * sb.count[1] + vi) * sb.row_pad + k2;
  };
  V x[5][5];
  auto lin = [](const V& p, const V& q) {
    V r;
#pragma unroll
    for (int e = 0; e < VEC; e++) r.v[e] = TAr<A>::lin(p.v[e], q.v[e]);
    return r;
  };
  // per-level linear prediction with step t (Alg. 1: t = 2 from the 4-grid,
  // t = 1 from the 2-grid); the v pass reads u-pass predictions
  auto pass_u = [&](int du, int dv, int t) -> V { return vu[du + t] ? lin(x[du - t][dv], x[du + t][dv]) : x[du - t][dv]; };
  auto predict = [&](int du, int dv, int t) -> V {
    if (dv % (2 * t) == 0) return pass_u(du, dv, t);
    const bool uc = du % (2 * t) == 0;
    const V lo = uc ? x[du][dv - t] : pass_u(du, dv - t, t);
    if (!vv[dv + t]) return lo;
    const V hi = uc ? x[du][dv + t] : pass_u(du, dv + t, t);
    return lin(lo, hi);
  };

  if (!a.retrieve) {
#pragma unroll
    for (int du = 0; du < 5; du++)
#pragma unroll
      for (int dv = 0; dv < 5; dv++) {
        if (vu[du] && vv[dv]) vld<A, VEC>(x[du][dv], comp + ((int64_t)(u0 + du) * cv + (v0 + dv)) * cw + k2);
        else
#pragma unroll
          for (int e = 0; e < VEC; e++) x[du][dv].v[e] = A(0);
      }
    A mx[5] = {A(0), A(0), A(0), A(0), A(0)};   // max |value| per sub-level
#pragma unroll
    for (int du = 0; du < 4; du++)
#pragma unroll
      for (int dv = 0; dv < 4; dv++) {
        if (!(vu[du] && vv[dv])) continue;
        const int sl = blk_slot(du, dv);
        V d = x[du][dv];
        if (sl != 0) {
          const V w = predict(du, dv, sl <= 2 ? 2 : 1);
#pragma unroll
          for (int e = 0; e < VEC; e++) d.v[e] = TAr<A>::sub(d.v[e], w.v[e]);
        }
        vst<A, VEC>(srow(sl, du, dv), d);
#pragma unroll
        for (int e = 0; e < VEC; e++) mx[sl] = fmax(mx[sl], fabs(d.v[e]));
      }
#pragma unroll
    for (int q = 0; q < 5; q++) push_max(a.subs[q].vmax, TAr<A>::mag(mx[q]), sizeof(A));
    return;
  }
  // recompose: decoded sub-level values of the block and of the next 4-grid
  // lines' 2-grid points; S2 from S1, then S3 from the 2-grid (Alg. 2)
#pragma unroll
  for (int du = 0; du < 5; du++)
#pragma unroll
    for (int dv = 0; dv < 5; dv++) {
      const bool need = (du < 4 && dv < 4) || ((du | dv) & 1) == 0;
      if (need && vu[du] && vv[dv]) vld<A, VEC>(x[du][dv], srow(blk_slot(du, dv), du, dv));
      else
#pragma unroll
        for (int e = 0; e < VEC; e++) x[du][dv].v[e] = A(0);
    }
#pragma unroll
  for (int du = 0; du < 5; du += 2)
#pragma unroll
    for (int dv = 0; dv < 5; dv += 2) {
      if (((du | dv) & 3) == 0 || !(vu[du] && vv[dv])) continue;
      const V w = predict(du, dv, 2);
#pragma unroll
      for (int e = 0; e < VEC; e++) x[du][dv].v[e] = TAr<A>::add(w.v[e], x[du][dv].v[e]);
    }
#pragma unroll
  for (int du = 0; du < 4; du++)
#pragma unroll
    for (int dv = 0; dv < 4; dv++) {
      if (!(vu[du] && vv[dv])) continue;
      V r = x[du][dv];
      if (((du | dv) & 1) != 0) {
        const V w = predict(du, dv, 1);
#pragma unroll
        for (int e = 0; e < VEC; e++) r.v[e] = TAr<A>::add(w.v[e], r.v[e]);
      }
      vst<A, VEC>(comp + ((int64_t)(u0 + du) * cv + (v0 + dv)) * cw + k2, r);
    }
}

// The forward decomposition of one 4 x 4 in-slice block (block indices ab,
// bb) at VEC consecutive points along the normal (starting at k2): S1 / S2 /
// S3 values written to their sub-level rows, their magnitudes folded into
// mx.  `ld(r, du, dv)` loads the block's point (du, dv), du, dv in 0..4 (the
// next 4-grid lines included); vu / vv flag the points inside the array.
// Same arithmetic as k_decomp_blk's forward direction.
template <typename A, int VEC, typename LD>
__device__ __forceinline__ void decomp_fwd_block(const DecompArgs& a, unsigned ab, unsigned bb, int64_t k2,
                                                 const bool* vu, const bool* vv, LD ld, A* mx) {
  using V = VecT<A, VEC>;
  auto srow = [&](int sl, int du, int dv) -> A* {
    const DecompSub& sb = a.subs[sl];
    const int64_t ui = ((int64_t)ab << (2 - blk_lu(sl))) + ((du - blk_su(sl)) >> blk_lu(sl));
    const int64_t vi = ((int64_t)bb << (2 - blk_lv(sl))) + ((dv - blk_sv(sl)) >> blk_lv(sl));
    return reinterpret_cast<A*>(sb.stage) + sb.base + (ui * sb.count[1] + vi) * sb.row_pad + k2;
  };
  auto lin = [](const V& p, const V& q) {
    V r;
#pragma unroll
    for (int e = 0; e < VEC; e++) r.v[e] = TAr<A>::lin(p.v[e], q.v[e]);
    return r;
  };
  // 2-grid values g[i][j] = c at (2i, 2j), i, j in 0..2
  V g[3][3];
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) ld(g[i][j], 2 * i, 2 * j);
  auto emit = [&](int sl, int du, int dv, const V& x, const V& w, bool sub) {
    V d = x;
    if (sub)
#pragma unroll
      for (int e = 0; e < VEC; e++) d.v[e] = TAr<A>::sub(d.v[e], w.v[e]);
    vst<A, VEC>(srow(sl, du, dv), d);
#pragma unroll
    for (int e = 0; e < VEC; e++) mx[sl] = fmax(mx[sl], fabs(d.v[e]));
  };
  // the per-level predictions of Alg. 1 (as in k_decomp_blk): t = 2 from the
  // 4-grid, t = 1 from the 2-grid; the v pass reads u-pass predictions
  // S1 (0,0)
  if (vu[0] && vv[0]) emit(0, 0, 0, g[0][0], g[0][0], false);
  // S2a (2,0): along u from the 4-grid
  if (vu[2] && vv[0]) emit(1, 2, 0, g[1][0], vu[4] ? lin(g[0][0], g[2][0]) : g[0][0], true);
  // S2b (0,2): u on the 4-grid, along v
  if (vu[0] && vv[2]) emit(2, 0, 2, g[0][1], vv[4] ? lin(g[0][0], g[0][2]) : g[0][0], true);
  // S2b (2,2): u pass at v = 0 and v = 4, then along v
  if (vu[2] && vv[2]) {
    const V lo = vu[4] ? lin(g[0][0], g[2][0]) : g[0][0];
    const V w = vv[4] ? lin(lo, vu[4] ? lin(g[0][2], g[2][2]) : g[0][2]) : lo;
    emit(2, 2, 2, g[1][1], w, true);
  }
  // S3 from the 2-grid (t = 1): value at 2-grid point (du, dv) even
  auto G = [&](int du, int dv) -> const V& { return g[du >> 1][dv >> 1]; };
  auto pass_u1 = [&](int du, int dv) -> V { return vu[du + 1] ? lin(G(du - 1, dv), G(du + 1, dv)) : G(du - 1, dv); };
#pragma unroll
  for (int du = 0; du < 4; du++)
#pragma unroll
    for (int dv = 0; dv < 4; dv++) {
      if (((du | dv) & 1) == 0 || !(vu[du] && vv[dv])) continue;
      V w;
      if ((dv & 1) == 0) {
        w = pass_u1(du, dv);
      } else {
        const bool uc = (du & 1) == 0;
        const V lo = uc ? G(du, dv - 1) : pass_u1(du, dv - 1);
        if (!vv[dv + 1]) w = lo;
        else w = lin(lo, uc ? G(du, dv + 1) : pass_u1(du, dv + 1));
      }
      V x;
      ld(x, du, dv);
      emit(blk_slot(du, dv), du, dv, x, w, true);
    }
}

// Decomposition only (same values as k_decomp_blk's forward direction):
// the 2-grid of the block's neighbourhood stays in registers while S1/S2 are
// written, then each S3 point is loaded and predicted on its own, so fewer
// vectors are live at once and more CTAs fit on an SM.
template <typename A, int VEC>
__device__ __forceinline__ void decomp_fwd_body(const DecompArgs& a, unsigned item) {
  using V = VecT<A, VEC>;
  const unsigned nvec = (unsigned)a.ntiles[2], nbb = (unsigned)a.ntiles[1], nab = (unsigned)a.ntiles[0];
  const unsigned iv = item % nvec + (unsigned)a.tlo[2], rest = item / nvec;
  const unsigned bb = rest % nbb + (unsigned)a.tlo[1], ab = rest / nbb + (unsigned)a.tlo[0];
  const bool live = rest / nbb < nab;
  const int cu = (int)a.cnt[0], cv = (int)a.cnt[1];
  const int64_t cw = a.cnt[2], pw = a.pitch ? a.pitch : cw;
  const int u0 = 4 * (int)ab, v0 = 4 * (int)bb;
  const int64_t k2 = (int64_t)iv * VEC;
  const A* __restrict__ comp = reinterpret_cast<const A*>(a.comp);
  bool vu[5], vv[5];
#pragma unroll
  for (int d = 0; d < 5; d++) {
    vu[d] = live && u0 + d < cu;
    vv[d] = live && v0 + d < cv;
  }
  auto ld = [&](V& r, int du, int dv) {
    if (vu[du] && vv[dv]) vld<A, VEC>(r, comp + ((int64_t)(u0 + du) * cv + (v0 + dv)) * pw + k2);
    else
#pragma unroll
      for (int e = 0; e < VEC; e++) r.v[e] = A(0);
  };
  A mx[5] = {A(0), A(0), A(0), A(0), A(0)};
  decomp_fwd_block<A, VEC>(a, ab, bb, k2, vu, vv, ld, mx);
#pragma unroll
  for (int q = 0; q < 5; q++) push_max(a.subs[q].vmax, TAr<A>::mag(mx[q]), sizeof(A));
}

template <typename A, int VEC>
__global__ void __launch_bounds__(128, 6) k_decomp_fwd(DecompArgs a) {
  decomp_fwd_body<A, VEC>(a, blockIdx.x * blockDim.x + threadIdx.x);
}

// the forward decomposition of several regions in one launch: item i owns
// blocks first[i] .. first[i + 1] - 1
constexpr int kMaxDecompFwdBatch = 40;
struct DecompBatch {
  int n;
  int64_t first[kMaxDecompFwdBatch + 1];
  DecompArgs a[kMaxDecompFwdBatch];
};
static_assert(sizeof(DecompBatch) <= 32764, "kernel parameter block");

template <typename A, int VEC>
__global__ void __launch_bounds__(128, 6) k_decomp_fwd_multi(const __grid_constant__ DecompBatch b) {
  const int i = batch_find(b.first, b.n);
  decomp_fwd_body<A, VEC>(b.a[i], (blockIdx.x - (unsigned)b.first[i]) * blockDim.x + threadIdx.x);
}

// ---------------------------------------------------------------------------
// Forward decomposition with TMA-staged tiles (FP32, slices normal to the
// fastest axis, rows a multiple of 4 values).  A persistent CTA walks tiles
// of 16 x 16 in-slice points x 32 points along the normal; each tile and its
// next 4-grid lines (17 x 17 x 32 values) arrive in shared memory by one
// cp.async.bulk.tensor copy, completed on an mbarrier, while the previous
// tile is decomposed (two stages).  One thread per (4 x 4 block, normal
// point): reads its 5 x 5 neighbourhood from shared memory (a warp = 32
// consecutive normal points: conflict-free) and writes its 16 values to the
// sub-level rows (a warp writes 128 contiguous bytes per row).  Waits are
// bounded: on a timeout the CTA records it in *a.err, waits (bounded) for
// the copy it still has in flight and returns.
// ---------------------------------------------------------------------------
constexpr int kDtU = 16, kDtV = 16, kDtW = 32;
constexpr int kDtBox = (kDtU + 1) * (kDtV + 1) * kDtW;          // floats per stage
constexpr int kDtSmem = 2 * kDtBox * 4 + 64 + 128;              // two stages + two mbarriers + alignment
constexpr int kDtSpin = 1 << 22;                                // bounded mbarrier polls

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }


__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < kDtSpin; i++) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
  }
  return false;
}

// Tile sources of the kernel below: one region (Dt1), or the regions of a
// batch of fields (DtBatch: item i owns tiles first[i] .. first[i + 1] - 1).
struct Dt1 {
  const CUtensorMap* tm;
  const DecompArgs* a;
  int ntu, ntv, ntw;
  __device__ int item(int) const { return 0; }
  __device__ int first(int) const { return 0; }
  __device__ const CUtensorMap* map(int) const { return tm; }
  __device__ const DecompArgs& args(int) const { return *a; }
  __device__ int nv(int) const { return ntv; }
  __device__ int nw(int) const { return ntw; }
};

constexpr int kMaxDecompBatch = 32;
struct DecompTmaBatch {
  CUtensorMap tm[kMaxDecompBatch];
  DecompArgs a[kMaxDecompBatch];
  int n;
  int first[kMaxDecompBatch + 1];
  int ntv[kMaxDecompBatch], ntw[kMaxDecompBatch];
};

struct DtBatch {
  const DecompTmaBatch* b;
  __device__ int item(int t) const {
    int i = 0;
    while (i + 1 < b->n && t >= b->first[i + 1]) i++;
    return i;
  }
  __device__ int first(int i) const { return b->first[i]; }
  __device__ const CUtensorMap* map(int i) const { return &b->tm[i]; }
  __device__ const DecompArgs& args(int i) const { return b->a[i]; }
  __device__ int nv(int i) const { return b->ntv[i]; }
  __device__ int nw(int i) const { return b->ntw[i]; }
};

template <class S>
__device__ __forceinline__ void decomp_tma_body(const S& src, int ntiles) {
  extern __shared__ __align__(128) float dsm_raw[];
  // stages on 128-byte boundaries (tensor copies land there)
  float* dsm = dsm_raw + ((128 - (smem_u32(dsm_raw) & 127)) & 127) / 4;
  uint64_t* bars = reinterpret_cast<uint64_t*>(dsm + 2 * kDtBox);
  const int tid = threadIdx.x;
  if ((int)blockIdx.x >= ntiles) return;
  const uint32_t bar0 = smem_u32(&bars[0]), bar1 = smem_u32(&bars[1]);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar0) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(bar1) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  __syncthreads();
  auto issue = [&](int t, int buf) {   // thread 0
    const int it = src.item(t), lt = t - src.first(it), ntw = src.nw(it), ntv = src.nv(it);
    const int tw = lt % ntw, r = lt / ntw, tv = r % ntv, tu = r / ntv;
    const uint32_t bar = buf ? bar1 : bar0;
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(kDtBox * 4) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n"
        ::"r"(smem_u32(dsm + buf * kDtBox)), "l"(reinterpret_cast<uint64_t>(src.map(it))), "r"(tw * kDtW),
        "r"(tv * kDtV), "r"(tu * kDtU), "r"(bar)
        : "memory");
  };
  float mx[5] = {0.f, 0.f, 0.f, 0.f, 0.f};
  int cur = src.item(blockIdx.x);   // item whose maxima mx holds
  uint32_t par = 0;                 // bit b: phase of stage b's next completion
  int buf = 0;
  if (tid == 0) issue(blockIdx.x, 0);
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x, buf ^= 1) {
    const int tn = t + gridDim.x;
    if (tid == 0 && tn < ntiles) issue(tn, buf ^ 1);   // that stage was released by the last barrier
    const bool ok = mbar_wait(buf ? bar1 : bar0, (par >> buf) & 1);
    if (__syncthreads_or(!ok)) {   // the whole CTA gives up together
      if (tid == 0) atomicExch(src.args(cur).err, 1);
      if (tn < ntiles) mbar_wait(buf ? bar0 : bar1, (par >> (buf ^ 1)) & 1);
      return;
    }
    par ^= 1u << buf;
    const int it = src.item(t);
    if (it != cur) {   // the maxima so far belong to the previous item
#pragma unroll
      for (int q = 0; q < 5; q++) {
        push_max(src.args(cur).subs[q].vmax, TAr<float>::mag(mx[q]), 4);
        mx[q] = 0.f;
      }
      cur = it;
    }
    const DecompArgs& a = src.args(it);
    const int lt = t - src.first(it), ntw = src.nw(it), ntv = src.nv(it);
    const int tw = lt % ntw, r = lt / ntw, tv = r % ntv, tu = r / ntv;
    const int cu = (int)a.cnt[0], cv = (int)a.cnt[1];
    const int64_t cw = a.cnt[2];
    const float* st = dsm + buf * kDtBox;
#pragma unroll
    for (int k = 0; k < 2; k++) {
      const int i = tid + 256 * k;
      const int w = i & 31, blk = i >> 5;
      const int ub = (blk >> 2) * 4, vb = (blk & 3) * 4;
      const int U0 = tu * kDtU + ub, V0 = tv * kDtV + vb;
      const int64_t W = (int64_t)tw * kDtW + w;
      const bool live = U0 < cu && V0 < cv && W < cw;
      bool vu[5], vv[5];
#pragma unroll
      for (int d = 0; d < 5; d++) {
        vu[d] = live && U0 + d < cu;
        vv[d] = live && V0 + d < cv;
      }
      auto ld = [&](VecT<float, 1>& rv, int du, int dv) {
        rv.v[0] = st[((ub + du) * (kDtV + 1) + (vb + dv)) * kDtW + w];
      };
      if (live) decomp_fwd_block<float, 1>(a, (unsigned)(U0 >> 2), (unsigned)(V0 >> 2), W, vu, vv, ld, mx);
    }
    __syncthreads();   // every read of this stage done: it may be refilled
  }
#pragma unroll
  for (int q = 0; q < 5; q++) push_max(src.args(cur).subs[q].vmax, TAr<float>::mag(mx[q]), 4);
}

__global__ void __launch_bounds__(256, 2) k_decomp_tma(const __grid_constant__ CUtensorMap tm,
                                                       const __grid_constant__ DecompArgs a, int ntu, int ntv,
                                                       int ntw) {
  decomp_tma_body(Dt1{&tm, &a, ntu, ntv, ntw}, ntu * ntv * ntw);
}

__global__ void __launch_bounds__(256, 2) k_decomp_tma_multi(const __grid_constant__ DecompTmaBatch b) {
  decomp_tma_body(DtBatch{&b}, b.first[b.n]);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library)
static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  });
  return fn;
}

// the TMA form applies to a whole array, FP32, slices normal to the fastest
// axis, 16-byte row strides and a tensor map the driver accepts
static bool decomp_tma_applies(const DecompArgs& a) {
  const int64_t pw = a.pitch ? a.pitch : a.cnt[2];
  return !a.retrieve && a.n == 2 && a.bhi[0] == 0 && pw % 4 == 0 && a.err && ((uintptr_t)a.comp & 15) == 0;
}

// tensor map of a region's compact array: boxes of kDtW x (kDtV + 1) x
// (kDtU + 1) values, zero fill beyond the array
static bool decomp_tensor_map(const DecompArgs& a, CUtensorMap& tm) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const int64_t cu = a.cnt[0], cv = a.cnt[1], cw = a.cnt[2], pw = a.pitch ? a.pitch : cw;
  const cuuint64_t gdim[3] = {(cuuint64_t)cw, (cuuint64_t)cv, (cuuint64_t)cu};
  const cuuint64_t gstride[2] = {(cuuint64_t)pw * 4, (cuuint64_t)(pw * cv) * 4};
  const cuuint32_t box[3] = {kDtW, kDtV + 1, kDtU + 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, a.comp, gdim, gstride, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// resident CTAs of the TMA kernels on this device (both forms take the same
// shared memory and registers per CTA)
static int decomp_tma_grid_cap() {
  static int grid_cache[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  int& per_dev = grid_cache[dev & 63];
  if (per_dev == 0) {
    int sms = 0, per = 0, per_m = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_decomp_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, kDtSmem);
    cudaFuncSetAttribute(k_decomp_tma_multi, cudaFuncAttributeMaxDynamicSharedMemorySize, kDtSmem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_decomp_tma, 256, kDtSmem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_m, k_decomp_tma_multi, 256, kDtSmem);
    per_dev = std::max(1, sms * std::max(std::min(per, per_m), 1));
  }
  return per_dev;
}

static bool run_decomp_tma(const DecompArgs& a, cudaStream_t s) {
  if (!decomp_tma_applies(a)) return false;
  const int64_t cu = a.cnt[0], cv = a.cnt[1], cw = a.cnt[2];
  if (cu <= 0 || cv <= 0 || cw <= 0) return true;   // nothing to do
  CUtensorMap tm;
  if (!decomp_tensor_map(a, tm)) return false;
  const int ntu = (int)((cu + kDtU - 1) / kDtU), ntv = (int)((cv + kDtV - 1) / kDtV),
            ntw = (int)((cw + kDtW - 1) / kDtW);
  const int64_t ntiles = (int64_t)ntu * ntv * ntw;
  const int grid = (int)std::min<int64_t>(ntiles, decomp_tma_grid_cap());
  count_launch();
  k_decomp_tma<<<grid, 256, kDtSmem, s>>>(tm, a, ntu, ntv, ntw);
  return true;
}

// several regions (of one field or of a batch's fields) in shared TMA
// launches; items the TMA form does not take go one by one
static void run_decomp_tma_multi(const DecompArgs* das, int n, cudaStream_t s, std::vector<int>& rest) {
  std::vector<int> tk;
  for (int k = 0; k < n; k++) {
    if (decomp_tma_applies(das[k])) tk.push_back(k);
    else rest.push_back(k);
  }
  if (tk.size() == 1) {
    if (!run_decomp_tma(das[tk[0]], s)) rest.push_back(tk[0]);
    return;
  }
  static_assert(sizeof(DecompTmaBatch) <= 32764, "kernel parameter block");
  size_t k = 0;
  while (k < tk.size()) {
    DecompTmaBatch b{};
    int tot = 0;
    for (; k < tk.size() && b.n < kMaxDecompBatch; k++) {
      const DecompArgs& a = das[tk[k]];
      const int64_t cu = a.cnt[0], cv = a.cnt[1], cw = a.cnt[2];
      if (cu <= 0 || cv <= 0 || cw <= 0) continue;
      if (!decomp_tensor_map(a, b.tm[b.n])) {
        rest.push_back(tk[k]);
        continue;
      }
      const int ntu = (int)((cu + kDtU - 1) / kDtU), ntv = (int)((cv + kDtV - 1) / kDtV),
                ntw = (int)((cw + kDtW - 1) / kDtW);
      b.a[b.n] = a;
      b.first[b.n] = tot;
      b.ntv[b.n] = ntv;
      b.ntw[b.n] = ntw;
      b.n++;
      tot += ntu * ntv * ntw;
    }
    b.first[b.n] = tot;
    if (!tot) continue;
    count_launch();
    k_decomp_tma_multi<<<std::min(tot, decomp_tma_grid_cap()), 256, kDtSmem, s>>>(b);
  }
}


// max |c| over a region's compact array (level-0 rounding term)
// running maximum of |c|: floating point in the value type, fixed point as
// an unsigned magnitude
template <typename A> struct MaxAbs {
  using T = A;
  __device__ static T upd(T m, A c) { return fmax(m, fabs(c)); }
  __device__ static unsigned long long bits(T m) { return TAr<A>::mag(m); }
};
template <> struct MaxAbs<float> {
  using T = float;
  __device__ static T upd(T m, float c) { return fmaxf(m, fabsf(c)); }
  __device__ static unsigned long long bits(T m) { return TAr<float>::mag(m); }
};
template <> struct MaxAbs<int64_t> {
  using T = unsigned long long;
  __device__ static T upd(T m, int64_t c) {
    const T g = TAr<int64_t>::mag(c);
    return g > m ? g : m;
  }
  __device__ static unsigned long long bits(T m) { return m; }
};

// ---------------------------------------------------------------------------
// level-0 per-level interpolation, 3-D, pass order (0, 1, 2): plane marching
// ---------------------------------------------------------------------------
// Alg. 1 (per-level) at level 0 predicts region 1 (odd i0, even i1, even i2)
// along axis 0 from the coarse grid, region 2 (odd i1, even i2) along axis 1
// and region 3 (odd i2) along axis 2, each pass reading the earlier passes'
// predictions.  Passes 2 and 3 stay inside one plane i0, and pass 1 reads
// only the coarse points (even i0, i1, i2) of planes i0 +- 1, +- 3.  One CTA
// owns a T1 x T2 column of the field and a chunk of planes, and walks the
// planes in order:
//   ring  : coarse values of the last four even planes over the column and
//           its halo (the inputs of pass 1)
//   Pe/Po : the current plane's values at even / odd i2 (tile + halo rows;
//           even i2 values are replaced by predictions as the passes run)
// The next plane's inputs (refactor: field rows and the coarse plane the
// ring needs next; retrieve: decoded coefficients of every point) are
// fetched into registers while the current plane's passes run.
// Refactor: c = x - W is stored to each region's staging as it is computed.
// Retrieve: the plane's reconstruction W + c_hat (coarse points: the ring)
// is assembled in Xo and written back with full-row vector stores.
// Region staging offsets use the level-0 lattices of this pass order:
// region 1 starts (1,0,0) step (2,2,2), region 2 (0,1,0) step (1,2,2),
// region 3 (0,0,1) step (1,1,2) (checked by the launcher).
// Arithmetic: the 1-D rules of the general tile kernel (same expressions).
// TMA (refactor): the field rows of a plane (tile + halo, PR x (T2 + 8)
// values, zero beyond the field) arrive in shared memory by one
// cp.async.bulk.tensor copy issued by thread 0 and completed on an mbarrier;
// two stages, so plane i0 + 2 is in flight while plane i0 is processed and
// plane i0 + 1 waits.  Waits are bounded: on a timeout the CTA records it in
// the field statistics, waits (bounded) for its other copy and returns.
template <typename A, int DEG, bool RET, bool IPR, int T1, int T2, bool TMA = false>
__device__ __forceinline__ void level0_march_body(const TileArgs& a, int zc, unsigned bid,
                                                  const CUtensorMap* tm = nullptr, int* err = nullptr,
                                                  const CUtensorMap* tmr = nullptr) {
  constexpr int NT = 256;
  constexpr int HR = DEG - 1;            // reach beyond the tile along i1, i2
  constexpr int PR = T1 + 2 * HR + 1;    // Pe rows: i1 in [b1 - HR, b1 + T1 + HR]
  constexpr int CE = T2 / 2 + DEG;       // even i2 in [b2 - HR, b2 + T2 + HR]
  constexpr int PAD = (HR / 2) & 1;      // Pe column pad: 16-byte vectors land on aligned pairs
  constexpr int CEP = (CE + PAD + 3) & ~3;
  constexpr int CR = T1 / 2 + DEG;       // even i1 rows of the ring
  constexpr int CO = T2 / 2;             // odd i2 in the tile (a power of two)
  constexpr int VEC = 16 / sizeof(A);
  constexpr int XL = 4;                  // loaded rows start 4 points before the tile (16-byte aligned)
  constexpr int NV = (T2 + 2 * XL) / VEC;
  constexpr int NLV = (PR * NV + NT - 1) / NT;        // plane vectors per thread
  constexpr int N1 = (CR * CE + NT - 1) / NT;         // ring / pass-1 points per thread
  constexpr int N2 = ((T1 / 2) * CE + NT - 1) / NT;   // pass-2 points per thread
  // FP32 cubic refactor: pass 2 in pairs of even columns (2k-1, 2k),
  // k = 1..CE/2, with column 0 alone: K2 items per row (the retrieval
  // measured faster with single points here)
  constexpr bool PAIR2 = sizeof(A) == 4 && DEG == 3 && !RET;
  constexpr int K2 = (CE + 1) / 2;
  constexpr int N2P = ((T1 / 2) * K2 + NT - 1) / NT;
  constexpr int N2V = PAIR2 ? 2 * N2P : N2;              // pass-2 values per thread
  constexpr int N3 = (T1 * CO) / NT;                  // pass-3 points per thread
  static_assert((T1 * CO) % NT == 0 && (CO & (CO - 1)) == 0, "tile shape");

  __shared__ __align__(16) A Pe[PR][CEP];
  __shared__ __align__(16) A Po[RET ? 1 : T1][CO];
  __shared__ __align__(16) A ring[4][CR][CE];
  // retrieve: the reconstructed plane, even columns of a tile row in
  // [0, T2 / 2), odd ones in [T2 / 2, T2) (conflict-free column writes)
  __shared__ __align__(16) A Xo[RET ? T1 : 1][RET ? T2 : 4];

  const int m0 = (int)a.m[0], m1 = (int)a.m[1], m2 = (int)a.m[2];
  const int64_t s0 = a.stride[0], s1 = a.stride[1];
  const unsigned nt2 = (unsigned)a.ntiles[2], nt1 = (unsigned)a.ntiles[1];
  const int b2 = (int)(bid % nt2 + a.tlo[2]) * T2;
  bid /= nt2;
  const int b1 = (int)(bid % nt1 + a.tlo[1]) * T1;
  const int z0 = (int)a.tlo[0] + (int)(bid / nt1) * zc;          // even
  const int z1 = min(z0 + zc, a.bhi[0] ? (int)a.bhi[0] : m0);
  const A* __restrict__ src = reinterpret_cast<const A*>(a.src);
  A* __restrict__ dst = reinterpret_cast<A*>(a.dst);
  const int tid = threadIdx.x;

  // TMA stages (dynamic shared memory, 128-byte aligned) and their mbarriers.
  // Refactor: a stage holds one plane's field rows (PR x XW values from
  // (b2 - XL, b1 - HR)); two stages.  Retrieve: a stage holds one plane's
  // c_hat boxes of the three regions' staging arrays -- region 1 (odd planes)
  // CR x W12 values from compact (b2 / 2 - 4, (b1 - HR) / 2), region 2
  // T1 / 2 x W12 from (b2 / 2 - 4, b1 / 2), region 3 T1 x T2 / 2 from
  // (b2 / 2, b1) -- zero beyond each array; two stages.
  constexpr int XW = T2 + 2 * XL;                                    // staged row length (refactor)
  constexpr int W12 = T2 / 2 + 8;                                    // region 1 / 2 box row (retrieve)
  constexpr int R1B = (CR * W12 * (int)sizeof(A) + 127) / 128 * 128;
  constexpr int R2B = ((T1 / 2) * W12 * (int)sizeof(A) + 127) / 128 * 128;
  constexpr int R3B = (T1 * (T2 / 2) * (int)sizeof(A) + 127) / 128 * 128;
  constexpr int SST = RET ? R1B + R2B + R3B : (PR * XW * (int)sizeof(A) + 127) / 128 * 128;   // bytes per stage
  constexpr int NSTG = 2;   // (three stages for the retrieval measured no faster)
  // retrieval with the coarse ring from the fixed-point 2-grid (tmr set):
  // each even plane's ring words (CR x RW from 2-grid column (b2 - HR) / 2
  // rounded down to even, a 16-byte boundary) arrive by one tensor copy
  // into a buffer after the mbarriers, with an mbarrier of its own
  constexpr int RW = T2 / 2 + 8;
  [[maybe_unused]] const bool rtma = TMA && RET && !std::is_same<A, int64_t>::value && tmr != nullptr;
  [[maybe_unused]] unsigned char* stg = nullptr;
  [[maybe_unused]] uint32_t barb = 0, par = 0, rbar = 0, rpar = 0;
  [[maybe_unused]] const int64_t* rbuf = nullptr;
  if constexpr (TMA) {
    extern __shared__ __align__(128) unsigned char march_dyn[];
    stg = march_dyn + ((128 - (smem_u32(march_dyn) & 127)) & 127);
    barb = smem_u32(stg + NSTG * SST);
    rbar = barb + 8 * NSTG;
    rbuf = reinterpret_cast<const int64_t*>(stg + NSTG * SST + 128);
    if (tid == 0) {
      for (int k = 0; k < NSTG + (rtma ? 1 : 0); k++)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(barb + 8 * k) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
  }
  [[maybe_unused]] auto tma3 = [&](const unsigned char* dst, const CUtensorMap* map, int x, int y, int z, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];\n"
        ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
        : "memory");
  };
  // thread 0: plane p's inputs into stage sl
  [[maybe_unused]] auto issue = [&](int p, int sl) {
    const uint32_t bar = barb + 8 * sl;
    unsigned char* d = stg + sl * SST;
    if constexpr (RET) {
      const bool o = p & 1;
      const int bytes = ((o ? CR : 0) * W12 + (T1 / 2) * W12 + T1 * (T2 / 2)) * (int)sizeof(A);
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
      if (o) tma3(d, tm, (b2 >> 1) - 4, (b1 - HR) >> 1, p >> 1, bar);
      tma3(d + R1B, tm + 1, (b2 >> 1) - 4, b1 >> 1, p, bar);
      tma3(d + R1B + R2B, tm + 2, b2 >> 1, b1, p, bar);
    } else {
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(PR * XW * (int)sizeof(A))
                   : "memory");
      tma3(d, tm, b2 - XL, b1 - HR, p, bar);
    }
  };
  const int rx = ((b2 - HR) >> 1) & ~1;           // ring box: first 2-grid column (even)
  const int ro = ((b2 - HR) >> 1) - rx;           // ... and the ring's offset in it (0 or 1)
  // thread 0: the ring words of even plane p into the ring buffer
  [[maybe_unused]] auto issue_ring = [&](int p) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(rbar), "r"(CR * RW * 8) : "memory");
    tma3(reinterpret_cast<const unsigned char*>(rbuf), tmr, rx, (b1 - HR) >> 1, p >> 1, rbar);
  };

  A* __restrict__ g1 = reinterpret_cast<A*>(a.reg[0].stage);
  A* __restrict__ g2 = reinterpret_cast<A*>(a.reg[1].stage);
  A* __restrict__ g3 = reinterpret_cast<A*>(a.reg[2].stage);
  const int64_t rp1 = a.reg[0].row_pad, rp2 = a.reg[1].row_pad, rp3 = a.reg[2].row_pad;
  auto base1 = [&](int i0) { return a.reg[0].base + (int64_t)(i0 >> 1) * a.reg[0].count[1] * rp1; };
  auto base2 = [&](int i0) { return a.reg[1].base + (int64_t)i0 * a.reg[1].count[1] * rp2; };
  auto base3 = [&](int i0) { return a.reg[2].base + (int64_t)i0 * a.reg[2].count[1] * rp3; };
  using MX = MaxAbs<A>;
  typename MX::T mx1 = 0, mx2 = 0, mx3 = 0;
  // refactor of a field's level 0: its statistics as the planes arrive
  // (minimum, maximum, and a sum of x - x that turns NaN at the first
  // non-finite value), kept per thread in shared memory: the kernel is
  // register-bound
  constexpr bool STATS = !RET && !std::is_same<A, int64_t>::value;
  __shared__ A sst[3][STATS ? NT : 1];
  const bool st_on = STATS && a.stats != nullptr;
  if constexpr (STATS) {
    if (st_on) {
      sst[0][tid] = A(INFINITY);
      sst[1][tid] = A(-INFINITY);
      sst[2][tid] = A(0);
    }
  }

  // point sets of the passes (thread-strided)
  auto p1pt = [&](int it, int& ci, int& cj, int& r, int& c) {
    const int i = tid + NT * it;
    ci = i / CE;
    cj = i - ci * CE;
    r = b1 - HR + 2 * ci;
    c = b2 - HR + 2 * cj;
    return i < CR * CE;
  };
  auto p2pt = [&](int it, int& ri, int& cj, int& r, int& c) {
    const int i = tid + NT * it;
    ri = i / CE;
    cj = i - ri * CE;
    r = b1 + 1 + 2 * ri;
    c = b2 - HR + 2 * cj;
    return i < (T1 / 2) * CE;
  };
  // pair item: column cj (and cj + 1 when pair), row r; false past the end
  auto p2pair = [&](int it, int& ri, int& cj, int& r, int& c, bool& pair) {
    const int i = tid + NT * it;
    ri = i / K2;
    const int k = i - ri * K2;
    pair = k > 0;
    cj = pair ? 2 * k - 1 : 0;
    r = b1 + 1 + 2 * ri;
    c = b2 - HR + 2 * cj;
    return i < (T1 / 2) * K2;
  };
  auto p3pt = [&](int it, int& ri, int& oj, int& r, int& c) {
    const int i = tid + NT * it;
    ri = i / CO;
    oj = i & (CO - 1);
    r = b1 + ri;
    c = b2 + 1 + 2 * oj;
  };
  // FP32 cubic: pass 3 takes pairs of adjacent odd columns (c, c + 2), which
  // share their even neighbours and whose coefficients are adjacent
  constexpr bool PAIR = sizeof(A) == 4 && DEG == 3;
  static_assert(!PAIR || (N3 % 2 == 0), "pairs");
  auto p3pair = [&](int pi, int& ri, int& oj, int& r, int& c) {
    const int q = tid + NT * pi;
    ri = q / (CO / 2);
    oj = 2 * (q & (CO / 2 - 1));
    r = b1 + ri;
    c = b2 + 1 + 2 * oj;
  };
  auto in_tile = [&](int r, int c) { return r >= b1 && r < b1 + T1 && c >= b2 && c < b2 + T2; };

  // ---- prefetch registers
  A rg[N1];                     // coarse values of one even plane (ring points)
  VecT<A, VEC> pv[RET || TMA ? 1 : NLV] = {};   // refactor: field rows of one plane
  [[maybe_unused]] const A* cur = nullptr;   // TMA: the stage holding the current plane
  // vector `it` of the current plane (registers, or the TMA stage)
  auto plane_vec = [&](int it) -> VecT<A, VEC> {
    if constexpr (TMA) {
      const int i = tid + NT * it;
      const int pr = i / NV, v = i - pr * NV;
      return *reinterpret_cast<const VecT<A, VEC>*>(cur + pr * XW + v * VEC);
    } else if constexpr (!RET) {
      return pv[it];
    } else {
      return VecT<A, VEC>{};
    }
  };
  A h1[RET && !TMA ? N1 : 1], h2[RET && !TMA ? N2V : 1], h3[RET && !TMA ? N3 : 1];   // retrieve: c_hat of one plane

  // retrieval: coarse values from the fixed-point 2-grid (rounded as the
  // coarse-point pass rounds them), else from the output.  The fixed-point
  // words stay in registers until the ring store, so the loads remain in
  // flight across the plane's passes.
  constexpr bool FIXR = RET && !std::is_same<A, int64_t>::value;
  [[maybe_unused]] const int64_t* __restrict__ cfix = FIXR ? a.cfix : nullptr;
  [[maybe_unused]] const A csc = FIXR ? A(a.cscale) : A(0);
  [[maybe_unused]] int64_t rgx[FIXR ? N1 : 1];
  const int64_t nc1 = (m1 - 1) / 2 + 1, nc2 = (m2 - 1) / 2 + 1;
  auto fetch_ring = [&](int p) {
#pragma unroll
    for (int it = 0; it < N1; it++) {
      int ci, cj, r, c;
      const bool ok = p1pt(it, ci, cj, r, c) && p >= 0 && p < m0 && r >= 0 && r < m1 && c >= 0 && c < m2;
      if constexpr (FIXR) {
        if (cfix) {
          rgx[it] = ok ? cfix[((int64_t)(p >> 1) * nc1 + (r >> 1)) * nc2 + (c >> 1)] : 0;
          continue;
        }
      }
      rg[it] = ok ? src[(int64_t)p * s0 + (int64_t)r * s1 + c] : A(0);
    }
  };
  auto store_ring = [&](int p) {
    if (p < 0 || p >= m0) return;
    A(*rs)[CE] = ring[(p >> 1) & 3];
#pragma unroll
    for (int it = 0; it < N1; it++) {
      int ci, cj, r, c;
      if (!p1pt(it, ci, cj, r, c)) continue;
      if constexpr (FIXR) {
        if (cfix) {
          rs[ci][cj] = from_fix<A>(rgx[it], csc);   // 0 outside the grid
          continue;
        }
      }
      rs[ci][cj] = rg[it];
    }
  };
  auto fetch_plane = [&](int i0) {
    if constexpr (!TMA) {
#pragma unroll
      for (int it = 0; it < NLV; it++) {
        const int i = tid + NT * it;
        const int pr = i / NV, v = i - pr * NV;
        const int r = b1 - HR + pr, c0 = b2 - XL + v * VEC;
        const bool need = i < PR * NV && ((pr >= HR && pr < HR + T1) || !(r & 1)) && r >= 0 && r < m1 && i0 < m0;
        if (need && c0 >= 0 && c0 + VEC <= m2) {
          const A* gp = src + (int64_t)i0 * s0 + (int64_t)r * s1 + c0;
          vld<A, VEC>(pv[it], gp);
        } else {
#pragma unroll
          for (int k = 0; k < VEC; k++) {
            const int c = c0 + k;
            pv[it].v[k] = (need && c >= 0 && c < m2) ? src[(int64_t)i0 * s0 + (int64_t)r * s1 + c] : A(0);
          }
        }
      }
    }
  };
  auto plane_stats = [&]() {   // the in-tile values of the plane in pv
    A lo = sst[0][tid], hi = sst[1][tid], nz = sst[2][tid];
    // min / max ignore NaN; nz = fma(x, 0, nz) stays 0 while every x is finite
    auto take = [&](A x) {
      if constexpr (std::is_same<A, float>::value) {
        lo = fminf(lo, x);
        hi = fmaxf(hi, x);
        nz = __fmaf_rn(x, 0.0f, nz);
      } else if constexpr (std::is_same<A, double>::value) {
        lo = fmin(lo, x);
        hi = fmax(hi, x);
        nz = __fma_rn(x, 0.0, nz);
      }
    };
#pragma unroll
    for (int it = 0; it < NLV; it++) {
      const int i = tid + NT * it;
      const int pr = i / NV, v = i - pr * NV;
      if (i >= PR * NV || pr < HR || pr >= HR + T1 || b1 - HR + pr >= m1) continue;
      const int c0 = b2 - XL + v * VEC;
      if (c0 < b2 || c0 >= b2 + T2) continue;   // vectors lie wholly inside or outside the tile's columns
      const VecT<A, VEC> x = plane_vec(it);
      if (c0 + VEC <= m2) {
#pragma unroll
        for (int k = 0; k < VEC; k++) take(x.v[k]);
      } else {
#pragma unroll
        for (int k = 0; k < VEC; k++)
          if (c0 + k < m2) take(x.v[k]);
      }
    }
    sst[0][tid] = lo;
    sst[1][tid] = hi;
    sst[2][tid] = nz;
  };
  auto store_plane = [&]() {
    if constexpr (STATS) {
      if (st_on) plane_stats();
    }
#pragma unroll
    for (int it = 0; it < NLV; it++) {
      const int i = tid + NT * it;
      const int pr = i / NV, v = i - pr * NV;
      if (i >= PR * NV) continue;
      const int r = b1 - HR + pr;
      const bool rows = pr >= HR && pr < HR + T1;
      if (!rows && (r & 1)) continue;
      const VecT<A, VEC> x = plane_vec(it);
      // element k sits at i2 = b2 - XL + VEC v + k: even k -> Pe, odd k -> Po
      if constexpr (VEC == 4) {
        const int ce = 2 * v - (XL - HR) / 2 + PAD;   // Pe column of element 0 (element 2: ce + 1)
        if (ce >= 0 && ce + 1 < CE + PAD) {
          *reinterpret_cast<float2*>(&Pe[pr][ce]) = make_float2(x.v[0], x.v[2]);
        } else {
          if (ce >= PAD && ce < CE + PAD) Pe[pr][ce] = x.v[0];
          if (ce + 1 >= PAD && ce + 1 < CE + PAD) Pe[pr][ce + 1] = x.v[2];
        }
        const int co = 2 * v - XL / 2;                 // Po column of element 1 (element 3: co + 1)
        if (rows && co >= 0 && co + 1 < CO) *reinterpret_cast<float2*>(&Po[pr - HR][co]) = make_float2(x.v[1], x.v[3]);
      } else {
        const int ce = v - (XL - HR) / 2 + PAD;       // element 0 (even)
        if (ce >= PAD && ce < CE + PAD) Pe[pr][ce] = x.v[0];
        const int co = v - XL / 2;                    // element 1 (odd)
        if (rows && co >= 0 && co < CO) Po[pr - HR][co] = x.v[1];
      }
    }
  };
  auto fetch_chat = [&](int i0) {
    if constexpr (!TMA) {
      if (i0 >= z1) return;
      if (i0 & 1) {
        const int64_t B1 = base1(i0);
#pragma unroll
        for (int it = 0; it < N1; it++) {
          int ci, cj, r, c;
          // per-region retrieval rebuilds halo points too: their c_hat as well
          const bool ok = p1pt(it, ci, cj, r, c) && (IPR || in_tile(r, c)) && r >= 0 && c >= 0 && r < m1 && c < m2;
          h1[it] = ok ? g1[B1 + (int64_t)(r >> 1) * rp1 + (c >> 1)] : A(0);
        }
      }
      const int64_t B2 = base2(i0), B3 = base3(i0);
      if constexpr (PAIR2) {
#pragma unroll
        for (int it = 0; it < N2P; it++) {
          int ri, cj, r, c;
          bool pair;
          float2 t = make_float2(0.0f, 0.0f);
          // pairs inside the tile: both points (c + 2 < m2 when c < m2)
          if (p2pair(it, ri, cj, r, c, pair) && pair && in_tile(r, c) && in_tile(r, c + 2) && r < m1 && c < m2)
            t = *reinterpret_cast<const float2*>(g2 + B2 + (int64_t)(r >> 1) * rp2 + (c >> 1));
          h2[2 * it] = t.x;
          h2[2 * it + 1] = t.y;
        }
      } else {
#pragma unroll
        for (int it = 0; it < N2; it++) {
          int ri, cj, r, c;
          const bool ok = p2pt(it, ri, cj, r, c) && (IPR || in_tile(r, c)) && r >= 0 && c >= 0 && r < m1 && c < m2;
          h2[it] = ok ? g2[B2 + (int64_t)(r >> 1) * rp2 + (c >> 1)] : A(0);
        }
      }
      if constexpr (PAIR) {
#pragma unroll
        for (int pi = 0; pi < N3 / 2; pi++) {
          int ri, oj, r, c;
          p3pair(pi, ri, oj, r, c);
          float2 t = make_float2(0.0f, 0.0f);
          if (r < m1 && c < m2) t = *reinterpret_cast<const float2*>(g3 + B3 + (int64_t)r * rp3 + (c >> 1));
          h3[2 * pi] = t.x;
          h3[2 * pi + 1] = t.y;
        }
      } else {
#pragma unroll
        for (int it = 0; it < N3; it++) {
          int ri, oj, r, c;
          p3pt(it, ri, oj, r, c);
          const bool ok = r < m1 && c < m2;
          h3[it] = ok ? g3[B3 + (int64_t)r * rp3 + (c >> 1)] : A(0);
        }
      }
    }
  };

  // warm-up: the ring holds planes z0 - 2, z0, z0 + 2 before the first odd
  // plane; the first plane's inputs are in registers
  fetch_ring(z0 - 2);
  store_ring(z0 - 2);
  fetch_ring(z0);
  store_ring(z0);
  fetch_ring(z0 + 2);
  store_ring(z0 + 2);
  int slot = 0;   // TMA: the stage of the current plane
  if constexpr (TMA) {
    if (tid == 0)
      for (int k = 0; k < NSTG && z0 + k < z1; k++) issue(z0 + k, k);
  } else if (!RET) {
    fetch_plane(z0);
  } else {
    fetch_chat(z0);
  }

  for (int i0 = z0; i0 < z1; i0++) {
    const bool odd = i0 & 1;
    if constexpr (TMA) {   // this plane's inputs have landed in stage `slot`
      const bool ok = mbar_wait(barb + 8 * slot, (par >> slot) & 1);
      if (__syncthreads_or(!ok)) {   // the whole CTA gives up together
        if (tid == 0) {
          atomicExch(err, 1);
          for (int k = 1; k < NSTG && i0 + k < z1; k++) {   // the copies still in flight
            const int s2 = (slot + k) % NSTG;
            mbar_wait(barb + 8 * s2, (par >> s2) & 1);
          }
          if (rtma && odd && i0 + 3 < m0) mbar_wait(rbar, rpar);   // the ring copy issued on plane i0 - 1
        }
        return;
      }
      par ^= 1u << slot;
      cur = reinterpret_cast<const A*>(stg + slot * SST);
    }
    // registers (or the TMA stage) -> shared memory: this plane's rows, and
    // (odd planes) the coarse plane i0 + 3 (the slot of plane i0 - 5)
    if (!RET) store_plane();
    if (rtma) {
      if (odd && i0 + 3 < m0) {   // ring words of plane i0 + 3 (issued on plane i0 - 1)
        const bool rok = mbar_wait(rbar, rpar);
        if (__syncthreads_or(!rok)) {
          if (tid == 0) {
            atomicExch(err, 1);
            for (int k = 1; k < NSTG && i0 + k < z1; k++) {
              const int s2 = (slot + k) % NSTG;
              mbar_wait(barb + 8 * s2, (par >> s2) & 1);
            }
          }
          return;
        }
        rpar ^= 1u;
        if constexpr (!std::is_same<A, int64_t>::value) {
          A(*rs)[CE] = ring[((i0 + 3) >> 1) & 3];
#pragma unroll
          for (int it = 0; it < N1; it++) {
            int ci, cj, r, c;
            if (p1pt(it, ci, cj, r, c)) rs[ci][cj] = from_fix<A>(rbuf[ci * RW + cj + ro], csc);   // 0 beyond the grid
          }
        }
      }
    } else if (odd) {
      store_ring(i0 + 3);
    }
    A c1[RET && !TMA ? N1 : 1], c2[RET && !TMA ? N2V : 1], c3[RET && !TMA ? N3 : 1];
    if (RET && !TMA) {
#pragma unroll
      for (int it = 0; it < N1; it++) c1[it] = h1[it];
#pragma unroll
      for (int it = 0; it < N2V; it++) c2[it] = h2[it];
#pragma unroll
      for (int it = 0; it < N3; it++) c3[it] = h3[it];
    }
    // c_hat of pass-1 item (ci, cj), pass-2 item (ri, cj), pass-3 point
    // (ri, oj): registers, or the regions' boxes in the TMA stage
    [[maybe_unused]] const A *sb1 = nullptr, *sb2 = nullptr, *sb3 = nullptr;
    if constexpr (TMA && RET) {
      sb1 = cur;
      sb2 = reinterpret_cast<const A*>(reinterpret_cast<const unsigned char*>(cur) + R1B);
      sb3 = reinterpret_cast<const A*>(reinterpret_cast<const unsigned char*>(cur) + R1B + R2B);
    }
    [[maybe_unused]] auto chat1 = [&](int it, int ci, int cj) -> A {
      if constexpr (TMA && RET) return sb1[ci * W12 + cj - HR / 2 + 4];
      else return c1[it];
    };
    [[maybe_unused]] auto chat2 = [&](int it, int ri, int cj) -> A {
      if constexpr (TMA && RET) return sb2[ri * W12 + cj - HR / 2 + 4];
      else return c2[it];
    };
    [[maybe_unused]] auto chat3 = [&](int it, int ri, int oj) -> A {
      if constexpr (TMA && RET) return sb3[ri * (T2 / 2) + oj];
      else return c3[it];
    };
    __syncthreads();
    // TMA refactor: the stage just read takes plane i0 + 2
    if constexpr (TMA && !RET) {
      if (tid == 0 && i0 + 2 < z1) issue(i0 + 2, slot);
    }
    // the next plane's inputs, in flight during this plane's passes
    if (i0 + 1 < z1) {
      if constexpr (!TMA) {
        if (!RET) fetch_plane(i0 + 1);
        else fetch_chat(i0 + 1);
      }
      if (rtma) {
        if (!odd && i0 + 4 < m0 && tid == 0) issue_ring(i0 + 4);   // needed by plane i0 + 1
      } else if (!odd) {
        fetch_ring(i0 + 4);               // needed by plane i0 + 1
      }
    }
    if (!odd && RET) {
      // even plane: the coarse points are the reconstruction already
      const A(*rs)[CE] = ring[(i0 >> 1) & 3];
#pragma unroll
      for (int it = 0; it < N1; it++) {
        int ci, cj, r, c;
        if (!p1pt(it, ci, cj, r, c)) continue;
        Pe[2 * ci][cj + PAD] = rs[ci][cj];
        if (in_tile(r, c)) Xo[r - b1][(c - b2) >> 1] = rs[ci][cj];
      }
      __syncthreads();
    }
    if (odd) {
      // pass 1 along axis 0 over the even (i1, i2) points of tile + halo
      const int64_t B1 = base1(i0);
      const int sm3 = ((i0 - 3) >> 1) & 3, sm1 = ((i0 - 1) >> 1) & 3, sp1 = ((i0 + 1) >> 1) & 3,
                sp3 = ((i0 + 3) >> 1) & 3;
      const bool fast = DEG == 3 && i0 >= 3 && i0 + 3 < m0;
#pragma unroll
      for (int it = 0; it < N1; it++) {
        int ci, cj, r, c;
        if (!p1pt(it, ci, cj, r, c) || r < 0 || r >= m1 || c < 0 || c >= m2) continue;
        A W;
        if (fast) {
          W = TAr<A>::cub(ring[sm3][ci][cj], ring[sm1][ci][cj], ring[sp1][ci][cj], ring[sp3][ci][cj]);
        } else {
          auto at = [&](int p) -> A { return ring[(p >> 1) & 3][ci][cj]; };
          W = rule<A>(i0, m0, DEG, at);
        }
        if (in_tile(r, c)) {
          if (!RET) {
            const A cv = TAr<A>::sub(Pe[2 * ci][cj + PAD], W);
            g1[B1 + (int64_t)(r >> 1) * rp1 + (c >> 1)] = cv;
            mx1 = MX::upd(mx1, cv);
          } else {
            Xo[r - b1][(c - b2) >> 1] = TAr<A>::add(W, chat1(it, ci, cj));
          }
        }
        // later passes read predictions (per-level), or originals /
        // reconstructed values (per-region refactor / retrieval)
        if (!IPR) Pe[2 * ci][cj + PAD] = W;
        else if (RET) Pe[2 * ci][cj + PAD] = TAr<A>::add(W, chat1(it, ci, cj));
      }
      __syncthreads();
    }
    // pass 2 along axis 1: odd i1 in the tile, even i2 over tile + halo
    if constexpr (PAIR2) {
      const int64_t B2 = base2(i0);
#pragma unroll
      for (int it = 0; it < N2P; it++) {
        int ri, cj, r, c;
        bool pair;
        if (!p2pair(it, ri, cj, r, c, pair) || r >= m1 || c < 0 || c >= m2) continue;
        const int pr = r - (b1 - HR);
        const int pc = cj + PAD;
        if (!pair) {   // column 0: the left halo column alone
          A W;
          if (r >= 3 && r + 3 < m1) {
            W = TAr<A>::cub(Pe[pr - 3][pc], Pe[pr - 1][pc], Pe[pr + 1][pc], Pe[pr + 3][pc]);
          } else {
            auto at = [&](int k) -> A { return Pe[pr + (k - r)][pc]; };
            W = rule<A>(r, m1, DEG, at);
          }
          if (!IPR) Pe[pr][pc] = W;
          continue;
        }
        float2 W;   // columns pc, pc + 1 (pc even)
        if (r >= 3 && r + 3 < m1) {
          const float2 a3 = *reinterpret_cast<const float2*>(&Pe[pr - 3][pc]);
          const float2 a1 = *reinterpret_cast<const float2*>(&Pe[pr - 1][pc]);
          const float2 p1 = *reinterpret_cast<const float2*>(&Pe[pr + 1][pc]);
          const float2 p3 = *reinterpret_cast<const float2*>(&Pe[pr + 3][pc]);
          W.x = TAr<A>::cub(a3.x, a1.x, p1.x, p3.x);
          W.y = TAr<A>::cub(a3.y, a1.y, p1.y, p3.y);
        } else {
          auto at0 = [&](int k) -> A { return Pe[pr + (k - r)][pc]; };
          auto at1 = [&](int k) -> A { return Pe[pr + (k - r)][pc + 1]; };
          W.x = rule<A>(r, m1, DEG, at0);
          W.y = rule<A>(r, m1, DEG, at1);
        }
        if (in_tile(r, c) && in_tile(r, c + 2)) {
          if (!RET) {
            const float2 x = *reinterpret_cast<const float2*>(&Pe[pr][pc]);
            const A c0v = TAr<A>::sub(x.x, W.x), c1v = TAr<A>::sub(x.y, W.y);
            *reinterpret_cast<float2*>(g2 + B2 + (int64_t)(r >> 1) * rp2 + (c >> 1)) = make_float2(c0v, c1v);
            mx2 = MX::upd(MX::upd(mx2, c0v), c1v);
          }
        }
        if (!IPR) *reinterpret_cast<float2*>(&Pe[pr][pc]) = W;
      }
    } else {
      const int64_t B2 = base2(i0);
#pragma unroll
      for (int it = 0; it < N2; it++) {
        int ri, cj, r, c;
        if (!p2pt(it, ri, cj, r, c) || r >= m1 || c < 0 || c >= m2) continue;
        const int pr = r - (b1 - HR);
        A W;
        if (DEG == 3 && r >= 3 && r + 3 < m1) {
          W = TAr<A>::cub(Pe[pr - 3][cj + PAD], Pe[pr - 1][cj + PAD], Pe[pr + 1][cj + PAD], Pe[pr + 3][cj + PAD]);
        } else {
          auto at = [&](int k) -> A { return Pe[pr + (k - r)][cj + PAD]; };
          W = rule<A>(r, m1, DEG, at);
        }
        if (c >= b2 && c < b2 + T2) {
          if (!RET) {
            const A cv = TAr<A>::sub(Pe[pr][cj + PAD], W);
            g2[B2 + (int64_t)(r >> 1) * rp2 + (c >> 1)] = cv;
            mx2 = MX::upd(mx2, cv);
          } else {
            Xo[r - b1][(c - b2) >> 1] = TAr<A>::add(W, chat2(it, ri, cj));
          }
        }
        if (!IPR) Pe[pr][cj + PAD] = W;
        else if (RET) Pe[pr][cj + PAD] = TAr<A>::add(W, chat2(it, ri, cj));
      }
    }
    __syncthreads();
    // pass 3 along axis 2: odd i2 of the tile rows
    if constexpr (PAIR) {
      const int64_t B3 = base3(i0);
#pragma unroll
      for (int pi = 0; pi < N3 / 2; pi++) {
        int ri, oj, r, c;
        p3pair(pi, ri, oj, r, c);
        if (r >= m1 || c >= m2) continue;   // c + 2 < m2 too: m2 is a multiple of 4
        const int pr = ri + HR;
        const int cj = oj + HR / 2 + PAD;   // Pe column of c - 1 (even)
        A W0, W1;
        if (c >= 3 && c + 5 < m2) {
          const A e0 = Pe[pr][cj - 1];
          const float2 e12 = *reinterpret_cast<const float2*>(&Pe[pr][cj]);
          const float2 e34 = *reinterpret_cast<const float2*>(&Pe[pr][cj + 2]);
          W0 = TAr<A>::cub(e0, e12.x, e12.y, e34.x);
          W1 = TAr<A>::cub(e12.x, e12.y, e34.x, e34.y);
        } else {
          auto at0 = [&](int k) -> A { return Pe[pr][cj + ((k - (c - 1)) >> 1)]; };
          auto at1 = [&](int k) -> A { return Pe[pr][cj + 1 + ((k - (c + 1)) >> 1)]; };
          W0 = rule<A>(c, m2, DEG, at0);
          W1 = rule<A>(c + 2, m2, DEG, at1);
        }
        if (!RET) {
          const float2 x = *reinterpret_cast<const float2*>(&Po[ri][oj]);
          const A c0v = TAr<A>::sub(x.x, W0), c1v = TAr<A>::sub(x.y, W1);
          *reinterpret_cast<float2*>(g3 + B3 + (int64_t)r * rp3 + (c >> 1)) = make_float2(c0v, c1v);
          mx3 = MX::upd(MX::upd(mx3, c0v), c1v);
        } else {
          A h0, h1v;
          if constexpr (TMA && RET) {   // adjacent in the region-3 box
            const float2 t = *reinterpret_cast<const float2*>(&sb3[ri * (T2 / 2) + oj]);
            h0 = t.x;
            h1v = t.y;
          } else {
            h0 = c3[2 * pi];
            h1v = c3[2 * pi + 1];
          }
          *reinterpret_cast<float2*>(&Xo[ri][T2 / 2 + oj]) = make_float2(TAr<A>::add(W0, h0), TAr<A>::add(W1, h1v));
        }
      }
    } else {
      const int64_t B3 = base3(i0);
#pragma unroll
      for (int it = 0; it < N3; it++) {
        int ri, oj, r, c;
        p3pt(it, ri, oj, r, c);
        if (r >= m1 || c >= m2) continue;
        const int pr = ri + HR;
        const int cj = oj + HR / 2 + PAD;           // Pe column of c - 1
        A W;
        if (DEG == 3 && c >= 3 && c + 3 < m2) {
          W = TAr<A>::cub(Pe[pr][cj - 1], Pe[pr][cj], Pe[pr][cj + 1], Pe[pr][cj + 2]);
        } else {
          auto at = [&](int k) -> A { return Pe[pr][cj + ((k - (c - 1)) >> 1)]; };
          W = rule<A>(c, m2, DEG, at);
        }
        if (!RET) {
          const A cv = TAr<A>::sub(Po[ri][oj], W);
          g3[B3 + (int64_t)r * rp3 + (c >> 1)] = cv;
          mx3 = MX::upd(mx3, cv);
        } else {
          Xo[ri][T2 / 2 + oj] = TAr<A>::add(W, chat3(it, ri, oj));
        }
      }
    }
    if (RET) {
      __syncthreads();
      // TMA retrieve: the passes are done with this stage; it takes plane
      // i0 + NSTG
      if constexpr (TMA && RET) {
        if (tid == 0 && i0 + NSTG < z1) issue(i0 + NSTG, slot);
      }
      // full tile rows of the reconstructed plane
      for (int i = tid; i < T1 * (T2 / VEC); i += NT) {
        const int ri = i / (T2 / VEC), v = i - ri * (T2 / VEC);
        const int r = b1 + ri, c0 = b2 + v * VEC;
        if (r >= m1) continue;
        A* gp = dst + (int64_t)i0 * s0 + (int64_t)r * s1 + c0;
        VecT<A, VEC> xv;   // interleave the even and odd halves
        if constexpr (VEC == 4) {
          const float2 e = *reinterpret_cast<const float2*>(&Xo[ri][2 * v]);
          const float2 o = *reinterpret_cast<const float2*>(&Xo[ri][T2 / 2 + 2 * v]);
          xv.v[0] = e.x;
          xv.v[1] = o.x;
          xv.v[2] = e.y;
          xv.v[3] = o.y;
        } else {
          xv.v[0] = Xo[ri][v];
          xv.v[1] = Xo[ri][T2 / 2 + v];
        }
        if (c0 + VEC <= m2) vst<A, VEC>(gp, xv);
        else
          for (int k = 0; k < VEC && c0 + k < m2; k++) gp[k] = xv.v[k];
      }
    }
    __syncthreads();
    if constexpr (TMA) slot = slot + 1 == NSTG ? 0 : slot + 1;
  }
  if constexpr (STATS) {
    if (st_on) {
      const A nz = sst[2][tid];
      stats_push_block(a.stats, (double)sst[0][tid], (double)sst[1][tid], nz != A(0));
    }
  }
  if (!RET) {
    const unsigned long long m[3] = {MX::bits(mx1), MX::bits(mx2), MX::bits(mx3)};
#pragma unroll
    for (int r = 0; r < 3; r++) {
      if (a.reg[r].vmax_double) push_max_double<A>(a.reg[r].vmax, m[r]);
      else push_max(a.reg[r].vmax, m[r], sizeof(A));
    }
  }
}

template <typename A, int DEG, bool RET, bool IPR, int T1, int T2>
__global__ void __launch_bounds__(256, 4) k_level0_march(TileArgs a, int zc) {
  level0_march_body<A, DEG, RET, IPR, T1, T2>(a, zc, blockIdx.x);
}

// refactor with TMA-staged field rows (tm: the field, boxes of
// (T2 + 8) x (T1 + 2 (DEG - 1) + 1) x 1 values)
template <typename A, int DEG, bool IPR, int T1, int T2>
__global__ void __launch_bounds__(256, 4) k_level0_march_tma(const __grid_constant__ CUtensorMap tm,
                                                             const __grid_constant__ TileArgs a, int zc) {
  level0_march_body<A, DEG, false, IPR, T1, T2, true>(a, zc, blockIdx.x, &tm, a.err);
}

// a bounded wait of a retrieval kernel gave up (read and cleared by
// read_device_timeouts)
__device__ int g_dev_timeout = 0;

// tensor maps of the three level-0 regions' staging arrays and (ring set)
// of the fixed-point 2-grid the coarse ring comes from
struct MarchMaps {
  CUtensorMap m[4];
  int ring;
};

// retrieval with TMA-staged c_hat boxes (mm: regions 1, 2, 3)
template <typename A, int DEG, bool IPR, int T1, int T2>
__global__ void __launch_bounds__(256, 4) k_level0_march_tma_ret(const __grid_constant__ MarchMaps mm,
                                                                 const __grid_constant__ TileArgs a, int zc) {
  level0_march_body<A, DEG, true, IPR, T1, T2, true>(a, zc, blockIdx.x, mm.m, a.err ? a.err : &g_dev_timeout,
                                                     mm.ring ? &mm.m[3] : nullptr);
}

int read_device_timeouts(bool clear) {
  int v = 0;
  if (cudaMemcpyFromSymbol(&v, g_dev_timeout, sizeof(int)) != cudaSuccess) return -1;
  if (clear && v) {
    const int z = 0;
    cudaMemcpyToSymbol(g_dev_timeout, &z, sizeof(int));
  }
  return v;
}

// the plane-marching kernel over several fields (or fixed-point levels) in
// one launch: item i owns blocks first[i] .. first[i + 1] - 1
struct MarchBatch {
  int n;
  int64_t first[kMaxTileBatch + 1];
  int zc[kMaxTileBatch];
  TileArgs args[kMaxTileBatch];
};
static_assert(sizeof(MarchBatch) <= 32764 && sizeof(TileBatch) <= 32764, "kernel parameter block");

template <typename A, int DEG, bool RET, bool IPR, int T1, int T2>
__global__ void __launch_bounds__(256, 4) k_level0_march_multi(const __grid_constant__ MarchBatch b) {
  const int i = batch_find(b.first, b.n);
  level0_march_body<A, DEG, RET, IPR, T1, T2>(b.args[i], b.zc[i], blockIdx.x - (unsigned)b.first[i]);
}

// the TMA-staged refactor over several fields (or fixed-point levels) in one
// launch: item i owns blocks first[i] .. first[i + 1] - 1 and reads its
// field through tm[i]
constexpr int kMaxMarchTmaBatch = 40;
struct MarchTmaBatch {
  CUtensorMap tm[kMaxMarchTmaBatch];
  int n;
  int64_t first[kMaxMarchTmaBatch + 1];
  int zc[kMaxMarchTmaBatch];
  TileArgs args[kMaxMarchTmaBatch];
};
static_assert(sizeof(MarchTmaBatch) <= 32764, "kernel parameter block");

template <typename A, int DEG, bool IPR, int T1, int T2>
__global__ void __launch_bounds__(256, 4) k_level0_march_tma_multi(const __grid_constant__ MarchTmaBatch b) {
  const int i = batch_find(b.first, b.n);
  level0_march_body<A, DEG, false, IPR, T1, T2, true>(b.args[i], b.zc[i], blockIdx.x - (unsigned)b.first[i], &b.tm[i],
                                                      b.args[i].err);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename A, int T0, int T1, int T2, int H0, int H>
static void run_tile(const TileArgs& a0, cudaStream_t s) {
  TileArgs a = a0;
  const int64_t T[3] = {T0, T1, T2};
  for (int k = 0; k < 3; k++) {   // tiles covering the box (or the grid)
    const int64_t lo = a.bhi[0] ? a.blo[k] : 0, hi = a.bhi[0] ? a.bhi[k] : a.m[k];
    a.tlo[k] = lo / T[k];
    a.ntiles[k] = hi > lo ? (hi + T[k] - 1) / T[k] - a.tlo[k] : 0;
  }
  if (!a.ntiles[0] || !a.ntiles[1] || !a.ntiles[2]) return;
  count_launch();
  const size_t smem = sizeof(A) * (T0 + 2 * H0) * (T1 + 2 * H) * (T2 + 8);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tile_interp<A, T0, T1, T2, H0, H>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  const int64_t nb = a.ntiles[0] * a.ntiles[1] * a.ntiles[2];
  k_tile_interp<A, T0, T1, T2, H0, H><<<(unsigned)nb, 256, smem, s>>>(a);
}

// independent grids of one kernel shape in as few launches as the batch
// parameter block allows
template <typename A, int T0, int T1, int T2, int H0, int H>
static void run_tile_multi(const std::vector<TileArgs>& v, cudaStream_t s) {
  const size_t smem = sizeof(A) * (T0 + 2 * H0) * (T1 + 2 * H) * (T2 + 8);
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tile_interp_multi<A, T0, T1, T2, H0, H>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    attr = true;
  }
  const int64_t T[3] = {T0, T1, T2};
  size_t k = 0;
  while (k < v.size()) {
    TileBatch b{};
    int64_t tot = 0;
    for (; k < v.size() && b.n < kMaxTileBatch; k++) {
      TileArgs a = v[k];
      int64_t nb = 1;
      for (int q = 0; q < 3; q++) {
        const int64_t lo = a.bhi[0] ? a.blo[q] : 0, hi = a.bhi[0] ? a.bhi[q] : a.m[q];
        a.tlo[q] = lo / T[q];
        a.ntiles[q] = hi > lo ? (hi + T[q] - 1) / T[q] - a.tlo[q] : 0;
        nb *= a.ntiles[q];
      }
      if (!nb) continue;
      b.first[b.n] = tot;
      b.args[b.n++] = a;
      tot += nb;
    }
    b.first[b.n] = tot;
    if (!tot) continue;
    count_launch();
    k_tile_interp_multi<A, T0, T1, T2, H0, H><<<(unsigned)tot, 256, smem, s>>>(b);
  }
}

// a retrieval of level 0 whose coarse points are still in fixed point: the
// tile kernels read them from the output, so they go there first
template <typename A>
static void coarse_into_output(const TileArgs& a, cudaStream_t s) {
  if constexpr (!std::is_same<A, int64_t>::value) {
    if (!a.retrieve || !a.cfix) return;
    FieldD f{};
    for (int k = 0; k < 3; k++) {
      f.n[k] = a.m[k];
      f.nc[k] = a.m[k] > 1 ? (a.m[k] - 1) / 2 + 1 : 1;
    }
    launch_coarse_out(sizeof(A) == 4 ? VK_F32 : VK_F64, f, a.cfix, a.cscale, a.dst, s);
  }
}

template <typename A>
static void run_tile_kind_multi(const std::vector<TileArgs>& all, cudaStream_t s) {
  std::vector<TileArgs> g[2][2];   // [3-D][cubic]
  for (const TileArgs& a : all) {
    coarse_into_output<A>(a, s);
    g[a.m[0] > 1][a.degree == 3].push_back(a);
  }
  constexpr bool wide = sizeof(A) == 4;
  if (!g[1][1].empty()) {
    if (wide) run_tile_multi<A, 8, 8, 64, 3, 3>(g[1][1], s); else run_tile_multi<A, 4, 4, 64, 3, 3>(g[1][1], s);
  }
  if (!g[1][0].empty()) {
    if (wide) run_tile_multi<A, 8, 8, 64, 1, 1>(g[1][0], s); else run_tile_multi<A, 4, 4, 64, 1, 1>(g[1][0], s);
  }
  if (!g[0][1].empty()) run_tile_multi<A, 1, 32, 64, 0, 3>(g[0][1], s);
  if (!g[0][0].empty()) run_tile_multi<A, 1, 32, 64, 0, 1>(g[0][0], s);
}

template <typename A>
static void run_tile_kind(const TileArgs& a, cudaStream_t s) {
  coarse_into_output<A>(a, s);
  const bool is3 = a.m[0] > 1;
  const bool cubic = a.degree == 3;
  constexpr bool wide = sizeof(A) == 4;
  if (is3) {
    if (cubic) {
      if (wide) run_tile<A, 8, 8, 64, 3, 3>(a, s); else run_tile<A, 4, 4, 64, 3, 3>(a, s);
    } else {
      if (wide) run_tile<A, 8, 8, 64, 1, 1>(a, s); else run_tile<A, 4, 4, 64, 1, 1>(a, s);
    }
  } else {
    if (cubic) run_tile<A, 1, 32, 64, 0, 3>(a, s); else run_tile<A, 1, 32, 64, 0, 1>(a, s);
  }
}

// schedule choice: the marching kernel with TMA-staged field rows and the
// default plane chunking (refactor levels whose statistics it takes; the
// register-prefetch form elsewhere)
constexpr int kMarchTma = -2;
// the same on 16 x 64 columns (FP32 levels; other value kinds: kMarchTma)
constexpr int kMarchTmaNarrow = -3;

// grid of the plane-marching kernel for one level: column tiles covering the
// box (or the grid) and chunks of zc planes; returns the block count (0:
// nothing to do) with a.ntiles / a.tlo set
template <int T1, int T2>
static int64_t march_grid(TileArgs& a, int zc_force, int& zc_out) {
  const bool box = a.bhi[0] != 0;
  const int64_t T[3] = {1, T1, T2};
  for (int k = 1; k < 3; k++) {
    const int64_t lo = box ? a.blo[k] : 0, hi = box ? a.bhi[k] : a.m[k];
    a.tlo[k] = lo / T[k];
    a.ntiles[k] = hi > lo ? (hi + T[k] - 1) / T[k] - a.tlo[k] : 0;
  }
  // planes [z_lo, z_end): chunks start on even planes (the ring holds even
  // planes)
  const int64_t zlo = box ? (a.blo[0] & ~int64_t(1)) : 0, zend = box ? a.bhi[0] : a.m[0];
  a.tlo[0] = zlo;
  if (zend <= zlo || !a.ntiles[1] || !a.ntiles[2]) return 0;
  // plane chunks (default): about eight full waves of 4 CTAs per SM, so the
  // last wave is not a sparse tail; at least 8 planes so the ring warm-up
  // (three coarse-plane loads) stays a small share of a chunk
  const int64_t cols = a.ntiles[1] * a.ntiles[2];
  int64_t zc;
  if (zc_force > 0) {
    zc = zc_force;
  } else {
    const int64_t want = (148 * 4 * 8 + cols - 1) / cols;
    zc = (zend - zlo + want - 1) / want;
    zc = std::max<int64_t>(8, (zc + 1) & ~int64_t(1));
  }
  a.ntiles[0] = (zend - zlo + zc - 1) / zc;
  zc_out = (int)zc;
  return a.ntiles[0] * cols;
}

// tensor map of the field for the TMA form of the marching kernel: boxes of
// (T2 + 8) x rows x 1 values, zero fill beyond the field (the launcher's
// contiguity and 16-byte row checks make the strides legal)
template <typename A>
static bool march_tensor_map(const TileArgs& a, int T2, int rows, CUtensorMap& tm) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  const CUtensorMapDataType dt = std::is_same<A, float>::value    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : std::is_same<A, double>::value ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                                                  : CU_TENSOR_MAP_DATA_TYPE_INT64;
  const cuuint64_t gdim[3] = {(cuuint64_t)a.m[2], (cuuint64_t)a.m[1], (cuuint64_t)a.m[0]};
  const cuuint64_t gstride[2] = {(cuuint64_t)a.stride[1] * sizeof(A), (cuuint64_t)a.stride[0] * sizeof(A)};
  const cuuint32_t box[3] = {(cuuint32_t)(T2 + 8), (cuuint32_t)rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(&tm, dt, 3, const_cast<void*>(a.src), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the TMA form: refactor of a level with a timeout flag to report a bounded
// wait that gives up, field base 16-byte aligned (march_applies)
template <typename A, int DEG, bool PR, int T1, int T2>
static bool run_level0_march_tma(const TileArgs& a0, cudaStream_t s, int zc_force) {
  if (a0.retrieve || !a0.err) return false;
  constexpr int ROWS = T1 + 2 * (DEG - 1) + 1;
  constexpr int SST = (ROWS * (T2 + 8) * (int)sizeof(A) + 127) / 128 * 128;
  constexpr int SMEM = 2 * SST + 128 + 16;
  CUtensorMap tm;
  if (!march_tensor_map<A>(a0, T2, ROWS, tm)) return false;
  TileArgs a = a0;
  int zc = 0;
  const int64_t nb = march_grid<T1, T2>(a, zc_force, zc);
  if (!nb) return true;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_level0_march_tma<A, DEG, PR, T1, T2>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
    cudaFuncSetAttribute(k_level0_march_tma<A, DEG, PR, T1, T2>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    attr = true;
  }
  count_launch();
  k_level0_march_tma<A, DEG, PR, T1, T2><<<(unsigned)nb, 256, SMEM, s>>>(tm, a, zc);
  return true;
}

// tensor map of one level-0 region's staging array ([count0][count1][row_pad]
// from element `base`): boxes of w x rows x 1 values, zero fill beyond the
// region's counts; false where the array is not 16-byte aligned or pitched
template <typename A>
static bool region_tensor_map(const TileRegion& g, int w, int rows, CUtensorMap& tm) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc || !g.stage || g.count[0] <= 0 || g.count[1] <= 0 || g.count[2] <= 0) return false;
  const char* base = static_cast<const char*>(g.stage) + g.base * (int64_t)sizeof(A);
  if (((uintptr_t)base & 15) != 0 || (g.row_pad * (int64_t)sizeof(A)) % 16 != 0) return false;
  const CUtensorMapDataType dt = std::is_same<A, float>::value    ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                 : std::is_same<A, double>::value ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64
                                                                  : CU_TENSOR_MAP_DATA_TYPE_INT64;
  const cuuint64_t gdim[3] = {(cuuint64_t)g.count[2], (cuuint64_t)g.count[1], (cuuint64_t)g.count[0]};
  const cuuint64_t gstride[2] = {(cuuint64_t)(g.row_pad * (int64_t)sizeof(A)),
                                 (cuuint64_t)(g.count[1] * g.row_pad * (int64_t)sizeof(A))};
  const cuuint32_t box[3] = {(cuuint32_t)w, (cuuint32_t)rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(&tm, dt, 3, const_cast<char*>(base), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// tensor map of the fixed-point 2-grid of a level-0 retrieval (cfix; shape
// ((m - 1) / 2 + 1) per axis, row-major): boxes of w x rows x 1 words, zero
// fill beyond the grid; false where its rows are not a multiple of 16 bytes
static bool ring_tensor_map(const TileArgs& a, int w, int rows, CUtensorMap& tm) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  const int64_t nc[3] = {(a.m[0] - 1) / 2 + 1, (a.m[1] - 1) / 2 + 1, (a.m[2] - 1) / 2 + 1};
  if (!enc || ((uintptr_t)a.cfix & 15) != 0 || (nc[2] * 8) % 16 != 0) return false;
  const cuuint64_t gdim[3] = {(cuuint64_t)nc[2], (cuuint64_t)nc[1], (cuuint64_t)nc[0]};
  const cuuint64_t gstride[2] = {(cuuint64_t)(nc[2] * 8), (cuuint64_t)(nc[1] * nc[2] * 8)};
  const cuuint32_t box[3] = {(cuuint32_t)w, (cuuint32_t)rows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  return enc(&tm, CU_TENSOR_MAP_DATA_TYPE_INT64, 3, const_cast<int64_t*>(a.cfix), gdim, gstride, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the TMA form of the retrieval: every region's staging array takes a
// tensor map (the level-0 lattices of pass order (0, 1, 2): march_applies)
template <typename A, int DEG, bool PR, int T1, int T2>
static bool run_level0_march_tma_ret(const TileArgs& a0, cudaStream_t s, int zc_force) {
  constexpr int CR = T1 / 2 + DEG, W12 = T2 / 2 + 8;
  constexpr int R1B = (CR * W12 * (int)sizeof(A) + 127) / 128 * 128;
  constexpr int R2B = ((T1 / 2) * W12 * (int)sizeof(A) + 127) / 128 * 128;
  constexpr int R3B = (T1 * (T2 / 2) * (int)sizeof(A) + 127) / 128 * 128;
  constexpr int NSTG = 2;   // as in level0_march_body
  // value kinds whose ring may come from the fixed-point grid: a 128-byte
  // mbarrier block, then the ring buffer (CR x RW words)
  constexpr bool FIX = !std::is_same<A, int64_t>::value;
  constexpr int RW = T2 / 2 + 8;
  constexpr int SMEM = NSTG * (R1B + R2B + R3B) + 128 + (FIX ? 128 + CR * RW * 8 : 8 * NSTG);
  MarchMaps mm;
  if (!region_tensor_map<A>(a0.reg[0], W12, CR, mm.m[0]) || !region_tensor_map<A>(a0.reg[1], W12, T1 / 2, mm.m[1]) ||
      !region_tensor_map<A>(a0.reg[2], T2 / 2, T1, mm.m[2]))
    return false;
  mm.ring = FIX && a0.cfix && ring_tensor_map(a0, RW, CR, mm.m[3]);
  TileArgs a = a0;
  int zc = 0;
  const int64_t nb = march_grid<T1, T2>(a, zc_force, zc);
  if (!nb) return true;
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_level0_march_tma_ret<A, DEG, PR, T1, T2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         SMEM);
    cudaFuncSetAttribute(k_level0_march_tma_ret<A, DEG, PR, T1, T2>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         100);
    attr = true;
  }
  count_launch();
  k_level0_march_tma_ret<A, DEG, PR, T1, T2><<<(unsigned)nb, 256, SMEM, s>>>(mm, a, zc);
  return true;
}

template <typename A, int DEG, bool RET, bool PR, int T1, int T2>
static void run_level0_march(const TileArgs& a0, cudaStream_t s, int zc_force, bool tma = false) {
  if constexpr (!RET) {
    if (tma && run_level0_march_tma<A, DEG, PR, T1, T2>(a0, s, zc_force)) return;
  } else {
    if (tma && run_level0_march_tma_ret<A, DEG, PR, T1, T2>(a0, s, zc_force)) return;
  }
  TileArgs a = a0;
  int zc = 0;
  const int64_t nb = march_grid<T1, T2>(a, zc_force, zc);
  if (!nb) return;
  count_launch();
  static bool attr = false;
  if (!attr) {   // shared memory for several CTAs per SM
    cudaFuncSetAttribute(k_level0_march<A, DEG, RET, PR, T1, T2>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    attr = true;
  }
  k_level0_march<A, DEG, RET, PR, T1, T2><<<(unsigned)nb, 256, 0, s>>>(a, zc);
}

template <typename A, int DEG, bool RET, bool PR, int T1, int T2>
static void run_level0_march_multi_reg(const std::vector<TileArgs>& v, const std::vector<int>& zcs, cudaStream_t s);

// the TMA-staged refactor of several levels in shared launches: items whose
// schedule is kMarchTma, with a timeout flag and a tensor map the driver
// accepts; the others are returned in (rest, rest_zc)
template <typename A, int DEG, bool PR, int T1, int T2>
static void run_level0_march_tma_multi(const std::vector<TileArgs>& v, const std::vector<int>& zcs, cudaStream_t s,
                                       std::vector<TileArgs>& rest, std::vector<int>& rest_zc) {
  constexpr int ROWS = T1 + 2 * (DEG - 1) + 1;
  constexpr int SST = (ROWS * (T2 + 8) * (int)sizeof(A) + 127) / 128 * 128;
  constexpr int SMEM = 2 * SST + 128 + 16;
  static bool attr = false;
  size_t k = 0;
  while (k < v.size()) {
    MarchTmaBatch b{};
    int64_t tot = 0;
    for (; k < v.size() && b.n < kMaxMarchTmaBatch; k++) {
      TileArgs a = v[k];
      if (zcs[k] != kMarchTma || a.retrieve || !a.err || !march_tensor_map<A>(a, T2, ROWS, b.tm[b.n])) {
        rest.push_back(v[k]);
        rest_zc.push_back(zcs[k]);
        continue;
      }
      int zc = 0;
      const int64_t nb = march_grid<T1, T2>(a, zcs[k], zc);
      if (!nb) continue;
      b.first[b.n] = tot;
      b.zc[b.n] = zc;
      b.args[b.n++] = a;
      tot += nb;
    }
    b.first[b.n] = tot;
    if (!tot) continue;
    if (!attr) {
      cudaFuncSetAttribute(k_level0_march_tma_multi<A, DEG, PR, T1, T2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           SMEM);
      cudaFuncSetAttribute(k_level0_march_tma_multi<A, DEG, PR, T1, T2>,
                           cudaFuncAttributePreferredSharedMemoryCarveout, 100);
      attr = true;
    }
    count_launch();
    k_level0_march_tma_multi<A, DEG, PR, T1, T2><<<(unsigned)tot, 256, SMEM, s>>>(b);
  }
}

// levels of one marching-kernel shape (value kind, degree, direction,
// interpolation) in shared launches; zcs[i]: the plane chunk of item i
// (<= 0: the default); a single item takes the one-level kernel
template <typename A, int DEG, bool RET, bool PR, int T1, int T2>
static void run_level0_march_multi(const std::vector<TileArgs>& v, const std::vector<int>& zcs, cudaStream_t s) {
  if (v.size() == 1) {
    run_level0_march<A, DEG, RET, PR, T1, T2>(v[0], s, zcs[0], zcs[0] == kMarchTma);
    return;
  }
  if constexpr (!RET) {   // the TMA form for the items whose schedule and arrays take it
    std::vector<TileArgs> rv;
    std::vector<int> rz;
    run_level0_march_tma_multi<A, DEG, PR, T1, T2>(v, zcs, s, rv, rz);
    if (rv.size() < v.size()) {
      if (rv.size() == 1) run_level0_march<A, DEG, RET, PR, T1, T2>(rv[0], s, rz[0], false);
      else if (!rv.empty()) run_level0_march_multi_reg<A, DEG, RET, PR, T1, T2>(rv, rz, s);
      return;
    }
  }
  run_level0_march_multi_reg<A, DEG, RET, PR, T1, T2>(v, zcs, s);
}

// the register-prefetch form of several levels in shared launches
template <typename A, int DEG, bool RET, bool PR, int T1, int T2>
static void run_level0_march_multi_reg(const std::vector<TileArgs>& v, const std::vector<int>& zcs, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_level0_march_multi<A, DEG, RET, PR, T1, T2>, cudaFuncAttributePreferredSharedMemoryCarveout,
                         100);
    attr = true;
  }
  size_t k = 0;
  while (k < v.size()) {
    MarchBatch b{};
    int64_t tot = 0;
    for (; k < v.size() && b.n < kMaxTileBatch; k++) {
      TileArgs a = v[k];
      int zc = 0;
      const int64_t nb = march_grid<T1, T2>(a, zcs[k], zc);
      if (!nb) continue;
      b.first[b.n] = tot;
      b.zc[b.n] = zc;
      b.args[b.n++] = a;
      tot += nb;
    }
    b.first[b.n] = tot;
    if (!tot) continue;
    count_launch();
    k_level0_march_multi<A, DEG, RET, PR, T1, T2><<<(unsigned)tot, 256, 0, s>>>(b);
  }
}

// the plane-marching kernel covers level 0 of 3-D per-level schemes in a
// contiguous field whose rows hold whole 16-byte vectors
template <typename A>
static bool march_applies(const TileArgs& a) {
  constexpr int VEC = 16 / sizeof(A);
  // per-level, or per-region in pass order (0, 1, 2): the same region lattices
  if (a.d != 3 || a.order[0] != 0 || a.order[1] != 1 || a.order[2] != 2) return false;
  if (a.degree != 1 && a.degree != 3) return false;
  if (a.stride[2] != 1 || a.stride[1] != a.m[2] || a.stride[0] != a.m[1] * a.m[2]) return false;
  if (a.m[2] % VEC != 0 || ((uintptr_t)a.src % 16) != 0 || ((uintptr_t)a.dst % 16) != 0) return false;
  // level-0 region lattices of pass order (0, 1, 2)
  static const int64_t st[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  static const int64_t sp[3][3] = {{2, 2, 2}, {1, 2, 2}, {1, 1, 2}};
  for (int r = 0; r < 3; r++)
    for (int k = 0; k < 3; k++)
      if (a.reg[r].start[k] != st[r][k] || a.reg[r].step[k] != sp[r][k]) return false;
  return true;
}

// one level on the marching kernel with T1 x T2 columns
template <typename A, int T1, int T2>
static void march_launch_t(const TileArgs& a, cudaStream_t s, int zc, bool tma) {
  const bool pr = a.interp != 0;
  if (a.retrieve) {
    if (a.degree == 3) {
      if (pr) run_level0_march<A, 3, true, true, T1, T2>(a, s, zc, tma);
      else run_level0_march<A, 3, true, false, T1, T2>(a, s, zc, tma);
    } else {
      if (pr) run_level0_march<A, 1, true, true, T1, T2>(a, s, zc, tma);
      else run_level0_march<A, 1, true, false, T1, T2>(a, s, zc, tma);
    }
  } else {
    if (a.degree == 3) {
      if (pr) run_level0_march<A, 3, false, true, T1, T2>(a, s, zc, tma);
      else run_level0_march<A, 3, false, false, T1, T2>(a, s, zc, tma);
    } else {
      if (pr) run_level0_march<A, 1, false, true, T1, T2>(a, s, zc, tma);
      else run_level0_march<A, 1, false, false, T1, T2>(a, s, zc, tma);
    }
  }
}

// zc > 0: chunks of zc planes; otherwise the default chunking (kMarchTma:
// with TMA-staged inputs where that form applies; kMarchTmaNarrow: the same
// on 16 x 64 columns for FP32, whose default columns are 16 x 128)
template <typename A>
static void march_launch(const TileArgs& a, cudaStream_t s, int zc) {
  if constexpr (sizeof(A) == 4) {
    if (zc == kMarchTmaNarrow) {
      march_launch_t<A, 16, 64>(a, s, zc, true);
      return;
    }
  }
  march_launch_t<A, 16, sizeof(A) == 4 ? 128 : 64>(a, s, zc, zc == kMarchTma || zc == kMarchTmaNarrow);
}

// ---------------------------------------------------------------------------
// autotuner of the level-interpolation schedule
// ---------------------------------------------------------------------------
// Where the marching kernel applies, a level can also run the general tile
// kernel, and the marching kernel's plane chunk sets its grid; all choices
// compute the same values (same expression trees).  Choice 0 = general tile
// kernel, -1 = marching with the default chunking, kMarchTma (-2, the
// default) = the same with TMA-staged inputs where that form applies,
// kMarchTmaNarrow (-3) = that on 16 x 64 columns (FP32), k > 0 = marching
// with chunks of k planes.  With tuning on, the first launch of an untuned (value
// kind, direction, degree, level grid) on a stream that is not being
// captured times every candidate (CUDA events, the best of two runs after a
// warm-up) and keeps the fastest; later launches, captured ones included,
// use the table.  A level runs the same points however often it is
// repeated, so the timing runs leave the same outputs behind.
namespace {
struct TuneKey {
  int vk, ret, deg, interp;
  int64_t m0, m1, m2;
  bool operator<(const TuneKey& o) const {
    if (vk != o.vk) return vk < o.vk;
    if (ret != o.ret) return ret < o.ret;
    if (deg != o.deg) return deg < o.deg;
    if (interp != o.interp) return interp < o.interp;
    if (m0 != o.m0) return m0 < o.m0;
    if (m1 != o.m1) return m1 < o.m1;
    return m2 < o.m2;
  }
};
struct TuneVal {
  int choice;
  float ms;
};
std::mutex g_tune_mu;
std::map<TuneKey, TuneVal> g_tune;
std::atomic<int> g_tune_on{0};
constexpr int kTuneCand[] = {0, 8, 16, 32, 64, -1, kMarchTma, kMarchTmaNarrow};

template <typename A>
void run_choice(const TileArgs& a, cudaStream_t s, int choice) {
  if (choice == 0) run_tile_kind<A>(a, s);
  else march_launch<A>(a, s, choice);
}

template <typename A>
TuneVal tune(const TileArgs& a, cudaStream_t s) {
  TuneVal best{-1, -1.0f};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return best;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return best;
  }
  for (int c : kTuneCand) {
    if (c > 0 && c >= 2 * a.m[0] && c != 8) continue;   // larger chunks than the field: same grid as a smaller one
    run_choice<A>(a, s, c);                            // warm-up
    float t = 1e30f;
    for (int r = 0; r < 2; r++) {
      cudaEventRecord(e0, s);
      run_choice<A>(a, s, c);
      cudaEventRecord(e1, s);
      float ms = 0.0f;
      if (cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
        t = std::min(t, ms);
    }
    if (best.ms < 0.0f || t < best.ms) best = {c, t};
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

// the schedule of a level the marching kernel applies to (timing the
// candidates first when tuning is on and the level is untuned)
template <typename A>
int tuned_choice(int vk, const TileArgs& a, cudaStream_t s) {
  const TuneKey key{vk, a.retrieve, a.degree, a.interp, a.m[0], a.m[1], a.m[2]};
  int choice = kMarchTma;
  bool have = false;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      choice = it->second.choice;
      have = true;
    }
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (!have && !a.bhi[0] && g_tune_on.load() && cudaStreamIsCapturing(s, &cs) == cudaSuccess &&
      cs == cudaStreamCaptureStatusNone) {
    const TuneVal v = tune<A>(a, s);
    if (v.ms >= 0.0f) {
      std::lock_guard<std::mutex> lk(g_tune_mu);
      g_tune[key] = v;
      choice = v.choice;
    }
  }
  return choice;
}

template <typename A>
int launch_tuned(int vk, const TileArgs& a, cudaStream_t s) {
  if (!march_applies<A>(a)) return -1;
  run_choice<A>(a, s, tuned_choice<A>(vk, a, s));
  return 1;
}
}  // namespace

int set_autotune(int on) { return g_tune_on.exchange(on ? 1 : 0); }

// pin one entry of the table (ms recorded as 0): every later launch of that
// (value kind, direction, degree, interpolation, level grid) uses `choice`
bool autotune_pin(const int64_t* key, int choice) {
  bool known = false;
  for (int c : kTuneCand) known = known || c == choice;
  if (!known || key[0] < 0 || key[0] > 2 || key[1] < 0 || key[1] > 1 || (key[2] != 1 && key[2] != 3) ||
      key[3] < 0 || key[3] > 1)
    return false;
  const TuneKey k{(int)key[0], (int)key[1], (int)key[2], (int)key[3], key[4], key[5], key[6]};
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[k] = TuneVal{choice, 0.0f};
  return true;
}

int autotune_entries(int max_entries, int64_t* keys, int* choice, double* ms) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  int k = 0;
  for (auto& kv : g_tune) {
    if (k < max_entries) {
      const TuneKey& t = kv.first;
      if (keys) {
        const int64_t v[7] = {t.vk, t.ret, t.deg, t.interp, t.m0, t.m1, t.m2};
        for (int i = 0; i < 7; i++) keys[7 * k + i] = v[i];
      }
      if (choice) choice[k] = kv.second.choice;
      if (ms) ms[k] = kv.second.ms;
    }
    k++;
  }
  return k;
}

void clear_autotune() {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune.clear();
}

// independent grids (no grid reads another's output): those the schedule
// gives the marching kernel in shared launches per kernel shape, the rest in
// shared launches of the tile kernel
template <typename A>
static void launch_multi_kind(int vk, const TileArgs* args, int n, cudaStream_t s) {
  constexpr int T1 = 16, T2 = sizeof(A) == 4 ? 128 : 64;
  std::vector<TileArgs> rest, mv[2][2];   // marching refactor levels [cubic][per-region]
  std::vector<int> mz[2][2];
  std::vector<const void*> sx;            // statistics the tile kernel does not take
  std::vector<int64_t> sn;
  std::vector<FieldStats*> ss;
  for (int i = 0; i < n; i++) {
    const TileArgs& a = args[i];
    const int c = march_applies<A>(a) ? tuned_choice<A>(vk, a, s) : 0;
    if (c == 0) {
      if (a.stats && !a.retrieve) {
        sx.push_back(a.src);
        sn.push_back(a.m[0] * a.m[1] * a.m[2]);
        ss.push_back(a.stats);
      }
      rest.push_back(a);
    } else if (a.retrieve || (c == kMarchTmaNarrow && sizeof(A) == 4)) {
      march_launch<A>(a, s, c);
    } else {
      mv[a.degree == 3][a.interp != 0].push_back(a);
      mz[a.degree == 3][a.interp != 0].push_back(c);
    }
  }
  if (!mv[1][0].empty()) run_level0_march_multi<A, 3, false, false, T1, T2>(mv[1][0], mz[1][0], s);
  if (!mv[1][1].empty()) run_level0_march_multi<A, 3, false, true, T1, T2>(mv[1][1], mz[1][1], s);
  if (!mv[0][0].empty()) run_level0_march_multi<A, 1, false, false, T1, T2>(mv[0][0], mz[0][0], s);
  if (!mv[0][1].empty()) run_level0_march_multi<A, 1, false, true, T1, T2>(mv[0][1], mz[0][1], s);
  if (!sx.empty()) launch_minmax_multi(vk, sx.data(), sn.data(), ss.data(), (int)sx.size(), s);
  run_tile_kind_multi<A>(rest, s);
}

void launch_tile_interp_multi(int vk, const TileArgs* args, int n, cudaStream_t s) {
  if (n <= 0) return;
  if (vk == VK_F32) launch_multi_kind<float>(vk, args, n, s);
  else if (vk == VK_F64) launch_multi_kind<double>(vk, args, n, s);
  else launch_multi_kind<int64_t>(vk, args, n, s);
}

void launch_tile_interp(int vk, const TileArgs& a, cudaStream_t s) {
  int r = -1;
  if (vk == VK_F32) r = launch_tuned<float>(vk, a, s);
  else if (vk == VK_F64) r = launch_tuned<double>(vk, a, s);
  else if (vk == VK_FIX) r = launch_tuned<int64_t>(vk, a, s);   // a contiguous fixed-point level (level 1)
  if (r > 0) return;
  if (vk == VK_F32) run_tile_kind<float>(a, s);
  else if (vk == VK_F64) run_tile_kind<double>(a, s);
  else run_tile_kind<int64_t>(a, s);
}

template <typename A, int N, int T0, int T1, int T2>
static void run_decomp(const DecompArgs& a0, cudaStream_t s) {
  count_launch();
  DecompArgs a = a0;
  a.ntiles[0] = (a.cnt[0] + T0 - 1) / T0;
  a.ntiles[1] = (a.cnt[1] + T1 - 1) / T1;
  a.ntiles[2] = (a.cnt[2] + T2 - 1) / T2;
  const size_t smem = sizeof(A) * (T0 + (N != 0)) * (T1 + (N != 1)) * (T2 + (N != 2));
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tile_decomp<A, N, T0, T1, T2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    attr = true;
  }
  const int64_t nb = a.ntiles[0] * a.ntiles[1] * a.ntiles[2];
  k_tile_decomp<A, N, T0, T1, T2><<<(unsigned)nb, 256, smem, s>>>(a);
}

// 4 x 4 blocks and vectors covering the box (or the array): sets a.tlo and
// a.ntiles, returns the thread items
template <int VEC>
static int64_t decomp_blk_grid(DecompArgs& a) {
  const bool box = a.bhi[0] != 0;
  const int64_t T[3] = {4, 4, VEC};
  for (int k = 0; k < 3; k++) {
    const int64_t lo = box ? a.blo[k] : 0, hi = box ? std::min(a.bhi[k], a.cnt[k]) : a.cnt[k];
    a.tlo[k] = lo / T[k];
    a.ntiles[k] = hi > lo ? (k == 2 ? hi / T[k] + (hi % T[k] != 0) : (hi + T[k] - 1) / T[k]) - a.tlo[k] : 0;
  }
  return a.ntiles[0] * a.ntiles[1] * a.ntiles[2];
}

template <typename A, int VEC>
static void run_decomp_fwd_multi(const std::vector<DecompArgs>& v, cudaStream_t s) {
  size_t k = 0;
  while (k < v.size()) {
    DecompBatch b{};
    int64_t tot = 0;
    for (; k < v.size() && b.n < kMaxDecompFwdBatch; k++) {
      DecompArgs a = v[k];
      const int64_t items = decomp_blk_grid<VEC>(a);
      if (!items) continue;
      b.first[b.n] = tot;
      b.a[b.n++] = a;
      tot += (items + 127) / 128;
    }
    b.first[b.n] = tot;
    if (!tot) continue;
    count_launch();
    k_decomp_fwd_multi<A, VEC><<<(unsigned)tot, 128, 0, s>>>(b);
  }
}

template <typename A, int VEC>
static void run_decomp_blk(const DecompArgs& a0, cudaStream_t s) {
  DecompArgs a = a0;
  const int64_t items = decomp_blk_grid<VEC>(a);
  if (items == 0) return;
  count_launch();
  if (a.retrieve) k_decomp_blk<A, VEC><<<(unsigned)((items + 127) / 128), 128, 0, s>>>(a);
  else k_decomp_fwd<A, VEC><<<(unsigned)((items + 127) / 128), 128, 0, s>>>(a);
}

void launch_tile_decomp(int vk, const DecompArgs& a, cudaStream_t s) {
  // tiles are multiples of 4 along the in-slice axes
  if (vk == VK_F32) {
    if (a.n == 2 && run_decomp_tma(a, s)) return;   // forward, whole array, 16-byte row pitch
    if (a.n == 2 && a.cnt[2] % 4 == 0) run_decomp_blk<float, 4>(a, s);
    else if (a.n == 2) run_decomp_blk<float, 1>(a, s);
    else if (a.n == 1) run_decomp<float, 1, 16, 4, 64>(a, s);
    else run_decomp<float, 0, 4, 16, 64>(a, s);
  } else {
    if (a.n == 2 && a.cnt[2] % 2 == 0) run_decomp_blk<double, 2>(a, s);
    else if (a.n == 2) run_decomp_blk<double, 1>(a, s);
    else if (a.n == 1) run_decomp<double, 1, 16, 4, 64>(a, s);
    else run_decomp<double, 0, 4, 16, 64>(a, s);
  }
}

// forward decompositions of several regions: the TMA form's in shared
// launches, the other slices-normal-to-the-fastest-axis ones in shared
// launches per value type and vector width, the rest one by one
void launch_tile_decomp_multi(int vk, const DecompArgs* das, int n, cudaStream_t s) {
  std::vector<int> rest;
  if (vk == VK_F32) run_decomp_tma_multi(das, n, s, rest);
  else
    for (int k = 0; k < n; k++) rest.push_back(k);
  std::vector<DecompArgs> g[4];   // F32 x4, F32 x1, F64 x2, F64 x1
  std::vector<int> one;
  for (int k : rest) {
    const DecompArgs& a = das[k];
    if (a.retrieve || a.n != 2) one.push_back(k);
    else if (vk == VK_F32) g[a.cnt[2] % 4 == 0 ? 0 : 1].push_back(a);   // whole vectors per row
    else g[a.cnt[2] % 2 == 0 ? 2 : 3].push_back(a);
  }
  for (int q = 0; q < 4; q++) {
    if (g[q].size() == 1) {
      launch_tile_decomp(vk, g[q][0], s);
    } else if (!g[q].empty()) {
      if (q == 0) run_decomp_fwd_multi<float, 4>(g[q], s);
      else if (q == 1) run_decomp_fwd_multi<float, 1>(g[q], s);
      else if (q == 2) run_decomp_fwd_multi<double, 2>(g[q], s);
      else run_decomp_fwd_multi<double, 1>(g[q], s);
    }
  }
  for (int k : one) launch_tile_decomp(vk, das[k], s);
}

// the row padding of many lattices (any value kinds) zeroed in one launch:
// item i owns blocks first[i] .. first[i + 1] - 1 and writes 32-bit words
constexpr int kMaxPadItems = 512;
struct PadItem {
  uint32_t* p;         // first padding word of the lattice's first row
  int64_t rows;        // rows of the lattice
  int64_t row_words;   // words from one row's padding to the next
  int64_t padw;        // padding words per row
};
struct PadBatch {
  int n;
  int64_t first[kMaxPadItems + 1];
  PadItem it[kMaxPadItems];
};

__global__ void __launch_bounds__(256) k_zero_pads_multi(const __grid_constant__ PadBatch b) {
  const int lo = batch_find(b.first, b.n);
  const PadItem& t = b.it[lo];
  const int64_t n = t.rows * t.padw;
  const int64_t nblk = b.first[lo + 1] - b.first[lo];
  for (int64_t e = (blockIdx.x - b.first[lo]) * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += nblk * (int64_t)blockDim.x) {
    const int64_t r = e / t.padw, c = e % t.padw;
    t.p[r * t.row_words + c] = 0u;
  }
}

void launch_zero_pads_multi(const int* vks, const LatD* lats, void* const* stages, int n, cudaStream_t s) {
  static_assert(sizeof(PadBatch) <= 32764, "kernel parameter block");
  int k = 0;
  while (k < n) {
    PadBatch b{};
    int64_t tot = 0;
    for (; k < n && b.n < kMaxPadItems; k++) {
      const LatD& l = lats[k];
      const int w = vks[k] == VK_F32 ? 1 : 2;
      const int64_t padw = (l.row_pad - l.count[2]) * w, rows = l.count[0] * l.count[1];
      if (padw <= 0 || rows <= 0) continue;
      const int64_t blocks = std::min<int64_t>((rows * padw + 255) / 256, 148 * 4);
      b.first[b.n] = tot;
      b.it[b.n] = {reinterpret_cast<uint32_t*>(stages[k]) + (l.base + l.count[2]) * w, rows, l.row_pad * w, padw};
      b.n++;
      tot += blocks;
    }
    b.first[b.n] = tot;
    if (!tot) continue;
    count_launch();
    k_zero_pads_multi<<<(unsigned)tot, 256, 0, s>>>(b);
  }
}



}  // namespace pcr
