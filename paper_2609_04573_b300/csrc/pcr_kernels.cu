// CUDA kernels of the progressive refactor / retrieve path (sm_103a).
//
// Section references are to arXiv 2609.04573 (ProAICD).  Arithmetic follows
// fixed expression trees (compiled with -fmad=false and written with _rn
// intrinsics) so that results are reproducible bit for bit:
//   level 0 and its coefficient decomposition in the field dtype;
//   levels >= 1 in exact 64-bit fixed point (quantum 2^(G-40)).
#include <cuda_runtime.h>
#include <cstdint>
#include <atomic>
#include <type_traits>

#include "pcr_internal.h"

namespace pcr {

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
long long launch_count() { return g_launches.load(); }
void add_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

#define FULL 0xFFFFFFFFu

// --------------------------------------------------------------------------
// 1-D interpolation rules (Sec. IV): cubic in the interior, 3-point Lagrange
// at either edge, 2-point mean, and the left neighbour when the line ends.
// Floating-point forms chosen to round little (inputs bounded by V, unit
// roundoff u): cubic as s1 / 2 + (s1 - s2) / 16 rounds at most 2.75 u V, the
// edge rules as 0.75 a + (0.375 b - 0.125 c) at most 2.875 u V, the mean u V;
// the host's level-0 rounding allowance is built on these constants.
// --------------------------------------------------------------------------
template <typename T> struct Ar;

template <> struct Ar<float> {
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
};

template <> struct Ar<double> {
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
};

template <> struct Ar<int64_t> {
  __device__ static int64_t lin(int64_t a, int64_t b) { return (a + b) >> 1; }
  __device__ static int64_t cub(int64_t m3, int64_t m1, int64_t p1, int64_t p3) {
    return (9 * (m1 + p1) - (m3 + p3)) >> 4;
  }
  __device__ static int64_t lft(int64_t m1, int64_t p1, int64_t p3) { return (3 * m1 + 6 * p1 - p3) >> 3; }
  __device__ static int64_t rgt(int64_t m3, int64_t m1, int64_t p1) { return (6 * m1 + 3 * p1 - m3) >> 3; }
  __device__ static int64_t add(int64_t a, int64_t b) { return a + b; }
  __device__ static int64_t sub(int64_t a, int64_t b) { return a - b; }
};

template <typename T, class F>
__device__ __forceinline__ T rule1d(int64_t j, int64_t m, int degree, const F& at) {
  const bool p1 = j + 1 < m, m3 = j - 3 >= 0, p3 = j + 3 < m;
  if (degree == 3 && p1 && m3 && p3) return Ar<T>::cub(at(j - 3), at(j - 1), at(j + 1), at(j + 3));
  if (degree == 3 && p1 && p3) return Ar<T>::lft(at(j - 1), at(j + 1), at(j + 3));
  if (degree == 3 && p1 && m3) return Ar<T>::rgt(at(j - 3), at(j - 1), at(j + 1));
  if (p1) return Ar<T>::lin(at(j - 1), at(j + 1));
  return at(j - 1);
}

// Tensor recursion of the per-level scheme: the rule along odd[I] applied to
// values that are themselves predictions along odd[0..I-1] (Sec. VI-C: the
// per-level interpolant equals sequential passes that read predictions).
template <typename T, int I, class G>
__device__ __forceinline__ T wrec(int64_t q0, int64_t q1, int64_t q2, const int* odd,
                                  const int64_t* m, int degree, const G& get) {
  if constexpr (I < 0) {
    return get(q0, q1, q2);
  } else {
    const int a = odd[I];
    const int64_t j = a == 0 ? q0 : (a == 1 ? q1 : q2);
    auto at = [&](int64_t t) -> T {
      return wrec<T, I - 1>(a == 0 ? t : q0, a == 1 ? t : q1, a == 2 ? t : q2, odd, m, degree, get);
    };
    return rule1d<T>(j, m[a], degree, at);
  }
}

// Prediction at level-grid coordinates q (some coordinate odd along a pass
// axis).  per-level: rules along every odd axis in pass order, innermost
// first; per-region: one rule along the last odd pass axis reading `get`.
template <typename T, class G>
__device__ __forceinline__ T predict(const int64_t* q, const int64_t* m, const int* order, int d,
                                     int interp, int degree, const G& get) {
  int odd[3];
  int k = 0;
  for (int i = 0; i < d; i++)
    if (q[order[i]] & 1) odd[k++] = order[i];
  if (interp == 1 && k > 1) {
    odd[0] = odd[k - 1];
    k = 1;
  }
  switch (k) {
    case 1: return wrec<T, 0>(q[0], q[1], q[2], odd, m, degree, get);
    case 2: return wrec<T, 1>(q[0], q[1], q[2], odd, m, degree, get);
    case 3: return wrec<T, 2>(q[0], q[1], q[2], odd, m, degree, get);
    default: return get(q[0], q[1], q[2]);
  }
}

// --------------------------------------------------------------------------
// helpers
// --------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ unsigned long long absbits(T v);
template <> __device__ __forceinline__ unsigned long long absbits<float>(float v) {
  return __float_as_uint(fabsf(v));
}
template <> __device__ __forceinline__ unsigned long long absbits<double>(double v) {
  return (unsigned long long)__double_as_longlong(fabs(v));
}
template <> __device__ __forceinline__ unsigned long long absbits<int64_t>(int64_t v) {
  return (unsigned long long)(v < 0 ? -v : v);
}

__device__ __forceinline__ unsigned long long warp_max(unsigned long long v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    unsigned long long t = __shfl_xor_sync(FULL, v, o);
    v = t > v ? t : v;
  }
  return v;
}

// floor(x 2^(F-G)) for finite x with |x| < 2^G (exact bit manipulation).
template <typename T> __device__ __forceinline__ int64_t fix_from(T x, int G, int F);
template <> __device__ __forceinline__ int64_t fix_from<float>(float x, int G, int F) {
  const uint32_t u = __float_as_uint(x);
  const int e = (u >> 23) & 0xFF;
  const int64_t val = e ? (int64_t)((u & 0x7FFFFFu) | 0x800000u) : (int64_t)(u & 0x7FFFFFu);
  if (val == 0) return 0;
  const int sh = (e ? e - 150 : -149) + F - G;
  const bool neg = u >> 31;
  if (sh >= 0) { const int64_t r = val << sh; return neg ? -r : r; }
  const int k = -sh;
  if (k >= 62) return neg ? -1 : 0;
  if (!neg) return val >> k;
  return -((val + ((int64_t(1) << k) - 1)) >> k);
}
template <> __device__ __forceinline__ int64_t fix_from<double>(double x, int G, int F) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((u >> 52) & 0x7FF);
  const int64_t val = e ? (int64_t)((u & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull)
                        : (int64_t)(u & 0xFFFFFFFFFFFFFull);
  if (val == 0) return 0;
  const int sh = (e ? e - 1075 : -1074) + F - G;
  const bool neg = u >> 63;
  if (sh >= 0) { const int64_t r = val << sh; return neg ? -r : r; }
  const int k = -sh;
  if (k >= 62) return neg ? -1 : 0;
  if (!neg) return val >> k;
  return -((val + ((int64_t(1) << k) - 1)) >> k);
}

// lattice element -> field coordinates; returns false for row padding
__device__ __forceinline__ bool lat_coords(const LatD& l, int64_t idx, int64_t* p) {
  const int64_t col = idx % l.row_pad;
  if (col >= l.count[2]) return false;
  const int64_t row = idx / l.row_pad;
  const int64_t k1 = row % l.count[1], k0 = row / l.count[1];
  p[0] = l.start[0] + l.step[0] * k0;
  p[1] = l.start[1] + l.step[1] * k1;
  p[2] = l.start[2] + l.step[2] * col;
  return true;
}

__device__ __forceinline__ int64_t lat_padded_index(const LatD& l, const int64_t* p) {
  const int64_t k0 = (p[0] - l.start[0]) / l.step[0];
  const int64_t k1 = (p[1] - l.start[1]) / l.step[1];
  const int64_t k2 = (p[2] - l.start[2]) / l.step[2];
  return l.base + (k0 * l.count[1] + k1) * l.row_pad + k2;
}

// --------------------------------------------------------------------------
// a1: field statistics
// --------------------------------------------------------------------------
// min, max and finiteness of x[0 .. n) by the threads tid = 0 .. nth - 1 of
// the blocks that share this field (a grid, or the field's blocks of a
// batched launch)
template <typename T>
__device__ __forceinline__ void minmax_body(const T* __restrict__ x, int64_t n, FieldStats* st, int64_t tid,
                                            int64_t nth) {
  T lo = x[0], hi = x[0];
  int bad = 0;
  auto take = [&](T v) {
    bad |= !isfinite(v);
    lo = v < lo ? v : lo;
    hi = v > hi ? v : hi;
  };
  int64_t tail = 0;
  if (((uintptr_t)x & 15) == 0) {   // 16-byte vectors, four loads in flight
    using V = typename std::conditional<sizeof(T) == 4, float4, double2>::type;
    const V* xv = reinterpret_cast<const V*>(x);
    const int64_t nv = n / (16 / (int64_t)sizeof(T));
#pragma unroll 4
    for (int64_t i = tid; i < nv; i += nth) {
      const V t = __ldg(xv + i);
      if constexpr (sizeof(T) == 4) {
        take(t.x); take(t.y); take(t.z); take(t.w);
      } else {
        take(t.x); take(t.y);
      }
    }
    tail = nv * (16 / (int64_t)sizeof(T));
  }
  for (int64_t i = tail + tid; i < n; i += nth) take(x[i]);
  stats_push_block(st, (double)lo, (double)hi, bad);
}

template <typename T>
__global__ void k_minmax(const T* __restrict__ x, int64_t n, FieldStats* st) {
  minmax_body<T>(x, n, st, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

// ---------------------------------------------------------------------------
// batched forms: one launch for the fields of a batch (blocks first[i] ..
// first[i + 1] - 1 belong to item i)
// ---------------------------------------------------------------------------
struct MinmaxBatch {
  int n;
  int64_t first[kMaxBatchItems + 1];
  const void* x[kMaxBatchItems];
  int64_t cnt[kMaxBatchItems];
  FieldStats* st[kMaxBatchItems];
};
static_assert(sizeof(MinmaxBatch) <= 32764, "kernel parameter block");

template <typename T>
__global__ void k_minmax_multi(const __grid_constant__ MinmaxBatch b) {
  const int i = batch_find(b.first, b.n);
  const int64_t nblk = b.first[i + 1] - b.first[i];
  minmax_body<T>(reinterpret_cast<const T*>(b.x[i]), b.cnt[i], b.st[i],
                 (blockIdx.x - b.first[i]) * (int64_t)blockDim.x + threadIdx.x, nblk * blockDim.x);
}

__device__ __forceinline__ double dkey_inv(unsigned long long k) {
  unsigned long long u = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  return __longlong_as_double((long long)u);
}

__global__ void k_stats_finalize_multi(const __grid_constant__ MinmaxBatch b) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= b.n) return;
  FieldStats* st = b.st[i];
  const double lo = dkey_inv(st->xmin_key), hi = dkey_inv(st->xmax_key);
  const double M = fmax(fabs(lo), fabs(hi));
  int G = 0;
  if (M > 0) frexp(M, &G);
  st->G = G;
}

__global__ void k_stats_finalize(FieldStats* st) {
  const double lo = dkey_inv(st->xmin_key), hi = dkey_inv(st->xmax_key);
  const double M = fmax(fabs(lo), fabs(hi));
  int G = 0;
  if (M > 0) frexp(M, &G);
  st->G = G;
}

// fixed-point copy of the 2-grid (coarse points of level 0)
template <typename T>
__device__ __forceinline__ void to_fixed_body(const T* __restrict__ x, const FieldD& f, const FieldStats* st,
                                              int64_t* __restrict__ xc, int64_t tid, int64_t nth) {
  const int G = st->G;
  const int64_t n = f.nc[0] * f.nc[1] * f.nc[2];
  const int s0 = f.n[0] > 1 ? 2 : 1;
  for (int64_t i = tid; i < n; i += nth) {
    const int64_t c2 = i % f.nc[2], t = i / f.nc[2];
    const int64_t c1 = t % f.nc[1], c0 = t / f.nc[1];
    xc[i] = fix_from<T>(x[((c0 * s0) * f.n[1] + 2 * c1) * f.n[2] + 2 * c2], G, f.fixb);
  }
}

template <typename T>
__global__ void k_to_fixed(const T* __restrict__ x, FieldD f, const FieldStats* st, int64_t* __restrict__ xc) {
  to_fixed_body<T>(x, f, st, xc, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

struct ToFixedBatch {
  int n;
  int64_t first[kMaxBatchItems + 1];
  const void* x[kMaxBatchItems];
  FieldD f[kMaxBatchItems];
  const FieldStats* st[kMaxBatchItems];
  int64_t* xc[kMaxBatchItems];
};
static_assert(sizeof(ToFixedBatch) <= 32764, "kernel parameter block");

template <typename T>
__global__ void k_to_fixed_multi(const __grid_constant__ ToFixedBatch b) {
  const int i = batch_find(b.first, b.n);
  const int64_t nblk = b.first[i + 1] - b.first[i];
  to_fixed_body<T>(reinterpret_cast<const T*>(b.x[i]), b.f[i], b.st[i], b.xc[i],
                   (blockIdx.x - b.first[i]) * (int64_t)blockDim.x + threadIdx.x, nblk * blockDim.x);
}

// --------------------------------------------------------------------------
// coefficients (Alg. 1): c = x - P(x) at the points of one lattice
// --------------------------------------------------------------------------
struct LevelGrid {
  int64_t m[3];     // level-grid lengths
  int64_t s;        // stride of the level in field units
};

__device__ __forceinline__ LevelGrid level_grid(const FieldD& f, int level) {
  LevelGrid g;
  g.s = int64_t(1) << level;
  for (int a = 0; a < 3; a++) g.m[a] = f.n[a] > 1 ? (f.n[a] - 1) / g.s + 1 : 1;
  return g;
}

// fixed-point levels >= 1: values from the 2-grid copy; raw = coarsest level
__device__ __forceinline__ void coef_fixed_body(const FieldD& f, int level, int raw, const LatD& lat,
                                                const int64_t* __restrict__ xc, int64_t* __restrict__ out,
                                                unsigned long long* vmax, int64_t tid, int64_t nth) {
  const LevelGrid g = level_grid(f, level);
  const int64_t half = g.s >> 1;
  const int64_t n = lat.count[0] * lat.count[1] * lat.row_pad;
  auto get = [&](int64_t a0, int64_t a1, int64_t a2) -> int64_t {
    return xc[((a0 * (f.n[0] > 1 ? half : 0)) * f.nc[1] + a1 * half) * f.nc[2] + a2 * half];
  };
  unsigned long long mx = 0;
  for (int64_t i = tid; i < n; i += nth) {
    int64_t p[3];
    int64_t c = 0;
    if (lat_coords(lat, i, p)) {
      int64_t q[3] = {p[0] / g.s, p[1] / g.s, p[2] / g.s};
      const int64_t v = get(q[0], q[1], q[2]);
      c = raw ? v : v - predict<int64_t>(q, g.m, f.order, f.d, f.interp, f.degree, get);
    }
    out[lat.base + i] = c;
    const unsigned long long a = absbits<int64_t>(c);
    mx = a > mx ? a : mx;
  }
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0 && mx) atomicMax(vmax, mx);
}

__global__ void k_coef_fixed(FieldD f, int level, int raw, LatD lat, const int64_t* __restrict__ xc,
                             int64_t* __restrict__ out, unsigned long long* vmax) {
  coef_fixed_body(f, level, raw, lat, xc, out, vmax, blockIdx.x * (int64_t)blockDim.x + threadIdx.x,
                  (int64_t)gridDim.x * blockDim.x);
}

struct CoefFixedBatch {
  int n;
  int64_t first[kMaxBatchItems + 1];
  FieldD f[kMaxBatchItems];
  LatD lat[kMaxBatchItems];
  int level[kMaxBatchItems];
  const int64_t* xc[kMaxBatchItems];
  int64_t* out[kMaxBatchItems];
  unsigned long long* vmax[kMaxBatchItems];
};
static_assert(sizeof(CoefFixedBatch) <= 32764, "kernel parameter block");

__global__ void k_coef_fixed_multi(const __grid_constant__ CoefFixedBatch b) {
  const int i = batch_find(b.first, b.n);
  const int64_t nblk = b.first[i + 1] - b.first[i];
  coef_fixed_body(b.f[i], b.level[i], 1, b.lat[i], b.xc[i], b.out[i], b.vmax[i],
                  (blockIdx.x - b.first[i]) * (int64_t)blockDim.x + threadIdx.x, nblk * blockDim.x);
}

// level 0 in the field dtype.  compact != 0: write the region's compact
// (unpadded) array for the decomposition; else the padded stream layout.
template <typename T>
__global__ void k_coef_l0(FieldD f, LatD lat, int compact, const T* __restrict__ x,
                          T* __restrict__ out, unsigned long long* vmax, unsigned long long* c0) {
  const LevelGrid g = level_grid(f, 0);
  const int64_t n = compact ? lat.count[0] * lat.count[1] * lat.count[2]
                            : lat.count[0] * lat.count[1] * lat.row_pad;
  auto get = [&](int64_t a0, int64_t a1, int64_t a2) -> T { return x[(a0 * f.n[1] + a1) * f.n[2] + a2]; };
  unsigned long long mx = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t p[3];
    bool real;
    if (compact) {
      const int64_t k2 = i % lat.count[2], t = i / lat.count[2];
      p[0] = lat.start[0] + lat.step[0] * (t / lat.count[1]);
      p[1] = lat.start[1] + lat.step[1] * (t % lat.count[1]);
      p[2] = lat.start[2] + lat.step[2] * k2;
      real = true;
    } else {
      real = lat_coords(lat, i, p);
    }
    T c = T(0);
    if (real) c = Ar<T>::sub(get(p[0], p[1], p[2]),
                             predict<T>(p, g.m, f.order, f.d, f.interp, f.degree, get));
    out[(compact ? 0 : lat.base) + i] = c;
    const unsigned long long a = absbits<T>(c);
    mx = a > mx ? a : mx;
  }
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0 && mx) {
    if (vmax) {
      if (sizeof(T) == 4) atomicMax((unsigned int*)vmax, (unsigned int)mx);
      else atomicMax(vmax, mx);
    }
    if (c0) {
      double dv = sizeof(T) == 4 ? (double)__uint_as_float((unsigned int)mx)
                                 : __longlong_as_double((long long)mx);
      atomicMax(c0, (unsigned long long)__double_as_longlong(dv));
    }
  }
}

// --------------------------------------------------------------------------
// coefficient decomposition (Sec. V-B, Alg. 1): 2-D per-level linear
// hierarchy on every slice normal to axis `nrm` of a region's compact array.
// sub 1: raw 4-grid; sub 2: predicted on the 2-grid from the 4-grid; sub 3:
// predicted on the full grid from the 2-grid (originals in both).
// --------------------------------------------------------------------------
template <typename T, class G>
__device__ __forceinline__ T decomp_predict(const DecompGeo& dg, const int64_t* kc, const G& getc) {
  // getc(k0, k1, k2) reads the region compact array
  const int64_t cu = dg.region.count[dg.u], cv = dg.region.count[dg.v];
  const int ord[2] = {dg.u, dg.v};
  if (dg.sub == 2) {
    int64_t m[3] = {1, 1, 1};
    m[dg.u] = (cu + 1) / 2;
    m[dg.v] = (cv + 1) / 2;
    int64_t q[3] = {kc[0], kc[1], kc[2]};
    q[dg.u] >>= 1;
    q[dg.v] >>= 1;
    const int u = dg.u, v = dg.v;
    auto get2 = [&](int64_t a0, int64_t a1, int64_t a2) -> T {
      int64_t k[3] = {a0, a1, a2};
      k[u] *= 2;
      k[v] *= 2;
      return getc(k[0], k[1], k[2]);
    };
    return predict<T>(q, m, ord, 2, 0, 1, get2);
  }
  int64_t m[3] = {1, 1, 1};
  m[dg.u] = cu;
  m[dg.v] = cv;
  return predict<T>(kc, m, ord, 2, 0, 1, getc);
}

template <typename T>
__global__ void k_decompose(DecompGeo dg, LatD sl, const T* __restrict__ comp, T* __restrict__ out,
                            unsigned long long* vmax) {
  const LatD& R = dg.region;
  const int64_t n = sl.count[0] * sl.count[1] * sl.row_pad;
  auto getc = [&](int64_t a0, int64_t a1, int64_t a2) -> T {
    return comp[(a0 * R.count[1] + a1) * R.count[2] + a2];
  };
  unsigned long long mx = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t p[3];
    T dv = T(0);
    if (lat_coords(sl, i, p)) {
      const int64_t kc[3] = {(p[0] - R.start[0]) / R.step[0], (p[1] - R.start[1]) / R.step[1],
                             (p[2] - R.start[2]) / R.step[2]};
      const T c = getc(kc[0], kc[1], kc[2]);
      dv = dg.sub == 1 ? c : Ar<T>::sub(c, decomp_predict<T>(dg, kc, getc));
    }
    out[sl.base + i] = dv;
    const unsigned long long a = absbits<T>(dv);
    mx = a > mx ? a : mx;
  }
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0 && mx) {
    if (sizeof(T) == 4) atomicMax((unsigned int*)vmax, (unsigned int)mx);
    else atomicMax(vmax, mx);
  }
}

// inverse (Alg. 2): comp[k] = d_hat (S1) or d_hat + prediction (S2, S3)
template <typename T>
__global__ void k_recompose(DecompGeo dg, LatD sl, const T* __restrict__ dec, T* __restrict__ comp) {
  const LatD& R = dg.region;
  const int64_t n = sl.count[0] * sl.count[1] * sl.count[2];
  auto getc = [&](int64_t a0, int64_t a1, int64_t a2) -> T {
    return comp[(a0 * R.count[1] + a1) * R.count[2] + a2];
  };
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k2 = i % sl.count[2], t = i / sl.count[2];
    const int64_t p[3] = {sl.start[0] + sl.step[0] * (t / sl.count[1]),
                          sl.start[1] + sl.step[1] * (t % sl.count[1]), sl.start[2] + sl.step[2] * k2};
    const int64_t kc[3] = {(p[0] - R.start[0]) / R.step[0], (p[1] - R.start[1]) / R.step[1],
                           (p[2] - R.start[2]) / R.step[2]};
    const T d = dec[sl.base + (t * sl.row_pad) + k2];
    const T r = dg.sub == 1 ? d : Ar<T>::add(decomp_predict<T>(dg, kc, getc), d);
    comp[(kc[0] * R.count[1] + kc[1]) * R.count[2] + kc[2]] = r;
  }
}

// --------------------------------------------------------------------------
// reconstruction (Alg. 2)
// --------------------------------------------------------------------------
// fixed-point levels >= 1: xc[p/2] = P(xc) + c_hat (raw: = c_hat)
__global__ void k_recon_fixed(FieldD f, int level, int raw, LatD lat, const int64_t* __restrict__ chat,
                              int64_t* __restrict__ xc) {
  const LevelGrid g = level_grid(f, level);
  const int64_t half = g.s >> 1;
  const int64_t n = lat.count[0] * lat.count[1] * lat.count[2];
  auto idx = [&](int64_t a0, int64_t a1, int64_t a2) -> int64_t {
    return ((a0 * (f.n[0] > 1 ? half : 0)) * f.nc[1] + a1 * half) * f.nc[2] + a2 * half;
  };
  auto get = [&](int64_t a0, int64_t a1, int64_t a2) -> int64_t { return xc[idx(a0, a1, a2)]; };
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k2 = i % lat.count[2], t = i / lat.count[2];
    const int64_t p[3] = {lat.start[0] + lat.step[0] * (t / lat.count[1]),
                          lat.start[1] + lat.step[1] * (t % lat.count[1]), lat.start[2] + lat.step[2] * k2};
    int64_t q[3] = {p[0] / g.s, p[1] / g.s, p[2] / g.s};
    const int64_t ch = chat[lat.base + t * lat.row_pad + k2];
    const int64_t v = raw ? ch : predict<int64_t>(q, g.m, f.order, f.d, f.interp, f.degree, get) + ch;
    xc[idx(q[0], q[1], q[2])] = v;
  }
}

// coarse points of level 0: out[2-grid] = x_int h rounded once, over the
// 2-grid box [lo, lo + cnt)
template <typename T>
__global__ void k_coarse_out(FieldD f, const int64_t* __restrict__ xc, T scale, T* __restrict__ out, Box3 b) {
  const int64_t n = b.cnt[0] * b.cnt[1] * b.cnt[2];
  const int s0 = f.n[0] > 1 ? 2 : 1;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c2 = i % b.cnt[2] + b.lo[2], t = i / b.cnt[2];
    const int64_t c1 = t % b.cnt[1] + b.lo[1], c0 = t / b.cnt[1] + b.lo[0];
    out[((c0 * s0) * f.n[1] + 2 * c1) * f.n[2] + 2 * c2] = from_fix<T>(xc[(c0 * f.nc[1] + c1) * f.nc[2] + c2], scale);
  }
}

// out[box] = field[lo + box] (row-major box of cnt points)
template <typename T>
__global__ void k_copy_box(FieldD f, const T* __restrict__ src, T* __restrict__ dst, Box3 b) {
  const int64_t n = b.cnt[0] * b.cnt[1] * b.cnt[2];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t c2 = i % b.cnt[2], t = i / b.cnt[2];
    const int64_t c1 = t % b.cnt[1], c0 = t / b.cnt[1];
    dst[i] = src[((c0 + b.lo[0]) * f.n[1] + c1 + b.lo[1]) * f.n[2] + c2 + b.lo[2]];
  }
}

// level 0: out[p] = P(out) + c_hat; c_hat from the padded stream layout of
// `lat` (compact == 0) or from the region's recomposed compact array.
template <typename T>
__global__ void k_recon_l0(FieldD f, LatD lat, int compact, const T* __restrict__ chat, T* __restrict__ out) {
  const LevelGrid g = level_grid(f, 0);
  const int64_t n = lat.count[0] * lat.count[1] * lat.count[2];
  auto get = [&](int64_t a0, int64_t a1, int64_t a2) -> T { return out[(a0 * f.n[1] + a1) * f.n[2] + a2]; };
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k2 = i % lat.count[2], t = i / lat.count[2];
    const int64_t p[3] = {lat.start[0] + lat.step[0] * (t / lat.count[1]),
                          lat.start[1] + lat.step[1] * (t % lat.count[1]), lat.start[2] + lat.step[2] * k2};
    const T ch = compact ? chat[i] : chat[lat.base + t * lat.row_pad + k2];
    out[(p[0] * f.n[1] + p[1]) * f.n[2] + p[2]] =
        Ar<T>::add(predict<T>(p, g.m, f.order, f.d, f.interp, f.degree, get), ch);
  }
}

// L == 1: the whole field is the raw coarse stream
template <typename T>
__global__ void k_copy_raw(FieldD f, LatD lat, const T* __restrict__ vals, T* __restrict__ out) {
  const int64_t n = lat.count[0] * lat.count[1] * lat.count[2];
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k2 = i % lat.count[2], t = i / lat.count[2];
    const int64_t p0 = t / lat.count[1], p1 = t % lat.count[1];
    out[(p0 * f.n[1] + p1) * f.n[2] + k2] = vals[t * lat.row_pad + k2];
  }
}

template <typename T>
__global__ void k_raw_stage(FieldD f, LatD lat, const T* __restrict__ x, T* __restrict__ out,
                            unsigned long long* vmax) {
  const int64_t n = lat.count[0] * lat.count[1] * lat.row_pad;
  unsigned long long mx = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t p[3];
    T v = T(0);
    if (lat_coords(lat, i, p)) v = x[(p[0] * f.n[1] + p[1]) * f.n[2] + p[2]];
    out[i] = v;
    const unsigned long long a = absbits<T>(v);
    mx = a > mx ? a : mx;
  }
  mx = warp_max(mx);
  if ((threadIdx.x & 31) == 0 && mx) {
    if (sizeof(T) == 4) atomicMax((unsigned int*)vmax, (unsigned int)mx);
    else atomicMax(vmax, mx);
  }
}

// --------------------------------------------------------------------------
// bitplanes (Sec. V-C; Sec. VI-A encodings)
// --------------------------------------------------------------------------
// 32 x 32 bit transpose across a warp: bit k of lane e <-> bit e of lane k
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
#pragma unroll
  for (int j = 16; j >= 1; j >>= 1) {
    const uint32_t m = j == 16 ? 0x0000FFFFu : j == 8 ? 0x00FF00FFu : j == 4 ? 0x0F0F0F0Fu
                     : j == 2 ? 0x33333333u : 0x55555555u;
    const uint32_t y = __shfl_xor_sync(FULL, x, j);
    x = (lane & j) ? ((x & ~m) | ((y & ~m) >> j)) : ((x & m) | ((y & m) << j));
  }
  return x;
}

__host__ __device__ __forceinline__ uint64_t nb_mask(int B) {
  uint64_t m = 0;
  for (int i = 1; i < B; i += 2) m |= uint64_t(1) << i;
  return m;
}

// quantisation parameters of one stream from its maximum
struct QParams {
  int E;      // float exponent, or fixed bit length
  int sh;     // fixed shift
  bool zero;
};

__device__ __forceinline__ QParams qparams(const StreamD& s) {
  QParams q;
  const unsigned long long vm = *s.vmax;
  q.zero = vm == 0;
  q.E = 0;
  q.sh = 0;
  if (s.vk == VK_F32) {
    if (vm) frexpf(__uint_as_float((unsigned)vm), &q.E);
  } else if (s.vk == VK_F64) {
    if (vm) frexp(__longlong_as_double((long long)vm), &q.E);
  } else {
    q.E = vm ? 64 - __clzll((long long)vm) : 0;
    const int lim = s.enc == 2 ? s.B - 3 : s.B;
    q.sh = q.E > lim ? q.E - lim : 0;
  }
  return q;
}

template <typename VT, int W> struct Code;  // W-bit code of one value

template <int W>
using code_t = typename std::conditional<W == 32, uint32_t, uint64_t>::type;

// exact power-of-two scaling: x * 2^k through one multiply when 2^k is a
// normal number (then the product is exact whenever it is >= 1 or a normal
// number), else through ldexp
__device__ __forceinline__ float scale2f(float x, int k) {
  return (k >= -126 && k <= 127) ? __fmul_rn(x, __int_as_float((k + 127) << 23)) : ldexpf(x, k);
}
__device__ __forceinline__ double scale2d(double x, int k) {
  return (k >= -1022 && k <= 1023) ? __dmul_rn(x, __longlong_as_double((long long)(k + 1023) << 52)) : ldexp(x, k);
}

// x * 2^k as two multiplies by normal powers of two, chosen per stream so
// that the first product is exact whenever the result can reach 1: for k in
// [-126, 127] (2^k, 1); above, (2^127, 2^(k-127)); below, (2^(k+126), 2^-126).
// Truncated to an integer this equals scale2f(x, k) for every |x| < 2^E;
// applied to a dequantised integer (>= 1 or 0) it rounds once, as scale2f.
struct Scale2 {
  float m1, m2;
};
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }   // k in [-126, 127]
__device__ __forceinline__ Scale2 scale_pair(int k) {
  if (k > 127) return {pow2f(127), pow2f(k - 127)};
  if (k < -126) return {pow2f(k + 126), pow2f(-126)};
  return {pow2f(k), 1.0f};
}

// S: any type with the stream's B and enc (StreamD, or a register copy)
template <typename VT, int W, typename S>
__device__ __forceinline__ code_t<W> quantize(VT v, const S& s, const QParams& qp, bool& neg) {
  using C = code_t<W>;
  const int B = s.B;
  const C M = (C)nb_mask(B);
  if constexpr (std::is_same<VT, int64_t>::value) {
    const uint64_t a = (uint64_t)(v < 0 ? -v : v);
    neg = v < 0;
    const uint64_t mag = a >> qp.sh;
    if (s.enc == 1) return (C)mag;
    const int64_t sv = neg ? -(int64_t)mag : (int64_t)mag;
    return (C)(((C)sv + M) ^ M);
  } else if constexpr (std::is_same<VT, float>::value) {
    neg = v < 0.0f;
    if (s.enc == 1) return (C)__float2uint_rz(scale2f(fabsf(v), B - qp.E));
    const int sv = __float2int_rz(scale2f(v, B - 3 - qp.E));
    return (C)(((C)(int64_t)sv + M) ^ M);
  } else {
    neg = v < 0.0;
    if (s.enc == 1) return (C)__double2ull_rz(scale2d(fabs(v), B - qp.E));
    const long long sv = __double2ll_rz(scale2d(v, B - 3 - qp.E));
    return (C)(((C)sv + M) ^ M);
  }
}

template <typename VT, int W>
__device__ __forceinline__ VT dequantize(code_t<W> q, bool neg, const StreamD& s) {
  const int B = s.B;
  if (s.enc == 1) {
    if constexpr (std::is_same<VT, int64_t>::value) {
      const int64_t mag = (int64_t)((uint64_t)q << s.sh);
      return neg ? -mag : mag;
    } else if constexpr (std::is_same<VT, float>::value) {
      const float mag = scale2f(__uint2float_rn((uint32_t)q), s.E - B);
      return neg ? -mag : mag;
    } else {
      const double mag = scale2d(__ull2double_rn((unsigned long long)q), s.E - B);
      return neg ? -mag : mag;
    }
  }
  const uint64_t M = nb_mask(B);
  int64_t val;
  if (W == 32) val = (int64_t)((uint64_t)(q ^ (code_t<W>)M)) - (int64_t)M;
  else val = (int64_t)(((uint64_t)q ^ M) - M);
  if constexpr (std::is_same<VT, int64_t>::value) {
    return (int64_t)((uint64_t)val << s.sh);
  } else if constexpr (std::is_same<VT, float>::value) {
    // |val| < 2^31 here: the quantised value is below 2^(B-3) <= 2^29 and the
    // digits dropped below plane b are worth less than (2/3) 2^31, so the
    // 32-bit conversion rounds the same integer as a 64-bit one would
    if (W == 32) return scale2f(__int2float_rn((int)val), s.E - B + 3);
    return scale2f(__ll2float_rn(val), s.E - B + 3);
  } else {
    return scale2d(__ll2double_rn(val), s.E - B + 3);
  }
}

template <int NP>
__device__ __forceinline__ int tri(int a, int b) {  // a <= b
  return a * NP - (a * (a - 1)) / 2 + (b - a);
}

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kWordsPerWarp = kSegWords / kWarps;   // 16

// most significant plane of code q (B for q == 0)
template <int W>
__device__ __forceinline__ int msb_plane(code_t<W> q, int B) {
  if (!q) return B;
  return W == 32 ? __clz((uint32_t)q << (32 - B)) : __clzll((long long)((uint64_t)q << (64 - B)));
}

// Generic-encoding sign bookkeeping for one word: the element's plane p and
// its rank among this warp's earlier elements of plane p (running per-warp
// counters in shared memory; match.any groups lanes of equal plane).
__device__ __forceinline__ uint32_t sign_record(int p, bool neg, int B, uint32_t* wc, int lane) {
  const unsigned grp = __match_any_sync(FULL, p);
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t rec = 0xFFFFFFFFu;
  uint32_t base = 0;
  if (p < B) base = wc[p];
  __syncwarp();
  if (p < B) {
    rec = (uint32_t)p | ((base + __popc(grp & lt)) << 7) | ((uint32_t)neg << 20);
    if ((grp & lt) == 0) wc[p] = base + __popc(grp);
  }
  __syncwarp();
  return rec;
}

// per-plane sign layout of a segment (32-bit codes): woff[w][k] = elements
// of plane k in warps before w, poff[k] = first sign word of plane k (an
// exclusive prefix of the planes' word counts over the lanes), poff[32] =
// the segment's sign words; wcnt[0][k] becomes the segment total of plane k.
// Run by warp 0.
__device__ __forceinline__ void sign_layout32(uint32_t (*wcnt)[32], uint32_t (*woff)[32], uint32_t* poff, int B,
                                              int lane) {
  uint32_t acc = 0;
#pragma unroll
  for (int w = 0; w < kWarps; w++) {
    const uint32_t c = wcnt[w][lane];
    woff[w][lane] = acc;
    acc += c;
  }
  wcnt[0][lane] = acc;
  const uint32_t words = lane < B ? (acc + 31) >> 5 : 0u;
  uint32_t inc = words;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(FULL, inc, o);
    inc += lane >= o ? t : 0u;
  }
  poff[lane] = inc - words;
  if (lane == 31) poff[32] = inc;
}

// Encode one (stream, segment) per CTA.  W = 32 (FP32 fields) or 64 (FP64).
template <typename VT, int W, bool PAIRS>
__global__ void __launch_bounds__(kThreads) k_encode(const StreamD* __restrict__ streams,
                                                     const WorkItem* __restrict__ items) {
  constexpr int NP = W;
  __shared__ uint32_t pbuf[NP][kSegWords + 1];
  __shared__ uint32_t sbuf[kSegWords + 64];
  __shared__ uint32_t wcnt[kWarps][NP];
  __shared__ uint32_t woff[kWarps][NP];
  __shared__ uint32_t poff[NP + 1];
  __shared__ uint32_t pnz[NP];
  __shared__ uint32_t pairs_s[PAIRS ? NP * (NP + 1) / 2 : 1];

  const WorkItem it = items[blockIdx.x];
  const StreamD& s = streams[it.stream];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int B = s.B;
  const int64_t e0 = (int64_t)it.seg * kSegElems;
  const int nw = (int)min((int64_t)kSegWords, (s.n_pad - e0) / 32);
  const QParams qp = qparams(s);
  const VT* vals = (const VT*)s.stage;
  const bool generic = s.enc == 1;

  for (int i = threadIdx.x; i < kSegWords + 64; i += kThreads) sbuf[i] = 0;
  if (threadIdx.x < NP) pnz[threadIdx.x] = 0;
  for (int i = threadIdx.x; i < kWarps * NP; i += kThreads) (&wcnt[0][0])[i] = 0;
  if (PAIRS)
    for (int i = threadIdx.x; i < NP * (NP + 1) / 2; i += kThreads) pairs_s[i] = 0;
  __syncthreads();

  uint32_t rec[kWordsPerWarp];
  uint32_t nz_lo = 0, nz_hi = 0;
  uint32_t acc_ll[PAIRS ? 17 : 1], acc_hh[PAIRS && W == 64 ? 17 : 1], acc_lh[PAIRS && W == 64 ? 32 : 1];
  if (PAIRS) {
#pragma unroll
    for (int t = 0; t < 17; t++) acc_ll[t] = 0;
    if (W == 64) {
#pragma unroll
      for (int t = 0; t < 17; t++) acc_hh[t] = 0;
#pragma unroll
      for (int t = 0; t < 32; t++) acc_lh[t] = 0;
    }
  }

#pragma unroll
  for (int jj = 0; jj < kWordsPerWarp; jj++) {
    rec[jj] = 0xFFFFFFFFu;
    const int j = warp * kWordsPerWarp + jj;
    if (j >= nw) continue;
    const VT v = vals[e0 + (int64_t)j * 32 + lane];
    bool neg = false;
    code_t<W> q = 0;
    if (!qp.zero) q = quantize<VT, W>(v, s, qp, neg);
    uint32_t dlo, dhi = 0;
    if (W == 32) {
      dlo = transpose32(__brev((uint32_t)q << (32 - B)), lane);
    } else {
      const uint64_t r = __brevll((unsigned long long)((uint64_t)q << (64 - B)));
      dlo = transpose32((uint32_t)r, lane);
      dhi = transpose32((uint32_t)(r >> 32), lane);
    }
    uint32_t slo = dlo, shi = dhi;
    if (!generic) {
      const uint32_t up = __shfl_up_sync(FULL, dlo, 1);
      slo = lane ? dlo ^ up : dlo;
      if (W == 64) {
        const uint32_t uph = __shfl_up_sync(FULL, dhi, 1);
        const uint32_t l31 = __shfl_sync(FULL, dlo, 31);
        shi = dhi ^ (lane ? uph : l31);
      }
    }
    if (lane < B) pbuf[lane][j] = slo;
    if (W == 64 && lane + 32 < B) pbuf[lane + 32][j] = shi;
    nz_lo += slo != 0;
    nz_hi += shi != 0;
    if (generic) rec[jj] = sign_record(msb_plane<W>(q, B), neg, B, wcnt[warp], lane);
    if (PAIRS) {
#pragma unroll
      for (int t = 0; t < 17; t++) {
        const uint32_t o = __shfl_sync(FULL, dlo, (lane + t) & 31);
        acc_ll[t] += __popc(dlo & o);
      }
      if (W == 64) {
#pragma unroll
        for (int t = 0; t < 17; t++) {
          const uint32_t o = __shfl_sync(FULL, dhi, (lane + t) & 31);
          acc_hh[t] += __popc(dhi & o);
        }
#pragma unroll
        for (int t = 0; t < 32; t++) {
          const uint32_t o = __shfl_sync(FULL, dhi, (lane + t) & 31);
          acc_lh[t] += __popc(dlo & o);
        }
      }
    }
  }
  if (lane < B && nz_lo) atomicAdd(&pnz[lane], nz_lo);
  if (W == 64 && lane + 32 < B && nz_hi) atomicAdd(&pnz[lane + 32], nz_hi);
  if (PAIRS) {
#pragma unroll
    for (int t = 0; t < 17; t++) {
      const int b = (lane + t) & 31;
      if ((t < 16 || lane < 16) && acc_ll[t]) atomicAdd(&pairs_s[tri<NP>(min(lane, b), max(lane, b))], acc_ll[t]);
      if (W == 64 && (t < 16 || lane < 16) && acc_hh[t])
        atomicAdd(&pairs_s[tri<NP>(min(lane, b) + 32, max(lane, b) + 32)], acc_hh[t]);
    }
    if (W == 64) {
#pragma unroll
      for (int t = 0; t < 32; t++)
        if (acc_lh[t]) atomicAdd(&pairs_s[tri<NP>(lane, 32 + ((lane + t) & 31))], acc_lh[t]);
    }
  }
  __syncthreads();
  if (generic) {
    if constexpr (W == 32) {
      if (warp == 0) sign_layout32(wcnt, woff, poff, B, lane);
    } else {
      if (threadIdx.x < NP) {
        const int k = threadIdx.x;
        uint32_t acc = 0;
        for (int w = 0; w < kWarps; w++) {
          woff[w][k] = acc;
          acc += wcnt[w][k];
        }
        wcnt[0][k] = acc;   // segment total of plane k
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        uint32_t o = 0;
        for (int k = 0; k < B; k++) {
          poff[k] = o;
          o += (wcnt[0][k] + 31) >> 5;
        }
        poff[B] = o;
      }
    }
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < kWordsPerWarp; jj++) {
      const uint32_t r = rec[jj];
      if (r != 0xFFFFFFFFu && (r >> 20)) {
        const int p = r & 127;
        const uint32_t pos = (r >> 7) & 8191;
        const uint32_t bit = poff[p] * 32 + woff[warp][p] + pos;
        atomicOr(&sbuf[bit >> 5], 1u << (bit & 31));
      }
    }
    __syncthreads();
    uint32_t* dst = s.signs + (int64_t)it.seg * s.slot_words;
    for (int i = threadIdx.x; i < (int)poff[B]; i += kThreads) dst[i] = sbuf[i];
    if (threadIdx.x < B) {
      const uint32_t c = wcnt[0][threadIdx.x];
      s.sign_counts[(int64_t)it.seg * B + threadIdx.x] = c;
      if (c) atomicAdd(&s.plane_nz[B + threadIdx.x], (c + 31) >> 5);   // sign words of plane k
    }
  }
  // plane words: coalesced per plane
  const int64_t w0 = (int64_t)it.seg * kSegWords;
  if (nw == kSegWords) {
    for (int i = threadIdx.x; i < B * kSegWords; i += kThreads)
      s.planes[(int64_t)(i >> 7) * s.words + w0 + (i & 127)] = pbuf[i >> 7][i & 127];
  } else {
    for (int i = threadIdx.x; i < B * nw; i += kThreads) {
      const int k = i / nw, j = i - k * nw;
      s.planes[(int64_t)k * s.words + w0 + j] = pbuf[k][j];
    }
  }
  if (threadIdx.x < B && pnz[threadIdx.x]) atomicAdd(&s.plane_nz[threadIdx.x], pnz[threadIdx.x]);
  if (PAIRS) {
    for (int i = threadIdx.x; i < NP * NP; i += kThreads) {
      const int a = i / NP, c = i % NP;
      if (a <= c && c < B && pairs_s[tri<NP>(a, c)])
        atomicAdd(&s.pairs[a * B + c], (unsigned long long)pairs_s[tri<NP>(a, c)]);
    }
  }
}

// per-lane constants of the warp bit transpose (hoisted out of word loops):
// byte permutes for the 16- and 8-bit stages, and for the 4-, 2- and 1-bit
// stages a rotation of the partner's word plus one masked merge
struct TrC {
  uint32_t sel16, sel8;
  uint32_t ml[3], sh[3];
};
__device__ __forceinline__ TrC tr_consts(int lane) {
  TrC c;
  c.sel16 = (lane & 16) ? 0x3276u : 0x5410u;
  c.sel8 = (lane & 8) ? 0x3715u : 0x6240u;
#pragma unroll
  for (int s = 0; s < 3; s++) {
    const int j = 4 >> s;
    const uint32_t m = j == 4 ? 0x0F0F0F0Fu : j == 2 ? 0x33333333u : 0x55555555u;
    const bool lower = (lane & j) == 0;
    c.ml[s] = lower ? m : ~m;
    c.sh[s] = lower ? j : 32 - j;
  }
  return c;
}
// the same transpose as transpose32 (bit k of lane e <-> bit e of lane k)
__device__ __forceinline__ uint32_t transpose32c(uint32_t x, const TrC& c) {
  uint32_t y = __shfl_xor_sync(FULL, x, 16);
  x = __byte_perm(x, y, c.sel16);
  y = __shfl_xor_sync(FULL, x, 8);
  x = __byte_perm(x, y, c.sel8);
#pragma unroll
  for (int s = 0; s < 3; s++) {
    y = __shfl_xor_sync(FULL, x, 4 >> s);
    const uint32_t yy = __funnelshift_l(y, y, c.sh[s]);
    x = (x & c.ml[s]) | (yy & ~c.ml[s]);
  }
  return x;
}

// Generic-encoding sign rank of one word from its plane words (lane k holds
// plane k): F_k = the elements whose leading one is in plane k (plane bits
// not covered by a more significant plane, an exclusive prefix OR over the
// lanes).  The element's rank within its plane is the warp's count of
// earlier words' elements of that plane (ctr, held by the plane's lane) plus
// the lanes below it in F_p.  Same ranks as sign_record, without match.any
// (used by the decoder; the encoder measured faster with sign_record).
__device__ __forceinline__ uint32_t sign_rank32(uint32_t d, int p, bool neg, int B, uint32_t& ctr, int lane,
                                                uint32_t lt) {
  // inclusive prefix OR over the lanes (a lane below o gets its own value
  // back from the shuffle, which leaves the OR unchanged)
  uint32_t incl = d;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) incl |= __shfl_up_sync(FULL, incl, o);
  uint32_t excl = __shfl_up_sync(FULL, incl, 1);
  excl = lane ? excl : 0u;
  const uint32_t F = d & ~excl;
  const uint32_t fp = __shfl_sync(FULL, F, p & 31), cp = __shfl_sync(FULL, ctr, p & 31);
  ctr += __popc(F);
  return p < B ? ((uint32_t)p | ((cp + __popc(fp & lt)) << 7) | ((uint32_t)neg << 20)) : 0xFFFFFFFFu;
}

// Decode one (stream, segment) per CTA: planes < b (zero-fill below).
template <typename VT, int W>
__global__ void __launch_bounds__(kThreads) k_decode(const StreamD* __restrict__ streams,
                                                     const WorkItem* __restrict__ items) {
  constexpr int NP = W;
  // plane rows padded to 132 words: 16-byte aligned rows, and the 16-byte
  // reads of 8 lanes from 8 rows fall on distinct banks
  __shared__ __align__(16) uint32_t pbuf[NP][kSegWords + 4];
  __shared__ uint32_t sbuf[kSegWords + 64];
  __shared__ uint32_t wcnt[kWarps][NP];
  __shared__ uint32_t woff[kWarps][NP];
  __shared__ uint32_t poff[NP + 1];

  const WorkItem it = items[blockIdx.x];
  const StreamD& s = streams[it.stream];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int B = s.B, b = s.b;
  const int64_t e0 = (int64_t)it.seg * kSegElems;
  const int nw = (int)min((int64_t)kSegWords, (s.n_pad - e0) / 32);
  const bool generic = s.enc == 1;
  const int64_t w0 = (int64_t)it.seg * kSegWords;
  VT* out = (VT*)s.stage;

  // 16-byte loads need 16-byte aligned plane rows: a whole number of
  // 4-word groups per plane and an aligned stream base (streams before this
  // one with B * words not a multiple of 4 shift it)
  if (nw == kSegWords && (s.words & 3) == 0 && ((uintptr_t)s.planes & 15) == 0) {
    for (int i = threadIdx.x; i < b * (kSegWords / 4); i += kThreads) {
      const int k = i >> 5, c = i & 31;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (s.plane_nz[k]) v = *reinterpret_cast<const uint4*>(s.planes + (int64_t)k * s.words + w0 + 4 * c);
      *reinterpret_cast<uint4*>(&pbuf[k][4 * c]) = v;
    }
  } else if (nw == kSegWords) {
    for (int i = threadIdx.x; i < b * kSegWords; i += kThreads) {
      const int k = i >> 7, j = i & 127;
      pbuf[k][j] = s.plane_nz[k] ? s.planes[(int64_t)k * s.words + w0 + j] : 0u;
    }
  } else {
    for (int i = threadIdx.x; i < b * nw; i += kThreads) {
      const int k = i / nw, j = i - k * nw;
      pbuf[k][j] = s.plane_nz[k] ? s.planes[(int64_t)k * s.words + w0 + j] : 0u;
    }
  }
  if (W == 64)
    for (int i = threadIdx.x; i < kWarps * NP; i += kThreads) (&wcnt[0][0])[i] = 0;
  if (generic) {
    if (W == 32) {
      if (threadIdx.x < 32) {   // first sign word of each plane: prefix of the planes' word counts
        const int k = threadIdx.x;
        const uint32_t words = k < B ? (s.sign_counts[(int64_t)it.seg * B + k] + 31) >> 5 : 0u;
        uint32_t inc = words;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t t = __shfl_up_sync(FULL, inc, o);
          inc += k >= o ? t : 0u;
        }
        poff[k] = inc - words;
        if (k == 31) poff[32] = inc;
      }
    } else if (threadIdx.x == 0) {
      uint32_t o = 0;
      for (int k = 0; k < B; k++) {
        poff[k] = o;
        o += (s.sign_counts[(int64_t)it.seg * B + k] + 31) >> 5;
      }
      poff[B] = o;
    }
    __syncthreads();
    const uint32_t* src = s.signs + (int64_t)it.seg * s.slot_words;
    for (int i = threadIdx.x; i < (int)poff[b]; i += kThreads) sbuf[i] = src[i];
  }
  __syncthreads();

  code_t<W> qs[kWordsPerWarp];
  uint32_t rec[kWordsPerWarp];
  const TrC tc = tr_consts(lane);
  const uint32_t lt = (1u << lane) - 1u;
  uint32_t ctr = 0;
  uint4 gl = make_uint4(0u, 0u, 0u, 0u), gh = gl;   // plane words of 4 consecutive words
#pragma unroll
  for (int jj = 0; jj < kWordsPerWarp; jj++) {
    const int j = warp * kWordsPerWarp + jj;
    qs[jj] = 0;
    rec[jj] = 0xFFFFFFFFu;
    if (j >= nw) continue;
    if ((jj & 3) == 0) {
      if (lane < b) gl = *reinterpret_cast<const uint4*>(&pbuf[lane][j]);
      if (W == 64 && lane + 32 < b) gh = *reinterpret_cast<const uint4*>(&pbuf[lane + 32][j]);
    }
    const int e4 = jj & 3;
    uint32_t xl = lane < b ? (e4 == 0 ? gl.x : e4 == 1 ? gl.y : e4 == 2 ? gl.z : gl.w) : 0u;
    uint32_t xh = (W == 64 && lane + 32 < b) ? (e4 == 0 ? gh.x : e4 == 1 ? gh.y : e4 == 2 ? gh.z : gh.w) : 0u;
    if (!generic) {
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(FULL, xl, o);
        if (lane >= o) xl ^= t;
      }
      if (W == 64) {
        const uint32_t tot = __shfl_sync(FULL, xl, 31);
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t t = __shfl_up_sync(FULL, xh, o);
          if (lane >= o) xh ^= t;
        }
        xh ^= tot;
      }
      if (lane >= b) xl = 0;
      if (lane + 32 >= b) xh = 0;
    }
    code_t<W> q;
    if (W == 32) {
      q = (code_t<W>)(__brev(transpose32c(xl, tc)) >> (32 - B));
    } else {
      const uint64_t lo = transpose32(xl, lane), hi = transpose32(xh, lane);
      q = (code_t<W>)(__brevll((unsigned long long)(lo | (hi << 32))) >> (64 - B));
    }
    qs[jj] = q;
    if (generic) {
      if constexpr (W == 32) rec[jj] = sign_rank32(xl, msb_plane<W>(q, B), false, B, ctr, lane, lt);
      else rec[jj] = sign_record(msb_plane<W>(q, B), false, B, wcnt[warp], lane);
    }
  }
  if (generic) {
    if (W == 32) wcnt[warp][lane] = ctr;
    __syncthreads();
    if (threadIdx.x < NP) {
      uint32_t acc = 0;
      for (int w = 0; w < kWarps; w++) {
        woff[w][threadIdx.x] = acc;
        acc += wcnt[w][threadIdx.x];
      }
    }
    __syncthreads();
  }
  // 32-bit codes: lane k holds the first sign bit of plane k for this warp,
  // fetched by each element with one shuffle
  uint32_t pbase = 0;
  if (W == 32 && generic && lane < B) pbase = poff[lane] * 32 + woff[warp][lane];
  VT* op = out + e0 + (int64_t)warp * kWordsPerWarp * 32 + lane;
  [[maybe_unused]] Scale2 dq{1.0f, 1.0f};
  [[maybe_unused]] uint32_t nbm = 0;
  if constexpr (std::is_same<VT, float>::value && W == 32) {
    dq = scale_pair(generic ? s.E - B : s.E - B + 3);
    nbm = (uint32_t)nb_mask(B);
  }
#pragma unroll
  for (int jj = 0; jj < kWordsPerWarp; jj++) {
    const int j = warp * kWordsPerWarp + jj;
    if (j >= nw) continue;
    bool neg = false;
    const uint32_t r = rec[jj];
    if (W == 32) {
      if (generic) {
        const uint32_t base = __shfl_sync(FULL, pbase, r & 31);
        if (r != 0xFFFFFFFFu) {
          const uint32_t bit = base + ((r >> 7) & 8191);
          neg = (sbuf[bit >> 5] >> (bit & 31)) & 1u;
        }
      }
    } else if (generic && r != 0xFFFFFFFFu) {
      const int p = r & 127;
      const uint32_t bit = poff[p] * 32 + woff[warp][p] + ((r >> 7) & 8191);
      neg = (sbuf[bit >> 5] >> (bit & 31)) & 1u;
    }
    if constexpr (std::is_same<VT, float>::value && W == 32) {
      // dequantize<float, 32> with the stream's scaling as two multipliers
      if (generic) {
        const float mag = __fmul_rn(__fmul_rn(__uint2float_rn((uint32_t)qs[jj]), dq.m1), dq.m2);
        op[jj * 32] = neg ? -mag : mag;
      } else {
        const int64_t val = (int64_t)((uint64_t)((uint32_t)qs[jj] ^ nbm)) - (int64_t)nbm;
        op[jj * 32] = __fmul_rn(__fmul_rn(__int2float_rn((int)val), dq.m1), dq.m2);
      }
    } else {
      op[jj * 32] = dequantize<VT, W>(qs[jj], neg, s);
    }
  }
}

// --------------------------------------------------------------------------
// host-callable launchers
// --------------------------------------------------------------------------
static int grid_for(int64_t n, int threads = 256) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 148 * 64) g = 148 * 64;
  return (int)(g < 1 ? 1 : g);
}

void launch_minmax(int vk, const void* x, int64_t n, FieldStats* st, cudaStream_t s) {
  count_launch();
  count_launch();
  int g = grid_for(n, 512);
  if (g > 148 * 4) g = 148 * 4;
  if (vk == VK_F32) k_minmax<float><<<g, 512, 0, s>>>((const float*)x, n, st);
  else k_minmax<double><<<g, 512, 0, s>>>((const double*)x, n, st);
  k_stats_finalize<<<1, 1, 0, s>>>(st);
}

// zeroing (src null) or copying of many word ranges in one launch
constexpr int kMaxWordsItems = 512;
struct WordsBatch {
  int n;
  int64_t first[kMaxWordsItems + 1];
  WordsItem it[kMaxWordsItems];
};
static_assert(sizeof(WordsBatch) <= 32764, "kernel parameter block");

__global__ void __launch_bounds__(256) k_words_multi(const __grid_constant__ WordsBatch b) {
  const int i = batch_find(b.first, b.n);
  const WordsItem& t = b.it[i];
  const int64_t nblk = b.first[i + 1] - b.first[i];
  for (int64_t e = (blockIdx.x - b.first[i]) * (int64_t)blockDim.x + threadIdx.x; e < t.words;
       e += nblk * (int64_t)blockDim.x)
    t.dst[e] = t.src ? t.src[e] : 0u;
}

void launch_words_multi(const WordsItem* items, int n, cudaStream_t s) {
  int k = 0;
  while (k < n) {
    WordsBatch b{};
    int64_t tot = 0;
    for (; k < n && b.n < kMaxWordsItems; k++) {
      if (items[k].words <= 0) continue;
      b.first[b.n] = tot;
      b.it[b.n++] = items[k];
      tot += std::min<int64_t>((items[k].words + 255) / 256, 148 * 4);
    }
    b.first[b.n] = tot;
    if (!tot) continue;
    count_launch();
    k_words_multi<<<(unsigned)tot, 256, 0, s>>>(b);
  }
}

// ---- batched launchers: items of one value kind, split into launches of at
// most kMaxBatchItems; each item gets blocks in proportion to its size (a
// single item takes the one-field kernel)
void launch_to_fixed(int vk, const void* x, const FieldD& f, const FieldStats* st, int64_t* xc, cudaStream_t s);
void launch_coef_fixed(const FieldD& f, int level, int raw, const LatD& lat, const int64_t* xc, int64_t* out,
                       unsigned long long* vmax, cudaStream_t s);

static int64_t blocks_for(int64_t n, int threads = 256, int64_t cap = 148 * 8) {
  return std::max<int64_t>(1, std::min<int64_t>((n + threads - 1) / threads, cap));
}

// minimum / maximum / finiteness of several fields (no exponent yet)
void launch_minmax_multi(int vk, const void* const* xs, const int64_t* ns, FieldStats* const* sts, int n,
                         cudaStream_t s) {
  if (n == 1) {
    count_launch();
    int g = grid_for(ns[0], 512);
    if (g > 148 * 4) g = 148 * 4;
    if (vk == VK_F32) k_minmax<float><<<g, 512, 0, s>>>((const float*)xs[0], ns[0], sts[0]);
    else k_minmax<double><<<g, 512, 0, s>>>((const double*)xs[0], ns[0], sts[0]);
    return;
  }
  for (int k0 = 0; k0 < n; k0 += kMaxBatchItems) {
    MinmaxBatch b{};
    int64_t tot = 0;
    for (int k = k0; k < n && b.n < kMaxBatchItems; k++) {
      b.first[b.n] = tot;
      b.x[b.n] = xs[k];
      b.cnt[b.n] = ns[k];
      b.st[b.n] = sts[k];
      b.n++;
      tot += blocks_for(ns[k], 512, 148 * 4);
    }
    b.first[b.n] = tot;
    count_launch();
    if (vk == VK_F32) k_minmax_multi<float><<<(unsigned)tot, 512, 0, s>>>(b);
    else k_minmax_multi<double><<<(unsigned)tot, 512, 0, s>>>(b);
  }
}

// the exponent G of each field from its completed minimum and maximum
void launch_finalize_multi(FieldStats* const* sts, int n, cudaStream_t s) {
  if (n == 1) {
    count_launch();
    k_stats_finalize<<<1, 1, 0, s>>>(sts[0]);
    return;
  }
  for (int k0 = 0; k0 < n; k0 += kMaxBatchItems) {
    MinmaxBatch b{};
    for (int k = k0; k < n && b.n < kMaxBatchItems; k++) b.st[b.n++] = sts[k];
    count_launch();
    k_stats_finalize_multi<<<(b.n + 63) / 64, 64, 0, s>>>(b);
  }
}

void launch_stats_multi(int vk, const void* const* xs, const int64_t* ns, FieldStats* const* sts, int n,
                        cudaStream_t s) {
  launch_minmax_multi(vk, xs, ns, sts, n, s);
  launch_finalize_multi(sts, n, s);
}

void launch_to_fixed_multi(int vk, const void* const* xs, const FieldD* fs, const FieldStats* const* sts,
                           int64_t* const* xcs, int n, cudaStream_t s) {
  if (n == 1) {
    launch_to_fixed(vk, xs[0], fs[0], sts[0], xcs[0], s);
    return;
  }
  for (int k0 = 0; k0 < n; k0 += kMaxBatchItems) {
    ToFixedBatch b{};
    int64_t tot = 0;
    for (int k = k0; k < n && b.n < kMaxBatchItems; k++) {
      b.first[b.n] = tot;
      b.x[b.n] = xs[k];
      b.f[b.n] = fs[k];
      b.st[b.n] = sts[k];
      b.xc[b.n] = xcs[k];
      b.n++;
      tot += blocks_for(fs[k].nc[0] * fs[k].nc[1] * fs[k].nc[2]);
    }
    b.first[b.n] = tot;
    count_launch();
    if (vk == VK_F32) k_to_fixed_multi<float><<<(unsigned)tot, 256, 0, s>>>(b);
    else k_to_fixed_multi<double><<<(unsigned)tot, 256, 0, s>>>(b);
  }
}

void launch_coarsest_multi(const FieldD* fs, const int* levels, const LatD* lats, const int64_t* const* xcs,
                           int64_t* const* outs, unsigned long long* const* vmaxs, int n, cudaStream_t s) {
  if (n == 1) {
    launch_coef_fixed(fs[0], levels[0], 1, lats[0], xcs[0], outs[0], vmaxs[0], s);
    return;
  }
  for (int k0 = 0; k0 < n; k0 += kMaxBatchItems) {
    CoefFixedBatch b{};
    int64_t tot = 0;
    for (int k = k0; k < n && b.n < kMaxBatchItems; k++) {
      const int64_t m = lats[k].count[0] * lats[k].count[1] * lats[k].row_pad;
      if (!m) continue;
      b.first[b.n] = tot;
      b.f[b.n] = fs[k];
      b.lat[b.n] = lats[k];
      b.level[b.n] = levels[k];
      b.xc[b.n] = xcs[k];
      b.out[b.n] = outs[k];
      b.vmax[b.n] = vmaxs[k];
      b.n++;
      tot += blocks_for(m);
    }
    b.first[b.n] = tot;
    if (!tot) continue;
    count_launch();
    k_coef_fixed_multi<<<(unsigned)tot, 256, 0, s>>>(b);
  }
}

void launch_to_fixed(int vk, const void* x, const FieldD& f, const FieldStats* st, int64_t* xc,
                     cudaStream_t s) {
  count_launch();
  const int64_t n = f.nc[0] * f.nc[1] * f.nc[2];
  if (vk == VK_F32) k_to_fixed<float><<<grid_for(n), 256, 0, s>>>((const float*)x, f, st, xc);
  else k_to_fixed<double><<<grid_for(n), 256, 0, s>>>((const double*)x, f, st, xc);
}

void launch_coef_fixed(const FieldD& f, int level, int raw, const LatD& lat, const int64_t* xc,
                       int64_t* out, unsigned long long* vmax, cudaStream_t s) {
  const int64_t n = lat.count[0] * lat.count[1] * lat.row_pad;
  if (n == 0) return;
  count_launch();
  k_coef_fixed<<<grid_for(n), 256, 0, s>>>(f, level, raw, lat, xc, out, vmax);
}

void launch_coef_l0(int vk, const FieldD& f, const LatD& lat, int compact, const void* x, void* out,
                    unsigned long long* vmax, unsigned long long* c0, cudaStream_t s) {
  const int64_t n = lat.count[0] * lat.count[1] * (compact ? lat.count[2] : lat.row_pad);
  if (n == 0) return;
  count_launch();
  if (vk == VK_F32)
    k_coef_l0<float><<<grid_for(n), 256, 0, s>>>(f, lat, compact, (const float*)x, (float*)out, vmax, c0);
  else
    k_coef_l0<double><<<grid_for(n), 256, 0, s>>>(f, lat, compact, (const double*)x, (double*)out, vmax, c0);
}

void launch_raw_stage(int vk, const FieldD& f, const LatD& lat, const void* x, void* out,
                      unsigned long long* vmax, cudaStream_t s) {
  count_launch();
  const int64_t n = lat.count[0] * lat.count[1] * lat.row_pad;
  if (vk == VK_F32) k_raw_stage<float><<<grid_for(n), 256, 0, s>>>(f, lat, (const float*)x, (float*)out, vmax);
  else k_raw_stage<double><<<grid_for(n), 256, 0, s>>>(f, lat, (const double*)x, (double*)out, vmax);
}

void launch_decompose(int vk, const DecompGeo& dg, const LatD& sl, const void* comp, void* out,
                      unsigned long long* vmax, cudaStream_t s) {
  const int64_t n = sl.count[0] * sl.count[1] * sl.row_pad;
  if (n == 0) return;
  count_launch();
  if (vk == VK_F32)
    k_decompose<float><<<grid_for(n), 256, 0, s>>>(dg, sl, (const float*)comp, (float*)out, vmax);
  else
    k_decompose<double><<<grid_for(n), 256, 0, s>>>(dg, sl, (const double*)comp, (double*)out, vmax);
}

void launch_recompose(int vk, const DecompGeo& dg, const LatD& sl, const void* dec, void* comp,
                      cudaStream_t s) {
  const int64_t n = sl.count[0] * sl.count[1] * sl.count[2];
  if (n == 0) return;
  count_launch();
  if (vk == VK_F32) k_recompose<float><<<grid_for(n), 256, 0, s>>>(dg, sl, (const float*)dec, (float*)comp);
  else k_recompose<double><<<grid_for(n), 256, 0, s>>>(dg, sl, (const double*)dec, (double*)comp);
}

void launch_recon_fixed(const FieldD& f, int level, int raw, const LatD& lat, const int64_t* chat,
                        int64_t* xc, cudaStream_t s) {
  const int64_t n = lat.count[0] * lat.count[1] * lat.count[2];
  if (n == 0) return;
  count_launch();
  k_recon_fixed<<<grid_for(n), 256, 0, s>>>(f, level, raw, lat, chat, xc);
}

void launch_coarse_out(int vk, const FieldD& f, const int64_t* xc, double scale, void* out, cudaStream_t s,
                       const Box3* box) {
  Box3 b;
  for (int k = 0; k < 3; k++) {
    b.lo[k] = box ? box->lo[k] : 0;
    b.cnt[k] = box ? box->cnt[k] : f.nc[k];
  }
  const int64_t n = b.cnt[0] * b.cnt[1] * b.cnt[2];
  if (n <= 0) return;
  count_launch();
  if (vk == VK_F32) k_coarse_out<float><<<grid_for(n), 256, 0, s>>>(f, xc, (float)scale, (float*)out, b);
  else k_coarse_out<double><<<grid_for(n), 256, 0, s>>>(f, xc, scale, (double*)out, b);
}

void launch_copy_box(int vk, const FieldD& f, const void* src, void* dst, const Box3& b, cudaStream_t s) {
  const int64_t n = b.cnt[0] * b.cnt[1] * b.cnt[2];
  if (n <= 0) return;
  count_launch();
  if (vk == VK_F32) k_copy_box<float><<<grid_for(n), 256, 0, s>>>(f, (const float*)src, (float*)dst, b);
  else k_copy_box<double><<<grid_for(n), 256, 0, s>>>(f, (const double*)src, (double*)dst, b);
}

void launch_recon_l0(int vk, const FieldD& f, const LatD& lat, int compact, const void* chat, void* out,
                     cudaStream_t s) {
  const int64_t n = lat.count[0] * lat.count[1] * lat.count[2];
  if (n == 0) return;
  count_launch();
  if (vk == VK_F32) k_recon_l0<float><<<grid_for(n), 256, 0, s>>>(f, lat, compact, (const float*)chat, (float*)out);
  else k_recon_l0<double><<<grid_for(n), 256, 0, s>>>(f, lat, compact, (const double*)chat, (double*)out);
}

void launch_copy_raw(int vk, const FieldD& f, const LatD& lat, const void* vals, void* out, cudaStream_t s) {
  count_launch();
  const int64_t n = lat.count[0] * lat.count[1] * lat.count[2];
  if (vk == VK_F32) k_copy_raw<float><<<grid_for(n), 256, 0, s>>>(f, lat, (const float*)vals, (float*)out);
  else k_copy_raw<double><<<grid_for(n), 256, 0, s>>>(f, lat, (const double*)vals, (double*)out);
}

// ---------------------------------------------------------------------------
// Persistent encoder for streams with 32-bit codes whose tables need no
// plane-pair counts: FP32 streams and fixed-point streams (Sec. V-C
// bitplanes, Sec. VI-A encodings).  Same planes, sign sub-streams, counts
// and tables as k_encode; organised for throughput:
//  * each CTA loops over work items; the next segment's values (16 KB FP32,
//    32 KB fixed point) are copied into shared memory with cp.async while the
//    current one is coded;
//  * sign ranks come from the transposed planes: F_k = D_k & ~(D_0 | .. |
//    D_{k-1}) marks the elements first significant at plane k; the word's
//    signs sorted by (plane, element) are one warp OR-reduction, and lane k
//    appends its slice of that word to plane k's per-warp bit string;
//  * plane words leave in 16-byte stores from rows of 132 words.
// ---------------------------------------------------------------------------
constexpr int kEncRow = kSegWords + 4;            // pbuf row (16-byte multiple, bank-spread)


__device__ __forceinline__ void cp_async16(uint32_t* smem, const void* gmem, int src_bytes) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// start the copy of one segment's staged values (zero fill past the stream)
template <typename VT>
__device__ __forceinline__ void enc_fetch(uint32_t* buf, const VT* stage, int64_t e0, int64_t n_pad) {
  constexpr int PER = 16 / sizeof(VT);           // values per 16-byte chunk
  const int64_t avail = n_pad - e0;              // elements of the stream from e0 (multiple of 32)
  for (int c = threadIdx.x; c < kSegElems / PER; c += kThreads) {
    const bool ok = (int64_t)c * PER < avail;
    cp_async16(buf + c * 4, ok ? (const void*)(stage + e0 + c * PER) : (const void*)(stage), ok ? 16 : 0);
  }
}

// sign bit-string of plane `lane` in this warp: index of word i in the
// warp's 32 x 16 buffer (swizzled so that lanes flushing the same word index
// hit different banks)
__device__ __forceinline__ int sb_index(int lane, int i) { return lane * 16 + (i ^ ((lane >> 1) & 15)); }

// two input buffers + plane rows (value type VT: 4 or 8 bytes)
template <typename VT>
constexpr int enc_dyn_smem() { return (2 * kSegElems * (int)(sizeof(VT) / 4) + 32 * kEncRow) * 4; }

// PAIRS (PSNR-mode streams): also the plane-pair counts of the exact
// squared-error tables, sum over values of d_a d_c for planes a <= c: per
// word lane a adds popc(D_a & D_(a+t)) for t = 0..16 (rotated lanes cover
// every unordered pair once, t = 16 only from the lower half), folded into
// shared counts per segment and added to the stream's table.
template <typename VT, bool PAIRS>
__global__ void __launch_bounds__(kThreads, PAIRS ? 2 : 4) k_encode_w32(const StreamD* __restrict__ streams,
                                                                        const WorkItem* __restrict__ items,
                                                                        int nitems) {
  constexpr int VW = sizeof(VT) / 4;   // 32-bit words per staged value
  extern __shared__ __align__(16) uint32_t enc_dyn[];
  uint32_t* const pbuf = enc_dyn + 2 * kSegElems * VW;
  __shared__ uint32_t sbuf[kSegWords + 64];
  __shared__ uint32_t wcnt[kWarps][32];
  __shared__ uint32_t woff[kWarps][32];
  __shared__ uint32_t poff[33];
  __shared__ uint32_t pnz[32];
  __shared__ uint32_t pairs_s[PAIRS ? 32 * 33 / 2 : 1];

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const TrC tc = tr_consts(lane);
  const uint32_t lt = (1u << lane) - 1u;

  int item = blockIdx.x;
  if (item >= nitems) return;
  if (threadIdx.x < 32) pnz[threadIdx.x] = 0;
  if constexpr (PAIRS)
    for (int i = threadIdx.x; i < 32 * 33 / 2; i += kThreads) pairs_s[i] = 0;
  [[maybe_unused]] uint32_t acc_p[PAIRS ? 17 : 1];
  if constexpr (PAIRS) {
#pragma unroll
    for (int t = 0; t < 17; t++) acc_p[t] = 0;
  }
  for (int i = threadIdx.x; i < kSegWords + 64; i += kThreads) sbuf[i] = 0;
  // the current item's stream fields needed to fetch it, and the next one's
  WorkItem it = items[item];
  {
    const StreamD& s0 = streams[it.stream];
    enc_fetch(enc_dyn, (const VT*)s0.stage, (int64_t)it.seg * kSegElems, s0.n_pad);
    cp_async_commit();
  }
  int nitem = item + gridDim.x;
  WorkItem nit = nitem < nitems ? items[nitem] : WorkItem{0, 0};
  const VT* nstage = nullptr;
  int64_t nn_pad = 0;
  if (nitem < nitems) {
    nstage = (const VT*)streams[nit.stream].stage;
    nn_pad = streams[nit.stream].n_pad;
  }

  for (int cur = 0; item < nitems; cur ^= 1) {
    // (A) the next item's values start moving; the one after is located
    if (nitem < nitems)
      enc_fetch(enc_dyn + (cur ^ 1) * kSegElems * VW, nstage, (int64_t)nit.seg * kSegElems, nn_pad);
    cp_async_commit();
    const int item2 = nitem + gridDim.x;
    WorkItem it2{0, 0};
    const VT* stage2 = nullptr;
    int64_t n_pad2 = 0;
    if (item2 < nitems) {
      it2 = items[item2];
      stage2 = (const VT*)streams[it2.stream].stage;
      n_pad2 = streams[it2.stream].n_pad;
    }
    const StreamD& s = streams[it.stream];
    const int B = s.B;
    const bool generic = s.enc == 1;
    const QParams qp = qparams(s);
    // quantisation (the arithmetic of quantize<VT, 32>) with per-item constants
    [[maybe_unused]] Scale2 sc{1.0f, 1.0f};
    if constexpr (std::is_same<VT, float>::value) sc = scale_pair(generic ? B - qp.E : B - 3 - qp.E);
    const uint32_t M = (uint32_t)nb_mask(B);
    const int64_t e0 = (int64_t)it.seg * kSegElems;
    const int nw = (int)min((int64_t)kSegWords, (s.n_pad - e0) / 32);

    // (B) this item's values have landed (S1)
    cp_async_wait<1>();
    __syncthreads();

    // (C) code this warp's 16 words
    uint32_t* wbuf = enc_dyn + (cur * kSegElems + warp * kWordsPerWarp * 32) * VW;
    // FP32: the values; fixed point: the codes and signs right away (the
    // arithmetic of quantize<int64_t, 32>), 32 bits per value in registers
    [[maybe_unused]] float v[std::is_same<VT, float>::value ? kWordsPerWarp : 1];
    [[maybe_unused]] uint32_t qv[std::is_same<VT, float>::value ? 1 : kWordsPerWarp];
    [[maybe_unused]] uint32_t negm = 0;
    if constexpr (std::is_same<VT, float>::value) {
#pragma unroll
      for (int jj = 0; jj < kWordsPerWarp; jj++) v[jj] = __uint_as_float(wbuf[jj * 32 + lane]);
    } else {
      const int64_t* wv = reinterpret_cast<const int64_t*>(wbuf);
#pragma unroll
      for (int jj = 0; jj < kWordsPerWarp; jj++) {
        const int64_t x = wv[jj * 32 + lane];
        const bool ng = x < 0;
        const uint64_t mag = (uint64_t)(ng ? -x : x) >> qp.sh;
        const int64_t sv = ng ? -(int64_t)mag : (int64_t)mag;
        qv[jj] = generic ? (uint32_t)mag : (((uint32_t)sv + M) ^ M);
        negm |= (uint32_t)ng << jj;
      }
    }
    __syncwarp();                       // the warp's region now holds its sign bit-strings
    uint32_t acc = 0, fill = 0, wpos = 0, count = 0, nz = 0;
    // the word loop, instantiated per encoding (the test then runs once)
    auto words = [&](auto gen_tag) {
      constexpr bool GEN = decltype(gen_tag)::value;
      uint32_t pw[4];
#pragma unroll
      for (int jj = 0; jj < kWordsPerWarp; jj++) {
        bool neg;
        uint32_t q;
        if constexpr (std::is_same<VT, float>::value) {
          neg = v[jj] < 0.0f;
          if constexpr (GEN) {
            q = __float2uint_rz(__fmul_rn(__fmul_rn(fabsf(v[jj]), sc.m1), sc.m2));
          } else {
            const int sv = __float2int_rz(__fmul_rn(__fmul_rn(v[jj], sc.m1), sc.m2));
            q = ((uint32_t)sv + M) ^ M;
          }
        } else {
          neg = (negm >> jj) & 1u;
          q = qv[jj];
        }
        if (qp.zero) q = 0;
        const uint32_t xr = q << (32 - B);
        const uint32_t x = __brev(xr);                   // bit t = plane t (from the top)
        const uint32_t D = transpose32c(x, tc);           // lane k: plane k of the 32 values
        if constexpr (PAIRS) {
#pragma unroll
          for (int t = 0; t < 17; t++) acc_p[t] += __popc(D & __shfl_sync(FULL, D, (lane + t) & 31));
        }
        uint32_t sl = D;
        if constexpr (!GEN) {
          const uint32_t up = __shfl_up_sync(FULL, D, 1);
          sl = lane ? D ^ up : D;
        }
        pw[jj & 3] = sl;
        if ((jj & 3) == 3 && lane < B)
          *reinterpret_cast<uint4*>(&pbuf[lane * kEncRow + warp * kWordsPerWarp + (jj & ~3)]) =
              make_uint4(pw[0], pw[1], pw[2], pw[3]);
        nz += sl != 0;
        if constexpr (GEN) {
          // planes above k that hold a one, per element (inclusive prefix OR)
          uint32_t inc = D;
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) inc |= __shfl_up_sync(FULL, inc, o);
          uint32_t exc = __shfl_up_sync(FULL, inc, 1);
          exc = lane ? exc : 0u;
          const uint32_t F = D & ~exc;                   // first significant at plane `lane`
          const uint32_t cnt = __popc(F), start = __popc(exc);
          // this element's place in the word's signs sorted by (plane, element)
          const int pe = __clz(xr) & 31;                 // its plane (any lane when q == 0)
          const uint32_t Fp = __shfl_sync(FULL, F, pe);
          const uint32_t sp = __shfl_sync(FULL, start, pe);
          const uint32_t dest = sp + __popc(Fp & lt);
          const uint32_t sorted = __reduce_or_sync(FULL, (neg && xr) ? (1u << dest) : 0u);
          // lane k: its plane's slice [start, start + cnt), appended to the plane's bit-string
          const uint32_t bits = __funnelshift_rc(sorted, 0u, start) & __funnelshift_lc(~0u, 0u, cnt);
          acc |= bits << fill;
          const uint32_t nf = fill + cnt;
          if (nf >= 32) {
            wbuf[sb_index(lane, wpos)] = acc;
            wpos++;
            acc = __funnelshift_rc(bits, 0u, 32 - fill);   // the part that did not fit (none if fill == 0)
          }
          fill = nf & 31;
          count += cnt;
        }
      }
    };
    if (generic) words(std::true_type{});
    else words(std::false_type{});
    if (generic) {
      if (fill) wbuf[sb_index(lane, wpos)] = acc;
      wcnt[warp][lane] = count;
    }
    if (lane < B && nz) atomicAdd(&pnz[lane], nz);
    if constexpr (PAIRS) {
#pragma unroll
      for (int t = 0; t < 17; t++) {
        const int b2 = (lane + t) & 31;
        if ((t < 16 || lane < 16) && acc_p[t]) atomicAdd(&pairs_s[tri<32>(min(lane, b2), max(lane, b2))], acc_p[t]);
        acc_p[t] = 0;
      }
    }
    __syncthreads();   // S2
    // (D) sign layout of the segment, then each plane's bit-strings in place
    if (generic) {
      if (warp == 0) sign_layout32(wcnt, woff, poff, B, lane);
      __syncthreads();   // S3
      if (count) {
        const uint32_t O = poff[lane] * 32 + woff[warp][lane];
        const uint32_t sh = O & 31, base = O >> 5, nwd = (count + 31) >> 5;
        for (uint32_t i = 0; i < nwd; i++) {
          const uint32_t w = wbuf[sb_index(lane, i)];
          atomicOr(&sbuf[base + i], w << sh);
          if (sh) {
            const uint32_t hi = w >> (32 - sh);
            if (hi) atomicOr(&sbuf[base + i + 1], hi);
          }
        }
      }
      __syncthreads();   // S4
      uint32_t* dst = s.signs + (int64_t)it.seg * s.slot_words;
      for (int i = threadIdx.x; i < (int)poff[B]; i += kThreads) dst[i] = sbuf[i];
      if (threadIdx.x < B) {
        const uint32_t c = wcnt[0][threadIdx.x];
        s.sign_counts[(int64_t)it.seg * B + threadIdx.x] = c;
        if (c) atomicAdd(&s.plane_nz[B + threadIdx.x], (c + 31) >> 5);
      }
    }
    // (E) plane words, four at a time where the rows allow it
    {
      const int64_t w0 = (int64_t)it.seg * kSegWords;
      const bool vec = ((s.words & 3) == 0) && ((((uintptr_t)s.planes) & 15) == 0);
      for (int c = threadIdx.x; c < B * (kSegWords / 4); c += kThreads) {
        const int k = c >> 5, j = (c & 31) * 4;
        if (j >= nw) continue;
        const uint4 w4 = *reinterpret_cast<const uint4*>(&pbuf[k * kEncRow + j]);
        uint32_t* g = s.planes + (int64_t)k * s.words + w0 + j;
        if (vec && j + 4 <= nw) {
          *reinterpret_cast<uint4*>(g) = w4;
        } else {
          g[0] = w4.x;
          if (j + 1 < nw) g[1] = w4.y;
          if (j + 2 < nw) g[2] = w4.z;
          if (j + 3 < nw) g[3] = w4.w;
        }
      }
      if (threadIdx.x < B && pnz[threadIdx.x]) atomicAdd(&s.plane_nz[threadIdx.x], pnz[threadIdx.x]);
      if constexpr (PAIRS) {
        for (int i = threadIdx.x; i < 32 * 32; i += kThreads) {
          const int a = i >> 5, c = i & 31;
          if (a <= c && c < B && pairs_s[tri<32>(a, c)])
            atomicAdd(&s.pairs[a * B + c], (unsigned long long)pairs_s[tri<32>(a, c)]);
        }
      }
    }
    // (F) every read of this item's shared memory is done (S5): clear for the next
    __syncthreads();
    if (threadIdx.x < 32) pnz[threadIdx.x] = 0;
    if constexpr (PAIRS)
      for (int i = threadIdx.x; i < 32 * 33 / 2; i += kThreads) pairs_s[i] = 0;
    for (int i = threadIdx.x; i < kSegWords + 64; i += kThreads) sbuf[i] = 0;
    item = nitem;
    it = nit;
    nitem = item2;
    nit = it2;
    nstage = stage2;
    nn_pad = n_pad2;
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Decoder for streams with 32-bit codes: one warp per segment, one pass, no
// shared memory (Sec. V-C bitplanes, Sec. VI-A encodings).  Lane k reads
// plane k's words of the segment directly (16-byte loads where the rows
// allow) and, for the generic encoding, plane k's sign sub-stream through a
// two-word bit reader.  Per word, the planes give F_k (values first
// significant at plane k, a prefix OR over lanes) and lane k takes the
// next |F_k| bits of its sign sub-stream; a value first significant at
// plane k reads its sign from lane k's slice at its rank in F_k.
// ---------------------------------------------------------------------------
template <typename VT>
__global__ void __launch_bounds__(kThreads) k_decode_w32(const StreamD* __restrict__ streams,
                                                         const WorkItem* __restrict__ items, int nitems) {
  const int lane = threadIdx.x & 31;
  const int item = (int)((blockIdx.x * (unsigned)blockDim.x + threadIdx.x) >> 5);
  if (item >= nitems) return;                       // whole warps
  const WorkItem it = items[item];
  const StreamD& s = streams[it.stream];
  const int B = s.B, b = s.b;
  const bool generic = s.enc == 1;
  const int64_t e0 = (int64_t)it.seg * kSegElems;
  const int nw = (int)min((int64_t)kSegWords, (s.n_pad - e0) / 32);
  const int64_t w0 = (int64_t)it.seg * kSegWords;
  VT* out = (VT*)s.stage + e0 + lane;
  const TrC tc = tr_consts(lane);
  const uint32_t lt = (1u << lane) - 1u;

  // this lane's plane row (planes >= b, and planes with no nonzero word in
  // the stream, read as zeros)
  const bool has = lane < b && s.plane_nz[lane] != 0;
  const uint32_t* row = s.planes + (int64_t)(has ? lane : 0) * s.words + w0;
  const bool vec = ((s.words & 3) == 0) && ((((uintptr_t)s.planes) & 15) == 0);

  // this lane's sign sub-stream: first word = exclusive prefix of the
  // planes' word counts over the lanes
  uint32_t win = 0, nxt = 0, pos = 0, idx = 2, nwords = 0;
  const uint32_t* sp = s.signs + (int64_t)it.seg * s.slot_words;
  if (generic) {
    const uint32_t cntk = lane < B ? s.sign_counts[(int64_t)it.seg * B + lane] : 0u;
    const uint32_t words = (cntk + 31) >> 5;
    uint32_t inc = words;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(FULL, inc, o);
      inc += lane >= o ? t : 0u;
    }
    sp += inc - words;
    nwords = lane < b ? words : 0u;
    if (nwords > 0) win = __ldg(sp);
    if (nwords > 1) nxt = __ldg(sp + 1);
  }
  // dequantisation constants (dequantize<VT, 32>)
  [[maybe_unused]] Scale2 dq{1.0f, 1.0f};
  const uint32_t nbm = (uint32_t)nb_mask(B);
  if constexpr (std::is_same<VT, float>::value) dq = scale_pair(generic ? s.E - B : s.E - B + 3);

  auto load4 = [&](int j) -> uint4 {
    if (!has || j >= nw) return make_uint4(0u, 0u, 0u, 0u);
    if (vec && j + 4 <= nw) return __ldg(reinterpret_cast<const uint4*>(row + j));
    uint4 g;
    g.x = __ldg(row + j);
    g.y = j + 1 < nw ? __ldg(row + j + 1) : 0u;
    g.z = j + 2 < nw ? __ldg(row + j + 2) : 0u;
    g.w = j + 3 < nw ? __ldg(row + j + 3) : 0u;
    return g;
  };

  // the word loop, instantiated per encoding and for whole / ragged segments
  // (neither test then runs per word)
  auto words = [&](auto gen_tag, auto whole_tag) {
    constexpr bool GEN = decltype(gen_tag)::value;
    constexpr bool WHOLE = decltype(whole_tag)::value;
    const int nwl = WHOLE ? kSegWords : nw;
    uint4 g = load4(0);
    for (int j4 = 0; j4 < nwl; j4 += 4) {
      const uint4 gn = load4(j4 + 4);               // next group in flight
#pragma unroll
      for (int e4 = 0; e4 < 4; e4++) {
        const int j = j4 + e4;
        if (!WHOLE && j >= nwl) break;
        uint32_t xl = e4 == 0 ? g.x : e4 == 1 ? g.y : e4 == 2 ? g.z : g.w;
        if constexpr (!GEN) {                       // negabinary planes are stored XOR-differenced
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(FULL, xl, o);
            if (lane >= o) xl ^= t;
          }
          if (lane >= b) xl = 0;
        }
        const uint32_t q = __brev(transpose32c(xl, tc)) >> (32 - B);
        bool neg = false;
        if constexpr (GEN) {
          uint32_t inc = xl;                        // a one in planes 0..lane
#pragma unroll
          for (int o = 1; o < 32; o <<= 1) inc |= __shfl_up_sync(FULL, inc, o);
          uint32_t exc = __shfl_up_sync(FULL, inc, 1);
          exc = lane ? exc : 0u;
          const uint32_t F = xl & ~exc;
          const uint32_t cnt = __popc(F);
          // the next cnt bits of this plane's signs
          const uint32_t slice = __funnelshift_r(win, nxt, pos) & __funnelshift_lc(~0u, 0u, cnt);
          pos += cnt;
          if (pos >= 32) {
            win = nxt;
            nxt = idx < nwords ? __ldg(sp + idx) : 0u;
            idx++;
            pos -= 32;
          }
          // a value's sign: bit (its rank among the values first significant
          // at its plane) of that plane's slice
          const uint32_t xr = q << (32 - B);
          const int pe = __clz(xr) & 31;
          const uint32_t Fp = __shfl_sync(FULL, F, pe);
          const uint32_t Sp = __shfl_sync(FULL, slice, pe);
          neg = xr && ((Sp >> __popc(Fp & lt)) & 1u);
        }
        if constexpr (std::is_same<VT, float>::value) {
          if constexpr (GEN) {
            const float mag = __fmul_rn(__fmul_rn(__uint2float_rn(q), dq.m1), dq.m2);
            out[(int64_t)j * 32] = neg ? -mag : mag;
          } else {
            const int64_t val = (int64_t)((uint64_t)(q ^ nbm)) - (int64_t)nbm;
            out[(int64_t)j * 32] = __fmul_rn(__fmul_rn(__int2float_rn((int)val), dq.m1), dq.m2);
          }
        } else {
          out[(int64_t)j * 32] = dequantize<VT, 32>(q, neg, s);
        }
      }
      g = gn;
    }
  };
  if (generic) {
    if (nw == kSegWords) words(std::true_type{}, std::true_type{});
    else words(std::true_type{}, std::false_type{});
  } else {
    if (nw == kSegWords) words(std::false_type{}, std::true_type{});
    else words(std::false_type{}, std::false_type{});
  }
}

// persistent grid of k_encode_w32: the CTAs that fit on the device at once
template <typename VT, bool PAIRS>
static int enc_w32_grid(int nitems) {
  static int cached[64] = {0};
  int dev = 0;
  cudaGetDevice(&dev);
  int& g = cached[dev & 63];
  if (g == 0) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaFuncSetAttribute(k_encode_w32<VT, PAIRS>, cudaFuncAttributeMaxDynamicSharedMemorySize, enc_dyn_smem<VT>());
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_encode_w32<VT, PAIRS>, kThreads, enc_dyn_smem<VT>());
    g = max(1, sms * max(per, 1));
  }
  return min(nitems, g);
}

// vk: value kind of the streams in this work list; w64: FP64-field word path
void launch_encode(int vk, int w64, int pairs, const StreamD* d_streams, const WorkItem* d_items,
                   int nitems, cudaStream_t s) {
  if (nitems == 0) return;
  count_launch();
#define ENC(VT, W, P) k_encode<VT, W, P><<<nitems, kThreads, 0, s>>>(d_streams, d_items)
#define ENC32(VT, P) \
  k_encode_w32<VT, P><<<enc_w32_grid<VT, P>(nitems), kThreads, enc_dyn_smem<VT>(), s>>>(d_streams, d_items, nitems)
  if (!w64) {
    if (vk == VK_F32) {
      if (pairs) ENC32(float, true);
      else ENC32(float, false);
    } else {
      if (pairs) ENC32(int64_t, true);
      else ENC32(int64_t, false);
    }
  } else {
    if (vk == VK_F64) { if (pairs) ENC(double, 64, true); else ENC(double, 64, false); }
    else { if (pairs) ENC(int64_t, 64, true); else ENC(int64_t, 64, false); }
  }
#undef ENC
#undef ENC32
}

void launch_decode(int vk, int w64, const StreamD* d_streams, const WorkItem* d_items, int nitems,
                   cudaStream_t s) {
  if (nitems == 0) return;
  count_launch();
  if (!w64) {
    const int grid = (nitems + kWarps - 1) / kWarps;   // one warp per segment
    if (vk == VK_F32) k_decode_w32<float><<<grid, kThreads, 0, s>>>(d_streams, d_items, nitems);
    else k_decode_w32<int64_t><<<grid, kThreads, 0, s>>>(d_streams, d_items, nitems);
  } else {
    if (vk == VK_F64) k_decode<double, 64><<<nitems, kThreads, 0, s>>>(d_streams, d_items);
    else k_decode<int64_t, 64><<<nitems, kThreads, 0, s>>>(d_streams, d_items);
  }
}

}  // namespace pcr
