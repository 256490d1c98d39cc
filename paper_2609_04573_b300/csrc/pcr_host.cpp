// Host side of the progressive refactor / retrieve library: geometry,
// error tables, bound composition, max ordering, the greedy planner, the
// container and the C ABI (include/pcr.h).  Section references are to
// arXiv 2609.04573 (ProAICD).
#include <new>
#include <queue>
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/pcr.h"
#include "pcr_internal.h"

namespace pcr {
// kernels (pcr_kernels.cu)
void launch_minmax(int vk, const void* x, int64_t n, FieldStats* st, cudaStream_t s);
void launch_to_fixed(int vk, const void* x, const FieldD& f, const FieldStats* st, int64_t* xc, cudaStream_t s);
void launch_coef_fixed(const FieldD& f, int level, int raw, const LatD& lat, const int64_t* xc, int64_t* out,
                       unsigned long long* vmax, cudaStream_t s);
void launch_coef_l0(int vk, const FieldD& f, const LatD& lat, int compact, const void* x, void* out,
                    unsigned long long* vmax, unsigned long long* c0, cudaStream_t s);
void launch_raw_stage(int vk, const FieldD& f, const LatD& lat, const void* x, void* out,
                      unsigned long long* vmax, cudaStream_t s);
void launch_decompose(int vk, const DecompGeo& dg, const LatD& sl, const void* comp, void* out,
                      unsigned long long* vmax, cudaStream_t s);
void launch_recompose(int vk, const DecompGeo& dg, const LatD& sl, const void* dec, void* comp, cudaStream_t s);
void launch_recon_fixed(const FieldD& f, int level, int raw, const LatD& lat, const int64_t* chat, int64_t* xc,
                        cudaStream_t s);
void launch_copy_box(int vk, const FieldD& f, const void* src, void* dst, const Box3& b, cudaStream_t s);
void launch_recon_l0(int vk, const FieldD& f, const LatD& lat, int compact, const void* chat, void* out,
                     cudaStream_t s);
void launch_copy_raw(int vk, const FieldD& f, const LatD& lat, const void* vals, void* out, cudaStream_t s);
void launch_encode(int vk, int w64, int pairs, const StreamD* d_streams, const WorkItem* d_items, int nitems,
                   cudaStream_t s);
void launch_decode(int vk, int w64, const StreamD* d_streams, const WorkItem* d_items, int nitems,
                   cudaStream_t s);
void launch_tile_interp(int vk, const TileArgs& a, cudaStream_t s);
void launch_tile_interp_multi(int vk, const TileArgs* args, int n, cudaStream_t s);
void launch_tile_decomp(int vk, const DecompArgs& a, cudaStream_t s);
void launch_zero_pads_multi(const int* vks, const LatD* lats, void* const* stages, int n, cudaStream_t s);
void launch_tile_decomp_multi(int vk, const DecompArgs* das, int n, cudaStream_t s);
// batched forms over the fields of a batch (pcr_kernels.cu)
void launch_stats_multi(int vk, const void* const* xs, const int64_t* ns, FieldStats* const* sts, int n,
                        cudaStream_t s);
void launch_to_fixed_multi(int vk, const void* const* xs, const FieldD* fs, const FieldStats* const* sts,
                           int64_t* const* xcs, int n, cudaStream_t s);
void launch_coarsest_multi(const FieldD* fs, const int* levels, const LatD* lats, const int64_t* const* xcs,
                           int64_t* const* outs, unsigned long long* const* vmaxs, int n, cudaStream_t s);
void launch_words_multi(const WordsItem* items, int n, cudaStream_t s);
void launch_finalize_multi(FieldStats* const* sts, int n, cudaStream_t s);
// lossless coding of plane words (pcr_pack.cu)
void launch_pack_sizes(const PackTask* tasks, int ntasks, uint32_t* headers, uint32_t* pwords, cudaStream_t s);
void launch_pack_write(const PackTask* tasks, int ntasks, const uint32_t* headers, const uint64_t* offsets,
                       uint32_t* out, cudaStream_t s);
void launch_unpack(const PackTask* tasks, int ntasks, const uint32_t* headers, const uint64_t* offsets,
                   const uint32_t* in, int* err, cudaStream_t s);
}  // namespace pcr

using namespace pcr;

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local std::string g_err;

static pcr_status fail(pcr_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

#define CUDA_TRY(expr)                                                                \
  do {                                                                                \
    cudaError_t _e = (expr);                                                          \
    if (_e != cudaSuccess)                                                            \
      return fail(PCR_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(_e)); \
  } while (0)

extern "C" const char* pcr_last_error(void) { return g_err.c_str(); }

// ---------------------------------------------------------------------------
// tracing: per-stage CUDA-event timing and kernel launch counts
// ---------------------------------------------------------------------------
namespace {
std::mutex g_prof_mu;
bool g_prof_on = false;
struct ProfRec {
  std::string name;
  cudaEvent_t a, b;
  long long launches;
};
std::vector<ProfRec> g_prof_recs;
std::map<std::string, std::pair<double, long long>> g_prof_tot;
std::vector<cudaEvent_t> g_prof_pool;   // events returned by pcr_profile_read, reused

cudaEvent_t prof_event() {
  {
    std::lock_guard<std::mutex> g(g_prof_mu);
    if (!g_prof_pool.empty()) {
      cudaEvent_t e = g_prof_pool.back();
      g_prof_pool.pop_back();
      return e;
    }
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

struct Prof {
  const char* name;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  long long c0;
  Prof(const char* n, cudaStream_t st) : name(n), s(st), c0(launch_count()) {
    if (g_prof_on && (a = prof_event())) cudaEventRecord(a, s);
  }
  ~Prof() {
    const long long dl = launch_count() - c0;
    if (!a) return;
    cudaEvent_t b = prof_event();
    if (!b) return;
    cudaEventRecord(b, s);
    std::lock_guard<std::mutex> g(g_prof_mu);
    g_prof_recs.push_back({name, a, b, dl});
  }
};
}  // namespace

extern "C" pcr_status pcr_profile_enable(int enable) try {
  g_prof_on = enable != 0;
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" int64_t pcr_launch_count(void) { return launch_count(); }

extern "C" pcr_status pcr_profile_read(int max_entries, char* names, double* ms, int64_t* launches, int* n_out,
                                       int reset) try {
  if (!n_out) return fail(PCR_ERR_INVALID_ARG, "null argument");
  std::lock_guard<std::mutex> g(g_prof_mu);
  for (auto& r : g_prof_recs) {
    float t = 0.0f;
    if (cudaEventSynchronize(r.b) == cudaSuccess) cudaEventElapsedTime(&t, r.a, r.b);
    auto& acc = g_prof_tot[r.name];
    acc.first += t;
    acc.second += r.launches;
    g_prof_pool.push_back(r.a);
    g_prof_pool.push_back(r.b);
  }
  g_prof_recs.clear();
  int k = 0;
  for (auto& kv : g_prof_tot) {
    if (k < max_entries) {
      if (names) std::snprintf(names + 48 * k, 48, "%s", kv.first.c_str());
      if (ms) ms[k] = kv.second.first;
      if (launches) launches[k] = kv.second.second;
    }
    k++;
  }
  *n_out = k;
  if (reset) g_prof_tot.clear();
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

// ---------------------------------------------------------------------------
// memory
// ---------------------------------------------------------------------------
namespace {

struct Mem {
  pcr_allocator a{};
  bool user = false;
  void* alloc(size_t bytes, cudaStream_t s) {
    if (bytes == 0) bytes = 16;
    if (user) return a.alloc(a.ctx, bytes, (void*)s);
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void free(void* p, cudaStream_t s) {
    if (!p) return;
    if (user) a.free(a.ctx, p, (void*)s);
    else cudaFreeAsync(p, s);
  }
};

Mem make_mem(const pcr_allocator* a) {
  Mem m;
  if (a && a->alloc && a->free) {
    m.a = *a;
    m.user = true;
  }
  return m;
}

// ---------------------------------------------------------------------------
// geometry (Sec. IV, V-B, V-C): levels, regions, decomposition sub-levels,
// streams as concatenated lattices with rows padded to 32 elements
// ---------------------------------------------------------------------------
int64_t count_from(int64_t n, int64_t start, int64_t step) {
  if (n - 1 < start) return 0;
  return (n - 1 - start) / step + 1;
}

struct Lat {
  int64_t start[3] = {0, 0, 0}, step[3] = {1, 1, 1}, count[3] = {1, 1, 1};
  int64_t row_pad() const { return (count[2] + 31) / 32 * 32; }
  int64_t n_real() const { return count[0] * count[1] * count[2]; }
  int64_t n_pad() const { return count[0] * count[1] * row_pad(); }
};

struct SGeo {
  int level = 0, region = 0, sub = 0;
  bool is_fix = false;
  std::vector<Lat> lats;
  int64_t n_real() const {
    int64_t t = 0;
    for (auto& l : lats) t += l.n_real();
    return t;
  }
  int64_t n_pad() const {
    int64_t t = 0;
    for (auto& l : lats) t += l.n_pad();
    return t;
  }
};

Lat region_lat(const int64_t* n3, int level, const std::vector<int>& order, int r) {
  const int64_t s = int64_t(1) << level;
  Lat l;
  const int a = order[r - 1];
  l.start[a] = s;
  l.step[a] = 2 * s;
  l.count[a] = count_from(n3[a], s, 2 * s);
  for (size_t i = r; i < order.size(); i++) {
    const int b = order[i];
    l.step[b] = 2 * s;
    l.count[b] = count_from(n3[b], 0, 2 * s);
  }
  for (int i = 0; i < r - 1; i++) {
    const int b = order[i];
    l.step[b] = s;
    l.count[b] = count_from(n3[b], 0, s);
  }
  return l;
}

Lat coarse_lat(const int64_t* n3, int L) {
  const int64_t S = int64_t(1) << (L - 1);
  Lat l;
  for (int a = 0; a < 3; a++)
    if (n3[a] > 1) {
      l.step[a] = S;
      l.count[a] = count_from(n3[a], 0, S);
    }
  return l;
}

Lat sub_lat(const Lat& R, int u, int v, int su, int tu, int sv, int tv) {
  Lat l = R;
  const int ax[2] = {u, v};
  const int s0[2] = {su, sv}, t0[2] = {tu, tv};
  for (int i = 0; i < 2; i++) {
    const int a = ax[i];
    l.start[a] = R.start[a] + R.step[a] * s0[i];
    l.step[a] = R.step[a] * t0[i];
    l.count[a] = count_from(R.count[a], s0[i], t0[i]);
  }
  return l;
}

// S1 = 4-grid, S2 = 2-grid minus 4-grid, S3 = the rest; each made of the
// regions of a 2-D per-level hierarchy (odd along u first, then v)
const int kSub[3][2][4] = {{{0, 4, 0, 4}, {-1, 0, 0, 0}},
                           {{2, 4, 0, 4}, {0, 2, 2, 4}},
                           {{1, 2, 0, 2}, {0, 1, 1, 2}}};

std::vector<SGeo> build_streams(const int64_t* n3, int L, int interp, const std::vector<int>& order, int dax) {
  std::vector<SGeo> out;
  SGeo c;
  c.level = L - 1;
  c.is_fix = L - 1 >= 1;
  c.lats.push_back(coarse_lat(n3, L));
  out.push_back(c);
  const int d = (int)order.size();
  for (int level = L - 2; level >= 0; level--) {
    std::vector<Lat> regs;
    for (int r = 1; r <= d; r++) regs.push_back(region_lat(n3, level, order, r));
    if (level == 0 && dax >= 0) {
      int u = -1, v = -1;
      for (int a = 0; a < 3; a++)
        if (a != dax) (u < 0 ? u : v) = a;
      for (int r = 1; r <= d; r++)
        for (int k = 0; k < 3; k++) {
          SGeo g;
          g.level = 0;
          g.region = r;
          g.sub = k + 1;
          for (int part = 0; part < 2; part++) {
            if (kSub[k][part][0] < 0) continue;
            const int* p = kSub[k][part];
            g.lats.push_back(sub_lat(regs[r - 1], u, v, p[0], p[1], p[2], p[3]));
          }
          out.push_back(g);
        }
    } else if (interp == 0) {
      SGeo g;
      g.level = level;
      g.is_fix = level >= 1;
      g.lats = regs;
      out.push_back(g);
    } else {
      for (int r = 1; r <= d; r++) {
        SGeo g;
        g.level = level;
        g.region = r;
        g.is_fix = level >= 1;
        g.lats.push_back(regs[r - 1]);
        out.push_back(g);
      }
    }
  }
  return out;
}

int auto_levels(const int64_t* n3) {
  int64_t m = INT64_MAX;
  for (int a = 0; a < 3; a++)
    if (n3[a] > 1) m = std::min(m, n3[a]);
  int L = 0;
  while ((int64_t(1) << (L + 1)) <= m - 1) L++;
  return std::max(1, L);
}

int max_levels(const int64_t* n3) {
  int64_t m = INT64_MAX;
  for (int a = 0; a < 3; a++)
    if (n3[a] > 1) m = std::min(m, n3[a]);
  int L = 1;
  while ((int64_t(1) << L) <= m - 1) L++;
  return L;
}

// ---------------------------------------------------------------------------
// exact integers for the squared-error tables (up to 384 bits)
// ---------------------------------------------------------------------------
struct Big {
  static constexpr int N = 6;
  uint64_t w[N] = {0, 0, 0, 0, 0, 0};
  static Big from(uint64_t v) {
    Big b;
    b.w[0] = v;
    return b;
  }
  void add(const Big& o) {
    unsigned __int128 c = 0;
    for (int i = 0; i < N; i++) {
      c += (unsigned __int128)w[i] + o.w[i];
      w[i] = (uint64_t)c;
      c >>= 64;
    }
  }
  void sub(const Big& o) {  // requires *this >= o
    unsigned __int128 br = 0;
    for (int i = 0; i < N; i++) {
      unsigned __int128 t = (unsigned __int128)w[i] - o.w[i] - br;
      w[i] = (uint64_t)t;
      br = (t >> 127) & 1;
    }
  }
  static Big shl(uint64_t v, int s) {  // v << s
    Big b;
    const int q = s / 64, r = s % 64;
    if (q < N) b.w[q] = v << r;
    if (r && q + 1 < N) b.w[q + 1] = v >> (64 - r);
    return b;
  }
  Big mul(uint64_t m) const {
    Big b;
    unsigned __int128 c = 0;
    for (int i = 0; i < N; i++) {
      c += (unsigned __int128)w[i] * m;
      b.w[i] = (uint64_t)c;
      c >>= 64;
    }
    return b;
  }
  Big mulb(const Big& o) const {
    Big b;
    for (int i = 0; i < N; i++) {
      unsigned __int128 c = 0;
      for (int j = 0; i + j < N; j++) {
        c += (unsigned __int128)w[i] * o.w[j] + b.w[i + j];
        b.w[i + j] = (uint64_t)c;
        c >>= 64;
      }
    }
    return b;
  }
  int cmp(const Big& o) const {
    for (int i = N - 1; i >= 0; i--)
      if (w[i] != o.w[i]) return w[i] < o.w[i] ? -1 : 1;
    return 0;
  }
  int bitlen() const {
    for (int i = N - 1; i >= 0; i--)
      if (w[i]) return 64 * i + 64 - __builtin_clzll(w[i]);
    return 0;
  }
  bool bit(int i) const { return (w[i / 64] >> (i % 64)) & 1; }
  void setbit(int i) { w[i / 64] |= uint64_t(1) << (i % 64); }
  // smallest double >= value
  double to_double_up() const {
    const int t = bitlen();
    if (t <= 53) {
      uint64_t v = w[0];
      return (double)v;
    }
    const int drop = t - 53;
    uint64_t m = 0;
    for (int i = t - 1; i >= drop; i--) m = (m << 1) | (uint64_t)bit(i);
    bool rest = false;
    for (int i = 0; i < drop && !rest; i++) rest = bit(i);
    if (rest) m += 1;
    return std::ldexp((double)m, drop);
  }
  // ceil(sqrt(value)), exact.  A long-double estimate e of sqrt(value)
  // (64-bit mantissa: relative error below 2^-62) gives the floor root
  // within e 2^-60 + 2; the bits below that margin are then set one at a
  // time from a lower bound (r = lo + sum of 2^i with (r + 2^i)^2 <= value),
  // so only a few multiplications remain.
  Big isqrt_ceil() const {
    const int t = bitlen();
    if (t == 0) return Big();
    long double v = 0.0L;   // value rounded to 64 bits, then the estimate
    {
      const int drop = t > 64 ? t - 64 : 0;
      uint64_t m = 0;
      for (int i = t - 1; i >= drop; i--) m = (m << 1) | (uint64_t)bit(i);
      v = std::ldexp((long double)m, drop);
    }
    const long double e = std::sqrt(v);
    const long double margin = std::ldexp(e, -60) + 4.0L;
    long double lo_f = std::floor(e - margin);
    if (lo_f < 0.0L) lo_f = 0.0L;
    // lo_f as a Big (an integer below 2^96 whose 64-bit mantissa is exact)
    Big lo;
    {
      int ex = 0;
      const long double fr = std::frexp(lo_f, &ex);   // lo_f = fr 2^ex, fr in [0.5, 1)
      if (lo_f > 0.0L) {
        const uint64_t mant = (uint64_t)std::ldexp(fr, 64);
        const int sh = ex - 64;
        if (sh >= 0) lo = Big::shl(mant, sh);
        else lo = Big::from(mant >> (-sh));
      }
    }
    int k = 0;   // bits to settle: the floor root lies in [lo, lo + 2^(k+1))
    {
      const long double span = 2.0L * margin + 2.0L;
      while (std::ldexp(1.0L, k + 1) <= span) k++;
      k++;
    }
    Big r = lo;
    for (int i = k; i >= 0; i--) {
      Big c = r;
      c.add(Big::shl(1, i));
      if (c.mulb(c).cmp(*this) <= 0) r = c;
    }
    if (r.mulb(r).cmp(*this) < 0) r.add(Big::from(1));
    return r;
  }
};

double up_u64(uint64_t v) { return Big::from(v).to_double_up(); }

// ---------------------------------------------------------------------------
// ||P^T P||_inf of the 1-D odd-point operator of a line of m points
// (L2 composition); weights are dyadic so every sum is exact
// ---------------------------------------------------------------------------
double rowsum_ptp(int64_t m, int degree) {
  static std::map<std::pair<int64_t, int>, double> cache;
  auto key = std::make_pair(m, degree);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  const int64_t mc = (m + 1) / 2;
  // rows of P: list of (column, weight)
  std::vector<std::vector<std::pair<int64_t, double>>> cols(mc);  // column -> (row, weight)
  std::vector<std::vector<std::pair<int64_t, double>>> rows(m / 2);
  for (int64_t t = 0, j = 1; j < m; j += 2, t++) {
    const bool p1 = j + 1 < m, m3 = j - 3 >= 0, p3 = j + 3 < m;
    std::vector<std::pair<int64_t, double>> w;
    if (degree == 3 && p1 && m3 && p3) w = {{j - 3, -1.0 / 16}, {j - 1, 9.0 / 16}, {j + 1, 9.0 / 16}, {j + 3, -1.0 / 16}};
    else if (degree == 3 && p1 && p3) w = {{j - 1, 3.0 / 8}, {j + 1, 6.0 / 8}, {j + 3, -1.0 / 8}};
    else if (degree == 3 && p1 && m3) w = {{j - 3, -1.0 / 8}, {j - 1, 6.0 / 8}, {j + 1, 3.0 / 8}};
    else if (p1) w = {{j - 1, 0.5}, {j + 1, 0.5}};
    else w = {{j - 1, 1.0}};
    for (auto& pr : w) {
      rows[t].push_back({pr.first / 2, pr.second});
      cols[pr.first / 2].push_back({t, pr.second});
    }
  }
  double best = 0.0;
  for (int64_t a = 0; a < mc; a++) {
    std::map<int64_t, double> acc;
    for (auto& rw : cols[a])
      for (auto& cw : rows[rw.first]) acc[cw.first] += rw.second * cw.second;
    double s = 0.0;
    for (auto& kv : acc) s += std::fabs(kv.second);
    best = std::max(best, s);
  }
  cache[key] = best;
  return best;
}

// ---------------------------------------------------------------------------
// tables, composition and planning
// ---------------------------------------------------------------------------
struct Tab {
  std::vector<double> maxerr, sq;
  std::vector<uint64_t> bytes;
};

constexpr double kMargin = 1.000000001;
constexpr double kRound2 = 1.0001;   // second-order rounding terms

struct Meta {
  int L = 1, d = 1, degree = 3, interp = 0, dtype = 0, decomp = -1;
  int enc = 1;   // 1 generic, 2 negabinary
  double h = 0, M = 0, C0 = 0, R = 0;
  double C0c = 0, Dm = 0;   // max |c| at level 0; max |S2 / S3 value|
  int64_t n = 0;
  std::map<int, int64_t> level_counts;
  std::map<std::pair<int, int>, int64_t> region_counts;
  std::map<int, double> level_factor;
  std::map<std::pair<int, int>, double> region_factor;
  std::map<int, std::pair<double, double>> decomp_factors;
};

struct SRef {
  int level, region, sub;
};

// Rounding at level 0 (field dtype, unit roundoff u).  The coarse values are
// the fixed-point reconstruction rounded once to the field dtype: conv() =
// G u Y joins the incoming error.  Every level-0 point then carries
// rho0() = G u (Pr + Y + Cr) + sub, with Y = M + Lam^d (E_1 + sum e_0)
// bounding |x'| and the retrieval's prediction inputs:
//   Pr     rounding of the prediction in refactoring and in retrieval: one
//          per-region pass rounds at most kappa (M + Y); per-level pass k
//          rounds at most kappa V_k, multiplied by Lam^(d-k) in the later
//          passes; pass 1 reads coarse values (V_1 = M; retrieval Y), pass
//          k >= 2 also earlier predictions, bounded by Lam^(k-1) V_1 and by
//          M + C0c (1 + 2u) (|W| <= |x| + |c| / (1 - u) at a level-0 point;
//          retrieval Y + C0c (1 + 2u)); kappa = 2.875 cubic (the rule forms of
//          the kernels), 1 linear;
//   Y      the final addition x' = P + c_hat;
//   Cr     the coefficient side, with C0c = max |c| over level 0 and Dm =
//          max |value| of the decomposition's sub-levels S2, S3: c = x - P
//          rounded once (C0c), negabinary dequantisation (C0c); with
//          decomposition S2's forward difference (Dm), two linear
//          predictions (2 C0c) and addition (C0c), S3's forward difference
//          (Dm), two 2-pass bilinear predictions (4 C0c), addition (C0c) and
//          the S2 points it reads: 9 C0c + 2 Dm generic, 10 C0c + 4 Dm
//          negabinary (dequantisation of S1, S2, S3);
//   sub    256 times the largest absolute error of a subnormal result;
//   G      1.0001, the second-order terms.
struct Composer {
  Meta m;
  std::vector<SRef> st;
  std::map<int, std::vector<int>> by_level;
  double lam, uw, lam_d, rho_fix, cr, sub, kap;

  void init(const Meta& meta, const std::vector<SRef>& streams) {
    m = meta;
    st = streams;
    lam = m.degree == 3 ? 1.25 : 1.0;
    uw = m.dtype == PCR_F32 ? std::ldexp(1.0, -24) : std::ldexp(1.0, -53);
    kap = m.degree == 3 ? 2.875 : 1.0;
    double lam_d1 = 1.0;
    for (int i = 0; i < m.d - 1; i++) lam_d1 *= lam;
    lam_d = lam_d1 * lam;
    rho_fix = (2.0 * (double)m.d * lam_d1 + 2.0) * m.h;
    const double neg = m.enc == 2 ? 1.0 : 0.0;
    cr = m.decomp >= 0 ? (9.0 + neg) * m.C0c + (2.0 + 2.0 * neg) * m.Dm : (1.0 + neg) * m.C0c;
    sub = m.dtype == PCR_F32 ? std::ldexp(1.0, -142) : std::ldexp(1.0, -1067);
    by_level.clear();
    for (size_t i = 0; i < st.size(); i++) by_level[st[i].level].push_back((int)i);
  }

  double mag(double E1, double e0sum) const { return m.M + lam_d * (E1 + e0sum); }

  double pred_rounding(double Y) const {
    if (m.interp != 0) return kap * (m.M + Y);
    const double cap = m.C0c * (1.0 + 2.0 * uw);
    double acc = 0.0, lk = 1.0;
    for (int k = 0; k < m.d; k++) {
      const double vr = k == 0 ? m.M : std::min(lk * m.M, m.M + cap);
      const double vt = k == 0 ? Y : std::min(lk * Y, Y + cap);
      double prop = 1.0;
      for (int j = 0; j < m.d - 1 - k; j++) prop *= lam;
      acc += prop * (vr + vt);
      lk *= lam;
    }
    return kap * acc;
  }

  double rho0(double E1, double e0sum) const {
    if (m.L == 1) return kMargin * 1.01 * uw * m.C0;
    const double Y = mag(E1, e0sum);
    return kRound2 * uw * (pred_rounding(Y) + Y + cr) + sub;
  }

  // rounding of the fixed-point coarse values to the field dtype
  double conv(double E1, double e0sum) const { return kRound2 * uw * mag(E1, e0sum); }

  // region -> summed error, in order of first appearance (stream order)
  std::vector<std::pair<int, double>> region_errors(int level, const std::vector<double>& err) const {
    std::vector<std::pair<int, double>> out;
    for (int i : by_level.at(level)) {
      const int r = st[i].region;
      bool found = false;
      for (auto& pr : out)
        if (pr.first == r) {
          pr.second = pr.second + err[i];
          found = true;
        }
      if (!found) out.push_back({r, 0.0 + err[i]});
    }
    return out;
  }

  double level_step(double E, const std::vector<std::pair<int, double>>& reg, double rho) const {
    if (m.interp == 0) {
      double e = reg[0].second;
      for (auto& pr : reg) e = std::max(e, pr.second);
      return lam_d * E + e + rho;
    }
    auto sorted = reg;
    std::sort(sorted.begin(), sorted.end());
    std::vector<double> F;
    for (auto& pr : sorted) {
      double base = E;
      for (double f : F) base = std::max(base, f);
      F.push_back(lam * base + pr.second + rho);
    }
    for (double f : F) E = std::max(E, f);
    return E;
  }

  static double sum_vals(const std::vector<std::pair<int, double>>& reg) {
    double s = 0.0;
    for (auto& pr : reg) s += pr.second;
    return s;
  }

  double linf(const std::vector<double>& err) const {
    const int L = m.L;
    double E = err[by_level.at(L - 1)[0]] + (L - 1 >= 1 ? m.h : 0.0);
    if (L == 1) return (E + rho0(0.0, 0.0)) * kMargin;
    for (int level = L - 2; level >= 0; level--) {
      auto reg = region_errors(level, err);
      const double rho = level == 0 ? rho0(E, sum_vals(reg)) : rho_fix;
      if (level == 0) E = E + conv(E, sum_vals(reg));
      E = level_step(E, reg, rho);
    }
    return E * kMargin;
  }

  void e1_e0(const std::vector<double>& err, double& E1, double& e0) const {
    const int L = m.L;
    if (L == 1) {
      E1 = e0 = 0.0;
      return;
    }
    double E = err[by_level.at(L - 1)[0]] + (L - 1 >= 1 ? m.h : 0.0);
    for (int level = L - 2; level >= 1; level--) E = level_step(E, region_errors(level, err), rho_fix);
    E1 = E;
    e0 = sum_vals(region_errors(0, err));
  }

  double l2(const std::vector<double>& sq, const std::vector<double>& err) const {
    const int L = m.L;
    double N = std::sqrt(sq[by_level.at(L - 1)[0]]);
    if (L == 1) {
      N += rho0(0.0, 0.0) * std::sqrt((double)m.level_counts.at(0));
      return (N * N) * kMargin;
    }
    N += m.h * std::sqrt((double)m.level_counts.at(L - 1));
    double E1, e0;
    e1_e0(err, E1, e0);
    for (int level = L - 2; level >= 0; level--) {
      const double rho = level == 0 ? rho0(E1, e0) : rho_fix;
      if (level == 0) N = N + conv(E1, e0) * std::sqrt((double)(m.n - m.level_counts.at(0)));
      std::map<int, std::vector<std::pair<int, int>>> groups;
      for (int i : by_level.at(level)) groups[st[i].region].push_back({st[i].sub, i});
      std::map<int, double> cnorm;
      for (auto& g : groups) {
        auto items = g.second;
        std::sort(items.begin(), items.end());
        if (items[0].first == 0) {
          cnorm[g.first] = std::sqrt(sq[items[0].second]);
        } else {
          const auto f = m.decomp_factors.at(g.first);
          const double n1 = std::sqrt(sq[items[0].second]);
          const double n2 = std::sqrt(sq[items[1].second]) + f.first * n1;
          const double n3 = std::sqrt(sq[items[2].second]) + f.second * std::sqrt(n1 * n1 + n2 * n2);
          cnorm[g.first] = std::sqrt(n1 * n1 + n2 * n2 + n3 * n3);
        }
      }
      if (m.interp == 0) {
        double c = 0.0;
        for (auto& kv : cnorm) c += kv.second * kv.second;
        const double t = m.level_factor.at(level) * N + std::sqrt(c) +
                         rho * std::sqrt((double)m.level_counts.at(level));
        N = std::sqrt(N * N + t * t);
      } else {
        double T = N * N;
        for (auto& kv : cnorm) {
          const double t = m.region_factor.at({level, kv.first}) * std::sqrt(T) + kv.second +
                           rho * std::sqrt((double)m.region_counts.at({level, kv.first}));
          T += t * t;
        }
        N = std::sqrt(T);
      }
    }
    return (N * N) * kMargin;
  }
};

struct Step {
  std::vector<std::pair<int, int>> upd;  // (stream, new planes)
  uint64_t db;
  double val;
};

std::vector<std::tuple<int, double, uint64_t>> useful_steps(const std::vector<double>& vals,
                                                             const std::vector<uint64_t>& bytes) {
  std::vector<std::tuple<int, double, uint64_t>> out;
  const int B = (int)vals.size() - 1;
  int b = 0;
  while (true) {
    int nb = b + 1;
    while (nb <= B && !(vals[nb] < vals[b])) nb++;
    if (nb > B) return out;
    out.push_back({nb, vals[nb], bytes[nb] - bytes[b]});
    b = nb;
  }
}

// greedy order inside one decomposed region (Sec. V-C)
std::vector<Step> region_sequence(const std::vector<int>& ids, const std::vector<Tab>& tabs) {
  std::map<int, int> b, pos;
  std::map<int, std::vector<std::tuple<int, double, uint64_t>>> steps;
  for (int i : ids) {
    b[i] = 0;
    pos[i] = 0;
    steps[i] = useful_steps(tabs[i].maxerr, tabs[i].bytes);
  }
  auto total = [&]() {
    double t = 0.0;
    for (int i : ids) t = t + tabs[i].maxerr[b[i]];
    return t;
  };
  std::vector<Step> seq;
  while (true) {
    bool have = false;
    double br = 0;
    int bi = -1, bnb = 0;
    uint64_t bdb = 0;
    for (int i : ids) {
      if (pos[i] >= (int)steps[i].size()) continue;
      const auto& stp = steps[i][pos[i]];
      const double de = tabs[i].maxerr[b[i]] - std::get<1>(stp);
      const uint64_t db = std::get<2>(stp);
      const double ratio = db == 0 ? std::numeric_limits<double>::infinity() : de / (double)db;
      if (!have || ratio > br) {
        have = true;
        br = ratio;
        bi = i;
        bnb = std::get<0>(stp);
        bdb = db;
      }
    }
    if (!have) return seq;
    b[bi] = bnb;
    pos[bi]++;
    seq.push_back({{{bi, bnb}}, bdb, total()});
  }
}

// Sec. V-C max ordering: (initial level error, segments)
std::pair<double, std::vector<Step>> max_ordering(const std::map<int, std::vector<int>>& by_region,
                                                  const std::vector<Tab>& tabs) {
  struct S {
    double e;
    int r, k;
    Step st;
  };
  std::vector<S> all;
  std::map<int, double> cur;
  for (auto& kv : by_region) {
    double t = 0.0;
    for (int i : kv.second) t = t + tabs[i].maxerr[0];
    cur[kv.first] = t;
    auto seq = region_sequence(kv.second, tabs);
    for (size_t k = 0; k < seq.size(); k++) all.push_back({seq[k].val, kv.first, (int)k, seq[k]});
  }
  std::sort(all.begin(), all.end(), [](const S& a, const S& b) {
    if (a.e != b.e) return a.e > b.e;
    if (a.r != b.r) return a.r < b.r;
    return a.k < b.k;
  });
  double init = -std::numeric_limits<double>::infinity();
  for (auto& kv : cur) init = std::max(init, kv.second);
  std::vector<Step> segs;
  size_t i = 0;
  while (i < all.size()) {
    size_t j = i;
    Step sg;
    sg.db = 0;
    while (j < all.size() && all[j].e == all[i].e) {
      for (auto& u : all[j].st.upd) sg.upd.push_back(u);
      sg.db += all[j].st.db;
      cur[all[j].r] = all[j].e;
      j++;
    }
    double mx = -std::numeric_limits<double>::infinity();
    for (auto& kv : cur) mx = std::max(mx, kv.second);
    sg.val = mx;
    segs.push_back(sg);
    i = j;
  }
  return {init, segs};
}

std::vector<Step> compress(double init, const std::vector<Step>& segs) {
  std::vector<Step> out;
  Step acc;
  acc.db = 0;
  double prev = init;
  for (auto& s : segs) {
    for (auto& u : s.upd) acc.upd.push_back(u);
    acc.db += s.db;
    if (s.val < prev) {
      acc.val = s.val;
      out.push_back(acc);
      acc = Step();
      acc.db = 0;
      prev = s.val;
    }
  }
  return out;
}

struct Unit {
  std::vector<int> ids;
  std::vector<Step> steps;
  double weight;
};

}  // namespace

// ---------------------------------------------------------------------------
// the handle
// ---------------------------------------------------------------------------
struct pcr_handle {
  int ndim = 3;
  int64_t dims[3] = {0, 0, 0};
  int64_t n3[3] = {1, 1, 1};
  int dtype = PCR_F32;
  int vk = VK_F32;
  int w64 = 0;
  pcr_scheme sch{};
  std::vector<int> order;
  int L = 1, B = 32, enc = 1, decomp = -1;
  double xmin = 0, xmax = 0, M = 0, h = 0, C0 = 0;
  double C0c = 0;   // max |c| over the level-0 coefficients (before decomposition)
  int G = 0;
  std::vector<SGeo> geo;
  std::vector<int> E, sh;
  std::vector<double> vmax;
  std::vector<Tab> tabs;
  std::vector<std::vector<uint32_t>> sign_words;    // per stream: sign words per plane (all segments)
  std::vector<std::vector<uint32_t>> plane_nz;
  std::vector<std::vector<uint64_t>> pairs;
  std::vector<int64_t> plane_off, sign_off, scnt_off, nz_off;
  int slot_words = 0;
  Mem mem;
  uint32_t* d_planes = nullptr;
  uint32_t* d_signs = nullptr;
  uint32_t* d_scnt = nullptr;
  uint32_t* d_nz = nullptr;
  Meta meta;
  Composer comp;
  bool has_m0 = false;
  double m0_init = 0;
  std::vector<Step> m0;
  size_t plane_words = 0, sign_area_words = 0, scnt_words = 0, nz_words = 0;
  // planner units ([0] l2, [1] L-infinity), built on first use from the tables
  mutable std::mutex plan_mu;
  mutable bool units_ok[2] = {false, false};
  mutable std::vector<Unit> units[2];
  // lossless-coded plane sizes (bytes per stream and plane), built on first use
  mutable bool packed_ok = false;
  mutable std::vector<std::vector<uint64_t>> packed;
  // work list of a whole retrieval (every segment of every stream; stream
  // numbers local to the handle), float streams then fixed-point streams;
  // built by the refactor while its kernels run, reused by every
  // single-handle retrieval
  WorkItem* d_items_all = nullptr;
  size_t items_n[2] = {0, 0};
  bool items_ready = false;
  void* d_block = nullptr;   // one allocation holding planes, signs, counts and the work list
  int device = -1;           // CUDA device holding d_block (current device at allocation)
  ~pcr_handle() {
    if (d_block) mem.free(d_block, 0);
  }
};

// exact integer squared-error tables (plane pair counts) are kept for PSNR
// and explicit schemes; error-bound schemes use n maxerr^2
static bool keeps_pairs(const pcr_handle* h) { return h->sch.mode != PCR_MODE_EB; }

static pcr_status resolve_auto(int n, const void* const* d_fields, const int* ndims, const int64_t* const* dims,
                               const int* dtypes, const pcr_scheme* schemes, const pcr_allocator* alloc,
                               void* cuda_stream, std::vector<pcr_scheme>& out);

namespace {

LatD to_latd(const Lat& l, int64_t base) {
  LatD d;
  for (int a = 0; a < 3; a++) {
    d.start[a] = l.start[a];
    d.step[a] = l.step[a];
    d.count[a] = l.count[a];
  }
  d.row_pad = l.row_pad();
  d.base = base;
  return d;
}

FieldD field_desc(const pcr_handle* h) {
  FieldD f{};
  for (int a = 0; a < 3; a++) {
    f.n[a] = h->n3[a];
    f.nc[a] = h->n3[a] > 1 ? (h->n3[a] - 1) / 2 + 1 : 1;
  }
  f.d = (int)h->order.size();
  for (int i = 0; i < 3; i++) f.order[i] = i < f.d ? h->order[i] : 0;
  f.interp = h->sch.interp;
  f.degree = h->sch.degree;
  f.L = h->L;
  f.fixb = fix_bits(h->vk, h->L);
  return f;
}

StreamD stream_desc(const pcr_handle* h, int i) {
  StreamD s{};
  const SGeo& g = h->geo[i];
  s.nlat = (int)g.lats.size();
  int64_t base = 0;
  for (int k = 0; k < s.nlat; k++) {
    s.lat[k] = to_latd(g.lats[k], base);
    base += g.lats[k].n_pad();
  }
  s.n_pad = g.n_pad();
  s.words = s.n_pad / 32;
  s.nseg = (s.n_pad + kSegElems - 1) / kSegElems;
  s.level = g.level;
  s.region = g.region;
  s.sub = g.sub;
  s.is_fix = g.is_fix;
  s.B = h->B;
  s.enc = h->enc;
  s.vk = g.is_fix ? VK_FIX : h->vk;
  s.slot_words = h->slot_words;
  s.planes = h->d_planes + h->plane_off[i];
  s.signs = h->d_signs + h->sign_off[i];
  s.sign_counts = h->d_scnt + h->scnt_off[i];
  s.plane_nz = h->d_nz + h->nz_off[i];
  s.pairs = nullptr;
  s.vmax = nullptr;
  s.stage = nullptr;
  s.b = 0;
  s.E = h->E.empty() ? 0 : h->E[i];
  s.sh = h->sh.empty() ? 0 : h->sh[i];
  return s;
}

// tiled-kernel arguments of one level (grid = the level's s-grid)
TileArgs level_args(const pcr_handle* h, int level, int retrieve, const void* src, void* dst) {
  TileArgs a{};
  const int64_t s = int64_t(1) << level;
  for (int k = 0; k < 3; k++) a.m[k] = h->n3[k] > 1 ? count_from(h->n3[k], 0, s) : 1;
  if (level == 0) {
    a.stride[0] = h->n3[1] * h->n3[2];
    a.stride[1] = h->n3[2];
    a.stride[2] = 1;
  } else {
    int64_t nc[3];
    for (int k = 0; k < 3; k++) nc[k] = h->n3[k] > 1 ? (h->n3[k] - 1) / 2 + 1 : 1;
    const int64_t xs[3] = {nc[1] * nc[2], nc[2], 1};
    for (int k = 0; k < 3; k++) a.stride[k] = (h->n3[k] > 1 ? s / 2 : 0) * xs[k];
  }
  a.d = (int)h->order.size();
  for (int i = 0; i < 3; i++) a.order[i] = i < a.d ? h->order[i] : 0;
  a.interp = h->sch.interp;
  a.degree = h->sch.degree;
  a.retrieve = retrieve;
  a.src = src;
  a.dst = dst;
  return a;
}

TileRegion tile_region(const pcr_handle* h, const Lat& l, int level, int64_t row_pad, int64_t base, void* stage,
                       unsigned long long* vmax) {
  TileRegion r{};
  const int64_t s = int64_t(1) << level;
  for (int k = 0; k < 3; k++) {
    if (h->n3[k] > 1) {
      r.start[k] = l.start[k] / s;
      r.step[k] = l.step[k] / s;
    } else {
      r.start[k] = 0;
      r.step[k] = 1;
    }
    r.count[k] = l.count[k];
  }
  r.row_pad = row_pad;
  r.base = base;
  r.stage = stage;
  r.vmax = vmax;
  return r;
}

// region lattices of `level` with the stream staging that holds them
void level_regions(const pcr_handle* h, int level, const std::vector<StreamD>& sds, TileArgs& a) {
  const int d = (int)h->order.size();
  for (size_t i = 0; i < h->geo.size(); i++) {
    const SGeo& g = h->geo[i];
    if (g.level != level || g.sub != 0) continue;
    int64_t base = 0;
    for (size_t k = 0; k < g.lats.size(); k++) {
      const int r = g.region == 0 ? (int)k : g.region - 1;
      if (r < d)
        a.reg[r] = tile_region(h, g.lats[k], level, g.lats[k].row_pad(), base, sds[i].stage, sds[i].vmax);
      base += g.lats[k].n_pad();
    }
  }
}

// sub-level lattices of a decomposed region in its compact coordinates
void decomp_subs(const pcr_handle* h, int region, const std::vector<StreamD>& sds, DecompArgs& a) {
  int u = -1, v = -1;
  for (int ax = 0; ax < 3; ax++)
    if (ax != h->decomp) (u < 0 ? u : v) = ax;
  const Lat R = region_lat(h->n3, 0, h->order, region);
  for (int k = 0; k < 3; k++) a.cnt[k] = R.count[k];
  a.u = u;
  a.v = v;
  a.n = h->decomp;
  Lat C;  // compact grid of the region
  for (int k = 0; k < 3; k++) {
    C.start[k] = 0;
    C.step[k] = 1;
    C.count[k] = R.count[k];
  }
  int slot = 0;
  for (size_t i = 0; i < h->geo.size(); i++) {
    const SGeo& g = h->geo[i];
    if (g.level != 0 || g.region != region || g.sub == 0) continue;
    const int sub = g.sub - 1;
    int64_t base = 0;
    for (int part = 0; part < 2; part++) {
      if (kSub[sub][part][0] < 0) continue;
      const int* p = kSub[sub][part];
      const Lat L = sub_lat(C, u, v, p[0], p[1], p[2], p[3]);
      DecompSub& ds = a.subs[slot++];
      for (int k = 0; k < 3; k++) {
        ds.start[k] = L.start[k];
        ds.step[k] = L.step[k];
        ds.count[k] = L.count[k];
      }
      ds.row_pad = L.row_pad();
      ds.base = base;
      ds.stage = sds[i].stage;
      ds.vmax = sds[i].vmax;
      base += L.n_pad();
    }
  }
}

void compute_tables(pcr_handle* h, int i, const std::vector<uint64_t>* pairs, bool psnr) {
  const SGeo& g = h->geo[i];
  const int B = h->B;
  const int64_t words = g.n_pad() / 32;
  const bool nb = h->enc == 2;
  Tab t;
  t.maxerr.assign(B + 1, 0.0);
  t.sq.assign(B + 1, 0.0);
  t.bytes.assign(B + 1, 0);
  uint64_t acc = 0;
  const int64_t nseg = (g.n_pad() + kSegElems - 1) / kSegElems;
  for (int k = 0; k < B; k++) {
    if (h->plane_nz[i][k]) acc += 4 * (uint64_t)words;
    if (!nb) acc += 4 * (uint64_t)h->sign_words[i][k];
    t.bytes[k + 1] = acc;
  }
  double unit, vmax_abs;
  const bool zero = h->vmax[i] == 0;
  if (g.is_fix) {
    vmax_abs = up_u64((uint64_t)h->vmax[i]) * h->h;
    unit = std::ldexp(h->h, h->sh[i] + (nb ? 3 : 0));
  } else {
    vmax_abs = h->vmax[i];
    unit = std::ldexp(1.0, h->E[i] - B + (nb ? 3 : 0));
  }
  if (!zero) {
    for (int b = 0; b <= B; b++) {
      if (b == 0) t.maxerr[b] = vmax_abs;
      else if (!nb) t.maxerr[b] = std::ldexp(unit, B - b);
      else {
        const int k = B - b;
        const uint64_t full = k + 1 >= 64 ? ~uint64_t(0) : ((uint64_t(1) << (k + 1)) - 1);
        const uint64_t dm = full / 3;   // largest |value| of k negabinary digits
        t.maxerr[b] = up_u64(dm + 1) * unit;
      }
    }
    const int64_t n_real = g.n_real();
    if (psnr && pairs) {
      const auto& C = *pairs;
      // the sums over planes j, jj >= b, from b = B down: step b adds the
      // pairs with min(j, jj) = b ((b, b) once, (b, jj) and (jj, b) as one
      // doubled term); exact integers, so the order does not matter
      Big pos, neg, s1g;
      for (int b = B; b >= 0; b--) {
        if (b < B) {
          for (int jj = b; jj < B; jj++) {
            const uint64_t c = C[b * B + jj];
            if (!c) continue;
            const int w = 2 * B - 2 - b - jj + (jj == b ? 0 : 1);
            const Big term = Big::shl(c, w);
            if (!nb || ((b + jj) % 2 == 0)) pos.add(term);
            else neg.add(term);
          }
          if (!nb) s1g.add(Big::shl(C[b * B + b], B - 1 - b));
        }
        Big s2 = pos;
        s2.sub(neg);
        Big s1;
        if (!nb) {
          s1 = s1g;
        } else {
          s1 = s2.mul((uint64_t)n_real).isqrt_ceil();
        }
        Big total = s2;
        Big s1x2 = s1;
        s1x2.add(s1);
        total.add(s1x2);
        total.add(Big::from((uint64_t)n_real));
        t.sq[b] = total.to_double_up() * unit * unit;
      }
    } else {
      for (int b = 0; b <= B; b++) t.sq[b] = (double)n_real * t.maxerr[b] * t.maxerr[b];
    }
  }
  h->tabs[i] = t;
}

void build_meta(pcr_handle* h) {
  Meta& m = h->meta;
  m.L = h->L;
  m.d = (int)h->order.size();
  m.degree = h->sch.degree;
  m.interp = h->sch.interp;
  m.dtype = h->dtype;
  m.decomp = h->decomp;
  m.enc = h->enc;
  m.h = h->h;
  m.M = h->M;
  m.C0 = h->C0;
  m.C0c = h->C0c;
  m.Dm = 0.0;
  for (size_t i = 0; i < h->geo.size(); i++)
    if (h->geo[i].level == 0 && !h->geo[i].is_fix && h->geo[i].sub >= 2) m.Dm = std::max(m.Dm, h->vmax[i]);
  m.R = h->xmax - h->xmin;
  m.n = h->n3[0] * h->n3[1] * h->n3[2];
  m.level_counts.clear();
  m.region_counts.clear();
  for (int l = 0; l < h->L; l++) m.level_counts[l] = 0;
  for (auto& g : h->geo) {
    m.level_counts[g.level] += g.n_real();
    m.region_counts[{g.level, g.region}] += g.n_real();
  }
  for (int level = 0; level < h->L - 1; level++) {
    const int64_t s = int64_t(1) << level;
    double prod = 1.0;
    for (int a : h->order) prod *= 1.0 + rowsum_ptp(count_from(h->n3[a], 0, s), m.degree);
    m.level_factor[level] = std::sqrt(prod - 1.0);
    for (int r = 1; r <= m.d; r++)
      m.region_factor[{level, r}] = std::sqrt(rowsum_ptp(count_from(h->n3[h->order[r - 1]], 0, s), m.degree));
  }
  if (h->decomp >= 0) {
    int u = -1, v = -1;
    for (int a = 0; a < 3; a++)
      if (a != h->decomp) (u < 0 ? u : v) = a;
    for (int r = 1; r <= m.d; r++) {
      const Lat R = region_lat(h->n3, 0, h->order, r);
      double p2 = 1.0, p3 = 1.0;
      for (int ax : {u, v}) {
        const int64_t c = R.count[ax];
        p3 *= 1.0 + rowsum_ptp(c, 1);
        p2 *= 1.0 + rowsum_ptp(count_from(c, 0, 2), 1);
      }
      m.decomp_factors[r] = {std::sqrt(p2 - 1.0), std::sqrt(p3 - 1.0)};
    }
  }
  std::vector<SRef> refs;
  for (auto& g : h->geo) refs.push_back({g.level, g.region, g.sub});
  h->comp.init(m, refs);
  h->has_m0 = false;
  h->m0.clear();
  if (h->sch.interp == 0 && h->decomp >= 0) {
    std::map<int, std::vector<int>> by_r;
    for (int i : h->comp.by_level.at(0)) by_r[h->geo[i].region].push_back(i);
    auto mo = max_ordering(by_r, h->tabs);
    h->has_m0 = true;
    h->m0_init = mo.first;
    h->m0 = mo.second;
  }
}

std::vector<Unit> build_units(const pcr_handle* h, bool linf) {
  std::vector<Unit> units;
  const Composer& c = h->comp;
  for (int level = h->L - 1; level >= 0; level--) {
    const auto& ids = c.by_level.at(level);
    const double w = std::ldexp(1.0, c.m.d * level);
    if (linf && h->sch.interp == 0 && ids.size() > 1) {
      std::map<int, std::vector<int>> by_r;
      for (int i : ids) by_r[h->geo[i].region].push_back(i);
      auto mo = max_ordering(by_r, h->tabs);
      units.push_back({ids, compress(mo.first, mo.second), w});
    } else {
      for (int i : ids) {
        Unit u;
        u.ids = {i};
        u.weight = w;
        for (auto& st : useful_steps(linf ? h->tabs[i].maxerr : h->tabs[i].sq, h->tabs[i].bytes))
          u.steps.push_back({{{i, std::get<0>(st)}}, std::get<2>(st), std::get<1>(st)});
        units.push_back(u);
      }
    }
  }
  return units;
}

// planner units of a handle (the tables never change after construction)
const std::vector<Unit>& cached_units(const pcr_handle* h, bool linf) {
  std::lock_guard<std::mutex> lk(h->plan_mu);
  if (!h->units_ok[linf]) {
    h->units[linf] = build_units(h, linf);
    h->units_ok[linf] = true;
  }
  return h->units[linf];
}

// Composer::linf and Composer::l2 with the partial results of the coarser
// levels kept: a step that changes streams of level l only needs levels
// l .. 0 again.  Every bound is computed with the same operations in the same
// order as the composer's, so the plans match it exactly.
struct BoundEval {
  struct Group {            // one region of a level for the L2 chain
    int region;
    std::vector<int> items; // streams in (sub, stream) order
    bool decomposed;
    double f1, f2, rfac, rcnt;
  };
  const Composer& c;
  int L;
  bool l2;
  std::vector<std::vector<int>> ids;     // stream ids per level (stream order)
  std::vector<std::vector<int>> slot;    // per stream of a level: its region's slot (first appearance)
  std::vector<int> nslot;
  std::vector<std::vector<int>> by_id;   // slots in ascending region id
  std::vector<std::vector<Group>> grp;   // per level, ascending region id
  std::vector<double> lfac, lcnt;        // per level: level factor, sqrt(point count)
  std::vector<int> grp_level, grp_index; // per stream: its L2 group's level and index (-1: none)
  std::vector<std::vector<double>> t_pre; // per-region L2 chain, kept: T before each group of a level
  std::vector<int> stream_level;          // per stream: its level
  double top_cnt = 0, n2grid = 0;
  // kept state for the current errors
  std::vector<double> E_in, N_in, csum;
  std::vector<std::vector<double>> acc, cn;
  std::vector<char> acc_ok, cn_ok;
  std::vector<double> tacc, tcn;

  BoundEval(const Composer& comp, bool use_l2) : c(comp), L(comp.m.L), l2(use_l2) {
    ids.resize(L);
    slot.resize(L);
    nslot.assign(L, 0);
    by_id.resize(L);
    grp.resize(L);
    lfac.assign(L, 0.0);
    lcnt.assign(L, 0.0);
    for (int l = 0; l < L; l++) {
      ids[l] = c.by_level.at(l);
      for (int i : ids[l]) {
        if ((int)stream_level.size() <= i) stream_level.resize(i + 1, -1);
        stream_level[i] = l;
      }
      std::vector<int> regs;
      for (int i : ids[l]) {
        const int r = c.st[i].region;
        int k = 0;
        while (k < (int)regs.size() && regs[k] != r) k++;
        if (k == (int)regs.size()) regs.push_back(r);
        slot[l].push_back(k);
      }
      nslot[l] = (int)regs.size();
      std::vector<int> o(regs.size());
      for (size_t k = 0; k < o.size(); k++) o[k] = (int)k;
      std::sort(o.begin(), o.end(), [&](int a, int b) { return regs[a] < regs[b]; });
      by_id[l] = o;
      if (!l2 || l == L - 1) continue;
      std::map<int, std::vector<std::pair<int, int>>> groups;
      for (int i : ids[l]) groups[c.st[i].region].push_back({c.st[i].sub, i});
      for (auto& g : groups) {
        auto items = g.second;
        std::sort(items.begin(), items.end());
        Group G;
        G.region = g.first;
        for (auto& it : items) G.items.push_back(it.second);
        G.decomposed = items[0].first != 0;
        G.f1 = G.f2 = 0.0;
        if (G.decomposed) {
          const auto f = c.m.decomp_factors.at(g.first);
          G.f1 = f.first;
          G.f2 = f.second;
        }
        G.rfac = G.rcnt = 0.0;
        if (c.m.interp != 0) {
          G.rfac = c.m.region_factor.at({l, g.first});
          G.rcnt = std::sqrt((double)c.m.region_counts.at({l, g.first}));
        }
        for (int i : G.items) {
          if ((int)grp_level.size() <= i) {
            grp_level.resize(i + 1, -1);
            grp_index.resize(i + 1, -1);
          }
          grp_level[i] = l;
          grp_index[i] = (int)grp[l].size();
        }
        grp[l].push_back(G);
      }
      if (c.m.interp == 0) {
        lfac[l] = c.m.level_factor.at(l);
        lcnt[l] = std::sqrt((double)c.m.level_counts.at(l));
      }
    }
    if (l2) top_cnt = std::sqrt((double)c.m.level_counts.at(L - 1));
    if (l2 && L >= 2) n2grid = std::sqrt((double)(c.m.n - c.m.level_counts.at(0)));
    E_in.assign(L, 0.0);
    t_pre.assign(L, {});
    N_in.assign(L, 0.0);
    csum.assign(L, 0.0);
    acc.resize(L);
    cn.resize(L);
    for (int l = 0; l < L; l++) {
      acc[l].assign(nslot[l], 0.0);
      cn[l].assign(grp[l].size(), 0.0);
    }
    acc_ok.assign(L, 0);
    cn_ok.assign(L, 0);
  }

  // region sums in stream order (Composer::region_errors)
  void sums(int l, const std::vector<double>& err, double* out) const {
    for (int k = 0; k < nslot[l]; k++) out[k] = 0.0;
    const auto& s = slot[l];
    const auto& id = ids[l];
    for (size_t j = 0; j < id.size(); j++) out[s[j]] = out[s[j]] + err[id[j]];
  }
  double sum_vals(int l, const double* a) const {
    double s = 0.0;
    for (int k = 0; k < nslot[l]; k++) s += a[k];
    return s;
  }
  // Composer::level_step; the running maximum equals its max over the list
  double level_step(int l, double E, const double* a, double rho) const {
    if (c.m.interp == 0) {
      double e = a[0];
      for (int k = 0; k < nslot[l]; k++) e = std::max(e, a[k]);
      return c.lam_d * E + e + rho;
    }
    double base = E;
    for (int k : by_id[l]) base = std::max(base, c.lam * base + a[k] + rho);
    return base;
  }
  // the norm of one region group (Composer::l2)
  static double group_norm(const Group& G, const std::vector<double>& sq) {
    if (!G.decomposed) return std::sqrt(sq[G.items[0]]);
    const double n1 = std::sqrt(sq[G.items[0]]);
    const double n2 = std::sqrt(sq[G.items[1]]) + G.f1 * n1;
    const double n3 = std::sqrt(sq[G.items[2]]) + G.f2 * std::sqrt(n1 * n1 + n2 * n2);
    return std::sqrt(n1 * n1 + n2 * n2 + n3 * n3);
  }
  // their root sum of squares (per-level interpolation)
  void norm_sum(int l, const double* out, double& cs) const {
    if (c.m.interp == 0) {
      double s = 0.0;
      for (size_t g = 0; g < grp[l].size(); g++) s += out[g] * out[g];
      cs = std::sqrt(s);
    }
  }
  // per-region norms of one level (Composer::l2)
  void norms(int l, const std::vector<double>& sq, double* out, double& cs) const {
    const auto& gs = grp[l];
    for (size_t g = 0; g < gs.size(); g++) out[g] = group_norm(gs[g], sq);
    norm_sum(l, out, cs);
  }
  double top(const std::vector<double>& err) const { return err[ids[L - 1][0]] + (L - 1 >= 1 ? c.m.h : 0.0); }

  // bound for the errors err / sq, of which only level `from`'s streams may
  // differ from the kept state; `keep` makes them the kept state
  // the bound of arbitrary errors, nothing kept or reused
  // whether eval_batch applies to stream i: an L2 evaluator, i one of the
  // streams of a level below the top one (in an L2 group), the kept state
  // current for every level (it is after any evaluation with keep)
  bool batch_ok(int i) const {
    if (L < 2 || i < 0 || i >= (int)stream_level.size() || stream_level[i] < 0 || stream_level[i] >= L - 1)
      return false;
    if (l2 && (i >= (int)grp_level.size() || grp_level[i] != stream_level[i])) return false;
    for (int l = 0; l <= stream_level[i]; l++)
      if (!acc_ok[l] || (l2 && !cn_ok[l])) return false;
    return true;
  }
  // The bounds of n candidates, candidate k being the kept state with stream
  // st[k]'s error and squared error replaced by nerr[k], nsq[k] (its level
  // l_k below the top one): eval_from(l_k, ..., false, st[k]) for each, with
  // the same operations in the same order per candidate, computed side by
  // side so that the candidates' dependent square-root chains overlap.
  // err / sq hold the kept state.
  void eval_batch(int n, const int* st, const double* nerr, const double* nsq, const std::vector<double>& err,
                  const std::vector<double>& sq, double* out) {
    b_lvl.resize(n);
    b_slot.resize(n);
    b_ssum.resize(n);
    b_E.resize(n);
    b_rho.resize(n);
    b_conv.resize(n);
    b_N.resize(n);
    b_gn.resize(n);
    b_cs.resize(n);
    int top = 0;
    for (int k = 0; k < n; k++) {
      const int i = st[k], l = stream_level[i];
      b_lvl[k] = l;
      top = std::max(top, l);
      // the changed stream's slot sum, in stream order as sums() forms it
      const auto& idl = ids[l];
      const auto& sll = slot[l];
      int si = -1;
      for (size_t j = 0; j < idl.size(); j++)
        if (idl[j] == i) si = sll[j];
      double ssum = 0.0;
      for (size_t j = 0; j < idl.size(); j++)
        if (sll[j] == si) ssum = ssum + (idl[j] == i ? nerr[k] : err[idl[j]]);
      b_slot[k] = si;
      b_ssum[k] = ssum;
      b_E[k] = E_in[l];
      if (!l2) continue;
      // the changed group's norm (group_norm with sq[i] replaced)
      const Group& Gi = grp[l][grp_index[i]];
      auto sqv = [&](int id) { return id == i ? nsq[k] : sq[id]; };
      if (!Gi.decomposed) {
        b_gn[k] = std::sqrt(sqv(Gi.items[0]));
      } else {
        const double n1 = std::sqrt(sqv(Gi.items[0]));
        const double n2 = std::sqrt(sqv(Gi.items[1])) + Gi.f1 * n1;
        const double n3 = std::sqrt(sqv(Gi.items[2])) + Gi.f2 * std::sqrt(n1 * n1 + n2 * n2);
        b_gn[k] = std::sqrt(n1 * n1 + n2 * n2 + n3 * n3);
      }
      if (c.m.interp == 0) {   // the level's root sum of squares with that group replaced
        double sacc = 0.0;
        for (size_t g = 0; g < grp[l].size(); g++) {
          const double v = (int)g == grp_index[i] ? b_gn[k] : cn[l][g];
          sacc += v * v;
        }
        b_cs[k] = std::sqrt(sacc);
      }
    }
    // the L-infinity chain from each candidate's level to level 1, then the
    // level-0 rounding terms
    for (int level = top; level >= 1; level--)
      for (int k = 0; k < n; k++) {
        if (b_lvl[k] < level) continue;
        const double* a = acc[level].data();
        if (b_lvl[k] == level) {
          tacc.assign(a, a + nslot[level]);
          tacc[b_slot[k]] = b_ssum[k];
          a = tacc.data();
        }
        b_E[k] = level_step(level, b_E[k], a, c.rho_fix);
      }
    for (int k = 0; k < n; k++) {
      double e0 = 0.0;
      for (int q = 0; q < nslot[0]; q++) e0 += (b_lvl[k] == 0 && q == b_slot[k]) ? b_ssum[k] : acc[0][q];
      b_rho[k] = c.rho0(b_E[k], e0);
      b_conv[k] = c.conv(b_E[k], e0);
      if (!l2) {   // the L-infinity bound: level 0's step
        const double* a = acc[0].data();
        if (b_lvl[k] == 0) {
          tacc.assign(a, a + nslot[0]);
          tacc[b_slot[k]] = b_ssum[k];
          a = tacc.data();
        }
        out[k] = level_step(0, b_E[k] + b_conv[k], a, b_rho[k]) * kMargin;
        continue;
      }
      b_N[k] = N_in[b_lvl[k]];
    }
    if (!l2) return;
    // the L2 chain from each candidate's level down to level 0
    for (int level = top; level >= 0; level--) {
      const auto& gs = grp[level];
      const int G = (int)gs.size();
      for (int k = 0; k < n; k++) {
        if (b_lvl[k] < level) continue;
        const double rho = level == 0 ? b_rho[k] : c.rho_fix;
        double N = b_N[k];
        if (level == 0) N = N + b_conv[k] * n2grid;
        const bool own = b_lvl[k] == level;
        const int gi = own ? grp_index[st[k]] : -1;
        if (c.m.interp == 0) {
          const double cs = own ? b_cs[k] : csum[level];
          const double t = lfac[level] * N + cs + rho * lcnt[level];
          N = std::sqrt(N * N + t * t);
        } else {
          double T = N * N;
          for (int g = 0; g < G; g++) {
            const double a = g == gi ? b_gn[k] : cn[level][g];
            const double t = gs[g].rfac * std::sqrt(T) + a + rho * gs[g].rcnt;
            T += t * t;
          }
          N = std::sqrt(T);
        }
        b_N[k] = N;
      }
    }
    for (int k = 0; k < n; k++) out[k] = (b_N[k] * b_N[k]) * kMargin;
  }
  std::vector<int> b_lvl, b_slot;
  std::vector<double> b_ssum, b_E, b_rho, b_conv, b_N, b_gn, b_cs;

  double eval_all(const std::vector<double>& err, const std::vector<double>& sq) {
    std::fill(acc_ok.begin(), acc_ok.end(), 0);
    std::fill(cn_ok.begin(), cn_ok.end(), 0);
    return eval_from(L - 1, err, sq, false);
  }
  // `changed` >= 0: the one stream whose sq may differ from the kept state
  // (the other groups' norms are taken from it, computed by the same
  // operations)
  double eval_from(int from, const std::vector<double>& err, const std::vector<double>& sq, bool keep,
                   int changed = -1) {
    if (L == 1) {
      if (!l2) return (top(err) + c.rho0(0.0, 0.0)) * kMargin;
      double N = std::sqrt(sq[ids[0][0]]);
      N += c.rho0(0.0, 0.0) * std::sqrt((double)c.m.level_counts.at(0));
      return (N * N) * kMargin;
    }
    const int start = std::min(from, L - 2);
    // the L-infinity chain (for L2: down to the rounding term of level 0)
    double E = from >= L - 1 ? top(err) : E_in[from];
    double rho_0 = 0.0, conv_0 = 0.0;
    for (int level = start; level >= 0; level--) {
      const double* a;
      if (level == from || !acc_ok[level]) {
        double* o;
        if (keep) {
          o = acc[level].data();
          acc_ok[level] = 1;
        } else {
          tacc.resize(nslot[level]);
          o = tacc.data();
        }
        sums(level, err, o);
        a = o;
      } else {
        a = acc[level].data();
      }
      if (keep) E_in[level] = E;
      if (level == 0) {
        rho_0 = c.rho0(E, sum_vals(0, a));
        conv_0 = c.conv(E, sum_vals(0, a));
        if (l2) break;
        E = level_step(0, E + conv_0, a, rho_0);
      } else {
        E = level_step(level, E, a, c.rho_fix);
      }
    }
    if (!l2) return E * kMargin;
    double N;
    if (from >= L - 1) {
      N = std::sqrt(sq[ids[L - 1][0]]);
      N += c.m.h * top_cnt;
    } else {
      N = N_in[from];
    }
    for (int level = start; level >= 0; level--) {
      const double rho = level == 0 ? rho_0 : c.rho_fix;
      if (level == 0 && keep) N_in[0] = N;
      if (level == 0) N = N + conv_0 * n2grid;
      const double* a;
      double cs;
      if (level == from || !cn_ok[level]) {
        double* o;
        if (keep) {
          o = cn[level].data();
          cn_ok[level] = 1;
        } else {
          tcn.resize(grp[level].size());
          o = tcn.data();
        }
        if (!keep && changed >= 0 && changed < (int)grp_level.size() && cn_ok[level] &&
            grp_level[changed] == level) {
          std::copy(cn[level].begin(), cn[level].end(), tcn.begin());
          o[grp_index[changed]] = group_norm(grp[level][grp_index[changed]], sq);
          norm_sum(level, o, cs);
        } else {
          norms(level, sq, o, cs);
        }
        if (keep) csum[level] = cs;
        a = o;
      } else {
        a = cn[level].data();
        cs = csum[level];
      }
      if (keep && level > 0) N_in[level] = N;
      if (c.m.interp == 0) {
        const double t = lfac[level] * N + cs + rho * lcnt[level];
        N = std::sqrt(N * N + t * t);
      } else {
        double T = N * N;
        const auto& gs = grp[level];
        size_t g0 = 0;
        // one changed group above level 0: the chain before it is the kept
        // one (the incoming N, the earlier groups and rho are unchanged; at
        // level 0 rho and the coarse rounding move with every error)
        if (!keep && changed >= 0 && level == from && level > 0 && changed < (int)grp_level.size() &&
            grp_level[changed] == level && t_pre.size() > (size_t)level && t_pre[level].size() == gs.size()) {
          g0 = (size_t)grp_index[changed];
          T = t_pre[level][g0];
        }
        if (keep) t_pre[level].resize(gs.size());
        for (size_t g = g0; g < gs.size(); g++) {
          if (keep) t_pre[level][g] = T;
          const double t = gs[g].rfac * std::sqrt(T) + a[g] + rho * gs[g].rcnt;
          T += t * t;
        }
        N = std::sqrt(T);
      }
    }
    return (N * N) * kMargin;
  }
};

// greedy interpreter: largest bound decrease per byte until the target holds.
// `have` (incremental invocation, Sec. III-A progressive refinement): planes
// already fetched per stream; the plan starts there and never drops a plane,
// a step costs only the bytes of planes not yet fetched, and steps whose
// planes are all fetched are passed over.
bool greedy(const pcr_handle* h, double target, bool linf, std::vector<int>& b, double& bound,
            const std::vector<int>* have = nullptr) {
  const int n = (int)h->tabs.size();
  if (have) b = *have;
  else b.assign(n, 0);
  const std::vector<Unit>& units = cached_units(h, linf);
  std::vector<size_t> pos(units.size(), 0);
  std::vector<double> err(n), sq(n);
  for (int i = 0; i < n; i++) {
    err[i] = h->tabs[i].maxerr[b[i]];
    sq[i] = h->tabs[i].sq[b[i]];
  }
  if (have)
    for (size_t ui = 0; ui < units.size(); ui++)
      for (; pos[ui] < units[ui].steps.size(); pos[ui]++) {
        bool covered = true;
        for (auto& up : units[ui].steps[pos[ui]].upd) covered = covered && up.second <= b[up.first];
        if (!covered) break;
      }
  // bytes a step adds to the current plan
  std::vector<std::pair<int, int>> top;
  auto step_cost = [&](const Step& st) -> uint64_t {
    if (!have) return st.db;
    top.clear();
    for (auto& up : st.upd) {
      bool found = false;
      for (auto& tp : top)
        if (tp.first == up.first) {
          tp.second = std::max(tp.second, up.second);
          found = true;
        }
      if (!found) top.push_back(up);
    }
    uint64_t c = 0;
    for (auto& tp : top) {
      const int i = tp.first;
      c += h->tabs[i].bytes[std::max(tp.second, b[i])] - h->tabs[i].bytes[b[i]];
    }
    return c;
  };
  BoundEval be(h->comp, !linf);
  std::vector<int> unit_level(units.size());
  for (size_t ui = 0; ui < units.size(); ui++) unit_level[ui] = h->geo[units[ui].ids[0]].level;
  auto evaluate = [&](int level, bool keep, int changed = -1) { return be.eval_from(level, err, sq, keep, changed); };
  std::vector<std::pair<int, double>> reg;
  auto unit_value = [&](const Unit& u) {
    if (u.ids.size() == 1) return linf ? err[u.ids[0]] : sq[u.ids[0]];
    reg.clear();
    for (int i : u.ids) {
      const int r = h->geo[i].region;
      bool found = false;
      for (auto& pr : reg)
        if (pr.first == r) {
          pr.second = pr.second + err[i];
          found = true;
        }
      if (!found) reg.push_back({r, 0.0 + err[i]});
    }
    double mx = reg[0].second;
    for (auto& pr : reg) mx = std::max(mx, pr.second);
    return mx;
  };
  // set the errors of one step's streams (returns the previous planes)
  std::vector<std::pair<int, int>> saved;
  auto apply = [&](const Step& st) {
    saved.clear();
    for (auto& up : st.upd) {
      saved.push_back({up.first, b[up.first]});
      const int nb = have ? std::max(b[up.first], up.second) : up.second;
      b[up.first] = nb;
      err[up.first] = h->tabs[up.first].maxerr[nb];
      sq[up.first] = h->tabs[up.first].sq[nb];
    }
  };
  auto undo = [&]() {
    for (auto it = saved.rbegin(); it != saved.rend(); ++it) {
      b[it->first] = it->second;
      err[it->first] = h->tabs[it->first].maxerr[it->second];
      sq[it->first] = h->tabs[it->first].sq[it->second];
    }
  };
  bound = evaluate(h->L - 1, true);
  // candidates that change one stream below the top level of an L2 plan:
  // evaluated side by side (BoundEval::eval_batch, the same values as one
  // by one)
  std::vector<int> bst, bunit;
  std::vector<double> berr, bsq, bval, nbv(units.size()), own1v(units.size());
  std::vector<char> batched(units.size(), 0);
  while (bound > target) {
    bool have_best = false, have_fb = false;
    double best_r = 0, fb_r = 0, best_bnd = 0, fb_bnd = 0;
    size_t best_u = 0, fb_u = 0;
    bst.clear();
    bunit.clear();
    berr.clear();
    bsq.clear();
    {
      for (size_t ui = 0; ui < units.size(); ui++) {
        batched[ui] = 0;
        const Unit& u = units[ui];
        if (pos[ui] >= u.steps.size() || u.ids.size() != 1) continue;
        const Step& st = u.steps[pos[ui]];
        const int i = u.ids[0];
        if (st.upd.size() != 1 || st.upd[0].first != i || !be.batch_ok(i)) continue;
        const int nbp = have ? std::max(b[i], st.upd[0].second) : st.upd[0].second;
        bst.push_back(i);
        bunit.push_back((int)ui);
        berr.push_back(h->tabs[i].maxerr[nbp]);
        bsq.push_back(h->tabs[i].sq[nbp]);
        own1v[ui] = linf ? h->tabs[i].maxerr[nbp] : h->tabs[i].sq[nbp];
        batched[ui] = 1;
      }
      if (!bst.empty()) {
        bval.resize(bst.size());
        be.eval_batch((int)bst.size(), bst.data(), berr.data(), bsq.data(), err, sq, bval.data());
        for (size_t k = 0; k < bst.size(); k++) nbv[bunit[k]] = bval[k];
      }
    }
    for (size_t ui = 0; ui < units.size(); ui++) {
      const Unit& u = units[ui];
      if (pos[ui] >= u.steps.size()) continue;
      const Step& st = u.steps[pos[ui]];
      const uint64_t db = step_cost(st);
      const double own0 = unit_value(u);
      double nb, own1;
      if (batched[ui]) {
        nb = nbv[ui];
        own1 = own1v[ui];
      } else {
        apply(st);
        nb = evaluate(unit_level[ui], false, u.ids.size() == 1 ? u.ids[0] : -1);
        own1 = unit_value(u);
        undo();
      }
      const double gain = bound - nb;
      const double inf = std::numeric_limits<double>::infinity();
      const double ratio = db == 0 ? inf : gain / (double)db;
      if (gain > 0 || db == 0) {
        if (!have_best || ratio > best_r) {
          have_best = true;
          best_r = ratio;
          best_u = ui;
          best_bnd = nb;
        }
      }
      const double own = (own0 - own1) * u.weight;
      const double fr = db == 0 ? inf : own / (double)db;
      if (!have_fb || fr > fb_r) {
        have_fb = true;
        fb_r = fr;
        fb_u = ui;
        fb_bnd = nb;
      }
    }
    if (!have_best) {
      if (!have_fb) return false;
      best_u = fb_u;
      best_bnd = fb_bnd;
    }
    apply(units[best_u].steps[pos[best_u]]);
    be.eval_from(unit_level[best_u], err, sq, true);   // refresh the kept partial results
    bound = best_bnd;
    pos[best_u]++;
  }
  return true;
}

// Best-first search for the fewest bytes whose bound meets the target
// (Sec. VI-B: best-first search with pruning and incremental invocation for
// per-level + decomposition, a dynamic program for per-region; both look for
// the smallest retrieval under the bound).  One search for every mode, over
// the greedy's planning units: a state is the number of steps taken in each
// unit, its cost the bytes it adds to `have` (or to nothing); the bound is
// monotone in every unit.  The greedy plan is the first incumbent; unit u
// starts at q_u, the fewest steps meeting the target with every other unit
// complete; states are expanded cheapest first (key: cost, then push
// order) over a tree that reaches every state once (a child advances only
// units at or after the one its parent advanced); a child that meets the
// target becomes the incumbent when cheaper, children costing at least the
// incumbent are cut, and the search ends when the cheapest open state costs
// at least the incumbent (proved minimum) or after max_nodes expansions.
struct SearchStats {
  int64_t expanded = 0;
  int optimal = 0;
  uint64_t greedy_bytes = 0;
};

bool search_plan(const pcr_handle* h, double target, bool linf, const std::vector<int>* have, int64_t max_nodes,
                 std::vector<int>& b, double& bound, SearchStats& ss) {
  const int n = (int)h->tabs.size();
  std::vector<int> base = have ? *have : std::vector<int>(n, 0);
  const bool ok = greedy(h, target, linf, b, bound, have);
  auto added = [&](const std::vector<int>& bb) {
    uint64_t c = 0;
    for (int i = 0; i < n; i++) c += h->tabs[i].bytes[bb[i]] - h->tabs[i].bytes[base[i]];
    return c;
  };
  ss = SearchStats();
  ss.greedy_bytes = added(b);
  if (!ok) return false;
  const std::vector<Unit>& units = cached_units(h, linf);
  const int U = (int)units.size();
  // planes of each unit's streams after p steps, and the bytes they add
  std::vector<std::vector<std::vector<std::pair<int, int>>>> pl(U);
  std::vector<std::vector<uint64_t>> cost(U);
  std::vector<int> S(U), start(U, 0);
  for (int u = 0; u < U; u++) {
    const Unit& un = units[u];
    S[u] = (int)un.steps.size();
    std::vector<std::pair<int, int>> cur;
    for (int i : un.ids) cur.push_back({i, base[i]});
    auto push = [&]() {
      pl[u].push_back(cur);
      uint64_t c = 0;
      for (auto& pr : cur) c += h->tabs[pr.first].bytes[pr.second] - h->tabs[pr.first].bytes[base[pr.first]];
      cost[u].push_back(c);
    };
    push();
    for (const Step& st : un.steps) {
      for (auto& up : st.upd)
        for (auto& pr : cur)
          if (pr.first == up.first) pr.second = have ? std::max(pr.second, up.second) : up.second;
      push();
    }
    if (have)
      while (start[u] < S[u]) {
        bool covered = true;
        for (auto& up : un.steps[start[u]].upd) covered = covered && up.second <= base[up.first];
        if (!covered) break;
        start[u]++;
      }
  }
  BoundEval be(h->comp, !linf);
  std::vector<double> err(n), sq(n);
  std::vector<int> bb(n);
  auto planes_of = [&](const uint16_t* pos) {
    bb = base;
    for (int u = 0; u < U; u++)
      for (auto& pr : pl[u][pos[u]]) bb[pr.first] = pr.second;
  };
  auto bound_of = [&](const uint16_t* pos) {
    planes_of(pos);
    for (int i = 0; i < n; i++) {
      err[i] = h->tabs[i].maxerr[bb[i]];
      sq[i] = h->tabs[i].sq[bb[i]];
    }
    return be.eval_all(err, sq);
  };
  std::vector<uint16_t> q(U), pos(U);
  for (int u = 0; u < U; u++) {
    for (int v = 0; v < U; v++) pos[v] = (uint16_t)S[v];
    int p = start[u];
    while (true) {
      pos[u] = (uint16_t)p;
      if (p == S[u] || bound_of(pos.data()) <= target) break;
      p++;
    }
    q[u] = (uint16_t)p;
  }
  // the incumbent: the greedy's positions (per unit the last position with
  // its planes), improved by local moves until none applies -- drop a unit's
  // last step, then move one step from unit a to unit b, each taken when it
  // is cheaper and still meets the target
  for (int u = 0; u < U; u++) {
    int p = 0;
    for (int k = 0; k <= S[u]; k++) {
      bool eq = true;
      for (auto& pr : pl[u][k]) eq = eq && b[pr.first] == pr.second;
      if (eq) p = k;
    }
    pos[u] = (uint16_t)p;
  }
  uint64_t c_best = ss.greedy_bytes;
  std::vector<uint16_t> t(U);
  for (bool changed = true; changed;) {
    changed = false;
    for (int a = 0; a < U; a++)
      while (pos[a] > std::max(start[a], (int)q[a])) {
        t = pos;
        t[a]--;
        const uint64_t ct = c_best - cost[a][pos[a]] + cost[a][t[a]];
        if (ct >= c_best) break;
        const double v = bound_of(t.data());
        if (v > target) break;
        pos = t;
        c_best = ct;
        bound = v;
        changed = true;
      }
    for (int a = 0; a < U; a++)
      for (int b2 = 0; b2 < U; b2++) {
        if (b2 == a || pos[a] <= std::max(start[a], (int)q[a]) || pos[b2] >= S[b2]) continue;
        t = pos;
        t[a]--;
        t[b2]++;
        const int64_t ct = (int64_t)c_best - (int64_t)cost[a][pos[a]] + (int64_t)cost[a][t[a]] -
                           (int64_t)cost[b2][pos[b2]] + (int64_t)cost[b2][t[b2]];
        if (ct >= (int64_t)c_best) continue;
        const double v = bound_of(t.data());
        if (v <= target) {
          pos = t;
          c_best = (uint64_t)ct;
          bound = v;
          changed = true;
        }
      }
  }
  planes_of(pos.data());
  b = bb;
  uint64_t c0 = 0;
  for (int u = 0; u < U; u++) c0 += cost[u][q[u]];
  if (c0 >= c_best) {
    ss.optimal = 1;
    return true;
  }
  const double v0 = bound_of(q.data());
  if (v0 <= target) {
    planes_of(q.data());
    b = bb;
    bound = v0;
    ss.optimal = 1;
    return true;
  }
  // open states: positions in a pool, heap of (cost, push order, slot, last unit)
  struct Open {
    uint64_t cost;
    int64_t seq;
    size_t slot;
    int last;
  };
  auto later = [](const Open& a, const Open& o) { return a.cost != o.cost ? a.cost > o.cost : a.seq > o.seq; };
  std::priority_queue<Open, std::vector<Open>, decltype(later)> heap(later);
  std::vector<uint16_t> pool(q.begin(), q.end());
  heap.push({c0, 0, 0, 0});
  int64_t seq = 1;
  std::vector<uint16_t> child(U);
  while (!heap.empty()) {
    const Open o = heap.top();
    heap.pop();
    if (o.cost >= c_best) break;
    if (ss.expanded >= max_nodes) return true;
    ss.expanded++;
    for (int u = o.last; u < U; u++) {
      const uint16_t* p = &pool[o.slot * U];
      if (p[u] >= S[u]) continue;
      const uint64_t nc = o.cost + cost[u][p[u] + 1] - cost[u][p[u]];
      if (nc >= c_best) continue;
      std::copy(p, p + U, child.begin());
      child[u]++;
      const double v = bound_of(child.data());
      if (v <= target) {
        b = bb;
        bound = v;
        c_best = nc;
      } else {
        const size_t slot = pool.size() / U;
        pool.insert(pool.end(), child.begin(), child.end());
        heap.push({nc, seq++, slot, u});
      }
    }
  }
  ss.optimal = 1;
  return true;
}

size_t vsize(int vk) { return vk == VK_F32 ? 4 : 8; }

}  // namespace

// ---------------------------------------------------------------------------
// refactor
// ---------------------------------------------------------------------------
// the device address of a field's timeout flag (no access: pointer arithmetic)
static int* timeout_flag(FieldStats* d_st) {
  return d_st ? reinterpret_cast<int*>(reinterpret_cast<char*>(d_st) + offsetof(FieldStats, timeout)) : nullptr;
}

static pcr_status validate(const void* d_field, int ndim, const int64_t* dims, int dtype, const pcr_scheme* sch) {
  if (!d_field || !dims || !sch) return fail(PCR_ERR_INVALID_ARG, "null argument");
  if (ndim != 2 && ndim != 3) return fail(PCR_ERR_INVALID_ARG, "ndim must be 2 or 3");
  for (int i = 0; i < ndim; i++)
    if (dims[i] < 2) return fail(PCR_ERR_INVALID_ARG, "every dimension must be >= 2");
  if (dtype != PCR_F32 && dtype != PCR_F64) return fail(PCR_ERR_INVALID_ARG, "dtype must be PCR_F32 or PCR_F64");
  if (sch->mode != PCR_MODE_EB && sch->mode != PCR_MODE_PSNR && sch->mode != PCR_MODE_EXPLICIT)
    return fail(PCR_ERR_INVALID_ARG, "bad mode");
  if (sch->interp != 0 && sch->interp != 1) return fail(PCR_ERR_INVALID_ARG, "bad interp");
  if (sch->degree != 1 && sch->degree != 3) return fail(PCR_ERR_INVALID_ARG, "degree must be 1 or 3");
  if (sch->encoding < 0 || sch->encoding > 2) return fail(PCR_ERR_INVALID_ARG, "bad encoding");
  return PCR_OK;
}

static pcr_status setup_handle(pcr_handle* h, int ndim, const int64_t* dims, int dtype, const pcr_scheme* sch) {
  h->ndim = ndim;
  for (int i = 0; i < 3; i++) h->dims[i] = 0;
  for (int i = 0; i < ndim; i++) h->dims[i] = dims[i];
  if (ndim == 2) {
    h->n3[0] = 1;
    h->n3[1] = dims[0];
    h->n3[2] = dims[1];
  } else {
    for (int i = 0; i < 3; i++) h->n3[i] = dims[i];
  }
  h->dtype = dtype;
  h->vk = dtype == PCR_F32 ? VK_F32 : VK_F64;
  h->w64 = dtype == PCR_F64;
  h->sch = *sch;
  std::vector<int> act;
  for (int a = 0; a < 3; a++)
    if (h->n3[a] > 1) act.push_back(a);
  const int d = (int)act.size();
  if (sch->interp == 1) {
    // user axes: 0..ndim-1; 2-D fields are stored as (1, n0, n1)
    std::vector<int> ord;
    for (int i = 0; i < d; i++) ord.push_back(sch->order[i] + (ndim == 2 ? 1 : 0));
    std::vector<int> s = ord;
    std::sort(s.begin(), s.end());
    if (s != act) return fail(PCR_ERR_INVALID_ARG, "order must be a permutation of the active axes");
    h->order = ord;
  } else {
    h->order = act;
  }
  const int Bmax = dtype == PCR_F32 ? 32 : 64;
  h->B = sch->nplanes ? sch->nplanes : Bmax;
  if (h->B < 1 || h->B > Bmax) return fail(PCR_ERR_INVALID_ARG, "nplanes out of range");
  h->L = sch->nlevels ? sch->nlevels : auto_levels(h->n3);
  if (h->L < 1 || h->L > max_levels(h->n3)) return fail(PCR_ERR_INVALID_ARG, "nlevels out of range");
  h->enc = sch->encoding == PCR_ENC_DEFAULT ? (sch->mode == PCR_MODE_PSNR ? 2 : 1) : sch->encoding;
  if (sch->decomp_axis < -1 || sch->decomp_axis > 2) return fail(PCR_ERR_INVALID_ARG, "decomp_axis must be -1..2");
  h->decomp = (d == 3 && h->L >= 2) ? sch->decomp_axis : -1;
  h->geo = build_streams(h->n3, h->L, sch->interp, h->order, h->decomp);
  if ((int)h->geo.size() > PCR_MAX_STREAMS) return fail(PCR_ERR_UNSUPPORTED, "too many streams");
  for (auto& g : h->geo)
    if (g.n_pad() >= (int64_t(1) << 31)) return fail(PCR_ERR_UNSUPPORTED, "stream longer than 2^31 elements");
  h->slot_words = kSegWords + h->B;
  // offsets of the device tables
  const int ns = (int)h->geo.size();
  h->plane_off.resize(ns);
  h->sign_off.resize(ns);
  h->scnt_off.resize(ns);
  h->nz_off.resize(ns);
  size_t po = 0, so = 0, co = 0, zo = 0;
  for (int i = 0; i < ns; i++) {
    const int64_t np = h->geo[i].n_pad();
    const int64_t nseg = (np + kSegElems - 1) / kSegElems;
    h->plane_off[i] = po;
    po += (size_t)h->B * (np / 32);
    h->sign_off[i] = so;
    if (h->enc == 1) so += (size_t)nseg * h->slot_words;
    h->scnt_off[i] = co;
    co += (size_t)nseg * h->B;
    h->nz_off[i] = zo;
    zo += 2 * (size_t)h->B;
  }
  h->plane_words = po;
  h->sign_area_words = so;
  h->scnt_words = co;
  h->nz_words = zo;
  return PCR_OK;
}

// Temporary device buffers of one call: from the caller's allocator, or
// carved (256-byte aligned, never freed) out of a fixed region when `bump`
// is set.
struct Scratch {
  Mem* mem;
  cudaStream_t s;
  std::vector<void*> ptrs;
  char* bump = nullptr;
  size_t cap = 0, off = 0;
  size_t* measure = nullptr;   // when set: bytes a bump carve of the same requests would need
  void* get(size_t bytes) {
    if (measure) *measure = ((*measure + 255) & ~size_t(255)) + bytes;
    if (bump) {
      const size_t o = (off + 255) & ~size_t(255);
      if (o + bytes > cap) return nullptr;
      off = o + bytes;
      return bump + o;
    }
    void* p = mem->alloc(bytes, s);
    if (p) ptrs.push_back(p);
    return p;
  }
  ~Scratch() {
    for (void* p : ptrs) mem->free(p, s);
  }
};

// ---------------------------------------------------------------------------
// a second stream beside a call's stream: the fixed-point coarse levels
// (1/8 of the points, small latency-bound kernels) run beside the level-0
// coefficient work, forked after the work both need and joined before the
// work that needs both
// ---------------------------------------------------------------------------
struct SideLane {
  cudaStream_t st = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};

static pcr_status lane_create(SideLane& l) {
  CUDA_TRY(cudaStreamCreateWithFlags(&l.st, cudaStreamNonBlocking));
  CUDA_TRY(cudaEventCreateWithFlags(&l.fork, cudaEventDisableTiming));
  CUDA_TRY(cudaEventCreateWithFlags(&l.join, cudaEventDisableTiming));
  return PCR_OK;
}

static void lane_destroy(SideLane& l) {
  if (l.join) cudaEventDestroy(l.join);
  if (l.fork) cudaEventDestroy(l.fork);
  if (l.st) cudaStreamDestroy(l.st);
  l = SideLane();
}

// lanes are taken for the enqueue of one call (its events must not be
// re-recorded by another thread meanwhile) and returned afterwards, kept per
// (device, main stream) so that calls on different streams do not queue
// their side work behind each other's; work an earlier call left queued on
// a lane's stream only delays the next user of that lane
static std::mutex g_lane_mu;
static std::map<std::pair<int, cudaStream_t>, std::vector<SideLane>> g_lane_free;

class Fork {
 public:
  // `fixed`: a lane owned by the caller (a graph being captured); else a
  // pooled one, unless the stream is being captured (then no fork).  With
  // stage tracing on there is no fork either: per-stage CUDA-event times
  // are only meaningful for stages that do not share the GPU.
  Fork(cudaStream_t main, const SideLane* fixed = nullptr) : main_(main) {
    if (g_prof_on) return;
    if (fixed) {
      lane_ = *fixed;
      return;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(main, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
      cudaGetLastError();
      return;
    }
    cudaGetDevice(&dev_);
    {
      std::lock_guard<std::mutex> lk(g_lane_mu);
      auto& v = g_lane_free[{dev_, main_}];
      if (!v.empty()) {
        lane_ = v.back();
        v.pop_back();
      }
    }
    if (!lane_.st && lane_create(lane_) != PCR_OK) {
      lane_destroy(lane_);
      cudaGetLastError();
    }
    pooled_ = lane_.st != nullptr;
  }
  ~Fork() {
    if (open_) join();   // an error path: the main stream still waits for the side work
    if (pooled_) {
      std::lock_guard<std::mutex> lk(g_lane_mu);
      g_lane_free[{dev_, main_}].push_back(lane_);
    }
  }
  cudaStream_t side() const { return open_ ? lane_.st : main_; }
  pcr_status fork() {
    if (!lane_.st) return PCR_OK;
    CUDA_TRY(cudaEventRecord(lane_.fork, main_));
    CUDA_TRY(cudaStreamWaitEvent(lane_.st, lane_.fork, 0));
    open_ = true;
    return PCR_OK;
  }
  pcr_status join() {
    if (!open_) return PCR_OK;
    open_ = false;
    CUDA_TRY(cudaEventRecord(lane_.join, lane_.st));
    CUDA_TRY(cudaStreamWaitEvent(main_, lane_.join, 0));
    return PCR_OK;
  }

 private:
  cudaStream_t main_;
  SideLane lane_;
  int dev_ = 0;
  bool pooled_ = false, open_ = false;
};

// elements per row of a decomposed region's compact array in the refactor:
// FP32 with slices normal to the fastest axis rounds rows up to 16 bytes
// (the TMA-staged decomposition needs 16-byte row strides); else dense
static int64_t comp_pitch(const pcr_handle* h, const Lat& R) {
  const int64_t cw = R.count[2];
  return (h->vk == VK_F32 && h->decomp == 2) ? (cw + 3) & ~int64_t(3) : cw;
}

// The refactor of one field, prepared on the host: its scratch carved, its
// stream descriptors filled and the arguments of every stage's launch
// recorded.  The stages of a batch then go out stage by stage across all its
// fields (enqueue_stages), each stage in as few launches as the batched
// kernels' parameter blocks allow.
struct FieldWork {
  pcr_handle* h = nullptr;
  const void* x = nullptr;
  FieldD f{};
  FieldStats* st = nullptr;
  int64_t n = 0;
  int64_t* xc = nullptr;   // fixed-point 2-grid (L >= 2)
  bool has_l0 = false;     // level 0 predicted from the original values
  TileArgs l0{};
  // coarsest level: fixed point (L >= 2) or the raw values (L = 1)
  bool coarse_fix = false;
  int coarse_level = 0;
  LatD coarse_lat{};
  void* coarse_stage = nullptr;
  unsigned long long* coarse_vmax = nullptr;
  std::vector<TileArgs> fixed;     // levels L-2 .. 1 (fixed point)
  std::vector<DecompArgs> dec;     // decomposed level-0 regions
  std::vector<int> pad_vk;         // row padding of every stream's staging
  std::vector<LatD> pad_lat;
  std::vector<void*> pad_stage;
};

// Scratch and launch arguments of one handle's refactor (geometry already
// set up, device outputs allocated); `st` receives field stats, `vmax`
// per-stream maxima.  Nothing is launched.
static pcr_status prepare_refactor(pcr_handle* h, const void* d_field, Scratch& sc, FieldStats* d_st,
                                   unsigned long long* d_vmax, unsigned long long* d_pairs,
                                   std::vector<StreamD>& sds, FieldWork& w) {
  const int ns = (int)h->geo.size();
  const FieldD f = field_desc(h);
  const size_t vb = vsize(h->vk);
  w.h = h;
  w.x = d_field;
  w.f = f;
  w.st = d_st;
  w.n = h->n3[0] * h->n3[1] * h->n3[2];
  // staging
  size_t fix_elems = 0, flt_elems = 0;
  std::vector<size_t> soff(ns);
  for (int i = 0; i < ns; i++) {
    if (h->geo[i].is_fix) {
      soff[i] = fix_elems;
      fix_elems += h->geo[i].n_pad();
    } else {
      soff[i] = flt_elems;
      flt_elems += h->geo[i].n_pad();
    }
  }
  int64_t* st_fix = (int64_t*)sc.get(fix_elems * 8);
  char* st_flt = (char*)sc.get(flt_elems * vb);
  if (!st_fix || !st_flt) return fail(PCR_ERR_OOM, "staging allocation failed");
  if (h->L >= 2) {
    w.xc = (int64_t*)sc.get((size_t)f.nc[0] * f.nc[1] * f.nc[2] * 8);
    if (!w.xc) return fail(PCR_ERR_OOM, "staging allocation failed");
  }
  // region compact arrays for the decomposition (rows pitched to 16 bytes
  // where the TMA-staged decomposition can then take them)
  std::vector<void*> comp(4, nullptr);
  std::vector<int64_t> pitch(4, 0);
  if (h->decomp >= 0)
    for (int r = 1; r <= f.d; r++) {
      const Lat R = region_lat(h->n3, 0, h->order, r);
      pitch[r] = comp_pitch(h, R);
      comp[r] = sc.get((size_t)(R.count[0] * R.count[1] * pitch[r]) * vb);
      if (!comp[r]) return fail(PCR_ERR_OOM, "staging allocation failed");
    }
  unsigned long long* c0 = &d_st->c0;
  for (int i = 0; i < ns; i++) {
    const SGeo& g = h->geo[i];
    sds[i] = stream_desc(h, i);
    sds[i].vmax = d_vmax + i;
    sds[i].pairs = d_pairs ? d_pairs + (size_t)i * h->B * h->B : nullptr;
    sds[i].stage = g.is_fix ? (void*)(st_fix + soff[i]) : (void*)(st_flt + soff[i] * vb);
  }
  // level 0 (Alg. 1 predicts it from the original values)
  if (h->L >= 2) {
    TileArgs a = level_args(h, 0, 0, d_field, nullptr);
    if (h->decomp >= 0) {
      for (int r = 1; r <= f.d; r++) {
        const Lat R = region_lat(h->n3, 0, h->order, r);
        // max |c| over level 0 for the rounding allowance, taken while the
        // coefficients are formed
        a.reg[r - 1] = tile_region(h, R, 0, pitch[r], 0, comp[r], c0);
        a.reg[r - 1].vmax_double = 1;
      }
    } else {
      level_regions(h, 0, sds, a);
    }
    w.has_l0 = true;
    w.l0 = a;
  }
  // coarsest level (raw) and the L = 1 case
  {
    const SGeo& g = h->geo[0];
    w.coarse_fix = g.is_fix;
    w.coarse_level = g.level;
    w.coarse_lat = to_latd(g.lats[0], 0);
    w.coarse_stage = sds[0].stage;
    w.coarse_vmax = sds[0].vmax;
  }
  // levels L-2 .. 1 in fixed point (Alg. 1 loop); each reads only the
  // fixed-point copy of the field, so they are independent grids
  for (int level = h->L - 2; level >= 1; level--) {
    TileArgs a = level_args(h, level, 0, (const void*)w.xc, nullptr);
    level_regions(h, level, sds, a);
    a.err = timeout_flag(w.st);
    w.fixed.push_back(a);
  }
  if (h->decomp >= 0)
    for (int r = 1; r <= f.d; r++) {
      DecompArgs da{};
      decomp_subs(h, r, sds, da);
      da.retrieve = 0;
      da.comp = comp[r];
      da.pitch = pitch[r];
      da.c0 = nullptr;   // max |c| taken by the level-0 prediction
      da.err = &d_st->timeout;
      w.dec.push_back(da);
    }
  // the row padding of every stream's staging (the kernels above write only
  // real elements, so this may run in any order with them)
  for (int i = 1; i < ns; i++)
    for (int k = 0; k < sds[i].nlat; k++)
      if (sds[i].lat[k].row_pad > sds[i].lat[k].count[2]) {
        w.pad_vk.push_back(h->geo[i].is_fix ? VK_FIX : h->vk);
        w.pad_lat.push_back(sds[i].lat[k]);
        w.pad_stage.push_back(sds[i].stage);
      }
  return PCR_OK;
}

// The coefficient stages of a batch's refactors, stage by stage across the
// fields; within a stage the fields' grids are independent, and each stage
// reads only what earlier stages wrote.
// Level 0 and what every later stage needs: statistics, level-0 prediction,
// the exponent, the row padding of every staging.
static void stages_level0(const std::vector<FieldWork>& ws, cudaStream_t s) {
  const int vks[2] = {VK_F32, VK_F64};
  {
    // fields without a level 0 (L = 1): a statistics pass of their own; the
    // others' statistics are taken while their level 0 is predicted
    Prof pf("stats", s);
    for (int vk : vks) {
      std::vector<const void*> xs;
      std::vector<int64_t> ns;
      std::vector<FieldStats*> sts;
      for (const FieldWork& w : ws)
        if (w.h->vk == vk && !w.has_l0) {
          xs.push_back(w.x);
          ns.push_back(w.n);
          sts.push_back(w.st);
        }
      if (!xs.empty()) launch_stats_multi(vk, xs.data(), ns.data(), sts.data(), (int)xs.size(), s);
    }
  }
  {
    Prof pf("interp_level0", s);
    for (int vk : vks) {
      std::vector<TileArgs> l0;
      for (const FieldWork& w : ws)
        if (w.h->vk == vk && w.has_l0) {
          l0.push_back(w.l0);
          l0.back().stats = w.st;
          l0.back().err = timeout_flag(w.st);
        }
      launch_tile_interp_multi(vk, l0.data(), (int)l0.size(), s);
    }
    std::vector<FieldStats*> fin;
    for (const FieldWork& w : ws)
      if (w.has_l0) fin.push_back(w.st);
    if (!fin.empty()) launch_finalize_multi(fin.data(), (int)fin.size(), s);
  }
  {
    std::vector<int> pv;
    std::vector<LatD> pl;
    std::vector<void*> ps;
    for (const FieldWork& w : ws) {
      pv.insert(pv.end(), w.pad_vk.begin(), w.pad_vk.end());
      pl.insert(pl.end(), w.pad_lat.begin(), w.pad_lat.end());
      ps.insert(ps.end(), w.pad_stage.begin(), w.pad_stage.end());
    }
    Prof pf("zero_pads", s);
    launch_zero_pads_multi(pv.data(), pl.data(), ps.data(), (int)pv.size(), s);
  }
}

// The fixed-point coarse levels: fixed-point copy, coarsest level, levels
// L-2 .. 1 (after stages_level0: they need the exponent).
static void stages_fixed(const std::vector<FieldWork>& ws, cudaStream_t s) {
  const int vks[2] = {VK_F32, VK_F64};
  {
    Prof pf("to_fixed", s);
    for (int vk : vks) {
      std::vector<const void*> xs;
      std::vector<FieldD> fs;
      std::vector<const FieldStats*> sts;
      std::vector<int64_t*> xcs;
      for (const FieldWork& w : ws)
        if (w.h->vk == vk && w.xc) {
          xs.push_back(w.x);
          fs.push_back(w.f);
          sts.push_back(w.st);
          xcs.push_back(w.xc);
        }
      if (!xs.empty()) launch_to_fixed_multi(vk, xs.data(), fs.data(), sts.data(), xcs.data(), (int)xs.size(), s);
    }
  }
  {
    Prof pf("coarsest", s);
    std::vector<FieldD> fs;
    std::vector<int> levels;
    std::vector<LatD> lats;
    std::vector<const int64_t*> xcs;
    std::vector<int64_t*> outs;
    std::vector<unsigned long long*> vms;
    for (const FieldWork& w : ws) {
      if (w.coarse_fix) {
        fs.push_back(w.f);
        levels.push_back(w.coarse_level);
        lats.push_back(w.coarse_lat);
        xcs.push_back(w.xc);
        outs.push_back((int64_t*)w.coarse_stage);
        vms.push_back(w.coarse_vmax);
      } else {
        launch_raw_stage(w.h->vk, w.f, w.coarse_lat, w.x, w.coarse_stage, w.coarse_vmax, s);
      }
    }
    if (!fs.empty())
      launch_coarsest_multi(fs.data(), levels.data(), lats.data(), xcs.data(), outs.data(), vms.data(),
                            (int)fs.size(), s);
  }
  {
    std::vector<TileArgs> lv;
    for (const FieldWork& w : ws) lv.insert(lv.end(), w.fixed.begin(), w.fixed.end());
    Prof pf("interp_fixed_levels", s);
    launch_tile_interp_multi(VK_FIX, lv.data(), (int)lv.size(), s);
  }
}

// The level-0 decomposition (after stages_level0).
static void stages_float(const std::vector<FieldWork>& ws, cudaStream_t s) {
  const int vks[2] = {VK_F32, VK_F64};
  {
    Prof pf("decompose", s);
    for (int vk : vks) {
      std::vector<DecompArgs> das;
      for (const FieldWork& w : ws)
        if (w.h->vk == vk) das.insert(das.end(), w.dec.begin(), w.dec.end());
      if (!das.empty()) launch_tile_decomp_multi(vk, das.data(), (int)das.size(), s);
    }
  }
}

static pcr_status finish_refactor(pcr_handle* h, const FieldStats& st, const std::vector<unsigned long long>& vm,
                                  const std::vector<uint32_t>& nz,
                                  const std::vector<uint64_t>* pairs) {
  if (st.bad) return fail(PCR_ERR_INVALID_ARG, "field contains NaN or Inf");
  if (st.timeout) return fail(PCR_ERR_TIMEOUT, "a device wait of the refactor gave up");
  auto inv = [](unsigned long long k) {
    unsigned long long u = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
    double d;
    std::memcpy(&d, &u, 8);
    return d;
  };
  h->xmin = inv(st.xmin_key);
  h->xmax = inv(st.xmax_key);
  h->M = std::max(std::fabs(h->xmin), std::fabs(h->xmax));
  h->G = st.G;
  h->h = std::ldexp(1.0, h->G - fix_bits(h->vk, h->L));
  const int ns = (int)h->geo.size();
  h->E.assign(ns, 0);
  h->sh.assign(ns, 0);
  h->vmax.assign(ns, 0);
  h->tabs.assign(ns, Tab());
  h->sign_words.assign(ns, {});
  h->plane_nz.assign(ns, {});
  h->pairs.assign(ns, {});
  double c0;
  std::memcpy(&c0, &st.c0, 8);
  h->C0 = h->L == 1 ? h->M : c0;
  h->C0c = h->C0;
  for (int i = 0; i < ns; i++) {
    const SGeo& g = h->geo[i];
    const unsigned long long v = vm[i];
    if (g.is_fix) {
      h->vmax[i] = (double)v;
      h->E[i] = v ? 64 - __builtin_clzll(v) : 0;
      const int lim = h->enc == 2 ? h->B - 3 : h->B;
      h->sh[i] = h->E[i] > lim ? h->E[i] - lim : 0;
    } else {
      double dv;
      if (h->vk == VK_F32) {
        float fv;
        const uint32_t b32 = (uint32_t)v;
        std::memcpy(&fv, &b32, 4);
        dv = fv;
      } else {
        std::memcpy(&dv, &v, 8);
      }
      h->vmax[i] = dv;
      int E = 0;
      if (dv > 0) std::frexp(dv, &E);
      h->E[i] = E;
      if (g.level == 0 && h->L >= 2) h->C0 = std::max(h->C0, dv);
      if (g.level == 0 && h->L >= 2 && g.sub <= 1) h->C0c = std::max(h->C0c, dv);
    }
    const int64_t nseg = (g.n_pad() + kSegElems - 1) / kSegElems;
    h->plane_nz[i].assign(nz.begin() + h->nz_off[i], nz.begin() + h->nz_off[i] + h->B);
    h->sign_words[i].assign(nz.begin() + h->nz_off[i] + h->B, nz.begin() + h->nz_off[i] + 2 * h->B);
    if (pairs) h->pairs[i].assign(pairs->begin() + (size_t)i * h->B * h->B, pairs->begin() + (size_t)(i + 1) * h->B * h->B);
  }
  for (int i = 0; i < ns; i++) compute_tables(h, i, pairs ? &h->pairs[i] : nullptr, keeps_pairs(h));
  build_meta(h);
  return PCR_OK;
}

static pcr_status alloc_handle_buffers(pcr_handle* h, cudaStream_t s) {
  // one allocation, carved in 256-byte aligned pieces
  size_t items = 0;
  for (auto& g : h->geo) items += (g.n_pad() + kSegElems - 1) / kSegElems;
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  const size_t b_pl = al(h->plane_words * 4), b_sg = al(std::max<size_t>(h->sign_area_words, 1) * 4),
               b_sc = al(std::max<size_t>(h->scnt_words, 1) * 4), b_nz = al(h->nz_words * 4),
               b_it = al(std::max<size_t>(items, 1) * sizeof(WorkItem));
  CUDA_TRY(cudaGetDevice(&h->device));
  h->d_block = h->mem.alloc(b_pl + b_sg + b_sc + b_nz + b_it + 256, s);
  if (!h->d_block) return fail(PCR_ERR_OOM, "handle allocation failed");
  char* p = (char*)(((uintptr_t)h->d_block + 255) & ~uintptr_t(255));
  h->d_planes = (uint32_t*)p;
  p += b_pl;
  h->d_signs = (uint32_t*)p;
  p += b_sg;
  h->d_scnt = (uint32_t*)p;
  p += b_sc;
  h->d_nz = (uint32_t*)p;
  p += b_nz;
  h->d_items_all = (WorkItem*)p;
  h->items_ready = false;
  // unused tails of sign slots stay zero, and so do the sign counts of
  // streams without sign sub-streams (negabinary), so a handle's contents
  // never depend on what the allocator handed back
  if (h->sign_area_words) CUDA_TRY(cudaMemsetAsync(h->d_signs, 0, h->sign_area_words * 4, s));
  if (h->scnt_words) CUDA_TRY(cudaMemsetAsync(h->d_scnt, 0, h->scnt_words * 4, s));
  return PCR_OK;
}

struct BatchDev {
  FieldStats* st;
  unsigned long long* vmax;
  unsigned long long* pairs;
};

// ---------------------------------------------------------------------------
// batched refactor: one work list per encode kind for the whole batch
// ---------------------------------------------------------------------------
// Offsets of each field's statistics in the batch's device blocks.
struct BatchLayout {
  std::vector<size_t> vm_off, pr_off, nz_off;
  size_t nv = 0, npairs = 0, nnz = 0;
  explicit BatchLayout(const std::vector<pcr_handle*>& hs) {
    for (pcr_handle* h : hs) {
      vm_off.push_back(nv);
      nv += h->geo.size();
      pr_off.push_back(npairs);
      if (keeps_pairs(h)) npairs += h->geo.size() * h->B * h->B;
      nz_off.push_back(nnz);
      nnz += h->nz_words;
    }
  }
};

// Host side of the batch's copies: the sources of the uploads (statistics
// initialisers, stream descriptors, work items) and the destinations of the
// read-backs.  Pageable vectors for a one-off call; for a captured graph the
// same roles are played by pinned buffers that outlive the graph (`pinned`).
struct BatchStage {
  bool pinned = false;
  bool pinned_out = false;   // only the read-backs (st, vm, pairs, nz) are pinned, set by the caller
  FieldStats* st_init = nullptr;
  StreamD* sd = nullptr;
  WorkItem* items = nullptr;
  size_t cap_sd = 0, cap_items = 0;
  FieldStats* st = nullptr;
  unsigned long long* vm = nullptr;
  uint64_t* pairs = nullptr;
  uint32_t* nz = nullptr;
  // pageable storage
  std::vector<FieldStats> v_init, v_st;
  std::vector<StreamD> v_sd;
  std::vector<WorkItem> v_items;
  std::vector<unsigned long long> v_vm;
  std::vector<uint64_t> v_pairs;
  std::vector<uint32_t> v_nz;
  size_t used_sd = 0, used_items = 0;   // descriptors and items the batch needed
};

// Enqueue the refactor of every handle of a batch (buffers allocated) and the
// read-back of its statistics; no synchronisation.  `clear_signs` zeroes the
// sign slots first (a replayed graph must not keep an earlier run's tails).
static pcr_status enqueue_batch(const std::vector<pcr_handle*>& hs, const void* const* d_fields, cudaStream_t s,
                                Scratch& sc, const BatchLayout& L, BatchStage& io, bool clear_signs,
                                const SideLane* lane = nullptr) {
  const int n = (int)hs.size();
  FieldStats* d_st = (FieldStats*)sc.get(sizeof(FieldStats) * n);
  unsigned long long* d_vm = (unsigned long long*)sc.get(L.nv * 8);
  unsigned long long* d_pairs = L.npairs ? (unsigned long long*)sc.get(L.npairs * 8) : nullptr;
  if (!d_st || !d_vm || (L.npairs && !d_pairs)) return fail(PCR_ERR_OOM, "statistics allocation failed");
  if (!io.pinned) {
    io.v_init.resize(n);
    io.st_init = io.v_init.data();
  }
  for (int k = 0; k < n; k++) {
    FieldStats& x = io.st_init[k];
    std::memset(&x, 0, sizeof(x));
    x.xmin_key = ~0ull;
  }
  CUDA_TRY(cudaMemcpyAsync(d_st, io.st_init, sizeof(FieldStats) * n, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemsetAsync(d_vm, 0, L.nv * 8, s));
  if (L.npairs) CUDA_TRY(cudaMemsetAsync(d_pairs, 0, L.npairs * 8, s));
  // every handle's plane counts (and, when asked, sign slots and counts)
  // zeroed in one launch
  {
    std::vector<WordsItem> z;
    for (int k = 0; k < n; k++) {
      z.push_back({hs[k]->d_nz, nullptr, (int64_t)hs[k]->nz_words});
      if (clear_signs) {
        z.push_back({hs[k]->d_signs, nullptr, (int64_t)hs[k]->sign_area_words});
        z.push_back({hs[k]->d_scnt, nullptr, (int64_t)hs[k]->scnt_words});
      }
    }
    launch_words_multi(z.data(), (int)z.size(), s);
  }
  // coefficient stages of every field, stage by stage; encode work lists
  // for the whole batch
  std::vector<FieldWork> ws(n);
  std::vector<StreamD> all;
  std::vector<WorkItem> items[2][2];  // [w64][fixed?]
  int pairs_mode[2][2] = {{-1, -1}, {-1, -1}};
  for (int k = 0; k < n; k++) {
    pcr_handle* h = hs[k];
    std::vector<StreamD> sds(h->geo.size());
    pcr_status e = prepare_refactor(h, d_fields[k], sc, d_st + k, d_vm + L.vm_off[k],
                                    keeps_pairs(h) ? d_pairs + L.pr_off[k] : nullptr, sds, ws[k]);
    if (e) return e;
    for (size_t i = 0; i < sds.size(); i++) {
      const int idx = (int)all.size();
      all.push_back(sds[i]);
      const int fx = sds[i].is_fix;
      const int pm = keeps_pairs(h);
      if (pairs_mode[h->w64][fx] < 0) pairs_mode[h->w64][fx] = pm;
      else if (pairs_mode[h->w64][fx] != pm) return fail(PCR_ERR_UNSUPPORTED, "mixed EB/PSNR modes in one batch");
      for (int64_t g = 0; g < sds[i].nseg; g++) items[h->w64][fx].push_back({idx, (int)g});
    }
  }
  size_t nit = 0;
  for (int a = 0; a < 2; a++)
    for (int b = 0; b < 2; b++) nit += items[a][b].size();
  io.used_sd = all.size();
  io.used_items = nit;
  StreamD* d_sd = (StreamD*)sc.get(all.size() * sizeof(StreamD));
  WorkItem* d_items = (WorkItem*)sc.get(std::max<size_t>(nit, 1) * sizeof(WorkItem));
  if (!d_sd || !d_items) return fail(PCR_ERR_OOM, "work list allocation failed");
  if (!io.pinned) {
    io.v_sd = all;
    io.sd = io.v_sd.data();
    io.v_items.resize(std::max<size_t>(nit, 1));
    io.items = io.v_items.data();
  } else if (all.size() > io.cap_sd || nit > io.cap_items) {
    return fail(PCR_ERR_INVALID_ARG, "batch work list larger than its staging");
  } else {
    std::memcpy(io.sd, all.data(), all.size() * sizeof(StreamD));
  }
  size_t off = 0;
  for (int a = 0; a < 2; a++)
    for (int b = 0; b < 2; b++) {
      if (items[a][b].empty()) continue;
      std::memcpy(io.items + off, items[a][b].data(), items[a][b].size() * sizeof(WorkItem));
      off += items[a][b].size();
    }
  CUDA_TRY(cudaMemcpyAsync(d_sd, io.sd, all.size() * sizeof(StreamD), cudaMemcpyHostToDevice, s));
  if (nit) CUDA_TRY(cudaMemcpyAsync(d_items, io.items, nit * sizeof(WorkItem), cudaMemcpyHostToDevice, s));
  // level 0 on the call's stream; then the fixed-point coarse levels and
  // their encode beside the decomposition and the level-0 encode
  stages_level0(ws, s);
  {
    Fork fk(s, lane);
    pcr_status e = fk.fork();
    if (e) return e;
    const cudaStream_t sf = fk.side();
    stages_fixed(ws, sf);
    stages_float(ws, s);
    off = 0;
    for (int a = 0; a < 2; a++)
      for (int b = 0; b < 2; b++) {
        if (items[a][b].empty()) continue;
        const int vk = b ? VK_FIX : (a ? VK_F64 : VK_F32);
        const cudaStream_t es = b ? sf : s;
        {
          Prof pf(b ? "encode_fixed" : "encode_float", es);
          launch_encode(vk, a, pairs_mode[a][b] > 0, d_sd, d_items + off, (int)items[a][b].size(), es);
        }
        off += items[a][b].size();
      }
    e = fk.join();
    if (e) return e;
  }
  // each handle's whole-retrieval work list, kept on the device (one upload
  // for the batch, scattered by one launch)
  std::vector<WorkItem> li;
  std::vector<std::pair<pcr_handle*, size_t>> li_at;
  // one handle: its encode work list (floating-point streams, then fixed
  // point, streams and segments in order) is that list already
  if (n == 1 && !hs[0]->items_ready && nit) {
    pcr_handle* h = hs[0];
    for (int fx = 0; fx < 2; fx++) {
      h->items_n[fx] = 0;
      for (int i = 0; i < (int)h->geo.size(); i++)
        if ((int)h->geo[i].is_fix == fx) h->items_n[fx] += (h->geo[i].n_pad() + kSegElems - 1) / kSegElems;
    }
    if ((size_t)(h->items_n[0] + h->items_n[1]) == nit) {
      CUDA_TRY(cudaMemcpyAsync(h->d_items_all, d_items, nit * sizeof(WorkItem), cudaMemcpyDeviceToDevice, s));
      h->items_ready = true;
    }
  }
  for (int k = 0; k < n; k++) {
    pcr_handle* h = hs[k];
    if (h->items_ready) continue;
    const size_t at = li.size();
    for (int fx = 0; fx < 2; fx++) {
      h->items_n[fx] = 0;
      for (int i = 0; i < (int)h->geo.size(); i++) {
        if ((int)h->geo[i].is_fix != fx) continue;
        const int64_t nseg = (h->geo[i].n_pad() + kSegElems - 1) / kSegElems;
        for (int64_t g = 0; g < nseg; g++) li.push_back({i, (int)g});
        h->items_n[fx] += nseg;
      }
    }
    if (li.size() > at) li_at.push_back({h, at});
  }
  if (!li.empty()) {
    static_assert(sizeof(WorkItem) % 4 == 0, "work items are whole words");
    if (li_at.size() == 1) {
      CUDA_TRY(cudaMemcpyAsync(li_at[0].first->d_items_all, li.data(), li.size() * sizeof(WorkItem),
                               cudaMemcpyHostToDevice, s));
    } else {
      WorkItem* d_li = (WorkItem*)sc.get(li.size() * sizeof(WorkItem));
      if (!d_li) return fail(PCR_ERR_OOM, "work list allocation failed");
      CUDA_TRY(cudaMemcpyAsync(d_li, li.data(), li.size() * sizeof(WorkItem), cudaMemcpyHostToDevice, s));
      std::vector<WordsItem> cp;
      for (size_t q = 0; q < li_at.size(); q++) {
        const size_t end = q + 1 < li_at.size() ? li_at[q + 1].second : li.size();
        cp.push_back({(uint32_t*)li_at[q].first->d_items_all, (const uint32_t*)(d_li + li_at[q].second),
                      (int64_t)((end - li_at[q].second) * sizeof(WorkItem) / 4)});
      }
      launch_words_multi(cp.data(), (int)cp.size(), s);
    }
    // (a copy from pageable memory has read its source when the call returns)
    for (auto& q : li_at) q.first->items_ready = true;
  }
  CUDA_TRY(cudaGetLastError());
  // read-back of the statistics the host tables need
  if (!io.pinned && !io.pinned_out) {
    io.v_st.resize(n);
    io.st = io.v_st.data();
    io.v_vm.resize(std::max<size_t>(L.nv, 1));
    io.vm = io.v_vm.data();
    io.v_pairs.resize(std::max<size_t>(L.npairs, 1));
    io.pairs = io.v_pairs.data();
    io.v_nz.resize(std::max<size_t>(L.nnz, 1));
    io.nz = io.v_nz.data();
  }
  CUDA_TRY(cudaMemcpyAsync(io.st, d_st, sizeof(FieldStats) * n, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(io.vm, d_vm, L.nv * 8, cudaMemcpyDeviceToHost, s));
  if (L.npairs) CUDA_TRY(cudaMemcpyAsync(io.pairs, d_pairs, L.npairs * 8, cudaMemcpyDeviceToHost, s));
  if (n == 1) {
    CUDA_TRY(cudaMemcpyAsync(io.nz, hs[0]->d_nz, hs[0]->nz_words * 4, cudaMemcpyDeviceToHost, s));
  } else {   // the handles' plane counts gathered by one launch, read back by one copy
    uint32_t* d_nz = (uint32_t*)sc.get(std::max<size_t>(L.nnz, 1) * 4);
    if (!d_nz) return fail(PCR_ERR_OOM, "statistics allocation failed");
    std::vector<WordsItem> cp;
    for (int k = 0; k < n; k++) cp.push_back({d_nz + L.nz_off[k], hs[k]->d_nz, (int64_t)hs[k]->nz_words});
    launch_words_multi(cp.data(), (int)cp.size(), s);
    CUDA_TRY(cudaMemcpyAsync(io.nz, d_nz, L.nnz * 4, cudaMemcpyDeviceToHost, s));
  }
  return PCR_OK;
}

// f(k) for k in [0, n) on up to 16 host threads (the caller's included):
// independent per-field host work of a batch.  Returns the failing status
// of the lowest k, with its message.
template <class F>
static pcr_status parallel_for(int n, F f) {
  const unsigned hw = std::thread::hardware_concurrency();
  const int nt = std::max(1, std::min(n, std::min(16, hw ? (int)hw : 1)));
  if (nt == 1 || n < 4) {
    for (int k = 0; k < n; k++) {
      pcr_status e = f(k);
      if (e) return e;
    }
    return PCR_OK;
  }
  std::vector<pcr_status> st(n, PCR_OK);
  std::vector<std::string> msg(n);
  std::atomic<int> next{0};
  auto work = [&]() {
    for (int k; (k = next.fetch_add(1)) < n;) {
      try {   // nothing thrown may leave a worker thread
        st[k] = f(k);
        if (st[k]) msg[k] = g_err;   // this thread's message
      } catch (const std::bad_alloc&) {
        st[k] = PCR_ERR_OOM;
        msg[k] = "host allocation failed";
      } catch (...) {
        st[k] = PCR_ERR_INVALID_ARG;
        msg[k] = "unexpected host error";
      }
    }
  };
  std::vector<std::thread> th;
  try {
    for (int t = 1; t < nt; t++) th.emplace_back(work);
  } catch (...) {   // fewer threads: this one takes the rest
  }
  work();
  for (auto& t : th) t.join();
  for (int k = 0; k < n; k++)
    if (st[k]) return fail(st[k], msg[k]);
  return PCR_OK;
}

// host tables of every handle from a completed batch's read-backs (the
// handles are independent: several at a time)
static pcr_status finish_batch(const std::vector<pcr_handle*>& hs, const BatchLayout& L, const BatchStage& io) {
  return parallel_for((int)hs.size(), [&](int k) -> pcr_status {
    pcr_handle* h = hs[k];
    std::vector<unsigned long long> v(io.vm + L.vm_off[k], io.vm + L.vm_off[k] + h->geo.size());
    std::vector<uint32_t> nz(io.nz + L.nz_off[k], io.nz + L.nz_off[k] + h->nz_words);
    std::vector<uint64_t> pk;
    if (keeps_pairs(h))
      pk.assign(io.pairs + L.pr_off[k], io.pairs + L.pr_off[k] + h->geo.size() * h->B * h->B);
    pcr_status e = finish_refactor(h, io.st[k], v, nz, keeps_pairs(h) ? &pk : nullptr);
    if (e) return e;
    std::lock_guard<std::mutex> lk(h->plan_mu);   // planner units follow the new tables
    h->units_ok[0] = h->units_ok[1] = false;
    return PCR_OK;
  });
}

static pcr_status make_batch_handles(int n, const void* const* d_fields, const int* ndims,
                                     const int64_t* const* dims, const int* dtypes, const pcr_scheme* schemes,
                                     const Mem& mem, cudaStream_t s, std::vector<std::unique_ptr<pcr_handle>>& hs) {
  hs.resize(n);
  for (int k = 0; k < n; k++) {
    pcr_status e = validate(d_fields[k], ndims[k], dims[k], dtypes[k], &schemes[k]);
    if (e) return e;
    hs[k].reset(new pcr_handle());
    hs[k]->mem = mem;
    e = setup_handle(hs[k].get(), ndims[k], dims[k], dtypes[k], &schemes[k]);
    if (e) return e;
    e = alloc_handle_buffers(hs[k].get(), s);
    if (e) return e;
  }
  return PCR_OK;
}

// bytes of temporary device memory the refactor of `h` takes inside a batch
// (upper bound with the 256-byte alignment of every piece): stream staging,
// the fixed-point 2-grid, the decomposed regions' compact arrays, and its
// share of the batch's statistics, descriptors and work items
static size_t refactor_scratch_bytes(const pcr_handle* h) {
  const size_t w = vsize(h->vk);
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  size_t fix = 0, flt = 0, items = 0;
  for (auto& g : h->geo) {
    (g.is_fix ? fix : flt) += g.n_pad();
    items += (g.n_pad() + kSegElems - 1) / kSegElems;
  }
  const size_t ns = h->geo.size();
  size_t t = al(fix * 8) + al(flt * w) + al(ns * sizeof(StreamD)) + al(std::max<size_t>(items, 1) * sizeof(WorkItem)) +
             al(sizeof(FieldStats)) + al(ns * 8);
  if (keeps_pairs(h)) t += al(ns * h->B * h->B * 8);
  // its share of the batch's work-list upload and plane-count gather
  t += al(std::max<size_t>(items, 1) * sizeof(WorkItem)) + al(std::max<size_t>(h->nz_words, 1) * 4);
  if (h->L >= 2) {
    size_t nc = 1;
    for (int a = 0; a < 3; a++) nc *= h->n3[a] > 1 ? (h->n3[a] - 1) / 2 + 1 : 1;
    t += al(nc * 8);
  }
  if (h->decomp >= 0)
    for (int r = 1; r <= (int)h->order.size(); r++) {
      const Lat R = region_lat(h->n3, 0, h->order, r);
      t += al((size_t)(R.count[0] * R.count[1] * comp_pitch(h, R)) * w);
    }
  return t + 256;
}

// one device block for all of a call's temporary buffers, carved in order:
// a single trip through the caller's allocator instead of one per buffer
struct ScratchBlock {
  Mem* mem;
  cudaStream_t s;
  void* p = nullptr;
  ScratchBlock(Mem* m, cudaStream_t st, size_t bytes, Scratch& sc) : mem(m), s(st) {
    p = mem->alloc(bytes + 256, s);
    if (p) {
      sc.bump = (char*)(((uintptr_t)p + 255) & ~uintptr_t(255));
      sc.cap = bytes;
    }
  }
  ~ScratchBlock() {
    if (p) mem->free(p, s);
  }
};

extern "C" pcr_status pcr_refactor_batch(int n, const void* const* d_fields, const int* ndims,
                                         const int64_t* const* dims, const int* dtypes, const pcr_scheme* schemes,
                                         const pcr_allocator* alloc, void* cuda_stream, pcr_handle** outs) try {
  if (n <= 0 || !d_fields || !ndims || !dims || !dtypes || !schemes || !outs)
    return fail(PCR_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  Mem mem = make_mem(alloc);
  std::vector<pcr_scheme> sch;
  pcr_status e = resolve_auto(n, d_fields, ndims, dims, dtypes, schemes, alloc, cuda_stream, sch);
  if (e) return e;
  std::vector<std::unique_ptr<pcr_handle>> own;
  e = make_batch_handles(n, d_fields, ndims, dims, dtypes, sch.data(), mem, s, own);
  if (e) return e;
  std::vector<pcr_handle*> hs;
  for (auto& h : own) hs.push_back(h.get());
  const BatchLayout L(hs);
  BatchStage io;
  {
    size_t need = 256 * 8;   // slack: the batch-level pieces are aligned once each
    for (pcr_handle* h : hs) need += refactor_scratch_bytes(h);
    Scratch sc{&mem, s, {}};
    ScratchBlock blk(&mem, s, need, sc);
    if (!blk.p) return fail(PCR_ERR_OOM, "scratch allocation failed");
    e = enqueue_batch(hs, d_fields, s, sc, L, io, false);
    if (e) return e;
    CUDA_TRY(cudaStreamSynchronize(s));
  }
  e = finish_batch(hs, L, io);
  if (e) return e;
  for (int k = 0; k < n; k++) outs[k] = own[k].release();
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

// ---------------------------------------------------------------------------
// asynchronous refactor: enqueue now, finish the host tables later
// ---------------------------------------------------------------------------
// pinned read-back blocks, kept for reuse by later jobs (a block is only
// returned once the copies into it have completed)
static std::mutex g_pin_mu;
static std::vector<std::pair<size_t, void*>> g_pin_free;

static void* pin_acquire(size_t bytes, size_t& got) {
  {
    std::lock_guard<std::mutex> lk(g_pin_mu);
    for (size_t i = 0; i < g_pin_free.size(); i++)
      if (g_pin_free[i].first >= bytes) {
        void* p = g_pin_free[i].second;
        got = g_pin_free[i].first;
        g_pin_free.erase(g_pin_free.begin() + (long)i);
        return p;
      }
  }
  const size_t sz = (bytes + 65535) & ~size_t(65535);
  void* p = nullptr;
  if (cudaMallocHost(&p, sz) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  got = sz;
  return p;
}

static void pin_release(void* p, size_t bytes) {
  std::lock_guard<std::mutex> lk(g_pin_mu);
  g_pin_free.push_back({bytes, p});
}

struct pcr_refactor_job {
  Mem mem;
  cudaStream_t s = nullptr;
  std::unique_ptr<pcr_handle> own;
  std::vector<pcr_handle*> hs;
  std::unique_ptr<BatchLayout> layout;
  BatchStage io;
  Scratch sc{nullptr, nullptr, {}};
  std::unique_ptr<ScratchBlock> blk;
  void* pin = nullptr;
  size_t pin_bytes = 0;
  cudaEvent_t done = nullptr;
  bool enqueued = false;
  ~pcr_refactor_job() {
    // nothing the job owns is released while its copies or kernels may run
    if (done) cudaEventSynchronize(done);
    else if (enqueued) cudaStreamSynchronize(s);
    blk.reset();
    if (done) cudaEventDestroy(done);
    if (pin) pin_release(pin, pin_bytes);
  }
};

extern "C" pcr_status pcr_refactor_begin(const void* d_field, int ndim, const int64_t* dims, int dtype,
                                         const pcr_scheme* scheme, const pcr_allocator* alloc, void* cuda_stream,
                                         pcr_refactor_job** out) try {
  if (!out || !d_field || !dims || !scheme) return fail(PCR_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  std::unique_ptr<pcr_refactor_job> j(new pcr_refactor_job());
  j->s = (cudaStream_t)cuda_stream;
  j->mem = make_mem(alloc);
  const void* f[1] = {d_field};
  const int nd[1] = {ndim};
  const int64_t* dm[1] = {dims};
  const int dt[1] = {dtype};
  std::vector<pcr_scheme> sch;
  pcr_status e = resolve_auto(1, f, nd, dm, dt, scheme, alloc, cuda_stream, sch);
  if (e) return e;
  std::vector<std::unique_ptr<pcr_handle>> own;
  e = make_batch_handles(1, f, nd, dm, dt, sch.data(), j->mem, j->s, own);
  if (e) return e;
  j->own = std::move(own[0]);
  j->hs.push_back(j->own.get());
  j->layout.reset(new BatchLayout(j->hs));
  const BatchLayout& L = *j->layout;
  // pinned targets of the read-backs, so that the enqueue does not wait
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t b_st = sizeof(FieldStats), b_vm = 8 * std::max<size_t>(L.nv, 1),
               b_pr = 8 * std::max<size_t>(L.npairs, 1), b_nz = 4 * std::max<size_t>(L.nnz, 1);
  j->pin = pin_acquire(al(b_st) + al(b_vm) + al(b_pr) + al(b_nz), j->pin_bytes);
  if (!j->pin) return fail(PCR_ERR_OOM, "pinned read-back allocation failed");
  char* p = (char*)j->pin;
  j->io.pinned_out = true;
  j->io.st = (FieldStats*)p;
  p += al(b_st);
  j->io.vm = (unsigned long long*)p;
  p += al(b_vm);
  j->io.pairs = (uint64_t*)p;
  p += al(b_pr);
  j->io.nz = (uint32_t*)p;
  j->sc.mem = &j->mem;
  j->sc.s = j->s;
  j->blk.reset(new ScratchBlock(&j->mem, j->s, 256 * 8 + refactor_scratch_bytes(j->own.get()), j->sc));
  if (!j->blk->p) return fail(PCR_ERR_OOM, "scratch allocation failed");
  j->enqueued = true;
  e = enqueue_batch(j->hs, f, j->s, j->sc, L, j->io, false);
  if (e) return e;
  CUDA_TRY(cudaEventCreateWithFlags(&j->done, cudaEventDisableTiming));
  CUDA_TRY(cudaEventRecord(j->done, j->s));
  *out = j.release();
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" pcr_status pcr_refactor_end(pcr_refactor_job* job, pcr_handle** out) try {
  if (!job || !out) return fail(PCR_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  std::unique_ptr<pcr_refactor_job> j(job);   // consumed, whatever the outcome
  CUDA_TRY(cudaEventSynchronize(j->done));
  pcr_status e = finish_batch(j->hs, *j->layout, j->io);
  if (e) return e;
  *out = j->own.release();
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" void pcr_refactor_job_free(pcr_refactor_job* job) { delete job; }

// ---------------------------------------------------------------------------
// batched refactor captured in one CUDA graph
// ---------------------------------------------------------------------------
struct pcr_refactor_graph {
  Mem mem;
  std::vector<std::unique_ptr<pcr_handle>> own;
  std::vector<pcr_handle*> hs;
  std::vector<const void*> fields;
  std::unique_ptr<BatchLayout> layout;
  BatchStage io;
  void* arena = nullptr;
  size_t arena_bytes = 0;
  void* pinned = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;
  size_t nodes = 0;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  double gpu_ms = 0.0, host_ms = 0.0;   // of the last run
  SideLane lane;                        // the captured fork's second stream
  ~pcr_refactor_graph() {
    for (cudaEvent_t e : ev)
      if (e) cudaEventDestroy(e);
    lane_destroy(lane);
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (cap) cudaStreamDestroy(cap);
    if (pinned) cudaFreeHost(pinned);
    if (arena) mem.free(arena, nullptr);
  }
};

extern "C" pcr_status pcr_refactor_graph_create(int n, const void* const* d_fields, const int* ndims,
                                                const int64_t* const* dims, const int* dtypes,
                                                const pcr_scheme* schemes, const pcr_allocator* alloc,
                                                void* cuda_stream, pcr_refactor_graph** out) try {
  if (n <= 0 || !d_fields || !ndims || !dims || !dtypes || !schemes || !out)
    return fail(PCR_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  std::unique_ptr<pcr_refactor_graph> g(new pcr_refactor_graph());
  g->mem = make_mem(alloc);
  std::vector<pcr_scheme> sch;
  pcr_status e = resolve_auto(n, d_fields, ndims, dims, dtypes, schemes, alloc, cuda_stream, sch);
  if (e) return e;
  e = make_batch_handles(n, d_fields, ndims, dims, dtypes, sch.data(), g->mem, s, g->own);
  if (e) return e;
  for (auto& h : g->own) g->hs.push_back(h.get());
  g->fields.assign(d_fields, d_fields + n);
  g->layout.reset(new BatchLayout(g->hs));
  const BatchLayout& L = *g->layout;
  // 1. one uncaptured run: autotunes the level schedule of these shapes,
  //    measures the scratch the batch needs and leaves valid handles
  size_t need = 0;
  {
    Scratch sc{&g->mem, s, {}};
    sc.measure = &need;
    BatchStage io;
    const int was = set_autotune(1);
    e = enqueue_batch(g->hs, d_fields, s, sc, L, io, false);
    set_autotune(was);
    if (e) return e;
    CUDA_TRY(cudaStreamSynchronize(s));
    e = finish_batch(g->hs, L, io);
    if (e) return e;
    g->io.cap_sd = io.used_sd;
    g->io.cap_items = std::max<size_t>(io.used_items, 1);
  }
  // 2. one scratch arena and pinned staging that live as long as the graph
  g->arena_bytes = need + 256;
  g->arena = g->mem.alloc(g->arena_bytes, s);
  if (!g->arena) return fail(PCR_ERR_OOM, "graph scratch arena allocation failed");
  const size_t b_init = sizeof(FieldStats) * n, b_sd = sizeof(StreamD) * g->io.cap_sd,
               b_it = sizeof(WorkItem) * g->io.cap_items, b_st = sizeof(FieldStats) * n,
               b_vm = 8 * std::max<size_t>(L.nv, 1), b_pr = 8 * std::max<size_t>(L.npairs, 1),
               b_nz = 4 * std::max<size_t>(L.nnz, 1);
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  const size_t total = al(b_init) + al(b_sd) + al(b_it) + al(b_st) + al(b_vm) + al(b_pr) + al(b_nz);
  CUDA_TRY(cudaMallocHost(&g->pinned, total));
  char* p = (char*)g->pinned;
  g->io.pinned = true;
  g->io.st_init = (FieldStats*)p;
  p += al(b_init);
  g->io.sd = (StreamD*)p;
  p += al(b_sd);
  g->io.items = (WorkItem*)p;
  p += al(b_it);
  g->io.st = (FieldStats*)p;
  p += al(b_st);
  g->io.vm = (unsigned long long*)p;
  p += al(b_vm);
  g->io.pairs = (uint64_t*)p;
  p += al(b_pr);
  g->io.nz = (uint32_t*)p;
  // 3. capture the whole batch on a stream of its own (tracing off while capturing)
  CUDA_TRY(cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking));
  e = lane_create(g->lane);
  if (e) return e;
  CUDA_TRY(cudaStreamSynchronize(s));
  const bool prof = g_prof_on;
  g_prof_on = false;
  const long long k0 = launch_count();
  CUDA_TRY(cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
  {
    Scratch sc{&g->mem, g->cap, {}};
    sc.bump = (char*)(((uintptr_t)g->arena + 255) & ~uintptr_t(255));
    sc.cap = need;
    e = enqueue_batch(g->hs, d_fields, g->cap, sc, L, g->io, true, &g->lane);
  }
  cudaGraph_t graph = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(g->cap, &graph);
  g_prof_on = prof;
  g->graph = graph;
  if (e) return e;
  if (ce != cudaSuccess) return fail(PCR_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
  g->kernels = launch_count() - k0;
  add_launches(-g->kernels);   // recorded, not launched
  CUDA_TRY(cudaGraphGetNodes(g->graph, nullptr, &g->nodes));
  CUDA_TRY(cudaGraphInstantiate(&g->exec, g->graph, 0));
  *out = g.release();
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" pcr_status pcr_refactor_graph_run(pcr_refactor_graph* g, void* cuda_stream) try {
  if (!g) return fail(PCR_ERR_INVALID_ARG, "null graph");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  for (cudaEvent_t& e : g->ev)
    if (!e) CUDA_TRY(cudaEventCreate(&e));
  CUDA_TRY(cudaEventRecord(g->ev[0], s));
  CUDA_TRY(cudaGraphLaunch(g->exec, s));
  CUDA_TRY(cudaEventRecord(g->ev[1], s));
  add_launches(g->kernels);
  CUDA_TRY(cudaStreamSynchronize(s));
  float ms = 0.0f;
  CUDA_TRY(cudaEventElapsedTime(&ms, g->ev[0], g->ev[1]));
  g->gpu_ms = ms;
  const auto t0 = std::chrono::steady_clock::now();
  const pcr_status e = finish_batch(g->hs, *g->layout, g->io);
  g->host_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return e;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" pcr_status pcr_refactor_graph_times(const pcr_refactor_graph* g, double* gpu_ms, double* host_ms) try {
  if (!g) return fail(PCR_ERR_INVALID_ARG, "null graph");
  if (gpu_ms) *gpu_ms = g->gpu_ms;
  if (host_ms) *host_ms = g->host_ms;
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" pcr_status pcr_refactor_graph_handle(const pcr_refactor_graph* g, int k, const pcr_handle** out) try {
  if (!g || !out || k < 0 || k >= (int)g->hs.size()) return fail(PCR_ERR_INVALID_ARG, "bad graph or index");
  *out = g->hs[k];
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" pcr_status pcr_refactor_graph_info(const pcr_refactor_graph* g, int64_t* nodes, int64_t* kernels,
                                              int64_t* arena_bytes) try {
  if (!g) return fail(PCR_ERR_INVALID_ARG, "null graph");
  if (nodes) *nodes = (int64_t)g->nodes;
  if (kernels) *kernels = g->kernels;
  if (arena_bytes) *arena_bytes = (int64_t)g->arena_bytes;
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" void pcr_refactor_graph_free(pcr_refactor_graph* g) { delete g; }

extern "C" pcr_status pcr_device_status(int* timeouts, int clear) try {
  if (!timeouts) return fail(PCR_ERR_INVALID_ARG, "null argument");
  const int v = read_device_timeouts(clear != 0);
  if (v < 0) return fail(PCR_ERR_CUDA, "reading the device status failed");
  *timeouts = v;
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" pcr_status pcr_autotune_enable(int enable) try {
  set_autotune(enable);
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" pcr_status pcr_autotune_set(const int64_t* key, int choice) try {
  if (!key) return fail(PCR_ERR_INVALID_ARG, "null key");
  if (!autotune_pin(key, choice)) return fail(PCR_ERR_INVALID_ARG, "unknown key field or schedule choice");
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" pcr_status pcr_autotune_read(int max_entries, int64_t* keys, int* choice, double* ms, int* n_out,
                                        int reset) try {
  if (!n_out) return fail(PCR_ERR_INVALID_ARG, "null argument");
  *n_out = autotune_entries(max_entries, keys, choice, ms);
  if (reset) clear_autotune();
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" pcr_status pcr_refactor(const void* d_field, int ndim, const int64_t* dims, int dtype,
                                   const pcr_scheme* scheme, const pcr_allocator* alloc, void* cuda_stream,
                                   pcr_handle** out) try {
  if (!out) return fail(PCR_ERR_INVALID_ARG, "null output");
  const void* f[1] = {d_field};
  const int nd[1] = {ndim};
  const int64_t* dm[1] = {dims};
  const int dt[1] = {dtype};
  return pcr_refactor_batch(1, f, nd, dm, dt, scheme, alloc, cuda_stream, out);
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

// ---------------------------------------------------------------------------
// plan
// ---------------------------------------------------------------------------
static pcr_status plan_impl(const pcr_handle* h, const pcr_target* t, const std::vector<int>* have,
                            pcr_retrieval_plan* out, int64_t search_nodes = -1, SearchStats* ss = nullptr) {
  if (!(t->value >= 0) || !std::isfinite(t->value)) return fail(PCR_ERR_INVALID_ARG, "bad target value");
  std::vector<int> b;
  double bound = 0;
  bool ok;
  const double R = h->xmax - h->xmin;
  std::memset(out, 0, sizeof(*out));
  if (t->kind == PCR_TARGET_ABS || t->kind == PCR_TARGET_REL) {
    const double tau = t->value * (t->kind == PCR_TARGET_REL ? R : 1.0);
    ok = search_nodes >= 0 ? search_plan(h, tau, true, have, search_nodes, b, bound, *ss)
                           : greedy(h, tau, true, b, bound, have);
    out->psnr_bound = 0;
  } else if (t->kind == PCR_TARGET_PSNR) {
    const double ratio = R / std::pow(10.0, t->value / 20.0);
    const double sse_max = (double)h->meta.n * ratio * ratio;
    ok = search_nodes >= 0 ? search_plan(h, sse_max, false, have, search_nodes, b, bound, *ss)
                           : greedy(h, sse_max, false, b, bound, have);
    const double rmse = std::sqrt(bound / (double)h->meta.n);
    out->psnr_bound = rmse > 0 ? 20.0 * std::log10(R / rmse) : std::numeric_limits<double>::infinity();
  } else {
    return fail(PCR_ERR_INVALID_ARG, "bad target kind");
  }
  out->nstreams = (int)b.size();
  uint64_t bytes = 0;
  for (size_t i = 0; i < b.size(); i++) {
    out->planes[i] = b[i];
    bytes += h->tabs[i].bytes[b[i]];
  }
  out->bytes = bytes;
  out->bound = bound;
  out->satisfied = ok ? 1 : 0;
  if (!ok) return fail(PCR_ERR_UNSATISFIABLE, "target tighter than the all-planes bound");
  return PCR_OK;
}

// ---------------------------------------------------------------------------
// one target for several blocks of a field (axis-0 slabs refactored one by
// one, Sec. VII): error bounds per block at the field's absolute tolerance;
// PSNR with one squared-error budget spent by one greedy over every block's
// units (the largest decrease of its own block's L2 bound per byte, ties to
// the earlier block then unit; when nothing lowers a bound, the largest
// decrease of the stream's own squared-error entry times the unit's weight
// per byte); one block gives the block's own plan
// ---------------------------------------------------------------------------
namespace {
struct BlockPlan {
  const pcr_handle* h;
  std::vector<int> b;
  std::vector<double> err, sq;
  std::unique_ptr<BoundEval> be;
  const std::vector<Unit>* units;
  std::vector<size_t> pos;
  std::vector<int> unit_level;
  double E = 0;
  // each unit's next-step bound and own squared error, valid until this
  // block takes a step (a step elsewhere leaves them unchanged)
  std::vector<double> cne, cown1;
  bool cvalid = false;
};
}  // namespace

static bool greedy_l2_global(std::vector<BlockPlan>& bp, double budget, double& total) {
  for (BlockPlan& p : bp) {
    const int n = (int)p.h->tabs.size();
    p.b.assign(n, 0);
    p.err.resize(n);
    p.sq.resize(n);
    for (int i = 0; i < n; i++) {
      p.err[i] = p.h->tabs[i].maxerr[0];
      p.sq[i] = p.h->tabs[i].sq[0];
    }
    p.be.reset(new BoundEval(p.h->comp, true));
    p.units = &cached_units(p.h, false);
    p.pos.assign(p.units->size(), 0);
    p.unit_level.resize(p.units->size());
    for (size_t ui = 0; ui < p.units->size(); ui++) p.unit_level[ui] = p.h->geo[(*p.units)[ui].ids[0]].level;
    p.E = p.be->eval_from(p.h->L - 1, p.err, p.sq, true);
  }
  total = 0.0;
  for (BlockPlan& p : bp) total += p.E;
  std::vector<std::pair<int, int>> saved;
  auto apply = [&](BlockPlan& p, const Step& st) {
    saved.clear();
    for (auto& up : st.upd) {
      saved.push_back({up.first, p.b[up.first]});
      p.b[up.first] = up.second;
      p.err[up.first] = p.h->tabs[up.first].maxerr[up.second];
      p.sq[up.first] = p.h->tabs[up.first].sq[up.second];
    }
  };
  auto undo = [&](BlockPlan& p) {
    for (auto it = saved.rbegin(); it != saved.rend(); ++it) {
      p.b[it->first] = it->second;
      p.err[it->first] = p.h->tabs[it->first].maxerr[it->second];
      p.sq[it->first] = p.h->tabs[it->first].sq[it->second];
    }
  };
  const double inf = std::numeric_limits<double>::infinity();
  std::vector<int> bst, bunit;
  std::vector<double> berr, bsq, bval;
  while (total > budget) {
    bool have_best = false, have_fb = false;
    double best_r = 0, fb_r = 0, best_e = 0, fb_e = 0;
    size_t best_k = 0, best_u = 0, fb_k = 0, fb_u = 0;
    for (size_t k = 0; k < bp.size(); k++) {
      BlockPlan& p = bp[k];
      if (!p.cvalid) {   // this block's candidates: batched where they change one stream
        const size_t nu = p.units->size();
        p.cne.assign(nu, 0.0);
        p.cown1.assign(nu, 0.0);
        bst.clear();
        bunit.clear();
        berr.clear();
        bsq.clear();
        for (size_t ui = 0; ui < nu; ui++) {
          const Unit& u = (*p.units)[ui];
          if (p.pos[ui] >= u.steps.size()) continue;
          const Step& st = u.steps[p.pos[ui]];
          const int i0 = u.ids[0];
          if (u.ids.size() == 1 && st.upd.size() == 1 && st.upd[0].first == i0 && p.be->batch_ok(i0)) {
            bst.push_back(i0);
            bunit.push_back((int)ui);
            berr.push_back(p.h->tabs[i0].maxerr[st.upd[0].second]);
            bsq.push_back(p.h->tabs[i0].sq[st.upd[0].second]);
            p.cown1[ui] = bsq.back();
            continue;
          }
          apply(p, st);
          p.cne[ui] = p.be->eval_from(p.unit_level[ui], p.err, p.sq, false, u.ids.size() == 1 ? i0 : -1);
          p.cown1[ui] = p.sq[i0];
          undo(p);
        }
        if (!bst.empty()) {
          bval.resize(bst.size());
          p.be->eval_batch((int)bst.size(), bst.data(), berr.data(), bsq.data(), p.err, p.sq, bval.data());
          for (size_t q = 0; q < bst.size(); q++) p.cne[bunit[q]] = bval[q];
        }
        p.cvalid = true;
      }
      for (size_t ui = 0; ui < p.units->size(); ui++) {
        const Unit& u = (*p.units)[ui];
        if (p.pos[ui] >= u.steps.size()) continue;
        const Step& st = u.steps[p.pos[ui]];
        const int i0 = u.ids[0];
        const double own0 = p.sq[i0];
        const double ne = p.cne[ui];
        const double own1 = p.cown1[ui];
        const double gain = p.E - ne;
        const double ratio = st.db == 0 ? inf : gain / (double)st.db;
        if (gain > 0 || st.db == 0) {
          if (!have_best || ratio > best_r) {
            have_best = true;
            best_r = ratio;
            best_k = k;
            best_u = ui;
            best_e = ne;
          }
        }
        const double own = (own0 - own1) * u.weight;
        const double fr = st.db == 0 ? inf : own / (double)st.db;
        if (!have_fb || fr > fb_r) {
          have_fb = true;
          fb_r = fr;
          fb_k = k;
          fb_u = ui;
          fb_e = ne;
        }
      }
    }
    if (!have_best) {
      if (!have_fb) return false;
      best_k = fb_k;
      best_u = fb_u;
      best_e = fb_e;
    }
    BlockPlan& p = bp[best_k];
    apply(p, (*p.units)[best_u].steps[p.pos[best_u]]);
    p.be->eval_from(p.unit_level[best_u], p.err, p.sq, true);   // refresh the kept partial results
    p.pos[best_u]++;
    p.cvalid = false;
    total = total - p.E + best_e;
    p.E = best_e;
  }
  return true;
}

extern "C" pcr_status pcr_plan_global(int n, const pcr_handle* const* hs, const pcr_target* t,
                                      pcr_retrieval_plan* plans, double* bound, int* satisfied) try {
  if (n <= 0 || !hs || !t || !plans) return fail(PCR_ERR_INVALID_ARG, "null argument");
  for (int k = 0; k < n; k++)
    if (!hs[k]) return fail(PCR_ERR_INVALID_ARG, "null handle");
  if (!(t->value >= 0) || !std::isfinite(t->value)) return fail(PCR_ERR_INVALID_ARG, "bad target value");
  double lo = hs[0]->xmin, hi = hs[0]->xmax;
  int64_t N = 0;
  for (int k = 0; k < n; k++) {
    lo = std::min(lo, hs[k]->xmin);
    hi = std::max(hi, hs[k]->xmax);
    N += hs[k]->meta.n;
  }
  const double R = hi - lo;
  bool ok = true;
  double bnd = 0;
  if (t->kind == PCR_TARGET_ABS || t->kind == PCR_TARGET_REL) {
    const double tau = t->value * (t->kind == PCR_TARGET_REL ? R : 1.0);
    const pcr_target ta{PCR_TARGET_ABS, tau, 0, {0, 0, 0}, {0, 0, 0}};
    for (int k = 0; k < n; k++) {
      const pcr_status e = plan_impl(hs[k], &ta, nullptr, &plans[k]);
      if (e && e != PCR_ERR_UNSATISFIABLE) return e;
      ok = ok && plans[k].satisfied;
      bnd = k ? std::max(bnd, plans[k].bound) : plans[k].bound;
    }
  } else if (t->kind == PCR_TARGET_PSNR) {
    const double ratio = R / std::pow(10.0, t->value / 20.0);
    const double budget = (double)N * ratio * ratio;
    std::vector<BlockPlan> bp(n);
    for (int k = 0; k < n; k++) bp[k].h = hs[k];
    ok = greedy_l2_global(bp, budget, bnd);
    for (int k = 0; k < n; k++) {
      pcr_retrieval_plan& o = plans[k];
      std::memset(&o, 0, sizeof(o));
      o.nstreams = (int)bp[k].b.size();
      uint64_t bytes = 0;
      for (int i = 0; i < o.nstreams; i++) {
        o.planes[i] = bp[k].b[i];
        bytes += hs[k]->tabs[i].bytes[bp[k].b[i]];
      }
      o.bytes = bytes;
      o.bound = bp[k].E;
      o.satisfied = ok ? 1 : 0;
    }
  } else {
    return fail(PCR_ERR_INVALID_ARG, "bad target kind");
  }
  if (bound) *bound = bnd;
  if (satisfied) *satisfied = ok ? 1 : 0;
  if (!ok) return fail(PCR_ERR_UNSATISFIABLE, "target tighter than the all-planes bound of some block");
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" pcr_status pcr_plan(const pcr_handle* h, const pcr_target* t, pcr_retrieval_plan* out) try {
  if (!h || !t || !out) return fail(PCR_ERR_INVALID_ARG, "null argument");
  return plan_impl(h, t, nullptr, out);
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" pcr_status pcr_plan_more(const pcr_handle* h, const pcr_target* t, const pcr_retrieval_plan* have,
                                    pcr_retrieval_plan* out) try {
  if (!h || !t || !have || !out) return fail(PCR_ERR_INVALID_ARG, "null argument");
  const int ns = (int)h->tabs.size();
  if (have->nstreams != ns) return fail(PCR_ERR_INVALID_ARG, "plan does not match the handle");
  std::vector<int> hv(ns);
  for (int i = 0; i < ns; i++) {
    if (have->planes[i] < 0 || have->planes[i] > h->B) return fail(PCR_ERR_INVALID_ARG, "plan plane count out of range");
    hv[i] = have->planes[i];
  }
  return plan_impl(h, t, &hv, out);
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" pcr_status pcr_plan_search(const pcr_handle* h, const pcr_target* t, const pcr_retrieval_plan* have,
                                      int64_t max_nodes, pcr_retrieval_plan* out, pcr_search_info* info) try {
  if (!h || !t || !out) return fail(PCR_ERR_INVALID_ARG, "null argument");
  if (max_nodes < 0) return fail(PCR_ERR_INVALID_ARG, "max_nodes must be >= 0");
  const int ns = (int)h->tabs.size();
  std::vector<int> hv;
  if (have) {
    if (have->nstreams != ns) return fail(PCR_ERR_INVALID_ARG, "plan does not match the handle");
    hv.resize(ns);
    for (int i = 0; i < ns; i++) {
      if (have->planes[i] < 0 || have->planes[i] > h->B)
        return fail(PCR_ERR_INVALID_ARG, "plan plane count out of range");
      hv[i] = have->planes[i];
    }
  }
  SearchStats ss;
  const auto t0 = std::chrono::steady_clock::now();
  const pcr_status st = plan_impl(h, t, have ? &hv : nullptr, out, max_nodes, &ss);
  if (info) {
    info->expanded = ss.expanded;
    info->optimal = ss.optimal;
    info->greedy_bytes = ss.greedy_bytes;
    info->plan_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return st;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

// ---------------------------------------------------------------------------
// retrieve
// ---------------------------------------------------------------------------
static pcr_status enqueue_retrieve_one(const pcr_handle* h, const pcr_retrieval_plan* p, void* d_out, cudaStream_t s,
                                       Scratch& sc, std::vector<StreamD>& sds, std::vector<int>& stage_kind) {
  const int ns = (int)h->geo.size();
  if (!p || p->nstreams != ns) return fail(PCR_ERR_INVALID_ARG, "plan does not match the handle");
  for (int i = 0; i < ns; i++)
    if (p->planes[i] < 0 || p->planes[i] > h->B) return fail(PCR_ERR_INVALID_ARG, "plan plane count out of range");
  const size_t w = vsize(h->vk);
  size_t fix_elems = 0, flt_elems = 0;
  std::vector<size_t> soff(ns);
  for (int i = 0; i < ns; i++) {
    if (h->geo[i].is_fix) {
      soff[i] = fix_elems;
      fix_elems += h->geo[i].n_pad();
    } else {
      soff[i] = flt_elems;
      flt_elems += h->geo[i].n_pad();
    }
  }
  int64_t* st_fix = (int64_t*)sc.get(fix_elems * 8);
  char* st_flt = (char*)sc.get(flt_elems * w);
  if (!st_fix || !st_flt) return fail(PCR_ERR_OOM, "staging allocation failed");
  sds.resize(ns);
  stage_kind.resize(ns);
  for (int i = 0; i < ns; i++) {
    sds[i] = stream_desc(h, i);
    sds[i].b = p->planes[i];
    sds[i].stage = h->geo[i].is_fix ? (void*)(st_fix + soff[i]) : (void*)(st_flt + soff[i] * w);
    stage_kind[i] = h->geo[i].is_fix ? VK_FIX : h->vk;
  }
  return PCR_OK;
}

// Reconstruction up to level 0 (Alg. 2): the level-0 recomposition on `s`
// (after the float decode there), the fixed-point coarse levels on `sf`
// (after the fixed-point decode there); `l0` receives the level-0 pass,
// which needs both.
struct ReconL0 {
  bool on = false;
  TileArgs a{};
};

static pcr_status enqueue_reconstruct_coarse(const pcr_handle* h, const std::vector<StreamD>& sds, void* d_out,
                                             cudaStream_t s, cudaStream_t sf, Scratch& sc, ReconL0& l0) {
  const FieldD f = field_desc(h);
  const size_t w = vsize(h->vk);
  l0.on = false;
  if (h->L == 1) {
    Prof pf("copy_raw", s);
    launch_copy_raw(h->vk, f, to_latd(h->geo[0].lats[0], 0), sds[0].stage, d_out, s);
    return PCR_OK;
  }
  // level-0 recomposition (Alg. 2)
  std::vector<void*> comp(4, nullptr);
  if (h->decomp >= 0) {
    for (int r = 1; r <= f.d; r++) {
      const Lat R = region_lat(h->n3, 0, h->order, r);
      comp[r] = sc.get((size_t)R.n_real() * w);
      if (!comp[r]) return fail(PCR_ERR_OOM, "staging allocation failed");
      DecompArgs da{};
      decomp_subs(h, r, sds, da);
      da.retrieve = 1;
      da.comp = comp[r];
      Prof pf("recompose", s);
      launch_tile_decomp(h->vk, da, s);
    }
  }
  // coarse levels in fixed point: raw coarsest, then L-2 .. 1
  int64_t* xc = (int64_t*)sc.get((size_t)f.nc[0] * f.nc[1] * f.nc[2] * 8);
  if (!xc) return fail(PCR_ERR_OOM, "staging allocation failed");
  {
    Prof pf("recon_coarsest", sf);
    launch_recon_fixed(f, h->L - 1, 1, to_latd(h->geo[0].lats[0], 0), (const int64_t*)sds[0].stage, xc, sf);
  }
  for (int level = h->L - 2; level >= 1; level--) {
    TileArgs a = level_args(h, level, 1, xc, xc);
    level_regions(h, level, sds, a);
    Prof pf("recon_fixed_levels", sf);
    launch_tile_interp(VK_FIX, a, sf);
  }
  // level 0, which takes the coarse points from the fixed-point grid: the
  // marching kernel reads them there, the tile kernels have them written
  // into the output first
  TileArgs a = level_args(h, 0, 1, d_out, d_out);
  a.cfix = xc;
  a.cscale = std::ldexp(1.0, h->G - fix_bits(h->vk, h->L));
  if (h->decomp >= 0) {
    for (int r = 1; r <= f.d; r++) {
      const Lat R = region_lat(h->n3, 0, h->order, r);
      a.reg[r - 1] = tile_region(h, R, 0, R.count[2], 0, comp[r], nullptr);
    }
  } else {
    level_regions(h, 0, sds, a);
  }
  l0.on = true;
  l0.a = a;
  return PCR_OK;
}

static void enqueue_reconstruct_l0(const pcr_handle* h, const ReconL0& l0, cudaStream_t s) {
  if (!l0.on) return;
  Prof pf("recon_level0", s);
  launch_tile_interp(h->vk, l0.a, s);
}

// `fork`: the fixed-point chain (decode, coarse levels, coarse output) runs
// on a second stream beside the float decode and recomposition
static pcr_status retrieve_batch_impl(int n, const pcr_handle* const* hs, const pcr_retrieval_plan* plans,
                                      void* const* d_outs, cudaStream_t s, Scratch& sc, bool fork = true) {
  for (int k = 0; k < n; k++)
    if (!hs[k]->d_block) return fail(PCR_ERR_UNSUPPORTED, "a planning-only handle holds no planes");
  std::vector<std::vector<StreamD>> sds(n);
  std::vector<StreamD> all;
  std::vector<WorkItem> items[2][2];
  // decodes (fixed point on the side stream), then the reconstruction up to
  // level 0, then, joined, every level 0
  auto run = [&](auto decode_all) -> pcr_status {
    std::unique_ptr<Fork> fk;
    if (fork) fk.reset(new Fork(s));
    if (fk) {
      pcr_status e = fk->fork();
      if (e) return e;
    }
    const cudaStream_t sf = fk ? fk->side() : s;
    pcr_status e = decode_all(sf);
    if (e) return e;
    std::vector<ReconL0> l0(n);
    for (int k = 0; k < n; k++) {
      e = enqueue_reconstruct_coarse(hs[k], sds[k], d_outs[k], s, sf, sc, l0[k]);
      if (e) return e;
    }
    if (fk) {
      e = fk->join();
      if (e) return e;
    }
    for (int k = 0; k < n; k++) enqueue_reconstruct_l0(hs[k], l0[k], s);
    CUDA_TRY(cudaGetLastError());
    return PCR_OK;
  };
  if (n == 1 && hs[0]->items_ready) {   // one handle: its kept work list
    const pcr_handle* h = hs[0];
    std::vector<int> kinds;
    pcr_status e = enqueue_retrieve_one(h, &plans[0], d_outs[0], s, sc, sds[0], kinds);
    if (e) return e;
    StreamD* d_sd = (StreamD*)sc.get(sds[0].size() * sizeof(StreamD));
    if (!d_sd) return fail(PCR_ERR_OOM, "work list allocation failed");
    CUDA_TRY(cudaMemcpyAsync(d_sd, sds[0].data(), sds[0].size() * sizeof(StreamD), cudaMemcpyHostToDevice, s));
    return run([&](cudaStream_t sf) -> pcr_status {
      size_t off = 0;
      for (int fx = 0; fx < 2; fx++) {
        if (!h->items_n[fx]) continue;
        const int vk = fx ? VK_FIX : h->vk;
        const cudaStream_t ds = fx ? sf : s;
        {
          Prof pf(fx ? "decode_fixed" : "decode_float", ds);
          launch_decode(vk, h->w64, d_sd, h->d_items_all + off, (int)h->items_n[fx], ds);
        }
        off += h->items_n[fx];
      }
      return PCR_OK;
    });
  }
  for (int k = 0; k < n; k++) {
    std::vector<int> kinds;
    pcr_status e = enqueue_retrieve_one(hs[k], &plans[k], d_outs[k], s, sc, sds[k], kinds);
    if (e) return e;
    for (size_t i = 0; i < sds[k].size(); i++) {
      const int idx = (int)all.size();
      all.push_back(sds[k][i]);
      const int fx = sds[k][i].is_fix;
      for (int64_t g = 0; g < sds[k][i].nseg; g++) items[hs[k]->w64][fx].push_back({idx, (int)g});
    }
  }
  StreamD* d_sd = (StreamD*)sc.get(all.size() * sizeof(StreamD));
  size_t nit = 0;
  for (int a = 0; a < 2; a++)
    for (int b = 0; b < 2; b++) nit += items[a][b].size();
  WorkItem* d_items = (WorkItem*)sc.get(std::max<size_t>(nit, 1) * sizeof(WorkItem));
  if (!d_sd || !d_items) return fail(PCR_ERR_OOM, "work list allocation failed");
  CUDA_TRY(cudaMemcpyAsync(d_sd, all.data(), all.size() * sizeof(StreamD), cudaMemcpyHostToDevice, s));
  size_t off = 0;
  for (int a = 0; a < 2; a++)
    for (int b = 0; b < 2; b++) {
      if (items[a][b].empty()) continue;
      CUDA_TRY(cudaMemcpyAsync(d_items + off, items[a][b].data(), items[a][b].size() * sizeof(WorkItem),
                               cudaMemcpyHostToDevice, s));
      off += items[a][b].size();
    }
  return run([&](cudaStream_t sf) -> pcr_status {
    size_t o = 0;
    for (int a = 0; a < 2; a++)
      for (int b = 0; b < 2; b++) {
        if (items[a][b].empty()) continue;
        const int vk = b ? VK_FIX : (a ? VK_F64 : VK_F32);
        const cudaStream_t ds = b ? sf : s;
        {
          Prof pf(b ? "decode_fixed" : "decode_float", ds);
          launch_decode(vk, a, d_sd, d_items + o, (int)items[a][b].size(), ds);
        }
        o += items[a][b].size();
      }
    return PCR_OK;
  });
}

// ---------------------------------------------------------------------------
// retrieval of a box of the field
// ---------------------------------------------------------------------------
// A reconstructed point at level l depends on the coarser grid and on level
// l's decoded coefficients within 3 points of the level grid per axis (the
// cubic rules; every region pass reads one axis once), i.e. 3 * 2^l field
// points.  So with B_0 = the box and B_(l+1) = B_l grown by 3 * 2^l, level l
// is reconstructed over B_l from coefficients decoded over B_l grown by
// 3 * 2^l (level 0 with decomposition: grown further by the recomposition's
// reach, 2 sub-level lines of 4 compact points, at most 16 field points).
// Only the stream segments meeting those boxes are decoded and only the
// tiles meeting B_l are run; values the kernels produce outside B_l (tile
// rounding) may use undecoded inputs but are never read by a point inside.
namespace {
struct FBox {
  int64_t lo[3], hi[3];   // field coordinates, [lo, hi)
};
int64_t floordiv(int64_t a, int64_t b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }
int64_t ceildiv(int64_t a, int64_t b) { return -floordiv(-a, b); }

FBox grow(const FBox& b, int64_t r, const int64_t* n3) {
  FBox o = b;
  for (int k = 0; k < 3; k++)
    if (n3[k] > 1) {
      o.lo[k] = std::max<int64_t>(0, b.lo[k] - r);
      o.hi[k] = std::min<int64_t>(n3[k], b.hi[k] + r);
    }
  return o;
}

// lattice index ranges [k0, k1) of the lattice points inside box b
bool lat_range(const Lat& L, const FBox& b, int64_t* k0, int64_t* k1) {
  for (int a = 0; a < 3; a++) {
    k0[a] = std::max<int64_t>(0, ceildiv(b.lo[a] - L.start[a], L.step[a]));
    k1[a] = std::min<int64_t>(L.count[a], floordiv(b.hi[a] - 1 - L.start[a], L.step[a]) + 1);
    if (k1[a] <= k0[a]) return false;
  }
  return true;
}
}  // namespace

// decode only the segments of stream i that hold lattice points of box b
static void mark_segments(const SGeo& g, const FBox& b, std::vector<char>& mark) {
  const int64_t nseg = (g.n_pad() + kSegElems - 1) / kSegElems;
  mark.assign(nseg, 0);
  int64_t base = 0;
  for (const Lat& L : g.lats) {
    int64_t k0[3], k1[3];
    if (lat_range(L, b, k0, k1)) {
      const int64_t rp = L.row_pad();
      for (int64_t a = k0[0]; a < k1[0]; a++)
        for (int64_t c = k0[1]; c < k1[1]; c++) {
          const int64_t row = base + (a * L.count[1] + c) * rp;
          for (int64_t sg = (row + k0[2]) / kSegElems; sg <= (row + k1[2] - 1) / kSegElems; sg++) mark[sg] = 1;
        }
    }
    base += L.n_pad();
  }
}

// level-grid box of a field box at level l (points q with q 2^l in [lo, hi))
static void level_box(const pcr_handle* h, const FBox& b, int level, int64_t* lo, int64_t* hi) {
  for (int k = 0; k < 3; k++) {
    if (h->n3[k] > 1) {
      lo[k] = ceildiv(b.lo[k], int64_t(1) << level);
      hi[k] = ceildiv(b.hi[k], int64_t(1) << level);
    } else {
      lo[k] = 0;
      hi[k] = 1;
    }
  }
}

static pcr_status enqueue_reconstruct_box(const pcr_handle* h, const std::vector<StreamD>& sds, void* d_full,
                                          const std::vector<FBox>& B, cudaStream_t s, Scratch& sc) {
  const FieldD f = field_desc(h);
  const size_t w = vsize(h->vk);
  if (h->L == 1) {
    Prof pf("copy_raw", s);
    launch_copy_raw(h->vk, f, to_latd(h->geo[0].lats[0], 0), sds[0].stage, d_full, s);
    return PCR_OK;
  }
  std::vector<void*> comp(4, nullptr);
  if (h->decomp >= 0) {
    const FBox rb = grow(B[0], 3, h->n3);   // level-0 coefficients the level-0 pass reads
    for (int r = 1; r <= f.d; r++) {
      const Lat R = region_lat(h->n3, 0, h->order, r);
      comp[r] = sc.get((size_t)R.n_real() * w);
      if (!comp[r]) return fail(PCR_ERR_OOM, "staging allocation failed");
      DecompArgs da{};
      decomp_subs(h, r, sds, da);
      da.retrieve = 1;
      da.comp = comp[r];
      int64_t k0[3], k1[3];
      if (!lat_range(R, rb, k0, k1)) continue;
      for (int k = 0; k < 3; k++) {
        da.blo[k] = k0[k];
        da.bhi[k] = k1[k];
      }
      Prof pf("recompose", s);
      launch_tile_decomp(h->vk, da, s);
    }
  }
  int64_t* xc = (int64_t*)sc.get((size_t)f.nc[0] * f.nc[1] * f.nc[2] * 8);
  if (!xc) return fail(PCR_ERR_OOM, "staging allocation failed");
  {
    Prof pf("recon_coarsest", s);
    launch_recon_fixed(f, h->L - 1, 1, to_latd(h->geo[0].lats[0], 0), (const int64_t*)sds[0].stage, xc, s);
  }
  for (int level = h->L - 2; level >= 1; level--) {
    TileArgs a = level_args(h, level, 1, xc, xc);
    level_regions(h, level, sds, a);
    level_box(h, B[level], level, a.blo, a.bhi);
    if (a.bhi[0] <= a.blo[0] || a.bhi[1] <= a.blo[1] || a.bhi[2] <= a.blo[2]) continue;
    Prof pf("recon_fixed_levels", s);
    launch_tile_interp(VK_FIX, a, s);
  }
  {
    int64_t lo[3], hi[3];
    level_box(h, B[1], 1, lo, hi);   // the 2-grid points level 0 reads
    Box3 cb;
    for (int k = 0; k < 3; k++) {
      cb.lo[k] = lo[k];
      cb.cnt[k] = std::max<int64_t>(0, hi[k] - lo[k]);
    }
    Prof pf("coarse_out", s);
    launch_coarse_out(h->vk, f, xc, std::ldexp(1.0, h->G - fix_bits(h->vk, h->L)), d_full, s, &cb);
  }
  TileArgs a = level_args(h, 0, 1, d_full, d_full);
  if (h->decomp >= 0) {
    for (int r = 1; r <= f.d; r++) {
      const Lat R = region_lat(h->n3, 0, h->order, r);
      a.reg[r - 1] = tile_region(h, R, 0, R.count[2], 0, comp[r], nullptr);
    }
  } else {
    level_regions(h, 0, sds, a);
  }
  level_box(h, B[0], 0, a.blo, a.bhi);
  Prof pf("recon_level0", s);
  launch_tile_interp(h->vk, a, s);
  return PCR_OK;
}

extern "C" pcr_status pcr_retrieve_box(const pcr_handle* h, const pcr_retrieval_plan* plan, const int64_t* lo,
                                       const int64_t* hi, void* d_out, void* cuda_stream) try {
  if (!h || !plan || !lo || !hi || !d_out) return fail(PCR_ERR_INVALID_ARG, "null argument");
  if (!h->d_block) return fail(PCR_ERR_UNSUPPORTED, "a planning-only handle holds no planes");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // user axes -> the internal 3-D view (2-D fields are 1 x n0 x n1)
  FBox B0{{0, 0, 0}, {1, 1, 1}};
  const int off = 3 - h->ndim;
  for (int k = 0; k < h->ndim; k++) {
    if (lo[k] < 0 || hi[k] > h->dims[k] || lo[k] >= hi[k]) return fail(PCR_ERR_INVALID_ARG, "box outside the field");
    B0.lo[off + k] = lo[k];
    B0.hi[off + k] = hi[k];
  }
  Mem mem = h->mem;
  Scratch sc{&mem, s, {}};
  std::vector<StreamD> sds;
  std::vector<int> kinds;
  pcr_status e = enqueue_retrieve_one(h, plan, d_out, s, sc, sds, kinds);
  if (e) return e;
  // level boxes and the decode work list
  std::vector<FBox> B(h->L);
  B[0] = B0;
  for (int l = 0; l + 1 < h->L; l++) B[l + 1] = grow(B[l], int64_t(3) << l, h->n3);
  std::vector<WorkItem> items[2];
  std::vector<char> mark;
  for (int i = 0; i < (int)h->geo.size(); i++) {
    const SGeo& g = h->geo[i];
    const int l = g.level;
    FBox need;
    if (l == h->L - 1) {
      need = FBox{{0, 0, 0}, {h->n3[0], h->n3[1], h->n3[2]}};
    } else {
      const int64_t r = (int64_t(3) << l) + (l == 0 && h->decomp >= 0 ? 16 : 0);
      need = grow(B[l], r, h->n3);
    }
    mark_segments(g, need, mark);
    for (int64_t sg = 0; sg < (int64_t)mark.size(); sg++)
      if (mark[sg]) items[g.is_fix].push_back({i, (int)sg});
  }
  StreamD* d_sd = (StreamD*)sc.get(sds.size() * sizeof(StreamD));
  WorkItem* d_items = (WorkItem*)sc.get(std::max<size_t>(items[0].size() + items[1].size(), 1) * sizeof(WorkItem));
  void* d_full = sc.get((size_t)h->n3[0] * h->n3[1] * h->n3[2] * vsize(h->vk));
  if (!d_sd || !d_items || !d_full) return fail(PCR_ERR_OOM, "box retrieval allocation failed");
  CUDA_TRY(cudaMemcpyAsync(d_sd, sds.data(), sds.size() * sizeof(StreamD), cudaMemcpyHostToDevice, s));
  size_t o = 0;
  for (int fx = 0; fx < 2; fx++) {
    if (items[fx].empty()) continue;
    CUDA_TRY(cudaMemcpyAsync(d_items + o, items[fx].data(), items[fx].size() * sizeof(WorkItem),
                             cudaMemcpyHostToDevice, s));
    {
      Prof pf(fx ? "decode_fixed" : "decode_float", s);
      launch_decode(fx ? VK_FIX : h->vk, h->w64, d_sd, d_items + o, (int)items[fx].size(), s);
    }
    o += items[fx].size();
  }
  e = enqueue_reconstruct_box(h, sds, d_full, B, s, sc);
  if (e) return e;
  Box3 ob;
  for (int k = 0; k < 3; k++) {
    ob.lo[k] = B0.lo[k];
    ob.cnt[k] = B0.hi[k] - B0.lo[k];
  }
  {
    Prof pf("copy_box", s);
    launch_copy_box(h->vk, field_desc(h), d_full, d_out, ob, s);
  }
  CUDA_TRY(cudaGetLastError());
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

static size_t retrieve_scratch_bytes(const pcr_handle* h);

extern "C" pcr_status pcr_retrieve_batch_plan(int n, const pcr_handle* const* hs, const pcr_retrieval_plan* plans,
                                              void* const* d_outs, void* cuda_stream) try {
  if (n <= 0 || !hs || !plans || !d_outs) return fail(PCR_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  for (int k = 0; k < n; k++)
    if (!hs[k] || !d_outs[k]) return fail(PCR_ERR_INVALID_ARG, "null handle or output");
  Mem mem = hs[0]->mem;
  size_t need = 256 * 4;
  for (int k = 0; k < n; k++) need += retrieve_scratch_bytes(hs[k]);
  Scratch sc{&mem, s, {}};
  ScratchBlock blk(&mem, s, need, sc);
  if (!blk.p) return fail(PCR_ERR_OOM, "scratch allocation failed");
  return retrieve_batch_impl(n, hs, plans, d_outs, s, sc);
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

// bytes of temporary device memory one retrieval of `h` uses (upper bound,
// including 256-byte alignment of every piece)
static size_t retrieve_scratch_bytes(const pcr_handle* h) {
  const size_t w = vsize(h->vk);
  auto al = [](size_t b) { return (b + 255) & ~size_t(255); };
  size_t fix = 0, flt = 0, items = 0;
  for (auto& g : h->geo) {
    (g.is_fix ? fix : flt) += g.n_pad();
    items += (g.n_pad() + kSegElems - 1) / kSegElems;
  }
  size_t t = al(fix * 8) + al(flt * w) + al(h->geo.size() * sizeof(StreamD)) + al(std::max<size_t>(items, 1) * sizeof(WorkItem));
  if (h->L >= 2) {
    size_t nc = 1;
    for (int a = 0; a < 3; a++) nc *= h->n3[a] > 1 ? (h->n3[a] - 1) / 2 + 1 : 1;
    t += al(nc * 8);
  }
  if (h->decomp >= 0)
    for (int r = 1; r <= (int)h->order.size(); r++) {
      const Lat R = region_lat(h->n3, 0, h->order, r);
      t += al((size_t)(R.count[0] * R.count[1] * comp_pitch(h, R)) * w);
    }
  return t + 256;
}

extern "C" pcr_status pcr_retrieve_scratch_bytes(const pcr_handle* h, size_t* bytes) try {
  if (!h || !bytes) return fail(PCR_ERR_INVALID_ARG, "null argument");
  *bytes = retrieve_scratch_bytes(h);
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

// Retrieval whose temporary buffers live in the library's fixed device array
// (pcr_static.cu); see pcr_retrieve_static in include/pcr.h.
extern "C" pcr_status pcr_retrieve_static(const pcr_handle* h, const pcr_retrieval_plan* plan, void* d_out,
                                          void* cuda_stream) try {
  if (!h || !plan || !d_out) return fail(PCR_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  // the scratch array is per device: it must be the one holding the handle
  int dev = -1;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev != h->device)
    return fail(PCR_ERR_INVALID_ARG, "current device " + std::to_string(dev) + " is not the handle's device " +
                                         std::to_string(h->device));
  // the call uploads its stream descriptors (and, for handles without a kept
  // work list, the work list) from host memory that does not outlive it
  cudaStreamCaptureStatus cap_st = cudaStreamCaptureStatusNone;
  CUDA_TRY(cudaStreamIsCapturing(s, &cap_st));
  if (cap_st != cudaStreamCaptureStatusNone)
    return fail(PCR_ERR_UNSUPPORTED, "pcr_retrieve_static does not accept a stream that is being captured");
  size_t cap = 0;
  std::string why;
  char* base = (char*)static_scratch(&cap, &why);
  if (!base) return fail(PCR_ERR_CUDA, "static scratch set-up failed: " + why);
  const size_t need = retrieve_scratch_bytes(h);
  if (need > cap)
    return fail(PCR_ERR_UNSUPPORTED, "retrieval needs " + std::to_string(need) +
                                         " bytes of scratch; the static array holds " + std::to_string(cap));
  Mem mem = h->mem;
  Scratch sc{&mem, s, {}};
  sc.bump = base;
  sc.cap = cap;
  return retrieve_batch_impl(1, &h, plan, &d_out, s, sc, false);
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" pcr_status pcr_retrieve_plan(const pcr_handle* h, const pcr_retrieval_plan* plan, void* d_out,
                                        void* cuda_stream) try {
  if (!h || !plan || !d_out) return fail(PCR_ERR_INVALID_ARG, "null argument");
  return pcr_retrieve_batch_plan(1, &h, plan, &d_out, cuda_stream);
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

// ---------------------------------------------------------------------------
// one-call retrieval: plan + retrieve (Sec. III-A problem statement)
// ---------------------------------------------------------------------------
namespace {
double ms_since(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

int64_t out_points(const pcr_handle* h, const pcr_target* t) {
  int64_t n = 1;
  for (int k = 0; k < h->ndim; k++) n *= t->has_box ? (t->hi[k] - t->lo[k]) : h->dims[k];
  return n;
}

void fill_info(const pcr_handle* h, const pcr_target* t, const pcr_retrieval_plan& p, double plan_ms,
               pcr_retrieval_info* info) {
  const int want = info->want_gpu_ms;
  std::memset(info, 0, sizeof(*info));
  info->want_gpu_ms = want;
  info->nstreams = p.nstreams;
  for (int i = 0; i < p.nstreams; i++) info->planes[i] = p.planes[i];
  info->bytes = p.bytes;
  const int64_t n = out_points(h, t);
  info->bits_per_value = n > 0 ? 8.0 * (double)p.bytes / (double)n : 0.0;
  info->bound = p.bound;
  info->psnr_bound = p.psnr_bound;
  info->satisfied = p.satisfied;
  info->plan_ms = plan_ms;
  info->gpu_ms = -1.0;
}
}  // namespace

extern "C" pcr_status pcr_retrieve(const pcr_handle* h, const pcr_target* target, void* d_out, void* cuda_stream,
                                   pcr_retrieval_info* info) try {
  if (!h || !target || !d_out) return fail(PCR_ERR_INVALID_ARG, "null argument");
  if (target->has_box) {
    for (int k = 0; k < h->ndim; k++)
      if (target->lo[k] < 0 || target->hi[k] > h->dims[k] || target->lo[k] >= target->hi[k])
        return fail(PCR_ERR_INVALID_ARG, "box outside the field");
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const auto t0 = std::chrono::steady_clock::now();
  pcr_retrieval_plan p{};
  const pcr_status ps = pcr_plan(h, target, &p);
  const double plan_ms = ms_since(t0);
  if (info) fill_info(h, target, p, plan_ms, info);
  if (ps != PCR_OK) return ps;   // unsatisfiable: nothing enqueued, info filled
  const bool timed = info && info->want_gpu_ms;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  if (timed) {
    CUDA_TRY(cudaEventCreate(&ev[0]));
    CUDA_TRY(cudaEventCreate(&ev[1]));
    CUDA_TRY(cudaEventRecord(ev[0], s));
  }
  const auto t1 = std::chrono::steady_clock::now();
  const pcr_status st = target->has_box ? pcr_retrieve_box(h, &p, target->lo, target->hi, d_out, cuda_stream)
                                        : pcr_retrieve_plan(h, &p, d_out, cuda_stream);
  if (info) info->enqueue_ms = ms_since(t1);
  if (timed) {
    float ms = -1.0f;
    if (st == PCR_OK && cudaEventRecord(ev[1], s) == cudaSuccess && cudaEventSynchronize(ev[1]) == cudaSuccess)
      cudaEventElapsedTime(&ms, ev[0], ev[1]);
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    info->gpu_ms = ms;
    // the call waited for its work: a bounded device wait that gave up
    // during it is reported here
    if (st == PCR_OK && read_device_timeouts(true) > 0)
      return fail(PCR_ERR_TIMEOUT, "a device wait of the retrieval gave up");
  }
  return st;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" pcr_status pcr_retrieve_batch(int n, const pcr_handle* const* hs, const pcr_target* targets,
                                         void* const* d_outs, void* cuda_stream, pcr_retrieval_info* infos) try {
  if (n <= 0 || !hs || !targets || !d_outs) return fail(PCR_ERR_INVALID_ARG, "null argument");
  std::vector<pcr_retrieval_plan> plans(n);
  for (int k = 0; k < n; k++) {
    if (!hs[k]) return fail(PCR_ERR_INVALID_ARG, "null handle");
    if (targets[k].has_box) return fail(PCR_ERR_UNSUPPORTED, "box targets go through pcr_retrieve");
    const auto t0 = std::chrono::steady_clock::now();
    const pcr_status ps = pcr_plan(hs[k], &targets[k], &plans[k]);
    if (infos) {
      infos[k].want_gpu_ms = 0;
      fill_info(hs[k], &targets[k], plans[k], ms_since(t0), &infos[k]);
    }
    if (ps != PCR_OK) return ps;
  }
  const auto t1 = std::chrono::steady_clock::now();
  const pcr_status st = pcr_retrieve_batch_plan(n, hs, plans.data(), d_outs, cuda_stream);
  if (infos) {
    const double e = ms_since(t1);
    for (int k = 0; k < n; k++) infos[k].enqueue_ms = e;
  }
  return st;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

// ---------------------------------------------------------------------------
// error tables of every stream (Sec. V-C)
// ---------------------------------------------------------------------------
extern "C" pcr_status pcr_get_tables(const pcr_handle* h, pcr_tables* out) try {
  if (!h || !out) return fail(PCR_ERR_INVALID_ARG, "null argument");
  const int ns = (int)h->geo.size();
  out->nstreams = ns;
  out->nplanes = h->B;
  for (int i = 0; i < PCR_MAX_STREAMS; i++) out->exponent[i] = i < ns ? h->E[i] : 0;
  for (int i = 0; i < ns; i++) {
    const Tab& t = h->tabs[i];
    const size_t o = (size_t)i * (h->B + 1);
    for (int b = 0; b <= h->B; b++) {
      if (out->maxerr) out->maxerr[o + b] = t.maxerr[b];
      if (out->sq) out->sq[o + b] = t.sq[b];
      if (out->bytes) out->bytes[o + b] = t.bytes[b];
    }
  }
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

// ---------------------------------------------------------------------------
// introspection
// ---------------------------------------------------------------------------
extern "C" pcr_status pcr_num_streams(const pcr_handle* h, int* n) try {
  if (!h || !n) return fail(PCR_ERR_INVALID_ARG, "null argument");
  *n = (int)h->geo.size();
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" pcr_status pcr_stream_info_get(const pcr_handle* h, int i, pcr_stream_info* o) try {
  if (!h || !o || i < 0 || i >= (int)h->geo.size()) return fail(PCR_ERR_INVALID_ARG, "bad stream index");
  const SGeo& g = h->geo[i];
  o->level = g.level;
  o->region = g.region;
  o->sub = g.sub;
  o->is_fixed = g.is_fix;
  o->nplanes = h->B;
  o->n_real = g.n_real();
  o->n_pad = g.n_pad();
  o->words = g.n_pad() / 32;
  o->nseg = (g.n_pad() + kSegElems - 1) / kSegElems;
  o->exponent = h->E[i];
  o->shift = h->sh[i];
  o->vmax = h->vmax[i];
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" pcr_status pcr_stream_tables(const pcr_handle* h, int i, double* maxerr, double* sq, uint64_t* bytes) try {
  if (!h || i < 0 || i >= (int)h->geo.size()) return fail(PCR_ERR_INVALID_ARG, "bad stream index");
  const Tab& t = h->tabs[i];
  for (int b = 0; b <= h->B; b++) {
    if (maxerr) maxerr[b] = t.maxerr[b];
    if (sq) sq[b] = t.sq[b];
    if (bytes) bytes[b] = t.bytes[b];
  }
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" pcr_status pcr_field_stats(const pcr_handle* h, double* xmin, double* xmax, int* G) try {
  if (!h) return fail(PCR_ERR_INVALID_ARG, "null handle");
  if (xmin) *xmin = h->xmin;
  if (xmax) *xmax = h->xmax;
  if (G) *G = h->G;
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" pcr_status pcr_stream_copy(const pcr_handle* h, int i, uint32_t* planes_host, uint32_t* signs_host,
                                      uint32_t* sign_counts_host, uint64_t* pairs_host) try {
  if (!h || i < 0 || i >= (int)h->geo.size()) return fail(PCR_ERR_INVALID_ARG, "bad stream index");
  if (!h->d_block) return fail(PCR_ERR_UNSUPPORTED, "a planning-only handle holds no planes");
  const int64_t words = h->geo[i].n_pad() / 32;
  const int64_t nseg = (h->geo[i].n_pad() + kSegElems - 1) / kSegElems;
  if (planes_host) CUDA_TRY(cudaMemcpy(planes_host, h->d_planes + h->plane_off[i], (size_t)h->B * words * 4, cudaMemcpyDeviceToHost));
  if (signs_host && h->enc == 1)
    CUDA_TRY(cudaMemcpy(signs_host, h->d_signs + h->sign_off[i], (size_t)nseg * h->slot_words * 4, cudaMemcpyDeviceToHost));
  if (sign_counts_host)
    CUDA_TRY(cudaMemcpy(sign_counts_host, h->d_scnt + h->scnt_off[i], (size_t)nseg * h->B * 4, cudaMemcpyDeviceToHost));
  if (pairs_host && !h->pairs[i].empty()) std::memcpy(pairs_host, h->pairs[i].data(), h->pairs[i].size() * 8);
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" pcr_status pcr_max_ordering(const pcr_handle* h, double* errs, int* n) try {
  if (!h || !n) return fail(PCR_ERR_INVALID_ARG, "null argument");
  if (!h->has_m0) {
    *n = 0;
    return PCR_OK;
  }
  *n = (int)h->m0.size() + 1;
  if (errs) {
    errs[0] = h->m0_init;
    for (size_t k = 0; k < h->m0.size(); k++) errs[k + 1] = h->m0[k].val;
  }
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" void pcr_free(pcr_handle* h) { delete h; }
extern "C" void pcr_buffer_free(void* p) { std::free(p); }

// ---------------------------------------------------------------------------
// container: magic, version, header, tables, directory, payload; CRC32 of
// each section (Sec. III-A: the refactored segments are the stored artifact)
// ---------------------------------------------------------------------------
namespace {
uint32_t crc32(const void* data, size_t n, uint32_t c = 0) {
  static uint32_t table[256];
  static bool init = false;
  if (!init) {
    for (uint32_t i = 0; i < 256; i++) {
      uint32_t r = i;
      for (int k = 0; k < 8; k++) r = (r >> 1) ^ (0xEDB88320u & (0u - (r & 1u)));
      table[i] = r;
    }
    init = true;
  }
  c = ~c;
  const uint8_t* p = (const uint8_t*)data;
  for (size_t i = 0; i < n; i++) c = table[(c ^ p[i]) & 0xFF] ^ (c >> 8);
  return ~c;
}

struct Writer {
  std::vector<uint8_t> buf;
  template <class T> void put(const T& v) {
    const uint8_t* p = (const uint8_t*)&v;
    buf.insert(buf.end(), p, p + sizeof(T));
  }
  void raw(const void* p, size_t n) { buf.insert(buf.end(), (const uint8_t*)p, (const uint8_t*)p + n); }
};

struct Reader {
  const uint8_t* p;
  size_t n, o = 0;
  bool ok = true;
  template <class T> T get() {
    T v{};
    if (o + sizeof(T) > n) {
      ok = false;
      return v;
    }
    std::memcpy(&v, p + o, sizeof(T));
    o += sizeof(T);
    return v;
  }
  const uint8_t* take(size_t k) {
    if (o + k > n) {
      ok = false;
      return nullptr;
    }
    const uint8_t* q = p + o;
    o += k;
    return q;
  }
};
const uint64_t kMagic = 0x3230524350ull;        // "PCR02": planes stored raw
const uint64_t kPackedMagic = 0x3250524350ull;  // "PCRP2": planes stored coded (pcr_serialize_packed)
}  // namespace

// what a handle's tables and planner need: dims, dtype, scheme, field
// statistics, per stream its maximum, exponent, shift, nonzero-plane counts,
// sign counts per segment and plane-pair counts
static pcr_status write_header(const pcr_handle* h, Writer& hd) {
  hd.put(h->ndim);
  for (int i = 0; i < 3; i++) hd.put(h->dims[i]);
  hd.put(h->dtype);
  hd.put(h->sch);
  hd.put(h->xmin);
  hd.put(h->xmax);
  hd.put(h->G);
  hd.put(h->C0);
  hd.put(h->C0c);
  const int ns = (int)h->geo.size();
  for (int i = 0; i < ns; i++) {
    hd.put(h->vmax[i]);
    hd.put(h->E[i]);
    hd.put(h->sh[i]);
    hd.raw(h->plane_nz[i].data(), h->plane_nz[i].size() * 4);
    {
      const int64_t nseg = (h->geo[i].n_pad() + kSegElems - 1) / kSegElems;
      std::vector<uint32_t> sc((size_t)nseg * h->B);
      CUDA_TRY(cudaMemcpy(sc.data(), h->d_scnt + h->scnt_off[i], sc.size() * 4, cudaMemcpyDeviceToHost));
      hd.raw(sc.data(), sc.size() * 4);
    }
    const uint64_t np = h->pairs[i].size();
    hd.put(np);
    hd.raw(h->pairs[i].data(), np * 8);
  }
  return PCR_OK;
}

extern "C" pcr_status pcr_serialize(const pcr_handle* h, void** buf, size_t* len) try {
  if (!h || !buf || !len) return fail(PCR_ERR_INVALID_ARG, "null argument");
  if (!h->d_block) return fail(PCR_ERR_UNSUPPORTED, "a planning-only handle holds no planes");
  Writer w;
  w.put(kMagic);
  Writer hd;
  pcr_status e = write_header(h, hd);
  if (e) return e;
  w.put((uint64_t)hd.buf.size());
  w.put(crc32(hd.buf.data(), hd.buf.size()));
  w.raw(hd.buf.data(), hd.buf.size());
  // payload: planes then signs
  std::vector<uint32_t> planes(h->plane_words), signs(h->sign_area_words);
  CUDA_TRY(cudaMemcpy(planes.data(), h->d_planes, h->plane_words * 4, cudaMemcpyDeviceToHost));
  if (h->sign_area_words)
    CUDA_TRY(cudaMemcpy(signs.data(), h->d_signs, h->sign_area_words * 4, cudaMemcpyDeviceToHost));
  w.put((uint64_t)planes.size());
  w.put(crc32(planes.data(), planes.size() * 4));
  w.raw(planes.data(), planes.size() * 4);
  w.put((uint64_t)signs.size());
  w.put(crc32(signs.data(), signs.size() * 4));
  w.raw(signs.data(), signs.size() * 4);
  void* out = std::malloc(w.buf.size());
  if (!out) return fail(PCR_ERR_OOM, "host allocation failed");
  std::memcpy(out, w.buf.data(), w.buf.size());
  *buf = out;
  *len = w.buf.size();
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

static pcr_status read_header(Reader& hr, pcr_handle* h, std::vector<std::vector<uint32_t>>& scnts) {
  const int ndim = hr.get<int>();
  int64_t dims[3];
  for (int i = 0; i < 3; i++) dims[i] = hr.get<int64_t>();
  const int dtype = hr.get<int>();
  const pcr_scheme sch = hr.get<pcr_scheme>();
  if (!hr.ok) return fail(PCR_ERR_CORRUPT, "truncated header");
  pcr_status e = validate((const void*)1, ndim, dims, dtype, &sch);
  if (e) return fail(PCR_ERR_CORRUPT, std::string("invalid header: ") + g_err);
  e = setup_handle(h, ndim, dims, dtype, &sch);
  if (e) return fail(PCR_ERR_CORRUPT, std::string("invalid header: ") + g_err);
  h->xmin = hr.get<double>();
  h->xmax = hr.get<double>();
  h->G = hr.get<int>();
  h->C0 = hr.get<double>();
  h->C0c = hr.get<double>();
  h->M = std::max(std::fabs(h->xmin), std::fabs(h->xmax));
  h->h = std::ldexp(1.0, h->G - fix_bits(h->vk, h->L));
  const int ns = (int)h->geo.size();
  h->vmax.resize(ns);
  h->E.resize(ns);
  h->sh.resize(ns);
  h->plane_nz.resize(ns);
  scnts.assign(ns, {});
  h->sign_words.assign(ns, std::vector<uint32_t>(h->B, 0));
  h->pairs.resize(ns);
  h->tabs.resize(ns);
  for (int i = 0; i < ns; i++) {
    h->vmax[i] = hr.get<double>();
    h->E[i] = hr.get<int>();
    h->sh[i] = hr.get<int>();
    h->plane_nz[i].resize(h->B);
    for (int k = 0; k < h->B; k++) h->plane_nz[i][k] = hr.get<uint32_t>();
    const int64_t nseg = (h->geo[i].n_pad() + kSegElems - 1) / kSegElems;
    scnts[i].resize(nseg * h->B);
    for (auto& x : scnts[i]) x = hr.get<uint32_t>();
    for (int64_t sg = 0; sg < nseg; sg++)
      for (int k = 0; k < h->B; k++) h->sign_words[i][k] += (scnts[i][sg * h->B + k] + 31) / 32;
    const uint64_t np = hr.get<uint64_t>();
    if (!hr.ok || (np != 0 && np != (uint64_t)h->B * h->B)) return fail(PCR_ERR_CORRUPT, "bad table section");
    h->pairs[i].resize(np);
    for (auto& x : h->pairs[i]) x = hr.get<uint64_t>();
  }
  if (!hr.ok || hr.o != hr.n) return fail(PCR_ERR_CORRUPT, "header length mismatch");
  return PCR_OK;
}

static void pack_tasks(const pcr_handle* h, uint32_t* planes, std::vector<PackTask>& tasks);

extern "C" pcr_status pcr_deserialize(const void* buf, size_t len, const pcr_allocator* alloc, void* cuda_stream,
                                      pcr_handle** out) try {
  if (!buf || !out) return fail(PCR_ERR_INVALID_ARG, "null argument");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  Reader r{(const uint8_t*)buf, len};
  const uint64_t magic = r.get<uint64_t>();
  if (!r.ok || (magic != kMagic && magic != kPackedMagic)) return fail(PCR_ERR_CORRUPT, "bad magic");
  const bool packed = magic == kPackedMagic;
  const uint64_t hl = r.get<uint64_t>();
  const uint32_t hc = r.get<uint32_t>();
  const uint8_t* hp = r.take(hl);
  if (!r.ok || crc32(hp, hl) != hc) return fail(PCR_ERR_CORRUPT, "header checksum or length mismatch");
  Reader hr{hp, hl};
  std::unique_ptr<pcr_handle> h(new pcr_handle());
  h->mem = make_mem(alloc);
  std::vector<std::vector<uint32_t>> scnts;
  pcr_status e = read_header(hr, h.get(), scnts);
  if (e) return e;
  const int ns = (int)h->geo.size();
  const uint8_t* pp = nullptr;   // raw planes
  uint64_t npw = 0;
  std::vector<PackTask> tasks;   // coded planes: per task header, payload offsets
  const uint32_t* heads = nullptr;
  const uint32_t* pay = nullptr;
  std::vector<uint64_t> off;
  if (!packed) {
    npw = r.get<uint64_t>();
    const uint32_t pc = r.get<uint32_t>();
    pp = r.take(npw * 4);
    if (!r.ok || npw != h->plane_words || crc32(pp, npw * 4) != pc)
      return fail(PCR_ERR_CORRUPT, "plane section mismatch");
  } else {
    pack_tasks(h.get(), nullptr, tasks);
    const uint64_t nt = r.get<uint64_t>();
    const uint32_t hcrc = r.get<uint32_t>();
    heads = (const uint32_t*)r.take(nt * 4);
    if (!r.ok || nt != tasks.size() || crc32(heads, nt * 4) != hcrc)
      return fail(PCR_ERR_CORRUPT, "coded plane headers mismatch");
    // every header must describe its segment: mode, ones, payload length
    off.assign(nt + 1, 0);
    for (size_t t = 0; t < nt; t++) {
      uint32_t hw;
      std::memcpy(&hw, (const uint8_t*)heads + 4 * t, 4);
      const int64_t w0 = (int64_t)tasks[t].seg * kSegWords;
      const uint32_t nw = (uint32_t)std::min<int64_t>(kSegWords, tasks[t].words - w0);
      const uint32_t mode = hw & 3, m = (hw >> 6) & 0x1FFF, pw = hw >> 19;
      const bool good = (mode == 0 && hw == 0) || (mode == 2 && pw == nw) ||
                        (mode == 1 && m >= 1 && m <= 32 * nw && pw >= 1 && pw <= nw);
      if (!good) return fail(PCR_ERR_CORRUPT, "coded plane header out of range");
      off[t + 1] = off[t] + pw;
    }
    const uint64_t np = r.get<uint64_t>();
    const uint32_t pcrc = r.get<uint32_t>();
    pay = (const uint32_t*)r.take(np * 4);
    if (!r.ok || np != off[nt] || crc32(pay, np * 4) != pcrc) return fail(PCR_ERR_CORRUPT, "coded plane payload mismatch");
  }
  const uint64_t nsw = r.get<uint64_t>();
  const uint32_t sgc = r.get<uint32_t>();
  const uint8_t* sp = r.take(nsw * 4);
  if (!r.ok || nsw != h->sign_area_words || crc32(sp, nsw * 4) != sgc)
    return fail(PCR_ERR_CORRUPT, "sign section mismatch");
  if (r.o != len) return fail(PCR_ERR_CORRUPT, "trailing bytes");
  e = alloc_handle_buffers(h.get(), s);
  if (e) return e;
  if (!packed) {
    CUDA_TRY(cudaMemcpyAsync(h->d_planes, pp, npw * 4, cudaMemcpyHostToDevice, s));
  } else if (!tasks.empty()) {
    // planes with no nonzero word are not stored: zero, then decode the rest
    CUDA_TRY(cudaMemsetAsync(h->d_planes, 0, h->plane_words * 4, s));
    pack_tasks(h.get(), h->d_planes, tasks);   // the same tasks, now over this handle's planes
    const size_t nt = tasks.size();
    Scratch sc{&h->mem, s, {}};
    PackTask* d_t = (PackTask*)sc.get(nt * sizeof(PackTask));
    uint32_t* d_h = (uint32_t*)sc.get(nt * 4);
    uint64_t* d_o = (uint64_t*)sc.get((nt + 1) * 8);
    uint32_t* d_p = (uint32_t*)sc.get(std::max<uint64_t>(off[nt], 1) * 4);
    int* d_err = (int*)sc.get(sizeof(int));
    if (!d_t || !d_h || !d_o || !d_p || !d_err) return fail(PCR_ERR_OOM, "unpacking allocation failed");
    CUDA_TRY(cudaMemcpyAsync(d_t, tasks.data(), nt * sizeof(PackTask), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(d_h, heads, nt * 4, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(d_o, off.data(), (nt + 1) * 8, cudaMemcpyHostToDevice, s));
    if (off[nt]) CUDA_TRY(cudaMemcpyAsync(d_p, pay, off[nt] * 4, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemsetAsync(d_err, 0, sizeof(int), s));
    launch_unpack(d_t, (int)nt, d_h, d_o, d_p, d_err, s);
    CUDA_TRY(cudaGetLastError());
    int err = 0;
    CUDA_TRY(cudaMemcpyAsync(&err, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    CUDA_TRY(cudaStreamSynchronize(s));
    if (err) return fail(PCR_ERR_CORRUPT, "coded plane payload does not decode");
  }
  if (nsw) CUDA_TRY(cudaMemcpyAsync(h->d_signs, sp, nsw * 4, cudaMemcpyHostToDevice, s));
  std::vector<uint32_t> scnt, nz;
  for (int i = 0; i < ns; i++) {
    scnt.insert(scnt.end(), scnts[i].begin(), scnts[i].end());
    nz.insert(nz.end(), h->plane_nz[i].begin(), h->plane_nz[i].end());
    nz.insert(nz.end(), h->sign_words[i].begin(), h->sign_words[i].end());
  }
  if (!scnt.empty()) CUDA_TRY(cudaMemcpyAsync(h->d_scnt, scnt.data(), scnt.size() * 4, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(h->d_nz, nz.data(), nz.size() * 4, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  for (int i = 0; i < ns; i++)
    compute_tables(h.get(), i, h->pairs[i].empty() ? nullptr : &h->pairs[i], keeps_pairs(h.get()));
  build_meta(h.get());
  *out = h.release();
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

// ---------------------------------------------------------------------------
// planning state: what the interpreter needs, without planes (block
// sharding: ranks exchange their blocks' states and plan the whole field)
// ---------------------------------------------------------------------------
const uint64_t kPlanMagic = 0x3230534C50ull;  // "PLS02"

extern "C" pcr_status pcr_export_plan_state(const pcr_handle* h, void** buf, size_t* len) try {
  if (!h || !buf || !len) return fail(PCR_ERR_INVALID_ARG, "null argument");
  if (!h->d_block) return fail(PCR_ERR_UNSUPPORTED, "a planning-only handle is exported by its owner");
  Writer w;
  w.put(kPlanMagic);
  Writer hd;
  pcr_status e = write_header(h, hd);
  if (e) return e;
  w.put((uint64_t)hd.buf.size());
  w.put(crc32(hd.buf.data(), hd.buf.size()));
  w.raw(hd.buf.data(), hd.buf.size());
  void* out = std::malloc(w.buf.size());
  if (!out) return fail(PCR_ERR_OOM, "host allocation failed");
  std::memcpy(out, w.buf.data(), w.buf.size());
  *buf = out;
  *len = w.buf.size();
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" pcr_status pcr_import_plan_state(const void* buf, size_t len, pcr_handle** out) try {
  if (!buf || !out) return fail(PCR_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  Reader r{(const uint8_t*)buf, len};
  if (r.get<uint64_t>() != kPlanMagic || !r.ok) return fail(PCR_ERR_CORRUPT, "bad magic");
  const uint64_t hl = r.get<uint64_t>();
  const uint32_t hc = r.get<uint32_t>();
  const uint8_t* hp = r.take(hl);
  if (!r.ok || crc32(hp, hl) != hc) return fail(PCR_ERR_CORRUPT, "header checksum or length mismatch");
  if (r.o != len) return fail(PCR_ERR_CORRUPT, "trailing bytes");
  Reader hr{hp, hl};
  std::unique_ptr<pcr_handle> h(new pcr_handle());
  h->mem = make_mem(nullptr);
  std::vector<std::vector<uint32_t>> scnts;
  pcr_status e = read_header(hr, h.get(), scnts);
  if (e) return e;
  for (int i = 0; i < (int)h->geo.size(); i++)
    compute_tables(h.get(), i, h->pairs[i].empty() ? nullptr : &h->pairs[i], keeps_pairs(h.get()));
  build_meta(h.get());
  *out = h.release();
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

// ---------------------------------------------------------------------------
// lossless coding of plane words (Sec. V): every nonzero plane of every
// stream coded per 4096-value segment (pcr_pack.cu); sizes for the tables,
// and a container whose planes are stored coded
// ---------------------------------------------------------------------------
// tasks in (stream, plane, segment) order over the planes with a nonzero word
static void pack_tasks(const pcr_handle* h, uint32_t* planes, std::vector<PackTask>& tasks) {
  tasks.clear();
  for (int i = 0; i < (int)h->geo.size(); i++) {
    const int64_t words = h->geo[i].n_pad() / 32;
    const int nseg = (int)((words + kSegWords - 1) / kSegWords);
    for (int k = 0; k < h->B; k++) {
      if (!h->plane_nz[i][k]) continue;
      for (int g = 0; g < nseg; g++) tasks.push_back({planes + h->plane_off[i] + (size_t)k * words, words, g});
    }
  }
}

// headers and payload words of every task of a live handle (synchronous)
static pcr_status pack_headers(const pcr_handle* h, const std::vector<PackTask>& tasks, cudaStream_t s,
                               std::vector<uint32_t>& headers, std::vector<uint32_t>& pwords) {
  const size_t nt = tasks.size();
  headers.assign(nt, 0);
  pwords.assign(nt, 0);
  if (!nt) return PCR_OK;
  Mem mem = h->mem;
  Scratch sc{&mem, s, {}};
  PackTask* d_t = (PackTask*)sc.get(nt * sizeof(PackTask));
  uint32_t* d_h = (uint32_t*)sc.get(nt * 4);
  uint32_t* d_w = (uint32_t*)sc.get(nt * 4);
  if (!d_t || !d_h || !d_w) return fail(PCR_ERR_OOM, "packing allocation failed");
  CUDA_TRY(cudaMemcpyAsync(d_t, tasks.data(), nt * sizeof(PackTask), cudaMemcpyHostToDevice, s));
  launch_pack_sizes(d_t, (int)nt, d_h, d_w, s);
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(headers.data(), d_h, nt * 4, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaMemcpyAsync(pwords.data(), d_w, nt * 4, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return PCR_OK;
}

extern "C" pcr_status pcr_packed_tables(const pcr_handle* h, uint64_t* bytes) try {
  if (!h || !bytes) return fail(PCR_ERR_INVALID_ARG, "null argument");
  if (!h->d_block) return fail(PCR_ERR_UNSUPPORTED, "a planning-only handle holds no planes");
  const int ns = (int)h->geo.size();
  {
    std::lock_guard<std::mutex> lk(h->plan_mu);
    if (!h->packed_ok) {
      std::vector<PackTask> tasks;
      pack_tasks(h, h->d_planes, tasks);
      std::vector<uint32_t> hd, pw;
      pcr_status e = pack_headers(h, tasks, nullptr, hd, pw);
      if (e) return e;
      h->packed.assign(ns, std::vector<uint64_t>(h->B, 0));
      size_t t = 0;
      for (int i = 0; i < ns; i++) {
        const int64_t words = h->geo[i].n_pad() / 32;
        const int nseg = (int)((words + kSegWords - 1) / kSegWords);
        for (int k = 0; k < h->B; k++) {
          if (!h->plane_nz[i][k]) continue;
          for (int g = 0; g < nseg; g++, t++) h->packed[i][k] += 4 + 4 * (uint64_t)pw[t];
        }
      }
      h->packed_ok = true;
    }
  }
  const bool nb = h->enc == 2;
  for (int i = 0; i < ns; i++) {
    uint64_t acc = 0;
    bytes[(size_t)i * (h->B + 1)] = 0;
    for (int k = 0; k < h->B; k++) {
      acc += h->packed[i][k];
      if (!nb) acc += 4 * (uint64_t)h->sign_words[i][k];
      bytes[(size_t)i * (h->B + 1) + k + 1] = acc;
    }
  }
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

// test entry: the coded form of one segment's plane words (at most 128
// words in device memory): header and payload words (payload: room for 128)
extern "C" pcr_status pcr_debug_pack(const uint32_t* d_words, int nwords, uint32_t* header, uint32_t* payload,
                                     int* npayload) try {
  if (!d_words || !header || !payload || !npayload || nwords < 1 || nwords > kSegWords)
    return fail(PCR_ERR_INVALID_ARG, "bad argument");
  const PackTask tk{const_cast<uint32_t*>(d_words), nwords, 0};
  PackTask* d_t = nullptr;
  uint32_t *d_h = nullptr, *d_w = nullptr, *d_p = nullptr;
  uint64_t* d_o = nullptr;
  auto release = [&]() {
    cudaFree(d_t);
    cudaFree(d_h);
    cudaFree(d_w);
    cudaFree(d_p);
    cudaFree(d_o);
  };
  if (cudaMalloc(&d_t, sizeof(PackTask)) != cudaSuccess || cudaMalloc(&d_h, 4) != cudaSuccess ||
      cudaMalloc(&d_w, 4) != cudaSuccess || cudaMalloc(&d_p, kSegWords * 4) != cudaSuccess ||
      cudaMalloc(&d_o, 16) != cudaSuccess) {
    release();
    cudaGetLastError();
    return fail(PCR_ERR_OOM, "debug allocation failed");
  }
  const uint64_t off[2] = {0, (uint64_t)kSegWords};
  uint32_t pw = 0;
  cudaError_t ce = cudaMemcpy(d_t, &tk, sizeof(PackTask), cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(d_o, off, 16, cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) {
    launch_pack_sizes(d_t, 1, d_h, d_w, nullptr);
    launch_pack_write(d_t, 1, d_h, d_o, d_p, nullptr);
    ce = cudaGetLastError();
  }
  if (ce == cudaSuccess) ce = cudaMemcpy(header, d_h, 4, cudaMemcpyDeviceToHost);
  if (ce == cudaSuccess) ce = cudaMemcpy(&pw, d_w, 4, cudaMemcpyDeviceToHost);
  if (ce == cudaSuccess && pw) ce = cudaMemcpy(payload, d_p, pw * 4, cudaMemcpyDeviceToHost);
  release();
  if (ce != cudaSuccess) return fail(PCR_ERR_CUDA, cudaGetErrorString(ce));
  *npayload = (int)pw;
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

extern "C" pcr_status pcr_serialize_packed(const pcr_handle* h, void** buf, size_t* len) try {
  if (!h || !buf || !len) return fail(PCR_ERR_INVALID_ARG, "null argument");
  if (!h->d_block) return fail(PCR_ERR_UNSUPPORTED, "a planning-only handle holds no planes");
  Writer w;
  w.put(kPackedMagic);
  Writer hd;
  pcr_status e = write_header(h, hd);
  if (e) return e;
  w.put((uint64_t)hd.buf.size());
  w.put(crc32(hd.buf.data(), hd.buf.size()));
  w.raw(hd.buf.data(), hd.buf.size());
  // coded planes: every task's header, then the payloads in task order
  std::vector<PackTask> tasks;
  pack_tasks(h, h->d_planes, tasks);
  std::vector<uint32_t> heads, pw;
  e = pack_headers(h, tasks, nullptr, heads, pw);
  if (e) return e;
  const size_t nt = tasks.size();
  std::vector<uint64_t> off(nt + 1, 0);
  for (size_t t = 0; t < nt; t++) off[t + 1] = off[t] + pw[t];
  std::vector<uint32_t> payload(off[nt]);
  if (nt && off[nt]) {
    Mem mem = h->mem;
    Scratch sc{&mem, nullptr, {}};
    PackTask* d_t = (PackTask*)sc.get(nt * sizeof(PackTask));
    uint32_t* d_h = (uint32_t*)sc.get(nt * 4);
    uint64_t* d_o = (uint64_t*)sc.get((nt + 1) * 8);
    uint32_t* d_p = (uint32_t*)sc.get(off[nt] * 4);
    if (!d_t || !d_h || !d_o || !d_p) return fail(PCR_ERR_OOM, "packing allocation failed");
    CUDA_TRY(cudaMemcpy(d_t, tasks.data(), nt * sizeof(PackTask), cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_h, heads.data(), nt * 4, cudaMemcpyHostToDevice));
    CUDA_TRY(cudaMemcpy(d_o, off.data(), (nt + 1) * 8, cudaMemcpyHostToDevice));
    launch_pack_write(d_t, (int)nt, d_h, d_o, d_p, nullptr);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpy(payload.data(), d_p, off[nt] * 4, cudaMemcpyDeviceToHost));
  }
  w.put((uint64_t)nt);
  w.put(crc32(heads.data(), nt * 4));
  w.raw(heads.data(), nt * 4);
  w.put((uint64_t)payload.size());
  w.put(crc32(payload.data(), payload.size() * 4));
  w.raw(payload.data(), payload.size() * 4);
  std::vector<uint32_t> signs(h->sign_area_words);
  if (h->sign_area_words)
    CUDA_TRY(cudaMemcpy(signs.data(), h->d_signs, h->sign_area_words * 4, cudaMemcpyDeviceToHost));
  w.put((uint64_t)signs.size());
  w.put(crc32(signs.data(), signs.size() * 4));
  w.raw(signs.data(), signs.size() * 4);
  void* out = std::malloc(w.buf.size());
  if (!out) return fail(PCR_ERR_OOM, "host allocation failed");
  std::memcpy(out, w.buf.data(), w.buf.size());
  *buf = out;
  *len = w.buf.size();
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

// ---------------------------------------------------------------------------
// target-driven sampled tuning (Sec. VI-A and its tuning table)
// ---------------------------------------------------------------------------
// Sample: whole blocks of b^D points (b = min(edge, n) per axis) centred on a
// regular k_0 x .. x k_(D-1) grid, the counts grown one axis at a time (the
// axis with the most points per block slot first) while the blocks stay
// within `fraction` of the field, at least one block; each block refactored
// as a field of its own with every candidate; at each of 9 tolerances tau
// (relative to the whole field's range R) the candidate needing the fewest
// bytes over all blocks gets a vote (error-bound mode: max |x - x'| <= tau R
// per block; PSNR mode: squared errors <= n_block (tau R)^2 per block); a
// candidate unable to meet tau in some block takes no part in that vote;
// ties go to the earlier candidate.
namespace {
const double kTuneTol[PCR_TUNE_NTOL] = {1e-3, 5e-4, 1e-4, 5e-5, 1e-5, 5e-6, 1e-6, 5e-7, 1e-7};

std::vector<pcr_scheme> tune_candidates(int mode, int ndim) {
  std::vector<std::array<int, 3>> orders;
  std::array<int, 3> o = {0, 1, 2};
  const int d = ndim == 3 ? 3 : 2;
  do {
    orders.push_back(o);
  } while (std::next_permutation(o.begin(), o.begin() + d));
  std::vector<int> decomps = ndim == 3 ? std::vector<int>{-1, 0, 1, 2} : std::vector<int>{-1};
  std::vector<std::pair<int, std::array<int, 3>>> interps;
  if (mode == PCR_MODE_EB) interps.push_back({PCR_INTERP_LEVEL, {0, 1, 2}});
  for (auto& od : orders) interps.push_back({PCR_INTERP_REGION, od});
  std::vector<pcr_scheme> out;
  for (auto& it : interps)
    for (int dax : decomps) {
      pcr_scheme c{};
      c.mode = mode;
      c.interp = it.first;
      c.degree = PCR_CUBIC;
      for (int k = 0; k < 3; k++) c.order[k] = it.second[k];
      c.decomp_axis = dax;
      c.encoding = mode == PCR_MODE_PSNR ? PCR_ENC_NEGABINARY : PCR_ENC_GENERIC;
      out.push_back(c);
    }
  return out;
}

void tune_blocks(const int64_t* dims, int ndim, double fraction, int edge, std::vector<std::array<int64_t, 3>>& org,
                 int64_t* b) {
  int64_t k[3] = {1, 1, 1};
  int64_t N = 1, per = 1;
  for (int d = 0; d < ndim; d++) {
    b[d] = std::min<int64_t>(edge, dims[d]);
    N *= dims[d];
    per *= b[d];
  }
  while (true) {
    int best = -1;
    for (int d = 0; d < ndim; d++) {
      const double r = (double)dims[d] / (double)(k[d] + 1), rb = best < 0 ? 0.0 : (double)dims[best] / (double)(k[best] + 1);
      if ((k[d] + 1) * b[d] <= dims[d] && (best < 0 || r > rb)) best = d;
    }
    if (best < 0) break;
    int64_t tot = per;
    for (int d = 0; d < ndim; d++) tot *= d == best ? k[d] + 1 : k[d];
    if ((double)tot > fraction * (double)N) break;
    k[best]++;
  }
  org.clear();
  int64_t idx[3] = {0, 0, 0};
  const int64_t nb = k[0] * (ndim > 1 ? k[1] : 1) * (ndim > 2 ? k[2] : 1);
  for (int64_t t = 0; t < nb; t++) {
    int64_t r = t;
    for (int d = ndim - 1; d >= 0; d--) {
      idx[d] = r % k[d];
      r /= k[d];
    }
    std::array<int64_t, 3> o = {0, 0, 0};
    for (int d = 0; d < ndim; d++) {
      const int64_t c = ((2 * idx[d] + 1) * dims[d]) / (2 * k[d]);
      o[d] = std::min(std::max<int64_t>(c - b[d] / 2, 0), dims[d] - b[d]);
    }
    org.push_back(o);
  }
}

double key_to_double(unsigned long long k) {
  unsigned long long u = (k >> 63) ? (k & 0x7FFFFFFFFFFFFFFFull) : ~k;
  double d;
  std::memcpy(&d, &u, 8);
  return d;
}
}  // namespace

extern "C" pcr_status pcr_tune(const void* d_field, int ndim, const int64_t* dims, int dtype, int mode, double fraction,
                               int edge, const pcr_allocator* alloc, void* cuda_stream, pcr_scheme* out,
                               pcr_tune_info* info) try {
  const auto t0 = std::chrono::steady_clock::now();
  if (!d_field || !dims || !out) return fail(PCR_ERR_INVALID_ARG, "null argument");
  if (ndim != 2 && ndim != 3) return fail(PCR_ERR_INVALID_ARG, "ndim must be 2 or 3");
  if (mode != PCR_MODE_EB && mode != PCR_MODE_PSNR) return fail(PCR_ERR_INVALID_ARG, "tuning needs EB or PSNR mode");
  if (dtype != PCR_F32 && dtype != PCR_F64) return fail(PCR_ERR_INVALID_ARG, "bad dtype");
  for (int d = 0; d < ndim; d++)
    if (dims[d] < 2) return fail(PCR_ERR_INVALID_ARG, "every dimension must be >= 2");
  if (fraction <= 0) fraction = 0.01;
  if (edge <= 0) edge = 64;
  if (edge < 4) return fail(PCR_ERR_INVALID_ARG, "block edge must be >= 4");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  Mem mem = make_mem(alloc);
  const int vk = dtype == PCR_F64 ? VK_F64 : VK_F32;
  const size_t w = vsize(vk);
  int64_t n3[3] = {1, 1, 1};
  for (int d = 0; d < ndim; d++) n3[3 - ndim + d] = dims[d];
  const int64_t n = n3[0] * n3[1] * n3[2];
  // the whole field's range
  std::vector<std::array<int64_t, 3>> org;
  int64_t b[3] = {1, 1, 1};
  tune_blocks(dims, ndim, fraction, edge, org, b);
  int64_t bsz = 1;
  for (int d = 0; d < ndim; d++) bsz *= b[d];
  Scratch sc{&mem, s, {}};
  FieldStats* d_st = (FieldStats*)sc.get(sizeof(FieldStats));
  char* d_blocks = (char*)sc.get(org.size() * bsz * w);
  if (!d_st || !d_blocks) return fail(PCR_ERR_OOM, "tuning allocation failed");
  FieldStats st0{};
  st0.xmin_key = ~0ull;
  CUDA_TRY(cudaMemcpyAsync(d_st, &st0, sizeof(st0), cudaMemcpyHostToDevice, s));
  launch_minmax(vk, d_field, n, d_st, s);
  FieldD f{};
  for (int a = 0; a < 3; a++) f.n[a] = n3[a];
  for (size_t k = 0; k < org.size(); k++) {
    Box3 bx;
    for (int a = 0; a < 3; a++) {
      const int d = a - (3 - ndim);
      bx.lo[a] = d >= 0 ? org[k][d] : 0;
      bx.cnt[a] = d >= 0 ? b[d] : 1;
    }
    launch_copy_box(vk, f, d_field, d_blocks + k * bsz * w, bx, s);
  }
  FieldStats st;
  CUDA_TRY(cudaMemcpyAsync(&st, d_st, sizeof(st), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (st.bad) return fail(PCR_ERR_INVALID_ARG, "field contains NaN or Inf");
  const double R = key_to_double(st.xmax_key) - key_to_double(st.xmin_key);
  const std::vector<pcr_scheme> cands = tune_candidates(mode, ndim);
  const int nc = (int)cands.size(), nb = (int)org.size();
  std::vector<const void*> ptrs(nb);
  std::vector<int> nds(nb, ndim), dts(nb, dtype);
  std::vector<const int64_t*> dms(nb, b);
  for (int k = 0; k < nb; k++) ptrs[k] = d_blocks + k * bsz * w;
  const uint64_t kNone = ~uint64_t(0);
  std::vector<std::array<uint64_t, PCR_TUNE_NTOL>> table(nc);
  for (int c = 0; c < nc; c++) {
    std::vector<pcr_scheme> sch(nb, cands[c]);
    std::vector<pcr_handle*> hs(nb, nullptr);
    pcr_status e = pcr_refactor_batch(nb, ptrs.data(), nds.data(), dms.data(), dts.data(), sch.data(), alloc,
                                      cuda_stream, hs.data());
    if (e) return e;
    std::vector<std::unique_ptr<pcr_handle>> own(nb);
    for (int k = 0; k < nb; k++) own[k].reset(hs[k]);
    for (int t = 0; t < PCR_TUNE_NTOL; t++) {
      const double tau = kTuneTol[t] * R;
      uint64_t tot = 0;
      for (int k = 0; k < nb && tot != kNone; k++) {
        std::vector<int> bv;
        double bound = 0;
        const bool ok = mode == PCR_MODE_PSNR ? greedy(hs[k], (double)hs[k]->meta.n * tau * tau, false, bv, bound)
                                              : greedy(hs[k], tau, true, bv, bound);
        if (!ok) {
          tot = kNone;
          break;
        }
        for (size_t i = 0; i < bv.size(); i++) tot += hs[k]->tabs[i].bytes[bv[i]];
      }
      table[c][t] = tot;
    }
  }
  std::vector<int> votes(nc, 0);
  for (int t = 0; t < PCR_TUNE_NTOL; t++) {
    int best = -1;
    for (int c = 0; c < nc; c++)
      if (table[c][t] != kNone && (best < 0 || table[c][t] < table[best][t])) best = c;
    if (best >= 0) votes[best]++;
  }
  int win = 0;
  for (int c = 0; c < nc; c++)
    if (votes[c] > votes[win]) win = c;
  *out = cands[win];
  if (ndim == 2) {   // orders in user axes; the table keeps the 3-D view's natural fill
    out->order[2] = 0;
  }
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->ncand = nc;
    info->winner = win;
    for (int c = 0; c < nc && c < PCR_TUNE_MAX_CANDIDATES; c++) {
      info->votes[c] = votes[c];
      info->cand[c] = cands[c];
      for (int t = 0; t < PCR_TUNE_NTOL; t++) info->bytes[c][t] = table[c][t];
    }
    info->nblocks = nb;
    for (int d = 0; d < ndim; d++) info->block[d] = b[d];
    info->fraction = (double)(bsz * nb) / (double)n;
    info->ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

// Schemes whose interp is PCR_INTERP_AUTO are replaced by the tuner's choice
// for their field (degree, nlevels and nplanes of the request kept).
static pcr_status resolve_auto(int n, const void* const* d_fields, const int* ndims, const int64_t* const* dims,
                               const int* dtypes, const pcr_scheme* schemes, const pcr_allocator* alloc,
                               void* cuda_stream, std::vector<pcr_scheme>& out) {
  out.assign(schemes, schemes + n);
  for (int k = 0; k < n; k++) {
    if (schemes[k].interp != PCR_INTERP_AUTO) continue;
    if (schemes[k].mode == PCR_MODE_EXPLICIT)
      return fail(PCR_ERR_INVALID_ARG, "an explicit scheme cannot leave its interpolation to the tuner");
    pcr_scheme t{};
    pcr_status e = pcr_tune(d_fields[k], ndims[k], dims[k], dtypes[k], schemes[k].mode, 0.0, 0, alloc, cuda_stream,
                            &t, nullptr);
    if (e) return e;
    t.nlevels = schemes[k].nlevels;
    t.nplanes = schemes[k].nplanes;
    out[k] = t;
  }
  return PCR_OK;
}

extern "C" pcr_status pcr_get_scheme(const pcr_handle* h, pcr_scheme* out) try {
  if (!h || !out) return fail(PCR_ERR_INVALID_ARG, "null argument");
  *out = h->sch;
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}

// ---------------------------------------------------------------------------
// test entry: encode given values
// ---------------------------------------------------------------------------
extern "C" pcr_status pcr_debug_encode(const void* d_vals, int64_t n_pad, int value_kind, int B, int encoding,
                                       int want_pairs, void* cuda_stream, uint32_t* planes_host,
                                       uint32_t* signs_host, uint32_t* sign_counts_host, uint32_t* plane_nz_host,
                                       uint64_t* pairs_host, double* vmax_host) try {
  if (!d_vals || n_pad <= 0 || n_pad % 32) return fail(PCR_ERR_INVALID_ARG, "n_pad must be a positive multiple of 32");
  if (value_kind < 0 || value_kind > 2 || encoding < 1 || encoding > 2) return fail(PCR_ERR_INVALID_ARG, "bad kind");
  const int w64 = value_kind == VK_F64 ? 1 : (value_kind == VK_FIX && B > 32 ? 1 : 0);
  if (B < 1 || B > (w64 ? 64 : 32)) return fail(PCR_ERR_INVALID_ARG, "bad B");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  Mem mem = make_mem(nullptr);
  Scratch sc{&mem, s, {}};
  const int64_t words = n_pad / 32, nseg = (n_pad + kSegElems - 1) / kSegElems;
  const int slot = kSegWords + B;
  uint32_t* d_planes = (uint32_t*)sc.get(words * B * 4);
  uint32_t* d_signs = (uint32_t*)sc.get(nseg * slot * 4);
  uint32_t* d_scnt = (uint32_t*)sc.get(nseg * B * 4);
  uint32_t* d_nz = (uint32_t*)sc.get(2 * B * 4);
  unsigned long long* d_pairs = (unsigned long long*)sc.get((size_t)B * B * 8);
  unsigned long long* d_vmax = (unsigned long long*)sc.get(8);
  StreamD* d_sd = (StreamD*)sc.get(sizeof(StreamD));
  WorkItem* d_it = (WorkItem*)sc.get(nseg * sizeof(WorkItem));
  if (!d_planes || !d_signs || !d_scnt || !d_nz || !d_pairs || !d_vmax || !d_sd || !d_it)
    return fail(PCR_ERR_OOM, "allocation failed");
  CUDA_TRY(cudaMemsetAsync(d_nz, 0, 2 * B * 4, s));
  CUDA_TRY(cudaMemsetAsync(d_pairs, 0, (size_t)B * B * 8, s));
  CUDA_TRY(cudaMemsetAsync(d_signs, 0, nseg * slot * 4, s));
  // maximum |value| on the host side of the test entry: read back values
  std::vector<uint8_t> hv(n_pad * (value_kind == VK_F32 ? 4 : 8));
  CUDA_TRY(cudaMemcpyAsync(hv.data(), d_vals, hv.size(), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  unsigned long long vm = 0;
  double vmd = 0;
  for (int64_t i = 0; i < n_pad; i++) {
    if (value_kind == VK_F32) {
      float f;
      std::memcpy(&f, &hv[i * 4], 4);
      f = std::fabs(f);
      uint32_t b;
      std::memcpy(&b, &f, 4);
      vm = std::max<unsigned long long>(vm, b);
      vmd = std::max(vmd, (double)f);
    } else if (value_kind == VK_F64) {
      double f;
      std::memcpy(&f, &hv[i * 8], 8);
      f = std::fabs(f);
      unsigned long long b;
      std::memcpy(&b, &f, 8);
      vm = std::max(vm, b);
      vmd = std::max(vmd, f);
    } else {
      int64_t v;
      std::memcpy(&v, &hv[i * 8], 8);
      const unsigned long long a = (unsigned long long)(v < 0 ? -v : v);
      vm = std::max(vm, a);
      vmd = std::max(vmd, (double)a);
    }
  }
  CUDA_TRY(cudaMemcpyAsync(d_vmax, &vm, 8, cudaMemcpyHostToDevice, s));
  StreamD sd{};
  sd.nlat = 0;
  sd.n_pad = n_pad;
  sd.words = words;
  sd.nseg = nseg;
  sd.B = B;
  sd.enc = encoding;
  sd.vk = value_kind;
  sd.is_fix = value_kind == VK_FIX;
  sd.slot_words = slot;
  sd.planes = d_planes;
  sd.signs = d_signs;
  sd.sign_counts = d_scnt;
  sd.plane_nz = d_nz;
  sd.pairs = want_pairs ? d_pairs : nullptr;
  sd.vmax = d_vmax;
  sd.stage = (void*)d_vals;
  std::vector<WorkItem> it(nseg);
  for (int64_t g = 0; g < nseg; g++) it[g] = {0, (int)g};
  CUDA_TRY(cudaMemcpyAsync(d_sd, &sd, sizeof(sd), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(d_it, it.data(), nseg * sizeof(WorkItem), cudaMemcpyHostToDevice, s));
  launch_encode(value_kind, w64, want_pairs, d_sd, d_it, (int)nseg, s);
  CUDA_TRY(cudaGetLastError());
  if (planes_host) CUDA_TRY(cudaMemcpyAsync(planes_host, d_planes, words * B * 4, cudaMemcpyDeviceToHost, s));
  if (signs_host) CUDA_TRY(cudaMemcpyAsync(signs_host, d_signs, nseg * slot * 4, cudaMemcpyDeviceToHost, s));
  if (sign_counts_host) CUDA_TRY(cudaMemcpyAsync(sign_counts_host, d_scnt, nseg * B * 4, cudaMemcpyDeviceToHost, s));
  if (plane_nz_host) CUDA_TRY(cudaMemcpyAsync(plane_nz_host, d_nz, B * 4, cudaMemcpyDeviceToHost, s));
  if (pairs_host) CUDA_TRY(cudaMemcpyAsync(pairs_host, d_pairs, (size_t)B * B * 8, cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (vmax_host) *vmax_host = vmd;
  return PCR_OK;
} catch (const std::bad_alloc&) {
  return fail(PCR_ERR_OOM, "host allocation failed");
} catch (...) {
  return fail(PCR_ERR_INVALID_ARG, "unexpected host error");
}
