// Internal types shared by the CUDA kernels (pcr_kernels.cu) and the host
// library (pcr_host.cpp).  Not part of the ABI.
#pragma once
#include <cstdint>
#include <string>

namespace pcr {

constexpr int kWord = 32;          // elements per plane word
constexpr int kSegElems = 4096;    // elements per sign segment / encode CTA
constexpr int kSegWords = kSegElems / kWord;
// Fixed point of levels >= 1: x_int = floor(x 2^(F - G)), max |x| < 2^G,
// with F = fix_bits(value kind, L): 40 for FP32 fields; for FP64 fields 48,
// fewer for deep hierarchies (56 - L) so that every reconstruction
// numerator keeps int64 headroom (values <= 4.2 (Lam^d)^L 2^F, numerators
// <= 20 times that, Lam^d <= 1.953).
constexpr int kFixBitsF32 = 40;
inline int fix_bits(int vk, int L) {
  if (vk != 1) return kFixBitsF32;
  return 56 - L < 48 ? 56 - L : 48;
}
constexpr int kMaxLat = 3;

enum ValueKind { VK_F32 = 0, VK_F64 = 1, VK_FIX = 2 };

// One lattice of a stream: field coordinates start + step * k, k < count,
// row-major with every row (fixed k0, k1) padded to row_pad elements.
struct LatD {
  int64_t start[3], step[3], count[3];
  int64_t row_pad;
  int64_t base;        // padded element offset of this lattice in its stream
};

// Field description for the coefficient kernels.
struct FieldD {
  int64_t n[3];        // 3-D shape (2-D fields: n[0] = 1)
  int64_t nc[3];       // shape of the 2-grid (fixed-point copy of the coarse points)
  int order[3];        // pass order over active axes (d entries)
  int d;               // number of active axes
  int interp;          // 0 per-level, 1 per-region
  int degree;          // 1 linear, 3 cubic
  int L;
  int fixb;            // fixed-point fraction bits F (see fix_bits)
};

// Per-stream device descriptor; holds raw device pointers so kernels can run
// over work lists that mix streams of different handles (batched forms).
struct StreamD {
  int nlat;
  LatD lat[kMaxLat];
  int64_t n_pad, words, nseg;
  int level, region, sub, is_fix;
  int B, enc;          // planes; 1 generic, 2 negabinary
  int vk;              // value kind of the staged values (ValueKind)
  int slot_words;      // sign slot capacity (u32) per segment
  uint32_t* planes;    // [B][words]
  uint32_t* signs;     // [nseg][slot_words]
  uint32_t* sign_counts;   // [nseg][B]
  uint32_t* plane_nz;      // [2B]: nonzero words per plane, then sign words per plane
  unsigned long long* pairs; // [B][B] (PSNR mode) or nullptr
  unsigned long long* vmax;  // max |value| (float bits / double bits / u64)
  void* stage;         // staged values, padded canonical order
  int b;               // planes to decode (retrieval)
  int E;               // float streams: exponent; fixed: bit length e
  int sh;              // fixed streams: quantisation shift
};

// coefficient decomposition of one region (Sec. V-B): in-slice axes u, v and
// the sub-level (1 = raw 4-grid, 2 = 2-grid, 3 = full grid)
struct DecompGeo {
  LatD region;
  int u, v;
  int sub;
};

// one region of a level in level-grid coordinates, with the staging it
// writes (refactor: coefficients) or reads (retrieve: decoded coefficients)
struct TileRegion {
  int64_t start[3], step[3], count[3];
  int64_t row_pad;     // padded row length, or count[2] for compact arrays
  int64_t base;        // element offset of the region's lattice in `stage`
  void* stage;
  unsigned long long* vmax;   // refactor: stream maximum slot (may be null)
  int vmax_double;            // 1: the slot holds the bits of a double (field statistics' max |c|)
};

struct FieldStats;

// arguments of the tiled interpolation kernel (one level, all regions)
struct TileArgs {
  int64_t m[3];        // level-grid lengths (1 along an inactive axis)
  int64_t stride[3];   // element strides of src / dst per level-grid step
  int64_t ntiles[3];
  int d;
  int order[3];
  int interp, degree;
  int retrieve;
  const void* src;     // refactor: field (level 0) or fixed-point 2-grid copy
  void* dst;           // retrieve: same view as src
  TileRegion reg[3];
  // box retrieval: level-grid box [blo, bhi) whose values must be exact
  // (bhi[0] == 0: the whole grid); set by the host
  int64_t blo[3], bhi[3];
  // set by the launchers: first tile per axis (plane-marching: first plane)
  int64_t tlo[3];
  // refactor of level 0: the field's statistics (min, max, finiteness),
  // taken by the plane-marching kernel as it reads the field, else by a
  // separate pass the launcher adds (null: not wanted)
  FieldStats* stats;
  // set to 1 when a bounded device wait gives up (refactor: the field's
  // timeout flag; null: the library's device status word)
  int* err;
  // whole-field retrieval of level 0: the coarse points (the 2-grid) come
  // from the fixed-point copy cfix (x_int, shape ((m - 1) / 2 + 1) per axis,
  // row-major), each value x_int * cscale rounded once.  The marching kernel
  // reads its ring there and writes those points with its planes; the other
  // paths first write them into the output.  Null: the output holds them.
  const int64_t* cfix;
  double cscale;
};

// items of one batched (multi-field) launch of the per-field kernels
constexpr int kMaxBatchItems = 128;

// one task: stream, plane, segment (plane rows of `words` words, segments of
// kSegWords words, the last one possibly shorter)
struct PackTask {
  uint32_t* plane;         // the plane's row (read by the packer, written by the unpacker)
  int64_t words;           // words in the row
  int seg;
};

// a range of 32-bit words to zero (src null) or copy, one item of a batched
// launch
struct WordsItem {
  uint32_t* dst;
  const uint32_t* src;
  int64_t words;
};

#ifdef __CUDACC__
// item of a batched launch that owns this block: the last i < n with
// first[i] <= blockIdx.x (first[] ascending, first[0] = 0)
__device__ __forceinline__ int batch_find(const int64_t* first, int n) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= (int64_t)blockIdx.x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
#endif

// independent tile-kernel launches fused into one (the refactor's levels
// >= 1, or one level of several fields); first[i]: first block of args[i]
constexpr int kMaxTileBatch = 54;
struct TileBatch {
  int n;
  int64_t first[kMaxTileBatch + 1];
  TileArgs args[kMaxTileBatch];
};

// one sub-level lattice part of a decomposed region, in the region's compact
// coordinates, with its padded stream staging
struct DecompSub {
  int64_t start[3], step[3], count[3];
  int64_t row_pad, base;
  void* stage;
  unsigned long long* vmax;
};

struct DecompArgs {
  int64_t cnt[3];      // compact region dims
  int64_t ntiles[3];
  int u, v, n;         // in-slice axes and slice normal
  int retrieve;        // 0 decompose, 1 recompose
  void* comp;          // region compact array (c, or recomposed c_hat)
  DecompSub subs[5];   // S1, S2a, S2b, S3a, S3b
  // recompose of a box of the compact array [blo, bhi) (bhi[0] == 0: all);
  // first block per axis set by the launcher
  int64_t blo[3], bhi[3], tlo[3];
  unsigned long long* c0;  // decompose: running max |c| (bits of a double)
  int* err;                // set to 1 when a bounded device wait gives up (may be null)
  int64_t pitch;           // elements per compact row (0: cnt[2]); forward decomposition only
};

// an index box: points lo + [0, cnt) per axis
struct Box3 {
  int64_t lo[3], cnt[3];
};

struct WorkItem {
  int stream;          // index into the StreamD array of the launch
  int seg;
};

// Device statistics of one field.
struct FieldStats {
  unsigned long long xmin_key, xmax_key;   // order-preserving keys of doubles
  unsigned long long c0;                   // max |c| at level 0 (double bits)
  int G;                                   // max|x| < 2^G
  int bad;                                 // non-finite input seen
  int timeout;                             // a bounded device wait gave up
};

#ifdef __CUDACC__
// fixed-point value -> value type (v * scale, scale a power of two)
template <typename T> __device__ __forceinline__ T from_fix(int64_t v, T scale);
template <> __device__ __forceinline__ float from_fix<float>(int64_t v, float scale) {
  return __fmul_rn(__ll2float_rn(v), scale);
}
template <> __device__ __forceinline__ double from_fix<double>(int64_t v, double scale) {
  return __dmul_rn(__ll2double_rn(v), scale);
}

// order-preserving key of a double (unsigned comparison = numeric order)
__device__ __forceinline__ unsigned long long dkey(double x) {
  unsigned long long u = __double_as_longlong(x);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

// a block's minimum, maximum and non-finite flag merged into the field's
// statistics; every thread of the block calls it
__device__ __forceinline__ void stats_push_block(FieldStats* st, double lo, double hi, int bad) {
  __shared__ unsigned long long rlo[32], rhi[32];
  __shared__ int rbad;
  unsigned long long klo = dkey(lo), khi = dkey(hi);
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    const unsigned long long a = __shfl_xor_sync(0xFFFFFFFFu, klo, o), b = __shfl_xor_sync(0xFFFFFFFFu, khi, o);
    klo = a < klo ? a : klo;
    khi = b > khi ? b : khi;
  }
  bad = __any_sync(0xFFFFFFFFu, bad);
  if (threadIdx.x == 0) rbad = 0;
  __syncthreads();
  if ((threadIdx.x & 31) == 0) {
    rlo[threadIdx.x >> 5] = klo;
    rhi[threadIdx.x >> 5] = khi;
    if (bad) rbad = 1;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    const int nw = blockDim.x >> 5;
    klo = threadIdx.x < nw ? rlo[threadIdx.x] : ~0ull;
    khi = threadIdx.x < nw ? rhi[threadIdx.x] : 0ull;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
      const unsigned long long a = __shfl_xor_sync(0xFFFFFFFFu, klo, o), b = __shfl_xor_sync(0xFFFFFFFFu, khi, o);
      klo = a < klo ? a : klo;
      khi = b > khi ? b : khi;
    }
    if (threadIdx.x == 0) {
      atomicMin(&st->xmin_key, klo);
      atomicMax(&st->xmax_key, khi);
      if (rbad) st->bad = 1;
    }
  }
}
#endif

// Device address of the library's fixed scratch array on the current device
// (looked up once per device with cudaGetSymbolAddress); nullptr and a
// reason on failure.  *cap receives its size in bytes.
void* static_scratch(size_t* cap, std::string* why);

// kernels launched by this library since load (tracing); every launcher
// increments it right before its <<<...>>>
void count_launch();
long long launch_count();
void add_launches(long long n);
// autotuner of the level-interpolation schedule (pcr_tiles.cu)
int set_autotune(int on);   // returns the previous setting
bool autotune_pin(const int64_t* key, int choice);   // false: unknown key field or choice
// bounded waits of retrieval kernels that gave up on the current device
// since the last clear (-1: the read failed); clear resets the count
int read_device_timeouts(bool clear);
// out[2-grid] = x_int * scale rounded once, over the whole 2-grid or a box
// of it (pcr_kernels.cu)
void launch_coarse_out(int vk, const FieldD& f, const int64_t* xc, double scale, void* out, cudaStream_t s,
                       const Box3* box = nullptr);
int autotune_entries(int max_entries, int64_t* keys, int* choice, double* ms);
void clear_autotune();

}  // namespace pcr
