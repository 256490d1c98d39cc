/*
 * pcr.h -- C ABI of the B300 progressive refactor / retrieve library.
 *
 * The library implements the data-parallel path of the adaptive progressive
 * compressor of arXiv 2609.04573 ("ProAICD"): a 2-D or 3-D FP32/FP64 field is
 * refactored into hierarchical coefficients by multilevel interpolation
 * (per-level or per-region, linear or cubic; Sec. IV), the finest level's
 * coefficients are further decomposed by 2-D per-level linear interpolation
 * of each slice (Sec. V-B, Algorithm 1), and every stream is quantised and
 * split into bitplanes with per-plane error tables (Sec. V-C).  Retrieval picks
 * the planes that provably meet a max-abs-error or PSNR target (Sec. III-A,
 * V-C) and reconstructs the field from them (Algorithm 2).
 *
 * Conventions shared by every entry point
 *   - Status codes only: no exceptions cross the ABI, nothing aborts, no
 *     device trap.  pcr_last_error() gives a thread-local message for the last
 *     non-OK status of the calling thread.
 *   - Device pointers are CUDA device addresses on the current device; the
 *     caller owns them and must keep them alive until the work enqueued on
 *     `cuda_stream` (a cudaStream_t, NULL = legacy default stream) completes.
 *   - A pcr_handle owns its device buffers (allocated through the caller's
 *     pcr_allocator, or cudaMallocAsync when that pointer is NULL) and its host
 *     tables; pcr_free releases both.  Handles are immutable after
 *     pcr_refactor / pcr_deserialize, so several threads may plan and retrieve
 *     from one handle concurrently, each on its own stream.
 *   - Fields are row-major (C order, last axis fastest).  ndim is 2 or 3 and
 *     every dimension must be >= 2.
 */
#ifndef PCR_H
#define PCR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  PCR_OK = 0,
  PCR_ERR_INVALID_ARG = 1,   /* bad pointer, size, enum or combination      */
  PCR_ERR_UNSUPPORTED = 2,   /* valid request outside what is implemented   */
  PCR_ERR_OOM = 3,           /* the allocator returned NULL                 */
  PCR_ERR_CUDA = 4,          /* a CUDA runtime call failed (message given)  */
  PCR_ERR_TIMEOUT = 5,       /* a bounded device wait gave up               */
  PCR_ERR_UNSATISFIABLE = 6, /* even all planes cannot meet the target      */
  PCR_ERR_CORRUPT = 7        /* container failed length / checksum checks   */
} pcr_status;

enum { PCR_F32 = 0, PCR_F64 = 1 };
enum { PCR_MODE_EB = 0, PCR_MODE_PSNR = 1, PCR_MODE_EXPLICIT = 2 };
enum { PCR_INTERP_AUTO = -1, PCR_INTERP_LEVEL = 0, PCR_INTERP_REGION = 1 };
enum { PCR_LINEAR = 1, PCR_CUBIC = 3 };
enum { PCR_ENC_DEFAULT = 0, PCR_ENC_GENERIC = 1, PCR_ENC_NEGABINARY = 2 };
enum { PCR_TARGET_ABS = 0, PCR_TARGET_REL = 1, PCR_TARGET_PSNR = 2 };

#define PCR_MAX_STREAMS 64

/* Device memory provider.  alloc(ctx, bytes, stream) returns a device pointer
 * usable in stream order on `stream` (NULL on failure -> PCR_ERR_OOM);
 * free(ctx, p, stream) returns it.  Pass NULL for cudaMallocAsync/FreeAsync. */
typedef struct {
  void* ctx;
  void* (*alloc)(void* ctx, size_t bytes, void* stream);
  void (*free)(void* ctx, void* p, void* stream);
} pcr_allocator;

/* Refactoring scheme (Sec. IV-VI; tuning table of Sec. VI-A).
 *   mode        PCR_MODE_EB: error-bound mode, L-inf tables only (sq tables
 *               are the L-inf bound times the count);
 *               PCR_MODE_PSNR: also exact integer squared-error tables;
 *               PCR_MODE_EXPLICIT: every field taken as given, exact integer
 *               squared-error tables kept, so the handle serves error-bound
 *               and PSNR targets alike (encoding default: generic).
 *   interp      per-level (pass order = natural axis order) or per-region;
 *               PCR_INTERP_AUTO: the target-driven tuner (pcr_tune, Sec. VI-A)
 *               picks interp, order, decomposition axis and encoding for the
 *               mode (EB or PSNR) from a sample of the field, then the field
 *               is refactored with that choice (pcr_get_scheme reads it).
 *   degree      PCR_LINEAR or PCR_CUBIC.
 *   order       per-region pass order: a permutation of the field's axes
 *               (3-D: of 0,1,2; 2-D: of 0,1 in order[0..1]); ignored per-level.
 *   decomp_axis slice normal (0..2) of the level-0 coefficient decomposition
 *               (Sec. V-B), or -1 for none; 3-D only.
 *   encoding    PCR_ENC_DEFAULT picks negabinary+XOR for PSNR, generic otherwise.
 *   nlevels     L (0 = auto: coarsest grid keeps >= 3 points per axis).
 *   nplanes     B (0 = auto: 32 for FP32, 64 for FP64; otherwise 1..B_auto). */
typedef struct {
  int mode;
  int interp;
  int degree;
  int order[3];
  int decomp_axis;
  int encoding;
  int nlevels;
  int nplanes;
} pcr_scheme;

/* Retrieval target (Sec. III-A): PCR_TARGET_ABS max|x - x'| <= value;
 * PCR_TARGET_REL max|x - x'| <= value * (max x - min x);
 * PCR_TARGET_PSNR 20 log10((max x - min x) / RMSE) >= value (dB).
 * has_box != 0 asks for the box [lo, hi) of the field only (user axes,
 * 0 <= lo < hi <= dims; entries past ndim are ignored): the plan is the
 * whole field's (its L-inf bound holds at every point, so inside the box;
 * a PSNR target is planned on the whole field) and the output holds the
 * box, row-major. */
typedef struct {
  int kind;
  double value;
  int has_box;
  int64_t lo[3], hi[3];
} pcr_target;

/* A retrieval plan: how many planes of every stream to read (host data). */
typedef struct {
  int nstreams;
  int planes[PCR_MAX_STREAMS];
  double bound;       /* a-priori L-inf bound (ABS/REL) or SSE bound (PSNR) */
  double psnr_bound;  /* PSNR implied by the SSE bound (PSNR targets)       */
  uint64_t bytes;     /* payload bytes read: plane words + sign words       */
  int satisfied;      /* 1 when the bound meets the target                  */
} pcr_retrieval_plan;

/* What one pcr_retrieve call read and how long it took. */
typedef struct {
  int nstreams;
  int planes[PCR_MAX_STREAMS];  /* planes read per stream                    */
  uint64_t bytes;               /* plane words + sign words read             */
  double bits_per_value;        /* 8 bytes / points of the output            */
  double bound;                 /* L-inf bound (ABS/REL) or SSE bound (PSNR) */
  double psnr_bound;            /* PSNR implied by the SSE bound (PSNR)      */
  int satisfied;                /* 1 when the bound meets the target         */
  double plan_ms;               /* host time of the interpreter              */
  double enqueue_ms;            /* host time enqueueing the GPU work         */
  int want_gpu_ms;              /* input: 1 = time the GPU work (the call
                                   then waits for it)                        */
  double gpu_ms;                /* GPU time of the call's work, -1 untimed   */
} pcr_retrieval_info;

/* Error tables of every stream (Sec. V-C).  The library fills nstreams,
 * nplanes (B) and exponent[]; maxerr / sq / bytes, when not NULL, are
 * caller arrays of nstreams * (nplanes + 1) entries, row i = stream i,
 * column b = b planes read (call once with NULL arrays to learn the sizes). */
typedef struct {
  int nstreams, nplanes;
  int exponent[PCR_MAX_STREAMS];  /* E (float streams) or bit length (fixed) */
  double* maxerr;                 /* L-inf error bound                        */
  double* sq;                     /* squared-error bound (sum over the stream)*/
  uint64_t* bytes;                /* bytes of the first b planes              */
} pcr_tables;

/* Per-stream description (tests, tools, serialisation). */
typedef struct {
  int level, region, sub;      /* sub 0 = undecomposed, 1..3 = S1..S3        */
  int is_fixed;                /* 1: 64-bit fixed point (levels >= 1)       */
  int nplanes;                 /* B                                         */
  int64_t n_real, n_pad, words;/* elements, padded elements, words / plane  */
  int64_t nseg;                /* sign segments (generic encoding)          */
  int exponent;                /* E (float streams) or bit length e (fixed) */
  int shift;                   /* fixed streams: quantisation shift sh      */
  double vmax;                 /* max |coefficient| (fixed: in quanta)      */
} pcr_stream_info;

typedef struct pcr_handle pcr_handle;

/* ---- refactor (Algorithm 1) ------------------------------------------- */
/* Refactor the device field `d_field` (dims[ndim], dtype PCR_F32/PCR_F64).
 * Enqueues all work on `cuda_stream` and synchronises it once at the end to
 * read the ~KB of tables.  On success *out owns the streams. */
pcr_status pcr_refactor(const void* d_field, int ndim, const int64_t* dims, int dtype,
                        const pcr_scheme* scheme, const pcr_allocator* alloc,
                        void* cuda_stream, pcr_handle** out);

/* ---- asynchronous refactor (pipelining of independent fields) ----------
 * begin: arguments as pcr_refactor.  Allocates the handle's buffers and
 *   scratch (stream-ordered, through `alloc`), enqueues every kernel and the
 *   small read-backs of the statistics into pinned host memory on
 *   `cuda_stream`, records an event and returns without waiting.  The field
 *   must stay unchanged at `d_field` until the job's work has run.  While a
 *   job is pending the host may plan, retrieve or begin other jobs; work
 *   enqueued later on the same stream runs after this job's kernels.
 * end: waits for the job's event, builds the host tables (Sec. V-C error
 *   tables) and returns the handle in *out (the caller owns it and frees it
 *   with pcr_free).  The job is consumed whatever the outcome.
 * job_free: abandons a job without a handle; waits for its work first.
 * The handle equals the one pcr_refactor returns for the same field.  Its
 *   buffers come from `alloc` on `cuda_stream` and go back there at
 *   pcr_free without waiting: work on other streams that reads the handle
 *   (a retrieval on a second stream) must have completed before pcr_free.
 * Errors: as pcr_refactor; PCR_ERR_OOM also when pinned host memory for the
 *   read-backs cannot be allocated. */
typedef struct pcr_refactor_job pcr_refactor_job;
pcr_status pcr_refactor_begin(const void* d_field, int ndim, const int64_t* dims, int dtype,
                              const pcr_scheme* scheme, const pcr_allocator* alloc,
                              void* cuda_stream, pcr_refactor_job** out);
pcr_status pcr_refactor_end(pcr_refactor_job* job, pcr_handle** out);
void pcr_refactor_job_free(pcr_refactor_job* job);

/* Batched form: n independent fields refactored with one work list per
 * kernel (one launch per pipeline stage for the whole batch).  Arrays are
 * length n; fields may have different shapes and dtypes. */
pcr_status pcr_refactor_batch(int n, const void* const* d_fields, const int* ndims,
                              const int64_t* const* dims, const int* dtypes,
                              const pcr_scheme* schemes, const pcr_allocator* alloc,
                              void* cuda_stream, pcr_handle** outs);

/* ---- batched refactor captured in one CUDA graph ----------------------
 * For batches refactored again and again with the same shapes (variables of
 * successive timesteps): the whole batch -- every kernel, memset and the
 * small uploads and read-backs -- is captured once into one CUDA graph and
 * each run is one graph launch plus the host finish of the tables.
 * create: arguments as pcr_refactor_batch.  The fields stay at these device
 *   addresses for the graph's lifetime; the caller refills them between
 *   runs.  Creation refactors the batch once uncaptured (with the level
 *   autotuner on, see pcr_autotune_enable, and measuring the scratch it
 *   needs), allocates one scratch arena through `alloc` and pinned host
 *   staging, captures on a stream of its own and instantiates; it
 *   synchronises `cuda_stream`.  The handles are valid after create.
 * run: launches the graph on `cuda_stream`, synchronises it and rebuilds
 *   every handle's tables from the new data.
 * handle: the k-th handle, owned by the graph (do not pcr_free it); valid
 *   until pcr_refactor_graph_free, its contents replaced by every run.
 * info: graph nodes, kernels per run, scratch arena bytes (any may be NULL).
 * times: of the last run, the graph's device time (CUDA events around the
 *   launch, ms) and the host finish of the tables (ms); zeros before the
 *   first run (either may be NULL).
 * Errors: as pcr_refactor_batch; PCR_ERR_CUDA when capture or instantiation
 *   fails. */
typedef struct pcr_refactor_graph pcr_refactor_graph;
pcr_status pcr_refactor_graph_create(int n, const void* const* d_fields, const int* ndims,
                                     const int64_t* const* dims, const int* dtypes,
                                     const pcr_scheme* schemes, const pcr_allocator* alloc,
                                     void* cuda_stream, pcr_refactor_graph** out);
pcr_status pcr_refactor_graph_run(pcr_refactor_graph* g, void* cuda_stream);
pcr_status pcr_refactor_graph_handle(const pcr_refactor_graph* g, int k, const pcr_handle** out);
pcr_status pcr_refactor_graph_info(const pcr_refactor_graph* g, int64_t* nodes, int64_t* kernels,
                                   int64_t* arena_bytes);
pcr_status pcr_refactor_graph_times(const pcr_refactor_graph* g, double* gpu_ms, double* host_ms);
void pcr_refactor_graph_free(pcr_refactor_graph* g);

/* ---- autotuner of the level-interpolation schedule (GPU tuning;
 * the paper tunes its interpolation choices, Sec. VI-A, but not GPU tiles) -
 * Where a level can run either the general tile kernel or the plane-marching
 * kernel, and the marching kernel's plane chunk sets its grid, all choices
 * compute identical values.  enable(1): the first launch of an untuned
 * (value kind, direction, degree, level grid) on a stream that is not being
 * captured times every candidate with CUDA events and keeps the fastest;
 * later launches use the table (enable(0) keeps using it without adding).
 * read: up to max_entries entries, keys = 7 int64 per entry (value kind
 * PCR-internal 0 f32 / 1 f64 / 2 fixed point, retrieve 0/1, degree,
 * interpolation 0 per-level / 1 per-region, level grid lengths m0, m1, m2),
 * choice (0 general tile kernel, -1 marching with the default chunk and
 * register prefetch, -2 marching with the default chunk and its inputs
 * staged by TMA copies where that form applies (register prefetch
 * elsewhere; the schedule of untuned levels), -3 the same on 16 x 64
 * columns instead of 16 x 128 (FP32 levels; -2 for other value kinds), k > 0
 * marching with k-plane chunks), ms (the winner's time); *n_out = entries
 * in the table; reset clears it afterwards. */
pcr_status pcr_autotune_enable(int enable);
/* Device status of the current device: *timeouts = 1 when a bounded wait
 * of a retrieval kernel (TMA-staged level-0 reconstruction) gave up since
 * the last clear -- the tiles of that CTA were left unwritten -- else 0;
 * clear != 0 resets it.  Synchronous (waits for the device's pending work
 * to read it).  pcr_retrieve with want_gpu_ms set checks and clears it
 * itself and returns PCR_ERR_TIMEOUT.  Refactor waits report through the
 * refactor's own status. */
pcr_status pcr_device_status(int* timeouts, int clear);
/* Pin one schedule: `key` = the 7 int64 of an entry (as pcr_autotune_read
 * gives them), `choice` one of the candidates (0, 8, 16, 32, 64, -1, -2, -3);
 * every later launch of that level grid uses it (a level the marching
 * kernel cannot take runs the general tile kernel whatever the choice).
 * PCR_ERR_INVALID_ARG for an unknown key field or choice. */
pcr_status pcr_autotune_set(const int64_t* key, int choice);
pcr_status pcr_autotune_read(int max_entries, int64_t* keys, int* choice, double* ms, int* n_out, int reset);

/* ---- target-driven sampled tuning (Sec. VI-A and its tuning table) ----
 * Picks the scheme of `mode` (PCR_MODE_EB: per-level or per-region with each
 * of the d! pass orders, decomposition off or along each axis, generic
 * planes; PCR_MODE_PSNR: per-region only, negabinary + XOR; cubic) for the
 * device field: whole blocks of min(edge, n)^d points sampled on a regular
 * grid (at most `fraction` of the field, at least one block; 0 = defaults
 * 0.01 and 64) are refactored with every candidate; at each of the 9
 * tolerances tau = 1e-3, 5e-4, 1e-4, .., 1e-7 (relative to the field's
 * range R) the candidate needing the fewest bytes gets a vote (EB: max error
 * tau R in every block; PSNR: squared-error sum n_block (tau R)^2, i.e.
 * RMSE tau R); most votes wins, ties to the earlier candidate.  Synchronises
 * `cuda_stream`; temporary memory through `alloc`.  info (nullable) receives
 * the candidates, votes and byte counts (UINT64_MAX: tolerance not met). */
#define PCR_TUNE_NTOL 9
#define PCR_TUNE_MAX_CANDIDATES 32
typedef struct {
  int ncand, winner;
  pcr_scheme cand[PCR_TUNE_MAX_CANDIDATES];
  int votes[PCR_TUNE_MAX_CANDIDATES];
  uint64_t bytes[PCR_TUNE_MAX_CANDIDATES][PCR_TUNE_NTOL];
  int nblocks;
  int64_t block[3];      /* block edge per field axis (ndim entries) */
  double fraction;       /* sampled points / field points */
  double ms;             /* wall time of the call */
} pcr_tune_info;
pcr_status pcr_tune(const void* d_field, int ndim, const int64_t* dims, int dtype, int mode, double fraction,
                    int edge, const pcr_allocator* alloc, void* cuda_stream, pcr_scheme* out,
                    pcr_tune_info* info);
/* The scheme a handle was refactored with (the tuner's choice for
 * PCR_INTERP_AUTO requests). */
pcr_status pcr_get_scheme(const pcr_handle* h, pcr_scheme* out);

/* ---- plan (retrieval interpreter, Sec. V-C / VI-B) -------------------- */
/* Host only.  Greedy selection of planes meeting `target`; returns
 * PCR_ERR_UNSATISFIABLE (plan still filled with all planes) when the bound
 * with every plane exceeds the target. */
pcr_status pcr_plan(const pcr_handle* h, const pcr_target* target, pcr_retrieval_plan* out);
/* Incremental invocation (progressive refinement, Sec. III-A: a retrieval
 * refines an earlier one and re-uses the planes it fetched): plan `target`
 * starting from `have` (a plan of this handle whose planes the caller
 * holds).  The result contains `have` stream by stream; the greedy steps
 * are ranked by the bytes they add beyond `have`, and steps whose planes
 * `have` already holds are passed over.  out->bytes is the whole plan's
 * size; the bytes to fetch are out->bytes - have->bytes.  From an empty
 * plan it equals pcr_plan.  Errors: as pcr_plan; PCR_ERR_INVALID_ARG when
 * `have` does not match the handle (stream count, plane counts). */
pcr_status pcr_plan_more(const pcr_handle* h, const pcr_target* target, const pcr_retrieval_plan* have,
                         pcr_retrieval_plan* out);

/* Best-first search interpreter (Sec. VI-B: per-level + decomposition is
 * planned by a best-first search with pruning and incremental invocation,
 * per-region by a dynamic program; both seek the fewest bytes whose bound
 * meets the target).  One search serves every mode: over the greedy's
 * planning units (the steps pcr_plan takes), a state is the number of steps
 * taken per unit and costs the bytes it adds to `have`.  The greedy plan is
 * the first incumbent; each unit starts at the fewest steps that meet the
 * target with every other unit complete; states are expanded cheapest
 * first (ties: the earlier pushed), each reached once (a child advances
 * units at or after the one its parent advanced); a child meeting the
 * target replaces a dearer incumbent; children costing at least the
 * incumbent are cut.  The search ends when the cheapest open state costs at
 * least the incumbent (the plan is then the minimum over unit positions:
 * info->optimal = 1) or after `max_nodes` expansions (the best plan found).
 * The plan never costs more than pcr_plan's (pcr_plan_more's with `have`).
 * have: NULL or a plan of this handle whose planes the caller holds (as
 * pcr_plan_more).  info (may be NULL): expansions, whether the minimum was
 * proved, the greedy's bytes beyond `have`, host milliseconds.  Errors: as
 * pcr_plan_more; PCR_ERR_INVALID_ARG for max_nodes < 0; host memory grows
 * with the budget (about 2 U^2 bytes per expansion for U planning units;
 * PCR_ERR_OOM when it cannot be had). */
typedef struct {
  int64_t expanded;       /* states expanded                                 */
  int optimal;            /* 1 when the plan is proved the minimum           */
  uint64_t greedy_bytes;  /* bytes the greedy plan adds beyond `have`        */
  double plan_ms;         /* host time of the search                         */
} pcr_search_info;
pcr_status pcr_plan_search(const pcr_handle* h, const pcr_target* target, const pcr_retrieval_plan* have,
                           int64_t max_nodes, pcr_retrieval_plan* out, pcr_search_info* info);

/* ---- block sharding of one field (Sec. VII: independent blocks) -------
 * A field split along axis 0 into slabs, each refactored as a field of its
 * own (on this GPU or on the ranks that hold them), retrieved for one
 * whole-field target:
 * plan_global: plans[k] for hs[k] (n blocks of one field).  abs / rel
 *   targets: relative to the whole field's range (max of the blocks'
 *   maxima minus min of their minima); every block planned by pcr_plan for
 *   that absolute tolerance; *bound = the largest block bound.  PSNR: one
 *   budget N (R 10^(-psnr/20))^2 of squared errors (N points in all
 *   blocks) spent by one greedy over every block's planning units (the step
 *   with the largest decrease of its own block's L2 bound per byte; ties to
 *   the earlier block, then the earlier unit); *bound = the blocks' summed
 *   bound, plans[k].bound each block's.  One block gives its pcr_plan.
 *   Errors: as pcr_plan (PCR_ERR_UNSATISFIABLE: some block cannot meet its
 *   share even with every plane; the plans are still filled).
 * export_plan_state: what the planner needs of a handle (statistics and
 *   per-stream tables, no planes) as a host buffer (free with
 *   pcr_buffer_free) that another process can import.
 * import_plan_state: a planning-only handle from such a buffer: it plans
 *   (pcr_plan, pcr_plan_more, pcr_plan_global) but holds no planes, so
 *   retrievals, stream copies and pcr_serialize return PCR_ERR_UNSUPPORTED.
 *   PCR_ERR_CORRUPT on a bad magic, length or checksum. */
/* ---- lossless coding of plane words (Sec. V: bitplane encoding then
 * lossless compression) -------------------------------------------------
 * Every plane of every 4096-value segment of a stream is coded on its own:
 * nothing when it has no one-bit, else the Rice code of the zero runs
 * before its ones (parameter k the largest value <= 15 with m 2^k <= n - m,
 * m ones in n bits), else -- when that code is not shorter -- the raw words;
 * one header word per segment and plane (mode, k, m, payload words).
 * Planes with no nonzero word in a stream are not stored.
 * packed_tables: bytes[i * (B + 1) + b] = stored bytes of stream i's first
 *   b planes coded (plus their sign words, as in the raw tables); computed
 *   on the GPU on first use (synchronises the device's default stream).
 * serialize_packed: a container like pcr_serialize with the planes stored
 *   coded; pcr_deserialize reads both kinds (it decodes the planes on the
 *   GPU; a header out of range or a code that does not decode into its
 *   segment is PCR_ERR_CORRUPT).
 * Planning-only handles: PCR_ERR_UNSUPPORTED. */
pcr_status pcr_packed_tables(const pcr_handle* h, uint64_t* bytes);
/* Test entry: the coded form of one segment's plane (nwords <= 128 words at
 * d_words in device memory): *header and the payload words (room for 128)
 * into host memory, *npayload their count. */
pcr_status pcr_debug_pack(const uint32_t* d_words, int nwords, uint32_t* header, uint32_t* payload, int* npayload);
pcr_status pcr_serialize_packed(const pcr_handle* h, void** buf, size_t* len);

pcr_status pcr_plan_global(int n, const pcr_handle* const* hs, const pcr_target* target,
                           pcr_retrieval_plan* plans, double* bound, int* satisfied);
pcr_status pcr_export_plan_state(const pcr_handle* h, void** buf, size_t* len);
pcr_status pcr_import_plan_state(const void* buf, size_t len, pcr_handle** out);

/* ---- retrieve (Algorithm 2) ------------------------------------------- */
/* One call: plan `target` (as pcr_plan) and reconstruct into the caller's
 * device buffer `d_out` (the field's shape and dtype, or the box's when
 * target->has_box).  Returns after enqueueing, unless info->want_gpu_ms is
 * set (then it waits for the work and reports its GPU time).  `info` may be
 * NULL.  PCR_ERR_UNSATISFIABLE: even every plane cannot meet the target;
 * nothing is enqueued and info (bound, planes = all) is still filled. */
pcr_status pcr_retrieve(const pcr_handle* h, const pcr_target* target, void* d_out, void* cuda_stream,
                        pcr_retrieval_info* info);

/* Decode the planes of `plan` (from pcr_plan on the same handle, or any
 * plane counts 0..B), recompose and reconstruct into `d_out` (same shape
 * and dtype as the refactored field).  Returns after enqueueing. */
pcr_status pcr_retrieve_plan(const pcr_handle* h, const pcr_retrieval_plan* plan, void* d_out,
                             void* cuda_stream);

/* Batched retrieval: n (handle, target, output) triples planned one by one
 * and retrieved with one work list per stage (whole-field targets only;
 * box targets go through pcr_retrieve).  infos: n entries or NULL. */
pcr_status pcr_retrieve_batch(int n, const pcr_handle* const* hs, const pcr_target* targets,
                              void* const* d_outs, void* cuda_stream, pcr_retrieval_info* infos);

/* The same with plans given (the serving loop plans on its own). */
pcr_status pcr_retrieve_batch_plan(int n, const pcr_handle* const* hs, const pcr_retrieval_plan* plans,
                                   void* const* d_outs, void* cuda_stream);

/* Retrieval of a box [lo, hi) of the field (user axes, 0 <= lo < hi <= dims)
 * under `plan` (from pcr_plan: the bound holds at every point, so inside the
 * box too).  d_out: device buffer of the box, row-major, prod(hi - lo)
 * values of the field dtype.  Returns exactly the box of what
 * pcr_retrieve_plan with the same plan returns.  A point at level l depends on the coarser
 * grid and on level l's coefficients within 3 * 2^l field points per axis
 * (Alg. 2's rules), so only the stream segments meeting the box's
 * dependency region are decoded and only the tiles meeting it are
 * reconstructed.  Temporary device memory as pcr_retrieve plus one field.
 * Enqueue only; errors: PCR_ERR_INVALID_ARG for a box outside the field. */
pcr_status pcr_retrieve_box(const pcr_handle* h, const pcr_retrieval_plan* plan, const int64_t* lo,
                            const int64_t* hi, void* d_out, void* cuda_stream);

/* Upper bound on the temporary device memory one retrieval of `h` takes
 * (staging, work lists, recomposition); used for memory-based admission. */
pcr_status pcr_retrieve_scratch_bytes(const pcr_handle* h, size_t* bytes);

/* ---- retrieval without device allocation -------------------------------- */
/* Same plans, same kernels and the same output as pcr_retrieve_plan, for callers
 * that must not allocate device memory: applications whose own pool or arena
 * owns all device memory, hosts that forbid libraries to allocate on their
 * behalf, and latency-bound loops where cudaMalloc / cudaFree would
 * synchronise the device.  Every temporary buffer of the call is carved out
 * of one fixed 32 MiB array compiled into the library
 * (PCR_STATIC_SCRATCH_BYTES); each GPU that loads the library holds that
 * array until the process exits.  Nothing is allocated: no cudaMalloc /
 * cudaMallocAsync / cudaFree and no call to the handle's allocator.  Every
 * byte of the array that a call reads is written earlier in the same call,
 * so nothing needs clearing between calls.
 *   - A retrieval needing more scratch than the array holds returns
 *     PCR_ERR_UNSUPPORTED with the required size in pcr_last_error() (with
 *     FP32 and coefficient decomposition the limit is about 3.5 M points).
 *   - The current device must be the one the handle was created on
 *     (PCR_ERR_INVALID_ARG otherwise): the array is per device.
 *   - The first call on a device looks the array's device address up with
 *     cudaGetSymbolAddress (device-wide set-up): make that first call on each
 *     device before any stream capture begins.
 *   - The call copies its per-call stream descriptors (and, for a handle from
 *     pcr_deserialize, its work list) from host memory that lives only for
 *     the call, so a stream that is being captured is refused with
 *     PCR_ERR_UNSUPPORTED.
 *   - All calls share the one array, so calls that can run at the same time
 *     on the GPU (different streams, or host threads without ordering) race
 *     and corrupt each other; calls enqueued on one stream are ordered.
 * The paper has no counterpart: this is an interface for such callers. */
#define PCR_STATIC_SCRATCH_BYTES (32u << 20)
pcr_status pcr_retrieve_static(const pcr_handle* h, const pcr_retrieval_plan* plan, void* d_out,
                               void* cuda_stream);

/* ---- introspection / persistence -------------------------------------- */
pcr_status pcr_num_streams(const pcr_handle* h, int* n);
pcr_status pcr_stream_info_get(const pcr_handle* h, int i, pcr_stream_info* out);
/* Error tables of every stream at once (see pcr_tables). */
pcr_status pcr_get_tables(const pcr_handle* h, pcr_tables* out);
/* Error tables of stream i: maxerr[B+1], sq[B+1] (FP64) and bytes[B+1]. */
pcr_status pcr_stream_tables(const pcr_handle* h, int i, double* maxerr, double* sq,
                             uint64_t* bytes);
/* Field statistics: min, max, fixed-point exponent G (max|x| < 2^G). */
pcr_status pcr_field_stats(const pcr_handle* h, double* xmin, double* xmax, int* G);
/* Copy stream i's plane words ([B][words] u32) and sign area to host. */
pcr_status pcr_stream_copy(const pcr_handle* h, int i, uint32_t* planes_host,
                           uint32_t* signs_host, uint32_t* sign_counts_host,
                           uint64_t* pairs_host);
/* Max-ordering segment errors of a per-level decomposed level 0 (M_0 of
 * Algorithm 1); *n receives the count (0 when not applicable), errs may be
 * NULL to query the count. */
pcr_status pcr_max_ordering(const pcr_handle* h, double* errs, int* n);
/* Container: header + tables + stream directory + payload, CRC32 per
 * section.  *buf is malloc'ed; release with pcr_buffer_free. */
pcr_status pcr_serialize(const pcr_handle* h, void** buf, size_t* len);
pcr_status pcr_deserialize(const void* buf, size_t len, const pcr_allocator* alloc,
                           void* cuda_stream, pcr_handle** out);
void pcr_buffer_free(void* buf);
void pcr_free(pcr_handle* h);
const char* pcr_last_error(void);

/* ---- tracing ------------------------------------------------------------ */
/* enable != 0: every pipeline stage enqueued afterwards records a pair of
 * CUDA events on its stream.  pcr_profile_read synchronises the recorded
 * events and returns, per stage name (48-byte NUL-terminated slots of
 * `names`), the summed milliseconds and kernel launches; *n_out receives the
 * number of stages (entries beyond max_entries are counted, not written);
 * reset != 0 clears the totals.  Not for use inside stream capture. */
pcr_status pcr_profile_enable(int enable);
pcr_status pcr_profile_read(int max_entries, char* names, double* ms, int64_t* launches, int* n_out,
                            int reset);
/* Kernels this library has launched since it was loaded (all threads). */
int64_t pcr_launch_count(void);

/* ---- test entry: encode given coefficients ---------------------------- */
/* Encode one stream of n_pad values already in canonical padded order
 * (`d_vals`: float, double or int64 fixed point per `value_kind` 0/1/2)
 * with B planes and `encoding`; writes plane words [B][n_pad/32], the sign
 * area, sign counts, plane nonzero-word counts and (want_pairs) plane pair
 * counts to host arrays.  Lets tests feed the oracle's own coefficients. */
pcr_status pcr_debug_encode(const void* d_vals, int64_t n_pad, int value_kind, int B,
                            int encoding, int want_pairs, void* cuda_stream,
                            uint32_t* planes_host, uint32_t* signs_host,
                            uint32_t* sign_counts_host, uint32_t* plane_nz_host,
                            uint64_t* pairs_host, double* vmax_host);

#ifdef __cplusplus
}
#endif
#endif /* PCR_H */
