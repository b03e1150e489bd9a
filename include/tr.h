/*
 * tr.h -- C ABI of libtr, a B300 (sm_103a) transform-reduce-scan library.
 *
 * The library evaluates a fixed family of "hdc" maps -- functions written once
 * and callable from host code, device code and at compile time, the subject of
 * Mejstrik, "__host__ __device__ -- Generic programming in Cuda" (Sec. 2.3
 * "host device everything", Sec. 2.6 "Experimental relaxed constexpr" and the
 * hdc helper of Sec. 4) -- over large device arrays:
 *
 *     y_i = f(x_i)                               tr_map
 *     sum / min / max of f over the array        tr_reduce
 *     the same per segment [off[s], off[s+1])    tr_segmented_reduce
 *     inclusive prefix sums of f                 tr_scan
 *     thousands of arrays, mixed maps, one graph tr_batched_*
 *     many polynomials at many points (GEMM)     tr_vandermonde
 *
 * Conventions (all entry points):
 *   - Every pointer named d_* or documented "device" is CUDA device memory
 *     owned by the caller; the library never frees it and never allocates
 *     per call.  Host pointers (map coefficients) are read during the call
 *     only.
 *   - Work is enqueued asynchronously on exec->stream (a cudaStream_t; NULL is
 *     the legacy default stream).  No call synchronises, except tr_check.
 *   - Errors follow the paper's convention (Sec. 1.2.1 "Cuda error checking"):
 *     a status code, 0 = success.  Argument errors are detected before any
 *     launch and nothing is enqueued.  Errors found on the device are never
 *     raised with a trap (the paper's release_assert of Sec. 2.4 calls
 *     __trap(), which poisons the CUDA context); instead the kernel writes a
 *     status word into the workspace and returns, and tr_check() reports it.
 *   - The workspace is caller-owned device memory of at least the size the
 *     matching *_workspace_size() call reports, 256-byte aligned and
 *     zero-filled before its first use (tr_workspace_init, or cudaMemset to
 *     0).  Every op leaves it ready for the next op; after an op reported an
 *     error, re-initialise it.  Ops that may run concurrently need distinct
 *     workspaces.
 *   - n = 0 is valid everywhere: sums are 0, min is +inf (UINT32_MAX for u32),
 *     max is -inf (0 for u32), scans and maps write nothing.
 */
#ifndef TR_H
#define TR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum tr_status {
  TR_OK = 0,
  TR_ERR_INVALID_ARG = 1,   /* null pointer, negative size, bad enum, overlap */
  TR_ERR_ALIGNMENT = 2,     /* a pointer not aligned to its element size */
  TR_ERR_UNSUPPORTED = 3,   /* (dtype, map, op) combination not provided */
  TR_ERR_WORKSPACE = 4,     /* workspace missing or smaller than required */
  TR_ERR_CUDA = 5,          /* a CUDA runtime call failed (see tr_last_error) */
  TR_ERR_TIMEOUT = 6,       /* a bounded device-side wait ran out */
  TR_ERR_DEVICE_ASSERT = 7  /* a device-side input check failed (e.g. offsets) */
} tr_status;

typedef enum tr_dtype {
  TR_F16 = 0,
  TR_BF16 = 1,
  TR_F32 = 2,
  TR_F64 = 3,
  TR_U32 = 4,
  TR_U64 = 5,
  TR_NONE = 15
} tr_dtype;

/* The map family.  Float maps compute in FP32 for f16/bf16/f32 storage and in
 * FP64 for f64 storage; the integer mixers take u32. */
typedef enum tr_map_kind {
  TR_MAP_IDENTITY = 0,    /* f(x) = x                                        */
  TR_MAP_SQUARE = 1,      /* f(x) = x * x                                    */
  TR_MAP_HORNER = 2,      /* p(x) = c_d; p = fma(p, x, c_k), k = d-1..0       */
  TR_MAP_RATIONAL = 3,    /* P(x) / Q(x), each by Horner, one IEEE division   */
  TR_MAP_NEWTON_CBRT = 4, /* y0 = sign(x); y <- (2y + x/(y*y))/3, iters times */
  TR_MAP_XORSHIFT32 = 5,  /* x^=x<<13; x^=x>>17; x^=x<<5 (Marsaglia 2003)     */
  TR_MAP_SPLITMIX32 = 6   /* z=x+0x9E3779B9; z=(z^z>>16)*0x6A09E667;
                             z=(z^z>>13)*0xBB67AE85; z^=z>>16 (mod 2^32)      */
} tr_map_kind;

#define TR_MAX_DEGREE 31

/* A map of the family.  coef_p / coef_q: host arrays of deg+1 FP64
 * coefficients in ascending powers (c_0 first); copied at the call and rounded
 * to FP32 for FP32-compute paths.  deg_p, deg_q in [0, TR_MAX_DEGREE]; unused
 * fields are ignored.  iters in [0, 64] for TR_MAP_NEWTON_CBRT. */
typedef struct tr_map_desc {
  int32_t kind; /* tr_map_kind */
  int32_t deg_p;
  int32_t deg_q;
  int32_t iters;
  const double* coef_p;
  const double* coef_q;
} tr_map_desc;

enum { TR_SUM = 1, TR_MIN = 2, TR_MAX = 4 };

/* Execution context of one call. */
typedef struct tr_exec {
  void* stream;            /* cudaStream_t, NULL = legacy default stream */
  void* workspace;         /* device memory, see conventions above */
  size_t workspace_bytes;
  uint32_t wait_timeout_us;  /* bound on each device-side wait; 0 = 1,000,000 */
  int32_t reserved;
  int64_t debug_stall_tile;  /* scan only, for fault tests: the tile with this
                                id never publishes its prefix, so its
                                successors' waits run out; -1 = off */
} tr_exec;

/* ---- status and workspace ------------------------------------------------ */

/* Static text for a status code. */
const char* tr_status_string(tr_status s);

/* Text describing the last failing call on this host thread ("" if none). */
const char* tr_last_error(void);

/* Number of kernels this library has enqueued in this process so far: one per
 * kernel launch, the kernels of a graph each time the graph is launched
 * (launches recorded during a stream capture count when recorded).  A
 * relaxed atomic counter, for counting the kernels of a timed region. */
uint64_t tr_launch_count(void);

/* Zero-fill a workspace (cudaMemsetAsync on stream). */
tr_status tr_workspace_init(void* d_workspace, size_t bytes, void* stream);

/* Synchronise exec->stream, then read and clear the device status word in
 * exec->workspace -- the host side of the paper's error convention (Sec. 1.2.1
 * "Cuda error checking") for errors a kernel found (Sec. 2.4's release_assert
 * reports instead of trapping here).  Returns TR_ERR_CUDA if the stream reported an error,
 * otherwise the first device-side error recorded since the last tr_check
 * (TR_ERR_TIMEOUT, TR_ERR_DEVICE_ASSERT) or TR_OK. */
tr_status tr_check(const tr_exec* exec);

/* ---- map ------------------------------------------------------------------ */

/* y_i = f(x_i), i < n: the map family of tr_map_kind, written once as hdc
 * functions (the paper's Sec. 2.3 "host device everything" and Sec. 2.6) and
 * evaluated on the device with the same operation sequence as on the host.
 * xt: F16/BF16/F32 (FP32 compute), F64 (FP64 compute) or
 * U32 (mixers and identity).  yt is the compute type: F32 for FP32 compute,
 * F64 for F64, U32 for U32.  y may equal x when xt == yt; partial overlap is
 * an error.  Needs no workspace (exec->workspace may be NULL).  Pointers must
 * be aligned to their element size; 16-byte aligned x and y take the 128-bit
 * vector path. */
tr_status tr_map(const tr_map_desc* map, const void* d_x, tr_dtype xt, void* d_y, tr_dtype yt, int64_t n,
                 const tr_exec* exec);

/* ---- full reduction ------------------------------------------------------ */

tr_status tr_reduce_workspace_size(int64_t n, tr_dtype xt, size_t* bytes);

/* sum / min / max of f(x_i), i < n, selected by ops (TR_SUM|TR_MIN|TR_MAX) -- the
 * plain transform-reduce (e.g. 2^20 FP64 values through a degree-8 Horner
 * polynomial, or 2^30 FP16-stored values with FP32 compute); compensated sums
 * (Kahan 1965) combined with error-free additions (Knuth's TwoSum).
 * Results are written to DEVICE memory (one element each):
 *   FP32 compute: per-thread compensated (Kahan) sums of pairwise vector sums,
 *                 float-float warp/block combination, FP64 across blocks;
 *                 sum_t F32 or F64; min/max F32.
 *   FP64 compute: FP64 sums; sum_t F64; min/max F64.
 *   U32 mixers:   exact sum_t U64 (or U32 modulo 2^32); min/max U32.
 * min/max ignore NaN (IEEE minNum/maxNum).  Deterministic for a given
 * (n, device): the combination order is fixed. */
tr_status tr_reduce(const tr_map_desc* map, const void* d_x, tr_dtype xt, int64_t n, unsigned ops, void* d_sum,
                    tr_dtype sum_t, void* d_min, void* d_max, const tr_exec* exec);

/* ---- segmented reduction -------------------------------------------------- */

tr_status tr_segmented_reduce_workspace_size(int64_t n, int64_t n_seg, tr_dtype xt, size_t* bytes);

/* The segmented transform-reduce (e.g. 2^28 FP32 values through a rational
 * map of degree 6/6 into 65,536 segments).
 * For each segment s < n_seg, elements [d_offsets[s], d_offsets[s+1]) of x:
 * sum / min / max of f into d_sums[s], d_mins[s], d_maxs[s] (device arrays).
 * d_offsets: n_seg + 1 int64 device values, offsets[0] = 0,
 * offsets[n_seg] = n, non-decreasing; empty segments get the identities.
 * Offsets that violate this are reported as TR_ERR_DEVICE_ASSERT by tr_check
 * (results are then unspecified).  xt: F16, BF16, F32 (FP32 compute with
 * compensated sums, FP64 combination of segment pieces); sum_t F32 or F64;
 * mins/maxs F32.  Deterministic for a given (n, device). */
tr_status tr_segmented_reduce(const tr_map_desc* map, const void* d_x, tr_dtype xt, int64_t n,
                              const int64_t* d_offsets, int64_t n_seg, unsigned ops, void* d_sums, tr_dtype sum_t,
                              void* d_mins, void* d_maxs, const tr_exec* exec);

/* tr_segmented_reduce from and to host memory, for callers whose data lives
 * on the host: copies h_x (n elements of xt) and h_offsets (n_seg + 1 int64)
 * into the caller's device buffers d_x and d_offsets, runs
 * tr_segmented_reduce on them into the caller's device result buffers d_sums /
 * d_mins / d_maxs, and copies the selected results back into h_sums / h_mins /
 * h_maxs.  Every step is enqueued on exec->stream (cudaMemcpyAsync: page-locked
 * host buffers make the copies asynchronous; pageable ones are staged by the
 * driver); the host results are valid after the stream is synchronised (e.g.
 * by tr_check).  Arguments and errors as for tr_segmented_reduce; NULL
 * buffers for selected outputs are TR_ERR_INVALID_ARG. */
tr_status tr_segmented_reduce_host(const tr_map_desc* map, const void* h_x, tr_dtype xt, int64_t n,
                                   const int64_t* h_offsets, int64_t n_seg, unsigned ops, void* h_sums,
                                   tr_dtype sum_t, void* h_mins, void* h_maxs, void* d_x, int64_t* d_offsets,
                                   void* d_sums, void* d_mins, void* d_maxs, const tr_exec* exec);

/* ---- inclusive scan ------------------------------------------------------- */

tr_status tr_scan_workspace_size(int64_t n, tr_dtype xt, tr_dtype yt, size_t* bytes);

/* The inclusive scan of f (e.g. 2^28 u32 through splitmix32 modulo 2^32, or
 * 2^28 f32 of x^2 with compensated sums):
 * y_i = f(x_0) + ... + f(x_i), single pass with decoupled look-back between
 * tiles (Merrill & Garland, "Single-pass parallel prefix scan with decoupled
 * look-back", NVIDIA NVR-2016-002).  Supported (xt -> yt):
 *   U32 -> U32  modulo 2^32 (bit exact)
 *   U32 -> U64  exact
 *   F16/BF16/F32 -> F32  float-float within and between tiles, each output
 *                 rounded once from the compensated prefix.
 * d_carry_in (nullable, device, one element of yt's type) is added to every
 * output.  y may equal x when the element sizes match.  4-byte inputs and
 * outputs on 16-byte aligned arrays move through the TMA engine; the
 * workspace holds one 128-byte look-back line per tile of 8,192 elements.
 * Each look-back wait
 * is bounded by exec->wait_timeout_us; on expiry tr_check returns
 * TR_ERR_TIMEOUT and the output is unspecified.  Float scans may differ in
 * the last bit between runs (where the look-back stops depends on timing). */
tr_status tr_scan(const tr_map_desc* map, const void* d_x, tr_dtype xt, void* d_y, tr_dtype yt, int64_t n,
                  const void* d_carry_in, const tr_exec* exec);

/* ---- scan with reduction, exclusive scan ------------------------------------- */

enum { TR_SCAN_INCLUSIVE = 0, TR_SCAN_EXCLUSIVE = 1 };

/* tr_scan in either mode, plus, from the same single read of x, the sum, min
 * and max of f over the whole array (ops: a mask of TR_SUM|TR_MIN|TR_MAX, 0 for
 * none).  mode TR_SCAN_EXCLUSIVE writes y_0 = carry (or 0) and
 * y_i = carry + f(x_0) + ... + f(x_{i-1}); TR_SCAN_INCLUSIVE is tr_scan.
 * Results of the reduction (device memory, one element each) do not include
 * the carry-in:
 *   U32 -> U32:   sum_t U32 (modulo 2^32);  U32 -> U64: sum_t U64 (exact);
 *   float scans:  sum_t F64 (the scan's float-float total of the tiles'
 *                 compensated sums, rounded once) or F32;  min / max: F32 for
 *                 float input, U32 for u32, ignoring NaN; for n = 0 the
 *                 identities.
 * The sum equals the last inclusive output when there is no carry-in (bit for
 * bit for integers).  Same workspace as tr_scan; dtypes, carry, in-place and
 * timeout rules as tr_scan.  The last tile writes the sum; min / max are
 * folded once per block and written by the last block to finish. */
tr_status tr_scan_reduce(const tr_map_desc* map, const void* d_x, tr_dtype xt, void* d_y, tr_dtype yt, int64_t n,
                         int mode, const void* d_carry_in, unsigned ops, void* d_sum, tr_dtype sum_t, void* d_min,
                         void* d_max, const tr_exec* exec);

/* ---- batched reduction ------------------------------------------------------ */

typedef struct tr_batch_plan tr_batch_plan; /* opaque, owned by the library */

/* Plan the reduction of n_arrays independent device arrays of storage type xt
 * (F32, F16 or BF16; FP32 compute), each with its own map (Horner, rational,
 * Newton cube root, square, identity), in ONE persistent kernel launch
 * replayed from a CUDA graph -- the batched workload (e.g. 10,000 arrays with
 * lengths log-uniform in [1, 2^20] and mixed maps), with an autotuned launch
 * shape.
 *   d_xs[i]   (host array of device pointers) array i, lens[i] elements,
 *             aligned to the element size
 *   maps[i]   its map (host descriptors, copied)
 *   d_sums / d_mins / d_maxs  device arrays of n_arrays F64 / F32 / F32
 *             (those selected by ops must be non-NULL)
 * Each array is cut into work items; warps pull items from an atomic queue
 * (costliest first), reduce them with compensated FP32 sums, and the warp that
 * finishes an array's last item joins its partials in FP64 in item order, so
 * results are bitwise deterministic.  autotune != 0 times the launch shapes
 * -- item size T in {8K, 16K, 32K, 64K}, 128 or 256 threads, items equal in
 * elements or balanced by map cost, 4 or 2 16-byte vectors in flight per lane
 * (fewer registers, more resident warps) -- on this data (it writes the outputs and
 * synchronises the device; TR_AUTOTUNE_CACHE names an optional cache file);
 * 0 takes a fixed default.  Plan creation allocates the plan's device buffers
 * and instantiates the graph; the arrays and outputs must stay valid while
 * the plan is used. */
tr_status tr_batched_plan_create(int64_t n_arrays, const void* const* d_xs, const int64_t* lens,
                                 const tr_map_desc* maps, tr_dtype xt, unsigned ops, double* d_sums, float* d_mins,
                                 float* d_maxs, int autotune, void* stream, tr_batch_plan** out);

/* Launch the plan's graph on stream (one cudaGraphLaunch).  Runs of one plan
 * must not overlap on the GPU. */
tr_status tr_batched_run(tr_batch_plan* plan, void* stream);

/* The unbatched baseline: the same results with one tr_reduce launch per
 * array; use_graph != 0 records those launches into a graph on first use and
 * replays it.  Allocates the baseline's workspace on first use. */
tr_status tr_batched_run_unbatched(tr_batch_plan* plan, int use_graph, void* stream);

/* Text describing the chosen tile, block size, grid and item count. */
const char* tr_batched_plan_describe(const tr_batch_plan* plan);

tr_status tr_batched_plan_destroy(tr_batch_plan* plan);

/* ---- dense Vandermonde product ---------------------------------------------- */

enum { TR_PREC_BF16X3 = 0, TR_PREC_FP32 = 1, TR_PREC_BF16X6 = 2 };

/* Workspace of tr_vandermonde for npoly polynomials: a status header and the
 * per-column partial results of the tensor path. */
tr_status tr_vandermonde_workspace_size(int64_t m, int64_t npoly, size_t* bytes);

/* Many polynomials at many points (the dense workload, e.g. 4096 polynomials
 * of degree 31 at 2^20 points), as a Vandermonde product on the tensor cores:
 * Y = V(x) C, Y[i][j] = sum_k C[k][j] x_i^k, written out and/or reduced per
 * column (polynomial j) over the points.
 *   d_x     m FP32 points;  d_coef (deg+1) x npoly FP32, row-major, row k
 *           holding the power-k coefficients of all polynomials (deg <= 31);
 *   d_y     m x npoly row-major in yt: TR_F32, TR_BF16 (rounded to nearest
 *           even from the FP32 result) or TR_NONE (not written; d_y ignored);
 *   d_colsum / d_colmin / d_colmax (each nullable, npoly FP32, device): sum,
 *           minimum and maximum of column j over the m points, taken from the
 *           FP32 results in the same pass (partials combined in FP64 in a
 *           fixed order: deterministic).
 * precision
 *   TR_PREC_BF16X3 / TR_PREC_BF16X6: split-BF16 on the tcgen05 tensor cores
 *     (Henry, Tang & Heinecke, ARITH 2019): powers and coefficients are split
 *     into 2 (x3: V1C1 + V1C2 + V2C1) or 3 (x6: all products of parts whose
 *     orders sum to at most 2) bf16 parts, accumulated in FP32 in tensor
 *     memory; V is generated on the fly from x.  Error, normwise against
 *     S[i][j] = sum_k |C[k][j]| |x_i|^k: about 2e-5 (x3), 1e-6 (x6).  Any m;
 *     FP32 output needs npoly % 4 == 0, BF16 output npoly % 8 == 0, and a
 *     16-byte aligned d_y; TR_NONE output any npoly.  Needs a workspace of
 *     tr_vandermonde_workspace_size() bytes (its status word reports a
 *     device-side timeout through tr_check).  Two launches when a column
 *     result is requested, one otherwise.
 *   TR_PREC_FP32: FP32 Horner with fma on the CUDA cores (the comparison);
 *     FP32 output only, no column results, any m and npoly, no workspace.
 * Rows of C beyond deg are treated as zero.  Nothing requested (TR_NONE and
 * no column output) is TR_ERR_INVALID_ARG. */
tr_status tr_vandermonde(const float* d_x, int64_t m, const float* d_coef, int32_t deg, int64_t npoly,
                         int precision, void* d_y, tr_dtype yt, float* d_colsum, float* d_colmin, float* d_colmax,
                         const tr_exec* exec);

/* ---- inclusive scan without a workspace -------------------------------------- */

/* The scan of tr_scan (same dtypes, maps, arithmetic and results) for callers
 * that cannot allocate device memory -- for example code running inside a
 * memory allocator, plugins handed only input and output pointers, or loops
 * that must not allocate once started -- and so cannot provide a workspace.
 * The paper has no counterpart to this entry point.
 *
 * The scratch lives in one fixed device array inside the library (about
 * 1 MiB, reserved on every GPU that loads the library and held until the
 * process exits), so n is limited to 2^26 elements; larger n is rejected with
 * TR_ERR_INVALID_ARG and a message naming the limit.  The call makes no
 * allocation of any kind.  Its first call on a device looks up the array's
 * device address for that device; make that first call before any stream
 * capture.  Every call shares the one array, so calls that may overlap on the
 * GPU (other streams, other host threads) race and must be serialised by the
 * caller.  The error words of the array are cleared at the start of each call.
 * d_status (nullable, device, one uint32) receives the device-side status of
 * this call: 0, or TR_ERR_TIMEOUT if a look-back wait ran out (1 s bound).
 * stream: cudaStream_t, NULL = legacy default stream. */
tr_status tr_scan_noalloc(const tr_map_desc* map, const void* d_x, tr_dtype xt, void* d_y, tr_dtype yt, int64_t n,
                          const void* d_carry_in, uint32_t* d_status, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* TR_H */
