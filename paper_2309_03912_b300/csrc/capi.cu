// capi.cu -- the extern "C" boundary of libtr: argument validation, map
// descriptors, workspace sizing, status reporting; dispatch to the launchers.
#include <atomic>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <unordered_map>

#include "internal.h"

namespace tr {

static thread_local char g_last_error[512] = "";
static std::atomic<unsigned long long> g_launches{0};

void count_launches(unsigned long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

tr_status fail(tr_status s, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
  va_end(ap);
  return s;
}

tr_status cuda_status(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return TR_OK;
  return fail(TR_ERR_CUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

const DevInfo& dev_info() {
  static std::mutex mu;
  static std::unordered_map<int, DevInfo> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  DevInfo d;
  d.device = dev;
  cudaDeviceGetAttribute(&d.sm_count, cudaDevAttrMultiProcessorCount, dev);
  cudaDeviceGetAttribute(&d.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (d.sm_count <= 0) d.sm_count = 1;
  return cache.emplace(dev, d).first->second;
}

namespace {
struct KernelKey {
  int device;
  const void* kernel;
  int threads;
  size_t bytes;
  bool operator<(const KernelKey& o) const {
    if (device != o.device) return device < o.device;
    if (kernel != o.kernel) return kernel < o.kernel;
    if (threads != o.threads) return threads < o.threads;
    return bytes < o.bytes;
  }
};
}  // namespace

int blocks_per_sm(const void* kernel, int threads, size_t dyn_smem) {
  static std::mutex mu;
  static std::map<KernelKey, int> cache;
  const KernelKey key{dev_info().device, kernel, threads, dyn_smem};
  std::lock_guard<std::mutex> lk(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int b = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, dyn_smem) != cudaSuccess || b < 1) b = 1;
  cache[key] = b;
  return b;
}

tr_status ensure_dyn_smem(const void* kernel, int bytes, const char* what) {
  static std::mutex mu;
  static std::set<KernelKey> done;
  const KernelKey key{dev_info().device, kernel, 0, (size_t)bytes};
  std::lock_guard<std::mutex> lk(mu);
  if (done.count(key)) return TR_OK;
  tr_status s = cuda_status(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes), what);
  if (s == TR_OK) done.insert(key);
  return s;
}

tr_status make_tensor_map_2d(CUtensorMap* out, const void* base, CUtensorMapDataType type, uint64_t inner,
                             uint64_t rows, uint64_t row_bytes, uint32_t box_inner, uint32_t box_rows,
                             CUtensorMapSwizzle swizzle) {
  typedef CUresult (*EncodeFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                               const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                               CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  static EncodeFn fn = nullptr;
  static std::mutex mu;
  {
    std::lock_guard<std::mutex> lk(mu);
    if (!fn) {
      void* p = nullptr;
      cudaDriverEntryPointQueryResult q;
      if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
          q != cudaDriverEntryPointSuccess || !p)
        return fail(TR_ERR_CUDA, "cuTensorMapEncodeTiled is not available");
      fn = reinterpret_cast<EncodeFn>(p);
    }
  }
  const cuuint64_t dims[2] = {inner, rows};
  const cuuint64_t strides[1] = {row_bytes};
  const cuuint32_t box[2] = {box_inner, box_rows};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r = fn(out, type, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(TR_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
  return TR_OK;
}

size_t dtype_size(tr_dtype t) {
  switch (t) {
    case TR_F16:
    case TR_BF16: return 2;
    case TR_F32:
    case TR_U32: return 4;
    case TR_F64:
    case TR_U64: return 8;
    default: return 0;
  }
}

tr_status make_map_params(const tr_map_desc* d, bool int_input, MapParams* P) {
  if (!d) return fail(TR_ERR_INVALID_ARG, "map descriptor is NULL");
  std::memset(P, 0, sizeof(*P));
  if (d->kind < TR_MAP_IDENTITY || d->kind > TR_MAP_SPLITMIX32) return fail(TR_ERR_INVALID_ARG, "unknown map kind %d", d->kind);
  P->kind = d->kind;
  const bool int_map = d->kind == TR_MAP_XORSHIFT32 || d->kind == TR_MAP_SPLITMIX32;
  if (int_input && !(int_map || d->kind == TR_MAP_IDENTITY))
    return fail(TR_ERR_UNSUPPORTED, "map kind %d needs float input", d->kind);
  if (!int_input && int_map) return fail(TR_ERR_UNSUPPORTED, "integer mixer %d needs u32 input", d->kind);
  if (d->kind == TR_MAP_HORNER || d->kind == TR_MAP_RATIONAL) {
    if (d->deg_p < 0 || d->deg_p > TR_MAX_DEGREE || !d->coef_p)
      return fail(TR_ERR_INVALID_ARG, "numerator degree %d or coefficients invalid", d->deg_p);
    P->deg_p = d->deg_p;
    for (int k = 0; k <= d->deg_p; ++k) {
      P->dp[k] = d->coef_p[k];
      P->fp[k] = (float)d->coef_p[k];
    }
  }
  if (d->kind == TR_MAP_RATIONAL) {
    if (d->deg_q < 0 || d->deg_q > TR_MAX_DEGREE || !d->coef_q)
      return fail(TR_ERR_INVALID_ARG, "denominator degree %d or coefficients invalid", d->deg_q);
    P->deg_q = d->deg_q;
    for (int k = 0; k <= d->deg_q; ++k) {
      P->dq[k] = d->coef_q[k];
      P->fq[k] = (float)d->coef_q[k];
    }
  }
  if (d->kind == TR_MAP_NEWTON_CBRT) {
    if (d->iters < 0 || d->iters > 64) return fail(TR_ERR_INVALID_ARG, "newton iterations %d out of [0, 64]", d->iters);
    P->iters = d->iters;
  }
  return TR_OK;
}

static bool is_float_storage(tr_dtype t) { return t == TR_F16 || t == TR_BF16 || t == TR_F32; }

static tr_status check_exec(const tr_exec* e, size_t need, bool ws_required) {
  if (!e) return fail(TR_ERR_INVALID_ARG, "exec is NULL");
  if (ws_required) {
    if (!e->workspace) return fail(TR_ERR_WORKSPACE, "workspace is NULL (need %zu bytes)", need);
    if (e->workspace_bytes < need)
      return fail(TR_ERR_WORKSPACE, "workspace has %zu bytes, need %zu", e->workspace_bytes, need);
    if (!aligned_to(e->workspace, 256)) return fail(TR_ERR_ALIGNMENT, "workspace must be 256-byte aligned");
  }
  return TR_OK;
}

static tr_status check_ptr(const void* p, tr_dtype t, int64_t n, const char* name) {
  if (n > 0 && !p) return fail(TR_ERR_INVALID_ARG, "%s is NULL", name);
  if (p && !aligned_to(p, dtype_size(t))) return fail(TR_ERR_ALIGNMENT, "%s is not aligned to its element size", name);
  return TR_OK;
}

// [a, a + an) and [b, b + bn) overlap without being identical
static bool partial_overlap(const void* a, size_t an, const void* b, size_t bn) {
  const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
  if (x == y && an == bn) return false;
  return x < y + bn && y < x + an;
}

}  // namespace tr

using namespace tr;

extern "C" {

const char* tr_status_string(tr_status s) {
  switch (s) {
    case TR_OK: return "TR_OK";
    case TR_ERR_INVALID_ARG: return "TR_ERR_INVALID_ARG: invalid argument";
    case TR_ERR_ALIGNMENT: return "TR_ERR_ALIGNMENT: misaligned pointer";
    case TR_ERR_UNSUPPORTED: return "TR_ERR_UNSUPPORTED: unsupported dtype/map/op combination";
    case TR_ERR_WORKSPACE: return "TR_ERR_WORKSPACE: workspace missing or too small";
    case TR_ERR_CUDA: return "TR_ERR_CUDA: CUDA runtime error";
    case TR_ERR_TIMEOUT: return "TR_ERR_TIMEOUT: a bounded device-side wait ran out";
    case TR_ERR_DEVICE_ASSERT: return "TR_ERR_DEVICE_ASSERT: device-side input check failed";
  }
  return "unknown tr_status";
}

const char* tr_last_error(void) { return g_last_error; }

uint64_t tr_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

tr_status tr_workspace_init(void* ws, size_t bytes, void* stream) {
  if (!ws && bytes) return fail(TR_ERR_INVALID_ARG, "workspace is NULL");
  if (!bytes) return TR_OK;
  return cuda_status(cudaMemsetAsync(ws, 0, bytes, static_cast<cudaStream_t>(stream)), "cudaMemsetAsync(workspace)");
}

tr_status tr_check(const tr_exec* e) {
  if (!e) return fail(TR_ERR_INVALID_ARG, "exec is NULL");
  tr_status st = cuda_status(cudaStreamSynchronize(stream_of(e)), "cudaStreamSynchronize");
  if (st != TR_OK) return st;
  if (!e->workspace || e->workspace_bytes < sizeof(WsHeader)) return TR_OK;
  uint32_t h[3] = {0, 0, 0};
  st = cuda_status(cudaMemcpy(h, e->workspace, sizeof(h), cudaMemcpyDeviceToHost), "cudaMemcpy(status)");
  if (st != TR_OK) return st;
  if (h[0] != 0) {
    static const uint32_t zero[3] = {0, 0, 0};
    cudaMemcpy(e->workspace, zero, sizeof(zero), cudaMemcpyHostToDevice);
    return fail((tr_status)h[0], "device reported %s (detail %u)", tr_status_string((tr_status)h[0]), h[1]);
  }
  return TR_OK;
}

tr_status tr_map(const tr_map_desc* map, const void* x, tr_dtype xt, void* y, tr_dtype yt, int64_t n,
                 const tr_exec* e) {
  MapParams P;
  if (n < 0) return fail(TR_ERR_INVALID_ARG, "n < 0");
  tr_status s = make_map_params(map, xt == TR_U32, &P);
  if (s) return s;
  if ((s = check_exec(e, 0, false))) return s;
  if (!(is_float_storage(xt) || xt == TR_F64 || xt == TR_U32)) return fail(TR_ERR_UNSUPPORTED, "map input dtype %d", xt);
  const tr_dtype want = is_float_storage(xt) ? TR_F32 : xt;
  if (yt != want) return fail(TR_ERR_UNSUPPORTED, "map output dtype must be the compute type (%d)", want);
  if ((s = check_ptr(x, xt, n, "x")) || (s = check_ptr(y, yt, n, "y"))) return s;
  if (partial_overlap(x, n * dtype_size(xt), y, n * dtype_size(yt)))
    return fail(TR_ERR_INVALID_ARG, "x and y overlap partially");
  if (n == 0) return TR_OK;
  return launch_map(P, x, xt, y, n, e);
}

tr_status tr_reduce_workspace_size(int64_t n, tr_dtype xt, size_t* bytes) {
  if (!bytes || n < 0) return fail(TR_ERR_INVALID_ARG, "bad arguments");
  *bytes = reduce_ws_bytes(n, xt);
  return TR_OK;
}

tr_status tr_reduce(const tr_map_desc* map, const void* x, tr_dtype xt, int64_t n, unsigned ops, void* sum,
                    tr_dtype sum_t, void* mn, void* mx, const tr_exec* e) {
  MapParams P;
  if (n < 0) return fail(TR_ERR_INVALID_ARG, "n < 0");
  if (ops == 0 || (ops & ~7u)) return fail(TR_ERR_INVALID_ARG, "ops must be a non-empty mask of TR_SUM|TR_MIN|TR_MAX");
  tr_status s = make_map_params(map, xt == TR_U32, &P);
  if (s) return s;
  if (!(is_float_storage(xt) || xt == TR_F64 || xt == TR_U32)) return fail(TR_ERR_UNSUPPORTED, "reduce input dtype %d", xt);
  if (ops & TR_SUM) {
    const bool ok = xt == TR_U32 ? (sum_t == TR_U64 || sum_t == TR_U32)
                                 : (xt == TR_F64 ? sum_t == TR_F64 : (sum_t == TR_F32 || sum_t == TR_F64));
    if (!ok) return fail(TR_ERR_UNSUPPORTED, "sum dtype %d for input dtype %d", sum_t, xt);
    if (!sum) return fail(TR_ERR_INVALID_ARG, "sum output is NULL");
    if ((s = check_ptr(sum, sum_t, 1, "sum"))) return s;
  }
  const tr_dtype mt = xt == TR_U32 ? TR_U32 : (xt == TR_F64 ? TR_F64 : TR_F32);
  if ((ops & TR_MIN) && ((s = check_ptr(mn, mt, 1, "min")))) return s;
  if ((ops & TR_MAX) && ((s = check_ptr(mx, mt, 1, "max")))) return s;
  if ((s = check_ptr(x, xt, n, "x"))) return s;
  if ((s = check_exec(e, reduce_ws_bytes(n, xt), true))) return s;
  return launch_reduce(P, x, xt, n, ops, sum, sum_t, mn, mx, e);
}

tr_status tr_segmented_reduce_workspace_size(int64_t n, int64_t n_seg, tr_dtype xt, size_t* bytes) {
  if (!bytes || n < 0 || n_seg < 0) return fail(TR_ERR_INVALID_ARG, "bad arguments");
  *bytes = segreduce_ws_bytes(n, n_seg, xt);
  return TR_OK;
}

tr_status tr_segmented_reduce(const tr_map_desc* map, const void* x, tr_dtype xt, int64_t n, const int64_t* off,
                              int64_t n_seg, unsigned ops, void* sums, tr_dtype sum_t, void* mins, void* maxs,
                              const tr_exec* e) {
  MapParams P;
  if (n < 0 || n_seg < 0) return fail(TR_ERR_INVALID_ARG, "n < 0 or n_seg < 0");
  if (n_seg >= (int64_t(1) << 40) || n >= (int64_t(1) << 40)) return fail(TR_ERR_INVALID_ARG, "size too large");
  if (ops == 0 || (ops & ~7u)) return fail(TR_ERR_INVALID_ARG, "ops must be a non-empty mask of TR_SUM|TR_MIN|TR_MAX");
  tr_status s = make_map_params(map, false, &P);
  if (s) return s;
  if (!is_float_storage(xt)) return fail(TR_ERR_UNSUPPORTED, "segmented reduce input dtype %d", xt);
  if ((ops & TR_SUM) && !(sum_t == TR_F32 || sum_t == TR_F64)) return fail(TR_ERR_UNSUPPORTED, "sum dtype %d", sum_t);
  if (!off) return fail(TR_ERR_INVALID_ARG, "offsets are NULL");
  if ((s = check_ptr(off, TR_U64, n_seg + 1, "offsets"))) return s;
  if ((ops & TR_SUM) && ((s = check_ptr(sums, sum_t, n_seg, "sums")))) return s;
  if ((ops & TR_MIN) && ((s = check_ptr(mins, TR_F32, n_seg, "mins")))) return s;
  if ((ops & TR_MAX) && ((s = check_ptr(maxs, TR_F32, n_seg, "maxs")))) return s;
  if ((s = check_ptr(x, xt, n, "x"))) return s;
  if ((s = check_exec(e, segreduce_ws_bytes(n, n_seg, xt), true))) return s;
  if (n_seg == 0) return TR_OK;
  return launch_segreduce(P, x, xt, n, off, n_seg, ops, sums, sum_t, mins, maxs, e);
}

tr_status tr_segmented_reduce_host(const tr_map_desc* map, const void* h_x, tr_dtype xt, int64_t n,
                                   const int64_t* h_off, int64_t n_seg, unsigned ops, void* h_sums, tr_dtype sum_t,
                                   void* h_mins, void* h_maxs, void* d_x, int64_t* d_off, void* d_sums, void* d_mins,
                                   void* d_maxs, const tr_exec* e) {
  if (n < 0 || n_seg < 0) return fail(TR_ERR_INVALID_ARG, "n < 0 or n_seg < 0");
  if (!e) return fail(TR_ERR_INVALID_ARG, "exec is NULL");
  if ((n > 0 && (!h_x || !d_x)) || !h_off || !d_off) return fail(TR_ERR_INVALID_ARG, "input buffer is NULL");
  const size_t xs = dtype_size(xt), ss = dtype_size(sum_t);
  if (!xs) return fail(TR_ERR_UNSUPPORTED, "storage dtype %d", xt);
  if ((ops & TR_SUM) && (!h_sums || !d_sums || !ss)) return fail(TR_ERR_INVALID_ARG, "sum buffers or dtype invalid");
  if ((ops & TR_MIN) && (!h_mins || !d_mins)) return fail(TR_ERR_INVALID_ARG, "min buffers are NULL");
  if ((ops & TR_MAX) && (!h_maxs || !d_maxs)) return fail(TR_ERR_INVALID_ARG, "max buffers are NULL");
  cudaStream_t st = stream_of(e);
  tr_status s = TR_OK;
  if (n > 0) s = cuda_status(cudaMemcpyAsync(d_x, h_x, (size_t)n * xs, cudaMemcpyHostToDevice, st), "copy x");
  if (!s) s = cuda_status(cudaMemcpyAsync(d_off, h_off, (size_t)(n_seg + 1) * 8, cudaMemcpyHostToDevice, st),
                          "copy offsets");
  if (!s) s = tr_segmented_reduce(map, d_x, xt, n, d_off, n_seg, ops, d_sums, sum_t, d_mins, d_maxs, e);
  if (s) return s;
  if (ops & TR_SUM)
    s = cuda_status(cudaMemcpyAsync(h_sums, d_sums, (size_t)n_seg * ss, cudaMemcpyDeviceToHost, st), "copy sums");
  if (!s && (ops & TR_MIN))
    s = cuda_status(cudaMemcpyAsync(h_mins, d_mins, (size_t)n_seg * 4, cudaMemcpyDeviceToHost, st), "copy mins");
  if (!s && (ops & TR_MAX))
    s = cuda_status(cudaMemcpyAsync(h_maxs, d_maxs, (size_t)n_seg * 4, cudaMemcpyDeviceToHost, st), "copy maxs");
  return s;
}

tr_status tr_scan_workspace_size(int64_t n, tr_dtype xt, tr_dtype yt, size_t* bytes) {
  if (!bytes || n < 0) return fail(TR_ERR_INVALID_ARG, "bad arguments");
  *bytes = scan_ws_bytes(n, xt, yt);
  return TR_OK;
}

tr_status tr_scan(const tr_map_desc* map, const void* x, tr_dtype xt, void* y, tr_dtype yt, int64_t n,
                  const void* carry, const tr_exec* e) {
  MapParams P;
  if (n < 0) return fail(TR_ERR_INVALID_ARG, "n < 0");
  if (n >= (int64_t(1) << 40)) return fail(TR_ERR_INVALID_ARG, "n too large");
  tr_status s = make_map_params(map, xt == TR_U32, &P);
  if (s) return s;
  const bool ok = (xt == TR_U32 && (yt == TR_U32 || yt == TR_U64)) || (is_float_storage(xt) && yt == TR_F32);
  if (!ok) return fail(TR_ERR_UNSUPPORTED, "scan %d -> %d", xt, yt);
  if ((s = check_ptr(x, xt, n, "x")) || (s = check_ptr(y, yt, n, "y"))) return s;
  if (carry && !aligned_to(carry, dtype_size(yt))) return fail(TR_ERR_ALIGNMENT, "carry_in misaligned");
  if (partial_overlap(x, n * dtype_size(xt), y, n * dtype_size(yt)))
    return fail(TR_ERR_INVALID_ARG, "x and y overlap partially");
  if (x == y && n > 0 && dtype_size(xt) != dtype_size(yt))
    return fail(TR_ERR_INVALID_ARG, "in-place scan needs equal element sizes");
  if ((s = check_exec(e, scan_ws_bytes(n, xt, yt), true))) return s;
  if (n == 0) return TR_OK;
  return launch_scan(P, x, xt, y, yt, n, carry, e);
}

tr_status tr_scan_reduce(const tr_map_desc* map, const void* x, tr_dtype xt, void* y, tr_dtype yt, int64_t n,
                         int mode, const void* carry, unsigned ops, void* sum, tr_dtype sum_t, void* mn, void* mx,
                         const tr_exec* e) {
  MapParams P;
  if (n < 0) return fail(TR_ERR_INVALID_ARG, "n < 0");
  if (n >= (int64_t(1) << 40)) return fail(TR_ERR_INVALID_ARG, "n too large");
  if (mode != TR_SCAN_INCLUSIVE && mode != TR_SCAN_EXCLUSIVE) return fail(TR_ERR_INVALID_ARG, "scan mode %d", mode);
  if (ops & ~7u) return fail(TR_ERR_INVALID_ARG, "ops must be a mask of TR_SUM|TR_MIN|TR_MAX");
  tr_status s = make_map_params(map, xt == TR_U32, &P);
  if (s) return s;
  const bool ok = (xt == TR_U32 && (yt == TR_U32 || yt == TR_U64)) || (is_float_storage(xt) && yt == TR_F32);
  if (!ok) return fail(TR_ERR_UNSUPPORTED, "scan %d -> %d", xt, yt);
  if (ops & TR_SUM) {
    const bool st_ok = xt == TR_U32 ? sum_t == yt : (sum_t == TR_F32 || sum_t == TR_F64);
    if (!st_ok) return fail(TR_ERR_UNSUPPORTED, "sum dtype %d for scan %d -> %d", sum_t, xt, yt);
    if (!sum) return fail(TR_ERR_INVALID_ARG, "sum output is NULL");
    if ((s = check_ptr(sum, sum_t, 1, "sum"))) return s;
  }
  const tr_dtype mt = xt == TR_U32 ? TR_U32 : TR_F32;
  if ((ops & TR_MIN) && (!mn || (s = check_ptr(mn, mt, 1, "min")))) return s ? s : fail(TR_ERR_INVALID_ARG, "min is NULL");
  if ((ops & TR_MAX) && (!mx || (s = check_ptr(mx, mt, 1, "max")))) return s ? s : fail(TR_ERR_INVALID_ARG, "max is NULL");
  if ((s = check_ptr(x, xt, n, "x")) || (s = check_ptr(y, yt, n, "y"))) return s;
  if (carry && !aligned_to(carry, dtype_size(yt))) return fail(TR_ERR_ALIGNMENT, "carry_in misaligned");
  if (partial_overlap(x, n * dtype_size(xt), y, n * dtype_size(yt)))
    return fail(TR_ERR_INVALID_ARG, "x and y overlap partially");
  if (x == y && n > 0 && dtype_size(xt) != dtype_size(yt))
    return fail(TR_ERR_INVALID_ARG, "in-place scan needs equal element sizes");
  if ((s = check_exec(e, scan_ws_bytes(n, xt, yt), true))) return s;
  if (n == 0 && ops == 0) return TR_OK;
  ScanOpts o;
  o.exclusive = mode == TR_SCAN_EXCLUSIVE;
  o.ops = ops;
  o.sum = sum;
  o.sum_t = sum_t;
  o.mn = mn;
  o.mx = mx;
  return launch_scan(P, x, xt, y, yt, n, carry, e, o);
}

}  // extern "C"
