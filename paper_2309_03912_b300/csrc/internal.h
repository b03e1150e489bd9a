// internal.h -- host-side helpers shared by the launchers of libtr.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdint>

#include "common.cuh"

namespace tr {

struct DevInfo {
  int device = -1;
  int sm_count = 0;
  int smem_optin = 0;
};

// Properties of the current device (queried once per device).
const DevInfo& dev_info();

// Record a failure for tr_last_error() on this thread and return `s`.
tr_status fail(tr_status s, const char* fmt, ...);

// Turn a CUDA error into TR_ERR_CUDA (TR_OK for cudaSuccess).
tr_status cuda_status(cudaError_t e, const char* what);

// Kernel launches enqueued by the library (tr_launch_count).
void count_launches(unsigned long long k);

// Check the launch of the kernel just enqueued (and count it).
inline tr_status launch_status(const char* what) {
  const tr_status s = cuda_status(cudaGetLastError(), what);
  if (s == TR_OK) count_launches(1);
  return s;
}

size_t dtype_size(tr_dtype t);

inline bool aligned_to(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// Validate a map descriptor for the given input kind and fill kernel params.
// int_input: u32 storage (mixers / identity only).
tr_status make_map_params(const tr_map_desc* d, bool int_input, MapParams* P);

// Resident blocks per SM of a kernel at a block size and dynamic shared
// memory size (cached per device, kernel and shape).
int blocks_per_sm(const void* kernel, int threads, size_t dyn_smem = 0);

// Allow `kernel` `bytes` of dynamic shared memory on the current device
// (cudaFuncSetAttribute, which acts per device), once per (device, kernel,
// bytes); thread-safe.
tr_status ensure_dyn_smem(const void* kernel, int bytes, const char* what);

inline WsHeader* ws_header(const tr_exec* e) { return static_cast<WsHeader*>(e->workspace); }
inline char* ws_body(const tr_exec* e) { return static_cast<char*>(e->workspace) + kWsHeader; }

inline cudaStream_t stream_of(const tr_exec* e) { return static_cast<cudaStream_t>(e->stream); }

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// 2-D tiled tensor map over a row-major array: `rows` rows of `inner`
// elements, `row_bytes` apart; boxes of box_inner x box_rows elements.
// (cuTensorMapEncodeTiled through the runtime's driver entry point.)
tr_status make_tensor_map_2d(CUtensorMap* out, const void* base, CUtensorMapDataType type, uint64_t inner,
                             uint64_t rows, uint64_t row_bytes, uint32_t box_inner, uint32_t box_rows,
                             CUtensorMapSwizzle swizzle);

// ---- launchers (one per kernel family) ------------------------------------
size_t reduce_ws_bytes(int64_t n, tr_dtype xt);
tr_status launch_reduce(const MapParams& P, const void* x, tr_dtype xt, int64_t n, unsigned ops, void* sum,
                        tr_dtype sum_t, void* mn, void* mx, const tr_exec* e);

tr_status launch_map(const MapParams& P, const void* x, tr_dtype xt, void* y, int64_t n, const tr_exec* e);

size_t segreduce_ws_bytes(int64_t n, int64_t n_seg, tr_dtype xt);
tr_status launch_segreduce(const MapParams& P, const void* x, tr_dtype xt, int64_t n, const int64_t* off,
                           int64_t n_seg, unsigned ops, void* sums, tr_dtype sum_t, void* mins, void* maxs,
                           const tr_exec* e);

size_t scan_ws_bytes(int64_t n, tr_dtype xt, tr_dtype yt);
// Options of a scan: exclusive outputs, and the sum / min / max of f taken in
// the same pass (ops = 0: none; outputs in device memory).
struct ScanOpts {
  int exclusive = 0;
  unsigned ops = 0;
  void* sum = nullptr;
  tr_dtype sum_t = TR_NONE;
  void* mn = nullptr;
  void* mx = nullptr;
};
tr_status launch_scan(const MapParams& P, const void* x, tr_dtype xt, void* y, tr_dtype yt, int64_t n,
                      const void* carry, const tr_exec* e, const ScanOpts& opt = ScanOpts());

}  // namespace tr
