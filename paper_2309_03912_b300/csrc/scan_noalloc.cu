// scan_noalloc.cu -- tr_scan_noalloc: the inclusive scan of tr_scan for
// callers that cannot allocate device memory.
//
// Some callers have no way to obtain a workspace: code running inside a
// custom memory allocator or an allocation-free real-time loop, plugins that
// are handed only input and output pointers by a host framework, or programs
// that have reserved all device memory up front.  For them this entry point
// keeps the scan's scratch (tile flags, aggregates, inclusive prefixes and the
// status header) in one file-scope device array of fixed size, reserved when
// the library is loaded on a GPU and held until the process exits.  It makes no
// cudaMalloc / cudaFree call and uses no allocating library routine.
//
// The scan kernel itself is the one tr_scan launches; only where its scratch
// lives differs.
#include <mutex>

#include "internal.h"

namespace tr {

namespace {

// Largest input accepted: 2^26 elements.
constexpr int64_t kNoAllocMaxN = int64_t(1) << 26;
// Header + one 128-byte look-back line per tile for up to 8,192 tiles (the
// scan's tiles hold 8,192 elements, so 2^26 elements need no more); the call
// checks the scan's own workspace size against it before launching.
constexpr size_t kNoAllocScratchBytes = 256 + (size_t)8192 * 128;

// The scratch.  In host code this name is only a stand-in for the symbol, not
// a device address: the address is obtained with cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_scan_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (the first call on a device does this set-up).
tr_status scratch_address(void** out) {
  int dev = -1;
  tr_status s = cuda_status(cudaGetDevice(&dev), "cudaGetDevice");
  if (s) return s;
  if (dev < 0 || dev >= kMaxDevices) return fail(TR_ERR_UNSUPPORTED, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    s = cuda_status(cudaGetSymbolAddress(&p, g_scan_scratch), "cudaGetSymbolAddress(scan scratch)");
    if (s) return s;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return TR_OK;
}

bool float_storage(tr_dtype t) { return t == TR_F16 || t == TR_BF16 || t == TR_F32; }

}  // namespace

}  // namespace tr

using namespace tr;

extern "C" tr_status tr_scan_noalloc(const tr_map_desc* map, const void* x, tr_dtype xt, void* y, tr_dtype yt,
                                     int64_t n, const void* carry, uint32_t* d_status, void* stream) {
  MapParams P;
  if (n < 0) return fail(TR_ERR_INVALID_ARG, "n < 0");
  if (n > kNoAllocMaxN)
    return fail(TR_ERR_INVALID_ARG,
                "n = %lld exceeds the %lld-element limit of tr_scan_noalloc's fixed scratch; use tr_scan with a "
                "workspace for larger inputs",
                (long long)n, (long long)kNoAllocMaxN);
  tr_status s = make_map_params(map, xt == TR_U32, &P);
  if (s) return s;
  const bool ok = (xt == TR_U32 && (yt == TR_U32 || yt == TR_U64)) || (float_storage(xt) && yt == TR_F32);
  if (!ok) return fail(TR_ERR_UNSUPPORTED, "scan %d -> %d", xt, yt);
  if (n > 0 && (!x || !y)) return fail(TR_ERR_INVALID_ARG, "x or y is NULL");
  if ((x && !aligned_to(x, dtype_size(xt))) || (y && !aligned_to(y, dtype_size(yt))) ||
      (carry && !aligned_to(carry, dtype_size(yt))) || (d_status && !aligned_to(d_status, 4)))
    return fail(TR_ERR_ALIGNMENT, "a pointer is not aligned to its element size");
  const uintptr_t xa = (uintptr_t)x, ya = (uintptr_t)y;
  const size_t xb = (size_t)n * dtype_size(xt), yb = (size_t)n * dtype_size(yt);
  if (n > 0 && !(xa == ya && xb == yb) && xa < ya + yb && ya < xa + xb)
    return fail(TR_ERR_INVALID_ARG, "x and y overlap partially");
  if (scan_ws_bytes(n, xt, yt) > kNoAllocScratchBytes)
    return fail(TR_ERR_WORKSPACE, "the fixed scratch is smaller than the scan needs for n = %lld", (long long)n);
  void* scratch = nullptr;
  if ((s = scratch_address(&scratch))) return s;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // The array keeps the previous call's contents.  Clear the error words
  // (status, detail, abort) and the two counters; the scan itself clears its
  // tile flags before it starts.
  auto* hdr = static_cast<WsHeader*>(scratch);
  if ((s = cuda_status(cudaMemsetAsync(hdr, 0, 3 * sizeof(uint32_t), st), "cudaMemsetAsync(status)"))) return s;
  if ((s = cuda_status(cudaMemsetAsync(&hdr->ticket, 0, 2 * sizeof(uint32_t), st), "cudaMemsetAsync(counters)")))
    return s;
  if (n > 0) {
    const tr_exec e{stream, scratch, kNoAllocScratchBytes, 0u, 0, -1};
    if ((s = launch_scan(P, x, xt, y, yt, n, carry, &e))) return s;
  }
  if (d_status)
    return cuda_status(cudaMemcpyAsync(d_status, &hdr->status, sizeof(uint32_t), cudaMemcpyDeviceToDevice, st),
                       "cudaMemcpyAsync(status)");
  return TR_OK;
}
