// k_map.cu -- tr_map for the map family of the C ABI: dtype and map dispatch to
// the kernel template of map_kernel.cuh.
#include "dispatch.cuh"
#include "map_kernel.cuh"

namespace tr {

tr_status launch_map(const MapParams& P, const void* x, tr_dtype xt, void* y, int64_t n, const tr_exec* e) {
  cudaStream_t st = stream_of(e);
  return dispatch_any(xt, P, [&](auto in_tag, auto map_tag) -> tr_status {
    using In = decltype(in_tag);
    using F = decltype(map_tag);
    return mapk::launch<In, F>(P, static_cast<const In*>(x), static_cast<typename Storage<In>::C*>(y), n, st);
  });
}

}  // namespace tr
