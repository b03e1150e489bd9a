// k_reduce.cu -- tr_reduce for the map family of the C ABI: dtype and map
// dispatch to the kernel template of reduce_kernel.cuh.
#include "dispatch.cuh"
#include "reduce_kernel.cuh"

namespace tr {

size_t reduce_ws_bytes(int64_t, tr_dtype) { return kWsHeader + redk::kMaxGrid * sizeof(PartialF); }

tr_status launch_reduce(const MapParams& P, const void* x, tr_dtype xt, int64_t n, unsigned ops, void* sum,
                        tr_dtype sum_t, void* mn, void* mx, const tr_exec* e) {
  const RedOut out{sum, mn, mx, (int32_t)sum_t, ops};
  return dispatch_any(xt, P, [&](auto in_tag, auto map_tag) -> tr_status {
    using In = decltype(in_tag);
    using F = decltype(map_tag);
    return redk::launch<In, F>(P, static_cast<const In*>(x), n, out, e);
  });
}

}  // namespace tr
