// k_scan.cu -- tr_scan / tr_scan_reduce for the map family of the C ABI: dtype,
// map and output-arithmetic dispatch to the kernel template of scan_kernel.cuh.
#include "dispatch.cuh"
#include "scan_kernel.cuh"

namespace tr {

// One look-back line per tile of 8,192 elements.
size_t scan_ws_bytes(int64_t n, tr_dtype, tr_dtype) {
  const int64_t tiles = std::max<int64_t>(1, ceil_div(n, scank::kTile));
  return (size_t)(kWsHeader + tiles * scank::kLineBytes);
}

tr_status launch_scan(const MapParams& P, const void* x, tr_dtype xt, void* y, tr_dtype yt, int64_t n, const void* carry,
                      const tr_exec* e, const ScanOpts& opt) {
  auto go = [&](auto op_tag) {
    using Op = decltype(op_tag);
    return [&](auto in_tag, auto map_tag) -> tr_status {
      using In = decltype(in_tag);
      using F = decltype(map_tag);
      using Out = typename Op::Out;
      return scank::launch<In, F, Op>(P, static_cast<const In*>(x), static_cast<Out*>(y), n,
                                       static_cast<const Out*>(carry), e, opt);
    };
  };
  if (xt == TR_U32 && yt == TR_U32) return dispatch_u32_map(P, go(scank::OpU32{}));
  if (xt == TR_U32 && yt == TR_U64) return dispatch_u32_map(P, go(scank::OpU64{}));
  if (yt == TR_F32) return dispatch_float_storage(xt, P, go(scank::OpF32{}));
  return fail(TR_ERR_UNSUPPORTED, "scan %d -> %d", xt, yt);
}

}  // namespace tr
