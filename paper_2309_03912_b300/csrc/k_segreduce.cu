// k_segreduce.cu -- tr_segmented_reduce for the map family of the C ABI: dtype
// and map dispatch to the kernel templates of segreduce_kernel.cuh, and the
// join kernel for segments cut by warp-range ends.
#include "dispatch.cuh"
#include "segreduce_kernel.cuh"

namespace tr {
namespace segk {

// Second launch: every warp of the walk has written its two slots.  One
// thread per warp w takes w's tail piece (a segment that continues past w's
// range) and adds the head pieces of the following warps in warp order, in
// FP64, until the segment ends.  Threads work independently, so the slot reads
// of all cut segments are in flight at once (a single joining block, as in the
// usual last-block scheme, took ~20 us of serial L2 round trips at the
// benchmark size and ~100 us with very long segments).
__global__ void __launch_bounds__(256) k_join_cut(RedOut out, WsHeader* hdr, const SegSlot* __restrict__ slots,
                                                  int64_t nw) {
  const int64_t w = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (w >= nw) return;
  const long long sg = slots[2 * w + 1].seg;
  if (sg < 0) return;
  double sum = slots[2 * w + 1].sum;
  float mn = slots[2 * w + 1].mn, mx = slots[2 * w + 1].mx;
  for (int64_t w2 = w + 1; w2 < nw; ++w2) {
    const SegSlot* h = &slots[2 * w2];
    if (h->seg != sg) {
      set_status(hdr, TR_ERR_DEVICE_ASSERT, (uint32_t)sg);
      break;
    }
    sum += h->sum;
    mn = fminf(mn, h->mn);
    mx = fmaxf(mx, h->mx);
    if (!h->through) break;
  }
  store_result(out, sg, PartialF{sum, (double)mn, (double)mx}, true);
}

tr_status launch_join(const RedOut& out, WsHeader* hdr, const SegSlot* slots, int64_t nw, cudaStream_t st) {
  k_join_cut<<<(unsigned)ceil_div(nw, (int64_t)256), 256, 0, st>>>(out, hdr, slots, nw);
  return launch_status("k_join_cut");
}

}  // namespace segk

size_t segreduce_ws_bytes(int64_t, int64_t, tr_dtype) {
  return kWsHeader + (size_t)segk::kMaxGrid * segk::kWarps * 2 * sizeof(segk::SegSlot);
}

tr_status launch_segreduce(const MapParams& P, const void* x, tr_dtype xt, int64_t n, const int64_t* off,
                           int64_t n_seg, unsigned ops, void* sums, tr_dtype sum_t, void* mins, void* maxs,
                           const tr_exec* e) {
  const RedOut out{sums, mins, maxs, (int32_t)sum_t, ops};
  return dispatch_float_storage(xt, P, [&](auto in_tag, auto map_tag) -> tr_status {
    using In = decltype(in_tag);
    using F = decltype(map_tag);
    return segk::launch<In, F>(P, static_cast<const In*>(x), n, off, n_seg, out, e);
  });
}

}  // namespace tr
