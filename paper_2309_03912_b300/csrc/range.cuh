// range.cuh -- one warp reduces f over the elements [pa, pb) of an array:
// 128-bit loads with U vectors in flight per lane (kRangeUnroll unless the
// caller picks another count; fewer vectors take fewer registers), a scalar
// head and tail around the 16-byte-aligned body, the map in registers, and
// the per-lane Kahan-compensated accumulator of accum.cuh.  Every lane returns
// its own accumulator; combine with Acc<float>::warp().  While it streams,
// lane 0 asks L2 for the data kPrefetchAhead chunks ahead (up to element
// pf_limit, the end of the region this warp will read).
#pragma once

#include "accum.cuh"

namespace tr {

constexpr int kRangeUnroll = 4;
// Chunks (32 lanes x U vectors) requested into L2 ahead of use.
constexpr int kPrefetchAhead = 4;

template <class In, class F, int U = kRangeUnroll>
__device__ __forceinline__ Acc<float> warp_reduce_range(const In* __restrict__ x, int64_t pa, int64_t pb, int x_aligned,
                                                        const F& f, int lane, int64_t pf_limit) {
  using S = Storage<In>;
  constexpr int V = S::kVec;
  Acc<float> acc;
  if (pa >= pb) return acc;
  const int64_t va = (pa + V - 1) / V, vb = pb / V;
  if (!x_aligned || va >= vb) {  // misaligned base, or under two vectors' worth: element-wise
    for (int64_t i = pa + lane; i < pb; i += 32) acc.add(f(S::cvt(x[i])));
    return acc;
  }
  if (pa + lane < va * V) acc.add(f(S::cvt(x[pa + lane])));      // head (< V elements)
  if (vb * V + lane < pb) acc.add(f(S::cvt(x[vb * V + lane])));  // tail (< V elements)
  const uint4* xv = reinterpret_cast<const uint4*>(x);
  int64_t v = va + lane;
  const int64_t vpf_end = pf_limit / V;  // prefetches stay below element pf_limit
  for (; v + 32 * (U - 1) < vb; v += 32 * U) {
    if (lane == 0) {
      const int64_t pv = v + (int64_t)kPrefetchAhead * 32 * U;
      if (pv + 32 * U <= vpf_end) prefetch_l2(xv + pv, 32 * U * 16);
    }
    uint4 raw[U];
#pragma unroll
    for (int u = 0; u < U; ++u) raw[u] = ld_stream(xv + v + 32 * u);
    float e[U * V];
#pragma unroll
    for (int u = 0; u < U; ++u) S::unpack(raw[u], e + u * V);
    map_vec<U * V>(f, e);
    acc.template add_vec<U * V>(e);
  }
  for (; v < vb; v += 32) {
    float e[V];
    S::unpack(ld_stream(xv + v), e);
    map_vec<V>(f, e);
    acc.template add_vec<V>(e);
  }
  return acc;
}

}  // namespace tr
