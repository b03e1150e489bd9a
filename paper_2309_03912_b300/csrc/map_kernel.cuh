// map_kernel.cuh -- the kernel of tr_map, y_i = f(x_i), as a template over the
// storage type, the map and the map's source (the family's MapParams, or a
// user-supplied functor passed by value), with its launcher.
//
// Grid-stride over groups of kUnroll 128-bit input vectors per thread (all
// loads of a group in flight together); outputs leave as 128-bit streaming
// stores.  Arrays whose base addresses are not both 16-byte aligned take an
// element-wise path (still coalesced).
#pragma once

#include "internal.h"

namespace tr {
namespace mapk {

constexpr int kThreads = 256;
constexpr int kUnroll = 4;

template <class In, class F, class Src>
__global__ void __launch_bounds__(kThreads) k_map(const In* __restrict__ x, typename Storage<In>::C* y, int64_t n,
                                                  int vec_ok, const __grid_constant__ Src P) {
  using S = Storage<In>;
  using C = typename S::C;
  constexpr int V = S::kVec;
  constexpr int kOut16 = V * (int)sizeof(C) / 16;  // 16-byte output chunks per input vector
  const auto f = kernel_map<F>(P);
  const int64_t tid = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const int64_t nthreads = (int64_t)gridDim.x * kThreads;
  int64_t done = 0;
  if (vec_ok) {
    const int64_t nvec = n / V;
    const uint4* xv = reinterpret_cast<const uint4*>(x);
    uint4* yv = reinterpret_cast<uint4*>(y);
    constexpr int64_t kGroup = (int64_t)kThreads * kUnroll;
    for (int64_t g = (int64_t)blockIdx.x * kGroup; g < nvec; g += (int64_t)gridDim.x * kGroup) {
      uint4 raw[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int64_t vi = g + u * kThreads + threadIdx.x;
        if (vi < nvec) raw[u] = ld_stream(xv + vi);
      }
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) {
        const int64_t vi = g + u * kThreads + threadIdx.x;
        if (vi < nvec) {
          C v[V];
          S::unpack(raw[u], v);
          map_vec<V>(f, v);
#pragma unroll
          for (int j = 0; j < kOut16; ++j) st_stream(yv + vi * kOut16 + j, pack16(v + j * (16 / (int)sizeof(C))));
        }
      }
    }
    done = nvec * V;
  }
  for (int64_t i = done + tid; i < n; i += nthreads) y[i] = f(S::cvt(x[i]));
}

template <class In, class F, class Src>
tr_status launch(const Src& P, const In* x, typename Storage<In>::C* y, int64_t n, cudaStream_t st) {
  using S = Storage<In>;
  auto kern = k_map<In, F, Src>;
  const int vec_ok = aligned_to(x, 16) && aligned_to(y, 16);
  const int64_t work = vec_ok ? ceil_div(n / S::kVec, kUnroll) : n;
  const int64_t resident = (int64_t)dev_info().sm_count * blocks_per_sm((const void*)kern, kThreads);
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(resident, ceil_div(work, kThreads)));
  kern<<<(unsigned)grid, kThreads, 0, st>>>(x, y, n, vec_ok, P);
  return launch_status("k_map");
}

}  // namespace mapk
}  // namespace tr
