// k_map.cu -- tr_map: y_i = f(x_i).
//
// Grid-stride over groups of kUnroll 128-bit input vectors per thread (all
// loads of a group in flight together); outputs leave as 128-bit streaming
// stores.  Arrays whose base addresses are not both 16-byte aligned take an
// element-wise path (still coalesced).
#include "dispatch.cuh"

namespace tr {

namespace {

constexpr int kThreads = 256;
constexpr int kUnroll = 4;

template <class In, class F>
__global__ void __launch_bounds__(kThreads) k_map(const In* __restrict__ x, typename Storage<In>::C* y, int64_t n,
                                                  int vec_ok, const __grid_constant__ MapParams P) {
  using S = Storage<In>;
  using C = typename S::C;
  constexpr int V = S::kVec;
  constexpr int kOut16 = V * (int)sizeof(C) / 16;  // 16-byte output chunks per input vector
  const auto f = make_kernel_map<F>(P);
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

}  // namespace

tr_status launch_map(const MapParams& P, const void* x, tr_dtype xt, void* y, int64_t n, const tr_exec* e) {
  cudaStream_t st = stream_of(e);
  return dispatch_any(xt, P, [&](auto in_tag, auto map_tag) -> tr_status {
    using In = decltype(in_tag);
    using F = decltype(map_tag);
    using S = Storage<In>;
    auto kern = k_map<In, F>;
    const int vec_ok = aligned_to(x, 16) && aligned_to(y, 16);
    const int64_t work = vec_ok ? ceil_div(n / S::kVec, kUnroll) : n;
    const int64_t resident = (int64_t)dev_info().sm_count * blocks_per_sm((const void*)kern, kThreads);
    const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(resident, ceil_div(work, kThreads)));
    kern<<<(unsigned)grid, kThreads, 0, st>>>(static_cast<const In*>(x), static_cast<typename S::C*>(y), n, vec_ok, P);
    return launch_status("k_map");
  });
}

}  // namespace tr
