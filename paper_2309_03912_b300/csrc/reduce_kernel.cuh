// reduce_kernel.cuh -- the kernel of tr_reduce, sum / min / max of f(x) over one
// array, as a template over the storage type, the map and the map's source
// (the family's MapParams, or a user-supplied functor passed by value), with
// its launcher.
//
// One launch sized to the resident grid: each block strides over groups of
// kThreads x kUnroll 128-bit vectors (all loads of a group issued before any
// use), applies the map in registers and accumulates per thread (Kahan over
// pairwise vector sums for FP32 compute).  Blocks combine warp-wise in
// float-float, publish an FP64 (or u64) partial, and the last block to finish
// (atomic ticket after a fence) combines all partials in a fixed order and
// writes the result -- a single kernel, deterministic for a given grid.
#pragma once

#include "accum.cuh"
#include "internal.h"

namespace tr {
namespace redk {

constexpr int kThreads = 256;
constexpr int kUnroll = 4;
constexpr int kMaxGrid = 2048;

template <class In, class F, class Src>
__device__ __forceinline__ void reduce_body(const In* __restrict__ x, int64_t n, int32_t head, const Src& P,
                                            RedOut out, WsHeader* hdr,
                                            typename Acc<typename Storage<In>::C>::Partial* partials) {
  using S = Storage<In>;
  using C = typename S::C;
  using A = Acc<C>;
  using Partial = typename A::Partial;
  constexpr int V = S::kVec;
  const auto f = kernel_map<F>(P);
  A acc;

  const int64_t nvec = (n - head) / V;
  if (blockIdx.x == 0) {  // scalar head (to 16-byte alignment) and ragged tail
    if ((int)threadIdx.x < head) acc.add(f(S::cvt(x[threadIdx.x])));
    const int64_t t = head + nvec * V + threadIdx.x;
    if (t < n) acc.add(f(S::cvt(x[t])));
  }
  const uint4* xv = reinterpret_cast<const uint4*>(x + head);
  constexpr int64_t kGroup = (int64_t)kThreads * kUnroll;
  for (int64_t g = (int64_t)blockIdx.x * kGroup; g < nvec; g += (int64_t)gridDim.x * kGroup) {
    if (g + kGroup <= nvec) {
      uint4 raw[kUnroll];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) raw[u] = ld_stream(xv + g + u * kThreads + threadIdx.x);
      C v[kUnroll * V];
#pragma unroll
      for (int u = 0; u < kUnroll; ++u) S::unpack(raw[u], v + u * V);
      map_vec<kUnroll * V>(f, v);
      acc.template add_vec<kUnroll * V>(v);
    } else {
      for (int u = 0; u < kUnroll; ++u) {
        const int64_t vi = g + u * kThreads + threadIdx.x;
        if (vi < nvec) {
          C v[V];
          S::unpack(ld_stream(xv + vi), v);
          map_vec<V>(f, v);
          acc.template add_vec<V>(v);
        }
      }
    }
  }

  __shared__ typename A::W smw[kThreads / 32];
  __shared__ Partial smp[kThreads / 32];
  __shared__ bool last;
  const typename A::W w = block_combine<C>(acc, smw);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = A::to_partial(w);
    __threadfence();
    last = atomicAdd(&hdr->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  const Partial r = combine_partials(partials, gridDim.x, smp);
  if (threadIdx.x == 0) {
    store_result(out, 0, r, std::is_same<C, float>::value);
    hdr->ticket = 0;  // leave the workspace ready for the next call
  }
}

template <class In, class F, class Src>
__global__ void __launch_bounds__(kThreads) k_reduce(const In* __restrict__ x, int64_t n, int32_t head,
                                                     const __grid_constant__ Src P, RedOut out, WsHeader* hdr,
                                                     typename Acc<typename Storage<In>::C>::Partial* partials) {
  reduce_body<In, F, Src>(x, n, head, P, out, hdr, partials);
}

// The same with at most 64 registers (4 blocks per SM): on B300 the FP32
// Horner reductions run ~5 % faster this way, other maps and storage types
// slower, so only those use it.
template <class In, class F, class Src>
__global__ void __launch_bounds__(kThreads, 4) k_reduce_b4(const In* __restrict__ x, int64_t n, int32_t head,
                                                           const __grid_constant__ Src P, RedOut out,
                                                           WsHeader* hdr,
                                                           typename Acc<typename Storage<In>::C>::Partial* partials) {
  reduce_body<In, F, Src>(x, n, head, P, out, hdr, partials);
}

template <class In, class F>
struct FourBlocks : std::false_type {};
template <int D>
struct FourBlocks<float, Horner<float, D>> : std::true_type {};

template <class In, class F, class Src>
tr_status launch(const Src& P, const In* x, int64_t n, const RedOut& out, const tr_exec* e) {
  using S = Storage<In>;
  using Partial = typename Acc<typename S::C>::Partial;
  WsHeader* hdr = ws_header(e);
  auto kern = [] {
    if constexpr (FourBlocks<In, F>::value) {
      return k_reduce_b4<In, F, Src>;
    } else {
      return k_reduce<In, F, Src>;
    }
  }();
  const int64_t addr = (int64_t)reinterpret_cast<uintptr_t>(x);
  int64_t head = ((16 - addr % 16) % 16) / (int64_t)sizeof(In);
  if (head > n) head = n;
  const int64_t nvec = (n - head) / S::kVec;
  const int64_t groups = ceil_div(nvec, (int64_t)kThreads * kUnroll);
  const int64_t resident = (int64_t)dev_info().sm_count * blocks_per_sm((const void*)kern, kThreads);
  const int64_t grid = std::min<int64_t>(std::min<int64_t>(resident, kMaxGrid), std::max<int64_t>(groups, 1));
  kern<<<(unsigned)grid, kThreads, 0, stream_of(e)>>>(x, n, (int32_t)head, P, out, hdr,
                                                       reinterpret_cast<Partial*>(ws_body(e)));
  return launch_status("k_reduce");
}

}  // namespace redk
}  // namespace tr
