// accum.cuh -- per-thread accumulators for sum / min / max and their warp and
// block combination, one flavour per compute type:
//   float    : Kahan-compensated sum of pairwise vector sums; warps and blocks
//              combine in float-float; the value leaving a block is FP64.
//   double   : plain FP64 sums (FP64 compute paths only).
//   uint32_t : exact 64-bit integer sums.
// min / max follow IEEE minNum / maxNum (a NaN operand is ignored).
#pragma once

#include <math.h>

#include "common.cuh"

namespace tr {

// Partial results that cross block boundaries (workspace records).
struct PartialF {
  double sum, mn, mx;
};
struct PartialU {
  unsigned long long sum;
  uint32_t mn, mx;
};

template <class C>
struct Acc;

// Pairwise sum of V values.  From four values up the first levels run on
// packed pairs (add.rn.f32x2: pair j of the first half plus pair j of the
// second half), so every value still passes through log2(V) additions.
template <int V>
__device__ __forceinline__ float pairwise(const float* v) {
  if constexpr (V == 1) {
    return v[0];
  } else if constexpr (V == 2 || V % 4 != 0) {
    return pairwise<V / 2>(v) + pairwise<V - V / 2>(v + V / 2);
  } else {
    unsigned long long p[V / 2];
#pragma unroll
    for (int j = 0; j < V / 2; ++j) p[j] = pack_f32x2(v[2 * j], v[2 * j + 1]);
#pragma unroll
    for (int w = V / 4; w >= 1; w /= 2)
#pragma unroll
      for (int j = 0; j < w; ++j) p[j] = add_f32x2(p[j], p[j + w]);
    float lo, hi;
    unpack_f32x2(p[0], lo, hi);
    return lo + hi;
  }
}

template <>
struct Acc<float> {
  using Partial = PartialF;
  Kahan k;
  float mn = INFINITY, mx = -INFINITY;
  __device__ __forceinline__ void add(float v) {
    k.add(v);
    mn = fminf(mn, v);
    mx = fmaxf(mx, v);
  }
  template <int V>
  __device__ __forceinline__ void add_vec(const float* v) {
    k.add(pairwise<V>(v));
#pragma unroll
    for (int i = 0; i + 1 < V; i += 2) {
      mn = min3f(mn, v[i], v[i + 1]);
      mx = max3f(mx, v[i], v[i + 1]);
    }
    if constexpr (V % 2 == 1) {
      mn = fminf(mn, v[V - 1]);
      mx = fmaxf(mx, v[V - 1]);
    }
  }
  // Only the values v[i] with take(i) true (take: index -> bool, evaluated
  // for compile-time i); the others are never combined.
  template <int V, class Take>
  __device__ __forceinline__ void add_if(const float* v, Take take) {
    float t[V];
#pragma unroll
    for (int i = 0; i < V; ++i) t[i] = take(i) ? v[i] : 0.0f;
    k.add(pairwise<V>(t));
#pragma unroll
    for (int i = 0; i + 1 < V; i += 2) {
      const bool a = take(i), b = take(i + 1);
      mn = min3f(mn, a ? v[i] : INFINITY, b ? v[i + 1] : INFINITY);
      mx = max3f(mx, a ? v[i] : -INFINITY, b ? v[i + 1] : -INFINITY);
    }
    if constexpr (V % 2 == 1) {
      if (take(V - 1)) {
        mn = fminf(mn, v[V - 1]);
        mx = fmaxf(mx, v[V - 1]);
      }
    }
  }
  // warp-combined value (every lane holds it)
  struct W {
    FF s;
    float mn, mx;
  };
  __device__ __forceinline__ W warp() const { return W{warp_sum_ff(k.ff()), warp_min(mn), warp_max(mx)}; }
  __device__ static __forceinline__ W identity() { return W{FF{0.f, 0.f}, INFINITY, -INFINITY}; }
  __device__ static __forceinline__ W warp_combine(W a) { return W{warp_sum_ff(a.s), warp_min(a.mn), warp_max(a.mx)}; }
  __device__ static __forceinline__ Partial to_partial(W a) { return Partial{ff_to_double(a.s), (double)a.mn, (double)a.mx}; }
};

template <>
struct Acc<double> {
  using Partial = PartialF;
  double s = 0.0, mn = INFINITY, mx = -INFINITY;
  __device__ __forceinline__ void add(double v) {
    s += v;
    mn = fmin(mn, v);
    mx = fmax(mx, v);
  }
  template <int V>
  __device__ __forceinline__ void add_vec(const double* v) {
#pragma unroll
    for (int i = 0; i < V; ++i) add(v[i]);
  }
  struct W {
    double s, mn, mx;
  };
  __device__ __forceinline__ W warp() const { return W{warp_sum(s), warp_min(mn), warp_max(mx)}; }
  __device__ static __forceinline__ W identity() { return W{0.0, INFINITY, -INFINITY}; }
  __device__ static __forceinline__ W warp_combine(W a) { return W{warp_sum(a.s), warp_min(a.mn), warp_max(a.mx)}; }
  __device__ static __forceinline__ Partial to_partial(W a) { return Partial{a.s, a.mn, a.mx}; }
};

template <>
struct Acc<uint32_t> {
  using Partial = PartialU;
  unsigned long long s = 0;
  uint32_t mn = 0xFFFFFFFFu, mx = 0u;
  __device__ __forceinline__ void add(uint32_t v) {
    s += v;
    mn = min(mn, v);
    mx = max(mx, v);
  }
  template <int V>
  __device__ __forceinline__ void add_vec(const uint32_t* v) {
#pragma unroll
    for (int i = 0; i < V; ++i) add(v[i]);
  }
  struct W {
    unsigned long long s;
    uint32_t mn, mx;
  };
  __device__ __forceinline__ W warp() const { return W{warp_sum(s), warp_min(mn), warp_max(mx)}; }
  __device__ static __forceinline__ W identity() { return W{0ull, 0xFFFFFFFFu, 0u}; }
  __device__ static __forceinline__ W warp_combine(W a) { return W{warp_sum(a.s), warp_min(a.mn), warp_max(a.mx)}; }
  __device__ static __forceinline__ Partial to_partial(W a) { return Partial{a.s, a.mn, a.mx}; }
};

// Combine the per-thread accumulators of a block; the result is valid in
// warp 0.  `sm` must hold blockDim.x / 32 elements of Acc<C>::W.
template <class C>
__device__ __forceinline__ typename Acc<C>::W block_combine(const Acc<C>& a, typename Acc<C>::W* sm) {
  using W = typename Acc<C>::W;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const W w = a.warp();
  if (lane == 0) sm[wid] = w;
  __syncthreads();
  W r = Acc<C>::identity();
  if (wid == 0) {
    r = lane < nw ? sm[lane] : Acc<C>::identity();
    r = Acc<C>::warp_combine(r);
  }
  __syncthreads();
  return r;
}

// FP64 / integer combination of block partials (fixed order: thread t takes
// partials t, t + blockDim, ...; then a fixed butterfly).  Valid in warp 0.
__device__ __forceinline__ PartialF combine_partials(const PartialF* p, int count, PartialF* sm) {
  double s = 0.0, mn = INFINITY, mx = -INFINITY;
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    s += __ldcg(&p[i].sum);
    mn = fmin(mn, __ldcg(&p[i].mn));
    mx = fmax(mx, __ldcg(&p[i].mx));
  }
  s = warp_sum(s);
  mn = warp_min(mn);
  mx = warp_max(mx);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) sm[wid] = PartialF{s, mn, mx};
  __syncthreads();
  PartialF r{0.0, INFINITY, -INFINITY};
  if (wid == 0) {
    const PartialF v = lane < nw ? sm[lane] : r;
    r = PartialF{warp_sum(v.sum), warp_min(v.mn), warp_max(v.mx)};
  }
  __syncthreads();
  return r;
}

__device__ __forceinline__ PartialU combine_partials(const PartialU* p, int count, PartialU* sm) {
  unsigned long long s = 0;
  uint32_t mn = 0xFFFFFFFFu, mx = 0;
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    s += __ldcg(&p[i].sum);
    mn = min(mn, __ldcg(&p[i].mn));
    mx = max(mx, __ldcg(&p[i].mx));
  }
  s = warp_sum(s);
  mn = warp_min(mn);
  mx = warp_max(mx);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) sm[wid] = PartialU{s, mn, mx};
  __syncthreads();
  PartialU r{0ull, 0xFFFFFFFFu, 0u};
  if (wid == 0) {
    const PartialU v = lane < nw ? sm[lane] : r;
    r = PartialU{warp_sum(v.sum), warp_min(v.mn), warp_max(v.mx)};
  }
  __syncthreads();
  return r;
}

// Device output pointers of a reduction and their types.
struct RedOut {
  void* sum;
  void* mn;
  void* mx;
  int32_t sum_t;  // tr_dtype
  uint32_t ops;
};

// Store a finished (sum, min, max) at index i of the outputs.
__device__ __forceinline__ void store_result(const RedOut& o, int64_t i, const PartialF& r, bool f32minmax) {
  if ((o.ops & TR_SUM) && o.sum) {
    if (o.sum_t == TR_F64)
      static_cast<double*>(o.sum)[i] = r.sum;
    else
      static_cast<float*>(o.sum)[i] = (float)r.sum;
  }
  if (f32minmax) {
    if ((o.ops & TR_MIN) && o.mn) static_cast<float*>(o.mn)[i] = (float)r.mn;
    if ((o.ops & TR_MAX) && o.mx) static_cast<float*>(o.mx)[i] = (float)r.mx;
  } else {
    if ((o.ops & TR_MIN) && o.mn) static_cast<double*>(o.mn)[i] = r.mn;
    if ((o.ops & TR_MAX) && o.mx) static_cast<double*>(o.mx)[i] = r.mx;
  }
}

__device__ __forceinline__ void store_result(const RedOut& o, int64_t i, const PartialU& r, bool) {
  if ((o.ops & TR_SUM) && o.sum) {
    if (o.sum_t == TR_U64)
      static_cast<unsigned long long*>(o.sum)[i] = r.sum;
    else
      static_cast<uint32_t*>(o.sum)[i] = (uint32_t)r.sum;
  }
  if ((o.ops & TR_MIN) && o.mn) static_cast<uint32_t*>(o.mn)[i] = r.mn;
  if ((o.ops & TR_MAX) && o.mx) static_cast<uint32_t*>(o.mx)[i] = r.mx;
}

}  // namespace tr
