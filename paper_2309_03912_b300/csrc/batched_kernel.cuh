// batched_kernel.cuh -- the device side of tr_batched_*: the descriptors of
// arrays, work items and partials, and the persistent kernel whose warps pull
// items from an atomic queue, reduce each with its array's map, and join an
// array's partials in item order once its last item is done.
//
// The kernel is a template over the storage type, the block size and U, the
// 16-byte vectors each lane has in flight (U x 4 values for FP32, U x 8 for
// FP16/BF16).  Fewer vectors per lane take fewer registers and so leave room
// for more resident warps; which count is faster depends on the mix of maps,
// so the plan's autotuner times both.  Each count is instantiated in a
// translation unit of its own (k_batched.cu: 4, k_batched_u2.cu: 2) so that
// the two compile in parallel.
#pragma once

#include "accum.cuh"
#include "dispatch.cuh"
#include "range.cuh"

namespace tr {

struct BatchArray {
  const void* x;  // storage type of the plan
  int64_t len;
  int32_t kind, deg_p, deg_q, iters;
  int32_t first_slot, n_items;
  int32_t aligned, pad;
  float cp[TR_MAX_DEGREE + 1];
  float cq[TR_MAX_DEGREE + 1];
};

struct BatchItem {
  int32_t array;
  int32_t slot;  // partial slot of this item (array's first slot + its index)
  int64_t start;
  int64_t count;
};

struct BatchPartial {
  double sum;
  float mn, mx;
};

struct BatchOut {
  double* sums;
  float* mins;
  float* maxs;
  unsigned ops;
};

template <class F>
struct MakeBatchMap {
  __device__ __forceinline__ static F make(const BatchArray&) { return F{}; }
};
template <int D>
struct MakeBatchMap<Horner<float, D>> {
  __device__ __forceinline__ static Horner<float, D> make(const BatchArray& A) {
    Horner<float, D> h{};
#pragma unroll
    for (int k = 0; k <= D; ++k) h.c[k] = A.cp[k];
    return h;
  }
};
template <>
struct MakeBatchMap<HornerN<float>> {
  __device__ __forceinline__ static HornerN<float> make(const BatchArray& A) { return HornerN<float>{A.cp, A.deg_p}; }
};
template <>
struct MakeBatchMap<Rational<float, 6, 6>> {
  __device__ __forceinline__ static Rational<float, 6, 6> make(const BatchArray& A) {
    Rational<float, 6, 6> r{};
#pragma unroll
    for (int k = 0; k <= 6; ++k) {
      r.p[k] = A.cp[k];
      r.q[k] = A.cq[k];
    }
    return r;
  }
};
template <>
struct MakeBatchMap<RationalN<float>> {
  __device__ __forceinline__ static RationalN<float> make(const BatchArray& A) {
    return RationalN<float>{A.cp, A.cq, A.deg_p, A.deg_q};
  }
};
template <>
struct MakeBatchMap<NewtonCbrt<float, -1>> {
  __device__ __forceinline__ static NewtonCbrt<float, -1> make(const BatchArray& A) {
    NewtonCbrt<float, -1> m{};
    m.iters = A.iters;
    return m;
  }
};

template <class In, int U, class F>
__device__ __forceinline__ Acc<float> run_item(const BatchArray& A, const BatchItem& it, int lane) {
  const auto f = Packed<F>::make(MakeBatchMap<F>::make(A));  // coefficient pairs in registers
  return warp_reduce_range<In, typename Packed<F>::type, U>(static_cast<const In*>(A.x), it.start, it.start + it.count,
                                                             A.aligned, f, lane, it.start + it.count);
}

template <class In, int U>
__device__ __noinline__ Acc<float> dispatch_item(const BatchArray& A, const BatchItem& it, int lane) {
  switch (A.kind) {
    case TR_MAP_HORNER:
      switch (A.deg_p) {
        case 4: return run_item<In, U, Horner<float, 4>>(A, it, lane);
        case 5: return run_item<In, U, Horner<float, 5>>(A, it, lane);
        case 6: return run_item<In, U, Horner<float, 6>>(A, it, lane);
        case 7: return run_item<In, U, Horner<float, 7>>(A, it, lane);
        case 8: return run_item<In, U, Horner<float, 8>>(A, it, lane);
        case 9: return run_item<In, U, Horner<float, 9>>(A, it, lane);
        case 10: return run_item<In, U, Horner<float, 10>>(A, it, lane);
        case 11: return run_item<In, U, Horner<float, 11>>(A, it, lane);
        case 12: return run_item<In, U, Horner<float, 12>>(A, it, lane);
        case 13: return run_item<In, U, Horner<float, 13>>(A, it, lane);
        case 14: return run_item<In, U, Horner<float, 14>>(A, it, lane);
        case 15: return run_item<In, U, Horner<float, 15>>(A, it, lane);
        case 16: return run_item<In, U, Horner<float, 16>>(A, it, lane);
        default: return run_item<In, U, HornerN<float>>(A, it, lane);
      }
    case TR_MAP_RATIONAL:
      if (A.deg_p == 6 && A.deg_q == 6) return run_item<In, U, Rational<float, 6, 6>>(A, it, lane);
      return run_item<In, U, RationalN<float>>(A, it, lane);
    case TR_MAP_NEWTON_CBRT:
      if (A.iters == 6) return run_item<In, U, NewtonCbrt<float, 6>>(A, it, lane);
      return run_item<In, U, NewtonCbrt<float, -1>>(A, it, lane);
    case TR_MAP_SQUARE: return run_item<In, U, Square<float>>(A, it, lane);
    default: return run_item<In, U, Identity<float>>(A, it, lane);
  }
}

__device__ __forceinline__ void store_batch(const BatchOut& o, int64_t a, double s, float mn, float mx) {
  if ((o.ops & TR_SUM) && o.sums) o.sums[a] = s;
  if ((o.ops & TR_MIN) && o.mins) o.mins[a] = mn;
  if ((o.ops & TR_MAX) && o.maxs) o.maxs[a] = mx;
}

template <class In, int THREADS, int U>
__global__ void __launch_bounds__(THREADS) k_batched(const BatchArray* __restrict__ arrays,
                                                     const BatchItem* __restrict__ items, int32_t n_items,
                                                     BatchPartial* partials, uint32_t* counters, uint32_t* queue,
                                                     BatchOut out) {
  const int lane = threadIdx.x & 31;
  while (true) {
    int32_t i = 0;
    if (lane == 0) i = (int32_t)atomicAdd(queue, 1u);
    i = __shfl_sync(kFull, i, 0);
    if (i >= n_items) break;
    const BatchItem it = items[i];
    const BatchArray& A = arrays[it.array];
    const Acc<float>::W w = dispatch_item<In, U>(A, it, lane).warp();
    const int32_t n_it = A.n_items;
    if (n_it == 1) {
      if (lane == 0) store_batch(out, it.array, ff_to_double(w.s), w.mn, w.mx);
      continue;
    }
    int last = 0;
    if (lane == 0) {
      partials[it.slot] = BatchPartial{ff_to_double(w.s), w.mn, w.mx};
      __threadfence();
      last = atomicAdd(&counters[it.array], 1u) == (uint32_t)(n_it - 1);
    }
    last = __shfl_sync(kFull, last, 0);
    if (!last) continue;
    __threadfence();
    double s = 0.0;
    float mn = INFINITY, mx = -INFINITY;
    for (int j = lane; j < n_it; j += 32) {  // fixed order: lane j takes slots j, j+32, ...
      const BatchPartial* p = &partials[A.first_slot + j];
      s += __ldcg(&p->sum);
      mn = fminf(mn, __ldcg(&p->mn));
      mx = fmaxf(mx, __ldcg(&p->mx));
    }
    s = warp_sum(s);
    mn = warp_min(mn);
    mx = warp_max(mx);
    if (lane == 0) {
      store_batch(out, it.array, s, mn, mx);
      counters[it.array] = 0;  // ready for the next run
    }
  }
}

typedef void (*BatchedKernel)(const BatchArray*, const BatchItem*, int32_t, BatchPartial*, uint32_t*, uint32_t*,
                              BatchOut);

// The kernel for a storage type and block size at U vectors per lane; each
// translation unit instantiates one U.
template <int U>
BatchedKernel batched_kernel(tr_dtype xt, int threads) {
  if (xt == TR_F16) return threads == 128 ? k_batched<__half, 128, U> : k_batched<__half, 256, U>;
  if (xt == TR_BF16) return threads == 128 ? k_batched<__nv_bfloat16, 128, U> : k_batched<__nv_bfloat16, 256, U>;
  return threads == 128 ? k_batched<float, 128, U> : k_batched<float, 256, U>;
}
BatchedKernel batched_kernel_u4(tr_dtype xt, int threads);  // k_batched.cu
BatchedKernel batched_kernel_u2(tr_dtype xt, int threads);  // k_batched_u2.cu

}  // namespace tr
