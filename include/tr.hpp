/*
 * tr.hpp -- C++ entry points of libtr for maps supplied by the caller.
 *
 * The C ABI (tr.h) serves a fixed family of maps.  This header instantiates
 * the same kernel templates for any map type F written the way the paper
 * teaches (Mejstrik, "__host__ __device__ -- Generic programming in Cuda"):
 * a functor whose call operator is callable on host and device -- and, where
 * its body allows, at compile time -- and that declares so through the
 * host-device-compatibility tag of the paper's Sec. 4 helper:
 *
 *     struct MyMap {
 *       static constexpr tr::HDC hdc = tr::HDC::HstDev;
 *       TR_HD constexpr float operator()(float x) const { return ...; }
 *     };
 *     tr::reduce(MyMap{}, d_x, n, TR_SUM | TR_MIN | TR_MAX, d_sum, d_min, d_max, &exec);
 *
 * A map without the tag is rejected at compile time (static_assert on
 * tr::hdc<F>), which is exactly what the trait is for.  A lambda can serve as
 * well (the paper's Sec. 2.6 "Variant with lambdas: C++17"): a
 * __host__ __device__ lambda (compile with --extended-lambda) wrapped by
 * tr::hd_lambda, or a lambda defined inside a TR_HD function, which inherits
 * that function's execution space.
 *
 * Storage may be float, __half or __nv_bfloat16 (values widened to FP32); the
 * map computes in FP32 (float operator()(float)).  Sums are compensated FP32
 * per thread, combined in float-float and then FP64, exactly as for the
 * family's maps; results, workspaces, streams and errors follow tr.h (the
 * workspace sizes are those of the matching *_workspace_size call).  Compile
 * the calling translation unit with nvcc for sm_103a with -fmad=false (so that
 * device code keeps the map's operation sequence), put the library's source
 * directory (paper_2309_03912_b300/csrc) and include/ on the include path, and
 * link against libtr.so.
 */
#ifndef TR_HPP
#define TR_HPP

#include "tr.h"

#include "map_kernel.cuh"
#include "reduce_kernel.cuh"
#include "scan_kernel.cuh"
#include "segreduce_kernel.cuh"

namespace tr {

// The compile-time gate: F must declare itself callable on host and device.
template <class F>
constexpr bool is_hd_map = hdc<F> == HDC::HstDev;

// A __host__ __device__ lambda as a map: the wrapper carries the tag the
// closure type cannot declare itself (nvcc tells extended host-device
// lambdas apart, so only those are accepted).
template <class L>
struct HdLambda {
  static constexpr HDC hdc = HDC::HstDev;
  L fn;
  TR_HD constexpr float operator()(float x) const { return fn(x); }
};
template <class L>
constexpr HdLambda<L> hd_lambda(L fn) {
#if defined(__CUDACC__) && defined(__CUDACC_EXTENDED_LAMBDA__)
  static_assert(__nv_is_extended_host_device_lambda_closure_type(L),
                "tr::hd_lambda takes a __host__ __device__ lambda (compile with --extended-lambda)");
#endif
  return HdLambda<L>{fn};
}

namespace user {
template <class In>
constexpr bool is_storage = std::is_same<In, float>::value || std::is_same<In, __half>::value ||
                            std::is_same<In, __nv_bfloat16>::value;

inline tr_status check_ws(const tr_exec* e, size_t need) {
  if (!e) return fail(TR_ERR_INVALID_ARG, "exec is NULL");
  if (!e->workspace || e->workspace_bytes < need) return fail(TR_ERR_WORKSPACE, "workspace missing or too small");
  if (!aligned_to(e->workspace, 256)) return fail(TR_ERR_ALIGNMENT, "workspace must be 256-byte aligned");
  return TR_OK;
}
}  // namespace user

// y_i = f(x_i), i < n (FP32 output).  No workspace needed.
template <class F, class In>
tr_status map(const F& f, const In* d_x, float* d_y, int64_t n, const tr_exec* e) {
  static_assert(is_hd_map<F>, "the map must declare static constexpr tr::HDC hdc = tr::HDC::HstDev");
  static_assert(user::is_storage<In>, "storage: float, __half or __nv_bfloat16");
  if (!e || n < 0 || (n > 0 && (!d_x || !d_y))) return fail(TR_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return TR_OK;
  return mapk::launch<In, F>(f, d_x, d_y, n, stream_of(e));
}

// sum (FP64) / min / max (FP32) of f(x_i), i < n, selected by ops; device outputs.
template <class F, class In>
tr_status reduce(const F& f, const In* d_x, int64_t n, unsigned ops, double* d_sum, float* d_min, float* d_max,
                 const tr_exec* e) {
  static_assert(is_hd_map<F>, "the map must declare static constexpr tr::HDC hdc = tr::HDC::HstDev");
  static_assert(user::is_storage<In>, "storage: float, __half or __nv_bfloat16");
  if (n < 0 || ops == 0 || (ops & ~7u) || (n > 0 && !d_x) || ((ops & TR_SUM) && !d_sum) ||
      ((ops & TR_MIN) && !d_min) || ((ops & TR_MAX) && !d_max))
    return fail(TR_ERR_INVALID_ARG, "bad arguments");
  size_t need = 0;
  tr_reduce_workspace_size(n, TR_F32, &need);
  if (tr_status s = user::check_ws(e, need)) return s;
  return redk::launch<In, F>(f, d_x, n, RedOut{d_sum, d_min, d_max, TR_F64, ops}, e);
}

// Per segment [d_off[s], d_off[s+1]) of x: sum (FP64) / min / max (FP32) of f;
// offsets as for tr_segmented_reduce (checked on the device).
template <class F, class In>
tr_status segmented_reduce(const F& f, const In* d_x, int64_t n, const int64_t* d_off, int64_t n_seg, unsigned ops,
                           double* d_sums, float* d_mins, float* d_maxs, const tr_exec* e) {
  static_assert(is_hd_map<F>, "the map must declare static constexpr tr::HDC hdc = tr::HDC::HstDev");
  static_assert(user::is_storage<In>, "storage: float, __half or __nv_bfloat16");
  if (n < 0 || n_seg < 0 || ops == 0 || (ops & ~7u) || !d_off || (n > 0 && !d_x) ||
      ((ops & TR_SUM) && !d_sums) || ((ops & TR_MIN) && !d_mins) || ((ops & TR_MAX) && !d_maxs))
    return fail(TR_ERR_INVALID_ARG, "bad arguments");
  size_t need = 0;
  tr_segmented_reduce_workspace_size(n, n_seg, TR_F32, &need);
  if (tr_status s = user::check_ws(e, need)) return s;
  if (n_seg == 0) return TR_OK;
  return segk::launch<In, F>(f, d_x, n, d_off, n_seg, RedOut{d_sums, d_mins, d_maxs, TR_F64, ops}, e);
}

// Inclusive (or exclusive) scan of f into d_y (FP32, float-float within and
// between tiles); d_carry (nullable, device) is added to every output;
// the optional sum (FP64) / min / max of f come from the same pass.
template <class F, class In>
tr_status scan(const F& f, const In* d_x, float* d_y, int64_t n, const tr_exec* e, int mode = TR_SCAN_INCLUSIVE,
               const float* d_carry = nullptr, unsigned ops = 0, double* d_sum = nullptr, float* d_min = nullptr,
               float* d_max = nullptr) {
  static_assert(is_hd_map<F>, "the map must declare static constexpr tr::HDC hdc = tr::HDC::HstDev");
  static_assert(user::is_storage<In>, "storage: float, __half or __nv_bfloat16");
  if (n < 0 || (n > 0 && (!d_x || !d_y)) || (mode != TR_SCAN_INCLUSIVE && mode != TR_SCAN_EXCLUSIVE) ||
      (ops & ~7u) || ((ops & TR_SUM) && !d_sum) || ((ops & TR_MIN) && !d_min) || ((ops & TR_MAX) && !d_max))
    return fail(TR_ERR_INVALID_ARG, "bad arguments");
  size_t need = 0;
  tr_scan_workspace_size(n, TR_F32, TR_F32, &need);
  if (tr_status s = user::check_ws(e, need)) return s;
  if (n == 0 && ops == 0) return TR_OK;
  ScanOpts o;
  o.exclusive = mode == TR_SCAN_EXCLUSIVE;
  o.ops = ops;
  o.sum = d_sum;
  o.sum_t = TR_F64;
  o.mn = d_min;
  o.mx = d_max;
  return scank::launch<In, F, scank::OpF32>(f, d_x, d_y, n, d_carry, e, o);
}

}  // namespace tr

#endif /* TR_HPP */
