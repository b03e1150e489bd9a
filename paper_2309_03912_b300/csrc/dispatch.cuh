// dispatch.cuh -- run-time (dtype, map) -> template instantiation.
//
// Each kernel family is instantiated for a fixed set of map types: the
// fixed-degree forms used by the benchmark workloads (degree-8 Horner,
// degree-6/6 rational) keep their coefficients in registers; every other
// degree runs through the run-time-degree forms.  `fn` is a generic host
// lambda receiving a value of the storage type and of the map type.
#pragma once

#include "internal.h"

namespace tr {

template <class In, class Fn>
tr_status dispatch_float_map(const MapParams& P, Fn&& fn) {
  using C = typename Storage<In>::C;
  switch (P.kind) {
    case TR_MAP_IDENTITY: return fn(In{}, Identity<C>{});
    case TR_MAP_SQUARE: return fn(In{}, Square<C>{});
    case TR_MAP_HORNER:
      if (P.deg_p == 8) return fn(In{}, Horner<C, 8>{});
      return fn(In{}, HornerN<C>{});
    case TR_MAP_RATIONAL:
      if (P.deg_p == 6 && P.deg_q == 6) return fn(In{}, Rational<C, 6, 6>{});
      return fn(In{}, RationalN<C>{});
    case TR_MAP_NEWTON_CBRT: return fn(In{}, NewtonCbrt<C, -1>{});
    default: return fail(TR_ERR_UNSUPPORTED, "map kind %d for float input", P.kind);
  }
}

template <class Fn>
tr_status dispatch_u32_map(const MapParams& P, Fn&& fn) {
  switch (P.kind) {
    case TR_MAP_IDENTITY: return fn(uint32_t{}, Identity<uint32_t>{});
    case TR_MAP_XORSHIFT32: return fn(uint32_t{}, Xorshift32{});
    case TR_MAP_SPLITMIX32: return fn(uint32_t{}, Splitmix32{});
    default: return fail(TR_ERR_UNSUPPORTED, "map kind %d for u32 input", P.kind);
  }
}

// f16 / bf16 / f32 storage with FP32 compute
template <class Fn>
tr_status dispatch_float_storage(tr_dtype xt, const MapParams& P, Fn&& fn) {
  switch (xt) {
    case TR_F16: return dispatch_float_map<__half>(P, fn);
    case TR_BF16: return dispatch_float_map<__nv_bfloat16>(P, fn);
    case TR_F32: return dispatch_float_map<float>(P, fn);
    default: return fail(TR_ERR_UNSUPPORTED, "storage dtype %d", xt);
  }
}

// every storage type: f16 / bf16 / f32 / f64 / u32
template <class Fn>
tr_status dispatch_any(tr_dtype xt, const MapParams& P, Fn&& fn) {
  if (xt == TR_U32) return dispatch_u32_map(P, fn);
  if (xt == TR_F64) return dispatch_float_map<double>(P, fn);
  return dispatch_float_storage(xt, P, fn);
}

}  // namespace tr
