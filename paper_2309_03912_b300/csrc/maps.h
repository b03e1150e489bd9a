// maps.h -- the map family f, written once for host, device and compile time.
//
// Every functor is TR_HD + constexpr and declares `hdc = HDC::HstDev`, the
// host-device-compatibility tag of the paper's Sec. 4 helper; the
// compile-time checks assert tr::hdc<F> == HDC::HstDev for the whole family.
// The operation sequence of each map is fixed (explicit fused multiply-adds,
// one correctly rounded division where a quotient appears, div_hd) so that
// host code compiled with -ffp-contract=off, device code compiled with
// -fmad=false and constant evaluation on exactly representable inputs give
// identical bits.
//
//   Horner     p = c_d; p = fma(p, x, c_k), k = d-1 .. 0 (ascending c)
//   Rational   P(x) / Q(x), both by Horner, one correctly rounded division
//   NewtonCbrt y_0 = sign(x); y <- (2y + x / (y*y)) / 3, a fixed number of
//              steps; the result is the iterate (not cbrt(x))
//   Square     x * x
//   Xorshift32 Marsaglia, "Xorshift RNGs" (2003), shift triple 13/17/5
//   Splitmix32 Weyl increment floor(2^32/phi), then (z ^ z>>16) * m1,
//              (z ^ z>>13) * m2, z ^ z>>16 with m1, m2 the first 32 bits of
//              the fractional parts of sqrt(2) and sqrt(3), all mod 2^32
#pragma once

#include "hd.h"

namespace tr {

// Two maps at once.  On the device, FP32 Horner steps of two points run as one
// packed instruction (fma.rn.f32x2: each half is an IEEE fma, so results are
// bit-identical to two scalar fmas); elsewhere the scalar form is used.  The
// signature is the same in every pass (the paper's Sec. 2.4 rule); only the
// body differs.
#if defined(__CUDACC__)  // device helpers: declared in both nvcc passes, used in device code
__device__ __forceinline__ unsigned long long pack_f32x2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void unpack_f32x2(unsigned long long r, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}
__device__ __forceinline__ unsigned long long fma_f32x2(unsigned long long a, unsigned long long b,
                                                         unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long add_f32x2(unsigned long long a, unsigned long long b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
#endif

// Horner on two points with the same coefficients: (p0, p1) = (P(x0), P(x1)).
template <class T, int D>
TR_HD inline void horner_pair(const T* c, T x0, T x1, T& p0, T& p1) {
#if defined(__CUDA_ARCH__)
  if constexpr (std::is_same<T, float>::value) {
    const unsigned long long xx = pack_f32x2(x0, x1);
    unsigned long long p = pack_f32x2(c[D], c[D]);
#pragma unroll
    for (int k = D - 1; k >= 0; --k) p = fma_f32x2(p, xx, pack_f32x2(c[k], c[k]));
    unpack_f32x2(p, p0, p1);
    return;
  }
#endif
  p0 = c[D];
  p1 = c[D];
  for (int k = D - 1; k >= 0; --k) {
    p0 = fma_hd(p0, x0, c[k]);
    p1 = fma_hd(p1, x1, c[k]);
  }
}

// Trait: does map F provide eval2 (two points per call)?  Member detection in
// the manner of the paper's has_xxx helper (Sec. 4).
template <class F, class = void>
struct has_eval2 : std::false_type {};
template <class F>
struct has_eval2<F, std::void_t<decltype(&F::eval2)>> : std::true_type {};

template <class T>
struct Identity {
  static constexpr HDC hdc = HDC::HstDev;
  TR_HD constexpr T operator()(T x) const { return x; }
};

template <class T>
struct Square {
  static constexpr HDC hdc = HDC::HstDev;
  TR_HD constexpr T operator()(T x) const { return x * x; }
};

// Horner's rule on d+1 ascending coefficients held anywhere addressable.
template <class T>
TR_HD constexpr T horner_eval(const T* c, int d, T x) {
  T p = c[d];
  for (int k = d - 1; k >= 0; --k) p = fma_hd(p, x, c[k]);
  return p;
}

// Compile-time degree D: coefficients by value (registers on the device).
template <class T, int D>
struct Horner {
  static constexpr HDC hdc = HDC::HstDev;
  T c[D + 1];
  TR_HD constexpr T operator()(T x) const {
    T p = c[D];
#pragma unroll
    for (int k = D - 1; k >= 0; --k) p = fma_hd(p, x, c[k]);
    return p;
  }
  TR_HD void eval2(T x0, T x1, T& y0, T& y1) const { horner_pair<T, D>(c, x0, x1, y0, y1); }
};

// Run-time degree: coefficients by pointer.
template <class T>
struct HornerN {
  static constexpr HDC hdc = HDC::HstDev;
  const T* c;
  int d;
  TR_HD constexpr T operator()(T x) const { return horner_eval(c, d, x); }
};

template <class T, int DP, int DQ>
struct Rational {
  static constexpr HDC hdc = HDC::HstDev;
  T p[DP + 1];
  T q[DQ + 1];
  TR_HD constexpr T operator()(T x) const {
    T a = p[DP];
#pragma unroll
    for (int k = DP - 1; k >= 0; --k) a = fma_hd(a, x, p[k]);
    T b = q[DQ];
#pragma unroll
    for (int k = DQ - 1; k >= 0; --k) b = fma_hd(b, x, q[k]);
    return div_hd(a, b);
  }
  TR_HD void eval2(T x0, T x1, T& y0, T& y1) const {
    T a0, a1, b0, b1;
    horner_pair<T, DP>(p, x0, x1, a0, a1);
    horner_pair<T, DQ>(q, x0, x1, b0, b1);
    y0 = div_hd(a0, b0);
    y1 = div_hd(a1, b1);
  }
};

template <class T>
struct RationalN {
  static constexpr HDC hdc = HDC::HstDev;
  const T* p;
  const T* q;
  int dp, dq;
  TR_HD constexpr T operator()(T x) const { return div_hd(horner_eval(p, dp, x), horner_eval(q, dq, x)); }
};

// ITERS >= 0: fixed step count; ITERS < 0: run-time count in `iters`.
template <class T, int ITERS>
struct NewtonCbrt {
  static constexpr HDC hdc = HDC::HstDev;
  int iters = ITERS;
  TR_HD constexpr T operator()(T x) const {
    T y = copysign_one(x);
    const int n = ITERS >= 0 ? ITERS : iters;
    for (int k = 0; k < n; ++k) {
      const T s = fma_hd(T(2), y, div_hd(x, y * y));  // 2y is exact, so this is RN(2y + x/y^2)
      if constexpr (std::is_same<T, float>::value) {
        y = div3_hd(s);  // = RN(s / 3), division-free
      } else {
        y = s / T(3);
      }
    }
    return y;
  }
};

struct Xorshift32 {
  static constexpr HDC hdc = HDC::HstDev;
  TR_HD constexpr uint32_t operator()(uint32_t x) const {
    x ^= x << 13;
    x ^= x >> 17;
    x ^= x << 5;
    return x;
  }
};

struct Splitmix32 {
  static constexpr HDC hdc = HDC::HstDev;
  static constexpr uint32_t kWeyl = 0x9E3779B9u;  // floor(2^32 / golden ratio)
  static constexpr uint32_t kM1 = 0x6A09E667u;    // frac(sqrt 2) * 2^32
  static constexpr uint32_t kM2 = 0xBB67AE85u;    // frac(sqrt 3) * 2^32
  TR_HD constexpr uint32_t operator()(uint32_t x) const {
    uint32_t z = x + kWeyl;
    z = (z ^ (z >> 16)) * kM1;
    z = (z ^ (z >> 13)) * kM2;
    return z ^ (z >> 16);
  }
};

}  // namespace tr
