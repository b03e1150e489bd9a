// user_map_check.cu -- test-side maps written by a "user" of libtr and run
// through the C++ entry points of tr.hpp (the library's kernel templates,
// instantiated here).  Built by tests/test_gpu_user_maps.py; test
// infrastructure only.
//
//   * UserHorner8: a hand-written degree-8 Horner polynomial (the same fma
//     sequence as the family's Horner map);
//   * UserRational: P/Q of any degrees up to 15 with the library's correctly
//     rounded division helper;
//   * a __host__ __device__ lambda computing fma(x, x, 1) (= Horner [1, 0, 1]).
// Compile-time checks (the paper's Sec. 2.6 and Sec. 4): the maps evaluate in
// constant expressions, the hdc trait marks the tagged maps host-device and an
// untagged functor host-only.
#include <cstdint>

#include "tr.hpp"

struct UserHorner8 {
  static constexpr tr::HDC hdc = tr::HDC::HstDev;
  float c[9];
  TR_HD constexpr float operator()(float x) const {
    float p = c[8];
    for (int k = 7; k >= 0; --k) p = tr::fma_hd(p, x, c[k]);
    return p;
  }
};

struct UserRational {
  static constexpr tr::HDC hdc = tr::HDC::HstDev;
  float p[16], q[16];
  int dp, dq;
  TR_HD constexpr float operator()(float x) const {
    float a = p[dp], b = q[dq];
    for (int k = dp - 1; k >= 0; --k) a = tr::fma_hd(a, x, p[k]);
    for (int k = dq - 1; k >= 0; --k) b = tr::fma_hd(b, x, q[k]);
    return tr::div_hd(a, b);
  }
};

struct Untagged {
  TR_HD float operator()(float x) const { return x; }
};

// compile time: evaluation in a constant expression (exactly representable
// intermediate values, so the unfused a * b + c of constant evaluation equals
// the fused result) and the trait
constexpr UserHorner8 kH{{1.0f, 2.0f, 3.0f, 0.0f, 0.0f, 0.0f, 0.0f, 0.0f, 1.0f}};
static_assert(kH(2.0f) == 1.0f + 4.0f + 12.0f + 256.0f, "constexpr evaluation of a user map");
constexpr UserRational kR{{3.0f, 1.0f}, {2.0f}, 1, 0};
static_assert(kR(5.0f) == 4.0f, "constexpr evaluation of a user rational map");
static_assert(tr::is_hd_map<UserHorner8> && tr::is_hd_map<UserRational>, "tagged maps are host-device");
static_assert(!tr::is_hd_map<Untagged>, "an untagged functor is host-only (tr::reduce would reject it)");

namespace {
UserHorner8 horner8(const double* c) {
  UserHorner8 h{};
  for (int k = 0; k <= 8; ++k) h.c[k] = (float)c[k];
  return h;
}
UserRational rational(const double* p, int dp, const double* q, int dq) {
  UserRational r{};
  for (int k = 0; k <= dp; ++k) r.p[k] = (float)p[k];
  for (int k = 0; k <= dq; ++k) r.q[k] = (float)q[k];
  r.dp = dp;
  r.dq = dq;
  return r;
}
tr_exec exec_of(void* ws, size_t ws_bytes) { return tr_exec{nullptr, ws, ws_bytes, 0u, 0, -1}; }
}  // namespace

extern "C" {

// Host evaluation of UserHorner8 (the same function compiled for the host).
void user_horner8_host(const double* c, const float* x, float* y, int64_t n) {
  const UserHorner8 h = horner8(c);
  for (int64_t i = 0; i < n; ++i) y[i] = h(x[i]);
}

int user_horner8_map(const double* c, const float* x, float* y, int64_t n) {
  const tr_exec e = exec_of(nullptr, 0);
  int s = tr::map(horner8(c), x, y, n, &e);
  return s ? s : (int)cudaStreamSynchronize(nullptr);
}

int user_horner8_reduce(const double* c, const float* x, int64_t n, double* sum, float* mn, float* mx, void* ws,
                        size_t ws_bytes) {
  const tr_exec e = exec_of(ws, ws_bytes);
  int s = tr::reduce(horner8(c), x, n, TR_SUM | TR_MIN | TR_MAX, sum, mn, mx, &e);
  return s ? s : (int)tr_check(&e);
}

int user_rational_segreduce_f16(const double* p, int dp, const double* q, int dq, const __half* x, int64_t n,
                                const int64_t* off, int64_t nseg, double* sums, float* mins, float* maxs, void* ws,
                                size_t ws_bytes) {
  const tr_exec e = exec_of(ws, ws_bytes);
  int s = tr::segmented_reduce(rational(p, dp, q, dq), x, n, off, nseg, TR_SUM | TR_MIN | TR_MAX, sums, mins, maxs,
                               &e);
  return s ? s : (int)tr_check(&e);
}

int user_lambda_scan(const float* x, float* y, int64_t n, int exclusive, double* sum, float* mn, float* mx, void* ws,
                     size_t ws_bytes) {
  const tr_exec e = exec_of(ws, ws_bytes);
  const auto f = tr::hd_lambda([] __host__ __device__(float v) { return tr::fma_hd(v, v, 1.0f); });
  static_assert(tr::is_hd_map<decltype(f)>, "the lambda wrapper carries the tag");
  int s = tr::scan(f, x, y, n, &e, exclusive ? TR_SCAN_EXCLUSIVE : TR_SCAN_INCLUSIVE, nullptr,
                   TR_SUM | TR_MIN | TR_MAX, sum, mn, mx);
  return s ? s : (int)tr_check(&e);
}

}  // extern "C"
