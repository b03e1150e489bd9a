// div_check.cu -- test-side CUDA checks of the library's division-free FP32
// quotient (div_hd / div_vec in hd.h and common.cuh) against the IEEE division
// (__fdiv_rn).  Built by tests/test_gpu_division.py into a small shared
// library; it is test infrastructure and no product code links it.
//
//   div_check_rcp_invariance : rcp.approx is sign- and scale-invariant over
//                              every normal input of the fast domain's range
//                              (rcp(-b) = -rcp(b), rcp(b 2^k) = rcp(b) 2^-k);
//   div_check_significands   : div_vec<2> (the packed path the kernels run)
//                              equals a / b, and div_vec_neg<2> equals
//                              -(a / b), for every pair of significands in
//                              [1, 2) x [b_first, b_first + b_count) x 2^-23;
//   div_check_values         : div_hd and div_vec<2> equal a / b, and
//                              div_vec_neg<2> equals -(a / b) (bitwise, NaN
//                              matched as NaN), on caller-supplied operands.
#include <cstdint>

#include "common.cuh"

// Result of a check (mirrored by the ctypes structure of the test).
struct Report {
  unsigned long long mismatches;
  unsigned int recorded;
  unsigned int pad;
  unsigned int a[16], b[16];
};

namespace {

__device__ void record(Report* r, float a, float b) {
  atomicAdd(&r->mismatches, 1ull);
  const unsigned k = atomicAdd(&r->recorded, 1u);
  if (k < 16) {
    r->a[k] = __float_as_uint(a);
    r->b[k] = __float_as_uint(b);
  }
}

__device__ bool same(float x, float y) {
  return __float_as_uint(x) == __float_as_uint(y) || (x != x && y != y);
}

__global__ void k_rcp(unsigned long long base, Report* rep) {
  const unsigned long long i = base + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (1ull << 32)) return;
  const unsigned u = (unsigned)i;
  const unsigned ex = (u >> 23) & 0xffu;
  if (ex < 2 || ex > 252) return;  // |b| in [2^-125, 2^126): reciprocals stay normal
  const float b = __uint_as_float(u);
  const float m = __uint_as_float((u & 0x807fffffu) | 0x3f800000u);  // sign * significand
  const float scale = __uint_as_float((unsigned)(254 - ex) << 23);  // 2^-(ex - 127), exact
  const float y = tr::rcp_approx(b);
  if (__float_as_uint(y) != __float_as_uint(__fmul_rn(tr::rcp_approx(m), scale)) ||
      __float_as_uint(tr::rcp_approx(-b)) != (__float_as_uint(y) ^ 0x80000000u))
    record(rep, b, m);
}

// one block per divisor significand, threads over the dividend significands
__global__ void __launch_bounds__(256) k_sig(unsigned b_first, Report* rep) {
  const float b = __uint_as_float(0x3f800000u | (b_first + blockIdx.x));
  for (unsigned j = 2 * threadIdx.x; j < (1u << 23); j += 512) {
    const float a[2] = {__uint_as_float(0x3f800000u | j), __uint_as_float(0x3f800000u | (j + 1))};
    const float bb[2] = {b, b};
    float q[2], nq[2];
    tr::div_vec<2>(a, bb, q);
    tr::div_vec_neg<2>(a, bb, nq, a[0], a[1]);  // a[0] < a[1], both in [1, 2)
    for (int t = 0; t < 2; ++t) {
      const unsigned ref = __float_as_uint(__fdiv_rn(a[t], b));
      if (__float_as_uint(q[t]) != ref || __float_as_uint(nq[t]) != (ref ^ 0x80000000u)) record(rep, a[t], b);
    }
  }
}

__global__ void k_values(const float* a, const float* b, int64_t n, Report* rep) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * i + 1 >= n + 1) return;
  const int64_t j = 2 * i + 1 < n ? 2 * i + 1 : 2 * i;  // odd n: the last pair repeats its element
  const float aa[2] = {a[2 * i], a[j]}, bb[2] = {b[2 * i], b[j]};
  float q[2], nq[2];
  tr::div_vec<2>(aa, bb, q);
  const float alo = fminf(fabsf(aa[0]), fabsf(aa[1])), ahi = fmaxf(fabsf(aa[0]), fabsf(aa[1]));
  // a NaN operand must fail the guard, as it does in the callers (their scans propagate NaN)
  const bool nan = aa[0] != aa[0] || aa[1] != aa[1];
  tr::div_vec_neg<2>(aa, bb, nq, nan ? __int_as_float(0x7fffffff) : alo, nan ? __int_as_float(0x7fffffff) : ahi);
  for (int t = 0; t < 2; ++t) {
    const float ref = __fdiv_rn(aa[t], bb[t]);
    if (!same(q[t], ref) || !same(tr::div_hd(aa[t], bb[t]), ref) || !same(nq[t], -ref)) record(rep, aa[t], bb[t]);
  }
}

int finish(Report* d, Report* h) {
  const cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return (int)e;
  cudaMemcpy(h, d, sizeof(Report), cudaMemcpyDeviceToHost);
  cudaFree(d);
  return 0;
}

}  // namespace

extern "C" {

int div_check_rcp_invariance(Report* out) {
  Report* d = nullptr;
  if (cudaMalloc(&d, sizeof(Report)) != cudaSuccess) return -1;
  cudaMemset(d, 0, sizeof(Report));
  for (unsigned long long base = 0; base < (1ull << 32); base += (1ull << 28))
    k_rcp<<<(1u << 28) / 256, 256>>>(base, d);
  return finish(d, out);
}

int div_check_significands(unsigned b_first, unsigned b_count, Report* out) {
  if (b_first >= (1u << 23) || b_count > (1u << 23) - b_first) return -2;
  Report* d = nullptr;
  if (cudaMalloc(&d, sizeof(Report)) != cudaSuccess) return -1;
  cudaMemset(d, 0, sizeof(Report));
  for (unsigned b0 = 0; b0 < b_count; b0 += 8192)
    k_sig<<<b_count - b0 < 8192 ? b_count - b0 : 8192, 256>>>(b_first + b0, d);
  return finish(d, out);
}

int div_check_values(const float* a, const float* b, int64_t n, Report* out) {
  Report* d = nullptr;
  if (n <= 0) return -2;
  if (cudaMalloc(&d, sizeof(Report)) != cudaSuccess) return -1;
  cudaMemset(d, 0, sizeof(Report));
  const int64_t pairs = (n + 1) / 2;
  k_values<<<(unsigned)((pairs + 255) / 256), 256>>>(a, b, n, d);
  return finish(d, out);
}

}  // extern "C"
