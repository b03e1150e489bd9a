// k_vandermonde.cu -- tr_vandermonde: many polynomials at many points,
// Y[i][j] = sum_k C[k][j] x_i^k, i.e. Y = V(x) C with V the Vandermonde matrix.
//
// TR_PREC_BF16X3 (tensor cores, tcgen05 + TMEM):
//   Split-BF16 product in the manner of Henry, Tang & Heinecke, "Leveraging
//   the bfloat16 artificial intelligence datatype for higher-precision
//   computations" (ARITH 2019): V = Vh + Vl and C = Ch + Cl with bf16 parts,
//   Y ~= Vh Ch + Vh Cl + Vl Ch accumulated in FP32 (the Vl Cl term is below
//   FP32 resolution of the result and is dropped).
//   * A persistent grid (two CTAs per SM, 128 threads each) walks 128 x 256
//     output tiles in column-tile-major order, so a CTA reloads its C tile
//     only when the column tile changes.
//   * V is never stored: each thread forms the 32 powers of its point in FP32
//     and writes their bf16 high and low parts to shared memory in the
//     tensor-core K-major core-matrix layout (8 rows x 16 bytes per core
//     matrix; K-adjacent core matrices 128 B apart, 8-row groups 512 B apart).
//   * One thread issues 6 tcgen05.mma (kind::f16, bf16 inputs, FP32
//     accumulate, M = 128, N = 256, K = 16 each) into a 256-column TMEM
//     accumulator and commits them to an mbarrier; the other CTA on the SM
//     overlaps its own tile with this one.
//   * The epilogue reads the accumulator with tcgen05.ld (32 lanes x 32
//     columns per warp and step), stages each 32 x 32 block in shared memory
//     in the 128-byte-swizzled layout and writes it with one 2-D TMA tensor
//     store (bulk async-groups, two staging blocks per warp in rotation).
//   Every mbarrier wait is bounded; on expiry the CTA records TR_ERR_TIMEOUT in
//   the workspace, stops, and still frees its TMEM.
//
// TR_PREC_FP32 (CUDA cores): the plain comparison -- one thread per
// polynomial holding its coefficients in registers, FP32 Horner with fma over
// a block of points, coalesced row stores.
#include <cuda_bf16.h>

#include "internal.h"

namespace tr {

namespace {

// ---------------------------------------------------------------- FP32 Horner
constexpr int kF32Threads = 256;
constexpr int kF32Points = 32;

__global__ void __launch_bounds__(kF32Threads) k_vander_fp32(const float* __restrict__ x, int64_t m,
                                                             const float* __restrict__ coef, int deg, int64_t npoly,
                                                             float* __restrict__ y) {
  const int64_t j = (int64_t)blockIdx.x * kF32Threads + threadIdx.x;
  float c[TR_MAX_DEGREE + 1];
#pragma unroll
  for (int k = 0; k <= TR_MAX_DEGREE; ++k) c[k] = (j < npoly && k <= deg) ? coef[(int64_t)k * npoly + j] : 0.0f;
  __shared__ float xs[kF32Points];
  for (int64_t i0 = (int64_t)blockIdx.y * kF32Points; i0 < m; i0 += (int64_t)gridDim.y * kF32Points) {
    __syncthreads();
    if (threadIdx.x < kF32Points) xs[threadIdx.x] = (i0 + threadIdx.x < m) ? x[i0 + threadIdx.x] : 0.0f;
    __syncthreads();
    if (j >= npoly) continue;
    for (int p = 0; p < kF32Points && i0 + p < m; ++p) {
      const float xi = xs[p];
      // leading zero coefficients leave the Horner value exactly unchanged
      float acc = c[TR_MAX_DEGREE];
#pragma unroll
      for (int k = TR_MAX_DEGREE - 1; k >= 0; --k) acc = __fmaf_rn(acc, xi, c[k]);
      __stcs(&y[(i0 + p) * npoly + j], acc);
    }
  }
}

// ------------------------------------------------------------- tcgen05 bf16x3
constexpr int kTcThreads = 128;
constexpr int kTileM = 128, kTileN = 256, kK = 32;
constexpr uint32_t kTmemCols = 256;
// K-major core-matrix layout (bytes): element (row r, k) of a tile at
// (r / 8) * kSBO + (k / 8) * kLBO + (r % 8) * 16 + (k % 8) * 2
constexpr uint32_t kLBO = 128;   // between K-adjacent core matrices
constexpr uint32_t kSBO = 512;   // between 8-row groups (K = 32: 4 core matrices)
constexpr uint32_t kABytes = kTileM * kK * 2;  // 8 KiB per bf16 part
constexpr uint32_t kBBytes = kTileN * kK * 2;  // 16 KiB per bf16 part
constexpr uint32_t kStageBytes = 32 * 32 * 4;                  // one warp's 32 x 32 FP32 output block
constexpr uint32_t kSmemUsed = 2 * kABytes + 2 * kBBytes + 4 * 2 * kStageBytes + 64;
// request more dynamic shared memory than used so that at most two CTAs share
// an SM: two 256-column accumulators fill the SM's 512 TMEM columns
constexpr uint32_t kSmemRequest = 96 * 1024;
constexpr long long kWaitLimit = 1ll << 26;  // mbarrier polls before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9 = 1, bits 10-12 = 1), both K-major (bits 15, 16 = 0),
// N >> 3 at bits 17-22, M >> 4 at bits 24-28
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTileN >> 3) << 17) |
                            ((uint32_t)(kTileM >> 4) << 24);

// shared-memory matrix descriptor: start >> 4 (bits 0-13), LBO >> 4
// (bits 16-29), SBO >> 4 (bits 32-45), descriptor version 1 (bits 46-47),
// base offset 0, no swizzle (bits 61-63 = 0)
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(kLBO >> 4) << 16) | ((uint64_t)(kSBO >> 4) << 32) |
         (1ull << 46);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(kIdesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Pack 8 floats as bf16 (round to nearest even).
__device__ __forceinline__ uint4 pack_bf16x8(const float* v) {
  uint32_t w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 b = __floats2bfloat162_rn(v[2 * i], v[2 * i + 1]);
    w[i] = *reinterpret_cast<const uint32_t*>(&b);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

// Split v into bf16 high part and bf16 remainder, both packed in K-major
// core-matrix layout for row `r` of a tile starting at hi / lo.
__device__ __forceinline__ void store_split_row(unsigned char* hi, unsigned char* lo, int r, const float* v) {
  float h[kK], l[kK];
#pragma unroll
  for (int k = 0; k < kK; ++k) {
    h[k] = __bfloat162float(__float2bfloat16_rn(v[k]));
    l[k] = v[k] - h[k];  // exact in FP32
  }
  const uint32_t row_off = (uint32_t)(r / 8) * kSBO + (uint32_t)(r % 8) * 16;
#pragma unroll
  for (int kc = 0; kc < kK / 8; ++kc) {
    *reinterpret_cast<uint4*>(hi + row_off + kc * kLBO) = pack_bf16x8(h + 8 * kc);
    *reinterpret_cast<uint4*>(lo + row_off + kc * kLBO) = pack_bf16x8(l + 8 * kc);
  }
}

__global__ void __launch_bounds__(kTcThreads, 1) k_vander_tc(const __grid_constant__ CUtensorMap ymap,
                                                             const float* __restrict__ x, int64_t m,
                                                             const float* __restrict__ coef, int deg, int64_t npoly,
                                                             WsHeader* hdr) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  unsigned char* sAh = base;
  unsigned char* sAl = sAh + kABytes;
  unsigned char* sBh = sAl + kABytes;
  unsigned char* sBl = sBh + kBBytes;
  unsigned char* sOut = sBl + kBBytes;  // 4 warps x 2 staging blocks, 1024-byte aligned
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sOut + 4 * 2 * kStageBytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t m_tiles = m / kTileM, n_tiles = npoly / kTileN, tiles = m_tiles * n_tiles;
  const int64_t t_begin = tiles * blockIdx.x / gridDim.x, t_end = tiles * (blockIdx.x + 1) / gridDim.x;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  uint32_t phase = 0;
  int64_t loaded_n = -1;
  bool ok = true;
  for (int64_t t = t_begin; t < t_end && ok; ++t) {
    const int64_t nt = t / m_tiles, mt = t % m_tiles;
    const int64_t m0 = mt * kTileM, n0 = nt * kTileN;
    if (nt != loaded_n) {  // C tile: columns n0 .. n0+255, powers 0 .. 31 (zero beyond deg)
      for (int half = 0; half < 2; ++half) {
        const int r = tid + half * kTcThreads;
        float v[kK];
#pragma unroll
        for (int k = 0; k < kK; ++k) v[k] = (k <= deg) ? __ldg(&coef[(int64_t)k * npoly + n0 + r]) : 0.0f;
        store_split_row(sBh, sBl, r, v);
      }
      loaded_n = nt;
    }
    {  // V tile: the 32 powers of point m0 + tid, by repeated FP32 multiplication
      const float xi = __ldg(&x[m0 + tid]);
      float v[kK];
      v[0] = 1.0f;
#pragma unroll
      for (int k = 1; k < kK; ++k) v[k] = v[k - 1] * xi;
      store_split_row(sAh, sAl, tid, v);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic-proxy smem writes -> tensor core
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t ah = smem_u32(sAh), al = smem_u32(sAl), bh = smem_u32(sBh), bl = smem_u32(sBl);
#pragma unroll
      for (int s = 0; s < 2; ++s)  // K = 16 per instruction: skip two core matrices per step
        mma_bf16(tmem, smem_desc(ah + s * 2 * kLBO), smem_desc(bh + s * 2 * kLBO), s > 0 ? 1u : 0u);
#pragma unroll
      for (int s = 0; s < 2; ++s) mma_bf16(tmem, smem_desc(ah + s * 2 * kLBO), smem_desc(bl + s * 2 * kLBO), 1u);
#pragma unroll
      for (int s = 0; s < 2; ++s) mma_bf16(tmem, smem_desc(al + s * 2 * kLBO), smem_desc(bh + s * 2 * kLBO), 1u);
      mma_commit(smem_u32(mbar));
    }
    long long polls = 0;
    while (!mbar_try_wait(smem_u32(mbar), phase)) {
      if (++polls > kWaitLimit) {
        ok = false;
        break;
      }
    }
    phase ^= 1u;
    if (!__syncthreads_and(ok ? 1 : 0)) {
      ok = false;
      if (tid == 0) set_status(hdr, TR_ERR_TIMEOUT, (uint32_t)t);
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: warp w owns TMEM lanes (rows) 32w .. 32w+31.  Each 32 x 32 block goes
    // registers -> swizzled shared staging (row r's 16-byte chunk q at q ^ (r % 8), the
    // 128-byte swizzle of the tensor map) -> one TMA tensor store issued by lane 0.
    // Two staging blocks per warp alternate; lane 0 waits until the store issued two
    // blocks earlier has finished reading its block before it is overwritten.
#pragma unroll 1
    for (int c = 0; c < kTileN / 32; ++c) {
      float v[32];
      tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 32), v);
      unsigned char* stg = sOut + (uint32_t)(warp * 2 + (c & 1)) * kStageBytes;
      if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 1;" ::: "memory");
      __syncwarp();
#pragma unroll
      for (int q = 0; q < 8; ++q)
        *reinterpret_cast<uint4*>(stg + lane * 128 + ((q ^ (lane & 7)) * 16)) = pack16(v + 4 * q);
      fence_async_smem();
      __syncwarp();
      if (lane == 0) {
        asm volatile(
            "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(&ymap),
            "r"((int)(n0 + c * 32)), "r"((int)(m0 + warp * 32)), "r"(smem_u32(stg))
            : "memory");
        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // TMEM and the A / B tiles are free for the next tile
  }
  if (lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // this warp's stores are done
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace

}  // namespace tr

using namespace tr;

extern "C" {

tr_status tr_vandermonde_workspace_size(size_t* bytes) {
  if (!bytes) return fail(TR_ERR_INVALID_ARG, "bytes is NULL");
  *bytes = kWsHeader;
  return TR_OK;
}

tr_status tr_vandermonde(const float* x, int64_t m, const float* coef, int32_t deg, int64_t npoly, int precision,
                         float* y, const tr_exec* e) {
  if (!e) return fail(TR_ERR_INVALID_ARG, "exec is NULL");
  if (m < 0 || npoly < 0) return fail(TR_ERR_INVALID_ARG, "m or npoly < 0");
  if (deg < 0 || deg > TR_MAX_DEGREE) return fail(TR_ERR_INVALID_ARG, "degree %d out of [0, %d]", deg, TR_MAX_DEGREE);
  if (precision != TR_PREC_BF16X3 && precision != TR_PREC_FP32) return fail(TR_ERR_INVALID_ARG, "precision %d", precision);
  if (m > 0 && npoly > 0 && (!x || !coef || !y)) return fail(TR_ERR_INVALID_ARG, "x, coef or y is NULL");
  if ((x && !aligned_to(x, 4)) || (coef && !aligned_to(coef, 4)) || (y && !aligned_to(y, 4)))
    return fail(TR_ERR_ALIGNMENT, "pointers must be 4-byte aligned");
  if (m == 0 || npoly == 0) return TR_OK;
  cudaStream_t st = stream_of(e);
  if (precision == TR_PREC_FP32) {
    if (ceil_div(npoly, kF32Threads) > 0x7FFFFFFF) return fail(TR_ERR_INVALID_ARG, "npoly too large");
    const dim3 grid((unsigned)ceil_div(npoly, kF32Threads), (unsigned)std::min<int64_t>(ceil_div(m, kF32Points), 65535));
    k_vander_fp32<<<grid, kF32Threads, 0, st>>>(x, m, coef, deg, npoly, y);
    return launch_status("k_vander_fp32");
  }
  if (m % kTileM || npoly % kTileN)
    return fail(TR_ERR_UNSUPPORTED, "bf16x3 tensor path needs m %% %d == 0 and npoly %% %d == 0", kTileM, kTileN);
  if (!aligned_to(y, 16)) return fail(TR_ERR_ALIGNMENT, "y must be 16-byte aligned for the tensor path");
  if (!e->workspace || e->workspace_bytes < (size_t)kWsHeader)
    return fail(TR_ERR_WORKSPACE, "the tensor path needs a %d-byte workspace (status word)", kWsHeader);
  static_assert(kSmemUsed + 1024 <= kSmemRequest, "shared memory budget");
  tr_status s = cuda_status(
      cudaFuncSetAttribute(k_vander_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemRequest),
      "cudaFuncSetAttribute(k_vander_tc)");
  if (s) return s;
  if (m > 0x7FFFFFFF || npoly > 0x7FFFFFFF) return fail(TR_ERR_INVALID_ARG, "m or npoly beyond 32-bit coordinates");
  CUtensorMap ymap;
  if ((s = make_tensor_map_2d(&ymap, y, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (uint64_t)npoly, (uint64_t)m,
                              (uint64_t)npoly * 4, 32, 32, CU_TENSOR_MAP_SWIZZLE_128B)))
    return s;
  const int64_t tiles = (m / kTileM) * (npoly / kTileN);
  const int64_t grid = std::min<int64_t>(tiles, 2 * (int64_t)dev_info().sm_count);
  k_vander_tc<<<(unsigned)grid, kTcThreads, kSmemRequest, st>>>(ymap, x, m, coef, deg, npoly, ws_header(e));
  return launch_status("k_vander_tc");
}

}  // extern "C"
