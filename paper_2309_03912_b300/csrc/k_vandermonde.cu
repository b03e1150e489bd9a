// k_vandermonde.cu -- tr_vandermonde: many polynomials at many points,
// Y[i][j] = sum_k C[k][j] x_i^k, i.e. Y = V(x) C with V the Vandermonde matrix,
// written out (FP32 or BF16) and/or reduced per column (polynomial) to its sum,
// minimum and maximum over the points.
//
// Split-BF16 on the tensor cores (tcgen05 + TMEM), in the manner of Henry,
// Tang & Heinecke, "Leveraging the bfloat16 artificial intelligence datatype
// for higher-precision computations" (ARITH 2019): every FP32 value v is
// carried as bf16 parts v = v1 + v2 (+ v3), and the product keeps the terms
// whose parts sum to at most the split's order -- bf16x3: V1C1 + V1C2 + V2C1
// (about 2^-16 relative); bf16x6: also V1C3 + V2C2 + V3C1 (about FP32
// accuracy) -- accumulated in FP32 in tensor memory.
//   * A persistent grid (two CTAs per SM, 128 threads each) walks 128 x 256
//     output tiles in column-tile-major order, so a CTA reloads its C tile
//     only when the column tile changes.
//   * V is never stored: each thread forms the 32 powers of its point in FP32
//     (zero above the degree) and writes their bf16 parts to shared memory in
//     the tensor-core K-major core-matrix layout (8 rows x 16 bytes per core
//     matrix; K-adjacent core matrices 128 B apart, 8-row groups 512 B apart).
//   * One thread issues the products' tcgen05.mma (kind::f16, bf16 inputs,
//     FP32 accumulate, M = 128, N = 256, K = 16 each) into a 256-column TMEM
//     accumulator and commits them to an mbarrier; the other CTA on the SM
//     overlaps its own tile with this one.
//   * The epilogue reads the accumulator with tcgen05.ld (32 lanes x 32
//     columns per warp and step) and stages each 32 x 32 block in shared
//     memory (128-byte swizzle), from where
//       - FP32 Y leaves by one 2-D TMA tensor store (bulk async-groups, two
//         staging blocks per warp in rotation; the tensor map clips rows and
//         columns beyond m and npoly);
//       - BF16 Y is rounded (nearest even) and leaves by coalesced 16-byte
//         stores from a second, 64-byte-swizzled staging block;
//       - the column reduction reads the block column-wise: each lane takes
//         one column's 32 rows (conflict-free under the swizzle) and folds
//         them into its running compensated sum, minimum and maximum, so one
//         lane owns 8 of the tile's 256 columns across the CTA's row tiles.
//     When the CTA's column tile changes, its four warps' running results are
//     combined in FP64 and written to a workspace slot (CTA + column tile),
//     and a second small kernel joins each column's slots in CTA order, in
//     FP64: deterministic results.
//   Every mbarrier wait is bounded by %globaltimer; on expiry the CTA records
//   TR_ERR_TIMEOUT, waits once more (bounded) for the committed products to
//   drain, stops, and still frees its TMEM.
//
// TR_PREC_FP32 (CUDA cores): the plain comparison -- one thread per
// polynomial holding its coefficients in registers, FP32 Horner with fma over
// a block of points, coalesced row stores.
#include <cuda_bf16.h>

#include <cstring>

#include "accum.cuh"
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

// ------------------------------------------------------------- tcgen05 split-bf16
constexpr int kTcThreads = 256;  // 8 warps: warps w and w + 4 share TMEM lanes 32 (w % 4) ..
constexpr int kTcWarps = kTcThreads / 32;
constexpr int kTileM = 128, kTileN = 256, kK = 32;
constexpr uint32_t kTmemCols = 256;
// K-major core-matrix layout (bytes): element (row r, k) of a tile at
// (r / 8) * kSBO + (k / 8) * kLBO + (r % 8) * 16 + (k % 8) * 2
constexpr uint32_t kLBO = 128;   // between K-adjacent core matrices
constexpr uint32_t kSBO = 512;   // between 8-row groups (K = 32: 4 core matrices)
constexpr uint32_t kABytes = kTileM * kK * 2;  // 8 KiB per bf16 part
constexpr uint32_t kBBytes = kTileN * kK * 2;  // 16 KiB per bf16 part
constexpr uint32_t kStageBytes = 32 * 32 * 4;  // one warp's 32 x 32 FP32 block
constexpr uint32_t kStageBf16 = 32 * 32 * 2;   // the same in BF16
constexpr uint64_t kMmaWaitNs = 1000000000ull; // 1 s for a tile's products
constexpr int kMaxTcGrid = 512;                // workspace slots are sized for this many CTAs

enum { kOutNone = 0, kOutF32 = 1, kOutBf16 = 2 };

// Shared-memory layout of a CTA: NS A parts, NS B parts, one 4 KiB staging
// block per warp (FP32 for the TMA store and the column reads; the BF16 output
// block overlays it), mbarrier and TMEM slot.  The request is at least 80 KiB
// so that at most two CTAs share an SM: two 256-column accumulators fill its
// 512 TMEM columns.
template <int NS, int OUT, bool RED>
struct TcLayout {
  static constexpr uint32_t a = 0;
  static constexpr uint32_t b = NS * kABytes;
  static constexpr uint32_t stage = b + NS * kBBytes;
  static constexpr uint32_t bar = stage + kTcWarps * kStageBytes;
  static constexpr uint32_t used = bar + 64;
  static constexpr uint32_t request = used + 1024 > 80 * 1024 ? used + 1024 : 80 * 1024;
  static_assert(request <= 110 * 1024, "two CTAs per SM");
  static_assert(kTcWarps * kStageBytes >= kTcWarps * 4 * 32 * sizeof(double) * 2, "room for the column combination");
};

// Per-column partial result of one CTA (one workspace slot entry).
struct ColPart {
  double sum;
  float mn, mx;
};

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

// 32 lanes x 64 columns: lane l of the warp receives columns 0..63 of its TMEM lane.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, float* v) {
  uint32_t r[64];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,"
      "%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]),
        "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]),
        "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]),
        "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]),
        "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 64; ++i) v[i] = __uint_as_float(r[i]);
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

// Two floats as bf16x2 (round to nearest even): `hi` in the upper half.
__device__ __forceinline__ uint32_t cvt_bf16x2(float hi, float lo) {
  uint32_t d;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(d) : "f"(hi), "f"(lo));
  return d;
}

// Split v into NS bf16 parts (v = p0 + p1 + ..., each remainder exact in FP32)
// and store them in K-major core-matrix layout for row `r` of tiles starting at
// part[0], part[0] + stride, ...  Powers are handled in pairs: one packed
// conversion rounds both, the pair word is stored as is, and its two bf16
// values (widened by shifts) leave the remainders by one packed subtraction.
// Only the k-chunks [KC0, KC0 + NKC) of 8 powers each are written (the row's
// two halves can be written by two threads).
template <int NS, int KC0 = 0, int NKC = kK / 8>
__device__ __forceinline__ void store_split_row(unsigned char* part0, uint32_t stride, int r, const float* v) {
  constexpr int k0 = KC0 * 8, np = NKC * 4;  // pairs of powers
  unsigned long long rem[np];
#pragma unroll
  for (int i = 0; i < np; ++i) rem[i] = pack_f32x2(v[k0 + 2 * i], v[k0 + 2 * i + 1]);
  const uint32_t row_off = (uint32_t)(r / 8) * kSBO + (uint32_t)(r % 8) * 16;
#pragma unroll
  for (int p = 0; p < NS; ++p) {
    uint32_t w[np];
#pragma unroll
    for (int i = 0; i < np; ++i) {
      float lo, hi;
      unpack_f32x2(rem[i], lo, hi);
      w[i] = cvt_bf16x2(hi, lo);
      if (p + 1 < NS)  // exact in FP32
        rem[i] = sub_f32x2(rem[i], pack_f32x2(__uint_as_float(w[i] << 16), __uint_as_float(w[i] & 0xFFFF0000u)));
    }
#pragma unroll
    for (int kc = 0; kc < NKC; ++kc)
      *reinterpret_cast<uint4*>(part0 + p * stride + row_off + (KC0 + kc) * kLBO) =
          make_uint4(w[4 * kc], w[4 * kc + 1], w[4 * kc + 2], w[4 * kc + 3]);
  }
}

// The tile ranges of a CTA (contiguous, column-tile-major): [t_begin, t_end).
__host__ __device__ __forceinline__ int64_t tc_tile_begin(int64_t tiles, int64_t cta, int64_t grid) {
  return tiles * cta / grid;
}

template <int NS, int OUT, bool RED>
__global__ void __launch_bounds__(kTcThreads, 2) k_vander_tc(const __grid_constant__ CUtensorMap ymap,
                                                             const float* __restrict__ x, int64_t m,
                                                             const float* __restrict__ coef, int deg, int64_t npoly,
                                                             __nv_bfloat16* __restrict__ ybf, ColPart* parts,
                                                             WsHeader* hdr) {
  using L = TcLayout<NS, OUT, RED>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  unsigned char* sA = base + L::a;
  unsigned char* sB = base + L::b;
  unsigned char* sF = base + L::stage;  // 1024-byte aligned (part sizes are multiples of 8 KiB)
  uint64_t* mbar = reinterpret_cast<uint64_t*>(base + L::bar);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t m_tiles = (m + kTileM - 1) / kTileM, n_tiles = (npoly + kTileN - 1) / kTileN;
  const int64_t tiles = m_tiles * n_tiles;
  const int64_t t_begin = tc_tile_begin(tiles, blockIdx.x, gridDim.x),
                t_end = tc_tile_begin(tiles, blockIdx.x + 1, gridDim.x);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(smem_u32(mbar), 1);
    mbar_init_fence();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // warp w works on TMEM lanes (rows) 32 (w % 4) .. + 31 and on the column half w / 4 of the tile
  const int lane_grp = warp & 3, half = warp >> 2;
  // running column results of this lane: column 128 half + 32 c + lane of the current column
  // tile, over this warp's rows of every row tile seen so far
  float cs_hi[4], cs_lo[4], cmn[4], cmx[4];
  auto reset_cols = [&]() {
#pragma unroll
    for (int c = 0; c < 4; ++c) cs_hi[c] = cs_lo[c] = 0.0f, cmn[c] = INFINITY, cmx[c] = -INFINITY;
  };
  // the CTA's results for column tile nt into its workspace slot (CTA + nt): the four row warps
  // of each column combined in FP64, in row order, through the staging blocks (every TMA store
  // has finished reading them)
  auto flush_cols = [&](int64_t nt) {
    if constexpr (OUT == kOutF32) {
      if (lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
    }
    __syncthreads();
    ColPart* cp = reinterpret_cast<ColPart*>(sF);  // [warp][c][lane]
#pragma unroll
    for (int c = 0; c < 4; ++c)
      cp[(warp * 4 + c) * 32 + lane] = ColPart{(double)cs_hi[c] + (double)cs_lo[c], cmn[c], cmx[c]};
    __syncthreads();
    {
      const int col = tid, h = col / 128, c = (col % 128) / 32, l = col % 32;  // kTcThreads == kTileN
      double sum = 0.0;
      float mn = INFINITY, mx = -INFINITY;
      for (int g = 0; g < 4; ++g) {
        const ColPart q = cp[((h * 4 + g) * 4 + c) * 32 + l];
        sum += q.sum;
        mn = fminf(mn, q.mn);
        mx = fmaxf(mx, q.mx);
      }
      parts[(blockIdx.x + nt) * kTileN + col] = ColPart{sum, mn, mx};
    }
    __syncthreads();
    reset_cols();
  };
  if constexpr (RED) reset_cols();

  uint32_t phase = 0;
  int64_t loaded_n = -1;
  bool ok = true;
  // point m0 + tid % 128 of a tile, loaded one tile ahead so that its latency hides behind the
  // products and the epilogue of the tile before
  auto load_x = [&](int64_t t) {
    const int64_t i = (t % m_tiles) * kTileM + (tid & (kTileM - 1));
    return t < t_end && i < m ? __ldg(&x[i]) : 0.0f;
  };
  float x_next = load_x(t_begin);
  for (int64_t t = t_begin; t < t_end && ok; ++t) {
    const int64_t nt = t / m_tiles, mt = t % m_tiles;
    const int64_t m0 = mt * kTileM, n0 = nt * kTileN;
    if (nt != loaded_n) {
      if constexpr (RED) {
        if (loaded_n >= 0) flush_cols(loaded_n);
      }
      // C tile: columns n0 .. n0+255 (zero beyond npoly), powers 0 .. 31 (zero beyond deg), one
      // column per thread
      {
        const bool in = n0 + tid < npoly;
        float v[kK];
#pragma unroll
        for (int k = 0; k < kK; ++k) v[k] = (in && k <= deg) ? __ldg(&coef[(int64_t)k * npoly + n0 + tid]) : 0.0f;
        store_split_row<NS>(sB, kBBytes, tid, v);
      }
      loaded_n = nt;
    }
    {  // V tile: the powers of point m0 + tid % 128 by repeated FP32 multiplication, zero above
       // deg; the two halves of the block write powers 0..15 and 16..31
      const int r = tid & (kTileM - 1);
      const float xi = x_next;
      x_next = load_x(t + 1);
      float v[kK];
      v[0] = 1.0f;
#pragma unroll
      for (int k = 1; k < kK; ++k) v[k] = k <= deg ? v[k - 1] * xi : 0.0f;
      if (tid < kTileM)
        store_split_row<NS, 0, 2>(sA, kABytes, r, v);
      else
        store_split_row<NS, 2, 2>(sA, kABytes, r, v);
    }
    fence_async_smem();  // generic-proxy smem writes -> tensor core
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
      // the products V_i C_j with i + j <= NS - 1 (parts numbered from 0), largest first;
      // K = 16 per instruction: two steps of two core matrices each
      bool first = true;
#pragma unroll
      for (int d = 0; d < NS; ++d)
#pragma unroll
        for (int i = 0; i <= d; ++i) {
          const uint32_t ai = a0 + i * kABytes, bj = b0 + (d - i) * kBBytes;
#pragma unroll
          for (int s = 0; s < 2; ++s) {
            mma_bf16(tmem, smem_desc(ai + s * 2 * kLBO), smem_desc(bj + s * 2 * kLBO), first ? 0u : 1u);
            first = false;
          }
        }
      mma_commit(smem_u32(mbar));
    }
    if (!mbar_wait_until(smem_u32(mbar), phase, kMmaWaitNs)) ok = false;
    phase ^= 1u;
    if (!__syncthreads_and(ok ? 1 : 0)) {
      ok = false;
      if (tid == 0) set_status(hdr, TR_ERR_TIMEOUT, (uint32_t)t);
      break;
    }
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // epilogue: warp w reads its 32 TMEM lanes (rows 32 (w % 4) ..) for the 128 columns of its
    // half, 64 columns per TMEM load handled as two 32 x 32 blocks; the steps are unrolled so that
    // the running column results stay in registers and the blocks' dependency chains overlap
    const int64_t row0 = m0 + lane_grp * 32;
    const int valid_rows = (int)imax<int64_t>(0, imin<int64_t>(32, m - row0));
    unsigned char* stg = sF + (uint32_t)warp * kStageBytes;
#pragma unroll
    for (int cp = 0; cp < 2; ++cp) {
      float v64[64];
      tmem_ld64(tmem + ((uint32_t)(lane_grp * 32) << 16) + (uint32_t)(half * 128 + cp * 64), v64);
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int c = 2 * cp + hh;  // block of this warp's half
        const float* v = v64 + 32 * hh;
        const int64_t col0 = n0 + half * 128 + c * 32;
        if constexpr (OUT == kOutF32 || RED) {
          // row `lane`'s 16-byte chunk q at chunk q ^ (lane % 8): the 128-byte swizzle of the tensor map
          if (OUT == kOutF32 && lane == 0) asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
          __syncwarp();
#pragma unroll
          for (int q = 0; q < 8; ++q)
            *reinterpret_cast<uint4*>(stg + lane * 128 + ((q ^ (lane & 7)) * 16)) = pack16(v + 4 * q);
          if constexpr (OUT == kOutF32) {
            fence_async_smem();
            __syncwarp();
            if (lane == 0) {
              if (valid_rows > 0 && col0 < npoly) {
                asm volatile(
                    "cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(&ymap),
                    "r"((int)col0), "r"((int)row0), "r"(smem_u32(stg))
                    : "memory");
                asm volatile("cp.async.bulk.commit_group;" ::: "memory");
              }
            }
          } else {
            __syncwarp();
          }
          if constexpr (RED) {
            // column `lane` of the block, rows 0..31: element (r, lane) at
            // r * 128 + ((lane / 4) ^ (r % 8)) * 16 + (lane % 4) * 4 (one bank per lane)
            const float* colp = reinterpret_cast<const float*>(stg);
            float e[32];
#pragma unroll
            for (int r = 0; r < 32; ++r) e[r] = colp[r * 32 + (((lane >> 2) ^ (r & 7)) << 2) + (lane & 3)];
            float tmn, tmx;
            if (valid_rows == 32) {
              tmn = min3f(e[0], e[1], e[2]);
              tmx = max3f(e[0], e[1], e[2]);
#pragma unroll
              for (int r = 3; r + 1 < 32; r += 2) {
                tmn = min3f(tmn, e[r], e[r + 1]);
                tmx = max3f(tmx, e[r], e[r + 1]);
              }
              tmn = fminf(tmn, e[31]);
              tmx = fmaxf(tmx, e[31]);
            } else {  // the last row tile: rows beyond m are left out
              tmn = INFINITY;
              tmx = -INFINITY;
#pragma unroll
              for (int r = 0; r < 32; ++r) {
                const bool in = r < valid_rows;
                tmn = fminf(tmn, in ? e[r] : INFINITY);
                tmx = fmaxf(tmx, in ? e[r] : -INFINITY);
                e[r] = in ? e[r] : 0.0f;
              }
            }
            const float ts = pairwise<32>(e);
            // compensated running sum (Kahan) of the per-tile partial sums
            const float yk = ts - (-cs_lo[c]);
            const float tt = cs_hi[c] + yk;
            cs_lo[c] = -((tt - cs_hi[c]) - yk);
            cs_hi[c] = tt;
            cmn[c] = fminf(cmn[c], tmn);
            cmx[c] = fmaxf(cmx[c], tmx);
          }
        }
        if constexpr (OUT == kOutBf16) {
          // row `lane`'s four 16-byte chunks (8 bf16 each) at chunk q ^ ((lane / 2) % 4) of the
          // warp's staging block (64-byte rows, conflict-free writes; after the column reads);
          // then 8 rows per instruction leave as 16-byte stores
          __syncwarp();
#pragma unroll
          for (int q = 0; q < 4; ++q)
            *reinterpret_cast<uint4*>(stg + lane * 64 + ((q ^ ((lane >> 1) & 3)) * 16)) = pack_bf16x8(v + 8 * q);
          __syncwarp();
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const int r = i * 8 + (lane >> 2), q = lane & 3;
            const uint4 w = *reinterpret_cast<const uint4*>(stg + r * 64 + ((q ^ ((r >> 1) & 3)) * 16));
            const int64_t col = col0 + q * 8;
            if (r < valid_rows && col < npoly) st_stream(ybf + (row0 + r) * npoly + col, w);
          }
        }
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();  // TMEM and the A / B tiles are free for the next tile
  }
  if constexpr (RED) {
    if (ok && loaded_n >= 0) flush_cols(loaded_n);
  }
  if (!ok) mbar_wait_until(smem_u32(mbar), phase ^ 1u, kMmaWaitNs);  // let committed products drain
  if (OUT == kOutF32 && lane == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // stores done
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

// Second launch of the column reduction: thread j joins column j's slots in CTA
// order (the CTAs whose tile range meets j's column block of `width` columns,
// blocks_per_col tiles per column block), in FP64.  Slot (CTA c, column block
// nt) lives at (c + nt) * width: a CTA's tile range is contiguous in
// column-block-major order, so no two (c, nt) it meets share c + nt.
__global__ void __launch_bounds__(256) k_vander_join(const ColPart* __restrict__ parts, int64_t blocks_per_col,
                                                     int64_t tiles, int64_t grid, int64_t width, int64_t npoly,
                                                     float* colsum, float* colmin, float* colmax) {
  const int64_t j = (int64_t)blockIdx.x * 256 + threadIdx.x;
  if (j >= npoly) return;
  const int64_t nt = j / width, lo = nt * blocks_per_col, hi = lo + blocks_per_col;
  double sum = 0.0;
  float mn = INFINITY, mx = -INFINITY;
  for (int64_t c = 0; c < grid; ++c) {
    const int64_t tb = tc_tile_begin(tiles, c, grid), te = tc_tile_begin(tiles, c + 1, grid);
    if (te <= lo || tb >= hi || tb == te) continue;
    const ColPart q = parts[(c + nt) * width + j % width];
    sum += q.sum;
    mn = fminf(mn, q.mn);
    mx = fmaxf(mx, q.mx);
  }
  if (colsum) colsum[j] = (float)sum;
  if (colmin) colmin[j] = mn;
  if (colmax) colmax[j] = mx;
}

// ---- the column results alone: the transposed product ----------------------
//
// Without a Y output the product is formed transposed, Y^T = C^T V^T, tile by
// tile: 128 polynomials (the M side: a C tile, K-major) by 256 points (the N
// side: the V tile, K-major).  The accumulator's TMEM lanes are then
// polynomials and its columns points, so a thread owns one polynomial of its
// warp's lanes and folds that polynomial's values at the warp's 128 points
// into its running compensated sum, minimum and maximum in registers -- no
// shared memory and no exchange between lanes.  The unit of work is a group of
// NB polynomial blocks at one point block: the V tile (the powers of the points
// and their bf16 split, about half of the non-tensor work) is built once and
// multiplied by the NB C tiles in turn -- four for bf16x3, two for bf16x6 (its
// three parts per tile leave shared memory for two).  A CTA walks its units
// group-major, so the running results carry over all of its point blocks, and
// are written to the CTA's workspace slot when the group changes.  (Measured on
// B300 at 2^20 points x 4096 polynomials, bf16x3 / bf16x6: one V tile per
// polynomial block, 1.045 / 1.304 ms; per two blocks, 0.876 / 1.180 ms.)
constexpr int kPolyBlk = 128, kPtBlk = 256;
template <int NS>
constexpr int kGroupBlocks = NS == 2 ? 4 : 2;  // polynomial blocks per unit

template <int NS>
struct ColLayout {
  static constexpr int NB = kGroupBlocks<NS>;
  static constexpr uint32_t a = 0;                        // C parts: NB blocks x NS x 128 polynomials x 32 powers
  static constexpr uint32_t b = NB * NS * kABytes;        // V parts: NS x 256 points x 32 powers
  static constexpr uint32_t comb = b + NS * kBBytes;      // the warps' halves combined: NB x 4 x 32 ColPart
  static constexpr uint32_t bar = comb + NB * 4 * 32 * sizeof(ColPart);
  static constexpr uint32_t used = bar + 64;
  static constexpr uint32_t request = used + 1024 > 80 * 1024 ? used + 1024 : 80 * 1024;
  static_assert(request <= 110 * 1024, "two CTAs per SM");
};

// min / max / sum of 64 values: four independent min3 / max3 chains, pairwise sums
__device__ __forceinline__ void stats64(const float* v, float& mn, float& mx, float& sum) {
  float a[4], b[4];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    a[c] = fminf(v[16 * c], v[16 * c + 1]);
    b[c] = fmaxf(v[16 * c], v[16 * c + 1]);
#pragma unroll
    for (int r = 2; r < 16; r += 2) {
      a[c] = min3f(a[c], v[16 * c + r], v[16 * c + r + 1]);
      b[c] = max3f(b[c], v[16 * c + r], v[16 * c + r + 1]);
    }
  }
  mn = min3f(min3f(a[0], a[1], a[2]), a[3], a[3]);
  mx = max3f(max3f(b[0], b[1], b[2]), b[3], b[3]);
  sum = pairwise<64>(v);
}

template <int NS>
__global__ void __launch_bounds__(kTcThreads, 2) k_vander_colred(const float* __restrict__ x, int64_t m,
                                                                 const float* __restrict__ coef, int deg,
                                                                 int64_t npoly, ColPart* parts, WsHeader* hdr) {
  using L = ColLayout<NS>;
  constexpr int NB = L::NB, kGroup = NB * kPolyBlk;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  unsigned char* sA = base + L::a;
  unsigned char* sB = base + L::b;
  ColPart* comb = reinterpret_cast<ColPart*>(base + L::comb);
  uint64_t* mbar = reinterpret_cast<uint64_t*>(base + L::bar);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(mbar + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = warp & 3, h = warp >> 2;  // TMEM lanes 32 g .. (polynomials), point half h
  const int64_t m_blocks = (m + kPtBlk - 1) / kPtBlk, p_blocks = (npoly + kPolyBlk - 1) / kPolyBlk;
  const int64_t groups = (p_blocks + NB - 1) / NB;
  const int64_t units = m_blocks * groups;
  const int64_t t_begin = tc_tile_begin(units, blockIdx.x, gridDim.x),
                t_end = tc_tile_begin(units, blockIdx.x + 1, gridDim.x);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(smem_u32(mbar), 1);
    mbar_init_fence();
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  // running results of polynomial kGroup pp + 128 s + 32 g + lane (block s of the group) over the
  // points of half h seen so far
  float cs_hi[NB], cs_lo[NB], cmn[NB], cmx[NB];
#pragma unroll
  for (int s = 0; s < NB; ++s) cs_hi[s] = cs_lo[s] = 0.0f, cmn[s] = INFINITY, cmx[s] = -INFINITY;
  auto flush = [&](int64_t pp) {  // both halves combined in FP64 into the slot (CTA + pp)
#pragma unroll
    for (int s = 0; s < NB; ++s)
      if (h == 1) comb[s * kPolyBlk + g * 32 + lane] = ColPart{(double)cs_hi[s] + (double)cs_lo[s], cmn[s], cmx[s]};
    __syncthreads();
    if (h == 0) {
#pragma unroll
      for (int s = 0; s < NB; ++s) {
        const ColPart q = comb[s * kPolyBlk + g * 32 + lane];
        parts[(blockIdx.x + pp) * kGroup + s * kPolyBlk + g * 32 + lane] =
            ColPart{((double)cs_hi[s] + (double)cs_lo[s]) + q.sum, fminf(cmn[s], q.mn), fmaxf(cmx[s], q.mx)};
      }
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < NB; ++s) cs_hi[s] = cs_lo[s] = 0.0f, cmn[s] = INFINITY, cmx[s] = -INFINITY;
  };

  uint32_t phase = 0;
  int64_t loaded_p = -1;
  bool ok = true;
  // point i0 + tid of a unit, loaded one unit ahead (its latency hides behind the unit before)
  auto load_x = [&](int64_t t) {
    const int64_t i = (t % m_blocks) * kPtBlk + tid;
    return t < t_end && i < m ? __ldg(&x[i]) : 0.0f;
  };
  float x_next = load_x(t_begin);
  for (int64_t t = t_begin; t < t_end && ok; ++t) {
    const int64_t pp = t / m_blocks, qb = t % m_blocks;
    const int64_t i0 = qb * kPtBlk;
    if (pp != loaded_p) {
      if (loaded_p >= 0) flush(loaded_p);
#pragma unroll
      for (int r = 0; r < NB / 2; ++r) {  // the NB C tiles: polynomial kGroup pp + 256 r + tid (zero beyond
        // npoly), powers 0 .. 31 (zero beyond deg); threads 0..127 block 2 r, 128..255 block 2 r + 1
        const int64_t j = pp * kGroup + r * 2 * kPolyBlk + tid;
        const bool in = j < npoly;
        float v[kK];
#pragma unroll
        for (int k = 0; k < kK; ++k) v[k] = (in && k <= deg) ? __ldg(&coef[(int64_t)k * npoly + j]) : 0.0f;
        store_split_row<NS>(sA + (2 * r + (tid >> 7)) * NS * kABytes, kABytes, tid & (kPolyBlk - 1), v);
      }
      loaded_p = pp;
    }
    {  // V tile: the powers of point i0 + tid (zero beyond m) by repeated FP32 multiplication, zero above deg
      const float xi = x_next;
      x_next = load_x(t + 1);
      float v[kK];
      v[0] = 1.0f;
#pragma unroll
      for (int k = 1; k < kK; ++k) v[k] = k <= deg ? v[k - 1] * xi : 0.0f;
      store_split_row<NS>(sB, kBBytes, tid, v);
    }
    fence_async_smem();
    __syncthreads();
    const int valid = (int)imax<int64_t>(0, imin<int64_t>(128, m - (i0 + h * 128)));
#pragma unroll
    for (int s = 0; s < NB; ++s) {
      if (NB * pp + s >= p_blocks) break;  // (the last group may hold fewer blocks)
      if (tid == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = smem_u32(sA + s * NS * kABytes), b0 = smem_u32(sB);
        bool first = true;
#pragma unroll
        for (int d = 0; d < NS; ++d)
#pragma unroll
          for (int i = 0; i <= d; ++i) {
            const uint32_t ai = a0 + i * kABytes, bj = b0 + (d - i) * kBBytes;
#pragma unroll
            for (int q = 0; q < 2; ++q) {
              mma_bf16(tmem, smem_desc(ai + q * 2 * kLBO), smem_desc(bj + q * 2 * kLBO), first ? 0u : 1u);
              first = false;
            }
          }
        mma_commit(smem_u32(mbar));
      }
      if (!mbar_wait_until(smem_u32(mbar), phase, kMmaWaitNs)) ok = false;
      phase ^= 1u;
      if (!__syncthreads_and(ok ? 1 : 0)) {
        ok = false;
        if (tid == 0) set_status(hdr, TR_ERR_TIMEOUT, (uint32_t)t);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // this thread's polynomial of block s at the 128 points of half h, 64 per TMEM load
#pragma unroll
      for (int cp = 0; cp < 2; ++cp) {
        float v[64];
        tmem_ld64(tmem + ((uint32_t)(g * 32) << 16) + (uint32_t)(h * 128 + cp * 64), v);
        float tmn, tmx, ts;
        if (valid >= (cp + 1) * 64) {
          stats64(v, tmn, tmx, ts);
        } else {  // points beyond m are left out (the last point block only)
#pragma unroll
          for (int r = 0; r < 64; ++r) v[r] = cp * 64 + r < valid ? v[r] : NAN;
          tmn = INFINITY;
          tmx = -INFINITY;
#pragma unroll
          for (int r = 0; r < 64; ++r) {
            tmn = fminf(tmn, v[r]);  // NaN (left out) is ignored
            tmx = fmaxf(tmx, v[r]);
            v[r] = v[r] == v[r] ? v[r] : 0.0f;
          }
          ts = pairwise<64>(v);
        }
        const float yk = ts - (-cs_lo[s]);  // compensated running sum (Kahan)
        const float tt = cs_hi[s] + yk;
        cs_lo[s] = -((tt - cs_hi[s]) - yk);
        cs_hi[s] = tt;
        cmn[s] = fminf(cmn[s], tmn);
        cmx[s] = fmaxf(cmx[s], tmx);
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncthreads();  // TMEM free for the next product; after the second block, the tiles too
    }
  }
  if (ok && loaded_p >= 0) flush(loaded_p);
  if (!ok) mbar_wait_until(smem_u32(mbar), phase ^ 1u, kMmaWaitNs);  // let committed products drain
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

template <int NS>
tr_status launch_colred(const float* x, int64_t m, const float* coef, int deg, int64_t npoly, float* colsum,
                        float* colmin, float* colmax, const tr_exec* e) {
  using L = ColLayout<NS>;
  auto kern = k_vander_colred<NS>;
  tr_status s = ensure_dyn_smem((const void*)kern, (int)L::request, "cudaFuncSetAttribute(k_vander_colred)");
  if (s) return s;
  constexpr int NB = L::NB;
  const int64_t m_blocks = ceil_div(m, kPtBlk), units = m_blocks * ceil_div(ceil_div(npoly, kPolyBlk), NB);
  const int64_t grid = std::min<int64_t>(std::min<int64_t>(units, 2 * (int64_t)dev_info().sm_count), kMaxTcGrid);
  ColPart* parts = reinterpret_cast<ColPart*>(ws_body(e));
  cudaStream_t st = stream_of(e);
  kern<<<(unsigned)grid, kTcThreads, L::request, st>>>(x, m, coef, deg, npoly, parts, ws_header(e));
  if ((s = launch_status("k_vander_colred"))) return s;
  // slot (CTA c, group pp) at (c + pp) x NB x 128: the join's column blocks are the groups
  k_vander_join<<<(unsigned)ceil_div(npoly, 256), 256, 0, st>>>(parts, m_blocks, units, grid, NB * kPolyBlk, npoly,
                                                               colsum, colmin, colmax);
  return launch_status("k_vander_join");
}

template <int NS, int OUT, bool RED>
tr_status launch_tc(const CUtensorMap& ymap, const float* x, int64_t m, const float* coef, int deg, int64_t npoly,
                    void* y, float* colsum, float* colmin, float* colmax, const tr_exec* e) {
  using L = TcLayout<NS, OUT, RED>;
  auto kern = k_vander_tc<NS, OUT, RED>;
  tr_status s = ensure_dyn_smem((const void*)kern, (int)L::request, "cudaFuncSetAttribute(k_vander_tc)");
  if (s) return s;
  const int64_t m_tiles = ceil_div(m, kTileM), tiles = m_tiles * ceil_div(npoly, kTileN);
  const int64_t grid = std::min<int64_t>(std::min<int64_t>(tiles, 2 * (int64_t)dev_info().sm_count), kMaxTcGrid);
  ColPart* parts = reinterpret_cast<ColPart*>(ws_body(e));
  cudaStream_t st = stream_of(e);
  kern<<<(unsigned)grid, kTcThreads, L::request, st>>>(ymap, x, m, coef, deg, npoly,
                                                       static_cast<__nv_bfloat16*>(y), parts, ws_header(e));
  if ((s = launch_status("k_vander_tc"))) return s;
  if constexpr (RED) {
    k_vander_join<<<(unsigned)ceil_div(npoly, 256), 256, 0, st>>>(parts, m_tiles, tiles, grid, kTileN, npoly, colsum,
                                                                 colmin, colmax);
    return launch_status("k_vander_join");
  }
  return TR_OK;
}

template <int NS>
tr_status launch_tc_ns(int out, bool red, const CUtensorMap& ymap, const float* x, int64_t m, const float* coef,
                       int deg, int64_t npoly, void* y, float* cs, float* cn, float* cx, const tr_exec* e) {
  if (out == kOutF32) return red ? launch_tc<NS, kOutF32, true>(ymap, x, m, coef, deg, npoly, y, cs, cn, cx, e)
                                 : launch_tc<NS, kOutF32, false>(ymap, x, m, coef, deg, npoly, y, cs, cn, cx, e);
  if (out == kOutBf16) return red ? launch_tc<NS, kOutBf16, true>(ymap, x, m, coef, deg, npoly, y, cs, cn, cx, e)
                                  : launch_tc<NS, kOutBf16, false>(ymap, x, m, coef, deg, npoly, y, cs, cn, cx, e);
  return launch_colred<NS>(x, m, coef, deg, npoly, cs, cn, cx, e);  // column results alone
}

// Slots of either form: (grid + column blocks) x block width, at most
// (kMaxTcGrid + npoly / 128 + 1) x 512 entries (column blocks of up to 512
// polynomials).
size_t vander_ws_bytes(int64_t npoly) {
  return (size_t)kWsHeader + (size_t)(kMaxTcGrid + ceil_div(std::max<int64_t>(npoly, 1), kPolyBlk)) * 4 * kPolyBlk *
                                 sizeof(ColPart);
}

}  // namespace

}  // namespace tr

using namespace tr;

extern "C" {

tr_status tr_vandermonde_workspace_size(int64_t m, int64_t npoly, size_t* bytes) {
  if (!bytes || m < 0 || npoly < 0) return fail(TR_ERR_INVALID_ARG, "bad arguments");
  *bytes = vander_ws_bytes(npoly);
  return TR_OK;
}

tr_status tr_vandermonde(const float* x, int64_t m, const float* coef, int32_t deg, int64_t npoly, int precision,
                         void* y, tr_dtype yt, float* colsum, float* colmin, float* colmax, const tr_exec* e) {
  if (!e) return fail(TR_ERR_INVALID_ARG, "exec is NULL");
  if (m < 0 || npoly < 0) return fail(TR_ERR_INVALID_ARG, "m or npoly < 0");
  if (deg < 0 || deg > TR_MAX_DEGREE) return fail(TR_ERR_INVALID_ARG, "degree %d out of [0, %d]", deg, TR_MAX_DEGREE);
  if (precision != TR_PREC_BF16X3 && precision != TR_PREC_FP32 && precision != TR_PREC_BF16X6)
    return fail(TR_ERR_INVALID_ARG, "precision %d", precision);
  if (yt != TR_F32 && yt != TR_BF16 && yt != TR_NONE) return fail(TR_ERR_UNSUPPORTED, "output dtype %d", yt);
  const bool red = colsum || colmin || colmax;
  if (yt == TR_NONE && !red) return fail(TR_ERR_INVALID_ARG, "no output requested (y and column results)");
  if (m > 0 && npoly > 0 && (!x || !coef || (yt != TR_NONE && !y)))
    return fail(TR_ERR_INVALID_ARG, "x, coef or y is NULL");
  if ((x && !aligned_to(x, 4)) || (coef && !aligned_to(coef, 4)) || (y && !aligned_to(y, yt == TR_BF16 ? 2 : 4)) ||
      (colsum && !aligned_to(colsum, 4)) || (colmin && !aligned_to(colmin, 4)) || (colmax && !aligned_to(colmax, 4)))
    return fail(TR_ERR_ALIGNMENT, "pointers must be aligned to their element size");
  if (m > 0x7FFFFFFF || npoly > 0x7FFFFFFF) return fail(TR_ERR_INVALID_ARG, "m or npoly beyond 32-bit coordinates");
  cudaStream_t st = stream_of(e);
  if (precision == TR_PREC_FP32) {
    if (yt != TR_F32 || red)
      return fail(TR_ERR_UNSUPPORTED, "the FP32 Horner path writes FP32 Y only (no BF16 or column results)");
    if (m == 0 || npoly == 0) return TR_OK;
    if (ceil_div(npoly, kF32Threads) > 0x7FFFFFFF) return fail(TR_ERR_INVALID_ARG, "npoly too large");
    const dim3 grid((unsigned)ceil_div(npoly, kF32Threads), (unsigned)std::min<int64_t>(ceil_div(m, kF32Points), 65535));
    k_vander_fp32<<<grid, kF32Threads, 0, st>>>(x, m, coef, deg, npoly, static_cast<float*>(y));
    return launch_status("k_vander_fp32");
  }
  if (yt == TR_F32 && (npoly % 4 || !aligned_to(y, 16)))
    return fail(TR_ERR_ALIGNMENT, "FP32 output on the tensor path needs npoly %% 4 == 0 and a 16-byte aligned y");
  if (yt == TR_BF16 && (npoly % 8 || !aligned_to(y, 16)))
    return fail(TR_ERR_ALIGNMENT, "BF16 output on the tensor path needs npoly %% 8 == 0 and a 16-byte aligned y");
  const size_t need = vander_ws_bytes(npoly);
  if (!e->workspace || e->workspace_bytes < need)
    return fail(TR_ERR_WORKSPACE, "the tensor path needs a %zu-byte workspace", need);
  if (!aligned_to(e->workspace, 256)) return fail(TR_ERR_ALIGNMENT, "workspace must be 256-byte aligned");
  if (m == 0 || npoly == 0) return TR_OK;
  CUtensorMap ymap;
  std::memset(&ymap, 0, sizeof(ymap));
  tr_status s;
  if (yt == TR_F32 &&
      (s = make_tensor_map_2d(&ymap, y, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, (uint64_t)npoly, (uint64_t)m,
                              (uint64_t)npoly * 4, 32, 32, CU_TENSOR_MAP_SWIZZLE_128B)))
    return s;
  const int out = yt == TR_F32 ? kOutF32 : (yt == TR_BF16 ? kOutBf16 : kOutNone);
  return precision == TR_PREC_BF16X6
             ? launch_tc_ns<3>(out, red, ymap, x, m, coef, deg, npoly, y, colsum, colmin, colmax, e)
             : launch_tc_ns<2>(out, red, ymap, x, m, coef, deg, npoly, y, colsum, colmin, colmax, e);
}

}  // extern "C"
