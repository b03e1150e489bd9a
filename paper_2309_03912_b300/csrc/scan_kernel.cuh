// scan_kernel.cuh -- the kernel of tr_scan / tr_scan_reduce, prefix sums of f(x)
// in one pass, as a template over the storage type, the map, the output
// arithmetic and the map's source (the family's MapParams, or a user-supplied
// functor passed by value), with its launcher.
//
// Single-pass scan with decoupled look-back (Merrill & Garland, "Single-pass
// parallel prefix scan with decoupled look-back", NVR-2016-002):
//   * each block takes tile ids from an atomic counter, at most one tile ahead
//     of the one it computes (dynamic ids: every tile's predecessors have
//     already started, so waiting on them ends);
//   * the tile is mapped and totalled in shared memory (threads total their
//     rows, warps scan the row totals with shuffles, the block combines warp
//     totals) and its aggregate is published at once (flag A);
//   * a dedicated look-back warp reads 256 predecessors per round (128 for u64
//     carries), summing aggregates until it meets an inclusive prefix (flag P),
//     publishes the tile's inclusive prefix and hands the exclusive prefix to
//     the compute warps, which meanwhile work on the next tile.  Each tile's
//     state has its own 128-byte line; u32 and float-float carries share one
//     64-bit status word with their flag (one relaxed load, no fence), a u64
//     carry sits beside a flag released after it;
//   * every wait is bounded by a %globaltimer deadline and an abort word: on
//     expiry the block records TR_ERR_TIMEOUT and finishes instead of hanging.
// Two kernels share this: k_scan (tiles loaded by the compute warps into
// registers, any storage and output type) and k_scan_tma (4-byte inputs and
// outputs on aligned arrays: tiles moved by TMA box loads and stores through a
// ring of shared-memory stages fed by a producer warp).  Each call clears the
// look-back lines and the tile counter with one memset on the stream
// (graph-capturable) before the kernel.
//
// Arithmetic: u32 wraps modulo 2^32; u32 -> u64 is exact; float scans keep
// float-float (hi, lo) pairs inside a tile and between tiles, and round each
// output once from the compensated prefix.
#pragma once

#include "internal.h"

namespace tr {
namespace scank {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kItems = 32;
constexpr int kTile = kThreads * kItems;  // 8192 elements

constexpr uint32_t kFlagA = 1, kFlagP = 2;

// ---- per-output arithmetic -------------------------------------------------
struct OpU32 {
  using T = uint32_t;      // in-tile running value
  using Carry = uint32_t;  // between tiles
  using Out = uint32_t;
  __device__ static T zero() { return 0u; }
  __device__ static Carry carry_of(Out v) { return v; }
  __device__ static T lift(uint32_t v) { return v; }
  __device__ static T add(T a, T b) { return a + b; }
  __device__ static Carry to_carry(T a) { return a; }
  __device__ static Carry cadd(Carry a, Carry b) { return a + b; }
  __device__ static T shfl_up(T a, int d) { return __shfl_up_sync(kFull, a, d); }
  __device__ static Carry shfl_xor_c(Carry a, int d) { return __shfl_xor_sync(kFull, a, d); }
};

struct OpU64 {
  using T = unsigned long long;
  using Carry = unsigned long long;
  using Out = unsigned long long;
  __device__ static T zero() { return 0ull; }
  __device__ static Carry carry_of(Out v) { return v; }
  __device__ static T lift(uint32_t v) { return v; }
  __device__ static T add(T a, T b) { return a + b; }
  __device__ static Carry to_carry(T a) { return a; }
  __device__ static Carry cadd(Carry a, Carry b) { return a + b; }
  __device__ static T shfl_up(T a, int d) { return __shfl_up_sync(kFull, a, d); }
  __device__ static Carry shfl_xor_c(Carry a, int d) { return __shfl_xor_sync(kFull, a, d); }
};

// Float scans carry float-float pairs between tiles as well: B300 issues an
// FP64 add for a warp in about 60 cycles, and FP64 carries made the look-back
// (a dozen adds per round) and every thread's prefix conversion the bound of
// the f32 scan.
struct OpF32 {
  using T = FF;
  using Carry = FF;
  using Out = float;
  __device__ static T zero() { return FF{0.f, 0.f}; }
  __device__ static Carry carry_of(Out v) { return FF{v, 0.f}; }
  __device__ static T add(T a, T b) { return ff_add(a, b); }
  __device__ static Carry to_carry(T a) { return a; }
  __device__ static Carry cadd(Carry a, Carry b) { return ff_add(a, b); }
  __device__ static T shfl_up(T a, int d) { return FF{__shfl_up_sync(kFull, a.hi, d), __shfl_up_sync(kFull, a.lo, d)}; }
  __device__ static Carry shfl_xor_c(Carry a, int d) {
    return FF{__shfl_xor_sync(kFull, a.hi, d), __shfl_xor_sync(kFull, a.lo, d)};
  }
};

template <class Op>
__device__ __forceinline__ typename Op::T warp_incl_scan(typename Op::T v, int lane) {
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const typename Op::T o = Op::shfl_up(v, d);
    if (lane >= d) v = Op::add(o, v);
  }
  return v;
}

template <class Op>
__device__ __forceinline__ typename Op::Carry warp_sum_carry(typename Op::Carry v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v = Op::cadd(v, Op::shfl_xor_c(v, d));
  return v;
}

// Look-back state: one 128-byte line per tile, so that the polls of hundreds
// of waiting tiles spread over many L2 lines instead of hammering a few (with
// the state packed contiguously the polls contended for a handful of lines and
// the u32 scan ran 25 % slower).  Where the carry and its flag fit one 64-bit
// status word, one relaxed load sees both and no fence is needed: a u32 carry
// takes the high half and the flag the low bits; a float-float carry (float
// scans) keeps its high part whole in the high half and gives up the two
// lowest significand bits of its low part to the flag (a relative change
// below 2^-44 of the carry, far below the FP32 outputs' resolution).  A u64 carry sits in the same line (aggregate at byte
// 8, inclusive prefix at byte 16) and its flag (byte 0) is released after it.
constexpr int kLineBytes = 128;
struct ScanWs {
  unsigned char* lines;  // tiles x kLineBytes
};

template <class Op>
constexpr bool kPackedStatus = !std::is_same<typename Op::Carry, unsigned long long>::value;

template <class Op>
__device__ __forceinline__ unsigned long long pack_status(typename Op::Carry v, uint32_t flag) {
  if constexpr (std::is_same<typename Op::Carry, FF>::value) {
    return ((unsigned long long)__float_as_uint(v.hi) << 32) | (__float_as_uint(v.lo) & ~3u) | flag;
  } else {
    return ((unsigned long long)v << 32) | flag;
  }
}
template <class Op>
__device__ __forceinline__ typename Op::Carry status_value(unsigned long long w) {
  if constexpr (std::is_same<typename Op::Carry, FF>::value) {
    return FF{__uint_as_float((uint32_t)(w >> 32)), __uint_as_float((uint32_t)w & ~3u)};
  } else {
    return (typename Op::Carry)(w >> 32);
  }
}

__device__ __forceinline__ unsigned char* status_line(ScanWs ws, int64_t tile) {
  return ws.lines + tile * kLineBytes;
}

template <class Op>
__device__ __forceinline__ void publish(ScanWs ws, int64_t tile, uint32_t flag, typename Op::Carry v) {
  unsigned char* line = status_line(ws, tile);
  if constexpr (kPackedStatus<Op>) {
    st_relaxed_u64(reinterpret_cast<unsigned long long*>(line), pack_status<Op>(v, flag));
  } else {
    *reinterpret_cast<typename Op::Carry*>(line + (flag == kFlagP ? 16 : 8)) = v;
    st_release_u32(reinterpret_cast<uint32_t*>(line), flag);
  }
}

// Decoupled look-back for `tile` by one warp (its aggregate, flag A, has been
// published by the compute warps): reads the nearest unread predecessors (256
// or 128 per round), summing aggregates until an inclusive prefix (flag P)
// bounds the sum, and publishes its own inclusive prefix.  Returns the exclusive prefix in
// every lane; sets `gave_up` (and the status word) when a wait runs past the
// deadline or another block has aborted.
// Predecessors read per lane and round: eight (a 256-tile window) with packed
// status words, four (128) for u64 carries, whose rounds cost a fence and a
// second load.  A round costs about one L2 round trip whatever its width, and
// with ~300 tiles in flight at once a tile's nearest inclusive prefix is
// usually one batch of tiles back: a 32-tile window needed several rounds per
// look-back and bounded the scan by look-back latency (measured on B300:
// 953 us for the 2^28 u32 scan with 4,096-element tiles).
template <class Op>
constexpr int kLookbackSlots = kPackedStatus<Op> ? 8 : 4;

template <class Op>
__device__ __forceinline__ typename Op::Carry warp_lookback(int64_t tile, typename Op::Carry aggregate, ScanWs ws,
                                                            WsHeader* hdr, uint64_t timeout_ns, bool stall, int lane,
                                                            bool& gave_up) {
  using Carry = typename Op::Carry;
  constexpr int kSlots = kLookbackSlots<Op>;
  Carry excl = Carry{};
  gave_up = false;
  if (tile == 0) return excl;  // (its inclusive prefix is its aggregate, published with it)
  const uint64_t deadline = globaltimer_ns() + timeout_ns;
  int64_t pos = tile - 1;
  while (true) {
    // slot m of lane l reads the predecessor at distance 32 m + l from pos
    uint32_t st[kSlots];
    Carry val[kSlots];
    int stop = 0;
#pragma unroll
    for (int m = 0; m < kSlots; ++m) {
      st[m] = kFlagP;  // before tile 0: an inclusive prefix of 0
      val[m] = Carry{};
    }
    for (int polls = 0;; ++polls) {  // the window's loads are issued together; waits are bounded
      bool pending = false;
#pragma unroll
      for (int m = 0; m < kSlots; ++m) {
        const int64_t idx = pos - 32 * m - lane;
        if (idx >= 0 && (polls == 0 || st[m] == 0)) {
          const unsigned char* line = status_line(ws, idx);
          if constexpr (kPackedStatus<Op>) {
            const unsigned long long w = ld_relaxed_u64(reinterpret_cast<const unsigned long long*>(line));
            st[m] = (uint32_t)w & 3u;
            val[m] = status_value<Op>(w);
          } else {
            st[m] = ld_relaxed_u32(reinterpret_cast<const uint32_t*>(line)) & 3u;
          }
          pending |= st[m] == 0;
        }
      }
      if (!pending) break;
      if ((polls & 15) == 15 && (globaltimer_ns() > deadline || ld_relaxed_u32(&hdr->abort) != 0u)) {
        stop = 1;
        break;
      }
    }
    if (__any_sync(kFull, stop)) {
      if (lane == 0 && !ld_relaxed_u32(&hdr->abort)) set_status(hdr, TR_ERR_TIMEOUT, (uint32_t)tile);
      gave_up = true;
      return excl;
    }
    if constexpr (!kPackedStatus<Op>) {
      fence_acq_rel_gpu();  // orders the value reads after the flags
#pragma unroll
      for (int m = 0; m < kSlots; ++m) {
        const int64_t idx = pos - 32 * m - lane;
        if (idx >= 0) val[m] = *reinterpret_cast<const Carry*>(status_line(ws, idx) + (st[m] == kFlagP ? 16 : 8));
      }
    }
    // the nearest predecessor holding an inclusive prefix: everything up to it is summed
    int first = 32 * kSlots;
#pragma unroll
    for (int m = kSlots - 1; m >= 0; --m) {
      const unsigned pm = __ballot_sync(kFull, st[m] == kFlagP);
      if (pm) first = 32 * m + __ffs(pm) - 1;
    }
    Carry part = Carry{};
#pragma unroll
    for (int m = 0; m < kSlots; ++m)
      if (32 * m + lane <= first) part = Op::cadd(part, val[m]);
    excl = Op::cadd(excl, warp_sum_carry<Op>(part));
    if (first < 32 * kSlots) break;
    pos -= 32 * kSlots;
  }
  if (lane == 0 && !stall) publish<Op>(ws, tile, kFlagP, Op::cadd(excl, aggregate));
  return excl;
}

// Run by one compute thread as soon as the tile's total is known: the tile's
// aggregate (flag A), or for tile 0 its inclusive prefix (flag P).  Publishing
// it here rather than in the look-back warp matters: the look-back warp may
// still be busy with the block's previous tile, and successors that cannot
// see this tile's aggregate cannot look past it -- the look-backs then chain
// tile by tile (measured on B300: the TMA-fed 2^28 scan took 4.6 ms so).
template <class Op>
__device__ __forceinline__ void publish_aggregate(ScanWs ws, int64_t tile, typename Op::Carry aggregate, bool stall) {
  if (!stall) publish<Op>(ws, tile, tile == 0 ? kFlagP : kFlagA, aggregate);
}

// ---- reduction in the same pass (tr_scan_reduce) ---------------------------
// min / max travel as order-preserving unsigned keys so that one unsigned
// maximum serves both (the minimum as the maximum of complemented keys): float
// keys flip the sign bit of non-negative values and every bit of negative ones;
// u32 values are their own keys.  A zero word means "no value yet" for both
// (no non-NaN float has key 0 or complemented key 0; for u32, 0 is the identity
// of max and ~0 that of min), so the cleared header words are the identities.
__device__ __forceinline__ uint32_t mm_key(float v) {
  const uint32_t b = __float_as_uint(v);
  return b ^ ((b >> 31) ? 0xFFFFFFFFu : 0x80000000u);
}
__device__ __forceinline__ uint32_t mm_key(uint32_t v) { return v; }
__device__ __forceinline__ float mm_float(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k ^ 0x80000000u) : ~k);
}
__device__ __forceinline__ float mm_min(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ float mm_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ uint32_t mm_min(uint32_t a, uint32_t b) { return min(a, b); }
__device__ __forceinline__ uint32_t mm_max(uint32_t a, uint32_t b) { return max(a, b); }
template <class C>
__device__ __forceinline__ C mm_lowest();
template <>
__device__ __forceinline__ float mm_lowest<float>() { return -INFINITY; }
template <>
__device__ __forceinline__ uint32_t mm_lowest<uint32_t>() { return 0u; }
template <class C>
__device__ __forceinline__ C mm_highest();
template <>
__device__ __forceinline__ float mm_highest<float>() { return INFINITY; }
template <>
__device__ __forceinline__ uint32_t mm_highest<uint32_t>() { return 0xFFFFFFFFu; }

__device__ __forceinline__ void red_max_u32(uint32_t* p, uint32_t v) {
  asm volatile("red.relaxed.gpu.global.max.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// The reduction outputs of a scan (ops = 0: plain scan).
struct ScanRed {
  void* sum;
  void* mn;
  void* mx;
  int32_t sum_t;  // tr_dtype
  uint32_t ops;
};

// Run by thread 0 of the last tile after its look-back: `total` is the sum of f
// over all tiles (without the carry-in).
template <class Op>
__device__ __noinline__ void finish_sum(const ScanRed& red, typename Op::Carry total) {
  if (!(red.ops & TR_SUM) || !red.sum) return;
  if constexpr (std::is_same<Op, OpF32>::value) {
    if (red.sum_t == TR_F64)
      *static_cast<double*>(red.sum) = ff_to_double(total);
    else
      *static_cast<float*>(red.sum) = (float)ff_to_double(total);
  } else if constexpr (std::is_same<Op, OpU64>::value) {
    *static_cast<unsigned long long*>(red.sum) = total;
  } else {
    *static_cast<uint32_t*>(red.sum) = total;
  }
}

// ---- the pipelined tile loop --------------------------------------------------
//
// A block is 8 compute warps plus one look-back warp and stays resident,
// taking tile ids from the counter one ahead of use.  Per tile i the compute
// warps map it into a padded row buffer (one of two), total the rows, hand
// the tile's aggregate to the look-back warp, then -- while that warp resolves
// tile i's prefix -- fetch tile i+1's vectors into registers and write tile
// i-1's outputs, whose prefix the look-back warp delivered meanwhile.  So the
// compute warps never wait out a look-back of their own tile, the loads of one
// tile overlap the stores of another, and two tiles per block are in flight.
// Hand-overs use named barriers, two per direction (by tile parity) so that a
// barrier is never arrived at twice within one phase:
//   kBarAgg + (i & 1)  compute warps arrive after publishing tile i's
//                      aggregate; the look-back warp waits on it;
//   kBarExcl + (i & 1) the look-back warp arrives after publishing tile i's
//                      exclusive prefix; the compute warps wait on it before
//                      writing tile i's outputs (one iteration later).
// The look-back warp stops on a tile id of -1.
constexpr int kBlockThreads = kThreads + 32;
constexpr int kBarCompute = 1, kBarAgg = 2, kBarExcl = 4;

__device__ __forceinline__ void bar_sync_n(int id, int count) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void bar_arrive_n(int id, int count) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(count) : "memory");
}
__device__ __forceinline__ void compute_sync() { bar_sync_n(kBarCompute, kThreads); }

// Min / max: every compute thread keeps its own running min / max over all the
// rows it maps; at its end a block combines them and folds the result into the
// header words (fire-and-forget red.max of order-preserving keys), then counts
// itself with one acquire-release add; the block that completes the count
// writes the results.  One fence per block -- counting every tile with a
// release add stalled the warp that hands tiles to the look-back once per tile
// (measured on B300: the fused 2^28 u32 scan took 502 us against 382 us for
// the plain scan).  All compute threads of the block call it.
template <class C>
__device__ __forceinline__ void block_minmax(C mn, C mx, const ScanRed& red, WsHeader* hdr, C* s_mn, C* s_mx) {
  const int tid = threadIdx.x, lane = tid & 31;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mn = mm_min(mn, __shfl_xor_sync(kFull, mn, o));
    mx = mm_max(mx, __shfl_xor_sync(kFull, mx, o));
  }
  if (lane == 0) {
    s_mn[tid >> 5] = mn;
    s_mx[tid >> 5] = mx;
  }
  compute_sync();
  if (tid != 0) return;
  mn = s_mn[0];
  mx = s_mx[0];
#pragma unroll
  for (int w = 1; w < kWarps; ++w) {
    mn = mm_min(mn, s_mn[w]);
    mx = mm_max(mx, s_mx[w]);
  }
  if (mn == mn) red_max_u32(&hdr->red_min, ~mm_key(mn));  // NaN (only NaN values) adds nothing
  if (mx == mx) red_max_u32(&hdr->red_max, mm_key(mx));
  if (atom_add_acq_rel_u32(&hdr->red_done, 1u) != gridDim.x - 1) return;
  const uint32_t kmn = ld_relaxed_u32(&hdr->red_min), kmx = ld_relaxed_u32(&hdr->red_max);
  if constexpr (std::is_same<C, float>::value) {
    if ((red.ops & TR_MIN) && red.mn) *static_cast<float*>(red.mn) = kmn ? mm_float(~kmn) : INFINITY;
    if ((red.ops & TR_MAX) && red.mx) *static_cast<float*>(red.mx) = kmx ? mm_float(kmx) : -INFINITY;
  } else {
    if ((red.ops & TR_MIN) && red.mn) *static_cast<uint32_t*>(red.mn) = ~kmn;
    if ((red.ops & TR_MAX) && red.mx) *static_cast<uint32_t*>(red.mx) = kmx;
  }
}

// A row's min / max over its first `valid` values (all V when the row is
// full): full rows fold as a tree of three-operand min / max for floats (two
// new values per instruction, independent levels) or as two independent
// chains for u32, with no per-value test; only partial rows mask.
template <class C, int V>
__device__ __forceinline__ void row_minmax(const C* v, int valid, C& mn, C& mx) {
  if (valid == V) {
    if constexpr (std::is_same<C, float>::value) {
      mn = fold3<V>(INFINITY, v, Min3());
      mx = fold3<V>(-INFINITY, v, Max3());
    } else {
      C a0 = v[0], a1 = v[1], b0 = v[0], b1 = v[1];
#pragma unroll
      for (int k = 2; k + 1 < V; k += 2) {
        a0 = mm_min(a0, v[k]);
        a1 = mm_min(a1, v[k + 1]);
        b0 = mm_max(b0, v[k]);
        b1 = mm_max(b1, v[k + 1]);
      }
      mn = mm_min(a0, a1);
      mx = mm_max(b0, b1);
    }
  } else {
    mn = mm_highest<C>();
    mx = mm_lowest<C>();
#pragma unroll
    for (int k = 0; k < V; ++k) {
      if (k < valid) {
        mn = mm_min(mn, v[k]);
        mx = mm_max(mx, v[k]);
      }
    }
  }
}

// Blocks per SM: two (each with two 33 KiB row buffers and 9 warps).  Measured
// on B300 at 2^28 (u32 splitmix32 / f32 x^2): two blocks 447 / 520 us, three
// blocks (72 registers, spilling) 532 / 605 us; one tile per block with six
// blocks per SM and the look-back in warp 0, 460 / 550 us.
constexpr int kBlocksPerSm = 2;

// The look-back warp of a block: per tile handed over by the compute warps
// (barrier kBarAgg + i % kN), the decoupled look-back, then the exclusive
// prefix back (barrier kBarAgg + kN + i % kN); the last tile also finishes the
// fused reduction.  It stops on a tile id of -1.  kN hand-over slots (and
// barriers each way) are in use at once: 2 when the compute warps consume a
// prefix one tile after handing the tile over, 4 when they consume it two
// tiles later (a barrier is never arrived at twice within one phase).
template <class Op, class C, int kN>
__device__ __forceinline__ void lookback_warp(const int64_t* s_tile_of, const typename Op::Carry* s_agg,
                                              typename Op::Carry* s_excl, ScanWs ws, WsHeader* hdr,
                                              uint64_t timeout_ns, int64_t stall_tile, const ScanRed& red,
                                              int64_t tiles, int lane) {
  using Carry = typename Op::Carry;
  for (int i = 0;; ++i) {
    const int slot = i % kN;
    bar_sync_n(kBarAgg + slot, kBlockThreads);
    const int64_t tile = s_tile_of[slot];
    if (tile < 0) break;
    const Carry agg = s_agg[slot];
    bool gave_up;
    const Carry e = warp_lookback<Op>(tile, agg, ws, hdr, timeout_ns, tile == stall_tile, lane, gave_up);
    if (lane == 0) {
      s_excl[slot] = e;
      if (tile == tiles - 1 && !gave_up) finish_sum<Op>(red, Op::cadd(e, agg));
    }
    __syncwarp();
    bar_arrive_n(kBarAgg + kN + slot, kBlockThreads);
  }
}

// One item into a running in-tile value (TwoSum into (hi, lo) for floats).
template <class Op, class C>
__device__ __forceinline__ void run_add(typename Op::T& run, C v) {
  if constexpr (std::is_same<Op, OpF32>::value) {
    float sm, e;
    two_sum(run.hi, v, sm, e);
    run.hi = sm;
    run.lo += e;
  } else {
    run = Op::add(run, Op::lift(v));
  }
}
template <class Op>
__device__ __forceinline__ typename Op::Out run_out(const typename Op::T& run) {
  if constexpr (std::is_same<Op, OpF32>::value) {
    return run.hi + run.lo;  // the compensated prefix, rounded once
  } else {
    return run;
  }
}

// The total of a thread's row (V values): float scans run two interleaved
// TwoSum chains on packed pairs (even and odd positions, add.rn.f32x2 /
// sub.rn.f32x2, each half an IEEE operation) and join them with one
// float-float add -- the same float-float accuracy as one chain in half the
// instructions; the other outputs add in order.
template <class Op, int V, class C>
__device__ __forceinline__ typename Op::T row_total(const C* v) {
  if constexpr (std::is_same<Op, OpF32>::value && V % 2 == 0) {
    unsigned long long s = pack_f32x2(v[0], v[1]), e = pack_f32x2(0.0f, 0.0f);
#pragma unroll
    for (int k = 2; k < V; k += 2) {
      const unsigned long long x = pack_f32x2(v[k], v[k + 1]);
      const unsigned long long t = add_f32x2(s, x);
      const unsigned long long bb = sub_f32x2(t, s);
      e = add_f32x2(e, add_f32x2(sub_f32x2(s, sub_f32x2(t, bb)), sub_f32x2(x, bb)));
      s = t;
    }
    float s0, s1, e0, e1;
    unpack_f32x2(s, s0, s1);
    unpack_f32x2(e, e0, e1);
    return ff_add(FF{s0, e0}, FF{s1, e1});
  } else {
    typename Op::T acc = Op::zero();
#pragma unroll
    for (int k = 0; k < V; ++k) run_add<Op>(acc, v[k]);
    return acc;
  }
}

// Lane totals warp-scanned; block totals in shared memory (compute warps only).
template <class Op>
__device__ __forceinline__ void block_totals(typename Op::T acc, typename Op::T* s_warp, typename Op::T& warp_off,
                                             typename Op::T& excl_lane, typename Op::T& tile_tot) {
  using T = typename Op::T;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const T incl_lane = warp_incl_scan<Op>(acc, lane);
  excl_lane = Op::shfl_up(incl_lane, 1);
  if (lane == 0) excl_lane = Op::zero();
  if (lane == 31) s_warp[wid] = incl_lane;
  compute_sync();
  warp_off = Op::zero();
  tile_tot = Op::zero();
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    if (w < wid) warp_off = Op::add(warp_off, s_warp[w]);
    tile_tot = Op::add(tile_tot, s_warp[w]);
  }
}

// Tiles move through shared memory in both directions so that every global
// access is a coalesced 16-byte-per-lane access: lanes load consecutive
// vectors, map them and scatter the values into per-thread rows (thread t owns
// the kItems contiguous elements t*kItems...; rows padded to kItems + 1 words,
// which makes the scatter, the row reads and the final gather free of bank
// conflicts).  For the outputs each thread scans its row on top of its prefix
// in place (outputs of 4 bytes) and the block stores the rows back out as
// coalesced vectors; 8-byte outputs are stored from the thread's registers.
constexpr int kRow = kItems + 1;  // padded row, in 4-byte words
constexpr size_t kRowsBytes = (size_t)kThreads * kRow * 4;  // one row buffer
constexpr size_t kDynBytes = 2 * kRowsBytes;                 // dynamic shared memory per block

template <class In, class F, class Op, class Src>
__global__ void __launch_bounds__(kBlockThreads, kBlocksPerSm)
    k_scan(const In* __restrict__ x, typename Op::Out* y, int64_t n, int vec_ok, const __grid_constant__ Src P,
           WsHeader* hdr, ScanWs ws, const typename Op::Out* carry_in, uint64_t timeout_ns, int64_t stall_tile,
           int exclusive, ScanRed red, int64_t tiles) {
  using S = Storage<In>;
  using C = typename S::C;
  using T = typename Op::T;
  using Carry = typename Op::Carry;
  using Out = typename Op::Out;
  static_assert(sizeof(C) == 4, "4-byte compute values");
  constexpr int V = S::kVec;
  constexpr int kVecs = kTile / V;  // input vectors per tile
  constexpr int kLoads = kVecs / kThreads;

  __shared__ int64_t s_tile_of[2];  // tile handed to the look-back warp, by parity (-1: stop)
  __shared__ Carry s_agg[2], s_excl[2];
  __shared__ uint32_t s_next;
  __shared__ T s_warp[kWarps];
  __shared__ C s_mn[kWarps], s_mx[kWarps];
  extern __shared__ __align__(16) unsigned char s_dyn[];
  const int tid = threadIdx.x, lane = tid & 31;

  if (tid >= kThreads) {  // ---- the look-back warp
    lookback_warp<Op, C, 2>(s_tile_of, s_agg, s_excl, ws, hdr, timeout_ns, stall_tile, red, tiles, lane);
    return;
  }

  // ---- the compute warps
  const auto f = kernel_map<F>(P);
  const bool minmax = (red.ops & (TR_MIN | TR_MAX)) != 0;
  const Carry carry = carry_in ? Op::carry_of(*carry_in) : Carry{};
  C* const rows0 = reinterpret_cast<C*>(s_dyn);
  uint4 raw[kLoads];
  auto full_tile = [&](int64_t t) { return vec_ok && t * kTile + kTile <= n; };
  auto fetch = [&](int64_t t) {  // a full tile's vectors into registers (loads in flight)
    const uint4* xv = reinterpret_cast<const uint4*>(x + t * kTile);
#pragma unroll
    for (int j = 0; j < kLoads; ++j) raw[j] = ld_stream(xv + j * kThreads + tid);
  };
  // tile t's outputs from its scanned-in-place row buffer, given its exclusive prefix
  auto write_out = [&](int64_t t, C* rows, Carry excl, const T& thread_off) {
    const int64_t t0 = t * kTile;
    const bool full = full_tile(t);
    C* row = rows + tid * kRow;
    const Carry prefix = Op::cadd(carry, excl);
    T run;
    if constexpr (std::is_same<Op, OpF32>::value) {
      run = ff_add(prefix, thread_off);
    } else {
      run = Op::add((T)prefix, thread_off);
    }
    if constexpr (sizeof(Out) == 4) {
      Out* orow = reinterpret_cast<Out*>(row);
      if (exclusive) {
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
          const Out o = run_out<Op>(run);
          run_add<Op>(run, row[i]);
          orow[i] = o;  // in place: this thread alone reads and writes its row
        }
      } else {
#pragma unroll
        for (int i = 0; i < kItems; ++i) {
          run_add<Op>(run, row[i]);
          orow[i] = run_out<Op>(run);
        }
      }
      compute_sync();
      const Out* orows = reinterpret_cast<const Out*>(rows);
      if (full) {
        uint4* yv = reinterpret_cast<uint4*>(y + t0);
#pragma unroll
        for (int j = 0; j < kTile / 4 / kThreads; ++j) {
          const int p0 = (j * kThreads + tid) * 4;
          Out o[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) o[q] = orows[((p0 + q) / kItems) * kRow + (p0 + q) % kItems];
          st_stream(yv + j * kThreads + tid, pack16(o));
        }
      } else {
        for (int p = tid; p < kTile && t0 + p < n; p += kThreads) y[t0 + p] = orows[(p / kItems) * kRow + p % kItems];
      }
    } else {
      const int64_t base = t0 + (int64_t)tid * kItems;
      constexpr int kPer = 16 / (int)sizeof(Out);
#pragma unroll
      for (int g = 0; g < kItems / kPer; ++g) {
        Out o[kPer];
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
          if (exclusive) {
            o[q] = run_out<Op>(run);
            run_add<Op>(run, row[g * kPer + q]);
          } else {
            run_add<Op>(run, row[g * kPer + q]);
            o[q] = run_out<Op>(run);
          }
        }
        if (full) {
          st_stream(reinterpret_cast<uint4*>(y + base) + g, pack16(o));
        } else {
#pragma unroll
          for (int q = 0; q < kPer; ++q)
            if (base + g * kPer + q < n) y[base + g * kPer + q] = o[q];
        }
      }
    }
    compute_sync();  // the buffer is free for the tile after next
  };

  C run_mn = mm_highest<C>(), run_mx = mm_lowest<C>();
  if (tid == 0) s_next = atomicAdd(&hdr->tile_counter, 1u);
  compute_sync();
  int64_t t = s_next;
  if (t < tiles && full_tile(t)) fetch(t);
  int64_t t_prev = -1;
  T prev_off = Op::zero();  // tile t_prev: this thread's offset within it (warp offset + lane offset)
  int i = 0;
  while (t < tiles) {
    compute_sync();  // everyone has read s_next
    if (tid == 0) s_next = atomicAdd(&hdr->tile_counter, 1u);  // the next tile's id, one ahead
    C* rows = rows0 + (i & 1) * (kThreads * kRow);
    const int64_t t0 = t * kTile;
    const bool full = full_tile(t);
    if (full) {
#pragma unroll
      for (int j = 0; j < kLoads; ++j) {
        C e[V];
        S::unpack(raw[j], e);
        map_vec<V>(f, e);
        const int p0 = (j * kThreads + tid) * V;
#pragma unroll
        for (int q = 0; q < V; ++q) rows[((p0 + q) / kItems) * kRow + (p0 + q) % kItems] = e[q];
      }
    } else {
      for (int p = tid; p < kTile; p += kThreads)
        rows[(p / kItems) * kRow + p % kItems] = (t0 + p < n) ? f(S::cvt(x[t0 + p])) : C(0);
    }
    compute_sync();
    C* row = rows + tid * kRow;
    const T acc = row_total<Op, kItems>(row);
    if (minmax) {  // this thread's running min / max of f over its valid elements
      const int valid =
          full ? kItems : (int)imax<int64_t>(0, imin<int64_t>(kItems, n - t0 - (int64_t)tid * kItems));
      C mn, mx;
      row_minmax<C, kItems>(row, valid, mn, mx);
      run_mn = mm_min(run_mn, mn);
      run_mx = mm_max(run_mx, mx);
    }
    T warp_off, excl_lane, tile_tot;
    block_totals<Op>(acc, s_warp, warp_off, excl_lane, tile_tot);  // (its barrier also publishes s_next)
    if (tid == 0) {
      s_agg[i & 1] = Op::to_carry(tile_tot);
      s_tile_of[i & 1] = t;
      publish_aggregate<Op>(ws, t, Op::to_carry(tile_tot), t == stall_tile);
    }
    bar_arrive_n(kBarAgg + (i & 1), kBlockThreads);  // tile t goes to the look-back warp
    const int64_t t_next = s_next;
    if (t_next < tiles && full_tile(t_next)) fetch(t_next);  // in flight during the outputs below
    if (t_prev >= 0) {
      bar_sync_n(kBarExcl + ((i - 1) & 1), kBlockThreads);
      write_out(t_prev, rows0 + ((i - 1) & 1) * (kThreads * kRow), s_excl[(i - 1) & 1], prev_off);
    }
    t_prev = t;
    prev_off = Op::add(warp_off, excl_lane);
    t = t_next;
    ++i;
  }
  if (t_prev >= 0) {
    bar_sync_n(kBarExcl + ((i - 1) & 1), kBlockThreads);
    write_out(t_prev, rows0 + ((i - 1) & 1) * (kThreads * kRow), s_excl[(i - 1) & 1], prev_off);
  }
  if (tid == 0) s_tile_of[i & 1] = -1;
  bar_arrive_n(kBarAgg + (i & 1), kBlockThreads);  // the look-back warp stops
  if (minmax) block_minmax<C>(run_mn, run_mx, red, hdr, s_mn, s_mx);
}

// ---- the TMA-fed tile loop (4-byte inputs and outputs) -----------------------
//
// The same look-back schedule as k_scan, with the tiles moved by the TMA
// engine instead of by the compute warps.  x and y are viewed as 2-D tensors
// of rows of kI elements (the rows that lie wholly inside [0, n)); a tile is
// 256 rows, one per compute thread.  A box load with the kI * 4-byte swizzle
// (64 or 128 bytes) lands a thread's row as kI / 4 16-byte chunks whose
// positions are permuted by the row index, so the eight threads of a quarter
// warp read their own rows from eight different bank groups: each thread
// reads its row with 16-byte loads, conflict-free, with no scatter and no
// gather.  The stage is then used in place: phase 1 maps the row and writes
// the mapped values back (tile total, min / max, aggregate to the look-back
// warp); phase 2 -- kD tiles later, once the look-back warp has delivered the
// prefix -- turns them into the outputs, and one box store writes the tile
// back.  Loads outside the tensor read zeros and stores outside it are
// clipped, so a partial last tile needs no special case; the elements of a
// last, partial row (fewer than kI) are read and written by their thread.
//
// A block is 8 compute warps, the look-back warp and a producer warp, with a
// ring of kD + 2 stages.  The producer takes the tile ids from the atomic
// counter and issues the box loads; the compute warps' thread 0 issues the box
// stores and, at the top of each iteration, waits for the store issued one
// iteration earlier to finish reading its stage and hands that stage back to
// the producer (an mbarrier per stage each way).  The producer takes the id of
// a block's next tile only once the current tile's data has landed, so a
// block holds at most one tile beyond the one it computes: taking ids several
// tiles ahead made the first block to start hold consecutive ids, the next
// block's first tile wait for that block's later ones, and so on -- a cascade
// that ran the 2^28 scan ten times slower.  Within that limit a load still
// gets most of an iteration to land.
template <int kI_, int kD_>
struct TmaTile {
  static constexpr int kI = kI_;  // elements per row (per compute thread)
  static constexpr int kD = kD_;  // tiles between phase 1 and phase 2
  static_assert(kI == 16 || kI == 32, "rows of 64 or 128 bytes");
  static_assert(kThreads * kI <= scank::kTile, "a look-back line per 8,192 elements suffices");
  static_assert(kD == 1 || kD == 2, "phase-2 lag");
  static constexpr int kTile = kThreads * kI;                // elements per tile
  static constexpr uint32_t kStageBytes = (uint32_t)kTile * 4;
  static constexpr int kStages = kD + 2;
  static constexpr int kChunks = kI / 4;                     // 16-byte chunks per row
  static constexpr size_t kDynBytes = (size_t)kStages * kStageBytes + 1024;  // + alignment of the ring
  static constexpr CUtensorMapSwizzle kSwizzle = kI == 16 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
  // byte offset of chunk c of row r in a stage: the swizzle XORs the chunk
  // index with address bits 7.. (two bits for 64-byte, three for 128-byte rows)
  __device__ static __forceinline__ uint32_t chunk_off(int r, int c) {
    return (uint32_t)r * (kI * 4) + ((uint32_t)(c ^ ((kI == 16 ? r >> 1 : r) & (kChunks - 1))) << 4);
  }
};
constexpr int kTmaBlockThreads = kBlockThreads + 32;  // + the producer warp

__device__ __forceinline__ void tma_load_rows(uint32_t dst, const CUtensorMap* map, int row, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          dst),
      "l"(map), "r"(0), "r"(row), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_store_rows(const CUtensorMap* map, int row, uint32_t src) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(map), "r"(0),
               "r"(row), "r"(src)
               : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_plain(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// True in every compute thread iff `v` holds in all of them (a compute-warp barrier).
__device__ __forceinline__ bool compute_all(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\t"
      "setp.ne.u32 p, %1, 0;\n\t"
      "bar.red.and.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}\n"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kBarCompute), "n"(kThreads)
      : "memory");
  return r != 0;
}
constexpr uint64_t kStageWaitNs = 1000000000ull;  // 1 s for one stage hand-over before giving up
template <class C>
__device__ __forceinline__ C from_bits(uint32_t b);
template <>
__device__ __forceinline__ float from_bits<float>(uint32_t b) { return __uint_as_float(b); }
template <>
__device__ __forceinline__ uint32_t from_bits<uint32_t>(uint32_t b) { return b; }

template <class In, class F, class Op, class Src, class L>
__global__ void __launch_bounds__(kTmaBlockThreads, kBlocksPerSm)
    k_scan_tma(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap ymap,
               const In* __restrict__ x, typename Op::Out* y, int64_t n, const __grid_constant__ Src P,
               WsHeader* hdr, ScanWs ws, const typename Op::Out* carry_in, uint64_t timeout_ns, int64_t stall_tile,
               int exclusive, ScanRed red, int64_t tiles) {
  constexpr int kI = L::kI, kD = L::kD, kR = L::kStages;
  constexpr int kN = kD == 1 ? 2 : 4;  // hand-over slots in use at once
  using C = In;
  using T = typename Op::T;
  using Carry = typename Op::Carry;
  using Out = typename Op::Out;
  static_assert(sizeof(C) == 4 && sizeof(Out) == 4, "4-byte inputs and outputs");
  static_assert(std::is_same<typename Storage<In>::C, In>::value, "the input is its own compute type");

  __shared__ int64_t s_tile_of[kN];
  __shared__ Carry s_agg[kN], s_excl[kN];
  __shared__ int64_t s_stage_tile[kR];  // tile id of a stage's fill (-1: none left)
  __shared__ __align__(8) uint64_t s_full[kR], s_empty[kR];
  __shared__ T s_warp[kWarps];
  __shared__ C s_mn[kWarps], s_mx[kWarps];
  extern __shared__ __align__(16) unsigned char s_dyn[];
  const int tid = threadIdx.x, lane = tid & 31;
  unsigned char* const ring = s_dyn + ((1024u - (smem_addr(s_dyn) & 1023u)) & 1023u);
  const uint32_t ring_s = smem_addr(ring), full0 = smem_addr(&s_full[0]), empty0 = smem_addr(&s_empty[0]);
  if (tid == 0) {
    for (int st = 0; st < kR; ++st) {
      mbar_init(full0 + 8 * st, 1);
      mbar_init(empty0 + 8 * st, 1);
    }
    mbar_init_fence();
  }
  __syncthreads();

  if (tid >= kBlockThreads) {  // ---- the producer warp (one lane)
    if (lane != 0) return;
    for (int q = 0;; ++q) {
      const int st = q % kR;
      // the block's previous tile has landed (at most one tile held beyond the computed one),
      // and this stage's last tile has been stored out of it
      bool ok = q == 0 || mbar_wait_quiet(full0 + 8 * ((q - 1) % kR), (uint32_t)(((q - 1) / kR) & 1), kStageWaitNs);
      if (ok && q >= kR) ok = mbar_wait_quiet(empty0 + 8 * st, (uint32_t)(((q - kR) / kR) & 1), kStageWaitNs);
      const uint32_t id = ok ? atomicAdd(&hdr->tile_counter, 1u) : 0xFFFFFFFFu;
      if (!ok) set_status(hdr, TR_ERR_TIMEOUT, (uint32_t)q);
      const uint32_t bar = full0 + 8 * st;
      if ((int64_t)id < tiles) {
        s_stage_tile[st] = id;
        mbar_expect_tx(bar, L::kStageBytes);
        tma_load_rows(ring_s + (uint32_t)st * L::kStageBytes, &xmap, (int)id * kThreads, bar);
      } else {  // no tile left (or a failed hand-over): the compute warps stop at this stage
        s_stage_tile[st] = -1;
        mbar_arrive_plain(bar);
        return;
      }
    }
  }
  if (tid >= kThreads) {  // ---- the look-back warp
    lookback_warp<Op, C, kN>(s_tile_of, s_agg, s_excl, ws, hdr, timeout_ns, stall_tile, red, tiles, lane);
    return;
  }

  // ---- the compute warps
  const auto f = kernel_map<F>(P);
  const bool minmax = (red.ops & (TR_MIN | TR_MAX)) != 0;
  const Carry carry = carry_in ? Op::carry_of(*carry_in) : Carry{};
  const int64_t ragged = (n / kI) * kI;  // the first element of a last, partial row (== n: none)
  auto stage_of = [&](int st) { return ring + (size_t)st * L::kStageBytes; };
  auto load_row = [&](const unsigned char* stage, C* v) {
#pragma unroll
    for (int c = 0; c < L::kChunks; ++c) {
      const uint4 w = *reinterpret_cast<const uint4*>(stage + L::chunk_off(tid, c));
      v[4 * c] = from_bits<C>(w.x);
      v[4 * c + 1] = from_bits<C>(w.y);
      v[4 * c + 2] = from_bits<C>(w.z);
      v[4 * c + 3] = from_bits<C>(w.w);
    }
  };
  auto store_row = [&](unsigned char* stage, const auto* v) {
#pragma unroll
    for (int c = 0; c < L::kChunks; ++c) *reinterpret_cast<uint4*>(stage + L::chunk_off(tid, c)) = pack16(v + 4 * c);
  };
  // phase 2 of tile t (stage st): outputs from the mapped row and the tile's exclusive prefix
  auto finish_tile = [&](int64_t t, int st, Carry excl, const T& thread_off) {
    unsigned char* stage = stage_of(st);
    const int64_t e0 = t * L::kTile + (int64_t)tid * kI;
    C v[kI];
    load_row(stage, v);
    const Carry prefix = Op::cadd(carry, excl);
    T run;
    if constexpr (std::is_same<Op, OpF32>::value) {
      run = ff_add(prefix, thread_off);
    } else {
      run = Op::add((T)prefix, thread_off);
    }
    Out o[kI];
    if (exclusive) {
#pragma unroll
      for (int k = 0; k < kI; ++k) {
        o[k] = run_out<Op>(run);
        run_add<Op>(run, v[k]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < kI; ++k) {
        run_add<Op>(run, v[k]);
        o[k] = run_out<Op>(run);
      }
    }
    if (e0 == ragged && e0 < n) {  // the partial last row: outside the tensor, written directly
      for (int k = 0; k < kI; ++k)
        if (e0 + k < n) y[e0 + k] = o[k];
    }
    store_row(stage, o);
    fence_async_smem();  // the rows, before the box store reads them
    compute_sync();
    if (tid == 0) tma_store_rows(&ymap, (int)(t * kThreads), ring_s + (uint32_t)st * L::kStageBytes);
  };

  // tiles in phase-2 order: pend_t[k] / pend_off[k] hold the tile handed over k + 1 iterations ago
  int64_t pend_t[kD];
  T pend_off[kD];
#pragma unroll
  for (int k = 0; k < kD; ++k) {
    pend_t[k] = -1;
    pend_off[k] = Op::zero();
  }
  C run_mn = mm_highest<C>(), run_mx = mm_lowest<C>();
  int stored = 0;  // box stores issued (the stage of store s is s % kR: stores go in fill order)
  int j = 0;
  bool ok = true;
  // the oldest pending tile: wait for its prefix, write it out, shift the queue
  auto drain_one = [&](int jj) {
    const int64_t tp = pend_t[kD - 1];
    if (tp >= 0) {
      const int q = jj - kD;  // its fill (and iteration) number
      bar_sync_n(kBarAgg + kN + q % kN, kBlockThreads);
      finish_tile(tp, q % kR, s_excl[q % kN], pend_off[kD - 1]);
      ++stored;
    }
#pragma unroll
    for (int k = kD - 1; k > 0; --k) {
      pend_t[k] = pend_t[k - 1];
      pend_off[k] = pend_off[k - 1];
    }
    pend_t[0] = -1;
  };
  while (true) {
    // hand the stage of the store issued one iteration ago back to the producer
    if (tid == 0 && stored > 0) {
      asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
      mbar_arrive_plain(empty0 + 8 * ((stored - 1) % kR));
    }
    const int st = j % kR;
    ok = compute_all(mbar_wait_quiet(full0 + 8 * st, (uint32_t)((j / kR) & 1), kStageWaitNs));
    if (!ok) {
      if (tid == 0) set_status(hdr, TR_ERR_TIMEOUT, (uint32_t)j);
      break;
    }
    const int64_t t = s_stage_tile[st];
    if (t < 0) break;
    // ---- phase 1: map the row in place, total it
    unsigned char* stage = stage_of(st);
    const int64_t e0 = t * L::kTile + (int64_t)tid * kI;
    const int valid = (int)imax<int64_t>(0, imin<int64_t>(kI, n - e0));
    C v[kI];
    load_row(stage, v);
    if (valid == kI) {
#pragma unroll
      for (int h = 0; h < kI; h += 16) map_vec<16>(f, v + h);  // 16 values at a time (registers)
    } else {
#pragma unroll
      for (int k = 0; k < kI; ++k) {
        C xv = v[k];
        if (e0 == ragged && k < valid) xv = x[e0 + k];  // the partial last row is not in the tensor
        v[k] = k < valid ? f(xv) : C(0);
      }
    }
    store_row(stage, v);
    const T acc = row_total<Op, kI>(v);
    if (minmax) {  // this thread's running min / max of f over its valid elements
      C mn, mx;
      row_minmax<C, kI>(v, valid, mn, mx);
      run_mn = mm_min(run_mn, mn);
      run_mx = mm_max(run_mx, mx);
    }
    T warp_off, excl_lane, tile_tot;
    block_totals<Op>(acc, s_warp, warp_off, excl_lane, tile_tot);
    if (tid == 0) {
      s_agg[j % kN] = Op::to_carry(tile_tot);
      s_tile_of[j % kN] = t;
      publish_aggregate<Op>(ws, t, Op::to_carry(tile_tot), t == stall_tile);
    }
    bar_arrive_n(kBarAgg + j % kN, kBlockThreads);  // tile t goes to the look-back warp
    // ---- phase 2 of the tile handed over kD iterations ago
    drain_one(j);
    pend_t[0] = t;
    pend_off[0] = Op::add(warp_off, excl_lane);
    ++j;
  }
#pragma unroll
  for (int k = 0; k < kD; ++k) drain_one(j + k);
  if (tid == 0) {
    s_tile_of[j % kN] = -1;
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");  // the box stores are complete
  }
  bar_arrive_n(kBarAgg + j % kN, kBlockThreads);  // the look-back warp stops
  if (minmax) block_minmax<C>(run_mn, run_mx, red, hdr, s_mn, s_mx);
  if (!ok && tid == 0)  // after a failed wait: the producer's load for this stage, if any, lands first
    mbar_wait_quiet(full0 + 8 * (j % kR), (uint32_t)((j / kR) & 1), kStageWaitNs);
}

// Clear the scan state and launch the scan for the storage type In, map F and
// output arithmetic Op; P is the map's source.  4-byte inputs and outputs on
// 16-byte aligned arrays of at least one tile take the TMA-fed kernel; the
// rest take k_scan.  Both use tiles of 8,192 elements.
template <class In, class F, class Op, class Src>
tr_status launch(const Src& P, const In* x, typename Op::Out* y, int64_t n, const typename Op::Out* carry,
                 const tr_exec* e, const ScanOpts& opt) {
  const ScanWs ws{reinterpret_cast<unsigned char*>(ws_body(e))};
  const uint64_t timeout_ns = (uint64_t)(e->wait_timeout_us ? e->wait_timeout_us : 1000000u) * 1000ull;
  const int vec_ok = aligned_to(x, 16) && aligned_to(y, 16);
  cudaStream_t st = stream_of(e);
  WsHeader* hdr = ws_header(e);
  const ScanRed red{opt.sum, opt.mn, opt.mx, (int32_t)opt.sum_t, opt.ops};
  // every call starts from a zero tile counter, cleared reduction words and clear look-back
  // lines: one memset from the counter through the last line (the error words before the
  // counter are left alone)
  auto clear = [&](int64_t tiles) {
    unsigned char* from = reinterpret_cast<unsigned char*>(&hdr->tile_counter);
    const size_t bytes = (size_t)(reinterpret_cast<unsigned char*>(ws.lines) - from) + (size_t)tiles * kLineBytes;
    return cuda_status(cudaMemsetAsync(from, 0, bytes, st), "cudaMemsetAsync(scan state)");
  };
  const int64_t lines = e->workspace_bytes > (size_t)kWsHeader
                            ? (int64_t)((e->workspace_bytes - (size_t)kWsHeader) / (size_t)kLineBytes)
                            : 0;
  if constexpr (sizeof(In) == 4 && sizeof(typename Op::Out) == 4) {
    auto go_tma = [&](auto layout_tag) -> tr_status {
      using L = decltype(layout_tag);
      constexpr int kI = L::kI;
      const int64_t tiles = ceil_div(n, L::kTile);
      const uint64_t rows = (uint64_t)(n / kI);
      const CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_UINT32;
      CUtensorMap xm, ym;
      tr_status s = make_tensor_map_2d(&xm, x, dt, kI, rows, kI * 4, kI, kThreads, L::kSwizzle);
      if (!s) s = make_tensor_map_2d(&ym, y, dt, kI, rows, kI * 4, kI, kThreads, L::kSwizzle);
      if (!s) s = clear(tiles);
      if (s) return s;
      auto kern = k_scan_tma<In, F, Op, Src, L>;
      if ((s = ensure_dyn_smem((const void*)kern, (int)L::kDynBytes, "cudaFuncSetAttribute(k_scan_tma)"))) return s;
      const int64_t resident =
          (int64_t)dev_info().sm_count * blocks_per_sm((const void*)kern, kTmaBlockThreads, L::kDynBytes);
      const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(tiles, resident));
      kern<<<(unsigned)grid, kTmaBlockThreads, L::kDynBytes, st>>>(xm, ym, x, y, n, P, hdr, ws, carry, timeout_ns,
                                                                    e->debug_stall_tile, opt.exclusive, red, tiles);
      return launch_status("k_scan_tma");
    };
    // 32-element rows, phase 2 one tile after phase 1 (measured on B300 at 2^28, u32 splitmix32 /
    // f32 x^2: 382 / 447 us; 16-element rows with phase 2 two tiles later: 455 / 570 us)
    using L = TmaTile<32, 1>;
    // (the row coordinates of the boxes are 32-bit)
    if (vec_ok && n >= L::kTile && n / 32 < 0x7FFFFFFF && ceil_div(n, L::kTile) <= lines) return go_tma(L());
  }
  const int64_t tiles = std::max<int64_t>(1, ceil_div(n, kTile));  // n = 0 (with a reduction): one empty tile
  if (tiles > 0x7FFFFFFF) return fail(TR_ERR_INVALID_ARG, "too many tiles");
  tr_status s = clear(tiles);
  if (s) return s;
  auto kern = k_scan<In, F, Op, Src>;
  if ((s = ensure_dyn_smem((const void*)kern, (int)kDynBytes, "cudaFuncSetAttribute(k_scan)"))) return s;
  // persistent: at most the resident blocks (every block that holds a tile id runs)
  const int64_t resident = (int64_t)dev_info().sm_count * blocks_per_sm((const void*)kern, kBlockThreads, kDynBytes);
  const int64_t grid = std::max<int64_t>(1, std::min<int64_t>(tiles, resident));
  kern<<<(unsigned)grid, kBlockThreads, kDynBytes, st>>>(x, y, n, vec_ok, P, hdr, ws, carry, timeout_ns,
                                                         e->debug_stall_tile, opt.exclusive, red, tiles);
  return launch_status("k_scan");
}

}  // namespace scank
}  // namespace tr
