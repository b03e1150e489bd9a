// segreduce_kernel.cuh -- the kernels of tr_segmented_reduce, sum / min / max of
// f per segment, as templates over the storage type, the map and the map's
// source (the family's MapParams, or a user-supplied functor passed by
// value), with their launcher.
//
// Layout of the work: the array is cut into equal contiguous element ranges,
// one per warp of a resident grid.  A warp finds the first segment touching
// its range with a 32-ary search over the offsets (log32 dependent loads),
// then walks the segments in order, keeping a window of 32 offsets in
// registers (one per lane).  Each segment piece -- the intersection of a
// segment with the range -- is reduced by the whole warp: 128-bit loads,
// kRangeUnroll vectors in flight per lane, the map in registers, Kahan-compensated
// per-lane sums of pairwise vector sums, then a float-float warp butterfly.
//   * a piece that is the whole segment is written out directly;
//   * a piece cut by the range start (head) or end (tail) goes to a per-warp
//     workspace slot as FP64, and a second, small kernel (one thread per
//     warp) joins each cut segment's pieces in warp order in FP64.
// The combination order is fixed by the grid, so results are deterministic.
// Offsets are checked while walking (monotone, within [0, n]); a violation is
// reported through the workspace status word instead of faulting.
#pragma once

#include "accum.cuh"
#include "internal.h"
#include "range.cuh"

namespace tr {
namespace segk {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kMaxGrid = 2048;

struct SegSlot {
  long long seg;  // segment id, -1 = unused
  double sum;
  float mn, mx;
  int32_t through;  // the piece covers the whole range (segment continues)
  int32_t pad;
};
static_assert(sizeof(SegSlot) == 32, "slot size");

// First index i in [0, m] with off[i] >= a (off non-decreasing, off[m] >= a),
// found by the warp with 32-ary narrowing; every lane returns it.
__device__ __forceinline__ int64_t warp_lower_bound(const int64_t* off, int64_t m, int64_t a, int lane) {
  int64_t lo = 0, hi = m + 1;  // answer in [lo, hi)
  while (hi - lo > 32) {
    const int64_t step = (hi - lo + 31) / 32;
    const int64_t p = lo + (int64_t)lane * step;
    const bool ge = p < hi ? (__ldg(off + p) >= a) : true;
    const unsigned mask = __ballot_sync(kFull, ge);
    const int k = mask ? __ffs(mask) - 1 : 32;
    const int64_t nlo = k == 0 ? lo : lo + (int64_t)(k - 1) * step + 1;
    const int64_t nhi = imin<int64_t>(hi, lo + (int64_t)k * step + 1);
    lo = nlo;
    hi = imax<int64_t>(nhi, nlo + 1);
  }
  const int64_t p = lo + lane;
  const bool ge = p < hi ? (__ldg(off + p) >= a) : true;
  const unsigned mask = __ballot_sync(kFull, ge);
  return lo + (mask ? __ffs(mask) - 1 : 0);
}

__device__ __forceinline__ void write_slot(SegSlot* sl, long long seg, const Acc<float>::W& w, int through) {
  sl->seg = seg;
  sl->sum = ff_to_double(w.s);
  sl->mn = w.mn;
  sl->mx = w.mx;
  sl->through = through;
}

// The two ends of the offsets contract (off[0] = 0, off[nseg] = n): the warp
// whose range starts at element 0 and the warp whose range ends at n check
// them; the walk itself checks every segment it visits (lo <= hi, within
// [0, n]).  A violation is reported, never trapped.
__device__ __forceinline__ void check_ends(const int64_t* off, int64_t nseg, int64_t n, bool first, bool last,
                                           WsHeader* hdr) {
  if (first && __ldg(off) != 0) set_status(hdr, TR_ERR_DEVICE_ASSERT, 0u);
  if (last && __ldg(off + nseg) != n) set_status(hdr, TR_ERR_DEVICE_ASSERT, (uint32_t)nseg);
}

template <class In, class F, class Src>
__global__ void __launch_bounds__(kThreads) k_segreduce(const In* __restrict__ x, int64_t n,
                                                        const int64_t* __restrict__ off, int64_t nseg, int64_t range,
                                                        int x_aligned, const __grid_constant__ Src P,
                                                        RedOut out, WsHeader* hdr, SegSlot* slots) {
  const int lane = threadIdx.x & 31;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int64_t a = gw * range;
  const int64_t b = imin<int64_t>(n, a + range);
  const bool active = a < n || (n == 0 && gw == 0);
  const bool last = active && b == n;
  bool wrote_head = false, wrote_tail = false;

  if (active) {
    if (lane == 0) check_ends(off, nseg, n, gw == 0, last, hdr);
    const auto f = kernel_map<F>(P);
    const int64_t i0 = warp_lower_bound(off, nseg, a, lane);
    int64_t s = (i0 <= nseg && __ldg(off + i0) == a) ? i0 : i0 - 1;
    if (s < 0) s = 0;
    int64_t wbase = s;
    int64_t win = (wbase + lane <= nseg) ? __ldg(off + wbase + lane) : n;
    while (s < nseg) {
      if (s + 1 - wbase >= 32) {
        wbase = s;
        win = (wbase + lane <= nseg) ? __ldg(off + wbase + lane) : n;
      }
      const int64_t lo_s = __shfl_sync(kFull, win, (int)(s - wbase));
      const int64_t hi_s = __shfl_sync(kFull, win, (int)(s + 1 - wbase));
      if (lo_s >= b && !(last && lo_s == n)) break;
      if (hi_s < lo_s || lo_s < 0 || hi_s > n) {
        if (lane == 0) set_status(hdr, TR_ERR_DEVICE_ASSERT, (uint32_t)s);
        break;
      }
      const int64_t pa = imax(lo_s, a), pb = imin(hi_s, b);
      const Acc<float> acc = warp_reduce_range<In>(x, pa, pb, x_aligned, f, lane, b);
      const Acc<float>::W w = acc.warp();
      const bool head_open = lo_s < a, tail_open = hi_s > b;
      if (lane == 0) {
        if (!head_open && !tail_open) {
          store_result(out, s, Acc<float>::to_partial(w), true);
        } else if (head_open) {
          write_slot(&slots[2 * gw], s, w, tail_open ? 1 : 0);
          wrote_head = true;
        } else {
          write_slot(&slots[2 * gw + 1], s, w, 0);
          wrote_tail = true;
        }
      }
      ++s;
    }
  }
  if (lane == 0) {
    if (!wrote_head) slots[2 * gw].seg = -1;
    if (!wrote_tail) slots[2 * gw + 1].seg = -1;
  }

}


// ---------------------------------------------------------------------------
// The same walk with the loads decoupled from the arithmetic (16-byte aligned
// x): every warp streams its range through a private ring of stages in shared
// memory, filled by TMA bulk copies (one lane issues them, an mbarrier per
// stage tracks the bytes), so all but one stage are in flight while the warp
// maps and accumulates the current one.  A chunk (one stage) holds 16 elements
// per lane whatever the storage type: 4 vectors per lane in 2 KiB stages for
// FP32, 2 vectors per lane in 1 KiB stages for FP16 / BF16.  Segment boundaries
// are handled inside a chunk: the common case (the chunk lies in one segment)
// accumulates all 16 values at once; a chunk holding boundaries makes one masked
// pass per piece and emits each finished segment.
//
// Ring size and blocks per SM follow the cost of the map (measured on B300 at
// 2^28 elements, 65,536 segments): maps of a few instructions per element run
// best as few warps with deep rings (one block of 8 warps, 16 KiB rings: 90 %
// of the copy bandwidth), the division-bound maps need every warp the
// registers allow (three blocks, 8 KiB rings), and Horner polynomials sit in
// between (two blocks, 8 KiB rings).
// ---------------------------------------------------------------------------
//
// A ring stage holds `sub` consecutive chunks: one mbarrier wait and one bulk
// copy serve them all, so the per-stage costs (wait, release, copy issue) are
// shared by sub x 16 elements per lane.
// (Measured on B300 for rational 6/6 at 2^28: two chunks per 4 KiB stage, 279
// us; one per 2 KiB stage, 290 us.)
template <class F>
struct SegShape {  // division-bound maps (rational, Newton) and the rest
  static constexpr int ring = 8192, blocks = 3, sub = 2;
  // warp ranges per resident warp: twice as many, half as long, run in two waves (measured on B300 for
  // rational 6/6 at 2^28: 267 us against 272 us with one range per resident warp; four: 267 us)
  static constexpr int waves = 2;
};
template <class T>
struct SegShape<Identity<T>> {
  static constexpr int ring = 16384, blocks = 1, sub = 1;
  static constexpr int waves = 1;
};
template <class T>
struct SegShape<Square<T>> {
  static constexpr int ring = 16384, blocks = 1, sub = 1;
  static constexpr int waves = 1;
};
template <class T, int D>
struct SegShape<Horner<T, D>> {
  static constexpr int ring = 8192, blocks = 2, sub = 1;
  static constexpr int waves = 1;
};
template <class T>
struct SegShape<HornerN<T>> {
  static constexpr int ring = 8192, blocks = 2, sub = 1;
  static constexpr int waves = 1;
};
constexpr int kMaxStages = 16;
constexpr uint64_t kTmaWaitNs = 1000000000ull;         // 1 s for one bulk copy before giving up

template <class In, class F, class Src>
__global__ void __launch_bounds__(kThreads, SegShape<F>::blocks) k_segreduce_tma(const In* __restrict__ x, int64_t n,
                                                            const int64_t* __restrict__ off, int64_t nseg,
                                                            int64_t range, int /*x_aligned: always*/,
                                                            const __grid_constant__ Src P, RedOut out,
                                                            WsHeader* hdr, SegSlot* slots) {
  using S = Storage<In>;
  constexpr int V = S::kVec;
  constexpr int E = 16;                      // elements per lane per chunk
  constexpr int kU = E / V;                  // vectors per lane per chunk
  constexpr int kChunkVec = 32 * kU;         // 16-byte vectors per chunk
  constexpr int kSub = SegShape<F>::sub;     // chunks per ring stage
  constexpr int kStageVec = kChunkVec * kSub;
  constexpr int kRingBytes = SegShape<F>::ring;  // per warp
  constexpr int kStages = kRingBytes / (kStageVec * 16);
  static_assert(kStages >= 2 && kStages <= kMaxStages, "ring layout");
  extern __shared__ __align__(128) uint4 ring_all[];
  __shared__ __align__(8) uint64_t bars[kWarps][kMaxStages];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t gw = (int64_t)blockIdx.x * kWarps + wid;
  const int64_t a = gw * range;
  const int64_t b = imin<int64_t>(n, a + range);
  const bool last = a < n && b == n;
  const uint4* ring = ring_all + (size_t)wid * kStages * kStageVec;
  const uint32_t ring_s = smem_addr(ring), bar0 = smem_addr(&bars[wid][0]);
  bool wrote_head = false, wrote_tail = false;
  if (lane == 0) {
    for (int st = 0; st < kStages; ++st) mbar_init(bar0 + 8 * st, 1);
    mbar_init_fence();
  }
  __syncwarp();

  if (a < n) {
    const uint4* xv = reinterpret_cast<const uint4*>(x);
    const int64_t va = a / V, vend = b / V;  // whole vectors [va, vend); elements [vend*V, b) are the tail
    const int nchunks = (int)((vend - va + kChunkVec - 1) / kChunkVec);
    const int nfull = (int)((vend - va) / kChunkVec);  // chunks holding kChunkVec vectors
    const int nstages = (nchunks + kSub - 1) / kSub;    // stage fills over the range
    auto issue = [&](int j) {  // lane 0: fetch stage fill j (chunks j*kSub ..) into its slot
      const int st = j % kStages;
      const int64_t v0 = va + (int64_t)j * kStageVec;
      const uint32_t bytes = (uint32_t)imin<int64_t>(kStageVec, vend - v0) * 16u;
      mbar_expect_tx(bar0 + 8 * st, bytes);
      bulk_load(ring_s + (uint32_t)st * kStageVec * 16u, xv + v0, bytes, bar0 + 8 * st);
    };
    if (lane == 0)
      for (int j = 0; j < imin(kStages, nstages); ++j) issue(j);

    const auto f = kernel_map<F>(P);
    const int64_t i0 = warp_lower_bound(off, nseg, a, lane);
    int64_t s = (i0 <= nseg && __ldg(off + i0) == a) ? i0 : i0 - 1;
    if (s < 0) s = 0;
    int64_t wbase = s;
    int64_t win = (wbase + lane <= nseg) ? __ldg(off + wbase + lane) : n;
    int64_t lo_s = 0, hi_s = 0;
    int kfast = 0;  // chunks [.., kfast) are full and lie wholly inside segment s
    bool ok = true;
    auto bounds = [&]() {  // lo_s, hi_s of segment s (warp-uniform); false on invalid offsets
      if (s + 1 - wbase >= 32) {
        wbase = s;
        win = (wbase + lane <= nseg) ? __ldg(off + wbase + lane) : n;
      }
      lo_s = __shfl_sync(kFull, win, (int)(s - wbase));
      hi_s = __shfl_sync(kFull, win, (int)(s + 1 - wbase));
      if (hi_s < lo_s || lo_s < 0 || hi_s > n) {
        if (lane == 0) set_status(hdr, TR_ERR_DEVICE_ASSERT, (uint32_t)s);
        return false;
      }
      kfast = (int)imin<int64_t>(nfull, imax<int64_t>(0, hi_s - a) / (kChunkVec * V));
      return true;
    };
    if (lane == 0) check_ends(off, nseg, n, a == 0, last, hdr);
    ok = s < nseg && bounds();
    // With valid offsets the first segment starts at or before a; one that starts
    // later (off[0] > 0, reported above) must not take whole chunks before it.
    if (lo_s > a) kfast = 0;
    bool head_open = ok && lo_s < a;
    Acc<float> acc;
    auto finish = [&]() {  // segment s ends inside this range
      const Acc<float>::W w = acc.warp();
      if (lane == 0) {
        if (head_open) {
          write_slot(&slots[2 * gw], s, w, 0);
          wrote_head = true;
        } else {
          store_result(out, s, Acc<float>::to_partial(w), true);
        }
      }
      head_open = false;
      acc = Acc<float>();
    };
    auto advance = [&]() { return ++s < nseg && bounds(); };
    // chunk k: vectors [v0, v0 + cnt) of x, staged in ring stage st.  Every lane maps
    // its kU vectors once; a chunk inside one segment is accumulated whole, any other
    // (segment boundaries inside it, or a short last chunk) by one masked pass per
    // piece of a segment, on chunk-relative element positions.
    auto chunk = [&](int st, int k) -> bool {
      const uint4* src = ring + st * kStageVec + (k % kSub) * kChunkVec;
      float e[E];
#pragma unroll
      for (int u = 0; u < kU; ++u) S::unpack(src[u * 32 + lane], e + u * V);  // stale past cnt: masked
      map_vec<E>(f, e);  // all 16 values at once: independent chains interleave
      if (k < kfast) {
        acc.template add_vec<E>(e);
        return true;
      }
      const int64_t v0 = va + (int64_t)k * kChunkVec;
      const int cnt = (int)imin<int64_t>(kChunkVec, vend - v0);
      const int64_t ca = v0 * V, cb = (v0 + cnt) * V;
      if (lo_s >= cb) return true;  // the chunk lies before segment s (offsets breaking the contract)
      int lo = (int)imax<int64_t>(lo_s - ca, 0);
      while (true) {
        const int end = (int)(imin(hi_s, cb) - ca);
        const int base = lane * V - lo;
        const unsigned len = (unsigned)(end - lo);
        acc.template add_if<E>(e, [&](int i) { return (unsigned)(base + (i / V) * 32 * V + i % V) < len; });
        if (hi_s > cb) return true;
        finish();
        if (!advance()) return false;
        lo = (int)(lo_s - ca);
        if (lo_s >= cb) return true;
      }
    };

    // Stage fills issued at any point: [0, min(nstages, j + kStages)) while chunks of fill j
    // are processed (fill j - 1 has been released).  After an early stop, fills
    // [pending, min(nstages, j + kStages)) may still be in flight.
    int k = 0, pending = ok ? nstages : 0;  // not ok already: the first fills are in flight
    for (; k < nchunks && ok; ++k) {
      const int j = k / kSub, st = j % kStages;
      if (k % kSub == 0 && !mbar_wait_until(bar0 + 8 * st, (uint32_t)((j / kStages) & 1), kTmaWaitNs)) {
        if (lane == 0) set_status(hdr, TR_ERR_TIMEOUT, (uint32_t)gw);
        ok = false;
        pending = j;  // fill j itself may still be landing
        break;
      }
      ok = chunk(st, k);
      if (!ok) {
        pending = j + 1;  // fill j was waited for
        break;
      }
      // after the stage's last chunk every lane has read it: hand it back to the copy engine
      if (k % kSub == kSub - 1 || k == nchunks - 1) {
        __syncwarp();
        if (lane == 0 && j + kStages < nstages) {
          fence_async_smem();
          issue(j + kStages);
        }
      }
    }
    if (ok && vend * V < b) {  // ragged tail (last range only): one element per lane
      const int64_t ca = vend * V;
      const int tl = (int)(b - ca);
      const bool has = lane < tl;
      const float ev = has ? f(S::cvt(x[ca + lane])) : 0.0f;
      if (hi_s >= b) {
        if (has) acc.add(ev);
      } else {
        int lo = 0;
        while (true) {
          const int end = (int)(imin(hi_s, b) - ca);
          if (has && lane >= lo && lane < end) acc.add(ev);
          if (hi_s > b) break;
          finish();
          if (!advance()) {
            ok = false;
            break;
          }
          lo = (int)(lo_s - ca);
          if (lo_s >= b) break;
        }
        // (here every fill has been waited for and none is in flight: pending stays nstages)
      }
    }
    if (ok) {
      if (lo_s < b) {     // segment s started in (or before) this range
        if (hi_s == b) {  // ... and ends exactly at its end
          finish();
          advance();
        } else {          // ... and continues into the next range
          const Acc<float>::W w = acc.warp();
          if (lane == 0) {
            if (head_open) {
              write_slot(&slots[2 * gw], s, w, 1);
              wrote_head = true;
            } else {
              write_slot(&slots[2 * gw + 1], s, w, 0);
              wrote_tail = true;
            }
          }
        }
      }
      // a segment starting at b belongs to the next range; only the last range also
      // emits the empty segments sitting at n
      if (last)
        while (s < nseg && lo_s == n && hi_s == n) {
          finish();
          if (!advance()) break;
        }
    }
    // after an early stop, wait (bounded) for the copies still in flight before the shared
    // memory is released: chunks issued but not yet taken from the ring
    if (!ok && pending < nstages) {
      const int to = imin(nstages, k / kSub + kStages);
      for (int j = pending; j < to; ++j)
        mbar_wait_until(bar0 + 8 * (j % kStages), (uint32_t)((j / kStages) & 1), kTmaWaitNs);
    }
  }
  if (lane == 0) {
    if (!wrote_head) slots[2 * gw].seg = -1;
    if (!wrote_tail) slots[2 * gw + 1].seg = -1;
  }
}

// The second launch (k_join_cut, defined once in the library): joins the
// pieces of segments cut by warp-range ends.
tr_status launch_join(const RedOut& out, WsHeader* hdr, const SegSlot* slots, int64_t nw, cudaStream_t st);

template <class In, class F, class Src>
tr_status launch(const Src& P, const In* x, int64_t n, const int64_t* off, int64_t n_seg, const RedOut& out,
                 const tr_exec* e) {
  cudaStream_t st = stream_of(e);
  const int x_aligned = aligned_to(x, 16);
  constexpr int V = Storage<In>::kVec;
  const bool tma = x_aligned && n > 0;
  auto kern = tma ? k_segreduce_tma<In, F, Src> : k_segreduce<In, F, Src>;
  const size_t smem = tma ? (size_t)kWarps * SegShape<F>::ring : 0;  // kStages * stage bytes == ring
  if (tma) {
    tr_status s = ensure_dyn_smem((const void*)kern, (int)smem, "cudaFuncSetAttribute(k_segreduce_tma)");
    if (s) return s;
  }
  const int64_t resident = (int64_t)dev_info().sm_count * blocks_per_sm((const void*)kern, kThreads, smem);
  const int64_t grid_full = std::min<int64_t>(resident * (tma ? SegShape<F>::waves : 1), kMaxGrid);
  const int64_t quantum = 32 * V;  // range starts stay 16-byte aligned
  int64_t range = ceil_div(std::max<int64_t>(n, 1), grid_full * kWarps);
  range = ceil_div(range, quantum) * quantum;
  const int64_t warps_needed = std::max<int64_t>(1, ceil_div(n, range));
  const int64_t grid = ceil_div(warps_needed, kWarps);
  SegSlot* slots = reinterpret_cast<SegSlot*>(ws_body(e));
  kern<<<(unsigned)grid, kThreads, smem, st>>>(x, n, off, n_seg, range, x_aligned, P, out, ws_header(e), slots);
  tr_status ls = launch_status("k_segreduce");
  if (ls) return ls;
  return launch_join(out, ws_header(e), slots, grid * kWarps, st);
}

}  // namespace segk
}  // namespace tr
