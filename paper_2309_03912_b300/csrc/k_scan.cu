// k_scan.cu -- tr_scan: inclusive prefix sums of f(x) in one pass.
//
// Single-pass scan with decoupled look-back (Merrill & Garland, "Single-pass
// parallel prefix scan with decoupled look-back", NVR-2016-002):
//   * each block takes a tile id from an atomic counter (dynamic ids: every
//     tile's predecessors have already started, so waiting on them ends);
//   * a thread owns kItems contiguous elements (128-bit loads) and keeps only
//     the mapped values in registers; warps scan lane totals with shuffles and
//     the block combines warp totals in shared memory;
//   * the tile publishes its aggregate (flag A), then the whole block looks
//     back over kThreads predecessors per round (one flag per thread), summing
//     aggregates until it meets an inclusive prefix (flag P), and publishes its
//     own inclusive prefix.  With hundreds of tiles in flight the nearest P is
//     usually several hundred tiles back, so a block-wide window takes one or
//     two rounds where a single warp would need tens;
//   * every wait is bounded by a %globaltimer deadline and an abort word: on
//     expiry the block records TR_ERR_TIMEOUT and finishes instead of hanging.
// Each call clears the tile flags and the tile counter with two memsets on
// the stream (graph-capturable) before the kernel.  Predecessor flags are
// polled with relaxed loads; one acquire fence per thread and round orders the
// reads of the values behind them.
//
// Arithmetic: u32 wraps modulo 2^32; u32 -> u64 is exact; float scans keep
// float-float (hi, lo) pairs inside a tile, FP64 between tiles, and round each
// output once from the compensated prefix.
#include "dispatch.cuh"

namespace tr {

namespace {

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
  __device__ static T lift(uint32_t v) { return v; }
  __device__ static T add(T a, T b) { return a + b; }
  __device__ static Carry to_carry(T a) { return a; }
  __device__ static Carry cadd(Carry a, Carry b) { return a + b; }
  __device__ static T shfl_up(T a, int d) { return __shfl_up_sync(kFull, a, d); }
  __device__ static Carry shfl_xor_c(Carry a, int d) { return __shfl_xor_sync(kFull, a, d); }
};

struct OpF32 {
  using T = FF;
  using Carry = double;
  using Out = float;
  __device__ static T zero() { return FF{0.f, 0.f}; }
  __device__ static T add(T a, T b) { return ff_add(a, b); }
  __device__ static Carry to_carry(T a) { return ff_to_double(a); }
  __device__ static Carry cadd(Carry a, Carry b) { return a + b; }
  __device__ static T shfl_up(T a, int d) { return FF{__shfl_up_sync(kFull, a.hi, d), __shfl_up_sync(kFull, a.lo, d)}; }
  __device__ static Carry shfl_xor_c(Carry a, int d) { return __shfl_xor_sync(kFull, a, d); }
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

struct ScanWs {
  uint32_t* flags;
  void* agg;
  void* incl;
};

// Decoupled look-back by the whole block for `tile` (aggregate already known):
// publishes A, then scans kThreads predecessors per round (one flag per
// thread) until an inclusive prefix P bounds the sum, publishes its own P and
// returns the exclusive prefix (the same value in every thread).  Every wait
// is bounded by `deadline` and the abort word.
template <class Op>
struct LookbackSmem {
  typename Op::Carry red[kWarps];
  int first[kWarps];
};

template <class Op>
__device__ __forceinline__ typename Op::Carry block_lookback(int64_t tile, typename Op::Carry aggregate, ScanWs ws,
                                                             WsHeader* hdr, uint64_t timeout_ns, bool stall,
                                                             LookbackSmem<Op>& sm) {
  using Carry = typename Op::Carry;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  Carry* agg = static_cast<Carry*>(ws.agg);
  Carry* incl = static_cast<Carry*>(ws.incl);
  Carry excl = Carry(0);
  if (tile == 0) {
    if (tid == 0 && !stall) {
      incl[0] = aggregate;
      st_release_u32(&ws.flags[0], kFlagP);
    }
    return excl;
  }
  if (tid == 0 && !stall) {
    agg[tile] = aggregate;
    st_release_u32(&ws.flags[tile], kFlagA);
  }
  const uint64_t deadline = globaltimer_ns() + timeout_ns;
  int64_t pos = tile - 1;
  while (true) {
    const int64_t idx = pos - tid;
    uint32_t st = kFlagP;  // before tile 0: an inclusive prefix of 0
    int gave_up = 0;
    if (idx >= 0) {  // relaxed polling; one acquire fence once the flag is seen
      for (int polls = 0;; ++polls) {
        st = ld_relaxed_u32(&ws.flags[idx]) & 3u;
        if (st) break;
        if ((polls & 15) == 15 && (globaltimer_ns() > deadline || ld_relaxed_u32(&hdr->abort) != 0u)) {
          gave_up = 1;
          break;
        }
        if (polls > 8) __nanosleep(20);
      }
      fence_acq_rel_gpu();
    }
    if (__syncthreads_or(gave_up)) {
      if (tid == 0 && !ld_relaxed_u32(&hdr->abort)) set_status(hdr, TR_ERR_TIMEOUT, (uint32_t)tile);
      break;
    }
    Carry val = Carry(0);
    if (idx >= 0) val = (st == kFlagP) ? incl[idx] : agg[idx];
    const unsigned pm = __ballot_sync(kFull, st == kFlagP);
    if (lane == 0) sm.first[wid] = pm ? __ffs(pm) - 1 : 32;
    __syncthreads();
    int first = kThreads;  // nearest predecessor holding an inclusive prefix (block-wide)
#pragma unroll
    for (int w = 0; w < kWarps; ++w)
      if (first == kThreads && sm.first[w] < 32) first = w * 32 + sm.first[w];
    const Carry part = warp_sum_carry<Op>(tid <= first ? val : Carry(0));
    if (lane == 0) sm.red[wid] = part;
    __syncthreads();
    Carry round = Carry(0);
#pragma unroll
    for (int w = 0; w < kWarps; ++w) round = Op::cadd(round, sm.red[w]);  // fixed order
    excl = Op::cadd(excl, round);
    __syncthreads();  // sm is reused next round
    if (first < kThreads) break;
    pos -= kThreads;
  }
  if (tid == 0 && !stall) {
    incl[tile] = Op::cadd(excl, aggregate);
    st_release_u32(&ws.flags[tile], kFlagP);
  }
  return excl;
}

// The thread's kItems outputs: its running prefix on top of everything before it.
template <class Op, class C>
__device__ __forceinline__ void scan_outputs(const C* v, typename Op::Carry prefix, typename Op::T warp_off,
                                             typename Op::T excl_lane, typename Op::Out* o) {
  using T = typename Op::T;
  if constexpr (std::is_same<Op, OpF32>::value) {
    FF run = ff_add(ff_add(ff_from_double(prefix), warp_off), excl_lane);
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      float sm, e;
      two_sum(run.hi, v[i], sm, e);
      run.hi = sm;
      run.lo += e;
      o[i] = run.hi + run.lo;  // the compensated prefix, rounded once
    }
  } else {
    T run = Op::add(Op::add((T)prefix, warp_off), excl_lane);
#pragma unroll
    for (int i = 0; i < kItems; ++i) {
      run = Op::add(run, Op::lift(v[i]));
      o[i] = run;
    }
  }
}

// Thread totals of the kItems values, warp-scanned; block totals in shared memory.
template <class Op, class C>
__device__ __forceinline__ void scan_totals(const C* v, typename Op::T* s_warp, typename Op::T& warp_off,
                                            typename Op::T& excl_lane, typename Op::T& tile_tot) {
  using T = typename Op::T;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T acc = Op::zero();
#pragma unroll
  for (int i = 0; i < kItems; ++i) {
    if constexpr (std::is_same<Op, OpF32>::value) {  // TwoSum into (hi, lo)
      float sm, e;
      two_sum(acc.hi, v[i], sm, e);
      acc.hi = sm;
      acc.lo += e;
    } else {
      acc = Op::add(acc, Op::lift(v[i]));
    }
  }
  const T incl_lane = warp_incl_scan<Op>(acc, lane);
  excl_lane = Op::shfl_up(incl_lane, 1);
  if (lane == 0) excl_lane = Op::zero();
  if (lane == 31) s_warp[wid] = incl_lane;
  __syncthreads();
  warp_off = Op::zero();
  tile_tot = Op::zero();
#pragma unroll
  for (int w = 0; w < kWarps; ++w) {
    if (w < wid) warp_off = Op::add(warp_off, s_warp[w]);
    tile_tot = Op::add(tile_tot, s_warp[w]);
  }
}

template <class Out>
__device__ __forceinline__ void store_items(Out* y, int64_t base, int64_t n, bool vec, const Out* o) {
  if (vec && base + kItems <= n) {
    uint4* yv = reinterpret_cast<uint4*>(y + base);
    constexpr int kPer = 16 / (int)sizeof(Out);
#pragma unroll
    for (int j = 0; j < kItems / kPer; ++j) st_stream(yv + j, pack16(o + j * kPer));
  } else {
#pragma unroll
    for (int i = 0; i < kItems; ++i)
      if (base + i < n) y[base + i] = o[i];
  }
}

// Plain form: one tile per block, tile ids drawn in launch order, loads
// straight to registers (any alignment).
template <class In, class F, class Op>
__global__ void __launch_bounds__(kThreads) k_scan(const In* __restrict__ x, typename Op::Out* y, int64_t n, int vec_ok,
                                                   const __grid_constant__ MapParams P, WsHeader* hdr, ScanWs ws,
                                                   const typename Op::Out* carry_in, uint64_t timeout_ns,
                                                   int64_t stall_tile) {
  using S = Storage<In>;
  using C = typename S::C;
  using T = typename Op::T;
  using Carry = typename Op::Carry;
  using Out = typename Op::Out;
  constexpr int V = S::kVec;
  constexpr int kLoads = kItems / V;

  __shared__ uint32_t s_tile;
  __shared__ T s_warp[kWarps];
  __shared__ LookbackSmem<Op> s_lb;
  const int tid = threadIdx.x;
  if (tid == 0) s_tile = atomicAdd(&hdr->tile_counter, 1u);
  __syncthreads();
  const int64_t tile = s_tile;

  const auto f = make_kernel_map<F>(P);
  const int64_t base = tile * kTile + (int64_t)tid * kItems;
  C v[kItems];
  if (vec_ok && base + kItems <= n) {
    const uint4* xv = reinterpret_cast<const uint4*>(x + base);
    uint4 raw[kLoads];
#pragma unroll
    for (int j = 0; j < kLoads; ++j) raw[j] = ld_cached(xv + j);
#pragma unroll
    for (int j = 0; j < kLoads; ++j) S::unpack(raw[j], v + j * V);
    map_vec<kItems>(f, v);
  } else {
#pragma unroll
    for (int i = 0; i < kItems; ++i) v[i] = (base + i < n) ? f(S::cvt(x[base + i])) : C(0);
  }
  T warp_off, excl_lane, tile_tot;
  scan_totals<Op>(v, s_warp, warp_off, excl_lane, tile_tot);
  const Carry excl = block_lookback<Op>(tile, Op::to_carry(tile_tot), ws, hdr, timeout_ns, tile == stall_tile, s_lb);
  const Carry prefix = Op::cadd(carry_in ? Carry(*carry_in) : Carry(0), excl);
  Out o[kItems];
  scan_outputs<Op>(v, prefix, warp_off, excl_lane, o);
  store_items(y, base, n, vec_ok, o);
}

}  // namespace

size_t scan_ws_bytes(int64_t n, tr_dtype, tr_dtype) {
  const int64_t tiles = std::max<int64_t>(1, ceil_div(n, kTile));
  const int64_t flags = ceil_div(tiles * 4, 256) * 256;
  const int64_t vals = ceil_div(tiles * 8, 256) * 256;
  return (size_t)(kWsHeader + flags + 2 * vals);
}

tr_status launch_scan(const MapParams& P, const void* x, tr_dtype xt, void* y, tr_dtype yt, int64_t n, const void* carry,
                      const tr_exec* e) {
  const int64_t tiles = ceil_div(n, kTile);
  if (tiles > 0x7FFFFFFF) return fail(TR_ERR_INVALID_ARG, "too many tiles");
  const int64_t flags_b = ceil_div(tiles * 4, 256) * 256;
  const int64_t vals_b = ceil_div(tiles * 8, 256) * 256;
  const ScanWs ws{reinterpret_cast<uint32_t*>(ws_body(e)), ws_body(e) + flags_b, ws_body(e) + flags_b + vals_b};
  const uint64_t timeout_ns = (uint64_t)(e->wait_timeout_us ? e->wait_timeout_us : 1000000u) * 1000ull;
  const int vec_ok = aligned_to(x, 16) && aligned_to(y, 16);
  cudaStream_t st = stream_of(e);
  WsHeader* hdr = ws_header(e);
  const int64_t stall = e->debug_stall_tile;
  // every call starts from clear tile flags and a zero tile counter
  tr_status s = cuda_status(cudaMemsetAsync(ws.flags, 0, (size_t)tiles * 4, st), "cudaMemsetAsync(scan flags)");
  if (!s) s = cuda_status(cudaMemsetAsync(&hdr->tile_counter, 0, sizeof(uint32_t), st), "cudaMemsetAsync(counter)");
  if (s) return s;
  auto go = [&](auto op_tag) {
    using Op = decltype(op_tag);
    return [&](auto in_tag, auto map_tag) -> tr_status {
      using In = decltype(in_tag);
      using F = decltype(map_tag);
      using Out = typename Op::Out;
      k_scan<In, F, Op><<<(unsigned)tiles, kThreads, 0, st>>>(static_cast<const In*>(x), static_cast<Out*>(y), n,
                                                              vec_ok, P, hdr, ws, static_cast<const Out*>(carry),
                                                              timeout_ns, stall);
      return launch_status("k_scan");
    };
  };
  if (xt == TR_U32 && yt == TR_U32) return dispatch_u32_map(P, go(OpU32{}));
  if (xt == TR_U32 && yt == TR_U64) return dispatch_u32_map(P, go(OpU64{}));
  if (yt == TR_F32) return dispatch_float_storage(xt, P, go(OpF32{}));
  return fail(TR_ERR_UNSUPPORTED, "scan %d -> %d", xt, yt);
}

}  // namespace tr
