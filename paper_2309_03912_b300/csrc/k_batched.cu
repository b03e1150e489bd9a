// k_batched.cu -- tr_batched_*: sum / min / max of f over thousands of
// independent arrays of uneven length, each with its own map, in one
// persistent launch replayed from a CUDA graph.
//
// Plan (host, once): every array is cut into work items of at most T elements;
// items are queued in decreasing order of estimated cost (elements x map cost)
// so the long ones start first.  The device arrays of descriptors, items,
// per-item partial slots and per-array counters are owned by the plan.
//
// Kernel (device, every run): a resident grid of warps pulls items from an
// atomic queue.  A warp reduces its item with 128-bit loads and the item's map
// chosen by a warp-uniform switch (fixed-degree forms keep coefficients in
// registers), combines lanes in float-float, and either writes the array's
// result (single-item arrays) or stores an FP64 partial; the warp that
// finishes an array's last item (atomic counter after a fence) joins its
// partials in item order in FP64 and resets the counter.  Results are
// therefore independent of scheduling: bitwise deterministic.
//
// Graph: a memset of the queue head and the kernel, captured once; each run is
// one cudaGraphLaunch.  Tile size T, block size, cost balancing and the
// vectors per lane (4 or 2: registers, hence resident warps, against loads in
// flight) come from a small autotuner that times the candidates on the plan's
// own data.  The device side is in batched_kernel.cuh.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "batched_kernel.cuh"

namespace tr {

BatchedKernel batched_kernel_u4(tr_dtype xt, int threads) { return batched_kernel<4>(xt, threads); }

namespace {

BatchedKernel kernel_for(tr_dtype xt, int threads, int unroll) {
  return unroll == 2 ? batched_kernel_u2(xt, threads) : batched_kernel_u4(xt, threads);
}

// rough per-element instruction cost of a map, for ordering the queue
double map_cost(const tr_map_desc& m) {
  switch (m.kind) {
    case TR_MAP_HORNER: return 4.0 + m.deg_p;
    case TR_MAP_RATIONAL: return 12.0 + m.deg_p + m.deg_q;
    case TR_MAP_NEWTON_CBRT: return 6.0 + 16.0 * m.iters;
    default: return 4.0;
  }
}

// Autotuned launch shape: the work-item size T, the block size, whether
// items are balanced by map cost (an array's items then hold about
// T x cost(Horner 8) / cost(map) elements, so costly maps get shorter items),
// and the 16-byte vectors each lane has in flight (4 or 2).  The grid is the
// kernel's full occupancy, which the vectors per lane set through registers.
struct Config {
  int64_t tile = 32768;
  int threads = 256;
  int balance = 0;
  int unroll = 4;
};

}  // namespace

}  // namespace tr

using namespace tr;

struct tr_batch_plan {
  int64_t n_arrays = 0;
  tr_dtype xt = TR_F32;
  unsigned ops = 0;
  double* sums = nullptr;
  float* mins = nullptr;
  float* maxs = nullptr;
  std::vector<BatchArray> h_arrays;
  std::vector<tr_map_desc> maps;
  std::vector<std::vector<double>> coef_p, coef_q;
  std::vector<int64_t> lens;
  Config cfg;
  int grid = 0;
  int32_t n_items = 0;
  // device buffers owned by the plan
  BatchArray* d_arrays = nullptr;
  BatchItem* d_items = nullptr;
  BatchPartial* d_partials = nullptr;
  uint32_t* d_counters = nullptr;  // n_arrays counters + the queue head at the end
  void* d_reduce_ws = nullptr;     // workspace of the per-array baseline
  size_t reduce_ws_bytes = 0;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  cudaGraphExec_t unbatched_graph = nullptr;
  std::string desc;
};

namespace tr {
namespace {

void free_items(tr_batch_plan* p) {
  if (p->d_items) cudaFree(p->d_items);
  if (p->d_partials) cudaFree(p->d_partials);
  p->d_items = nullptr;
  p->d_partials = nullptr;
}

// Build the item list for tile size T (balanced by map cost or not) and upload
// it (with the partial slots).
tr_status build_items(tr_batch_plan* p, int64_t T, int balance) {
  std::vector<BatchItem> items;
  std::vector<double> cost;
  int32_t slot = 0;
  for (int64_t a = 0; a < p->n_arrays; ++a) {
    const int64_t L = p->lens[a];
    int64_t Ta = T;
    if (balance) {  // about T x cost(Horner 8) / cost(map), multiples of 256 (vector alignment kept)
      const double r = 12.0 / map_cost(p->maps[a]);
      Ta = std::max<int64_t>(1024, std::min<int64_t>(T, ((int64_t)(T * r) / 256) * 256));
    }
    const int64_t n_it = std::max<int64_t>(1, (L + Ta - 1) / Ta);
    p->h_arrays[a].first_slot = slot;
    p->h_arrays[a].n_items = (int32_t)n_it;
    const double mc = map_cost(p->maps[a]);
    for (int64_t k = 0; k < n_it; ++k) {
      const int64_t st = k * Ta, cnt = std::min<int64_t>(Ta, L - st);
      items.push_back(BatchItem{(int32_t)a, slot + (int32_t)k, st, std::max<int64_t>(cnt, 0)});
      cost.push_back(mc * (double)std::max<int64_t>(cnt, 1) + 200.0);
    }
    slot += (int32_t)n_it;
  }
  std::vector<size_t> order(items.size());
  for (size_t i = 0; i < order.size(); ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](size_t u, size_t v) { return cost[u] > cost[v]; });
  std::vector<BatchItem> sorted(items.size());
  for (size_t i = 0; i < order.size(); ++i) sorted[i] = items[order[i]];
  free_items(p);
  p->n_items = (int32_t)sorted.size();
  tr_status s;
  if ((s = cuda_status(cudaMalloc(&p->d_items, sorted.size() * sizeof(BatchItem)), "cudaMalloc(items)"))) return s;
  if ((s = cuda_status(cudaMalloc(&p->d_partials, std::max<size_t>(1, slot) * sizeof(BatchPartial)),
                       "cudaMalloc(partials)")))
    return s;
  if ((s = cuda_status(cudaMemcpy(p->d_items, sorted.data(), sorted.size() * sizeof(BatchItem), cudaMemcpyHostToDevice),
                       "cudaMemcpy(items)")))
    return s;
  return cuda_status(cudaMemcpy(p->d_arrays, p->h_arrays.data(), p->h_arrays.size() * sizeof(BatchArray),
                                cudaMemcpyHostToDevice),
                     "cudaMemcpy(arrays)");
}

tr_status enqueue(tr_batch_plan* p, cudaStream_t st) {
  tr_status s = cuda_status(cudaMemsetAsync(p->d_counters + p->n_arrays, 0, sizeof(uint32_t), st), "memset(queue)");
  if (s) return s;
  const BatchOut out{p->sums, p->mins, p->maxs, p->ops};
  kernel_for(p->xt, p->cfg.threads, p->cfg.unroll)<<<p->grid, p->cfg.threads, 0, st>>>(p->d_arrays, p->d_items, p->n_items, p->d_partials,
                                                                  p->d_counters, p->d_counters + p->n_arrays, out);
  return launch_status("k_batched");
}

tr_status set_config(tr_batch_plan* p, const Config& c) {
  p->cfg = c;
  const BatchedKernel k = kernel_for(p->xt, c.threads, c.unroll);
  p->grid = dev_info().sm_count * blocks_per_sm((const void*)k, c.threads);
  return build_items(p, c.tile, c.balance);
}

tr_status time_config(tr_batch_plan* p, cudaStream_t st, float* ms) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  tr_status s = enqueue(p, st);  // warm-up
  cudaEventRecord(a, st);
  for (int r = 0; r < 3 && !s; ++r) s = enqueue(p, st);
  cudaEventRecord(b, st);
  if (!s) s = cuda_status(cudaEventSynchronize(b), "cudaEventSynchronize");
  float t = 0.f;
  cudaEventElapsedTime(&t, a, b);
  *ms = t / 3.f;
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return s;
}

std::string cache_key(const tr_batch_plan* p) {
  cudaDeviceProp prop;
  cudaGetDeviceProperties(&prop, dev_info().device);
  int64_t total = 0;
  for (int64_t L : p->lens) total += L;
  std::ostringstream k;
  k << prop.name << "|xt=" << (int)p->xt << "|arrays=" << p->n_arrays
    << "|log2n=" << (int)std::log2((double)std::max<int64_t>(total, 1));
  return k.str();
}

bool cache_lookup(const std::string& key, Config* c) {
  const char* path = getenv("TR_AUTOTUNE_CACHE");
  if (!path) return false;
  std::ifstream f(path);
  std::string line;
  while (std::getline(f, line)) {
    // key, tile, threads, balance[, vectors per lane]
    const size_t t1 = line.find('\t'), t2 = line.find('\t', t1 + 1), t3 = line.find('\t', t2 + 1);
    if (t1 == std::string::npos || t2 == std::string::npos || t3 == std::string::npos) continue;
    if (line.substr(0, t1) == key) {
      const size_t t4 = line.find('\t', t3 + 1);
      c->tile = atoll(line.substr(t1 + 1, t2 - t1 - 1).c_str());
      c->threads = atoi(line.substr(t2 + 1, t3 - t2 - 1).c_str());
      c->balance = atoi(line.substr(t3 + 1, t4 == std::string::npos ? std::string::npos : t4 - t3 - 1).c_str()) != 0;
      c->unroll = t4 == std::string::npos ? 4 : atoi(line.substr(t4 + 1).c_str());
      return c->tile > 0 && (c->threads == 128 || c->threads == 256) && (c->unroll == 2 || c->unroll == 4);
    }
  }
  return false;
}

void cache_store(const std::string& key, const Config& c) {
  const char* path = getenv("TR_AUTOTUNE_CACHE");
  if (!path) return;
  std::ofstream f(path, std::ios::app);
  f << key << '\t' << c.tile << '\t' << c.threads << '\t' << c.balance << '\t' << c.unroll << '\n';
}

tr_status capture(tr_batch_plan* p, bool unbatched, cudaGraphExec_t* out);

}  // namespace
}  // namespace tr

extern "C" {

tr_status tr_batched_plan_destroy(tr_batch_plan* p) {
  if (!p) return TR_OK;
  if (p->graph) cudaGraphExecDestroy(p->graph);
  if (p->unbatched_graph) cudaGraphExecDestroy(p->unbatched_graph);
  free_items(p);
  if (p->d_arrays) cudaFree(p->d_arrays);
  if (p->d_counters) cudaFree(p->d_counters);
  if (p->d_reduce_ws) cudaFree(p->d_reduce_ws);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  delete p;
  return TR_OK;
}

tr_status tr_batched_plan_create(int64_t n_arrays, const void* const* d_xs, const int64_t* lens,
                                 const tr_map_desc* maps, tr_dtype xt, unsigned ops, double* d_sums, float* d_mins,
                                 float* d_maxs, int autotune, void* stream, tr_batch_plan** out) {
  if (!out) return fail(TR_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (xt != TR_F32 && xt != TR_F16 && xt != TR_BF16) return fail(TR_ERR_UNSUPPORTED, "batched storage dtype %d", xt);
  const size_t esz = dtype_size(xt);
  if (n_arrays <= 0 || n_arrays > (int64_t(1) << 30)) return fail(TR_ERR_INVALID_ARG, "n_arrays out of range");
  if (!d_xs || !lens || !maps) return fail(TR_ERR_INVALID_ARG, "arrays, lengths or maps are NULL");
  if (ops == 0 || (ops & ~7u)) return fail(TR_ERR_INVALID_ARG, "ops must be a non-empty mask of TR_SUM|TR_MIN|TR_MAX");
  if (((ops & TR_SUM) && !d_sums) || ((ops & TR_MIN) && !d_mins) || ((ops & TR_MAX) && !d_maxs))
    return fail(TR_ERR_INVALID_ARG, "an output selected by ops is NULL");
  if ((d_sums && !aligned_to(d_sums, 8)) || (d_mins && !aligned_to(d_mins, 4)) || (d_maxs && !aligned_to(d_maxs, 4)))
    return fail(TR_ERR_ALIGNMENT, "outputs misaligned");
  auto* p = new tr_batch_plan();
  p->n_arrays = n_arrays;
  p->xt = xt;
  p->ops = ops;
  p->sums = d_sums;
  p->mins = d_mins;
  p->maxs = d_maxs;
  p->h_arrays.resize(n_arrays);
  p->maps.resize(n_arrays);
  p->coef_p.resize(n_arrays);
  p->coef_q.resize(n_arrays);
  p->lens.assign(lens, lens + n_arrays);
  for (int64_t a = 0; a < n_arrays; ++a) {
    MapParams P;
    tr_status s = make_map_params(&maps[a], false, &P);
    if (s) {
      const std::string msg = tr_last_error();
      tr_batched_plan_destroy(p);
      return fail(s, "array %lld: %s", (long long)a, msg.c_str());
    }
    if (lens[a] < 0 || (lens[a] > 0 && !d_xs[a]) || (d_xs[a] && !aligned_to(d_xs[a], esz))) {
      tr_batched_plan_destroy(p);
      return fail(TR_ERR_INVALID_ARG, "array %lld: bad pointer or length", (long long)a);
    }
    BatchArray& A = p->h_arrays[a];
    std::memset(&A, 0, sizeof(A));
    A.x = d_xs[a];
    A.len = lens[a];
    A.kind = P.kind;
    A.deg_p = P.deg_p;
    A.deg_q = P.deg_q;
    A.iters = P.iters;
    A.aligned = aligned_to(d_xs[a], 16) ? 1 : 0;
    for (int k = 0; k <= TR_MAX_DEGREE; ++k) {
      A.cp[k] = P.fp[k];
      A.cq[k] = P.fq[k];
    }
    p->coef_p[a].assign(P.dp, P.dp + P.deg_p + 1);
    p->coef_q[a].assign(P.dq, P.dq + P.deg_q + 1);
    p->maps[a] = maps[a];
    p->maps[a].coef_p = p->coef_p[a].data();
    p->maps[a].coef_q = p->coef_q[a].data();
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  tr_status s;
  if ((s = cuda_status(cudaMalloc(&p->d_arrays, n_arrays * sizeof(BatchArray)), "cudaMalloc(arrays)")) ||
      (s = cuda_status(cudaMalloc(&p->d_counters, (n_arrays + 64) * sizeof(uint32_t)), "cudaMalloc(counters)")) ||
      (s = cuda_status(cudaMemset(p->d_counters, 0, (n_arrays + 64) * sizeof(uint32_t)), "cudaMemset(counters)")) ||
      (s = cuda_status(cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking), "cudaStreamCreate"))) {
    tr_batched_plan_destroy(p);
    return s;
  }
  // configuration: cache, autotuner, or the fixed default
  Config best;
  std::string how = "default";
  const std::string key = cache_key(p);
  if (autotune && cache_lookup(key, &best)) {
    how = "autotune cache";
  } else if (autotune) {
    float best_ms = 1e30f;
    int tried = 0;
    for (int64_t T : {8192, 16384, 32768, 65536})
      for (int th : {128, 256})
        for (int bal : {0, 1})
          for (int u : {4, 2}) {
            Config c;
            c.tile = T;
            c.threads = th;
            c.balance = bal;
            c.unroll = u;
            float ms = 0.f;
            if ((s = set_config(p, c)) || (s = time_config(p, st, &ms))) {
              tr_batched_plan_destroy(p);
              return s;
            }
            ++tried;
            if (ms < best_ms) {
              best_ms = ms;
              best = c;
            }
          }
    cache_store(key, best);
    char b[96];
    snprintf(b, sizeof b, "autotuned over %d candidates (best %.3f ms)", tried, best_ms);
    how = b;
  }
  if ((s = set_config(p, best))) {
    tr_batched_plan_destroy(p);
    return s;
  }
  if ((s = cuda_status(cudaDeviceSynchronize(), "cudaDeviceSynchronize")) || (s = capture(p, false, &p->graph))) {
    tr_batched_plan_destroy(p);
    return s;
  }
  char b[256];
  snprintf(b, sizeof b, "tile=%lld threads=%d balance=%d vectors_per_lane=%d grid=%d items=%d arrays=%lld (%s)",
           (long long)best.tile, best.threads, best.balance, best.unroll, p->grid, p->n_items, (long long)n_arrays,
           how.c_str());
  p->desc = b;
  *out = p;
  return TR_OK;
}

tr_status tr_batched_run(tr_batch_plan* p, void* stream) {
  if (!p || !p->graph) return fail(TR_ERR_INVALID_ARG, "plan is NULL");
  const tr_status s = cuda_status(cudaGraphLaunch(p->graph, static_cast<cudaStream_t>(stream)), "cudaGraphLaunch");
  if (s == TR_OK) count_launches(1);  // the graph holds one kernel (and a memset)
  return s;
}

tr_status tr_batched_run_unbatched(tr_batch_plan* p, int use_graph, void* stream) {
  if (!p) return fail(TR_ERR_INVALID_ARG, "plan is NULL");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (!p->d_reduce_ws) {
    p->reduce_ws_bytes = reduce_ws_bytes(0, p->xt);
    tr_status s = cuda_status(cudaMalloc(&p->d_reduce_ws, p->reduce_ws_bytes), "cudaMalloc(reduce workspace)");
    if (!s) s = cuda_status(cudaMemset(p->d_reduce_ws, 0, p->reduce_ws_bytes), "cudaMemset(reduce workspace)");
    if (s) return s;
  }
  if (use_graph) {
    if (!p->unbatched_graph) {
      tr_status s = capture(p, true, &p->unbatched_graph);
      if (s) return s;
    }
    const tr_status s = cuda_status(cudaGraphLaunch(p->unbatched_graph, st), "cudaGraphLaunch");
    if (s == TR_OK) count_launches((unsigned long long)p->n_arrays);  // one reduce kernel per array
    return s;
  }
  const tr_exec e{stream, p->d_reduce_ws, p->reduce_ws_bytes, 0, 0, -1};
  for (int64_t a = 0; a < p->n_arrays; ++a) {
    tr_status s = tr_reduce(&p->maps[a], p->h_arrays[a].x, p->xt, p->lens[a], p->ops, p->sums ? p->sums + a : nullptr,
                            TR_F64, p->mins ? p->mins + a : nullptr, p->maxs ? p->maxs + a : nullptr, &e);
    if (s) return s;
  }
  return TR_OK;
}

const char* tr_batched_plan_describe(const tr_batch_plan* p) { return p ? p->desc.c_str() : ""; }

}  // extern "C"

namespace tr {
namespace {

tr_status capture(tr_batch_plan* p, bool unbatched, cudaGraphExec_t* out) {
  cudaStream_t cs = p->cap_stream;
  tr_status s = cuda_status(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
  if (s) return s;
  if (unbatched) {
    const tr_exec e{cs, p->d_reduce_ws, p->reduce_ws_bytes, 0, 0, -1};
    for (int64_t a = 0; a < p->n_arrays && !s; ++a)
      s = tr_reduce(&p->maps[a], p->h_arrays[a].x, p->xt, p->lens[a], p->ops, p->sums ? p->sums + a : nullptr, TR_F64,
                    p->mins ? p->mins + a : nullptr, p->maxs ? p->maxs + a : nullptr, &e);
  } else {
    s = enqueue(p, cs);
  }
  cudaGraph_t g = nullptr;
  const tr_status s2 = cuda_status(cudaStreamEndCapture(cs, &g), "cudaStreamEndCapture");
  if (s || s2) {
    if (g) cudaGraphDestroy(g);
    return s ? s : s2;
  }
  s = cuda_status(cudaGraphInstantiate(out, g, 0), "cudaGraphInstantiate");
  cudaGraphDestroy(g);
  return s;
}

}  // namespace
}  // namespace tr
