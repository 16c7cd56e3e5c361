// Batched embedding of many independent graphs (Alg. 6 lines 1-5 for each).
//
// A graph of a few thousand vertices fills a small part of the GPU, so the
// graphs of a batch run side by side on a pool of streams ("lanes") forked from
// the caller's stream.  The graphs are placed largest first, each on the lane
// with the least estimated work so far (longest-processing-time order), and
// every lane owns one slice of the workspace, sized for the largest graph it
// runs.  The single-graph path never waits on the host, so a whole batch can
// be captured into a CUDA graph and replayed.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <numeric>
#include <vector>

#include "sne_internal.cuh"

using namespace sne;

namespace {

constexpr int kMaxLanes = 16;
constexpr int kDefaultLanes = 8;

// Lane counts chosen by the autotuner for lockstep batches, by (number of
// graphs, log2 of their total vertices, k, precision); lanes = 0 in
// sne_embed_batched looks here first.
struct LaneKey {
  int G, lg, k, prec;
  bool operator==(const LaneKey &o) const {
    return G == o.G && lg == o.lg && k == o.k && prec == o.prec;
  }
};
std::mutex g_lane_mu;
std::vector<std::pair<LaneKey, int>> g_lanes;
LaneKey lane_key(int32_t G, const sne_csr *graphs, const sne_params *p) {
  int64_t sum = 0;
  for (int i = 0; i < G; ++i) sum += graphs[i].n;
  int lg = 0;
  while (lg < 62 && ((int64_t)1 << (lg + 1)) <= sum) ++lg;
  return LaneKey{G, lg, p->k, p->precision};
}
int tuned_lanes(int32_t G, const sne_csr *graphs, const sne_params *p) {
  const LaneKey k = lane_key(G, graphs, p);
  std::lock_guard<std::mutex> lk(g_lane_mu);
  for (const auto &e : g_lanes)
    if (e.first == k) return e.second;
  return kDefaultLanes;
}
constexpr int kMaxDevices = 64;

struct LanePool {
  bool ready = false;
  cudaStream_t stream[kMaxLanes];
  cudaEvent_t fork;
  cudaEvent_t join[kMaxLanes];
};

std::mutex g_pool_mu;  // guards the pools and serializes the enqueue of a batch
LanePool g_pool[kMaxDevices];

// Streams and events of the current device, created on first use (held
// until the process exits).  Called with g_pool_mu held.
int lane_pool(LanePool **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SNE_ERR_CUDA;
  LanePool &pl = g_pool[dev];
  if (!pl.ready) {
    for (int l = 0; l < kMaxLanes; ++l) {
      if (cudaStreamCreateWithFlags(&pl.stream[l], cudaStreamNonBlocking) != cudaSuccess)
        return SNE_ERR_CUDA;
      if (cudaEventCreateWithFlags(&pl.join[l], cudaEventDisableTiming) != cudaSuccess)
        return SNE_ERR_CUDA;
    }
    if (cudaEventCreateWithFlags(&pl.fork, cudaEventDisableTiming) != cudaSuccess)
      return SNE_ERR_CUDA;
    pl.ready = true;
  }
  *out = &pl;
  return SNE_OK;
}

// Relative cost of one embedding: the SpMMs and small-dimension products of
// Alg. 5 and the reconstruction of Eq. 4.
double graph_cost(const sne_csr &g, const sne_params &p) {
  const double K = (double)p.k + p.s_eig;
  const double n = (double)g.n, nnz = (double)g.nnz;
  const double z = std::min<double>(n, (double)p.zeta);
  return (2.0 * p.q + 2.0) * nnz * K + (p.q + 2.0) * 4.0 * n * K * K + n * p.h * z * p.k;
}

struct Plan {
  int lanes = 0;
  bool lockstep = false;       // tensor-core sketch: one launch for the whole batch
  std::vector<int> order;      // graphs, largest first
  std::vector<int> lane_of;    // lane of each graph
  std::vector<size_t> bytes;   // workspace of each lane (lockstep: of each graph)
  std::vector<size_t> offset;  // byte offset of each lane's (graph's) slice
  size_t total = 0;
};

int make_plan(int32_t G, const sne_csr *graphs, const sne_params *p, int32_t lanes, Plan *plan) {
  if (G <= 0 || !graphs || !p || lanes < 0 || lanes > kMaxLanes) return SNE_ERR_ARG;
  std::vector<size_t> wsb(G);
  std::vector<double> cost(G);
  for (int i = 0; i < G; ++i) {
    const sne_csr &g = graphs[i];
    if (g.n <= 0 || g.nnz < 0 || !g.row_ptr || (g.nnz > 0 && !g.col_idx)) return SNE_ERR_ARG;
    if (g.nnz == 0) return SNE_ERR_GRAPH;  // no edges: vol(G) = 0, Eq. 1 undefined
    const int rc = sne_workspace_bytes(g.n, g.nnz, p, SNE_WS_EMBED, &wsb[i]);
    if (rc) return rc;
    cost[i] = graph_cost(g, *p);
  }
  const int L = std::min<int>(G, lanes > 0 ? lanes : tuned_lanes(G, graphs, p));
  plan->lanes = L;
  plan->order.resize(G);
  std::iota(plan->order.begin(), plan->order.end(), 0);
  std::stable_sort(plan->order.begin(), plan->order.end(),
                   [&](int a, int b) { return cost[a] > cost[b]; });
  plan->lane_of.assign(G, 0);
  plan->bytes.assign(L, 0);
  std::vector<double> load(L, 0.0);
  for (int i : plan->order) {
    const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    plan->lane_of[i] = l;
    load[l] += cost[i];
    plan->bytes[l] = std::max(plan->bytes[l], wsb[i]);
  }
  TcShape shp;
  plan->lockstep = G > 1 && embed_tc_shape(&graphs[0], p, &shp);
  if (!plan->lockstep) {
    plan->offset.assign(L, 0);
    size_t off = 0;
    for (int l = 0; l < L; ++l) {
      plan->offset[l] = off;
      off += (plan->bytes[l] + 255) & ~(size_t)255;
    }
    plan->total = off;
    return SNE_OK;
  }
  // every graph keeps its own slice from its first half to its second; the
  // slices start on operand-row boundaries of the one arena the batched
  // sketch reads
  const size_t rb = tc_row_bytes(p);
  const size_t al = std::lcm((size_t)256, rb);
  plan->bytes = wsb;
  plan->offset.assign(G, 0);
  size_t off = 0;
  for (int i = 0; i < G; ++i) {
    plan->offset[i] = off;
    off += (wsb[i] + al - 1) / al * al;
  }
  plan->total = off;
  return SNE_OK;
}

// The lockstep form: the first halves of all embeddings on the lanes, one
// persistent tensor-core launch for the sketches of all of them (grouped by
// z, which is min(n, zeta)), the second halves on the lanes.
int run_lockstep(const Plan &plan, int32_t G, const sne_csr *graphs, const sne_params *p, void *ws,
                 float *const *E, double *const *sigma, int32_t *status, LanePool *pool,
                 cudaStream_t st) {
  std::vector<TcSketchJobDesc> jobs((size_t)2 * G);
  std::vector<TcShape> shape(G);
  for (int i = 0; i < G; ++i)
    if (!embed_tc_shape(&graphs[i], p, &shape[i])) return SNE_ERR_ARG;
  int first_error = SNE_OK;
  for (int i : plan.order) {
    const int l = plan.lane_of[i];
    char *slice = static_cast<char *>(ws) + plan.offset[i];
    const int r = embed_phase(&graphs[i], p, slice, plan.bytes[i], E[i], sigma[i], 1,
                              &jobs[(size_t)2 * i], pool->stream[l]);
    if (r != SNE_OK) {
      first_error = r;
      break;
    }
  }
  for (int l = 0; l < plan.lanes; ++l) {
    if (cudaEventRecord(pool->join[l], pool->stream[l]) != cudaSuccess) return SNE_ERR_CUDA;
    if (cudaStreamWaitEvent(st, pool->join[l], 0) != cudaSuccess) return SNE_ERR_CUDA;
  }
  if (first_error) return first_error;
  std::vector<int> zs;
  for (int i = 0; i < G; ++i)
    if (std::find(zs.begin(), zs.end(), shape[i].z) == zs.end()) zs.push_back(shape[i].z);
  for (int z : zs) {
    std::vector<TcSketchJobDesc> grp;
    int64_t rows = 0;
    for (int i = 0; i < G; ++i)
      if (shape[i].z == z) {
        grp.push_back(jobs[(size_t)2 * i]);
        grp.push_back(jobs[(size_t)2 * i + 1]);
        rows += jobs[(size_t)2 * i].nrows_max + jobs[(size_t)2 * i + 1].nrows_max;
      }
    const TcShape &s0 = shape[0];
    const TcTune tune = tc_tune_lookup(s0.kpad, s0.split, s0.fp16, z, rows);
    if (launch_fused_sketch_tc_jobs(s0.fp16, s0.split, ws, plan.total, s0.kpad, z,
                                    1.0f / sqrtf((float)z), s0.f, grp.data(), (int)grp.size(),
                                    tune, grp[0].ctrl, st) != cudaSuccess)
      return SNE_ERR_CUDA;
  }
  if (cudaEventRecord(pool->fork, st) != cudaSuccess) return SNE_ERR_CUDA;
  for (int l = 0; l < plan.lanes; ++l)
    if (cudaStreamWaitEvent(pool->stream[l], pool->fork, 0) != cudaSuccess) return SNE_ERR_CUDA;
  for (int i : plan.order) {
    const int l = plan.lane_of[i];
    char *slice = static_cast<char *>(ws) + plan.offset[i];
    const int r = embed_phase(&graphs[i], p, slice, plan.bytes[i], E[i], sigma[i], 2, nullptr,
                              pool->stream[l]);
    if (r != SNE_OK) {
      first_error = r;
      break;
    }
    if (status && cudaMemcpyAsync(status + i, slice, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                  pool->stream[l]) != cudaSuccess) {
      first_error = SNE_ERR_CUDA;
      break;
    }
  }
  return first_error;
}

// One timed launch of the batch's sketches with launch shape t (ms).
float time_sketch(const std::vector<TcSketchJobDesc> &jobs, const TcShape &s0, void *arena,
                  size_t arena_bytes, const TcTune &t, cudaStream_t st, int reps) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return -1.f;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return -1.f;
  }
  float best = -1.f;
  for (int r = 0; r < reps; ++r) {
    cudaEventRecord(e0, st);
    const cudaError_t e = launch_fused_sketch_tc_jobs(
        s0.fp16, s0.split, arena, arena_bytes, s0.kpad, s0.z, 1.0f / sqrtf((float)s0.z), s0.f,
        jobs.data(), (int)jobs.size(), t, jobs[0].ctrl, st);
    cudaEventRecord(e1, st);
    if (e != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
      best = -1.f;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (best < 0.f || ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

}  // namespace

extern "C" {

int sne_autotune_sketch(int32_t G, const sne_csr *graphs, const sne_params *p, int32_t lanes,
                        void *ws, size_t ws_bytes, float *const *E, double *const *sigma,
                        sne_tune_result *out, sne_stream_t stream) {
  if (G <= 0 || !graphs || !p || !out) return SNE_ERR_ARG;
  TcShape s0;
  if (!embed_tc_shape(&graphs[0], p, &s0)) return SNE_ERR_ARG;  // FP32 path: nothing to tune
  for (int i = 1; i < G; ++i) {
    TcShape si;
    if (!embed_tc_shape(&graphs[i], p, &si) || si.z != s0.z) return SNE_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<TcSketchJobDesc> jobs((size_t)2 * G);
  // the sketch operands of every graph, as the embedding prepares them (the
  // outputs E and sigma are not written by the first half)
  size_t arena_bytes = ws_bytes;
  int64_t rows = 0;
  if (G == 1) {
    size_t need = 0;
    int rc = sne_workspace_bytes(graphs[0].n, graphs[0].nnz, p, SNE_WS_EMBED, &need);
    if (rc) return rc;
    if (!ws || ((uintptr_t)ws % 256) != 0 || ws_bytes < need) return SNE_ERR_WORKSPACE;
    float dummyE = 0.f;
    double dummyS = 0.0;
    rc = embed_phase(&graphs[0], p, ws, ws_bytes, &dummyE, &dummyS, 1, jobs.data(), st);
    if (rc) return rc;
    arena_bytes = need;
    rows = graphs[0].n;
  } else {
    Plan plan;
    int rc = make_plan(G, graphs, p, lanes, &plan);
    if (rc) return rc;
    if (!plan.lockstep) return SNE_ERR_ARG;
    if (!ws || ((uintptr_t)ws % 256) != 0 || ws_bytes < plan.total) return SNE_ERR_WORKSPACE;
    float dummyE = 0.f;
    double dummyS = 0.0;
    for (int i = 0; i < G; ++i) {
      char *slice = static_cast<char *>(ws) + plan.offset[i];
      rc = embed_phase(&graphs[i], p, slice, plan.bytes[i], &dummyE, &dummyS, 1, &jobs[(size_t)2 * i],
                       st);
      if (rc) return rc;
      rows += jobs[(size_t)2 * i].nrows_max + jobs[(size_t)2 * i + 1].nrows_max;
    }
    arena_bytes = plan.total;
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return SNE_ERR_CUDA;
  // candidates: column tile 256 or 128, every stage count that fits from 2,
  // Z-core column split aiming at 1, 2 or 4 items per SM
  std::vector<TcTune> cand;
  for (int tn : {256, 128}) {
    const int smax = tc_max_stages(s0.kpad, s0.split, tn);
    for (int stg = 2; stg <= smax; ++stg)
      for (int sm : {1, 2, 4}) {
        TcTune t;
        t.tn = tn;
        t.stages = stg;
        t.split_mult = sm;
        cand.push_back(t);
      }
  }
  const TcTune dflt;
  const float dms = time_sketch(jobs, s0, ws, arena_bytes, dflt, st, 3);
  if (dms < 0.f) return SNE_ERR_CUDA;
  TcTune best = dflt;
  float bms = dms;
  for (const TcTune &t : cand) {
    const float ms = time_sketch(jobs, s0, ws, arena_bytes, t, st, 3);
    if (ms < 0.f) return SNE_ERR_CUDA;
    if (ms < bms) {
      bms = ms;
      best = t;
    }
  }
  tc_tune_store(s0.kpad, s0.split, s0.fp16, s0.z, rows, best);
  // a batch: the number of stream lanes, timed over whole lockstep batches
  // (the workspace of a lockstep batch does not depend on it)
  out->lanes = 0;
  out->batch_ms = 0.f;
  if (G > 1 && lanes <= 0) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return SNE_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
      cudaEventDestroy(e0);
      return SNE_ERR_CUDA;
    }
    if (E && sigma) {
      int bestL = 0;
      float bestB = -1.f;
      for (int L : {4, 8, 12, 16}) {
        if (L > G) continue;
        float tb = -1.f;
        for (int r = 0; r < 2; ++r) {
          cudaEventRecord(e0, st);
          const int rc = sne_embed_batched(G, graphs, p, L, ws, arena_bytes, E, sigma, nullptr,
                                           stream);
          cudaEventRecord(e1, st);
          if (rc != SNE_OK || cudaEventSynchronize(e1) != cudaSuccess) {
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            return rc != SNE_OK ? rc : SNE_ERR_CUDA;
          }
          float ms = 0.f;
          cudaEventElapsedTime(&ms, e0, e1);
          if (tb < 0.f || ms < tb) tb = ms;
        }
        if (bestB < 0.f || tb < bestB) {
          bestB = tb;
          bestL = L;
        }
      }
      if (bestL > 0) {
        const LaneKey key = lane_key(G, graphs, p);
        std::lock_guard<std::mutex> lk(g_lane_mu);
        bool found = false;
        for (auto &e : g_lanes)
          if (e.first == key) {
            e.second = bestL;
            found = true;
          }
        if (!found) g_lanes.emplace_back(key, bestL);
        out->lanes = bestL;
        out->batch_ms = bestB;
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
  }
  out->tn = best.tn;
  out->stages = best.stages > 0 ? best.stages : tc_max_stages(s0.kpad, s0.split, best.tn);
  out->split_mult = best.split_mult;
  out->candidates = (int32_t)cand.size() + 1;
  out->best_ms = bms;
  out->default_ms = dms;
  return SNE_OK;
}


int sne_embed_batched_workspace_bytes(int32_t G, const sne_csr *graphs, const sne_params *p,
                                      int32_t lanes, size_t *bytes) {
  if (!bytes) return SNE_ERR_ARG;
  Plan plan;
  const int rc = make_plan(G, graphs, p, lanes, &plan);
  if (rc) return rc;
  *bytes = plan.total;
  return SNE_OK;
}

int sne_embed_batched(int32_t G, const sne_csr *graphs, const sne_params *p, int32_t lanes,
                      void *ws, size_t ws_bytes, float *const *E, double *const *sigma,
                      int32_t *status, sne_stream_t stream) {
  Plan plan;
  int rc = make_plan(G, graphs, p, lanes, &plan);
  if (rc) return rc;
  if (!E || !sigma) return SNE_ERR_ARG;
  for (int i = 0; i < G; ++i)
    if (!E[i] || !sigma[i]) return SNE_ERR_ARG;
  if (!ws || ((uintptr_t)ws % 256) != 0 || ws_bytes < plan.total) return SNE_ERR_WORKSPACE;
  std::lock_guard<std::mutex> lk(g_pool_mu);
  LanePool *pool = nullptr;
  rc = lane_pool(&pool);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaEventRecord(pool->fork, st) != cudaSuccess) return SNE_ERR_CUDA;
  for (int l = 0; l < plan.lanes; ++l)
    if (cudaStreamWaitEvent(pool->stream[l], pool->fork, 0) != cudaSuccess) return SNE_ERR_CUDA;
  int first_error = SNE_OK;
  if (plan.lockstep) {
    first_error = run_lockstep(plan, G, graphs, p, ws, E, sigma, status, pool, st);
  } else {
  for (int i : plan.order) {
    const int l = plan.lane_of[i];
    char *slice = static_cast<char *>(ws) + plan.offset[l];
    const int r = sne_embed(&graphs[i], p, slice, plan.bytes[l], E[i], sigma[i],
                            (sne_stream_t)pool->stream[l]);
    if (r != SNE_OK) {
      first_error = r;
      break;
    }
    if (status && cudaMemcpyAsync(status + i, slice, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                  pool->stream[l]) != cudaSuccess) {
      first_error = SNE_ERR_CUDA;
      break;
    }
  }
  }
  // the caller's stream waits for every lane, also after an error, so that
  // nothing enqueued above outlives the call's stream order
  for (int l = 0; l < plan.lanes; ++l) {
    if (cudaEventRecord(pool->join[l], pool->stream[l]) != cudaSuccess) return SNE_ERR_CUDA;
    if (cudaStreamWaitEvent(st, pool->join[l], 0) != cudaSuccess) return SNE_ERR_CUDA;
  }
  return first_error;
}

}  // extern "C"
