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
#include <mutex>
#include <numeric>
#include <vector>

#include "sne_internal.cuh"

namespace {

constexpr int kMaxLanes = 16;
constexpr int kDefaultLanes = 8;
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
  std::vector<int> order;      // graphs, largest first
  std::vector<int> lane_of;    // lane of each graph
  std::vector<size_t> bytes;   // workspace of each lane
  std::vector<size_t> offset;  // byte offset of each lane's slice
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
  const int L = std::min<int>(G, lanes > 0 ? lanes : kDefaultLanes);
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
  plan->offset.assign(L, 0);
  size_t off = 0;
  for (int l = 0; l < L; ++l) {
    plan->offset[l] = off;
    off += (plan->bytes[l] + 255) & ~(size_t)255;
  }
  plan->total = off;
  return SNE_OK;
}

}  // namespace

extern "C" {

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
  // the caller's stream waits for every lane, also after an error, so that
  // nothing enqueued above outlives the call's stream order
  for (int l = 0; l < plan.lanes; ++l) {
    if (cudaEventRecord(pool->join[l], pool->stream[l]) != cudaSuccess) return SNE_ERR_CUDA;
    if (cudaStreamWaitEvent(st, pool->join[l], 0) != cudaSuccess) return SNE_ERR_CUDA;
  }
  return first_error;
}

}  // extern "C"
