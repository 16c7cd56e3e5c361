// Launch accounting and optional per-kernel-class timing.  Every launcher
// opens a ProfScope: it counts the kernels it enqueues and, while profiling is
// on, brackets them with a pair of CUDA events recorded on the same stream.
#include <atomic>
#include <cstring>
#include <mutex>
#include <vector>

#include "sne_internal.cuh"

namespace sne {

namespace {
std::atomic<long long> g_launches{0};
std::mutex g_mu;
bool g_prof = false;
struct Rec {
  int cls;
  int nk;
  cudaEvent_t a, b;
};
std::vector<Rec> g_recs;
std::vector<cudaEvent_t> g_pool;
constexpr int kMaxDev = 64;
std::atomic<int> g_sms[kMaxDev];

cudaEvent_t take_event() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

const char *kClassNames[K_COUNT] = {"spmm",   "gram",  "tall_gemm", "small_gemm", "sym_eig",
                                    "cholesky", "triu_inverse", "fused_sketch", "gather",
                                    "rng", "unique", "misc", "fused_sketch_tc", "gram_tc",
                                    "tall_gemm_tc", "propagate"};
}  // namespace

int sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return 148;
  int v = g_sms[dev].load(std::memory_order_relaxed);
  if (v <= 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
      v = 148;
    g_sms[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

ProfScope::ProfScope(int cls, cudaStream_t st, int nk) : cls_(cls), nk_(nk), st_(st) {
  g_launches.fetch_add(nk, std::memory_order_relaxed);
  if (!g_prof) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_prof) return;
  a_ = take_event();
  b_ = take_event();
  if (a_ && b_) cudaEventRecord(a_, st_);
}

ProfScope::~ProfScope() {
  if (!a_ || !b_) return;
  cudaEventRecord(b_, st_);
  std::lock_guard<std::mutex> lk(g_mu);
  g_recs.push_back({cls_, nk_, a_, b_});
}

}  // namespace sne

using namespace sne;

extern "C" {

long long sne_kernel_launches(void) { return g_launches.load(); }

int sne_profile_start(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (auto &r : g_recs) {
    g_pool.push_back(r.a);
    g_pool.push_back(r.b);
  }
  g_recs.clear();
  g_prof = true;
  return SNE_OK;
}

int sne_profile_stop(sne_kernel_time *out, int max_entries, int *count) {
  std::vector<Rec> recs;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_prof = false;
    recs.swap(g_recs);
  }
  double ms[K_COUNT] = {0};
  long long nl[K_COUNT] = {0}, ns[K_COUNT] = {0};
  int rc = SNE_OK;
  for (auto &r : recs) {
    if (cudaEventSynchronize(r.b) != cudaSuccess) rc = SNE_ERR_CUDA;
    float t = 0.f;
    if (cudaEventElapsedTime(&t, r.a, r.b) != cudaSuccess) rc = SNE_ERR_CUDA;
    ms[r.cls] += t;
    nl[r.cls] += r.nk;
    ns[r.cls] += 1;
  }
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &r : recs) {
      g_pool.push_back(r.a);
      g_pool.push_back(r.b);
    }
  }
  int c = 0;
  for (int k = 0; k < K_COUNT; ++k) {
    if (ns[k] == 0) continue;
    if (out && c < max_entries) {
      std::memset(&out[c], 0, sizeof(out[c]));
      std::strncpy(out[c].name, kClassNames[k], sizeof(out[c].name) - 1);
      out[c].calls = ns[k];
      out[c].launches = nl[k];
      out[c].total_ms = ms[k];
    }
    ++c;
  }
  if (count) *count = c;
  return rc;
}

}  // extern "C"
