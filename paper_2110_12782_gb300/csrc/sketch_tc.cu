// Mixed-precision fused reconstruct + f + sparse-sign sketch (Eq. 4 and the
// Z core of Alg. 4) on the fifth-generation tensor cores of sm_103a.
//
// The entries are evaluated in the centred form of center.cu,
//   x_ie - c0 = rowf_i colf_e <A_i, B_e> + rho_i + mask_i kappa_e,
// where A_i = L~_i / rowf_i and B_e = B~_e / colf_e are the centred factors
// scaled by powers of two into [-1, 1] and stored in BF16 or FP16.  With
// SPLIT each operand is a pair hi + lo (lo = the rounding error of hi, in the
// same type) and the accumulator takes A_hi B_hi + A_lo B_hi + A_hi B_lo, so
// the product keeps about twice the operand precision (FP16 pairs: 22 bits);
// without SPLIT one product A_hi B_hi.  Accumulation is FP32 in TMEM.
//
// One CTA owns a tile of 128 rows and walks over all evaluated columns in
// tiles of 256:
//   warp 0   TMA producer: the 128 x k A tile (hi, and lo) once, then
//            256 x 64 B k-blocks (hi, then lo) through a ring of
//            shared-memory stages (128-byte swizzle);
//   warp 1   allocates 512 TMEM columns (two 128 x 256 FP32 accumulators)
//            and issues tcgen05.mma (M 128, N 256, K 16) from one thread;
//   warps 2.. epilogue (kSketchEpiWarps of them): tcgen05.ld of the
//            accumulator rows, r = x - c0, f(r), sign, and the z-column
//            segmented sums in registers, then the Y (or Y') row segment is
//            stored.  Warp w reads TMEM lane quarter w % 4 and 256 /
//            (kSketchEpiWarps / 4) of the 256 columns.
// Double-buffered accumulators let the epilogue of tile j overlap the MMAs
// of tile j+1.  When the rows are few (the Z core: v_O rows, thousands of
// columns) blockIdx.y splits a row tile's column tiles over several CTAs.
// Every mbarrier wait is bounded (about 2 s of %globaltimer); on timeout the
// CTA records SNE_ERR_TIMEOUT, stops issuing work, waits for its in-flight
// MMAs and copies, frees TMEM and returns.
#include <cuda.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

#include "sne_internal.cuh"
#include "tc_ptx.cuh"

namespace sne {

// PTX helpers: tc_ptx.cuh

// One launch works through the (row tile, column split) items of up to
// kMaxTcJobs jobs (a job: one sketch of one graph, Y or the Z core).  Every
// operand lives in one arena (the caller's workspace) seen through two tensor
// maps of rows of kpad half values: job operands are given as arena rows.
struct TcJob {
  int64_t a_row, a_lo_row;  // arena rows of A (hi, lo): row i of the job is a_row + i
  int64_t b_row, b_lo_row;  // arena rows of B (hi, lo), zero padded to whole column tiles
  int64_t nrows_max;        // rows of A; nrows_dev (if set) holds the rows actually used
  const int32_t *nrows_dev;
  const float *rowf;
  const float2 *rowdat;
  const float4 *coldat;     // readable (zero padded) up to a multiple of 256 entries
  float *out;
  int64_t ldo;
  Ctrl *ctrl;               // status word of the job's graph
  int32_t ncols_eval, cols_out, splits, item_begin;  // items: row tiles x splits
};
constexpr int kMaxTcJobs = 160;

struct TcJobs {
  int32_t njobs, total_items;
  TcJob job[kMaxTcJobs];
};

// A CTA that stops early leaves items of any job undone: every job's status
// word records the timeout.
__device__ __forceinline__ void tc_abort_all(const TcJobs &P) {
  for (int q = 0; q < P.njobs; ++q) record_error(P.job[q].ctrl, SNE_ERR_TIMEOUT, W_TC);
}

// The work items of a CTA (w = blockIdx.x + i gridDim.x) in job order; all
// three roles walk the same sequence and skip the same items.
struct TcItem {
  const TcJob *J;
  int64_t row0, nrows;
  int s, S, ntiles;
};
template <int TN>
__device__ __forceinline__ bool tc_item(const TcJobs &P, int w, int &q, TcItem &it) {
  while (q + 1 < P.njobs && w >= P.job[q + 1].item_begin) ++q;
  const TcJob &J = P.job[q];
  const int local = w - J.item_begin;
  it.J = &J;
  it.S = J.splits;
  it.s = local % J.splits;
  it.row0 = (int64_t)(local / J.splits) * tc::BM;
  it.nrows = J.nrows_dev ? (int64_t)(*J.nrows_dev) : J.nrows_max;
  it.ntiles = (J.ncols_eval + TN - 1) / TN;
  return it.row0 < it.nrows;
}

template <int F, int Z, bool SPLIT, int TN>
__global__ void __launch_bounds__(tc::kThreadsSketch, 1) fused_sketch_tc_kernel(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
    const __grid_constant__ TcJobs P, int kblocks, int stages, float out_scale, uint32_t idesc,
    Ctrl *ctrl, int stall, uint64_t wait_ns) {
  using namespace tc;
  constexpr int NPART = SPLIT ? 2 : 1;
  constexpr int kStageBytes = TN * BK * 2;
  constexpr int kAlloc = 2 * TN;  // two accumulators of TN columns (a power of two >= 32)
  constexpr int CPW = TN / (kSketchEpiWarps / 4);  // columns per epilogue warp and tile
  static_assert(kSketchEpiWarps % 4 == 0 && CPW % 32 == 0, "epilogue warp split");
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char *sA = smem;                                     // hi k-blocks, then lo
  unsigned char *sB = sA + (size_t)NPART * kblocks * kABlockBytes;
  uint64_t *bars = reinterpret_cast<uint64_t *>(sB + (size_t)stages * kStageBytes);
  uint64_t *a_full = bars;
  uint64_t *a_empty = bars + 1;
  uint64_t *full = bars + 2;
  uint64_t *empty = full + stages;
  uint64_t *tfull = empty + stages;   // 2
  uint64_t *tempty = tfull + 2;       // 2
  uint64_t *done = tempty + 2;        // 1
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
  int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int steps = kblocks * NPART;  // B stages per column tile
  // the N = TN / 2 form of the instruction descriptor, for a tile at most half full
  const uint32_t idesc_half =
      (idesc & ~(0x3fu << 17)) | ((uint32_t)(TN / 2 >> 3) << 17);

  if (threadIdx.x == 0) {
    mbar_init(a_full, 1);
    mbar_init(a_empty, 1);
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 32 * kSketchEpiWarps);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kAlloc));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int *abortv = abort_flag;

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      int it = 0, q = 0, ai = 0;
      int last_it = -1;  // the ring index of the last copy issued
      bool ok = true;
      for (int w = blockIdx.x; w < P.total_items && ok; w += gridDim.x) {
        TcItem I;
        if (!tc_item<TN>(P, w, q, I)) continue;
        // A: once the MMAs of the previous item have read it
        if (!mbar_wait(a_empty, (uint32_t)(ai & 1) ^ 1u, abortv, ctrl, wait_ns)) {
          ok = false;
          break;
        }
        mbar_expect_tx(a_full, (uint32_t)(NPART * kblocks * kABlockBytes));
        for (int kb = 0; kb < kblocks; ++kb) {
          tma_load_2d(sA + (size_t)kb * kABlockBytes, &tmA, a_full, kb * BK,
                      (int)(I.J->a_row + I.row0));
          if (SPLIT)
            tma_load_2d(sA + (size_t)(kblocks + kb) * kABlockBytes, &tmA, a_full, kb * BK,
                        (int)(I.J->a_lo_row + I.row0));
        }
        ++ai;
        for (int j = I.s; j < I.ntiles && ok; j += I.S) {
          for (int qq = 0; qq < steps; ++qq, ++it) {
            const int kb = qq / NPART, part = qq % NPART;
            const int s = it % stages;
            const uint32_t ph = (uint32_t)((it / stages) & 1);
            if (!mbar_wait(&empty[s], ph ^ 1u, abortv, ctrl, wait_ns)) {
              ok = false;
              break;
            }
            // fault injection (tests only): the first stage is never loaded,
            // so the MMA warp's wait on it runs out
            if (stall && it == 0) continue;
            mbar_expect_tx(&full[s], (uint32_t)kStageBytes);
            tma_load_2d(sB + (size_t)s * kStageBytes, &tmB, &full[s], kb * BK,
                        (int)((part ? I.J->b_lo_row : I.J->b_row) + (int64_t)j * TN));
            last_it = it;
          }
        }
      }
      if (!ok) {
        tc_abort_all(P);
        // let the copies already issued land before the CTA exits (the last
        // A tile, and the last `stages` B stages: the others completed
        // before their stage was reused)
        if (ai > 0) mbar_drain(a_full, (uint32_t)((ai - 1) & 1), wait_ns);
        for (int qq = (last_it - stages + 1 > 0 ? last_it - stages + 1 : 0); qq <= last_it; ++qq) {
          if (stall && qq == 0) continue;
          mbar_drain(&full[qq % stages], (uint32_t)((qq / stages) & 1), wait_ns);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      int it = 0, q = 0, mi = 0;
      int jj = 0;  // tile count (accumulator buffer and phase)
      bool ok = true;
      for (int w = blockIdx.x; w < P.total_items && ok; w += gridDim.x) {
        TcItem I;
        if (!tc_item<TN>(P, w, q, I)) continue;
        if (!mbar_wait(a_full, (uint32_t)(mi & 1), abortv, ctrl, wait_ns)) {
          ok = false;
          break;
        }
        fence_after();
        for (int j = I.s; j < I.ntiles && ok; j += I.S, ++jj) {
          const int buf = jj & 1;
          const uint32_t use = (uint32_t)(jj >> 1);
          if (!mbar_wait(&tempty[buf], (use & 1u) ^ 1u, abortv, ctrl, wait_ns)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t dt = tmem + (uint32_t)(buf * TN);
          // a last column tile at most half full runs at N = TN / 2: the
          // columns past it are neither multiplied nor read by the epilogue
          const uint32_t id = (I.J->ncols_eval - j * TN <= TN / 2) ? idesc_half : idesc;
          for (int qq = 0; qq < steps; ++qq, ++it) {
            const int kb = qq / NPART, part = qq % NPART;
            const int s = it % stages;
            if (!mbar_wait(&full[s], (uint32_t)((it / stages) & 1), abortv, ctrl, wait_ns)) {
              ok = false;
              break;
            }
            fence_after();
            const uint32_t ahi = smem_u32(sA + (size_t)kb * kABlockBytes);
            const uint32_t b0 = smem_u32(sB + (size_t)s * kStageBytes);
            if (part == 0) {
              // A_hi B_hi (the first product of the tile starts the accumulator)
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk)
                mma_f16(dt, sdesc(ahi + kk * 32), sdesc(b0 + kk * 32), id, (kb | kk) ? 1u : 0u);
              if (SPLIT) {
                const uint32_t alo = smem_u32(sA + (size_t)(kblocks + kb) * kABlockBytes);
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)
                  mma_f16(dt, sdesc(alo + kk * 32), sdesc(b0 + kk * 32), id, 1u);
              }
            } else {
              // A_hi B_lo
#pragma unroll
              for (int kk = 0; kk < BK / 16; ++kk)
                mma_f16(dt, sdesc(ahi + kk * 32), sdesc(b0 + kk * 32), id, 1u);
            }
            mma_commit(&empty[s]);
          }
          if (!ok) break;
          mma_commit(&tfull[buf]);
        }
        if (!ok) break;
        mma_commit(a_empty);  // the next A may land once these products are done
        ++mi;
      }
      if (!ok) tc_abort_all(P);
      // wait for every MMA issued by this thread before TMEM is released
      mma_commit(done);
      mbar_drain(done, 0, wait_ns);
    }
  } else {
    // ---------------- epilogue warps: warp w reads TMEM lane quarter w % 4
    // (rows 32(w%4) .. +32) and column slice (w - 2) / 4 of the TN columns
    const int ew = warp & 3;
    const int quarter = (warp - 2) >> 2;
    constexpr int G = 32 / Z;  // output columns per 32-column chunk
    int q = 0, jj = 0;
    bool ok = true;
    for (int w = blockIdx.x; w < P.total_items && ok; w += gridDim.x) {
      TcItem I;
      if (!tc_item<TN>(P, w, q, I)) continue;
      const TcJob &J = *I.J;
      const int64_t row = I.row0 + 32 * ew + lane;
      const bool row_ok = row < I.nrows;
      const float rf = row_ok ? J.rowf[row] : 0.0f;
      const float2 rd = row_ok ? J.rowdat[row] : make_float2(0.0f, 0.0f);
      for (int j = I.s; j < I.ntiles; j += I.S, ++jj) {
        const int buf = jj & 1;
        const uint32_t use = (uint32_t)(jj >> 1);
        if (!mbar_wait(&tfull[buf], use & 1u, abortv, ctrl, wait_ns)) {
          ok = false;
          break;
        }
        fence_after();
        // a tile at most half full (the N = TN / 2 product) is split over the
        // warps of a lane quarter in half as many columns each
        const int cpw = (J.ncols_eval - j * TN <= TN / 2 && CPW >= 64) ? CPW / 2 : CPW;
        const int nch = cpw / 32;
        const int ebase = j * TN + quarter * cpw;
        const uint32_t taddr =
            tmem + ((uint32_t)(32 * ew) << 16) + (uint32_t)(buf * TN + quarter * cpw);
        // the warp's columns in chunks of 32; the accumulator goes back to
        // the MMA warp once the last chunk is in registers
#pragma unroll 1
        for (int c = 0; c < nch; ++c) {
          if (ebase + 32 * c >= J.ncols_eval) {
            // past the evaluated columns (a partial last tile): nothing to read
            if (c == nch - 1) {
              fence_before();
              mbar_arrive(&tempty[buf]);
            }
            continue;
          }
          float vc[32];
          tmem_ld32_nw(taddr + 32 * c, vc);
          tmem_wait_ld();
          if (c == nch - 1) {
            fence_before();
            mbar_arrive(&tempty[buf]);
          }
          // the chunk's column data, lane t holding column t, broadcast by
          // shuffles (32 uniform loads per chunk, hoisted by the compiler to
          // the top of the loop, would spill)
          const float4 cdl = __ldg(J.coldat + ebase + c * 32 + lane);
          float acc[G];
#pragma unroll
          for (int g = 0; g < G; ++g) acc[g] = 0.0f;
#pragma unroll
          for (int t = 0; t < 32; ++t) {
            const float colf = __shfl_sync(0xffffffffu, cdl.x, t);
            const float kappa = __shfl_sync(0xffffffffu, cdl.y, t);
            const float sgn = __shfl_sync(0xffffffffu, cdl.z, t);
            const float r = fmaf(vc[t], rf * colf, fmaf(rd.y, kappa, rd.x));
            acc[t / Z] = fmaf(sgn, tc::fr<F>(r), acc[t / Z]);
          }
          // G consecutive outputs of this row: columns (ebase + 32 c) / Z ..
          const int oc0 = (ebase + 32 * c) / Z;
          if (row_ok && oc0 < J.cols_out) {
            float *o = J.out + row * J.ldo + oc0;
            if (G % 4 == 0 && oc0 + G <= J.cols_out &&
                ((reinterpret_cast<uintptr_t>(o) & 15) == 0)) {
#pragma unroll
              for (int g = 0; g < G; g += 4)
                *reinterpret_cast<float4 *>(o + g) =
                    make_float4(out_scale * acc[g], out_scale * acc[g + 1],
                                out_scale * acc[g + 2], out_scale * acc[g + 3]);
            } else {
#pragma unroll
              for (int g = 0; g < G; ++g)
                if (oc0 + g < J.cols_out) o[g] = out_scale * acc[g];
            }
          }
        }
      }
    }
  }
  if (warp >= 2 && lane == 0 && *abortv) tc_abort_all(P);
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kAlloc));
}

// ---------------------------------------------------------------------------
// Tensor maps (driver entry point looked up through the runtime)
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

static bool make_map(CUtensorMap *tm, bool fp16, const void *ptr, int64_t rows, int kpad,
                     int box_rows) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  cuuint64_t gdim[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)kpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)tc::BK, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(tm, fp16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                   const_cast<void *>(ptr), gdim, gstride, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// Shared memory of a launch with column tiles of tn: the A tile (hi, and lo)
// and a ring of `stages` B stages (at most the requested number, at least 2).
static size_t fused_tc_smem_bytes(int kpad, bool split, int tn, int want_stages, int *stages_out) {
  const int kblocks = kpad / tc::BK;
  const size_t abytes = (size_t)(split ? 2 : 1) * kblocks * tc::kABlockBytes;
  const size_t stage = (size_t)tn * tc::BK * 2;
  // 1 KB alignment slack and 256 bytes of barriers next to A and the B ring
  const size_t budget = 227 * 1024 - 1024 - 256;
  int stages = want_stages > 0 ? want_stages : 8;
  while (stages > 2 && abytes + (size_t)stages * stage > budget) --stages;
  if (stages_out) *stages_out = stages;
  return 1024 + abytes + (size_t)stages * stage + 256;
}

// Tuned launch shapes, by key (process-wide; written by the autotuner).
namespace {
struct TuneKey {
  int kpad, split, fp16, z, lg;
  bool operator==(const TuneKey &o) const {
    return kpad == o.kpad && split == o.split && fp16 == o.fp16 && z == o.z && lg == o.lg;
  }
};
std::mutex g_tune_mu;
std::vector<std::pair<TuneKey, TcTune>> g_tune;
int lg_rows(int64_t rows) {
  int lg = 0;
  while (lg < 62 && ((int64_t)1 << (lg + 1)) <= rows) ++lg;
  return lg;
}
int env_int(const char *name, int dflt) {
  const char *v = getenv(name);
  return v && *v ? atoi(v) : dflt;
}
}  // namespace

TcTune tc_tune_lookup(int kpad, bool split, bool fp16, int z, int64_t rows) {
  TcTune t;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    const TuneKey k{kpad, split, fp16, z, lg_rows(rows)};
    for (const auto &e : g_tune)
      if (e.first == k) t = e.second;
  }
  t.tn = env_int("SNE_TC_TN", t.tn);
  t.stages = env_int("SNE_TC_STAGES", t.stages);
  t.split_mult = env_int("SNE_TC_SPLIT", t.split_mult);
  return t;
}

void tc_tune_store(int kpad, bool split, bool fp16, int z, int64_t rows, const TcTune &t) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  const TuneKey k{kpad, split, fp16, z, lg_rows(rows)};
  for (auto &e : g_tune)
    if (e.first == k) {
      e.second = t;
      return;
    }
  g_tune.emplace_back(k, t);
}

int tc_max_stages(int kpad, bool split, int tn) {
  int s = 0;
  fused_tc_smem_bytes(kpad, split, tn, 0, &s);
  return s;
}

template <int F, int Z, bool SPLIT, int TN>
static cudaError_t launch_tc_kernel(const CUtensorMap &tmA, const CUtensorMap &tmB,
                                    const TcJobs &P, int grid, int kblocks, int stages,
                                    size_t smem, float out_scale, uint32_t idesc, Ctrl *ctrl,
                                    int stall, uint64_t wait_ns, cudaStream_t st) {
  auto kern = fused_sketch_tc_kernel<F, Z, SPLIT, TN>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, tc::kThreadsSketch, smem, st>>>(tmA, tmB, P, kblocks, stages, out_scale, idesc, ctrl,
                                               stall, wait_ns);
  return cudaGetLastError();
}

template <int F, bool SPLIT, int TN>
static cudaError_t launch_tc_z(int z, const CUtensorMap &tmA, const CUtensorMap &tmB,
                               const TcJobs &P, int grid, int kblocks, int stages, size_t smem,
                               float out_scale, uint32_t idesc, Ctrl *ctrl, int stall,
                               uint64_t wait_ns, cudaStream_t st) {
#define SNE_TC_Z(ZV)                                                                           \
  case ZV:                                                                                     \
    return launch_tc_kernel<F, ZV, SPLIT, TN>(tmA, tmB, P, grid, kblocks, stages, smem,        \
                                              out_scale, idesc, ctrl, stall, wait_ns, st);
  switch (z) {
    SNE_TC_Z(1)
    SNE_TC_Z(2)
    SNE_TC_Z(4)
    SNE_TC_Z(8)
    SNE_TC_Z(16)
    SNE_TC_Z(32)
    default:
      return cudaErrorInvalidValue;
  }
#undef SNE_TC_Z
}

cudaError_t launch_fused_sketch_tc_jobs(bool fp16, bool split, const void *arena,
                                        size_t arena_bytes, int kpad, int z, float sv, int f,
                                        const TcSketchJobDesc *jobs, int njobs, const TcTune &tune,
                                        Ctrl *ctrl, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  if (kpad % tc::BK != 0 || kpad <= 0 || !arena || ((uintptr_t)arena % 16)) return cudaErrorInvalidValue;
  if (!(z == 1 || z == 2 || z == 4 || z == 8 || z == 16 || z == 32)) return cudaErrorInvalidValue;
  const int tn = tune.tn == 128 ? 128 : 256;
  const int64_t rb = (int64_t)kpad * 2;  // bytes of one operand row
  const int64_t arena_rows = (int64_t)(arena_bytes / (size_t)rb);
  if (arena_rows <= 0 || arena_rows > INT32_MAX) return cudaErrorInvalidValue;
  // arena row of an operand: it must start on a row boundary of the arena
  auto row_of = [&](const void *ptr, int64_t rows, int64_t *out) -> bool {
    if (!ptr) return false;
    const int64_t off = (int64_t)((const char *)ptr - (const char *)arena);
    if (off < 0 || off % rb != 0) return false;
    *out = off / rb;
    return *out + rows <= arena_rows;
  };
  int stages = 0;
  const size_t smem = fused_tc_smem_bytes(kpad, split, tn, tune.stages, &stages);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  CUtensorMap tmA, tmB;
  if (!make_map(&tmA, fp16, arena, arena_rows, kpad, tc::BM)) return cudaErrorInvalidValue;
  if (!make_map(&tmB, fp16, arena, arena_rows, kpad, tn)) return cudaErrorInvalidValue;
  // instruction descriptor: D F32, A/B F16 (0) or BF16 (1), K-major, N = tn, M = 128
  const uint32_t fmt = fp16 ? 0u : 1u;
  const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(tn >> 3) << 17) |
                         ((uint32_t)(tc::BM >> 4) << 24);
  // SNE_FAULT_INJECT=tc_stall (tests of the failure path only): the kernel
  // leaves one shared-memory stage unloaded, and every bounded wait runs out
  // after 20 ms instead of 2 s
  int stall = 0;
  uint64_t wait_ns = tc::kTimeoutNs;
  if (const char *fi = getenv("SNE_FAULT_INJECT")) {
    if (std::strcmp(fi, "tc_stall") == 0) {
      stall = 1;
      wait_ns = 20000000ull;
    }
  }
  const int split_mult = tune.split_mult > 0 ? tune.split_mult : 2;
  for (int j0 = 0; j0 < njobs; j0 += kMaxTcJobs) {
    thread_local TcJobs P;  // host staging of the parameter block (copied at launch)
    P.njobs = 0;
    int64_t items = 0;
    for (int jq = j0; jq < njobs && jq < j0 + kMaxTcJobs; ++jq) {
      const TcSketchJobDesc &d = jobs[jq];
      if (d.nrows_max <= 0 || d.cols_out <= 0 || d.ncols_eval <= 0) continue;
      TcJob &J = P.job[P.njobs];
      const int64_t bpad = (d.ncols_eval + 255) / 256 * 256;
      if (!row_of(d.Ahi, d.nrows_max, &J.a_row) || !row_of(d.Bhi, bpad, &J.b_row))
        return cudaErrorInvalidValue;
      if (split) {
        if (!row_of(d.Alo, d.nrows_max, &J.a_lo_row) || !row_of(d.Blo, bpad, &J.b_lo_row))
          return cudaErrorInvalidValue;
      } else {
        J.a_lo_row = J.a_row;
        J.b_lo_row = J.b_row;
      }
      J.nrows_max = d.nrows_max;
      J.nrows_dev = d.nrows_dev;
      J.rowf = d.rowf;
      J.rowdat = d.rowdat;
      J.coldat = d.coldat;
      J.out = d.out;
      J.ldo = d.ldo;
      J.ctrl = d.ctrl ? d.ctrl : ctrl;
      J.ncols_eval = d.ncols_eval;
      J.cols_out = d.cols_out;
      const int64_t rowtiles = (d.nrows_max + tc::BM - 1) / tc::BM;
      const int ntiles = (d.ncols_eval + tn - 1) / tn;
      // few row tiles (the Z core): spread their column tiles over items so
      // that every SM has work
      const int64_t want = (split_mult * (int64_t)sm_count() + rowtiles - 1) / rowtiles;
      J.splits = (int32_t)std::max<int64_t>(1, std::min<int64_t>(ntiles, want));
      J.item_begin = (int32_t)items;
      items += rowtiles * J.splits;
      if (items > INT32_MAX) return cudaErrorInvalidValue;
      ++P.njobs;
    }
    if (P.njobs == 0) continue;
    P.total_items = (int32_t)items;
    const int grid = (int)std::min<int64_t>(items, (int64_t)sm_count());
    const int kblocks = kpad / tc::BK;
    ProfScope ps_(K_FUSED_TC, st);
    cudaError_t e;
#define SNE_TC_TN(FV, SV)                                                                     \
  e = tn == 128 ? launch_tc_z<FV, SV, 128>(z, tmA, tmB, P, grid, kblocks, stages, smem, sv,   \
                                           idesc, ctrl, stall, wait_ns, st)                   \
                : launch_tc_z<FV, SV, 256>(z, tmA, tmB, P, grid, kblocks, stages, smem, sv,   \
                                           idesc, ctrl, stall, wait_ns, st)
    if (f == SNE_F_TRUNC_LOG) {
      if (split) SNE_TC_TN(SNE_F_TRUNC_LOG, true); else SNE_TC_TN(SNE_F_TRUNC_LOG, false);
    } else {
      if (split) SNE_TC_TN(SNE_F_IDENTITY, true); else SNE_TC_TN(SNE_F_IDENTITY, false);
    }
#undef SNE_TC_TN
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace sne
