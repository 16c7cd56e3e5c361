// Mixed-precision fused reconstruct + f + sparse-sign sketch (Eq. 4 and the
// Z core of Alg. 4) on the fifth-generation tensor cores of sm_103a.
//
// The reconstruction L' R'(:, p) runs as a BF16 or FP16 GEMM with FP32
// accumulation.  Per-row and per-column scaling keeps both operands in
// [-1, 1]: A_hat[i, :] = U[i, :] / max|U[i, :]| with row factor
// rowf_i = max|U[i, :]| * vol/(bT) * d_i^(-1+alpha), and
// B_hat[e, :] = R'(:, idx_e)^T / colf_e with colf_e = max|R'(:, idx_e)|, so
// that x_ie = rowf_i * colf_e * <A_hat_i, B_hat_e> is formed in FP32 before f.
//
// One CTA owns a tile of 128 rows and walks over all evaluated columns in
// tiles of 256:
//   warp 0   TMA producer: the 128 x k A tile once, then 256 x 64 B k-blocks
//            through a ring of shared-memory stages (128-byte swizzle);
//   warp 1   allocates 512 TMEM columns (two 128 x 256 FP32 accumulators)
//            and issues tcgen05.mma (M 128, N 256, K 16) from one thread;
//   warps 2-17 epilogue: tcgen05.ld of the accumulator rows, x = scale * acc,
//            f(x), sign, and the z-column segmented sums in registers, then
//            the Y (or Y') row segment is stored.  Warp w reads TMEM lane
//            quarter w % 4 and 64 of the 256 columns; sixteen warps keep
//            enough loads, MUFU logs and stores in flight per scheduler.
// Double-buffered accumulators let the epilogue of tile j overlap the MMAs
// of tile j+1.  When the rows are few (the Z core: v_O rows, thousands of
// columns) blockIdx.y splits a row tile's column tiles over several CTAs.  Every mbarrier wait is bounded (about 2 s of %globaltimer);
// on timeout the CTA records SNE_ERR_TIMEOUT, stops issuing work, waits for
// its in-flight MMAs and copies, frees TMEM and returns.
#include <cuda.h>

#include <algorithm>

#include "sne_internal.cuh"
#include "tc_ptx.cuh"

namespace sne {

// PTX helpers: tc_ptx.cuh

template <int F, int Z>
__global__ void __launch_bounds__(tc::kThreadsSketch, 1) fused_sketch_tc_kernel(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
    int64_t nrows_max, const int32_t *__restrict__ nrows_dev, int kblocks, int stages,
    int ncols_eval, int cols_out, const float *__restrict__ rowf, const float *__restrict__ colf,
    float out_scale, uint32_t idesc, float *__restrict__ out, int64_t ldo, Ctrl *ctrl) {
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char *sA = smem;
  unsigned char *sB = sA + (size_t)kblocks * kABlockBytes;
  uint64_t *bars = reinterpret_cast<uint64_t *>(sB + (size_t)stages * kBStageBytes);
  uint64_t *a_full = bars;
  uint64_t *full = bars + 1;
  uint64_t *empty = full + stages;
  uint64_t *tfull = empty + stages;   // 2
  uint64_t *tempty = tfull + 2;       // 2
  uint64_t *done = tempty + 2;        // 1
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
  int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nrows = nrows_dev ? (int64_t)(*nrows_dev) : nrows_max;
  const int64_t row0 = (int64_t)blockIdx.x * BM;
  if (row0 >= nrows) return;  // uniform for the CTA
  const int ntiles = (ncols_eval + BN - 1) / BN;

  if (threadIdx.x == 0) {
    mbar_init(a_full, 1);
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 512);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512));
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
      mbar_expect_tx(a_full, (uint32_t)(kblocks * kABlockBytes));
      for (int kb = 0; kb < kblocks; ++kb)
        tma_load_2d(sA + (size_t)kb * kABlockBytes, &tmA, a_full, kb * BK, (int)row0);
      int it = 0;
      int issued = 0;
      bool ok = true;
      for (int j = blockIdx.y; j < ntiles && ok; j += gridDim.y) {
        for (int kb = 0; kb < kblocks; ++kb, ++it) {
          const int s = it % stages;
          const uint32_t ph = (uint32_t)((it / stages) & 1);
          if (!mbar_wait(&empty[s], ph ^ 1u, abortv, ctrl)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full[s], (uint32_t)kBStageBytes);
          tma_load_2d(sB + (size_t)s * kBStageBytes, &tmB, &full[s], kb * BK, j * BN);
          ++issued;
        }
      }
      if (!ok) {
        // let the copies already issued land before the CTA exits
        (void)mbar_wait(a_full, 0, abortv, ctrl);
        const int first = issued > stages ? issued - stages : 0;
        for (int q = first; q < issued; ++q) {
          const uint64_t t0 = gtimer();
          while (!mbar_try_wait(&full[q % stages], (uint32_t)((q / stages) & 1)) &&
                 gtimer() - t0 < kTimeoutNs) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      bool ok = mbar_wait(a_full, 0, abortv, ctrl);
      int it = 0;
      int jj = 0;  // local tile count (accumulator buffer and phase)
      for (int j = blockIdx.y; j < ntiles && ok; j += gridDim.y, ++jj) {
        const int buf = jj & 1;
        const uint32_t use = (uint32_t)(jj >> 1);
        if (!mbar_wait(&tempty[buf], (use & 1u) ^ 1u, abortv, ctrl)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t dt = tmem + (uint32_t)(buf * BN);
        for (int kb = 0; kb < kblocks; ++kb, ++it) {
          const int s = it % stages;
          if (!mbar_wait(&full[s], (uint32_t)((it / stages) & 1), abortv, ctrl)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t a0 = smem_u32(sA + (size_t)kb * kABlockBytes);
          const uint32_t b0 = smem_u32(sB + (size_t)s * kBStageBytes);
#pragma unroll
          for (int kk = 0; kk < BK / 16; ++kk)
            mma_f16(dt, sdesc(a0 + kk * 32), sdesc(b0 + kk * 32), idesc, (kb | kk) ? 1u : 0u);
          mma_commit(&empty[s]);
        }
        if (!ok) break;
        mma_commit(&tfull[buf]);
      }
      // wait for every MMA issued by this thread before TMEM is released
      mma_commit(done);
      const uint64_t t0 = gtimer();
      while (!mbar_try_wait(done, 0) && gtimer() - t0 < kTimeoutNs) {
      }
    }
  } else {
    // ---------------- epilogue warps 2..17: warp w reads TMEM lane quarter
    // w % 4 (rows 32(w%4) .. +32) and quarter (w - 2) / 4 of the 256 columns
    const int ew = warp & 3;
    const int quarter = (warp - 2) >> 2;
    const int64_t row = row0 + 32 * ew + lane;
    const bool row_ok = row < nrows;
    const float rf = row_ok ? rowf[row] : 0.0f;
    constexpr int G = 32 / Z;        // output columns per 32-column chunk
    int jj = 0;
    for (int j = blockIdx.y; j < ntiles; j += gridDim.y, ++jj) {
      const int buf = jj & 1;
      const uint32_t use = (uint32_t)(jj >> 1);
      if (!mbar_wait(&tfull[buf], use & 1u, abortv, ctrl)) break;
      fence_after();
      const int ebase = j * BN + quarter * 64;
      float v[2][32];
      const uint32_t taddr = tmem + ((uint32_t)(32 * ew) << 16) + (uint32_t)(buf * BN + quarter * 64);
      tmem_ld32_nw(taddr, v[0]);
      tmem_ld32_nw(taddr + 32, v[1]);
      tmem_wait_ld();
      // the accumulator is in registers: release it to the MMA warp early
      fence_before();
      mbar_arrive(&tempty[buf]);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const float4 *cf4 = reinterpret_cast<const float4 *>(colf + ebase + c * 32);
        float acc[G];
#pragma unroll
        for (int g = 0; g < G; ++g) acc[g] = 0.0f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const float4 cf = __ldg(cf4 + q);
          const float cfv[4] = {cf.x, cf.y, cf.z, cf.w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int t = 4 * q + u;
            const float x = rf * fabsf(cfv[u]) * v[c][t];
            const float l = tc::fx2<F>(x);
            // trunc_log is >= 0, so the sign of cf can be copied onto it
            if (F == SNE_F_TRUNC_LOG) acc[t / Z] += copysignf(l, cfv[u]);
            else acc[t / Z] += (cfv[u] < 0.0f) ? -l : l;
          }
        }
        // G consecutive outputs of this row: columns (ebase + 32 c) / Z ..
        const int oc0 = (ebase + 32 * c) / Z;
        if (row_ok && oc0 < cols_out) {
          float *o = out + row * ldo + oc0;
          if (G % 4 == 0 && oc0 + G <= cols_out && ((reinterpret_cast<uintptr_t>(o) & 15) == 0)) {
#pragma unroll
            for (int g = 0; g < G; g += 4)
              *reinterpret_cast<float4 *>(o + g) =
                  make_float4(out_scale * acc[g], out_scale * acc[g + 1], out_scale * acc[g + 2],
                              out_scale * acc[g + 3]);
          } else {
#pragma unroll
            for (int g = 0; g < G; ++g)
              if (oc0 + g < cols_out) o[g] = out_scale * acc[g];
          }
        }
      }
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// ---------------------------------------------------------------------------
// Row-normalized half-precision copies of the GEMM operands
// ---------------------------------------------------------------------------
template <typename H>
__device__ __forceinline__ H to_h(float x);
template <>
__device__ __forceinline__ __nv_bfloat16 to_h<__nv_bfloat16>(float x) {
  return __float2bfloat16_rn(x);
}
template <>
__device__ __forceinline__ __half to_h<__half>(float x) {
  return __float2half_rn(x);
}

// dst[r, :kpad] = src[s(r), :k] / max|src[s(r), :k]| (zero padded); scale[r] =
// max|src[s(r), :]| * extra[s(r)].  Rows r >= *nrows_dev (when given) are zero.
template <typename H>
__global__ void __launch_bounds__(256) to_half_rows_kernel(
    const float *__restrict__ src, int64_t lds, const int32_t *__restrict__ ridx,
    const int32_t *__restrict__ nrows_dev, int64_t nrows_max, int k, int kpad,
    const float *__restrict__ extra, const int8_t *__restrict__ sgn, H *__restrict__ dst,
    float *__restrict__ scale) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (r >= nrows_max) return;
  const int64_t nrows = nrows_dev ? (int64_t)(*nrows_dev) : nrows_max;
  H *d = dst + r * kpad;
  if (r >= nrows) {
    for (int c = lane; c < kpad; c += 32) d[c] = to_h<H>(0.0f);
    if (lane == 0) scale[r] = 0.0f;
    return;
  }
  const int64_t s = ridx ? (int64_t)ridx[r] : r;
  const float *x = src + s * lds;
  float m = 0.0f;
  for (int c = lane; c < k; c += 32) m = fmaxf(m, fabsf(x[c]));
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  const float inv = m > 0.0f ? 1.0f / m : 0.0f;
  for (int c = lane; c < kpad; c += 32) d[c] = to_h<H>(c < k ? x[c] * inv : 0.0f);
  if (lane == 0) {
    const float sc = m * (extra ? extra[s] : 1.0f);
    scale[r] = (sgn && sgn[r] < 0) ? -sc : sc;
  }
}

cudaError_t launch_to_half_rows(bool fp16, const float *src, int64_t lds, const int32_t *ridx,
                                const int32_t *nrows_dev, int64_t nrows_max, int k, int kpad,
                                const float *extra, const int8_t *sgn, void *dst, float *scale,
                                cudaStream_t st) {
  if (nrows_max <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((nrows_max + 7) / 8);
  ProfScope ps_(K_MISC, st);
  if (fp16)
    to_half_rows_kernel<__half><<<blocks, 256, 0, st>>>(src, lds, ridx, nrows_dev, nrows_max, k, kpad,
                                                        extra, sgn, static_cast<__half *>(dst), scale);
  else
    to_half_rows_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(
        src, lds, ridx, nrows_dev, nrows_max, k, kpad, extra, sgn, static_cast<__nv_bfloat16 *>(dst),
        scale);
  return cudaGetLastError();
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

size_t fused_tc_smem_bytes(int kpad, int *stages_out) {
  const int kblocks = kpad / tc::BK;
  int stages = 4;
  while (stages > 2 && (size_t)kblocks * tc::kABlockBytes + (size_t)stages * tc::kBStageBytes >
                           200 * 1024)
    --stages;
  if (stages_out) *stages_out = stages;
  return 1024 + (size_t)kblocks * tc::kABlockBytes + (size_t)stages * tc::kBStageBytes + 256;
}

cudaError_t launch_fused_sketch_tc(bool fp16, const void *Ahat, int64_t nrows_max,
                                   const int32_t *nrows_dev, int kpad, const void *Bhat,
                                   int ncols_eval, int cols_out, int z, const float *rowf,
                                   const float *colf, const int8_t *sign, float sv, int f, float *out,
                                   int64_t ldo, Ctrl *ctrl, cudaStream_t st) {
  if (nrows_max <= 0 || cols_out <= 0) return cudaSuccess;
  if (kpad % tc::BK != 0 || kpad <= 0) return cudaErrorInvalidValue;
  if (!(z == 1 || z == 2 || z == 4 || z == 8 || z == 16 || z == 32)) return cudaErrorInvalidValue;
  if (((uintptr_t)Ahat % 16) || ((uintptr_t)Bhat % 16)) return cudaErrorInvalidValue;
  int stages = 0;
  const size_t smem = fused_tc_smem_bytes(kpad, &stages);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  CUtensorMap tmA, tmB;
  if (!make_map(&tmA, fp16, Ahat, nrows_max, kpad, tc::BM)) return cudaErrorInvalidValue;
  if (!make_map(&tmB, fp16, Bhat, ncols_eval, kpad, tc::BN)) return cudaErrorInvalidValue;
  // instruction descriptor: D F32, A/B F16 (0) or BF16 (1), K-major, N = 256, M = 128
  const uint32_t fmt = fp16 ? 0u : 1u;
  const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(tc::BN >> 3) << 17) |
                         ((uint32_t)(tc::BM >> 4) << 24);
  const unsigned grid_x = (unsigned)((nrows_max + tc::BM - 1) / tc::BM);
  // few row tiles (the Z core): spread their column tiles over CTAs so that
  // at least two CTAs per SM's worth of work exists
  const int ntiles = (ncols_eval + tc::BN - 1) / tc::BN;
  const unsigned splits = (unsigned)std::max(
      1, std::min(ntiles, (int)((2 * sm_count() + grid_x - 1) / grid_x)));
  const dim3 grid(grid_x, splits);
  const int kblocks = kpad / tc::BK;
  // f = trunc_log: the kernel sums signed log2 values; ln 2 joins sv here
  const float out_scale = (f == SNE_F_TRUNC_LOG) ? sv * 0.69314718055994530942f : sv;
  (void)sign;
#define SNE_TC_LAUNCH(FV, ZV)                                                                     \
  do {                                                                                            \
    auto kern = fused_sketch_tc_kernel<FV, ZV>;                                                   \
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                         (int)smem);                                              \
    if (e != cudaSuccess) return e;                                                               \
    ProfScope ps_(K_FUSED_TC, st);                                                                \
    kern<<<grid, tc::kThreadsSketch, smem, st>>>(tmA, tmB, nrows_max, nrows_dev, kblocks, stages, \
                                                 ncols_eval, cols_out, rowf, colf, out_scale,     \
                                                 idesc, out, ldo, ctrl);                          \
  } while (0)
#define SNE_TC_Z(FV)             \
  switch (z) {                   \
    case 1: SNE_TC_LAUNCH(FV, 1); break;  \
    case 2: SNE_TC_LAUNCH(FV, 2); break;  \
    case 4: SNE_TC_LAUNCH(FV, 4); break;  \
    case 8: SNE_TC_LAUNCH(FV, 8); break;  \
    case 16: SNE_TC_LAUNCH(FV, 16); break; \
    default: SNE_TC_LAUNCH(FV, 32); break; \
  }
  if (f == SNE_F_TRUNC_LOG) {
    SNE_TC_Z(SNE_F_TRUNC_LOG)
  } else {
    SNE_TC_Z(SNE_F_IDENTITY)
  }
#undef SNE_TC_Z
#undef SNE_TC_LAUNCH
  return cudaGetLastError();
}

}  // namespace sne
