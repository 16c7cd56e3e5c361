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
#include <cstdlib>
#include <cstring>

#include "sne_internal.cuh"
#include "tc_ptx.cuh"

namespace sne {

// PTX helpers: tc_ptx.cuh

template <int F, int Z, bool SPLIT>
__global__ void __launch_bounds__(tc::kThreadsSketch, 1) fused_sketch_tc_kernel(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmA2,
    const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmB2,
    int64_t nrows_max, const int32_t *__restrict__ nrows_dev, int kblocks, int stages,
    int ncols_eval, int cols_out, const float *__restrict__ rowf,
    const float2 *__restrict__ rowdat, const float4 *__restrict__ coldat, float out_scale,
    uint32_t idesc, float *__restrict__ out, int64_t ldo, Ctrl *ctrl, int stall,
    uint64_t wait_ns) {
  using namespace tc;
  constexpr int NPART = SPLIT ? 2 : 1;
  extern __shared__ __align__(1024) unsigned char tc_smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
  unsigned char *sA = smem;                                     // hi k-blocks, then lo
  unsigned char *sB = sA + (size_t)NPART * kblocks * kABlockBytes;
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
  const int steps = kblocks * NPART;  // B stages per column tile

  if (threadIdx.x == 0) {
    mbar_init(a_full, 1);
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
      mbar_expect_tx(a_full, (uint32_t)(NPART * kblocks * kABlockBytes));
      for (int kb = 0; kb < kblocks; ++kb) {
        tma_load_2d(sA + (size_t)kb * kABlockBytes, &tmA, a_full, kb * BK, (int)row0);
        if (SPLIT)
          tma_load_2d(sA + (size_t)(kblocks + kb) * kABlockBytes, &tmA2, a_full, kb * BK,
                      (int)row0);
      }
      int it = 0;
      int last_it = -1;  // the ring index of the last copy issued
      bool ok = true;
      for (int j = blockIdx.y; j < ntiles && ok; j += gridDim.y) {
        for (int q = 0; q < steps; ++q, ++it) {
          const int kb = q / NPART, part = q % NPART;
          const int s = it % stages;
          const uint32_t ph = (uint32_t)((it / stages) & 1);
          if (!mbar_wait(&empty[s], ph ^ 1u, abortv, ctrl, wait_ns)) {
            ok = false;
            break;
          }
          // fault injection (tests only): the first stage is never loaded,
          // so the MMA warp's wait on it runs out
          if (stall && it == 0) continue;
          mbar_expect_tx(&full[s], (uint32_t)kBStageBytes);
          tma_load_2d(sB + (size_t)s * kBStageBytes, part ? &tmB2 : &tmB, &full[s], kb * BK, j * BN);
          last_it = it;
        }
      }
      if (!ok) {
        // let the copies already issued land before the CTA exits (the
        // last `stages` of them; the others completed before their stage
        // was reused)
        mbar_drain(a_full, 0, wait_ns);
        for (int q = (last_it - stages + 1 > 0 ? last_it - stages + 1 : 0); q <= last_it; ++q) {
          if (stall && q == 0) continue;
          mbar_drain(&full[q % stages], (uint32_t)((q / stages) & 1), wait_ns);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer
      bool ok = mbar_wait(a_full, 0, abortv, ctrl, wait_ns);
      int it = 0;
      int jj = 0;  // local tile count (accumulator buffer and phase)
      for (int j = blockIdx.y; j < ntiles && ok; j += gridDim.y, ++jj) {
        const int buf = jj & 1;
        const uint32_t use = (uint32_t)(jj >> 1);
        if (!mbar_wait(&tempty[buf], (use & 1u) ^ 1u, abortv, ctrl, wait_ns)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t dt = tmem + (uint32_t)(buf * BN);
        // a last column tile at most half full runs at N = 128: the columns
        // past it are neither multiplied nor read by the epilogue
        const uint32_t id = (ncols_eval - j * BN <= BN / 2)
                                ? ((idesc & ~(0x3fu << 17)) | ((uint32_t)(BN / 2 >> 3) << 17))
                                : idesc;
        for (int q = 0; q < steps; ++q, ++it) {
          const int kb = q / NPART, part = q % NPART;
          const int s = it % stages;
          if (!mbar_wait(&full[s], (uint32_t)((it / stages) & 1), abortv, ctrl, wait_ns)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t ahi = smem_u32(sA + (size_t)kb * kABlockBytes);
          const uint32_t b0 = smem_u32(sB + (size_t)s * kBStageBytes);
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
      // wait for every MMA issued by this thread before TMEM is released
      mma_commit(done);
      mbar_drain(done, 0, wait_ns);
    }
  } else {
    // ---------------- epilogue warps: warp w reads TMEM lane quarter w % 4
    // (rows 32(w%4) .. +32) and column slice (w - 2) / 4 of the 256 columns
    constexpr int CPW = BN / (kSketchEpiWarps / 4);  // columns per warp and tile
    static_assert(kSketchEpiWarps % 4 == 0 && CPW % 32 == 0, "epilogue warp split");
    const int ew = warp & 3;
    const int quarter = (warp - 2) >> 2;
    const int64_t row = row0 + 32 * ew + lane;
    const bool row_ok = row < nrows;
    const float rf = row_ok ? rowf[row] : 0.0f;
    const float2 rd = row_ok ? rowdat[row] : make_float2(0.0f, 0.0f);
    constexpr int G = 32 / Z;        // output columns per 32-column chunk
    int jj = 0;
    for (int j = blockIdx.y; j < ntiles; j += gridDim.y, ++jj) {
      const int buf = jj & 1;
      const uint32_t use = (uint32_t)(jj >> 1);
      if (!mbar_wait(&tfull[buf], use & 1u, abortv, ctrl, wait_ns)) break;
      fence_after();
      const int ebase = j * BN + quarter * CPW;
      const uint32_t taddr = tmem + ((uint32_t)(32 * ew) << 16) + (uint32_t)(buf * BN + quarter * CPW);
      // the warp's columns in chunks of 32; the accumulator goes back to the
      // MMA warp once the last chunk is in registers
#pragma unroll 1
      for (int c = 0; c < CPW / 32; ++c) {
        if (ebase + 32 * c >= ncols_eval) {
          // past the evaluated columns (a partial last tile): nothing to read
          if (c == CPW / 32 - 1) {
            fence_before();
            mbar_arrive(&tempty[buf]);
          }
          continue;
        }
        float vc[32];
        tmem_ld32_nw(taddr + 32 * c, vc);
        tmem_wait_ld();
        if (c == CPW / 32 - 1) {
          fence_before();
          mbar_arrive(&tempty[buf]);
        }
        // the chunk's column data, lane t holding column t, broadcast by
        // shuffles (32 uniform loads per chunk, hoisted by the compiler to
        // the top of the loop, would spill)
        const float4 cdl = __ldg(coldat + ebase + c * 32 + lane);
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

size_t fused_tc_smem_bytes(int kpad, bool split, int *stages_out) {
  const int kblocks = kpad / tc::BK;
  const size_t abytes = (size_t)(split ? 2 : 1) * kblocks * tc::kABlockBytes;
  // 1 KB alignment slack and 256 bytes of barriers next to A and the B ring
  const size_t budget = 227 * 1024 - 1024 - 256;
  int stages = 4;
  while (stages > 2 && abytes + (size_t)stages * tc::kBStageBytes > budget) --stages;
  if (stages_out) *stages_out = stages;
  return 1024 + abytes + (size_t)stages * tc::kBStageBytes + 256;
}

cudaError_t launch_fused_sketch_tc(bool fp16, bool split, const void *Ahi, const void *Alo,
                                   int64_t nrows_max, const int32_t *nrows_dev, int kpad,
                                   const void *Bhi, const void *Blo, int ncols_eval, int cols_out,
                                   int z, const float *rowf, const float2 *rowdat,
                                   const float4 *coldat, float sv, int f, float *out, int64_t ldo,
                                   Ctrl *ctrl, cudaStream_t st) {
  if (nrows_max <= 0 || cols_out <= 0) return cudaSuccess;
  if (kpad % tc::BK != 0 || kpad <= 0) return cudaErrorInvalidValue;
  if (!(z == 1 || z == 2 || z == 4 || z == 8 || z == 16 || z == 32)) return cudaErrorInvalidValue;
  if (((uintptr_t)Ahi % 16) || ((uintptr_t)Bhi % 16)) return cudaErrorInvalidValue;
  if (split && (!Alo || !Blo || ((uintptr_t)Alo % 16) || ((uintptr_t)Blo % 16)))
    return cudaErrorInvalidValue;
  int stages = 0;
  const size_t smem = fused_tc_smem_bytes(kpad, split, &stages);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  CUtensorMap tmA, tmA2, tmB, tmB2;
  if (!make_map(&tmA, fp16, Ahi, nrows_max, kpad, tc::BM)) return cudaErrorInvalidValue;
  if (!make_map(&tmB, fp16, Bhi, ncols_eval, kpad, tc::BN)) return cudaErrorInvalidValue;
  if (split) {
    if (!make_map(&tmA2, fp16, Alo, nrows_max, kpad, tc::BM)) return cudaErrorInvalidValue;
    if (!make_map(&tmB2, fp16, Blo, ncols_eval, kpad, tc::BN)) return cudaErrorInvalidValue;
  } else {
    tmA2 = tmA;
    tmB2 = tmB;
  }
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
  const float out_scale = sv;
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
#define SNE_TC_LAUNCH(FV, ZV, SV)                                                                 \
  do {                                                                                            \
    auto kern = fused_sketch_tc_kernel<FV, ZV, SV>;                                               \
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,       \
                                         (int)smem);                                              \
    if (e != cudaSuccess) return e;                                                               \
    ProfScope ps_(K_FUSED_TC, st);                                                                \
    kern<<<grid, tc::kThreadsSketch, smem, st>>>(tmA, tmA2, tmB, tmB2, nrows_max, nrows_dev,      \
                                                 kblocks, stages, ncols_eval, cols_out, rowf,     \
                                                 rowdat, coldat, out_scale, idesc, out, ldo,      \
                                                 ctrl, stall, wait_ns);                           \
  } while (0)
#define SNE_TC_Z(FV, SV)                        \
  switch (z) {                                  \
    case 1: SNE_TC_LAUNCH(FV, 1, SV); break;    \
    case 2: SNE_TC_LAUNCH(FV, 2, SV); break;    \
    case 4: SNE_TC_LAUNCH(FV, 4, SV); break;    \
    case 8: SNE_TC_LAUNCH(FV, 8, SV); break;    \
    case 16: SNE_TC_LAUNCH(FV, 16, SV); break;  \
    default: SNE_TC_LAUNCH(FV, 32, SV); break;  \
  }
  if (f == SNE_F_TRUNC_LOG) {
    if (split) {
      SNE_TC_Z(SNE_F_TRUNC_LOG, true)
    } else {
      SNE_TC_Z(SNE_F_TRUNC_LOG, false)
    }
  } else {
    if (split) {
      SNE_TC_Z(SNE_F_IDENTITY, true)
    } else {
      SNE_TC_Z(SNE_F_IDENTITY, false)
    }
  }
#undef SNE_TC_Z
#undef SNE_TC_LAUNCH
  return cudaGetLastError();
}

}  // namespace sne
