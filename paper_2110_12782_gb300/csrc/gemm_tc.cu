// FP32-accurate tall-skinny products on tcgen05 (kind::tf32, three passes):
//   TALL  C[i, :] = A[i, :] M            (A n x K row-major, M K x Kc; the
//                                          operand B is M^T, K-major)
//   GRAM  P[c]    = sum_{i in chunk c} w_i A[i, :]^T B[i, :]
//                                        (the row-major tall matrices arrive
//                                          as 32 x 32 boxes and are transposed
//                                          into K-major tiles in shared memory)
// used for the eigSVD / Cholesky-QR orthonormalizations and the Rayleigh-Ritz
// product of Alg. 5, the sketch QR of Alg. 4 and E = Q U_hat.
//
// Each operand x is split into hi = rna_tf32(x) and lo = x - hi (exact), and
// the accumulator takes A_hi B_hi + A_hi B_lo + A_lo B_hi, so the product
// carries about 2^-21 relative error per term (the FP32 result up to the
// dropped A_lo B_lo term).  Four split warps do this in shared memory between
// the TMA load and the MMA of every stage, for the tall operands.
//
// TALL: a persistent CTA per SM walks (128-row tile, column half) work items
// over Npad <= 288 output columns (halves of at most 160 columns, one MMA of
// N = half width per k-step and product); the small operand M^T is split into
// TF32 hi/lo once per call and loaded by TMA, so only A is split in shared
// memory.  Warp 0: TMA; warp 1: TMEM and MMA issue; warps 2-5: split of A;
// warps 6-9: epilogue (tcgen05.ld, store) from two alternating accumulators.
#include <cuda.h>
#include <cuda.h>

#include "sne_internal.cuh"
#include "tc_ptx.cuh"

namespace sne {

namespace gt {
constexpr int BM = 128;        // output rows per tile (MMA M)
constexpr int BK = 32;         // FP32 elements per k-block (128 bytes)
constexpr int kMaxN = 288;     // padded output columns
constexpr int kHalfFrom = 160; // wider outputs go in two column halves
constexpr int kStages = 3;
constexpr int kThreads = 320;  // TMA, MMA, 4 split warps, 4 epilogue warps
constexpr int kABytes = BM * BK * 4;  // 16 KB
}  // namespace gt

// Column halves of an npad-column output: N0 (the wider, a multiple of 32) and
// N1 (0 for one pass).
__host__ __device__ inline void tall_halves(int npad, int *N0, int *N1) {
  if (npad <= gt::kHalfFrom) {
    *N0 = npad;
    *N1 = 0;
  } else {
    *N0 = ((npad / 2) + 31) / 32 * 32;
    *N1 = npad - *N0;
  }
}

// Persistent: CTA b takes the work items b, b + gridDim.x, ... of the list
// (row tile, column half); the second half of a tile re-reads the tile's A
// rows, from L2.  The operand B = M^T arrives already split (rows 0 .. npad
// hi, rows npad .. 2 npad lo; split once per call), so the split warps only
// split A, and with halves of at most 160 columns a stage (A hi, A lo, B hi,
// B lo) is at most 72 KB: three stages.  The two TMEM accumulators (columns
// 0 and 256) alternate between work items, so that the epilogue of one
// overlaps the MMAs of the next; the stage ring and the barrier phases run on
// across work items.
//
// PAIR: the CTAs run in clusters of two that take the row tiles 2t and 2t + 1
// of the same work items in lockstep; each CTA loads half of every B stage
// and multicasts it to both, so that the split M^T (the same for every tile)
// is read from L2 once per pair instead of once per CTA.  A stage is free
// again only when the MMAs of both CTAs are done with it (the MMA commits
// arrive on the empty barriers of both), and the cluster synchronizes after
// its barriers are initialized and before it exits.
template <bool PAIR>
__global__ void __launch_bounds__(gt::kThreads, 1) tall_tf32x3_kernel(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB0,
    const __grid_constant__ CUtensorMap tmB1, int npad, int nkb, int64_t ntiles, int64_t nrows,
    int ncols, float *__restrict__ out, int64_t ldo, int vec4, Ctrl *ctrl) {
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char g_smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(g_smem_raw) + 1023) & ~(uintptr_t)1023);
  int N0, N1;
  tall_halves(npad, &N0, &N1);
  const int nhalf = N1 > 0 ? 2 : 1;
  const int bmax = N0 * gt::BK * 4;                    // B bytes (hi or lo) of the wider half
  const int stage_bytes = 2 * gt::kABytes + 2 * bmax;  // A hi | A lo | B hi | B lo
  uint64_t *bars = reinterpret_cast<uint64_t *>(smem + (size_t)gt::kStages * stage_bytes);
  uint64_t *full = bars;                    // [stages] TMA landed
  uint64_t *split = full + gt::kStages;     // [stages] A split
  uint64_t *empty = split + gt::kStages;    // [stages] MMA done with the stage
  uint64_t *accfull = empty + gt::kStages;  // [2] accumulator of a work item complete
  uint64_t *accfree = accfull + 2;          // [2] the epilogue has read it out
  uint64_t *done = accfree + 2;             // every MMA issued has completed
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
  int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // work items (tile pair or tile, half); this CTA's tile of item w
  const uint32_t rank = PAIR ? cluster_ctarank() : 0u;
  const int64_t nitems = (PAIR ? (ntiles + 1) / 2 : ntiles) * nhalf;
  const int64_t first = PAIR ? (int64_t)(blockIdx.x >> 1) : (int64_t)blockIdx.x;
  const int64_t step = PAIR ? (int64_t)(gridDim.x >> 1) : (int64_t)gridDim.x;
  auto item = [&](int64_t w, int64_t &tile, int &half) {
    const int64_t tq = w / nhalf;
    half = (int)(w - tq * nhalf);
    tile = PAIR ? 2 * tq + rank : tq;
  };

  if (threadIdx.x == 0) {
    for (int s = 0; s < gt::kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&split[s], 128);
      mbar_init(&empty[s], PAIR ? 2 : 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accfull[b], 1);
      mbar_init(&accfree[b], 128);
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
  if (PAIR) cluster_sync_all();  // the peer's barriers exist before any multicast
  const uint32_t tmem = *tmem_slot;
  volatile int *abortv = abort_flag;

  auto stage_ptr = [&](int s) { return smem + (size_t)s * stage_bytes; };
  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      uint32_t it = 0;
      bool ok = true;
      for (int64_t w = first; w < nitems && ok; w += step) {
        int64_t tile;
        int half;
        item(w, tile, half);
        const int N = half ? N1 : N0, c0 = half ? N0 : 0;
        const CUtensorMap *tmB = half ? &tmB1 : &tmB0;
        const int m0 = (int)(tile * gt::BM);
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = it % gt::kStages;
          if (!mbar_wait(&empty[s], ((it / gt::kStages) & 1) ^ 1, abortv, ctrl)) {
            ok = false;
            break;
          }
          unsigned char *st = stage_ptr(s);
          mbar_expect_tx(&full[s], (uint32_t)(gt::kABytes + 2 * N * gt::BK * 4));
          // A box {32 k, 128 rows}; B boxes {32 k, N rows}: hi rows c0 ..,
          // lo rows npad + c0 ..
          tma_load_2d(st, &tmA, &full[s], kb * gt::BK, m0);
          if (PAIR) {
            // this CTA's half of the B rows, to both CTAs of the pair
            const int Nh = N / 2, off = (int)rank * Nh;
            tma_load_2d_mc(st + 2 * gt::kABytes + off * 128, tmB, &full[s], kb * gt::BK, c0 + off,
                           (uint16_t)3);
            tma_load_2d_mc(st + 2 * gt::kABytes + bmax + off * 128, tmB, &full[s], kb * gt::BK,
                           npad + c0 + off, (uint16_t)3);
          } else {
            tma_load_2d(st + 2 * gt::kABytes, tmB, &full[s], kb * gt::BK, c0);
            tma_load_2d(st + 2 * gt::kABytes + bmax, tmB, &full[s], kb * gt::BK, npad + c0);
          }
        }
      }
      if (!ok) {
        // let the copies this CTA issued land before it exits
        const uint32_t first = it > (uint32_t)gt::kStages ? it - gt::kStages : 0;
        for (uint32_t q = first; q < it; ++q)
          mbar_drain(&full[q % gt::kStages], (q / gt::kStages) & 1, kTimeoutNs);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---------------- MMA issuer.  Instruction descriptor: D F32, A/B TF32
      // (2), K-major, N, M = 128
      const uint32_t base = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(gt::BM >> 4) << 24);
      uint32_t it = 0, u = 0;
      bool ok = true;
      for (int64_t w = first; w < nitems && ok; w += step, ++u) {
        int64_t tile;
        int half;
        item(w, tile, half);
        const int N = half ? N1 : N0;
        const uint32_t idesc = base | ((uint32_t)(N >> 3) << 17);
        const int buf = u & 1;
        if (!mbar_wait(&accfree[buf], ((u >> 1) & 1) ^ 1, abortv, ctrl)) break;
        fence_after();
        const uint32_t dt = tmem + (uint32_t)(buf * 256);
        for (int kb = 0; kb < nkb; ++kb, ++it) {
          const int s = it % gt::kStages;
          if (!mbar_wait(&split[s], (it / gt::kStages) & 1, abortv, ctrl)) {
            ok = false;
            break;
          }
          fence_after();
          const uint32_t ahi = smem_u32(stage_ptr(s));
          const uint32_t alo = ahi + gt::kABytes;
          const uint32_t bhi = ahi + 2 * gt::kABytes;
          const uint32_t blo = bhi + bmax;
#pragma unroll
          for (int kk = 0; kk < gt::BK / 8; ++kk) {
            const uint32_t acc = (kb | kk) ? 1u : 0u;
            const uint64_t da_hi = sdesc2(ahi + kk * 32, 16, 1024);
            const uint64_t db_hi = sdesc2(bhi + kk * 32, 16, 1024);
            mma_tf32(dt, da_hi, db_hi, idesc, acc);
            mma_tf32(dt, da_hi, sdesc2(blo + kk * 32, 16, 1024), idesc, 1u);
            mma_tf32(dt, sdesc2(alo + kk * 32, 16, 1024), db_hi, idesc, 1u);
          }
          if (PAIR)
            mma_commit_mc(&empty[s], (uint16_t)3);
          else
            mma_commit(&empty[s]);
        }
        if (ok) mma_commit(&accfull[buf]);
      }
      // every issued MMA has completed before TMEM is released
      mma_commit(done);
      mbar_drain(done, 0, kTimeoutNs);
    }
  } else if (warp < 6) {
    // ---------------- warps 2..5: split of A (elementwise, in place)
    const int t = threadIdx.x - 64;  // 0..127
    uint32_t it = 0;
    bool ok = true;
    for (int64_t w = first; w < nitems && ok; w += step) {
      for (int kb = 0; kb < nkb; ++kb, ++it) {
        const int s = it % gt::kStages;
        if (!mbar_wait(&full[s], (it / gt::kStages) & 1, abortv, ctrl)) {
          ok = false;
          break;
        }
        unsigned char *st = stage_ptr(s);
        float4 *ahi = reinterpret_cast<float4 *>(st);
        float4 *alo = reinterpret_cast<float4 *>(st + gt::kABytes);
#pragma unroll 4
        for (int q = t; q < gt::kABytes / 16; q += 128) {
          const float4 x = ahi[q];
          const float4 h = make_float4(tf32_rna(x.x), tf32_rna(x.y), tf32_rna(x.z), tf32_rna(x.w));
          ahi[q] = h;
          alo[q] = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&split[s]);
      }
    }
  } else {
    // ---------------- warps 6..9: epilogue, one accumulator row per thread
    const int ew = warp & 3;  // TMEM lane quarter of this warp
    uint32_t u = 0;
    for (int64_t w = first; w < nitems; w += step, ++u) {
      int64_t tile;
      int half;
      item(w, tile, half);
      const int N = half ? N1 : N0, c0 = half ? N0 : 0;
      const int buf = u & 1;
      if (!mbar_wait(&accfull[buf], (u >> 1) & 1, abortv, ctrl)) break;
      fence_after();
      const int64_t r = tile * gt::BM + 32 * ew + lane;
      float *orow = out + r * ldo + c0;
      const bool rok = r < nrows;
      for (int c = 0; c < N; c += 32) {
        float v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * ew) << 16) + (uint32_t)(buf * 256 + c), v);
        if (rok) {
          if (vec4 && c0 + c + 32 <= ncols) {
#pragma unroll
            for (int q = 0; q < 32; q += 4)
              *reinterpret_cast<float4 *>(orow + c + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
          } else {
#pragma unroll
            for (int q = 0; q < 32; ++q)
              if (c0 + c + q < ncols) orow[c + q] = v[q];
          }
        }
      }
      fence_before();
      mbar_arrive(&accfree[buf]);
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  // no copy or MMA commit of the peer targets this CTA after this point
  if (PAIR) cluster_sync_all();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// ---------------------------------------------------------------------------
// Gram kernel.  The row-major tall matrices arrive from TMA as 32 x 32 boxes in
// which the contiguous direction is the output index (a or b) and the rows are
// the reduction index i.  The split warps transpose every box into the
// K-major 128-byte-swizzled layout (row = a or b, 32 consecutive i per
// 128-byte row, 16-byte chunk c of row r stored at chunk c ^ (r % 8)) while
// forming hi and lo, so the MMA reads K-major operands.
//
// The tensor-core accumulator does not round like IEEE addition: summing a
// long chain of small products into a large total drifts.  So each TMEM
// accumulator takes only kSeg k-blocks (kSeg * 32 rows, 3 * 4 * kSeg MMA
// updates) before the MMA moves to the other accumulator, and eight drain
// warps (two per TMEM lane quarter, 64 columns each) add the finished one into
// FP32 registers with ordinary (round-to-nearest) additions.  Output tile
// 128 (a) x 128 (b).  The transposing split is the costliest part of the
// kernel (without it a launch takes 58% of the time), so eight warps share it.
// Warps: 0 TMA, 1 MMA, 2-9 split, 10-17 drain.
// ---------------------------------------------------------------------------
namespace gg {
constexpr int BN = 128;
constexpr int kSeg = 4;
constexpr int kSplitThreads = 256;        // warps 2-9
constexpr int kDrainThreads = 256;        // warps 10-17
constexpr int kThreads = 64 + kSplitThreads + kDrainThreads;
constexpr int kTileBytes = 128 * 32 * 4;  // 16 KB: 128 rows x 32 fp32
constexpr int kRawStages = 3;             // TMA stages of raw boxes
}  // namespace gg

__global__ void __launch_bounds__(gg::kThreads, 1) gram_tf32x3_kernel(
    const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int ntb,
    int symmetric, int64_t rows_per_chunk, int64_t nrows_total, const float *__restrict__ w,
    int mrows, int ncols, float *__restrict__ out, int64_t ldo, int64_t chunk_stride, Ctrl *ctrl) {
  using namespace tc;
  extern __shared__ __align__(1024) unsigned char gg_smem_raw[];
  unsigned char *smem = reinterpret_cast<unsigned char *>(
      (reinterpret_cast<uintptr_t>(gg_smem_raw) + 1023) & ~(uintptr_t)1023);
  // raw[3] = {A 16 KB, B 16 KB}; hilo[2] = {A_hi, A_lo, B_hi, B_lo} 16 KB each
  unsigned char *raw = smem;
  unsigned char *hilo = smem + gg::kRawStages * 2 * gg::kTileBytes;
  uint64_t *bars = reinterpret_cast<uint64_t *>(hilo + 2 * 4 * gg::kTileBytes);
  uint64_t *full = bars;                        // [kRawStages]
  uint64_t *rawfree = full + gg::kRawStages;    // [kRawStages]
  uint64_t *ready = rawfree + gg::kRawStages;   // [2]
  uint64_t *hfree = ready + 2;     // [2]
  uint64_t *accfull = hfree + 2;   // [2]
  uint64_t *accfree = accfull + 2; // [2]
  uint64_t *done = accfree + 2;    // [1]
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);
  int *abort_flag = reinterpret_cast<int *>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // output tile (ta, tb): symmetric -> tb >= ta enumerated row by row
  int ta = 0, tb = 0;
  {
    int t = blockIdx.x;
    if (symmetric) {
      int rowlen = ntb;
      while (t >= rowlen) {
        t -= rowlen;
        ++ta;
        --rowlen;
      }
      tb = ta + t;
    } else {
      ta = t / ntb;
      tb = t % ntb;
    }
  }
  const int a0 = ta * gt::BM, b0 = tb * gg::BN;
  const int npad = min(gg::BN, ((ncols - b0) + 31) / 32 * 32);
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t r1 = min64(nrows_total, r0 + rows_per_chunk);
  const int kblocks = r1 > r0 ? (int)((r1 - r0 + gt::BK - 1) / gt::BK) : 0;
  const int nseg = (kblocks + gg::kSeg - 1) / gg::kSeg;
  const int bbytes = npad * 128;
  // a diagonal tile of the unweighted symmetric Gram reads its B columns from
  // the A tile (with weights, A holds w_i A[i, :] and B must stay unweighted)
  const bool diag = symmetric && ta == tb && w == nullptr;
  const uint32_t raw_bytes = (uint32_t)(gt::kABytes + (diag ? 0 : bbytes));

  if (threadIdx.x == 0) {
    for (int s = 0; s < gg::kRawStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&rawfree[s], gg::kSplitThreads);
    }
    for (int s = 0; s < 2; ++s) {
      mbar_init(&ready[s], gg::kSplitThreads);
      mbar_init(&hfree[s], 1);
      mbar_init(&accfull[s], 1);
      mbar_init(&accfree[s], gg::kDrainThreads);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(256));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;
  volatile int *abortv = abort_flag;

  if (warp == 0) {
    if (lane == 0) {
      int issued = 0;
      for (int kb = 0; kb < kblocks; ++kb) {
        const int s = kb % gg::kRawStages;
        if (!mbar_wait(&rawfree[s], (uint32_t)(((kb / gg::kRawStages) & 1) ^ 1), abortv, ctrl)) break;
        unsigned char *rb = raw + (size_t)s * 2 * gg::kTileBytes;
        mbar_expect_tx(&full[s], raw_bytes);
        const int y = (int)(r0 + (int64_t)kb * gt::BK);
        for (int m = 0; m < 4; ++m) tma_load_2d(rb + m * 4096, &tmA, &full[s], a0 + 32 * m, y);
        if (!diag)
          for (int t = 0; t < npad / 32; ++t)
            tma_load_2d(rb + gg::kTileBytes + t * 4096, &tmB, &full[s], b0 + 32 * t, y);
        ++issued;
      }
      const int first = issued > gg::kRawStages ? issued - gg::kRawStages : 0;
      for (int q = first; q < issued; ++q)
        mbar_drain(&full[q % gg::kRawStages], (uint32_t)((q / gg::kRawStages) & 1), kTimeoutNs);
    }
  } else if (warp == 1) {
    if (lane == 0) {
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(npad >> 3) << 17) |
                             ((uint32_t)(gt::BM >> 4) << 24);
      bool ok = true;
      for (int kb = 0; kb < kblocks && ok; ++kb) {
        const int seg = kb / gg::kSeg, buf = seg & 1;
        const bool seg_first = (kb % gg::kSeg) == 0;
        const bool seg_last = ((kb % gg::kSeg) == gg::kSeg - 1) || (kb == kblocks - 1);
        if (seg_first) {
          // the drain warps must have emptied this accumulator (its use seg/2 - 1)
          if (!mbar_wait(&accfree[buf], (uint32_t)(((seg >> 1) & 1) ^ 1), abortv, ctrl)) {
            ok = false;
            break;
          }
          fence_after();
        }
        const int s = kb & 1;
        if (!mbar_wait(&ready[s], (uint32_t)((kb >> 1) & 1), abortv, ctrl)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t base = smem_u32(hilo + (size_t)s * 4 * gg::kTileBytes);
        const uint32_t ahi = base, alo = base + gg::kTileBytes;
        const uint32_t bhi = diag ? ahi : base + 2 * gg::kTileBytes;
        const uint32_t blo = diag ? alo : base + 3 * gg::kTileBytes;
        const uint32_t dt = tmem + (uint32_t)(buf * gg::BN);
#pragma unroll
        for (int kk = 0; kk < gt::BK / 8; ++kk) {
          const uint32_t acc = (!seg_first || kk) ? 1u : 0u;
          const uint64_t da_hi = sdesc2(ahi + kk * 32, 16, 1024);
          mma_tf32(dt, da_hi, sdesc2(bhi + kk * 32, 16, 1024), idesc, acc);
          mma_tf32(dt, da_hi, sdesc2(blo + kk * 32, 16, 1024), idesc, 1u);
          mma_tf32(dt, sdesc2(alo + kk * 32, 16, 1024), sdesc2(bhi + kk * 32, 16, 1024), idesc, 1u);
        }
        mma_commit(&hfree[s]);
        if (seg_last) mma_commit(&accfull[buf]);
      }
      // every issued MMA has completed before TMEM is released
      mma_commit(done);
      const uint64_t t0 = gtimer();
      while (!mbar_try_wait(done, 0u) && gtimer() - t0 < kTimeoutNs) {
      }
    }
  } else if (warp < 2 + gg::kSplitThreads / 32) {
    // ---------------- split warps: raw (MN boxes) -> transposed hi / lo
    const int t = threadIdx.x - 64;
    for (int kb = 0; kb < kblocks; ++kb) {
      const int s = kb & 1, rs = kb % gg::kRawStages;
      if (!mbar_wait(&full[rs], (uint32_t)((kb / gg::kRawStages) & 1), abortv, ctrl)) break;
      if (kb >= 2 && !mbar_wait(&hfree[s], (uint32_t)(((kb >> 1) - 1) & 1), abortv, ctrl)) break;
      const float *rawf = reinterpret_cast<const float *>(raw + (size_t)rs * 2 * gg::kTileBytes);
      float *hA = reinterpret_cast<float *>(hilo + (size_t)s * 4 * gg::kTileBytes);
      float *lA = hA + gg::kTileBytes / 4;
      float *hB = lA + gg::kTileBytes / 4;
      float *lB = hB + gg::kTileBytes / 4;
      const int64_t ibase = r0 + (int64_t)kb * gt::BK;
      // task (box, ic, j): the 4 x 4 block rows i = 4 ic .. 4 ic + 3, columns
      // 4 j .. 4 j + 3 of a raw box (16-byte chunk j of row i sits at chunk
      // j ^ (i % 8)), read as four float4, transposed in registers and
      // written as four hi and four lo float4: K-major row r = 32 m + 4 j + v,
      // K-chunk ic at chunk ic ^ (r % 8).  The 8 lanes of a quarter-warp take
      // ic = 0..7 with j = ic ^ g, so both their loads (chunks j ^ 4(ic & 1) ^ u)
      // and their stores (chunks ic ^ 4(j & 1) ^ v) fall on 8 distinct chunks:
      // no bank conflicts.
      const int ntask = (4 + (diag ? 0 : npad / 32)) * 64;
      for (int tau = t; tau < ntask; tau += gg::kSplitThreads) {
        const int box = tau >> 6, g = (tau >> 3) & 7, ic = tau & 7, j = ic ^ g;
        const bool isA = box < 4;
        const int m = isA ? box : box - 4;
        const float *bx = rawf + (isA ? 0 : gg::kTileBytes / 4) + m * 1024;
        float4 X[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int i = 4 * ic + u;
          X[u] = *reinterpret_cast<const float4 *>(bx + i * 32 + ((j ^ (i & 7)) << 2));
        }
        if (isA && w) {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int64_t gi = ibase + 4 * ic + u;
            const float wi = gi < nrows_total ? __ldg(w + gi) : 0.0f;
            X[u].x *= wi;
            X[u].y *= wi;
            X[u].z *= wi;
            X[u].w *= wi;
          }
        }
        float *dh = isA ? hA : hB;
        float *dl = isA ? lA : lB;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const float x0 = v == 0 ? X[0].x : v == 1 ? X[0].y : v == 2 ? X[0].z : X[0].w;
          const float x1 = v == 0 ? X[1].x : v == 1 ? X[1].y : v == 2 ? X[1].z : X[1].w;
          const float x2 = v == 0 ? X[2].x : v == 1 ? X[2].y : v == 2 ? X[2].z : X[2].w;
          const float x3 = v == 0 ? X[3].x : v == 1 ? X[3].y : v == 2 ? X[3].z : X[3].w;
          const float4 h = make_float4(tf32_rna(x0), tf32_rna(x1), tf32_rna(x2), tf32_rna(x3));
          const int r = 32 * m + 4 * j + v;
          const int off = r * 32 + ((ic ^ (r & 7)) << 2);
          *reinterpret_cast<float4 *>(dh + off) = h;
          *reinterpret_cast<float4 *>(dl + off) = make_float4(x0 - h.x, x1 - h.y, x2 - h.z, x3 - h.w);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(&rawfree[rs]);
      mbar_arrive(&ready[s]);
    }
  } else {
    // ---------------- drain warps: finished accumulators -> FP32 registers;
    // warp w reads TMEM lane quarter w % 4 and columns 64 h .. 64 h + 63,
    // h = (w - 10) / 4
    constexpr int DW = gg::BN / 2;
    const int ew = warp & 3;
    const int cb = DW * ((warp - 2 - gg::kSplitThreads / 32) >> 2);
    const int64_t r = a0 + 32 * ew + lane;
    float acc[DW];
#pragma unroll
    for (int c = 0; c < DW; ++c) acc[c] = 0.0f;
    bool ok = true;
    for (int seg = 0; seg < nseg; ++seg) {
      const int buf = seg & 1;
      if (!mbar_wait(&accfull[buf], (uint32_t)((seg >> 1) & 1), abortv, ctrl)) {
        ok = false;
        break;
      }
      fence_after();
#pragma unroll
      for (int c = 0; c < DW; c += 32) {
        if (cb + c < npad) {
          float v[32];
          tmem_ld32(tmem + ((uint32_t)(32 * ew) << 16) + (uint32_t)(buf * gg::BN + cb + c), v);
#pragma unroll
          for (int q = 0; q < 32; ++q) acc[c + q] += v[q];
        }
      }
      fence_before();
      mbar_arrive(&accfree[buf]);
    }
    if (r < mrows) {
      float *orow = out + (int64_t)blockIdx.y * chunk_stride + r * ldo + b0 + cb;
#pragma unroll
      for (int c = 0; c < DW; ++c)
        if (b0 + cb + c < ncols && (ok || kblocks == 0)) orow[c] = acc[c];
    }
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn2)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                   const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                   const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                   CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn2 encode_fn2() {
  static EncodeTiledFn2 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn2>(p);
  }
  return fn;
}

// 2-D FP32 tensor map over rows x cols (leading dimension ld floats),
// box {bx columns, by rows}, 128-byte swizzle.
static bool map_f32(CUtensorMap *tm, const float *ptr, int64_t rows, int64_t cols, int64_t ld, int bx,
                    int by) {
  EncodeTiledFn2 enc = encode_fn2();
  if (!enc) return false;
  if ((uintptr_t)ptr % 16 || (ld * 4) % 16) return false;
  cuuint64_t gdim[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t gstride[1] = {(cuuint64_t)ld * 4};
  cuuint32_t box[2] = {(cuuint32_t)bx, (cuuint32_t)by};
  cuuint32_t estr[2] = {1, 1};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(ptr), gdim, gstride, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

static size_t gemm_tc_smem(int npad) {
  int N0, N1;
  tall_halves(npad, &N0, &N1);
  const size_t stage = 2 * (size_t)gt::kABytes + 2 * (size_t)N0 * gt::BK * 4;
  return 1024 + gt::kStages * stage + 256;
}

bool tc_gemm_supported(int ncols) {
  const int npad = (ncols + 31) / 32 * 32;
  return npad <= gt::kMaxN && gemm_tc_smem(npad) <= 227 * 1024;
}

// Mt2 (2 npad x K): rows c < Kc of M^T split into TF32 hi (row c) and lo
// (row npad + c); rows Kc .. npad of both halves zero.
__global__ void split_mt_kernel(const float *__restrict__ M, int K, int Kc, int ldm, int npad,
                                float *__restrict__ Mt2) {
  const int64_t total = (int64_t)npad * K;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(q / K), a = (int)(q % K);
    const float x = c < Kc ? M[(int64_t)a * ldm + c] : 0.0f;
    const float h = tc::tf32_rna(x);
    Mt2[q] = h;
    Mt2[(int64_t)npad * K + q] = x - h;
  }
}

size_t tall_tc_scratch_floats(int K, int Kc) {
  const int npad = (Kc + 31) / 32 * 32;
  return (size_t)2 * npad * K;
}

// C[i, :Kc] = A[i, :K] M  (M K x Kc, leading dimension ldm); Mt2: scratch of
// tall_tc_scratch_floats(K, Kc) floats for the split M^T.
cudaError_t launch_tall_gemm_tc(const float *A, int64_t lda, int64_t n, int K, const float *M,
                                int ldm, int Kc, float *C, int64_t ldc, float *Mt2, Ctrl *ctrl,
                                cudaStream_t st) {
  if (n <= 0 || Kc <= 0) return cudaSuccess;
  const int npad = (Kc + 31) / 32 * 32;
  if (!tc_gemm_supported(Kc) || n > (int64_t)INT32_MAX - gt::BM) return cudaErrorInvalidValue;
  {
    ProfScope ps_(K_MISC, st);
    split_mt_kernel<<<(unsigned)min64(1024, ((int64_t)npad * K + 255) / 256), 256, 0, st>>>(
        M, K, Kc, ldm, npad, Mt2);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int N0, N1;
  tall_halves(npad, &N0, &N1);
  const int nkb = (K + gt::BK - 1) / gt::BK;
  const int64_t ntiles = (n + gt::BM - 1) / gt::BM;
  const int nhalf = N1 > 0 ? 2 : 1;
  const int vec4 = (ldc % 4 == 0 && (uintptr_t)C % 16 == 0) ? 1 : 0;
  const size_t smem = gemm_tc_smem(npad);
  CUtensorMap tmA;
  if (!map_f32(&tmA, A, n, K, lda, gt::BK, gt::BM)) return cudaErrorInvalidValue;
  ProfScope ps_(K_TALL_TC, st);
  // pairs of CTAs sharing each B stage, when the tiles are at least two
  if (ntiles >= 2 && sm_count() >= 2) {
    CUtensorMap tmB0, tmB1;
    if (!map_f32(&tmB0, Mt2, 2 * npad, K, K, gt::BK, N0 / 2)) return cudaErrorInvalidValue;
    if (!map_f32(&tmB1, Mt2, 2 * npad, K, K, gt::BK, N1 > 0 ? N1 / 2 : 16))
      return cudaErrorInvalidValue;
    auto kern = tall_tf32x3_kernel<true>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int64_t items = ((ntiles + 1) / 2) * nhalf;
    const int grid = 2 * (int)min64(items, (int64_t)(sm_count() / 2));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3(gt::kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 2;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, tmA, tmB0, tmB1, npad, nkb, ntiles, n, Kc, C, ldc, vec4, ctrl);
    if (e == cudaSuccess) return cudaSuccess;
    (void)cudaGetLastError();  // clusters unavailable: one CTA per work item below
  }
  CUtensorMap tmB0, tmB1;
  if (!map_f32(&tmB0, Mt2, 2 * npad, K, K, gt::BK, N0)) return cudaErrorInvalidValue;
  if (!map_f32(&tmB1, Mt2, 2 * npad, K, K, gt::BK, N1 > 0 ? N1 : 32)) return cudaErrorInvalidValue;
  auto kern = tall_tf32x3_kernel<false>;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int grid = (int)min64(ntiles * nhalf, (int64_t)sm_count());
  kern<<<grid, gt::kThreads, smem, st>>>(tmA, tmB0, tmB1, npad, nkb, ntiles, n, Kc, C, ldc, vec4,
                                         ctrl);
  return cudaGetLastError();
}

static void gram_tc_grid(int64_t n, int Ka, int Kb, bool symmetric, int *tiles, int *ntb,
                         int *chunks) {
  const int nta = (Ka + gt::BM - 1) / gt::BM;
  *ntb = (Kb + gg::BN - 1) / gg::BN;
  *tiles = symmetric ? (*ntb) * (*ntb + 1) / 2 : nta * (*ntb);
  int c = (sm_count() * 2) / *tiles;  // at most two full waves of one CTA per SM
  const int64_t maxc = (n + 4 * gt::BK - 1) / (4 * gt::BK);
  if (c > maxc) c = (int)maxc;
  if (c < 1) c = 1;
  *chunks = c;
}

size_t gram_tc_partial_floats(int64_t n, int Ka, int Kb) {
  int tiles, ntb, chunks;
  gram_tc_grid(n, Ka, Kb, false, &tiles, &ntb, &chunks);
  int t2, nb2, c2;
  gram_tc_grid(n, Ka, Kb, Ka == Kb, &t2, &nb2, &c2);
  if (c2 > chunks) chunks = c2;
  return (size_t)chunks * Ka * Kb;
}

// partial[c][a][b] = sum_{i in chunk c} w_i A[i, a] B[i, b]; C = sum_c partial (FP64).
cudaError_t launch_gram_tc(const float *A, int64_t lda, int Ka, const float *B, int64_t ldb, int Kb,
                           int64_t n, const float *w, bool symmetric, float *partial, double *C,
                           int ldc, Ctrl *ctrl, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (symmetric && Ka != Kb) return cudaErrorInvalidValue;
  int tiles, ntb, chunks;
  gram_tc_grid(n, Ka, Kb, symmetric, &tiles, &ntb, &chunks);
  int64_t rpc = (n + chunks - 1) / chunks;
  rpc = (rpc + gt::BK - 1) / gt::BK * gt::BK;  // chunks never share a 32-row k-block
  CUtensorMap tmA, tmB;
  if (!map_f32(&tmA, A, n, Ka, lda, 32, gt::BK)) return cudaErrorInvalidValue;
  if (!map_f32(&tmB, B, n, Kb, ldb, 32, gt::BK)) return cudaErrorInvalidValue;
  const size_t smem =
      1024 + (size_t)gg::kRawStages * 2 * gg::kTileBytes + (size_t)2 * 4 * gg::kTileBytes + 256;
  auto kern = gram_tf32x3_kernel;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  {
    ProfScope ps_(K_GRAM_TC, st);
    kern<<<dim3((unsigned)tiles, (unsigned)chunks), gg::kThreads, smem, st>>>(
        tmA, tmB, ntb, symmetric ? 1 : 0, rpc, n, w, Ka, Kb, partial, Kb, (int64_t)Ka * Kb, ctrl);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  return launch_gram_reduce(partial, Ka, Kb, chunks, symmetric ? gg::BN : 0, C, ldc, st);
}

}  // namespace sne
