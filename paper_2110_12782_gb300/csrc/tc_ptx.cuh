// Inline-PTX helpers for the tcgen05 / TMA / mbarrier kernels of sm_103a.
#pragma once

#include <cuda.h>

#include "sne_internal.cuh"

namespace sne {

namespace tc {

constexpr int BM = 128;
constexpr int BN = 256;
constexpr int BK = 64;                        // elements per k-block (128 bytes)
constexpr int kABlockBytes = BM * BK * 2;     // 16 KB
constexpr int kBStageBytes = BN * BK * 2;     // 32 KB
constexpr int kThreads = 192;
#ifndef SNE_SKETCH_EPI_WARPS
#define SNE_SKETCH_EPI_WARPS 16
#endif
// Fused sketch: TMA warp, MMA warp and kSketchEpiWarps epilogue warps (a
// multiple of 4: one TMEM lane quarter each, the columns of a tile split
// between the warps of a quarter).  With 18 warps a thread gets at most 96
// registers (the column data are broadcast by shuffles so that the epilogue
// fits); 8 epilogue warps (168 registers) hide less latency and run slower.
constexpr int kSketchEpiWarps = SNE_SKETCH_EPI_WARPS;
constexpr int kThreadsSketch = 64 + 32 * kSketchEpiWarps;
constexpr unsigned long long kTimeoutNs = 2000000000ull;

// Shared-memory descriptor with explicit byte offsets (128-byte swizzle).
// K-major: lbo unused, sbo = distance between 8-row groups.
// MN-major: lbo = distance between 128-byte MN chunks, sbo = distance between
// 8-row K groups.
__device__ __forceinline__ uint64_t sdesc2(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}
__device__ __forceinline__ void mma_tf32(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint64_t gtimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait; false on timeout (after limit_ns of %globaltimer) or when
// another role aborted.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                          Ctrl *ctrl, uint64_t limit_ns = kTimeoutNs) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = gtimer();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (gtimer() - t0 > limit_ns) {
      *abort_flag = 1;
      record_error(ctrl, SNE_ERR_TIMEOUT, W_TC);
      return false;
    }
  }
}
// Bounded wait that ignores the abort flag: for a CTA that is about to exit
// and must let its own copies and MMAs land first.
__device__ __forceinline__ void mbar_drain(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
  const uint64_t t0 = gtimer();
  while (!mbar_try_wait(bar, parity) && gtimer() - t0 < limit_ns) {
  }
}
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *tm, uint64_t *bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, "
      "%4}], [%2];" ::"r"(smem_u32(dst)),
      "l"(tm), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}
// Thread-block clusters: rank of this CTA, a barrier over every thread of
// every CTA of the cluster, a TMA load multicast to the CTAs of `mask` (the
// same shared-memory offset and mbarrier in each), and an MMA commit that
// arrives on the mbarrier at the same offset in each CTA of `mask`.
__device__ __forceinline__ uint32_t cluster_ctarank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cluster_sync_all() {
  asm volatile("barrier.cluster.arrive.release;\n\tbarrier.cluster.wait.acquire;" ::: "memory");
}
__device__ __forceinline__ void tma_load_2d_mc(void *dst, const CUtensorMap *tm, uint64_t *bar, int x,
                                               int y, uint16_t mask) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.multicast::cluster "
      "[%0], [%1, {%3, %4}], [%2], %5;" ::"r"(smem_u32(dst)),
      "l"(tm), "r"(smem_u32(bar)), "r"(x), "r"(y), "h"(mask)
      : "memory");
}
__device__ __forceinline__ void mma_commit_mc(uint64_t *bar, uint16_t mask) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], "
      "%1;" ::"r"(smem_u32(bar)),
      "h"(mask)
      : "memory");
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;             // leading byte offset (unused for swizzled K-major)
  d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
  d |= (uint64_t)1 << 46;             // descriptor version
  d |= (uint64_t)2 << 61;             // 128-byte swizzle
  return d;
}
__device__ __forceinline__ void mma_f16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.u32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// tcgen05.ld of 32 columns without the wait: several loads can be in flight
// before one tmem_wait_ld().
__device__ __forceinline__ void tmem_ld32_nw(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() {
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]),
        "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]),
        "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// p(t), t = r - 1/2, by Horner (coefficients c_8 .. c_0 of fit_log1p.py)
__device__ __forceinline__ float log1p_poly(float t) {
  float p = 5.232623778e-03f;
  p = fmaf(p, t, -8.574461564e-03f);
  p = fmaf(p, t, 1.158651151e-02f);
  p = fmaf(p, t, -2.022824623e-02f);
  p = fmaf(p, t, 3.663385287e-02f);
  p = fmaf(p, t, -6.771145016e-02f);
  p = fmaf(p, t, 1.326090842e-01f);
  p = fmaf(p, t, -2.885266542e-01f);
  return fmaf(p, t, 8.109301925e-01f);
}

// f of r = x - c0: trunc_log(x) = log1p(r) for r > 0, else 0; the identity r.
// For 0 <= r < 1, log1p(r) = r p(r - 1/2) with p the degree-8 polynomial
// fitted to log1p(r)/r on [0, 1] (fit_log1p.py: minimax relative error by
// iteratively reweighted least squares), which keeps the relative accuracy as
// r -> 0 and stays within 2e-7 relative in FP32 (Horner with fused
// multiply-adds); r <= 0 enters the polynomial as 0 and gives 0.  For r >= 1,
// log(1 + r) = ln 2 log2(1 + r) with the special function unit's base-2
// logarithm (lg2.approx), whose absolute error of about 2^-22 is below 2e-7 of
// log(1 + r) >= ln 2; the rounding of 1 + r moves log(1 + r) by at most 2^-24.
// Both sides are evaluated and selected (no divergence within a warp): about
// sixteen instructions, half of a full-range logf with its argument
// correction, and the base-2 logarithm runs on the otherwise idle MUFU pipe.
template <int F>
__device__ __forceinline__ float fr(float r) {
  if (F == SNE_F_TRUNC_LOG) {
    const float rs = fminf(fmaxf(r, 0.0f), 1.0f);
    const float small = log1p_poly(rs - 0.5f) * rs;
    float l2;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(l2) : "f"(1.0f + r));
    return r < 1.0f ? small : l2 * 0.693147182f;
  }
  return r;
}

}  // namespace tc

}  // namespace sne
