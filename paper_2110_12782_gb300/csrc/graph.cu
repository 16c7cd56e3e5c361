// Graph kernels: degrees and vol(G) (Sec. 2), the implicit SpMM with the
// modified Laplacian X = D^-a A D^-a (Alg. 5, Sec. 4.4 "Parallelization"),
// and CSR validation.
#include <cstdlib>

#include "sne_internal.cuh"

namespace sne {

__global__ void degrees_kernel(int64_t n, const int64_t *__restrict__ row_ptr,
                               const float *__restrict__ val, float *__restrict__ deg,
                               double *__restrict__ vol) {
  double local = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int64_t b = row_ptr[i], e = row_ptr[i + 1];
    float d;
    if (val == nullptr) {
      d = (float)(e - b);
    } else {
      double acc = 0.0;  // exact order-independent enough: per-row FP64 sum
      for (int64_t p = b; p < e; ++p) acc += (double)val[p];
      d = (float)acc;
    }
    deg[i] = d;
    local += (double)d;
  }
  for (int o = 16; o > 0; o >>= 1) local += __shfl_xor_sync(0xffffffffu, local, o);
  __shared__ double ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = local;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? ws[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (threadIdx.x == 0) atomicAdd(vol, v);
  }
}

cudaError_t launch_degrees(const sne_csr &g, float *deg, double *vol, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(vol, 0, sizeof(double), st);
  if (e != cudaSuccess) return e;
  if (g.n <= 0) return cudaSuccess;
  int64_t blocks = (g.n + 255) / 256;
  if (blocks > sm_count() * 8) blocks = sm_count() * 8;
  ProfScope ps_(K_MISC, st);
  degrees_kernel<<<(unsigned)blocks, 256, 0, st>>>(g.n, g.row_ptr, g.val, deg, vol);
  return cudaGetLastError();
}

__global__ void degree_power_kernel(const float *__restrict__ deg, int64_t n, float beta, float scale,
                                    float *__restrict__ out) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const float d = deg[i];
    out[i] = d > 0.0f ? scale * powf(d, beta) : 0.0f;
  }
}

cudaError_t launch_degree_power(const float *deg, int64_t n, double beta, float *out, float scale,
                                cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > sm_count() * 8) blocks = sm_count() * 8;
  ProfScope ps_(K_MISC, st);
  degree_power_kernel<<<(unsigned)blocks, 256, 0, st>>>(deg, n, (float)beta, scale, out);
  return cudaGetLastError();
}

// L2 priorities of the SpMM's loads and stores (PTX createpolicy / cache_hint).
__device__ __forceinline__ uint64_t l2_policy_normal() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint64_t l2_policy_first() {
  uint64_t pol;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ float4 ld_nc_f4(const float4 *ptr, uint64_t pol) {
  float4 v;
  asm("ld.global.nc.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(ptr), "l"(pol));
  return v;
}
__device__ __forceinline__ float ld_nc_f32(const float *ptr, uint64_t pol) {
  float v;
  asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(ptr), "l"(pol));
  return v;
}
__device__ __forceinline__ int32_t ld_nc_s32(const int32_t *ptr, uint64_t pol) {
  int32_t v;
  asm("ld.global.nc.L2::cache_hint.s32 %0, [%1], %2;" : "=r"(v) : "l"(ptr), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_f4(float4 *ptr, float4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(ptr), "f"(v.x),
               "f"(v.y), "f"(v.z), "f"(v.w), "l"(pol)
               : "memory");
}

// Y[i, :] = s_i * sum_{p in row i} w_p s_{col_p} B[col_p, :],  s = d^-a.
// One warp per row; each lane owns VPL float4 column groups of the row; the
// row's (col, weight) pairs are fetched 32 at a time and broadcast by shuffle.
// On power-law graphs the dense operand does not fit in L2 and the kernel is
// bound by the latency of its gathers: the per-nonzero weights come
// precomputed (one dependent load less) and two blocks stay resident per SM.
// Row j of B is gathered deg(j) times, so L2 holds the rows of the vertices of
// largest degree best: those rows (weight bits below *hot) load with the
// normal priority, while the other rows, the CSR arrays and Y go evict-first
// and do not push them out.
template <int VPL>
__global__ void __launch_bounds__(256, 2) spmm_vec4_kernel(
    int64_t n, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
    const float *__restrict__ val, const float *__restrict__ dpow, const float *__restrict__ wnz,
    const float *__restrict__ B, int64_t ldb, int32_t nvec, float *__restrict__ Y, int64_t ldy,
    const uint32_t *__restrict__ hot) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  const uint64_t pol_keep = l2_policy_normal(), pol_stream = l2_policy_first();
  const uint32_t thr = hot ? *hot : 0xffffffffu;
  float4 acc[VPL];
#pragma unroll
  for (int v = 0; v < VPL; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
  const int64_t beg = row_ptr[row], end = row_ptr[row + 1];
  for (int64_t p0 = beg; p0 < end; p0 += 32) {
    const int64_t p = p0 + lane;
    int32_t c = 0;
    float w = 0.f;
    if (p < end) {
      c = ld_nc_s32(col + p, pol_stream);
      w = wnz ? ld_nc_f32(wnz + p, pol_stream) : dpow[c] * (val ? val[p] : 1.0f);
    }
    const int cnt = (int)min64(32, end - p0);
    int t = 0;
    for (; t + 2 <= cnt; t += 2) {
      const int32_t c0 = __shfl_sync(0xffffffffu, c, t);
      const int32_t c1 = __shfl_sync(0xffffffffu, c, t + 1);
      const float w0 = __shfl_sync(0xffffffffu, w, t);
      const float w1 = __shfl_sync(0xffffffffu, w, t + 1);
      const uint64_t pl0 = __float_as_uint(w0) < thr ? pol_keep : pol_stream;
      const uint64_t pl1 = __float_as_uint(w1) < thr ? pol_keep : pol_stream;
      const float4 *r0 = reinterpret_cast<const float4 *>(B + (int64_t)c0 * ldb);
      const float4 *r1 = reinterpret_cast<const float4 *>(B + (int64_t)c1 * ldb);
#pragma unroll
      for (int v = 0; v < VPL; ++v) {
        const int q = lane + 32 * v;
        if (q < nvec) {
          const float4 x0 = ld_nc_f4(r0 + q, pl0);
          const float4 x1 = ld_nc_f4(r1 + q, pl1);
          acc[v].x += w0 * x0.x + w1 * x1.x;
          acc[v].y += w0 * x0.y + w1 * x1.y;
          acc[v].z += w0 * x0.z + w1 * x1.z;
          acc[v].w += w0 * x0.w + w1 * x1.w;
        }
      }
    }
    for (; t < cnt; ++t) {
      const int32_t c0 = __shfl_sync(0xffffffffu, c, t);
      const float w0 = __shfl_sync(0xffffffffu, w, t);
      const uint64_t pl0 = __float_as_uint(w0) < thr ? pol_keep : pol_stream;
      const float4 *r0 = reinterpret_cast<const float4 *>(B + (int64_t)c0 * ldb);
#pragma unroll
      for (int v = 0; v < VPL; ++v) {
        const int q = lane + 32 * v;
        if (q < nvec) {
          const float4 x0 = ld_nc_f4(r0 + q, pl0);
          acc[v].x += w0 * x0.x;
          acc[v].y += w0 * x0.y;
          acc[v].z += w0 * x0.z;
          acc[v].w += w0 * x0.w;
        }
      }
    }
  }
  const float si = dpow[row];
  float4 *yr = reinterpret_cast<float4 *>(Y + row * ldy);
#pragma unroll
  for (int v = 0; v < VPL; ++v) {
    const int q = lane + 32 * v;
    if (q < nvec)
      st_f4(yr + q, make_float4(si * acc[v].x, si * acc[v].y, si * acc[v].z, si * acc[v].w),
            pol_stream);
  }
}

// Column-panel SpMM for operands larger than L2: Y[:, panel] = X B[:, panel]
// for P panels of nqp float4 columns each, one panel after the other
// (blockIdx.y; the hardware dispatches the CTAs of one panel before the next),
// so that the L2 holds P times as many rows of the panel as of whole rows:
// a row j of B is gathered deg(j) times, and on power-law graphs the share of
// those gathers that land on the rows L2 keeps grows with the number of rows
// it keeps.  The CSR arrays are read once per panel.  One warp per row; the 32
// lanes form G = 32 / L groups of L lanes, each group gathering the panel
// segment of a different nonzero (V float4 per lane, two nonzeros per group in
// flight); the groups' partial sums are added by shuffles at the end of the
// row.
template <int L, int V>
__global__ void __launch_bounds__(256) spmm_panel_kernel(
    int64_t n, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
    const float *__restrict__ val, const float *__restrict__ dpow, const float *__restrict__ wnz,
    const float *__restrict__ B, int64_t ldb, int nq, int nqp, float *__restrict__ Y, int64_t ldy,
    const uint32_t *__restrict__ hot) {
  constexpr int G = 32 / L;
  const int lane = threadIdx.x & 31;
  const int grp = lane / L, sub = lane % L;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  const uint64_t pol_keep = l2_policy_normal(), pol_stream = l2_policy_first();
  const uint32_t thr = hot ? *hot : 0xffffffffu;
  const int q0 = blockIdx.y * nqp;
  const int qn = min(nqp, nq - q0);
  const float4 *Bp = reinterpret_cast<const float4 *>(B) + q0;  // row j at Bp + j * ldb / 4
  const int64_t ldb4 = ldb / 4;
  float4 acc[V];
#pragma unroll
  for (int v = 0; v < V; ++v) acc[v] = make_float4(0.f, 0.f, 0.f, 0.f);
  const int64_t beg = row_ptr[row], end = row_ptr[row + 1];
  for (int64_t p0 = beg; p0 < end; p0 += 32) {
    const int64_t p = p0 + lane;
    int32_t c = 0;
    float w = 0.f;
    if (p < end) {
      c = ld_nc_s32(col + p, pol_stream);
      w = wnz ? ld_nc_f32(wnz + p, pol_stream) : dpow[c] * (val ? val[p] : 1.0f);
    }
    const int cnt = (int)min64(32, end - p0);
    for (int t = 0; t < cnt; t += 2 * G) {
      const int ta = t + grp, tb = t + G + grp;  // both < 32
      const int32_t ca = __shfl_sync(0xffffffffu, c, ta);
      const int32_t cb = __shfl_sync(0xffffffffu, c, tb);
      const float wa = __shfl_sync(0xffffffffu, w, ta);
      const float wb = __shfl_sync(0xffffffffu, w, tb);
      const bool va = ta < cnt, vb = tb < cnt;
      const uint64_t pa = __float_as_uint(wa) < thr ? pol_keep : pol_stream;
      const uint64_t pb = __float_as_uint(wb) < thr ? pol_keep : pol_stream;
      const float4 *ra = Bp + (int64_t)ca * ldb4;
      const float4 *rb = Bp + (int64_t)cb * ldb4;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        const int q = sub + L * v;
        if (q < qn) {
          const float4 xa = va ? ld_nc_f4(ra + q, pa) : make_float4(0.f, 0.f, 0.f, 0.f);
          const float4 xb = vb ? ld_nc_f4(rb + q, pb) : make_float4(0.f, 0.f, 0.f, 0.f);
          acc[v].x += wa * xa.x + wb * xb.x;
          acc[v].y += wa * xa.y + wb * xb.y;
          acc[v].z += wa * xa.z + wb * xb.z;
          acc[v].w += wa * xa.w + wb * xb.w;
        }
      }
    }
  }
#pragma unroll
  for (int v = 0; v < V; ++v) {
#pragma unroll
    for (int o = L; o < 32; o <<= 1) {
      acc[v].x += __shfl_xor_sync(0xffffffffu, acc[v].x, o);
      acc[v].y += __shfl_xor_sync(0xffffffffu, acc[v].y, o);
      acc[v].z += __shfl_xor_sync(0xffffffffu, acc[v].z, o);
      acc[v].w += __shfl_xor_sync(0xffffffffu, acc[v].w, o);
    }
  }
  if (grp == 0) {
    const float si = dpow[row];
    float4 *yr = reinterpret_cast<float4 *>(Y + row * ldy) + q0;
#pragma unroll
    for (int v = 0; v < V; ++v) {
      const int q = sub + L * v;
      if (q < qn)
        st_f4(yr + q, make_float4(si * acc[v].x, si * acc[v].y, si * acc[v].z, si * acc[v].w),
              pol_stream);
    }
  }
}

// Scalar fallback for widths that are not a multiple of 4 (or unaligned).
__global__ void __launch_bounds__(256) spmm_scalar_kernel(
    int64_t n, const int64_t *__restrict__ row_ptr, const int32_t *__restrict__ col,
    const float *__restrict__ val, const float *__restrict__ dpow, const float *__restrict__ B,
    int64_t ldb, int32_t ncols, float *__restrict__ Y, int64_t ldy) {
  const int lane = threadIdx.x & 31;
  const int64_t row = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (row >= n) return;
  const int64_t beg = row_ptr[row], end = row_ptr[row + 1];
  const float si = dpow[row];
  for (int c0 = 0; c0 < ncols; c0 += 32 * 8) {
    float acc[8];
#pragma unroll
    for (int v = 0; v < 8; ++v) acc[v] = 0.f;
    for (int64_t p = beg; p < end; ++p) {
      const int32_t c = col[p];
      const float w = dpow[c] * (val ? val[p] : 1.0f);
      const float *br = B + (int64_t)c * ldb;
#pragma unroll
      for (int v = 0; v < 8; ++v) {
        const int q = c0 + lane + 32 * v;
        if (q < ncols) acc[v] += w * br[q];
      }
    }
#pragma unroll
    for (int v = 0; v < 8; ++v) {
      const int q = c0 + lane + 32 * v;
      if (q < ncols) Y[row * ldy + q] = si * acc[v];
    }
  }
}

__global__ void spmm_weights_kernel(int64_t nnz, const int32_t *__restrict__ col,
                                    const float *__restrict__ val, const float *__restrict__ dpow,
                                    float *__restrict__ wnz) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz; p += stride)
    wnz[p] = dpow[col[p]] * (val ? val[p] : 1.0f);
}

cudaError_t launch_spmm_weights(const sne_csr &g, const float *dpow, float *wnz, cudaStream_t st) {
  if (g.nnz <= 0) return cudaSuccess;
  ProfScope ps_(K_MISC, st);
  spmm_weights_kernel<<<(unsigned)min64(sm_count() * 16, (g.nnz + 255) / 256), 256, 0, st>>>(
      g.nnz, g.col_idx, g.val, dpow, wnz);
  return cudaGetLastError();
}

// The keep bound: a strided sample of kHotSample values of d^-a, sorted
// (bitonic, one CTA); the bound is the sample's quantile at the fraction of
// vertices whose rows fit kSpmmKeepBytes, so that weights strictly below it
// (the largest degrees) are kept.  With weighted edges the per-nonzero weight
// val_p d_j^-a only approximates the degree order, which moves rows between
// the two L2 classes and never changes a result.
constexpr int kHotSample = 2048;
constexpr int64_t kSpmmKeepBytes = 80ll << 20;  // of the 129 MB L2

__global__ void __launch_bounds__(1024) spmm_hot_threshold_kernel(const float *__restrict__ dpow,
                                                                   int64_t n, int64_t keep_rows,
                                                                   Ctrl *ctrl) {
  __shared__ uint32_t sv[kHotSample];
  const int tid = threadIdx.x;
  if (keep_rows >= n) {
    if (tid == 0) ctrl->hot_bits = 0xffffffffu;
    return;
  }
  // d^-a = 0 marks an isolated vertex, whose row is never gathered: it sorts
  // last so that it takes no place in the kept set
  for (int i = tid; i < kHotSample; i += blockDim.x) {
    const uint32_t b = __float_as_uint(dpow[(int64_t)((double)i * (double)n / kHotSample)]);
    sv[i] = b == 0u ? 0xffffffffu : b;
  }
  __syncthreads();
  for (int k = 2; k <= kHotSample; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < kHotSample; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const uint32_t a = sv[i], b = sv[l];
          if ((a > b) == ((i & k) == 0)) {
            sv[i] = b;
            sv[l] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  if (tid == 0) {
    const int at = (int)((double)keep_rows / (double)n * kHotSample);  // < kHotSample
    ctrl->hot_bits = sv[at < 0 ? 0 : at];
  }
}

cudaError_t launch_spmm_hot_threshold(const float *dpow, int64_t n, int64_t row_bytes, Ctrl *ctrl,
                                      cudaStream_t st) {
  if (n <= 0 || row_bytes <= 0) return cudaSuccess;
  ProfScope ps_(K_MISC, st);
  spmm_hot_threshold_kernel<<<1, 1024, 0, st>>>(dpow, n, kSpmmKeepBytes / row_bytes, ctrl);
  return cudaGetLastError();
}

// Number of column panels of the SpMM (1: whole rows at once).  Operands of
// at most kSpmmPanelFromBytes use one panel; above, SNE_SPMM_PANELS (1, 2, 4
// or 8) when set, else kSpmmPanelsDefault.
constexpr double kSpmmPanelFromBytes = 256.0 * 1024 * 1024;
constexpr int kSpmmPanelsDefault = 1;
int spmm_panels(int64_t n, int32_t ncols) {
  if ((double)n * ncols * 4.0 <= kSpmmPanelFromBytes) return 1;
  static int env = -1;
  if (env < 0) {
    const char *v = getenv("SNE_SPMM_PANELS");
    env = 0;
    if (v && (v[0] == '1' || v[0] == '2' || v[0] == '4' || v[0] == '8') && v[1] == 0) env = v[0] - '0';
  }
  return env > 0 ? env : kSpmmPanelsDefault;
}

// Bytes of one gathered row segment when the SpMM runs with spmm_panels():
// the row size the L2 keep bound is computed for.
int64_t spmm_row_bytes(int64_t n, int32_t ncols) {
  const int P = spmm_panels(n, ncols);
  const int nq = (ncols + 3) / 4;
  return (int64_t)16 * ((nq + P - 1) / P);
}

cudaError_t launch_spmm(const sne_csr &g, const float *dpow, const float *wnz, const float *B,
                        int64_t ldb, int32_t ncols, float *Y, int64_t ldy, cudaStream_t st,
                        const uint32_t *hot) {
  if (g.n <= 0 || ncols <= 0) return cudaSuccess;

  ProfScope ps_(K_SPMM, st);
  const unsigned blocks = (unsigned)((g.n + 7) / 8);
  const bool vec = (ncols % 4 == 0) && (ldb % 4 == 0) && (ldy % 4 == 0) &&
                   ((uintptr_t)B % 16 == 0) && ((uintptr_t)Y % 16 == 0);
  const int nvec = ncols / 4;
  // operands beyond L2: column panels (lanes per nonzero L and float4 per lane
  // V chosen for the panel width, at most 4 float4 per lane)
  const int P = vec ? spmm_panels(g.n, ncols) : 1;
  if (P > 1) {
    const int nqp = (nvec + P - 1) / P;
    const int L = nqp <= 32 ? 8 : (nqp <= 64 ? 16 : 32);
    const int V = (nqp + L - 1) / L;
    const dim3 grid(blocks, (unsigned)((nvec + nqp - 1) / nqp));
#define SNE_PANEL(LV, VV)                                                                    \
  spmm_panel_kernel<LV, VV><<<grid, 256, 0, st>>>(g.n, g.row_ptr, g.col_idx, g.val, dpow, wnz, B, \
                                                  ldb, nvec, nqp, Y, ldy, hot)
    if (V > 4) return cudaErrorInvalidValue;
    if (L == 8) {
      if (V == 1) SNE_PANEL(8, 1); else if (V == 2) SNE_PANEL(8, 2); else if (V == 3) SNE_PANEL(8, 3); else SNE_PANEL(8, 4);
    } else if (L == 16) {
      if (V == 1) SNE_PANEL(16, 1); else if (V == 2) SNE_PANEL(16, 2); else if (V == 3) SNE_PANEL(16, 3); else SNE_PANEL(16, 4);
    } else {
      if (V == 1) SNE_PANEL(32, 1); else if (V == 2) SNE_PANEL(32, 2); else if (V == 3) SNE_PANEL(32, 3); else SNE_PANEL(32, 4);
    }
#undef SNE_PANEL
    return cudaGetLastError();
  }
  if (vec && nvec <= 32 * 12) {
    const int vpl = (nvec + 31) / 32;
#define SNE_SPMM_CASE(V)                                                                     \
  case V:                                                                                    \
    spmm_vec4_kernel<V><<<blocks, 256, 0, st>>>(g.n, g.row_ptr, g.col_idx, g.val, dpow, wnz, B, \
                                                ldb, nvec, Y, ldy, hot);                     \
    break;
    switch (vpl) {
      SNE_SPMM_CASE(1)
      SNE_SPMM_CASE(2)
      SNE_SPMM_CASE(3)
      SNE_SPMM_CASE(4)
      SNE_SPMM_CASE(5)
      SNE_SPMM_CASE(6)
      SNE_SPMM_CASE(7)
      SNE_SPMM_CASE(8)
      SNE_SPMM_CASE(9)
      SNE_SPMM_CASE(10)
      SNE_SPMM_CASE(11)
      SNE_SPMM_CASE(12)
      default:
        break;
    }
#undef SNE_SPMM_CASE
  } else {
    spmm_scalar_kernel<<<blocks, 256, 0, st>>>(g.n, g.row_ptr, g.col_idx, g.val, dpow, B, ldb, ncols,
                                               Y, ldy);
  }
  return cudaGetLastError();
}

// CSR validation: row_ptr[0] = 0, nondecreasing, row_ptr[n] = nnz; columns in
// range, strictly increasing within a row, no self-loop; every (i, j, w) has
// its mirror (j, i, w).
__global__ void validate_kernel(int64_t n, int64_t nnz, const int64_t *__restrict__ row_ptr,
                                const int32_t *__restrict__ col, const float *__restrict__ val,
                                Ctrl *ctrl) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int64_t b = row_ptr[i], e = row_ptr[i + 1];
    bool bad = (b > e) || (b < 0) || (e > nnz) || (i == 0 && b != 0) || (i == n - 1 && e != nnz);
    if (!bad) {
      for (int64_t p = b; p < e; ++p) {
        const int32_t j = col[p];
        if (j < 0 || j >= n || j == i || (p > b && col[p - 1] >= j)) {
          bad = true;
          break;
        }
        // mirror (j, i): binary search in row j
        int64_t lo = row_ptr[j], hi = row_ptr[j + 1] - 1;
        if (lo < 0 || hi >= nnz) {
          bad = true;
          break;
        }
        bool found = false;
        while (lo <= hi) {
          const int64_t mid = (lo + hi) >> 1;
          const int32_t cm = col[mid];
          if (cm == i) {
            found = (val == nullptr) || (val[mid] == val[p]);
            break;
          }
          if (cm < i) lo = mid + 1;
          else hi = mid - 1;
        }
        if (!found) {
          bad = true;
          break;
        }
      }
    }
    if (bad) record_error(ctrl, SNE_ERR_GRAPH, W_VALIDATE);
  }
}

cudaError_t launch_validate(const sne_csr &g, Ctrl *ctrl, cudaStream_t st) {
  if (g.n <= 0) return cudaSuccess;
  int64_t blocks = (g.n + 255) / 256;
  if (blocks > sm_count() * 8) blocks = sm_count() * 8;
  ProfScope ps_(K_MISC, st);
  validate_kernel<<<(unsigned)blocks, 256, 0, st>>>(g.n, g.nnz, g.row_ptr, g.col_idx, g.val, ctrl);
  return cudaGetLastError();
}

}  // namespace sne
