// Fused reconstruct + f + sparse-sign contraction (Eq. 4, Alg. 4 lines 4 and
// 7), FP32 SIMT form, and the signed gathers O^T Y' and O^T Q.
//
// The sparse-sign matrix is kept as its list of (column, slot) nonzeros: entry
// e = c*z + t has row idx[e] and sign[e].  The kernel evaluates one column of
// L R per nonzero, B[e, :] = R(:, idx[e])^T, so that
//   out[i, c] = sv * sum_{t<z} sign[c*z+t] * f(rs_i * <A[i, :], B[c*z+t, :]>)
// is a sum over z consecutive evaluated columns.  This equals
// f(L R(:, p)) S(p, :) of Eq. 4 exactly: duplicated coordinates only repeat
// an evaluation.  M-hat is never stored.
#include "sne_internal.cuh"

namespace sne {

constexpr int kFM = 64;    // rows per CTA
constexpr int kFN = 128;   // evaluated columns per CTA
constexpr int kFK = 16;    // k step

template <int F>
__device__ __forceinline__ float apply_f(float x) {
  if (F == SNE_F_TRUNC_LOG) return x > 1.0f ? logf(x) : 0.0f;
  return x;
}

template <int F>
__global__ void __launch_bounds__(256) fused_sketch_f32_kernel(
    const float *__restrict__ A, int64_t lda, const int32_t *__restrict__ ridx,
    const int32_t *__restrict__ nrows_dev, int64_t nrows_max, int32_t k,
    const float *__restrict__ rs, const float *__restrict__ rs_lo, const float *__restrict__ B,
    const int8_t *__restrict__ sign, int32_t cols_out, int32_t z, float sv,
    float *__restrict__ out, int64_t ldo) {
  __shared__ __align__(16) float As[kFK][kFM + 4];
  __shared__ __align__(16) float Bs[kFK][kFN + 4];
  __shared__ float Fs[kFM][kFN + 1];
  const int64_t nrows = nrows_dev ? (int64_t)(*nrows_dev) : nrows_max;
  const int64_t i0 = (int64_t)blockIdx.x * kFM;
  if (i0 >= nrows) return;
  const int cpt = kFN / z;            // output columns per CTA
  const int c_begin = blockIdx.y * cpt;
  const int e_begin = c_begin * z;    // first evaluated column
  const int e_count = min(cpt, cols_out - c_begin) * z;
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;  // rows ty*4.., evaluated columns tx*8..
  float acc[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  for (int k0 = 0; k0 < k; k0 += kFK) {
#pragma unroll
    for (int q = 0; q < (kFM * kFK) / 256; ++q) {
      const int lin = tid + 256 * q;
      const int r = lin / kFK, kk = lin % kFK;
      const int64_t i = i0 + r;
      float v = 0.f;
      if (i < nrows && k0 + kk < k) {
        const int64_t src = ridx ? (int64_t)ridx[i] : i;
        v = A[src * lda + k0 + kk];
      }
      As[kk][r] = v;
    }
#pragma unroll
    for (int q = 0; q < (kFN * kFK) / 256; ++q) {
      const int lin = tid + 256 * q;
      const int c = lin / kFK, kk = lin % kFK;
      float v = 0.f;
      if (c < e_count && k0 + kk < k) v = B[(int64_t)(e_begin + c) * k + k0 + kk];
      Bs[kk][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kFK; ++kk) {
      const float4 a = *reinterpret_cast<const float4 *>(&As[kk][ty * 4]);
      const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 8]);
      const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[kk][tx * 8 + 4]);
      const float av[4] = {a.x, a.y, a.z, a.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
  // epilogue: scale, f, sign -> shared; then segmented sums over z columns
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t row = i0 + ty * 4 + i;
    float s = 0.f, s_lo = 0.f;
    if (row < nrows) {
      const int64_t src = ridx ? ridx[row] : row;
      s = rs[src];
      if (rs_lo) s_lo = rs_lo[src];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = tx * 8 + j;
      float v = 0.f;
      // the scale is the pair s + s_lo, so the only rounding of x is its own
      if (c < e_count) v = (float)sign[e_begin + c] * apply_f<F>(fmaf(s, acc[i][j], s_lo * acc[i][j]));
      Fs[ty * 4 + i][c] = v;
    }
  }
  __syncthreads();
  const int ncol = e_count / z;
  for (int q = tid; q < kFM * cpt; q += 256) {
    const int r = q / cpt, c = q % cpt;
    const int64_t row = i0 + r;
    if (c >= ncol || row >= nrows) continue;
    float sum = 0.f;
    for (int t = 0; t < z; ++t) sum += Fs[r][c * z + t];
    out[row * ldo + c_begin + c] = sv * sum;
  }
}

cudaError_t launch_fused_sketch_f32(const float *A, int64_t lda, const int32_t *ridx,
                                    const int32_t *nrows_dev, int64_t nrows, int32_t k,
                                    const float *rs, const float *rs_lo, const float *B,
                                    const int8_t *sign, int32_t cols_out, int32_t z, float sv,
                                    int32_t f, float *out, int64_t ldo, cudaStream_t st) {
  if (nrows <= 0 || cols_out <= 0) return cudaSuccess;
  if (z <= 0 || z > kFN) return cudaErrorInvalidValue;
  const int cpt = kFN / z;
  dim3 grid((unsigned)((nrows + kFM - 1) / kFM), (unsigned)((cols_out + cpt - 1) / cpt));
  ProfScope ps_(K_FUSED, st);
  if (f == SNE_F_TRUNC_LOG)
    fused_sketch_f32_kernel<SNE_F_TRUNC_LOG><<<grid, 256, 0, st>>>(
        A, lda, ridx, nrows_dev, nrows, k, rs, rs_lo, B, sign, cols_out, z, sv, out, ldo);
  else
    fused_sketch_f32_kernel<SNE_F_IDENTITY><<<grid, 256, 0, st>>>(
        A, lda, ridx, nrows_dev, nrows, k, rs, rs_lo, B, sign, cols_out, z, sv, out, ldo);
  return cudaGetLastError();
}

// out[c, :] = sv * sum_t sign[c*z+t] * In[idx[c*z+t], :]  (one CTA per output row)
__global__ void signed_gather_sum_kernel(const float *__restrict__ In, int64_t ldi, int32_t width,
                                         const int32_t *__restrict__ idx,
                                         const int8_t *__restrict__ sign, int32_t z, float sv,
                                         float *__restrict__ out, int64_t ldo) {
  const int c = blockIdx.x;
  for (int q = threadIdx.x; q < width; q += blockDim.x) {
    float s = 0.f;
    for (int t = 0; t < z; ++t) {
      const int64_t e = (int64_t)c * z + t;
      s += (float)sign[e] * In[(int64_t)idx[e] * ldi + q];
    }
    out[(int64_t)c * ldo + q] = sv * s;
  }
}

cudaError_t launch_signed_gather_sum(const float *In, int64_t ldi, int32_t width, const int32_t *idx,
                                     const int8_t *sign, int32_t cols, int32_t z, float sv,
                                     float *out, int64_t ldo, cudaStream_t st) {
  if (cols <= 0 || width <= 0) return cudaSuccess;
  ProfScope ps_(K_GATHER, st);
  signed_gather_sum_kernel<<<cols, 256, 0, st>>>(In, ldi, width, idx, sign, z, sv, out, ldo);
  return cudaGetLastError();
}

// R'(:, j)^T for the gathered vertices j = idx[i] (Eq. 11):
//   out[i, :] = a_j U[j, :] (C_hi + C_lo)^T,  a_j = deg_j^beta in FP64 (0 if deg_j = 0).
// C^T is carried as a pair of FP32 matrices so that its rounding, which every
// column of R' would otherwise share, cancels; the sums over the k terms are
// FP32 FMA chains, and each output is rounded to FP32 once.
constexpr int kRpRows = 8;
__global__ void __launch_bounds__(256) rprime_rows_kernel(
    const float *__restrict__ U, int32_t k, const int32_t *__restrict__ idx, int32_t count,
    const float *__restrict__ CThi, const float *__restrict__ CTlo, const float *__restrict__ deg,
    double beta, float *__restrict__ out) {
  extern __shared__ float us[];  // kRpRows x k
  const int i0 = blockIdx.x * kRpRows;
  const int rows = min(kRpRows, count - i0);
  for (int e = threadIdx.x; e < kRpRows * k; e += blockDim.x) {
    const int r = e / k, a = e % k;
    us[e] = r < rows ? U[(int64_t)idx[i0 + r] * k + a] : 0.f;
  }
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    float hi[kRpRows], lo[kRpRows];
#pragma unroll
    for (int r = 0; r < kRpRows; ++r) hi[r] = lo[r] = 0.f;
    for (int a = 0; a < k; ++a) {
      const float ch = CThi[(int64_t)a * k + c], cl = CTlo[(int64_t)a * k + c];
#pragma unroll
      for (int r = 0; r < kRpRows; ++r) {
        const float u = us[r * k + a];
        hi[r] = fmaf(u, ch, hi[r]);
        lo[r] = fmaf(u, cl, lo[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < kRpRows; ++r) {
      if (r >= rows) break;
      const float dj = deg[idx[i0 + r]];
      const double aj = dj > 0.f ? pow((double)dj, beta) : 0.0;
      out[(int64_t)(i0 + r) * k + c] = (float)(aj * ((double)hi[r] + (double)lo[r]));
    }
  }
}

cudaError_t launch_rprime_rows(const float *U, int32_t k, const int32_t *idx, int32_t count,
                               const float *CThi, const float *CTlo, const float *deg, double beta,
                               float *out, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const size_t smem = (size_t)kRpRows * k * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(rprime_rows_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  ProfScope ps_(K_TALL_GEMM, st);
  rprime_rows_kernel<<<(count + kRpRows - 1) / kRpRows, 256, smem, st>>>(U, k, idx, count, CThi,
                                                                        CTlo, deg, beta, out);
  return cudaGetLastError();
}

// FP64 version (FP32 input rows, FP64 sums): out[c, :] = sv * sum_t sign * In[idx, :]
__global__ void signed_gather_sum64_kernel(const float *__restrict__ In, int64_t ldi, int32_t width,
                                           const int32_t *__restrict__ idx,
                                           const int8_t *__restrict__ sign, int32_t z, double sv,
                                           double *__restrict__ out, int64_t ldo) {
  const int c = blockIdx.x;
  for (int q = threadIdx.x; q < width; q += blockDim.x) {
    double s = 0.0;
    for (int t = 0; t < z; ++t) {
      const int64_t e = (int64_t)c * z + t;
      s += (double)sign[e] * (double)In[(int64_t)idx[e] * ldi + q];
    }
    out[(int64_t)c * ldo + q] = sv * s;
  }
}

cudaError_t launch_signed_gather_sum64(const float *In, int64_t ldi, int32_t width,
                                       const int32_t *idx, const int8_t *sign, int32_t cols,
                                       int32_t z, double sv, double *out, int64_t ldo,
                                       cudaStream_t st) {
  if (cols <= 0 || width <= 0) return cudaSuccess;
  ProfScope ps_(K_GATHER, st);
  signed_gather_sum64_kernel<<<cols, 256, 0, st>>>(In, ldi, width, idx, sign, z, sv, out, ldo);
  return cudaGetLastError();
}

}  // namespace sne
