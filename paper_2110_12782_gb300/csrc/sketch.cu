// Fused reconstruct + f + sparse-sign contraction (Eq. 4, Alg. 4 lines 4 and
// 7), FP32 SIMT form, and the signed gathers O^T Y' and O^T Q.
//
// The sparse-sign matrix is kept as its list of (column, slot) nonzeros: entry
// e = c*z + t has row idx[e] and sign[e].  The kernel evaluates one column of
// L'R' per nonzero, so that
//   out[i, c] = sv * sum_{t<z} sgn[c*z+t] * f(x_{i, idx[c*z+t]})
// is a sum over z consecutive evaluated columns.  This equals
// f(L'R'(:, p)) S(p, :) of Eq. 4 exactly: duplicated coordinates only repeat
// an evaluation.  M-hat is never stored.
//
// The entries are evaluated in the centred form of center.cu:
//   x_ie - c0 = <A[i, :], B[e, :]> + rho_i + mask_i kappa_e,
// A = L~ (rows s (W_i - w)), B = B~ (rows (W_j - w) C^T), rowdat[i] =
// (rho_i, mask_i), coldat[e] = (scale, kappa_e, sgn_e, 0); trunc_log(x) is
// log1p(x - 1) for x - 1 > 0 (c0 = 1) and the identity is x itself (c0 = 0).
#include "sne_internal.cuh"

namespace sne {

constexpr int kFM = 64;    // rows per CTA
constexpr int kFN = 128;   // evaluated columns per CTA
constexpr int kFK = 16;    // k step

// f from r = x - c0 (CUDA's log1pf: in this kernel, bound by the FP32
// products of k terms per entry, the polynomial form of the tensor-core
// epilogue measured slower)
template <int F>
__device__ __forceinline__ float apply_f(float r) {
  if (F == SNE_F_TRUNC_LOG) return r > 0.0f ? log1pf(r) : 0.0f;
  return r;
}

template <int F>
__global__ void __launch_bounds__(256) fused_sketch_f32_kernel(
    const float *__restrict__ A, int64_t lda, const int32_t *__restrict__ ridx,
    const int32_t *__restrict__ nrows_dev, int64_t nrows_max, int32_t k,
    const float2 *__restrict__ rowdat, const float *__restrict__ B,
    const float4 *__restrict__ coldat, int32_t cols_out, int32_t z, float sv,
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
  // epilogue: r = x - c0, f, sign -> shared; then segmented sums over z columns
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int64_t row = i0 + ty * 4 + i;
    float2 rd = make_float2(0.f, 0.f);
    if (row < nrows) rd = rowdat[ridx ? ridx[row] : row];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int c = tx * 8 + j;
      float v = 0.f;
      if (c < e_count) {
        const float4 cd = coldat[e_begin + c];
        v = cd.z * apply_f<F>(acc[i][j] + fmaf(rd.y, cd.y, rd.x));
      }
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

// Register-tiled form: CTA tile 128 rows x 128 evaluated columns, 256
// threads with 8 x 8 outputs each, k in steps of 8 through two shared-memory
// buffers (the next step's operands are loaded into registers while the
// current one is multiplied).  A thread's 8 columns are consecutive, so for
// z = 1, 2, 4, 8 the segmented sum over z columns stays in registers; for
// z = 16, 32 it adds the partial sums of 2 or 4 neighbouring lanes.
constexpr int kGM = 128, kGN = 128, kGK = 8;

template <int F, int Z>
__global__ void __launch_bounds__(256, 2) fused_sketch_f32_tiled_kernel(
    const float *__restrict__ A, int64_t lda, const int32_t *__restrict__ ridx,
    const int32_t *__restrict__ nrows_dev, int64_t nrows_max, int32_t k,
    const float2 *__restrict__ rowdat, const float *__restrict__ B,
    const float4 *__restrict__ coldat, int32_t cols_out, float sv, float *__restrict__ out,
    int64_t ldo) {
  __shared__ __align__(16) float As[2][kGK][kGM + 4];
  __shared__ __align__(16) float Bs[2][kGK][kGN + 4];
  const int64_t nrows = nrows_dev ? (int64_t)(*nrows_dev) : nrows_max;
  constexpr int CPT = kGN / Z;  // output columns per CTA
  // linear block index, column groups fastest: the CTAs that share a row tile
  // of A run together and read it from L2 after the first
  const int ncg = (cols_out + CPT - 1) / CPT;
  const int64_t i0 = (int64_t)(blockIdx.x / ncg) * kGM;
  if (i0 >= nrows) return;
  const int c_begin = (int)(blockIdx.x % ncg) * CPT;
  const int e_begin = c_begin * Z;
  const int e_count = min(CPT, cols_out - c_begin) * Z;
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;  // rows ty*8.., columns tx*8..
  // the two float4 of a thread's 8 columns are read in swapped order by
  // threads 4..7 of every 8 (sw = 1): the 8 threads of a 128-bit shared load
  // phase then cover all 32 banks (in order, columns 8 tx + 0 and 8 tx + 32
  // fall on the same banks: 2-way conflicts that made the loop bound by shared
  // memory); the accumulator halves are swapped back before the epilogue
  const int sw = (tx >> 2) & 1;
  // loader: thread t brings row (t >> 1) of A's tile and column (t >> 1) of
  // B's tile, k-part 4 (t & 1) .. +4, as one float4 each
  const int lr = tid >> 1, lk = 4 * (tid & 1);
  const int64_t arow = i0 + lr;
  const bool a_ok = arow < nrows;
  const float *ap = A + (a_ok ? (ridx ? (int64_t)ridx[arow] : arow) : 0) * lda;
  const bool b_ok = lr < e_count;
  const float *bp = B + (int64_t)(e_begin + (b_ok ? lr : 0)) * k;
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  float4 pa = (a_ok && lk < k) ? __ldg(reinterpret_cast<const float4 *>(ap + lk)) : zero4;
  float4 pb = (b_ok && lk < k) ? __ldg(reinterpret_cast<const float4 *>(bp + lk)) : zero4;
  int buf = 0;
  for (int k0 = 0; k0 < k; k0 += kGK) {
    As[buf][lk + 0][lr] = pa.x;
    As[buf][lk + 1][lr] = pa.y;
    As[buf][lk + 2][lr] = pa.z;
    As[buf][lk + 3][lr] = pa.w;
    Bs[buf][lk + 0][lr] = pb.x;
    Bs[buf][lk + 1][lr] = pb.y;
    Bs[buf][lk + 2][lr] = pb.z;
    Bs[buf][lk + 3][lr] = pb.w;
    __syncthreads();
    const int kn = k0 + kGK + lk;
    pa = (a_ok && kn < k) ? __ldg(reinterpret_cast<const float4 *>(ap + kn)) : zero4;
    pb = (b_ok && kn < k) ? __ldg(reinterpret_cast<const float4 *>(bp + kn)) : zero4;
#pragma unroll
    for (int kk = 0; kk < kGK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 8]);
      const float4 a1 = *reinterpret_cast<const float4 *>(&As[buf][kk][ty * 8 + 4]);
      const float4 b0 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 8 + 4 * sw]);
      const float4 b1 = *reinterpret_cast<const float4 *>(&Bs[buf][kk][tx * 8 + 4 * (sw ^ 1)]);
      const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    buf ^= 1;
  }
  if (sw) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float t = acc[i][j];
        acc[i][j] = acc[i][j + 4];
        acc[i][j + 4] = t;
      }
  }
  // epilogue: r = acc + rho_i + mask_i kappa_e, f, sign, segmented sums over Z columns
  float sg[8], kp[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int c = tx * 8 + j;
    const float4 cd = c < e_count ? coldat[e_begin + c] : make_float4(0.f, 0.f, 0.f, 0.f);
    kp[j] = cd.y;
    sg[j] = cd.z;
  }
  constexpr int PER = Z < 8 ? 8 / Z : 1;  // outputs per thread per row
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t row = i0 + ty * 8 + i;
    const bool rok = row < nrows;
    float2 rd = make_float2(0.f, 0.f);
    if (rok) rd = rowdat[ridx ? ridx[row] : row];
    float part[PER];
#pragma unroll
    for (int g = 0; g < PER; ++g) part[g] = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const float r = acc[i][j] + fmaf(rd.y, kp[j], rd.x);
      part[Z < 8 ? j / Z : 0] += sg[j] * apply_f<F>(r);
    }
    if (Z > 8) {
      // combine the Z / 8 lanes of one output column (consecutive tx)
#pragma unroll
      for (int o = 1; o < Z / 8; o <<= 1) part[0] += __shfl_xor_sync(0xffffffffu, part[0], o);
    }
    if (!rok) continue;
    if (Z <= 8) {
#pragma unroll
      for (int g = 0; g < PER; ++g) {
        const int oc = c_begin + (tx * 8) / Z + g;
        if (tx * 8 + g * Z < e_count) out[row * ldo + oc] = sv * part[g];
      }
    } else if ((tx & (Z / 8 - 1)) == 0) {
      const int oc = c_begin + (tx * 8) / Z;
      if (tx * 8 < e_count) out[row * ldo + oc] = sv * part[0];
    }
  }
}

cudaError_t launch_fused_sketch_f32(const float *A, int64_t lda, const int32_t *ridx,
                                    const int32_t *nrows_dev, int64_t nrows, int32_t k,
                                    const float2 *rowdat, const float *B, const float4 *coldat,
                                    int32_t cols_out, int32_t z, float sv, int32_t f, float *out,
                                    int64_t ldo, cudaStream_t st) {
  if (nrows <= 0 || cols_out <= 0) return cudaSuccess;
  if (z <= 0 || z > kFN) return cudaErrorInvalidValue;
  if (k % 4 == 0 && lda % 4 == 0 && (uintptr_t)A % 16 == 0 && (uintptr_t)B % 16 == 0 &&
      (z == 1 || z == 2 || z == 4 || z == 8 || z == 16 || z == 32)) {
    const int cptz = kGN / z;
    const dim3 grid2((unsigned)(((nrows + kGM - 1) / kGM) * ((cols_out + cptz - 1) / cptz)));
    ProfScope ps_(K_FUSED, st);
#define SNE_F32_CASE(FV, ZV)                                                                    \
  fused_sketch_f32_tiled_kernel<FV, ZV><<<grid2, 256, 0, st>>>(A, lda, ridx, nrows_dev, nrows, k, \
                                                             rowdat, B, coldat, cols_out, sv,   \
                                                             out, ldo)
#define SNE_F32_Z(FV)                         \
  switch (z) {                                \
    case 1: SNE_F32_CASE(FV, 1); break;       \
    case 2: SNE_F32_CASE(FV, 2); break;       \
    case 4: SNE_F32_CASE(FV, 4); break;       \
    case 8: SNE_F32_CASE(FV, 8); break;       \
    case 16: SNE_F32_CASE(FV, 16); break;     \
    default: SNE_F32_CASE(FV, 32); break;     \
  }
    if (f == SNE_F_TRUNC_LOG) {
      SNE_F32_Z(SNE_F_TRUNC_LOG)
    } else {
      SNE_F32_Z(SNE_F_IDENTITY)
    }
#undef SNE_F32_Z
#undef SNE_F32_CASE
    return cudaGetLastError();
  }
  const int cpt = kFN / z;
  dim3 grid((unsigned)((nrows + kFM - 1) / kFM), (unsigned)((cols_out + cpt - 1) / cpt));
  ProfScope ps_(K_FUSED, st);
  if (f == SNE_F_TRUNC_LOG)
    fused_sketch_f32_kernel<SNE_F_TRUNC_LOG><<<grid, 256, 0, st>>>(
        A, lda, ridx, nrows_dev, nrows, k, rowdat, B, coldat, cols_out, z, sv, out, ldo);
  else
    fused_sketch_f32_kernel<SNE_F_IDENTITY><<<grid, 256, 0, st>>>(
        A, lda, ridx, nrows_dev, nrows, k, rowdat, B, coldat, cols_out, z, sv, out, ldo);
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

// Centred columns of R' for the gathered vertices j = idx[e] (Eq. 11):
//   out[e, :] = (W_j - w) (C_hi + C_lo)^T,  W_j = d_j^beta U[j, :],
//   coldat[e] = (1, kappa_e, sgn_e, 0),  kappa_e = s q (W_j - w)^T,
// with w, q = w C and s from the centring statistics (stats: w | p | q |
// gamma | s).  W_j - w is formed in FP64 and rounded to FP32 once; the sums
// over the k terms are FP32 FMA chains against the FP32 pair C^T = C_hi + C_lo
// (so that the rounding of C, which every column would otherwise share,
// cancels), each output rounded to FP32 once; kappa_e is summed in FP64 from
// the same rounded W_j - w.  A vertex of degree 0 has R'(:, j) = 0, so its
// columns get sgn_e = 0.
constexpr int kRpRows = 8;
__global__ void __launch_bounds__(256) rtilde_rows_kernel(
    const float *__restrict__ U, int32_t k, const int32_t *__restrict__ idx, int32_t count,
    const float *__restrict__ CThi, const float *__restrict__ CTlo, const float *__restrict__ deg,
    double beta, const double *__restrict__ stats, const int8_t *__restrict__ sign,
    float *__restrict__ out, float4 *__restrict__ coldat) {
  extern __shared__ float us[];  // kRpRows x k
  const int i0 = blockIdx.x * kRpRows;
  const int rows = min(kRpRows, count - i0);
  for (int e = threadIdx.x; e < kRpRows * k; e += blockDim.x) {
    const int r = e / k, a = e % k;
    float v = 0.f;
    if (r < rows) {
      const int j = idx[i0 + r];
      const float dj = deg[j];
      const double aj = dj > 0.f ? pow((double)dj, beta) : 0.0;
      v = (float)(aj * (double)U[(int64_t)j * k + a] - stats[a]);
    }
    us[e] = v;
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
      out[(int64_t)(i0 + r) * k + c] = (float)((double)hi[r] + (double)lo[r]);
    }
  }
  // kappa_e: one warp per row
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp < rows) {
    const double *q = stats + 2 * k;
    double acc = 0.0;
    for (int a = lane; a < k; a += 32) acc = fma(q[a], (double)us[warp * k + a], acc);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) {
      const int e = i0 + warp;
      const int j = idx[e];
      const float sg = deg[j] > 0.f ? (float)sign[e] : 0.f;
      coldat[e] = make_float4(1.0f, (float)(stats[3 * k + 1] * acc), sg, 0.f);
    }
  }
}

cudaError_t launch_rtilde_rows(const float *U, int32_t k, const int32_t *idx, int32_t count,
                               const float *CThi, const float *CTlo, const float *deg, double beta,
                               const double *stats, const int8_t *sign, float *out, float4 *coldat,
                               cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  const size_t smem = (size_t)kRpRows * k * sizeof(float);
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(rtilde_rows_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  ProfScope ps_(K_TALL_GEMM, st);
  rtilde_rows_kernel<<<(count + kRpRows - 1) / kRpRows, 256, smem, st>>>(
      U, k, idx, count, CThi, CTlo, deg, beta, stats, sign, out, coldat);
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
