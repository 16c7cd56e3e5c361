// Centred evaluation of the entries of L'R' (Eq. 11) near the trunc_log
// threshold.
//
// With W = D^(-1+a) U (n x k), s = vol(G)/(bT) and C = Lambda sum_{r<T} K^r,
// Eq. 11 gives x_ij = s W_i C W_j^T.  For any reference row w,
//   x_ij - c0 = s (W_i - w) C (W_j - w)^T + rho_i + kappa_j,
//   rho_i   = s (W_i - w) C w^T + (s w C w^T - c0),
//   kappa_j = s w C (W_j - w)^T,
// is an identity.  Taking w as the degree-weighted mean of the rows of W,
// w = sum_i d_i W_i / vol(G), removes the component that every entry shares:
// the degree-weighted mean over i of any column of the NetMF matrix of Eq. 1
// is exactly 1/b (1^T D (D^-1 A)^r = 1^T D for every r), so on a connected
// graph with b = 1 the entries of L'R' sit near 1 and the stationary
// eigenvector (D^(1/2) 1 at a = 1/2) contributes a constant row of W, which
// the subtraction cancels exactly.  The products that remain are of the
// small, centred factors, so their rounding is relative to |x - 1| rather
// than to 1, and trunc_log(x) = log1p(x - 1) for x - 1 > 0 is evaluated from
// x - 1 directly.  c0 = 1 for trunc_log and 0 for f = identity.
//
// Kernels here:
//  * center_mean_partial_kernel / center_finish_kernel: w (FP32 sums of
//    64-row groups added in FP64, fixed-order two-stage sum), p = C w^T,
//    q = w C, gamma = s w C w^T - c0, s w as an FP32 hi/lo pair;
//  * center_rows_kernel: L~_i = s (W_i - w) in double-float, rounded once
//    (FP32 rows, or FP16/BF16 rows scaled by a power of two and split into a
//    hi part and a lo part), and (rho_i, mask_i);
//  * split_rows_kernel: FP32 rows -> power-of-two-scaled FP16/BF16 hi/lo rows.
#include <algorithm>
#include <type_traits>

#include "sne_internal.cuh"

namespace sne {

namespace {

constexpr int kMeanThreads = 256;

// Partial sums of d_i W_i = d_i^a U_i over row chunks.  The reference row w
// only has to remove the component the entries share: the centred form is an
// identity for any w, and rho and kappa are computed from the w this gives.
// So the weights are FP32 powers, each group of 64 rows is summed in FP32
// (loads of eight rows issued before their multiply-adds) and only the group
// sums are added in FP64: GB300's FP64 rate would make a per-row FP64 sum the
// bound of this kernel.
__global__ void __launch_bounds__(kMeanThreads) center_mean_partial_kernel(
    const float *__restrict__ U, int64_t ldu, int k, int64_t n, const float *__restrict__ deg,
    double alpha, int64_t rows_per_chunk, double *__restrict__ partial) {
  __shared__ float wsh[64];
  const int64_t r0 = (int64_t)blockIdx.x * rows_per_chunk;
  const int64_t r1 = min64(n, r0 + rows_per_chunk);
  const float af = (float)alpha;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};  // columns tid + 256 m, k <= 1024
  for (int64_t t0 = r0; t0 < r1; t0 += 64) {
    __syncthreads();
    if (threadIdx.x < 64) {
      const int64_t i = t0 + threadIdx.x;
      float wv = 0.f;
      if (i < r1) {
        const float d = deg[i];
        wv = d > 0.f ? powf(d, af) : 0.f;
      }
      wsh[threadIdx.x] = wv;
    }
    __syncthreads();
    const int rows = (int)min64(64, r1 - t0);
    float a32[4] = {0.f, 0.f, 0.f, 0.f};
    for (int r = 0; r < rows; r += 8) {
      float x[8][4];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float *row = U + (t0 + (r + u < rows ? r + u : 0)) * ldu;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int c = threadIdx.x + kMeanThreads * m;
          x[u][m] = c < k ? row[c] : 0.0f;
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const float wv = r + u < rows ? wsh[r + u] : 0.f;
#pragma unroll
        for (int m = 0; m < 4; ++m) a32[m] = fmaf(wv, x[u][m], a32[m]);
      }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) acc[m] += (double)a32[m];
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
    const int c = threadIdx.x + kMeanThreads * m;
    if (c < k) partial[(int64_t)blockIdx.x * k + c] = acc[m];
  }
}

// One CTA.  stats: w[k] | p[k] | q[k] | gamma | s.
__global__ void __launch_bounds__(kMeanThreads) center_finish_kernel(
    const double *__restrict__ partial, int chunks, int k, const double *__restrict__ vol_dev,
    const double *__restrict__ lam, const double *__restrict__ Csum, double smult, double c0,
    double *__restrict__ stats, float *__restrict__ ws_hi, float *__restrict__ ws_lo) {
  extern __shared__ double csh[];  // w[k], then reduction scratch
  double *wv = csh;
  double *red = csh + k;
  const double vol = *vol_dev;
  const double s = smult * vol;
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    double acc = 0.0;
    for (int b = 0; b < chunks; ++b) acc += partial[(int64_t)b * k + c];
    const double w = vol > 0.0 ? acc / vol : 0.0;
    wv[c] = w;
    stats[c] = w;
    const double sw = s * w;
    const float hi = (float)sw;
    ws_hi[c] = hi;
    ws_lo[c] = (float)(sw - (double)hi);
  }
  __syncthreads();
  double part = 0.0;
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    // p_c = sum_a C[c][a] w_a, C[c][a] = lam_c Csum[c][a]
    double pc = 0.0;
    for (int a = 0; a < k; ++a) pc = fma(Csum[(int64_t)c * k + a], wv[a], pc);
    pc *= lam[c];
    stats[k + c] = pc;
    part = fma(wv[c], pc, part);
    // q_a = sum_c w_c C[c][a]  (here a = this thread's column)
    double qa = 0.0;
    for (int cc = 0; cc < k; ++cc) qa = fma(wv[cc] * lam[cc], Csum[(int64_t)cc * k + c], qa);
    stats[2 * k + c] = qa;
  }
  red[threadIdx.x] = part;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    stats[3 * k] = s * red[0] - c0;  // gamma
    stats[3 * k + 1] = s;
  }
}

template <typename H>
__device__ __forceinline__ H cvt_h(float x);
template <>
__device__ __forceinline__ __half cvt_h<__half>(float x) {
  return __float2half_rn(x);
}
template <>
__device__ __forceinline__ __nv_bfloat16 cvt_h<__nv_bfloat16>(float x) {
  return __float2bfloat16_rn(x);
}
template <typename H>
__device__ __forceinline__ float h2f(H x);
template <>
__device__ __forceinline__ float h2f<__half>(__half x) {
  return __half2float(x);
}
template <>
__device__ __forceinline__ float h2f<__nv_bfloat16>(__nv_bfloat16 x) {
  return __bfloat162float(x);
}

// Power of two sc >= max_abs with max_abs / sc in (1/2, 1]; 1 for a zero row.
__device__ __forceinline__ float pow2_scale(float max_abs) {
  if (!(max_abs > 0.f)) return 1.0f;
  int e;
  const float f = frexpf(max_abs, &e);  // max_abs = f 2^e, f in [1/2, 1)
  (void)f;
  return ldexpf(1.0f, e);
}

constexpr int kMaxPerLane = 32;  // k <= 1024

// Warp per output row r (source row src = ridx ? ridx[r] : r).
//  OUT = 0: FP32 row L~ (ld ldl);  OUT = 1: FP16, OUT = 2: BF16 rows of
//  L~ / rowf (rowf a power of two) into hi (and lo when SPLIT) with kpad
//  columns, zero padded.
// rowdat[r] = (rho, mask).  Rows past *nrows_dev are zero (half outputs only).
template <int OUT, bool SPLIT>
__global__ void __launch_bounds__(256) center_rows_kernel(
    const float *__restrict__ U, int64_t ldu, int k, const int32_t *__restrict__ ridx,
    const int32_t *__restrict__ nrows_dev, int64_t nrows_max, const float *__restrict__ rsc,
    const float *__restrict__ rsc_lo, const float *__restrict__ ws_hi,
    const float *__restrict__ ws_lo, const double *__restrict__ stats, int trunc_log, double c0,
    float *__restrict__ Lt, int64_t ldl, void *__restrict__ Ahi, void *__restrict__ Alo, int kpad,
    float *__restrict__ rowf, float2 *__restrict__ rowdat) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (r >= nrows_max) return;
  const int64_t nrows = nrows_dev ? (int64_t)(*nrows_dev) : nrows_max;
  using H = typename std::conditional<OUT == 2, __nv_bfloat16, __half>::type;
  if (r >= nrows) {
    if (OUT != 0) {
      H *hi = static_cast<H *>(Ahi) + r * kpad;
      for (int c = lane; c < kpad; c += 32) hi[c] = cvt_h<H>(0.f);
      if (SPLIT) {
        H *lo = static_cast<H *>(Alo) + r * kpad;
        for (int c = lane; c < kpad; c += 32) lo[c] = cvt_h<H>(0.f);
      }
      if (lane == 0) rowf[r] = 0.f;
    }
    if (lane == 0) rowdat[r] = make_float2(0.f, 0.f);
    return;
  }
  const int64_t src = ridx ? (int64_t)ridx[r] : r;
  const float a_hi = rsc[src], a_lo = rsc_lo ? rsc_lo[src] : 0.f;  // s d^(-1+a), hi/lo
  const bool isolated = (a_hi == 0.f && a_lo == 0.f);
  const float *u = U + src * ldu;
  const double *pbar = stats + k;
  const double gamma = stats[3 * k];
  float v[kMaxPerLane];
  float dot = 0.f, mx = 0.f;
#pragma unroll
  for (int m = 0; m < kMaxPerLane; ++m) {
    const int c = lane + 32 * m;
    float x = 0.f;
    if (c < k && !isolated) {
      // s a_i U_ic - s w_c in double-float, one rounding at the end
      const float uc = u[c];
      const float p = __fmul_rn(a_hi, uc);
      float e = __fmaf_rn(a_hi, uc, -p);  // exact low part of a_hi uc
      e = __fmaf_rn(a_lo, uc, e);
      const float d = __fsub_rn(p, ws_hi[c]);
      const float t = __fsub_rn(e, ws_lo[c]);
      x = __fadd_rn(d, t);
      dot = fmaf(x, (float)pbar[c], dot);
      mx = fmaxf(mx, fabsf(x));
    }
    v[m] = x;
    if (32 * (m + 1) >= k) break;
  }
  // rho = sum_c L~_c p_c + gamma (lane partials in FP32, summed in FP64)
  double dsum = (double)dot;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
  if (OUT == 0) {
    float *o = Lt + r * ldl;
#pragma unroll
    for (int m = 0; m < kMaxPerLane; ++m) {
      const int c = lane + 32 * m;
      if (c < k) o[c] = v[m];
      if (32 * (m + 1) >= k) break;
    }
  } else {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    const float sc = pow2_scale(mx);
    const float inv = 1.0f / sc;  // exact: a power of two
    H *hi = static_cast<H *>(Ahi) + r * kpad;
    H *lo = SPLIT ? static_cast<H *>(Alo) + r * kpad : nullptr;
#pragma unroll
    for (int m = 0; m < kMaxPerLane; ++m) {
      const int c = lane + 32 * m;
      if (c < k) {
        const float y = v[m] * inv;
        const H h = cvt_h<H>(y);
        hi[c] = h;
        if (SPLIT) lo[c] = cvt_h<H>(__fsub_rn(y, h2f<H>(h)));
      }
      if (32 * (m + 1) >= k) break;
    }
    for (int c = k + lane; c < kpad; c += 32) {
      hi[c] = cvt_h<H>(0.f);
      if (SPLIT) lo[c] = cvt_h<H>(0.f);
    }
    if (lane == 0) rowf[r] = isolated ? 0.f : sc;
  }
  if (lane == 0) {
    float rho, mask;
    if (isolated) {
      // x_ij = 0 exactly: trunc_log gives 0 (rho = -inf), the identity 0 - c0
      rho = trunc_log ? -INFINITY : (float)(-c0);
      mask = 0.f;
    } else {
      rho = (float)(dsum + gamma);
      mask = 1.f;
    }
    rowdat[r] = make_float2(rho, mask);
  }
}

// FP32 rows (ld lds) -> rows / sc split into FP16/BF16 hi (+ lo), kpad columns;
// sc (a power of two) is written to scale[r * sstride].
template <typename H, bool SPLIT>
__global__ void __launch_bounds__(256) split_rows_kernel(const float *__restrict__ src,
                                                         int64_t lds, int64_t rows, int k, int kpad,
                                                         H *__restrict__ hi, H *__restrict__ lo,
                                                         float *__restrict__ scale, int sstride) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (r >= rows) return;
  const float *x = src + r * lds;
  float mx = 0.f;
  for (int c = lane; c < k; c += 32) mx = fmaxf(mx, fabsf(x[c]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const float sc = pow2_scale(mx);
  const float inv = 1.0f / sc;
  for (int c = lane; c < kpad; c += 32) {
    const float y = c < k ? x[c] * inv : 0.f;
    const H h = cvt_h<H>(y);
    hi[r * kpad + c] = h;
    if (SPLIT) lo[r * kpad + c] = cvt_h<H>(__fsub_rn(y, h2f<H>(h)));
  }
  if (lane == 0) scale[r * sstride] = sc;
}

}  // namespace

size_t center_partial_doubles(int64_t n, int k) {
  const int64_t chunks = std::min<int64_t>((n + 255) / 256, 4 * 1024);
  return (size_t)chunks * (size_t)k;
}

cudaError_t launch_center_stats(const float *U, int64_t ldu, int k, int64_t n, const float *deg,
                                double alpha, const double *vol_dev, const double *lam,
                                const double *Csum, double smult, double c0, double *partial,
                                double *stats, float *ws_hi, float *ws_lo, cudaStream_t st) {
  if (k <= 0 || k > 1024 || n <= 0) return cudaErrorInvalidValue;
  int64_t chunks = std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 4);
  if (chunks < 1) chunks = 1;
  if ((size_t)chunks * k > center_partial_doubles(n, k)) chunks = center_partial_doubles(n, k) / k;
  const int64_t rpc = (n + chunks - 1) / chunks;
  {
    ProfScope ps_(K_MISC, st);
    center_mean_partial_kernel<<<(unsigned)chunks, kMeanThreads, 0, st>>>(U, ldu, k, n, deg, alpha,
                                                                          rpc, partial);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t smem = (size_t)(k + kMeanThreads) * sizeof(double);
  ProfScope ps_(K_MISC, st);
  center_finish_kernel<<<1, kMeanThreads, smem, st>>>(partial, (int)chunks, k, vol_dev, lam, Csum,
                                                       smult, c0, stats, ws_hi, ws_lo);
  return cudaGetLastError();
}

cudaError_t launch_center_rows(int out, bool split, const float *U, int64_t ldu, int k,
                               const int32_t *ridx, const int32_t *nrows_dev, int64_t nrows_max,
                               const float *rsc, const float *rsc_lo, const float *ws_hi,
                               const float *ws_lo, const double *stats, bool trunc_log, double c0,
                               float *Lt, int64_t ldl, void *Ahi, void *Alo, int kpad, float *rowf,
                               float2 *rowdat, cudaStream_t st) {
  if (nrows_max <= 0) return cudaSuccess;
  if (k <= 0 || k > 32 * kMaxPerLane) return cudaErrorInvalidValue;
  const unsigned blocks = (unsigned)((nrows_max + 7) / 8);
  ProfScope ps_(K_MISC, st);
#define SNE_CR(O, S)                                                                             \
  center_rows_kernel<O, S><<<blocks, 256, 0, st>>>(U, ldu, k, ridx, nrows_dev, nrows_max, rsc,  \
                                                   rsc_lo, ws_hi, ws_lo, stats, trunc_log ? 1 : 0, \
                                                   c0, Lt, ldl, Ahi, Alo, kpad, rowf, rowdat)
  if (out == 0) SNE_CR(0, false);
  else if (out == 1 && split) SNE_CR(1, true);
  else if (out == 1) SNE_CR(1, false);
  else if (split) SNE_CR(2, true);
  else SNE_CR(2, false);
#undef SNE_CR
  return cudaGetLastError();
}

cudaError_t launch_split_rows(bool fp16, bool split, const float *src, int64_t lds, int64_t rows,
                              int k, int kpad, void *hi, void *lo, float *scale, int sstride,
                              cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((rows + 7) / 8);
  ProfScope ps_(K_MISC, st);
  if (fp16) {
    if (split)
      split_rows_kernel<__half, true><<<blocks, 256, 0, st>>>(
          src, lds, rows, k, kpad, static_cast<__half *>(hi), static_cast<__half *>(lo), scale, sstride);
    else
      split_rows_kernel<__half, false><<<blocks, 256, 0, st>>>(
          src, lds, rows, k, kpad, static_cast<__half *>(hi), nullptr, scale, sstride);
  } else {
    if (split)
      split_rows_kernel<__nv_bfloat16, true><<<blocks, 256, 0, st>>>(
          src, lds, rows, k, kpad, static_cast<__nv_bfloat16 *>(hi),
          static_cast<__nv_bfloat16 *>(lo), scale, sstride);
    else
      split_rows_kernel<__nv_bfloat16, false><<<blocks, 256, 0, st>>>(
          src, lds, rows, k, kpad, static_cast<__nv_bfloat16 *>(hi), nullptr, scale, sstride);
  }
  return cudaGetLastError();
}

}  // namespace sne
