// Dense building blocks of Alg. 4 and Alg. 5: the tall-skinny Gram Y^T Y and
// Q^T (XQ) (eigSVD, Rayleigh-Ritz, CholeskyQR), the tall-by-small product
// Y M, small GEMMs, and single-CTA small factorizations (Cholesky, triangular
// inverse, symmetric eigendecomposition by Householder tridiagonalization and
// implicit shifted QR).
#include <cfloat>
#include <cstdlib>
#include <cmath>

#include "sne_internal.cuh"

namespace sne {

// ---------------------------------------------------------------------------
// Tall-skinny Gram: C = sum_i w_i A[i,:]^T B[i,:]  (FP32 products, FP32 partial
// sums per row chunk, FP64 reduction over chunks in a fixed order).
// CTA = one 64x64 output tile over one row chunk; 64 threads, 8x8 each.
// ---------------------------------------------------------------------------
constexpr int kGT = 64;   // output tile edge
constexpr int kGR = 32;   // rows per shared-memory stage
constexpr int kGThreads = 64;

static inline int ceil_div(int64_t a, int64_t b) { return (int)((a + b - 1) / b); }

static void gram_grid(int64_t n, int Ka, int Kb, bool symmetric, int *tiles, int *chunks) {
  const int ta = ceil_div(Ka, kGT), tb = ceil_div(Kb, kGT);
  *tiles = symmetric ? ta * (ta + 1) / 2 : ta * tb;
  int want = (sm_count() * 10 + *tiles - 1) / *tiles;
  const int maxc = ceil_div(n, 4 * kGR);
  if (want > maxc) want = maxc;
  if (want < 1) want = 1;
  *chunks = want;
}

bool tc_gemm_enabled() {
  static int enabled = -1;
  if (enabled < 0) {
    const char *v = getenv("SNE_SIMT_GEMM");
    enabled = (v && v[0] == '1') ? 0 : 1;
  }
  return enabled == 1;
}

size_t gram_partial_floats(int64_t n, int32_t Ka, int32_t Kb) {
  const size_t tcf = gram_tc_partial_floats(n, Ka, Kb);
  int tiles, chunks;
  gram_grid(n, Ka, Kb, false, &tiles, &chunks);
  int tiles_s, chunks_s;
  gram_grid(n, Ka, Kb, Ka == Kb, &tiles_s, &chunks_s);
  if (chunks_s > chunks) chunks = chunks_s;
  // FP64 partials of the double-float Gram take two floats per entry
  const size_t simt = 2 * (size_t)chunks * (size_t)Ka * (size_t)Kb;
  return simt > tcf ? simt : tcf;
}

__global__ void __launch_bounds__(kGThreads) gram_partial_kernel(
    const float *__restrict__ A, int64_t lda, int32_t Ka, const float *__restrict__ B, int64_t ldb,
    int32_t Kb, int64_t n, const float *__restrict__ w, int symmetric, int32_t tiles_a,
    int64_t rows_per_chunk, float *__restrict__ partial) {
  __shared__ __align__(16) float As[kGR][kGT];
  __shared__ __align__(16) float Bs[kGR][kGT];
  // decode the tile pair
  int ta, tb;
  int t = blockIdx.x;
  if (symmetric) {
    ta = 0;
    int rowlen = tiles_a;
    while (t >= rowlen) {
      t -= rowlen;
      ++ta;
      --rowlen;
    }
    tb = ta + t;
  } else {
    ta = t / ((Kb + kGT - 1) / kGT);
    tb = t % ((Kb + kGT - 1) / kGT);
  }
  const int a0 = ta * kGT, b0 = tb * kGT;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t r1 = min64(n, r0 + rows_per_chunk);
  const int tid = threadIdx.x;
  const int ty = tid >> 3, tx = tid & 7;
  // two-level sum: acc takes 256 rows at a time and is then added into tot,
  // so no FP32 chain grows longer than 256 + rows/256 terms
  float acc[8][8], tot[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = tot[i][j] = 0.f;

  int blk = 0;
  for (int64_t rs = r0; rs < r1; rs += kGR) {
    // load 32 rows x 64 columns of A and B (one column per thread)
#pragma unroll 4
    for (int r = 0; r < kGR; ++r) {
      const int64_t row = rs + r;
      float av = 0.f, bv = 0.f;
      if (row < r1) {
        const float wr = w ? w[row] : 1.0f;
        if (a0 + tid < Ka) av = wr * A[row * lda + a0 + tid];
        if (b0 + tid < Kb) bv = B[row * ldb + b0 + tid];
      }
      As[r][tid] = av;
      Bs[r][tid] = bv;
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < kGR; ++r) {
      const float4 a_lo = *reinterpret_cast<const float4 *>(&As[r][ty * 8]);
      const float4 a_hi = *reinterpret_cast<const float4 *>(&As[r][ty * 8 + 4]);
      const float4 b_lo = *reinterpret_cast<const float4 *>(&Bs[r][tx * 8]);
      const float4 b_hi = *reinterpret_cast<const float4 *>(&Bs[r][tx * 8 + 4]);
      const float av[8] = {a_lo.x, a_lo.y, a_lo.z, a_lo.w, a_hi.x, a_hi.y, a_hi.z, a_hi.w};
      const float bv[8] = {b_lo.x, b_lo.y, b_lo.z, b_lo.w, b_hi.x, b_hi.y, b_hi.z, b_hi.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
    }
    __syncthreads();
    if (++blk == 256 / kGR) {
      blk = 0;
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          tot[i][j] += acc[i][j];
          acc[i][j] = 0.f;
        }
    }
  }
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) tot[i][j] += acc[i][j];
  float *P = partial + (size_t)blockIdx.y * Ka * Kb;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int a = a0 + ty * 8 + i;
    if (a >= Ka) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int b = b0 + tx * 8 + j;
      if (b < Kb) P[(size_t)a * Kb + b] = tot[i][j];
    }
  }
}

__global__ void gram_reduce_kernel(const float *__restrict__ partial, int32_t Ka, int32_t Kb,
                                   int32_t chunks, int sym_tile, double *__restrict__ C,
                                   int32_t ldc) {
  const int64_t total = (int64_t)Ka * Kb;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int a = (int)(e / Kb), b = (int)(e % Kb);
    int sa = a, sb = b;
    if (sym_tile > 0 && (a / sym_tile) > (b / sym_tile)) {
      sa = b;
      sb = a;
    }
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += (double)partial[(size_t)c * Ka * Kb + (size_t)sa * Kb + sb];
    C[(int64_t)a * ldc + b] = s;
  }
}

cudaError_t launch_gram_reduce(const float *partial, int Ka, int Kb, int chunks, int sym_tile,
                               double *C, int ldc, cudaStream_t st) {
  const int64_t total = (int64_t)Ka * Kb;
  ProfScope ps_(K_GRAM_TC, st);
  gram_reduce_kernel<<<(unsigned)min64(1024, (total + 255) / 256), 256, 0, st>>>(
      partial, Ka, Kb, chunks, sym_tile, C, ldc);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// FP64-accurate Gram.  Every output is accumulated over groups of 16 rows
// with FP32 FMA; each group sum is then added into a double-float pair
// (hi, lo) with Knuth's TwoSum, which is exact, so the rounding error does not
// grow with n: the group sums carry a relative error of a few units of 2^-24
// of a group, and the pair keeps about 48 bits of the total.  64 x 64
// output tile per CTA, 128 threads with 4 x 8 outputs each; one FP64 partial
// per row chunk.
// ---------------------------------------------------------------------------
constexpr int kDThreads = 128;

// (hi, lo) += x with the rounding error of hi + x carried into lo (TwoSum;
// the _rn intrinsics keep the compiler from contracting or reordering it)
__device__ __forceinline__ void two_sum_into(float &hi, float &lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bp = __fsub_rn(s, hi);
  const float ap = __fsub_rn(s, bp);
  lo = __fadd_rn(lo, __fadd_rn(__fsub_rn(hi, ap), __fsub_rn(x, bp)));
  hi = s;
}

// With weights (WEIGHTED), row i of A is scaled by w_i = w_hi[i] + w_lo[i] (an
// FP32 pair carrying the weight to FP64 accuracy): the scaled entry is kept as
// the pair (fl(w_hi a), fma(w_hi, a, -fl(w_hi a)) + w_lo a), whose second part
// enters the products' error terms.
template <bool WEIGHTED, bool EXACT>
__global__ void __launch_bounds__(kDThreads) gram_df_partial_kernel(
    const float *__restrict__ A, int64_t lda, int32_t Ka, const float *__restrict__ B, int64_t ldb,
    int32_t Kb, int64_t n, const float *__restrict__ w, const float *__restrict__ w_lo,
    int symmetric, int32_t tiles_a, int64_t rows_per_chunk, double *__restrict__ partial) {
  __shared__ __align__(16) float As[kGR][kGT];
  __shared__ __align__(16) float Al[WEIGHTED ? kGR : 1][kGT];
  __shared__ __align__(16) float Bs[kGR][kGT];
  int ta, tb;
  int t = blockIdx.x;
  if (symmetric) {
    ta = 0;
    int rowlen = tiles_a;
    while (t >= rowlen) {
      t -= rowlen;
      ++ta;
      --rowlen;
    }
    tb = ta + t;
  } else {
    ta = t / ((Kb + kGT - 1) / kGT);
    tb = t % ((Kb + kGT - 1) / kGT);
  }
  const int a0 = ta * kGT, b0 = tb * kGT;
  const int64_t r0 = (int64_t)blockIdx.y * rows_per_chunk;
  const int64_t r1 = min64(n, r0 + rows_per_chunk);
  const int tid = threadIdx.x;
  const int ty = tid >> 3, tx = tid & 7;  // 16 x 8 threads: rows ty*4.., cols tx*8..
  // threads 4..7 of every 8 read the two float4 of their 8 columns in swapped
  // order (sw = 1), so that the 8 threads of a 128-bit shared load phase fall
  // on all 32 banks (else columns 8 tx and 8 tx + 32 share banks: 2-way
  // conflicts); j < 4 of hi, lo then hold columns 8 tx + 4 sw + j
  const int sw = (tx >> 2) & 1;
  float hi[4][8], lo[4][8];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) hi[i][j] = lo[i][j] = 0.f;
  // a stage is 32 rows x 64 columns of A and of B = 1024 float4, 8 per thread;
  // float4 q of the stage: matrix q / 512, row (q / 16) % 32, column 4 (q % 16)
  const bool vec = (lda % 4 == 0) && (ldb % 4 == 0) && ((uintptr_t)A % 16 == 0) &&
                   ((uintptr_t)B % 16 == 0);
  float4 pre[8];
  float2 wpre[4];  // (w_hi, w_lo) of the A rows this thread fetches
  auto fetch = [&](int64_t rs) {
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int q = tid + kDThreads * m;
      const bool isA = q < 512;
      const int r = (q >> 4) & 31, c = 4 * (q & 15);
      const int64_t row = rs + r;
      const int cbase = (isA ? a0 : b0) + c;
      const int K = isA ? Ka : Kb;
      const float *src = isA ? A + row * lda : B + row * ldb;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (row < r1) {
        if (vec && cbase + 3 < K) {
          v = __ldg(reinterpret_cast<const float4 *>(src + cbase));
        } else {
          if (cbase < K) v.x = src[cbase];
          if (cbase + 1 < K) v.y = src[cbase + 1];
          if (cbase + 2 < K) v.z = src[cbase + 2];
          if (cbase + 3 < K) v.w = src[cbase + 3];
        }
      }
      if (WEIGHTED && isA)
        wpre[m] = row < r1 ? make_float2(w[row], w_lo ? w_lo[row] : 0.f) : make_float2(0.f, 0.f);
      pre[m] = v;
    }
  };
  if (r0 < r1) fetch(r0);
  for (int64_t rs = r0; rs < r1; rs += kGR) {
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int q = tid + kDThreads * m;
      const int r = (q >> 4) & 31, c = 4 * (q & 15);
      if (WEIGHTED && q < 512) {
        // w a as the pair (hi, lo), elementwise
        const float wh = wpre[m].x, wl = wpre[m].y;
        const float4 a = pre[m];
        float4 h, l;
        h.x = __fmul_rn(wh, a.x); l.x = __fmaf_rn(wl, a.x, __fmaf_rn(wh, a.x, -h.x));
        h.y = __fmul_rn(wh, a.y); l.y = __fmaf_rn(wl, a.y, __fmaf_rn(wh, a.y, -h.y));
        h.z = __fmul_rn(wh, a.z); l.z = __fmaf_rn(wl, a.z, __fmaf_rn(wh, a.z, -h.z));
        h.w = __fmul_rn(wh, a.w); l.w = __fmaf_rn(wl, a.w, __fmaf_rn(wh, a.w, -h.w));
        *reinterpret_cast<float4 *>(&As[r][c]) = h;
        *reinterpret_cast<float4 *>(&Al[WEIGHTED ? r : 0][c]) = l;
      } else {
        *reinterpret_cast<float4 *>(q < 512 ? &As[r][c] : &Bs[r][c]) = pre[m];
      }
    }
    __syncthreads();
    if (rs + kGR < r1) fetch(rs + kGR);  // in flight while this stage is summed
    if (!EXACT) {
      // FP32 FMA sums over groups of 16 rows, each group sum added into the
      // pair (hi, lo) by TwoSum: relative error about 16 eps32 of the largest
      // group sum
#pragma unroll
      for (int g = 0; g < kGR; g += 16) {
        float acc[4][8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
#pragma unroll
        for (int r = g; r < g + 16; ++r) {
          const float4 av = *reinterpret_cast<const float4 *>(&As[r][ty * 4]);
          const float4 b_lo = *reinterpret_cast<const float4 *>(&Bs[r][tx * 8 + 4 * sw]);
          const float4 b_hi = *reinterpret_cast<const float4 *>(&Bs[r][tx * 8 + 4 * (sw ^ 1)]);
          const float a4[4] = {av.x, av.y, av.z, av.w};
          const float b8[8] = {b_lo.x, b_lo.y, b_lo.z, b_lo.w, b_hi.x, b_hi.y, b_hi.z, b_hi.w};
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a4[i], b8[j], acc[i][j]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) two_sum_into(hi[i][j], lo[i][j], acc[i][j]);
      }
      __syncthreads();
      continue;
    }
    // EXACT: every product is split exactly into p + e (p = fl(a b),
    // e = fma(a, b, -p)) and p is added into the pair (hi, lo) by TwoSum, e into
    // lo: no rounding of a product or of a running sum is lost, only the final
    // rounding of lo, whose terms are about 2^-24 of the sum's
#pragma unroll 4
    for (int r = 0; r < kGR; ++r) {
      const float4 av = *reinterpret_cast<const float4 *>(&As[r][ty * 4]);
      const float4 b_lo = *reinterpret_cast<const float4 *>(&Bs[r][tx * 8 + 4 * sw]);
      const float4 b_hi = *reinterpret_cast<const float4 *>(&Bs[r][tx * 8 + 4 * (sw ^ 1)]);
      const float a4[4] = {av.x, av.y, av.z, av.w};
      const float b8[8] = {b_lo.x, b_lo.y, b_lo.z, b_lo.w, b_hi.x, b_hi.y, b_hi.z, b_hi.w};
      float al4[4] = {0.f, 0.f, 0.f, 0.f};
      if (WEIGHTED) {
        const float4 alv = *reinterpret_cast<const float4 *>(&Al[WEIGHTED ? r : 0][ty * 4]);
        al4[0] = alv.x; al4[1] = alv.y; al4[2] = alv.z; al4[3] = alv.w;
      }
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          const float pr = __fmul_rn(a4[i], b8[j]);
          float er = __fmaf_rn(a4[i], b8[j], -pr);
          if (WEIGHTED) er = __fmaf_rn(al4[i], b8[j], er);
          two_sum_into(hi[i][j], lo[i][j], pr);
          lo[i][j] = __fadd_rn(lo[i][j], er);
        }
    }
    __syncthreads();
  }
  double *P = partial + (size_t)blockIdx.y * Ka * Kb;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int a = a0 + ty * 4 + i;
    if (a >= Ka) continue;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int b = b0 + tx * 8 + 4 * ((j >> 2) ^ sw) + (j & 3);
      if (b < Kb) P[(size_t)a * Kb + b] = (double)hi[i][j] + (double)lo[i][j];
    }
  }
}

__global__ void gram_reduce64_kernel(const double *__restrict__ partial, int32_t Ka, int32_t Kb,
                                     int32_t chunks, int sym_tile, double *__restrict__ C,
                                     int32_t ldc) {
  const int64_t total = (int64_t)Ka * Kb;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    int a = (int)(e / Kb), b = (int)(e % Kb);
    int sa = a, sb = b;
    if (sym_tile > 0 && (a / sym_tile) > (b / sym_tile)) {
      sa = b;
      sb = a;
    }
    double s = 0.0;
    for (int c = 0; c < chunks; ++c) s += partial[(size_t)c * Ka * Kb + (size_t)sa * Kb + sb];
    C[(int64_t)a * ldc + b] = s;
  }
}

cudaError_t launch_gram_accurate(const float *A, int64_t lda, int32_t Ka, const float *B,
                                 int64_t ldb, int32_t Kb, int64_t n, const float *w,
                                 const float *w_lo, bool symmetric, float *partial, double *C,
                                 int32_t ldc, cudaStream_t st, bool exact) {
  if (symmetric && (A != B || Ka != Kb || lda != ldb)) return cudaErrorInvalidValue;
  if (n <= 0 || Ka <= 0 || Kb <= 0) return cudaErrorInvalidValue;
  int tiles, chunks;
  gram_grid(n, Ka, Kb, symmetric, &tiles, &chunks);
  int64_t rpc = (n + chunks - 1) / chunks;
  rpc = (rpc + kGR - 1) / kGR * kGR;
  double *p64 = reinterpret_cast<double *>(partial);
  {
    ProfScope ps_(K_GRAM, st, 2);
#define SNE_GDF(WV, EV)                                                                      \
  gram_df_partial_kernel<WV, EV><<<dim3(tiles, chunks), kDThreads, 0, st>>>(                  \
      A, lda, Ka, B, ldb, Kb, n, w, w_lo, symmetric ? 1 : 0, ceil_div(Ka, kGT), rpc, p64)
    if (w && exact) SNE_GDF(true, true);
    else if (w) SNE_GDF(true, false);
    else if (exact) SNE_GDF(false, true);
    else SNE_GDF(false, false);
#undef SNE_GDF
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t total = (int64_t)Ka * Kb;
    gram_reduce64_kernel<<<(unsigned)min64(1024, (total + 255) / 256), 256, 0, st>>>(
        p64, Ka, Kb, chunks, symmetric ? kGT : 0, C, ldc);
  }
  return cudaGetLastError();
}

cudaError_t launch_gram(const float *A, int64_t lda, int32_t Ka, const float *B, int64_t ldb,
                        int32_t Kb, int64_t n, const float *w, bool symmetric, float *partial,
                        double *C, int32_t ldc, cudaStream_t st, Ctrl *ctrl) {
  if (symmetric && (A != B || Ka != Kb || lda != ldb)) return cudaErrorInvalidValue;
  if (tc_gemm_enabled() && tc_gemm_supported(Kb) && lda % 4 == 0 && ldb % 4 == 0 &&
      (uintptr_t)A % 16 == 0 && (uintptr_t)B % 16 == 0 && n >= 256)
    return launch_gram_tc(A, lda, Ka, B, ldb, Kb, n, w, symmetric && A == B && Ka == Kb, partial, C,
                          ldc, ctrl, st);
  int tiles, chunks;
  gram_grid(n, Ka, Kb, symmetric, &tiles, &chunks);
  const int64_t rpc = (n + chunks - 1) / chunks;
  ProfScope ps_(K_GRAM, st, 2);
  gram_partial_kernel<<<dim3(tiles, chunks), kGThreads, 0, st>>>(
      A, lda, Ka, B, ldb, Kb, n, w, symmetric ? 1 : 0, ceil_div(Ka, kGT), rpc, partial);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t total = (int64_t)Ka * Kb;
  gram_reduce_kernel<<<(unsigned)min64(1024, (total + 255) / 256), 256, 0, st>>>(
      partial, Ka, Kb, chunks, symmetric ? kGT : 0, C, ldc);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Tall-by-small product C[i,:] = rs_i * A[r(i),:] M  (FP32).
// CTA tile 128 rows x 64 columns, K step 16, 256 threads with 8x4 outputs.
// ---------------------------------------------------------------------------
constexpr int kTM = 128, kTN = 64, kTK = 16;

__global__ void __launch_bounds__(256) tall_gemm_kernel(
    const float *__restrict__ A, int64_t lda, const int32_t *__restrict__ ridx, int64_t n,
    int32_t Ka, const float *__restrict__ M, int32_t ldm, int32_t Kc, const float *__restrict__ rs,
    float *__restrict__ C, int64_t ldc) {
  __shared__ __align__(16) float As[kTK][kTM + 4];
  __shared__ __align__(16) float Ms[kTK][kTN];
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  const int64_t i0 = (int64_t)blockIdx.x * kTM;
  const int c0 = blockIdx.y * kTN;
  float acc[8][4];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  for (int k0 = 0; k0 < Ka; k0 += kTK) {
#pragma unroll
    for (int e = 0; e < (kTM * kTK) / 256; ++e) {
      const int lin = tid + 256 * e;
      const int r = lin / kTK, kk = lin % kTK;
      const int64_t i = i0 + r;
      float v = 0.f;
      if (i < n && k0 + kk < Ka) {
        const int64_t src = ridx ? (int64_t)ridx[i] : i;
        v = A[src * lda + k0 + kk];
      }
      As[kk][r] = v;
    }
#pragma unroll
    for (int e = 0; e < (kTK * kTN) / 256; ++e) {
      const int lin = tid + 256 * e;
      const int kk = lin / kTN, c = lin % kTN;
      float v = 0.f;
      if (k0 + kk < Ka && c0 + c < Kc) v = M[(int64_t)(k0 + kk) * ldm + c0 + c];
      Ms[kk][c] = v;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTK; ++kk) {
      const float4 alo = *reinterpret_cast<const float4 *>(&As[kk][ty * 8]);
      const float4 ahi = *reinterpret_cast<const float4 *>(&As[kk][ty * 8 + 4]);
      const float4 m = *reinterpret_cast<const float4 *>(&Ms[kk][tx * 4]);
      const float av[8] = {alo.x, alo.y, alo.z, alo.w, ahi.x, ahi.y, ahi.z, ahi.w};
      const float mv[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], mv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int64_t row = i0 + ty * 8 + i;
    if (row >= n) continue;
    const float s = rs ? rs[ridx ? ridx[row] : row] : 1.0f;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx * 4 + j;
      if (c < Kc) C[row * ldc + c] = s * acc[i][j];
    }
  }
}

cudaError_t launch_tall_gemm_auto(const float *A, int64_t lda, int64_t n, int32_t Ka, const float *M,
                                  int32_t ldm, int32_t Kc, float *C, int64_t ldc, float *Mt,
                                  Ctrl *ctrl, cudaStream_t st) {
  if (tc_gemm_enabled() && tc_gemm_supported(Kc) && Mt && lda % 4 == 0 && ldc % 4 == 0 &&
      Ka % 4 == 0 && (uintptr_t)A % 16 == 0 && (uintptr_t)Mt % 16 == 0 && n >= 256)
    return launch_tall_gemm_tc(A, lda, n, Ka, M, ldm, Kc, C, ldc, Mt, ctrl, st);
  return launch_tall_gemm(A, lda, nullptr, n, Ka, M, ldm, Kc, nullptr, C, ldc, st);
}

cudaError_t launch_tall_gemm(const float *A, int64_t lda, const int32_t *ridx, int64_t n, int32_t Ka,
                             const float *M, int32_t ldm, int32_t Kc, const float *rs, float *C,
                             int64_t ldc, cudaStream_t st) {
  if (n <= 0 || Kc <= 0) return cudaSuccess;
  dim3 grid((unsigned)((n + kTM - 1) / kTM), (unsigned)ceil_div(Kc, kTN));
  ProfScope ps_(K_TALL_GEMM, st);
  tall_gemm_kernel<<<grid, 256, 0, st>>>(A, lda, ridx, n, Ka, M, ldm, Kc, rs, C, ldc);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Small GEMM: C = alpha op(A) op(B) + beta C.  TB x TB output tiles, (TB/2)^2
// threads with 2 x 2 outputs each, K in slabs of 32 through shared memory.
// GB300's FP64 rate is low (about 2 FMA per clock and SM), so a double GEMM of
// a few hundred rows is bound by how many SMs take part: 16 x 16 tiles when
// 32 x 32 ones would leave SMs idle.
// ---------------------------------------------------------------------------
template <typename T, int TB>
__global__ void __launch_bounds__((TB / 2) * (TB / 2)) small_gemm_kernel(
    int ta, int tb, int M, int N, int K, T alpha, const T *__restrict__ A, int lda,
    const T *__restrict__ B, int ldb, T beta, T *__restrict__ C, int ldc,
    const int *__restrict__ skip) {
  if (skip && *skip) return;
  constexpr int NT = (TB / 2) * (TB / 2);
  __shared__ T As[TB][33];  // As[r][c] = op(A)[m0 + r][k0 + c]
  __shared__ T Bs[32][TB + 1];  // Bs[r][c] = op(B)[k0 + r][n0 + c]
  const int tid = threadIdx.x;
  const int ty = tid / (TB / 2), tx = tid % (TB / 2);
  const int m0 = blockIdx.y * TB, n0 = blockIdx.x * TB;
  T acc[2][2] = {{0, 0}, {0, 0}};
  for (int k0 = 0; k0 < K; k0 += 32) {
    for (int e = tid; e < TB * 32; e += NT) {
      // A slab: TB rows x 32 k; with ta the k index runs fastest in memory
      // order of A's rows, so walk (k, m) with m fastest for coalescing
      {
        int r, c;
        if (ta) { c = e / TB; r = e % TB; } else { r = e / 32; c = e % 32; }
        const int m = m0 + r, k = k0 + c;
        T av = 0;
        if (m < M && k < K) av = ta ? A[(int64_t)k * lda + m] : A[(int64_t)m * lda + k];
        As[r][c] = av;
      }
      {
        int r, c;
        if (tb) { c = e / 32; r = e % 32; } else { r = e / TB; c = e % TB; }
        const int kb = k0 + r, nb = n0 + c;
        T bv = 0;
        if (kb < K && nb < N) bv = tb ? B[(int64_t)nb * ldb + kb] : B[(int64_t)kb * ldb + nb];
        Bs[r][c] = bv;
      }
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < 32; ++kk) {
      const T a0 = As[ty * 2][kk], a1 = As[ty * 2 + 1][kk];
      const T b0 = Bs[kk][tx * 2], b1 = Bs[kk][tx * 2 + 1];
      acc[0][0] += a0 * b0;
      acc[0][1] += a0 * b1;
      acc[1][0] += a1 * b0;
      acc[1][1] += a1 * b1;
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int m = m0 + ty * 2 + i, nn = n0 + tx * 2 + j;
      if (m < M && nn < N) {
        T *c = C + (int64_t)m * ldc + nn;
        *c = alpha * acc[i][j] + (beta == T(0) ? T(0) : beta * *c);
      }
    }
}

template <typename T>
cudaError_t launch_small_gemm(bool ta, bool tb, int32_t M, int32_t N, int32_t K, T alpha,
                              const T *A, int32_t lda, const T *B, int32_t ldb, T beta, T *C,
                              int32_t ldc, cudaStream_t st, const int *skip) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  ProfScope ps_(K_SMALL_GEMM, st);
  if ((int64_t)ceil_div(N, 32) * ceil_div(M, 32) < 2 * (int64_t)sm_count()) {
    dim3 grid((unsigned)ceil_div(N, 16), (unsigned)ceil_div(M, 16));
    small_gemm_kernel<T, 16><<<grid, 64, 0, st>>>(ta ? 1 : 0, tb ? 1 : 0, M, N, K, alpha, A, lda,
                                                  B, ldb, beta, C, ldc, skip);
  } else {
    dim3 grid((unsigned)ceil_div(N, 32), (unsigned)ceil_div(M, 32));
    small_gemm_kernel<T, 32><<<grid, 256, 0, st>>>(ta ? 1 : 0, tb ? 1 : 0, M, N, K, alpha, A, lda,
                                                   B, ldb, beta, C, ldc, skip);
  }
  return cudaGetLastError();
}
template cudaError_t launch_small_gemm<float>(bool, bool, int32_t, int32_t, int32_t, float,
                                              const float *, int32_t, const float *, int32_t, float,
                                              float *, int32_t, cudaStream_t, const int *);
template cudaError_t launch_small_gemm<double>(bool, bool, int32_t, int32_t, int32_t, double,
                                               const double *, int32_t, const double *, int32_t,
                                               double, double *, int32_t, cudaStream_t, const int *);

// ---------------------------------------------------------------------------
// Symmetric eigendecomposition, one CTA of 1024 threads.
//  1. Householder tridiagonalization: for column k, the reflector
//     H_k = I - 2 v v^T (|v| = 1) maps A[k+1:, k] to alpha e_1; the trailing
//     block becomes A - v w^T - w v^T with p = A v, w = 2p - 2(v^T p) v.
//     v is kept in column k below the subdiagonal.
//  2. Implicit symmetric QR steps with the Wilkinson shift on the tridiagonal
//     (d, e), chasing the bulge with Givens rotations from the top of the
//     unreduced block to its bottom; thread 0 computes each sweep's rotations,
//     all threads apply them to the rows of Z^T (eigenvector j = row j).
//  3. Back-transformation V^T = Z^T H_{n-3} ... H_0, then V = (V^T)^T.
// scratch: n*n (Z^T) + 4n.
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  T s = 0;
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : T(0);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[32] = s;
  }
  __syncthreads();
  return red[32];
}

template <typename T>
__device__ __forceinline__ T eps_of();
template <>
__device__ __forceinline__ float eps_of<float>() {
  return FLT_EPSILON;
}
template <>
__device__ __forceinline__ double eps_of<double>() {
  return DBL_EPSILON;
}

constexpr int kMaxEigN = 1024;

template <typename T>
__global__ void __launch_bounds__(1024) sym_eig_kernel(T *A, int n, int lda, T *w, T *V, int ldv,
                                                       T *scratch, Ctrl *ctrl) {
  __shared__ T red[33];
  __shared__ int sweep_lm[2];
  extern __shared__ __align__(16) unsigned char eig_smem[];
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  T *Zt = scratch;                               // n x n, global
  T *d = reinterpret_cast<T *>(eig_smem);        // n
  T *e = d + n;                                  // n
  T *p = e + n;                                  // n
  T *vv = p + n;                                 // n
  T *rc = vv + n;                                // n  rotation cosines of a sweep
  T *rs = rc + n;                                // n  rotation sines

  // ---- 1. tridiagonalization
  for (int k = 0; k + 2 < n; ++k) {
    const int m0 = k + 1;
    T part = 0;
    for (int i = m0 + tid; i < n; i += nt) {
      const T x = A[(int64_t)i * lda + k];
      vv[i] = x;
      part += x * x;
    }
    const T x0 = A[(int64_t)m0 * lda + k];
    const T sigma = block_sum(part, red);
    const T tail = sigma - x0 * x0;
    if (!(tail > T(0))) {  // already reduced (or zero column): H_k = I
      for (int i = m0 + tid; i < n; i += nt) A[(int64_t)i * lda + k] = T(0);
      if (tid == 0) {
        e[k] = x0;
        d[k] = A[(int64_t)k * lda + k];
      }
      __syncthreads();
      continue;
    }
    const T alpha = (x0 >= T(0)) ? -sqrt(sigma) : sqrt(sigma);
    const T inv_vnorm = T(1) / sqrt(T(2) * (sigma - x0 * alpha));
    for (int i = m0 + tid; i < n; i += nt) vv[i] = ((i == m0) ? (vv[i] - alpha) : vv[i]) * inv_vnorm;
    __syncthreads();
    // p = A' v (warp per row)
    for (int i = m0 + warp; i < n; i += nwarps) {
      T s = 0;
      for (int j = m0 + lane; j < n; j += 32) s += A[(int64_t)i * lda + j] * vv[j];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) p[i] = s;
    }
    __syncthreads();
    T part2 = 0;
    for (int i = m0 + tid; i < n; i += nt) part2 += vv[i] * p[i];
    const T beta = block_sum(part2, red);
    for (int i = m0 + tid; i < n; i += nt) p[i] = T(2) * p[i] - T(2) * beta * vv[i];  // w
    __syncthreads();
    // trailing update, warp per row, lanes over columns (no index division)
    for (int i = m0 + warp; i < n; i += nwarps) {
      const T vi = vv[i], pi = p[i];
      T *ai = A + (int64_t)i * lda;
      for (int j = m0 + lane; j < n; j += 32) ai[j] -= vi * p[j] + pi * vv[j];
    }
    for (int i = m0 + tid; i < n; i += nt) A[(int64_t)i * lda + k] = vv[i];
    if (tid == 0) {
      e[k] = alpha;
      d[k] = A[(int64_t)k * lda + k];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      d[n - 2] = A[(int64_t)(n - 2) * lda + (n - 2)];
      e[n - 2] = A[(int64_t)(n - 1) * lda + (n - 2)];
    }
    d[n - 1] = A[(int64_t)(n - 1) * lda + (n - 1)];
    e[n - 1] = T(0);
  }
  for (int64_t q = tid; q < (int64_t)n * n; q += nt) Zt[q] = (q / n == q % n) ? T(1) : T(0);
  __syncthreads();

  // ---- 2. implicit QR sweeps (thread 0 computes, everyone applies)
  const T eps = eps_of<T>();
  int hi_idx = n - 1;
  int sweeps = 0;
  for (;;) {
    if (tid == 0) {
      int lq = -1, mq = -1;
      while (hi_idx > 0) {
        const T tol = eps * (fabs(d[hi_idx - 1]) + fabs(d[hi_idx]));
        if (fabs(e[hi_idx - 1]) <= tol) {
          e[hi_idx - 1] = T(0);
          --hi_idx;
          continue;
        }
        int lo = hi_idx - 1;
        while (lo > 0 && fabs(e[lo - 1]) > eps * (fabs(d[lo - 1]) + fabs(d[lo]))) --lo;
        if (lo > 0) e[lo - 1] = T(0);
        lq = lo;
        mq = hi_idx;
        break;
      }
      if (lq >= 0 && ++sweeps > 40 * n) {
        record_error(ctrl, SNE_ERR_NUMERIC, W_EIG);
        lq = -1;
      }
      if (lq >= 0) {
        const T dd = (d[mq - 1] - d[mq]) * T(0.5);
        const T bb = e[mq - 1];
        const T den = dd + (dd >= T(0) ? T(1) : T(-1)) * hypot(dd, bb);
        const T mu = d[mq] - ((den != T(0)) ? bb * bb / den : T(0));
        T x = d[lq] - mu, y = e[lq];
        T bulge = T(0);
        for (int k = lq; k < mq; ++k) {
          if (k > lq) {
            x = e[k - 1];
            y = bulge;
          }
          const T r = hypot(x, y);
          T c = T(1), s = T(0);
          if (r != T(0)) {
            const T ir = T(1) / r;
            c = x * ir;
            s = y * ir;
          }
          if (k > lq) e[k - 1] = r;
          const T a = d[k], a2 = d[k + 1], b = e[k];
          const T cc = c * c, ss = s * s, cs = c * s;
          d[k] = cc * a + T(2) * cs * b + ss * a2;
          d[k + 1] = ss * a - T(2) * cs * b + cc * a2;
          e[k] = cs * (a2 - a) + (cc - ss) * b;
          if (k + 1 < mq) {
            bulge = s * e[k + 1];
            e[k + 1] = c * e[k + 1];
          }
          rc[k] = c;
          rs[k] = s;
        }
      }
      sweep_lm[0] = lq;
      sweep_lm[1] = mq;
    }
    __syncthreads();
    const int lq = sweep_lm[0], mq = sweep_lm[1];
    if (lq < 0) break;
    // apply the sweep to the rows of Z^T (thread r owns entry r of every row);
    // loads are issued 8 rotations ahead of their use
    for (int r = tid; r < n; r += nt) {
      T zk = Zt[(int64_t)lq * n + r];
      int k = lq;
      for (; k + 8 <= mq; k += 8) {
        T z1[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) z1[u] = Zt[(int64_t)(k + 1 + u) * n + r];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const T c = rc[k + u], s = rs[k + u];
          Zt[(int64_t)(k + u) * n + r] = c * zk + s * z1[u];
          zk = -s * zk + c * z1[u];
        }
      }
      for (; k < mq; ++k) {
        const T c = rc[k], s = rs[k];
        const T zk1 = Zt[(int64_t)(k + 1) * n + r];
        Zt[(int64_t)k * n + r] = c * zk + s * zk1;
        zk = -s * zk + c * zk1;
      }
      Zt[(int64_t)mq * n + r] = zk;
    }
    __syncthreads();
  }
  for (int i = tid; i < n; i += nt) w[i] = d[i];

  // ---- 3. back-transformation: V^T = Z^T H_{n-3} ... H_0 (warp per row j)
  for (int k = n - 3; k >= 0; --k) {
    const int m0 = k + 1;
    for (int i = m0 + tid; i < n; i += nt) vv[i] = A[(int64_t)i * lda + k];
    __syncthreads();
    for (int j = warp; j < n; j += nwarps) {
      T s = 0;
      for (int i = m0 + lane; i < n; i += 32) s += Zt[(int64_t)j * n + i] * vv[i];
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      s *= T(2);
      for (int i = m0 + lane; i < n; i += 32) Zt[(int64_t)j * n + i] -= s * vv[i];
    }
    __syncthreads();
  }
  for (int64_t q = tid; q < (int64_t)n * n; q += nt) {
    const int r = (int)(q / n), c = (int)(q % n);
    V[(int64_t)r * ldv + c] = Zt[(int64_t)c * n + r];
  }
}

template <typename T>
cudaError_t launch_sym_eig(T *A, int32_t n, int32_t lda, T *w, T *V, int32_t ldv, void *scratch_v,
                           Ctrl *ctrl, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (n > kMaxEigN) return cudaErrorInvalidValue;
  if (n <= kFastEigMaxN) return launch_sym_eig_fast(A, n, lda, w, V, ldv, scratch_v, ctrl, st);
  T *scratch = static_cast<T *>(scratch_v);
  const size_t smem = (size_t)6 * n * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(sym_eig_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  ProfScope ps_(K_EIG, st);
  sym_eig_kernel<T><<<1, 1024, smem, st>>>(A, n, lda, w, V, ldv, scratch, ctrl);
  return cudaGetLastError();
}
template cudaError_t launch_sym_eig<float>(float *, int32_t, int32_t, float *, float *, int32_t,
                                           void *, Ctrl *, cudaStream_t);
template cudaError_t launch_sym_eig<double>(double *, int32_t, int32_t, double *, double *, int32_t,
                                            void *, Ctrl *, cudaStream_t);

// perm[j] = index of the j-th largest key (|w| or w), ties by index (rank sort).
template <typename T>
__global__ void eig_order_kernel(const T *w, int n, int by_abs, int32_t *perm) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const T ki = by_abs ? fabs(w[i]) : w[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const T kj = by_abs ? fabs(w[j]) : w[j];
      rank += (kj > ki) || (kj == ki && j < i);
    }
    perm[rank] = i;
  }
}

template <typename T>
cudaError_t launch_eig_order(const T *w, int32_t n, bool by_abs, int32_t *perm, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  ProfScope ps_(K_MISC, st);
  eig_order_kernel<T><<<1, 1024, 0, st>>>(w, n, by_abs ? 1 : 0, perm);
  return cudaGetLastError();
}
template cudaError_t launch_eig_order<float>(const float *, int32_t, bool, int32_t *, cudaStream_t);
template cudaError_t launch_eig_order<double>(const double *, int32_t, bool, int32_t *,
                                              cudaStream_t);

// ---------------------------------------------------------------------------
// Elementwise helpers
// ---------------------------------------------------------------------------
__global__ void d2f_kernel(const double *src, int rows, int cols, int lds, float *dst, int ldd) {
  const int64_t total = (int64_t)rows * cols;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(q / cols), c = (int)(q % cols);
    dst[(int64_t)r * ldd + c] = (float)src[(int64_t)r * lds + c];
  }
}
__global__ void f2d_kernel(const float *src, int rows, int cols, int lds, double *dst, int ldd) {
  const int64_t total = (int64_t)rows * cols;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(q / cols), c = (int)(q % cols);
    dst[(int64_t)r * ldd + c] = (double)src[(int64_t)r * lds + c];
  }
}
cudaError_t launch_d2f(const double *src, int32_t rows, int32_t cols, int32_t lds, float *dst,
                       int32_t ldd, cudaStream_t st) {
  const int64_t total = (int64_t)rows * cols;
  if (total <= 0) return cudaSuccess;
  ProfScope ps_(K_MISC, st);
  d2f_kernel<<<(unsigned)min64(1024, (total + 255) / 256), 256, 0, st>>>(src, rows, cols, lds,
                                                                               dst, ldd);
  return cudaGetLastError();
}
cudaError_t launch_f2d(const float *src, int32_t rows, int32_t cols, int32_t lds, double *dst,
                       int32_t ldd, cudaStream_t st) {
  const int64_t total = (int64_t)rows * cols;
  if (total <= 0) return cudaSuccess;
  ProfScope ps_(K_MISC, st);
  f2d_kernel<<<(unsigned)min64(1024, (total + 255) / 256), 256, 0, st>>>(src, rows, cols, lds,
                                                                               dst, ldd);
  return cudaGetLastError();
}

__global__ void symmetrize_kernel(double *A, int n, int lda) {
  const int64_t total = (int64_t)n * n;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(q / n), c = (int)(q % n);
    if (c > r) {
      const double v = 0.5 * (A[(int64_t)r * lda + c] + A[(int64_t)c * lda + r]);
      A[(int64_t)r * lda + c] = v;
      A[(int64_t)c * lda + r] = v;
    }
  }
}
cudaError_t launch_symmetrize(double *A, int32_t n, int32_t lda, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  ProfScope ps_(K_MISC, st);
  symmetrize_kernel<<<(unsigned)min64(1024, ((int64_t)n * n + 255) / 256), 256, 0, st>>>(A, n,
                                                                                               lda);
  return cudaGetLastError();
}

__global__ void check_finite_kernel(const float *x, int64_t count, Ctrl *ctrl, int where) {
  bool bad = false;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count;
       q += (int64_t)gridDim.x * blockDim.x)
    bad |= !isfinite(x[q]);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) record_error(ctrl, SNE_ERR_NUMERIC, where);
}
cudaError_t launch_check_finite_f(const float *x, int64_t count, Ctrl *ctrl, int32_t where,
                                  cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  ProfScope ps_(K_MISC, st);
  check_finite_kernel<<<(unsigned)min64(sm_count() * 4, (count + 255) / 256), 256, 0, st>>>(
      x, count, ctrl, where);
  return cudaGetLastError();
}

}  // namespace sne
