// Small symmetric eigensolver and Cholesky factorization for the Gram and
// reduced matrices of Alg. 4 and Alg. 5 (sizes up to a few hundred).
//
// FP32 eigendecomposition: cyclic Jacobi with the round-robin ("circle")
// ordering.  A round pairs all indices into m/2 disjoint pairs (m = n rounded
// up to even); the m/2 rotations are computed from the current matrix and
// applied at once as independent 2x2 blocks J_i^T A_(i,j) J_j, with the
// symmetric matrix packed (lower triangle) in shared memory of one CTA.  A
// sweep is m-1 rounds; sweeps stop when every off-diagonal element is below
// 2 eps * max(sqrt(|a_pp a_qq|), |A|_F / (2 sqrt(n))).  Each round's rotations are recorded; a second,
// multi-CTA kernel accumulates V = J_1 J_2 ... row block by row block.
//
// FP64 eigendecomposition (Rayleigh-Ritz, svd(W)): the FP32 result refined in
// FP64 by the iteration of Ogita and Aishima ("Iterative refinement for
// symmetric eigenvalue decomposition", Japan J. Indust. Appl. Math. 35, 2018):
// R = I - X^T X, S = X^T A X, lambda_i = s_ii / (1 - r_ii),
// delta = 2 (|S - diag(lambda)| + |A| |R|) (Frobenius norms, floored at
// 1e-4 max |lambda|), E_ij = (s_ij + lambda_j r_ij) / (lambda_j - lambda_i) when
// |lambda_i - lambda_j| > delta, else r_ij / 2, X <- X + X E; at most six
// iterations, the rest skipped on the device once max |E| < 1e-14.  Clusters
// (pairs closer than the floor) are then resolved exactly by a small FP64
// Jacobi on each cluster's block of X^T A X.
#include <cfloat>
#include <climits>
#include <cmath>
#include <cstdlib>

#include <algorithm>

#include "sne_internal.cuh"

namespace sne {

constexpr int kJacobiMaxSweeps = 30;
constexpr int kRefineSteps = 6;
constexpr double kClusterFloor = 1e-4;  // eigenvalue gaps below this x max|lambda| form clusters

struct Rot {
  int p, q;
  float c, s;
};

__device__ __forceinline__ int packed_lower(int a, int b) {  // a >= b
  return a * (a + 1) / 2 + b;
}
__device__ __forceinline__ int packed_any(int a, int b) {
  return a >= b ? packed_lower(a, b) : packed_lower(b, a);
}

// circle method: pair t of round r among m players (m even)
__device__ __forceinline__ void rr_pair(int m, int r, int t, int *p, int *q) {
  int a, b;
  if (t == 0) {
    a = 0;
    b = 1 + (r % (m - 1));
  } else {
    a = 1 + ((r + t) % (m - 1));
    b = 1 + ((r + m - 1 - t) % (m - 1));
  }
  *p = min(a, b);
  *q = max(a, b);
}

size_t jacobi_rot_capacity(int n) {
  const int m = n + (n & 1);
  return (size_t)kJacobiMaxSweeps * (m - 1) * (m / 2);
}

__global__ void __launch_bounds__(1024) jacobi_kernel(const float *__restrict__ A, int n, int lda,
                                                      float *__restrict__ w, Rot *__restrict__ rot,
                                                      int *__restrict__ nrounds, Ctrl *ctrl) {
  extern __shared__ __align__(16) float jsm[];
  const int m = n + (n & 1);
  const int P = m / 2;
  float *Ap = jsm;                                   // n(n+1)/2
  float *rc = Ap + n * (n + 1) / 2;                  // P
  float *rs = rc + P;                                // P
  int *rp = reinterpret_cast<int *>(rs + P);         // P
  int *rq = rp + P;                                  // P
  __shared__ unsigned int off_bits;
  __shared__ float offmax_final;
  __shared__ float fro_sq;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < n * (n + 1) / 2; e += nt) {
    const int a = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
    int aa = a;
    while (aa * (aa + 1) / 2 > e) --aa;
    while ((aa + 1) * (aa + 2) / 2 <= e) ++aa;
    const int b = e - aa * (aa + 1) / 2;
    Ap[e] = A[(int64_t)aa * lda + b];
  }
  if (tid == 0) fro_sq = 0.0f;
  __syncthreads();
  {
    float part = 0.0f;
    for (int e = tid; e < n * (n + 1) / 2; e += nt) {
      const int a = (int)((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
      int aa = a;
      while (aa * (aa + 1) / 2 > e) --aa;
      while ((aa + 1) * (aa + 2) / 2 <= e) ++aa;
      const float v = Ap[e];
      part += (e - aa * (aa + 1) / 2 == aa) ? v * v : 2.0f * v * v;
    }
    for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
    if ((tid & 31) == 0) atomicAdd(&fro_sq, part);
  }
  __syncthreads();
  const float tol = 2.0f * FLT_EPSILON;
  // a pair is rotated while |a_pq| exceeds tol * sqrt(|a_pp a_qq|) (relative
  // accuracy for graded matrices) and also eps * rms(lambda) = eps |A|_F /
  // sqrt(n): below that the element is FP32 rounding noise
  const float denom_floor = 0.5f * sqrtf(fro_sq / (float)n);
  const int warp_id = tid >> 5, lane_id = tid & 31, nwarps = nt >> 5;
  int round = 0;
  int sweep = 0;
  for (; sweep < kJacobiMaxSweeps; ++sweep) {
    if (tid == 0) off_bits = 0u;
    __syncthreads();
    for (int r = 0; r < m - 1; ++r) {
      for (int t = tid; t < P; t += nt) {
        int p, q;
        rr_pair(m, r, t, &p, &q);
        float c = 1.0f, s = 0.0f;
        if (q < n) {
          const float apq = Ap[packed_lower(q, p)];
          const float app = Ap[packed_lower(p, p)], aqq = Ap[packed_lower(q, q)];
          const float scale = fmaxf(sqrtf(fabsf(app * aqq)), denom_floor);
          const float rel = (apq == 0.0f) ? 0.0f : (scale > 0.0f ? fabsf(apq) / scale : FLT_MAX);
          atomicMax(&off_bits, __float_as_uint(rel));
          if (rel > tol) {
            const float tau = (aqq - app) / (2.0f * apq);
            const float tt = (tau >= 0.0f ? 1.0f : -1.0f) / (fabsf(tau) + sqrtf(1.0f + tau * tau));
            c = rsqrtf(1.0f + tt * tt);
            s = tt * c;
          }
        }
        rc[t] = c;
        rs[t] = s;
        rp[t] = p;
        rq[t] = q;
        rot[(int64_t)round * P + t] = Rot{p, q, c, s};
      }
      __syncthreads();
      // 2x2 blocks (i, j), i <= j: warp per block row i, lanes over j
      for (int i = warp_id; i < P; i += nwarps) {
        const float c1 = rc[i], s1 = rs[i];
        const int p1 = rp[i], q1 = rq[i];
        for (int j = i + lane_id; j < P; j += 32) {
          const float c2 = rc[j], s2 = rs[j];
          if (s1 == 0.0f && s2 == 0.0f) continue;
          const int p2 = rp[j], q2 = rq[j];
          if (i == j) {
            if (q1 >= n) continue;
            const float app = Ap[packed_lower(p1, p1)], aqq = Ap[packed_lower(q1, q1)];
            const float apq = Ap[packed_lower(q1, p1)];
            const float t_ = s1 / c1;
            Ap[packed_lower(p1, p1)] = app - t_ * apq;
            Ap[packed_lower(q1, q1)] = aqq + t_ * apq;
            Ap[packed_lower(q1, p1)] = 0.0f;
            continue;
          }
          // block rows (p1, q1), columns (p2, q2): B' = J1^T B J2
          const bool v1q = q1 < n, v2q = q2 < n;
          const float b00 = Ap[packed_any(p1, p2)];
          const float b01 = v2q ? Ap[packed_any(p1, q2)] : 0.0f;
          const float b10 = v1q ? Ap[packed_any(q1, p2)] : 0.0f;
          const float b11 = (v1q && v2q) ? Ap[packed_any(q1, q2)] : 0.0f;
          const float x1 = c1 * b00 - s1 * b10, x2 = c1 * b01 - s1 * b11;
          const float x3 = s1 * b00 + c1 * b10, x4 = s1 * b01 + c1 * b11;
          Ap[packed_any(p1, p2)] = x1 * c2 - x2 * s2;
          if (v2q) Ap[packed_any(p1, q2)] = x1 * s2 + x2 * c2;
          if (v1q) Ap[packed_any(q1, p2)] = x3 * c2 - x4 * s2;
          if (v1q && v2q) Ap[packed_any(q1, q2)] = x3 * s2 + x4 * c2;
        }
      }
      __syncthreads();
      ++round;
    }
    const float om = __uint_as_float(off_bits);  // read by all before anyone resets it
    __syncthreads();
    if (om <= tol) {
      ++sweep;
      break;
    }
  }
  if (tid == 0) {
    offmax_final = __uint_as_float(off_bits);
    *nrounds = round;
  }
  __syncthreads();
  if (offmax_final > 1e-4f && tid == 0) record_error(ctrl, SNE_ERR_NUMERIC, W_EIG);
  for (int i = tid; i < n; i += nt) w[i] = Ap[packed_lower(i, i)];
}

// V = J_1 J_2 ... J_R.  Rows of V are independent (row i of V is e_i^T times
// the rotations), so one warp owns a row, held in shared memory, and applies
// each round's m/2 disjoint rotations across its lanes, with only warp-level
// synchronization between rounds.
constexpr int kVWarps = 8;
__global__ void __launch_bounds__(32 * kVWarps) jacobi_vectors_kernel(
    const Rot *__restrict__ rot, const int *__restrict__ nrounds, int n, float *__restrict__ V,
    int ldv) {
  extern __shared__ __align__(16) float vs[];  // kVWarps x n
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * kVWarps + warp;
  if (row >= n) return;
  float *v = vs + (size_t)warp * n;
  for (int c = lane; c < n; c += 32) v[c] = (c == row) ? 1.0f : 0.0f;
  __syncwarp();
  const int m = n + (n & 1);
  const int P = m / 2;
  const int R = *nrounds;
  for (int r = 0; r < R; ++r) {
    const Rot *rr = rot + (int64_t)r * P;
    for (int t = lane; t < P; t += 32) {
      const Rot g = rr[t];
      if (g.s == 0.0f || g.q >= n) continue;
      const float vp = v[g.p], vq = v[g.q];
      v[g.p] = g.c * vp - g.s * vq;
      v[g.q] = g.s * vp + g.c * vq;
    }
    __syncwarp();
  }
  for (int c = lane; c < n; c += 32) V[(int64_t)row * ldv + c] = v[c];
}

cudaError_t launch_jacobi_f32(const float *A, int32_t n, int32_t lda, float *w, float *V, int32_t ldv,
                              void *rot_scratch, int *nrounds, Ctrl *ctrl, cudaStream_t st) {
  const int m = n + (n & 1);
  const size_t smem = ((size_t)n * (n + 1) / 2 + 2 * (m / 2)) * sizeof(float) + 2 * (m / 2) * sizeof(int);
  cudaError_t e = cudaFuncSetAttribute(jacobi_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  {
    ProfScope ps_(K_EIG, st);
    jacobi_kernel<<<1, 1024, smem, st>>>(A, n, lda, w, reinterpret_cast<Rot *>(rot_scratch), nrounds,
                                         ctrl);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const size_t vsm = (size_t)kVWarps * n * sizeof(float);
  e = cudaFuncSetAttribute(jacobi_vectors_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)vsm);
  if (e != cudaSuccess) return e;
  {
    ProfScope ps_(K_EIG, st);
    jacobi_vectors_kernel<<<(n + kVWarps - 1) / kVWarps, 32 * kVWarps, vsm, st>>>(
        reinterpret_cast<const Rot *>(rot_scratch), nrounds, n, V, ldv);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Ogita-Aishima refinement step (FP64), over many CTAs: given T1 = X^T X and
// S = X^T A X, oa_stats_kernel forms lambda_i = S_ii / T1_ii and the sums
// |S - diag(lambda)|_F^2, |A|_F^2, |I - T1|_F^2 and max |lambda| (acc[0..3],
// zeroed before the launch); oa_apply_kernel writes the correction E over T1
// and the largest |E| (acc[4], as bits); oa_done_kernel marks the refinement
// converged when that correction is at rounding level (this step is applied,
// later ones are skipped).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void atomic_max_nonneg(double *addr, double v) {
  // non-negative doubles order like their bit patterns
  atomicMax(reinterpret_cast<unsigned long long *>(addr), (unsigned long long)__double_as_longlong(v));
}

__global__ void __launch_bounds__(256) oa_stats_kernel(const double *T1, const double *S,
                                                       const double *A, int lda, int n,
                                                       double *lam, double *acc, const int *done) {
  __shared__ double red[3][8];
  __shared__ double rmax[8];
  if (*done) return;
  const int tid = threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double so = 0.0, sa = 0.0, sr = 0.0, lmax = 0.0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + tid; q < (int64_t)n * n; q += stride) {
    const int i = (int)(q / n), j = (int)(q % n);
    double s = S[q];
    double r = -T1[q];
    if (i == j) {
      const double li = S[q] / T1[q];
      lam[i] = li;
      lmax = fmax(lmax, fabs(li));
      s -= li;
      r += 1.0;
    }
    so += s * s;
    const double av = A[(int64_t)i * lda + j];
    sa += av * av;
    sr += r * r;
  }
  for (int o = 16; o > 0; o >>= 1) {
    so += __shfl_xor_sync(0xffffffffu, so, o);
    sa += __shfl_xor_sync(0xffffffffu, sa, o);
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    lmax = fmax(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
  }
  if ((tid & 31) == 0) {
    red[0][tid >> 5] = so;
    red[1][tid >> 5] = sa;
    red[2][tid >> 5] = sr;
    rmax[tid >> 5] = lmax;
  }
  __syncthreads();
  if (tid == 0) {
    double a = 0, b = 0, c = 0, m = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      a += red[0][w];
      b += red[1][w];
      c += red[2][w];
      m = fmax(m, rmax[w]);
    }
    atomicAdd(&acc[0], a);
    atomicAdd(&acc[1], b);
    atomicAdd(&acc[2], c);
    atomic_max_nonneg(&acc[3], m);
  }
}

__global__ void __launch_bounds__(256) oa_apply_kernel(double *T1, const double *S, int n,
                                                       const double *lam, double *acc,
                                                       const int *done) {
  __shared__ double rmax[8];
  if (*done) return;
  const int tid = threadIdx.x;
  // pairs closer than 1e-4 max|lambda| are treated as one cluster (only
  // re-orthogonalized).  The FP32 start mixes such a pair by an angle of up
  // to eps_32 |A| / gap, too large for the first-order correction to
  // converge; left unresolved, the pair's residual stays at the FP32
  // rounding level and its eigenvalues within the gap.
  const double delta = fmax(2.0 * (sqrt(acc[0]) + sqrt(acc[1]) * sqrt(acc[2])), kClusterFloor * acc[3]);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double emax = 0.0;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + tid; q < (int64_t)n * n; q += stride) {
    const int i = (int)(q / n), j = (int)(q % n);
    const double r = (i == j ? 1.0 : 0.0) - T1[q];
    const double gap = lam[j] - lam[i];
    double e;
    if (i != j && fabs(gap) > delta) e = (S[q] + lam[j] * r) / gap;
    else e = 0.5 * r;
    T1[q] = e;
    emax = fmax(emax, fabs(e));
  }
  for (int o = 16; o > 0; o >>= 1) emax = fmax(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  if ((tid & 31) == 0) rmax[tid >> 5] = emax;
  __syncthreads();
  if (tid == 0) {
    double m = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, rmax[w]);
    atomic_max_nonneg(&acc[4], m);
  }
}

__global__ void oa_done_kernel(const double *acc, int *done) {
  if (*done == 0 && acc[4] < 1e-14) *done = 1;
}

__global__ void add_inplace_kernel(double *X, const double *Y, int64_t count, const int *skip) {
  if (*skip) return;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count;
       q += (int64_t)gridDim.x * blockDim.x)
    X[q] += Y[q];
}

// ---------------------------------------------------------------------------
// Cholesky A = R^T R and R^-1 in shared memory (packed upper triangle).
// Row i of the packed upper triangle starts at i*n - i*(i-1)/2.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int packed_upper(int n, int i, int j) {  // j >= i
  return i * n - i * (i - 1) / 2 + (j - i);
}

constexpr int kCholColBufs = 32;  // warps that build columns of R^-1 at once

// Upper-triangle storage of the matrix being factored: packed in shared memory
// when it fits, else dense (row-major, leading dimension n) in global scratch.
template <typename T, bool PACKED>
struct CholStore {
  T *base;
  int n;
  __device__ __forceinline__ T &at(int i, int j) const {  // i <= j
    return PACKED ? base[packed_upper(n, i, j)] : base[(int64_t)i * n + j];
  }
  __device__ __forceinline__ T *row(int i) const {  // row(i)[c] = at(i, c), c >= i
    return PACKED ? base + packed_upper(n, i, i) - i : base + (int64_t)i * n;
  }
};

// A = R^T R and M = P R^-1 (one CTA).  Without pivoting (tol < 0), P = I and a
// non-positive or non-finite pivot is recorded as SNE_ERR_NUMERIC and replaced
// by 1.  With pivoting (tol >= 0; diagonal pivoting as in LAPACK's pstrf), step
// j swaps the largest remaining diagonal entry into place and the factorization
// stops at the numerical rank r, the first step whose largest remaining
// diagonal is at most tol times the largest diagonal of A; then M = P [R11^-1 0;
// 0 0], so that A^+ = M M^T on the range of A and Y M is an orthonormal basis of
// range(Y) padded with zero columns (A = Y^T Y).
template <typename T, bool PACKED>
__global__ void __launch_bounds__(1024) chol_inv_kernel(const T *__restrict__ A, int n, int lda,
                                                        T *__restrict__ Rinv, int ldi,
                                                        T *__restrict__ scratch, double tol,
                                                        Ctrl *ctrl) {
  extern __shared__ __align__(16) unsigned char csm[];
  T *packed = reinterpret_cast<T *>(csm);
  T *colbuf = packed + (PACKED ? (size_t)n * (n + 1) / 2 : 0);  // kCholColBufs x n (PACKED)
  T *dinv = colbuf + (PACKED ? (size_t)kCholColBufs * n : 0);   // n: 1 / R[i][i]
  int *perm = reinterpret_cast<int *>(dinv + n);
  __shared__ T piv;
  __shared__ T wmax[32];
  __shared__ int widx[32];
  __shared__ int rank_s;
  __shared__ double dmax0_s;
  const CholStore<T, PACKED> U{PACKED ? packed : scratch, n};
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const bool pivoting = tol >= 0.0;
  for (int i = 0; i < n; ++i)
    for (int j = i + tid; j < n; j += nt) U.at(i, j) = A[(int64_t)i * lda + j];
  for (int i = tid; i < n; i += nt) perm[i] = i;
  if (tid == 0) {
    rank_s = n;
    double m = 0.0;
    for (int i = 0; i < n; ++i) m = fmax(m, (double)A[(int64_t)i * lda + i]);
    dmax0_s = m;
  }
  __syncthreads();
  const double cut = tol * dmax0_s;
  for (int j = 0; j < n; ++j) {
    if (pivoting) {
      // largest remaining diagonal entry
      T best = -INFINITY;
      int bi = j;
      for (int i = j + tid; i < n; i += nt) {
        const T v = U.at(i, i);
        if (v > best) {
          best = v;
          bi = i;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > best || (ov == best && oi < bi)) {
          best = ov;
          bi = oi;
        }
      }
      if (lane == 0) {
        wmax[warp] = best;
        widx[warp] = bi;
      }
      __syncthreads();
      if (tid == 0) {
        T bv = wmax[0];
        int ib = widx[0];
        for (int w = 1; w < (nt >> 5); ++w)
          if (wmax[w] > bv || (wmax[w] == bv && widx[w] < ib)) {
            bv = wmax[w];
            ib = widx[w];
          }
        widx[0] = ib;
        if (!((double)bv > cut) || !isfinite((double)bv)) rank_s = j;
      }
      __syncthreads();
      if (rank_s == j) break;
      const int p = widx[0];
      if (p != j) {
        // swap rows and columns j and p of the symmetric matrix (and the
        // columns j, p of the rows of R already computed)
        for (int k = tid; k < n; k += nt) {
          if (k == j || k == p) continue;
          T &x = k < j ? U.at(k, j) : U.at(j, k);
          T &y = k < p ? U.at(k, p) : U.at(p, k);
          const T t = x;
          x = y;
          y = t;
        }
        if (tid == 0) {
          const T t = U.at(j, j);
          U.at(j, j) = U.at(p, p);
          U.at(p, p) = t;
          const int q = perm[j];
          perm[j] = perm[p];
          perm[p] = q;
        }
        __syncthreads();
      }
    }
    if (tid == 0) {
      T d = U.at(j, j);
      if (!(d > T(0)) || !isfinite((double)d)) {
        record_error(ctrl, SNE_ERR_NUMERIC, W_CHOL);
        d = T(1);
      }
      d = sqrt(d);
      U.at(j, j) = d;
      piv = T(1) / d;
    }
    __syncthreads();
    const T inv = piv;
    for (int c = j + 1 + tid; c < n; c += nt) U.at(j, c) *= inv;
    __syncthreads();
    // trailing update U(r, c) -= U(j, r) U(j, c), j < r <= c: warp per row r
    const T *ujrow = U.row(j);
    for (int rr = j + 1 + warp; rr < n; rr += (nt >> 5)) {
      const T ujr = ujrow[rr];
      T *urow = U.row(rr);
      for (int cc = rr + lane; cc < n; cc += 32) urow[cc] -= ujr * ujrow[cc];
    }
    __syncthreads();
  }
  const int r = rank_s;
  for (int i = tid; i < n; i += nt) dinv[i] = i < r ? T(1) / U.at(i, i) : T(0);
  if (!PACKED) {
    // the multi-CTA back substitution (chol_backsub_kernel) follows
    int *gperm = reinterpret_cast<int *>(scratch + (size_t)n * n + n);
    for (int i = tid; i < n; i += nt) {
      gperm[i] = perm[i];
      scratch[(size_t)n * n + i] = dinv[i];
    }
    if (tid == 0) gperm[n] = r;
    return;
  }
  __syncthreads();
  // X = R11^-1 (upper triangular, r x r) by back substitution, one warp per
  // column: X[j][j] = 1 / R[j][j], X[i][j] = -(sum_{k=i+1..j} R[i][k] X[k][j]) /
  // R[i][i] for i = j-1 .. 0; the warp splits each sum over its lanes.  Column j
  // of M is written to the rows perm[i].
  if (warp < kCholColBufs) {
    T *xcol = colbuf + (size_t)warp * n;
    for (int j = warp; j < n; j += min(nt >> 5, kCholColBufs)) {
      if (j < r) {
        if (lane == 0) xcol[j] = dinv[j];
        __syncwarp();
        for (int i = j - 1; i >= 0; --i) {
          const T *urow = U.row(i);
          T sum = 0;
          for (int k = i + 1 + lane; k <= j; k += 32) sum += urow[k] * xcol[k];
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
          if (lane == 0) xcol[i] = -sum * dinv[i];
          __syncwarp();
        }
      }
      for (int i = lane; i < n; i += 32)
        Rinv[(int64_t)perm[i] * ldi + j] = (j < r && i <= j) ? xcol[i] : T(0);
      __syncwarp();
    }
  }
}

// ---------------------------------------------------------------------------
// Pivoted FP64 Cholesky over a cluster of C CTAs (16 where the device allows
// clusters of that size, else 8; left-looking form of
// the diagonal pivoting of LAPACK's pstrf).  GB300 executes about two FP64
// fused multiply-adds per clock and SM, so one CTA cannot factor a 272 x 272
// matrix in less than a millisecond and a half; here the rows of L (A = L L^T,
// rows in the original order) are spread cyclically over the cluster's shared
// memory, row i in CTA i % C.  Step j:
//   each CTA proposes its largest remaining diagonal d_i (lowest index on
//   ties); after a cluster barrier every CTA reads the C proposals
//   through distributed shared memory and takes the same pivot p (stopping
//   at the numerical rank: d_p <= tol max_i A_ii, or not finite);
//   L(p, j) = sqrt(d_p); every CTA copies L(p, 0..j-1) from p's CTA and, for
//   its rows i not yet pivots, L(i, j) = (A(i, p) - sum_{k<j} L(i, k) L(p, k))
//   / L(p, j) and d_i -= L(i, j)^2 (a warp per row).
// In exact arithmetic the pivots and the factor are those of the right-looking
// kernel above.  The result goes to the same global scratch layout (R = L^T in
// pivot order, 1 / R_jj, the pivot order and the rank), for chol_backsub_kernel.
// The waits are the cluster barriers, whose CTAs are co-scheduled.
// ---------------------------------------------------------------------------
constexpr int kCholClThreads = 512;

__device__ __forceinline__ uint32_t cl_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cl_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::
                   : "memory");
}
__device__ __forceinline__ uint32_t cl_map(const void *p, uint32_t cta) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(cta));
  return r;
}
__device__ __forceinline__ double cl_ld_f64(const double *p, uint32_t cta) {
  double v;
  asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(cl_map(p, cta)) : "memory");
  return v;
}
__device__ __forceinline__ int cl_ld_s32(const int *p, uint32_t cta) {
  int v;
  asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(cl_map(p, cta)) : "memory");
  return v;
}

// larger value wins, then lower index
__device__ __forceinline__ void piv_better(double &v, int &i, double ov, int oi) {
  if (ov > v || (ov == v && oi < i)) {
    v = ov;
    i = oi;
  }
}

size_t chol_piv_cluster_smem(int n, int C) {
  const int nloc = (n + C - 1) / C;
  return ((size_t)nloc * n + n + nloc + 2) * sizeof(double) + (2 + 2 * (size_t)n) * sizeof(int) +
         (size_t)n + 16;
}

template <int C>
__global__ void __launch_bounds__(kCholClThreads) chol_piv_cluster_kernel(
    const double *__restrict__ A, int n, int lda, double *__restrict__ scratch, double tol) {
  extern __shared__ __align__(16) unsigned char ccm[];
  const int nloc = (n + C - 1) / C;
  double *L = reinterpret_cast<double *>(ccm);  // nloc x n: L[t n + k] = L(me + C t, k)
  double *rp = L + (size_t)nloc * n;            // n: L(p, k), k < j
  double *dloc = rp + n;                        // nloc: remaining diagonal of the local rows
  double *cval = dloc + nloc;                   // 2 slots (step parity): proposed d
  int *cidx = reinterpret_cast<int *>(cval + 2);  // 2 slots: proposed row
  int *perm = cidx + 2;                         // n: pivot order (replicated in every CTA)
  int *pos = perm + n;                          // n: position of each row in perm
  unsigned char *chosen = reinterpret_cast<unsigned char *>(pos + n);  // n (replicated)
  __shared__ double s_v;
  __shared__ int s_p;
  const uint32_t me = cl_rank();
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int t = tid; t < nloc; t += blockDim.x) {
    const int i = (int)me + C * t;
    dloc[t] = i < n ? A[(int64_t)i * lda + i] : 0.0;
  }
  for (int i = tid; i < n; i += blockDim.x) chosen[i] = 0;
  if (warp == 0) {  // max_i A_ii, the same in every CTA
    double m = 0.0;
    for (int i = lane; i < n; i += 32) m = fmax(m, A[(int64_t)i * lda + i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) s_v = m;
  }
  __syncthreads();
  const double cut = tol * s_v;
  int r = n;
  for (int j = 0; j < n; ++j) {
    const int slot = j & 1;
    if (warp == 0) {
      double v = -INFINITY;
      int ix = INT_MAX;
      for (int t = lane; t < nloc; t += 32) {
        const int i = (int)me + C * t;
        if (i < n && !chosen[i]) piv_better(v, ix, dloc[t], i);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        piv_better(v, ix, __shfl_xor_sync(0xffffffffu, v, o), __shfl_xor_sync(0xffffffffu, ix, o));
      if (lane == 0) {
        cval[slot] = v;
        cidx[slot] = ix;
      }
    }
    cl_sync();  // the proposals of step j are visible cluster-wide
    if (warp == 0) {
      double v = -INFINITY;
      int ix = INT_MAX;
      if (lane < C) {
        v = cl_ld_f64(&cval[slot], (uint32_t)lane);
        ix = cl_ld_s32(&cidx[slot], (uint32_t)lane);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
        piv_better(v, ix, __shfl_xor_sync(0xffffffffu, v, o), __shfl_xor_sync(0xffffffffu, ix, o));
      if (lane == 0) {
        s_v = v;
        s_p = ix;
      }
    }
    __syncthreads();
    const double dmax = s_v;
    const int p = s_p;
    if (!(dmax > cut) || !isfinite(dmax) || p < 0 || p >= n) {  // the same in every CTA
      r = j;
      break;
    }
    const double ljj = sqrt(dmax);
    const double inv = 1.0 / ljj;
    const uint32_t owner = (uint32_t)(p % C);
    const int tp = p / C;
    for (int k = tid; k < j; k += blockDim.x)
      rp[k] = owner == me ? L[(size_t)tp * n + k] : cl_ld_f64(&L[(size_t)tp * n + k], owner);
    if (tid == 0) {
      chosen[p] = 1;
      perm[j] = p;
      if (owner == me) L[(size_t)tp * n + j] = ljj;
    }
    __syncthreads();
    for (int t = warp; t < nloc; t += nw) {
      const int i = (int)me + C * t;
      if (i >= n || chosen[i]) continue;  // uniform for the warp
      const double *li = L + (size_t)t * n;
      double acc = 0.0;
      for (int k = lane; k < j; k += 32) acc = fma(li[k], rp[k], acc);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) {
        const double lij = (A[(int64_t)i * lda + p] - acc) * inv;
        L[(size_t)t * n + j] = lij;
        dloc[t] -= lij * lij;
      }
    }
    __syncthreads();
  }
  // positions r .. n-1: the rows never pivoted, in increasing order
  if (tid == 0) {
    int q = r;
    for (int i = 0; i < n; ++i)
      if (!chosen[i]) perm[q++] = i;
  }
  __syncthreads();
  for (int c = tid; c < n; c += blockDim.x) pos[perm[c]] = c;
  __syncthreads();
  double *R = scratch;  // R[k][c] = L(perm[c], k), k <= c < r
  double *dinv = scratch + (size_t)n * n;
  int *gperm = reinterpret_cast<int *>(dinv + n);
  for (int t = warp; t < nloc; t += nw) {
    const int i = (int)me + C * t;
    if (i >= n) continue;
    const int c = pos[i];
    if (c >= r) continue;
    for (int k = lane; k <= c; k += 32) R[(size_t)k * n + c] = L[(size_t)t * n + k];
    if (lane == 0) dinv[c] = 1.0 / L[(size_t)t * n + c];
  }
  if (me == 0) {
    for (int c = tid; c < n; c += blockDim.x) {
      gperm[c] = perm[c];
      if (c >= r) dinv[c] = 0.0;
    }
    if (tid == 0) gperm[n] = r;
  }
  cl_sync();  // no CTA leaves while another may still read its shared memory
}

// Back substitution for the factor left in global scratch by chol_inv_kernel
// (dense n x n R, then dinv[n], then perm[n] and the rank): one warp per
// column of M = P [R11^-1 0; 0 0], eight columns per CTA.
template <typename T>
__global__ void __launch_bounds__(256) chol_backsub_kernel(const T *__restrict__ scratch, int n,
                                                           T *__restrict__ Rinv, int ldi) {
  extern __shared__ __align__(16) unsigned char bsm[];
  T *xcol = reinterpret_cast<T *>(bsm) + (threadIdx.x >> 5) * n;
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (j >= n) return;
  const T *R = scratch;
  const T *dinv = scratch + (size_t)n * n;
  const int *perm = reinterpret_cast<const int *>(dinv + n);
  const int r = perm[n];
  if (j < r) {
    if (lane == 0) xcol[j] = dinv[j];
    __syncwarp();
    for (int i = j - 1; i >= 0; --i) {
      const T *urow = R + (size_t)i * n;
      T sum = 0;
      for (int k = i + 1 + lane; k <= j; k += 32) sum += urow[k] * xcol[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
      if (lane == 0) xcol[i] = -sum * dinv[i];
      __syncwarp();
    }
  }
  for (int i = lane; i < n; i += 32)
    Rinv[(int64_t)perm[i] * ldi + j] = (j < r && i <= j) ? xcol[i] : T(0);
}

// Unpivoted Cholesky and R^-1 by blocks of kCB columns, packed upper triangle
// in shared memory (one CTA).
//  Factorization: within a panel of kCB columns every thread derives the pivot
//  d_j = sqrt(U(j, j)) itself (kept in diag[j]; U(j, j) is left as is), scales
//  row j and updates the panel's remaining rows, two block barriers per column;
//  the rows below the panel then take the panel's rank-kCB update in one pass
//  (kCB products per element in registers, one read-modify-write).
//  Inverse: X = R^-1 in place by block columns (as LAPACK's trtri): for block
//  column J, X_JJ = R_JJ^-1, then X(0:J, J) = -X(0:J, 0:J) R(0:J, J) X_JJ, using
//  the already inverted leading block.
constexpr int kCB = 16;

template <typename T>
__global__ void __launch_bounds__(1024) chol_inv_blocked_kernel(const T *__restrict__ A, int n,
                                                                int lda, T *__restrict__ Rinv,
                                                                int ldi, Ctrl *ctrl) {
  extern __shared__ __align__(16) unsigned char cbm[];
  T *U = reinterpret_cast<T *>(cbm);                    // packed upper, n(n+1)/2
  T *diag = U + (size_t)n * (n + 1) / 2;                // n: d_j = R[j][j]
  T *tb = diag + n;                                     // n x kCB scratch
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int nw = nt >> 5;
  auto at = [&](int i, int j) -> T & { return U[packed_upper(n, i, j)]; };
  for (int i = warp; i < n; i += nw) {
    T *ui = U + packed_upper(n, i, i) - i;
    for (int j = i + lane; j < n; j += 32) ui[j] = A[(int64_t)i * lda + j];
  }
  __syncthreads();
  // ---- factorization
  for (int j0 = 0; j0 < n; j0 += kCB) {
    const int j1 = min(n, j0 + kCB);
    for (int j = j0; j < j1; ++j) {
      T d2 = at(j, j);
      if (!(d2 > T(0)) || !isfinite((double)d2)) {
        if (tid == 0) record_error(ctrl, SNE_ERR_NUMERIC, W_CHOL);
        d2 = T(1);
      }
      const T d = sqrt(d2), inv = T(1) / d;
      if (tid == 0) diag[j] = d;
      T *uj = U + packed_upper(n, j, j) - j;
      for (int c = j + 1 + tid; c < n; c += nt) uj[c] *= inv;
      __syncthreads();
      // remaining rows of the panel: U(r, c) -= U(j, r) U(j, c), j < r < j1, c >= r
      for (int r = j + 1 + warp; r < j1; r += nw) {
        const T f = uj[r];
        T *ur = U + packed_upper(n, r, r) - r;
        for (int c = r + lane; c < n; c += 32) ur[c] -= f * uj[c];
      }
      __syncthreads();
    }
    // rows below the panel: U(r, c) -= sum_{k=j0}^{j1-1} U(k, r) U(k, c), j1 <= r <= c
    const int nk = j1 - j0;
    for (int r = j1 + warp; r < n; r += nw) {
      T ukr[kCB];
#pragma unroll
      for (int q = 0; q < kCB; ++q) ukr[q] = q < nk ? at(j0 + q, r) : T(0);
      T *ur = U + packed_upper(n, r, r) - r;
      for (int c = r + lane; c < n; c += 32) {
        T acc = 0;
#pragma unroll
        for (int q = 0; q < kCB; ++q)
          if (q < nk) acc += ukr[q] * U[packed_upper(n, j0 + q, j0 + q) - (j0 + q) + c];
        ur[c] -= acc;
      }
    }
    __syncthreads();
  }
  // ---- inverse in place: the diagonal of U becomes 1 / d
  for (int J0 = 0; J0 < n; J0 += kCB) {
    const int J1 = min(n, J0 + kCB), nb = J1 - J0;
    // X_JJ = R_JJ^-1 (one warp, column by column: x_jj = 1/d_j, x_ij for i < j)
    if (warp == 0) {
      for (int jj = 0; jj < nb; ++jj) {
        const int j = J0 + jj;
        // column j of X_JJ, rows i = j .. J0 (bottom-up), lane i - J0 holds x_ij
        T x = (lane == jj) ? T(1) / diag[j] : T(0);
        for (int ii = jj - 1; ii >= 0; --ii) {
          const int i = J0 + ii;
          // x_ij = -(sum_{k=i+1..j} R_ik x_kj) / d_i
          T part = (lane > ii && lane <= jj) ? at(i, J0 + lane) * x : T(0);
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
          if (lane == ii) x = -part / diag[i];
        }
        if (lane < nb) tb[(size_t)lane * kCB + jj] = x;  // X_JJ[ii][jj]
      }
    }
    __syncthreads();
    // T(0:J0, jj) = X(0:J0, 0:J0) R(0:J0, J0 + jj)  (X upper, in U's leading block,
    // whose diagonal already holds 1/d)
    T *tcol = tb + (size_t)kCB * kCB;  // J0 x kCB
    for (int e = tid; e < J0 * nb; e += nt) {
      const int i = e / nb, jj = e % nb;
      T acc = 0;
      for (int k = i; k < J0; ++k) acc += at(i, k) * at(k, J0 + jj);
      tcol[(size_t)i * kCB + jj] = acc;
    }
    __syncthreads();
    // X(0:J0, J) = -T X_JJ; X_JJ into the diagonal block
    for (int e = tid; e < J0 * nb; e += nt) {
      const int i = e / nb, jj = e % nb;
      T acc = 0;
      for (int k = 0; k <= jj; ++k) acc += tcol[(size_t)i * kCB + k] * tb[(size_t)k * kCB + jj];
      at(i, J0 + jj) = -acc;
    }
    for (int e = tid; e < nb * nb; e += nt) {
      const int ii = e / nb, jj = e % nb;
      if (jj >= ii) at(J0 + ii, J0 + jj) = tb[(size_t)ii * kCB + jj];
    }
    __syncthreads();
  }
  for (int i = warp; i < n; i += nw)
    for (int j = lane; j < n; j += 32) Rinv[(int64_t)i * ldi + j] = j >= i ? at(i, j) : T(0);
}

// ---------------------------------------------------------------------------
// FP32 Cholesky and inverse in 32 x 32 blocks (n <= 288), one CTA, for the
// orthonormalizations inside the power iteration of Alg. 5 (Q = Y R^-1 with
// Y^T Y = R^T R).  The upper triangle is held as nb (nb + 1) / 2 blocks of
// 32 x 33 floats (the padding keeps column walks free of bank conflicts);
// rows and columns past n are those of the identity, so the factor of the
// padded matrix is diag(R, I).
//   factor, panel p: the 1024 threads factor block (p, p) (thread per entry,
//   two barriers per column) and invert it, X_pp = R_pp^-1 (warp per column,
//   back substitution with the sums as warp reductions; kept for the
//   inverse); all warps form R_pq = X_pp^T A_pq for q > p and update the
//   trailing blocks A_qr -= R_pq^T R_pr with 4 x 4 register tiles.
//   inverse, block column j: T_i = sum_{m=i}^{j-1} X_im R_mj for i < j (X = R^-1,
//   columns < j already done), then X_ij = -T_i X_jj; two barriers per block
//   column.
// A non-positive or non-finite pivot records SNE_ERR_NUMERIC and is replaced
// by 1.
// ---------------------------------------------------------------------------
constexpr int kQB = 32;
constexpr int kQLd = 33;
constexpr int kQMaxNb = 9;

__device__ __forceinline__ int qblk(int nb, int bi, int bj) {  // bi <= bj
  return bi * nb - bi * (bi - 1) / 2 + (bj - bi);
}

size_t chol_quick_smem(int n) {
  const int nb = (n + kQB - 1) / kQB;
  return ((size_t)nb * (nb + 1) / 2 * kQB * kQLd + (size_t)nb * kQB * kQB) * sizeof(float);
}

__global__ void __launch_bounds__(1024) chol_inv_quick_kernel(const float *__restrict__ A, int n,
                                                              int lda, float *__restrict__ Rinv,
                                                              int ldi, Ctrl *ctrl) {
  extern __shared__ __align__(16) float qsm[];
  const int nb = (n + kQB - 1) / kQB;
  float *blk = qsm;                                              // triangle of blocks
  float *tmp = qsm + (size_t)nb * (nb + 1) / 2 * kQB * kQLd;     // nb blocks of 32 x 32
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  auto B = [&](int bi, int bj) { return blk + (size_t)qblk(nb, bi, bj) * kQB * kQLd; };
  // ---- load (upper triangle; identity past n)
  for (int bi = 0; bi < nb; ++bi)
    for (int bj = bi; bj < nb; ++bj) {
      float *b = B(bi, bj);
      for (int e = tid; e < kQB * kQB; e += blockDim.x) {
        const int r = e >> 5, c = e & 31;
        const int i = bi * kQB + r, j = bj * kQB + c;
        float v = 0.f;
        if (i < n && j < n) v = (i <= j) ? A[(int64_t)i * lda + j] : 0.f;
        else if (i == j) v = 1.f;
        b[r * kQLd + c] = v;
      }
    }
  __syncthreads();
  // ---- factorization
  for (int p = 0; p < nb; ++p) {
    float *bpp = B(p, p);
    // the diagonal block by all 1024 threads, thread (r, c) = (warp, lane):
    // step j scales row j (warp j) and updates the trailing triangle
    for (int j = 0; j < kQB; ++j) {
      if (warp == j) {
        float djj = bpp[j * kQLd + j];
        if (!(djj > 0.f) || !isfinite(djj)) {
          if (lane == 0) record_error(ctrl, SNE_ERR_NUMERIC, W_CHOL);
          djj = 1.f;
        }
        const float d = sqrtf(djj);
        __syncwarp();
        if (lane == j) bpp[j * kQLd + j] = d;
        else if (lane > j) bpp[j * kQLd + lane] /= d;
      }
      __syncthreads();
      if (warp > j && lane >= warp) bpp[warp * kQLd + lane] -= bpp[j * kQLd + warp] * bpp[j * kQLd + lane];
      __syncthreads();
    }
    // X_pp = R_pp^-1 into tmp block p: warp c takes column c, lane m holds
    // X[m][c]; row r = c .. 0: X[r][c] = (delta_rc - sum_{m>r} R[r][m] X[m][c]) / R[r][r]
    {
      float *xpp = tmp + (size_t)p * kQB * kQB;
      const int c = warp;
      float xm = 0.f;
      for (int r = c; r >= 0; --r) {
        float part = (lane > r && lane <= c) ? bpp[r * kQLd + lane] * xm : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
        const float xr = ((r == c ? 1.f : 0.f) - part) / bpp[r * kQLd + r];
        if (lane == r) xm = xr;
      }
      xpp[lane * kQB + c] = lane <= c ? xm : 0.f;
    }
    __syncthreads();
    // R_pq = X_pp^T A_pq, q > p, in 4 x 4 tiles (at most 8 blocks x 64 tiles,
    // one tile per thread): products first, then the blocks are overwritten
    {
      const float *xpp = tmp + (size_t)p * kQB * kQB;
      const int ntask = (nb - p - 1) * 64;
      float acc[4][4] = {};
      int q = 0, a0 = 0, b0 = 0;
      if (tid < ntask) {
        q = p + 1 + (tid >> 6);
        const int t = tid & 63;
        a0 = 4 * (t >> 3);
        b0 = 4 * (t & 7);
        const float *apq = B(p, q);
        // X_pp[m][a] = 0 for m > a: m runs to a0 + 3
        for (int m = 0; m < a0 + 4; ++m) {
          float av[4], bv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            av[u] = xpp[m * kQB + a0 + u];
            bv[u] = apq[m * kQLd + b0 + u];
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
        }
      }
      __syncthreads();
      if (tid < ntask) {
        float *dst = B(p, q);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) dst[(a0 + u) * kQLd + b0 + v] = acc[u][v];
      }
    }
    __syncthreads();
    // trailing update A_qr -= R_pq^T R_pr, p < q <= r, in 4 x 4 tiles
    {
      const int nrem = nb - p - 1;
      const int nblocks = nrem * (nrem + 1) / 2;
      for (int task = tid; task < nblocks * 64; task += blockDim.x) {
        const int bl = task >> 6, t = task & 63;
        // decode block bl -> (q, r), q <= r, among the remaining blocks
        int q = 0, rem = bl, len = nrem;
        while (rem >= len) {
          rem -= len;
          ++q;
          --len;
        }
        const int qq = p + 1 + q, rr = qq + rem;
        const int a0 = 4 * (t >> 3), b0 = 4 * (t & 7);
        const float *rq = B(p, qq), *rr_ = B(p, rr);
        float acc[4][4] = {};
#pragma unroll 4
        for (int m = 0; m < kQB; ++m) {
          float av[4], bv[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            av[u] = rq[m * kQLd + a0 + u];
            bv[u] = rr_[m * kQLd + b0 + u];
          }
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
        }
        float *dst = B(qq, rr);
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) dst[(a0 + u) * kQLd + b0 + v] -= acc[u][v];
      }
    }
    __syncthreads();
  }
  // ---- inverse X = R^-1, block column by block column
  for (int j = 0; j < nb; ++j) {
    const float *xjj = tmp + (size_t)j * kQB * kQB;  // X_jj from the factorization
    // T_i = sum_{m=i}^{j-1} X_im R_mj for i < j (into tmp block i), 4 x 4 tiles
    {
      for (int task = tid; task < j * 64; task += blockDim.x) {
        const int i = task >> 6, t = task & 63;
        const int a0 = 4 * (t >> 3), b0 = 4 * (t & 7);
        float acc[4][4] = {};
        for (int m = i; m < j; ++m) {
          const float *xim = B(i, m), *rmj = B(m, j);
#pragma unroll 4
          for (int kk = 0; kk < kQB; ++kk) {
            float av[4], bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              av[u] = xim[(a0 + u) * kQLd + kk];
              bv[u] = rmj[kk * kQLd + b0 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
          }
        }
        float *ti = tmp + (size_t)i * kQB * kQB;
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) ti[(a0 + u) * kQB + b0 + v] = acc[u][v];
      }
    }
    __syncthreads();
    // X_ij = -T_i X_jj (i < j), X_jj into block (j, j)
    for (int task = tid; task < (j + 1) * 64; task += blockDim.x) {
      const int i = task >> 6, t = task & 63;
      const int a0 = 4 * (t >> 3), b0 = 4 * (t & 7);
      float *dst = B(i, j);
      if (i == j) {
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) dst[(a0 + u) * kQLd + b0 + v] = xjj[(a0 + u) * kQB + b0 + v];
        continue;
      }
      const float *ti = tmp + (size_t)i * kQB * kQB;
      float acc[4][4] = {};
#pragma unroll 4
      for (int kk = 0; kk < kQB; ++kk) {
        float av[4], bv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          av[u] = ti[(a0 + u) * kQB + kk];
          bv[u] = xjj[kk * kQB + b0 + u];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) dst[(a0 + u) * kQLd + b0 + v] = -acc[u][v];
    }
    __syncthreads();
  }
  // ---- write R^-1 (upper triangular, zeros below)
  for (int e = tid; e < n * n; e += blockDim.x) {
    const int i = e / n, j = e % n;
    float v = 0.f;
    if (j >= i) v = B(i / kQB, j / kQB)[(i % kQB) * kQLd + (j % kQB)];
    Rinv[(int64_t)i * ldi + j] = v;
  }
}

template <typename T>
size_t chol_blocked_smem(int n) {
  return ((size_t)n * (n + 1) / 2 + n + (size_t)kCB * kCB + (size_t)n * kCB) * sizeof(T);
}

template <typename T>
size_t chol_inv_smem(int n, bool packed) {
  return ((packed ? (size_t)n * (n + 1) / 2 + (size_t)kCholColBufs * n : 0) + n) * sizeof(T) +
         (size_t)n * sizeof(int);
}

// The cluster kernel for pivoted FP64 factors, unless SNE_CHOL_CLUSTER=0 (for
// comparisons: the one-CTA kernel).
static bool chol_cluster_enabled() {
  static int on = -1;
  if (on < 0) {
    const char *v = getenv("SNE_CHOL_CLUSTER");
    on = (v && v[0] == '0') ? 0 : 1;
  }
  return on == 1;
}

// The blocked FP32 kernel above, unless SNE_CHOL_QUICK=0 (for comparisons).
static bool chol_quick_enabled() {
  static int on = -1;
  if (on < 0) {
    const char *v = getenv("SNE_CHOL_QUICK");
    on = (v && v[0] == '0') ? 0 : 1;
  }
  return on == 1;
}

template <typename T>
cudaError_t launch_chol_inverse(const T *A, int32_t n, int32_t lda, T *Rinv, int32_t ldi, T *scratch,
                                Ctrl *ctrl, cudaStream_t st, double tol) {
  if (n <= 0) return cudaSuccess;
  if (n > 1024) return cudaErrorInvalidValue;
  if (sizeof(T) == 4 && tol < 0.0 && n <= kQB * kQMaxNb && chol_quick_smem(n) <= 226 * 1024 &&
      chol_quick_enabled()) {
    const size_t smem = chol_quick_smem(n);
    cudaError_t e = cudaFuncSetAttribute(chol_inv_quick_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ProfScope ps_(K_CHOL, st);
    chol_inv_quick_kernel<<<1, 1024, smem, st>>>(reinterpret_cast<const float *>(A), n, lda,
                                                 reinterpret_cast<float *>(Rinv), ldi, ctrl);
    return cudaGetLastError();
  }
  if (tol < 0.0 && chol_blocked_smem<T>(n) <= 220 * 1024) {
    const size_t smem = chol_blocked_smem<T>(n);
    cudaError_t e = cudaFuncSetAttribute(chol_inv_blocked_kernel<T>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    ProfScope ps_(K_CHOL, st);
    chol_inv_blocked_kernel<T><<<1, 1024, smem, st>>>(A, n, lda, Rinv, ldi, ctrl);
    return cudaGetLastError();
  }
  const bool packed = chol_inv_smem<T>(n, true) <= 220 * 1024;
  if (!packed && !scratch) return cudaErrorInvalidValue;
  if (sizeof(T) == 8 && tol >= 0.0 && scratch && chol_cluster_enabled()) {
    // pivoted FP64: the cluster kernel (16 CTAs, else 8), then the multi-CTA
    // back substitution
    cudaError_t e = cudaErrorInvalidValue;
    bool launched = false;
    for (int C : {16, 8}) {
      const size_t csm = chol_piv_cluster_smem(n, C);
      if (csm > 220 * 1024) continue;
      auto kern = C == 16 ? chol_piv_cluster_kernel<16> : chol_piv_cluster_kernel<8>;
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csm);
      if (e != cudaSuccess) return e;
      if (C > 8) {
        if (cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
            cudaSuccess) {
          (void)cudaGetLastError();
          continue;
        }
      }
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(C, 1, 1);
      cfg.blockDim = dim3(kCholClThreads, 1, 1);
      cfg.dynamicSmemBytes = csm;
      cfg.stream = st;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributeClusterDimension;
      attr[0].val.clusterDim.x = C;
      attr[0].val.clusterDim.y = 1;
      attr[0].val.clusterDim.z = 1;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      if (C > 8) {
        // a cluster of 16 must fit the device (one GPC's SMs): ask first
        int ncl = 0;
        if (cudaOccupancyMaxActiveClusters(&ncl, kern, &cfg) != cudaSuccess || ncl < 1) {
          (void)cudaGetLastError();
          continue;
        }
      }
      ProfScope ps_(K_CHOL, st);
      e = cudaLaunchKernelEx(&cfg, kern, reinterpret_cast<const double *>(A), n, lda,
                             reinterpret_cast<double *>(scratch), tol);
      if (e != cudaSuccess) return e;
      launched = true;
      break;
    }
    if (launched) {
      ProfScope ps_(K_CHOL, st);
      const size_t bsmem = (size_t)8 * n * sizeof(T);
      e = cudaFuncSetAttribute(chol_backsub_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)bsmem);
      if (e != cudaSuccess) return e;
      chol_backsub_kernel<T><<<(n + 7) / 8, 256, bsmem, st>>>(scratch, n, Rinv, ldi);
      return cudaGetLastError();
    }
  }
  const size_t smem = chol_inv_smem<T>(n, packed);
  auto kern = packed ? chol_inv_kernel<T, true> : chol_inv_kernel<T, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  ProfScope ps_(K_CHOL, st);
  kern<<<1, 1024, smem, st>>>(A, n, lda, Rinv, ldi, scratch, tol, ctrl);
  e = cudaGetLastError();
  if (e != cudaSuccess || packed) return e;
  const size_t bsmem = (size_t)8 * n * sizeof(T);
  e = cudaFuncSetAttribute(chol_backsub_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)bsmem);
  if (e != cudaSuccess) return e;
  chol_backsub_kernel<T><<<(n + 7) / 8, 256, bsmem, st>>>(scratch, n, Rinv, ldi);
  return cudaGetLastError();
}
template cudaError_t launch_chol_inverse<float>(const float *, int32_t, int32_t, float *, int32_t,
                                                float *, Ctrl *, cudaStream_t, double);
template cudaError_t launch_chol_inverse<double>(const double *, int32_t, int32_t, double *, int32_t,
                                                 double *, Ctrl *, cudaStream_t, double);

// ---------------------------------------------------------------------------
// Public eigensolver entry (replaces the tridiagonal QR for n <= 320)
// scratch layout (bytes): see eig_scratch_bytes.
// ---------------------------------------------------------------------------
size_t eig_scratch_bytes(int n) {
  const size_t n2 = (size_t)n * n;
  return 256 + jacobi_rot_capacity(n) * sizeof(Rot) + 2 * n2 * sizeof(float) + n * sizeof(float) +
         3 * n2 * sizeof(double) + 1024;
}

// The FP32 eigensolver: Householder tridiagonalization, bisection and
// inverse iteration (tridiag.cu) for n >= 32, cyclic Jacobi for smaller n or
// when SNE_EIG_JACOBI=1 (for comparisons).  The scratch region of the Jacobi
// rotations holds the tridiagonal solver's arrays.
static bool eig_use_tridiag(int n) {
  static int jac = -1;
  if (jac < 0) {
    const char *v = getenv("SNE_EIG_JACOBI");
    jac = (v && v[0] == '1') ? 1 : 0;
  }
  return jac == 0 && n >= 32 && tri_eig_smem(n) <= 227 * 1024 &&
         tri_eig_scratch_floats(n) * sizeof(float) <= jacobi_rot_capacity(n) * sizeof(Rot);
}

static cudaError_t eig_f32(const float *A, int32_t n, int32_t lda, float *w, float *V, int32_t ldv,
                           char *base, Ctrl *ctrl, cudaStream_t st) {
  int *nrounds = reinterpret_cast<int *>(base);
  void *rot = base + 256;
  if (eig_use_tridiag(n))
    return launch_sym_eig_tridiag(A, n, lda, w, V, ldv, static_cast<float *>(rot), ctrl, st);
  return launch_jacobi_f32(A, n, lda, w, V, ldv, rot, nrounds, ctrl, st);
}

cudaError_t launch_sym_eig_fast(float *A, int32_t n, int32_t lda, float *w, float *V, int32_t ldv,
                                void *scratch, Ctrl *ctrl, cudaStream_t st) {
  return eig_f32(A, n, lda, w, V, ldv, static_cast<char *>(scratch), ctrl, st);
}

// ---------------------------------------------------------------------------
// Clusters after the refinement.  Eigenvalue pairs closer than the cluster
// floor are only re-orthogonalized by the Ogita-Aishima step, so within a
// cluster the vectors keep the FP32 start's mixing and the eigenvalues an
// error up to the cluster's width.  Each cluster (consecutive eigenvalues in
// ascending order, gaps at most the floor, 2..kMaxCluster members) is
// resolved exactly: its block S_C = X_C^T A X_C (taken from S = X^T A X) is
// diagonalized by cyclic FP64 Jacobi, S_C = V_C D V_C^T, and X_C <- X_C V_C.
// ---------------------------------------------------------------------------
constexpr int kMaxCluster = 64;

// w = diag(S); perm = indices by ascending w; start[s] = 1 where sorted
// position s begins a cluster
__global__ void __launch_bounds__(1024) cluster_prep_kernel(const double *__restrict__ S, int n,
                                                            double floor_rel, double *__restrict__ w,
                                                            int *__restrict__ perm,
                                                            int *__restrict__ start) {
  __shared__ double red[32];
  const int tid = threadIdx.x, nt = blockDim.x;
  double lm = 0.0;
  for (int i = tid; i < n; i += nt) {
    const double v = S[(int64_t)i * n + i];
    w[i] = v;
    lm = fmax(lm, fabs(v));
  }
  for (int o = 16; o > 0; o >>= 1) lm = fmax(lm, __shfl_xor_sync(0xffffffffu, lm, o));
  if ((tid & 31) == 0) red[tid >> 5] = lm;
  __syncthreads();
  double lmax = 0.0;
  for (int q = 0; q < (nt >> 5); ++q) lmax = fmax(lmax, red[q]);
  for (int i = tid; i < n; i += nt) {
    const double wi = w[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      const double wj = w[j];
      rank += (wj < wi || (wj == wi && j < i)) ? 1 : 0;
    }
    perm[rank] = i;
  }
  __syncthreads();
  const double fl = floor_rel * lmax;
  for (int q = tid; q < n; q += nt)
    start[q] = (q == 0 || w[perm[q]] - w[perm[q - 1]] > fl) ? 1 : 0;
}

__global__ void __launch_bounds__(256) cluster_eig_kernel(const double *__restrict__ S, int n,
                                                          const int *__restrict__ perm,
                                                          const int *__restrict__ start,
                                                          double *__restrict__ X,
                                                          double *__restrict__ Xtmp,
                                                          double *__restrict__ w) {
  extern __shared__ __align__(16) double csh[];
  const int b = blockIdx.x;
  if (!start[b]) return;
  int m = 1;
  while (b + m < n && !start[b + m]) ++m;
  if (m < 2 || m > kMaxCluster) return;
  double *Sc = csh;            // m x m
  double *Vc = Sc + m * m;     // m x m
  __shared__ double rot_c, rot_s;
  __shared__ int go;
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < m * m; e += nt) {
    const int a = e / m, c = e % m;
    Sc[e] = 0.5 * (S[(int64_t)perm[b + a] * n + perm[b + c]] + S[(int64_t)perm[b + c] * n + perm[b + a]]);
    Vc[e] = (a == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int sweep = 0; sweep < 12; ++sweep) {
    if (tid == 0) {
      double off = 0.0, tot = 0.0;
      for (int e = 0; e < m * m; ++e) {
        tot += Sc[e] * Sc[e];
        if (e / m != e % m) off += Sc[e] * Sc[e];
      }
      go = off > 1e-30 * tot;
    }
    __syncthreads();
    if (!go) break;
    for (int p = 0; p < m - 1; ++p)
      for (int q = p + 1; q < m; ++q) {
        if (tid == 0) {
          const double apq = Sc[p * m + q];
          double c = 1.0, sn = 0.0;
          if (apq != 0.0) {
            const double tau = (Sc[q * m + q] - Sc[p * m + p]) / (2.0 * apq);
            const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
            c = 1.0 / sqrt(1.0 + t * t);
            sn = t * c;
          }
          rot_c = c;
          rot_s = sn;
        }
        __syncthreads();
        const double c = rot_c, sn = rot_s;
        if (sn != 0.0) {
          // columns p, q of S and V
          for (int r = tid; r < m; r += nt) {
            const double sp = Sc[r * m + p], sq = Sc[r * m + q];
            Sc[r * m + p] = c * sp - sn * sq;
            Sc[r * m + q] = sn * sp + c * sq;
            const double vp = Vc[r * m + p], vq = Vc[r * m + q];
            Vc[r * m + p] = c * vp - sn * vq;
            Vc[r * m + q] = sn * vp + c * vq;
          }
          __syncthreads();
          // rows p, q of S
          for (int r = tid; r < m; r += nt) {
            const double sp = Sc[p * m + r], sq = Sc[q * m + r];
            Sc[p * m + r] = c * sp - sn * sq;
            Sc[q * m + r] = sn * sp + c * sq;
          }
        }
        __syncthreads();
      }
  }
  // X_C <- X_C V_C (through Xtmp: every new column reads all old ones)
  for (int e = tid; e < n * m; e += nt) {
    const int r = e / m, c = e % m;
    double acc = 0.0;
    for (int a = 0; a < m; ++a) acc += X[(int64_t)r * n + perm[b + a]] * Vc[a * m + c];
    Xtmp[(int64_t)r * n + perm[b + c]] = acc;
  }
  __syncthreads();
  for (int e = tid; e < n * m; e += nt) {
    const int r = e / m, c = e % m;
    X[(int64_t)r * n + perm[b + c]] = Xtmp[(int64_t)r * n + perm[b + c]];
  }
  for (int c = tid; c < m; c += nt) w[perm[b + c]] = Sc[c * m + c];
}

cudaError_t launch_sym_eig_fast(double *A, int32_t n, int32_t lda, double *w, double *V, int32_t ldv,
                                void *scratch, Ctrl *ctrl, cudaStream_t st) {
  char *base = static_cast<char *>(scratch);
  int *nrounds = reinterpret_cast<int *>(base);
  Rot *rot = reinterpret_cast<Rot *>(base + 256);
  float *A32 = reinterpret_cast<float *>(rot + jacobi_rot_capacity(n));
  float *V32 = A32 + (size_t)n * n;
  float *w32 = V32 + (size_t)n * n;
  double *T1 = reinterpret_cast<double *>(
      (reinterpret_cast<uintptr_t>(w32 + n) + 255) & ~(uintptr_t)255);
  double *T2 = T1 + (size_t)n * n;
  double *T3 = T2 + (size_t)n * n;
  if (ldv != n) return cudaErrorInvalidValue;
  cudaError_t e = launch_d2f(A, n, n, lda, A32, n, st);
  if (e != cudaSuccess) return e;
  e = eig_f32(A32, n, n, w32, V32, n, base, ctrl, st);
  if (e != cudaSuccess) return e;
  // X = V (FP64), A copied compact into T3's neighbour: use T3 for S
  e = launch_f2d(V32, n, n, n, V, ldv, st);
  if (e != cudaSuccess) return e;
  double *Ac = T3;  // S
  int *done = nrounds + 1;  // set once a correction is at rounding level
  double *oacc = reinterpret_cast<double *>(base + 64);  // refinement sums (8 doubles)
  e = cudaMemsetAsync(done, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  for (int it = 0; it < kRefineSteps; ++it) {
    e = launch_small_gemm<double>(true, false, n, n, n, 1.0, V, ldv, V, ldv, 0.0, T1, n, st, done);  // X^T X
    if (e != cudaSuccess) return e;
    e = launch_small_gemm<double>(false, false, n, n, n, 1.0, A, lda, V, ldv, 0.0, T2, n, st, done);  // A X
    if (e != cudaSuccess) return e;
    e = launch_small_gemm<double>(true, false, n, n, n, 1.0, V, ldv, T2, n, 0.0, Ac, n, st, done);  // S
    if (e != cudaSuccess) return e;
    {
      ProfScope ps_(K_EIG, st, 3);
      e = cudaMemsetAsync(oacc, 0, 8 * sizeof(double), st);
      if (e != cudaSuccess) return e;
      const unsigned g = (unsigned)std::min<int64_t>(sm_count() * 2, ((int64_t)n * n + 255) / 256);
      oa_stats_kernel<<<g, 256, 0, st>>>(T1, Ac, A, lda, n, w, oacc, done);
      oa_apply_kernel<<<g, 256, 0, st>>>(T1, Ac, n, w, oacc, done);
      oa_done_kernel<<<1, 1, 0, st>>>(oacc, done);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = launch_small_gemm<double>(false, false, n, n, n, 1.0, V, ldv, T1, n, 0.0, T2, n, st, done);  // X E
    if (e != cudaSuccess) return e;
    {
      ProfScope ps_(K_EIG, st);
      add_inplace_kernel<<<(unsigned)min64(1024, ((int64_t)n * n + 255) / 256), 256, 0, st>>>(
          V, T2, (int64_t)n * n, done);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  // resolve the clusters: S = X^T A X, then one small FP64 Jacobi per cluster
  e = launch_small_gemm<double>(false, false, n, n, n, 1.0, A, lda, V, ldv, 0.0, T2, n, st);  // A X
  if (e != cudaSuccess) return e;
  e = launch_small_gemm<double>(true, false, n, n, n, 1.0, V, ldv, T2, n, 0.0, Ac, n, st);  // S
  if (e != cudaSuccess) return e;
  int *perm = reinterpret_cast<int *>(T1);
  int *start = perm + n;
  {
    ProfScope ps_(K_EIG, st);
    cluster_prep_kernel<<<1, 1024, 0, st>>>(Ac, n, kClusterFloor, w, perm, start);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t csmem = (size_t)2 * kMaxCluster * kMaxCluster * sizeof(double);
    e = cudaFuncSetAttribute(cluster_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)csmem);
    if (e != cudaSuccess) return e;
    cluster_eig_kernel<<<n, 256, csmem, st>>>(Ac, n, perm, start, V, T2, w);
  }
  return cudaGetLastError();
}

}  // namespace sne
