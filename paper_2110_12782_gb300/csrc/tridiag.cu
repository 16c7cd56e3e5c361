// FP32 symmetric eigendecomposition by Householder tridiagonalization,
// bisection and inverse iteration: the starting point of the FP64
// eigensolver of the Rayleigh-Ritz step of Alg. 5 and of svd(W) in Alg. 4
// (the Ogita-Aishima refinement in eig.cu takes it to FP64 accuracy).
//
//  1. tridiag_kernel (one CTA; the lower triangle packed in shared memory):
//     for k = 0 .. n-3 the reflection H_k = I - beta_k v_k v_k^T that zeroes
//     column k below the subdiagonal is formed and applied to the trailing
//     matrix as A <- A - v w^T - w v^T with p = beta A v,
//     w = p - (beta p^T v / 2) v (Householder; Golub and Van Loan, Sec. 8.3).
//     Out: the diagonal d, the off-diagonal e, the v_k and beta_k.
//  2. tri_eig_kernel (one CTA): the tridiagonal T is split where an
//     off-diagonal is negligible against its neighbouring diagonal entries;
//     the eigenvalues of every unreduced block are found by bisection on the
//     Sturm count (the number of negative pivots of the LDL^T factorization
//     of T - x I, Sylvester's law of inertia); eigenvectors by inverse
//     iteration with T - lambda I factored by Gaussian elimination with
//     partial pivoting, from a pseudo-random start, one thread per vector
//     (O(size) sequential steps per factorization or solve, all vectors at
//     once).  Members of a cluster (eigenvalues of one block closer than
//     1e-3 |T_block|, the grouping of LAPACK's stein, with shifts kept at least
//     10 eps |T| apart) are re-orthogonalized by modified Gram-Schmidt by the
//     whole CTA: two solves, the cluster pass, a third solve, the cluster pass
//     again.
//  3. tri_backtransform_kernel: V = H_0 H_1 ... H_{n-3} Z, a warp per column.
#include <cfloat>
#include <cmath>

#include <algorithm>

#include "sne_internal.cuh"

namespace sne {

namespace {

__device__ __forceinline__ int lp(int i, int j) {  // packed lower, i >= j
  return i * (i + 1) / 2 + j;
}

__device__ __forceinline__ float block_sum(float v, float *red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();  // red may still be read from the previous call
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float t = 0.f;
  for (int w = 0; w < nw; ++w) t += red[w];
  return t;
}

__global__ void __launch_bounds__(1024) tridiag_kernel(const float *__restrict__ A, int n, int lda,
                                                       float *__restrict__ d,
                                                       float *__restrict__ e,
                                                       float *__restrict__ Hv,
                                                       float *__restrict__ beta) {
  extern __shared__ __align__(16) float tsm[];
  float *L = tsm;                                // n(n+1)/2
  float *v = L + (size_t)n * (n + 1) / 2;        // n
  float *p = v + n;                              // n
  float *red = p + n;                            // 32
  __shared__ float s_beta, s_alpha;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int i = warp; i < n; i += nw)
    for (int j = lane; j <= i; j += 32) L[lp(i, j)] = A[(int64_t)i * lda + j];
  __syncthreads();
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - 1 - k;  // length of the column below the diagonal
    float part = 0.f;
    for (int j = tid; j < m; j += blockDim.x) {
      const float x = L[lp(k + 1 + j, k)];
      v[j] = x;
      part += x * x;
    }
    const float sigma2 = block_sum(part, red);
    if (tid == 0) {
      const float x0 = v[0];
      const float rest = sigma2 - x0 * x0;
      if (!(rest > FLT_MIN)) {
        s_beta = 0.f;   // the column is already zero below the subdiagonal
        s_alpha = x0;
      } else {
        const float alpha = -copysignf(sqrtf(sigma2), x0);
        v[0] = x0 - alpha;
        s_beta = 1.0f / (sigma2 - x0 * alpha);
        s_alpha = alpha;
      }
      d[k] = L[lp(k, k)];
      e[k] = s_alpha;
      beta[k] = s_beta;
    }
    __syncthreads();
    const float b = s_beta;
    for (int j = tid; j < n - 1; j += blockDim.x) Hv[(int64_t)k * (n - 1) + j] = (j < m && b != 0.f) ? v[j] : 0.f;
    if (b == 0.f) continue;  // uniform
    // p = b A_sub v (A_sub: rows and columns k+1 .. n-1)
    for (int i = warp; i < m; i += nw) {
      const int gi = k + 1 + i;
      float acc = 0.f;
      for (int j = lane; j < m; j += 32) {
        const int gj = k + 1 + j;
        acc += (gj <= gi ? L[lp(gi, gj)] : L[lp(gj, gi)]) * v[j];
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) p[i] = b * acc;
    }
    __syncthreads();
    part = 0.f;
    for (int j = tid; j < m; j += blockDim.x) part += p[j] * v[j];
    const float K = 0.5f * b * block_sum(part, red);
    for (int j = tid; j < m; j += blockDim.x) p[j] -= K * v[j];  // w
    __syncthreads();
    // A_sub -= v w^T + w v^T (lower triangle)
    for (int i = warp; i < m; i += nw) {
      const int gi = k + 1 + i;
      const float vi = v[i], wi = p[i];
      float *row = L + lp(gi, k + 1);
      for (int j = lane; j <= i; j += 32) row[j] -= vi * p[j] + wi * v[j];
    }
    __syncthreads();
  }
  if (tid == 0) {
    if (n >= 2) {
      d[n - 2] = L[lp(n - 2, n - 2)];
      e[n - 2] = L[lp(n - 1, n - 2)];
    }
    d[n - 1] = L[lp(n - 1, n - 1)];
    if (n >= 2) beta[n - 2] = 0.f;
    if (n >= 1) beta[n - 1] = 0.f;
  }
  for (int k = (n >= 2 ? n - 2 : 0); k < n - 1; ++k)
    for (int j = tid; j < n - 1; j += blockDim.x) Hv[(int64_t)k * (n - 1) + j] = 0.f;
}

// Number of eigenvalues below x of the tridiagonal block (d[s..t], e[s..t-1]).
__device__ __forceinline__ int sturm_count(const float *d, const float *e2, int s, int t, float x,
                                           float pivmin) {
  int c = 0;
  float q = d[s] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  if (q < 0.f) ++c;
  for (int i = s + 1; i <= t; ++i) {
    // the division needs no IEEE rounding: the count only takes signs, and
    // bisection tolerates an error of a few ulp in q
    q = d[i] - x - __fdividef(e2[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    if (q < 0.f) ++c;
  }
  return c;
}

constexpr int kTriMaxN = 1024;
// threads of tri_eig_kernel: one per eigenvector up to 512 (more per thread
// beyond), leaving each thread registers for the blocked solves
constexpr int kTriEigThreads = 512;

__device__ __forceinline__ float hash_unit(uint32_t a, uint32_t b) {
  uint64_t z = ((uint64_t)a << 32) ^ (uint64_t)b ^ 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  z ^= z >> 31;
  return (float)(z >> 40) * (2.0f / 16777216.0f) - 1.0f;  // [-1, 1)
}

// Inverse iteration: one thread per eigenvector.  The factors of
// T_b - shift_m I and the iterate of vector m live in global scratch at
// [i * n + m], so that the 32 threads of a warp, which run their sequential
// loops in lockstep over the same row i, touch 32 consecutive words.
struct TriLU {
  float *r0, *u1, *u2, *lm, *pv;  // 1/U(i,i), U(i,i+1), U(i,i+2), multiplier, swap flag
};

// LU of T_b - shift I with partial pivoting for the column m (rows s .. t).
__device__ void tri_lu(const float *d, const float *e, int s, int sz, float shift, float pertol,
                       const TriLU &f, int n, int m) {
  float a = d[s] - shift, bnext = e[s];
  for (int i = 0; i < sz - 1; ++i) {
    const float sub = e[s + i];             // T(i+1, i)
    const float dn = d[s + i + 1] - shift;  // T(i+1, i+1)
    const float sup2 = (i + 2 < sz) ? e[s + i + 1] : 0.f;
    float u0, u1, u2, l, pv;
    if (fabsf(a) >= fabsf(sub)) {
      l = (a != 0.f) ? sub / a : 0.f;
      u0 = a; u1 = bnext; u2 = 0.f; pv = 0.f;
      a = dn - l * bnext;
      bnext = sup2;
    } else {
      l = a / sub;
      u0 = sub; u1 = dn; u2 = sup2; pv = 1.f;
      a = bnext - l * dn;
      bnext = -l * sup2;
    }
    if (fabsf(u0) < pertol) u0 = copysignf(pertol, u0 == 0.f ? 1.f : u0);
    const int64_t q = (int64_t)i * n + m;
    f.r0[q] = 1.0f / u0; f.u1[q] = u1; f.u2[q] = u2; f.lm[q] = l; f.pv[q] = pv;
  }
  const float u0 = (fabsf(a) < pertol) ? copysignf(pertol, a == 0.f ? 1.f : a) : a;
  const int64_t q = (int64_t)(sz - 1) * n + m;
  f.r0[q] = 1.0f / u0; f.u1[q] = 0.f; f.u2[q] = 0.f; f.lm[q] = 0.f; f.pv[q] = 0.f;
}

// x <- (T_b - shift I)^-1 x (x = column m of X, rows s ..), then scaled to
// max |x_i| = 1.
__device__ void tri_solve(const TriLU &f, float *X, int s, int sz, int n, int m) {
  // Rows are taken in blocks of kSB: the loads of a block (independent of the
  // recurrence) are issued together, so that one L2 latency covers kSB steps.
  constexpr int kSB = 4;
  float *x = X + (int64_t)s * n + m;
  const float *__restrict__ lm = f.lm + m;
  const float *__restrict__ pv = f.pv + m;
  const float *__restrict__ u1 = f.u1 + m;
  const float *__restrict__ u2 = f.u2 + m;
  const float *__restrict__ r0 = f.r0 + m;
  // forward: the row swaps and multipliers (step i reads x[i + 1] before step
  // i + 1 overwrites it)
  float cur = x[0];
  for (int i0 = 0; i0 < sz - 1; i0 += kSB) {
    float xn[kSB], lv[kSB], pw[kSB], o[kSB];
#pragma unroll
    for (int u = 0; u < kSB; ++u) {
      const int i = i0 + u;
      if (i < sz - 1) {
        xn[u] = x[(int64_t)(i + 1) * n];
        lv[u] = lm[(int64_t)i * n];
        pw[u] = pv[(int64_t)i * n];
      }
    }
#pragma unroll
    for (int u = 0; u < kSB; ++u) {
      if (i0 + u < sz - 1) {
        if (pw[u] != 0.f) {
          o[u] = xn[u];
          cur = cur - lv[u] * xn[u];
        } else {
          o[u] = cur;
          cur = xn[u] - lv[u] * cur;
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kSB; ++u)
      if (i0 + u < sz - 1) x[(int64_t)(i0 + u) * n] = o[u];
  }
  x[(int64_t)(sz - 1) * n] = cur;
  // back substitution with U, rows sz - 1 .. 0
  float x1 = 0.f, x2 = 0.f, mx = 0.f;
  for (int i0 = sz - 1; i0 >= 0; i0 -= kSB) {
    float xv[kSB], a1[kSB], a2[kSB], rr[kSB];
#pragma unroll
    for (int u = 0; u < kSB; ++u) {
      const int i = i0 - u;
      if (i >= 0) {
        const int64_t q = (int64_t)i * n;
        xv[u] = x[q];
        a1[u] = u1[q];
        a2[u] = u2[q];
        rr[u] = r0[q];
      }
    }
#pragma unroll
    for (int u = 0; u < kSB; ++u) {
      if (i0 - u >= 0) {
        const float r = (xv[u] - a1[u] * x1 - a2[u] * x2) * rr[u];
        xv[u] = r;
        x2 = x1;
        x1 = r;
        mx = fmaxf(mx, fabsf(r));
      }
    }
#pragma unroll
    for (int u = 0; u < kSB; ++u)
      if (i0 - u >= 0) x[(int64_t)(i0 - u) * n] = xv[u];
  }
  const float inv = mx > 0.f ? 1.f / mx : 1.f;
  for (int i0 = 0; i0 < sz; i0 += kSB) {
    float xv[kSB];
#pragma unroll
    for (int u = 0; u < kSB; ++u)
      if (i0 + u < sz) xv[u] = x[(int64_t)(i0 + u) * n];
#pragma unroll
    for (int u = 0; u < kSB; ++u)
      if (i0 + u < sz) x[(int64_t)(i0 + u) * n] = xv[u] * inv;
  }
}

// Modified Gram-Schmidt inside every cluster of two or more members, by the
// whole CTA: member j is normalized, then its component is removed from the
// later members (a warp per member).  Clusters in order, members in order.
// A cluster whose members fit in the shared buffer `cb` (cap floats) is
// copied there first (member-major, coalesced loads and stores of Z's rows):
// the member vectors are columns of Z, strided in global memory.
__device__ void tri_cluster_mgs(float *X, int n, const int *cstart, int nc, const int *blk_of,
                                const int *bstart, float *red, Ctrl *ctrl, float *cb, int cap) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  for (int c = 0; c < nc; ++c) {
    const int m0 = cstart[c], m1 = cstart[c + 1];
    if (m1 - m0 < 2) continue;
    const int b = blk_of[m0];
    const int s = bstart[b], sz = bstart[b + 1] - s;
    const int mc = m1 - m0;
    const bool shared = (int64_t)mc * sz <= cap;
    if (shared) {
      for (int e = tid; e < mc * sz; e += blockDim.x) {
        const int i = e / mc, q = e % mc;
        cb[q * sz + i] = X[(int64_t)(s + i) * n + m0 + q];
      }
      __syncthreads();
    }
    for (int j = m0; j < m1; ++j) {
      float *xj = shared ? cb + (j - m0) * sz : nullptr;
      float part = 0.f;
      for (int i = tid; i < sz; i += blockDim.x) {
        const float v = shared ? xj[i] : X[(int64_t)(s + i) * n + j];
        part += v * v;
      }
      const float nrm = block_sum(part, red);
      if (!(nrm > 0.f)) {
        if (tid == 0) record_error(ctrl, SNE_ERR_NUMERIC, W_EIG);
      }
      const float rn = nrm > 0.f ? 1.0f / sqrtf(nrm) : 0.f;
      for (int i = tid; i < sz; i += blockDim.x) {
        if (shared)
          xj[i] *= rn;
        else
          X[(int64_t)(s + i) * n + j] *= rn;
      }
      __syncthreads();
      for (int q = j + 1 + warp; q < m1; q += nw) {
        float dot = 0.f;
        if (shared) {
          const float *xq = cb + (q - m0) * sz;
          for (int i = lane; i < sz; i += 32) dot += xj[i] * xq[i];
        } else {
          for (int i = lane; i < sz; i += 32)
            dot += X[(int64_t)(s + i) * n + j] * X[(int64_t)(s + i) * n + q];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
        if (shared) {
          float *xq = cb + (q - m0) * sz;
          for (int i = lane; i < sz; i += 32) xq[i] -= dot * xj[i];
        } else {
          for (int i = lane; i < sz; i += 32)
            X[(int64_t)(s + i) * n + q] -= dot * X[(int64_t)(s + i) * n + j];
        }
      }
      __syncthreads();
    }
    if (shared) {
      for (int e = tid; e < mc * sz; e += blockDim.x) {
        const int i = e / mc, q = e % mc;
        X[(int64_t)(s + i) * n + m0 + q] = cb[q * sz + i];
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(kTriEigThreads) tri_eig_kernel(const float *__restrict__ dg,
                                                       const float *__restrict__ eg, int n,
                                                       float *__restrict__ w,
                                                       float *__restrict__ Z,
                                                       float *__restrict__ scratch,
                                                       Ctrl *ctrl, int cbuf_cap) {
  extern __shared__ __align__(16) float cbuf[];  // cbuf_cap floats: a cluster's vectors
  __shared__ float d[kTriMaxN], e[kTriMaxN], e2[kTriMaxN], lam[kTriMaxN], shift[kTriMaxN];
  __shared__ int bstart[kTriMaxN + 1], blk_of[kTriMaxN], cstart[kTriMaxN + 1];
  __shared__ float bnorm[kTriMaxN];
  __shared__ int csz[kTriMaxN];  // size of the cluster of eigenvalue m
  __shared__ float red[32];
  __shared__ int nblk_s, nclu_s;
  __shared__ float tnorm_s;
  const int tid = threadIdx.x;
  for (int i = tid; i < n; i += blockDim.x) {
    d[i] = dg[i];
    e[i] = i + 1 < n ? eg[i] : 0.f;
  }
  __syncthreads();
  if (tid == 0) {
    float tn = 0.f;
    for (int i = 0; i < n; ++i)
      tn = fmaxf(tn, fabsf(d[i]) + (i > 0 ? fabsf(e[i - 1]) : 0.f) + fabsf(e[i]));
    tnorm_s = tn;
    // split where e_i is negligible
    int nb = 0;
    bstart[nb++] = 0;
    for (int i = 0; i + 1 < n; ++i) {
      if (fabsf(e[i]) <= 2.0f * FLT_EPSILON * (fabsf(d[i]) + fabsf(d[i + 1])) ||
          fabsf(e[i]) <= FLT_MIN) {
        e[i] = 0.f;
        bstart[nb++] = i + 1;
      }
    }
    bstart[nb] = n;
    nblk_s = nb;
  }
  __syncthreads();
  for (int i = tid; i < n; i += blockDim.x) e2[i] = e[i] * e[i];
  const int nb = nblk_s;
  for (int b = tid; b < nb; b += blockDim.x) {
    float bn = 0.f;
    for (int i = bstart[b]; i < bstart[b + 1]; ++i) {
      blk_of[i] = b;
      bn = fmaxf(bn, fabsf(d[i]) + 2.f * fabsf(e[i]));
    }
    bnorm[b] = bn;
  }
  __syncthreads();
  const float tnorm = tnorm_s;
  const float pivmin = fmaxf(FLT_MIN, tnorm * 1e-30f);
  // eigenvalues: global index m -> block blk_of[m] (blocks are contiguous in
  // index), local index m - bstart
  for (int m = tid; m < n; m += blockDim.x) {
    const int b = blk_of[m];
    const int s = bstart[b], t = bstart[b + 1] - 1;
    const int loc = m - s;
    float lo = FLT_MAX, hi = -FLT_MAX;
    for (int i = s; i <= t; ++i) {
      const float r = (i > s ? fabsf(e[i - 1]) : 0.f) + (i < t ? fabsf(e[i]) : 0.f);
      lo = fminf(lo, d[i] - r);
      hi = fmaxf(hi, d[i] + r);
    }
    const float pad = 2.0f * FLT_EPSILON * fmaxf(fabsf(lo), fabsf(hi)) + pivmin;
    lo -= pad;
    hi += pad;
    for (int it = 0; it < 64; ++it) {
      const float mid = 0.5f * (lo + hi);
      if (mid == lo || mid == hi) break;
      if (sturm_count(d, e2, s, t, mid, pivmin) <= loc) lo = mid;
      else hi = mid;
    }
    lam[m] = 0.5f * (lo + hi);
    w[m] = lam[m];
  }
  __syncthreads();
  // clusters: consecutive eigenvalues of one block closer than 1e-3 |T_block|;
  // the shifts inside a cluster kept at least 10 eps |T| apart
  const float pertol = 10.0f * FLT_EPSILON * tnorm;
  if (tid == 0) {
    int nc = 0;
    for (int m = 0; m < n; ++m) {
      const int b = blk_of[m];
      bool newc = (m == 0) || (blk_of[m - 1] != b);
      if (!newc) newc = (lam[m] - lam[m - 1]) > 1e-3f * bnorm[b];
      if (newc) cstart[nc++] = m;
      shift[m] = (!newc && lam[m] - shift[m - 1] < pertol) ? shift[m - 1] + pertol : lam[m];
    }
    cstart[nc] = n;
    nclu_s = nc;
  }
  __syncthreads();
  const int nc = nclu_s;
  for (int c = tid; c < nc; c += blockDim.x)
    for (int m = cstart[c]; m < cstart[c + 1]; ++m) csz[m] = cstart[c + 1] - cstart[c];
  __syncthreads();
  const int64_t n2 = (int64_t)n * n;
  TriLU f{scratch, scratch + n2, scratch + 2 * n2, scratch + 3 * n2, scratch + 4 * n2};
  // two inverse-iteration solves per vector from a pseudo-random start
  for (int m = tid; m < n; m += blockDim.x) {
    const int b = blk_of[m];
    const int s = bstart[b], sz = bstart[b + 1] - s;
    for (int i = 0; i < n; ++i) Z[(int64_t)i * n + m] = 0.f;
    if (sz == 1) {
      Z[(int64_t)s * n + m] = 1.f;
      continue;
    }
    tri_lu(d, e, s, sz, shift[m], pertol, f, n, m);
    for (int i = 0; i < sz; ++i) Z[(int64_t)(s + i) * n + m] = hash_unit((uint32_t)m, (uint32_t)i);
    tri_solve(f, Z, s, sz, n, m);
    tri_solve(f, Z, s, sz, n, m);
  }
  __syncthreads();
  tri_cluster_mgs(Z, n, cstart, nc, blk_of, bstart, red, ctrl, cbuf, cbuf_cap);
  // a third solve, then orthonormal again (clusters) or normalized (the rest)
  for (int m = tid; m < n; m += blockDim.x) {
    const int b = blk_of[m];
    const int s = bstart[b], sz = bstart[b + 1] - s;
    if (sz > 1) tri_solve(f, Z, s, sz, n, m);
  }
  __syncthreads();
  tri_cluster_mgs(Z, n, cstart, nc, blk_of, bstart, red, ctrl, cbuf, cbuf_cap);
  for (int m = tid; m < n; m += blockDim.x) {
    const int b = blk_of[m];
    const int s = bstart[b], sz = bstart[b + 1] - s;
    // members of clusters are orthonormal after the cluster pass
    if (csz[m] > 1 || sz == 1) continue;
    float nrm = 0.f;
    for (int i = 0; i < sz; ++i) {
      const float v = Z[(int64_t)(s + i) * n + m];
      nrm += v * v;
    }
    if (!(nrm > 0.f)) record_error(ctrl, SNE_ERR_NUMERIC, W_EIG);
    const float rn = nrm > 0.f ? 1.0f / sqrtf(nrm) : 0.f;
    for (int i = 0; i < sz; ++i) Z[(int64_t)(s + i) * n + m] *= rn;
  }
}

// V[:, m] = H_0 H_1 ... H_{n-3} Z[:, m]: a warp per column, the column in
// registers (lane i holds rows i, i + 32, ...).
constexpr int kBtPer = 32;  // n <= 1024
__global__ void __launch_bounds__(256) tri_backtransform_kernel(const float *__restrict__ Z, int ldz,
                                                                const float *__restrict__ Hv,
                                                                const float *__restrict__ beta,
                                                                int n, float *__restrict__ V,
                                                                int ldv) {
  const int lane = threadIdx.x & 31;
  const int col = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (col >= n) return;
  float z[kBtPer];
#pragma unroll
  for (int r = 0; r < kBtPer; ++r) {
    const int i = lane + 32 * r;
    z[r] = i < n ? Z[(int64_t)i * ldz + col] : 0.f;
  }
  for (int k = n - 3; k >= 0; --k) {
    const float b = beta[k];
    if (b == 0.f) continue;
    const float *vk = Hv + (int64_t)k * (n - 1);  // v_k[j] acts on row k + 1 + j
    float dot = 0.f;
#pragma unroll
    for (int r = 0; r < kBtPer; ++r) {
      const int i = lane + 32 * r;
      if (i > k && i < n) dot += vk[i - k - 1] * z[r];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dot += __shfl_xor_sync(0xffffffffu, dot, o);
    dot *= b;
#pragma unroll
    for (int r = 0; r < kBtPer; ++r) {
      const int i = lane + 32 * r;
      if (i > k && i < n) z[r] -= dot * vk[i - k - 1];
    }
  }
#pragma unroll
  for (int r = 0; r < kBtPer; ++r) {
    const int i = lane + 32 * r;
    if (i < n) V[(int64_t)i * ldv + col] = z[r];
  }
}

}  // namespace

size_t tri_eig_scratch_floats(int n) {
  // Hv (n-1 x n-1 rounded to n x n), Z (n x n), d, e, beta, the LU factors of
  // every inverse iteration (5 n x n)
  return 7 * (size_t)n * n + 3 * (size_t)n + 64;
}

size_t tri_eig_smem(int n) { return ((size_t)n * (n + 1) / 2 + 2 * (size_t)n + 32) * sizeof(float); }

cudaError_t launch_sym_eig_tridiag(const float *A, int32_t n, int32_t lda, float *w, float *V,
                                   int32_t ldv, float *scratch, Ctrl *ctrl, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (n > kTriMaxN || tri_eig_smem(n) > 227 * 1024) return cudaErrorInvalidValue;
  float *Hv = scratch;
  float *Z = Hv + (size_t)n * n;
  float *d = Z + (size_t)n * n;
  float *e = d + n;
  float *beta = e + n;
  float *wsc = beta + n;
  const size_t smem = tri_eig_smem(n);
  cudaError_t err = cudaFuncSetAttribute(tridiag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
  if (err != cudaSuccess) return err;
  {
    ProfScope ps_(K_EIG, st);
    tridiag_kernel<<<1, 1024, smem, st>>>(A, n, lda, d, e, Hv, beta);
  }
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  {
    ProfScope ps_(K_EIG, st);
    // the cluster buffer: as much shared memory as the kernel may take next
    // to its static arrays (48 KB of them at kTriMaxN = 1024), at most n^2 floats
    const int cap = (int)std::min<size_t>((size_t)n * n, (size_t)(160 * 1024) / sizeof(float));
    err = cudaFuncSetAttribute(tri_eig_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                               (int)(cap * sizeof(float)));
    if (err != cudaSuccess) return err;
    tri_eig_kernel<<<1, kTriEigThreads, cap * sizeof(float), st>>>(d, e, n, w, Z, wsc, ctrl, cap);
  }
  err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  ProfScope ps_(K_EIG, st);
  tri_backtransform_kernel<<<(n + 7) / 8, 256, 0, st>>>(Z, n, Hv, beta, n, V, ldv);
  return cudaGetLastError();
}

}  // namespace sne
