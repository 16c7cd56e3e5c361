// C entry points of libsketchne.so: argument checks, the workspace layout, and
// the stream-ordered sequence of kernels for Alg. 5 (freigs), Eq. 11 and
// Alg. 4 (sparse-sign randomized single-pass SVD), i.e. Alg. 6 lines 1-5.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstring>
#include <mutex>

#include "sne_internal.cuh"

using namespace sne;

namespace {

// --------------------------------------------------------------------------
// Sizes and workspace layout
// --------------------------------------------------------------------------
struct Dims {
  int64_t n, nnz;
  int k, K, h, l, z, d, nS, nO, Sm, Wab;
  bool half;   // mixed-precision reconstruction (BF16 / FP16 operands)
  bool split;  // operands as hi/lo pairs (SNE_BF16X2 / SNE_FP16X2)
  bool fp16;   // FP16 (else BF16) operands
  int kpad;    // k rounded up to a multiple of 64 for the tensor-core operands
};

int make_dims(int64_t n, int64_t nnz, const sne_params *p, int mode, Dims *D) {
  if (!p || n <= 0 || nnz < 0) return SNE_ERR_ARG;
  if (mode == SNE_WS_EMBED_HOST) mode = SNE_WS_EMBED;
  if (p->k <= 0 || p->d <= 0 || p->h <= 0 || p->l <= 0 || p->zeta <= 0 || p->T <= 0 ||
      p->q < 0 || p->s_eig < 0 || !(p->b > 0) || !(p->alpha > 0) || p->alpha > 1.0)
    return SNE_ERR_ARG;
  if (p->precision != SNE_FP32 && p->precision != SNE_BF16 && p->precision != SNE_FP16 &&
      p->precision != SNE_BF16X2 && p->precision != SNE_FP16X2)
    return SNE_ERR_ARG;
  if (p->f != SNE_F_TRUNC_LOG && p->f != SNE_F_IDENTITY) return SNE_ERR_ARG;
  if (p->orth != SNE_ORTH_EIGSVD && p->orth != SNE_ORTH_CHOLQR) return SNE_ERR_ARG;
  Dims d{};
  d.n = n;
  d.nnz = nnz;
  d.k = p->k;
  d.K = p->k + p->s_eig;
  d.h = p->h;
  d.l = p->l;
  d.d = p->d;
  d.z = (int)min64(n, p->zeta);
  d.nS = d.h * d.z;
  d.nO = d.l * d.z;
  if (d.z > 64) return SNE_ERR_SIZE;
  if (mode != SNE_WS_SKETCH && (d.K > n || d.K > 1024)) return SNE_ERR_SIZE;
  if (mode != SNE_WS_FREIGS) {
    if (d.d > d.h || d.h > d.l || d.h > n || d.h > 1024 || d.k > 1024) return SNE_ERR_SIZE;
    if (d.nS > kUniqueMax || d.nO > kUniqueMax) return SNE_ERR_SIZE;
  }
  d.Sm = std::max(std::max(d.K, d.h), d.k);
  d.half = p->precision != SNE_FP32;
  d.split = p->precision == SNE_BF16X2 || p->precision == SNE_FP16X2;
  d.fp16 = p->precision == SNE_FP16 || p->precision == SNE_FP16X2;
  d.kpad = (d.k + 63) / 64 * 64;
  if (d.half && mode != SNE_WS_FREIGS) {
    if (!(d.z == 1 || d.z == 2 || d.z == 4 || d.z == 8 || d.z == 16 || d.z == 32)) return SNE_ERR_SIZE;
    // the A tile stays in shared memory: k <= 384 (k <= 320 for hi/lo pairs)
    if (d.kpad > (d.split ? 320 : 384)) return SNE_ERR_SIZE;
  }
  // the tall buffers also hold the centred rows L~ (n x k) during the sketch
  d.Wab = (mode == SNE_WS_SKETCH) ? std::max(d.h, d.k)
                                  : (mode == SNE_WS_FREIGS ? d.K : std::max(d.K, d.h));
  *D = d;
  return SNE_OK;
}

struct Bump {
  char *base;
  size_t off = 0;
  template <class T>
  T *take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    T *ptr = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += count * sizeof(T);
    return ptr;
  }
  // rows of row_bytes starting at a multiple of row_bytes from the base (the
  // tensor-core sketch reads its operands as rows of one arena)
  template <class T>
  T *take_rows(size_t rows, size_t row_bytes) {
    off = (off + row_bytes - 1) / row_bytes * row_bytes;
    T *ptr = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += rows * row_bytes;
    return ptr;
  }
};

struct Bufs {
  Ctrl *ctrl;
  float *deg, *dpow, *wnz, *rsc, *rsc_lo, *wgt, *wgt_lo;
  float *A, *B, *C;  // tall buffers
  float *partial;
  double *m64[5];
  void *eigscr;
  float *m32[4];
  float *mT;  // transposed small factor for the tensor-core tall product
  double *w64, *lam;
  float *w32;
  int32_t *perm;
  int32_t *idxS, *idxO, *uniqS, *uniqO, *posS, *posO;
  int8_t *signS, *signO;
  float *RpS, *RpO, *Yo, *Zf, *Gf;
  double *G64, *Gp, *Tm, *Z64;
  void *Ah, *AhO, *BhS, *BhO;  // half operands of the tensor-core sketch (hi parts)
  void *Al, *AlO, *BlS, *BlO;  // their lo parts (split precisions)
  float *rowfA, *rowfO;
  double *cpart, *cstats;      // centring: partial sums, statistics (w, p, q, gamma, s)
  float *ws_hi, *ws_lo;        // s w as an FP32 pair
  float2 *rowdat, *rowdatO;    // (rho, mask) per row of L~ and of L~(p_O, :)
  float4 *coldatS, *coldatO;   // (scale, kappa, sign, 0) per evaluated column
  char *arena;        // the workspace: base of the tensor-core operand rows
  size_t arena_bytes;
  int64_t *h_rowptr;  // device staging of a host graph (SNE_WS_EMBED_HOST)
  int32_t *h_col;
  float *h_val, *h_E;
  double *h_sigma;
};

inline int64_t pad256(int64_t x) { return (x + 255) / 256 * 256; }

size_t carve(const Dims &D, int mode, void *base, Bufs *b) {
  Bump bp{static_cast<char *>(base)};
  Bufs x{};
  const bool host_mode = (mode == SNE_WS_EMBED_HOST);
  if (host_mode) mode = SNE_WS_EMBED;
  x.ctrl = bp.take<Ctrl>(1);
  const int64_t n = D.n;
  x.deg = bp.take<float>(n);
  x.dpow = bp.take<float>(n);
  x.wnz = mode != SNE_WS_SKETCH ? bp.take<float>((size_t)D.nnz) : nullptr;
  x.rsc = bp.take<float>(n);
  x.rsc_lo = bp.take<float>(n);
  x.wgt = bp.take<float>(n);
  x.wgt_lo = bp.take<float>(n);
  x.A = bp.take<float>((size_t)n * D.Wab);
  x.B = bp.take<float>((size_t)n * D.Wab);
  if (mode != SNE_WS_SKETCH) x.C = bp.take<float>((size_t)n * D.K);
  size_t pf = 0;
  if (mode != SNE_WS_SKETCH) pf = std::max(pf, gram_partial_floats(n, D.K, D.K));
  if (mode != SNE_WS_FREIGS) {
    pf = std::max(pf, gram_partial_floats(n, D.h, D.h));
    pf = std::max(pf, gram_partial_floats(n, D.k, D.k));
  }
  x.partial = bp.take<float>(pf);
  // n x n plus room for the Cholesky scratch tail (1/R[i][i], permutation, rank)
  const size_t S2 = (size_t)D.Sm * D.Sm + 2 * (size_t)D.Sm + 8;
  for (auto &m : x.m64) m = bp.take<double>(S2);
  x.eigscr = bp.take<char>(std::max(eig_scratch_bytes(D.Sm), (S2 + 4 * (size_t)D.Sm) * 8 + 1024));
  for (auto &m : x.m32) m = bp.take<float>(S2);
  x.mT = bp.take<float>(tall_tc_scratch_floats(D.Sm, D.Sm));
  x.w64 = bp.take<double>(D.Sm);
  x.lam = bp.take<double>(D.Sm);
  x.w32 = bp.take<float>(D.Sm);
  x.perm = bp.take<int32_t>(D.Sm);
  if (mode != SNE_WS_FREIGS) {
    x.idxS = bp.take<int32_t>(D.nS);
    x.uniqS = bp.take<int32_t>(D.nS);
    x.posS = bp.take<int32_t>(D.nS);
    x.signS = bp.take<int8_t>(D.nS);
    x.idxO = bp.take<int32_t>(D.nO);
    x.uniqO = bp.take<int32_t>(D.nO);
    x.posO = bp.take<int32_t>(D.nO);
    x.signO = bp.take<int8_t>(D.nO);
    x.RpS = bp.take<float>((size_t)D.nS * D.k);
    x.RpO = bp.take<float>((size_t)D.nO * D.k);
    const int64_t vmax = min64(n, D.nO);
    x.Yo = bp.take<float>((size_t)vmax * D.l);
    x.Zf = bp.take<float>((size_t)D.l * D.l);
    x.Gf = bp.take<float>((size_t)D.l * D.h);
    x.G64 = bp.take<double>((size_t)D.l * D.h);
    x.Gp = bp.take<double>((size_t)D.h * D.l);
    x.Tm = bp.take<double>((size_t)D.h * D.l);
    x.Z64 = bp.take<double>((size_t)D.l * D.l);
    x.cpart = bp.take<double>(center_partial_doubles(n, D.k));
    x.cstats = bp.take<double>(3 * (size_t)D.k + 2);
    x.ws_hi = bp.take<float>(D.k);
    x.ws_lo = bp.take<float>(D.k);
    x.rowdat = bp.take<float2>(n);
    x.rowdatO = bp.take<float2>(vmax);
    x.coldatS = bp.take<float4>(D.nS + 256);
    x.coldatO = bp.take<float4>(D.nO + 256);
    if (D.half) {
      // operand rows of the arena; B zero padded to whole 256-column tiles
      const size_t rb = (size_t)D.kpad * 2;
      x.Ah = bp.take_rows<uint16_t>(n, rb);
      x.AhO = bp.take_rows<uint16_t>(vmax, rb);
      x.BhS = bp.take_rows<uint16_t>(pad256(D.nS), rb);
      x.BhO = bp.take_rows<uint16_t>(pad256(D.nO), rb);
      if (D.split) {
        x.Al = bp.take_rows<uint16_t>(n, rb);
        x.AlO = bp.take_rows<uint16_t>(vmax, rb);
        x.BlS = bp.take_rows<uint16_t>(pad256(D.nS), rb);
        x.BlO = bp.take_rows<uint16_t>(pad256(D.nO), rb);
      }
      x.rowfA = bp.take<float>(n);
      x.rowfO = bp.take<float>(vmax);
    }
  }
  if (host_mode) {
    x.h_rowptr = bp.take<int64_t>(D.n + 1);
    x.h_col = bp.take<int32_t>(D.nnz);
    x.h_val = bp.take<float>(D.nnz);
    x.h_E = bp.take<float>((size_t)D.n * D.d);
    x.h_sigma = bp.take<double>(D.d);
  }
  const size_t total = (bp.off + 255) & ~(size_t)255;
  x.arena = static_cast<char *>(base);
  x.arena_bytes = total;
  if (b) *b = x;
  return total;
}

#define CK(call)                               \
  do {                                         \
    cudaError_t e__ = (call);                  \
    if (e__ != cudaSuccess) return SNE_ERR_CUDA; \
  } while (0)

constexpr int kMaxPropagationSteps = 1000;
constexpr int kMaxPropagationWidth = 1024;

int check_graph(const sne_csr *g) {
  if (!g || g->n <= 0 || g->nnz < 0 || !g->row_ptr || (g->nnz > 0 && !g->col_idx))
    return SNE_ERR_ARG;
  if (g->n > (int64_t)INT32_MAX - 1) return SNE_ERR_SIZE;
  return SNE_OK;
}

// The embedding needs at least one edge: with none, vol(G) = 0 and the matrix
// of Eq. 1 (and every power of X in Alg. 5) is undefined.
int check_has_edges(const sne_csr *g) { return g->nnz > 0 ? SNE_OK : SNE_ERR_GRAPH; }

int check_ws(void *ws, size_t bytes, size_t need) {
  if (!ws || ((uintptr_t)ws % 256) != 0 || bytes < need) return SNE_ERR_WORKSPACE;
  return SNE_OK;
}

// --------------------------------------------------------------------------
// Small kernels local to the orchestration
// --------------------------------------------------------------------------
// out_i = mult * vol * deg_i^beta  (0 for isolated vertices)
// out_i + out_lo_i = mult * vol * deg_i^beta evaluated in FP64 and split into
// two FP32 parts: one rounding shared by all rows (of the scalar, or of the
// power of a common degree) would shift every entry of L'R' alike
__global__ void rowscale_kernel(const float *deg, int64_t n, double beta, const double *vol,
                                double mult, float *out, float *out_lo) {
  const double s = mult * (vol ? *vol : 1.0);
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float d = deg[i];
    const double x = d > 0.f ? s * pow((double)d, beta) : 0.0;
    const float hi = (float)x;
    out[i] = hi;
    if (out_lo) out_lo[i] = (float)(x - (double)hi);
  }
}

// eigSVD step: M[:, j] = V[:, j] / sqrt(w_j)
__global__ void inv_sqrt_cols_kernel(const float *V, int n, int ldv, const float *w, float *M, int ldm,
                                     Ctrl *ctrl) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n * n; q += gridDim.x * blockDim.x) {
    const int r = q / n, c = q % n;
    const float wc = w[c];
    if (!(wc > 0.f)) {
      if (r == 0) record_error(ctrl, SNE_ERR_NUMERIC, W_EIGSVD);
      M[(int64_t)r * ldm + c] = 0.f;
    } else {
      M[(int64_t)r * ldm + c] = V[(int64_t)r * ldv + c] * rsqrtf(wc);
    }
  }
}

// out[a][j] = V[a][perm[j]] * colscale_j  (FP32), j < ncols; optional value outputs
__global__ void select_cols_kernel(const double *V, int rows, int ldv, const int32_t *perm,
                                   const double *w, int ncols, int scale_mode, float *out, int ldo,
                                   double *vals_out, int vals_abs) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < rows * ncols; q += gridDim.x * blockDim.x) {
    const int a = q / ncols, j = q % ncols;
    const int src = perm[j];
    double s = 1.0;
    if (scale_mode == 1) s = sqrt(fabs(w[src]));
    out[(int64_t)a * ldo + j] = (float)(V[(int64_t)a * ldv + src] * s);
    if (a == 0 && vals_out) vals_out[j] = vals_abs ? fabs(w[src]) : w[src];
  }
}

// K = G diag(lam) (FP64, k x k)
__global__ void scale_cols_kernel(const double *G, int k, const double *lam, double *K) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < k * k; q += gridDim.x * blockDim.x) {
    const int c = q % k;
    K[q] = G[q] * lam[c];
  }
}

// I (k x k FP64)
__global__ void eye_kernel(double *I, int k) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < k * k; q += gridDim.x * blockDim.x)
    I[q] = (q / k == q % k) ? 1.0 : 0.0;
}

// CfT + CfT_lo = (diag(lam) Csum)^T, i.e. [a][c] = lam_c Csum[c][a], as an
// FP32 pair
__global__ void core_transpose_kernel(const double *Csum, int k, const double *lam, float *CfT,
                                      float *CfT_lo) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < k * k; q += gridDim.x * blockDim.x) {
    const int a = q / k, c = q % k;
    const double v = lam[c] * Csum[(int64_t)c * k + a];
    const float hi = (float)v;
    CfT[q] = hi;
    CfT_lo[q] = (float)(v - (double)hi);
  }
}

inline unsigned grid_for(int64_t work, int per = 256, int cap = 0) {
  if (cap <= 0) cap = sm_count() * 8;
  int64_t b = (work + per - 1) / per;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (unsigned)b;
}

// --------------------------------------------------------------------------
// Pipeline pieces
// --------------------------------------------------------------------------
// Q (n x w) = orth(Y) with eigSVD (frPCA: B = Y^T Y = V diag(w) V^T,
// Q = Y V diag(w)^-1/2) or Cholesky QR (B = R^T R, Q = Y R^-1).  The small
// factorization runs in FP64 when `fp64` (sketch QR), else in FP32 (the
// orthonormalizations inside the power iteration of Alg. 5).
int orth_tall(const Dims &D, const Bufs &b, int method, bool fp64, const float *Y, int64_t ldy, int w,
              float *Q, int64_t ldq, cudaStream_t st, bool accurate_gram = false) {
  if (accurate_gram)
    CK(launch_gram_accurate(Y, ldy, w, Y, ldy, w, D.n, nullptr, nullptr, true, b.partial, b.m64[0], w,
                            st));
  else
    CK(launch_gram(Y, ldy, w, Y, ldy, w, D.n, nullptr, true, b.partial, b.m64[0], w, st, b.ctrl));
  if (method == SNE_ORTH_EIGSVD) {
    CK(launch_d2f(b.m64[0], w, w, w, b.m32[0], w, st));
    CK(launch_sym_eig<float>(b.m32[0], w, w, b.w32, b.m32[1], w, b.eigscr, b.ctrl, st));
    { ProfScope ps_(K_MISC, st); inv_sqrt_cols_kernel<<<grid_for((int64_t)w * w), 256, 0, st>>>(b.m32[1], w, w, b.w32, b.m32[2],
                                                                   w, b.ctrl); }
    CK(cudaGetLastError());
  } else if (fp64) {
    // the sketch QR, in FP64: Y can be ill-conditioned (with half-precision
    // operands its small singular values are rounding noise), and an FP32
    // Cholesky of Y^T Y loses kappa(Y)^2 eps_32.  Pivoted, and cut only at the
    // FP64 noise floor (1e-13 of the largest diagonal), like the Householder
    // QR it stands for, which keeps every direction of Y: Y is rank-deficient
    // when trunc_log(L'R') has rank below h (a graph with more components than
    // sketch columns), and then the factorization stops instead of meeting a
    // non-positive pivot; columns of Q past the stop are zero.
    CK(launch_chol_inverse<double>(b.m64[0], w, w, b.m64[1], w, b.m64[2], b.ctrl, st, 1e-13));
    CK(launch_d2f(b.m64[1], w, w, w, b.m32[2], w, st));
  } else {
    CK(launch_d2f(b.m64[0], w, w, w, b.m32[0], w, st));
    CK(launch_chol_inverse<float>(b.m32[0], w, w, b.m32[2], w, b.m32[1], b.ctrl, st));
  }
  CK(launch_tall_gemm_auto(Y, ldy, D.n, w, b.m32[2], w, w, Q, ldq, b.mT, b.ctrl, st));
  return SNE_OK;
}

// Alg. 5.  Leaves U_k (n x k, ld k) in `U` and lambda (k) in `lam`.
int run_freigs(const sne_csr &g, const sne_params &p, const Dims &D, const Bufs &b, float *U,
               double *lam, cudaStream_t st) {
  const int K = D.K;
  const int64_t ld = D.Wab;
  float *Q = b.A, *T1 = b.B, *T2 = b.C;
  CK(launch_degree_power(b.deg, D.n, -p.alpha, b.dpow, 1.0f, st));
  CK(launch_spmm_weights(g, b.dpow, b.wnz, st));                  // d_j^-alpha a_ij per nonzero
  CK(launch_spmm_hot_threshold(b.dpow, D.n, spmm_row_bytes(D.n, K), b.ctrl, st));  // rows kept in L2
  const uint32_t *hot = &b.ctrl->hot_bits;
  CK(launch_gaussian(D.n, K, p.seed, 1, T1, ld, st));              // Omega
  CK(launch_spmm(g, b.dpow, b.wnz, T1, ld, K, T2, K, st, hot));   // Y = X Omega
  int rc = orth_tall(D, b, p.orth, false, T2, K, K, Q, ld, st);    // Q = eigSVD(Y)
  if (rc) return rc;
  for (int it = 0; it < p.q; ++it) {
    CK(launch_spmm(g, b.dpow, b.wnz, Q, ld, K, T1, ld, st, hot));  // X Q
    CK(launch_spmm(g, b.dpow, b.wnz, T1, ld, K, T2, K, st, hot));  // X X Q
    rc = orth_tall(D, b, p.orth, false, T2, K, K, Q, ld, st);      // Q = eigSVD(X X Q)
    if (rc) return rc;
  }
  // one more FP32 Cholesky-QR pass over the final basis (a no-op in exact
  // arithmetic) so that Q is orthonormal to working precision before the
  // Rayleigh-Ritz step assumes Q^T Q = I
  CK(cudaMemcpy2DAsync(T2, K * sizeof(float), Q, ld * sizeof(float), K * sizeof(float), D.n,
                       cudaMemcpyDeviceToDevice, st));
  rc = orth_tall(D, b, SNE_ORTH_CHOLQR, false, T2, K, K, Q, ld, st);
  if (rc) return rc;
  // Rayleigh-Ritz: S = Q^T X Q (FP64), eig(S), U = Q U_hat, top k by |lambda|
  CK(launch_spmm(g, b.dpow, b.wnz, Q, ld, K, T1, ld, st, hot));
  CK(launch_gram(Q, ld, K, T1, ld, K, D.n, nullptr, false, b.partial, b.m64[0], K, st, b.ctrl));
  CK(launch_symmetrize(b.m64[0], K, K, st));
  CK(launch_sym_eig<double>(b.m64[0], K, K, b.w64, b.m64[1], K, b.eigscr, b.ctrl, st));
  CK(launch_eig_order<double>(b.w64, K, true, b.perm, st));
  { ProfScope ps_(K_MISC, st); select_cols_kernel<<<grid_for((int64_t)K * D.k), 256, 0, st>>>(b.m64[1], K, K, b.perm, b.w64, D.k,
                                                                 0, b.m32[0], D.k, lam, 0); }
  CK(cudaGetLastError());
  CK(launch_tall_gemm_auto(Q, ld, D.n, K, b.m32[0], D.k, D.k, U, D.k, b.mT, b.ctrl, st));
  return SNE_OK;
}

// Eq. 11 + Alg. 4 from U_k (ld k), lambda.  Optional outputs Y, Z, E, sigma.
// The two tensor-core sketches of one graph: Y = f(L'R'(:, p_S)) S(p_S, :)
// (Alg. 4 line 4) and the Z core's Y' = f(L'(p_O, :) R'(:, p_O)) O(p_O, :)
// (Alg. 4 line 7), on the rows p_O (device count v_o).
void tc_jobs(const Dims &D, const Bufs &b, float *Y, int h, int l, TcSketchJobDesc *jobs) {
  const int64_t vmax = min64(D.n, D.nO);
  jobs[0] = TcSketchJobDesc{b.Ah, b.Al, b.BhS, b.BlS, D.n, nullptr, (int32_t)D.nS, h,
                            b.rowfA, b.rowdat, b.coldatS, Y, h, b.ctrl};
  jobs[1] = TcSketchJobDesc{b.AhO, b.AlO, b.BhO, b.BlO, vmax, &b.ctrl->v_o, (int32_t)D.nO, l,
                            b.rowfO, b.rowdatO, b.coldatO, b.Yo, l, b.ctrl};
}

TcTune tc_tune_for(const Dims &D) {
  return tc_tune_lookup(D.kpad, D.split, D.fp16, D.z, D.n);
}

// phase 0: all of it.  Phase 1 (half-precision reconstructions only): up to
// the tensor-core sketch, whose two jobs go to jobs_out instead of being
// launched (a batch runs the sketches of all its graphs in one launch).
// Phase 2: from the sketch results on.
int run_sketch(const sne_csr &g, const sne_params &p, const Dims &D, const Bufs &b, const float *U,
               const double *lam, float *Yout, float *Zout, float *E, double *sigma,
               cudaStream_t st, int phase = 0, TcSketchJobDesc *jobs_out = nullptr) {
  const int k = D.k, h = D.h, l = D.l, z = D.z;
  const float sv = 1.0f / sqrtf((float)z);
  float *Y = Yout ? Yout : b.A;
  if (phase == 1 && (!D.half || !jobs_out)) return SNE_ERR_ARG;
  if (phase != 2) {
  // --- Eq. 11 factors
  // d^(-1+2alpha) in FP64, as the FP32 pair (wgt, wgt_lo)
  { ProfScope ps_(K_MISC, st); rowscale_kernel<<<grid_for(D.n), 256, 0, st>>>(b.deg, D.n, -1.0 + 2.0 * p.alpha, nullptr,
                                                 1.0, b.wgt, b.wgt_lo); }
  CK(cudaGetLastError());
  { ProfScope ps_(K_MISC, st); rowscale_kernel<<<grid_for(D.n), 256, 0, st>>>(b.deg, D.n, -1.0 + p.alpha, &b.ctrl->vol,
                                                 1.0 / (p.b * p.T), b.rsc, b.rsc_lo); }    // vol/(bT) a
  CK(cudaGetLastError());
  // G = U^T D^(-1+2 alpha) U in FP64 accuracy: most entries of L'R' lie just
  // above the trunc_log threshold, where an error in the core C shifts every
  // one of them, and the Horner sum multiplies the error of G by up to T^2/2
  CK(launch_gram_accurate(U, k, k, U, k, k, D.n, b.wgt, b.wgt_lo, true, b.partial, b.m64[0], k, st,
                          true));
  { ProfScope ps_(K_MISC, st); scale_cols_kernel<<<grid_for((int64_t)k * k), 256, 0, st>>>(b.m64[0], k, lam, b.m64[1]); }  // K
  { ProfScope ps_(K_MISC, st); eye_kernel<<<grid_for((int64_t)k * k), 256, 0, st>>>(b.m64[2], k); }                        // I
  CK(cudaGetLastError());
  // Horner in FP64: Csum = I + K (I + K (... (I))) = sum_{r=1..T} K^(r-1)
  double *cur = b.m64[2], *nxt = b.m64[3];
  for (int r = 1; r < p.T; ++r) {
    { ProfScope ps_(K_MISC, st); eye_kernel<<<grid_for((int64_t)k * k), 256, 0, st>>>(nxt, k); }
    CK(cudaGetLastError());
    CK(launch_small_gemm<double>(false, false, k, k, k, 1.0, b.m64[1], k, cur, k, 1.0, nxt, k, st));
    std::swap(cur, nxt);
  }
  { ProfScope ps_(K_MISC, st); core_transpose_kernel<<<grid_for((int64_t)k * k), 256, 0, st>>>(cur, k, lam, b.m32[3], b.m32[2]); }  // C^T
  CK(cudaGetLastError());
  // --- centring of L'R' (the degree-weighted mean row w of W = D^(-1+a) U):
  // x - c0 = s (W_i - w) C (W_j - w)^T + rho_i + kappa_j, c0 = 1 for trunc_log
  const bool tlog = p.f == SNE_F_TRUNC_LOG;
  const double c0 = tlog ? 1.0 : 0.0;
  CK(launch_center_stats(U, k, k, D.n, b.deg, p.alpha, &b.ctrl->vol, lam, cur, 1.0 / (p.b * p.T),
                         c0, b.cpart, b.cstats, b.ws_hi, b.ws_lo, st));
  // --- Alg. 3: S (stream 2) and O (stream 3); unique coordinates
  CK(launch_sparse_sign(D.n, h, z, p.seed, 2, b.idxS, b.signS, b.ctrl, st));
  CK(launch_sparse_sign(D.n, l, z, p.seed, 3, b.idxO, b.signO, b.ctrl, st));
  CK(launch_unique(b.idxS, D.nS, b.uniqS, &b.ctrl->v_s, b.posS, b.ctrl, W_UNIQUE, st));
  CK(launch_unique(b.idxO, D.nO, b.uniqO, &b.ctrl->v_o, b.posO, b.ctrl, W_UNIQUE, st));
  // centred columns R~(:, idx)^T = (W_idx - w) C^T and their (scale, kappa, sign);
  // the padding past the last column reads as zero
  CK(cudaMemsetAsync(b.coldatS, 0, (size_t)(D.nS + 256) * sizeof(float4), st));
  CK(cudaMemsetAsync(b.coldatO, 0, (size_t)(D.nO + 256) * sizeof(float4), st));
  CK(launch_rtilde_rows(U, k, b.idxS, D.nS, b.m32[3], b.m32[2], b.deg, -1.0 + p.alpha, b.cstats,
                        b.signS, b.RpS, b.coldatS, st));
  CK(launch_rtilde_rows(U, k, b.idxO, D.nO, b.m32[3], b.m32[2], b.deg, -1.0 + p.alpha, b.cstats,
                        b.signO, b.RpO, b.coldatO, st));
  // --- Alg. 4 line 4: Y = f(L' R'(:, p)) S(p, :)
  // --- Alg. 4 line 7: Y' = f(L'(p,:) R'(:,p)) O(p,:) on the rows p = p_O
  const int64_t vmax = min64(D.n, D.nO);
  if (!D.half) {
    // centred rows L~ = s (W - w) (FP32) in the free tall buffer
    float *Lt = b.B;
    CK(launch_center_rows(0, false, U, k, k, nullptr, nullptr, D.n, b.rsc, b.rsc_lo, b.ws_hi,
                          b.ws_lo, b.cstats, tlog, c0, Lt, k, nullptr, nullptr, 0, nullptr,
                          b.rowdat, st));
    CK(launch_fused_sketch_f32(Lt, k, nullptr, nullptr, D.n, k, b.rowdat, b.RpS, b.coldatS, h, z,
                               sv, p.f, Y, h, st));
    CK(launch_fused_sketch_f32(Lt, k, b.uniqO, &b.ctrl->v_o, vmax, k, b.rowdat, b.RpO, b.coldatO,
                               l, z, sv, p.f, b.Yo, l, st));
  } else {
    const int outk = D.fp16 ? 1 : 2;
    CK(launch_center_rows(outk, D.split, U, k, k, nullptr, nullptr, D.n, b.rsc, b.rsc_lo, b.ws_hi,
                          b.ws_lo, b.cstats, tlog, c0, nullptr, 0, b.Ah, b.Al, D.kpad, b.rowfA,
                          b.rowdat, st));
    CK(launch_center_rows(outk, D.split, U, k, k, b.uniqO, &b.ctrl->v_o, vmax, b.rsc, b.rsc_lo,
                          b.ws_hi, b.ws_lo, b.cstats, tlog, c0, nullptr, 0, b.AhO, b.AlO, D.kpad,
                          b.rowfO, b.rowdatO, st));
    // column scales go to coldat[e].x
    CK(launch_split_rows(D.fp16, D.split, b.RpS, k, D.nS, k, D.kpad, b.BhS, b.BlS,
                         reinterpret_cast<float *>(b.coldatS), 4, st));
    CK(launch_split_rows(D.fp16, D.split, b.RpO, k, D.nO, k, D.kpad, b.BhO, b.BlO,
                         reinterpret_cast<float *>(b.coldatO), 4, st));
    // zero rows past the evaluated columns up to the 256-row tile boundary
    const size_t rb = (size_t)D.kpad * 2;
    CK(cudaMemsetAsync(static_cast<char *>(b.BhS) + (size_t)D.nS * rb, 0,
                       (size_t)(pad256(D.nS) - D.nS) * rb, st));
    CK(cudaMemsetAsync(static_cast<char *>(b.BhO) + (size_t)D.nO * rb, 0,
                       (size_t)(pad256(D.nO) - D.nO) * rb, st));
    if (D.split) {
      CK(cudaMemsetAsync(static_cast<char *>(b.BlS) + (size_t)D.nS * rb, 0,
                         (size_t)(pad256(D.nS) - D.nS) * rb, st));
      CK(cudaMemsetAsync(static_cast<char *>(b.BlO) + (size_t)D.nO * rb, 0,
                         (size_t)(pad256(D.nO) - D.nO) * rb, st));
    }
    // Y and the Z core's Y' in one persistent launch
    TcSketchJobDesc jobs[2];
    tc_jobs(D, b, Y, h, l, jobs);
    if (phase == 1) {
      jobs_out[0] = jobs[0];
      jobs_out[1] = jobs[1];
      return SNE_OK;
    }
    CK(launch_fused_sketch_tc_jobs(D.fp16, D.split, b.arena, b.arena_bytes, D.kpad, z, sv, p.f, jobs,
                                   2, tc_tune_for(D), b.ctrl, st));
  }
  }  // phase != 2
  // --- Z = O(p,:)^T Y'  (Alg. 4 line 7)
  float *Z = Zout ? Zout : b.Zf;
  CK(launch_signed_gather_sum(b.Yo, l, l, b.posO, b.signO, l, z, sv, Z, l, st));
  if (!E && !sigma) return SNE_OK;
  // O^T Y (FP64), taken before Y's buffer is reused for Q
  CK(launch_signed_gather_sum64(Y, h, h, b.idxO, b.signO, l, z, (double)sv, b.Tm, h, st));
  // --- Alg. 4 line 5: Q = orth(Y) = Y R^-1 by Cholesky QR, twice (R = R2 R1)
  // the first pass sees Y itself: Cholesky QR loses about kappa(Y)^2 times the
  // Gram's relative error, so this Gram is the FP64-accurate one
  int rc = orth_tall(D, b, SNE_ORTH_CHOLQR, true, Y, h, h, b.B, h, st, true);  // Q1 = Y R1^-1
  if (rc) return rc;
  CK(cudaMemcpyAsync(b.m64[3], b.m64[1], (size_t)h * h * sizeof(double), cudaMemcpyDeviceToDevice,
                     st));                                                  // R1^-1
  rc = orth_tall(D, b, SNE_ORTH_CHOLQR, true, b.B, h, h, b.A, h, st);    // Q = Q1 R2^-1
  if (rc) return rc;
  float *Q = b.A;
  CK(launch_small_gemm<double>(false, false, h, h, h, 1.0, b.m64[3], h, b.m64[1], h, 0.0, b.m64[4],
                               h, st));                                     // R^-1 = R1^-1 R2^-1
  // --- Alg. 4 line 8: W = (O^T Q)^+ Z (Q^T O)^+ via the normal equations (FP64).
  // G = O^T Q is formed as (O^T Y) R^-1 in FP64: the solves magnify errors in
  // G by cond(G) (several thousand on large power-law graphs), so G must not
  // carry the FP32 rounding of Q
  CK(launch_small_gemm<double>(false, false, l, h, h, 1.0, b.Tm, h, b.m64[4], h, 0.0, b.G64, h, st));
  CK(launch_f2d(Z, l, l, l, b.Z64, l, st));
  CK(launch_small_gemm<double>(true, false, h, h, l, 1.0, b.G64, h, b.G64, h, 0.0, b.m64[0], h, st));
  // (G^T G)^+ = M M^T with M = P R^-1 from the pivoted Cholesky G^T G = P R^T R P^T;
  // zero columns of G (directions Q lacks) are cut, which gives the
  // minimum-norm least-squares solutions
  CK(launch_chol_inverse<double>(b.m64[0], h, h, b.m64[1], h, b.m64[2], b.ctrl, st, 1e-12));
  CK(launch_small_gemm<double>(false, true, h, h, h, 1.0, b.m64[1], h, b.m64[1], h, 0.0, b.m64[2], h,
                               st));                                               // (G^T G)^-1
  CK(launch_small_gemm<double>(false, true, h, l, h, 1.0, b.m64[2], h, b.G64, h, 0.0, b.Gp, l, st));
  CK(launch_small_gemm<double>(false, false, h, l, l, 1.0, b.Gp, l, b.Z64, l, 0.0, b.Tm, l, st));
  CK(launch_small_gemm<double>(false, true, h, h, l, 1.0, b.Tm, l, b.Gp, l, 0.0, b.m64[3], h, st));
  // --- Alg. 4 line 9: svd(W).  W is symmetric (Z is), so its singular values
  // are |eigenvalues| and its left singular vectors are eigenvectors (Lemma 1).
  CK(launch_symmetrize(b.m64[3], h, h, st));
  CK(launch_sym_eig<double>(b.m64[3], h, h, b.w64, b.m64[4], h, b.eigscr, b.ctrl, st));
  CK(launch_eig_order<double>(b.w64, h, true, b.perm, st));
  // E = Q U_hat(:, 1:d) Sigma_d^(1/2)  (Alg. 4 line 10, Alg. 6 line 5)
  { ProfScope ps_(K_MISC, st); select_cols_kernel<<<grid_for((int64_t)h * D.d), 256, 0, st>>>(b.m64[4], h, h, b.perm, b.w64, D.d,
                                                                 1, b.m32[0], D.d, sigma, 1); }
  CK(cudaGetLastError());
  if (E) CK(launch_tall_gemm_auto(Q, h, D.n, h, b.m32[0], D.d, D.d, E, D.d, b.mT, b.ctrl, st));
  return SNE_OK;
}

}  // namespace

// ==========================================================================
// extern "C" entry points
// ==========================================================================
extern "C" {

int sne_params_init(sne_params *p, int32_t d, int32_t k) {
  if (!p || d <= 0 || k <= 0) return SNE_ERR_ARG;
  std::memset(p, 0, sizeof(*p));
  p->k = k;
  p->q = 20;
  p->T = 10;
  p->d = d;
  p->h = 2 * d + 16;
  p->l = d + 1000;
  p->zeta = 8;
  p->s_eig = 16;
  p->row_block = 0;
  p->precision = SNE_FP32;
  p->f = SNE_F_TRUNC_LOG;
  p->orth = SNE_ORTH_EIGSVD;
  p->alpha = 0.5;
  p->b = 1.0;
  p->seed = 0;
  return SNE_OK;
}

const char *sne_error_string(int code) {
  switch (code) {
    case SNE_OK: return "ok";
    case SNE_ERR_ARG: return "invalid argument";
    case SNE_ERR_GRAPH: return "invalid graph (CSR not monotone, out of range or asymmetric, or no edges)";
    case SNE_ERR_SIZE: return "inconsistent or unsupported sizes";
    case SNE_ERR_WORKSPACE: return "workspace missing, too small or misaligned";
    case SNE_ERR_CUDA: return "CUDA error";
    case SNE_ERR_TIMEOUT: return "bounded device wait timed out";
    case SNE_ERR_NUMERIC: return "numerical failure (NaN/Inf or non-positive pivot)";
    default: return "unknown error";
  }
}

int sne_workspace_bytes(int64_t n, int64_t nnz, const sne_params *p, int mode, size_t *bytes) {
  if (!bytes || mode < SNE_WS_EMBED || mode > SNE_WS_EMBED_HOST) return SNE_ERR_ARG;
  Dims D;
  int rc = make_dims(n, nnz, p, mode, &D);
  if (rc) return rc;
  *bytes = carve(D, mode, nullptr, nullptr);
  return SNE_OK;
}

int sne_status_reset(void *ws, sne_stream_t stream) {
  if (!ws) return SNE_ERR_WORKSPACE;
  return cudaMemsetAsync(ws, 0, sizeof(Ctrl), (cudaStream_t)stream) == cudaSuccess ? SNE_OK
                                                                                 : SNE_ERR_CUDA;
}

int sne_status(const void *ws, sne_stream_t stream) {
  if (!ws) return SNE_ERR_WORKSPACE;
  int32_t st = 0;
  if (cudaMemcpyAsync(&st, ws, sizeof(int32_t), cudaMemcpyDeviceToHost, (cudaStream_t)stream) !=
      cudaSuccess)
    return SNE_ERR_CUDA;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return SNE_ERR_CUDA;
  return st;
}

int sne_stats_read(const void *ws, sne_stats *out, sne_stream_t stream) {
  if (!ws || !out) return SNE_ERR_ARG;
  Ctrl c;
  if (cudaMemcpyAsync(&c, ws, sizeof(Ctrl), cudaMemcpyDeviceToHost, (cudaStream_t)stream) !=
      cudaSuccess)
    return SNE_ERR_CUDA;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return SNE_ERR_CUDA;
  out->status = c.status;
  out->where = c.where;
  out->v_s = c.v_s;
  out->v_o = c.v_o;
  out->vol = c.vol;
  return SNE_OK;
}

int sne_sparse_sign(int64_t n, int32_t cols, int32_t zeta, uint64_t seed, int32_t stream_id,
                    int32_t *idx, int8_t *sign, sne_stream_t stream) {
  if (n <= 0 || cols < 0 || zeta <= 0 || !idx || !sign || n > (int64_t)INT32_MAX - 1)
    return SNE_ERR_ARG;
  const int z = (int)min64(n, zeta);
  if (z > 64) return SNE_ERR_SIZE;
  return launch_sparse_sign(n, cols, z, seed, stream_id, idx, sign, nullptr, (cudaStream_t)stream) ==
                 cudaSuccess
             ? SNE_OK
             : SNE_ERR_CUDA;
}

int sne_gaussian(int64_t n, int32_t cols, uint64_t seed, int32_t stream_id, float *out,
                 sne_stream_t stream) {
  if (n < 0 || cols < 0 || (!out && n * cols > 0)) return SNE_ERR_ARG;
  return launch_gaussian(n, cols, seed, stream_id, out, cols, (cudaStream_t)stream) == cudaSuccess
             ? SNE_OK
             : SNE_ERR_CUDA;
}

int sne_degrees(const sne_csr *g, float *deg, double *vol, sne_stream_t stream) {
  int rc = check_graph(g);
  if (rc) return rc;
  if (!deg || !vol) return SNE_ERR_ARG;
  return launch_degrees(*g, deg, vol, (cudaStream_t)stream) == cudaSuccess ? SNE_OK : SNE_ERR_CUDA;
}

int sne_degree_power(const float *deg, int64_t n, double beta, float *out, sne_stream_t stream) {
  if (n < 0 || (n > 0 && (!deg || !out))) return SNE_ERR_ARG;
  return launch_degree_power(deg, n, beta, out, 1.0f, (cudaStream_t)stream) == cudaSuccess
             ? SNE_OK
             : SNE_ERR_CUDA;
}

int sne_spmm_weights(const sne_csr *g, const float *dpow, float *w_nz, sne_stream_t stream) {
  int rc = check_graph(g);
  if (rc) return rc;
  if (!dpow || (!w_nz && g->nnz > 0)) return SNE_ERR_ARG;
  return launch_spmm_weights(*g, dpow, w_nz, (cudaStream_t)stream) == cudaSuccess ? SNE_OK
                                                                                 : SNE_ERR_CUDA;
}

int sne_spmm(const sne_csr *g, const float *dpow, const float *w_nz, const float *B, int32_t ncols,
             float *Y, sne_stream_t stream) {
  int rc = check_graph(g);
  if (rc) return rc;
  if (!dpow || !B || !Y || ncols <= 0 || B == Y) return SNE_ERR_ARG;
  return launch_spmm(*g, dpow, w_nz, B, ncols, ncols, Y, ncols, (cudaStream_t)stream) == cudaSuccess
             ? SNE_OK
             : SNE_ERR_CUDA;
}

int sne_validate_csr(const sne_csr *g, void *ws, size_t ws_bytes, sne_stream_t stream) {
  int rc = check_graph(g);
  if (rc) return rc;
  rc = check_ws(ws, ws_bytes, sizeof(Ctrl));
  if (rc) return rc;
  return launch_validate(*g, reinterpret_cast<Ctrl *>(ws), (cudaStream_t)stream) == cudaSuccess
             ? SNE_OK
             : SNE_ERR_CUDA;
}

static int general_check(int64_t n, int64_t m, int32_t k, const sne_params *p) {
  if (!p || n <= 0 || m <= 0 || k <= 0 || p->d <= 0 || p->h <= 0 || p->l <= 0 || p->zeta <= 0)
    return SNE_ERR_ARG;
  if (p->f != SNE_F_TRUNC_LOG && p->f != SNE_F_IDENTITY) return SNE_ERR_ARG;
  if (n > (int64_t)INT32_MAX - 1 || m > (int64_t)INT32_MAX - 1 || k > 4096) return SNE_ERR_SIZE;
  const int64_t zn = std::min<int64_t>(n, p->zeta), zm = std::min<int64_t>(m, p->zeta);
  if (zn > 64 || zm > 64) return SNE_ERR_SIZE;
  if (p->d > p->h || p->h > p->l || p->h > std::min(n, m) || p->h > kFastEigMaxN) return SNE_ERR_SIZE;
  if ((int64_t)p->l * zn > kUniqueMax || (int64_t)p->l * zm > kUniqueMax) return SNE_ERR_SIZE;
  return SNE_OK;
}

int sne_single_pass_svd_workspace_bytes(int64_t n, int64_t m, int32_t k, const sne_params *p,
                                        size_t *bytes) {
  if (!bytes) return SNE_ERR_ARG;
  const int rc = general_check(n, m, k, p);
  if (rc) return rc;
  *bytes = general_workspace_bytes(n, m, k, p->d, p->h, p->l, p->zeta);
  return SNE_OK;
}

int sne_single_pass_svd(int64_t n, int64_t m, int32_t k, const float *L, int64_t ldl,
                        const float *Rt, int64_t ldr, const sne_params *p, void *ws,
                        size_t ws_bytes, float *U, int64_t ldu, double *sigma, float *V,
                        int64_t ldv, sne_stream_t stream) {
  int rc = general_check(n, m, k, p);
  if (rc) return rc;
  if (!L || !Rt || !sigma || ldl < k || ldr < k || (U && ldu < p->d) || (V && ldv < p->d))
    return SNE_ERR_ARG;
  rc = check_ws(ws, ws_bytes, general_workspace_bytes(n, m, k, p->d, p->h, p->l, p->zeta));
  if (rc) return rc;
  return run_general_svd(n, m, k, L, ldl, Rt, ldr, *p, ws, U, ldu, sigma, V, ldv,
                         (cudaStream_t)stream);
}

int sne_propagation_coefficients(int32_t steps, double theta, double *c) {
  if (!c || steps < 0 || steps > kMaxPropagationSteps || !(theta >= 0.0) || !std::isfinite(theta))
    return SNE_ERR_ARG;
  propagation_coefficients(steps, theta, c);
  return SNE_OK;
}

int sne_spectral_propagate_workspace_bytes(int64_t n, int32_t d, size_t *bytes) {
  if (!bytes || n <= 0 || d <= 0 || d > kMaxPropagationWidth) return SNE_ERR_ARG;
  *bytes = propagate_workspace_bytes(n, d);
  return SNE_OK;
}

int sne_spectral_propagate(const sne_csr *g, int32_t steps, double theta, double mu, float *E,
                           int64_t lde, int32_t d, void *ws, size_t ws_bytes, sne_stream_t stream) {
  int rc = check_graph(g);
  if (rc) return rc;
  if (!E || d <= 0 || d > kMaxPropagationWidth || lde < d || steps < 0 ||
      steps > kMaxPropagationSteps || !(theta >= 0.0) || !std::isfinite(theta) || !(mu >= 0.0) ||
      !(mu <= 2.0))
    return SNE_ERR_ARG;
  rc = check_ws(ws, ws_bytes, propagate_workspace_bytes(g->n, d));
  if (rc) return rc;
  return run_propagate(*g, steps, theta, mu, E, lde, d, ws, (cudaStream_t)stream);
}

int sne_freigs(const sne_csr *g, const sne_params *p, void *ws, size_t ws_bytes, float *U,
               double *lambda, sne_stream_t stream) {
  int rc = check_graph(g);
  if (rc) return rc;
  rc = check_has_edges(g);
  if (rc) return rc;
  Dims D;
  rc = make_dims(g->n, g->nnz, p, SNE_WS_FREIGS, &D);
  if (rc) return rc;
  Bufs b;
  rc = check_ws(ws, ws_bytes, carve(D, SNE_WS_FREIGS, nullptr, nullptr));
  if (rc) return rc;
  if (!U || !lambda) return SNE_ERR_ARG;
  carve(D, SNE_WS_FREIGS, ws, &b);
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemsetAsync(b.ctrl, 0, sizeof(Ctrl), st));
  CK(launch_degrees(*g, b.deg, &b.ctrl->vol, st));
  return run_freigs(*g, *p, D, b, U, lambda, st);
}

int sne_sketch_from_factors(const sne_csr *g, const sne_params *p, const float *U,
                            const double *lambda, void *ws, size_t ws_bytes, float *Y, float *Z,
                            float *E, double *sigma, sne_stream_t stream) {
  int rc = check_graph(g);
  if (rc) return rc;
  rc = check_has_edges(g);
  if (rc) return rc;
  Dims D;
  rc = make_dims(g->n, g->nnz, p, SNE_WS_SKETCH, &D);
  if (rc) return rc;
  rc = check_ws(ws, ws_bytes, carve(D, SNE_WS_SKETCH, nullptr, nullptr));
  if (rc) return rc;
  if (!U || !lambda) return SNE_ERR_ARG;
  Bufs b;
  carve(D, SNE_WS_SKETCH, ws, &b);
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemsetAsync(b.ctrl, 0, sizeof(Ctrl), st));
  CK(launch_degrees(*g, b.deg, &b.ctrl->vol, st));
  return run_sketch(*g, *p, D, b, U, lambda, Y, Z, E, sigma, st);
}

int sne_embed(const sne_csr *g, const sne_params *p, void *ws, size_t ws_bytes, float *E,
              double *sigma, sne_stream_t stream) {
  int rc = check_graph(g);
  if (rc) return rc;
  rc = check_has_edges(g);
  if (rc) return rc;
  Dims D;
  rc = make_dims(g->n, g->nnz, p, SNE_WS_EMBED, &D);
  if (rc) return rc;
  rc = check_ws(ws, ws_bytes, carve(D, SNE_WS_EMBED, nullptr, nullptr));
  if (rc) return rc;
  if (!E || !sigma) return SNE_ERR_ARG;
  Bufs b;
  carve(D, SNE_WS_EMBED, ws, &b);
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemsetAsync(b.ctrl, 0, sizeof(Ctrl), st));
  CK(launch_degrees(*g, b.deg, &b.ctrl->vol, st));
  // U_k goes to the third tall buffer, lambda to the FP64 scratch tail
  float *Uk = b.C;
  double *lam = b.lam;
  rc = run_freigs(*g, *p, D, b, Uk, lam, st);
  if (rc) return rc;
  return run_sketch(*g, *p, D, b, Uk, lam, nullptr, nullptr, E, sigma, st);
}

int sne_embed_host(const sne_csr *g, const sne_params *p, void *ws, size_t ws_bytes, float *E_host,
                   double *sigma_host, sne_stream_t stream) {
  int rc = check_graph(g);
  if (rc) return rc;
  rc = check_has_edges(g);
  if (rc) return rc;
  Dims D;
  rc = make_dims(g->n, g->nnz, p, SNE_WS_EMBED_HOST, &D);
  if (rc) return rc;
  rc = check_ws(ws, ws_bytes, carve(D, SNE_WS_EMBED_HOST, nullptr, nullptr));
  if (rc) return rc;
  if (!E_host || !sigma_host) return SNE_ERR_ARG;
  Bufs b;
  carve(D, SNE_WS_EMBED_HOST, ws, &b);
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemcpyAsync(b.h_rowptr, g->row_ptr, (D.n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
  if (D.nnz > 0)
    CK(cudaMemcpyAsync(b.h_col, g->col_idx, D.nnz * sizeof(int32_t), cudaMemcpyHostToDevice, st));
  if (g->val && D.nnz > 0)
    CK(cudaMemcpyAsync(b.h_val, g->val, D.nnz * sizeof(float), cudaMemcpyHostToDevice, st));
  sne_csr dg{g->n, g->nnz, b.h_rowptr, b.h_col, g->val ? b.h_val : nullptr};
  rc = sne_embed(&dg, p, ws, ws_bytes, b.h_E, b.h_sigma, stream);
  if (rc) return rc;
  CK(cudaMemcpyAsync(E_host, b.h_E, (size_t)D.n * D.d * sizeof(float), cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(sigma_host, b.h_sigma, D.d * sizeof(double), cudaMemcpyDeviceToHost, st));
  return SNE_OK;
}

}  // extern "C"

// ==========================================================================
// Allocation-free variant of sne_freigs.  Its workspace is a static device
// array of this library (one per device the library is used on), so the
// caller passes only inputs and outputs.
// ==========================================================================
namespace {

constexpr size_t kStaticWorkspaceBytes = (size_t)32 << 20;  // 32 MiB
__device__ __align__(256) unsigned char g_static_workspace[kStaticWorkspaceBytes];

constexpr int kMaxDevices = 64;
std::mutex g_static_mu;
void *g_static_ptr[kMaxDevices] = {nullptr};

// Device address of g_static_workspace on the current device.  The host name
// of a __device__ array is only a stand-in, so the address is looked up once
// per device with cudaGetSymbolAddress and cached.
int static_workspace_ptr(void **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return SNE_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_static_mu);
  if (g_static_ptr[dev] == nullptr) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_static_workspace) != cudaSuccess || ptr == nullptr)
      return SNE_ERR_CUDA;
    g_static_ptr[dev] = ptr;
  }
  *out = g_static_ptr[dev];
  return SNE_OK;
}

}  // namespace

extern "C" int sne_freigs_static(const sne_csr *g, const sne_params *p, float *U, double *lambda,
                                 int32_t *status, sne_stream_t stream) {
  int rc = check_graph(g);
  if (rc) return rc;
  rc = check_has_edges(g);
  if (rc) return rc;
  Dims D;
  rc = make_dims(g->n, g->nnz, p, SNE_WS_FREIGS, &D);
  if (rc) return rc;
  if (!U || !lambda) return SNE_ERR_ARG;
  if (carve(D, SNE_WS_FREIGS, nullptr, nullptr) > kStaticWorkspaceBytes) return SNE_ERR_SIZE;
  void *ws = nullptr;
  rc = static_workspace_ptr(&ws);
  if (rc) return rc;
  Bufs b;
  carve(D, SNE_WS_FREIGS, ws, &b);
  cudaStream_t st = (cudaStream_t)stream;
  CK(cudaMemsetAsync(b.ctrl, 0, sizeof(Ctrl), st));  // the array keeps the previous call's status
  CK(launch_degrees(*g, b.deg, &b.ctrl->vol, st));
  rc = run_freigs(*g, *p, D, b, U, lambda, st);
  if (rc) return rc;
  if (status)
    CK(cudaMemcpyAsync(status, &b.ctrl->status, sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
  return SNE_OK;
}

namespace sne {

bool embed_tc_shape(const sne_csr *g, const sne_params *p, TcShape *out) {
  Dims D;
  if (!g || make_dims(g->n, g->nnz, p, SNE_WS_EMBED, &D) != SNE_OK || !D.half) return false;
  out->kpad = D.kpad;
  out->fp16 = D.fp16;
  out->split = D.split;
  out->z = D.z;
  out->f = p->f;
  return true;
}

size_t tc_row_bytes(const sne_params *p) {
  Dims D;
  if (make_dims(1 << 20, 1 << 20, p, SNE_WS_EMBED, &D) != SNE_OK) return 256;
  return D.half ? (size_t)D.kpad * 2 : 256;
}

int embed_phase(const sne_csr *g, const sne_params *p, void *ws, size_t ws_bytes, float *E,
                double *sigma, int phase, TcSketchJobDesc *jobs, cudaStream_t st) {
  int rc = check_graph(g);
  if (rc) return rc;
  rc = check_has_edges(g);
  if (rc) return rc;
  Dims D;
  rc = make_dims(g->n, g->nnz, p, SNE_WS_EMBED, &D);
  if (rc) return rc;
  if (!D.half || (phase != 1 && phase != 2)) return SNE_ERR_ARG;
  rc = check_ws(ws, ws_bytes, carve(D, SNE_WS_EMBED, nullptr, nullptr));
  if (rc) return rc;
  if (!E || !sigma) return SNE_ERR_ARG;
  Bufs b;
  carve(D, SNE_WS_EMBED, ws, &b);
  float *Uk = b.C;
  double *lam = b.lam;
  if (phase == 1) {
    CK(cudaMemsetAsync(b.ctrl, 0, sizeof(Ctrl), st));
    CK(launch_degrees(*g, b.deg, &b.ctrl->vol, st));
    rc = run_freigs(*g, *p, D, b, Uk, lam, st);
    if (rc) return rc;
    return run_sketch(*g, *p, D, b, Uk, lam, nullptr, nullptr, E, sigma, st, 1, jobs);
  }
  return run_sketch(*g, *p, D, b, Uk, lam, nullptr, nullptr, E, sigma, st, 2, nullptr);
}

}  // namespace sne
