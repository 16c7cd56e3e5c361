// The general randomized single-pass SVD of Eqs. 5-10 (Sec. 4.1) for a
// rectangular, not necessarily symmetric f(L R): L is n x k, R = Rt^T is
// k x m, f is trunc_log or the identity applied entrywise, and neither the
// n x m matrix nor f of it is ever stored.
//
//   C (n x h), S (m x h), H (n x l), O (m x l)   sparse-sign (Alg. 3; random
//                                               streams 4, 2, 5, 3)
//   Y = f(LR) S,  K = f(LR)^T C,  Z = H^T f(LR) O                 (Eq. 5)
//   Q = orth(Y),  P = orth(K)                                      (Eq. 6)
//   W = (H^T Q)^+ Z (P^T O)^+                                      (Eq. 9)
//   f(LR) ~ Q W P^T,  svd(W) = U_w Sigma V_w^T  ->  U = Q U_w, V = P V_w (Eq. 10)
//
// Y, K and the l columns of f(LR) O on the rows of H are the fused FP32
// reconstruct + f + sparse-sign kernel of sketch.cu (every evaluated entry
// x = <L_i, R_j>, f(x) = log1p(x - 1) for x > 1 or x itself); Z is a signed
// gather of those rows.  orth is Cholesky QR twice with an FP64 pivoted
// Cholesky on the double-float Gram (as for the sketch QR of Alg. 4), and
// H^T Q, O^T P are formed in FP64 as (H^T Y) R_Y^-1 and (O^T K) R_K^-1.  The
// two least-squares solves go through the normal equations in FP64 with the
// pivoted Cholesky, and the SVD of the general h x h W comes from the FP64
// symmetric eigendecomposition W^T W = V_w Sigma^2 V_w^T, U_w = W V_w Sigma^-1
// (the leading d triplets, whose relative accuracy the squaring costs only
// (sigma_1 / sigma_d)^2 eps_64).
#include <algorithm>
#include <cmath>

#include "sne_internal.cuh"

namespace sne {

namespace {

inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

struct GenBufs {
  Ctrl *ctrl;
  int32_t *idxC, *idxS, *idxH, *idxO, *uniqH, *posH;
  int8_t *sgnC, *sgnS, *sgnH, *sgnO;
  float *BS, *BC, *BO;        // gathered rows of Rt (S, O) and L (C), k columns
  float4 *cdS, *cdC, *cdO;    // (1, 0, sign, 0) per sparse-sign nonzero
  float2 *rowdat;             // (-c0, 0) for every row
  float *Y, *K, *tmp;         // n x h, m x h, max(n, m) x h
  float *Yh, *Z;              // rows of f(LR) O on the rows of H (l z_n x l), Z (l x l)
  float *partial;             // Gram scratch
  float *m32;                 // 3 h x h FP32
  float *Mt;                  // tall-product scratch (the split M^T)
  double *HY, *OK, *G1, *G2;  // l x h FP64
  double *R1, *R2, *RY, *RK;  // h x h FP64
  double *N, *Ni, *NN;        // h x h FP64 (normal equations)
  double *Gp1, *Gp2, *Tm;     // h x l FP64
  double *W, *Z64;            // h x h, l x l
  double *WtW, *Vw64, *ww;    // h x h, h x h, h
  double *Vsel, *Usel;        // h x d
  double *chs;                // Cholesky scratch (h^2 + 2h + 8)
  int32_t *perm;              // h
  void *eigscr;
};

struct GenDims {
  int64_t n, m;
  int k, d, h, l, zn, zm;
};

size_t gen_carve(const GenDims &D, void *base, GenBufs *b) {
  size_t off = 0;
  char *p = static_cast<char *>(base);
  auto take = [&](size_t bytes) {
    void *r = p ? p + off : nullptr;
    off += a256(bytes);
    return r;
  };
  const int64_t nC = (int64_t)D.h * D.zn, nS = (int64_t)D.h * D.zm;
  const int64_t nH = (int64_t)D.l * D.zn, nO = (int64_t)D.l * D.zm;
  const size_t hh = (size_t)D.h * D.h, lh = (size_t)D.l * D.h;
  GenBufs x{};
  x.ctrl = static_cast<Ctrl *>(take(sizeof(Ctrl)));
  x.idxC = static_cast<int32_t *>(take(nC * 4));
  x.idxS = static_cast<int32_t *>(take(nS * 4));
  x.idxH = static_cast<int32_t *>(take(nH * 4));
  x.idxO = static_cast<int32_t *>(take(nO * 4));
  x.uniqH = static_cast<int32_t *>(take(nH * 4));
  x.posH = static_cast<int32_t *>(take(nH * 4));
  x.sgnC = static_cast<int8_t *>(take(nC));
  x.sgnS = static_cast<int8_t *>(take(nS));
  x.sgnH = static_cast<int8_t *>(take(nH));
  x.sgnO = static_cast<int8_t *>(take(nO));
  x.BS = static_cast<float *>(take(nS * D.k * 4));
  x.BC = static_cast<float *>(take(nC * D.k * 4));
  x.BO = static_cast<float *>(take(nO * D.k * 4));
  x.cdS = static_cast<float4 *>(take(nS * 16));
  x.cdC = static_cast<float4 *>(take(nC * 16));
  x.cdO = static_cast<float4 *>(take(nO * 16));
  x.rowdat = static_cast<float2 *>(take((size_t)std::max(D.n, D.m) * 8));
  x.Y = static_cast<float *>(take((size_t)D.n * D.h * 4));
  x.K = static_cast<float *>(take((size_t)D.m * D.h * 4));
  x.tmp = static_cast<float *>(take((size_t)std::max(D.n, D.m) * D.h * 4));
  x.Yh = static_cast<float *>(take((size_t)nH * D.l * 4));
  x.Z = static_cast<float *>(take((size_t)D.l * D.l * 4));
  x.partial = static_cast<float *>(
      take(std::max(gram_partial_floats(D.n, D.h, D.h), gram_partial_floats(D.m, D.h, D.h)) * 4));
  x.m32 = static_cast<float *>(take(3 * hh * 4));
  x.Mt = static_cast<float *>(take(tall_tc_scratch_floats(D.h, D.h) * 4));
  x.HY = static_cast<double *>(take(lh * 8));
  x.OK = static_cast<double *>(take(lh * 8));
  x.G1 = static_cast<double *>(take(lh * 8));
  x.G2 = static_cast<double *>(take(lh * 8));
  x.R1 = static_cast<double *>(take(hh * 8));
  x.R2 = static_cast<double *>(take(hh * 8));
  x.RY = static_cast<double *>(take(hh * 8));
  x.RK = static_cast<double *>(take(hh * 8));
  x.N = static_cast<double *>(take(hh * 8));
  x.Ni = static_cast<double *>(take(hh * 8));
  x.NN = static_cast<double *>(take(hh * 8));
  x.Gp1 = static_cast<double *>(take(lh * 8));
  x.Gp2 = static_cast<double *>(take(lh * 8));
  x.Tm = static_cast<double *>(take(lh * 8));
  x.W = static_cast<double *>(take(hh * 8));
  x.Z64 = static_cast<double *>(take((size_t)D.l * D.l * 8));
  x.WtW = static_cast<double *>(take(hh * 8));
  x.Vw64 = static_cast<double *>(take(hh * 8));
  x.ww = static_cast<double *>(take((size_t)D.h * 8));
  x.Vsel = static_cast<double *>(take((size_t)D.h * D.d * 8));
  x.Usel = static_cast<double *>(take((size_t)D.h * D.d * 8));
  x.chs = static_cast<double *>(take((hh + 2 * (size_t)D.h + 8) * 8));
  x.perm = static_cast<int32_t *>(take((size_t)D.h * 4));
  x.eigscr = take(eig_scratch_bytes(D.h));
  if (b) *b = x;
  return off;
}

// out[e, :] = src[idx[e], :] (k columns), coldat[e] = (1, 0, sign_e, 0)
__global__ void gather_rows_kernel(const float *__restrict__ src, int64_t lds, int k,
                                   const int32_t *__restrict__ idx, const int8_t *__restrict__ sgn,
                                   int64_t count, float *__restrict__ out, float4 *__restrict__ cd) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count * k; q += stride) {
    const int64_t e = q / k;
    const int c = (int)(q % k);
    out[q] = src[(int64_t)idx[e] * lds + c];
    if (c == 0) cd[e] = make_float4(1.f, 0.f, (float)sgn[e], 0.f);
  }
}

__global__ void fill_rowdat_kernel(float2 *rowdat, int64_t count, float rho) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < count; q += stride)
    rowdat[q] = make_float2(rho, 0.f);
}

// Vsel[a][j] = V[a][perm[j]] (h x d), sigma[j] = sqrt(max(w[perm[j]], 0))
__global__ void select_right_kernel(const double *__restrict__ V, int h,
                                    const int32_t *__restrict__ perm, const double *__restrict__ w,
                                    int d, double *__restrict__ Vsel, double *__restrict__ sigma) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < h * d; q += gridDim.x * blockDim.x) {
    const int a = q / d, j = q % d;
    const int src = perm[j];
    Vsel[q] = V[(int64_t)a * h + src];
    if (a == 0) sigma[j] = sqrt(fmax(w[src], 0.0));
  }
}

// Uw = Usel Sigma^-1, Vw = Vsel (FP32, h x d); a zero singular value gives a
// zero column
__global__ void finish_uv_kernel(const double *__restrict__ Usel, const double *__restrict__ Vsel,
                                 const double *__restrict__ sigma, int h, int d,
                                 float *__restrict__ Uw, float *__restrict__ Vw) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < h * d; q += gridDim.x * blockDim.x) {
    const int j = q % d;
    const double s = sigma[j];
    Uw[q] = s > 0.0 ? (float)(Usel[q] / s) : 0.f;
    Vw[q] = (float)Vsel[q];
  }
}

inline unsigned grid_for_g(int64_t work) {
  int64_t b = (work + 255) / 256;
  b = std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)sm_count() * 8));
  return (unsigned)b;
}

#define GK(call)                                  \
  do {                                            \
    cudaError_t e__ = (call);                     \
    if (e__ != cudaSuccess) return SNE_ERR_CUDA;  \
  } while (0)

// Q = orth(Yin) (rows x w) by Cholesky QR twice, FP64 pivoted Cholesky on the
// double-float Gram; Rinv = R^-1 of Yin = Q R (FP64, w x w).
int orth64(const GenDims &D, const GenBufs &b, const float *Yin, int64_t rows, int w, float *tmp,
           float *Qout, double *Rinv, cudaStream_t st) {
  const size_t ww = (size_t)w * w;
  double *Gm = b.N;
  GK(launch_gram_accurate(Yin, w, w, Yin, w, w, rows, nullptr, nullptr, true, b.partial, Gm, w, st));
  GK(launch_chol_inverse<double>(Gm, w, w, b.R1, w, b.chs, b.ctrl, st, 1e-13));
  GK(launch_d2f(b.R1, w, w, w, b.m32, w, st));
  GK(launch_tall_gemm_auto(Yin, w, rows, w, b.m32, w, w, tmp, w, b.Mt, b.ctrl, st));
  GK(launch_gram_accurate(tmp, w, w, tmp, w, w, rows, nullptr, nullptr, true, b.partial, Gm, w, st));
  GK(launch_chol_inverse<double>(Gm, w, w, b.R2, w, b.chs, b.ctrl, st, 1e-13));
  GK(launch_d2f(b.R2, w, w, w, b.m32, w, st));
  GK(launch_tall_gemm_auto(tmp, w, rows, w, b.m32, w, w, Qout, w, b.Mt, b.ctrl, st));
  GK(launch_small_gemm<double>(false, false, w, w, w, 1.0, b.R1, w, b.R2, w, 0.0, Rinv, w, st));
  (void)D;
  (void)ww;
  return SNE_OK;
}

// Gp = G^+ (h x l) for G (l x h) via the normal equations: (G^T G)^+ = M M^T
// with M from the pivoted Cholesky (columns past the numerical rank cut).
int pinv64(const GenBufs &b, const double *G, int l, int h, double *Gp, cudaStream_t st) {
  GK(launch_small_gemm<double>(true, false, h, h, l, 1.0, G, h, G, h, 0.0, b.N, h, st));
  GK(launch_chol_inverse<double>(b.N, h, h, b.Ni, h, b.chs, b.ctrl, st, 1e-12));
  GK(launch_small_gemm<double>(false, true, h, h, h, 1.0, b.Ni, h, b.Ni, h, 0.0, b.NN, h, st));
  GK(launch_small_gemm<double>(false, true, h, l, h, 1.0, b.NN, h, G, h, 0.0, Gp, l, st));
  return SNE_OK;
}

}  // namespace

size_t general_workspace_bytes(int64_t n, int64_t m, int32_t k, int32_t d, int32_t h, int32_t l,
                               int32_t zeta) {
  GenDims D{n, m, k, d, h, l, (int)std::min<int64_t>(n, zeta), (int)std::min<int64_t>(m, zeta)};
  return gen_carve(D, nullptr, nullptr);
}

int run_general_svd(int64_t n, int64_t m, int32_t k, const float *L, int64_t ldl, const float *Rt,
                    int64_t ldr, const sne_params &p, void *ws, float *U, int64_t ldu, double *sigma,
                    float *V, int64_t ldv, cudaStream_t st) {
  GenDims D{n, m, k, p.d, p.h, p.l, (int)std::min<int64_t>(n, p.zeta),
            (int)std::min<int64_t>(m, p.zeta)};
  GenBufs b;
  gen_carve(D, ws, &b);
  const int h = D.h, l = D.l, d = D.d;
  const int64_t nC = (int64_t)h * D.zn, nS = (int64_t)h * D.zm;
  const int64_t nH = (int64_t)l * D.zn, nO = (int64_t)l * D.zm;
  GK(cudaMemsetAsync(b.ctrl, 0, sizeof(Ctrl), st));
  // Alg. 3: the four sparse-sign matrices, and the unique rows of H
  GK(launch_sparse_sign(n, h, D.zn, p.seed, 4, b.idxC, b.sgnC, b.ctrl, st));
  GK(launch_sparse_sign(m, h, D.zm, p.seed, 2, b.idxS, b.sgnS, b.ctrl, st));
  GK(launch_sparse_sign(n, l, D.zn, p.seed, 5, b.idxH, b.sgnH, b.ctrl, st));
  GK(launch_sparse_sign(m, l, D.zm, p.seed, 3, b.idxO, b.sgnO, b.ctrl, st));
  GK(launch_unique(b.idxH, (int32_t)nH, b.uniqH, &b.ctrl->v_o, b.posH, b.ctrl, W_UNIQUE, st));
  // the gathered rows of the other factor, one per sparse-sign nonzero
  {
    ProfScope ps_(K_MISC, st, 4);
    gather_rows_kernel<<<grid_for_g(nS * k), 256, 0, st>>>(Rt, ldr, k, b.idxS, b.sgnS, nS, b.BS, b.cdS);
    gather_rows_kernel<<<grid_for_g(nC * k), 256, 0, st>>>(L, ldl, k, b.idxC, b.sgnC, nC, b.BC, b.cdC);
    gather_rows_kernel<<<grid_for_g(nO * k), 256, 0, st>>>(Rt, ldr, k, b.idxO, b.sgnO, nO, b.BO, b.cdO);
    fill_rowdat_kernel<<<grid_for_g(std::max(n, m)), 256, 0, st>>>(
        b.rowdat, std::max(n, m), p.f == SNE_F_TRUNC_LOG ? -1.0f : 0.0f);
  }
  GK(cudaGetLastError());
  // Eq. 5: Y = f(LR) S, K = f(LR)^T C = f(Rt L^T) C, f(LR)(p_H, :) O, Z = H^T (that)
  const float svn = 1.0f / sqrtf((float)D.zn), svm = 1.0f / sqrtf((float)D.zm);
  GK(launch_fused_sketch_f32(L, ldl, nullptr, nullptr, n, k, b.rowdat, b.BS, b.cdS, h, D.zm, svm,
                             p.f, b.Y, h, st));
  GK(launch_fused_sketch_f32(Rt, ldr, nullptr, nullptr, m, k, b.rowdat, b.BC, b.cdC, h, D.zn, svn,
                             p.f, b.K, h, st));
  GK(launch_fused_sketch_f32(L, ldl, b.uniqH, &b.ctrl->v_o, nH, k, b.rowdat, b.BO, b.cdO, l, D.zm,
                             svm, p.f, b.Yh, l, st));
  GK(launch_signed_gather_sum(b.Yh, l, l, b.posH, b.sgnH, l, D.zn, svn, b.Z, l, st));
  // H^T Y and O^T K in FP64, before Y and K are replaced by Q and P
  GK(launch_signed_gather_sum64(b.Y, h, h, b.idxH, b.sgnH, l, D.zn, (double)svn, b.HY, h, st));
  GK(launch_signed_gather_sum64(b.K, h, h, b.idxO, b.sgnO, l, D.zm, (double)svm, b.OK, h, st));
  // Eq. 6
  int rc = orth64(D, b, b.Y, n, h, b.tmp, b.Y, b.RY, st);
  if (rc) return rc;
  rc = orth64(D, b, b.K, m, h, b.tmp, b.K, b.RK, st);
  if (rc) return rc;
  // Eq. 9: H^T Q = (H^T Y) R_Y^-1, O^T P = (O^T K) R_K^-1, W = (H^T Q)^+ Z ((O^T P)^+)^T
  GK(launch_small_gemm<double>(false, false, l, h, h, 1.0, b.HY, h, b.RY, h, 0.0, b.G1, h, st));
  GK(launch_small_gemm<double>(false, false, l, h, h, 1.0, b.OK, h, b.RK, h, 0.0, b.G2, h, st));
  rc = pinv64(b, b.G1, l, h, b.Gp1, st);
  if (rc) return rc;
  rc = pinv64(b, b.G2, l, h, b.Gp2, st);
  if (rc) return rc;
  GK(launch_f2d(b.Z, l, l, l, b.Z64, l, st));
  GK(launch_small_gemm<double>(false, false, h, l, l, 1.0, b.Gp1, l, b.Z64, l, 0.0, b.Tm, l, st));
  GK(launch_small_gemm<double>(false, true, h, h, l, 1.0, b.Tm, l, b.Gp2, l, 0.0, b.W, h, st));
  // Eq. 10: svd(W) from W^T W = V_w Sigma^2 V_w^T, the d largest
  GK(launch_small_gemm<double>(true, false, h, h, h, 1.0, b.W, h, b.W, h, 0.0, b.WtW, h, st));
  GK(launch_symmetrize(b.WtW, h, h, st));
  GK(launch_sym_eig<double>(b.WtW, h, h, b.ww, b.Vw64, h, b.eigscr, b.ctrl, st));
  GK(launch_eig_order<double>(b.ww, h, false, b.perm, st));
  {
    ProfScope ps_(K_MISC, st);
    select_right_kernel<<<grid_for_g((int64_t)h * d), 256, 0, st>>>(b.Vw64, h, b.perm, b.ww, d,
                                                                    b.Vsel, sigma);
  }
  GK(cudaGetLastError());
  GK(launch_small_gemm<double>(false, false, h, d, h, 1.0, b.W, h, b.Vsel, d, 0.0, b.Usel, d, st));
  float *Uw = b.m32, *Vw = b.m32 + (size_t)h * h;
  {
    ProfScope ps_(K_MISC, st);
    finish_uv_kernel<<<grid_for_g((int64_t)h * d), 256, 0, st>>>(b.Usel, b.Vsel, sigma, h, d, Uw, Vw);
  }
  GK(cudaGetLastError());
  if (U) GK(launch_tall_gemm_auto(b.Y, h, n, h, Uw, d, d, U, ldu, b.Mt, b.ctrl, st));
  if (V) GK(launch_tall_gemm_auto(b.K, h, m, h, Vw, d, d, V, ldv, b.Mt, b.ctrl, st));
  return SNE_OK;
}

}  // namespace sne
