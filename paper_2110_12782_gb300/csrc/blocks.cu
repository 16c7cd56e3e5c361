// C entry points for the dense building blocks that Alg. 5 (freigs, with
// eigSVD) and Alg. 4 (orth and the small SVD) are made of: the tall Gram
// matrix, the tall-times-small product and the small symmetric
// eigensolver.  The pipelines in api.cu call the same launchers; these entry
// points expose them one by one so that each can be checked at full size.
#include <algorithm>

#include "sne_internal.cuh"
#include "tc_ptx.cuh"

using namespace sne;

namespace {

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

int check_ws_(void *ws, size_t bytes, size_t need) {
  if (!ws || ((uintptr_t)ws % 256) != 0 || bytes < need) return SNE_ERR_WORKSPACE;
  return SNE_OK;
}

size_t gram_ws(int64_t n, int32_t ka, int32_t kb) {
  const size_t pf = std::max(gram_partial_floats(n, ka, kb), gram_tc_partial_floats(n, ka, kb));
  return align256(sizeof(Ctrl)) + align256(pf * sizeof(float));
}

size_t eig_ws(int32_t n) {
  const size_t nn = (size_t)n * n;
  return align256(sizeof(Ctrl)) + 2 * align256(nn * sizeof(double)) + align256(n * sizeof(double)) +
         align256(n * sizeof(int32_t)) + align256(eig_scratch_bytes(n));
}

__global__ void trunc_log_eval_kernel(const float *__restrict__ r, float *out, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = tc::fr<SNE_F_TRUNC_LOG>(r[i]);
}

// Vout[a][j] = V[a][perm[j]], lam[j] = w[perm[j]]
__global__ void permute_cols_kernel(const double *V, int n, const int32_t *perm, const double *w,
                                    double *Vout, int ldo, double *lam) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < n * n; q += gridDim.x * blockDim.x) {
    const int a = q / n, j = q % n;
    const int src = perm[j];
    Vout[(int64_t)a * ldo + j] = V[(int64_t)a * n + src];
    if (a == 0) lam[j] = w[src];
  }
}

}  // namespace

extern "C" {

int sne_gram_workspace_bytes(int64_t n, int32_t ka, int32_t kb, size_t *bytes) {
  if (!bytes || n <= 0 || ka <= 0 || kb <= 0) return SNE_ERR_ARG;
  *bytes = gram_ws(n, ka, kb);
  return SNE_OK;
}

int sne_gram(int64_t n, int32_t ka, int32_t kb, const float *A, int64_t lda, const float *B,
             int64_t ldb, const float *w, double *C, int32_t ldc, int32_t accurate, void *ws,
             size_t ws_bytes, sne_stream_t stream) {
  if (n <= 0 || ka <= 0 || kb <= 0 || !A || !B || !C || lda < ka || ldb < kb || ldc < kb ||
      (accurate != 0 && accurate != 1))
    return SNE_ERR_ARG;
  const int rc = check_ws_(ws, ws_bytes, gram_ws(n, ka, kb));
  if (rc) return rc;
  Ctrl *ctrl = reinterpret_cast<Ctrl *>(ws);
  if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), (cudaStream_t)stream) != cudaSuccess) return SNE_ERR_CUDA;
  float *partial = reinterpret_cast<float *>(static_cast<char *>(ws) + align256(sizeof(Ctrl)));
  const bool sym = A == B && ka == kb && lda == ldb;
  if (accurate)
    return launch_gram_accurate(A, lda, ka, B, ldb, kb, n, w, nullptr, sym, partial, C, ldc,
                                (cudaStream_t)stream) == cudaSuccess
               ? SNE_OK
               : SNE_ERR_CUDA;
  return launch_gram(A, lda, ka, B, ldb, kb, n, w, sym, partial, C, ldc, (cudaStream_t)stream,
                     ctrl) == cudaSuccess
             ? SNE_OK
             : SNE_ERR_CUDA;
}

int sne_tall_gemm_workspace_bytes(int32_t ka, int32_t kc, size_t *bytes) {
  if (!bytes || ka <= 0 || kc <= 0) return SNE_ERR_ARG;
  *bytes = align256(sizeof(Ctrl)) + align256(tall_tc_scratch_floats(ka, kc) * sizeof(float));
  return SNE_OK;
}

int sne_tall_gemm(int64_t n, int32_t ka, int32_t kc, const float *A, int64_t lda, const float *M,
                  int32_t ldm, float *C, int64_t ldc, void *ws, size_t ws_bytes,
                  sne_stream_t stream) {
  if (n <= 0 || ka <= 0 || kc <= 0 || !A || !M || !C || lda < ka || ldm < kc || ldc < kc)
    return SNE_ERR_ARG;
  const int rc = check_ws_(ws, ws_bytes,
                           align256(sizeof(Ctrl)) +
                               align256(tall_tc_scratch_floats(ka, kc) * sizeof(float)));
  if (rc) return rc;
  Ctrl *ctrl = reinterpret_cast<Ctrl *>(ws);
  if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), (cudaStream_t)stream) != cudaSuccess) return SNE_ERR_CUDA;
  float *Mt = reinterpret_cast<float *>(static_cast<char *>(ws) + align256(sizeof(Ctrl)));
  return launch_tall_gemm_auto(A, lda, n, ka, M, ldm, kc, C, ldc, Mt, ctrl,
                               (cudaStream_t)stream) == cudaSuccess
             ? SNE_OK
             : SNE_ERR_CUDA;
}

int sne_sym_eig_workspace_bytes(int32_t n, size_t *bytes) {
  if (!bytes || n <= 0 || n > 1024) return SNE_ERR_ARG;
  *bytes = eig_ws(n);
  return SNE_OK;
}

int sne_sym_eig(int32_t n, const double *S, int32_t lds, double *lambda, double *V, int32_t ldv,
                void *ws, size_t ws_bytes, sne_stream_t stream) {
  if (n <= 0 || n > 1024 || !S || !lambda || !V || lds < n || ldv < n) return SNE_ERR_ARG;
  const int rc = check_ws_(ws, ws_bytes, eig_ws(n));
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nn = (size_t)n * n;
  char *p = static_cast<char *>(ws);
  Ctrl *ctrl = reinterpret_cast<Ctrl *>(p);
  p += align256(sizeof(Ctrl));
  double *A = reinterpret_cast<double *>(p);
  p += align256(nn * sizeof(double));
  double *Vu = reinterpret_cast<double *>(p);
  p += align256(nn * sizeof(double));
  double *w = reinterpret_cast<double *>(p);
  p += align256(n * sizeof(double));
  int32_t *perm = reinterpret_cast<int32_t *>(p);
  p += align256(n * sizeof(int32_t));
  void *scratch = p;
  if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st) != cudaSuccess) return SNE_ERR_CUDA;
  if (cudaMemcpy2DAsync(A, n * sizeof(double), S, lds * sizeof(double), n * sizeof(double), n,
                        cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return SNE_ERR_CUDA;
  if (launch_sym_eig<double>(A, n, n, w, Vu, n, scratch, ctrl, st) != cudaSuccess) return SNE_ERR_CUDA;
  if (launch_eig_order<double>(w, n, true, perm, st) != cudaSuccess) return SNE_ERR_CUDA;
  const int64_t total = (int64_t)n * n;
  permute_cols_kernel<<<(unsigned)std::min<int64_t>(1024, (total + 255) / 256), 256, 0, st>>>(
      Vu, n, perm, w, V, ldv, lambda);
  return cudaGetLastError() == cudaSuccess ? SNE_OK : SNE_ERR_CUDA;
}

int sne_chol_inverse_workspace_bytes(int32_t n, int32_t fp64, size_t *bytes) {
  if (!bytes || n <= 0 || n > 1024) return SNE_ERR_ARG;
  const size_t el = fp64 ? sizeof(double) : sizeof(float);
  *bytes = align256(sizeof(Ctrl)) + align256(((size_t)n * n + 2 * (size_t)n + 8) * el);
  return SNE_OK;
}

int sne_chol_inverse(int32_t n, const void *A, int32_t lda, void *M, int32_t ldm, int32_t fp64,
                     double tol, void *ws, size_t ws_bytes, sne_stream_t stream) {
  if (n <= 0 || n > 1024 || !A || !M || lda < n || ldm < n) return SNE_ERR_ARG;
  size_t need = 0;
  int rc = sne_chol_inverse_workspace_bytes(n, fp64, &need);
  if (rc) return rc;
  rc = check_ws_(ws, ws_bytes, need);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  Ctrl *ctrl = reinterpret_cast<Ctrl *>(ws);
  if (cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st) != cudaSuccess) return SNE_ERR_CUDA;
  void *scratch = static_cast<char *>(ws) + align256(sizeof(Ctrl));
  cudaError_t e =
      fp64 ? launch_chol_inverse<double>(static_cast<const double *>(A), n, lda,
                                         static_cast<double *>(M), ldm,
                                         static_cast<double *>(scratch), ctrl, st, tol)
           : launch_chol_inverse<float>(static_cast<const float *>(A), n, lda,
                                        static_cast<float *>(M), ldm,
                                        static_cast<float *>(scratch), ctrl, st, tol);
  return e == cudaSuccess ? SNE_OK : SNE_ERR_CUDA;
}

int sne_trunc_log_eval(int64_t n, const float *r, float *out, sne_stream_t stream) {
  if (n < 0 || (n > 0 && (!r || !out))) return SNE_ERR_ARG;
  if (n == 0) return SNE_OK;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 8);
  trunc_log_eval_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(r, out, n);
  return cudaGetLastError() == cudaSuccess ? SNE_OK : SNE_ERR_CUDA;
}

}  // extern "C"
