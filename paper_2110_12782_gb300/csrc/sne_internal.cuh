// Internal declarations shared by the translation units of libsketchne.so.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sketchne.h"

namespace sne {

__host__ __device__ __forceinline__ int64_t min64(int64_t a, int64_t b) { return a < b ? a : b; }
__host__ __device__ __forceinline__ int64_t max64(int64_t a, int64_t b) { return a > b ? a : b; }

// ---------------------------------------------------------------------------
// Device control block: first 256 bytes of every workspace.
// ---------------------------------------------------------------------------
struct Ctrl {
  int32_t status;  // first error code recorded on the device (0 = none)
  int32_t where;   // id of the kernel that recorded it
  int32_t v_s;     // unique rows of S (Alg. 4 line 3)
  int32_t v_o;     // unique rows of O (Alg. 4 line 6)
  double vol;      // vol(G)
  uint32_t hot_bits;  // SpMM L2 split: weights whose bits are below it mark kept rows
  int32_t pad[57];
};
static_assert(sizeof(Ctrl) == 256, "control block is 256 bytes");

enum Where : int32_t {
  W_NONE = 0,
  W_VALIDATE = 1,
  W_CHOL = 2,
  W_EIG = 3,
  W_TRIINV = 4,
  W_EIGSVD = 5,
  W_NAN = 6,
  W_SPARSE_SIGN = 7,
  W_UNIQUE = 8,
  W_TC = 9,
};

// Number of SMs of the current device (queried once per device and cached);
// grids are sized in multiples of it.
int sm_count();

__device__ __forceinline__ void record_error(Ctrl *c, int32_t code, int32_t where) {
  if (c == nullptr) return;
  if (atomicCAS(&c->status, 0, code) == 0) c->where = where;
}

// ---------------------------------------------------------------------------
// Launch accounting / profiling (prof.cu).  A ProfScope covers the `nk`
// kernels one launcher enqueues on `st`.
// ---------------------------------------------------------------------------
enum KClass : int {
  K_SPMM = 0, K_GRAM, K_TALL_GEMM, K_SMALL_GEMM, K_EIG, K_CHOL, K_TRIINV, K_FUSED, K_GATHER, K_RNG,
  K_UNIQUE, K_MISC, K_FUSED_TC, K_GRAM_TC, K_TALL_TC, K_PROP, K_COUNT
};
class ProfScope {
 public:
  ProfScope(int cls, cudaStream_t st, int nk = 1);
  ~ProfScope();
  ProfScope(const ProfScope &) = delete;
  ProfScope &operator=(const ProfScope &) = delete;

 private:
  int cls_, nk_;
  cudaStream_t st_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
};

// ---------------------------------------------------------------------------
// Counter-based random numbers: SplitMix64 (Steele, Lea, Flood 2014) read as a
// counter-based generator.  Output i (1-based) of SplitMix64 started at state s
// is mix64(s + i * GOLDEN).  stream_key(seed, stream) is output stream+1 of
// SplitMix64(seed); draw(key, ctr) is output ctr+1 of SplitMix64(key).
// ---------------------------------------------------------------------------
constexpr uint64_t kGolden = 0x9E3779B97F4A7C15ull;

__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
__host__ __device__ __forceinline__ uint64_t stream_key(uint64_t seed, uint32_t stream) {
  return mix64(seed + kGolden * (uint64_t)(stream + 1));
}
__host__ __device__ __forceinline__ uint64_t draw(uint64_t key, uint64_t ctr) {
  return mix64(key + kGolden * (ctr + 1));
}

// ---------------------------------------------------------------------------
// Launchers (host functions; every one enqueues on `st` and returns a
// cudaError_t from cudaGetLastError()).
// ---------------------------------------------------------------------------
// rng.cu
cudaError_t launch_gaussian(int64_t n, int32_t cols, uint64_t seed, int32_t stream_id, float *out,
                            int64_t ld, cudaStream_t st);
cudaError_t launch_sparse_sign(int64_t n, int32_t cols, int32_t z, uint64_t seed, int32_t stream_id,
                               int32_t *idx, int8_t *sign, Ctrl *ctrl, cudaStream_t st);
// Sorts `count` row indices, writes the unique ones to uniq (ascending), their
// number to *nuniq (device), and for every input its position in uniq to pos.
constexpr int kUniqueMax = 32768;
cudaError_t launch_unique(const int32_t *keys, int32_t count, int32_t *uniq, int32_t *nuniq,
                          int32_t *pos, Ctrl *ctrl, int32_t where, cudaStream_t st);

// graph.cu
cudaError_t launch_degrees(const sne_csr &g, float *deg, double *vol, cudaStream_t st);
cudaError_t launch_degree_power(const float *deg, int64_t n, double beta, float *out, float scale,
                                cudaStream_t st);
// wnz: per-nonzero weights dpow[col_p] * val_p (launch_spmm_weights), or NULL
// to form them on the fly.
cudaError_t launch_spmm_weights(const sne_csr &g, const float *dpow, float *wnz, cudaStream_t st);
// Picks the rows of the dense SpMM operand that stay in L2: the vertices of
// largest degree (smallest d^-a), as many as fill kSpmmKeepBytes at
// `row_bytes` a row; writes the bit pattern bound to ctrl->hot_bits.
cudaError_t launch_spmm_hot_threshold(const float *dpow, int64_t n, int64_t row_bytes, Ctrl *ctrl,
                                      cudaStream_t st);
// Column panels launch_spmm uses for an n x ncols operand, and the bytes of the
// row segment one panel gathers (the row size for the keep bound).
int spmm_panels(int64_t n, int32_t ncols);
int64_t spmm_row_bytes(int64_t n, int32_t ncols);
// hot: that bound (a gathered row whose weight bits are below it is loaded with
// the normal L2 priority, every other row and the CSR streams evict-first), or
// NULL to load every row with the normal priority.
cudaError_t launch_spmm(const sne_csr &g, const float *dpow, const float *wnz, const float *B,
                        int64_t ldb, int32_t ncols, float *Y, int64_t ldy, cudaStream_t st,
                        const uint32_t *hot = nullptr);
cudaError_t launch_validate(const sne_csr &g, Ctrl *ctrl, cudaStream_t st);

// dense.cu
// C (Ka x Kb, FP64, ldc) = sum_i w_i A[i, :]^T B[i, :]  over i < n; w may be NULL.
// `partial` is FP32 scratch of gram_partial_floats(n, Ka, Kb) floats.
size_t gram_partial_floats(int64_t n, int32_t Ka, int32_t Kb);
cudaError_t launch_gram(const float *A, int64_t lda, int32_t Ka, const float *B, int64_t ldb,
                        int32_t Kb, int64_t n, const float *w, bool symmetric, float *partial,
                        double *C, int32_t ldc, cudaStream_t st, Ctrl *ctrl = nullptr);
// The same Gram summed in double-float on the FP32 pipes (FP32 sums of 16
// products added into hi/lo pairs, relative error ~1e-8), or with `exact`
// every product split exactly and added into the pair by TwoSum (FP64
// accuracy, about 1e-9 absolute at n = 10^6 for sums of size 1), for sums
// whose errors later steps amplify; same scratch.  The weight may be given as
// an FP32 pair w + w_lo (w_lo NULL: w exact).
cudaError_t launch_gram_accurate(const float *A, int64_t lda, int32_t Ka, const float *B,
                                 int64_t ldb, int32_t Kb, int64_t n, const float *w,
                                 const float *w_lo, bool symmetric, float *partial, double *C,
                                 int32_t ldc, cudaStream_t st, bool exact = false);
// gemm_tc.cu: FP32-accurate (3 x TF32) tensor-core versions, used when
// tc_gemm_supported(columns) and the operands are 16-byte aligned.
bool tc_gemm_supported(int ncols);
bool tc_gemm_enabled();
size_t gram_tc_partial_floats(int64_t n, int Ka, int Kb);
cudaError_t launch_gram_tc(const float *A, int64_t lda, int Ka, const float *B, int64_t ldb, int Kb,
                           int64_t n, const float *w, bool symmetric, float *partial, double *C,
                           int ldc, Ctrl *ctrl, cudaStream_t st);
// C = sum over chunks of partial[c] (FP64); with sym_tile > 0 the entries
// (a, b) with a / sym_tile > b / sym_tile are read from (b, a).
cudaError_t launch_gram_reduce(const float *partial, int Ka, int Kb, int chunks, int sym_tile,
                               double *C, int ldc, cudaStream_t st);
// C = A M with M (K x Kc, leading dimension ldm); Mt2: scratch of
// tall_tc_scratch_floats(K, Kc) floats (M^T split into TF32 hi and lo rows).
size_t tall_tc_scratch_floats(int K, int Kc);
cudaError_t launch_tall_gemm_tc(const float *A, int64_t lda, int64_t n, int K, const float *M,
                                int ldm, int Kc, float *C, int64_t ldc, float *Mt2, Ctrl *ctrl,
                                cudaStream_t st);
// C = A M through the tensor-core path when possible (Mt: scratch of
// tall_tc_scratch_floats(Ka, Kc) floats for the split M^T), else the SIMT
// tall_gemm.
cudaError_t launch_tall_gemm_auto(const float *A, int64_t lda, int64_t n, int32_t Ka, const float *M,
                                  int32_t ldm, int32_t Kc, float *C, int64_t ldc, float *Mt,
                                  Ctrl *ctrl, cudaStream_t st);
// C[i, :] = rs_i * sum_a A[r(i), a] M[a, :]   (r(i) = ridx[i] or i; rs = 1 if NULL)
cudaError_t launch_tall_gemm(const float *A, int64_t lda, const int32_t *ridx, int64_t n, int32_t Ka,
                             const float *M, int32_t ldm, int32_t Kc, const float *rs, float *C,
                             int64_t ldc, cudaStream_t st);
// Small dense GEMM (multi-CTA): C = alpha * op(A) op(B) + beta * C, row-major.
// With `skip` (device flag) set the kernel returns without touching C.
template <typename T>
cudaError_t launch_small_gemm(bool ta, bool tb, int32_t M, int32_t N, int32_t K, T alpha,
                              const T *A, int32_t lda, const T *B, int32_t ldb, T beta, T *C,
                              int32_t ldc, cudaStream_t st, const int *skip = nullptr);
// Symmetric eigendecomposition: A (n x n) = V diag(w) V^T, w unordered.
// V is returned row-major n x n (column j = eigenvector j), ldv = n.  A may be
// overwritten.  scratch: eig_scratch_bytes(n) bytes, 256-byte aligned.
size_t eig_scratch_bytes(int n);
template <typename T>
cudaError_t launch_sym_eig(T *A, int32_t n, int32_t lda, T *w, T *V, int32_t ldv, void *scratch,
                           Ctrl *ctrl, cudaStream_t st);
cudaError_t launch_sym_eig_fast(float *A, int32_t n, int32_t lda, float *w, float *V, int32_t ldv,
                                void *scratch, Ctrl *ctrl, cudaStream_t st);
cudaError_t launch_sym_eig_fast(double *A, int32_t n, int32_t lda, double *w, double *V,
                                int32_t ldv, void *scratch, Ctrl *ctrl, cudaStream_t st);
constexpr int kFastEigMaxN = 320;
// tridiag.cu: FP32 symmetric eigendecomposition (Householder tridiagonalization,
// bisection, inverse iteration); w unordered, column j of V the eigenvector of
// w[j]; scratch: tri_eig_scratch_floats(n) floats.
size_t tri_eig_scratch_floats(int n);
size_t tri_eig_smem(int n);  // shared memory of the tridiagonalization
cudaError_t launch_sym_eig_tridiag(const float *A, int32_t n, int32_t lda, float *w, float *V,
                                   int32_t ldv, float *scratch, Ctrl *ctrl, cudaStream_t st);

// M = R^-1 where A = R^T R (Cholesky); scratch: n*n + 2n + 8 T (used only for
// n too large for shared memory).  tol >= 0 selects diagonal pivoting with a rank
// cut at tol * max(diag A): then M = P [R11^-1 0; 0 0] (zero columns past the
// numerical rank) and no pivot is ever non-positive.
template <typename T>
cudaError_t launch_chol_inverse(const T *A, int32_t n, int32_t lda, T *Rinv, int32_t ldi, T *scratch,
                                Ctrl *ctrl, cudaStream_t st, double tol = -1.0);
// Orders eigenpairs: perm[j] = index of the j-th largest (|w| if by_abs else w).
template <typename T>
cudaError_t launch_eig_order(const T *w, int32_t n, bool by_abs, int32_t *perm, cudaStream_t st);
// Elementwise helpers.
cudaError_t launch_d2f(const double *src, int32_t rows, int32_t cols, int32_t lds, float *dst,
                       int32_t ldd, cudaStream_t st);
cudaError_t launch_f2d(const float *src, int32_t rows, int32_t cols, int32_t lds, double *dst,
                       int32_t ldd, cudaStream_t st);
cudaError_t launch_symmetrize(double *A, int32_t n, int32_t lda, cudaStream_t st);
cudaError_t launch_check_finite_f(const float *x, int64_t count, Ctrl *ctrl, int32_t where,
                                  cudaStream_t st);

// center.cu: centred evaluation of L'R' (x - c0 = s (W_i - w) C (W_j - w)^T +
// rho_i + kappa_j with W = D^(-1+a) U and w the degree-weighted mean row).
// stats (FP64, 3k + 2): w | p = C w^T | q = w C | gamma = s w C w^T - c0 | s.
size_t center_partial_doubles(int64_t n, int k);
cudaError_t launch_center_stats(const float *U, int64_t ldu, int k, int64_t n, const float *deg,
                                double alpha, const double *vol_dev, const double *lam,
                                const double *Csum, double smult, double c0, double *partial,
                                double *stats, float *ws_hi, float *ws_lo, cudaStream_t st);
// Rows r < nrows_max (source row ridx[r] or r) of L~ = s (W - w): out = 0 FP32
// (Lt, ld ldl); out = 1 FP16, 2 BF16 rows of L~ / rowf (rowf a power of two)
// into Ahi (and Alo, the rounding error of Ahi, when split), kpad columns.
// rowdat[r] = (rho_r, mask_r).  rsc + rsc_lo = s d^(-1+a) (0 for isolated
// vertices), ws_hi + ws_lo = s w.
cudaError_t launch_center_rows(int out, bool split, const float *U, int64_t ldu, int k,
                               const int32_t *ridx, const int32_t *nrows_dev, int64_t nrows_max,
                               const float *rsc, const float *rsc_lo, const float *ws_hi,
                               const float *ws_lo, const double *stats, bool trunc_log, double c0,
                               float *Lt, int64_t ldl, void *Ahi, void *Alo, int kpad, float *rowf,
                               float2 *rowdat, cudaStream_t st);
// FP32 rows -> FP16/BF16 rows / sc (sc a power of two, written to
// scale[r * sstride]) as hi (+ lo) with kpad columns.
cudaError_t launch_split_rows(bool fp16, bool split, const float *src, int64_t lds, int64_t rows,
                              int k, int kpad, void *hi, void *lo, float *scale, int sstride,
                              cudaStream_t st);

// sketch.cu
// out[i, c] = sv * sum_{t<z} sgn_e f(<A[r(i), :], B[e, :]> + rho_r(i) + mask_r(i) kappa_e),
// e = c*z + t, rowdat[r] = (rho, mask), coldat[e] = (scale, kappa, sgn, 0).
cudaError_t launch_fused_sketch_f32(const float *A, int64_t lda, const int32_t *ridx,
                                    const int32_t *nrows_dev, int64_t nrows, int32_t k,
                                    const float2 *rowdat, const float *B, const float4 *coldat,
                                    int32_t cols_out, int32_t z, float sv, int32_t f, float *out,
                                    int64_t ldo, cudaStream_t st);
// Centred columns of R' for j = idx[e]: out[e, :] = (W_j - w) C^T (C^T as
// the FP32 pair CThi + CTlo), coldat[e] = (1, kappa_e, sgn_e, 0).
cudaError_t launch_rtilde_rows(const float *U, int32_t k, const int32_t *idx, int32_t count,
                               const float *CThi, const float *CTlo, const float *deg, double beta,
                               const double *stats, const int8_t *sign, float *out, float4 *coldat,
                               cudaStream_t st);
// sketch_tc.cu: the same sums with half-precision operands (BF16 or FP16,
// optionally hi/lo pairs) on tcgen05 with FP32 accumulation; A rows scaled by
// rowf, B rows by coldat[e].x; kpad = k rounded up to 64.  One persistent
// launch runs any number of such sketches (jobs).  Every operand lies in the
// arena [arena, arena + arena_bytes) at a byte offset that is a multiple of
// 2 kpad (one row), B zero padded to a multiple of 256 rows; coldat readable
// (zero padded) up to a multiple of 256 entries.
struct TcSketchJobDesc {
  const void *Ahi, *Alo, *Bhi, *Blo;  // Alo, Blo: split precisions only
  int64_t nrows_max;                  // rows of A
  const int32_t *nrows_dev;           // if set: the rows used (device count)
  int32_t ncols_eval, cols_out;
  const float *rowf;
  const float2 *rowdat;
  const float4 *coldat;
  float *out;
  int64_t ldo;
  Ctrl *ctrl;                         // status word (timeouts); null: the launch's
};
// Launch shape of the fused tensor-core sketch: column tile width (128 or
// 256), B stages (0: as many as fit), and the column split of jobs with few
// row tiles (items per SM to aim for).  None of them changes a result.
struct TcTune {
  int tn = 256;
  int stages = 0;
  int split_mult = 2;
};
int tc_max_stages(int kpad, bool split, int tn);
// The launch shape for a sketch of this kind: the autotuner's choice for the
// key (kpad, split, fp16, z, log2 of the rows) if it has tuned one, else the
// default; SNE_TC_TN, SNE_TC_STAGES and SNE_TC_SPLIT override it (for
// comparisons).
TcTune tc_tune_lookup(int kpad, bool split, bool fp16, int z, int64_t rows);
// api.cu: the shape of a graph's tensor-core sketch (false for the FP32 path),
// the operand row bytes for the parameters, and an embedding in two halves
// around that sketch (phase 1: up to the sketch, its two jobs returned instead
// of launched; phase 2: from the sketch results on; the same workspace).
struct TcShape {
  int kpad, z, f;
  bool fp16, split;
};
bool embed_tc_shape(const sne_csr *g, const sne_params *p, TcShape *out);
size_t tc_row_bytes(const sne_params *p);
int embed_phase(const sne_csr *g, const sne_params *p, void *ws, size_t ws_bytes, float *E,
                double *sigma, int phase, TcSketchJobDesc *jobs, cudaStream_t st);
void tc_tune_store(int kpad, bool split, bool fp16, int z, int64_t rows, const TcTune &t);
cudaError_t launch_fused_sketch_tc_jobs(bool fp16, bool split, const void *arena,
                                        size_t arena_bytes, int kpad, int z, float sv, int f,
                                        const TcSketchJobDesc *jobs, int njobs, const TcTune &tune,
                                        Ctrl *ctrl, cudaStream_t st);
// The same sum of FP32 rows accumulated and written in FP64.
cudaError_t launch_signed_gather_sum64(const float *In, int64_t ldi, int32_t width,
                                       const int32_t *idx, const int8_t *sign, int32_t cols,
                                       int32_t z, double sv, double *out, int64_t ldo,
                                       cudaStream_t st);
// out[c, :] = sv * sum_t sign[c*z+t] * In[idx[c*z+t], :]
cudaError_t launch_signed_gather_sum(const float *In, int64_t ldi, int32_t width, const int32_t *idx,
                                     const int8_t *sign, int32_t cols, int32_t z, float sv,
                                     float *out, int64_t ldo, cudaStream_t st);

// Spectral propagation (propagate.cu): c_0 .. c_steps of the filter's
// Chebyshev series, the workspace of run_propagate, and the run itself (E in
// place, n x d with leading dimension lde).
double bessel_i(int r, double theta);
void propagation_coefficients(int steps, double theta, double *c);
size_t propagate_workspace_bytes(int64_t n, int32_t d);
int run_propagate(const sne_csr &g, int steps, double theta, double mu, float *E, int64_t lde, int d,
                  void *ws, cudaStream_t st);

// The general single-pass SVD of Eqs. 5-10 (general.cu): workspace bytes and
// the run (L n x k, Rt = R^T m x k, outputs U n x d, sigma d (FP64), V m x d;
// U or V may be NULL).
size_t general_workspace_bytes(int64_t n, int64_t m, int32_t k, int32_t d, int32_t h, int32_t l,
                               int32_t zeta);
int run_general_svd(int64_t n, int64_t m, int32_t k, const float *L, int64_t ldl, const float *Rt,
                    int64_t ldr, const sne_params &p, void *ws, float *U, int64_t ldu, double *sigma,
                    float *V, int64_t ldv, cudaStream_t st);

}  // namespace sne
