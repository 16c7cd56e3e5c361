/*
 * sketchne.h -- C ABI of libsketchne.so, the GB300 (sm_103a) hot path of
 * SketchNE ("SketchNE: Embedding Billion-Scale Networks Accurately in One
 * Hour", arXiv 2110.12782): the fast randomized eigendecomposition of the
 * modified Laplacian D^-a A D^-a (Alg. 5), the factors L', R' of Eq. 11, and
 * the sparse-sign randomized single-pass SVD of trunc_log(L'R') (Alg. 3, 4),
 * giving the initial embedding E = U_d Sigma_d^(1/2) (Alg. 6 lines 1-5).
 *
 * Conventions for every entry point below:
 *  - All array arguments are DEVICE pointers (memory of the current CUDA
 *    device) unless the comment says "host".  The caller allocates and owns
 *    every input, output and workspace; the library never allocates, frees or
 *    keeps a pointer after the call returns.
 *  - Dense matrices are row-major FP32 or FP64 with the leading dimension equal
 *    to the column count stated for the argument.
 *  - Every call is stream-ordered and asynchronous on `stream` (NULL = legacy
 *    default stream); the host returns as soon as the work is enqueued.
 *    Argument errors found on the host are returned immediately and enqueue
 *    nothing.  Errors found on the device (NaN, a non-positive pivot, a bad
 *    graph) are recorded in the workspace's status word and are read with
 *    sne_status(), which synchronizes the stream.
 *  - Return value: SNE_OK (0) or a negative SNE_ERR_* code.
 *  - Calls that share a workspace must not overlap on the GPU.
 */
#ifndef SKETCHNE_H
#define SKETCHNE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *sne_stream_t; /* the same type as cudaStream_t */

enum {
  SNE_OK = 0,
  SNE_ERR_ARG = -1,       /* bad argument (NULL pointer, negative size, ...) */
  SNE_ERR_GRAPH = -2,     /* CSR not valid (row_ptr not monotone, index out of range, asymmetric),
                             or no edges for an embedding (vol(G) = 0, Eq. 1 undefined) */
  SNE_ERR_SIZE = -3,      /* inconsistent sizes: k+s > n, d > h, h > l, z > 64, ... */
  SNE_ERR_WORKSPACE = -4, /* workspace NULL, too small or not 256-byte aligned */
  SNE_ERR_CUDA = -5,      /* a CUDA launch or runtime call failed */
  SNE_ERR_TIMEOUT = -6,   /* a bounded device-side wait ran out */
  SNE_ERR_NUMERIC = -7    /* NaN/Inf or a non-positive pivot in a small solve */
};

/* Precision of the L'R' reconstruction GEMM of Eq. 4 and the Z core: FP32
 * (FP32 FMA), or half-precision operands on the tensor cores with FP32
 * accumulation: BF16 / FP16 (one product), or BF16X2 / FP16X2 (each operand a
 * pair hi + lo of that type, lo the rounding error of hi; three products
 * hi*hi + lo*hi + hi*lo, about twice the operand precision). */
enum { SNE_FP32 = 0, SNE_BF16 = 1, SNE_FP16 = 2, SNE_BF16X2 = 3, SNE_FP16X2 = 4 };
enum { SNE_F_TRUNC_LOG = 0, SNE_F_IDENTITY = 1 };          /* elementwise f of Problem 1 */
enum { SNE_ORTH_EIGSVD = 0, SNE_ORTH_CHOLQR = 1 };         /* orthonormalization inside Alg. 5 */

/* Undirected graph G = (V, E, A) in CSR (Sec. 2): both directions of every
 * edge stored, no self-loops.  row_ptr int64 [n+1] (row_ptr[0] = 0,
 * nondecreasing, row_ptr[n] = nnz), col_idx int32 [nnz] in [0, n),
 * val FP32 [nnz] positive edge weights or NULL for an unweighted graph. */
typedef struct sne_csr {
  int64_t n;
  int64_t nnz;
  const int64_t *row_ptr;
  const int32_t *col_idx;
  const float *val;
} sne_csr;

/* Parameters (Table 2 and Alg. 4-6).
 *  k      eigen rank (Alg. 5/6)                    q      power-iteration count (Alg. 5)
 *  T      context window size (Eq. 1)              d      embedding dimension
 *  h      sketch size of Y  (h = d + s1, Alg. 4)   l      sketch size of Z (l = d + s2, Alg. 4)
 *  zeta   sparse-sign column density z (Alg. 3); the library uses z = min(n, zeta) <= 64
 *  s_eig  oversampling of Alg. 5 (k + s_eig columns of Omega)
 *  row_block  rows of L' per batch of Eq. 4 in the paper; the fused kernels never
 *             store a block of M-hat and work in 128-row tiles whatever it is
 *  precision  SNE_FP32 | SNE_BF16 | SNE_FP16 | SNE_BF16X2 | SNE_FP16X2 (L'R' reconstruction)
 *  f      SNE_F_TRUNC_LOG (NetMF) or SNE_F_IDENTITY (Problem 1 with f = id)
 *  orth   SNE_ORTH_EIGSVD (Alg. 5 as printed) or SNE_ORTH_CHOLQR
 *  alpha  exponent of the modified Laplacian D^-alpha A D^-alpha, in (0, 1] (paper: 0.5, 0.4)
 *  b      number of negative samples (Eq. 1)       seed   seed of all random draws */
typedef struct sne_params {
  int32_t k, q, T, d, h, l, zeta, s_eig, row_block, precision, f, orth;
  double alpha, b;
  uint64_t seed;
} sne_params;

/* Counters filled by sne_stats_read() (host struct). */
typedef struct sne_stats {
  int32_t status;   /* device status word (SNE_OK or SNE_ERR_*) */
  int32_t where;    /* id of the kernel that set the status (0 = none) */
  int64_t v_s;      /* v of Alg. 4 line 3: unique rows of S */
  int64_t v_o;      /* v of Alg. 4 line 6: unique rows of O */
  double vol;       /* vol(G) */
} sne_stats;

/* Fills *p with the defaults: alpha = 0.5, q = 20, T = 10, b = 1, zeta = 8,
 * s_eig = 16, h = 2d + 16, l = d + 1000 (s2 = 1000, Sec. 5.2), FP32, trunc_log,
 * eigSVD, seed 0, and the given d and k. */
int sne_params_init(sne_params *p, int32_t d, int32_t k);

/* Static message for an SNE_* code (host). */
const char *sne_error_string(int code);

/* Workspace modes. */
enum { SNE_WS_EMBED = 0, SNE_WS_FREIGS = 1, SNE_WS_SKETCH = 2, SNE_WS_EMBED_HOST = 3 };

/* Bytes of device workspace needed by sne_embed (mode SNE_WS_EMBED),
 * sne_freigs (SNE_WS_FREIGS) or sne_sketch_from_factors (SNE_WS_SKETCH) for a
 * graph with n vertices and nnz stored entries.  Host-only. */
int sne_workspace_bytes(int64_t n, int64_t nnz, const sne_params *p, int mode, size_t *bytes);

/* Alg. 6 lines 1-5.  E: n x d FP32 (row i = embedding of vertex i), sigma: d
 * FP64 singular values Sigma_d (descending).  Workspace from
 * sne_workspace_bytes(..., SNE_WS_EMBED). */
int sne_embed(const sne_csr *g, const sne_params *p, void *workspace, size_t ws_bytes,
              float *E, double *sigma, sne_stream_t stream);

/* sne_embed with the graph and the outputs in HOST memory.  g's row_ptr,
 * col_idx and val point to host arrays (page-locked for the copies to be
 * asynchronous); E_host (n x d FP32) and sigma_host (d FP64) are host arrays.
 * The call copies the graph into the workspace, runs Alg. 6 lines 1-5 and
 * copies E and sigma back, all on `stream`; the outputs are valid after the
 * stream is synchronized.  Workspace: sne_workspace_bytes(..., SNE_WS_EMBED_HOST). */
int sne_embed_host(const sne_csr *g_host, const sne_params *p, void *workspace, size_t ws_bytes,
                   float *E_host, double *sigma_host, sne_stream_t stream);

/* Alg. 6 lines 1-5 for a batch of G independent graphs (many graphs of uneven
 * sizes, one call).  graphs: HOST array of G sne_csr (each with device arrays);
 * E, sigma: HOST arrays of G device pointers (E[i]: n_i x d FP32, sigma[i]: d
 * FP64); status: DEVICE int32 [G] receiving each graph's status word, or NULL.
 * The paper embeds one graph per call; this entry point has no counterpart
 * there.  The graphs run concurrently on `lanes` streams forked from `stream`
 * (0 = the library's choice, at most 16): largest first, each on the lane
 * with the least estimated work, and the caller's stream waits for all of
 * them, so the outputs are complete when `stream` reaches the end of the call.
 * Each graph's results equal those of sne_embed on that graph.  With a
 * half-precision reconstruction (SNE_BF16 .. SNE_FP16X2) the batch runs in
 * lockstep: the first halves of all embeddings (up to the sketch operands) on
 * the lanes, ONE persistent tensor-core launch for the sketches Y and Z of
 * all graphs (one per distinct z = min(n, zeta)), then the second halves on
 * the lanes.  lanes = 0 takes the count sne_autotune_sketch chose for a batch
 * of this kind, else 8.  The lanes are created on the first call on a device
 * (make it before any stream capture); after that the call enqueues work
 * only, and a batch can be captured into a CUDA graph.  Workspace:
 * sne_embed_batched_workspace_bytes (same G, graphs, p and lanes): with FP32
 * reconstruction every lane owns a slice sized for its largest graph; in
 * lockstep every graph owns one (the sum of the graphs' sne_embed
 * workspaces, each rounded up to an operand row).  Errors: those of
 * sne_embed, checked for every graph before anything is enqueued. */
int sne_embed_batched_workspace_bytes(int32_t G, const sne_csr *graphs, const sne_params *p,
                                      int32_t lanes, size_t *bytes);
int sne_embed_batched(int32_t G, const sne_csr *graphs, const sne_params *p, int32_t lanes,
                      void *workspace, size_t ws_bytes, float *const *E, double *const *sigma,
                      int32_t *status, sne_stream_t stream);

/* Alg. 5 on X = D^-alpha A D^-alpha: U: n x k FP32 (orthonormal columns),
 * lambda: k FP64, ordered by |lambda| descending. */
int sne_freigs(const sne_csr *g, const sne_params *p, void *workspace, size_t ws_bytes,
               float *U, double *lambda, sne_stream_t stream);

/* Alg. 6 lines 2-5 from given eigenpairs (U: n x k FP32, lambda: k FP64, on the
 * device): Eq. 11 factors, Alg. 4 sketches and the embedding.  Outputs (each
 * may be NULL): Y n x h FP32 (Alg. 4 line 4), Z l x l FP32 (line 7), E n x d
 * FP32, sigma d FP64. */
int sne_sketch_from_factors(const sne_csr *g, const sne_params *p, const float *U,
                            const double *lambda, void *workspace, size_t ws_bytes, float *Y,
                            float *Z, float *E, double *sigma, sne_stream_t stream);

/* Alg. 3: sparse-sign matrix with `cols` columns over n rows, z = min(n, zeta)
 * nonzeros per column.  idx: cols x z int32 rows (distinct within a column),
 * sign: cols x z int8 (+1/-1); the value of an entry is sign / sqrt(z).  Bit
 * for bit the SplitMix64 / Lemire draws of stream `stream_id` (2 = S, 3 = O). */
int sne_sparse_sign(int64_t n, int32_t cols, int32_t zeta, uint64_t seed, int32_t stream_id,
                    int32_t *idx, int8_t *sign, sne_stream_t stream);

/* Omega = randn(n, cols) of Alg. 5 line 3 (Box-Muller on SplitMix64 draws of
 * stream `stream_id`, 1 for Omega).  out: n x cols FP32. */
int sne_gaussian(int64_t n, int32_t cols, uint64_t seed, int32_t stream_id, float *out,
                 sne_stream_t stream);

/* d_i = sum_j A_ij (FP32 [n]) and vol(G) = sum_i d_i (FP64 [1]) (Sec. 2). */
int sne_degrees(const sne_csr *g, float *deg, double *vol, sne_stream_t stream);

/* out_i = deg_i^beta, 0 where deg_i = 0 (FP32 [n]). */
int sne_degree_power(const float *deg, int64_t n, double beta, float *out, sne_stream_t stream);

/* Per-nonzero weights of X = D^-a A D^-a for sne_spmm: w_nz[p] = dpow[col_p]
 * * val_p (val_p = 1 for an unweighted graph); w_nz: nnz FP32. */
int sne_spmm_weights(const sne_csr *g, const float *dpow, float *w_nz, sne_stream_t stream);

/* One SpMM of Alg. 5: Y = D^-a A D^-a B, given dpow_i = d_i^-a and optionally
 * the per-nonzero weights of sne_spmm_weights (NULL: formed on the fly, one
 * more dependent load per nonzero).  B, Y: n x ncols FP32 row-major, distinct
 * buffers.  The CSR arrays and Y pass through L2 evict-first and the rows of B
 * at the normal priority (inside sne_embed and sne_freigs only the rows of the
 * vertices of largest degree keep the normal priority, as many as fill 80 MB);
 * the priorities never change a result. */
int sne_spmm(const sne_csr *g, const float *dpow, const float *w_nz, const float *B, int32_t ncols,
             float *Y, sne_stream_t stream);

/* The general randomized single-pass SVD of Eqs. 5-10 (Sec. 4.1) for a
 * rectangular f(L R), not necessarily symmetric: L n x k and Rt = R^T m x k
 * (device, FP32, row-major, leading dimensions ldl, ldr >= k, caller-owned),
 * f = p->f (trunc_log or the identity).  With sparse-sign C (n x h),
 * S (m x h), H (n x l), O (m x l) drawn by Alg. 3 from p->seed (streams 4, 2,
 * 5, 3): K = f(LR)^T C, Y = f(LR) S, Z = H^T f(LR) O (Eq. 5); P = orth(K),
 * Q = orth(Y) (Eq. 6); W = (H^T Q)^+ Z (P^T O)^+ (Eq. 9); svd(W) =
 * U_w Sigma V_w^T and f(LR) ~ (Q U_w) Sigma (P V_w)^T (Eq. 10).  Writes the
 * leading d = p->d triplets: U (n x d, ldu), sigma (d, FP64, descending),
 * V (m x d, ldv), all device and caller-owned; U or V may be NULL.  Uses
 * p->d, h, l, zeta, seed and f only (the sketch sizes need d <= h <= l,
 * h <= min(n, m), h <= 320).  FP32 sketches, FP64 small solves.  The
 * workspace (device, 256-byte aligned, sne_single_pass_svd_workspace_bytes)
 * is caller-owned; the unique rows of H are counted in the stats' v_o.
 * Errors: SNE_ERR_ARG, SNE_ERR_SIZE, SNE_ERR_WORKSPACE, SNE_ERR_CUDA on the
 * host; numerical failures in the workspace status word. */
int sne_single_pass_svd_workspace_bytes(int64_t n, int64_t m, int32_t k, const sne_params *p,
                                        size_t *bytes);
int sne_single_pass_svd(int64_t n, int64_t m, int32_t k, const float *L, int64_t ldl,
                        const float *Rt, int64_t ldr, const sne_params *p, void *workspace,
                        size_t ws_bytes, float *U, int64_t ldu, double *sigma, float *V,
                        int64_t ldv, sne_stream_t stream);

/* Spectral propagation, Alg. 6 line 6 (Sec. 4.3): E <- sum_{r=0..steps}
 * c_r T_r(X) E with L = I - D^-1 A (the normalized graph Laplacian of
 * Sec. 4.3) and X = (L - mu I)^2 / 2 - I.  The paper names c_r "coefficients
 * of Chebyshev polynomials" and takes p = 10, theta = 0.5, mu = 0.2 (Sec. 5.2)
 * from ProNE without printing them; here they are those of ProNE's band-pass
 * filter g(lambda) = exp(-theta/2 [(lambda - mu)^2 - 1]):
 * c_0 = e^(-theta/2) I_0(theta), c_r = 2 e^(-theta/2) (-1)^r I_r(theta), with
 * I_r the modified Bessel functions of the first kind (the Chebyshev series
 * of exp(-theta x) on [-1, 1]).
 *
 * sne_propagation_coefficients: host only; writes c_0 .. c_steps (steps + 1
 * doubles) to c.  SNE_ERR_ARG for c == NULL, steps outside [0, 1000], theta
 * negative or not finite.
 *
 * sne_spectral_propagate: E (device, n x d FP32, row-major, leading dimension
 * lde >= d, caller-owned) is replaced by the propagated embedding.  Each step
 * is two SpMMs by D^-1 A at width d (a vertex without edges is scaled by
 * g(1)); FP32 arithmetic.  The workspace (device, 256-byte aligned, at least
 * sne_spectral_propagate_workspace_bytes bytes, caller-owned) holds the status
 * word, 1/d and four n x d buffers.  Errors: SNE_ERR_ARG (graph or pointer
 * missing, d outside [1, 1024], lde < d, steps outside [0, 1000], theta < 0,
 * mu outside [0, 2]), SNE_ERR_SIZE (n above the int32 range),
 * SNE_ERR_WORKSPACE, SNE_ERR_CUDA (a launch or copy failed).  Stream-ordered;
 * nothing is synchronized. */
int sne_propagation_coefficients(int32_t steps, double theta, double *c);
int sne_spectral_propagate_workspace_bytes(int64_t n, int32_t d, size_t *bytes);
int sne_spectral_propagate(const sne_csr *g, int32_t steps, double theta, double mu, float *E,
                           int64_t lde, int32_t d, void *workspace, size_t ws_bytes,
                           sne_stream_t stream);

/* Checks the CSR on the device (monotone row_ptr, indices in range, symmetric
 * pattern and weights) and records SNE_ERR_GRAPH in the workspace status word
 * (any workspace of at least 256 bytes).  Read the result with sne_status(). */
int sne_validate_csr(const sne_csr *g, void *workspace, size_t ws_bytes, sne_stream_t stream);

/* Clears the status word of a workspace (stream-ordered). */
int sne_status_reset(void *workspace, sne_stream_t stream);

/* Synchronizes `stream` and returns the workspace's device status word. */
int sne_status(const void *workspace, sne_stream_t stream);

/* Synchronizes `stream` and copies the workspace counters into *out (host). */
int sne_stats_read(const void *workspace, sne_stats *out, sne_stream_t stream);

/* Allocation-free sne_freigs, for callers that cannot allocate device memory:
 * for example a plug-in running inside a host framework whose allocator owns
 * all device memory and forbids raw cudaMalloc, or a caller that may not
 * allocate (or wait for an allocator) in the middle of a latency-bound step.
 * The paper has no counterpart; this is an interface convenience.
 * The workspace is a static 32 MiB device array compiled into this library
 * (every GPU that loads the library holds it until the process exits).  A
 * graph whose freigs workspace (sne_workspace_bytes(..., SNE_WS_FREIGS)) is
 * larger than 32 MiB is rejected with SNE_ERR_SIZE before any work is
 * enqueued.  The call allocates nothing: the first call on a device looks up
 * the array's device address once (cudaGetSymbolAddress) and caches it; make
 * that first call before any stream capture.  Every call shares the array, so
 * calls that overlap on the GPU (other streams, other host threads) race: the
 * caller must serialize them.  The call clears the status word it uses and
 * performs the same computation as sne_freigs, with the same outputs.
 * `status` (a DEVICE int32, or NULL) receives the device status word (SNE_OK
 * or SNE_ERR_*) at the end of the enqueued work, and is written only when
 * the call returns SNE_OK: on any other return value nothing past the failing
 * step is enqueued, the return value is the result and `status` keeps its
 * previous contents.  U: n x k FP32 and lambda: k FP64 as in sne_freigs. */
int sne_freigs_static(const sne_csr *g, const sne_params *p, float *U, double *lambda,
                      int32_t *status, sne_stream_t stream);

/* ------------------------------------------------------------------------
 * Dense building blocks of Alg. 5 and Alg. 4, callable one by one.  Same
 * conventions as above: device pointers, row-major, stream-ordered; a
 * workspace of the stated size (256-byte aligned) whose first bytes hold the
 * device status word (read with sne_status).
 * ------------------------------------------------------------------------ */

/* Gram matrix of tall row-major FP32 matrices:
 *   C (ka x kb, FP64, row stride ldc) = sum_{i<n} w_i A[i, :]^T B[i, :]
 * A: n x ka (row stride lda), B: n x kb (ldb), w: n FP32 or NULL (all ones).
 * This is B = Y^T Y of eigSVD (Alg. 5), the Cholesky-QR Gram of Alg. 4's
 * orth(Y), S = Q^T (X Q) of the Rayleigh-Ritz step and U_k^T D^(-1+2 alpha)
 * U_k of Eq. 11.  accurate = 0: products FP32-accurate (3 x TF32 on the
 * tensor cores, or FP32 FMA), summed in FP32 over row blocks and in FP64
 * across blocks (relative error ~1e-6).  accurate = 1: FP32 FMA over groups of
 * 8 rows, the group sums added exactly into double-float pairs (relative
 * error ~1e-9), the form Eq. 11's core uses.  A == B with ka == kb and lda ==
 * ldb computes only the upper block triangle and mirrors it.
 * Errors: SNE_ERR_ARG (bad sizes or NULL), SNE_ERR_WORKSPACE. */
int sne_gram_workspace_bytes(int64_t n, int32_t ka, int32_t kb, size_t *bytes);
int sne_gram(int64_t n, int32_t ka, int32_t kb, const float *A, int64_t lda, const float *B,
             int64_t ldb, const float *w, double *C, int32_t ldc, int32_t accurate,
             void *workspace, size_t ws_bytes, sne_stream_t stream);

/* Tall-times-small product C (n x kc, row stride ldc) = A (n x ka, lda) M
 * (ka x kc, ldm), all FP32, FP32-accurate: Q = Y V Delta^-1/2 of eigSVD,
 * Q = Y R^-1 of Cholesky QR, U_k = Q U_hat of Alg. 5 and U_d = Q U_hat(:, 1:d)
 * of Alg. 4.  Errors as sne_gram. */
int sne_tall_gemm_workspace_bytes(int32_t ka, int32_t kc, size_t *bytes);
int sne_tall_gemm(int64_t n, int32_t ka, int32_t kc, const float *A, int64_t lda, const float *M,
                  int32_t ldm, float *C, int64_t ldc, void *workspace, size_t ws_bytes,
                  sne_stream_t stream);

/* Cholesky factor inverse of Cholesky QR (Alg. 4 line 5's orth(Y) = Y R^-1)
 * and of the normal equations of Alg. 4 line 8: for a symmetric positive
 * semidefinite A (n x n, lda; n <= 1024; FP64 if fp64 else FP32; only the
 * upper triangle is read) writes M (n x n, ldm, same type) with M^T A M = I.
 * tol < 0: A = R^T R and M = R^-1 (upper triangular); a non-positive pivot sets
 * SNE_ERR_NUMERIC.  tol >= 0: diagonal pivoting stopped at the numerical rank r
 * (the first remaining diagonal <= tol * max_i A_ii); M = P [R11^-1 0; 0 0],
 * so M^T A M = diag(I_r, 0) and the last n - r columns of M are zero.  Errors
 * as sne_gram. */
int sne_chol_inverse_workspace_bytes(int32_t n, int32_t fp64, size_t *bytes);
int sne_chol_inverse(int32_t n, const void *A, int32_t lda, void *M, int32_t ldm, int32_t fp64,
                     double tol, void *workspace, size_t ws_bytes, sne_stream_t stream);

/* Eigendecomposition of a symmetric FP64 matrix S (n x n, lds; n <= 1024) as
 * in the Rayleigh-Ritz step of Alg. 5: lambda (n) ordered by |lambda|
 * descending, V (n x n, ldv) with column j the eigenvector of lambda[j].  S is
 * not modified.  A failure to converge sets SNE_ERR_NUMERIC in the status
 * word.  Errors as sne_gram. */
int sne_sym_eig_workspace_bytes(int32_t n, size_t *bytes);
int sne_sym_eig(int32_t n, const double *S, int32_t lds, double *lambda, double *V, int32_t ldv,
                void *workspace, size_t ws_bytes, sne_stream_t stream);

/* Autotuner of the fused tensor-core sketch (Eq. 4 and the Z core of Alg. 4
 * with the half-precision reconstructions; the FP32 path has nothing to
 * tune): prepares the sketch operands of graph graphs[0] (G = 1, workspace of
 * sne_workspace_bytes(SNE_WS_EMBED)) or of the whole batch (G > 1, workspace
 * of sne_embed_batched_workspace_bytes with the same lanes), then times the
 * persistent sketch launch for every candidate shape: column tile width 128
 * or 256, every number of B stages that fits shared memory, and the column
 * split of the Z core (aiming at 1, 2 or 4 work items per SM).  The fastest
 * shape is kept for this kind of sketch (k, precision, z and log2 of the
 * rows) and used by later sne_embed / sne_embed_batched calls in this process.
 * For a batch with lanes <= 0 and output arrays E, sigma (as sne_embed_batched
 * takes them; null: skipped) the number of stream lanes (4, 8, 12 or 16) is
 * then timed over whole batched embeddings and kept for batches of this kind
 * (G, log2 of the total vertices, k, precision): sne_embed_batched with
 * lanes = 0 uses it.  No shape and no lane count changes a result.
 * Synchronizes the stream; out receives the choices and the times.  Errors:
 * SNE_ERR_ARG (FP32 precision, graphs of different z), SNE_ERR_WORKSPACE,
 * the errors of sne_embed. */
typedef struct sne_tune_result {
  int32_t tn, stages, split_mult; /* chosen launch shape */
  int32_t candidates;             /* shapes timed */
  float best_ms, default_ms;      /* one sketch launch: chosen and default shape */
  int32_t lanes;                  /* chosen lanes of a batch (0: not tuned) */
  float batch_ms;                 /* one batched embedding with them */
} sne_tune_result;
int sne_autotune_sketch(int32_t G, const sne_csr *graphs, const sne_params *p, int32_t lanes,
                        void *workspace, size_t ws_bytes, float *const *E, double *const *sigma,
                        sne_tune_result *out, sne_stream_t stream);

/* trunc_log as the tensor-core sketch epilogue evaluates it (Eq. 4 with
 * f = trunc_log, f(x) = max(0, log x)): out[i] = log1p(r[i]) for r[i] > 0 and
 * 0 otherwise, where r = x - 1 is the centred entry.  r and out are device
 * arrays of n FP32 values (may be the same array).  Relative error below 3e-7
 * for r > 0.  Errors: SNE_ERR_ARG for n < 0 or a null pointer with n > 0,
 * SNE_ERR_CUDA for a failed launch. */
int sne_trunc_log_eval(int64_t n, const float *r, float *out, sne_stream_t stream);

/* Kernel accounting (host only).  sne_kernel_launches returns the number of
 * kernels this library has enqueued since it was loaded.  Between
 * sne_profile_start and sne_profile_stop every launcher brackets its kernels
 * with CUDA events on its stream; sne_profile_stop synchronizes those events
 * and writes one sne_kernel_time per kernel class (at most max_entries,
 * *count = number of classes seen). */
typedef struct sne_kernel_time {
  char name[24];       /* kernel class */
  int64_t calls;       /* launcher calls */
  int64_t launches;    /* kernels enqueued */
  double total_ms;     /* summed event time */
} sne_kernel_time;

long long sne_kernel_launches(void);
int sne_profile_start(void);
int sne_profile_stop(sne_kernel_time *out, int max_entries, int *count);

#ifdef __cplusplus
}
#endif
#endif /* SKETCHNE_H */
