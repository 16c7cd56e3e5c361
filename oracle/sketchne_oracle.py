"""SketchNE oracle: a plain, slow, obviously correct FP64 CPU implementation.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports, links or runs
this file: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` use it.  It shares no code with the CUDA library; the two
sides meet only at the seeded graphs of ``paper_2110_12782_gb300.synth`` and at
the published definition of the counter-based random generator below, which
each side implements on its own.

Everything is FP64 NumPy/SciPy.  Library primitives (dense matmul, sparse
matmul, LAPACK ``eigh``/``qr``/``lstsq``/``svd``, ``unique``) serve as single
steps; there is no blocking, fusion or reordering beyond what the paper states.

Paper: "SketchNE: Embedding Billion-Scale Networks Accurately in One Hour"
(arXiv 2110.12782).  Section, equation and algorithm numbers below are the
paper's.

Readings of points the paper leaves open:

* ``unique`` (Alg. 3) returns the coordinates sorted ascending.
* ``randperm(n, z)`` (Alg. 3) is z distinct rows drawn uniformly without
  replacement; z = min(n, zeta) (Sec. 4.1); the signs are +-1 with equal
  probability, scaled by 1/sqrt(z).
* ``freigs`` (Alg. 5) returns the k eigenpairs of largest |lambda| (the
  quantity of Lemma 4 / Theorem 1), ordered by |lambda| descending.
* For an isolated vertex (degree 0) every power of its degree is taken as 0
  (pseudo-inverse), so its rows of X, L', R', Y and E are 0.  A graph with no
  edges at all (vol(G) = 0, Eq. 1 undefined) is rejected.
* trunc_log(x) = max(0, ln x), with trunc_log(x) = 0 for x <= 1 (including
  x <= 0, where log is undefined).
* eigSVD (Alg. 5, from frPCA) is  B = Y^T Y, eig(B) = V D V^T,
  Q = Y V D^(-1/2).
* The sketch sizes are h = d + s1 and l = d + s2 (Alg. 4); the default is
  s1 = d + 16 (sketch size 2d + 16) and s2 = 1000 (Sec. 5.2).

Random numbers: SplitMix64 (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) used as a counter-based
generator: output number i (1-based) of a SplitMix64 generator whose state
starts at s is mix64(s + i * 0x9E3779B97F4A7C15).  Bounded integers use
Lemire's multiply-shift with rejection ("Fast random integer generation in an
interval", ACM TOMACS 2019); Gaussians use the Box-Muller transform on 24-bit
uniforms.  Stream ids: 1 = Omega (Alg. 5), 2 = S (Alg. 4 line 3),
3 = O (Alg. 4 line 6), 4 = C and 5 = H (the general single-pass SVD of
Eqs. 5-10).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

# ---------------------------------------------------------------------------
# Counter-based random numbers (published definitions, see module docstring)
# ---------------------------------------------------------------------------
MASK64 = (1 << 64) - 1
GOLDEN = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB

STREAM_OMEGA = 1
STREAM_S = 2
STREAM_O = 3
STREAM_C = 4
STREAM_H = 5


def mix64(z: int) -> int:
    """SplitMix64 output function."""
    z &= MASK64
    z = ((z ^ (z >> 30)) * MIX1) & MASK64
    z = ((z ^ (z >> 27)) * MIX2) & MASK64
    return z ^ (z >> 31)


def splitmix64_output(state: int, i: int) -> int:
    """Output number ``i`` (1-based) of SplitMix64 seeded with ``state``."""
    return mix64((state + i * GOLDEN) & MASK64)


def stream_key(seed: int, stream: int) -> int:
    return splitmix64_output(seed & MASK64, stream + 1)


def draw(key: int, ctr: int) -> int:
    return splitmix64_output(key, ctr + 1)


def bounded(key: int, ctr: int, n: int):
    """Uniform integer in [0, n) by Lemire's multiply-shift with rejection.

    Returns (value, next counter)."""
    x = draw(key, ctr)
    ctr += 1
    m = x * n
    lo = m & MASK64
    if lo < n:
        threshold = ((1 << 64) - n) % n
        while lo < threshold:
            x = draw(key, ctr)
            ctr += 1
            m = x * n
            lo = m & MASK64
    return m >> 64, ctr


def _mix64_np(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
    return z ^ (z >> np.uint64(31))


def draw_np(key: int, ctr: np.ndarray) -> np.ndarray:
    with np.errstate(over="ignore"):
        return _mix64_np(np.uint64(key) + np.uint64(GOLDEN) * (ctr.astype(np.uint64) + np.uint64(1)))


# ---------------------------------------------------------------------------
# Alg. 3: gen_sparse_sign_matrix(n, h, z)
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class SparseSign:
    """Sparse-sign matrix of Alg. 3 in coordinate form.

    ``idx[j, t]`` is the row of the t-th nonzero of column j, ``sign[j, t]`` its
    sign (+-1); every nonzero has value ``sign / sqrt(z)``.  ``p`` is
    ``unique(idx)`` (Alg. 3 line 8)."""

    n: int
    idx: np.ndarray
    sign: np.ndarray
    p: np.ndarray
    scale: float = 0.0  # value of a +1 entry; 0 -> 1/sqrt(z)

    @property
    def value(self) -> float:
        return self.scale if self.scale > 0 else 1.0 / math.sqrt(self.z)

    @property
    def cols(self) -> int:
        return self.idx.shape[0]

    @property
    def z(self) -> int:
        return self.idx.shape[1]

    def dense(self) -> np.ndarray:
        """The full n x cols matrix (for brute-force checks on small n)."""
        M = np.zeros((self.n, self.cols))
        for j in range(self.cols):
            M[self.idx[j], j] = self.sign[j] * self.value
        return M

    def rows_at_p(self) -> np.ndarray:
        """S(p, :), the v x cols restriction to the unique coordinates."""
        M = np.zeros((len(self.p), self.cols))
        pos = np.searchsorted(self.p, self.idx)
        for j in range(self.cols):
            M[pos[j], j] = self.sign[j] * self.value
        return M


def gen_sparse_sign(n: int, cols: int, zeta: int, seed: int, stream: int) -> SparseSign:
    """Alg. 3.  For each column j: z = min(n, zeta) distinct rows (randperm),
    each with an independent random sign; then p = unique(all rows).

    Column j draws its rows from counters (j << 32) + c, c = 0, 1, 2, ...,
    skipping a row already taken in the column; its t-th sign is the top bit
    of draw((j << 32) | (1 << 31) | t) (0 -> +1, 1 -> -1)."""
    z = min(n, zeta)
    key = stream_key(seed, stream)
    idx = np.empty((cols, z), dtype=np.int64)
    sign = np.empty((cols, z), dtype=np.int8)
    for j in range(cols):
        ctr = j << 32
        chosen: list[int] = []
        while len(chosen) < z:
            r, ctr = bounded(key, ctr, n)
            if r not in chosen:
                chosen.append(r)
        idx[j] = chosen
        for t in range(z):
            bit = draw(key, (j << 32) | (1 << 31) | t) >> 63
            sign[j, t] = 1 if bit == 0 else -1
    p = np.unique(idx)
    return SparseSign(n=n, idx=idx, sign=sign, p=p)


# ---------------------------------------------------------------------------
# Gaussian test matrix Omega = randn(n, k+s)  (Alg. 5 line 3)
# ---------------------------------------------------------------------------
def gaussian_matrix(n: int, cols: int, seed: int, stream: int = STREAM_OMEGA,
                    row0: int = 0, rows: int | None = None) -> np.ndarray:
    """Rows [row0, row0+rows) of the n x cols standard normal matrix.

    Entry e = i*cols + c uses the pair of draws at counters 2*(e//2) and
    2*(e//2)+1: u1 = (hi24(x1) + 1) / 2^24, u2 = hi24(x2) / 2^24,
    r = sqrt(-2 ln u1); the entry is r cos(2 pi u2) for even e and
    r sin(2 pi u2) for odd e (Box-Muller)."""
    if rows is None:
        rows = n - row0
    key = stream_key(seed, stream)
    e = np.arange(row0 * cols, (row0 + rows) * cols, dtype=np.uint64)
    pair = e >> np.uint64(1)
    x1 = draw_np(key, pair * np.uint64(2))
    x2 = draw_np(key, pair * np.uint64(2) + np.uint64(1))
    u1 = ((x1 >> np.uint64(40)).astype(np.float64) + 1.0) * 2.0 ** -24
    u2 = (x2 >> np.uint64(40)).astype(np.float64) * 2.0 ** -24
    r = np.sqrt(-2.0 * np.log(u1))
    theta = 2.0 * np.pi * u2
    g = np.where((e & np.uint64(1)) == 0, r * np.cos(theta), r * np.sin(theta))
    return g.reshape(rows, cols)


# ---------------------------------------------------------------------------
# Graph quantities (Sec. 2, Table 2)
# ---------------------------------------------------------------------------
def adjacency(row_ptr, col_idx, n, val=None) -> sp.csr_matrix:
    data = np.ones(len(col_idx)) if val is None else np.asarray(val, dtype=np.float64)
    return sp.csr_matrix((data, np.asarray(col_idx, dtype=np.int64), np.asarray(row_ptr, dtype=np.int64)),
                         shape=(n, n))


def degrees(A: sp.csr_matrix) -> np.ndarray:
    """d_i = sum_j A_ij."""
    return np.asarray(A.sum(axis=1)).ravel()


def volume(A: sp.csr_matrix) -> float:
    """vol(G) = sum_i sum_j A_ij."""
    return float(A.sum())


def degree_power(deg: np.ndarray, beta: float) -> np.ndarray:
    """deg**beta with isolated vertices mapped to 0 (pseudo-inverse reading)."""
    out = np.zeros_like(deg, dtype=np.float64)
    nz = deg > 0
    out[nz] = deg[nz] ** beta
    return out


def normalized_operator(A: sp.csr_matrix, alpha: float) -> sp.csr_matrix:
    """X = D^-alpha A D^-alpha, the modified Laplacian of Sec. 4.2."""
    s = degree_power(degrees(A), -alpha)
    Ds = sp.diags(s)
    return (Ds @ A @ Ds).tocsr()


def trunc_log(x: np.ndarray) -> np.ndarray:
    """trunc_log(x) = max(0, log x), elementwise (Eq. 1); 0 wherever x <= 1."""
    out = np.zeros_like(x, dtype=np.float64)
    m = x > 1.0
    out[m] = np.log(x[m])
    return out


def identity(x: np.ndarray) -> np.ndarray:
    return np.array(x, dtype=np.float64, copy=True)


F_TABLE = {"trunc_log": trunc_log, "identity": identity}


# ---------------------------------------------------------------------------
# Alg. 5: freigs(X, k, q), with eigSVD from frPCA
# ---------------------------------------------------------------------------
def eigsvd(Y: np.ndarray):
    """eigSVD: B = Y^T Y; eig(B) = V D V^T; S = D^(1/2); Q = Y V S^-1.

    Returns (Q, S, V) with the eigenvalues in LAPACK's ascending order."""
    B = Y.T @ Y
    Dv, V = np.linalg.eigh(B)
    S = np.sqrt(Dv)
    Q = Y @ (V / S[None, :])
    return Q, S, V


def freigs(X: sp.csr_matrix, k: int, q: int, s: int, seed: int):
    """Alg. 5.  Returns (U_k, lambda_k) with |lambda| descending."""
    n = X.shape[1]
    Omega = gaussian_matrix(n, k + s, seed, STREAM_OMEGA)
    Y = X @ Omega
    Q, _, _ = eigsvd(Y)
    for _ in range(q):
        Q, _, _ = eigsvd(X @ (X @ Q))
    Sred = Q.T @ (X @ Q)
    Sred = 0.5 * (Sred + Sred.T)  # symmetric in exact arithmetic
    lam, Uhat = np.linalg.eigh(Sred)
    order = np.argsort(-np.abs(lam), kind="stable")
    lam = lam[order]
    U = Q @ Uhat[:, order]
    return U[:, :k], lam[:k]


# ---------------------------------------------------------------------------
# Eq. 11 / Alg. 6 lines 2-3: the factors L', R'
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Factors:
    Lp: np.ndarray  # n x k
    Rp: np.ndarray  # k x n
    K: np.ndarray   # k x k
    Csum: np.ndarray  # sum_{r=1..T} K^(r-1)


def netmf_factors(U: np.ndarray, lam: np.ndarray, deg: np.ndarray, vol: float,
                  alpha: float, T: int, b: float) -> Factors:
    """K = U^T D^(-1+2a) U Lambda;  L' = vol/(bT) D^(-1+a) U;
    R' = Lambda (sum_{r=1..T} K^(r-1)) U^T D^(-1+a)."""
    a = degree_power(deg, -1.0 + alpha)
    w = degree_power(deg, -1.0 + 2.0 * alpha)
    Lam = np.diag(lam)
    K = U.T @ (w[:, None] * U) @ Lam
    k = len(lam)
    Csum = np.zeros((k, k))
    Kpow = np.eye(k)
    for _ in range(T):
        Csum += Kpow
        Kpow = Kpow @ K
    Lp = (vol / (b * T)) * (a[:, None] * U)
    Rp = (Lam @ Csum @ U.T) * a[None, :]
    return Factors(Lp=Lp, Rp=Rp, K=K, Csum=Csum)


def netmf_factor_rows(U: np.ndarray, lam: np.ndarray, deg: np.ndarray, vol: float, alpha: float,
                      T: int, b: float, rows: np.ndarray, cols: np.ndarray,
                      chunk: int = 1 << 20):
    """Eq. 11 as in ``netmf_factors``, returning only the rows ``rows`` of L'
    and the columns ``cols`` of R' (for graphs whose n x k factors do not fit
    in host memory): K = U^T D^(-1+2a) U Lambda is summed over row chunks of
    U, the rest is the same arithmetic on the selected rows and columns."""
    k = len(lam)
    a = degree_power(deg, -1.0 + alpha)
    w = degree_power(deg, -1.0 + 2.0 * alpha)
    G = np.zeros((k, k))
    for r0 in range(0, U.shape[0], chunk):
        Uc = np.asarray(U[r0:r0 + chunk], dtype=np.float64)
        G += Uc.T @ (w[r0:r0 + chunk, None] * Uc)
    Lam = np.diag(lam)
    K = G @ Lam
    Csum = np.zeros((k, k))
    Kpow = np.eye(k)
    for _ in range(T):
        Csum += Kpow
        Kpow = Kpow @ K
    Lp_rows = (vol / (b * T)) * (a[rows, None] * np.asarray(U[rows], dtype=np.float64))
    Rp_cols = (Lam @ Csum @ np.asarray(U[cols], dtype=np.float64).T) * a[None, cols]
    return Lp_rows, Rp_cols


def sketch_Y_rows_at(Lp_rows: np.ndarray, Rp_at_p: np.ndarray, S: "SparseSign", f=None):
    """Rows of Y of Eq. 4 given the rows of L' and the columns R'(:, p) at the
    unique coordinates p of S."""
    f = trunc_log if f is None else f
    return f(Lp_rows @ Rp_at_p) @ S.rows_at_p()


# ---------------------------------------------------------------------------
# Alg. 4: sparse-sign randomized single-pass SVD of f(L R)
# ---------------------------------------------------------------------------
def sketch_Y(Lp: np.ndarray, Rp: np.ndarray, S: SparseSign, f=trunc_log, row_block: int = 8192):
    """Eq. 4 / Alg. 4 line 4: Y = f(L R(:, p)) S(p, :), evaluated in fixed-size
    row blocks of L (the batched multiplication of Sec. 4.1)."""
    n = Lp.shape[0]
    Rsub = Rp[:, S.p]
    Ssub = S.rows_at_p()
    Y = np.empty((n, S.cols))
    for r0 in range(0, n, row_block):
        r1 = min(n, r0 + row_block)
        Y[r0:r1] = f(Lp[r0:r1] @ Rsub) @ Ssub
    return Y


def sketch_Y_rows(Lp_rows: np.ndarray, Rp: np.ndarray, S: SparseSign, f=trunc_log):
    """Selected rows of Y (rows of L given explicitly)."""
    return f(Lp_rows @ Rp[:, S.p]) @ S.rows_at_p()


def sketch_Z(Lp: np.ndarray, Rp: np.ndarray, O: SparseSign, f=trunc_log):
    """Alg. 4 line 7: Z = O(p,:)^T f(L(p,:) R(:,p)) O(p,:)."""
    Osub = O.rows_at_p()
    core = f(Lp[O.p] @ Rp[:, O.p])
    return Osub.T @ core @ Osub


@dataclasses.dataclass
class SinglePassResult:
    U: np.ndarray      # n x d
    sigma: np.ndarray  # d
    Y: np.ndarray
    Q: np.ndarray
    Z: np.ndarray
    W: np.ndarray
    S: SparseSign
    O: SparseSign


def single_pass_svd(Lp: np.ndarray, Rp: np.ndarray, d: int, h: int, l: int, zeta: int,
                    seed: int, f=trunc_log, row_block: int = 8192,
                    sign_scale: float = 0.0) -> SinglePassResult:
    """Alg. 4 with the two least-squares solves of Sec. 4.1 for W.

    ``sign_scale`` overrides the value 1/sqrt(z) of the sparse-sign entries
    (the result is invariant to it)."""
    n = Lp.shape[0]
    S = gen_sparse_sign(n, h, zeta, seed, STREAM_S)
    S.scale = sign_scale
    Y = sketch_Y(Lp, Rp, S, f, row_block)
    Q, _ = np.linalg.qr(Y)  # Householder QR (LAPACK)
    O = gen_sparse_sign(n, l, zeta, seed, STREAM_O)
    O.scale = sign_scale
    Z = sketch_Z(Lp, Rp, O, f)
    G = O.rows_at_p().T @ Q[O.p]          # O^T Q, l x h
    Tm = np.linalg.lstsq(G, Z, rcond=None)[0]       # (O^T Q) T = Z
    Wt = np.linalg.lstsq(G, Tm.T, rcond=None)[0]    # (O^T Q) W^T = T^T
    W = Wt.T
    Uh, sig, _ = np.linalg.svd(W)
    return SinglePassResult(U=Q @ Uh[:, :d], sigma=sig[:d], Y=Y, Q=Q, Z=Z, W=W, S=S, O=O)


@dataclasses.dataclass
class GeneralSinglePassResult:
    U: np.ndarray      # n x d, left singular vectors
    sigma: np.ndarray  # d
    V: np.ndarray      # m x d, right singular vectors
    Y: np.ndarray
    K: np.ndarray
    Z: np.ndarray
    W: np.ndarray


def single_pass_svd_general(L: np.ndarray, Rt: np.ndarray, d: int, h: int, l: int, zeta: int,
                            seed: int, f=trunc_log) -> GeneralSinglePassResult:
    """Eqs. 5-10 (Sec. 4.1) for a general, not necessarily symmetric or square,
    f(L R) with L n x k and R = Rt^T k x m: sparse-sign C (n x h), S (m x h),
    H (n x l), O (m x l) (Alg. 3; random streams 4, 2, 5, 3);
    K = f(LR)^T C, Y = f(LR) S, Z = H^T f(LR) O (Eq. 5); P = orth(K),
    Q = orth(Y) (Eq. 6); W = (H^T Q)^+ Z (P^T O)^+ (Eq. 9), taken as two
    least-squares solves; svd(W) = U_w Sigma V_w^T, f(LR) ~ (Q U_w) Sigma
    (P V_w)^T (Eq. 10), the leading d triplets."""
    n, m = L.shape[0], Rt.shape[0]
    C = gen_sparse_sign(n, h, zeta, seed, STREAM_C)
    S = gen_sparse_sign(m, h, zeta, seed, STREAM_S)
    H = gen_sparse_sign(n, l, zeta, seed, STREAM_H)
    O = gen_sparse_sign(m, l, zeta, seed, STREAM_O)
    Y = f(L @ Rt[S.p].T) @ S.rows_at_p()
    K = f(Rt @ L[C.p].T) @ C.rows_at_p()
    Z = H.rows_at_p().T @ f(L[H.p] @ Rt[O.p].T) @ O.rows_at_p()
    P, _ = np.linalg.qr(K)
    Q, _ = np.linalg.qr(Y)
    HQ = H.rows_at_p().T @ Q[H.p]     # H^T Q, l x h
    OP = O.rows_at_p().T @ P[O.p]     # O^T P = (P^T O)^T, l x h
    Tm = np.linalg.lstsq(HQ, Z, rcond=None)[0]          # (H^T Q) T = Z
    W = np.linalg.lstsq(OP, Tm.T, rcond=None)[0].T      # W (P^T O) = T
    Uw, sig, Vwt = np.linalg.svd(W)
    return GeneralSinglePassResult(U=Q @ Uw[:, :d], sigma=sig[:d], V=P @ Vwt.T[:, :d], Y=Y, K=K, Z=Z,
                                   W=W)


# ---------------------------------------------------------------------------
# Alg. 6 lines 1-5: SketchNE (initial embedding)
# ---------------------------------------------------------------------------
@dataclasses.dataclass
class Params:
    k: int = 256
    d: int = 128
    q: int = 20
    T: int = 10
    b: float = 1.0
    alpha: float = 0.5
    zeta: int = 8
    s_eig: int = 16
    h: int = 0        # 0 -> 2d + 16
    l: int = 0        # 0 -> d + 1000
    seed: int = 0
    f: str = "trunc_log"
    row_block: int = 8192

    def resolved(self) -> "Params":
        p = dataclasses.replace(self)
        if p.h <= 0:
            p.h = 2 * p.d + 16
        if p.l <= 0:
            p.l = p.d + 1000
        return p


@dataclasses.dataclass
class EmbedResult:
    E: np.ndarray
    sigma: np.ndarray
    U_k: np.ndarray
    lam: np.ndarray
    deg: np.ndarray
    vol: float
    factors: Factors
    sp: SinglePassResult


def embed(row_ptr, col_idx, n, params: Params, val=None, U_k=None, lam=None) -> EmbedResult:
    """Alg. 6 lines 1-5.  ``U_k``/``lam`` may be given to skip line 1."""
    p = params.resolved()
    A = adjacency(row_ptr, col_idx, n, val)
    deg = degrees(A)
    vol = volume(A)
    if not vol > 0:
        raise ValueError("a graph without edges has vol(G) = 0: Eq. 1 is undefined")
    if U_k is None:
        X = normalized_operator(A, p.alpha)
        U_k, lam = freigs(X, p.k, p.q, p.s_eig, p.seed)
    fac = netmf_factors(U_k, lam, deg, vol, p.alpha, p.T, p.b)
    res = single_pass_svd(fac.Lp, fac.Rp, p.d, p.h, p.l, p.zeta, p.seed, F_TABLE[p.f], p.row_block)
    E = res.U * np.sqrt(res.sigma)[None, :]
    return EmbedResult(E=E, sigma=res.sigma, U_k=U_k, lam=lam, deg=deg, vol=vol, factors=fac, sp=res)


# ---------------------------------------------------------------------------
# Alg. 6 line 6: spectral propagation
# ---------------------------------------------------------------------------
def propagation_coefficients(steps: int, theta: float) -> np.ndarray:
    """c_0 .. c_steps of exp(-theta/2 [(lam - mu)^2 - 1]) as a Chebyshev series
    in x = (lam - mu)^2 / 2 - 1: the filter is exp(-theta/2) exp(-theta x), and
    exp(-theta x) = I_0(theta) + 2 sum_{r>=1} (-1)^r I_r(theta) T_r(x) on
    [-1, 1] (the generating function of the modified Bessel functions of the
    first kind I_r).  Reading of the coefficients the paper leaves to ProNE
    (Zhang et al., IJCAI 2019: band-pass filter g, Chebyshev expansion with
    Bessel coefficients)."""
    import scipy.special
    r = np.arange(steps + 1)
    c = 2.0 * (-1.0) ** r * scipy.special.iv(r, theta)
    c[0] = scipy.special.iv(0, theta)
    return math.exp(-0.5 * theta) * c


def spectral_propagation(A: sp.csr_matrix, E: np.ndarray, steps: int = 10, theta: float = 0.5,
                         mu: float = 0.2) -> np.ndarray:
    """Alg. 6 line 6: E <- sum_{r=0..steps} c_r T_r(X) E, the Chebyshev series
    of g(L) = exp(-theta/2 [(L - mu I)^2 - I]) for the normalized Laplacian
    L = I - D^-1 A (Sec. 4.3), in the variable X = (L - mu I)^2 / 2 - I, whose
    spectrum lies in [-1, 1] when 0 <= mu <= 2 (that of L lies in [0, 2]).
    T_0 = E, T_1 = X E, T_{r+1} = 2 X T_r - T_{r-1}.  Defaults p = 10,
    theta = 0.5, mu = 0.2 (Sec. 5.2).  Isolated vertices: D^-1 A has a zero
    row, so their rows are scaled by g(1)."""
    deg = degrees(A)
    P = (sp.diags(degree_power(deg, -1.0)) @ A).tocsr()  # D^-1 A

    def M(V):  # (L - mu I) V
        return (1.0 - mu) * V - P @ V

    def X(V):
        return 0.5 * M(M(V)) - V

    c = propagation_coefficients(steps, theta)
    E = np.asarray(E, dtype=np.float64)
    F = c[0] * E
    if steps >= 1:
        T_prev, T_cur = E, X(E)
        F = F + c[1] * T_cur
        for r in range(2, steps + 1):
            T_prev, T_cur = T_cur, 2.0 * X(T_cur) - T_prev
            F = F + c[r] * T_cur
    return F


# ---------------------------------------------------------------------------
# Dense references for tiny graphs
# ---------------------------------------------------------------------------
def netmf_matrix_dense(A_dense: np.ndarray, T: int, b: float) -> np.ndarray:
    """Eq. 1 before trunc_log: vol/(bT) sum_{r=1..T} (D^-1 A)^r D^-1."""
    deg = A_dense.sum(axis=1)
    vol = A_dense.sum()
    Dinv = np.diag(degree_power(deg, -1.0))
    P = Dinv @ A_dense
    acc = np.zeros_like(A_dense, dtype=np.float64)
    Pr = np.eye(A_dense.shape[0])
    for _ in range(T):
        Pr = Pr @ P
        acc += Pr
    return vol / (b * T) * acc @ Dinv


def netmf_eq2_dense(A_dense: np.ndarray, U: np.ndarray, lam: np.ndarray, T: int, b: float) -> np.ndarray:
    """Eq. 2 before trunc_log: vol/(bT) D^-1/2 U (sum_r Lambda^r) U^T D^-1/2."""
    deg = A_dense.sum(axis=1)
    vol = A_dense.sum()
    s = degree_power(deg, -0.5)
    lam_sum = sum(lam ** r for r in range(1, T + 1))
    return vol / (b * T) * (s[:, None] * U) @ np.diag(lam_sum) @ (U.T * s[None, :])


def theorem1_bound(eig_abs_desc: np.ndarray, k: int, deg: np.ndarray, vol: float, n: int,
                   alpha: float, T: int, b: float, eps: float = 0.0) -> float:
    """Right-hand side of Theorem 1."""
    dmin = deg[deg > 0].min()
    dmax = deg.max()
    tail = math.sqrt(float(np.sum(eig_abs_desc[k:] ** 2)))
    c = n * (dmax / dmin) ** (1.0 - 2.0 * alpha)
    B = tail * ((c ** T - 1.0) * (1.0 + n / (c - 1.0)) - n * T) * vol
    return (1.0 + eps) * dmin ** (-1.0 + 2.0 * alpha) * B / ((c - 1.0) * b * T)


def principal_angle_sines(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Sines of the principal angles between span(A) and span(B), descending."""
    Qa, _ = np.linalg.qr(A)
    Qb, _ = np.linalg.qr(B)
    c = np.linalg.svd(Qa.T @ Qb, compute_uv=False)
    c = np.clip(c, 0.0, 1.0)
    return np.sort(np.sqrt(np.maximum(0.0, 1.0 - c * c)))[::-1]
