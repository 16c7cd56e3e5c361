"""The dense building blocks of Alg. 5 and Alg. 4 through the C-ABI, one by one,
against their plain FP64 definitions (numpy) on the same FP32 inputs.

Sizes run from a few rows (the FP32-FMA path) through several tiles with a
ragged tail up to the benchmark's full size (n = 1,000,000 rows, 272
columns).  The tall inputs mimic the basis matrices the pipeline feeds these
blocks: a heavy-tailed first column (proportional to sqrt(degree) for a
power-law degree sequence, as the top eigenvector of D^-1/2 A D^-1/2) and
Gaussian columns with row scales spread over three decades.
"""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sk():
    from paper_2110_12782_gb300 import build
    build.build()
    from paper_2110_12782_gb300 import sketchne
    sketchne.lib()
    return sketchne


def tall_basis(n, k, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, k)).astype(np.float32)
    A *= np.exp(rng.uniform(-3.5, 3.5, size=(n, 1))).astype(np.float32)
    deg = np.floor(rng.pareto(1.1, size=n) + 1.0)
    A[:, 0] = np.sqrt(deg / deg.sum())
    A[:, 1:] /= np.linalg.norm(A[:, 1:], axis=0, keepdims=True)
    return A


def gram_error(C, ref):
    d = np.sqrt(np.abs(np.diag(ref)))
    if ref.shape[0] != ref.shape[1]:
        raise ValueError
    return float(np.max(np.abs(C - ref) / np.outer(d, d)))


def cross_error(C, ref, A, B):
    na = np.sqrt((A.astype(np.float64) ** 2).sum(axis=0))
    nb = np.sqrt((B.astype(np.float64) ** 2).sum(axis=0))
    return float(np.max(np.abs(C - ref) / np.outer(na, nb)))


# The accurate form's error is that of one FP32 sum over a 16-row group, so it
# is largest relative to the total when n is small and shrinks as n grows.
TOL = {False: 1e-5, True: 1e-7}


@pytest.mark.parametrize("accurate", [False, True])
@pytest.mark.parametrize("n,k", [(300, 16), (4097, 144), (100_003, 272), (1_000_000, 272)])
def test_gram_symmetric(sk, n, k, accurate):
    A = tall_basis(n, k, seed=n)
    ref = A.astype(np.float64).T @ A.astype(np.float64)
    Ad = torch.from_numpy(A).cuda()
    C = torch.empty(k, k, dtype=torch.float64, device="cuda")
    ws = sk.gram_workspace(n, k, k)
    sk.sne_gram(Ad, Ad, C, ws, accurate=accurate)
    assert sk.sne_status(ws) == 0
    err = gram_error(C.cpu().numpy(), ref)
    print(f"gram n={n} k={k} accurate={accurate}: max |C - ref| / sqrt(ref_aa ref_bb) = {err:.2e}")
    assert err < (1e-8 if accurate and n >= 1_000_000 else TOL[accurate])


@pytest.mark.parametrize("accurate", [False, True])
@pytest.mark.parametrize("n,k", [(4097, 144), (1_000_000, 256)])
def test_gram_weighted(sk, n, k, accurate):
    """U^T D^(-1+2 alpha) U of Eq. 11 with positive weights over four decades."""
    A = tall_basis(n, k, seed=7 + n)
    rng = np.random.default_rng(3)
    w = np.exp(rng.uniform(-4.6, 4.6, size=n)).astype(np.float32)
    ref = (A.astype(np.float64) * w[:, None].astype(np.float64)).T @ A.astype(np.float64)
    Ad = torch.from_numpy(A).cuda()
    C = torch.empty(k, k, dtype=torch.float64, device="cuda")
    ws = sk.gram_workspace(n, k, k)
    sk.sne_gram(Ad, Ad, C, ws, w=torch.from_numpy(w).cuda(), accurate=accurate)
    assert sk.sne_status(ws) == 0
    err = gram_error(C.cpu().numpy(), ref)
    print(f"weighted gram n={n} k={k} accurate={accurate}: {err:.2e}")
    assert err < TOL[accurate]


@pytest.mark.parametrize("accurate", [False, True])
@pytest.mark.parametrize("n,ka,kb", [(1000, 100, 37), (65_537, 272, 272), (1_000_000, 272, 272)])
def test_gram_cross(sk, n, ka, kb, accurate):
    """S = Q^T (X Q) of the Rayleigh-Ritz step: two different tall matrices."""
    A = tall_basis(n, ka, seed=11)
    B = tall_basis(n, kb, seed=12)
    ref = A.astype(np.float64).T @ B.astype(np.float64)
    C = torch.empty(ka, kb, dtype=torch.float64, device="cuda")
    ws = sk.gram_workspace(n, ka, kb)
    sk.sne_gram(torch.from_numpy(A).cuda(), torch.from_numpy(B).cuda(), C, ws, accurate=accurate)
    assert sk.sne_status(ws) == 0
    err = cross_error(C.cpu().numpy(), ref, A, B)
    print(f"cross gram n={n} {ka}x{kb} accurate={accurate}: {err:.2e}")
    assert err < TOL[accurate]


@pytest.mark.parametrize("n,ka,kc", [(500, 40, 24), (4097, 272, 272), (20_000, 272, 200),
                                     (1_000_000, 272, 256), (1_000_000, 272, 128)])
def test_tall_gemm(sk, n, ka, kc):
    A = tall_basis(n, ka, seed=5)
    rng = np.random.default_rng(6)
    M = rng.standard_normal((ka, kc)).astype(np.float32)
    C = torch.empty(n, kc, dtype=torch.float32, device="cuda")
    ws = sk.tall_gemm_workspace(ka, kc)
    sk.sne_tall_gemm(torch.from_numpy(A).cuda(), torch.from_numpy(M).cuda(), C, ws)
    assert sk.sne_status(ws) == 0
    rows = np.unique(np.concatenate([np.arange(min(n, 64)), np.arange(max(0, n - 64), n),
                                     np.random.default_rng(9).choice(n, min(n, 4096), replace=False)]))
    ref = A[rows].astype(np.float64) @ M.astype(np.float64)
    got = C[torch.as_tensor(rows, device="cuda")].cpu().numpy().astype(np.float64)
    scale = np.sqrt((A[rows].astype(np.float64) ** 2) @ (M.astype(np.float64) ** 2))
    err = float(np.max(np.abs(got - ref) / scale))
    print(f"tall gemm n={n} {ka}x{kc}: {err:.2e}")
    # 3 x TF32 products; the tensor-core accumulator rounds each of the
    # 3 * ka / 8 updates of a K-chain, about 0.5 ulp of the running sum each
    assert err < 3e-5


def clustered_symmetric(n, seed, n_plus=19, n_minus=18, n_zero=23):
    """V diag(lam) V^T with eigenvalue clusters at +1, -1 and 0 (each split by
    1e-9), as the Rayleigh-Ritz matrix of a graph with many small components."""
    rng = np.random.default_rng(seed)
    V, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = rng.uniform(-0.9, 0.9, size=n)
    lam[:n_plus] = 1.0 - 1e-9 * rng.random(n_plus)
    lam[n_plus:n_plus + n_minus] = -1.0 + 1e-9 * rng.random(n_minus)
    lam[n_plus + n_minus:n_plus + n_minus + n_zero] = 1e-9 * rng.standard_normal(n_zero)
    S = (V * lam) @ V.T
    return 0.5 * (S + S.T), lam, V


@pytest.mark.parametrize("n", [8, 144, 272, 320, 600])
def test_sym_eig_clustered(sk, n):
    c = min(19, n // 4)
    S, lam_true, V_true = clustered_symmetric(n, seed=n, n_plus=c, n_minus=c, n_zero=c)
    Sd = torch.from_numpy(S).cuda()
    lam = torch.empty(n, dtype=torch.float64, device="cuda")
    V = torch.empty(n, n, dtype=torch.float64, device="cuda")
    ws = sk.sym_eig_workspace(n)
    sk.sne_sym_eig(Sd, lam, V, ws)
    assert sk.sne_status(ws) == 0
    l, Vh = lam.cpu().numpy(), V.cpu().numpy()
    assert np.all(np.diff(np.abs(l)) <= 1e-12)
    orth = np.abs(Vh.T @ Vh - np.eye(n)).max()
    lam_err = np.abs(np.sort(l) - np.sort(lam_true)).max()
    res = np.linalg.norm(S @ Vh - Vh * l[None, :], axis=0)
    # eigenvalues isolated by more than 1e-3 are resolved to FP64 accuracy.
    # Pairs closer than 1e-4 max|lambda| keep the FP32 solver's mixing, which
    # is bounded by its rounding: residual and eigenvalue error at FP32 level.
    # Inside a cluster (gaps of 1e-9) any orthonormal basis of the cluster's
    # invariant subspace is correct, and that subspace must be exact.
    gaps = (np.abs(l[:, None] - l[None, :]) + np.diag(np.full(n, np.inf))).min(axis=1)
    iso = gaps > 1e-3
    sub_err = 0.0
    for center in (1.0, -1.0, 0.0):
        cols_true = np.abs(lam_true - center) < 1e-6
        cols_got = np.abs(l - center) < 1e-6
        assert cols_true.sum() == cols_got.sum()
        P = V_true[:, cols_true]
        Vc = Vh[:, cols_got]
        sub_err = max(sub_err, np.abs(Vc - P @ (P.T @ Vc)).max())
    print(f"sym eig n={n}: |V^T V - I| {orth:.1e}, |lam - ref| {lam_err:.1e}, residual isolated "
          f"{res[iso].max():.1e} all {res.max():.1e}, cluster subspace {sub_err:.1e}")
    assert orth < 1e-11
    assert lam_err < 1e-7
    assert res[iso].max() < 1e-10
    assert res.max() < 5e-6
    assert sub_err < 1e-9


@pytest.mark.parametrize("weights", [False, True])
@pytest.mark.parametrize("width", [272, 144, 36])
def test_spmm_fullsize(sk, width, weights):
    """X B with X = D^-1/2 A D^-1/2 on the Chung-Lu graph of the benchmark
    (n = 1,000,000, mean degree 20, exponent 2.1; the hubs are the first rows):
    sampled rows, hubs included, against FP64."""
    from oracle import sketchne_oracle as o
    from paper_2110_12782_gb300 import synth
    g = synth.chung_lu(1_000_000, 20.0, 2.1, seed=0)
    G = sk.DeviceGraph.from_numpy(g.row_ptr, g.col_idx)
    deg = torch.empty(g.n, device="cuda")
    vol = torch.empty(1, dtype=torch.float64, device="cuda")
    sk.sne_degrees(G, deg, vol)
    dpow = torch.empty(g.n, device="cuda")
    sk.sne_degree_power(deg, -0.5, dpow)
    rng = np.random.default_rng(width)
    B = rng.standard_normal((g.n, width)).astype(np.float32)
    Y = torch.empty(g.n, width, device="cuda")
    w_nz = None
    if weights:
        w_nz = torch.empty(g.nnz, device="cuda")
        sk.sne_spmm_weights(G, dpow, w_nz)
    sk.sne_spmm(G, dpow, torch.from_numpy(B).cuda(), Y, w_nz=w_nz)
    rows = np.unique(np.concatenate([np.arange(64), np.arange(g.n - 64, g.n),
                                     rng.choice(g.n, 4096, replace=False)]))
    X = o.normalized_operator(o.adjacency(g.row_ptr, g.col_idx, g.n), 0.5)
    ref = X[rows] @ B.astype(np.float64)
    got = Y[torch.as_tensor(rows, device="cuda")].cpu().numpy()
    scale = np.sqrt(abs(X[rows]).power(2) @ (B.astype(np.float64) ** 2)) + 1e-30
    err = float(np.max(np.abs(got - ref) / scale))
    print(f"spmm n=1M width {width}: {err:.2e}")
    assert err < 1e-5


def test_freigs_with_l2_row_split(sk):
    """freigs on a Chung-Lu graph (n = 300,000, mean degree 20, exponent 2.1)
    whose 272-column SpMM operand (326 MB) holds more rows than the SpMM keeps
    in L2 (80 MB), so that its gathers split between the normal and the
    evict-first class: U orthonormal, and the eigenpairs of magnitude 1
    converged (Rayleigh-Ritz residual)."""
    from oracle import sketchne_oracle as o
    from paper_2110_12782_gb300 import synth
    g = synth.chung_lu(300_000, 20.0, 2.1, seed=1)
    G = sk.DeviceGraph.from_numpy(g.row_ptr, g.col_idx)
    k = 256
    p = sk.sne_params_init(128, k, orth=sk.SNE_ORTH_CHOLQR)
    ws = sk.workspace(g.n, g.nnz, p, sk.SNE_WS_FREIGS)
    U = torch.empty(g.n, k, dtype=torch.float32, device="cuda")
    lam = torch.empty(k, dtype=torch.float64, device="cuda")
    sk.sne_freigs(G, p, ws, U, lam)
    assert sk.sne_status(ws) == 0
    eye = torch.eye(k, dtype=torch.float64, device="cuda")
    orth = float((U.T.double() @ U.double() - eye).abs().max())
    Uh = U.cpu().numpy().astype(np.float64)
    lh = lam.cpu().numpy()
    X = o.normalized_operator(o.adjacency(g.row_ptr, g.col_idx, g.n), 0.5)
    res = np.linalg.norm(X @ Uh - Uh * lh[None, :], axis=0)
    top = np.abs(np.abs(lh) - 1.0) < 1e-3
    print(f"freigs n=300k: |U^T U - I| {orth:.1e}, {top.sum()} eigenvalues of magnitude 1, "
          f"their max residual {res[top].max() if top.any() else 0:.1e}, median {np.median(res):.1e}")
    assert orth < 3e-5
    assert top.sum() >= 1 and res[top].max() < 1e-4


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("n", [5, 16, 17, 100, 272, 300])
@pytest.mark.parametrize("pivot", [False, True])
def test_chol_inverse(sk, n, dtype, pivot):
    """M^T A M = I for the Cholesky-QR factor inverse, unpivoted (blocked
    shared-memory kernel, or global memory when A does not fit) and pivoted."""
    rng = np.random.default_rng(n)
    Y = rng.standard_normal((3 * n, n)) * np.exp(rng.uniform(-1, 1, size=n))[None, :]
    A = Y.T @ Y
    Ad = torch.tensor(A, dtype=dtype, device="cuda")
    M = torch.empty_like(Ad)
    ws = sk.chol_inverse_workspace(n, dtype == torch.float64)
    sk.sne_chol_inverse(Ad, M, ws, tol=(1e-12 if pivot else -1.0))
    assert sk.sne_status(ws) == 0
    Mh = M.cpu().numpy().astype(np.float64)
    err = np.abs(Mh.T @ A @ Mh - np.eye(n)).max()
    if not pivot:
        # upper triangular with a positive diagonal and M^T A M = I: M = R^-1
        assert np.allclose(np.tril(Mh, -1), 0)
        assert np.all(np.diag(Mh) > 0)
    tol = 2e-3 if dtype == torch.float32 else 1e-10
    print(f"chol inverse n={n} {dtype} pivot={pivot}: |M^T A M - I| {err:.1e}")
    assert err < tol


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("n,r", [(96, 80), (300, 211)])
def test_chol_inverse_rank_deficient(sk, dtype, n, r):
    """Pivoting stops at the numerical rank; n = 300 in FP64 runs the cluster
    kernel past its early exit (the FP32 kernel is the one-CTA one at both
    sizes, checked at n = 96)."""
    if dtype == torch.float32 and n == 300:
        pytest.skip("FP32 pivoted factor: covered at n = 96")
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((2 * r + 40, r)) @ rng.standard_normal((r, n))
    A = Y.T @ Y
    Ad = torch.tensor(A, dtype=dtype, device="cuda")
    M = torch.empty_like(Ad)
    ws = sk.chol_inverse_workspace(n, dtype == torch.float64)
    sk.sne_chol_inverse(Ad, M, ws, tol=(1e-6 if dtype == torch.float32 else 1e-10))
    assert sk.sne_status(ws) == 0
    Mh = M.cpu().numpy().astype(np.float64)
    G = Mh.T @ A @ Mh
    nz = np.abs(Mh).max(axis=0) > 0
    assert nz.sum() == r
    assert np.abs(G[np.ix_(nz, nz)] - np.eye(r)).max() < (1e-2 if dtype == torch.float32 else 1e-8)
