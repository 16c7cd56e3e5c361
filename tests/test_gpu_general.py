"""The general single-pass SVD of Eqs. 5-10 (rectangular f(L R), co-range
sketch K = f(LR)^T C) through the C ABI against the FP64 oracle with the same
sparse-sign matrices.

* f = identity and rank(LR) = k <= h: Eq. 10 is exact, so the singular values
  equal those of LR (numpy SVD) up to the FP32 sketches (relative 1e-5) and U,
  V span the exact singular subspaces (principal-angle sines 1e-4 on the
  leading block with a relative gap of at least 1e-2).
* f = trunc_log of a rectangular product (n != m): singular values within
  1e-4 and sines within 1e-3 of the oracle's on the gapped leading block.
* (slow) n = 200,000 by m = 100,000, k = 64.
"""
import numpy as np
import pytest
import torch

from oracle import sketchne_oracle as o

pytestmark = pytest.mark.gpu
GAP = 1e-2


@pytest.fixture(scope="module")
def sk():
    from paper_2110_12782_gb300 import build
    build.build()
    from paper_2110_12782_gb300 import sketchne
    sketchne.lib()
    return sketchne


def leading_gap_block(sigma, max_d):
    best = 0
    for j in range(1, min(max_d, len(sigma) - 1) + 1):
        if (sigma[j - 1] - sigma[j]) / sigma[j - 1] >= GAP:
            best = j
    return best


def run(sk, L, Rt, d, h, l, f, seed=0):
    p = sk.sne_params_init(d, 8)
    p.h, p.l, p.seed = h, l, seed
    p.f = sk.SNE_F_TRUNC_LOG if f == "trunc_log" else sk.SNE_F_IDENTITY
    Ld = torch.from_numpy(L.astype(np.float32)).cuda()
    Rd = torch.from_numpy(Rt.astype(np.float32)).cuda()
    n, m = L.shape[0], Rt.shape[0]
    ws = sk.single_pass_svd_workspace(n, m, L.shape[1], p)
    U = torch.empty(n, d, dtype=torch.float32, device="cuda")
    V = torch.empty(m, d, dtype=torch.float32, device="cuda")
    sig = torch.empty(d, dtype=torch.float64, device="cuda")
    sk.sne_single_pass_svd(Ld, Rd, p, ws, U, sig, V)
    sk.check_status(ws, "single-pass svd")
    return (U.cpu().double().numpy(), sig.cpu().numpy(), V.cpu().double().numpy())


def compare(U, s, V, rU, rs, rV, d, stol, atol):
    blk = leading_gap_block(rs, d)
    assert blk >= 1
    srel = np.max(np.abs(s[:blk] - rs[:blk]) / rs[:blk])
    su = o.principal_angle_sines(U[:, :blk], rU[:, :blk]).max()
    sv = o.principal_angle_sines(V[:, :blk], rV[:, :blk]).max()
    return blk, srel, su, sv


@pytest.mark.parametrize("n,m,k", [(6000, 4000, 24), (5000, 5000, 40)])
def test_identity_low_rank_is_recovered(sk, n, m, k):
    rng = np.random.default_rng(k)
    L = rng.standard_normal((n, k)).astype(np.float32)
    Rt = (rng.standard_normal((m, k)) * np.linspace(1.0, 0.1, k)[None, :]).astype(np.float32)
    U, s, V = run(sk, L, Rt, d=k, h=k + 8, l=k + 200, f="identity")
    Uf, sf, Vft = np.linalg.svd(L.astype(np.float64) @ Rt.astype(np.float64).T, full_matrices=False)
    blk, srel, su, sv = compare(U, s, V, Uf, sf[:k], Vft.T, k, 1e-5, 1e-4)
    print(f"identity n={n} m={m} k={k}: block {blk}, sigma rel {srel:.1e}, sines U {su:.1e} V {sv:.1e}")
    assert srel < 1e-5 and su < 1e-4 and sv < 1e-4


def trunc_log_case(n, m, k, seed):
    """x_ij = 1 + 0.9 <u_i, v_j> with Gaussian u, v on geometrically falling
    scales: half of the entries are truncated and the spectrum of trunc_log(x)
    falls off with clear gaps."""
    rng = np.random.default_rng(seed)
    sc = np.geomspace(1.0, 0.05, k - 1)
    u = rng.standard_normal((n, k - 1)) * sc
    v = rng.standard_normal((m, k - 1)) * sc
    L = np.hstack([np.ones((n, 1)), 0.9 * u]).astype(np.float32)
    Rt = np.hstack([np.ones((m, 1)), v]).astype(np.float32)
    return L, Rt


@pytest.mark.parametrize("n,m,k,d", [(8000, 3000, 16, 8), (3000, 8000, 32, 16)])
def test_trunc_log_matches_oracle(sk, n, m, k, d):
    L, Rt = trunc_log_case(n, m, k, seed=n + m)
    h, l = 2 * d + 16, d + 400
    U, s, V = run(sk, L, Rt, d, h, l, "trunc_log", seed=2)
    ref = o.single_pass_svd_general(L.astype(np.float64), Rt.astype(np.float64), d, h, l, 8, 2,
                                    o.trunc_log)
    blk, srel, su, sv = compare(U, s, V, ref.U, ref.sigma, ref.V, d, 1e-4, 1e-3)
    print(f"trunc_log n={n} m={m} k={k}: block {blk}, sigma rel {srel:.1e}, sines U {su:.1e} V {sv:.1e}")
    assert srel < 1e-4 and su < 1e-3 and sv < 1e-3


@pytest.mark.slow
def test_trunc_log_large(sk):
    n, m, k, d = 200_000, 100_000, 64, 32
    L, Rt = trunc_log_case(n, m, k, seed=11)
    h, l = 2 * d + 16, d + 600
    U, s, V = run(sk, L, Rt, d, h, l, "trunc_log", seed=4)
    ref = o.single_pass_svd_general(L.astype(np.float64), Rt.astype(np.float64), d, h, l, 8, 4,
                                    o.trunc_log)
    blk, srel, su, sv = compare(U, s, V, ref.U, ref.sigma, ref.V, d, 1e-4, 1e-3)
    print(f"trunc_log n={n} m={m}: block {blk}, sigma rel {srel:.1e}, sines U {su:.1e} V {sv:.1e}")
    assert srel < 1e-4 and su < 1e-3 and sv < 1e-3
