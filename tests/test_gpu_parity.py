"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: sparse-sign indices and signs bit-exact; FP32 sketches Y, Z within
relative Frobenius error 1e-4; embedding subspace within principal-angle sine
1e-3 on the leading block of singular directions separated from the rest by a
relative gap of at least 1e-2 (Davis-Kahan: only such a block is determined).
"""
import math

import numpy as np
import pytest
import torch

from oracle import sketchne_oracle as o
from paper_2110_12782_gb300 import synth

pytestmark = pytest.mark.gpu

SKETCH_RTOL = 1e-4
ANGLE_TOL = 1e-3
GAP = 1e-2


@pytest.fixture(scope="module")
def sk():
    from paper_2110_12782_gb300 import build
    build.build()
    from paper_2110_12782_gb300 import sketchne
    sketchne.lib()
    return sketchne


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def leading_gap_block(sigma, max_d):
    """Largest j <= max_d with (s_j - s_{j+1}) / s_j >= GAP."""
    best = 0
    for j in range(1, min(max_d, len(sigma) - 1) + 1):
        if (sigma[j - 1] - sigma[j]) / sigma[j - 1] >= GAP:
            best = j
    return best


def dev_graph(sk, g, val=None):
    return sk.DeviceGraph.from_numpy(g.row_ptr, g.col_idx, val)


@pytest.fixture(scope="module")
def c1():
    g = synth.named("sbm4096")
    p = o.Params(k=128, d=32)
    ref = o.embed(g.row_ptr, g.col_idx, g.n, p)
    return g, p, ref


def gpu_params(sk, p: o.Params, **kw):
    pr = p.resolved()
    q = sk.sne_params_init(pr.d, pr.k, q=pr.q, T=pr.T, h=pr.h, l=pr.l, zeta=pr.zeta, s_eig=pr.s_eig,
                           alpha=pr.alpha, b=pr.b, seed=pr.seed,
                           f=sk.SNE_F_TRUNC_LOG if pr.f == "trunc_log" else sk.SNE_F_IDENTITY)
    for key, v in kw.items():
        setattr(q, key, v)
    return q


# ---------------------------------------------------------------- Alg. 3 / randn
@pytest.mark.parametrize("n,cols,zeta,seed,stream", [
    (4096, 80, 8, 0, 2), (4096, 1032, 8, 0, 3), (1_000_000, 272, 8, 7, 2), (50, 300, 8, 3, 3),
    (8, 5, 8, 1, 2), (5, 7, 8, 2, 3), (2_000_000_000, 16, 4, 11, 2), (100, 1, 64, 5, 2)])
def test_sparse_sign_bit_exact(sk, n, cols, zeta, seed, stream):
    ref = o.gen_sparse_sign(n, cols, zeta, seed, stream)
    z = ref.z
    idx = torch.empty(cols * z, dtype=torch.int32, device="cuda")
    sign = torch.empty(cols * z, dtype=torch.int8, device="cuda")
    sk.sne_sparse_sign(n, cols, zeta, seed, stream, idx, sign)
    torch.cuda.synchronize()
    assert np.array_equal(idx.cpu().numpy().reshape(cols, z), ref.idx)
    assert np.array_equal(sign.cpu().numpy().reshape(cols, z), ref.sign)


def test_gaussian_matches_oracle(sk):
    n, cols = 1001, 37
    out = torch.empty(n, cols, dtype=torch.float32, device="cuda")
    sk.sne_gaussian(n, cols, 5, 1, out)
    ref = o.gaussian_matrix(n, cols, 5, 1)
    got = out.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(got - ref) / (1.0 + np.abs(ref))) < 2e-6


# ---------------------------------------------------------------- degrees / SpMM
def test_degrees_and_volume(sk, c1):
    g, _, _ = c1
    G = dev_graph(sk, g)
    deg = torch.empty(g.n, dtype=torch.float32, device="cuda")
    vol = torch.empty(1, dtype=torch.float64, device="cuda")
    sk.sne_degrees(G, deg, vol)
    A = o.adjacency(g.row_ptr, g.col_idx, g.n)
    assert np.array_equal(deg.cpu().numpy(), o.degrees(A).astype(np.float32))
    assert vol.item() == o.volume(A)
    # weighted
    rng = np.random.default_rng(0)
    w = rng.uniform(0.5, 2.0, g.nnz)
    Aw = o.adjacency(g.row_ptr, g.col_idx, g.n, w)
    Aw = (Aw + Aw.T) * 0.5
    val = Aw[np.repeat(np.arange(g.n), np.diff(g.row_ptr)), g.col_idx].A1.astype(np.float32)
    Gw = dev_graph(sk, g, val)
    sk.sne_degrees(Gw, deg, vol)
    ref = o.degrees(o.adjacency(g.row_ptr, g.col_idx, g.n, val.astype(np.float64)))
    assert np.allclose(deg.cpu().numpy(), ref, rtol=1e-6)
    assert abs(vol.item() - ref.sum()) < 1e-6 * ref.sum()


@pytest.mark.parametrize("alpha,width", [(0.5, 144), (0.4, 272), (0.5, 37), (0.35, 80)])
def test_spmm_matches_oracle(sk, c1, alpha, width):
    g, _, _ = c1
    G = dev_graph(sk, g)
    A = o.adjacency(g.row_ptr, g.col_idx, g.n)
    deg = torch.tensor(o.degrees(A), dtype=torch.float32, device="cuda")
    dpow = torch.empty_like(deg)
    sk.sne_degree_power(deg, -alpha, dpow)
    B = np.random.default_rng(1).standard_normal((g.n, width))
    Y = torch.empty(g.n, width, dtype=torch.float32, device="cuda")
    sk.sne_spmm(G, dpow, torch.tensor(B, dtype=torch.float32, device="cuda"), Y)
    ref = o.normalized_operator(A, alpha) @ B
    assert rel(Y.cpu().numpy(), ref) < 2e-6


# ---------------------------------------------------------------- Alg. 4 with oracle factors
def run_sketch(sk, g, p, U, lam, want_E=True):
    pr = p.resolved()
    G = dev_graph(sk, g)
    q = gpu_params(sk, p)
    ws = sk.workspace(g.n, g.nnz, q, sk.SNE_WS_SKETCH)
    Ud = torch.tensor(U, dtype=torch.float32, device="cuda").contiguous()
    ld = torch.tensor(lam, dtype=torch.float64, device="cuda")
    Y = torch.empty(g.n, pr.h, dtype=torch.float32, device="cuda")
    Z = torch.empty(pr.l, pr.l, dtype=torch.float32, device="cuda")
    E = torch.empty(g.n, pr.d, dtype=torch.float32, device="cuda") if want_E else None
    sig = torch.empty(pr.d, dtype=torch.float64, device="cuda") if want_E else None
    sk.sne_sketch_from_factors(G, q, Ud, ld, ws, Y=Y, Z=Z, E=E, sigma=sig)
    st = sk.sne_stats_read(ws)
    assert st.status == 0, sk.sne_error_string(st.status)
    return (Y.cpu().numpy(), Z.cpu().numpy(), None if E is None else E.cpu().numpy(),
            None if sig is None else sig.cpu().numpy(), st)


def test_sketch_Y_Z_E_match_oracle_with_oracle_factors(sk, c1):
    g, p, ref = c1
    Y, Z, E, sig, st = run_sketch(sk, g, p, ref.U_k, ref.lam)
    assert st.v_s == len(ref.sp.S.p) and st.v_o == len(ref.sp.O.p)
    assert rel(Y, ref.sp.Y) < SKETCH_RTOL
    assert rel(Z, ref.sp.Z) < SKETCH_RTOL
    blk = leading_gap_block(ref.sigma, p.resolved().d)
    assert blk >= 1
    assert np.allclose(sig, ref.sigma, rtol=1e-3)
    sines = o.principal_angle_sines(E[:, :blk], ref.E[:, :blk])
    assert sines.max() < ANGLE_TOL
    # E = U_d Sigma^(1/2) with orthonormal U_d
    Ud = E / np.sqrt(sig)[None, :]
    assert np.allclose(Ud.T @ Ud, np.eye(Ud.shape[1]), atol=1e-4)



@pytest.fixture(scope="module")
def c1_alpha04():
    g = synth.named("sbm4096")
    p = o.Params(k=128, d=32, alpha=0.4)
    return g, p, o.embed(g.row_ptr, g.col_idx, g.n, p)


def test_sketch_matches_oracle_at_alpha_04(sk, c1_alpha04):
    """Eq. 11 with a full core: at alpha = 0.4, G = U^T D^(-0.2) U is not the
    identity, so K = G Lambda and the Horner sum are dense k x k matrices.
    Y, Z, the singular values and the 8 block directions of the SBM (relative
    gap 7%) against the oracle, from the oracle's factors."""
    g, p, ref = c1_alpha04
    Y, Z, E, sig, st = run_sketch(sk, g, p, ref.U_k, ref.lam)
    assert st.v_s == len(ref.sp.S.p) and st.v_o == len(ref.sp.O.p)
    assert rel(Y, ref.sp.Y) < SKETCH_RTOL
    assert rel(Z, ref.sp.Z) < SKETCH_RTOL
    assert np.allclose(sig[:8], ref.sigma[:8], rtol=1e-3)
    sines = o.principal_angle_sines(E[:, :8], ref.E[:, :8])
    print(f"alpha 0.4: Y rel {rel(Y, ref.sp.Y):.1e}, Z rel {rel(Z, ref.sp.Z):.1e}, "
          f"8-block sine {sines.max():.1e}")
    assert sines.max() < ANGLE_TOL

def test_identity_f_single_pass_is_exact(sk):
    # f = identity, rank(L'R') = k = h: Y has full column rank and spans
    # range(L'), so the sketch recovers the SVD of L'R' exactly
    g = synth.sbm(1500, 3, 0.05, 0.005, seed=4)
    A = o.adjacency(g.row_ptr, g.col_idx, g.n)
    k = 24
    U, lam = o.freigs(o.normalized_operator(A, 0.5), k, 8, 8, 1)
    p = o.Params(k=k, d=8, h=24, l=200, f="identity", T=3)
    fac = o.netmf_factors(U, lam, o.degrees(A), o.volume(A), 0.5, 3, 1.0)
    M = fac.Lp @ fac.Rp
    sv = np.linalg.svd(M, compute_uv=False)
    _, _, E, sig, _ = run_sketch(sk, g, p, U, lam)
    assert np.allclose(sig, sv[:8], rtol=1e-4)


def test_isolated_vertices_rows_are_zero(sk):
    g0 = synth.sbm(600, 3, 0.05, 0.005, seed=8)
    n = g0.n + 7
    row_ptr = np.concatenate([g0.row_ptr, np.full(7, g0.row_ptr[-1])])
    g = synth.Graph(n=n, row_ptr=row_ptr, col_idx=g0.col_idx)
    p = o.Params(k=16, d=8, q=4, h=24, l=80)
    ref = o.embed(row_ptr, g0.col_idx, n, p)
    Y, Z, E, sig, _ = run_sketch(sk, g, p, ref.U_k, ref.lam)
    assert np.all(Y[g0.n:] == 0) and np.all(E[g0.n:] == 0)
    assert rel(Y, ref.sp.Y) < SKETCH_RTOL


# ---------------------------------------------------------------- Alg. 5 and Alg. 6
@pytest.mark.parametrize("orth", ["eigsvd", "cholqr"])
def test_freigs_matches_oracle(sk, c1, orth):
    g, p, ref = c1
    pr = p.resolved()
    G = dev_graph(sk, g)
    q = gpu_params(sk, p, orth=sk.SNE_ORTH_EIGSVD if orth == "eigsvd" else sk.SNE_ORTH_CHOLQR)
    ws = sk.workspace(g.n, g.nnz, q, sk.SNE_WS_FREIGS)
    U = torch.empty(g.n, pr.k, dtype=torch.float32, device="cuda")
    lam = torch.empty(pr.k, dtype=torch.float64, device="cuda")
    sk.sne_freigs(G, q, ws, U, lam)
    assert sk.sne_status(ws) == 0
    U = U.cpu().numpy().astype(np.float64)
    lam = lam.cpu().numpy()
    assert np.allclose(lam[:8], ref.lam[:8], atol=1e-5)
    assert np.max(np.abs(lam - ref.lam)) < 5e-3
    # the top eigenvector (lambda = 1) and the block of 8 leading ones
    sines = o.principal_angle_sines(U[:, :8], ref.U_k[:, :8])
    assert sines.max() < ANGLE_TOL
    assert np.allclose(U.T @ U, np.eye(pr.k), atol=1e-4)



def test_freigs_matches_oracle_at_alpha_04(sk, c1_alpha04):
    """Alg. 5 on D^-0.4 A D^-0.4 (largest eigenvalue 1.56, not 1): the top
    eigenvalues and the leading 8-dimensional subspace against the oracle's
    freigs from the same Omega."""
    g, p, ref = c1_alpha04
    pr = p.resolved()
    G = dev_graph(sk, g)
    q = gpu_params(sk, p, orth=sk.SNE_ORTH_CHOLQR)
    ws = sk.workspace(g.n, g.nnz, q, sk.SNE_WS_FREIGS)
    U = torch.empty(g.n, pr.k, dtype=torch.float32, device="cuda")
    lam = torch.empty(pr.k, dtype=torch.float64, device="cuda")
    sk.sne_freigs(G, q, ws, U, lam)
    assert sk.sne_status(ws) == 0
    U = U.cpu().numpy().astype(np.float64)
    lam = lam.cpu().numpy()
    scale = abs(ref.lam[0])
    print(f"alpha 0.4 freigs: top-8 eigenvalue error {np.max(np.abs(lam[:8] - ref.lam[:8])):.1e}")
    assert np.allclose(lam[:8], ref.lam[:8], atol=1e-5 * scale)
    assert np.max(np.abs(lam - ref.lam)) < 5e-3 * scale
    assert o.principal_angle_sines(U[:, :8], ref.U_k[:, :8]).max() < ANGLE_TOL
    assert np.allclose(U.T @ U, np.eye(pr.k), atol=1e-4)

def test_embed_matches_oracle(sk, c1):
    g, p, ref = c1
    pr = p.resolved()
    G = dev_graph(sk, g)
    q = gpu_params(sk, p)
    ws = sk.workspace(g.n, g.nnz, q, sk.SNE_WS_EMBED)
    E = torch.empty(g.n, pr.d, dtype=torch.float32, device="cuda")
    sig = torch.empty(pr.d, dtype=torch.float64, device="cuda")
    sk.sne_embed(G, q, ws, E, sig)
    assert sk.sne_status(ws) == 0
    E = E.cpu().numpy()
    sig = sig.cpu().numpy()
    blk = leading_gap_block(ref.sigma, pr.d)
    sines = o.principal_angle_sines(E[:, :blk], ref.E[:, :blk])
    assert sines.max() < ANGLE_TOL, (blk, sines)
    assert np.allclose(sig[:blk], ref.sigma[:blk], rtol=1e-3)


@pytest.mark.parametrize("pinned", [True, False])
def test_embed_host_equals_embed_and_matches_oracle(sk, c1, pinned):
    """sne_embed_host (graph and outputs in host memory, the copies inside the
    call) runs the same kernels on the same data as sne_embed: E and sigma are
    equal bit for bit, and so match the oracle at the stated tolerance."""
    g, p, ref = c1
    pr = p.resolved()
    G = dev_graph(sk, g)
    q = gpu_params(sk, p)
    ws = sk.workspace(g.n, g.nnz, q, sk.SNE_WS_EMBED)
    E = torch.empty(g.n, pr.d, dtype=torch.float32, device="cuda")
    sig = torch.empty(pr.d, dtype=torch.float64, device="cuda")
    sk.sne_embed(G, q, ws, E, sig)
    assert sk.sne_status(ws) == 0
    rp = torch.from_numpy(g.row_ptr)
    ci = torch.from_numpy(g.col_idx)
    Eh = torch.full((g.n, pr.d), float("nan"), dtype=torch.float32)
    sh = torch.full((pr.d,), float("nan"), dtype=torch.float64)
    if pinned:
        rp, ci, Eh, sh = rp.pin_memory(), ci.pin_memory(), Eh.pin_memory(), sh.pin_memory()
    wsh = sk.workspace(g.n, g.nnz, q, sk.SNE_WS_EMBED_HOST)
    sk.sne_embed_host(rp, ci, None, g.n, q, wsh, Eh, sh)
    torch.cuda.synchronize()
    assert sk.sne_status(wsh) == 0
    assert torch.equal(Eh, E.cpu())
    assert torch.equal(sh, sig.cpu())
    blk = leading_gap_block(ref.sigma, pr.d)
    sines = o.principal_angle_sines(Eh.numpy()[:, :blk], ref.E[:, :blk])
    assert sines.max() < ANGLE_TOL, (blk, sines)
    assert np.allclose(sh.numpy()[:blk], ref.sigma[:blk], rtol=1e-3)


# ---------------------------------------------------------------- validation
def test_validate_flags_bad_graphs(sk):
    g = synth.sbm(300, 3, 0.05, 0.01, seed=2)
    G = dev_graph(sk, g)
    ws = torch.zeros(4096, dtype=torch.uint8, device="cuda")
    sk.sne_status_reset(ws)
    sk.sne_validate_csr(G, ws)
    assert sk.sne_status(ws) == 0
    # drop the mirror of one edge: asymmetric
    col = g.col_idx.copy()
    i = int(np.argmax(np.diff(g.row_ptr) > 0))
    col[g.row_ptr[i]] = (col[g.row_ptr[i]] + 1) % g.n if col[g.row_ptr[i]] + 1 != i else (i + 2) % g.n
    Gb = sk.DeviceGraph.from_numpy(g.row_ptr, col)
    sk.sne_status_reset(ws)
    sk.sne_validate_csr(Gb, ws)
    assert sk.sne_status(ws) == sk.SNE_ERR_GRAPH
    # column index out of range
    col = g.col_idx.copy()
    col[-1] = g.n + 5
    Gc = sk.DeviceGraph.from_numpy(g.row_ptr, col)
    sk.sne_status_reset(ws)
    sk.sne_validate_csr(Gc, ws)
    assert sk.sne_status(ws) == sk.SNE_ERR_GRAPH


@pytest.fixture(scope="module")
def cl_k256():
    """Chung-Lu n = 30,000 (mean degree 20, exponent 2.1) at the benchmark's
    k = 256, d = 128, h = 272, l = 1128: several row blocks, 2176 sketch
    columns and ~7,800 unique O rows, small enough for the dense oracle."""
    g = synth.chung_lu(30_000, 20.0, 2.1, seed=3)
    p = o.Params(k=256, d=128, q=3)
    A = o.adjacency(g.row_ptr, g.col_idx, g.n)
    U, lam = o.freigs(o.normalized_operator(A, 0.5), p.k, p.q, p.s_eig, p.seed)
    U = U.astype(np.float32).astype(np.float64)
    pr = p.resolved()
    fac = o.netmf_factors(U, lam, o.degrees(A), o.volume(A), pr.alpha, pr.T, pr.b)
    S = o.gen_sparse_sign(g.n, pr.h, pr.zeta, pr.seed, o.STREAM_S)
    O = o.gen_sparse_sign(g.n, pr.l, pr.zeta, pr.seed, o.STREAM_O)
    return g, p, U, lam, o.sketch_Y_rows(fac.Lp, fac.Rp, S), o.sketch_Z(fac.Lp, fac.Rp, O), S, O


def test_sketch_k256_matches_oracle(sk, cl_k256):
    g, p, U, lam, Yref, Zref, S, O = cl_k256
    Y, Z, _, _, st = run_sketch(sk, g, p, U, lam, want_E=False)
    assert st.v_s == len(S.p) and st.v_o == len(O.p)
    ey, ez = rel(Y, Yref), rel(Z, Zref)
    print(f"k=256 sketch: Y rel {ey:.2e}, Z rel {ez:.2e}")
    assert ey < SKETCH_RTOL
    assert ez < SKETCH_RTOL


def test_rank_deficient_sketch_matches_oracle(sk):
    """40 cliques of 4..8 vertices and 40 single edges, k = 120 = the dimension
    of the |lambda| = 1 eigenspace: U_k spans the component indicators, L'R' is
    constant on every component, and trunc_log(L'R') has rank 80 < h = 96.  The
    sketch QR and the least-squares solves must still reproduce the oracle (whose
    Householder QR and lstsq are rank-revealing)."""
    edges, off = [], 0
    for i in range(40):
        m = 4 + i % 5
        edges += [(off + a, off + b) for a in range(m) for b in range(a + 1, m)]
        off += m
    for i in range(40):
        edges.append((off, off + 1))
        off += 2
    g = synth.from_edges(off, np.array(edges))
    p = o.Params(k=120, d=40, h=96, l=200)
    ref = o.embed(g.row_ptr, g.col_idx, g.n, p)
    assert np.linalg.matrix_rank(ref.sp.Y) < p.h
    for orth in ("cholqr", "eigsvd"):
        q = gpu_params(sk, p, orth=sk.SNE_ORTH_CHOLQR if orth == "cholqr" else sk.SNE_ORTH_EIGSVD)
        G = dev_graph(sk, g)
        ws = sk.workspace(g.n, g.nnz, q, sk.SNE_WS_EMBED)
        E = torch.empty(g.n, p.d, dtype=torch.float32, device="cuda")
        sig = torch.empty(p.d, dtype=torch.float64, device="cuda")
        sk.sne_embed(G, q, ws, E, sig)
        st = sk.sne_stats_read(ws)
        assert st.status == 0, (orth, sk.sne_error_string(st.status), st.where)
        s = sig.cpu().numpy()
        assert np.allclose(s, ref.sigma, rtol=1e-4), (orth, s[:8], ref.sigma[:8])
        Eh = E.cpu().numpy()
        for blk in (8, 16, 24, 32):
            sines = o.principal_angle_sines(Eh[:, :blk], ref.E[:, :blk])
            assert sines.max() < ANGLE_TOL, (orth, blk, sines.max())
