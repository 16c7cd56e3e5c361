"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
test vectors, closed forms, textbook spectra, exactness statements of the
paper, library routines that reach the same result by another algorithm, and
brute force on tiny inputs.  CPU only.
"""
import math
import os

import numpy as np
import pytest
import scipy.stats

from oracle import sketchne_oracle as o
from paper_2110_12782_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _dense(g):
    return o.adjacency(g.row_ptr, g.col_idx, g.n).toarray()


# ---------------------------------------------------------------- random numbers
def test_splitmix64_published_vectors():
    want = [int(line, 16) for line in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if line.strip() and not line.startswith("#")]
    got = [o.splitmix64_output(0, i) for i in range(1, len(want) + 1)]
    assert got == want
    # the vectorised form used for Omega agrees with the scalar one
    key = o.stream_key(7, 1)
    ctr = np.arange(100, dtype=np.uint64)
    assert [int(x) for x in o.draw_np(key, ctr)] == [o.draw(key, int(c)) for c in range(100)]


def test_lemire_bounded_definition_and_uniformity():
    key = o.stream_key(3, 2)
    n = 7
    counts = np.zeros(n)
    ctr = 0
    for _ in range(14000):
        x = o.draw(key, ctr)
        v, ctr2 = o.bounded(key, ctr, n)
        if ctr2 == ctr + 1:  # not rejected: the value is floor(x * n / 2^64)
            assert v == (x * n) >> 64
        ctr = ctr2
        counts[v] += 1
    chi2 = ((counts - counts.mean()) ** 2 / counts.mean()).sum()
    assert scipy.stats.chi2.sf(chi2, n - 1) > 1e-4
    # a bound just above 2^63 rejects about half of the draws
    big = (1 << 63) + 1
    ctr, rejected = 0, 0
    for _ in range(400):
        v, ctr2 = o.bounded(o.stream_key(1, 1), ctr, big)
        rejected += ctr2 - ctr - 1
        assert 0 <= v < big
        ctr = ctr2
    assert 100 < rejected < 800


def test_sparse_sign_structure():
    for n, cols, zeta in [(1000, 50, 8), (20, 30, 8), (5, 4, 8), (8, 3, 8), (100000, 40, 4)]:
        S = o.gen_sparse_sign(n, cols, zeta, seed=11, stream=2)
        z = min(n, zeta)
        assert S.idx.shape == (cols, z)
        for j in range(cols):
            assert len(set(S.idx[j].tolist())) == z
        assert S.idx.min() >= 0 and S.idx.max() < n
        assert set(np.unique(S.sign).tolist()) <= {-1, 1}
        assert np.array_equal(S.p, np.array(sorted(set(S.idx.ravel().tolist()))))
        D = S.dense()
        assert np.count_nonzero(D) == cols * z
        assert np.allclose(np.abs(D[D != 0]), 1 / math.sqrt(z))
    # deterministic, stream-dependent
    a = o.gen_sparse_sign(1000, 20, 8, 5, 2)
    b = o.gen_sparse_sign(1000, 20, 8, 5, 2)
    c = o.gen_sparse_sign(1000, 20, 8, 5, 3)
    assert np.array_equal(a.idx, b.idx) and np.array_equal(a.sign, b.sign)
    assert not np.array_equal(a.idx, c.idx)


def test_sparse_sign_uniform_rows_and_signs():
    n = 50
    S = o.gen_sparse_sign(n, 2000, 8, seed=1, stream=3)
    counts = np.bincount(S.idx.ravel(), minlength=n)
    chi2 = ((counts - counts.mean()) ** 2 / counts.mean()).sum()
    assert scipy.stats.chi2.sf(chi2, n - 1) > 1e-4
    plus = (S.sign == 1).sum()
    assert abs(plus - S.sign.size / 2) < 4 * math.sqrt(S.sign.size / 4)


def test_gaussian_omega_distribution_and_slicing():
    G = o.gaussian_matrix(4000, 37, seed=2)
    x = G.ravel()
    assert scipy.stats.kstest(x, "norm").pvalue > 1e-4
    assert abs(x.mean()) < 4 / math.sqrt(x.size)
    assert abs(x.var() - 1) < 4 * math.sqrt(2 / x.size)
    # rows are independent of how the matrix is chunked
    part = o.gaussian_matrix(4000, 37, seed=2, row0=1234, rows=77)
    assert np.array_equal(part, G[1234:1311])


# ---------------------------------------------------------------- graph quantities
def test_degrees_volume_star():
    g = synth.from_edges(6, [(0, i) for i in range(1, 6)])
    A = o.adjacency(g.row_ptr, g.col_idx, g.n)
    assert np.array_equal(o.degrees(A), [5, 1, 1, 1, 1, 1])
    assert o.volume(A) == 10


def test_normalized_operator_textbook_spectra():
    # K_n: D^-1/2 A D^-1/2 = (J - I)/(n-1): eigenvalues 1 (once), -1/(n-1)
    n = 9
    g = synth.complete_graph(n)
    X = o.normalized_operator(o.adjacency(g.row_ptr, g.col_idx, n), 0.5).toarray()
    ev = np.sort(np.linalg.eigvalsh(X))
    assert np.allclose(ev, np.r_[np.full(n - 1, -1 / (n - 1)), 1.0], atol=1e-13)
    # connected graph: top eigenvalue 1 with eigenvector D^1/2 1
    g = synth.sbm(300, 3, 0.2, 0.05, seed=4)
    A = o.adjacency(g.row_ptr, g.col_idx, g.n)
    X = o.normalized_operator(A, 0.5).toarray()
    ev, V = np.linalg.eigh(X)
    assert abs(ev[-1] - 1) < 1e-12 and ev[0] >= -1 - 1e-12
    u = np.sqrt(o.degrees(A))
    u /= np.linalg.norm(u)
    assert abs(abs(V[:, -1] @ u) - 1) < 1e-10


# ---------------------------------------------------------------- Alg. 5
def test_eigsvd_is_an_orthonormal_basis_of_range():
    rng = np.random.default_rng(0)
    Y = rng.standard_normal((500, 30)) @ np.diag(np.logspace(0, -3, 30))
    Q, S, V = o.eigsvd(Y)
    assert np.allclose(Q.T @ Q, np.eye(30), atol=1e-9)
    U, sv, _ = np.linalg.svd(Y, full_matrices=False)
    assert np.allclose(np.sort(S), np.sort(sv), rtol=1e-9)
    assert np.allclose(Q @ Q.T, U @ U.T, atol=1e-9)


def test_freigs_exact_on_bipartite_union():
    # each K_{a,b} contributes eigenvalues +1 and -1 of D^-1/2 A D^-1/2, all
    # other eigenvalues are 0; the 2c-dimensional eigenspace is found exactly.
    # (k + s must not exceed rank(X) = 2c: eigSVD divides by the square roots
    # of the Gram eigenvalues, which are 0 beyond the rank.)
    parts = [(3, 5), (4, 4), (2, 7), (6, 3), (5, 5), (3, 9)]
    g = synth.complete_bipartite_union(parts)
    X = o.normalized_operator(o.adjacency(g.row_ptr, g.col_idx, g.n), 0.5)
    k = 2 * len(parts)
    U, lam = o.freigs(X, k, q=2, s=0, seed=1)
    assert np.allclose(np.abs(lam), 1.0, atol=1e-10)
    assert (lam > 0).sum() == len(parts)
    assert np.allclose(X @ U, U * lam[None, :], atol=1e-9)
    assert np.allclose(U.T @ U, np.eye(k), atol=1e-9)


def test_freigs_matches_dense_eigh_on_leading_eigenvalues():
    g = synth.sbm(600, 4, 0.08, 0.005, seed=3)
    A = o.adjacency(g.row_ptr, g.col_idx, g.n)
    for alpha in (0.5, 0.4):
        X = o.normalized_operator(A, alpha)
        ev = np.linalg.eigvalsh(X.toarray())
        ev = ev[np.argsort(-np.abs(ev))]
        U, lam = o.freigs(X, 16, q=30, s=16, seed=2)
        # the four community eigenvalues are well separated from the bulk
        assert np.allclose(lam[:4], ev[:4], rtol=1e-8)
        assert np.all(np.abs(np.abs(lam) - np.abs(ev[:16])) < 0.05)


def test_freigs_with_householder_qr_gives_same_eigenvalues():
    # the span after each step does not depend on the orthonormal basis chosen
    g = synth.sbm(400, 4, 0.1, 0.01, seed=5)
    X = o.normalized_operator(o.adjacency(g.row_ptr, g.col_idx, g.n), 0.5)
    k, s, q = 10, 6, 4
    U, lam = o.freigs(X, k, q, s, seed=9)
    Om = o.gaussian_matrix(g.n, k + s, 9)
    Q, _ = np.linalg.qr(X @ Om)
    for _ in range(q):
        Q, _ = np.linalg.qr(X @ (X @ Q))
    Sred = Q.T @ (X @ Q)
    ev = np.linalg.eigvalsh(0.5 * (Sred + Sred.T))
    ev = ev[np.argsort(-np.abs(ev))][:k]
    assert np.allclose(lam, ev, rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------- Eq. 1 / Eq. 2 / Eq. 11
def test_netmf_matrix_closed_form_complete_graph():
    for n, T, b in [(5, 10, 1.0), (12, 3, 2.0)]:
        M = o.netmf_matrix_dense(_dense(synth.complete_graph(n)), T, b)
        mu = -1.0 / (n - 1)
        off = sum(1 - mu ** r for r in range(1, T + 1)) / (b * T)
        diag = sum(1 + (n - 1) * mu ** r for r in range(1, T + 1)) / (b * T)
        assert np.allclose(M[~np.eye(n, dtype=bool)], off, rtol=1e-13)
        assert np.allclose(np.diag(M), diag, rtol=1e-13)
    # n=5, T=10, b=1 puts every off-diagonal entry just above the threshold 1
    M = o.netmf_matrix_dense(_dense(synth.complete_graph(5)), 10, 1.0)
    assert 1.0 < M[0, 1] < 1.05 and o.trunc_log(M)[0, 1] > 0


@pytest.mark.parametrize("alpha", [0.5, 0.4, 0.35])
def test_eq11_equals_eq1_at_full_rank(alpha):
    # with all n eigenpairs of D^-a A D^-a, L'R' of Eq. 11 is exactly Eq. 1's matrix
    g = synth.sbm(60, 2, 0.4, 0.1, seed=1)
    Ad = _dense(g)
    A = o.adjacency(g.row_ptr, g.col_idx, g.n)
    assert (o.degrees(A) > 0).all()
    X = o.normalized_operator(A, alpha).toarray()
    lam, U = np.linalg.eigh(X)
    fac = o.netmf_factors(U, lam, o.degrees(A), o.volume(A), alpha, T=5, b=1.0)
    M = o.netmf_matrix_dense(Ad, T=5, b=1.0)
    assert np.allclose(fac.Lp @ fac.Rp, M, rtol=1e-9, atol=1e-9 * np.abs(M).max())
    if alpha == 0.5:
        M2 = o.netmf_eq2_dense(Ad, U, lam, T=5, b=1.0)
        assert np.allclose(M2, M, rtol=1e-9, atol=1e-9 * np.abs(M).max())


def test_top_eigenpair_contributes_exactly_one_over_b():
    # alpha = 1/2: lambda_1 = 1, u_1 ~ D^1/2 1 give vol/(bT) d_i^-1/2 u_1i T u_1j d_j^-1/2 = 1/b
    g = synth.sbm(200, 2, 0.2, 0.05, seed=2)
    A = o.adjacency(g.row_ptr, g.col_idx, g.n)
    deg = o.degrees(A)
    u = np.sqrt(deg) / np.linalg.norm(np.sqrt(deg))
    for b in (1.0, 3.0):
        fac = o.netmf_factors(u[:, None], np.array([1.0]), deg, o.volume(A), 0.5, T=10, b=b)
        assert np.allclose(fac.Lp @ fac.Rp, 1.0 / b, rtol=1e-12)


def test_trunc_log_cases_and_lipschitz():
    x = np.array([-3.0, 0.0, 0.5, 1.0, math.e, math.e ** 2])
    assert np.allclose(o.trunc_log(x), [0, 0, 0, 0, 1, 2])
    rng = np.random.default_rng(1)
    a, b = rng.uniform(-2, 20, 10000), rng.uniform(-2, 20, 10000)
    # trunc_log is 1-Lipschitz where both arguments are >= 1 or the log is flat
    lhs = np.abs(o.trunc_log(a) - o.trunc_log(b))
    assert np.all(lhs <= np.abs(np.maximum(a, 1) - np.maximum(b, 1)) + 1e-15)


# ---------------------------------------------------------------- Alg. 4
def _small_factors(n=300, k=24, seed=3, alpha=0.5):
    g = synth.sbm(n, 3, 0.1, 0.01, seed=seed)
    A = o.adjacency(g.row_ptr, g.col_idx, g.n)
    X = o.normalized_operator(A, alpha)
    U, lam = o.freigs(X, k, q=5, s=8, seed=seed)
    return g, o.netmf_factors(U, lam, o.degrees(A), o.volume(A), alpha, 10, 1.0)


def test_eq4_column_sampling_is_exact():
    g, fac = _small_factors()
    S = o.gen_sparse_sign(g.n, 40, 8, seed=4, stream=2)
    Y = o.sketch_Y(fac.Lp, fac.Rp, S, row_block=64)
    Yd = o.trunc_log(fac.Lp @ fac.Rp) @ S.dense()
    assert np.linalg.norm(Y - Yd) <= 1e-12 * np.linalg.norm(Yd)
    assert len(S.p) < g.n


def test_z_core_is_exact():
    g, fac = _small_factors()
    O = o.gen_sparse_sign(g.n, 70, 8, seed=4, stream=3)
    Z = o.sketch_Z(fac.Lp, fac.Rp, O)
    Od = O.dense()
    Zd = Od.T @ o.trunc_log(fac.Lp @ fac.Rp) @ Od
    assert np.linalg.norm(Z - Zd) <= 1e-12 * np.linalg.norm(Zd)
    assert np.allclose(Z, Z.T, rtol=0, atol=1e-12 * np.abs(Z).max())


def test_single_pass_exact_for_identity_f():
    # f = identity and rank(L'R') = k <= h: Alg. 4 recovers the SVD exactly
    g, fac = _small_factors(k=12)
    M = fac.Lp @ fac.Rp
    d = 8
    res = o.single_pass_svd(fac.Lp, fac.Rp, d, h=20, l=120, zeta=8, seed=6, f=o.identity)
    U, sv, _ = np.linalg.svd(M)
    assert np.allclose(res.sigma, sv[:d], rtol=1e-8)
    gap_ok = [i for i in range(1, d + 1) if i == d or (sv[i - 1] - sv[i]) > 1e-3 * sv[0]]
    dd = gap_ok[-1]
    sines = o.principal_angle_sines(res.U[:, :dd], U[:, :dd])
    assert sines.max() < 1e-6


def test_single_pass_invariant_to_sign_scale_and_w_symmetric():
    g, fac = _small_factors()
    a = o.single_pass_svd(fac.Lp, fac.Rp, 8, 32, 150, 8, seed=2)
    b = o.single_pass_svd(fac.Lp, fac.Rp, 8, 32, 150, 8, seed=2, sign_scale=1.0)
    assert np.allclose(a.sigma, b.sigma, rtol=1e-10)
    assert o.principal_angle_sines(a.U, b.U).max() < 1e-6  # sqrt(1-cos^2) floor ~1e-8
    assert np.linalg.norm(a.W - a.W.T) <= 1e-12 * np.linalg.norm(a.W)


def test_graph_without_edges_is_rejected():
    # Eq. 1 divides by vol(G) = sum of degrees; with no edges it is undefined
    n = 50
    with pytest.raises(ValueError, match="vol"):
        o.embed(np.zeros(n + 1, dtype=np.int64), np.zeros(0, dtype=np.int32), n,
                o.Params(k=8, d=4, q=2, h=12, l=40))


def test_isolated_vertices_have_zero_rows():
    g0 = synth.sbm(200, 2, 0.2, 0.02, seed=8)
    # append 5 isolated vertices
    n = g0.n + 5
    row_ptr = np.concatenate([g0.row_ptr, np.full(5, g0.row_ptr[-1])])
    p = o.Params(k=16, d=8, q=4, h=24, l=80)
    r = o.embed(row_ptr, g0.col_idx, n, p)
    assert np.all(r.sp.Y[g0.n:] == 0)
    assert np.all(r.E[g0.n:] == 0)
    assert np.all(r.U_k[g0.n:] == 0)


def test_theorem1_bound_holds():
    g = synth.sbm(400, 4, 0.08, 0.01, seed=12)
    A = o.adjacency(g.row_ptr, g.col_idx, g.n)
    deg = o.degrees(A)
    assert (deg > 0).all()
    for alpha in (0.5, 0.45):
        X = o.normalized_operator(A, alpha)
        k = 32
        U, lam = o.freigs(X, k, q=10, s=16, seed=1)
        fac = o.netmf_factors(U, lam, deg, o.volume(A), alpha, 10, 1.0)
        lhs = np.linalg.norm(o.trunc_log(o.netmf_matrix_dense(A.toarray(), 10, 1.0))
                             - o.trunc_log(fac.Lp @ fac.Rp))
        ev = np.sort(np.abs(np.linalg.eigvalsh(X.toarray())))[::-1]
        assert lhs <= o.theorem1_bound(ev, k, deg, o.volume(A), g.n, alpha, 10, 1.0)


def test_theorem1_bound_hand_values():
    """The right-hand side of Theorem 1 at two tiny graphs, worked by hand
    from the known spectra (not from the oracle's eigensolver):

    * K_4, alpha = 1/2, k = 1, T = 2, b = 1: D^-1/2 A D^-1/2 has eigenvalues
      1 and -1/3 (three times), so the tail is sqrt(3 / 9) = 1/sqrt(3); every
      degree is 3, vol = 12, c = n (d_max/d_min)^0 = 4.  Then
      (c^T - 1)(1 + n/(c-1)) - nT = 15 * 7/3 - 8 = 27,
      B = 27 * 12 / sqrt(3) = 108 sqrt(3), and the bound is
      d_min^0 B / ((c - 1) b T) = 108 sqrt(3) / 6 = 18 sqrt(3).
    * K_{2,4}, alpha = 1/4, k = 1, T = 2, b = 1: D^-a A D^-a is
      (2*4)^(-1/4) times the all-ones biadjacency block, eigenvalues
      +-(2*4)^(1/2 - 1/4) = +-8^(1/4) and 0, so the tail is 8^(1/4); degrees 4
      (twice) and 2 (four times), vol = 16, d_min^(-1+2a) = 2^(-1/2),
      c = 6 (4/2)^(1/2) = 6 sqrt(2), c^2 = 72.  The bound is
      2^(-1/2) 8^(1/4) (71 (1 + 6/(6 sqrt(2) - 1)) - 12) 16 / ((6 sqrt(2) - 1) 2)
      = 147.32...
    A dropped (c - 1), a wrong power of c or of d_min, or a missing vol moves
    either value."""
    deg = np.full(4, 3.0)
    ev = np.array([1.0, 1 / 3, 1 / 3, 1 / 3])
    assert math.isclose(o.theorem1_bound(ev, 1, deg, 12.0, 4, 0.5, 2, 1.0), 18 * math.sqrt(3),
                        rel_tol=1e-12)
    deg = np.array([4.0, 4.0, 2.0, 2.0, 2.0, 2.0])
    ev = np.array([8 ** 0.25, 8 ** 0.25, 0, 0, 0, 0])
    r2 = math.sqrt(2.0)
    want = 2 ** -0.5 * 8 ** 0.25 * (71 * (1 + 6 / (6 * r2 - 1)) - 12) * 16 / ((6 * r2 - 1) * 2)
    assert math.isclose(want, 147.32, rel_tol=1e-4)
    assert math.isclose(o.theorem1_bound(ev, 1, deg, 16.0, 6, 0.25, 2, 1.0), want, rel_tol=1e-12)
    # the spectra used above are those of the graphs
    for g, alpha, spec in ((synth.complete_graph(4), 0.5, [1.0, -1 / 3, -1 / 3, -1 / 3]),
                           (synth.complete_bipartite_union([(2, 4)]), 0.25,
                            [8 ** 0.25, -(8 ** 0.25), 0, 0, 0, 0])):
        A = o.adjacency(g.row_ptr, g.col_idx, g.n)
        X = o.normalized_operator(A, alpha).toarray()
        assert np.allclose(np.sort(np.linalg.eigvalsh(X)), np.sort(spec), atol=1e-12)


def test_embedding_dominant_subspace_matches_dense_svd():
    # the four block directions of trunc_log(L'R') are separated from the rest
    # by a wide gap; the single-pass sketch recovers them (randomized, so loose
    # bounds), and its rank-d projection is close to the Eckart-Young optimum
    g = synth.sbm(800, 4, 0.05, 0.005, seed=1)
    p = o.Params(k=32, d=8, q=10, h=64, l=600)
    r = o.embed(g.row_ptr, g.col_idx, g.n, p)
    F = o.trunc_log(r.factors.Lp @ r.factors.Rp)
    U, sv, _ = np.linalg.svd(F)
    assert sv[3] > 2 * sv[4]
    assert np.all(np.abs(r.sigma[:4] - sv[:4]) < 2e-2 * sv[:4])
    assert o.principal_angle_sines(r.sp.U[:, :4], U[:, :4]).max() < 0.2
    Ud = r.sp.U
    resid = np.linalg.norm(F - Ud @ (Ud.T @ F))
    optimum = math.sqrt(float(np.sum(sv[8:] ** 2)))
    assert optimum <= resid <= 1.1 * optimum


def test_principal_angle_sines_known_angles():
    # span{e1, e2} against span{e1, cos(t) e2 + sin(t) e3}: principal angles
    # (t, 0) by construction; the spans do not depend on the bases chosen
    rng = np.random.default_rng(11)
    n, t = 7, 0.3
    E = np.eye(n)
    A = E[:, :2]
    B = np.stack([E[:, 0], np.cos(t) * E[:, 1] + np.sin(t) * E[:, 2]], axis=1)
    s = o.principal_angle_sines(A @ rng.standard_normal((2, 2)), B @ rng.standard_normal((2, 2)))
    assert np.allclose(s, [np.sin(t), 0.0], atol=1e-7)
    # orthogonal spans: every angle is pi/2; a span against itself: 0
    assert np.allclose(o.principal_angle_sines(E[:, :3], E[:, 3:6]), 1.0)
    assert o.principal_angle_sines(A, A[:, ::-1]).max() < 1e-7
    # a rotation by t in the (e1, e4) plane and by 2t in the (e2, e5) plane
    C = np.stack([np.cos(t) * E[:, 0] + np.sin(t) * E[:, 3],
                  np.cos(2 * t) * E[:, 1] + np.sin(2 * t) * E[:, 4]], axis=1)
    assert np.allclose(o.principal_angle_sines(A, C), [np.sin(2 * t), np.sin(t)], atol=1e-12)


def test_sketch_rows_equal_dense_definition():
    g, fac = _small_factors()
    S = o.gen_sparse_sign(g.n, 40, 8, seed=5, stream=2)
    rows = np.array([0, 3, 17, g.n - 1])
    got = o.sketch_Y_rows(fac.Lp[rows], fac.Rp, S)
    ref = o.trunc_log(fac.Lp[rows] @ fac.Rp) @ S.dense()
    assert np.linalg.norm(got - ref) <= 1e-12 * np.linalg.norm(ref)


def test_lemire_rejection_leaves_exactly_one_preimage(monkeypatch):
    """Lemire's theorem for bounds n > 2^63: every output v in [0, n) keeps
    exactly floor(2^64 / n) = 1 accepted 64-bit draw.  The draws mapping to v
    (x with floor(x n / 2^64) = v) are fed to the oracle one at a time and the
    accepted ones counted, so a wrong rejection threshold or a missing rejection
    leaves some v with 0 or 2 preimages."""
    rng = np.random.default_rng(5)
    for n in [(1 << 63) + 1, (1 << 63) + 12345, (1 << 64) - 5, 3 << 62]:
        assert (1 << 64) // n == 1
        vs = [0, 1, 2, n - 1, n - 2] + [int(v) for v in rng.integers(0, n, size=60, dtype=np.uint64)
                                        if int(v) < n]
        for v in vs:
            lo_x = -((-v << 64) // n)                 # ceil(v 2^64 / n)
            hi_x = -((-(v + 1) << 64) // n)           # ceil((v+1) 2^64 / n)
            accepted = 0
            for x in range(lo_x, min(hi_x, 1 << 64)):
                # the draw under test at counter 0; any later draw is 2^64 - 1,
                # which is accepted for these n (its low word 2^64 - n equals
                # the threshold 2^64 mod n), so a rejection ends after one redraw
                monkeypatch.setattr(o, "draw",
                                    lambda key, ctr, x=x: x if ctr == 0 else (1 << 64) - 1)
                val, ctr2 = o.bounded(0, 0, n)
                assert ctr2 in (1, 2)
                if ctr2 == 1:
                    assert val == v
                    accepted += 1
            assert accepted == 1, (n, v, lo_x, hi_x)


def test_factor_rows_equal_full_factors():
    """netmf_factor_rows (chunked Gram, selected rows and columns) is the same
    arithmetic as netmf_factors; with chunks smaller than n it agrees to
    rounding on the selected rows and columns, and sketch_Y_rows_at gives the
    same rows of Y as sketch_Y."""
    g = synth.sbm(600, 3, 0.05, 0.005, seed=9)
    A = o.adjacency(g.row_ptr, g.col_idx, g.n)
    deg = o.degrees(A)
    X = o.normalized_operator(A, 0.4)
    U, lam = o.freigs(X, 24, q=6, s=8, seed=2)
    fac = o.netmf_factors(U, lam, deg, o.volume(A), 0.4, 10, 1.0)
    S = o.gen_sparse_sign(g.n, 40, 8, 0, o.STREAM_S)
    rows = np.array([0, 7, 123, 599])
    Lr, Rc = o.netmf_factor_rows(U, lam, deg, o.volume(A), 0.4, 10, 1.0, rows, S.p, chunk=97)
    assert np.allclose(Lr, fac.Lp[rows], rtol=1e-12, atol=0)
    assert np.allclose(Rc, fac.Rp[:, S.p], rtol=1e-10, atol=1e-14 * np.abs(fac.Rp).max())
    Y = o.sketch_Y(fac.Lp, fac.Rp, S)
    assert np.allclose(o.sketch_Y_rows_at(Lr, Rc, S), Y[rows], rtol=1e-10, atol=1e-12)


# ---------------------------------------------------------------- spectral propagation (Alg. 6 line 6)
@pytest.mark.parametrize("steps,theta", [(10, 0.5), (24, 2.0)])
def test_propagation_coefficients_sum_to_the_exponential(steps, theta):
    """sum_r c_r T_r(x) = exp(-theta/2) exp(-theta x) on [-1, 1]: the Bessel
    generating function, truncated where its terms are below rounding."""
    c = o.propagation_coefficients(steps, theta)
    x = np.linspace(-1.0, 1.0, 201)
    got = np.polynomial.chebyshev.chebval(x, c)
    want = np.exp(-0.5 * theta) * np.exp(-theta * x)
    assert np.max(np.abs(got - want)) < 1e-12 * want.max()


def _filter_dense(A_dense, E, theta, mu):
    """g(L) E through the spectrum: L = I - D^-1 A = D^-1/2 L_sym D^1/2 with
    L_sym = I - D^-1/2 A D^-1/2 = V diag(lam) V^T, g applied to lam."""
    deg = A_dense.sum(axis=1)
    s = 1.0 / np.sqrt(deg)
    Ls = np.eye(len(deg)) - s[:, None] * A_dense * s[None, :]
    lam, V = np.linalg.eigh(Ls)
    g = np.exp(-0.5 * theta * ((lam - mu) ** 2 - 1.0))
    return (s[:, None] * V) @ (g[:, None] * (V.T @ (np.sqrt(deg)[:, None] * E)))


@pytest.mark.parametrize("theta,mu", [(0.5, 0.2), (1.0, 1.0)])
def test_spectral_propagation_equals_the_filter_through_the_spectrum(theta, mu):
    g = synth.sbm(240, 4, 0.1, 0.02, seed=5)
    A = o.adjacency(g.row_ptr, g.col_idx, g.n)
    assert np.all(o.degrees(A) > 0)
    E = np.random.default_rng(0).standard_normal((g.n, 7))
    want = _filter_dense(A.toarray(), E, theta, mu)
    got = o.spectral_propagation(A, E, steps=10, theta=theta, mu=mu)
    assert np.max(np.abs(got - want)) < 1e-10 * np.max(np.abs(want))
    # no propagation steps: the constant term only
    got0 = o.spectral_propagation(A, E, steps=0, theta=theta, mu=mu)
    assert np.allclose(got0, o.propagation_coefficients(0, theta)[0] * E, rtol=0, atol=1e-15)


def test_spectral_propagation_isolated_rows_scale_by_g_of_one():
    """A vertex without edges is an eigenvector of L with eigenvalue 1."""
    n = 60
    edges = [(i, (i + 1) % 50) for i in range(50)] + [(i, (i + 7) % 50) for i in range(50)]
    g = synth.from_edges(n, edges)  # vertices 50..59 isolated
    A = o.adjacency(g.row_ptr, g.col_idx, g.n)
    E = np.random.default_rng(1).standard_normal((n, 3))
    got = o.spectral_propagation(A, E)
    g1 = math.exp(-0.25 * ((1.0 - 0.2) ** 2 - 1.0))
    assert np.allclose(got[50:], g1 * E[50:], rtol=1e-13, atol=0)
    want = _filter_dense(A.toarray()[:50, :50], E[:50], 0.5, 0.2)
    assert np.max(np.abs(got[:50] - want)) < 1e-10 * np.max(np.abs(want))


# ---------------------------------------------------------------- general single-pass SVD (Eqs. 5-10)
@pytest.mark.parametrize("n,m,k", [(400, 300, 12), (250, 250, 20)])
def test_general_single_pass_recovers_a_low_rank_product_exactly(n, m, k):
    """With f the identity and rank(LR) = k <= h, the sketches span the row
    and column spaces, and Eq. 10 reproduces LR and its SVD (to rounding)."""
    rng = np.random.default_rng(n + k)
    L = rng.standard_normal((n, k))
    Rt = rng.standard_normal((m, k)) * np.linspace(1.0, 0.05, k)[None, :]
    M = L @ Rt.T
    r = o.single_pass_svd_general(L, Rt, d=k, h=k + 6, l=k + 40, zeta=8, seed=3, f=o.identity)
    ref = np.linalg.svd(M, compute_uv=False)[:k]
    assert np.allclose(r.sigma, ref, rtol=1e-9)
    assert np.allclose((r.U * r.sigma) @ r.V.T, M, atol=1e-9 * np.abs(M).max())
    assert np.allclose(r.U.T @ r.U, np.eye(k), atol=1e-10)
    assert np.allclose(r.V.T @ r.V, np.eye(k), atol=1e-10)


def test_general_single_pass_trunc_log_against_dense_svd():
    """f = trunc_log of a rectangular product whose result has a decaying
    spectrum: the leading singular values within the randomized-sketch error
    of the dense SVD, and the sketches equal their definitions (Eq. 5) with
    dense sparse-sign matrices."""
    rng = np.random.default_rng(9)
    n, m, k = 300, 200, 6
    L = np.abs(rng.standard_normal((n, k))) * 1.5
    Rt = np.abs(rng.standard_normal((m, k)))
    F = o.trunc_log(L @ Rt.T)
    r = o.single_pass_svd_general(L, Rt, d=4, h=40, l=160, zeta=8, seed=1, f=o.trunc_log)
    ref = np.linalg.svd(F, compute_uv=False)
    assert np.allclose(r.sigma, ref[:4], rtol=2e-2)
    C = o.gen_sparse_sign(n, 40, 8, 1, o.STREAM_C).dense()
    S = o.gen_sparse_sign(m, 40, 8, 1, o.STREAM_S).dense()
    H = o.gen_sparse_sign(n, 160, 8, 1, o.STREAM_H).dense()
    O = o.gen_sparse_sign(m, 160, 8, 1, o.STREAM_O).dense()
    assert np.allclose(r.Y, F @ S)
    assert np.allclose(r.K, F.T @ C)
    assert np.allclose(r.Z, H.T @ F @ O)
