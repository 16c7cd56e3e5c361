"""Spectral propagation (Alg. 6 line 6) through the C ABI against the FP64
oracle, element by element.

FP32 recurrence error: every term T_r of the series stays within |E| (the
Chebyshev polynomials are bounded by 1 on the spectrum of X), each pass adds
a few FP32 roundings per gathered row, and the coefficients fall off like
(theta/2)^r / r!, so the result carries a relative error of a few 1e-7 of
max|E|; the stated bound is 1e-5 of max|F| (F the oracle's result).

Cases: an SBM and a Chung-Lu graph at widths 32 and 30 (a width that is not a
multiple of 4, leading dimension 40), a graph with isolated vertices, no
steps, the C1 embedding from sne_embed, and (slow) the n = 1M Chung-Lu graph
at width 128, the width and graph of the benchmark.
"""
import numpy as np
import pytest
import torch

from oracle import sketchne_oracle as o
from paper_2110_12782_gb300 import synth

pytestmark = pytest.mark.gpu
TOL = 1e-5


@pytest.fixture(scope="module")
def sk():
    from paper_2110_12782_gb300 import build
    build.build()
    from paper_2110_12782_gb300 import sketchne
    sketchne.lib()
    return sketchne


def run(sk, g, E_host, steps=10, theta=0.5, mu=0.2, lde=None):
    n, d = E_host.shape
    lde = lde or d
    buf = torch.zeros(n, lde, dtype=torch.float32, device="cuda")
    buf[:, :d] = torch.from_numpy(E_host.astype(np.float32)).cuda()
    G = sk.DeviceGraph.from_numpy(g.row_ptr, g.col_idx)
    ws = sk.propagate_workspace(n, d)
    sk.sne_spectral_propagate(G, buf[:, :d], ws, steps=steps, theta=theta, mu=mu)
    sk.check_status(ws, "propagate")
    out = buf.cpu().numpy()
    assert np.all(out[:, d:] == 0.0)  # the columns past d are not touched
    return out[:, :d].astype(np.float64)


def check(sk, g, E, **kw):
    lde = kw.pop("lde", None)
    A = o.adjacency(g.row_ptr, g.col_idx, g.n)
    want = o.spectral_propagation(A, E.astype(np.float32).astype(np.float64), **kw)
    got = run(sk, g, E, lde=lde, **kw)
    err = np.max(np.abs(got - want)) / np.max(np.abs(want))
    return err


@pytest.mark.parametrize("kind,d,lde", [("sbm", 32, None), ("chung_lu", 32, None),
                                        ("chung_lu", 30, 40)])
def test_propagation_matches_oracle(sk, kind, d, lde):
    g = synth.sbm(4096, 8, 0.01, 0.001, seed=0) if kind == "sbm" else \
        synth.chung_lu(20000, 12.0, 2.1, seed=2)
    E = np.random.default_rng(3).standard_normal((g.n, d))
    err = check(sk, g, E, lde=lde)
    print(f"propagation {kind} n={g.n} d={d}: max |F - F_ref| / max |F_ref| = {err:.2e}")
    assert err < TOL


@pytest.mark.parametrize("steps,theta,mu", [(0, 0.5, 0.2), (1, 0.5, 0.2), (10, 1.0, 1.0),
                                            (24, 2.0, 0.0)])
def test_propagation_parameters(sk, steps, theta, mu):
    g = synth.sbm(2048, 4, 0.02, 0.002, seed=1)
    E = np.random.default_rng(4).standard_normal((g.n, 16))
    err = check(sk, g, E, steps=steps, theta=theta, mu=mu)
    assert err < TOL, (steps, theta, mu, err)


def test_propagation_isolated_vertices(sk):
    n = 3000
    g0 = synth.chung_lu(2500, 8.0, 2.2, seed=5)
    # vertices 2500 .. 2999 have no edges
    rp = np.concatenate([g0.row_ptr, np.full(n - g0.n, g0.row_ptr[-1], dtype=np.int64)])
    g = synth.Graph(n=n, row_ptr=rp, col_idx=g0.col_idx)
    E = np.random.default_rng(6).standard_normal((n, 8))
    err = check(sk, g, E)
    assert err < TOL


def test_propagation_of_the_embedding(sk):
    """The embedding of sne_embed on the C1 graph, propagated on the GPU and by
    the oracle from the same FP32 E."""
    g = synth.sbm(4096, 8, 0.01, 0.001, seed=0)
    G = sk.DeviceGraph.from_numpy(g.row_ptr, g.col_idx)
    p = sk.sne_params_init(32, 128, orth=sk.SNE_ORTH_CHOLQR)
    ws = sk.workspace(g.n, g.nnz, p, sk.SNE_WS_EMBED)
    E = torch.empty(g.n, p.d, dtype=torch.float32, device="cuda")
    sig = torch.empty(p.d, dtype=torch.float64, device="cuda")
    sk.sne_embed(G, p, ws, E, sig)
    sk.check_status(ws, "embed")
    err = check(sk, g, E.cpu().numpy().astype(np.float64))
    assert err < TOL


@pytest.mark.slow
def test_propagation_full_size(sk):
    g = synth.chung_lu(1_000_000, 20.0, 2.1, seed=0)
    E = np.random.default_rng(7).standard_normal((g.n, 128)).astype(np.float32)
    err = check(sk, g, E)
    print(f"propagation n=1M d=128: {err:.2e}")
    assert err < TOL
