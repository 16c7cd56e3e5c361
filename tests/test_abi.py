"""The C ABI without a GPU: the library loads, exports every function that
include/sketchne.h declares, and rejects bad arguments on the host (calls that
return before any CUDA work)."""
import ctypes
import math
import os
import re
import types

import pytest

from paper_2110_12782_gb300 import build
from paper_2110_12782_gb300 import sketchne as sk

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return sk.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "sketchne.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sne_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(sk.EXPORTS)


def test_struct_layouts_match_header(L):
    assert ctypes.sizeof(sk.sne_params) == 12 * 4 + 2 * 8 + 8
    assert ctypes.sizeof(sk.sne_csr) == 40
    assert ctypes.sizeof(sk.sne_stats) == 32


def test_params_defaults(L):
    p = sk.sne_params_init(128, 256)
    assert (p.k, p.d, p.h, p.l, p.q, p.T, p.zeta, p.s_eig) == (256, 128, 272, 1128, 20, 10, 8, 16)
    assert p.alpha == 0.5 and p.b == 1.0 and p.precision == sk.SNE_FP32
    assert p.f == sk.SNE_F_TRUNC_LOG and p.orth == sk.SNE_ORTH_EIGSVD
    with pytest.raises(sk.SketchNEError):
        sk.sne_params_init(0, 10)


def test_error_strings(L):
    for code in range(0, -8, -1):
        assert sk.sne_error_string(code)
    assert "unknown" in sk.sne_error_string(-99)


def test_workspace_bytes_and_size_checks(L):
    p = sk.sne_params_init(32, 128)
    small = sk.sne_workspace_bytes(4096, 35000, p, sk.SNE_WS_EMBED)
    big = sk.sne_workspace_bytes(1_000_000, 20_000_000, sk.sne_params_init(128, 256), sk.SNE_WS_EMBED)
    assert 0 < small < big
    assert small % 256 == 0
    # k + s larger than n
    with pytest.raises(sk.SketchNEError) as e:
        sk.sne_workspace_bytes(100, 1000, p, sk.SNE_WS_FREIGS)
    assert e.value.code == sk.SNE_ERR_SIZE
    # d > h
    q = sk.sne_params_init(32, 64, h=16)
    with pytest.raises(sk.SketchNEError) as e:
        sk.sne_workspace_bytes(4096, 1000, q, sk.SNE_WS_SKETCH)
    assert e.value.code == sk.SNE_ERR_SIZE
    # bad enum
    q = sk.sne_params_init(32, 64, precision=7)
    with pytest.raises(sk.SketchNEError) as e:
        sk.sne_workspace_bytes(4096, 1000, q, sk.SNE_WS_EMBED)
    assert e.value.code == sk.SNE_ERR_ARG


def test_host_side_argument_errors_enqueue_nothing(L):
    p = sk.sne_params_init(32, 128)
    # NULL graph / workspace: rejected on the host
    assert L.sne_embed(None, ctypes.byref(p), None, 0, None, None, None) == sk.SNE_ERR_ARG
    g = sk.sne_csr(4096, 10, None, None, None)
    assert L.sne_embed(ctypes.byref(g), ctypes.byref(p), None, 0, None, None, None) == sk.SNE_ERR_ARG
    g = sk.sne_csr(4096, 10, 256, 512, None)  # fake, never dereferenced
    assert L.sne_embed(ctypes.byref(g), ctypes.byref(p), None, 0, None, None, None) == \
        sk.SNE_ERR_WORKSPACE
    assert L.sne_embed(ctypes.byref(g), ctypes.byref(p), 257, 1 << 40, None, None, None) == \
        sk.SNE_ERR_WORKSPACE
    assert L.sne_sparse_sign(0, 10, 8, 0, 2, None, None, None) == sk.SNE_ERR_ARG
    assert L.sne_sparse_sign(1000, 10, 65, 0, 2, 256, 512, None) == sk.SNE_ERR_SIZE
    assert L.sne_status(None, None) == sk.SNE_ERR_WORKSPACE


def test_building_block_argument_errors_on_the_host(L):
    """The dense building blocks reject bad sizes, leading dimensions, flags and
    workspaces before any CUDA call (fake device addresses, never read)."""
    ARG, WS = sk.SNE_ERR_ARG, sk.SNE_ERR_WORKSPACE
    nb = ctypes.c_size_t(0)
    assert L.sne_gram_workspace_bytes(1000, 16, 16, ctypes.byref(nb)) == 0 and nb.value > 0
    assert L.sne_gram_workspace_bytes(0, 16, 16, ctypes.byref(nb)) == ARG
    A, C = 1 << 20, 1 << 21
    need = nb.value
    assert L.sne_gram(0, 16, 16, A, 16, A, 16, None, C, 16, 0, 256, need, None) == ARG
    assert L.sne_gram(1000, 16, 16, A, 8, A, 16, None, C, 16, 0, 256, need, None) == ARG  # lda < ka
    assert L.sne_gram(1000, 16, 16, A, 16, A, 16, None, C, 16, 2, 256, need, None) == ARG  # flag
    assert L.sne_gram(1000, 16, 16, None, 16, A, 16, None, C, 16, 0, 256, need, None) == ARG
    assert L.sne_gram(1000, 16, 16, A, 16, A, 16, None, C, 16, 0, None, need, None) == WS
    assert L.sne_gram(1000, 16, 16, A, 16, A, 16, None, C, 16, 0, 257, need, None) == WS  # unaligned
    assert L.sne_gram(1000, 16, 16, A, 16, A, 16, None, C, 16, 0, 256, need - 1, None) == WS
    assert L.sne_tall_gemm_workspace_bytes(16, 8, ctypes.byref(nb)) == 0
    assert L.sne_tall_gemm(1000, 16, 8, A, 16, A, 4, C, 8, 256, nb.value, None) == ARG  # ldm < kc
    assert L.sne_tall_gemm(1000, 16, 8, A, 16, A, 8, C, 8, 256, nb.value - 1, None) == WS
    assert L.sne_sym_eig_workspace_bytes(1025, ctypes.byref(nb)) == ARG
    assert L.sne_sym_eig_workspace_bytes(272, ctypes.byref(nb)) == 0
    assert L.sne_sym_eig(272, A, 271, C, C, 272, 256, nb.value, None) == ARG  # lds < n
    assert L.sne_sym_eig(272, A, 272, C, C, 272, 256, nb.value - 1, None) == WS
    assert L.sne_chol_inverse_workspace_bytes(300, 1, ctypes.byref(nb)) == 0
    assert L.sne_chol_inverse(300, A, 300, C, 299, 1, -1.0, 256, nb.value, None) == ARG
    assert L.sne_chol_inverse(300, A, 300, C, 300, 1, -1.0, 256, nb.value - 1, None) == WS
    assert L.sne_trunc_log_eval(-1, A, C, None) == ARG
    assert L.sne_trunc_log_eval(10, None, C, None) == ARG
    assert L.sne_trunc_log_eval(10, A, None, None) == ARG
    assert L.sne_trunc_log_eval(0, None, None, None) == 0  # nothing to do
    res = sk.sne_tune_result()
    p32 = sk.sne_params_init(16, 32)
    g1 = (sk.sne_csr * 1)()
    g1[0] = sk.sne_csr(1000, 2000, 256, 256, None)
    assert L.sne_autotune_sketch(0, g1, ctypes.byref(p32), 0, 256, 1 << 20, None, None, ctypes.byref(res), None) == ARG
    assert L.sne_autotune_sketch(1, g1, ctypes.byref(p32), 0, 256, 1 << 20, None, None, None, None) == ARG
    # the FP32 path has no tensor-core sketch to tune
    assert L.sne_autotune_sketch(1, g1, ctypes.byref(p32), 0, 256, 1 << 20, None, None, ctypes.byref(res), None) == ARG


def test_lockstep_batch_workspace_on_the_host(L):
    """With a half-precision reconstruction the batch runs in lockstep and
    every graph keeps its own workspace slice: the batch workspace is the sum
    of the graphs' sne_embed workspaces (each rounded up to a multiple of 256
    bytes and of an operand row, 2 * kpad bytes) and does not depend on the
    number of lanes; with FP32 it is the lanes' slices."""
    p16 = sk.sne_params_init(16, 64, precision=sk.SNE_FP16X2)
    graphs = (sk.sne_csr * 3)(sk.sne_csr(5000, 40000, 256, 512, None),
                              sk.sne_csr(3000, 20000, 768, 1024, None),
                              sk.sne_csr(7000, 50000, 1280, 1536, None))
    each = []
    for g in graphs:
        b = ctypes.c_size_t(0)
        assert L.sne_workspace_bytes(g.n, g.nnz, ctypes.byref(p16), sk.SNE_WS_EMBED, ctypes.byref(b)) == 0
        each.append(b.value)
    row = 2 * 64  # kpad = 64
    al = 256 * row // math.gcd(256, row)
    want = sum((b + al - 1) // al * al for b in each)
    for lanes in (0, 1, 3):
        nb = ctypes.c_size_t(0)
        assert L.sne_embed_batched_workspace_bytes(3, graphs, ctypes.byref(p16), lanes, ctypes.byref(nb)) == 0
        assert nb.value == want, (lanes, nb.value, want)
    p32 = sk.sne_params_init(16, 64)
    one = ctypes.c_size_t(0)
    assert L.sne_embed_batched_workspace_bytes(3, graphs, ctypes.byref(p32), 1, ctypes.byref(one)) == 0
    b32 = ctypes.c_size_t(0)
    assert L.sne_workspace_bytes(7000, 50000, ctypes.byref(p32), sk.SNE_WS_EMBED, ctypes.byref(b32)) == 0
    assert one.value == (b32.value + 255) // 256 * 256  # one lane: the largest graph's slice


def test_batched_argument_errors_on_the_host(L):
    p = sk.sne_params_init(16, 32)
    graphs = (sk.sne_csr * 2)(sk.sne_csr(5000, 40000, 256, 512, None),
                              sk.sne_csr(3000, 20000, 768, 1024, None))
    nb = ctypes.c_size_t(0)
    assert L.sne_embed_batched_workspace_bytes(2, graphs, ctypes.byref(p), 0, ctypes.byref(nb)) == 0
    one = ctypes.c_size_t(0)
    assert L.sne_embed_batched_workspace_bytes(2, graphs, ctypes.byref(p), 1, ctypes.byref(one)) == 0
    # two lanes hold both graphs' workspaces, one lane only the larger one
    assert nb.value > one.value > 0
    assert L.sne_embed_batched_workspace_bytes(0, graphs, ctypes.byref(p), 0, ctypes.byref(nb)) == \
        sk.SNE_ERR_ARG
    assert L.sne_embed_batched_workspace_bytes(2, graphs, ctypes.byref(p), 17, ctypes.byref(nb)) == \
        sk.SNE_ERR_ARG
    bad = (sk.sne_csr * 1)(sk.sne_csr(0, 0, 256, None, None))
    assert L.sne_embed_batched_workspace_bytes(1, bad, ctypes.byref(p), 0, ctypes.byref(nb)) == \
        sk.SNE_ERR_ARG
    E = (ctypes.c_void_p * 2)(1 << 20, None)
    S = (ctypes.c_void_p * 2)(1 << 21, 1 << 22)
    assert L.sne_embed_batched(2, graphs, ctypes.byref(p), 0, 256, 1 << 40, E, S, None, None) == \
        sk.SNE_ERR_ARG
    E = (ctypes.c_void_p * 2)(1 << 20, 1 << 23)
    assert L.sne_embed_batched(2, graphs, ctypes.byref(p), 0, None, 1 << 40, E, S, None, None) == \
        sk.SNE_ERR_WORKSPACE
    assert L.sne_embed_batched(2, graphs, ctypes.byref(p), 0, 256, 1000, E, S, None, None) == \
        sk.SNE_ERR_WORKSPACE


def test_no_cpu_fallback(L, monkeypatch):
    """Host tensors are refused before any call, and a missing library is an
    error, never a silent switch to another implementation."""
    import torch
    with pytest.raises(ValueError, match="CUDA tensor"):
        sk.DeviceGraph(torch.zeros(5, dtype=torch.int64), torch.zeros(4, dtype=torch.int32))
    p = sk.sne_params_init(8, 16)
    with pytest.raises(ValueError, match="CUDA tensor"):
        g = types.SimpleNamespace(csr=sk.sne_csr(4, 0, None, None, None))
        sk.sne_spmm(g, torch.zeros(4), torch.zeros(4, 4), torch.zeros(4, 4))
    monkeypatch.setattr(sk, "_lib", None)
    monkeypatch.setattr(sk, "LIB_PATH", os.path.join(ROOT, "no_such_library.so"))
    with pytest.raises(RuntimeError, match="missing"):
        sk.sne_params_init(8, 16)
    assert p.d == 8


def test_graph_without_edges_is_rejected_on_the_host(L):
    """vol(G) = 0 leaves Eq. 1 undefined: every embedding entry point returns
    SNE_ERR_GRAPH for a graph with no edges before touching the device."""
    p = sk.sne_params_init(8, 16)
    g = sk.sne_csr(1000, 0, 256, None, None)  # fake row_ptr address, never read
    GR = sk.SNE_ERR_GRAPH
    assert L.sne_embed(ctypes.byref(g), ctypes.byref(p), 256, 1 << 40, 512, 768, None) == GR
    assert L.sne_embed_host(ctypes.byref(g), ctypes.byref(p), 256, 1 << 40, 512, 768, None) == GR
    assert L.sne_freigs(ctypes.byref(g), ctypes.byref(p), 256, 1 << 40, 512, 768, None) == GR
    assert L.sne_sketch_from_factors(ctypes.byref(g), ctypes.byref(p), 512, 768, 256, 1 << 40,
                                     None, None, None, None, None) == GR
    assert L.sne_freigs_static(ctypes.byref(g), ctypes.byref(p), 512, 768, None, None) == GR
    graphs = (sk.sne_csr * 1)(g)
    nb = ctypes.c_size_t(0)
    assert L.sne_embed_batched_workspace_bytes(1, graphs, ctypes.byref(p), 0, ctypes.byref(nb)) == GR
    assert "no edges" in sk.sne_error_string(GR)


def test_pair_precision_rejects_k_beyond_the_resident_tile(L):
    """hi/lo pair operands keep 2 x k half columns of the 128-row A tile in
    shared memory, so the pair precisions take k <= 320 (single: k <= 384)."""
    for prec, k, ok in ((sk.SNE_FP16X2, 320, True), (sk.SNE_FP16X2, 384, False),
                        (sk.SNE_BF16X2, 384, False), (sk.SNE_FP16, 384, True)):
        q = sk.sne_params_init(64, k, precision=prec)
        if ok:
            assert sk.sne_workspace_bytes(100_000, 1_000_000, q, sk.SNE_WS_SKETCH) > 0
        else:
            with pytest.raises(sk.SketchNEError) as e:
                sk.sne_workspace_bytes(100_000, 1_000_000, q, sk.SNE_WS_SKETCH)
            assert e.value.code == sk.SNE_ERR_SIZE


def test_propagation_coefficients_match_the_oracle_on_the_host(L):
    """The library's host-side Bessel series (Alg. 6 line 6 coefficients)
    against the oracle's, which calls SciPy's modified Bessel functions."""
    import numpy as np
    from oracle import sketchne_oracle as o
    for steps, theta in ((10, 0.5), (0, 0.5), (30, 4.0), (5, 0.0)):
        got = sk.sne_propagation_coefficients(steps, theta)
        want = o.propagation_coefficients(steps, theta)
        assert np.allclose(got, want, rtol=1e-14, atol=1e-300), (steps, theta)
    c = (ctypes.c_double * 4)()
    ARG = sk.SNE_ERR_ARG
    assert L.sne_propagation_coefficients(-1, 0.5, c) == ARG
    assert L.sne_propagation_coefficients(1001, 0.5, c) == ARG
    assert L.sne_propagation_coefficients(3, -0.1, c) == ARG
    assert L.sne_propagation_coefficients(3, float("nan"), c) == ARG
    assert L.sne_propagation_coefficients(3, 0.5, None) == ARG


def test_spectral_propagate_argument_errors_on_the_host(L):
    ARG, WS = sk.SNE_ERR_ARG, sk.SNE_ERR_WORKSPACE
    nb = ctypes.c_size_t(0)
    assert L.sne_spectral_propagate_workspace_bytes(1000, 32, ctypes.byref(nb)) == 0
    assert L.sne_spectral_propagate_workspace_bytes(1000, 1025, ctypes.byref(nb)) == ARG
    assert L.sne_spectral_propagate_workspace_bytes(1000, 32, ctypes.byref(nb)) == 0
    need = nb.value
    g = sk.sne_csr(1000, 10, 1 << 20, 1 << 21, None)
    E = 1 << 22
    call = lambda steps=10, theta=0.5, mu=0.2, e=E, lde=32, d=32, ws=256, nbytes=need: \
        L.sne_spectral_propagate(ctypes.byref(g), steps, theta, mu, e, lde, d, ws, nbytes, None)
    assert call(steps=-1) == ARG
    assert call(steps=1001) == ARG
    assert call(theta=-1.0) == ARG
    assert call(mu=2.5) == ARG
    assert call(mu=-0.1) == ARG
    assert call(lde=31) == ARG
    assert call(e=None) == ARG
    assert call(ws=None) == WS
    assert call(ws=257) == WS
    assert call(nbytes=need - 1) == WS


def test_single_pass_svd_argument_errors_on_the_host(L):
    ARG, SIZE, WS = sk.SNE_ERR_ARG, sk.SNE_ERR_SIZE, sk.SNE_ERR_WORKSPACE
    p = sk.sne_params_init(16, 32)
    p.h, p.l = 24, 200
    nb = ctypes.c_size_t(0)
    assert L.sne_single_pass_svd_workspace_bytes(5000, 3000, 32, ctypes.byref(p), ctypes.byref(nb)) == 0
    need = nb.value
    assert L.sne_single_pass_svd_workspace_bytes(0, 3000, 32, ctypes.byref(p), ctypes.byref(nb)) == ARG
    q = sk.sne_params_init(16, 32)
    q.h, q.l = 12, 200                              # d > h
    assert L.sne_single_pass_svd_workspace_bytes(5000, 3000, 32, ctypes.byref(q), ctypes.byref(nb)) == SIZE
    q.h, q.l = 24, 20                               # h > l
    assert L.sne_single_pass_svd_workspace_bytes(5000, 3000, 32, ctypes.byref(q), ctypes.byref(nb)) == SIZE
    q.h, q.l = 400, 1000                            # h beyond the small eigensolver
    assert L.sne_single_pass_svd_workspace_bytes(5000, 3000, 32, ctypes.byref(q), ctypes.byref(nb)) == SIZE
    A, B, U, S, V = 1 << 20, 1 << 21, 1 << 22, 1 << 23, 1 << 24
    call = lambda ldl=32, ldr=32, ldu=16, ldv=16, s=S, ws=256, nbytes=need: L.sne_single_pass_svd(
        5000, 3000, 32, A, ldl, B, ldr, ctypes.byref(p), ws, nbytes, U, ldu, s, V, ldv, None)
    assert call(ldl=31) == ARG
    assert call(ldr=31) == ARG
    assert call(ldu=15) == ARG
    assert call(s=None) == ARG
    assert call(ws=None) == WS
    assert call(nbytes=need - 1) == WS
