"""The C ABI without a GPU: the library loads, exports every function that
include/sketchne.h declares, and rejects bad arguments on the host (calls that
return before any CUDA work)."""
import ctypes
import os
import re

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
