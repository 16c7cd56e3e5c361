"""ctypes binding of libsketchne.so (declared in include/sketchne.h).

Argument marshalling only: every function here has the name of the C entry
point it calls, checks that the tensors it is given live on the GPU with the
expected dtype and layout, passes their device pointers and the current torch
stream, and raises ``SketchNEError`` on a nonzero return code.  PyTorch is used
for device memory and streams; no arithmetic of the method happens here.

The library must have been built (``paper_2110_12782_gb300.build.build()``);
importing a function fails loudly otherwise -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libsketchne.so")

SNE_OK = 0
SNE_ERR_ARG = -1
SNE_ERR_GRAPH = -2
SNE_ERR_SIZE = -3
SNE_ERR_WORKSPACE = -4
SNE_ERR_CUDA = -5
SNE_ERR_TIMEOUT = -6
SNE_ERR_NUMERIC = -7

SNE_FP32, SNE_BF16, SNE_FP16, SNE_BF16X2, SNE_FP16X2 = 0, 1, 2, 3, 4
PRECISIONS = {"fp32": SNE_FP32, "bf16": SNE_BF16, "fp16": SNE_FP16, "bf16x2": SNE_BF16X2,
              "fp16x2": SNE_FP16X2}
SNE_F_TRUNC_LOG, SNE_F_IDENTITY = 0, 1
SNE_ORTH_EIGSVD, SNE_ORTH_CHOLQR = 0, 1
SNE_WS_EMBED, SNE_WS_FREIGS, SNE_WS_SKETCH, SNE_WS_EMBED_HOST = 0, 1, 2, 3

EXPORTS = [
    "sne_params_init", "sne_error_string", "sne_workspace_bytes", "sne_embed", "sne_freigs",
    "sne_sketch_from_factors", "sne_sparse_sign", "sne_gaussian", "sne_degrees",
    "sne_degree_power", "sne_spmm_weights", "sne_spmm", "sne_validate_csr", "sne_status_reset", "sne_status",
    "sne_stats_read", "sne_embed_host", "sne_kernel_launches", "sne_profile_start",
    "sne_profile_stop", "sne_freigs_static", "sne_gram_workspace_bytes", "sne_gram",
    "sne_tall_gemm_workspace_bytes", "sne_tall_gemm", "sne_sym_eig_workspace_bytes", "sne_sym_eig",
    "sne_embed_batched_workspace_bytes", "sne_embed_batched", "sne_chol_inverse_workspace_bytes",
    "sne_chol_inverse", "sne_propagation_coefficients", "sne_spectral_propagate_workspace_bytes",
    "sne_spectral_propagate", "sne_single_pass_svd_workspace_bytes", "sne_single_pass_svd",
    "sne_trunc_log_eval", "sne_autotune_sketch",
]


class SketchNEError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {sne_error_string(code)} ({code})")


class sne_csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("row_ptr", ctypes.c_void_p),
                ("col_idx", ctypes.c_void_p), ("val", ctypes.c_void_p)]


class sne_tune_result(ctypes.Structure):
    _fields_ = [("tn", ctypes.c_int32), ("stages", ctypes.c_int32), ("split_mult", ctypes.c_int32),
                ("candidates", ctypes.c_int32), ("best_ms", ctypes.c_float),
                ("default_ms", ctypes.c_float), ("lanes", ctypes.c_int32),
                ("batch_ms", ctypes.c_float)]


class sne_params(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int32) for f in
                ("k", "q", "T", "d", "h", "l", "zeta", "s_eig", "row_block", "precision", "f",
                 "orth")] + [("alpha", ctypes.c_double), ("b", ctypes.c_double),
                             ("seed", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class sne_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("where", ctypes.c_int32), ("v_s", ctypes.c_int64),
                ("v_o", ctypes.c_int64), ("vol", ctypes.c_double)]


class sne_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("calls", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double)]


_lib = None


def lib() -> ctypes.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "paper_2110_12782_gb300.build.build() (requires nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, u64, dbl = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                  ctypes.c_double)
        P = ctypes.POINTER
        sig = {
            "sne_params_init": [P(sne_params), i32, i32],
            "sne_error_string": [ctypes.c_int],
            "sne_workspace_bytes": [i64, i64, P(sne_params), ctypes.c_int, P(ctypes.c_size_t)],
            "sne_embed": [P(sne_csr), P(sne_params), vp, ctypes.c_size_t, vp, vp, vp],
            "sne_freigs": [P(sne_csr), P(sne_params), vp, ctypes.c_size_t, vp, vp, vp],
            "sne_sketch_from_factors": [P(sne_csr), P(sne_params), vp, vp, vp, ctypes.c_size_t, vp,
                                        vp, vp, vp, vp],
            "sne_sparse_sign": [i64, i32, i32, u64, i32, vp, vp, vp],
            "sne_gaussian": [i64, i32, u64, i32, vp, vp],
            "sne_degrees": [P(sne_csr), vp, vp, vp],
            "sne_degree_power": [vp, i64, dbl, vp, vp],
            "sne_spmm_weights": [P(sne_csr), vp, vp, vp],
            "sne_spmm": [P(sne_csr), vp, vp, vp, i32, vp, vp],
            "sne_validate_csr": [P(sne_csr), vp, ctypes.c_size_t, vp],
            "sne_status_reset": [vp, vp],
            "sne_status": [vp, vp],
            "sne_stats_read": [vp, P(sne_stats), vp],
            "sne_embed_host": [P(sne_csr), P(sne_params), vp, ctypes.c_size_t, vp, vp, vp],
            "sne_kernel_launches": [],
            "sne_profile_start": [],
            "sne_profile_stop": [P(sne_kernel_time), ctypes.c_int, P(ctypes.c_int)],
            "sne_freigs_static": [P(sne_csr), P(sne_params), vp, vp, vp, vp],
            "sne_gram_workspace_bytes": [i64, i32, i32, P(ctypes.c_size_t)],
            "sne_gram": [i64, i32, i32, vp, i64, vp, i64, vp, vp, i32, i32, vp, ctypes.c_size_t, vp],
            "sne_tall_gemm_workspace_bytes": [i32, i32, P(ctypes.c_size_t)],
            "sne_tall_gemm": [i64, i32, i32, vp, i64, vp, i32, vp, i64, vp, ctypes.c_size_t, vp],
            "sne_sym_eig_workspace_bytes": [i32, P(ctypes.c_size_t)],
            "sne_sym_eig": [i32, vp, i32, vp, vp, i32, vp, ctypes.c_size_t, vp],
            "sne_chol_inverse_workspace_bytes": [i32, i32, P(ctypes.c_size_t)],
            "sne_chol_inverse": [i32, vp, i32, vp, i32, i32, dbl, vp, ctypes.c_size_t, vp],
            "sne_trunc_log_eval": [i64, vp, vp, vp],
            "sne_autotune_sketch": [i32, vp, P(sne_params), i32, vp, ctypes.c_size_t, vp, vp,
                                    P(sne_tune_result), vp],
            "sne_single_pass_svd_workspace_bytes": [i64, i64, i32, P(sne_params),
                                                    P(ctypes.c_size_t)],
            "sne_single_pass_svd": [i64, i64, i32, vp, i64, vp, i64, P(sne_params), vp,
                                    ctypes.c_size_t, vp, i64, vp, vp, i64, vp],
            "sne_propagation_coefficients": [i32, dbl, vp],
            "sne_spectral_propagate_workspace_bytes": [i64, i32, P(ctypes.c_size_t)],
            "sne_spectral_propagate": [P(sne_csr), i32, dbl, dbl, vp, i64, i32, vp,
                                       ctypes.c_size_t, vp],
            "sne_embed_batched_workspace_bytes": [i32, P(sne_csr), P(sne_params), i32,
                                                  P(ctypes.c_size_t)],
            "sne_embed_batched": [i32, P(sne_csr), P(sne_params), i32, vp, ctypes.c_size_t,
                                  P(ctypes.c_void_p), P(ctypes.c_void_p), vp, vp],
        }
        for name, args in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = {"sne_error_string": ctypes.c_char_p,
                          "sne_kernel_launches": ctypes.c_longlong}.get(name, ctypes.c_int)
        _lib = L
    return _lib


# ----------------------------------------------------------------------------- helpers
def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, torch.cuda.Stream):
        return stream.cuda_stream
    return int(stream)


def _ptr(t, dtype=None, name="tensor", allow_none=False, row_major=False) -> int | None:
    """Device pointer of t; with row_major a 2-D view with unit column stride
    (a leading dimension passed separately) is accepted as well."""
    if t is None:
        if allow_none:
            return None
        raise ValueError(f"{name} is required")
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if row_major:
        if t.dim() != 2 or t.stride(1) != 1:
            raise ValueError(f"{name} must be a row-major matrix")
    elif not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return t.data_ptr()


def _check(rc: int, where: str) -> None:
    if rc != SNE_OK:
        raise SketchNEError(rc, where)


class DeviceGraph:
    """A symmetric CSR graph held in device tensors, with its sne_csr struct."""

    def __init__(self, row_ptr: torch.Tensor, col_idx: torch.Tensor, val: torch.Tensor | None = None):
        self.row_ptr = row_ptr
        self.col_idx = col_idx
        self.val = val
        self.n = row_ptr.numel() - 1
        self.nnz = col_idx.numel()
        self.csr = sne_csr(self.n, self.nnz, _ptr(row_ptr, torch.int64, "row_ptr"),
                           _ptr(col_idx, torch.int32, "col_idx") if self.nnz else None,
                           _ptr(val, torch.float32, "val", allow_none=True))

    @classmethod
    def from_numpy(cls, row_ptr, col_idx, val=None, device="cuda"):
        rp = torch.as_tensor(row_ptr, dtype=torch.int64).to(device)
        ci = torch.as_tensor(col_idx, dtype=torch.int32).to(device)
        v = None if val is None else torch.as_tensor(val, dtype=torch.float32).to(device)
        return cls(rp, ci, v)


# ----------------------------------------------------------------------------- entry points
def sne_params_init(d: int, k: int, **overrides) -> sne_params:
    p = sne_params()
    _check(lib().sne_params_init(ctypes.byref(p), d, k), "sne_params_init")
    for key, v in overrides.items():
        if not hasattr(p, key):
            raise KeyError(key)
        setattr(p, key, v)
    return p


def sne_error_string(code: int) -> str:
    return lib().sne_error_string(code).decode()


def sne_workspace_bytes(n: int, nnz: int, p: sne_params, mode: int = SNE_WS_EMBED) -> int:
    out = ctypes.c_size_t(0)
    _check(lib().sne_workspace_bytes(n, nnz, ctypes.byref(p), mode, ctypes.byref(out)),
           "sne_workspace_bytes")
    return out.value


def workspace(n: int, nnz: int, p: sne_params, mode: int = SNE_WS_EMBED, device="cuda") -> torch.Tensor:
    """A device byte tensor large enough for the given mode (256-byte aligned)."""
    nbytes = sne_workspace_bytes(n, nnz, p, mode)
    t = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    off = (-t.data_ptr()) % 256
    return t[off:off + nbytes]


def sne_embed(g: DeviceGraph, p: sne_params, ws: torch.Tensor, E: torch.Tensor, sigma: torch.Tensor,
              stream=None) -> None:
    _check(lib().sne_embed(ctypes.byref(g.csr), ctypes.byref(p), _ptr(ws, torch.uint8, "workspace"),
                           ws.numel(), _ptr(E, torch.float32, "E"), _ptr(sigma, torch.float64, "sigma"),
                           _stream(stream)), "sne_embed")


def sne_freigs(g: DeviceGraph, p: sne_params, ws: torch.Tensor, U: torch.Tensor, lam: torch.Tensor,
               stream=None) -> None:
    _check(lib().sne_freigs(ctypes.byref(g.csr), ctypes.byref(p), _ptr(ws, torch.uint8, "workspace"),
                            ws.numel(), _ptr(U, torch.float32, "U"), _ptr(lam, torch.float64, "lambda"),
                            _stream(stream)), "sne_freigs")


def sne_sketch_from_factors(g: DeviceGraph, p: sne_params, U: torch.Tensor, lam: torch.Tensor,
                            ws: torch.Tensor, Y=None, Z=None, E=None, sigma=None, stream=None) -> None:
    _check(lib().sne_sketch_from_factors(
        ctypes.byref(g.csr), ctypes.byref(p), _ptr(U, torch.float32, "U"),
        _ptr(lam, torch.float64, "lambda"), _ptr(ws, torch.uint8, "workspace"), ws.numel(),
        _ptr(Y, torch.float32, "Y", True), _ptr(Z, torch.float32, "Z", True),
        _ptr(E, torch.float32, "E", True), _ptr(sigma, torch.float64, "sigma", True),
        _stream(stream)), "sne_sketch_from_factors")


def sne_sparse_sign(n: int, cols: int, zeta: int, seed: int, stream_id: int, idx: torch.Tensor,
                    sign: torch.Tensor, stream=None) -> None:
    _check(lib().sne_sparse_sign(n, cols, zeta, seed, stream_id, _ptr(idx, torch.int32, "idx"),
                                 _ptr(sign, torch.int8, "sign"), _stream(stream)), "sne_sparse_sign")


def sne_gaussian(n: int, cols: int, seed: int, stream_id: int, out: torch.Tensor, stream=None) -> None:
    _check(lib().sne_gaussian(n, cols, seed, stream_id, _ptr(out, torch.float32, "out"),
                              _stream(stream)), "sne_gaussian")


def sne_degrees(g: DeviceGraph, deg: torch.Tensor, vol: torch.Tensor, stream=None) -> None:
    _check(lib().sne_degrees(ctypes.byref(g.csr), _ptr(deg, torch.float32, "deg"),
                             _ptr(vol, torch.float64, "vol"), _stream(stream)), "sne_degrees")


def sne_degree_power(deg: torch.Tensor, beta: float, out: torch.Tensor, stream=None) -> None:
    _check(lib().sne_degree_power(_ptr(deg, torch.float32, "deg"), deg.numel(), beta,
                                  _ptr(out, torch.float32, "out"), _stream(stream)),
           "sne_degree_power")


def sne_spmm_weights(g: DeviceGraph, dpow: torch.Tensor, w_nz: torch.Tensor, stream=None) -> None:
    _check(lib().sne_spmm_weights(ctypes.byref(g.csr), _ptr(dpow, torch.float32, "dpow"),
                                  _ptr(w_nz, torch.float32, "w_nz"), _stream(stream)),
           "sne_spmm_weights")


def sne_spmm(g: DeviceGraph, dpow: torch.Tensor, B: torch.Tensor, Y: torch.Tensor,
             w_nz: torch.Tensor | None = None, stream=None) -> None:
    _check(lib().sne_spmm(ctypes.byref(g.csr), _ptr(dpow, torch.float32, "dpow"),
                          _ptr(w_nz, torch.float32, "w_nz", True), _ptr(B, torch.float32, "B"),
                          B.shape[1], _ptr(Y, torch.float32, "Y"), _stream(stream)), "sne_spmm")


def single_pass_svd_workspace(n: int, m: int, k: int, p: sne_params, device="cuda") -> torch.Tensor:
    nb = ctypes.c_size_t(0)
    _check(lib().sne_single_pass_svd_workspace_bytes(n, m, k, ctypes.byref(p), ctypes.byref(nb)),
           "sne_single_pass_svd_workspace_bytes")
    return _aligned_bytes(nb.value, device)


def sne_single_pass_svd(L: torch.Tensor, Rt: torch.Tensor, p: sne_params, ws: torch.Tensor,
                        U: torch.Tensor | None, sigma: torch.Tensor, V: torch.Tensor | None,
                        stream=None) -> None:
    """Eqs. 5-10 for f(L Rt^T): L (n x k), Rt (m x k) row-major CUDA float32;
    U (n x d), V (m x d) float32 or None, sigma (d) float64."""
    if L.shape[1] != Rt.shape[1]:
        raise ValueError("L and Rt need the same number of columns")
    _check(lib().sne_single_pass_svd(
        L.shape[0], Rt.shape[0], L.shape[1], _ptr(L, torch.float32, "L", row_major=True), L.stride(0),
        _ptr(Rt, torch.float32, "Rt", row_major=True), Rt.stride(0), ctypes.byref(p),
        _ptr(ws, torch.uint8, "workspace"), ws.numel(),
        _ptr(U, torch.float32, "U", True, row_major=True), U.stride(0) if U is not None else 0,
        _ptr(sigma, torch.float64, "sigma"), _ptr(V, torch.float32, "V", True, row_major=True),
        V.stride(0) if V is not None else 0, _stream(stream)), "sne_single_pass_svd")


def sne_propagation_coefficients(steps: int = 10, theta: float = 0.5) -> np.ndarray:
    """c_0 .. c_steps of the spectral-propagation filter (host only)."""
    c = np.zeros(steps + 1, dtype=np.float64)
    _check(lib().sne_propagation_coefficients(steps, theta, c.ctypes.data), "sne_propagation_coefficients")
    return c


def propagate_workspace(n: int, d: int, device="cuda") -> torch.Tensor:
    nb = ctypes.c_size_t(0)
    _check(lib().sne_spectral_propagate_workspace_bytes(n, d, ctypes.byref(nb)),
           "sne_spectral_propagate_workspace_bytes")
    return _aligned_bytes(nb.value, device)


def sne_spectral_propagate(g: DeviceGraph, E: torch.Tensor, ws: torch.Tensor, steps: int = 10,
                           theta: float = 0.5, mu: float = 0.2, stream=None) -> None:
    """Alg. 6 line 6 on the CUDA FP32 row-major E (n x d), in place."""
    _check(lib().sne_spectral_propagate(ctypes.byref(g.csr), steps, theta, mu,
                                        _ptr(E, torch.float32, "E", row_major=True), E.stride(0),
                                        E.shape[1],
                                        _ptr(ws, torch.uint8, "workspace"), ws.numel(),
                                        _stream(stream)), "sne_spectral_propagate")


def sne_validate_csr(g: DeviceGraph, ws: torch.Tensor, stream=None) -> None:
    _check(lib().sne_validate_csr(ctypes.byref(g.csr), _ptr(ws, torch.uint8, "workspace"), ws.numel(),
                                  _stream(stream)), "sne_validate_csr")


def sne_status_reset(ws: torch.Tensor, stream=None) -> None:
    _check(lib().sne_status_reset(_ptr(ws, torch.uint8, "workspace"), _stream(stream)),
           "sne_status_reset")


def sne_status(ws: torch.Tensor, stream=None) -> int:
    return lib().sne_status(_ptr(ws, torch.uint8, "workspace"), _stream(stream))


def sne_stats_read(ws: torch.Tensor, stream=None) -> sne_stats:
    out = sne_stats()
    _check(lib().sne_stats_read(_ptr(ws, torch.uint8, "workspace"), ctypes.byref(out), _stream(stream)),
           "sne_stats_read")
    return out


def check_status(ws: torch.Tensor, where: str = "device", stream=None) -> None:
    """Raises if the workspace's device status word records an error."""
    _check(sne_status(ws, stream), where)


def sne_embed_host(row_ptr, col_idx, val, n: int, p: sne_params, ws: torch.Tensor, E_host: torch.Tensor,
                   sigma_host: torch.Tensor, stream=None) -> None:
    """sne_embed from host arrays (torch CPU tensors, pinned for asynchronous copies)."""
    for t, nm in ((row_ptr, "row_ptr"), (col_idx, "col_idx"), (E_host, "E"), (sigma_host, "sigma")):
        if t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{nm} must be a contiguous host tensor")
    g = sne_csr(n, col_idx.numel(), row_ptr.data_ptr(), col_idx.data_ptr(),
                None if val is None else val.data_ptr())
    _check(lib().sne_embed_host(ctypes.byref(g), ctypes.byref(p), _ptr(ws, torch.uint8, "workspace"),
                                ws.numel(), E_host.data_ptr(), sigma_host.data_ptr(), _stream(stream)),
           "sne_embed_host")


def sne_kernel_launches() -> int:
    return int(lib().sne_kernel_launches())


def sne_profile_start() -> None:
    _check(lib().sne_profile_start(), "sne_profile_start")


def sne_profile_stop() -> dict:
    """Per kernel class: {name: (calls, launches, total_ms)}."""
    arr = (sne_kernel_time * 32)()
    cnt = ctypes.c_int(0)
    _check(lib().sne_profile_stop(arr, 32, ctypes.byref(cnt)), "sne_profile_stop")
    return {arr[i].name.decode(): (arr[i].calls, arr[i].launches, arr[i].total_ms)
            for i in range(cnt.value)}


def sne_freigs_static(g: DeviceGraph, p: sne_params, U: torch.Tensor, lam: torch.Tensor,
                      status: torch.Tensor | None = None, stream=None) -> None:
    """Alg. 5 with the library's static device workspace (no allocation)."""
    _check(lib().sne_freigs_static(ctypes.byref(g.csr), ctypes.byref(p), _ptr(U, torch.float32, "U"),
                                   _ptr(lam, torch.float64, "lambda"),
                                   _ptr(status, torch.int32, "status", True), _stream(stream)),
           "sne_freigs_static")


# ----------------------------------------------------------------------------- dense building blocks
def _aligned_bytes(nbytes: int, device) -> torch.Tensor:
    t = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
    off = (-t.data_ptr()) % 256
    return t[off:off + nbytes]


def _row_stride(t: torch.Tensor, name: str) -> int:
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError(f"{name} must be a row-major 2-D tensor")
    return t.stride(0)


def gram_workspace(n: int, ka: int, kb: int, device="cuda") -> torch.Tensor:
    nb = ctypes.c_size_t(0)
    _check(lib().sne_gram_workspace_bytes(n, ka, kb, ctypes.byref(nb)), "sne_gram_workspace_bytes")
    return _aligned_bytes(nb.value, device)


def sne_gram(A: torch.Tensor, B: torch.Tensor, C: torch.Tensor, ws: torch.Tensor,
             w: torch.Tensor | None = None, accurate: bool = False, stream=None) -> None:
    """C (FP64) = A^T diag(w) B for tall row-major FP32 A (n x ka) and B (n x kb);
    ``accurate`` selects the double-float accumulation."""
    for t, nm in ((A, "A"), (B, "B")):
        if not (t.is_cuda and t.dtype == torch.float32):
            raise ValueError(f"{nm} must be a CUDA float32 tensor")
    if C.dtype != torch.float64 or not C.is_cuda:
        raise ValueError("C must be a CUDA float64 tensor")
    n, ka = A.shape
    kb = B.shape[1]
    if B.shape[0] != n or tuple(C.shape) != (ka, kb):
        raise ValueError("shape mismatch")
    _check(lib().sne_gram(n, ka, kb, A.data_ptr(), _row_stride(A, "A"), B.data_ptr(), _row_stride(B, "B"),
                          _ptr(w, torch.float32, "w", True), C.data_ptr(), _row_stride(C, "C"),
                          1 if accurate else 0, _ptr(ws, torch.uint8, "workspace"), ws.numel(),
                          _stream(stream)), "sne_gram")


def tall_gemm_workspace(ka: int, kc: int, device="cuda") -> torch.Tensor:
    nb = ctypes.c_size_t(0)
    _check(lib().sne_tall_gemm_workspace_bytes(ka, kc, ctypes.byref(nb)), "sne_tall_gemm_workspace_bytes")
    return _aligned_bytes(nb.value, device)


def sne_tall_gemm(A: torch.Tensor, M: torch.Tensor, C: torch.Tensor, ws: torch.Tensor, stream=None) -> None:
    """C = A M for tall row-major FP32 A (n x ka) and small M (ka x kc)."""
    for t, nm in ((A, "A"), (M, "M"), (C, "C")):
        if not (t.is_cuda and t.dtype == torch.float32):
            raise ValueError(f"{nm} must be a CUDA float32 tensor")
    n, ka = A.shape
    kc = M.shape[1]
    if M.shape[0] != ka or tuple(C.shape) != (n, kc):
        raise ValueError("shape mismatch")
    _check(lib().sne_tall_gemm(n, ka, kc, A.data_ptr(), _row_stride(A, "A"), M.data_ptr(),
                               _row_stride(M, "M"), C.data_ptr(), _row_stride(C, "C"),
                               _ptr(ws, torch.uint8, "workspace"), ws.numel(), _stream(stream)),
           "sne_tall_gemm")


def sym_eig_workspace(n: int, device="cuda") -> torch.Tensor:
    nb = ctypes.c_size_t(0)
    _check(lib().sne_sym_eig_workspace_bytes(n, ctypes.byref(nb)), "sne_sym_eig_workspace_bytes")
    return _aligned_bytes(nb.value, device)


def sne_sym_eig(S: torch.Tensor, lam: torch.Tensor, V: torch.Tensor, ws: torch.Tensor, stream=None) -> None:
    """Symmetric FP64 S = V diag(lam) V^T, lam ordered by |lam| descending."""
    n = S.shape[0]
    for t, nm in ((S, "S"), (lam, "lambda"), (V, "V")):
        if not (t.is_cuda and t.dtype == torch.float64):
            raise ValueError(f"{nm} must be a CUDA float64 tensor")
    if tuple(S.shape) != (n, n) or tuple(V.shape) != (n, n) or lam.numel() != n:
        raise ValueError("shape mismatch")
    _check(lib().sne_sym_eig(n, S.data_ptr(), _row_stride(S, "S"), _ptr(lam, torch.float64, "lambda"),
                             V.data_ptr(), _row_stride(V, "V"), _ptr(ws, torch.uint8, "workspace"),
                             ws.numel(), _stream(stream)), "sne_sym_eig")


# ----------------------------------------------------------------------------- batches of graphs
def _csr_array(graphs):
    arr = (sne_csr * len(graphs))()
    for i, g in enumerate(graphs):
        arr[i] = g.csr
    return arr


def batched_workspace(graphs, p: sne_params, lanes: int = 0, device="cuda") -> torch.Tensor:
    nb = ctypes.c_size_t(0)
    _check(lib().sne_embed_batched_workspace_bytes(len(graphs), _csr_array(graphs), ctypes.byref(p),
                                                   lanes, ctypes.byref(nb)),
           "sne_embed_batched_workspace_bytes")
    return _aligned_bytes(nb.value, device)


def sne_embed_batched(graphs, p: sne_params, ws: torch.Tensor, E, sigma, status: torch.Tensor | None = None,
                      lanes: int = 0, stream=None) -> None:
    """Alg. 6 lines 1-5 for every DeviceGraph of ``graphs`` (outputs E[i], sigma[i])."""
    G = len(graphs)
    if len(E) != G or len(sigma) != G:
        raise ValueError("one E and one sigma per graph")
    e_ptrs = (ctypes.c_void_p * G)(*[_ptr(e, torch.float32, "E") for e in E])
    s_ptrs = (ctypes.c_void_p * G)(*[_ptr(s_, torch.float64, "sigma") for s_ in sigma])
    _check(lib().sne_embed_batched(G, _csr_array(graphs), ctypes.byref(p), lanes,
                                   _ptr(ws, torch.uint8, "workspace"), ws.numel(), e_ptrs, s_ptrs,
                                   _ptr(status, torch.int32, "status", True), _stream(stream)),
           "sne_embed_batched")


def sne_autotune_sketch(graphs, p: sne_params, ws: torch.Tensor, lanes: int = 0, E=None, sigma=None,
                        stream=None) -> dict:
    """Time the fused tensor-core sketch over its launch shapes for one graph
    (workspace of ``workspace(..., SNE_WS_EMBED)``) or a batch (workspace of
    ``batched_workspace(graphs, p, lanes)``); the fastest shape is used from
    then on.  For a batch with outputs E, sigma (one per graph) and lanes 0,
    also the number of stream lanes.  Returns the choices and the times."""
    if isinstance(graphs, DeviceGraph):
        graphs = [graphs]
    G = len(graphs)
    e_ptrs = s_ptrs = None
    if E is not None and sigma is not None:
        if len(E) != G or len(sigma) != G:
            raise ValueError("one E and one sigma per graph")
        e_ptrs = (ctypes.c_void_p * G)(*[_ptr(e, torch.float32, "E") for e in E])
        s_ptrs = (ctypes.c_void_p * G)(*[_ptr(s_, torch.float64, "sigma") for s_ in sigma])
    res = sne_tune_result()
    _check(lib().sne_autotune_sketch(G, _csr_array(graphs), ctypes.byref(p), lanes,
                                     _ptr(ws, torch.uint8, "workspace"), ws.numel(), e_ptrs, s_ptrs,
                                     ctypes.byref(res), _stream(stream)), "sne_autotune_sketch")
    return {"tn": res.tn, "stages": res.stages, "split_mult": res.split_mult,
            "candidates": res.candidates, "best_ms": res.best_ms, "default_ms": res.default_ms,
            "lanes": res.lanes, "batch_ms": res.batch_ms}


def chol_inverse_workspace(n: int, fp64: bool, device="cuda") -> torch.Tensor:
    nb = ctypes.c_size_t(0)
    _check(lib().sne_chol_inverse_workspace_bytes(n, 1 if fp64 else 0, ctypes.byref(nb)),
           "sne_chol_inverse_workspace_bytes")
    return _aligned_bytes(nb.value, device)


def sne_trunc_log_eval(r: torch.Tensor, out: torch.Tensor, stream=None) -> None:
    """out = trunc_log(1 + r) elementwise, as the tensor-core sketch evaluates it."""
    if r.numel() != out.numel():
        raise ValueError("r and out must have the same size")
    _check(lib().sne_trunc_log_eval(r.numel(), _ptr(r, torch.float32, "r"), _ptr(out, torch.float32, "out"),
                                    _stream(stream)), "sne_trunc_log_eval")


def sne_chol_inverse(A: torch.Tensor, M: torch.Tensor, ws: torch.Tensor, tol: float = -1.0,
                     stream=None) -> None:
    """M with M^T A M = I (tol < 0) or diag(I_r, 0) (pivoted, rank cut at tol)."""
    if A.dtype != M.dtype or A.dtype not in (torch.float32, torch.float64):
        raise ValueError("A and M must both be float32 or both float64")
    n = A.shape[0]
    if tuple(A.shape) != (n, n) or tuple(M.shape) != (n, n):
        raise ValueError("shape mismatch")
    _check(lib().sne_chol_inverse(n, A.data_ptr(), _row_stride(A, "A"), M.data_ptr(), _row_stride(M, "M"),
                                  1 if A.dtype == torch.float64 else 0, tol,
                                  _ptr(ws, torch.uint8, "workspace"), ws.numel(), _stream(stream)),
           "sne_chol_inverse")
