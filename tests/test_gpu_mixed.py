"""Mixed-precision (BF16 / FP16 operands, FP32 accumulation on tcgen05) fused
sketch against the FP32 path and the FP64 oracle.

The tolerances are derived from the operand rounding: after row/column
normalization every product term carries a relative error of at most
2^-11 (FP16) or 2^-8 (BF16) per operand; x = sum_c a_c b_c near the trunc_log
threshold has an absolute error of a few units of that times the largest
term, which f passes through with slope <= 1.  The errors measured against the
FP64 oracle are printed and asserted below the stated bounds.
"""
import numpy as np
import pytest
import torch

from oracle import sketchne_oracle as o
from paper_2110_12782_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"fp16": {"Y": 5e-3, "Z": 5e-3}, "bf16": {"Y": 4e-2, "Z": 4e-2}}


@pytest.fixture(scope="module")
def sk():
    from paper_2110_12782_gb300 import build
    build.build()
    from paper_2110_12782_gb300 import sketchne
    sketchne.lib()
    return sketchne


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def c1():
    g = synth.named("sbm4096")
    p = o.Params(k=128, d=32)
    return g, p, o.embed(g.row_ptr, g.col_idx, g.n, p)


def sketch(sk, g, p, U, lam, precision, f=None):
    pr = p.resolved()
    G = sk.DeviceGraph.from_numpy(g.row_ptr, g.col_idx)
    prec = {"fp32": sk.SNE_FP32, "fp16": sk.SNE_FP16, "bf16": sk.SNE_BF16}[precision]
    q = sk.sne_params_init(pr.d, pr.k, q=pr.q, T=pr.T, h=pr.h, l=pr.l, precision=prec,
                           f=sk.SNE_F_TRUNC_LOG if (f or pr.f) == "trunc_log" else sk.SNE_F_IDENTITY)
    ws = sk.workspace(g.n, g.nnz, q, sk.SNE_WS_SKETCH)
    Y = torch.empty(g.n, pr.h, dtype=torch.float32, device="cuda")
    Z = torch.empty(pr.l, pr.l, dtype=torch.float32, device="cuda")
    E = torch.empty(g.n, pr.d, dtype=torch.float32, device="cuda")
    sig = torch.empty(pr.d, dtype=torch.float64, device="cuda")
    sk.sne_sketch_from_factors(G, q, torch.tensor(U, dtype=torch.float32, device="cuda"),
                               torch.tensor(lam, dtype=torch.float64, device="cuda"), ws,
                               Y=Y, Z=Z, E=E, sigma=sig)
    st = sk.sne_stats_read(ws)
    assert st.status == 0, sk.sne_error_string(st.status)
    return Y.cpu().numpy(), Z.cpu().numpy(), E.cpu().numpy(), sig.cpu().numpy()


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_tc_identity_f_matches_fp32_path(sk, c1, precision):
    # f = identity isolates the GEMM + segmented sum of the tensor-core kernel
    g, p, ref = c1
    Y32, Z32, _, _ = sketch(sk, g, p, ref.U_k, ref.lam, "fp32", f="identity")
    Yh, Zh, _, _ = sketch(sk, g, p, ref.U_k, ref.lam, precision, f="identity")
    ey, ez = rel(Yh, Y32), rel(Zh, Z32)
    print(f"{precision} identity: Y rel {ey:.2e}  Z rel {ez:.2e}")
    assert ey < TOL[precision]["Y"] and ez < TOL[precision]["Z"]


@pytest.mark.parametrize("precision", ["fp16", "bf16"])
def test_tc_trunc_log_sketch_vs_oracle(sk, c1, precision):
    g, p, ref = c1
    Y, Z, E, sig = sketch(sk, g, p, ref.U_k, ref.lam, precision)
    ey, ez = rel(Y, ref.sp.Y), rel(Z, ref.sp.Z)
    es = np.max(np.abs(sig - ref.sigma) / ref.sigma)
    print(f"{precision} trunc_log: Y rel {ey:.2e}  Z rel {ez:.2e}  sigma rel {es:.2e}")
    assert ey < TOL[precision]["Y"] and ez < TOL[precision]["Z"]


def test_tc_ragged_rows_and_columns(sk):
    # n = 1500 is not a multiple of the 128-row tile; h*z and l*z are not
    # multiples of the 256-column tile
    g = synth.sbm(1500, 3, 0.05, 0.005, seed=4)
    p = o.Params(k=64, d=8, q=6, h=36, l=150)
    ref = o.embed(g.row_ptr, g.col_idx, g.n, p)
    Y, Z, _, _ = sketch(sk, g, p, ref.U_k, ref.lam, "fp16")
    ey, ez = rel(Y, ref.sp.Y), rel(Z, ref.sp.Z)
    print(f"ragged fp16: Y rel {ey:.2e}  Z rel {ez:.2e}")
    assert ey < TOL["fp16"]["Y"] and ez < TOL["fp16"]["Z"]
