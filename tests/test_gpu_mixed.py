"""Mixed-precision fused sketch (half-precision operands on tcgen05, FP32
accumulation) against the FP32 path and the FP64 oracle, and the embedding
it leads to.

Every path evaluates the entries of L'R' in the centred form
x - 1 = s (W_i - w) C (W_j - w)^T + rho_i + kappa_j (w the degree-weighted
mean row of W = D^(-1+a) U), so the operand rounding is relative to the
centred factors.  Tolerances, from the operand rounding (unit roundoff u of
the operand format after power-of-two row and column scaling: FP16 2^-11,
BF16 2^-8; hi/lo pairs about u^2, i.e. 2^-22 and 2^-16): a product of two
rounded operands carries at most 2u relative error per term, the k-term sum a
few times that relative to the sum of |terms|, and trunc_log passes it with
slope <= 1.  Stated bounds on Y and Z (relative Frobenius): FP16 5e-3,
BF16 4e-2, FP16 pairs 1e-4 (the sketch bound stated for FP32), BF16 pairs
1e-3.  The embedding is compared on the leading block of singular directions
separated by a relative gap >= 1e-2 (Davis-Kahan): principal-angle sine and
singular values within 1e-3 for the pairs (the FP32 bound), 1e-2 for FP16
and 5e-2 for BF16 (ten times the Y bound: the least-squares solves of Alg. 4
line 8 amplify the error of Y by cond(O^T Q), about 10 on this graph).
"""
import numpy as np
import pytest
import torch

from oracle import sketchne_oracle as o
from paper_2110_12782_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {"fp16": {"Y": 5e-3, "Z": 5e-3, "E": 1e-2},
       "bf16": {"Y": 4e-2, "Z": 4e-2, "E": 5e-2},
       "fp16x2": {"Y": 1e-4, "Z": 1e-4, "E": 1e-3},
       "bf16x2": {"Y": 1e-3, "Z": 1e-3, "E": 1e-3}}
PRECS = ["fp16", "bf16", "fp16x2", "bf16x2"]


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
    q = sk.sne_params_init(pr.d, pr.k, q=pr.q, T=pr.T, h=pr.h, l=pr.l,
                           precision=sk.PRECISIONS[precision],
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


def gapped_block(sigma):
    """Size of the leading block of singular directions separated from the
    rest by a relative gap >= 1e-2."""
    blk = 0
    for j in range(1, len(sigma)):
        if (sigma[j - 1] - sigma[j]) / sigma[j - 1] >= 1e-2:
            blk = j
    return blk


@pytest.mark.parametrize("precision", PRECS)
def test_tc_identity_f_matches_fp32_path(sk, c1, precision):
    # f = identity isolates the GEMM + segmented sum of the tensor-core kernel
    g, p, ref = c1
    Y32, Z32, _, _ = sketch(sk, g, p, ref.U_k, ref.lam, "fp32", f="identity")
    Yh, Zh, _, _ = sketch(sk, g, p, ref.U_k, ref.lam, precision, f="identity")
    ey, ez = rel(Yh, Y32), rel(Zh, Z32)
    print(f"{precision} identity: Y rel {ey:.2e}  Z rel {ez:.2e}")
    assert ey < TOL[precision]["Y"] and ez < TOL[precision]["Z"]


@pytest.mark.parametrize("precision", PRECS)
def test_tc_trunc_log_sketch_and_embedding_vs_oracle(sk, c1, precision):
    g, p, ref = c1
    Y, Z, E, sig = sketch(sk, g, p, ref.U_k, ref.lam, precision)
    ey, ez = rel(Y, ref.sp.Y), rel(Z, ref.sp.Z)
    blk = gapped_block(ref.sigma)
    sine = o.principal_angle_sines(E[:, :blk].astype(np.float64), ref.E[:, :blk]).max()
    es = np.max(np.abs(sig[:blk] - ref.sigma[:blk]) / ref.sigma[:blk])
    print(f"{precision} trunc_log: Y rel {ey:.2e}  Z rel {ez:.2e}  block {blk}: sine {sine:.2e} "
          f"sigma rel {es:.2e}")
    assert blk >= 8
    assert ey < TOL[precision]["Y"] and ez < TOL[precision]["Z"]
    assert sine < TOL[precision]["E"] and es < TOL[precision]["E"]


@pytest.mark.parametrize("precision", ["fp16", "fp16x2"])
def test_tc_ragged_rows_and_columns(sk, precision):
    # n = 1500 is not a multiple of the 128-row tile; h*z and l*z are not
    # multiples of the 256-column tile
    g = synth.sbm(1500, 3, 0.05, 0.005, seed=4)
    p = o.Params(k=64, d=8, q=6, h=36, l=150)
    ref = o.embed(g.row_ptr, g.col_idx, g.n, p)
    Y, Z, _, _ = sketch(sk, g, p, ref.U_k, ref.lam, precision)
    ey, ez = rel(Y, ref.sp.Y), rel(Z, ref.sp.Z)
    print(f"ragged {precision}: Y rel {ey:.2e}  Z rel {ez:.2e}")
    assert ey < TOL[precision]["Y"] and ez < TOL[precision]["Z"]

