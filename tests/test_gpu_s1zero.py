"""The very-large-graph setting of Sec. 5.2 (Table 3's ClueWeb and Hyperlink
rows): no oversampling of the single-pass sketch (s1 = 0, so h = d), small k
and d (k = d = 32 or 16), T = 5, alpha = 0.45, few power iterations.  The
embedding through the C ABI against the FP64 oracle run with the same
parameters from the GPU's eigenpairs, on a Chung-Lu graph, FP32 and the FP16
hi/lo pair reconstruction: singular values within 1e-3 relative and
principal-angle sines within 1e-3 on the leading block whose relative gap is
at least 1e-2 (both the paper-level tolerances of the full-size tests).
"""
import numpy as np
import pytest
import torch

from oracle import sketchne_oracle as o
from paper_2110_12782_gb300 import synth

pytestmark = pytest.mark.gpu
GAP, TOL = 1e-2, 1e-3


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


@pytest.mark.parametrize("d,q", [(32, 6), (16, 5)])
@pytest.mark.parametrize("precision", ["fp32", "fp16x2"])
def test_s1_zero_embedding_matches_oracle(sk, d, q, precision):
    g = synth.chung_lu(30000, 10.0, 2.2, seed=4)
    G = sk.DeviceGraph.from_numpy(g.row_ptr, g.col_idx)
    p = sk.sne_params_init(d, d, q=q, T=5, h=d, alpha=0.45, orth=sk.SNE_ORTH_CHOLQR,
                           precision=sk.PRECISIONS[precision])
    # eigenpairs from the GPU, so that the comparison isolates lines 2-5
    ws = sk.workspace(g.n, g.nnz, p, sk.SNE_WS_FREIGS)
    U = torch.empty(g.n, p.k, dtype=torch.float32, device="cuda")
    lam = torch.empty(p.k, dtype=torch.float64, device="cuda")
    sk.sne_freigs(G, p, ws, U, lam)
    sk.check_status(ws, "freigs")
    wss = sk.workspace(g.n, g.nnz, p, sk.SNE_WS_SKETCH)
    E = torch.empty(g.n, d, dtype=torch.float32, device="cuda")
    sig = torch.empty(d, dtype=torch.float64, device="cuda")
    sk.sne_sketch_from_factors(G, p, U, lam, wss, E=E, sigma=sig)
    sk.check_status(wss, "sketch")
    op = o.Params(k=d, d=d, q=q, T=5, h=d, alpha=0.45)
    ref = o.embed(g.row_ptr, g.col_idx, g.n, op, U_k=U.cpu().double().numpy(),
                  lam=lam.cpu().numpy())
    s = sig.cpu().numpy()
    blk = leading_gap_block(ref.sigma, d)
    assert blk >= 1
    srel = np.max(np.abs(s[:blk] - ref.sigma[:blk]) / ref.sigma[:blk])
    sines = o.principal_angle_sines(E.cpu().double().numpy()[:, :blk], ref.E[:, :blk])
    print(f"s1=0 d={d} q={q} {precision}: leading block {blk}, sigma rel {srel:.1e}, "
          f"max sine {sines.max():.1e}")
    assert srel < TOL
    assert sines.max() < TOL
