"""Failure detection on the GPU without a fault: every mbarrier wait of the
tensor-core sketch kernel is bounded.  With SNE_FAULT_INJECT=tc_stall the
kernel leaves one shared-memory stage unloaded (an mbarrier that nothing
completes) and its waits are limited to 20 ms: the MMA warp's wait runs out,
the CTA records SNE_ERR_TIMEOUT in the workspace status word, lets its own
copies and MMAs land, frees its tensor memory and returns.  The context stays
usable: the next call, without the injection, succeeds and matches the
oracle."""
import numpy as np
import pytest
import torch

from oracle import sketchne_oracle as o
from paper_2110_12782_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sk():
    from paper_2110_12782_gb300 import build
    build.build()
    from paper_2110_12782_gb300 import sketchne
    sketchne.lib()
    return sketchne


def test_bounded_wait_runs_out_and_context_stays_usable(sk, monkeypatch):
    g = synth.sbm(1500, 3, 0.05, 0.005, seed=4)
    op = o.Params(k=64, d=8, q=6, h=36, l=150)
    ref = o.embed(g.row_ptr, g.col_idx, g.n, op)
    pr = op.resolved()
    G = sk.DeviceGraph.from_numpy(g.row_ptr, g.col_idx)
    q = sk.sne_params_init(pr.d, pr.k, q=pr.q, h=pr.h, l=pr.l, precision=sk.SNE_FP16)
    U = torch.tensor(ref.U_k, dtype=torch.float32, device="cuda")
    lam = torch.tensor(ref.lam, dtype=torch.float64, device="cuda")
    ws = sk.workspace(g.n, g.nnz, q, sk.SNE_WS_SKETCH)
    Y = torch.empty(g.n, pr.h, dtype=torch.float32, device="cuda")
    Z = torch.empty(pr.l, pr.l, dtype=torch.float32, device="cuda")
    monkeypatch.setenv("SNE_FAULT_INJECT", "tc_stall")
    sk.sne_sketch_from_factors(G, q, U, lam, ws, Y=Y, Z=Z)
    st = sk.sne_stats_read(ws)
    assert st.status == sk.SNE_ERR_TIMEOUT, sk.sne_error_string(st.status)
    monkeypatch.delenv("SNE_FAULT_INJECT")
    # the same call again: the status word is cleared by the call, the
    # kernels (tensor memory allocated afresh) complete
    sk.sne_sketch_from_factors(G, q, U, lam, ws, Y=Y, Z=Z)
    st = sk.sne_stats_read(ws)
    assert st.status == 0, sk.sne_error_string(st.status)
    ey = float(np.linalg.norm(Y.cpu().numpy() - ref.sp.Y) / np.linalg.norm(ref.sp.Y))
    ez = float(np.linalg.norm(Z.cpu().numpy() - ref.sp.Z) / np.linalg.norm(ref.sp.Z))
    print(f"after the injected timeout: Y rel {ey:.2e}, Z rel {ez:.2e}")
    assert ey < 5e-3 and ez < 5e-3
