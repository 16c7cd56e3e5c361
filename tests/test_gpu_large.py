"""The two largest workloads through the C ABI, drawn on the GPU with the
Chung-Lu recipe (synth.chung_lu_device):

* n = 10^7, mean degree 30, exponent 2.2, k = 256, d = 128, BF16 and FP32
  reconstruction: Y on a seeded sample of 100,000 rows against the FP64
  oracle from the GPU's own eigenpairs (the Gram of U_k summed over row
  chunks: oracle.netmf_factor_rows), at the stated tolerances (FP32 1e-4,
  BF16 4e-2); the two embeddings agree on their singular values within the
  BF16 bound.
* n = 5 * 10^7, mean degree 40 (about 2 * 10^9 stored entries, near the
  int32 limit of the column indices), exponent 2.1, k = 128, d = 128, FP16
  reconstruction: sne_embed runs through (status OK; singular values positive
  and descending; U_d = E Sigma^-1/2 orthonormal; rows of isolated vertices
  zero), and Y on a seeded sample of 20,000 rows is within the FP16 bound 5e-3
  of the oracle.
"""
import numpy as np
import pytest
import torch

from oracle import sketchne_oracle as o
from paper_2110_12782_gb300 import synth

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module")
def sk():
    from paper_2110_12782_gb300 import build
    build.build()
    from paper_2110_12782_gb300 import sketchne
    sketchne.lib()
    return sketchne


def freigs(sk, G, n, nnz, p):
    ws = sk.workspace(n, nnz, p, sk.SNE_WS_FREIGS)
    U = torch.empty(n, p.k, dtype=torch.float32, device="cuda")
    lam = torch.empty(p.k, dtype=torch.float64, device="cuda")
    sk.sne_freigs(G, p, ws, U, lam)
    sk.check_status(ws, "freigs")
    del ws
    torch.cuda.empty_cache()
    return U, lam


def sample_error(sk, G, n, nnz, rp_host, p, U, lam, precision, rows):
    """Relative error of Y on the seeded rows against the oracle."""
    deg = np.diff(rp_host).astype(np.float64)
    sel = np.sort(np.random.default_rng(1).choice(n, size=rows, replace=False))
    S = o.gen_sparse_sign(n, p.h, p.zeta, p.seed, o.STREAM_S)
    Lr, Rc = o.netmf_factor_rows(U.cpu().numpy(), lam.cpu().numpy(), deg, float(deg.sum()),
                                 p.alpha, p.T, p.b, sel, S.p)
    ref = o.sketch_Y_rows_at(Lr, Rc, S)
    q = sk.sne_params_init(p.d, p.k, precision=precision, orth=sk.SNE_ORTH_CHOLQR)
    wss = sk.workspace(n, nnz, q, sk.SNE_WS_SKETCH)
    Y = torch.empty(n, q.h, dtype=torch.float32, device="cuda")
    sk.sne_sketch_from_factors(G, q, U, lam, wss, Y=Y)
    sk.check_status(wss, "sketch")
    got = Y[torch.as_tensor(sel, device="cuda")].cpu().double().numpy()
    del wss, Y
    torch.cuda.empty_cache()
    return float(np.linalg.norm(got - ref) / np.linalg.norm(ref))


def embed(sk, G, n, nnz, p):
    ws = sk.workspace(n, nnz, p, sk.SNE_WS_EMBED)
    E = torch.empty(n, p.d, dtype=torch.float32, device="cuda")
    sig = torch.empty(p.d, dtype=torch.float64, device="cuda")
    sk.sne_embed(G, p, ws, E, sig)
    sk.check_status(ws, "embed")
    del ws
    torch.cuda.empty_cache()
    return E, sig.cpu().numpy()


def test_cl10m_bf16_and_fp32_sample_against_oracle(sk):
    n = 10_000_000
    rp, ci = synth.chung_lu_device(n, 30.0, 2.2, seed=0)
    nnz = int(ci.numel())
    G = sk.DeviceGraph(rp, ci)
    p = sk.sne_params_init(128, 256, orth=sk.SNE_ORTH_CHOLQR)
    U, lam = freigs(sk, G, n, nnz, p)
    rph = rp.cpu().numpy()
    errs = {prec: sample_error(sk, G, n, nnz, rph, p, U, lam, code, 100_000)
            for prec, code in (("fp32", sk.SNE_FP32), ("bf16", sk.SNE_BF16))}
    del U, lam
    torch.cuda.empty_cache()
    sig = {}
    for prec, code in (("fp32", sk.SNE_FP32), ("bf16", sk.SNE_BF16)):
        q = sk.sne_params_init(128, 256, orth=sk.SNE_ORTH_CHOLQR, precision=code)
        E, s = embed(sk, G, n, nnz, q)
        assert np.all(s > 0) and np.all(np.diff(s) <= 1e-9 * s[0])
        sig[prec] = s
        del E
    sdiff = np.max(np.abs(sig["bf16"] - sig["fp32"]) / sig["fp32"])
    print(f"n=10^7 (nnz {nnz}): Y sample rel fp32 {errs['fp32']:.2e}, bf16 {errs['bf16']:.2e}; "
          f"sigma bf16 vs fp32 {sdiff:.2e}")
    assert errs["fp32"] < 1e-4
    assert errs["bf16"] < 4e-2
    assert sdiff < 4e-2


def test_cl50m_fp16_runs_through_and_sample_against_oracle(sk):
    n = 50_000_000
    rp, ci = synth.chung_lu_device(n, 40.0, 2.1, seed=0)
    nnz = int(ci.numel())
    assert nnz < 2 ** 31
    G = sk.DeviceGraph(rp, ci)
    p = sk.sne_params_init(128, 128, orth=sk.SNE_ORTH_CHOLQR, precision=sk.SNE_FP16)
    E, s = embed(sk, G, n, nnz, p)
    assert np.all(s > 0) and np.all(np.diff(s) <= 1e-9 * s[0])
    deg = (rp[1:] - rp[:-1])
    iso = deg == 0
    if bool(iso.any()):
        assert float(E[iso].abs().max()) == 0.0
    Ud = E.double() / torch.as_tensor(np.sqrt(s), device="cuda")[None, :]
    orth = float((Ud.T @ Ud - torch.eye(p.d, dtype=torch.float64, device="cuda")).abs().max())
    del E, Ud
    torch.cuda.empty_cache()
    U, lam = freigs(sk, G, n, nnz, p)
    err = sample_error(sk, G, n, nnz, rp.cpu().numpy(), p, U, lam, sk.SNE_FP16, 20_000)
    print(f"n=5*10^7 (nnz {nnz}): |U_d^T U_d - I| {orth:.1e}, sigma[:3] {s[:3]}, "
          f"Y sample rel (fp16) {err:.2e}")
    assert orth < 1e-3
    assert err < 5e-3
