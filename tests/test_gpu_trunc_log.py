"""trunc_log as the tensor-core sketch epilogue evaluates it
(sne_trunc_log_eval), against log1p in FP64: relative error below 3e-7 for
r = x - 1 > 0 (polynomial on (0, 1), the hardware base-2 logarithm above),
exactly 0 for r <= 0, across 2^-30 .. 2^20 and at the switch r = 1."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sk():
    from paper_2110_12782_gb300 import build
    build.build()
    from paper_2110_12782_gb300 import sketchne
    sketchne.lib()
    return sketchne


def test_trunc_log_eval(sk):
    rng = np.random.default_rng(11)
    pos = np.exp(rng.uniform(np.log(2.0 ** -30), np.log(2.0 ** 20), 1_000_000))
    near1 = 1.0 + rng.uniform(-1e-3, 1e-3, 100_000)
    special = np.array([0.0, -0.0, -1e-30, -0.5, -1.0, -3.0, 1.0, np.nextafter(1.0, 0.0),
                        np.nextafter(1.0, 2.0), 2.0 ** -149, 1e-38, 0.5, 0.999999])
    r = np.concatenate([pos, near1, -pos[:1000], special]).astype(np.float32)
    rd = torch.from_numpy(r).cuda()
    out = torch.empty_like(rd)
    sk.sne_trunc_log_eval(rd, out)
    y = out.cpu().numpy().astype(np.float64)
    r64 = r.astype(np.float64)
    ref = np.where(r64 > 0, np.log1p(np.maximum(r64, 0.0)), 0.0)
    p = r64 > 0
    rel = np.abs(y[p] - ref[p]) / ref[p]
    print(f"trunc_log eval: max rel {rel.max():.2e}, mean {rel.mean():.2e}")
    assert rel.max() < 3e-7
    assert np.all(y[~p] == 0.0)


def test_trunc_log_eval_in_place_and_empty(sk):
    r = torch.linspace(-1.0, 3.0, 4097, device="cuda")
    ref = torch.where(r > 0, torch.log1p(r.double().clamp(min=0)), torch.zeros_like(r.double()))
    sk.sne_trunc_log_eval(r, r)
    assert torch.max(torch.abs(r.double() - ref) / ref.clamp(min=1e-30)).item() < 3e-7
    e = torch.empty(0, device="cuda")
    sk.sne_trunc_log_eval(e, e)
