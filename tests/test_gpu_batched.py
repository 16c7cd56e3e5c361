"""sne_embed_batched: a batch of uneven graphs (8-block SBMs and Chung-Lu
graphs, as in the 64-graph batch workload, smaller) embedded in one call on
several streams, against one sne_embed per graph, against the FP64 oracle, and
captured into a CUDA graph and replayed."""
import numpy as np
import pytest
import torch

from oracle import sketchne_oracle as o
from paper_2110_12782_gb300 import synth

pytestmark = pytest.mark.gpu

K, D = 64, 32


@pytest.fixture(scope="module")
def sk():
    from paper_2110_12782_gb300 import build
    build.build()
    from paper_2110_12782_gb300 import sketchne
    sketchne.lib()
    return sketchne


@pytest.fixture(scope="module")
def batch(sk):
    graphs = synth.batched_mix(count=7, n_lo=2000, n_hi=12000, seed=5)
    dev = [sk.DeviceGraph.from_numpy(g.row_ptr, g.col_idx) for g in graphs]
    p = sk.sne_params_init(D, K, orth=sk.SNE_ORTH_CHOLQR)
    return graphs, dev, p


def outputs(graphs):
    E = [torch.empty(g.n, D, dtype=torch.float32, device="cuda") for g in graphs]
    s = [torch.empty(D, dtype=torch.float64, device="cuda") for _ in graphs]
    return E, s


def run_single(sk, graphs, dev, p):
    E, s = outputs(graphs)
    for g, G, e, sg in zip(graphs, dev, E, s):
        ws = sk.workspace(g.n, g.nnz, p, sk.SNE_WS_EMBED)
        sk.sne_embed(G, p, ws, e, sg)
        sk.check_status(ws)
    return E, s


@pytest.mark.parametrize("lanes", [1, 3, 0])
def test_batched_equals_single(sk, batch, lanes):
    graphs, dev, p = batch
    E1, s1 = run_single(sk, graphs, dev, p)
    E, s = outputs(graphs)
    ws = sk.batched_workspace(dev, p, lanes)
    status = torch.full((len(graphs),), -99, dtype=torch.int32, device="cuda")
    sk.sne_embed_batched(dev, p, ws, E, s, status=status, lanes=lanes)
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [0] * len(graphs)
    worst = 0.0
    for a, b, sa, sb in zip(E, E1, s, s1):
        worst = max(worst, float((a - b).abs().max() / b.abs().max()))
        assert torch.allclose(sa, sb, rtol=1e-9, atol=0)
    print(f"lanes={lanes}: max relative difference to single calls {worst:.1e}")
    assert worst < 1e-6


def test_batched_matches_oracle(sk, batch):
    graphs, dev, p = batch
    E, s = outputs(graphs)
    ws = sk.batched_workspace(dev, p)
    sk.sne_embed_batched(dev, p, ws, E, s)
    torch.cuda.synchronize()
    for i, g in enumerate(graphs):
        ref = o.embed(g.row_ptr, g.col_idx, g.n, o.Params(k=K, d=D, q=20))
        sig = s[i].cpu().numpy()
        srel = np.max(np.abs(sig - ref.sigma) / ref.sigma)
        blk = 0
        for j in range(1, D):
            if (ref.sigma[j - 1] - ref.sigma[j]) / ref.sigma[j - 1] >= 1e-2:
                blk = j
        sines = o.principal_angle_sines(E[i].cpu().numpy()[:, :blk], ref.E[:, :blk]) if blk else [0.0]
        kind = "SBM" if i % 2 == 0 else "Chung-Lu"
        srel_blk = np.max(np.abs(sig[:blk] - ref.sigma[:blk]) / ref.sigma[:blk]) if blk else 0.0
        print(f"graph {i} ({kind}, n={g.n}): sigma rel {srel:.1e} (block {srel_blk:.1e}), "
              f"block {blk} sine {np.max(sines):.1e}")
        # every graph, SBM and Chung-Lu: the stated tolerance on the gapped block
        assert blk >= 1 and np.max(sines) < 1e-3, (i, kind)
        assert srel_blk < 1e-3, (i, kind)


def test_batched_cuda_graph_replay(sk, batch):
    graphs, dev, p = batch
    E, s = outputs(graphs)
    ws = sk.batched_workspace(dev, p)
    sk.sne_embed_batched(dev, p, ws, E, s)  # creates the lanes before capture
    torch.cuda.synchronize()
    ref_E = [e.clone() for e in E]
    for e in E:
        e.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        sk.sne_embed_batched(dev, p, ws, E, s)
    for _ in range(2):
        graph.replay()
    torch.cuda.synchronize()
    for a, b in zip(E, ref_E):
        assert torch.equal(a, b)
