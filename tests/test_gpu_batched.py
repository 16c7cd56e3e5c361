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


def gapped_block(sigma):
    blk = 0
    for j in range(1, D):
        if (sigma[j - 1] - sigma[j]) / sigma[j - 1] >= 1e-2:
            blk = j
    return blk


def test_batched_matches_oracle(sk, batch):
    """Every graph of the batch, SBM and Chung-Lu, at the stated tolerance
    (principal-angle sine and singular values within 1e-3 on the leading block
    separated by a relative gap >= 1e-2):

    * the batched embedding against the oracle's Alg. 6 lines 2-5 run on the
      GPU's own eigenpairs (sne_freigs on the same graph: the kernels and
      inputs of the batch), which isolates the sketch of Alg. 4;
    * freigs against the oracle's freigs: the magnitudes of the eight
      eigenvalues of largest magnitude within 1e-5 (relative to the largest);
    * the SBM graphs, whose spectrum is gapped at k, also against the fully
      independent oracle embedding (its own freigs in FP64).  On the
      Chung-Lu graphs the eigenvalues around the k-th are dense, so two
      freigs runs in different arithmetic keep different near-degenerate
      eigenvectors there and the embeddings built from them may differ."""
    graphs, dev, p = batch
    E, s = outputs(graphs)
    ws = sk.batched_workspace(dev, p)
    sk.sne_embed_batched(dev, p, ws, E, s)
    torch.cuda.synchronize()
    for i, g in enumerate(graphs):
        kind = "SBM" if i % 2 == 0 else "Chung-Lu"
        wsf = sk.workspace(g.n, g.nnz, p, sk.SNE_WS_FREIGS)
        U = torch.empty(g.n, K, dtype=torch.float32, device="cuda")
        lam = torch.empty(K, dtype=torch.float64, device="cuda")
        sk.sne_freigs(dev[i], p, wsf, U, lam)
        sk.check_status(wsf)
        Uh, lh = U.cpu().numpy().astype(np.float64), lam.cpu().numpy()
        ref_g = o.embed(g.row_ptr, g.col_idx, g.n, o.Params(k=K, d=D, q=20), U_k=Uh, lam=lh)
        ref = o.embed(g.row_ptr, g.col_idx, g.n, o.Params(k=K, d=D, q=20))
        Ei, sig = E[i].cpu().numpy().astype(np.float64), s[i].cpu().numpy()
        blk = gapped_block(ref_g.sigma)
        sine = o.principal_angle_sines(Ei[:, :blk], ref_g.E[:, :blk]).max()
        srel = np.max(np.abs(sig[:blk] - ref_g.sigma[:blk]) / ref_g.sigma[:blk])
        # freigs orders by |lambda|; +1 and -1 (a bipartite component) tie, so
        # the magnitudes are compared
        lam_err = np.max(np.abs(np.abs(lh[:8]) - np.abs(ref.lam[:8]))) / np.abs(ref.lam[0])
        print(f"graph {i} ({kind}, n={g.n}): vs oracle on GPU eigenpairs: block {blk} sine "
              f"{sine:.1e} sigma {srel:.1e}; freigs top-8 eigenvalues {lam_err:.1e}")
        assert blk >= 1 and sine < 1e-3 and srel < 1e-3, (i, kind)
        assert lam_err < 1e-5, (i, kind)
        if kind == "SBM":
            blk2 = gapped_block(ref.sigma)
            sine2 = o.principal_angle_sines(Ei[:, :blk2], ref.E[:, :blk2]).max()
            srel2 = np.max(np.abs(sig[:blk2] - ref.sigma[:blk2]) / ref.sigma[:blk2])
            print(f"    vs the independent oracle: block {blk2} sine {sine2:.1e} sigma {srel2:.1e}")
            assert blk2 >= 1 and sine2 < 1e-3 and srel2 < 1e-3, i


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


@pytest.mark.parametrize("precision", ["fp16x2", "fp16"])
def test_lockstep_batch_equals_single(sk, batch, precision):
    """Half-precision reconstructions run the batch in lockstep: the first
    halves of all embeddings on the lanes, one persistent tensor-core launch
    for the sketches of every graph, the second halves on the lanes.  Each
    entry of every sketch is computed by the same arithmetic as in a single
    sne_embed, so the embeddings are the same bit for bit, also under a CUDA
    graph."""
    graphs, dev, _ = batch
    p = sk.sne_params_init(D, K, orth=sk.SNE_ORTH_CHOLQR, precision=sk.PRECISIONS[precision])
    E1, s1 = run_single(sk, graphs, dev, p)
    E, s = outputs(graphs)
    ws = sk.batched_workspace(dev, p, 3)
    status = torch.full((len(graphs),), -99, dtype=torch.int32, device="cuda")
    sk.sne_embed_batched(dev, p, ws, E, s, status=status, lanes=3)
    torch.cuda.synchronize()
    assert status.cpu().tolist() == [0] * len(graphs)
    for a, b, sa, sb in zip(E, E1, s, s1):
        assert torch.equal(a, b) and torch.equal(sa, sb)
    for e in E:
        e.zero_()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        sk.sne_embed_batched(dev, p, ws, E, s, lanes=3)
    graph.replay()
    torch.cuda.synchronize()
    for a, b in zip(E, E1):
        assert torch.equal(a, b)


@pytest.mark.parametrize("tn,stages,split", [(128, 2, 1), (128, 0, 4), (256, 2, 1), (256, 3, 8)])
def test_tc_launch_shape_leaves_results_unchanged(sk, batch, monkeypatch, tn, stages, split):
    """The launch shapes the autotuner chooses between (column tile width,
    B stages, column split of the Z core) give the same embedding bit for bit."""
    graphs, dev, _ = batch
    g, G = graphs[1], dev[1]
    p = sk.sne_params_init(D, K, orth=sk.SNE_ORTH_CHOLQR, precision=sk.SNE_FP16X2)
    E0, s0 = run_single(sk, [g], [G], p)
    monkeypatch.setenv("SNE_TC_TN", str(tn))
    monkeypatch.setenv("SNE_TC_STAGES", str(stages))
    monkeypatch.setenv("SNE_TC_SPLIT", str(split))
    E1, s1 = run_single(sk, [g], [G], p)
    assert torch.equal(E0[0], E1[0]) and torch.equal(s0[0], s1[0])


def test_autotune_sketch(sk, batch):
    """The autotuner times the candidate launch shapes of the fused
    tensor-core sketch for one graph and for the batch, keeps the fastest, and
    the embeddings computed afterwards (with the tuned shape) are the ones
    computed before, bit for bit."""
    graphs, dev, _ = batch
    p = sk.sne_params_init(D, K, orth=sk.SNE_ORTH_CHOLQR, precision=sk.SNE_FP16X2)
    E0, s0 = run_single(sk, graphs[:1], dev[:1], p)
    ws = sk.workspace(graphs[0].n, graphs[0].nnz, p, sk.SNE_WS_EMBED)
    r = sk.sne_autotune_sketch(dev[0], p, ws)
    print(f"autotune one graph: {r}")
    assert r["tn"] in (128, 256) and r["stages"] >= 2 and r["split_mult"] in (1, 2, 4)
    assert r["candidates"] > 4 and 0 < r["best_ms"] <= r["default_ms"]
    E1, s1 = run_single(sk, graphs[:1], dev[:1], p)
    assert torch.equal(E0[0], E1[0]) and torch.equal(s0[0], s1[0])
    wsb = sk.batched_workspace(dev, p, 3)
    E, s = outputs(graphs)
    rb = sk.sne_autotune_sketch(dev, p, wsb, lanes=0, E=E, sigma=s)
    print(f"autotune batch of {len(dev)}: {rb}")
    assert 0 < rb["best_ms"] <= rb["default_ms"]
    assert rb["lanes"] in (4, 8, 12, 16) and rb["batch_ms"] > 0
    for e in E:
        e.zero_()
    sk.sne_embed_batched(dev, p, wsb, E, s)  # lanes = 0: the tuned count
    torch.cuda.synchronize()
    assert torch.equal(E[0], E0[0])
