"""The seeded graph generators against their recipes.  These graphs are the
only inputs the oracle and the CUDA path share, so their structure is pinned
here: symmetric CSR without self-loops or repeats, SBM block densities within
binomial bounds, the Chung-Lu power-law tail and degree order, the batch mix."""
import numpy as np
import pytest

from paper_2110_12782_gb300 import synth


def check_csr(g):
    rp, ci = g.row_ptr, g.col_idx
    assert rp.dtype == np.int64 and ci.dtype == np.int32
    assert rp[0] == 0 and rp[-1] == len(ci) and np.all(np.diff(rp) >= 0)
    rows = np.repeat(np.arange(g.n), np.diff(rp))
    assert np.all(ci >= 0) and np.all(ci < g.n)
    assert not np.any(rows == ci)
    same_row = rows[1:] == rows[:-1]
    assert np.all(ci[1:][same_row] > ci[:-1][same_row])  # sorted, no repeats
    fwd = rows.astype(np.int64) * g.n + ci
    rev = ci.astype(np.int64) * g.n + rows
    assert np.array_equal(np.sort(fwd), np.sort(rev))  # both directions stored
    return rows


def test_sbm_block_densities_and_seeding():
    n, B, p_in, p_out = 4096, 8, 0.01, 0.001
    g = synth.sbm(n, B, p_in, p_out, seed=0)
    rows = check_csr(g)
    blk = n // B
    inside = (rows // blk) == (g.col_idx // blk)
    e_in, e_out = inside.sum() // 2, (~inside).sum() // 2
    pairs_in = B * blk * (blk - 1) // 2
    pairs_out = n * (n - 1) // 2 - pairs_in
    for e, m, p in ((e_in, pairs_in, p_in), (e_out, pairs_out, p_out)):
        assert abs(e - m * p) < 5 * np.sqrt(m * p * (1 - p))
    assert g.nnz == 35782  # the parity workload's size, as documented
    assert np.array_equal(g.col_idx, synth.sbm(n, B, p_in, p_out, seed=0).col_idx)
    assert not np.array_equal(g.col_idx, synth.sbm(n, B, p_in, p_out, seed=1).col_idx)


def test_chung_lu_power_law_and_degree_order():
    n, avg, gamma = 100_000, 20.0, 2.1
    g = synth.chung_lu(n, avg, gamma, seed=0)
    check_csr(g)
    deg = g.degrees()
    mean = g.nnz / n
    assert avg <= mean <= 1.01 * avg
    assert deg.max() <= 1.1 * np.sqrt(n * avg)  # weights capped at sqrt(n avg)
    # P(deg >= x) ~ x^-(gamma - 1) between the mean and the cap
    slope = np.log((deg >= 400).mean() / (deg >= 40).mean()) / np.log(10.0)
    assert abs(slope + (gamma - 1.0)) < 0.15
    # ids sorted by expected degree: the first 1% are hubs
    assert deg[: n // 100].mean() > 50 * deg[n // 2:].mean()


def test_batched_mix_alternates_families_within_ranges():
    graphs = synth.batched_mix(count=6, n_lo=2000, n_hi=5000, seed=3)
    assert len(graphs) == 6
    for g_id, g in enumerate(graphs):
        check_csr(g)
        assert 2000 <= g.n <= 5000
        assert g.name.startswith("sbm" if g_id % 2 == 0 else "chung_lu")
        assert 8.0 * 0.7 <= g.nnz / g.n <= 32.0 * 1.3


def test_closed_form_graphs():
    k = synth.complete_graph(7)
    check_csr(k)
    assert np.all(k.degrees() == 6)
    u = synth.complete_bipartite_union([(2, 3), (1, 4)])
    check_csr(u)
    assert u.n == 10 and u.nnz == 2 * (2 * 3 + 1 * 4)
    assert list(u.degrees()) == [3, 3, 2, 2, 2, 4, 1, 1, 1, 1]


def test_chung_lu_device_recipe_on_cpu():
    """The torch form of the Chung-Lu recipe (run here on the CPU): a
    symmetric CSR without self-loops or repeated edges, at least the target
    number of edges, and the same expected-degree order as the NumPy form."""
    torch = pytest.importorskip("torch")
    n, avg = 50_000, 20.0
    rp, ci = synth.chung_lu_device(n, avg, 2.1, seed=3, device="cpu")
    rp, ci = rp.numpy(), ci.numpy().astype(np.int64)
    nnz = int(rp[-1])
    assert rp[0] == 0 and np.all(np.diff(rp) >= 0) and len(ci) == nnz
    assert nnz >= n * avg and nnz < 1.02 * n * avg
    rows = np.repeat(np.arange(n), np.diff(rp))
    assert np.all(rows != ci)
    key = rows * n + ci
    assert np.all(np.diff(key) > 0)                      # sorted, no repeats
    assert np.array_equal(np.sort(ci * n + rows), key)  # symmetric
    deg = np.diff(rp)
    ref = synth.chung_lu(n, avg, 2.1, seed=3).degrees()
    # same weights: the hubs are the low ids in both, with matching mean degrees
    assert abs(deg[:100].mean() / ref[:100].mean() - 1.0) < 0.1
    assert deg.argmax() < 50  # the largest weights are capped alike
