#!/usr/bin/env python
"""Benchmark of the SketchNE hot path (Alg. 6 lines 1-5) on GB300.

One step = one full embedding of the workload graph: freigs (Alg. 5) with its
CSR SpMM power iterations, the Eq. 11 factors, the sparse-sign single-pass SVD
(Alg. 3, 4) with the fused trunc_log(M-hat) sketches Y and Z, the small QR /
least-squares / SVD, and E = U_d Sigma_d^(1/2).

Metric: M-hat entries evaluated by the sketches per second, n*v_S + v_O^2 per
step (v_S, v_O = unique sparse-sign coordinates), over the whole step; the
end-to-end embed time is ms_per_step.  Inputs resident in HBM for `value`;
`e2e` repeats the measurement through sne_embed_host (graph in pinned host
memory, copies inside the timed region, E and sigma read back every step).

Default workload "cl1m": Chung-Lu power-law graph, n = 1,000,000, mean degree
20, exponent 2.1, seed 0; T = 10, b = 1, k = 256, d = 128, zeta = 8,
h = 2d + 16, l = d + 1000, q = 20, alpha = 0.5, plain FP32 path.

--impl reference times the FP64 oracle (the CPU reference of this repo) on a
bounded sample of the same workload on the host cores.

Multi-GPU: one process per GPU (torchrun); the path does not shard, so every
rank runs an independent replica (weak scaling) and `value` sums the ranks'
work over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "trunc_log(M̂)·Ω entries/s and end-to-end embed time, mixed vs FP32 plain"
UNIT = "entries/s"

WORKLOADS = {
    "cl1m": dict(kind="chung_lu", n=1_000_000, avg=20.0, gamma=2.1, d=128, k=256, T=10, q=20,
                 label="Chung-Lu n=1M avg-degree 20 gamma 2.1, T=10 b=1 k=256 d=128 zeta=8 "
                       "h=2d+16 l=d+1000 q=20 alpha=0.5, row block 8192"),
    "cl200k": dict(kind="chung_lu", n=200_000, avg=20.0, gamma=2.1, d=128, k=256, T=10, q=20,
                   label="Chung-Lu n=200k avg-degree 20 gamma 2.1, T=10 b=1 k=256 d=128 zeta=8 "
                         "h=2d+16 l=d+1000 q=20 alpha=0.5 (the n=1M workload at 1/5 size, for "
                         "kernel captures)"),
    "sbm4096": dict(kind="sbm", n=4096, d=32, k=128, T=10, q=20,
                    label="SBM n=4096 8 blocks p_in=0.01 p_out=0.001, T=10 b=1 k=128 d=32 zeta=8"),
    "cl10m": dict(kind="chung_lu_device", n=10_000_000, avg=30.0, gamma=2.2, d=128, k=256, T=10,
                  q=20, precision="bf16",
                  label="Chung-Lu n=10M avg-degree 30 gamma 2.2 (drawn on the GPU), T=10 b=1 k=256 "
                        "d=128 zeta=8 h=2d+16 l=d+1000 q=20 alpha=0.5; BF16 reconstruction with "
                        "FP32 accumulation, FP64 Rayleigh-Ritz/QR/SVD"),
    "cl50m": dict(kind="chung_lu_device", n=50_000_000, avg=40.0, gamma=2.1, d=128, k=128, T=10,
                  q=20, precision="fp16",
                  label="Chung-Lu n=50M avg-degree 40 gamma 2.1 (drawn on the GPU), T=10 b=1 k=128 "
                        "d=128 zeta=8 h=2d+16 l=d+1000 q=20 alpha=0.5; FP16 reconstruction with "
                        "FP32 accumulation"),
    "cl1m_a04": dict(kind="chung_lu", n=1_000_000, avg=20.0, gamma=2.1, d=128, k=256, T=10,
                     q=20, alpha=0.4, precision="fp16x2",
                     label="Chung-Lu n=1M avg-degree 20 gamma 2.1, T=10 b=1 k=256 d=128 zeta=8 "
                           "h=2d+16 l=d+1000 q=20 alpha=0.4; FP16 hi/lo pair reconstruction "
                           "against plain FP32"),
    "cl50m_s0": dict(kind="chung_lu_device", n=50_000_000, avg=40.0, gamma=2.1, d=32, k=32, T=5,
                     q=6, alpha=0.45, h=32, precision="fp16x2",
                     label="Chung-Lu n=50M avg-degree 40 gamma 2.1 (drawn on the GPU), the "
                           "very-large-graph setting: s1=0 (h=d=32), k=32, T=5, q=6, alpha=0.45, "
                           "l=d+1000 zeta=8; FP16 hi/lo pair reconstruction against plain FP32"),
    "batch64": dict(kind="batch", count=64, d=64, k=64, T=10, q=20,
                    label="64 graphs, n ~ U[2000, 200000], mean degree ~ U[8, 32], even: 8-block "
                          "SBM p_in/p_out = 10, odd: Chung-Lu gamma 2.1, graph g seeded g; "
                          "T=10 b=1 k=64 d=64 zeta=8 h=2d+16 l=d+1000 q=20, one batched call"),
}


class DeviceDrawnGraph:
    """A graph drawn on the GPU (synth.chung_lu_device): the device CSR, and
    the host arrays on demand."""

    def __init__(self, n, row_ptr, col_idx):
        self.n, self.row_ptr_dev, self.col_idx_dev = n, row_ptr, col_idx
        self.nnz = int(col_idx.numel())

    @property
    def row_ptr(self):
        return self.row_ptr_dev.cpu().numpy()

    @property
    def col_idx(self):
        return self.col_idx_dev.cpu().numpy()


def make_graph(w):
    from paper_2110_12782_gb300 import synth
    if w["kind"] == "chung_lu_device":
        rp, ci = synth.chung_lu_device(w["n"], w["avg"], w["gamma"], seed=0)
        return DeviceDrawnGraph(w["n"], rp, ci)
    if w["kind"] == "batch":
        # the reference arm samples the largest graph of the batch
        return max(synth.batched_mix(w["count"]), key=lambda g: g.n)
    if w["kind"] == "chung_lu":
        return synth.chung_lu(w["n"], w["avg"], w["gamma"], seed=0)
    return synth.sbm(w["n"], 8, 0.01, 0.001, seed=0)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", str(gpu_index)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def profiled_traffic(kernel: str, workload: str):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summary table (profiles/traffic.json), or None when the table has no
    capture of that kernel on that workload."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        tab = json.load(f)
    ent = tab.get(kernel)
    if ent is None or ent.get("workload") != workload:
        return None
    return ent.get("dram_bytes_per_launch")


def measured_peaks() -> tuple[dict, str]:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


# --------------------------------------------------------------------------- algorithmic work
def algorithmic_work(cls: str, n: int, nnz: int, p, v_s: int, v_o: int) -> tuple[float, str, str]:
    """Algorithmic work of one step for a kernel class: bytes for the SpMM (row
    pointers, column indices, the vector d^-a, one read of the dense operand and
    one write of the result per call; the per-nonzero weights the kernel streams
    are derived data and not counted), flops for the
    products (2 n K K' per Gram or tall product, symmetric Grams counted in full)
    and for Eq. 4 (2k per evaluated entry of L'R')."""
    K = p.k + p.s_eig
    h, l, z, k, d = p.h, p.l, min(n, p.zeta), p.k, p.d
    if cls == "spmm":
        calls = 2 * p.q + 2
        per = 8 * (n + 1) + 4 * nnz + 4 * n + 2 * 4 * n * K
        return calls * per, "hbm", "GB/s"
    if cls == "gram":
        flops = (p.q + 2) * n * K * (K + 1) + 2 * n * K * K + n * k * (k + 1) + 2 * n * h * (h + 1)
        return flops, "alu", "TFLOP/s"
    if cls == "tall_gemm":
        flops = (p.q + 2) * 2 * n * K * K + 2 * n * K * k + 2 * (h + l) * z * k * k \
            + 2 * 2 * n * h * h + 2 * n * h * d
        return flops, "alu", "TFLOP/s"
    if cls == "gram_tc":
        # symmetric Grams counted as full products (the kernel skips lower tiles)
        flops = (p.q + 2) * 2 * n * K * K + 2 * n * K * K + 2 * n * k * k + 2 * 2 * n * h * h
        return flops, "tensor_tf32x3", "TFLOP/s"
    if cls == "tall_gemm_tc":
        flops = (p.q + 2) * 2 * n * K * K + 2 * n * K * k + 2 * 2 * n * h * h + 2 * n * h * d
        return flops, "tensor_tf32x3", "TFLOP/s"
    if cls in ("fused_sketch", "fused_sketch_tc"):
        flops = 2 * k * (n * h * z + v_o * l * z)
        return flops, ("tensor" if cls.endswith("_tc") else "alu"), "TFLOP/s"
    return 0.0, "alu", "TFLOP/s"


def device_sms() -> int:
    """SM count of the current device."""
    import torch
    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


def alu_peak_tflops(sm_mhz: float, sms: int) -> float:
    """FP32 FFMA peak: SMs x 128 FP32 lanes x 2 flops x clock."""
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


# --------------------------------------------------------------------------- oracle timing
def oracle_sample_rate(g, p, U_k: np.ndarray, lam: np.ndarray, budget_s: float) -> dict:
    """Eq. 4 in the FP64 oracle on a row sample; entries evaluated per second."""
    from oracle import sketchne_oracle as o
    A = o.adjacency(g.row_ptr, g.col_idx, g.n)
    deg = o.degrees(A)
    fac = o.netmf_factors(U_k, lam, deg, o.volume(A), p.alpha, p.T, p.b)
    S = o.gen_sparse_sign(g.n, p.h, p.zeta, p.seed, o.STREAM_S)
    v = len(S.p)
    rows, done, spent = 512, 0, 0.0
    rng = np.random.default_rng(0)
    while spent < budget_s:
        sel = np.sort(rng.choice(g.n, size=min(rows, g.n), replace=False))
        t0 = time.perf_counter()
        o.sketch_Y_rows(fac.Lp[sel], fac.Rp, S)
        spent += time.perf_counter() - t0
        done += len(sel)
        rows = min(rows * 2, 16384)
    return {"value": done * v / spent, "rows": done, "seconds": spent, "v": v}


def sketch_error_vs_oracle(sk, g, G, p, U, lam, Uh, lh, op, precisions, rows=1024) -> dict:
    """Relative Frobenius error of Y = trunc_log(L'R'(:, p)) S (Eq. 4) on a
    seeded sample of rows against the FP64 oracle, for each reconstruction
    precision, from the same eigenpairs (this run's freigs), so that the
    comparison isolates the sketch arithmetic."""
    import torch
    from oracle import sketchne_oracle as o
    sel = np.sort(np.random.default_rng(1).choice(g.n, size=min(rows, g.n), replace=False))
    A = o.adjacency(g.row_ptr, g.col_idx, g.n)
    fac = o.netmf_factors(Uh, lh, o.degrees(A), o.volume(A), op.alpha, op.T, op.b)
    S = o.gen_sparse_sign(g.n, op.h, op.zeta, op.seed, o.STREAM_S)
    ref = o.sketch_Y_rows(fac.Lp[sel], fac.Rp, S)
    out = {"rows": int(len(sel)), "seed": 1, "metric": "relative Frobenius error of Y rows"}
    for prec in precisions:
        q = sk.sne_params_init(p.d, p.k, q=p.q, T=p.T, precision=sk.PRECISIONS[prec], orth=p.orth)
        wss = sk.workspace(g.n, g.nnz, q, sk.SNE_WS_SKETCH)
        Y = torch.empty(g.n, q.h, dtype=torch.float32, device="cuda")
        sk.sne_sketch_from_factors(G, q, U, lam, wss, Y=Y)
        sk.check_status(wss, f"sketch {prec}")
        got = Y[torch.as_tensor(sel, device="cuda")].cpu().double().numpy()
        out[prec] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        del wss, Y
    return out


def cpu_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


# --------------------------------------------------------------------------- multi-rank
def max_over_ranks(x: float, world: int) -> float:
    """The largest of the ranks' values: the job takes as long as its slowest
    rank.  NCCL reduces device tensors, gloo host tensors."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_step: float, world: int, steps: int, total_ms: float) -> float:
    """Whole-job throughput: every rank processes `units_per_step` per step (an
    independent replica), over the slowest rank's total time."""
    return world * steps * units_per_step / (total_ms / 1e3)


# --------------------------------------------------------------------------- reference arm
def run_reference(args, rank: int) -> None:
    if rank != 0:
        return
    from oracle import sketchne_oracle as o
    w = WORKLOADS[args.workload]
    g = make_graph(w)
    p = o.Params(k=w["k"], d=w["d"], q=w["q"], T=w["T"]).resolved()
    A = o.adjacency(g.row_ptr, g.col_idx, g.n)
    # factors for the sampled sketch: freigs with a bounded number of power
    # iterations (the sketch arithmetic timed below does not depend on q)
    X = o.normalized_operator(A, p.alpha)
    U, lam = o.freigs(X, p.k, min(p.q, 1), p.s_eig, p.seed)
    budget = args.ref_step_seconds
    for _ in range(args.warmup):
        oracle_sample_rate(g, p, U, lam, budget * 0.2)
    vals, secs = [], []
    for _ in range(args.steps):
        r = oracle_sample_rate(g, p, U, lam, budget)
        vals.append(r["value"])
        secs.append(r["seconds"])
    value = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * float(np.mean(secs)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w["label"], "sample": "Eq. 4 rows of trunc_log(L'R'(:,p))S on "
                   f"random row samples, ~{budget:.0f} s of CPU work per step",
                   "parallelism": "host cores"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                         "sample": f"row samples of Eq. 4, {budget:.0f} s per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- our arm
def run_ours(args, rank: int, world: int) -> None:
    import torch
    import torch.distributed as dist

    from paper_2110_12782_gb300 import build
    from paper_2110_12782_gb300 import sketchne as sk

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build.build()
    w = WORKLOADS[args.workload]
    g = make_graph(w)
    prec = sk.PRECISIONS[args.precision]
    orth = {"eigsvd": sk.SNE_ORTH_EIGSVD, "cholqr": sk.SNE_ORTH_CHOLQR}[args.orth]
    p = sk.sne_params_init(w["d"], w["k"], q=w["q"], T=w["T"], precision=prec, orth=orth,
                           row_block=8192)
    sms = device_sms()
    G = sk.DeviceGraph.from_numpy(g.row_ptr, g.col_idx)
    ws = sk.workspace(g.n, g.nnz, p, sk.SNE_WS_EMBED)
    E = torch.empty(g.n, p.d, dtype=torch.float32, device="cuda")
    sig = torch.empty(p.d, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2

    def step():
        sk.sne_embed(G, p, ws, E, sig)

    if args.profile_run:
        # one embed (for ncu launch lists and kernel captures), no timing
        step()
        sk.check_status(ws, "profile run")
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"profile_run": "ok", "workload": w["label"], "precision": args.precision}))
        return
    for _ in range(args.warmup):
        step()
    sk.check_status(ws, "warm-up")
    st = sk.sne_stats_read(ws)
    entries = g.n * st.v_s + st.v_o * st.v_o

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- timed region: inputs resident in HBM, L2 flushed between steps
    clocks = ClockSampler(local)
    times = []
    launches0 = sk.sne_kernel_launches()
    for _ in range(args.steps):
        flush.zero_()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        step()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    launches = sk.sne_kernel_launches() - launches0
    clk = clocks.stop()
    sk.check_status(ws, "timed steps")
    total_ms = max_over_ranks(float(sum(times)), world)
    value = job_value(entries, world, args.steps, total_ms)

    # ---- per-kernel-class times (events on the launching stream), same steps
    sk.sne_profile_start()
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        step()
    prof = sk.sne_profile_stop()
    prof_total = sum(v[2] for v in prof.values())

    # ---- end to end through the public host-buffer entry point
    h_rp = torch.from_numpy(g.row_ptr).pin_memory()
    h_ci = torch.from_numpy(g.col_idx).pin_memory()
    h_E = torch.empty(g.n, p.d, dtype=torch.float32).pin_memory()
    h_sig = torch.empty(p.d, dtype=torch.float64).pin_memory()
    ws_h = sk.workspace(g.n, g.nnz, p, sk.SNE_WS_EMBED_HOST)
    sk.sne_embed_host(h_rp, h_ci, None, g.n, p, ws_h, h_E, h_sig)
    torch.cuda.synchronize()
    e2e_t = []
    for _ in range(args.steps):
        flush.zero_()
        barrier()
        t0 = time.perf_counter()
        sk.sne_embed_host(h_rp, h_ci, None, g.n, p, ws_h, h_E, h_sig)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    sk.check_status(ws_h, "e2e steps")
    e2e_total = max_over_ranks(float(sum(e2e_t)), world)
    h2d = 8 * (g.n + 1) + 4 * g.nnz
    d2h = 4 * g.n * p.d + 8 * p.d

    # ---- roofline of the dominant kernel class
    peaks, peak_kind = measured_peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][2])[0] if prof else None
    roofline = None
    if dom:
        calls, nlaunch, ms = prof[dom]
        work, bound, unit = algorithmic_work(dom, g.n, g.nnz, p, st.v_s, st.v_o)
        per_step_ms = ms / args.steps
        if work > 0:
            if bound == "hbm":
                achieved = work / (per_step_ms / 1e3) / 1e9
                peak = float(peaks["hbm_gbs"])
            elif bound == "tensor":
                achieved = work / (per_step_ms / 1e3) / 1e12
                peak = float(peaks["bf16_tflops"])
            elif bound == "tensor_tf32x3":
                # FP32-accurate products as three TF32 passes: ceiling = TF32 peak / 3,
                # TF32 peak = measured BF16 peak x nominal 1.1 / 2.25
                achieved = work / (per_step_ms / 1e3) / 1e12
                peak = float(peaks["bf16_tflops"]) * (1.1 / 2.25) / 3.0
            else:
                achieved = work / (per_step_ms / 1e3) / 1e12
                peak = alu_peak_tflops(float(peaks.get("sm_max_mhz", 2070.0)), sms)
            roofline = {"kernel": dom, "bound": bound, "achieved": achieved, "peak": peak,
                        "unit": unit, "frac": achieved / peak, "traffic": profiled_traffic(dom, args.workload),
                        "peak_source": {"alu": f"derived: {sms} SMs x 128 FP32 lanes x 2 x max SM clock",
                                        "tensor_tf32x3": f"{peak_kind} bf16 x 1.1/2.25 / 3"}.get(
                                            bound, f"{peak_kind}"),
                        "share_of_step": ms / prof_total if prof_total else None}

    # ---- mixed precision (half-precision reconstruction) on the same graph and steps
    mixed = None
    if not args.no_mixed and prec == sk.SNE_FP32:
        pm = sk.sne_params_init(w["d"], w["k"], q=w["q"], T=w["T"],
                                precision=sk.PRECISIONS[args.mixed_precision], orth=orth,
                                row_block=8192)
        wsm = sk.workspace(g.n, g.nnz, pm, sk.SNE_WS_EMBED)
        Em = torch.empty_like(E)
        sigm = torch.empty_like(sig)
        # launch shape of the fused tensor-core sketch, timed over its candidates
        tune = sk.sne_autotune_sketch(G, pm, wsm)
        for _ in range(args.warmup):
            sk.sne_embed(G, pm, wsm, Em, sigm)
        mt = []
        for _ in range(args.steps):
            flush.zero_()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            sk.sne_embed(G, pm, wsm, Em, sigm)
            e1.record()
            torch.cuda.synchronize()
            mt.append(e0.elapsed_time(e1))
        sk.check_status(wsm, "mixed steps")
        sk.sne_profile_start()
        for _ in range(args.steps):
            flush.zero_()
            torch.cuda.synchronize()
            sk.sne_embed(G, pm, wsm, Em, sigm)
        profm = sk.sne_profile_stop()
        # agreement of the two embeddings on the leading singular values
        s32 = sig.cpu().numpy()
        s16 = sigm.cpu().numpy()
        mixed_total = max_over_ranks(float(sum(mt)), world)
        mixed = {"precision": args.mixed_precision, "ms_per_step": mixed_total / args.steps,
                 "autotune": tune,
                 "value": job_value(entries, world, args.steps, mixed_total),
                 "sigma_rel_diff_vs_fp32": float(np.max(np.abs(s16 - s32) / np.abs(s32))),
                 "kernel_ms_per_step": {k: v[2] / args.steps for k, v in
                                        sorted(profm.items(), key=lambda kv: -kv[1][2])}}
        if "fused_sketch_tc" in profm:
            ms = profm["fused_sketch_tc"][2] / args.steps
            work, _, _ = algorithmic_work("fused_sketch_tc", g.n, g.nnz, p, st.v_s, st.v_o)
            # hi/lo pair operands: three tensor-core products per entry
            products = 3 if args.mixed_precision.endswith("x2") else 1
            ach = products * work / (ms / 1e3) / 1e12
            # the kernel runs inside seconds-long embeddings: sustained peak
            pk = float(peaks.get("bf16_tflops_sustained", peaks["bf16_tflops"]))
            mixed["roofline_fused_sketch"] = {
                "kernel": "fused_sketch_tc", "bound": "tensor", "achieved": ach, "peak": pk,
                "unit": "TFLOP/s", "frac": ach / pk, "products_per_entry": products,
                "algorithmic_tflops": work / (ms / 1e3) / 1e12,
                "peak_source": f"{peak_kind} bf16 dense sustained (FP16 has the same tensor rate)",
                "ms_per_step": ms}

    # ---- spectral propagation (Alg. 6 line 6) of this run's embedding
    propagation = None
    if not args.no_extra:
        propagation = measure_propagation(sk, G, E, g.n, g.nnz, args.steps, args.warmup, flush,
                                          peaks, peak_kind)

    cpu = None
    accuracy = None
    if rank == 0 and not args.no_cpu_baseline:
        U = torch.empty(g.n, p.k, dtype=torch.float32, device="cuda")
        lam = torch.empty(p.k, dtype=torch.float64, device="cuda")
        ws_f = sk.workspace(g.n, g.nnz, p, sk.SNE_WS_FREIGS)
        sk.sne_freigs(G, p, ws_f, U, lam)
        sk.check_status(ws_f, "freigs")
        del ws_f
        from oracle import sketchne_oracle as o
        op = o.Params(k=p.k, d=p.d, q=p.q, T=p.T, h=p.h, l=p.l).resolved()
        Uh, lh = U.cpu().double().numpy(), lam.cpu().numpy()
        r = oracle_sample_rate(g, op, Uh, lh, args.cpu_seconds)
        cpu = {"value": r["value"], "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
               "sample": f"Eq. 4 (trunc_log(L'R'(:,p))S, FP64) on {r['rows']} random rows, "
                         f"{r['seconds']:.1f} s, factors from this run's freigs"}
        accuracy = sketch_error_vs_oracle(sk, g, G, p, U, lam, Uh, lh, op,
                                          ["fp32"] + ([] if args.no_mixed else [args.mixed_precision]))

    # ---- the other workloads of the configuration list, fewer steps each
    extra = None
    if not args.no_extra and args.workload == "cl1m":
        del ws, E, sig, flush
        torch.cuda.empty_cache()
        ek, ew = min(args.steps, 3), max(3, min(args.warmup, 3))
        extra = {}
        for name in ("cl10m", "cl1m_a04", "cl50m_s0"):
            extra[name] = measure_single(args, name, ek, ew) if rank == 0 or world > 1 else None
        bline = measure_batch(args, rank, world, "batch64", "fp16", ek, ew)
        if bline is not None:
            extra["batch64"] = {k: bline[k] for k in ("value", "ms_per_step", "steps", "warmup",
                                                       "config", "e2e", "gpu_launches", "autotune",
                                                       "kernel_ms_per_step_summed_over_lanes")
                                if k in bline}
            # the same batch in plain FP32 and with FP16 hi/lo pairs
            for prec_b in ("fp32", "fp16x2"):
                bl = measure_batch(args, rank, world, "batch64", prec_b, ek, ew)
                if bl is not None:
                    extra["batch64"][prec_b] = {k: bl[k] for k in ("value", "ms_per_step", "autotune")
                                                if k in bl}
            if rank == 0 and not args.no_cpu_baseline:
                extra["batch64"]["error_vs_oracle"] = batch_error_vs_oracle(
                    "batch64", ["fp16", "fp16x2", "fp32"])
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == sk.SNE_FP32 else args.precision,
            "data": "synthetic",
            "config": {"workload": w["label"], "n": g.n, "nnz": g.nnz, "v_S": st.v_s, "v_O": st.v_o,
                       "entries_per_step": entries, "precision": args.precision, "orth": args.orth,
                       "l2": "flushed between steps (256 MB write)",
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "e2e": {"value": job_value(entries, world, args.steps, 1e3 * e2e_total), "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": 1e3 * e2e_total / args.steps},
            "gpu_launches": int(launches),
            "roofline": roofline,
            "mixed": mixed,
            "propagation": propagation,
            "error_vs_oracle": accuracy,
            "workloads": extra,
            "cpu_baseline": cpu,
            "clocks": clk,
            "kernel_ms_per_step": {k: v[2] / args.steps for k, v in sorted(prof.items(), key=lambda kv: -kv[1][2])},
        }
        print(json.dumps(line), flush=True)


def measure_propagation(sk, G, E, n, nnz, steps, warmup, flush, peaks, peak_kind,
                        p_steps=10, theta=0.5, mu=0.2) -> dict:
    """sne_spectral_propagate (p = 10, theta = 0.5, mu = 0.2) of the embedding E,
    L2 flushed before each call.  Algorithmic bytes of one Chebyshev step (two
    passes): the CSR arrays and 1/d twice, and 4 n d bytes for each of the
    operand read and result write of the first pass and the operand read, the
    two earlier terms, the result write and the read and write of the running
    sum of the second."""
    import torch
    d = E.shape[1]
    wsp = sk.propagate_workspace(n, d)
    Ep = torch.empty_like(E)
    times = []
    for it in range(warmup + steps):
        Ep.copy_(E)
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        sk.sne_spectral_propagate(G, Ep, wsp, steps=p_steps, theta=theta, mu=mu)
        e1.record()
        torch.cuda.synchronize()
        if it >= warmup:
            times.append(e0.elapsed_time(e1))
    sk.check_status(wsp, "propagate")
    ms = float(np.mean(times))
    per_step = 2 * (8 * (n + 1) + 4 * nnz + 4 * n) + 8 * 4 * n * d
    work = p_steps * per_step + 2 * 4 * n * d
    ach = work / (ms / 1e3) / 1e9
    peak = float(peaks["hbm_gbs"])
    del wsp, Ep
    return {"ms": ms, "steps": p_steps, "theta": theta, "mu": mu, "d": d, "calls_timed": steps,
            "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                         "frac": ach / peak, "algorithmic_bytes": work, "peak_source": peak_kind}}


def workload_params(sk, w, precision="fp32"):
    """sne_params of a workload (alpha 0.5 and h = 2d + 16 unless it says otherwise)."""
    p = sk.sne_params_init(w["d"], w["k"], q=w["q"], T=w["T"], precision=sk.PRECISIONS[precision],
                           orth=sk.SNE_ORTH_CHOLQR, alpha=w.get("alpha", 0.5))
    if "h" in w:
        p.h = w["h"]
    return p


def measure_single(args, workload: str, steps: int, warmup: int) -> dict:
    """One graph of a large workload at its configured (mixed) precision and
    at plain FP32, steps embeddings each after `warmup` untimed ones (L2
    flushed between steps); with the CPU-baseline leg on, the error of Y on a
    seeded sample of 100,000 rows against the FP64 oracle from this run's
    eigenpairs."""
    import torch

    from paper_2110_12782_gb300 import sketchne as sk
    w = WORKLOADS[workload]
    t0 = time.perf_counter()
    g = make_graph(w)
    gen_s = time.perf_counter() - t0
    if isinstance(g, DeviceDrawnGraph):
        G = sk.DeviceGraph(g.row_ptr_dev, g.col_idx_dev)
    else:
        G = sk.DeviceGraph.from_numpy(g.row_ptr, g.col_idx)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    out = {"workload": w["label"], "n": g.n, "nnz": g.nnz, "steps": steps, "warmup": warmup,
           "graph_generation_s": gen_s, "l2": "flushed between steps (256 MB write)"}
    sigmas = {}
    for prec in (w["precision"], "fp32"):
        p = workload_params(sk, w, prec)
        ws = sk.workspace(g.n, g.nnz, p, sk.SNE_WS_EMBED)
        E = torch.empty(g.n, p.d, dtype=torch.float32, device="cuda")
        sig = torch.empty(p.d, dtype=torch.float64, device="cuda")
        for _ in range(warmup):
            sk.sne_embed(G, p, ws, E, sig)
        sk.check_status(ws, f"{workload} {prec}")
        st = sk.sne_stats_read(ws)
        entries = g.n * st.v_s + st.v_o * st.v_o
        times = []
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            sk.sne_embed(G, p, ws, E, sig)
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        sk.check_status(ws, f"{workload} {prec} timed")
        sk.sne_profile_start()
        flush.zero_()
        torch.cuda.synchronize()
        sk.sne_embed(G, p, ws, E, sig)
        prof = sk.sne_profile_stop()
        ms = float(np.mean(times))
        out[prec] = {"ms_per_step": ms, "value": entries / (ms / 1e3), "unit": UNIT,
                     "entries_per_step": entries,
                     "kernel_ms_per_step": {k: v[2] for k, v in sorted(prof.items(), key=lambda kv: -kv[1][2])}}
        sigmas[prec] = sig.cpu().numpy()
        del ws, E, sig
        torch.cuda.empty_cache()
    out["sigma_rel_diff_vs_fp32"] = float(np.max(np.abs(sigmas[w["precision"]] - sigmas["fp32"]) /
                                                 np.abs(sigmas["fp32"])))
    if not args.no_cpu_baseline:
        out["error_vs_oracle"] = large_sample_error(sk, g, G, w, [w["precision"], "fp32"])
    del G, g, flush
    torch.cuda.empty_cache()
    return out


def large_sample_error(sk, g, G, w, precisions, rows=100_000) -> dict:
    """Part of the CPU-baseline leg: Y = trunc_log(L'R'(:, p)) S on a seeded
    sample of rows, FP64 oracle (factors of Eq. 11 for the sampled rows and
    the columns p only, the Gram of U summed in row chunks) against the
    library at each precision, from the same eigenpairs."""
    import torch
    from oracle import sketchne_oracle as o
    p = workload_params(sk, w)
    ws = sk.workspace(g.n, g.nnz, p, sk.SNE_WS_FREIGS)
    U = torch.empty(g.n, p.k, dtype=torch.float32, device="cuda")
    lam = torch.empty(p.k, dtype=torch.float64, device="cuda")
    sk.sne_freigs(G, p, ws, U, lam)
    sk.check_status(ws, "freigs")
    del ws
    t0 = time.perf_counter()
    Uh, lh = U.cpu().numpy(), lam.cpu().numpy()
    deg = np.diff(g.row_ptr).astype(np.float64)
    sel = np.sort(np.random.default_rng(1).choice(g.n, size=min(rows, g.n), replace=False))
    S = o.gen_sparse_sign(g.n, p.h, p.zeta, p.seed, o.STREAM_S)
    Lr, Rc = o.netmf_factor_rows(Uh, lh, deg, float(deg.sum()), p.alpha, p.T, p.b, sel, S.p)
    ref = o.sketch_Y_rows_at(Lr, Rc, S)
    out = {"rows": int(len(sel)), "seed": 1, "metric": "relative Frobenius error of Y rows",
           "oracle_s": time.perf_counter() - t0}
    del Uh
    for prec in precisions:
        q = workload_params(sk, w, prec)
        wss = sk.workspace(g.n, g.nnz, q, sk.SNE_WS_SKETCH)
        Y = torch.empty(g.n, q.h, dtype=torch.float32, device="cuda")
        sk.sne_sketch_from_factors(G, q, U, lam, wss, Y=Y)
        sk.check_status(wss, f"sketch {prec}")
        got = Y[torch.as_tensor(sel, device="cuda")].cpu().double().numpy()
        out[prec] = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
        del wss, Y
        torch.cuda.empty_cache()
    del U, lam
    torch.cuda.empty_cache()
    return out


def run_ours_batch(args, rank: int, world: int) -> None:
    """The many-graphs workload as the main line."""
    line = measure_batch(args, rank, world, args.workload, args.precision, args.steps, args.warmup)
    if rank == 0:
        print(json.dumps(line), flush=True)


def batch_error_vs_oracle(workload: str, precisions, count: int = 4) -> dict:
    """Part of the CPU-baseline leg: the embeddings of the `count` smallest
    graphs of the batch (sne_embed, the per-graph pipeline the batched call
    runs on its lanes) against the FP64 oracle's embedding with the same
    parameters: the largest relative error of the singular values and the
    largest principal-angle sine over the leading block whose relative gap is
    at least 1e-2, per precision (maximum over the graphs)."""
    import torch
    from oracle import sketchne_oracle as o
    from paper_2110_12782_gb300 import synth
    from paper_2110_12782_gb300 import sketchne as sk
    w = WORKLOADS[workload]
    graphs = sorted(synth.batched_mix(w["count"]), key=lambda g: g.n)[:count]
    out = {"graphs": [int(g.n) for g in graphs],
           "metric": "max over graphs: sigma relative error, principal-angle sine (leading gapped block)"}
    refs = [o.embed(g.row_ptr, g.col_idx, g.n, o.Params(k=w["k"], d=w["d"], q=w["q"], T=w["T"]))
            for g in graphs]
    for prec in precisions:
        se, ss = 0.0, 0.0
        for g, ref in zip(graphs, refs):
            p = sk.sne_params_init(w["d"], w["k"], q=w["q"], T=w["T"], precision=sk.PRECISIONS[prec],
                                   orth=sk.SNE_ORTH_CHOLQR)
            G = sk.DeviceGraph.from_numpy(g.row_ptr, g.col_idx)
            ws = sk.workspace(g.n, g.nnz, p, sk.SNE_WS_EMBED)
            E = torch.empty(g.n, p.d, dtype=torch.float32, device="cuda")
            sig = torch.empty(p.d, dtype=torch.float64, device="cuda")
            sk.sne_embed(G, p, ws, E, sig)
            sk.check_status(ws, f"batch graph {prec}")
            s_ = sig.cpu().numpy()
            blk = 0
            for j in range(1, min(p.d, len(ref.sigma) - 1) + 1):
                if (ref.sigma[j - 1] - ref.sigma[j]) / ref.sigma[j - 1] >= 1e-2:
                    blk = j
            if blk == 0:
                continue
            se = max(se, float(np.max(np.abs(s_[:blk] - ref.sigma[:blk]) / ref.sigma[:blk])))
            ss = max(ss, float(o.principal_angle_sines(E.cpu().double().numpy()[:, :blk],
                                                       ref.E[:, :blk]).max()))
        out[prec] = {"sigma_rel": se, "sine": ss}
    return out


def measure_batch(args, rank: int, world: int, workload: str, precision: str, steps: int,
                  warmup: int) -> dict:
    """The many-graphs workload: every step embeds the whole batch with one
    sne_embed_batched call, replayed from a CUDA graph."""
    import torch
    import torch.distributed as dist

    from paper_2110_12782_gb300 import build, synth
    from paper_2110_12782_gb300 import sketchne as sk

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    build.build()
    w = WORKLOADS[workload]
    graphs = synth.batched_mix(w["count"])
    orth = {"eigsvd": sk.SNE_ORTH_EIGSVD, "cholqr": sk.SNE_ORTH_CHOLQR}[args.orth]
    prec = sk.PRECISIONS[precision]
    p = sk.sne_params_init(w["d"], w["k"], q=w["q"], T=w["T"], precision=prec, orth=orth)
    dev = [sk.DeviceGraph.from_numpy(g.row_ptr, g.col_idx) for g in graphs]
    E = [torch.empty(g.n, p.d, dtype=torch.float32, device="cuda") for g in graphs]
    sig = [torch.empty(p.d, dtype=torch.float64, device="cuda") for _ in graphs]
    status = torch.zeros(len(graphs), dtype=torch.int32, device="cuda")
    ws = sk.batched_workspace(dev, p)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    # v_S, v_O of every graph (one embedding each, untimed)
    entries = 0
    for g, G, e, sg in zip(graphs, dev, E, sig):
        wsg = sk.workspace(g.n, g.nnz, p, sk.SNE_WS_EMBED)
        sk.sne_embed(G, p, wsg, e, sg)
        st = sk.sne_stats_read(wsg)
        entries += g.n * st.v_s + st.v_o * st.v_o
        del wsg
    # half-precision reconstructions: the batch's sketches run as one
    # persistent launch, its shape timed over the candidates first
    tune = sk.sne_autotune_sketch(dev, p, ws, E=E, sigma=sig) if prec != sk.SNE_FP32 else None
    sk.sne_embed_batched(dev, p, ws, E, sig, status=status)  # creates the lanes
    torch.cuda.synchronize()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg):
        sk.sne_embed_batched(dev, p, ws, E, sig, status=status)
    for _ in range(warmup):
        cg.replay()
    torch.cuda.synchronize()
    if int(status.abs().sum()) != 0:
        raise RuntimeError(f"batch status {status.tolist()}")

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    times = []
    launches0 = sk.sne_kernel_launches()
    for _ in range(steps):
        flush.zero_()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        cg.replay()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    # kernels in one batch (a replay launches what the capture enqueued)
    l0 = sk.sne_kernel_launches()
    sk.sne_embed_batched(dev, p, ws, E, sig, status=status)
    torch.cuda.synchronize()
    launches = (sk.sne_kernel_launches() - l0) * steps
    total_ms = max_over_ranks(float(sum(times)), world)
    value = job_value(entries, world, steps, total_ms)
    # per-class times (eager batched calls; lanes overlap, so shares are of summed kernel time)
    sk.sne_profile_start()
    for _ in range(steps):
        flush.zero_()
        torch.cuda.synchronize()
        sk.sne_embed_batched(dev, p, ws, E, sig, status=status)
    torch.cuda.synchronize()
    prof = sk.sne_profile_stop()
    # end to end: graphs from pinned host memory, embeddings back to the host
    h_rp = [torch.from_numpy(g.row_ptr).pin_memory() for g in graphs]
    h_ci = [torch.from_numpy(g.col_idx).pin_memory() for g in graphs]
    d_rp = [torch.empty_like(t, device="cuda") for t in h_rp]
    d_ci = [torch.empty_like(t, device="cuda") for t in h_ci]
    devh = [sk.DeviceGraph(r, c) for r, c in zip(d_rp, d_ci)]
    h_E = [torch.empty(g.n, p.d, dtype=torch.float32).pin_memory() for g in graphs]
    h_s = [torch.empty(p.d, dtype=torch.float64).pin_memory() for g in graphs]
    e2e_t = []
    for _ in range(steps):
        flush.zero_()
        barrier()
        t0 = time.perf_counter()
        for a, b in zip(d_rp + d_ci, h_rp + h_ci):
            a.copy_(b, non_blocking=True)
        sk.sne_embed_batched(devh, p, ws, E, sig, status=status)
        for a, b in zip(h_E + h_s, E + sig):
            a.copy_(b, non_blocking=True)
        torch.cuda.synchronize()
        e2e_t.append(time.perf_counter() - t0)
    e2e_total = max_over_ranks(float(sum(e2e_t)), world)
    h2d = sum(8 * (g.n + 1) + 4 * g.nnz for g in graphs)
    d2h = sum(4 * g.n * p.d + 8 * p.d for g in graphs)
    peaks, peak_kind = measured_peaks()
    dom = max(prof.items(), key=lambda kv: kv[1][2])[0] if prof else None
    prof_total = sum(v[2] for v in prof.values())
    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": total_ms / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == sk.SNE_FP32 else precision, "data": "synthetic",
            "config": {"workload": w["label"], "graphs": len(graphs),
                       "sum_n": int(sum(g.n for g in graphs)),
                       "sum_nnz": int(sum(g.nnz for g in graphs)), "entries_per_step": entries,
                       "precision": precision, "orth": args.orth, "cuda_graph": True,
                       "l2": "flushed between steps (256 MB write)",
                       "parallelism": "replicas" if world > 1 else (
                           "single GPU, stream lanes" if prec == sk.SNE_FP32 else
                           "single GPU, stream lanes; the sketches of all graphs in one "
                           "persistent tensor-core launch")},
            "autotune": tune,
            "e2e": {"value": job_value(entries, world, steps, 1e3 * e2e_total), "unit": UNIT,
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": 1e3 * e2e_total / steps},
            "gpu_launches": int(launches),
            "roofline": {"kernel": dom, "bound": None, "achieved": None, "peak": None,
                         "unit": None, "frac": None, "traffic": None,
                         "note": "lanes overlap; see the single-graph workload "
                         "for per-kernel rooflines", "peak_source": peak_kind},
            "cpu_baseline": None,
            "clocks": clk,
            "kernel_ms_per_step_summed_over_lanes": {
                k: v[2] / steps for k, v in sorted(prof.items(), key=lambda kv: -kv[1][2])},
            "kernel_share": {k: v[2] / prof_total for k, v in prof.items()} if prof_total else None,
        }
    del ws, E, sig, dev, flush
    torch.cuda.empty_cache()
    return line


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cl1m", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32",
                    choices=["fp32", "bf16", "fp16", "bf16x2", "fp16x2"])
    ap.add_argument("--mixed-precision", default="fp16x2",
                    choices=["bf16", "fp16", "bf16x2", "fp16x2"],
                    help="precision of the mixed arm (pairs: hi/lo operands, three products)")
    ap.add_argument("--orth", default="cholqr", choices=["eigsvd", "cholqr"],
                    help="orthonormalization inside freigs (Alg. 5): Cholesky QR (default) or "
                         "eigSVD as printed; both give the same subspace")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-step-seconds", type=float, default=8.0)
    ap.add_argument("--profile-run", action="store_true",
                    help="run one embedding and exit (for ncu)")
    ap.add_argument("--no-mixed", action="store_true",
                    help="skip the mixed-precision comparison steps")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the n=10M and 64-graph workloads measured after the main line")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if WORKLOADS[args.workload]["kind"] == "batch":
        run_ours_batch(args, rank, world)
    else:
        run_ours(args, rank, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
