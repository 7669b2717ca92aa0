#!/usr/bin/env python3
"""Benchmark of the SF-GRASS hot path on one GB300: filter + score throughput.

Workload (one step): the 3-D 6-neighbour grid 128^3 (2,097,152 nodes, 6,242,304 edges, weights
10^U[-2,2)), K = 32 seeded vectors, 20 weighted-Jacobi sweeps (omega 0.7) on the Laplacian of G and
on that of its maximum spanning tree P, projection, RATIO scores of all 4,145,153 off-tree edges and
the top round(0.05 N) = 104,858 of them (sfg_filter_score + sfg_select_topk). G, P and the off-tree id list are built once before the
timed region (they are the inputs of the filter); every step recomputes everything else.

Metric: filter+score algorithmic GB/s = bytes / step time with
  B_sweep(L)  = 4(N+1) + 8 nnz(L) + 4N + 2 N K s     (row_ptr, (col, w), D^-1, X read + X written)
  B_score     = 20 E_off + 2 N K s                    (id, endpoints, weight, score; both blocks)
  B_step      = T (B_sweep(G) + B_sweep(P)) + B_score
The timed region uses inputs larger than L2 (each vector block is 268 MB), so no L2 flush is done.

Multi-GPU: the workload is one graph; N > 1 runs N independent replicas (weak scaling, no
collective on the data path), one per rank, and the value is the sum over ranks.

Also in the line, measured outside the timed region: `sparsify_forms` (sparsify time and kappa of
each form against the plain two-level FP32 method), `mlp_forward` (learned-scorer inference on
the tensor cores over 28M feature rows) and `small_graph_latency` (the 64 x 64 oracle-size grid,
where launch and synchronisation costs dominate).

--impl reference times the CPU oracle (single thread, FP64) on a bounded sample of the same
workload: the first 32 of the 128 planes (524,288 nodes), same K, sweeps and budget fraction.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

SIDE, K, T, OMEGA, SEED, BETA = 128, 32, 20, 0.7, 1002, 0.05
SAMPLE_PLANES = 32
METRIC = "filter+score GB/s (% HBM peak); sparsify time at matched kappa vs plain FP32"
UNIT = "GB/s"


def workload_name(side=SIDE):
    return f"grid3d-{side}^3 6-neighbour, w=10^U[-2,2), K={K}, T={T}, omega={OMEGA}, fp32, flat filter+score+top-5%N"


def sweep_bytes(n, nnz, k=K, s=4):
    return 4 * (n + 1) + 8 * nnz + 4 * n + 2 * n * k * s


def score_bytes(n, e_off, k=K, s=4):
    return 20 * e_off + 2 * n * k * s


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# Source region of each profiled kernel (start and end markers in its file, plus shared headers):
# the committed ncu counters stay valid while this text is unchanged.
KERNEL_SOURCES = {
    "k_jacobi": ("smooth.cu", "template <typename V>\n__device__ __forceinline__ V ldmeta",
                 "// Rows longer than kHeavy entries", ["vec.cuh"]),
    "k_score": ("score.cu", "// Scorer, warp-tile schedule", "// ||X_p||^2 in FP64", ["vec.cuh"]),
    "k_mlp_forward_tc": ("mlp.cu", "// ---- inference on the 5th-generation tensor cores",
                         "constexpr int kS64 = 72;", []),
}


def kernel_source_hash(kernel):
    fname, start, end, extra = KERNEL_SOURCES[kernel]
    csrc = os.path.join(ROOT, "paper_2008_07633_gb300", "csrc")
    text = open(os.path.join(csrc, fname)).read()
    a = text.index(start)
    b = text.index(end, a)
    h = hashlib.sha256(text[a:b].encode())
    for e in extra:
        h.update(open(os.path.join(csrc, e), "rb").read())
    return h.hexdigest()


def ncu_traffic(kernel, summary):
    """DRAM bytes per launch from the committed ncu summary (the mean of its captured launches,
    one on L_G and one on L_P, like `achieved`), or None if the kernel's source changed since the
    counters were taken or a capture is missing."""
    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    shas = re.findall(r"source_sha256:\s*([0-9a-f]{64})", text)
    vals = [float(x) for x in re.findall(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)]
    if len(vals) < 2 or not shas:
        return None
    cur = kernel_source_hash(kernel)
    if any(h != cur for h in shas):
        return None
    return sum(vals) / len(vals)


def summary_value(summary, key, kernel):
    """A per-unit figure from a committed ncu summary, or None once the kernel's source changed."""
    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    shas = re.findall(r"source_sha256:\s*([0-9a-f]{64})", text)
    m = re.search(key + r":\s*([0-9.eE+]+)", text)
    if not m or not shas or any(h != kernel_source_hash(kernel) for h in shas):
        return None
    return float(m.group(1))


# Learned-scorer inference (16 -> 64 -> 64 -> 1, ReLU): FLOPs and HBM bytes per feature row
MLP_FLOP_PER_ROW = 2 * (16 * 64 + 64 * 64 + 64)
MLP_BYTES_PER_ROW = 16 * 4 + 4


def mlp_report(S, ctx, dev, rows, iters):
    """Throughput of sfg_mlp_forward (the tcgen05 kernel) over `rows` FP32 feature rows, timed by
    the context's CUDA events around each launch on its own stream."""
    import torch

    net = S.sfg_mlp_create(ctx, seed=7)
    gen_ = torch.Generator(device=dev)
    gen_.manual_seed(5)
    X = torch.randn(rows, S.MLP_NFEAT, device=dev, generator=gen_)
    out = torch.empty(rows, dtype=torch.float32, device=dev)
    for _ in range(3):
        S.sfg_mlp_forward(ctx, net, X, out=out)
    S.sfg_ctx_timing(ctx, True)
    for _ in range(iters):
        S.sfg_mlp_forward(ctx, net, X, out=out)
    n, ms = S.sfg_ctx_kernel_time(ctx, "mlp_forward")
    S.sfg_ctx_timing(ctx, False)
    net.close()
    ms /= max(n, 1)
    peak, peak_kind = load_peaks()
    gbs = rows * MLP_BYTES_PER_ROW / (ms * 1e-3) / 1e9
    per_row = summary_value("k_mlp_forward_tc_rows4M.txt", "dram_bytes_per_row", "k_mlp_forward_tc")
    return {"kernel": "k_mlp_forward_tc", "rows": rows, "launches": n, "avg_launch_ms": ms,
            "rows_per_s": rows / (ms * 1e-3),
            "tflops": rows * MLP_FLOP_PER_ROW / (ms * 1e-3) / 1e12,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                         "frac": gbs / peak, "peak_kind": peak_kind,
                         "traffic": per_row * rows if per_row else None,
                         "bytes_per_row": MLP_BYTES_PER_ROW, "flop_per_row": MLP_FLOP_PER_ROW}}


def small_graph_latency(S, ctx, dev, reps=20):
    """Latency of the oracle-size configuration (64 x 64 grid, weights U[1,10), K = 8, 10 sweeps,
    10% of the off-tree edges), which launch and synchronisation costs dominate: one flat
    sfg_sparsify call and one filter+score step, wall clock per call after warm-up."""
    import torch

    from paper_2008_07633_gb300 import inputs as gen

    n, u, v, w = gen.grid2d(64, 64, seed=1)
    g = S.sfg_laplacian(ctx, n, *(torch.from_numpy(a).to(dev) for a in (u, v, w)))
    tree, _ = S.sfg_spanning_tree(ctx, g)
    p = S.sfg_graph_subgraph(ctx, g, tree)
    off = torch.nonzero(tree == 0).flatten().to(torch.int32)
    k = int(np.floor(0.1 * off.numel() + 0.5))

    def wall(f):
        for _ in range(3):
            f()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            f()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps * 1e3

    def fs():
        sc = S.sfg_filter_score(ctx, g, p, off, 8, 10, 0.7, 1001)
        S.sfg_select_topk(ctx, sc, off, k)

    out = {"workload": "grid2d-64x64, w=U[1,10), K=8, T=10, omega=0.7, fp32, 10% of off-tree edges",
           "sparsify_flat_ms": wall(lambda: S.sfg_sparsify(ctx, g, K=8, steps=10, levels=0, omega=0.7,
                                                           seed=1001, budget_frac=0.1, budget_unit=1)),
           "filter_score_topk_ms": wall(fs)}
    g.close()
    p.close()
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------------------------------------------
# reference arm / CPU baseline: the oracle on a bounded sample of the workload
# ------------------------------------------------------------------------------------------------
def oracle_sample():
    import oracle as O
    from paper_2008_07633_gb300 import inputs as gen

    n, u, v, w = gen.grid3d(SIDE, seed=2)
    ns = SAMPLE_PLANES * SIDE * SIDE
    keep = (u < ns) & (v < ns)
    g = O.canonicalize(ns, u[keep], v[keep], w[keep])
    tree = O.mst(g)
    p = g.subgraph(tree)
    off = np.nonzero(tree == 0)[0].astype(np.int32)
    k = int(np.floor(BETA * ns + 0.5))
    nbytes = T * (sweep_bytes(ns, 2 * g.m) + sweep_bytes(ns, 2 * p.m)) + score_bytes(ns, off.size)

    def step():
        xg = O.smooth(g, K, T, OMEGA, SEED)
        xp = O.smooth(p, K, T, OMEGA, SEED)
        s = O.score_edges(g, xg, xp, off)
        O.topk(s, off, k)

    desc = (f"oracle (1 thread, FP64) on the first {SAMPLE_PLANES} of {SIDE} planes: {ns} nodes, "
            f"{g.m} edges, {off.size} off-tree edges; full filter+score step (init, {T} sweeps on "
            f"G and P, projection, scoring, top-{k})")
    return step, nbytes, desc


def run_reference(args):
    world, rank, _ = dist_env()
    if world > 1 and rank != 0:
        return 0
    step, nbytes, desc = oracle_sample()
    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    value = nbytes / dt / 1e9
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": workload_name() + " (oracle sample)"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                            "sample": desc},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def cpu_baseline():
    step, nbytes, desc = oracle_sample()
    t0 = time.perf_counter()
    step()
    dt = time.perf_counter() - t0
    return {"value": nbytes / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": desc + f"; one step, {dt:.1f} s"}


# ------------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------------
def run_ours(args):
    import torch

    import paper_2008_07633_gb300.sfg as S
    from paper_2008_07633_gb300 import inputs as gen

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    def barrier():
        if pg:
            pg.barrier()
        torch.cuda.synchronize()

    if args.mlp_only:  # ncu captures of the tensor-core inference kernel alone
        ctx = S.sfg_ctx_create(local)
        if rank == 0:
            print(json.dumps({"mlp_forward": mlp_report(S, ctx, dev, args.mlp_rows, 3)}), flush=True)
        return 0
    n, u, v, w = gen.grid3d(SIDE, seed=2)
    ctx = S.sfg_ctx_create(local)
    U, V, W = (torch.from_numpy(a).to(dev) for a in (u, v, w))
    G = S.sfg_laplacian(ctx, n, U, V, W)
    tree, ntree = S.sfg_spanning_tree(ctx, G)
    P = S.sfg_graph_subgraph(ctx, G, tree)
    off = torch.nonzero(tree == 0).flatten().to(torch.int32)
    e_off = off.numel()
    # deployment-time tuning of the sweep's tile shape for each Laplacian (outside the timed
    # region; the choice is recorded per degree bucket and the result is bit-identical)
    # (--profile keeps the default shape: under a profiler the tuner's timings mean nothing)
    tuned = ({"G": (1, None), "P": (1, None)} if args.profile else
             {"G": S.sfg_autotune(ctx, G, K), "P": S.sfg_autotune(ctx, P, K)})
    kk = int(np.floor(BETA * n + 0.5))
    scores = torch.empty(e_off, dtype=torch.float32, device=dev)
    sel = torch.empty(kk, dtype=torch.int32, device=dev)
    b_sweep_g, b_sweep_p = sweep_bytes(n, 2 * G.m), sweep_bytes(n, 2 * P.m)
    b_step = T * (b_sweep_g + b_sweep_p) + score_bytes(n, e_off)

    def step():
        S.sfg_filter_score(ctx, G, P, off, K, T, OMEGA, SEED, out=scores)
        S.sfg_select_topk(ctx, scores, off, kk, out=sel)

    for _ in range(args.warmup):
        step()
    barrier()
    stream = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    S.sfg_ctx_timing(ctx, True)
    l0 = S.sfg_ctx_launches(ctx)
    with ClockSampler(local) as clk:
        barrier()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        barrier()
    launches = S.sfg_ctx_launches(ctx) - l0
    ms = e0.elapsed_time(e1) / args.steps
    nj, ms_j = S.sfg_ctx_kernel_time(ctx, "jacobi")
    ns_, ms_s = S.sfg_ctx_kernel_time(ctx, "score")
    S.sfg_ctx_timing(ctx, False)
    if pg:
        t = torch.tensor([ms], device=dev, dtype=torch.float64)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    value = world * b_step / (ms * 1e-3) / 1e9

    # roofline of the dominant kernel (the Jacobi sweep), from its live CUDA-event durations
    peak, peak_kind = load_peaks()
    achieved = (args.steps * T * (b_sweep_g + b_sweep_p)) / (ms_j * 1e-3) / 1e9 if ms_j > 0 else None
    traffic = ncu_traffic("k_jacobi", "k_jacobi_grid3d128_k32.txt")
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None, "traffic": traffic,
            "kernel": "k_jacobi", "peak_kind": peak_kind,
            "bytes_per_launch": (b_sweep_g + b_sweep_p) / 2, "launches": nj,
            "avg_launch_us": ms_j / nj * 1e3 if nj else None,
            "score_kernel_GBps": score_bytes(n, e_off) * ns_ / (ms_s * 1e-3) / 1e9 if ms_s else None}

    # sparsify time (device-resident G) and the end-to-end number through the public API with
    # host buffers: H2D of the edge list, Laplacian, flat sparsify, D2H of the mask
    mlp = mlp_report(S, ctx, dev, args.mlp_rows, 10) if args.mlp_rows > 0 and not args.profile else None
    if args.profile:  # launch-list / counter captures: the filter+score steps only
        if rank == 0:
            print(json.dumps({"profile": True, "ms_per_step": ms, "value": value,
                              "roofline": roof, "gpu_launches": launches}), flush=True)
        return 0
    hu, hv, hw = (torch.from_numpy(a).pin_memory() for a in (u, v, w))
    mask_host = torch.empty(G.m, dtype=torch.uint8).pin_memory()

    def sparsify_only():
        m_, _ = S.sfg_sparsify(ctx, G, K=K, steps=T, levels=0, omega=OMEGA, seed=SEED,
                               budget_frac=BETA, budget_unit=0)
        return m_

    def e2e_step():
        du, dv, dw = (t.to(dev, non_blocking=True) for t in (hu, hv, hw))
        g2 = S.sfg_laplacian(ctx, n, du, dv, dw)
        m_, _ = S.sfg_sparsify(ctx, g2, K=K, steps=T, levels=0, omega=OMEGA, seed=SEED,
                               budget_frac=BETA, budget_unit=0)
        mask_host.copy_(m_, non_blocking=True)
        torch.cuda.synchronize()
        g2.close()

    e2e_iters = max(2, args.steps // 3)
    sparsify_only()
    e2e_step()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_iters):
        sparsify_only()
    torch.cuda.synchronize()
    sparsify_ms = (time.perf_counter() - t0) / e2e_iters * 1e3
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_iters):
        e2e_step()
    barrier()
    e2e_ms = (time.perf_counter() - t0) / e2e_iters * 1e3
    if pg:
        t = torch.tensor([e2e_ms, sparsify_ms], device=dev, dtype=torch.float64)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        e2e_ms, sparsify_ms = (float(x) for x in t.tolist())

    # sparsify time at matched kappa against plain FP32: the reference is the plain method of the
    # 128^3 configuration (two-level coarsening, Jacobi, FP32 blocks); the forms are the flat
    # method, BF16 storage, and the multicolour Gauss-Seidel smoother with 2 sweeps, each timed
    # (device-resident G) and scored by sfg_kappa (200 Lanczos steps; lambda_min certified = 1 by
    # the component count when it applies). Rank 0 only, outside every timed region above.
    forms = None
    if rank == 0 and not args.no_kappa:
        forms = {}
        for name, levels, storage, smoother, steps_f, om in (
                ("fp32_2level", 2, torch.float32, S.SFG_SMOOTH_JACOBI, T, OMEGA),
                ("fp32_flat", 0, torch.float32, S.SFG_SMOOTH_JACOBI, T, OMEGA),
                ("bf16_2level", 2, torch.bfloat16, S.SFG_SMOOTH_JACOBI, T, OMEGA),
                ("gauss_seidel_T2_2level", 2, torch.float32, S.SFG_SMOOTH_GAUSS_SEIDEL, 2, 1.0),
                ("gauss_seidel_T2_flat", 0, torch.float32, S.SFG_SMOOTH_GAUSS_SEIDEL, 2, 1.0)):
            def sp_once():
                return S.sfg_sparsify(ctx, G, K=K, steps=steps_f, levels=levels, omega=om,
                                      seed=SEED, budget_frac=BETA, budget_unit=0, storage=storage,
                                      smoother=smoother)
            mk, nsel = sp_once()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(e2e_iters):
                mk, nsel = sp_once()
            torch.cuda.synchronize()
            ms_form = (time.perf_counter() - t0) / e2e_iters * 1e3
            t1 = time.perf_counter()
            kap, lmin, lmax, info = S.sfg_kappa(ctx, G, mk, steps=args.kappa_steps, seed=1, info=True)
            forms[name] = {"levels": levels, "storage": str(storage).replace("torch.", ""),
                           "smoother": "gauss_seidel" if smoother else "jacobi", "sweeps": steps_f,
                           "edges": nsel, "sparsify_ms": ms_form, "kappa": kap, "lambda_max": lmax,
                           "lambda_min": lmin, "lambda_min_exact": info["lambda_min_exact"],
                           "lanczos_steps": info["steps"],
                           "kappa_seconds": time.perf_counter() - t1}
        ref = forms["fp32_2level"]
        for name in forms:
            if name != "fp32_2level":
                forms[name]["kappa_vs_reference"] = forms[name]["kappa"] / ref["kappa"]
                forms[name]["speedup_vs_reference"] = ref["sparsify_ms"] / forms[name]["sparsify_ms"]

    small = small_graph_latency(S, ctx, dev) if rank == 0 else None
    if rank != 0:
        return 0
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": workload_name(), "nodes": n, "edges": G.m, "nnz_G": 2 * G.m,
                      "nnz_P": 2 * P.m, "off_tree_edges": e_off, "k_selected": kk,
                      "bytes_per_step": b_step,
                      "l2": "inputs larger than L2 (each N x K block is 268 MB); no flush",
                      "parallelism": f"replicas x{world}",
                      "tuned_tile_shape": {k: v[0] for k, v in tuned.items()}},
           "roofline": roof,
           "clocks": clk.summary(),
           "e2e": {"value": world * b_step / (e2e_ms * 1e-3) / 1e9, "unit": UNIT,
                   "h2d_bytes_per_step": int(u.nbytes + v.nbytes + w.nbytes),
                   "d2h_bytes_per_step": int(G.m), "ms_per_step": e2e_ms,
                   "what": "pinned host edge list -> H2D -> sfg_laplacian -> sfg_sparsify (flat) -> D2H mask"},
           "sparsify_ms": sparsify_ms,
           "gpu_launches": launches}
    if forms:
        out["sparsify_forms"] = forms
    if mlp:
        out["mlp_forward"] = mlp
    if small:
        out["small_graph_latency"] = small
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline()
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-kappa", action="store_true",
                    help="skip the sparsify-forms report (FP32 vs BF16 sparsify time and kappa)")
    ap.add_argument("--kappa-steps", type=int, default=200)
    ap.add_argument("--profile", action="store_true",
                    help="time only the filter+score steps (for ncu launch lists and counters)")
    ap.add_argument("--mlp-rows", type=int, default=28_000_000,
                    help="feature rows for the learned-scorer inference report (0 skips it)")
    ap.add_argument("--mlp-only", action="store_true",
                    help="run only the inference report (for ncu captures of its kernel)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
