#!/usr/bin/env python3
"""Benchmark of the SF-GRASS hot path on one GB300: filter + score throughput.

Headline workload (one step): the 3-D 6-neighbour grid 128^3 (2,097,152 nodes, 6,242,304 edges,
weights 10^U[-2,2)), K = 32 seeded vectors, 20 weighted-Jacobi sweeps (omega 0.7) on the Laplacian
of G and on that of its maximum spanning tree P, projection, RATIO scores of all 4,145,153
off-tree edges and the top round(0.05 N) = 104,858 of them (sfg_filter_score + sfg_select_topk).
G, P and the off-tree id list are built before the timed region (they are the inputs of the
filter); every step recomputes everything else.

Metric: filter+score algorithmic GB/s = bytes / step time with
  B_sweep(L)  = 4(N+1) + 8 nnz(L) + 4N + 2 N K s     (row_ptr, (col, w), D^-1, X read + X written)
  B_score     = 16 E_off + 2 N K s                    (per edge 16 bytes, both blocks once)
  B_step      = T (B_sweep(G) + B_sweep(P)) + B_score
B_score counts 16 bytes per scored edge: its id, its two endpoint ids and its score (the weight
lookup is left out of the byte model). The timed region uses inputs larger than
L2 (each vector block is 268 MB), so no L2 flush is done.

Also in the line (rank 0, outside the headline's timed region, each timed with CUDA events over
the same number of steps):
- `workloads`: filter+score on every workload shape -- the 2048^2 power-grid mesh with vias
  (K = 64, FP32 and BF16 blocks), the 4M-node Chung-Lu power-law graph (K = 32), and the batch of
  512 10-NN graphs (K = 16, T = 15) as a batch-plan run replayed from a CUDA graph (graphs/s) --
  each with its algorithmic GB/s and the sweep's roofline against the measured HBM peak;
- `sparsify_forms`: sparsify time at matched kappa on the 128^3 grid. The reference is the plain
  method of that configuration (two-level coarsening, Jacobi, FP32 blocks, 5% of N); every other
  form (flat FP32, BF16 blocks, the Gauss-Seidel smoother) has its budget searched until its kappa
  is within 5% of the reference's (kappa by sfg_kappa, 100 Lanczos steps);
- `batched_forms`: the batch plan against one sfg_sparsify call per graph, kappa compared on a
  sample of the graphs; `learned_forms`: the learned-proposal form on the Chung-Lu graph with the
  proposal fraction raised until its kappa is within 5% of the plain flat method's;
- `mlp_forward` (learned-scorer inference on the tensor cores) and `small_graph_latency` (the
  64 x 64 oracle-size grid, where launch and synchronisation costs dominate).

Multi-GPU: the workload is one graph; N > 1 runs N independent replicas (weak scaling, no
collective on the data path), one per rank, and the value is the sum over ranks.

--impl reference times the CPU oracle (single thread, FP64) on a bounded sample of the headline
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
    return 16 * e_off + 2 * n * k * s


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
                         "// ---- training on the 5th-generation tensor cores", []),
    "k_mlp_fwdbwd_tc": ("mlp.cu", "// ---- training on the 5th-generation tensor cores",
                        "// grad[i] = sum over CTAs (in order) of part[cta][i]", []),
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


def ncu_traffic_single(kernel, summary):
    """DRAM bytes per launch from a committed ncu summary with one capture (or None, as above)."""
    path = os.path.join(ROOT, "profiles", summary)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    shas = re.findall(r"source_sha256:\s*([0-9a-f]{64})", text)
    vals = [float(x) for x in re.findall(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", text)]
    if not vals or not shas or any(h != kernel_source_hash(kernel) for h in shas):
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


# Training step of the learned scorer (forward and backward of every row): FLOPs of the network's
# own products per row (forward 10,368; delta_1 = delta_2 W2^T, dW2, dW1, dw3)
MLP_TRAIN_FLOP_PER_ROW = MLP_FLOP_PER_ROW + 2 * 64 * 64 + 2 * 64 * 64 + 2 * 16 * 64 + 2 * 64


def load_tensor_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return float(json.load(open(p))["bf16_tflops"]), "measured (bf16, burst)"
    return 1900.0, "fallback"


def mlp_train_report(S, ctx, dev, rows, iters):
    """Throughput of sfg_mlp_gradient (the tcgen05 training kernel: forward and backward over
    `rows` feature rows), timed by the context's CUDA events around each launch."""
    import torch

    net = S.sfg_mlp_create(ctx, seed=7)
    gen_ = torch.Generator(device=dev)
    gen_.manual_seed(6)
    X = torch.randn(rows, S.MLP_NFEAT, device=dev, generator=gen_)
    t = torch.randn(rows, device=dev, generator=gen_)
    for _ in range(3):
        S.sfg_mlp_gradient(ctx, net, X, t)
    S.sfg_ctx_timing(ctx, True)
    for _ in range(iters):
        S.sfg_mlp_gradient(ctx, net, X, t)
    n, ms = S.sfg_ctx_kernel_time(ctx, "mlp_fwdbwd")
    S.sfg_ctx_timing(ctx, False)
    net.close()
    ms /= max(n, 1)
    peak, kind = load_tensor_peak()
    tf = rows * MLP_TRAIN_FLOP_PER_ROW / (ms * 1e-3) / 1e12
    return {"kernel": "k_mlp_fwdbwd_tc", "rows": rows, "launches": n, "avg_launch_ms": ms,
            "rows_per_s": rows / (ms * 1e-3),
            "roofline": {"bound": "tensor", "achieved": tf, "peak": peak, "unit": "TFLOP/s",
                         "frac": tf / peak, "peak_kind": kind, "flop_per_row": MLP_TRAIN_FLOP_PER_ROW,
                         "hbm_GBps": rows * MLP_BYTES_PER_ROW / (ms * 1e-3) / 1e9}}


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


def host_cpu():
    """Host cores and CPU model of this machine (for the CPU-baseline lines)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                if line.startswith("Model name"):
                    break
    except Exception:
        pass
    if not model:
        import platform

        model = platform.processor() or platform.machine()
    return {"nproc": os.cpu_count(), "cpu_model": model}


# ------------------------------------------------------------------------------------------------
# input generation in worker processes (started with spawn before the first GPU call)
# ------------------------------------------------------------------------------------------------
C5_NODES, C4_GRAPHS = 4_000_000, 512
LEARN_TRAIN_SEEDS = (101, 102, 103, 104)


def _gen_chung_lu(args):
    from paper_2008_07633_gb300 import inputs as gen

    n, seed = args
    return gen.chung_lu(n, 16.0, 2.3, seed=seed)


def _gen_knn(args):
    from paper_2008_07633_gb300 import inputs as gen

    n, seed = args
    return gen.knn3d(int(n), k=10, seed=seed)


def start_generators():
    """Worker pool generating the large workloads' inputs while the headline runs: the C5
    Chung-Lu graph, the 512 k-NN graphs of the batch and the learned scorer's training graphs."""
    import multiprocessing as mp

    from paper_2008_07633_gb300 import inputs as gen

    pool = mp.get_context("spawn").Pool(max(1, min(16, (os.cpu_count() or 2) - 1)))
    sizes = gen.batch_sizes(C4_GRAPHS, seed=3)
    jobs = {"c5": pool.apply_async(_gen_chung_lu, ((C5_NODES, 5),)),
            "c4": pool.map_async(_gen_knn, [(int(n), 3000 + i) for i, n in enumerate(sizes)]),
            "train": pool.map_async(_gen_chung_lu, [(1 << 18, s) for s in LEARN_TRAIN_SEEDS])}
    return pool, jobs


def _timed_steps(ctx, S, fn, steps, warmup):
    """CUDA-event time per step of fn() on the context's stream, plus the context's per-kernel
    event times of the sweep ("jacobi*") and scorer ("score") launches of the timed steps."""
    import torch

    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    S.sfg_ctx_timing(ctx, True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    nj, ms_j = S.sfg_ctx_kernel_time(ctx, "jacobi")
    ns, ms_s = S.sfg_ctx_kernel_time(ctx, "score")
    S.sfg_ctx_timing(ctx, False)
    return e0.elapsed_time(e1) / steps, ms_j / steps, ms_s / steps


def time_filter_score(S, ctx, dev, spec, name, K_, T_, storage, steps, warmup, peak, peak_kind,
                      traffic=None, autotune=True):
    """Filter+score throughput of one workload (inputs device-resident, as the headline)."""
    import torch

    n, u, v, w = spec
    G = S.sfg_laplacian(ctx, n, *(torch.from_numpy(a).to(dev) for a in (u, v, w)))
    tree, _ = S.sfg_spanning_tree(ctx, G)
    P = S.sfg_graph_subgraph(ctx, G, tree)
    off = torch.nonzero(tree == 0).flatten().to(torch.int32)
    if autotune:
        S.sfg_autotune(ctx, G, K_, storage)
        S.sfg_autotune(ctx, P, K_, storage)
    s = 2 if storage == torch.bfloat16 else 4
    out = torch.empty(off.numel(), dtype=torch.float32, device=dev)
    ms, ms_sweeps, ms_score = _timed_steps(
        ctx, S, lambda: S.sfg_filter_score(ctx, G, P, off, K_, T_, OMEGA, SEED, storage=storage,
                                           out=out), steps, warmup)
    bs_g, bs_p = sweep_bytes(n, 2 * G.m, K_, s), sweep_bytes(n, 2 * P.m, K_, s)
    b_sweeps = T_ * (bs_g + bs_p)
    b_score = score_bytes(n, off.numel(), K_, s)
    gbs = (b_sweeps + b_score) / (ms * 1e-3) / 1e9
    sweeps_gbs = b_sweeps / (ms_sweeps * 1e-3) / 1e9
    res = {"workload": name, "nodes": n, "edges": G.m, "off_tree_edges": off.numel(), "K": K_,
           "T": T_, "storage": str(storage).replace("torch.", ""), "bytes_per_step": b_sweeps + b_score,
           "ms_per_step": ms, "value": gbs, "unit": "GB/s", "frac_of_peak": gbs / peak,
           "roofline": {"bound": "hbm", "kernel": "sweep (k_jacobi and its hub-row kernels)",
                        "achieved": sweeps_gbs, "peak": peak, "unit": "GB/s",
                        "frac": sweeps_gbs / peak, "peak_kind": peak_kind,
                        "bytes_per_launch": (bs_g + bs_p) / 2,
                        "avg_sweep_us": ms_sweeps / (2 * T_) * 1e3, "traffic": traffic},
           "score_kernel": {"achieved": b_score / (ms_score * 1e-3) / 1e9, "frac": b_score / (ms_score * 1e-3) / 1e9 / peak,
                            "us": ms_score * 1e3}}
    return res, (G, P, tree, off)


def time_batch(S, ctx, dev, specs, steps, warmup, peak, peak_kind, K_=16, T_=15, beta=0.05):
    """The batch configuration: a batch plan of all graphs, its run captured in a CUDA graph and
    replayed; graphs/s and the algorithmic GB/s of the union's filter+score."""
    import torch

    graphs = [S.sfg_laplacian(ctx, n, *(torch.from_numpy(a).to(dev) for a in (u, v, w)))
              for n, u, v, w in specs]
    torch.cuda.synchronize()
    stream = torch.cuda.Stream()
    bctx = S.sfg_ctx_create(dev.index, stream)
    def timed(locality):
        with torch.cuda.stream(stream):
            plan = S.Batch(bctx, graphs, K=K_, steps=T_, budget_frac=beta, autotune=True,
                           locality=locality)
            ref = plan.run(SEED)
            out = torch.empty_like(ref)
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream, capture_error_mode="relaxed"):
            plan.run(SEED, out=out)
        with torch.cuda.stream(stream):     # replays run on the current stream: time them there
            for _ in range(warmup):
                graph.replay()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(steps):
                graph.replay()
            e1.record(stream)
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
        return plan, e0.elapsed_time(e1) / steps

    _, ms_input_order = timed(False)
    plan, ms = timed(True)
    n_all = sum(g.n for g in graphs)
    m_all = sum(g.m for g in graphs)
    # union sizes: G has 2 m_all entries; P, the forests, 2 (count_g - k_g) entries per graph, with
    # k_g = round(beta n_g) (every 10-NN graph has more off-forest edges than its budget)
    forest = sum(int(c) - int(np.floor(beta * g.n + 0.5)) for c, g in zip(plan.counts, graphs))
    e_off = m_all - forest
    b_step = T_ * (sweep_bytes(n_all, 2 * m_all, K_) + sweep_bytes(n_all, 2 * forest, K_)) + \
        score_bytes(n_all, e_off, K_)
    gbs = b_step / (ms * 1e-3) / 1e9
    res = {"workload": f"{len(graphs)} symmetrised 10-NN graphs, n log-uniform in [1e3, 2e5), "
                       f"Gaussian-kernel weights, K={K_}, T={T_}, flat, 5% of N",
           "graphs": len(graphs), "nodes": n_all, "edges": m_all, "ms_per_batch": ms,
           "value": len(graphs) / (ms * 1e-3), "unit": "graphs/s", "bytes_per_batch": b_step,
           "GBps": gbs, "frac_of_peak": gbs / peak, "peak_kind": peak_kind,
           "how": "sfg_batch_run captured in a CUDA graph and replayed (plan built once, nodes in "
                  "locality order)",
           "ms_per_batch_input_order": ms_input_order}
    return res, graphs, plan, bctx


def kappa_of(S, ctx, G, mask, steps):
    k, lmin, lmax, info = S.sfg_kappa(ctx, G, mask, steps=steps, seed=1, info=True)
    return k, info


def search_budget(S, ctx, G, kappa_ref, form, beta0, kappa_steps, reps, max_probes=8, tol=0.04):
    """Budget beta at which a sparsify form's kappa is within tol of kappa_ref. kappa falls as beta
    grows, but in steps on some forms (a few poorly approximated edges hold it up until they are
    recovered), so: secant steps on (log beta, log kappa) from the slope -1 until the target is
    bracketed, then bisection in log beta. A probe whose kappa evaluation fails is recorded and
    treated as above the target. Returns the closest probe and all probes."""
    import math

    import torch

    probes = []
    lo = hi = None          # log beta with kappa above / below the target
    lb, prev = math.log(beta0), None
    for _ in range(max_probes):
        beta = math.exp(lb)
        mk, nsel = form(beta)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            mk, nsel = form(beta)
        torch.cuda.synchronize()
        ms = (time.perf_counter() - t0) / reps * 1e3
        try:
            kap, info = kappa_of(S, ctx, G, mk, kappa_steps)
            err = None
        except S.SfgError as e:
            kap, info, err = float("inf"), {"steps": None, "lambda_min_exact": None}, str(e)
        probes.append({"budget_frac": beta, "edges": nsel, "sparsify_ms": ms, "kappa": kap,
                       "lanczos_steps": info["steps"], "lambda_min_exact": info["lambda_min_exact"],
                       "error": err})
        if math.isfinite(kap) and abs(kap / kappa_ref - 1.0) <= tol:
            break
        above = not math.isfinite(kap) or kap > kappa_ref
        if above:
            lo = lb if lo is None else max(lo, lb)
        else:
            hi = lb if hi is None else min(hi, lb)
        if lo is not None and hi is not None:
            nxt = 0.5 * (lo + hi)
        else:
            r = math.log(kap / kappa_ref) if math.isfinite(kap) else 1.0
            slope = -1.0
            if prev is not None and lb != prev[0] and math.isfinite(prev[1]):
                slope = max(-4.0, min(-0.1, (r - prev[1]) / (lb - prev[0])))
            prev = (lb, r)
            step_ = max(-math.log(4.0), min(math.log(4.0), -r / slope))   # at most 4x per step
            nxt = min(max(lb + step_, math.log(1e-4)), math.log(0.6))
        if abs(nxt - lb) < 1e-6:
            break
        lb = nxt
    best = min(probes, key=lambda p: abs(p["kappa"] / kappa_ref - 1.0) if math.isfinite(p["kappa"]) else 1e30)
    return best, probes


def matched_forms_c2(S, ctx, G, reps, kappa_steps):
    """Sparsify time at matched kappa on the 128^3 grid (see the module docstring)."""
    import torch

    forms_def = {
        "fp32_2level": dict(levels=2, storage=torch.float32, smoother=S.SFG_SMOOTH_JACOBI, steps=T, omega=OMEGA),
        "fp32_flat": dict(levels=0, storage=torch.float32, smoother=S.SFG_SMOOTH_JACOBI, steps=T, omega=OMEGA),
        "bf16_flat": dict(levels=0, storage=torch.bfloat16, smoother=S.SFG_SMOOTH_JACOBI, steps=T, omega=OMEGA),
        "bf16_2level": dict(levels=2, storage=torch.bfloat16, smoother=S.SFG_SMOOTH_JACOBI, steps=T, omega=OMEGA),
        "gauss_seidel_T2_flat": dict(levels=0, storage=torch.float32, smoother=S.SFG_SMOOTH_GAUSS_SEIDEL, steps=2, omega=1.0),
        "gauss_seidel_T2_2level": dict(levels=2, storage=torch.float32, smoother=S.SFG_SMOOTH_GAUSS_SEIDEL, steps=2, omega=1.0),
    }

    def make(kw):
        def form(beta):
            return S.sfg_sparsify(ctx, G, K=K, seed=SEED, budget_frac=beta, budget_unit=0, **kw)
        return form

    out = {}
    ref_form = make(forms_def["fp32_2level"])
    mk, nsel = ref_form(BETA)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        mk, nsel = ref_form(BETA)
    torch.cuda.synchronize()
    ref_ms = (time.perf_counter() - t0) / reps * 1e3
    kref, info = kappa_of(S, ctx, G, mk, kappa_steps)
    out["fp32_2level"] = {"reference": True, "budget_frac": BETA, "edges": nsel, "sparsify_ms": ref_ms,
                          "kappa": kref, "lanczos_steps": info["steps"],
                          "lambda_min_exact": info["lambda_min_exact"]}
    start = {}
    for name, kw in forms_def.items():
        if name == "fp32_2level":
            continue
        beta0 = start.get(kw["levels"], BETA) if kw["smoother"] == S.SFG_SMOOTH_JACOBI else start.get(("gs", kw["levels"]), start.get(kw["levels"], BETA))
        best, probes = search_budget(S, ctx, G, kref, make(kw), beta0, kappa_steps, reps)
        start.setdefault(kw["levels"], best["budget_frac"])
        if kw["smoother"] != S.SFG_SMOOTH_JACOBI:
            start.setdefault(("gs", kw["levels"]), best["budget_frac"])
        best = dict(best)
        best.update({"levels": kw["levels"], "storage": str(kw["storage"]).replace("torch.", ""),
                     "smoother": "gauss_seidel" if kw["smoother"] else "jacobi", "sweeps": kw["steps"],
                     "kappa_vs_reference": best["kappa"] / kref,
                     "matched": abs(best["kappa"] / kref - 1.0) <= 0.05,
                     "speedup_vs_reference": ref_ms / best["sparsify_ms"],
                     "probes": [{"budget_frac": round(p["budget_frac"], 6), "kappa": round(p["kappa"], 1),
                                 "lanczos_steps": p["lanczos_steps"], "error": p["error"]} for p in probes]})
        out[name] = best
    return out


def batched_forms(S, ctx, graphs, plan, kappa_steps, sample=16):
    """The batch plan against one sfg_sparsify per graph (same parameters): time per batch and
    kappa on a sample of graphs across sizes."""
    import torch

    kw = dict(K=16, steps=15, levels=0, seed=SEED, budget_frac=0.05, budget_unit=0)
    mask = plan.run(SEED)
    parts = plan.split(mask)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan.run(SEED, out=mask)
    torch.cuda.synchronize()
    t_batch = (time.perf_counter() - t0) * 1e3
    singles = []
    t0 = time.perf_counter()
    for g in graphs:
        singles.append(S.sfg_sparsify(ctx, g, **kw)[0])
    torch.cuda.synchronize()
    t_loop = (time.perf_counter() - t0) * 1e3
    order = sorted(range(len(graphs)), key=lambda i: graphs[i].n)
    idx = order[:: max(1, len(order) // sample)][:sample]
    ratios = []
    for i in idx:
        kb = kappa_of(S, ctx, graphs[i], parts[i], kappa_steps)[0]
        ks = kappa_of(S, ctx, graphs[i], singles[i], kappa_steps)[0]
        ratios.append(kb / ks)
    return {"reference": "one sfg_sparsify call per graph (plain flat FP32)",
            "reference_ms": t_loop, "batched_ms": t_batch, "speedup_vs_reference": t_loop / t_batch,
            "kappa_vs_reference_sample": {"graphs": len(idx), "min": min(ratios), "max": max(ratios),
                                          "median": float(np.median(ratios))},
            "matched": all(abs(r - 1.0) <= 0.05 for r in ratios)}


def learned_forms(S, ctx, dev, spec, train_specs, kappa_steps=60):
    """Learned proposals on the Chung-Lu graph against the plain flat method (K = 32, T = 20, 5% of
    N): the network is trained on the GPU by the library's own kernels on method-generated data
    (2-step features -> ln 20-step score) of the training graphs; the proposal fraction is raised
    until the learned form's kappa is within 5% of the plain method's."""
    import torch

    feats, targs = [], []
    for (n, u, v, w), sd in zip(train_specs, LEARN_TRAIN_SEEDS):
        g = S.sfg_laplacian(ctx, n, *(torch.from_numpy(a).to(dev) for a in (u, v, w)))
        tree, _ = S.sfg_spanning_tree(ctx, g)
        p = S.sfg_graph_subgraph(ctx, g, tree)
        off = torch.nonzero(tree == 0).flatten().to(torch.int32)
        feats.append(S.sfg_edge_features(ctx, g, p, off, 32, 2, 0.7, seed=sd))
        targs.append(torch.log(S.sfg_filter_score(ctx, g, p, off, 32, 20, 0.7, seed=sd) + 1e-30))
    net = S.sfg_mlp_create(ctx, seed=21)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = S.sfg_mlp_train(ctx, net, torch.cat(feats), torch.cat(targs), batch=16384, epochs=10, lr=2e-3)
    t_train = time.perf_counter() - t0
    n, u, v, w = spec
    G = S.sfg_laplacian(ctx, n, *(torch.from_numpy(a).to(dev) for a in (u, v, w)))
    kw = dict(K=32, steps=20, seed=5, budget_frac=0.05)

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            mk, cnt = fn()
        torch.cuda.synchronize()
        return mk, cnt, (time.perf_counter() - t0) / reps * 1e3

    mk, cnt, ms_plain = timed(lambda: S.sfg_sparsify(ctx, G, levels=0, budget_unit=0, **kw))
    kp = kappa_of(S, ctx, G, mk, kappa_steps)[0]
    probes = []
    for frac in (0.02, 0.05, 0.1, 0.2, 0.35, 0.5, 0.75):
        ml, cl, ms = timed(lambda: S.sfg_sparsify_learned(ctx, G, net, feat_steps=2, propose_frac=frac, **kw))
        kl = kappa_of(S, ctx, G, ml, kappa_steps)[0]
        probes.append({"propose_frac": frac, "sparsify_ms": ms, "kappa": kl, "kappa_vs_reference": kl / kp,
                       "speedup_vs_reference": ms_plain / ms})
        if abs(kl / kp - 1.0) <= 0.05:
            break
    best = min(probes, key=lambda p: abs(p["kappa_vs_reference"] - 1.0))
    net.close()
    return {"workload": f"Chung-Lu n={G.n}, m={G.m}, K=32, T=20, 5% of N",
            "train_seconds": t_train, "train_loss": loss,
            "reference": {"form": "plain flat FP32", "sparsify_ms": ms_plain, "kappa": kp, "edges": cnt},
            "learned": best, "matched": abs(best["kappa_vs_reference"] - 1.0) <= 0.05, "probes": probes}


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


def max_over_ranks(pg, values, device):
    """Element-wise maximum of `values` over all ranks (a replica job takes as long as its
    slowest rank); `values` unchanged without a process group."""
    if pg is None:
        return [float(x) for x in values]
    import torch

    t_ = torch.tensor([float(x) for x in values], device=device, dtype=torch.float64)
    pg.all_reduce(t_, op=pg.ReduceOp.MAX)
    return [float(x) for x in t_.tolist()]


def whole_job_gbps(world, bytes_per_step, ms):
    """Whole-job throughput of `world` replicas that each move bytes_per_step per step."""
    return world * bytes_per_step / (ms * 1e-3) / 1e9


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
           "cpu_baseline": dict({"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "sample": desc}, **host_cpu()),
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def cpu_baseline():
    step, nbytes, desc = oracle_sample()
    t0 = time.perf_counter()
    step()
    dt = time.perf_counter() - t0
    return dict({"value": nbytes / dt / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
                 "sample": desc + f"; one step, {dt:.1f} s"}, **host_cpu())


# ------------------------------------------------------------------------------------------------
# our arm
# ------------------------------------------------------------------------------------------------
def run_ours(args):
    world, rank, local = dist_env()
    extra = rank == 0 and not args.profile and not args.headline_only
    pool, jobs = start_generators() if extra and not args.no_workloads else (None, None)

    import torch

    import paper_2008_07633_gb300.sfg as S
    from paper_2008_07633_gb300 import inputs as gen

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

    if args.mlp_only:  # ncu captures of the tensor-core inference and training kernels alone
        ctx = S.sfg_ctx_create(local)
        if rank == 0:
            print(json.dumps({"mlp_forward": mlp_report(S, ctx, dev, args.mlp_rows, 3),
                              "mlp_train": mlp_train_report(S, ctx, dev, args.mlp_rows, 3)}), flush=True)
        return 0
    if args.profile and args.profile_workload == "chunglu":
        # ncu captures on the power-law workload: filter+score steps only (default tile shape)
        ctx = S.sfg_ctx_create(local)
        spec = gen.chung_lu(C5_NODES, 16.0, 2.3, seed=5)
        r_, _ = time_filter_score(S, ctx, dev, spec, "chunglu", 32, T, torch.float32, args.steps,
                                  args.warmup, *load_peaks(), autotune=False)
        if rank == 0:
            print(json.dumps({"profile": True, "workload": r_}), flush=True)
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
    ms = max_over_ranks(pg, [ms], dev)[0]
    value = whole_job_gbps(world, b_step, ms)

    # roofline of the dominant kernel (the Jacobi sweep), from its live CUDA-event durations
    peak, peak_kind = load_peaks()
    achieved = (args.steps * T * (b_sweep_g + b_sweep_p)) / (ms_j * 1e-3) / 1e9 if ms_j > 0 else None
    traffic = ncu_traffic("k_jacobi", "k_jacobi_grid3d128_k32.txt")
    b_score = score_bytes(n, e_off)
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak if achieved else None, "traffic": traffic,
            "kernel": "k_jacobi", "peak_kind": peak_kind,
            "bytes_per_launch": (b_sweep_g + b_sweep_p) / 2, "launches": nj,
            "avg_launch_us": ms_j / nj * 1e3 if nj else None,
            "score_kernel_GBps": b_score * ns_ / (ms_s * 1e-3) / 1e9 if ms_s else None,
            "score_kernel_frac": b_score * ns_ / (ms_s * 1e-3) / 1e9 / peak if ms_s else None}

    if args.profile:  # launch-list / counter captures: the filter+score steps only
        if rank == 0:
            print(json.dumps({"profile": True, "ms_per_step": ms, "value": value,
                              "roofline": roof, "gpu_launches": launches}), flush=True)
        return 0

    # sparsify time (device-resident G) and the end-to-end number through the public API with
    # host buffers: H2D of the edge list, Laplacian, flat sparsify, D2H of the mask
    mlp = mlp_report(S, ctx, dev, args.mlp_rows, 10) if args.mlp_rows > 0 and extra else None
    mlp_tr = mlp_train_report(S, ctx, dev, 4_000_000, 10) if args.mlp_rows > 0 and extra else None
    hu, hv, hw = (torch.from_numpy(a).pin_memory() for a in (u, v, w))
    mask_host = torch.empty(G.m, dtype=torch.uint8).pin_memory()

    def sparsify_only():
        m_, _ = S.sfg_sparsify(ctx, G, K=K, steps=T, levels=0, omega=OMEGA, seed=SEED,
                               budget_frac=BETA, budget_unit=0)
        return m_

    def e2e_step():
        du, dv, dw = (t_.to(dev, non_blocking=True) for t_ in (hu, hv, hw))
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
    e2e_ms, sparsify_ms = max_over_ranks(pg, [e2e_ms, sparsify_ms], dev)
    if rank != 0:
        return 0

    # every workload shape of the configuration list (rank 0, outside the headline's timed region)
    workloads, forms, bforms, lforms = None, None, None, None
    if extra and not args.no_workloads:
        workloads = {}
        wsteps, wwarm = max(3, min(args.steps, 10)), max(3, args.warmup)
        c3 = gen.power_grid(2048, seed=3)
        for st in (torch.float32, torch.bfloat16):
            r_, objs = time_filter_score(S, ctx, dev, c3, "power-grid mesh 2048^2 + 1% vias, "
                                         "log-normal weights", 64, T, st, wsteps, wwarm, peak, peak_kind)
            workloads["C3_powergrid_" + ("fp32" if st == torch.float32 else "bf16")] = r_
            del objs
        c5 = jobs["c5"].get()
        r_, objs = time_filter_score(S, ctx, dev, c5, "Chung-Lu power-law graph, 4M nodes requested "
                                     "(largest component), mean degree 16, exponent 2.3", 32, T,
                                     torch.float32, wsteps, wwarm, peak, peak_kind,
                                     traffic=ncu_traffic_single("k_jacobi", "k_jacobi_chunglu4m_k32.txt"))
        r_["roofline"]["note"] = ("random neighbour rows of a power-law graph mostly miss L2: the "
                                  "sweep's DRAM traffic is about 3x its algorithmic bytes (traffic)")
        workloads["C5_chunglu_fp32"] = r_
        del objs
        c4 = jobs["c4"].get()
        r_, graphs, plan, bctx = time_batch(S, ctx, dev, c4, wsteps, wwarm, peak, peak_kind)
        workloads["C4_batch_knn"] = r_
        if not args.no_kappa:
            bforms = batched_forms(S, ctx, graphs, plan, args.kappa_steps)
        plan.close()
        for g_ in graphs:
            g_.close()
        bctx.close()
        if not args.no_kappa:
            lforms = learned_forms(S, ctx, dev, c5, jobs["train"].get())
        pool.close()
    if extra and not args.no_kappa:
        forms = matched_forms_c2(S, ctx, G, max(2, e2e_iters // 2), args.kappa_steps)

    small = small_graph_latency(S, ctx, dev) if extra else None
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": workload_name(), "nodes": n, "edges": G.m, "nnz_G": 2 * G.m,
                      "nnz_P": 2 * P.m, "off_tree_edges": e_off, "k_selected": kk,
                      "bytes_per_step": b_step,
                      "l2": "inputs larger than L2 (each N x K block is 268 MB); no flush",
                      "parallelism": f"replicas x{world}",
                      "tuned_tile_shape": {k_: v_[0] for k_, v_ in tuned.items()}},
           "roofline": roof,
           "clocks": clk.summary(),
           "e2e": {"value": whole_job_gbps(world, b_step, e2e_ms), "unit": UNIT,
                   "h2d_bytes_per_step": int(u.nbytes + v.nbytes + w.nbytes),
                   "d2h_bytes_per_step": int(G.m), "ms_per_step": e2e_ms,
                   "what": "pinned host edge list -> H2D -> sfg_laplacian -> sfg_sparsify (flat) -> D2H mask"},
           "sparsify_ms": sparsify_ms,
           "gpu_launches": launches}
    if workloads:
        out["workloads"] = workloads
    if forms:
        out["sparsify_forms"] = forms
    if bforms:
        out["batched_forms"] = bforms
    if lforms:
        out["learned_forms"] = lforms
    if mlp:
        out["mlp_forward"] = mlp
    if mlp_tr:
        out["mlp_train"] = mlp_tr
    if small:
        out["small_graph_latency"] = small
    if world == 1 and not args.no_cpu_baseline and extra:
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
    ap.add_argument("--kappa-steps", type=int, default=100,
                    help="Lanczos steps of every kappa in the matched-kappa reports")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the other workload shapes (power grid, Chung-Lu, batch)")
    ap.add_argument("--headline-only", action="store_true",
                    help="only the headline line (no workloads, forms, reports or CPU baseline)")
    ap.add_argument("--profile", action="store_true",
                    help="time only the filter+score steps (for ncu launch lists and counters)")
    ap.add_argument("--profile-workload", default="grid", choices=["grid", "chunglu"],
                    help="workload of --profile: the 128^3 grid or the 4M-node Chung-Lu graph")
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
