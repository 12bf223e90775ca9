"""Benchmark of the EbV solver on one GB300 (or N replicas under torchrun).

Workload: dense, unit-diagonal, strictly row-diagonally-dominant A, n=16384,
off-diagonals U[-0.9, 0.9]/(n-1), 32 planted right-hand sides (b = A x_true),
seeded.  One step = mixed-precision EbV factorisation (bfloat16 trailing
updates on the tensor cores, FP32 factors) + FP64 iterative refinement of the
32 solutions until the relative residual max_c ||b_c - A x_c|| / ||b_c|| is
<= 1e-12.  The plain FP64 EbV path on the same GPU is measured beside it.

Metric: nominal factor+solve GFLOP/s, 2n^3/3 + 2 n^2 nrhs flops per step (the
HPL convention: refinement work is not credited), and solves/s.

Output: one JSON line (rank 0).  --impl reference runs the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "factor+solve GFLOP/s & solves/s, mixed vs FP64 EbV at rel. resid ≤1e-12"
N_FULL, NRHS_FULL = 16384, 32
TOL = 1e-12


def nominal_flops(n, nrhs):
    return 2.0 * n ** 3 / 3.0 + 2.0 * n * n * nrhs


def oracle_sample_flops(n, kstop):
    k = np.arange(kstop, dtype=np.float64)
    m = n - k - 1
    return float(np.sum(m + 2.0 * m * m))


def workload_desc(n, nrhs):
    return (f"dense DD n={n}, {nrhs} RHS, offdiag U[-0.9,0.9]/(n-1); EbV factor with bf16 tensor-core Schur "
            f"updates + FP64 iterative refinement to rel. resid <= {TOL:g}")


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    INTERVAL_MS = 100

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self, first_sample_s: float = 3.0):
        """Start sampling; returns once the first sample is in (at most
        first_sample_s seconds), so the timed region that follows is covered
        from its start."""
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", str(self.INTERVAL_MS)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        deadline = time.monotonic() + first_sample_s
        while not self.lines and self.proc.poll() is None and time.monotonic() < deadline:
            time.sleep(0.005)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": float(np.median(loaded)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm), "interval_ms": self.INTERVAL_MS}


# ----------------------------------------------------------------------------
# CPU oracle baseline
# ----------------------------------------------------------------------------

def cpu_oracle_rate(a: np.ndarray, kstop: int, threads: int = 0):
    """Time the oracle's FP64 Doolittle on the first kstop elimination steps of
    the full workload matrix; returns (GFLOP/s, seconds, threads)."""
    import oracle
    used = oracle.set_threads(threads if threads > 0 else (os.cpu_count() or 1))
    t0 = time.perf_counter()
    oracle.lu(a, kstop=kstop)
    dt = time.perf_counter() - t0
    return oracle_sample_flops(a.shape[0], kstop) / dt / 1e9, dt, used


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name"):
                return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def max_over_ranks(ms, dist, device):
    """The slowest rank's time (every rank gets it); the time itself at N = 1."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gflops(world, flops_per_replica, ms):
    """Replicas only (no data-path collective): every rank solves its own
    system per step, so the job's rate is world systems per slowest step."""
    return world * flops_per_replica / (ms / 1e3) / 1e9


def shard_of_rank(ns, rs, world, rank):
    """Indices (ascending) of the systems of a batch that rank `rank` of
    `world` solves: the library's size-balanced split (long/short pairs of
    Eq. 7 across systems, then longest-first onto the least-loaded rank).
    Every rank computes the same split; no data moves between ranks."""
    import paper_1907_05767_gb300 as ebv
    rank_of, cost = ebv.ebv_batch_partition(ns, rs, world)
    return np.flatnonzero(rank_of == rank), rank_of, cost


def gather_by_system(values, idx, batch, dist, device):
    """Every rank's per-system values (int64, in the order of its `idx`) put
    back into system order on every rank: the batched workload's only
    exchange, done once after the timed region (per-system info words)."""
    import torch
    full = torch.zeros(batch, dtype=torch.int64, device=device)
    full[torch.as_tensor(idx, dtype=torch.int64, device=device)] = torch.as_tensor(values, dtype=torch.int64,
                                                                                   device=device)
    if dist is not None:
        dist.all_reduce(full, op=dist.ReduceOp.SUM)  # each system is owned by exactly one rank
    return full.cpu().numpy()


def run_batched(args, rank, world, dist):
    """The batched workload: 4096 dense systems n ~ U{16..512}, 1-4 RHS, in
    FP64 or FP32, split across the ranks by size (no exchange in the data
    path); each rank solves its share in one persistent launch replayed from
    a CUDA graph.  The value is systems (and nominal flops) of the whole job
    per slowest rank's step."""
    import torch

    import paper_1907_05767_gb300 as ebv
    import synthetic
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    ns, rs = synthetic.config3_sizes()
    idx, _, cost = shard_of_rank(ns, rs, world, rank)
    vmap, tuned = None, None
    if args.autotune:
        vmap, tuned = ebv.batch_autotune_buckets(args.batched_prec, cache_path=args.tune_cache)
    bt = ebv.Batch(ns[idx], rs[idx], args.batched_prec, device=dev, variant_of_n=vmap)
    for k, s in enumerate(idx):
        a, _, b = synthetic.config3_system(int(s), int(ns[s]), int(rs[s]))
        bt.a_view(k).copy_(torch.from_numpy(a))
        bt.b_view(k).copy_(torch.from_numpy(b))
    a0, b0 = bt.a_buf.clone(), bt.b_buf.clone()

    def restore():
        bt.a_buf.copy_(a0)
        bt.b_buf.copy_(b0)

    def step():
        restore()
        bt.run()

    ms_restore = _dev_ms(restore, args.steps, args.warmup)
    ms_all = _dev_ms(step, args.steps, max(3, args.warmup))
    ms = max_over_ranks(ms_all - ms_restore, dist, dev)
    info = gather_by_system(bt.info.cpu().numpy(), idx, len(ns), dist, dev)
    flops = float(sum(nominal_flops(int(n), int(r)) for n, r in zip(ns, rs)))
    line = {"metric": "batched factor+solve solves/s & GFLOP/s (4096 systems n~U{16..512}, 1-4 RHS)",
            "value": len(ns) * 1e3 / ms, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
            "gflops": flops / (ms / 1e3) / 1e9, "dtype": args.batched_prec, "data": "synthetic (seeded)",
            "config": {"workload": "batched 4096 systems n~U{16..512}, 1-4 RHS, offdiag U[-0.5,0.5]/(n-1)",
                       "parallelism": f"systems split over {world} rank(s) by cost, no exchange",
                       "cuda_graph": True, "l2": "restore of the inputs (1.5-3 GB) between steps flushes L2",
                       "rank_cost_spread": float(cost.max() / max(cost.min(), 1.0))},
            "info_nonzero": int(np.count_nonzero(info)), "gpu_launches": 1,
            "tuned_variants": tuned}
    return line


def run_gpu(args, rank, world, dist):
    import torch

    import paper_1907_05767_gb300 as ebv
    import synthetic

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, nrhs = args.n, args.nrhs
    prec = args.prec

    t_gen = time.perf_counter()
    a_np, x_true, b_np = synthetic.config2(n, nrhs)
    t_gen = time.perf_counter() - t_gen

    a = torch.from_numpy(a_np).to(dev)
    b0 = torch.from_numpy(b_np).to(dev)
    lowp = torch.empty((n, n), dtype=torch.float32, device=dev)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = ebv.workspace(n, prec, nrhs, dev)
    rep = torch.zeros(3, dtype=torch.float64, device=dev)
    x = torch.empty_like(b0)
    stream = torch.cuda.current_stream(dev)

    def step():
        x.copy_(b0)
        ebv.ebv_factor(a, prec, lowp=lowp, info=info, ws=ws)
        ebv.ebv_solve(lowp, x, prec, a_orig=a, refine=(TOL, args.max_iter), report=rep, ws=ws, ld=n)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    rep_np = ebv.read_report(rep)
    launches_per_step = ebv.launch_count()
    step()
    torch.cuda.synchronize()
    launches_per_step = ebv.launch_count() - launches_per_step

    # The whole step (factor + refined solve) as one CUDA graph: the library
    # never synchronises or allocates inside a call, so it captures as is.
    graph = None
    if args.graph:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step()
        graph.replay()
        torch.cuda.synchronize()
    run = graph.replay if graph is not None else step

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        run()
    e1.record(stream)
    barrier()
    clk = clocks.stop()
    launches = launches_per_step * args.steps
    ms_total = e0.elapsed_time(e1)
    ms = ms_total / args.steps
    ms = max_over_ranks(ms, dist, dev)
    rep_np = ebv.read_report(rep)
    info_v = int(info.item())

    # accuracy of the last step against the planted solution and by the oracle residual (sampled rows)
    import oracle
    xs = x.cpu().numpy()
    rows = synthetic.pick_indices(7, 256, [n])[:, 0]
    r_s = oracle.residual(a_np, xs, b_np, rows=rows)
    rel_resid_sampled = float((np.abs(r_s).max(axis=0) / np.abs(b_np).max(axis=0)).max())
    err_true = float(np.abs(xs - x_true).max() / np.abs(x_true).max())

    flops = nominal_flops(n, nrhs)
    value = whole_job_gflops(world, flops, ms)

    # per-kernel-class device times of one more (profiled) step
    ebv.profile(True)
    step()
    torch.cuda.synchronize()
    prof = ebv.profile_read()
    ebv.profile(False)

    # end to end through the C ABI from pinned host buffers: ebv_gesv_host
    # copies A (column blocks, overlapped with the factorisation) and B in,
    # factors, solves with refinement and copies X back.
    a_host = torch.from_numpy(a_np).pin_memory()
    b_host = torch.from_numpy(b_np).pin_memory()
    x_host = torch.empty_like(b_host).pin_memory()
    rep_host = torch.zeros(32, dtype=torch.uint8).pin_memory()
    ws_host_path = ebv.gesv_host_workspace(n, nrhs, prec)

    def e2e_step():
        ebv.ebv_gesv_host(a_host, b_host, x_host, prec=prec, refine=(TOL, args.max_iter), report_host=rep_host,
                          ws=ws_host_path)

    e2e_step()
    barrier()
    e2e_run = e2e_step
    if args.graph:
        g2 = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g2):
            e2e_step()
        g2.replay()
        e2e_run = g2.replay
    barrier()
    f0 = torch.cuda.Event(enable_timing=True)
    f1 = torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.e2e_steps):
        e2e_run()
    f1.record(stream)
    barrier()
    e2e_ms = f0.elapsed_time(f1) / args.e2e_steps
    e2e_val = world * flops / (e2e_ms / 1e3) / 1e9
    e2e_rep = ebv.read_report(rep_host)
    e2e_err = float(np.abs(x_host.numpy() - x_true).max() / np.abs(x_true).max())
    del ws_host_path

    # plain FP64 EbV on the same GPU (same matrix and right-hand sides)
    fp64 = None
    if args.fp64_steps > 0:
        lu64 = torch.empty_like(a)
        x64 = torch.empty_like(b0)
        ws64 = ebv.workspace(n, "fp64", nrhs, dev)

        def step64():
            lu64.copy_(a)
            x64.copy_(b0)
            ebv.ebv_factor(lu64, "fp64", info=info, ws=ws64)
            ebv.ebv_solve(lu64, x64, "fp64", ws=ws64)

        torch.cuda.synchronize()
        g0 = torch.cuda.Event(enable_timing=True)
        g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        for _ in range(args.fp64_steps):
            step64()
        g1.record(stream)
        torch.cuda.synchronize()
        ms64 = g0.elapsed_time(g1) / args.fp64_steps
        x64n = x64.cpu().numpy()
        r64 = oracle.residual(a_np, x64n, b_np, rows=rows)
        fp64 = {"gflops": flops / (ms64 / 1e3) / 1e9, "ms_per_step": ms64,
                "rel_resid_sampled": float((np.abs(r64).max(axis=0) / np.abs(b_np).max(axis=0)).max()),
                "speedup_mixed_vs_fp64": ms64 / ms}
        del lu64, x64, ws64

    # roofline of the dominant kernel class
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    dom = max(prof.items(), key=lambda kv: kv[1][0])
    dom_name, (dom_ms, dom_work, dom_cnt) = dom
    roofline = roofline_for(dom_name, dom_ms, dom_work, dom_cnt, peaks, args, active=active_launches(dom_name, rep_np))

    cpu = None
    if rank == 0 and world == 1 and args.cpu_kstop > 0:
        rate, secs, used = cpu_oracle_rate(a_np, args.cpu_kstop)
        cpu = {"value": rate, "unit": "GFLOP/s", "cores": used, "kind": "oracle",
               "sample": f"oracle FP64 Doolittle (kij, OpenMP rows) on the first {args.cpu_kstop} elimination "
                         f"steps of the n={n} workload matrix ({secs:.1f} s, {cpu_model()}); GFLOP/s of those steps",
               "est_solve_s": flops / (rate * 1e9)}

    line = {
        "metric": METRIC, "value": value, "unit": "GFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16 (tensor-core updates) / fp32 (factors) / fp64 (refinement)",
        "data": "synthetic (seeded, planted solutions)",
        "config": {"workload": workload_desc(n, nrhs), "n": n, "nrhs": nrhs, "precision": prec,
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "cuda_graph": bool(args.graph),
                   "l2": "inputs larger than L2 (A is %.2f GB FP64)" % (n * n * 8 / 1e9)},
        "solves_per_s": world * 1e3 / ms, "rhs_per_s": world * nrhs * 1e3 / ms,
        "refinement": {"iters": rep_np["iters"], "status": rep_np["status"], "resid_first": rep_np["resid_first"],
                       "resid_final": rep_np["resid_final"], "rel_resid_sampled_oracle": rel_resid_sampled,
                       "err_vs_x_true": err_true, "info": info_v},
        "fp64_plain": fp64,
        "roofline": roofline,
        "rooflines_by_class": {k: roofline_for(k, v[0], v[1], v[2], peaks, args, active=active_launches(k, rep_np))
                               for k, v in prof.items() if v[2] > 0},
        "kernel_classes_ms": {k: round(v[0], 4) for k, v in prof.items() if v[2] > 0},
        "kernel_classes_launches": {k: v[2] for k, v in prof.items() if v[2] > 0},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_val, "unit": "GFLOP/s", "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": int(a_np.nbytes + b_np.nbytes), "d2h_bytes_per_step": int(b_np.nbytes),
                "api": "ebv_gesv_host (host A, B -> host X)", "resid_final": e2e_rep["resid_final"],
                "err_vs_x_true": e2e_err},
        "gpu_launches": int(launches),
        "clocks": clk,
        "input_gen_s": t_gen,
    }
    return line


def active_launches(name, rep):
    """Launches of a refinement-loop class that did work: iters + 1 residuals,
    2 (iters + 1) triangles."""
    it = int(rep["iters"]) + 1
    return {"residual": it, "trsv": 2 * it}.get(name)


def roofline_for(name, ms, work, cnt, peaks, args, active=None):
    if cnt == 0 or ms <= 0:
        return None
    per_launch_ms = ms / cnt
    if name in ("lowp_gemm",):
        tc = args.tc_used
        if tc:
            peak = peaks.get("bf16_tflops_sustained") or 1700.0
            src = "measured bf16 sustained" if "bf16_tflops_sustained" in peaks else "fallback"
            bound = "tensor"
        else:
            peak, src, bound = 75.1, "measured FFMA probe (FP32 SIMT fallback)", "alu"
        achieved = work / (ms / 1e3) / 1e12
        return {"bound": bound, "kernel": name, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "peak_source": src, "launches": cnt,
                "avg_launch_ms": per_launch_ms}
    if name == "residual":
        # Tensor-core residual: reads A (8 n^2 bytes, FP64) once per evaluation;
        # reported against HBM bandwidth.  Launches after the stop test has
        # passed exit at once: only `active` of them evaluate a residual.
        act = active if active else cnt
        n = args.n
        bytes_per = 8.0 * n * n
        achieved = bytes_per * act / (ms / 1e3) / 1e9
        peak = peaks.get("hbm_gbs") or 6800.0
        src = "measured HBM copy" if "hbm_gbs" in peaks else "fallback"
        return {"bound": "hbm", "kernel": name, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": None, "peak_source": src,
                "launches": act, "avg_launch_ms": ms / act}
    if name == "trsv" and active:
        # Substitution launches after the stop test has passed exit at once:
        # only the diagonal inverses and `active` triangles do work.
        work = work * (active + 1) / cnt
    achieved = work / (ms / 1e3) / 1e12
    return {"bound": "alu", "kernel": name, "achieved": achieved, "peak": 75.1, "unit": "TFLOP/s",
            "frac": achieved / 75.1, "traffic": None, "peak_source": "measured FFMA probe", "launches": cnt,
            "avg_launch_ms": per_launch_ms}


# ----------------------------------------------------------------------------
# single-kernel mode: the mixed-precision trailing update alone
# ----------------------------------------------------------------------------

def run_update_only(args):
    """Time C -= L21 U12 (bf16 operands, FP32 C) for one M x N x K update with
    the tcgen05 kernel, as in the top level of the n = 2M factorisation."""
    import torch

    import paper_1907_05767_gb300 as ebv
    m, n, k = (int(v) for v in args.update_only.split(","))
    dev = torch.device("cuda")
    g = torch.Generator(device="cpu").manual_seed(1)
    ld = (k + 63) // 64 * 64
    lb = ((torch.rand((m, ld), generator=g) - 0.5) * 1e-3).to(torch.bfloat16).to(dev)
    ut = ((torch.rand((n, ld), generator=g) - 0.5) * 1e-3).to(torch.bfloat16).to(dev)
    c = torch.rand((m, n), generator=g, dtype=torch.float32).to(dev)
    scale = torch.tensor([1.0, 1.0, 1.0, 0.0], device=dev)
    ws = torch.zeros(256, dtype=torch.uint8, device=dev)
    for _ in range(args.warmup):
        ebv.debug_lowp_update(c, lb, ut, scale, 0, 0, 0, m, n, k, "tc", ws=ws)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        ebv.debug_lowp_update(c, lb, ut, scale, 0, 0, 0, m, n, k, "tc", ws=ws, check=False)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    tf = 2.0 * m * n * k / (ms / 1e3) / 1e12
    peak = peaks.get("bf16_tflops", 1900.0)
    return {"kernel": "k_tc_update", "m": m, "n": n, "k": k, "ms": ms, "tflops": tf, "peak_bf16_burst": peak,
            "frac": tf / peak, "bytes_min": 8.0 * m * n + 2.0 * k * (m + n),
            "hbm_gbs_at_min_bytes": (8.0 * m * n + 2.0 * k * (m + n)) / (ms / 1e3) / 1e9}


# ----------------------------------------------------------------------------
# --configs: the other workloads (parity cases of the test suite), one JSON
# line each, for the results table; not the bench line
# ----------------------------------------------------------------------------

def _dev_ms(fn, steps, warmup, graph=True):
    """Device ms per call of fn (CUDA events on the launching stream), replayed
    from a CUDA graph unless graph is False."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    run = fn
    if graph:
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            fn()
        g.replay()
        torch.cuda.synchronize()
        run = g.replay
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        run()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


def _peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def run_configs(args):
    import torch

    import oracle
    import paper_1907_05767_gb300 as ebv
    import synthetic
    dev = torch.device("cuda")
    hbm = _peaks().get("hbm_gbs", 6800.0)
    out = []
    names = set(str(args.configs).split(","))

    def want(name):
        return "all" in names or name in names

    if want("dense256"):
        out.append(_config_dense256(args, dev))
    if want("band"):
        out.extend(_config_band(args, dev))
    if want("fp16"):
        out.append(_config_fp16(args, dev))
    if want("batched"):
        out.extend(_config_batched(args, dev))
    if want("adjoint"):
        out.append(_config_adjoint(args, dev, hbm))
    if want("inverse"):
        out.append(run_inverse_config(args))
    if want("profile"):
        out.append(run_profile_config(args))
    if want("band_mixed"):
        out.append(run_band_mixed_config(args))
    if want("dense_sym"):
        out.append(_config_dense_sym(args, dev))
    return out


def _config_dense256(args, dev):
    import torch

    import oracle
    import paper_1907_05767_gb300 as ebv
    import synthetic
    out = []
    # n = 256 dense FP64, one RHS (L2-resident: the whole problem is 0.5 MB)
    a, x_true, b = synthetic.config0()
    n = a.shape[0]
    A, B = torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)
    lu, x = torch.empty_like(A), torch.empty_like(B)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = ebv.workspace(n, "fp64", 1, dev)

    def c0():
        lu.copy_(A)
        x.copy_(B)
        ebv.ebv_factor(lu, "fp64", info=info, ws=ws)
        ebv.ebv_solve(lu, x, "fp64", ws=ws)

    def c0_factor():
        lu.copy_(A)
        ebv.ebv_factor(lu, "fp64", info=info, ws=ws)

    ebv.lib().ebv_debug_set_small_dense(0)  # the same on one thread-block cluster
    ms_cluster = _dev_ms(c0, 200, 10)
    ebv.lib().ebv_debug_set_small_dense(1)
    ms_factor = _dev_ms(c0_factor, 200, 10)
    ms = _dev_ms(c0, 200, 10)
    x_ref = oracle.solve(oracle.lu(a)[0], b)
    xs = x.cpu().numpy()
    r = oracle.residual(a, xs, b)
    out.append({"config": "dense FP64 n=256, 1 RHS", "ms": ms, "ms_factor_incl_copy": ms_factor,
                "ms_on_cluster_panel": ms_cluster,
                "solves_per_s": 1e3 / ms,
                "gflops": nominal_flops(n, 1) / (ms / 1e3) / 1e9,
                "x_relerr_vs_oracle": float(np.abs(xs - x_ref).max() / np.abs(x_ref).max()),
                "backward_error": float(np.abs(r).max() / (np.abs(a).sum(axis=1).max() * np.abs(xs).max())),
                "note": "whole problem L2-resident (CUDA graph); 64-column panels with substitution L21/U12, "
                        "one-CTA block substitution solve"})
    print(json.dumps(out[-1]), flush=True)
    return out[-1]


def _config_band(args, dev):
    import torch

    import oracle
    import paper_1907_05767_gb300 as ebv
    import synthetic
    out = []
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    # banded FP64 5-point Laplacian on a 512 x 512 grid (--band-grid), 8 RHS
    ab, kl, ku, x_true, b = synthetic.config1(args.band_grid)
    n = ab.shape[0]
    AB, B = torch.from_numpy(ab).to(dev), torch.from_numpy(b).to(dev)
    lu, x = torch.empty_like(AB), torch.empty_like(B)
    ws = ebv.workspace(n, "fp64", b.shape[1], dev, kl=kl, ku=ku, storage=ebv.BAND)

    def c1():
        lu.copy_(AB)
        x.copy_(B)
        ebv.ebv_factor(lu, "fp64", info=info, ws=ws, kl=kl, ku=ku, storage=ebv.BAND)
        ebv.ebv_solve(lu, x, "fp64", ws=ws, kl=kl, ku=ku, storage=ebv.BAND)

    # the same with the panels on thread-block clusters
    ebv.lib().ebv_debug_set_band_cluster(1)
    ms_cluster = _dev_ms(c1, 3, 2)
    ebv.lib().ebv_debug_set_band_cluster(0)
    # the same with the blocked 16 x 16 sub-block diagonal-block kernel
    ebv.lib().ebv_debug_set_diag_lu(0)
    ms_diag_blocked = _dev_ms(c1, 3, 2)
    ebv.lib().ebv_debug_set_diag_lu(1)
    # every panel's kernels serial, and without the general band's look-ahead
    ebv.lib().ebv_debug_set_band_lookahead(0)
    ms_serial = _dev_ms(c1, 3, 2)
    ebv.lib().ebv_debug_set_band_lookahead(1)
    ms_no_lookahead = _dev_ms(c1, 3, 2)
    ebv.lib().ebv_debug_set_band_lookahead(2)
    # per kernel class (CUDA events around every launch; classes on the
    # look-ahead's side stream overlap the others)
    ebv.profile(True)
    c1()
    torch.cuda.synchronize()
    classes = {k: round(v[0], 2) for k, v in ebv.profile_read().items() if v[2] > 0}
    ebv.profile(False)
    ms = _dev_ms(c1, 3, 2)
    xs = x.cpu().numpy()
    rows = synthetic.pick_indices(11, 512, [n])[:, 0]
    r = oracle.band_residual(ab, kl, ku, xs, b)[rows]
    flops = 2.0 * n * kl * ku + 2.0 * n * (kl + ku) * b.shape[1]
    g = args.band_grid
    out.append({"config": f"band FP64 Laplacian {g}x{g} (n={n}, kl=ku={kl}), 8 RHS", "ms": ms,
                "ms_cluster_panels": ms_cluster, "ms_blocked_diag_kernel": ms_diag_blocked,
                "ms_serial_panels": ms_serial, "ms_without_lookahead": ms_no_lookahead,
                "class_ms_profiled_run": classes,
                "solves_per_s": 1e3 / ms, "gflops": flops / (ms / 1e3) / 1e9,
                "err_vs_x_true": float(np.abs(xs - x_true).max() / np.abs(x_true).max()),
                "backward_error_sampled": float(np.abs(r).max() / (np.abs(ab).sum(axis=1).max() * np.abs(xs).max())),
                "band_bytes": int(ab.nbytes), "info": int(info.item())})
    print(json.dumps(out[-1]), flush=True)

    # the same Laplacian as a symmetric band (EBV_BAND_SYM: U12 = D11 L21^T,
    # block-lower trailing updates); same output, same nominal flops
    def c1s():
        lu.copy_(AB)
        x.copy_(B)
        ebv.ebv_factor(lu, "fp64", info=info, ws=ws, kl=kl, ku=ku, storage=ebv.BAND_SYM)
        ebv.ebv_solve(lu, x, "fp64", ws=ws, kl=kl, ku=ku, storage=ebv.BAND)

    ebv.lib().ebv_debug_set_band_lookahead(0)
    ms_sym_no_lookahead = _dev_ms(c1s, 3, 2)
    ebv.lib().ebv_debug_set_band_lookahead(2)
    ms = _dev_ms(c1s, 3, 2)
    xs = x.cpu().numpy()
    r = oracle.band_residual(ab, kl, ku, xs, b)[rows]
    out.append({"config": f"band FP64 Laplacian {g}x{g}, symmetric storage mode, 8 RHS", "ms": ms,
                "ms_without_lookahead": ms_sym_no_lookahead,
                "solves_per_s": 1e3 / ms, "gflops": flops / (ms / 1e3) / 1e9,
                "err_vs_x_true": float(np.abs(xs - x_true).max() / np.abs(x_true).max()),
                "backward_error_sampled": float(np.abs(r).max() / (np.abs(ab).sum(axis=1).max() * np.abs(xs).max())),
                "info": int(info.item())})
    print(json.dumps(out[-1]), flush=True)
    del AB, lu, ws

    # the same Laplacian with only the lower half of its band stored
    # (EBV_BAND_SYM_LOWER: kl + 1 entries per row, the LDL^T factors in place)
    ablo = np.ascontiguousarray(ab[:, :kl + 1])
    ABL = torch.from_numpy(ablo).to(dev)
    lul = torch.empty_like(ABL)
    wsl = ebv.workspace(n, "fp64", b.shape[1], dev, ld=kl + 1, kl=kl, ku=ku, storage=ebv.BAND_SYM_LOWER)

    def c1l():
        lul.copy_(ABL)
        x.copy_(B)
        ebv.ebv_factor(lul, "fp64", info=info, ws=wsl, kl=kl, ku=ku, storage=ebv.BAND_SYM_LOWER)
        ebv.ebv_solve(lul, x, "fp64", ws=wsl, kl=kl, ku=ku, storage=ebv.BAND_SYM_LOWER)

    ms = _dev_ms(c1l, 3, 2)
    xs = x.cpu().numpy()
    r = oracle.band_residual(ab, kl, ku, xs, b)[rows]
    out.append({"config": f"band FP64 Laplacian {g}x{g}, symmetric, lower half of the band stored, 8 RHS",
                "ms": ms,
                "solves_per_s": 1e3 / ms, "gflops": flops / (ms / 1e3) / 1e9,
                "err_vs_x_true": float(np.abs(xs - x_true).max() / np.abs(x_true).max()),
                "backward_error_sampled": float(np.abs(r).max() / (np.abs(ab).sum(axis=1).max() * np.abs(xs).max())),
                "band_bytes": int(ablo.nbytes), "band_bytes_full": int(ab.nbytes), "info": int(info.item())})
    print(json.dumps(out[-1]), flush=True)
    del ABL, lul, wsl, B, x
    return out


def _config_fp16(args, dev):
    import torch

    import paper_1907_05767_gb300 as ebv
    import synthetic
    out = []
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    # dense n = 16384, 32 RHS: FP16 updates + refinement (bf16 is the bench line)
    a, x_true, b = synthetic.config2(args.n, args.nrhs)
    n, nrhs = a.shape[0], b.shape[1]
    A, B = torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)
    lowp = torch.empty((n, n), dtype=torch.float32, device=dev)
    x = torch.empty_like(B)
    rep = torch.zeros(3, dtype=torch.float64, device=dev)
    ws = ebv.workspace(n, "fp16", nrhs, dev)

    def c2():
        x.copy_(B)
        ebv.ebv_factor(A, "fp16", lowp=lowp, info=info, ws=ws)
        ebv.ebv_solve(lowp, x, "fp16", a_orig=A, refine=(TOL, args.max_iter), report=rep, ws=ws, ld=n)

    ms = _dev_ms(c2, 3, 3)
    rp = ebv.read_report(rep)
    xs = x.cpu().numpy()
    out.append({"config": f"dense n={n}, {nrhs} RHS, fp16 tensor-core updates + FP64 refinement", "ms": ms,
                "solves_per_s": 1e3 / ms, "gflops": nominal_flops(n, nrhs) / (ms / 1e3) / 1e9,
                "refine_iters": rp["iters"], "resid_first": rp["resid_first"], "resid_final": rp["resid_final"],
                "err_vs_x_true": float(np.abs(xs - x_true).max() / np.abs(x_true).max())})
    print(json.dumps(out[-1]), flush=True)
    del A, B, lowp, x, ws
    return out[-1]


def _config_dense_sym(args, dev):
    """The symmetric mode on the dense n = 16384, 32 RHS matrix made
    symmetric: FP64 LDL^T in the lower triangle (n^3/3 flops) against the
    general FP64 factorisation of the same matrix (2n^3/3)."""
    import torch

    import oracle
    import paper_1907_05767_gb300 as ebv
    import synthetic
    a, _, _ = synthetic.config2(args.n, args.nrhs)
    a = np.tril(a) + np.tril(a, -1).T  # symmetric, still strictly diagonally dominant
    n, nrhs = a.shape[0], args.nrhs
    x_true = synthetic.planted_x(n, nrhs, 90_001)
    b = synthetic.rhs_for(a, x_true)
    A, B = torch.from_numpy(a).to(dev), torch.from_numpy(b).to(dev)
    lu, x = torch.empty_like(A), torch.empty_like(B)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = ebv.workspace(n, "fp64", nrhs, dev, storage=ebv.DENSE_SYM)
    wsg = ebv.workspace(n, "fp64", nrhs, dev)

    def sym():
        lu.copy_(A)
        x.copy_(B)
        ebv.ebv_factor(lu, "fp64", info=info, ws=ws, storage=ebv.DENSE_SYM)
        ebv.ebv_solve(lu, x, "fp64", ws=ws, storage=ebv.DENSE_SYM)

    def gen():
        lu.copy_(A)
        x.copy_(B)
        ebv.ebv_factor(lu, "fp64", info=info, ws=wsg)
        ebv.ebv_solve(lu, x, "fp64", ws=wsg)

    ms_gen = _dev_ms(gen, 1, 1)
    ms = _dev_ms(sym, 2, 1)
    xs = x.cpu().numpy()
    r = oracle.residual(a, xs, b)
    flops = n ** 3 / 3 + 2 * n * n * nrhs
    line = {"config": f"dense symmetric n={n}, {nrhs} RHS, FP64 LDL^T in the lower triangle", "ms": ms,
            "gflops": flops / (ms / 1e3) / 1e9, "ms_general_fp64": ms_gen,
            "speedup_vs_general": ms_gen / ms, "info": int(info.item()),
            "backward_error": float(np.abs(r).max() / (np.abs(a).sum(axis=1).max() * np.abs(xs).max())),
            "err_vs_x_true": float(np.abs(xs - x_true).max() / np.abs(x_true).max()),
            "note": "flops credited: n^3/3 + 2 n^2 nrhs (the symmetric factorisation's own work)"}
    print(json.dumps(line), flush=True)
    del A, B, lu, x, ws, wsg
    torch.cuda.empty_cache()
    return line


def _config_batched(args, dev):
    import torch

    import paper_1907_05767_gb300 as ebv
    import synthetic
    out = []
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    # batched: 4096 systems, n ~ U{16..512}, 1-4 RHS, FP64 and FP32
    ns, rs = synthetic.config3_sizes()
    systems = [synthetic.config3_system(s, int(ns[s]), int(rs[s])) for s in range(len(ns))]
    flops = float(sum(nominal_flops(int(nn), int(rr)) for nn, rr in zip(ns, rs)))
    pick = synthetic.pick_indices(99, 16, [len(ns)])[:, 0]
    for prec in ("fp64", "fp32"):
        # the autotuner's variant per size bucket (block width x update tile)
        vmap, tuned = ebv.batch_autotune_buckets(prec, cache_path=args.tune_cache)
        bt = ebv.Batch(ns, rs, prec, variant_of_n=vmap)
        for s, (a, _, b) in enumerate(systems):
            bt.a_view(s).copy_(torch.from_numpy(a))
            bt.b_view(s).copy_(torch.from_numpy(b))
        a0, b0 = bt.a_buf.clone(), bt.b_buf.clone()
        sched_tuned = bt.sched.clone()
        sched_default = torch.from_numpy(ebv.ebv_batch_schedule(ns, rs)).to(dev)

        def restore():
            bt.a_buf.copy_(a0)
            bt.b_buf.copy_(b0)

        def c3():
            restore()
            bt.run()

        ms_restore = _dev_ms(restore, 10, 3)
        bt.sched = sched_default
        ms_default = _dev_ms(c3, 10, 3) - ms_restore
        bt.sched = sched_tuned
        ms_all = _dev_ms(c3, 10, 3)  # last: the buffers hold the factors and X
        err = 0.0
        for s in pick:
            _, xt, _ = systems[s]
            err = max(err, float(np.abs(bt.b_view(int(s)).double().cpu().numpy() - xt).max() / np.abs(xt).max()))
        ms_run = ms_all - ms_restore
        line = {"config": f"batched 4096 systems n~U{{16..512}}, 1-4 RHS, {prec}", "ms": ms_run,
                "ms_incl_restore": ms_all, "solves_per_s": len(ns) * 1e3 / ms_run,
                "gflops": flops / (ms_run / 1e3) / 1e9, "launches": 1,
                "ms_default_variants": ms_default, "tuned_variants": tuned,
                "err_vs_x_true_sampled": err, "info_max": int(bt.info.abs().max())}
        if prec == "fp64":
            # the same systems one at a time through ebv_factor + ebv_solve
            wsp = ebv.workspace(512, "fp64", 4, dev)
            views = [(bt.a_view(s), bt.b_view(s)) for s in range(len(ns))]
            restore()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for av, bv in views:
                ebv.ebv_factor(av, "fp64", info=info, ws=wsp)
                ebv.ebv_solve(av, bv, "fp64", ws=wsp)
            e1.record()
            torch.cuda.synchronize()
            line["per_system_launches_ms"] = e0.elapsed_time(e1)
            line["speedup_vs_per_system"] = line["per_system_launches_ms"] / ms_run
        out.append(line)
        print(json.dumps(out[-1]), flush=True)
        del bt, a0, b0
    del systems
    return out


def _config_adjoint(args, dev, hbm):
    import torch

    import oracle
    import paper_1907_05767_gb300 as ebv
    import synthetic
    # differentiable batch: 256 FP64 systems n = 1024, 4 RHS; forward + adjoint
    nb, n, nrhs = 256, 1024, 4
    data = [synthetic.config4_system(i, n, nrhs) for i in range(nb)]
    A = torch.from_numpy(np.stack([d[0] for d in data])).to(dev)
    B = torch.from_numpy(np.stack([d[2] for d in data])).to(dev)
    W = torch.from_numpy(np.stack([d[3] for d in data])).to(dev)
    lu, x = torch.empty_like(A), torch.empty_like(B)
    bt = ebv.uniform_batch(lu, x)

    def fwd():
        lu.copy_(A)
        x.copy_(B)
        bt.run()

    ms_copy = _dev_ms(lambda: (lu.copy_(A), x.copy_(B)), 5, 2)
    ms_f = _dev_ms(fwd, 5, 2)  # last: lu and x hold the factors and X
    g_b, g_a = ebv.ebv_solve_adjoint(lu, x, W)
    torch.cuda.synchronize()
    ms_b = _dev_ms(lambda: ebv.ebv_solve_adjoint(lu, x, W), 5, 2, graph=False)
    err = 0.0
    for i in synthetic.pick_indices(5, 3, [nb])[:, 0]:
        luo = oracle.lu(data[i][0])[0]
        xo = oracle.solve(luo, data[i][2])
        gbo, gao = oracle.adjoint(luo, xo, data[i][3])
        err = max(err, float(np.abs(g_b[i].cpu().numpy() - gbo).max() / np.abs(gbo).max()),
                  float(np.abs(g_a[i].cpu().numpy() - gao).max() / np.abs(gao).max()))
    # backward: two transposed substitutions (n^2 nrhs / 2 multiply-adds each)
    # and grad_A = -grad_B X^T (n^2 nrhs) -- FP64-pipe bound on this GPU;
    # bytes: each triangle of the factors read once, grad_A written
    bwd_flops = nb * 4.0 * n * n * nrhs
    bwd_bytes = nb * 8.0 * n * n * 2
    line = {"config": "adjoint batch 256 x FP64 n=1024, 4 RHS", "ms_forward": ms_f - ms_copy,
                "ms_backward": ms_b, "forward_gflops": nb * nominal_flops(n, nrhs) / ((ms_f - ms_copy) / 1e3) / 1e9,
                "backward_gflops_fp64": bwd_flops / (ms_b / 1e3) / 1e9,
                "backward_gbs": bwd_bytes / (ms_b / 1e3) / 1e9, "backward_hbm_frac": bwd_bytes / (ms_b / 1e3) / 1e9 / hbm,
                "grad_relerr_vs_oracle_sampled": err, "info_max": int(bt.info.abs().max())}
    print(json.dumps(line), flush=True)
    return line


def run_band_mixed_config(args):
    """The banded Laplacian (512 x 512 grid, 8 RHS) in mixed precision: FP32
    factors of the FP64 band, refinement in FP64 to a relative residual of
    1e-12; one step = factor + refined solve, as a CUDA graph."""
    import torch

    import oracle
    import paper_1907_05767_gb300 as ebv
    import synthetic
    dev = torch.device("cuda")
    ab, kl, ku, x_true, b = synthetic.config1()
    n, nrhs = ab.shape[0], b.shape[1]
    AB, B = torch.from_numpy(ab).to(dev), torch.from_numpy(b).to(dev)
    lowp = torch.empty(AB.shape, dtype=torch.float32, device=dev)
    x = torch.empty_like(B)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    rep = torch.zeros(3, dtype=torch.float64, device=dev)
    ws = ebv.workspace(n, "bf16", nrhs, dev, kl=kl, ku=ku, storage=ebv.BAND)

    def step():
        x.copy_(B)
        ebv.ebv_factor(AB, "bf16", lowp=lowp, info=info, ws=ws, kl=kl, ku=ku, storage=ebv.BAND)
        ebv.ebv_solve(lowp, x, "bf16", a_orig=AB, refine=(1e-12, 10), report=rep, ws=ws, kl=kl, ku=ku,
                      storage=ebv.BAND)

    ms = _dev_ms(step, 3, 1)
    r = ebv.read_report(rep)
    xs = x.cpu().numpy()
    rows = synthetic.pick_indices(11, 512, [n])[:, 0]
    res = oracle.band_residual(ab, kl, ku, xs, b)[rows]
    flops = 2.0 * n * kl * ku + 2.0 * n * (kl + ku) * nrhs
    line = {"config": "band Laplacian 512x512 (n=262144, kl=ku=512), 8 RHS, FP32 factors + FP64 refinement to 1e-12",
            "ms": ms, "gflops_nominal_fp64": flops / (ms / 1e3) / 1e9, "iters": r["iters"],
            "resid_first": r["resid_first"], "resid_final": r["resid_final"], "status": r["status"],
            "err_vs_x_true": float(np.abs(xs - x_true).max() / np.abs(x_true).max()),
            "backward_error_sampled": float(np.abs(res).max() / (np.abs(ab).sum(axis=1).max() * np.abs(xs).max())),
            "info": int(info.item())}
    print(json.dumps(line), flush=True)
    return line


def profile_work(ab, kl, ku):
    """Flops of a no-pivot LU confined to the profile: sum over steps k of
    2 r_k c_k, r_k (c_k) = the rows below (columns right of) k whose first
    non-zero left of (above) the diagonal is at or before k."""
    n = ab.shape[0]
    i = np.arange(n)
    low = ab[:, :kl] != 0.0
    f = np.where(low.any(axis=1), i - kl + np.argmax(low, axis=1), i)
    g = i.copy()
    for d in range(ku, 0, -1):  # column j, row j - d: slot kl + d of row j - d
        j = np.arange(d, n)
        hit = ab[j - d, kl + d] != 0.0
        g[j[hit]] = np.minimum(g[j[hit]], j[hit] - d)
    r = np.zeros(n + 1)
    c = np.zeros(n + 1)
    np.add.at(r, f, 1.0)
    np.add.at(r, i, -1.0)
    np.add.at(c, g, 1.0)
    np.add.at(c, i, -1.0)
    r, c = np.cumsum(r)[:n], np.cumsum(c)[:n]
    return float(2.0 * (r * c).sum()), float(r.sum()), float(c.sum())


def run_profile_config(args):
    """Variable band: the 5-point Laplacian on a disc of radius 289 (n = 262341,
    stored in its widest band kl = ku = 578), FP64, 8 RHS; factorisation with
    and without the block-envelope skipping."""
    import torch

    import oracle
    import paper_1907_05767_gb300 as ebv
    import synthetic
    dev = torch.device("cuda")
    ab, kl, ku = synthetic.laplacian_disc_band(289)
    n, nrhs = ab.shape[0], 8
    x_true = synthetic.planted_x(n, nrhs, synthetic.seed_for(1, 7))
    b = synthetic.band_rhs(ab, kl, ku, x_true)
    AB, B = torch.from_numpy(ab).to(dev), torch.from_numpy(b).to(dev)
    lu, x = torch.empty_like(AB), torch.empty_like(B)
    info = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = ebv.workspace(n, "fp64", nrhs, dev, kl=kl, ku=ku, storage=ebv.BAND)

    def step():
        lu.copy_(AB)
        x.copy_(B)
        ebv.ebv_factor(lu, "fp64", info=info, ws=ws, kl=kl, ku=ku, storage=ebv.BAND)
        ebv.ebv_solve(lu, x, "fp64", ws=ws, kl=kl, ku=ku, storage=ebv.BAND)

    ebv.lib().ebv_debug_set_band_envelope(0)
    ms_full = _dev_ms(step, 3, 1)
    ebv.lib().ebv_debug_set_band_envelope(1)
    ms = _dev_ms(step, 3, 1)
    xs = x.cpu().numpy()
    rows = synthetic.pick_indices(12, 512, [n])[:, 0]
    r = oracle.band_residual(ab, kl, ku, xs, b)[rows]
    del AB, lu, ws

    # the same matrix in profile storage (EBV_PROFILE: per 64-block from the
    # envelope start), factors in place
    buf, klp, kup = ebv.ebv_profile_from_band(ab, kl, ku, "fp64")
    P0 = torch.from_numpy(buf).to(dev)
    P = torch.empty_like(P0)
    wsp = ebv.workspace(n, "fp64", nrhs, dev, ld=0, kl=klp, ku=kup, storage=ebv.PROFILE)

    def pstep():
        P.copy_(P0)
        x.copy_(B)
        ebv.ebv_factor(P, "fp64", info=info, ws=wsp, kl=klp, ku=kup, storage=ebv.PROFILE, n=n)
        ebv.ebv_solve(P, x, "fp64", ws=wsp, kl=klp, ku=kup, storage=ebv.PROFILE, ld=0)

    ms_prof = _dev_ms(pstep, 3, 1)
    xp = x.cpu().numpy()
    rp = oracle.band_residual(ab, kl, ku, xp, b)[rows]
    del P0, P, wsp
    work, rsum, csum = profile_work(ab, kl, ku)
    flops = work + 2.0 * (rsum + csum) * nrhs
    line = {"config": f"variable band FP64: Laplacian on a disc of radius 289 (n={n}, widest band kl=ku={kl}), "
                      f"{nrhs} RHS", "ms": ms, "ms_without_envelope": ms_full, "speedup_envelope": ms_full / ms,
            "profile_gflop": flops / 1e9, "band_gflop": (2.0 * n * kl * ku + 2.0 * n * (kl + ku) * nrhs) / 1e9,
            "gflops_profile": flops / (ms / 1e3) / 1e9,
            "err_vs_x_true": float(np.abs(xs - x_true).max() / np.abs(x_true).max()),
            "backward_error_sampled": float(np.abs(r).max() / (np.abs(ab).sum(axis=1).max() * np.abs(xs).max())),
            "band_bytes": int(ab.nbytes),
            "profile_storage": {"ms": ms_prof, "bytes": int(buf.nbytes), "bytes_vs_band": buf.nbytes / ab.nbytes,
                                "kl_ku_bounds": [klp, kup],
                                "err_vs_x_true": float(np.abs(xp - x_true).max() / np.abs(x_true).max()),
                                "backward_error_sampled": float(np.abs(rp).max() / (np.abs(ab).sum(axis=1).max() *
                                                                                    np.abs(xp).max()))},
            "info": int(info.item())}
    print(json.dumps(line), flush=True)
    return line


# FP64 SIMT peak derived from the unit counts and the clock: 152 SMs x 2 DFMA
# per clock x 2 flops x 2.07 GHz (an FMA-chain probe reads 1.01 and under-reads:
# the inverse's products run at 1.21).
DFMA_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12


def run_inverse_config(args):
    """Explicit FP64 inverse from FP64 factors (product form, Eq. 4c), n = 8192
    (--inverse-n).
    Checked through properties that hold at any size: sampled rows of A X - I
    and X A - I (the oracle inverse itself is O(n^3) on the host)."""
    import torch

    import paper_1907_05767_gb300 as ebv
    import synthetic
    dev = torch.device("cuda")
    n = args.inverse_n
    a = synthetic.dense_dd(n, 0.9, synthetic.seed_for(2))
    A = torch.from_numpy(a).to(dev)
    lu = A.clone()
    info = ebv.ebv_factor(lu, "fp64")
    x = torch.empty_like(A)
    ws = torch.empty(ebv.lib().ebv_inverse_workspace_size(n, ebv.FP64), dtype=torch.uint8, device=dev)
    ms = _dev_ms(lambda: ebv.ebv_inverse(lu, x, "fp64", ws=ws), 3, 1, graph=False)
    launches0 = ebv.launch_count()
    ebv.ebv_inverse(lu, x, "fp64", ws=ws)
    torch.cuda.synchronize()
    launches = ebv.launch_count() - launches0
    rows = synthetic.pick_indices(13, 16, [n])[:, 0]
    xs = x.cpu().numpy()
    eye = np.eye(n)[rows]
    r_ax = float(np.abs(a[rows] @ xs - eye).max())
    r_xa = float(np.abs(xs[rows] @ a - eye).max())
    flops = 4.0 * n ** 3 / 3.0
    gf = flops / (ms / 1e3) / 1e9
    line = {"config": f"explicit inverse FP64 n={n} from FP64 factors (product form)", "ms": ms,
            "gflops_fp64": gf, "fp64_alu_frac": gf / 1e3 / DFMA_TFLOPS,
            "fp64_peak_tflops": DFMA_TFLOPS,
            "fp64_peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flops x 2.07 GHz", "launches": launches,
            "max_abs_AX_minus_I_sampled_rows": r_ax, "max_abs_XA_minus_I_sampled_rows": r_xa,
            "info": int(info.item())}
    print(json.dumps(line), flush=True)
    return line


# ----------------------------------------------------------------------------
# reference arm: the CPU oracle on a bounded sample of the same workload
# ----------------------------------------------------------------------------

def run_reference(args):
    import synthetic
    n = args.n
    a_np, _, _ = synthetic.config2(n, args.nrhs)
    kstop = args.ref_kstop
    rates = []
    for i in range(args.warmup + args.steps):
        rate, secs, used = cpu_oracle_rate(a_np, kstop)
        if i >= args.warmup:
            rates.append((rate, secs))
    rate = float(np.median([r for r, _ in rates]))
    ms = float(np.median([s for _, s in rates])) * 1e3
    sample = (f"oracle FP64 Doolittle on the first {kstop} elimination steps of the n={n} workload matrix "
              f"({cpu_model()})")
    return {"metric": METRIC, "value": rate, "unit": "GFLOP/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "fp64", "data": "synthetic (seeded)", "impl": "reference",
            "config": {"workload": workload_desc(n, args.nrhs), "n": n, "nrhs": args.nrhs},
            "cpu_baseline": {"value": rate, "unit": "GFLOP/s", "cores": used, "kind": "oracle", "sample": sample},
            "e2e": {"value": rate, "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ebv", choices=["ebv", "reference"])
    p.add_argument("--n", type=int, default=N_FULL)
    p.add_argument("--nrhs", type=int, default=NRHS_FULL)
    p.add_argument("--prec", default="bf16", choices=["bf16", "fp16"])
    p.add_argument("--max-iter", type=int, default=10)
    p.add_argument("--fp64-steps", type=int, default=1)
    p.add_argument("--e2e-steps", type=int, default=3)
    p.add_argument("--cpu-kstop", type=int, default=384)
    p.add_argument("--ref-kstop", type=int, default=96)
    p.add_argument("--no-graph", dest="graph", action="store_false")
    p.add_argument("--update-only", default=None, help="M,N,K: time the tensor-core update alone and exit")
    p.add_argument("--configs", nargs="?", const="all", default=None,
                   help="time the other workloads (one JSON line each) and exit; --configs inverse / profile / band_mixed / dense_sym: "
                        "one alone")
    p.add_argument("--inverse-n", type=int, default=8192, help="order of the explicit-inverse workload")
    p.add_argument("--band-grid", type=int, default=512, help="grid edge of the banded Laplacian workload")
    p.add_argument("--workload", default="dense", choices=["dense", "batched"],
                   help="batched: the 4096-system batch split across the ranks (one JSON line)")
    p.add_argument("--batched-prec", default="fp64", choices=["fp64", "fp32"])
    p.add_argument("--autotune", action="store_true", help="batched: tuned variant per size bucket")
    p.add_argument("--tune-cache", default=os.path.join(os.path.expanduser("~"), ".cache", "ebv_batch_autotune.json"),
                   help="JSON cache of the batched autotuner (keyed by GPU, precision and repetitions)")
    args = p.parse_args()
    if args.update_only:
        print(json.dumps(run_update_only(args)), flush=True)
        return
    if args.configs == "inverse":
        run_inverse_config(args)
        return
    if args.configs == "profile":
        run_profile_config(args)
        return
    if args.configs == "band_mixed":
        run_band_mixed_config(args)
        return
    if args.configs:
        run_configs(args)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        if rank != 0:
            return
        print(json.dumps(run_reference(args)), flush=True)
        return

    import paper_1907_05767_gb300 as ebv
    args.tc_used = ebv.tc_available() if hasattr(ebv, "tc_available") else False

    dist = None
    if world > 1:
        import torch.distributed as tdist
        tdist.init_process_group("nccl")
        dist = tdist
    line = run_batched(args, rank, world, dist) if args.workload == "batched" else run_gpu(args, rank, world, dist)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
