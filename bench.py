"""Benchmark of the KRR hot path on GB300: Build -> Factor -> Solve (+ refinement)
-> Predict on synthetic genotypes, one JSON line on stdout.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--config c3|c2|c1]
                    [--impl ours|reference] [--no-compare] [--no-e2e] [--no-cpu]

A step is one pass of the whole path on resident inputs; value = algorithmic
TOp/s of build + factor + solve (N(N+1)M + N^3/3 + 2N^2P) over the step time
(predict is inside the step but not counted).  Under torchrun (N > 1) every
rank runs an independent replica (the path has no data-path collective);
value = all ranks' operations / the slowest rank's time.

--impl reference times the CPU oracle (the method's plain FP64 definition) on
this machine's host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "KRR build+factor+solve TOp/s and s at N=131072: mixed vs FP32, rel err<=1e-4"
CONFIGS = {
    # name: (N, M, P, N_test, tile)
    "c1": (2048, 512, 1, 512, 256),
    "c2": (32768, 8192, 10, 4096, 1024),
    "c3": (131072, 16384, 20, 4096, 1024),
    # small case for ncu captures (about 1.5 GB on the device, K tiles > L2)
    "p1": (16384, 4096, 8, 1024, 1024),
    # FP8-dominant regime: the precision workload's shapes on structured cohorts
    "c2s": (32768, 8192, 10, 4096, 1024),
}
# structured cohorts (Balding-Nichols subpopulations) and gamma = gamma_m / M
STRUCTURED = {"c2s": {"populations": 8, "fst": 0.3, "gamma_m": 8.0}}
# batching workload: 64 problems = 16 cohorts x 4 lambdas, N ~ U[1024, 16384]
C4 = {"problems": 64, "cohorts": 16, "n_lo": 1024, "n_hi": 16384, "m": 4096, "p": 4, "n_test": 512,
      "lambdas": (1e-3, 1e-2, 1e-1, 1.0)}
LAMBDA = 0.1
SEED = 2409017120
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "update_kernel_traffic.txt")
TC_SRC = os.path.join(ROOT, "paper_2409_01712_gb300", "csrc", "tc_gemm.cu")


def metric_ops(n, m, p):
    return n * (n + 1) * m + n ** 3 / 3.0 + 2.0 * n * n * p


def workload_name(cfg):
    n, m, p, nt, b = CONFIGS[cfg]
    if cfg in STRUCTURED:
        st = STRUCTURED[cfg]
        return (f"{cfg}: N={n} M={m} P={p} N_test={nt} tile={b} gamma={st['gamma_m']:g}/M lambda={LAMBDA}, "
                f"{st['populations']} Balding-Nichols cohorts F={st['fst']} around p_j~U(0.05,0.5), "
                f"phenotypes 20 SNP-pair products + N(0,0.5)")
    return (f"{cfg}: N={n} M={m} P={p} N_test={nt} tile={b} gamma=1/M lambda={LAMBDA}, "
            f"genotypes Binomial(2,p_j) p_j~U(0.05,0.5), phenotypes 20 SNP-pair products + N(0,0.5)")


def gamma_of(cfg):
    m = CONFIGS[cfg][1]
    return STRUCTURED[cfg]["gamma_m"] / m if cfg in STRUCTURED else 1.0 / m


def make_problem(cfg, n, m, p, n_test, seed, device="cpu"):
    from paper_2409_01712_gb300 import inputs

    if cfg in STRUCTURED:
        st = STRUCTURED[cfg]
        return inputs.structured_problem(n, m, p, n_test, seed=seed, populations=st["populations"], fst=st["fst"],
                                         device=device)
    return inputs.problem(n, m, p, n_test, seed=seed, device=device)


PREC_CHARS = {0: "D", 1: "S", 2: "h", 3: "8", 255: " "}
PREC_LEGEND = "D FP64, S FP32 (diagonal tiles: their factorisation precision), h FP16, 8 E4M3; row i = tiles (i, 0..i)"


def heatmap_rows(pmap):
    """The precision mosaic as text rows: D = FP64, S = FP32 (FP32 class),
    h = FP16, 8 = E4M3 (row i lists tiles (i, 0..i))."""
    return ["".join(PREC_CHARS.get(int(v), "?") for v in pmap[i, : i + 1]) for i in range(pmap.shape[0])]


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def update_traffic():
    """DRAM bytes per algorithmic flop of the trailing-update kernel from the
    committed ncu summary (key = value lines), if it was taken on the current
    tensor-core source; else None."""
    try:
        rec = {}
        with open(TRAFFIC_FILE) as f:
            for line in f:
                if "=" in line and not line.lstrip().startswith("#"):
                    k, v = line.split("=", 1)
                    rec[k.strip()] = v.strip()
        with open(TC_SRC, "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
        if rec.get("tc_gemm_sha256") != sha:
            return None
        return float(rec["dram_bytes_per_flop"])
    except (OSError, ValueError, KeyError):
        return None


class ClockSampler:
    """nvidia-smi samples (200 ms) while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
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
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def slowest_ms(ms, dist=None, device=None):
    """The job's time per step: the largest of the ranks' times (replicas run
    independently; the job ends with the slowest)."""
    if dist is None:
        return ms
    import torch

    tt = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(tt, op=dist.ReduceOp.MAX)
    return float(tt.item())


def job_value(world, ops_per_rank, ms):
    """Whole-job TOp/s: every rank's operations over the slowest rank's time."""
    return world * ops_per_rank / (ms / 1e3) / 1e12


def cpu_sample(cfg, n_sample, g_host=None, y_host=None):
    """Times the oracle's build + factor + solve on the first n_sample rows."""
    import oracle
    from paper_2409_01712_gb300 import inputs

    n, m, p, _, _ = CONFIGS[cfg]
    if g_host is None:
        prob = make_problem(cfg, n_sample, m, p, 1, seed=SEED)
        g_host, y_host = prob["G"].numpy(), prob["Y"].numpy()
    g = np.ascontiguousarray(g_host[:n_sample])
    y = np.ascontiguousarray(y_host[:n_sample]).astype(np.float64)
    t0 = time.perf_counter()
    k = oracle.build_kernel(gamma_of(cfg), g)
    t1 = time.perf_counter()
    oracle.associate(LAMBDA, k, y)
    dt = time.perf_counter() - t0
    ops = metric_ops(n_sample, m, p)
    # the plain loops scale as N^2 M (distances) and N^3 (factorisation)
    scale = n / n_sample
    extrap = (t1 - t0) * scale ** 2 + (dt - (t1 - t0)) * scale ** 3
    return {"value": ops / dt / 1e12, "unit": "TOp/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"first {n_sample} rows of the {cfg} workload (M={m}, P={p}): brute-force "
                      f"distances, FP64 Cholesky, substitution; {dt:.2f} s",
            "seconds": dt, "build_s": t1 - t0, "associate_s": dt - (t1 - t0),
            "extrapolated_full_s": extrap,
            "extrapolation": f"labelled extrapolation to N={n}: build x (N/{n_sample})^2, associate x (N/{n_sample})^3"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    cfg = args.config if args.config in CONFIGS else "c3"
    n_sample = args.ref_rows
    times = []
    res = None
    for i in range(args.warmup + args.steps):
        res = cpu_sample(cfg, n_sample)
        if i >= args.warmup:
            times.append(res["seconds"])
    n, m, p, _, _ = CONFIGS[cfg]
    ops = metric_ops(n_sample, m, p)
    t = float(np.mean(times))
    value = ops / t / 1e12
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "TOp/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": workload_name(cfg), "sample_rows": n_sample},
            "cpu_baseline": {"value": value, "unit": "TOp/s", "cores": res["cores"], "kind": "oracle",
                             "sample": res["sample"], "extrapolated_full_s": res["extrapolated_full_s"],
                             "extrapolation": res["extrapolation"]},
            "e2e": {"value": value, "unit": "TOp/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def subproblem_accuracy(args, g, y, t, gamma, tile, stream):
    """The first sub_rows rows of the workload (same held-out rows) through the
    same mixed path, against the full FP64 oracle solution of that
    subproblem (float64 library Gram products and factorisation)."""
    import oracle
    from paper_2409_01712_gb300 import KRR

    ns = args.sub_rows
    gs, ys = g[:ns].contiguous(), y[:ns].contiguous()
    with KRR(tile=tile, mode=args.mode, stream=stream.cuda_stream) as sub:
        sub.build_kernel(gs, gamma)
        fi = sub.factor(LAMBDA)
        a_s, si = sub.solve(ys)
        yt_s = sub.predict(t, a_s)
    g_h, y_h, t_h = gs.cpu().numpy(), ys.double().cpu().numpy(), t.cpu().numpy()
    a_h, yt_h = a_s.double().cpu().numpy(), yt_s.double().cpu().numpy()
    t0 = time.perf_counter()
    k_ref, a_ref, yt_ref = oracle.krr(gamma, LAMBDA, g_h, y_h, t_h, method="lapack")
    osec = time.perf_counter() - t0
    res = y_h - LAMBDA * a_h - k_ref @ a_h
    return {"rows": ns, "held_out_rows": int(t.shape[0]),
            "rel_err_yt": float(np.linalg.norm(yt_h - yt_ref) / np.linalg.norm(yt_ref)),
            "rel_err_a": float(np.linalg.norm(a_h - a_ref) / np.linalg.norm(a_ref)),
            "rel_residual_fp64": float(np.linalg.norm(res) / np.linalg.norm(y_h)),
            "rel_residual_device": si["rel_residual"], "iterations": si["iterations"],
            "tiles_fp32_fp16_e4m3": [fi["tiles_fp32"], fi["tiles_fp16"], fi["tiles_e4m3"]],
            "oracle": "FP64, float64 library Gram product + LAPACK Cholesky / triangular solves",
            "oracle_s": osec}


def run_ours(args):
    import torch

    from paper_2409_01712_gb300 import KRR, inputs

    world, rank, local = dist_env()
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    cfg = args.config
    n, m, p, n_test, tile = CONFIGS[cfg]
    gamma = gamma_of(cfg)

    prob = make_problem(cfg, n, m, p, n_test, seed=SEED + rank, device=dev)
    g, y, t = prob["G"], prob["Y"], prob["T"]
    torch.cuda.synchronize()
    a_out = torch.empty((n, p), dtype=torch.float32, device=dev)
    yt_out = torch.empty((n_test, p), dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    model = KRR(tile=tile, mode=args.mode, stream=stream.cuda_stream, prec_rule=args.prec_rule, eps=args.eps)

    def step():
        model.build_kernel(g, gamma)
        fi = model.factor(LAMBDA)
        _, si = model.solve(y, out=a_out)
        model.predict(t, a_out, out=yt_out)
        return fi, si

    for _ in range(args.warmup):
        fi, si = step()
    torch.cuda.synchronize()
    model.set_profiling(True)
    model.profile(reset=True)
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    infos = []
    for _ in range(args.steps):
        infos.append(step())
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1) / args.steps
    prof = model.profile(reset=True)
    model.set_profiling(False)
    ms = slowest_ms(ms, dist, dev)
    ops = metric_ops(n, m, p)
    value = job_value(world, ops, ms)
    fi, si = infos[-1]

    pk, pk_kind = peaks()
    # every launch of the trailing-update kernel: those with the whole GPU
    # and those beside the next column's diagonal step (lookahead)
    full, shared = prof["update"], prof.get("update_shared", {"count": 0, "ms": 0.0, "flops": 0.0})
    upd = {k: full[k] + shared[k] for k in ("count", "ms", "flops")}
    roof = None
    if upd["count"] > 0 and upd["ms"] > 0:
        ach = upd["flops"] / (upd["ms"] / 1e3) / 1e12
        peak = float(pk.get("bf16_tflops_sustained", pk.get("bf16_tflops")))
        bpf = update_traffic() if args.mode == "mixed" else None
        # the capture is of a small case: scale its bytes per flop to the
        # average launch here (operand and C traffic grow with the tiles)
        traffic = bpf * upd["flops"] / upd["count"] if bpf else None
        roof = {"bound": "tensor", "kernel": "tc_kernel<F16, OP_UPDATE> (trailing update)",
                "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "peak_source": f"{pk_kind}: bf16 dense sustained (FP16 dense runs at the same rate)",
                "traffic": traffic, "launches": upd["count"],
                "avg_launch_ms": upd["ms"] / upd["count"]}
        if shared["count"] > 0 and full["ms"] > 0:
            ach_full = full["flops"] / (full["ms"] / 1e3) / 1e12
            roof["lookahead"] = {
                "note": "lookahead launches: the diagonal target alone, then targets beside the next column's "
                        "diagonal step on the SMs it leaves free; full_gpu = the other update launches",
                "shared_launches": shared["count"], "shared_ms_per_step": shared["ms"] / args.steps,
                "shared_tflops": shared["flops"] / (shared["ms"] / 1e3) / 1e12 if shared["ms"] > 0 else None,
                "full_gpu_launches": full["count"], "full_gpu_tflops": ach_full, "full_gpu_frac": ach_full / peak}
    bld = prof["build"]
    if bld["count"] > 0 and bld["ms"] > 0 and args.mode == "mixed":
        # the distance GEMM on E4M3 operands: its peak is the measured BF16
        # rate times the nominal E4M3 : BF16 ratio (2)
        ach = bld["flops"] / (bld["ms"] / 1e3) / 1e12
        peak8 = 2.0 * float(pk.get("bf16_tflops_sustained", pk.get("bf16_tflops")))
        line_build_roof = {"bound": "tensor", "kernel": "tc_kernel<F8, OP_DIST> (distance GEMM + exp epilogue)",
                           "achieved": ach, "peak": peak8, "unit": "TFLOP/s", "frac": ach / peak8,
                           "peak_source": f"{pk_kind}: bf16 dense sustained x 2 (nominal E4M3 : BF16 ratio)",
                           "launches": bld["count"], "avg_launch_ms": bld["ms"] / bld["count"]}
    else:
        line_build_roof = None
    phases = {k: {"ms_per_step": v["ms"] / args.steps, "count_per_step": v["count"] / args.steps}
              for k, v in prof.items() if isinstance(v, dict) and v["count"] > 0}
    for k, v in prof.items():
        if isinstance(v, dict) and v["count"] > 0 and v["ms"] > 0:
            if v["flops"] > 0:
                phases[k]["tflops"] = v["flops"] / (v["ms"] / 1e3) / 1e12
            if v["bytes"] > 0:
                phases[k]["gbs"] = v["bytes"] / (v["ms"] / 1e3) / 1e9
    line = {"metric": METRIC, "value": value, "unit": "TOp/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": "e4m3+f16 tensor, f32/f64 refine" if args.mode == "mixed" else "f32",
            "data": "synthetic",
            "config": {"workload": workload_name(cfg), "mode": args.mode,
                       "l2": "inputs larger than L2 (K tiles alone are "
                             f"{(n // tile) * (n // tile + 1) // 2 * tile * tile * 4 / 1e9:.1f} GB)",
                       "parallelism": f"replicas x{world}"},
            "gpu_launches": int(prof["launches"]),
            "clocks": clk,
            "phases": phases,
            "phases_note": "CUDA-event time per class; diagonal steps of the lookahead run on a second stream "
                           "at the same time as update_shared, so the classes add up to more than the step",
            "factor": {k: fi[k] for k in ("tiles_fp32", "tiles_fp16", "tiles_e4m3", "factor_bytes",
                                          "min_pivot")},
            "precision_map": ({"legend": PREC_LEGEND,
                               "rows": heatmap_rows(model.precision_map())} if fi["nt"] <= 32 else
                              {"note": f"{fi['nt']} x {fi['nt']} tiles: counts under factor"}),
            "solve": {"iterations": si["iterations"], "rel_residual": si["rel_residual"],
                      "converged": si["converged"], "history": si["history"]}}
    if roof:
        line["roofline"] = roof
    if line_build_roof:
        line["roofline_build"] = line_build_roof

    # ---- e2e: the same step through host buffers (pinned), copies inside the timing
    if not args.no_e2e:
        gh = g.cpu().pin_memory()
        yh = y.cpu().pin_memory()
        th = t.cpu().pin_memory()
        ah = torch.empty((n, p), dtype=torch.float32).pin_memory()
        yth = torch.empty((n_test, p), dtype=torch.float32).pin_memory()

        def step_host():
            model.build_kernel(gh, gamma)
            model.factor(LAMBDA)
            model.solve(yh, out=ah)
            model.predict(th, ah, out=yth)

        step_host()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        w0 = time.perf_counter()
        e0.record(stream)
        for _ in range(args.steps):
            step_host()
        e1.record(stream)
        torch.cuda.synchronize()
        wall = (time.perf_counter() - w0) / args.steps
        ems = max(e0.elapsed_time(e1) / args.steps, wall * 1e3)
        ems = slowest_ms(ems, dist, dev)
        h2d = n * m + n * p * 4 + n_test * m + n * p * 4
        d2h = n * p * 4 + n_test * p * 4
        line["e2e"] = {"value": job_value(world, ops, ems), "unit": "TOp/s", "ms_per_step": ems,
                       "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # ---- sampled accuracy check against the oracle (outside the timing)
    if not args.no_cpu and rank == 0:
        import oracle

        a_host = a_out.double().cpu().numpy()
        rows = np.random.default_rng(7).choice(n, size=args.check_rows, replace=False)
        gh_np = g.cpu().numpy()
        krows = oracle.kernel_rows(gamma, gh_np, rows, gh_np)
        yh_np = y.double().cpu().numpy()
        r = yh_np[rows] - (krows @ a_host + LAMBDA * a_host[rows])
        line["accuracy"] = {"sampled_rows": int(args.check_rows),
                            "rel_residual_fp64_oracle_rows": float(np.linalg.norm(r) / np.linalg.norm(yh_np[rows])),
                            "rel_residual_device": si["rel_residual"]}
        if args.sub_rows > 0 and args.sub_rows < n:
            line["accuracy"]["subproblem"] = subproblem_accuracy(args, g, y, t, gamma, tile, stream)

    # ---- plain FP32 comparator: the same engine with every step in FP32 on CUDA cores
    if not args.no_compare and args.mode == "mixed":
        model.close()
        del model
        torch.cuda.empty_cache()
        cmp_model = KRR(tile=tile, mode="fp32", stream=stream.cuda_stream)

        def step32():
            cmp_model.build_kernel(g, gamma)
            cmp_model.factor(LAMBDA)
            cmp_model.solve(y, out=a_out)
            cmp_model.predict(t, a_out, out=yt_out)

        # one untimed step allocates the FP32 tiles and sets up the kernels,
        # then the timed steps (the mixed arm's own warm-up runs before its timing)
        for _ in range(args.fp32_warmup):
            step32()
        torch.cuda.synchronize()
        c0 = torch.cuda.Event(enable_timing=True)
        c1 = torch.cuda.Event(enable_timing=True)
        c0.record(stream)
        for _ in range(args.fp32_steps):
            step32()
        c1.record(stream)
        torch.cuda.synchronize()
        cms = c0.elapsed_time(c1) / args.fp32_steps
        line["fp32_comparator"] = {"ms_per_step": cms, "value": ops / (cms / 1e3) / 1e12, "unit": "TOp/s",
                                   "steps": args.fp32_steps, "warmup": args.fp32_warmup,
                                   "speedup_mixed_over_fp32": cms / ms}
        cmp_model.close()

    # ---- CPU baseline: the oracle on this host's cores, bounded sample
    if not args.no_cpu and rank == 0:
        res = cpu_sample(cfg, args.cpu_rows, g.cpu().numpy(), y.cpu().numpy())
        for key in ("seconds", "build_s", "associate_s"):
            res.pop(key)
        line["cpu_baseline"] = res

    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """C4: 64 KRR problems (16 cohorts x 4 lambdas, ragged N) as one captured
    CUDA graph, against the same 64 problems solved one after another."""
    import torch

    from paper_2409_01712_gb300 import KRR, KRRBatch, inputs

    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(SEED + 4)
    ns = [int(x) for x in rng.integers(C4["n_lo"], C4["n_hi"] + 1, size=C4["cohorts"])]
    m, p = C4["m"], C4["p"]
    problems = []
    for ci, n in enumerate(ns):
        prob = inputs.problem(n, m, p, C4["n_test"], seed=SEED + 100 + ci, device=dev)
        for lam in C4["lambdas"]:
            problems.append({"G": prob["G"], "Y": prob["Y"], "T": prob["T"], "gamma": 1.0 / m, "lam": lam})
    ops = sum(metric_ops(pr["G"].shape[0], m, p) for pr in problems)
    t0 = time.perf_counter()
    bt = KRRBatch(problems, ir_iters=3, autotune=2)
    setup_s = time.perf_counter() - t0
    for _ in range(args.warmup):
        bt.run()
    torch.cuda.synchronize()
    times = []
    for _ in range(args.steps):
        t1 = time.perf_counter()
        res = bt.run()
        times.append(time.perf_counter() - t1)
    ms = float(np.median(times)) * 1e3
    tiles = sorted({r["tile"] for r in res})
    bad = [i for i, r in enumerate(res) if r["status"] != 0 or not (r["rel_residual"] > 0.0)]
    worst_res = max((r["rel_residual"] for r in res), key=lambda v: (v != v, v))  # NaN counts as worst
    bt.close()
    # the same problems one after another, eagerly (refinement with host
    # checks), each on a context of its own made and warmed up before the
    # timing: in plain FP32 (the comparison path) and in mixed precision
    def sequential(mode):
        models = [KRR(tile=1024, mode=mode) for _ in problems]

        def one_pass():
            for model, pr in zip(models, problems):
                model.build_kernel(pr["G"], pr["gamma"])
                model.factor(pr["lam"])
                a, _ = model.solve(pr["Y"], raise_on_noconv=False)
                model.predict(pr["T"], a)

        one_pass()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        one_pass()
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t1) * 1e3
        for model in models:
            model.close()
        torch.cuda.empty_cache()
        return dt

    seq_ms = sequential("mixed") if not args.no_compare else None
    seq32_ms = sequential("fp32") if not args.no_compare else None
    line = {"metric": "batched KRR: 64 CV problems (16 cohorts x 4 lambdas, N~U[1024,16384]) TOp/s",
            "value": ops / (ms / 1e3) / 1e12, "unit": "TOp/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "e4m3+f16 tensor, f32/f64 refine", "data": "synthetic",
            "config": {"workload": f"c4: 64 problems, cohort N = {ns}, M={m}, P={p}, N_test={C4['n_test']}, "
                                   f"lambda in {C4['lambdas']}, gamma=1/M", "graph": "one CUDA graph per run"},
            "batch": {"tiles_chosen": tiles, "setup_s": setup_s,
                      "autotune": "per-size trial runs, then the whole batch timed for that choice and every uniform "
                                  "tile edge (256 / 512 / 1024); the fastest kept", "worst_rel_residual": worst_res,
                      "problems_failed_or_zero_residual": bad, "residuals": [r["rel_residual"] for r in res],
                      "shared_builds": "the 4 lambdas of a cohort share one Build",
                      "sequential_fp32_ms": seq32_ms,
                      "speedup_over_sequential_fp32": seq32_ms / ms if seq32_ms else None,
                      "sequential_mixed_ms": seq_ms,
                      "speedup_over_sequential_mixed": seq_ms / ms if seq_ms else None}}
    print(json.dumps(line), flush=True)
    return 0


def run_peaks(args):
    """Dense tensor-core peaks of this GPU for the dtypes the path uses, by
    library GEMMs (cuBLAS / cuBLASLt through torch) timed with CUDA events:
    FP16 (torch.matmul) and E4M3 with FP32 accumulation (torch._scaled_mm),
    n x n x n with n = 8192; burst = best of 10 single products, sustained =
    back-to-back products for about 4 s; SM clocks sampled meanwhile."""
    import torch

    dev = torch.device("cuda", 0)
    n = 8192
    flops = 2.0 * n ** 3
    a16 = torch.randn((n, n), device=dev, dtype=torch.float16)
    b16 = torch.randn((n, n), device=dev, dtype=torch.float16)
    a8 = a16.to(torch.float8_e4m3fn)
    b8 = b16.t().contiguous().to(torch.float8_e4m3fn).t()  # column-major second operand
    one = torch.ones((), device=dev, dtype=torch.float32)
    cases = {"fp16": lambda: torch.matmul(a16, b16),
             "e4m3": lambda: torch._scaled_mm(a8, b8, scale_a=one, scale_b=one, out_dtype=torch.bfloat16)}
    out = {"metric": "dense tensor-core peaks (library GEMM, n=8192)", "n": n, "unit": "TFLOP/s"}
    clocks = ClockSampler(0)
    clocks.start()
    for name, fn in cases.items():
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        best = 0.0
        for _ in range(10):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            best = max(best, flops / (e0.elapsed_time(e1) / 1e3) / 1e12)
        reps, t_total = 0, 0.0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        w0 = time.perf_counter()
        while time.perf_counter() - w0 < 4.0:
            for _ in range(20):
                fn()
            reps += 20
            torch.cuda.synchronize()
        e1.record()
        torch.cuda.synchronize()
        t_total = e0.elapsed_time(e1) / 1e3
        out[name] = {"burst": best, "sustained": flops * reps / t_total / 1e12, "reps": reps}
    out["clocks"] = clocks.stop()
    print(json.dumps(out), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--config", default="c3", choices=sorted(CONFIGS) + ["c4"])
    ap.add_argument("--prec-rule", default="lambda", choices=["lambda", "knorm"])
    ap.add_argument("--eps", type=float, default=None, help="threshold of the precision rule")
    ap.add_argument("--mode", default="mixed", choices=["mixed", "fp32"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-compare", action="store_true", help="skip the plain-FP32 comparator step")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle baseline and sampled check")
    ap.add_argument("--cpu-rows", type=int, default=4096, help="rows of the oracle sample (cpu_baseline)")
    ap.add_argument("--ref-rows", type=int, default=2048, help="rows of each --impl reference step")
    ap.add_argument("--sub-rows", type=int, default=16384,
                    help="rows of the subproblem compared with the full FP64 oracle (0: skip)")
    ap.add_argument("--fp32-warmup", type=int, default=1)
    ap.add_argument("--fp32-steps", type=int, default=2)
    ap.add_argument("--check-rows", type=int, default=32, help="rows of the sampled oracle residual")
    ap.add_argument("--peaks", action="store_true", help="measure the dense FP16 / E4M3 library GEMM peaks")
    args = ap.parse_args()
    if args.peaks:
        return run_peaks(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.config == "c4":
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
