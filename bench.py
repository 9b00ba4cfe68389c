"""Benchmark of the Spectral Ewald Stokes hot path on GB300.

Workload (N = 1): the triply periodic stresslet and rotlet potentials of N = 20,000 points
uniform in the unit box (strengths N(0,1), stresslet normals normalised), FP32 path,
parameters from the selection procedure of Sec. 4.6 at 1e-6 RMS relative tolerance (PKB
window), targets = sources. One step = one full evaluation of both kernels (real-space sum,
Fourier-space part of Alg. 1, corrections). value = targets per second of the FP32 batched
form (both evaluations replayed as one CUDA graph through se_batch_launch), counting each
(kernel, target) evaluation; the eager form (one se_eval per kernel, with per-kernel events
for the stage times and the roofline), the FP64 plain form and the end-to-end form through
host buffers are reported beside it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank runs the same workload on its own GPU (replicas, weak
scaling, no collective in the data path); value = all ranks' targets / the slowest rank's time.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "3p_stresslet_rotlet_n20000"   # default (--workload selects another configuration)
METRIC_FMT = "targets/sec at 1e-6 RMS rel error (FP32 batched vs FP64 plain), %s"
METRIC = METRIC_FMT % "3P stresslet+rotlet, N=20000"
METRIC_NAMES = {"3p_stresslet_rotlet_n20000": "3P stresslet+rotlet, N=20000",
                "2p_stokeslet_n200000_rhs8": "2P stokeslet, N=200000, 8 RHS"}
UNIT = "targets/s"
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # SMs x FP32 lanes x 2 flop x max clock


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {"hbm_gbs": 6800.0, "fallback": True}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
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
                "sm_max_mhz": float(max(smax)) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(ms, dist, device):
    """The slowest rank's time (each rank times its own replica; the job ends with the last)."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(targets_per_step, world, steps, ms_max):
    """Whole-job throughput of `world` replicas (weak scaling): every rank's targets over the
    slowest rank's time."""
    return targets_per_step * world * steps / (ms_max / 1e3)


def make_inputs():
    """Positions (N, 3) and per-kernel strengths (n_rhs, N, c) of the selected workload."""
    from paper_2210_01255_gb300 import workloads as W
    cfg = W.CONFIGS[WORKLOAD]
    N, R = cfg["N"], cfg.get("n_rhs", 1)
    x = W.uniform_points(N, cfg["box"], seed=cfg["seed"])
    fs = {}
    for k in cfg["kernels"]:
        f = W.strengths(k, N, seed=cfg["seed"] + (0 if k == "stresslet" else 100), n_rhs=R if R > 1 else None)
        fs[k] = np.ascontiguousarray(f.reshape(R, N, -1).astype(np.float32))
    return cfg, x, fs


def tuned(cfg, kernel, f):
    import paper_2210_01255_gb300 as se
    from paper_2210_01255_gb300 import workloads as W
    # the selection targets E <= 10 tau (Sec. 4.6); ask for tol/10 so the result meets tol
    Q = W.source_quantity(kernel, f[0])
    o = se.se_opts_default()
    o.n_rc = cfg.get("n_rc", {}).get(kernel, 0.0)
    o.P_margin = cfg.get("P_margin", -1)
    return se.se_autotune(cfg["D"], cfg["box"], se.KERNELS[kernel], Q, cfg["N"], cfg["tol"] / 10.0, opts=o)


KERNEL_SOURCES = {"real": "se_core.cu", "spread": "se_core.cu", "gather": "se_core.cu"}


def kernel_traffic(stage, params, gridding="cuda"):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of the stage's kernel
    from the committed ncu summary profiles/traffic_3p_stresslet_rotlet_n20000.txt, averaged over
    the stresslet and rotlet launches; None when the summary is missing, was taken for other
    parameters, or the kernel's source file changed since (sha256 recorded with the counters)."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "traffic_3p_stresslet_rotlet_n20000.txt")
    try:
        lines = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    except OSError:
        return None
    if stage == "spread" and gridding == "tc":
        return None  # the summary covers the CUDA-core gridding kernel only
    src = os.path.join(ROOT, "paper_2210_01255_gb300", "csrc", KERNEL_SOURCES[stage])
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    vals = []
    for f in lines:
        # stage kernel M P bytes_per_launch source_sha
        if len(f) == 6 and f[0] == stage and f[5] == sha:
            for k, p in params.items():
                if f[1] == k and int(f[2]) == p["M"][0] and int(f[3]) == p["P"]:
                    vals.append(float(f[4]))
    return sum(vals) / len(vals) if len(vals) == len(params) else None


def oracle_sample(cfg, x, fs, nsample, seed=7):
    """The exact Ewald oracle (FP64, all host cores) at a bounded sample of targets."""
    from oracle import ewald as E
    idx = np.random.default_rng(seed).choice(cfg["N"], nsample, replace=False)
    out, t0 = {}, time.perf_counter()
    for k in cfg["kernels"]:
        out[k] = E.potential(cfg["D"], list(cfg["box"]), k, x, fs[k][0].astype(np.float64), targets=x[idx])
    return idx, out, time.perf_counter() - t0


def run_reference(args):
    """Reference arm: the oracle as it stands, timed on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cfg, x, fs = make_inputs()
    ns = 512 if cfg["N"] <= 50000 else 32  # targets per step: ~1-2 s of oracle work
    for _ in range(args.warmup):
        oracle_sample(cfg, x, fs, ns, seed=11)
    tot = 0.0
    for s in range(args.steps):
        _, _, dt = oracle_sample(cfg, x, fs, ns, seed=100 + s)
        tot += dt
    targets = ns * len(cfg["kernels"]) * args.steps
    value = targets / tot
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": cfg["N"], "box": list(cfg["box"]),
                       "kernels": list(cfg["kernels"]), "tol_rel": cfg["tol"], "parallelism": "single"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d sampled targets x %d kernels per step, all N sources" %
                                       (ns, len(cfg["kernels"]))},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    global WORKLOAD, METRIC
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(METRIC_NAMES),
                    help="configuration from paper_2210_01255_gb300.workloads.CONFIGS")
    ap.add_argument("--gridding", choices=["cuda", "tc"], default="cuda",
                    help="FP32 gridding on the CUDA cores (default) or the tensor cores (tcgen05)")
    args = ap.parse_args()
    WORKLOAD = args.workload
    METRIC = METRIC_FMT % METRIC_NAMES[WORKLOAD]
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2210_01255_gb300 as se

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    cfg, x, fs = make_inputs()
    N, R = cfg["N"], cfg.get("n_rhs", 1)
    stream = torch.cuda.current_stream()
    plans, fdev, params = {}, {}, {}
    for k in cfg["kernels"]:
        t = tuned(cfg, k, fs[k])
        params[k] = dict(xi=t["xi"], rc=t["rc"], M=t["M"], P=t["P"])
        o = se.se_opts_default()
        o.flags = se.FLAG_TC_GRIDDING if args.gridding == "tc" else 0
        plans[k] = se.Plan(cfg["D"], cfg["box"], t["xi"], t["rc"], t["M"], t["P"], cfg["window"], "fp32",
                           opts=o, stream=stream)
        fdev[k] = torch.tensor(fs[k], device=dev)
    grid_n = {k: list(plans[k].info().n) for k in cfg["kernels"]}
    xdev = torch.tensor(x, device=dev)
    udev = {k: torch.empty((R, N, 3), dtype=torch.float32, device=dev) for k in cfg["kernels"]}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2

    def step():
        for k in cfg["kernels"]:
            plans[k].evaluate(k, xdev, fdev[k], out=udev[k])

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()

    # ---- timed region: K steps, L2 flushed between steps (outside the events)
    for p in plans.values():
        se.se_set_timing(p.handle, True)
    stage_ms = {k: np.zeros(8) for k in cfg["kernels"]}
    launches = 0
    sampler = ClockSampler(local)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for s in range(args.steps):
        flush.zero_()
        ev[s][0].record(stream)
        step()
        ev[s][1].record(stream)
        for k in cfg["kernels"]:
            info = plans[k].info()       # waits for this step's stage events
            stage_ms[k] += np.array(list(info.times_ms))
            launches += info.launches
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    targets_per_step = N * R * len(cfg["kernels"])  # (target, RHS) evaluations per step
    # FP32 batched: both evaluations of a step captured into one CUDA graph (se_batch_*) on a
    # stream of their own and replayed; L2 flushed between replays, timed with events
    graph = None
    gstream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(gstream):
        gplans, gu = {}, {}
        for k in cfg["kernels"]:
            t = params[k]
            o = se.se_opts_default()
            o.flags = se.FLAG_TC_GRIDDING if args.gridding == "tc" else 0
            gplans[k] = se.Plan(cfg["D"], cfg["box"], t["xi"], t["rc"], t["M"], t["P"], cfg["window"], "fp32",
                                opts=o, stream=gstream)
            gu[k] = torch.empty((R, N, 3), dtype=torch.float32, device=dev)
        ks = list(cfg["kernels"])
        bh = se.se_batch_create([gplans[k].handle for k in ks], [se.KERNELS[k] for k in ks], [xdev] * len(ks),
                                [fdev[k] for k in ks], [R] * len(ks), [gu[k] for k in ks])
        for _ in range(max(3, args.warmup)):
            se.se_batch_launch(bh)
        gstream.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        evg = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for s_ in range(args.steps):
            flush.zero_()
            evg[s_][0].record(gstream)
            se.se_batch_launch(bh)
            evg[s_][1].record(gstream)
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        tg = sum(a.elapsed_time(b) for a, b in evg)
        gerr = max(float((gu[k] - udev[k]).abs().max() / udev[k].abs().max()) for k in ks)
        se.se_batch_destroy(bh)
    graph = {"value": targets_per_step * args.steps / (tg / 1e3), "unit": UNIT, "ms_per_step": tg / args.steps,
             "form": "FP32 batched: the step's evaluations replayed as one CUDA graph (se_batch_launch); "
                     "the headline value",
             "max_rel_diff_vs_eager": gerr}

    clocks = sampler.stop()
    for p in plans.values():
        se.se_set_timing(p.handle, False)
    tot_ms = max_over_ranks(sum(a.elapsed_time(b) for a, b in ev), dist, dev)
    value = replica_value(targets_per_step, world, args.steps, tot_ms)

    # ---- dominant kernel and its roofline
    names = ["bin", "spread", "fft", "scale", "ifft", "gather", "real", "corr"]
    per_stage = {n: sum(stage_ms[k][i] for k in cfg["kernels"]) / args.steps for i, n in enumerate(names)}
    work, hbm = {}, {}
    for k in cfg["kernels"]:
        P = params[k]["P"]
        C = (6 if k == "stresslet" else 3) * R
        G = float(np.prod(grid_n[k]))
        H = float(grid_n[k][0] * grid_n[k][1] * (grid_n[k][2] // 2 + 1))
        work.setdefault("spread", 0.0)
        work["spread"] += 2.0 * N * P ** 3 * C        # one FMA per tap per component
        work.setdefault("gather", 0.0)
        work["gather"] += 2.0 * N * P ** 3 * 3 * R
        # algorithmic HBM bytes: spread N (24 + 4 C) + 4 G C; gather 4 G 3R + 12 N R;
        # k-space multiply (3P) (C + 3R) x 8 B per half-spectrum mode
        hbm["spread"] = hbm.get("spread", 0.0) + N * (24 + 4 * C) + 4 * G * C
        hbm["gather"] = hbm.get("gather", 0.0) + 4 * G * 3 * R + 12 * N * R
        if cfg["D"] == 3:
            hbm["scale"] = hbm.get("scale", 0.0) + (C + 3 * R) * 8 * H
    # real space: pairs within rc for the uniform density of this workload, 60 flops per pair
    vol = float(np.prod(cfg["box"]))
    work["real"] = sum(60.0 * N * (N - 1) / vol * 4.0 / 3.0 * math.pi * params[k]["rc"] ** 3
                       for k in cfg["kernels"])
    # the dominant kernel among those with a per-launch algorithmic work figure
    dom = max(work, key=lambda n: per_stage[n])
    ach = work[dom] / (per_stage[dom] * 1e-3) / 1e12
    roof = {"bound": "alu", "kernel": dom, "achieved": ach, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": ach / FP32_PEAK_TFLOPS, "traffic": kernel_traffic(dom, params, args.gridding),
            "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz (derived from unit counts and "
                           "the maximum SM clock)"}
    roof["per_stage_tflops"] = {k: work[k] / (per_stage[k] * 1e-3) / 1e12 for k in work if per_stage[k] > 0}
    pk = peaks()
    roof["per_stage_hbm"] = {k: {"algorithmic_bytes": hbm[k], "achieved_gbs": hbm[k] / (per_stage[k] * 1e-3) / 1e9,
                                 "frac_of_measured_peak": hbm[k] / (per_stage[k] * 1e-3) / 1e9 / pk["hbm_gbs"]}
                             for k in hbm if per_stage[k] > 0}

    # ---- end to end through the C ABI with host buffers (copies inside the timed region)
    e2e = None
    if rank == 0 or True:
        xh = np.ascontiguousarray(x)
        uh = {k: np.empty((R, N, 3), dtype=np.float32) for k in cfg["kernels"]}
        fh = {k: np.ascontiguousarray(fs[k]) for k in cfg["kernels"]}
        for _ in range(2):
            for k in cfg["kernels"]:
                se.se_eval_host(plans[k].handle, se.KERNELS[k], xh, fh[k], R, None, uh[k])
        t0 = time.perf_counter()
        for _ in range(args.steps):
            for k in cfg["kernels"]:
                se.se_eval_host(plans[k].handle, se.KERNELS[k], xh, fh[k], R, None, uh[k])
        dt = time.perf_counter() - t0
        h2d = sum(xh.nbytes + fh[k].nbytes for k in cfg["kernels"])
        d2h = sum(uh[k].nbytes for k in cfg["kernels"])
        e2e = {"value": targets_per_step * args.steps / dt, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    # the plain FP64 single-RHS form of the same workload and tolerance (comparison of the metric)
    fp64 = None
    if not args.no_fp64:
        plans64, f64 = {}, {}
        for k in cfg["kernels"]:
            t = params[k]
            plans64[k] = se.Plan(cfg["D"], cfg["box"], t["xi"], t["rc"], t["M"], t["P"], cfg["window"], "fp64",
                                 stream=stream)
            f64[k] = torch.tensor(fs[k].astype(np.float64), device=dev)
        u64 = {k: torch.empty((1, N, 3), dtype=torch.float64, device=dev) for k in cfg["kernels"]}

        def step64():
            for k in cfg["kernels"]:
                for r in range(R):
                    plans64[k].evaluate(k, xdev, f64[k][r], out=u64[k])

        for _ in range(3):
            step64()
        torch.cuda.synchronize()
        n64 = max(3, args.steps // 4)
        ev64 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n64)]
        for s_ in range(n64):
            flush.zero_()
            ev64[s_][0].record(stream)
            step64()
            ev64[s_][1].record(stream)
        torch.cuda.synchronize()
        t64 = sum(a.elapsed_time(b) for a, b in ev64)
        fp64 = {"value": targets_per_step * n64 / (t64 / 1e3), "unit": UNIT, "ms_per_step": t64 / n64,
                "form": "FP64, one RHS per evaluation, same parameters"}

    # headline: the FP32 batched form (the metric compares it with the FP64 plain form); the
    # eager per-call form, whose per-kernel events give the stage times and the roofline, beside it
    eager = {"value": value, "unit": UNIT, "ms_per_step": tot_ms / args.steps,
             "form": "FP32, one se_eval call per kernel per step"}
    g_ms = max_over_ranks(graph["ms_per_step"] * args.steps, dist, dev)
    value = replica_value(targets_per_step, world, args.steps, g_ms)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": g_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "N": N, "n_rhs": R, "box": list(cfg["box"]),
                       "kernels": list(cfg["kernels"]), "periodicity": cfg["D"],
                       "tol_rel": cfg["tol"], "window": cfg["window"], "params": params,
                       "selection": {"n_rc": cfg.get("n_rc"), "P_margin": cfg.get("P_margin", -1),
                                     "tol_requested": cfg["tol"] / 10.0},
                       "targets_per_step": targets_per_step, "l2": "flushed between steps (256 MB write)",
                       "gridding": "tcgen05" if args.gridding == "tc" else "cuda cores",
                       "parallelism": "replicas" if world > 1 else "single"},
            "stage_ms_per_step": per_stage, "roofline": roof, "clocks": clocks, "e2e": e2e,
            "gpu_launches": launches, "fp32_eager": eager, "fp32_graph": graph, "fp64_plain": fp64}

    # ---- CPU baseline (rank 0, N = 1): the oracle on a bounded sample; also the GPU error there
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # a bounded sample (a few seconds of oracle work); the oracle's per-call cost (the
        # k-space structure factors) is amortised over the sample's targets
        ns = 1024 if N <= 50000 else 64
        idx, ref, dt = oracle_sample(cfg, x, fs, ns)
        err = {}
        from oracle import ewald as E
        for k in cfg["kernels"]:
            err[k] = E.rms_rel(udev[k][0].cpu().numpy()[idx].astype(np.float64), ref[k])
        line["cpu_baseline"] = {"value": ns * len(cfg["kernels"]) / dt, "unit": UNIT, "cores": os.cpu_count(),
                                "kind": "oracle",
                                "sample": "%d sampled targets x %d kernels (RHS 0) against all %d sources" %
                                          (ns, len(cfg["kernels"]), N)}
        line["rms_rel_err_vs_oracle"] = err
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
