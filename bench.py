#!/usr/bin/env python
"""Benchmark of the GB300 NKS time step (arXiv 2209.08001, Sec. 4).

Metric: point-steps/s = grid points x accepted time steps / seconds of the
step loop.  Default workload: the 2-D 1024x1024 periodic FP64 configuration
(200 adaptive DVD steps with the energy-change dt driver, GMRES(30), RAS on
16x16 subdomains with overlap 2, ILU(0)-reuse); seeded synthetic initial
fields.  A bench "step" is one accepted time step (one NKS solve).  Timed
steps start from the workload's initial state (steps 1..K), after W warm-up
steps whose state is discarded.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs one independent replica per GPU (launched by torch.distributed.run;
the method has no data-path exchange on one GPU per problem), weak scaling.
--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.  One JSON line is printed by rank 0.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic as S  # noqa: E402

METRIC = "point-steps/s"
# FP64 FMA peak derived from the unit counts: 152 SMs x 2 FP64 FMA/clk x 2 FLOP x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# DRAM traffic per launch of the dominant kernel (dram__bytes.sum.per_second x duration),
# keyed by (workload, precision, kernel class), from one ncu capture of the 1024^2 probe
# (bench.py --probe gmres1024: the bench workload's own 256-box launch); an entry is
# removed whenever the kernel changes
NCU_TRAFFIC = {("2d1024", "fp64", "schwarz_apply"): 932.815680e9 * 969.792e-6,
               ("2d1024", "mixed", "schwarz_apply"): 1435.653e9 * 275.168e-6}


def kernel_rates(st, cfg, mixed, pk):
    """Achieved rates per kernel class from the CUDA-event times of the timed steps:
    HBM-bound classes against the measured copy bandwidth, FP64-bound ones against
    the derived FP64 peak (algorithmic bytes / FLOPs per unit as in the design notes)."""
    d = cfg["dim"]
    N = float(np.prod(cfg["n"]))
    f = 2 + d
    b = 4.0 if mixed else 8.0
    out = {}
    hbm = pk.get("hbm_gbs")

    def rate(cls, nbytes, nflops=None, bound="hbm"):
        ms = st["ms"].get(cls, 0.0)
        if ms <= 0 or nbytes <= 0:
            return
        gbs = nbytes / (ms / 1e3) / 1e9
        e = {"algorithmic_bytes": nbytes, "ms": ms, "launches": st["launches"][cls], "achieved_gbs": gbs,
             "hbm_frac": gbs / hbm if hbm else None, "bound": bound}
        if nflops:
            e["achieved_tflops"] = nflops / (ms / 1e3) / 1e12
            e["fp64_frac"] = e["achieved_tflops"] / FP64_PEAK_TFLOPS
        out[cls] = e

    # Jacobian action: (2f + 5) words per point per application (v, 4 coefficients + edge
    # mobility, J v), FP32 words in the Arnoldi step of the mixed mode
    rate("jacobian_action", st["launches"]["jacobian_action"] * (2 * f + 5) * b * N,
         bound="hbm" if mixed else "alu")
    # Gram-Schmidt: (2j + 5) basis-vector transfers per pass of Arnoldi step j (counted by the library)
    gs_ms = st["ms"].get("gs_dots", 0.0) + st["ms"].get("gs_update", 0.0)
    if gs_ms > 0 and st.get("cgs_bytes", 0) > 0:
        gbs = st["cgs_bytes"] / (gs_ms / 1e3) / 1e9
        out["gram_schmidt"] = {"algorithmic_bytes": st["cgs_bytes"], "ms": gs_ms, "achieved_gbs": gbs,
                               "hbm_frac": gbs / hbm if hbm else None, "bound": "hbm" if mixed else "alu",
                               "second_passes": st.get("reorth"), "arnoldi_steps": st["gmres_its"]}
    # Schwarz sweeps
    rate("schwarz_apply", st["launches"]["schwarz_apply"] * st["schwarz_bytes"],
         None if mixed else st["launches"]["schwarz_apply"] * st["schwarz_flops"], bound="hbm" if mixed else "alu")
    return out


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.Q, "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.dev)], stdout=open(self.path, "w"),
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def init_dist(ws, backend):
    if ws <= 1:
        return None
    import torch.distributed as dist
    dist.init_process_group(backend=backend)
    return dist


def max_over_ranks(dist, value, device=None):
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(dist, value, device=None):
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ---------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------

def oracle_sample(cfg, gmres_per_step, newton_per_step, its=(2, 6)):
    """Times the FP64 oracle on the full-size workload: Jacobian assembly, the
    RAS/ILU(0) set-up and GMRES iterations of the first Newton solve, at two
    iteration caps.  One time step is then estimated as newton_per_step set-ups
    (assembly + factorisation) plus gmres_per_step GMRES iterations (the counts
    of the same algorithm on the same workload)."""
    import oracle
    op = S.options(**cfg["opts"])
    c, e = S.config_fields(cfg)
    N = c.size
    times = []
    O = None
    for m in its:
        O = oracle.Problem(cfg["dim"], cfg["n"], cfg["h"], S.config_coefficients(cfg), dict(op, gmres_maxit=m))
        X = O.interleave(c, e)
        cb = float(np.sum(c) / N)
        F = O.residual(X, X, cb, op["dt_init"])
        t0 = time.perf_counter()
        O.linear_solve(X, X, cb, op["dt_init"], -F, 0.0)
        times.append(time.perf_counter() - t0)
    t_it = max((times[1] - times[0]) / (its[1] - its[0]), 1e-9)
    t_setup = max(times[0] - its[0] * t_it, 0.0)
    step_s = newton_per_step * t_setup + gmres_per_step * t_it
    return {"value": N / step_s, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": ("full-size %s workload, first Newton solve: Jacobian assembly + RAS/ILU(0) set-up + %d and %d "
                       "GMRES iterations timed (%.1f s, %.1f s); step = %.2f set-ups + %.1f iterations (per-step "
                       "counts of the same method); single-threaded FP64 C oracle"
                       % ("x".join(str(v) for v in cfg["n"]), its[0], its[1], times[0], times[1],
                          newton_per_step, gmres_per_step)),
            "seconds_per_step": step_s, "t_setup_s": t_setup, "t_gmres_iteration_s": t_it}


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = init_dist(ws, "nccl")
    import __graft_entry__ as g
    if rank == 0 or ws == 1:
        g.build()
    if dist is not None:
        dist.barrier()
    import paper_2209_08001_gb300 as nks

    cfg = S.CONFIGS[args.config]
    op = S.options(**cfg["opts"])
    if args.precision:
        op["precision"] = args.precision
    if args.variant:
        op["ras_variant"] = args.variant
    if args.overlap is not None:
        op["overlap"] = args.overlap
    if args.u0_maxit is not None:
        op["u0_maxit"] = args.u0_maxit
    c, e = S.config_fields(cfg, 1000 * rank)  # independent replica per rank (seeded workloads)
    N = c.size
    tuned = None
    if args.autotune:
        # owned box sides 8..16 (3-D) or 32..128 (2-D), overlap 1 and 2; one timed step each
        sides = (8, 12, 16) if cfg["dim"] == 3 else (32, 64, 128)
        cands = [(tuple(max(2, (nn + b // 2) // b) for nn in cfg["n"]), ov) for b in sides for ov in (1, 2)]
        op, table, chosen = nks.autotune(cfg["dim"], cfg["n"], cfg["h"], c, e, S.config_coefficients(cfg), op,
                                         candidates=cands, dt_trial=op["dt_init"])
        tuned = {"candidates": [{"sub": list(sb), "overlap": ov, "step_s": t} for sb, ov, t in table],
                 "chosen": {"sub": list(op["sub"]), "overlap": op["overlap"]}}
    stream = torch.cuda.current_stream()
    alloc = nks.torch_allocator()
    torch.cuda.synchronize()
    t_setup = time.perf_counter()
    P = nks.Problem(cfg["dim"], cfg["n"], cfg["h"], c, e, S.config_coefficients(cfg), op, stream=stream.cuda_stream,
                    allocator=alloc, timing=True)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup
    sst = P.get_stats()
    setup = {"seconds": t_setup, "u0_newton_its": sst["newton_its"], "u0_gmres_its": sst["gmres_its"],
             "device_bytes": P.device_bytes(),
             "includes": "problem creation: plan, factor tables, upload, initial mechanical equilibrium (Newton on "
                         "the displacement rows, tolerance u0_rtol)"}
    state0 = P.get_state()
    for _ in range(args.warmup):
        P.step()
    P.set_state(state0)
    P.reset_stats()
    clocks = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    infos = [P.step() for _ in range(args.steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    if dist is not None:
        dist.barrier()
    ms_max = max_over_ranks(dist, ms, torch.device("cuda", local))
    points_all = sum_over_ranks(dist, float(N * args.steps), torch.device("cuda", local))
    st = P.get_stats()
    value = points_all / (ms_max / 1e3)

    # roofline of the dominant kernel class, and achieved rates of the others
    pk = peaks()
    mixed = op["precision"] == "mixed"
    kernels = kernel_rates(st, cfg, mixed, pk)
    cls = max(st["ms"], key=lambda k: st["ms"][k])
    launches = max(st["launches"][cls], 1)
    avg_s = st["ms"][cls] / launches / 1e3
    if cls == "schwarz_apply" and not mixed:
        # FP64 sweeps: 2 FLOP per stored factor entry per point; bound by the FP64 pipe on GB300
        flops = st["schwarz_flops"]
        roof = {"kernel": "k_ras_apply<FP64> (ILU(0) sweeps, TMA-staged factors)", "bound": "alu",
                "achieved": flops / avg_s / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": flops / avg_s / 1e12 / FP64_PEAK_TFLOPS,
                "peak_source": "derived FP64 FMA peak: 152 SMs x 2 FP64 FMA/clk x 2 FLOP x 2.07 GHz "
                               "(a measured FMA loop reached 1.20)",
                "algorithmic_flops_per_launch": flops, "algorithmic_bytes_per_launch": st["schwarz_bytes"],
                "hbm_achieved_gbs": st["schwarz_bytes"] / avg_s / 1e9, "hbm_peak_gbs": pk.get("hbm_gbs"),
                "traffic": NCU_TRAFFIC.get((args.config, op["precision"], cls)), "avg_launch_ms": avg_s * 1e3,
                "launches": launches}
    elif cls == "schwarz_apply":
        # FP32 sweeps (mixed precision): factors and sub-vectors streamed once per sweep
        by = st["schwarz_bytes"]
        roof = {"kernel": "k_ras_apply<FP32> (ILU(0) sweeps, TMA-staged factors)", "bound": "hbm",
                "achieved": by / avg_s / 1e9, "peak": pk.get("hbm_gbs"), "unit": "GB/s",
                "frac": by / avg_s / 1e9 / pk.get("hbm_gbs"), "peak_source": "measured copy bandwidth (burst)",
                "algorithmic_bytes_per_launch": by, "algorithmic_flops_per_launch": st["schwarz_flops"],
                "traffic": NCU_TRAFFIC.get((args.config, op["precision"], cls)), "avg_launch_ms": avg_s * 1e3,
                "launches": launches}
    else:
        roof = dict(kernels.get(cls, {}), kernel=cls, traffic=NCU_TRAFFIC.get((args.config, op["precision"], cls)))
    # mixed precision: error per field against the FP64 path on the same dt sequence
    accuracy = None
    if mixed and not args.no_accuracy and rank == 0:
        cm, em, um = P.get_fields()
        Q = nks.Problem(cfg["dim"], cfg["n"], cfg["h"], c, e, S.config_coefficients(cfg), dict(op, precision="fp64"),
                        stream=stream.cuda_stream, allocator=alloc)
        for i in infos:
            Q.step(i["dt"])
        cd, ed, ud = Q.get_fields()
        Q.destroy()
        rel = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
        accuracy = {"reference": "FP64 GPU path (parity-tested against the FP64 oracle), same dt sequence, "
                                 "after the K timed steps",
                    "rel_l2": {"c": rel(cm, cd), "eta": rel(em, ed), "u": rel(um, ud) if um is not None else None},
                    "tolerance": 1e-8}
    total_ms = sum(st["ms"].values())
    breakdown = {k: round(v / max(total_ms, 1e-9), 4) for k, v in st["ms"].items() if v > 0}

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        cpin = torch.from_numpy(c).pin_memory().numpy()
        epin = torch.from_numpy(e).pin_memory().numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        Q = nks.Problem(cfg["dim"], cfg["n"], cfg["h"], cpin, epin, S.config_coefficients(cfg), op, stream=stream.cuda_stream,
                        allocator=alloc)
        outs = []
        for _ in range(args.steps):
            Q.step()
            outs.append(Q.get_fields()[0])
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        Q.destroy()
        t_e2e = max_over_ranks(dist, t_e2e, torch.device("cuda", local))
        e2e = {"value": points_all / t_e2e, "unit": METRIC,
               "h2d_bytes_per_step": int(2 * N * 8 / args.steps),
               "d2h_bytes_per_step": int((2 + (cfg["dim"] if S.config_coefficients(cfg).get("Lscale", 1.0) else 0)) * N * 8),
               "includes": "problem creation from host fields (upload + initial mechanical equilibrium solve), "
                           "K steps, fields read back to host after every step"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        gm = st["gmres_its"] / max(st["steps"], 1)
        nw = st["newton_its"] / max(st["steps"], 1)
        cpu = oracle_sample(cfg, gm, nw)
        cpu = {k: cpu[k] for k in ("value", "unit", "cores", "kind", "sample")}

    out = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if op["precision"] == "fp64" else "f64+f32",
        "data": "synthetic (seeded SplitMix64 initial fields)",
        "config": {"workload": cfg["desc"], "precision": op["precision"], "grid": list(cfg["n"]), "points": N,
                   "decomposition": {"sub": list(op["sub"]), "overlap": op["overlap"],
                                     "schwarz": op.get("ras_variant", "left-ras")},
                   "steps_in_workload": cfg["steps"],
                   "timed_steps": "steps 1..K of the workload from its initial state",
                   "initial_equilibrium": ("Newton on the displacement rows, FP64 residual to u0_rtol, inner GMRES in "
                                           "the mixed form" if op.get("u0_mixed") else
                                           "Newton on the displacement rows in the solver's precision"),
                   "l2": "working set (state, Krylov basis, ~0.65 GB of Schwarz factors) far above the 129 MB L2",
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "gpu_launches": None,
        "setup": setup,
        "autotune": tuned,
        "roofline": roof,
        "kernels": kernels,
        "accuracy": accuracy,
        "kernel_time_share": breakdown,
        "iterations": {"newton_per_step": st["newton_its"] / max(st["steps"], 1),
                       "gmres_per_step": st["gmres_its"] / max(st["steps"], 1),
                       "dt": [i["dt"] for i in infos]},
        "clocks": clk,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    # kernels this library launched inside the timed region (counted at every launch site)
    out["gpu_launches"] = int(st["kernel_launches"])
    P.destroy()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    cfg = S.CONFIGS[args.config]
    # per-step iteration counts of the method on this workload (same algorithm as the oracle)
    gm, nw = args.ref_gmres_per_step, args.ref_newton_per_step
    samples = []
    for _ in range(args.warmup + args.steps):
        samples.append(oracle_sample(cfg, gm, nw, its=(1, 3)))
    timed = samples[args.warmup:]
    step_s = statistics.mean(s["seconds_per_step"] for s in timed)
    N = int(np.prod(cfg["n"]))
    v = N / step_s
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded SplitMix64 initial fields)",
           "config": {"workload": cfg["desc"], "grid": list(cfg["n"]), "points": N},
           "cpu_baseline": {"value": v, "unit": METRIC, "cores": 1, "kind": "oracle", "sample": timed[0]["sample"]},
           "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_batch(args):
    """--batch B: B instances of the workload (seeds seed, seed + 1, ...) stepped as
    one batch (one launch per solver phase, GMRES iterations replayed from CUDA
    graphs), beside the same workload stepped alone; one JSON line."""
    import torch
    import paper_2209_08001_gb300 as nks
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)
    cfg = S.CONFIGS[args.config]
    op = S.options(**cfg["opts"])
    if args.precision:
        op["precision"] = args.precision
    B = args.batch
    fields = [S.config_fields(cfg, i) for i in range(B)]
    c = np.stack([f[0] for f in fields])
    e = np.stack([f[1] for f in fields])
    N = c.shape[1]
    stream = torch.cuda.current_stream()

    def timed(run_steps, reset):
        for _ in range(args.warmup):
            run_steps()
        reset()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        ev0.record(stream)
        for _ in range(args.steps):
            run_steps()
        ev1.record(stream)
        torch.cuda.synchronize()
        return ev0.elapsed_time(ev1), (time.perf_counter() - t0) * 1e3

    Bt = nks.Batch(cfg["dim"], cfg["n"], cfg["h"], B, S.config_coefficients(cfg), op, c=c, eta=e,
                   allocator=nks.torch_allocator())
    st0 = [Bt.get_state(i) for i in range(B)]
    clocks = ClockSampler(0)
    clocks.start()
    ms_b, wall_b = timed(lambda: Bt.step(), lambda: [Bt.set_state(i, st0[i]) for i in range(B)])
    clk = clocks.stop()
    stats = Bt.get_stats()
    P = nks.Problem(cfg["dim"], cfg["n"], cfg["h"], c[0], e[0], S.config_coefficients(cfg), op,
                    allocator=nks.torch_allocator())
    s1 = P.get_state()
    ms_1, _ = timed(lambda: P.step(), lambda: P.set_state(s1))
    value = B * N * args.steps / (wall_b / 1e3)
    out = {"metric": METRIC, "value": value, "unit": METRIC, "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": wall_b / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64" if op["precision"] == "fp64" else "f64+f32",
           "data": "synthetic (seeded SplitMix64 initial fields, one seed per instance)",
           "config": {"workload": "%d instances of: %s" % (B, cfg["desc"]), "batch": B, "precision": op["precision"],
                      "grid": list(cfg["n"]), "points_per_instance": N,
                      "timed_steps": "steps 1..K of every instance from its initial state",
                      "l2": "small grids: the working set fits in L2 (latency- and launch-bound, no HBM fraction)"},
           "device_ms_per_step": ms_b / args.steps,
           "single_instance": {"value": N * args.steps / (ms_1 / 1e3), "ms_per_step": ms_1 / args.steps},
           "batch_speedup_over_single": (value / (N * args.steps / (ms_1 / 1e3))),
           "gpu_launches": int(stats["kernel_launches"]),
           "iterations": {"gmres_per_instance_step": stats["gmres_its"] / max(stats["steps"], 1),
                          "newton_per_instance_step": stats["newton_its"] / max(stats["steps"], 1)},
           "device_bytes": Bt.device_bytes(), "clocks": clk, "roofline": None}
    Bt.destroy()
    P.destroy()
    print(json.dumps(out), flush=True)


def run_serve(args):
    """--serve: the serving workload.  Requests from the synthetic stream (2-D grids
    64^2..512^2 or 3-D 32^3..96^3, log-uniform sides, mean composition U(0.10,
    0.25), mixed precision, adaptive dt) go through the native request loop.  A
    closed-loop pass over the first requests measures the saturated request
    rate; the timed pass submits every request at its Poisson arrival time with
    rate 0.8 x that, and reports p50 / p99 time-to-completion and the aggregate
    point-steps/s (points x steps of all requests / makespan)."""
    import threading
    import torch
    import paper_2209_08001_gb300 as nks
    import __graft_entry__ as g
    g.build()
    torch.cuda.set_device(0)
    op = S.options(precision=args.precision or "mixed", dt_mode="energy", overlap=1)
    R, steps = args.requests, args.req_steps

    def stream_run(reqs, rate):
        srv = nks.Server(S.coefficients(), op, max_slots=args.slots, max_groups=args.groups)
        ids = {}
        t0 = time.perf_counter()

        def feeder():
            for r in reqs:
                if rate > 0:
                    dt = r["arrival"] - (time.perf_counter() - t0)
                    if dt > 0:
                        time.sleep(dt)
                c, e = S.initial_fields(r["dim"], r["n"], r["cbar"], r["seed"])
                ids[r["id"]] = srv.submit(r["dim"], r["n"], r["h"], c, e, steps)

        th = threading.Thread(target=feeder)
        th.start()
        th.join()
        res = [srv.wait(ids[r["id"]])[0] for r in reqs]
        wall = time.perf_counter() - t0
        srv.destroy()
        return res, wall

    base = S.serving_requests(count=R, seed=4, rate=1.0)
    # saturated rate: the first requests all at once
    nsat = min(R, max(8, R // 4))
    sat, wall_sat = stream_run(base[:nsat], 0.0)
    span = max(r["t_done"] for r in sat) - min(r["t_submit"] for r in sat)
    rate_sat = nsat / max(span, 1e-9)
    rate = 0.8 * rate_sat
    reqs = S.serving_requests(count=R, seed=4, rate=rate)
    clocks = ClockSampler(0)
    clocks.start()
    res, wall = stream_run(reqs, rate)
    clk = clocks.stop()
    lat = np.array([r["t_done"] - r["t_submit"] for r in res])
    qwait = np.array([r["t_admit"] - r["t_submit"] for r in res])
    bad = sum(1 for r in res if r["status"] != 0)
    t_first = min(r["t_submit"] for r in res)
    makespan = max(r["t_done"] for r in res) - t_first
    pts = float(sum(r["points"] * r["steps"] for r in res))
    out = {"metric": "serving p50/p99 time-to-completion; aggregate point-steps/s", "value": pts / makespan,
           "unit": METRIC, "n_gpus": 1, "steps": steps, "warmup": 0, "ms_per_step": None, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32" if op["precision"] == "mixed" else "f64",
           "data": "synthetic request stream (seeded; Poisson arrivals)",
           "config": {"workload": "%d requests, %d adaptive steps each: 2-D 64^2..512^2 or 3-D 32^3..96^3 "
                                  "(log-uniform sides, multiples of 16), cbar ~ U(0.10, 0.25), %s precision"
                                  % (R, steps, op["precision"]),
                      "requests": R, "steps_per_request": steps, "slots_per_group": args.slots,
                      "groups": args.groups},
           "latency_s": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                         "mean": float(lat.mean()), "max": float(lat.max())},
           "queue_wait_s": {"p50": float(np.percentile(qwait, 50)), "p99": float(np.percentile(qwait, 99))},
           "arrival_rate_req_s": rate, "saturated_rate_req_s": rate_sat, "makespan_s": makespan,
           "failed_requests": bad, "clocks": clk, "roofline": None}
    print(json.dumps(out), flush=True)


def run_probe(args):
    """Small fixed cases for profiling single kernels (ncu -k ...): 'gmres512' builds
    the 2-D 512^2 problem with 8x8 subdomains, overlap 2 (the 68x68 boxes of the
    1024^2 workload), 'gmres1024' the 1024^2 problem itself with its 16x16
    subdomains (the bench's launch configuration, about 2.5 GB on the device);
    both run 40 GMRES iterations of the first Newton solve (FP64, or FP32 sweeps
    and basis with --precision mixed) after a one-iteration set-up solve."""
    import torch
    import paper_2209_08001_gb300 as nks
    torch.cuda.set_device(0)
    if args.probe in ("gmres512", "gmres1024"):
        side, sub = (512, 8) if args.probe == "gmres512" else (1024, 16)
        n = (side, side)
        op = S.options(sub=(sub, sub), overlap=2, u0_maxit=1, gmres_maxit=40, u0_rtol=1e-2,
                       precision=args.precision or "fp64")
        c, e = S.initial_fields(2, n, 0.2, 1)
        P = nks.Problem(2, n, 0.25, c, e, S.coefficients(), op)
        cg, eg, ug = P.get_fields()
        X = np.concatenate([cg, eg, ug[0], ug[1]])
        b = -P.eval_residual(X, X, 0.01)
        x, its, res = P.linear_solve(X, X, 0.01, b, 1e-30)
        print(json.dumps({"probe": args.probe, "gmres_its": its, "res": res}))
        P.destroy()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="2d1024", choices=sorted(S.CONFIGS))
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed"],
                    help="override the workload's precision mode (default: the workload's own)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true", help="mixed precision: skip the FP64 comparison")
    # iteration counts used to scale the oracle sample in the reference arm (measured on the GPU arm)
    ap.add_argument("--ref-gmres-per-step", type=float, default=1700.0)
    ap.add_argument("--ref-newton-per-step", type=float, default=5.67)
    ap.add_argument("--probe", default=None, choices=["gmres512", "gmres1024"], help="small profiling case, no JSON bench line")
    ap.add_argument("--batch", type=int, default=0,
                    help="B > 0: B instances of the workload stepped as one batch (beside one alone)")
    ap.add_argument("--serve", action="store_true", help="the serving workload (p50/p99 latency, throughput)")
    ap.add_argument("--variant", default=None, choices=["left-ras", "as", "right-ras"],
                    help="Schwarz preconditioner type (default: the workload's, left-RAS)")
    ap.add_argument("--overlap", type=int, default=None, help="override the workload's Schwarz overlap delta")
    ap.add_argument("--u0-maxit", type=int, default=None,
                    help="Newton iterations allowed to the initial mechanical equilibrium (set-up, not timed)")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the Schwarz decomposition with nks_autotune before timing")
    ap.add_argument("--requests", type=int, default=64, help="--serve: requests in the stream")
    ap.add_argument("--req-steps", type=int, default=10, help="--serve: time steps per request")
    ap.add_argument("--slots", type=int, default=16, help="--serve: slots per shape group")
    ap.add_argument("--groups", type=int, default=8, help="--serve: shape groups alive at once")
    args = ap.parse_args()
    if args.probe:
        run_probe(args)
    elif args.batch > 0 and args.impl == "ours":
        run_batch(args)
    elif args.serve and args.impl == "ours":
        run_serve(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
