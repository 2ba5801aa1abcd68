#!/usr/bin/env python
"""Benchmark of the GB300 NKS time step (arXiv 2209.08001, Sec. 4).

Metric: point-steps/s = grid points x accepted time steps / seconds of the
step loop, with the mixed-precision solver (FP32 Schwarz factors, sweeps and
Krylov basis; FP64 residual, update, logarithms, energy and mass) beside the
plain FP64 solver on the same steps.  Default workload: the 3-D 128^3 periodic
configuration (c = 0.18 + U(-0.005, 0.005), seed 2, 50 adaptive DVD steps with
the energy-change dt driver, GMRES(30), left-RAS on 8x8x8 subdomains with
overlap 1, ILU(0)-reuse); seeded synthetic initial fields.  A bench "step" is
one accepted time step (one NKS solve).  Timed steps start from the workload's
initial state (steps 1..K), after W warm-up steps whose state is discarded;
the FP64 solver replays the mixed run's dt sequence.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--config 3d128] [--precision mixed|fp64] [--grid SIDE]

N > 1 runs one independent replica per GPU (launched by torch.distributed.run;
the method has no data-path exchange on one GPU per problem), weak scaling.
--impl reference times the FP64 CPU oracle on the host cores (real time steps
of a bounded sample of the workload).  One JSON line is printed by rank 0.
"""
import argparse
import json
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
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic.json")


def peaks():
    try:
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        pk.setdefault("source", "measured (MEASURED_PEAKS.json)")
        return pk
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback (no MEASURED_PEAKS.json)"}


def workload(name, side=None):
    """The workload's description, optionally on a smaller cubic / square grid of
    `side` cells per axis with the same Schwarz box size (sub = side / box)."""
    cfg = dict(S.CONFIGS[name])
    cfg["opts"] = dict(cfg["opts"])
    if side:
        d = cfg["dim"]
        box = [cfg["n"][J] // cfg["opts"]["sub"][J] for J in range(d)]
        cfg["n"] = tuple([side] * d)
        cfg["opts"]["sub"] = tuple(max(1, side // b) for b in box)
        cfg["desc"] = "%s [on a %s grid, sub %s]" % (cfg["desc"], "x".join([str(side)] * d),
                                                    "x".join(str(v) for v in cfg["opts"]["sub"]))
    return cfg


def kernel_rates(st, cfg, mixed, pk):
    """Achieved rates per kernel class from the CUDA-event times of the timed steps:
    algorithmic bytes per unit (as in the design notes) over the class's device time."""
    d = cfg["dim"]
    N = float(np.prod(cfg["n"]))
    ne, f = layout(cfg)
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

    # Jacobian action: 2f + (1 + ne)^2 + d words per point per application (v, the
    # pointwise derivative block, the d edge mobilities, J v), FP32 words in the
    # Arnoldi step of the mixed mode
    rate("jacobian_action", st["launches"]["jacobian_action"] * (2 * f + (1 + ne) ** 2 + d) * b * N,
         bound="hbm" if mixed else "fp64")
    # the FP64 action on the true residual at the end of every GMRES cycle (both precisions)
    rate("true_residual_jv", st["launches"].get("true_residual_jv", 0) * (2 * f + (1 + ne) ** 2 + d) * 8.0 * N,
         bound="fp64")
    # Gram-Schmidt: (2j + 5) basis-vector transfers per pass of Arnoldi step j (counted by the library)
    gs_ms = st["ms"].get("gs_dots", 0.0) + st["ms"].get("gs_update", 0.0)
    if gs_ms > 0 and st.get("cgs_bytes", 0) > 0:
        gbs = st["cgs_bytes"] / (gs_ms / 1e3) / 1e9
        out["gram_schmidt"] = {"algorithmic_bytes": st["cgs_bytes"], "ms": gs_ms, "achieved_gbs": gbs,
                               "hbm_frac": gbs / hbm if hbm else None, "bound": "hbm" if mixed else "fp64",
                               "second_passes": st.get("reorth"), "arnoldi_steps": st["gmres_its"]}
    rate("schwarz_apply", st["launches"]["schwarz_apply"] * st["schwarz_bytes"],
         None if mixed else st["launches"]["schwarz_apply"] * st["schwarz_flops"],
         bound="hbm" if mixed else "fp64")
    return out


def traffic_for(workload_name, side, precision, kernel):
    """DRAM bytes per launch of `kernel` from the ncu summary recorded for this
    workload, precision and the library's current source hash; None (with the
    reason) when no capture of the current kernels exists."""
    from paper_2209_08001_gb300 import build
    h = build.source_hash(kernel)
    try:
        entries = json.load(open(TRAFFIC_FILE))["entries"]
    except Exception:
        return None, "no ncu traffic record (profiles/traffic.json)"
    for e in entries:
        if (e["workload"], e.get("side"), e["precision"], e["kernel"]) == (workload_name, side, precision, kernel):
            if e["source_hash"] != h:
                return None, "ncu capture %s is of other kernel sources (%s, now %s)" % (e["profile"],
                                                                                       e["source_hash"], h)
            return e["dram_bytes_per_launch"], "ncu dram__bytes_read.sum + dram__bytes_write.sum, %s" % e["profile"]
    return None, "no ncu traffic record for this workload, precision and kernel"


def roofline(st, kernels, mixed, pk, wl, side, precision):
    """Roofline of the dominant kernel class of the timed steps."""
    cls = max(st["ms"], key=lambda k: st["ms"][k])
    launches = max(st["launches"][cls], 1)
    avg_s = st["ms"][cls] / launches / 1e3
    if cls == "schwarz_apply":
        by, fl = st["schwarz_bytes"], st["schwarz_flops"]
        if mixed:
            tr, why = traffic_for(wl, side, precision, "k_ras_apply_lane")
            roof = {"kernel": "k_ras_apply_lane<FP32> (ILU(0) sweeps, TMA-staged point-major factors)",
                    "bound": "hbm", "achieved": by / avg_s / 1e9, "peak": pk.get("hbm_gbs"), "unit": "GB/s",
                    "frac": by / avg_s / 1e9 / pk.get("hbm_gbs"),
                    "peak_source": "%s, copy bandwidth" % pk.get("source"),
                    "limiter": "wavefront latency: each box is a chain of dependent level steps (one "
                               "point's rows per thread, then a block barrier) at one warp per scheduler",
                    "algorithmic_bytes_per_launch": by, "algorithmic_flops_per_launch": fl}
        else:
            tr, why = traffic_for(wl, side, precision, "k_ras_apply")
            roof = {"kernel": "k_ras_apply<FP64> (ILU(0) sweeps, TMA-staged factors)", "bound": "alu",
                    "achieved": fl / avg_s / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": fl / avg_s / 1e12 / FP64_PEAK_TFLOPS,
                    "peak_source": "derived FP64 FMA peak: 152 SMs x 2 FP64 FMA/clk x 2 FLOP x 2.07 GHz "
                                   "(a measured FMA loop reached 1.20)",
                    "limiter": "FP64 pipe and wavefront latency (barriers between levels)",
                    "algorithmic_flops_per_launch": fl, "algorithmic_bytes_per_launch": by,
                    "hbm_achieved_gbs": by / avg_s / 1e9, "hbm_peak_gbs": pk.get("hbm_gbs")}
    else:
        tr, why = None, "no ncu traffic record for this kernel class"
        roof = dict(kernels.get(cls, {}), kernel=cls)
    roof.update({"traffic": tr, "traffic_source": why, "avg_launch_ms": avg_s * 1e3, "launches": launches,
                 "timing": "CUDA events around every launch of the class on the solver's stream"})
    return roof


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


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def layout(cfg):
    """(order parameters, fields per point) of a workload"""
    cf = S.config_coefficients(cfg)
    ne = 3 if cf.get("n_eta", 1) == 3 else 1
    elastic = cf.get("Lscale", 1.0) != 0.0 and any(cf[k] != 0.0 for k in ("C11", "C12", "C44"))
    return ne, 1 + ne + (cfg["dim"] if elastic else 0)


def field_dict(c, e, u):
    e = np.asarray(e)
    out = {"c": c, "eta": e} if e.ndim == 1 else {"c": c, **{"eta%d" % (j + 1): e[j] for j in range(len(e))}}
    if u is not None:
        for I in range(len(u)):
            out["u%d" % (I + 1)] = u[I]
    return out


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample of the workload (cpu_baseline, --impl reference)
# ---------------------------------------------------------------------------

def cpu_sample_config(name):
    """The bounded sample of a workload that the CPU oracle runs: the same recipe
    (initial state, coefficients, solver settings, Schwarz box size and overlap)
    on a periodic grid of three boxes per axis (3-D 48^3 for 16^3 boxes, 2-D
    192^2 for 64^2 boxes), or the workload itself when it is no larger."""
    cfg = S.CONFIGS[name]
    d = cfg["dim"]
    box = [cfg["n"][J] // cfg["opts"]["sub"][J] for J in range(d)]
    side = 3 * max(box)
    if side >= max(cfg["n"][:d]):
        return cfg, None
    return workload(name, side), side


def oracle_steps(cfg, warmup, steps, threads=None):
    """Real oracle time steps: the initial mechanical equilibrium (set-up, not
    timed), then warmup + steps NKS steps with the workload's dt rule (dt_init,
    then the oracle's predictor of Eq. sencondt, divergence retries), each timed.
    Returns (per-step seconds of the timed steps, infos, set-up seconds, threads)."""
    import oracle
    oracle.set_threads(threads or 0)
    op = S.options(**cfg["opts"])
    op["precision"] = "fp64"
    c, e = S.config_fields(cfg)
    O = oracle.Problem(cfg["dim"], cfg["n"], cfg["h"], S.config_coefficients(cfg), op)
    X = O.interleave(c, e)
    cb = float(np.sum(c) / c.size)
    t0 = time.perf_counter()
    rc, X, _ = O.equilibrate(X, cb)
    t_setup = time.perf_counter() - t0
    if rc != 0:
        raise RuntimeError("oracle equilibrium failed (%d)" % rc)
    E, Eprev, dt_prev, zeta = O.energy(X, cb), None, op["dt_init"], op["zeta"]
    secs, infos = [], []
    for st in range(warmup + steps):
        if st == 0 or op["dt_mode"] == "fixed":
            dt = op["dt_init"]
        else:
            dt = oracle.dt_predict(op["dt_min"], op["dt_max"], zeta, abs(E - Eprev) / dt_prev)
        zeta = op["zeta"]
        t0 = time.perf_counter()
        for _ in range(op["max_retries"] + 1):
            rc, Xn, info = O.newton_step(X, cb, dt)
            if rc == 0:
                break
            dt /= 2 ** 0.5
            zeta *= 2.0
        if rc != 0:
            raise RuntimeError("oracle step failed (%d)" % rc)
        Eprev, E = E, O.energy(Xn, cb)
        dt_prev, X = dt, Xn
        el = time.perf_counter() - t0
        if st >= warmup:
            secs.append(el)
            infos.append(info)
    return secs, infos, t_setup, oracle.num_threads()


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "hardware")):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(name, steps=2):
    cfg, side = cpu_sample_config(name)
    N = int(np.prod(cfg["n"]))
    secs, infos, t_setup, thr = oracle_steps(cfg, 0, steps)
    v = N * len(secs) / sum(secs)
    out = {"value": v, "unit": METRIC, "cores": thr, "kind": "oracle",
           "sample": ("%d real FP64 oracle time steps (all %d host threads, OpenMP) of the workload's recipe on a "
                      "periodic %s grid (%d points, the workload's Schwarz box size: %s); %.1f s of steps, "
                      "%.1f s equilibrium set-up untimed; %.1f Newton, %.0f GMRES per step; the full-size grid has "
                      "more boxes per axis and needs more GMRES iterations per Newton solve"
                      % (len(secs), thr, "x".join(str(v) for v in cfg["n"]), N, cfg["desc"].split("[")[-1].rstrip("]")
                         if side else "the workload itself", sum(secs), t_setup,
                         np.mean([i["newton_its"] for i in infos]), np.mean([i["gmres_its"] for i in infos]))),
           "nproc": os.cpu_count(), "cpu_model": cpu_model()}
    # one thread on the small 2-D workload (64^2, 16^2 boxes), for the per-core rate
    import oracle
    try:
        secs1, infos1, _, thr1 = oracle_steps(S.CONFIGS["2d64"], 0, 2, threads=1)
        out["single_thread_2d64"] = {"value": 4096 * len(secs1) / sum(secs1), "unit": METRIC, "cores": thr1,
                                     "sample": "2 real oracle steps of the 2-D 64^2 workload on one thread"}
    finally:
        oracle.set_threads(0)
    return out


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------

def timed_run(P, steps, warmup, stream, dts=None):
    """W warm-up steps (state restored afterwards), then K steps between CUDA
    events on the solver's stream (dts: replay those step sizes)."""
    import torch
    state0 = P.get_state()
    for i in range(warmup):
        P.step(dts[i] if dts and i < len(dts) else 0.0)
    P.set_state(state0)
    P.reset_stats()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    infos = [P.step(dts[i] if dts else 0.0) for i in range(steps)]
    ev1.record(stream)
    torch.cuda.synchronize()
    return ev0.elapsed_time(ev1), infos


def golden_accuracy(nks, name, cfg, op, stream, alloc):
    """Per-field error against the full-size FP64 oracle reference of the
    workload (tests/golden/full_<workload>.json, written by the oracle alone):
    both GPU solvers replay the oracle's dt sequence for its steps; the relative
    L2 error per field is estimated from the reference's 256-row sign sketch,
    and the error at its 1024 sampled points is exact."""
    path = os.path.join(ROOT, "tests", "golden", "full_%s.json" % name)
    if not os.path.exists(path):
        return None
    G = json.load(open(path))
    dts = [s["dt"] for s in G["per_step"]]
    c, e = S.config_fields(cfg)
    idx = np.array(G["samples"]["index"], dtype=np.int64)
    out = {"reference": "FP64 oracle, %d steps of the full-size workload (dt replayed), %s; both GPU solvers at its "
                        "Newton tolerance %.0e" % (len(dts), G["_source"], G["newton_rtol"]),
           "estimator": "relative L2 from a %d-row seeded sign sketch (Johnson-Lindenstrauss; the estimate lies "
                        "within a factor 0.7..1.3 of the true value with probability > 1 - 1e-6); max relative "
                        "error over %d sampled points" % (G["sketch"]["k"], idx.size)}
    for prec in ("mixed", "fp64"):
        # at the reference's Newton tolerance: the workload's own leaves the 1024^2 displacement
        # settled only to a few 1e-7 (its rows carry about 1e-12 of the residual norm)
        Q = nks.Problem(cfg["dim"], cfg["n"], cfg["h"], c, e, S.config_coefficients(cfg),
                        dict(op, precision=prec, newton_rtol=G["newton_rtol"]), stream=stream.cuda_stream,
                        allocator=alloc)
        infos = [Q.step(dt) for dt in dts]
        fl = field_dict(*Q.get_fields())
        Q.destroy()
        sk = S.sign_sketch([fl[f] for f in G["fields"]], G["sketch"]["k"], G["sketch"]["seed"])
        r = {}
        for i, f in enumerate(G["fields"]):
            ref = G["fields"][f]
            scale = ref["norm"] / np.sqrt(fl[f].size)
            r[f] = {"rel_l2_est": float(np.linalg.norm(sk[i] - np.array(ref["sketch"])) / ref["norm"]),
                    "max_rel_at_samples": float(np.max(np.abs(fl[f][idx] - np.array(ref["at_samples"]))) / scale)}
        r["energy_rel"] = max(abs(i["energy"] - s["energy"]) / abs(s["energy"]) for i, s in zip(infos, G["per_step"]))
        r["mass_rel"] = max(abs(i["mass"] - s["mass"]) / abs(s["mass"]) for i, s in zip(infos, G["per_step"]))
        r["max_rel_l2_est"] = max(r[f]["rel_l2_est"] for f in G["fields"])
        out[prec] = r
    out["tolerance"] = 1e-8
    out["within_tolerance"] = all(out[p]["max_rel_l2_est"] <= 1e-8 for p in ("mixed", "fp64"))
    return out


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

    cfg = workload(args.config, args.grid)
    op = S.options(**cfg["opts"])
    prec = args.precision or "mixed"
    op["precision"] = prec
    if args.variant:
        op["ras_variant"] = args.variant
    if args.overlap is not None:
        op["overlap"] = args.overlap
    if args.sub:
        op["sub"] = tuple(int(v) for v in args.sub.split(","))
        args.no_accuracy = True
    if args.u0_maxit is not None:
        op["u0_maxit"] = args.u0_maxit
    if args.gmres_maxit is not None:
        op["gmres_maxit"] = args.gmres_maxit
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
    dev = torch.device("cuda", local)
    pk = peaks()

    def create(o, timing=False):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        P = nks.Problem(cfg["dim"], cfg["n"], cfg["h"], c, e, S.config_coefficients(cfg), o,
                        stream=stream.cuda_stream, allocator=alloc, timing=timing)
        torch.cuda.synchronize()
        sst = P.get_stats()
        return P, {"seconds": time.perf_counter() - t0, "u0_newton_its": sst["newton_its"],
                   "u0_gmres_its": sst["gmres_its"], "device_bytes": P.device_bytes(),
                   "includes": "problem creation: plan, factor tables, upload, initial mechanical equilibrium "
                               "(Newton on the displacement rows, tolerance u0_rtol)"}

    def instrumented(o, dts):
        """the same K steps (dt replayed) on a problem that times every kernel class with
        CUDA events on its stream (graph replay off): the per-class breakdown"""
        T, _ = create(o, timing=True)
        ms_t, infos_t = timed_run(T, args.steps, args.warmup, stream, dts=dts)
        st = T.get_stats()
        T.destroy()
        return st, ms_t, infos_t

    def summary(P, ms, infos, mixed, st, ms_t, infos_t):
        kernels = kernel_rates(st, cfg, mixed, pk)
        total_ms = sum(st["ms"].values())
        return {
            "value": sum_over_ranks(dist, float(N * len(infos)), dev) / (max_over_ranks(dist, ms, dev) / 1e3),
            "ms_per_step": max_over_ranks(dist, ms, dev) / len(infos),
            "roofline": roofline(st, kernels, mixed, pk, args.config, args.grid, "mixed" if mixed else "fp64"),
            "kernels": kernels,
            "kernel_time_share": {k: round(v / max(total_ms, 1e-9), 4) for k, v in st["ms"].items() if v > 0},
            "instrumented": {"ms_per_step": ms_t / len(infos_t),
                             "same_iterations": [(i["newton_its"], i["gmres_its"]) for i in infos] ==
                                                [(i["newton_its"], i["gmres_its"]) for i in infos_t],
                             "about": "roofline, kernels and kernel_time_share come from a replay of the same K "
                                      "steps (dt replayed) with CUDA events around every kernel class on the "
                                      "solver's stream and graph replay off; value and ms_per_step from the run "
                                      "as a user runs it (GMRES iterations replayed from CUDA graphs)"},
            "iterations": {"newton_per_step": sum(i["newton_its"] for i in infos) / max(len(infos), 1),
                           "gmres_per_step": sum(i["gmres_its"] for i in infos) / max(len(infos), 1),
                           "dt": [i["dt"] for i in infos]},
            "gpu_launches": int(P.get_stats()["kernel_launches"])}

    # --- the headline solver: K timed steps from the initial state ---------------
    P, setup = create(op)
    clocks = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    clocks.start()
    ms, infos = timed_run(P, args.steps, args.warmup, stream)
    clk = clocks.stop()
    if dist is not None:
        dist.barrier()
    mixed = prec == "mixed"
    dts = [i["dt"] for i in infos]
    head = summary(P, ms, infos, mixed, *instrumented(op, dts))
    value = head["value"]

    # --- the FP64 solver beside it on the same steps (same K, W, dt sequence) ---
    fp64 = None
    accuracy = {}
    if mixed and not args.no_fp64:
        Q, qsetup = create(dict(op, precision="fp64"))
        clocks64 = ClockSampler(local)
        clocks64.start()
        ms64, infos64 = timed_run(Q, args.steps, args.warmup, stream, dts=dts)
        clk64 = clocks64.stop()
        fp64 = summary(Q, ms64, infos64, False, *instrumented(dict(op, precision="fp64"), dts))
        fp64.update({"setup": qsetup, "clocks": clk64, "dt_sequence": "replayed from the mixed-precision run",
                     "mixed_over_fp64": value / fp64["value"]})
        fm = field_dict(*P.get_fields())
        fd = field_dict(*Q.get_fields())
        accuracy["vs_fp64_gpu"] = {
            "reference": "FP64 GPU path after the same K steps (same dt sequence)",
            "rel_l2": {f: rel(fm[f], fd[f]) for f in fm}}
        Q.destroy()
    if not args.no_accuracy and rank == 0:
        ga = golden_accuracy(nks, args.config if not args.grid else "-", cfg, op, stream, alloc)
        if ga:
            accuracy["vs_oracle"] = ga
    accuracy["tolerance"] = 1e-8

    # --- end to end through the public API with host buffers ---------------------
    e2e = None
    if not args.no_e2e:
        cpin = torch.from_numpy(c).pin_memory().numpy()
        epin = torch.from_numpy(np.ascontiguousarray(e)).pin_memory().numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        R = nks.Problem(cfg["dim"], cfg["n"], cfg["h"], cpin, epin, S.config_coefficients(cfg), op,
                        stream=stream.cuda_stream, allocator=alloc)
        for _ in range(args.steps):
            R.step()
            R.get_fields()
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        R.destroy()
        t_e2e = max_over_ranks(dist, t_e2e, dev)
        ne, nfr = layout(cfg)
        e2e = {"value": sum_over_ranks(dist, float(N * args.steps), dev) / t_e2e, "unit": METRIC,
               "h2d_bytes_per_step": int((1 + ne) * N * 8 / args.steps), "d2h_bytes_per_step": int(nfr * N * 8),
               "includes": "problem creation from host fields (upload + initial mechanical equilibrium solve), "
                           "K adaptive steps, all fields read back to host after every step"}

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.config)

    out = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32" if mixed else "f64",
        "data": "synthetic (seeded SplitMix64 initial fields)",
        "config": {"workload": cfg["desc"], "precision": prec, "grid": list(cfg["n"]), "points": N,
                   "decomposition": {"sub": list(op["sub"]), "overlap": op["overlap"],
                                     "schwarz": op.get("ras_variant", "left-ras")},
                   "steps_in_workload": cfg["steps"],
                   "timed_steps": "steps 1..K of the workload from its initial state",
                   "initial_equilibrium": ("Newton on the displacement rows, FP64 residual to u0_rtol, inner GMRES in "
                                           "the mixed form" if op.get("u0_mixed") else
                                           "Newton on the displacement rows in the solver's precision"),
                   "l2": "inputs larger than L2: the working set (state, Krylov basis, Schwarz factors; %.1f GB) is "
                         "far above the 129 MB L2" % (setup["device_bytes"] / 1e9),
                   "parallelism": "replicas" if ws > 1 else "single GPU"},
        "gpu_launches": head["gpu_launches"],
        "setup": setup,
        "autotune": tuned,
        "roofline": head["roofline"],
        "kernels": head["kernels"],
        "kernel_time_share": head["kernel_time_share"],
        "instrumented": head["instrumented"],
        "iterations": head["iterations"],
        "fp64": fp64,
        "accuracy": accuracy,
        "clocks": clk,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    P.destroy()
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_reference(args):
    """The oracle (the paper's method in plain FP64 C) on the host cores: W
    warm-up and K timed real time steps of the bounded sample of the workload."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    cfg, side = cpu_sample_config(args.config)
    N = int(np.prod(cfg["n"]))
    secs, infos, t_setup, thr = oracle_steps(cfg, args.warmup, args.steps)
    step_s = sum(secs) / len(secs)
    v = N / step_s
    sample = ("%d real FP64 oracle time steps after %d warm-up steps (all %d host threads, OpenMP) of the workload's "
              "recipe on a periodic %s grid (%d points) with the workload's Schwarz box size; %.1f Newton, %.0f GMRES "
              "per step" % (len(secs), args.warmup, thr, "x".join(str(x) for x in cfg["n"]), N,
                            np.mean([i["newton_its"] for i in infos]), np.mean([i["gmres_its"] for i in infos])))
    full = workload(args.config)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded SplitMix64 initial fields)",
           "config": {"workload": full["desc"], "grid": list(full["n"]), "points": int(np.prod(full["n"])),
                      "sample_grid": list(cfg["n"]), "sample_points": N},
           "cpu_baseline": {"value": v, "unit": METRIC, "cores": thr, "kind": "oracle", "sample": sample,
                            "nproc": os.cpu_count(), "cpu_model": cpu_model()},
           "setup_s": t_setup,
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
    cfg = workload(args.config, args.grid)
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
        srv.destroy()
        return res

    base = S.serving_requests(count=R, seed=4, rate=1.0)
    # saturated rate: the first requests all at once
    nsat = min(R, max(8, R // 4))
    sat = stream_run(base[:nsat], 0.0)
    span = max(r["t_done"] for r in sat) - min(r["t_submit"] for r in sat)
    rate_sat = nsat / max(span, 1e-9)
    rate = 0.8 * rate_sat
    reqs = S.serving_requests(count=R, seed=4, rate=rate)
    clocks = ClockSampler(0)
    clocks.start()
    res = stream_run(reqs, rate)
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="3d128", choices=sorted(S.CONFIGS))
    ap.add_argument("--grid", type=int, default=None,
                    help="run the workload's recipe on a smaller grid of this many cells per axis (same box size)")
    ap.add_argument("--precision", default=None, choices=["fp64", "mixed"],
                    help="the headline solver (default mixed, with the FP64 solver beside it)")
    ap.add_argument("--no-fp64", action="store_true", help="mixed precision without the FP64 solver beside it")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true", help="skip the comparison with the oracle reference")
    ap.add_argument("--batch", type=int, default=0,
                    help="B > 0: B instances of the workload stepped as one batch (beside one alone)")
    ap.add_argument("--serve", action="store_true", help="the serving workload (p50/p99 latency, throughput)")
    ap.add_argument("--variant", default=None, choices=["left-ras", "as", "right-ras"],
                    help="Schwarz preconditioner type (default: the workload's, left-RAS)")
    ap.add_argument("--overlap", type=int, default=None, help="override the workload's Schwarz overlap delta")
    ap.add_argument("--sub", default=None,
                    help="override the workload's subdomains per axis, e.g. 8,8,16 (the oracle comparison is skipped)")
    ap.add_argument("--gmres-maxit", type=int, default=None, help="override the GMRES iteration cap per solve")
    ap.add_argument("--u0-maxit", type=int, default=None,
                    help="Newton iterations allowed to the initial mechanical equilibrium (set-up, not timed)")
    ap.add_argument("--autotune", action="store_true",
                    help="pick the Schwarz decomposition with nks_autotune before timing")
    ap.add_argument("--requests", type=int, default=64, help="--serve: requests in the stream")
    ap.add_argument("--req-steps", type=int, default=10, help="--serve: time steps per request")
    ap.add_argument("--slots", type=int, default=16, help="--serve: slots per shape group")
    ap.add_argument("--groups", type=int, default=8, help="--serve: shape groups alive at once")
    args = ap.parse_args()
    if args.batch > 0 and args.impl == "ours":
        run_batch(args)
    elif args.serve and args.impl == "ours":
        run_serve(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
