"""Benchmark: a/j/s pair interactions per second of the Hermite-6 block-step
hot path on a Plummer sphere of N = 65536 (equal masses, G = M = 1 Henon
units, eps = 1e-4, eta = 0.4, power-of-two steps in [2^-20, 2^-3]) integrated
to t = 0.25, FP64 (the headline), with the EX and FP32 arithmetics measured on
the same workload beside it.

One timed "step" is one slice of 1/64 N-body time units of that integration
(select -> predict -> evaluate -> correct block steps until the slice end);
sixteen slices make the whole t = 0.25 run, after which the start-up state is
restored (a device copy, inside the step) and the slices repeat.  Inputs are
resident in HBM; L2 is flushed (a 256 MB write) before every timed slice,
outside its CUDA-event window.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle
(test infrastructure) on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 65536
EPS = 1e-4
ETA = 0.4
DT_MIN, DT_MAX = 2.0 ** -20, 2.0 ** -3
T_END = 0.25
SLICE = 1.0 / 64
SLICES = int(round(T_END / SLICE))
SEED = 1
FLOPS_PER_INTERACTION = 79  # add/sub/mul = 1, FMA = 2, rsqrt = 1 (stated convention)
METRIC = "a/j/s pair interactions/s"
UNIT = "interactions/s"
WORKLOAD = (f"Plummer N={N}, equal masses, Henon units, eps={EPS:g}, block steps "
            f"dt in [2^-20, 2^-3], eta={ETA}, integrated to t={T_END} in slices of 1/64")

# DRAM traffic of the FP64 step-evaluation kernel, bytes per launch: the mean
# of dram__bytes_read.sum + dram__bytes_write.sum over five consecutive
# k_eval<FP64, step> launches (block steps 301-305 of the 1/64-slice run) of
# one ncu capture of this workload (summary and command in profiles/).  It
# holds for the kernel sources it was taken on (SHA-256 of EVAL_SOURCES
# below); after any change to them it is reported as null.
EVAL_TRAFFIC = {"bytes_per_launch": 7354880, "launches": 5,
                "sources_sha256": "7de9ad53402fc3bce54e3bb2241dc3169b9f7108d3dff80642e0fe229e2193c4"}
EVAL_SOURCES = ("nb_eval.cuh", "nb_eval_fp64.cu", "nb_step.cuh", "nb_internal.cuh")


def eval_sources_sha256() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in EVAL_SOURCES:
        with open(os.path.join(ROOT, "paper_1812_00367_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def eval_traffic():
    """Measured bytes per launch if the kernel is unchanged since, else None."""
    if EVAL_TRAFFIC["bytes_per_launch"] is None:
        return None
    return EVAL_TRAFFIC["bytes_per_launch"] if eval_sources_sha256() == EVAL_TRAFFIC["sources_sha256"] else None


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def emit(obj, rank):
    if rank == 0:
        print(json.dumps(obj), flush=True)


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        import tempfile
        self.path = os.path.join(tempfile.gettempdir(), f"nb_clocks_{os.getpid()}_{id(self)}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
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
        self.fh.close()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); smax.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "power_w_median": statistics.median(power), "samples": len(sm),
                "reasons": sorted(reasons)}


# ------------------------------------------------------------ GPU arm
def gpu_arm(args, ws, rank, local):
    import torch
    from paper_1812_00367_gb300 import build as nbbuild
    from paper_1812_00367_gb300 import ic, nb

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    nbbuild.build()
    nb.load()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)

    m, x, v = ic.plummer(N, seed=SEED)

    def probe_peaks():
        """Best of five runs of each FMA probe."""
        p64 = max(nb.nb_probe_fma_peak(nb.NB_FP64, 8192)[0] for _ in range(5))
        p32 = max(nb.nb_probe_fma_peak(nb.NB_FP32, 65536)[0] for _ in range(5))
        return p64, p32

    peak64, peak32 = probe_peaks()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    import tempfile
    tune_dir = tempfile.mkdtemp(prefix="nbtune_")

    def tune(sim, precision):
        """The autotuner picks lanes-per-i and splits per active-set size
        before anything is timed (one table per arithmetic for this run)."""
        if not args.no_autotune:
            sim.autotune(os.path.join(tune_dir, f"{precision}.txt"))

    def run_precision(precision, steps, warmup, timed_eval):
        sim = nb.Simulation(m, x, v, eps=EPS, eta=ETA, dt_min=DT_MIN, dt_max=DT_MAX,
                            precision=precision, time_eval=timed_eval)
        tune(sim, precision)
        snap = {k: t.clone() for k, t in sim.buf.items()}
        stream = torch.cuda.current_stream(dev)

        def restore():
            for k, t in sim.buf.items():
                t.copy_(snap[k])

        slice_idx = 0
        inter_tot, ms_tot, ev_ms, ev_n, launches = 0.0, 0.0, 0.0, 0, 0
        for k in range(warmup + steps):
            timed = k >= warmup
            if timed:
                flush.zero_()
            c0 = sim.counters() if timed else None
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if slice_idx == 0 and k > 0:
                restore()
            _, inter = sim.run((slice_idx + 1) * args.slice)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            slice_idx = (slice_idx + 1) % int(round(T_END / args.slice))
            if timed:
                c1 = sim.counters()
                ms_tot += e0.elapsed_time(e1)
                inter_tot += inter
                ev_ms += c1["eval_ms"] - c0["eval_ms"]
                ev_n += c1["eval_launches"] - c0["eval_launches"]
                launches += c1["kernel_launches"] - c0["kernel_launches"]
        c = sim.counters()
        sim.close()
        return {"interactions": inter_tot, "ms": ms_tot, "eval_ms": ev_ms, "eval_launches": ev_n,
                "kernel_launches": launches, "underflows": c["dt_underflows"]}

    def e2e_run(steps, warmup):
        """Same slices through the public C ABI with HOST buffers: each step copies
        the state in from pinned host memory, runs the slice, copies it back."""
        sim = nb.Simulation(m, x, v, eps=EPS, eta=ETA, dt_min=DT_MIN, dt_max=DT_MAX,
                            precision="fp64")
        tune(sim, "fp64")
        host0 = {}
        for f, t in sim.buf.items():
            host0[f] = torch.empty(t.shape, dtype=t.dtype, pin_memory=True)
            host0[f].copy_(t)
        host = {f: torch.empty_like(t).pin_memory() for f, t in host0.items()}
        for f in host:
            host[f].copy_(host0[f])
        hst = nb.nb_state(*[nb.C.c_void_p(host[f].data_ptr()) for f in nb.STATE_FIELDS])
        nbytes = sum(t.numel() * t.element_size() for t in host.values())
        slice_idx = 0
        inter_tot, sec_tot = 0.0, 0.0
        for k in range(warmup + steps):
            timed = k >= warmup
            if timed:
                flush.zero_()
            if slice_idx == 0 and k > 0:
                for f in host:
                    host[f].copy_(host0[f])
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            nb.nb_set_state(sim.ctx, hst)
            _, inter = sim.run((slice_idx + 1) * args.slice)
            nb.nb_get_state(sim.ctx, hst)
            t1 = time.perf_counter()
            slice_idx = (slice_idx + 1) % int(round(T_END / args.slice))
            if timed:
                inter_tot += inter
                sec_tot += t1 - t0
        sim.close()
        return inter_tot / sec_tot, nbytes

    # ---- headline FP64 run
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    t_wall0 = time.perf_counter()
    r64 = run_precision("fp64", args.steps, args.warmup, True)
    barrier()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    # the probes again right after the timed region, at the clocks it ran at;
    # the peak is the larger reading (a cold start can read low)
    p64b, p32b = probe_peaks()
    peak64, peak32 = max(peak64, p64b), max(peak32, p32b)

    from paper_1812_00367_gb300.replicas import combine_timing
    ms_max, inter_all = combine_timing(r64["ms"], r64["interactions"], dev)
    value = inter_all / (ms_max * 1e-3)

    # ---- EX on the same slices (shorter); per-precision evaluation kernel rates
    # on the same system (FP32 block-step runs are not used: its force noise
    # makes the interpolated 6th-order derivatives collapse the time steps);
    # and the end-to-end number through the C ABI with host buffers.
    k2 = max(1, min(args.steps, args.other_steps))
    rex = run_precision("ex", k2, args.warmup, False) if not args.only_fp64 else None
    r32x = run_precision("fp32x", k2, args.warmup, False) if not args.only_fp64 else None
    kern = {}
    if not args.only_fp64:
        for prec in ("fp64", "ex", "fp32x", "fp32"):
            kern[prec] = {f"A={a}": eval_rate(nb, torch, dev, m, x, v, prec, a, 2 if a == N else 10)
                          for a in (1024, N)}
    e2e_val, state_bytes = (e2e_run(k2, args.warmup) if not args.only_fp64 else (None, 0))
    # configurations 1, 3, 4, 5 beside the headline (rank 0 of a replica run)
    configs, samples = (config_suite(nb, torch, dev, flush, peak64, ic)
                        if not (args.only_fp64 or args.no_configs) and rank == 0 else (None, None))

    eval_avg_ms = r64["eval_ms"] / max(r64["eval_launches"], 1)
    # algorithmic flops of the evaluation launches in the timed region
    eval_flops = FLOPS_PER_INTERACTION * r64["interactions"]
    achieved = eval_flops / (r64["eval_ms"] * 1e-3) if r64["eval_ms"] > 0 else None

    def rate(r):
        return r["interactions"] / (r["ms"] * 1e-3)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N, "eps": EPS, "eta": ETA, "dt_min": DT_MIN,
                   "dt_max": DT_MAX, "t_end": T_END, "step": f"{args.slice:g} N-body time slice",
                   "l2": "flushed (256 MB write) before each timed step",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "plan_table": "default" if args.no_autotune else "nb_autotune before timing",
                   "potential": "the FP64 path sums the potential m/r in float-float on the FP32 "
                                "pipe (about 2^-45 per 64-pair tile, FP64 across tiles); a, jerk "
                                "and snap are all FP64",
                   "seed": SEED},
        "gflops_79": value * FLOPS_PER_INTERACTION / 1e9,
        "fp64_fma_peak_tflops_measured": peak64 / 1e12,
        "fp32_fma_peak_tflops_measured": peak32 / 1e12,
        "pct_fp64_peak": 100.0 * value * FLOPS_PER_INTERACTION / peak64,
        "roofline": {"bound": "alu", "kernel": "k_eval<FP64, step>",
                     "achieved": None if achieved is None else achieved / 1e12,
                     "peak": peak64 / 1e12, "unit": "TFLOP/s",
                     "peak_source": "FP64 FMA probe (nb_probe_fma_peak) in this run: best of 5 runs before and 5 after the timed region",
                     "frac": None if achieved is None else achieved / peak64,
                     "traffic": eval_traffic(),
                     "traffic_unit": "DRAM bytes per launch (ncu, mean of 5 launches), null if the kernel changed",
                     "avg_launch_ms": eval_avg_ms, "launches": r64["eval_launches"],
                     "share_of_step_time": r64["eval_ms"] / r64["ms"] if r64["ms"] else None,
                     "flops_per_interaction": FLOPS_PER_INTERACTION},
        "precisions": {
            "block_steps": {"f64": value,
                            "ex": None if rex is None else rate(rex),
                            "ex_speedup_vs_f64": None if rex is None else rate(rex) / rate(r64),
                            "f32x": None if r32x is None else rate(r32x),
                            "f32x_speedup_vs_f64": None if r32x is None else rate(r32x) / rate(r64),
                            "f32x_note": "float-float acceleration and potential, FP32 jerk and snap",
                            "f32": "not run: FP32 acceleration errors (up to 4e-7) collapse the "
                                   "6th-order time steps",
                            "slices_ex_f32x": k2},
            "eval_kernel": kern,
        },
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                "d2h_bytes_per_step": state_bytes, "steps": k2,
                "api": "nb_set_state(host) + nb_run + nb_get_state(host)"},
        "gpu_launches": r64["kernel_launches"],
        "clocks": clk,
        # board power (nvidia-smi, median over the timed region) x time / work
        "energy_nj_per_interaction": (None if not clk.get("power_w_median") else
                                      clk["power_w_median"] * r64["ms"] * 1e-3
                                      / r64["interactions"] * 1e9),
        "wall_s_timed_region": t_wall,
        "dt_underflows": r64["underflows"],
    }
    if configs is not None:
        out["configs"] = configs
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        if samples is not None:
            out["cpu_baseline"]["configs"] = cpu_config_checks(samples)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return out


def eval_rate(nb, torch, dev, m, x, v, precision, A, reps, order=6):
    """Evaluation-kernel throughput: A active particles against all N of the
    start-up state (nb_predict then nb_evaluate), CUDA events on the stream."""
    n = len(m)
    # no start-up evaluations: the launches of this case are the timed ones
    sim = nb.Simulation(m, x, v, eps=EPS, eta=ETA, dt_min=DT_MIN, dt_max=DT_MAX,
                        precision=precision, keep_state=True, order=order)
    sim.predict(0.0, out=False)
    act = torch.arange(A, dtype=torch.int32, device=dev)
    out = torch.empty((10, A), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    nb.nb_evaluate(sim.ctx, 0, act, A, out)          # warm-up launch
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        nb.nb_evaluate(sim.ctx, 0, act, A, out)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    sim.sync()
    sim.close()
    ms = e0.elapsed_time(e1) / reps
    return {"interactions_per_s": A * (n - 1) / (ms * 1e-3), "ms_per_launch": ms}


def _keep_state_sim(nb, m, x, v, a, eps, precision, order=6):
    """A context over (m, x, v) at t = 0 holding the given accelerations
    (they enter the snap terms) with no start-up evaluations of its own."""
    n = len(m)
    sim = nb.Simulation(m, x, v, eps=eps, precision=precision, keep_state=True, order=order)
    st = {"m": m, "x": x, "v": v, "a": a, "j": np.zeros((n, 3)), "s": np.zeros((n, 3)),
          "c": np.zeros((n, 3)), "t": np.zeros(n), "dt": np.full(n, 2.0 ** -6),
          "pot": np.zeros(n)}
    sim.set_state_numpy(st)
    sim.predict(0.0, out=False)
    return sim


def timed_evals(nb, torch, dev, sim, n, actives, flush, keep_largest=True):
    """Evaluation-kernel rate of each active-set size: the active particles are
    spread evenly over the index range; L2 is flushed before every timed
    launch (CUDA events on the stream around the launches only).  Returns the
    rates and, for the largest size, its index list and outputs (host)."""
    stream = torch.cuda.current_stream(dev)
    res, kept = {}, None
    for A in actives:
        idx = np.linspace(0, n - 1, A).astype(np.int32)
        act = torch.as_tensor(idx, device=dev)
        o = torch.empty((10, A), dtype=torch.float64, device=dev)
        nb.nb_evaluate(sim.ctx, 0, act[:min(A, 1024)], min(A, 1024), o)   # warm-up
        reps = 5 if A <= 4096 else 1
        ms = 0.0
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            nb.nb_evaluate(sim.ctx, 0, act, A, o)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms += e0.elapsed_time(e1)
        ms /= reps
        res[f"A={A}"] = {"interactions_per_s": A * (n - 1) / (ms * 1e-3), "ms_per_launch": ms}
        if keep_largest and A == max(actives):
            kept = (idx, o.cpu().numpy())
    sim.sync()
    return res, kept


def config_suite(nb, torch, dev, flush, peak64, ic):
    """Configurations 1, 3, 4 and 5 beside the headline (configuration 2):
    GPU rates, each FP64 rate also as a fraction of the measured DFMA peak.
    Returns (results, samples): the samples are what the CPU-baseline leg
    evaluates with the oracle (timed) and compares."""
    out, samples = {}, {}
    rng = np.random.default_rng(2024)

    # -- configuration 1: Plummer N=1024, eps 1e-4, one full evaluation and 16
    # shared steps of 1/256 (FP64)
    n1, eps1, h1 = 1024, 1e-4, 1.0 / 256
    m1, x1, v1 = ic.plummer(n1, seed=1)
    r_eval = eval_rate(nb, torch, dev, m1, x1, v1, "fp64", n1, 50)
    sim = nb.Simulation(m1, x1, v1, eps=eps1, precision="fp64", dt_min=h1, dt_max=h1)
    E0 = sim.energy(0.0)
    flush.zero_()
    steps, inter, sec = _timed_run(sim, torch, dev, 16 * h1)
    E1 = sim.energy(16 * h1)
    st1 = sim.state_numpy()
    sim.close()
    out["c1_plummer_n1024"] = {
        "workload": "Plummer N=1024, eps=1e-4, FP64: one all-active evaluation; 16 shared steps dt=1/256",
        "eval_interactions_per_s": r_eval["interactions_per_s"],
        "eval_frac_of_fp64_peak": r_eval["interactions_per_s"] * FLOPS_PER_INTERACTION / peak64,
        "shared_steps": steps, "ms_per_shared_step": 1e3 * sec / steps,
        "step_interactions_per_s": inter / sec,
        "rel_energy_change": abs((E1[0] + E1[1]) - (E0[0] + E0[1])) / abs(E0[0] + E0[1]),
        "dP": float(np.linalg.norm(E1[2] - E0[2]))}
    samples["c1"] = {"m": m1, "x0": x1, "v0": v1, "eps": eps1, "h": h1, "x": st1["x"],
                     "v": st1["v"], "E0": E0[0] + E0[1], "E1": E1[0] + E1[1]}

    # -- configuration 3: Plummer N=2^20, Kroupa masses, eps 1e-5: a 1/16
    # slice of the full evaluation in FP64, the full evaluation in EX and FP32
    n3, eps3 = 1 << 20, 1e-5
    m3, x3, v3 = ic.plummer(n3, seed=3, masses=ic.kroupa_masses(n3, seed=3))
    a3 = rng.normal(size=(n3, 3)) * 0.3
    c3 = {"workload": "Plummer N=2^20, Kroupa-like masses (0.1-100), eps=1e-5: all-active "
                      "evaluation (FP64: 65536 active, 1/16 of it)"}
    samples["c3"] = {"m": m3, "x": x3, "v": v3, "a": a3, "eps": eps3, "gpu": {}}
    for prec in ("fp64", "ex", "fp32x", "fp32"):
        A = 65536 if prec == "fp64" else n3
        sim = _keep_state_sim(nb, m3, x3, v3, a3, eps3, prec)
        rates, (idx, o) = timed_evals(nb, torch, dev, sim, n3, (A,), flush)
        sim.close()
        c3[prec] = rates
        pick = np.sort(rng.choice(len(idx), 256, replace=False))
        samples["c3"]["gpu"][prec] = (idx[pick], o[:, pick])
    c3["fp64_frac_of_fp64_peak"] = (c3["fp64"]["A=65536"]["interactions_per_s"]
                                   * FLOPS_PER_INTERACTION / peak64)
    c3["ex_speedup_vs_fp64"] = (c3["ex"][f"A={n3}"]["interactions_per_s"]
                                / c3["fp64"]["A=65536"]["interactions_per_s"])
    out["c3_kroupa_plummer_n2p20"] = c3
    del m3, x3, v3

    # -- configuration 4: 512 Plummer clusters, N log-uniform in [256, 16384],
    # eps 1e-4: start-up, block steps to t = 1/256 (untimed), then a timed
    # window of 1/256 of block steps of every cluster, graph-replayed
    batch = ic.plummer_batch(512, seed=1)
    c4 = {"workload": "512 Plummer clusters, N log-uniform in [256, 16384] (sum "
                      f"{int(batch.offsets[-1])}), eps=1e-4, own block steps per cluster; timed "
                      "window t = 1/256 .. 2/256", "clusters": 512,
          "n_total": int(batch.offsets[-1])}
    sizes = batch.sizes
    order = np.argsort(sizes)
    csample = sorted({int(order[-1]), int(order[0]), *rng.choice(512, 6, replace=False).tolist()})
    samples["c4"] = {"batch": batch, "eps": 1e-4, "clusters": csample, "gpu": {}}
    for prec in ("fp64", "ex"):
        sim = nb.Simulation(batch.m, batch.x, batch.v, eps=1e-4, eta=ETA, dt_min=DT_MIN,
                            dt_max=DT_MAX, precision=prec, offsets=batch.offsets)
        st = sim.state_numpy()
        samples["c4"]["gpu"][prec] = {f: st[f] for f in ("a", "j", "s", "pot")}
        t0, t1 = 1.0 / 256, 2.0 / 256
        sim.run(t0)
        e0 = sim.energy_all(t0)[:, :2].sum(axis=1)
        flush.zero_()
        steps, inter, sec = _timed_run(sim, torch, dev, t1)
        e1 = sim.energy_all(t1)[:, :2].sum(axis=1)
        sim.close()
        drift = np.abs(e1 - e0) / np.abs(e0) / (t1 - t0)
        c4[prec] = {"interactions_per_s": inter / sec, "seconds": sec, "cluster_block_steps": steps,
                    "interactions": inter,
                    "energy_drift_per_time_max": float(drift.max()),
                    "energy_drift_per_time_median": float(np.median(drift))}
    c4["fp64_frac_of_fp64_peak"] = c4["fp64"]["interactions_per_s"] * FLOPS_PER_INTERACTION / peak64
    c4["ex_speedup_vs_fp64"] = c4["ex"]["interactions_per_s"] / c4["fp64"]["interactions_per_s"]
    out["c4_batched_512"] = c4

    # -- configuration 5: two Hernquist spheres of 2^21 each, eps 1e-3:
    # evaluation of 64, 1024 and 65536 active particles against all 4,194,304
    m5, x5, v5 = ic.hernquist_merger(1 << 21, seed=5)
    n5 = len(m5)
    a5 = rng.normal(size=(n5, 3)) * 0.1
    c5 = {"workload": "two Hernquist spheres 2 x 2^21 on a parabolic orbit at separation 20, "
                      "eps=1e-3: A active (evenly spread) against all 4,194,304"}
    samples["c5"] = {"m": m5, "x": x5, "v": v5, "a": a5, "eps": 1e-3, "gpu": {}}
    for prec, acts in (("fp64", (64, 1024, 65536)), ("ex", (64, 1024, 65536)),
                       ("fp32x", (65536,)), ("fp32", (65536,))):
        sim = _keep_state_sim(nb, m5, x5, v5, a5, 1e-3, prec)
        rates, (idx, o) = timed_evals(nb, torch, dev, sim, n5, acts, flush)
        sim.close()
        c5[prec] = rates
        pick = np.sort(rng.choice(len(idx), 64, replace=False))
        samples["c5"]["gpu"][prec] = (idx[pick], o[:, pick])
    c5["fp64_frac_of_fp64_peak"] = {k: r["interactions_per_s"] * FLOPS_PER_INTERACTION / peak64
                                    for k, r in c5["fp64"].items()}
    c5["ex_speedup_vs_fp64"] = (c5["ex"]["A=65536"]["interactions_per_s"]
                                / c5["fp64"]["A=65536"]["interactions_per_s"])
    out["c5_hernquist_merger_n4194304"] = c5
    return out, samples


def _rel_errs(out, ref):
    acc, jrk, snp, pot = ref
    e = {}
    for name, lo, r in (("a", 0, acc), ("j", 3, jrk), ("s", 6, snp)):
        d = np.linalg.norm(out[lo:lo + 3].T - r, axis=1) / np.linalg.norm(r, axis=1)
        e[name] = float(d.max())
    e["pot"] = float((np.abs(out[9] - pot) / np.abs(pot)).max())
    return e


def cpu_config_checks(samples):
    """CPU-baseline leg of configurations 1, 3, 4, 5: the oracle, as it stands,
    on the host cores over a bounded sample of each workload (timed:
    interactions/s), and the largest relative difference of the GPU's results
    from the oracle's on that same sample (a, jerk, snap, potential; per
    arithmetic)."""
    from oracle import nb_oracle
    nb_oracle.build()
    res = {}
    c = samples["c1"]
    t0 = time.perf_counter()
    ref = nb_oracle.Sim(c["m"], c["x0"], c["v0"], eps=c["eps"], dt_min=c["h"], dt_max=c["h"]).init()
    r0 = ref.energy(0.0)
    ref.run(16 * c["h"])
    sec = time.perf_counter() - t0
    r1 = ref.energy(16 * c["h"])
    ex = np.linalg.norm(c["x"] - ref.x, axis=1) / np.linalg.norm(ref.x, axis=1)
    ev = np.linalg.norm(c["v"] - ref.v, axis=1) / np.linalg.norm(ref.v, axis=1)
    res["c1"] = {"sample": "the whole run: start-up and 16 shared steps",
                 "interactions_per_s": ref.interactions / sec, "seconds": sec,
                 "gpu_vs_oracle": {"x_max_rel": float(ex.max()), "v_max_rel": float(ev.max()),
                                   "x_median_rel": float(np.median(ex)),
                                   "energy_change_gpu": c["E1"] - c["E0"],
                                   "energy_change_oracle": (r1[0] + r1[1]) - (r0[0] + r0[1])}}
    for key in ("c3", "c5"):
        c = samples[key]
        idx = next(iter(c["gpu"].values()))[0]
        errs, sec, ninter = {}, 0.0, 0.0
        refs = {}
        for prec, (ix, o) in c["gpu"].items():
            k = tuple(ix.tolist())
            if k not in refs:
                t0 = time.perf_counter()
                refs[k] = nb_oracle.force(c["m"], c["x"], c["v"], c["a"], c["eps"], active=ix)
                sec += time.perf_counter() - t0
                ninter += len(ix) * (len(c["m"]) - 1)
            errs[prec] = _rel_errs(o, refs[k])
        res[key] = {"sample": f"{len(idx)} active particles (per arithmetic, from its largest "
                              f"timed set) against all {len(c['m'])}",
                    "interactions_per_s": ninter / sec, "seconds": sec,
                    "gpu_vs_oracle_max_rel": errs}
    c = samples["c4"]
    b = c["batch"]
    errs = {p: {"a": 0.0, "j": 0.0, "s": 0.0, "pot": 0.0} for p in c["gpu"]}
    sec, ninter = 0.0, 0.0
    for k in c["clusters"]:
        lo, hi = b.offsets[k], b.offsets[k + 1]
        t0 = time.perf_counter()
        ref = nb_oracle.Sim(b.m[lo:hi], b.x[lo:hi], b.v[lo:hi], eps=c["eps"]).init()
        sec += time.perf_counter() - t0
        ninter += ref.interactions
        for prec, g in c["gpu"].items():
            for f in ("a", "j", "s"):
                d = (np.linalg.norm(g[f][lo:hi] - getattr(ref, f), axis=1)
                     / np.linalg.norm(getattr(ref, f), axis=1))
                errs[prec][f] = max(errs[prec][f], float(d.max()))
            d = np.abs(g["pot"][lo:hi] - ref.pot) / np.abs(ref.pot)
            errs[prec]["pot"] = max(errs[prec]["pot"], float(d.max()))
    res["c4"] = {"sample": f"start-up (two passes) of {len(c['clusters'])} clusters "
                           "(the largest, the smallest, six at random)",
                 "interactions_per_s": ninter / sec, "seconds": sec,
                 "gpu_vs_oracle_max_rel": errs}
    return res


def eval_case(args):
    """--case eval: one evaluation launch size, for kernel profiling."""
    import torch
    from paper_1812_00367_gb300 import build as nbbuild
    from paper_1812_00367_gb300 import ic, nb
    nbbuild.build()
    nb.load()
    dev = torch.device("cuda", 0)
    m, x, v = ic.plummer(args.n, seed=SEED)
    r = eval_rate(nb, torch, dev, m, x, v, args.precision, args.active, args.reps,
                  order=args.order)
    print(json.dumps({"case": "eval", "precision": args.precision, "n": args.n,
                      "active": args.active, "order": args.order, **r,
                      "gflops_79": r["interactions_per_s"] * FLOPS_PER_INTERACTION / 1e9}))


def _timed_run(sim, torch, dev, t_end):
    stream = torch.cuda.current_stream(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(stream)
    steps, inter = sim.run(t_end)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    return steps, inter, e0.elapsed_time(e1) * 1e-3


def batched_case(args):
    """512 independent Plummer clusters, N log-uniform in [256, 16384], eps 1e-4,
    each on its own block steps, all advanced together (one persistent
    evaluation launch per block step, graph-replayed): FP64 and EX."""
    import torch
    from paper_1812_00367_gb300 import build as nbbuild
    from paper_1812_00367_gb300 import ic, nb
    nbbuild.build()
    nb.load()
    dev = torch.device("cuda", 0)
    batch = ic.plummer_batch(args.clusters, seed=SEED)
    out = {"case": "batched", "clusters": args.clusters, "n_total": int(batch.offsets[-1]),
           "n_min": int(batch.sizes.min()), "n_max": int(batch.sizes.max()), "eps": EPS,
           "t_warm": args.t_warm, "t_end": args.t_warm + args.t_run}
    for prec in ("fp64", "ex"):
        sim = nb.Simulation(batch.m, batch.x, batch.v, eps=EPS, eta=ETA, dt_min=DT_MIN,
                            dt_max=DT_MAX, precision=prec, offsets=batch.offsets)
        if args.batched_target > 0:   # one split target for every active-set size
            import tempfile
            path = os.path.join(tempfile.mkdtemp(), "table.txt")
            with open(path, "w") as f:
                f.write(f"nbtune {nb.PRECISIONS[prec]} 0\n")
                for b in range(32):
                    gl = 32 if b < 6 else (8 if b < 10 else (2 if b < 12 else 1))
                    f.write(f"{gl} {args.batched_target}\n")
            sim.autotune(path)
            out["batched_target"] = args.batched_target
        e0 = list(sim.energy_all(0.0)[:, :2].sum(axis=1))
        sim.run(args.t_warm)
        steps, inter, sec = _timed_run(sim, torch, dev, args.t_warm + args.t_run)
        t1 = args.t_warm + args.t_run
        e1 = list(sim.energy_all(t1)[:, :2].sum(axis=1))
        drift = [abs(b - a) / abs(a) / t1 for a, b in zip(e0, e1)]
        out[prec] = {"interactions_per_s": inter / sec, "seconds": sec, "cluster_block_steps": steps,
                     "interactions": inter, "energy_drift_per_time_max": max(drift),
                     "energy_drift_per_time_median": statistics.median(drift)}
        sim.close()
    out["ex_speedup_vs_f64"] = out["ex"]["interactions_per_s"] / out["fp64"]["interactions_per_s"]
    print(json.dumps(out))


def config3_case(args):
    """Plummer N = 2^20 with Kroupa-like masses, eps = 1e-5: evaluation
    throughput per arithmetic, a/j/s/pot errors on a 4096-particle subsample
    against the FP64 oracle (whose evaluation of the subsample is timed: this
    case's CPU-baseline leg), and energy drift over a short block-step run."""
    import torch
    from oracle import nb_oracle
    from paper_1812_00367_gb300 import build as nbbuild
    from paper_1812_00367_gb300 import ic, nb
    nbbuild.build()
    nb.load()
    nb_oracle.build()
    dev = torch.device("cuda", 0)
    n, eps = 1 << 20, 1e-5
    masses = ic.kroupa_masses(n, seed=3)
    m, x, v = ic.plummer(n, seed=3, masses=masses)
    rng = np.random.default_rng(3)
    sub = np.sort(rng.choice(n, 4096, replace=False)).astype(np.int32)
    t0 = time.perf_counter()
    ref = nb_oracle.force(m, x, v, np.zeros_like(x), eps, active=sub)
    t_oracle = time.perf_counter() - t0
    out = {"case": "config3", "n": n, "eps": eps, "subsample": len(sub),
           "oracle_seconds_subsample": t_oracle, "oracle_threads": nb_oracle.num_threads()}
    for prec in ("fp64", "ex", "fp32x", "fp32"):
        sim = nb.Simulation(m, x, v, eps=eps, precision=prec, keep_state=True)
        st = {"m": m, "x": x, "v": v, "a": np.zeros((n, 3)), "j": np.zeros((n, 3)),
              "s": np.zeros((n, 3)), "c": np.zeros((n, 3)), "t": np.zeros(n),
              "dt": np.full(n, 2.0 ** -6), "pot": np.zeros(n)}
        sim.set_state_numpy(st)
        sim.predict(0.0, out=False)
        got = sim.evaluate(torch.as_tensor(sub, device=dev)).cpu().numpy()
        errs = {}
        for name, lo, r in (("a", 0, ref[0]), ("j", 3, ref[1]), ("s", 6, ref[2])):
            e = np.linalg.norm(got[lo:lo + 3].T - r, axis=1) / np.linalg.norm(r, axis=1)
            errs[name] = {"max": float(e.max()), "p99.9": float(np.quantile(e, 0.999))}
        e = np.abs(got[9] - ref[3]) / np.abs(ref[3])
        errs["pot"] = {"max": float(e.max()), "p99.9": float(np.quantile(e, 0.999))}
        A = n if (prec != "fp64" or args.c3_full_fp64) else args.c3_active
        act = torch.arange(A, dtype=torch.int32, device=dev)
        o = torch.empty((10, A), dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream(dev)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        nb.nb_evaluate(sim.ctx, 0, act, A, o)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        sec = ev0.elapsed_time(ev1) * 1e-3
        sim.close()
        out[prec] = {"errors": errs, "eval_active": A, "eval_seconds": sec,
                     "interactions_per_s": A * (n - 1) / sec,
                     "gflops_79": A * (n - 1) / sec * FLOPS_PER_INTERACTION / 1e9}
    if args.c3_run_t > 0:
        # "prec" or "prec:4" (the 4th-order scheme, eta 0.02)
        for spec in args.c3_run_precisions.split(","):
            prec, _, order = spec.partition(":")
            order = int(order or 6)
            sim = nb.Simulation(m, x, v, eps=eps, precision=prec, order=order,
                                eta=ETA4 if order == 4 else ETA)
            E0 = sum(sim.energy(0.0)[:2])
            steps, inter, sec = _timed_run(sim, torch, dev, args.c3_run_t)
            E1 = sum(sim.energy(args.c3_run_t)[:2])
            c = sim.counters()
            out.setdefault("block_runs", {})[spec] = {
                "order": order, "t_end": args.c3_run_t, "block_steps": steps,
                "interactions": inter, "interactions_per_s": inter / sec, "seconds": sec,
                "energy_drift_per_time": abs(E1 - E0) / abs(E0) / args.c3_run_t,
                "dt_underflows": c["dt_underflows"]}
            sim.close()
    print(json.dumps(out))


def _lagrangian_radii(m, x, fractions=(0.1, 0.5, 0.9)):
    com = (m[:, None] * x).sum(0) / m.sum()
    r = np.linalg.norm(x - com, axis=1)
    order = np.argsort(r)
    cm = np.cumsum(m[order]) / m.sum()
    return [float(r[order][np.searchsorted(cm, f)]) for f in fractions]


def config2_check(args):
    """The benchmark's integration run to t = 0.25 on the GPU (FP64, EX and
    FP32X by default) and, as this case's CPU-baseline leg, by the oracle
    (timed): block steps, interactions, energy error, momentum and
    Lagrangian radii at the end (block-step runs diverge per particle, so the
    comparison is statistical)."""
    import torch
    from paper_1812_00367_gb300 import build as nbbuild
    from paper_1812_00367_gb300 import ic, nb
    nbbuild.build()
    nb.load()
    dev = torch.device("cuda", 0)
    m, x, v = ic.plummer(N, seed=SEED)
    out = {"case": "config2_check", "n": N, "t_end": T_END}
    for prec in args.c2_precisions.split(","):
        sim = nb.Simulation(m, x, v, eps=EPS, eta=ETA, dt_min=DT_MIN, dt_max=DT_MAX, precision=prec)
        ek0, ep0, P0, L0 = sim.energy(0.0)
        steps, inter, sec = _timed_run(sim, torch, dev, T_END)
        ek1, ep1, P1, L1 = sim.energy(T_END)
        st = sim.state_numpy()
        out[prec] = {"block_steps": steps, "interactions": inter, "seconds": sec,
                     "interactions_per_s": inter / sec,
                     "rel_energy_error": abs((ek1 + ep1) - (ek0 + ep0)) / abs(ek0 + ep0),
                     "dP": float(np.linalg.norm(P1 - P0)), "dL": float(np.linalg.norm(L1 - L0)),
                     "lagrangian_radii_10_50_90": _lagrangian_radii(m, st["x"]),
                     "dt_underflows": sim.counters()["dt_underflows"]}
        sim.close()
    if args.c2_skip_oracle:
        print(json.dumps(out))
        return
    from oracle import nb_oracle
    nb_oracle.build()
    t0 = time.perf_counter()
    ref = nb_oracle.Sim(m, x, v, eps=EPS, eta=ETA, dt_min=DT_MIN, dt_max=DT_MAX).init()
    e0 = ref.energy(0.0)
    ref.run(T_END)
    e1 = ref.energy(T_END)
    sec = time.perf_counter() - t0
    out["oracle"] = {"block_steps": ref.block_steps, "interactions": ref.interactions,
                     "seconds_incl_startup": sec, "threads": nb_oracle.num_threads(),
                     "rel_energy_error": abs((e1[0] + e1[1]) - (e0[0] + e0[1])) / abs(e0[0] + e0[1]),
                     "dP": float(np.linalg.norm(e1[2] - e0[2])), "dL": float(np.linalg.norm(e1[3] - e0[3])),
                     "lagrangian_radii_10_50_90": _lagrangian_radii(m, ref.x),
                     "dt_underflows": ref.underflows}
    print(json.dumps(out))


def merger_case(args):
    """Two Hernquist spheres of 2^21 particles each on a parabolic orbit,
    eps = 1e-3: evaluation throughput of an active subset against all
    4,194,304 particles in FP64 and EX."""
    import torch
    from paper_1812_00367_gb300 import build as nbbuild
    from paper_1812_00367_gb300 import ic, nb
    nbbuild.build()
    nb.load()
    dev = torch.device("cuda", 0)
    m, x, v = ic.hernquist_merger(1 << 21, seed=5)
    n = len(m)
    out = {"case": "merger", "n": n, "eps": 1e-3, "active": args.merger_active}
    for prec in ("fp64", "ex", "fp32"):
        sim = nb.Simulation(m, x, v, eps=1e-3, precision=prec, keep_state=True)
        st = {"m": m, "x": x, "v": v, "a": np.zeros((n, 3)), "j": np.zeros((n, 3)),
              "s": np.zeros((n, 3)), "c": np.zeros((n, 3)), "t": np.zeros(n),
              "dt": np.full(n, 2.0 ** -6), "pot": np.zeros(n)}
        sim.set_state_numpy(st)
        sim.predict(0.0, out=False)
        A = args.merger_active
        act = torch.as_tensor(np.linspace(0, n - 1, A).astype(np.int32), device=dev)
        o = torch.empty((10, A), dtype=torch.float64, device=dev)
        stream = torch.cuda.current_stream(dev)
        nb.nb_evaluate(sim.ctx, 0, act[:1024], 1024, o)   # warm-up
        torch.cuda.synchronize(dev)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        nb.nb_evaluate(sim.ctx, 0, act, A, o)
        ev1.record(stream)
        torch.cuda.synchronize(dev)
        sec = ev0.elapsed_time(ev1) * 1e-3
        sim.close()
        out[prec] = {"interactions_per_s": A * (n - 1) / sec, "seconds": sec,
                     "gflops_79": A * (n - 1) / sec * FLOPS_PER_INTERACTION / 1e9}
    print(json.dumps(out))


def merger_window_case(args):
    """Configuration 5 block steps within a fixed wall-clock window: two
    Hernquist spheres of 2^21 particles each (parabolic orbit, separation 20),
    eps = 1e-3, eta = 0.4, steps in [2^-20, 2^-3], in the given arithmetic.
    Reports the start-up cost separately, then block steps for about
    --window-seconds: block steps, interactions, the time reached, the
    evaluation share of the step time (CUDA events around every evaluation
    launch) and the extrapolation of interactions and time to t = 1 at the
    window's rate."""
    import torch
    from paper_1812_00367_gb300 import build as nbbuild
    from paper_1812_00367_gb300 import ic, nb
    nbbuild.build()
    nb.load()
    dev = torch.device("cuda", 0)
    m, x, v = ic.hernquist_merger(1 << 21, seed=5)
    n = len(m)
    out = {"case": "merger-window", "n": n, "eps": 1e-3, "precision": args.precision,
           "window_seconds_target": args.window_seconds}
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    sim = nb.Simulation(m, x, v, eps=1e-3, eta=ETA, dt_min=DT_MIN, dt_max=DT_MAX,
                        precision=args.precision, time_eval=True)
    torch.cuda.synchronize(dev)
    t_start = time.perf_counter() - t0
    out["startup_seconds"] = t_start
    out["startup_interactions"] = 2.0 * n * (n - 1) if sim.order == 6 else 1.0 * n * (n - 1)
    st = sim.state_numpy()
    dts = st["dt"]
    out["startup_dt_histogram_log2"] = {int(k): int(c) for k, c in
                                        zip(*np.unique(np.log2(dts).astype(int), return_counts=True))}
    stream = torch.cuda.current_stream(dev)
    steps_tot, inter_tot, sec_tot, t_reached = 0, 0.0, 0.0, 0.0
    c0 = sim.counters()
    chunk = 64
    while sec_tot < args.window_seconds:
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        k, inter = sim.run(1.0, chunk)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        sec_tot += e0.elapsed_time(e1) * 1e-3
        steps_tot += k
        inter_tot += inter
        if k == 0:
            break
    c1 = sim.counters()
    st = sim.state_numpy()
    t_reached = float(st["t"].max())   # the last block time taken
    out["end_dt_histogram_log2"] = {int(k): int(c) for k, c in
                                    zip(*np.unique(np.log2(st["dt"]).astype(int), return_counts=True))}
    eval_s = (c1["eval_ms"] - c0["eval_ms"]) * 1e-3
    sim.close()
    out.update({
        "window_seconds": sec_tot, "block_steps": steps_tot, "interactions": inter_tot,
        "interactions_per_s": inter_tot / sec_tot, "t_reached": t_reached,
        "eval_share_of_step_time": eval_s / sec_tot if sec_tot > 0 else None,
        "eval_interactions_per_s": inter_tot / eval_s if eval_s > 0 else None,
        "dt_underflows": c1["dt_underflows"],
        "extrapolated_interactions_to_t1": inter_tot / t_reached if t_reached > 0 else None,
        "extrapolated_seconds_to_t1": sec_tot / t_reached if t_reached > 0 else None})
    print(json.dumps(out))


def histogram_case(args):
    """Configuration 2 (Plummer N=65536, eps 1e-4, eta 0.4, block steps)
    from start-up to t = 0.25 one block step at a time, FP64: the active-set
    histogram in floor(log2 A) buckets with each bucket's block steps,
    interactions, evaluation time (CUDA events around each evaluation launch)
    and interactions/s; the energy error at the end."""
    import torch
    import tempfile
    from paper_1812_00367_gb300 import build as nbbuild
    from paper_1812_00367_gb300 import ic, nb
    nbbuild.build()
    nb.load()
    m, x, v = ic.plummer(N, seed=SEED)
    sim = nb.Simulation(m, x, v, eps=EPS, eta=ETA, dt_min=DT_MIN, dt_max=DT_MAX,
                        precision="fp64", time_eval=True)
    if not args.no_autotune:
        sim.autotune(os.path.join(tempfile.mkdtemp(prefix="nbtune_"), "fp64.txt"))
    e0 = sum(sim.energy(0.0)[:2])
    buckets = {}
    tn, steps = 0.0, 0
    while tn < T_END:
        c0 = sim.counters()["eval_ms"]
        tn, na = sim.step()
        ms = sim.counters()["eval_ms"] - c0
        b = int(math.floor(math.log2(max(na, 1))))
        r = buckets.setdefault(b, [0, 0.0, 0.0, {}])
        r[0] += 1
        r[1] += float(na) * (N - 1)
        r[2] += ms
        r[3][na] = r[3].get(na, 0) + 1
        steps += 1
    e1 = sum(sim.energy(T_END)[:2])
    sim.close()
    rows = [{"log2_active": b, "block_steps": r[0], "interactions": r[1], "eval_ms": r[2],
             "interactions_per_s": r[1] / (r[2] * 1e-3) if r[2] > 0 else None,
             "share_of_interactions": None,
             "most_common_active": sorted(r[3].items(), key=lambda kv: -kv[1])[:4]}
            for b, r in sorted(buckets.items())]
    tot_i = sum(r["interactions"] for r in rows)
    tot_ms = sum(r["eval_ms"] for r in rows)
    for r in rows:
        r["share_of_interactions"] = r["interactions"] / tot_i
    print(json.dumps({"case": "histogram", "n": N, "t_end": T_END, "block_steps": steps,
                      "interactions": tot_i, "eval_seconds": tot_ms * 1e-3,
                      "eval_interactions_per_s": tot_i / (tot_ms * 1e-3),
                      "rel_energy_error": abs(e1 - e0) / abs(e0), "buckets": rows}))


ETA4 = 0.02


def order4_case(args):
    """The 4th-order Hermite variant on the headline workload (Plummer
    N=65536, eps=1e-4, block steps, eta=0.02): block-step throughput from
    t_warm over t_run, its evaluation share (CUDA events inside the graphs),
    the energy drift over the timed run, and the all-active evaluation
    kernel rate, in FP64, EX and FP32; the 6th-order FP64 run beside it."""
    import torch
    from paper_1812_00367_gb300 import build as nbbuild
    from paper_1812_00367_gb300 import ic, nb
    nbbuild.build()
    nb.load()
    dev = torch.device("cuda", 0)
    m, x, v = ic.plummer(N, seed=SEED)
    out = {"case": "order4", "n": N, "eps": EPS, "eta4": ETA4, "eta6": ETA,
           "t_warm": args.t_warm, "t_run": args.t_run}
    runs = [("fp64", 4), ("ex", 4), ("fp32x", 4), ("fp32", 4), ("fp64", 6), ("fp32x", 6)]
    for prec, order in runs:
        sim = nb.Simulation(m, x, v, eps=EPS, eta=ETA4 if order == 4 else ETA, dt_min=DT_MIN,
                            dt_max=DT_MAX, precision=prec, order=order, time_eval=True)
        sim.run(args.t_warm)
        e0 = sum(sim.energy(args.t_warm)[:2])
        c0 = sim.counters()
        steps, inter, sec = _timed_run(sim, torch, dev, args.t_warm + args.t_run)
        c1 = sim.counters()
        e1 = sum(sim.energy(args.t_warm + args.t_run)[:2])
        ev_ms = c1["eval_ms"] - c0["eval_ms"]
        sim.close()
        r = eval_rate(nb, torch, dev, m, x, v, prec, N, 2, order=order)
        out[f"{prec}/order{order}"] = {
            "block_steps": steps, "interactions": inter, "seconds": sec,
            "interactions_per_s": inter / sec,
            "eval_interactions_per_s": inter / (ev_ms * 1e-3) if ev_ms > 0 else None,
            "energy_drift": abs(e1 - e0) / abs(e0),
            "all_active_eval_per_s": r["interactions_per_s"]}
    print(json.dumps(out))


def energy_case(args):
    """Energy per interaction: board power (nvidia-smi, every 200 ms) while the
    all-active evaluation of the Plummer N=65536 system repeats for about
    four seconds, times the CUDA-event time, over the interactions; FP64, EX
    and FP32, 6th- and 4th-order pair terms."""
    import torch
    from paper_1812_00367_gb300 import build as nbbuild
    from paper_1812_00367_gb300 import ic, nb
    nbbuild.build()
    nb.load()
    dev = torch.device("cuda", 0)
    m, x, v = ic.plummer(N, seed=SEED)
    out = {"case": "energy", "n": N, "active": N, "seconds_target": args.energy_seconds}
    stream = torch.cuda.current_stream(dev)
    for prec in ("fp64", "ex", "fp32x", "fp32"):
        for order in (6, 4):
            sim = nb.Simulation(m, x, v, eps=EPS, eta=ETA, dt_min=DT_MIN, dt_max=DT_MAX,
                                precision=prec, keep_state=True, order=order)
            sim.predict(0.0, out=False)
            act = torch.arange(N, dtype=torch.int32, device=dev)
            o = torch.empty((10, N), dtype=torch.float64, device=dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            nb.nb_evaluate(sim.ctx, 0, act, N, o)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            reps = max(2, int(math.ceil(args.energy_seconds / (e0.elapsed_time(e1) * 1e-3))))
            clocks = ClockSampler(0)
            clocks.start()
            time.sleep(0.3)
            e0.record(stream)
            for _ in range(reps):
                nb.nb_evaluate(sim.ctx, 0, act, N, o)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            clk = clocks.stop()
            sim.sync()
            sim.close()
            sec = e0.elapsed_time(e1) * 1e-3
            inter = reps * N * (N - 1)
            p = clk.get("power_w_median")
            out[f"{prec}/order{order}"] = {
                "interactions_per_s": inter / sec, "seconds": sec, "power_w_median": p,
                "nj_per_interaction": None if not p else p * sec / inter * 1e9,
                "sm_mhz": clk.get("sm_mhz"), "reasons": clk.get("reasons"),
                "samples": clk.get("samples")}
    print(json.dumps(out))


# ------------------------------------------------------------ CPU oracle
def _oracle_setup():
    from oracle import nb_oracle
    from paper_1812_00367_gb300 import ic
    nb_oracle.build()
    m, x, v = ic.plummer(N, seed=SEED)
    return nb_oracle, m, x, v


def cpu_baseline(seconds: float):
    """The FP64 oracle, as it stands, on the host cores: its own start-up of
    the same Plummer system, then block steps of the same integration for
    about `seconds` (bounded sample)."""
    nb_oracle, m, x, v = _oracle_setup()
    sim = nb_oracle.Sim(m, x, v, eps=EPS, eta=ETA, dt_min=DT_MIN, dt_max=DT_MAX)
    t0 = time.perf_counter()
    sim.init()
    t_init = time.perf_counter() - t0
    inter0 = sim.interactions
    t1 = time.perf_counter()
    steps = 0
    while time.perf_counter() - t1 < seconds:
        sim.step()
        steps += 1
    dt = time.perf_counter() - t1
    value = (sim.interactions - inter0) / dt
    cores = nb_oracle.num_threads()
    # one core: the oracle's evaluation of 2048 active particles against all
    # N on the current state (a block step of one core could last minutes)
    nb_oracle.set_threads(1)
    act1 = np.arange(0, N, N // 2048, dtype=np.int64)[:2048]
    t2 = time.perf_counter()
    nb_oracle.force(sim.m, sim.x, sim.v, sim.a, EPS, active=act1)
    dt1 = time.perf_counter() - t2
    nb_oracle.set_threads(cores)
    return {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"oracle start-up of the same N={N} Plummer system ({t_init:.1f} s, untimed), "
                      f"then its first {steps} block steps ({dt:.1f} s timed)",
            "value_single_core": len(act1) * (N - 1) / dt1,
            "init_interactions_per_s": inter0 / t_init,
            "single_core": {"value": len(act1) * (N - 1) / dt1, "cores": 1,
                            "sample": f"evaluation of {len(act1)} active particles against all "
                                      f"{N} ({dt1:.1f} s) on one thread"}}


def reference_arm(args, ws, rank):
    """--impl reference: the oracle on this arm's config/metric, on host cores."""
    if rank != 0:
        return None
    nb_oracle, m, x, v = _oracle_setup()
    sim = nb_oracle.Sim(m, x, v, eps=EPS, eta=ETA, dt_min=DT_MIN, dt_max=DT_MAX)
    sim.init()
    per_step = args.ref_interactions
    inter_t, sec_t = 0.0, 0.0
    for k in range(args.warmup + args.steps):
        i0 = sim.interactions
        t0 = time.perf_counter()
        while sim.interactions - i0 < per_step:
            sim.step()
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            inter_t += sim.interactions - i0
            sec_t += dt
    value = inter_t / sec_t
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * sec_t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": N, "eps": EPS, "eta": ETA,
                       "step": f"oracle block steps of the same integration, >= {per_step:.0e} "
                               "interactions per step (bounded sample)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": nb_oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"{args.steps} steps of >= {per_step:.0e} interactions "
                                       "after the oracle's own start-up"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=13)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["native", "reference"], default="native")
    ap.add_argument("--other-steps", type=int, default=4, help="slices timed for EX, FP32, e2e")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--ref-interactions", type=float, default=5e8)
    ap.add_argument("--only-fp64", action="store_true", help="headline run only (profiling)")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the configuration 1/3/4/5 measurements beside the headline")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default plan table")
    ap.add_argument("--slice", type=float, default=SLICE,
                    help="N-body time per step (a power of two dividing 0.25); shorter for profiling")
    ap.add_argument("--case", choices=["run", "eval", "batched", "config3", "merger", "config2-check",
                                       "order4", "energy", "histogram", "merger-window"],
                    default="run")
    ap.add_argument("--clusters", type=int, default=512)
    ap.add_argument("--batched-target", type=int, default=0,
                    help="split target per cluster for --case batched (0: library default)")
    ap.add_argument("--t-warm", type=float, default=1.0 / 256)
    ap.add_argument("--t-run", type=float, default=1.0 / 64)
    ap.add_argument("--c3-active", type=int, default=65536)
    ap.add_argument("--c2-precisions", default="fp64,ex,fp32x", help="--case config2-check")
    ap.add_argument("--c2-skip-oracle", action="store_true",
                    help="--case config2-check: GPU runs only (no CPU-baseline leg)")
    ap.add_argument("--c3-full-fp64", action="store_true")
    ap.add_argument("--c3-run-t", type=float, default=0.0)
    ap.add_argument("--c3-run-precisions", default="ex")
    ap.add_argument("--merger-active", type=int, default=65536)
    ap.add_argument("--precision", default="fp64", choices=["fp64", "ex", "fp32", "fp32x"])
    ap.add_argument("--n", type=int, default=N)
    ap.add_argument("--active", type=int, default=N)
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--energy-seconds", type=float, default=4.0)
    ap.add_argument("--order", type=int, default=6, choices=[4, 6], help="--case eval only")
    ap.add_argument("--window-seconds", type=float, default=300.0, help="--case merger-window")
    args = ap.parse_args()
    if args.case != "run":
        {"eval": eval_case, "batched": batched_case, "config3": config3_case,
         "merger": merger_case, "config2-check": config2_check,
         "order4": order4_case, "energy": energy_case,
         "histogram": histogram_case, "merger-window": merger_window_case}[args.case](args)
        return
    args.warmup = max(args.warmup, 3)
    ws, rank, local = dist_env()
    if args.impl == "reference":
        out = reference_arm(args, ws, rank)
        if out is not None:
            emit(out, rank)
        return
    out = gpu_arm(args, ws, rank, local)
    emit(out, rank)


if __name__ == "__main__":
    main()
