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
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
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
    peak64, _ = nb.nb_probe_fma_peak(nb.NB_FP64, 4096)
    peak32, _ = nb.nb_probe_fma_peak(nb.NB_FP32, 65536)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def run_precision(precision, steps, warmup, timed_eval):
        sim = nb.Simulation(m, x, v, eps=EPS, eta=ETA, dt_min=DT_MIN, dt_max=DT_MAX,
                            precision=precision, time_eval=timed_eval)
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
            _, inter = sim.run((slice_idx + 1) * SLICE)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            slice_idx = (slice_idx + 1) % SLICES
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
            _, inter = sim.run((slice_idx + 1) * SLICE)
            nb.nb_get_state(sim.ctx, hst)
            t1 = time.perf_counter()
            slice_idx = (slice_idx + 1) % SLICES
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

    ms_max = r64["ms"]
    inter_all = r64["interactions"]
    if ws > 1:
        import torch.distributed as dist
        tt = torch.tensor([ms_max], dtype=torch.float64, device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms_max = float(tt.item())
        ii = torch.tensor([inter_all], dtype=torch.float64, device=dev)
        dist.all_reduce(ii, op=dist.ReduceOp.SUM)
        inter_all = float(ii.item())
    value = inter_all / (ms_max * 1e-3)

    # ---- EX on the same slices (shorter); per-precision evaluation kernel rates
    # on the same system (FP32 block-step runs are not used: its force noise
    # makes the interpolated 6th-order derivatives collapse the time steps);
    # and the end-to-end number through the C ABI with host buffers.
    k2 = max(1, min(args.steps, args.other_steps))
    rex = run_precision("ex", k2, args.warmup, False) if not args.only_fp64 else None
    kern = {}
    if not args.only_fp64:
        for prec in ("fp64", "ex", "fp32"):
            kern[prec] = {f"A={a}": eval_rate(nb, torch, dev, m, x, v, prec, a, 2 if a == N else 10)
                          for a in (1024, N)}
    e2e_val, state_bytes = (e2e_run(k2, args.warmup) if not args.only_fp64 else (None, 0))

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
                   "dt_max": DT_MAX, "t_end": T_END, "step": "1/64 N-body time slice",
                   "l2": "flushed (256 MB write) before each timed step",
                   "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "seed": SEED},
        "gflops_79": value * FLOPS_PER_INTERACTION / 1e9,
        "fp64_fma_peak_tflops_measured": peak64 / 1e12,
        "fp32_fma_peak_tflops_measured": peak32 / 1e12,
        "pct_fp64_peak": 100.0 * value * FLOPS_PER_INTERACTION / peak64,
        "roofline": {"bound": "alu", "kernel": "k_eval<FP64, step>",
                     "achieved": None if achieved is None else achieved / 1e12,
                     "peak": peak64 / 1e12, "unit": "TFLOP/s",
                     "peak_source": "FP64 FMA probe (nb_probe_fma_peak) in this run",
                     "frac": None if achieved is None else achieved / peak64,
                     "traffic": None,
                     "avg_launch_ms": eval_avg_ms, "launches": r64["eval_launches"],
                     "share_of_step_time": r64["eval_ms"] / r64["ms"] if r64["ms"] else None,
                     "flops_per_interaction": FLOPS_PER_INTERACTION},
        "precisions": {
            "block_steps": {"f64": value,
                            "ex": None if rex is None else rate(rex),
                            "ex_speedup_vs_f64": None if rex is None else rate(rex) / rate(r64),
                            "f32": "not run: FP32 force noise collapses the 6th-order time steps",
                            "slices_ex": k2},
            "eval_kernel": kern,
        },
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": state_bytes,
                "d2h_bytes_per_step": state_bytes, "steps": k2,
                "api": "nb_set_state(host) + nb_run + nb_get_state(host)"},
        "gpu_launches": r64["kernel_launches"],
        "clocks": clk,
        "wall_s_timed_region": t_wall,
        "dt_underflows": r64["underflows"],
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return out


def eval_rate(nb, torch, dev, m, x, v, precision, A, reps):
    """Evaluation-kernel throughput: A active particles against all N of the
    start-up state (nb_predict then nb_evaluate), CUDA events on the stream."""
    n = len(m)
    sim = nb.Simulation(m, x, v, eps=EPS, eta=ETA, dt_min=DT_MIN, dt_max=DT_MAX,
                        precision=precision)
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


def eval_case(args):
    """--case eval: one evaluation launch size, for kernel profiling."""
    import torch
    from paper_1812_00367_gb300 import build as nbbuild
    from paper_1812_00367_gb300 import ic, nb
    nbbuild.build()
    nb.load()
    dev = torch.device("cuda", 0)
    m, x, v = ic.plummer(args.n, seed=SEED)
    r = eval_rate(nb, torch, dev, m, x, v, args.precision, args.active, args.reps)
    print(json.dumps({"case": "eval", "precision": args.precision, "n": args.n,
                      "active": args.active, **r,
                      "gflops_79": r["interactions_per_s"] * FLOPS_PER_INTERACTION / 1e9}))


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
    return {"value": value, "unit": UNIT, "cores": nb_oracle.num_threads(), "kind": "oracle",
            "sample": f"oracle start-up of the same N={N} Plummer system ({t_init:.1f} s, untimed), "
                      f"then its first {steps} block steps ({dt:.1f} s timed)",
            "init_interactions_per_s": inter0 / t_init}


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
    ap.add_argument("--case", choices=["run", "eval"], default="run")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "ex", "fp32"])
    ap.add_argument("--n", type=int, default=N)
    ap.add_argument("--active", type=int, default=N)
    ap.add_argument("--reps", type=int, default=2)
    args = ap.parse_args()
    if args.case == "eval":
        eval_case(args)
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
