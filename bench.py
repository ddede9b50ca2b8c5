"""Benchmark of the adaptive-resolution WCSPH hot path on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload NAME]

One step = one pass of the method's hot path over the workload's resident
particle state (see WORKLOADS).  Prints ONE JSON line on rank 0.  For N > 1
(torchrun) each rank advances its own independent replica (no data-path
collective; weak scaling); the barrier and the max-over-ranks time are the
only cross-rank operations.

--impl reference times the CPU oracle (the slow FP64 reference program) on
a bounded sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2107_01276_gb300 import workloads as wl  # noqa: E402

# FP32 flops of one pass-B pair evaluation (formula operation count, FMA = 2;
# derivation in the design doc) and of one pass-A pair.
PASS_B_FLOP_PER_PAIR = 90
PASS_A_FLOP_PER_PAIR = 60

WORKLOADS = {
    # pair-kernel sweep shape at N ~ 1M: 2-D periodic square, spacing
    # graded over 1:250 by C_r per column, u,v ~ N(0, 0.1),
    # rho = 1 + U(-0.01, 0.01)
    "graded-1M": dict(kind="graded", n_target=1 << 20, ratio=250.0),
}
DEFAULT_WORKLOAD = "graded-1M"


def make_workload(name):
    w = WORKLOADS[name]
    if w["kind"] == "graded":
        d = wl.graded_strip(n_target=w["n_target"], ratio=w["ratio"])
        desc = ("2-D periodic square, column spacing graded by C_r=1.08 per "
                "column from a fine core to 1:%g, N=%d, h/dx=1.2, "
                "u,v~N(0,0.1), rho=1+U(-0.01,0.01), PEC steps, no "
                "adaptation" % (w["ratio"], len(d["particles"]["x"])))
        return d, desc
    raise KeyError(name)


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed
    region (every 200 ms)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,"
         "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
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


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def fp32_alu_peak_tflops(sm_mhz):
    """Non-tensor FP32 peak: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


# ------------------------------------------------------------ reference --
def cpu_sample(d, frac=0.08, seed=0):
    """A spatial window of the workload (x in a band of width frac*L around
    the middle of the strip) as a standalone non-periodic set: bounded CPU
    work with the same particle shapes."""
    pt = d["particles"]
    L = d["params"]["hi"][0] - d["params"]["lo"][0]
    c = 0.5 * L
    sel = np.abs(pt["x"] - c) < 0.5 * frac * L
    sub = {k: v[sel].copy() for k, v in pt.items()}
    prm = dict(d["params"], periodic=(0, 1))
    return {"particles": sub, "params": prm}, int(sel.sum())


def run_oracle_sample(d, steps, frac):
    import oracle
    sd, n = cpu_sample(d, frac)
    P = oracle.params(**sd["params"])
    st = oracle.make_state(sd["particles"])
    t0 = time.perf_counter()
    oracle.step(P, st, steps)
    el = time.perf_counter() - t0
    return n, el, oracle.num_threads()


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    d, desc = make_workload(args.workload)
    frac = 0.1
    for _ in range(max(args.warmup, 0)):
        run_oracle_sample(d, 1, frac)
    tot_el, tot_ps = 0.0, 0
    for _ in range(args.steps):
        n, el, cores = run_oracle_sample(d, 1, frac)
        tot_el += el
        tot_ps += n
    v = tot_ps / tot_el
    line = {"impl": "reference", "metric": "particle-steps/s", "value": v,
            "unit": "particle-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": desc},
            "cpu_baseline": {"value": v, "unit": "particle-steps/s",
                             "cores": cores, "kind": "oracle",
                             "sample": "window |x-L/2|<%.3gL of the workload "
                                       "(%d particles), 1 PEC step per "
                                       "timed step" % (frac / 2, n)},
            "e2e": {"value": v, "unit": "particle-steps/s",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- ours ----
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    from paper_2107_01276_gb300 import sph

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    sph.lib()
    stream = torch.cuda.current_stream().cuda_stream

    d, desc = make_workload(args.workload)
    pt = d["particles"]
    n = len(pt["x"])

    def new_sim(precision):
        P = sph.make_params(d["params"], precision=precision,
                            capacity=int(n * 1.1) + 16)
        s = sph.Simulation(P, stream)
        s.load(pt)
        return s

    # L2 flush buffer (> 129 MB L2), written between timed steps
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed_steps(sim, K, W):
        for _ in range(W):
            sim.step(1, want_time=False)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True),
                torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        sim.set_timing(True)
        for fam in range(5):
            sim.kernel_time(fam, reset=True)
        l0 = sim.info()["launches"]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        for k in range(K):
            flush.zero_()
            evs[k][0].record()
            sim.step(1, want_time=False)
            evs[k][1].record()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        sim.set_timing(False)
        ms = [a.elapsed_time(b) for a, b in evs]
        fams = [sim.kernel_time(f) for f in range(5)]
        return ms, fams, sim.info()["launches"] - l0

    sim = new_sim(sph.SPH_MIXED)
    clk = ClockSampler(local)
    clk.start()
    ms, fams, nlaunch = timed_steps(sim, args.steps, args.warmup)
    clocks = clk.stop()
    sim.rhs()
    nnb = sim.read("nnb")
    pairs = int(nnb.sum()) - n            # ordered pairs j != i per pass
    info = sim.info()
    launches_per_step = None
    tot_ms = float(np.sum(ms))
    my_time = torch.tensor([tot_ms], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(my_time, op=dist.ReduceOp.MAX)
    tmax = float(my_time.item())
    value = world * n * args.steps / (tmax / 1e3)

    passb_ms, passb_cnt = fams[0]
    passa_ms, passa_cnt = fams[1]
    avg_b = passb_ms / max(passb_cnt, 1)
    sm_mhz = clocks.get("sm_mhz") or 2070.0
    peak_alu = fp32_alu_peak_tflops(2070.0)
    ach_b = PASS_B_FLOP_PER_PAIR * pairs / (avg_b / 1e3) / 1e12
    # launches per step: count of this context's launches over the region
    info2 = sim.info()

    # e2e through the C ABI with pinned host buffers: H2D load of the
    # step's particle state, one PEC step, D2H read of x, y, u, v, p.
    fields_in = ("x", "y", "u", "v", "p", "rho", "m", "h")
    pinned = {k: torch.from_numpy(np.ascontiguousarray(pt[k], np.float64)
                                  ).pin_memory() for k in fields_in}
    src = sph.Particles()
    for k in fields_in:
        setattr(src, k, __import__("ctypes").cast(
            pinned[k].data_ptr(), sph._D))
    outs = {k: torch.empty(n, dtype=torch.float64).pin_memory()
            for k in ("x", "y", "u", "v", "p")}
    out_np = {k: v.numpy() for k, v in outs.items()}
    for _ in range(2):
        sim.load_raw(sph.SPH_FLUID, n, src)
        sim.step(1, want_time=False)
        for k in out_np:
            sim.read_into(k, out_np[k])
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ke = max(3, args.steps // 2)
    for _ in range(ke):
        sim.load_raw(sph.SPH_FLUID, n, src)
        sim.step(1, want_time=False)
        for k in out_np:
            sim.read_into(k, out_np[k])
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_val = world * n * ke / float(e2e_t.item())
    sim.close()

    # plain FP64 GPU form on the same workload (spec: mixed vs FP64)
    fp64 = None
    if not args.no_fp64:
        s64 = new_sim(sph.SPH_FP64)
        ms64, f64, _ = timed_steps(s64, max(3, args.steps // 4), 3)
        fp64 = n / (float(np.mean(ms64)) / 1e3)
        s64.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        frac = 0.1
        run_oracle_sample(d, 1, 0.01)           # warm (build, caches)
        nn, el, cores = run_oracle_sample(d, 2, frac)
        el /= 2
        cpu = {"value": nn / el, "unit": "particle-steps/s", "cores": cores,
               "kind": "oracle",
               "sample": "window |x-L/2|<%.3gL of the workload (%d particles,"
                         " non-periodic in x), 2 PEC steps" % (frac / 2, nn)}

    peaks, pk_kind = measured_peaks()
    line = {
        "metric": "particle-steps/s", "value": value,
        "unit": "particle-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tmax / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32-pair/f64-state", "data": "synthetic",
        "config": {"workload": args.workload, "desc": desc, "n": n,
                   "precision": "mixed", "l2": "flushed between steps "
                   "(256 MiB write)"},
        "pair_interactions_per_s": pairs * 2 / (tmax / 1e3 / args.steps),
        "pass_b_pair_interactions_per_s": pairs / (avg_b / 1e3),
        "fp64_particle_steps_per_s": fp64,
        "mixed_over_fp64": (value / world / fp64) if fp64 else None,
        "kernel_ms_per_step": {
            "pass_b": passb_ms / args.steps, "pass_a": passa_ms / args.steps,
            "rebuild": fams[2][0] / args.steps, "pec": fams[3][0] / args.steps},
        "roofline": {"bound": "alu", "kernel": "k_pass_b<float>",
                     "achieved": ach_b, "peak": peak_alu, "unit": "TFLOP/s",
                     "frac": ach_b / peak_alu, "traffic": None,
                     "peak_kind": "derived FP32 non-tensor peak at 2070 MHz "
                                  "(152 SM x 128 lanes x 2)"},
        "clocks": clocks,
        "e2e": {"value": e2e_val, "unit": "particle-steps/s",
                "h2d_bytes_per_step": 8 * len(fields_in) * n,
                "d2h_bytes_per_step": 8 * len(outs) * n},
        "gpu_launches": None,
        "cpu_baseline": cpu,
        "peaks": {"hbm_gbs": peaks.get("hbm_gbs"), "kind": pk_kind},
        "neighbours_mean": float(nnb.mean()),
    }
    line["gpu_launches"] = int(nlaunch)
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
