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

# FP32 flops of one pass-B pair evaluation (formula operation count, FMA = 2)
# and of one pass-A pair.
PASS_B_FLOP_PER_PAIR = 90
PASS_A_FLOP_PER_PAIR = 60
# Compulsory bytes of the neighbour walk: per particle its x, y, h (FP64)
# and anchor record read and its own-entry count written (44 B), per list
# entry 4 B (the walk stages own entries and counts reverse ones).
WALK_BYTES_PER_PARTICLE = 44
WALK_BYTES_PER_ENTRY = 4
NFAM = 6   # timed kernel families of the library (sph_kernel_time)
FAM_NAMES = ["pass_b", "pass_a", "rebuild", "pec", "adapt", "walk"]
# kernel sources a DRAM-traffic capture is tied to
WALK_SOURCES = ["paper_2107_01276_gb300/csrc/lists.cu",
                "paper_2107_01276_gb300/csrc/neighbors.cuh",
                "paper_2107_01276_gb300/csrc/team.cuh"]


def sources_sha(paths):
    import hashlib
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), p),
                  "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def walk_kernel(n):
    """Name of the neighbour-walk kernel the library launches for n
    particles (the size rule of the list build)."""
    if n >= 60000:
        return "k_list_tile<1> (neighbour walk, cell tiles)"
    if n >= 12000:
        return "k_list_tile<4> (neighbour walk, cell tiles)"
    return "k_list_gather<T> (neighbour walk, per-particle teams)"


def walk_traffic(workload):
    """DRAM bytes per launch of the neighbour walk from the committed ncu
    summary, or None if there is none for this workload or the kernel
    sources changed since it was taken."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                        "profiles", "walk_dram_traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(workload)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("sources_sha") != sources_sha(WALK_SOURCES):
        return None
    return rec.get("dram_bytes_per_launch")

WORKLOADS = {
    # flow past a cylinder at Re 40, spacing graded from D/50 at
    # the wall to D/2 (1:25), split/merge every step
    "cylinder-re40": dict(kind="cylinder", Re=40.0, refine_calls=12),
    # pair-kernel sweep shape at N ~ 1M: 2-D periodic square, spacing
    # graded over 1:250 by C_r per column, u,v ~ N(0, 0.1),
    # rho = 1 + U(-0.01, 0.01); PEC steps, no adaptation
    "graded-1M": dict(kind="graded", n_target=1 << 20, ratio=250.0),
    # solution-adaptive cylinder at Re 1000, spacing D/1000 at the wall to
    # D/4 (1:250), vorticity marking (k = 0.05) with a background iteration
    # every 100 adaptations; fluid initialised from the graded ring
    # background and settled by 6 sph_adapt calls before timing
    "cylinder-re1000": dict(kind="cylinder", Re=1000.0,
                            ds_min_over_D=1 / 1000, ds_max_over_D=1 / 4,
                            background="rings", fluid="rings", vort_k=0.05,
                            n_bg=100, refine_calls=6, oracle_refine=0,
                            cpu_steps=1, capacity=2_000_000),
    # a stream of independent adaptive simulations (half
    # cylinders at Re log-uniform in [20, 2000], half Taylor-Green vortices
    # at Re in [50, 500]), Poisson arrivals at 20/s, served concurrently
    "serving": dict(kind="serving", requests=32, rate=20.0, slots=8,
                    steps=40, sizes=(5000, 50000)),
    # the same stream of requests with the Taylor-Green half stepped
    # together by the batch stepper (continuous batching of the steps)
    "serving-batched": dict(kind="serving", requests=32, rate=20.0, slots=8,
                            steps=40, sizes=(5000, 50000), batch=True),
    # 32 resident Taylor-Green vortices (Re uniform in [50, 500], particle
    # counts log-uniform in [1.6k, 20k]) advanced together by the batched
    # step (one persistent launch per phase over all of them, replayed as
    # a captured graph); compared with the same instances stepped one by
    # one on their own streams
    "batched-tg32": dict(kind="batch", instances=32, sizes=(1600, 20000)),
}
DEFAULT_WORKLOAD = "cylinder-re40"


def make_workload(name):
    w = WORKLOADS[name]
    if w["kind"] == "cylinder":
        dmin = w.get("ds_min_over_D", 1 / 50)
        dmax = w.get("ds_max_over_D", 0.5)
        d = wl.cylinder(Re=w["Re"], ds_min_over_D=dmin, ds_max_over_D=dmax,
                        background=w.get("background", "construct"),
                        fluid=w.get("fluid", "lattice"))
        d["params"] = dict(d["params"], vort_k=w.get("vort_k", 0.0),
                           n_bg=w.get("n_bg", 0))
        if w.get("background", "construct") == "construct":
            bgdesc = ("background built by sph_background (%d iterations) "
                      "from a D/%g lattice"
                      % (3 * math.ceil(math.log(dmax / dmin) / math.log(1.08)),
                         1 / dmax))
        else:
            bgdesc = "C_r-graded ring background"
        fdesc = ("coarse fluid lattice" if w.get("fluid", "lattice") == "lattice"
                 else "fluid initialised from the ring background")
        vdesc = (", vorticity adaptivity k=%g with a background iteration "
                 "every %d adaptations" % (w["vort_k"], w["n_bg"])
                 if w.get("vort_k", 0) > 0 else "")
        desc = ("flow past a cylinder, Re %g, D=2, rho0=1000, c_s=10, "
                "h/dx=1.2, C_r=1.08, spacing D/%g at the wall to D/%g "
                "(1:%g), 25D x 15D periodic box, impulsive start%s; %s, "
                "%s refined by %d sph_adapt calls before timing; a step is "
                "sph_adapt (split/merge/shift/h) + one PEC step"
                % (w["Re"], 1 / dmin, 1 / dmax, round(dmax / dmin), vdesc,
                   bgdesc, fdesc, w["refine_calls"]))
        return d, desc
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


def replica_totals(dist, time_s, units, device="cuda"):
    """Whole-job totals of a replica run: the slowest rank's time and the
    units all ranks processed (all_gather over the process group; the
    local values without one)."""
    if dist is None:
        return float(time_s), float(units)
    import torch
    my = torch.tensor([float(time_s), float(units)], dtype=torch.float64,
                      device=device)
    t_all = [torch.zeros_like(my) for _ in range(dist.get_world_size())]
    dist.all_gather(t_all, my)
    return max(float(t[0]) for t in t_all), sum(float(t[1]) for t in t_all)


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def fp32_alu_peak_tflops(sm_mhz):
    """Non-tensor FP32 peak: 152 SMs x 128 FP32 lanes x 2 flop (FMA) x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


# ------------------------------------------------------------ reference --
def cpu_sample(d, frac=0.1):
    """A band 0 <= y - lo < frac * Ly of the graded workload (its columns
    are graded along x, so the band holds every resolution in the
    workload's proportions) as a standalone set, non-periodic in y:
    bounded CPU work with the same particle shapes."""
    pt = d["particles"]
    lo, hi = d["params"]["lo"][1], d["params"]["hi"][1]
    sel = pt["y"] - lo < frac * (hi - lo)
    sub = {k: v[sel].copy() for k, v in pt.items()}
    per = d["params"]["periodic"]
    prm = dict(d["params"], periodic=(per[0], 0))
    return {"particles": sub, "params": prm}, int(sel.sum()), frac


def oracle_steps(d, state, steps, adaptive):
    """Time `steps` steps of the oracle (adaptation + PEC step when
    adaptive) from `state`; returns (particle-steps, seconds, threads)."""
    import oracle
    P = oracle.params(**d["params"])
    st = oracle.make_state(state, cap=max(4 * len(state["x"]), 1000))
    oracle.set_walls(d.get("walls"))
    bg = d.get("background_rings", d.get("background"))
    nid = int(np.max(state["id"])) + 1 if "id" in state else None
    ps, el = 0, 0.0
    try:
        for _ in range(steps):
            t0 = time.perf_counter()
            if adaptive:
                _, _, nid = oracle.adapt(P, st, bg=bg, next_id=nid)
            oracle.step(P, st, 1)
            el += time.perf_counter() - t0
            ps += st["n"]
    finally:
        oracle.set_walls(None)
    return ps, el, oracle.num_threads()


def reference_state(d, kind, w=None):
    """The state the oracle starts from: for the cylinder, the coarse set
    refined by the oracle's own adaptation (as the GPU set-up does) against
    the C_r-graded ring background, standing in for the constructed one
    (the oracle's construction alone takes minutes; its m_ref search is
    brute force over the background, so the smaller ring set makes the
    oracle's step faster, not slower)."""
    if kind != "cylinder":
        sd, n, frac = cpu_sample(d)
        return sd, sd["particles"], "band 0 <= y < %.2f L of the workload " \
            "(%d particles, all resolutions, non-periodic in y)" % (frac, n)
    import oracle
    P = oracle.params(**d["params"])
    st = oracle.make_state(d["particles"], cap=400000)
    oracle.set_walls(d["walls"])
    nid = None
    try:
        refine = (w or {}).get("oracle_refine",
                               (w or WORKLOADS["cylinder-re40"])["refine_calls"])
        for _ in range(refine):
            _, _, nid = oracle.adapt(P, st, bg=d["background_rings"],
                                     next_id=nid)
    finally:
        oracle.set_walls(None)
    n = st["n"]
    state = {k: st[k][:n].copy() for k in oracle.STATE_FIELDS}
    state["id"] = st["id"][:n].copy()
    how = ("after %d adaptations of the oracle's own" % refine if refine
           else "the generator's state, before any adaptation")
    return d, state, ("the whole workload (%d particles, %s; ring background "
                      "of %d particles)" % (n, how, len(d["background_rings"]["x"])))


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if WORKLOADS[args.workload]["kind"] in ("serving", "batch"):
        print(json.dumps({"impl": "reference", "unavailable":
                          "the oracle runs one simulation at a time; the "
                          "%s workload has no reference arm"
                          % WORKLOADS[args.workload]["kind"]}))
        return 0
    d, desc = make_workload(args.workload)
    kind = WORKLOADS[args.workload]["kind"]
    dd, state, sample = reference_state(d, kind, WORKLOADS[args.workload])
    adaptive = kind == "cylinder"
    oracle_steps(dd, state, max(args.warmup, 0) and 1, adaptive)
    ps, el, cores = oracle_steps(dd, state, args.steps, adaptive)
    v = ps / el
    line = {"impl": "reference", "metric": "particle-steps/s", "value": v,
            "unit": "particle-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": desc},
            "cpu_baseline": {"value": v, "unit": "particle-steps/s",
                             "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "particle-steps/s",
                    "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------- serving ----
def serving_arm(args):
    """The serving workload: requests admitted by free HBM and slots, each
    simulation resident in its own context on its own stream; value is the
    particle-steps of all requests over the wall time of the whole run
    (set-up of each request included), with per-step latency percentiles."""
    import torch
    from paper_2107_01276_gb300 import serve, sph
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    sph.lib()
    w = WORKLOADS[args.workload]
    reqs = serve.c5_requests(n=w["requests"], rate=w["rate"],
                             seed=7 + rank, steps=w["steps"], sizes=w["sizes"])
    srv = serve.Server(slots=w["slots"], batch=w.get("batch", False))
    clk = ClockSampler(local)
    clk.start()
    rep = srv.run(reqs)
    clocks = clk.stop()
    # every rank serves its own stream: the particle-steps of all ranks
    # over the slowest rank's wall time
    wall, units = replica_totals(dist, rep["wall_s"], rep["particle_steps"])
    value = units / wall if wall > 0 else 0.0
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    line = {
        "metric": "particle-steps/s", "value": value,
        "unit": "particle-steps/s", "n_gpus": world, "steps": rep["steps"],
        "warmup": 0, "ms_per_step": rep["step_ms_p50"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32-pair/f64-state", "data": "synthetic",
        "config": {"workload": args.workload, "requests": w["requests"],
                   "batched_steps": bool(w.get("batch", False)),
                   "arrival_rate_per_s": w["rate"], "slots": w["slots"],
                   "steps_per_request": w["steps"],
                   "particles": list(w["sizes"]),
                   "desc": "half flow past a cylinder (Re log-uniform "
                           "[20, 2000], adapt every step), half Taylor-Green "
                           "(Re uniform [50, 500]); Poisson arrivals; each "
                           "request's set-up (background construction, "
                           "refinement) inside the wall time"},
        "latency_ms": {"p50": rep["step_ms_p50"], "p99": rep["step_ms_p99"]},
        "serving": rep,
        "clocks": clocks,
        "e2e": {"value": value,
                "unit": "particle-steps/s", "h2d_bytes_per_step": None,
                "d2h_bytes_per_step": None},
    }
    print(json.dumps(line))
    return 0


# ------------------------------------------------------------ batched ----
def batch_arm(args):
    """Many small simulations advanced together by sph_batch_step.  value:
    particle-steps of all instances per second over K timed batch steps
    (CUDA events on the batch stream, L2 flushed between steps);
    streams_value: the same instances stepped one by one with sph_step on
    their own streams (host clock around K steps); e2e: every step loads
    each instance from pinned host buffers, runs the batch step and reads
    x, y, u, v, p back."""
    import ctypes

    import torch
    from paper_2107_01276_gb300 import sph, workloads as wl
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    sph.lib()
    w = WORKLOADS[args.workload]
    rng = np.random.default_rng(11 + rank)
    lo, hi = np.log(w["sizes"][0]), np.log(w["sizes"][1])
    nxs = [int(round(np.sqrt(np.exp(rng.uniform(lo, hi))))) for _ in range(w["instances"])]
    Res = [float(rng.uniform(50.0, 500.0)) for _ in nxs]
    bs = torch.cuda.Stream()
    own = [torch.cuda.Stream() for _ in nxs]
    sims, states = [], []
    for nx, Re, st in zip(nxs, Res, own):
        d = wl.taylor_green(nx=nx, Re=Re)
        n = len(d["particles"]["x"])
        P = sph.make_params(d["params"], precision=sph.SPH_MIXED, capacity=n)
        sm = sph.Simulation(P, st.cuda_stream)
        sm.load(d["particles"])
        sims.append(sm)
        states.append(d["particles"])
    ntot = sum(sm.info()["n"] for sm in sims)
    b = sph.Batch(len(sims), bs.cuda_stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    K, W = args.steps, args.warmup
    for _ in range(W):
        b.step(sims)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(K)]
    l0 = b.launches + sum(sm.info()["launches"] for sm in sims)
    g0 = b.graph_steps
    clk = ClockSampler(local)
    clk.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if args.profile_region:
        torch.cuda.cudart().cudaProfilerStart()
    with torch.cuda.stream(bs):
        for k in range(K):
            flush.zero_()
            evs[k][0].record(bs)
            b.step(sims)
            evs[k][1].record(bs)
    torch.cuda.synchronize()
    if args.profile_region:
        torch.cuda.cudart().cudaProfilerStop()
    if dist:
        dist.barrier()
    clocks = clk.stop()
    launches = b.launches + sum(sm.info()["launches"] for sm in sims) - l0
    graph_steps = b.graph_steps - g0
    ms = [a.elapsed_time(c) for a, c in evs]
    tmax, units = replica_totals(dist, float(np.sum(ms)), ntot * K)
    value = units / (tmax / 1e3)
    # the same instances, one sph_step each on its own stream
    for _ in range(W):
        for sm in sims:
            sm.step(1, want_time=False)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(K):
        for sm in sims:
            sm.step(1, want_time=False)
    torch.cuda.synchronize()
    streams_value = ntot * K / (time.perf_counter() - t0)
    # e2e: pinned host state in, batch step, x, y, u, v, p out
    fields_in = ("x", "y", "u", "v", "p", "rho", "m", "h")
    keep, srcs, outs = [], [], []
    h2d = d2h = 0
    for sm, st0 in zip(sims, states):
        n = len(st0["x"])
        src = sph.Particles()
        for k in fields_in:
            t = torch.from_numpy(np.ascontiguousarray(st0[k], np.float64)).pin_memory()
            keep.append(t)
            setattr(src, k, ctypes.cast(t.data_ptr(), sph._D))
            h2d += 8 * n
        srcs.append((n, src))
        outs.append({k: torch.empty(n, dtype=torch.float64).pin_memory().numpy()
                     for k in ("x", "y", "u", "v", "p")})

    def e2e_step():
        for sm, (n, src) in zip(sims, srcs):
            sm.load_raw(sph.SPH_FLUID, n, src)
        b.step(sims)
        nb = 0
        for sm, o in zip(sims, outs):
            for k in o:
                nb += 8 * sm.read_into(k, o[k])
        return nb

    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    ke = max(3, K // 2)
    t0 = time.perf_counter()
    for _ in range(ke):
        d2h = e2e_step()
    torch.cuda.synchronize()
    e2e_val = world * ntot * ke / (time.perf_counter() - t0)
    b.close()
    for sm in sims:
        sm.close()
    if dist:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    line = {
        "metric": "particle-steps/s", "value": value, "unit": "particle-steps/s",
        "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": float(np.mean(ms)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32-pair/f64-state",
        "data": "synthetic",
        "config": {"workload": args.workload, "instances": len(sims),
                   "particles_total": ntot,
                   "particles_per_instance": [min(x * x for x in nxs), max(x * x for x in nxs)],
                   "precision": "mixed", "l2": "flushed between steps (256 MiB write)",
                   "desc": "Taylor-Green vortices, Re uniform [50, 500], periodic unit "
                           "square, h/dx 1.2; one sph_batch_step per step"},
        "streams_value": streams_value,
        "batch_over_streams": value / streams_value,
        "graph_steps": graph_steps,
        "roofline": None,
        "clocks": clocks,
        "e2e": {"value": e2e_val, "unit": "particle-steps/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "cpu_baseline": None,
    }
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- ours ----
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--autotune", action="store_true",
                    help="run sph_autotune on the set-up state (untimed)")
    ap.add_argument("--profile-region", action="store_true",
                    help="bracket the timed steps of the mixed run with "
                         "cudaProfilerStart/Stop (for ncu "
                         "--profile-from-start off)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return reference_arm(args)
    if WORKLOADS[args.workload]["kind"] == "serving":
        return serving_arm(args)
    if WORKLOADS[args.workload]["kind"] == "batch":
        return batch_arm(args)

    import ctypes

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
    # a stream of the bench's own (the legacy default stream cannot be
    # captured, so the library could not replay its step graphs there)
    torch.cuda.set_stream(torch.cuda.Stream())
    stream = torch.cuda.current_stream().cuda_stream

    wdef = WORKLOADS[args.workload]
    kind = wdef["kind"]
    adaptive = kind == "cylinder"
    d, desc = make_workload(args.workload)
    pt = d["particles"]

    tuned = {}

    def new_sim(precision):
        cap = wdef.get("capacity", 400000) if adaptive else int(len(pt["x"]) * 1.1) + 16
        P = sph.make_params(d["params"], precision=precision, capacity=cap)
        s = sph.Simulation(P, stream)
        s.load(pt)
        if "walls" in d:
            s.load(d["walls"], kind=sph.SPH_WALL)
        if "background" in d:
            s.load(d["background"], kind=sph.SPH_BACKGROUND)
            if d.get("construct_background"):
                s.background()
        for _ in range(wdef.get("refine_calls", 0)):
            s.adapt()
        if args.autotune:
            tuned.update(s.autotune())
        return s

    def one_step(s):
        n = None
        if adaptive:
            n = s.adapt()["n_after"]
        s.step(1, want_time=False)
        return n

    # L2 flush buffer (> 129 MB L2), written between timed steps
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed_steps(s, K, W, profile=False, lib_timing=False):
        """K timed steps after W untimed ones; lib_timing: also the
        library's per-family CUDA events (which keep it from replaying
        captured step graphs)."""
        for _ in range(W):
            one_step(s)
        torch.cuda.synchronize()
        n_fixed = s.info()["n"]
        evs = [(torch.cuda.Event(enable_timing=True),
                torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        s.set_timing(lib_timing)
        for fam in range(NFAM):
            s.kernel_time(fam, reset=True)
        l0 = s.info()["launches"]
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        if profile:
            torch.cuda.cudart().cudaProfilerStart()
        ns = []
        for k in range(K):
            flush.zero_()
            evs[k][0].record()
            n = one_step(s)
            evs[k][1].record()
            ns.append(n if n is not None else n_fixed)
        torch.cuda.synchronize()
        if profile:
            torch.cuda.cudart().cudaProfilerStop()
        if dist:
            dist.barrier()
        s.set_timing(False)
        ms = [a.elapsed_time(b) for a, b in evs]
        fams = [s.kernel_time(f) for f in range(NFAM)]
        return ms, ns, fams, s.info()["launches"] - l0

    sim = new_sim(sph.SPH_MIXED)
    n_bg = sim.info()["n_bg"]
    clk = ClockSampler(local)
    clk.start()
    ms, ns, _, nlaunch = timed_steps(sim, args.steps, args.warmup,
                                     profile=args.profile_region)
    clocks = clk.stop()
    # the kernel breakdown (and the roofline's kernel times) from further
    # steps with the library's per-family events
    k_breakdown = max(5, args.steps // 4)
    _, _, fams, _ = timed_steps(sim, k_breakdown, 1, lib_timing=True)
    tot_ms = float(np.sum(ms))
    tmax, units = replica_totals(dist, tot_ms, float(np.sum(ns)))
    value = units / (tmax / 1e3)

    # force on the body after the timed steps (Eq. force-sph, Eq. cdcl);
    # a diagnostic of the state reached, outside the timed region
    forces = None
    if "walls" in d:
        f = sim.forces()
        forces = dict(sph.coefficients(f, d["params"]["rho0"], d.get("U", 1.0),
                                       d.get("D", 1.0)),
                      t=float(sim.info()["t"]))

    # pass-B pairs of the final state (rate of the pair loop)
    sim.rhs()
    nnb = sim.read("nnb")
    n_now = len(nnb)
    pairs = int(nnb.sum()) - n_now
    passb_ms, passb_cnt = fams[0]
    avg_b = passb_ms / max(passb_cnt, 1)
    peak_alu = fp32_alu_peak_tflops(2070.0)
    ach_b = PASS_B_FLOP_PER_PAIR * pairs / (avg_b / 1e3) / 1e12
    # the dominant kernel of the step: the neighbour walk
    walk_ms, walk_cnt = fams[5]
    avg_w = walk_ms / max(walk_cnt, 1)
    walk_bytes = WALK_BYTES_PER_PARTICLE * n_now + WALK_BYTES_PER_ENTRY * int(nnb.sum())
    peaks0, _ = measured_peaks()
    hbm_peak = peaks0.get("hbm_gbs") or 6800.0
    ach_w = walk_bytes / (avg_w / 1e3) / 1e9

    # e2e through the C ABI with pinned host buffers: H2D of the step's
    # fluid state, the step (adaptation + PEC), D2H of x, y, u, v, p
    state = {k: sim.read(k) for k in ("x", "y", "u", "v", "p", "rho", "m",
                                      "h", "mmin", "mmax")}
    state["id"] = sim.read("id")
    n_e = len(state["x"])
    fields_in = ("x", "y", "u", "v", "p", "rho", "m", "h", "mmin", "mmax")
    pinned = {k: torch.from_numpy(np.ascontiguousarray(state[k], np.float64)
                                  ).pin_memory() for k in fields_in}
    pid = torch.from_numpy(state["id"].astype(np.int64)).pin_memory()
    src = sph.Particles()
    for k in fields_in:
        setattr(src, k, ctypes.cast(pinned[k].data_ptr(), sph._D))
    src.id = ctypes.cast(pid.data_ptr(), ctypes.POINTER(ctypes.c_int64))
    cap_out = (wdef.get("capacity", 400000) if adaptive else 0) + 2 * n_e
    outs = {k: torch.empty(cap_out, dtype=torch.float64).pin_memory()
            for k in ("x", "y", "u", "v", "p")}
    out_np = {k: v.numpy() for k, v in outs.items()}
    d2h = 0

    def e2e_step():
        sim.load_raw(sph.SPH_FLUID, n_e, src)
        one_step(sim)
        nb = 0
        for k in out_np:
            nb += 8 * sim.read_into(k, out_np[k])
        return nb

    for _ in range(2):
        e2e_step()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ke = max(3, args.steps // 2)
    t0 = time.perf_counter()
    for _ in range(ke):
        d2h = e2e_step()
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_t = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(e2e_t, op=dist.ReduceOp.MAX)
    e2e_val = world * n_e * ke / float(e2e_t.item())
    bg_state = sim.read_background() if "background" in d else None
    sim.close()

    # mixed-precision error report: the mixed and FP64 paths on one state
    # (the mixed run's final one): right-hand sides field by field
    # (max |mixed - fp64| / max |fp64|) and the counts of one adaptation
    def error_report():
        out = {"rhs_rel_err": {}, "adapt": {}}
        res = {}
        for name, prec in (("mixed", sph.SPH_MIXED), ("fp64", sph.SPH_FP64)):
            cap = 400000 if adaptive else n_e + 16
            P = sph.make_params(d["params"], precision=prec, capacity=cap,
                                bg_capacity=400000)
            sx = sph.Simulation(P, stream)
            sx.load(dict(state))
            if "walls" in d:
                sx.load(d["walls"], kind=sph.SPH_WALL)
            if bg_state is not None:
                sx.load(bg_state, kind=sph.SPH_BACKGROUND)
            sx.rhs()
            ids = sx.read("id")
            order = np.argsort(ids)
            res[name] = {f: sx.read(f)[order] for f in
                         ("rho", "beta", "pavg", "drx", "dry", "dpdt", "dudt",
                          "dvdt")}
            if adaptive:
                g = sx.adapt()
                out["adapt"][name] = {k: int(g[k]) for k in
                                      ("n_split", "n_merged", "n_after")}
            sx.close()
        for f, ref in res["fp64"].items():
            sc = float(np.abs(ref).max()) or 1.0
            out["rhs_rel_err"][f] = float(np.abs(res["mixed"][f] - ref).max()) / sc
        return out

    err_rep = error_report() if world == 1 else None

    # the plain FP64 GPU form on the same workload
    fp64 = None
    if not args.no_fp64:
        s64 = new_sim(sph.SPH_FP64)
        ms64, ns64, _, _ = timed_steps(s64, max(4, args.steps // 4), 3)
        fp64 = float(np.sum(ns64)) / (float(np.sum(ms64)) / 1e3)
        s64.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return 0

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        dd, st0, sample = reference_state(d, kind, wdef)
        steps_cpu = wdef.get("cpu_steps", 2)
        ps, el, cores = oracle_steps(dd, st0, steps_cpu, adaptive)
        cpu = {"value": ps / el, "unit": "particle-steps/s", "cores": cores,
               "kind": "oracle",
               "sample": "%s, %d oracle steps (%s)" % (
                   sample, steps_cpu,
                   "adaptation + PEC step each" if adaptive else "PEC")}

    peaks, pk_kind = measured_peaks()
    fam_names = FAM_NAMES
    line = {
        "metric": "particle-steps/s", "value": value,
        "unit": "particle-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tmax / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32-pair/f64-state", "data": "synthetic",
        "config": {"workload": args.workload, "desc": desc,
                   "n_particles": int(np.mean(ns)),
                   "n_walls": len(d["walls"]["x"]) if "walls" in d else 0,
                   "n_background": int(n_bg),
                   "precision": "mixed",
                   "l2": "flushed between steps (256 MiB write)",
                   "timing": "value: CUDA events around each step on the "
                             "bench's stream, library timing off (sph_step "
                             "replays captured graphs where it can); kernel "
                             "breakdown and roofline: further steps with "
                             "per-family library events"},
        "pair_interactions_per_s": 4 * pairs / (tmax / 1e3 / args.steps),
        "pass_b_pair_interactions_per_s": pairs / (avg_b / 1e3),
        "fp64_particle_steps_per_s": fp64,
        "mixed_over_fp64": (value / world / fp64) if fp64 else None,
        "kernel_ms_per_step": {fam_names[f]: fams[f][0] / k_breakdown
                               for f in range(NFAM)},
        "roofline": {"bound": "hbm", "kernel": walk_kernel(int(np.mean(ns))),
                     "achieved": ach_w, "peak": hbm_peak, "unit": "GB/s",
                     "frac": ach_w / hbm_peak,
                     "traffic": walk_traffic(args.workload),
                     "bytes_per_launch": walk_bytes,
                     "ms_per_launch": avg_w,
                     "peak_kind": "measured copy bandwidth",
                     "note": "instruction- and latency-bound, not "
                             "bandwidth-bound: ncu shows high issue activity "
                             "and a few % DRAM throughput for this kernel"},
        "roofline_pass_b": {"bound": "alu", "kernel": "k_pass_b<float>",
                     "achieved": ach_b, "peak": peak_alu, "unit": "TFLOP/s",
                     "frac": ach_b / peak_alu, "traffic": None,
                     "peak_kind": "derived FP32 non-tensor peak at 2070 MHz "
                                  "(152 SM x 128 lanes x 2)"},
        "clocks": clocks,
        "e2e": {"value": e2e_val, "unit": "particle-steps/s",
                "h2d_bytes_per_step": 8 * len(fields_in) * n_e + 8 * n_e,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(nlaunch),
        "cpu_baseline": cpu,
        "peaks": {"hbm_gbs": peaks.get("hbm_gbs"), "kind": pk_kind},
        "neighbours_mean": float(nnb.mean()),
        "mixed_vs_fp64": err_rep,
        "forces": forces,
        "tuning": ({k: tuned[k] for k in ("cell_scale", "walk", "team_a", "team_b", "walls")}
                   if tuned else None),
    }
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
