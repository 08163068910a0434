"""Benchmark: vehicle-steps/s of the traffic microsimulation hot path on one GB300.

Workload (default): the metropolitan network (225,000 nodes, 550,000 links, 3,000,000
gravity-OD trips; dt = 0.5 s) with every trip on its GPU-planned shortest-path route
and all of them on the road at once (the saturated snapshot: every trip placed on a
random hop of its route, evenly spaced in its lane, at half the speed limit).  One
bench step = one simulation step of the whole hot path (occupancy rebuild,
neighbours, lane changes, IDM, admission and transitions, departures, counters).

Prints one JSON line.  ``--impl reference`` times the CPU oracle instead (the
reference arm: the plain single-threaded C implementation of the same model), on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "vehicle-steps/s"
UNIT = "vehicle-steps/s"

# Roofline bytes of the method per vehicle-step (the algorithmic traffic of one step,
# neighbour re-reads not counted): the plain step kernel (neighbours, lane change, car
# following, admission and transition) reads and writes x, v, link/lane slot, route
# cursor and flags once (5 x 4 B each way); the whole step adds the occupancy rebuild,
# one pass over nearly sorted (u64 key + u32 id) records (24 B).
STEP_KERNEL_BYTES = 40
WHOLE_STEP_BYTES = 64
# kernels that make up the plain step kernel (the lane-front and chunk kernels)
STEP_KERNELS = ("front", "chunk")

# Implementation bytes per vehicle that each kernel of this design moves (every array
# element it reads or writes once, its own scratch included; per-link and per-lane
# records not counted): these explain the kernels, the roofline above judges the step.
IMPL_BYTES = {
    "scatter": 20 + 4 + 16,          # link, lane id, arrival index, x, vid; lane start; 4 scatter words
    "rank": 16 + 4 + 21 + 29,        # scatter words; lane starts; link, nxt, lane, v, cursor, movement
                                     # gathered from A; sorted state written to B
    "chunk": 21 + 8 + 38 + 8,        # staged x, v, vid, lane id, link, movement; nxt, cursor; next state
                                     # (with lane id, arrival index, decision); lane count
}


# DRAM bytes (read + write) per active vehicle per launch of the plain step kernel
# (front + chunk), from the ncu capture summarised under profiles/, valid only for the
# kernel sources it was taken on.
PROFILED_SRC_SHA = "13600078790119c1"
PROFILED_STEP_TRAFFIC = 149.0   # k_front 67.4 + k_chunk 81.5 B per active vehicle (987,466 vehicles)


def kernel_source_sha():
    import hashlib
    h = hashlib.sha256()
    for f in ("gbt_fused.cu", "gbt_rebuild.cuh", "gbt_stepdev.cuh", "gbt_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1807_01148_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def flush_l2(torch, buf):
    """Write a buffer larger than the L2 cache (on the current stream)."""
    buf.zero_()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="cuda", choices=["cuda", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the 64-scenario batched-ensemble comparison")
    ap.add_argument("--batched-steps", type=int, default=7200)
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint/forward time ratio")
    ap.add_argument("--no-assign", action="store_true", help="skip the static-assignment timing")
    ap.add_argument("--no-outputs", action="store_true",
                    help="skip the measured-output overhead and the equilibrium timing")
    ap.add_argument("--no-day", action="store_true", help="skip the natural 24 h metro run")
    ap.add_argument("--no-jam", action="store_true", help="skip the standing-queue (jammed lanes) case")
    ap.add_argument("--workload", default="metro", choices=["metro", "metro-walk"],
                    help="metro: GPU-planned shortest-path routes; metro-walk: the first --trips trips on "
                         "random-walk routes (no trip planning; smaller cases for profiling)")
    ap.add_argument("--trips", type=int, default=0,
                    help="use only the first N trips of the metro demand (0 = all; smaller cases for profiling)")
    ap.add_argument("--sample-frac", type=float, default=0.1,
                    help="fraction of trips in the CPU oracle's bounded sample")
    return ap.parse_args()


# ---------------------------------------------------------------------------- helpers
class ClockSampler:
    """nvidia-smi clock / throttle sampling while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0, period_ms=50):
        self.index = index
        self.period = period_ms
        self.proc = None
        self.lines = []
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 f"-lms", str(self.period)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def mark(self, which):
        setattr(self, which, time.time())

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        rows = []
        for ts, line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            rows.append((ts, f))
        inside = [f for ts, f in rows if self.t0 and self.t1 and self.t0 - 0.05 <= ts <= self.t1 + 0.05]
        use = inside if inside else [f for _, f in rows]
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        sm = [float(f[1]) for f in use if f[1].replace(".", "").isdigit()]
        mx = [float(f[2]) for f in use if f[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for f in use for i in range(4) if f[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(use), "samples_in_timed_region": len(inside)}


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_over_ranks(secs, veh_steps, world, device):
    """Replicas (one per GPU, no exchange): the job takes the slowest rank's time and
    advances the vehicle-steps of all ranks."""
    if world <= 1:
        return secs, veh_steps
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(secs)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    v = torch.tensor([float(veh_steps)], dtype=torch.float64, device=device)
    dist.all_reduce(v, op=dist.ReduceOp.SUM)
    return float(t.item()), float(v.item())


def lscpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu model")):
                return line.split(":", 1)[1].strip()
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for line in out.splitlines():
            if "Model name" in line:
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


# ---------------------------------------------------------------------------- oracle arm
def oracle_sample(frac, seed=1807011499):
    """Bounded sample of the workload for the CPU oracle: the same metro network and
    snapshot recipe with a random ``frac`` of the trips, routed by the oracle itself is
    too slow (one Dijkstra per origin over 225k nodes), so the sample's trips follow
    random-walk routes of the same mean length (inputs, not derived from the GPU)."""
    from paper_1807_01148_gb300 import scenarios as S
    m = S.metro()
    rng = np.random.default_rng(seed)
    keep = np.sort(rng.choice(m["demand"]["n_trips"], int(m["demand"]["n_trips"] * frac), replace=False))
    d = m["demand"]
    m["demand"] = S._demand(d["origin"][keep], d["dest"][keep], d["depart_step"][keep])
    off, links = S.random_walk_routes(m, min_hops=20, max_hops=90)
    st = S.saturate(m, off, links)
    return m, off, links, st


def time_oracle(frac, steps, warmup, budget_s=None):
    import oracle
    m, off, links, st = oracle_sample(frac)
    o = oracle.OracleSim(m)
    o.set_routes(off, links)
    o.write_state(st)
    o.step(warmup)
    c0 = o.counters()
    t0 = time.perf_counter()
    n = 0
    while n < steps:
        o.step(1)
        n += 1
        if budget_s and time.perf_counter() - t0 > budget_s and n >= 1:
            break
    dt = time.perf_counter() - t0
    c1 = o.counters()
    vs = c1["veh_steps"] - c0["veh_steps"]
    return dict(value=vs / dt, steps=n, seconds=dt, veh_steps=vs, trips=m["demand"]["n_trips"])


def time_oracle_routing(n_trips=100):
    """The oracle's trip planning (one Dijkstra tree per distinct origin, canonical
    routes) for the first n_trips trips of the metro demand on the full network:
    trees per second on one core."""
    import oracle
    from paper_1807_01148_gb300 import scenarios as S
    m = S.metro()
    d = m["demand"]
    m["demand"] = S._demand(d["origin"][:n_trips], d["dest"][:n_trips], d["depart_step"][:n_trips])
    n_orig = int(len(np.unique(m["demand"]["origin"])))
    o = oracle.OracleSim(m)
    t0 = time.perf_counter()
    o.route()
    dt = time.perf_counter() - t0
    return {"trees_per_s": n_orig / dt, "seconds": dt, "cores": 1,
            "sample": f"{n_orig} origin trees (the first {n_trips} trips of the metro demand) on the full "
                      f"225000-node network, single-threaded"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    r = time_oracle(args.sample_frac, args.steps, args.warmup)
    cores = 1
    sample = (f"{r['trips']} of 3,000,000 metro trips ({args.sample_frac:.0%}) in the saturated snapshot "
              f"recipe on the full 225k-node network, random-walk routes; {r['steps']} steps")
    line = {"impl": "reference", "metric": METRIC, "value": r["value"], "unit": UNIT, "n_gpus": args.gpus,
            "steps": r["steps"], "warmup": args.warmup, "ms_per_step": 1e3 * r["seconds"] / max(1, r["steps"]),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "metro saturated snapshot (bounded sample for the CPU oracle)",
                       "network": "225000 nodes / 550000 links", "trips_in_sample": r["trips"]},
            "cpu_baseline": {"value": r["value"], "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample,
                             "cpu": lscpu_model()},
            "e2e": {"value": r["value"], "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------- batched ensemble
def measure_batched(G, S, torch, steps):
    """64 grid scenarios of uneven size (side 10..40, 5k..80k trips, per-scenario IDM
    parameters) advanced together by one handle (sim_create_batch) against the same 64
    scenarios run one after another, each in its own handle; device time of the stepping
    only (trip planning excluded on both sides)."""
    scs = S.ensemble(steps=steps)
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b = G.Sim.batch(scs)
    b.set_stream(stream.cuda_stream)
    b.route()
    # block shape / execution mode picked by the autotuner on a copy advanced to the middle
    # of the run (the early steps, with few vehicles, favour the persistent launch; the
    # busy ones the graph)
    tune = G.Sim.batch(scs)
    tune.set_stream(stream.cuda_stream)
    tune.route()
    tune.step(steps // 2)
    choice = tune.autotune(trial_steps=100)
    tune.close()
    # both execution modes over the whole run, the autotuner's pick for the headline
    modes = {}
    for name, ex in (("graph", dict(mode=0, grid_per_sm=8)),
                     ("persistent", choice if choice["mode"] == 1 else dict(mode=1, threads=256, blocks_per_sm=4))):
        m = G.Sim.batch(scs)
        m.set_stream(stream.cuda_stream)
        m.route()
        m.set_exec(**ex)
        m.step(1)
        torch.cuda.synchronize()
        e0.record(stream)
        m.step(steps - 1)
        e1.record(stream)
        torch.cuda.synchronize()
        modes[name] = {"us_per_step": 1e3 * e0.elapsed_time(e1) / (steps - 1), "exec": ex}
        m.close()
    b.set_exec(**choice)
    torch.cuda.synchronize()
    e0.record(stream)
    b.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    tb = e0.elapsed_time(e1) / 1e3
    vb = b.counters()["veh_steps"]
    b.close()
    ts, vs = 0.0, 0
    for sc in scs:
        g = G.Sim(sc)
        g.set_stream(stream.cuda_stream)
        g.route()
        torch.cuda.synchronize()
        e0.record(stream)
        g.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ts += e0.elapsed_time(e1) / 1e3
        vs += g.counters()["veh_steps"]
        g.close()
    return {"scenarios": len(scs), "steps": steps, "trips": int(sum(s["demand"]["n_trips"] for s in scs)),
            "batched": {"value": vb / tb, "seconds": tb, "veh_steps": vb},
            "sequential": {"value": vs / ts, "seconds": ts, "veh_steps": vs},
            "ratio": (vb / tb) / (vs / ts), "unit": UNIT, "exec": choice, "modes": modes,
            "note": "one handle over the disjoint union of the 64 scenarios, execution configuration chosen by "
                    "sim_autotune (mode 1 = all steps in one persistent cooperative launch captured as a CUDA "
                    "graph, mode 0 = one graph of the step kernels per step) vs 64 handles stepped one after "
                    "another; identical vehicle-steps"}


# ---------------------------------------------------------------------------- adjoint
def measure_adjoint(G, S, torch, reps=3):
    """Calibration workload: the 20x20 grid with 20,000 trips and three link classes,
    1800 steps, loss = squared route-progress error every 20 steps against trajectories
    of perturbed parameters.  Ratio = wall time of sim_adjoint (forward with checkpoints
    every 64 steps, per-segment taped replay, binary64 reverse sweep) / wall time of the
    plain forward sim_step(1800); best of `reps` each."""
    sc = S.calib()
    n = sc["demand"]["n_trips"]
    steps, every = sc["steps"], sc["obs_every"]
    keys = ("v0", "T", "a", "b", "s0")
    g = G.Sim(sc)
    g.route()
    tp = sc["target_params"]
    g.set_class_params(*[tp[k] for k in keys])
    target = g.observe(steps, every)
    p = sc["params"]
    g.set_class_params(*[p[k] for k in keys])
    start = dict(status=np.zeros(n, np.uint8), link=np.zeros(n, np.int32), lane=np.zeros(n, np.int32),
                 cursor=np.zeros(n, np.int32), x=np.zeros(n, np.float32), v=np.zeros(n, np.float32))
    tf, ta = [], []
    grad = loss = None
    for _ in range(reps):
        g.write_state(start)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g.step(steps)
        torch.cuda.synchronize()
        tf.append(time.perf_counter() - t0)
        g.write_state(start)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        grad, loss = g.adjoint(steps, every, target, 3)
        torch.cuda.synchronize()
        ta.append(time.perf_counter() - t0)
    g.close()
    return {"workload": "20x20 grid, 20000 trips, 3 link classes x (v0, T, a, b, s0), 1800 steps, "
                        "observations every 20 steps, checkpoints every 64",
            "forward_s": min(tf), "adjoint_s": min(ta), "ratio": min(ta) / min(tf), "loss": loss,
            "grad_norm": float(np.linalg.norm(grad))}


# ---------------------------------------------------------------------------- outputs
def measure_outputs(G, g, snap, args, stream, torch, plain_ms):
    """The metro snapshot stepped again with every measured output on: fuel and CO per
    trip (Eq. 8-9), link traversal times (Sec. 6.3.1) and per-edge samples every 60 s in
    6-minute windows (Sec. 6.4).  Device time per step against the plain steps."""
    g.set_outputs(G.OUT_EMISSIONS | G.OUT_LINK_TIMES | G.OUT_EDGE_SAMPLES, 120, 6,
                  (args.warmup + args.steps) // 720 + 1)
    g.write_state(snap)
    g.step(args.warmup)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    g.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    fuel, co = g.emissions()
    _, n_exit = g.link_times()
    g.set_outputs(0)
    return {"ms_per_step": ms, "overhead_frac": ms / plain_ms - 1.0, "every_steps": 120, "per_window": 6,
            "fuel_l_total": float(fuel.sum() / 1e3), "co_kg_total": float(co.sum() / 1e3),
            "link_exits": int(n_exit.sum())}


def measure_equilibrium(G, S, torch):
    """Sec. 6.3.1 iterative decaying equilibrium on the 20x20 signalised grid (20,000
    trips, 9,000 steps per run): four runs routed on 100%, 100%, 50% and 25% of the trips,
    the first on sqrt(lanes) * length / speed, the others on the travel times measured in
    the previous run.  Wall time of the whole sim_equilibrium call."""
    sc = S.grid()
    sc["params"]["cost_mode"] = 1
    g = G.Sim(sc)
    g.set_outputs(G.OUT_LINK_TIMES)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    cost, gap = g.equilibrium([65536, 65536, 32768, 16384], sc["steps"])
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    c = g.counters()
    g.close()
    return {"workload": "20x20 grid, 20000 trips, 4 x 9000 steps", "seconds": secs, "gap": [float(x) for x in gap],
            "last_run_arrived": c["arrived"], "last_run_veh_steps": c["veh_steps"]}


def measure_assignment(G, S, torch, iters=2):
    """Static user equilibrium (Sec. 5.2) of the full metro demand (3,000,000 trips over
    24 h, Table 3 capacities) on the 550,000-link network: the initial all-or-nothing
    assignment plus `iters` Frank-Wolfe iterations, each one a full set of 225,000
    shortest-path trees.  Wall time of sim_assign_static."""
    sc = S.metro()
    cap = S.bpr_capacity(sc, 24.0, S.METRO_EDGE_TYPES)
    g = G.Sim(sc)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    r = g.assign_static(cap, max_iter=iters)
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    g.close()
    return {"workload": f"metro, 3000000 trips, capacities over 24 h, {iters} Frank-Wolfe iterations "
                        f"({iters + 1} all-or-nothing assignments of 225000 trees)",
            "seconds": secs, "seconds_per_assignment": secs / (iters + 1),
            "gap": [float(x) for x in r["gap"]], "step": [float(x) for x in r["step"]],
            "objective": [float(x) for x in r["objective"]]}


# ---------------------------------------------------------------------------- natural day, queues
def measure_natural_day(G, S, torch, stream):
    """The metro network with its natural demand (3,000,000 gravity-OD trips, bimodal
    departures): trip planning on the GPU, then all 172,800 steps of the day from t = 0,
    in the execution configuration the autotuner picks on a copy advanced to 8 h (the
    morning peak), and again with the per-step graph.  Vehicle-steps/s over the stepping
    (CUDA events), wall time with and without routing, the active count every 30
    simulated minutes."""
    sc = S.metro()
    g = G.Sim(sc)
    g.set_stream(stream.cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g.route()
    torch.cuda.synchronize()
    route_s = time.perf_counter() - t0
    off, links = g.routes()
    tune = G.Sim(sc)
    tune.set_stream(stream.cuda_stream)
    tune.set_routes(off, links)
    tune.step(57600)
    choice = tune.autotune(trial_steps=200)
    tune.close()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def day(h):
        samples = []
        step_ms = 0.0
        t1 = time.perf_counter()
        for _ in range(48):
            e0.record(stream)
            h.step(3600)
            e1.record(stream)
            torch.cuda.synchronize()
            step_ms += e0.elapsed_time(e1)
            samples.append(int(h.counters()["active"]))
        return step_ms, time.perf_counter() - t1, samples

    g.set_exec(**choice)
    step_ms, wall, samples = day(g)
    c = g.counters()
    g.close()
    gg = G.Sim(sc)
    gg.set_stream(stream.cuda_stream)
    gg.set_routes(off, links)
    gg.set_exec(mode=0, grid_per_sm=8)
    graph_ms, _, _ = day(gg)
    cg = gg.counters()
    gg.close()
    assert cg["veh_steps"] == c["veh_steps"] and cg["arrived"] == c["arrived"]
    return {"workload": "metro, 3000000 trips, gravity OD, bimodal departures, GPU-planned routes, 172800 steps "
                        "(24 h at 0.5 s)",
            "value": c["veh_steps"] / (step_ms / 1e3), "unit": UNIT, "vehicle_steps": int(c["veh_steps"]),
            "step_seconds": step_ms / 1e3, "wall_seconds": wall, "routing_seconds": route_s,
            "end_to_end_seconds": wall + route_s, "peak_active_30min_samples": max(samples),
            "active_every_30min": samples, "arrived": int(c["arrived"]), "departed": int(c["departed"]),
            "exec": choice, "graph_step_seconds": graph_ms / 1e3,
            "note": "exec: sim_autotune's pick on a copy at 8 h; graph_step_seconds: the same day with one graph "
                    "of the step kernels per step (identical vehicle-steps and arrivals)"}


def measure_jam(G, S, torch, stream, steps=300):
    """Standing queues: 1000 corridors, each a 2 km two-lane link into a signalised node
    (15 s of green per minute) holding about 285 vehicles per lane at rest.  Device time
    per step and per kernel (the in-lane rank of the occupancy rebuild grows with the
    queue length)."""
    sc = S.jammed_corridors(n_corr=1000)
    g = G.Sim(sc)
    g.set_stream(stream.cuda_stream)
    g.set_routes(sc["routes"]["offsets"], sc["routes"]["links"])
    g.write_state(sc["init_state"])
    g.step(10)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    c0 = g.counters()
    torch.cuda.synchronize()
    e0.record(stream)
    g.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    c1 = g.counters()
    lane_start, _ = g.occupancy()
    g.write_state(sc["init_state"])
    g.step(10)
    kms = g.step_timed(steps)
    g.close()
    vs = (c1["veh_steps"] - c0["veh_steps"]) / steps
    return {"workload": "1000 corridors x 2 lanes x 2 km, queues at rest behind signals (green 15 s / 60 s)",
            "ms_per_step": ms, "value": vs / (ms / 1e3), "unit": UNIT, "avg_active": vs,
            "longest_lane_queue": int(np.diff(lane_start).max()),
            "per_kernel_ms_per_step": {k: v / steps for k, v in kms.items()}}


# ---------------------------------------------------------------------------- cuda arm
def run_cuda(args):
    import torch

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    from paper_1807_01148_gb300 import gbtraffic as G
    from paper_1807_01148_gb300 import scenarios as S

    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    m = S.metro()
    if args.trips:
        d = m["demand"]
        k = args.trips
        m["demand"] = S._demand(d["origin"][:k], d["dest"][:k], d["depart_step"][:k])
    stream = torch.cuda.current_stream()
    g = G.Sim(m)
    g.set_stream(stream.cuda_stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if args.workload == "metro":
        g.route()
        off, links = g.routes()
    else:
        off, links = S.random_walk_routes(m, min_hops=20, max_hops=90)
        g.set_routes(off, links)
    torch.cuda.synchronize()
    route_s = time.perf_counter() - t0
    snap = S.saturate(m, off, links)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local).start()

    # -- main timed region: K graph-launched steps from the snapshot
    g.write_state(snap)
    g.step(args.warmup)
    c0 = g.counters()
    n_launch0 = g.launch_count()
    barrier()
    clocks.mark("t0")
    ev0.record(stream)
    g.step(args.steps)
    ev1.record(stream)
    barrier()
    clocks.mark("t1")
    ms = ev0.elapsed_time(ev1)
    c1 = g.counters()
    veh_steps = c1["veh_steps"] - c0["veh_steps"]
    launches = g.launch_count() - n_launch0
    clk = clocks.stop()

    # -- per-kernel device times over the same K steps (events after every kernel),
    #    back to back, then again with the L2 cache flushed before every step (the flush
    #    is outside the events)
    g.write_state(snap)
    g.step(args.warmup)
    c2 = g.counters()
    kms = g.step_timed(args.steps)
    c3 = g.counters()
    avg_active = (c3["veh_steps"] - c2["veh_steps"]) / max(1, args.steps)
    avg_cand = (c3["lc_evals"] - c2["lc_evals"]) / max(1, args.steps)
    l2_bytes = torch.cuda.get_device_properties(local).L2_cache_size
    flush_buf = torch.empty(2 * l2_bytes // 4 + 1024, dtype=torch.float32, device="cuda")
    g.write_state(snap)
    g.step(args.warmup)
    c4 = g.counters()
    kms_fl = {}
    for _ in range(args.steps):
        flush_l2(torch, flush_buf)
        for k, v in g.step_timed(1).items():
            kms_fl[k] = kms_fl.get(k, 0.0) + v
    c5 = g.counters()
    avg_active_fl = (c5["veh_steps"] - c4["veh_steps"]) / max(1, args.steps)
    del flush_buf
    step_ms = sum(kms[k] for k in STEP_KERNELS) / args.steps
    step_ms_fl = sum(kms_fl[k] for k in STEP_KERNELS) / args.steps
    achieved_fl = STEP_KERNEL_BYTES * avg_active_fl / (step_ms_fl * 1e-3) / 1e9
    achieved = STEP_KERNEL_BYTES * avg_active / (step_ms * 1e-3) / 1e9
    whole = WHOLE_STEP_BYTES * (veh_steps / args.steps) / (ms / args.steps * 1e-3) / 1e9
    impl_gbs = {k: IMPL_BYTES[k] * avg_active / (kms[k] / args.steps * 1e-3) / 1e9 for k in IMPL_BYTES if k in kms}

    # -- end to end through the C ABI with host buffers: load the snapshot from pinned host
    #    memory, then every step read positions and speeds back to pinned host memory.  The
    #    device-to-host copy of step k runs on a second stream while step k + 1 computes
    #    (double-buffered device staging); all copies finish inside the timed region.
    e2e = None
    if not args.no_e2e:
        pin = {k: torch.from_numpy(np.ascontiguousarray(v)).pin_memory() for k, v in snap.items()}
        n = m["demand"]["n_trips"]
        hx = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in range(2)]
        hv = [torch.empty(n, dtype=torch.float32).pin_memory() for _ in range(2)]
        dx = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(2)]
        dv = [torch.empty(n, dtype=torch.float32, device="cuda") for _ in range(2)]
        views = [G.sim_state_view(None, None, None, None, dx[k].data_ptr(), dv[k].data_ptr(), None, None, None)
                 for k in range(2)]
        copy_stream = torch.cuda.Stream()
        done = [torch.cuda.Event(), torch.cuda.Event()]
        ready = [torch.cuda.Event(), torch.cuda.Event()]
        import ctypes
        L = G.lib()
        e_steps = min(args.steps, 100)
        barrier()
        t0 = time.perf_counter()
        rc = L.sim_write_state(g.h, *[ctypes.c_void_p(pin[k].data_ptr()) for k in
                                       ("status", "link", "lane", "cursor", "x", "v")])
        assert rc == 0, L.sim_last_error(g.h)
        ce0 = g.counters()
        for k in range(e_steps):
            b = k % 2
            done[b].synchronize()                  # step k-2's x, v are in host memory
            rc = L.sim_step(g.h, 1)
            assert rc == 0
            # gather into staging b, enqueued behind the step on the handle's stream; the
            # copy to pinned host memory waits for it on a second stream, while step k+1
            # is already queued behind it
            rc = L.sim_read_state(g.h, ctypes.byref(views[b]), G.F_X | G.F_V, 2)
            assert rc == 0
            ready[b].record(stream)
            copy_stream.wait_event(ready[b])
            with torch.cuda.stream(copy_stream):
                hx[b].copy_(dx[b], non_blocking=True)
                hv[b].copy_(dv[b], non_blocking=True)
                done[b].record(copy_stream)
        copy_stream.synchronize()
        ce1 = g.counters()
        barrier()
        e2e_s = time.perf_counter() - t0
        h2d = sum(int(v.numel() * v.element_size()) for v in pin.values())
        e2e = {"value": (ce1["veh_steps"] - ce0["veh_steps"]) / e2e_s, "unit": UNIT,
               "h2d_bytes_per_step": h2d / e_steps, "d2h_bytes_per_step": 8 * n + 64,
               "steps": e_steps, "pattern": "sim_write_state(host snapshot) then per step sim_step(1) + "
                                            "sim_read_state(x, v -> device staging, enqueued on the step's stream) "
                                            "+ copy to pinned host on a second stream after an event, overlapping "
                                            "the next step; the host waits for step k's copy two steps later and "
                                            "for every copy before the clock stops"}

    day = jam = None
    if not args.no_day:
        day = measure_natural_day(G, S, torch, stream)
    if not args.no_jam:
        jam = measure_jam(G, S, torch, stream)
    outputs = equilibrium = assignment = None
    if not args.no_outputs:
        outputs = measure_outputs(G, g, snap, args, stream, torch, ms / args.steps)
        equilibrium = measure_equilibrium(G, S, torch)
    if not args.no_assign:
        g.close()
        assignment = measure_assignment(G, S, torch)

    # -- aggregate over ranks (replicas only: each rank runs its own copy)
    secs, tot_vs = reduce_over_ranks(ms / 1e3, veh_steps, world, "cuda")
    adjoint = None
    if not args.no_adjoint:
        adjoint = measure_adjoint(G, S, torch)
    batched = None
    if not args.no_batched:
        batched = measure_batched(G, S, torch, args.batched_steps)
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline:
        r = time_oracle(args.sample_frac, 50, 1, budget_s=20.0)
        cpu = {"value": r["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{r['trips']} trips ({args.sample_frac:.0%} of the metro demand) in the saturated "
                         f"snapshot recipe on the full network, random-walk routes; {r['steps']} steps, "
                         f"{r['seconds']:.1f} s single-threaded",
               "cpu": lscpu_model(),
               "routing": time_oracle_routing()}
    line = {
        "metric": METRIC, "value": tot_vs / secs, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": (f"metro (225000 nodes, 550000 links, {m['demand']['n_trips']} trips) saturated "
                                "snapshot: all trips on their GPU-planned shortest-path routes at once")
                               if args.workload == "metro" else
                               f"metro network, {m['demand']['n_trips']} trips on random-walk routes, saturated",
                   "dt_s": 0.5, "avg_active_vehicles": tot_vs / world / args.steps,
                   "l2": "headline steps back to back: working set > L2 (state, scratch and per-lane arrays "
                         "~0.5 GB); roofline: L2 flushed before every timed step",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": {"bound": "hbm", "kernel": "plain step kernel (front + chunk: neighbours, lane change, "
                                                 "car following, admission, transition)",
                     "achieved": achieved_fl, "peak": hbm_peak, "unit": "GB/s", "frac": achieved_fl / hbm_peak,
                     "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                     "alg_bytes_per_unit": STEP_KERNEL_BYTES, "unit_of_work": "vehicle-step",
                     "units_per_launch": avg_active_fl, "ms_per_launch": step_ms_fl,
                     "timing": "CUDA events around the two kernels, L2 flushed before every step",
                     "back_to_back": {"achieved": achieved, "frac": achieved / hbm_peak, "ms_per_launch": step_ms},
                     "traffic": (PROFILED_STEP_TRAFFIC * avg_active_fl
                                 if PROFILED_STEP_TRAFFIC and kernel_source_sha() == PROFILED_SRC_SHA else None),
                     "traffic_note": "ncu dram bytes (read + write) of the front and chunk kernels per vehicle on a "
                                     "smaller capture of the same network, scaled to this launch's vehicles; null "
                                     "when the kernel sources changed since",
                     "whole_step": {"alg_bytes_per_unit": WHOLE_STEP_BYTES, "achieved": whole,
                                    "frac": whole / hbm_peak, "ms_per_step": ms / args.steps,
                                    "timing": "graph-launched steps back to back (the headline value)"}},
        "per_kernel_ms_per_step": {k: v / args.steps for k, v in kms.items()},
        "per_kernel_ms_per_step_l2_flushed": {k: v / args.steps for k, v in kms_fl.items()},
        "per_kernel_impl_gbs": impl_gbs,
        "impl_bytes_note": "per_kernel_impl_gbs: this design's own bytes per vehicle (IMPL_BYTES, scratch "
                           "included) / back-to-back kernel time; explains the kernels, not a roofline",
        "lane_change_candidates_per_step": avg_cand,
        "routing": {"seconds": route_s, "mode": "gpu sim_route" if args.workload == "metro" else "set_routes",
                    "origins_trees": int(len(np.unique(m["demand"]["origin"]))),
                    "trees_per_s": int(len(np.unique(m["demand"]["origin"]))) / route_s,
                    "trips": m["demand"]["n_trips"], "hops": int(off[-1])},
        "natural_day": day,
        "jammed_lanes": jam,
        "outputs": outputs,
        "equilibrium": equilibrium,
        "static_assignment": assignment,
        "batched_ensemble": batched,
        "adjoint_forward": adjoint,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk,
        "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_cuda(args)


if __name__ == "__main__":
    main()
