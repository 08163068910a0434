"""Python binding of libgbtraffic (argument marshalling only; every step runs in the
CUDA library).  Names follow the C ABI in include/gbtraffic.h.

The library is built in-tree by ``paper_1807_01148_gb300.build``; importing this module
without it raises at first use, and there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

SIM_OK, SIM_EINVAL, SIM_ENOMEM, SIM_ECUDA, SIM_EUNREACHABLE, SIM_ETIMEOUT, SIM_ESTATE, SIM_EDEVICE = \
    0, -1, -2, -3, -4, -5, -6, -7
ERR_NAMES = {0: "SIM_OK", -1: "SIM_EINVAL", -2: "SIM_ENOMEM", -3: "SIM_ECUDA", -4: "SIM_EUNREACHABLE",
             -5: "SIM_ETIMEOUT", -6: "SIM_ESTATE", -7: "SIM_EDEVICE"}
F_STATUS, F_LINK, F_LANE, F_CURSOR, F_X, F_V, F_INSERT, F_ARRIVE, F_LANECHANGE = (1 << k for k in range(9))
F_ALL = (1 << 9) - 1

EXPORTS = ["sim_create", "sim_create_batch", "sim_set_stream", "sim_route", "sim_set_routes", "sim_route_size",
           "sim_read_routes", "sim_step", "sim_step_timed", "sim_kernel_name", "sim_read_state", "sim_write_state", "sim_occupancy", "sim_n_lanes",
           "sim_counters", "sim_last_error", "sim_destroy", "sim_set_class_params", "sim_observe", "sim_adjoint",
           "sim_set_exec", "sim_get_exec", "sim_autotune", "sim_set_outputs", "sim_reset_outputs",
           "sim_read_emissions", "sim_read_link_times", "sim_read_edge_samples", "sim_measured_costs",
           "sim_reroute", "sim_equilibrium", "sim_assign_static", "sim_set_vehicle_types", "sim_loss",
           "sim_launch_count"]
OUT_EMISSIONS, OUT_LINK_TIMES, OUT_EDGE_SAMPLES = 1, 2, 4
SIM_EXEC_GRAPH, SIM_EXEC_PERSISTENT = 0, 1


def n_kernels():
    """Kernels of one step (the names sim_kernel_name reports, in launch order)."""
    n = 0
    while lib().sim_kernel_name(n):
        n += 1
    return n


class sim_network(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("n_links", C.c_int32),
                ("node_x_dm", C.c_void_p), ("node_y_dm", C.c_void_p), ("node_control", C.c_void_p),
                ("signal_offset_ds", C.c_void_p), ("signal_cycle_ds", C.c_void_p),
                ("signal_green_ds", C.c_void_p), ("link_from", C.c_void_p), ("link_to", C.c_void_p),
                ("link_length_m", C.c_void_p), ("link_speed_mps", C.c_void_p),
                ("link_lanes", C.c_void_p), ("link_class", C.c_void_p)]


class sim_demand(C.Structure):
    _fields_ = [("n_trips", C.c_int32), ("origin", C.c_void_p), ("dest", C.c_void_p),
                ("depart_step", C.c_void_p)]


class sim_params(C.Structure):
    _fields_ = [("dt", C.c_float), ("veh_len", C.c_float), ("s_min", C.c_float), ("n_class", C.c_int32),
                ("v0", C.c_void_p), ("T", C.c_void_p), ("a", C.c_void_p), ("b", C.c_void_p), ("s0", C.c_void_p),
                ("mobil_p", C.c_float), ("mobil_athr", C.c_float), ("mobil_bsafe", C.c_float),
                ("mobil_bias_right", C.c_float), ("lambda_mand", C.c_float), ("stop_acquire_m", C.c_float),
                ("seed", C.c_uint64), ("cost_mode", C.c_int32), ("loop_routes", C.c_int32),
                ("max_device_bytes", C.c_uint64)]


class sim_counters_t(C.Structure):
    _fields_ = [(k, C.c_int64) for k in
                ("t", "departed", "waiting", "active", "arrived", "veh_steps", "pending", "active_last",
                 "lc_evals")]


class sim_exec(C.Structure):
    _fields_ = [("mode", C.c_int32), ("threads", C.c_int32), ("blocks_per_sm", C.c_int32),
                ("grid_per_sm", C.c_int32), ("barrier_timeout_cycles", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class sim_loss_spec(C.Structure):
    _fields_ = [("n_steps", C.c_int32), ("obs_every", C.c_int32), ("checkpoint_every", C.c_int32),
                ("target", C.c_void_p)]


class sim_sampling(C.Structure):
    _fields_ = [("every_steps", C.c_int32), ("per_window", C.c_int32), ("max_windows", C.c_int32)]


class sim_vehicle_type(C.Structure):
    _fields_ = [("length_m", C.c_float), ("accel_scale", C.c_float), ("max_speed_mps", C.c_float)]


class sim_assign_spec(C.Structure):
    _fields_ = [("capacity", C.c_void_p), ("alpha", C.c_double), ("beta", C.c_int32), ("max_iter", C.c_int32),
                ("bisect_iter", C.c_int32)]


class sim_state_view(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in
                ("status", "link", "lane", "cursor", "x", "v", "insert_step", "arrive_step", "lane_change")]


_lib = None


def lib(path: str | None = None):
    """Load libgbtraffic.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is None:
        so = path or _build.build()
        if not os.path.exists(so):
            raise RuntimeError(f"libgbtraffic not built: {so}")
        L = C.CDLL(so)
        vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
        L.sim_create.argtypes = [C.POINTER(sim_network), C.POINTER(sim_demand), C.POINTER(sim_params),
                                 C.POINTER(vp)]
        L.sim_create_batch.argtypes = [i32, C.POINTER(C.POINTER(sim_network)), C.POINTER(C.POINTER(sim_demand)),
                                       C.POINTER(C.POINTER(sim_params)), C.POINTER(vp)]
        L.sim_set_stream.argtypes = [vp, vp]
        L.sim_route.argtypes = [vp, vp]
        L.sim_set_routes.argtypes = [vp, vp, vp]
        L.sim_route_size.argtypes = [vp, C.POINTER(i64)]
        L.sim_read_routes.argtypes = [vp, vp, vp]
        L.sim_step.argtypes = [vp, i32]
        L.sim_step_timed.argtypes = [vp, i32, vp]
        L.sim_kernel_name.argtypes = [i32]
        L.sim_kernel_name.restype = C.c_char_p
        L.sim_launch_count.argtypes = [vp, C.POINTER(i64)]
        L.sim_read_state.argtypes = [vp, C.POINTER(sim_state_view), C.c_uint32, C.c_int]
        L.sim_write_state.argtypes = [vp] * 7
        L.sim_occupancy.argtypes = [vp, vp, vp]
        L.sim_n_lanes.argtypes = [vp, C.POINTER(i64)]
        L.sim_counters.argtypes = [vp, C.POINTER(sim_counters_t)]
        L.sim_last_error.argtypes = [vp]
        L.sim_last_error.restype = C.c_char_p
        L.sim_destroy.argtypes = [vp]
        L.sim_destroy.restype = None
        L.sim_set_class_params.argtypes = [vp] * 6
        L.sim_observe.argtypes = [vp, i32, i32, vp]
        L.sim_adjoint.argtypes = [vp, C.POINTER(sim_loss_spec), vp, vp]
        L.sim_loss.argtypes = [vp, C.POINTER(sim_loss_spec), vp]
        L.sim_set_exec.argtypes = [vp, C.POINTER(sim_exec)]
        L.sim_get_exec.argtypes = [vp, C.POINTER(sim_exec)]
        L.sim_autotune.argtypes = [vp, i32, C.c_char_p, C.POINTER(sim_exec)]
        u32 = C.c_uint32
        L.sim_set_outputs.argtypes = [vp, u32, C.POINTER(sim_sampling)]
        L.sim_reset_outputs.argtypes = [vp]
        L.sim_read_emissions.argtypes = [vp, vp, vp]
        L.sim_read_link_times.argtypes = [vp, vp, vp]
        L.sim_read_edge_samples.argtypes = [vp, vp, vp, vp]
        L.sim_measured_costs.argtypes = [vp, vp, vp, vp]
        L.sim_reroute.argtypes = [vp, vp, u32, u32]
        L.sim_equilibrium.argtypes = [vp, i32, vp, i32, vp, vp]
        L.sim_assign_static.argtypes = [vp, C.POINTER(sim_assign_spec), vp, vp, vp, vp, vp]
        L.sim_set_vehicle_types.argtypes = [vp, i32, C.POINTER(sim_vehicle_type), vp]
        _lib = L
    return _lib


class SimError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERR_NAMES.get(code, code)}: {msg}")
        self.code = code


def _p(a):
    return None if a is None else C.c_void_p(a.ctypes.data)


class _Keep:
    """Holds the numpy arrays behind a ctypes struct until the call returns."""

    def __init__(self):
        self.arrs = []

    def __call__(self, a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        self.arrs.append(a)
        return a.ctypes.data


def _structs(sc, keep):
    net, dem, par = sc["network"], sc["demand"], sc["params"]
    n = sim_network(net["n_nodes"], net["n_links"], keep(net["node_x_dm"], np.int32),
                    keep(net["node_y_dm"], np.int32), keep(net["node_control"], np.uint8),
                    keep(net["signal_offset_ds"], np.int32), keep(net["signal_cycle_ds"], np.int32),
                    keep(net["signal_green_ds"], np.int32), keep(net["link_from"], np.int32),
                    keep(net["link_to"], np.int32), keep(net["link_length_m"], np.float32),
                    keep(net["link_speed_mps"], np.float32), keep(net["link_lanes"], np.uint8),
                    keep(net["link_class"], np.uint8))
    nt = dem["n_trips"]
    d = sim_demand(nt, keep(dem["origin"], np.int32) if nt else None,
                   keep(dem["dest"], np.int32) if nt else None,
                   keep(dem["depart_step"], np.int32) if nt else None)
    p = sim_params(par["dt"], par["veh_len"], par["s_min"], par["n_class"],
                   keep(par["v0"], np.float32), keep(par["T"], np.float32), keep(par["a"], np.float32),
                   keep(par["b"], np.float32), keep(par["s0"], np.float32),
                   par["mobil_p"], par["mobil_athr"], par["mobil_bsafe"], par["mobil_bias_right"],
                   par["lambda_mand"], par["stop_acquire_m"], par["seed"] & (2**64 - 1),
                   par["cost_mode"], par["loop_routes"], int(par.get("max_device_bytes", 0)))
    return n, d, p


class Sim:
    """One simulation handle of libgbtraffic.

    ``Sim(scenario)`` wraps ``sim_create``; ``Sim.batch([scenarios])`` wraps
    ``sim_create_batch``.  Scenarios are the dicts of ``paper_1807_01148_gb300.scenarios``.
    """

    def __init__(self, scenario=None, *, _handle=None, n_trips=None, n_nodes=None, n_links=None):
        L = lib()
        self._max_windows = 0
        if _handle is not None:
            self.h = _handle
            self.n_trips = n_trips
            self.n_nodes = n_nodes
            self.n_links = n_links
        else:
            keep = _Keep()
            n, d, p = _structs(scenario, keep)
            h = C.c_void_p()
            rc = L.sim_create(C.byref(n), C.byref(d), C.byref(p), C.byref(h))
            if rc != SIM_OK:
                raise SimError(rc, L.sim_last_error(None).decode())
            self.h = h
            self.n_trips = scenario["demand"]["n_trips"]
            self.n_nodes = scenario["network"]["n_nodes"]
            self.n_links = scenario["network"]["n_links"]
        ln = C.c_int64()
        L.sim_n_lanes(self.h, C.byref(ln))
        self.n_lanes = ln.value

    @classmethod
    def batch(cls, scenarios):
        L = lib()
        keep = _Keep()
        structs = [_structs(s, keep) for s in scenarios]
        k = len(structs)
        nets = (C.POINTER(sim_network) * k)(*[C.pointer(s[0]) for s in structs])
        dems = (C.POINTER(sim_demand) * k)(*[C.pointer(s[1]) for s in structs])
        pars = (C.POINTER(sim_params) * k)(*[C.pointer(s[2]) for s in structs])
        h = C.c_void_p()
        rc = L.sim_create_batch(k, nets, dems, pars, C.byref(h))
        if rc != SIM_OK:
            raise SimError(rc, L.sim_last_error(None).decode())
        return cls(_handle=h, n_trips=sum(s["demand"]["n_trips"] for s in scenarios),
                   n_nodes=sum(s["network"]["n_nodes"] for s in scenarios),
                   n_links=sum(s["network"]["n_links"] for s in scenarios))

    def _check(self, rc):
        if rc != SIM_OK:
            raise SimError(rc, lib().sim_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib().sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_handle):
        """stream_handle: an integer cudaStream_t (e.g. torch.cuda.current_stream().cuda_stream)."""
        self._check(lib().sim_set_stream(self.h, C.c_void_p(stream_handle)))

    def route(self, costs=None):
        c = None if costs is None else np.ascontiguousarray(costs, np.int32)
        self._check(lib().sim_route(self.h, _p(c)))

    def set_routes(self, offsets, links):
        o = np.ascontiguousarray(offsets, np.int32)
        l_ = np.ascontiguousarray(links, np.int32)
        self._check(lib().sim_set_routes(self.h, _p(o), _p(l_)))

    def routes(self):
        n = C.c_int64()
        self._check(lib().sim_route_size(self.h, C.byref(n)))
        off = np.zeros(self.n_trips + 1, np.int32)
        links = np.zeros(max(1, n.value), np.int32)
        self._check(lib().sim_read_routes(self.h, _p(off), _p(links)))
        return off, links[: n.value]

    def step(self, n=1):
        self._check(lib().sim_step(self.h, int(n)))

    def step_timed(self, n=1):
        """Advance n steps with an event after every kernel; returns {kernel name: ms}."""
        nk = n_kernels()
        ms = np.zeros(nk, np.float32)
        self._check(lib().sim_step_timed(self.h, int(n), _p(ms)))
        return {lib().sim_kernel_name(k).decode(): float(ms[k]) for k in range(nk)}

    def state(self, fields=F_ALL):
        n = self.n_trips
        out = dict(status=np.zeros(n, np.uint8), link=np.zeros(n, np.int32), lane=np.zeros(n, np.int32),
                   cursor=np.zeros(n, np.int32), x=np.zeros(n, np.float32), v=np.zeros(n, np.float32),
                   insert_step=np.zeros(n, np.int32), arrive_step=np.zeros(n, np.int32),
                   lane_change=np.zeros(n, np.int8))
        names = ("status", "link", "lane", "cursor", "x", "v", "insert_step", "arrive_step", "lane_change")
        view = sim_state_view(*[out[k].ctypes.data if (fields >> i) & 1 else None for i, k in enumerate(names)])
        self._check(lib().sim_read_state(self.h, C.byref(view), fields, 0))
        return {k: out[k] for i, k in enumerate(names) if (fields >> i) & 1}

    def state_device(self, tensors: dict, fields: int, wait: bool = True):
        """Read fields into caller-owned device buffers (e.g. torch CUDA tensors).  wait
        False: only enqueued on the handle's stream (sim_read_state mode 2)."""
        names = ("status", "link", "lane", "cursor", "x", "v", "insert_step", "arrive_step", "lane_change")
        view = sim_state_view(*[tensors[k].data_ptr() if (fields >> i) & 1 else None for i, k in enumerate(names)])
        self._check(lib().sim_read_state(self.h, C.byref(view), fields, 1 if wait else 2))

    def write_state(self, st):
        self._check(lib().sim_write_state(
            self.h, _p(np.ascontiguousarray(st["status"], np.uint8)),
            _p(np.ascontiguousarray(st["link"], np.int32)), _p(np.ascontiguousarray(st["lane"], np.int32)),
            _p(np.ascontiguousarray(st["cursor"], np.int32)), _p(np.ascontiguousarray(st["x"], np.float32)),
            _p(np.ascontiguousarray(st["v"], np.float32))))

    def occupancy(self):
        start = np.zeros(self.n_lanes + 1, np.int32)
        vids = np.zeros(max(1, self.n_trips), np.int32)
        self._check(lib().sim_occupancy(self.h, _p(start), _p(vids)))
        return start, vids[: start[-1]]

    def set_class_params(self, v0, T, a, b, s0):
        arrs = [np.ascontiguousarray(q, np.float32) for q in (v0, T, a, b, s0)]
        self._check(lib().sim_set_class_params(self.h, *[_p(q) for q in arrs]))

    def observe(self, n_steps, obs_every):
        out = np.zeros((n_steps // obs_every, self.n_trips), np.float64)
        self._check(lib().sim_observe(self.h, int(n_steps), int(obs_every), _p(out)))
        return out

    def adjoint(self, n_steps, obs_every, target, n_class, checkpoint_every=64):
        """Loss and dL/d(v0, T, a, b, s0) per class from the current state (see sim_adjoint)."""
        t = np.ascontiguousarray(target, np.float64)
        spec = sim_loss_spec(int(n_steps), int(obs_every), int(checkpoint_every), t.ctypes.data)
        g = np.zeros(n_class * 5, np.float64)
        loss = np.zeros(1, np.float64)
        self._check(lib().sim_adjoint(self.h, C.byref(spec), _p(g), _p(loss)))
        return g.reshape(n_class, 5), float(loss[0])

    def loss(self, n_steps, obs_every, target):
        """The calibration loss alone, computed on the device from the current state (see
        sim_loss); the state advances by n_steps."""
        t = np.ascontiguousarray(target, np.float64)
        spec = sim_loss_spec(int(n_steps), int(obs_every), 0, t.ctypes.data)
        loss = np.zeros(1, np.float64)
        self._check(lib().sim_loss(self.h, C.byref(spec), _p(loss)))
        return float(loss[0])

    def set_exec(self, mode=SIM_EXEC_GRAPH, threads=256, blocks_per_sm=1, grid_per_sm=8,
                 barrier_timeout_cycles=0):
        e = sim_exec(mode, threads, blocks_per_sm, grid_per_sm, barrier_timeout_cycles)
        self._check(lib().sim_set_exec(self.h, C.byref(e)))

    def get_exec(self):
        e = sim_exec()
        self._check(lib().sim_get_exec(self.h, C.byref(e)))
        return e.as_dict()

    def autotune(self, trial_steps=20, cache_path=None):
        e = sim_exec()
        self._check(lib().sim_autotune(self.h, int(trial_steps),
                                       cache_path.encode() if cache_path else None, C.byref(e)))
        return e.as_dict()

    # ---- measured outputs (Eq. 8-9, Sec. 6.3.1, Sec. 6.4)
    def set_outputs(self, flags, sample_every=120, per_window=6, max_windows=0):
        smp = sim_sampling(int(sample_every), int(per_window), int(max_windows))
        self._check(lib().sim_set_outputs(self.h, int(flags), C.byref(smp)))
        self._max_windows = int(max_windows) if flags & OUT_EDGE_SAMPLES else 0

    def reset_outputs(self):
        self._check(lib().sim_reset_outputs(self.h))

    def emissions(self):
        fuel = np.zeros(self.n_trips, np.float64)
        co = np.zeros(self.n_trips, np.float64)
        self._check(lib().sim_read_emissions(self.h, _p(fuel), _p(co)))
        return fuel, co

    def link_times(self):
        s = np.zeros(self.n_links, np.int64)
        n = np.zeros(self.n_links, np.int32)
        self._check(lib().sim_read_link_times(self.h, _p(s), _p(n)))
        return s, n

    def edge_samples(self):
        w = self._max_windows
        u = np.zeros((w, self.n_links), np.float64)
        sp = np.zeros((w, self.n_links), np.float64)
        n = np.zeros(w, np.int32)
        self._check(lib().sim_read_edge_samples(self.h, _p(u), _p(sp), _p(n)))
        return u, sp, n

    def measured_costs(self, prev):
        prev = np.ascontiguousarray(prev, np.int32)
        out = np.zeros(self.n_links, np.int32)
        gap = np.zeros(1, np.float64)
        self._check(lib().sim_measured_costs(self.h, _p(prev), _p(out), _p(gap)))
        return out, float(gap[0])

    def reroute(self, costs, fraction_q16, round_):
        c = np.ascontiguousarray(costs, np.int32)
        self._check(lib().sim_reroute(self.h, _p(c), int(fraction_q16), int(round_)))

    def equilibrium(self, fractions_q16, n_steps):
        f = np.ascontiguousarray(fractions_q16, np.uint32)
        cost = np.zeros(self.n_links, np.int32)
        gap = np.zeros(len(f), np.float64)
        self._check(lib().sim_equilibrium(self.h, len(f), _p(f), int(n_steps), _p(cost), _p(gap)))
        return cost, gap

    def set_vehicle_types(self, types, trip_type):
        """types: list of (length_m, accel_scale, max_speed_mps); trip_type: per-trip index
        (Sec. 6.3.5 trucks).  An empty list returns to the single vehicle class."""
        n = len(types)
        arr = (sim_vehicle_type * max(1, n))(*[sim_vehicle_type(*map(float, t)) for t in types])
        tt = np.ascontiguousarray(trip_type, np.uint8) if n else None
        self._check(lib().sim_set_vehicle_types(self.h, n, arr, _p(tt)))

    # ---- static user equilibrium (Sec. 5.2, Eq. 3, Eq. 6)
    def assign_static(self, capacity, alpha=0.15, beta=4, max_iter=20, bisect_iter=30):
        cap = np.ascontiguousarray(capacity, np.float64)
        spec = sim_assign_spec(cap.ctypes.data, float(alpha), int(beta), int(max_iter), int(bisect_iter))
        flow = np.zeros(self.n_links, np.float64)
        time = np.zeros(self.n_links, np.float64)
        gap = np.zeros(max(1, max_iter), np.float64)
        step = np.zeros(max(1, max_iter), np.float64)
        obj = np.zeros(max_iter + 1, np.float64)
        self._check(lib().sim_assign_static(self.h, C.byref(spec), _p(flow), _p(time), _p(gap), _p(step), _p(obj)))
        return dict(flow=flow, time=time, gap=gap[:max_iter], step=step[:max_iter], objective=obj)

    def launch_count(self):
        """Kernel launches sim_step has made on this handle (sim_launch_count)."""
        n = C.c_int64()
        self._check(lib().sim_launch_count(self.h, C.byref(n)))
        return int(n.value)

    def counters(self):
        c = sim_counters_t()
        self._check(lib().sim_counters(self.h, C.byref(c)))
        return {k: getattr(c, k) for k, _ in sim_counters_t._fields_}


def setup(scenario, sim=None):
    """Create (or reuse) a handle and give it the scenario's routes and initial state."""
    s = sim or Sim(scenario)
    if "routes" in scenario:
        s.set_routes(scenario["routes"]["offsets"], scenario["routes"]["links"])
    else:
        s.route()
    if "init_state" in scenario:
        s.write_state(scenario["init_state"])
    return s


PARAM_ORDER = ("v0", "T", "a", "b", "s0")


def calibration_loss_fn():
    """torch.autograd.Function for trajectory calibration: loss(theta), theta a
    [n_class, 5] float64 tensor of (v0, T, a, b, s0) per class.  Forward sets the class
    parameters, restores the start state and runs sim_adjoint (taped forward pass with
    checkpoints + binary64 reverse sweep) when a gradient is needed, sim_loss (the
    loss alone, on the device) otherwise; backward returns the stored gradient scaled by the incoming one."""
    import torch

    class CalibrationLoss(torch.autograd.Function):
        @staticmethod
        def forward(ctx, theta, sim, start_state, target, n_steps, obs_every, checkpoint_every):
            th = theta.detach().cpu().double().numpy()
            sim.set_class_params(*[th[:, k] for k in range(5)])
            sim.write_state(start_state)
            if theta.requires_grad:
                g, loss = sim.adjoint(n_steps, obs_every, target, th.shape[0], checkpoint_every)
                ctx.save_for_backward(torch.from_numpy(g).to(theta.device, theta.dtype))
            else:
                loss = sim.loss(n_steps, obs_every, target)
            return torch.tensor(loss, dtype=theta.dtype, device=theta.device)

        @staticmethod
        def backward(ctx, gout):
            (g,) = ctx.saved_tensors
            return gout * g, None, None, None, None, None, None

    return CalibrationLoss
