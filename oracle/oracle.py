"""ctypes wrapper of the C oracle (test infrastructure only; never used by the product path)."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with plain gcc (no fused multiply-add, no fast-math)."""
    with _lock:
        if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < max(
                os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
            tmp = _SO + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
                                   "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _SO)
    return _SO


class _Net(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("n_links", C.c_int32),
                ("node_x_dm", C.c_void_p), ("node_y_dm", C.c_void_p), ("node_control", C.c_void_p),
                ("signal_offset_ds", C.c_void_p), ("signal_cycle_ds", C.c_void_p),
                ("signal_green_ds", C.c_void_p), ("link_from", C.c_void_p), ("link_to", C.c_void_p),
                ("link_length_m", C.c_void_p), ("link_speed_mps", C.c_void_p),
                ("link_lanes", C.c_void_p), ("link_class", C.c_void_p)]


class _Dem(C.Structure):
    _fields_ = [("n_trips", C.c_int32), ("origin", C.c_void_p), ("dest", C.c_void_p),
                ("depart_step", C.c_void_p)]


class _Par(C.Structure):
    _fields_ = [("dt", C.c_float), ("veh_len", C.c_float), ("s_min", C.c_float),
                ("n_class", C.c_int32),
                ("v0", C.c_void_p), ("T", C.c_void_p), ("a", C.c_void_p), ("b", C.c_void_p),
                ("s0", C.c_void_p),
                ("mobil_p", C.c_float), ("mobil_athr", C.c_float), ("mobil_bsafe", C.c_float),
                ("mobil_bias_right", C.c_float), ("lambda_mand", C.c_float),
                ("stop_acquire_m", C.c_float), ("seed", C.c_uint64),
                ("cost_mode", C.c_int32), ("loop_routes", C.c_int32)]


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        vp, i32, i64, f32 = C.c_void_p, C.c_int32, C.c_int64, C.c_float
        L.orc_create.argtypes = [C.POINTER(_Net), C.POINTER(_Dem), C.POINTER(_Par), C.POINTER(vp)]
        L.orc_destroy.argtypes = [vp]
        L.orc_route.argtypes = [vp, vp]
        L.orc_set_routes.argtypes = [vp, vp, vp]
        L.orc_route_size.argtypes = [vp, C.POINTER(i64)]
        L.orc_read_routes.argtypes = [vp, vp, vp]
        L.orc_write_state.argtypes = [vp] + [vp] * 6
        L.orc_step.argtypes = [vp, i32]
        L.orc_read_state.argtypes = [vp] + [vp] * 9
        L.orc_occupancy.argtypes = [vp, vp, vp]
        L.orc_n_lanes.argtypes = [vp]
        L.orc_counters.argtypes = [vp, vp]
        L.orc_node_holder.argtypes = [vp, vp]
        L.orc_observe.argtypes = [vp, i32, i32, vp]
        L.orc_adjoint.argtypes = [vp, i32, i32, vp, vp, vp]
        L.orc_replay_loss.argtypes = [vp] + [vp] * 6
        L.orc_set_class_params.argtypes = [vp] * 6
        L.orc_record.argtypes = [vp, i32]
        L.orc_tape_digest.argtypes = [vp, vp, vp, vp]
        L.orc_idm.argtypes = [f32] * 9 + [C.c_int]
        L.orc_idm.restype = f32
        L.orc_ballistic.argtypes = [f32, f32, f32, f32, C.POINTER(f32), C.POINTER(f32)]
        L.orc_link_cost.argtypes = [f32, f32, C.c_int, C.c_int]
        L.orc_link_cost.restype = i32
        L.orc_sssp.argtypes = [i32, i32, vp, vp, vp, i32, vp]
        L.orc_mand_index.argtypes = [C.c_uint64, i32, i32]
        L.orc_mand_index.restype = C.c_uint32
        L.orc_mand_tau.argtypes = [C.c_int]
        L.orc_mand_tau.restype = f32
        L.orc_turn.argtypes = [i64] * 6
        L.orc_signal_green.argtypes = [i64, i32, i32, i32, i32, C.c_int]
        u32 = C.c_uint32
        L.orc_set_outputs.argtypes = [vp, u32, i32, i32, i32]
        L.orc_reset_outputs.argtypes = [vp]
        L.orc_read_emissions.argtypes = [vp, vp, vp]
        L.orc_read_link_times.argtypes = [vp, vp, vp]
        L.orc_read_edge_samples.argtypes = [vp, vp, vp, vp]
        L.orc_measured_costs.argtypes = [vp, vp, vp, vp]
        L.orc_reroute.argtypes = [vp, vp, u32, u32]
        L.orc_equilibrium.argtypes = [vp, i32, vp, i32, vp, vp]
        L.orc_reroute_selected.argtypes = [C.c_uint64, i32, u32, u32]
        L.orc_set_vehicle_types.argtypes = [vp, i32, vp, vp, vp, vp]
        L.orc_assign_static.argtypes = [vp, vp, C.c_double, i32, i32, i32, vp, vp, vp, vp, vp]
        L.orc_aon.argtypes = [vp, vp, vp]
        L.orc_co_rate.argtypes = [f32]
        L.orc_co_rate.restype = f32
        L.orc_fuel_rate.argtypes = [f32, f32]
        L.orc_fuel_rate.restype = f32
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class OracleError(RuntimeError):
    pass


def _check(rc, what):
    if rc != 0:
        raise OracleError(f"{what} failed with code {rc}")


class OracleSim:
    """One simulation instance of the oracle (same inputs as the CUDA library)."""

    def __init__(self, scenario: dict):
        L = lib()
        net, dem, par = scenario["network"], scenario["demand"], scenario["params"]
        self._keep = []

        def arr(a, dt):
            a = np.ascontiguousarray(a, dtype=dt)
            self._keep.append(a)
            return _p(a)
        n = _Net(net["n_nodes"], net["n_links"], arr(net["node_x_dm"], np.int32),
                 arr(net["node_y_dm"], np.int32), arr(net["node_control"], np.uint8),
                 arr(net["signal_offset_ds"], np.int32), arr(net["signal_cycle_ds"], np.int32),
                 arr(net["signal_green_ds"], np.int32), arr(net["link_from"], np.int32),
                 arr(net["link_to"], np.int32), arr(net["link_length_m"], np.float32),
                 arr(net["link_speed_mps"], np.float32), arr(net["link_lanes"], np.uint8),
                 arr(net["link_class"], np.uint8))
        d = _Dem(dem["n_trips"], arr(dem["origin"], np.int32), arr(dem["dest"], np.int32),
                 arr(dem["depart_step"], np.int32))
        p = _Par(par["dt"], par["veh_len"], par["s_min"], par["n_class"],
                 arr(par["v0"], np.float32), arr(par["T"], np.float32), arr(par["a"], np.float32),
                 arr(par["b"], np.float32), arr(par["s0"], np.float32),
                 par["mobil_p"], par["mobil_athr"], par["mobil_bsafe"], par["mobil_bias_right"],
                 par["lambda_mand"], par["stop_acquire_m"], par["seed"] & (2**64 - 1),
                 par["cost_mode"], par["loop_routes"])
        h = C.c_void_p()
        _check(L.orc_create(C.byref(n), C.byref(d), C.byref(p), C.byref(h)), "orc_create")
        self._keep = []
        self.h = h
        self.n_trips = dem["n_trips"]
        self.n_nodes = net["n_nodes"]
        self.n_links = net["n_links"]
        self._max_windows = 0
        self.n_lanes = L.orc_n_lanes(h)

    def close(self):
        if self.h:
            lib().orc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def route(self, costs=None):
        c = None if costs is None else np.ascontiguousarray(costs, np.int32)
        _check(lib().orc_route(self.h, _p(c)), "orc_route")

    def set_routes(self, offsets, links):
        o = np.ascontiguousarray(offsets, np.int32)
        l_ = np.ascontiguousarray(links, np.int32)
        _check(lib().orc_set_routes(self.h, _p(o), _p(l_)), "orc_set_routes")

    def routes(self):
        n = C.c_int64()
        _check(lib().orc_route_size(self.h, C.byref(n)), "orc_route_size")
        off = np.zeros(self.n_trips + 1, np.int32)
        links = np.zeros(max(1, n.value), np.int32)
        _check(lib().orc_read_routes(self.h, _p(off), _p(links)), "orc_read_routes")
        return off, links[: n.value]

    def write_state(self, st):
        _check(lib().orc_write_state(
            self.h, _p(np.ascontiguousarray(st["status"], np.uint8)),
            _p(np.ascontiguousarray(st["link"], np.int32)),
            _p(np.ascontiguousarray(st["lane"], np.int32)),
            _p(np.ascontiguousarray(st["cursor"], np.int32)),
            _p(np.ascontiguousarray(st["x"], np.float32)),
            _p(np.ascontiguousarray(st["v"], np.float32))), "orc_write_state")

    def step(self, n=1):
        _check(lib().orc_step(self.h, int(n)), "orc_step")

    def state(self):
        n = self.n_trips
        out = dict(status=np.zeros(n, np.uint8), link=np.zeros(n, np.int32), lane=np.zeros(n, np.int32),
                   cursor=np.zeros(n, np.int32), x=np.zeros(n, np.float32), v=np.zeros(n, np.float32),
                   insert_step=np.zeros(n, np.int32), arrive_step=np.zeros(n, np.int32),
                   lane_change=np.zeros(n, np.int8))
        _check(lib().orc_read_state(self.h, *[_p(out[k]) for k in
                                              ("status", "link", "lane", "cursor", "x", "v",
                                               "insert_step", "arrive_step", "lane_change")]),
               "orc_read_state")
        return out

    def occupancy(self):
        start = np.zeros(self.n_lanes + 1, np.int32)
        vids = np.zeros(max(1, self.n_trips), np.int32)
        _check(lib().orc_occupancy(self.h, _p(start), _p(vids)), "orc_occupancy")
        return start, vids[: start[-1]]

    def counters(self):
        c = np.zeros(9, np.int64)
        _check(lib().orc_counters(self.h, _p(c)), "orc_counters")
        keys = ("t", "departed", "waiting", "active", "arrived", "veh_steps", "pending", "active_last", "lc_evals")
        return {k: int(v) for k, v in zip(keys, c)}

    def set_class_params(self, v0, T, a, b, s0):
        arrs = [np.ascontiguousarray(q, np.float32) for q in (v0, T, a, b, s0)]
        _check(lib().orc_set_class_params(self.h, *[_p(q) for q in arrs]), "orc_set_class_params")

    def observe(self, n_steps, obs_every):
        out = np.zeros((n_steps // obs_every, self.n_trips), np.float64)
        _check(lib().orc_observe(self.h, int(n_steps), int(obs_every), _p(out)), "orc_observe")
        return out

    def adjoint(self, n_steps, obs_every, target, n_class):
        t = np.ascontiguousarray(target, np.float64)
        g = np.zeros(n_class * 5, np.float64)
        loss = np.zeros(1, np.float64)
        _check(lib().orc_adjoint(self.h, int(n_steps), int(obs_every), _p(t), _p(g), _p(loss)), "orc_adjoint")
        return g, float(loss[0])

    def replay_loss(self, v0, T, a, b, s0):
        arrs = [np.ascontiguousarray(q, np.float64) for q in (v0, T, a, b, s0)]
        loss = np.zeros(1, np.float64)
        _check(lib().orc_replay_loss(self.h, *[_p(q) for q in arrs], _p(loss)), "orc_replay_loss")
        return float(loss[0])

    # ---- measured outputs (Eq. 8-9, Sec. 6.3.1, Sec. 6.4)
    def record(self, n_steps):
        """Run n_steps with the adjoint's tape recorded (no observation, no sweep)."""
        _check(lib().orc_record(self.h, int(n_steps)), "orc_record")

    def tape_digest(self, per_step=False):
        """(digest, records) of the discrete decisions of the last recorded run; with
        per_step also the array whose entry j digests steps 0 .. j-1."""
        dg = np.zeros(1, np.uint64)
        n = np.zeros(1, np.int64)
        steps = np.zeros(max(1, int(self.counters()["t"])) + 1, np.uint64) if per_step else None
        _check(lib().orc_tape_digest(self.h, _p(dg), _p(n), _p(steps) if per_step else None), "orc_tape_digest")
        return (int(dg[0]), int(n[0]), steps) if per_step else (int(dg[0]), int(n[0]))

    def set_outputs(self, flags, sample_every=120, per_window=6, max_windows=0):
        _check(lib().orc_set_outputs(self.h, int(flags), int(sample_every), int(per_window), int(max_windows)),
               "orc_set_outputs")
        self._max_windows = int(max_windows) if flags & 4 else 0

    def reset_outputs(self):
        _check(lib().orc_reset_outputs(self.h), "orc_reset_outputs")

    def emissions(self):
        fuel = np.zeros(self.n_trips, np.float64)
        co = np.zeros(self.n_trips, np.float64)
        _check(lib().orc_read_emissions(self.h, _p(fuel), _p(co)), "orc_read_emissions")
        return fuel, co

    def link_times(self):
        s = np.zeros(self.n_links, np.int64)
        n = np.zeros(self.n_links, np.int32)
        _check(lib().orc_read_link_times(self.h, _p(s), _p(n)), "orc_read_link_times")
        return s, n

    def edge_samples(self):
        w = self._max_windows
        u = np.zeros((w, self.n_links), np.float64)
        sp = np.zeros((w, self.n_links), np.float64)
        n = np.zeros(w, np.int32)
        _check(lib().orc_read_edge_samples(self.h, _p(u), _p(sp), _p(n)), "orc_read_edge_samples")
        return u, sp, n

    def measured_costs(self, prev):
        prev = np.ascontiguousarray(prev, np.int32)
        out = np.zeros(self.n_links, np.int32)
        gap = np.zeros(1, np.float64)
        _check(lib().orc_measured_costs(self.h, _p(prev), _p(out), _p(gap)), "orc_measured_costs")
        return out, float(gap[0])

    def reroute(self, costs, fraction_q16, round_):
        c = np.ascontiguousarray(costs, np.int32)
        _check(lib().orc_reroute(self.h, _p(c), int(fraction_q16), int(round_)), "orc_reroute")

    def equilibrium(self, fractions_q16, n_steps):
        f = np.ascontiguousarray(fractions_q16, np.uint32)
        cost = np.zeros(self.n_links, np.int32)
        gap = np.zeros(len(f), np.float64)
        _check(lib().orc_equilibrium(self.h, len(f), _p(f), int(n_steps), _p(cost), _p(gap)), "orc_equilibrium")
        return cost, gap

    def set_vehicle_types(self, types, trip_type):
        """types: list of (length_m, accel_scale, max_speed_mps); trip_type: per-trip index."""
        n = len(types)
        cols = [np.ascontiguousarray([t[k] for t in types], np.float32) for k in range(3)] if n else [None] * 3
        tt = np.ascontiguousarray(trip_type, np.uint8) if n else None
        _check(lib().orc_set_vehicle_types(self.h, n, *[_p(c) for c in cols], _p(tt)), "orc_set_vehicle_types")

    # ---- static user equilibrium (Sec. 5.2, Eq. 3, Eq. 6)
    def assign_static(self, capacity, alpha=0.15, beta=4, max_iter=20, bisect_iter=30):
        cap = np.ascontiguousarray(capacity, np.float64)
        flow = np.zeros(self.n_links, np.float64)
        time = np.zeros(self.n_links, np.float64)
        gap = np.zeros(max(1, max_iter), np.float64)
        step = np.zeros(max(1, max_iter), np.float64)
        obj = np.zeros(max_iter + 1, np.float64)
        _check(lib().orc_assign_static(self.h, _p(cap), float(alpha), int(beta), int(max_iter), int(bisect_iter),
                                       _p(flow), _p(time), _p(gap), _p(step), _p(obj)), "orc_assign_static")
        return dict(flow=flow, time=time, gap=gap[:max_iter], step=step[:max_iter], objective=obj)

    def aon(self, costs):
        c = np.ascontiguousarray(costs, np.int32)
        flow = np.zeros(self.n_links, np.float64)
        _check(lib().orc_aon(self.h, _p(c), _p(flow)), "orc_aon")
        return flow

    def node_holder(self):
        h = np.zeros(self.n_nodes, np.int32)
        _check(lib().orc_node_holder(self.h, _p(h)), "orc_node_holder")
        return h


def oracle_idm(a, b, T, s0, v0, s_min, s, v, v_lead, has_leader=True):
    return lib().orc_idm(a, b, T, s0, v0, s_min, s, v, v_lead, int(has_leader))


def oracle_ballistic(x, v, acc, dt):
    xo, vo = C.c_float(), C.c_float()
    lib().orc_ballistic(x, v, acc, dt, C.byref(xo), C.byref(vo))
    return xo.value, vo.value


def oracle_link_cost(length, speed, lanes=1, mode=0):
    return lib().orc_link_cost(length, speed, lanes, mode)


def oracle_sssp(n_nodes, link_from, link_to, cost, origin):
    lf = np.ascontiguousarray(link_from, np.int32)
    lt = np.ascontiguousarray(link_to, np.int32)
    c = np.ascontiguousarray(cost, np.int32)
    dist = np.zeros(n_nodes, np.int64)
    _check(lib().orc_sssp(n_nodes, len(lf), _p(lf), _p(lt), _p(c), origin, _p(dist)), "orc_sssp")
    return dist


def oracle_mand_index(seed, vid, hop):
    return lib().orc_mand_index(seed & (2**64 - 1), vid, hop)


def oracle_mand_tau(k):
    return lib().orc_mand_tau(k)


def oracle_turn(a, b, c):
    return lib().orc_turn(a[0], a[1], b[0], b[1], c[0], c[1])


def oracle_signal_green(t, dt_ds, offset, cycle, green, ew):
    return lib().orc_signal_green(t, dt_ds, offset, cycle, green, int(ew))


def oracle_reroute_selected(seed, vid, round_, fraction_q16):
    return bool(lib().orc_reroute_selected(seed & (2**64 - 1), vid, round_, fraction_q16))


def oracle_co_rate(v):
    return lib().orc_co_rate(v)


def oracle_fuel_rate(v, a):
    return lib().orc_fuel_rate(v, a)
