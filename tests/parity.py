"""Helpers that run the CUDA library and the CPU oracle side by side on the same
seeded scenario and compare their results element by element (bit patterns for
binary32 state, exact equality for integers)."""
from __future__ import annotations

import numpy as np

STATE_KEYS = ("status", "link", "lane", "cursor", "x", "v", "insert_step", "arrive_step", "lane_change")


def setup_pair(sc, sim_cls, oracle_cls):
    g = sim_cls(sc)
    o = oracle_cls(sc)
    if "routes" in sc:
        g.set_routes(sc["routes"]["offsets"], sc["routes"]["links"])
        o.set_routes(sc["routes"]["offsets"], sc["routes"]["links"])
    else:
        g.route()
        o.route()
    if "init_state" in sc:
        g.write_state(sc["init_state"])
        o.write_state(sc["init_state"])
    return g, o


def diff_state(a: dict, b: dict, keys=STATE_KEYS):
    """Return a list of (field, first differing vids, values) for fields that differ."""
    out = []
    for k in keys:
        x, y = a[k], b[k]
        if x.dtype == np.float32:
            x, y = x.view(np.uint32), y.view(np.uint32)
        bad = np.flatnonzero(x != y)
        if len(bad):
            out.append((k, bad[:8].tolist(), a[k][bad[:8]].tolist(), b[k][bad[:8]].tolist(), len(bad)))
    return out


def compare(g, o, label="", check_occ=True):
    sg, so = g.state(), o.state()
    d = diff_state(sg, so)
    assert not d, f"{label}: state differs (field, vids, gpu, oracle, count): {d}"
    cg, co = g.counters(), o.counters()
    for k in ("t", "departed", "waiting", "active", "arrived", "veh_steps", "pending", "active_last", "lc_evals"):
        assert cg[k] == co[k], f"{label}: counter {k} gpu {cg[k]} oracle {co[k]}"
    if check_occ:
        lg, vg = g.occupancy()
        lo, vo = o.occupancy()
        assert np.array_equal(lg, lo), f"{label}: lane_start differs"
        assert np.array_equal(vg, vo), f"{label}: sorted vids differ at {np.flatnonzero(vg != vo)[:8]}"
    return sg


def run_lockstep(g, o, steps, every, check_occ=True):
    done = 0
    compare(g, o, "start", check_occ)
    while done < steps:
        n = min(every, steps - done)
        g.step(n)
        o.step(n)
        done += n
        compare(g, o, f"after step {done}", check_occ)
    return done
