"""The batched ensemble at its configured size, bit for bit against the oracle.

64 grid scenarios of uneven size (side 10, 15, 20, 30 or 40 intersections, 200 m links,
2 lanes, signals; 5,000 to 80,000 trips scaled to the network; departures over the
first hour; per-scenario IDM parameters), all 7,200 steps, in one batched handle
(sim_create_batch: the disjoint union of the scenarios).  Every 1,200 steps each
scenario's slice of the batched state (status, link, lane, route cursor, x, v,
insertion and arrival steps, lane-change decisions) must equal the oracle's run of
that scenario alone, field by field (compared by SHA-256 of the bytes), and at the end
the batched counters must equal the sums of the oracle's.  The oracle scenarios run in
a process pool started with spawn before the first GPU call."""
import hashlib
import multiprocessing as mp

import numpy as np
import pytest

from paper_1807_01148_gb300 import scenarios as S

from .parity import STATE_KEYS

pytestmark = pytest.mark.gpu

EVERY = 1200
COUNTERS = ("departed", "arrived", "veh_steps", "lc_evals", "active", "waiting", "pending")


def _digest(st):
    return {k: hashlib.sha256(np.ascontiguousarray(st[k]).tobytes()).hexdigest() for k in STATE_KEYS}


def _oracle_run(k):
    """Scenario k of the ensemble, run alone by the oracle: digests every EVERY steps."""
    import oracle
    sc = S.ensemble()[k]
    o = oracle.OracleSim(sc)
    o.route()
    out = []
    for _ in range(sc["steps"] // EVERY):
        o.step(EVERY)
        out.append(_digest(o.state()))
    c = o.counters()
    return out, {q: int(c[q]) for q in COUNTERS}


def test_ensemble_64_scenarios_7200_steps_bitexact():
    scs = S.ensemble()
    assert len(scs) == 64 and all(sc["steps"] == 7200 for sc in scs)
    sides = sorted({int(round(sc["network"]["n_nodes"] ** 0.5)) for sc in scs})
    assert set(sides) <= {10, 15, 20, 30, 40} and len(sides) >= 4
    # the biggest scenarios first, so that the pool's last jobs are short
    order = sorted(range(len(scs)), key=lambda k: -scs[k]["demand"]["n_trips"])
    pool = mp.get_context("spawn").Pool(min(16, mp.cpu_count()))
    try:
        pending = {k: pool.apply_async(_oracle_run, (k,)) for k in order}
        from paper_1807_01148_gb300 import gbtraffic as G
        b = G.Sim.batch(scs)
        b.route()
        gpu = [[] for _ in scs]
        for _ in range(7200 // EVERY):
            b.step(EVERY)
            sb = b.state()
            base = link_base = 0
            for k, sc in enumerate(scs):
                n = sc["demand"]["n_trips"]
                sl = {q: v[base:base + n].copy() for q, v in sb.items()}
                act = sl["status"] == 1
                sl["link"][act] -= link_base
                gpu[k].append(_digest(sl))
                base += n
                link_base += sc["network"]["n_links"]
        cb = b.counters()
        b.close()
        tot = {q: 0 for q in COUNTERS}
        for k in order:
            ref, cnt = pending[k].get(timeout=3000)
            for j, (dg, do) in enumerate(zip(gpu[k], ref)):
                bad = [q for q in STATE_KEYS if dg[q] != do[q]]
                assert not bad, f"scenario {k} ({scs[k]['name']}) differs after {(j + 1) * EVERY} steps in {bad}"
            for q in COUNTERS:
                tot[q] += cnt[q]
    finally:
        pool.terminate()
        pool.join()
    for q in COUNTERS:
        assert cb[q] == tot[q], (q, cb[q], tot[q])
    assert tot["arrived"] > 0.5 * sum(sc["demand"]["n_trips"] for sc in scs)
