"""Seeded synthetic inputs for the traffic microsimulation (networks, demand, parameters).

This module is the only code the CUDA path and the CPU oracle have in common.  It
draws inputs and holds none of the method's arithmetic: no link costs, no turn or
lane-mask rules, no car-following, no signal logic.  Every scenario is a plain dict
of numpy arrays that both sides take as input.

Stand-ins for the paper's data (Sec. 4 builds the Bay Area network from
OpenStreetMap; Sec. 3 produces the OD table with ActivitySim; neither is available
here):

* ``ring``      single-lane ring road used to check car following (Sec. 6, Eq. 7).
* ``grid``      Manhattan grid with fixed-time signals (Sec. 6, intersection control).
* ``metro``     planar lattice-based road hierarchy of metropolitan size, lognormal
                link lengths, gravity OD and a bimodal (AM/PM) departure mixture,
                shaped like the Bay Area run of Sec. 6 (31 k nodes / 66 k edges there;
                225 k nodes / ~550 k links here).
* ``ensemble``  many independent grid scenarios with per-scenario IDM parameters.
* ``calib``     the grid with three link classes and perturbed target parameters.

Node positions are integer decimetres, lengths are float32 metres, speeds float32 m/s,
departure times are integer step indices (dt = 0.5 s, Sec. 6 "Per-vehicle ... simulation").
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 1807011480

CTRL_NONE, CTRL_STOP, CTRL_SIGNAL = 0, 1, 2
ST_PENDING, ST_ACTIVE, ST_ARRIVED = 0, 1, 2


def default_params(n_class: int = 1, **over) -> dict:
    """Model parameters.  IDM defaults follow Treiber et al. (2000), the source Sec. 6
    cites for the per-vehicle driver variables; MOBIL constants follow Kesting et al. (2007).
    ``v0 <= 0`` for a class means "use the link speed limit" (Sec. 6: v0 is the edge speed limit)."""
    p = dict(
        dt=0.5, veh_len=5.0, s_min=0.1,
        n_class=n_class,
        v0=[0.0] * n_class, T=[1.5] * n_class, a=[1.0] * n_class,
        b=[1.5] * n_class, s0=[2.0] * n_class,
        mobil_p=0.2, mobil_athr=0.1, mobil_bsafe=4.0, mobil_bias_right=0.0,
        lambda_mand=100.0, stop_acquire_m=3.0,
        seed=BASE_SEED, cost_mode=0, loop_routes=0,
    )
    p.update(over)
    return p


def _net(n_nodes, nx_dm, ny_dm, ctrl, off, cyc, grn, lf, lt, length, speed, lanes, cls):
    return dict(
        n_nodes=int(n_nodes), n_links=int(len(lf)),
        node_x_dm=np.ascontiguousarray(nx_dm, np.int32),
        node_y_dm=np.ascontiguousarray(ny_dm, np.int32),
        node_control=np.ascontiguousarray(ctrl, np.uint8),
        signal_offset_ds=np.ascontiguousarray(off, np.int32),
        signal_cycle_ds=np.ascontiguousarray(cyc, np.int32),
        signal_green_ds=np.ascontiguousarray(grn, np.int32),
        link_from=np.ascontiguousarray(lf, np.int32),
        link_to=np.ascontiguousarray(lt, np.int32),
        link_length_m=np.ascontiguousarray(length, np.float32),
        link_speed_mps=np.ascontiguousarray(speed, np.float32),
        link_lanes=np.ascontiguousarray(lanes, np.uint8),
        link_class=np.ascontiguousarray(cls, np.uint8),
    )


def _demand(o, d, dep):
    return dict(n_trips=int(len(o)),
                origin=np.ascontiguousarray(o, np.int32),
                dest=np.ascontiguousarray(d, np.int32),
                depart_step=np.ascontiguousarray(dep, np.int32))


# --------------------------------------------------------------------------- ring
def ring(n_veh: int = 50, circumference: float = 1000.0, jitter: float = 2.0,
         steps: int = 3600, v_init: float = 0.0, seed: int = BASE_SEED + 0) -> dict:
    """Single-lane ring: one node, one self-loop link (the paper's network is a
    multigraph with self-loops, Sec. 4).  Vehicles start evenly spaced with uniform
    jitter; every route is the loop link, followed forever."""
    rng = np.random.default_rng(seed)
    net = _net(1, [0], [0], [CTRL_NONE], [0], [600], [300], [0], [0],
               [circumference], [30.0], [1], [0])
    dem = _demand(np.zeros(n_veh), np.zeros(n_veh), np.zeros(n_veh))
    spacing = circumference / n_veh
    x = np.arange(n_veh) * spacing + spacing / 2 + rng.uniform(-jitter, jitter, n_veh)
    init = dict(status=np.full(n_veh, ST_ACTIVE, np.uint8),
                link=np.zeros(n_veh, np.int32), lane=np.zeros(n_veh, np.int32),
                cursor=np.zeros(n_veh, np.int32),
                x=x.astype(np.float32), v=np.full(n_veh, v_init, np.float32))
    routes = dict(offsets=np.arange(n_veh + 1, dtype=np.int32),
                  links=np.zeros(n_veh, np.int32))
    par = default_params(1, v0=[30.0], loop_routes=1, seed=seed)
    return dict(name="ring", network=net, demand=dem, params=par, routes=routes,
                init_state=init, steps=steps)


# --------------------------------------------------------------------------- grid
def _grid_network(n: int, spacing: float, lanes: int, speed: float, rng,
                  cycle_ds=600, green_ds=300):
    ids = np.arange(n * n).reshape(n, n)          # ids[j, i]: row j (y), column i (x)
    jj, ii = np.divmod(np.arange(n * n), n)
    xs = (ii * spacing * 10).round().astype(np.int64)
    ys = (jj * spacing * 10).round().astype(np.int64)
    lf, lt = [], []
    for j in range(n):
        for i in range(n):
            u = ids[j, i]
            for di, dj in ((1, 0), (0, 1), (-1, 0), (0, -1)):   # E, N, W, S
                a, b = i + di, j + dj
                if 0 <= a < n and 0 <= b < n:
                    lf.append(u)
                    lt.append(ids[b, a])
    lf = np.array(lf)
    lt = np.array(lt)
    nl = len(lf)
    off = rng.integers(0, cycle_ds, n * n)
    net = _net(n * n, xs, ys, np.full(n * n, CTRL_SIGNAL), off,
               np.full(n * n, cycle_ds), np.full(n * n, green_ds), lf, lt,
               np.full(nl, spacing), np.full(nl, speed), np.full(nl, lanes),
               np.zeros(nl))
    return net


def _uniform_od(n_nodes: int, n_trips: int, window_steps: int, rng):
    o = rng.integers(0, n_nodes, n_trips)
    d = rng.integers(0, n_nodes, n_trips)
    same = o == d
    while same.any():
        d[same] = rng.integers(0, n_nodes, int(same.sum()))
        same = o == d
    dep = rng.integers(0, window_steps, n_trips)
    return _demand(o, d, dep)


def grid(n: int = 20, n_trips: int = 20000, steps: int = 9000, spacing: float = 200.0,
         lanes: int = 2, speed: float = 13.9, depart_window_s: float = 3600.0,
         seed: int = BASE_SEED + 1) -> dict:
    """n x n signalised Manhattan grid, 4-neighbour two-way links, fixed-time two-phase
    signals 30 s / 30 s with offsets uniform on [0, 60) s, uniform OD (o != d) and
    departures uniform over the first ``depart_window_s`` seconds."""
    rng = np.random.default_rng(seed)
    net = _grid_network(n, spacing, lanes, speed, rng)
    dt = 0.5
    dem = _uniform_od(n * n, n_trips, int(round(depart_window_s / dt)), rng)
    return dict(name=f"grid{n}", network=net, demand=dem, params=default_params(1, seed=seed),
                steps=steps)


def grid_link_classes(net: dict, n: int) -> np.ndarray:
    """Three link classes on an n x n grid: 0 = perimeter links, 1 = links along every
    5th row or column, 2 = all others."""
    xs = net["node_x_dm"]
    ys = net["node_y_dm"]
    lf, lt = net["link_from"], net["link_to"]
    ci = np.arange(n * n) % n
    cj = np.arange(n * n) // n
    i0, j0, i1, j1 = ci[lf], cj[lf], ci[lt], cj[lt]
    horiz = j0 == j1
    row_or_col = np.where(horiz, j0, i0)
    perim = (row_or_col == 0) | (row_or_col == n - 1)
    fifth = (row_or_col % 5 == 0)
    cls = np.where(perim, 0, np.where(fifth, 1, 2)).astype(np.uint8)
    del xs, ys, i1, j1
    return cls


# --------------------------------------------------------------------------- metro
def metro(nx: int = 500, ny: int = 450, n_undirected: int = 275_000, n_trips: int = 3_000_000,
          spacing: float = 150.0, jitter: float = 40.0, steps: int = 172_800,
          seed: int = BASE_SEED + 2) -> dict:
    """Metropolitan-scale planar road network and demand.

    Topology: jittered nx x ny lattice.  Freeway corridors run along every 20th
    lattice row/column (offset 10), arterial corridors along every 7th (offset 3);
    all corridor edges are kept, a random spanning tree over local edges connects
    the rest, and random extra local edges bring the total to ``n_undirected``
    two-way roads (so the directed graph is strongly connected and planar).
    Hierarchy (Sec. 4 Tables 1-2 give OSM-based defaults; here three classes):
    local 1 lane 11 m/s, arterial 2 lanes 18 m/s, freeway 3-4 lanes 29 m/s.
    Lengths: lognormal with arithmetic mean 150 m, sigma 0.8, clamped to [20, 2000] m.
    Controls: signal where >= 3 incoming links and one of them non-local, stop where
    >= 3 incoming and all local, none otherwise; signals 60 s cycle, 30 s per phase.
    Demand: origins uniform over nodes; destination displacement with density
    proportional to max(r, 100 m)^-2 (gravity exponent 2) snapped to the lattice;
    departures 50/50 from N(8 h, 1 h) and N(17.5 h, 1.2 h), clipped to the day."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import minimum_spanning_tree

    rng = np.random.default_rng(seed)
    nn = nx * ny
    node = np.arange(nn)
    r_of, c_of = np.divmod(node, nx)
    px = c_of * spacing + rng.uniform(-jitter, jitter, nn)
    py = r_of * spacing + rng.uniform(-jitter, jitter, nn)

    # undirected lattice edges: horizontal then vertical
    hr, hc = np.divmod(np.arange(ny * (nx - 1)), nx - 1)
    hu = hr * nx + hc
    hw = hu + 1
    vr, vc = np.divmod(np.arange((ny - 1) * nx), nx)
    vu = vr * nx + vc
    vw = vu + nx
    eu = np.concatenate([hu, vu])
    ew = np.concatenate([hw, vw])
    line_row = np.concatenate([hr, np.full(len(vu), -1)])
    line_col = np.concatenate([np.full(len(hu), -1), vc])
    fwy = ((line_row >= 0) & (line_row % 20 == 10)) | ((line_col >= 0) & (line_col % 20 == 10))
    art = ~fwy & (((line_row >= 0) & (line_row % 7 == 3)) | ((line_col >= 0) & (line_col % 7 == 3)))
    corridor = fwy | art
    ne = len(eu)

    w = rng.uniform(1.0, 2.0, ne)
    w[corridor] = 1e-6
    mst = minimum_spanning_tree(coo_matrix((w, (eu, ew)), shape=(nn, nn)).tocsr()).tocoo()
    key_all = eu.astype(np.int64) * nn + ew
    key_mst = np.minimum(mst.row, mst.col).astype(np.int64) * nn + np.maximum(mst.row, mst.col)
    in_tree = np.isin(key_all, key_mst)
    keep = corridor | in_tree
    extra_pool = np.flatnonzero(~keep)
    n_extra = max(0, n_undirected - int(keep.sum()))
    keep[rng.choice(extra_pool, size=min(n_extra, len(extra_pool)), replace=False)] = True
    eu, ew = eu[keep], ew[keep]
    cls_u = np.where(fwy[keep], 2, np.where(art[keep], 1, 0))
    # freeway lanes: one draw (3 or 4) per freeway line, shared by its edges
    fwy_lanes_row = rng.integers(3, 5, ny)
    fwy_lanes_col = rng.integers(3, 5, nx)
    lr, lc = line_row[keep], line_col[keep]
    lanes_u = np.where(cls_u == 0, 1, np.where(cls_u == 1, 2,
                       np.where(lr >= 0, fwy_lanes_row[np.maximum(lr, 0)],
                                fwy_lanes_col[np.maximum(lc, 0)])))
    speed_u = np.array([11.0, 18.0, 29.0])[cls_u]
    mu = np.log(150.0) - 0.5 * 0.8 ** 2
    len_u = np.clip(np.exp(mu + 0.8 * rng.standard_normal(len(eu))), 20.0, 2000.0)

    lf = np.concatenate([eu, ew])
    lt = np.concatenate([ew, eu])
    rep = lambda a: np.concatenate([a, a])
    order = np.lexsort((lt, lf))
    lf, lt = lf[order], lt[order]
    length = rep(len_u)[order]
    speed = rep(speed_u)[order]
    lanes = rep(lanes_u)[order]
    cls = rep(cls_u)[order]

    n_in = np.bincount(lt, minlength=nn)
    nonlocal_in = np.bincount(lt, weights=(cls > 0), minlength=nn) > 0
    ctrl = np.where(n_in >= 3, np.where(nonlocal_in, CTRL_SIGNAL, CTRL_STOP), CTRL_NONE)
    off = rng.integers(0, 600, nn)

    net = _net(nn, np.round(px * 10), np.round(py * 10), ctrl, off,
               np.full(nn, 600), np.full(nn, 300), lf, lt, length, speed, lanes, cls)

    # gravity demand, sampled as a lattice displacement
    o = rng.integers(0, nn, n_trips)
    d = np.full(n_trips, -1, np.int64)
    rmax = float(np.hypot(nx * spacing, ny * spacing))
    z = 0.5 + np.log(rmax / 100.0)
    todo = np.arange(n_trips)
    while len(todo):
        u = rng.uniform(0.0, z, len(todo))
        rad = np.where(u <= 0.5, 100.0 * np.sqrt(2.0 * u), 100.0 * np.exp(u - 0.5))
        th = rng.uniform(0.0, 2 * np.pi, len(todo))
        dc = np.rint(rad * np.cos(th) / spacing).astype(np.int64)
        dr = np.rint(rad * np.sin(th) / spacing).astype(np.int64)
        cc = c_of[o[todo]] + dc
        rr = r_of[o[todo]] + dr
        ok = (cc >= 0) & (cc < nx) & (rr >= 0) & (rr < ny) & ((dc != 0) | (dr != 0))
        d[todo[ok]] = rr[ok] * nx + cc[ok]
        todo = todo[~ok]
    dt = 0.5
    am = rng.uniform(size=n_trips) < 0.5
    tsec = np.where(am, rng.normal(8 * 3600.0, 3600.0, n_trips),
                    rng.normal(17.5 * 3600.0, 1.2 * 3600.0, n_trips))
    tsec = np.clip(tsec, 0.0, 24 * 3600.0 - dt)
    dep = np.floor(tsec / dt).astype(np.int64)
    dem = _demand(o, d, dep)
    par = default_params(3, seed=seed)
    return dict(name="metro", network=net, demand=dem, params=par, steps=steps)


# --------------------------------------------------------------------------- ensemble
def ensemble_fleet(side: int) -> int:
    """Fleet size scaled with network size: 5 000 trips at side 10, 80 000 at side 40."""
    return 5000 + 75000 * (side * side - 100) // 1500


def ensemble(n_scen: int = 64, sides=(10, 15, 20, 30, 40), steps: int = 7200,
             seed: int = BASE_SEED + 3) -> list:
    """Independent grid scenarios (200 m links, 2 lanes, signals) with uneven sizes and
    per-scenario IDM parameters v0~U(25,33), T~U(1,2), a~U(0.8,1.5), b~U(1.2,2.5).
    The drawn v0 replaces the link speed limit in the car-following model."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_scen):
        side = int(rng.choice(sides))
        v0 = float(rng.uniform(25, 33))
        T = float(rng.uniform(1.0, 2.0))
        a = float(rng.uniform(0.8, 1.5))
        b = float(rng.uniform(1.2, 2.5))
        sub = int(rng.integers(0, 2**31 - 1))
        r2 = np.random.default_rng(sub)
        net = _grid_network(side, 200.0, 2, 13.9, r2)
        dem = _uniform_od(side * side, ensemble_fleet(side), 7200, r2)
        par = default_params(1, v0=[v0], T=[T], a=[a], b=[b], seed=sub)
        out.append(dict(name=f"ens{k}_side{side}", network=net, demand=dem, params=par,
                        steps=steps))
    return out


# --------------------------------------------------------------------------- calibration
def calib(steps: int = 1800, n: int = 20, n_trips: int = 20000, seed: int = BASE_SEED + 4) -> dict:
    """The 20 x 20 grid demand with three link classes (perimeter / every 5th line / other).
    Nominal per-class IDM parameters v0=13.9, T=1.5, a=1.0, b=1.5, s0=2; target
    parameters are the nominal ones scaled by (1 + U(-0.1, 0.1)) each."""
    sc = grid(n=n, n_trips=n_trips, steps=steps)
    sc["network"]["link_class"] = grid_link_classes(sc["network"], n)
    rng = np.random.default_rng(seed)
    nom = dict(v0=[13.9] * 3, T=[1.5] * 3, a=[1.0] * 3, b=[1.5] * 3, s0=[2.0] * 3)
    tgt = {k: [float(x * (1.0 + rng.uniform(-0.1, 0.1))) for x in v] for k, v in nom.items()}
    sc["params"] = default_params(3, **nom)
    sc["target_params"] = default_params(3, **tgt)
    sc["name"] = "calib"
    sc["steps"] = steps
    sc["obs_every"] = 20
    return sc


def small_grid(n: int = 6, n_trips: int = 600, steps: int = 900, lanes: int = 2,
               seed: int = BASE_SEED + 11, window_steps: int = 600) -> dict:
    """A small grid for quick parity cases (several lanes, signals, transitions)."""
    rng = np.random.default_rng(seed)
    net = _grid_network(n, 200.0, lanes, 13.9, rng)
    dem = _uniform_od(n * n, n_trips, window_steps, rng)
    return dict(name=f"grid{n}", network=net, demand=dem, params=default_params(1, seed=seed),
                steps=steps)


def small_metro(nx: int = 24, ny: int = 20, n_trips: int = 4000, steps: int = 1200,
                seed: int = BASE_SEED + 12) -> dict:
    """A reduced metro network (same recipe) with departures compressed into the
    first ``steps`` steps so that stops, signals and lane changes all occur."""
    n_und = int(round(275_000 * (nx * ny) / 225_000))
    sc = metro(nx=nx, ny=ny, n_undirected=n_und, n_trips=n_trips, steps=steps, seed=seed)
    dep = sc["demand"]["depart_step"].astype(np.int64)
    sc["demand"]["depart_step"] = np.ascontiguousarray(dep * (steps // 2) // 172_800, np.int32)
    sc["name"] = f"metro{nx}x{ny}"
    return sc


# --------------------------------------------------------------------------- BPR capacities
# Table 3 (capacity defaults, vehicles per lane per hour, by edge type and lanes 1/2/3/4+)
CAPACITY_VPHPL = {
    "motorway": (1900, 2000, 2000, 2200), "trunk": (1900, 2000, 2000, 2000),
    "primary": (1000, 1000, 1000, 1000), "secondary": (900, 900, 900, 900),
    "tertiary": (900, 900, 900, 900), "unclassified": (800, 800, 800, 800), "road": (900, 900, 900, 900),
}
# edge type standing for each class of the synthetic networks: metro local / arterial /
# freeway; the uniform grid's links are plain roads
METRO_EDGE_TYPES = ("unclassified", "primary", "motorway")


def bpr_capacity(sc: dict, period_h: float, edge_types=None) -> np.ndarray:
    """Capacity of every link over an assignment period of period_h hours: the Table 3
    lane capacity of its edge type and lane count, times lanes, times period_h."""
    net = sc["network"]
    lanes = net["link_lanes"].astype(np.int64)
    cls = net["link_class"].astype(np.int64)
    kinds = edge_types or ("road",) * (int(cls.max()) + 1 if len(cls) else 1)
    per_lane = np.array([[CAPACITY_VPHPL[kinds[c]][min(k, 4) - 1] for k in (1, 2, 3, 4)]
                         for c in range(len(kinds))], np.float64)
    return per_lane[cls, np.minimum(lanes, 4) - 1] * lanes * float(period_h)


# --------------------------------------------------------------------------- snapshots
def random_walk_routes(sc: dict, min_hops: int = 20, max_hops: int = 120, seed: int = BASE_SEED + 20):
    """Explicit routes for every trip: a random walk from the trip's origin that never
    takes the link straight back (unless it is the only way on), of uniform length in
    [min_hops, max_hops].  An input recipe for large stepping cases that need routes
    without running trip planning; returns (offsets, links)."""
    net = sc["network"]
    nn, lf, lt = net["n_nodes"], net["link_from"].astype(np.int64), net["link_to"].astype(np.int64)
    order = np.argsort(lf, kind="stable")
    start = np.zeros(nn + 1, np.int64)
    np.add.at(start, lf + 1, 1)
    start = np.cumsum(start)
    outl = order
    deg = start[1:] - start[:-1]
    rng = np.random.default_rng(seed)
    nt = sc["demand"]["n_trips"]
    hops = rng.integers(min_hops, max_hops + 1, nt)
    node = sc["demand"]["origin"].astype(np.int64).copy()
    prev_from = np.full(nt, -1, np.int64)
    out = np.full((max_hops, nt), -1, np.int64)
    for k in range(max_hops):
        live = k < hops
        d = deg[node]
        pick = rng.integers(0, 1 << 30, nt) % np.maximum(d, 1)
        e = outl[start[node] + pick]
        back = (lt[e] == prev_from) & (d > 1)
        pick2 = (pick + 1) % np.maximum(d, 1)
        e = np.where(back, outl[start[node] + pick2], e)
        out[k] = np.where(live, e, -1)
        prev_from = np.where(live, node, prev_from)
        node = np.where(live, lt[e], node)
    links = out.T[out.T >= 0]
    offsets = np.zeros(nt + 1, np.int64)
    offsets[1:] = np.cumsum(hops)
    return offsets.astype(np.int32), links.astype(np.int32)


def jammed_corridors(n_corr: int = 1000, length: float = 2000.0, lanes: int = 2, spacing: float = 7.0,
                     fill: float = 1.0, seed: int = BASE_SEED + 30) -> dict:
    """Standing queues: n_corr separate corridors A -> B -> C, each a ``length`` m link
    of ``lanes`` lanes into a signalised node B (cycle 60 s, the corridor's east-west
    approach green 15 s, offsets uniform) and a 200 m exit link.  Every lane of the
    long link holds a queue at rest, one vehicle per ``spacing`` m from the stop line
    back over ``fill`` of the link (about 285 per lane at the defaults), routed A -> B
    -> C; nothing departs later.  Returns a scenario with routes and initial state."""
    rng = np.random.default_rng(seed)
    n_nodes = 3 * n_corr
    y = np.repeat(np.arange(n_corr) * 500.0, 3)
    x = np.tile([0.0, length, length + 200.0], n_corr)
    ctrl = np.tile([CTRL_NONE, CTRL_SIGNAL, CTRL_NONE], n_corr)
    off = np.zeros(n_nodes, np.int64)
    off[1::3] = rng.integers(0, 600, n_corr)
    cyc = np.full(n_nodes, 600)
    grn = np.full(n_nodes, 450)   # north-south green 45 s: the east-west corridor gets 15 s
    a = np.arange(n_corr) * 3
    lf = np.stack([a, a + 1], 1).ravel()
    lt = np.stack([a + 1, a + 2], 1).ravel()
    length_m = np.tile([length, 200.0], n_corr)
    net = _net(n_nodes, np.round(x * 10), np.round(y * 10), ctrl, off, cyc, grn, lf, lt, length_m,
               np.full(2 * n_corr, 13.9), np.full(2 * n_corr, lanes), np.zeros(2 * n_corr))
    per_lane = int(np.floor(length * fill / spacing))
    n_per = per_lane * lanes
    nt = n_corr * n_per
    corr = np.repeat(np.arange(n_corr), n_per)
    k = np.tile(np.arange(n_per), n_corr)
    lane = (k % lanes).astype(np.int32)
    pos = k // lanes
    xq = length - 1.0 - pos * spacing
    routes_links = np.stack([2 * corr, 2 * corr + 1], 1).ravel().astype(np.int32)
    offsets = (np.arange(nt + 1) * 2).astype(np.int32)
    dem = _demand(3 * corr, 3 * corr + 2, np.zeros(nt, np.int64))
    st = dict(status=np.full(nt, ST_ACTIVE, np.uint8), link=(2 * corr).astype(np.int32), lane=lane,
              cursor=np.zeros(nt, np.int32), x=xq.astype(np.float32), v=np.zeros(nt, np.float32))
    return dict(name=f"jam{n_corr}", network=net, demand=dem, params=default_params(1, seed=seed),
                routes=dict(offsets=offsets, links=routes_links), init_state=st, steps=600)


def saturate(sc: dict, offsets, links, spacing: float = 8.0, v_frac: float = 0.5,
             seed: int = BASE_SEED + 21) -> dict:
    """A saturated snapshot: every trip on the road at once.  Trip i sits on hop
    k ~ U{0..len_i-1} of its route, in a uniformly drawn lane; vehicles of one lane are
    spread evenly along it (at most one per ``spacing`` metres, excess trips are
    re-drawn onto other hops, and after 30 rounds left pending), moving at ``v_frac``
    of the link speed limit.  Returns a per-trip state dict (status, link, lane,
    cursor, x, v)."""
    net = sc["network"]
    L = net["link_length_m"].astype(np.float64)
    lanes = net["link_lanes"].astype(np.int64)
    base = np.zeros(len(L) + 1, np.int64)
    base[1:] = np.cumsum(lanes)
    cap = np.maximum(1, np.floor(L / spacing)).astype(np.int64)
    off = np.asarray(offsets, np.int64)
    lk = np.asarray(links, np.int64)
    nt = len(off) - 1
    rlen = off[1:] - off[:-1]
    rng = np.random.default_rng(seed)
    cursor = np.zeros(nt, np.int64)
    lane = np.zeros(nt, np.int64)
    placed = np.zeros(nt, bool)
    todo = np.arange(nt)
    fill = np.zeros(base[-1], np.int64)
    for _ in range(30):
        if len(todo) == 0:
            break
        k = (rng.random(len(todo)) * rlen[todo]).astype(np.int64)
        e = lk[off[todo] + k]
        ln = (rng.random(len(todo)) * lanes[e]).astype(np.int64)
        g = base[e] + ln
        order = np.argsort(g, kind="stable")
        gs = g[order]
        first = np.r_[0, np.flatnonzero(gs[1:] != gs[:-1]) + 1]
        run_start = np.repeat(first, np.diff(np.r_[first, len(gs)]))
        rank = np.arange(len(gs)) - run_start + fill[gs]
        ok_sorted = rank < cap[e[order]]
        ok = np.zeros(len(todo), bool)
        ok[order] = ok_sorted
        np.add.at(fill, g[ok], 1)
        idx = todo[ok]
        cursor[idx], lane[idx], placed[idx] = k[ok], ln[ok], True
        todo = todo[~ok]
    link = np.where(placed, lk[off[:-1] + cursor], -1)
    g = np.where(placed, base[np.maximum(link, 0)] + lane, -1)
    key = rng.random(nt)
    order = np.lexsort((key, g))
    order = order[placed[order]]
    gs = g[order]
    first = np.r_[0, np.flatnonzero(gs[1:] != gs[:-1]) + 1]
    counts = np.diff(np.r_[first, len(gs)])
    rank = np.arange(len(gs)) - np.repeat(first, counts)
    cnt = np.repeat(counts, counts)
    x = np.zeros(nt, np.float64)
    x[order] = (rank + 0.5) * L[link[order]] / cnt
    v = np.where(placed, v_frac * net["link_speed_mps"].astype(np.float64)[np.maximum(link, 0)], 0.0)
    return dict(status=np.where(placed, ST_ACTIVE, ST_PENDING).astype(np.uint8),
                link=np.where(placed, link, 0).astype(np.int32), lane=lane.astype(np.int32),
                cursor=cursor.astype(np.int32), x=x.astype(np.float32), v=v.astype(np.float32))
