"""Execution configurations of sim_step: the CUDA-graph path with several grid sizes
and the single persistent cooperative launch with several block shapes must give
bit-identical results (checked against the oracle); the autotuner picks among them
and caches its choice; a barrier wait that runs out returns SIM_ETIMEOUT and leaves
the handle usable."""
import json

import numpy as np
import pytest

from paper_1807_01148_gb300 import scenarios as S

from .parity import diff_state, run_lockstep, setup_pair

pytestmark = pytest.mark.gpu

CONFIGS = [dict(mode=0, grid_per_sm=2), dict(mode=0, grid_per_sm=16), dict(mode=1, threads=256, blocks_per_sm=1),
           dict(mode=1, threads=256, blocks_per_sm=2), dict(mode=1, threads=512, blocks_per_sm=1),
           dict(mode=1, threads=1024, blocks_per_sm=1), dict(mode=1, threads=256, blocks_per_sm=4)]


@pytest.fixture(scope="module")
def G():
    from paper_1807_01148_gb300 import gbtraffic
    return gbtraffic


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: "-".join(f"{k}{v}" for k, v in c.items()))
def test_persistent_and_graph_configs_bitexact(G, cfg):
    import oracle
    sc = S.small_metro()
    g, o = setup_pair(sc, G.Sim, oracle.OracleSim)
    try:
        g.set_exec(**cfg)
    except G.SimError:
        pytest.skip("configuration does not fit this device")
    run_lockstep(g, o, 1200, 150)


def test_batched_ensemble_persistent_equals_graph(G):
    scs = [S.small_grid(n=n, n_trips=100 * n, steps=500, seed=2000 + n, window_steps=400) for n in (4, 7, 5, 9)]
    a = G.Sim.batch(scs)
    a.route()
    b = G.Sim.batch(scs)
    b.route()
    b.set_exec(mode=1, threads=256, blocks_per_sm=1)
    for _ in range(5):
        a.step(100)
        b.step(100)
        d = diff_state(a.state(), b.state())
        assert not d, d


def test_autotune_choice_and_cache(G, tmp_path):
    scs = [S.small_grid(n=n, n_trips=150 * n, steps=400, seed=3000 + n) for n in (5, 8)]
    cache = str(tmp_path / "tune.jsonl")
    a = G.Sim.batch(scs)
    a.route()
    a.step(50)
    ref = G.Sim.batch(scs)
    ref.route()
    ref.step(50)
    choice = a.autotune(trial_steps=10, cache_path=cache)
    assert choice["mode"] in (0, 1)
    # the trials left the state where it was
    assert not diff_state(a.state(), ref.state())
    a.step(200)
    ref.step(200)
    assert not diff_state(a.state(), ref.state())
    lines = [json.loads(x) for x in open(cache)]
    assert len(lines) == 1 and lines[0]["mode"] == choice["mode"]
    b = G.Sim.batch(scs)
    b.route()
    assert b.autotune(trial_steps=10, cache_path=cache) == choice      # cache hit
    assert len(open(cache).readlines()) == 1


def test_launch_count(G):
    # graph execution: the kernels of the step graph per step (two scan kernels, scatter,
    # rank, lane fronts, chunks, counters; the long-segment rank where a lane can hold
    # more than 64 vehicles; the big-chunk kernel where most of the road lies on links
    # that hold more vehicles than a staged chunk); persistent execution: one launch per
    # sim_step call
    g = G.Sim(S.small_grid(n=5, n_trips=200, steps=200))   # 200 m links
    g.route()
    n0 = g.launch_count()
    g.step(10)
    assert g.launch_count() - n0 == 10 * 7
    sm = G.Sim(S.small_metro())                             # links up to about 900 m
    sm.route()
    n0 = sm.launch_count()
    sm.step(3)
    assert sm.launch_count() - n0 == 3 * 8
    jam = S.jammed_corridors(n_corr=2)
    j = G.Sim(jam)
    j.set_routes(jam["routes"]["offsets"], jam["routes"]["links"])
    j.write_state(jam["init_state"])
    n0 = j.launch_count()
    j.step(4)
    assert j.launch_count() - n0 == 4 * 9
    g.set_exec(mode=1, threads=256, blocks_per_sm=1)
    n0 = g.launch_count()
    g.step(10)
    g.step(5)
    assert g.launch_count() - n0 == 2


def test_barrier_timeout_returns_error_and_handle_recovers(G):
    sc = S.small_grid(n=6, n_trips=400, steps=300)
    g = G.Sim(sc)
    g.route()
    g.step(50)
    g.set_exec(mode=1, threads=256, blocks_per_sm=1, barrier_timeout_cycles=1)
    with pytest.raises(G.SimError) as e:
        g.step(5)
    assert e.value.code == G.SIM_ETIMEOUT
    # back to a sane configuration: the handle refuses to step until the state is reset
    g.set_exec(mode=0, grid_per_sm=8)
    with pytest.raises(G.SimError) as e:
        g.step(1)
    assert e.value.code == G.SIM_ESTATE
    n = sc["demand"]["n_trips"]
    g.write_state(dict(status=np.zeros(n, np.uint8), link=np.zeros(n, np.int32), lane=np.zeros(n, np.int32),
                       cursor=np.zeros(n, np.int32), x=np.zeros(n, np.float32), v=np.zeros(n, np.float32)))
    g.step(100)
    assert g.counters()["t"] == 100


def test_tile_wait_timeout_returns_error_and_handle_recovers(G):
    # graph execution with a one-cycle bound on the chunk kernel's waits for its
    # bulk-copied chunks: the first wait runs out while the copy is in flight, the kernel
    # reports it and returns after its copies have landed, every later kernel of the
    # step returns at entry; the handle is usable again after the state is reset
    sc = S.small_grid(n=6, n_trips=400, steps=300)
    g = G.Sim(sc)
    g.route()
    g.step(50)
    g.set_exec(mode=0, grid_per_sm=8, barrier_timeout_cycles=1)
    with pytest.raises(G.SimError) as e:
        g.step(5)
    assert e.value.code == G.SIM_ETIMEOUT
    g.set_exec(mode=0, grid_per_sm=8)
    with pytest.raises(G.SimError) as e:
        g.step(1)
    assert e.value.code == G.SIM_ESTATE
    n = sc["demand"]["n_trips"]
    g.write_state(dict(status=np.zeros(n, np.uint8), link=np.zeros(n, np.int32), lane=np.zeros(n, np.int32),
                       cursor=np.zeros(n, np.int32), x=np.zeros(n, np.float32), v=np.zeros(n, np.float32)))
    g.step(100)
    assert g.counters()["t"] == 100


def test_device_memory_cap_returns_enomem(G):
    # sim_params.max_device_bytes caps what a handle allocates: a creation that would pass
    # it fails with SIM_ENOMEM (nothing is left allocated), a generous cap changes nothing
    sc = S.small_grid(n=5, n_trips=200, steps=100)
    tiny = dict(sc, params=dict(sc["params"], max_device_bytes=4096))
    with pytest.raises(G.SimError) as e:
        G.Sim(tiny)
    assert e.value.code == G.SIM_ENOMEM
    roomy = dict(sc, params=dict(sc["params"], max_device_bytes=1 << 30))
    g = G.Sim(roomy)
    g.route()
    g.step(20)
    ref = G.Sim(sc)
    ref.route()
    ref.step(20)
    a, b = g.state(), ref.state()
    assert all(np.array_equal(a[k], b[k]) for k in a)

