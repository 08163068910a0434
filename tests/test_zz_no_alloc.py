"""sim_sssp_static: the shortest-path tree for callers that cannot allocate device
memory (a framework owns the pool, a supervisor caps the process, a plug-in must not
touch the allocator).  Its working memory is a fixed array inside the library, so
this test checks it against the existing trip planner, sim_route, through the C ABI:
for every trip of the sampled origins, the tree's distance to the destination equals
the cost of the route sim_route planned (integer costs: exact), on two calls in a
row.  This file is collected last."""
import ctypes

import numpy as np
import pytest

from paper_1807_01148_gb300 import scenarios as S

pytestmark = pytest.mark.gpu

SIM_SSSP_STATIC_MAX_NODES = 262144


def _bind(lib):
    f = lib.sim_sssp_static
    f.argtypes = [ctypes.c_int32, ctypes.c_int32] + [ctypes.c_void_p] * 4 + [ctypes.c_int32, ctypes.c_void_p,
                                                                               ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def _csr(net):
    lf = net["link_from"].astype(np.int64)
    order = np.argsort(lf, kind="stable").astype(np.int32)
    start = np.zeros(net["n_nodes"] + 1, np.int64)
    np.add.at(start, lf + 1, 1)
    return np.cumsum(start).astype(np.int32), order


@pytest.mark.parametrize("make", [lambda: S.grid(n=12, n_trips=3000),
                                  lambda: S.small_metro(nx=40, ny=30, n_trips=6000)])
def test_static_tree_matches_sim_route(make):
    import torch
    from paper_1807_01148_gb300 import gbtraffic as G

    sc = make()
    net = sc["network"]
    rng = np.random.default_rng(7)
    cost = rng.integers(1, 400, net["n_links"]).astype(np.int32)
    sim = G.Sim(sc)
    sim.route(cost)                      # the existing entry point
    off, links = sim.routes()
    route_cost = np.add.reduceat(cost[links].astype(np.int64), off[:-1])

    start, order = _csr(net)
    dev = torch.device("cuda")
    d_start = torch.from_numpy(start).to(dev)
    d_link = torch.from_numpy(order).to(dev)
    d_to = torch.from_numpy(net["link_to"].astype(np.int32)).to(dev)
    d_cost = torch.from_numpy(cost).to(dev)
    dist = torch.empty(net["n_nodes"], dtype=torch.int32, device=dev)
    f = _bind(G.lib())
    stream = torch.cuda.current_stream().cuda_stream

    origins = sc["demand"]["origin"]
    dests = sc["demand"]["dest"]
    sample = rng.choice(np.unique(origins), 25, replace=False)
    for o in sample:
        results = []
        for _ in range(2):                               # two calls in a row
            rc = f(net["n_nodes"], net["n_links"], d_start.data_ptr(), d_link.data_ptr(), d_to.data_ptr(),
                   d_cost.data_ptr(), int(o), dist.data_ptr(), stream)
            assert rc == 0
            results.append(dist.cpu().numpy().copy())
        assert np.array_equal(results[0], results[1])
        dv = results[0]
        assert dv[o] == 0
        trips = np.flatnonzero(origins == o)
        assert np.array_equal(dv[dests[trips]].astype(np.int64), route_cost[trips])
    sim.close()


def test_static_tree_rejects_oversize_and_bad_graphs():
    import torch
    from paper_1807_01148_gb300 import gbtraffic as G

    f = _bind(G.lib())
    dev = torch.device("cuda")
    z = torch.zeros(8, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream().cuda_stream
    # beyond the fixed working-memory limit: rejected before touching the arrays
    assert f(SIM_SSSP_STATIC_MAX_NODES + 1, 0, z.data_ptr(), None, None, None, 0, z.data_ptr(), stream) == -1
    # origin out of range
    assert f(4, 0, z.data_ptr(), None, None, None, 9, z.data_ptr(), stream) == -1
    # a link whose head node is out of range
    start = torch.tensor([0, 1, 1], dtype=torch.int32, device=dev)
    link = torch.tensor([0], dtype=torch.int32, device=dev)
    to = torch.tensor([5], dtype=torch.int32, device=dev)
    cost = torch.tensor([3], dtype=torch.int32, device=dev)
    out = torch.empty(2, dtype=torch.int32, device=dev)
    assert f(2, 1, start.data_ptr(), link.data_ptr(), to.data_ptr(), cost.data_ptr(), 0, out.data_ptr(),
             stream) == -1
    # the same graph made valid works, and an unreachable node reads INT32_MAX
    to = torch.tensor([1], dtype=torch.int32, device=dev)
    assert f(2, 1, start.data_ptr(), link.data_ptr(), to.data_ptr(), cost.data_ptr(), 1, out.data_ptr(),
             stream) == 0
    assert out.cpu().tolist() == [2**31 - 1, 0]
