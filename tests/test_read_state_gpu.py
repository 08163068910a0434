"""sim_read_state's paths: host reads of any subset of fields (through the handle's
staging buffers, kept between calls) and device reads into caller-owned CUDA tensors
give the same bits, and both equal the CPU oracle's state after the same steps."""
import ctypes

import numpy as np
import pytest

from paper_1807_01148_gb300 import scenarios as S

from .parity import diff_state

pytestmark = pytest.mark.gpu

NAMES = ("status", "link", "lane", "cursor", "x", "v", "insert_step", "arrive_step", "lane_change")
DTYPES = {"status": np.uint8, "lane_change": np.int8, "x": np.float32, "v": np.float32}


def _bits(a):
    return a.view(np.uint32) if a.dtype == np.float32 else a


def test_host_device_and_partial_reads_agree():
    import torch

    import oracle
    from paper_1807_01148_gb300 import gbtraffic as G
    sc = S.small_grid(n=6, n_trips=500, steps=400)
    g = G.Sim(sc)
    g.set_stream(torch.cuda.current_stream().cuda_stream)
    g.route()
    o = oracle.OracleSim(sc)
    o.route()
    for steps in (150, 250):
        g.step(steps)
        o.step(steps)
        full = g.state()
        assert not diff_state(full, o.state())
        # one field at a time, in an order that reuses every staging buffer
        for i, k in reversed(list(enumerate(NAMES))):
            part = g.state(1 << i)
            assert list(part) == [k]
            assert np.array_equal(_bits(part[k]), _bits(full[k])), k
        # two fields together
        xv = g.state(G.F_X | G.F_V)
        assert np.array_equal(_bits(xv["x"]), _bits(full["x"])) and np.array_equal(_bits(xv["v"]), _bits(full["v"]))
        # device buffers
        n = g.n_trips
        tens = {k: torch.zeros(n, dtype=getattr(torch, np.dtype(DTYPES.get(k, np.int32)).name), device="cuda")
                for k in NAMES}
        g.state_device(tens, G.F_ALL)
        torch.cuda.synchronize()
        for k in NAMES:
            assert np.array_equal(_bits(tens[k].cpu().numpy()), _bits(full[k])), k
        # enqueued only (mode 2) on the handle's stream, which is torch's current one:
        # torch's later reads are ordered after the gather
        late = {k: torch.zeros_like(v) for k, v in tens.items()}
        g.state_device(late, G.F_X | G.F_V | G.F_LINK, wait=False)
        for k in ("x", "v", "link"):
            assert np.array_equal(_bits(late[k].cpu().numpy()), _bits(full[k])), k
        assert not late["status"].any()                     # not requested, untouched


def test_requested_field_without_buffer_is_rejected():
    from paper_1807_01148_gb300 import gbtraffic as G
    sc = S.small_grid(n=5, n_trips=100, steps=100)
    g = G.Sim(sc)
    g.route()
    g.step(10)
    view = G.sim_state_view(None, None, None, None, None, None, None, None, None)
    rc = G.lib().sim_read_state(g.h, ctypes.byref(view), G.F_X, 0)
    assert rc == G.SIM_EINVAL
    assert G.lib().sim_read_state(g.h, ctypes.byref(view), G.F_X, 3) == G.SIM_EINVAL   # no such mode
    g.step(10)                                     # the handle stays usable
    assert g.counters()["t"] == 20
