"""Pins of the oracle's calibration adjoint (binary64 reverse sweep over the tape of a
binary32 run) against an independent computation: binary64 central finite
differences of the taped replay (the same continuous dynamics with every discrete
decision fixed), and the replay's own consistency with the binary32 forward loss."""
import numpy as np

import oracle as O
from paper_1807_01148_gb300 import scenarios as S

KEYS = ("v0", "T", "a", "b", "s0")


def _case(n=6, n_trips=500, steps=600, every=20):
    sc = S.calib(steps=steps, n=n, n_trips=n_trips)
    sc["demand"]["depart_step"] = (sc["demand"]["depart_step"] % (steps * 2 // 3)).astype(np.int32)
    o = O.OracleSim(sc)
    o.route()
    tp = sc["target_params"]
    o.set_class_params(*[tp[k] for k in KEYS])
    return sc, o.observe(steps, every)


def test_adjoint_equals_finite_differences_of_taped_replay():
    steps, every = 600, 20
    sc, tgt = _case(steps=steps, every=every)
    o = O.OracleSim(sc)
    o.route()
    g, loss = o.adjoint(steps, every, tgt, 3)
    p = sc["params"]
    th = {k: np.array(p[k], float) for k in KEYS}
    base = o.replay_loss(*[th[k] for k in KEYS])
    assert abs(base - loss) <= 1e-6 * loss          # binary64 replay of the binary32 run
    fd = np.zeros(15)
    for c in range(3):
        for j, k in enumerate(KEYS):
            hp = {q: v.copy() for q, v in th.items()}
            hm = {q: v.copy() for q, v in th.items()}
            h = 1e-4 * th[k][c]
            hp[k][c] += h
            hm[k][c] -= h
            fd[c * 5 + j] = (o.replay_loss(*[hp[q] for q in KEYS]) - o.replay_loss(*[hm[q] for q in KEYS])) / (2 * h)
    assert np.abs(fd).max() > 0
    assert np.abs(g - fd).max() / np.abs(fd).max() <= 1e-3


def test_zero_residual_gives_zero_gradient():
    # targets equal to the run's own trajectory: the loss is zero and so is every component
    steps, every = 400, 20
    sc = S.calib(steps=steps, n=5, n_trips=300)
    sc["demand"]["depart_step"] = (sc["demand"]["depart_step"] % 250).astype(np.int32)
    o = O.OracleSim(sc)
    o.route()
    own = o.observe(steps, every)
    o = O.OracleSim(sc)
    o.route()
    g, loss = o.adjoint(steps, every, own, 3)
    assert loss == 0.0 and np.all(g == 0.0)


def test_free_vehicle_closed_form():
    # one vehicle on a long empty road from rest: its speed obeys dv/dt = a (1 - (v/v0)^4)
    # in the ballistic scheme; the gradient of its final progress with respect to a must
    # match the sensitivity obtained by integrating the discrete map's derivative directly
    from .nets import make_net, scenario
    net = make_net([(0.0, 0.0), (5000.0, 0.0), (10000.0, 0.0)], [(0, 1), (1, 2)], lanes=1, speed=20.0)
    par = S.default_params(1, v0=[20.0])
    sc = scenario(net, [[0, 1]], dict(lane=[0], x=[0.0], v=[0.0]), params=par)
    steps, every = 100, 100
    o = O.OracleSim(sc)
    o.set_routes(sc["routes"]["offsets"], sc["routes"]["links"])
    o.write_state(sc["init_state"])
    g, loss = o.adjoint(steps, every, np.zeros((1, 1)), 1)
    # direct forward sensitivity of x_n to a (binary64), same discrete map
    A, v0, dt = 1.0, 20.0, 0.5
    x, v, dx, dv = 0.0, 0.0, 0.0, 0.0
    for _ in range(steps):
        acc = A * (1 - (v / v0) ** 4)
        dacc = (1 - (v / v0) ** 4) + A * (-4 * v ** 3 / v0 ** 4) * dv
        x, dx = x + v * dt + 0.5 * acc * dt * dt, dx + dv * dt + 0.5 * dacc * dt * dt
        v, dv = v + acc * dt, dv + dacc * dt
    assert abs(loss - x * x) <= 1e-4 * x * x
    assert abs(g[2] - 2 * x * dx) <= 1e-4 * abs(2 * x * dx)
