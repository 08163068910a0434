"""Calibration adjoint (GPU) against the oracle and against finite differences.

The gradient of L = sum_k sum_v (p_v(t_k) - target)^2 with respect to the 15 IDM
parameters (3 link classes x v0, T, a, b, s0) on a grid with three link classes,
discrete decisions held fixed:
- the GPU forward observations equal the oracle's exactly (binary64 progress of
  bit-identical binary32 states);
- the GPU loss and gradient equal the oracle's binary64 reverse sweep of the same tape
  up to summation order;
- the gradient matches binary64 central finite differences (eps = 1e-4 relative) of the
  oracle's taped replay: ||g - g_FD||_inf / ||g_FD||_inf <= 1e-3;
- the torch.autograd.Function returns the same gradient."""
import numpy as np
import pytest

from paper_1807_01148_gb300 import scenarios as S

pytestmark = pytest.mark.gpu
KEYS = ("v0", "T", "a", "b", "s0")


def _case(n=8, n_trips=900, steps=600):
    sc = S.calib(steps=steps, n=n, n_trips=n_trips)
    sc["demand"]["depart_step"] = (sc["demand"]["depart_step"] % (steps * 2 // 3)).astype(np.int32)
    return sc


def _targets(sc, steps, every):
    import oracle
    o = oracle.OracleSim(sc)
    o.route()
    tp = sc["target_params"]
    o.set_class_params(*[tp[k] for k in KEYS])
    return o.observe(steps, every)


@pytest.mark.parametrize("seg", [64, 50])
def test_adjoint_matches_oracle_and_fd(seg):
    import oracle
    from paper_1807_01148_gb300 import gbtraffic as G
    steps, every = 600, 20
    sc = _case(steps=steps)
    tgt = _targets(sc, steps, every)
    # forward observations: GPU == oracle, exactly
    g = G.Sim(sc)
    g.route()
    o = oracle.OracleSim(sc)
    o.route()
    assert np.array_equal(g.observe(steps, every), o.observe(steps, every))
    # adjoint
    g = G.Sim(sc)
    g.route()
    grad, loss = g.adjoint(steps, every, tgt, 3, checkpoint_every=seg)
    o = oracle.OracleSim(sc)
    o.route()
    og, oloss = o.adjoint(steps, every, tgt, 3)
    assert abs(loss - oloss) <= 1e-12 * abs(oloss)
    og = og.reshape(3, 5)
    assert np.allclose(grad, og, rtol=1e-9, atol=1e-9 * np.abs(og).max())
    # binary64 central differences of the taped replay
    p = sc["params"]
    th = {k: np.array(p[k], float) for k in KEYS}
    fd = np.zeros((3, 5))
    for c in range(3):
        for j, k in enumerate(KEYS):
            if th[k][c] == 0.0:
                continue
            hp = {q: v.copy() for q, v in th.items()}
            hm = {q: v.copy() for q, v in th.items()}
            h = 1e-4 * th[k][c]
            hp[k][c] += h
            hm[k][c] -= h
            fd[c, j] = (o.replay_loss(*[hp[q] for q in KEYS]) - o.replay_loss(*[hm[q] for q in KEYS])) / (2 * h)
    err = np.abs(grad - fd).max() / np.abs(fd).max()
    assert err <= 1e-3, (err, grad, fd)
    # the state after the call is the one after the horizon
    assert g.counters()["t"] == steps


def test_autograd_function():
    import torch
    from paper_1807_01148_gb300 import gbtraffic as G
    steps, every = 400, 20
    sc = _case(n=6, n_trips=500, steps=steps)
    tgt = _targets(sc, steps, every)
    g = G.Sim(sc)
    g.route()
    n = sc["demand"]["n_trips"]
    start = dict(status=np.zeros(n, np.uint8), link=np.zeros(n, np.int32), lane=np.zeros(n, np.int32),
                 cursor=np.zeros(n, np.int32), x=np.zeros(n, np.float32), v=np.zeros(n, np.float32))
    p = sc["params"]
    theta = torch.tensor(np.stack([np.array(p[k], float) for k in KEYS], 1), requires_grad=True)
    fn = G.calibration_loss_fn()
    loss = fn.apply(theta, g, start, tgt, steps, every, 64)
    loss.backward()
    g2 = G.Sim(sc)
    g2.route()
    ref, ref_loss = g2.adjoint(steps, every, tgt, 3)
    assert abs(loss.item() - ref_loss) <= 1e-12 * ref_loss
    assert np.allclose(theta.grad.numpy(), ref, rtol=1e-10, atol=1e-10 * np.abs(ref).max())
    # without requires_grad the loss comes from the plain forward pass
    with torch.no_grad():
        l2 = fn.apply(theta.detach(), g, start, tgt, steps, every, 64)
    assert abs(l2.item() - ref_loss) <= 1e-9 * ref_loss
