"""The calibration adjoint at its configured size: the 20x20 signalised grid with three
link classes, 20,000 trips, 1800 steps, observations every 20 steps (checkpoints every
64), gradient of the squared route-progress error with respect to the 15 IDM
parameters (3 classes x v0, T, a, b, s0), discrete decisions held fixed.

1. Over the whole configured horizon, the GPU gradient (sim_adjoint) equals the
   oracle's binary64 reverse sweep of the same tape up to summation order, and matches
   binary64 central finite differences (eps = 1e-4 relative) of the taped replay:
   ||g - g_FD||_inf / ||g_FD||_inf <= 1e-3 (the relative error of every component is
   printed beside it).
2. Untaped +-eps runs.  The oracle's own binary32 model is rerun at theta +- eps with
   its discrete tape recorded; runs whose tape (leaders, forms of Eq. 7, its floors,
   moves, crossings, departures, arrivals) equals the base run's took no discrete
   flip.  Over the full 1800 steps every such run flips something (2.7M taped
   vehicle-steps, and eps moves positions by about 1e-3 m), so for each parameter the
   comparison is made over the longest prefix (a whole number of observation periods)
   on which both of its runs keep the base tape: there the taped replay IS the model,
   and the GPU gradient over that horizon must match its binary64 central difference.
Targets come from the oracle (binary32 forward at perturbed parameters).  The oracle
runs go to a process pool started with spawn."""
import multiprocessing as mp

import numpy as np
import pytest

from paper_1807_01148_gb300 import scenarios as S

pytestmark = pytest.mark.gpu
KEYS = ("v0", "T", "a", "b", "s0")
EPS = 1e-4


def _theta(sc):
    return {k: np.array(sc["params"][k], np.float64) for k in KEYS}


def _shift(th, c, k, rel):
    out = {q: v.copy() for q, v in th.items()}
    out[k][c] = out[k][c] * (1.0 + rel)
    return out


def _targets(sc):
    import oracle
    o = oracle.OracleSim(sc)
    o.route()
    tp = sc["target_params"]
    o.set_class_params(*[tp[k] for k in KEYS])
    return o.observe(sc["steps"], sc["obs_every"])


def _flip_free_prefix(args):
    """Steps at the start of the run at theta shifted by rel on (c, k) whose discrete
    tape equals the base run's (per-step digests of the oracle's recorded tape)."""
    c, k, rel = args
    import oracle
    sc = S.calib()
    steps = sc["steps"]
    base = oracle.OracleSim(sc)
    base.route()
    base.record(steps)
    _, nb, db = base.tape_digest(per_step=True)
    o = oracle.OracleSim(sc)
    o.route()
    th = _shift(_theta(sc), c, k, rel)
    o.set_class_params(*[th[q].astype(np.float32) for q in KEYS])
    o.record(steps)
    _, no, do = o.tape_digest(per_step=True)
    bad = np.flatnonzero(db[:steps] != do[:steps])
    if len(bad):
        return int(bad[0]) - 1
    return steps if (no == nb and base.tape_digest() == o.tape_digest()) else steps - 1


def _taped_fd(o, th, c, k):
    h = EPS * th[k][c]
    hp, hm = _shift(th, c, k, EPS), _shift(th, c, k, -EPS)
    return (o.replay_loss(*[hp[q] for q in KEYS]) - o.replay_loss(*[hm[q] for q in KEYS])) / (2 * h)


@pytest.fixture(scope="module")
def calib():
    sc = S.calib()
    assert (sc["network"]["n_nodes"], sc["demand"]["n_trips"], sc["steps"], sc["obs_every"]) == (400, 20000, 1800,
                                                                                                  20)
    return sc, _targets(sc)


def test_calib_full_horizon_gradient(calib):
    import oracle
    from paper_1807_01148_gb300 import gbtraffic as G
    sc, tgt = calib
    steps, every = sc["steps"], sc["obs_every"]
    g = G.Sim(sc)
    g.route()
    grad, loss = g.adjoint(steps, every, tgt, 3, checkpoint_every=64)
    o = oracle.OracleSim(sc)
    o.route()
    og, oloss = o.adjoint(steps, every, tgt, 3)
    og = og.reshape(3, 5)
    assert abs(loss - oloss) <= 1e-12 * abs(oloss)
    assert np.allclose(grad, og, rtol=1e-9, atol=1e-9 * np.abs(og).max())
    th = _theta(sc)
    fd = np.zeros((3, 5))
    for c in range(3):
        for j, k in enumerate(KEYS):
            fd[c, j] = _taped_fd(o, th, c, k)
    err = np.abs(grad - fd)
    scale = np.abs(fd).max()
    rel = err / np.maximum(np.abs(fd), 1e-300)
    print("per-parameter relative error (rows: class, cols: v0 T a b s0):\n", rel)
    assert err.max() / scale <= 1e-3, (err.max() / scale, grad, fd)


def test_calib_untaped_runs_flip_free_horizons(calib):
    import oracle
    from paper_1807_01148_gb300 import gbtraffic as G
    sc, tgt = calib
    every = sc["obs_every"]
    jobs = [(c, k, s * EPS) for c in range(3) for k in KEYS for s in (1, -1)]
    with mp.get_context("spawn").Pool(min(16, mp.cpu_count())) as pool:
        prefix = dict(zip(jobs, pool.map(_flip_free_prefix, jobs)))
    th = _theta(sc)
    checked = []
    for c in range(3):
        for j, k in enumerate(KEYS):
            common = min(prefix[(c, k, EPS)], prefix[(c, k, -EPS)])
            H = (common // every) * every
            assert H >= 4 * every, f"class {c} {k}: only {common} flip-free steps"
            g = G.Sim(sc)
            g.route()
            grad, _ = g.adjoint(H, every, tgt[: H // every], 3, checkpoint_every=64)
            o = oracle.OracleSim(sc)
            o.route()
            o.adjoint(H, every, tgt[: H // every], 3)
            fd = _taped_fd(o, th, c, k)
            rel = abs(grad[c, j] - fd) / abs(fd)
            checked.append((c, k, H, rel))
            assert rel <= 1e-3, (c, k, H, grad[c, j], fd)
    print("flip-free horizon and relative error per parameter:", checked)
