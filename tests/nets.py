"""Small hand-built networks for unit cases (inputs only)."""
import numpy as np

from paper_1807_01148_gb300 import scenarios as S


def make_net(nodes_xy, links, ctrl=None, offsets=None, lanes=2, length=None, speed=30.0):
    """nodes_xy: list of (x_m, y_m); links: list of (from, to)."""
    nn = len(nodes_xy)
    xy = np.array(nodes_xy, float)
    lf = np.array([a for a, _ in links])
    lt = np.array([b for _, b in links])
    if length is None:
        length = np.hypot(*(xy[lt] - xy[lf]).T)
    length = np.broadcast_to(np.asarray(length, float), (len(links),))
    lanes = np.broadcast_to(np.asarray(lanes), (len(links),))
    ctrl = np.zeros(nn) if ctrl is None else np.asarray(ctrl)
    offsets = np.zeros(nn) if offsets is None else np.asarray(offsets)
    return S._net(nn, np.round(xy[:, 0] * 10), np.round(xy[:, 1] * 10), ctrl, offsets,
                  np.full(nn, 600), np.full(nn, 300), lf, lt, length,
                  np.full(len(links), speed), lanes, np.zeros(len(links)))


def scenario(net, routes, state=None, depart=None, params=None):
    """routes: list of link lists (one per trip); state: dict of per-trip arrays or None."""
    nt = len(routes)
    off = np.zeros(nt + 1, np.int32)
    off[1:] = np.cumsum([len(r) for r in routes])
    links = np.concatenate([np.asarray(r, np.int32) for r in routes]) if nt else np.zeros(0, np.int32)
    lf, lt = net["link_from"], net["link_to"]
    o = np.array([lf[r[0]] for r in routes], np.int32)
    d = np.array([lt[r[-1]] for r in routes], np.int32)
    dep = np.zeros(nt, np.int32) if depart is None else np.asarray(depart, np.int32)
    sc = dict(name="hand", network=net, demand=S._demand(o, d, dep),
              params=params or S.default_params(1), routes=dict(offsets=off, links=links))
    if state is not None:
        st = dict(status=np.full(nt, S.ST_ACTIVE, np.uint8), link=np.zeros(nt, np.int32),
                  lane=np.zeros(nt, np.int32), cursor=np.zeros(nt, np.int32), x=np.zeros(nt, np.float32),
                  v=np.zeros(nt, np.float32))
        for k, val in state.items():
            st[k] = np.asarray(val, st[k].dtype)
        sc["init_state"] = st
    return sc
