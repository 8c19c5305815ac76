"""Pins of the oracle's static 3-D immersed boxes (ib3d): solid / IB faces face by face, the
partition of unity of the 3-D delta on a uniform grid, the transpose identity of the force
gather, and zero velocity on forced faces after a step."""
import numpy as np
import torch

import oracle as O
import synthetic as S
from oracle import ib3d
from helpers import grid_of

P, NS = S.PERIODIC, S.NOSLIP


def _grid():
    wl = S.box_3d(16, 12, 16, (P, P), (NS, NS), L=(1.0, 0.75, 1.0), nu=0.01)
    return wl, grid_of(wl)


def test_classify_face_by_face():
    wl, g = _grid()
    body = ib3d.Boxes([[0.3, 0.55, 0.0, 0.2, 0.4, 0.6]], np.zeros((1, 3)), [1.0])
    masks = ib3d.classify(g, body)
    b = body.boxes[0]
    for c in range(3):
        solid, ibm = masks[c]
        fx, fy, fz = [t.expand(g.shape(c)) for t in g.face_coords(c)]
        ez, ey, ex = g.shape(c)
        for k in range(ez):
            for j in range(ey):
                for i in range(ex):
                    x, y, z = float(fx[k, j, i]), float(fy[k, j, i]), float(fz[k, j, i])
                    inside = b[0] < x < b[1] and b[2] < y < b[3] and b[4] < z < b[5]
                    assert bool(solid[k, j, i]) == inside
                    nbs = []
                    for d, (n, idx) in enumerate(((ex, i), (ey, j), (ez, k))):
                        for s in (-1, 1):
                            q = [i, j, k]
                            q[d] = idx + s
                            if g.periodic(d):
                                q[d] %= n
                            elif not 0 <= q[d] < n:
                                continue
                            nbs.append(bool(solid[q[2], q[1], q[0]]))
                    assert bool(ibm[k, j, i]) == ((not inside) and any(nbs))


def test_uniform_forcing_gives_minus_f_per_marker():
    """sum_faces delta_h(x - X) dv = 1 for markers whose support lies inside a uniform grid."""
    wl = S.box_3d(16, 16, 16, (P, P), (P, P), L=(1.0, 1.0, 1.0))
    g = grid_of(wl)
    rng = np.random.default_rng(0)
    X = rng.uniform(0.2, 0.8, size=(20, 3))
    body = ib3d.Boxes(np.zeros((0, 6)), X, np.ones(20))
    for kind in (O.ib.PESKIN4, O.ib.ROMA3):
        f = [torch.full(g.shape(c), 0.7 + c, dtype=torch.float64) for c in range(3)]
        q, F = ib3d.marker_forces(g, body, kind, f)
        for c in range(3):
            assert torch.allclose(q[:, c], torch.full((20,), -(0.7 + c), dtype=torch.float64), rtol=1e-13, atol=0)


def test_force_gather_transpose_identity():
    """<q, Q>_markers = -<f, S Q>_faces with S the spreading by the same weights."""
    wl, g = _grid()
    rng = np.random.default_rng(1)
    X = rng.uniform([0.2, 0.2, 0.2], [0.8, 0.55, 0.8], size=(7, 3))
    body = ib3d.Boxes(np.zeros((0, 6)), X, np.ones(7))
    f = [torch.tensor(rng.standard_normal(g.shape(c))) for c in range(3)]
    Q = torch.tensor(rng.standard_normal((7, 3)))
    q, _ = ib3d.marker_forces(g, body, O.ib.ROMA3, f)
    lhs = float((q * Q).sum())
    rhs = 0.0
    for c in range(3):
        W = ib3d.weights(g, c, O.ib.ROMA3, body.X)
        spread = (W * Q[:, c].reshape(-1, 1, 1, 1)).sum(dim=0)
        rhs -= float((f[c] * g.face_volume(c) * spread).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_forced_faces_are_zero_before_the_correction():
    """u* = u_s = 0 on forced faces, so after the step u^{n+1} = -G phi there exactly,
    and the forcing f is zero off the forced faces."""
    from oracle import fluid
    wl, g = _grid()
    wl.u0 = S.random_fields(wl, 3, 1.0)
    body = ib3d.Boxes([[0.3, 0.55, 0.0, 0.2, 0.4, 0.6]], [[0.3, 0.1, 0.5]], [1e-3])
    st = O.State([torch.tensor(a) for a in wl.u0])
    new, dg = O.step(g, st, 0.002, body=body, kernel=O.ib.ROMA3)
    G = fluid.gradient(g, dg.phi)
    for c in range(3):
        e = dg.eps[c]
        assert int(e.sum()) > 0
        assert torch.equal(new.u[c][e], -G[c][e])
        assert float(dg.f[c][~e].abs().max()) == 0.0
    assert dg.F.shape == (3,)
