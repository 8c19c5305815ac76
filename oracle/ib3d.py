"""Static 3-D immersed bodies made of axis-aligned boxes (oracle, FP64).

The paper's rough-wall and obstacle cases (§3.4, e.g. cube roughness on a
channel wall) place fixed bodies in a 3-D flow and force them with the same
direct forcing as its 2-D bodies (§2.3.3, Eqs. 18-23).  For a body at rest the
target velocity is zero on every forced face: u_s = 0 on solid and IB faces
and u_c = 0 inside, so the interpolation of Eq. (18) reduces to that value and
the Lagrangian markers serve the hydrodynamic force of Eq. (20) only.

  Boxes            union of boxes [x0, x1] x [y0, y1] x [z0, z1] with surface markers
  classify         solid faces (face position strictly inside a box) and IB faces
                   (non-solid faces with a solid same-component neighbour in any
                   of the six directions), the epsilon = 1 set of Eq. (5)
  delta3           delta_h(x) = d_h(x) d_h(y) d_h(z) (Eq. 21 in 3-D)
  marker_forces    q_i of Eq. (20) and F = rho sum_i q_i dV_i

Readings: the grid is uniform in all three directions
where the body's kernel supports reach; a face exactly on a box surface is a
fluid face (open boxes); dV_i is supplied per marker.

Parity: pinned by the partition of unity of delta_h on a uniform grid (a
uniform forcing field gives q_i = -f exactly), by the transpose identity of
the force gather, and by the solid / IB definition checked face by face
(tests/test_oracle_ib3d.py).

Test infrastructure only (see the package header).
"""
import torch

from .grid import F64
from .ib import kernel_fn


class Boxes:
    """boxes: (nb, 6) rows x0, x1, y0, y1, z0, z1; X: (nm, 3) marker positions; dV: (nm,) marker volumes."""

    def __init__(self, boxes, X, dV):
        self.boxes = torch.as_tensor(boxes, dtype=F64).reshape(-1, 6)
        self.X = torch.as_tensor(X, dtype=F64).reshape(-1, 3)
        self.dV = torch.as_tensor(dV, dtype=F64).reshape(-1)


def _shift(m, g, d, s):
    """Neighbour values m[index - s along d] (periodic wrap or zero outside the domain)."""
    ax = 2 - d
    if g.periodic(d):
        return torch.roll(m, s, dims=ax)
    e = m.shape[ax]
    z = torch.zeros_like(m.narrow(ax, 0, 1))
    if s == 1:
        return torch.cat([z, m.narrow(ax, 0, e - 1)], dim=ax)
    return torch.cat([m.narrow(ax, 1, e - 1), z], dim=ax)


def classify(g, body):
    """Per velocity component: (solid, ib) boolean masks of its faces."""
    out = []
    for c in range(g.dim):
        fx, fy, fz = [t.expand(g.shape(c)) for t in g.face_coords(c)]
        solid = torch.zeros(g.shape(c), dtype=torch.bool)
        for b in body.boxes:
            solid = solid | ((fx > b[0]) & (fx < b[1]) & (fy > b[2]) & (fy < b[3]) & (fz > b[4]) & (fz < b[5]))
        nb = torch.zeros_like(solid)
        for d in range(g.dim):
            for s in (-1, 1):
                nb = nb | _shift(solid, g, d, s)
        out.append((solid, (~solid) & nb))
    return out


def delta3(kind, dx, dy, dz, hx, hy, hz):
    phi = kernel_fn(kind)
    return phi(dx / hx) * phi(dy / hy) * phi(dz / hz) / (hx * hy * hz)


def weights(g, c, kind, X):
    """delta_h(x_face - X_i) for every face of component c: shape (nm,) + shape(c)."""
    hx, hy, hz = float(g.h[0][0]), float(g.h[1][0]), float(g.h[2][0])
    fx, fy, fz = g.face_coords(c)
    d = [fx.unsqueeze(0) - X[:, 0].reshape(-1, 1, 1, 1),
         fy.unsqueeze(0) - X[:, 1].reshape(-1, 1, 1, 1),
         fz.unsqueeze(0) - X[:, 2].reshape(-1, 1, 1, 1)]
    return delta3(kind, d[0], d[1], d[2], hx, hy, hz)


def marker_forces(g, body, kind, f):
    """q_i = -sum_faces f_c delta_h(x - X_i) dv_c (Eq. 20) and F = rho sum_i q_i dV_i."""
    q = []
    for c in range(g.dim):
        W = weights(g, c, kind, body.X)
        q.append(-(W * (f[c] * g.face_volume(c)).unsqueeze(0)).sum(dim=(1, 2, 3)))
    q = torch.stack(q, dim=1)
    F = g.rho * (q * body.dV.reshape(-1, 1)).sum(dim=0)
    return q, F
