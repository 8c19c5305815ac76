"""Immersed boundary of §2.2 and §2.3.3 (oracle, FP64; 2-D bodies).

  phi_peskin4, phi_roma3   1-D regularised kernels; Eq. (22) is the 4-point
                           kernel of the paper, the 3-point kernel (Roma,
                           Peskin & Berger 1999) is the one the FSI workload asks for
  delta                    tensor product delta_h = d_h(x) d_h(y), Eq. (21)
  inside_polygon           solid test of a point against the marker polygon (one or
                           several closed contours)
  classify                 solid faces (Omega_s) and IB faces (Omega_IB, fluid
                           faces with a solid neighbour, §2.2)
  half_distribution_sum    F_N_i of Eq. (19)
  target_velocity          u_s of Eq. (5): body velocity on solid faces
                           (Eq. 23), normalised marker interpolation on IB
                           faces (Eqs. 18-19)
  marker_forces            q_i of Eq. (20) and the body force F

Readings of the paper taken here:
* epsilon = 1 on solid faces and on IB faces (the direct forcing acts "in
  cells intersecting the immersed region", §2.3.1, and u_s is defined on IB
  points).
* Eq. (18) is applied in its normalised (convex) form
  u_IB(x) = sum_i w_i(x) wdot_i / sum_i w_i(x),  w_i = delta_h(x - X_i) dV_i / F_N_i,
  with F_N_i of Eq. (19) summed over the non-solid faces of the same velocity
  component.  A uniform marker velocity is then reproduced exactly.  An IB
  face outside every marker's support takes the body velocity.
* dV_i = (arc length of marker i) * h, the thin shell of one grid spacing of §2.3.3.
* F = rho sum_i q_i dV_i (the "integration over all Lagrangian nodes" of
  §2.3.2 with the nodal volume), torque likewise.
* The solid test is the crossing-number point-in-polygon test of the face
  position minus the body displacement against the rest polygon; it is an
  integer decision taken in FP64 with each operation rounded separately.

Parity: kernels pinned by their moment conditions; interpolation / spreading
by the transpose identity and exact reproduction of a uniform velocity; F_N
by the half-distribution value 1 / (2 h_x h_y) of a marker on a flat wall;
the normalised interpolation with non-uniform marker velocities by a
scalar-loop brute force; q_i, F and the torque by uniform (q = -f), rigid-
rotation (closed-form torque) and radial (zero torque) forcings
(tests/test_oracle_ib.py).  The coupled FSI trajectory is "parity unpinned"
against physics (no reference data); only GPU-vs-oracle applies there.
"""
import torch

from .grid import F64

PESKIN4, ROMA3 = 0, 1


def phi_peskin4(r):
    """Eq. (22) with h = 1: the 4-point kernel, support |r| < 2."""
    a = r.abs()
    inner = (3.0 - 2.0 * a + torch.sqrt(torch.clamp(1.0 + 4.0 * a - 4.0 * a * a, min=0.0))) / 8.0
    outer = (5.0 - 2.0 * a - torch.sqrt(torch.clamp(-7.0 + 12.0 * a - 4.0 * a * a, min=0.0))) / 8.0
    return torch.where(a <= 1.0, inner, torch.where(a <= 2.0, outer, torch.zeros_like(a)))


def phi_roma3(r):
    """3-point kernel (Roma, Peskin & Berger 1999), support |r| < 1.5."""
    a = r.abs()
    inner = (1.0 + torch.sqrt(torch.clamp(1.0 - 3.0 * a * a, min=0.0))) / 3.0
    b = 1.0 - a
    outer = (5.0 - 3.0 * a - torch.sqrt(torch.clamp(1.0 - 3.0 * b * b, min=0.0))) / 6.0
    return torch.where(a <= 0.5, inner, torch.where(a <= 1.5, outer, torch.zeros_like(a)))


def kernel_fn(kind):
    return phi_peskin4 if kind == PESKIN4 else phi_roma3


def delta(kind, dx, dy, hx, hy):
    """delta_h(x) = d_h(x) d_h(y), d_h(r) = phi(r / h) / h (Eqs. 21-22)."""
    phi = kernel_fn(kind)
    return phi(dx / hx) * phi(dy / hy) / (hx * hy)


def contour_next(nm, starts=None):
    """Index of the vertex after each vertex: closed contours [starts[k], starts[k+1]) (one contour
    of all nm markers when starts is None), each closing back to its first vertex."""
    starts = [0] if starts is None else [int(a) for a in starts]
    ends = starts[1:] + [nm]
    nxt = []
    for a, b in zip(starts, ends):
        nxt += list(range(a + 1, b)) + [a]
    return nxt


def inside_polygon(px, py, X, Y, nxt=None):
    """Crossing-number test of points (px, py) against the closed polygon (X, Y), or against a set of
    closed contours (vertex i joined to vertex nxt[i]): a point is inside when a ray from it crosses
    the edges an odd number of times, i.e. when it lies inside an odd number of the contours.

    Each operation is one IEEE-rounded FP64 operation in the order written."""
    inside = torch.zeros(torch.broadcast_shapes(px.shape, py.shape), dtype=torch.bool)
    nm = X.numel()
    if nxt is None:
        nxt = contour_next(nm)
    for i in range(nm):
        ax, ay = X[i], Y[i]
        bx, by = X[nxt[i]], Y[nxt[i]]
        cond = (ay > py) != (by > py)
        if float(by - ay) == 0.0:
            continue
        xint = ax + (py - ay) * (bx - ax) / (by - ay)
        inside = inside ^ (cond & (px < xint))
    return inside


class Body:
    """Rigid 2-D body: rest polygon of markers, arc-length weights, reference centre.

    X0, Y0      marker rest positions, ordered around the closed surface
    ds          arc length per marker
    contours    first marker of each closed contour when the body is made of several
                disjoint parts (an array of cylinders moving as one rigid body); None:
                one contour
    xc0         reference point (rotation centre) at rest
    omega       prescribed angular velocity (surface velocity only; the
                geometry translates but does not turn)
    """

    def __init__(self, X0, Y0, ds, xc0, omega=0.0, contours=None):
        self.X0 = torch.as_tensor(X0, dtype=F64)
        self.Y0 = torch.as_tensor(Y0, dtype=F64)
        self.ds = torch.as_tensor(ds, dtype=F64)
        self.xc0 = (float(xc0[0]), float(xc0[1]))
        self.omega = float(omega)
        self.next = contour_next(self.X0.numel(), contours)

    def markers(self, w):
        return self.X0 + w[0], self.Y0 + w[1]

    def velocity_at(self, x, y, w, wdot):
        """Rigid velocity V + omega x (r - r_c) at points (x, y)."""
        cx = self.xc0[0] + w[0]
        cy = self.xc0[1] + w[1]
        return wdot[0] - self.omega * (y - cy), wdot[1] + self.omega * (x - cx)


def classify(g, body, w):
    """Per velocity component: (solid, ib) boolean masks of its faces (§2.2, Fig. 2)."""
    out = []
    for c in range(g.dim):
        fx, fy, _ = g.face_coords(c)
        px = (fx - w[0]).expand(g.shape(c))
        py = (fy - w[1]).expand(g.shape(c))
        solid = inside_polygon(px, py, body.X0, body.Y0, body.next)
        nb = torch.zeros_like(solid)
        for d in range(2):
            ax = 2 - d
            for s in (-1, 1):
                if g.periodic(d):
                    sh = torch.roll(solid, s, dims=ax)
                else:
                    e = solid.shape[ax]
                    z = torch.zeros_like(solid.narrow(ax, 0, 1))
                    if s == 1:
                        sh = torch.cat([z, solid.narrow(ax, 0, e - 1)], dim=ax)
                    else:
                        sh = torch.cat([solid.narrow(ax, 1, e - 1), z], dim=ax)
                nb = nb | sh
        out.append((solid, (~solid) & nb))
    return out


def _spacing(g):
    return float(g.h[0][0]), float(g.h[1][0])


def weights_matrix(g, c, kind, Xm, Ym):
    """delta_h(x_face - X_i) for every face of component c and marker i: shape (nm,) + shape(c)."""
    hx, hy = _spacing(g)
    fx, fy, _ = g.face_coords(c)
    dx = fx.unsqueeze(0) - Xm.reshape(-1, 1, 1, 1)
    dy = fy.unsqueeze(0) - Ym.reshape(-1, 1, 1, 1)
    return delta(kind, dx, dy, hx, hy)


def half_distribution_sum(g, c, kind, Xm, Ym, solid):
    """F_N_i of Eq. (19) for component c: sum over the c-faces that are not solid of delta_h(x - X_i)."""
    W = weights_matrix(g, c, kind, Xm, Ym)
    return (W * (~solid).unsqueeze(0)).sum(dim=(1, 2, 3))


def target_velocity(g, body, kind, w, wdot, masks):
    """u_s of Eq. (5) on forced faces and the exact solid velocity u_c of Eq. (8).

    Returns (ut, uc) lists over components; values off forced faces are 0.
    """
    hx, hy = _spacing(g)
    Xm, Ym = body.markers(w)
    dV = body.ds * hx                                 # shell of thickness h (§2.3.3)
    mvx, mvy = body.velocity_at(Xm, Ym, w, wdot)
    mv = (mvx, mvy)
    ut, ucl = [], []
    for c in range(g.dim):
        solid, ib = masks[c]
        fx, fy, _ = g.face_coords(c)
        bvx, bvy = body.velocity_at(fx.expand(g.shape(c)), fy.expand(g.shape(c)), w, wdot)
        bv = (bvx, bvy)[c]
        W = weights_matrix(g, c, kind, Xm, Ym)         # (nm, ez, ey, ex)
        FN = half_distribution_sum(g, c, kind, Xm, Ym, solid)          # Eq. (19)
        FNs = torch.where(FN > 0, FN, torch.ones_like(FN))
        wgt = W * (dV / FNs).reshape(-1, 1, 1, 1)
        num = (wgt * mv[c].reshape(-1, 1, 1, 1)).sum(dim=0)
        den = wgt.sum(dim=0)
        uib = torch.where(den > 0, num / torch.where(den > 0, den, torch.ones_like(den)), bv)
        zero = torch.zeros_like(bv)
        ut.append(torch.where(solid, bv, torch.where(ib, uib, zero)))
        ucl.append(torch.where(solid | ib, bv, zero))
    return ut, ucl


def marker_forces(g, body, kind, w, f):
    """q_i of Eq. (20) per marker and component, and (F, torque) = rho sum_i dV_i (q_i, r_i x q_i)."""
    hx, hy = _spacing(g)
    Xm, Ym = body.markers(w)
    dV = body.ds * hx
    q = []
    for c in range(g.dim):
        W = weights_matrix(g, c, kind, Xm, Ym)
        dv = g.face_volume(c)
        q.append(-(W * (f[c] * dv).unsqueeze(0)).sum(dim=(1, 2, 3)))
    q = torch.stack(q, dim=1)                          # (nm, 2)
    F = g.rho * (q * dV.reshape(-1, 1)).sum(dim=0)
    rx = Xm - (body.xc0[0] + w[0])
    ry = Ym - (body.xc0[1] + w[1])
    torque = g.rho * (dV * (rx * q[:, 1] - ry * q[:, 0])).sum()
    return q, F, torque
