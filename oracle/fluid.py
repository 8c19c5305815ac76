"""Finite-volume operators of §2.3.1 on the MAC grid (oracle, FP64).

  momentum_rhs   R(u) = -div(u (x) u) + nu lap(u) + body force, the bracket of
                 the predictor Eq. (4) without the IB forcing term
  divergence     D u at cell centres (the divergence in Eqs. 7-9)
  gradient       G p on faces (the gradient in Eqs. 6 and 10)

Discretisation (the paper fixes the scheme family, §2.3.1 and Table 1: 2nd-order
central diffusion, 1st-order upwind or 2nd-order central convection, FV on a
staggered grid); the details below are this project's reading of it:

* convection is in divergence form.  For the c-momentum control volume around
  a c-face, the flux through its faces normal to direction d is T * Q where T
  is the transporting velocity u_d interpolated to the flux point and Q is the
  transported u_c there: central takes Q linearly interpolated, upwind takes
  the upstream c-face value.  Along d == c the flux points are cell centres
  (T = Q = mean of the two c-faces of the cell for central); along d != c
  they are cell edges, T is interpolated along c, Q along d.  Interpolation is
  linear in the coordinate (metric-weighted on stretched grids).
* diffusion: nu times the difference of the two face gradients divided by the
  control-volume width.
* boundary ghosts for tangential components: no-slip / inflow reflect
  linearly about the wall value (ghost = 2 u_wall - u_interior), free-slip and
  zero-gradient outflow copy the interior value; ghost centres are mirrored
  across the boundary.  Normal components on non-periodic boundaries are
  stored boundary values (walls 0, inflow U) and are not updated by R.

Parity: pinned by tests against polynomial exactness, Taylor-Green decay in
closed form, Poiseuille flow against an independent tridiagonal solve, and
momentum conservation (tests/test_oracle_operators.py, test_oracle_flows.py).
The stretched-grid interpolation weights of the transported and transporting
velocities are pinned by exact linear fields on a tanh-stretched grid (hand
values from the face coordinates), the upwind direction by step profiles with
hand-computed first-order fluxes for both signs of the transport velocity.
"""
import torch

from .grid import PERIODIC, NOSLIP, FREESLIP, INFLOW, OUTFLOW


def pad_ghosts(g, c, uc):
    """Return component c with one ghost layer on every side: shape + (2, 2, 2).

    Ghost rules (module docstring).  Filling x, then y, then z makes corner
    ghosts consistent.  Ghosts along the component's own non-periodic
    direction are never read by an update of an interior face; they copy the
    boundary value.
    """
    E = uc
    for d in range(3):
        ax = 2 - d
        size = E.shape[ax]
        first = E.narrow(ax, 0, 1)
        last = E.narrow(ax, size - 1, 1)
        if g.periodic(d):
            lo, hi = last, first
        elif d == c:
            lo, hi = first, last
        else:
            ghosts = []
            for side, inner in ((0, first), (1, last)):
                kind = g.bc[d][side]
                if kind in (NOSLIP, INFLOW):
                    val = g.bc_val[d][side][c]
                    ghosts.append(2.0 * val - inner)
                elif kind in (FREESLIP, OUTFLOW):
                    ghosts.append(inner)
                else:
                    raise ValueError("unknown boundary type %r" % kind)
            lo, hi = ghosts
        E = torch.cat([lo, E, hi], dim=ax)
    return E


def shifted(E, shape, off):
    """Slice of a ghost-padded array seen from storage index + off (off per direction x, y, z)."""
    ez, ey, ex = shape
    ox, oy, oz = off
    return E[1 + oz:1 + oz + ez, 1 + oy:1 + oy + ey, 1 + ox:1 + ox + ex]


def _unit(d, s=1):
    o = [0, 0, 0]
    o[d] = s
    return o


def _add(a, b):
    return [a[i] + b[i] for i in range(3)]


def momentum_rhs(g, u):
    """R(u) = -div(u u) + nu lap(u) + f_body on every interior face (Eq. 4 bracket, §2.3.1).

    Returns a list of tensors with the shapes of u; boundary faces carry 0.
    """
    E = [pad_ghosts(g, c, u[c]) for c in range(g.dim)]
    R = []
    for c in range(g.dim):
        shp = g.shape(c)
        uc = lambda off: shifted(E[c], shp, off)  # noqa: E731
        conv = torch.zeros(shp, dtype=u[c].dtype)
        diff = torch.zeros(shp, dtype=u[c].dtype)
        for d in range(g.dim):
            if d == c:
                # flux points are the cell centres east (cell f) and west (cell f-1) of face f
                uW, u0, uE = uc(_unit(c, -1)), uc([0, 0, 0]), uc(_unit(c, 1))
                TE = 0.5 * (u0 + uE)
                TW = 0.5 * (uW + u0)
                if g.conv == "upwind":
                    QE = torch.where(TE > 0, u0, uE)
                    QW = torch.where(TW > 0, uW, u0)
                else:
                    QE, QW = TE, TW
                hf = g.along(c, _faces(g, c, g.hf[c]))
                hE = g.along(c, _cells_right(g, c))
                hW = g.along(c, _cells_left(g, c))
                conv = conv + (TE * QE - TW * QW) / hf
                diff = diff + ((uE - u0) / hE - (u0 - uW) / hW) / hf
            else:
                # flux points are the edges on d-faces m+1 (north) and m (south) of d-cell m
                ud = lambda off: shifted(E[d], shp, off)  # noqa: E731
                th_c = g.along(c, _faces(g, c, g.theta[c]))
                # transport u_d interpolated along c to the c-face: c-cells f-1 (off -1) and f (off 0)
                TN = (1 - th_c) * ud(_add(_unit(c, -1), _unit(d, 1))) + th_c * ud(_unit(d, 1))
                TS = (1 - th_c) * ud(_unit(c, -1)) + th_c * ud([0, 0, 0])
                uS, u0, uN = uc(_unit(d, -1)), uc([0, 0, 0]), uc(_unit(d, 1))
                th_d = g.theta[d]
                thN = g.along(d, _face_right(g, d, th_d))
                thS = g.along(d, th_d[:g.n[d]])
                if g.conv == "upwind":
                    QN = torch.where(TN > 0, u0, uN)
                    QS = torch.where(TS > 0, uS, u0)
                else:
                    QN = (1 - thN) * u0 + thN * uN
                    QS = (1 - thS) * uS + thS * u0
                hd = g.along(d, g.h[d])
                hfN = g.along(d, _face_right(g, d, g.hf[d]))
                hfS = g.along(d, g.hf[d][:g.n[d]])
                conv = conv + (TN * QN - TS * QS) / hd
                diff = diff + ((uN - u0) / hfN - (u0 - uS) / hfS) / hd
        Rc = -conv + g.nu * diff
        if c == 0 and g.body_force is not None:
            Rc = Rc + g.along(1, g.body_force)
        Rc = torch.where(g.interior_mask(c), Rc, torch.zeros_like(Rc))
        R.append(Rc)
    return R


def _faces(g, d, arr):
    """Per-face metric along d restricted to the stored faces of the normal component."""
    return arr[:g.n[d]] if g.periodic(d) else arr


def _face_right(g, d, arr):
    """Metric at the right face (m+1) of each cell m along d (wraps when periodic)."""
    if g.periodic(d):
        return torch.roll(arr[:g.n[d]], -1)
    return arr[1:g.n[d] + 1]


def _cells_right(g, c):
    """Width of the cell east of each stored c-face (cell f)."""
    h = g.h[c]
    if g.periodic(c):
        return h
    # faces 0..n: cell f for f < n, boundary face n has no east cell (value unused)
    return torch.cat([h, h[-1:]])


def _cells_left(g, c):
    """Width of the cell west of each stored c-face (cell f-1)."""
    h = g.h[c]
    if g.periodic(c):
        return torch.roll(h, 1)
    return torch.cat([h[:1], h])


def divergence(g, u):
    """(D u)_cell = sum_d (u_d[face m+1] - u_d[face m]) / h_d[m] at every cell centre."""
    out = torch.zeros(g.cshape(), dtype=u[0].dtype)
    nshape = g.cshape()
    for d in range(g.dim):
        ax = 2 - d
        nd = g.n[d]
        ud = u[d]
        if g.periodic(d):
            right = torch.roll(ud, -1, dims=ax)
            left = ud
        else:
            right = ud.narrow(ax, 1, nd)
            left = ud.narrow(ax, 0, nd)
        out = out + ((right - left) / g.along(d, g.h[d])).expand(nshape)
    return out


def gradient(g, p):
    """(G p)_c[face f] = (p[f] - p[f-1]) / hf_c[f] on interior faces, 0 on non-periodic boundary faces."""
    G = []
    for c in range(g.dim):
        ax = 2 - c
        nd = g.n[c]
        if g.periodic(c):
            Gc = (p - torch.roll(p, 1, dims=ax)) / g.along(c, g.hf[c])
        else:
            inner = (p.narrow(ax, 1, nd - 1) - p.narrow(ax, 0, nd - 1)) / g.along(c, g.hf[c][1:nd])
            zshape = list(p.shape)
            zshape[ax] = 1
            z = torch.zeros(zshape, dtype=p.dtype)
            Gc = torch.cat([z, inner, z], dim=ax)
        G.append(Gc)
    return G


def apply_boundary_values(g, u):
    """Normal velocity on non-periodic boundary faces: 0 on walls, U on the inflow face.

    The outflow face is set separately (outflow_faces)."""
    out = []
    for c in range(g.dim):
        uc = u[c]
        if not g.periodic(c):
            ax = 2 - c
            e = g.ext(c)[c]
            idx = g.along(c, torch.arange(e))
            for side, pos in ((0, 0), (1, e - 1)):
                kind = g.bc[c][side]
                if kind == OUTFLOW:
                    continue
                val = g.bc_val[c][side][c] if kind == INFLOW else 0.0
                uc = torch.where(idx == pos, torch.full_like(uc, val), uc)
        out.append(uc)
    return out


def boundary_flux_in(g, u):
    """Volume flux entering through every non-outflow boundary face (0 for walls and periodic)."""
    q = torch.zeros((), dtype=u[0].dtype)
    for c in range(g.dim):
        if g.periodic(c):
            continue
        ax = 2 - c
        e = g.ext(c)[c]
        area = _face_area(g, c)
        for side, pos in ((0, 0), (1, e - 1)):
            if g.bc[c][side] == OUTFLOW:
                continue
            sign = 1.0 if side == 0 else -1.0
            q = q + sign * (u[c].narrow(ax, pos, 1) * area).sum()
    return q


def _face_area(g, c):
    a = None
    for d in range(3):
        if d == c:
            continue
        v = g.along(d, g.h[d])
        a = v if a is None else a * v
    return a


def outflow_faces(g, u_prev, u_new):
    """Zero-gradient outflow at x-high (§3.1 "Neumann outflow du/dx = 0"), flux-corrected.

    The outflow face takes the last interior face of the previous state,
    u*[n] = s u[n-1], with s chosen so that the volume leaving equals the volume
    entering through the other boundaries.  That keeps the discrete Poisson
    problem with Neumann conditions on every side solvable.
    """
    if g.periodic(0) or g.bc[0][1] != OUTFLOW:
        return u_new
    nx = g.n[0]
    area = _face_area(g, 0)
    inner = u_prev[0].narrow(2, nx - 1, 1)
    q_out = (inner * area).sum()
    q_in = boundary_flux_in(g, u_new)
    s = q_in / q_out
    idx = g.along(0, torch.arange(nx + 1))
    u0 = torch.where(idx == nx, (s * inner).expand_as(u_new[0]), u_new[0])
    return [u0] + list(u_new[1:])
