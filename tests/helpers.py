"""Test helpers: build oracle grids and states from synthetic workloads."""
import numpy as np
import torch

import oracle as O
from oracle import ib as oib
from oracle.body import RigidParams


def grid_of(wl):
    return O.Grid(wl.dim, wl.n, wl.xf, wl.bc, wl.bc_val, wl.nu, wl.rho, wl.conv,
                  None if wl.body_force is None else wl.body_force)


def state_of(wl, u=None):
    u = wl.u0 if u is None else u
    tu = [torch.tensor(np.asarray(a), dtype=torch.float64) for a in u]
    if wl.body is not None:
        return O.State(tu, torch.tensor(wl.body.w0, dtype=torch.float64),
                       torch.tensor(wl.body.wd0, dtype=torch.float64))
    return O.State(tu)


def body_of(wl):
    bx = getattr(wl, "boxes", None)
    if bx is not None:
        from oracle import ib3d
        return ib3d.Boxes(bx.boxes, bx.X, bx.dV), None
    b = wl.body
    if b is None:
        return None, None
    body = oib.Body(b.X0, b.Y0, b.ds, b.centre, b.omega, getattr(b, "contours", None))
    params = RigidParams(b.mass, b.stiffness, b.damping, b.active) if b.mass > 0 else None
    return body, params


def rel_l2(a, b):
    num = sum(float(((x - y) ** 2).sum()) for x, y in zip(a, b))
    den = sum(float((y ** 2).sum()) for y in b)
    return (num / max(den, 1e-300)) ** 0.5
