"""Build a Grid from any object describing a workload (duck-typed attributes:
dim, n, xf, bc, bc_val, nu, rho, conv, scheme, precision, body_force, body)."""
import torch

from . import fsstep as F


def grid_from_workload(wl, precision=None, stream=None):
    prec = precision if precision is not None else wl.precision
    prec = F.MIXED if prec in ("mixed", F.MIXED) else F.FP64
    g = F.Grid(wl.dim, wl.n, wl.xf, wl.bc, wl.bc_val, wl.nu, wl.rho,
               conv=F.UPWIND1 if wl.conv == "upwind" else F.CENTRAL2,
               scheme=F.RK3 if wl.scheme == "rk3" else F.FE, precision=prec,
               body_force=wl.body_force, stream=stream)
    b = getattr(wl, "body", None)
    if b is not None:
        g.set_body(b.X0, b.Y0, b.ds, b.centre, b.omega, b.mass, b.stiffness, b.damping, b.active,
                   kernel=wl.kernel, contours=getattr(b, "contours", None))
    bx = getattr(wl, "boxes", None)
    if bx is not None:
        g.set_boxes(bx.boxes, bx.X, bx.dV, wl.kernel)
    return g


def body_tensor(wl, device="cuda"):
    """Device FP64 body state [w_x, w_y, wdot_x, wdot_y] of a workload, or None."""
    b = getattr(wl, "body", None)
    if b is None:
        return None
    return torch.tensor([b.w0[0], b.w0[1], b.wd0[0], b.wd0[1]], dtype=torch.float64, device=device)
