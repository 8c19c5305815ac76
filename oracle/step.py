"""One fractional-step time step (oracle, FP64): Eqs. (4)-(10) of §2.3.1, the
immersed-boundary coupling of §2.3.3 and the rigid body of §2.3.2.

Forward Euler (the scheme of every run in §3):
  1. markers X_i = X_i^0 + w^n; solid / IB faces; u_s and u_c (ib.py)
  2. predictor with direct forcing, Eqs. (4)-(5):
        f  = eps [ -R(u^n) + (u_s - u^n) / dt ]
        u* = u^n + dt (R(u^n) + f) = (1 - eps)(u^n + dt R) + eps u_s
  3. pressure Poisson Eq. (9) and correction Eq. (10), with phi = dt p / rho:
        L phi = D[(1 - eps) u* + eps u_c],   u^{n+1} = u* - G phi
  4. q_i from f (Eq. 20), F = rho sum q_i dV_i, then the body by RK4 (Eq. 12)
A static 3-D body (ib3d.Boxes) is forced the same way with u_s = u_c = 0.

Runge-Kutta ("explicit Runge-Kutta", §2.5; tableau not given): the strong-
stability-preserving three-stage scheme of Shu and Osher with a projection
after every stage, for grids without a body or an outflow:
  u1 = P(u^n + dt R(u^n)),  u2 = P(3/4 u^n + 1/4 (u1 + dt R(u1))),
  u^{n+1} = P(1/3 u^n + 2/3 (u2 + dt R(u2))).

The outflow face (zero gradient, flux-corrected) and the boundary values are
applied to u* before the projection.

Parity: the pieces are pinned in their own modules; the composition is
pinned by Taylor-Green decay, Poiseuille flow, divergence-free projection and
momentum conservation (tests/test_oracle_flows.py), the SSP-RK3 tableau by
third-order convergence in dt (error ratios ~8 per halving; a swapped stage
weight drops it to ~2), and its autograd adjoint by central finite
differences (tests/test_oracle_adjoint.py).  The implicit-differentiation
adjoint of the strongly coupled step (step_coupled_adjoint) is pinned by
central finite differences of the coupled step converged to rounding and by
reverse-mode AD through the unrolled sub-iterations
(tests/test_oracle_coupling.py).
"""
import torch

from . import body as body_mod
from . import fluid, ib, ib3d, les, poisson
from .grid import F64

SSPRK3 = ((0.0, 1.0), (0.75, 0.25), (1.0 / 3.0, 2.0 / 3.0))


class State:
    """u: list of velocity components; w, wd: body displacement and velocity (2,), or None."""

    def __init__(self, u, w=None, wd=None):
        self.u = u
        self.w = w
        self.wd = wd


class Diagnostics:
    def __init__(self):
        self.f = None
        self.q = None
        self.F = None
        self.torque = None
        self.phi = None
        self.eps = None


def _predictor(g, u_in, dt, eps=None, ut=None, cs=0.0):
    """Eq. (4)-(5): returns (u*, f).  cs > 0 adds the Smagorinsky subgrid term (les.py)."""
    R = fluid.momentum_rhs(g, u_in)
    if cs > 0.0:
        R = [a + b for a, b in zip(R, les.sgs_term(g, u_in, cs))]
    ustar, f = [], []
    for c in range(g.dim):
        base = u_in[c] + dt * R[c]
        if eps is None:
            ustar.append(base)
            f.append(torch.zeros_like(base))
        else:
            e = eps[c]
            ustar.append(torch.where(e, ut[c], base))
            f.append(torch.where(e, -R[c] + (ut[c] - u_in[c]) / dt, torch.zeros_like(base)))
    return ustar, f


def step(g, st, dt, scheme="fe", body=None, kernel=ib.ROMA3, params=None, cs=0.0):
    """Advance one step; returns (new State, Diagnostics).  cs: Smagorinsky constant (0: no model)."""
    dg = Diagnostics()
    u = fluid.apply_boundary_values(g, st.u)
    if scheme == "rk3":
        assert body is None and not (not g.periodic(0) and g.bc[0][1] == fluid.OUTFLOW), \
            "RK3 is provided for grids without a body or an outflow"
        v = u
        for a, b in SSPRK3:
            ustar, _ = _predictor(g, v, dt, cs=cs)
            ut = [a * u[c] + b * ustar[c] for c in range(g.dim)]
            ut = fluid.apply_boundary_values(g, ut)
            v, phi = poisson.project(g, ut)
        dg.phi = phi
        return State(v, st.w, st.wd), dg

    eps = ut = ucl = masks = None
    static3d = isinstance(body, ib3d.Boxes)
    if static3d:
        # body at rest: u_s = 0 on every forced face, u_c = 0
        masks = ib3d.classify(g, body)
        ut = [torch.zeros(g.shape(c), dtype=F64) for c in range(g.dim)]
        ucl = ut
        eps = [m[0] | m[1] for m in masks]
        dg.eps = eps
    elif body is not None:
        masks = ib.classify(g, body, st.w)
        ut, ucl = ib.target_velocity(g, body, kernel, st.w, st.wd, masks)
        eps = [m[0] | m[1] for m in masks]
        dg.eps = eps
    ustar, f = _predictor(g, u, dt, eps, ut, cs=cs)
    ustar = fluid.apply_boundary_values(g, ustar)
    ustar = fluid.outflow_faces(g, u, ustar)
    unew, phi = poisson.project(g, ustar, ucl, eps)
    dg.phi = phi
    dg.f = f
    w_new, wd_new = st.w, st.wd
    if static3d:
        dg.q, dg.F = ib3d.marker_forces(g, body, kernel, f)
    elif body is not None:
        q, F, torque = ib.marker_forces(g, body, kernel, st.w, f)
        dg.q, dg.F, dg.torque = q, F, torque
        if params is not None:
            w_new, wd_new = body_mod.rk4(params, st.w, st.wd, F, dt)
    return State(unew, w_new, wd_new), dg


def step_coupled(g, st, dt, body, kernel=ib.ROMA3, params=None, max_iter=100, tol=1e-5):
    """Strongly coupled FSI step: the sub-iteration of the paper's strong-coupling
    procedure (§2.3.3, Algorithm 1), from the fluid state and body state of time level n.

    Iterate k = 1, 2, ...: advance the fluid from u^n with the body kinematics of
    the current iterate (iterate 0 = the body at level n), take the force of that
    fluid step, advance the body ODE from its level-n state with that force, and
    measure xi = |w_k - w_{k-1}|^2 / |w_{k-1}|^2 (the plain |w_k - w_{k-1}|^2 while
    w_{k-1} = 0).  Stop when xi < tol or after max_iter fluid solves.  One
    sub-iteration is the weakly coupled step.

    Returns (new State, Diagnostics of the last fluid solve, sub-iterations, last xi).
    """
    w_it, wd_it = st.w, st.wd
    xi = float("inf")
    k = 0
    while k < max_iter:
        new, dg = step(g, State(st.u, w_it, wd_it), dt, "fe", body, kernel, params=None)
        k += 1
        w_new, wd_new = body_mod.rk4(params, st.w, st.wd, dg.F, dt)
        den = float((w_it * w_it).sum().detach())
        num = float(((w_new - w_it) ** 2).sum().detach())
        xi = num / den if den > 0.0 else num
        w_it, wd_it = w_new, wd_new
        if xi < tol:
            break
    return State(new.u, w_it, wd_it), dg, k, xi


def step_coupled_adjoint(g, st, dt, body, kernel, params, lam_u, lam_body, dJdF, max_iter=100, tol=1e-5):
    """Reverse of the strongly coupled step by implicit differentiation (§2.4.1) of its fixed point.

    The converged body state s* = (w*, wdot*) of Algorithm 1 satisfies
        R(s*, theta) = s* - B(s^n, F(u^n, s*), k) = 0,
    where F(u^n, s) is the force of the fluid step advanced from u^n with the body kinematics s
    and B the RK4 step of Eq. (12) from the level-n body state s^n; the new velocity is
    u^{n+1} = U(u^n, s*).  For the loss L(u^{n+1}, s*, F) with adjoint seeds (lam_u, lam_body,
    dJdF) the paper's adjoint equation reads
        (dR/ds)^T lam = (dL/ds)^T,  dL/dtheta = (explicit part) - lam^T dR/dtheta,
    with theta = (u^n, s^n, k).  The fluid step and the body step are linearised at the converged
    iterate (the body state step_coupled returns); their partial derivatives come from
    torch.autograd, dR/ds = I - dB/ds is formed column by column (4 x 4) and the 4-unknown system
    is solved directly.

    Returns (lam_u^n, lam_body^n (4,), dJ/dk) and the sub-iteration count of the forward solve.
    """
    with torch.no_grad():
        new, _, iters, _ = step_coupled(g, State([x.detach() for x in st.u], st.w.detach(), st.wd.detach()), dt,
                                        body, kernel, params, max_iter, tol)
    s_star = torch.cat([new.w, new.wd]).detach().clone().requires_grad_(True)
    u_n = [x.detach().clone().requires_grad_(True) for x in st.u]
    s_n = torch.cat([st.w, st.wd]).detach().clone().requires_grad_(True)
    k = torch.tensor(float(params.k), dtype=F64, requires_grad=True)
    p = body_mod.RigidParams(params.m, k, params.c, params.active)
    fl, dg = step(g, State(u_n, s_star[:2], s_star[2:]), dt, "fe", body, kernel, params=None)
    w_b, wd_b = body_mod.rk4(p, s_n[:2], s_n[2:], dg.F, dt)
    B = torch.cat([w_b, wd_b])
    seeds_u = [torch.as_tensor(a, dtype=F64) for a in lam_u]
    sig = torch.as_tensor(lam_body, dtype=F64)
    fbar = torch.as_tensor(dJdF, dtype=F64)
    # partial dL/ds at s*: lam_body directly, plus the fluid outputs' dependence on the kinematics
    dLds = torch.autograd.grad(list(fl.u) + [dg.F], s_star, seeds_u + [fbar], retain_graph=True)[0] + sig
    # dR/ds = I - dB/ds, row i of dB/ds from the vector-Jacobian product with e_i
    dBds = torch.stack([torch.autograd.grad(B, s_star, torch.eye(4, dtype=F64)[i], retain_graph=True,
                                            allow_unused=True)[0] for i in range(4)])
    lam = torch.linalg.solve((torch.eye(4, dtype=F64) - dBds).T, dLds)
    # explicit part through U and F, then -lam^T dR/dtheta = lam^T dB/dtheta
    ex = torch.autograd.grad(list(fl.u) + [dg.F], u_n, seeds_u + [fbar], retain_graph=True)
    th = torch.autograd.grad(B, u_n + [s_n, k], lam, allow_unused=True)
    lam_un = [a + (b if b is not None else torch.zeros_like(a)) for a, b in zip(ex, th[:len(u_n)])]
    lam_sn = th[len(u_n)] if th[len(u_n)] is not None else torch.zeros(4, dtype=F64)
    dk = th[len(u_n) + 1] if th[len(u_n) + 1] is not None else torch.zeros((), dtype=F64)
    return [x.detach() for x in lam_un], lam_sn.detach(), dk.detach(), iters


def kinetic_energy(g, u):
    """1/2 sum over faces of u_c^2 times the face control volume."""
    ke = torch.zeros((), dtype=F64)
    for c in range(g.dim):
        ke = ke + 0.5 * (u[c] * u[c] * g.face_volume(c)).sum()
    return ke
