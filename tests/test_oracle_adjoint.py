"""Pin of the oracle's adjoint (reverse-mode AD through step(), as the paper differentiates its
solver, §2.4.1): directional derivatives against central finite differences in FP64."""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S
from helpers import grid_of, body_of

P, NS = S.PERIODIC, S.NOSLIP


def _fd_check(J, x0, direction, grad):
    """Best agreement over a scan of central-difference steps (1e-2 .. 1e-7 of |x0|)."""
    ad = float((grad * direction).sum())
    scale = max(float(x0.abs().max()), 1e-3)
    best = np.inf
    for k in range(2, 8):
        e = scale * 10.0 ** (-k)
        with torch.no_grad():
            fd = (float(J(x0 + e * direction)) - float(J(x0 - e * direction))) / (2 * e)
        best = min(best, abs(fd - ad) / max(abs(ad), 1e-300))
    return best


def _rollout_ke(g, u0, steps, dt, scheme):
    st = O.State(u0)
    for _ in range(steps):
        st, _ = O.step(g, st, dt, scheme=scheme)
    return O.kinetic_energy(g, st.u)


@pytest.mark.parametrize("scheme,conv", [("fe", "central"), ("rk3", "central"), ("fe", "upwind")])
def test_adjoint_initial_field_periodic_3d(scheme, conv):
    wl = S.box_3d(6, 6, 6, (P, P), (P, P), nu=0.05)
    wl.conv = conv
    g = grid_of(wl)
    rng = np.random.default_rng(21)
    u0 = [torch.tensor(rng.uniform(-1, 1, size=g.shape(c)), requires_grad=True) for c in range(3)]
    J = _rollout_ke(g, u0, 3, 0.02, scheme)
    grads = torch.autograd.grad(J, u0)
    dirs = [torch.tensor(rng.uniform(-1, 1, size=g.shape(c))) for c in range(3)]
    flat0 = torch.cat([u.detach().reshape(-1) for u in u0])
    flatd = torch.cat([d.reshape(-1) for d in dirs])
    flatg = torch.cat([gr.reshape(-1) for gr in grads])

    def Jf(x):
        parts, o = [], 0
        for c in range(3):
            n = int(np.prod(g.shape(c)))
            parts.append(x[o:o + n].reshape(g.shape(c)))
            o += n
        return _rollout_ke(g, parts, 3, 0.02, scheme)

    assert _fd_check(Jf, flat0, flatd, flatg) < 1e-6


def test_adjoint_body_force_channel():
    wl = S.box_3d(6, 8, 4, (P, P), (NS, NS), L=(2.0, 2.0, 1.0), stretched=1.5, nu=0.05)
    rng = np.random.default_rng(22)
    u0 = [torch.tensor(rng.uniform(-1, 1, size=grid_of(wl).shape(c))) for c in range(3)]
    u0[1][:, 0, :] = 0
    u0[1][:, -1, :] = 0
    fx0 = torch.tensor(rng.uniform(0.5, 1.5, size=8), requires_grad=True)

    def J(fx):
        wl.body_force = fx
        g = grid_of(wl)
        g.body_force = fx
        st = O.State(u0)
        for _ in range(3):
            st, _ = O.step(g, st, 0.01)
        return O.kinetic_energy(g, st.u)

    grad, = torch.autograd.grad(J(fx0), fx0)
    d = torch.tensor(rng.uniform(-1, 1, size=8))
    assert _fd_check(J, fx0.detach(), d, grad) < 1e-6


def test_adjoint_stiffness_fsi():
    """d/dk of sum_n C_L(n)^2 over a short FSI rollout (no face changes solid/fluid in the horizon)."""
    wl = S.cylinder_2d(nx=40, ny=32, cells_per_d=8, nm=26, dt=0.01, centre_d=(2.0, 2.0),
                       seed=3, perturb=0.05)
    g = grid_of(wl)
    body, params = body_of(wl)
    k0 = torch.tensor(wl.body.stiffness, dtype=torch.float64, requires_grad=True)
    u0 = [torch.tensor(a) for a in wl.u0]

    def J(k):
        params.k = k
        st = O.State(u0, torch.tensor([0.0, 0.02], dtype=torch.float64), torch.zeros(2, dtype=torch.float64))
        tot = torch.zeros((), dtype=torch.float64)
        for _ in range(4):
            st, dg = O.step(g, st, wl.dt, body=body, kernel=wl.kernel, params=params)
            tot = tot + (2.0 * dg.F[1]) ** 2
        return tot + st.w[1] ** 2 * 100

    grad, = torch.autograd.grad(J(k0), k0)
    assert abs(float(grad)) > 0
    assert _fd_check(J, k0.detach(), torch.ones((), dtype=torch.float64), grad) < 1e-6
