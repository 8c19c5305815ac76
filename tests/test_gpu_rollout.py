"""Whole-rollout gradients through FsRollout (revolve checkpointing + fs_step_adjoint) vs the
oracle's reverse-mode AD of the same rollout: dJ/du0 (isotropic RK3), dJ/df_x(y) (channel),
dJ/dk and dJ/du0 (elastically mounted cylinder with a force-history loss)."""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S
from helpers import body_of, grid_of, rel_l2

pytestmark = pytest.mark.gpu
P, NS = S.PERIODIC, S.NOSLIP


def face_volumes(wl, dev):
    g = grid_of(wl)
    return [g.face_volume(c).contiguous().to(dev) for c in range(wl.dim)]


@pytest.mark.parametrize("slots", [1, 3, None])
def test_rollout_gradient_initial_field_rk3(slots):
    from paper_2505_23940_b300 import grid_from_workload
    from paper_2505_23940_b300.autodiff import rollout
    wl = S.isotropic_3d(n=16, steps=6)
    n = 6
    # oracle
    g = grid_of(wl)
    u = [torch.tensor(a, requires_grad=True) for a in wl.u0]
    st = O.State(u)
    for _ in range(n):
        st, _ = O.step(g, st, wl.dt, scheme="rk3")
    J = O.kinetic_energy(g, st.u)
    go = torch.autograd.grad(J, u)
    # GPU, FP64
    G = grid_from_workload(wl, "fp64")
    u0 = [torch.tensor(a, device="cuda", requires_grad=True) for a in wl.u0]
    uT, _, _ = rollout(G, u0, wl.dt, n, slots=slots)
    V = face_volumes(wl, "cuda")
    Jg = sum(0.5 * (x * x * v).sum() for x, v in zip(uT, V))
    gg = torch.autograd.grad(Jg, u0)
    assert abs(float(Jg) - float(J)) < 1e-12 * abs(float(J))
    assert rel_l2([x.cpu() for x in gg], list(go)) < 1e-11


def test_rollout_gradient_body_force_channel():
    from paper_2505_23940_b300 import grid_from_workload
    from paper_2505_23940_b300.autodiff import rollout
    wl = S.channel_3d(nx=16, ny=12, nz=8, steps=5)
    n = 5
    g = grid_of(wl)
    fx = torch.tensor(wl.body_force, requires_grad=True)
    g.body_force = fx
    st = O.State([torch.tensor(a) for a in wl.u0])
    for _ in range(n):
        st, _ = O.step(g, st, wl.dt)
    J = O.kinetic_energy(g, st.u)
    go, = torch.autograd.grad(J, fx)
    G = grid_from_workload(wl, "fp64")
    u0 = [torch.tensor(a, device="cuda") for a in wl.u0]
    fxg = torch.tensor(wl.body_force, device="cuda", requires_grad=True)
    uT, _, _ = rollout(G, u0, wl.dt, n, slots=2, body_force=fxg)
    V = face_volumes(wl, "cuda")
    Jg = sum(0.5 * (x * x * v).sum() for x, v in zip(uT, V))
    gg, = torch.autograd.grad(Jg, fxg)
    assert rel_l2([gg.cpu()], [go]) < 1e-11


def test_rollout_gradient_stiffness_fsi():
    from paper_2505_23940_b300 import body_tensor, grid_from_workload
    from paper_2505_23940_b300.autodiff import rollout
    wl = S.cylinder_2d(nx=48, ny=32, cells_per_d=8, nm=26, dt=0.01, centre_d=(2.0, 2.0), precision="fp64",
                       seed=3, perturb=0.05)
    wl.body.w0 = (0.0, 0.03)
    n = 5
    g = grid_of(wl)
    body, params = body_of(wl)
    k = torch.tensor(wl.body.stiffness, dtype=torch.float64, requires_grad=True)
    params.k = k
    u = [torch.tensor(a, requires_grad=True) for a in wl.u0]
    st = O.State(u, torch.tensor(wl.body.w0, dtype=torch.float64), torch.tensor(wl.body.wd0, dtype=torch.float64))
    J = torch.zeros((), dtype=torch.float64)
    for _ in range(n):
        st, dg = O.step(g, st, wl.dt, body=body, kernel=wl.kernel, params=params)
        J = J + dg.F[1] ** 2
    J = J + 50.0 * st.w[1] ** 2
    go = torch.autograd.grad(J, [k] + u)
    G = grid_from_workload(wl, "fp64")
    u0 = [torch.tensor(a, device="cuda", requires_grad=True) for a in wl.u0]
    kg = torch.tensor([wl.body.stiffness], dtype=torch.float64, device="cuda", requires_grad=True)
    uT, bT, forces = rollout(G, u0, wl.dt, n, slots=2, body0=body_tensor(wl), stiffness=kg)
    Jg = (forces[:, 1] ** 2).sum() + 50.0 * bT[1] ** 2
    gg = torch.autograd.grad(Jg, [kg] + u0)
    assert abs(float(Jg) - float(J)) < 1e-10 * abs(float(J))
    assert abs(float(gg[0]) - float(go[0])) < 1e-9 * abs(float(go[0]))
    assert rel_l2([x.cpu() for x in gg[1:]], list(go[1:])) < 1e-10


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_recorded_stages_match_recomputed_adjoint(precision):
    """fs_step_record leaves the state fs_step gives, and fs_step_adjoint_recorded on its
    stage states gives fs_step_adjoint's result (same kernels on the same stage values)."""
    from paper_2505_23940_b300 import grid_from_workload
    wl = S.isotropic_3d(n=16, steps=3)
    G = grid_from_workload(wl, precision)
    dt_ = G.dtype
    u0 = [torch.tensor(np.asarray(a), dtype=dt_, device="cuda").contiguous() for a in wl.u0]
    ua = [x.clone() for x in u0]
    ub = [x.clone() for x in u0]
    G.step(ua, wl.dt, 1)
    v1 = [torch.empty_like(x) for x in u0]
    v2 = [torch.empty_like(x) for x in u0]
    G.step_record(ub, wl.dt, v1, v2)
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(ua, ub))
    rng = np.random.default_rng(4)
    lam = [torch.tensor(rng.standard_normal(tuple(x.shape)), dtype=dt_, device="cuda") for x in u0]
    la = [x.clone() for x in lam]
    lb = [x.clone() for x in lam]
    G.step_adjoint(u0, la, wl.dt)
    G.step_adjoint_recorded(u0, v1, v2, lb, wl.dt)
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(la, lb))


def test_rollout_gradient_stiffness_strong_coupling():
    """dJ/dk and dJ/du0 of a 3-step strongly coupled FSI rollout (2-DOF, sub-iterations converged to
    rounding) through FsRollout against the oracle's implicit-differentiation adjoint chained over the
    same steps (each step reversed at its own converged fixed point)."""
    from oracle.step import step_coupled, step_coupled_adjoint
    from paper_2505_23940_b300 import body_tensor, grid_from_workload
    from paper_2505_23940_b300.autodiff import rollout
    wl = S.cylinder_2d(nx=48, ny=32, cells_per_d=8, nm=26, dt=0.01, centre_d=(2.0, 2.0), precision="fp64",
                       seed=3, perturb=0.05, mass_ratio=1.0)
    wl.body.w0 = (0.02, 0.05)
    wl.body.active = (True, True)
    n, tol = 3, 1e-28
    g = grid_of(wl)
    body, params = body_of(wl)
    f64 = torch.float64
    st = O.State([torch.tensor(a, dtype=f64) for a in wl.u0], torch.tensor(wl.body.w0, dtype=f64),
                 torch.tensor(wl.body.wd0, dtype=f64))
    states, Fy = [], []
    for _ in range(n):
        states.append(st)
        st, dg, _, _ = step_coupled(g, st, wl.dt, body, wl.kernel, params, max_iter=200, tol=tol)
        Fy.append(float(dg.F[1]))
    J = sum(f * f for f in Fy) + 50.0 * float(st.w[1]) ** 2
    lam_u = [np.zeros(g.shape(c)) for c in range(2)]
    lam_b = [0.0, 100.0 * float(st.w[1]), 0.0, 0.0]
    dk = 0.0
    for t in range(n - 1, -1, -1):
        lu, ls, dkt, _ = step_coupled_adjoint(g, states[t], wl.dt, body, wl.kernel, params, lam_u, lam_b,
                                              [0.0, 2.0 * Fy[t]], max_iter=200, tol=tol)
        lam_u, lam_b, dk = [x.numpy() for x in lu], ls.tolist(), dk + float(dkt)
    G = grid_from_workload(wl, "fp64")
    G.set_coupling(200, tol)
    u0 = [torch.tensor(a, device="cuda", requires_grad=True) for a in wl.u0]
    kg = torch.tensor([wl.body.stiffness], dtype=f64, device="cuda", requires_grad=True)
    uT, bT, forces = rollout(G, u0, wl.dt, n, slots=2, body0=body_tensor(wl), stiffness=kg)
    Jg = (forces[:, 1] ** 2).sum() + 50.0 * bT[1] ** 2
    gg = torch.autograd.grad(Jg, [kg] + u0)
    assert abs(float(Jg) - J) < 1e-10 * abs(J)
    assert abs(float(gg[0]) - dk) < 1e-9 * abs(dk), (float(gg[0]), dk)
    assert rel_l2([x.cpu() for x in gg[1:]], [torch.tensor(a) for a in lam_u]) < 1e-9
