"""GPU discrete adjoint (fs_step_adjoint) vs the oracle's reverse-mode AD of the same step (§2.4.1).

For random adjoint seeds lam^{n+1} (velocity, body state) and dJ/dF, the GPU must return
lam^n = (d step / d state^n)^T lam^{n+1} and the parameter gradients (body-force profile,
spring stiffness) that torch.autograd gives through the oracle's step.
Tolerances: relative L2 1e-11 (FP64 grids), 1e-5 (mixed grids)."""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S
from helpers import body_of, grid_of, rel_l2

pytestmark = pytest.mark.gpu
P, NS, FS, IN, OUT = S.PERIODIC, S.NOSLIP, S.FREESLIP, S.INFLOW, S.OUTFLOW


def oracle_vjp(wl, u0, lam_u, dt, lam_body=None, dJdF=None):
    g = grid_of(wl)
    body, params = body_of(wl)
    u = [torch.tensor(np.asarray(a), dtype=torch.float64, requires_grad=True) for a in u0]
    inputs = list(u)
    fx = None
    if wl.body_force is not None:
        fx = torch.tensor(np.asarray(wl.body_force), dtype=torch.float64, requires_grad=True)
        g.body_force = fx
        inputs.append(fx)
    k = None
    if body is not None:
        w = torch.tensor(wl.body.w0, dtype=torch.float64, requires_grad=True)
        wd = torch.tensor(wl.body.wd0, dtype=torch.float64, requires_grad=True)
        inputs += [w, wd]
        if params is not None:
            k = torch.tensor(float(params.k), dtype=torch.float64, requires_grad=True)
            params.k = k
            inputs.append(k)
        st = O.State(u, w, wd)
    else:
        st = O.State(u)
    st1, dg = O.step(g, st, dt, scheme=wl.scheme, body=body, kernel=wl.kernel, params=params)
    outs, seeds = list(st1.u), [torch.tensor(np.asarray(a)) for a in lam_u]
    if body is not None:
        outs += [st1.w, st1.wd, dg.F]
        f64 = torch.float64
        seeds += [torch.tensor(lam_body[:2], dtype=f64), torch.tensor(lam_body[2:], dtype=f64),
                  torch.tensor(dJdF, dtype=f64)]
    grads = torch.autograd.grad(outs, inputs, seeds, allow_unused=True)
    gr = [torch.zeros_like(x) if gx is None else gx for gx, x in zip(grads, inputs)]
    out = {"u": gr[:wl.dim]}
    i = wl.dim
    if fx is not None:
        out["fx"] = gr[i]
        i += 1
    if body is not None:
        out["body"] = torch.cat([gr[i], gr[i + 1]])
        i += 2
        if k is not None:
            out["k"] = gr[i]
    return out


def gpu_vjp(wl, u0, lam_u, dt, precision, lam_body=None, dJdF=None, tuning=()):
    from paper_2505_23940_b300 import body_tensor, grid_from_workload
    g = grid_from_workload(wl, precision)
    for key, value in tuning:
        g.set_tuning(key, value)
    u = [torch.tensor(np.asarray(a), dtype=g.dtype, device="cuda").contiguous() for a in u0]
    lam = [torch.tensor(np.asarray(a), dtype=g.dtype, device="cuda").contiguous() for a in lam_u]
    body = body_tensor(wl)
    lb = torch.tensor(lam_body, dtype=torch.float64, device="cuda") if lam_body is not None else None
    gfx = torch.zeros(wl.n[1], dtype=torch.float64, device="cuda") if wl.body_force is not None else None
    gk = torch.zeros(1, dtype=torch.float64, device="cuda") if wl.body is not None else None
    g.step_adjoint(u, lam, dt, body_n=body, lam_body=lb, dJdF=dJdF, g_body_force=gfx, g_stiffness=gk)
    torch.cuda.synchronize()
    out = {"u": [x.double().cpu() for x in lam]}
    if gfx is not None:
        out["fx"] = gfx.cpu()
    if lb is not None:
        out["body"] = lb.cpu()
        out["k"] = gk.cpu()[0]
    return out


def seeds(wl, seed):
    return S.random_fields(wl, seed + 100, 1.0)


def check(o, gp, tol):
    assert rel_l2(gp["u"], o["u"]) < tol, rel_l2(gp["u"], o["u"])
    if "fx" in o:
        assert rel_l2([gp["fx"]], [o["fx"]]) < tol
    if "body" in o:
        assert rel_l2([gp["body"]], [o["body"]]) < max(tol, 1e-10), (gp["body"], o["body"])
        assert abs(float(gp["k"]) - float(o["k"])) <= max(tol, 1e-10) * max(abs(float(o["k"])), 1e-12)


@pytest.mark.parametrize("scheme,conv", [("fe", "central"), ("fe", "upwind"), ("rk3", "central"), ("rk3", "upwind")])
def test_adjoint_periodic_3d_fp64(scheme, conv):
    wl = S.box_3d(12, 10, 8, (P, P), (P, P), L=(1.0, 0.8, 0.6), nu=0.03)
    wl.conv, wl.scheme = conv, scheme
    u0 = S.random_fields(wl, 1, 1.0)
    lam = seeds(wl, 1)
    check(oracle_vjp(wl, u0, lam, 0.004), gpu_vjp(wl, u0, lam, 0.004, "fp64"), 1e-11)


def test_adjoint_channel_body_force_fp64():
    wl = S.box_3d(12, 10, 8, (P, P), (NS, NS), L=(2.0, 2.0, 1.0), stretched=1.5, nu=0.05)
    wl.body_force = np.linspace(0.5, 1.5, 10)
    u0 = S.random_fields(wl, 2, 1.0)
    lam = seeds(wl, 2)
    check(oracle_vjp(wl, u0, lam, 0.002), gpu_vjp(wl, u0, lam, 0.002, "fp64"), 1e-11)


@pytest.mark.parametrize("bcx,bcy,gamma,n", [
    ((IN, OUT), (FS, FS), 0.0, (16, 10)),
    ((NS, NS), (FS, FS), 0.0, (9, 10)),
    ((P, P), (NS, NS), 1.3, (12, 10)),
    ((P, P), (P, P), 0.0, (14, 8)),
])
def test_adjoint_2d_boundaries_fp64(bcx, bcy, gamma, n):
    bc_val = [[[1.0, 0, 0], [0, 0, 0]], [[0.3, 0, 0], [0.0, 0, 0]]]
    wl = S.box_2d(n[0], n[1], bcx, bcy, Lx=1.3, Ly=1.0, stretched=gamma, nu=0.02, bc_val=bc_val)
    u0 = S.random_fields(wl, 3, 1.0)
    lam = seeds(wl, 3)
    check(oracle_vjp(wl, u0, lam, 0.002), gpu_vjp(wl, u0, lam, 0.002, "fp64"), 1e-11)


@pytest.mark.parametrize("kernel", [S.ROMA3, S.PESKIN4])
def test_adjoint_cylinder_fsi_fp64(kernel):
    wl = S.cylinder_2d(nx=48, ny=32, cells_per_d=8, nm=26, dt=0.01, kernel=kernel, centre_d=(2.0, 2.0),
                       precision="fp64", seed=3, perturb=0.05)
    wl.body.w0 = (0.0, 0.05)
    wl.body.wd0 = (0.0, 0.2)
    u0 = S.random_fields(wl, 4, 0.5)
    u0[0] += 1.0
    lam = seeds(wl, 4)
    lb = [0.3, -0.7, 0.2, 0.9]
    dJdF = [0.4, -1.1]
    o = oracle_vjp(wl, u0, lam, wl.dt, lb, dJdF)
    gp = gpu_vjp(wl, u0, lam, wl.dt, "fp64", lb, dJdF)
    check(o, gp, 1e-11)


def test_adjoint_mixed_isotropic_rk3():
    wl = S.isotropic_3d(n=16, steps=1)
    lam = seeds(wl, 5)
    o = oracle_vjp(wl, wl.u0, lam, wl.dt)
    gp = gpu_vjp(wl, wl.u0, lam, wl.dt, "mixed")
    assert rel_l2(gp["u"], o["u"]) < 1e-5


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-11), ("mixed", 1e-5)])
@pytest.mark.parametrize("twisted", [1, 0])
def test_adjoint_fp64_periodic_y_solve(precision, tol, twisted):
    """The adjoint step with the y part of its Poisson solves as the FP64 cyclic tridiagonal
    (y_spectral = 0), twisted (tensor-map tiles in mixed precision) or partitioned, against
    the oracle's reverse-mode AD."""
    wl = S.isotropic_3d(n=32, steps=1)
    lam = seeds(wl, 7)
    o = oracle_vjp(wl, wl.u0, lam, wl.dt)
    gp = gpu_vjp(wl, wl.u0, lam, wl.dt, precision, tuning=[("y_spectral", 0), ("ysolve_twisted", twisted)])
    assert rel_l2(gp["u"], o["u"]) < tol


def test_adjoint_mixed_cylinder():
    wl = S.cylinder_2d(nx=48, ny=32, cells_per_d=8, nm=26, dt=0.01, centre_d=(2.0, 2.0), precision="mixed",
                       seed=3, perturb=0.05)
    u0 = S.random_fields(wl, 6, 0.5)
    u0[0] += 1.0
    lam = seeds(wl, 6)
    lb = [0.1, 0.5, -0.2, 0.3]
    o = oracle_vjp(wl, u0, lam, wl.dt, lb, [0.0, 1.0])
    gp = gpu_vjp(wl, u0, lam, wl.dt, "mixed", lb, [0.0, 1.0])
    assert rel_l2(gp["u"], o["u"]) < 1e-5
    assert rel_l2([gp["body"]], [o["body"]]) < 1e-5


def _coupled_case(active, precision):
    wl = S.cylinder_2d(nx=48, ny=32, cells_per_d=8, nm=26, dt=0.01, centre_d=(2.0, 2.0), precision=precision,
                       seed=3, perturb=0.05, mass_ratio=1.0)
    wl.body.w0 = (0.02, 0.05)
    wl.body.wd0 = (0.1 if active[0] else 0.0, -0.2)
    wl.body.active = active
    return wl


@pytest.mark.parametrize("active", [(False, True), (True, True)])
def test_adjoint_strong_coupling_fp64(active):
    """Adjoint of the strongly coupled step (Algorithm 1 differentiated implicitly at its fixed point,
    §2.4.1) against the oracle's implicit differentiation: lam of u^n, of the body state and dJ/dk, both
    sides converging the sub-iteration to rounding (xi < 1e-28).  dJdF is passed in device memory."""
    from oracle.step import step_coupled_adjoint
    from paper_2505_23940_b300 import body_tensor, grid_from_workload
    wl = _coupled_case(active, "fp64")
    g = grid_of(wl)
    body, params = body_of(wl)
    f64 = torch.float64
    st = O.State([torch.tensor(a, dtype=f64) for a in wl.u0], torch.tensor(wl.body.w0, dtype=f64),
                 torch.tensor(wl.body.wd0, dtype=f64))
    lam_u = seeds(wl, 9)
    lb, fb = [0.3, -0.7, 0.2, 0.9], [0.4, -1.1]
    lu, ls, dk, iters = step_coupled_adjoint(g, st, wl.dt, body, wl.kernel, params, lam_u, lb, fb,
                                             max_iter=200, tol=1e-28)
    G = grid_from_workload(wl, "fp64")
    G.set_coupling(200, 1e-28)
    u = [torch.tensor(a, dtype=f64, device="cuda") for a in wl.u0]
    lam = [torch.tensor(a, dtype=f64, device="cuda") for a in lam_u]
    bt = body_tensor(wl)
    lbt = torch.tensor(lb, dtype=f64, device="cuda")
    gk = torch.zeros(1, dtype=f64, device="cuda")
    G.step_adjoint(u, lam, wl.dt, body_n=bt, lam_body=lbt, dJdF=torch.tensor(fb, dtype=f64, device="cuda"),
                   g_stiffness=gk)
    torch.cuda.synchronize()
    eu = rel_l2([x.cpu() for x in lam], lu)
    eb = float((lbt.cpu() - ls).norm() / ls.norm())
    ek = abs(float(gk[0]) - float(dk)) / abs(float(dk))
    print("strong coupling adjoint %s: %d sub-iterations, lam_u %.2e, lam_body %.2e, dJ/dk %.2e"
          % (active, iters, eu, eb, ek))
    assert eu < 1e-9 and eb < 1e-9 and ek < 1e-9
    assert torch.equal(u[0].cpu(), torch.tensor(wl.u0[0], dtype=f64))   # st_n is not modified


def test_adjoint_strong_coupling_mixed():
    """The same in mixed precision (FP32 fluid, FP64 body and coupling system) against the FP64 oracle;
    the FP32 force limits how far the sub-iteration converges (xi < 1e-12 here)."""
    from oracle.step import step_coupled_adjoint
    from paper_2505_23940_b300 import body_tensor, grid_from_workload
    wl = _coupled_case((True, True), "mixed")
    g = grid_of(wl)
    body, params = body_of(wl)
    f64 = torch.float64
    st = O.State([torch.tensor(a, dtype=f64) for a in wl.u0], torch.tensor(wl.body.w0, dtype=f64),
                 torch.tensor(wl.body.wd0, dtype=f64))
    lam_u = seeds(wl, 9)
    lb, fb = [0.3, -0.7, 0.2, 0.9], [0.4, -1.1]
    lu, ls, dk, _ = step_coupled_adjoint(g, st, wl.dt, body, wl.kernel, params, lam_u, lb, fb,
                                         max_iter=200, tol=1e-28)
    G = grid_from_workload(wl, "mixed")
    G.set_coupling(100, 1e-12)
    u = [torch.tensor(a, dtype=torch.float32, device="cuda") for a in wl.u0]
    lam = [torch.tensor(a, dtype=torch.float32, device="cuda") for a in lam_u]
    bt = body_tensor(wl)
    lbt = torch.tensor(lb, dtype=f64, device="cuda")
    gk = torch.zeros(1, dtype=f64, device="cuda")
    G.step_adjoint(u, lam, wl.dt, body_n=bt, lam_body=lbt, dJdF=fb, g_stiffness=gk)
    torch.cuda.synchronize()
    eu = rel_l2([x.double().cpu() for x in lam], lu)
    eb = float((lbt.cpu() - ls).norm() / ls.norm())
    ek = abs(float(gk[0]) - float(dk)) / abs(float(dk))
    print("strong coupling adjoint, mixed: lam_u %.2e, lam_body %.2e, dJ/dk %.2e" % (eu, eb, ek))
    assert eu < 1e-5 and eb < 1e-4 and ek < 1e-4


def test_adjoint_device_and_host_force_sensitivity_agree():
    """fs_step_adjoint_dev (dJ/dF in device memory) gives fs_step_adjoint's result (up to the order of
    the adjoint's atomic FP64 sums)."""
    from paper_2505_23940_b300 import body_tensor, grid_from_workload
    wl = S.cylinder_2d(nx=48, ny=32, cells_per_d=8, nm=26, dt=0.01, centre_d=(2.0, 2.0), precision="fp64",
                       seed=3, perturb=0.05)
    wl.body.w0 = (0.0, 0.05)
    G = grid_from_workload(wl, "fp64")
    u = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in wl.u0]
    out = []
    for dev in (False, True):
        lam = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in seeds(wl, 11)]
        lbt = torch.tensor([0.3, -0.7, 0.2, 0.9], dtype=torch.float64, device="cuda")
        fb = [0.4, -1.1]
        G.step_adjoint(u, lam, wl.dt, body_n=body_tensor(wl), lam_body=lbt,
                       dJdF=torch.tensor(fb, dtype=torch.float64, device="cuda") if dev else fb)
        torch.cuda.synchronize()
        out.append([x.cpu() for x in lam] + [lbt.cpu()])
    for a, b in zip(*out):
        assert float((a - b).norm()) <= 1e-13 * float(b.norm())
