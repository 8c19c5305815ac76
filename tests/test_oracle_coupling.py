"""Pins of the oracle's strongly coupled FSI step (§2.3.3, Algorithm 1): one sub-iteration is
the weakly coupled step, and a converged iterate is a fixed point of the coupled fluid-structure
map (one more sub-iteration changes it by less than the tolerance)."""
import pytest
import torch

import oracle as O
import synthetic as S
from helpers import body_of, grid_of


def _cyl(mass_ratio=2.0, w0=(0.0, 0.05), active=(False, True)):
    wl = S.cylinder_2d(nx=48, ny=32, cells_per_d=8, nm=26, dt=0.01, centre_d=(2.0, 2.0), precision="fp64",
                       seed=3, perturb=0.05, mass_ratio=mass_ratio)
    wl.body.w0 = w0
    wl.body.active = active
    return wl


def _state(wl):
    u = [torch.tensor(a, dtype=torch.float64) for a in wl.u0]
    return O.State(u, torch.tensor(wl.body.w0, dtype=torch.float64), torch.tensor(wl.body.wd0, dtype=torch.float64))


def test_one_subiteration_is_the_weak_step():
    from oracle.step import step_coupled
    wl = _cyl()
    g = grid_of(wl)
    body, params = body_of(wl)
    st = _state(wl)
    weak, _ = O.step(g, st, wl.dt, body=body, kernel=wl.kernel, params=params)
    strong, _, k, _ = step_coupled(g, st, wl.dt, body, wl.kernel, params, max_iter=1)
    assert k == 1
    for a, b in zip(weak.u, strong.u):
        assert torch.equal(a, b)
    assert torch.equal(weak.w, strong.w) and torch.equal(weak.wd, strong.wd)


def test_converged_iterate_is_a_fixed_point():
    from oracle.step import step_coupled
    for active in [(False, True), (True, True)]:
        wl = _cyl(mass_ratio=1.0, w0=(0.02, 0.05), active=active)
        g = grid_of(wl)
        body, params = body_of(wl)
        st = _state(wl)
        tol = 1e-12
        new, dg, k, xi = step_coupled(g, st, wl.dt, body, wl.kernel, params, max_iter=50, tol=tol)
        assert xi < tol and 1 < k < 50
        # one more fluid solve with the converged kinematics, structure from level n again
        nxt, dg2 = O.step(g, O.State(st.u, new.w, new.wd), wl.dt, body=body, kernel=wl.kernel, params=None)
        w2, wd2 = O.body.rk4(params, st.w, st.wd, dg2.F, wl.dt)
        assert float(((w2 - new.w) ** 2).sum()) <= tol * float((new.w ** 2).sum())
        # the coupled answer differs from the weak one (the sub-iteration did something)
        weak, _ = O.step(g, st, wl.dt, body=body, kernel=wl.kernel, params=params)
        assert float((weak.w - new.w).abs().max()) > 0.0


def _loss(new, dg, lam_u, lb, fb):
    f64 = torch.float64
    return (sum((a * torch.as_tensor(b, dtype=f64)).sum() for a, b in zip(new.u, lam_u))
            + (new.w * torch.tensor(lb[:2], dtype=f64)).sum() + (new.wd * torch.tensor(lb[2:], dtype=f64)).sum()
            + (dg.F * torch.tensor(fb, dtype=f64)).sum())


def _adjoint_case(active):
    import numpy as np
    wl = _cyl(mass_ratio=1.0, w0=(0.02, 0.05), active=active)
    wl.body.wd0 = (0.1, -0.2) if active[0] else (0.0, -0.2)
    g = grid_of(wl)
    body, params = body_of(wl)
    st = _state(wl)
    rng = np.random.default_rng(5)
    lam_u = [rng.uniform(-1, 1, size=g.shape(c)) for c in range(2)]
    return wl, g, body, params, st, lam_u, [0.3, -0.7, 0.2, 0.9], [0.4, -1.1], rng


@pytest.mark.parametrize("active", [(False, True), (True, True)])
def test_coupled_adjoint_against_central_differences(active):
    """Implicit differentiation of the converged sub-iteration (§2.4.1) against central finite
    differences of the coupled step converged to rounding (xi < 1e-30): the spring stiffness k and a
    random joint direction in (u^n, w^n, wdot^n).  Best agreement over steps 1e-3 .. 1e-5 within 1e-7."""
    import numpy as np
    from oracle.step import step_coupled, step_coupled_adjoint
    from oracle import body as body_mod
    wl, g, body, params, st, lam_u, lb, fb, rng = _adjoint_case(active)
    lu, ls, dk, iters = step_coupled_adjoint(g, st, wl.dt, body, wl.kernel, params, lam_u, lb, fb,
                                             max_iter=200, tol=1e-30)
    assert 5 < iters < 200
    du = [torch.tensor(rng.uniform(-1, 1, size=g.shape(c))) for c in range(2)]
    ds = torch.tensor(rng.uniform(-0.1, 0.1, size=4), dtype=torch.float64)
    if not active[0]:
        ds[0] = ds[2] = 0.0
    k0 = float(params.k)

    def L(kv, e):
        p = body_mod.RigidParams(params.m, kv, params.c, params.active)
        s = O.State([a + e * b for a, b in zip(st.u, du)], st.w + e * ds[:2], st.wd + e * ds[2:])
        new, dg, _, _ = step_coupled(g, s, wl.dt, body, wl.kernel, p, max_iter=200, tol=1e-30)
        return float(_loss(new, dg, lam_u, lb, fb))

    ad_dir = sum(float((a * b).sum()) for a, b in zip(lu, du)) + float((ls * ds).sum())
    best_dir = min(abs((L(k0, e) - L(k0, -e)) / (2 * e) - ad_dir) / abs(ad_dir) for e in (1e-3, 1e-4, 1e-5))
    best_k = min(abs((L(k0 + e, 0.0) - L(k0 - e, 0.0)) / (2 * e) - float(dk)) / abs(float(dk))
                 for e in (1e-3, 1e-4, 1e-5))
    assert best_dir < 1e-7, best_dir
    assert best_k < 1e-7, best_k


def test_coupled_adjoint_matches_unrolled_reverse_mode():
    """The same gradients by reverse-mode AD through 40 unrolled sub-iterations (no implicit
    function theorem); the unrolled derivative of this contraction settles to within 1e-6."""
    from oracle.step import step_coupled, step_coupled_adjoint
    from oracle import body as body_mod
    wl, g, body, params, st, lam_u, lb, fb, _ = _adjoint_case((True, True))
    lu, ls, dk, _ = step_coupled_adjoint(g, st, wl.dt, body, wl.kernel, params, lam_u, lb, fb,
                                         max_iter=200, tol=1e-30)
    uu = [x.clone().requires_grad_(True) for x in st.u]
    w, wd = st.w.clone().requires_grad_(True), st.wd.clone().requires_grad_(True)
    k = torch.tensor(float(params.k), dtype=torch.float64, requires_grad=True)
    p = body_mod.RigidParams(params.m, k, params.c, params.active)
    new, dg, _, _ = step_coupled(g, O.State(uu, w, wd), wl.dt, body, wl.kernel, p, max_iter=40, tol=0.0)
    gr = torch.autograd.grad(_loss(new, dg, lam_u, lb, fb), uu + [w, wd, k])
    num = sum(float(((a - b) ** 2).sum()) for a, b in zip(gr[:2], lu))
    assert (num / sum(float((b ** 2).sum()) for b in lu)) ** 0.5 < 1e-10
    assert float((torch.cat([gr[2], gr[3]]) - ls).norm() / ls.norm()) < 1e-6
    assert abs(float(gr[4]) - float(dk)) < 1e-6 * abs(float(dk))
