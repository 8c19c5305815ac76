"""Pins of the oracle's strongly coupled FSI step (§2.3.3, Algorithm 1): one sub-iteration is
the weakly coupled step, and a converged iterate is a fixed point of the coupled fluid-structure
map (one more sub-iteration changes it by less than the tolerance)."""
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
