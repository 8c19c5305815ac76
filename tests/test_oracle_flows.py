"""Pins of the oracle's whole step (Eqs. 4-10) against closed forms and independent solves."""
import math

import numpy as np
import pytest
import torch
from scipy.linalg import solve_banded

import oracle as O
import synthetic as S
from oracle import fluid
from helpers import grid_of, state_of, rel_l2


def _tg_error(n, steps, dt, scheme):
    wl = S.taylor_green_2d(n=n, nu=0.01)
    g = grid_of(wl)
    st = state_of(wl)
    for _ in range(steps):
        st, _ = O.step(g, st, dt, scheme=scheme)
    ex = [torch.tensor(a) for a in S.taylor_green_exact(n, 0.01, steps * dt)]
    return rel_l2(st.u, ex), st, g


def test_taylor_green_second_order_in_space():
    """Closed-form decay u = sin x cos y e^{-2 nu t}: spatial error ratio ~4 per halving of h."""
    e16, _, _ = _tg_error(16, 50, 0.004, "rk3")
    e32, _, _ = _tg_error(32, 50, 0.004, "rk3")
    assert 3.6 < e16 / e32 < 4.4
    assert e32 < 2e-4


def test_taylor_green_forward_euler_workload():
    """The 64^2, CFL 0.5, 100-step forward-Euler case: within 5e-3 of closed form, divergence-free."""
    wl = S.taylor_green_2d(64, 0.01)
    err, st, g = _tg_error(64, 100, wl.dt, "fe")
    assert err < 5e-3
    assert float(fluid.divergence(g, st.u).abs().max()) < 1e-10


def _poiseuille_discrete(yf, nu, fx):
    """Steady 1-D FV diffusion nu u'' = -fx with ghost reflection u_ghost = -u (no-slip), solved banded."""
    yc = 0.5 * (yf[:-1] + yf[1:])
    h = np.diff(yf)
    n = yc.size
    ab = np.zeros((3, n))
    rhs = np.full(n, -fx / nu)
    for j in range(n):
        dn = (yc[j] - yc[j - 1]) if j > 0 else 2 * (yc[0] - yf[0])
        up = (yc[j + 1] - yc[j]) if j < n - 1 else 2 * (yf[-1] - yc[-1])
        lo_c, up_c = 1.0 / (dn * h[j]), 1.0 / (up * h[j])
        diag = -lo_c - up_c
        if j == 0:
            diag -= lo_c          # ghost = -u_0
        else:
            ab[2, j - 1] = lo_c
        if j == n - 1:
            diag -= up_c
        else:
            ab[0, j + 1] = up_c
        ab[1, j] = diag
    return solve_banded((1, 1), ab, rhs), yc


@pytest.mark.parametrize("gamma", [0.0, 1.3])
def test_poiseuille_steady_state(gamma):
    """Marched to steady state the step reproduces the discrete 1-D profile to 1e-10 and the
    parabola (fx / 2 nu)(1 - y^2) to O(h^2)."""
    wl = S.poiseuille_2d(nx=4, ny=16, nu=1.0, fx=1.0, stretched=gamma, steps=0)
    g = grid_of(wl)
    st = state_of(wl)
    ud, yc = _poiseuille_discrete(wl.xf[1], 1.0, 1.0)
    for it in range(40000):
        st, _ = O.step(g, st, wl.dt)
        if it % 500 == 0:
            if float((st.u[0][0, :, 0] - torch.tensor(ud)).abs().max()) < 1e-11:
                break
    prof = st.u[0][0, :, :]
    assert float((prof - torch.tensor(ud).reshape(-1, 1)).abs().max()) < 1e-10
    assert float(st.u[1].abs().max()) < 1e-12
    par = 0.5 * (1 - yc ** 2)
    err = np.abs(ud - par).max()
    assert err < 0.02


def test_poiseuille_second_order_vs_parabola():
    errs = []
    for ny in (16, 32, 64):
        yf = S.uniform_faces(ny, 2.0, -1.0)
        ud, yc = _poiseuille_discrete(yf, 1.0, 1.0)
        errs.append(np.abs(ud - 0.5 * (1 - yc ** 2)).max())
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5


def test_periodic_step_conserves_momentum():
    wl = S.box_3d(8, 8, 8, (S.PERIODIC,) * 2, (S.PERIODIC,) * 2, nu=0.02)
    g = grid_of(wl)
    rng = np.random.default_rng(11)
    st = O.State([torch.tensor(rng.uniform(-1, 1, size=g.shape(c))) for c in range(3)])
    m0 = [float((st.u[c] * g.face_volume(c)).sum()) for c in range(3)]
    for _ in range(3):
        st, _ = O.step(g, st, 0.01)
    m1 = [float((st.u[c] * g.face_volume(c)).sum()) for c in range(3)]
    assert max(abs(a - b) for a, b in zip(m0, m1)) < 1e-13


def _rk3_order_ratios():
    """Time-step refinement of SSP-RK3 on one 16^2 periodic grid (so the spatial error is the same in
    every run and cancels): a random projected field with u ~ 1, nu = 0.02, T = 0.8 with dt = T/8,
    T/16, T/32, each compared with dt = T/256 on the same grid.  Returns the two error ratios."""
    from oracle import poisson
    wl = S.box_2d(16, 16, (S.PERIODIC,) * 2, (S.PERIODIC,) * 2, Lx=2 * math.pi, Ly=2 * math.pi, nu=0.02)
    g = grid_of(wl)
    rng = np.random.default_rng(3)
    u0 = [torch.tensor(rng.uniform(-1, 1, size=g.shape(c))) for c in range(2)]
    u0, _ = poisson.project(g, u0)
    T = 0.8

    def run(n):
        st = O.State([x.clone() for x in u0])
        for _ in range(n):
            st, _ = O.step(g, st, T / n, scheme="rk3")
        return st.u

    ref = run(256)
    es = [rel_l2(run(n), ref) for n in (8, 16, 32)]
    return es[0] / es[1], es[1] / es[2]


def test_ssp_rk3_is_third_order_in_time():
    """The explicit Runge-Kutta scheme (§2.5; read as Shu-Osher SSP-RK3 with a projection per stage)
    converges at third order in dt: error ratios ~8 per halving of dt."""
    r1, r2 = _rk3_order_ratios()
    assert 7.0 < r1 < 9.5 and 7.0 < r2 < 9.5, (r1, r2)


def test_rk3_order_check_rejects_a_wrong_tableau(monkeypatch):
    """The order check is sensitive to the stage weights: with the second stage's weights swapped
    (1/4, 3/4) the scheme drops to about second order and the ratios fall near 2-4."""
    import sys
    mod = sys.modules["oracle.step"]
    monkeypatch.setattr(mod, "SSPRK3", ((0.0, 1.0), (0.25, 0.75), (1.0 / 3.0, 2.0 / 3.0)))
    r1, r2 = _rk3_order_ratios()
    assert r1 < 5.0 and r2 < 5.0, (r1, r2)
