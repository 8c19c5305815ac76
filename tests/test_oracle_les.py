"""Pins of the oracle's Smagorinsky subgrid term (les.py): the discrete energy identity
sum u . d_j tau_ij dv = -sum tau_ij S_ij dV <= 0, zero stress for a uniform translation, a
shear that varies in y only acts on u only, and C_s = 0 reproduces the plain step."""
import numpy as np
import torch

import oracle as O
import synthetic as S
from oracle import les
from helpers import grid_of

P = S.PERIODIC


def _box(n=(12, 10, 8), L=(1.0, 0.8, 0.6)):
    wl = S.box_3d(*n, (P, P), (P, P), L=L, nu=0.01)
    return wl, grid_of(wl)


def test_subgrid_term_removes_energy_exactly_as_tau_S():
    wl, g = _box()
    u = [torch.tensor(a) for a in S.random_fields(wl, 5, 1.0)]
    cs = 0.17
    R = les.sgs_term(g, u, cs)
    dv = float(g.h[0][0] * g.h[1][0] * g.h[2][0])
    power = sum(float((a * b).sum()) for a, b in zip(u, R)) * dv
    nt = les.nu_t(g, u, cs)
    Sxx, Syy, Szz, Sxy, Sxz, Syz = les.strain(g, u)
    diss = float((2 * nt * (Sxx ** 2 + Syy ** 2 + Szz ** 2)).sum())
    for e, a1, a2 in ((Sxy, 2, 1), (Sxz, 2, 0), (Syz, 1, 0)):
        ne = les._centre_to_edge(nt, a1, a2)
        diss += float((4.0 * ne * e * e).sum())
    diss *= dv
    assert power < 0.0
    assert abs(power + diss) <= 1e-12 * diss


def test_uniform_translation_has_no_subgrid_stress():
    wl, g = _box()
    u = [torch.full(g.shape(c), 0.3 + c, dtype=torch.float64) for c in range(3)]
    assert float(les.nu_t(g, u, 0.2).abs().max()) == 0.0
    assert all(float(r.abs().max()) == 0.0 for r in les.sgs_term(g, u, 0.2))


def test_shear_in_y_acts_on_u_only_and_nu_t_matches_closed_form():
    wl, g = _box(n=(8, 64, 8), L=(1.0, 1.0, 1.0))
    yc = torch.tensor(0.5 * (wl.xf[1][:-1] + wl.xf[1][1:]))
    U = torch.sin(2 * np.pi * yc).reshape(1, -1, 1).expand(g.shape(0)).clone()
    u = [U, torch.zeros(g.shape(1), dtype=torch.float64), torch.zeros(g.shape(2), dtype=torch.float64)]
    R = les.sgs_term(g, u, 0.1)
    assert float(R[1].abs().max()) == 0.0 and float(R[2].abs().max()) == 0.0
    # nu_t = (C_s Delta)^2 |du/dy| at the centres, to second order in h
    delta = (1.0 / 8 * 1.0 / 64 * 1.0 / 8) ** (1.0 / 3.0)
    exact = (0.1 * delta) ** 2 * 2 * np.pi * torch.abs(torch.cos(2 * np.pi * yc))
    got = les.nu_t(g, u, 0.1)[0, :, 0]
    assert float((got - exact).abs().max()) < 0.01 * float(exact.max())


def test_zero_constant_is_the_plain_step():
    wl, g = _box()
    st = O.State([torch.tensor(a) for a in S.random_fields(wl, 6, 1.0)])
    a, _ = O.step(g, st, 0.002)
    b, _ = O.step(g, st, 0.002, cs=0.0)
    assert all(torch.equal(x, y) for x, y in zip(a.u, b.u))
