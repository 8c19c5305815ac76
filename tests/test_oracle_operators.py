"""Pins of the oracle's FV operators (§2.3.1): exactness on polynomials, conservation, energy."""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import fluid, poisson
from helpers import grid_of

P, NS, FS, IN, OUT = S.PERIODIC, S.NOSLIP, S.FREESLIP, S.INFLOW, S.OUTFLOW


def test_gradient_exact_on_linear_pressure_stretched():
    """G of p = a + b x + c y is exactly (b, c) on interior faces of a stretched wall-bounded grid."""
    wl = S.box_2d(10, 9, (FS, FS), (NS, NS), Lx=1.7, Ly=2.0, stretched=1.4)
    g = grid_of(wl)
    X = g.along(0, g.xc[0])
    Y = g.along(1, g.xc[1])
    p = (0.3 + 1.25 * X - 0.75 * Y).expand(g.cshape())
    G = fluid.gradient(g, p)
    gu = G[0][..., 1:-1]
    gv = G[1][:, 1:-1, :]
    assert torch.allclose(gu, torch.full_like(gu, 1.25), rtol=0, atol=1e-12)
    assert torch.allclose(gv, torch.full_like(gv, -0.75), rtol=0, atol=1e-12)
    assert float(G[0][..., 0].abs().max()) == 0.0 and float(G[1][:, -1, :].abs().max()) == 0.0


def test_divergence_exact_on_linear_field_stretched():
    """D of u = 2x, v = -3y is exactly -1 in every cell (stretched y)."""
    wl = S.box_2d(7, 9, (FS, FS), (NS, NS), Lx=1.0, Ly=2.0, stretched=1.1)
    g = grid_of(wl)
    fx, _, _ = g.face_coords(0)
    _, fy, _ = g.face_coords(1)
    u = [(2.0 * fx).expand(g.shape(0)).clone(), (-3.0 * fy).expand(g.shape(1)).clone()]
    D = fluid.divergence(g, u)
    assert torch.allclose(D, torch.full_like(D, -1.0), rtol=0, atol=1e-12)


@pytest.mark.parametrize("conv", ["central", "upwind"])
@pytest.mark.parametrize("dim", [2, 3])
def test_momentum_conservation_periodic(conv, dim):
    """Divergence form conserves momentum: sum_faces R_c * dV_c = 0 on a periodic (stretch-free) grid."""
    if dim == 2:
        wl = S.box_2d(12, 10, (P, P), (P, P), Lx=1.3, Ly=0.7, nu=0.05)
    else:
        wl = S.box_3d(8, 6, 10, (P, P), (P, P), L=(1.0, 0.8, 1.2), nu=0.05)
    wl.conv = conv
    g = grid_of(wl)
    rng = np.random.default_rng(5)
    u = [torch.tensor(rng.uniform(-1, 1, size=g.shape(c))) for c in range(dim)]
    R = fluid.momentum_rhs(g, u)
    for c in range(dim):
        total = float((R[c] * g.face_volume(c)).sum())
        scale = float((R[c].abs() * g.face_volume(c)).sum())
        assert abs(total) < 1e-13 * scale


@pytest.mark.parametrize("dim", [2, 3])
def test_central_convection_conserves_energy(dim):
    """With D u = 0 and nu = 0, sum_c sum_f u_c R_c dV_c = 0 (energy conservation of the
    divergence-form central MAC scheme on uniform periodic grids, Morinishi et al. 1998)."""
    if dim == 2:
        wl = S.box_2d(16, 12, (P, P), (P, P), Lx=1.0, Ly=0.75, nu=0.0)
    else:
        wl = S.box_3d(8, 8, 8, (P, P), (P, P), nu=0.0)
    g = grid_of(wl)
    rng = np.random.default_rng(7)
    u = [torch.tensor(rng.uniform(-1, 1, size=g.shape(c))) for c in range(dim)]
    u, _ = poisson.project(g, u)
    R = fluid.momentum_rhs(g, u)
    e = sum(float((u[c] * R[c] * g.face_volume(c)).sum()) for c in range(dim))
    scale = sum(float((u[c].abs() * R[c].abs() * g.face_volume(c)).sum()) for c in range(dim))
    assert abs(e) < 1e-13 * scale


def test_diffusion_exact_on_quadratic_uniform():
    """nu lap(u) of u = y^2 (x-periodic, y-periodic-free interior rows) is exactly 2 nu in the interior."""
    wl = S.box_2d(6, 10, (P, P), (FS, FS), Lx=1.0, Ly=1.0, nu=0.3)
    g = grid_of(wl)
    _, fy, _ = g.face_coords(0)
    u = [(fy * fy).expand(g.shape(0)).clone(), torch.zeros(g.shape(1), dtype=torch.float64)]
    R = fluid.momentum_rhs(g, u)
    # u-momentum: convection vanishes (v = 0 and u independent of x); interior rows only
    inner = R[0][:, 1:-1, :]
    assert torch.allclose(inner, torch.full_like(inner, 0.6), rtol=0, atol=1e-11)


def test_noslip_ghost_reflection():
    """Wall-adjacent diffusion uses ghost = -u: for a constant u the wall row sees nu * (-2u / h^2)... divided per metric."""
    wl = S.box_2d(4, 8, (P, P), (NS, NS), Lx=1.0, Ly=1.0, nu=1.0)
    g = grid_of(wl)
    u = [torch.ones(g.shape(0), dtype=torch.float64), torch.zeros(g.shape(1), dtype=torch.float64)]
    R = fluid.momentum_rhs(g, u)
    h = 1.0 / 8
    # bottom row: ((u1 - u0)/h - (u0 - (-u0))/h) / h = -2/h^2
    assert torch.allclose(R[0][:, 0, :], torch.full_like(R[0][:, 0, :], -2.0 / h ** 2), atol=1e-9)
    assert torch.allclose(R[0][:, 3, :], torch.zeros_like(R[0][:, 3, :]), atol=1e-9)


def test_inflow_outflow_flux_balance():
    """After the outflow correction the net boundary flux is zero, so D u sums to zero."""
    wl = S.box_2d(12, 8, (IN, OUT), (FS, FS), bc_val=[[[1.0, 0, 0], [0, 0, 0]], [[0] * 3, [0] * 3]])
    g = grid_of(wl)
    rng = np.random.default_rng(9)
    u = [torch.tensor(rng.uniform(0.5, 1.5, size=g.shape(c))) for c in range(2)]
    u = fluid.apply_boundary_values(g, u)
    assert float(u[0][..., 0].min()) == 1.0 and float(u[1][:, 0, :].abs().max()) == 0.0
    un = fluid.outflow_faces(g, u, u)
    D = fluid.divergence(g, un)
    assert abs(float((D * g.cell_volume()).sum())) < 1e-13
