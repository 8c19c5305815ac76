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


def _stretched_box(nu=0.0):
    """x periodic and uniform, y wall-bounded and tanh-stretched (the channel's geometry, §3.4.1)."""
    wl = S.box_2d(8, 12, (P, P), (NS, NS), Lx=1.0, Ly=2.0, stretched=1.6, nu=nu)
    return grid_of(wl), wl


def test_convection_exact_linear_interpolation_of_transported_u_on_stretched_y():
    """u = a + b y (stored at the u faces, i.e. at the cell-centre heights yc_j) carried by a uniform
    v = V: the y flux at the cell edge y = yf_j is V (a + b yf_j) when u is interpolated linearly in y
    between yc_{j-1} and yc_j, so on every row away from the walls R_u = -(V (a + b yf_{j+1}) -
    V (a + b yf_j)) / (yf_{j+1} - yf_j) = -V b exactly (§2.3.1, stretched-grid interpolation).  Equal
    weights 1/2 instead of the metric weights give -V b (yc_{j+1} - yc_{j-1}) / (2 h_j) there."""
    g, wl = _stretched_box()
    a, b, V = 0.4, 1.7, -0.6
    yc = 0.5 * (wl.xf[1][:-1] + wl.xf[1][1:])
    h = np.diff(wl.xf[1])
    assert np.ptp(h) > 0.2 * h.max()          # the grid is strongly stretched
    u = torch.tensor(np.broadcast_to((a + b * yc)[None, :, None], g.shape(0)).copy())
    v = torch.full(g.shape(1), V, dtype=torch.float64)
    R = fluid.momentum_rhs(g, [u, v])
    inner = R[0][:, 1:-1, :]
    assert float((inner + V * b).abs().max()) < 1e-12
    # the equal-weight value differs by far more than that on this grid
    half = -V * b * (yc[2:] - yc[:-2]) / (2 * h[1:-1])
    assert np.abs(half + V * b).max() > 1e-2


def test_convection_exact_linear_interpolation_of_transport_velocity_on_stretched_y():
    """v = W uniform carried by u = sin(k x) (a + b y): the x flux of v momentum at the edge (x_i, yf_j)
    is u interpolated linearly in y to the v face times W, u(x_i, yf_j) = sin(k x_i) (a + b yf_j), so
    R_v = -W (sin(k x_{i+1}) - sin(k x_i)) (a + b yf_j) / h_x on every interior v face; the y flux
    cancels (v uniform).  Hand value from the face coordinates alone."""
    g, wl = _stretched_box()
    a, b, W, k = 0.3, -1.1, 0.8, 2 * np.pi
    xf = wl.xf[0]
    yc = 0.5 * (wl.xf[1][:-1] + wl.xf[1][1:])
    hx = xf[1] - xf[0]
    xu = xf[:-1]                                   # u faces (periodic x: n faces)
    u = torch.tensor(np.broadcast_to((np.sin(k * xu)[None, :] * (a + b * yc)[:, None])[None], g.shape(0)).copy())
    v = torch.full(g.shape(1), W, dtype=torch.float64)
    R = fluid.momentum_rhs(g, [u, v])
    yfj = wl.xf[1][1:-1]                           # interior v faces j = 1 .. ny-1
    sx = (np.sin(k * np.roll(xu, -1)) - np.sin(k * xu)) / hx
    sx[-1] = (np.sin(k * (xu[0] + 1.0)) - np.sin(k * xu[-1])) / hx   # periodic wrap
    expect = -W * sx[None, :] * (a + b * yfj)[:, None]
    got = R[1][0, 1:-1, :].numpy()
    assert np.abs(got - expect).max() < 1e-12 * np.abs(expect).max()


def _upwind_periodic(nx=16):
    wl = S.box_2d(nx, 4, (P, P), (P, P), Lx=1.0, Ly=0.25, nu=0.0)
    wl.conv = "upwind"
    return grid_of(wl), 1.0 / nx


@pytest.mark.parametrize("U", [0.7, -0.7])
def test_upwind_takes_the_upstream_value_cross_direction(U):
    """v = step in x (1 on faces i < 8, 0 from i = 8) carried by a uniform u = U: first-order upwind
    flux through the edge between v faces i and i+1 is U times the upstream v, so R_v is nonzero only on
    the face just downstream of each jump: U > 0: R_v[8] = U / h (the 1 -> 0 jump) and R_v[0] = -U / h
    (the 0 -> 1 jump at the periodic wrap); U < 0: the faces i = 7 and 15 instead (§2.3.1, Table 1)."""
    g, h = _upwind_periodic()
    u = torch.full(g.shape(0), U, dtype=torch.float64)
    step = (torch.arange(16) < 8).double()
    v = step.reshape(1, 1, -1).expand(g.shape(1)).clone()
    R = fluid.momentum_rhs(g, [u, v])[1][0, 0, :]
    expect = torch.zeros(16, dtype=torch.float64)
    if U > 0:
        expect[8], expect[0] = U / h, -U / h
    else:
        expect[7], expect[15] = U / h, -U / h
    assert float((R - expect).abs().max()) < 1e-12


def test_upwind_takes_the_upstream_value_own_direction():
    """u = 1 on faces i < 8 and 1.5 from i = 8 (all positive, so every cell-centre transport velocity
    T = (u_i + u_{i+1}) / 2 > 0 and the upstream u is the west face of the cell): by hand
    R_u[7] = -(1.25 * 1 - 1 * 1) / h = -0.25 / h, R_u[8] = -(1.5 * 1.5 - 1.25 * 1) / h = -1 / h,
    R_u[9] = 0 (the downstream values would give -0.875 / h, -0.5 / h, 0)."""
    g, h = _upwind_periodic()
    uu = torch.where(torch.arange(16) < 8, 1.0, 1.5).double()
    u = uu.reshape(1, 1, -1).expand(g.shape(0)).clone()
    v = torch.zeros(g.shape(1), dtype=torch.float64)
    R = fluid.momentum_rhs(g, [u, v])[0][0, 0, :]
    assert abs(float(R[7]) + 0.25 / h) < 1e-12
    assert abs(float(R[8]) + 1.0 / h) < 1e-12
    assert abs(float(R[9])) < 1e-12
