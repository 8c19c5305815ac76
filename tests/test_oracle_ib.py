"""Pins of the oracle's immersed boundary (§2.3.3): kernel moments, interpolation, classification."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S
from oracle import ib
from helpers import grid_of, state_of, body_of

RNG = np.random.default_rng(0)
R = torch.tensor(RNG.uniform(0.0, 1.0, size=1000), dtype=torch.float64)
J = torch.arange(-4, 5, dtype=torch.float64).reshape(-1, 1)


@pytest.mark.parametrize("phi,second", [(ib.phi_peskin4, 3.0 / 8.0), (ib.phi_roma3, 0.5)])
def test_kernel_moments(phi, second):
    """sum_j phi(r - j) = 1, sum_j (r - j) phi(r - j) = 0, sum_j phi(r - j)^2 = const."""
    w = phi(R.reshape(1, -1) - J)
    assert float((w.sum(0) - 1).abs().max()) < 1e-14
    assert float(((R.reshape(1, -1) - J) * w).sum(0).abs().max()) < 1e-14
    assert float(((w * w).sum(0) - second).abs().max()) < 1e-14


def test_peskin_even_odd_split():
    w = ib.phi_peskin4(R.reshape(1, -1) - J)
    even = w[(J.reshape(-1).long() % 2) == 0].sum(0)
    assert float((even - 0.5).abs().max()) < 1e-14


@pytest.mark.parametrize("phi,knots", [(ib.phi_peskin4, (0.0, 1.0, 2.0)), (ib.phi_roma3, (0.5, 1.5))])
def test_kernel_continuity_and_support(phi, knots):
    for k in knots:
        lo = phi(torch.tensor(k - 1e-12, dtype=torch.float64))
        hi = phi(torch.tensor(k + 1e-12, dtype=torch.float64))
        assert abs(float(lo - hi)) < 1e-9
    big = torch.tensor([2.0, 2.5, 3.0, -2.1], dtype=torch.float64)
    assert float(phi(big).abs().max()) == 0.0


def test_delta_scaling_eq21():
    """delta_h integrates to one on the grid: sum_x delta_h(x - X) hx hy = 1."""
    hx, hy = 0.1, 0.07
    X, Y = 0.4321, -0.1234
    xs = torch.arange(-40, 41, dtype=torch.float64) * hx
    ys = torch.arange(-40, 41, dtype=torch.float64) * hy
    for kind in (ib.PESKIN4, ib.ROMA3):
        d = ib.delta(kind, xs.reshape(1, -1) - X, ys.reshape(-1, 1) - Y, hx, hy)
        assert abs(float(d.sum()) * hx * hy - 1.0) < 1e-13


def test_point_in_polygon_matches_circle():
    X, Y, _ = S.circle_markers(126, 1.0, (0.0, 0.0))
    pts = torch.tensor(RNG.uniform(-0.8, 0.8, size=(2, 4000)))
    r = torch.sqrt(pts[0] ** 2 + pts[1] ** 2)
    keep = (r < 0.499) | (r > 0.501)
    inside = ib.inside_polygon(pts[0], pts[1], torch.tensor(X), torch.tensor(Y))
    assert bool((inside[keep] == (r[keep] < 0.5)).all())


def _small_cylinder(kernel=S.ROMA3, omega=0.0):
    return S.cylinder_2d(nx=48, ny=32, cells_per_d=8, nm=26, dt=0.01, steps=5, kernel=kernel,
                         centre_d=(2.0, 2.0), omega=omega)


def test_ib_faces_are_fluid_faces_next_to_solid():
    """Brute force over every face: IB = not solid and some same-component neighbour solid (§2.2)."""
    wl = _small_cylinder()
    g = grid_of(wl)
    body, _ = body_of(wl)
    w = torch.tensor([0.013, -0.021], dtype=torch.float64)
    masks = ib.classify(g, body, w)
    for c in range(2):
        solid, isib = masks[c]
        ez, ey, ex = solid.shape
        for j in range(ey):
            for i in range(ex):
                nbrs = [(j, i - 1), (j, i + 1), (j - 1, i), (j + 1, i)]
                adj = any(0 <= a < ey and 0 <= b < ex and bool(solid[0, a, b]) for a, b in nbrs)
                assert bool(isib[0, j, i]) == ((not bool(solid[0, j, i])) and adj)
        assert int(solid.sum()) > 0 and int(isib.sum()) > 0


@pytest.mark.parametrize("kernel", [S.ROMA3, S.PESKIN4])
def test_normalised_interpolation_reproduces_uniform_velocity(kernel):
    """Eq. (18) in normalised form returns the body velocity exactly when all markers share it."""
    wl = _small_cylinder(kernel)
    g = grid_of(wl)
    body, _ = body_of(wl)
    w = torch.tensor([0.0, 0.031], dtype=torch.float64)
    wd = torch.tensor([0.25, -0.4], dtype=torch.float64)
    masks = ib.classify(g, body, w)
    ut, uc = ib.target_velocity(g, body, kernel, w, wd, masks)
    for c in range(2):
        forced = masks[c][0] | masks[c][1]
        assert float((ut[c][forced] - wd[c]).abs().max()) < 1e-14
        assert float((uc[c][forced] - wd[c]).abs().max()) < 1e-14


def test_spread_interp_transpose_identity():
    """<S F, u>_{h^2} = <F, J u>_{dV} for the raw delta-weighted spread S and interpolation J."""
    wl = _small_cylinder(S.PESKIN4)
    g = grid_of(wl)
    body, _ = body_of(wl)
    Xm, Ym = body.markers(torch.tensor([0.0, 0.0], dtype=torch.float64))
    hx, hy = float(g.h[0][0]), float(g.h[1][0])
    dV = body.ds * hx
    W = ib.weights_matrix(g, 0, S.PESKIN4, Xm, Ym)
    F = torch.tensor(RNG.uniform(-1, 1, size=Xm.numel()))
    u = torch.tensor(RNG.uniform(-1, 1, size=g.shape(0)))
    SF = (W * (F * dV).reshape(-1, 1, 1, 1)).sum(0)
    Ju = (W * u.unsqueeze(0)).sum(dim=(1, 2, 3)) * hx * hy
    lhs = float((SF * u).sum()) * hx * hy
    rhs = float((F * Ju * dV).sum())
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_rotating_surface_interpolation_is_convex():
    """With a spinning surface the IB velocity is a convex combination of marker velocities."""
    wl = _small_cylinder(S.ROMA3, omega=2.0)
    g = grid_of(wl)
    body, _ = body_of(wl)
    w = torch.zeros(2, dtype=torch.float64)
    wd = torch.zeros(2, dtype=torch.float64)
    masks = ib.classify(g, body, w)
    ut, _ = ib.target_velocity(g, body, S.ROMA3, w, wd, masks)
    vmax = 2.0 * 0.5
    for c in range(2):
        isib = masks[c][1]
        assert float(ut[c][isib].abs().max()) <= vmax + 1e-14
        assert float(ut[c][isib].abs().max()) > 0.1


def test_fsi_step_runs_and_forces_sane():
    """A short cylinder run: divergence-free outside the body, finite drag of the right sign."""
    wl = _small_cylinder()
    g = grid_of(wl)
    body, params = body_of(wl)
    st = state_of(wl)
    for _ in range(3):
        st, dg = O.step(g, st, wl.dt, body=body, kernel=wl.kernel, params=params)
    assert float(dg.F[0]) > 0.0
    assert torch.isfinite(st.w).all() and torch.isfinite(st.wd).all()
