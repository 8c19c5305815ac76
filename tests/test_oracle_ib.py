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


def _wall_polygon(Y, xs_top):
    """Closed polygon of a rectangle x in [0.3, 1.7], y in [0.2, Y] whose top edge carries markers at xs_top."""
    X = [0.3, 1.7, 1.7] + [float(x) for x in sorted(xs_top, reverse=True)] + [0.3]
    Yp = [0.2, 0.2, Y] + [Y] * len(xs_top) + [Y]
    return X, Yp


@pytest.mark.parametrize("kernel", [ib.ROMA3, ib.PESKIN4])
@pytest.mark.parametrize("c", [0, 1])
def test_half_distribution_on_a_straight_wall(kernel, c):
    """Eq. (19) on a flat wall: a marker on a straight, grid-aligned wall midway between two face rows
    of component c has half of its delta distribution on solid faces, so F_N = 1 / (2 h_x h_y) exactly
    (both kernels are symmetric about the marker and sum to one along x).  Top-edge markers at
    arbitrary x, at least 2 h from the corners."""
    wl = S.box_2d(32, 24, (S.PERIODIC, S.PERIODIC), (S.FREESLIP, S.FREESLIP), Lx=2.0, Ly=1.5)
    g = grid_of(wl)
    h = 1.0 / 16
    Y = 12 * h if c == 0 else 11.5 * h        # midway between two rows of c-faces
    xs = np.array([0.71, 0.8333, 0.97, 1.0, 1.123, 1.29])
    X, Yp = _wall_polygon(Y, xs)
    body = ib.Body(X, Yp, np.ones(len(X)), (1.0, 0.5))
    masks = ib.classify(g, body, torch.zeros(2, dtype=torch.float64))
    solid = masks[c][0]
    Xm = torch.tensor(xs, dtype=torch.float64)
    Ym = torch.full_like(Xm, Y)
    FN = ib.half_distribution_sum(g, c, kernel, Xm, Ym, solid)
    assert float((FN * h * h - 0.5).abs().max()) < 1e-14


def _scalar_phi(kernel, r):
    a = abs(r)
    if kernel == ib.PESKIN4:
        if a <= 1.0:
            return (3.0 - 2.0 * a + math.sqrt(max(1.0 + 4.0 * a - 4.0 * a * a, 0.0))) / 8.0
        if a <= 2.0:
            return (5.0 - 2.0 * a - math.sqrt(max(-7.0 + 12.0 * a - 4.0 * a * a, 0.0))) / 8.0
        return 0.0
    if a <= 0.5:
        return (1.0 + math.sqrt(max(1.0 - 3.0 * a * a, 0.0))) / 3.0
    if a <= 1.5:
        return (5.0 - 3.0 * a - math.sqrt(max(1.0 - 3.0 * (1.0 - a) ** 2, 0.0))) / 6.0
    return 0.0


@pytest.mark.parametrize("kernel", [ib.ROMA3, ib.PESKIN4])
def test_target_velocity_brute_force_with_nonuniform_marker_velocity(kernel):
    """Eqs. (18)-(19) summed by hand with scalar loops over every (marker, face) pair, for a translating
    cylinder with a spinning surface (marker velocities differ): F_N_i = sum over non-solid faces of
    phi phi / (h_x h_y), w_i = delta_h dV_i / F_N_i, u_IB = sum w_i v_i / sum w_i on every IB face."""
    wl = _small_cylinder(kernel, omega=1.7)
    g = grid_of(wl)
    body, _ = body_of(wl)
    w = torch.tensor([0.0123, -0.0217], dtype=torch.float64)
    wd = torch.tensor([0.3, -0.2], dtype=torch.float64)
    masks = ib.classify(g, body, w)
    ut, _ = ib.target_velocity(g, body, kernel, w, wd, masks)
    hx, hy = float(g.h[0][0]), float(g.h[1][0])
    X0, Y0, ds = wl.body.X0, wl.body.Y0, wl.body.ds
    cx, cy = wl.body.centre[0] + float(w[0]), wl.body.centre[1] + float(w[1])
    Xm = [float(x) + float(w[0]) for x in X0]
    Ym = [float(y) + float(w[1]) for y in Y0]
    vel = [(float(wd[0]) - 1.7 * (Ym[i] - cy), float(wd[1]) + 1.7 * (Xm[i] - cx)) for i in range(len(Xm))]
    for c in range(2):
        fx, fy, _ = g.face_coords(c)
        ex, ey = g.ext(c)[0], g.ext(c)[1]
        xs = [float(fx.reshape(-1)[i if fx.numel() > 1 else 0]) for i in range(ex)]
        ys = [float(fy.reshape(-1)[j if fy.numel() > 1 else 0]) for j in range(ey)]
        solid = masks[c][0][0].numpy()
        isib = masks[c][1][0].numpy()
        FN = []
        for i in range(len(Xm)):
            s = 0.0
            for jj in range(ey):
                py = _scalar_phi(kernel, (ys[jj] - Ym[i]) / hy)
                if py == 0.0:
                    continue
                for ii in range(ex):
                    if not solid[jj, ii]:
                        s += _scalar_phi(kernel, (xs[ii] - Xm[i]) / hx) * py / (hx * hy)
            FN.append(s)
        checked = 0
        for jj in range(ey):
            for ii in range(ex):
                if not isib[jj, ii]:
                    continue
                num = den = 0.0
                for i in range(len(Xm)):
                    d = _scalar_phi(kernel, (xs[ii] - Xm[i]) / hx) * _scalar_phi(kernel, (ys[jj] - Ym[i]) / hy) / (hx * hy)
                    if d == 0.0:
                        continue
                    wgt = d * ds[i] * hx / FN[i]
                    num += wgt * vel[i][c]
                    den += wgt
                assert den > 0.0
                assert abs(float(ut[c][0, jj, ii]) - num / den) < 1e-13
                checked += 1
        assert checked > 20


def _periodic_circle(kernel, nm=40):
    """A circle of diameter 0.5 in a periodic unit box of 32^2 cells: every support is complete."""
    wl = S.box_2d(32, 32, (S.PERIODIC, S.PERIODIC), (S.PERIODIC, S.PERIODIC), Lx=1.0, Ly=1.0)
    g = grid_of(wl)
    X, Y, ds = S.circle_markers(nm, 0.5, (0.5, 0.5))
    return g, ib.Body(X, Y, ds, (0.5, 0.5)), 0.25


@pytest.mark.parametrize("kernel", [ib.ROMA3, ib.PESKIN4])
def test_marker_forces_of_uniform_forcing(kernel):
    """Eq. (20) with a uniform forcing f: the kernel sums to one over the faces (Eq. 21), so q_i = -f for
    every marker and component, and F = rho sum_i q_i dV_i = -rho f sum_i dV_i (dV_i = ds_i h)."""
    g, body, _ = _periodic_circle(kernel)
    g.rho = 1.3
    w = torch.tensor([0.0131, -0.0207], dtype=torch.float64)
    fv = (0.7, -1.9)
    f = [torch.full(g.shape(c), fv[c], dtype=torch.float64) for c in range(2)]
    q, F, torque = ib.marker_forces(g, body, kernel, w, f)
    for c in range(2):
        assert float((q[:, c] + fv[c]).abs().max()) < 1e-13
    sdV = float(body.ds.sum()) / 32
    for c in range(2):
        assert abs(float(F[c]) + 1.3 * fv[c] * sdV) < 1e-13


@pytest.mark.parametrize("kernel", [ib.ROMA3, ib.PESKIN4])
def test_marker_torque_closed_forms(kernel):
    """A rigid-rotation forcing f = Om (-(y - y_c), x - x_c) is linear, which the kernel reproduces at
    each marker (first moment, Eq. 22), so q_i = -f(X_i) and the torque rho sum dV_i (r_i x q_i) is
    -rho Om R^2 sum_i dV_i for markers on a circle of radius R; a radial forcing f = (x - x_c, y - y_c)
    gives zero torque."""
    g, body, R = _periodic_circle(kernel)
    w = torch.tensor([0.0131, -0.0207], dtype=torch.float64)
    cx, cy = 0.5 + float(w[0]), 0.5 + float(w[1])
    Om = 0.9
    fxu, fyu, _ = g.face_coords(0)
    fxv, fyv, _ = g.face_coords(1)
    f = [(-Om * (fyu - cy)).expand(g.shape(0)).clone(), (Om * (fxv - cx)).expand(g.shape(1)).clone()]
    q, F, torque = ib.marker_forces(g, body, kernel, w, f)
    Xm, Ym = body.markers(w)
    assert float((q[:, 0] - Om * (Ym - cy)).abs().max()) < 1e-13
    assert float((q[:, 1] + Om * (Xm - cx)).abs().max()) < 1e-13
    sdV = float(body.ds.sum()) / 32
    assert abs(float(torque) + Om * R * R * sdV) < 1e-13
    f = [(fxu - cx).expand(g.shape(0)).clone(), (fyv - cy).expand(g.shape(1)).clone()]
    _, _, torque = ib.marker_forces(g, body, kernel, w, f)
    assert abs(float(torque)) < 1e-14


def test_inside_test_of_several_contours_is_their_union():
    """A body of several closed contours (an array of cylinders moving as one): a point is solid when
    it lies inside one of the cylinders, against the distance to every centre (points within 2e-3 D of
    a circle, where the 40-gon's chords depart from it, skipped), and the solid faces are the union of the single-cylinder classifications."""
    wl = S.cylinder_array_2d(rows=2, cols=3, cells_per_d=8, nm_per=40)
    b = wl.body
    body = ib.Body(b.X0, b.Y0, b.ds, b.centre, 0.0, b.contours)
    assert len(set(body.next)) == len(body.next) == b.X0.size
    rng = np.random.default_rng(3)
    px = torch.tensor(rng.uniform(3.5, 10.5, 6000))
    py = torch.tensor(rng.uniform(0.5, 5.5, 6000))
    cs = [(4.0 + (q + 0.5) * 2.0, 1.0 + (r + 0.5) * 2.0) for r in range(2) for q in range(3)]
    dmin = torch.stack([torch.sqrt((px - cx) ** 2 + (py - cy) ** 2) for cx, cy in cs]).min(0).values
    keep = (dmin - 0.5).abs() > 2e-3        # beyond the chords' sagitta 0.5 (1 - cos(pi / 40)) = 1.5e-3
    inside = ib.inside_polygon(px, py, body.X0, body.Y0, body.next)
    assert bool((inside[keep] == (dmin[keep] < 0.5)).all()) and int(inside.sum()) > 500
    g = grid_of(wl)
    w = torch.tensor([0.0, 0.037], dtype=torch.float64)
    masks = ib.classify(g, body, w)
    for c in range(2):
        union = torch.zeros_like(masks[c][0])
        for k in range(6):
            sl = slice(b.contours[k], b.contours[k] + 40)
            one = ib.Body(b.X0[sl], b.Y0[sl], b.ds[sl], b.centre)
            union |= ib.classify(g, one, w)[c][0]
        assert torch.equal(masks[c][0], union)
