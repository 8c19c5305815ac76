"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the solver.  It produces grid geometry
(face coordinates), boundary descriptions, initial fields sampled at face
positions, marker sets and body parameters as plain float64 numpy arrays.
Both the oracle and the CUDA path receive the identical arrays.

Workloads (sizes and parameters from the paper's cases, §3):
  taylor_green_2d   periodic [0, 2 pi]^2 vortex, closed-form initial field
  isotropic_3d      periodic 128^3 random solenoidal field, E(k) ~ k^4 exp(-2 (k/4)^2), u_rms = 1
  channel_3d        2 pi x 2 x pi channel, tanh-stretched walls in y, laminar
                    profile plus 10 % seeded noise, constant-pressure-gradient forcing (§3.4.1)
  cylinder_2d       cylinder of diameter D = 40 cells in a 16 D x 8 D box, uniform inflow,
                    free-slip sides, outflow, 126 markers (§3.1-3.2)
  cylinder_array_2d an array of cylinders moving as one elastically mounted body (the
                    immersed-boundary stress case: 12 x 116 cylinders, 104,400 markers)
  poiseuille_2d     periodic channel with no-slip walls and a uniform body force

The initial fields are not made discretely divergence-free here; the first
projection of the first step does that on each side from identical inputs.
"""
import math
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

PERIODIC, NOSLIP, FREESLIP, INFLOW, OUTFLOW = 0, 1, 2, 3, 4
PESKIN4, ROMA3 = 0, 1


@dataclass
class BodySpec:
    X0: np.ndarray            # marker rest x (nm,)
    Y0: np.ndarray            # marker rest y (nm,)
    ds: np.ndarray            # arc length per marker (nm,)
    centre: tuple             # reference point at rest
    omega: float = 0.0        # prescribed surface angular velocity
    mass: float = 0.0         # 0: body held fixed (static)
    stiffness: float = 0.0
    damping: float = 0.0
    active: tuple = (False, False)
    w0: tuple = (0.0, 0.0)
    wd0: tuple = (0.0, 0.0)
    contours: Optional[list] = None   # first marker of each closed contour (None: one contour)


@dataclass
class BoxSpec:
    boxes: np.ndarray         # (nb, 6) x0, x1, y0, y1, z0, z1
    X: np.ndarray             # (nm, 3) surface marker positions
    dV: np.ndarray            # (nm,) marker volumes (surface area per marker x h)


@dataclass
class Workload:
    name: str
    dim: int
    n: List[int]
    xf: List[np.ndarray]
    bc: List[tuple]
    bc_val: list
    nu: float
    rho: float = 1.0
    conv: str = "central"
    scheme: str = "fe"
    dt: float = 0.0
    steps: int = 1
    precision: str = "fp64"
    kernel: int = ROMA3
    body_force: Optional[np.ndarray] = None
    body: Optional[BodySpec] = None
    boxes: Optional[BoxSpec] = None
    u0: List[np.ndarray] = field(default_factory=list)   # (ez, ey, ex) arrays per component

    def cells(self):
        return int(np.prod(self.n))


def uniform_faces(n, length, x0=0.0):
    return x0 + length * np.arange(n + 1, dtype=np.float64) / n


def tanh_faces(n, gamma):
    """y_j = tanh(gamma (2 j / n - 1)) / tanh(gamma), j = 0..n, on [-1, 1]."""
    j = np.arange(n + 1, dtype=np.float64)
    return np.tanh(gamma * (2.0 * j / n - 1.0)) / math.tanh(gamma)


def _centres(xf):
    return 0.5 * (xf[:-1] + xf[1:])


def _ext(n, c, bc):
    e = list(n)
    if bc[c][0] != PERIODIC:
        e[c] += 1
    return e


def _face_positions(n, xf, c, bc):
    """Broadcastable (x, y, z) coordinates of the c-faces (x fastest layout (ez, ey, ex))."""
    out = []
    for d in range(3):
        if d == c:
            v = xf[d] if bc[d][0] != PERIODIC else xf[d][:-1]
        else:
            v = _centres(xf[d])
        s = [1, 1, 1]
        s[2 - d] = v.size
        out.append(v.reshape(s))
    return out


def taylor_green_2d(n=64, nu=0.01, cfl=0.5, steps=100):
    """u = sin x cos y, v = -cos x sin y on [0, 2 pi]^2; dt = cfl h / max|u0| (= 0.5 h)."""
    L = 2.0 * math.pi
    xf = [uniform_faces(n, L), uniform_faces(n, L), np.array([0.0, 1.0])]
    bc = [(PERIODIC, PERIODIC)] * 3
    nn = [n, n, 1]
    x, y, _ = _face_positions(nn, xf, 0, bc)
    u = np.sin(x) * np.cos(y) * np.ones((1, n, n))
    x, y, _ = _face_positions(nn, xf, 1, bc)
    v = -np.cos(x) * np.sin(y) * np.ones((1, n, n))
    h = L / n
    return Workload("taylor_green_2d", 2, nn, xf, bc[:2], None, nu, dt=cfl * h / 1.0,
                    steps=steps, u0=[u, v])


def taylor_green_exact(n, nu, t):
    """Closed-form decaying vortex sampled at the faces of an n x n periodic grid."""
    L = 2.0 * math.pi
    xf = [uniform_faces(n, L), uniform_faces(n, L), np.array([0.0, 1.0])]
    bc = [(PERIODIC, PERIODIC)] * 3
    nn = [n, n, 1]
    dec = math.exp(-2.0 * nu * t)
    x, y, _ = _face_positions(nn, xf, 0, bc)
    u = np.sin(x) * np.cos(y) * dec * np.ones((1, n, n))
    x, y, _ = _face_positions(nn, xf, 1, bc)
    v = -np.cos(x) * np.sin(y) * dec * np.ones((1, n, n))
    return [u, v]


def isotropic_3d(n=128, seed=0, nu=1.0 / 400.0, cfl=0.5, steps=500, scheme="rk3", k0=4.0):
    """Random solenoidal field with E(k) ~ k^4 exp(-2 (k/k0)^2), rescaled to u_rms = 1.

    Fourier amplitudes |u_hat|^2 ~ E(k) / (4 pi k^2) with random phases, the
    spectral solenoidal projection applied, sampled at face positions by
    interpolation-free inverse FFT on staggered positions (half-cell phase shifts).
    dt = cfl h / max|u0|.
    """
    rng = np.random.default_rng(seed)
    L = 2.0 * math.pi
    h = L / n
    k1 = np.fft.fftfreq(n, d=1.0 / n)
    KZ, KY, KX = np.meshgrid(k1, k1, k1, indexing="ij")
    K2 = KX ** 2 + KY ** 2 + KZ ** 2
    Kmag = np.sqrt(K2)
    E = np.where(Kmag > 0, Kmag ** 4 * np.exp(-2.0 * (Kmag / k0) ** 2), 0.0)
    amp = np.sqrt(np.where(Kmag > 0, E / (4.0 * math.pi * np.where(K2 > 0, K2, 1.0)), 0.0))
    comps = []
    for _ in range(3):
        phase = rng.uniform(0.0, 2.0 * math.pi, size=(n, n, n))
        comps.append(amp * np.exp(1j * phase))
    kv = (KX, KY, KZ)
    kdotu = sum(kv[c] * comps[c] for c in range(3))
    K2s = np.where(K2 > 0, K2, 1.0)
    comps = [comps[c] - kv[c] * kdotu / K2s for c in range(3)]
    fields = []
    for c in range(3):
        # face c sits half a cell below the centre along c: shift by exp(-i k h/2) before inversion
        shift = np.exp(-1j * kv[c] * h * 0.5) * np.exp(1j * sum(kv[d] * h * 0.5 for d in range(3)))
        fields.append(np.real(np.fft.ifftn(comps[c] * shift)))
    rms = math.sqrt(sum(float(np.mean(f * f)) for f in fields) / 3.0)
    fields = [f / rms for f in fields]
    umax = max(float(np.abs(f).max()) for f in fields)
    xf = [uniform_faces(n, L)] * 3
    bc = [(PERIODIC, PERIODIC)] * 3
    return Workload("isotropic_3d", 3, [n, n, n], xf, bc, None, nu, scheme=scheme,
                    dt=cfl * h / umax, steps=steps, precision="mixed", u0=fields)


def channel_3d(nx=192, ny=128, nz=128, seed=1, gamma=1.5, re_tau=180.0, dt_plus=4e-3,
               ub=15.6, noise=0.1, steps=2000):
    """Re_tau = 180 channel in outer units (u_tau = delta = 1, nu = 1 / Re_tau, f_x = 1).

    u = 1.5 U_b (1 - y^2) plus noise * U_b seeded uniform noise on every
    component; dt = dt+ nu / u_tau^2.
    """
    rng = np.random.default_rng(seed)
    Lx, Lz = 2.0 * math.pi, math.pi
    xf = [uniform_faces(nx, Lx), tanh_faces(ny, gamma), uniform_faces(nz, Lz)]
    bc = [(PERIODIC, PERIODIC), (NOSLIP, NOSLIP), (PERIODIC, PERIODIC)]
    nn = [nx, ny, nz]
    nu = 1.0 / re_tau
    u0 = []
    for c in range(3):
        e = _ext(nn, c, bc)
        shp = (e[2], e[1], e[0])
        x, y, z = _face_positions(nn, xf, c, bc)
        base = 1.5 * ub * (1.0 - y * y) if c == 0 else 0.0
        fld = base + noise * ub * rng.uniform(-1.0, 1.0, size=shp)
        if c == 1:
            fld[:, 0, :] = 0.0
            fld[:, -1, :] = 0.0
        u0.append(np.ascontiguousarray(np.broadcast_to(fld, shp), dtype=np.float64))
    return Workload("channel_3d", 3, nn, xf, bc, None, nu, dt=dt_plus * nu, steps=steps,
                    precision="mixed", body_force=np.ones(ny), u0=u0)


def circle_markers(nm, D, centre):
    """nm markers equally spaced on a circle (counter-clockwise), arc length pi D / nm each."""
    t = 2.0 * math.pi * (np.arange(nm, dtype=np.float64) + 0.5) / nm
    X = centre[0] + 0.5 * D * np.cos(t)
    Y = centre[1] + 0.5 * D * np.sin(t)
    return X, Y, np.full(nm, math.pi * D / nm)


def cylinder_2d(nx=640, ny=320, cells_per_d=40, nm=126, re=150.0, mass_ratio=2.0,
                reduced_velocity=5.0, zeta=0.0, U=1.0, dt=0.005, steps=20000, kernel=ROMA3,
                k_factor=1.0, centre_d=(4.0, 4.0), precision="mixed", seed=None, perturb=0.0,
                omega=0.0):
    """Elastically mounted cylinder, 1-DOF transverse (the FSI workload of §3.2.1).

    Lengths in cylinder diameters (D = 1, h = 1 / cells_per_d), uniform inflow
    U at x = 0, zero-gradient outflow at x = Lx, free-slip y walls.  Body
    parameters m = m* rho pi D^2 / 4, f_n = U / (U_r D), k = k_factor m (2 pi f_n)^2,
    c = 2 m (2 pi f_n) zeta (§2.3.2).
    """
    D = 1.0
    h = D / cells_per_d
    Lx, Ly = nx * h, ny * h
    xf = [uniform_faces(nx, Lx), uniform_faces(ny, Ly), np.array([0.0, 1.0])]
    bc = [(INFLOW, OUTFLOW), (FREESLIP, FREESLIP)]
    bc_val = [[[U, 0.0, 0.0], [0.0, 0.0, 0.0]], [[0.0] * 3, [0.0] * 3]]
    nn = [nx, ny, 1]
    centre = (centre_d[0] * D, centre_d[1] * D)
    X, Y, ds = circle_markers(nm, D, centre)
    m = mass_ratio * math.pi * D * D / 4.0
    fn = U / (reduced_velocity * D)
    k = k_factor * m * (2.0 * math.pi * fn) ** 2
    c = 2.0 * m * 2.0 * math.pi * fn * zeta
    body = BodySpec(X, Y, ds, centre, omega=omega, mass=m, stiffness=k, damping=c,
                    active=(False, True))
    u = np.full((1, ny, nx + 1), U)
    v = np.zeros((1, ny + 1, nx))
    if seed is not None and perturb > 0:
        rng = np.random.default_rng(seed)
        v[:, 1:-1, :] = perturb * U * rng.uniform(-1.0, 1.0, size=(1, ny - 1, nx))
    return Workload("cylinder_2d", 2, nn, xf, bc, bc_val, U * D / re, dt=dt, steps=steps,
                    precision=precision, kernel=kernel, body=body, u0=[u, v])


def cylinder_array_2d(rows=12, cols=116, cells_per_d=24, pitch_d=2.0, margin_d=(4.0, 1.0), nm_per=None,
                      re=150.0, mass_ratio=2.0, reduced_velocity=5.0, U=1.0, dt=None, steps=100, kernel=ROMA3,
                      precision="mixed", seed=5, perturb=0.01):
    """A rows x cols array of cylinders (diameter D = 1 = cells_per_d cells, centres pitch_d D apart)
    moving as one elastically mounted rigid body (1-DOF transverse), in the FSI set-up of
    cylinder_2d: uniform inflow, zero-gradient outflow, free-slip y walls.  The immersed-boundary
    stress case: nm_per markers per cylinder (default one per grid spacing, pi cells_per_d), each
    cylinder a closed contour of its own.  Mass and stiffness scale with the number of cylinders
    (m = m* rho N pi D^2 / 4), so the body has the single cylinder's natural frequency."""
    D = 1.0
    h = D / cells_per_d
    nm_per = int(round(math.pi * cells_per_d)) if nm_per is None else int(nm_per)
    nx = int(round((2 * margin_d[0] + cols * pitch_d) * cells_per_d))
    ny = int(round((2 * margin_d[1] + rows * pitch_d) * cells_per_d))
    nx += nx % 2
    ny += ny % 2
    Lx, Ly = nx * h, ny * h
    xf = [uniform_faces(nx, Lx), uniform_faces(ny, Ly), np.array([0.0, 1.0])]
    bc = [(INFLOW, OUTFLOW), (FREESLIP, FREESLIP)]
    bc_val = [[[U, 0.0, 0.0], [0.0, 0.0, 0.0]], [[0.0] * 3, [0.0] * 3]]
    Xs, Ys, Ss, starts = [], [], [], []
    for r in range(rows):
        for q in range(cols):
            c = ((margin_d[0] + (q + 0.5) * pitch_d) * D, (margin_d[1] + (r + 0.5) * pitch_d) * D)
            X, Y, ds = circle_markers(nm_per, D, c)
            starts.append(len(Xs) * nm_per)
            Xs.append(X)
            Ys.append(Y)
            Ss.append(ds)
    X, Y, ds = np.concatenate(Xs), np.concatenate(Ys), np.concatenate(Ss)
    ncyl = rows * cols
    centre = (0.5 * Lx, 0.5 * Ly)
    m = mass_ratio * ncyl * math.pi * D * D / 4.0
    fn = U / (reduced_velocity * D)
    k = m * (2.0 * math.pi * fn) ** 2
    body = BodySpec(X, Y, ds, centre, mass=m, stiffness=k, damping=0.0, active=(False, True),
                    contours=starts)
    u = np.full((1, ny, nx + 1), U)
    v = np.zeros((1, ny + 1, nx))
    if seed is not None and perturb > 0:
        rng = np.random.default_rng(seed)
        v[:, 1:-1, :] = perturb * U * rng.uniform(-1.0, 1.0, size=(1, ny - 1, nx))
    if dt is None:
        dt = 0.2 * h
    return Workload("cylinder_array_2d", 2, [nx, ny, 1], xf, bc, bc_val, U * D / re, dt=dt, steps=steps,
                    precision=precision, kernel=kernel, body=body, u0=[u, v])


def ensemble_cylinders(members=64, seed=2, steps=500, precision="mixed", kmin=128, kmax=512):
    """Members of the batched-ensemble workload: 2-D cylinder flows (16 D x 8 D boxes) with
    nx drawn uniformly from the multiples of 32 in [kmin, kmax], ny = nx / 2, D = nx / 16
    cells, Re uniform in [50, 200], 1 % seeded noise on the initial cross-flow velocity,
    elastically mounted (m* = 2, U_r = 5) as in the FSI workload.  dt = min(0.2 h, 0.6 / Re) (D = U = 1):
    0.2 h keeps the advective CFL number at 0.2, and forward Euler with central convection also
    needs dt < 2 nu / |u|^2 (|u| up to about 1.5 U near the cylinder), which 0.2 h breaks on the
    coarse, high-Re members (those diverged within 500 steps)."""
    rng = np.random.default_rng(seed)
    sizes = np.arange(kmin, kmax + 1, 32)
    out = []
    for m in range(members):
        nx = int(rng.choice(sizes))
        re = float(rng.uniform(50.0, 200.0))
        cpd = nx // 16
        nm = int(round(math.pi * cpd))
        wl = cylinder_2d(nx=nx, ny=nx // 2, cells_per_d=cpd, nm=nm, re=re, dt=min(0.2 / cpd, 0.6 / re), steps=steps,
                         precision=precision, seed=int(seed * 1000 + m), perturb=0.01)
        wl.name = "cylinder_2d_member_%d" % m
        out.append(wl)
    return out


def poiseuille_2d(nx=8, ny=16, nu=1.0, fx=1.0, dt=None, steps=2000, stretched=0.0, slip=False):
    """Periodic-in-x channel y in [-1, 1] with no-slip (or free-slip) walls and body force fx."""
    Lx = 1.0
    yf = tanh_faces(ny, stretched) if stretched > 0 else uniform_faces(ny, 2.0, -1.0)
    xf = [uniform_faces(nx, Lx), yf, np.array([0.0, 1.0])]
    wall = FREESLIP if slip else NOSLIP
    bc = [(PERIODIC, PERIODIC), (wall, wall)]
    hmin = float(np.min(np.diff(yf)))
    if dt is None:
        dt = 0.2 * hmin * hmin / nu
    u = np.zeros((1, ny, nx))
    v = np.zeros((1, ny + 1, nx))
    return Workload("poiseuille_2d", 2, [nx, ny, 1], xf, bc, None, nu, dt=dt, steps=steps,
                    body_force=np.full(ny, fx), u0=[u, v])


def random_fields(wl, seed, scale=1.0):
    """Uniform random velocity on every face of a workload's grid (boundary faces included)."""
    rng = np.random.default_rng(seed)
    out = []
    for c in range(wl.dim):
        e = _ext(wl.n, c, wl.bc + [(PERIODIC, PERIODIC)] * (3 - len(wl.bc)))
        out.append(scale * rng.uniform(-1.0, 1.0, size=(e[2], e[1], e[0])))
    return out


def box_2d(nx, ny, bcx, bcy, Lx=1.0, Ly=1.0, stretched=0.0, nu=0.01, bc_val=None):
    """A generic small 2-D grid for operator tests."""
    yf = (Ly / 2) * (1 + tanh_faces(ny, stretched)) if stretched > 0 else uniform_faces(ny, Ly)
    xf = [uniform_faces(nx, Lx), yf, np.array([0.0, 1.0])]
    return Workload("box_2d", 2, [nx, ny, 1], xf, [bcx, bcy], bc_val, nu)


def box_3d(nx, ny, nz, bcx, bcy, bcz=(PERIODIC, PERIODIC), L=(1.0, 1.0, 1.0), stretched=0.0,
           nu=0.01, bc_val=None):
    yf = (L[1] / 2) * (1 + tanh_faces(ny, stretched)) if stretched > 0 else uniform_faces(ny, L[1])
    xf = [uniform_faces(nx, L[0]), yf, uniform_faces(nz, L[2])]
    return Workload("box_3d", 3, [nx, ny, nz], xf, [bcx, bcy, bcz], bc_val, nu)


def box_markers(box, spacing, h):
    """Markers on the six faces of a box at a lattice of the given spacing (cell-centred on each face);
    dV = (area per marker) * h, the shell of one grid spacing."""
    x0, x1, y0, y1, z0, z1 = box
    pts, vol = [], []

    def lattice(a0, a1):
        n = max(1, int(round((a1 - a0) / spacing)))
        return a0 + (np.arange(n) + 0.5) * (a1 - a0) / n, (a1 - a0) / n

    ax, dx = lattice(x0, x1)
    ay, dy = lattice(y0, y1)
    az, dz = lattice(z0, z1)
    for xv in (x0, x1):
        Y, Z = np.meshgrid(ay, az, indexing="ij")
        pts.append(np.stack([np.full(Y.size, xv), Y.ravel(), Z.ravel()], axis=1))
        vol.append(np.full(Y.size, dy * dz * h))
    for yv in (y0, y1):
        X, Z = np.meshgrid(ax, az, indexing="ij")
        pts.append(np.stack([X.ravel(), np.full(X.size, yv), Z.ravel()], axis=1))
        vol.append(np.full(X.size, dx * dz * h))
    for zv in (z0, z1):
        X, Y = np.meshgrid(ax, ay, indexing="ij")
        pts.append(np.stack([X.ravel(), Y.ravel(), np.full(X.size, zv)], axis=1))
        vol.append(np.full(X.size, dx * dy * h))
    return np.concatenate(pts), np.concatenate(vol)


def rough_channel_3d(nx=32, ny=32, nz=32, L=(2.0, 2.0, 2.0), cube=4, pitch=8, nu=0.01, dt=None, seed=4,
                     kernel=ROMA3, both_walls=False, noise=0.1, marker_spacing=1.0):
    """Channel with cube roughness on the wall(s): uniform grid, x and z periodic, no-slip y walls,
    constant x-momentum source f_x = 1, cubes of `cube` cells at a pitch of `pitch` cells
    (the rough-wall case of §3.4 in miniature), surface markers every `marker_spacing` h.
    Initial field: the laminar profile
    u = (1 - y^2) (y in [-1, 1]) plus `noise` seeded uniform noise on every component."""
    rng = np.random.default_rng(seed)
    xf = [uniform_faces(nx, L[0]), uniform_faces(ny, L[1], -L[1] / 2), uniform_faces(nz, L[2])]
    h = L[0] / nx
    bc = [(PERIODIC, PERIODIC), (NOSLIP, NOSLIP), (PERIODIC, PERIODIC)]
    boxes = []
    walls = [(-L[1] / 2, 1)] + ([(L[1] / 2, -1)] if both_walls else [])
    for i0 in range(pitch // 2, nx, pitch):
        for k0 in range(pitch // 2, nz, pitch):
            for yw, sgn in walls:
                x0 = xf[0][0] + (i0 - cube / 2) * h
                z0 = xf[2][0] + (k0 - cube / 2) * h
                ya, yb = sorted((yw, yw + sgn * cube * h))
                boxes.append([x0, x0 + cube * h, ya, yb, z0, z0 + cube * h])
    X, dV = [], []
    for b in boxes:
        x, v = box_markers(b, marker_spacing * h, h)
        X.append(x)
        dV.append(v)
    spec = BoxSpec(np.array(boxes), np.concatenate(X), np.concatenate(dV))
    nn = [nx, ny, nz]
    u0 = []
    for c in range(3):
        e = _ext(nn, c, bc)
        shp = (e[2], e[1], e[0])
        x, y, z = _face_positions(nn, xf, c, bc)
        base = (1.0 - (2.0 * y / L[1]) ** 2) if c == 0 else 0.0
        fld = base + noise * rng.uniform(-1.0, 1.0, size=shp)
        if c == 1:
            fld[:, 0, :] = 0.0
            fld[:, -1, :] = 0.0
        u0.append(np.ascontiguousarray(np.broadcast_to(fld, shp), dtype=np.float64))
    return Workload("rough_channel_3d", 3, nn, xf, bc, None, nu, dt=dt if dt else 0.2 * h, steps=10,
                    precision="fp64", kernel=kernel, body_force=np.ones(ny), boxes=spec, u0=u0)
