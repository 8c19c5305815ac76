"""GPU vs oracle parity of the forward step through the C ABI (Eqs. 4-10, 18-23, 12).

Tolerances: relative L2 over all velocity components <= 1e-11 for FP64 grids,
<= 1e-5 for mixed-precision grids (FP32 stencils / transforms, FP64 tridiagonal,
reductions and body ODE): FP64 to the rounding of a few steps, mixed precision to the FP32
rounding of the stencils and transforms, unless a test states a reason for another bound."""
import math

import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S
from gpu_util import field_err, run_gpu, run_oracle
from helpers import grid_of

pytestmark = pytest.mark.gpu
P, NS, FS, IN, OUT = S.PERIODIC, S.NOSLIP, S.FREESLIP, S.INFLOW, S.OUTFLOW
TOL64, TOLMIX = 1e-11, 1e-5


def test_taylor_green_64_fp64_100_steps():
    """The 2-D Taylor-Green workload: 64^2, nu = 0.01, CFL 0.5, 100 forward-Euler steps."""
    wl = S.taylor_green_2d(64, 0.01)
    gp = run_gpu(wl, 100)
    st, _, g = run_oracle(wl, 100)
    assert field_err(gp["u"], st.u) < TOL64
    ex = [torch.tensor(a) for a in S.taylor_green_exact(64, 0.01, 100 * wl.dt)]
    assert field_err(gp["u"], ex) < 5e-3
    d = gp["grid"].diagnostics(gp["u_dev"])
    assert d["divmax"] < 1e-10


@pytest.mark.parametrize("scheme", ["fe", "rk3"])
@pytest.mark.parametrize("conv", ["central", "upwind"])
def test_periodic_3d_fp64(scheme, conv):
    wl = S.box_3d(16, 12, 8, (P, P), (P, P), L=(1.0, 0.75, 0.5), nu=0.02)
    wl.conv, wl.scheme, wl.dt = conv, scheme, 0.004
    wl.u0 = S.random_fields(wl, 4, 0.5)
    gp = run_gpu(wl, 8)
    st, _, _ = run_oracle(wl, 8)
    assert field_err(gp["u"], st.u) < TOL64


def test_channel_stretched_fp64_with_pressure():
    wl = S.box_3d(16, 12, 8, (P, P), (NS, NS), L=(2.0, 2.0, 1.0), stretched=1.5, nu=0.05)
    wl.body_force = np.linspace(0.5, 1.5, 12)
    wl.dt = 0.002
    wl.u0 = S.random_fields(wl, 5, 1.0)
    gp = run_gpu(wl, 10, want_p=True)
    st, dg, g = run_oracle(wl, 10)
    assert field_err(gp["u"], st.u) < TOL64
    p_or = dg.phi * g.rho / wl.dt
    assert float((gp["p"] - p_or).abs().max()) < 1e-9 * float(p_or.abs().max())


@pytest.mark.parametrize("bcx,bcy,gamma,n", [
    ((P, P), (NS, NS), 0.0, (16, 12)),
    ((P, P), (FS, FS), 1.2, (12, 10)),
    ((IN, OUT), (FS, FS), 0.0, (24, 12)),
    ((NS, NS), (FS, FS), 0.0, (9, 10)),        # odd DCT length
    ((FS, FS), (NS, NS), 1.1, (14, 8)),        # radix 7
    ((P, P), (P, P), 0.0, (22, 26)),           # radices 11 and 13
])
def test_2d_boundary_combinations_fp64(bcx, bcy, gamma, n):
    bc_val = [[[1.0, 0, 0], [0, 0, 0]], [[0.3, 0, 0], [0.0, 0, 0]]]
    wl = S.box_2d(n[0], n[1], bcx, bcy, Lx=1.3, Ly=1.0, stretched=gamma, nu=0.02, bc_val=bc_val)
    wl.dt = 0.002
    wl.u0 = S.random_fields(wl, 6, 1.0)
    gp = run_gpu(wl, 6)
    st, _, _ = run_oracle(wl, 6)
    assert field_err(gp["u"], st.u) < TOL64
    assert gp["grid"].diagnostics(gp["u_dev"])["divmax"] < 1e-10


@pytest.mark.parametrize("kind,wl", [
    ("2d", S.box_2d(12, 10, (P, P), (NS, NS), stretched=1.3)),
    ("2d", S.box_2d(9, 7, (IN, OUT), (FS, FS))),
    ("2d", S.box_2d(28, 6, (P, P), (P, P))),
    ("3d", S.box_3d(16, 12, 8, (P, P), (NS, NS), stretched=1.5)),
    ("3d", S.box_3d(12, 8, 10, (P, P), (P, P))),
])
def test_solve_pressure_fp64(kind, wl):
    from paper_2505_23940_b300 import grid_from_workload
    from oracle import fluid, poisson
    g = grid_of(wl)
    rng = np.random.default_rng(8)
    u = [torch.tensor(rng.uniform(-1, 1, size=g.shape(c))) for c in range(g.dim)]
    u = fluid.apply_boundary_values(g, u)
    u = fluid.outflow_faces(g, u, u)
    b = fluid.divergence(g, u)
    ref = poisson.solve(g, b)
    G = grid_from_workload(wl, "fp64")
    p = G.solve_pressure(b.cuda().contiguous())
    torch.cuda.synchronize()
    assert float((p.cpu() - ref).abs().max()) < 1e-12 * float(ref.abs().max())


@pytest.mark.parametrize("segments", [4, 8, 16])
@pytest.mark.parametrize("wl", [
    S.box_2d(40, 70, (P, P), (NS, NS), stretched=1.3),
    S.box_2d(24, 37, (IN, OUT), (FS, FS)),
    S.box_3d(10, 66, 6, (P, P), (NS, NS), stretched=1.5),
])
def test_solve_pressure_segments_fp64(wl, segments):
    """The partitioned wall-normal solve with 4, 8 and 16 segments per column
    (ragged segment lengths) against the oracle's direct solve."""
    from paper_2505_23940_b300 import grid_from_workload
    from oracle import fluid, poisson
    g = grid_of(wl)
    rng = np.random.default_rng(11)
    u = [torch.tensor(rng.uniform(-1, 1, size=g.shape(c))) for c in range(g.dim)]
    u = fluid.apply_boundary_values(g, u)
    u = fluid.outflow_faces(g, u, u)
    b = fluid.divergence(g, u)
    ref = poisson.solve(g, b)
    G = grid_from_workload(wl, "fp64")
    G.set_tuning("ysolve_segments", segments)
    p = G.solve_pressure(b.cuda().contiguous())
    torch.cuda.synchronize()
    assert float((p.cpu() - ref).abs().max()) < 1e-12 * float(ref.abs().max())


_CT_CASES = {
    "x320": lambda: S.box_2d(320, 6, (P, P), (NS, NS), stretched=1.2),   # x DFT, compile-time 320
    "x160dct": lambda: S.box_2d(160, 8, (IN, OUT), (FS, FS)),            # x DCT-II, 160
    "z224": lambda: S.box_3d(8, 6, 224, (P, P), (NS, NS)),               # z, 224 (radix 7)
    "y352": lambda: S.box_3d(6, 352, 4, (P, P), (P, P)),                 # periodic y, 352 (radix 11)
    "x640dct": lambda: S.box_2d(640, 8, (IN, OUT), (FS, FS)),            # x DCT-II, 640 (FP32 plan only)
    "z512": lambda: S.box_3d(4, 4, 512, (P, P), (P, P)),                 # z, 512 (FP32 plan only)
}


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", sorted(_CT_CASES))
def test_solve_pressure_compile_time_lengths(case, precision):
    """Transform lengths with compile-time plans (and, in FP64, the generic plans of the
    lengths whose compile-time kernels would not fit in shared memory) against the
    oracle's direct solve; in mixed precision, two steps against the oracle's."""
    from paper_2505_23940_b300 import grid_from_workload
    wl = _CT_CASES[case]()
    from oracle import fluid, poisson
    if precision == "mixed":   # FP32 transforms inside the step (the pressure entry point is FP64)
        hmin = min(float(np.diff(wl.xf[d]).min()) for d in range(wl.dim))
        wl.dt = 0.1 * hmin
        wl.u0 = S.random_fields(wl, 9, 1.0)
        gp = run_gpu(wl, 2, precision="mixed")
        st, _, _ = run_oracle(wl, 2)
        assert field_err(gp["u"], st.u) < TOLMIX
        return
    g = grid_of(wl)
    rng = np.random.default_rng(9)
    u = [torch.tensor(rng.uniform(-1, 1, size=g.shape(c))) for c in range(g.dim)]
    u = fluid.apply_boundary_values(g, u)
    u = fluid.outflow_faces(g, u, u)
    b = fluid.divergence(g, u)
    ref = poisson.solve(g, b)
    G = grid_from_workload(wl, precision)
    p = G.solve_pressure(b.cuda().contiguous())
    torch.cuda.synchronize()
    assert float((p.cpu() - ref).abs().max()) < 1e-12 * float(ref.abs().max())


@pytest.mark.parametrize("wl", [
    S.box_3d(12, 16, 10, (P, P), (P, P)),
    S.box_3d(8, 70, 6, (P, P), (P, P)),          # ragged segments, 8 segments (narrow 8-column blocks)
    S.box_2d(24, 40, (P, P), (P, P)),
])
def test_periodic_y_cyclic_tridiagonal_fp64(wl):
    """Periodic y solved by the FP64 cyclic partitioned tridiagonal (y_spectral = 0)
    against the oracle's direct solve and against the spectral y solve."""
    from paper_2505_23940_b300 import grid_from_workload
    from oracle import fluid, poisson
    g = grid_of(wl)
    rng = np.random.default_rng(12)
    u = [torch.tensor(rng.uniform(-1, 1, size=g.shape(c))) for c in range(g.dim)]
    b = fluid.divergence(g, u)
    ref = poisson.solve(g, b)
    out = []
    for spectral in (0, 1):
        G = grid_from_workload(wl, "fp64")
        G.set_tuning("y_spectral", spectral)
        out.append(G.solve_pressure(b.cuda().contiguous()).cpu())
    torch.cuda.synchronize()
    scale = float(ref.abs().max())
    assert float((out[0] - ref).abs().max()) < 1e-12 * scale
    assert float((out[0] - out[1]).abs().max()) < 1e-12 * scale


_TWIST_CASES = [
    S.box_2d(40, 70, (P, P), (NS, NS), stretched=1.3),     # walls, stretched, 40 of 64 columns active
    S.box_2d(24, 37, (IN, OUT), (FS, FS)),                 # x DCT-II, odd chain length
    S.box_3d(10, 66, 6, (P, P), (NS, NS), stretched=1.5),
    S.box_3d(12, 16, 10, (P, P), (P, P)),                  # periodic y: cyclic, chain of 15
    S.box_2d(24, 6, (P, P), (P, P)),                       # shortest cyclic chain (5 rows)
    S.box_2d(18, 5, (P, P), (NS, NS)),                     # walls, 5 rows
    S.box_2d(20, 300, (P, P), (NS, NS), stretched=1.1),    # 300 rows (32-column blocks)
    S.box_2d(24, 200, (P, P), (NS, NS), stretched=1.1),    # 200 rows, one 64-column block per SM
    S.box_3d(8, 256, 4, (P, P), (P, P)),                   # cyclic, 256 rows
    S.box_2d(16, 400, (P, P), (P, P)),                     # largest twisted column (200 KB tile), cyclic
]


@pytest.mark.parametrize("wl", _TWIST_CASES)
def test_solve_pressure_twisted_fp64(wl):
    """The twisted two-thread y solve (forced on small grids) against the oracle's direct
    solve and against the partitioned solve of the same grid."""
    from paper_2505_23940_b300 import grid_from_workload
    from oracle import fluid, poisson
    g = grid_of(wl)
    rng = np.random.default_rng(13)
    u = [torch.tensor(rng.uniform(-1, 1, size=g.shape(c))) for c in range(g.dim)]
    u = fluid.apply_boundary_values(g, u)
    u = fluid.outflow_faces(g, u, u)
    b = fluid.divergence(g, u)
    ref = poisson.solve(g, b)
    out = []
    for tw in (1, 0):
        G = grid_from_workload(wl, "fp64")
        if wl.bc[1][0] == P:
            G.set_tuning("y_spectral", 0)
        G.set_tuning("ysolve_twisted", tw)
        out.append(G.solve_pressure(b.cuda().contiguous()).cpu())
    torch.cuda.synchronize()
    # the FP64 field tolerance (1e-11): the 400-row cyclic column, condition number ~ (400 / pi)^2,
    # lands near 1e-12 with either solve form
    scale = float(ref.abs().max())
    assert float((out[0] - ref).abs().max()) < 1e-11 * scale
    assert float((out[0] - out[1]).abs().max()) < 1e-11 * scale


@pytest.mark.parametrize("tiled", [1, 0, "cols32"])
@pytest.mark.parametrize("make", [
    lambda: S.isotropic_3d(n=32, steps=5),
    lambda: S.box_3d(16, 24, 8, (P, P), (NS, NS), stretched=1.2),
    lambda: S.box_2d(18, 24, (P, P), (NS, NS), stretched=1.2),    # rows not 16-byte multiples: plain loads
    lambda: S.box_3d(64, 66, 4, (P, P), (NS, NS), stretched=1.2),  # three 32-row boxes, ragged
    lambda: S.box_3d(32, 100, 4, (P, P), (P, P)),                  # cyclic, four boxes overlapping
    lambda: S.box_3d(16, 200, 4, (P, P), (NS, NS), stretched=1.1),  # 200 rows: 13 boxes
])
def test_mixed_twisted_y_solve(make, tiled):
    """Mixed precision with the twisted FP64 y solve (integer-pipe FP32 <-> FP64
    conversions, FP32 gauge of the zero mode; tiles as tensor-map boxes or row copies)
    against the FP64 oracle over steps."""
    wl = make()
    from paper_2505_23940_b300 import grid_from_workload
    if not wl.u0:
        hmin = min(float(np.diff(wl.xf[d]).min()) for d in range(wl.dim))
        wl.dt = 0.1 * hmin
        wl.u0 = S.random_fields(wl, 14, 1.0)
    n = 5
    st, _, _ = run_oracle(wl, n)
    G = grid_from_workload(wl, "mixed")
    if wl.bc[1][0] == P:
        G.set_tuning("y_spectral", 0)
    G.set_tuning("ysolve_twisted", 1)
    if tiled == "cols32":   # 32-column blocks (sweep and helper warps trading places in every other block)
        G.set_tuning("ysolve_twist_columns", 32)
    else:
        G.set_tuning("ysolve_tiled", tiled)
    u = [torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda").contiguous() for a in wl.u0]
    G.step(u, wl.dt, n)
    torch.cuda.synchronize()
    assert G.device_status() == 0
    assert field_err([x.double().cpu() for x in u], st.u) < TOLMIX


def test_mixed_isotropic_fp64_y_solve():
    """The isotropic RK3 step in mixed precision with the FP64 cyclic tridiagonal y solve
    (FP32 stencils and x/z transforms, FP64 Poisson along y) against the FP64 oracle."""
    from paper_2505_23940_b300 import grid_from_workload
    wl = S.isotropic_3d(n=32, steps=5)
    st, _, _ = run_oracle(wl, 5)
    G = grid_from_workload(wl, "mixed")
    G.set_tuning("y_spectral", 0)
    u = [torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda").contiguous() for a in wl.u0]
    G.step(u, wl.dt, 5)
    torch.cuda.synchronize()
    assert field_err([x.double().cpu() for x in u], st.u) < TOLMIX


def _small_cyl(kernel, precision="fp64", omega=0.0):
    wl = S.cylinder_2d(nx=48, ny=32, cells_per_d=8, nm=26, dt=0.01, kernel=kernel, centre_d=(2.0, 2.0),
                       precision=precision, seed=3, perturb=0.05, omega=omega)
    wl.body.w0 = (0.0, 0.05)
    return wl


@pytest.mark.parametrize("kernel", [S.ROMA3, S.PESKIN4])
def test_cylinder_fsi_fp64(kernel):
    wl = _small_cyl(kernel)
    gp = run_gpu(wl, 10)
    st, dg, _ = run_oracle(wl, 10)
    assert field_err(gp["u"], st.u) < TOL64
    assert float((gp["body"][:2] - st.w).abs().max()) < 1e-12
    assert float((gp["body"][2:] - st.wd).abs().max()) < 1e-11
    F, _ = gp["F"]
    assert abs(F[0] - float(dg.F[0])) < 1e-10 * abs(float(dg.F[0]))
    assert abs(F[1] - float(dg.F[1])) < 1e-9 * max(abs(float(dg.F[1])), 1e-3)


@pytest.mark.parametrize("kernel", [S.ROMA3, S.PESKIN4])
def test_cylinder_array_fsi_fp64_and_mixed(kernel):
    """A 2 x 3 array of cylinders moving as one elastically mounted body (six closed contours; the
    solid test over several contours, the cell-binned IB gather across contours): fields, body state
    and force against the oracle after 6 steps, FP64 and mixed precision."""
    wl = S.cylinder_array_2d(rows=2, cols=3, cells_per_d=8, nm_per=25, kernel=kernel)
    wl.body.w0 = (0.0, 0.02)
    st, dg, _ = run_oracle(wl, 6)
    gp = run_gpu(wl, 6, precision="fp64")
    assert field_err(gp["u"], st.u) < TOL64
    assert float((gp["body"][:2] - st.w).abs().max()) < 1e-12
    assert float((gp["body"][2:] - st.wd).abs().max()) < 1e-11
    F, _ = gp["F"]
    assert abs(F[1] - float(dg.F[1])) < 1e-9 * max(abs(float(dg.F[1])), 1e-3)
    gm = run_gpu(wl, 6, precision="mixed")
    assert field_err(gm["u"], st.u) < TOLMIX


def test_fsi_step_is_bitwise_reproducible():
    """The IB interpolation is a per-face gather in a fixed order and the force sums have a fixed
    order, so two FP64 runs of the 640 x 320 FSI workload give identical bits (fields and body)."""
    wl = S.cylinder_2d(seed=2, perturb=0.01)
    wl.body.w0 = (0.0, 0.1)
    a = run_gpu(wl, 5, precision="fp64")
    b = run_gpu(wl, 5, precision="fp64")
    assert all(torch.equal(x, y) for x, y in zip(a["u"], b["u"]))
    assert torch.equal(a["body"], b["body"])


def test_cylinder_rotating_surface_fp64():
    wl = _small_cyl(S.ROMA3, omega=1.5)
    gp = run_gpu(wl, 5)
    st, _, _ = run_oracle(wl, 5)
    assert field_err(gp["u"], st.u) < TOL64


def test_mixed_taylor_green_100_steps():
    wl = S.taylor_green_2d(64, 0.01)
    gp = run_gpu(wl, 100, precision="mixed")
    st, _, _ = run_oracle(wl, 100)
    assert field_err(gp["u"], st.u) < TOLMIX


def test_mixed_isotropic_32_rk3():
    wl = S.isotropic_3d(n=32, steps=20)
    gp = run_gpu(wl, 20, precision="mixed")
    st, _, _ = run_oracle(wl, 20)
    assert field_err(gp["u"], st.u) < TOLMIX


@pytest.mark.parametrize("n", [(64, 64, 64), (128, 64, 128), (64, 128, 64), (64, 256, 64), (256, 64, 64),
                               (64, 64, 256)])
def test_mixed_periodic_transform_shapes(n):
    """Fully periodic 3-D mixed grids whose x, z and periodic-y transforms take
    the register FFT kernels of lengths 64 / 128 / 256, against the FP64 oracle."""
    L = (1.0, 0.8, 1.2)
    wl = S.box_3d(*n, (P, P), (P, P), L=L, nu=0.001)
    hmin = min(L[d] / n[d] for d in range(3))
    wl.scheme, wl.dt, wl.precision = "rk3", 0.25 * hmin, "mixed"   # CFL 0.25 for |u| <= 1
    wl.u0 = S.random_fields(wl, 11, 1.0)
    gp = run_gpu(wl, 5, precision="mixed")
    st, _, _ = run_oracle(wl, 5)
    assert field_err(gp["u"], st.u) < TOLMIX
    d = gp["grid"].diagnostics(gp["u_dev"])
    assert d["divmax"] < 1e-3 * d["umax"] * max(n)


@pytest.mark.parametrize("n,kz,chunk", [((128, 16, 8), 8, 0), ((128, 14, 10), 8, 0), ((128, 10, 12), 5, 0),
                                        ((256, 6, 6), 4, 0), ((256, 12, 6), 1, 0),
                                        ((128, 14, 10), 8, 3), ((256, 12, 8), 4, 3), ((128, 10, 12), 5, 5)])
def test_mixed_staged_predictor(n, kz, chunk):
    """The shared-memory staged predictor (bulk asynchronous copies of whole
    planes; n_x = 128 / 256, ragged y blocks and z chunks, plane ring reuse; equal
    shares of the units (chunk 0 on these small grids) and runs aligned across row
    blocks, ragged last run) against the FP64 oracle and the unstaged z-marching kernel."""
    from paper_2505_23940_b300 import grid_from_workload
    L = (1.0, 0.8, 1.2)
    wl = S.box_3d(*n, (P, P), (P, P), L=L, nu=0.001)
    hmin = min(L[d] / n[d] for d in range(3))
    wl.scheme, wl.dt, wl.precision = "rk3", 0.25 * hmin, "mixed"
    wl.u0 = S.random_fields(wl, 12, 1.0)
    st, _, _ = run_oracle(wl, 3)
    out = []
    for staged in (1, 0):
        g = grid_from_workload(wl, "mixed")
        g.set_tuning("predictor_zmarch", kz)
        g.set_tuning("predictor_staged", staged)
        g.set_tuning("predictor_chunk", chunk)
        u = [torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda").contiguous() for a in wl.u0]
        g.step(u, wl.dt, 3)
        assert g.device_status() == 0
        out.append([x.double().cpu() for x in u])
        assert field_err(out[-1], st.u) < TOLMIX
    assert field_err(out[0], out[1]) < 1e-6


def test_mixed_channel_small_100_steps():
    wl = S.channel_3d(nx=24, ny=16, nz=16, steps=100)
    gp = run_gpu(wl, 100, precision="mixed")
    st, _, _ = run_oracle(wl, 100)
    assert field_err(gp["u"], st.u) < TOLMIX


def test_mixed_cylinder_small():
    wl = _small_cyl(S.ROMA3, precision="mixed")
    gp = run_gpu(wl, 20)
    st, _, _ = run_oracle(wl, 20)
    assert field_err(gp["u"], st.u) < TOLMIX
    assert float((gp["body"][:2] - st.w).abs().max()) < 1e-7


def test_zero_steps_is_identity():
    wl = S.taylor_green_2d(16, 0.01)
    gp = run_gpu(wl, 0)
    assert field_err(gp["u"], [torch.tensor(a) for a in wl.u0]) == 0.0


@pytest.mark.parametrize("active", [(False, True), (True, True)])
def test_strong_coupling_fp64(active):
    """Strongly coupled FSI (Algorithm 1, 1-DOF and 2-DOF) against the oracle's sub-iteration:
    fields, body state and the number of sub-iterations of every step."""
    from oracle.step import step_coupled
    from helpers import body_of
    from paper_2505_23940_b300 import body_tensor, grid_from_workload
    wl = S.cylinder_2d(nx=48, ny=32, cells_per_d=8, nm=26, dt=0.01, centre_d=(2.0, 2.0), precision="fp64",
                       seed=3, perturb=0.05, mass_ratio=1.0)
    wl.body.w0 = (0.02, 0.05)
    wl.body.active = active
    g = grid_of(wl)
    body, params = body_of(wl)
    st = O.State([torch.tensor(a, dtype=torch.float64) for a in wl.u0],
                 torch.tensor(wl.body.w0, dtype=torch.float64), torch.tensor(wl.body.wd0, dtype=torch.float64))
    G = grid_from_workload(wl, "fp64")
    G.set_coupling(30, 1e-10)
    u = [torch.tensor(a, dtype=torch.float64, device="cuda") for a in wl.u0]
    bt = body_tensor(wl)
    for _ in range(4):
        st, _, k, xi = step_coupled(g, st, wl.dt, body, wl.kernel, params, max_iter=30, tol=1e-10)
        G.step(u, wl.dt, 1, body=bt)
        kg, xig = G.coupling_stats()
        assert kg == k and k > 1
    torch.cuda.synchronize()
    assert field_err([x.cpu() for x in u], st.u) < TOL64
    assert float((bt[:2].cpu() - st.w).abs().max()) < 1e-12
    assert float((bt[2:].cpu() - st.wd).abs().max()) < 1e-11


@pytest.mark.parametrize("kernel", [S.ROMA3, S.PESKIN4])
def test_rough_channel_static_boxes_fp64(kernel):
    """Static 3-D box body (cube roughness on a channel wall): fields, the force on the body and
    every marker force against the oracle."""
    wl = S.rough_channel_3d(16, 16, 16, cube=4, pitch=8, kernel=kernel)
    gp = run_gpu(wl, 10)
    st, dg, _ = run_oracle(wl, 10)
    assert field_err(gp["u"], st.u) < TOL64
    F, q = gp["grid"].box_forces(with_q=True)
    for d in range(3):
        assert abs(F[d] - float(dg.F[d])) <= 1e-10 * float(dg.F.abs().max())
    qo = dg.q.numpy()
    assert np.abs(np.array(q) - qo).max() <= 1e-10 * np.abs(qo).max()


def test_rough_channel_static_boxes_mixed():
    wl = S.rough_channel_3d(32, 16, 32, cube=4, pitch=8, both_walls=True)
    gp = run_gpu(wl, 10, precision="mixed")
    st, dg, _ = run_oracle(wl, 10)
    assert field_err(gp["u"], st.u) < TOLMIX
    F = gp["grid"].box_forces()
    assert abs(F[0] - float(dg.F[0])) <= 1e-4 * abs(float(dg.F[0]))


@pytest.mark.parametrize("scheme,precision", [("fe", "fp64"), ("rk3", "fp64"), ("rk3", "mixed")])
def test_smagorinsky_les(scheme, precision):
    """Constant-coefficient Smagorinsky LES on a periodic box against the oracle's subgrid term."""
    from paper_2505_23940_b300 import FsError, grid_from_workload
    wl = S.box_3d(16, 12, 8, (P, P), (P, P), L=(1.0, 0.75, 0.5), nu=0.002)
    wl.scheme, wl.dt = scheme, 0.004
    wl.u0 = S.random_fields(wl, 9, 1.0)
    cs = 0.17
    g = grid_of(wl)
    st = O.State([torch.tensor(a) for a in wl.u0])
    for _ in range(8):
        st, _ = O.step(g, st, wl.dt, scheme=scheme, cs=cs)
    G = grid_from_workload(wl, precision)
    G.set_les(cs)
    u = [torch.tensor(a, dtype=G.dtype, device="cuda") for a in wl.u0]
    G.step(u, wl.dt, 8)
    torch.cuda.synchronize()
    assert field_err([x.double().cpu() for x in u], st.u) < (TOL64 if precision == "fp64" else TOLMIX)
    # the model changes the result (the comparison is not vacuous)
    st0 = O.State([torch.tensor(a) for a in wl.u0])
    for _ in range(8):
        st0, _ = O.step(g, st0, wl.dt, scheme=scheme)
    assert field_err(st.u, st0.u) > 1e-6
    with pytest.raises(FsError):
        G.step_adjoint(u, [torch.zeros_like(x) for x in u], wl.dt)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_split_two_stream_poisson_matches_single_stream(precision):
    """The periodic-z Poisson solve with the twisted FP64 y solve split into two independent
    z / y / z chains on two streams (two column blocks along x) gives the single-stream result bit for
    bit, and the oracle's within the stated tolerance, over 3 SSP-RK3 steps."""
    wl = S.box_3d(128, 24, 64, (S.PERIODIC, S.PERIODIC), (S.PERIODIC, S.PERIODIC), L=(2.0, 0.375, 1.0), nu=0.01)
    wl.scheme = "rk3"
    wl.u0 = S.random_fields(wl, 17, 1.0)
    wl.dt = 0.002
    tune = [("y_spectral", 0), ("ysolve_twisted", 1)]
    a = run_gpu(wl, 3, precision=precision, tuning=tune + [("ysplit", 1)])
    b = run_gpu(wl, 3, precision=precision, tuning=tune + [("ysplit", 0)])
    assert a["grid"].device_status() == 0 and b["grid"].device_status() == 0
    assert all(torch.equal(x, y) for x, y in zip(a["u"], b["u"]))
    st, _, _ = run_oracle(wl, 3)
    assert field_err(a["u"], st.u) < (TOL64 if precision == "fp64" else TOLMIX)


@pytest.mark.parametrize("scheme", ["fe", "rk3"])
@pytest.mark.parametrize("n", [(64, 48), (36, 20)])
def test_2d_periodic_four_cell_predictor_mixed(n, scheme):
    """The four-cell 2-D predictor of fully periodic FP32 grids (a row of 36 cells: a partial
    warp) against the FP64 oracle over steps, and against the one-cell kernel it replaces."""
    wl = S.box_2d(n[0], n[1], (P, P), (P, P), Lx=1.3, nu=0.02)
    wl.scheme = scheme
    wl.dt = 0.002
    wl.body_force = np.linspace(0.2, 0.8, n[1])
    wl.u0 = S.random_fields(wl, 7, 1.0)
    st, _, _ = run_oracle(wl, 6)
    a = run_gpu(wl, 6, precision="mixed")
    b = run_gpu(wl, 6, precision="mixed", tuning=[("predictor_cells", 1)])
    assert field_err(a["u"], st.u) < TOLMIX
    assert field_err(a["u"], b["u"]) < 1e-6


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("make", [
    lambda: S.box_3d(16, 24, 8, (P, P), (P, P)),                     # cyclic y
    lambda: S.box_3d(16, 24, 8, (P, P), (NS, NS), stretched=1.3),    # walls, stretched y
])
def test_twisted_pressure_gauge(make, precision):
    """The twisted y solve sets the zero mode's gauge (zero hy-weighted mean, the oracle's) in the
    solve whose pressure is written out, and only there: the written pressure matches the
    oracle's, and the velocity does not depend on whether the pressure was asked for (the stage
    solves keep the factorisation's gauge, which the pressure gradient does not see)."""
    wl = make()
    wl.dt = 0.002
    wl.u0 = S.random_fields(wl, 5, 1.0)
    tune = [("ysolve_twisted", 1)] + ([("y_spectral", 0)] if wl.bc[1][0] == P else [])
    a = run_gpu(wl, 4, precision=precision, want_p=True, tuning=tune)
    b = run_gpu(wl, 4, precision=precision, tuning=tune)
    st, dg, g = run_oracle(wl, 4)
    fp64 = precision == "fp64"
    assert field_err(a["u"], st.u) < (TOL64 if fp64 else TOLMIX)
    assert field_err(a["u"], b["u"]) < (1e-13 if fp64 else 1e-6)
    p_or = dg.phi * g.rho / wl.dt
    # FP32 fields: the pressure carries the FP32 rounding of u* through the solve; a wrong gauge
    # would be off by the column's mean, O(1) of max |p|
    tol = 1e-9 if fp64 else 1e-4
    assert float((a["p"] - p_or).abs().max()) < tol * float(p_or.abs().max())


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("axis", ["x", "z", "y"])
@pytest.mark.parametrize("n", [384, 512])
def test_register_fft_384_512(n, axis, precision):
    """The 384- and 512-point register transforms (first pass: three 16-point and sixteen 3-point
    DFTs, or two 16-point DFTs and a radix-2 step; second pass: 8- or 16-point DFTs) along x, z
    and the spectral y, through whole steps against the FP64 oracle."""
    if axis == "x":
        wl = S.box_3d(n, 6, 4, (P, P), (NS, NS), stretched=1.2)
    elif axis == "z":
        wl = S.box_3d(8, 6, n, (P, P), (NS, NS), L=(1.0, 1.0, 4.0))
    else:
        wl = S.box_3d(8, n, 4, (P, P), (P, P), L=(1.0, 4.0, 1.0))
    wl.dt = 0.001
    wl.u0 = S.random_fields(wl, 9, 1.0)
    gp = run_gpu(wl, 3, precision=precision)
    st, _, _ = run_oracle(wl, 3)
    assert field_err(gp["u"], st.u) < (TOL64 if precision == "fp64" else TOLMIX)


@pytest.mark.parametrize("precision,ny", [("mixed", 4096), ("fp64", 2000), ("mixed", 2000)])
def test_long_periodic_y_spectral(precision, ny):
    """Periodic y on long columns against the FP64 oracle: 2000 rows by the mixed-radix kernels (a
    few lines per block, 1024 threads per block where the block holds at most four lines), 4096
    rows by the three-launch four-step form."""
    # square cells of h = 8 / ny; |u| <= 1, CFL <= 0.1 and nu dt / h^2 <= 0.01 (stable steps)
    wl = S.box_2d(16, ny, (P, P), (P, P), Lx=16 * 8.0 / ny, Ly=8.0, nu=1e-4)
    wl.dt = 0.0002
    wl.u0 = S.random_fields(wl, 4, 1.0)
    gp = run_gpu(wl, 3, precision=precision)
    st, _, _ = run_oracle(wl, 3)
    assert field_err(gp["u"], st.u) < (TOL64 if precision == "fp64" else TOLMIX)


@pytest.mark.parametrize("form", [1, 2])
@pytest.mark.parametrize("n,ny,bcy,yspec", [(64, 24, (NS, NS), None), (128, 16, (P, P), 0),
                                             (128, 16, (P, P), 1), (64, 64, (P, P), 0)])
def test_xz_plane_transforms(n, ny, bcy, yspec, form):
    """Mixed precision, the x and z transforms fused per y position (nx = nz of 64 or 128: the
    x-z plane in shared memory, one pass each way, the divergence formed on the fly; form 1 one
    block per plane, form 2 the plane split over a two-block cluster exchanging its halves
    through distributed shared memory): whole RK3 steps against the FP64 oracle, and against
    the separate x and z kernels (xz_plane off) to FP32 rounding; walls in y (stretched) and
    periodic y by the FP64 twisted solve and by the FP32 DFT."""
    wl = S.box_3d(n, ny, n, (P, P), bcy, stretched=1.2 if bcy == (NS, NS) else 0.0, nu=1e-3)
    wl.dt = 0.002
    wl.u0 = S.random_fields(wl, 11, 1.0)
    tune = [] if yspec is None else [("y_spectral", yspec)]
    gp = run_gpu(wl, 3, precision="mixed", tuning=tune + [("xz_plane", form)])
    gs = run_gpu(wl, 3, precision="mixed", tuning=tune + [("xz_plane", 0)])
    st, _, _ = run_oracle(wl, 3)
    assert field_err(gp["u"], st.u) < TOLMIX
    # both forms round in FP32 (about 6e-8 per operation); their difference stays well below TOLMIX
    assert field_err(gp["u"], gs["u"]) < 1e-6


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("shape", [(40, 4096), (8, 4096, 4)])
def test_four_step_periodic_y(precision, shape):
    """Periodic y of 4096-row columns in three launches (64-point DFTs over the rows of each
    residue class mod 64 with the 4096-point twiddles; the eigenvalue division in the middle
    launch, whose blocks hold the row groups k1 and 64 - k1): two slot tiles, the second
    holding 8 slots, in 2-D, and four z planes in 3-D, against the FP64 oracle."""
    h = 8.0 / 4096   # square cells; |u| <= 1, CFL <= 0.1, nu dt / h^2 <= 0.01
    if len(shape) == 2:
        wl = S.box_2d(shape[0], 4096, (P, P), (P, P), Lx=shape[0] * h, Ly=8.0, nu=1e-4)
    else:
        wl = S.box_3d(shape[0], 4096, shape[2], (P, P), (P, P), L=(shape[0] * h, 8.0, shape[2] * h), nu=1e-4)
    wl.dt = 0.0002
    wl.u0 = S.random_fields(wl, 7, 1.0)
    gp = run_gpu(wl, 3, precision=precision)
    st, _, _ = run_oracle(wl, 3)
    assert field_err(gp["u"], st.u) < (TOL64 if precision == "fp64" else TOLMIX)


@pytest.mark.parametrize("precision,nx,bcx,ny", [("mixed", 4096, (P, P), 16), ("fp64", 4096, (P, P), 16),
                                                 ("fp64", 4096, (P, P), 15), ("fp64", 4096, (IN, OUT), 16),
                                                 ("mixed", 4096, (IN, OUT), 15), ("fp64", 2000, (IN, OUT), 16),
                                                 ("mixed", 2000, (IN, OUT), 16), ("fp64", 5760, (IN, OUT), 16),
                                                 ("mixed", 5760, (IN, OUT), 16)])
def test_long_x_lines(precision, nx, bcx, ny):
    """x transforms of long rows with one line per block (4096 points: the radix-16 kernels;
    5760: the compile-time plan; 2000: the runtime plan; FP64: lines beyond the usual
    shared-memory budget): the periodic DFT with the divergence fused, and the DCT-II of an
    inflow/outflow channel, with an odd row count (the last line's second row empty), against
    the FP64 oracle."""
    h = 1.0 / 256
    bcy = (NS, NS) if bcx == (P, P) else (FS, FS)
    bc_val = None if bcx == (P, P) else [[[1.0, 0, 0], [0, 0, 0]], [[0, 0, 0], [0, 0, 0]]]
    wl = S.box_2d(nx, ny, bcx, bcy, Lx=nx * h, Ly=ny * h, nu=1e-4, bc_val=bc_val)
    wl.dt = 0.1 * h
    wl.u0 = S.random_fields(wl, 6, 1.0)
    gp = run_gpu(wl, 3, precision=precision)
    st, _, _ = run_oracle(wl, 3)
    # FP32 rounding of the Neumann x solve grows about linearly with the row length: 3.8e-6 at
    # 640 points and 1.2e-5 at 2000 (the same with one or two lines per block)
    tol_mixed = 2.5e-5 * nx / 2000 if bcx != (P, P) else TOLMIX
    assert field_err(gp["u"], st.u) < (TOL64 if precision == "fp64" else tol_mixed)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("ny,bcy", [(37, (NS, NS)), (33, (NS, NS)), (25, (P, P))])
def test_twisted_requested_on_odd_ny(precision, ny, bcy):
    """The twisted y solve requested on odd ny: on walls it runs with row copies (the tensor-map
    boxes assume the lower thread's first chunk covers the bottom box), on periodic y the
    partitioned form takes over (the cyclic twisted form needs an odd chain, ny even)."""
    wl = S.box_3d(16, ny, 4, (P, P), bcy, stretched=0.0 if bcy == (P, P) else 1.2)
    wl.dt = 0.002
    wl.u0 = S.random_fields(wl, 5, 1.0)
    tune = [("ysolve_twisted", 1), ("ysolve_tiled", 1)] + ([("y_spectral", 0)] if bcy == (P, P) else [])
    gp = run_gpu(wl, 3, precision=precision, tuning=tune)
    st, _, _ = run_oracle(wl, 3)
    assert gp["grid"].device_status() == 0
    assert field_err(gp["u"], st.u) < (TOL64 if precision == "fp64" else TOLMIX)



@pytest.mark.parametrize("bcy", [(NS, NS), (P, P)])
def test_twisted_mixed_long_columns(bcy):
    """Mixed precision, the twisted y solve on 300-row columns: 32-column blocks (the sweep and
    helper warps trading places in every other block), tensor-map tiles of 19 boxes, the scaled
    outward pass; walls (stretched) and periodic y, against the FP64 oracle."""
    wl = S.box_3d(16, 300, 4, (P, P), bcy, stretched=1.1 if bcy == (NS, NS) else 0.0, L=(1.0, 3.0, 1.0))
    wl.dt = 0.001
    wl.u0 = S.random_fields(wl, 8, 1.0)
    tune = [("ysolve_twisted", 1)] + ([("y_spectral", 0)] if bcy == (P, P) else [])
    gp = run_gpu(wl, 3, precision="mixed", tuning=tune)
    st, _, _ = run_oracle(wl, 3)
    assert gp["grid"].device_status() == 0
    assert field_err(gp["u"], st.u) < TOLMIX
