"""Pins of the oracle's pressure solve (Eq. 9): dense LU of the assembled L = D G and closed-form eigenvalues."""
import math

import numpy as np
import pytest
import torch

import synthetic as S
from oracle import fluid, poisson
from helpers import grid_of

P, NS, FS, IN, OUT = S.PERIODIC, S.NOSLIP, S.FREESLIP, S.INFLOW, S.OUTFLOW

CASES_2D = [
    ((P, P), (P, P), 0.0),
    ((P, P), (NS, NS), 0.0),
    ((P, P), (NS, NS), 1.5),
    ((IN, OUT), (FS, FS), 0.0),
    ((NS, NS), (FS, FS), 1.2),
]
CASES_3D = [
    ((P, P), (NS, NS), 1.5),
    ((P, P), (P, P), 0.0),
    ((FS, FS), (NS, NS), 1.0),
]


def assembled_L(g):
    """Dense matrix of D(G(.)) built column by column from unit vectors."""
    N = int(np.prod(g.cshape()))
    L = torch.zeros((N, N), dtype=torch.float64)
    for i in range(N):
        e = torch.zeros(N, dtype=torch.float64)
        e[i] = 1.0
        L[:, i] = fluid.divergence(g, fluid.gradient(g, e.reshape(g.cshape()))).reshape(-1)
    return L


def dense_solve(g, b):
    """Bordered system [L  V; V^T 0][p; mu] = [b; 0]: the zero volume-mean solution."""
    L = assembled_L(g)
    N = L.shape[0]
    V = g.cell_volume().reshape(-1)
    A = torch.zeros((N + 1, N + 1), dtype=torch.float64)
    A[:N, :N] = L
    A[:N, N] = V
    A[N, :N] = V
    rhs = torch.cat([b.reshape(-1), torch.zeros(1, dtype=torch.float64)])
    return torch.linalg.solve(A, rhs)[:N].reshape(g.cshape())


def compatible_rhs(g, seed):
    rng = np.random.default_rng(seed)
    u = [torch.tensor(rng.uniform(-1, 1, size=g.shape(c))) for c in range(g.dim)]
    u = fluid.apply_boundary_values(g, u)
    if not g.periodic(0) and g.bc[0][1] == OUT:
        u = fluid.outflow_faces(g, u, u)
    return fluid.divergence(g, u)


@pytest.mark.parametrize("bcx,bcy,gamma", CASES_2D)
def test_poisson_dense_lu_2d(bcx, bcy, gamma):
    wl = S.box_2d(8, 6, bcx, bcy, Lx=1.3, Ly=0.9, stretched=gamma)
    g = grid_of(wl)
    b = compatible_rhs(g, 1)
    p = poisson.solve(g, b)
    pd = dense_solve(g, b)
    assert float((p - pd).abs().max()) <= 1e-12 * float(pd.abs().max())


@pytest.mark.parametrize("bcx,bcy,gamma", CASES_3D)
def test_poisson_dense_lu_3d(bcx, bcy, gamma):
    wl = S.box_3d(8, 8, 8, bcx, bcy, stretched=gamma)
    g = grid_of(wl)
    b = compatible_rhs(g, 2)
    p = poisson.solve(g, b)
    pd = dense_solve(g, b)
    assert float((p - pd).abs().max()) <= 1e-12 * float(pd.abs().max())


def test_poisson_fourier_eigenvalue():
    """A single Fourier mode is an eigenvector of L with eigenvalue -(2 - 2 cos(kh))/h^2 per direction."""
    n, L = 16, 2.0
    wl = S.box_2d(n, n, (P, P), (P, P), Lx=L, Ly=L)
    g = grid_of(wl)
    h = L / n
    x = (torch.arange(n, dtype=torch.float64) + 0.5) * h
    kx, ky = 3, 5
    p = torch.cos(2 * math.pi * kx * x / L).reshape(1, 1, n) * torch.sin(2 * math.pi * ky * x / L).reshape(1, n, 1)
    lam = -(2 - 2 * math.cos(2 * math.pi * kx / n)) / h ** 2 - (2 - 2 * math.cos(2 * math.pi * ky / n)) / h ** 2
    Lp = fluid.divergence(g, fluid.gradient(g, p))
    assert float((Lp - lam * p).abs().max()) < 1e-11 * abs(lam)
    sol = poisson.solve(g, lam * p)
    assert float((sol - p).abs().max()) < 1e-12


def test_poisson_dct_eigenvalue():
    """cos(pi k (i + 1/2) / n) is an eigenvector of the Neumann operator."""
    n = 12
    wl = S.box_2d(n, 4, (FS, FS), (P, P), Lx=1.0, Ly=1.0)
    g = grid_of(wl)
    h = 1.0 / n
    i = torch.arange(n, dtype=torch.float64)
    k = 4
    p = torch.cos(math.pi * k * (i + 0.5) / n).reshape(1, 1, n).expand(1, 4, n)
    lam = -(2 - 2 * math.cos(math.pi * k / n)) / h ** 2
    Lp = fluid.divergence(g, fluid.gradient(g, p))
    assert float((Lp - lam * p).abs().max()) < 1e-10 * abs(lam)


def test_projection_divergence_free():
    """Eq. (10) after Eq. (9) with eps = 0: ||D u^{n+1}||_inf < 1e-10 for every boundary combination."""
    for bcx, bcy, gamma in CASES_2D:
        wl = S.box_2d(16, 12, bcx, bcy, stretched=gamma)
        g = grid_of(wl)
        rng = np.random.default_rng(3)
        u = [torch.tensor(rng.uniform(-1, 1, size=g.shape(c))) for c in range(2)]
        u = fluid.apply_boundary_values(g, u)
        u = fluid.outflow_faces(g, u, u)
        un, _ = poisson.project(g, u)
        assert float(fluid.divergence(g, un).abs().max()) < 1e-10


@pytest.mark.parametrize("jacobi", [False, True])
@pytest.mark.parametrize("bcx,bcy,gamma", CASES_2D)
def test_oracle_cg_matches_dense_lu_2d(bcx, bcy, gamma, jacobi):
    """The paper's Krylov solver (CG, optionally Jacobi-preconditioned) reaches the same
    zero volume-mean solution as the dense LU of the assembled operator."""
    from oracle import krylov
    wl = S.box_2d(8, 6, bcx, bcy, Lx=1.3, Ly=0.9, stretched=gamma)
    g = grid_of(wl)
    b = compatible_rhs(g, 3)
    p, it, rel = krylov.cg_solve(g, b, tol=1e-14, jacobi=jacobi)
    pd = dense_solve(g, b)
    assert rel < 1e-14 and it <= 4 * b.numel()
    assert float((p - pd).abs().max()) <= 1e-10 * float(pd.abs().max())


@pytest.mark.parametrize("bcx,bcy,gamma", CASES_3D)
def test_oracle_cg_matches_direct_3d(bcx, bcy, gamma):
    from oracle import krylov
    wl = S.box_3d(8, 8, 8, bcx, bcy, stretched=gamma)
    g = grid_of(wl)
    b = compatible_rhs(g, 4)
    p, it, rel = krylov.cg_solve(g, b, tol=1e-14, jacobi=True)
    pd = dense_solve(g, b)
    assert float((p - pd).abs().max()) <= 1e-10 * float(pd.abs().max())


def test_oracle_jacobi_diagonal_is_the_operator_diagonal():
    from oracle import krylov
    for wl in [S.box_2d(6, 5, (P, P), (NS, NS), stretched=1.2), S.box_3d(4, 6, 4, (FS, FS), (P, P)),
               S.box_2d(5, 4, (IN, OUT), (FS, FS))]:
        g = grid_of(wl)
        A = -g.cell_volume().reshape(-1, 1) * assembled_L(g)
        assert torch.allclose(krylov.diag_A(g).reshape(-1), torch.diagonal(A), rtol=1e-13, atol=0)
