"""Exact solve of the discrete pressure Poisson equation, Eq. (9) of §2.3.1 (oracle, FP64).

The paper solves L p = b with an iterative Krylov method (CG/BiCG/GMRES,
Table 1; unpreconditioned CG in §3.5).  Those iterations converge to the
unique zero-mean solution of the same linear system L = D G, so the oracle
computes that solution directly:

* x (and z in 3-D) must be uniform.  Periodic directions are diagonalised by
  the DFT (eigenvalues -(2 - 2 cos(2 pi k / n)) / h^2), Neumann directions
  (walls, inflow, outflow: G p . n = 0) by the DCT-II (eigenvalues
  -(2 - 2 cos(pi k / n)) / h^2).
* y may be stretched.  For each x/z wavenumber the remaining operator is
  tridiagonal in y and is solved by the Thomas algorithm; a periodic y must be
  uniform and is diagonalised by the DFT instead.
* The one singular mode (all wavenumbers zero, no Dirichlet pressure
  anywhere) is solved with p_0 = 0 in place of its first row, then shifted to
  zero volume-weighted mean.  Every solution returned has sum(p V) = 0.

torch.fft is used as a library primitive for the DFT; the DCT is a dense
orthonormal cosine matrix.

Parity: pinned against a dense LU solve of the assembled operator L = D G on
small grids for every boundary combination, including stretched y
(tests/test_oracle_poisson.py), and against the closed-form eigenvalues.
"""
import math

import torch

from .grid import F64


def dct_matrix(n):
    """Orthonormal DCT-II matrix C[k, i] = s_k cos(pi k (i + 1/2) / n)."""
    k = torch.arange(n, dtype=F64).reshape(-1, 1)
    i = torch.arange(n, dtype=F64).reshape(1, -1)
    C = torch.cos(math.pi * k * (i + 0.5) / n) * math.sqrt(2.0 / n)
    C[0] = C[0] / math.sqrt(2.0)
    return C


def _eig(n, h, periodic):
    k = torch.arange(n, dtype=F64)
    if periodic:
        return -(2.0 - 2.0 * torch.cos(2.0 * math.pi * k / n)) / (h * h)
    return -(2.0 - 2.0 * torch.cos(math.pi * k / n)) / (h * h)


def _uniform_h(g, d):
    h = g.h[d]
    if float((h - h[0]).abs().max()) > 1e-12 * float(h[0]):
        raise ValueError("direction %d must be uniform for the transform solver" % d)
    return float(h[0])


def _fwd(x, ax, periodic, n):
    if periodic:
        return torch.fft.fft(x, dim=ax)
    C = dct_matrix(n).to(x.dtype)
    return torch.movedim(torch.tensordot(C, torch.movedim(x, ax, 0), dims=([1], [0])), 0, ax)


def _inv(x, ax, periodic, n):
    if periodic:
        return torch.fft.ifft(x, dim=ax)
    C = dct_matrix(n).to(x.dtype)
    return torch.movedim(torch.tensordot(C.t(), torch.movedim(x, ax, 0), dims=([1], [0])), 0, ax)


def y_coefficients(g):
    """Tridiagonal couplings of L along y: a_j (to j-1), c_j (to j+1); boundary terms dropped."""
    ny = g.n[1]
    h, hf = g.h[1], g.hf[1]
    a = 1.0 / (hf[:ny] * h)
    if g.periodic(1):
        c = 1.0 / (torch.roll(hf[:ny], -1) * h)
    else:
        c = 1.0 / (hf[1:ny + 1] * h)
        a = torch.cat([torch.zeros(1, dtype=F64), a[1:]])      # G p = 0 on the wall face
        c = torch.cat([c[:-1], torch.zeros(1, dtype=F64)])
    return a, c


def solve(g, b):
    """Zero-mean solution p of D G p = b (cell-centred, shape (nz, ny, nx))."""
    nx, ny, nz = g.n
    B = b.to(torch.complex128)
    lam = torch.zeros((1, 1, 1), dtype=F64)
    for d, ax in ((0, 2), (2, 0)):
        if d >= g.dim:
            continue
        hd = _uniform_h(g, d)
        B = _fwd(B, ax, g.periodic(d), g.n[d])
        lam = lam + g.along(d, _eig(g.n[d], hd, g.periodic(d)))
    lam = lam.expand(nz, 1, nx)

    if g.periodic(1):
        hy = _uniform_h(g, 1)
        B = torch.fft.fft(B, dim=1)
        lam3 = lam + g.along(1, _eig(ny, hy, True))
        zero = lam3 == 0
        P = torch.where(zero, torch.zeros_like(B), B / torch.where(zero, torch.ones_like(lam3), lam3))
        P = torch.fft.ifft(P, dim=1)
    else:
        a, c = y_coefficients(g)
        P = _thomas_modes(a, c, lam, B, g.h[1])
    for d, ax in ((2, 0), (0, 2)):
        if d >= g.dim:
            continue
        P = _inv(P, ax, g.periodic(d), g.n[d])
    p = P.real
    V = g.cell_volume()
    return p - (p * V).sum() / V.sum()


def _thomas_modes(a, c, lam, B, hy):
    """Solve a_j p_{j-1} + (-(a_j + c_j) + lam) p_j + c_j p_{j+1} = B_j for every (z, x) mode.

    The mode with lam == 0 is singular (constant null vector): its row 0 is
    replaced by p_0 = 0 and its solution shifted to zero hy-weighted mean.
    """
    ny = a.numel()
    nz, _, nx = B.shape
    lam2 = lam.reshape(nz, nx)
    singular = lam2 == 0
    diag = [(-(a[j] + c[j]) + lam2).to(torch.complex128) for j in range(ny)]
    rhs = [B[:, j, :] for j in range(ny)]
    one = torch.ones_like(diag[0])
    # row 0 of the singular mode: p_0 = 0
    diag[0] = torch.where(singular, one, diag[0])
    c0 = torch.where(singular, torch.zeros_like(diag[0]), c[0] * one)
    rhs[0] = torch.where(singular, torch.zeros_like(rhs[0]), rhs[0])
    # forward elimination
    cp = [c0 / diag[0]]
    dp = [rhs[0] / diag[0]]
    for j in range(1, ny):
        beta = diag[j] - a[j] * cp[j - 1]
        cp.append(c[j] / beta)
        dp.append((rhs[j] - a[j] * dp[j - 1]) / beta)
    # back substitution
    x = [None] * ny
    x[ny - 1] = dp[ny - 1]
    for j in range(ny - 2, -1, -1):
        x[j] = dp[j] - cp[j] * x[j + 1]
    P = torch.stack(x, dim=1)
    w = hy.to(torch.complex128).reshape(1, ny, 1)
    mean = (P * w).sum(dim=1, keepdim=True) / w.sum()
    return torch.where(singular.reshape(nz, 1, nx), P - mean, P)


def project(g, u, uc=None, eps=None):
    """Projection of Eqs. (9)-(10): solve L phi = D[(1 - eps) u + eps uc], return (u - G phi, phi).

    phi is the pressure scaled by dt / rho (Eq. 10: u^{n+1} = u* - (dt/rho) grad p).
    Only interior faces are corrected (G phi is zero on non-periodic boundary faces).
    """
    from .fluid import divergence, gradient
    if eps is None:
        ut = u
    else:
        ut = [torch.where(eps[c], uc[c], u[c]) for c in range(g.dim)]
    b = divergence(g, ut)
    phi = solve(g, b)
    G = gradient(g, phi)
    return [u[c] - G[c] for c in range(g.dim)], phi
