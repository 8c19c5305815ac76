"""Conjugate-gradient solve of the pressure Poisson equation, Eq. (9) (oracle, FP64).

The paper's own pressure solver is a Krylov iteration: unpreconditioned CG by
default (§2.5 and Table 1; §3.5 names it as the solver of its timing runs).
This is that iteration written plainly, on the operator L = D G that the
oracle's divergence and gradient define, so that a CG solve on the GPU can be
checked against it and against the direct solve (poisson.solve, itself pinned
to a dense LU of the assembled L).

L is symmetric in the cell-volume inner product, so CG runs on the symmetric
positive semi-definite system
    A x = r,   A = -V L,   r = -V b,
whose null space (when no pressure is imposed anywhere) is the constant
vector; the right-hand side is first projected onto the range of A (its plain
mean removed), and the result is shifted to zero volume-weighted mean, the
gauge of poisson.solve.  Optional Jacobi preconditioning divides by diag(A).

Test infrastructure: imported only by the tests, the smoke check and the
benchmark's CPU baseline.
"""
import torch

from . import fluid


def apply_A(g, x):
    """A x = -V (D G x) at every cell."""
    return -g.cell_volume() * fluid.divergence(g, fluid.gradient(g, x))


def diag_A(g):
    """diag(A): V times sum_d (1/hf[lo] + 1/hf[hi]) / h, boundary faces of non-periodic directions
    carrying no gradient (G p . n = 0 there)."""
    d = torch.zeros(g.cshape(), dtype=torch.float64)
    for k in range(g.dim):
        n = g.n[k]
        ihf = 1.0 / g.hf[k]
        lo = ihf[0:n].clone()               # face f of cell f (periodic: n faces, face n = face 0)
        if g.periodic(k):
            hi = torch.roll(lo, -1)
        else:
            hi = ihf[1:n + 1].clone()
            lo[0] = 0.0
            hi[n - 1] = 0.0
        d = d + g.along(k, (lo + hi) / g.h[k])
    return g.cell_volume() * d


def cg_solve(g, b, tol=1e-13, maxit=None, jacobi=False):
    """Solve D G p = b by (preconditioned) CG.  Returns (p, iterations, final relative residual)."""
    n = b.numel()
    maxit = maxit or 4 * n
    V = g.cell_volume().expand(g.cshape())
    r = -V * b
    r = r - r.mean()
    r0 = float(torch.sqrt((r * r).sum()))
    x = torch.zeros_like(b)
    if r0 == 0.0:
        return x, 0, 0.0
    Minv = 1.0 / diag_A(g) if jacobi else None
    z = r * Minv if jacobi else r
    p = z.clone()
    rz = float((r * z).sum())
    it = 0
    rel = 1.0
    while it < maxit:
        q = apply_A(g, p)
        alpha = rz / float((p * q).sum())
        x = x + alpha * p
        r = r - alpha * q
        it += 1
        rel = float(torch.sqrt((r * r).sum())) / r0
        if rel < tol:
            break
        z = r * Minv if jacobi else r
        rz_new = float((r * z).sum())
        p = z + (rz_new / rz) * p
        rz = rz_new
    x = x - (V * x).sum() / V.sum()
    return x, it, rel
