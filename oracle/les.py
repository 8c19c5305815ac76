"""Constant-coefficient Smagorinsky subgrid model (oracle, FP64), the LES option of §2.5
(constant Smagorinsky model; its use in the paper's channel LES, §3.4).

The paper states the model (eddy viscosity nu_t = (C_s Delta)^2 |S|, |S| = sqrt(2 S_ij S_ij))
but not its discretisation; the readings taken here are:
* uniform grids periodic in every direction (the decaying-turbulence LES case);
  Delta = (h_x h_y h_z)^(1/3);
* on the MAC grid the normal strains S_xx = du/dx, ... live at cell centres, the
  shear strains S_xy = (du/dy + dv/dx) / 2, ... at the cell edges where those two
  differences meet; |S| at a centre takes the shear strains averaged from the
  four edges around it;
* nu_t lives at cell centres and is averaged to an edge from its four cells;
* the subgrid stress tau_ij = 2 nu_t S_ij enters R as its divergence,
  R_i += d_j tau_ij, with tau_ii at centres and tau_ij (i != j) at edges.
With this arrangement the discrete subgrid term can only remove kinetic energy:
sum_faces u_i (d_j tau_ij) dv = -sum tau_ij S_ij dV <= 0 (tests/test_oracle_les.py).

Edge (i, j) of the xy family sits at (x_{i-1/2}, y_{j-1/2}), the corner of cells
(i-1, j-1) .. (i, j); likewise xz and yz.  Arrays are (z, y, x).

Test infrastructure only (see the package header).
"""
import torch


def _d(a, ax, h):
    """Forward difference (a[i+1] - a[i]) / h along array axis ax, periodic."""
    return (torch.roll(a, -1, dims=ax) - a) / h


def _b(a, ax, h):
    """Backward difference (a[i] - a[i-1]) / h along array axis ax, periodic."""
    return (a - torch.roll(a, 1, dims=ax)) / h


def strain(g, u):
    """(Sxx, Syy, Szz) at centres and (Sxy, Sxz, Syz) at edges."""
    hx, hy, hz = (float(g.h[d][0]) for d in range(3))
    U, V, W = u
    Sxx = _d(U, 2, hx)
    Syy = _d(V, 1, hy)
    Szz = _d(W, 0, hz)
    Sxy = 0.5 * (_b(U, 1, hy) + _b(V, 2, hx))
    Sxz = 0.5 * (_b(U, 0, hz) + _b(W, 2, hx))
    Syz = 0.5 * (_b(V, 0, hz) + _b(W, 1, hy))
    return Sxx, Syy, Szz, Sxy, Sxz, Syz


def _edge_to_centre(e, ax1, ax2):
    """Average of the four edges around each centre: edges (i, j), (i+1, j), (i, j+1), (i+1, j+1)."""
    a = e + torch.roll(e, -1, dims=ax1)
    return 0.25 * (a + torch.roll(a, -1, dims=ax2))


def _centre_to_edge(c, ax1, ax2):
    """Average of the four cells around each edge: cells (i-1, j-1), (i, j-1), (i-1, j), (i, j)."""
    a = c + torch.roll(c, 1, dims=ax1)
    return 0.25 * (a + torch.roll(a, 1, dims=ax2))


def nu_t(g, u, cs):
    """Eddy viscosity at cell centres."""
    hx, hy, hz = (float(g.h[d][0]) for d in range(3))
    delta = (hx * hy * hz) ** (1.0 / 3.0)
    Sxx, Syy, Szz, Sxy, Sxz, Syz = strain(g, u)
    cxy = _edge_to_centre(Sxy, 2, 1)
    cxz = _edge_to_centre(Sxz, 2, 0)
    cyz = _edge_to_centre(Syz, 1, 0)
    ss = Sxx * Sxx + Syy * Syy + Szz * Szz + 2.0 * (cxy * cxy + cxz * cxz + cyz * cyz)
    return (cs * delta) ** 2 * torch.sqrt(2.0 * ss)


def sgs_term(g, u, cs):
    """d_j tau_ij on the faces of each component, tau_ij = 2 nu_t S_ij."""
    hx, hy, hz = (float(g.h[d][0]) for d in range(3))
    nt = nu_t(g, u, cs)
    Sxx, Syy, Szz, Sxy, Sxz, Syz = strain(g, u)
    txx, tyy, tzz = 2.0 * nt * Sxx, 2.0 * nt * Syy, 2.0 * nt * Szz
    txy = 2.0 * _centre_to_edge(nt, 2, 1) * Sxy
    txz = 2.0 * _centre_to_edge(nt, 2, 0) * Sxz
    tyz = 2.0 * _centre_to_edge(nt, 1, 0) * Syz
    Ru = _b(txx, 2, hx) + _d(txy, 1, hy) + _d(txz, 0, hz)
    Rv = _d(txy, 2, hx) + _b(tyy, 1, hy) + _d(tyz, 0, hz)
    Rw = _d(txz, 2, hx) + _d(tyz, 1, hy) + _b(tzz, 0, hz)
    return [Ru, Rv, Rw]
