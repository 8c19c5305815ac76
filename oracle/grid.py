"""Staggered (MAC) finite-volume grid of §2.3.1 ("Fluid discretization").

Pressure lives at cell centres, velocity component c on the faces normal to
direction c.  Directions are x (d=0), y (d=1), z (d=2); a 2-D grid has a dummy
periodic z of one cell of unit width and no w component.

Storage of a velocity component c is a tensor of shape (ez, ey, ex), x fastest:
along its own direction c it holds n_c faces when that direction is periodic
(face f is the left face of cell f) and n_c + 1 faces otherwise (faces 0 and
n_c lie on the boundary); along the other directions it is cell-indexed.

Uniform and stretched spacing are both expressed through the face
coordinates ``xf[d]`` (n_d + 1 values), as in §2.5 ("uniform and smoothly
stretched grids").

Parity: the metrics are pinned by tests that difference polynomials exactly
(tests/test_oracle_operators.py).
"""
import torch

PERIODIC, NOSLIP, FREESLIP, INFLOW, OUTFLOW = 0, 1, 2, 3, 4
F64 = torch.float64


class Grid:
    """Metrics of the MAC grid.

    Arguments
      dim      2 or 3
      n        cell counts (nx, ny[, nz])
      xf       list of face-coordinate sequences, one per direction (n_d + 1)
      bc       bc[d] = (low, high) boundary types, PERIODIC on both sides or
               none; INFLOW only at x-low, OUTFLOW only at x-high
      bc_val   bc_val[d][side] = velocity vector imposed there (wall velocity
               for NOSLIP, inflow velocity for INFLOW); zeros by default
      nu, rho  kinematic viscosity and density (Eq. 1)
      conv     "central" (2nd-order) or "upwind" (1st-order) convection (§2.3.1)
      body_force  x-momentum source per y-row (ny values), the constant
               pressure-gradient forcing of §3.4.1; None for no source
    """

    def __init__(self, dim, n, xf, bc, bc_val=None, nu=0.0, rho=1.0,
                 conv="central", body_force=None):
        assert dim in (2, 3)
        self.dim = dim
        n = list(n)
        self.n = n + [1] * (3 - len(n))
        self.nu = float(nu)
        self.rho = float(rho)
        self.conv = conv
        bc = [tuple(b) for b in bc] + [(PERIODIC, PERIODIC)] * (3 - len(bc))
        self.bc = bc
        bc_val = list(bc_val or [])
        self.bc_val = []
        for d in range(3):
            sides = bc_val[d] if d < len(bc_val) else [[], []]
            self.bc_val.append([[float(x) for x in sides[s]] + [0.0] * (3 - len(sides[s]))
                                for s in range(2)])
        xf = list(xf) + [[0.0, 1.0]] * (3 - len(xf))
        self.xf = [torch.as_tensor(xf[d], dtype=F64).clone() for d in range(3)]
        for d in range(3):
            assert self.xf[d].numel() == self.n[d] + 1, "xf[%d] needs n+1 values" % d
            lo, hi = self.bc[d]
            assert (lo == PERIODIC) == (hi == PERIODIC), "periodic on one side only"
        self.body_force = None if body_force is None else torch.as_tensor(body_force, dtype=F64)

        # per-direction metrics
        self.L, self.xc, self.h, self.hf, self.theta = [], [], [], [], []
        for d in range(3):
            xfd = self.xf[d]
            nd = self.n[d]
            L = float(xfd[-1] - xfd[0])
            xc = 0.5 * (xfd[:-1] + xfd[1:])          # cell centres
            h = xfd[1:] - xfd[:-1]                   # cell widths
            if self.periodic(d):
                # face f (0..n-1) sits between cell f-1 and cell f (cell -1 wraps)
                xl = torch.roll(xc, 1)
                xl[0] = xl[0] - L
                hf = xc - xl                         # centre-to-centre spacing at face f
                theta = (xfd[:-1] - xl) / hf         # linear interpolation weight of the right cell
            else:
                hf = torch.empty(nd + 1, dtype=F64)
                theta = torch.full((nd + 1,), 0.5, dtype=F64)
                hf[1:nd] = xc[1:] - xc[:-1]
                theta[1:nd] = (xfd[1:nd] - xc[:-1]) / hf[1:nd]
                hf[0] = h[0]                         # ghost centre mirrored across the wall
                hf[nd] = h[nd - 1]
            self.L.append(L)
            self.xc.append(xc)
            self.h.append(h)
            self.hf.append(hf)
            self.theta.append(theta)

    # ---- topology -------------------------------------------------------
    def periodic(self, d):
        return self.bc[d][0] == PERIODIC

    def ncomp(self):
        return self.dim

    def ext(self, c):
        """(ex, ey, ez) extents of velocity component c."""
        e = list(self.n)
        if not self.periodic(c):
            e[c] += 1
        return e

    def shape(self, c):
        ex, ey, ez = self.ext(c)
        return (ez, ey, ex)

    def cshape(self):
        nx, ny, nz = self.n
        return (nz, ny, nx)

    def zeros(self):
        return [torch.zeros(self.shape(c), dtype=F64) for c in range(self.dim)]

    # ---- broadcasting helpers --------------------------------------------
    @staticmethod
    def along(d, v):
        """Reshape a 1-D tensor to broadcast along axis of direction d in (z, y, x) layout."""
        s = [1, 1, 1]
        s[2 - d] = v.numel()
        return v.reshape(s)

    def face_coords(self, c):
        """Coordinates (x, y, z) of the faces of component c, each broadcastable to shape(c)."""
        out = []
        for d in range(3):
            if d == c:
                xfd = self.xf[d] if not self.periodic(d) else self.xf[d][:-1]
                out.append(self.along(d, xfd))
            else:
                out.append(self.along(d, self.xc[d]))
        return out

    def face_volume(self, c):
        """Control volume of each c-face (hf along c times cell widths across)."""
        v = self.along(c, self.hf[c] if not self.periodic(c) else self.hf[c])
        for d in range(3):
            if d != c:
                v = v * self.along(d, self.h[d])
        return v.expand(self.shape(c))

    def cell_volume(self):
        v = self.along(0, self.h[0]) * self.along(1, self.h[1]) * self.along(2, self.h[2])
        return v.expand(self.cshape())

    def interior_mask(self, c):
        """True on the faces of component c whose velocity is an unknown (not on a non-periodic boundary)."""
        m = torch.ones(self.shape(c), dtype=torch.bool)
        if not self.periodic(c):
            e = self.ext(c)[c]
            idx = torch.arange(e)
            inner = (idx > 0) & (idx < e - 1)
            m = m & self.along(c, inner)
        return m
