"""The paper's Krylov pressure solver (CG, §2.5 / Table 1) on the GPU, fs_solve_pressure_cg,
against the oracle: the same zero volume-mean solution as the direct solve (pinned to a dense LU)
and the same iteration count as the oracle's own CG."""
import numpy as np
import pytest
import torch

import synthetic as S
from oracle import fluid, krylov, poisson
from helpers import grid_of

pytestmark = pytest.mark.gpu
P, NS, FS, IN, OUT = S.PERIODIC, S.NOSLIP, S.FREESLIP, S.INFLOW, S.OUTFLOW


def compatible_rhs(g, seed):
    rng = np.random.default_rng(seed)
    u = [torch.tensor(rng.uniform(-1, 1, size=g.shape(c))) for c in range(g.dim)]
    u = fluid.apply_boundary_values(g, u)
    if not g.periodic(0) and g.bc[0][1] == OUT:
        u = fluid.outflow_faces(g, u, u)
    return fluid.divergence(g, u)


CASES = [
    S.box_2d(32, 24, (P, P), (NS, NS), Lx=1.3, Ly=0.9, stretched=1.5),
    S.box_2d(40, 20, (IN, OUT), (FS, FS)),
    S.box_2d(15, 13, (NS, NS), (FS, FS), stretched=1.2),
    S.box_3d(16, 12, 8, (P, P), (NS, NS), L=(2.0, 2.0, 1.0), stretched=1.5),
    S.box_3d(12, 10, 8, (P, P), (P, P)),
]


@pytest.mark.parametrize("jacobi", [False, True])
@pytest.mark.parametrize("case", range(len(CASES)))
def test_cg_matches_direct_and_oracle(case, jacobi):
    from paper_2505_23940_b300 import grid_from_workload
    wl = CASES[case]
    g = grid_of(wl)
    b = compatible_rhs(g, 10 + case)
    pd = poisson.solve(g, b)
    _, it_o, _ = krylov.cg_solve(g, b, tol=1e-12, jacobi=jacobi)
    G = grid_from_workload(wl, "fp64")
    bd = b.cuda().contiguous()
    p, it, rel = G.solve_pressure_cg(bd, tol=1e-12, jacobi=jacobi)
    torch.cuda.synchronize()
    assert rel <= 1e-12
    err = float((p.cpu() - pd).abs().max()) / float(pd.abs().max())
    assert err < 1e-9, err
    # same algorithm, same iteration count (the GPU tests convergence every 8 iterations)
    assert it_o <= it < it_o + 8, (it, it_o)
    # and the GPU direct solver agrees
    pg = G.solve_pressure(bd)
    assert float((p - pg).abs().max()) < 1e-9 * float(pg.abs().max())


def test_cg_zero_rhs_and_mixed_grid():
    from paper_2505_23940_b300 import FsError, grid_from_workload
    wl = S.box_2d(8, 8, (P, P), (NS, NS))
    G = grid_from_workload(wl, "fp64")
    p, it, rel = G.solve_pressure_cg(torch.zeros((1, 8, 8), dtype=torch.float64, device="cuda"))
    assert it == 0 and float(p.abs().max()) == 0.0
    Gm = grid_from_workload(wl, "mixed")
    with pytest.raises(FsError):
        Gm.solve_pressure_cg(torch.zeros((1, 8, 8), dtype=torch.float64, device="cuda"))
