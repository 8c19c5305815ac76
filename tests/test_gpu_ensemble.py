"""Batched ensemble: one CUDA-graph launch over members of uneven size reproduces the same
members stepped one by one, and matches the oracle on a member; autotuned launch
parameters leave results unchanged."""
import numpy as np
import pytest
import torch

import synthetic as S
from gpu_util import run_oracle
from helpers import rel_l2

pytestmark = pytest.mark.gpu


def test_graph_ensemble_matches_sequential_and_oracle():
    from paper_2505_23940_b300.ensemble import Ensemble
    wls = S.ensemble_cylinders(members=6, seed=5, precision="fp64", kmin=64, kmax=160)
    ens = Ensemble(wls, "fp64", streams=3)
    snap = ens.snapshot()
    ens.step_sequential(4)
    torch.cuda.synchronize()
    seq = [[x.clone() for x in m.u] for m in ens.members]
    ens.restore(snap)
    ens.capture(2)
    ens.restore(snap)
    ens.replay()
    ens.replay()
    torch.cuda.synchronize()
    for m, ref in zip(ens.members, seq):
        assert rel_l2([x.cpu() for x in m.u], [x.cpu() for x in ref]) < 1e-13
    st, _, _ = run_oracle(wls[0], 4)
    assert rel_l2([x.cpu() for x in ens.members[0].u], st.u) < 1e-11


def test_autotune_keeps_results(tmp_path, monkeypatch):
    from paper_2505_23940_b300 import autotune, grid_from_workload
    monkeypatch.setenv("FS_TUNE_CACHE", str(tmp_path / "tune.json"))
    wl = S.channel_3d(nx=32, ny=16, nz=16, steps=4)
    g = grid_from_workload(wl, "fp64")
    u0 = [torch.tensor(a, device="cuda") for a in wl.u0]
    ref = [x.clone() for x in u0]
    g.step(ref, wl.dt, 3)
    best = autotune.tune(g, u0, wl.dt)
    assert set(best) == set(autotune.CANDIDATES)
    out = [x.clone() for x in u0]
    g.step(out, wl.dt, 3)
    torch.cuda.synchronize()
    assert rel_l2([x.cpu() for x in out], [x.cpu() for x in ref]) < 1e-14
    assert autotune.tune(g, u0, wl.dt) == best     # served from the cache


def test_graph_ensemble_forward_adjoint_matches_rollouts_and_oracle():
    """Windowed forward + adjoint of an ensemble through two CUDA graphs (2 windows of 3 steps, members
    on parallel branches): dJ/du_0 of J = 1/2 sum_members sum u_T^2 h^2 equals the same sweep launched
    member by member, each member's FsRollout gradient, and the oracle's reverse-mode AD on a member."""
    import oracle as O
    from helpers import body_of, grid_of
    from paper_2505_23940_b300.autodiff import Rollout
    from paper_2505_23940_b300.ensemble import Ensemble
    wls = S.ensemble_cylinders(members=5, seed=6, precision="fp64", kmin=64, kmax=128)
    ens = Ensemble(wls, "fp64", streams=3)
    hs = [wl.xf[0][1] - wl.xf[0][0] for wl in wls]
    weights = [[torch.tensor(h * h, dtype=torch.float64, device="cuda")] * 2 for h in hs]
    ens.setup_adjoint(window=3, windows=2, weights=weights)
    ens.capture_windows()
    ens.fwd_adj_graph()
    torch.cuda.synchronize()
    graph = [[x.clone() for x in lu] for lu, _ in ens.lam_v]
    ens.fwd_adj_sequential()
    torch.cuda.synchronize()
    seq = [[x.clone() for x in lu] for lu, _ in ens.lam_v]
    for a, b in zip(graph, seq):
        assert rel_l2([x.cpu() for x in a], [x.cpu() for x in b]) < 1e-13
    for m, a, w in zip(ens.members, graph, weights):
        ro = Rollout(m.grid, m.dt, 6)
        u0 = [torch.tensor(np.asarray(x), dtype=torch.float64, device="cuda") for x in m.wl.u0]
        b0 = m.body.clone()
        uT, bT, _ = ro.forward(u0, b0)
        lam0, _ = ro.backward(u0, b0, [x * w[0] for x in uT], torch.zeros_like(bT))
        assert rel_l2([x.cpu() for x in a], [x.cpu() for x in lam0]) < 1e-12
    # the oracle's reverse-mode AD for member 0
    wl = wls[0]
    g = grid_of(wl)
    body, params = body_of(wl)
    u = [torch.tensor(np.asarray(x), dtype=torch.float64, requires_grad=True) for x in wl.u0]
    st = O.State(u, torch.tensor(wl.body.w0, dtype=torch.float64), torch.tensor(wl.body.wd0, dtype=torch.float64))
    for _ in range(6):
        st, _ = O.step(g, st, wl.dt, body=body, kernel=wl.kernel, params=params)
    J = sum(0.5 * (x * x).sum() for x in st.u) * hs[0] ** 2
    go = torch.autograd.grad(J, u)
    assert rel_l2([x.cpu() for x in graph[0]], list(go)) < 1e-11
