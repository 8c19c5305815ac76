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
