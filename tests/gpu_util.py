"""Helpers of the GPU parity tests: run a workload through the C ABI and through the oracle."""
import numpy as np
import torch

import oracle as O
from helpers import body_of, grid_of, rel_l2


def run_gpu(wl, steps, dt=None, precision="fp64", u0=None, want_p=False, tuning=()):
    from paper_2505_23940_b300 import body_tensor, grid_from_workload
    g = grid_from_workload(wl, precision)
    for key, value in tuning:
        g.set_tuning(key, value)
    u = [torch.tensor(np.asarray(a), dtype=g.dtype, device="cuda").contiguous() for a in (u0 or wl.u0)]
    body = body_tensor(wl)
    p = torch.zeros(g.shape(-1), dtype=torch.float64, device="cuda") if want_p else None
    g.step(u, wl.dt if dt is None else dt, steps, p=p, body=body)
    torch.cuda.synchronize()
    out = {"u": [x.double().cpu() for x in u], "grid": g, "u_dev": u}
    if body is not None:
        out["body"] = body.cpu()
        out["F"] = g.forces()
    if want_p:
        out["p"] = p.cpu()
    return out


def run_oracle(wl, steps, dt=None, u0=None):
    g = grid_of(wl)
    body, params = body_of(wl)
    u = [torch.tensor(np.asarray(a), dtype=torch.float64) for a in (u0 or wl.u0)]
    if wl.body is not None:
        st = O.State(u, torch.tensor(wl.body.w0, dtype=torch.float64), torch.tensor(wl.body.wd0, dtype=torch.float64))
    else:
        st = O.State(u)
    dg = None
    for _ in range(steps):
        st, dg = O.step(g, st, wl.dt if dt is None else dt, scheme=wl.scheme, body=body, kernel=wl.kernel,
                        params=params)
    return st, dg, g


def field_err(a, b):
    return rel_l2(a, b)
