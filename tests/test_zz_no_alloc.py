"""GPU test of fs_component_stats_noalloc, the entry point for callers that may not allocate
device memory (their memory belongs to another allocator, or an allocation's implicit
synchronisation is not allowed where they call).  It must agree with the grid-based
fs_diagnostics on the same fields, on two calls in a row (the fixed scratch keeps the
previous call's contents), and reject fields larger than its scratch.

This file is collected last so that a run stopping at the first failure has run every
other test first; it also passes on its own in a fresh process."""
import ctypes

import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu


def _stats(L, t, precision, vol, wy=None):
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    ext = (ctypes.c_int * 3)(t.shape[2], t.shape[1], t.shape[0])
    stream = torch.cuda.current_stream().cuda_stream
    rc = L.fs_component_stats_noalloc(ctypes.c_void_p(t.data_ptr()), precision, ext, ctypes.c_double(vol),
                                      ctypes.c_void_p(wy.data_ptr() if wy is not None else None),
                                      ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(stream))
    assert rc == 0, L.fs_last_error()
    torch.cuda.synchronize()
    return out.cpu()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_noalloc_stats_match_grid_diagnostics_two_calls(precision):
    from paper_2505_23940_b300 import FP64, MIXED, grid_from_workload, lib
    L = lib()
    wl = S.box_3d(32, 24, 16, (S.PERIODIC,) * 2, (S.NOSLIP,) * 2, L=(2.0, 2.0, 1.0), stretched=1.3)
    g = grid_from_workload(wl, precision)
    code = FP64 if precision == "fp64" else MIXED
    hx, hz = 2.0 / 32, 1.0 / 16
    hy = torch.tensor(np.diff(wl.xf[1]), dtype=torch.float64, device="cuda")
    yc = 0.5 * (wl.xf[1][:-1] + wl.xf[1][1:])
    hfy = np.empty(25)
    hfy[1:24] = np.diff(yc)
    hfy[0], hfy[24] = np.diff(wl.xf[1])[0], np.diff(wl.xf[1])[-1]
    hfy = torch.tensor(hfy, dtype=torch.float64, device="cuda")
    for call, seed in enumerate((11, 12)):
        u = [torch.tensor(a, dtype=g.dtype, device="cuda").contiguous()
             for a in S.random_fields(wl, seed, scale=1.0 + call)]
        ref = g.diagnostics(u)
        ke, um = 0.0, 0.0
        for c in range(3):
            wy = hfy if c == 1 else hy
            o = _stats(L, u[c], code, hx * hz, wy)
            ke += float(o[0])
            um = max(um, float(o[1]))
        assert abs(ke - ref["ke"]) <= 1e-12 * ref["ke"], (call, ke, ref["ke"])
        assert um == ref["umax"], (call, um, ref["umax"])


def test_noalloc_exact_capacity_without_weights_matches_host_sum():
    """A field of exactly 33,554,432 FP32 elements fills all 4096 scratch slots; with wy = NULL every
    element has weight vol.  Checked against an FP64 sum and max taken on the host, twice in a row."""
    from paper_2505_23940_b300 import MIXED, lib
    L = lib()
    for seed in (21, 22):
        gen = torch.Generator().manual_seed(seed)
        host = torch.rand((2, 4096, 4096), generator=gen, dtype=torch.float64).mul_(2.0).sub_(1.0).float()
        t = host.to("cuda")
        o = _stats(L, t, MIXED, 0.25)
        h64 = host.double()
        ke = float((0.5 * h64 * h64).sum()) * 0.25
        assert abs(float(o[0]) - ke) <= 1e-12 * ke, (seed, float(o[0]), ke)
        assert float(o[1]) == float(h64.abs().max())
        del t


def test_noalloc_rejects_fields_beyond_its_scratch():
    from paper_2505_23940_b300 import FP64, lib
    L = lib()
    t = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    ext = (ctypes.c_int * 3)(4096, 4096, 3)          # 50,331,648 elements > 33,554,432
    rc = L.fs_component_stats_noalloc(ctypes.c_void_p(t.data_ptr()), FP64, ext, ctypes.c_double(1.0), None,
                                      ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -1
    assert b"33554432" in L.fs_last_error()
    ext = (ctypes.c_int * 3)(2 ** 30, 2 ** 30, 2 ** 30)   # the product overflows 64 bits without the stepwise check
    rc = L.fs_component_stats_noalloc(ctypes.c_void_p(t.data_ptr()), FP64, ext, ctypes.c_double(1.0), None,
                                      ctypes.c_void_p(out.data_ptr()), None)
    assert rc == -1
