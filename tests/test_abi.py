"""CPU checks of the C ABI: the library builds, loads, exports every declared symbol, and
rejects invalid grid descriptions on the host before touching a device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2505_23940_b300 import build
    build.build()
    from paper_2505_23940_b300 import fsstep
    return fsstep.lib()


def declared():
    src = open(os.path.join(ROOT, "include", "fs.h")).read()
    return sorted(set(re.findall(r"\b(fs_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary_calls():
    names = declared()
    for required in ("fs_create_grid", "fs_set_ib_markers", "fs_step", "fs_step_adjoint", "fs_solve_pressure",
                     "fs_forces", "fs_destroy_grid", "fs_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol(L):
    for name in declared():
        assert hasattr(L, name), name


def _desc(fsstep, dim=2, n=(8, 8, 1), bc=None, xf=None, bad_dim=None):
    d = fsstep.GridDesc()
    d.dim = dim
    for i in range(3):
        d.n[i] = n[i]
    keep = []
    for i in range(dim):
        a = np.ascontiguousarray(xf[i] if xf else np.linspace(0, 1, n[i] + 1))
        keep.append(a)
        d.xf[i] = a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    bc = bc or [(0, 0)] * 3
    for i in range(3):
        for s in range(2):
            d.bc[i][s] = bc[i][s] if i < len(bc) else 0
    d.nu, d.rho = 0.01, 1.0
    if bad_dim is not None:
        d.dim = bad_dim
    return d, keep


@pytest.mark.parametrize("case,code", [
    (dict(bad_dim=4), -1),
    (dict(n=(1, 8, 1)), -1),
    (dict(bc=[(0, 1), (0, 0)]), -1),                      # periodic on one side only
    (dict(bc=[(4, 3), (2, 2)]), -1),                      # outflow at x-low
    (dict(bc=[(0, 0), (3, 4)]), -1),                      # inflow in y
    (dict(n=(7, 8, 1)), -1),                              # odd periodic transform length
    (dict(n=(34, 8, 1)), -5),                             # prime factor 17
    (dict(xf=[np.linspace(0, 1, 9) ** 2, np.linspace(0, 1, 9)]), -1),   # stretched x
])
def test_invalid_descriptions_rejected_on_host(L, case, code):
    from paper_2505_23940_b300 import fsstep
    d, keep = _desc(fsstep, **case)
    h = ctypes.c_void_p()
    rc = L.fs_create_grid(ctypes.byref(d), None, ctypes.byref(h))
    assert rc == code
    assert len(L.fs_last_error()) > 0
    assert not h.value


def test_null_arguments(L):
    assert L.fs_create_grid(None, None, None) == -1
    assert L.fs_step(None, None, ctypes.c_double(0.1), 1) == -1
    assert L.fs_destroy_grid(None) == 0
