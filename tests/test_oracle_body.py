"""Pins of the rigid-body RK4 (Eq. 12): closed-form free vibration and static offset."""
import math

import torch

from oracle.body import RigidParams, rk4


def _run(dt, T, F=0.0, y0=0.1, k=2.4805, m=math.pi / 2, c=0.0):
    p = RigidParams(m, k, c, (False, True))
    w = torch.tensor([0.0, y0], dtype=torch.float64)
    wd = torch.zeros(2, dtype=torch.float64)
    Ft = torch.tensor([0.0, F], dtype=torch.float64)
    for _ in range(int(round(T / dt))):
        w, wd = rk4(p, w, wd, Ft, dt)
    return w, wd


def test_free_vibration_fourth_order():
    k, m = 2.4805, math.pi / 2
    om = math.sqrt(k / m)
    T = 4.3  # away from an extremum of cos, where the phase error would vanish
    errs = []
    for dt in (0.1, 0.05, 0.025):
        w, _ = _run(dt, T)
        errs.append(abs(float(w[1]) - 0.1 * math.cos(om * T)))
    assert 14.0 < errs[0] / errs[1] < 18.0 and 14.0 < errs[1] / errs[2] < 18.0


def test_static_offset_under_constant_force():
    k, m, c = 2.0, 1.0, 1.5
    w, wd = _run(0.01, 60.0, F=0.6, y0=0.0, k=k, m=m, c=c)
    assert abs(float(w[1]) - 0.6 / k) < 1e-10 and abs(float(wd[1])) < 1e-10


def test_inactive_dof_stays_at_rest():
    w, wd = _run(0.01, 1.0, F=1.0)
    assert float(w[0]) == 0.0 and float(wd[0]) == 0.0


def test_reduced_parameters():
    p = RigidParams.from_reduced(2.0, 5.0, 1.0, 1.0)
    assert abs(p.m - math.pi / 2) < 1e-15
    assert abs(float(p.k) - 0.08 * math.pi ** 3) < 1e-12
