"""Values the paper prints, checked against the oracle's grid conventions (tests/golden/)."""
import json
import os

import numpy as np

import synthetic as S
from helpers import grid_of

HERE = os.path.dirname(os.path.abspath(__file__))


def test_channel_setup_table_wall_units():
    """Cell widths of the oracle grid in wall units reproduce the printed Delta x+, y+, z+
    (uniform grid of the stated cell counts on the stated domain, Re_tau = u_tau delta / nu)."""
    gd = json.load(open(os.path.join(HERE, "golden", "channel_re180_setup.json")))
    L, n, re = gd["domain"], gd["cells"], gd["re_tau"]
    wl = S.box_3d(n[0], n[1], n[2], (S.PERIODIC,) * 2, (S.NOSLIP,) * 2, L=tuple(L))
    g = grid_of(wl)
    got = {"dx_plus": float(g.h[0][0]) * re, "dy_plus": float(g.h[1][0]) * re, "dz_plus": float(g.h[2][0]) * re}
    for k, v in gd["printed_wall_units"].items():
        assert round(got[k], gd["printed_digits"][k]) == v, (k, got[k], v)
    # the time step of the channel workload is Delta t+ nu / u_tau^2 in outer units
    wl2 = S.channel_3d(nx=8, ny=8, nz=8)
    assert abs(wl2.dt * re - gd["dt_plus"]) < 1e-15
