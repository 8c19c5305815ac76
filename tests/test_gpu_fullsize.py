"""Parity at the full workload sizes, in the configuration the benchmark times (mixed precision),
against the oracle over a few steps (the oracle finishes these in seconds to a minute)."""
import pytest

import synthetic as S
from gpu_util import field_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu


def test_isotropic_128_mixed_full_size():
    wl = S.isotropic_3d(n=128)
    gp = run_gpu(wl, 2, precision="mixed")
    st, _, _ = run_oracle(wl, 2)
    assert field_err(gp["u"], st.u) < 1e-5


def test_isotropic_128_mixed_fp64_y_full_size():
    """The benchmark's step: FP32 stencils and x/z transforms, the periodic y part of the
    Poisson solve as the FP64 cyclic tridiagonal (twisted factorisation, tensor-map tiles)."""
    wl = S.isotropic_3d(n=128)
    gp = run_gpu(wl, 2, precision="mixed", tuning=[("y_spectral", 0)])
    assert gp["grid"].device_status() == 0
    st, _, _ = run_oracle(wl, 2)
    assert field_err(gp["u"], st.u) < 1e-5


def test_channel_192x128x128_mixed_full_size():
    wl = S.channel_3d()
    gp = run_gpu(wl, 2, precision="mixed")
    st, _, _ = run_oracle(wl, 2)
    assert field_err(gp["u"], st.u) < 1e-5


def test_cylinder_640x320_fp64_and_mixed_full_size():
    wl = S.cylinder_2d(seed=2, perturb=0.01)
    wl.body.w0 = (0.0, 0.1)
    st, dg, _ = run_oracle(wl, 2)
    g64 = run_gpu(wl, 2, precision="fp64")
    assert field_err(g64["u"], st.u) < 1e-11
    assert abs(g64["F"][0][0] - float(dg.F[0])) < 1e-9 * abs(float(dg.F[0]))
    gm = run_gpu(wl, 2, precision="mixed")
    assert field_err(gm["u"], st.u) < 1e-5
