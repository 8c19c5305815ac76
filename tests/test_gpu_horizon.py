"""Parity over 100 steps at the full workload sizes, in the configurations the benchmark times:
every GPU field against the FP64 oracle after the whole horizon, within 1e-5 relative L2 for the
mixed-precision (FP32 stencil) runs and 1e-11 for FP64 runs.  The oracle takes about 0.2 s per
128^3 RK3 step on the host cores, so each case costs tens of seconds of oracle time."""
import pytest
import torch

import synthetic as S
from gpu_util import field_err, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

STEPS = 100


def test_isotropic_128_mixed_fp64_y_100_steps():
    """The benchmark's step (FP32 stencils and x/z transforms, periodic y as the FP64 cyclic
    tridiagonal solve, SSP-RK3 at CFL 0.5) over 100 steps."""
    wl = S.isotropic_3d(n=128)
    gp = run_gpu(wl, STEPS, precision="mixed", tuning=[("y_spectral", 0)])
    assert gp["grid"].device_status() == 0
    st, _, _ = run_oracle(wl, STEPS)
    err = field_err(gp["u"], st.u)
    print("isotropic 128^3 mixed, FP64 y, %d steps: rel L2 %.3e" % (STEPS, err))
    assert err < 1e-5


def test_isotropic_128_fp64_10_steps():
    wl = S.isotropic_3d(n=128)
    gp = run_gpu(wl, 10, precision="fp64")
    st, _, _ = run_oracle(wl, 10)
    err = field_err(gp["u"], st.u)
    print("isotropic 128^3 FP64, 10 steps: rel L2 %.3e" % err)
    assert err < 1e-11


def test_channel_192x129x128_mixed_100_steps():
    wl = S.channel_3d()
    gp = run_gpu(wl, STEPS, precision="mixed")
    assert gp["grid"].device_status() == 0
    st, _, _ = run_oracle(wl, STEPS)
    err = field_err(gp["u"], st.u)
    print("channel 192x129x128 mixed, %d steps: rel L2 %.3e" % (STEPS, err))
    assert err < 1e-5


def test_cylinder_640x320_100_steps_fields_and_body():
    """The FSI workload (Roma-3 kernel, 126 markers, elastically mounted, released from w_y = 0.1)
    over 100 steps: fields and the body state (displacement, velocity) in FP64 and mixed precision."""
    wl = S.cylinder_2d(seed=2, perturb=0.01)
    wl.body.w0 = (0.0, 0.1)
    st, dg, _ = run_oracle(wl, STEPS)
    ob = torch.cat([st.w, st.wd])
    for precision, tol in (("fp64", 1e-11), ("mixed", 1e-5)):
        gp = run_gpu(wl, STEPS, precision=precision)
        err = field_err(gp["u"], st.u)
        berr = float((gp["body"] - ob).norm() / ob.norm())
        ferr = abs(gp["F"][0][1] - float(dg.F[1])) / abs(float(dg.F[1]))
        print("cylinder 640x320 %s, %d steps: fields %.3e, body %.3e, lift %.3e" % (precision, STEPS, err, berr, ferr))
        assert err < tol
        assert berr < tol
