"""Host check of the y solve's integer-pipe FP32 <-> FP64 conversions
(csrc/fpconv.cuh): every binary32 value widened and binary64 values across every
exponent, with rounding ties, narrowed, bit-compared with the host's IEEE 754
conversions (round to nearest even)."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2505_23940_b300", "csrc")


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_fp32_fp64_conversions_match_ieee(tmp_path):
    exe = str(tmp_path / "fpconv_check")
    subprocess.check_call(["gcc", "-O2", "-I", CSRC, "-o", exe, os.path.join(HERE, "fpconv_check.c"), "-lm"])
    out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout
    assert out.stdout.strip() == "ok"
