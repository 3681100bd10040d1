"""The identity behind the FP32 step kernels' packed unfused products
(mul2_nf): fma(a, b, -0) is the rounded product a*b bit for bit, zeros
keeping their sign, checked on the host with C's correctly rounded fmaf
(tests/fma_negzero.c) on special values and 2^24 random pairs.  The GPU
tests check the kernels built on it bit for bit against the scalar
kernels, whose products are plain rounded multiplies."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_fma_with_negative_zero_addend_is_the_rounded_product(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "fma_negzero")
    subprocess.run([cc, "-O2", "-ffp-contract=off", "-o", exe, os.path.join(HERE, "fma_negzero.c"), "-lm"],
                   check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout
