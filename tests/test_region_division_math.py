"""The mathematics of the region statements' FP32 division, checked on the
host with C's correctly rounded fmaf (tests/region_division_math.c): the
two Newton corrections give RN(1/b) from any starting value within the
documented rcp.approx bound (every significand but the all-ones one, which
the division sends to its exact fallback), and the last FMA then gives
RN(a/b) (Markstein's theorem), on quotient midpoints and at random.  The GPU
tests check the same steps on the hardware's own rcp.approx values."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_division_steps_round_correctly_for_every_admissible_start(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    exe = str(tmp_path / "region_division_math")
    subprocess.run([cc, "-O2", "-ffp-contract=off", "-o", exe, os.path.join(HERE, "region_division_math.c"), "-lm"],
                   check=True)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("ok"), r.stdout
