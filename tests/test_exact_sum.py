"""The FP32 mass accumulator (paper_1107_2157_gb300/csrc/swe_exact_sum.h,
compiled here for the host from the same header the mass kernel includes)
against the exactly rounded sum of its inputs (math.fsum).

Values whose exponents lie within 5 binades of the first, largest one reach
the integer accumulator exactly and the result is the exact sum itself;
otherwise only the few FP64 additions of flushed parts and of small values
round, so the result stays within a few units in the last place."""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1107_2157_gb300", "csrc")


@pytest.fixture(scope="module")
def exe(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    out = str(tmp_path_factory.mktemp("exact_sum") / "exact_sum_host")
    subprocess.run([cxx, "-O2", "-std=c++17", "-I", CSRC, "-o", out, os.path.join(HERE, "exact_sum_host.cpp")],
                   check=True)
    return out


def _sum(exe, x, tmp_path):
    p = tmp_path / "x.bin"
    np.asarray(x, np.float32).tofile(p)
    r = subprocess.run([exe, str(p)], capture_output=True, text=True, check=True)
    return float.fromhex(r.stdout.strip())


def _ulp(v):
    return math.ulp(abs(v)) if v != 0 else 5e-324


def test_depths_of_one_binade_sum_exactly(exe, tmp_path):
    rng = np.random.default_rng(1)
    x = (1.0 + 0.9 * rng.random(1_000_003)).astype(np.float32)
    assert _sum(exe, x, tmp_path) == math.fsum(x.astype(np.float64))


def test_mixed_binades_after_the_largest_sum_exactly(exe, tmp_path):
    rng = np.random.default_rng(2)
    x = np.concatenate([[3.5], 0.15 + 3.0 * rng.random(100_001)]).astype(np.float32)
    assert np.log2(x.max()) - np.log2(x.min()) < 5
    assert _sum(exe, x, tmp_path) == math.fsum(x.astype(np.float64))


@pytest.mark.parametrize("case", ["rising", "wide", "signs", "tiny", "subnormal", "zeros", "huge"])
def test_general_inputs_within_a_few_ulps(exe, tmp_path, case):
    rng = np.random.default_rng(hash(case) % 2**32)
    n = 50_001
    if case == "rising":      # every new maximum flushes
        x = np.sort(0.01 + 100 * rng.random(n))
    elif case == "wide":      # 40 binades, values far below the reference go to FP64
        x = 2.0 ** rng.uniform(-20, 20, n)
    elif case == "signs":
        x = rng.standard_normal(n) * 2.0 ** rng.uniform(-3, 3, n)
    elif case == "tiny":
        x = np.concatenate([[1.0], 1e-9 * rng.random(n)])
    elif case == "subnormal":
        x = rng.random(n) * 1e-39
    elif case == "zeros":
        x = np.where(rng.random(n) < 0.5, 0.0, 1.0 + rng.random(n))
        x[::7] = -0.0
    else:
        x = (1e38 * rng.random(n)).astype(np.float32)
    x = np.asarray(x, np.float32)
    got = _sum(exe, x, tmp_path)
    want = math.fsum(x.astype(np.float64))
    assert abs(got - want) <= 4 * _ulp(want), (case, got, want)


def test_non_finite_values_propagate(exe, tmp_path):
    x = np.ones(11, np.float32)
    x[5] = np.inf
    assert _sum(exe, x, tmp_path) == np.inf
    x[6] = -np.inf
    assert math.isnan(_sum(exe, x, tmp_path))
    y = np.ones(9, np.float32)
    y[8] = np.nan
    assert math.isnan(_sum(exe, y, tmp_path))

