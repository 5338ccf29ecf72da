"""The bounds-checked build (libcasim_checked.so, -DCASIM_CHECKED), the
stand-in for a memory checker: small cases agree with the oracle and end with
status 0 (no gather index out of range), and an out-of-range index planted
on the device ends the step with CASIM_E_BOUNDS without any out-of-range
access, after which the context runs normally."""
import json
import os
import subprocess
import sys

import pytest

from paper_2203_02054_gb300 import build as casim_build
from paper_2203_02054_gb300 import casim

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def results():
    if not os.path.exists(casim.LIB_CHECKED_PATH):
        casim_build.build()
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_runner.py")], capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_library_is_loaded(results):
    assert results["checked"] == 1


def test_checked_runs_equal_the_oracle_without_bound_errors(results):
    assert results["fp64_status"] == 0 and results["fp64_err"] <= 1e-9 and results["fp64_springs"]
    assert results["mixed_status"] in (0, casim.CASIM_W_PCG_MAXIT)
    assert results["mixed_pairs_equal"] and results["mixed_err"] <= 1e-5
    assert results["gripper_status"] == 0 and results["gripper_finite"]
    assert results["batch_status"] == 0


def test_planted_out_of_range_index_is_reported(results):
    assert results["corrupt_status"] == casim.CASIM_E_BOUNDS
    assert results["corrupt_bits"] & 64
    assert results["after_status"] == 0
