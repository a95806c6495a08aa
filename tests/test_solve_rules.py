"""CPU tests of the restart loop's stopping and precision-switch rules (the
paper states none; the readings are in csrc/solve_rules.h): the host header
is compiled with g++ into a small driver that replays per-iteration counts."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NONE = 1e300          # "no unconverged in-window pair"


@pytest.fixture(scope="module")
def driver(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    exe = str(tmp_path_factory.mktemp("rules") / "solve_rules_driver")
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", os.path.join(ROOT, "paper_1803_02156_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "native", "solve_rules_driver.cpp"), "-o", exe], check=True)
    return exe


def run(driver, mixed, n_t, its):
    """its: per iteration (c, cl, m, ml); returns [(iteration, low, done)]."""
    args = [driver, str(int(mixed)), str(n_t)]
    for c, cl, m, ml in its:
        args += [str(c), str(cl), repr(float(m)), repr(float(ml))]
    out = subprocess.run(args, capture_output=True, text=True, check=True).stdout.split("\n")
    return [tuple(int(v) for v in line.split()) for line in out if line.strip()]


def test_fp64_stops_at_target_count(driver):
    r = run(driver, False, 4, [(0, 0, 1e-3, 1e-3), (2, 3, 1e-9, 1e-5), (4, 6, NONE, NONE), (6, 6, NONE, NONE)])
    assert r[-1] == (3, 0, 1)


def test_fp64_stops_when_count_stable_and_nothing_converging(driver):
    # the window holds 3 states: the count stays 3, the other in-window Ritz
    # values are spurious and their residual no longer halves
    its = [(3, 3, 1e-3, 1e-3), (3, 3, 0.9e-3, 0.9e-3), (3, 3, 0.8e-3, 0.8e-3), (3, 3, 0.8e-3, 0.8e-3)]
    assert run(driver, False, 10, its)[-1] == (3, 0, 1)


def test_fp64_waits_while_a_pair_still_converges(driver):
    its = [(3, 3, 1e-3, 1e-3), (3, 3, 1e-5, 1e-5), (3, 4, 1e-7, 1e-7), (3, 4, 0.9e-7, 0.9e-7),
           (3, 4, 0.8e-7, 0.8e-7), (3, 4, 0.8e-7, 0.8e-7)]
    r = run(driver, False, 10, its)
    assert r[-1][2] == 1 and r[-1][0] == 5       # not at 3 (the residual still halves), at 5
    assert run(driver, False, 10, its[:3])[-1][2] == 0


def test_no_target_stops_only_on_stable_count(driver):
    its = [(1, 1, 1e-2, 1e-2), (5, 5, 1e-3, 1e-3), (5, 5, 0.9e-3, 0.9e-3), (5, 5, 0.9e-3, 0.9e-3)]
    assert run(driver, False, 0, its)[-1] == (4, 0, 1)


def test_mixed_switches_at_target_count_then_stops_in_fp64(driver):
    its = [(0, 1, 1e-2, 1e-2), (0, 3, 1e-3, 1e-3), (0, 4, 1e-4, 1e-5),    # fp32 phase: 4 at switch_tol
           (2, 4, 1e-8, NONE), (4, 4, NONE, NONE)]
    r = run(driver, True, 4, its)
    assert [x[1] for x in r] == [1, 1, 1, 0, 0]       # three fp32 iterations, then fp64
    assert r[-1] == (5, 0, 1)


def test_mixed_switches_when_fp32_stalls_and_fp64_confirms(driver):
    # fp32 stalls at 2 pairs below switch_tol (count flat, residual not halving)
    its = [(0, 2, 1e-3, 1e-3), (0, 2, 0.9e-3, 0.9e-3),
           # one fp64 sweep: the 2 pairs reach tol and the rest do not improve
           (2, 2, 0.9e-3, 0.9e-3)]
    r = run(driver, True, 8, its)
    assert [x[1] for x in r] == [1, 1, 0]
    assert r[-1] == (3, 0, 1)


def test_mixed_keeps_going_while_fp64_still_improves(driver):
    its = [(0, 2, 1e-3, 1e-3), (0, 2, 0.9e-3, 0.9e-3), (2, 2, 1e-4, 1e-4), (3, 3, 1e-6, 1e-6)]
    r = run(driver, True, 8, its)
    assert all(x[2] == 0 for x in r)
