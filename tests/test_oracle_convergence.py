"""The oracle's periodic Cahn-Hilliard scheme against the convergence study the
paper prints (section 5.2, Table 3; `tests/golden/paper_table3.json`): gamma = 0.01,
L = 2 pi, dt = 0.1 dx, C(x, 0) = 1e-6 cos(5 x), run to T = 20 on N = 64, 128 and
256 points.  The errors E_128 and E_256 and the order log2(E_128 / E_256) must equal
the printed values to the printed digits.  These numbers come from the paper, not
from this library, so they pin the whole step (matrix, right-hand side, cyclic
solve) at once: a wrong sign, a dropped term or a wrong corner moves them."""
import json
import math
import os

import numpy as np
import pytest

import synth
from oracle import matrices, steppers

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_table3.json")


def half_unit(v):
    """Half a unit in the last printed digit of a value printed with 3 significant
    digits (0.0310, 0.0022 and 5.45e-4 are printed this way, 0.0022 with 2)."""
    return 0.5 * 10.0 ** (math.floor(math.log10(abs(v))) - 2)


def run_oracle(N):
    gamma, dt, steps, _, C = synth.ch_convergence_case(N)
    A = steppers.SharedPentaPeriodic(*matrices.ch_matrix_periodic(N, dt * gamma))
    for _ in range(steps):
        C = steppers.ch_step_periodic(A, C, dt)
    return C[:, 0]


@pytest.fixture(scope="module")
def runs():
    return {N: run_oracle(N) for N in (64, 128, 256)}


def test_table3_errors_and_order(runs):
    rows = {int(r[0]): r for r in json.load(open(GOLDEN))["rows"]}
    E128 = steppers.convergence_error(runs[64], runs[128])
    E256 = steppers.convergence_error(runs[128], runs[256])
    assert abs(E128 - rows[128][1]) <= half_unit(rows[128][1]), E128
    assert abs(E256 - rows[256][1]) <= 0.5e-4, E256      # printed 0.0022
    assert abs(math.log2(E128 / E256) - rows[128][2]) <= 0.5e-4, math.log2(E128 / E256)


def test_runs_reach_the_steady_five_domain_state(runs):
    """By T = 20 the small cosine has grown into five domains near +-0.95 and
    stopped moving (the time error of a fixed point is zero, so the differences
    above are spatial)."""
    for N, C in runs.items():
        assert 0.94 < np.max(C) < 0.97 and -0.97 < np.min(C) < -0.94, (N, np.max(C), np.min(C))
        assert abs(np.mean(C)) <= 1e-10  # mean conserved up to roundoff over 8149 steps
        crossings = np.count_nonzero(np.sign(C) != np.sign(np.roll(C, 1)))
        assert crossings == 10, (N, crossings)


def test_convergence_error_definition():
    fine = np.arange(8.0)
    half = fine[::2] + np.array([1.0, -1.0, 0.5, 0.0])
    assert steppers.convergence_error(half, fine) == pytest.approx(2.5 / 4)
