"""The oracle against the numbers the paper prints (tests/golden/
paper_printed_values.txt, each line citing where the paper prints it)."""
import math
import os

import numpy as np
import pytest

import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_printed_values.txt")


def _golden():
    out = {}
    with open(GOLDEN) as fh:
        for line in fh:
            if not line.strip() or line.startswith("#"):
                continue
            name, value, tol, where, what = (s.strip() for s in line.split("|"))
            out[name] = (float(value), float(tol), where)
    return out


G = _golden()


def test_golden_file_lists_every_pin():
    assert set(G) == {"a_proposal", "S_low_coef", "S_high_coef", "F_norm",
                      "omega_c_circular"}


def test_proposal_constant_a_as_printed():
    v, tol, _ = G["a_proposal"]
    assert abs(O.const_a() - v) <= tol


@pytest.mark.parametrize("x", [1e-9, 1e-3, 0.1, 0.5, 0.69])
def test_proposal_low_branch_as_printed(x):
    v, tol, _ = G["S_low_coef"]
    assert O.S(x) == pytest.approx(v * x ** (1.0 / 3.0), rel=tol * 10)


@pytest.mark.parametrize("x", [0.7, 1.0, 3.0, 20.0])
def test_proposal_high_branch_as_printed(x):
    v, tol, _ = G["S_high_coef"]
    assert O.S(x) == pytest.approx(v * math.exp(-x), rel=tol * 10)


def test_spectrum_normalisation_as_printed():
    v, tol, _ = G["F_norm"]
    total = (9.0 * math.sqrt(3.0) / (8.0 * math.pi)) * O.int_F(np.inf)
    assert abs(total - v) <= tol


@pytest.mark.parametrize("gamma", [10.0, 1000.0, 3.0e4])
def test_omega_c_of_circular_motion_as_printed(gamma):
    """A particle moving perpendicular to a pure B (normalised units, c = 1,
    B in units of the non-relativistic gyro-frequency): the gyro-radius is
    rho = gamma beta / B.  The caption's omega_c = (3/2)(c/rho) gamma^3 is the
    ultra-relativistic form; the oracle's omega_c = (3/2) Omega gamma^2 with
    Omega = |beta x B| from the effective field equals it times beta^2, i.e.
    to O(1/gamma^2)."""
    v, tol, _ = G["omega_c_circular"]
    B = 2.5
    beta = math.sqrt(1.0 - 1.0 / gamma ** 2)
    H = O.heff_field([0.0, 0.0, 0.0], [0.0, 0.0, B], [beta, 0.0, 0.0])
    omega_c = 1.5 * H * gamma ** 2
    rho = gamma * beta / B
    printed = v * (1.0 / rho) * gamma ** 3
    assert omega_c / printed == pytest.approx(beta ** 2, rel=max(tol, 1e-12))
    assert abs(omega_c / printed - 1.0) <= 1.0 / gamma ** 2 * (1 + 1e-9)
