"""Pins of the comparison measures the parity tests use.

The factor-match score is not part of the method, but every parity claim on
factors goes through it, so it is checked against values fixed by geometry:
a model compared with itself scores 1; the score ignores column order and
column scales (signs included); with orthonormal columns and one column of
one mode turned by an angle theta in a plane orthogonal to all other
columns, only one matched product changes, to cos(theta), so the score is
(R - 1 + cos theta) / R.  Both matching branches are exercised: brute force
(R <= 8) and the assignment solver (R > 8).
"""
import math

import numpy as np
import pytest

from tests._metrics import fms, rel_fro


def _orthonormal(n, R, seed):
    q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, R)))
    return q


@pytest.mark.parametrize("R", [3, 8, 10])
def test_fms_of_a_model_with_itself_is_one(R):
    rng = np.random.default_rng(R)
    model = tuple(rng.standard_normal((n, R)) for n in (12, 11, 13))
    assert fms(model, model) == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("R", [4, 8, 10])
def test_fms_ignores_column_order_and_scales(R):
    rng = np.random.default_rng(100 + R)
    ref = tuple(rng.standard_normal((n, R)) for n in (14, 15, 16))
    perm = rng.permutation(R)
    model = []
    for F in ref:
        s = rng.uniform(0.2, 5.0, R) * rng.choice([-1.0, 1.0], R)
        model.append(F[:, perm] * s)
    assert fms(tuple(model), ref) == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("R,theta", [(3, 0.3), (8, 1.1), (10, 0.7), (10, math.pi / 2)])
def test_fms_turned_column_closed_form(R, theta):
    n = R + 2
    A, B, C = (_orthonormal(n, R + 1, s) for s in (1, 2, 3))
    ref = (A[:, :R], B[:, :R], C[:, :R])
    At = ref[0].copy()
    # column 0 turned towards the (R+1)-th orthonormal direction, orthogonal to
    # every column of the reference
    At[:, 0] = math.cos(theta) * A[:, 0] + math.sin(theta) * A[:, R]
    got = fms((At, ref[1], ref[2]), ref)
    assert got == pytest.approx((R - 1 + abs(math.cos(theta))) / R, abs=1e-12)


def test_fms_takes_the_best_matching_not_the_identity():
    # two columns swapped in every mode: the identity pairing scores 0 on
    # them, the best pairing 1
    A, B, C = (_orthonormal(9, 4, s) for s in (4, 5, 6))
    swap = [1, 0, 2, 3]
    assert fms((A[:, swap], B[:, swap], C[:, swap]), (A, B, C)) == pytest.approx(1.0, abs=1e-12)


def test_rel_fro_values():
    ref = np.array([3.0, 4.0])
    assert rel_fro(ref, ref) == 0.0
    assert rel_fro(np.zeros(2), ref) == pytest.approx(1.0)
    assert rel_fro(np.array([3.0, 4.5]), ref) == pytest.approx(0.1)
    assert rel_fro(np.array([1.0, 0.0]), np.zeros(2)) == pytest.approx(1.0)
