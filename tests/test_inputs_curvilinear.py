"""The seeded curved-grid generators (paper_2608_09615_b300/inputs.py) produce what the
library requires: periodic images one period vector away, positive Jacobians at the
solution points, proper rotations."""
import math

import numpy as np
import pytest

from oracle.curvilinear import CurvGrid
from paper_2608_09615_b300 import inputs

LO, HI = (0.0, -1.0, 0.5), (2.0, 1.5, 3.0)


@pytest.mark.parametrize("kind", ["uniform", "jitter", "wavy"])
def test_periodic_images(kind):
    ne = (4, 3, 5)
    N = {"uniform": lambda: inputs.periodic_lattice(ne, LO, HI),
         "jitter": lambda: inputs.jittered_lattice(ne, LO, HI, seed=3, amp=0.15),
         "wavy": lambda: inputs.wavy_lattice(ne, LO, HI, amp=0.15)}[kind]()
    assert N.shape == (3, ne[2] + 1, ne[1] + 1, ne[0] + 1)
    T = [np.array([HI[0] - LO[0], 0, 0]), np.array([0, HI[1] - LO[1], 0]), np.array([0, 0, HI[2] - LO[2]])]
    assert np.allclose(N[:, :, :, -1] - N[:, :, :, 0], T[0][:, None, None], atol=1e-14)
    assert np.allclose(N[:, :, -1, :] - N[:, :, 0, :], T[1][:, None, None], atol=1e-14)
    assert np.allclose(N[:, -1, :, :] - N[:, 0, :, :], T[2][:, None, None], atol=1e-14)


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("p", [1, 4])
def test_jittered_elements_valid(seed, p):
    ne = (5, 4, 3)
    g = CurvGrid(inputs.jittered_lattice(ne, LO, HI, seed=seed, amp=0.15), p)   # raises if J <= 0
    vol = (HI[0] - LO[0]) * (HI[1] - LO[1]) * (HI[2] - LO[2])
    assert abs(g.volume.sum() - vol) <= 1e-12 * vol


def test_rotation_matrix_is_a_rotation():
    R = inputs.rotation_matrix((1.0, -2.0, 0.5), 0.9)
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-15)
    assert abs(np.linalg.det(R) - 1.0) <= 1e-14
    a = np.array([1.0, -2.0, 0.5])
    assert np.allclose(R @ a, a)                       # the axis is fixed
    R2 = inputs.rotation_matrix((0.0, 0.0, 1.0), math.pi / 2)
    assert np.allclose(R2 @ np.array([1.0, 0, 0]), [0, 1.0, 0], atol=1e-15)


def test_curvilinear_coordinates_match_uniform_grid():
    ne, p = (3, 4, 2), 3
    X = inputs.curvilinear_coordinates(inputs.periodic_lattice(ne, LO, HI), p)
    Y = inputs.coordinates(3, ne, LO, HI, p)
    for a, b in zip(X, Y):
        assert np.allclose(a, b, atol=1e-14)
