"""Pins of the oracle's grid, stencil and index sets (Sec. 2, eq:25, App. A)."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle.lattice import STENCILS, Box, n_gamma

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.mark.parametrize("R", [1, 2, 3, 4])
def test_stencil_moments(R):
    """A (2R+1)-point central second difference is exact on x^p, p <= 2R+1:
    sum_m c_m m^p = 2 delta_{p,2} (m from -R to R)."""
    c = STENCILS[R]
    for p in range(0, 2 * R + 2):
        tot = Fraction(0)
        for m in range(-R, R + 1):
            tot += c[abs(m)] * Fraction(m) ** p
        assert tot == (2 if p == 2 else 0), (R, p, tot)


def test_five_point_matches_paper():
    g = GOLDEN["five_point_over_12"]
    c = STENCILS[2]
    printed = [Fraction(v, g["denominator"]) for v in g["coefficients"]]
    assert printed == [c[2], c[1], c[0], c[1], c[2]]


def test_paper_gamma_count():
    """Sec. 4.2: 31^3 interior, 7-point per axis (R = 3) -> 14166 boundary nodes."""
    for e in GOLDEN["n_gamma"]:
        box = Box(tuple(e["dims"]), 0.1, e["R"])
        assert len(box.gamma()) == e["value"]
        assert n_gamma(e["dims"], e["R"]) == e["value"]


def test_gamma_counts_r1():
    assert n_gamma((96, 96, 96), 1) == 54152
    assert n_gamma((64, 64, 64), 1) == 23816
    for dims in [(4, 5, 6), (7, 3, 4), (16, 16, 16)]:
        box = Box(dims, 0.5)
        assert len(box.gamma()) == n_gamma(dims, 1)


@pytest.mark.parametrize("dims", [(5, 6, 7), (4, 4, 4), (9,), (4, 6)])
def test_sigma_structure_r1(dims):
    """With the 3-point stencil every Sigma node touches exactly one Gamma node, a
    Gamma node touches 1..d exterior nodes, and |Sigma| = 2 sum_k prod_{j!=k} N_j."""
    box = Box(dims, 0.7)
    S, HGS = box.sigma()
    assert HGS.shape == (len(box.gamma()), len(S))
    assert np.all((HGS != 0).sum(axis=0) == 1)
    assert np.allclose(HGS[HGS != 0], -0.5 / 0.7 ** 2)
    cnt = (HGS != 0).sum(axis=1)
    assert cnt.min() >= 1 and cnt.max() <= box.d
    expect = 2 * sum(int(np.prod([n for j, n in enumerate(dims) if j != k])) for k in range(len(dims)))
    assert len(S) == expect
    # corners have d exterior neighbours
    assert (cnt == box.d).sum() == 2 ** box.d


def test_hamiltonian_symmetric_and_laplacian():
    """H_{I,I} is real symmetric; on a quadratic far from the faces the kinetic part
    returns -1/2 * Laplacian exactly."""
    box = Box((7, 6, 8), 0.3)
    Hk = box.H_II_kinetic()
    assert abs(Hk - Hk.T).max() == 0
    C = box.coords() * box.h
    f = C[:, 0] ** 2 + 2 * C[:, 1] ** 2 - C[:, 2] ** 2 + C[:, 0] * C[:, 2]
    Hf = Hk @ f
    inner = np.all((box.coords() > 0) & (box.coords() < np.array(box.dims) - 1), axis=1)
    assert np.allclose(Hf[inner], -0.5 * (2 + 4 - 2), atol=1e-10)
