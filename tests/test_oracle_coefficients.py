"""Pins of the order-0 / order-1 ABC coefficients (Thm 3.1, Thm 3.2)."""
import numpy as np
import pytest

from oracle.coefficients import order0, order1
from oracle.lattice import Box


@pytest.fixture(scope="module")
def box():
    return Box((5, 4, 6), 0.5)


def test_hgg_diagonal(box):
    """For the 3-point stencil H_{Gamma,II} H_{II,Gamma} = diag(c_gamma)/(4h^4), with c_gamma
    the number of exterior neighbours (each Sigma node touches one Gamma node)."""
    _, HGS = box.sigma()
    Hgg = HGS @ HGS.T
    c = box.exterior_neighbour_count()
    assert np.allclose(Hgg, np.diag(c / (4 * box.h ** 4)), atol=0)


@pytest.mark.parametrize("s1", [0.5, 1.0, 3.0])
def test_order1_identities(box, s1):
    co = order1(box, s1)
    A, B, Q, K1 = co["A"], co["B"], co["Q"], co["K1"]
    n = len(A)
    # i I + Q A = 0 (the cross terms of dW/dt vanish, eq:11)
    assert np.abs(Q @ A + 1j * np.eye(n)).max() < 1e-13
    # interpolation at s1: (s1 I - B)^{-1} A = K(s1)
    R11 = np.linalg.solve(s1 * np.eye(n) - B, A)
    assert np.abs(R11 - K1).max() < 1e-11 * np.abs(K1).max()
    # Q B + B^* Q is negative semi-definite (eq:35)
    S = Q @ B + B.conj().T @ Q
    assert np.abs(S - S.conj().T).max() < 1e-10 * np.abs(S).max()
    ev = np.linalg.eigvalsh((S + S.conj().T) / 2)
    assert ev.max() <= 1e-12 * np.abs(ev).max()
    # Q symmetric positive definite
    assert np.linalg.eigvalsh(Q).min() > 0


def test_order0_dissipative(box):
    """i (M^* - M) <= 0 for M = K(s0) (Thm 3.1)."""
    M = order0(box, 1.0)["M"]
    D = 1j * (M.conj().T - M)
    ev = np.linalg.eigvalsh((D + D.conj().T) / 2)
    assert ev.max() < 0
