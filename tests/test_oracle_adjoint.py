"""Pins of the oracle's adjoint (reverse mode through the Taylor propagator)."""
import numpy as np
import pytest

from oracle.adjoint import absorbed, gradient
from oracle.coefficients import order0, order1
from oracle.lattice import Box
from oracle.propagate import System
from paper_1908_02456_gb300 import inputs


def _cplx(rng, *shape):
    return rng.normal(size=shape) + 1j * rng.normal(size=shape)


@pytest.mark.parametrize("order", [0, 1])
def test_dot_product(order):
    """<L x, y> = <x, L^H y> for the augmented operator."""
    box = Box((5, 4, 6), 0.5)
    rng = np.random.default_rng(3)
    co = order0(box, 1.0) if order == 0 else order1(box, 1.0)
    sy = System(box, V_ext=rng.normal(size=box.n), coeffs=co)
    ng = len(box.gamma())
    xp, yp = _cplx(rng, 2, box.n), _cplx(rng, 2, box.n)
    xf = _cplx(rng, 2, ng) if order == 1 else None
    yf = _cplx(rng, 2, ng) if order == 1 else None
    Lp, Lf = sy.L(xp, xf, sy.V_ext)
    Hp, Hf = sy.LH(yp, yf, sy.V_ext)
    lhs = np.vdot(yp, Lp) + (np.vdot(yf, Lf) if order == 1 else 0)
    rhs = np.vdot(Hp, xp) + (np.vdot(Hf, xf) if order == 1 else 0)
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


@pytest.mark.parametrize("order", [0, 1])
def test_gradient_vs_central_differences(order):
    N, h, dt, n = 6, 0.5, 0.01, 30
    box = Box((N,) * 3, h)
    rng = np.random.default_rng(4)
    V = inputs.smooth_random((N,) * 3, h, rng).reshape(-1)
    co = order0(box, 1.0) if order == 0 else order1(box, 1.0)
    psi = inputs.gaussian_packet((N,) * 3, h, (0, 0, 0), (2.0, 0.5, 0), 1.0).reshape(1, -1)
    J, g = gradient(System(box, V_ext=V, coeffs=co), psi, dt, n)
    assert abs(J - absorbed(System(box, V_ext=V, coeffs=co), psi, dt, n)) < 1e-14
    for t in range(3):
        dV = inputs.smooth_random((N,) * 3, h, rng).reshape(-1)
        eps = 1e-4
        Jp = absorbed(System(box, V_ext=V + eps * dV, coeffs=co), psi, dt, n)
        Jm = absorbed(System(box, V_ext=V - eps * dV, coeffs=co), psi, dt, n)
        fd = (Jp - Jm) / (2 * eps)
        an = float(g @ dV)
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-12, (fd, an)
