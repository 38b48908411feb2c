"""Pins of the oracle's K'(s) and of the two other first-order fits of
R_11(s) = (sI - B)^{-1} A: two finite interpolation points (Sec. 3.2's closing remark)
and value + derivative at one point (App. C, eq:39).

* K'(s) from differentiating eq:eval equals (a) central differences of the pinned
  K(s), (b) the definition K'(s) = -i H_{Gamma,II} (H_{II,II} - i s)^{-2} H_{II,Gamma} on a
  truncated exterior (the brute-force route, solved twice), and (c) in 1D the
  derivative of the closed form K = -u(s) / (2 h^2), u + 1/u = 2 - 2 i s h^2, which is
  i u^2 / (u^2 - 1).
* The two-point fit, evaluated as a rational function, equals K at both points; as
  the second point goes to infinity it tends to the Thm 3.2 fit (A = -i H H).
* The Hermite fit matches K(s1) and, by central differences of R_11 itself, K'(s1)
  (a route that does not use the closed form of the fit).
* Both fits give stable, absorbing dynamics on a packet leaving a small box over a
  long run (the paper reports the two-point variant as numerically stable; no proof
  covers either fit)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle.coefficients import order1, order1_hermite, order1_two_point, rational11
from oracle.dtn import decay_root_1d, dtn_eval, dtn_eval_deriv
from oracle.lattice import Box
from oracle.propagate import System
from paper_1908_02456_gb300 import inputs


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _dtn_deriv_bruteforce(box: Box, s: float, L: int) -> np.ndarray:
    """-i H_{Gamma,e} (H_e - i s)^{-2} H_{e,Gamma} on an exterior shell L nodes thick."""
    big = Box(tuple(n + 2 * L for n in box.dims), box.h, box.R)
    Hb = big.H_II_kinetic().tocsr()
    Cb = big.coords()
    inner = np.ones(big.n, dtype=bool)
    for k in range(box.d):
        inner &= (Cb[:, k] >= L) & (Cb[:, k] < L + box.dims[k])
    ext = np.nonzero(~inner)[0]
    gam = big.linear(box.coords()[box.gamma()] + L)
    lu = spla.splu((Hb[ext][:, ext] - 1j * s * sp.identity(len(ext))).tocsc())
    X = lu.solve(lu.solve(Hb[ext][:, gam].toarray().astype(np.complex128)))
    return -1j * (Hb[gam][:, ext] @ X)


@pytest.mark.parametrize("s", [0.6, 2.5])
def test_dK_matches_central_differences(s):
    box = Box((4, 5, 6), 0.5)
    d = 1e-4 * s
    fd = (dtn_eval(box, s + d) - dtn_eval(box, s - d)) / (2 * d)
    assert rel(dtn_eval_deriv(box, s), fd) < 1e-7


def test_dK_matches_truncated_definition():
    box = Box((4, 4, 5), 0.5)
    s = 3.0                      # fast exterior decay: a 14-node shell is exact to ~1e-10
    assert rel(dtn_eval_deriv(box, s), _dtn_deriv_bruteforce(box, s, 14)) < 1e-8


@pytest.mark.parametrize("s,h", [(2.0, 0.3), (0.5, 0.7)])
def test_dK_1d_closed_form(s, h):
    box = Box((9,), h)
    u = decay_root_1d(s, h)
    Kd = dtn_eval_deriv(box, s)
    for e in (0, 1):             # each end sees a half-line
        assert abs(Kd[e, e] - 1j * u * u / (u * u - 1)) < 1e-11 * abs(Kd[e, e])


def test_two_point_fit_interpolates_and_tends_to_thm32():
    box = Box((5, 4, 6), 0.5)
    co = order1_two_point(box, 1.0, 2.0)
    for sj in (1.0, 2.0):
        K = dtn_eval(box, sj)
        assert rel(rational11(co, sj), K) < 1e-12
    K3 = dtn_eval(box, 3.0)
    assert rel(rational11(co, 3.0), K3) > 1e-6          # the points belong to the fit
    lim = order1(box, 1.0)
    far = order1_two_point(box, 1.0, 1e8, K1=lim["K1"])
    assert rel(far["A"], lim["A"]) < 1e-6
    assert rel(far["B"], lim["B"]) < 1e-6


def test_hermite_fit_matches_value_and_slope():
    box = Box((5, 5, 4), 0.5)
    s1 = 1.3
    co = order1_hermite(box, s1)
    assert rel(rational11(co, s1), dtn_eval(box, s1)) < 1e-12
    d = 1e-4
    dR = (rational11(co, s1 + d) - rational11(co, s1 - d)) / (2 * d)
    dK = (dtn_eval(box, s1 + d) - dtn_eval(box, s1 - d)) / (2 * d)
    assert rel(dR, dK) < 1e-6
    # a planted slip (the sign of eq:39's second condition flipped) fails the slope pin
    X = dtn_eval_deriv(box, s1) @ np.linalg.inv(co["K1"])
    bad = {"A": np.linalg.inv(X) @ co["K1"], "B": s1 * np.eye(len(X)) - np.linalg.inv(X)}
    dRb = (rational11(bad, s1 + d) - rational11(bad, s1 - d)) / (2 * d)
    assert rel(dRb, dK) > 1e-2


@pytest.mark.parametrize("fit", ["two_point", "hermite"])
def test_fitted_dynamics_stable_and_absorbing(fit):
    """A slow packet (k = 1.5) over 2000 steps: the norm left in the box decays
    steadily to below 0.2 % (no late growth, the sign of an unstable fit)."""
    dims, h, dt, steps = (8, 8, 8), 0.5, 0.01, 2000
    box = Box(dims, h)
    co = order1_two_point(box, 1.0, 2.0) if fit == "two_point" else order1_hermite(box, 1.0)
    psi0 = inputs.gaussian_packet(dims, h, (0.0, 0.0, 0.0), (1.5, 0.0, 0.0), 0.8).reshape(1, -1)
    _, _, d = System(box, coeffs=co).run(psi0, dt, steps, diag_every=200)
    norms = d[:, 0, 0]
    assert np.all(np.diff(norms[3:]) < 0)
    assert norms[-1] < 2e-3
