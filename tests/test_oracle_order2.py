"""Pins of the oracle's second-order ABC (Sec. 3.3, eq:dynamics2).

* The fitted R_22(s) = (s^2 I - s B1 - B0)^{-1}(s A1 + A0), evaluated as a rational
  function, equals K(s) at the four interpolation points (the fit is a different
  linear system).
* The Laplace transform of eq:dynamics2 from the oracle's initial data (f = 0,
  g = A1 E phi(0)) eliminates f, g: (s + iH + i E^T R_22(s) E) phi_hat = phi(0).  The
  resolvent (s I - L)^{-1}, with L assembled column by column from the oracle's own
  operator, applied to that initial state must give this phi_hat at any s (every term
  of the g equation enters it).
* With B1 = B, B0 = 0, A1 = A, A0 = 0 (the order-1 coefficients) the set
  g = B f + A E phi is invariant under L, and on it the (phi, f) dynamics is
  eq:dynamics1: started there, the order-2 stepper reproduces the order-1 stepper.
* A planted slip (the A1 E phidot term dropped) fails the transfer-function pin."""
import numpy as np
import pytest

from oracle.coefficients import order1, order2, rational22
from oracle.dtn import dtn_eval
from oracle.lattice import Box
from oracle.propagate import System
from paper_1908_02456_gb300 import inputs


@pytest.fixture(scope="module")
def small():
    box = Box((4, 5, 4), 0.5)
    return box, order2(box, (0.7, 1.5, 3.0, 8.0))


def test_order2_interpolates_at_its_points(small):
    box, co = small
    for sj, Kj in zip(co["points"], co["Ks"]):
        R = rational22(co, sj)
        assert np.abs(R - Kj).max() < 1e-9 * np.abs(Kj).max()
    # the points are a property of the fit, not of K: between them R_22 differs from K
    s = 2.2
    K = dtn_eval(box, s)
    assert np.abs(rational22(co, s) - K).max() > 1e-9 * np.abs(K).max()


def _dense_L(sysm, V):
    """Matrix of the oracle's L on (phi, f, g) for one orbital, column by column."""
    n, ng = sysm.box.n, len(sysm.G)
    N = n + 2 * ng
    L = np.zeros((N, N), dtype=np.complex128)
    for c in range(N):
        y = np.zeros(N, dtype=np.complex128)
        y[c] = 1.0
        dphi, df = sysm.L(y[None, :n], y[None, n:], V)
        L[:n, c] = dphi[0]
        L[n:, c] = df[0]
    return L


def _transfer_residual(box, co, used, s):
    rng = np.random.default_rng(8)
    V = rng.uniform(-0.5, 0.5, box.n)
    sysm = System(box, V_ext=V, coeffs=used)
    n = box.n
    phi0 = rng.normal(size=(1, n)) + 1j * rng.normal(size=(1, n))
    y0 = np.concatenate([phi0, sysm.initial_aux(phi0)], axis=1)[0]
    yhat = np.linalg.solve(s * np.eye(len(y0)) - _dense_L(sysm, V), y0)
    H = sysm.Hk.toarray() + np.diag(V)
    E = np.zeros((len(sysm.G), n))
    E[np.arange(len(sysm.G)), sysm.G] = 1.0
    ref = np.linalg.solve(s * np.eye(n) + 1j * H + 1j * E.T @ rational22(co, s) @ E, phi0[0])
    return np.linalg.norm(yhat[:n] - ref) / np.linalg.norm(ref)


@pytest.mark.parametrize("s", [0.4, 2.2])
def test_order2_transfer_function(small, s):
    box, co = small
    assert _transfer_residual(box, co, co, s) < 1e-11


def test_order2_with_order1_coefficients_reproduces_order1():
    dims, h, dt, steps = (5, 4, 6), 0.5, 0.01, 20
    box = Box(dims, h)
    c1 = order1(box, 1.3)
    n_g = c1["A"].shape[0]
    Z = np.zeros_like(c1["A"])
    c2 = {"order": 2, "B1": c1["B"], "B0": Z, "A1": c1["A"], "A0": Z}
    rng = np.random.default_rng(4)
    V = rng.uniform(-0.5, 0.5, box.n)
    phi0 = inputs.random_state(dims, 2, rng).reshape(2, -1)
    f0 = rng.normal(size=(2, n_g)) + 1j * rng.normal(size=(2, n_g))
    s1 = System(box, V_ext=V, coeffs=c1)
    s2 = System(box, V_ext=V, coeffs=c2)
    g0 = (c1["B"] @ f0.T).T + (c1["A"] @ s1.E(phi0).T).T
    p1, f1, _ = s1.run(phi0, dt, steps, f0=f0)
    p2, a2, _ = s2.run(phi0, dt, steps, f0=np.concatenate([f0, g0], axis=1))
    assert np.linalg.norm(p2 - p1) / np.linalg.norm(p1) < 1e-12
    assert np.linalg.norm(a2[:, :n_g] - f1) / np.linalg.norm(f1) < 1e-12
    g1 = (c1["B"] @ f1.T).T + (c1["A"] @ s1.E(p1).T).T
    assert np.linalg.norm(a2[:, n_g:] - g1) / np.linalg.norm(g1) < 1e-11


def test_dropped_a1_term_is_caught(small):
    box, co = small
    broken = dict(co)
    broken["A1"] = np.zeros_like(co["A1"])       # the A1 E phidot term dropped from the g equation
    assert _transfer_residual(box, co, broken, 2.2) > 1e-6


def test_swapped_b0_b1_is_caught(small):
    box, co = small
    broken = dict(co, B1=co["B0"], B0=co["B1"])
    assert _transfer_residual(box, co, broken, 2.2) > 1e-6


def test_radius3_fit_is_a_stable_basic_solution():
    """Radius 3 (Sec. 4.2's stencil): the four-point system is nearly singular; the
    oracle's fit (basic solution of a column-pivoted QR) interpolates K at the points
    and keeps every root of det(s^2 I - s B1 - B0) in the closed left half-plane, and
    its free unknowns (one per dropped pivot, shared by all rows) are exactly zero."""
    box = Box((9, 8, 9), 0.5, 3)
    pts = (1.0, 2.0, 3.0, 10.0)
    co = order2(box, pts)
    n = co["B1"].shape[0]
    roots = np.linalg.eigvals(np.block([[np.zeros((n, n)), np.eye(n)], [co["B0"], co["B1"]]]))
    assert roots.real.max() < 1e-9
    for sj, K in zip(pts, co["Ks"]):
        assert np.abs(rational22(co, sj) - K).max() < 1e-7 * np.abs(K).max()
    X = np.concatenate([co[k] for k in ("B1", "B0", "A1", "A0")], axis=1)
    zero_cols = np.sum(np.all(X == 0, axis=0))
    assert 1 <= zero_cols < X.shape[1] // 4
