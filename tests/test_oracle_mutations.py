"""Planted mistakes in the oracle (CPU only) must be caught by its pins.

Each case patches one plausible slip into a copy of an oracle routine -- a dropped
term, a wrong sign, a transposed operand -- and checks that the corresponding pin
fails on it.  This shows the pins are sharp enough to trust."""
import math

import numpy as np
import scipy.fft as sfft

import oracle.dtn as dtn
from oracle.coefficients import order1
from oracle.lattice import Box
from oracle.propagate import System
from paper_1908_02456_gb300 import inputs


def test_dropped_taylor_term_is_caught(monkeypatch):
    def taylor3(self, op, phi, f, V, dt):
        out_p, tp, tf = phi.copy(), phi, f
        for k in range(1, 4):                          # quartic term dropped
            tp, tf = op(tp, tf, V)
            out_p = out_p + dt ** k / math.factorial(k) * tp
        return out_p, None
    monkeypatch.setattr(System, "taylor", taylor3)
    dims, h, dt, n = (5, 4, 6), 0.5, 0.02, 10
    box = Box(dims, h)
    phi0 = inputs.random_state(dims, 1, np.random.default_rng(0))
    phi, _, _ = System(box).run(phi0.reshape(1, -1), dt, n)
    lam = np.zeros(box.shape)
    for ax, N in zip((2, 1, 0), dims):
        shp = [1, 1, 1]
        shp[ax] = N
        lam = lam + ((1 - np.cos(np.pi * np.arange(1, N + 1) / (N + 1))) / h ** 2).reshape(shp)
    P = sum((-1j * dt * lam) ** k / math.factorial(k) for k in range(5))
    ref = sfft.idstn(sfft.dstn(phi0[0], type=1, norm="ortho") * P ** n, type=1, norm="ortho")
    assert np.linalg.norm(phi[0] - ref.reshape(-1)) / np.linalg.norm(ref) > 1e-8


def test_wrong_sign_of_shift_is_caught(monkeypatch):
    orig = dtn.FreeGreen.__init__

    def flipped(self, d, h, R, s, max_offset, P=None):
        orig(self, d, h, R, -s, max_offset, P)        # +is instead of -is
    monkeypatch.setattr(dtn.FreeGreen, "__init__", flipped)
    K = dtn.dtn_eval(Box((4, 5, 4), 0.5), 1.0)
    assert np.linalg.eigvalsh((K - K.conj().T) / 2j).max() > 0   # Im K <= 0 pin fails


def test_transposed_b_is_caught():
    box = Box((5, 4, 6), 0.5)
    co = order1(box, 1.0)
    A, B, K1 = co["A"], co["B"], co["K1"]
    n = len(A)
    bad = np.linalg.solve(np.eye(n) - B.T, A)
    assert np.abs(bad - K1).max() > 1e-6 * np.abs(K1).max()


def test_dropped_boundary_forcing_is_caught(monkeypatch):
    orig_L = System.L

    def L_no_forcing(self, phi, f, V):
        dphi, df = orig_L(self, phi, f, V)
        if self.order == 1:
            dphi = dphi + 1j * self.ET(f, phi.shape[1])   # removes -i E^T f
        return dphi, df
    monkeypatch.setattr(System, "L", L_no_forcing)
    N, h = 8, 0.5
    box = Box((N,) * 3, h)
    psi = inputs.gaussian_packet((N,) * 3, h, (0, 0, 0), (3.0, 0.5, 0), 1.0).reshape(1, -1)
    _, _, d = System(box, coeffs=order1(box, 1.0)).run(psi, 0.01, 100, diag_every=1)
    W = np.concatenate([[1.0], d[:, 0, 1]])
    assert not np.all(W[1:] <= W[:-1] * (1 + 1e-12))              # Lyapunov pin fails


# ---------------------------------------------------------------------------
# mean-field potential and energy functional (Sec. 4.3)
# ---------------------------------------------------------------------------
from meanfield_pins import energy_drift_ok, energy_scaling_ok, potential_scaling_ok  # noqa: E402


class _PowerAlpha(System):
    def potential(self, phi):                          # rho^alpha for rho^(1+alpha)
        a, b, al = self.meanfield
        rho = self.density(phi)
        return self.V_ext + a * rho + b * np.power(rho, al)


class _OneOrbitalDensity(System):
    def density(self, phi):                            # orbital sum dropped
        return np.abs(phi[0]) ** 2


class _WeightedDensityPotential(System):
    def potential(self, phi):                          # stray h^3 weight
        a, b, al = self.meanfield
        rho = self.w * self.density(phi)
        return self.V_ext + a * rho + b * np.power(rho, 1.0 + al)


class _EnergyFullA(System):
    def energy_functional(self, phi):                  # a rho^2 for (a/2) rho^2
        a, b, al = self.meanfield if self.meanfield else (0.0, 0.0, 0.0)
        rho = self.density(phi)
        kin = self.w * np.real(np.sum(phi.conj() * (self.Hk @ phi.T).T))
        return kin + self.w * np.sum(self.V_ext * rho + a * rho ** 2 + b / (2 + al) * rho ** (2 + al))


class _EnergyWrongB(System):
    def energy_functional(self, phi):                  # b/(1+alpha) for b/(2+alpha)
        a, b, al = self.meanfield if self.meanfield else (0.0, 0.0, 0.0)
        rho = self.density(phi)
        kin = self.w * np.real(np.sum(phi.conj() * (self.Hk @ phi.T).T))
        return kin + self.w * np.sum(self.V_ext * rho + 0.5 * a * rho ** 2 + b / (1 + al) * rho ** (2 + al))


class _EnergyPowerOnePlusAlpha(System):
    def energy_functional(self, phi):                  # rho^(1+alpha) in the energy
        a, b, al = self.meanfield if self.meanfield else (0.0, 0.0, 0.0)
        rho = self.density(phi)
        kin = self.w * np.real(np.sum(phi.conj() * (self.Hk @ phi.T).T))
        return kin + self.w * np.sum(self.V_ext * rho + 0.5 * a * rho ** 2 + b / (2 + al) * rho ** (1 + al))


def test_meanfield_potential_mistakes_are_caught():
    for bad in (_PowerAlpha, _OneOrbitalDensity, _WeightedDensityPotential):
        assert not energy_drift_ok(bad), bad.__name__
    assert not potential_scaling_ok(_PowerAlpha)
    assert not potential_scaling_ok(_OneOrbitalDensity)
    assert not potential_scaling_ok(_WeightedDensityPotential)


def test_meanfield_energy_mistakes_are_caught():
    for bad in (_EnergyFullA, _EnergyWrongB, _EnergyPowerOnePlusAlpha):
        assert not energy_drift_ok(bad), bad.__name__
    assert not energy_scaling_ok(_EnergyPowerOnePlusAlpha)


# ---- the second-order fit on a 1D box (hidden root at -min(s_j)) ----
from order2_pins import end_blocks, fit_ok, system  # noqa: E402


def _fit_copy(pts, Ks, sign=-1.0, place=True, ypow=2):
    """A copy of the oracle's one-end order-2 fit with one slip selectable."""
    M, Y = system(pts, Ks)
    if ypow != 2:
        Y = Y / np.repeat(np.asarray(pts), 2)[None, :] ** (2 - ypow)
    U, S, Vh = np.linalg.svd(M)
    x = U[:, -1].conj()
    X0 = Y @ (Vh[:-1].conj().T @ np.diag(1.0 / S[:-1]) @ U[:, :-1].conj().T)
    if not place:
        return X0
    lam = sign * min(pts)
    D0 = lam * lam * np.eye(2) - lam * X0[:, 0:2] - X0[:, 2:4]
    adj = np.array([[D0[1, 1], -D0[0, 1]], [-D0[1, 0], D0[0, 0]]])
    c = (lam * x[0:2] + x[2:4]) @ adj
    w = np.conj(c) * np.linalg.det(D0) / np.vdot(c, c)
    return X0 + np.outer(w, x)


def test_order2_1d_fit_mistakes_are_caught():
    pts = (10.0, 11.0, 20.0, 21.0)
    _, Ks = end_blocks(0.05, 240, pts)
    assert fit_ok(pts, Ks, _fit_copy(pts, Ks))                    # the copy itself passes
    assert not fit_ok(pts, Ks, _fit_copy(pts, Ks, sign=1.0))      # hidden root at +min(s_j)
    assert not fit_ok(pts, Ks, _fit_copy(pts, Ks, place=False))   # hidden root left where it falls
    assert not fit_ok(pts, Ks, _fit_copy(pts, Ks, ypow=1))        # s_j K_j for s_j^2 K_j
