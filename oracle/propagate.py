"""Reduced dynamics with the ABC, the Taylor propagator and diagnostics (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

State y = (phi, f): phi holds b orbitals on the interior nodes (shape (b, n_I)),
f the auxiliary boundary variable f_Gamma of the first-order ABC (shape (b, n_Gamma),
f(0) = 0 because phi_II(0) = 0, Sec. 2).  For the second-order ABC f holds [f | g]
with g = df/dt (shape (b, 2 n_Gamma)).  The linear operator L of y' = L y is

  no ABC  : L phi = -i H_{I,I} phi                            (zero Dirichlet)
  order 0 : L phi = -i H_{I,I} phi - i E^T M E phi            (eq:dynamics0)
  order 1 : L (phi, f) = (-i H_{I,I} phi - i E^T f,  B f + A E phi)   (eq:dynamics1)
  order 2 : L (phi, f, g) = (phidot, g, B1 g + B0 f + A1 E phidot + A0 E phi),
            phidot = -i H_{I,I} phi - i E^T f                 (eq:dynamics2)

with H_{I,I} = kinetic + diag(V).  One time step applies the degree-4 Taylor
polynomial of exp(dt L) (eq:21, read as sum_{k=0..4} (dt L)^k / k!; the printed
signs of its cubic and quartic terms are garbled) term by term.

Mean field (Sec. 4.3, eq:ham_tdhf, in the simplified density-dependent form
V = V_ext + a rho + b rho^(1+alpha), rho = sum_j |phi_j|^2): V is computed from the
state at the start of each step and held fixed within the step.  The energy that the
exact mean-field dynamics conserves (with a closed box) is the functional whose
derivative with respect to rho is V (Sec. 4.3 reports the energy released):

  E[phi] = h^d sum_j Re <phi_j, H_kin phi_j>
         + h^d sum_x [ V_ext rho + (a/2) rho^2 + b/(2+alpha) rho^(2+alpha) ].
"""
from __future__ import annotations

import math

import numpy as np

from .lattice import Box


class System:
    def __init__(self, box: Box, V_ext=None, coeffs: dict | None = None, meanfield=None):
        self.box = box
        self.Hk = box.H_II_kinetic().tocsr()
        self.G = box.gamma()
        self.V_ext = np.zeros(box.n) if V_ext is None else np.asarray(V_ext, dtype=np.float64).reshape(-1)
        self.coeffs = coeffs
        self.order = None if coeffs is None else coeffs["order"]
        self.meanfield = meanfield
        self.w = box.h ** box.d              # quadrature weight of the discrete norm

    # ---- potential ----------------------------------------------------
    def density(self, phi):
        return np.sum(np.abs(phi) ** 2, axis=0)

    def potential(self, phi):
        """V = V_ext + a rho + b rho^(1+alpha) (mean field), else V_ext."""
        if self.meanfield is None:
            return self.V_ext
        a, b, alpha = self.meanfield
        rho = self.density(phi)
        return self.V_ext + a * rho + b * np.power(rho, 1.0 + alpha)

    def energy_potential(self, phi):
        """V_ext + e(rho) with e(rho) = (a/2) rho + b/(2+alpha) rho^(1+alpha), the
        interaction energy per unit density: h^d sum_x rho e(rho) is the interaction
        term of E[phi].  Without a mean field this is V_ext."""
        if self.meanfield is None:
            return self.V_ext
        a, b, alpha = self.meanfield
        rho = self.density(phi)
        return self.V_ext + 0.5 * a * rho + b / (2.0 + alpha) * np.power(rho, 1.0 + alpha)

    def energy_functional(self, phi):
        """E[phi] = h^d sum_j Re<phi_j, H_kin phi_j> + h^d sum_x [V_ext rho + (a/2) rho^2
        + b/(2+alpha) rho^(2+alpha)] (no mean field: the last two terms are absent)."""
        kin = self.w * np.real(np.sum(phi.conj() * (self.Hk @ phi.T).T))
        rho = self.density(phi)
        pot = self.w * np.sum(self.V_ext * rho)
        if self.meanfield is not None:
            a, b, alpha = self.meanfield
            pot += self.w * np.sum(0.5 * a * rho ** 2 + b / (2.0 + alpha) * np.power(rho, 2.0 + alpha))
        return kin + pot

    # ---- operators ----------------------------------------------------
    def H(self, phi, V):
        """H_{I,I} phi for every orbital."""
        return (self.Hk @ phi.T).T + V[None, :] * phi

    def E(self, phi):
        return phi[:, self.G]

    def ET(self, g, n):
        out = np.zeros((g.shape[0], n), dtype=np.complex128)
        out[:, self.G] = g
        return out

    def L(self, phi, f, V):
        dphi = -1j * self.H(phi, V)
        df = None
        if self.order == 0:
            M = self.coeffs["M"]
            dphi = dphi - 1j * self.ET((M @ self.E(phi).T).T, phi.shape[1])
        elif self.order == 1:
            A, B = self.coeffs["A"], self.coeffs["B"]
            dphi = dphi - 1j * self.ET(f, phi.shape[1])
            df = (B @ f.T).T + (A @ self.E(phi).T).T
        elif self.order == 2:
            co = self.coeffs
            ng = len(self.G)
            fa, ga = f[:, :ng], f[:, ng:]
            dphi = dphi - 1j * self.ET(fa, phi.shape[1])
            dg = (co["B1"] @ ga.T).T + (co["B0"] @ fa.T).T + (co["A1"] @ self.E(dphi).T).T \
                + (co["A0"] @ self.E(phi).T).T
            df = np.concatenate([ga, dg], axis=1)
        return dphi, df

    def LH(self, phi, f, V):
        """Adjoint operator L^H (for the reverse sweep; orders 0 and 1)."""
        if self.order == 2:
            raise NotImplementedError("the reverse sweep covers orders 0 and 1")
        dphi = 1j * self.H(phi, V)
        df = None
        if self.order == 0:
            M = self.coeffs["M"]
            dphi = dphi + 1j * self.ET((M.conj().T @ self.E(phi).T).T, phi.shape[1])
        elif self.order == 1:
            A, B = self.coeffs["A"], self.coeffs["B"]
            dphi = dphi + self.ET((A.conj().T @ f.T).T, phi.shape[1])
            df = 1j * self.E(phi) + (B.conj().T @ f.T).T
        return dphi, df

    # ---- time stepping ------------------------------------------------
    def initial_aux(self, phi):
        """Auxiliary data at t = 0.  Order 1: f(0) = 0 (phi_II(0) = 0, Sec. 2).  Order 2:
        f(0) = 0 and g(0) = A1 E phi(0), the value for which the Laplace transform of
        eq:dynamics2 gives f_hat = R_22(s) E phi_hat (the A1 E phidot term carries phi(0);
        the exact exterior solution likewise has df/dt(0) = -i H_{Gamma,II} H_{II,Gamma} phi(0))."""
        aux = self.zero_aux(phi.shape[0])
        if self.order == 2:
            aux[:, len(self.G):] = (self.coeffs["A1"] @ self.E(phi).T).T
        return aux

    def zero_aux(self, b):
        if self.order == 1:
            return np.zeros((b, len(self.G)), dtype=np.complex128)
        if self.order == 2:
            return np.zeros((b, 2 * len(self.G)), dtype=np.complex128)
        return None

    def taylor(self, op, phi, f, V, dt):
        """sum_{k=0..4} (dt op)^k / k! applied to (phi, f), term by term."""
        out_p, out_f = phi.copy(), None if f is None else f.copy()
        tp, tf = phi, f
        for k in range(1, 5):
            tp, tf = op(tp, tf, V)
            c = dt ** k / math.factorial(k)
            out_p = out_p + c * tp
            if tf is not None:
                out_f = out_f + c * tf
        return out_p, out_f

    def step(self, phi, f, dt):
        V = self.potential(phi)
        return self.taylor(self.L, phi, f, V, dt)

    def diagnostics(self, phi, f):
        """Per orbital: [norm, W, interior energy] (all with the h^d weight).

        norm = h^d |phi_j|^2; W = norm + h^d f_j^* Q f_j (eq:lyapunov1; = norm for
        order 0 / no ABC, eq:lyapunov0, and for order 2, which has no proven
        Lyapunov functional); energy = h^d Re <phi_j, (H_kin + V_ext + e(rho)) phi_j>
        with e the interaction energy per unit density (``energy_potential``), so
        that the orbitals' energies sum to E[phi] (``energy_functional``); without a
        mean field it is h^d Re <phi_j, H_{I,I} phi_j>."""
        V = self.energy_potential(phi)
        norm = self.w * np.sum(np.abs(phi) ** 2, axis=1)
        W = norm.copy()
        if self.order == 1:
            Q = self.coeffs["Q"]
            W = W + self.w * np.real(np.einsum("bi,ij,bj->b", f.conj(), Q, f))
        en = self.w * np.real(np.sum(phi.conj() * self.H(phi, V), axis=1))
        return np.stack([norm, W, en], axis=1)

    def run(self, phi0, dt, nsteps, f0=None, diag_every=0):
        phi = np.asarray(phi0, dtype=np.complex128).reshape(phi0.shape[0], -1)
        f = self.initial_aux(phi) if f0 is None else np.asarray(f0, dtype=np.complex128)
        diags = []
        for n in range(1, nsteps + 1):
            phi, f = self.step(phi, f, dt)
            if diag_every and n % diag_every == 0:
                diags.append(self.diagnostics(phi, f))
        return phi, f, (np.array(diags) if diag_every else None)
