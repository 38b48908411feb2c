"""Reverse-mode gradient of the absorbed probability w.r.t. the potential (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

J(V) = sum_j (1 - h^d |phi_j(T)|^2), the probability that left the box, for a
static potential V (no mean field).  With the Wirtinger convention dJ = 2 Re <g, dy>,
g_N = dJ/dy_N^* = (-h^d phi_N, 0).  Each step is y_{n+1} = U y_n with
U = sum_{k=0..4} (dt L)^k / k! and L = L_0 - i diag(V) on the phi part, so

  g_n      = U^H g_{n+1},
  dJ/dV_x  = sum_n sum_{k=1..4} dt^k/k! sum_{j=0..k-1}
             2 Re[ sum_orb conj(((L^H)^j g_{n+1})_phi,x) * (-i) (L^{k-1-j} y_n)_phi,x ].

All states are kept (no checkpointing): plain and slow by design.
"""
from __future__ import annotations

import math

import numpy as np

from .propagate import System


def absorbed(system: System, phi0, dt, nsteps):
    phi, f, _ = system.run(phi0, dt, nsteps)
    return float(np.sum(1.0 - system.w * np.sum(np.abs(phi) ** 2, axis=1)))


def gradient(system: System, phi0, dt, nsteps):
    """Returns (J, dJ/dV) with dJ/dV of shape (n_I,)."""
    if system.meanfield is not None:
        raise ValueError("the adjoint covers a static potential only")
    V = system.V_ext
    phi = np.asarray(phi0, dtype=np.complex128).reshape(phi0.shape[0], -1)
    f = system.zero_aux(phi.shape[0])
    states = [(phi, f)]
    for _ in range(nsteps):
        phi, f = system.taylor(system.L, phi, f, V, dt)
        states.append((phi, f))
    J = float(np.sum(1.0 - system.w * np.sum(np.abs(phi) ** 2, axis=1)))
    gp = -system.w * phi
    gf = None if f is None else np.zeros_like(f)
    grad = np.zeros(system.box.n)
    for n in range(nsteps - 1, -1, -1):
        yp, yf = states[n]
        # b_i = L^i y_n, i = 0..3 ; a_j = (L^H)^j g_{n+1}, j = 0..3
        bs = [(yp, yf)]
        for _ in range(3):
            bs.append(system.L(*bs[-1], V))
        as_ = [(gp, gf)]
        for _ in range(3):
            as_.append(system.LH(*as_[-1], V))
        for k in range(1, 5):
            c = dt ** k / math.factorial(k)
            for j in range(k):
                a_phi = as_[j][0]
                b_phi = bs[k - 1 - j][0]
                grad += c * 2.0 * np.real(np.sum(a_phi.conj() * (-1j) * b_phi, axis=0))
        gp, gf = system.taylor(system.LH, gp, gf, V, dt)
    return J, grad
