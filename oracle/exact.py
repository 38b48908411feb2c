"""Closed-form solutions used as references (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The free Gaussian packet of the continuum equation i psi_t = -(1/2) Delta psi
(hbar = m = 1, Sec. 2):

    psi(x, 0) = exp(-|x - c|^2 / (2 sigma^2) + i k.(x - c))
    psi(x, t) = (sigma^2 / a)^{d/2} exp(-|x - c - k t|^2 / (2 a) + i k.(x - c) - i |k|^2 t / 2),
                a = sigma^2 + i t.

With d = 3, c = 0, k = (k0, 0, 0) and sigma^2 = 1/2 this is the paper's eq:15 (Sec.
4.2); with d = 1 it is eq:14 read with k0^2 t / 2 in the exponent (the printed k0^2 t
cannot solve the free equation).  It solves the continuum equation, not the lattice
one; the discrete solution approaches it at the order of the stencil in h.
"""
from __future__ import annotations

import numpy as np


def free_packet(X, t, center, k, sigma2):
    """psi(X, t) for coordinate arrays X = (x1[, x2[, x3]])."""
    d = len(X)
    a = sigma2 + 1j * t
    r2 = sum((X[i] - center[i] - k[i] * t) ** 2 for i in range(d))
    kx = sum(k[i] * (X[i] - center[i]) for i in range(d))
    k2 = sum(ki * ki for ki in k)
    return (sigma2 / a) ** (d / 2) * np.exp(-r2 / (2 * a) + 1j * kx - 0.5j * k2 * t)
