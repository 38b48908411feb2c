"""The discrete DtN map K(s) of eq:17 (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Two independent routes to the same matrix:

* ``dtn_bruteforce`` -- the definition K(s) = -H_{Gamma,II} [H_{II,II} - i s]^{-1} H_{II,Gamma}
  (eq:17), with the infinite exterior truncated to a wide shell with zero Dirichlet
  values on its outer face.  The truncation error decays like |u|^L for a shell L
  nodes thick, so this is the exact map up to a controlled error.
* ``dtn_eval`` -- App. A, eq:eval:
  K = -(I - H_{Gamma,Sigma} G_{Sigma,Gamma})^{-1} H_{Gamma,Sigma} G_{Sigma,Sigma} H_{Sigma,Gamma},
  with G = (H_0 - i s)^{-1} the free lattice Green's function (V = 0 everywhere;
  App. A's definition, normalised as H~ G~ = I).  G is taken from a periodic lattice
  of P nodes per axis by one inverse FFT of the symbol (the Brillouin-zone integral of
  App. D sampled on P points); the periodic Green's function is the sum of the free one
  over all images, so P is chosen so that the images are below 1e-17.

``dtn_eval_deriv`` gives K'(s) (the Hermite fit, eq:39) by differentiating eq:eval.

Plus the 1D closed form: with R = 1 each end of a 1D box sees a half-line, and
f_Gamma = H_{Gamma,II} phi_II = -(1/2h^2) u phi_Gamma, where u is the root with |u| < 1
of u + 1/u = 2 - 2 i s h^2 (the exterior equation (H - i s) phi = 0 solved by phi_j ~ u^j).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .lattice import Box


def decay_root_1d(s: float, h: float) -> complex:
    """Root |u| < 1 of u + 1/u = 2 - 2 i s h^2 (3-point exterior recursion)."""
    q = 1.0 - 1j * s * h * h
    r = np.sqrt(q * q - 1.0 + 0j)
    u1, u2 = q - r, q + r
    return u1 if abs(u1) < 1 else u2


def dtn_1d_closed(h: float, s: float) -> complex:
    """K(s) on one end of a 1D box with the 3-point stencil: -u/(2h^2)."""
    return -decay_root_1d(s, h) / (2.0 * h * h)


# ----------------------------------------------------------------------
# free lattice Green's function
# ----------------------------------------------------------------------
class FreeGreen:
    """G(Delta) = [(H_0 - i s)^{-1}](Delta) on the infinite lattice, V = 0."""

    def __init__(self, d: int, h: float, R: int, s: float, max_offset: int, P: int | None = None,
                 deriv: bool = False):
        """deriv: the table of dG/ds = i G^2 instead of G (symbol i / (sigma - i s)^2)."""
        self.d, self.h, self.R, self.s = d, h, R, s
        if P is None:
            rate = -math.log(abs(decay_root_1d(s, h)))
            P = max_offset + 1 + int(math.ceil(40.0 / rate))
            P += (-P) % 8
        self.P = P
        from .lattice import stencil
        c = stencil(R)
        xi = 2.0 * np.pi * np.fft.fftfreq(P)
        sym1 = -0.5 * (c[0] + 2.0 * sum(c[m] * np.cos(m * xi) for m in range(1, R + 1))) / h ** 2
        symbol = np.zeros((P,) * d, dtype=np.complex128)
        for k in range(d):
            shp = [1] * d
            shp[k] = P
            symbol = symbol + sym1.reshape(shp)
        symbol = symbol - 1j * s
        if deriv:
            self.table = np.fft.ifftn(1j / symbol ** 2)
        else:
            self.table = np.fft.ifftn(1.0 / symbol)   # periodic Green's function

    def __call__(self, delta: np.ndarray) -> np.ndarray:
        delta = np.asarray(delta) % self.P
        return self.table[tuple(delta[..., k] for k in range(self.d))]


def dtn_eval(box: Box, s: float, P: int | None = None) -> np.ndarray:
    """K(s) by eq:eval (App. A) with the periodic-FFT free Green's function."""
    G_idx = box.gamma()
    Cg = box.coords()[G_idx]
    Sg, HGS = box.sigma()
    HSG = HGS.T                                   # H is symmetric
    span = max(box.dims) + 2 * box.R
    g = FreeGreen(box.d, box.h, box.R, s, span, P)
    G_SG = g(Sg[:, None, :] - Cg[None, :, :])     # (n_sigma, n_gamma)
    G_SS = g(Sg[:, None, :] - Sg[None, :, :])     # (n_sigma, n_sigma)
    X = np.eye(len(G_idx)) - HGS @ G_SG
    Y = HGS @ G_SS @ HSG
    return -np.linalg.solve(X, Y)


def dtn_eval_deriv(box: Box, s: float, P: int | None = None) -> np.ndarray:
    """K'(s) = dK/ds by differentiating eq:eval: with X = I - H_{Gamma,Sigma} G_{Sigma,Gamma}
    and Y = H_{Gamma,Sigma} G_{Sigma,Sigma} H_{Sigma,Gamma}, X K = -Y gives
    K' = -X^{-1} (Y' + X' K), and G' = dG/ds = i G^2 (G = (H_0 - i s)^{-1})."""
    G_idx = box.gamma()
    Cg = box.coords()[G_idx]
    Sg, HGS = box.sigma()
    HSG = HGS.T
    span = max(box.dims) + 2 * box.R
    g = FreeGreen(box.d, box.h, box.R, s, span, P)
    gd = FreeGreen(box.d, box.h, box.R, s, span, g.P, deriv=True)
    dSG = Sg[:, None, :] - Cg[None, :, :]
    dSS = Sg[:, None, :] - Sg[None, :, :]
    X = np.eye(len(G_idx)) - HGS @ g(dSG)
    Y = HGS @ g(dSS) @ HSG
    K = -np.linalg.solve(X, Y)
    Xd = -(HGS @ gd(dSG))
    Yd = HGS @ gd(dSS) @ HSG
    return -np.linalg.solve(X, Yd + Xd @ K)


def dtn_bruteforce(box: Box, s: float, L: int) -> np.ndarray:
    """K(s) = -H_{Gamma,II}(H_{II,II} - i s)^{-1} H_{II,Gamma} (eq:17) on an exterior shell
    L nodes thick around the box, zero Dirichlet beyond it."""
    big = Box(tuple(n + 2 * L for n in box.dims), box.h, box.R)
    Hb = big.H_II_kinetic().tocsr()
    Cb = big.coords()
    inner = np.ones(big.n, dtype=bool)
    for k in range(box.d):
        inner &= (Cb[:, k] >= L) & (Cb[:, k] < L + box.dims[k])
    ext = np.nonzero(~inner)[0]
    # Gamma of the small box, expressed as big-box indices (same ascending order)
    Cg = box.coords()[box.gamma()] + L
    gam_big = big.linear(Cg)
    A = (Hb[ext][:, ext] - 1j * s * sp.identity(len(ext))).tocsc()
    Rhs = Hb[ext][:, gam_big].toarray().astype(np.complex128)
    X = spla.splu(A).solve(Rhs)
    return -(Hb[gam_big][:, ext] @ X)
