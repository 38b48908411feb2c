"""Grid, finite-difference stencil and the index sets of Sec. 2 (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The interior Omega_I is a box of nodes with spacing h; the exterior Omega_II is
the rest of the infinite lattice (Sec. 2).  H = -1/2 Delta_h + V with the
Laplacian applied axis by axis with a (2R+1)-point central formula
(Sec. 2, the 5-point example; "7-point scheme in each direction" of Sec. 4.2).
Nodes are ordered with x fastest: linear index ((k*Ny)+j)*Nx + i.
"""
from __future__ import annotations

import itertools
from fractions import Fraction

import numpy as np
import scipy.sparse as sp

# Central second-derivative coefficients c_0..c_R (c_{-m} = c_m).
# R = 2 is the paper's five-point formula (Sec. 2, App. B); R = 4 is App. D's
# nine-point formula with c_0 = -205/72 (the printed +205/72 cannot be right:
# the coefficients of a consistent second difference sum to zero).
STENCILS = {
    1: [Fraction(-2), Fraction(1)],
    2: [Fraction(-5, 2), Fraction(4, 3), Fraction(-1, 12)],
    3: [Fraction(-49, 18), Fraction(3, 2), Fraction(-3, 20), Fraction(1, 90)],
    4: [Fraction(-205, 72), Fraction(8, 5), Fraction(-1, 5), Fraction(8, 315), Fraction(-1, 560)],
}


def stencil(R: int) -> np.ndarray:
    return np.array([float(c) for c in STENCILS[R]])


class Box:
    """Interior box Omega_I: ``dims`` = (Nx[, Ny[, Nz]]), spacing ``h``, radius ``R``."""

    def __init__(self, dims, h: float, R: int = 1):
        self.dims = tuple(int(n) for n in dims)
        self.d = len(self.dims)
        self.h = float(h)
        self.R = int(R)
        self.shape = self.dims[::-1]          # numpy array shape (z, y, x)
        self.n = int(np.prod(self.dims))
        self.c = stencil(self.R)

    # ---- coordinates -------------------------------------------------
    def coords(self) -> np.ndarray:
        """(n, d) integer coordinates in (x, y, z) order, row = linear index."""
        idx = np.indices(self.shape).reshape(self.d, -1)
        return np.ascontiguousarray(idx[::-1].T)

    def linear(self, c: np.ndarray) -> np.ndarray:
        c = np.asarray(c)
        return np.ravel_multi_index(tuple(c[..., k] for k in reversed(range(self.d))), self.shape)

    def inside(self, c: np.ndarray) -> np.ndarray:
        c = np.asarray(c)
        ok = np.ones(c.shape[:-1], dtype=bool)
        for k in range(self.d):
            ok &= (c[..., k] >= 0) & (c[..., k] < self.dims[k])
        return ok

    # ---- the Hamiltonian ---------------------------------------------
    def offsets(self):
        """Axis-aligned stencil offsets with their H weights -c_m/(2h^2), m != 0."""
        out = []
        for k in range(self.d):
            for m in range(1, self.R + 1):
                w = -0.5 * self.c[m] / self.h ** 2
                for sgn in (1, -1):
                    e = np.zeros(self.d, dtype=np.int64)
                    e[k] = sgn * m
                    out.append((e, w))
        return out

    def diag_weight(self) -> float:
        return -0.5 * self.d * self.c[0] / self.h ** 2

    def H_II_kinetic(self) -> sp.csr_matrix:
        """Kinetic block of H_{I,I} (eq:32): couplings that leave the box are omitted
        here, because they belong to H_{I,II} and enter only through the boundary term."""
        C = self.coords()
        rows, cols, vals = [np.arange(self.n)], [np.arange(self.n)], [np.full(self.n, self.diag_weight())]
        for e, w in self.offsets():
            nb = C + e
            ok = self.inside(nb)
            rows.append(np.nonzero(ok)[0])
            cols.append(self.linear(nb[ok]))
            vals.append(np.full(int(ok.sum()), w))
        return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(self.n, self.n))

    # ---- index sets ---------------------------------------------------
    def gamma(self) -> np.ndarray:
        """Gamma (eq:25): interior nodes coupled by H to some exterior node, i.e. within
        R of a face.  Returned as ascending linear indices (the ordering E uses)."""
        C = self.coords()
        near = np.zeros(self.n, dtype=bool)
        for k in range(self.d):
            near |= (C[:, k] < self.R) | (C[:, k] > self.dims[k] - 1 - self.R)
        return np.nonzero(near)[0]

    def sigma(self):
        """Sigma (App. A): exterior nodes coupled by H to some interior node.

        Returns (coords (n_sigma, d), H_{Gamma,Sigma} as a dense (n_gamma, n_sigma) array)."""
        G = self.gamma()
        C = self.coords()
        sig = {}
        entries = []
        for e, w in self.offsets():
            nb = C[G] + e
            out = ~self.inside(nb)
            for gi, sc in zip(np.nonzero(out)[0], nb[out]):
                key = tuple(int(v) for v in sc)
                if key not in sig:
                    sig[key] = len(sig)
                entries.append((gi, sig[key], w))
        S = np.array(sorted(sig, key=sig.get), dtype=np.int64).reshape(-1, self.d)
        HGS = np.zeros((len(G), len(sig)))
        for gi, si, w in entries:
            HGS[gi, si] += w
        return S, HGS

    def exterior_neighbour_count(self) -> np.ndarray:
        """c_gamma: number of exterior nodes coupled to each Gamma node (R = 1)."""
        _, HGS = self.sigma()
        return (HGS != 0).sum(axis=1)


def n_gamma(dims, R: int) -> int:
    """|Gamma| = prod N - prod (N - 2R): used by the paper's 14166 count (Sec. 4.2)."""
    return int(np.prod(dims) - np.prod([max(n - 2 * R, 0) for n in dims]))


def all_offsets(d: int, rng_max: int):
    return itertools.product(range(-rng_max, rng_max + 1), repeat=d)
