"""Pins of the second-order fit on a 1D box (Sec. 3.3 applied to the five-point scheme
of Sec. 4.1), shared by the oracle's tests and its planted-mistake tests.

The interpolation conditions R_22(s_j) = K(s_j) of one end are linear in
X = [B1 B0 A1 A0] (2 x 8): X M = Y.  For the five-point scheme M is singular, with a
one-dimensional null space that comes from K itself: a fixed row combination of K(s)
obeys (s b1 + b0) K(s) = -(s a1 + a0) at every s.  The oracle picks one member of the
solution family (the hidden root of det(s^2 I - s B1 - B0) at -min(s_j)); these pins
check each of those facts independently of how the oracle computes them."""
import numpy as np

from oracle.dtn import dtn_eval
from oracle.lattice import Box


def end_blocks(h, n, pts):
    """K(s_j) of the left end (Gamma nodes 0, 1) of a 1D box of n nodes."""
    box = Box((n,), h, 2)
    return box, [dtn_eval(box, s)[0:2, 0:2] for s in pts]


def system(pts, Ks):
    """M, Y of X M = Y, written out block column by block column."""
    M = np.zeros((8, 8), dtype=np.complex128)
    Y = np.zeros((2, 8), dtype=np.complex128)
    for j, (s, K) in enumerate(zip(pts, Ks)):
        for c in range(2):
            col = 2 * j + c
            M[0:2, col] = s * K[:, c]
            M[2:4, col] = K[:, c]
            M[4 + c, col] = s
            M[6 + c, col] = 1.0
            Y[:, col] = s * s * K[:, c]
    return M, Y


def null_row(pts, Ks):
    """The singular values of M and its left null row x (x M = 0)."""
    M, _ = system(pts, Ks)
    U, S, _ = np.linalg.svd(M)
    return S, U[:, -1].conj()


def identity_residual(box, x, s):
    """|(s b1 + b0) K(s) + s a1 + a0| / (|x| |K(s)|) at a point s off the fit."""
    K = dtn_eval(box, s)[0:2, 0:2]
    r = (s * x[0:2] + x[2:4]) @ K + s * x[4:6] + x[6:8]
    return np.abs(r).max() / (np.abs(x).max() * np.abs(K).max())


def roots(B1, B0):
    """The roots of det(s^2 I - s B1 - B0) (companion linearisation)."""
    C = np.block([[np.zeros((2, 2)), np.eye(2)], [B0, B1]])
    return np.linalg.eigvals(C)


def r22(X, s):
    B1, B0, A1, A0 = (X[:, 2 * k:2 * k + 2] for k in range(4))
    return np.linalg.solve(s * s * np.eye(2) - s * B1 - B0, s * A1 + A0)


def fit_ok(pts, Ks, X, tol=1e-6):
    """The fit's three properties: it interpolates K at the four points, its four
    roots lie in the left half-plane, and one of them is -min(s_j)."""
    interp = max(np.abs(r22(X, s) - K).max() / np.abs(K).max() for s, K in zip(pts, Ks)) < tol
    z = roots(X[:, 0:2], X[:, 2:4])
    smin = min(pts)
    return bool(interp and z.real.max() < 0 and np.abs(z + smin).min() < 1e-6 * smin)
