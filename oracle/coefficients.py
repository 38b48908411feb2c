"""Coefficient matrices of the zeroth- and first-order ABCs (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

* Order 0 (Sec. 3.1, eq:dynamics0, Thm 3.1): M = K(s0), s0 > 0.  The paper's remark
  that M be "Hermitian" is read as complex-symmetric: K(s0) is used unmodified, since a
  Hermitian M would give dW/dt = 0 in the proof of Thm 3.1 (no absorption at all).
* Order 1 (Sec. 3.2, eq:dynamics1, Thm 3.2): R_11(s) = (sI - B)^{-1} A with
    A = -i H_{Gamma,II} H_{II,Gamma}     (matching the s -> infinity limit),
    B = s1 I - A K(s1)^{-1}              (interpolation at s1),
    Q = (H_{Gamma,II} H_{II,Gamma})^{-1} (the Lyapunov weight of eq:lyapunov1).
  H_{Gamma,II} H_{II,Gamma} = H_{Gamma,Sigma} H_{Sigma,Gamma} because H_{Gamma,II} is
  non-zero only on Sigma.
* Order 1, other fits of the same R_11(s) = (sI - B)^{-1} A (both B and A dense):
    two finite points (Sec. 3.2's closing remark: still stable with s2 finite):
      R_11(s1) = K(s1), R_11(s2) = K(s2), i.e. (s_j I - B) K_j = A for j = 1, 2;
    value and derivative at s1 (App. C, eq:39):
      (s1 I - B)^{-1} A = K(s1),  (s1 I - B)^{-2} A = -K'(s1).
  Both are solved here as the linear systems they are.  Q stays the Thm 3.2 weight
  (H_{Gamma,II} H_{II,Gamma})^{-1}, used for the diagnostic W only.
* Order 2 (Sec. 3.3, eq:dynamics2): R_22(s) = (s^2 I - s B1 - B0)^{-1} (s A1 + A0),
  fitted by interpolation at four points s_j (R_22(s_j) = K(s_j)); each condition
  s_j^2 K_j = s_j B1 K_j + B0 K_j + s_j A1 + A0 is linear in [B1, B0, A1, A0].
* Order 2 in 1D (Sec. 4.1, five-point scheme): each end's 2 x 2 block is fitted on its
  own (the ends see disjoint half-lines, so K is block diagonal).  There the 8 x 8
  interpolation system has a one-dimensional null space: a fixed row combination of
  K(s) obeys a first-degree identity (s b1 + b0) K(s) = -(s a1 + a0) for every s.  The
  solutions [B1 B0 A1 A0] = X0 + w x (x the null row, w any 2-vector) share R_22(s)
  for every s but differ in one hidden mode, a root of det(s^2 I - s B1 - B0) that R_22
  does not show and that rounding excites; for some w it lies in the right half-plane
  and the run diverges.  The paper does not address this; the reading taken here: X0 is
  the minimum-norm solution (pseudo-inverse of rank 7) and w the shortest vector that
  puts the hidden root at s = -min(s_j), a decaying mode.  By the determinant lemma
  det(D0(l) - w r) = det D0(l) - r adj(D0(l)) w with D0(l) = l^2 I - l B1 - B0 of X0 and
  r = l x_B1 + x_B0, so the condition is one linear equation in w.
* Order 2 with a wider stencil in 3D (radius R >= 2, Sec. 4.2's seven-point scheme per
  axis): the 4 n x 4 n system has many near-null directions with no clear gap (131
  singular values below 1e-11 sigma_1 at 7 x 8 x 7), and a plain LU solution puts roots
  of det(s^2 I - s B1 - B0) deep in the right half-plane (real parts ~1e3 at 11^3,
  h = 0.1: the fitted dynamics diverge).  Reading: the basic solution of a
  column-pivoted QR at numerical rank, pivots below 1e-13 |R_11| dropped (the free
  unknowns set to zero; Golub and Van Loan, Sec. 5.5).  It interpolates K to ~1e-9 and
  keeps every root at Re <= ~1e-7 on the boxes checked.  Radius 1 keeps the plain solve.
"""
from __future__ import annotations

import numpy as np

from .dtn import dtn_eval, dtn_eval_deriv
from .lattice import Box


def order0(box: Box, s0: float, K=None) -> dict:
    M = dtn_eval(box, s0) if K is None else K
    return {"order": 0, "s": s0, "M": M}


def order1(box: Box, s1: float, K1=None) -> dict:
    _, HGS = box.sigma()
    Hgg = HGS @ HGS.T                      # H_{Gamma,II} H_{II,Gamma}
    A = -1j * Hgg
    K1 = dtn_eval(box, s1) if K1 is None else K1
    B = s1 * np.eye(len(Hgg)) - A @ np.linalg.inv(K1)
    Q = np.linalg.inv(Hgg)
    return {"order": 1, "s": s1, "A": A, "B": B, "Q": Q, "K1": K1}


def order1_two_point(box: Box, s1: float, s2: float, K1=None, K2=None) -> dict:
    """B and A from (s1 I - B) K1 = A and (s2 I - B) K2 = A: subtracting gives
    B (K1 - K2) = s1 K1 - s2 K2; then A = (s1 I - B) K1."""
    if not (s1 > 0 and s2 > 0) or s1 == s2:
        raise ValueError("two distinct positive interpolation points are needed")
    K1 = dtn_eval(box, s1) if K1 is None else K1
    K2 = dtn_eval(box, s2) if K2 is None else K2
    n = K1.shape[0]
    # B D = C  <=>  D^T B^T = C^T
    B = np.linalg.solve((K1 - K2).T, (s1 * K1 - s2 * K2).T).T
    A = (s1 * np.eye(n) - B) @ K1
    _, HGS = box.sigma()
    Q = np.linalg.inv(HGS @ HGS.T)
    return {"order": 1, "fit": "two_point", "s": s1, "s2": s2, "A": A, "B": B, "Q": Q, "K1": K1, "K2": K2}


def order1_hermite(box: Box, s1: float, K1=None, dK1=None) -> dict:
    """eq:39: with X = (s1 I - B)^{-1}, X A = K1 and X (X A) = -K1' give X K1 = -K1', so
    X = -K1' K1^{-1}; then B = s1 I - X^{-1} and A = X^{-1} K1."""
    if not s1 > 0:
        raise ValueError("the interpolation point must be positive")
    K1 = dtn_eval(box, s1) if K1 is None else K1
    dK1 = dtn_eval_deriv(box, s1) if dK1 is None else dK1
    n = K1.shape[0]
    X = -dK1 @ np.linalg.inv(K1)
    Xi = np.linalg.inv(X)
    B = s1 * np.eye(n) - Xi
    A = Xi @ K1
    _, HGS = box.sigma()
    Q = np.linalg.inv(HGS @ HGS.T)
    return {"order": 1, "fit": "hermite", "s": s1, "A": A, "B": B, "Q": Q, "K1": K1, "dK1": dK1}


def rational11(co: dict, s: float) -> np.ndarray:
    """R_11(s) = (sI - B)^{-1} A."""
    n = co["B"].shape[0]
    return np.linalg.solve(s * np.eye(n) - co["B"], co["A"])


def order2(box: Box, points=(1.0, 2.0, 3.0, 10.0), Ks=None) -> dict:
    """Second-order coefficients from interpolation at four distinct points s_j > 0:
    [B1, B0, A1, A0] M = [s_1^2 K_1, ..., s_4^2 K_4] with block column j of M equal to
    (s_j K_j; K_j; s_j I; I)."""
    pts = [float(x) for x in points]
    if len(pts) != 4 or len(set(pts)) != 4 or min(pts) <= 0:
        raise ValueError("order 2 needs four distinct positive interpolation points")
    Ks = [dtn_eval(box, sj) for sj in pts] if Ks is None else list(Ks)
    if box.d == 1:
        return _order2_1d(pts, Ks)
    n = Ks[0].shape[0]
    M, Y = _interp2_system(pts, Ks)
    if box.R >= 2:
        X = _basic_solution(M.T, Y.T, 1e-13).T
    else:
        X = np.linalg.solve(M.T, Y.T).T
    B1, B0, A1, A0 = (X[:, k * n:(k + 1) * n] for k in range(4))
    return {"order": 2, "points": tuple(pts), "B1": B1, "B0": B0, "A1": A1, "A0": A0, "Ks": Ks}


def _interp2_system(pts, Ks):
    """M and Y of the order-2 interpolation conditions X M = Y, X = [B1 B0 A1 A0]."""
    n = Ks[0].shape[0]
    I = np.eye(n)
    M = np.zeros((4 * n, 4 * n), dtype=np.complex128)
    Y = np.zeros((n, 4 * n), dtype=np.complex128)
    for j, (sj, Kj) in enumerate(zip(pts, Ks)):
        cols = slice(j * n, (j + 1) * n)
        M[0:n, cols] = sj * Kj
        M[n:2 * n, cols] = Kj
        M[2 * n:3 * n, cols] = sj * I
        M[3 * n:4 * n, cols] = I
        Y[:, cols] = sj * sj * Kj
    return M, Y


def _basic_solution(A, B, rtol):
    """Z with A Z = B by column-pivoted QR, at the rank of the pivots above rtol |R_11|,
    the remaining unknowns zero."""
    import scipy.linalg as sla
    Q, R, P = sla.qr(A, pivoting=True)
    d = np.abs(np.diag(R))
    r = int(np.sum(d > rtol * d[0]))
    Z = np.zeros((A.shape[1], B.shape[1]), dtype=np.complex128)
    Z[P[:r]] = sla.solve_triangular(R[:r, :r], (Q.conj().T @ B)[:r])
    return Z


def order2_end(pts, Ks) -> np.ndarray:
    """One end of the 1D box: X = [B1 B0 A1 A0] (2 x 8) for the 2 x 2 blocks Ks at the
    four points, the null direction fixed by the hidden-root rule of the module doc."""
    M, Y = _interp2_system(pts, Ks)
    U, S, Vh = np.linalg.svd(M)
    if S[-1] > 1e-6 * S[-2]:                        # full rank: the unique solution
        return np.linalg.solve(M.T, Y.T).T
    x = U[:, -1].conj()                             # x M = 0
    X0 = Y @ (Vh[:-1].conj().T @ np.diag(1.0 / S[:-1]) @ U[:, :-1].conj().T)
    lam = -min(pts)
    D0 = lam * lam * np.eye(2) - lam * X0[:, 0:2] - X0[:, 2:4]
    adj = np.array([[D0[1, 1], -D0[0, 1]], [-D0[1, 0], D0[0, 0]]])
    c = (lam * x[0:2] + x[2:4]) @ adj
    w = np.conj(c) * np.linalg.det(D0) / np.vdot(c, c)
    return X0 + np.outer(w, x)


def _order2_1d(pts, Ks) -> dict:
    """Order 2 on a 1D box: Gamma = [0, 1, n-2, n-1], K block diagonal over the ends."""
    out = {k: np.zeros((4, 4), dtype=np.complex128) for k in ("B1", "B0", "A1", "A0")}
    for ends in (slice(0, 2), slice(2, 4)):
        X = order2_end(pts, [K[ends, ends] for K in Ks])
        for k, key in enumerate(("B1", "B0", "A1", "A0")):
            out[key][ends, ends] = X[:, 2 * k:2 * k + 2]
    return {"order": 2, "points": tuple(pts), **out, "Ks": Ks}


def rational22(co: dict, s: float) -> np.ndarray:
    """R_22(s) = (s^2 I - s B1 - B0)^{-1} (s A1 + A0)."""
    n = co["B1"].shape[0]
    return np.linalg.solve(s * s * np.eye(n) - s * co["B1"] - co["B0"], s * co["A1"] + co["A0"])
