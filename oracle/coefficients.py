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
* Order 2 (Sec. 3.3, eq:dynamics2): R_22(s) = (s^2 I - s B1 - B0)^{-1} (s A1 + A0),
  fitted by interpolation at four points s_j (R_22(s_j) = K(s_j)); each condition
  s_j^2 K_j = s_j B1 K_j + B0 K_j + s_j A1 + A0 is linear in [B1, B0, A1, A0].
"""
from __future__ import annotations

import numpy as np

from .dtn import dtn_eval
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


def order2(box: Box, points=(1.0, 2.0, 3.0, 10.0), Ks=None) -> dict:
    """Second-order coefficients from interpolation at four distinct points s_j > 0:
    [B1, B0, A1, A0] M = [s_1^2 K_1, ..., s_4^2 K_4] with block column j of M equal to
    (s_j K_j; K_j; s_j I; I)."""
    pts = [float(x) for x in points]
    if len(pts) != 4 or len(set(pts)) != 4 or min(pts) <= 0:
        raise ValueError("order 2 needs four distinct positive interpolation points")
    Ks = [dtn_eval(box, sj) for sj in pts] if Ks is None else list(Ks)
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
    X = np.linalg.solve(M.T, Y.T).T
    B1, B0, A1, A0 = (X[:, k * n:(k + 1) * n] for k in range(4))
    return {"order": 2, "points": tuple(pts), "B1": B1, "B0": B0, "A1": A1, "A0": A0, "Ks": Ks}


def rational22(co: dict, s: float) -> np.ndarray:
    """R_22(s) = (s^2 I - s B1 - B0)^{-1} (s A1 + A0)."""
    n = co["B1"].shape[0]
    return np.linalg.solve(s * s * np.eye(n) - s * co["B1"] - co["B0"], s * co["A1"] + co["A0"])
