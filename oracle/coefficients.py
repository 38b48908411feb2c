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
