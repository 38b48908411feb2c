"""Pins of the oracle's DtN map K(s) (eq:17, eq:eval, App. A/D)."""
import numpy as np
import pytest

from oracle.dtn import FreeGreen, decay_root_1d, dtn_1d_closed, dtn_bruteforce, dtn_eval
from oracle.lattice import Box


@pytest.mark.parametrize("s,h,N", [(1.0, 0.5, 6), (20.0, 0.1, 9), (0.3, 1.0, 4)])
def test_1d_closed_form(s, h, N):
    """1D, R = 1: the exterior is two half-lines, K = diag(-u/(2h^2)) with |u| < 1 and
    u + 1/u = 2 - 2ish^2.  Both oracle routes must reproduce it."""
    box = Box((N,), h)
    Kc = dtn_1d_closed(h, s)
    u = decay_root_1d(s, h)
    assert abs(u) < 1 and abs(u + 1 / u - (2 - 2j * s * h * h)) < 1e-14
    Ke = dtn_eval(box, s)
    assert np.allclose(Ke, np.diag([Kc, Kc]), atol=1e-13 * abs(Kc))
    Kb = dtn_bruteforce(box, s, 400)
    assert np.allclose(Kb, Ke, atol=1e-13 * abs(Kc))


@pytest.mark.parametrize("dims,h,s", [((3, 4), 1.0, 1.0), ((3, 3, 4), 1.0, 4.0), ((4, 4, 4), 1.0, 3.0),
                                      ((3, 4), 0.7, 0.5)])
def test_eval_matches_bruteforce(dims, h, s):
    """App. A's eq:eval equals the definition eq:17 on a truncated exterior (shell of L
    nodes, zero Dirichlet beyond); the shell is grown until the brute force converges."""
    box = Box(dims, h)
    Ke = dtn_eval(box, s)
    L = int(np.ceil(17.0 / -np.log(abs(decay_root_1d(s, h)))))
    Kb1 = dtn_bruteforce(box, s, L)
    Kb2 = dtn_bruteforce(box, s, L + 3)
    scale = np.abs(Ke).max()
    assert np.abs(Kb1 - Kb2).max() < 1e-13 * scale
    assert np.abs(Ke - Kb2).max() < 1e-12 * scale


def test_eval_converges_in_fft_lattice():
    box = Box((5, 4, 6), 0.5)
    K1 = dtn_eval(box, 1.0)
    g = FreeGreen(3, 0.5, 1, 1.0, 8)
    K2 = dtn_eval(box, 1.0, P=g.P + 32)
    assert np.abs(K1 - K2).max() < 1e-14 * np.abs(K1).max()


@pytest.mark.parametrize("s", [0.5, 1.0, 4.0])
def test_symmetry_and_negative_imaginary_part(s):
    """K(s) is complex symmetric (H is real symmetric) and Im K(s) <= 0 for s > 0
    (proof of Thm 3.1)."""
    box = Box((5, 6, 4), 0.5)
    K = dtn_eval(box, s)
    assert np.abs(K - K.T).max() < 1e-13 * np.abs(K).max()
    imK = (K - K.conj().T) / 2j
    ev = np.linalg.eigvalsh(imK)
    assert ev.max() < 0
    assert ev.max() < -1e-6 * np.abs(ev).max()


def test_large_s_asymptote():
    """s K(s) -> -H_{Gamma,II} H_{II,Gamma} i as s -> infinity (the second interpolation
    condition of Thm 3.2); the remainder decays like 1/s."""
    box = Box((4, 5, 4), 0.5)
    _, HGS = box.sigma()
    Hgg = HGS @ HGS.T
    errs = []
    for s in (100.0, 200.0, 400.0):
        K = dtn_eval(box, s)
        errs.append(np.abs(s * K + 1j * Hgg).max() / np.abs(Hgg).max())
    assert errs[0] < 0.15
    assert 1.7 < errs[0] / errs[1] < 2.3 and 1.7 < errs[1] / errs[2] < 2.3


def test_green_continuum_limit():
    """Far from the source the free lattice Green's function approaches h^3 times the
    continuum kernel of (-Delta/2 - i s): exp(-kappa r)/(2 pi r), kappa = sqrt(-2is)
    (App. D's fundamental solution up to the normalisation of App. A)."""
    h, s = 0.1, 1.0
    g = FreeGreen(3, h, 1, s, 30, P=192)
    kappa = np.sqrt(-2j * s)
    errs = []
    for n in (10, 15, 20):
        r = n * h
        lat = g(np.array([n, 0, 0]))
        cont = h ** 3 * np.exp(-kappa * r) / (2 * np.pi * r)
        errs.append(abs(lat - cont) / abs(cont))
    assert max(errs) < 1e-2
    assert errs[2] < errs[0]


@pytest.mark.parametrize("dims,h,s,L,tol", [((7, 8), 1.0, 1.0, 16, 1e-12), ((7, 7, 7), 1.0, 4.0, 8, 1e-11)])
def test_eval_matches_bruteforce_radius3(dims, h, s, L, tol):
    """The same two routes with the 7-point-per-axis stencil of Sec. 4.2 (R = 3): a
    three-node-deep Gamma and exterior couplings c_1 .. c_3 across it."""
    box = Box(dims, h, 3)
    Ke = dtn_eval(box, s)
    Kb = dtn_bruteforce(box, s, L)
    assert np.abs(Ke - Kb).max() < tol * np.abs(Ke).max()
