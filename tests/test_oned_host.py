"""Host set-up of the one-dimensional stepper (include/abc1d.h) against the oracle, on
CPU: the boundary blocks of the five-point scheme (Sec. 4.1, App. B).

The oracle builds K(s) for the whole Gamma of the 1D box (both ends at once) from an
FFT Green's function; the library builds the left end's 2 x 2 block from the closed
form of App. B and mirrors it for the right end.  Orders 0 and 1 must agree to
rounding.  The second-order fit at four points has one null direction per end (an
identity of K(s)); both sides fix it by placing the hidden root at -min(s_j), so the
blocks agree entry by entry to the fit's conditioning."""
import numpy as np
import pytest

from oracle.coefficients import order0, order1, order1_two_point, order2
from oracle.dtn import dtn_eval
from oracle.lattice import Box
from paper_1908_02456_gb300 import abc

from order2_pins import end_blocks, fit_ok

N, H = 40, 0.05


@pytest.fixture(scope="module")
def box():
    return Box((N,), H, 2)


def blocks_agree(lib, ora, tol):
    left, right = ora[0:2, 0:2], ora[2:4, 2:4]
    scale = np.abs(left).max()
    assert np.abs(lib - left).max() < tol * scale
    assert np.abs(lib[::-1, ::-1] - right).max() < tol * scale       # the right end is the mirror image
    assert np.abs(ora[0:2, 2:4]).max() < 1e-12 * scale                # the ends do not couple (to rounding)


def test_order0_block(box):
    blocks_agree(abc.abc1d_host_block(N, H, 0, 20.0, abc.MAT_M), order0(box, 20.0)["M"], 1e-13)


def test_order1_limit_blocks(box):
    co = order1(box, 10.0)
    blocks_agree(abc.abc1d_host_block(N, H, 1, 10.0, abc.MAT_A), co["A"], 1e-13)
    blocks_agree(abc.abc1d_host_block(N, H, 1, 10.0, abc.MAT_B), co["B"], 1e-11)


def test_order1_two_point_blocks(box):
    co = order1_two_point(box, 10.0, 20.0)
    for which, key in ((abc.MAT_A, "A"), (abc.MAT_B, "B")):
        blocks_agree(abc.abc1d_host_block(N, H, 1, (10.0, 20.0), which, fit1="two_point"), co[key], 1e-10)


def test_order2_blocks(box):
    """Both sides fix the one null direction of the 1D order-2 fit the same way (the
    hidden root of det(s^2 I - s B1 - B0) at -min(s_j)), so the blocks agree entry by
    entry to the fit's conditioning (eps sigma_1 / sigma_7 of the 8 x 8 system)."""
    pts = (10.0, 11.0, 20.0, 21.0)
    ora = order2(box, pts)
    lib = {}
    for key, which in (("B1", abc.MAT_B1), ("B0", abc.MAT_B0), ("A1", abc.MAT_A1), ("A0", abc.MAT_A0)):
        lib[key] = abc.abc1d_host_block(N, H, 2, pts, which)
        blocks_agree(lib[key], ora[key], 1e-6)
    X = np.concatenate([lib[k] for k in ("B1", "B0", "A1", "A0")], axis=1)
    Ks = [dtn_eval(box, s)[0:2, 0:2] for s in pts]
    assert fit_ok(pts, Ks, X)


@pytest.mark.parametrize("h,n,pts", [(0.01, 1501, (10.0, 11.0, 20.0, 21.0)), (0.02, 400, (1.0, 2.0, 3.0, 10.0)),
                                     (0.1, 60, (0.5, 4.0, 9.0, 30.0))])
def test_order2_fit_properties(h, n, pts):
    """The library's fit at the paper's h = 0.01 and elsewhere: it interpolates K, its
    four roots lie in the left half-plane, the hidden one at -min(s_j)."""
    X = np.concatenate([abc.abc1d_host_block(n, h, 2, pts, w)
                        for w in (abc.MAT_B1, abc.MAT_B0, abc.MAT_A1, abc.MAT_A0)], axis=1)
    _, Ks = end_blocks(h, n, pts)
    assert fit_ok(pts, Ks, X)


def test_rejects_bad_parameters():
    with pytest.raises(abc.AbcError):
        abc.abc1d_host_block(4, H, 1, 10.0, abc.MAT_B)               # n < 8
    with pytest.raises(abc.AbcError):
        abc.abc1d_host_block(N, H, 2, (10.0, 10.0, 20.0, 21.0), abc.MAT_B1)   # repeated point
    with pytest.raises(abc.AbcError):
        abc.abc1d_host_block(N, H, 1, (10.0, 10.0), abc.MAT_B, fit1="two_point")
