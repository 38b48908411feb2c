"""Host set-up of the one-dimensional stepper (include/abc1d.h) against the oracle, on
CPU: the boundary blocks of the five-point scheme (Sec. 4.1, App. B).

The oracle builds K(s) for the whole Gamma of the 1D box (both ends at once) from an
FFT Green's function; the library builds the left end's 2 x 2 block from the closed
form of App. B and mirrors it for the right end.  Orders 0 and 1 must agree to
rounding.  The second-order fit at the paper's points s = 10, 11, 20, 21 is an
ill-conditioned interpolation (two pairs of nearly equal points), so its coefficient
matrices are only determined up to that conditioning: the test checks the
interpolation conditions R_22(s_j) = K(s_j) and the rational function R_22 itself on
the imaginary axis, not the coefficients entry by entry."""
import numpy as np
import pytest

from oracle.coefficients import order0, order1, order1_two_point, order2
from oracle.dtn import dtn_eval
from oracle.lattice import Box
from paper_1908_02456_gb300 import abc

N, H = 40, 0.05


@pytest.fixture(scope="module")
def box():
    return Box((N,), H, 2)


def blocks_agree(lib, ora, tol):
    left, right = ora[0:2, 0:2], ora[2:4, 2:4]
    scale = np.abs(left).max()
    assert np.abs(lib - left).max() < tol * scale
    assert np.abs(lib[::-1, ::-1] - right).max() < tol * scale       # the right end is the mirror image
    assert np.abs(ora[0:2, 2:4]).max() < 1e-14 * scale                # the ends do not couple


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


def test_order2_rational_function(box):
    pts = (10.0, 11.0, 20.0, 21.0)
    lib = {k: abc.abc1d_host_block(N, H, 2, pts, w)
           for k, w in (("B1", abc.MAT_B1), ("B0", abc.MAT_B0), ("A1", abc.MAT_A1), ("A0", abc.MAT_A0))}
    ora = order2(box, pts)

    def r22(c, s):
        return np.linalg.solve(s * s * np.eye(2) - s * c["B1"] - c["B0"], s * c["A1"] + c["A0"])
    left = {k: ora[k][0:2, 0:2] for k in lib}
    for s in pts:                                          # the interpolation conditions
        K = dtn_eval(box, s)[0:2, 0:2]
        assert np.abs(r22(lib, s) - K).max() < 1e-8 * np.abs(K).max()
    for s in (2j, 10j, 50j, 5.0, 30.0):                    # the same rational function
        ref = r22(left, s)
        assert np.abs(r22(lib, s) - ref).max() < 1e-5 * np.abs(ref).max()


def test_rejects_bad_parameters():
    with pytest.raises(abc.AbcError):
        abc.abc1d_host_block(4, H, 1, 10.0, abc.MAT_B)               # n < 8
    with pytest.raises(abc.AbcError):
        abc.abc1d_host_block(N, H, 2, (10.0, 10.0, 20.0, 21.0), abc.MAT_B1)   # repeated point
    with pytest.raises(abc.AbcError):
        abc.abc1d_host_block(N, H, 1, (10.0, 10.0), abc.MAT_B, fit1="two_point")
