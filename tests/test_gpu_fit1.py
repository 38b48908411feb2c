"""The two-point and Hermite first-order fits (Sec. 3.2's finite-s2 remark, eq:39) on
the GPU against the FP64 oracle (marked gpu): runs from f = 0 on a cube and on a box
with unequal odd axes, one and three orbitals, element by element (1e-10 FP64,
1e-5 complex64 relative L2), through the dense class-block rows [B | A]."""
import ctypes

import numpy as np
import pytest

from oracle.coefficients import order1_hermite, order1_two_point
from oracle.lattice import Box
from oracle.propagate import System
from paper_1908_02456_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "c64": 1e-5, "tf32x3": 1e-5}


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    from paper_1908_02456_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _coeffs(box, fit):
    return order1_two_point(box, 1.0, 2.0) if fit == "two_point" else order1_hermite(box, 1.0)


@pytest.mark.parametrize("dims,b", [((8, 8, 8), 1), ((7, 6, 9), 3)])
@pytest.mark.parametrize("prec", ["fp64", "c64", "tf32x3"])
@pytest.mark.parametrize("fit", ["two_point", "hermite"])
def test_fit1_run_matches_oracle(torch_cuda, dims, b, prec, fit):
    torch = torch_cuda
    from paper_1908_02456_gb300 import abc
    h, dt, steps = 0.5, 0.01, 40
    rng = np.random.default_rng(80 + b)
    V = inputs.smooth_random(dims, h, rng)
    psi0 = np.concatenate([inputs.gaussian_packet(dims, h, (0.3 * j, -0.2, 0.1), (2.0, 0.5 * j, -1.0), 1.0)[None]
                           for j in range(b)])
    box = Box(dims, h)
    sy = System(box, V_ext=V.reshape(-1), coeffs=_coeffs(box, fit))
    ctx = abc.Context(dims, h, 1, 1.0, precision=prec, max_orbitals=b, fit1=fit, s1b=2.0)
    psi = torch.from_numpy(psi0).to("cuda", ctx.complex_dtype).contiguous()
    Vt = torch.from_numpy(V).to("cuda", ctx.real_dtype).contiguous()
    aux = ctx.new_aux(b)
    ref_p, ref_f, ref_d = sy.run(psi0.reshape(b, -1), dt, steps, diag_every=10)
    d = ctx.run(psi, aux, Vt, dt, steps, diag_every=10)
    torch.cuda.synchronize()
    assert rel(psi.cpu().numpy().reshape(b, -1), ref_p) < TOL[prec]
    assert rel(aux.cpu().numpy().T, ref_f) < TOL[prec]
    assert rel(d, ref_d) < TOL[prec]
    ctx.close()


def test_fit1_matrices_from_device_context(torch_cuda):
    """abc_get_matrices returns the context's own fitted B and A (natural order)."""
    from paper_1908_02456_gb300 import abc
    dims, h = (6, 7, 5), 0.5
    box = Box(dims, h)
    co = _coeffs(box, "hermite")
    ctx = abc.Context(dims, h, 1, 1.0, precision="c64", fit1="hermite")
    for which, key in [(abc.MAT_B, "B"), (abc.MAT_A, "A")]:
        X = ctx.matrix(which)
        assert np.abs(X - co[key]).max() < 1e-9 * np.abs(co[key]).max(), key
    ctx.close()


def test_fit1_refuses_adjoint_and_noalloc(torch_cuda):
    torch = torch_cuda
    from paper_1908_02456_gb300 import abc
    ctx = abc.Context((6, 6, 6), 0.5, 1, 1.0, precision="fp64", fit1="two_point", s1b=2.0)
    p = torch.zeros((1, 6, 6, 6), dtype=torch.complex128, device="cuda")
    V = torch.zeros((6, 6, 6), dtype=torch.float64, device="cuda")
    lib = abc.load()
    J = ctypes.c_double()
    g = torch.zeros_like(V)
    assert lib.abc_adjoint_run(ctx.ctx, p.data_ptr(), V.data_ptr(), 1, 0.01, 2, 1, ctypes.byref(J), g.data_ptr(),
                               None) == 7
    aux = ctx.new_aux(1)
    assert lib.abc_step_noalloc(ctx.ctx, p.data_ptr(), aux.data_ptr(), V.data_ptr(), 1, 0.01, None) == 7
    ctx.close()
