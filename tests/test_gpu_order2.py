"""Second-order ABC (Sec. 3.3, eq:dynamics2) on the GPU against the FP64 oracle
(marked gpu): the consistent initial auxiliary state (f = 0, g = A1 E psi) and runs
from it, element by element, on a cube (irreducible classes) and a box with unequal
odd axes, one and three orbitals, FP64 and complex64 (1e-10 / 1e-5 relative L2)."""
import numpy as np
import pytest

from oracle.coefficients import order2
from oracle.lattice import Box
from oracle.propagate import System
from paper_1908_02456_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "c64": 1e-5, "tf32x3": 1e-5}
PTS = (1.0, 2.0, 3.0, 10.0)


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    from paper_1908_02456_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _aux_to_oracle(aux):
    """[2][n_gamma][b] -> (b, 2 n_gamma) = [f | g] per orbital."""
    a = aux.cpu().numpy().astype(np.complex128)
    return a.transpose(2, 0, 1).reshape(a.shape[2], -1)


@pytest.mark.parametrize("dims,b", [((8, 8, 8), 1), ((7, 6, 9), 3)])
@pytest.mark.parametrize("prec", ["fp64", "c64", "tf32x3"])
def test_order2_run_matches_oracle(torch_cuda, dims, b, prec):
    torch = torch_cuda
    from paper_1908_02456_gb300 import abc
    h, dt, steps = 0.5, 0.01, 40
    rng = np.random.default_rng(60 + b)
    V = inputs.smooth_random(dims, h, rng)
    psi0 = np.concatenate([inputs.gaussian_packet(dims, h, (0.3 * j, -0.2, 0.1), (2.0, 0.5 * j, -1.0), 1.0)[None]
                           for j in range(b)])
    sy = System(Box(dims, h), V_ext=V.reshape(-1), coeffs=order2(Box(dims, h), PTS))
    ctx = abc.Context(dims, h, 2, PTS, precision=prec, max_orbitals=b)
    psi = torch.from_numpy(psi0).to("cuda", ctx.complex_dtype).contiguous()
    Vt = torch.from_numpy(V).to("cuda", ctx.real_dtype).contiguous()
    aux = ctx.init_aux(psi)
    torch.cuda.synchronize()
    a0 = sy.initial_aux(psi0.reshape(b, -1))
    assert rel(_aux_to_oracle(aux), a0) < (1e-12 if prec == "fp64" else 1e-6)
    ref_p, ref_a, ref_d = sy.run(psi0.reshape(b, -1), dt, steps, diag_every=10)
    d = ctx.run(psi, aux, Vt, dt, steps, diag_every=10)
    torch.cuda.synchronize()
    assert rel(psi.cpu().numpy().reshape(b, -1), ref_p) < TOL[prec]
    assert rel(_aux_to_oracle(aux), ref_a) < TOL[prec]
    assert rel(d, ref_d) < TOL[prec]
    assert d[-1, 0, 0] < d[0, 0, 0]                    # the packet is being absorbed
    ctx.close()


def test_order2_refuses_adjoint_and_noalloc(torch_cuda):
    torch = torch_cuda
    from paper_1908_02456_gb300 import abc
    dims = (6, 6, 6)
    ctx = abc.Context(dims, 0.5, 2, PTS, precision="fp64", max_orbitals=1)
    p = torch.zeros((1, 6, 6, 6), dtype=torch.complex128, device="cuda")
    V = torch.zeros((6, 6, 6), dtype=torch.float64, device="cuda")
    lib = abc.load()
    import ctypes
    J = ctypes.c_double()
    g = torch.zeros_like(V)
    assert lib.abc_adjoint_run(ctx.ctx, p.data_ptr(), V.data_ptr(), 1, 0.01, 2, 1, ctypes.byref(J), g.data_ptr(),
                               None) == 7
    aux = ctx.new_aux(1)
    assert lib.abc_step_noalloc(ctx.ctx, p.data_ptr(), aux.data_ptr(), V.data_ptr(), 1, 0.01, None) == 7
    ctx.close()
