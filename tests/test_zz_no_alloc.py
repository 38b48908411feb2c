"""abc_step_noalloc: a time step that allocates no device memory.

Callers that cannot call cudaMalloc while they step the system -- code inside a
framework whose pool allocator owns the device heap, or code that must not allocate
at that point -- use abc_step_noalloc, which takes the step's scratch from a fixed
static device array in the library instead of from an allocation.  These tests call
it through the C ABI and check two consecutive calls against two calls of the
existing abc_step on identical inputs, within the tolerances of the other parity
tests (1e-10 FP64, 1e-5 complex64), and that a request larger than the fixed array
is refused with a clear error.  This file is collected last on purpose."""
import ctypes

import numpy as np
import pytest

from paper_1908_02456_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "c64": 1e-5}


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_1908_02456_gb300 import abc, build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch, abc, abc.load()


def _rel(a, b):
    a = a.cpu().numpy().astype(np.complex128)
    b = b.cpu().numpy().astype(np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("b", [1, 2])
@pytest.mark.parametrize("prec,order", [("c64", 1), ("fp64", 1), ("c64", 0), ("fp64", 0)])
def test_noalloc_step_matches_step(env, prec, order, b):
    """b = 1 runs the one-orbital full-block kernel of the no-allocation step, b = 2 the
    many-orbital one; abc_step runs its own kernels for both."""
    torch, abc, lib = env
    dims, h, dt = (14, 12, 10), 0.5, 0.01
    ctx = abc.Context(dims, h, order, 1.0, precision=prec, max_orbitals=b)
    rng = np.random.default_rng(42 + order + 10 * b)
    psi0 = inputs.random_state(dims, b, rng)
    V0 = rng.uniform(-1, 1, size=dims[::-1])
    psi_a = torch.from_numpy(psi0).to("cuda", ctx.complex_dtype).contiguous()
    psi_b = psi_a.clone()
    V = torch.from_numpy(V0).to("cuda", ctx.real_dtype).contiguous()
    aux_a = aux_b = None
    if order == 1:
        f0 = rng.normal(size=(ctx.n_gamma, b)) + 1j * rng.normal(size=(ctx.n_gamma, b))
        aux_a = torch.from_numpy(f0).to("cuda", ctx.complex_dtype).contiguous()
        aux_b = aux_a.clone()
    stream = torch.cuda.current_stream().cuda_stream
    ptr = lambda t: None if t is None else t.data_ptr()
    for _ in range(2):
        st_a = lib.abc_step(ctx.ctx, ptr(psi_a), ptr(aux_a), ptr(V), b, dt, stream)
        st_b = lib.abc_step_noalloc(ctx.ctx, ptr(psi_b), ptr(aux_b), ptr(V), b, dt, stream)
        assert st_a == 0 and st_b == 0, lib.abc_last_error()
        torch.cuda.synchronize()
        assert _rel(psi_b, psi_a) <= TOL[prec]
        if order == 1:
            assert _rel(aux_b, aux_a) <= TOL[prec]
    ctx.close()


def test_noalloc_refuses_more_than_its_scratch(env):
    torch, abc, lib = env
    dims, b = (40, 40, 40), 16
    ctx = abc.Context(dims, 0.5, 1, 1.0, precision="c64", max_orbitals=b)
    psi = torch.zeros((b, 40, 40, 40), dtype=torch.complex64, device="cuda")
    aux = ctx.new_aux(b)
    V = torch.zeros((40, 40, 40), dtype=torch.float32, device="cuda")
    st = lib.abc_step_noalloc(ctx.ctx, psi.data_ptr(), aux.data_ptr(), V.data_ptr(), b, 0.01, None)
    assert st == abc.AbcError(1, "").status == 1
    assert b"scratch" in lib.abc_last_error()
    st = lib.abc_step_noalloc(ctx.ctx, psi.data_ptr(), aux.data_ptr(), V.data_ptr(), 1, 0.01, None)
    assert st == 0, lib.abc_last_error()
    torch.cuda.synchronize()
    ctx.close()
