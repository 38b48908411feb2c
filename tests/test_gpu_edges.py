"""Edge cases of the GPU path (marked gpu), element by element against the FP64 oracle
or exactly:

* the smallest boxes the radius-1 stencil admits, 3 nodes per axis (Gamma is every
  node but the centre) and 3 x 4 x 5, for orders 0, 1 and 2, in FP64, complex64 with
  one and three orbitals, and on the tensor cores with five orbitals (a ragged group of
  the four-orbital transforms and a 16-column tile holding five);
* zero steps (the state is returned bit for bit) and the zero state (it stays exactly
  zero, its norms and W are zero, and the divergence monitor stays quiet);
* orbital counts at the context's limit and past it (refused with ABC_ERR_ARG), and
  a run with fewer orbitals than the context was set up for."""
import numpy as np
import pytest

from oracle.coefficients import order0, order1, order2
from oracle.lattice import Box
from oracle.propagate import System
from paper_1908_02456_gb300 import inputs

pytestmark = pytest.mark.gpu

PTS = (1.0, 2.0, 3.0, 10.0)
TOL = {"fp64": 1e-10, "c64": 1e-5, "tf32x3": 1e-5, "fp16x3": 1e-5}


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_1908_02456_gb300 import abc, build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch, abc


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def coeffs(box, order):
    return order0(box, 1.0) if order == 0 else order1(box, 1.0) if order == 1 else order2(box, PTS)


def aux_to_oracle(aux, order):
    a = aux.cpu().numpy().astype(np.complex128)
    if order == 2:                                   # [2][n_gamma][b] -> (b, 2 n_gamma)
        return a.transpose(2, 0, 1).reshape(a.shape[2], -1)
    return a.T                                       # [n_gamma][b] -> (b, n_gamma)


@pytest.mark.parametrize("dims", [(3, 3, 3), (3, 4, 5)])
@pytest.mark.parametrize("order", [0, 1, 2])
@pytest.mark.parametrize("prec,b", [("fp64", 1), ("c64", 1), ("c64", 3), ("fp16x3", 5), ("tf32x3", 5)])
def test_smallest_boxes_vs_oracle(env, dims, order, prec, b):
    torch, abc = env
    if order == 2 and prec == "fp16x3":
        prec = "c64"                                 # the tensor-core forms cover orders 0 and 1
    h, dt, steps = 0.5, 0.004, 30
    rng = np.random.default_rng(400 + 10 * order + b + dims[2])
    psi0 = inputs.random_state(dims, b, rng)
    V = rng.uniform(-0.5, 0.5, size=dims[::-1])
    box = Box(dims, h)
    sy = System(box, V_ext=V.reshape(-1), coeffs=coeffs(box, order))
    ctx = abc.Context(dims, h, order, PTS if order == 2 else 1.0, precision=prec, max_orbitals=b)
    psi = torch.from_numpy(psi0).to("cuda", ctx.complex_dtype).contiguous()
    Vt = torch.from_numpy(V).to("cuda", ctx.real_dtype).contiguous()
    aux = ctx.init_aux(psi) if order == 2 else ctx.new_aux(b)
    ref_p, ref_a, ref_d = sy.run(psi0.reshape(b, -1), dt, steps, diag_every=10)
    d = ctx.run(psi, aux, Vt, dt, steps, diag_every=10)
    torch.cuda.synchronize()
    assert rel(psi.cpu().numpy().reshape(b, -1), ref_p) < TOL[prec]
    if order >= 1:
        assert rel(aux_to_oracle(aux, order), ref_a) < TOL[prec]
    assert rel(d[:, :, 0], ref_d[:, :, 0]) < TOL[prec]
    ctx.close()


@pytest.mark.parametrize("prec,b", [("fp64", 1), ("c64", 1), ("fp16x3", 8)])
def test_zero_steps_and_zero_state(env, prec, b):
    torch, abc = env
    dims, h, dt = (10, 9, 8), 0.5, 0.005
    ctx = abc.Context(dims, h, 1, 1.0, precision=prec, max_orbitals=b)
    psi0 = inputs.random_state(dims, b, np.random.default_rng(5))
    psi = torch.from_numpy(psi0).to("cuda", ctx.complex_dtype).contiguous()
    aux = ctx.new_aux(b)
    aux.normal_()
    V = torch.zeros(dims[::-1], dtype=ctx.real_dtype, device="cuda")
    p_before, a_before = psi.clone(), aux.clone()
    ctx.run(psi, aux, V, dt, 0)
    torch.cuda.synchronize()
    assert torch.equal(psi, p_before) and torch.equal(aux, a_before)
    psi.zero_()
    aux.zero_()
    d = ctx.run(psi, aux, V, dt, 12, meanfield=(-1.0, 0.8, 1.0 / 6.0), diag_every=4)
    torch.cuda.synchronize()
    assert not torch.any(psi != 0) and not torch.any(aux != 0)
    assert np.all(d[:, :, :2] == 0.0)
    ctx.close()


def test_orbital_count_limits(env):
    torch, abc = env
    dims, h, dt, bmax = (8, 8, 8), 0.5, 0.005, 4
    ctx = abc.Context(dims, h, 1, 1.0, precision="c64", max_orbitals=bmax)
    V = torch.zeros(dims[::-1], dtype=torch.float32, device="cuda")
    over = torch.zeros((bmax + 1,) + dims[::-1], dtype=torch.complex64, device="cuda")
    with pytest.raises(abc.AbcError) as e:
        ctx.run(over, ctx.new_aux(bmax + 1), V, dt, 1)
    assert e.value.status == 1
    # fewer orbitals than the context holds, and exactly as many: both match the oracle
    box = Box(dims, h)
    for b in (3, bmax):
        psi0 = inputs.random_state(dims, b, np.random.default_rng(50 + b))
        sy = System(box, coeffs=order1(box, 1.0))
        ref_p, ref_f, _ = sy.run(psi0.reshape(b, -1), dt, 10)
        psi = torch.from_numpy(psi0).to("cuda", torch.complex64).contiguous()
        aux = ctx.new_aux(b)
        ctx.run(psi, aux, V, dt, 10)
        torch.cuda.synchronize()
        assert rel(psi.cpu().numpy().reshape(b, -1), ref_p) < 1e-5
        assert rel(aux.cpu().numpy().astype(np.complex128).T, ref_f) < 1e-5
    ctx.close()
