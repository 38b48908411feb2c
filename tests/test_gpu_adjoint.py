"""GPU adjoint (gradient of the absorbed probability w.r.t. V) against the FP64
oracle's reverse mode and against central finite differences (marked gpu)."""
import numpy as np
import pytest

from oracle.adjoint import gradient as oracle_gradient
from oracle.coefficients import order0, order1
from oracle.lattice import Box
from oracle.propagate import System
from paper_1908_02456_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_1908_02456_gb300 import abc, build
    build.build()
    assert torch.cuda.is_available()
    return torch, abc


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _gpu_adjoint(torch, abc, dims, h, order, s, prec, psi0, V, dt, steps, ckpt):
    ctx = abc.Context(dims, h, order, s, precision=prec, max_orbitals=psi0.shape[0])
    p = torch.from_numpy(psi0.reshape((psi0.shape[0],) + tuple(dims[::-1]))).to("cuda", ctx.complex_dtype).contiguous()
    Vt = torch.from_numpy(V.reshape(dims[::-1])).to("cuda", ctx.real_dtype).contiguous()
    J, g = ctx.adjoint(p, Vt, dt, steps, ckpt)
    out = J, g.cpu().numpy().reshape(-1).astype(np.float64)
    ctx.close()
    return out


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("b", [1, 2])
def test_adjoint_matches_oracle_fp64(env, order, b):
    """FP64 discrete adjoint vs the oracle's reverse mode of the Taylor form; 30 steps with
    checkpoints every 7 (a ragged last segment)."""
    torch, abc = env
    dims, h, dt, steps = (8, 7, 9), 0.5, 0.01, 30
    rng = np.random.default_rng(20 + order + b)
    V = inputs.smooth_random(dims, h, rng).reshape(-1)
    psi = np.concatenate([inputs.gaussian_packet(dims, h, (0.3 * j, 0, 0), (2.0, 0.5 - j, 0), 1.0)[None]
                          for j in range(b)]).reshape(b, -1)
    box = Box(dims, h)
    co = order0(box, 1.0) if order == 0 else order1(box, 1.0)
    Jo, go = oracle_gradient(System(box, V_ext=V, coeffs=co), psi, dt, steps)
    J, g = _gpu_adjoint(torch, abc, dims, h, order, 1.0, "fp64", psi, V, dt, steps, 7)
    assert abs(J - Jo) < 1e-12 * max(1.0, abs(Jo))
    assert rel(g, go) < 1e-10


def test_adjoint_complex64_vs_fp64(env):
    torch, abc = env
    dims, h, dt, steps = (12, 12, 12), 0.4, 0.005, 120
    w = inputs.WORKLOADS[4]
    psi0, V = inputs.make_inputs(w, n=12)
    J64, g64 = _gpu_adjoint(torch, abc, dims, h, 1, 1.0, "fp64", psi0.reshape(1, -1), V, dt, steps, 50)
    J32, g32 = _gpu_adjoint(torch, abc, dims, h, 1, 1.0, "c64", psi0.reshape(1, -1), V, dt, steps, 50)
    assert abs(J32 - J64) < 1e-5 * max(abs(J64), 1e-3)
    assert rel(g32, g64) < 1e-4


@pytest.mark.parametrize("tc", ["tf32x3", "fp16x3"])
@pytest.mark.parametrize("order", [0, 1])
def test_adjoint_tensor_core_vs_fp64(env, order, tc):
    """Three orbitals through the tensor-core contraction (its conjugated form runs in
    the reverse sweep) against the FP64 gradient, next to the FP32 CUDA-core form."""
    torch, abc = env
    dims, h, dt, steps = (12, 12, 12), 0.4, 0.005, 60
    rng = np.random.default_rng(5 + order)
    V = inputs.smooth_random(dims, h, rng).reshape(-1)
    psi = np.concatenate([inputs.gaussian_packet(dims, h, (0.4 * j - 0.4, 0, 0.2), (2.0, 1.0 - j, 0.5), 1.2)[None]
                          for j in range(3)]).reshape(3, -1)
    J64, g64 = _gpu_adjoint(torch, abc, dims, h, order, 1.0, "fp64", psi, V, dt, steps, 20)
    Jtc, gtc = _gpu_adjoint(torch, abc, dims, h, order, 1.0, tc, psi, V, dt, steps, 20)
    Jc, gc = _gpu_adjoint(torch, abc, dims, h, order, 1.0, "c64", psi, V, dt, steps, 20)
    assert abs(Jtc - J64) < 1e-5 * max(abs(J64), 1e-3)
    # the tensor-core path is as accurate as the FP32 CUDA-core path on the same case
    e_tc, e_c = rel(gtc, g64), rel(gc, g64)
    assert e_tc < max(2.0 * e_c, 1e-5) and e_tc < 1e-3, (e_tc, e_c)


def _absorbed(torch, ctx, psi0, V, dt, steps):
    p = psi0.clone()
    aux = ctx.new_aux(p.shape[0]) if ctx.order == 1 else None
    ctx.run(p, aux, V, dt, steps)
    d = ctx.diagnostics(p, aux, V)
    return float(np.sum(1.0 - d[:, 0]))


@pytest.mark.parametrize("prec", ["fp64", "c64"])
def test_adjoint_full_workload_vs_finite_differences(env, prec):
    """The 48^3 adjoint workload (first-order ABC, 1000 steps, checkpoints every 50):
    <dJ/dV, dV> against central differences of the FP64 forward in 3 seeded smooth
    directions, to 1e-4 relative."""
    torch, abc = env
    w = inputs.WORKLOADS[4]
    psi0, V = inputs.make_inputs(w)
    dims = w.shape
    J, g = _gpu_adjoint(torch, abc, dims, w.h, 1, w.s, prec, psi0.reshape(1, -1), V, w.dt, w.steps, 50)
    ctx = abc.Context(dims, w.h, 1, w.s, precision="fp64")
    p0 = torch.from_numpy(psi0).to("cuda")
    rng = np.random.default_rng(99)
    assert 0.0 < J < 1.0
    for _ in range(3):
        dV = inputs.smooth_random(dims, w.h, rng)
        eps = 1e-3
        Jp = _absorbed(torch, ctx, p0, torch.from_numpy(V + eps * dV).to("cuda"), w.dt, w.steps)
        Jm = _absorbed(torch, ctx, p0, torch.from_numpy(V - eps * dV).to("cuda"), w.dt, w.steps)
        fd = (Jp - Jm) / (2 * eps)
        an = float(g @ dV.reshape(-1))
        assert abs(fd - an) <= 1e-4 * abs(fd), (prec, fd, an)
    ctx.close()


def test_autograd_function(env):
    torch, abc = env
    from paper_1908_02456_gb300.autograd import absorbed_probability
    dims, h, dt, steps = (10, 10, 10), 0.5, 0.01, 40
    psi0 = inputs.gaussian_packet(dims, h, (0, 0, 0), (2.5, 0, 0), 1.0)[None]
    ctx = abc.Context(dims, h, 1, 1.0, precision="fp64")
    V = torch.zeros(dims, dtype=torch.float64, device="cuda", requires_grad=True)
    p = torch.from_numpy(psi0).to("cuda")
    J = absorbed_probability(V, p, ctx, dt, steps, 8)
    (gV,) = torch.autograd.grad(2.0 * J, V)
    J2, g2 = ctx.adjoint(p, V.detach(), dt, steps, 8)
    assert abs(float(J.detach()) - J2) < 1e-14
    assert torch.allclose(gV, 2.0 * g2, rtol=0, atol=1e-14)
    ctx.close()
