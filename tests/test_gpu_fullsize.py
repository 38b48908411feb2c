"""Parity at the workloads' full sizes and step counts (marked gpu and slow).

The reduced-precision forms are compared element by element (relative L2 per result:
psi of every orbital, f, and the norm / W / energy series) with

* the FP64 oracle directly where it finishes in about a minute (32^3, one orbital,
  1000 steps; 32^3 with 32 mean-field orbitals, 100 steps), and
* the FP64 GPU path (held to the oracle at 1e-10 by the small-box tests) at the full
  sizes: the 64^3 single-orbital workload for its 2000 steps, the 64^3 x 32
  mean-field workload for its 1000 steps, and the 96^3 x 128 mean-field workload for
  50 of its 500 steps (the FP64 form takes about a second per step there).

Tolerances: 1e-5 for the complex64 forms (FP32 CUDA cores, 3xTF32, split FP16).  The
auxiliary variable f is held to that bound in the norm of the Lyapunov functional W of
Thm 3.2 (|d phi|^2 + d f^* Q d f over |phi|^2 + f^* Q f, Q = 4 h^4 / c_gamma): in the
harmonic-well workload the packet stays trapped, f is ~1e-8 of the state, and the FP32
rounding noise that reaches the boundary (its high-wavenumber part is not held back by
the well) is ~1e-3 of f itself, so a bare relative error of f is reported with a looser
bound beside the W-norm one."""
import numpy as np
import pytest

from oracle.coefficients import order1
from oracle.lattice import Box
from oracle.propagate import System
from paper_1908_02456_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL = 1e-5


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_1908_02456_gb300 import abc, build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch, abc


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def exterior_counts(n):
    """c_gamma (faces the node lies on) for the Gamma nodes of an n^3 box, ascending order."""
    i = np.arange(n)
    on = (i == 0).astype(int) + (i == n - 1)
    c = on[None, None, :] + on[None, :, None] + on[:, None, None]
    return c.reshape(-1)[c.reshape(-1) > 0]


def rel_w(p, f, p_ref, f_ref, n, h):
    """Relative error of (phi, f) in the W norm (radius 1)."""
    q = 4.0 * h ** 4 / exterior_counts(n)
    num = h ** 3 * np.sum(np.abs(p - p_ref) ** 2) + np.sum(q[None, :] * np.abs(f - f_ref) ** 2)
    den = h ** 3 * np.sum(np.abs(p_ref) ** 2) + np.sum(q[None, :] * np.abs(f_ref) ** 2)
    return float(np.sqrt(num / den))


def gpu(torch, abc, w, prec, psi0, V, steps, diag_every, n=None):
    dims = (n or w.n,) * 3
    b = psi0.shape[0]
    ctx = abc.Context(dims, w.h, 1, w.s, precision=prec, max_orbitals=b)
    psi = torch.from_numpy(psi0).to("cuda", ctx.complex_dtype).contiguous()
    aux = ctx.new_aux(b)
    Vt = torch.from_numpy(V).to("cuda", ctx.real_dtype).contiguous()
    d = ctx.run(psi, aux, Vt, w.dt, steps, meanfield=w.meanfield, diag_every=diag_every)
    torch.cuda.synchronize()
    out = (psi.cpu().numpy().reshape(b, -1).astype(np.complex128), aux.cpu().numpy().T.astype(np.complex128), d)
    ctx.close()
    return out


@pytest.fixture(scope="module")
def oracle32():
    """The order-1 coefficients of the 32^3, h = 0.4 box (the oracle's own set-up)."""
    box = Box((32, 32, 32), 0.4)
    return box, order1(box, 1.0)


def test_single_orbital_32cube_1000_steps_vs_oracle(env, oracle32):
    torch, abc = env
    w = inputs.WORKLOADS[2]
    box, co = oracle32
    psi0, V = inputs.make_inputs(w, n=32)
    ref_p, ref_f, ref_d = System(box, V_ext=V.reshape(-1), coeffs=co).run(psi0.reshape(1, -1), w.dt, 1000,
                                                                         diag_every=100)
    p, f, d = gpu(torch, abc, w, "c64", psi0, V, 1000, 100, n=32)
    assert rel(p, ref_p) < TOL
    assert rel(f, ref_f) < TOL
    assert rel(d, ref_d) < TOL


@pytest.mark.parametrize("prec", ["fp16x3", "tf32x3"])
def test_meanfield_32cube_32orb_vs_oracle(env, oracle32, prec):
    torch, abc = env
    w = inputs.WORKLOADS[3]
    box, co = oracle32
    psi0, V = inputs.make_inputs(w, n=32)
    ref_p, ref_f, ref_d = System(box, V_ext=V.reshape(-1), coeffs=co, meanfield=w.meanfield).run(
        psi0.reshape(w.n_orb, -1), w.dt, 100, diag_every=25)
    p, f, d = gpu(torch, abc, w, prec, psi0, V, 100, 25, n=32)
    assert rel(p, ref_p) < TOL
    assert rel(f, ref_f) < TOL
    assert rel(d, ref_d) < TOL


def test_single_orbital_64cube_2000_steps_vs_fp64(env):
    torch, abc = env
    w = inputs.WORKLOADS[2]
    psi0, V = inputs.make_inputs(w)
    p64, f64, d64 = gpu(torch, abc, w, "fp64", psi0, V, w.steps, 200)
    p, f, d = gpu(torch, abc, w, "c64", psi0, V, w.steps, 200)
    assert rel(p, p64) < TOL
    assert rel_w(p, f, p64, f64, w.n, w.h) < TOL
    assert rel(f, f64) < 1e-2                    # measured 4.7e-3: f is ~1e-8 of the state here
    assert rel(d, d64) < TOL


_FP64_RUNS = {}


@pytest.mark.parametrize("prec", ["fp16x3", "tf32x3", "c64"])
def test_meanfield_64cube_32orb_1000_steps_vs_fp64(env, prec):
    torch, abc = env
    w = inputs.WORKLOADS[3]
    psi0, V = inputs.make_inputs(w)
    if w.name not in _FP64_RUNS:                 # one FP64 run serves the three forms
        _FP64_RUNS[w.name] = gpu(torch, abc, w, "fp64", psi0, V, w.steps, 100)
    p64, f64, d64 = _FP64_RUNS[w.name]
    p, f, d = gpu(torch, abc, w, prec, psi0, V, w.steps, 100)
    assert rel(p, p64) < TOL
    assert rel(f, f64) < TOL
    assert rel(d, d64) < TOL


def test_meanfield_96cube_128orb_vs_fp64(env):
    torch, abc = env
    w = inputs.WORKLOADS[5]
    psi0, V = inputs.make_inputs(w)
    steps = 50
    p64, f64, d64 = gpu(torch, abc, w, "fp64", psi0, V, steps, 10)
    p, f, d = gpu(torch, abc, w, "fp16x3", psi0, V, steps, 10)
    assert rel(p, p64) < TOL
    assert rel(f, f64) < TOL
    assert rel(d, d64) < TOL
    # per orbital as well: no orbital hides behind the others' norm
    for j in range(0, w.n_orb, 17):
        assert rel(p[j], p64[j]) < TOL
