"""The order-1 step with the interior stencil fused in time (ABC_TUNE_FUSED) against the
stage-by-stage step and against the FP64 oracle (marked gpu).

The fused form evaluates the same stage formula; only the FP32 rounding of fused
multiply-adds may differ, so after a few steps the two agree to ~1e-6.  The boxes
cover partial tiles in x and y (tiles are 32 x 16), the thinnest box the form
accepts (8 planes), odd step counts (the result comes back from the alternate
buffer), the mean field and the fitted first-order forms."""
import numpy as np
import pytest

from oracle.coefficients import order1
from oracle.lattice import Box
from oracle.propagate import System
from paper_1908_02456_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_1908_02456_gb300 import abc, build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch, abc


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def _run(torch, abc, dims, h, prec, b, fused, steps, mf, fit1="limit", s1b=0.0, diag_every=0):
    ctx = abc.Context(dims, h, 1, 1.0, precision=prec, max_orbitals=b, fit1=fit1, s1b=s1b)
    ctx.set_tuning(abc.TUNE_FUSED, fused)
    rng = np.random.default_rng(11 + b)
    psi0 = inputs.orbital_set(dims, h, rng, b)
    V = inputs.smooth_random(dims, h, rng)
    psi = torch.from_numpy(psi0).to("cuda", ctx.complex_dtype).contiguous()
    aux = ctx.new_aux(b)
    Vt = torch.from_numpy(V).to("cuda", ctx.real_dtype).contiguous()
    d = ctx.run(psi, aux, Vt, 0.005, steps, meanfield=mf, diag_every=diag_every)
    torch.cuda.synchronize()
    out = (psi.cpu().numpy().astype(np.complex128), aux.cpu().numpy().astype(np.complex128), d)
    ctx.close()
    return out, psi0, V


@pytest.mark.parametrize("dims,b,prec,fit1,mf", [
    ((16, 16, 16), 3, "c64", "limit", None),
    ((18, 20, 9), 2, "tf32x3", "limit", (-1.0, 0.8, 1.0 / 6.0)),
    ((34, 17, 8), 4, "fp16x3", "limit", (-20.0, 10.0, 1.0 / 6.0)),
    ((14, 12, 11), 1, "c64", "limit", None),
    ((16, 14, 12), 2, "c64", "two_point", None),
])
@pytest.mark.parametrize("steps", [1, 6, 7])
def test_fused_matches_stage_by_stage(env, dims, b, prec, fit1, mf, steps):
    torch, abc = env
    s1b = 2.0 if fit1 == "two_point" else 0.0
    (p0, f0, d0), _, _ = _run(torch, abc, dims, 0.45, prec, b, 0, steps, mf, fit1, s1b, diag_every=1)
    (p1, f1, d1), _, _ = _run(torch, abc, dims, 0.45, prec, b, 1, steps, mf, fit1, s1b, diag_every=1)
    assert rel(p1, p0) < 2e-6
    assert rel(f1, f0) < 2e-6
    assert rel(d1, d0) < 2e-6


def test_fused_meanfield_against_oracle(env):
    """Five orbitals of the mean field on a 14^3 box, 60 steps, fused form vs the FP64
    oracle at the reduced-precision tolerance."""
    torch, abc = env
    dims, h, b, steps = (14, 14, 14), 0.45, 5, 60
    mf = (-1.0, 0.8, 1.0 / 6.0)
    (p, f, d), psi0, V = _run(torch, abc, dims, h, "c64", b, 1, steps, mf, diag_every=20)
    box = Box(dims, h)
    sy = System(box, V_ext=V.reshape(-1), coeffs=order1(box, 1.0), meanfield=mf)
    ref_p, ref_f, ref_d = sy.run(psi0.reshape(b, -1), 0.005, steps, diag_every=20)
    assert rel(p.reshape(b, -1), ref_p) < 1e-5
    assert rel(f.T, ref_f) < 1e-5
    assert rel(d, ref_d) < 1e-5
