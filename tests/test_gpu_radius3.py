"""Radius 3 (the "7-point scheme in each direction" of Sec. 4.2) on the GPU against the
FP64 oracle (marked gpu): a Gamma three nodes deep, the 19-point interior stencil,
order 0 (packed symmetric tiles for one complex64 orbital) and order 1 (Thm 3.2's fit
and the two-point fit, both as dense class rows [B | A], since A = -i H_{Gamma,II}
H_{II,Gamma} is not diagonal), a cube (irreducible classes) and a box with unequal odd
axes, one and three orbitals, element by element; order 2 in FP64; and the paper's 31^3
experiment with orders 0, 1 and 2."""
import numpy as np
import pytest

from oracle.coefficients import order0, order1, order1_two_point, order2
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


def _coeffs(box, order, fit):
    if order == 0:
        return order0(box, 1.0)
    return order1(box, 1.0) if fit == "limit" else order1_two_point(box, 1.0, 2.0)


@pytest.mark.parametrize("dims,b", [((9, 9, 9), 1), ((8, 7, 9), 3)])
@pytest.mark.parametrize("prec", ["fp64", "c64", "tf32x3"])
@pytest.mark.parametrize("order,fit", [(0, "limit"), (1, "limit"), (1, "two_point")])
def test_radius3_run_matches_oracle(torch_cuda, dims, b, prec, order, fit):
    torch = torch_cuda
    from paper_1908_02456_gb300 import abc
    h, dt, steps = 0.5, 0.005, 40
    rng = np.random.default_rng(90 + b)
    V = inputs.smooth_random(dims, h, rng)
    psi0 = np.concatenate([inputs.gaussian_packet(dims, h, (0.3 * j, -0.2, 0.1), (2.0, 0.5 * j, -1.0), 1.0)[None]
                           for j in range(b)])
    box = Box(dims, h, 3)
    sy = System(box, V_ext=V.reshape(-1), coeffs=_coeffs(box, order, fit))
    ctx = abc.Context(dims, h, order, 1.0, precision=prec, max_orbitals=b, fit1=fit, s1b=2.0, radius=3)
    assert ctx.n_gamma == np.prod(dims) - np.prod([n - 6 for n in dims])
    psi = torch.from_numpy(psi0).to("cuda", ctx.complex_dtype).contiguous()
    Vt = torch.from_numpy(V).to("cuda", ctx.real_dtype).contiguous()
    aux = ctx.new_aux(b) if order == 1 else None
    ref_p, ref_f, ref_d = sy.run(psi0.reshape(b, -1), dt, steps, diag_every=10)
    d = ctx.run(psi, aux, Vt, dt, steps, diag_every=10)
    torch.cuda.synchronize()
    assert rel(psi.cpu().numpy().reshape(b, -1), ref_p) < TOL[prec]
    if order == 1:
        # Thm 3.2's B = s1 I - A K(s1)^{-1} at radius 3: K and H H have condition numbers
        # near 3e8 on these boxes, so two FP64 setups (library by class blocks, oracle
        # dense) agree on B only to cond * eps ~ 3e-8 (pinned on the CPU through the
        # interpolation condition); f inherits that in FP64, phi does not
        tol_f = 1e-8 if (prec == "fp64" and fit == "limit") else TOL[prec]
        assert rel(aux.cpu().numpy().T, ref_f) < tol_f
    # norm and energy as the oracle (W: with radius 3 the library reports |phi|^2)
    assert rel(d[:, :, 0], ref_d[:, :, 0]) < TOL[prec]
    assert rel(d[:, :, 2], ref_d[:, :, 2]) < TOL[prec]
    ctx.close()


@pytest.mark.parametrize("dims,b", [((9, 8, 9), 2), ((8, 8, 8), 1)])
def test_radius3_order2_matches_oracle(torch_cuda, dims, b):
    """The second-order ABC (s = 1, 2, 3, 10 as in Sec. 4.2) with the radius-3 stencil, in
    FP64 (the library refuses complex64 here: its fitted entries near 1e5 cancel and
    FP32 drifts by ~1e-4).  The four-point system is nearly singular, so its solution is
    a family; both sides take the basic solution of a column-pivoted QR, the oracle on
    the natural-order system, the library per irreducible class, i.e. in another basis,
    so they pick different members (coefficients differing O(1)) that both interpolate K
    to ~1e-9 with every root of det(s^2 I - s B1 - B0) at Re <= ~1e-13 here
    (`tests/test_library_host.py`, `tests/test_oracle_order2.py`).  The trajectories they
    drive differ by 3e-7 to 7e-7 (phi) and 2e-4 to 3e-4 ([f | g]) after 40 steps on these
    boxes (measured with both coefficient sets in the oracle's stepper), so phi is held
    to 3e-6 and the auxiliary state to 1e-3."""
    torch = torch_cuda
    from paper_1908_02456_gb300 import abc
    prec = "fp64"
    h, dt, steps = 0.5, 0.005, 40
    pts = (1.0, 2.0, 3.0, 10.0)
    rng = np.random.default_rng(95)
    V = inputs.smooth_random(dims, h, rng)
    psi0 = np.concatenate([inputs.gaussian_packet(dims, h, (0.2 * j, 0.1, -0.1), (2.0, -0.5 * j, 1.0), 1.0)[None]
                           for j in range(b)])
    box = Box(dims, h, 3)
    sy = System(box, V_ext=V.reshape(-1), coeffs=order2(box, pts))
    ctx = abc.Context(dims, h, 2, pts, precision=prec, max_orbitals=b, radius=3)
    psi = torch.from_numpy(psi0).to("cuda", ctx.complex_dtype).contiguous()
    Vt = torch.from_numpy(V).to("cuda", ctx.real_dtype).contiguous()
    aux = ctx.init_aux(psi)
    ref_p, ref_a, _ = sy.run(psi0.reshape(b, -1), dt, steps, f0=sy.initial_aux(psi0.reshape(b, -1)))
    ctx.run(psi, aux, Vt, dt, steps)
    torch.cuda.synchronize()
    assert rel(psi.cpu().numpy().reshape(b, -1), ref_p) < 3e-6
    a = aux.cpu().numpy().astype(np.complex128)
    assert rel(a.transpose(2, 0, 1).reshape(b, -1), ref_a) < 1e-3


def test_radius3_refuses_adjoint_and_noalloc(torch_cuda):
    import ctypes
    torch = torch_cuda
    from paper_1908_02456_gb300 import abc
    ctx = abc.Context((8, 8, 8), 0.5, 1, 1.0, precision="fp64", radius=3)
    p = torch.zeros((1, 8, 8, 8), dtype=torch.complex128, device="cuda")
    V = torch.zeros((8, 8, 8), dtype=torch.float64, device="cuda")
    lib = abc.load()
    J = ctypes.c_double()
    g = torch.zeros_like(V)
    assert lib.abc_adjoint_run(ctx.ctx, p.data_ptr(), V.data_ptr(), 1, 0.01, 2, 1, ctypes.byref(J), g.data_ptr(),
                               None) == 7
    aux = ctx.new_aux(1)
    assert lib.abc_step_noalloc(ctx.ctx, p.data_ptr(), aux.data_ptr(), V.data_ptr(), 1, 0.01, None) == 7
    ctx.close()
    with pytest.raises(abc.AbcError) as e:
        abc.Context((8, 8, 8), 0.5, 2, (1.0, 2.0, 3.0, 10.0), precision="c64", radius=3)
    assert e.value.status == 7


def test_paper_3d_experiment_replay(torch_cuda):
    """Sec. 4.2's experiment: box [-1.5, 1.5]^3 at h = 0.1 (31^3, 7 points per axis,
    n_Gamma = 14166), the free packet of eq:15 with k0 = 5, dt = 0.001, 600 steps.  The
    paper reports for the number of electrons in the box that about 20 % is reflected
    with the first-order ABC fitted at s = 1, 2; read here as the norm left in the box
    minus the closed form's norm in the box at t = 0.6.  Before the packet reaches the
    faces (t = 0.1) the run follows eq:15 up to the discretisation and the first
    absorption (< 7 %).  The zeroth order (s0 = 1) reflects more.  The second order at
    s = 1, 2, 3, 10 (FP64; its nearly singular four-point fit taken as the basic solution
    of a column-pivoted QR) reflects far less, as the paper reports (measured 0.011
    against 0.198), and stays stable: the norm keeps falling over 2400 further steps."""
    torch = torch_cuda
    from oracle.exact import free_packet
    from paper_1908_02456_gb300 import abc
    w1 = inputs.WORKLOADS[9]
    dims, h, dt = w1.shape, w1.h, w1.dt
    psi0, V = inputs.make_inputs(w1)
    ax = (np.arange(dims[0]) - 0.5 * (dims[0] - 1)) * h
    Z, Y, X = np.meshgrid(ax, ax, ax, indexing="ij")
    ex0 = free_packet([X, Y, Z], 0.0, (0, 0, 0), (5.0, 0, 0), 0.5)
    scale = psi0[0][0, 0, 0] / ex0[0, 0, 0]             # the inputs are h^3-normalised
    res = {}
    runs = [("order0", 0, 1.0, "c64", {}), ("order1", 1, 1.0, "c64", dict(fit1="two_point", s1b=2.0)),
            ("order2", 2, (1.0, 2.0, 3.0, 10.0), "fp64", {})]
    later = None
    for name, order, s, prec, kw in runs:
        ctx = abc.Context(dims, h, order, s, precision=prec, radius=3, **kw)
        assert ctx.n_gamma == 14166
        psi = torch.from_numpy(psi0).to("cuda", ctx.complex_dtype).contiguous()
        Vt = torch.from_numpy(V).to("cuda", ctx.real_dtype).contiguous()
        aux = ctx.init_aux(psi) if order == 2 else ctx.new_aux(1) if order == 1 else None
        d1 = ctx.run(psi, aux, Vt, dt, 100, diag_every=100)
        p1 = psi.cpu().numpy()[0].astype(np.complex128)
        d = ctx.run(psi, aux, Vt, dt, 500, diag_every=100)
        if order == 2:
            later = ctx.run(psi, aux, Vt, dt, 2400, diag_every=600)[:, 0, 0]
        torch.cuda.synchronize()
        norms = np.concatenate([d1[:, 0, 0], d[:, 0, 0]])
        ex1 = scale * free_packet([X, Y, Z], 0.1, (0, 0, 0), (5.0, 0, 0), 0.5)
        res[name] = (norms, float(np.linalg.norm(p1 - ex1) / np.linalg.norm(ex1)))
        ctx.close()
    ex6 = scale * free_packet([X, Y, Z], 0.6, (0, 0, 0), (5.0, 0, 0), 0.5)
    n_exact = float(np.sum(np.abs(ex6) ** 2) * h ** 3)
    refl = {k: v[0][-1] - n_exact for k, v in res.items()}
    assert res["order1"][1] < 0.07, res["order1"][1]
    assert np.all(np.diff(res["order1"][0][:4]) < 0), res["order1"][0]
    assert 0.1 < refl["order1"] < 0.3, refl
    assert refl["order0"] > refl["order1"], refl
    assert 0 < refl["order2"] < 0.05 and refl["order2"] < refl["order1"] / 5, refl
    assert np.all(np.diff(np.concatenate([res["order2"][0], later])) < 0), later
