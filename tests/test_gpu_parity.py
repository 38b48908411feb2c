"""GPU path vs FP64 oracle, element by element (marked gpu).

Tolerances (relative L2 over each result): 1e-10 for the FP64 path and 1e-5 for the
complex64 paths after the stated number of steps (the targets the method's
reduced-precision form is measured against)."""
import numpy as np
import pytest

from oracle.coefficients import order0, order1
from oracle.lattice import Box
from oracle.propagate import System
from paper_1908_02456_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "c64": 1e-5, "tf32x3": 1e-5, "fp16x3": 1e-5}


@pytest.fixture(scope="module")
def torch_cuda():
    import torch

    from paper_1908_02456_gb300 import build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b)))


def oracle_system(dims, h, order, s, V, meanfield=None):
    box = Box(dims, h)
    co = None if order is None else (order0(box, s) if order == 0 else order1(box, s))
    return System(box, V_ext=V.reshape(-1), coeffs=co, meanfield=meanfield)


def gpu_run(torch, dims, h, order, s, prec, psi0, V, dt, steps, aux0=None, meanfield=None, diag_every=0):
    from paper_1908_02456_gb300 import abc
    b = psi0.shape[0]
    ctx = abc.Context(dims, h, order, s, precision=prec, max_orbitals=b)
    psi = torch.from_numpy(psi0.reshape(b, dims[2], dims[1], dims[0])).to("cuda", ctx.complex_dtype).contiguous()
    aux = None
    if order == 1:
        aux = ctx.new_aux(b) if aux0 is None else torch.from_numpy(aux0.T.copy()).to("cuda", ctx.complex_dtype)
    Vt = torch.from_numpy(V.reshape(dims[2], dims[1], dims[0])).to("cuda", ctx.real_dtype).contiguous()
    diag = ctx.run(psi, aux, Vt, dt, steps, meanfield=meanfield, diag_every=diag_every)
    torch.cuda.synchronize()
    out = (psi.cpu().numpy().reshape(b, -1).astype(np.complex128),
           None if aux is None else aux.cpu().numpy().T.astype(np.complex128), diag)
    ctx.close()
    return out


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("b", [1, 3])
def test_one_step_random_state(torch_cuda, order, b):
    """One step from an unstructured state (and a random aux for order 1)."""
    dims, h, dt = (6, 7, 5), 0.5, 0.01
    rng = np.random.default_rng(10 + order + b)
    psi0 = inputs.random_state(dims, b, rng).reshape(b, -1)
    V = rng.uniform(-1, 1, size=dims[::-1])
    sy = oracle_system(dims, h, order, 1.0, V)
    f0 = (rng.normal(size=(b, len(sy.G))) + 1j * rng.normal(size=(b, len(sy.G)))) if order == 1 else None
    ref_p, ref_f = sy.step(psi0, f0, dt)
    p, f, _ = gpu_run(torch_cuda, dims, h, order, 1.0, "fp64", psi0, V, dt, 1, aux0=f0)
    assert rel(p, ref_p) < 1e-13
    if order == 1:
        assert rel(f, ref_f) < 1e-13


def test_free_packet_16cube_order0_fp64(torch_cuda):
    """The 16^3, h = 0.5, order-0 (s0 = 1) free packet, 300 steps in FP64, with the
    norm / W / energy series every 10 steps."""
    w = inputs.WORKLOADS[1]
    psi0, V = inputs.make_inputs(w)
    dims = w.shape
    sy = oracle_system(dims, w.h, 0, w.s, V)
    ref_p, _, ref_d = sy.run(psi0.reshape(1, -1), w.dt, w.steps, diag_every=10)
    p, _, d = gpu_run(torch_cuda, dims, w.h, 0, w.s, "fp64", psi0.reshape(1, -1), V, w.dt, w.steps, diag_every=10)
    assert rel(p, ref_p) < TOL["fp64"]
    assert rel(d, ref_d) < TOL["fp64"]
    assert d[-1, 0, 0] < 0.95 * d[0, 0, 0]      # the packet is being absorbed


@pytest.mark.parametrize("prec", ["fp64", "c64"])
def test_harmonic_order1_reduced(torch_cuda, prec):
    """The single-orbital harmonic-well workload (first-order ABC, s1 = 1, h = 0.4,
    dt = 0.005) on a 20^3 box for 200 steps."""
    w = inputs.WORKLOADS[2]
    n, steps = 20, 200
    psi0, V = inputs.make_inputs(w, n=n)
    dims = (n, n, n)
    sy = oracle_system(dims, w.h, 1, w.s, V)
    ref_p, ref_f, ref_d = sy.run(psi0.reshape(1, -1), w.dt, steps, diag_every=20)
    p, f, d = gpu_run(torch_cuda, dims, w.h, 1, w.s, prec, psi0.reshape(1, -1), V, w.dt, steps, diag_every=20)
    assert rel(p, ref_p) < TOL[prec]
    assert rel(f, ref_f) < TOL[prec]
    assert rel(d, ref_d) < TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "c64", "tf32x3", "fp16x3"])
def test_meanfield_batched_reduced(torch_cuda, prec):
    """Batched orbitals with the density-dependent potential V = a rho + b rho^(1+alpha)
    (a = -1, b = 0.8, alpha = 1/6), first-order ABC; 5 orbitals (a ragged tail of the
    32-wide orbital tiles) on a 12^3 box, 100 steps; a second, strong-coupling case
    makes the density term dominate."""
    w = inputs.WORKLOADS[3]
    n, b, steps = 12, 5, 100
    psi0, V = inputs.make_inputs(w, n=n, n_orb=b)
    dims = (n, n, n)
    for mf in (w.meanfield, (-40.0, 30.0, 1.0 / 6.0)):
        sy = oracle_system(dims, w.h, 1, w.s, V, meanfield=mf)
        ref_p, ref_f, ref_d = sy.run(psi0.reshape(b, -1), w.dt, steps, diag_every=25)
        p, f, d = gpu_run(torch_cuda, dims, w.h, 1, w.s, prec, psi0.reshape(b, -1), V, w.dt, steps,
                          meanfield=mf, diag_every=25)
        assert rel(p, ref_p) < TOL[prec]
        assert rel(f, ref_f) < TOL[prec]
        assert rel(d, ref_d) < TOL[prec]
        # the orbitals' energies sum to the mean-field functional E[phi] (Sec. 4.3)
        E_ref = sy.energy_functional(ref_p)
        assert abs(d[-1, :, 2].sum() - E_ref) < TOL[prec] * abs(E_ref)


def test_odd_nonuniform_box_fp64(torch_cuda):
    """Odd and unequal axes exercise reflection-fixed nodes (middle planes)."""
    dims, h, dt, steps = (9, 10, 11), 0.5, 0.01, 60
    psi0 = inputs.gaussian_packet(dims, h, (0.5, -0.3, 0.2), (2.0, 1.0, -1.5), 1.0).reshape(1, -1)
    V = inputs.smooth_random(dims, h, np.random.default_rng(3))
    for order in (0, 1):
        sy = oracle_system(dims, h, order, 0.7, V)
        ref_p, ref_f, _ = sy.run(psi0, dt, steps)
        p, f, _ = gpu_run(torch_cuda, dims, h, order, 0.7, "fp64", psi0, V, dt, steps)
        assert rel(p, ref_p) < TOL["fp64"]
        if order == 1:
            assert rel(f, ref_f) < TOL["fp64"]


def test_graph_run_equals_single_steps(torch_cuda):
    """abc_run (CUDA graph replay) and repeated abc_step give identical bits."""
    torch = torch_cuda
    from paper_1908_02456_gb300 import abc
    dims, h, dt = (10, 10, 10), 0.5, 0.01
    psi0 = inputs.gaussian_packet(dims, h, (0, 0, 0), (2.0, 0, 0), 1.0)[None]
    ctx = abc.Context(dims, h, 1, 1.0, precision="c64")
    V = torch.zeros(dims, dtype=torch.float32, device="cuda")
    p1 = torch.from_numpy(psi0).to("cuda", torch.complex64)
    p2 = p1.clone()
    a1, a2 = ctx.new_aux(1), ctx.new_aux(1)
    ctx.run(p1, a1, V, dt, 20)
    for _ in range(20):
        ctx.step(p2, a2, V, dt)
    torch.cuda.synchronize()
    assert torch.equal(p1, p2) and torch.equal(a1, a2)
    # host-buffer entry point
    ph = psi0.astype(np.complex64).copy()
    ah = np.zeros((ctx.n_gamma, 1), np.complex64)
    ctx.run_host(ph, ah, np.zeros(dims, np.float32), dt, 20)
    assert np.array_equal(ph, p1.cpu().numpy()) and np.array_equal(ah, a1.cpu().numpy())
    ctx.close()


def test_full_size_lyapunov_c64(torch_cuda):
    """At the full 64^3 harmonic-well size: W = |phi|^2 + f^* Q f does not grow (Thm 3.2),
    checked every 10 steps over 400 steps of the complex64 path."""
    w = inputs.WORKLOADS[2]
    psi0, V = inputs.make_inputs(w)
    p, f, d = gpu_run(torch_cuda, w.shape, w.h, 1, w.s, "c64", psi0.reshape(1, -1), V, w.dt, 400, diag_every=10)
    W = d[:, 0, 1]
    assert np.all(np.diff(W) <= 1e-6 * W[:-1])
    assert abs(d[0, 0, 0] - 1.0) < 1e-3


@pytest.mark.parametrize("prec", ["tf32x3", "fp16x3"])
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("dims,b", [((22, 22, 22), 48), ((13, 11, 12), 7)])
def test_tensor_core_contraction_many_tiles(torch_cuda, prec, order, dims, b):
    """The tensor-core many-orbital contraction (3xTF32 and split FP16) against the
    FP64 oracle, one step from an unstructured state: on the 22^3 cube the classes
    span several 128-row tiles and K blocks, and 3 x 48 columns split into two N tiles
    (80 + 64); the non-cube has eight R = 1 classes and a 16-column tile holding 7
    orbitals."""
    h, dt = 0.45, 0.005
    rng = np.random.default_rng(77 + order + b)
    psi0 = inputs.random_state(dims, b, rng).reshape(b, -1)
    V = rng.uniform(-0.5, 0.5, size=dims[::-1])
    sy = oracle_system(dims, h, order, 1.0, V)
    f0 = (rng.normal(size=(b, len(sy.G))) + 1j * rng.normal(size=(b, len(sy.G)))) if order == 1 else None
    ref_p, ref_f = sy.step(psi0, f0, dt)
    p, f, _ = gpu_run(torch_cuda, dims, h, order, 1.0, prec, psi0, V, dt, 1, aux0=f0)
    assert rel(p, ref_p) < 1e-6
    if order == 1:
        assert rel(f, ref_f) < 1e-6


@pytest.mark.parametrize("scale", [1e-20, 1e-6, 1e12])
def test_split_fp16_column_scales(torch_cuda, scale):
    """The split-FP16 contraction scales every right-hand-side column by a power of two
    found per contraction, so its relative accuracy does not depend on the state's
    magnitude: the linear step of a state (and aux) multiplied by `scale` equals
    `scale` times the oracle's step, far outside FP16's own range."""
    dims, h, dt, b = (14, 14, 14), 0.45, 0.005, 12
    rng = np.random.default_rng(91)
    psi0 = inputs.random_state(dims, b, rng).reshape(b, -1)
    V = rng.uniform(-0.5, 0.5, size=dims[::-1])
    sy = oracle_system(dims, h, 1, 1.0, V)
    f0 = rng.normal(size=(b, len(sy.G))) + 1j * rng.normal(size=(b, len(sy.G)))
    # one orbital's columns far smaller than the rest (a per-column scale, not a global one)
    psi0[3] *= 1e-9
    f0[3] *= 1e-9
    ref_p, ref_f = sy.step(psi0, f0, dt)
    p, f, _ = gpu_run(torch_cuda, dims, h, 1, 1.0, "fp16x3", psi0 * scale, V, dt, 1, aux0=f0 * scale)
    assert rel(p / scale, ref_p) < 1e-6
    assert rel(f / scale, ref_f) < 1e-6
    assert rel(f[3] / scale, ref_f[3]) < 1e-6


@pytest.mark.parametrize("prec", ["tf32x3", "fp16x3"])
def test_tensor_core_several_items_per_cta(torch_cuda, prec):
    """At 48^3 x 32 orbitals the persistent tensor-core contraction has about two
    (tile, split) items per SM, so many CTAs work through three, reusing each TMEM
    accumulator buffer after its epilogue drained it.  Three steps of the 3xTF32 path
    against the FP64 path on the same inputs (the FP64 path is the one the small-box
    tests hold to the oracle at 1e-10)."""
    dims, h, dt, b = (48, 48, 48), 0.4, 0.005, 32
    rng = np.random.default_rng(404)
    psi0 = inputs.random_state(dims, b, rng).reshape(b, -1)
    V = inputs.smooth_random(dims, h, rng)
    p64, f64, _ = gpu_run(torch_cuda, dims, h, 1, 1.0, "fp64", psi0, V, dt, 3)
    ptc, ftc, _ = gpu_run(torch_cuda, dims, h, 1, 1.0, prec, psi0, V, dt, 3)
    assert rel(ptc, p64) < 1e-6
    assert rel(ftc, f64) < 1e-5


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("c64", 1e-5), ("tf32x3", 1e-6), ("fp16x3", 1e-6)])
@pytest.mark.parametrize("order,dims,b", [(1, (13, 11, 12), 8), (0, (10, 9, 11), 4)])
def test_multi_orbital_forward_transform(torch_cuda, prec, tol, order, dims, b):
    """With the orbital count a multiple of four the forward transform handles four
    orbitals per cell group; one step from an unstructured state against the FP64
    oracle in every precision."""
    h, dt = 0.45, 0.005
    rng = np.random.default_rng(300 + order + b)
    psi0 = inputs.random_state(dims, b, rng).reshape(b, -1)
    V = rng.uniform(-0.5, 0.5, size=dims[::-1])
    sy = oracle_system(dims, h, order, 1.0, V)
    f0 = (rng.normal(size=(b, len(sy.G))) + 1j * rng.normal(size=(b, len(sy.G)))) if order == 1 else None
    ref_p, ref_f = sy.step(psi0, f0, dt)
    p, f, _ = gpu_run(torch_cuda, dims, h, order, 1.0, prec, psi0, V, dt, 1, aux0=f0)
    assert rel(p, ref_p) < tol
    if order == 1:
        assert rel(f, ref_f) < tol


@pytest.mark.parametrize("prec", ["c64", "tf32x3", "fp16x3"])
def test_one_orbital_complex64_uses_packed_tiles(torch_cuda, prec):
    """One complex64 orbital runs the packed symmetric-tile contraction, not the
    full-block fallback: the context holds tiles and the algorithmic bytes of a launch
    are the tiles' (64 x 64 complex64 each) plus the two boundary vectors."""
    from paper_1908_02456_gb300 import abc
    ctx = abc.Context((16, 16, 16), 0.5, 1, 1.0, precision=prec, max_orbitals=2)
    tiles = ctx.get_tuning(abc.TUNE_TILE_COUNT)
    assert tiles > 0
    assert ctx.kernel_bytes(abc.KERNEL_CONTRACTION, 1) == tiles * 64 * 64 * 8 + 2 * ctx.n_gamma * 8
    ctx.close()


@pytest.mark.parametrize("prec,b", [("c64", 1), ("fp64", 1), ("c64", 3), ("tf32x3", 3), ("fp16x3", 4)])
def test_chained_forward_matches_separate_forward(torch_cuda, prec, b):
    """ABC_TUNE_CHAIN (the back transform forms the next stage's adapted inputs) gives the
    same steps as separate forward transforms, to rounding."""
    torch = torch_cuda
    from paper_1908_02456_gb300 import abc
    dims, h, dt = (10, 9, 11), 0.5, 0.01
    rng = np.random.default_rng(70 + b)
    V = inputs.smooth_random(dims, h, rng)
    psi0 = np.concatenate([inputs.gaussian_packet(dims, h, (0.2 * j, 0.0, -0.2), (2.0, 1.0 - j, 0.5), 1.0)[None]
                           for j in range(b)])
    outs = []
    for chain in (0, 1):
        ctx = abc.Context(dims, h, 1, 1.0, precision=prec, max_orbitals=b)
        ctx.set_tuning(abc.TUNE_CHAIN, chain)
        psi = torch.from_numpy(psi0).to("cuda", ctx.complex_dtype).contiguous()
        Vt = torch.from_numpy(V).to("cuda", ctx.real_dtype).contiguous()
        aux = ctx.new_aux(b)
        ctx.run(psi, aux, Vt, dt, 30)
        torch.cuda.synchronize()
        outs.append((psi.cpu().numpy().astype(np.complex128), aux.cpu().numpy().astype(np.complex128)))
        ctx.close()
    tol = 1e-13 if prec == "fp64" else 1e-6
    for a, c in zip(outs[0], outs[1]):
        assert np.linalg.norm(a - c) <= tol * np.linalg.norm(a)


def test_bounded_wait_reports_timeout_and_context_survives(torch_cuda):
    """Failure detection without a fault: a device wait on a barrier that nothing
    completes gives up after a bounded number of polls, the host reads ABC_ERR_TIMEOUT
    from the context's flag, and the context keeps working afterwards."""
    torch = torch_cuda
    from paper_1908_02456_gb300 import abc
    dims, h = (8, 8, 8), 0.5
    ctx = abc.Context(dims, h, 1, 1.0, precision="c64")
    assert abc.abc_wait_selftest(ctx.ctx, 1000) == 5
    assert b"bounded device wait" in abc.load().abc_last_error()
    psi = torch.from_numpy(inputs.gaussian_packet(dims, h, (0, 0, 0), (2.0, 0, 0), 1.0)[None]).to(
        "cuda", torch.complex64).contiguous()
    aux = ctx.new_aux(1)
    V = torch.zeros(dims, dtype=torch.float32, device="cuda")
    ctx.run(psi, aux, V, 0.01, 10)                      # raises on a nonzero status
    torch.cuda.synchronize()
    assert torch.isfinite(torch.view_as_real(psi)).all()
    assert abc.abc_wait_selftest(ctx.ctx, 1000) == 5    # and the check works again
    ctx.close()
