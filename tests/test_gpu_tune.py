"""The autotuner and every setting it chooses among (marked gpu).

Each GEMM tile configuration and split count, and each stencil form, computes the
same step up to FP32 rounding: checked against the FP64 oracle on a box whose
classes span several 128-row tiles and K blocks, and the tuned setting against the
default one over a mean-field run."""
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


@pytest.mark.parametrize("prec", ["tf32x3", "fp16x3"])
@pytest.mark.parametrize("tile,split", [(0, 0), (0, 1), (0, 4), (1, 0), (1, 2), (1, 8), (2, 0), (2, 1), (2, 3)])
def test_gemm_settings_against_oracle(env, prec, tile, split):
    torch, abc = env
    dims, h, dt, b = (22, 22, 22), 0.45, 0.005, 40
    rng = np.random.default_rng(808)
    psi0 = inputs.random_state(dims, b, rng).reshape(b, -1)
    V = rng.uniform(-0.5, 0.5, size=dims[::-1])
    box = Box(dims, h)
    sy = System(box, V_ext=V.reshape(-1), coeffs=order1(box, 1.0))
    f0 = rng.normal(size=(b, len(sy.G))) + 1j * rng.normal(size=(b, len(sy.G)))
    ref_p, ref_f = sy.step(psi0, f0, dt)
    ctx = abc.Context(dims, h, 1, 1.0, precision=prec, max_orbitals=b)
    ctx.set_tuning(abc.TUNE_GEMM_TILE, tile)
    ctx.set_tuning(abc.TUNE_GEMM_SPLIT, split)
    psi = torch.from_numpy(psi0.reshape(b, *dims[::-1])).to("cuda", torch.complex64).contiguous()
    aux = torch.from_numpy(f0.T.copy()).to("cuda", torch.complex64).contiguous()
    Vt = torch.from_numpy(V).to("cuda", torch.float32).contiguous()
    ctx.run(psi, aux, Vt, dt, 1)
    torch.cuda.synchronize()
    assert rel(psi.cpu().numpy().reshape(b, -1), ref_p) < 1e-6
    assert rel(aux.cpu().numpy().T, ref_f) < 1e-6
    ctx.close()


def test_tuned_setting_matches_default(env, tmp_path, monkeypatch):
    """tune() picks a setting (timed on a copy of the state; the caller's state is not
    touched), caches it, and the tuned run equals the default run to FP32 rounding."""
    torch, abc = env
    from paper_1908_02456_gb300 import tune
    monkeypatch.setattr(tune, "CACHE", str(tmp_path / "cache.json"))
    dims, h, dt, b = (24, 24, 24), 0.4, 0.005, 16
    mf = (-1.0, 0.8, 1.0 / 6.0)
    psi0 = inputs.orbital_set(dims, h, np.random.default_rng(9), b)
    outs = []
    for tuned in (False, True):
        ctx = abc.Context(dims, h, 1, 1.0, precision="fp16x3", max_orbitals=b)
        psi = torch.from_numpy(psi0).to("cuda", torch.complex64).contiguous()
        aux = ctx.new_aux(b)
        V = torch.zeros(dims, dtype=torch.float32, device="cuda")
        if tuned:
            keep = psi.clone()
            res = tune.tune(ctx, psi, aux, V, dt, meanfield=mf, steps=3, repeats=1)
            assert res["tuned"] and res["setting"]
            assert torch.equal(psi, keep)
            again = tune.tune(ctx, psi, aux, V, dt, meanfield=mf)
            assert again["cached"] and again["setting"] == res["setting"]
        ctx.run(psi, aux, V, dt, 21, meanfield=mf)
        torch.cuda.synchronize()
        outs.append((psi.cpu().numpy().astype(np.complex128), aux.cpu().numpy().astype(np.complex128)))
        ctx.close()
    assert rel(outs[1][0], outs[0][0]) < 2e-6
    assert rel(outs[1][1], outs[0][1]) < 2e-6


@pytest.mark.parametrize("mode,bps", [(1, 3), (0, 4), (1, 0), (2, 0)])
def test_stencil_placements_give_identical_steps(env, mode, bps):
    """Where the stencil runs (second stream after the contraction, from the stage start,
    or serially) and the grid-stride grid of a bounded number of blocks per SM change
    only the schedule: every node is computed by the same expression, so the steps
    agree bit for bit with the default."""
    torch, abc = env
    dims, h, dt, b = (20, 18, 16), 0.45, 0.005, 8
    psi0 = inputs.orbital_set(dims, h, np.random.default_rng(4), b)
    outs = []
    for setting in ((0, 0), (mode, bps)):
        ctx = abc.Context(dims, h, 1, 1.0, precision="fp16x3", max_orbitals=b)
        ctx.set_tuning(abc.TUNE_STENCIL, setting[0])
        ctx.set_tuning(abc.TUNE_STENCIL_BPS, setting[1])
        psi = torch.from_numpy(psi0).to("cuda", torch.complex64).contiguous()
        aux = ctx.new_aux(b)
        V = torch.zeros(dims[::-1], dtype=torch.float32, device="cuda")
        ctx.run(psi, aux, V, dt, 9, meanfield=(-1.0, 0.8, 1.0 / 6.0))
        torch.cuda.synchronize()
        outs.append((psi.cpu(), aux.cpu()))
        ctx.close()
    assert torch.equal(outs[0][0], outs[1][0])
    assert torch.equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("knob,value", [("STENCIL_KZ", 1), ("STENCIL_KZ", 2), ("STENCIL_KZ", 4), ("STENCIL_KZ", 8),
                                        ("STENCIL_KZ", 16),
                                        ("BACK_MULTI", 1), ("BACK_MULTI", 2), ("FORWARD_RW", 1)])
@pytest.mark.parametrize("prec", ["fp16x3", "c64"])
def test_kernel_forms_match_default(env, knob, value, prec):
    """The z-marching stencil forms (2..16 planes per thread, the box's 13 planes leave a
    ragged last group) and the four-orbital back transform evaluate the same
    expressions as the default kernels."""
    torch, abc = env
    dims, h, dt, b = (18, 14, 13), 0.45, 0.005, 8
    psi0 = inputs.orbital_set(dims, h, np.random.default_rng(6), b)
    V0 = inputs.smooth_random(dims, h, np.random.default_rng(7))
    outs = []
    for setting in (0, value):
        ctx = abc.Context(dims, h, 1, 1.0, precision=prec, max_orbitals=b)
        ctx.set_tuning(getattr(abc, "TUNE_" + knob), setting)
        psi = torch.from_numpy(psi0).to("cuda", torch.complex64).contiguous()
        aux = ctx.new_aux(b)
        V = torch.from_numpy(V0).to("cuda", torch.float32).contiguous()
        ctx.run(psi, aux, V, dt, 7, meanfield=(-1.0, 0.8, 1.0 / 6.0))
        torch.cuda.synchronize()
        outs.append((psi.cpu().numpy().astype(np.complex128), aux.cpu().numpy().astype(np.complex128)))
        ctx.close()
    assert rel(outs[1][0], outs[0][0]) < 1e-6
    assert rel(outs[1][1], outs[0][1]) < 1e-6


@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("form", [(0, 1, 0), (1, 1, 0), (0, 0, 0), (0, 4, 0), (1, 0, 2)])
@pytest.mark.parametrize("prec", ["fp16x3", "c64"])
def test_gamma_copy_is_bit_identical(env, order, form, prec):
    """The forward transform reading w on Gamma from the copy the previous stage's stencil
    wrote (two alternating copies, the first filled from psi at the start of each call)
    sees exactly the values it would gather from the state: abc_run and abc_step give
    bit-identical results with the copy on and off, for every stencil form and placement
    (form = stencil placement, planes per thread, blocks per SM of the grid-stride form;
    placement 1 runs each stage's stencil beside its forward transform)."""
    torch, abc = env
    dims, h, dt, b = (18, 14, 13), 0.45, 0.005, 8
    psi0 = inputs.orbital_set(dims, h, np.random.default_rng(16), b)
    V0 = inputs.smooth_random(dims, h, np.random.default_rng(17))
    outs = []
    for gc in (0, 1):
        ctx = abc.Context(dims, h, order, 1.0, precision=prec, max_orbitals=b)
        ctx.set_tuning(abc.TUNE_GAMMA_COPY, gc)
        ctx.set_tuning(abc.TUNE_STENCIL, form[0])
        ctx.set_tuning(abc.TUNE_STENCIL_KZ, form[1])
        ctx.set_tuning(abc.TUNE_STENCIL_BPS, form[2])
        assert ctx.get_tuning(abc.TUNE_GAMMA_COPY) == gc
        psi = torch.from_numpy(psi0).to("cuda", torch.complex64).contiguous()
        aux = ctx.new_aux(b)
        V = torch.from_numpy(V0).to("cuda", torch.float32).contiguous()
        ctx.run(psi, aux, V, dt, 7, meanfield=(-1.0, 0.8, 1.0 / 6.0))
        ctx.step(psi, aux, V, dt)
        ctx.run(psi, aux, V, dt, 3)
        torch.cuda.synchronize()
        outs.append((psi.cpu(), None if aux is None else aux.cpu()))
        ctx.close()
    assert torch.equal(outs[0][0], outs[1][0])
    if order == 1:
        assert torch.equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("dims", [(18, 14, 13), (10, 17, 50), (96, 9, 26)])
@pytest.mark.parametrize("order", [0, 1])
@pytest.mark.parametrize("placement,gc", [(0, 0), (1, 1)])
def test_staged_stencil_is_bit_identical(env, dims, order, placement, gc):
    """The stencil with its planes staged in shared memory by bulk copies evaluates the
    same expressions in the same order as the direct-load forms, so whole runs are bit
    for bit the same: ragged row tiles (14 = 8 + 6 rows, 17 = 8 + 8 + 1) and plane runs
    (13 < 24, 50 = 24 + 24 + 2, 26 = 24 + 2), a full-width row of 96, orders 0 and 1,
    the stencil beside the forward transform, the Gamma copy written by it."""
    torch, abc = env
    h, dt, b = 0.45, 0.005, 4
    psi0 = inputs.orbital_set(dims, h, np.random.default_rng(36), b)
    V0 = inputs.smooth_random(dims, h, np.random.default_rng(37))
    outs = []
    for staged in (0, 1):
        ctx = abc.Context(dims, h, order, 1.0, precision="c64", max_orbitals=b)
        ctx.set_tuning(abc.TUNE_STENCIL, placement)
        ctx.set_tuning(abc.TUNE_GAMMA_COPY, gc)
        ctx.set_tuning(abc.TUNE_STENCIL_STAGED, staged)
        assert ctx.get_tuning(abc.TUNE_STENCIL_STAGED) == staged
        psi = torch.from_numpy(psi0).to("cuda", torch.complex64).contiguous()
        aux = ctx.new_aux(b)
        V = torch.from_numpy(V0).to("cuda", torch.float32).contiguous()
        ctx.run(psi, aux, V, dt, 6, meanfield=(-1.0, 0.8, 1.0 / 6.0))
        ctx.step(psi, aux, V, dt)
        torch.cuda.synchronize()
        outs.append((psi.cpu(), aux.cpu()))
        ctx.close()
    assert torch.equal(outs[0][0], outs[1][0])
    if order == 1:
        assert torch.equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("lanes", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("prec,b,tile,split,gc", [("fp16x3", 32, 0, 0, 0), ("fp16x3", 64, 1, 2, 1),
                                                  ("fp16x3", 96, 0, 1, 0), ("tf32x3", 32, 2, 3, 0),
                                                  ("tf32x3", 64, 0, 1, 1), ("fp16x3", 40, 0, 0, 0),
                                                  ("c64", 32, 0, 0, 0)])
def test_node_major_chain_is_bit_identical(env, lanes, prec, b, tile, split, gc):
    """The order-1 chain with node-major adapted vectors (ABC_TUNE_LANES: warp per cell
    and 32 orbitals; the column scales, the operand packing and the GEMM epilogue in that
    layout) forms the same sums in the same order as the orbital-major chain: runs and
    single steps are bit for bit the same, for each GEMM form, split count and the Gamma
    copy, on a box whose classes span several 128-row tiles and K blocks, with a warp per
    cell (lanes 1) or each cell split between two lanes (lanes 2 and 3, two register caps)
    or four (lanes 4 and 5).  Orbital counts that are not a multiple of 32, and plain complex64, keep the
    orbital-major chain."""
    torch, abc = env
    dims, h, dt = (22, 20, 18), 0.45, 0.005
    psi0 = inputs.orbital_set(dims, h, np.random.default_rng(46), b)
    V0 = inputs.smooth_random(dims, h, np.random.default_rng(47))
    outs = []
    for setting in (0, lanes):
        ctx = abc.Context(dims, h, 1, 1.0, precision=prec, max_orbitals=b)
        ctx.set_tuning(abc.TUNE_LANES, setting)
        assert ctx.get_tuning(abc.TUNE_LANES) == setting
        if prec != "c64":
            ctx.set_tuning(abc.TUNE_GEMM_TILE, tile)
            ctx.set_tuning(abc.TUNE_GEMM_SPLIT, split)
        ctx.set_tuning(abc.TUNE_GAMMA_COPY, gc)
        psi = torch.from_numpy(psi0).to("cuda", torch.complex64).contiguous()
        aux = ctx.new_aux(b)
        V = torch.from_numpy(V0).to("cuda", torch.float32).contiguous()
        ctx.run(psi, aux, V, dt, 5, meanfield=(-1.0, 0.8, 1.0 / 6.0))
        ctx.step(psi, aux, V, dt)
        ctx.run(psi, aux, V, dt, 2)
        torch.cuda.synchronize()
        outs.append((psi.cpu(), aux.cpu()))
        ctx.close()
    assert torch.equal(outs[0][0], outs[1][0])
    assert torch.equal(outs[0][1], outs[1][1])


@pytest.mark.parametrize("lanes", [1, 2, 4])
@pytest.mark.parametrize("prec", ["fp16x3", "tf32x3"])
def test_node_major_chain_against_oracle(env, prec, lanes):
    """One step of the node-major chain against the FP64 oracle (64 orbitals, random
    auxiliary state): the same 1e-6 as every other tensor-core setting."""
    torch, abc = env
    dims, h, dt, b = (22, 22, 22), 0.45, 0.005, 64
    rng = np.random.default_rng(818)
    psi0 = inputs.random_state(dims, b, rng).reshape(b, -1)
    V = rng.uniform(-0.5, 0.5, size=dims[::-1])
    box = Box(dims, h)
    sy = System(box, V_ext=V.reshape(-1), coeffs=order1(box, 1.0))
    f0 = rng.normal(size=(b, len(sy.G))) + 1j * rng.normal(size=(b, len(sy.G)))
    ref_p, ref_f = sy.step(psi0, f0, dt)
    ctx = abc.Context(dims, h, 1, 1.0, precision=prec, max_orbitals=b)
    ctx.set_tuning(abc.TUNE_LANES, lanes)
    ctx.set_tuning(abc.TUNE_GEMM_SPLIT, 1)               # the epilogue forms x
    psi = torch.from_numpy(psi0.reshape(b, *dims[::-1])).to("cuda", torch.complex64).contiguous()
    aux = torch.from_numpy(f0.T.copy()).to("cuda", torch.complex64).contiguous()
    Vt = torch.from_numpy(V).to("cuda", torch.float32).contiguous()
    ctx.run(psi, aux, Vt, dt, 1)
    torch.cuda.synchronize()
    assert rel(psi.cpu().numpy().reshape(b, -1), ref_p) < 1e-6
    assert rel(aux.cpu().numpy().T, ref_f) < 1e-6
    ctx.close()
