"""Checkpoint / resume and the divergence monitor through the C ABI (marked gpu).

The monitor is exercised without any device fault: the instability is made on the
host, either as a NaN planted in the input state or as a time step past the
stability limit of the degree-4 Taylor step on a tiny box, so the state grows (or
stays NaN) while every kernel runs normally."""
import numpy as np
import pytest

from paper_1908_02456_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    from paper_1908_02456_gb300 import abc, build
    build.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch, abc


def _state(torch, ctx, dims, h, b, order):
    psi0 = np.concatenate([inputs.gaussian_packet(dims, h, (0.3 * j - 0.3, 0.1, 0.0), (2.0, 0.5 * j, -0.5), 1.0)[None]
                           for j in range(b)])
    psi = torch.from_numpy(psi0).to("cuda", ctx.complex_dtype).contiguous()
    aux = ctx.init_aux(psi) if order == 2 else ctx.new_aux(b) if order == 1 else None
    return psi, aux


@pytest.mark.parametrize("prec,order,b", [("fp64", 1, 1), ("c64", 0, 2), ("tf32x3", 1, 3), ("fp64", 2, 1)])
def test_checkpoint_resume_is_bit_exact(env, prec, order, b):
    """Run 20 steps, checkpoint, run 30 more; restore the checkpoint into fresh buffers
    of a new context and run the same 30 steps: identical bits, and the progress
    counters (steps, time) come back with the blob."""
    torch, abc = env
    dims, h, dt = (10, 9, 11), 0.5, 0.01
    V = torch.from_numpy(inputs.smooth_random(dims, h, np.random.default_rng(4))).to("cuda")
    s = (1.0, 2.0, 3.0, 10.0) if order == 2 else 1.0
    ctx = abc.Context(dims, h, order, s, precision=prec, max_orbitals=b)
    Vt = V.to(ctx.real_dtype).contiguous()
    psi, aux = _state(torch, ctx, dims, h, b, order)
    ctx.run(psi, aux, Vt, dt, 20)
    blob = ctx.get_state(psi, aux)
    assert blob.nbytes == abc.abc_state_size(ctx.ctx, b)
    assert ctx.progress()[0] == 20
    ctx.run(psi, aux, Vt, dt, 30)
    torch.cuda.synchronize()
    ref_p, ref_a = psi.cpu().clone(), None if aux is None else aux.cpu().clone()
    ctx.close()

    ctx2 = abc.Context(dims, h, order, s, precision=prec, max_orbitals=b)
    psi2 = torch.zeros_like(psi)
    aux2 = None if aux is None else torch.zeros_like(aux)
    ctx2.set_state(psi2, aux2, blob)
    steps, t = ctx2.progress()
    assert steps == 20 and abs(t - 20 * dt) < 1e-15
    ctx2.run(psi2, aux2, Vt, dt, 30)
    torch.cuda.synchronize()
    assert torch.equal(psi2.cpu(), ref_p)
    if aux is not None:
        assert torch.equal(aux2.cpu(), ref_a)
    assert ctx2.progress()[0] == 50
    ctx2.close()


def test_state_blob_is_validated(env):
    """A blob from another grid, another orbital count or with a flipped payload byte is
    refused (ABC_ERR_ARG) and nothing is copied."""
    torch, abc = env
    dims, h = (8, 8, 8), 0.5
    ctx = abc.Context(dims, h, 1, 1.0, precision="c64", max_orbitals=2)
    psi, aux = _state(torch, ctx, dims, h, 2, 1)
    blob = ctx.get_state(psi, aux)
    other = abc.Context((8, 8, 9), h, 1, 1.0, precision="c64", max_orbitals=2)
    p_o, a_o = _state(torch, other, (8, 8, 9), h, 2, 1)
    with pytest.raises(abc.AbcError) as e:
        other.set_state(p_o, a_o, blob)
    assert e.value.status == 1
    with pytest.raises(abc.AbcError):
        ctx.set_state(psi[:1].contiguous(), aux[:, :1].contiguous(), blob)   # one orbital, blob has two
    bad = blob.copy()
    bad[-5] ^= 0x10
    keep = psi.clone()
    with pytest.raises(abc.AbcError) as e:
        ctx.set_state(psi, aux, bad)
    assert b"checksum" in abc.load().abc_last_error()
    assert torch.equal(psi, keep)
    ctx.set_state(psi, aux, blob)                     # the intact blob is accepted
    other.close()
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "c64", "tf32x3"])
def test_monitor_quiet_on_a_stable_run(env, prec):
    """A stable order-1 run with diagnostics every 5 steps returns ABC_OK and its W
    series does not grow (the monitor's own criterion, checked again on the host)."""
    torch, abc = env
    dims, h, dt, b = (12, 12, 12), 0.4, 0.005, 3
    ctx = abc.Context(dims, h, 1, 1.0, precision=prec, max_orbitals=b)
    psi, aux = _state(torch, ctx, dims, h, b, 1)
    V = torch.zeros(dims, dtype=ctx.real_dtype, device="cuda")
    d = ctx.run(psi, aux, V, dt, 100, meanfield=(-1.0, 0.8, 1.0 / 6.0), diag_every=5)
    W = d[:, :, 1]
    assert np.all(W[1:] <= W[:-1] * (1 + 5e-6))
    ctx.close()


@pytest.mark.parametrize("prec", ["fp64", "c64"])
def test_monitor_reports_nan_state(env, prec):
    torch, abc = env
    dims, h, dt = (8, 8, 8), 0.5, 0.01
    ctx = abc.Context(dims, h, 1, 1.0, precision=prec)
    psi, aux = _state(torch, ctx, dims, h, 1, 1)
    psi[0, 3, 4, 5] = complex("nan")
    V = torch.zeros(dims, dtype=ctx.real_dtype, device="cuda")
    with pytest.raises(abc.AbcError) as e:
        ctx.run(psi, aux, V, dt, 10, diag_every=2)
    assert e.value.status == 6
    assert b"divergence monitor" in abc.load().abc_last_error()
    # the context stays usable: a clean state runs without complaint
    psi, aux = _state(torch, ctx, dims, h, 1, 1)
    ctx.run(psi, aux, V, dt, 10, diag_every=2)
    ctx.close()


@pytest.mark.parametrize("order", [0, 1])
def test_monitor_reports_unstable_time_step(env, order):
    """dt far past the Taylor-4 stability limit (dt * rho(H) = 4.8 > 2 sqrt 2 on an 8^3
    box at h = 0.5): the state grows every step and the monitor names the first
    diagnostic step."""
    torch, abc = env
    dims, h, dt = (8, 8, 8), 0.5, 0.2
    ctx = abc.Context(dims, h, order, 1.0, precision="fp64")
    rng = np.random.default_rng(3)
    psi = torch.from_numpy(inputs.random_state(dims, 1, rng)).to("cuda").contiguous()
    aux = ctx.new_aux(1) if order == 1 else None
    V = torch.zeros(dims, dtype=torch.float64, device="cuda")
    with pytest.raises(abc.AbcError) as e:
        ctx.run(psi, aux, V, dt, 12, diag_every=3)
    assert e.value.status == 6
    assert b"at step 3 " in abc.load().abc_last_error()
    ctx.close()
