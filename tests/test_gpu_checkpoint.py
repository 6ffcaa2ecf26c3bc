"""Checkpoint and resume through the C ABI: a trajectory saved after a few steps and resumed
(in a fresh context, into fresh buffers) continues bit for bit like the uninterrupted run,
on both paths; snapshots of another grid or precision are refused.  The host-buffer step
(scfft_step_host) follows the device API's trajectory bit for bit."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_1803_01346_gb300 as S  # noqa: E402
import scfft_inputs as I  # noqa: E402

N_GRID, L_BOX = (16, 16, 16), (1.0, 1.0, 1.0)
PATH = ([0.0, 1.0, 2.0], [[0, 0, 0], [0, 0, 0.5], [0, 0, 0]])


def _ctx(prec, n=N_GRID):
    ctx = S.Context(n, L_BOX, n_power=20.0, rho_out=20.0, precision=prec, delta_it=2e-5, max_iter=50,
                    rtol=1e-5, atol=1e-7)
    ctx.set_geometry(I.cube(n, L_BOX, 1.0))
    ctx.set_field_path(*PATH)
    ctx.precompute_kernel()
    return ctx


def _steps(ctx, t, dt, h, warm, k):
    for _ in range(k):
        t, dt, _ = ctx.step(t, dt, 2.0, h, warm)
    return t, dt


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [S.PREC_F64, S.PREC_F32])
def test_resume_continues_bit_for_bit(prec):
    n3 = 3 * int(np.prod(N_GRID))
    a = _ctx(prec)
    h = torch.zeros(n3, dtype=torch.float64, device="cuda")
    warm = torch.zeros_like(h)
    warm.view(3, -1)[2] = 0.5  # dh_e/dt on the first segment of the path
    t, dt = _steps(a, 0.0, 1e-3, h, warm, 4)
    snap = a.checkpoint_save(t, dt, h, warm)
    t_ref, dt_ref = _steps(a, t, dt, h, warm, 3)
    h_ref, w_ref = h.cpu().numpy(), warm.cpu().numpy()

    b = _ctx(prec)
    h2 = torch.full_like(h, float("nan"))
    w2 = torch.full_like(h, float("nan"))
    t2, dt2 = b.checkpoint_load(snap, h2, w2)
    assert (t2, dt2) == (t, dt)
    t2, dt2 = _steps(b, t2, dt2, h2, w2, 3)
    assert (t2, dt2) == (t_ref, dt_ref)
    assert np.array_equal(h2.cpu().numpy(), h_ref)
    assert np.array_equal(w2.cpu().numpy(), w_ref)


@pytest.mark.gpu
def test_snapshots_of_another_grid_or_precision_are_refused():
    n3 = 3 * int(np.prod(N_GRID))
    a = _ctx(S.PREC_F64)
    h = torch.zeros(n3, dtype=torch.float64, device="cuda")
    warm = torch.zeros_like(h)
    snap = a.checkpoint_save(0.0, 1e-3, h, warm)
    for other in (_ctx(S.PREC_F32), _ctx(S.PREC_F64, (32, 16, 16))):
        hh = torch.zeros(3 * 32 * 16 * 16, dtype=torch.float64, device="cuda")
        with pytest.raises(S.ScfftError) as e:
            other.checkpoint_load(snap, hh, torch.zeros_like(hh))
        assert e.value.code == 1


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [S.PREC_F64, S.PREC_F32])
def test_step_host_matches_step_bit_for_bit(prec):
    """scfft_step_host (state and warm start in page-locked host memory) follows the device
    API's trajectory bit for bit and copies what it states: h in and h, warm out on every
    step; warm in on the first step of a trajectory, and on every step of the FP64 path
    (whose stages read it)."""
    n3 = 3 * int(np.prod(N_GRID))
    k = 4
    a = _ctx(prec)
    h = torch.zeros(n3, dtype=torch.float64, device="cuda")
    warm = torch.zeros_like(h)
    warm.view(3, -1)[2] = 0.5
    h_host = h.cpu().pin_memory()
    w_host = warm.cpu().pin_memory()
    t_ref, dt_ref = _steps(a, 0.0, 1e-3, h, warm, k)

    b = _ctx(prec)
    hd = torch.full_like(h, float("nan"))
    wd = torch.full_like(h, float("nan"))
    t, dt = 0.0, 1e-3
    for _ in range(k):
        t, dt, _ = b.step_host(t, dt, 2.0, h_host, w_host, hd, wd)
    assert (t, dt) == (t_ref, dt_ref)
    assert np.array_equal(h_host.numpy(), h.cpu().numpy())
    assert np.array_equal(w_host.numpy(), warm.cpu().numpy())
    st, nb = b.stats(), n3 * 8
    assert st["d2h_bytes"] == 2 * k * nb
    assert st["h2d_bytes"] == (2 * k * nb if prec == S.PREC_F64 else (k + 1) * nb)
    with pytest.raises(ValueError):
        b.step_host(t, dt, 2.0, hd, w_host, hd, wd)  # device tensor where a host one belongs
    # without warm_host the warm start stays in the device buffer: the same trajectory bit for
    # bit, with only h copied in and out on every step
    c = _ctx(prec)
    h_host2 = torch.zeros(n3, dtype=torch.float64).pin_memory()
    hd2 = torch.full_like(h, float("nan"))
    wd2 = torch.zeros_like(h)
    wd2.view(3, -1)[2] = 0.5
    t, dt = 0.0, 1e-3
    for _ in range(k):
        t, dt, _ = c.step_host(t, dt, 2.0, h_host2, None, hd2, wd2)
    assert (t, dt) == (t_ref, dt_ref)
    assert np.array_equal(h_host2.numpy(), h.cpu().numpy())
    assert np.array_equal(wd2.cpu().numpy(), warm.cpu().numpy())
    st = c.stats()
    assert st["h2d_bytes"] == k * nb and st["d2h_bytes"] == k * nb
