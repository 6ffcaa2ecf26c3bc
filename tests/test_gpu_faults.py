"""Device-side timeout path, exercised without a GPU fault: an injected fault makes one
bounded mbarrier wait of the TMA-fed y pass run out (its copy brings 16 bytes fewer than the
wait expects).  The pass must latch SCFFT_ETIMEOUT, which scfft_sync reports, within a few
seconds; the GPU must stay usable, and a fresh context must compute the right answer."""

import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
import paper_1803_01346_gb300 as S  # noqa: E402
import scfft_inputs as I  # noqa: E402

ETIMEOUT = 7


def _ctx(n, L):
    ctx = S.Context(n, L, n_power=20.0, rho_out=20.0, precision=S.PREC_F32, delta_it=0.0, max_iter=3)
    ctx.set_geometry(I.cube(n, L, 1.0))
    ctx.set_field_path([0.0, 1.0], [[0, 0, 0], [0, 0, 0.5]])
    ctx.precompute_kernel()
    return ctx


@pytest.mark.gpu
def test_tma_wait_timeout_is_latched_and_the_gpu_stays_usable():
    n, L = (32, 32, 32), (1.0, 1.0, 1.0)
    g = O.Grid(n, L)
    j = I.random_field((3,) + g.shape, 77, 1.0) * I.cube(n, L, 1.0)[None]
    jd = torch.from_numpy(j.ravel().copy()).cuda()
    out = torch.empty_like(jd)

    bad = _ctx(n, L)
    bad.inject_fault(S.FAULT_TMA_WAIT)
    t0 = time.perf_counter()
    bad.phi(jd, out)
    with pytest.raises(S.ScfftError) as e:
        bad.sync()
    assert e.value.code == ETIMEOUT
    assert time.perf_counter() - t0 < 30.0
    with pytest.raises(S.ScfftError) as e:  # the status stays latched in that context
        bad.sync()
    assert e.value.code == ETIMEOUT

    good = _ctx(n, L)
    good.phi(jd, out)
    good.sync()
    ref = O.phi_hockney(j, g)
    err = float(np.abs(out.cpu().numpy().reshape(ref.shape) - ref).max() / np.abs(ref).max())
    assert err < 2e-5, err


@pytest.mark.gpu
def test_inject_fault_rejects_unknown_kinds_and_fp64_contexts():
    n, L = (16, 16, 16), (1.0, 1.0, 1.0)
    with pytest.raises(S.ScfftError) as e:
        _ctx(n, L).inject_fault(5)
    assert e.value.code == 1
    ctx64 = S.Context(n, L)
    with pytest.raises(S.ScfftError) as e:
        ctx64.inject_fault(S.FAULT_TMA_WAIT)
    assert e.value.code == 1
    ctx64.inject_fault(0)  # disarming is always accepted


def _state(n, L, seed, scale=0.05):
    return torch.from_numpy(I.random_field((3,) + tuple(n[::-1]), seed, scale).ravel().copy()).cuda()


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [S.PREC_F64, S.PREC_F32])
def test_nan_in_the_state_latches_enonfinite(prec):
    n, L = (16, 16, 16), (1.0, 1.0, 1.0)
    ctx = S.Context(n, L, precision=prec, delta_it=2e-5, max_iter=20)
    ctx.set_geometry(I.cube(n, L, 1.0))
    ctx.set_field_path([0.0, 1.0], [[0, 0, 0], [0, 0, 0.5]])
    ctx.precompute_kernel()
    h = _state(n, L, 3)
    h[123] = float("nan")
    warm = torch.zeros_like(h)
    out = torch.empty_like(h)
    with pytest.raises(S.ScfftError) as e:
        ctx.rhs(0.2, h, warm, out)
    assert e.value.code == 6


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [S.PREC_F64, S.PREC_F32])
def test_iteration_cap_reports_enoconv_with_the_result_written(prec):
    import ctypes
    n, L = (16, 16, 16), (1.0, 1.0, 1.0)
    ctx = S.Context(n, L, n_power=20.0, rho_out=20.0, precision=prec, delta_it=1e-12, max_iter=1)
    ctx.set_geometry(I.cube(n, L, 1.0))
    ctx.set_field_path([0.0, 1.0], [[0, 0, 0], [0, 0, 0.5]])
    ctx.precompute_kernel()
    h = _state(n, L, 4)
    warm = torch.zeros_like(h)
    out = torch.full_like(h, float("nan"))
    it = ctypes.c_int(0)
    code = ctx._lib.scfft_rhs(ctx._h, 0.2, 0, ctypes.c_void_p(h.data_ptr()), ctypes.c_void_p(warm.data_ptr()),
                              ctypes.c_void_p(out.data_ptr()), ctypes.byref(it))
    torch.cuda.synchronize()
    assert code == 4 and it.value == 1
    assert bool(torch.isfinite(out).all())


@pytest.mark.gpu
def test_step_size_floor_reports_estep():
    n, L = (16, 16, 16), (1.0, 1.0, 1.0)
    ctx = S.Context(n, L, delta_it=2e-5, max_iter=20)
    ctx.set_geometry(I.cube(n, L, 1.0))
    ctx.set_field_path([0.0, 1.0], [[0, 0, 0], [0, 0, 0.5]])
    ctx.precompute_kernel()
    h = torch.zeros(3 * 16 ** 3, dtype=torch.float64, device="cuda")
    warm = torch.zeros_like(h)
    with pytest.raises(S.ScfftError) as e:
        ctx.step(0.0, 1e-20, 1.0, h, warm)
    assert e.value.code == 5


@pytest.mark.gpu
def test_calls_out_of_order_and_bad_sizes_are_rejected_on_the_host():
    n, L = (16, 16, 16), (1.0, 1.0, 1.0)
    ctx = S.Context(n, L)
    h = torch.zeros(3 * 16 ** 3, dtype=torch.float64, device="cuda")
    with pytest.raises(S.ScfftError) as e:  # no geometry, kernel or field path yet
        ctx.rhs(0.0, h, torch.zeros_like(h), torch.empty_like(h))
    assert e.value.code == 8
    with pytest.raises(S.ScfftError) as e:  # 20 is not a supported grid size
        S.Context((20, 16, 16), L)
    assert e.value.code == 1
    # corrupt geometry: a superconducting node within two cells of a face, or none at all
    near_face = I.cube(n, L, 1.0)
    near_face[1, 8, 8] = True
    for bad in (near_face, np.zeros_like(near_face)):
        with pytest.raises(S.ScfftError) as e:
            ctx.set_geometry(bad)
        assert e.value.code == 1
