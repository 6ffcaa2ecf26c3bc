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
