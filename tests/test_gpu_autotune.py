"""The schedule autotuner of the FP32 passes (scfft_autotune): it must choose among launch
schedules that give the same bits, cache its choice per grid, and leave the results alone."""

import itertools

import numpy as np
import pytest

import oracle as O
import scfft_inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1803_01346_gb300 as S  # noqa: E402
from paper_1803_01346_gb300 import build as B  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def _ctx(n, L, mask, prec=S.PREC_F32):
    ctx = S.Context(n, L, n_power=30.0, rho_out=100.0, precision=prec, delta_it=2e-5, max_iter=50)
    ctx.set_geometry(mask)
    ctx.set_field_path([0.0, 1.0], [[0, 0, 0], [0.3, -0.2, 0.9]])
    ctx.precompute_kernel()
    return ctx


def _rhs(ctx, h, g0):
    out = torch.empty_like(h)
    it = ctx.rhs(0.2, h, g0.clone(), out)
    torch.cuda.synchronize()
    return it, out.cpu().numpy()


@pytest.mark.parametrize("n,L", [((32, 32, 32), (1.0, 1.0, 1.0)), ((48, 32, 16), (1.2, 0.9, 0.8))])
def test_every_schedule_gives_the_same_bits(n, L):
    """All 64 schedules: the same Eq. 5 iteration count and the same dh/dt bit for bit (the
    loop graph is rebuilt after each change), and the oracle's answer.  On the first grid
    (nx = ny) the fused box passes run; on the second they do not apply and the three
    passes run whatever the knob says."""
    mask = I.lens(n, L, 0.6 * min(L), 0.5 * min(L), 0.1, 0.1)
    ctx = _ctx(n, L, mask)
    g = O.Grid(n, L)
    prob = O.Problem(g, mask, O.Material(n=30.0, rho_out=100.0), O.FieldPath([0.0, 1.0], [[0, 0, 0], [0.3, -0.2, 0.9]]))
    jr = O.curl_s(I.random_field((3,) + g.shape, 91, 0.3), g) * mask[None]
    hs = O.phi_hockney(jr, g) + np.array([0.05, -0.02, 0.1])[:, None, None, None]
    g0s = np.broadcast_to(prob.path.hedot(0.2)[:, None, None, None], hs.shape).copy()
    h = torch.from_numpy(hs.reshape(-1).copy()).cuda()
    g0 = torch.from_numpy(g0s.reshape(-1).copy()).cuda()
    ref_it, ref = _rhs(ctx, h, g0)
    for zk, zc, yu, yp, bf, xs in itertools.product((8, 4), (8, 16), (8, 16), (1, 0), (0, 1), (0, 1)):
        ctx.set_schedule(z_kernel_tile=zk, z_curl_tile=zc, y_unpadded_tile=yu, y_padded_tma=yp, box_fused=bf,
                         x_update_split=xs)
        assert ctx.get_schedule() == dict(z_kernel_tile=zk, z_curl_tile=zc, y_unpadded_tile=yu, y_padded_tma=yp,
                                          z_kernel_tmem=0, box_fused=bf, x_update_split=xs)
        it, out = _rhs(ctx, h, g0)
        assert it == ref_it and np.array_equal(out, ref), (zk, zc, yu, yp, bf, xs)
    o = O.rhs(prob, 0.2, hs, g0s, delta_it=2e-5, max_iter=50)
    assert abs(o.iters - ref_it) <= 1
    e = [float(np.abs(ref.reshape(hs.shape)[q] - o.hdot[q]).max() / np.abs(o.hdot[q]).max()) for q in range(3)]
    assert max(e) < 6e-6, e


def test_autotune_times_once_per_grid_and_keeps_the_results():
    n, L = (64, 64, 64), (1.0, 1.0, 1.0)
    mask = I.lens(n, L, 0.6, 0.5, 0.1, 0.1)
    a = _ctx(n, L, mask)
    b = _ctx(n, L, mask)
    h = torch.from_numpy(I.random_field((3 * 64 ** 3,), 92, 0.01)).cuda()
    g0 = torch.zeros_like(h)
    g0.view(3, -1)[2] = 0.9
    it0, out0 = _rhs(a, h, g0)
    sa = a.autotune(retune=True)
    assert sa["z_kernel_tile"] in (4, 8) and sa["z_curl_tile"] in (8, 16)
    assert sa["y_unpadded_tile"] in (8, 16) and sa["y_padded_tma"] in (0, 1)
    assert all(u > 0 for u in sa["us"][:8]), sa  # every candidate was timed
    assert sa["z_kernel_tmem"] == 0 and sa["us"][8:11] == [0.0] * 3  # no tensor-memory form at nz = 64
    assert sa["box_fused"] in (0, 1) and sa["us"][11] > 0 and sa["us"][12] > 0, sa  # three passes, fused
    assert sa["x_update_split"] in (0, 1) and sa["us"][13] > 0 and sa["us"][14] > 0, sa
    print(f"[autotune 64^3] {sa}")
    sb = b.autotune()  # the same grid: the cached choice, nothing timed
    assert {k: sb[k] for k in S.Context._SCHED_KEYS} == {k: sa[k] for k in S.Context._SCHED_KEYS}
    assert all(u == 0 for u in sb["us"])
    it1, out1 = _rhs(a, h, g0)
    it2, out2 = _rhs(b, h, g0)
    assert it0 == it1 == it2 and np.array_equal(out0, out1) and np.array_equal(out0, out2)


def test_autotune_is_a_no_op_without_a_schedule():
    n, L = (16, 16, 16), (1.0, 1.0, 1.0)
    mask = I.cube(n, L, 1.0)
    for prec in (S.PREC_F64, S.PREC_DF64):
        ctx = _ctx(n, L, mask, prec)
        s = ctx.autotune()
        assert all(u == 0 for u in s["us"])
        with pytest.raises(S.ScfftError):
            ctx.set_schedule(z_kernel_tile=4)
    ctx = _ctx(n, L, mask)
    with pytest.raises(S.ScfftError):
        ctx.set_schedule(z_kernel_tile=5)
    with pytest.raises(S.ScfftError):  # the tensor-memory z pass needs a 256-point z transform
        ctx.set_schedule(z_kernel_tmem=1)


def test_tensor_memory_z_pass_gives_the_same_bits():
    """nz = 128 (a 256-point padded z transform, 16 x 16 split): both column tiles with the
    spectra in shared memory, in tensor memory with three transpose buffers and in tensor
    memory with two give the same Eq. 5 iteration count and dh/dt bit for bit, and the
    oracle's answer; the autotuner times the three forms."""
    n, L = (32, 16, 128), (1.0, 0.5, 4.0)
    mask = I.lens(n, L, 0.4, 1.5, 0.08, 0.06)
    ctx = _ctx(n, L, mask)
    g = O.Grid(n, L)
    prob = O.Problem(g, mask, O.Material(n=30.0, rho_out=100.0), O.FieldPath([0.0, 1.0], [[0, 0, 0], [0.3, -0.2, 0.9]]))
    jr = O.curl_s(I.random_field((3,) + g.shape, 93, 0.3), g) * mask[None]
    hs = O.phi_hockney(jr, g) + np.array([0.05, -0.02, 0.1])[:, None, None, None]
    g0s = np.broadcast_to(prob.path.hedot(0.2)[:, None, None, None], hs.shape).copy()
    h = torch.from_numpy(hs.reshape(-1).copy()).cuda()
    g0 = torch.from_numpy(g0s.reshape(-1).copy()).cuda()
    ref_it, ref = _rhs(ctx, h, g0)
    for zk, zm in itertools.product((8, 4), (0, 1, 2)):
        ctx.set_schedule(z_kernel_tile=zk, z_kernel_tmem=zm)
        assert ctx.get_schedule()["z_kernel_tmem"] == zm
        it, out = _rhs(ctx, h, g0)
        assert it == ref_it and np.array_equal(out, ref), (zk, zm)
    o = O.rhs(prob, 0.2, hs, g0s, delta_it=2e-5, max_iter=50)
    assert abs(o.iters - ref_it) <= 1
    e = [float(np.abs(ref.reshape(hs.shape)[q] - o.hdot[q]).max() / np.abs(o.hdot[q]).max()) for q in range(3)]
    assert max(e) < 6e-6, e
    s = ctx.autotune(retune=True)
    assert s["z_kernel_tmem"] in (0, 1, 2) and all(u > 0 for u in s["us"][8:11]), s
    print(f"[autotune 32x16x128] {s}")
