"""Batched instances (scfft_batch_step): independent problems of different grid
sizes advanced together, each against the FP64 oracle.

A batch of shield instances on mixed grids (16^3, 32^3 and a non-cubic
48 x 32 x 16) takes adaptive BS23 steps (the method of lines of §2); the oracle
then integrates each instance alone over the step sizes the GPU chose, with
Eq. 5 iterated to its fixed point on both sides (delta_it = 1e-13), and the
states agree element by element: <= 1e-10 (FP64 path), <= 1e-4 (FP32 path,
the FP32 fixed-step bound of test_gpu_parity).  A second check: the batch gives
bit for bit the results of stepping the same instances one after another with the same
device-resident step (scfft_advance), and those of the host-driven scfft_step up to the
rounding of the step controller's pow (FP32 contexts run the batch as one CUDA graph)."""

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


GRIDS = [(16, 16, 16), (32, 32, 32), (48, 32, 16)]


def _configs():
    cfgs = I.batch_configs(len(GRIDS), seed=7)
    for c, n in zip(cfgs, GRIDS):
        c.n = n
        c.mask = I.shield(n, c.L, 1.0, 0.8, 2.0, 0.2)
    return cfgs


def _make(cfg, prec, stream, delta_it=1e-13, max_iter=80):
    ctx = S.Context(cfg.n, cfg.L, n_power=cfg.n_power, rho_out=cfg.rho_out, precision=prec, rtol=cfg.rtol,
                    atol=cfg.atol, delta_it=delta_it, max_iter=max_iter, stream=stream.cuda_stream)
    ctx.set_geometry(cfg.mask)
    ctx.set_field_path(cfg.knots_t, cfg.knots_he)
    ctx.precompute_kernel()
    N = int(np.prod(cfg.n))
    h = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    w = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    hd = np.asarray(cfg.knots_he[1]) / cfg.knots_t[1]  # dh_e/dt(0): the first warm start (reading R-warm)
    for q in range(3):
        w.view(3, N)[q] = float(hd[q])
    return ctx, h, w


@pytest.mark.parametrize("prec,tol", [(S.PREC_F64, 1e-10), (S.PREC_F32, 1e-4)])
def test_mixed_grid_batch_matches_oracle(prec, tol):
    cfgs = _configs()
    streams = [torch.cuda.Stream() for _ in cfgs]
    inst = [_make(c, prec, s) for c, s in zip(cfgs, streams)]
    nb = len(inst)
    t, dt = [0.0] * nb, [2e-3] * nb
    stop = [c.t_end for c in cfgs]
    hist = [[] for _ in range(nb)]
    for _ in range(3):
        t0 = list(t)
        t, dt, st = S.batch_step([a[0] for a in inst], t, dt, stop, [a[1] for a in inst], [a[2] for a in inst])
        assert all(v == 0 for v in st)
        for i in range(nb):
            hist[i].append(t[i] - t0[i])
    torch.cuda.synchronize()
    for (ctx, h, _), c, dts in zip(inst, cfgs, hist):
        prob = O.Problem(O.Grid(c.n, c.L), c.mask, O.Material(n=c.n_power, rho_out=c.rho_out),
                         O.FieldPath(c.knots_t, c.knots_he))
        ref = O.integrate(prob, 0.0, float(np.sum(dts)), np.zeros((3,) + prob.grid.shape), rtol=c.rtol,
                          atol=c.atol, dt0=dts[0], delta_it=1e-13, max_iter=80, dt_list=dts)
        assert ref.accepted == len(dts)
        got = h.cpu().numpy().reshape(ref.y.shape)
        err = float(np.abs(got - ref.y).max() / np.abs(ref.y).max())
        assert err < tol, (c.n, err)


@pytest.mark.parametrize("prec", [S.PREC_F64, S.PREC_F32])
def test_batch_step_equals_individual_steps(prec):
    cfgs = _configs()
    streams = [torch.cuda.Stream() for _ in cfgs]
    A = [_make(c, prec, s, delta_it=2e-5, max_iter=100) for c, s in zip(cfgs, streams)]
    Bv = [_make(c, prec, s, delta_it=2e-5, max_iter=100) for c, s in zip(cfgs, streams)]
    nb = len(cfgs)
    t = [0.0] * nb
    dt = [1e-4] * nb
    stop = [c.t_end for c in cfgs]
    for _ in range(3):
        t, dt, st = S.batch_step([a[0] for a in A], t, dt, stop, [a[1] for a in A], [a[2] for a in A])
        assert all(v == 0 for v in st)
    torch.cuda.synchronize()
    C = [_make(c, prec, s, delta_it=2e-5, max_iter=100) for c, s in zip(cfgs, streams)]
    for (ctx, h, w), (ctx2, h2, w2), c, tb in zip(Bv, C, cfgs, t):
        tt, d = 0.0, 1e-4
        for _ in range(3):  # the same device-resident step, one instance at a time
            tt, d, _ = ctx.advance(tt, d, c.t_end, 1, h, w)
        assert tt == tb
        tt, d = 0.0, 1e-4
        for _ in range(3):  # the host-driven step: the same up to the rounding of pow in the controller
            tt, d, _ = ctx2.step(tt, d, c.t_end, h2, w2)
        assert tt == pytest.approx(tb, rel=1e-12)
    torch.cuda.synchronize()
    for a, b, c2 in zip(A, Bv, C):
        assert torch.equal(a[1], b[1])
        assert float((a[1] - c2[1]).abs().max() / c2[1].abs().max()) < 1e-9


def test_bench_batch_sampled_instances_match_oracle():
    """The batch the bench times (64 shield instances on grids 32^3 ... 96^3, FP32, the autotuned
    schedules, one graph launch per batch step): two batch steps, then two sampled instances
    (the first of each of the two smallest grid sizes) against the oracle over the step sizes
    the GPU chose, Eq. 5 iterated to its fixed point on both sides."""
    cfgs = I.batch_configs(64, seed=1803)
    streams = [torch.cuda.Stream() for _ in cfgs]
    inst = []
    for c, s in zip(cfgs, streams):
        ctx, h, w = _make(c, S.PREC_F32, s)
        ctx.autotune()
        inst.append((ctx, h, w))
    nb = len(inst)
    t, dt = [0.0] * nb, [1e-4] * nb
    stop = [c.t_end for c in cfgs]
    hist = [[] for _ in range(nb)]
    for _ in range(2):
        t0 = list(t)
        t, dt, st = S.batch_step([a[0] for a in inst], t, dt, stop, [a[1] for a in inst], [a[2] for a in inst])
        assert all(v == 0 for v in st)
        for i in range(nb):
            hist[i].append(t[i] - t0[i])
    torch.cuda.synchronize()
    picked = {}
    for i, c in enumerate(cfgs):
        if c.n[0] in (32, 48) and c.n[0] not in picked:
            picked[c.n[0]] = i
    assert len(picked) == 2
    for size, i in sorted(picked.items()):
        c, (ctx, h, _), dts = cfgs[i], inst[i], hist[i]
        prob = O.Problem(O.Grid(c.n, c.L), c.mask, O.Material(n=c.n_power, rho_out=c.rho_out),
                         O.FieldPath(c.knots_t, c.knots_he))
        ref = O.integrate(prob, 0.0, float(np.sum(dts)), np.zeros((3,) + prob.grid.shape), rtol=c.rtol,
                          atol=c.atol, dt0=dts[0], delta_it=1e-13, max_iter=80, dt_list=dts)
        assert ref.accepted == len(dts)
        got = h.cpu().numpy().reshape(ref.y.shape)
        err = float(np.abs(got - ref.y).max() / np.abs(ref.y).max())
        print(f"[batch c4] instance {i} ({size}^3): {err:.2e}")
        assert err < 1e-4, (c.n, err)
