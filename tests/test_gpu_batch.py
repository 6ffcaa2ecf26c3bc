"""Batched instances (scfft_batch_step): independent contexts on their own
streams, stepped concurrently, give exactly the results of stepping each one
alone."""

import numpy as np
import pytest

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


def _make(cfg, prec, stream):
    ctx = S.Context(cfg.n, cfg.L, n_power=cfg.n_power, rho_out=cfg.rho_out, precision=prec, rtol=cfg.rtol,
                    atol=cfg.atol, stream=stream.cuda_stream)
    ctx.set_geometry(cfg.mask)
    ctx.set_field_path(cfg.knots_t, cfg.knots_he)
    ctx.precompute_kernel()
    N = int(np.prod(cfg.n))
    h = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    w = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    hd = np.asarray(cfg.knots_he[1]) / cfg.knots_t[1]
    for q in range(3):
        w.view(3, N)[q] = float(hd[q])
    return ctx, h, w


@pytest.mark.parametrize("prec", [S.PREC_F64, S.PREC_F32])
def test_batch_step_equals_individual_steps(prec):
    cfgs = I.batch_configs(4, seed=7)
    for c in cfgs:  # keep the test small: 32^3 copies of each instance
        c.n = (32, 32, 32)
        c.mask = I.shield(c.n, c.L, 1.0, 0.8, 2.0, 0.2)
    streams = [torch.cuda.Stream() for _ in cfgs]
    A = [_make(c, prec, s) for c, s in zip(cfgs, streams)]
    Bv = [_make(c, prec, s) for c, s in zip(cfgs, streams)]
    t = [0.0] * 4
    dt = [1e-4] * 4
    stop = [c.t_end for c in cfgs]
    for _ in range(3):
        t, dt, st = S.batch_step([a[0] for a in A], t, dt, stop, [a[1] for a in A], [a[2] for a in A])
        assert all(v == 0 for v in st)
    torch.cuda.synchronize()
    for (ctx, h, w), c, tb in zip(Bv, cfgs, t):
        tt, d = 0.0, 1e-4
        for _ in range(3):
            tt, d, _ = ctx.step(tt, d, c.t_end, h, w)
        assert tt == tb
    torch.cuda.synchronize()
    for a, b in zip(A, Bv):
        assert torch.equal(a[1], b[1])
