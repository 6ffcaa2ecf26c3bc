"""Device-resident stepping (scfft_advance): the whole sequence of BS23 trials of the FP32
path as one CUDA graph launch (trial step, stage parameters, stage right-hand sides with
their Eq. 5 loops, error norm and step controller on the device).  It must take the same
steps as the host-driven scfft_step (up to the rounding of the device's pow in the step
controller), stop exactly on a kink of the path, retry rejected trials, and track the FP64
oracle; with the stencil curl too."""

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


def _ctx(cfg, curl=S.CURL_SPECTRAL, rtol=1e-4, atol=1e-7):
    ctx = S.Context(cfg.n, cfg.L, n_power=cfg.n_power, rho_out=cfg.rho_out, precision=S.PREC_F32, delta_it=2e-5,
                    max_iter=100, rtol=rtol, atol=atol)
    ctx.set_geometry(cfg.mask)
    ctx.set_field_path(cfg.knots_t, cfg.knots_he)
    ctx.set_curl(curl)
    ctx.precompute_kernel()
    N = int(np.prod(cfg.n))
    h = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    w = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    hd = np.asarray(cfg.knots_he[1]) / cfg.knots_t[1]
    for q in range(3):
        w.view(3, N)[q] = float(hd[q])
    return ctx, h, w


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max().clamp_min(1e-300))


@pytest.mark.parametrize("curl", [S.CURL_SPECTRAL, S.CURL_FD])
def test_advance_takes_the_host_steps(curl):
    cfg = I.config("lens128", scale=(32, 32, 32))
    a, ha, wa = _ctx(cfg, curl)
    b, hb, wb = _ctx(cfg, curl)
    ta, da = 0.0, 1e-5
    tb, db = 0.0, 1e-5
    for _ in range(12):
        tb, db, _ = b.step(tb, db, 10.0, hb, wb)
    ta, da, n = a.advance(ta, da, 10.0, 12, ha, wa)
    assert n == 12
    assert ta == pytest.approx(tb, rel=1e-12)
    assert _rel(ha, hb) < 1e-9 and _rel(wa, wb) < 1e-9
    sa, sb = a.stats(), b.stats()
    assert sa["accepted"] == sb["accepted"] and sa["rhs_calls"] == sb["rhs_calls"]
    assert sa["iterations"] == sb["iterations"]
    # a second call continues the trajectory (FSAL) as the host steps do
    ta, da, n = a.advance(ta, da, 10.0, 5, ha, wa)
    for _ in range(5):
        tb, db, _ = b.step(tb, db, 10.0, hb, wb)
    assert ta == pytest.approx(tb, rel=1e-12) and _rel(ha, hb) < 1e-9


def test_advance_stops_on_the_kink_and_retries_rejected_trials():
    """The cube's path turns at t = 1 (ramp up, then down); an over-large first step is
    rejected and retried on the device; the call ends exactly on the kink and the next call
    restarts from it; the trajectory tracks the FP64 oracle's adaptive run."""
    cfg = I.config("cube16")
    cfg.knots_t = [0.0, 0.05, 0.1]
    cfg.knots_he = [[0, 0, 0], [0, 0, 0.025], [0, 0, 0.0]]
    a, h, w = _ctx(cfg, rtol=1e-4, atol=1e-7)
    t, dt = 0.0, 0.02  # far too large: rejected trials first
    t, dt, n = a.advance(t, dt, 0.1, 1000, h, w)
    assert t == 0.05 and n > 0
    assert a.stats()["rejected"] > 0
    t, dt, n2 = a.advance(t, dt, 0.1, 1000, h, w)
    assert t == 0.1
    prob = O.Problem(O.Grid(cfg.n, cfg.L), cfg.mask, O.Material(n=cfg.n_power, rho_out=cfg.rho_out),
                     O.FieldPath(cfg.knots_t, cfg.knots_he))
    ref = O.integrate(prob, 0.0, 0.1, np.zeros((3,) + prob.grid.shape), rtol=1e-4, atol=1e-7, dt0=1e-4)
    got = h.cpu().numpy().reshape(ref.y.shape)
    assert np.abs(got - ref.y).max() / np.abs(ref.y).max() < 2e-3
