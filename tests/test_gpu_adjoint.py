"""Reverse mode of the fixed-iteration rhs on the GPU (through the C ABI)
against the oracle's rhs_vjp, and the autograd wrapper against central
differences of the GPU rhs itself."""

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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).reshape(-1)).cuda()


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def _setup(n, L, prec, K=3):
    mask = I.cube(n, L, 0.6 * min(L) * 2)
    jc = I.jc_noise((n[2], n[1], n[0]), 5)
    path = ([0.0, 1.0], [[0, 0, 0], [0.3, -0.2, 0.9]])
    ctx = S.Context(n, L, n_power=7.0, rho_out=5.0, precision=prec, delta_it=0.0, max_iter=K)
    ctx.set_geometry(mask)
    ctx.set_field_path(*path)
    ctx.set_jc_map(dev(jc))
    ctx.precompute_kernel()
    g = O.Grid(n, L)
    prob = O.Problem(g, mask, O.Material(n=7.0, rho_out=5.0, jc=jc), O.FieldPath(*path))
    rng = np.random.default_rng(1)
    jr = O.curl_s(rng.standard_normal((3,) + g.shape) * 0.5, g) * mask
    h = O.phi_hockney(jr, g) + 0.05
    lam = rng.standard_normal(h.shape)
    return ctx, prob, h, lam


@pytest.mark.parametrize("n,L", [((16, 32, 16), (1.0, 1.4, 0.8)), ((48, 16, 32), (1.2, 0.6, 0.9))])
def test_rhs_vjp_fp64_matches_oracle(n, L):
    K = 3
    ctx, prob, h, lam = _setup(n, L, S.PREC_F64, K)
    ref = O.rhs_vjp(prob, 0.4, h, lam, K)
    N = int(np.prod(n))
    mu_h = torch.empty(3 * N, dtype=torch.float64, device="cuda")
    mu_g = torch.empty_like(mu_h)
    mu_jc = torch.empty(N, dtype=torch.float64, device="cuda")
    mu_a = ctx.rhs_vjp(dev(h), dev(lam), mu_h, mu_g, mu_jc)
    torch.cuda.synchronize()
    assert rel(mu_h.cpu().numpy().reshape(h.shape), ref.mu_h) < 1e-10
    assert rel(mu_g.cpu().numpy().reshape(h.shape), ref.mu_g) < 1e-10
    assert rel(mu_jc.cpu().numpy().reshape(ref.mu_jc.shape), ref.mu_jc) < 1e-10
    assert rel(np.array(mu_a), ref.mu_a) < 1e-10


def test_rhs_vjp_fp32_error_is_stated():
    K = 3
    n, L = (32, 32, 32), (1.0, 1.0, 1.0)
    ctx, prob, h, lam = _setup(n, L, S.PREC_F32, K)
    ref = O.rhs_vjp(prob, 0.4, h, lam, K)
    N = int(np.prod(n))
    mu_h = torch.empty(3 * N, dtype=torch.float64, device="cuda")
    mu_jc = torch.empty(N, dtype=torch.float64, device="cuda")
    ctx.rhs_vjp(dev(h), dev(lam), mu_h, None, mu_jc)
    torch.cuda.synchronize()
    assert rel(mu_h.cpu().numpy().reshape(h.shape), ref.mu_h) < 1e-4
    assert rel(mu_jc.cpu().numpy().reshape(ref.mu_jc.shape), ref.mu_jc) < 1e-4


def test_autograd_rhs_matches_central_differences():
    K = 3
    n, L = (16, 16, 16), (1.0, 1.0, 1.0)
    ctx, prob, h, lam = _setup(n, L, S.PREC_F64, K)
    N = int(np.prod(n))
    ht = dev(h).requires_grad_(True)
    warm = torch.zeros(3 * N, dtype=torch.float64, device="cuda", requires_grad=True)
    jc = dev(prob.mat.jc).requires_grad_(True)
    out = S.rhs_autograd(ctx, 0.4, ht, warm, jc)
    lt = dev(lam)
    (out * lt).sum().backward()
    rng = np.random.default_rng(7)
    v = dev(rng.standard_normal(3 * N))
    eps = 1e-5
    with torch.no_grad():
        fp = S.rhs_autograd(ctx, 0.4, ht + eps * v, warm, jc)
        fm = S.rhs_autograd(ctx, 0.4, ht - eps * v, warm, jc)
    fd = float(((fp - fm) * lt).sum() / (2 * eps))
    assert fd == pytest.approx(float((ht.grad * v).sum()), rel=1e-6)
    dj = dev(rng.standard_normal(N) * 0.01)
    eps = 1e-4
    with torch.no_grad():
        fp = S.rhs_autograd(ctx, 0.4, ht, warm, jc + eps * dj)
        fm = S.rhs_autograd(ctx, 0.4, ht, warm, jc - eps * dj)
    fd = float(((fp - fm) * lt).sum() / (2 * eps))
    assert fd == pytest.approx(float((jc.grad * dj).sum()), rel=1e-5)


@pytest.mark.parametrize("prec,tol", [(S.PREC_F64, 1e-10), (S.PREC_F32, 1e-3)])
def test_adjoint_integrate_matches_oracle(prec, tol):
    """Checkpointed reverse sweep (checkpoints every 2 of 5 steps, so segments
    are recomputed) against the oracle's step adjoint."""
    K = 3
    n, L = (16, 16, 16), (1.0, 1.0, 1.0)
    ctx, prob, h, lam = _setup(n, L, prec, K)
    dts = [0.002, 0.003, 0.002, 0.0025, 0.003]
    ref = O.integrate_adjoint(prob, 0.1, dts, h, lam, K)
    N = int(np.prod(n))
    mu_y0 = torch.empty(3 * N, dtype=torch.float64, device="cuda")
    y_end = torch.empty_like(mu_y0)
    mu_jc = torch.empty(N, dtype=torch.float64, device="cuda")
    mu_a = ctx.adjoint_integrate(0.1, dts, dev(h), dev(lam), mu_y0, y_end=y_end, mu_jc=mu_jc, checkpoint_every=2)
    torch.cuda.synchronize()
    assert rel(y_end.cpu().numpy().reshape(h.shape), ref.y) < tol
    assert rel(mu_y0.cpu().numpy().reshape(h.shape), ref.mu_y0) < tol
    assert rel(mu_jc.cpu().numpy().reshape(ref.mu_jc.shape), ref.mu_jc) < (tol if prec == S.PREC_F64 else 1e-2)
    assert rel(np.array(mu_a), ref.mu_a) < (tol if prec == S.PREC_F64 else 1e-2)
