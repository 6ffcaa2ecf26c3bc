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


def _lens_problem(n, prec, K):
    """The 96^3 lens adjoint workload at a small grid: the lens in a box of side 3.2,
    jc = 1 + U[-0.05, 0.05] (seeded), n = 30, rho_out = 100, an axial ramp at rate 1 to
    amplitude A then a hold (a kink at t = A)."""
    cfg = I.config("lens96", scale=n)
    jc = np.ascontiguousarray(I.jc_noise((n[2], n[1], n[0]), 1346))
    A = np.array([0.02, -0.01, 0.12])
    tk = [0.0, 0.12, 1.0]
    he = np.stack([np.zeros(3), A, A])
    ctx = S.Context(n, cfg.L, n_power=cfg.n_power, rho_out=cfg.rho_out, precision=prec, delta_it=0.0,
                    max_iter=K)
    ctx.set_geometry(cfg.mask)
    ctx.set_field_path(tk, he)
    ctx.set_jc_map(dev(jc))
    ctx.precompute_kernel()
    g = O.Grid(n, cfg.L)
    prob = O.Problem(g, cfg.mask, O.Material(n=cfg.n_power, rho_out=cfg.rho_out, jc=jc), O.FieldPath(tk, he))
    rng = np.random.default_rng(1346)
    # the field of a random current in the lens, scaled so that the largest |curl h| in the
    # lens is 0.8 jc (the power law of Eq. 1 is steep there but the steps below stay stable)
    P = O.phi_hockney(O.curl_s(rng.standard_normal((3,) + g.shape), g) * cfg.mask, g)
    jP = np.sqrt(np.sum(O.curl_s(P, g) ** 2, axis=0))[cfg.mask].max()
    y0 = (0.8 / jP) * P + np.array([0.0, 0.0, 0.1])[:, None, None, None]
    return ctx, prob, cfg, jc, tk, he, y0, rng


def _reverse(ctx, ts, y0, lam, N, P):
    y_end = torch.empty(3 * N, dtype=torch.float64, device="cuda")
    S_ = ctx.adjoint_record(ts, dev(y0), y_end=y_end, checkpoint_every=2)
    lam_h = dev(lam).clone()
    gjc = torch.zeros(N, dtype=torch.float64, device="cuda")
    gp = np.zeros(P)
    for k in range(S_ - 1, -1, -1):
        ctx.adjoint_step(k, lam_h, gjc, gp)
    torch.cuda.synchronize()
    return y_end, lam_h, gjc, gp


# five steps; the second ends on the ramp's kink (t = 0.12).  rho_out = 100 makes the
# explicit steps stiff: dt = 2e-4 keeps dt times the largest eigenvalue near 1 at 32^3
TS = [0.1196, 0.1198, 0.12, 0.1202, 0.12045, 0.1207]


@pytest.mark.parametrize("prec,tol", [(S.PREC_F64, 1e-10), (S.PREC_F32, 1e-3)])
def test_adjoint_step_lens_matches_oracle(prec, tol):
    """scfft_adjoint_step over a recorded trajectory that crosses the ramp-to-hold kink,
    checkpoints every 2 steps: the state, dJ/dy_0, dJ/djc and the path gradient (knot
    amplitudes) against the oracle's step adjoint."""
    K, n = 3, (32, 32, 32)
    ctx, prob, cfg, jc, tk, he, y0, rng = _lens_problem(n, prec, K)
    N = int(np.prod(n))
    lam = rng.standard_normal(y0.shape)
    ref = O.integrate_adjoint(prob, None, None, y0, lam, K, ts=TS)
    y_end, mu_y0, gjc, gp = _reverse(ctx, TS, y0, lam, N, 3 * len(tk) + 1)
    assert rel(y_end.cpu().numpy().reshape(y0.shape), ref.y) < tol
    assert rel(mu_y0.cpu().numpy().reshape(y0.shape), ref.mu_y0) < tol
    assert rel(gjc.cpu().numpy().reshape(ref.mu_jc.shape), ref.mu_jc) < (tol if prec == S.PREC_F64 else 1e-2)
    assert rel(gp, ref.mu_path) < (tol if prec == S.PREC_F64 else 1e-2)


def test_adjoint_step_lens_matches_central_differences_of_the_gpu_forward():
    """dJ/djc on 16 seeded voxels of the lens and dJ/dA for the three components of the
    ramp amplitude (A enters both knots of the ramp-then-hold path) against central
    differences (step 1e-4) of the GPU's own forward map over the same step times."""
    K, n = 3, (32, 32, 32)
    ctx, prob, cfg, jc, tk, he, y0, rng = _lens_problem(n, S.PREC_F64, K)
    N = int(np.prod(n))
    lam = rng.standard_normal(y0.shape)
    lt = dev(lam)
    _, _, gjc, gp = _reverse(ctx, TS, y0, lam, N, 3 * len(tk) + 1)
    gjc = gjc.cpu().numpy()

    def J():
        y = torch.empty(3 * N, dtype=torch.float64, device="cuda")
        ctx.adjoint_record(TS, dev(y0), y_end=y, checkpoint_every=2)
        return float((y * lt).sum())

    eps = 1e-4
    inside = np.flatnonzero(cfg.mask.reshape(-1))
    vox = np.random.default_rng(16).choice(inside, 16, replace=False)
    scale = np.abs(gjc).max()
    for v in vox:
        for sgn, store in ((1, "p"), (-1, "m")):
            j2 = jc.reshape(-1).copy()
            j2[v] += sgn * eps
            ctx.set_jc_map(dev(j2))
            if sgn > 0:
                jp = J()
            else:
                jm = J()
        fd = (jp - jm) / (2 * eps)
        # central differences err by about (eps^2 / 6) f'''/f' ~ 2e-6 relative here (rho ~ jc^-n, n = 30)
        assert abs(fd - gjc[v]) < 1e-6 * scale + 2e-5 * abs(gjc[v]), (v, fd, gjc[v])
    ctx.set_jc_map(dev(jc))
    dA = gp[3:6] + gp[6:9]
    for a in range(3):
        vals = []
        for sgn in (1, -1):
            h2 = he.copy()
            h2[1:, a] += sgn * eps
            ctx.set_field_path(tk, h2)
            vals.append(J())
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert fd == pytest.approx(dA[a], rel=2e-5, abs=1e-9 * np.abs(dA).max()), (a, fd, dA[a])
    ctx.set_field_path(tk, he)


def test_integrate_autograd_gradients():
    """The checkpointed reverse sweep behind torch.autograd: gradients of <lam, y_end>
    for y0, jc and the knot amplitudes equal the per-step calls'."""
    K, n = 3, (16, 16, 16)
    ctx, prob, cfg, jc, tk, he, y0, rng = _lens_problem(n, S.PREC_F64, K)
    N = int(np.prod(n))
    lam = rng.standard_normal(y0.shape)
    y0t = dev(y0).requires_grad_(True)
    jct = dev(jc).requires_grad_(True)
    het = torch.tensor(he, dtype=torch.float64, requires_grad=True)
    out = S.integrate_autograd(ctx, TS, y0t, jct, tk, het, checkpoint_every=2)
    (out * dev(lam)).sum().backward()
    ref = O.integrate_adjoint(prob, None, None, y0, lam, K, ts=TS)
    assert rel(y0t.grad.cpu().numpy().reshape(y0.shape), ref.mu_y0) < 1e-10
    assert rel(jct.grad.cpu().numpy().reshape(ref.mu_jc.shape), ref.mu_jc) < 1e-10
    assert rel(het.grad.numpy().reshape(-1), ref.mu_path[:-1]) < 1e-10


@pytest.mark.parametrize("prec,tol", [(S.PREC_F64, 1e-10), (S.PREC_F32, 1e-4)])
def test_rhs_vjp_lens96_matches_oracle(prec, tol):
    """The reverse mode's workload grid: the lens at 96^3 with its seeded +-5% jc map (the
    bench's reverse-mode leg), one rhs with three fixed Eq. 5 iterations, its vector-Jacobian
    product against the oracle's (FP64 tier and the FP32 path's stated bound)."""
    K = 3
    cfg = I.config("lens96")
    n, L = cfg.n, cfg.L
    ctx = S.Context(n, L, n_power=cfg.n_power, rho_out=cfg.rho_out, precision=prec, delta_it=0.0, max_iter=K)
    ctx.set_geometry(cfg.mask)
    ctx.set_field_path(cfg.knots_t, cfg.knots_he)
    ctx.set_jc_map(dev(cfg.jc))
    ctx.precompute_kernel()
    g = O.Grid(n, L)
    prob = O.Problem(g, cfg.mask, O.Material(n=cfg.n_power, rho_out=cfg.rho_out, jc=cfg.jc),
                     O.FieldPath(cfg.knots_t, cfg.knots_he))
    rng = np.random.default_rng(96)
    # the field of a random current in the lens, scaled so that the largest |curl h| in the lens
    # is 1.1 jc (the steep part of Eq. 1 at n = 30), plus a uniform field
    P = O.phi_hockney(O.curl_s(rng.standard_normal((3,) + g.shape) * 0.3, g) * cfg.mask, g)
    jP = np.sqrt(np.sum(O.curl_s(P, g) ** 2, axis=0))[cfg.mask].max()
    h = (1.1 / jP) * P + np.array([0.0, 0.0, 0.4])[:, None, None, None]
    lam = rng.standard_normal(h.shape)
    ref = O.rhs_vjp(prob, 0.4, h, lam, K)
    N = int(np.prod(n))
    mu_h = torch.empty(3 * N, dtype=torch.float64, device="cuda")
    mu_jc = torch.empty(N, dtype=torch.float64, device="cuda")
    ctx.rhs_vjp(dev(h), dev(lam), mu_h, None, mu_jc)
    torch.cuda.synchronize()
    e_h = rel(mu_h.cpu().numpy().reshape(h.shape), ref.mu_h)
    e_jc = rel(mu_jc.cpu().numpy().reshape(ref.mu_jc.shape), ref.mu_jc)
    print(f"[rhs_vjp lens96 precision {prec}] mu_h {e_h:.2e} mu_jc {e_jc:.2e}")
    assert e_h < tol and e_jc < tol


# the same five steps at the reverse-mode workload's own grid (96^3, a third of the cell size:
# the explicit steps' stiffness grows ninefold, so the steps are ten times shorter), the second
# again ending on the kink
TS96 = [0.11996, 0.11998, 0.12, 0.12002, 0.120045, 0.12007]


def test_adjoint_step_lens96_matches_central_differences_of_the_gpu_forward():
    """The reverse-mode workload's grid (lens 96^3 with its +-5% jc map, FP64): dJ/djc on 8
    seeded voxels of the lens and dJ/dA for the three ramp-amplitude components across the
    ramp-to-hold kink, against central differences (step 1e-4) of the GPU's own forward map."""
    K, n = 3, (96, 96, 96)
    ctx, prob, cfg, jc, tk, he, y0, rng = _lens_problem(n, S.PREC_F64, K)
    N = int(np.prod(n))
    lam = rng.standard_normal(y0.shape)
    lt = dev(lam)
    _, _, gjc, gp = _reverse(ctx, TS96, y0, lam, N, 3 * len(tk) + 1)
    gjc = gjc.cpu().numpy()

    def J():
        y = torch.empty(3 * N, dtype=torch.float64, device="cuda")
        ctx.adjoint_record(TS96, dev(y0), y_end=y, checkpoint_every=2)
        return float((y * lt).sum())

    eps = 1e-4
    inside = np.flatnonzero(cfg.mask.reshape(-1))
    vox = np.random.default_rng(96).choice(inside, 8, replace=False)
    scale = np.abs(gjc).max()
    for v in vox:
        vals = []
        for sgn in (1, -1):
            j2 = jc.reshape(-1).copy()
            j2[v] += sgn * eps
            ctx.set_jc_map(dev(j2))
            vals.append(J())
        fd = (vals[0] - vals[1]) / (2 * eps)
        assert abs(fd - gjc[v]) < 1e-6 * scale + 2e-5 * abs(gjc[v]), (v, fd, gjc[v])
    ctx.set_jc_map(dev(jc))
    dA = gp[3:6] + gp[6:9]
    for a in range(3):
        vals = []
        for sgn in (1, -1):
            h2 = he.copy()
            h2[1:, a] += sgn * eps
            ctx.set_field_path(tk, h2)
            vals.append(J())
        fd = (vals[0] - vals[1]) / (2 * eps)
        print(f"[adjoint lens96] dJ/dA_{a}: reverse {dA[a]:.6e}, central difference {fd:.6e}")
        assert fd == pytest.approx(dA[a], rel=2e-5, abs=1e-9 * np.abs(dA).max()), (a, fd, dA[a])
    ctx.set_field_path(tk, he)
