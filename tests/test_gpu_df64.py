"""GPU parity of the double-float path (SCFFT_PREC_DF64): every FFT pass in double-float
arithmetic (hi + lo FP32 pairs, unit roundoff 2^-48), the node-wise law in FP64, FP64 state
and stages, against the FP64 oracle, element by element.

Tolerance: the FP64 path's tier.  A double-float operation rounds at 2^-48 = 3.6e-15 where
FP64 rounds at 1.1e-16; a transform chain of the rhs adds up a few hundred such roundings per
output (relative to the field's magnitude), so the expected error is a few 1e-13 at most,
and the FP64 path's bounds (1e-12 for the operators, 1e-10 for the rhs and the integrator)
hold with room.  The observed errors are printed (pytest -s)."""

import numpy as np
import pytest

import oracle as O
import scfft_inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1803_01346_gb300 as S  # noqa: E402
from paper_1803_01346_gb300 import build as B  # noqa: E402

DF = S.PREC_DF64


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def check(name, a, b, bound):
    e = rel(a, b)
    print(f"[df64 error] {name}: {e:.2e}")
    assert e < bound, (name, e, bound)


def make(n, L, mask, n_power=20.0, rho_out=20.0, delta_it=0.0, max_iter=3, jc_map=None):
    path = ([0.0, 1.0], [[0, 0, 0], [0.3, -0.2, 0.9]])
    ctx = S.Context(n, L, n_power=n_power, rho_out=rho_out, precision=DF, delta_it=delta_it, max_iter=max_iter)
    ctx.set_geometry(mask)
    ctx.set_field_path(*path)
    if jc_map is not None:
        ctx.set_jc_map(dev(jc_map).reshape(-1))
    ctx.precompute_kernel()
    prob = O.Problem(O.Grid(tuple(n), tuple(L)), mask.astype(bool),
                     O.Material(n=n_power, rho_out=rho_out, jc=1.0 if jc_map is None else jc_map),
                     O.FieldPath(*path))
    return ctx, prob


def _state(prob, seed):
    g = prob.grid
    j = O.curl_s(I.random_field((3,) + g.shape, seed, 0.3), g) * prob.mask[None]
    return O.phi_hockney(j, g) + np.array([0.05, -0.02, 0.1])[:, None, None, None]


# every FFT length the passes support: 16 ... 128 unpadded, 32 ... 256 padded, and ragged
# column tiles
GRIDS = [((16, 32, 48), (0.8, 1.0, 1.2)),
         ((48, 64, 96), (1.0, 1.1, 1.5)),
         ((32, 96, 128), (0.7, 1.2, 1.6)),
         ((64, 128, 16), (1.0, 1.6, 0.5))]


@pytest.mark.parametrize("n,L", GRIDS)
def test_curl_df64_matches_oracle(n, L):
    g = O.Grid(n, L)
    f = I.random_field((3,) + g.shape, 71)
    ctx = S.Context(n, L, precision=DF)
    out = torch.empty(f.size, dtype=torch.float64, device="cuda")
    ctx.curl(dev(f).reshape(-1), out)
    check(f"curl {n}", host(out).reshape(f.shape), O.curl_s(f, g), 1e-12)


@pytest.mark.parametrize("n,L", GRIDS)
def test_phi_df64_matches_oracle(n, L):
    g = O.Grid(n, L)
    j = I.random_field((3,) + g.shape, 72)
    ctx = S.Context(n, L, precision=DF)
    ctx.precompute_kernel()
    out = torch.empty(j.size, dtype=torch.float64, device="cuda")
    ctx.phi(dev(j).reshape(-1), out)
    check(f"phi {n}", host(out).reshape(j.shape), O.phi_hockney(j, g), 1e-12)


def test_phi_df64_matches_direct_sum():
    n, L = (16, 16, 16), (1.0, 1.1, 0.9)
    g = O.Grid(n, L)
    j = I.random_field((3,) + g.shape, 73)
    ctx = S.Context(n, L, precision=DF)
    ctx.precompute_kernel()
    out = torch.empty(j.size, dtype=torch.float64, device="cuda")
    ctx.phi(dev(j).reshape(-1), out)
    check("phi vs direct sum", host(out).reshape(j.shape), O.phi_direct(j, g), 1e-12)


def test_df64_is_closer_to_the_oracle_than_fp32_by_orders():
    """The point of the mode: FP64-equivalent operators, not FP32 ones (FP32 passes give
    about 1e-7 here)."""
    n, L = (48, 32, 16), (1.2, 0.9, 0.8)
    g = O.Grid(n, L)
    j = I.random_field((3,) + g.shape, 74)
    ref = O.phi_hockney(j, g)
    err = {}
    for p in (S.PREC_F32, DF, S.PREC_F64):
        ctx = S.Context(n, L, precision=p)
        ctx.precompute_kernel()
        out = torch.empty(j.size, dtype=torch.float64, device="cuda")
        ctx.phi(dev(j).reshape(-1), out)
        err[p] = rel(host(out).reshape(j.shape), ref)
    print(f"[df64 error] phi 48x32x16: fp32 {err[S.PREC_F32]:.2e} df64 {err[DF]:.2e} fp64 {err[S.PREC_F64]:.2e}")
    assert err[DF] < 1e-5 * err[S.PREC_F32]


@pytest.mark.parametrize("n,L", [((16, 16, 16), (1.0, 1.0, 1.0)), ((48, 32, 16), (1.2, 0.9, 0.8)),
                                 ((32, 16, 96), (0.8, 0.5, 2.0))])
def test_rhs_df64_fixed_iterations_matches_oracle(n, L):
    mask = I.cube(n, L, 0.6 * min(L) * 2)
    ctx, prob = make(n, L, mask)
    h = _state(prob, 75)
    g0 = I.random_field(h.shape, 76, 0.1)
    ref = O.rhs(prob, 0.4, h, g0, delta_it=0.0, max_iter=3)
    hd = torch.empty(h.size, dtype=torch.float64, device="cuda")
    warm = dev(g0).reshape(-1)
    assert ctx.rhs(0.4, dev(h).reshape(-1), warm, hd) == 3
    check(f"rhs {n}", host(hd).reshape(h.shape), ref.hdot, 1e-10)
    check(f"rhs warm {n}", host(warm).reshape(h.shape), ref.hdot, 1e-10)


def test_rhs_df64_early_stop_and_jc_map():
    """Lens 32^3, n = 30, rho_out = 100, a jc map, the paper's delta_it: the same iteration
    count as the oracle and its dh/dt."""
    n, L = (32, 32, 32), (1.0, 1.0, 1.0)
    mask = I.lens(n, L, 0.6, 0.5, 0.1, 0.1)
    jc = I.jc_noise((32, 32, 32), 5)
    ctx, prob = make(n, L, mask, n_power=30.0, rho_out=100.0, delta_it=2e-5, max_iter=50, jc_map=jc)
    h = _state(prob, 77)
    g0 = np.broadcast_to(prob.path.hedot(0.2)[:, None, None, None], h.shape).copy()
    ref = O.rhs(prob, 0.2, h, g0, delta_it=2e-5, max_iter=50)
    hd = torch.empty(h.size, dtype=torch.float64, device="cuda")
    it = ctx.rhs(0.2, dev(h).reshape(-1), dev(g0).reshape(-1), hd)
    assert it == ref.iters
    check("rhs lens32 early stop", host(hd).reshape(h.shape), ref.hdot, 1e-10)


def test_rhs_df64_ej_law_and_stencil_curl():
    """The e(j, h) law (Kim jc(|h|), anisotropic norm) and the local-stencil curl through the
    double-float passes."""
    n, L = (32, 48, 32), (1.0, 1.2, 0.9)
    mask = I.cube(n, L, 0.6 * min(L) * 2)
    ctx, prob = make(n, L, mask, n_power=25.0)
    ctx.set_ej_law(kim_h0=0.3, aniso=(1.0, 0.7, 1.5))
    prob.mat.kim_h0 = 0.3
    prob.mat.aniso = (1.0, 0.7, 1.5)
    h = _state(prob, 78)
    g0 = I.random_field(h.shape, 79, 0.1)
    hd = torch.empty(h.size, dtype=torch.float64, device="cuda")
    ref = O.rhs(prob, 0.4, h, g0, delta_it=0.0, max_iter=3)
    assert ctx.rhs(0.4, dev(h).reshape(-1), dev(g0).reshape(-1), hd) == 3
    check("rhs e(j,h) law", host(hd).reshape(h.shape), ref.hdot, 1e-10)
    ctx.set_curl(S.CURL_FD)
    prob.curl = "fd"
    ref = O.rhs(prob, 0.4, h, g0, delta_it=0.0, max_iter=3)
    assert ctx.rhs(0.4, dev(h).reshape(-1), dev(g0).reshape(-1), hd) == 3
    check("rhs e(j,h) law, stencil curl", host(hd).reshape(h.shape), ref.hdot, 1e-10)


def test_integrate_fixed_steps_df64_matches_oracle():
    """Tier T2: fixed dt list, Eq. 5 iterated to its fixed point (delta_it 1e-13, which the
    double-float iterates reach: their differences round at a few 1e-15)."""
    cfg = I.config("cube16")
    prob = O.Problem(O.Grid(cfg.n, cfg.L), cfg.mask, O.Material(n=cfg.n_power, rho_out=cfg.rho_out),
                     O.FieldPath(cfg.knots_t, cfg.knots_he))
    dts = [0.002, 0.003, 0.004, 0.004, 0.005, 0.005]
    ctx = S.Context(cfg.n, cfg.L, n_power=cfg.n_power, rho_out=cfg.rho_out, delta_it=1e-13, max_iter=80,
                    precision=DF)
    ctx.set_geometry(cfg.mask)
    ctx.set_field_path(cfg.knots_t, cfg.knots_he)
    ctx.precompute_kernel()
    N = int(np.prod(cfg.n))
    h = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    t1 = float(np.sum(dts))
    st = ctx.integrate(0.0, t1, dts[0], h, dt_fixed=dts)
    ref = O.integrate(prob, 0.0, t1, np.zeros((3,) + prob.grid.shape), rtol=1e-6, atol=1e-9, dt0=dts[0],
                      delta_it=1e-13, max_iter=80, dt_list=dts)
    assert st["accepted"] == len(dts)
    check("integrate T2 cube16", host(h).reshape(ref.y.shape), ref.y, 1e-10)


def test_rhs_vjp_df64_matches_oracle():
    """The transposed passes in double-float: rhs_vjp against the oracle's reverse mode."""
    n, L = (16, 32, 16), (1.0, 1.4, 0.8)
    K = 3
    mask = I.cube(n, L, 0.6 * min(L) * 2)
    jc = I.jc_noise((n[2], n[1], n[0]), 5)
    path = ([0.0, 1.0], [[0, 0, 0], [0.3, -0.2, 0.9]])
    ctx = S.Context(n, L, n_power=7.0, rho_out=5.0, precision=DF, delta_it=0.0, max_iter=K)
    ctx.set_geometry(mask)
    ctx.set_field_path(*path)
    ctx.set_jc_map(dev(jc).reshape(-1))
    ctx.precompute_kernel()
    g = O.Grid(n, L)
    prob = O.Problem(g, mask, O.Material(n=7.0, rho_out=5.0, jc=jc), O.FieldPath(*path))
    rng = np.random.default_rng(1)
    h = O.phi_hockney(O.curl_s(rng.standard_normal((3,) + g.shape) * 0.5, g) * mask, g) + 0.05
    lam = rng.standard_normal(h.shape)
    ref = O.rhs_vjp(prob, 0.4, h, lam, K)
    N = int(np.prod(n))
    mu_h = torch.empty(3 * N, dtype=torch.float64, device="cuda")
    mu_g = torch.empty_like(mu_h)
    mu_jc = torch.empty(N, dtype=torch.float64, device="cuda")
    mu_a = ctx.rhs_vjp(dev(h).reshape(-1), dev(lam).reshape(-1), mu_h, mu_g, mu_jc)
    check("vjp mu_h", host(mu_h).reshape(h.shape), ref.mu_h, 1e-10)
    check("vjp mu_g", host(mu_g).reshape(h.shape), ref.mu_g, 1e-10)
    check("vjp mu_jc", host(mu_jc).reshape(ref.mu_jc.shape), ref.mu_jc, 1e-10)
    check("vjp mu_a", np.array(mu_a), ref.mu_a, 1e-10)


def test_df64_small_magnitudes_keep_their_relative_accuracy():
    """FP32's exponent range bounds the mode: a field scaled by 1e-20 keeps its low parts
    (about 1e-27) and their products with the twiddles in FP32's normal range, so it
    transforms with the same relative error (below about 1e-30 the low parts would turn
    subnormal and the error would grow)."""
    n, L = (32, 32, 32), (1.0, 1.0, 1.0)
    g = O.Grid(n, L)
    f = I.random_field((3,) + g.shape, 80)
    ctx = S.Context(n, L, precision=DF)
    out = torch.empty(f.size, dtype=torch.float64, device="cuda")
    ref = O.curl_s(f, g)
    ctx.curl(dev(f).reshape(-1), out)
    e1 = rel(host(out).reshape(f.shape), ref)
    ctx.curl(dev(f * 1e-20).reshape(-1), out)
    e2 = rel(host(out).reshape(f.shape), ref * 1e-20)
    print(f"[df64 error] curl at scale 1 / 1e-20: {e1:.2e} / {e2:.2e}")
    assert e1 < 1e-12 and e2 < 1e-12
