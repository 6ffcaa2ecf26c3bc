"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the
same seeded inputs, element by element.

Tolerances (relative to the largest oracle magnitude of each field):
  FP64 path      <= 1e-10 (every stage is a sum of at most ~1e3 rounded terms)
  FP32 path      stated per field in the tests below (FP32 FFT round-off
                 ~1e-6 amplified by the power law's exponent n).
"""

import math

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
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def rel3(a, b):
    """Per-component relative error of a (3, ...) field: max |a_q - b_q| / max |b_q|."""
    return [rel(a[q], b[q]) for q in range(3)]


def check3(name, a, b, bounds):
    """Assert the per-component error of the FP32 path against its stated bounds."""
    e = rel3(a, b)
    print(f"[fp32 error] {name}: " + " ".join(f"{v:.2e}" for v in e))
    assert all(v < bd for v, bd in zip(e, bounds)), (name, e, bounds)
    return e


def make(n, L, mask, n_power=20.0, rho_out=20.0, prec=S.PREC_F64, delta_it=0.0, max_iter=3, path=None,
         jc_map=None, sigma_scale=1.0, rtol=2e-4, atol=1e-6):
    ctx = S.Context(n, L, n_power=n_power, rho_out=rho_out, precision=prec, delta_it=delta_it,
                    max_iter=max_iter, sigma_scale=sigma_scale, rtol=rtol, atol=atol)
    ctx.set_geometry(mask)
    t, he = path if path is not None else ([0.0, 1.0], [[0, 0, 0], [0.3, -0.2, 0.9]])
    ctx.set_field_path(t, he)
    if jc_map is not None:
        ctx.set_jc_map(dev(jc_map))
    ctx.precompute_kernel()
    g = O.Grid(tuple(n), tuple(L), sigma_scale=sigma_scale)
    prob = O.Problem(g, mask.astype(bool), O.Material(n=n_power, rho_out=rho_out,
                                                      jc=1.0 if jc_map is None else jc_map),
                     O.FieldPath(t, he))
    return ctx, prob


# FP32 path: per-component bounds of max |GPU - oracle| / max |oracle| (about three times
# the errors observed on GB300, printed by check3 under pytest -s)
# (observed: curl and Phi <= 2.9e-7 per component, rhs with 3 Eq. 5 iterations <= 2.1e-6)
CURL32 = (1e-6, 1e-6, 1e-6)
PHI32 = (1e-6, 1e-6, 1e-6)
RHS32 = (6e-6, 6e-6, 6e-6)

GRIDS = [((16, 16, 16), (1.0, 1.0, 1.0)),
         ((48, 32, 16), (1.2, 0.9, 0.8)),     # ragged column tiles (25 and 17 spectral columns)
         ((32, 16, 96), (0.8, 0.5, 2.0))]


@pytest.mark.parametrize("n,L", GRIDS)
def test_curl_fp64_matches_oracle(n, L):
    g = O.Grid(n, L)
    f = I.random_field((3,) + g.shape, 7)
    ctx = S.Context(n, L)
    out = torch.empty(3 * g.shape[0] * g.shape[1] * g.shape[2], dtype=torch.float64, device="cuda")
    ctx.curl(dev(f).reshape(-1), out)
    assert rel(host(out).reshape(f.shape), O.curl_s(f, g)) < 1e-12


@pytest.mark.parametrize("n,L", GRIDS)
def test_phi_fp64_matches_oracle(n, L):
    g = O.Grid(n, L)
    j = I.random_field((3,) + g.shape, 8)
    ctx = S.Context(n, L)
    ctx.precompute_kernel()
    out = torch.empty(j.size, dtype=torch.float64, device="cuda")
    ctx.phi(dev(j).reshape(-1), out)
    assert rel(host(out).reshape(j.shape), O.phi_hockney(j, g)) < 1e-12


# every FFT length on both grids: 16 32 48 64 96 128 (unpadded), 32 ... 256 (padded)
GRIDS32 = [((16, 32, 48), (0.8, 1.0, 1.2)),
           ((48, 64, 96), (1.0, 1.1, 1.5)),
           ((32, 96, 128), (0.7, 1.2, 1.6)),
           ((64, 128, 16), (1.0, 1.6, 0.5))]


@pytest.mark.parametrize("n,L", GRIDS32)
def test_curl_fp32_matches_oracle(n, L):
    """FP32 register passes vs the FP64 oracle: FP32 FFT round-off only."""
    g = O.Grid(n, L)
    f = I.random_field((3,) + g.shape, 17)
    ctx = S.Context(n, L, precision=S.PREC_F32)
    out = torch.empty(f.size, dtype=torch.float64, device="cuda")
    ctx.curl(dev(f).reshape(-1), out)
    check3(f"curl {n}", host(out).reshape(f.shape), O.curl_s(f, g), CURL32)


@pytest.mark.parametrize("n,L", GRIDS32)
def test_phi_fp32_matches_oracle(n, L):
    g = O.Grid(n, L)
    j = I.random_field((3,) + g.shape, 18)
    ctx = S.Context(n, L, precision=S.PREC_F32)
    ctx.precompute_kernel()
    out = torch.empty(j.size, dtype=torch.float64, device="cuda")
    ctx.phi(dev(j).reshape(-1), out)
    check3(f"phi {n}", host(out).reshape(j.shape), O.phi_hockney(j, g), PHI32)


def test_phi_fp64_matches_direct_sum():
    n, L = (16, 16, 16), (1.0, 1.1, 0.9)
    g = O.Grid(n, L)
    j = I.random_field((3,) + g.shape, 9)
    ctx = S.Context(n, L)
    ctx.precompute_kernel()
    out = torch.empty(j.size, dtype=torch.float64, device="cuda")
    ctx.phi(dev(j).reshape(-1), out)
    assert rel(host(out).reshape(j.shape), O.phi_direct(j, g)) < 1e-12


def _state(prob, seed):
    """A smooth, nonzero field: h_e plus the field of a random current in Omega."""
    g = prob.grid
    j = O.curl_s(I.random_field((3,) + g.shape, seed, 0.3), g) * prob.mask[None]
    return O.phi_hockney(j, g) + np.array([0.05, -0.02, 0.1])[:, None, None, None]


@pytest.mark.parametrize("n,L", GRIDS)
def test_rhs_fp64_fixed_iterations_matches_oracle(n, L):
    mask = I.cube(n, L, 0.6 * min(L) * 2)
    ctx, prob = make(n, L, mask, max_iter=3)
    h = _state(prob, 3)
    g0 = I.random_field(h.shape, 4, 0.1)
    ref = O.rhs(prob, 0.4, h, g0, delta_it=0.0, max_iter=3)
    hd = torch.empty(h.size, dtype=torch.float64, device="cuda")
    warm = dev(g0).reshape(-1)
    it = ctx.rhs(0.4, dev(h).reshape(-1), warm, hd)
    assert it == 3
    assert rel(host(hd).reshape(h.shape), ref.hdot) < 1e-10
    assert rel(host(warm).reshape(h.shape), ref.hdot) < 1e-10


def test_rhs_fp64_early_stop_and_jc_map():
    n, L = (32, 32, 32), (1.0, 1.0, 1.0)
    mask = I.lens(n, L, 0.6, 0.5, 0.1, 0.1)
    jc = I.jc_noise((32, 32, 32), 5)
    ctx, prob = make(n, L, mask, n_power=30.0, rho_out=100.0, delta_it=2e-5, max_iter=50, jc_map=jc)
    h = _state(prob, 6)
    g0 = np.broadcast_to(prob.path.hedot(0.2)[:, None, None, None], h.shape).copy()
    ref = O.rhs(prob, 0.2, h, g0, delta_it=2e-5, max_iter=50)
    hd = torch.empty(h.size, dtype=torch.float64, device="cuda")
    it = ctx.rhs(0.2, dev(h).reshape(-1), dev(g0).reshape(-1), hd)
    assert it == ref.iters
    assert rel(host(hd).reshape(h.shape), ref.hdot) < 1e-10


@pytest.mark.parametrize("n,L", [((16, 32, 48), (0.8, 1.0, 1.2)), ((48, 64, 96), (1.0, 1.1, 1.5)),
                                 ((96, 32, 16), (1.5, 0.6, 0.4)), ((128, 16, 32), (1.6, 0.3, 0.6)),
                                 ((64, 48, 32), (1.0, 0.8, 0.6))])
def test_rhs_fp32_fixed_iterations_all_x_lengths(n, L):
    """FP32 x passes of every length (power law, assembly, mask + pad, Eq. 5
    update) against the oracle, fixed iteration count; FP32 round-off only."""
    mask = I.cube(n, L, 0.6 * min(L) * 2)
    ctx, prob = make(n, L, mask, n_power=15.0, prec=S.PREC_F32, max_iter=3)
    h = _state(prob, 23)
    g0 = I.random_field(h.shape, 24, 0.1)
    ref = O.rhs(prob, 0.4, h, g0, delta_it=0.0, max_iter=3)
    hd = torch.empty(h.size, dtype=torch.float64, device="cuda")
    it = ctx.rhs(0.4, dev(h).reshape(-1), dev(g0).reshape(-1), hd)
    assert it == 3
    check3(f"rhs {n}", host(hd).reshape(h.shape), ref.hdot, RHS32)


def test_rhs_fp32_graph_loop_equals_host_loop():
    """The FP32 Eq. 5 loop runs as one CUDA graph (a WHILE conditional node, one
    iteration per trip, condition set on the device).  While profiling, the host drives
    the same kernels one iteration at a time.  Both must give the same dh/dt bit for bit,
    the same iteration count and the oracle's answer; the graph body counts one extra
    kernel (the condition) per iteration, which shows that the graph really ran."""
    n, L = (32, 32, 32), (1.0, 1.0, 1.0)
    mask = I.lens(n, L, 0.6, 0.5, 0.1, 0.1)
    ctx, prob = make(n, L, mask, n_power=30.0, rho_out=100.0, prec=S.PREC_F32, delta_it=2e-5, max_iter=50)
    h = _state(prob, 31)
    g0 = np.broadcast_to(prob.path.hedot(0.2)[:, None, None, None], h.shape).copy()
    ref = O.rhs(prob, 0.2, h, g0, delta_it=2e-5, max_iter=50)
    out = {}
    for mode in ("host", "graph", "graph_again"):
        ctx.profile(mode == "host")
        hd = torch.empty(h.size, dtype=torch.float64, device="cuda")
        l0 = ctx.stats()["launches"]
        it = ctx.rhs(0.2, dev(h).reshape(-1), dev(g0).reshape(-1), hd)
        out[mode] = (it, ctx.stats()["launches"] - l0, host(hd))
        ctx.profile(False)
    it_h, l_h, v_h = out["host"]
    for mode in ("graph", "graph_again"):
        it_g, l_g, v_g = out[mode]
        assert it_g == it_h
        assert l_g - l_h == it_g
        assert np.array_equal(v_g, v_h)
    assert abs(it_h - ref.iters) <= 1
    check3("rhs lens32 early stop", v_h.reshape(h.shape), ref.hdot, RHS32)


def test_rhs_fp32_error_is_stated():
    n, L = (32, 32, 32), (1.0, 1.0, 1.0)
    mask = I.sphere(n, L, 0.6)
    ctx, prob = make(n, L, mask, n_power=25.0, prec=S.PREC_F32, max_iter=3)
    h = _state(prob, 11)
    g0 = I.random_field(h.shape, 12, 0.1)
    ref = O.rhs(prob, 0.4, h, g0, delta_it=0.0, max_iter=3)
    hd = torch.empty(h.size, dtype=torch.float64, device="cuda")
    ctx.rhs(0.4, dev(h).reshape(-1), dev(g0).reshape(-1), hd)
    check3("rhs sphere32", host(hd).reshape(h.shape), ref.hdot, RHS32)


def _cube_cfg():
    cfg = I.config("cube16")
    prob = O.Problem(O.Grid(cfg.n, cfg.L), cfg.mask, O.Material(n=cfg.n_power, rho_out=cfg.rho_out),
                     O.FieldPath(cfg.knots_t, cfg.knots_he))
    return cfg, prob


def test_integrate_fixed_steps_fp64_matches_oracle():
    """Parity tier T2: fixed dt list, Eq. 5 iterated to its fixed point."""
    cfg, prob = _cube_cfg()
    dts = [0.002, 0.003, 0.004, 0.004, 0.005, 0.005]
    ctx = S.Context(cfg.n, cfg.L, n_power=cfg.n_power, rho_out=cfg.rho_out, delta_it=1e-13, max_iter=80)
    ctx.set_geometry(cfg.mask)
    ctx.set_field_path(cfg.knots_t, cfg.knots_he)
    ctx.precompute_kernel()
    N = int(np.prod(cfg.n))
    h = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    t1 = float(np.sum(dts))
    st = ctx.integrate(0.0, t1, dts[0], h, dt_fixed=dts)
    ref = O.integrate(prob, 0.0, t1, np.zeros((3,) + prob.grid.shape), rtol=1e-6, atol=1e-9, dt0=dts[0],
                      delta_it=1e-13, max_iter=80, dt_list=dts)
    assert st["accepted"] == len(dts) == ref.accepted
    assert rel(host(h).reshape(ref.y.shape), ref.y) < 1e-10


def test_integrate_adaptive_fp64_tracks_oracle():
    """Parity tier T3: adaptive BS23 with the paper's iteration tolerance; the
    step sequences may differ, the states agree to a small multiple of rtol."""
    cfg, prob = _cube_cfg()
    rtol, atol = 1e-5, 1e-8
    ctx = S.Context(cfg.n, cfg.L, n_power=cfg.n_power, rho_out=cfg.rho_out, delta_it=2e-5, max_iter=100,
                    rtol=rtol, atol=atol)
    ctx.set_geometry(cfg.mask)
    ctx.set_field_path(cfg.knots_t, cfg.knots_he)
    ctx.precompute_kernel()
    N = int(np.prod(cfg.n))
    h = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    snaps = torch.zeros(2 * 3 * N, dtype=torch.float64, device="cuda")
    st = ctx.integrate(0.0, 0.2, 1e-4, h, tsnap=[0.1, 0.2], snaps=snaps)
    ref = O.integrate(prob, 0.0, 0.2, np.zeros((3,) + prob.grid.shape), rtol=rtol, atol=atol, dt0=1e-4,
                      snapshots=[0.1, 0.2])
    s = host(snaps).reshape((2,) + ref.y.shape)
    for i, (t, y) in enumerate(ref.snaps):
        assert rel(s[i], y) < 20 * rtol, (t, rel(s[i], y))
    assert abs(st["accepted"] - ref.accepted) <= max(3, 0.2 * ref.accepted)


def test_step_matches_integrate_and_counts_launches():
    cfg, prob = _cube_cfg()
    ctx = S.Context(cfg.n, cfg.L, n_power=cfg.n_power, rho_out=cfg.rho_out, delta_it=2e-5, max_iter=100,
                    rtol=1e-5, atol=1e-8)
    ctx.set_geometry(cfg.mask)
    ctx.set_field_path(cfg.knots_t, cfg.knots_he)
    ctx.precompute_kernel()
    N = int(np.prod(cfg.n))
    h = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    warm = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    warm.view(3, N)[2] = 0.5
    t, dt = 0.0, 1e-4
    s0 = ctx.stats()
    while t < 0.05:
        t, dt, _ = ctx.step(t, dt, 0.05, h, warm)
    assert t == 0.05
    s1 = ctx.stats()
    assert s1["launches"] > s0["launches"] and s1["rhs_calls"] > s0["rhs_calls"]
    ref = O.integrate(prob, 0.0, 0.05, np.zeros((3,) + prob.grid.shape), rtol=1e-5, atol=1e-8, dt0=1e-4)
    assert rel(host(h).reshape(ref.y.shape), ref.y) < 2e-4


def test_integrate_fp32_path_tracks_oracle():
    """FP32 FFTs, FP32 stages, compensated FP64 state: fixed steps and an
    adaptive run against the FP64 oracle (stated tolerance 1e-4 relative)."""
    cfg, prob = _cube_cfg()
    N = int(np.prod(cfg.n))
    dts = [0.002, 0.003, 0.004, 0.004, 0.005, 0.005]
    ctx = S.Context(cfg.n, cfg.L, n_power=cfg.n_power, rho_out=cfg.rho_out, delta_it=1e-13, max_iter=80,
                    precision=S.PREC_F32)
    ctx.set_geometry(cfg.mask)
    ctx.set_field_path(cfg.knots_t, cfg.knots_he)
    ctx.precompute_kernel()
    h = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    t1 = float(np.sum(dts))
    st = ctx.integrate(0.0, t1, dts[0], h, dt_fixed=dts)
    ref = O.integrate(prob, 0.0, t1, np.zeros((3,) + prob.grid.shape), rtol=1e-6, atol=1e-9, dt0=dts[0],
                      delta_it=1e-13, max_iter=80, dt_list=dts)
    assert st["accepted"] == len(dts)
    assert rel(host(h).reshape(ref.y.shape), ref.y) < 1e-4
    # adaptive, through scfft_step
    ctx2 = S.Context(cfg.n, cfg.L, n_power=cfg.n_power, rho_out=cfg.rho_out, delta_it=2e-5, max_iter=100,
                     rtol=1e-4, atol=1e-7, precision=S.PREC_F32)
    ctx2.set_geometry(cfg.mask)
    ctx2.set_field_path(cfg.knots_t, cfg.knots_he)
    ctx2.precompute_kernel()
    h2 = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    warm = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    warm.view(3, N)[2] = 0.5
    t, dt = 0.0, 1e-4
    while t < 0.1:
        t, dt, _ = ctx2.step(t, dt, 0.1, h2, warm)
    ref2 = O.integrate(prob, 0.0, 0.1, np.zeros((3,) + prob.grid.shape), rtol=1e-4, atol=1e-7, dt0=1e-4)
    assert rel(host(h2).reshape(ref2.y.shape), ref2.y) < 2e-3


@pytest.mark.parametrize("prec", [S.PREC_F64, S.PREC_F32])
def test_rhs_ej_law_kim_and_anisotropy_matches_oracle(prec):
    """The e(j, h) law of §2 (after Eq. 1) in place of the power law: Kim's jc(|h|) with the
    anisotropic norm |A j|, through the x pass that reads the state h at every node."""
    n, L = (32, 48, 32), (1.0, 1.2, 0.9)
    mask = I.cube(n, L, 0.6 * min(L) * 2)
    ctx, prob = make(n, L, mask, n_power=25.0, prec=prec, max_iter=3)
    ctx.set_ej_law(kim_h0=0.3, aniso=(1.0, 0.7, 1.5))
    prob.mat.kim_h0 = 0.3
    prob.mat.aniso = (1.0, 0.7, 1.5)
    h = _state(prob, 51)
    g0 = I.random_field(h.shape, 52, 0.1)
    ref = O.rhs(prob, 0.4, h, g0, delta_it=0.0, max_iter=3)
    hd = torch.empty(h.size, dtype=torch.float64, device="cuda")
    assert ctx.rhs(0.4, dev(h).reshape(-1), dev(g0).reshape(-1), hd) == 3
    if prec == S.PREC_F64:
        assert rel(host(hd).reshape(h.shape), ref.hdot) < 1e-10
    else:
        check3("rhs e(j,h) law", host(hd).reshape(h.shape), ref.hdot, RHS32)
    # the reverse mode covers Eq. 1 only
    mu = torch.empty_like(hd)
    with pytest.raises(S.ScfftError) as ei:
        ctx.rhs_vjp(dev(h).reshape(-1), hd, mu)
    assert ei.value.code == 8
    # back to Eq. 1: the plain power law again
    ctx.set_ej_law()
    prob.mat.kim_h0, prob.mat.aniso = 0.0, (1.0, 1.0, 1.0)
    ref1 = O.rhs(prob, 0.4, h, g0, delta_it=0.0, max_iter=3)
    ctx.rhs(0.4, dev(h).reshape(-1), dev(g0).reshape(-1), hd)
    assert rel(host(hd).reshape(h.shape), ref1.hdot) < (1e-10 if prec == S.PREC_F64 else 6e-6)


def test_integrate_ej_law_fixed_steps_fp64_matches_oracle():
    """Fixed-step BS23 with the Kim / anisotropic law (Eq. 5 iterated to its fixed point)."""
    cfg, prob = _cube_cfg()
    prob.mat.kim_h0 = 0.2
    prob.mat.aniso = (1.2, 1.0, 0.8)
    dts = [0.002, 0.003, 0.004]
    ctx = S.Context(cfg.n, cfg.L, n_power=cfg.n_power, rho_out=cfg.rho_out, delta_it=1e-13, max_iter=80)
    ctx.set_geometry(cfg.mask)
    ctx.set_field_path(cfg.knots_t, cfg.knots_he)
    ctx.set_ej_law(kim_h0=0.2, aniso=(1.2, 1.0, 0.8))
    ctx.precompute_kernel()
    N = int(np.prod(cfg.n))
    h = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    t1 = float(np.sum(dts))
    ctx.integrate(0.0, t1, dts[0], h, dt_fixed=dts)
    ref = O.integrate(prob, 0.0, t1, np.zeros((3,) + prob.grid.shape), rtol=1e-6, atol=1e-9, dt0=dts[0],
                      delta_it=1e-13, max_iter=80, dt_list=dts)
    assert rel(host(h).reshape(ref.y.shape), ref.y) < 1e-10


# ---------------------------------------------------------------- local-stencil curl option
def _fd_ctx(n, L, mask, prec, **kw):
    ctx, prob = make(n, L, mask, prec=prec, **kw)
    ctx.set_curl(S.CURL_FD)
    prob.curl = "fd"
    return ctx, prob


@pytest.mark.parametrize("n,L", [((16, 32, 48), (0.8, 1.0, 1.2)), ((48, 32, 16), (1.2, 0.9, 0.8))])
@pytest.mark.parametrize("prec", [S.PREC_F64, S.PREC_F32])
def test_rhs_stencil_curl_matches_oracle(n, L, prec):
    """Central-difference curls (the pre-stage's two stencil passes, the masked stencil curl
    of every Eq. 5 iterate) against the oracle's curl_fd, fixed iteration count."""
    mask = I.cube(n, L, 0.6 * min(L) * 2)
    ctx, prob = _fd_ctx(n, L, mask, prec, n_power=20.0, max_iter=3)
    h = _state(prob, 61)
    g0 = I.random_field(h.shape, 62, 0.1)
    ref = O.rhs(prob, 0.4, h, g0, delta_it=0.0, max_iter=3)
    hd = torch.empty(h.size, dtype=torch.float64, device="cuda")
    assert ctx.rhs(0.4, dev(h).reshape(-1), dev(g0).reshape(-1), hd) == 3
    if prec == S.PREC_F64:
        assert rel(host(hd).reshape(h.shape), ref.hdot) < 1e-10
    else:
        check3(f"rhs stencil curl {n}", host(hd).reshape(h.shape), ref.hdot, RHS32)


def test_rhs_stencil_curl_graph_loop_and_early_stop():
    """FP32 with the stencil curl: the Eq. 5 loop as one CUDA graph gives the host-driven
    loop's result bit for bit and stops with the oracle (lens 32^3, jc map, delta_it 2e-5)."""
    n, L = (32, 32, 32), (1.0, 1.0, 1.0)
    mask = I.lens(n, L, 0.6, 0.5, 0.1, 0.1)
    jc = I.jc_noise((32, 32, 32), 5)
    ctx, prob = _fd_ctx(n, L, mask, S.PREC_F32, n_power=30.0, rho_out=100.0, delta_it=2e-5, max_iter=50, jc_map=jc)
    h = _state(prob, 63)
    g0 = np.broadcast_to(prob.path.hedot(0.2)[:, None, None, None], h.shape).copy()
    ref = O.rhs(prob, 0.2, h, g0, delta_it=2e-5, max_iter=50)
    out = {}
    for mode in ("host", "graph"):
        ctx.profile(mode == "host")
        hd = torch.empty(h.size, dtype=torch.float64, device="cuda")
        it = ctx.rhs(0.2, dev(h).reshape(-1), dev(g0).reshape(-1), hd)
        out[mode] = (it, host(hd))
        ctx.profile(False)
    assert out["graph"][0] == out["host"][0]
    assert np.array_equal(out["graph"][1], out["host"][1])
    assert abs(out["host"][0] - ref.iters) <= 1
    check3("rhs stencil curl lens32 early stop", out["host"][1].reshape(h.shape), ref.hdot, RHS32)


def test_integrate_stencil_curl_fixed_steps_matches_oracle():
    """Fixed-step BS23 with the stencil curl, Eq. 5 iterated to its fixed point: FP64 and FP32."""
    cfg, prob = _cube_cfg()
    prob.curl = "fd"
    dts = [0.002, 0.003, 0.004, 0.004]
    t1 = float(np.sum(dts))
    ref = O.integrate(prob, 0.0, t1, np.zeros((3,) + prob.grid.shape), rtol=1e-6, atol=1e-9, dt0=dts[0],
                      delta_it=1e-13, max_iter=80, dt_list=dts)
    N = int(np.prod(cfg.n))
    for prec, tol in ((S.PREC_F64, 1e-10), (S.PREC_F32, 1e-4)):
        ctx = S.Context(cfg.n, cfg.L, n_power=cfg.n_power, rho_out=cfg.rho_out, delta_it=1e-13, max_iter=80,
                        precision=prec)
        ctx.set_geometry(cfg.mask)
        ctx.set_field_path(cfg.knots_t, cfg.knots_he)
        ctx.set_curl(S.CURL_FD)
        ctx.precompute_kernel()
        h = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
        ctx.integrate(0.0, t1, dts[0], h, dt_fixed=dts)
        assert rel(host(h).reshape(ref.y.shape), ref.y) < tol, prec


def _off_centre_mask(g, L):
    X, Y, Z = g.coords()
    return ((np.abs(X - 0.2 * L[0]) < 0.35 * L[0]) & (np.abs(Y + 0.29 * L[1]) < 0.27 * L[1]) &
            (np.abs(Z - 0.41 * L[2]) < 0.23 * L[2]))


@pytest.mark.parametrize("prec", [S.PREC_F64, S.PREC_DF64])
@pytest.mark.parametrize("curl", ["spectral", "fd"])
def test_rhs_fp64_and_df64_off_centre_source_box_matches_oracle(prec, curl):
    """The source box in the shared-memory passes (FP64, double-float), with either curl."""
    n, L = (32, 48, 64), (1.0, 1.2, 1.4)
    g = O.Grid(n, L)
    mask = _off_centre_mask(g, L)
    ctx, prob = make(n, L, mask, n_power=25.0, prec=prec, max_iter=4)
    if curl == "fd":
        ctx.set_curl(S.CURL_FD)
        prob.curl = "fd"
    h = _state(prob, 97)
    g0 = I.random_field(h.shape, 98, 0.1)
    ref = O.rhs(prob, 0.4, h, g0, delta_it=0.0, max_iter=4)
    hd = torch.empty(h.size, dtype=torch.float64, device="cuda")
    assert ctx.rhs(0.4, dev(h).reshape(-1), dev(g0).reshape(-1), hd) == 4
    assert rel(host(hd).reshape(h.shape), ref.hdot) < 1e-10


@pytest.mark.parametrize("n,L", [((32, 48, 64), (1.0, 1.2, 1.4)), ((64, 32, 16), (1.4, 0.9, 0.6))])
def test_rhs_fp32_off_centre_source_box_matches_oracle(n, L):
    """The forward padded passes of an Eq. 5 iteration skip everything outside Omega's
    bounding box (the source chi curl dh^i vanishes there): an off-centre solid whose box
    starts at odd rows and planes, on non-cubic grids, must still give the oracle's dh/dt
    at a fixed iteration count and through the graph-captured loop with its stop."""
    g = O.Grid(n, L)
    mask = _off_centre_mask(g, L)
    zs = np.nonzero(mask.any(axis=(1, 2)))[0]
    ys = np.nonzero(mask.any(axis=(0, 2)))[0]
    assert zs[0] > 2 and ys[0] > 2 and zs[-1] < n[2] - 3 and ys[-1] < n[1] - 3
    ctx, prob = make(n, L, mask, n_power=25.0, prec=S.PREC_F32, max_iter=4)
    h = _state(prob, 95)
    g0 = I.random_field(h.shape, 96, 0.1)
    ref = O.rhs(prob, 0.4, h, g0, delta_it=0.0, max_iter=4)
    hd = torch.empty(h.size, dtype=torch.float64, device="cuda")
    assert ctx.rhs(0.4, dev(h).reshape(-1), dev(g0).reshape(-1), hd) == 4
    check3(f"rhs off-centre box {n}", host(hd).reshape(h.shape), ref.hdot, RHS32)
    # host-driven (profiled) and graph loops: the same bits
    out = {}
    for mode in ("host", "graph"):
        ctx.profile(mode == "host")
        o = torch.empty_like(hd)
        ctx.rhs(0.4, dev(h).reshape(-1), dev(g0).reshape(-1), o)
        out[mode] = host(o)
        ctx.profile(False)
    assert np.array_equal(out["host"], out["graph"])


@pytest.mark.parametrize("n,L", [((16, 16, 32), (0.8, 0.8, 1.2)), ((32, 32, 16), (1.0, 1.0, 0.6)),
                                 ((48, 48, 32), (1.1, 1.1, 0.8)), ((64, 64, 16), (1.2, 1.2, 0.5)),
                                 ((96, 96, 16), (1.4, 1.4, 0.4)), ((128, 128, 16), (1.6, 1.6, 0.3))])
def test_rhs_fp32_fused_box_passes_match_three_passes_and_oracle(n, L):
    """The curl's inverse y pass, the mask/pad x pass and the padded forward y pass of an Eq.
    5 iteration fused into one launch over Omega's box (nx = ny, every x length): with an
    off-centre solid whose box starts at odd rows and planes, the same dh/dt bit for bit as
    the three launches (host-driven and graph loops) and the oracle's at a fixed iteration
    count."""
    g = O.Grid(n, L)
    mask = _off_centre_mask(g, L)
    ctx, prob = make(n, L, mask, n_power=25.0, prec=S.PREC_F32, max_iter=4)
    h = _state(prob, 99)
    g0 = I.random_field(h.shape, 100, 0.1)
    ref = O.rhs(prob, 0.4, h, g0, delta_it=0.0, max_iter=4)
    out = {}
    for bf in (0, 1):
        ctx.set_schedule(box_fused=bf)
        for mode in ("host", "graph"):
            ctx.profile(mode == "host")
            o = torch.empty(h.size, dtype=torch.float64, device="cuda")
            assert ctx.rhs(0.4, dev(h).reshape(-1), dev(g0).reshape(-1), o) == 4
            out[bf, mode] = host(o)
            if mode == "host":
                prof = ctx.profile_read()
                # the fused launch runs in place of the three (4 iterations per rhs)
                assert prof["box_fused"][0] == (4 if bf else 0), prof
                assert prof["x_maskpad"][0] == (0 if bf else 4), prof
            ctx.profile(False)
    assert all(np.array_equal(out[0, "host"], v) for v in out.values())
    check3(f"rhs fused box passes {n}", out[1, "graph"].reshape(h.shape), ref.hdot, RHS32)


# FP32 bound of the single-node case: the state is the field of a point current, whose curl at
# the node is far rougher than the smooth states above, and Eq. 1 amplifies its FP32 round-off
# by n - 1 = 24; observed 2.5e-5, 4.8e-6, 2.7e-5 per component at 32^3 (about 3x that here)
RHS32_POINT = (8e-5, 8e-5, 8e-5)


@pytest.mark.parametrize("n,L", [((32, 32, 32), (1.0, 1.0, 1.0)), ((48, 32, 16), (1.2, 0.9, 0.8))])
@pytest.mark.parametrize("prec", [S.PREC_F64, S.PREC_F32])
def test_rhs_single_node_omega_matches_oracle(n, L, prec):
    """The degenerate superconductor: Omega is one node at an odd row and plane, so the source
    box of the Eq. 5 convolution is one plane and one row pair.  The box passes (FP64; FP32 with
    three launches and, where nx = ny, the fused one, the same bits) against the oracle at a
    fixed iteration count."""
    mask = np.zeros((n[2], n[1], n[0]), dtype=bool)
    mask[n[2] // 2 + 1, n[1] // 2 + 1, n[0] // 2] = True
    ctx, prob = make(n, L, mask, n_power=25.0, prec=prec, max_iter=3)
    h = _state(prob, 101) + np.array([0.02, -0.01, 0.05])[:, None, None, None]
    g0 = I.random_field(h.shape, 102, 0.1)
    ref = O.rhs(prob, 0.4, h, g0, delta_it=0.0, max_iter=3)
    outs = []
    for bf in ((0, 1) if prec == S.PREC_F32 else (None,)):
        if bf is not None:
            ctx.set_schedule(box_fused=bf)
        o = torch.empty(h.size, dtype=torch.float64, device="cuda")
        assert ctx.rhs(0.4, dev(h).reshape(-1), dev(g0).reshape(-1), o) == 3
        outs.append(host(o))
    assert all(np.array_equal(outs[0], x) for x in outs[1:])
    if prec == S.PREC_F64:
        assert rel(outs[0].reshape(h.shape), ref.hdot) < 1e-10
    else:
        check3(f"rhs single-node Omega {n}", outs[0].reshape(h.shape), ref.hdot, RHS32_POINT)
