"""Physics checks of the GPU path (closed forms of the critical state).

A long superconducting cylinder (radius R, length d = 8R, n = 100, close to
the Bean limit) in a slowly ramped axial field screens its mid-plane centre
until the applied field reaches the full-penetration field, which for
j = jc phi_hat in the whole cylinder is
    H_p = jc (d/2) asinh(2R/d) = 0.990 jc R,
and at full penetration its moment is |m_z| = (pi/3) jc R^3 d.  Both follow
from integrating the loop field of an azimuthal current of density jc over
the cylinder.  Finite n, the Gaussian smoothing of the derivatives and the
voxelisation make the match approximate; the tolerances are stated below."""

import math

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


def test_bean_cylinder_penetration_field_and_moment():
    R, d = 0.5, 4.0
    n, L = (32, 32, 96), (0.8, 0.8, 2.4)
    mask = I.cylinder(n, L, R, d)
    he_max = 0.75
    ctx = S.Context(n, L, n_power=100.0, rho_out=20.0, precision=S.PREC_F32, delta_it=2e-5, max_iter=100,
                    rtol=1e-3, atol=1e-5)
    ctx.set_geometry(mask)
    ctx.set_field_path([0.0, he_max], [[0, 0, 0], [0, 0, he_max]])
    ctx.precompute_kernel()
    N = int(np.prod(n))
    h = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    ts = [0.05 * (i + 1) for i in range(15)]
    snaps = torch.zeros(len(ts) * 3 * N, dtype=torch.float64, device="cuda")
    ctx.integrate(0.0, he_max, 1e-5, h, tsnap=ts, snaps=snaps)
    s = snaps.cpu().numpy().reshape(len(ts), 3, n[2], n[1], n[0])
    cz, cy, cx = n[2] // 2, n[1] // 2, n[0] // 2
    centre = s[:, 2, cz - 1:cz + 1, cy - 1:cy + 1, cx - 1:cx + 1].mean(axis=(1, 2, 3))
    Hp = (d / 2) * math.asinh(2 * R / d)  # 0.495 for R = 0.5, d = 4
    # screened well below H_p, penetrated above it
    for t, hc in zip(ts, centre):
        if t <= 0.6 * Hp:
            assert hc < 0.05 * t, (t, hc)
    first = next(t for t, hc in zip(ts, centre) if hc > 0.05 * t)
    assert 0.75 * Hp <= first <= 1.25 * Hp, (first, Hp)
    # saturated moment at the end: m = 1/2 sum r x j dV with j = curl h
    j = torch.empty_like(h)
    ctx.curl(h, j)
    jn = j.cpu().numpy().reshape(3, n[2], n[1], n[0])
    x, y, z = I.node_axes(n, L)
    X, Y = x[None, None, :], y[None, :, None]
    dV = np.prod([2 * Lh / k for Lh, k in zip(L, n)])
    mz = 0.5 * dV * np.sum(X * jn[1] - Y * jn[0])
    m_sat = math.pi / 3 * R ** 3 * d
    assert -mz == pytest.approx(m_sat, rel=0.15), (mz, m_sat)
