"""FP64 NumPy oracle of the method-of-lines right-hand side dh/dt and its
time integrator (Prigozhin & Sokolovsky, §2, Eqs. 1-8).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg; never by the product path. Every step is written
in the paper's order and notation, with library FFTs as the only primitive; no
blocking, fusion or reordering.

Array layout: vector fields are numpy arrays of shape (3, nz, ny, nx), the
component index first (x, y, z), then z, y, x (x varies fastest).  Scalar node
fields (the mask of the superconductor Omega, a jc map) have shape (nz, ny, nx).

Readings of points where the paper is silent (each one named where it is used):
  R-grid   nodes are cell centres x_i = -L + (i + 1/2) dx, dx = 2L/N (§2: "uniform
           N_x x N_y x N_z grid" on D = {|x|<=L_x, ...}).
  R-smooth the Gaussian smoothing multiplies a derivative's symbol by
           exp(-sigma^2 |k|^2 / 2), sigma = half the cell diagonal (§2).
  R-nyq    the derivative symbol i k_a is 0 on the Nyquist plane of axis a, so
           that a real field has a real curl.
  R-phi    Phi of Eq. 6 is the free-space convolution with the gradient of the
           smoothed Green function G_sigma = G * Gaussian(sigma) (Fourier
           transform exp(-sigma^2 k^2/2)/k^2, cf. Eq. 7 and the smoothing of §2),
           sampled on the grid: Phi_d[j](r_a) = dV sum_b grad G_sigma(r_a - r_b) x j_b.
           It is evaluated either by this direct sum or by zero padding to
           2N_x x 2N_y x 2N_z and a cyclic FFT convolution (Hockney).  The
           sampled kernel is made exactly odd (the offset -N_a plane is zeroed,
           it never meets a cropped output) so its transform vanishes at k = 0,
           the paper's rule for k = 0 under Eq. 7.
  R-warm   the initial approximation of dh_out/dt (Eq. 5) is the warm-start
           array g passed in by the caller (the previous result, §2); the
           first call uses g = dh_e/dt.
  R-stop   the residual of Eq. 5 is the mean over the Omega_out nodes of the
           Euclidean norm |dh^{i+1} - dh^i|; iterate while it is not below
           delta_it * max(|dh_e/dt|, 1), at most max_iter times.
  R-ode    "ode23" is read as the Bogacki-Shampine 3(2) FSAL pair with the
           error norm max_i |err_i| / max(rtol |y_i|, rtol |y_new,i|, atol),
           accept if <= 1, dt <- dt * min(5, max(0.2, 0.9 err^(-1/3))).
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field
from typing import Callable, Optional, Sequence

import numpy as np
from scipy.special import erf

__all__ = [
    "Grid", "Material", "FieldPath", "Problem",
    "wavenumbers", "curl_s", "div_s", "curl_fd", "div_fd", "electric_field",
    "grad_green_sigma", "phi_direct", "phi_hockney", "hockney_kernel_spectrum",
    "rhs", "RhsResult",
    "BS23_C", "BS23_A", "BS23_B", "BS23_BHAT", "BS23_E",
    "bs23_step", "error_norm", "integrate", "IntegrateResult",
    "magnetic_moment", "dissipation", "rhs_vjp", "RhsVJP", "integrate_adjoint", "StepAdjoint",
]


# ----------------------------------------------------------------------------
# Grid (§2: uniform grid on D = {|x|<=Lx, |y|<=Ly, |z|<=Lz}; reading R-grid)
# ----------------------------------------------------------------------------
@dataclass(frozen=True)
class Grid:
    n: tuple  # (nx, ny, nz)
    L: tuple  # half extents (Lx, Ly, Lz)
    sigma_scale: float = 1.0  # multiplies the paper's sigma (half the cell diagonal)

    @property
    def shape(self):
        nx, ny, nz = self.n
        return (nz, ny, nx)

    @property
    def d(self):
        return tuple(2.0 * L / n for L, n in zip(self.L, self.n))

    @property
    def dV(self):
        dx, dy, dz = self.d
        return dx * dy * dz

    @property
    def sigma(self):
        # §2: "the smoothing parameter sigma was equal to a half of the grid cell diagonal"
        dx, dy, dz = self.d
        return self.sigma_scale * 0.5 * math.sqrt(dx * dx + dy * dy + dz * dz)

    def axes(self):
        """Node coordinates along x, y, z (cell centres, reading R-grid)."""
        return tuple(-L + (np.arange(n) + 0.5) * (2.0 * L / n) for L, n in zip(self.L, self.n))

    def coords(self):
        """Broadcastable (z, y, x) coordinate arrays: X[None,None,:], Y[None,:,None], Z[:,None,None]."""
        x, y, z = self.axes()
        return x[None, None, :], y[None, :, None], z[:, None, None]


def wavenumbers(n: int, L: float):
    """Angular wavenumbers of the periodic grid of n nodes on [-L, L) (period 2L),
    in numpy FFT order, and the derivative symbol i*k with the Nyquist entry set
    to zero (reading R-nyq)."""
    m = np.fft.fftfreq(n, d=1.0 / n)  # integers 0..n/2-1, -n/2..-1
    k = np.pi * m / L
    D = 1j * k
    if n % 2 == 0:
        D[n // 2] = 0.0
    return k, D


def _symbols(grid: Grid):
    nx, ny, nz = grid.n
    Lx, Ly, Lz = grid.L
    kx, Dx = wavenumbers(nx, Lx)
    ky, Dy = wavenumbers(ny, Ly)
    kz, Dz = wavenumbers(nz, Lz)
    k2 = kx[None, None, :] ** 2 + ky[None, :, None] ** 2 + kz[:, None, None] ** 2
    S = np.exp(-0.5 * grid.sigma ** 2 * k2)  # reading R-smooth
    return Dx[None, None, :], Dy[None, :, None], Dz[:, None, None], S


def curl_s(f: np.ndarray, grid: Grid) -> np.ndarray:
    """Smoothed spectral curl on the periodic unpadded grid (§2: derivatives of
    Eqs. 3-4 taken in Fourier space with Gaussian smoothing)."""
    Dx, Dy, Dz, S = _symbols(grid)
    F = np.fft.fftn(f, axes=(1, 2, 3))
    Fx, Fy, Fz = F[0], F[1], F[2]
    G = np.stack([
        (Dy * Fz - Dz * Fy) * S,
        (Dz * Fx - Dx * Fz) * S,
        (Dx * Fy - Dy * Fx) * S,
    ])
    return np.real(np.fft.ifftn(G, axes=(1, 2, 3)))


def div_s(f: np.ndarray, grid: Grid) -> np.ndarray:
    """Smoothed spectral divergence with the same symbols as curl_s (used by the
    div j = 0 check of §2)."""
    Dx, Dy, Dz, S = _symbols(grid)
    F = np.fft.fftn(f, axes=(1, 2, 3))
    return np.real(np.fft.ifftn((Dx * F[0] + Dy * F[1] + Dz * F[2]) * S))


def _dfd(f: np.ndarray, axis: int, d: float) -> np.ndarray:
    """Second-order central difference (f[i+1] - f[i-1]) / (2 d) along an array axis of the
    periodic grid."""
    return (np.roll(f, -1, axis=axis) - np.roll(f, 1, axis=axis)) / (2.0 * d)


def curl_fd(f: np.ndarray, grid: Grid) -> np.ndarray:
    """Local-stencil curl (reading R-fd, an alternative to the smoothed spectral derivatives of
    §2): second-order central differences on the periodic grid, no smoothing.  f has shape
    (3, nz, ny, nx): array axis 2 is y, 1 is z, 3 is x."""
    dx, dy, dz = grid.d
    fx, fy, fz = f[0], f[1], f[2]
    return np.stack([
        _dfd(fz, 1, dy) - _dfd(fy, 0, dz),
        _dfd(fx, 0, dz) - _dfd(fz, 2, dx),
        _dfd(fy, 2, dx) - _dfd(fx, 1, dy),
    ])


def div_fd(f: np.ndarray, grid: Grid) -> np.ndarray:
    """Divergence with the same central differences as curl_fd."""
    dx, dy, dz = grid.d
    return _dfd(f[0], 2, dx) + _dfd(f[1], 1, dy) + _dfd(f[2], 0, dz)


# ----------------------------------------------------------------------------
# Material law (Eq. 1) and the fictitious outer resistivity (§2, after Eq. 4)
# ----------------------------------------------------------------------------
@dataclass
class Material:
    n: float = 20.0       # power-law exponent
    e0: float = 1.0       # dimensionless units of Eq. 8: e0 = jc = mu0 = 1
    jc: object = 1.0      # scalar or (nz, ny, nx) map
    rho_out: float = 20.0  # fictitious resistivity in Omega_out
    mu0: float = 1.0
    # e(j, h) variants (§2 after Eq. 1: "e(j) or e(j, h), where h is the local magnetic field"):
    kim_h0: float = 0.0            # Kim-type jc(|h|) = jc / (1 + |h| / kim_h0); 0: jc independent of h
    aniso: tuple = (1.0, 1.0, 1.0)  # a_x, a_y, a_z of the anisotropic norm |j|_A = |(a_x j_x, a_y j_y, a_z j_z)|


def electric_field(j: np.ndarray, mask: np.ndarray, mat: Material, h: Optional[np.ndarray] = None) -> np.ndarray:
    """e = rho(|j|) j in Omega with rho = (e0/jc)|j/jc|^(n-1) (Eq. 1), e = rho_out j in
    Omega_out (the poor-conductor Ohm law of §2).

    The e(j, h) variants that §2 allows in place of Eq. 1 (readings R-kim, R-aniso):
    jc may depend on the local field, jc(h) = jc / (1 + |h| / kim_h0) (Kim's form), and
    the power law may be anisotropic: e = (e0/jc)(|j|_A/jc)^(n-1) A^2 j with
    A = diag(a_x, a_y, a_z) and |j|_A = |A j|, the gradient in j of the convex potential
    (e0 jc / (n + 1)) (|j|_A / jc)^(n + 1), so the critical current along axis a is jc / a_a.
    With kim_h0 = 0 and A = I this is Eq. 1."""
    jc = np.asarray(mat.jc, dtype=np.float64)
    if mat.kim_h0 > 0:
        if h is None:
            raise ValueError("a field-dependent jc needs the field h")
        jc = jc / (1.0 + np.sqrt(np.sum(h * h, axis=0)) / mat.kim_h0)
    A = np.asarray(mat.aniso, dtype=np.float64)[:, None, None, None]
    jA = np.sqrt(np.sum((A * j) ** 2, axis=0))
    rho = (mat.e0 / jc) * (jA / jc) ** (mat.n - 1.0)
    return np.where(mask[None], rho[None] * (A * A) * j, mat.rho_out * j)


def dissipation(j: np.ndarray, e: np.ndarray, mask: np.ndarray, dV: float) -> float:
    """Integral of e.j over Omega (nonnegative for Eq. 1)."""
    return float(np.sum(np.sum(e * j, axis=0)[mask]) * dV)


# ----------------------------------------------------------------------------
# Biot-Savart operator Phi (Eqs. 2, 6, 7; reading R-phi)
# ----------------------------------------------------------------------------
def grad_green_sigma(rx, ry, rz, sigma: float):
    """Gradient of G_sigma(r) = erf(r / (sqrt(2) sigma)) / (4 pi r), the Green
    function G = 1/(4 pi r) of Eq. 2 convolved with a Gaussian of std sigma.
    d G_sigma / dr = [ (2/sqrt(pi)) u exp(-u^2) - erf(u) ] / (4 pi r^2), u = r/(sqrt(2) sigma).
    The gradient is 0 at r = 0 (odd symmetry)."""
    rx, ry, rz = np.broadcast_arrays(np.asarray(rx, float), np.asarray(ry, float), np.asarray(rz, float))
    shape = rx.shape
    rx, ry, rz = (np.atleast_1d(a).copy() for a in (rx, ry, rz))
    r = np.sqrt(rx * rx + ry * ry + rz * rz)
    out = np.zeros((3,) + r.shape)
    nz = r > 0
    rr = r[nz]
    u = rr / (math.sqrt(2.0) * sigma)
    g = ((2.0 / math.sqrt(math.pi)) * u * np.exp(-u * u) - erf(u)) / (4.0 * math.pi * rr * rr)
    out[0][nz] = g * rx[nz] / rr
    out[1][nz] = g * ry[nz] / rr
    out[2][nz] = g * rz[nz] / rr
    return out.reshape((3,) + shape)


def _cross(a, b):
    return np.stack([
        a[1] * b[2] - a[2] * b[1],
        a[2] * b[0] - a[0] * b[2],
        a[0] * b[1] - a[1] * b[0],
    ])


def phi_direct(j: np.ndarray, grid: Grid) -> np.ndarray:
    """Phi_d[j](r_a) = dV sum_b grad G_sigma(r_a - r_b) x j_b: Eq. 6 as a plain
    O(N^2) sum over grid nodes (tiny grids only)."""
    x, y, z = grid.axes()
    nz_, ny_, nx_ = grid.shape
    Zg, Yg, Xg = np.meshgrid(z, y, x, indexing="ij")
    pts = np.stack([Xg.ravel(), Yg.ravel(), Zg.ravel()], axis=1)  # (N, 3)
    jv = j.reshape(3, -1).T  # (N, 3)
    out = np.zeros_like(jv)
    for a in range(pts.shape[0]):
        d = pts[a] - pts  # r_a - r_b
        K = grad_green_sigma(d[:, 0], d[:, 1], d[:, 2], grid.sigma)  # (3, N)
        out[a] = grid.dV * np.sum(_cross(K, jv.T), axis=1)
    return out.T.reshape(3, nz_, ny_, nx_)


def hockney_kernel_spectrum(grid: Grid) -> np.ndarray:
    """Complex spectrum (3, 2nz, 2ny, 2nx) of dV * grad G_sigma sampled at the
    offsets m_a * d_a, m_a in [-n_a, n_a) (cyclic order), with every m_a = -n_a
    plane set to zero so that the sampled kernel is exactly odd."""
    nx, ny, nz = grid.n
    dx, dy, dz = grid.d
    mx = np.fft.fftfreq(2 * nx, d=1.0 / (2 * nx))
    my = np.fft.fftfreq(2 * ny, d=1.0 / (2 * ny))
    mz = np.fft.fftfreq(2 * nz, d=1.0 / (2 * nz))
    K = grid.dV * grad_green_sigma(mx[None, None, :] * dx, my[None, :, None] * dy,
                                   mz[:, None, None] * dz, grid.sigma)
    K[:, :, :, nx] = 0.0
    K[:, :, ny, :] = 0.0
    K[:, nz, :, :] = 0.0
    return np.fft.fftn(K, axes=(1, 2, 3))


def phi_hockney(j: np.ndarray, grid: Grid, Khat: Optional[np.ndarray] = None) -> np.ndarray:
    """Phi_d[j] by zero padding to twice the grid along every axis, an FFT, the
    cross product K^ x J^ (Eq. 7 with the sampled-kernel spectrum) and an inverse
    FFT cropped to the original block."""
    nx, ny, nz = grid.n
    if Khat is None:
        Khat = hockney_kernel_spectrum(grid)
    jp = np.zeros((3, 2 * nz, 2 * ny, 2 * nx))
    jp[:, :nz, :ny, :nx] = j
    J = np.fft.fftn(jp, axes=(1, 2, 3))
    P = np.real(np.fft.ifftn(_cross(Khat, J), axes=(1, 2, 3)))
    return P[:, :nz, :ny, :nx].copy()


# ----------------------------------------------------------------------------
# Applied field path h_e(t) (§3: piecewise-linear ramps; plus a sinusoid)
# ----------------------------------------------------------------------------
@dataclass
class FieldPath:
    """h_e(t) = piecewise-linear interpolation of knots (t_k, he_k), constant
    outside [t_0, t_K], plus sin_amp * sin(2 pi (t - sin_t0)/sin_period) * sin_dir
    for sin_t0 <= t < sin_t1."""
    t: Sequence[float]
    he: Sequence[Sequence[float]]
    sin_amp: float = 0.0
    sin_period: float = 1.0
    sin_t0: float = 0.0
    sin_t1: float = 0.0
    sin_dir: Sequence[float] = (0.0, 0.0, 1.0)

    def _seg(self, t, left):
        tk = np.asarray(self.t, float)
        K = len(tk)
        for s in range(K - 1):
            lo, hi = tk[s], tk[s + 1]
            if (lo <= t < hi) if not left else (lo < t <= hi):
                return s
        return -1

    def he_at(self, t: float) -> np.ndarray:
        tk = np.asarray(self.t, float)
        hk = np.asarray(self.he, float).reshape(-1, 3)
        if t <= tk[0]:
            v = hk[0].copy()
        elif t >= tk[-1]:
            v = hk[-1].copy()
        else:
            s = int(np.searchsorted(tk, t, side="right") - 1)
            w = (t - tk[s]) / (tk[s + 1] - tk[s])
            v = (1 - w) * hk[s] + w * hk[s + 1]
        if self.sin_amp != 0.0 and self.sin_t0 <= t < self.sin_t1:
            v = v + self.sin_amp * math.sin(2 * math.pi * (t - self.sin_t0) / self.sin_period) * np.asarray(self.sin_dir, float)
        return v

    def hedot(self, t: float, left: bool = False) -> np.ndarray:
        """dh_e/dt at t; at a kink the right derivative, or the left one if left=True."""
        tk = np.asarray(self.t, float)
        hk = np.asarray(self.he, float).reshape(-1, 3)
        s = self._seg(t, left)
        v = np.zeros(3) if s < 0 else (hk[s + 1] - hk[s]) / (tk[s + 1] - tk[s])
        if self.sin_amp != 0.0:
            inside = (self.sin_t0 < t <= self.sin_t1) if left else (self.sin_t0 <= t < self.sin_t1)
            if inside:
                w = 2 * math.pi / self.sin_period
                v = v + self.sin_amp * w * math.cos(w * (t - self.sin_t0)) * np.asarray(self.sin_dir, float)
        return v

    def hedot_jacobian(self, t: float, left: bool = False) -> np.ndarray:
        """d(dh_e/dt)(t) / d(path parameters), shape (3, 3K + 1): the parameters are the
        knot amplitudes he[k][a] (knot-major, 3 per knot) and sin_amp.  On the linear
        piece (t_s, t_{s+1}) that holds t (on the side `left` picks at a kink) the rate
        (he_{s+1} - he_s) / (t_{s+1} - t_s) gives +-1/(t_{s+1} - t_s); inside the sine
        window the rate sin_amp w cos(w (t - sin_t0)) sin_dir gives w cos(.) sin_dir."""
        K = len(self.t)
        J = np.zeros((3, 3 * K + 1))
        s = self._seg(t, left)
        if s >= 0:
            w = 1.0 / (float(self.t[s + 1]) - float(self.t[s]))
            for a in range(3):
                J[a, 3 * (s + 1) + a] += w
                J[a, 3 * s + a] -= w
        inside = (self.sin_t0 < t <= self.sin_t1) if left else (self.sin_t0 <= t < self.sin_t1)
        if inside and self.sin_period > 0:
            w = 2 * math.pi / self.sin_period
            J[:, 3 * K] = w * math.cos(w * (t - self.sin_t0)) * np.asarray(self.sin_dir, float)
        return J

    def kinks(self):
        ks = list(np.asarray(self.t, float))
        if self.sin_amp != 0.0:
            ks += [self.sin_t0, self.sin_t1]
        return sorted(set(ks))


@dataclass
class Problem:
    grid: Grid
    mask: np.ndarray          # bool (nz, ny, nx): True in Omega
    mat: Material
    path: FieldPath
    Khat: Optional[np.ndarray] = None
    curl: str = "spectral"    # "spectral" (§2: smoothed spectral derivatives) or "fd" (reading R-fd)

    def kernel(self):
        if self.Khat is None:
            self.Khat = hockney_kernel_spectrum(self.grid)
        return self.Khat

    def curl_op(self) -> Callable:
        """The discrete curl of Eqs. 3-5 for this problem."""
        if self.curl == "fd":
            return lambda f: curl_fd(f, self.grid)
        return lambda f: curl_s(f, self.grid)


# ----------------------------------------------------------------------------
# Right-hand side dh/dt (§2: Eqs. 1, 3, 4, 5 and the iteration that follows)
# ----------------------------------------------------------------------------
@dataclass
class RhsResult:
    hdot: np.ndarray
    iters: int
    converged: bool
    residual: float
    residuals: list = field(default_factory=list)


def rhs(prob: Problem, t: float, h: np.ndarray, g: np.ndarray, delta_it: float = 2e-5,
        max_iter: int = 100, left: bool = False, phi: Optional[Callable] = None) -> RhsResult:
    """dh/dt at time t for the field h, warm start g (reading R-warm).

    1. j = curl h                                  (Eq. 4)
    2. e = rho(|j|) j in Omega, rho_out j outside  (Eq. 1 and §2)
    3. dh_in = -curl e / mu0 restricted to Omega   (Eq. 3)
    4. dh^0 = dh_in in Omega, g in Omega_out
    5. dh^{i+1} = dh^i in Omega, dh_e/dt + Phi[chi_Omega curl dh^i] in Omega_out (Eq. 5)
       until the residual test of reading R-stop passes or max_iter iterations.
    """
    grid, mask, mat = prob.grid, prob.mask, prob.mat
    if phi is None:
        Khat = prob.kernel()
        phi = lambda jj: phi_hockney(jj, grid, Khat)  # noqa: E731
    C = prob.curl_op()
    j = C(h)
    e = electric_field(j, mask, mat, h)
    hdot_in = -C(e) / mat.mu0
    hd = np.where(mask[None], hdot_in, g)
    hed = prob.path.hedot(t, left=left)
    tol = delta_it * max(float(np.linalg.norm(hed)), 1.0)
    out = ~mask
    nout = int(out.sum())
    iters, conv, r = 0, False, float("nan")
    res = []
    if nout == 0:  # Omega fills the box: Eq. 5 has nothing to iterate on
        return RhsResult(hd, 0, True, 0.0, res)
    for i in range(max_iter):
        jdot_in = C(hd) * mask[None]
        P = phi(jdot_in)
        new = np.where(mask[None], hd, hed[:, None, None, None] + P)
        r = float(np.sum(np.sqrt(np.sum((new - hd) ** 2, axis=0))[out]) / nout)
        res.append(r)
        hd = new
        iters = i + 1
        if r < tol:
            conv = True
            break
    return RhsResult(hd, iters, conv, r, res)


# ----------------------------------------------------------------------------
# Bogacki-Shampine 3(2) FSAL pair (the method behind Matlab ode23; reading R-ode)
# Coefficients from Bogacki & Shampine, Appl. Math. Lett. 2 (1989) 321-325.
# ----------------------------------------------------------------------------
BS23_C = (0.0, 0.5, 0.75, 1.0)
BS23_A = ((), (0.5,), (0.0, 0.75), (2.0 / 9.0, 1.0 / 3.0, 4.0 / 9.0))
BS23_B = (2.0 / 9.0, 1.0 / 3.0, 4.0 / 9.0, 0.0)          # third-order solution
BS23_BHAT = (7.0 / 24.0, 0.25, 1.0 / 3.0, 0.125)         # embedded second order
BS23_E = tuple(b - bh for b, bh in zip(BS23_B, BS23_BHAT))  # y3 - y2 weights


def bs23_step(f: Callable, t: float, y: np.ndarray, dt: float, k1: np.ndarray, end_left: bool = False,
              t_end: Optional[float] = None):
    """One BS23 step from (t, y) with first stage k1 = f(t, y).  Returns
    (y_new, k4, err_vec) with k4 = f(t_end, y_new) (the FSAL stage; t_end
    defaults to t+dt, a step clipped to a stop passes the stop itself) and
    err_vec = dt * sum_i (b_i - bhat_i) k_i."""
    k2 = f(t + BS23_C[1] * dt, y + dt * (BS23_A[1][0] * k1), False)
    k3 = f(t + BS23_C[2] * dt, y + dt * (BS23_A[2][0] * k1 + BS23_A[2][1] * k2), False)
    ynew = y + dt * (BS23_B[0] * k1 + BS23_B[1] * k2 + BS23_B[2] * k3)
    k4 = f(t + dt if t_end is None else t_end, ynew, end_left)
    err = dt * (BS23_E[0] * k1 + BS23_E[1] * k2 + BS23_E[2] * k3 + BS23_E[3] * k4)
    return ynew, k4, err


def error_norm(err: np.ndarray, y: np.ndarray, ynew: np.ndarray, rtol: float, atol: float) -> float:
    """max_i |err_i| / max(rtol |y_i|, rtol |ynew_i|, atol) (reading R-ode)."""
    w = np.maximum(np.maximum(rtol * np.abs(y), rtol * np.abs(ynew)), atol)
    return float(np.max(np.abs(err) / w))


@dataclass
class IntegrateResult:
    t: float
    y: np.ndarray
    snaps: list
    accepted: int
    rejected: int
    rhs_calls: int
    iters: list
    dts: list
    ts: list = field(default_factory=list)  # end time of every accepted step


def integrate(prob: Problem, t0: float, t1: float, y0: np.ndarray, rtol: float, atol: float,
              dt0: float, snapshots: Sequence[float] = (), delta_it: float = 2e-5,
              max_iter: int = 100, dt_list: Optional[Sequence[float]] = None,
              max_steps: int = 100000) -> IntegrateResult:
    """Method of lines (§2): integrate dh/dt = rhs from t0 to t1 by BS23.

    Steps are clipped to end exactly on the field-path kinks, the snapshot
    times and t1; a step that ends on a kink evaluates its last stage with the
    left derivative of h_e and the next step restarts its first stage with the
    right one.  With dt_list given, the steps are those dts (fixed-step mode,
    no error control).  The warm start g is the result of the most recent rhs
    call (reading R-warm)."""
    state = {"g": None, "calls": 0, "iters": []}

    def f(t, y, left):
        if state["g"] is None:
            state["g"] = np.broadcast_to(prob.path.hedot(t, left)[:, None, None, None], y.shape).copy()
        r = rhs(prob, t, y, state["g"], delta_it=delta_it, max_iter=max_iter, left=left)
        state["g"] = r.hdot
        state["calls"] += 1
        state["iters"].append(r.iters)
        return r.hdot

    stops = sorted(set([s for s in list(prob.path.kinks()) + list(snapshots) + [t1] if t0 < s <= t1]))
    kinks = set(prob.path.kinks())
    t, y = t0, y0.copy()
    k1 = f(t, y, False)
    dt = dt0
    snaps = []
    acc = rej = 0
    dts = []
    tends = []
    si = 0
    step = 0
    while t < t1 and step < max_steps:
        step += 1
        while si < len(stops) and stops[si] <= t:
            si += 1
        nxt = stops[si] if si < len(stops) else t1
        if dt_list is not None:
            dt = dt_list[acc]
        h_step = min(dt, nxt - t)
        hits = (h_step == nxt - t)
        end_left = hits and (nxt in kinks)
        ynew, k4, err = bs23_step(f, t, y, h_step, k1, end_left, t_end=nxt if hits else None)
        if dt_list is not None:
            en = 0.0
        else:
            en = error_norm(err, y, ynew, rtol, atol)
        if en <= 1.0:
            t = nxt if hits else t + h_step
            y = ynew
            acc += 1
            dts.append(h_step)
            tends.append(t)
            if end_left:
                k1 = f(t, y, False)
            else:
                k1 = k4
            if hits and nxt in snapshots:
                snaps.append((t, y.copy()))
            if dt_list is None:
                fac = 5.0 if en == 0 else min(5.0, max(0.2, 0.9 * en ** (-1.0 / 3.0)))
                dt = h_step * fac
        else:
            rej += 1
            dt = h_step * max(0.2, 0.9 * en ** (-1.0 / 3.0))
    return IntegrateResult(t, y, snaps, acc, rej, state["calls"], state["iters"], dts, tends)


# ----------------------------------------------------------------------------
# Diagnostics
# ----------------------------------------------------------------------------
def magnetic_moment(j: np.ndarray, grid: Grid) -> np.ndarray:
    """m = 1/2 sum r x j dV over the grid."""
    X, Y, Z = grid.coords()
    r = np.stack(np.broadcast_arrays(X, Y, Z))
    return 0.5 * grid.dV * np.sum(_cross(r, j), axis=(1, 2, 3))


# ----------------------------------------------------------------------------
# Adjoint of one right-hand side with a fixed number K of Eq. 5 iterations
# ----------------------------------------------------------------------------
@dataclass
class RhsVJP:
    mu_h: np.ndarray   # (dF/dh)^T lam
    mu_g: np.ndarray   # (dF/dg)^T lam
    mu_jc: np.ndarray  # (dF/djc)^T lam, one value per node (zero outside Omega)
    mu_a: np.ndarray   # (dF/da)^T lam for the applied rate a = dh_e/dt (3 values)


def rhs_vjp(prob: Problem, t: float, h: np.ndarray, lam: np.ndarray, K: int, left: bool = False) -> RhsVJP:
    """Reverse-mode derivative of F(h, g, jc, a) = dh^K of `rhs` (delta_it = 0,
    max_iter = K): the forward map is, in the order of §2,
        j = C h,  e = E(j; jc),  u = -C e / mu0,  d^0 = chi u + chib g,
        d^{i+1} = M d^i + chib a,  M = chi + chib Phi chi C   (Eq. 5)
    with chi the indicator of Omega and chib = 1 - chi.  The curl C (imaginary
    odd symbol, skew cross product) and Phi (odd kernel, skew cross product, the
    same offsets both ways after cropping) are symmetric, so
        M^T = chi + C chi Phi chib,
    and the transposed steps run in reverse order.  The power law's Jacobian is
    rho (I + (n-1) jhat jhat^T) in Omega (symmetric), rho_out I outside, and
    de/djc = -n rho j / jc in Omega (rho is proportional to jc^-n).  The warm
    start g does not enter (the result is linear in it: mu_g = chib lam_0)."""
    grid, mask, mat = prob.grid, prob.mask, prob.mat
    if mat.kim_h0 > 0 or tuple(mat.aniso) != (1.0, 1.0, 1.0):
        raise NotImplementedError("the reverse mode covers the isotropic, field-independent law of Eq. 1")
    chi = mask[None].astype(float)
    chib = 1.0 - chi
    Khat = prob.kernel()
    C = prob.curl_op()  # both curls are symmetric operators (odd symbols under a cross product)
    Phi = lambda f: phi_hockney(f, grid, Khat)  # noqa: E731
    # forward quantities the Jacobians need
    j = C(h)
    jn = np.sqrt(np.sum(j * j, axis=0))
    jc = np.asarray(mat.jc, dtype=np.float64) * np.ones(jn.shape)
    rho = (mat.e0 / jc) * (jn / jc) ** (mat.n - 1.0)
    # iterations, in reverse
    lam_i = lam.copy()
    mu_a = np.zeros(3)
    for _ in range(K):
        mu_a += np.sum(chib * lam_i, axis=(1, 2, 3))
        lam_i = chi * lam_i + C(chi * Phi(chib * lam_i))
    mu_g = chib * lam_i
    lam_u = chi * lam_i
    lam_e = -C(lam_u) / mat.mu0
    # power-law Jacobian transpose (Omega) / outer Ohm law (Omega_out)
    with np.errstate(invalid="ignore", divide="ignore"):
        jhat = np.where(jn > 0, j / np.where(jn > 0, jn, 1.0), 0.0)
    proj = np.sum(jhat * lam_e, axis=0)
    lam_j_in = rho[None] * (lam_e + (mat.n - 1.0) * proj[None] * jhat)
    lam_j = np.where(mask[None], lam_j_in, mat.rho_out * lam_e)
    mu_jc = np.where(mask, -mat.n * rho / jc * np.sum(j * lam_e, axis=0), 0.0)
    mu_h = C(lam_j)
    return RhsVJP(mu_h, mu_g, mu_jc, mu_a)


# ----------------------------------------------------------------------------
# Adjoint of fixed-step BS23 (frozen step list, fixed Eq. 5 iteration count)
# ----------------------------------------------------------------------------
@dataclass
class StepAdjoint:
    y: np.ndarray       # forward end state y_S
    mu_y0: np.ndarray   # dJ/dy_0 for J = <lam_T, y_S>
    mu_jc: np.ndarray   # dJ/djc (per node)
    mu_a: np.ndarray    # dJ/d(dh_e/dt), summed over every rhs call (and the first warm start)
    mu_path: np.ndarray  # dJ/d(path parameters): knot amplitudes (3 per knot) and sin_amp


def integrate_adjoint(prob: Problem, t0: float, dts: Sequence[float], y0: np.ndarray, lam_T: np.ndarray,
                      K: int, ts: Optional[Sequence[float]] = None) -> StepAdjoint:
    """Discrete adjoint of the fixed-step BS23 map y_0 -> y_S of `integrate` (Bogacki-
    Shampine pair, dt_list mode) with each rhs iterating Eq. 5 exactly K times.  The
    step times are ts (S + 1 values), or t0 + cumulative dts.  The forward chain of
    step n (t = t_n, dt = t_{n+1} - t_n) is
        Y2 = y + dt a21 k1,  k2 = F(t + dt/2, Y2; g=k1),  Y3 = y + dt a32 k2,
        k3 = F(t + 3dt/4, Y3; g=k2),  y' = y + dt (b1 k1 + b2 k2 + b3 k3),
        k4 = F(t_{n+1}, y'; g=k3)  (the left derivative of h_e when t_{n+1} is a kink),
        next k1 = k4 (FSAL), or, when t_{n+1} is a kink, next k1 = F(t_{n+1}, y'; g=k4)
        with the right derivative,
    with k1 = F(t_0, y_0; g_0) at the start and g_0 = dh_e/dt(t_0) (reading R-warm);
    F(t, h; g) depends on t only through the applied rate a = dh_e/dt(t).  The reverse
    sweep transposes it call by call with rhs_vjp; each call's cotangent of a (and that
    of g_0, summed over the nodes) maps to the path parameters through
    FieldPath.hedot_jacobian at that call's time and side."""
    a21, a32 = BS23_A[1][0], BS23_A[2][1]
    b1, b2, b3 = BS23_B[0], BS23_B[1], BS23_B[2]
    if ts is None:
        ts = [t0]
        for dt in dts:
            ts.append(ts[-1] + dt)
    ts = [float(v) for v in ts]
    S = len(ts) - 1
    kinks = set(prob.path.kinks())
    ends_on_kink = [ts[n + 1] in kinks for n in range(S)]
    F = lambda t, y, g, left=False: rhs(prob, t, y, g, delta_it=0.0, max_iter=K, left=left).hdot  # noqa: E731
    g0 = np.broadcast_to(prob.path.hedot(ts[0])[:, None, None, None], y0.shape).copy()

    def stages(n, y, k1):
        t, dt = ts[n], ts[n + 1] - ts[n]
        Y2 = y + dt * a21 * k1
        k2 = F(t + 0.5 * dt, Y2, k1)
        Y3 = y + dt * a32 * k2
        k3 = F(t + 0.75 * dt, Y3, k2)
        ynew = y + dt * (b1 * k1 + b2 * k2 + b3 * k3)
        k4 = F(ts[n + 1], ynew, k3, left=ends_on_kink[n])
        return Y2, k2, Y3, k3, ynew, k4

    # forward, storing y_n and k1_n
    ys, k1s = [y0.copy()], []
    k1 = F(ts[0], y0, g0)
    y = y0.copy()
    for n in range(S):
        k1s.append(k1)
        _, _, _, _, y, k4 = stages(n, y, k1)
        k1 = F(ts[n + 1], y, k4) if ends_on_kink[n] else k4
        ys.append(y.copy())
    # reverse
    P = 3 * len(prob.path.t) + 1
    mu_path = np.zeros(P)
    mu_jc = np.zeros(prob.mask.shape)
    mu_a = np.zeros(3)

    def back(t, left, Y, lam):
        v = rhs_vjp(prob, t, Y, lam, K, left=left)
        nonlocal mu_jc, mu_a, mu_path
        mu_jc = mu_jc + v.mu_jc
        mu_a = mu_a + v.mu_a
        mu_path = mu_path + prob.path.hedot_jacobian(t, left).T @ v.mu_a
        return v

    ybar = lam_T.copy()
    k1bar_next = np.zeros_like(y0)  # cotangent of the next step's first stage
    for n in range(S - 1, -1, -1):
        t, dt = ts[n], ts[n + 1] - ts[n]
        Y2, k2, Y3, k3, ynew, k4 = stages(n, ys[n], k1s[n])
        k1bar = np.zeros_like(y0)
        k2bar = np.zeros_like(y0)
        k3bar = np.zeros_like(y0)
        if ends_on_kink[n]:
            # next k1 = F(t_{n+1}, y'; g=k4) (right derivative), k4 = F(t_{n+1}, y'; g=k3) (left)
            v = back(ts[n + 1], False, ynew, k1bar_next)
            ybar = ybar + v.mu_h
            v = back(ts[n + 1], True, ynew, v.mu_g)
        else:
            v = back(ts[n + 1], False, ynew, k1bar_next)
        ybar = ybar + v.mu_h
        k3bar += v.mu_g
        # y' = y + dt (b1 k1 + b2 k2 + b3 k3)
        k1bar += dt * b1 * ybar
        k2bar += dt * b2 * ybar
        k3bar += dt * b3 * ybar
        # k3 = F(t + 3dt/4, Y3; g=k2), Y3 = y + dt a32 k2
        v = back(t + 0.75 * dt, False, Y3, k3bar)
        ybar = ybar + v.mu_h
        k2bar += v.mu_g + dt * a32 * v.mu_h
        # k2 = F(t + dt/2, Y2; g=k1), Y2 = y + dt a21 k1
        v = back(t + 0.5 * dt, False, Y2, k2bar)
        ybar = ybar + v.mu_h
        k1bar += v.mu_g + dt * a21 * v.mu_h
        k1bar_next = k1bar
    # k1 = F(t_0, y_0; g_0) with g_0 = dh_e/dt(t_0) at every node
    v = back(ts[0], False, ys[0], k1bar_next)
    ybar = ybar + v.mu_h
    mg0 = np.sum(v.mu_g, axis=(1, 2, 3))
    mu_a = mu_a + mg0
    mu_path = mu_path + prob.path.hedot_jacobian(ts[0], False).T @ mg0
    return StepAdjoint(ys[-1], ybar, mu_jc, mu_a, mu_path)
