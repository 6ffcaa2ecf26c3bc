"""Library-FFT yardstick for the zero-padded Biot-Savart convolution (Eqs. 6-7 by zero
padding), timed beside the library's own passes by bench.py.  Not part of the library:
libscfft.so never links cuFFT, and nothing here is called on the product path.

The same operator as scfft_phi: the three components of j (FP64 on the device) are
zero-padded to 2nx x 2ny x 2nz, transformed by a real-to-complex 3D FFT (cuFFT through
torch.fft, FP32), multiplied by the spectrum of the sampled kernel dV grad G_sigma (the
offset -N_a planes zeroed, so the kernel is odd and its transform vanishes at k = 0; Eq. 7's
rule), transformed back and cropped to the first nx x ny x nz block.  The kernel spectrum
is built once here with torch from the same sampling rule, and the result is checked
against scfft_phi on the same input before timing.
"""

from __future__ import annotations

import math


def kernel_spectrum(torch, n, L, sigma, device="cuda"):
    """rfftn over (z, y, x) of dV grad G_sigma sampled at the offsets m_a d_a, m_a in [-n_a, n_a)
    (cyclic order), with every m_a = -n_a plane zeroed: shape (3, 2nz, 2ny, nx + 1), complex64."""
    nx, ny, nz = n
    d = [2.0 * L[a] / n[a] for a in range(3)]
    dV = d[0] * d[1] * d[2]
    dev = device

    def offs(k, da):
        m = torch.fft.fftfreq(2 * k, d=1.0 / (2 * k), device=dev, dtype=torch.float64)
        return m * da

    rx = offs(nx, d[0])[None, None, :]
    ry = offs(ny, d[1])[None, :, None]
    rz = offs(nz, d[2])[:, None, None]
    r = torch.sqrt(rx * rx + ry * ry + rz * rz)
    u = r / (math.sqrt(2.0) * sigma)
    rs = torch.where(r > 0, r, torch.ones_like(r))
    g = ((2.0 / math.sqrt(math.pi)) * u * torch.exp(-u * u) - torch.special.erf(u)) / (4.0 * math.pi * rs * rs)
    g = torch.where(r > 0, g, torch.zeros_like(g))
    K = torch.stack([dV * g * rx / rs, dV * g * ry / rs, dV * g * rz / rs])
    K[:, :, :, nx] = 0.0
    K[:, :, ny, :] = 0.0
    K[:, nz, :, :] = 0.0
    return torch.fft.rfftn(K.to(torch.float32), dim=(1, 2, 3))


class PaddedPhi:
    """Phi_d[j] with cuFFT: FP64 j in, FP64 Phi out (the I/O of scfft_phi)."""

    def __init__(self, torch, n, L, sigma_scale=1.0):
        self.torch = torch
        self.n = tuple(n)
        d = [2.0 * L[a] / n[a] for a in range(3)]
        sigma = sigma_scale * 0.5 * math.sqrt(sum(v * v for v in d))
        self.K = kernel_spectrum(torch, n, L, sigma)
        nx, ny, nz = n
        self.pad = torch.zeros((3, 2 * nz, 2 * ny, 2 * nx), dtype=torch.float32, device="cuda")

    def __call__(self, j, out):
        torch = self.torch
        nx, ny, nz = self.n
        self.pad[:, :nz, :ny, :nx] = j.view(3, nz, ny, nx)
        J = torch.fft.rfftn(self.pad, dim=(1, 2, 3))
        K = self.K
        P = torch.stack([K[1] * J[2] - K[2] * J[1], K[2] * J[0] - K[0] * J[2], K[0] * J[1] - K[1] * J[0]])
        p = torch.fft.irfftn(P, s=(2 * nz, 2 * ny, 2 * nx), dim=(1, 2, 3))
        out.view(3, nz, ny, nx).copy_(p[:, :nz, :ny, :nx])


def compare(S, torch, n, L, reps=20, warmup=3):
    """Time scfft_phi (FP32 context) and the cuFFT version on the same FP64 input; both
    include the FP64 -> FP32 conversion of j and the FP32 -> FP64 write of Phi.  Returns a
    dict with the per-call times (CUDA events, inputs larger than L2 at 128^3), their ratio
    and the relative difference of the two results."""
    N = n[0] * n[1] * n[2]
    g = torch.Generator(device="cuda").manual_seed(1803)
    j = torch.randn(3 * N, dtype=torch.float64, device="cuda", generator=g)
    ctx = S.Context(n, L, precision=S.PREC_F32)
    ctx.precompute_kernel()
    ours = torch.empty_like(j)
    lib = torch.empty_like(j)
    base = PaddedPhi(torch, n, L)
    ctx.phi(j, ours)
    base(j, lib)
    torch.cuda.synchronize()
    diff = float((ours - lib).abs().max() / lib.abs().max())
    stream = torch.cuda.current_stream()

    def timed(f):
        for _ in range(warmup):
            f()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            f()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    t_ours = timed(lambda: ctx.phi(j, ours))
    t_lib = timed(lambda: base(j, lib))
    return {"grid": list(n), "padded": [2 * v for v in n], "ms_ours": t_ours, "ms_cufft": t_lib,
            "speedup_vs_cufft": t_lib / t_ours, "max_rel_diff": diff,
            "what": "Phi_d[j] of 3 components, FP64 in and out, FP32 transforms: scfft_phi (pruned passes, "
                    "kernel product fused into the z pass) vs torch.fft (cuFFT) rfftn / product / irfftn / crop"}
