"""The experiments of §3 of the paper, run through the library (FP32 FFTs, FP64 state).

    python paper_runs.py shield [--grid 128]      # cases A and B of the magnetic shield
    python paper_runs.py lens [--grid 128]        # field concentration of the magnetic lens

Shield (§3): a hollow cylinder closed at one end, centred in a cube of side 3.2, n = 30,
rho_out = 20.  The paper takes its sizes from its reference [2] and shows them only in a
figure, so two readings are run: "cup", a short cup (outer radius 1, inner 0.7, height 1.5,
end cap 0.2; the paper calls the cylinder short), and "long", the shield workload's
proportions (inner radius 0.8, height 3, cap 0.2).  Case A: h_e = (0, 0, t) for t <= tau,
then (t - tau, 0, tau); case B: the same ramps in the inverse order; tau = 0.09.  Reported:
the mean |h| over the "shielded zone" (a coaxial disk of thickness 0.143 and radius 0.667
whose middle plane lies 0.452 inside the closed end; reading: the closed end is the "top")
against |h_e|, the curves of the paper's Fig. 2.  (The paper finds that a field
perpendicular to the axis reaches the zone much more easily than an axial one; with these
guessed geometries the two cases stay within a factor of two of each other.)

Lens (§3): a cylinder of radius 1 and height 1 with a coaxial biconical hole (radius 0.25
at the mid-plane widening to 0.6 at the faces: readings, the paper shows the cone only in a
figure) and a radial slit of width 0.05, in a cube of side 3.6 (the paper's lateral extent;
its box is twice as long along z on a 128 x 128 x 256 grid, which the free-space Phi of this
library does not need), n = 30, rho_out = 100, h_e = (0, 0, t) for t <= 0.2.  Reported: the
concentration ratio <|h|> / |h_e| over {r <= 0.2, |z| <= 0.33}; the paper finds about 2 at
|h_e| = 0.05 and 1.6 at 0.2.

Prints one JSON line per run.  The averages over the zones are taken with torch on the
device snapshots (reporting only; every step of the method runs in the library).
"""

from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import scfft_inputs as I  # noqa: E402

TAU = 0.09


def _context(S, n, L, mask, n_power, rho_out, knots_t, knots_he, rtol=2e-4, atol=1e-7):
    ctx = S.Context(n, L, n_power=n_power, rho_out=rho_out, precision=S.PREC_F32, delta_it=2e-5, max_iter=100,
                    rtol=rtol, atol=atol)
    ctx.set_geometry(mask)
    ctx.set_field_path(knots_t, knots_he)
    ctx.precompute_kernel()
    return ctx


def _zone_mean_abs_h(torch, snaps, zone, N):
    z = torch.from_numpy(zone.reshape(-1)).cuda()
    s = snaps.view(-1, 3, N)
    mag = torch.sqrt((s * s).sum(dim=1))
    return (mag[:, z].mean(dim=1)).cpu().numpy()


SHIELDS = {"cup": (0.7, 1.5), "long": (0.8, 3.0)}  # inner radius, height (outer radius 1, cap 0.2)


def shield(S, torch, grid: int, case: str, geometry: str = "cup", nsnap: int = 18):
    n = (grid, grid, grid)
    L = (1.6, 1.6, 1.6)
    r_in, height = SHIELDS[geometry]
    mask = I.shield(n, L, 1.0, r_in, height, 0.2)
    kt, khe = I.shield_case_path(case, TAU)
    ctx = _context(S, n, L, mask, 30.0, 20.0, kt, khe)
    # the closed end is at z = -height/2; the zone's middle plane lies 0.452 inside it
    zone = I.disk_region(n, L, -0.5 * height + 0.452, 0.143, 0.667)
    assert not (zone & mask).any()
    N = int(np.prod(n))
    ts = [2 * TAU * (i + 1) / nsnap for i in range(nsnap)]
    h = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    snaps = torch.zeros(nsnap * 3 * N, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = ctx.integrate(0.0, 2 * TAU, 1e-5, h, tsnap=ts, snaps=snaps)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    hz = _zone_mean_abs_h(torch, snaps, zone, N)
    path = [np.interp(t, kt, np.asarray(khe)[:, 0]) for t in ts], [np.interp(t, kt, np.asarray(khe)[:, 2]) for t in ts]
    he = [float(np.hypot(a, b)) for a, b in zip(*path)]
    return {"run": f"shield ({geometry}) case {case}", "grid": list(n), "t": ts, "abs_he": he, "zone_mean_abs_h": hz.tolist(),
            "ratio": (hz / np.maximum(he, 1e-30)).tolist(), "steps": st["accepted"], "rejected": st["rejected"],
            "rhs_calls": st["rhs_calls"], "iters_per_rhs": st["iterations"] / max(st["rhs_calls"], 1),
            "seconds": wall}


def lens(S, torch, grid: int, shape: str, levels=(0.05, 0.1, 0.15, 0.2)):
    n = (grid, grid, grid)
    if shape == "biconical":
        L = (1.8, 1.8, 1.8)
        mask = I.biconical_lens(n, L, 1.0, 1.0, 0.25, 0.6, 0.05)
        zone = I.disk_region(n, L, 0.0, 0.66, 0.2)
    else:  # the straight bore of the benchmark's lens; the zone shrinks to fit the bore
        L = (1.6, 1.6, 1.6)
        mask = I.lens(n, L, 1.0, 1.0, 0.15, 0.05)
        zone = I.disk_region(n, L, 0.0, 0.66, 0.1)
    assert not (zone & mask).any()
    ctx = _context(S, n, L, mask, 30.0, 100.0, [0.0, 0.2], [[0, 0, 0], [0, 0, 0.2]])
    N = int(np.prod(n))
    h = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    snaps = torch.zeros(len(levels) * 3 * N, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = ctx.integrate(0.0, max(levels), 1e-5, h, tsnap=list(levels), snaps=snaps)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    hz = _zone_mean_abs_h(torch, snaps, zone, N)
    return {"run": f"lens ({shape} hole)", "grid": list(n), "abs_he": list(levels),
            "concentration": (hz / np.asarray(levels)).tolist(), "steps": st["accepted"],
            "rejected": st["rejected"], "rhs_calls": st["rhs_calls"],
            "iters_per_rhs": st["iterations"] / max(st["rhs_calls"], 1), "seconds": wall}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["shield", "lens", "all"])
    ap.add_argument("--grid", type=int, default=128)
    args = ap.parse_args()
    import torch
    import paper_1803_01346_gb300 as S
    from paper_1803_01346_gb300 import build as B
    B.build()
    if args.what in ("shield", "all"):
        for geometry in ("cup", "long"):
            for case in ("A", "B"):
                print(json.dumps(shield(S, torch, args.grid, case, geometry)), flush=True)
    if args.what in ("lens", "all"):
        for shape in ("biconical", "straight"):
            print(json.dumps(lens(S, torch, args.grid, shape)), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
