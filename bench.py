"""Benchmark: voxel-RHS evaluations per second of the method-of-lines
right-hand side (§2) on the 128^3 magnetic-lens workload, FP32 FFTs with FP64
integrator state, through the library's BS23 step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--t-start T]

One step = one accepted Bogacki-Shampine step of the lens workload (three
right-hand sides, each with its Eq. 5 iterations, plus the stage sums and the
error norm).  The timed steps start mid-ramp (t = T, default 0.3, on the ramp
of the applied field to 0.8): the trajectory is integrated from the virgin state
h = 0 (§3) up to T before the timed region, so the Eq. 5 iteration counts are
those of the regime the paper's runs spend their time in.  The first steps from
h = 0 are timed as well and reported as a separate, labelled figure.
value = grid nodes x right-hand sides evaluated / second, summed over ranks
(each rank runs its own replica; the method has no data-parallel exchange).
Prints one JSON line on rank 0.

--impl reference times the FP64 CPU oracle on the host cores instead: each
step is one Eq. 5 iteration of the oracle at 128^3 (the pre-stage is timed
once), converted to the same unit with the iteration count per right-hand side
that the GPU path measures over its default timed segment (REF_ITERS_PER_RHS).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import scfft_inputs as I  # noqa: E402

WORKLOAD = "lens128"
METRIC = "voxel-RHS evals/s at 128^3 (FP32 FFT, FP64 state)"
UNIT = "voxel-RHS evals/s"
# Eq. 5 iterations per right-hand side that the GPU path measures over its default timed
# segment of this workload (mid-ramp, t = 0.3: 5.0), used only to convert the reference
# arm's per-iteration samples to the metric's unit; the GPU arm's line states its own count.
REF_ITERS_PER_RHS = 5.0
T_START = 0.3  # start of the timed steps on the lens ramp (h_e reaches 0.8 at t = 0.8)
AUTOTUNE = True  # --no-autotune: keep the default launch schedule (profiling runs: under ncu the
                 # tuner's own timings are distorted and may pick another schedule)
# DRAM bytes (read + write) per launch from the committed ncu capture
# profiles/ncu_zpass_tm2_lens128_fp32.md; an entry is removed when its kernel changes.
NCU_TRAFFIC = {"z_kernel": 86768384 + 58679552}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def aggregate_ranks(ms: float, units: float, ws: int, device: str):
    """Whole-job figures of a multi-rank run: the slowest rank's time and the units all
    ranks processed (each rank runs its own replica).  Single rank: unchanged."""
    if ws <= 1:
        return ms, units
    import torch
    import torch.distributed as dist
    tm = torch.tensor([ms, units], dtype=torch.float64, device=device)
    dist.all_reduce(tm[0:1], op=dist.ReduceOp.MAX)
    dist.all_reduce(tm[1:2], op=dist.ReduceOp.SUM)
    return float(tm[0]), float(tm[1])


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms; `stop` keeps the
    samples whose nvidia-smi timestamp falls inside the timed region (marked by
    `begin`/`end` in the host's wall-clock time)."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.t_begin = self.t_end = None

    def _reader(self):
        import datetime
        for line in self.proc.stdout:
            try:
                ts = datetime.datetime.strptime(line.split(",")[0].strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                ts = time.time()
            self.lines.append((ts, line))

    def start(self):
        """Start sampling and wait (up to 3 s) for the first sample."""
        import threading
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        threading.Thread(target=self._reader, daemon=True).start()
        t0 = time.perf_counter()
        while not self.lines and time.perf_counter() - t0 < 3.0:
            time.sleep(0.01)

    def begin(self):
        self.t_begin = time.time()

    def end(self):
        self.t_end = time.time()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        inside = [ln for t, ln in self.lines if self.t_begin is not None and self.t_begin <= t <= self.t_end]
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in inside:
            parts = [p.strip() for p in line.split(",")][1:]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "window_ms": round((self.t_end - self.t_begin) * 1e3, 1) if self.t_begin is not None else None}


def source_box(mask) -> tuple:
    """Fractions of the planes (z) and of the rows (y, z) that hold Omega's bounding box, with
    the y bounds rounded out to even rows as the library does: the Eq. 5 convolution's source
    chi curl dh^i vanishes outside, and the forward padded passes skip the rest."""
    m = np.asarray(mask, dtype=bool)  # [z][y][x]
    zs = np.nonzero(m.any(axis=(1, 2)))[0]
    ys = np.nonzero(m.any(axis=(0, 2)))[0]
    nz, ny = m.shape[0], m.shape[1]
    y0, y1 = int(ys[0]) & ~1, min(ny, (int(ys[-1]) + 2) & ~1)
    nzb, nyb = int(zs[-1]) - int(zs[0]) + 1, y1 - y0
    return nzb / nz, nzb * nyb / (nz * ny)


def algorithmic_bytes(kind: str, n, fp_bytes: int, box=(1.0, 1.0)) -> float:
    """Bytes a pass must move per launch (each array read or written once); box = the plane
    and row fractions of the Eq. 5 source's support (source_box), which bound what the
    forward padded passes of an iteration must read and write."""
    nx, ny, nz = n
    N = nx * ny * nz
    fz, fyz = box
    c = 2 * fp_bytes                     # one complex value
    U = 3 * (nx // 2 + 1) * ny * nz * c  # unpadded half spectrum, 3 components
    Pin = 3 * (nx + 1) * ny * nz * c     # padded spectrum, rows y < ny
    Pall = 3 * (nx + 1) * 2 * ny * nz * c
    real = 3 * N * fp_bytes
    kap = 3 * (nx + 1) * (ny + 1) * (nz + 1) * fp_bytes
    table = {
        "x_fwd_state": 3 * N * 8 + U,
        "x_powerlaw": 2 * U + N,
        "x_assemble": 2 * U + N + real + 3 * N * 8,
        "x_maskpad": (U + N + Pin) * fyz,
        "x_update": Pin + 2 * real + N + U,
        "y_fwd_unpadded": 2 * U,
        "y_inv_unpadded": 2 * U,
        "z_curl": 2 * U,
        "y_fwd_padded": Pin * fyz + Pall * fz,
        "y_inv_padded": Pall + Pin,
        "z_kernel": Pall * fz + Pall + kap,
        # the curl's inverse y pass, mask/pad and the padded forward y pass as one launch: the
        # curl's half spectrum on the box's planes in, the mask on its rows, the padded spectrum
        # of its planes out
        "box_fused": U * fz + N * fyz + Pall * fz,
        "finalize": real + 2 * 3 * N * 8,
    }
    return float(table.get(kind, 0.0))


def make_ctx(S, cfg, precision, delta_it=2e-5, max_iter=100):
    ctx = S.Context(cfg.n, cfg.L, n_power=cfg.n_power, rho_out=cfg.rho_out, precision=precision,
                    delta_it=delta_it, max_iter=max_iter, rtol=cfg.rtol, atol=cfg.atol)
    ctx.set_geometry(cfg.mask)
    ctx.set_field_path(cfg.knots_t, cfg.knots_he)
    ctx.precompute_kernel()
    if AUTOTUNE:
        ctx.autotune()  # launch schedule of the FP32 passes (cached per grid; a no-op otherwise)
    return ctx


def run_steps(ctx, state, k):
    t, dt, h, warm = state
    for _ in range(k):
        t, dt, _ = ctx.step(t, dt, 10.0, h, warm)
    state[0], state[1] = t, dt


def cpu_oracle_sample(cfg, iters_per_rhs):
    """Time the oracle's pre-stage and one Eq. 5 iteration on the host cores."""
    import oracle as O
    g = O.Grid(cfg.n, cfg.L)
    prob = O.Problem(g, cfg.mask, O.Material(n=cfg.n_power, rho_out=cfg.rho_out),
                     O.FieldPath(cfg.knots_t, cfg.knots_he))
    prob.kernel()
    h = np.zeros((3,) + g.shape)
    gw = np.broadcast_to(prob.path.hedot(0.0)[:, None, None, None], h.shape).copy()
    t0 = time.perf_counter()
    O.rhs(prob, 0.0, h, gw, delta_it=0.0, max_iter=0)
    t_pre = time.perf_counter() - t0
    t0 = time.perf_counter()
    O.rhs(prob, 0.0, h, gw, delta_it=0.0, max_iter=1)
    t_iter = max(time.perf_counter() - t0 - t_pre, 1e-9)
    N = cfg.n[0] * cfg.n[1] * cfg.n[2]
    return N / (t_pre + iters_per_rhs * t_iter), t_pre, t_iter


def bench_reference(args, ws, rank):
    if rank != 0:
        return 0
    cfg = I.config(WORKLOAD)
    import oracle as O
    g = O.Grid(cfg.n, cfg.L)
    prob = O.Problem(g, cfg.mask, O.Material(n=cfg.n_power, rho_out=cfg.rho_out),
                     O.FieldPath(cfg.knots_t, cfg.knots_he))
    prob.kernel()
    h = np.zeros((3,) + g.shape)
    gw = np.broadcast_to(prob.path.hedot(0.0)[:, None, None, None], h.shape).copy()
    t0 = time.perf_counter()
    O.rhs(prob, 0.0, h, gw, delta_it=0.0, max_iter=0)
    t_pre = time.perf_counter() - t0
    # each step: one Eq. 5 iteration (pre-stage + 1 iteration, minus the pre-stage); at most
    # 30 timed and 2 warm-up samples (about 3.5 s each on a Grace core), so that the arm ends
    # within a few minutes whatever K is
    n_warm, n_timed = min(args.warmup, 2), max(1, min(args.steps, 30))
    for _ in range(n_warm):
        O.rhs(prob, 0.0, h, gw, delta_it=0.0, max_iter=1)
    times = []
    for _ in range(n_timed):
        t0 = time.perf_counter()
        O.rhs(prob, 0.0, h, gw, delta_it=0.0, max_iter=1)
        times.append(time.perf_counter() - t0 - t_pre)
    t_iter = statistics.mean(times)
    N = cfg.n[0] * cfg.n[1] * cfg.n[2]
    value = N / (t_pre + REF_ITERS_PER_RHS * t_iter)
    ms = (t_pre + t_iter) * 1e3
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": list(cfg.n), "padded": [2 * v for v in cfg.n],
                   "geometry": cfg.note, "step": "one Eq. 5 iteration of the FP64 NumPy oracle (pre-stage timed once)",
                   "iters_per_rhs": REF_ITERS_PER_RHS},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"pre-stage {t_pre:.2f}s once + {n_timed} Eq. 5 iterations (of {args.steps} steps asked) of mean {t_iter:.2f}s after {n_warm} warm-up, scaled to {REF_ITERS_PER_RHS} iterations per rhs"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def bench_batch(S, torch, steps: int, warmup: int):
    """64 independent shield instances (grids 32..96^3, FP32 FFTs) advanced by
    scfft_batch_step, each context on its own stream; compared with the same
    instances stepped one after another."""
    cfgs = I.batch_configs(64, seed=1803)
    streams = [torch.cuda.Stream() for _ in cfgs]
    inst = []
    schedules = {}
    for c, st in zip(cfgs, streams):
        ctx = S.Context(c.n, c.L, n_power=c.n_power, rho_out=c.rho_out, precision=S.PREC_F32, rtol=c.rtol,
                        atol=c.atol, stream=st.cuda_stream)
        ctx.set_geometry(c.mask)
        ctx.set_field_path(c.knots_t, c.knots_he)
        ctx.precompute_kernel()
        sched = ctx.autotune() if AUTOTUNE else ctx.get_schedule()  # timed once per grid size, then cached
        if c.n[0] not in schedules:
            schedules[c.n[0]] = sched
        N = int(np.prod(c.n))
        h = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
        w = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
        rate = np.asarray(c.knots_he[1]) / c.knots_t[1]
        for q in range(3):
            w.view(3, N)[q] = float(rate[q])
        inst.append((ctx, h, w, N))
    torch.cuda.synchronize()
    ctxs = [x[0] for x in inst]
    t = [0.0] * len(inst)
    dt = [1e-4] * len(inst)
    stop = [c.t_end for c in cfgs]
    hs = [x[1] for x in inst]
    wsv = [x[2] for x in inst]
    for _ in range(warmup):
        t, dt, _ = S.batch_step(ctxs, t, dt, stop, hs, wsv)
    torch.cuda.synchronize()
    c0 = [x[0].stats()["rhs_calls"] for x in inst]
    i0 = [x[0].stats()["iterations"] for x in inst]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    clocks.begin()
    t0 = time.perf_counter()
    for _ in range(steps):
        t, dt, _ = S.batch_step(ctxs, t, dt, stop, hs, wsv)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    clocks.end()
    clk = clocks.stop()
    evals = sum(x[3] * (x[0].stats()["rhs_calls"] - c) for x, c in zip(inst, c0))
    rcs = sum(x[0].stats()["rhs_calls"] - c for x, c in zip(inst, c0))
    its = sum(x[0].stats()["iterations"] - c for x, c in zip(inst, i0))
    # the same instances, one after another
    t1 = time.perf_counter()
    for i, (ctx, h, w, N) in enumerate(inst):
        ti, di = t[i], dt[i]
        for _ in range(steps):
            ti, di, _ = ctx.step(ti, di, stop[i], h, w)
    torch.cuda.synchronize()
    seq = time.perf_counter() - t1
    return {"instances": len(inst), "grids": sorted({c.n[0] for c in cfgs}), "steps": steps,
            "instance_steps_per_s": len(inst) * steps / el, "voxel_rhs_evals_per_s": evals / el,
            "sequential_instance_steps_per_s": len(inst) * steps / seq, "speedup_vs_sequential": seq / el,
            "iters_per_rhs": its / max(1, rcs),
            "schedules": {str(k): {kk: v[kk] for kk in ("z_kernel_tile", "z_curl_tile", "y_unpadded_tile",
                                                         "y_padded_tma", "z_kernel_tmem", "box_fused",
                                                         "x_update_split")}
                          for k, v in sorted(schedules.items())},
            "timing": "wall clock around synchronous batch calls, device synchronised on both sides",
            "clocks": clk}


def bench_adjoint(S, torch, nsteps: int, checkpoint: int, K: int):
    """Reverse mode on the lens at 96^3 with a seeded +-5% jc map (FP32 FFTs, FP64 state and
    gradients): an adaptive forward run of `nsteps` steps from the virgin state records its
    accepted step times; the frozen map over those times (K Eq. 5 iterations per rhs,
    checkpoints every `checkpoint` steps) is recorded and swept backwards step by step
    (scfft_adjoint_step) for J = |h(bore centre)|^2, giving dJ/djc per node, dJ/dy_0 and dJ/dA
    for the three components of the ramp amplitude A (the path ramps to A, then holds)."""
    cfg = I.config("lens96")
    N = int(np.prod(cfg.n))
    ctx = S.Context(cfg.n, cfg.L, n_power=cfg.n_power, rho_out=cfg.rho_out, precision=S.PREC_F32,
                    delta_it=2e-5, max_iter=K, rtol=cfg.rtol, atol=cfg.atol)
    ctx.set_geometry(cfg.mask)
    knots_t = [0.0, 0.8, 1.0]
    knots_he = [cfg.knots_he[0], cfg.knots_he[1], cfg.knots_he[1]]  # ramp to A = (0, 0, 0.8), then hold
    ctx.set_field_path(knots_t, knots_he)
    jc = torch.from_numpy(np.ascontiguousarray(cfg.jc).reshape(-1)).cuda()
    ctx.set_jc_map(jc)
    ctx.precompute_kernel()
    h = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    warm = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    warm.view(3, N)[2] = knots_he[1][2] / knots_t[1]
    t, dt, ts = 0.0, 1e-6, [0.0]
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(nsteps):
        t, dt, _ = ctx.step(t, dt, 10.0, h, warm)
        ts.append(t)
    torch.cuda.synchronize()
    fwd_s = time.perf_counter() - w0
    c = (cfg.n[2] // 2 * cfg.n[1] + cfg.n[1] // 2) * cfg.n[0] + cfg.n[0] // 2
    y0 = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    y_end = torch.empty_like(y0)
    gjc = torch.zeros(N, dtype=torch.float64, device="cuda")
    gp = np.zeros(3 * len(knots_t) + 1)
    s0 = ctx.stats()["rhs_calls"]
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    ctx.adjoint_record(ts, y0, y_end=y_end, checkpoint_every=checkpoint)
    lam = torch.zeros(3 * N, dtype=torch.float64, device="cuda")
    for q in range(3):
        lam[q * N + c] = 2.0 * float(y_end[q * N + c])
    for k in range(nsteps - 1, -1, -1):
        ctx.adjoint_step(k, lam, gjc, gp)
    torch.cuda.synchronize()
    rev_s = time.perf_counter() - w0
    calls = ctx.stats()["rhs_calls"] - s0
    dA = [float(gp[3 + a] + gp[6 + a]) for a in range(3)]
    J = float(sum(float(y_end[q * N + c]) ** 2 for q in range(3)))
    return {"workload": "lens96 (jc +-5%), FP32 FFTs", "steps": nsteps, "t_end": t, "checkpoint_every": checkpoint,
            "iters_per_rhs": K, "forward_adaptive_s": fwd_s, "record_and_reverse_s": rev_s,
            "adjoint_steps_per_s": nsteps / rev_s, "forward_rhs_in_record_and_reverse": int(calls),
            "objective": "|h(bore centre)|^2 at t_end", "J": J,
            "grad_jc_norm": float(gjc.norm()), "grad_amplitude": dA,
            "end_state_vs_adaptive_forward": float((y_end - h).abs().max() / h.abs().max().clamp_min(1e-300))}


def bench_ours(args, ws, rank, local):
    import torch
    import paper_1803_01346_gb300 as S
    from paper_1803_01346_gb300 import build as B

    torch.cuda.set_device(local)
    if rank == 0 or not os.path.exists(S.library_path()):
        B.build()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    cfg = I.config(WORKLOAD)
    N = cfg.n[0] * cfg.n[1] * cfg.n[2]
    n3 = 3 * N
    ctx = make_ctx(S, cfg, S.PREC_F32)
    sched_used = ctx.get_schedule()  # chosen by the autotuner in make_ctx
    h = torch.zeros(n3, dtype=torch.float64, device="cuda")
    warm = torch.zeros(n3, dtype=torch.float64, device="cuda")
    warm.view(3, N)[2] = cfg.knots_he[1][2] / cfg.knots_t[1]  # dh_e/dt at t = 0
    state = [0.0, 1e-6, h, warm]
    stream = torch.cuda.current_stream()
    # ---- the first steps from the virgin state h = 0 (a separate, labelled figure)
    run_steps(ctx, state, args.warmup)
    t_virgin = state[0]
    v0 = ctx.stats()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    run_steps(ctx, state, args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    v1 = ctx.stats()
    virgin = {"t_start": t_virgin, "steps": args.steps, "ms_per_step": ev0.elapsed_time(ev1) / args.steps,
              "value": N * (v1["rhs_calls"] - v0["rhs_calls"]) / (ev0.elapsed_time(ev1) * 1e-3),
              "rhs_per_step": (v1["rhs_calls"] - v0["rhs_calls"]) / args.steps,
              "iters_per_rhs": (v1["iterations"] - v0["iterations"]) / max(1, v1["rhs_calls"] - v0["rhs_calls"])}
    # ---- integrate on to the mid-ramp start of the timed steps (untimed), then warm up again
    wall = time.perf_counter()
    pre = 0
    while state[0] < args.t_start:
        state[0], state[1], _ = ctx.step(state[0], state[1], 10.0, h, warm)
        pre += 1
    pre_s = time.perf_counter() - wall
    # warm-up through the device-resident stepping (builds its graph before the timed region)
    state[0], state[1], _ = ctx.advance(state[0], state[1], 10.0, args.warmup, h, warm)
    # the timed segment's starting point: the profiled pass and the e2e pass below replay the
    # same steps from it (scfft_checkpoint_load continues a trajectory bit for bit)
    t_start = state[0]
    snap = ctx.checkpoint_save(state[0], state[1], h, warm)

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    # ---- timed region (device time, CUDA events on the library's stream)
    clocks = ClockSampler(local)
    clocks.start()
    s0 = ctx.stats()
    barrier()
    torch.cuda.synchronize()
    clocks.begin()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    # device-resident: the K steps are one graph launch (scfft_advance); no host between steps
    state[0], state[1], taken = ctx.advance(state[0], state[1], 10.0, args.steps, h, warm)
    e1.record(stream)
    torch.cuda.synchronize()
    clocks.end()
    barrier()
    ms = e0.elapsed_time(e1)
    s1 = ctx.stats()
    clk = clocks.stop()
    rhs_calls = s1["rhs_calls"] - s0["rhs_calls"]
    iters = s1["iterations"] - s0["iterations"]
    launches = s1["launches"] - s0["launches"]
    units = float(N * rhs_calls)
    t_max, units = aggregate_ranks(ms, units, ws, "cuda")
    value = units / (t_max * 1e-3)

    # ---- per-pass profile over the same number of steps (separate pass, events around each launch)
    ts = ctx.checkpoint_load(snap, h, warm)
    pstate = [ts[0], ts[1], h, warm]
    ctx.profile(True)
    # (the Eq. 5 loop runs host-driven while profiling, so every pass is a separate launch that
    # ncu --nvtx-include profiled_steps/ can list; inside the graph's conditional nodes it cannot)
    torch.cuda.nvtx.range_push("profiled_steps")
    run_steps(ctx, pstate, args.steps)
    torch.cuda.nvtx.range_pop()
    prof = ctx.profile_read()
    ctx.profile(False)
    kinds = {k: v for k, v in prof.items() if v[0] > 0}
    # the dominant pass among those with algorithmic HBM bytes (the one-thread stage kernels
    # of the device-resident step carry none)
    box = source_box(cfg.mask)
    dom = max((k for k in kinds if algorithmic_bytes(k, cfg.n, 4) > 0), key=lambda k: kinds[k][1])
    cnt, tot = kinds[dom]
    avg_ms = tot / cnt
    peak, peak_src = _peaks()
    # algorithmic bytes: the pass's per-unit figure for the whole grid (each array read or
    # written once); the same with the source box, the least the pass must move here
    achieved = algorithmic_bytes(dom, cfg.n, 4) / (avg_ms * 1e-3) / 1e9
    achieved_box = algorithmic_bytes(dom, cfg.n, 4, box) / (avg_ms * 1e-3) / 1e9
    total_prof_ms = sum(v[1] for v in kinds.values())
    shares = {k: round(v[1] / total_prof_ms, 4) for k, v in sorted(kinds.items(), key=lambda kv: -kv[1][1])}

    # ---- end to end through the public API with host buffers (pinned), copies inside the timed
    # region: the state h copied in and out on every step (the warm start stays on the device,
    # warm_host = None), and the same with the warm start copied out as well
    def e2e_run(with_warm):
        hd = torch.empty_like(h)
        wd = torch.empty_like(warm)
        te = ctx.checkpoint_load(snap, hd, wd)  # the same steps as the timed region
        h_host = hd.cpu().pin_memory()
        w_host = wd.cpu().pin_memory() if with_warm else None
        barrier()
        torch.cuda.synchronize()
        b0 = ctx.stats()
        st = [te[0], te[1]]
        e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e2.record(stream)
        for _ in range(args.steps):  # scfft_step_host: copies in, step, copies out, every step
            st[0], st[1], _ = ctx.step_host(st[0], st[1], 10.0, h_host, w_host, hd, wd)
        e3.record(stream)
        torch.cuda.synchronize()
        b1 = ctx.stats()
        ms = e2.elapsed_time(e3)
        return (ms, b1["rhs_calls"] - b0["rhs_calls"], (b1["h2d_bytes"] - b0["h2d_bytes"]) // args.steps,
                (b1["d2h_bytes"] - b0["d2h_bytes"]) // args.steps)

    ke = args.steps
    e2e_ms, e2e_rhs, e2e_h2d, e2e_d2h = e2e_run(False)
    e2e_value = N * e2e_rhs / (e2e_ms * 1e-3) * ws
    w_ms, w_rhs, w_h2d, w_d2h = e2e_run(True)
    e2e_warm = {"value": N * w_rhs / (w_ms * 1e-3) * ws, "h2d_bytes_per_step": w_h2d, "d2h_bytes_per_step": w_d2h,
                "api": "scfft_step_host with warm_host as well (the warm start copied out every step)"}

    # ---- the same steps driven from the host (scfft_step: one synchronisation per step)
    hh = torch.empty_like(h)
    wh = torch.empty_like(warm)
    th = ctx.checkpoint_load(snap, hh, wh)
    hstate = [th[0], th[1], hh, wh]
    torch.cuda.synchronize()
    q0 = ctx.stats()
    e8, e9 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e8.record(stream)
    run_steps(ctx, hstate, args.steps)
    e9.record(stream)
    torch.cuda.synchronize()
    q1 = ctx.stats()
    host_stepped = {"api": "scfft_step per step (host step control, one synchronisation per step)",
                    "value": N * (q1["rhs_calls"] - q0["rhs_calls"]) / (e8.elapsed_time(e9) * 1e-3),
                    "ms_per_step": e8.elapsed_time(e9) / args.steps, "rhs_calls": q1["rhs_calls"] - q0["rhs_calls"]}
    del hh, wh

    # ---- FP64 path on the same state (one step) and the FP32 error against it
    ctx64 = make_ctx(S, cfg, S.PREC_F64)
    hA = h.clone()
    w32 = warm.clone()
    w64 = warm.clone()
    o32 = torch.empty_like(h)
    o64 = torch.empty_like(h)
    ctx64.rhs(state[0], hA, w64, o64)
    ctx.rhs(state[0], hA, w32, o32)

    def per_comp(a_, b_):
        return {"dhdt_" + nm: float((a_.view(3, N)[ci] - b_.view(3, N)[ci]).abs().max()
                                    / b_.view(3, N)[ci].abs().max().clamp_min(1e-300))
                for ci, nm in enumerate(("x", "y", "z"))}
    # as run: each path stops Eq. 5 at its own first residual below delta_it (the iteration
    # truncation then dominates the difference)
    fp32_err_stop = per_comp(o32, o64)
    # FP32 arithmetic alone: the same state and warm start, 8 Eq. 5 iterations on both paths
    fixed_it = 8
    c32f = make_ctx(S, cfg, S.PREC_F32, delta_it=0.0, max_iter=fixed_it)
    c64f = make_ctx(S, cfg, S.PREC_F64, delta_it=0.0, max_iter=fixed_it)
    cdff = make_ctx(S, cfg, S.PREC_DF64, delta_it=0.0, max_iter=fixed_it)
    odf = torch.empty_like(h)
    c32f.rhs(state[0], hA, warm.clone(), o32)
    # (NVTX ranges: every pass of these calls does work, so ncu can pick any launch in them)
    torch.cuda.nvtx.range_push("fp64_fixed_iterations")
    c64f.rhs(state[0], hA, warm.clone(), o64)
    torch.cuda.nvtx.range_pop()
    torch.cuda.nvtx.range_push("df64_fixed_iterations")
    cdff.rhs(state[0], hA, warm.clone(), odf)
    torch.cuda.nvtx.range_pop()
    fp32_err = per_comp(o32, o64)
    fp32_err["iterations"] = fixed_it
    df64_err = per_comp(odf, o64)
    df64_err["iterations"] = fixed_it
    del c32f, c64f, cdff
    st64 = [state[0], state[1], h.clone(), warm.clone()]
    torch.cuda.synchronize()
    c0 = ctx64.stats()["rhs_calls"]
    k64 = max(1, min(args.steps, 3))
    e4, e5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e4.record(stream)
    run_steps(ctx64, st64, k64)
    e5.record(stream)
    torch.cuda.synchronize()
    fp64_value = N * (ctx64.stats()["rhs_calls"] - c0) / (e4.elapsed_time(e5) * 1e-3)
    fp64_ms_per_step = e4.elapsed_time(e5) / k64
    del ctx64
    # the double-float path (FP64-equivalent transforms on the FP32 pipes) over the same steps
    cdf = make_ctx(S, cfg, S.PREC_DF64)
    stdf = [state[0], state[1], h.clone(), warm.clone()]
    torch.cuda.synchronize()
    d0 = cdf.stats()
    e10, e11 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e10.record(stream)
    run_steps(cdf, stdf, k64)
    e11.record(stream)
    torch.cuda.synchronize()
    d1 = cdf.stats()
    df64 = {"value": N * (d1["rhs_calls"] - d0["rhs_calls"]) / (e10.elapsed_time(e11) * 1e-3), "unit": UNIT,
            "steps": k64, "ms_per_step": e10.elapsed_time(e11) / k64, "fp64_ms_per_step": fp64_ms_per_step,
            "speedup_vs_fp64": fp64_ms_per_step / (e10.elapsed_time(e11) / k64),
            "iters_per_rhs": (d1["iterations"] - d0["iterations"]) / max(1, d1["rhs_calls"] - d0["rhs_calls"]),
            "error_vs_fp64": df64_err,
            "what": "SCFFT_PREC_DF64: double-float FFT passes (hi + lo FP32), node-wise law and stages in FP64"}
    del cdf, stdf

    # the local-stencil curl option: its own trajectory from the virgin state (a state of the
    # spectral trajectory is not one of the stencil's: its unsmoothed curl at the voxel
    # staircase exceeds jc, and the n = 30 law makes that stiff), up to 800 device-resident
    # steps or t = 0.3, then K steps timed as the headline's are (one scfft_advance launch)
    fd = None
    if not args.no_fd and rank == 0:
        cfd = make_ctx(S, cfg, S.PREC_F32)
        cfd.set_curl(S.CURL_FD)
        hf, wf = torch.zeros_like(h), torch.zeros_like(warm)
        for q in range(3):
            wf.view(3, N)[q] = float(cfg.knots_he[1][q]) / cfg.knots_t[1]
        tf, dtf, npre = cfd.advance(0.0, 1e-5, 0.3, 800, hf, wf)
        tf, dtf, _ = cfd.advance(tf, dtf, 10.0, args.warmup, hf, wf)
        f0 = cfd.stats()
        torch.cuda.synchronize()
        e6, e7 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e6.record(stream)
        tf1, dtf, nf = cfd.advance(tf, dtf, 10.0, args.steps, hf, wf)
        e7.record(stream)
        torch.cuda.synchronize()
        f1 = cfd.stats()
        fd_ms = e6.elapsed_time(e7)
        # the cost of one rhs at a fixed count of 5 Eq. 5 iterations on the headline's mid-ramp
        # state, spectral against stencil curl (the same work per call, whatever the trajectory)
        per_rhs = {}
        for kind in (S.CURL_SPECTRAL, S.CURL_FD):
            cx = make_ctx(S, cfg, S.PREC_F32, delta_it=0.0, max_iter=5)
            cx.set_curl(kind)
            ox = torch.empty_like(h)
            wx = warm.clone()
            for _ in range(3):
                cx.rhs(state[0], h, wx, ox)
            torch.cuda.synchronize()
            ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ea.record(stream)
            for _ in range(10):
                cx.rhs(state[0], h, wx, ox)
            eb.record(stream)
            torch.cuda.synchronize()
            per_rhs["spectral" if kind == S.CURL_SPECTRAL else "stencil"] = ea.elapsed_time(eb) / 10
            del cx
        fd = {"curl": "second-order central differences (stencil passes, no unpadded FFTs)",
              "ms_per_rhs_5_iterations": per_rhs,
              "value": N * (f1["rhs_calls"] - f0["rhs_calls"]) / (fd_ms * 1e-3), "unit": UNIT,
              "ms_per_step": fd_ms / max(nf, 1), "steps": nf, "t_start": tf, "steps_before_t_start": npre,
              "rhs_per_step": (f1["rhs_calls"] - f0["rhs_calls"]) / max(nf, 1),
              "iters_per_rhs": (f1["iterations"] - f0["iterations"]) / max(1, f1["rhs_calls"] - f0["rhs_calls"])}
        del cfd
    cufft = None
    if not args.no_cufft and rank == 0:
        import cufft_baseline
        cufft = [cufft_baseline.compare(S, torch, n, (1.6, 1.6, 1.6)) for n in ((128, 128, 128), (96, 96, 96))]
    batch = None if (args.no_batch or rank != 0) else bench_batch(S, torch, max(2, min(args.steps, 5)), 2)
    adjoint = None if (args.no_adjoint or rank != 0) else bench_adjoint(S, torch, 2000, 50, 5)
    if rank != 0:
        return 0
    cpu = None
    if ws == 1 and not args.no_cpu:
        v, tp, ti = cpu_oracle_sample(cfg, iters / max(rhs_calls, 1))
        cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"FP64 NumPy oracle on the 128^3 lens: pre-stage {tp:.2f}s + one Eq. 5 iteration "
                         f"{ti:.2f}s, scaled to {iters / max(rhs_calls, 1):.2f} iterations per RHS"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": list(cfg.n), "padded": [2 * v for v in cfg.n],
                   "geometry": cfg.note, "state_dtype": "f64", "n": cfg.n_power, "rho_out": cfg.rho_out,
                   "rtol": cfg.rtol, "delta_it": 2e-5, "t_start": None, "steps_before_t_start": pre,
                   "seconds_to_t_start": round(pre_s, 2), "rhs_per_step": rhs_calls / args.steps,
                   "iters_per_rhs": iters / max(rhs_calls, 1), "steps_taken": taken,
                   "stepping": "device-resident: the K steps are one CUDA graph launch (scfft_advance)",
                   "schedule": sched_used,
                   "l2": "inputs larger than L2 (FP64 state and "
                   "stage buffers 7 x 50 MB, padded spectrum 101 MB per pass)",
                   "parallelism": f"replicas x{ws}"},
        "virgin_state": virgin,
        "host_stepped": host_stepped,
        "fp64_path": {"value": fp64_value, "unit": UNIT, "steps": k64, "ms_per_step": fp64_ms_per_step},
        "df64_path": df64,
        "fp32_error_vs_fp64": fp32_err,
        "fp32_error_vs_fp64_early_stop": fp32_err_stop,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": e2e_h2d, "d2h_bytes_per_step": e2e_d2h,
                "api": "scfft_step_host (the state h in pinned host memory, copied in and out every step)",
                "steps": ke, "rhs_calls": e2e_rhs, "same_steps_as_value": e2e_rhs == rhs_calls,
                "with_warm_start": e2e_warm},
        "gpu_launches": int(launches),
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "peak_source": peak_src, "traffic": NCU_TRAFFIC.get(dom),
                     "bytes_per_launch": algorithmic_bytes(dom, cfg.n, 4), "avg_launch_ms": avg_ms,
                     "source_box": {"plane_fraction": box[0], "row_fraction": box[1],
                                    "bytes_per_launch": algorithmic_bytes(dom, cfg.n, 4, box),
                                    "achieved": achieved_box, "frac": achieved_box / peak},
                     "launches": cnt},
        "pass_shares": shares,
        "clocks": clk,
        "cpu_baseline": cpu,
        "stencil_curl": fd,
        "cufft_baseline": cufft,
        "batch": batch,
        "adjoint": adjoint,
    }
    line["config"]["t_start"] = t_start
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--t-start", type=float, default=T_START, help="time at which the timed steps start")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-instances leg")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the reverse-mode leg")
    ap.add_argument("--no-cufft", action="store_true", help="skip the cuFFT baseline of the padded convolution")
    ap.add_argument("--no-fd", action="store_true", help="skip the stencil-curl leg")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch schedule")
    args = ap.parse_args()
    global AUTOTUNE
    AUTOTUNE = not args.no_autotune
    ws, rank, local = _dist()
    if args.impl == "reference":
        return bench_reference(args, ws, rank)
    if ws > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    try:
        return bench_ours(args, ws, rank, local)
    finally:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
