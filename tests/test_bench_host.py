"""Host logic of bench.py that needs no GPU: the clock sampler keeps the nvidia-smi samples
whose timestamps fall inside the timed region (a stand-in nvidia-smi prints them here), and
reports its absence instead of failing."""

import importlib.util
import os
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_clock_sampler_keeps_only_samples_inside_the_timed_region(tmp_path, monkeypatch):
    fake = tmp_path / "nvidia-smi"
    fake.write_text("#!/bin/bash\nwhile true; do\n"
                    "  echo \"$(date +'%Y/%m/%d %H:%M:%S.%3N'), 0, 1980, 2070, 900.0, 0x4, "
                    "Not Active, Not Active, Not Active, Active\"\n  sleep 0.02\ndone\n")
    fake.chmod(0o755)
    monkeypatch.setenv("PATH", f"{tmp_path}{os.pathsep}{os.environ['PATH']}")
    c = _bench().ClockSampler(0)
    c.start()
    time.sleep(0.3)  # samples before the region
    c.begin()
    time.sleep(0.3)
    c.end()
    time.sleep(0.3)  # and after it
    r = c.stop()
    total = len(c.lines)
    assert 3 <= r["samples"] < total, (r, total)
    assert r["sm_mhz"] == 1980.0 and r["sm_max_mhz"] == 2070.0
    assert r["reasons"] == ["sw_power_cap"]
    assert 250 <= r["window_ms"] <= 600


def test_clock_sampler_without_nvidia_smi(tmp_path, monkeypatch):
    monkeypatch.setenv("PATH", str(tmp_path))
    c = _bench().ClockSampler(0)
    c.start()
    c.begin()
    c.end()
    assert c.stop()["reasons"] == ["nvidia-smi unavailable"]


def test_algorithmic_bytes_of_the_padded_z_pass_and_one_eq5_iteration():
    """The roofline's numerator, counted from the layouts: the padded z pass reads and writes
    the N_z non-zero planes of the padded half spectrum (3 components x (N_x+1) x 2N_y x N_z
    complex FP32) and reads the kernel spectrum's octant (3 x (N_x+1)(N_y+1)(N_z+1) floats);
    the eight passes of one Eq. 5 iteration at 128^3 move 0.893 GB."""
    b = _bench()
    n = (128, 128, 128)
    p_all = 3 * 129 * 256 * 128 * 8
    assert b.algorithmic_bytes("z_kernel", n, 4) == 2 * p_all + 3 * 129 ** 3 * 4 == 228_659_724
    u = 3 * 65 * 128 * 128 * 8
    assert b.algorithmic_bytes("z_curl", n, 4) == 2 * u
    passes = ("x_update", "y_fwd_unpadded", "z_curl", "y_inv_unpadded", "x_maskpad", "y_fwd_padded",
              "z_kernel", "y_inv_padded")
    assert abs(sum(b.algorithmic_bytes(k, n, 4) for k in passes) - 0.8935e9) < 1e6


def test_cufft_baseline_kernel_spectrum_matches_the_oracle():
    """The cuFFT yardstick builds the same sampled-kernel spectrum as the oracle's Hockney
    convolution (checked here with torch on the CPU; on the GPU the bench compares its
    result with scfft_phi before timing)."""
    import numpy as np
    import pytest
    torch = pytest.importorskip("torch")
    import cufft_baseline as C
    import oracle as O

    n, L = (6, 8, 4), (1.0, 1.2, 0.7)
    g = O.Grid(n, L)
    ref = O.hockney_kernel_spectrum(g)[:, :, :, : n[0] + 1]
    K = C.kernel_spectrum(torch, n, L, g.sigma, device="cpu").numpy()
    assert np.abs(K - ref).max() < 1e-6 * np.abs(ref).max()


def test_source_box_fractions():
    """The bench's source box (for the box-aware bytes of the forward padded passes) takes
    Omega's bounding planes and rows, the rows rounded out to even bounds as the library
    rounds them for its row pairs."""
    import numpy as np
    bench = _bench()
    m = np.zeros((16, 20, 8), dtype=bool)  # [z][y][x]
    m[3:7, 5:9, 2:4] = True                # planes 3..6, rows 5..8 -> rows 4..9 after rounding
    fz, fyz = bench.source_box(m)
    assert fz == 4 / 16
    assert fyz == (4 * 6) / (16 * 20)
    m[:] = False
    m[2, 18, 1] = True                     # one node in the last even row pair: rows 18..19
    assert bench.source_box(m) == (1 / 16, 2 / (16 * 20))


def test_algorithmic_bytes_of_the_fused_box_passes():
    """The fused box passes (the curl's inverse y pass, the mask/pad x pass and the padded
    forward y pass in one launch) read the curl's half spectrum on the box's planes and the mask
    on its rows and write the padded spectrum of its planes once: fewer bytes than the three
    passes on the same box, which each make a round trip."""
    b = _bench()
    n = (128, 128, 128)
    N = 128 ** 3
    u = 3 * 65 * 128 * 128 * 8
    p_in = 3 * 129 * 128 * 128 * 8
    p_all = 3 * 129 * 256 * 128 * 8
    box = (40 / 128, 40 * 80 / (128 * 128))
    fused = b.algorithmic_bytes("box_fused", n, 4, box)
    assert fused == u * box[0] + N * box[1] + p_all * box[0]
    three = (2 * u + (u + N + p_in) * box[1] + p_in * box[1] + p_all * box[0])
    assert b.algorithmic_bytes("y_inv_unpadded", n, 4) + b.algorithmic_bytes("x_maskpad", n, 4, box) + \
        b.algorithmic_bytes("y_fwd_padded", n, 4, box) == three
    assert fused < three
