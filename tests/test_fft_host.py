"""The shared-memory FFT headers (paper_2505_07814_gb300/csrc/fft_smem.cuh and fft_cluster.cuh)
compiled for the host.

tests/fft_host_check.cpp runs the headers' transform steps one emulated thread at a time, with a
step finished by every thread before the next starts, as the barrier after each step guarantees
on the GPU.  The N = 256 transform runs on four emulated CTAs of a cluster
(tests/host_shim/cooperative_groups.h maps a CTA's shared-memory pointer to another CTA's buffer).
It compares them with a direct double-precision 2D DFT, read through the k-space digit layout
(kbin0 / kbin1).  Cases: N = 64 (128 threads), N = 128 (256 and 512 threads) and N = 256 (four CTAs
of 512 threads, or eight of 128 with PTY_N256_CTAS=8).  Each is checked with the default butterflies,
twiddle skip and preloads, with each switched off, and with other thread-group counts of the
row-local steps (PTY_GROUPS, PTY_GROUPS256: every task of a step must still be run exactly once).

Bounds: an FP32 FFT of N^2 = 2^14 points has a relative L2 error of a few 1e-7 (1.3e-7 measured
for one transform, 5e-7 for the two-transform fused chains); the bounds leave 5-8x headroom and are
far below the error of any wrong twiddle, sign or index (a 0.1% error in one butterfly constant
gives 3e-4, a cross-CTA write to the wrong rank 1.4).
"""
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CXX = shutil.which("g++") or shutil.which("c++")


@pytest.mark.skipif(CXX is None, reason="no host C++ compiler")
@pytest.mark.parametrize("defines", [[], ["-DPTY_DFT_FMA=0"], ["-DPTY_TW_SKIP=0"], ["-DPTY_PRELOAD=0", "-DPTY_PRELOAD_BLOCK=1"],
                                     ["-DPTY_N256_CTAS=8", "-DPTY_GROUPS256=2"], ["-DPTY_GROUPS=4", "-DPTY_GROUPS256=1"],
                                     ["-DPTY_GROUPS=2", "-DPTY_GROUPS256=2"]],
                         ids=["default", "plain-combine", "no-skip", "no-preload", "eight-ctas", "groups-4-1", "groups-2"])
def test_fft_steps_match_direct_dft(tmp_path, defines):
    exe = str(tmp_path / "fft_host_check")
    subprocess.run([CXX, "-O2", "-std=c++17", "-Wno-unknown-pragmas", *defines,
                    "-I", os.path.join(ROOT, "tests", "host_shim"),
                    "-I", os.path.join(ROOT, "paper_2505_07814_gb300", "csrc"),
                    os.path.join(ROOT, "tests", "fft_host_check.cpp"), "-o", exe], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    rows = re.findall(r"N (\d+) T (\d+) fwd (\S+) inv (\S+) fused (\S+)", out)
    t256 = 128 if "-DPTY_N256_CTAS=8" in defines else 512
    assert [(int(n), int(t)) for n, t, *_ in rows] == [(64, 128), (128, 256), (128, 512), (256, t256)], out
    for n, t, fwd, inv, fused in rows:
        assert float(fwd) <= 1e-6 and float(inv) <= 1e-6, (n, t, fwd, inv)
        assert float(fused) <= 2e-6, (n, t, fused)
