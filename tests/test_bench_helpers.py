"""Host-side arithmetic of the benchmark (CPU only): the 95 % interval of a
frame error rate, the exact PCE-ET FER curve over D_max and the matched
D_max of the equal-FER comparison, and the algorithmic bytes per
frame-iteration of QC and CSR codes."""
import math
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2507_03509_gb300 import gen  # noqa: E402


def test_wilson_interval_closed_forms():
    # k = 0: lower end 0, upper end z^2 / (n + z^2)
    z = 1.959964
    lo, hi = bench.wilson_interval(0, 100)
    assert lo == 0.0 and hi == pytest.approx(z * z / (100 + z * z), rel=1e-12)
    # symmetric about 1/2 at k = n/2, and k <-> n - k mirrors the interval
    lo, hi = bench.wilson_interval(50, 100)
    assert lo + hi == pytest.approx(1.0, abs=1e-12)
    a = bench.wilson_interval(7, 40)
    b = bench.wilson_interval(33, 40)
    assert a[0] == pytest.approx(1 - b[1], abs=1e-12) and a[1] == pytest.approx(1 - b[0], abs=1e-12)
    # large n: close to the normal interval p +- z sqrt(p(1-p)/n)
    lo, hi = bench.wilson_interval(300000, 1000000)
    half = z * math.sqrt(0.3 * 0.7 / 1e6)
    assert lo == pytest.approx(0.3 - half, abs=1e-6) and hi == pytest.approx(0.3 + half, abs=1e-6)


def test_fer_curve_and_matched_dmax():
    # 8 frames: decoded at 5, 10, 10, 40, 300, 700; two never decoded
    ok = np.array([1, 1, 1, 1, 1, 1, 0, 0], dtype=bool)
    it = np.array([5, 10, 10, 40, 300, 700, 1000, 1000])
    k = bench.pce_decoded_at(ok, it)
    assert bench.fer_at(k, 4) == 1.0
    assert bench.fer_at(k, 10) == pytest.approx(5 / 8)
    assert bench.fer_at(k, 1000) == pytest.approx(2 / 8)
    assert bench.matched_dmax(k, 5 / 8, 1000) == 10       # reached exactly at 10
    assert bench.matched_dmax(k, 0.5, 1000) == 40         # FER 4/8 first at 40
    assert bench.matched_dmax(k, 0.3, 1000) == 700        # FER 2/8 <= 0.3 first at 700
    assert bench.matched_dmax(k, 0.0, 1000) == 1000       # never reached: the largest D_max


def test_algorithmic_bytes():
    qc = gen.workload_code(2, Z=64)
    assert bench.algorithmic_bytes_per_frame_iter(qc) == 8 * qc.edges + 12 * qc.n
    csr = gen.workload_code(1)
    assert bench.algorithmic_bytes_per_frame_iter(csr) == 16 * csr.edges + 12 * csr.n


def test_frame_kernel_naming_follows_the_shared_memory_rule():
    """The bench names the frame-per-CTA (or per-pair) kernel for the n = 4096 CSR code (about
    148 KB of shared memory) and lock-step for QC codes and for a CSR code of
    60000 edges, whose messages alone exceed the 220 KB limit."""
    small = gen.workload_code(1)
    assert bench.frame_schedule_applies(small)
    assert bench.decoder_kernel_name(small) == "csr_frame_kernel<false,1>"
    # a CTA pair per frame when every frame gets its own pair (64 frames on 152 SMs), one CTA otherwise
    assert bench.decoder_kernel_name(small, "auto", 64, 152) == "csr_frame_kernel<false,2>"
    assert bench.decoder_kernel_name(small, "auto", 100, 152) == "csr_frame_kernel<false,1>"
    assert bench.decoder_kernel_name(small, "frame", 64, 152) == "csr_frame_kernel<false,1>"
    assert bench.decoder_kernel_name(small, "frame_pair") == "csr_frame_kernel<false,2>"
    assert bench.decoder_kernel_name(small, "lockstep") == "bp_decode_kernel<float,CsrDev>"
    big = gen.random_csr_code(20000, 10000, 3, {6: 10000}, seed=77)
    assert not bench.frame_schedule_applies(big)
    qc = gen.workload_code(2, Z=64)
    assert not bench.frame_schedule_applies(qc)
    assert bench.decoder_kernel_name(qc) == "bp_decode_kernel<float,QcDev>"


def test_mufu_count_follows_the_check_rule():
    """Special-function operations per check pass, counted by hand: degree 3
    takes 3 exponentials + 3 reciprocals + 3 logarithms = 9, degree 4 takes
    4 + 6 + 4 = 14, degree 7 (general path) 7 + 6 + 7 = 30 with its extra
    combination; degrees 1 and 2 take none."""
    rowptr = np.array([0, 1, 3, 6, 10, 17], dtype=np.int32)  # degrees 1, 2, 3, 4, 7
    colidx = np.concatenate([[0], [0, 1], [0, 1, 2], [0, 1, 2, 3], np.arange(7)]).astype(np.int32)
    code = gen.CSRCode(m=5, n=7, rowptr=rowptr, colidx=colidx)
    assert bench.mufu_per_frame_iter(code) == 9 + 14 + 30
    qc = gen.workload_code(2, Z=64)
    deg = (np.asarray(qc.shifts) >= 0).sum(axis=1)
    want = int(sum(5 * d - 6 for d in deg if 3 <= d <= 6)) * 64
    assert bench.mufu_per_frame_iter(qc) == want
