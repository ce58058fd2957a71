"""Input-generator checks: channel capacity pins, code structure, syndromes."""
import math
import os

import numpy as np
import pytest

from paper_2507_03509_gb300 import gen

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "biawgn_limits.txt")


def _golden_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            r, ebn0, tol, src = line.split()
            rows.append((float(r), float(ebn0), float(tol), src))
    return rows


@pytest.mark.parametrize("rate,ebn0_db,tol,src", _golden_rows())
def test_shannon_limits(rate, ebn0_db, tol, src):
    """sigma at C = R reproduces the textbook Eb/N0 limit (Eb/N0 = 1/(2 R sigma^2))."""
    sigma = gen.sigma_for_capacity(rate)
    ebn0 = 10 * math.log10(1.0 / (2.0 * rate * sigma * sigma))
    assert abs(ebn0 - ebn0_db) < tol, (src, ebn0)


def test_capacity_low_snr_slope():
    """For small SNR = 1/sigma^2, C ~ SNR / (2 ln 2)."""
    for sigma in (20.0, 40.0):
        snr = 1.0 / sigma ** 2
        assert gen.biawgn_capacity(sigma) == pytest.approx(snr / (2 * math.log(2)), rel=3e-3)


def test_capacity_quadrature_matches_adaptive_integration():
    from scipy.integrate import quad
    for sigma in (0.8, 2.449867, 5.748478):
        f = lambda y: (math.exp(-(y - 1) ** 2 / (2 * sigma * sigma)) / math.sqrt(2 * math.pi * sigma * sigma)
                       * math.log2(1 + math.exp(-2 * y / sigma ** 2)))
        ref = 1 - quad(f, 1 - 40 * sigma, 1 + 40 * sigma, limit=400)[0]
        assert gen.biawgn_capacity(sigma) == pytest.approx(ref, abs=1e-10)


def test_workload1_code_structure():
    c = gen.workload_code(1)
    assert (c.m, c.n) == (3686, 4096)
    assert c.edges <= 12288 and c.edges > 12200  # duplicates collapsed
    assert np.all(np.diff(c.rowptr) >= 1)
    for r in range(c.m):
        cols = c.colidx[c.rowptr[r]:c.rowptr[r + 1]]
        assert np.all(np.diff(cols) > 0)


def test_workload2_base_matrix_margins():
    q = gen.workload_code(2, Z=64)
    B = q.shifts >= 0
    assert B.shape == (49, 50)
    assert sorted(np.bincount(B.sum(0))[2:].tolist()) == [25, 25]
    assert np.bincount(B.sum(1)).tolist()[2:] == [22, 27]
    assert q.shifts.max() < 64 and q.shifts[B].min() >= 0
    full = gen.workload_code(2)
    assert (full.n, full.m, full.edges) == (1_000_000, 980_000, 2_500_000)
    assert ((full.shifts >= 0) == B).all()


def test_qc_lift_and_syndrome_match_dense():
    q = gen.random_qc_code(3, 5, 7, [2, 1, 3, 2, 2], seed=5)
    csr = q.to_csr()
    H = np.zeros((q.m, q.n), dtype=np.int64)
    for i in range(q.mb):
        for j in range(q.nb):
            s = q.shifts[i, j]
            if s >= 0:
                for t in range(q.Z):
                    H[i * q.Z + t, j * q.Z + (t + s) % q.Z] = 1
    Hc = np.zeros_like(H)
    for r in range(csr.m):
        Hc[r, csr.colidx[csr.rowptr[r]:csr.rowptr[r + 1]]] = 1
    assert (H == Hc).all()
    x = np.random.default_rng(1).integers(0, 2, size=(3, q.n)).astype(np.uint8)
    want = (x.astype(np.int64) @ H.T) % 2
    assert (gen.syndrome(q, x) == want).all()
    assert (gen.syndrome(csr, x) == want).all()


def test_frames_reproducible_and_llr_convention():
    c = gen.workload_code(1)
    a = gen.workload_frames(1, c, frames=2)
    b = gen.workload_frames(1, c, frames=1, first=1)
    assert (a.llr[1] == b.llr[0]).all() and (a.x[1] == b.x[0]).all()
    # LLR = 2y/sigma^2 with y = 1-2x + noise: sign agrees with 1-2x on most bits
    agree = ((a.llr > 0) == (a.x == 0)).mean()
    assert 0.6 < agree < 0.8
    assert a.sigma[0] == pytest.approx(2.449867, abs=2e-6)


def test_batch_workload_layout_and_reproducibility():
    codes = gen.batch_codes(3)
    assert [c.n for c in codes] == [65536, 262144, 1000000]
    assert [round(c.rate, 2) for c in codes] == [0.1, 0.05, 0.02]
    a = gen.workload_batch(3, codes, frames=6)
    b = gen.workload_batch(3, codes, frames=3, first=3)
    assert (a.frame_code[3:] == b.frame_code).all() and (a.beta[3:] == b.beta).all()
    assert (a.llr[a.var_off[3]:] == b.llr).all() and (a.syndrome[a.syn_off[3]:] == b.syndrome).all()
    for f in range(6):
        c = codes[a.frame_code[f]]
        assert a.var_off[f + 1] - a.var_off[f] == c.n and a.syn_off[f + 1] - a.syn_off[f] == c.m
        x = a.x[a.var_off[f]:a.var_off[f + 1]]
        assert (gen.syndrome(c, x) == a.syndrome[a.syn_off[f]:a.syn_off[f + 1]]).all()
        assert 0.85 <= a.beta[f] <= 0.97
        assert gen.biawgn_capacity(a.sigma[f]) == pytest.approx(c.rate / a.beta[f], rel=1e-9)


def test_tbp_like_code_structure():
    c = gen.tbp_like_qc_code(16)
    B = (c.shifts >= 0).astype(int)
    assert (c.mb, c.nb) == (196, 200) and abs(c.rate - 0.02) < 1e-12
    cols, rows = B.sum(0), B.sum(1)
    assert (cols[:8] == 51).all() and (cols[8:] == 1).all()          # core columns, degree-1 columns
    assert (rows[:4] == 6).all() and (rows[4:] == 3).all()           # core rows, lower rows
    assert (B[4:, 8:] == np.eye(192, dtype=int)).all()              # one degree-1 column per lower row
    assert B[:4, 8:].sum() == 0
    csr = c.to_csr()
    deg = np.bincount(csr.colidx, minlength=c.n)
    assert (deg[8 * 16:] == 1).all() and (deg[:8 * 16] == 51).all()


def test_rate_adapt_puncture_and_shorten():
    c = gen.workload_code(1)
    fr = gen.workload_frames(1, c, frames=3)
    p, sh = np.arange(0, 40), np.arange(100, 130)
    ad = gen.rate_adapt(fr, p, sh)
    assert (ad.llr[:, p] == 0).all()
    assert (ad.llr[:, sh] == gen.SHORTENED_LLR * (1 - 2 * fr.x[:, sh].astype(np.float32))).all()
    rest = np.setdiff1d(np.arange(c.n), np.concatenate([p, sh]))
    assert (ad.llr[:, rest] == fr.llr[:, rest]).all()
    assert ad.syndrome is fr.syndrome and ad.x is fr.x
    w = gen.workload_frames(7, gen.workload_code(7, Z=16), frames=2)
    assert (w.llr[:, :16] == 0).all() and (w.llr[:, 16:] != 0).all()   # core column 0 punctured
