"""GPU parity: the CUDA decoder (through the C ABI) against the FP64 oracle.

Messages over the first 10 iterations agree to 1e-4 relative + 1e-5 absolute;
decisions (bits, success/abort flags, iteration counts) agree on every frame,
with FP32 mismatches re-run in the decoder's FP64 mode, which must then agree
exactly.  Sizes span several tiles with a ragged tail (QC tiles are 1024
checks or variables of one base row / column).
"""
import numpy as np
import pytest

from paper_2507_03509_gb300 import gen
from _decode_helpers import (Q_LOG, TOL, assert_close_messages, check_decisions, gpu_decode, lib,
                             mismatched_frames, RULE_IDS)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ldpc():
    return lib()


@pytest.fixture(scope="module")
def oracle(oracle_mod):
    return oracle_mod


@pytest.fixture(scope="module")
def csr1():
    return gen.workload_code(1)


@pytest.fixture(scope="module")
def qc_small():
    # the n = 1e6 base matrix lifted with Z = 2600: 3 tiles per base column,
    # the last one ragged (2600 = 2*1024 + 552)
    return gen.workload_code(2, Z=2600)


def test_trace_messages_csr(ldpc, oracle, csr1):
    g = ldpc.Graph.from_code(csr1)
    fr = gen.workload_frames(1, csr1, frames=8)
    for rule in ("none", "pce_vnr"):
        orc = oracle.decode(csr1, fr.llr, fr.syndrome, 10, RULE_IDS[rule], trace_iters=10)
        got = gpu_decode(ldpc, g, fr.llr, fr.syndrome, 10, rule, trace_iters=10)
        assert_close_messages(got["c2v"], orc["c2v"], "c2v")
        assert_close_messages(got["app"], orc["app"], "app")
        np.testing.assert_allclose(got["q"][~np.isnan(orc["q"])], orc["q"][~np.isnan(orc["q"])], rtol=1e-5)


def test_trace_messages_qc(ldpc, oracle, qc_small):
    g = ldpc.Graph.from_code(qc_small)
    csr = qc_small.to_csr()
    fr = gen.workload_frames(2, qc_small, frames=4)
    orc = oracle.decode(csr, fr.llr, fr.syndrome, 10, 0, trace_iters=10)
    got = gpu_decode(ldpc, g, fr.llr, fr.syndrome, 10, "none", trace_iters=10)
    assert_close_messages(got["c2v"], orc["c2v"], "c2v")
    assert_close_messages(got["app"], orc["app"], "app")
    np.testing.assert_allclose(got["q"], orc["q"], rtol=1e-5)


@pytest.mark.parametrize("case", ["csr_n4096", "qc_z2600", "reg36_z64"])
def test_q_trace_within_tie_band(ldpc, oracle, csr1, qc_small, case):
    """q^(k) of the FP32 decoder (FP64 sums of FP32 APP values) against the
    oracle's FP64 q, rule NONE.  A VNR decision can only differ from the
    oracle's where the oracle's own step q^(k) - q^(k-1) is within the two
    iterations' q differences, so the near-tie band rtol_q of the decision
    checks must be at least twice the largest relative difference; the test
    holds the difference to half the band over the first 20 iterations and
    records it over 60 (unconverged frames drift apart later, A25)."""
    import torch
    if case == "csr_n4096":
        code, fr = csr1, gen.workload_frames(1, csr1, frames=16)
    elif case == "qc_z2600":
        code, fr = qc_small, gen.workload_frames(2, qc_small, frames=4)
    else:
        code = gen.workload_code(6, Z=64)
        fr = gen.workload_frames(6, code, frames=16, beta=0.8)
    K = 60
    csr = code.to_csr() if hasattr(code, "to_csr") else code
    orc = oracle.decode(csr, fr.llr, fr.syndrome, K, 0, trace_iters=K, trace=("q",))
    g = ldpc.Graph.from_code(code)
    dev = torch.device("cuda:0")
    tq = torch.full((K, fr.llr.shape[0]), float("nan"), dtype=torch.float64, device=dev)
    ldpc.decode(g, torch.from_numpy(fr.llr).to(dev), torch.from_numpy(fr.syndrome).to(dev), K, "none",
                trace_iters=K, trace_q=tq)
    torch.cuda.synchronize()
    q = tq.cpu().numpy()
    rel = np.abs(q - orc["q"]) / np.abs(orc["q"])
    Q_LOG.append(dict(case=case, max_rel=float(rel[:20].max()), iters=20, rtol_q=TOL["fp32"]["rtol_q"]))
    Q_LOG.append(dict(case=case, max_rel=float(rel.max()), iters=K, rtol_q=TOL["fp32"]["rtol_q"]))
    assert rel[:20].max() <= 0.5 * TOL["fp32"]["rtol_q"], f"max relative q difference {rel[:20].max():.3g}"
    g.close()


@pytest.mark.parametrize("rule", ["pce_vnr", "pce", "none"])
def test_decisions_csr_full_workload(ldpc, oracle, csr1, rule):
    """n = 4096 random code, all 64 frames, max 200 iterations."""
    g = ldpc.Graph.from_code(csr1)
    fr = gen.workload_frames(1, csr1)
    check_decisions(ldpc, g, csr1, oracle, fr.llr, fr.syndrome, 200, rule)


@pytest.mark.parametrize("rule", ["pce_vnr", "pce"])
def test_decisions_qc(ldpc, oracle, qc_small, rule):
    g = ldpc.Graph.from_code(qc_small)
    fr = gen.workload_frames(2, qc_small, frames=12)
    check_decisions(ldpc, g, qc_small.to_csr(), oracle, fr.llr, fr.syndrome, 60, rule)


def test_decisions_decodable_regime(ldpc, oracle):
    """A rate-1/2 code at a noise level where most frames decode, so PCE-ET
    successes (not only aborts and D_max) are exercised."""
    code = gen.random_csr_code(2000, 1000, 3, {6: 1000}, seed=4242)
    g = ldpc.Graph.from_code(code)
    fr = gen.make_frames(code, np.full(48, 0.75), seeds=range(7000, 7048))
    for rule in ("pce_vnr", "pce", "none"):
        bad, got, orc = check_decisions(ldpc, g, code, oracle, fr.llr, fr.syndrome, 80, rule)
        assert (got["flags"] & 1).sum() >= 24


def test_fp64_mode_follows_oracle(ldpc, oracle, csr1, qc_small):
    for code, F in ((csr1, 6), (qc_small, 2)):
        csr = code.to_csr() if hasattr(code, "to_csr") else code
        g = ldpc.Graph.from_code(code)
        fr = gen.workload_frames(1 if code is csr1 else 2, code, frames=F)
        orc = oracle.decode(csr, fr.llr, fr.syndrome, 40, 2, trace_iters=10)
        got = gpu_decode(ldpc, g, fr.llr, fr.syndrome, 40, "pce_vnr", trace_iters=10, fp64=True)
        ran = ~np.isnan(orc["c2v"])
        np.testing.assert_allclose(got["c2v"][ran], orc["c2v"][ran], rtol=1e-11, atol=1e-11)
        ran = ~np.isnan(orc["app"])
        np.testing.assert_allclose(got["app"][ran], orc["app"][ran], rtol=1e-11, atol=1e-11)
        assert mismatched_frames(got, orc).size == 0


@pytest.mark.parametrize("fp64", [False, True])
def test_sign_symmetry_bit_exact(ldpc, csr1, qc_small, fp64):
    """decode(Lch*(1-2u), s xor Hu) = decode(Lch, s) with bits xor u, equal
    flags and iteration counts, and messages equal up to the edge signs."""
    rng = np.random.default_rng(11)
    for code, wl in ((csr1, 1), (qc_small, 2)):
        csr = code.to_csr() if hasattr(code, "to_csr") else code
        g = ldpc.Graph.from_code(code)
        fr = gen.workload_frames(wl, code, frames=4)
        u = rng.integers(0, 2, size=fr.x.shape).astype(np.uint8)
        llr2 = (fr.llr * (1 - 2 * u.astype(np.float32))).astype(np.float32)
        s2 = fr.syndrome ^ gen.syndrome(code, u)
        a = gpu_decode(ldpc, g, fr.llr, fr.syndrome, 30, "pce_vnr", trace_iters=4, fp64=fp64)
        b = gpu_decode(ldpc, g, llr2, s2, 30, "pce_vnr", trace_iters=4, fp64=fp64)
        assert (b["bits"] == (a["bits"] ^ u)).all()
        assert (a["flags"] == b["flags"]).all() and (a["iters"] == b["iters"]).all()
        ue = (1 - 2 * u[:, csr.colidx].astype(np.float64))[None]
        ran = ~np.isnan(a["c2v"])
        assert (b["c2v"][ran] == (a["c2v"] * ue)[ran]).all()
        assert (b["app"] == a["app"] * (1 - 2 * u.astype(np.float64))[None])[~np.isnan(a["app"])].all()
        assert np.array_equal(a["q"], b["q"], equal_nan=True)


def test_success_means_zero_syndrome(ldpc):
    code = gen.random_csr_code(2000, 1000, 3, {6: 1000}, seed=4242)
    g = ldpc.Graph.from_code(code)
    fr = gen.make_frames(code, np.full(32, 0.8), seeds=range(100, 132))
    for rule in ("pce", "pce_vnr", "none"):
        got = gpu_decode(ldpc, g, fr.llr, fr.syndrome, 60, rule)
        ok = (gen.syndrome(code, got["bits"]) == fr.syndrome).all(1)
        assert (ok == ((got["flags"] & 1) > 0)).all()
        assert ok.sum() > 0


def test_noise_free_limit(ldpc, csr1, qc_small):
    rng = np.random.default_rng(5)
    for code in (csr1, qc_small):
        g = ldpc.Graph.from_code(code)
        x = rng.integers(0, 2, size=(3, code.n)).astype(np.uint8)
        llr = (30.0 * (1.0 - 2.0 * x)).astype(np.float32)
        s = gen.syndrome(code, x)
        got = gpu_decode(ldpc, g, llr, s, 25, "pce_vnr")
        assert (got["iters"] == 1).all() and (got["flags"] == 1).all() and (got["bits"] == x).all()


def test_groups_concurrency_and_grid_do_not_change_results(ldpc, csr1, qc_small):
    """Any number of CTA groups, slots (queue + refill) and CTAs gives
    bit-identical results and traces."""
    for code, wl in ((csr1, 1), (qc_small, 2)):
        g = ldpc.Graph.from_code(code)
        fr = gen.workload_frames(wl, code, frames=9)
        ref = gpu_decode(ldpc, g, fr.llr, fr.syndrome, 40, "pce_vnr", trace_iters=3, groups=1,
                         max_active_frames=9, schedule="lockstep")
        for slots, ctas, groups in ((0, 0, 0), (3, 0, 1), (3, 0, 3), (1, 0, 0), (9, 1, 0), (9, 0, 4),
                                    (4, 7, 0), (8, 0, 2), (0, 0, 8)):
            got = gpu_decode(ldpc, g, fr.llr, fr.syndrome, 40, "pce_vnr", trace_iters=3,
                             max_active_frames=slots, grid_ctas=ctas, groups=groups, schedule="lockstep")
            for key in ("bits", "flags", "iters"):
                assert np.array_equal(got[key], ref[key]), (slots, ctas, groups, key)
            for key in ("c2v", "app", "q"):
                assert np.array_equal(got[key], ref[key], equal_nan=True), (slots, ctas, groups, key)
            assert got["stats"].active_frames >= max(1, slots)


def test_degenerate_graph_shapes(ldpc, oracle):
    """Degree-0 and degree-1 checks, a variable in no check, a degree-7 check."""
    rows = [[0], [0, 1], [1, 2, 3], [], [2, 4, 5, 6, 7, 8, 9, 10], [3, 4], [5, 11]]
    rowptr = np.cumsum([0] + [len(r) for r in rows]).astype(np.int32)
    code = gen.CSRCode(len(rows), 13, rowptr, np.concatenate([np.asarray(r, np.int32) for r in rows]))
    g = ldpc.Graph.from_code(code)
    rng = np.random.default_rng(2)
    x = rng.integers(0, 2, size=(20, code.n)).astype(np.uint8)
    llr = ((1.0 - 2.0 * x) + 1.1 * rng.standard_normal(x.shape)).astype(np.float32) * 1.3
    s = gen.syndrome(code, x)
    for rule in ("pce_vnr", "pce", "none"):
        check_decisions(ldpc, g, code, oracle, llr, s, 15, rule)
    orc = oracle.decode(code, llr, s, 6, 0, trace_iters=6)
    got = gpu_decode(ldpc, g, llr, s, 6, "none", trace_iters=6)
    assert_close_messages(got["c2v"], orc["c2v"], "c2v")
    assert_close_messages(got["app"], orc["app"], "app")


def test_degenerate_qc_shapes(ldpc, oracle):
    """A base row with no block, a weight-1 row, weight-1 columns, a weight-7 row."""
    sh = -np.ones((4, 9), np.int32)
    sh[1, 0] = 3
    sh[2, [0, 1, 2]] = [0, 5, 9]
    sh[3, 2:9] = [1, 2, 3, 4, 5, 6, 7]
    code = gen.QCCode(4, 9, 11, sh)
    g = ldpc.Graph.from_code(code)
    rng = np.random.default_rng(3)
    x = rng.integers(0, 2, size=(40, code.n)).astype(np.uint8)
    llr = ((1.0 - 2.0 * x) + 0.9 * rng.standard_normal(x.shape)).astype(np.float32) * 2.0
    s = gen.syndrome(code, x)
    orc = oracle.decode(code.to_csr(), llr, s, 10, 0, trace_iters=10)
    got = gpu_decode(ldpc, g, llr, s, 10, "none", trace_iters=10)
    assert_close_messages(got["c2v"], orc["c2v"], "c2v")
    assert_close_messages(got["app"], orc["app"], "app")
    # Nearly a forest: every frame reaches an exact fixed point within three
    # iterations, after which q is flat in exact arithmetic, so each VNR test is
    # a tie (A5) that FP32 rounding may break either way.  Every such frame
    # still has to pass the trajectory check and agree exactly in FP64.
    for rule in ("pce_vnr", "pce"):
        check_decisions(ldpc, g, code.to_csr(), oracle, llr, s, 12, rule, fp32_escape_frac=1.0)


@pytest.mark.parametrize("opts", [dict(vnr_first_iter=1), dict(clamp=8.0), dict(vnr_first_iter=4)])
def test_options_follow_oracle(ldpc, oracle, csr1, opts):
    g = ldpc.Graph.from_code(csr1)
    fr = gen.workload_frames(1, csr1, frames=24)
    check_decisions(ldpc, g, csr1, oracle, fr.llr, fr.syndrome, 100, "pce_vnr", **opts)


def test_single_iteration_and_single_frame(ldpc, oracle, qc_small):
    g = ldpc.Graph.from_code(qc_small)
    fr = gen.workload_frames(2, qc_small, frames=1)
    for rule in ("none", "pce", "pce_vnr"):
        check_decisions(ldpc, g, qc_small.to_csr(), oracle, fr.llr, fr.syndrome, 1, rule)


def test_zero_frames_and_errors(ldpc, csr1):
    import torch
    g = ldpc.Graph.from_code(csr1)
    dev = torch.device("cuda:0")
    e = torch.empty((0, csr1.n), dtype=torch.float32, device=dev)
    s = torch.empty((0, csr1.m), dtype=torch.uint8, device=dev)
    bits, flags, iters = ldpc.decode(g, e, s, 10, "pce_vnr")
    assert bits.shape == (0, csr1.n)
    fr = gen.workload_frames(1, csr1, frames=2)
    llr = torch.from_numpy(fr.llr).to(dev)
    syn = torch.from_numpy(fr.syndrome).to(dev)
    bad = syn.clone()
    bad[1, 17] = 2
    with pytest.raises(ldpc.LdpcError) as ei:
        ldpc.decode(g, llr, bad, 10, "pce_vnr")
    assert ei.value.status == ldpc.LDPC_ERR_INVALID_ARG
    with pytest.raises(ldpc.LdpcError):
        ldpc.decode(g, llr, syn, 0, "pce_vnr")
    out = ldpc.decode(g, llr, syn, 10, "pce_vnr")  # the context is still usable
    assert out[2].min().item() >= 1


def test_host_entry_point_matches_device(ldpc, qc_small):
    g = ldpc.Graph.from_code(qc_small)
    fr = gen.workload_frames(2, qc_small, frames=5)
    dev = gpu_decode(ldpc, g, fr.llr, fr.syndrome, 30, "pce_vnr")
    bits, flags, iters = ldpc.decode_host(g, fr.llr, fr.syndrome, 30, "pce_vnr")
    assert (bits == dev["bits"]).all() and (flags == dev["flags"]).all() and (iters == dev["iters"]).all()


@pytest.mark.parametrize("groups", [1, 0])
def test_expired_grid_wait_returns_timeout_and_context_survives(ldpc, qc_small, groups):
    """Failure detection without a fault: the test hook makes the first
    barrier of every group wait for one CTA more than the group has (nothing
    ever arrives), so the waits run out after 200 ms; the call returns
    LDPC_ERR_TIMEOUT and the next decode on the same context works."""
    import time
    import torch
    g = ldpc.Graph.from_code(qc_small)
    fr = gen.workload_frames(2, qc_small, frames=3)
    dev = torch.device("cuda:0")
    llr = torch.from_numpy(fr.llr).to(dev)
    syn = torch.from_numpy(fr.syndrome).to(dev)
    t0 = time.perf_counter()
    with pytest.raises(ldpc.LdpcError) as ei:
        ldpc.decode(g, llr, syn, 20, "pce_vnr", barrier_timeout_ms=200, test_unreachable_barrier=True,
                    groups=groups)
    assert ei.value.status == ldpc.LDPC_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 30.0
    bits, flags, iters = ldpc.decode(g, llr, syn, 20, "pce_vnr", groups=groups)
    ref = gpu_decode(ldpc, g, fr.llr, fr.syndrome, 20, "pce_vnr")
    assert (iters.cpu().numpy() == ref["iters"]).all() and (bits.cpu().numpy() == ref["bits"]).all()


def test_regular_36_qc_code_in_its_waterfall(ldpc, oracle):
    """The (3,6)-regular QC family of the beta sweep (weight-6 rows, weight-3
    columns), at a noise level inside its BP waterfall: successes, VNR aborts
    and D_max all occur; decisions and messages follow the oracle."""
    code = gen.workload_code(6, Z=200)
    g = ldpc.Graph.from_code(code)
    csr = code.to_csr()
    fr = gen.workload_frames(6, code, frames=48, beta=0.87)
    orc = oracle.decode(csr, fr.llr[:4], fr.syndrome[:4], 10, 0, trace_iters=10)
    got = gpu_decode(ldpc, g, fr.llr[:4], fr.syndrome[:4], 10, "none", trace_iters=10)
    assert_close_messages(got["c2v"], orc["c2v"], "c2v")
    assert_close_messages(got["app"], orc["app"], "app")
    seen = set()
    for rule in ("pce_vnr", "pce"):
        bad, res, _ = check_decisions(ldpc, g, csr, oracle, fr.llr, fr.syndrome, 200, rule)
        seen |= {int(x) for x in res["flags"]}
    assert {0, 1, 2} <= seen
