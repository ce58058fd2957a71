"""Helpers shared by the GPU tests: run the CUDA decoder through the C ABI and
the FP64 oracle on the same seeded inputs, and compare what the decoding fixes.

Tolerances: per-edge messages and APP values agree to 1e-4 relative plus
1e-5 absolute over the first 10 iterations; decisions (bits, flags,
iterations) agree on every frame, and a frame whose FP32 decisions differ is
re-run in the decoder's FP64 mode, which must agree with the oracle exactly.

How many frames may take either way out is capped per call (FP32_ESCAPE_FRAC,
FP64_TIE_FRAC), and every call's counts are kept in PARITY_LOG, which the
test session prints at its end.
"""
import os

import numpy as np

RTOL, ATOL = 1e-4, 1e-5

# At most this fraction of a call's frames (at least one frame) may differ in
# FP32 and be accepted through the FP64 re-run and the trajectory check ...
FP32_ESCAPE_FRAC = 0.10
# ... and at most this fraction (at least one frame) may still differ in the
# FP64 re-run and be accepted as an FP64-level near-tie of the trajectory.
# Such frames reached a fixed point that is not a codeword: q then rises by
# geometrically shrinking steps, and the VNR test stops the frame once a step
# falls below FP64 rounding noise, at an iteration that the summation order
# decides.  The most seen is 2 of the 64 frames of the n = 4096 workload.
FP64_TIE_FRAC = 0.05

# One entry per decision comparison of the session: test, rule, frames, the
# frames that differed in FP32 and those accepted as FP64 near-ties.
PARITY_LOG = []


# Largest relative difference |q_gpu - q_oracle| / q_oracle seen per traced
# comparison (test_q_trace_within_tie_band), printed at the session's end.
Q_LOG = []


def escape_caps(frames, fp32_escape_frac=FP32_ESCAPE_FRAC):
    """(FP32 escapes, FP64 near-ties) allowed for a comparison of `frames` frames."""
    return max(1, int(fp32_escape_frac * frames)), max(1, int(FP64_TIE_FRAC * frames))


def log_parity(rule, frames, fp32_mismatch, fp64_ties):
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    PARITY_LOG.append(dict(test=test, rule=rule, frames=int(frames), fp32_mismatch=[int(f) for f in fp32_mismatch],
                           fp64_ties=[int(f) for f in fp64_ties]))


def lib():
    from paper_2507_03509_gb300 import build
    build.build()
    from paper_2507_03509_gb300 import ldpc
    return ldpc


def gpu_decode(ldpc, graph, llr, syn, max_iter, rule, trace_iters=0, fp64=False, **opts):
    """Decode numpy inputs on cuda:0; returns numpy outputs (+ traces).  The
    decode places guard words around its workspace arrays (debug_guards) and
    the guards are checked afterwards, unless debug_guards=False is passed."""
    import torch
    dev = torch.device("cuda:0")
    F = llr.shape[0]
    t_llr = torch.from_numpy(np.ascontiguousarray(llr)).to(dev)
    t_syn = torch.from_numpy(np.ascontiguousarray(syn)).to(dev)
    dt = torch.float64 if fp64 else torch.float32
    tc = ta = tq = None
    if trace_iters:
        tc = torch.full((trace_iters, F, graph.edges), float("nan"), dtype=dt, device=dev)
        ta = torch.full((trace_iters, F, graph.n), float("nan"), dtype=dt, device=dev)
        tq = torch.full((trace_iters, F), float("nan"), dtype=torch.float64, device=dev)
    stats = ldpc.ldpc_decode_stats()
    opts.setdefault("debug_guards", True)
    bits, flags, iters = ldpc.decode(graph, t_llr, t_syn, max_iter, rule, fp64=fp64, trace_iters=trace_iters,
                                     trace_c2v=tc, trace_app=ta, trace_q=tq, stats=stats, **opts)
    torch.cuda.synchronize()
    if opts["debug_guards"]:  # the decode wrote nothing outside its workspace arrays
        st = ldpc.ldpc_graph_check_guards(graph.handle)
        assert st == ldpc.LDPC_OK, ldpc.ldpc_status_str(st)
    out = dict(bits=bits.cpu().numpy(), flags=flags.cpu().numpy(), iters=iters.cpu().numpy(), stats=stats)
    if trace_iters:
        out.update(c2v=tc.cpu().numpy().astype(np.float64), app=ta.cpu().numpy().astype(np.float64),
                   q=tq.cpu().numpy())
    return out


def assert_close_messages(got, want, what):
    ran = ~np.isnan(want)
    assert np.array_equal(ran, ~np.isnan(got)), f"{what}: iterations run differ"
    g, w = got[ran], want[ran]
    err = np.abs(g - w)
    tol = ATOL + RTOL * np.abs(w)
    bad = err > tol
    assert not bad.any(), (f"{what}: {bad.sum()} of {bad.size} values out of tolerance; "
                           f"worst |d|={err.max():.3g}, worst ratio={np.max(err / tol):.3g}")
    return float(np.max(err / tol)) if err.size else 0.0


def mismatched_frames(a, b):
    return np.nonzero((a["iters"] != b["iters"]) | (a["flags"] != b["flags"])
                      | (a["bits"] != b["bits"]).any(axis=1))[0]


RULE_IDS = {"none": 0, "pce": 1, "pce_vnr": 2}

# Rounding levels: a q step |q(k) - q(k-1)| at most RTOL_Q * q, or an APP
# value within ATOL_APP of zero, is a near-tie whose outcome the arithmetic
# does not fix.
TOL = {"fp32": dict(rtol_q=2e-6, atol_app=1e-3), "fp64": dict(rtol_q=1e-11, atol_app=1e-9)}


def decision_is_input_sensitive(oracle, code, llr_f, syn_f, D, bits, kw, tries=3):
    """Whether the oracle's own decision after D iterations changes when one
    channel value moves by one float32 ulp.  A frame that never converges
    follows a chaotic trajectory on a loopy graph; once its decision depends
    on the inputs below their own precision, the bits of that failed frame are
    not a unique result, and two arithmetics may end on different ones."""
    free = np.nonzero(np.abs(llr_f) < 50.0)[0]  # not shortened
    free = free[llr_f[free] != 0.0]             # not punctured
    for v in free[:: max(1, free.size // tries)][:tries]:
        pert = llr_f.copy()
        pert[v] = np.nextafter(pert[v], np.float32(np.inf))
        alt = oracle.decode(code, pert[None], syn_f[None], D, 0, **kw)["bits"][0]
        if (alt != bits).any():
            return True
    return False


def validate_trajectory(oracle, code, llr_f, syn_f, res, orc, max_iter, rule, precision,
                        vnr_first_iter=2, clamp=25.0):
    """Check one frame's decoder result against the oracle's own trajectory.

    Returns a list of problems (empty when the result is valid): the bits must
    be the oracle's hard decision at the decoder's stopping iteration D (up to
    APP near-ties, or, for a frame both sides ran to D_max without success or
    abort, unless the oracle's own decision there moves with a one-ulp change
    of one channel value); success must mean H x^ = s; every termination test the
    decoder passed or took must agree with the oracle's q and decisions up to
    near-ties (a VNR step within rounding, a PCE success hanging on an APP
    near-tie)."""
    from paper_2507_03509_gb300 import gen
    tol = TOL[precision]
    rid = RULE_IDS[rule]
    D, Do = int(res["iters"]), int(orc["iters"])
    fl, flo = int(res["flags"]), int(orc["flags"])
    K = max(D, Do)
    kw = dict(vnr_first_iter=vnr_first_iter, lmax=clamp)
    tr = oracle.decode(code, llr_f[None], syn_f[None], K, 0, trace_iters=K, trace=("q",), **kw)
    q = tr["q"][:, 0]
    deg = np.bincount(code.colidx, minlength=code.n)
    q0 = float(np.abs(llr_f.astype(np.float64))[deg > 1].sum())
    at = oracle.decode(code, llr_f[None], syn_f[None], D, 0, final_app=True, **kw)
    app, xo = at["app_final"][0], at["bits"][0]
    probs = []
    diff = res["bits"] != xo
    if diff.any() and np.abs(app[diff]).max() > tol["atol_app"]:
        unconverged = D == Do == max_iter and fl == flo == 0
        if not (unconverged and decision_is_input_sensitive(oracle, code, llr_f, syn_f, D, xo, kw)):
            probs.append(f"{int(diff.sum())} bits differ from the oracle's decision at k={D}, "
                         f"max |APP| there {np.abs(app[diff]).max():.3g}")
    synd_ok = bool((gen.syndrome(code, res["bits"]) == syn_f).all())
    if bool(fl & 1) != synd_ok:
        probs.append("success flag disagrees with H x^ = s")

    def step(k):
        prev = q[k - 2] if k >= 2 else q0
        return q[k - 1] - prev

    def tie(k):
        return abs(step(k)) <= tol["rtol_q"] * abs(q[k - 1])

    if rid == 0 and D != max_iter:
        probs.append("rule none stopped early")
    if fl & 2:
        if not (rid == 2 and D >= vnr_first_iter and (step(D) < 0 or tie(D))):
            probs.append(f"VNR abort at k={D} without a drop of q (step {step(D):.3g})")
    if rid == 2:
        for k in range(vnr_first_iter, D):
            if step(k) < 0 and not tie(k):
                probs.append(f"q fell clearly at k={k} (step {step(k):.3g}) but decoding went on")
                break
    if rid in (1, 2) and Do < D and (flo & 1):
        ao = oracle.decode(code, llr_f[None], syn_f[None], Do, 0, final_app=True, **kw)["app_final"][0]
        if np.abs(ao).min() > tol["atol_app"]:
            probs.append(f"oracle met the syndrome at k={Do} with no APP near-tie, decoder went on")
    if rid in (1, 2) and not (fl & 1) and D < max_iter and not (fl & 2):
        probs.append("stopped without success, abort or D_max")
    return probs


def check_decisions(ldpc, graph, code_csr, oracle, llr, syn, max_iter, rule, report=None,
                    fp32_escape_frac=FP32_ESCAPE_FRAC, **opts):
    """FP32 GPU decisions vs the oracle on every frame.

    Frames that differ are re-run in the decoder's FP64 mode, which must agree
    with the oracle exactly -- or, where the FP64 decision itself hangs on a
    near-tie at FP64 rounding level, pass validate_trajectory at FP64
    tolerance.  The FP32 result of every differing frame must pass
    validate_trajectory at FP32 tolerance (so no difference is accepted unless
    the oracle's own trajectory shows a near-tie there).  escape_caps() bounds
    how many frames may take each way out.  FP32 differences are mostly VNR
    aborts on frames that reached a fixed point: there the FP64 q stays flat (a
    tie, decoding goes on) while the FP32 q moves by rounding and may fall.
    Returns (differing frames, gpu result, oracle result)."""
    kw = dict(vnr_first_iter=opts.get("vnr_first_iter", 2), clamp=opts.get("clamp", 25.0))
    orc = oracle.decode(code_csr, llr, syn, max_iter, RULE_IDS[rule], vnr_first_iter=kw["vnr_first_iter"],
                        lmax=kw["clamp"])
    got = gpu_decode(ldpc, graph, llr, syn, max_iter, rule, **opts)
    bad = mismatched_frames(got, orc)
    cap32, cap64 = escape_caps(llr.shape[0], fp32_escape_frac)
    assert bad.size <= cap32, \
        (f"FP32 decisions differ on {bad.size} of {llr.shape[0]} frames: "
         + "; ".join(f"f{f}: gpu D={got['iters'][f]} fl={got['flags'][f]} / oracle D={orc['iters'][f]} "
                     f"fl={orc['flags'][f]}, {(got['bits'][f] != orc['bits'][f]).sum()} bits" for f in bad))
    fp64_ties = []
    if bad.size:
        g64 = gpu_decode(ldpc, graph, llr[bad], syn[bad], max_iter, rule, fp64=True, **opts)
        for i, f in enumerate(bad):
            one = lambda r, j: {k: r[k][j] for k in ("bits", "flags", "iters")}
            o = one(orc, f)
            p32 = validate_trajectory(oracle, code_csr, llr[f], syn[f], one(got, f), o, max_iter, rule, "fp32", **kw)
            assert not p32, f"frame {f} (FP32): {p32}"
            r64 = one(g64, i)
            if mismatched_frames({k: v[None] for k, v in r64.items()}, {k: v[None] for k, v in o.items()}).size:
                p64 = validate_trajectory(oracle, code_csr, llr[f], syn[f], r64, o, max_iter, rule, "fp64", **kw)
                assert not p64, f"frame {f} (FP64 re-run): {p64}"
                fp64_ties.append(int(f))
    log_parity(rule, llr.shape[0], bad, fp64_ties)
    assert len(fp64_ties) <= cap64, f"{len(fp64_ties)} frames hang on FP64 near-ties: {fp64_ties}"
    if report is not None:
        report.append(dict(rule=rule, frames=int(llr.shape[0]), fp32_mismatch=bad.tolist(), fp64_ties=fp64_ties))
    return bad.tolist(), got, orc
