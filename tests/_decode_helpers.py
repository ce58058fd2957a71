"""Helpers shared by the GPU tests: run the CUDA decoder through the C ABI and
the FP64 oracle on the same seeded inputs, and compare what the decoding fixes.

Tolerances: per-edge messages and APP values agree to 1e-4 relative plus
1e-5 absolute over the first 10 iterations; decisions (bits, flags,
iterations) agree on every frame, and a frame whose FP32 decisions differ is
re-run in the decoder's FP64 mode, which must agree with the oracle exactly.
"""
import numpy as np

RTOL, ATOL = 1e-4, 1e-5


def lib():
    from paper_2507_03509_gb300 import build
    build.build()
    from paper_2507_03509_gb300 import ldpc
    return ldpc


def gpu_decode(ldpc, graph, llr, syn, max_iter, rule, trace_iters=0, fp64=False, **opts):
    """Decode numpy inputs on cuda:0; returns numpy outputs (+ traces)."""
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
    bits, flags, iters = ldpc.decode(graph, t_llr, t_syn, max_iter, rule, fp64=fp64, trace_iters=trace_iters,
                                     trace_c2v=tc, trace_app=ta, trace_q=tq, stats=stats, **opts)
    torch.cuda.synchronize()
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


def check_decisions(ldpc, graph, code_csr, oracle, llr, syn, max_iter, rule, report=None,
                    max_mismatch_frac=0.1, **opts):
    """FP32 GPU decisions vs oracle on every frame; mismatches re-run in FP64
    on the GPU must then agree exactly.  Near-ties (a q step or an APP value
    within FP32 rounding of zero) are the only accepted cause, so at most
    max_mismatch_frac of the frames may need the re-run.  Returns the list of
    frames that needed it."""
    orc = oracle.decode(code_csr, llr, syn, max_iter, RULE_IDS[rule],
                        vnr_first_iter=opts.get("vnr_first_iter", 2), lmax=opts.get("clamp", 25.0))
    got = gpu_decode(ldpc, graph, llr, syn, max_iter, rule, **opts)
    bad = mismatched_frames(got, orc)
    assert bad.size <= max(1, int(max_mismatch_frac * llr.shape[0])), \
        f"FP32 decisions differ on {bad.size} of {llr.shape[0]} frames: {bad.tolist()}"
    if bad.size:
        g64 = gpu_decode(ldpc, graph, llr[bad], syn[bad], max_iter, rule, fp64=True, **opts)
        sub = {k: orc[k][bad] for k in ("bits", "flags", "iters")}
        still = mismatched_frames(g64, sub)
        assert still.size == 0, f"FP64 re-run still differs on frames {bad[still].tolist()}"
    if report is not None:
        report.append(dict(rule=rule, frames=int(llr.shape[0]), fp32_mismatch=bad.tolist()))
    return bad.tolist(), got, orc
