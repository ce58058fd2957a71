"""The dataflow schedule (no grid barriers) and the frame-per-CTA schedule
(small CSR codes in shared memory) against the lock-step schedule.

Both run the same check and variable items and take the same decisions with
the same fixed-order q, so every result must be bit-identical: decided bits,
flags, iteration counts and the traced messages, APP values and q.  Cases
cover ragged item tails, frames refilled from the queue (fewer slots than
frames), every lag from 1 to the slot count, degree-0/1 rows and columns,
degree-1 variables with a punctured column, learned weights, batches of
codes with different item geometries, and the timeout path.
"""
import numpy as np
import pytest

from paper_2507_03509_gb300 import gen
from _decode_helpers import gpu_decode, lib

pytestmark = pytest.mark.gpu

KEYS = ("bits", "flags", "iters")


@pytest.fixture(scope="module")
def ldpc():
    return lib()


def same(a, b, what, traces=False):
    for key in KEYS + (("c2v", "app", "q") if traces else ()):
        assert np.array_equal(a[key], b[key], equal_nan=True), (what, key)


def degenerate_qc():
    sh = -np.ones((4, 9), np.int32)
    sh[1, 0] = 3
    sh[2, [0, 1, 2]] = [0, 5, 9]
    sh[3, 2:9] = [1, 2, 3, 4, 5, 6, 7]
    return gen.QCCode(4, 9, 11, sh)


@pytest.mark.parametrize("case", ["z2600", "reg36_z64", "tbp_z64", "degenerate"])
def test_dataflow_equals_lockstep(ldpc, case):
    if case == "z2600":
        code = gen.workload_code(2, Z=2600)
        fr = gen.workload_frames(2, code, frames=9)
        T = 60
    elif case == "reg36_z64":
        code = gen.workload_code(6, Z=64)
        fr = gen.workload_frames(6, code, frames=24, beta=0.8)
        T = 80
    elif case == "tbp_z64":
        code = gen.workload_code(7, Z=64)
        fr = gen.workload_frames(7, code, frames=16, beta=0.8)
        T = 120
    else:
        code = degenerate_qc()
        rng = np.random.default_rng(3)
        x = rng.integers(0, 2, size=(12, code.n)).astype(np.uint8)
        llr = ((1.0 - 2.0 * x) + 0.9 * rng.standard_normal(x.shape)).astype(np.float32) * 2.0
        fr = gen.Frames(x, llr, gen.syndrome(code, x), np.full(12, 0.9))
        T = 12
    g = ldpc.Graph.from_code(code)
    F = fr.llr.shape[0]
    for rule in ("pce_vnr", "pce", "none"):
        ref = gpu_decode(ldpc, g, fr.llr, fr.syndrome, T, rule, trace_iters=4, schedule="lockstep")
        for slots, lag in ((0, 0), (0, 1), (3, 3), (1, 1), (5, 2), (F, F)):
            got = gpu_decode(ldpc, g, fr.llr, fr.syndrome, T, rule, trace_iters=4, schedule="dataflow",
                             max_active_frames=slots, flow_lag=lag)
            same(got, ref, (case, rule, slots, lag), traces=True)
    g.close()


def test_dataflow_small_grids(ldpc):
    """Few CTAs: every CTA walks many items of each pass; results unchanged."""
    code = gen.workload_code(2, Z=600)
    fr = gen.workload_frames(2, code, frames=6)
    g = ldpc.Graph.from_code(code)
    ref = gpu_decode(ldpc, g, fr.llr, fr.syndrome, 40, "pce_vnr", schedule="lockstep")
    for ctas in (1, 2, 7, 150):
        same(gpu_decode(ldpc, g, fr.llr, fr.syndrome, 40, "pce_vnr", schedule="dataflow", grid_ctas=ctas), ref,
             ctas)
    g.close()


def test_dataflow_learned_weights(ldpc):
    import torch
    code = gen.workload_code(6, Z=64)
    fr = gen.workload_frames(6, code, frames=12, beta=0.8)
    nblk = int((code.shifts >= 0).sum())
    g = ldpc.Graph.from_code(code)
    plan = ldpc.WeightedBP(g, 2, 5, np.arange(nblk, dtype=np.int32) % 5, 5)
    dev = torch.device("cuda:0")
    w = torch.from_numpy(np.random.default_rng(4).uniform(0.7, 1.1, size=(5, 5)).astype(np.float32)).to(dev)
    llr, syn = torch.from_numpy(fr.llr).to(dev), torch.from_numpy(fr.syndrome).to(dev)
    out = {}
    for sched in ("lockstep", "dataflow"):
        b, f, i = plan.decode(llr, syn, w, 60, "pce_vnr", schedule=sched)
        out[sched] = dict(bits=b.cpu().numpy(), flags=f.cpu().numpy(), iters=i.cpu().numpy())
    same(out["dataflow"], out["lockstep"], "weights")
    plan.close()
    g.close()


def test_dataflow_batch_of_codes(ldpc):
    """Frames of three QC codes with different item counts back to back:
    slots change code when they refill, so a new frame waits for the whole
    previous frame's variable pass."""
    import torch
    codes = [gen.workload_code(2, Z=2600), gen.workload_code(6, Z=64), gen.workload_code(7, Z=64)]
    rng = np.random.default_rng(8)
    fc = rng.integers(0, 3, size=20).astype(np.int32)
    parts = []
    for f, c in enumerate(fc):
        wl = (2, 6, 7)[c]
        beta = (0.93, 0.8, 0.8)[c]
        parts.append(gen.workload_frames(wl, codes[c], frames=1, first=100 + f, beta=beta))
    llr = np.concatenate([p.llr[0] for p in parts])
    syn = np.concatenate([p.syndrome[0] for p in parts])
    graphs = [ldpc.Graph.from_code(c) for c in codes]
    batch = ldpc.Batch(graphs, fc)
    dev = torch.device("cuda:0")
    t_llr, t_syn = torch.from_numpy(llr).to(dev), torch.from_numpy(syn).to(dev)
    res = {}
    for sched, slots in (("lockstep", 0), ("dataflow", 0), ("dataflow", 4), ("dataflow", 1)):
        out = batch.decode(t_llr, t_syn, 60, "pce_vnr", schedule=sched, max_active_frames=slots)
        res[(sched, slots)] = dict(bits=out[0].cpu().numpy(), flags=out[1].cpu().numpy(), iters=out[2].cpu().numpy())
    for key, r in res.items():
        same(r, res[("lockstep", 0)], key)
    batch.close()
    for g in graphs:
        g.close()


def test_dataflow_timeout_returns_error_and_context_survives(ldpc):
    import torch
    code = gen.workload_code(2, Z=600)
    fr = gen.workload_frames(2, code, frames=4)
    g = ldpc.Graph.from_code(code)
    dev = torch.device("cuda:0")
    llr, syn = torch.from_numpy(fr.llr).to(dev), torch.from_numpy(fr.syndrome).to(dev)
    with pytest.raises(ldpc.LdpcError) as ei:
        ldpc.decode(g, llr, syn, 20, "pce_vnr", schedule="dataflow", barrier_timeout_ms=200,
                    test_unreachable_barrier=True)
    assert ei.value.status == ldpc.LDPC_ERR_TIMEOUT
    ref = gpu_decode(ldpc, g, fr.llr, fr.syndrome, 20, "pce_vnr", schedule="lockstep")
    same(gpu_decode(ldpc, g, fr.llr, fr.syndrome, 20, "pce_vnr", schedule="dataflow"), ref, "after timeout")
    g.close()


def test_dataflow_refused_for_csr(ldpc):
    import torch
    code = gen.workload_code(1)
    fr = gen.workload_frames(1, code, frames=2)
    g = ldpc.Graph.from_code(code)
    dev = torch.device("cuda:0")
    with pytest.raises(ldpc.LdpcError) as ei:
        ldpc.decode(g, torch.from_numpy(fr.llr).to(dev), torch.from_numpy(fr.syndrome).to(dev), 5, "pce",
                    schedule="dataflow")
    assert ei.value.status == ldpc.LDPC_ERR_INVALID_ARG
    g.close()


def degenerate_csr():
    rows = [[0], [0, 1], [1, 2, 3], [], [2, 4, 5, 6, 7, 8, 9, 10], [3, 4], [5, 11]]
    rowptr = np.cumsum([0] + [len(r) for r in rows]).astype(np.int32)
    return gen.CSRCode(len(rows), 13, rowptr, np.concatenate([np.asarray(r, np.int32) for r in rows]))


@pytest.mark.parametrize("case", ["csr_n4096", "fd_n256", "degenerate", "decodable", "degree24"])
def test_frame_schedule_equals_lockstep(ldpc, case):
    if case == "csr_n4096":
        code = gen.workload_code(1)
        fr = gen.workload_frames(1, code, frames=20)
    elif case == "fd_n256":
        code = gen.wbp_fd_code()
        fr = gen.make_frames(code, np.full(9, gen.sigma_for_capacity(code.rate / 0.9)), range(300, 309))
    elif case == "degenerate":
        code = degenerate_csr()
        rng = np.random.default_rng(2)
        x = rng.integers(0, 2, size=(11, code.n)).astype(np.uint8)
        llr = ((1.0 - 2.0 * x) + 1.1 * rng.standard_normal(x.shape)).astype(np.float32) * 1.3
        fr = gen.Frames(x, llr, gen.syndrome(code, x), np.full(11, 1.1))
    elif case == "decodable":
        code = gen.random_csr_code(2000, 1000, 3, {6: 1000}, seed=4242)
        fr = gen.make_frames(code, np.full(12, 0.78), seeds=range(800, 812))
    else:
        # checks of degree about 24 (the generic check path) spread over both CTAs of a
        # pair, with variables in both CTAs' blocks
        code = gen.random_csr_code(2048, 256, 3, {24: 256}, seed=4343)
        fr = gen.make_frames(code, np.full(10, 0.6), seeds=range(900, 910))
    g = ldpc.Graph.from_code(code)
    for rule in ("pce_vnr", "pce", "none"):
        ref = gpu_decode(ldpc, g, fr.llr, fr.syndrome, 60, rule, trace_iters=5, schedule="lockstep")
        for opts in (dict(schedule="frame"), dict(schedule="auto"), dict(schedule="frame", grid_ctas=2),
                     dict(schedule="frame", vnr_first_iter=1), dict(schedule="frame_pair"),
                     dict(schedule="frame_pair", grid_ctas=2), dict(schedule="frame_pair", grid_ctas=6),
                     dict(schedule="frame_pair", vnr_first_iter=1)):
            r = ref
            if opts.get("vnr_first_iter") == 1:
                r = gpu_decode(ldpc, g, fr.llr, fr.syndrome, 60, rule, trace_iters=5, schedule="lockstep",
                               vnr_first_iter=1)
            got = gpu_decode(ldpc, g, fr.llr, fr.syndrome, 60, rule, trace_iters=5, **opts)
            same(got, r, (case, rule, opts), traces=True)
    g.close()


def test_frame_schedule_learned_weights_and_batch(ldpc):
    import torch
    code = gen.workload_code(1)
    fr = gen.workload_frames(1, code, frames=10)
    g = ldpc.Graph.from_code(code)
    cls, C, _ = gen.edge_classes_by_check_degree(code)
    plan = ldpc.WeightedBP(g, 2, 4, cls, C)
    dev = torch.device("cuda:0")
    w = torch.from_numpy(np.random.default_rng(5).uniform(0.7, 1.1, size=(4, C)).astype(np.float32)).to(dev)
    llr, syn = torch.from_numpy(fr.llr).to(dev), torch.from_numpy(fr.syndrome).to(dev)
    out = {}
    for sched in ("lockstep", "frame", "frame_pair"):
        b, f, i = plan.decode(llr, syn, w, 80, "pce_vnr", schedule=sched)
        out[sched] = dict(bits=b.cpu().numpy(), flags=f.cpu().numpy(), iters=i.cpu().numpy())
    same(out["frame"], out["lockstep"], "weights")
    same(out["frame_pair"], out["lockstep"], "weights, pair")
    plan.close()
    batch = ldpc.Batch([g], np.zeros(10, dtype=np.int32))
    res = {}
    for sched in ("lockstep", "frame", "frame_pair"):
        o = batch.decode(llr.reshape(-1), syn.reshape(-1), 80, "pce_vnr", schedule=sched, debug_guards=True)
        torch.cuda.synchronize()
        assert ldpc.ldpc_batch_check_guards(batch.handle) == ldpc.LDPC_OK
        res[sched] = dict(bits=o[0].cpu().numpy(), flags=o[1].cpu().numpy(), iters=o[2].cpu().numpy())
    same(res["frame"], res["lockstep"], "batch")
    same(res["frame_pair"], res["lockstep"], "batch, pair")
    batch.close()
    g.close()


def test_frame_schedule_refused_where_it_does_not_apply(ldpc):
    import torch
    dev = torch.device("cuda:0")
    big = gen.random_csr_code(20000, 10000, 3, {6: 10000}, seed=77)  # 60000 edges: beyond shared memory
    for code, kw in ((gen.workload_code(2, Z=64), {}), (gen.workload_code(1), dict(fp64=True)), (big, {})):
        if code is big:
            fr = gen.make_frames(code, np.full(2, 0.8), seeds=range(2))
        else:
            fr = gen.workload_frames(2 if hasattr(code, "shifts") else 1, code, frames=2)
        g = ldpc.Graph.from_code(code)
        for sched in ("frame", "frame_pair"):
            with pytest.raises(ldpc.LdpcError) as ei:
                ldpc.decode(g, torch.from_numpy(fr.llr).to(dev), torch.from_numpy(fr.syndrome).to(dev), 5, "pce",
                            schedule=sched, **kw)
            assert ei.value.status == ldpc.LDPC_ERR_INVALID_ARG
        g.close()
