"""Batches of frames of several codes in one persistent kernel (lengths,
rates and noise levels mixed; frames that stop are replaced by waiting ones of
any code).  A batch must decode every frame exactly as ldpc_decode decodes it
with its own code alone; the stream-ordered variant must work inside a CUDA
graph; the autotuner must keep results unchanged."""
import numpy as np
import pytest

from paper_2507_03509_gb300 import gen
from _decode_helpers import gpu_decode, lib

pytestmark = pytest.mark.gpu


def three_codes():
    a = gen.workload_code(2, Z=1000)                                     # n = 50000, R = 0.02
    b = gen.workload_code(6, Z=400)                                      # n = 19200, R = 0.5
    c = gen.random_qc_code(45, 50, 601, np.full(50, 3), seed=3003)       # n = 30050, R = 0.1
    # (n = 2 mod 4: frames after a frame of c start off the 16-byte grid, so
    # the decoder must take the scalar variable-node path for them, with the
    # same results as the vector path the per-code decodes take)
    return [a, b, c]


def make_batch(codes, F, seed):
    rng = np.random.default_rng(seed)
    which = rng.integers(0, len(codes), size=F)
    llr, syn, xs, per = [], [], [], []
    for f in range(F):
        code = codes[which[f]]
        beta = rng.uniform(0.85, 0.97) if code.rate < 0.4 else rng.uniform(0.84, 0.88)
        fr = gen.make_frames(code, [gen.sigma_for_capacity(code.rate / beta)], seeds=[900000 + seed * 1000 + f])
        llr.append(fr.llr[0]); syn.append(fr.syndrome[0]); xs.append(fr.x[0]); per.append(fr)
    return which, np.concatenate(llr), np.concatenate(syn), xs, per


def test_mixed_batch_matches_per_code_decodes():
    import torch
    ldpc = lib()
    codes = three_codes()
    graphs = [ldpc.Graph.from_code(c) for c in codes]
    F = 30
    which, llr, syn, xs, per = make_batch(codes, F, seed=1)
    batch = ldpc.Batch(graphs, which)
    assert batch.llr_len == sum(codes[w].n for w in which)
    dev = torch.device("cuda:0")
    bits, flags, iters = batch.decode(torch.from_numpy(llr).to(dev), torch.from_numpy(syn).to(dev), 120,
                                      "pce_vnr", max_active_frames=6)
    bits, flags, iters = bits.cpu().numpy(), flags.cpu().numpy(), iters.cpu().numpy()
    off = np.concatenate([[0], np.cumsum([codes[w].n for w in which])])
    for c, (code, g) in enumerate(zip(codes, graphs)):
        idx = np.nonzero(which == c)[0]
        if idx.size == 0:
            continue
        ref = gpu_decode(ldpc, g, np.stack([per[f].llr[0] for f in idx]), np.stack([per[f].syndrome[0] for f in idx]),
                         120, "pce_vnr")
        for i, f in enumerate(idx):
            assert (bits[off[f]:off[f + 1]] == ref["bits"][i]).all(), f
            assert flags[f] == ref["flags"][i] and iters[f] == ref["iters"][i], f
    assert len(set(flags.tolist())) >= 2  # successes and failures both occur
    batch.close()


def test_batch_async_replays_in_a_cuda_graph():
    import torch
    ldpc = lib()
    codes = three_codes()
    graphs = [ldpc.Graph.from_code(c) for c in codes]
    F = 12
    which, llr1, syn1, _, _ = make_batch(codes, F, seed=2)
    # a second input set with the same frame-to-code map
    rng = np.random.default_rng(4)
    llr2 = (llr1 + rng.normal(0.0, 0.05, size=llr1.shape)).astype(np.float32)
    batch = ldpc.Batch(graphs, which)
    dev = torch.device("cuda:0")
    s_llr = torch.from_numpy(llr1).to(dev)
    s_syn = torch.from_numpy(syn1).to(dev)
    out = batch.outputs(dev)
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    ref1 = [t.clone() for t in batch.decode(s_llr, s_syn, 80, "pce_vnr")]        # sizes the workspace
    ref2 = [t.clone() for t in batch.decode(torch.from_numpy(llr2).to(dev), s_syn, 80, "pce_vnr")]
    torch.cuda.synchronize()
    stream = torch.cuda.Stream(dev)
    stream.wait_stream(torch.cuda.current_stream(dev))
    with torch.cuda.stream(stream):
        batch.decode_async(s_llr, s_syn, 80, "pce_vnr", out, status)            # warm up on the side stream
    torch.cuda.current_stream(dev).wait_stream(stream)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        batch.decode_async(s_llr, s_syn, 80, "pce_vnr", out, status)
    for llr, ref in ((llr1, ref1), (llr2, ref2)):
        s_llr.copy_(torch.from_numpy(llr).to(dev))
        status.fill_(-1)
        graph.replay()
        torch.cuda.synchronize()
        assert status.item() == 0
        for a, b in zip(out, ref):
            assert torch.equal(a, b)
    batch.close()


def test_autotune_picks_a_schedule_and_keeps_results():
    import torch
    ldpc = lib()
    codes = three_codes()
    graphs = [ldpc.Graph.from_code(c) for c in codes]
    which, llr, syn, _, _ = make_batch(codes, 16, seed=5)
    batch = ldpc.Batch(graphs, which)
    dev = torch.device("cuda:0")
    t_llr, t_syn = torch.from_numpy(llr).to(dev), torch.from_numpy(syn).to(dev)
    ref = [t.clone() for t in batch.decode(t_llr, t_syn, 60, "pce_vnr", groups=1)]
    g, s = batch.autotune(t_llr, t_syn, 60, "pce_vnr")
    assert g in (1, 2, 4, 8) and 1 <= s <= 16
    st = ldpc.ldpc_decode_stats()
    got = batch.decode(t_llr, t_syn, 60, "pce_vnr", stats=st)
    assert st.active_frames >= s
    for a, b in zip(got, ref):
        assert torch.equal(a, b)
    batch.close()


def test_batch_argument_errors():
    ldpc = lib()
    code = gen.workload_code(1)
    g = ldpc.Graph.from_code(code)
    q = ldpc.Graph.from_code(gen.workload_code(2, Z=64))
    with pytest.raises(ldpc.LdpcError):
        ldpc.Batch([g, q], [0, 1])          # CSR and QC mixed
    with pytest.raises(ldpc.LdpcError):
        ldpc.Batch([g], [0, 1])             # frame_graph out of range


def test_csr_batch_matches_per_code_decodes():
    """A batch of two general (CSR) codes: the n = 4096 code and the n = 256
    code, frames interleaved; every frame as decoded by its own code alone."""
    import torch
    ldpc = lib()
    codes = [gen.workload_code(1), gen.wbp_fd_code()]
    graphs = [ldpc.Graph.from_code(c) for c in codes]
    which = np.array([0, 1, 1, 0, 1, 0, 0, 1, 1, 1], dtype=np.int32)
    per = []
    for f, c in enumerate(which):
        code = codes[c]
        per.append(gen.make_frames(code, [gen.sigma_for_capacity(code.rate / 0.88)], [6100 + f]))
    llr = np.concatenate([fr.llr[0] for fr in per])
    syn = np.concatenate([fr.syndrome[0] for fr in per])
    batch = ldpc.Batch(graphs, which)
    dev = torch.device("cuda:0")
    bits, flags, iters = (t.cpu().numpy() for t in batch.decode(torch.from_numpy(llr).to(dev),
                                                                 torch.from_numpy(syn).to(dev), 100, "pce_vnr"))
    off = np.concatenate([[0], np.cumsum([codes[c].n for c in which])])
    for c, g in enumerate(graphs):
        idx = np.nonzero(which == c)[0]
        ref = gpu_decode(ldpc, g, np.stack([per[f].llr[0] for f in idx]), np.stack([per[f].syndrome[0] for f in idx]),
                         100, "pce_vnr")
        for i, f in enumerate(idx):
            assert (bits[off[f]:off[f + 1]] == ref["bits"][i]).all(), f
            assert flags[f] == ref["flags"][i] and iters[f] == ref["iters"][i], f
    batch.close()


def test_batch_async_timeout_comes_back_in_the_status_word():
    """Failure detection on the stream-ordered path: with the test hook that
    makes the first barrier wait for one CTA more than exist, every wait ends
    at its 200 ms limit, the device status word reads LDPC_ERR_TIMEOUT (5),
    and the next decode on the same plan and context is correct."""
    import torch
    ldpc = lib()
    codes = three_codes()
    graphs = [ldpc.Graph.from_code(c) for c in codes]
    which, llr, syn, _, _ = make_batch(codes, 6, seed=11)
    batch = ldpc.Batch(graphs, which)
    dev = torch.device("cuda:0")
    t_llr, t_syn = torch.from_numpy(llr).to(dev), torch.from_numpy(syn).to(dev)
    ref = [t.clone() for t in batch.decode(t_llr, t_syn, 40, "pce_vnr")]
    out = batch.outputs(dev)
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    batch.decode_async(t_llr, t_syn, 40, "pce_vnr", out, status, test_unreachable_barrier=True,
                       barrier_timeout_ms=200)
    torch.cuda.synchronize()
    assert status.item() == ldpc.LDPC_ERR_TIMEOUT
    status.fill_(-1)
    batch.decode_async(t_llr, t_syn, 40, "pce_vnr", out, status)
    torch.cuda.synchronize()
    assert status.item() == 0
    for a, b in zip(out, ref):
        assert torch.equal(a, b)
    batch.close()
