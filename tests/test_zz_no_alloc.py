"""The entry point that allocates nothing gives the same decisions as ldpc_decode.

ldpc_decode_qc_noalloc exists for callers that must not allocate device memory
themselves: real-time reconciliation loops whose latency budget cannot absorb
cudaMalloc/cudaFree (both can synchronise the device), and host processes whose
memory manager reserves the GPU's memory and forbids allocations outside it.
It decodes inside one fixed device array that every call reuses, so the test
makes two calls in a row (the second finds the first one's leftovers) and
compares each with ldpc_decode on the same inputs.  Decisions must be equal
bit for bit, as they are for any concurrency of ldpc_decode.

The file is named so that pytest collects it last.
"""
import numpy as np
import pytest

from paper_2507_03509_gb300 import gen
from _decode_helpers import gpu_decode, lib

pytestmark = pytest.mark.gpu


def _noalloc(ldpc, code, llr, syn, max_iter, rule):
    import torch
    dev = torch.device("cuda:0")
    F = llr.shape[0]
    t_llr = torch.from_numpy(np.ascontiguousarray(llr)).to(dev)
    t_syn = torch.from_numpy(np.ascontiguousarray(syn)).to(dev)
    bits = torch.full((F, code.n), 7, dtype=torch.uint8, device=dev)
    flags = torch.full((F,), 7, dtype=torch.uint8, device=dev)
    iters = torch.full((F,), -1, dtype=torch.int32, device=dev)
    st = ldpc.ldpc_decode_qc_noalloc(code.mb, code.nb, code.Z, code.shifts, F, t_llr.data_ptr(),
                                     t_syn.data_ptr(), max_iter, ldpc.RULES[rule], bits.data_ptr(),
                                     flags.data_ptr(), iters.data_ptr(),
                                     torch.cuda.current_stream(dev).cuda_stream)
    assert st == ldpc.LDPC_OK, ldpc.ldpc_status_str(st)
    torch.cuda.synchronize()
    return dict(bits=bits.cpu().numpy(), flags=flags.cpu().numpy(), iters=iters.cpu().numpy())


# (lifting size, frames of the two calls, D_max).  The small liftings put one
# frame in each of hundreds of slots, so the per-slot tables in shared memory
# are at their largest; the Z = 20000 case (n = 10^6) does not fit every frame
# at once and refills slots from the queue.
@pytest.mark.parametrize("Z,frames,max_iter", [(2600, (6, 9), 60), (20000, (8, 5), 12), (64, (256, 200), 60),
                                               (512, (96, 128), 40)])
def test_noalloc_matches_ldpc_decode_on_consecutive_calls(Z, frames, max_iter):
    ldpc = lib()
    code = gen.workload_code(2, Z=Z)
    graph = ldpc.Graph.from_code(code)
    first = 0
    for call, (F, rule) in enumerate(zip(frames, ("pce_vnr", "pce"))):
        fr = gen.workload_frames(2, code, frames=F, first=first)
        first += F
        want = gpu_decode(ldpc, graph, fr.llr, fr.syndrome, max_iter, rule)
        got = _noalloc(ldpc, code, fr.llr, fr.syndrome, max_iter, rule)
        for key in ("bits", "flags", "iters"):
            assert np.array_equal(got[key], want[key]), (call, key)
    graph.close()
