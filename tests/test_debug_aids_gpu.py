"""Debug aids on the GPU: guard words around the decoder's workspace arrays
(opts.debug_guards, checked by ldpc_graph_check_guards / ldpc_batch_check_guards)
and the index-checking build (-DLDPC_BOUNDS_CHECK), which must find no index
outside its array on decodes that cover every kernel path: QC and CSR codes,
lock-step, dataflow, frame-per-CTA and frame-per-pair schedules, FP32 and FP64, learned weights, a batch of
codes, ragged item tails and refilled slots.  Every other GPU parity test
already decodes with guards and checks them (tests/_decode_helpers.py)."""
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_2507_03509_gb300 import gen
from _decode_helpers import gpu_decode, lib

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_guards_hold_for_graph_and_batch_decodes():
    import torch
    ldpc = lib()
    code = gen.workload_code(2, Z=600)
    fr = gen.workload_frames(2, code, frames=5)
    g = ldpc.Graph.from_code(code)
    for sched in ("lockstep", "dataflow"):
        gpu_decode(ldpc, g, fr.llr, fr.syndrome, 30, "pce_vnr", schedule=sched, max_active_frames=3)
    # a decode without guards leaves none to check
    gpu_decode(ldpc, g, fr.llr, fr.syndrome, 5, "pce", debug_guards=False)
    assert ldpc.ldpc_graph_check_guards(g.handle) == ldpc.LDPC_ERR_INVALID_ARG
    codes = [code, gen.workload_code(6, Z=64)]
    fc = np.array([0, 1, 1, 0, 1], dtype=np.int32)
    parts = [gen.workload_frames((2, 6)[c], codes[c], frames=1, first=50 + i, beta=(0.93, 0.8)[c])
             for i, c in enumerate(fc)]
    graphs = [g, ldpc.Graph.from_code(codes[1])]
    batch = ldpc.Batch(graphs, fc)
    dev = torch.device("cuda:0")
    llr = torch.from_numpy(np.concatenate([p.llr[0] for p in parts])).to(dev)
    syn = torch.from_numpy(np.concatenate([p.syndrome[0] for p in parts])).to(dev)
    for sched in ("lockstep", "dataflow"):
        batch.decode(llr, syn, 40, "pce_vnr", schedule=sched, debug_guards=True)
        torch.cuda.synchronize()
        assert ldpc.ldpc_batch_check_guards(batch.handle) == ldpc.LDPC_OK
    batch.close()
    for gr in graphs:
        gr.close()


CHECKED_SCRIPT = r"""
import numpy as np, torch
from paper_2507_03509_gb300 import build, gen
build.build(checked=True)
from paper_2507_03509_gb300 import ldpc
assert ldpc.library_path().endswith("libldpc_gb300_checked.so")
dev = torch.device("cuda:0")
def run(code, fr, T, **opt):
    g = ldpc.Graph.from_code(code)
    llr, syn = torch.from_numpy(fr.llr).to(dev), torch.from_numpy(fr.syndrome).to(dev)
    for rule in ("pce_vnr", "pce", "none"):
        ldpc.decode(g, llr, syn, T, rule, **opt)  # raises LdpcError(LDPC_ERR_BOUNDS) on a bad index
    torch.cuda.synchronize()
    g.close()
qc = gen.workload_code(2, Z=2600)
run(qc, gen.workload_frames(2, qc, frames=7), 40)
run(qc, gen.workload_frames(2, qc, frames=7), 40, max_active_frames=3, groups=2)
run(qc, gen.workload_frames(2, qc, frames=7), 40, schedule="dataflow", max_active_frames=3)
run(qc, gen.workload_frames(2, qc, frames=3), 10, fp64=True)
tbp = gen.workload_code(7, Z=64)
run(tbp, gen.workload_frames(7, tbp, frames=6, beta=0.8), 60)
run(tbp, gen.workload_frames(7, tbp, frames=6, beta=0.8), 60, schedule="dataflow")
csr = gen.workload_code(1)
run(csr, gen.workload_frames(1, csr, frames=9), 50)
run(csr, gen.workload_frames(1, csr, frames=9), 50, schedule="frame", grid_ctas=2)
run(csr, gen.workload_frames(1, csr, frames=9), 50, schedule="frame_pair", grid_ctas=4)
run(csr, gen.workload_frames(1, csr, frames=3), 10, fp64=True)
reg = gen.workload_code(6, Z=64)
codes = [qc, reg]
fc = np.array([0, 1, 1, 0, 1, 1], dtype=np.int32)
parts = [gen.workload_frames((2, 6)[c], codes[c], frames=1, first=70 + i, beta=(0.93, 0.8)[c]) for i, c in enumerate(fc)]
graphs = [ldpc.Graph.from_code(c) for c in codes]
batch = ldpc.Batch(graphs, fc)
llr = torch.from_numpy(np.concatenate([p.llr[0] for p in parts])).to(dev)
syn = torch.from_numpy(np.concatenate([p.syndrome[0] for p in parts])).to(dev)
for sched in ("lockstep", "dataflow"):
    batch.decode(llr, syn, 40, "pce_vnr", schedule=sched, max_active_frames=2)
nblk = int((reg.shifts >= 0).sum())
plan = ldpc.WeightedBP(graphs[1], 2, 4, np.arange(nblk, dtype=np.int32) % 3, 3)
fr = gen.workload_frames(6, reg, frames=4, beta=0.8)
w = torch.full((4, 3), 0.9, dtype=torch.float32, device=dev)
plan.decode(torch.from_numpy(fr.llr).to(dev), torch.from_numpy(fr.syndrome).to(dev), w, 30, "pce_vnr")
torch.cuda.synchronize()
print("checked decodes ok")
"""


def test_index_checking_build_finds_no_bad_index():
    env = dict(os.environ, LDPC_GB300_CHECKED="1")
    out = subprocess.run([sys.executable, "-c", CHECKED_SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=900)
    assert out.returncode == 0, out.stdout[-2000:] + out.stderr[-4000:]
    assert "checked decodes ok" in out.stdout
