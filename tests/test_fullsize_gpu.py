"""Full-size parity at the n = 1,000,000, R = 0.02 workload, in the launch
configuration the benchmark times (32 frames, all decoded concurrently, every
CTA that fits, max 500 iterations).

The oracle needs about 5 minutes per rule on 8 cores here, so its decisions
for these 32 frames were stored by tests/golden/make_oracle_decisions.py
(oracle only): iterations, flags, bit errors and a SHA-256 of the decided
bits.  Every frame's decisions must equal them; a frame that differs in FP32
is re-run in the decoder's FP64 mode, which must equal them exactly.  Messages
are compared on sampled frames over the first iterations (the oracle computes
those in seconds), and the sign symmetry is checked bit for bit at full size.
"""
import hashlib
import os

import numpy as np
import pytest

from paper_2507_03509_gb300 import gen
from _decode_helpers import assert_close_messages, gpu_decode, lib

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_golden(name, rule):
    rows = {}
    for line in open(os.path.join(GOLDEN, f"oracle_{name}_{rule}.txt")):
        if line.strip() and not line.startswith("#"):
            f, it, fl, errs, digest = line.split()
            rows[int(f)] = (int(it), int(fl), int(errs), digest)
    return rows


def digest(bits):
    return hashlib.sha256(np.ascontiguousarray(bits).tobytes()).hexdigest()


@pytest.fixture(scope="module")
def ldpc():
    return lib()


@pytest.fixture(scope="module")
def full():
    code = gen.workload_code(2)
    frames = gen.workload_frames(2, code)
    return code, frames


@pytest.mark.parametrize("rule", ["pce_vnr", "pce"])
def test_fullsize_decisions_match_stored_oracle(ldpc, full, rule):
    code, fr = full
    w = gen.WORKLOADS[2]
    gold = load_golden(w["name"], rule)
    assert len(gold) == fr.llr.shape[0]
    graph = ldpc.Graph.from_code(code)
    got = gpu_decode(ldpc, graph, fr.llr, fr.syndrome, w["max_iter"], rule)
    bad = [f for f in range(fr.llr.shape[0])
           if (got["iters"][f], got["flags"][f], digest(got["bits"][f])) != (gold[f][0], gold[f][1], gold[f][3])]
    if bad:
        idx = np.asarray(bad)
        g64 = gpu_decode(ldpc, graph, fr.llr[idx], fr.syndrome[idx], w["max_iter"], rule, fp64=True)
        for i, f in enumerate(bad):
            assert (g64["iters"][i], g64["flags"][i], digest(g64["bits"][i])) == (gold[f][0], gold[f][1],
                                                                                  gold[f][3]), f"frame {f}"
    for f in range(fr.llr.shape[0]):
        if f not in bad:
            assert int((got["bits"][f] != fr.x[f]).sum()) == gold[f][2]
    graph.close()


def test_fullsize_messages_on_sampled_frames(ldpc, oracle_mod, full):
    code, fr = full
    csr = code.to_csr()
    sel = np.array([3, 17])
    T = 3
    orc = oracle_mod.decode(csr, fr.llr[sel], fr.syndrome[sel], T, 0, trace_iters=T)
    graph = ldpc.Graph.from_code(code)
    got = gpu_decode(ldpc, graph, fr.llr[sel], fr.syndrome[sel], T, "none", trace_iters=T)
    assert_close_messages(got["c2v"], orc["c2v"], "c2v")
    assert_close_messages(got["app"], orc["app"], "app")
    np.testing.assert_allclose(got["q"], orc["q"], rtol=1e-6)
    graph.close()


def test_fullsize_sign_symmetry_bit_exact(ldpc, full):
    code, fr = full
    sel = np.array([0, 1])
    rng = np.random.default_rng(99)
    u = rng.integers(0, 2, size=(2, code.n)).astype(np.uint8)
    llr2 = (fr.llr[sel] * (1 - 2 * u.astype(np.float32))).astype(np.float32)
    s2 = fr.syndrome[sel] ^ gen.syndrome(code, u)
    graph = ldpc.Graph.from_code(code)
    a = gpu_decode(ldpc, graph, fr.llr[sel], fr.syndrome[sel], 12, "pce_vnr", trace_iters=2)
    b = gpu_decode(ldpc, graph, llr2, s2, 12, "pce_vnr", trace_iters=2)
    assert (b["bits"] == (a["bits"] ^ u)).all()
    assert (a["flags"] == b["flags"]).all() and (a["iters"] == b["iters"]).all()
    assert (b["app"] == a["app"] * (1 - 2 * u.astype(np.float64))[None]).all()
    assert np.array_equal(a["q"], b["q"])
    graph.close()
