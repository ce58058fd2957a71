"""Early termination against what the method itself fixes, on the FP64 oracle.

Paper, section "Early Termination": PCE-ET stops a frame once its decision
meets the parity checks; VNR-ET stops it as soon as q^(k) < q^(k-1); both
run inside the same flooding BP, with the parity test first.  At equal D_max
the three rules therefore see the same trajectory up to the iteration where
one of them stops, which fixes, frame by frame:
- D(PCE+VNR) <= D(PCE) <= D(NONE) = D_max;
- a frame PCE+VNR does not abort ends exactly as under PCE (same D, flags, bits);
- a frame PCE+VNR aborts at k is one PCE had not decoded by k;
so FER(PCE+VNR) >= FER(PCE).  The section "Simulations" also states the
regime: VNR-ET raises the FER, cuts the mean iteration count where frames do
not decode and leaves it alone where they do, and so raises K = N R (1 - FER)/D
(Eq. 2) except where every frame decodes.  These are checked on a
(3,6)-regular QC code (the base matrix of the n = 960,000 sweep code, lifted by
Z = 64) across its waterfall.  CPU only.
"""
import os

import numpy as np
import pytest

from paper_2507_03509_gb300 import gen

D_MAX = 100
FRAMES = 48
BETAS = (0.7, 0.8, 0.85, 0.9, 0.95)
SUCCESS, ABORTED = 1, 2


@pytest.fixture(scope="module")
def runs(oracle_mod):
    code = gen.workload_code(6, Z=64)
    csr = code.to_csr()
    out = {}
    for beta in BETAS:
        fr = gen.workload_frames(6, code, frames=FRAMES, beta=beta)
        out[beta] = {rule: oracle_mod.decode(csr, fr.llr, fr.syndrome, D_MAX, r, trace_iters=0)
                     for rule, r in (("none", oracle_mod.RULE_NONE), ("pce", oracle_mod.RULE_PCE),
                                     ("vnr", oracle_mod.RULE_PCE_VNR))}
    return out


@pytest.mark.parametrize("beta", BETAS)
def test_per_frame_order_of_the_three_rules(runs, beta):
    r = runs[beta]
    none, pce, vnr = r["none"], r["pce"], r["vnr"]
    assert (none["iters"] == D_MAX).all()
    assert (vnr["iters"] <= pce["iters"]).all() and (pce["iters"] <= none["iters"]).all()
    kept = (vnr["flags"] & ABORTED) == 0
    assert np.array_equal(vnr["iters"][kept], pce["iters"][kept])
    assert np.array_equal(vnr["flags"][kept], pce["flags"][kept])
    assert np.array_equal(vnr["bits"][kept], pce["bits"][kept])
    # an abort at k: PCE had not decoded that frame by k
    ab = ~kept
    assert ((pce["iters"][ab] > vnr["iters"][ab]) | ((pce["flags"][ab] & SUCCESS) == 0)).all()
    assert ((vnr["flags"][ab] & SUCCESS) == 0).all()
    # PCE never aborts; a PCE success stops before D_max or exactly at it
    assert ((pce["flags"] & ABORTED) == 0).all()


def fer(run):
    return float(np.mean((run["flags"] & SUCCESS) == 0))


def test_paper_regime_on_the_waterfall(runs):
    # below the waterfall every frame decodes and VNR-ET changes nothing
    for beta in (0.7, 0.8):
        r = runs[beta]
        assert fer(r["pce"]) == 0.0 and fer(r["vnr"]) == 0.0
        assert np.array_equal(r["vnr"]["iters"], r["pce"]["iters"])
    # in and above it VNR-ET raises the FER and cuts the mean iteration count
    for beta in (0.85, 0.9, 0.95):
        r = runs[beta]
        assert fer(r["vnr"]) >= fer(r["pce"])
        assert r["vnr"]["iters"].mean() < 0.6 * r["pce"]["iters"].mean()
    # where frames fail, throughput K = (1 - FER) / mean D rises with VNR-ET
    for beta in (0.85, 0.9):
        r = runs[beta]
        k = lambda run: (1.0 - fer(run)) / run["iters"].mean()
        assert k(r["vnr"]) > k(r["pce"])
    # far above it no frame decodes: both fail every frame, VNR-ET far sooner
    r = runs[0.95]
    assert fer(r["pce"]) == 1.0 and fer(r["vnr"]) == 1.0
    assert r["vnr"]["iters"].mean() < 0.3 * D_MAX


def _stored(name):
    """Stored oracle decisions: {frame: (iters, flags, bits sha256)}."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", name)
    rows = {}
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            f, it, fl, _, h = line.split()
            rows[int(f)] = (int(it), int(fl), h)
    return rows


@pytest.mark.parametrize("workload,rules,d_max", [
    ("csr_n4096_r0.1", ("none", "pce", "pce_vnr"), 200),
    ("qc_n1e6_r0.02", ("pce", "pce_vnr"), 500),
])
def test_stored_full_size_decisions_keep_the_order_of_the_rules(workload, rules, d_max):
    # the decisions the GPU parity tests compare with obey the same per-frame order
    runs = {r: _stored(f"oracle_{workload}_{r}.txt") for r in rules}
    frames = runs["pce"].keys()
    assert all(runs[r].keys() == frames for r in rules)
    for f in frames:
        pce, vnr = runs["pce"][f], runs["pce_vnr"][f]
        if "none" in runs:
            assert runs["none"][f][0] == d_max
        assert vnr[0] <= pce[0] <= d_max
        if not vnr[1] & ABORTED:
            assert vnr == pce
        else:
            assert not vnr[1] & SUCCESS and (pce[0] > vnr[0] or not pce[1] & SUCCESS)
