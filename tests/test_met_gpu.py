"""The paper's code features on the GPU against the oracle: a type-based-
protograph-like multi-edge-type code at R = 1/50 (core columns of degree 51,
degree-1 columns that q leaves out), punctured bits (Lch = 0: core column 0,
never sent) and shortened bits (known to both sides: Lch = +-100; here 64
degree-1 bits).

At Z = 64 (n = 12800) the code's BP waterfall lies at beta ~0.6-0.9, so
frames decode, fail and get aborted by VNR-ET in the same run."""
import numpy as np
import pytest

from paper_2507_03509_gb300 import gen
from _decode_helpers import assert_close_messages, check_decisions, gpu_decode, lib

pytestmark = pytest.mark.gpu

Z = 64


def met_frames(beta, frames, seed):
    code = gen.tbp_like_qc_code(Z)
    sigma = gen.sigma_for_capacity(code.rate / beta)
    fr = gen.make_frames(code, np.full(frames, sigma), [7700 + 100 * seed + f for f in range(frames)])
    rng = np.random.default_rng(seed)
    short = rng.choice(np.arange(8 * Z, code.n), size=64, replace=False)   # degree-1 bits
    return code, gen.rate_adapt(fr, np.arange(Z), short)


def test_met_messages_match_oracle(oracle_mod):
    ldpc = lib()
    code, fr = met_frames(0.75, 4, 0)
    csr = code.to_csr()
    T = 10
    orc = oracle_mod.decode(csr, fr.llr, fr.syndrome, T, 0, trace_iters=T)
    g = ldpc.Graph.from_code(code)
    got = gpu_decode(ldpc, g, fr.llr, fr.syndrome, T, "none", trace_iters=T)
    assert_close_messages(got["c2v"], orc["c2v"], "c2v")
    assert_close_messages(got["app"], orc["app"], "app")
    np.testing.assert_allclose(got["q"], orc["q"], rtol=1e-6)
    deg = np.bincount(csr.colidx, minlength=code.n)
    assert (deg == 1).sum() == 192 * Z  # q covers only the 8 core columns
    q_core = np.abs(orc["app"][T - 1]).T[deg > 1].sum(0)
    np.testing.assert_allclose(orc["q"][T - 1], q_core, rtol=1e-12)
    g.close()


@pytest.mark.parametrize("beta", [0.7, 0.85])
@pytest.mark.parametrize("rule", ["pce_vnr", "pce"])
def test_met_decisions_match_oracle(oracle_mod, beta, rule):
    ldpc = lib()
    code, fr = met_frames(beta, 16, 1)
    g = ldpc.Graph.from_code(code)
    report = []
    _, got, orc = check_decisions(ldpc, g, code.to_csr(), oracle_mod, fr.llr, fr.syndrome, 200, rule, report=report)
    ok = ((got["flags"] & 1) > 0) & (got["bits"] == fr.x).all(1)
    if beta == 0.7:
        assert ok.sum() >= 4  # the waterfall: some frames decode
    # a shortened degree-1 bit has |APP| >= 100 - 25: its decision is the known bit in every frame
    short = np.abs(fr.llr[0]) == 100.0
    assert short.sum() == 64
    assert (got["bits"][:, short] == fr.x[:, short]).all()
    if rule == "pce_vnr" and beta == 0.85:
        assert ((got["flags"] & 2) > 0).any()  # VNR-ET aborts failing frames
    g.close()


@pytest.mark.parametrize("fp64", [True, False])
def test_met_weighted_bp_matches_oracle(oracle_mod, fp64):
    """Weighted BP on the same code: rows of degree 6 and columns of degree 51
    take the kernels' general paths."""
    import torch
    ldpc = lib()
    code, fr = met_frames(0.75, 3, 2)
    nblk = int((code.shifts >= 0).sum())
    cls = (np.arange(nblk) % 5).astype(np.int32)
    cls_csr = cls[gen.qc_csr_edge_blocks(code)]
    T = 8
    w = np.random.default_rng(3).uniform(0.7, 1.2, size=(T, 5))
    dev = torch.device("cuda:0")
    g = ldpc.Graph.from_code(code)
    plan = ldpc.WeightedBP(g, 3, T, cls, 5, checkpoint_every=3, fp64=fp64)
    llr, syn, x = (torch.from_numpy(a).to(dev) for a in (fr.llr, fr.syndrome, fr.x))
    wt = torch.tensor(w, dtype=plan.dtype, device=dev)
    app = plan.forward(llr, syn, wt)
    loss, gapp = plan.loss(app, x)
    gw, gl = plan.backward(llr, syn, wt, gapp, want_llr=True)
    ref = oracle_mod.wbp(code.to_csr(), fr.llr, fr.syndrome, fr.x, T, cls_csr, w if fp64 else w.astype(np.float32))
    a = app.double().cpu().numpy()
    sc, scl = np.abs(ref["grad_w"]).max(), np.abs(ref["grad_llr"]).max()
    if fp64:
        np.testing.assert_allclose(a, ref["app"], rtol=1e-9, atol=1e-9)
        np.testing.assert_allclose(gw.cpu().numpy(), ref["grad_w"], rtol=1e-9, atol=1e-9 * sc)
        np.testing.assert_allclose(gl.cpu().numpy(), ref["grad_llr"], rtol=1e-9, atol=1e-9 * scl)
    else:
        np.testing.assert_allclose(a, ref["app"], rtol=1e-4, atol=1e-4)
        assert np.abs(gw.double().cpu().numpy() - ref["grad_w"]).max() <= 2e-3 * sc
        assert np.abs(gl.double().cpu().numpy() - ref["grad_llr"]).max() <= 2e-3 * scl
    assert float(loss.item()) == pytest.approx(ref["loss"], rel=1e-5)
    plan.close()
    g.close()
