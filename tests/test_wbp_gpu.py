"""Weighted belief propagation on the GPU (ldpc_wbp_*) against the FP64 oracle.

Tolerances.  FP64 plans run the oracle's formulas (tanh rule, explicit
products) with other summation orders, so APP, loss and gradients agree to
~1e-12 relative, except where atanh is evaluated next to +-1 (condition number
up to ~1e10 at saturated inputs), hence 1e-9 here.  FP32 plans run the
decoder's r-domain check rule with fast exp/log (a few ulp per operation);
APP values agree with the oracle like the decoder's messages do (1e-4 relative
plus 1e-4 absolute after 10-20 iterations), and every gradient element, a sum
of products of such values over every iteration, to 2e-3 of its own value
plus 1e-4 of the largest element of its row.
"""
import numpy as np
import pytest

from paper_2507_03509_gb300 import gen
from _decode_helpers import lib

pytestmark = pytest.mark.gpu


def fd_setup(frames=4, beta=0.9, seed=0):
    code = gen.wbp_fd_code()
    cls, C, _ = gen.edge_classes_by_check_degree(code)
    sigma = gen.sigma_for_capacity(code.rate / beta)
    fr = gen.make_frames(code, np.full(frames, sigma), [9000 + 10 * seed + f for f in range(frames)])
    return code, cls, C, fr


def qc_setup(Z=64, frames=3, beta=0.9, seed=0):
    code = gen.random_qc_code(23, 26, Z, gen._qc_weights_2_3(26, 13, 41), seed=41)
    nblk = int((code.shifts >= 0).sum())
    cls_blk = (np.arange(nblk) % 7).astype(np.int32)         # 7 classes over the base blocks
    cls_csr = cls_blk[gen.qc_csr_edge_blocks(code)]
    sigma = gen.sigma_for_capacity(code.rate / beta)
    fr = gen.make_frames(code, np.full(frames, sigma), [9500 + 10 * seed + f for f in range(frames)])
    return code, cls_blk, cls_csr, 7, fr


def tensors(fr, dev):
    import torch
    return (torch.from_numpy(fr.llr).to(dev), torch.from_numpy(fr.syndrome).to(dev),
            torch.from_numpy(fr.x).to(dev))


def run_gpu(ldpc, code, cls, C, fr, T, w, fp64, every=5, want_llr=True):
    import torch
    dev = torch.device("cuda:0")
    g = ldpc.Graph.from_code(code)
    plan = ldpc.WeightedBP(g, fr.llr.shape[0], T, cls, C, checkpoint_every=every, fp64=fp64)
    llr, syn, x = tensors(fr, dev)
    wt = torch.tensor(w, dtype=plan.dtype, device=dev)
    app = plan.forward(llr, syn, wt)
    loss, gapp = plan.loss(app, x)
    gw, gl = plan.backward(llr, syn, wt, gapp, want_llr=want_llr)
    torch.cuda.synchronize()
    out = dict(app=app.double().cpu().numpy(), loss=float(loss.item()), grad_w=gw.double().cpu().numpy(),
               grad_llr=gl.double().cpu().numpy() if gl is not None else None)
    plan.close()
    g.close()
    return out


def oracle_code(code):
    return code.to_csr() if hasattr(code, "to_csr") else code


@pytest.mark.parametrize("fp64", [True, False])
def test_csr_forward_loss_gradient_match_oracle(oracle_mod, fp64):
    ldpc = lib()
    code, cls, C, fr = fd_setup()
    T = 10
    w = np.random.default_rng(1).uniform(0.6, 1.2, size=(T, C))
    got = run_gpu(ldpc, code, cls, C, fr, T, w, fp64)
    ref = oracle_mod.wbp(code, fr.llr, fr.syndrome, fr.x, T, cls, w if fp64 else w.astype(np.float32))
    check(got, ref, fp64)


@pytest.mark.parametrize("fp64", [True, False])
def test_qc_forward_loss_gradient_match_oracle(oracle_mod, fp64):
    ldpc = lib()
    code, cls_blk, cls_csr, C, fr = qc_setup()
    T = 12
    w = np.random.default_rng(2).uniform(0.6, 1.2, size=(T, C))
    got = run_gpu(ldpc, code, cls_blk, C, fr, T, w, fp64)
    ref = oracle_mod.wbp(code.to_csr(), fr.llr, fr.syndrome, fr.x, T, cls_csr, w if fp64 else w.astype(np.float32))
    check(got, ref, fp64)


def check(got, ref, fp64):
    if fp64:
        np.testing.assert_allclose(got["app"], ref["app"], rtol=1e-9, atol=1e-9)
        assert got["loss"] == pytest.approx(ref["loss"], rel=1e-11)
        sc = np.abs(ref["grad_w"]).max()
        np.testing.assert_allclose(got["grad_w"], ref["grad_w"], rtol=1e-9, atol=1e-9 * sc)
        scl = np.abs(ref["grad_llr"]).max()
        np.testing.assert_allclose(got["grad_llr"], ref["grad_llr"], rtol=1e-9, atol=1e-9 * scl)
    else:
        np.testing.assert_allclose(got["app"], ref["app"], rtol=1e-4, atol=1e-4)
        assert got["loss"] == pytest.approx(ref["loss"], rel=1e-5)
        # every element to FP32_GRAD_RTOL of its own FP64 value, with an absolute
        # floor of FP32_GRAD_FLOOR times the largest value of its row (one
        # iteration's weights, one frame's channel values), so a small class
        # gradient is held to its own size, not to the largest one's
        per_element_close(got["grad_w"], ref["grad_w"], "grad_w")
        per_element_close(got["grad_llr"], ref["grad_llr"], "grad_llr")


FP32_GRAD_RTOL, FP32_GRAD_FLOOR = 2e-3, 1e-4


def per_element_close(got, want, what):
    floor = FP32_GRAD_FLOOR * np.abs(want).max(axis=-1, keepdims=True)
    err = np.abs(got - want)
    tol = FP32_GRAD_RTOL * np.abs(want) + floor
    worst = np.unravel_index(np.argmax(err / np.maximum(tol, 1e-300)), err.shape)
    assert (err <= tol).all(), (f"{what}: {(err > tol).sum()} of {err.size} elements out of tolerance; worst at "
                                f"{worst}: got {got[worst]:.6g}, want {want[worst]:.6g}, ratio "
                                f"{err[worst] / tol[worst]:.3g}")


def test_fp64_gradient_matches_finite_differences():
    """Central differences (eps 1e-6) of the GPU's own FP64 loss against its
    adjoint, for every weight, on the n = 256 code."""
    import torch
    ldpc = lib()
    code, cls, C, fr = fd_setup(frames=3, seed=1)
    T = 8
    dev = torch.device("cuda:0")
    g = ldpc.Graph.from_code(code)
    plan = ldpc.WeightedBP(g, 3, T, cls, C, checkpoint_every=3, fp64=True)
    llr, syn, x = tensors(fr, dev)
    w0 = np.random.default_rng(3).uniform(0.7, 1.3, size=(T, C))

    def loss_of(w):
        wt = torch.tensor(w, dtype=torch.float64, device=dev)
        app = plan.forward(llr, syn, wt, save=False)
        return float(plan.loss(app, x, want_grad=False)[0].item())

    wt = torch.tensor(w0, dtype=torch.float64, device=dev)
    app = plan.forward(llr, syn, wt)
    _, gapp = plan.loss(app, x)
    gw, _ = plan.backward(llr, syn, wt, gapp)
    gw = gw.cpu().numpy()
    eps = 1e-6
    fd = np.zeros_like(w0)
    for k in range(T):
        for c in range(C):
            wp, wm = w0.copy(), w0.copy()
            wp[k, c] += eps
            wm[k, c] -= eps
            fd[k, c] = (loss_of(wp) - loss_of(wm)) / (2 * eps)
    sc = np.abs(gw).max()
    np.testing.assert_allclose(gw, fd, rtol=1e-5, atol=1e-6 * sc)
    plan.close()


@pytest.mark.parametrize("fp64", [False, True])
def test_checkpoint_interval_does_not_change_results(fp64):
    ldpc = lib()
    code, cls_blk, _, C, fr = qc_setup(seed=2)
    T = 11
    w = np.random.default_rng(4).uniform(0.6, 1.2, size=(T, C))
    runs = [run_gpu(ldpc, code, cls_blk, C, fr, T, w, fp64, every=e) for e in (1, 3, 5, T, 50)]
    for r in runs[1:]:
        assert np.array_equal(r["app"], runs[0]["app"])
        assert np.array_equal(r["grad_w"], runs[0]["grad_w"])
        assert np.array_equal(r["grad_llr"], runs[0]["grad_llr"])


def test_autograd_gradcheck():
    import torch
    ldpc = lib()
    code, cls, C, fr = fd_setup(frames=2, seed=3)
    T = 4
    dev = torch.device("cuda:0")
    g = ldpc.Graph.from_code(code)
    plan = ldpc.WeightedBP(g, 2, T, cls, C, checkpoint_every=2, fp64=True)
    llr, syn, _ = tensors(fr, dev)
    w = torch.tensor(np.random.default_rng(5).uniform(0.7, 1.3, size=(T, C)), dtype=torch.float64, device=dev,
                     requires_grad=True)
    assert torch.autograd.gradcheck(lambda ww: ldpc.weighted_bp(plan, ww, llr, syn), (w,), eps=1e-6, atol=1e-5,
                                    rtol=1e-4)
    # and a torch loss on top: the chain through the plan's adjoint
    ll = llr.clone().requires_grad_(False)
    app = ldpc.weighted_bp(plan, w, ll, syn)
    (app.tanh().sum()).backward()
    assert w.grad is not None and torch.isfinite(w.grad).all()
    plan.close()


def test_fullsize_training_step_and_sampled_parity(oracle_mod):
    """The training workload: QC n = 65536 (115 x 128 base, Z = 512), 128
    frames at capacity = R/0.9, 20 iterations, one weight per (iteration, base
    block), checkpoints every 5.  Frames are independent, so the first two
    frames of the 128-frame plan must give bit-for-bit the APP of a 2-frame
    plan, whose APP, loss and gradient are compared with the oracle; the
    128-frame step must be deterministic, and a few SGD steps must lower the
    loss."""
    import torch
    ldpc = lib()
    number = 4
    wl = gen.WORKLOADS[number]
    code = gen.workload_code(number)
    F, T = wl["frames"], wl["iters"]
    fr = gen.workload_frames(number, code, frames=F)
    nblk = int((code.shifts >= 0).sum())
    cls = np.arange(nblk, dtype=np.int32)
    dev = torch.device("cuda:0")
    g = ldpc.Graph.from_code(code)
    plan = ldpc.WeightedBP(g, F, T, cls, nblk, checkpoint_every=wl["checkpoint"])
    llr, syn, x = tensors(fr, dev)
    w = torch.ones((T, nblk), dtype=torch.float32, device=dev)
    app = plan.forward(llr, syn, w)
    loss, gapp = plan.loss(app, x)
    gw, _ = plan.backward(llr, syn, w, gapp)
    app2 = plan.forward(llr, syn, w)
    loss2, gapp2 = plan.loss(app2, x)
    gw2, _ = plan.backward(llr, syn, w, gapp2)
    assert torch.equal(app, app2) and torch.equal(gw, gw2) and torch.equal(loss, loss2)
    assert torch.isfinite(gw).all()
    # the first two frames alone
    small = ldpc.WeightedBP(g, 2, T, cls, nblk, checkpoint_every=wl["checkpoint"])
    app_s = small.forward(llr[:2].contiguous(), syn[:2].contiguous(), w)
    assert torch.equal(app_s, app[:2])
    # oracle on those two frames (weights 1.3 on the last iteration, so they matter)
    wv = np.ones((T, nblk))
    wv[-1] = 1.3
    w_t = torch.tensor(wv, dtype=torch.float32, device=dev)
    app_s = small.forward(llr[:2].contiguous(), syn[:2].contiguous(), w_t)
    loss_s, gapp_s = small.loss(app_s, x[:2].contiguous())
    gw_s, _ = small.backward(llr[:2].contiguous(), syn[:2].contiguous(), w_t, gapp_s)
    cls_csr = cls[gen.qc_csr_edge_blocks(code)]
    ref = oracle_mod.wbp(code.to_csr(), fr.llr[:2], fr.syndrome[:2], fr.x[:2], T, cls_csr, wv, grad=True)
    np.testing.assert_allclose(app_s.double().cpu().numpy(), ref["app"], rtol=1e-4, atol=1e-4)
    assert float(loss_s.item()) == pytest.approx(ref["loss"], rel=1e-5)
    per_element_close(gw_s.double().cpu().numpy(), ref["grad_w"], "grad_w")
    # SGD lowers the loss
    losses = []
    for _ in range(4):
        a = plan.forward(llr, syn, w)
        l, ga = plan.loss(a, x)
        gww, _ = plan.backward(llr, syn, w, ga)
        plan.sgd_step(w, gww, lr=20.0)
        losses.append(float(l.item()))
    assert losses[-1] < losses[0]
    small.close()
    plan.close()


def test_training_step_replays_in_a_cuda_graph():
    import torch
    ldpc = lib()
    code, cls_blk, _, C, fr = qc_setup(Z=128, frames=4, seed=4)
    T = 10
    dev = torch.device("cuda:0")
    g = ldpc.Graph.from_code(code)
    plan = ldpc.WeightedBP(g, 4, T, cls_blk, C, checkpoint_every=5)
    llr, syn, x = tensors(fr, dev)
    w0 = torch.tensor(np.random.default_rng(6).uniform(0.8, 1.1, size=(T, C)), dtype=torch.float32, device=dev)
    w = w0.clone()
    app = torch.empty((4, code.n), dtype=torch.float32, device=dev)
    gw = torch.empty_like(w)

    def step():
        plan.forward(llr, syn, w, app=app)
        loss, gapp = plan.loss(app, x)
        plan.backward(llr, syn, w, gapp, grad_w=gw)
        plan.sgd_step(w, gw, lr=0.5)
        return loss

    # eager reference: three steps
    ref = []
    for _ in range(3):
        ref.append(step().clone())
    w_ref = w.clone()
    w.copy_(w0)
    side = torch.cuda.Stream(dev)
    side.wait_stream(torch.cuda.current_stream(dev))
    torch.cuda.synchronize()
    cg = torch.cuda.CUDAGraph()
    with torch.cuda.graph(cg):
        loss_g = step()
    w.copy_(w0)  # capture does not run the work
    got = []
    for _ in range(3):
        cg.replay()
        got.append(loss_g.clone())
    torch.cuda.synchronize()
    for a, b in zip(got, ref):
        assert torch.equal(a, b)
    assert torch.equal(w, w_ref)
    plan.close()


def test_argument_errors():
    ldpc = lib()
    code, cls, C, fr = fd_setup(frames=1)
    g = ldpc.Graph.from_code(code)
    with pytest.raises(ldpc.LdpcError):
        ldpc.WeightedBP(g, 1, 4, cls, C - 1)                   # a class out of range
    with pytest.raises(ValueError):
        ldpc.WeightedBP(g, 1, 4, np.zeros(3, np.int32), 1)   # a map of the wrong length (checked in Python)
    with pytest.raises(ldpc.LdpcError):
        ldpc.WeightedBP(g, 1, 0, cls, C)                     # no iterations
    plan = ldpc.WeightedBP(g, 1, 6, cls, C, checkpoint_every=2)
    import torch
    dev = torch.device("cuda:0")
    llr, syn, _ = tensors(fr, dev)
    w = torch.ones((6, C), device=dev)
    with pytest.raises(ldpc.LdpcError):                      # checkpoints never saved
        plan.backward(llr, syn, w, torch.zeros((1, code.n), device=dev))
    plan.close()


# ---------------------------------------------------------------------------
# Early-terminating decoding with learned weights (ldpc_wbp_decode)
# ---------------------------------------------------------------------------
def weighted_decode(ldpc, plan, fr, w, max_iter, rule, **opt):
    import torch
    dev = torch.device("cuda:0")
    llr, syn, _ = tensors(fr, dev)
    wt = torch.tensor(w, dtype=torch.float32, device=dev)
    T = opt.pop("trace_iters", 0)
    F, n = fr.llr.shape
    tr = {}
    if T:
        dt = torch.float64 if opt.get("fp64") else torch.float32
        tr = dict(trace_iters=T, trace_app=torch.full((T, F, n), float("nan"), dtype=dt, device=dev),
                  trace_q=torch.full((T, F), float("nan"), dtype=torch.float64, device=dev))
    bits, flags, iters = plan.decode(llr, syn, wt, max_iter, rule, **opt, **tr)
    torch.cuda.synchronize()
    out = dict(bits=bits.cpu().numpy(), flags=flags.cpu().numpy(), iters=iters.cpu().numpy())
    if T:
        out.update(app=tr["trace_app"].double().cpu().numpy(), q=tr["trace_q"].cpu().numpy())
    return out


def test_weighted_decode_unit_weights_is_plain_decode():
    import torch
    ldpc = lib()
    code, cls_blk, _, C, fr = qc_setup(Z=128, frames=6, beta=0.9, seed=5)
    g = ldpc.Graph.from_code(code)
    plan = ldpc.WeightedBP(g, 1, 4, cls_blk, C)
    from _decode_helpers import gpu_decode
    ref = gpu_decode(ldpc, g, fr.llr, fr.syndrome, 60, "pce_vnr")
    got = weighted_decode(ldpc, plan, fr, np.ones((4, C)), 60, "pce_vnr")
    for k in ("bits", "flags", "iters"):
        assert np.array_equal(got[k], ref[k]), k
    plan.close()


@pytest.mark.parametrize("rule", ["pce_vnr", "none"])
def test_weighted_decode_matches_oracle(oracle_mod, rule):
    """Weighted messages and APP over the first iterations, and the decisions:
    a frame whose FP32 decisions differ from the oracle's is re-run in FP64,
    which must equal them."""
    ldpc = lib()
    code, cls_blk, cls_csr, C, fr = qc_setup(Z=128, frames=8, beta=0.75, seed=6)
    g = ldpc.Graph.from_code(code)
    plan = ldpc.WeightedBP(g, 1, 3, cls_blk, C)
    w = np.random.default_rng(7).uniform(0.7, 1.1, size=(3, C)).astype(np.float32)
    csr = code.to_csr()
    T = 6
    got = weighted_decode(ldpc, plan, fr, w, T, "none", trace_iters=T)
    orc = oracle_mod.decode(csr, fr.llr, fr.syndrome, T, 0, trace_iters=T, trace=("app", "q"), weights=w,
                            edge_class=cls_csr)
    np.testing.assert_allclose(got["app"], orc["app"], rtol=1e-4, atol=1e-4)
    np.testing.assert_allclose(got["q"], orc["q"], rtol=1e-5)
    rid = {"none": 0, "pce_vnr": 2}[rule]
    got = weighted_decode(ldpc, plan, fr, w, 80, rule)
    orc = oracle_mod.decode(csr, fr.llr, fr.syndrome, 80, rid, weights=w, edge_class=cls_csr)
    bad = np.nonzero((got["iters"] != orc["iters"]) | (got["flags"] != orc["flags"])
                     | (got["bits"] != orc["bits"]).any(1))[0]
    if bad.size:
        sub = gen.Frames(fr.x[bad], fr.llr[bad], fr.syndrome[bad], fr.sigma[bad])
        g64 = weighted_decode(ldpc, plan, sub, w, 80, rule, fp64=True)
        for i, f in enumerate(bad):
            assert (g64["iters"][i], g64["flags"][i]) == (orc["iters"][f], orc["flags"][f]), f
            assert np.array_equal(g64["bits"][i], orc["bits"][f]), f
    assert bad.size <= 2
    plan.close()


def test_weighted_decode_reuses_the_last_row():
    ldpc = lib()
    code, cls_blk, _, C, fr = qc_setup(Z=128, frames=4, beta=0.75, seed=7)
    g = ldpc.Graph.from_code(code)
    short = ldpc.WeightedBP(g, 1, 2, cls_blk, C)
    long = ldpc.WeightedBP(g, 1, 9, cls_blk, C)
    w = np.random.default_rng(8).uniform(0.7, 1.1, size=(2, C)).astype(np.float32)
    a = weighted_decode(ldpc, short, fr, w, 40, "pce_vnr")
    b = weighted_decode(ldpc, long, fr, np.concatenate([w, np.repeat(w[-1:], 7, axis=0)]), 40, "pce_vnr")
    for k in ("bits", "flags", "iters"):
        assert np.array_equal(a[k], b[k]), k
    short.close()
    long.close()


def test_weighted_decode_csr_matches_oracle(oracle_mod):
    """Learned-weight decoding of a general (CSR) code, one class per check
    degree: decisions equal the oracle's (FP64 re-run where FP32 differs)."""
    ldpc = lib()
    code, cls, C, fr = fd_setup(frames=8, beta=0.8, seed=9)
    g = ldpc.Graph.from_code(code)
    plan = ldpc.WeightedBP(g, 1, 4, cls, C)
    w = np.random.default_rng(10).uniform(0.7, 1.1, size=(4, C)).astype(np.float32)
    got = weighted_decode(ldpc, plan, fr, w, 60, "pce_vnr")
    orc = oracle_mod.decode(code, fr.llr, fr.syndrome, 60, 2, weights=w, edge_class=cls)
    bad = np.nonzero((got["iters"] != orc["iters"]) | (got["flags"] != orc["flags"])
                     | (got["bits"] != orc["bits"]).any(1))[0]
    if bad.size:
        sub = gen.Frames(fr.x[bad], fr.llr[bad], fr.syndrome[bad], fr.sigma[bad])
        g64 = weighted_decode(ldpc, plan, sub, w, 60, "pce_vnr", fp64=True)
        for i, f in enumerate(bad):
            assert (g64["iters"][i], g64["flags"][i]) == (orc["iters"][f], orc["flags"][f]), f
            assert np.array_equal(g64["bits"][i], orc["bits"][f]), f
    assert bad.size <= 2
    plan.close()
