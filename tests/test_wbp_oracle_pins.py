"""Pins of the weighted-BP oracle (oracle/wbp_oracle.c) to facts outside it.

- With every weight 1 its forward pass is the plain sum-product decoder, so
  the APP after T iterations must equal the decoder oracle's (itself pinned to
  brute-force MAP, closed forms and invariants in test_oracle_pins.py).
- Its gradient must equal central finite differences of its own loss: for
  every weight (eps 1e-6, weights in double) and for sampled channel values
  (eps 2^-16, which float32 inputs represent exactly).
- With every weight 0 the messages vanish: APP = Lch, the loss is the channel
  cross-entropy, and the gradient is written out here by hand (only the last
  iteration's weights get one, from the first check-node pass on Lch).
- Flipping bits u in the channel values, the syndrome (s + H u) and the
  reference bits (x + u) leaves loss and weight gradient bit-for-bit unchanged
  and flips the channel-value gradient's signs.
"""
import numpy as np
import pytest

from paper_2507_03509_gb300 import gen

LMAX = 25.0


def fd_case(frames=2, beta=0.9, seed=0):
    code = gen.wbp_fd_code()
    cls, C, _ = gen.edge_classes_by_check_degree(code)
    sigma = gen.sigma_for_capacity(code.rate / beta)
    fr = gen.make_frames(code, np.full(frames, sigma), [7000 + seed * 100 + f for f in range(frames)])
    return code, cls, C, fr


def random_weights(T, C, seed):
    return np.random.default_rng(seed).uniform(0.7, 1.3, size=(T, C))


def test_unit_weights_reproduce_the_decoder_oracle(oracle_mod):
    code, cls, C, fr = fd_case(frames=3)
    T = 6
    out = oracle_mod.wbp(code, fr.llr, fr.syndrome, fr.x, T, cls, np.ones((T, C)), grad=False)
    ref = oracle_mod.decode(code, fr.llr, fr.syndrome, T, oracle_mod.RULE_NONE, final_app=True)
    assert (ref["iters"] == T).all()
    np.testing.assert_allclose(out["app"], ref["app_final"], rtol=1e-12, atol=1e-12)


def _loss(oracle_mod, code, llr, fr, T, cls, w):
    return oracle_mod.wbp(code, llr, fr.syndrome, fr.x, T, cls, w, grad=False)["loss"]


def test_weight_gradient_matches_finite_differences(oracle_mod):
    code, cls, C, fr = fd_case(frames=2)
    T = 5
    w = random_weights(T, C, 1)
    g = oracle_mod.wbp(code, fr.llr, fr.syndrome, fr.x, T, cls, w)["grad_w"]
    eps = 1e-6
    fd = np.zeros_like(w)
    for k in range(T):
        for c in range(C):
            wp, wm = w.copy(), w.copy()
            wp[k, c] += eps
            wm[k, c] -= eps
            fd[k, c] = (_loss(oracle_mod, code, fr.llr, fr, T, cls, wp)
                        - _loss(oracle_mod, code, fr.llr, fr, T, cls, wm)) / (2 * eps)
    scale = np.abs(g).max()
    assert scale > 1e-4
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-6 * scale)


def test_channel_gradient_matches_finite_differences(oracle_mod):
    code, cls, C, fr = fd_case(frames=2, seed=1)
    T = 4
    w = random_weights(T, C, 2)
    gl = oracle_mod.wbp(code, fr.llr, fr.syndrome, fr.x, T, cls, w)["grad_llr"]
    rng = np.random.default_rng(3)
    eps = 2.0 ** -16
    picks = [(int(f), int(v)) for f, v in zip(rng.integers(0, 2, 10), rng.integers(0, code.n, 10))]
    for f, v in picks:
        lp, lm = fr.llr.copy(), fr.llr.copy()
        lp[f, v] += np.float32(eps)
        lm[f, v] -= np.float32(eps)
        assert lp[f, v] - fr.llr[f, v] == np.float32(eps)  # exact in float32
        fd = (_loss(oracle_mod, code, lp, fr, T, cls, w) - _loss(oracle_mod, code, lm, fr, T, cls, w)) / (2 * eps)
        assert fd == pytest.approx(gl[f, v], rel=1e-4, abs=1e-9), (f, v)


def test_zero_weights_closed_form(oracle_mod):
    code, cls, C, fr = fd_case(frames=2, seed=2)
    T = 3
    out = oracle_mod.wbp(code, fr.llr, fr.syndrome, fr.x, T, cls, np.zeros((T, C)))
    F, n = fr.llr.shape
    L = fr.llr.astype(np.float64)
    assert (out["app"] == L).all()
    sx = 1.0 - 2.0 * fr.x
    z = -sx * L
    assert out["loss"] == pytest.approx(np.sum(np.logaddexp(0.0, z)) / (F * n), rel=1e-13)
    gapp = -sx / (1.0 + np.exp(-z)) / (F * n)            # d loss / d APP
    np.testing.assert_allclose(out["grad_llr"], gapp, rtol=1e-13, atol=0)
    assert (out["grad_w"][:T - 1] == 0).all()
    # last iteration: sum over edges of class c of g(v) * t_e, with t_e the check
    # message computed from a = clamp(Lch) by its definition
    want = np.zeros(C)
    row = code.row_of_edge()
    for f in range(F):
        a = np.clip(L[f], -LMAX, LMAX)
        for e in range(code.edges):
            c = row[e]
            lo, hi = code.rowptr[c], code.rowptr[c + 1]
            sgn = -1.0 if fr.syndrome[f, c] else 1.0
            if hi - lo == 1:
                t = sgn * LMAX
            else:
                others = [code.colidx[i] for i in range(lo, hi) if i != e]
                t = sgn * 2.0 * np.arctanh(np.prod(np.tanh(a[others] / 2.0)))
            want[cls[e]] += gapp[f, code.colidx[e]] * t
    np.testing.assert_allclose(out["grad_w"][T - 1], want, rtol=1e-10)


def test_sign_symmetry_bit_exact(oracle_mod):
    code, cls, C, fr = fd_case(frames=2, seed=3)
    T = 5
    w = random_weights(T, C, 4)
    u = np.random.default_rng(5).integers(0, 2, size=fr.x.shape).astype(np.uint8)
    a = oracle_mod.wbp(code, fr.llr, fr.syndrome, fr.x, T, cls, w)
    b = oracle_mod.wbp(code, (fr.llr * (1 - 2 * u.astype(np.float32))).astype(np.float32),
                       fr.syndrome ^ gen.syndrome(code, u), fr.x ^ u, T, cls, w)
    assert a["loss"] == b["loss"]
    assert np.array_equal(a["grad_w"], b["grad_w"])
    flip = 1.0 - 2.0 * u
    assert np.array_equal(b["app"], a["app"] * flip)
    assert np.array_equal(b["grad_llr"], a["grad_llr"] * flip)


def test_gradient_fd_with_degree1_degree2_checks_and_saturation(oracle_mod):
    """Checks of degree 1 (constant message: no gradient through it), 2 (a
    copy: derivative 1) and 3, and channel values strong enough that many
    variable-to-check messages sit on the clamp (no gradient through them).

    The differences here use large steps with Richardson extrapolation,
    (4 D(eps/2) - D(eps)) / 3 with D the central difference and eps = 1e-2,
    not eps = 1e-6: with saturated inputs the check rule evaluates atanh at
    products within ~1e-10 of 1, whose condition number (~1e10) turns FP64
    rounding into ~2e-9 of noise in the loss (measured: the loss difference
    over [-H, H] departs from the integral of the analytic gradient by ~2e-9
    whatever H is).  A 1e-6 step would divide that noise up to ~1e-3; the
    extrapolated large steps leave O(eps^4) truncation and ~4e-7 of noise."""
    code = gen.random_csr_code(42, 34, 2, {1: 4, 2: 10, 3: 20}, seed=77)
    cls, C, degrees = gen.edge_classes_by_check_degree(code)
    assert list(degrees) == [1, 2, 3]
    sigma = gen.sigma_for_capacity(code.rate / 0.5)
    fr = gen.make_frames(code, np.full(2, sigma), [8100, 8101])
    fr.llr = (fr.llr * 6.0).astype(np.float32)
    T = 4
    w = random_weights(T, C, 9)
    out = oracle_mod.wbp(code, fr.llr, fr.syndrome, fr.x, T, cls, w)
    assert np.abs(out["app"]).max() > 2 * LMAX  # messages saturate
    def central(k, c, eps):
        wp, wm = w.copy(), w.copy()
        wp[k, c] += eps
        wm[k, c] -= eps
        return (_loss(oracle_mod, code, fr.llr, fr, T, cls, wp)
                - _loss(oracle_mod, code, fr.llr, fr, T, cls, wm)) / (2 * eps)

    eps = 1e-2
    for k in range(T):
        for c in range(C):
            fd = (4.0 * central(k, c, eps / 2) - central(k, c, eps)) / 3.0
            assert fd == pytest.approx(out["grad_w"][k, c], rel=1e-4, abs=1e-8), (k, c)
    def central_llr(f, v, eps):
        lp, lm = fr.llr.copy(), fr.llr.copy()
        lp[f, v] += np.float32(eps)
        lm[f, v] -= np.float32(eps)
        assert lp[f, v] - fr.llr[f, v] == np.float32(eps)  # exact in float32
        return (_loss(oracle_mod, code, lp, fr, T, cls, w) - _loss(oracle_mod, code, lm, fr, T, cls, w)) / (2 * eps)

    eps = 2.0 ** -6
    for f, v in [(0, 0), (0, 5), (1, 17), (1, 41), (0, 30), (1, 2)]:
        fd = (4.0 * central_llr(f, v, eps / 2) - central_llr(f, v, eps)) / 3.0
        assert fd == pytest.approx(out["grad_llr"][f, v], rel=1e-4, abs=5e-7), (f, v)
