"""Pins of the decoder oracle's learned-weight mode (oracle_decode_weighted):
the early-terminating decoder with check-to-variable messages of iteration k
scaled by w[min(k, w_iters) - 1][class(e)].

- Unit weights: bit-identical to the unweighted decoder, for every rule.
- Rule NONE for T iterations with T weight rows: the APP equals the forward
  pass of the weighted-BP oracle (wbp_oracle.c, an independent implementation
  pinned to finite differences and the decoder oracle).
- Iterations past the last row reuse it: weights [3, C] decode like the same
  weights with the last row repeated to max_iter rows.
- Zero weights: every message vanishes, APP = Lch, q is constant (so VNR-ET
  never fires: the test is strict), and PCE-ET succeeds at k = 1 exactly when
  the channel's hard decision meets the syndrome.
"""
import numpy as np
import pytest

from paper_2507_03509_gb300 import gen


def setup(frames=4, beta=0.9, seed=0):
    code = gen.wbp_fd_code()
    cls, C, _ = gen.edge_classes_by_check_degree(code)
    sigma = gen.sigma_for_capacity(code.rate / beta)
    fr = gen.make_frames(code, np.full(frames, sigma), [9900 + 10 * seed + f for f in range(frames)])
    return code, cls, C, fr


@pytest.mark.parametrize("rule", [0, 1, 2])
def test_unit_weights_are_the_plain_decoder(oracle_mod, rule):
    code, cls, C, fr = setup()
    a = oracle_mod.decode(code, fr.llr, fr.syndrome, 30, rule, trace_iters=5, final_app=True)
    b = oracle_mod.decode(code, fr.llr, fr.syndrome, 30, rule, trace_iters=5, final_app=True,
                          weights=np.ones((7, C)), edge_class=cls)
    for k in ("bits", "flags", "iters", "app_final", "c2v", "app", "q"):
        assert np.array_equal(a[k], b[k], equal_nan=True), k


def test_rule_none_equals_weighted_bp_forward(oracle_mod):
    code, cls, C, fr = setup(seed=1)
    T = 9
    w = np.random.default_rng(2).uniform(0.6, 1.3, size=(T, C))
    d = oracle_mod.decode(code, fr.llr, fr.syndrome, T, 0, final_app=True, weights=w, edge_class=cls)
    f = oracle_mod.wbp(code, fr.llr, fr.syndrome, fr.x, T, cls, w, grad=False)
    np.testing.assert_allclose(d["app_final"], f["app"], rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("rule", [0, 2])
def test_rows_past_the_last_repeat_it(oracle_mod, rule):
    code, cls, C, fr = setup(seed=2)
    w = np.random.default_rng(3).uniform(0.6, 1.3, size=(3, C))
    full = np.concatenate([w, np.repeat(w[-1:], 17, axis=0)])
    a = oracle_mod.decode(code, fr.llr, fr.syndrome, 20, rule, final_app=True, weights=w, edge_class=cls)
    b = oracle_mod.decode(code, fr.llr, fr.syndrome, 20, rule, final_app=True, weights=full, edge_class=cls)
    for k in ("bits", "flags", "iters", "app_final"):
        assert np.array_equal(a[k], b[k]), k


def test_zero_weights_closed_form(oracle_mod):
    code, cls, C, fr = setup(frames=6, seed=3)
    # two frames whose channel decision meets the syndrome by construction
    fr.syndrome[:2] = gen.syndrome(code, (fr.llr[:2] < 0).astype(np.uint8))
    w = np.zeros((2, C))
    out = oracle_mod.decode(code, fr.llr, fr.syndrome, 12, 2, final_app=True, trace_iters=12,
                            weights=w, edge_class=cls)
    assert (out["app_final"] == fr.llr.astype(np.float64)).all()
    meets = (gen.syndrome(code, (fr.llr < 0).astype(np.uint8)) == fr.syndrome).all(1)
    assert meets[:2].all() and not meets[2:].any()
    assert (out["iters"][meets] == 1).all() and (out["flags"][meets] == 1).all()
    assert (out["iters"][~meets] == 12).all() and (out["flags"][~meets] == 0).all()
    q = out["q"][:, ~meets]
    assert (q == q[0]).all()
