"""The check-node arithmetic the CUDA kernels use, restated in FP64 numpy and
held against the paper's tanh/atanh rule (section "Early Termination").

The FP32 kernels do not evaluate 2 atanh(prod tanh(x/2)) as written, since
FP32 tanh(x/2) rounds to 1 beyond x ~ 17.  A magnitude x maps to r = e^{-x},
two magnitudes combine as (r_a + r_b) / (1 + r_a r_b), and the result is
-ln r; signs are carried apart.  The weighted-BP adjoint differentiates the
same form: d(a [+] B)/da = sgn(B) r_a (1 - r_B^2) / ((r_a + r_B)(1 + r_a r_B)).
These tests check both identities on grids, so the GPU parity tests measure
rounding only, not a reformulation.  CPU only; no product code is imported.
"""
import numpy as np
import pytest


def boxplus_tanh(a, b):
    """The paper's rule for two inputs: 2 atanh(tanh(a/2) tanh(b/2))."""
    return 2.0 * np.arctanh(np.tanh(a / 2.0) * np.tanh(b / 2.0))


def boxplus_r(a, b):
    """Sign and magnitude apart, magnitudes in the r = e^{-|x|} domain."""
    ra, rb = np.exp(-np.abs(a)), np.exp(-np.abs(b))
    mag = -np.log((ra + rb) / (1.0 + ra * rb))
    return np.sign(a) * np.sign(b) * mag


def exclusive_r(v):
    """Every exclusive combination of one check by prefix and suffix products
    in the r domain (what the kernels do for degree >= 3)."""
    d = len(v)
    r = np.exp(-np.abs(v))
    comb = lambda x, y: (x + y) / (1.0 + x * y)
    pre, suf = [None] * d, [None] * d
    pre[0] = r[0]
    for k in range(1, d):
        pre[k] = comb(pre[k - 1], r[k])
    suf[d - 1] = r[d - 1]
    for k in range(d - 2, -1, -1):
        suf[k] = comb(r[k], suf[k + 1])
    sg = np.prod(np.sign(v))
    out = []
    for k in range(d):
        ex = suf[1] if k == 0 else pre[d - 2] if k == d - 1 else comb(pre[k - 1], suf[k + 1])
        out.append(sg * np.sign(v[k]) * -np.log(ex))
    return np.array(out)


def exclusive_tanh(v):
    """The rule as written: 2 atanh of the product over the other inputs."""
    t = np.tanh(v / 2.0)
    return np.array([2.0 * np.arctanh(np.prod(np.delete(t, k))) for k in range(len(v))])


def test_pairwise_r_domain_equals_tanh_rule():
    # both arguments up to 16 in magnitude: there atanh of the FP64 product is
    # still well conditioned (tanh(8) = 1 - 2.3e-7), so the comparison is fair
    g = np.linspace(-16.0, 16.0, 321)
    a, b = np.meshgrid(g, g)
    want, got = boxplus_tanh(a, b), boxplus_r(a, b)
    assert np.allclose(got, want, rtol=1e-9, atol=1e-12)


def test_r_domain_keeps_precision_where_tanh_saturates():
    # a, b = 24, 30: the exact value is within e^-24 of min(|a|, |b|); the r
    # form gets it from the sum of two tiny r's, never from 1 - tanh
    got = boxplus_r(np.float64(24.0), np.float64(30.0))
    assert got == pytest.approx(24.0 - np.log1p(np.exp(-6.0)), rel=1e-12)
    # and it is odd in each argument, exactly
    assert boxplus_r(-24.0, 30.0) == -got and boxplus_r(24.0, -30.0) == -got


@pytest.mark.parametrize("d", [3, 4, 5, 7])
def test_prefix_suffix_exclusives_equal_the_rule_as_written(d):
    rng = np.random.default_rng(100 + d)
    for _ in range(200):
        v = rng.normal(0.0, 4.0, size=d)
        assert np.allclose(exclusive_r(v), exclusive_tanh(v), rtol=1e-9, atol=1e-12)


def test_degree_two_check_copies_the_other_message():
    # with one other input the exclusive combination is that input itself
    v = np.array([3.25, -0.5])
    assert np.allclose(exclusive_tanh(v), v[::-1], rtol=1e-14)


def dbox_r(a, b):
    """The adjoint's derivative d(a [+] b)/da in the r domain."""
    ra, rb = np.exp(-np.abs(a)), np.exp(-np.abs(b))
    return np.sign(b) * ra * (1.0 - rb * rb) / ((ra + rb) * (1.0 + ra * rb))


def test_adjoint_derivative_equals_central_differences():
    g = np.concatenate([np.linspace(-12.0, -0.05, 40), np.linspace(0.05, 12.0, 40)])
    a, b = np.meshgrid(g, g)
    h = 1e-6
    fd = (boxplus_tanh(a + h, b) - boxplus_tanh(a - h, b)) / (2.0 * h)
    assert np.allclose(dbox_r(a, b), fd, rtol=1e-5, atol=1e-7)


def test_adjoint_derivative_closed_form_by_hand():
    # d/da 2 atanh(tanh(a/2) t_b) = t_b (1 - tanh^2(a/2)) / (1 - tanh^2(a/2) t_b^2)
    a, b = 0.7, -1.9
    ta, tb = np.tanh(a / 2.0), np.tanh(b / 2.0)
    want = tb * (1.0 - ta * ta) / (1.0 - ta * ta * tb * tb)
    assert dbox_r(a, b) == pytest.approx(want, rel=1e-12)
