"""Pins for the FP64 oracle: values fixed by the mathematics, not by the oracle.

Each test checks the oracle against something independent of its own code:
brute-force MAP marginals where BP is exact (cycle-free graphs), closed forms
of degree-1 / degree-2 checks, hand-solved small graphs, exact sign symmetry,
an independent GF(2) product, and the noise-free limit.  The method is the
paper's section "Early Termination" (flooding BP, tanh/atanh check rule,
PCE-ET, VNR-ET over variable nodes of degree > 1).
"""
import itertools

import numpy as np
import pytest

from paper_2507_03509_gb300 import gen

pytestmark = pytest.mark.filterwarnings("ignore")

NONE, PCE, PCE_VNR = 0, 1, 2
SUCCESS, ABORTED = 1, 2


def csr_from_rows(n, rows):
    """CSR code from a list of column lists (one per check)."""
    rowptr = np.zeros(len(rows) + 1, dtype=np.int32)
    cols = []
    for i, r in enumerate(rows):
        r = sorted(r)
        cols.extend(r)
        rowptr[i + 1] = rowptr[i] + len(r)
    return gen.CSRCode(len(rows), n, rowptr, np.asarray(cols, dtype=np.int32))


def random_tree(rng, n_target):
    """Cycle-free Tanner graph: each new check joins one existing variable to
    1..3 new ones, so every check has degree >= 2."""
    rows = []
    n = 1
    while n < n_target:
        parent = int(rng.integers(0, n))
        k = int(min(rng.integers(1, 4), n_target - n))
        rows.append([parent] + list(range(n, n + k)))
        n += k
    return csr_from_rows(n, rows)


def brute_force_app(code, llr, s):
    """Exact bitwise MAP log-ratios ln P(x_v=0 | y, Hx=s) / P(x_v=1 | y, Hx=s)
    by enumerating all 2^n words."""
    n = code.n
    X = np.array(list(itertools.product([0, 1], repeat=n)), dtype=np.uint8)
    ok = np.ones(X.shape[0], dtype=bool)
    for c in range(code.m):
        cols = code.colidx[code.rowptr[c]:code.rowptr[c + 1]]
        ok &= (X[:, cols].sum(1) % 2) == s[c]
    X = X[ok]
    logw = (llr.astype(np.float64)[None, :] * (1.0 - 2.0 * X) / 2.0).sum(1)
    out = np.empty(n)
    for v in range(n):
        a = logw[X[:, v] == 0]
        b = logw[X[:, v] == 1]
        out[v] = np.logaddexp.reduce(a) - np.logaddexp.reduce(b)
    return out


@pytest.mark.parametrize("seed", range(8))
def test_trees_match_bruteforce_map(oracle_mod, seed):
    """BP is exact on cycle-free graphs: after enough flooding iterations the
    APP values equal the bitwise MAP log-ratios."""
    rng = np.random.default_rng(100 + seed)
    code = random_tree(rng, int(rng.integers(6, 13)))
    llr = (rng.standard_normal(code.n) * 0.9).astype(np.float32)
    s = rng.integers(0, 2, code.m).astype(np.uint8)
    exact = brute_force_app(code, llr, s)
    assert np.abs(exact).max() < 15.0  # the +-25 clamp is out of reach
    iters = 2 * (code.n + code.m)
    out = oracle_mod.decode(code, llr[None], s[None], iters, NONE, trace_iters=iters)
    app = out["app"][iters - 1, 0]
    np.testing.assert_allclose(app, exact, rtol=1e-10, atol=1e-10)
    assert (out["bits"][0] == (exact < 0)).all()
    assert out["iters"][0] == iters


@pytest.mark.parametrize("seed", range(6))
def test_trees_with_punctured_and_shortened_bits_match_bruteforce_map(oracle_mod, seed):
    """Rate adaptation on trees: punctured bits (Lch = 0) and shortened bits
    (Lch = +-100, known) leave BP exact; only the clamp of a shortened bit's
    own outgoing messages at 25 departs from MAP, by ~e^-25.  Trees where a
    free bit's MAP value reaches 15 (a shortened bit copied through a
    degree-2 check, where the clamp itself binds) are redrawn."""
    rng = np.random.default_rng(300 + seed)
    for _ in range(100):
        code = random_tree(rng, int(rng.integers(7, 13)))
        llr = (rng.standard_normal(code.n) * 0.9).astype(np.float32)
        perm = rng.permutation(code.n)
        punct, short = perm[: max(1, code.n // 4)], perm[code.n // 4: code.n // 4 + max(1, code.n // 6)]
        llr[punct] = 0.0
        llr[short] = (100.0 * rng.choice([-1.0, 1.0], size=short.size)).astype(np.float32)
        s = rng.integers(0, 2, code.m).astype(np.uint8)
        exact = brute_force_app(code, llr, s)
        free = np.setdiff1d(np.arange(code.n), short)
        if np.abs(exact[free]).max() < 15.0:
            break
    else:
        pytest.fail("no tree without a binding clamp drawn")
    iters = 2 * (code.n + code.m)
    out = oracle_mod.decode(code, llr[None], s[None], iters, NONE, final_app=True)
    np.testing.assert_allclose(out["app_final"][0], exact, rtol=1e-8, atol=1e-8)
    assert (out["bits"][0][short] == (llr[short] < 0)).all()


def test_degree2_check_closed_form(oracle_mod):
    """A degree-2 check passes the other variable's message on, sign set by
    its syndrome bit: c2v = (1 - 2 s) * v2c_other."""
    code = csr_from_rows(2, [[0, 1]])
    llr = np.array([[1.75, -0.625]], dtype=np.float32)
    for sbit in (0, 1):
        s = np.array([[sbit]], dtype=np.uint8)
        out = oracle_mod.decode(code, llr, s, 1, NONE, trace_iters=1)
        sg = 1.0 - 2.0 * sbit
        np.testing.assert_allclose(out["c2v"][0, 0], [sg * -0.625, sg * 1.75], rtol=1e-14)
        np.testing.assert_allclose(out["app"][0, 0], [1.75 + sg * -0.625, -0.625 + sg * 1.75],
                                   rtol=1e-14)


def test_degree1_check_and_isolated_variable(oracle_mod):
    """A degree-1 check forces its bit: c2v = (1 - 2 s) * LMAX; a variable in
    no check keeps its channel value."""
    # v0 in a degree-1 check c0 and a degree-2 check c1 with v1; v2 isolated.
    code = csr_from_rows(3, [[0], [0, 1]])
    llr = np.array([[0.5, 2.0, -3.0]], dtype=np.float32)
    for s0 in (0, 1):
        s = np.array([[s0, 0]], dtype=np.uint8)
        out = oracle_mod.decode(code, llr, s, 3, NONE, trace_iters=3, lmax=25.0)
        for k in range(3):
            assert out["c2v"][k, 0, 0] == (1.0 - 2.0 * s0) * 25.0
            assert out["app"][k, 0, 2] == -3.0
        assert out["bits"][0, 2] == 1


def test_three_cycle_unsatisfiable_syndrome(oracle_mod):
    """Hand-solved 3-cycle (checks v0v1, v1v2, v2v0) with syndrome (1,0,0),
    which no word satisfies.  Solving the degree-2 message recursion by hand
    for Lch = (a, b, c):
        APP(1) = (a-b+c, b-a+c, a+b+c), APP(2) = (a, b, c), APP(3) = (-a,-b,-c)
    so with (1, 2, 4): q(1) = 15 > q(2) = 7 and VNR-ET aborts at k = 2."""
    code = csr_from_rows(3, [[0, 1], [1, 2], [0, 2]])
    a, b, c = 1.0, 2.0, 4.0
    llr = np.array([[a, b, c]], dtype=np.float32)
    s = np.array([[1, 0, 0]], dtype=np.uint8)
    out = oracle_mod.decode(code, llr, s, 50, NONE, trace_iters=3)
    np.testing.assert_allclose(out["app"][0, 0], [a - b + c, b - a + c, a + b + c], rtol=1e-13)
    np.testing.assert_allclose(out["app"][1, 0], [a, b, c], rtol=1e-13)
    np.testing.assert_allclose(out["app"][2, 0], [-a, -b, -c], rtol=1e-13)
    # iteration-1 messages in CSR edge order: c0->(v0,v1), c1->(v1,v2), c2->(v0,v2)
    np.testing.assert_allclose(out["c2v"][0, 0], [-b, -a, c, b, c, a], rtol=1e-13)
    np.testing.assert_allclose(out["q"][:2, 0], [15.0, 7.0], rtol=1e-13)
    r = oracle_mod.decode(code, llr, s, 50, PCE_VNR)
    assert r["iters"][0] == 2 and r["flags"][0] == ABORTED
    assert (r["bits"][0] == 0).all()
    r1 = oracle_mod.decode(code, llr, s, 50, PCE_VNR, vnr_first_iter=1)  # q(0) = 7 < q(1)
    assert r1["iters"][0] == 2 and r1["flags"][0] == ABORTED
    for rule in (NONE, PCE):
        r = oracle_mod.decode(code, llr, s, 50, rule)
        assert r["iters"][0] == 50 and r["flags"][0] == 0


def test_chain_success_wins_over_abort(oracle_mod):
    """Hand-solved chain v0-c0-v1-c1-v2-c2-v3, zero syndrome, Lch = (a,b,c,d).
    APP(1) = (a+b, a+b+c, b+c+d, c+d), APP(2) = (a+b+c, S, S, b+c+d), S = a+b+c+d.
    With (-1.5, 1, 1, 0.25) the decision fails the checks at k = 1, meets them
    at k = 2, and q (over v1, v2) falls from 2.75 to 1.5 at k = 2: the parity
    test comes first, so the frame ends as a success at k = 2."""
    code = csr_from_rows(4, [[0, 1], [1, 2], [2, 3]])
    a, b, c, d = -1.5, 1.0, 1.0, 0.25
    S = a + b + c + d
    llr = np.array([[a, b, c, d]], dtype=np.float32)
    s = np.zeros((1, 3), dtype=np.uint8)
    out = oracle_mod.decode(code, llr, s, 5, NONE, trace_iters=2)
    np.testing.assert_allclose(out["app"][0, 0], [a + b, a + b + c, b + c + d, c + d], rtol=1e-13)
    np.testing.assert_allclose(out["app"][1, 0], [a + b + c, S, S, b + c + d], rtol=1e-13)
    np.testing.assert_allclose(out["q"][:, 0], [2.75, 1.5], rtol=1e-13)
    for rule in (PCE, PCE_VNR):
        r = oracle_mod.decode(code, llr, s, 5, rule)
        assert r["iters"][0] == 2 and r["flags"][0] == SUCCESS
        assert (r["bits"][0] == 0).all()


def test_degree1_variables_excluded_from_q(oracle_mod):
    """q sums |APP| only over variables of degree > 1: on the chain above only
    v1 and v2 count, so q(1) = |a+b+c| + |b+c+d| whatever v0 and v3 hold."""
    code = csr_from_rows(4, [[0, 1], [1, 2], [2, 3]])
    llr = np.array([[-9.0, 1.0, 1.0, 7.0]], dtype=np.float32)
    out = oracle_mod.decode(code, llr, np.zeros((1, 3), np.uint8), 1, NONE, trace_iters=1)
    assert out["q"][0, 0] == pytest.approx(abs(-9 + 1 + 1) + abs(1 + 1 + 7), rel=1e-13)


def test_sign_symmetry_exact(oracle_mod):
    """Flipping Lch by (1-2u) and the syndrome by H u flips decisions by u and
    every message sign on the matching edges; magnitudes, flags and iteration
    counts are unchanged, bit for bit."""
    rng = np.random.default_rng(7)
    code = gen.random_csr_code(240, 216, 3, {3: 144, 4: 72}, seed=77)
    fr = gen.make_frames(code, np.full(6, 1.4), seeds=range(500, 506))
    u = rng.integers(0, 2, size=(6, code.n)).astype(np.uint8)
    llr2 = (fr.llr * (1 - 2 * u.astype(np.float32))).astype(np.float32)
    s2 = fr.syndrome ^ gen.syndrome(code, u)
    for rule in (NONE, PCE, PCE_VNR):
        r1 = oracle_mod.decode(code, fr.llr, fr.syndrome, 40, rule, trace_iters=5)
        r2 = oracle_mod.decode(code, llr2, s2, 40, rule, trace_iters=5)
        assert (r2["bits"] == (r1["bits"] ^ u)).all()
        assert (r2["flags"] == r1["flags"]).all() and (r2["iters"] == r1["iters"]).all()
        ue = u[:, code.colidx].astype(np.float64)
        ran = ~np.isnan(r1["app"][:, :, 0])
        assert (r2["c2v"][ran] == (r1["c2v"] * (1 - 2 * ue)[None])[ran]).all()
        assert (r2["app"][ran] == (r1["app"] * (1 - 2 * u.astype(np.float64))[None])[ran]).all()
        assert (r2["q"][ran] == r1["q"][ran]).all()


def test_success_means_zero_syndrome(oracle_mod):
    """Every frame flagged as a success satisfies H x^ = s, checked with an
    independent GF(2) product; the decoded word is then a valid one."""
    code = gen.random_csr_code(600, 300, 3, {6: 300}, seed=91)
    fr = gen.make_frames(code, np.full(24, 0.62), seeds=range(900, 924))
    for rule in (PCE, PCE_VNR, NONE):
        r = oracle_mod.decode(code, fr.llr, fr.syndrome, 60, rule)
        succ = (r["flags"] & SUCCESS) > 0
        assert succ.sum() >= 12
        synd = gen.syndrome(code, r["bits"])
        assert ((synd == fr.syndrome).all(1) == succ).all()


def test_noise_free_limit(oracle_mod):
    """With certain channel values (+-30) the first decision is the sent word:
    PCE-ET stops at k = 1 with success."""
    code = gen.workload_code(1)
    rng = np.random.default_rng(3)
    x = rng.integers(0, 2, size=(4, code.n)).astype(np.uint8)
    llr = (30.0 * (1.0 - 2.0 * x)).astype(np.float32)
    s = gen.syndrome(code, x)
    for rule in (PCE, PCE_VNR):
        r = oracle_mod.decode(code, llr, s, 20, rule)
        assert (r["iters"] == 1).all() and (r["flags"] == SUCCESS).all()
        assert (r["bits"] == x).all()
    r = oracle_mod.decode(code, llr, s, 7, NONE)
    assert (r["iters"] == 7).all() and (r["flags"] == SUCCESS).all() and (r["bits"] == x).all()


def test_rule_none_runs_every_iteration(oracle_mod):
    code = gen.workload_code(1)
    fr = gen.workload_frames(1, code, frames=3)
    r = oracle_mod.decode(code, fr.llr, fr.syndrome, 9, NONE)
    assert (r["iters"] == 9).all()
    assert ((r["flags"] & ABORTED) == 0).all()
