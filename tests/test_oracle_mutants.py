"""The oracle's pins catch plausible mistakes.

Each case below compiles a copy of oracle/bp_oracle.c with one deliberate,
plausible mistake (a dropped term, a wrong sign or index, a wrong order of the
termination tests, ...) and runs the pins of test_oracle_pins.py against it:
at least one pin must fail for every mutant.  The mistakes are planted in a
temporary copy of the oracle on the CPU only; the real oracle is untouched.
"""
import ctypes
import os
import subprocess

import pytest

import oracle
import test_oracle_pins as pins
import test_weighted_decode_pins as wpins

SRC = os.path.join(os.path.dirname(oracle.__file__), "bp_oracle.c")

PCE_BLOCK = """        if (rule != RULE_NONE && syndrome_ok(m, rowptr, colidx, xhat, s)) {
            success = 1; D = k; break;
        }
"""
VNR_BLOCK = """        if (rule == RULE_PCE_VNR && k >= vnr_first_iter && q < q_prev) {
            aborted = 1; D = k; break;
        }
"""

MUTANTS = {
    "syndrome sign dropped": [("double sgn = s[c] ? -1.0 : 1.0;", "double sgn = 1.0;")],
    "channel value dropped from APP": [("double L = Lch[v];", "double L = 0.0;")],
    "own c2v not excluded from v2c": [("if (b != a) sum += c2v[va->edge[b]];", "sum += c2v[va->edge[b]];")],
    "own v2c not excluded from c2v": [("if (f != e) prod *= tanh(0.5 * v2c[f]);", "prod *= tanh(0.5 * v2c[f]);")],
    "tanh of v2c instead of v2c/2": [("prod *= tanh(0.5 * v2c[f]);", "prod *= tanh(v2c[f]);")],
    "atanh without the factor 2": [("sgn * 2.0 * atanh(prod)", "sgn * atanh(prod)")],
    "c2v not clamped": [("c2v[e] = clampd(sgn * 2.0 * atanh(prod), lmax);", "c2v[e] = sgn * 2.0 * atanh(prod);")],
    "VNR comparison reversed": [("q < q_prev", "q > q_prev")],
    "signed q": [("if (va->ptr[v + 1] - va->ptr[v] > 1) q += fabs(app[v]);",
                  "if (va->ptr[v + 1] - va->ptr[v] > 1) q += app[v];")],
    "degree-1 variables counted in q": [("if (va->ptr[v + 1] - va->ptr[v] > 1) q += fabs(app[v]);",
                                         "if (va->ptr[v + 1] - va->ptr[v] > 0) q += fabs(app[v]);")],
    "first VNR test one iteration late": [("k >= vnr_first_iter && q < q_prev", "k > vnr_first_iter && q < q_prev")],
    "VNR tested before PCE": [(PCE_BLOCK + VNR_BLOCK, VNR_BLOCK + PCE_BLOCK)],
    "parity check ignores the syndrome": [("int par = s[c];", "int par = 0;")],
    "q history not updated": [("        q_prev = q;\n", "")],
    "learned weight ignores the edge class": [("* n_classes + edge_class[e]];", "* n_classes + 0];")],
    "past the last weight row, the first row is used": [("(k < w_iters ? k : w_iters) - 1", "(k < w_iters ? k : 1) - 1")],
}

PINS = [
    lambda o: [pins.test_trees_match_bruteforce_map(o, seed) for seed in range(3)],
    lambda o: [pins.test_trees_with_punctured_and_shortened_bits_match_bruteforce_map(o, seed) for seed in range(2)],
    pins.test_degree2_check_closed_form,
    pins.test_degree1_check_and_isolated_variable,
    pins.test_three_cycle_unsatisfiable_syndrome,
    pins.test_chain_success_wins_over_abort,
    pins.test_degree1_variables_excluded_from_q,
    pins.test_sign_symmetry_exact,
    pins.test_success_means_zero_syndrome,
    pins.test_noise_free_limit,
    lambda o: [wpins.test_unit_weights_are_the_plain_decoder(o, r) for r in (0, 2)],
    wpins.test_rule_none_equals_weighted_bp_forward,
    lambda o: [wpins.test_rows_past_the_last_repeat_it(o, r) for r in (0, 2)],
    wpins.test_zero_weights_closed_form,
]


class _MutantOracle:
    """The oracle module's decode() bound to a mutated library."""

    def __init__(self, lib):
        self._lib = lib
        for name in ("RULE_NONE", "RULE_PCE", "RULE_PCE_VNR", "FLAG_SUCCESS", "FLAG_ABORTED"):
            setattr(self, name, getattr(oracle, name))
        self.wbp = oracle.wbp  # the weighted-BP oracle is a separate library, not mutated here

    def decode(self, *args, **kwargs):
        saved = oracle._lib
        oracle._lib = self._lib
        try:
            return oracle.decode(*args, **kwargs)
        finally:
            oracle._lib = saved


def build_mutant(tmp_path, edits):
    src = open(SRC).read()
    for old, new in edits:
        assert old in src, f"mutation anchor not found: {old!r}"
        src = src.replace(old, new, 1)
    c = tmp_path / "mutant.c"
    c.write_text(src)
    so = tmp_path / "mutant.so"
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off", str(c),
                    "-o", str(so), "-lm"], check=True)
    lib = ctypes.CDLL(str(so))
    P, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.oracle_decode.argtypes = [i64, i64, P, P, i64, P, P, i32, i32, i32, dbl, P, P, P, P, i32, P, P, P, i32]
    lib.oracle_decode.restype = ctypes.c_int
    lib.oracle_decode_weighted.argtypes = [i64, i64, P, P, i64, P, P, i32, i32, i32, dbl, P, P, P, P, i32, P, P, P,
                                           i32, P, i32, i32, P]
    lib.oracle_decode_weighted.restype = ctypes.c_int
    lib.oracle_max_threads.restype = ctypes.c_int
    return lib


def test_unmutated_copy_passes_every_pin(tmp_path, oracle_mod):
    mutant = _MutantOracle(build_mutant(tmp_path, []))
    for pin in PINS:
        pin(mutant)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(tmp_path, oracle_mod, name):
    mutant = _MutantOracle(build_mutant(tmp_path, MUTANTS[name]))
    failed = []
    for pin in PINS:
        try:
            pin(mutant)
        except Exception:  # an assertion, or a numerical error the mistake causes
            failed.append(getattr(pin, "__name__", "pin"))
    assert failed, f"no pin catches the mutant '{name}'"
