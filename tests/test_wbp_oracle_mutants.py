"""The weighted-BP oracle's pins catch plausible mistakes.

Each case compiles a copy of oracle/wbp_oracle.c with one deliberate mistake
(a dropped mask, a missing sign, an exclusive sum that includes its own term,
a weight taken from the wrong iteration, ...) and runs the pins of
test_wbp_oracle_pins.py against it: at least one pin must fail for every
mutant.  The mistakes are planted in a temporary copy on the CPU only.
"""
import ctypes
import os
import subprocess

import pytest

import oracle
import test_wbp_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "wbp_oracle.c")

MUTANTS = {
    "variable-side clamp passes the gradient": [("du[j] = fabs(u[j]) <= lmax ? da : 0.0;", "du[j] = da;")],
    "syndrome sign missing in the backward pass": [("da += dt[e] * sgn * dphi;", "da += dt[e] * dphi;")],
    "own term kept in the backward exclusive sum": [("if (b != a) ex += du[g->vedge[b]];",
                                                     "ex += du[g->vedge[b]];")],
    "weight of the previous iteration used": [("cnew[e] = w[(size_t)(k - 1) * n_classes + cls[e]] * val;",
                                               "cnew[e] = w[(size_t)(k > 1 ? k - 2 : 0) * n_classes + cls[e]] * val;")],
    "weight left out of the backward pass": [("(e1 - e0 == 1) ? 0.0 : G[e] * wk[cls[e]];",
                                              "(e1 - e0 == 1) ? 0.0 : G[e];")],
    "sigmoid argument sign flipped": [("-sx * sigmoid(-sx * app[v]) * scale", "-sx * sigmoid(sx * app[v]) * scale")],
    "derivative without the sech^2 factor": [("(1.0 - tj * tj) * rest / (1.0 - P * P)", "rest / (1.0 - P * P)")],
    "direct channel term missing from the gradient": [("        gl[v] = gv;\n", "        gl[v] = 0.0;\n")],
    "weight gradient uses the weighted message": [("gwk[cls[e]] += G[e] * t[e];",
                                                   "gwk[cls[e]] += G[e] * t[e] * wk[cls[e]];")],
    "loss not averaged over bits": [("const double scale = (frames > 0 && n > 0) ? 1.0 / ((double)frames * (double)n) : 0.0;",
                                     "const double scale = (frames > 0 && n > 0) ? 1.0 / (double)frames : 0.0;")],
    "variable-side clamp missing in the forward pass": [("if (f != e) prod *= tanh(0.5 * clamp_lim(u[f], lmax));",
                                                         "if (f != e) prod *= tanh(0.5 * u[f]);")],
}

PINS = [
    pins.test_unit_weights_reproduce_the_decoder_oracle,
    pins.test_weight_gradient_matches_finite_differences,
    pins.test_channel_gradient_matches_finite_differences,
    pins.test_zero_weights_closed_form,
    pins.test_sign_symmetry_bit_exact,
    pins.test_gradient_fd_with_degree1_degree2_checks_and_saturation,
]


class _MutantOracle:
    """The oracle module with wbp() bound to a mutated library."""

    def __init__(self, lib):
        self._lib = lib
        self.decode = oracle.decode
        for name in ("RULE_NONE", "RULE_PCE", "RULE_PCE_VNR"):
            setattr(self, name, getattr(oracle, name))

    def wbp(self, *args, **kwargs):
        return oracle.wbp(*args, lib=self._lib, **kwargs)


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
    return oracle._bind_wbp(ctypes.CDLL(str(so)))


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
            failed.append(pin.__name__)
    assert failed, f"no pin catches the mutant '{name}'"
