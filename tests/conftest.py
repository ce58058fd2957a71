import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (sm_103a) and the built decoder library")
    config.addinivalue_line("markers", "slow: long-running (full-size workloads)")


@pytest.fixture(scope="session")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


def pytest_terminal_summary(terminalreporter):
    """Print how many frames of each decision comparison took the FP32 and the
    FP64 way out of exact agreement (tests/_decode_helpers.py caps both)."""
    helpers = sys.modules.get("_decode_helpers")
    tr = terminalreporter
    for e in getattr(helpers, "Q_LOG", None) or []:
        tr.write_line(f"q trace {e['case']}: max |q_gpu - q_oracle| / q_oracle = {e['max_rel']:.3g} over "
                      f"{e['iters']} iterations (tie band rtol_q = {e['rtol_q']:.3g})")
    log = getattr(helpers, "PARITY_LOG", None)
    if not log:
        return
    tr.write_sep("-", "decision parity: frames re-run in FP64 / accepted as FP64 near-ties")
    tot_f = tot32 = tot64 = 0
    for e in log:
        tot_f += e["frames"]
        tot32 += len(e["fp32_mismatch"])
        tot64 += len(e["fp64_ties"])
        tr.write_line(f"{e['test']} [{e['rule']}]: {len(e['fp32_mismatch'])}/{e['frames']} FP32 "
                      f"{e['fp32_mismatch'][:8]}, {len(e['fp64_ties'])} FP64 {e['fp64_ties']}")
    tr.write_line(f"total: {tot32} of {tot_f} frames re-run in FP64, {tot64} FP64 near-ties")
