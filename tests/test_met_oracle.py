"""Oracle-only evidence behind the parity reading for frames that never
converge: on the multi-edge-type code at beta = 0.85, a frame that runs to
D_max = 200 without meeting its syndrome ends on a decision that moves when
one channel value moves by one float32 ulp (a chaotic trajectory), while
frames that converge end on the same decision.  So the final bits of such a
failed frame are not a unique result; the GPU parity tests compare its flags
and iteration count and accept other bits only where this holds."""
import numpy as np

from paper_2507_03509_gb300 import gen
from _decode_helpers import decision_is_input_sensitive

Z = 64


def test_unconverged_frame_decision_moves_with_one_ulp(oracle_mod):
    code = gen.tbp_like_qc_code(Z)
    sigma = gen.sigma_for_capacity(code.rate / 0.85)
    fr = gen.make_frames(code, np.full(16, sigma), [7700 + 100 + f for f in range(16)])
    short = np.random.default_rng(1).choice(np.arange(8 * Z, code.n), size=64, replace=False)
    fr = gen.rate_adapt(fr, np.arange(Z), short)
    csr = code.to_csr()
    kw = dict(vnr_first_iter=2, lmax=25.0)
    out = oracle_mod.decode(csr, fr.llr, fr.syndrome, 200, oracle_mod.RULE_PCE)
    failed = np.nonzero((out["flags"] & 1) == 0)[0]
    done = np.nonzero(out["flags"] & 1)[0]
    assert failed.size >= 1 and done.size >= 4
    f = int(failed[0])
    assert decision_is_input_sensitive(oracle_mod, csr, fr.llr[f], fr.syndrome[f], 200, out["bits"][f], kw)
    for g in done[:3]:
        assert not decision_is_input_sensitive(oracle_mod, csr, fr.llr[g], fr.syndrome[g], int(out["iters"][g]),
                                               out["bits"][g], kw)
