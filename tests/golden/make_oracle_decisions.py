"""Write the FP64 oracle's per-frame decisions for a named workload.

Calls only the oracle (oracle/) and the seeded input generators; the values
it stores are the expected decisions that the full-size parity tests and the
CPU baseline use (the decoder is never involved).

Usage: python tests/golden/make_oracle_decisions.py <workload-number> <rule> [threads]
Writes tests/golden/oracle_<workload name>_<rule>.txt with one line per frame:
    frame iters flags bit_errors sha256(bits)
"""
import hashlib
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_2507_03509_gb300 import gen  # noqa: E402

RULES = {"none": 0, "pce": 1, "pce_vnr": 2}


def main():
    number = int(sys.argv[1])
    rule = sys.argv[2]
    threads = int(sys.argv[3]) if len(sys.argv) > 3 else 0
    w = gen.WORKLOADS[number]
    if w["kind"] == "batch":
        return main_batch(number, rule, threads)
    code = gen.workload_code(number)
    csr = code.to_csr() if hasattr(code, "to_csr") else code
    frames = gen.workload_frames(number, code)
    t0 = time.time()
    out = oracle.decode(csr, frames.llr, frames.syndrome, w["max_iter"], RULES[rule], threads=threads)
    dt = time.time() - t0
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"oracle_{w['name']}_{rule}.txt")
    with open(path, "w") as fh:
        fh.write(f"# FP64 oracle decisions: workload {w['name']} (frames {w['frames']}, beta {w['beta']},"
                 f" max_iter {w['max_iter']}), rule {rule}, vnr_first_iter 2, clamp 25\n")
        fh.write("# written by tests/golden/make_oracle_decisions.py (oracle only)\n")
        fh.write(f"# oracle wall time {dt:.1f} s, threads {threads or oracle.max_threads()}\n")
        fh.write("# frame iters flags bit_errors sha256(bits)\n")
        for f in range(frames.llr.shape[0]):
            bits = out["bits"][f]
            errs = int((bits != frames.x[f]).sum())
            digest = hashlib.sha256(np.ascontiguousarray(bits).tobytes()).hexdigest()
            fh.write(f"{f} {int(out['iters'][f])} {int(out['flags'][f])} {errs} {digest}\n")
    print(path, f"{dt:.1f}s")


def main_batch(number, rule, threads):
    """Frames of several codes: each code's frames decoded by the oracle with
    that code; lines in batch order."""
    w = gen.WORKLOADS[number]
    codes = gen.batch_codes(number)
    bf = gen.workload_batch(number, codes)
    F = bf.frame_code.size
    rows = [None] * F
    t0 = time.time()
    for c, code in enumerate(codes):
        idx = np.nonzero(bf.frame_code == c)[0]
        if idx.size == 0:
            continue
        csr = code.to_csr()
        llr = np.stack([bf.llr[bf.var_off[f]:bf.var_off[f + 1]] for f in idx])
        syn = np.stack([bf.syndrome[bf.syn_off[f]:bf.syn_off[f + 1]] for f in idx])
        out = oracle.decode(csr, llr, syn, w["max_iter"], RULES[rule], threads=threads)
        for i, f in enumerate(idx):
            bits = out["bits"][i]
            errs = int((bits != bf.x[bf.var_off[f]:bf.var_off[f + 1]]).sum())
            digest = hashlib.sha256(np.ascontiguousarray(bits).tobytes()).hexdigest()
            rows[f] = f"{f} {int(out['iters'][i])} {int(out['flags'][i])} {errs} {digest}\n"
    dt = time.time() - t0
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"oracle_{w['name']}_{rule}.txt")
    with open(path, "w") as fh:
        fh.write(f"# FP64 oracle decisions: workload {w['name']} (frames {F}, beta ~ U[{w['beta_lo']}, "
                 f"{w['beta_hi']}] per frame, max_iter {w['max_iter']}), rule {rule}, vnr_first_iter 2, clamp 25\n")
        fh.write("# written by tests/golden/make_oracle_decisions.py (oracle only)\n")
        fh.write(f"# oracle wall time {dt:.1f} s, threads {threads or oracle.max_threads()}\n")
        fh.write("# frame iters flags bit_errors sha256(bits)\n")
        fh.writelines(rows)
    print(path, f"{dt:.1f}s")


if __name__ == "__main__":
    main()
