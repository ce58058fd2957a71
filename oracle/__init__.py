"""FP64 CPU oracle for syndrome-based sum-product decoding with early termination.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package.  It is independent of the CUDA
decoder: it shares no source, header, table or helper with it, and imports
nothing from the product package.

The arithmetic lives in ``bp_oracle.c`` (plain C, FP64, OpenMP over frames);
this module compiles it with gcc on first use and marshals arguments.

Parity status of each function (what pins it, tests/test_oracle_pins.py):
  decode  -- pinned: brute-force bitwise MAP marginals on cycle-free graphs,
             closed forms of degree-1 and degree-2 checks, a hand-solved
             3-cycle with an unsatisfiable syndrome (APP values, q sequence,
             VNR abort iteration), channel/syndrome sign symmetry, zero
             syndrome on every success (independent GF(2) product), the
             noise-free limit.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bp_oracle.c")
_LIB = os.path.join(_HERE, "_bp_oracle.so")
_lock = threading.Lock()
_lib = None

RULE_NONE, RULE_PCE, RULE_PCE_VNR = 0, 1, 2
FLAG_SUCCESS, FLAG_ABORTED = 1, 2


def build(force: bool = False) -> str:
    """Compile bp_oracle.c into _bp_oracle.so (gcc, OpenMP, no FP contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.c_void_p
            i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            lib.oracle_decode.argtypes = [i64, i64, P, P, i64, P, P, i32, i32, i32, dbl,
                                          P, P, P, P, i32, P, P, P, i32]
            lib.oracle_decode.restype = ctypes.c_int
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def decode(code, llr, syndrome, max_iter: int, rule: int = RULE_PCE_VNR,
           vnr_first_iter: int = 2, lmax: float = 25.0, trace_iters: int = 0,
           threads: int = 0, trace=("c2v", "app", "q"), final_app: bool = False):
    """Decode frames with the FP64 oracle.

    code: any object with m, n, rowptr, colidx (check-major CSR, columns sorted).
    llr: float32 [F, n]; syndrome: uint8 [F, m] (0/1).
    Returns dict(bits uint8 [F,n], flags uint8 [F], iters int32 [F]); with
    final_app, app_final float64 [F,n] (APP of the last iteration run); and,
    if trace_iters > 0, the traces named in `trace`: c2v float64 [T,F,E] (CSR
    edge order), app [T,F,n], q [T,F] (NaN where a frame stopped earlier).
    """
    lib = _load()
    llr = np.ascontiguousarray(llr, dtype=np.float32)
    syndrome = np.ascontiguousarray(syndrome, dtype=np.uint8)
    if llr.ndim == 1:
        llr = llr[None]
    if syndrome.ndim == 1:
        syndrome = syndrome[None]
    F = llr.shape[0]
    m, n = int(code.m), int(code.n)
    if llr.shape != (F, n) or syndrome.shape != (F, m):
        raise ValueError("llr / syndrome shapes do not match the code")
    rowptr = np.ascontiguousarray(code.rowptr, dtype=np.int64)
    colidx = np.ascontiguousarray(code.colidx, dtype=np.int32)
    E = int(rowptr[-1])
    bits = np.zeros((F, n), dtype=np.uint8)
    flags = np.zeros(F, dtype=np.uint8)
    iters = np.zeros(F, dtype=np.int32)
    T = int(trace_iters)
    tc = np.full((T, F, E), np.nan) if T > 0 and "c2v" in trace else None
    ta = np.full((T, F, n), np.nan) if T > 0 and "app" in trace else None
    tq = np.full((T, F), np.nan) if T > 0 and "q" in trace else None
    af = np.zeros((F, n)) if final_app else None
    rc = lib.oracle_decode(m, n, _ptr(rowptr), _ptr(colidx), F, _ptr(llr), _ptr(syndrome),
                           int(max_iter), int(rule), int(vnr_first_iter), float(lmax),
                           _ptr(bits), _ptr(flags), _ptr(iters), _ptr(af), T, _ptr(tc), _ptr(ta),
                           _ptr(tq), int(threads))
    if rc != 0:
        raise RuntimeError("oracle_decode failed (bad arguments or out of memory)")
    out = dict(bits=bits, flags=flags, iters=iters)
    if final_app:
        out["app_final"] = af
    for key, arr in (("c2v", tc), ("app", ta), ("q", tq)):
        if arr is not None:
            out[key] = arr
    return out
