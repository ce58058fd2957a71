"""FP64 CPU oracle for syndrome-based sum-product decoding with early termination.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package.  It is independent of the CUDA
decoder: it shares no source, header, table or helper with it, and imports
nothing from the product package.

The arithmetic lives in ``bp_oracle.c`` (plain C, FP64, OpenMP over frames);
this module compiles it with gcc on first use and marshals arguments.

The weighted-BP reference (weights per iteration and edge class, T unrolled
iterations, binary cross-entropy loss and its exact reverse-mode gradient)
lives in ``wbp_oracle.c`` and is built the same way into its own library.

Parity status of each function (what pins it, tests/test_oracle_pins.py and
tests/test_wbp_oracle_pins.py):
  decode  -- pinned: brute-force bitwise MAP marginals on cycle-free graphs,
             closed forms of degree-1 and degree-2 checks, a hand-solved
             3-cycle with an unsatisfiable syndrome (APP values, q sequence,
             VNR abort iteration), channel/syndrome sign symmetry, zero
             syndrome on every success (independent GF(2) product), the
             noise-free limit.
  wbp     -- pinned: unit weights reproduce decode()'s APP after T
             iterations; the gradient equals central finite differences of the
             loss (eps 1e-6) for every weight and for sampled channel values;
             all-zero weights give APP = Lch and a gradient written out by hand
             in the test; sign symmetry of loss and gradient (bit-exact).
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


_WSRC = os.path.join(_HERE, "wbp_oracle.c")
_WLIB = os.path.join(_HERE, "_wbp_oracle.so")
_wlib = None


def _compile(src: str, lib: str, force: bool) -> str:
    if not force and os.path.exists(lib) and os.path.getmtime(lib) >= os.path.getmtime(src):
        return lib
    tmp = lib + f".{os.getpid()}.tmp"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", src, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


def build(force: bool = False) -> str:
    """Compile bp_oracle.c and wbp_oracle.c into their libraries (gcc, OpenMP,
    no FP contraction); returns the decoder library's path."""
    _compile(_WSRC, _WLIB, force)
    return _compile(_SRC, _LIB, force)


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
            lib.oracle_decode_weighted.argtypes = [i64, i64, P, P, i64, P, P, i32, i32, i32, dbl,
                                                   P, P, P, P, i32, P, P, P, i32, P, i32, i32, P]
            lib.oracle_decode_weighted.restype = ctypes.c_int
            lib.oracle_max_threads.restype = ctypes.c_int
            _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().oracle_max_threads())


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def decode(code, llr, syndrome, max_iter: int, rule: int = RULE_PCE_VNR,
           vnr_first_iter: int = 2, lmax: float = 25.0, trace_iters: int = 0,
           threads: int = 0, trace=("c2v", "app", "q"), final_app: bool = False, weights=None,
           edge_class=None):
    """Decode frames with the FP64 oracle.

    code: any object with m, n, rowptr, colidx (check-major CSR, columns sorted).
    llr: float32 [F, n]; syndrome: uint8 [F, m] (0/1).
    weights [w_iters, C] with edge_class [E] (CSR order): learned weights on
    the check-to-variable messages, row min(k, w_iters) in iteration k.
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
    args = (m, n, _ptr(rowptr), _ptr(colidx), F, _ptr(llr), _ptr(syndrome), int(max_iter), int(rule),
            int(vnr_first_iter), float(lmax), _ptr(bits), _ptr(flags), _ptr(iters), _ptr(af), T, _ptr(tc),
            _ptr(ta), _ptr(tq), int(threads))
    if weights is None:
        rc = lib.oracle_decode(*args)
    else:
        w = np.ascontiguousarray(weights, dtype=np.float64)
        cls = np.ascontiguousarray(edge_class, dtype=np.int32)
        if w.ndim != 2 or cls.shape != (E,):
            raise ValueError("weights [w_iters, classes] and edge_class [E] expected")
        rc = lib.oracle_decode_weighted(*args, _ptr(w), int(w.shape[0]), int(w.shape[1]), _ptr(cls))
    if rc != 0:
        raise RuntimeError("oracle_decode failed (bad arguments or out of memory)")
    out = dict(bits=bits, flags=flags, iters=iters)
    if final_app:
        out["app_final"] = af
    for key, arr in (("c2v", tc), ("app", ta), ("q", tq)):
        if arr is not None:
            out[key] = arr
    return out


def _load_wbp():
    global _wlib
    with _lock:
        if _wlib is None:
            _wlib = _bind_wbp(ctypes.CDLL(_compile(_WSRC, _WLIB, False)))
    return _wlib


def _bind_wbp(lib):
    P = ctypes.c_void_p
    i64, i32, dbl = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    lib.oracle_wbp.argtypes = [i64, i64, P, P, i64, P, P, P, i32, i32, P, P, dbl, P, P, P, P, i32]
    lib.oracle_wbp.restype = ctypes.c_int
    return lib


def wbp(code, llr, syndrome, x, iters: int, edge_class, weights, lmax: float = 25.0, grad: bool = True,
        threads: int = 0, lib=None):
    """Weighted BP over T = iters unrolled iterations, loss and gradient (FP64).

    code: m, n, rowptr, colidx (check-major CSR); llr float32 [F, n];
    syndrome uint8 [F, m]; x uint8 [F, n] (the bits the loss compares with);
    edge_class int [E] in CSR edge order; weights float [T, C].
    Returns dict(app [F, n], loss float, and with grad: grad_w [T, C],
    grad_llr [F, n]).
    """
    lib = lib or _load_wbp()
    llr = np.ascontiguousarray(llr, dtype=np.float32)
    syndrome = np.ascontiguousarray(syndrome, dtype=np.uint8)
    x = np.ascontiguousarray(x, dtype=np.uint8)
    if llr.ndim == 1:
        llr, syndrome, x = llr[None], syndrome[None], x[None]
    F = llr.shape[0]
    m, n = int(code.m), int(code.n)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    T, C = int(iters), int(w.shape[1])
    if w.shape != (T, C) or llr.shape != (F, n) or syndrome.shape != (F, m) or x.shape != (F, n):
        raise ValueError("shapes do not match the code / iterations")
    rowptr = np.ascontiguousarray(code.rowptr, dtype=np.int64)
    colidx = np.ascontiguousarray(code.colidx, dtype=np.int32)
    cls = np.ascontiguousarray(edge_class, dtype=np.int32)
    if cls.shape != (int(rowptr[-1]),):
        raise ValueError("edge_class must hold one class per edge")
    app = np.zeros((F, n))
    loss = np.zeros(1)
    gw = np.zeros((T, C)) if grad else None
    gl = np.zeros((F, n)) if grad else None
    rc = lib.oracle_wbp(m, n, _ptr(rowptr), _ptr(colidx), F, _ptr(llr), _ptr(syndrome), _ptr(x), T, C,
                        _ptr(cls), _ptr(w), float(lmax), _ptr(app), _ptr(loss), _ptr(gw), _ptr(gl),
                        int(threads))
    if rc != 0:
        raise RuntimeError("oracle_wbp failed (bad arguments or out of memory)")
    out = dict(app=app, loss=float(loss[0]))
    if grad:
        out.update(grad_w=gw, grad_llr=gl)
    return out
