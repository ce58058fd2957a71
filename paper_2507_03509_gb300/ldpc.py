"""Python binding of the decoder's C ABI (include/ldpc.h): argument marshalling only.

Every step of decoding runs in the CUDA library ``libldpc_gb300.so``; this
module only passes pointers, sizes and the current CUDA stream.  Importing it
raises ImportError when the library has not been built -- there is no
fallback decoder.

The functions keep the C names (``ldpc_graph_create_csr``,
``ldpc_graph_create_qc``, ``ldpc_graph_destroy``, ``ldpc_graph_info``,
``ldpc_decode``, ``ldpc_decode_host``, ``ldpc_status_str``); ``Graph`` and
``decode`` are small conveniences on top.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

# LDPC_GB300_CHECKED=1 selects the index-checking build (a debug aid, compiled with -DLDPC_BOUNDS_CHECK)
_CHECKED = os.environ.get("LDPC_GB300_CHECKED", "0") not in ("", "0")
_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)),
                         "libldpc_gb300_checked.so" if _CHECKED else "libldpc_gb300.so")

LDPC_OK = 0
LDPC_ERR_INVALID_ARG = 1
LDPC_ERR_INVALID_GRAPH = 2
LDPC_ERR_OOM = 3
LDPC_ERR_CUDA = 4
LDPC_ERR_TIMEOUT = 5
LDPC_ERR_TOO_LARGE = 6
LDPC_ERR_BOUNDS = 7

LDPC_TERM_NONE = 0
LDPC_TERM_PCE = 1
LDPC_TERM_PCE_VNR = 2

LDPC_FLAG_SUCCESS = 1
LDPC_FLAG_ABORTED = 2

RULES = {"none": LDPC_TERM_NONE, "pce": LDPC_TERM_PCE, "pce_vnr": LDPC_TERM_PCE_VNR}

EXPORTED = ("ldpc_decode_opts_init", "ldpc_graph_create_csr", "ldpc_graph_create_qc",
            "ldpc_graph_destroy", "ldpc_graph_info", "ldpc_decode", "ldpc_decode_host",
            "ldpc_status_str", "ldpc_decode_qc_noalloc", "ldpc_batch_create", "ldpc_batch_destroy",
            "ldpc_batch_info", "ldpc_batch_decode", "ldpc_batch_decode_async", "ldpc_batch_autotune",
            "ldpc_wbp_create", "ldpc_wbp_destroy", "ldpc_wbp_forward", "ldpc_wbp_loss", "ldpc_wbp_backward",
            "ldpc_wbp_sgd_step", "ldpc_wbp_decode", "ldpc_graph_check_guards", "ldpc_batch_check_guards")

NOALLOC_SCRATCH_BYTES = 64 * 1024 * 1024


class ldpc_decode_stats(ctypes.Structure):
    _fields_ = [("kernel_ms", ctypes.c_float), ("total_ms", ctypes.c_float),
                ("kernel_launches", ctypes.c_int32), ("grid_ctas", ctypes.c_int32),
                ("threads_per_cta", ctypes.c_int32), ("active_frames", ctypes.c_int32),
                ("frame_iterations", ctypes.c_int64)]


class ldpc_decode_opts(ctypes.Structure):
    _fields_ = [("vnr_first_iter", ctypes.c_int32), ("clamp", ctypes.c_float),
                ("fp64", ctypes.c_int32), ("max_active_frames", ctypes.c_int32),
                ("grid_ctas", ctypes.c_int32), ("trace_iters", ctypes.c_int32),
                ("trace_c2v", ctypes.c_void_p), ("trace_app", ctypes.c_void_p),
                ("trace_q", ctypes.c_void_p), ("stats", ctypes.POINTER(ldpc_decode_stats)),
                ("barrier_timeout_ms", ctypes.c_int32), ("test_unreachable_barrier", ctypes.c_int32),
                ("groups", ctypes.c_int32), ("schedule", ctypes.c_int32), ("flow_lag", ctypes.c_int32),
                ("debug_guards", ctypes.c_int32)]

SCHEDULES = {"auto": 0, "lockstep": 1, "dataflow": 2, "frame": 3, "frame_pair": 4}


def _load():
    if not os.path.exists(_LIB_PATH):
        raise ImportError(f"decoder library {_LIB_PATH} is missing: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
    lib = ctypes.CDLL(_LIB_PATH)
    P, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    pg = ctypes.POINTER(P)
    lib.ldpc_decode_opts_init.argtypes = [ctypes.POINTER(ldpc_decode_opts)]
    lib.ldpc_decode_opts_init.restype = None
    lib.ldpc_graph_create_csr.argtypes = [i32, i32, P, P, pg]
    lib.ldpc_graph_create_csr.restype = ctypes.c_int
    lib.ldpc_graph_create_qc.argtypes = [i32, i32, i32, P, pg]
    lib.ldpc_graph_create_qc.restype = ctypes.c_int
    lib.ldpc_graph_destroy.argtypes = [P]
    lib.ldpc_graph_destroy.restype = None
    lib.ldpc_graph_info.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i64)]
    lib.ldpc_graph_info.restype = ctypes.c_int
    dec = [P, i32, P, P, i32, ctypes.c_int, P, P, P, ctypes.POINTER(ldpc_decode_opts), P]
    lib.ldpc_decode.argtypes = dec
    lib.ldpc_decode.restype = ctypes.c_int
    lib.ldpc_decode_host.argtypes = dec
    lib.ldpc_decode_host.restype = ctypes.c_int
    lib.ldpc_status_str.argtypes = [ctypes.c_int]
    lib.ldpc_status_str.restype = ctypes.c_char_p
    lib.ldpc_decode_qc_noalloc.argtypes = [i32, i32, i32, P, i32, P, P, i32, ctypes.c_int, P, P, P, P]
    lib.ldpc_decode_qc_noalloc.restype = ctypes.c_int
    lib.ldpc_batch_create.argtypes = [P, i32, i32, P, pg]
    lib.ldpc_batch_create.restype = ctypes.c_int
    lib.ldpc_batch_destroy.argtypes = [P]
    lib.ldpc_batch_destroy.restype = None
    lib.ldpc_batch_info.argtypes = [P, ctypes.POINTER(i32), ctypes.POINTER(i64), ctypes.POINTER(i64)]
    lib.ldpc_batch_info.restype = ctypes.c_int
    lib.ldpc_batch_decode.argtypes = [P, P, P, i32, ctypes.c_int, P, P, P, ctypes.POINTER(ldpc_decode_opts), P]
    lib.ldpc_batch_decode.restype = ctypes.c_int
    lib.ldpc_batch_decode_async.argtypes = [P, P, P, i32, ctypes.c_int, P, P, P, P,
                                            ctypes.POINTER(ldpc_decode_opts), P]
    lib.ldpc_batch_decode_async.restype = ctypes.c_int
    lib.ldpc_batch_autotune.argtypes = [P, P, P, i32, ctypes.c_int, P, P, P, P, ctypes.POINTER(i32),
                                        ctypes.POINTER(i32)]
    lib.ldpc_batch_autotune.restype = ctypes.c_int
    lib.ldpc_wbp_create.argtypes = [P, i32, i32, i32, P, i32, i32, pg]
    lib.ldpc_wbp_create.restype = ctypes.c_int
    lib.ldpc_wbp_destroy.argtypes = [P]
    lib.ldpc_wbp_destroy.restype = None
    lib.ldpc_wbp_forward.argtypes = [P, P, P, P, P, i32, P]
    lib.ldpc_wbp_forward.restype = ctypes.c_int
    lib.ldpc_wbp_loss.argtypes = [P, P, P, P, P, P]
    lib.ldpc_wbp_loss.restype = ctypes.c_int
    lib.ldpc_wbp_backward.argtypes = [P, P, P, P, P, P, P, P]
    lib.ldpc_wbp_backward.restype = ctypes.c_int
    lib.ldpc_wbp_sgd_step.argtypes = [P, P, P, ctypes.c_double, P]
    lib.ldpc_wbp_sgd_step.restype = ctypes.c_int
    lib.ldpc_wbp_decode.argtypes = [P, i32, P, P, P, i32, ctypes.c_int, P, P, P, ctypes.POINTER(ldpc_decode_opts), P]
    lib.ldpc_wbp_decode.restype = ctypes.c_int
    lib.ldpc_graph_check_guards.argtypes = [P]
    lib.ldpc_graph_check_guards.restype = ctypes.c_int
    lib.ldpc_batch_check_guards.argtypes = [P]
    lib.ldpc_batch_check_guards.restype = ctypes.c_int
    return lib


_lib = _load()


def ldpc_graph_check_guards(handle) -> int:
    return _lib.ldpc_graph_check_guards(handle)


def ldpc_batch_check_guards(handle) -> int:
    return _lib.ldpc_batch_check_guards(handle)


class LdpcError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {ldpc_status_str(status)} (status {status})")
        self.status = status


def _check(status: int, what: str):
    if status != LDPC_OK:
        raise LdpcError(status, what)


def library_path() -> str:
    return _LIB_PATH


# --------------------------------------------------------------------------
# C-named entry points
# --------------------------------------------------------------------------
def ldpc_status_str(status: int) -> str:
    return _lib.ldpc_status_str(int(status)).decode()


def ldpc_decode_opts_init() -> ldpc_decode_opts:
    o = ldpc_decode_opts()
    _lib.ldpc_decode_opts_init(ctypes.byref(o))
    return o


def ldpc_graph_create_csr(m: int, n: int, row_ptr, col_idx) -> int:
    """Returns the opaque graph handle (int).  Raises LdpcError on failure."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(col_idx, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(_lib.ldpc_graph_create_csr(int(m), int(n), rp.ctypes.data, ci.ctypes.data if ci.size else None,
                                      ctypes.byref(h)), "ldpc_graph_create_csr")
    return h.value


def ldpc_graph_create_qc(mb: int, nb: int, Z: int, shifts) -> int:
    sh = np.ascontiguousarray(shifts, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(_lib.ldpc_graph_create_qc(int(mb), int(nb), int(Z), sh.ctypes.data, ctypes.byref(h)),
           "ldpc_graph_create_qc")
    return h.value


def ldpc_graph_destroy(handle: int) -> None:
    _lib.ldpc_graph_destroy(handle)


def ldpc_graph_info(handle: int):
    m, n, e = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64()
    _check(_lib.ldpc_graph_info(handle, ctypes.byref(m), ctypes.byref(n), ctypes.byref(e)), "ldpc_graph_info")
    return m.value, n.value, e.value


def ldpc_decode(handle: int, frames: int, llr_ptr: int, syndrome_ptr: int, max_iter: int, rule: int,
                bits_ptr: int, flags_ptr: int, iters_ptr: int, opts: ldpc_decode_opts | None,
                stream: int) -> int:
    """Raw call with device pointers; returns the status code."""
    return _lib.ldpc_decode(handle, int(frames), llr_ptr, syndrome_ptr, int(max_iter), int(rule), bits_ptr,
                            flags_ptr, iters_ptr, ctypes.byref(opts) if opts is not None else None, stream)


def ldpc_decode_host(handle: int, frames: int, llr_ptr: int, syndrome_ptr: int, max_iter: int, rule: int,
                     bits_ptr: int, flags_ptr: int, iters_ptr: int, opts: ldpc_decode_opts | None,
                     stream: int) -> int:
    """Raw call with host pointers; returns the status code."""
    return _lib.ldpc_decode_host(handle, int(frames), llr_ptr, syndrome_ptr, int(max_iter), int(rule), bits_ptr,
                                 flags_ptr, iters_ptr, ctypes.byref(opts) if opts is not None else None, stream)


def ldpc_decode_qc_noalloc(mb: int, nb: int, Z: int, shifts, frames: int, llr_ptr: int, syndrome_ptr: int,
                           max_iter: int, rule: int, bits_ptr: int, flags_ptr: int, iters_ptr: int,
                           stream: int) -> int:
    """Raw call of the entry point that allocates no device memory (for callers
    that must not allocate: real-time loops, hosts whose memory manager owns the
    GPU).  shifts is a host int32 mb x nb array; the other pointers are device
    buffers as in ldpc_decode.  Returns the status code."""
    sh = np.ascontiguousarray(shifts, dtype=np.int32)
    return _lib.ldpc_decode_qc_noalloc(int(mb), int(nb), int(Z), sh.ctypes.data, int(frames), llr_ptr,
                                       syndrome_ptr, int(max_iter), int(rule), bits_ptr, flags_ptr, iters_ptr,
                                       stream)


# --------------------------------------------------------------------------
# Conveniences (torch tensors as device buffers)
# --------------------------------------------------------------------------
class Graph:
    """Owns an ldpc_graph handle."""

    def __init__(self, handle: int):
        self.handle = handle
        self.m, self.n, self.edges = ldpc_graph_info(handle)

    @classmethod
    def from_csr(cls, m, n, row_ptr, col_idx):
        return cls(ldpc_graph_create_csr(m, n, row_ptr, col_idx))

    @classmethod
    def from_qc(cls, shifts, Z):
        shifts = np.asarray(shifts)
        g = cls(ldpc_graph_create_qc(shifts.shape[0], shifts.shape[1], Z, shifts))
        g.qc_blocks = int((shifts >= 0).sum())
        return g

    qc_blocks = None  # nonzero base blocks of a QC graph (None for CSR graphs)

    @property
    def class_keys(self) -> int:
        """Entries an edge-class map of this graph has (QC: base blocks, CSR: edges)."""
        return self.qc_blocks if self.qc_blocks is not None else self.edges

    @classmethod
    def from_code(cls, code):
        """From a gen.CSRCode / gen.QCCode (anything with those fields)."""
        if hasattr(code, "shifts"):
            return cls.from_qc(code.shifts, code.Z)
        return cls.from_csr(code.m, code.n, code.rowptr, code.colidx)

    def close(self):
        if self.handle:
            ldpc_graph_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def make_opts(vnr_first_iter=2, clamp=25.0, fp64=False, max_active_frames=0, grid_ctas=0,
              trace_iters=0, trace_c2v=None, trace_app=None, trace_q=None, stats=None,
              barrier_timeout_ms=0, test_unreachable_barrier=False, groups=0, schedule="auto", flow_lag=0,
              debug_guards=False):
    o = ldpc_decode_opts_init()
    o.debug_guards = 1 if debug_guards else 0
    o.groups = int(groups)
    o.schedule = SCHEDULES[schedule] if isinstance(schedule, str) else int(schedule)
    o.flow_lag = int(flow_lag)
    o.barrier_timeout_ms = barrier_timeout_ms
    o.test_unreachable_barrier = 1 if test_unreachable_barrier else 0
    o.vnr_first_iter = vnr_first_iter
    o.clamp = clamp
    o.fp64 = 1 if fp64 else 0
    o.max_active_frames = max_active_frames
    o.grid_ctas = grid_ctas
    o.trace_iters = trace_iters
    o.trace_c2v = trace_c2v.data_ptr() if trace_c2v is not None else None
    o.trace_app = trace_app.data_ptr() if trace_app is not None else None
    o.trace_q = trace_q.data_ptr() if trace_q is not None else None
    if stats is not None:
        o.stats = ctypes.pointer(stats)
    return o


def decode(graph: Graph, llr, syndrome, max_iter: int, rule="pce_vnr", out=None, stream=None, **opt):
    """Decode with device tensors (torch, cuda).  llr float32 [F, n], syndrome
    uint8 [F, m].  Returns (bits uint8 [F, n], flags uint8 [F], iters int32 [F]).
    Keyword options are those of make_opts()."""
    import torch
    rule = RULES[rule] if isinstance(rule, str) else int(rule)
    if llr.dtype != torch.float32 or syndrome.dtype != torch.uint8:
        raise TypeError("llr must be float32 and syndrome uint8")
    if not (llr.is_cuda and syndrome.is_cuda and llr.is_contiguous() and syndrome.is_contiguous()):
        raise ValueError("llr and syndrome must be contiguous CUDA tensors")
    F = llr.shape[0]
    if llr.shape != (F, graph.n) or syndrome.shape != (F, graph.m):
        raise ValueError("llr / syndrome shapes do not match the graph")
    if out is None:
        out = (torch.empty((F, graph.n), dtype=torch.uint8, device=llr.device),
               torch.empty(F, dtype=torch.uint8, device=llr.device),
               torch.empty(F, dtype=torch.int32, device=llr.device))
    bits, flags, iters = out
    s = stream if stream is not None else torch.cuda.current_stream(llr.device)
    o = make_opts(**opt)
    st = ldpc_decode(graph.handle, F, llr.data_ptr(), syndrome.data_ptr(), max_iter, rule, bits.data_ptr(),
                     flags.data_ptr(), iters.data_ptr(), o, s.cuda_stream)
    _check(st, "ldpc_decode")
    return bits, flags, iters


def decode_host(graph: Graph, llr: np.ndarray, syndrome: np.ndarray, max_iter: int, rule="pce_vnr",
                out=None, stream: int = 0, **opt):
    """Decode host arrays (numpy, or pinned torch CPU tensors via .numpy()).
    Returns numpy (bits, flags, iters); copies happen inside the call."""
    rule = RULES[rule] if isinstance(rule, str) else int(rule)
    llr = np.ascontiguousarray(llr, dtype=np.float32)
    syndrome = np.ascontiguousarray(syndrome, dtype=np.uint8)
    F = llr.shape[0]
    if out is None:
        out = (np.empty((F, graph.n), np.uint8), np.empty(F, np.uint8), np.empty(F, np.int32))
    bits, flags, iters = out
    o = make_opts(**opt)
    st = ldpc_decode_host(graph.handle, F, llr.ctypes.data, syndrome.ctypes.data, max_iter, rule,
                          bits.ctypes.data, flags.ctypes.data, iters.ctypes.data, o, stream)
    _check(st, "ldpc_decode_host")
    return bits, flags, iters


# --------------------------------------------------------------------------
# Batches of frames of several codes
# --------------------------------------------------------------------------
def ldpc_batch_create(graph_handles, frame_graph) -> int:
    arr = (ctypes.c_void_p * len(graph_handles))(*graph_handles)
    fg = np.ascontiguousarray(frame_graph, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(_lib.ldpc_batch_create(arr, len(graph_handles), fg.size, fg.ctypes.data, ctypes.byref(h)),
           "ldpc_batch_create")
    return h.value


def ldpc_batch_destroy(handle: int) -> None:
    _lib.ldpc_batch_destroy(handle)


def ldpc_batch_info(handle: int):
    f, a, b = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
    _check(_lib.ldpc_batch_info(handle, ctypes.byref(f), ctypes.byref(a), ctypes.byref(b)), "ldpc_batch_info")
    return f.value, a.value, b.value


def ldpc_batch_decode(handle, llr_ptr, syndrome_ptr, max_iter, rule, bits_ptr, flags_ptr, iters_ptr, opts,
                      stream) -> int:
    return _lib.ldpc_batch_decode(handle, llr_ptr, syndrome_ptr, int(max_iter), int(rule), bits_ptr, flags_ptr,
                                  iters_ptr, ctypes.byref(opts) if opts is not None else None, stream)


def ldpc_batch_decode_async(handle, llr_ptr, syndrome_ptr, max_iter, rule, bits_ptr, flags_ptr, iters_ptr,
                            status_ptr, opts, stream) -> int:
    return _lib.ldpc_batch_decode_async(handle, llr_ptr, syndrome_ptr, int(max_iter), int(rule), bits_ptr,
                                        flags_ptr, iters_ptr, status_ptr,
                                        ctypes.byref(opts) if opts is not None else None, stream)


def ldpc_batch_autotune(handle, llr_ptr, syndrome_ptr, max_iter, rule, bits_ptr, flags_ptr, iters_ptr, stream):
    g, s = ctypes.c_int32(), ctypes.c_int32()
    _check(_lib.ldpc_batch_autotune(handle, llr_ptr, syndrome_ptr, int(max_iter), int(rule), bits_ptr, flags_ptr,
                                    iters_ptr, stream, ctypes.byref(g), ctypes.byref(s)), "ldpc_batch_autotune")
    return g.value, s.value


class Batch:
    """Frames of up to four codes decoded together (owns an ldpc_batch plan).
    Buffers hold the frames back to back: llr / bits [llr_len], syndrome
    [syndrome_len], flags / iters [frames]."""

    def __init__(self, graphs, frame_graph):
        self.graphs = list(graphs)  # keep the graphs alive
        self.handle = ldpc_batch_create([g.handle for g in self.graphs], frame_graph)
        self.frames, self.llr_len, self.syndrome_len = ldpc_batch_info(self.handle)

    def outputs(self, device):
        """Fresh (bits, flags, iters) device tensors for this batch."""
        import torch
        return (torch.empty(self.llr_len, dtype=torch.uint8, device=device),
                torch.empty(self.frames, dtype=torch.uint8, device=device),
                torch.empty(self.frames, dtype=torch.int32, device=device))

    def decode(self, llr, syndrome, max_iter, rule="pce_vnr", out=None, stream=None, **opt):
        import torch
        rule = RULES[rule] if isinstance(rule, str) else int(rule)
        out = out or self.outputs(llr.device)
        s = stream if stream is not None else torch.cuda.current_stream(llr.device)
        _check(ldpc_batch_decode(self.handle, llr.data_ptr(), syndrome.data_ptr(), max_iter, rule,
                                 out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), make_opts(**opt),
                                 s.cuda_stream), "ldpc_batch_decode")
        return out

    def decode_async(self, llr, syndrome, max_iter, rule, out, status, stream=None, **opt):
        """Stream-ordered; writes the ldpc_status code to the device int32 tensor `status`."""
        import torch
        rule = RULES[rule] if isinstance(rule, str) else int(rule)
        s = stream if stream is not None else torch.cuda.current_stream(llr.device)
        _check(ldpc_batch_decode_async(self.handle, llr.data_ptr(), syndrome.data_ptr(), max_iter, rule,
                                       out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), status.data_ptr(),
                                       make_opts(**opt), s.cuda_stream), "ldpc_batch_decode_async")

    def autotune(self, llr, syndrome, max_iter, rule="pce_vnr", out=None, stream=None):
        import torch
        rule = RULES[rule] if isinstance(rule, str) else int(rule)
        out = out or self.outputs(llr.device)
        s = stream if stream is not None else torch.cuda.current_stream(llr.device)
        return ldpc_batch_autotune(self.handle, llr.data_ptr(), syndrome.data_ptr(), max_iter, rule,
                                   out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), s.cuda_stream)

    def close(self):
        if self.handle:
            ldpc_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# --------------------------------------------------------------------------
# Weighted belief propagation (trainable decoder)
# --------------------------------------------------------------------------
def ldpc_wbp_create(graph_handle: int, frames: int, iters: int, n_classes: int, edge_class,
                    checkpoint_every: int, fp64: int) -> int:
    cls = np.ascontiguousarray(edge_class, dtype=np.int32)
    h = ctypes.c_void_p()
    _check(_lib.ldpc_wbp_create(graph_handle, int(frames), int(iters), int(n_classes), cls.ctypes.data,
                                int(checkpoint_every), int(fp64), ctypes.byref(h)), "ldpc_wbp_create")
    return h.value


def ldpc_wbp_destroy(handle: int) -> None:
    _lib.ldpc_wbp_destroy(handle)


def ldpc_wbp_forward(handle, llr_ptr, syndrome_ptr, weights_ptr, app_ptr, save_for_backward, stream) -> int:
    return _lib.ldpc_wbp_forward(handle, llr_ptr, syndrome_ptr, weights_ptr, app_ptr, int(save_for_backward),
                                 stream)


def ldpc_wbp_loss(handle, app_ptr, x_ptr, loss_ptr, grad_app_ptr, stream) -> int:
    return _lib.ldpc_wbp_loss(handle, app_ptr, x_ptr, loss_ptr, grad_app_ptr, stream)


def ldpc_wbp_backward(handle, llr_ptr, syndrome_ptr, weights_ptr, grad_app_ptr, grad_w_ptr, grad_llr_ptr,
                      stream) -> int:
    return _lib.ldpc_wbp_backward(handle, llr_ptr, syndrome_ptr, weights_ptr, grad_app_ptr, grad_w_ptr,
                                  grad_llr_ptr, stream)


def ldpc_wbp_decode(handle, frames, llr_ptr, syndrome_ptr, weights_ptr, max_iter, rule, bits_ptr, flags_ptr,
                    iters_ptr, opts, stream) -> int:
    return _lib.ldpc_wbp_decode(handle, int(frames), llr_ptr, syndrome_ptr, weights_ptr, int(max_iter), int(rule),
                                bits_ptr, flags_ptr, iters_ptr, ctypes.byref(opts) if opts is not None else None,
                                stream)


def ldpc_wbp_sgd_step(handle, weights_ptr, grad_ptr, lr, stream) -> int:
    return _lib.ldpc_wbp_sgd_step(handle, weights_ptr, grad_ptr, float(lr), stream)


class WeightedBP:
    """A weighted-BP plan (ldpc_wbp): `frames` frames of `graph`, `iters`
    unrolled iterations, weights [iters, n_classes] of the plan's dtype
    (float32, or float64 with fp64=True).  edge_class: QC graphs one class per
    nonzero base block (row-major), CSR graphs one per edge (CSR order)."""

    def __init__(self, graph: Graph, frames: int, iters: int, edge_class, n_classes: int,
                 checkpoint_every: int = 5, fp64: bool = False):
        self.graph = graph
        self.frames, self.iters, self.n_classes = int(frames), int(iters), int(n_classes)
        self.fp64 = bool(fp64)
        edge_class = np.ascontiguousarray(edge_class, dtype=np.int32)
        if edge_class.shape != (graph.class_keys,):
            raise ValueError(f"edge_class needs {graph.class_keys} entries, got {edge_class.shape}")
        self.handle = None
        self.handle = ldpc_wbp_create(graph.handle, frames, iters, n_classes, edge_class, checkpoint_every,
                                      int(self.fp64))
        self.generation = 0  # forward passes with save_for_backward so far

    @property
    def dtype(self):
        import torch
        return torch.float64 if self.fp64 else torch.float32

    def _stream(self, t, stream):
        import torch
        return (stream if stream is not None else torch.cuda.current_stream(t.device)).cuda_stream

    def forward(self, llr, syndrome, weights, app=None, save=True, stream=None):
        import torch
        app = app if app is not None else torch.empty((self.frames, self.graph.n), dtype=self.dtype,
                                                      device=llr.device)
        _check(ldpc_wbp_forward(self.handle, llr.data_ptr(), syndrome.data_ptr(), weights.data_ptr(),
                                app.data_ptr(), save, self._stream(llr, stream)), "ldpc_wbp_forward")
        if save:
            self.generation += 1
        return app

    def loss(self, app, x, want_grad=True, stream=None):
        """Mean binary cross-entropy of the soft output against x; returns
        (loss [1] tensor, dloss/dAPP or None)."""
        import torch
        loss = torch.empty(1, dtype=self.dtype, device=app.device)
        g = torch.empty_like(app) if want_grad else None
        _check(ldpc_wbp_loss(self.handle, app.data_ptr(), x.data_ptr(), loss.data_ptr(),
                             g.data_ptr() if g is not None else None, self._stream(app, stream)), "ldpc_wbp_loss")
        return loss, g

    def backward(self, llr, syndrome, weights, grad_app, want_llr=False, grad_w=None, stream=None):
        import torch
        gw = grad_w if grad_w is not None else torch.empty_like(weights)
        gl = torch.empty((self.frames, self.graph.n), dtype=self.dtype, device=llr.device) if want_llr else None
        _check(ldpc_wbp_backward(self.handle, llr.data_ptr(), syndrome.data_ptr(), weights.data_ptr(),
                                 grad_app.data_ptr(), gw.data_ptr(), gl.data_ptr() if gl is not None else None,
                                 self._stream(llr, stream)), "ldpc_wbp_backward")
        return gw, gl

    def decode(self, llr, syndrome, weights, max_iter, rule="pce_vnr", out=None, stream=None, **opt):
        """Early-terminating decode with these learned weights (float32
        [iters, n_classes]); llr [F, n] float32, syndrome [F, m] uint8 on the
        device; returns (bits, flags, iters) as ldpc.decode does."""
        import torch
        rule = RULES[rule] if isinstance(rule, str) else int(rule)
        F = llr.shape[0]
        if out is None:
            out = (torch.empty((F, self.graph.n), dtype=torch.uint8, device=llr.device),
                   torch.empty(F, dtype=torch.uint8, device=llr.device),
                   torch.empty(F, dtype=torch.int32, device=llr.device))
        w = weights.to(torch.float32).contiguous()
        _check(ldpc_wbp_decode(self.handle, F, llr.data_ptr(), syndrome.data_ptr(), w.data_ptr(), max_iter, rule,
                               out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr(), make_opts(**opt),
                               self._stream(llr, stream)), "ldpc_wbp_decode")
        return out

    def sgd_step(self, weights, grad, lr, stream=None):
        _check(ldpc_wbp_sgd_step(self.handle, weights.data_ptr(), grad.data_ptr(), lr,
                                 self._stream(weights, stream)), "ldpc_wbp_sgd_step")

    def close(self):
        if self.handle:
            ldpc_wbp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def weighted_bp(plan: WeightedBP, weights, llr, syndrome):
    """APP after the plan's iterations as a differentiable function of the
    weights (and of the channel LLRs), for torch.autograd."""
    import torch

    class _WBP(torch.autograd.Function):
        @staticmethod
        def forward(ctx, w, l):
            app = plan.forward(l, syndrome, w.contiguous(), save=True)
            ctx.save_for_backward(w, l)
            ctx.generation = plan.generation
            return app

        @staticmethod
        def backward(ctx, grad_app):
            w, l = ctx.saved_tensors
            if plan.generation != ctx.generation:  # another forward replaced the checkpoints
                plan.forward(l, syndrome, w.contiguous(), save=True)
            gw, gl = plan.backward(l, syndrome, w.contiguous(), grad_app.contiguous().to(plan.dtype),
                                   want_llr=ctx.needs_input_grad[1])
            return gw, (gl.to(l.dtype) if gl is not None else None)

    return _WBP.apply(weights, llr)
