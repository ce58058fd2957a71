"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports
every function that include/ldpc.h declares, and rejects malformed graphs and
arguments on the host before any GPU work is queued."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "ldpc.h")


@pytest.fixture(scope="module")
def ldpc():
    from paper_2507_03509_gb300 import build
    build.build()
    from paper_2507_03509_gb300 import ldpc as mod
    return mod


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(?:LDPC_API\s+)?(?:ldpc_status|void|const char\s*\*)\s+(ldpc_\w+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("ldpc_graph_create_csr", "ldpc_graph_create_qc", "ldpc_graph_destroy", "ldpc_graph_info",
              "ldpc_decode", "ldpc_decode_host", "ldpc_status_str", "ldpc_decode_opts_init"):
        assert n in names


def test_library_exports_every_declared_symbol(ldpc):
    lib = ctypes.CDLL(ldpc.library_path())
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(ldpc.EXPORTED)


def test_struct_layout_matches_header(ldpc):
    # opts: 6 x 4-byte fields, 4 pointers, 6 x 4-byte fields; stats: 2 floats, 4 ints, 1 int64
    assert ctypes.sizeof(ldpc.ldpc_decode_opts) == 24 + 4 * 8 + 24
    assert ctypes.sizeof(ldpc.ldpc_decode_stats) == 32
    o = ldpc.ldpc_decode_opts_init()
    assert o.vnr_first_iter == 2 and o.clamp == 25.0 and o.fp64 == 0 and o.trace_iters == 0
    assert o.barrier_timeout_ms == 0 and o.test_unreachable_barrier == 0 and o.groups == 0
    assert o.schedule == 0 and o.flow_lag == 0 and o.debug_guards == 0


def test_status_strings(ldpc):
    assert ldpc.ldpc_status_str(0) == "ok"
    assert "graph" in ldpc.ldpc_status_str(2)
    assert ldpc.ldpc_status_str(99) == "unknown status"


@pytest.mark.parametrize("rows,cols,n,why", [
    ([1, 1], [0], 4, "row_ptr[0] != 0"),
    ([0, 2, 1], [0, 1], 4, "decreasing row_ptr"),
    ([0, 2], [1, 1], 4, "repeated column"),
    ([0, 2], [2, 1], 4, "unsorted row"),
    ([0, 1], [4], 4, "column out of range"),
    ([0, 1], [-1], 4, "negative column"),
    ([0, 65], list(range(65)), 70, "check degree above 64"),
])
def test_malformed_csr_is_rejected_on_host(ldpc, rows, cols, n, why):
    with pytest.raises(ldpc.LdpcError) as ei:
        ldpc.ldpc_graph_create_csr(len(rows) - 1, n, rows, cols)
    assert ei.value.status == ldpc.LDPC_ERR_INVALID_GRAPH, why


@pytest.mark.parametrize("shifts,Z,status", [
    ([[0, 5]], 5, 2),          # shift == Z
    ([[0, -2]], 5, 2),         # below -1
    ([[0]], 0, 1),             # Z = 0
    ([[0] * 65], 4, 2),        # row weight 65
])
def test_malformed_qc_is_rejected_on_host(ldpc, shifts, Z, status):
    with pytest.raises(ldpc.LdpcError) as ei:
        ldpc.ldpc_graph_create_qc(len(shifts), len(shifts[0]), Z, np.asarray(shifts))
    assert ei.value.status == status


def test_noalloc_rejects_oversize_before_any_gpu_work(ldpc):
    # one Z = 2^30 circulant: its packed syndrome alone exceeds the fixed scratch
    st = ldpc.ldpc_decode_qc_noalloc(1, 1, 1 << 30, np.zeros((1, 1), np.int32), 1, 16, 16, 10, 2, 16, 16, 16, None)
    assert st == ldpc.LDPC_ERR_TOO_LARGE
    assert "too large" in ldpc.ldpc_status_str(st)
    assert ldpc.ldpc_decode_qc_noalloc(1, 1, 4, np.full((1, 1), 4, np.int32), 1, 16, 16, 10, 2, 16, 16, 16,
                                       None) == ldpc.LDPC_ERR_INVALID_GRAPH


def test_decode_argument_errors_need_no_gpu(ldpc):
    # a null graph and bad sizes are refused before any CUDA call
    assert ldpc.ldpc_decode(None, 1, 1, 1, 10, 2, 1, 1, 1, None, None) == ldpc.LDPC_ERR_INVALID_ARG
    assert ldpc.ldpc_decode_host(None, 1, 1, 1, 10, 2, 1, 1, 1, None, None) == ldpc.LDPC_ERR_INVALID_ARG


def test_guard_check_needs_a_guarded_decode(ldpc):
    # no graph, and a graph whose workspace holds no guards yet: refused on the host
    assert ldpc.ldpc_graph_check_guards(None) == ldpc.LDPC_ERR_INVALID_ARG
    assert ldpc.ldpc_batch_check_guards(None) == ldpc.LDPC_ERR_INVALID_ARG
    assert "guard" in ldpc.ldpc_status_str(ldpc.LDPC_ERR_BOUNDS)


def test_index_checking_build_compiles_and_exports(ldpc):
    """The debug build (-DLDPC_BOUNDS_CHECK) builds for sm_103a and exports the
    same boundary."""
    from paper_2507_03509_gb300 import build
    path = build.build(checked=True)
    assert path.endswith("libldpc_gb300_checked.so")
    lib = ctypes.CDLL(path)
    for name in declared_functions():
        assert hasattr(lib, name), name


def header_constants():
    """Integer constants of include/ldpc.h: enum members (NAME = value) and
    #define NAME value lines (a value of the form (a * b * c) is multiplied out)."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    consts = {k: int(v) for k, v in re.findall(r"\b(LDPC_[A-Z0-9_]+)\s*=\s*(\d+)", text)}
    for name, expr in re.findall(r"#define\s+(LDPC_[A-Z0-9_]+)\s+(.+)", text):
        factors = re.findall(r"(\d+)u?", expr)
        if factors and re.fullmatch(r"[\s()*\du]+", expr.strip()):
            val = 1
            for f in factors:
                val *= int(f)
            consts[name] = val
    return consts


def test_binding_constants_match_the_header(ldpc):
    """The Python binding's status codes, rules, flags, schedule values and
    no-alloc scratch size are the header's (the binding restates them)."""
    h = header_constants()
    for name in ("LDPC_OK", "LDPC_ERR_INVALID_ARG", "LDPC_ERR_INVALID_GRAPH", "LDPC_ERR_OOM", "LDPC_ERR_CUDA",
                 "LDPC_ERR_TIMEOUT", "LDPC_ERR_TOO_LARGE", "LDPC_ERR_BOUNDS", "LDPC_TERM_NONE", "LDPC_TERM_PCE",
                 "LDPC_TERM_PCE_VNR", "LDPC_FLAG_SUCCESS", "LDPC_FLAG_ABORTED"):
        assert getattr(ldpc, name) == h[name], name
    assert ldpc.NOALLOC_SCRATCH_BYTES == h["LDPC_NOALLOC_SCRATCH_BYTES"]
    schedules = {"auto": "LDPC_SCHEDULE_AUTO", "lockstep": "LDPC_SCHEDULE_LOCKSTEP",
                 "dataflow": "LDPC_SCHEDULE_DATAFLOW", "frame": "LDPC_SCHEDULE_FRAME",
                 "frame_pair": "LDPC_SCHEDULE_FRAME_PAIR"}
    assert set(ldpc.SCHEDULES) == set(schedules)
    for key, name in schedules.items():
        assert ldpc.SCHEDULES[key] == h[name], key
    assert ldpc.RULES == {"none": h["LDPC_TERM_NONE"], "pce": h["LDPC_TERM_PCE"], "pce_vnr": h["LDPC_TERM_PCE_VNR"]}
