"""Seeded synthetic inputs for syndrome-based LDPC reconciliation.

This module builds parity-check matrices and channel frames.  It holds none of
the decoder's arithmetic: it draws codes, bits, Gaussian noise and channel
LLRs, and forms the syndrome s = H x (mod 2) that Alice would send (the
decoder's input in syndrome-based reconciliation, paper section "Early
Termination").  Both the CUDA decoder's tests/benchmark and the FP64 oracle
consume what it returns; neither side imports the other.

Conventions
-----------
* H is m x n (rows = check nodes, columns = variable nodes).
* LLR L = ln P(x=0)/P(x=1); BPSK maps bit 0 -> +1, bit 1 -> -1, so with
  y = (1 - 2x) + sigma * z the channel LLR is Lch = 2 y / sigma^2.
* The noise level is set through the reconciliation efficiency
  beta = R / C (section "Secret Key Rate"), with C the binary-input AWGN
  capacity, solved for sigma by bisection.

Seeds: a code of workload number c uses seed 1000 + c; frame f of workload c
uses seed 2000 * c + f, each an independent numpy PCG64 stream.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "CSRCode", "QCCode", "Frames", "random_csr_code", "qc_base_matrix",
    "random_qc_code", "biawgn_capacity", "sigma_for_capacity", "make_frames",
    "syndrome", "WORKLOADS", "workload_code", "workload_frames",
]


# --------------------------------------------------------------------------
# Parity-check matrices
# --------------------------------------------------------------------------
@dataclass
class CSRCode:
    """Binary H in compressed-sparse-row form; columns sorted in each row."""
    m: int
    n: int
    rowptr: np.ndarray  # int32 [m+1]
    colidx: np.ndarray  # int32 [E]

    @property
    def edges(self) -> int:
        return int(self.rowptr[-1])

    @property
    def rate(self) -> float:
        """Design rate 1 - m/n (assumes full-rank H)."""
        return 1.0 - self.m / self.n

    def check_degrees(self) -> np.ndarray:
        return np.diff(self.rowptr).astype(np.int64)

    def var_degrees(self) -> np.ndarray:
        return np.bincount(self.colidx, minlength=self.n).astype(np.int64)

    def row_of_edge(self) -> np.ndarray:
        return np.repeat(np.arange(self.m, dtype=np.int64), self.check_degrees())


@dataclass
class QCCode:
    """Quasi-cyclic H: an mb x nb base matrix of circulant shifts.

    shifts[i, j] = -1 is an all-zero Z x Z block; shifts[i, j] = s >= 0 is the
    identity cyclically shifted so that check i*Z + t meets variable
    j*Z + (t + s) mod Z.
    """
    mb: int
    nb: int
    Z: int
    shifts: np.ndarray  # int32 [mb, nb]

    @property
    def m(self) -> int:
        return self.mb * self.Z

    @property
    def n(self) -> int:
        return self.nb * self.Z

    @property
    def edges(self) -> int:
        return int((self.shifts >= 0).sum()) * self.Z

    @property
    def rate(self) -> float:
        return 1.0 - self.mb / self.nb

    def to_csr(self) -> CSRCode:
        """Lift to the binary m x n matrix, rows in order, columns ascending."""
        Z = self.Z
        t = np.arange(Z, dtype=np.int64)
        degs = []
        cols_per_row = []
        for i in range(self.mb):
            js = [j for j in range(self.nb) if self.shifts[i, j] >= 0]
            blk = np.empty((Z, len(js)), dtype=np.int64)
            for k, j in enumerate(js):  # ascending j => ascending column index
                blk[:, k] = j * Z + (t + int(self.shifts[i, j])) % Z
            cols_per_row.append(blk.reshape(-1))
            degs.append(np.full(Z, len(js), dtype=np.int64))
        colidx = np.concatenate(cols_per_row) if cols_per_row else np.zeros(0, np.int64)
        rowptr = np.concatenate([[0], np.cumsum(np.concatenate(degs))]) if degs else np.zeros(1)
        return CSRCode(self.m, self.n, rowptr.astype(np.int32), colidx.astype(np.int32))


def _collapse_rows(m: int, n: int, rows: np.ndarray, cols: np.ndarray) -> CSRCode:
    """Sort (row, col) pairs, drop repeated pairs (H is a 0/1 adjacency)."""
    key = np.unique(rows.astype(np.int64) * n + cols.astype(np.int64))
    r = key // n
    c = key % n
    rowptr = np.zeros(m + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return CSRCode(m, n, rowptr.astype(np.int32), c.astype(np.int32))


def random_csr_code(n: int, m: int, var_degree: int, check_degrees: dict[int, int],
                    seed: int) -> CSRCode:
    """Random code by seeded socket matching.

    Every variable node gets `var_degree` sockets; `check_degrees` maps a check
    degree to how many checks carry it (assigned to checks by a seeded
    permutation).  A seeded permutation matches the two socket lists; repeated
    (check, variable) pairs collapse to one edge, so a few degrees may drop.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    degs = np.concatenate([np.full(cnt, d, dtype=np.int64)
                           for d, cnt in sorted(check_degrees.items())])
    if degs.size != m:
        raise ValueError("check degree counts must add up to m")
    if int(degs.sum()) != n * var_degree:
        raise ValueError("socket counts of the two sides differ")
    degs = rng.permutation(degs)
    check_sockets = np.repeat(np.arange(m, dtype=np.int64), degs)
    var_sockets = np.repeat(np.arange(n, dtype=np.int64), var_degree)
    var_sockets = var_sockets[rng.permutation(var_sockets.size)]
    return _collapse_rows(m, n, check_sockets, var_sockets)


def qc_base_matrix(mb: int, nb: int, col_weights: np.ndarray, seed: int) -> np.ndarray:
    """Seeded 0/1 base matrix with the given column weights and row weights
    as equal as the total allows (balanced assignment).

    Columns are placed in a seeded order, heaviest first; each takes the rows
    with the most remaining capacity, ties broken by a seeded random key.
    Row capacities are floor/ceil of (total weight / mb), the larger ones on
    seeded rows.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    col_weights = np.asarray(col_weights, dtype=np.int64)
    if col_weights.size != nb or col_weights.max(initial=0) > mb:
        raise ValueError("bad column weights")
    total = int(col_weights.sum())
    lo, extra = divmod(total, mb)
    cap = np.full(mb, lo, dtype=np.int64)
    cap[rng.permutation(mb)[:extra]] += 1
    B = np.zeros((mb, nb), dtype=np.int8)
    order = rng.permutation(nb)
    order = order[np.argsort(-col_weights[order], kind="stable")]
    for j in order:
        w = int(col_weights[j])
        tie = rng.random(mb)
        rows = np.lexsort((tie, -cap))[:w]
        if np.any(cap[rows] <= 0):
            raise RuntimeError("row capacities exhausted")
        B[rows, j] = 1
        cap[rows] -= 1
    return B


def random_qc_code(mb: int, nb: int, Z: int, col_weights, seed: int) -> QCCode:
    """QC code: seeded balanced base matrix, circulant shifts uniform in [0, Z)."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    B = qc_base_matrix(mb, nb, np.asarray(col_weights), seed)
    shifts = np.where(B > 0, rng.integers(0, Z, size=B.shape), -1).astype(np.int32)
    return QCCode(mb, nb, Z, shifts)


# --------------------------------------------------------------------------
# Channel: BIAWGN capacity and sigma for a target efficiency
# --------------------------------------------------------------------------
_GH_X, _GH_W = np.polynomial.hermite.hermgauss(160)


def biawgn_capacity(sigma: float) -> float:
    """Capacity (bits/use) of BPSK over AWGN with noise std sigma.

    C = 1 - E[log2(1 + exp(-2Y/sigma^2))], Y ~ N(1, sigma^2), by
    Gauss-Hermite quadrature (160 nodes).
    """
    y = 1.0 + math.sqrt(2.0) * sigma * _GH_X
    f = np.logaddexp(0.0, -2.0 * y / (sigma * sigma)) / math.log(2.0)
    return float(1.0 - (_GH_W * f).sum() / math.sqrt(math.pi))


def sigma_for_capacity(target: float, lo: float = 0.05, hi: float = 80.0) -> float:
    """Noise std at which biawgn_capacity(sigma) = target (bisection; C falls with sigma)."""
    if not (0.0 < target < 1.0):
        raise ValueError("capacity target must lie in (0, 1)")
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if biawgn_capacity(mid) > target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


# --------------------------------------------------------------------------
# Frames
# --------------------------------------------------------------------------
@dataclass
class Frames:
    x: np.ndarray         # uint8 [F, n]  Alice's bits
    llr: np.ndarray       # float32 [F, n] channel LLRs at Bob
    syndrome: np.ndarray  # uint8 [F, m]  s = H x mod 2
    sigma: np.ndarray     # float64 [F]


def syndrome(code, x: np.ndarray) -> np.ndarray:
    """s = H x (mod 2) for x of shape [F, n] (or [n]); uint8 result."""
    x = np.asarray(x, dtype=np.uint8)
    squeeze = x.ndim == 1
    x2 = x[None, :] if squeeze else x
    if isinstance(code, QCCode):
        Z = code.Z
        out = np.zeros((x2.shape[0], code.mb, Z), dtype=np.uint8)
        xb = x2.reshape(x2.shape[0], code.nb, Z)
        for i in range(code.mb):
            for j in range(code.nb):
                s = int(code.shifts[i, j])
                if s >= 0:
                    out[:, i, :] ^= np.roll(xb[:, j, :], -s, axis=1)
        out = out.reshape(x2.shape[0], code.m)
    else:
        vals = x2[:, code.colidx].astype(np.uint8)
        deg = code.check_degrees()
        out = np.zeros((x2.shape[0], code.m), dtype=np.uint8)
        nz = deg > 0
        starts = code.rowptr[:-1][nz]
        if vals.shape[1] > 0:
            red = np.bitwise_xor.reduceat(vals, starts, axis=1)
            out[:, nz] = red
    return out[0] if squeeze else out


def _draw_frame(n: int, seed: int, sigmas, x_out, llr_outs, f: int) -> None:
    """Frame f from its own generator: x ~ U{0,1}^n, z ~ N(0,1)^n, and for
    each sigma Lch = 2y/sigma^2 with y = (1-2x) + sigma z, rounded once to
    float32."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    xf = rng.integers(0, 2, size=n, dtype=np.uint8)
    z = rng.standard_normal(n)
    x_out[f] = xf
    bpsk = 1.0 - 2.0 * xf.astype(np.float64)
    for sigma, llr in zip(sigmas, llr_outs):
        y = bpsk + sigma * z
        llr[f] = (2.0 * y / (sigma ** 2)).astype(np.float32)


def _frame_threads(frames: int, n: int) -> int:
    """Host threads for drawing frames (numpy's generators release the GIL);
    one thread for small jobs."""
    import os
    if frames * n < 4_000_000:
        return 1
    return max(1, min(16, os.cpu_count() or 1, frames))


def make_frames_sigmas(code, sigma_sets, seeds) -> list[Frames]:
    """make_frames for several noise levels at once: frame f uses the same
    generator (seed) and hence the same x and z at every level, so the frames
    of level i equal make_frames(code, sigma_sets[i], seeds).  Frames are
    drawn by a thread pool; each has its own generator, so the result does not
    depend on the threads."""
    sets = [np.asarray(sg, dtype=np.float64) for sg in sigma_sets]
    F = len(seeds)
    n = code.n
    x = np.empty((F, n), dtype=np.uint8)
    llrs = [np.empty((F, n), dtype=np.float32) for _ in sets]
    work = lambda f: _draw_frame(n, seeds[f], [sg[f] for sg in sets], x, llrs, f)
    threads = _frame_threads(F, n)
    if threads == 1:
        for f in range(F):
            work(f)
    else:
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(work, range(F)))
    s = syndrome(code, x)
    return [Frames(x, llr, s, sg) for llr, sg in zip(llrs, sets)]


def make_frames(code, sigmas, seeds) -> Frames:
    """One frame per (sigma, seed): x ~ U{0,1}^n, y = (1-2x) + sigma z,
    Lch = 2y/sigma^2 rounded once to float32, s = H x."""
    sigmas = np.asarray(sigmas, dtype=np.float64)
    return make_frames_sigmas(code, [sigmas], [int(sd) for sd in seeds][:sigmas.size])[0]


# --------------------------------------------------------------------------
# The named workloads
# --------------------------------------------------------------------------
def _qc_weights_2_3(nb: int, n_w2: int, seed: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(seed + 104729))
    w = np.full(nb, 3, dtype=np.int64)
    w[rng.permutation(nb)[:n_w2]] = 2
    return w


# number -> description; sizes follow the workloads the paper simulates
# (N = 1e6, R = 1/50, section "Simulations") and a small oracle-sized code.
WORKLOADS = {
    1: dict(name="csr_n4096_r0.1", kind="csr", n=4096, m=3686, var_degree=3,
            check_degrees={3: 2456, 4: 1230}, frames=64, beta=0.9, rate=0.1,
            max_iter=200),
    2: dict(name="qc_n1e6_r0.02", kind="qc", mb=49, nb=50, Z=20000, n_w2=25,
            frames=32, beta=0.93, rate=0.02, max_iter=500),
    5: dict(name="qc_n1e6_r0.02_stream", kind="qc", mb=49, nb=50, Z=20000, n_w2=25,
            frames=512, beta=0.95, rate=0.02, max_iter=1000, code_from=2),
    # frames of three codes of different length and rate, decoded together; each
    # frame draws its code and its efficiency beta ~ U[beta_lo, beta_hi]
    3: dict(name="qc_mix3_n64k-1e6_256f", kind="batch", frames=256, beta_lo=0.85, beta_hi=0.97, max_iter=500,
            codes=[dict(name="qc_n65536_r0.1", mb=115, nb=128, Z=512, n_w2=64, seed=1031),
                   dict(name="qc_n262144_r0.05", mb=243, nb=256, Z=1024, n_w2=128, seed=1032),
                   dict(name="qc_n1e6_r0.02", code_from=2)]),
    # weighted BP trained by gradient descent: T unrolled iterations, one weight
    # per (iteration, base block); gradients checked against finite differences
    # on the small random code `fd` (one weight per (iteration, check degree))
    4: dict(name="wbp_qc_n65536_r0.1_T20", kind="wbp", mb=115, nb=128, Z=512, n_w2=64, frames=128, beta=0.9,
            rate=0.1, iters=20, checkpoint=5,
            fd=dict(n=256, m=230, var_degree=3, check_degrees={3: 152, 4: 78}, seed=1404)),
    # a type-based-protograph-like multi-edge-type code at the paper's rate and
    # length (R = 1/50, n = 10^6): 8 core columns (core column 0 punctured),
    # 192 degree-1 columns; used for the VNR-ET beta sweep on degree-1 variables
    7: dict(name="qc_tbp_like_n1e6_r0.02", kind="tbp", Z=5000, frames=32, beta=0.9, rate=0.02, max_iter=500,
            punctured_cols=(0,)),
    # a (3,6)-regular QC code of the same length class whose BP waterfall lies at
    # beta ~ 0.86-0.89, where early termination changes FER and mean iterations
    # (the regime of the paper's Figs. 1-2); used for the beta sweep
    6: dict(name="qc_n960k_r0.5_reg36", kind="qc", mb=24, nb=48, Z=20000, col_weight=3,
            frames=32, beta=0.87, rate=0.5, max_iter=500),
}


def workload_code(number: int, Z: int | None = None):
    """Code of a named workload; Z overrides the lifting size (same base matrix)."""
    w = WORKLOADS[number]
    code_no = w.get("code_from", number)
    seed = 1000 + code_no
    if w["kind"] == "csr":
        return random_csr_code(w["n"], w["m"], w["var_degree"], w["check_degrees"], seed)
    if w["kind"] == "batch":
        raise ValueError("a batch workload has several codes: use batch_codes()")
    if w["kind"] == "tbp":
        return tbp_like_qc_code(Z or w["Z"], seed=seed)
    if "col_weight" in w:
        weights = np.full(w["nb"], w["col_weight"], dtype=np.int64)
    else:
        weights = _qc_weights_2_3(w["nb"], w["n_w2"], seed)
    return random_qc_code(w["mb"], w["nb"], Z or w["Z"], weights, seed)


def edge_classes_by_check_degree(code: CSRCode):
    """Edge classes of a CSR code: the class of edge (c, v) is the rank of
    deg(c) among the code's distinct check degrees.  Returns (class per edge
    in CSR order, number of classes, the degrees in class order)."""
    deg = code.check_degrees()
    degrees = np.unique(deg[deg > 0])
    rank = np.searchsorted(degrees, deg)
    return rank[code.row_of_edge()].astype(np.int32), int(degrees.size), degrees


def qc_block_index(code: QCCode) -> np.ndarray:
    """[mb, nb] -> index of each nonzero base block in row-major order (-1 elsewhere)."""
    nz = code.shifts >= 0
    idx = np.full(code.shifts.shape, -1, dtype=np.int64)
    idx[nz] = np.arange(int(nz.sum()))
    return idx


def qc_csr_edge_blocks(code: QCCode) -> np.ndarray:
    """Base block of every edge of code.to_csr(), in CSR edge order."""
    csr = code.to_csr()
    rows = csr.row_of_edge() // code.Z
    cols = csr.colidx.astype(np.int64) // code.Z
    return qc_block_index(code)[rows, cols]


def wbp_fd_code(number: int = 4) -> CSRCode:
    """The small random code of a weighted-BP workload's finite-difference check."""
    d = WORKLOADS[number]["fd"]
    return random_csr_code(d["n"], d["m"], d["var_degree"], d["check_degrees"], d["seed"])


def tbp_like_base(k_core: int, core_rows: int, lower_rows: int, core_deg: int, lower_core_deg: int,
                  seed: int) -> np.ndarray:
    """Base matrix of a multi-edge-type protograph in the style of the paper's
    type-based protograph (TBP) codes for low rates (section "Simulations",
    R = 1/50): k_core core columns and lower_rows degree-1 columns.

    Rows 0 .. core_rows-1 tie the core columns together (each core column
    meets core_deg of them).  Row core_rows + r holds degree-1 column
    k_core + r and lower_core_deg core columns.  Core columns are spread over
    the lower rows as evenly as the totals allow (seeded).  Rate
    1 - (core_rows + lower_rows) / (k_core + lower_rows)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mb, nb = core_rows + lower_rows, k_core + lower_rows
    B = np.zeros((mb, nb), dtype=np.int8)
    core = qc_base_matrix(core_rows, k_core, np.full(k_core, core_deg), seed + 1)
    B[:core_rows, :k_core] = core
    use = np.zeros(k_core, dtype=np.int64)  # lower-row connections per core column so far
    for r in range(lower_rows):
        tie = rng.random(k_core)
        cols = np.lexsort((tie, use))[:lower_core_deg]  # least used first, ties at random
        B[core_rows + r, cols] = 1
        use[cols] += 1
        B[core_rows + r, k_core + r] = 1
    return B


def tbp_like_qc_code(Z: int, k_core: int = 8, core_rows: int = 4, lower_rows: int = 192, core_deg: int = 3,
                     lower_core_deg: int = 2, seed: int = 1007) -> QCCode:
    """QC lift of tbp_like_base with circulant shifts uniform in [0, Z).  The
    defaults give R = 4/200 = 1/50 (n = 200 Z): core columns of degree 3 + 48,
    core rows of degree 6, lower rows of degree 3 (two core bits and one
    degree-1 bit), the shape of published low-rate multi-edge-type codes."""
    B = tbp_like_base(k_core, core_rows, lower_rows, core_deg, lower_core_deg, seed)
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    shifts = np.where(B > 0, rng.integers(0, Z, size=B.shape), -1).astype(np.int32)
    return QCCode(B.shape[0], B.shape[1], Z, shifts)


SHORTENED_LLR = 100.0  # channel value of a shortened (known) bit: strong, finite


def rate_adapt(frames: Frames, punctured, shortened) -> Frames:
    """Rate adaptation of received frames.  Punctured bits were never sent:
    Lch = 0.  Shortened bits are known to both sides: Lch = +-SHORTENED_LLR
    with the sign of the known bit.  x and the syndrome are unchanged."""
    llr = frames.llr.copy()
    p = np.asarray(punctured, dtype=np.int64)
    sh = np.asarray(shortened, dtype=np.int64)
    llr[:, p] = 0.0
    llr[:, sh] = (SHORTENED_LLR * (1.0 - 2.0 * frames.x[:, sh].astype(np.float64))).astype(np.float32)
    return Frames(frames.x, llr, frames.syndrome, frames.sigma)


def batch_codes(number: int):
    """The codes of a batch workload, in the order frames index them."""
    codes = []
    for c in WORKLOADS[number]["codes"]:
        if "code_from" in c:
            codes.append(workload_code(c["code_from"]))
        else:
            codes.append(random_qc_code(c["mb"], c["nb"], c["Z"], _qc_weights_2_3(c["nb"], c["n_w2"], c["seed"]),
                                        c["seed"]))
    return codes


@dataclass
class BatchFrames:
    frame_code: np.ndarray  # int32 [F]  code of each frame
    beta: np.ndarray        # float64 [F]
    sigma: np.ndarray       # float64 [F]
    var_off: np.ndarray     # int64 [F + 1]  frame f's bits / LLRs at var_off[f] .. var_off[f + 1]
    syn_off: np.ndarray     # int64 [F + 1]
    x: np.ndarray           # uint8 [sum n]  all frames' bits, back to back
    llr: np.ndarray         # float32 [sum n]
    syndrome: np.ndarray    # uint8 [sum m]


def workload_batch(number: int, codes, frames: int | None = None, first: int = 0) -> BatchFrames:
    """Frames first..first+frames-1 of a batch workload.  Frame f draws its code
    and beta from its own seeded generator, so a frame does not depend on how
    many frames are drawn; then x, Lch and s as make_frames makes them, with
    sigma such that capacity = R_code / beta."""
    w = WORKLOADS[number]
    F = w["frames"] if frames is None else frames
    fc = np.empty(F, dtype=np.int32)
    beta = np.empty(F)
    for i in range(F):
        rng = np.random.Generator(np.random.PCG64([number, first + i]))
        fc[i] = rng.integers(0, len(codes))
        beta[i] = rng.uniform(w["beta_lo"], w["beta_hi"])
    sigma = np.array([sigma_for_capacity(codes[c].rate / b) for c, b in zip(fc, beta)])
    var_off = np.concatenate([[0], np.cumsum([codes[c].n for c in fc])]).astype(np.int64)
    syn_off = np.concatenate([[0], np.cumsum([codes[c].m for c in fc])]).astype(np.int64)
    x = np.empty(var_off[-1], dtype=np.uint8)
    llr = np.empty(var_off[-1], dtype=np.float32)
    syn = np.empty(syn_off[-1], dtype=np.uint8)
    def one(i):
        fr = make_frames(codes[fc[i]], [sigma[i]], [2000 * number + first + i])
        x[var_off[i]:var_off[i + 1]] = fr.x[0]
        llr[var_off[i]:var_off[i + 1]] = fr.llr[0]
        syn[syn_off[i]:syn_off[i + 1]] = fr.syndrome[0]

    threads = _frame_threads(F, int(var_off[-1]) // max(1, F))
    if threads == 1:
        for i in range(F):
            one(i)
    else:  # each frame has its own generator, so the threads do not change the result
        from concurrent.futures import ThreadPoolExecutor
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(one, range(F)))
    return BatchFrames(fc, beta, sigma, var_off, syn_off, x, llr, syn)


def workload_frames(number: int, code, frames: int | None = None, first: int = 0,
                    beta: float | None = None) -> Frames:
    """Frames first..first+frames-1 of a named workload at efficiency beta."""
    w = WORKLOADS[number]
    return workload_frames_betas(number, code, [w["beta"] if beta is None else beta], frames, first)[0]


def workload_frames_betas(number: int, code, betas, frames: int | None = None, first: int = 0) -> list[Frames]:
    """workload_frames at several efficiencies: the same frames (bits, noise
    draws, syndromes), each at its own sigma; element i equals
    workload_frames(number, code, frames, first, betas[i])."""
    w = WORKLOADS[number]
    F = w["frames"] if frames is None else frames
    rate = w["rate"]
    seeds = [2000 * number + f for f in range(first, first + F)]
    sets = [np.full(F, sigma_for_capacity(rate / b)) for b in betas]
    out = make_frames_sigmas(code, sets, seeds)
    if w.get("punctured_cols"):
        Z = code.Z
        punct = np.concatenate([np.arange(j * Z, (j + 1) * Z) for j in w["punctured_cols"]])
        out = [rate_adapt(fr, punct, []) for fr in out]
    return out
