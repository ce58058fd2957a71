"""Host-side model of how the frame-per-pair decoder splits a frame between
the two CTAs of a cluster (csr_frame_kernel<W, 2>): CTA r runs the runs of 32
checks of the degree-sorted order whose run index is r mod 2, owns the
1024-variable blocks b with b mod 2 = r, and stores a new message into the
other CTA's copy when the message's variable lies in the other CTA's blocks.

The model checks, for the codes the GPU tests decode with this schedule, that
every check and variable has exactly one owner and that every message a pass
reads in either CTA's copy was written in the current iteration (no stale
read); a pair that dropped the remote store, or gave a check or a variable to
both CTAs or to neither, fails it."""
import numpy as np
import pytest

from paper_2507_03509_gb300 import gen

THREADS = 1024      # threads of one CTA of the pair
PAIR_SHIFT = 10     # variable v belongs to CTA (v >> 10) & 1


def check_owner(m):
    """CTA that runs each check (by position in the degree-sorted order)."""
    owner = np.full(m, -1)
    for r in (0, 1):
        for tid in range(THREADS):
            i = ((tid >> 5) * 2 + r) * 32 + (tid & 31)
            while i < m:
                assert owner[i] == -1
                owner[i] = r
                i += 2 * THREADS
    return owner


def variable_owner(n):
    owner = np.full(n, -1)
    for r in (0, 1):
        v0 = r << PAIR_SHIFT
        while v0 < n:
            for tid in range(THREADS):
                if v0 + tid < n:
                    assert owner[v0 + tid] == -1
                    owner[v0 + tid] = r
            v0 += 2 << PAIR_SHIFT
    return owner


def degenerate_csr():
    rows = [[0], [0, 1], [1, 2, 3], [], [2, 4, 5, 6, 7, 8, 9, 10], [3, 4], [5, 11]]
    rowptr = np.cumsum([0] + [len(r) for r in rows]).astype(np.int32)
    return gen.CSRCode(len(rows), 13, rowptr, np.concatenate([np.asarray(r, np.int32) for r in rows]))


CODES = {
    "csr_n4096": lambda: gen.workload_code(1),
    "fd_n256": gen.wbp_fd_code,
    "degenerate": degenerate_csr,
    "decodable": lambda: gen.random_csr_code(2000, 1000, 3, {6: 1000}, seed=4242),
    "degree24": lambda: gen.random_csr_code(2048, 256, 3, {24: 256}, seed=4343),
}


@pytest.mark.parametrize("name", sorted(CODES))
def test_pair_partition_covers_and_reads_fresh_messages(name):
    code = CODES[name]()
    m, n = code.m, code.n
    rowptr, colidx = np.asarray(code.rowptr), np.asarray(code.colidx)
    E = colidx.size
    own_c = check_owner(m)
    own_v = variable_owner(n)
    assert (own_c >= 0).all() and (own_v >= 0).all()
    # a permutation of the rows stands for the degree-sorted order: ownership is by position
    order = np.random.default_rng(0).permutation(m)
    row_owner = np.empty(m, int)
    row_owner[order] = own_c
    edge_row = np.repeat(np.arange(m), np.diff(rowptr))
    edge_cta = row_owner[edge_row]
    var_cta = own_v[colidx]
    for it in (1, 2, 3):
        version = {0: np.zeros(E, int), 1: np.zeros(E, int)}
        for r in (0, 1):  # check pass: local store, and a remote one for the other CTA's variables
            mine = edge_cta == r
            version[r][mine] = it
            version[1 - r][mine & (var_cta != r)] = it
        # variable pass: each edge read in the copy of its variable's owner
        assert (np.where(var_cta == 0, version[0], version[1]) == it).all()
        # next check pass: each edge's old message read in the copy of its check's owner
        assert (np.where(edge_cta == 0, version[0], version[1]) == it).all()
