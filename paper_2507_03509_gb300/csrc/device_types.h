// Plain structures shared by the device code and the host side of the
// decoder library: the per-group control words and the two graph layouts
// the kernels walk.
#pragma once

namespace ldpcgb {

// One per group (its barrier), 128 bytes apart; the first one also holds the
// error word, the iteration total and the queue of waiting frames.
struct alignas(128) Ctrl {
    unsigned bar_count;
    unsigned bar_gen;
    int err;
    int next_frame;                  // frames handed out so far
    unsigned long long frame_iters;  // sum over frames of D
    int bad_site;                    // index-checking build: where the first bad index was seen
    long long bad_index;             // ... and its value
};

// Quasi-cyclic code: nonzero base blocks in row-major order (block id b).
// Check i*Z + t meets variable col[b]*Z + (t + shift[b]) mod Z.
// Messages of block b live at c2v[b*Z + p], p the variable's offset in its
// column block, so the variable-node side reads them unrotated.
struct QcDev {
    int mb, nb, Z, nblk;
    const int* row_ptr;            // [mb+1] first block of row i
    const int* blk_col;            // [nblk]
    const int* blk_shift;          // [nblk]
    const int* col_ptr;            // [nb+1] into col_blk
    const int* col_blk;            // [nblk] block ids of column j, ascending row
    const int* blk_row;            // [nblk] base row of block b
};

// General code: check-major CSR plus a variable-major list of edge ids.
struct CsrDev {
    int m, n;
    const int* row_ptr;            // [m+1]
    const int* col_idx;            // [E]
    const int* var_ptr;            // [n+1]
    const int* var_edge;           // [E] edge ids of variable v, ascending
    const int* row_order;          // [m] checks by ascending degree, ascending within a degree
};

}  // namespace ldpcgb
