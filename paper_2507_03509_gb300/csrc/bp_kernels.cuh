// Device code of the GB300 syndrome-based sum-product decoder.
//
// One cooperative, persistent kernel runs the whole decode (paper, section
// "Early Termination"): every step is
//   phase A  check-node update of iteration k+1 for each running frame, with
//            the syndrome test of the decision x^(k) fused into the same pass
//            (the APP values it reads are the ones the decision uses);
//            FP64 reduction of q^(k) = sum_{v in V} |APP_v^(k)|;
//   barrier;
//   decide   PCE-ET / VNR-ET / D_max for each running frame (every CTA takes
//            the same decisions from the same global words);
//   phase B  variable-node update APP^(k+1) = Lch + sum of c2v^(k+1) for the
//            frames that go on, per-tile partials of q^(k+1); the hard
//            decision of frames that stopped is written out, and their slot
//            is refilled from the queue of waiting frames;
//   barrier.
// Frames run in "slots" (at most max_active_frames at once); stopped frames
// cost no more work.  Barriers spin with a time limit and turn an expired
// wait into an error word, never a hang.
#pragma once

#include <cstdint>
#include <type_traits>
#include <cuda_runtime.h>

#include "cn_math.cuh"
#include "device_types.h"

namespace ldpcgb {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kCPT = 2;                  // checks per thread in a check-node tile
constexpr int kVPT = 4;                  // variables per thread in a variable-node tile
constexpr int kCnTile = kThreads * kCPT;
constexpr int kVnTile = kThreads * kVPT;
constexpr int kMaxSlots = 1024;

enum : int { kErrNone = 0, kErrTimeout = 1, kErrSyndrome = 2, kErrBounds = 3 };

// Index checking (a build with -DLDPC_BOUNDS_CHECK): LDPC_IX(ctrl, i, len, site)
// yields i when 0 <= i < len; otherwise it records the first such index and
// its site in the control words, sets the error word (the decode returns
// LDPC_ERR_BOUNDS at its next synchronisation) and yields 0, an index inside
// every array, so the access stays in bounds.  Other builds: plain i.
#ifdef LDPC_BOUNDS_CHECK
static __device__ __noinline__ long long bounds_fail(Ctrl* c, long long i, int site) {
    if (atomicCAS(&c->err, kErrNone, kErrBounds) == kErrNone) {
        c->bad_site = site;
        c->bad_index = i;
    }
    return 0;
}
#define LDPC_IX(ctrl, i, len, site) \
    (((unsigned long long)(long long)(i) < (unsigned long long)(long long)(len)) ? (long long)(i) \
                                                                               : ldpcgb::bounds_fail((ctrl), (i), (site)))
// LDPC_IXN(ctrl, i, cnt, len, site): the same for the cnt elements i .. i + cnt - 1.
#define LDPC_IXN(ctrl, i, cnt, len, site) \
    (((long long)(i) >= 0 && (long long)(i) + (cnt) <= (long long)(len)) ? (long long)(i) \
                                                                         : ldpcgb::bounds_fail((ctrl), (i), (site)))
#else
#define LDPC_IX(ctrl, i, len, site) (i)
#define LDPC_IXN(ctrl, i, cnt, len, site) (i)
#endif
// Sites of the checks (reported with the bad index).
enum : int {
    kIxCnLlr = 1, kIxCnApp, kIxCnMsg, kIxCnSyn, kIxVnLlr, kIxVnMsg, kIxVnApp, kIxVnPart, kIxBits,
    kIxCsrVar, kIxCsrMsg, kIxSlot, kIxFrame, kIxFlowFlag, kIxFlowSlot
};
enum : int { kModeFirst = 0, kModeFull = 1, kModeSynd = 2 };
enum : int { kRuleNone = 0, kRulePce = 1, kRulePceVnr = 2 };

constexpr int kMaxGrid = 4096;            // largest grid either decoder kernel is launched with

constexpr int kMaxGroups = 64;

constexpr int kMaxCodes = 4;              // codes one decode call may mix

// Dynamic shared memory of bp_decode_kernel for a group of `slots_per_group`
// slots: per slot its q^(k-1) (double) and five ints (frame, iteration, code,
// and the two slot lists of a step), rounded up to 128 bytes.  Both launchers
// size the launch, the attribute and the occupancy query with it.
constexpr int kSmemPerSlot = (int)(sizeof(double) + 5 * sizeof(int));
__host__ __device__ constexpr size_t decode_smem_bytes(int slots_per_group) {
    return (size_t)((slots_per_group * kSmemPerSlot + 127) / 128) * 128;
}

// Sizes of one code as the decoder walks it.
template <class Code>
struct CodeInfo {
    Code code;
    int n, m;
    long long E;
    int swords;                    // packed syndrome words per frame
    int cn_tiles, vn_tiles;        // check-node / variable-node items per frame
    int cn_chunk, vn_chunk;        // QC items: checks of one base row / variables of one base column
    int nqb;                       // q-blocks per frame: fixed runs of kQBlock variables
    int vec4;                      // 16-byte variable-node path allowed (Z % 4 == 0, aligned Lch)
};

template <class Code>
struct CodeSet {
    CodeInfo<Code> c[kMaxCodes];
    int count;
};

template <typename T>
struct Params {
    int frames, max_iter, rule, vnr_first_iter;
    T lmax;
    // frames: code, and where its values start in the concatenated buffers
    // (NULL arrays: one code, frame f at f*n and f*swords)
    const int* frame_code;         // [frames]
    const long long* var_off;      // [frames] offset of frame f in llr / bits_out
    const long long* sb_off;       // [frames] offset of frame f in sbits (words)
    const float* llr;              // channel LLRs of all frames
    const unsigned* sbits;         // packed syndromes of all frames
    unsigned char* bits_out;       // decisions of all frames
    unsigned char* flags_out;      // [frames]
    int* iters_out;                // [frames]
    int slots;
    long long slot_E;              // per-slot strides (the largest code's sizes)
    int slot_n, slot_nqb;
    int cn_tiles_max, vn_tiles_max;
    T* c2v;                        // [slots][slot_E]
    T* app;                        // [slots][slot_n]
    double* qpart;                 // [slots][slot_nqb * kWarps] per-warp partial sums of q
    double* q0part;                // [slots][slot_nqb * kWarps]
    double* qval;                  // [slots][kQParts] q^(k) summed over fixed ranges of partials
    double* q0val;                 // [slots][kQParts] the same for q^(0)
    int* unsat;                    // [2][slots]
    Ctrl* ctrl;
    int trace_iters;
    T* trace_c2v;                  // [trace_iters][frames][E]
    T* trace_app;                  // [trace_iters][frames][n]
    double* trace_q;               // [trace_iters][frames]
    unsigned long long timeout_ns;
    unsigned bar_extra;            // test hook: arrivals the first barrier waits for beyond the grid
    int groups;                    // independent CTA groups, each with its own slots and barrier
    int slots_per_group;           // slots = groups * slots_per_group
    int* new_frame;                // [slots] frame taken from the queue by a slot that stopped
    // learned weights (NULL: none): check-to-variable messages of iteration k are
    // scaled by wts[min(k, w_iters) - 1][wcls[key]], key = base block (QC) or edge (CSR)
    const float* wts;
    const int* wcls;
    int w_iters, w_classes;
};

// Where one running frame's data lives (slot s decoding frame f of code ci).
template <typename T>
struct FrameCtx {
    T* c2v;                        // the slot's messages
    T* app;                        // the slot's APP values
    const float* llr;              // the frame's channel LLRs
    const unsigned* sbits;         // the frame's packed syndrome
    unsigned char* bits;           // the frame's decision (output)
    double* qpart;                 // the slot's partial sums of q
    double* q0part;
    int f, n;
    long long E;
    int cn_chunk, vn_chunk, nqb, vec4;
    int swords;                    // packed syndrome words of the frame
    const float* wrow;             // weights of the iteration the check pass computes (NULL: none)
    Ctrl* ctrl;                    // control words (error reports of the index-checking build)
};

// A check message scaled by its learned weight (W: the weighted kernel); the
// unweighted kernel stores the message as computed.
template <bool W, typename T>
__device__ __forceinline__ T weighted(const Params<T>& p, const FrameCtx<T>& fc, T msg, int key) {
    if constexpr (W) return msg * T(__ldg(fc.wrow + __ldg(p.wcls + key)));
    else return msg;
}

template <typename T, class Code>
__device__ __forceinline__ FrameCtx<T> frame_ctx(const Params<T>& p, const CodeInfo<Code>& ci, int s, int f) {
    s = (int)LDPC_IX(p.ctrl, s, p.slots, kIxSlot);
    f = (int)LDPC_IX(p.ctrl, f, p.frames, kIxFrame);
    FrameCtx<T> c;
    c.c2v = p.c2v + (size_t)s * (size_t)p.slot_E;
    c.app = p.app + (size_t)s * (size_t)p.slot_n;
    const long long vo = p.var_off ? p.var_off[f] : (long long)f * ci.n;
    const long long so = p.sb_off ? p.sb_off[f] : (long long)f * ci.swords;
    c.llr = p.llr + vo;
    c.bits = p.bits_out + vo;
    c.sbits = p.sbits + so;
    c.qpart = p.qpart + (size_t)s * p.slot_nqb * kWarps;
    c.q0part = p.q0part + (size_t)s * p.slot_nqb * kWarps;
    c.f = f;
    c.n = ci.n;
    c.E = ci.E;
    c.cn_chunk = ci.cn_chunk;
    c.vn_chunk = ci.vn_chunk;
    c.nqb = ci.nqb;
    c.vec4 = ci.vec4;
    c.swords = ci.swords;
    c.wrow = nullptr;
    c.ctrl = p.ctrl;
    return c;
}

// The weight row of the check pass that follows k completed iterations.
template <typename T>
__device__ __forceinline__ const float* weight_row(const Params<T>& p, int k) {
    if (!p.wts) return nullptr;
    const int r = min(k + 1, p.w_iters) - 1;
    return p.wts + (size_t)r * p.w_classes;
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ int ld_volatile(const int* p) { return *(const volatile int*)p; }
__device__ __forceinline__ double ld_volatile(const double* p) { return *(const volatile double*)p; }


// Barrier over the nblocks CTAs of one group (a cooperative launch keeps them
// all resident).  The group's arrival counter only grows: thread 0 of each
// CTA adds 1 with a release reduction (no reply to wait for) and then waits,
// with acquire loads, until the counter reaches nblocks times the number of
// barriers passed so far (`epoch`, counted locally).  A wait longer than
// timeout_ns (or any error raised elsewhere) ends it with the error word set;
// the return value says whether the decode may go on.  `extra` (a test hook)
// makes the barrier wait for more CTAs than exist.
__device__ __forceinline__ void red_release_add(unsigned* p, unsigned v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ bool grid_sync(Ctrl* bar, int* err, unsigned nblocks, unsigned epoch,
                                          unsigned long long timeout_ns, unsigned extra = 0) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned target = epoch * nblocks + extra;
        red_release_add(&bar->bar_count, 1u);
        unsigned spins = 0;
        unsigned long long t0 = 0;
        while ((int)(ld_acquire(&bar->bar_count) - target) < 0) {
            if (++spins > 32) {
                if (t0 == 0) t0 = global_ns();
                __nanosleep(64);
                if (ld_volatile(err) != kErrNone) break;
                if (global_ns() - t0 > timeout_ns) {
                    atomicCAS(err, kErrNone, kErrTimeout);
                    break;
                }
            }
        }
    }
    __syncthreads();
    return ld_volatile(err) == kErrNone;
}

__device__ __forceinline__ unsigned syndrome_bit(const unsigned* sb, int row) {
    return (__ldg(sb + (row >> 5)) >> (row & 31)) & 1u;
}

// ---------------------------------------------------------------------------
// Quasi-cyclic check-node item: checks t in [t0, t0 + cn_chunk) of base row
// i.  The row's block pointers are set up once; each thread then walks the
// chunk two checks at a time (both checks' loads issued before any
// arithmetic).  MODE and SYND are compile-time so the hot loop carries no
// mode tests: kModeFirst reads Lch with c2v = 0, kModeFull reads APP and the
// old c2v, kModeSynd only tests the syndrome of the current decision.
// ---------------------------------------------------------------------------
constexpr int kQcCnChunk = 2048;         // default checks of one base row per item (multiple of 2*kThreads)
constexpr int kQcVnChunk = 4096;         // default variables of one base column per item (multiple of kQBlock)
constexpr int kQBlock = 4 * kThreads;    // variables per q partial sum (per warp: 128)
constexpr int kQParts = 8;               // a frame's q is reduced in this many fixed ranges, by different CTAs

// Bulk L2 prefetch of a window [ptr, ptr + bytes) by the copy engine: one
// instruction for the whole window, no registers held while the lines arrive.
// Only its 16-byte-aligned interior is requested (the bulk copy needs 16-byte
// alignment), so no byte outside the window is touched.
__device__ __forceinline__ void prefetch_l2_range(const void* ptr, size_t bytes) {
    const uintptr_t lo = ((uintptr_t)ptr + 15) & ~uintptr_t(15);
    const uintptr_t hi = ((uintptr_t)ptr + bytes) & ~uintptr_t(15);
    if (hi > lo) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(lo), "r"((unsigned)(hi - lo)) : "memory");
}

// Bulk L2 prefetch of a QC check item's windows: per block of the row, the
// rotated run of positions the item reads, in one or two pieces, of the
// messages and of the APP values (of Lch in the first iteration).  Issued by
// one thread: one copy-engine request per piece, no registers held while the
// lines arrive.  (Prefetching the CTA's next item as well measured slower.)
template <bool FIRST, typename T>
__device__ __forceinline__ void qc_cn_prefetch(const QcDev& q, const FrameCtx<T>& fc, int i, int t0, int b0, int d) {
    const int Z = q.Z;
    const int len = min(t0 + fc.cn_chunk, Z) - t0;
    for (int j = 0; j < d; ++j) {
        int st = t0 + __ldg(q.blk_shift + b0 + j);
        st = st >= Z ? st - Z : st;
        const int first = min(len, Z - st);
        if constexpr (FIRST) {
            const float* b = fc.llr + (size_t)__ldg(q.blk_col + b0 + j) * Z;
            prefetch_l2_range(b + st, (size_t)first * sizeof(float));
            if (len > first) prefetch_l2_range(b, (size_t)(len - first) * sizeof(float));
        } else {
            const T* b = fc.c2v + (size_t)(b0 + j) * Z;
            prefetch_l2_range(b + st, (size_t)first * sizeof(T));
            if (len > first) prefetch_l2_range(b, (size_t)(len - first) * sizeof(T));
            const T* a = fc.app + (size_t)__ldg(q.blk_col + b0 + j) * Z;
            prefetch_l2_range(a + st, (size_t)first * sizeof(T));
            if (len > first) prefetch_l2_range(a, (size_t)(len - first) * sizeof(T));
        }
    }
}

template <int D, int MODE, bool SYND, bool W, typename T>
__device__ __forceinline__ bool qc_cn_item(const Params<T>& p, const QcDev& q, const FrameCtx<T>& fc, int i, int t0,
                                           int b0) {
    const int Z = q.Z;
    const int t_end = min(t0 + fc.cn_chunk, Z);
    T* c2v = fc.c2v;
    const T* app = fc.app;
    const float* llr = fc.llr;
    const unsigned* sb = fc.sbits + (size_t)i * Z / 32;
    const int sbit0 = (i * Z) & 31;  // bit offset of check (i, 0) in its word
    // per-block offsets: variable column (col*Z) and message block ((b0+j)*Z)
    int sh[D], vo[D], mo[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        sh[j] = __ldg(q.blk_shift + b0 + j);
        vo[j] = __ldg(q.blk_col + b0 + j) * Z;
        mo[j] = (b0 + j) * Z;
    }
    // L2 prefetch of the item's windows: many more lines in flight than the
    // loads below could keep
#ifndef LDPC_BOUNDS_CHECK  // the index-checking build issues no unchecked prefetches
    if constexpr (MODE != kModeSynd) {
        if (threadIdx.x == 0) qc_cn_prefetch<MODE == kModeFirst, T>(q, fc, i, t0, b0, D);
    }
#endif
    // checks in flight per thread
    constexpr int NC = 2;
    bool unsat = false;
    for (int tb = t0 + (int)threadIdx.x; tb < t_end; tb += NC * kThreads) {
        int pos[NC][D];
        T a[NC][D], o[NC][D];
        bool ok[NC];
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const int t = tb + c * kThreads;
            ok[c] = t < t_end;
#pragma unroll
            for (int j = 0; j < D; ++j) {
                int pp = t + sh[j];
                pp = pp >= Z ? pp - Z : pp;
                pp = ok[c] ? pp : 0;  // in-bounds dummy position for the guarded tail
                pos[c][j] = pp;
                if constexpr (MODE == kModeFirst) {
                    a[c][j] = T(__ldg(llr + LDPC_IX(p.ctrl, vo[j] + pp, fc.n, kIxCnLlr)));
                    o[c][j] = T(0);
                } else {
                    a[c][j] = app[LDPC_IX(p.ctrl, vo[j] + pp, fc.n, kIxCnApp)];
                    o[c][j] = MODE == kModeFull ? c2v[LDPC_IX(p.ctrl, mo[j] + pp, fc.E, kIxCnMsg)] : T(0);
                }
            }
        }
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if (!ok[c]) continue;
            const int t = tb + c * kThreads;
            const int bit = sbit0 + t;
            const unsigned sbit =
                (__ldg(sb + LDPC_IX(p.ctrl, (sb - fc.sbits) + (bit >> 5), fc.swords, kIxCnSyn) - (sb - fc.sbits)) >>
                 (bit & 31)) & 1u;
            if constexpr (SYND) {
                unsigned pr = sbit;
#pragma unroll
                for (int j = 0; j < D; ++j) pr ^= (unsigned)(a[c][j] < T(0));
                unsat |= pr != 0u;
            }
            if constexpr (MODE != kModeSynd) {
                T v[D], out[D];
#pragma unroll
                for (int j = 0; j < D; ++j) v[j] = clampm(a[c][j] - o[c][j], p.lmax);
                cn_core<D>(v, sbit, p.lmax, out);
#pragma unroll
                for (int j = 0; j < D; ++j)
                    c2v[LDPC_IX(p.ctrl, mo[j] + pos[c][j], fc.E, kIxCnMsg)] = weighted<W>(p, fc, out[j], b0 + j);
            }
        }
    }
    return unsat;
}

// Rows of weight > 6: runtime degree, local arrays.
template <int MODE, bool SYND, bool W, typename T>
__device__ bool qc_cn_item_n(const Params<T>& p, const QcDev& q, const FrameCtx<T>& fc, int i, int t0, int b0,
                             int d) {
    const int Z = q.Z;
    const int t_end = min(t0 + fc.cn_chunk, Z);
    T* c2v = fc.c2v;
    const T* app = fc.app;
    const float* llr = fc.llr;
    const unsigned* sb = fc.sbits;
    bool unsat = false;
    for (int t = t0 + (int)threadIdx.x; t < t_end; t += kThreads) {
        (void)LDPC_IX(p.ctrl, (i * Z + t) >> 5, fc.swords, kIxCnSyn);
        const unsigned sbit = syndrome_bit(sb, i * Z + t);
        T v[kMaxDeg], out[kMaxDeg];
        unsigned pr = sbit;
        for (int j = 0; j < d; ++j) {
            int pp = t + __ldg(q.blk_shift + b0 + j);
            pp = pp >= Z ? pp - Z : pp;
            const int vi = (int)LDPC_IX(p.ctrl, __ldg(q.blk_col + b0 + j) * Z + pp, fc.n, kIxCnApp);
            T a, o = T(0);
            if (MODE == kModeFirst) {
                a = T(__ldg(llr + vi));
            } else {
                a = app[vi];
                if (MODE == kModeFull) o = c2v[LDPC_IX(p.ctrl, (b0 + j) * Z + pp, fc.E, kIxCnMsg)];
            }
            pr ^= (unsigned)(a < T(0));
            v[j] = clampm(a - o, p.lmax);
        }
        if (SYND) unsat |= pr != 0u;
        if constexpr (MODE != kModeSynd) {
            cn_core_n(v, d, sbit, p.lmax, out);
            for (int j = 0; j < d; ++j) {
                int pp = t + __ldg(q.blk_shift + b0 + j);
                pp = pp >= Z ? pp - Z : pp;
                c2v[LDPC_IX(p.ctrl, (b0 + j) * Z + pp, fc.E, kIxCnMsg)] = weighted<W>(p, fc, out[j], b0 + j);
            }
        }
    }
    return unsat;
}

template <int MODE, bool SYND, bool W, typename T>
__device__ __forceinline__ bool qc_cn_dispatch(const Params<T>& p, const QcDev& q, const FrameCtx<T>& fc, int i,
                                               int t0, int b0, int d) {
    switch (d) {
        case 0: {
            bool unsat = false;
            if (SYND) {
                const unsigned* sb = fc.sbits;
                const int t_end = min(t0 + fc.cn_chunk, q.Z);
                for (int t = t0 + (int)threadIdx.x; t < t_end; t += kThreads)
                    unsat |= syndrome_bit(sb, i * q.Z + t) != 0u;
            }
            return unsat;
        }
        case 1: return qc_cn_item<1, MODE, SYND, W, T>(p, q, fc, i, t0, b0);
        case 2: return qc_cn_item<2, MODE, SYND, W, T>(p, q, fc, i, t0, b0);
        case 3: return qc_cn_item<3, MODE, SYND, W, T>(p, q, fc, i, t0, b0);
        case 4: return qc_cn_item<4, MODE, SYND, W, T>(p, q, fc, i, t0, b0);
        case 5: return qc_cn_item<5, MODE, SYND, W, T>(p, q, fc, i, t0, b0);
        case 6: return qc_cn_item<6, MODE, SYND, W, T>(p, q, fc, i, t0, b0);
        default: return qc_cn_item_n<MODE, SYND, W, T>(p, q, fc, i, t0, b0, d);
    }
}

template <bool W, typename T>
__device__ __forceinline__ bool cn_tile(const Params<T>& p, const QcDev& q, const FrameCtx<T>& fc, int mode,
                                        bool want_synd, int tile) {
    const int per_row = (q.Z + fc.cn_chunk - 1) / fc.cn_chunk;
    const int i = tile / per_row;
    const int t0 = (tile - i * per_row) * fc.cn_chunk;
    const int b0 = __ldg(q.row_ptr + i);
    const int d = __ldg(q.row_ptr + i + 1) - b0;
    if (mode == kModeFirst) return qc_cn_dispatch<kModeFirst, false, W, T>(p, q, fc, i, t0, b0, d);
    if (mode == kModeSynd) return qc_cn_dispatch<kModeSynd, true, false, T>(p, q, fc, i, t0, b0, d);
    if (want_synd) return qc_cn_dispatch<kModeFull, true, W, T>(p, q, fc, i, t0, b0, d);
    return qc_cn_dispatch<kModeFull, false, W, T>(p, q, fc, i, t0, b0, d);
}

// ---------------------------------------------------------------------------
// CSR check-node tile: checks tile*kCnTile ...; one check per thread-slot.
// ---------------------------------------------------------------------------
template <int D, bool W, typename T>
__device__ __forceinline__ bool csr_cn_check(const Params<T>& p, const CsrDev& g, const FrameCtx<T>& fc, int mode,
                                             bool want_synd, int row, int e0) {
    T* c2v = fc.c2v;
    const T* app = fc.app;
    const float* llr = fc.llr;
    const unsigned sbit = syndrome_bit(fc.sbits, row);
    T a[D], o[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const int vi = (int)LDPC_IX(p.ctrl, __ldg(g.col_idx + e0 + j), fc.n, kIxCsrVar);
        o[j] = T(0);
        if (mode == kModeFirst) {
            a[j] = T(__ldg(llr + vi));
        } else {
            a[j] = app[vi];
            if (mode == kModeFull) o[j] = c2v[LDPC_IX(p.ctrl, e0 + j, fc.E, kIxCsrMsg)];
        }
    }
    bool unsat = false;
    if (want_synd) {
        unsigned pr = sbit;
#pragma unroll
        for (int j = 0; j < D; ++j) pr ^= (unsigned)(a[j] < T(0));
        unsat = pr != 0u;
    }
    if (mode == kModeSynd) return unsat;
    T v[D], out[D];
#pragma unroll
    for (int j = 0; j < D; ++j) v[j] = clampm(a[j] - o[j], p.lmax);
    cn_core<D>(v, sbit, p.lmax, out);
#pragma unroll
    for (int j = 0; j < D; ++j) c2v[LDPC_IX(p.ctrl, e0 + j, fc.E, kIxCsrMsg)] = weighted<W>(p, fc, out[j], e0 + j);
    return unsat;
}

template <bool W, typename T>
__device__ bool csr_cn_check_n(const Params<T>& p, const CsrDev& g, const FrameCtx<T>& fc, int mode, bool want_synd,
                               int row, int e0, int d) {
    T* c2v = fc.c2v;
    const T* app = fc.app;
    const float* llr = fc.llr;
    const unsigned sbit = syndrome_bit(fc.sbits, row);
    if (d == 0) return want_synd && sbit != 0u;
    T v[kMaxDeg], out[kMaxDeg];
    unsigned pr = sbit;
    for (int j = 0; j < d; ++j) {
        const int vi = (int)LDPC_IX(p.ctrl, __ldg(g.col_idx + e0 + j), fc.n, kIxCsrVar);
        T a, o = T(0);
        if (mode == kModeFirst) {
            a = T(__ldg(llr + vi));
        } else {
            a = app[vi];
            if (mode == kModeFull) o = c2v[LDPC_IX(p.ctrl, e0 + j, fc.E, kIxCsrMsg)];
        }
        pr ^= (unsigned)(a < T(0));
        v[j] = clampm(a - o, p.lmax);
    }
    const bool unsat = want_synd && pr != 0u;
    if (mode == kModeSynd) return unsat;
    cn_core_n(v, d, sbit, p.lmax, out);
    for (int j = 0; j < d; ++j) c2v[LDPC_IX(p.ctrl, e0 + j, fc.E, kIxCsrMsg)] = weighted<W>(p, fc, out[j], e0 + j);
    return unsat;
}

template <bool W, typename T>
__device__ __forceinline__ bool cn_tile(const Params<T>& p, const CsrDev& g, const FrameCtx<T>& fc, int mode,
                                        bool want_synd, int tile) {
    bool unsat = false;
    for (int c = 0; c < kCPT; ++c) {
        const int row = tile * kCnTile + c * kThreads + (int)threadIdx.x;
        if (row >= g.m) break;
        const int e0 = __ldg(g.row_ptr + row);
        const int d = __ldg(g.row_ptr + row + 1) - e0;
        switch (d) {
            case 1: unsat |= csr_cn_check<1, W, T>(p, g, fc, mode, want_synd, row, e0); break;
            case 2: unsat |= csr_cn_check<2, W, T>(p, g, fc, mode, want_synd, row, e0); break;
            case 3: unsat |= csr_cn_check<3, W, T>(p, g, fc, mode, want_synd, row, e0); break;
            case 4: unsat |= csr_cn_check<4, W, T>(p, g, fc, mode, want_synd, row, e0); break;
            case 5: unsat |= csr_cn_check<5, W, T>(p, g, fc, mode, want_synd, row, e0); break;
            case 6: unsat |= csr_cn_check<6, W, T>(p, g, fc, mode, want_synd, row, e0); break;
            default: unsat |= csr_cn_check_n<W, T>(p, g, fc, mode, want_synd, row, e0, d); break;
        }
    }
    return unsat;
}

// ---------------------------------------------------------------------------
// Variable-node tiles: APP^(k+1) = Lch + sum of c2v^(k+1) over the variable's
// checks in ascending check order; per-warp sums of |APP| over V (degree > 1)
// and, for the first iteration, of |Lch| over V.  The per-warp partials go to
// fixed positions (tile * kWarps + warp), so q is a fixed-order sum.
// ---------------------------------------------------------------------------
// The warp's butterfly adds in the message type (each lane adds the same two
// operands, commuted, so all lanes hold the same sum); its result is widened
// to FP64, and every addition above the warp is an FP64 addition in a fixed
// order.  An FP64 butterfly was measured 11 % slower on the whole decoder
// (GB300's FP64 rate is a small fraction of its FP32 rate); q differs from the
// oracle's by FP32 APP rounding far more than by this tree.
template <typename T>
__device__ __forceinline__ void warp_sum_to(T acc, double* slot) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) *slot = double(acc);
}
template <typename T>
__device__ __forceinline__ void warp_sum_store(T acc, double* dst) {
    warp_sum_to(acc, dst + (threadIdx.x >> 5));
}

// Trace of c2v^(k+1) for variable j*Z + u, written from the variable side so
// that only iterations a frame completes are recorded.  Edge order is the
// lifted matrix's row-major order: row i*Z + t, blocks of row i in turn.
template <typename T>
__device__ void trace_c2v_qc(const Params<T>& p, const QcDev& q, const FrameCtx<T>& fc, int k, int u, int cb0,
                             int dv) {
    const int Z = q.Z;
    const T* c2v = fc.c2v;
    T* tr = p.trace_c2v + ((size_t)k * p.frames + fc.f) * (size_t)fc.E;
    for (int b = 0; b < dv; ++b) {
        const int blk = __ldg(q.col_blk + cb0 + b);
        const int i = __ldg(q.blk_row + blk);
        const int r0 = __ldg(q.row_ptr + i);
        const int d = __ldg(q.row_ptr + i + 1) - r0;
        int t = u - __ldg(q.blk_shift + blk);
        t = t < 0 ? t + Z : t;
        tr[(size_t)r0 * Z + (size_t)t * d + (blk - r0)] = c2v[(size_t)blk * Z + u];
    }
}

// Quasi-cyclic variable-node item: variables u in [u0, u0 + vn_chunk) of
// base column j.  DV > 0: compile-time column degree; DV == 0: runtime dv.
// The item is walked in q-blocks of kQBlock variables (u0 is a multiple of
// kQBlock); in each, thread t handles variables 4t .. 4t+3, so q's partial
// sums -- one per q-block and warp, at a fixed position -- do not depend on
// the item size or on the load path.  With vec (Z % 4 == 0, aligned Lch) the
// four variables move as 16-byte loads and stores.
template <int DV, typename T>
__device__ __forceinline__ void qc_vn_cols(const Params<T>& p, const QcDev& q, const FrameCtx<T>& fc, int k, int j,
                                           int u0, int cb0, int dv) {
    constexpr bool kFixed = DV > 0;
    const int Z = q.Z;
    const int u_end = min(u0 + fc.vn_chunk, Z);
    const int nd = kFixed ? DV : dv;
    const bool inV = nd > 1;
    const bool want_q0 = (k == 0) && p.vnr_first_iter <= 1;
    const bool tracing = k < p.trace_iters;
    const T* c2v = fc.c2v;
    T* app = fc.app + j * Z;
    const float* llr = fc.llr + j * Z;
    const T* cb[kFixed ? DV : 1];
    if constexpr (kFixed) {
#pragma unroll
        for (int b = 0; b < DV; ++b) cb[b] = c2v + __ldg(q.col_blk + cb0 + b) * Z;
    }
    bool vec = false;
    if constexpr (sizeof(T) == 4) vec = fc.vec4 != 0;
    const int qb_per_col = (Z + kQBlock - 1) / kQBlock;
#ifndef LDPC_BOUNDS_CHECK
    // bulk L2 prefetch of the item's message blocks and channel values (contiguous), by one thread
    if (threadIdx.x == 0) {
        prefetch_l2_range(llr + u0, (size_t)(u_end - u0) * sizeof(float));
        for (int b = 0; b < nd; ++b)
            prefetch_l2_range(c2v + (size_t)__ldg(q.col_blk + cb0 + b) * Z + u0, (size_t)(u_end - u0) * sizeof(T));
    }
#endif
    for (int ub = u0; ub < u_end; ub += kQBlock) {
        const int u = ub + 4 * (int)threadIdx.x;
        T acc = T(0), acc0 = T(0);
        if (u < u_end) {
            T L[4], sum[4];
            if (vec) {
                (void)LDPC_IXN(p.ctrl, (long long)j * Z + u, 4, fc.n, kIxVnLlr);
                const float4 l4 = __ldg(reinterpret_cast<const float4*>(llr + u));
                float4 s4 = l4;
                if constexpr (kFixed) {
                    float4 m[DV];
#pragma unroll
                    for (int b = 0; b < DV; ++b) {
                        (void)LDPC_IXN(p.ctrl, (cb[b] - c2v) + u, 4, fc.E, kIxVnMsg);
                        m[b] = *reinterpret_cast<const float4*>(cb[b] + u);
                    }
#pragma unroll
                    for (int b = 0; b < DV; ++b) {
                        s4.x += m[b].x;
                        s4.y += m[b].y;
                        s4.z += m[b].z;
                        s4.w += m[b].w;
                    }
                } else {
                    for (int b = 0; b < nd; ++b) {
                        const long long mi =
                            LDPC_IXN(p.ctrl, (long long)__ldg(q.col_blk + cb0 + b) * Z + u, 4, fc.E, kIxVnMsg);
                        const float4 m = *reinterpret_cast<const float4*>(c2v + mi);
                        s4.x += m.x;
                        s4.y += m.y;
                        s4.z += m.z;
                        s4.w += m.w;
                    }
                }
                *reinterpret_cast<float4*>(reinterpret_cast<float*>(app) + u) = s4;
                L[0] = T(l4.x), L[1] = T(l4.y), L[2] = T(l4.z), L[3] = T(l4.w);
                sum[0] = T(s4.x), sum[1] = T(s4.y), sum[2] = T(s4.z), sum[3] = T(s4.w);
            } else {
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if (u + e < u_end) {
                        (void)LDPC_IX(p.ctrl, (long long)j * Z + u + e, fc.n, kIxVnApp);
                        L[e] = T(__ldg(llr + u + e));
                        T t = L[e];
                        if constexpr (kFixed) {
#pragma unroll
                            for (int b = 0; b < DV; ++b)
                                t += cb[b][LDPC_IX(p.ctrl, (cb[b] - c2v) + u + e, fc.E, kIxVnMsg) - (cb[b] - c2v)];
                        } else {
                            for (int b = 0; b < nd; ++b)
                                t += c2v[LDPC_IX(p.ctrl, (long long)__ldg(q.col_blk + cb0 + b) * Z + u + e, fc.E,
                                                 kIxVnMsg)];
                        }
                        sum[e] = t;
                        app[u + e] = t;
                    } else {
                        L[e] = T(0);
                        sum[e] = T(0);
                    }
                }
            }
            if (inV) {
                acc = (absm(sum[0]) + absm(sum[1])) + (absm(sum[2]) + absm(sum[3]));
                acc0 = (absm(L[0]) + absm(L[1])) + (absm(L[2]) + absm(L[3]));
            }
            if (tracing) {
                for (int e = 0; e < 4 && u + e < u_end; ++e) {
                    if (p.trace_app) p.trace_app[((size_t)k * p.frames + fc.f) * (size_t)fc.n + j * Z + u + e] = sum[e];
                    if (p.trace_c2v) trace_c2v_qc(p, q, fc, k, u + e, cb0, nd);
                }
            }
        }
        const size_t part = (size_t)LDPC_IXN(p.ctrl, ((long long)j * qb_per_col + ub / kQBlock) * kWarps, kWarps,
                                             (long long)p.slot_nqb * kWarps, kIxVnPart);
        warp_sum_store(acc, fc.qpart + part);
        if (want_q0) warp_sum_store(acc0, fc.q0part + part);
    }
}

template <typename T>
__device__ __forceinline__ void vn_tile(const Params<T>& p, const QcDev& q, const FrameCtx<T>& fc, int k, int tile) {
    const int per_col = (q.Z + fc.vn_chunk - 1) / fc.vn_chunk;
    const int j = tile / per_col;
    const int u0 = (tile - j * per_col) * fc.vn_chunk;
    const int cb0 = __ldg(q.col_ptr + j);
    const int dv = __ldg(q.col_ptr + j + 1) - cb0;
    switch (dv) {
        case 1: qc_vn_cols<1, T>(p, q, fc, k, j, u0, cb0, dv); break;
        case 2: qc_vn_cols<2, T>(p, q, fc, k, j, u0, cb0, dv); break;
        case 3: qc_vn_cols<3, T>(p, q, fc, k, j, u0, cb0, dv); break;
        case 4: qc_vn_cols<4, T>(p, q, fc, k, j, u0, cb0, dv); break;
        default: qc_vn_cols<0, T>(p, q, fc, k, j, u0, cb0, dv); break;
    }
}

template <typename T>
__device__ __forceinline__ void vn_tile(const Params<T>& p, const CsrDev& g, const FrameCtx<T>& fc, int k, int tile) {
    const bool want_q0 = (k == 0) && p.vnr_first_iter <= 1;
    const T* c2v = fc.c2v;
    T* app = fc.app;
    const float* llr = fc.llr;
    T acc = T(0), acc0 = T(0);
#pragma unroll
    for (int c = 0; c < kVPT; ++c) {
        const int v = tile * kVnTile + c * kThreads + (int)threadIdx.x;
        if (v < g.n) {
            const int a0 = __ldg(g.var_ptr + v), a1 = __ldg(g.var_ptr + v + 1);
            const T L = T(__ldg(llr + v));
            T sum = L;
            for (int a = a0; a < a1; ++a) sum += c2v[LDPC_IX(p.ctrl, __ldg(g.var_edge + a), fc.E, kIxCsrMsg)];
            app[v] = sum;
            if (a1 - a0 > 1) {
                acc += absm(sum);
                acc0 += absm(L);
            }
            if (k < p.trace_iters) {
                if (p.trace_app) p.trace_app[((size_t)k * p.frames + fc.f) * (size_t)fc.n + v] = sum;
                if (p.trace_c2v) {
                    T* tr = p.trace_c2v + ((size_t)k * p.frames + fc.f) * (size_t)fc.E;
                    for (int a = a0; a < a1; ++a) tr[__ldg(g.var_edge + a)] = c2v[__ldg(g.var_edge + a)];
                }
            }
        }
    }
    const size_t part = (size_t)tile * kWarps;
    warp_sum_store(acc, fc.qpart + part);
    if (want_q0) warp_sum_store(acc0, fc.q0part + part);
}

// Hard decision of a stopped frame: bits = [APP < 0] over the tile's variables.
template <typename T>
__device__ __forceinline__ void final_tile(const FrameCtx<T>& fc, int tile) {
    for (int c = 0; c < kVPT; ++c) {
        const long long v = (long long)tile * kVnTile + c * kThreads + threadIdx.x;
        if (v < fc.n) fc.bits[v] = (unsigned char)(fc.app[v] < T(0));
    }
}

// QC items run per column block, so the variable range of an item differs.
template <typename T>
__device__ __forceinline__ void final_tile(const QcDev& q, const FrameCtx<T>& fc, int tile) {
    const int per_col = (q.Z + fc.vn_chunk - 1) / fc.vn_chunk;
    const int j = tile / per_col;
    const int u0 = (tile - j * per_col) * fc.vn_chunk;
    const int u_end = min(u0 + fc.vn_chunk, q.Z);
    const T* app = fc.app + j * q.Z;
    unsigned char* bits = fc.bits + j * q.Z;
    for (int u = u0 + (int)threadIdx.x; u < u_end; u += kThreads) {
        (void)LDPC_IX(fc.ctrl, (long long)j * q.Z + u, fc.n, kIxBits);
        bits[u] = (unsigned char)(app[u] < T(0));
    }
}
template <typename T>
__device__ __forceinline__ void final_tile(const CsrDev&, const FrameCtx<T>& fc, int tile) {
    final_tile(fc, tile);
}

// Deterministic FP64 sum of a frame's per-tile partials (fixed order); the
// result is valid in thread 0, its only reader.  Additions of a known +0.0 are
// skipped: groups of kThreads elements that lie wholly past `count`, butterfly
// steps and warps without elements.  They would add +0.0 to a sum of
// non-negative terms, which changes nothing, and FP64 instructions are scarce
// on this part (about two per clock per SM).
__device__ __forceinline__ double block_sum_fixed(const double* part, int count, double* s_red) {
    double acc = 0.0;
    for (int base = 0; base < count; base += 8 * kThreads) {  // 8 loads in flight per thread
        const int groups = min(8, (count - base + kThreads - 1) / kThreads);
        double v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int t = base + u * kThreads + (int)threadIdx.x;
            v[u] = (u < groups && t < count) ? part[t] : 0.0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            if (u < groups) acc += v[u];
    }
    // the warp's butterfly: step o adds nothing to lane 0 when lanes o .. 31 of
    // the warp hold no element (live <= o), so it is skipped
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int live = count - warp * 32;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double b = __shfl_xor_sync(0xffffffffu, acc, o);
        if (o < live) acc += b;
    }
    __syncthreads();
    if (lane == 0) s_red[warp] = acc;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x == 0) {
#pragma unroll
        for (int w = 0; w < kWarps; ++w)
            if (w * 32 < count) t += s_red[w];
    }
    return t;
}

// ---------------------------------------------------------------------------
// The persistent decoder.
//
// The grid is split into `groups` independent groups (by default one CTA of
// each group per SM).  A group owns slots_per_group slots and advances its
// frames in lock-step between its own barriers; frames that stop are replaced
// from one queue shared by all groups.  While one group waits at a barrier,
// the other groups' CTAs on the same SMs keep computing, and only the few
// frames in flight have to stay in L2.
// ---------------------------------------------------------------------------
template <typename T, class Code, bool W>
__global__ void __launch_bounds__(kThreads, 4) bp_decode_kernel(Params<T> p, CodeSet<Code> cs) {
    const int SG = p.slots_per_group;
    // the carve below takes kSmemPerSlot bytes per slot (decode_smem_bytes)
    extern __shared__ double smem_dyn[];
    double* st_qprev = smem_dyn;                  // [SG]
    int* st_frame = (int*)(st_qprev + SG);        // [SG]
    int* st_k = st_frame + SG;                    // [SG]
    int* st_code = st_k + SG;                     // [SG]
    int* listA = st_code + SG;                    // [SG]
    int* listB = listA + SG;                      // [SG]
    __shared__ double s_red[kWarps];
    __shared__ int s_nA, s_nB;

    const int gsize = gridDim.x / p.groups;
    const int g = blockIdx.x / gsize;
    if (g >= p.groups) return;
    const int lb = blockIdx.x - g * gsize;        // CTA index within the group
    const int s0 = g * SG;                        // first (global) slot of the group
    Ctrl* bar = p.ctrl + g;
    int* err = &p.ctrl->err;

    for (int l = threadIdx.x; l < SG; l += kThreads) {
        const int f = s0 + l < p.frames ? s0 + l : -1;
        st_frame[l] = f;
        st_code[l] = (f >= 0 && p.frame_code) ? p.frame_code[f] : 0;
        st_k[l] = 0;
        st_qprev[l] = 0.0;
    }
    __syncthreads();
    if (ld_volatile(err) != kErrNone) return;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned lt_mask = (1u << lane) - 1u;

    for (int step = 0;; ++step) {
        const int par = step & 1;
        // ---- running slots ------------------------------------------------
        if (warp == 0) {
            int cnt = 0;
            for (int base = 0; base < SG; base += 32) {
                const int l = base + lane;
                const bool occ = l < SG && st_frame[l] >= 0;
                const unsigned m = __ballot_sync(0xffffffffu, occ);
                if (occ) listA[cnt + __popc(m & lt_mask)] = l;
                cnt += __popc(m);
            }
            if (lane == 0) s_nA = cnt;
        }
        __syncthreads();
        const int nA = s_nA;
        if (nA == 0) break;

        // ---- phase A: check nodes + syndrome of the current decision -----
        // (every slot owns cn_tiles_max items; a frame of a smaller code skips the rest)
        const unsigned totalA = (unsigned)nA * (unsigned)p.cn_tiles_max;
        for (unsigned it = lb; it < totalA; it += gsize) {
            const unsigned si = it / (unsigned)p.cn_tiles_max;
            const int l = listA[si];
            const int tile = (int)(it - si * (unsigned)p.cn_tiles_max);
            const CodeInfo<Code>& ci = cs.c[st_code[l]];
            if (tile >= ci.cn_tiles) continue;
            const int s = s0 + l;
            const int k = st_k[l];
            const int mode = k == 0 ? kModeFirst : (k >= p.max_iter ? kModeSynd : kModeFull);
            const bool want_synd = k >= 1 && (p.rule != kRuleNone || k >= p.max_iter);
            FrameCtx<T> fc = frame_ctx(p, ci, s, st_frame[l]);
            if constexpr (W) fc.wrow = weight_row(p, k);
            const bool unsat = cn_tile<W, T>(p, ci.code, fc, mode, want_synd, tile);
            if (want_synd && __any_sync(0xffffffffu, unsat) && lane == 0)
                atomicOr(&p.unsat[par * p.slots + s], 1);
        }
        // q^(k) of every running frame that has done an iteration: the partials
        // are summed in kQParts fixed ranges, each by its own CTA (counted from
        // the end of the group, where CTAs get one item fewer when the items
        // do not divide evenly); the decision adds the kQParts sums in order
        for (int w = gsize - 1 - lb; w >= 0 && w < nA * kQParts; w += gsize) {
            const int l = listA[w / kQParts];
            const int r = w % kQParts;
            const int s = s0 + l;
            const int k = st_k[l];
            if (k < 1) continue;
            const int np = cs.c[st_code[l]].nqb * kWarps;
            const int per = (np + kQParts - 1) / kQParts;
            const int lo = r * per, cnt = max(0, min(np, lo + per) - lo);
            const double* qp = p.qpart + (size_t)s * p.slot_nqb * kWarps;
            const double* q0p = p.q0part + (size_t)s * p.slot_nqb * kWarps;
            const double qv = block_sum_fixed(qp + lo, cnt, s_red);
            const bool with_q0 = k == 1 && p.vnr_first_iter <= 1;
            double q0 = 0.0;
            if (with_q0) q0 = block_sum_fixed(q0p + lo, cnt, s_red);
            if (threadIdx.x == 0) {
                p.qval[(size_t)s * kQParts + r] = qv;
                if (with_q0) p.q0val[(size_t)s * kQParts + r] = q0;
            }
        }
        if (!grid_sync(bar, err, gsize, 2u * step + 1u, p.timeout_ns, step == 0 ? p.bar_extra : 0u)) return;

        // ---- decisions (warp 0 of every CTA of the group, all alike) ------
        if (warp == 0) {
            int cnt = 0;
            for (int base = 0; base < SG; base += 32) {
                const int l = base + lane;
                const int s = s0 + l;
                int act = -1;  // 0 = continue, 1 = stop
                if (l < SG && st_frame[l] >= 0) {
                    const int k = st_k[l];
                    const int f = st_frame[l];
                    if (k == 0) {
                        act = 0;
                    } else {
                        const bool sat = ld_volatile(&p.unsat[par * p.slots + s]) == 0;
                        double qr[kQParts], q0r[kQParts];
                        const bool with_q0 = k == 1 && p.vnr_first_iter <= 1;
#pragma unroll
                        for (int r = 0; r < kQParts; ++r) {
                            qr[r] = ld_volatile(&p.qval[(size_t)s * kQParts + r]);
                            q0r[r] = with_q0 ? ld_volatile(&p.q0val[(size_t)s * kQParts + r]) : 0.0;
                        }
                        double qv = 0.0, q0 = 0.0;
#pragma unroll
                        for (int r = 0; r < kQParts; ++r) qv += qr[r];
                        if (with_q0) {
#pragma unroll
                            for (int r = 0; r < kQParts; ++r) q0 += q0r[r];
                        }
                        if (lb == 0 && k <= p.trace_iters && p.trace_q)
                            p.trace_q[(long long)(k - 1) * p.frames + f] = qv;
                        const double qprev = with_q0 ? q0 : st_qprev[l];
                        const bool succ = p.rule != kRuleNone && sat;
                        const bool abort_ = !succ && p.rule == kRulePceVnr && k >= p.vnr_first_iter && qv < qprev;
                        const bool end = k >= p.max_iter;
                        if (succ || abort_ || end) {
                            act = 1;
                            if (lb == 0) {
                                p.flags_out[f] = (unsigned char)((sat ? 1 : 0) | (abort_ ? 2 : 0));
                                p.iters_out[f] = k;
                                atomicAdd(&p.ctrl->frame_iters, (unsigned long long)k);
                                const int nf = atomicAdd(&p.ctrl->next_frame, 1);
                                p.new_frame[s] = nf < p.frames ? nf : -1;
                            }
                        } else {
                            act = 0;
                            st_qprev[l] = qv;
                        }
                    }
                }
                const unsigned mAny = __ballot_sync(0xffffffffu, act >= 0);
                if (act >= 0) listB[cnt + __popc(mAny & lt_mask)] = l | (act << 16);
                cnt += __popc(mAny);
            }
            if (lane == 0) s_nB = cnt;
        }
        __syncthreads();
        const int nB = s_nB;

        // ---- phase B: variable nodes / write-out of stopped frames -------
        const unsigned totalB = (unsigned)nB * (unsigned)p.vn_tiles_max;
        for (unsigned it = lb; it < totalB; it += gsize) {
            // phase B walks the slots in the reverse order of phase A, so it starts
            // on the frames whose messages phase A wrote last (still in L2)
            const unsigned si = it / (unsigned)p.vn_tiles_max;
            const int e = listB[nB - 1 - (int)si];
            const int l = e & 0xffff;
            const int tile = (int)(it - si * (unsigned)p.vn_tiles_max);
            const CodeInfo<Code>& ci = cs.c[st_code[l]];
            if (tile >= ci.vn_tiles) continue;
            const FrameCtx<T> fc = frame_ctx(p, ci, s0 + l, st_frame[l]);
            if ((e >> 16) == 0)
                vn_tile<T>(p, ci.code, fc, st_k[l], tile);
            else
                final_tile<T>(ci.code, fc, tile);
        }
        if (lb == 0)
            for (int l = threadIdx.x; l < SG; l += kThreads) p.unsat[(par ^ 1) * p.slots + s0 + l] = 0;
        if (!grid_sync(bar, err, gsize, 2u * step + 2u, p.timeout_ns)) return;
        // new state: continuing frames did one more iteration; stopped ones are
        // replaced by the frame the group's first CTA took from the queue
        for (int i = threadIdx.x; i < nB; i += kThreads) {
            const int e = listB[i];
            const int l = e & 0xffff;
            if ((e >> 16) == 0) {
                st_k[l] += 1;
            } else {
                const int nf = ld_volatile(&p.new_frame[s0 + l]);
                st_frame[l] = nf;
                st_code[l] = (nf >= 0 && p.frame_code) ? p.frame_code[nf] : 0;
                st_k[l] = 0;
                st_qprev[l] = 0.0;
            }
        }
        __syncthreads();
    }
}

// Where each frame's syndrome bytes are and where its packed words go.
struct PackInfo {
    int m[kMaxCodes];              // checks per frame of each code
    int swords[kMaxCodes];
    const int* frame_code;         // [frames], NULL = all code 0
    const long long* syn_off;      // [frames] byte offset, NULL = f * m
    const long long* sb_off;       // [frames] word offset, NULL = f * swords
};

// Pack the syndrome bytes into bits, 32 checks per word, one warp per word:
// blockIdx.y walks the frames, blockIdx.x the frame's words; any byte other
// than 0/1 raises kErrSyndrome (the decode kernel then returns at once).
__global__ void pack_syndrome_kernel(const unsigned char* __restrict__ syn, int frames, PackInfo pi,
                                     unsigned* __restrict__ out, Ctrl* ctrl) {
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    const int warp = (int)blockIdx.x * nw + (threadIdx.x >> 5), wstride = (int)gridDim.x * nw;
    for (int f = blockIdx.y; f < frames; f += gridDim.y) {
        const int c = pi.frame_code ? pi.frame_code[f] : 0;
        const int m = pi.m[c], swords = pi.swords[c];
        const unsigned char* s = syn + (pi.syn_off ? pi.syn_off[f] : (long long)f * m);
        unsigned* o = out + (pi.sb_off ? pi.sb_off[f] : (long long)f * swords);
        bool bad = false;
        for (int w = warp; w < swords; w += wstride) {
            const int i = w * 32 + lane;
            const unsigned char b = i < m ? s[i] : (unsigned char)0;
            const unsigned bits = __ballot_sync(0xffffffffu, (b & 1u) != 0u);
            bad |= __any_sync(0xffffffffu, b > 1u);
            if (lane == 0) o[w] = bits;
        }
        if (bad && lane == 0) atomicCAS(&ctrl->err, kErrNone, kErrSyndrome);
    }
}

// Start-of-decode control words: every group's barrier cleared, the error word
// and totals zeroed, the queue of waiting frames starting at `next_frame`.
// (A kernel rather than a host copy, so a whole decode can be captured in a
// CUDA graph.)
__global__ void init_ctrl_kernel(Ctrl* ctrl, int groups, int next_frame, int* unsat, int unsat_words) {
    for (int i = threadIdx.x; i < groups; i += blockDim.x) {
        ctrl[i].bar_count = 0u;
        ctrl[i].bar_gen = 0u;
        ctrl[i].err = kErrNone;
        ctrl[i].next_frame = i == 0 ? next_frame : 0;
        ctrl[i].frame_iters = 0ull;
    }
    for (int i = threadIdx.x; i < unsat_words; i += blockDim.x) unsat[i] = 0;
}

// The decode's outcome as an ldpc_status code (0 ok, 1 bad syndrome byte, 5 timeout,
// 7 an index check of the index-checking build failed).
__global__ void status_kernel(const Ctrl* ctrl, int* out) {
    const int e = ctrl->err;
    *out = e == kErrNone ? 0 : (e == kErrSyndrome ? 1 : (e == kErrTimeout ? 5 : (e == kErrBounds ? 7 : 4)));
}

}  // namespace ldpcgb
