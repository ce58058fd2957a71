// Dataflow schedule of the persistent QC decoder (no grid barriers).
//
// The work of a decode is one endless list of items, cut into "pairs".  Pair t
// holds the variable-node items of slot-step t - lag followed by the check-
// node items of slot-step t, where slot-step u = c * slots + s is cycle c of
// slot s (one decoding iteration of the frame in that slot).  CTA b takes the
// items b, b + grid, b + 2 grid, ... in order.  An item starts once the items
// of the other pass that it reads are done:
//   check item  (slot s, cycle c, base row i, checks t0..t1) reads APP^(c-1)
//               at columns j of row i, i.e. variable items of cycle c - 1;
//   variable item (slot s, cycle c, base column j, variables u0..u1) reads the
//               new check messages of the rows meeting j, i.e. check items of
//               cycle c, and needs the decision taken after cycle c's checks.
// Every item flags its completion with 1 + its cycle.  Every dependency lies
// earlier in the list, and a cooperative launch keeps every CTA resident, so
// the earliest unfinished item can always run: the schedule cannot deadlock.
// The same dependencies order every overwrite after the reads of the old
// value (a variable item rewrites the APP values that exactly the check items
// it waits for read; a check item rewrites the messages that exactly the
// variable items it waits for read).  With lag 2 a frame's new messages are
// read back about two pairs (~60 MB of traffic) after they were written, so
// they are still in L2.
//
// The last check item of a slot's cycle to finish (an acq_rel counter) takes
// the frame's decision (PCE-ET, VNR-ET, D_max) with the same q as the
// lock-step kernel, bit for bit: the eight fixed ranges of per-warp partials
// are summed in block_sum_fixed's order, one range per warp.  A stopped frame
// hands its slot to the next queued frame; the variable items of the stop
// cycle write its decision out.  Waits spin with a time limit and turn an
// expired wait into the error word.
#pragma once

#include <climits>

#include "bp_kernels.cuh"

namespace ldpcgb {

// Per code: the items of the other pass each item waits for (CSR lists).
struct FlowDeps {
    const int* cn_ptr;   // [cn_tiles + 1]
    const int* cn_dep;   // variable items (previous cycle) read by each check item
    const int* vn_ptr;   // [vn_tiles + 1]
    const int* vn_dep;   // check items (same cycle) read by each variable item
};

struct FlowParams {
    int lag;                      // 1 .. slots
    int cn_items, vn_items;       // items per slot-step of each pass (largest code)
    int* cn_flag;                 // [slots][cn_items] 1 + cycle of the item's last completion
    int* vn_flag;                 // [slots][vn_items]
    unsigned* cn_count;           // [slots][2] check items of cycle c (by parity) done
    int* unsat;                   // [slots][2] any unsatisfied check in cycle c
    int* dec;                     // [slots] last cycle whose decision is published
    unsigned long long* rec;      // [slots] frame (low 32 bits, -1 none) and its start cycle (high)
    int* prev;                    // [slots] the slot's previous frame (-1 none)
    double* qprev;                // [slots] q of the previous iteration
    int* retired;                 // slots left without a frame
    unsigned* progress;           // decisions taken so far (watchdog of CTAs that only skip)
    FlowDeps dep[kMaxCodes];
};

__device__ __forceinline__ int ld_acquire_s32(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_s32(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned* p, unsigned v) {
    unsigned old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}

__host__ __device__ __forceinline__ unsigned long long flow_rec(int frame, int start) {
    return ((unsigned long long)(unsigned)start << 32) | (unsigned long long)(unsigned)frame;
}
__device__ __forceinline__ int rec_frame(unsigned long long r) { return (int)(unsigned)(r & 0xffffffffull); }
__device__ __forceinline__ int rec_start(unsigned long long r) { return (int)(unsigned)(r >> 32); }

// Bounded spinning shared by the waits: cheap spins first, then sleeps with a
// wall-clock limit; false once the decode must stop (error set here or elsewhere).
struct Spin {
    unsigned n = 0;
    unsigned long long t0 = 0;
    __device__ __forceinline__ bool again(int* err, unsigned long long timeout_ns) {
        if (++n <= 16) return true;
        if (t0 == 0) t0 = global_ns();
        __nanosleep(100);
        if (ld_volatile(err) != kErrNone) return false;
        if (global_ns() - t0 > timeout_ns) {
            atomicCAS(err, kErrNone, kErrTimeout);
            return false;
        }
        return true;
    }
};

// Warp-wide wait (all 32 lanes of one warp call it) until flag[idx[i]] >= want
// for every i < n (idx NULL: flag[i] for i < n).  Lanes check disjoint entries
// with acquire loads; false on error or timeout.
__device__ __forceinline__ bool warp_wait_flags(const int* flag, const int* idx, int n, int want, int* err,
                                                unsigned long long timeout_ns, Ctrl* ctrl = nullptr, int len = 0) {
    const int lane = threadIdx.x & 31;
    Spin sp;
    (void)ctrl;
    (void)len;
    for (;;) {
        bool ok = true;
        for (int i = lane; i < n; i += 32) {
            int f = idx ? __ldg(idx + i) : i;
#ifdef LDPC_BOUNDS_CHECK
            if (ctrl) f = (int)LDPC_IX(ctrl, f, len, kIxFlowFlag);
#endif
            ok &= ld_acquire_s32(flag + f) >= want;
        }
        if (__all_sync(0xffffffffu, ok)) return true;
        const bool go = sp.again(err, timeout_ns);
        if (__any_sync(0xffffffffu, !go)) return false;
    }
}

// One warp computes block_sum_fixed(part, count) bit for bit: lane l plays
// the threads w * 32 + l (w = 0 .. kWarps - 1) of that 256-thread sum, each
// accumulating its elements in the same order, then each emulated warp's
// butterfly, then the sum over the emulated warps in order.  Additions whose
// other operand is known to be +0.0 are skipped (they change nothing in a sum
// of non-negative terms, and FP64 instructions are scarce on this part, about
// two per clock per SM): element groups past `count`, emulated warps that hold
// no element, and butterfly steps o whose partner lanes o .. 31 hold none.  The
// skipped steps leave some lanes' partial sums unfinished, never lane 0's:
// the result is valid in lane 0, the only reader.
__device__ __forceinline__ double warp_block_sum_fixed(const double* part, int count) {
    const int lane = threadIdx.x & 31;
    double tot = 0.0;
#pragma unroll
    for (int w = 0; w < kWarps; ++w) {
        const int live = count - w * 32;  // elements of the emulated warp's first group
        if (live <= 0) break;             // this and later emulated warps hold only zeros
        double a = lane < live ? part[w * 32 + lane] : 0.0;  // 0.0 + x == x
        for (int base = 0; base < count; base += 8 * kThreads) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int t0 = base + u * kThreads + w * 32;
                if (base + u == 0) continue;  // the first group is loaded above
                if (t0 >= count) break;       // uniform: later groups of this pass are past the end
                const int t = t0 + lane;
                a += t < count ? part[t] : 0.0;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double b = __shfl_xor_sync(0xffffffffu, a, o);
            if (o < live) a += b;  // lanes o .. 31 of this emulated warp hold elements
        }
        tot = w == 0 ? a : tot + a;  // 0.0 + a == a
    }
    return tot;  // valid in lane 0
}

// Shared-memory state of one CTA's current item (written by warp 0).
struct FlowItem {
    int kind;      // 0 skip, 1 check item, 2 variable item, 3 write-out of a stopped frame
    int s, c, tile, frame, k, code, prev_code;
    int fail;      // a wait gave up: leave the kernel
};

// Decision of slot it.s after the check items of cycle it.c, taken by the CTA
// that finished the last of them (every thread of it calls this).  Same rule
// and the same q, bit for bit, as the lock-step kernel's decision block.
// Returns false if a wait gave up.
template <typename T>
__device__ bool flow_decide(const Params<T>& p, const CodeSet<QcDev>& cs, const FlowParams& fp, const FlowItem& it,
                            int* err, double* s_q, double* s_q0, int* s_ok) {
    const int s = it.s, c = it.c, k = it.k, f = it.frame;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // every variable item of cycle c - 1 is done: its q partials are final, and
    // nothing reads the slot record that this decision may replace
    if (warp == 0) {
        bool ok = true;
        const int code_prev = k >= 1 ? it.code : it.prev_code;
        if (c >= 1 && code_prev >= 0)
            ok = warp_wait_flags(fp.vn_flag + (size_t)s * fp.vn_items, nullptr, cs.c[code_prev].vn_tiles, c, err,
                                 p.timeout_ns);
        if (lane == 0) *s_ok = ok ? 1 : 0;
    }
    __syncthreads();
    if (!*s_ok) return false;
    const bool with_q0 = k == 1 && p.vnr_first_iter <= 1;
    if (k >= 1) {
        static_assert(kQParts == kWarps, "one q range per warp");
        const int np = cs.c[it.code].nqb * kWarps;
        const int per = (np + kQParts - 1) / kQParts;
        const int lo = warp * per, cnt = max(0, min(np, lo + per) - lo);
        const size_t base = (size_t)s * p.slot_nqb * kWarps + lo;
        const double qv = warp_block_sum_fixed(p.qpart + base, cnt);
        const double q0 = with_q0 ? warp_block_sum_fixed(p.q0part + base, cnt) : 0.0;
        if (lane == 0) {
            s_q[warp] = qv;
            s_q0[warp] = q0;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        bool stop = false, sat = false, abort_ = false;
        double qv = 0.0;
        if (k >= 1) {
            sat = ld_volatile(&fp.unsat[2 * s + (c & 1)]) == 0;
            double q0 = 0.0;
#pragma unroll
            for (int r = 0; r < kQParts; ++r) {
                qv += s_q[r];
                q0 += s_q0[r];
            }
            if (k <= p.trace_iters && p.trace_q) p.trace_q[(long long)(k - 1) * p.frames + f] = qv;
            const double qprev = with_q0 ? q0 : fp.qprev[s];
            const bool succ = p.rule != kRuleNone && sat;
            abort_ = !succ && p.rule == kRulePceVnr && k >= p.vnr_first_iter && qv < qprev;
            stop = succ || abort_ || k >= p.max_iter;
        }
        // the counters of this parity start again at zero for cycle c + 2
        fp.cn_count[2 * s + (c & 1)] = 0u;
        fp.unsat[2 * s + (c & 1)] = 0;
        if (stop) {
            p.flags_out[f] = (unsigned char)((sat ? 1 : 0) | (abort_ ? 2 : 0));
            p.iters_out[f] = k;
            atomicAdd(&p.ctrl->frame_iters, (unsigned long long)k);
            const int nf = atomicAdd(&p.ctrl->next_frame, 1);
            const int next = nf < p.frames ? nf : -1;
            fp.prev[s] = f;
            fp.qprev[s] = 0.0;
            st_relaxed_u64(&fp.rec[s], flow_rec(next, c + 1));
            if (next < 0) {
                __threadfence();  // the record before the count that announces it
                atomicAdd(fp.retired, 1);
            }
        } else if (k >= 1) {
            fp.qprev[s] = qv;
        }
        st_release_s32(&fp.dec[s], c);
        atomicAdd(fp.progress, 1u);
    }
    return true;
}

// What the next item of this CTA is, with its waits done (warp 0 only; the
// result is broadcast through shared memory).
template <typename T>
__device__ FlowItem flow_next_item(const Params<T>& p, const CodeSet<QcDev>& cs, const FlowParams& fp, long long t,
                                   int r, bool hook, int* err, unsigned* gone) {
    const int lane = threadIdx.x & 31;
    FlowItem m{};
    const bool vn = r < fp.vn_items;
    const long long u = vn ? t - fp.lag : t;  // slot-step of the item
    if (u < 0) return m;
    const int S = p.slots;
    m.s = (int)(u % S);
    m.c = (int)(u / S);
    m.tile = vn ? r : r - fp.vn_items;
    if ((gone[m.s >> 5] >> (m.s & 31)) & 1u) return m;  // this CTA already saw the slot without frames
    // slot state: valid once the decision of cycle c (variable item) or c - 1
    // (check item) is published, or final once the slot has no frame left
    const int need = vn ? m.c : m.c - 1;
    int state = 0;  // 1 valid, 2 empty, 3 gave up
    unsigned long long rv = 0;
    if (lane == 0) {
        Spin sp;
        for (;;) {
            const int d = ld_acquire_s32(fp.dec + m.s);
            rv = ld_acquire_u64(fp.rec + m.s);
            if (!hook && d >= need) { state = 1; break; }
            if (!hook && rec_frame(rv) < 0 && rec_start(rv) <= m.c) { state = 2; break; }
            if (!sp.again(err, p.timeout_ns)) { state = 3; break; }
        }
    }
    state = __shfl_sync(0xffffffffu, state, 0);
    rv = __shfl_sync(0xffffffffu, rv, 0);
    if (state == 3) {
        m.fail = 1;
        return m;
    }
    if (state == 2) {  // no frame left for the slot: for good
        if (lane == 0) gone[m.s >> 5] |= 1u << (m.s & 31);
        return m;
    }
    const int f = rec_frame(rv), start = rec_start(rv);
    auto code_of = [&](int frame) { return p.frame_code ? __ldg(p.frame_code + frame) : 0; };
    bool ok = true;
    if (!vn) {
        // a record that starts after cycle c belongs to a later frame: the frame of
        // cycle c was decided without this item, so the item lay past its code's
        // check items (a batch of codes) and has nothing to do
        if (f < 0 || start > m.c) return m;
        m.frame = f;
        m.k = m.c - start;
        m.code = code_of(f);
        if (m.tile >= cs.c[m.code].cn_tiles) return m;
        const int pv = ld_volatile(fp.prev + m.s);
        m.prev_code = (m.k == 0 && m.c >= 1 && pv >= 0) ? code_of(pv) : -1;
        const int* flags = fp.vn_flag + (size_t)m.s * fp.vn_items;
        if (m.k == 0) {
            // a new frame: the previous frame's variable items (its write-out) must be done,
            // whatever the two codes' item geometries
            if (m.prev_code >= 0) ok = warp_wait_flags(flags, nullptr, cs.c[m.prev_code].vn_tiles, m.c, err,
                                                        p.timeout_ns, p.ctrl, fp.vn_items);
        } else {
            const FlowDeps& dp = fp.dep[m.code];
            const int a = __ldg(dp.cn_ptr + m.tile), b = __ldg(dp.cn_ptr + m.tile + 1);
            ok = warp_wait_flags(flags, dp.cn_dep + a, b - a, m.c, err, p.timeout_ns, p.ctrl, fp.vn_items);
        }
        m.kind = 1;
    } else if (f >= 0 && start <= m.c) {
        m.frame = f;
        m.k = m.c - start;
        m.code = code_of(f);
        if (m.tile >= cs.c[m.code].vn_tiles) return m;
        const FlowDeps& dp = fp.dep[m.code];
        const int a = __ldg(dp.vn_ptr + m.tile), b = __ldg(dp.vn_ptr + m.tile + 1);
        ok = warp_wait_flags(fp.cn_flag + (size_t)m.s * fp.cn_items, dp.vn_dep + a, b - a, m.c + 1, err,
                             p.timeout_ns, p.ctrl, fp.cn_items);
        m.kind = 2;
    } else if (start == m.c + 1) {
        // the frame stopped at cycle c: write its decision out
        const int pv = ld_volatile(fp.prev + m.s);
        m.frame = pv;
        m.code = code_of(pv);
        if (m.tile >= cs.c[m.code].vn_tiles) return m;
        m.kind = 3;
    }
    if (!ok) m.fail = 1;
    return m;
}

template <typename T, bool W>
__global__ void __launch_bounds__(kThreads, 4) bp_flow_kernel(Params<T> p, CodeSet<QcDev> cs, FlowParams fp) {
    __shared__ FlowItem s_it;
    __shared__ double s_q[kWarps], s_q0[kWarps];
    __shared__ int s_dec, s_ok, s_all_retired;
    __shared__ long long s_t_end;
    __shared__ unsigned s_gone[kMaxSlots / 32];  // slots this CTA has seen without frames (for good)
    __shared__ int s_stop;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int* err = &p.ctrl->err;
    const long long I = (long long)fp.cn_items + fp.vn_items;
    if (threadIdx.x == 0) {
        s_t_end = LLONG_MAX;
        s_stop = 0;
    }
    for (int i = threadIdx.x; i < kMaxSlots / 32; i += kThreads) s_gone[i] = 0u;
    __syncthreads();
    // watchdog: a CTA whose items all fall on slots without frames only skips; it
    // gives up (error word) only if no decision is taken anywhere for timeout_ns
    unsigned skips = 0, seen_progress = 0;
    unsigned long long skip_t0 = 0;
    bool hook = p.bar_extra != 0 && blockIdx.x == 0;  // test hook: CTA 0's first slot wait never ends
    const volatile FlowItem* vit = &s_it;  // re-read after an item's work rather than held in registers
    unsigned n_items = 0;
    for (long long it = blockIdx.x;; it += gridDim.x, ++n_items) {
        const long long t = it / I;
        if (t > s_t_end) break;
        const int r = (int)(it - t * I);
        if (warp == 0) {
            const FlowItem m = flow_next_item(p, cs, fp, t, r, hook && r >= fp.vn_items && t >= 0, err, s_gone);
            if (lane == 0) s_it = m;
        }
        __syncthreads();
        const int kind = vit->kind;
        if (vit->fail) return;
        if (kind == 1) hook = false;
        if (kind == 0) {
            if (++skips > 2u * (unsigned)p.slots) __nanosleep(200);  // a long run of slots without frames
            if ((skips & 255u) == 0u) {
                if (threadIdx.x == 0) {
                    const unsigned pr = ld_volatile((const int*)fp.progress);
                    const unsigned long long now = global_ns();
                    if (skip_t0 == 0 || pr != seen_progress) {
                        skip_t0 = now;
                        seen_progress = pr;
                    } else if (now - skip_t0 > p.timeout_ns) {
                        atomicCAS(err, kErrNone, kErrTimeout);
                    }
                    s_stop = ld_volatile(err) != kErrNone;
                }
                __syncthreads();
                if (s_stop) return;
            }
        } else {
            skips = 0;
            skip_t0 = 0;
        }
        if (kind != 0) {
            const CodeInfo<QcDev>& ci = cs.c[vit->code];
            const int k = vit->k, tile = vit->tile;
            FrameCtx<T> fc = frame_ctx(p, ci, vit->s, vit->frame);
            if (kind == 1) {
                if constexpr (W) fc.wrow = weight_row(p, k);
                const int mode = k == 0 ? kModeFirst : (k >= p.max_iter ? kModeSynd : kModeFull);
                const bool want_synd = k >= 1 && (p.rule != kRuleNone || k >= p.max_iter);
                const bool unsat = cn_tile<W, T>(p, ci.code, fc, mode, want_synd, tile);
                if (want_synd && __any_sync(0xffffffffu, unsat) && lane == 0)
                    atomicOr(&fp.unsat[2 * vit->s + (vit->c & 1)], 1);
                __syncthreads();
                if (threadIdx.x == 0) {
                    const int sl = vit->s, cy = vit->c;
                    st_release_s32(fp.cn_flag + (size_t)sl * fp.cn_items +
                                       LDPC_IX(p.ctrl, vit->tile, fp.cn_items, kIxFlowFlag), cy + 1);
                    const unsigned old = atom_add_acq_rel(&fp.cn_count[2 * sl + (cy & 1)], 1u);
                    s_dec = old + 1u == (unsigned)cs.c[vit->code].cn_tiles;
                }
                __syncthreads();
                if (s_dec) {
                    const FlowItem m = s_it;
                    if (!flow_decide<T>(p, cs, fp, m, err, s_q, s_q0, &s_ok)) return;
                }
            } else {
                if (kind == 2)
                    vn_tile<T>(p, ci.code, fc, k, tile);
                else
                    final_tile<T>(ci.code, fc, tile);
                __syncthreads();
                if (threadIdx.x == 0)
                    st_release_s32(fp.vn_flag + (size_t)vit->s * fp.vn_items +
                                       LDPC_IX(p.ctrl, vit->tile, fp.vn_items, kIxFlowFlag), vit->c + 1);
            }
        }
        // every few items: once no slot has a frame left, find the last pair that
        // still holds work (the write-out of each slot's last frame)
        if ((n_items & 3) == 3 && s_t_end == LLONG_MAX) {
            if (threadIdx.x == 0) s_all_retired = ld_acquire_s32(fp.retired) >= p.slots;
            __syncthreads();
            if (s_all_retired) {
                long long te = -1;
                for (int q = threadIdx.x; q < p.slots; q += kThreads) {
                    const int st = rec_start(ld_acquire_u64(fp.rec + q));
                    if (st >= 1) te = max(te, (long long)(st - 1) * p.slots + q + fp.lag);
                }
                for (int o = 16; o > 0; o >>= 1) te = max(te, __shfl_xor_sync(0xffffffffu, te, o));
                if (lane == 0) s_q[warp] = (double)te;  // reuse: item counts are exact in double
                __syncthreads();
                if (threadIdx.x == 0) {
                    long long m2 = -1;
                    for (int w = 0; w < kWarps; ++w) m2 = max(m2, (long long)s_q[w]);
                    s_t_end = m2;
                }
            }
        }
        __syncthreads();
    }
}

// Start-of-decode state of the dataflow schedule: the first `slots` frames in
// the slots (cycle 0), every completion word and counter at zero, the queue of
// waiting frames after them, no decision published.
__global__ void flow_init_kernel(FlowParams fp, int slots, int frames, Ctrl* ctrl) {
    const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = gridDim.x * blockDim.x;
    for (long long i = tid; i < (long long)slots * fp.cn_items; i += nth) fp.cn_flag[i] = 0;
    for (long long i = tid; i < (long long)slots * fp.vn_items; i += nth) fp.vn_flag[i] = 0;
    for (int s = tid; s < slots; s += nth) {
        fp.rec[s] = flow_rec(s < frames ? s : -1, 0);
        fp.dec[s] = -1;
        fp.prev[s] = -1;
        fp.qprev[s] = 0.0;
        fp.cn_count[2 * s] = fp.cn_count[2 * s + 1] = 0u;
        fp.unsat[2 * s] = fp.unsat[2 * s + 1] = 0;
    }
    if (tid == 0) {
        *fp.retired = slots - min(slots, frames);
        *fp.progress = 0u;
        ctrl->bar_count = 0u;
        ctrl->bar_gen = 0u;
        ctrl->err = kErrNone;
        ctrl->next_frame = min(slots, frames);
        ctrl->frame_iters = 0ull;
    }
}

}  // namespace ldpcgb
