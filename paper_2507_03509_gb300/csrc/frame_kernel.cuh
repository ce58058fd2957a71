// Frame-per-CTA schedule of the decoder for small CSR codes (whole frame and
// the code's index lists in shared memory).
//
// When a frame's messages, APP values and channel LLRs, and the code's edge
// lists as 16-bit indices, fit one CTA's shared memory (about 8E + 12n + 4m
// bytes; the n = 4096 workload code needs 155 KB), a CTA of kFrameThreads
// threads decodes whole frames on its own, taking them from the shared queue.
// It runs the lock-step kernel's steps (check pass with the fused syndrome
// test, q^(k), decision, variable pass), separated by CTA barriers instead of
// grid barriers, and touches global memory inside an iteration only for
// learned weights and traces.
//
// Bit-identity with the lock-step kernel: every check and variable does the
// same arithmetic; the variable pass runs as kFrameThreads / kThreads virtual
// 256-thread CTAs, so each per-warp q partial (tile * kWarps + warp) sums the
// same variables in the same order; the eight fixed q ranges are summed by
// one warp each with the 256-thread CTA's tree (warp_block_sum_fixed).
//
// FP64 work is scarce on this part (about two FP64 operations per clock per
// SM), so only the eight range warps sum q and only warp 0 takes the decision;
// the other warps wait at the CTA barrier.
//
// Frame per cluster (NC = 2): when there are fewer frames than SMs, a
// thread-block cluster of two CTAs on two SMs decodes each frame.  Both CTAs
// hold the whole frame; CTA r runs the runs of 32 checks of the degree-sorted
// order with index mod 2 = r and the variables of the 1024-variable blocks b
// with b mod 2 = r.  A
// new message whose variable lies in the other CTA's blocks, and every APP
// value, is also stored into the other CTA's copy through distributed shared
// memory (st.shared::cluster: stores only, so no pass waits on a remote load),
// and cluster barriers separate the passes.  Both CTAs then read identical
// copies, so they compute the same q^(k) (its per-warp partials are formed
// from the shared APP copy, in the variable pass's order) and take the same
// decisions in lock-step; CTA 0 alone writes the frame's outputs.
#pragma once

#include "bp_kernels.cuh"
#include "flow_kernel.cuh"

namespace ldpcgb {

constexpr int kFrameThreads = 1024;
constexpr int kFrameVirt = kFrameThreads / kThreads;  // virtual 256-thread CTAs per frame CTA
// frame per cluster: variable v belongs to CTA (v >> kPairShift) & 1, one variable per thread
constexpr int kPairShift = 10;
static_assert(kVnTile == (1 << kPairShift) && kFrameThreads == (1 << kPairShift), "pair blocks are q tiles");

// ---- thread-block cluster primitives (inline PTX, sm_90 and later) ----
__device__ __forceinline__ unsigned cluster_ctarank() {
    unsigned r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// address, in the cluster's shared window, of this CTA's shared variable p in CTA `rank`
__device__ __forceinline__ unsigned dsmem_addr(const void* p, unsigned rank) {
    const unsigned a = (unsigned)__cvta_generic_to_shared(p);
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
__device__ __forceinline__ void dsmem_st_f32(unsigned addr, float v) {
    asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(addr), "f"(v) : "memory");
}
__device__ __forceinline__ void dsmem_st_s32(unsigned addr, int v) {
    asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}
// returns the word's previous value
__device__ __forceinline__ unsigned dsmem_or_b32(unsigned addr, unsigned v) {
    unsigned old;
    asm volatile("atom.shared::cluster.or.b32 %0, [%1], %2;" : "=r"(old) : "r"(addr), "r"(v) : "memory");
    return old;
}
// All threads of every CTA of the cluster: the cluster's shared-memory writes
// before it are visible to every thread's reads after it.
__device__ __forceinline__ void cluster_barrier() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__host__ __device__ constexpr long long frame_round(long long x, long long a) { return (x + a - 1) / a * a; }

// Byte offsets of the pieces of csr_frame_kernel's shared memory (16-byte aligned).
struct FrameSmem {
    long long part, part0, c2v, app, lch, sbits, col, vedge, rptr, rord, vptr, total;
};

__host__ __device__ constexpr FrameSmem frame_smem_layout(long long E, int n, int m, int nqb, int swords) {
    FrameSmem s{};
    long long o = 0;
    s.part = o;  o += frame_round((long long)nqb * kWarps * 8, 16);
    s.part0 = o; o += frame_round((long long)nqb * kWarps * 8, 16);
    s.c2v = o;   o += frame_round(E * 4, 16);
    s.app = o;   o += frame_round((long long)n * 4, 16);
    s.lch = o;   o += frame_round((long long)n * 4, 16);
    s.sbits = o; o += frame_round((long long)swords * 4, 16);
    s.col = o;   o += frame_round(E * 2, 16);
    s.vedge = o; o += frame_round(E * 2, 16);
    s.rptr = o;  o += frame_round((long long)(m + 1) * 2, 16);
    s.rord = o;  o += frame_round((long long)m * 2, 16);
    s.vptr = o;  o += frame_round((long long)(n + 1) * 2, 16);
    s.total = o;
    return s;
}

// Shared memory of csr_frame_kernel, or 0 if the code's indices do not fit 16 bits.
__host__ __device__ constexpr size_t frame_smem_bytes(long long E, int n, int m, int nqb, int swords) {
    return (E > 65535 || n > 65535 || m > 65535) ? 0 : (size_t)frame_smem_layout(E, n, m, nqb, swords).total;
}

// One check of degree D (compile time) from shared memory: the arithmetic of csr_cn_check.
// NC = 2: a message whose variable belongs to the other CTA of the pair is
// also stored into that CTA's copy (peer_c2v: its c2v array in the cluster window).
template <int D, bool W, int NC>
__device__ __forceinline__ bool smem_cn_check(const Params<float>& p, const FrameCtx<float>& fc, int mode,
                                              bool want_synd, unsigned sbit, int e0, const unsigned short* col,
                                              const float* app, const float* lch, float* c2v, unsigned peer_c2v,
                                              unsigned rank) {
    float a[D], o[D];
    int vis[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const int vi = (int)LDPC_IX(p.ctrl, col[e0 + j], fc.n, kIxCsrVar);
        vis[j] = vi;
        o[j] = 0.0f;
        if (mode == kModeFirst) {
            a[j] = lch[vi];
        } else {
            a[j] = app[vi];
            if (mode == kModeFull) o[j] = c2v[e0 + j];
        }
    }
    bool unsat = false;
    if (want_synd) {
        unsigned pr = sbit;
#pragma unroll
        for (int j = 0; j < D; ++j) pr ^= (unsigned)(a[j] < 0.0f);
        unsat = pr != 0u;
    }
    if (mode == kModeSynd) return unsat;
    float v[D], out[D];
#pragma unroll
    for (int j = 0; j < D; ++j) v[j] = clampm(a[j] - o[j], p.lmax);
    cn_core<D>(v, sbit, p.lmax, out);
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const float msg = weighted<W>(p, fc, out[j], e0 + j);
        c2v[e0 + j] = msg;
        if constexpr (NC == 2)
            if ((unsigned)((vis[j] >> kPairShift) & 1) != rank) dsmem_st_f32(peer_c2v + 4u * (unsigned)(e0 + j), msg);
    }
    return unsat;
}

// Any degree (0 and > 6): the arithmetic of csr_cn_check_n.
template <bool W, int NC>
__device__ __noinline__ bool smem_cn_check_n(const Params<float>& p, const FrameCtx<float>& fc, int mode,
                                             bool want_synd, unsigned sbit, int e0, int d,
                                             const unsigned short* col, const float* app, const float* lch,
                                             float* c2v, unsigned peer_c2v, unsigned rank) {
    if (d == 0) return want_synd && sbit != 0u;
    float v[kMaxDeg], out[kMaxDeg];
    unsigned pr = sbit;
    for (int j = 0; j < d; ++j) {
        const int vi = (int)LDPC_IX(p.ctrl, col[e0 + j], fc.n, kIxCsrVar);
        float a, o = 0.0f;
        if (mode == kModeFirst) {
            a = lch[vi];
        } else {
            a = app[vi];
            if (mode == kModeFull) o = c2v[e0 + j];
        }
        pr ^= (unsigned)(a < 0.0f);
        v[j] = clampm(a - o, p.lmax);
    }
    const bool unsat = want_synd && pr != 0u;
    if (mode == kModeSynd) return unsat;
    cn_core_n(v, d, sbit, p.lmax, out);
    for (int j = 0; j < d; ++j) {
        const float msg = weighted<W>(p, fc, out[j], e0 + j);
        c2v[e0 + j] = msg;
        if constexpr (NC == 2) {
            const int vi = (int)LDPC_IX(p.ctrl, col[e0 + j], fc.n, kIxCsrVar);
            if ((unsigned)((vi >> kPairShift) & 1) != rank) dsmem_st_f32(peer_c2v + 4u * (unsigned)(e0 + j), msg);
        }
    }
    return unsat;
}

template <bool W, int NC>
__global__ void __launch_bounds__(kFrameThreads, 1) csr_frame_kernel(Params<float> p, CodeInfo<CsrDev> ci,
                                                                      FrameSmem L) {
    static_assert(NC == 1 || NC == 2, "one CTA or a pair per frame");
    extern __shared__ __align__(16) unsigned char smem_frame[];
    double* part = (double*)(smem_frame + L.part);      // [nqb * kWarps] q partials of APP^(k)
    double* part0 = (double*)(smem_frame + L.part0);    // [nqb * kWarps] the same for q^(0)
    float* c2v = (float*)(smem_frame + L.c2v);          // [E]
    float* app = (float*)(smem_frame + L.app);          // [n]
    float* lch = (float*)(smem_frame + L.lch);          // [n] the frame's channel LLRs
    unsigned* sb = (unsigned*)(smem_frame + L.sbits);   // [swords] the frame's packed syndrome
    unsigned short* col = (unsigned short*)(smem_frame + L.col);      // [E] variable of each edge
    unsigned short* vedge = (unsigned short*)(smem_frame + L.vedge);  // [E] edges of each variable
    unsigned short* rptr = (unsigned short*)(smem_frame + L.rptr);    // [m + 1]
    unsigned short* rord = (unsigned short*)(smem_frame + L.rord);    // [m] checks by degree
    unsigned short* vptr = (unsigned short*)(smem_frame + L.vptr);    // [n + 1]
    __shared__ double s_q[kQParts], s_q0[kQParts];
    __shared__ int s_frame, s_unsat[2], s_stop;
    const int tid = (int)threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const CsrDev& g = ci.code;
    const int n = ci.n, m = ci.m;
    const long long E = ci.E;
    // the pair's other CTA: its copies of c2v, APP, the syndrome flags and the frame number
    const unsigned rank = NC == 2 ? cluster_ctarank() : 0u;
    unsigned peer_c2v = 0, peer_app = 0, peer_unsat = 0, peer_frame = 0;
    if constexpr (NC == 2) {
        peer_c2v = dsmem_addr(c2v, rank ^ 1u);
        peer_app = dsmem_addr(app, rank ^ 1u);
        peer_unsat = dsmem_addr(s_unsat, rank ^ 1u);
        peer_frame = dsmem_addr(&s_frame, rank ^ 1u);
    }
    // the code's index lists, once per CTA (values < 2^16: checked by the launcher)
    for (long long e = tid; e < E; e += kFrameThreads) {
        col[e] = (unsigned short)__ldg(g.col_idx + e);
        vedge[e] = (unsigned short)__ldg(g.var_edge + e);
    }
    for (int i = tid; i <= m; i += kFrameThreads) rptr[i] = (unsigned short)__ldg(g.row_ptr + i);
    for (int i = tid; i < m; i += kFrameThreads) rord[i] = (unsigned short)__ldg(g.row_order + i);
    for (int v = tid; v <= n; v += kFrameThreads) vptr[v] = (unsigned short)__ldg(g.var_ptr + v);
    const int npart = ci.nqb * kWarps;
    const int per = (npart + kQParts - 1) / kQParts;
    const int vt = tid & (kThreads - 1);  // thread of the virtual 256-thread CTA
    // this CTA's checks: runs of 32 in the degree-sorted order, alternating between the CTAs of a pair
    const int c_first = (warp * NC + (int)rank) * 32 + lane, c_step = NC * kFrameThreads;

    for (;;) {
        if (tid == 0 && rank == 0) {
            const int nf = atomicAdd(&p.ctrl->next_frame, 1);
            s_frame = nf;
            if constexpr (NC == 2) dsmem_st_s32(peer_frame, nf);
        }
        if constexpr (NC == 2) cluster_barrier(); else __syncthreads();
        const int f = s_frame;
        if (f >= p.frames) break;
        FrameCtx<float> fc = frame_ctx(p, ci, 0, f);
        for (int v = tid; v < n; v += kFrameThreads) lch[v] = __ldg(fc.llr + v);
        for (int w = tid; w < ci.swords; w += kFrameThreads) sb[w] = __ldg(fc.sbits + w);
        __syncthreads();
        double qprev = 0.0;  // used by warp 0 only
        for (int k = 0;; ++k) {
            // ---- check pass of iteration k + 1 with the syndrome test of x^(k) ----
            const int mode = k == 0 ? kModeFirst : (k >= p.max_iter ? kModeSynd : kModeFull);
            const bool want_synd = k >= 1 && (p.rule != kRuleNone || k >= p.max_iter);
            if constexpr (W) fc.wrow = weight_row(p, k);
            bool unsat = false;
            for (int i = c_first; i < m; i += c_step) {  // checks by degree: warps run one degree's code
                const int row = rord[i];
                const int e0 = rptr[row];
                const int d = (int)rptr[row + 1] - e0;
                const unsigned sbit = (sb[row >> 5] >> (row & 31)) & 1u;
#define LDPC_FRAME_CHECK(D) \
    unsat |= smem_cn_check<D, W, NC>(p, fc, mode, want_synd, sbit, e0, col, app, lch, c2v, peer_c2v, rank)
                switch (d) {
                    case 1: LDPC_FRAME_CHECK(1); break;
                    case 2: LDPC_FRAME_CHECK(2); break;
                    case 3: LDPC_FRAME_CHECK(3); break;
                    case 4: LDPC_FRAME_CHECK(4); break;
                    case 5: LDPC_FRAME_CHECK(5); break;
                    case 6: LDPC_FRAME_CHECK(6); break;
                    default:
                        unsat |= smem_cn_check_n<W, NC>(p, fc, mode, want_synd, sbit, e0, d, col, app, lch, c2v,
                                                        peer_c2v, rank);
                        break;
                }
#undef LDPC_FRAME_CHECK
            }
            if (want_synd && __any_sync(0xffffffffu, unsat) && lane == 0) {
                atomicOr(&s_unsat[k & 1], 1);
                if constexpr (NC == 2) (void)dsmem_or_b32(peer_unsat + 4u * (unsigned)(k & 1), 1u);
            }
            const bool with_q0 = k == 1 && p.vnr_first_iter <= 1;
            if constexpr (NC == 2) {
                // q partials of APP^(k) (and of Lch for q^(0)) from this CTA's full APP copy:
                // slot tile * kWarps + w sums, per lane, the tile's variables
                // tile * kVnTile + c * kThreads + 32 w + lane for c = 0 .. kVPT - 1 in order,
                // exactly as the variable pass of the one-CTA schedule does
                if (k >= 1) {
                    for (int sl = warp; sl < npart; sl += kFrameThreads / 32) {
                        const int tile = sl / kWarps, wv = sl - tile * kWarps;
                        float acc = 0.0f, acc0 = 0.0f;
#pragma unroll
                        for (int c = 0; c < kVPT; ++c) {
                            const int v = tile * kVnTile + c * kThreads + wv * 32 + lane;
                            if (v < n && (int)vptr[v + 1] - (int)vptr[v] > 1) {
                                acc += fabsf(app[v]);
                                acc0 += fabsf(lch[v]);
                            }
                        }
                        warp_sum_to(acc, part + sl);
                        if (with_q0) warp_sum_to(acc0, part0 + sl);
                    }
                }
                cluster_barrier();  // both CTAs' messages and syndrome flags are in place
            } else {
                __syncthreads();
            }
            // ---- q^(k): one warp per fixed range, the 256-thread CTA's tree; then warp 0
            //      takes the decision ----
            if (k >= 1 && warp < kQParts) {
                const int lo = warp * per, cnt = max(0, min(npart, lo + per) - lo);
                const double qr = warp_block_sum_fixed(part + lo, cnt);
                const double q0r = with_q0 ? warp_block_sum_fixed(part0 + lo, cnt) : 0.0;
                if (lane == 0) {
                    s_q[warp] = qr;
                    s_q0[warp] = q0r;
                }
                asm volatile("bar.sync 1, %0;" ::"r"(kQParts * 32) : "memory");  // the range warps only
                if (warp == 0) {
                    // 0.0 + s_q[0] == s_q[0]; empty ranges hold +0.0 and are skipped
                    double qv = s_q[0], q0 = s_q0[0];
#pragma unroll
                    for (int r = 1; r < kQParts; ++r)
                        if (r * per < npart) qv += s_q[r];
                    if (with_q0) {
#pragma unroll
                        for (int r = 1; r < kQParts; ++r)
                            if (r * per < npart) q0 += s_q0[r];
                    }
                    const bool sat = s_unsat[k & 1] == 0;
                    const double qp = with_q0 ? q0 : qprev;
                    const bool succ = p.rule != kRuleNone && sat;
                    const bool abort_ = !succ && p.rule == kRulePceVnr && k >= p.vnr_first_iter && qv < qp;
                    const bool stop_k = succ || abort_ || k >= p.max_iter;
                    if (lane == 0) {
                        if (rank == 0) {  // both CTAs of a pair decide alike; one writes
                            if (k <= p.trace_iters && p.trace_q) p.trace_q[(long long)(k - 1) * p.frames + f] = qv;
                            if (stop_k) {
                                p.flags_out[f] = (unsigned char)((sat ? 1 : 0) | (abort_ ? 2 : 0));
                                p.iters_out[f] = k;
                                atomicAdd(&p.ctrl->frame_iters, (unsigned long long)k);
                            }
                        }
                        s_stop = stop_k ? 1 : 0;
                    }
                    qprev = qv;
                }
            }
            if (tid == 0) s_unsat[(k + 1) & 1] = 0;  // the flag of the next check pass
            __syncthreads();
            if (k >= 1 && s_stop != 0) {
                for (int v0 = (int)rank << kPairShift; v0 < n; v0 += NC << kPairShift) {
                    const int v = v0 + tid;
                    if (v < n) fc.bits[v] = (unsigned char)(app[v] < 0.0f);
                }
                break;  // the next frame starts behind a barrier
            }
            // ---- variable pass: APP^(k+1) (and, one CTA per frame, its q partials) ----
            const bool trace = k < p.trace_iters;
            if constexpr (NC == 2) {
                // one variable per thread, in this CTA's 1024-variable blocks; APP into both copies
                for (int v0 = (int)rank << kPairShift; v0 < n; v0 += NC << kPairShift) {
                    const int v = v0 + tid;
                    if (v < n) {
                        const int a0 = vptr[v], a1 = vptr[v + 1];
                        float sum = lch[v];
                        for (int a = a0; a < a1; ++a) sum += c2v[LDPC_IX(p.ctrl, vedge[a], E, kIxCsrMsg)];
                        app[v] = sum;
                        dsmem_st_f32(peer_app + 4u * (unsigned)v, sum);
                        if (trace && p.trace_app) p.trace_app[((size_t)k * p.frames + f) * (size_t)n + v] = sum;
                    }
                }
            } else {
                // as virtual 256-thread CTAs, with the q partials
                const bool want_q0 = k == 0 && p.vnr_first_iter <= 1;
                for (int tile = tid / kThreads; tile < ci.vn_tiles; tile += kFrameVirt) {
                    float acc = 0.0f, acc0 = 0.0f;
#pragma unroll
                    for (int c = 0; c < kVPT; ++c) {
                        const int v = tile * kVnTile + c * kThreads + vt;
                        if (v < n) {
                            const int a0 = vptr[v], a1 = vptr[v + 1];
                            const float Lv = lch[v];
                            float sum = Lv;
                            for (int a = a0; a < a1; ++a) sum += c2v[LDPC_IX(p.ctrl, vedge[a], E, kIxCsrMsg)];
                            app[v] = sum;
                            if (a1 - a0 > 1) {
                                acc += fabsf(sum);
                                acc0 += fabsf(Lv);
                            }
                            if (trace && p.trace_app) p.trace_app[((size_t)k * p.frames + f) * (size_t)n + v] = sum;
                        }
                    }
                    const int slot = tile * kWarps + (vt >> 5);
                    warp_sum_to(acc, part + slot);
                    if (want_q0) warp_sum_to(acc0, part0 + slot);
                }
            }
            if (trace && p.trace_c2v) {
                float* tr = p.trace_c2v + ((size_t)k * p.frames + f) * (size_t)E;
                if constexpr (NC == 2) {  // the messages of this CTA's checks
                    for (int i = c_first; i < m; i += c_step) {
                        const int row = rord[i];
                        for (int e = rptr[row]; e < (int)rptr[row + 1]; ++e) tr[e] = c2v[e];
                    }
                } else {
                    for (long long e = tid; e < E; e += kFrameThreads) tr[e] = c2v[e];
                }
            }
            if constexpr (NC == 2) cluster_barrier(); else __syncthreads();
        }
    }
}

}  // namespace ldpcgb
