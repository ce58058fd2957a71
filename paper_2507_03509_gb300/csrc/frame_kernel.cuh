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
#pragma once

#include "bp_kernels.cuh"
#include "flow_kernel.cuh"

namespace ldpcgb {

constexpr int kFrameThreads = 1024;
constexpr int kFrameVirt = kFrameThreads / kThreads;  // virtual 256-thread CTAs per frame CTA

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
template <int D, bool W>
__device__ __forceinline__ bool smem_cn_check(const Params<float>& p, const FrameCtx<float>& fc, int mode,
                                              bool want_synd, unsigned sbit, int e0, const unsigned short* col,
                                              const float* app, const float* lch, float* c2v) {
    float a[D], o[D];
#pragma unroll
    for (int j = 0; j < D; ++j) {
        const int vi = (int)LDPC_IX(p.ctrl, col[e0 + j], fc.n, kIxCsrVar);
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
    for (int j = 0; j < D; ++j) c2v[e0 + j] = weighted<W>(p, fc, out[j], e0 + j);
    return unsat;
}

// Any degree (0 and > 6): the arithmetic of csr_cn_check_n.
template <bool W>
__device__ __noinline__ bool smem_cn_check_n(const Params<float>& p, const FrameCtx<float>& fc, int mode,
                                             bool want_synd, unsigned sbit, int e0, int d,
                                             const unsigned short* col, const float* app, const float* lch,
                                             float* c2v) {
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
    for (int j = 0; j < d; ++j) c2v[e0 + j] = weighted<W>(p, fc, out[j], e0 + j);
    return unsat;
}

template <bool W>
__global__ void __launch_bounds__(kFrameThreads, 1) csr_frame_kernel(Params<float> p, CodeInfo<CsrDev> ci,
                                                                      FrameSmem L) {
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

    for (;;) {
        if (tid == 0) s_frame = atomicAdd(&p.ctrl->next_frame, 1);
        __syncthreads();
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
            for (int i = tid; i < m; i += kFrameThreads) {  // checks by degree: warps run one degree's code
                const int row = rord[i];
                const int e0 = rptr[row];
                const int d = (int)rptr[row + 1] - e0;
                const unsigned sbit = (sb[row >> 5] >> (row & 31)) & 1u;
                switch (d) {
                    case 1: unsat |= smem_cn_check<1, W>(p, fc, mode, want_synd, sbit, e0, col, app, lch, c2v); break;
                    case 2: unsat |= smem_cn_check<2, W>(p, fc, mode, want_synd, sbit, e0, col, app, lch, c2v); break;
                    case 3: unsat |= smem_cn_check<3, W>(p, fc, mode, want_synd, sbit, e0, col, app, lch, c2v); break;
                    case 4: unsat |= smem_cn_check<4, W>(p, fc, mode, want_synd, sbit, e0, col, app, lch, c2v); break;
                    case 5: unsat |= smem_cn_check<5, W>(p, fc, mode, want_synd, sbit, e0, col, app, lch, c2v); break;
                    case 6: unsat |= smem_cn_check<6, W>(p, fc, mode, want_synd, sbit, e0, col, app, lch, c2v); break;
                    default:
                        unsat |= smem_cn_check_n<W>(p, fc, mode, want_synd, sbit, e0, d, col, app, lch, c2v);
                        break;
                }
            }
            if (want_synd && __any_sync(0xffffffffu, unsat) && lane == 0) atomicOr(&s_unsat[k & 1], 1);
            __syncthreads();
            // ---- q^(k): one warp per fixed range, the 256-thread CTA's tree; then warp 0
            //      takes the decision ----
            const bool with_q0 = k == 1 && p.vnr_first_iter <= 1;
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
                        if (k <= p.trace_iters && p.trace_q) p.trace_q[(long long)(k - 1) * p.frames + f] = qv;
                        if (stop_k) {
                            p.flags_out[f] = (unsigned char)((sat ? 1 : 0) | (abort_ ? 2 : 0));
                            p.iters_out[f] = k;
                            atomicAdd(&p.ctrl->frame_iters, (unsigned long long)k);
                        }
                        s_stop = stop_k ? 1 : 0;
                    }
                    qprev = qv;
                }
            }
            if (tid == 0) s_unsat[(k + 1) & 1] = 0;  // the flag of the next check pass
            __syncthreads();
            if (k >= 1 && s_stop != 0) {
                for (int v = tid; v < n; v += kFrameThreads) fc.bits[v] = (unsigned char)(app[v] < 0.0f);
                break;  // the next frame starts behind a barrier
            }
            // ---- variable pass: APP^(k+1) and its q partials, as virtual 256-thread CTAs ----
            const bool want_q0 = k == 0 && p.vnr_first_iter <= 1;
            const bool trace = k < p.trace_iters;
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
            if (trace && p.trace_c2v) {
                float* tr = p.trace_c2v + ((size_t)k * p.frames + f) * (size_t)E;
                for (long long e = tid; e < E; e += kFrameThreads) tr[e] = c2v[e];
            }
            __syncthreads();
        }
    }
}

}  // namespace ldpcgb
