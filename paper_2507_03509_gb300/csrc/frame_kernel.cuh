// Frame-per-CTA schedule of the decoder for small CSR codes (whole frame in
// shared memory).
//
// When a frame's messages and APP values fit one CTA's shared memory (about
// 4E + 4n bytes; the n = 4096 workload code needs 65 KB), a CTA decodes whole
// frames on its own, taking them from the shared queue: the same steps as the
// lock-step kernel (check pass with the fused syndrome test, q^(k), decision,
// variable pass), separated by CTA barriers instead of grid barriers, with
// the code's index lists read through the read-only cache.  The check and
// variable items, the per-warp q partials (tile * kWarps + warp) and the eight
// fixed q ranges are the lock-step kernel's, so every result is bit-identical.
// Opt-in (LDPC_SCHEDULE_FRAME): with fewer frames than SMs each SM runs one
// 8-warp CTA whose dependent index and shared-memory loads set its pace.
#pragma once

#include "bp_kernels.cuh"

namespace ldpcgb {

// Shared memory of csr_frame_kernel for a code of n variables, E edges and
// vn_tiles variable tiles: messages, APP values and the q partials of the
// frame (and of q^(0)), 16-byte aligned pieces.
__host__ __device__ constexpr size_t frame_smem_bytes(long long E, int n, int vn_tiles) {
    return (size_t)((E + 3) / 4 * 4) * 4 + (size_t)((n + 3) / 4 * 4) * 4 + 2 * (size_t)vn_tiles * kWarps * 8;
}

template <bool W>
__global__ void __launch_bounds__(kThreads) csr_frame_kernel(Params<float> p, CodeInfo<CsrDev> ci) {
    extern __shared__ double smem_frame[];
    const long long Ep = (ci.E + 3) / 4 * 4;
    double* part = smem_frame;                                  // [vn_tiles * kWarps]
    double* part0 = part + (size_t)ci.vn_tiles * kWarps;        // [vn_tiles * kWarps]
    float* c2v = (float*)(part0 + (size_t)ci.vn_tiles * kWarps);  // [E]
    float* app = c2v + Ep;                                       // [n]
    __shared__ double s_red[kWarps];
    __shared__ int s_frame, s_unsat;
    const int lane = threadIdx.x & 31;
    const CsrDev& g = ci.code;

    for (;;) {
        if (threadIdx.x == 0) s_frame = atomicAdd(&p.ctrl->next_frame, 1);
        __syncthreads();
        const int f = s_frame;
        if (f >= p.frames) break;
        FrameCtx<float> fc = frame_ctx(p, ci, 0, f);
        fc.c2v = c2v;
        fc.app = app;
        fc.qpart = part;
        fc.q0part = part0;
        double qprev = 0.0;
        for (int k = 0;; ++k) {
            // ---- check pass of iteration k + 1 with the syndrome test of x^(k) ----
            if (threadIdx.x == 0) s_unsat = 0;
            __syncthreads();
            const int mode = k == 0 ? kModeFirst : (k >= p.max_iter ? kModeSynd : kModeFull);
            const bool want_synd = k >= 1 && (p.rule != kRuleNone || k >= p.max_iter);
            if constexpr (W) fc.wrow = weight_row(p, k);
            bool unsat = false;
            for (int tile = 0; tile < ci.cn_tiles; ++tile) unsat |= cn_tile<W, float>(p, g, fc, mode, want_synd, tile);
            if (want_synd && __any_sync(0xffffffffu, unsat) && lane == 0) atomicOr(&s_unsat, 1);
            // ---- q^(k): the eight fixed ranges of the per-warp partials, in order ----
            double qv = 0.0, q0 = 0.0;
            const bool with_q0 = k == 1 && p.vnr_first_iter <= 1;
            if (k >= 1) {
                const int npart = ci.nqb * kWarps;
                const int per = (npart + kQParts - 1) / kQParts;
                for (int r = 0; r < kQParts; ++r) {
                    const int lo = r * per, cnt = max(0, min(npart, lo + per) - lo);
                    qv += block_sum_fixed(part + lo, cnt, s_red);
                    if (with_q0) q0 += block_sum_fixed(part0 + lo, cnt, s_red);
                }
            }
            __syncthreads();
            // ---- decision (every thread takes the same one) ----
            bool stop = false;
            if (k >= 1) {
                const bool sat = s_unsat == 0;
                if (k <= p.trace_iters && p.trace_q && threadIdx.x == 0) p.trace_q[(long long)(k - 1) * p.frames + f] = qv;
                const double qp = with_q0 ? q0 : qprev;
                const bool succ = p.rule != kRuleNone && sat;
                const bool abort_ = !succ && p.rule == kRulePceVnr && k >= p.vnr_first_iter && qv < qp;
                stop = succ || abort_ || k >= p.max_iter;
                if (stop && threadIdx.x == 0) {
                    p.flags_out[f] = (unsigned char)((sat ? 1 : 0) | (abort_ ? 2 : 0));
                    p.iters_out[f] = k;
                    atomicAdd(&p.ctrl->frame_iters, (unsigned long long)k);
                }
                qprev = qv;
            }
            if (stop) {
                for (int tile = 0; tile < ci.vn_tiles; ++tile) final_tile(fc, tile);
                __syncthreads();
                break;
            }
            // ---- variable pass: APP^(k+1) and its q partials ----
            for (int tile = 0; tile < ci.vn_tiles; ++tile) vn_tile<float>(p, g, fc, k, tile);
            __syncthreads();
        }
    }
}

}  // namespace ldpcgb
