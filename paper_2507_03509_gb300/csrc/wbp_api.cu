// C ABI of weighted belief propagation (ldpc_wbp_* in include/ldpc.h).
//
// Host side: builds the per-class lists of message slots, owns the plan's
// workspace (allocated once at creation), and issues the stream-ordered
// kernel sequences of wbp_kernels.cuh -- forward with checkpoints, loss,
// backward with recomputation between checkpoints, gradient step.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/ldpc.h"
#include "host_common.h"
#include "wbp_kernels.cuh"

using namespace ldpcgb;

struct ldpc_wbp {
    const ldpc_graph* graph = nullptr;
    int device = 0;
    int F = 0, T = 0, C = 0, every = 1, fp64 = 0;
    int m = 0, n = 0;
    long long E = 0;
    int nckpt = 0;               // checkpoints kept by the forward pass (iterations every, 2 every, ... < T)
    int nseg = 0;                // recomputed iterations held during the backward pass (every - 1)
    int k0_last = 0;             // first iteration of the last checkpoint segment
    int ntail = 0;               // iterations of the last segment kept by the forward pass (T - 1 - k0_last)
    bool saved = false;          // a forward pass has stored checkpoints
    void* tables = nullptr;      // cls | class_ptr | class_slot
    const int* cls = nullptr;
    const int* class_ptr = nullptr;
    const int* class_slot = nullptr;
    void* buf = nullptr;
    size_t elem = 4;
    // state, offsets into buf
    char* c2v_work = nullptr;    // [F][E]
    char* app_work = nullptr;    // [F][n]
    std::vector<char*> ck_c2v, ck_app;    // [nckpt] of [F][E] / [F][n]
    std::vector<char*> seg_c2v, seg_app;  // [nseg]
    std::vector<char*> tail_c2v, tail_app;  // [max(ntail, nseg)]: iterations k0_last + 1 .. T - 1 from the
                                            // forward pass; later the second recompute buffer set
    cudaStream_t s2 = nullptr;              // interleaved plans: the backward pass's recompute stream
    std::vector<cudaEvent_t> ev;            // [1 + 2 * segments]: ordering between the two streams
    char* G = nullptr;           // [F][E]
    char* pbuf = nullptr;        // [F][E]
    double* partial = nullptr;   // loss partial sums [loss_blocks]
    int loss_blocks = 0;
    int grid_cn = 1, grid_vn = 1, grid_w = 1;
    // QC plans: tiled kernels, per-tile sums of G * t, classes as lists of blocks
    int tiles_cn = 1;            // check tiles per base row
    int fpc_cn = 1, fpc_vn = 1;  // frames per CTA group, check / variable side
    int groups_cn = 1;
    long long grid_qcn = 1, grid_qvn = 1;
    double* wpart = nullptr;     // [iters][groups_cn][nblk][tiles_cn]
    size_t wpart_per = 0;        // doubles of wpart per iteration
    const int* cblk_ptr = nullptr;
    const int* cblk = nullptr;
    // FP32 QC plans: state interleaved by frame quads (wbp_kernels.cuh, Args4);
    // F4 = ceil(F / 4) quads, the state arrays hold 4 * F4 frames
    bool x4 = false;
    int F4 = 0;
    int fpq_cn = 1, fpq_vn = 1;  // quads per CTA group, check / variable side
    float* llr4 = nullptr;       // [F4][n][4] interleaved Lch
    unsigned char* syn4 = nullptr;  // [F4][m] syndrome bits of the quad's frames
    float* grad4 = nullptr;      // [F4][n][4] accumulated dloss/dLch
    int grid_pack = 1;
};

namespace {

template <typename T, class Code>
struct Runner {
    ldpc_wbp* p;
    Code code;
    cudaStream_t s;

    wbp::Args<T> base(const float* llr, const uint8_t* syn) const {
        wbp::Args<T> a{};
        a.F = p->F;
        a.m = p->m;
        a.n = p->n;
        a.E = p->E;
        a.lmax = T(25);
        a.llr = llr;
        a.syn = syn;
        a.cls = p->cls;
        return a;
    }
    static constexpr bool kQc = std::is_same_v<Code, QcDev>;
    static bool aligned(const void* ptr) { return ptr == nullptr || ((uintptr_t)ptr % 16) == 0; }

    // iteration k (1-based) forward: c2v^(k) into c2v_dst, APP^(k) into app_dst
    ldpc_status fwd(const float* llr, const uint8_t* syn, const T* w, int k, const T* c2v_prev,
                    const T* app_prev, T* c2v_dst, T* app_dst) const {
        wbp::Args<T> a = base(llr, syn);
        a.w = w + (size_t)(k - 1) * p->C;
        a.c2v_prev = c2v_prev;
        a.app_prev = app_prev;
        a.c2v_out = c2v_dst;
        a.app_out = app_dst;
        if constexpr (kQc) {
            a.vec = p->graph->Z % 4 == 0 && aligned(llr) && aligned(app_dst);
            wbp::qc_cn_kernel<false, T><<<(unsigned)p->grid_qcn, wbp::kThreads, 0, s>>>(a, code, p->tiles_cn,
                                                                                          p->fpc_cn, nullptr);
            LDPC_TRY(cudaGetLastError());
            wbp::qc_vn_kernel<wbp::kVnFwd, T><<<(unsigned)p->grid_qvn, wbp::kThreads, 0, s>>>(a, code, p->fpc_vn,
                                                                                              nullptr);
        } else {
            wbp::cn_kernel<false, T, Code><<<p->grid_cn, wbp::kThreads, 0, s>>>(a, code);
            LDPC_TRY(cudaGetLastError());
            wbp::vn_fwd_kernel<T, Code><<<p->grid_vn, wbp::kThreads, 0, s>>>(a, code);
        }
        LDPC_TRY(cudaGetLastError());
        return LDPC_OK;
    }
    T* ck_c2v(int i) const { return (T*)p->ck_c2v[i]; }
    T* ck_app(int i) const { return (T*)p->ck_app[i]; }

    // ---- interleaved (x4) path of FP32 QC plans -------------------------
    wbp::Args4 base4() const {
        wbp::Args4 a{};
        a.F = p->F;
        a.F4 = p->F4;
        a.m = p->m;
        a.n = p->n;
        a.E = p->E;
        a.lmax = 25.0f;
        a.llr4 = (const float4*)p->llr4;
        a.syn4 = p->syn4;
        a.cls = p->cls;
        return a;
    }
    ldpc_status pack4(const float* llr, const uint8_t* syn) const {
        wbp::pack4_kernel<<<p->grid_pack, wbp::kThreads, 0, s>>>(llr, syn, p->F, p->F4, p->n, p->m,
                                                                 (float4*)p->llr4, p->syn4);
        LDPC_TRY(cudaGetLastError());
        return LDPC_OK;
    }
    // iteration k forward on the interleaved state; app_rows (the caller's
    // frame-major buffer) receives APP^(k) instead of app_dst when given
    ldpc_status fwd4(const float* w, int k, const float* c2v_prev, const float* app_prev, float* c2v_dst,
                     float* app_dst, float* app_rows) const {
        return fwd4_on(s, w, k, c2v_prev, app_prev, c2v_dst, app_dst, app_rows);
    }
    ldpc_status fwd4_on(cudaStream_t st, const float* w, int k, const float* c2v_prev, const float* app_prev,
                        float* c2v_dst, float* app_dst, float* app_rows) const {
        if constexpr (kQc) {
            wbp::Args4 a = base4();
            a.w = w + (size_t)(k - 1) * p->C;
            a.c2v_prev = (const float4*)c2v_prev;
            a.app_prev = (const float4*)app_prev;
            a.c2v_out = (float4*)c2v_dst;
            a.app_out = app_rows ? nullptr : (float4*)app_dst;
            a.app_rows = app_rows;
            wbp::qc_cn4_kernel<false><<<(unsigned)p->grid_qcn, wbp::kThreads, 0, st>>>(a, code, p->tiles_cn,
                                                                                        p->fpq_cn, nullptr);
            LDPC_TRY(cudaGetLastError());
            wbp::qc_vn4_kernel<wbp::kVnFwd><<<(unsigned)p->grid_qvn, wbp::kThreads, 0, st>>>(a, code, p->fpq_vn);
            LDPC_TRY(cudaGetLastError());
        }
        return LDPC_OK;
    }
    ldpc_status forward4(const float* llr, const uint8_t* syn, const float* w, float* app_out, bool save) {
        ldpc_status st = pack4(llr, syn);
        if (st != LDPC_OK) return st;
        const float* cprev = nullptr;
        const float* aprev = nullptr;
        for (int k = 1; k <= p->T; ++k) {
            float* cdst = (float*)p->c2v_work;
            float* adst = (float*)p->app_work;
            if (save && k % p->every == 0 && k < p->T) {
                cdst = (float*)ck_c2v(k / p->every - 1);
                adst = (float*)ck_app(k / p->every - 1);
            } else if (save && k > p->k0_last && k < p->T) {  // the last segment, kept whole
                cdst = (float*)p->tail_c2v[k - p->k0_last - 1];
                adst = (float*)p->tail_app[k - p->k0_last - 1];
            }
            st = fwd4(w, k, cprev, aprev, cdst, adst, k == p->T ? app_out : nullptr);
            if (st != LDPC_OK) return st;
            cprev = cdst;
            aprev = adst;
        }
        return LDPC_OK;
    }
    ldpc_status backward4(const float* llr, const uint8_t* syn, const float* w, const float* grad_app, float* gw,
                          float* gl) {
        if constexpr (kQc) {
            ldpc_status st = pack4(llr, syn);
            if (st != LDPC_OK) return st;
            wbp::Args4 a = base4();
            a.G = (float4*)p->G;
            a.grad4 = gl ? (float4*)p->grad4 : nullptr;
            a.grad_app = grad_app;
            wbp::qc_vn4_kernel<wbp::kVnSeed><<<(unsigned)p->grid_qvn, wbp::kThreads, 0, s>>>(a, code, p->fpq_vn);
            LDPC_TRY(cudaGetLastError());
            const int every = p->every;
            const int L = (p->T + every - 1) / every - 1;  // the last segment
            // Segment sg works in buffer set A (the kept tail) if L - sg is even, else in set B (the
            // recompute buffers).  The recomputation of segment sg - 1 runs on the second stream
            // while segment sg's adjoint runs on the caller's; recomputing segment sg - 2, which
            // reuses segment sg's set, waits for that adjoint.  No result depends on this overlap.
            const bool overlap = p->s2 != nullptr && (int)p->ev.size() >= 2 * (L + 1) + 1;
            cudaStream_t rs = overlap ? p->s2 : s;
            auto set_c = [&](int sg) -> const std::vector<char*>& { return (L - sg) % 2 == 0 ? p->tail_c2v : p->seg_c2v; };
            auto set_a = [&](int sg) -> const std::vector<char*>& { return (L - sg) % 2 == 0 ? p->tail_app : p->seg_app; };
            auto recompute = [&](int sg) -> ldpc_status {
                const int k0 = sg * every, k1 = std::min((sg + 1) * every, p->T);
                const float* c0 = k0 == 0 ? nullptr : (const float*)ck_c2v(sg - 1);
                const float* a0 = k0 == 0 ? nullptr : (const float*)ck_app(sg - 1);
                const std::vector<char*>& sc = set_c(sg);
                const std::vector<char*>& sa = set_a(sg);
                for (int k = k0 + 1; k < k1; ++k) {
                    const float* cp = k - 1 == k0 ? c0 : (const float*)sc[k - 1 - k0 - 1];
                    const float* ap = k - 1 == k0 ? a0 : (const float*)sa[k - 1 - k0 - 1];
                    const ldpc_status s3 =
                        fwd4_on(rs, w, k, cp, ap, (float*)sc[k - k0 - 1], (float*)sa[k - k0 - 1], nullptr);
                    if (s3 != LDPC_OK) return s3;
                }
                if (overlap) LDPC_TRY(cudaEventRecord(p->ev[1 + 2 * sg], rs));  // recomputed
                return LDPC_OK;
            };
            if (overlap) {
                LDPC_TRY(cudaEventRecord(p->ev[0], s));  // packed inputs and the seed are in place
                LDPC_TRY(cudaStreamWaitEvent(rs, p->ev[0], 0));
            }
            if (L >= 1 && overlap) {
                st = recompute(L - 1);
                if (st != LDPC_OK) return st;
            }
            for (int sg = L; sg >= 0; --sg) {
                const int k0 = sg * every, k1 = std::min((sg + 1) * every, p->T);
                const float* c0 = k0 == 0 ? nullptr : (const float*)ck_c2v(sg - 1);
                const float* a0 = k0 == 0 ? nullptr : (const float*)ck_app(sg - 1);
                const std::vector<char*>& sc = set_c(sg);
                const std::vector<char*>& sa = set_a(sg);
                if (sg < L) {
                    if (overlap) {
                        LDPC_TRY(cudaStreamWaitEvent(s, p->ev[1 + 2 * sg], 0));
                    } else {
                        st = recompute(sg);  // the last segment was kept by the forward pass
                        if (st != LDPC_OK) return st;
                    }
                }
                for (int k = k1; k > k0; --k) {
                    a.w = w + (size_t)(k - 1) * p->C;
                    a.c2v_prev = (const float4*)(k - 1 == k0 ? c0 : (const float*)sc[k - 1 - k0 - 1]);
                    a.app_prev = (const float4*)(k - 1 == k0 ? a0 : (const float*)sa[k - 1 - k0 - 1]);
                    wbp::qc_cn4_kernel<true><<<(unsigned)p->grid_qcn, wbp::kThreads, 0, s>>>(
                        a, code, p->tiles_cn, p->fpq_cn, p->wpart + (size_t)(k - 1) * p->wpart_per);
                    LDPC_TRY(cudaGetLastError());
                    wbp::qc_vn4_kernel<wbp::kVnBwd><<<(unsigned)p->grid_qvn, wbp::kThreads, 0, s>>>(a, code,
                                                                                                    p->fpq_vn);
                    LDPC_TRY(cudaGetLastError());
                }
                if (overlap && sg >= 2) {  // segment sg - 2 reuses this segment's buffers
                    LDPC_TRY(cudaEventRecord(p->ev[2 + 2 * sg], s));
                    LDPC_TRY(cudaStreamWaitEvent(rs, p->ev[2 + 2 * sg], 0));
                    st = recompute(sg - 2);
                    if (st != LDPC_OK) return st;
                }
            }
            LDPC_TRY(class_reduce_all(gw));
            if (gl) {
                wbp::unpack4_kernel<<<p->grid_pack, wbp::kThreads, 0, s>>>((const float4*)p->grad4, p->F, p->n, gl);
                LDPC_TRY(cudaGetLastError());
            }
        }
        return LDPC_OK;
    }

    ldpc_status forward(const float* llr, const uint8_t* syn, const T* w, T* app_out, bool save) {
        if constexpr (kQc && std::is_same_v<T, float>) {
            if (p->x4) return forward4(llr, syn, w, app_out, save);
        }
        const T* cprev = nullptr;
        const T* aprev = nullptr;
        for (int k = 1; k <= p->T; ++k) {
            T* cdst = (T*)p->c2v_work;
            T* adst = k == p->T ? app_out : (T*)p->app_work;
            if (save && k % p->every == 0 && k < p->T) {
                cdst = ck_c2v(k / p->every - 1);
                adst = ck_app(k / p->every - 1);
            } else if (save && k > p->k0_last && k < p->T) {  // the last segment, kept whole
                cdst = (T*)p->tail_c2v[k - p->k0_last - 1];
                adst = (T*)p->tail_app[k - p->k0_last - 1];
            }
            ldpc_status st = fwd(llr, syn, w, k, cprev, aprev, cdst, adst);
            if (st != LDPC_OK) return st;
            cprev = cdst;
            aprev = adst;
        }
        return LDPC_OK;
    }

    ldpc_status backward(const float* llr, const uint8_t* syn, const T* w, const T* grad_app, T* gw, T* gl) {
        if constexpr (kQc && std::is_same_v<T, float>) {
            if (p->x4) return backward4(llr, syn, w, grad_app, gw, gl);
        }
        wbp::Args<T> a = base(llr, syn);
        a.G = (T*)p->G;
        a.pbuf = (T*)p->pbuf;
        a.grad_llr = gl;
        if constexpr (kQc) {
            a.vec = p->graph->Z % 4 == 0 && aligned(llr) && aligned(grad_app) && aligned(gl);
            wbp::qc_vn_kernel<wbp::kVnSeed, T><<<(unsigned)p->grid_qvn, wbp::kThreads, 0, s>>>(a, code, p->fpc_vn,
                                                                                               grad_app);
        } else {
            wbp::seed_kernel<T, Code><<<p->grid_vn, wbp::kThreads, 0, s>>>(a, code, grad_app);
        }
        LDPC_TRY(cudaGetLastError());
        const int every = p->every;
        const int nseg_total = (p->T + every - 1) / every;
        for (int sg = nseg_total - 1; sg >= 0; --sg) {
            const int k0 = sg * every, k1 = std::min((sg + 1) * every, p->T);
            const T* c0 = k0 == 0 ? nullptr : ck_c2v(sg - 1);
            const T* a0 = k0 == 0 ? nullptr : ck_app(sg - 1);
            // recompute c2v^(k), APP^(k) for k0 < k < k1; the last segment was kept by the forward pass
            const bool last = sg == nseg_total - 1;
            const std::vector<char*>& sc = last ? p->tail_c2v : p->seg_c2v;
            const std::vector<char*>& sa = last ? p->tail_app : p->seg_app;
            for (int k = k0 + 1; k < k1 && !last; ++k) {
                const T* cp = k - 1 == k0 ? c0 : (T*)sc[k - 1 - k0 - 1];
                const T* ap = k - 1 == k0 ? a0 : (T*)sa[k - 1 - k0 - 1];
                ldpc_status st = fwd(llr, syn, w, k, cp, ap, (T*)sc[k - k0 - 1], (T*)sa[k - k0 - 1]);
                if (st != LDPC_OK) return st;
            }
            for (int k = k1; k > k0; --k) {
                a.w = w + (size_t)(k - 1) * p->C;
                a.c2v_prev = k - 1 == k0 ? c0 : (T*)sc[k - 1 - k0 - 1];
                a.app_prev = k - 1 == k0 ? a0 : (T*)sa[k - 1 - k0 - 1];
                if constexpr (kQc) {
                    wbp::qc_cn_kernel<true, T><<<(unsigned)p->grid_qcn, wbp::kThreads, 0, s>>>(
                        a, code, p->tiles_cn, p->fpc_cn, p->wpart + (size_t)(k - 1) * p->wpart_per);
                    LDPC_TRY(cudaGetLastError());
                    wbp::qc_vn_kernel<wbp::kVnBwd, T><<<(unsigned)p->grid_qvn, wbp::kThreads, 0, s>>>(
                        a, code, p->fpc_vn, nullptr);
                } else {
                    wbp::cn_kernel<true, T, Code><<<p->grid_cn, wbp::kThreads, 0, s>>>(a, code);
                    LDPC_TRY(cudaGetLastError());
                    wbp::wgrad_kernel<T><<<p->grid_w, wbp::kThreads, 0, s>>>(
                        (const T*)p->pbuf, p->F, p->E, p->class_ptr, p->class_slot, p->C,
                        gw + (size_t)(k - 1) * p->C);
                    LDPC_TRY(cudaGetLastError());
                    wbp::vn_bwd_kernel<T, Code><<<p->grid_vn, wbp::kThreads, 0, s>>>(a, code);
                }
                LDPC_TRY(cudaGetLastError());
            }
        }
        if constexpr (kQc) LDPC_TRY(class_reduce_all(gw));
        return LDPC_OK;
    }
    // dloss/dw of every iteration and class from the adjoint check passes' per-tile
    // partials, in one launch once the backward pass is done (QC plans)
    template <typename G>
    cudaError_t class_reduce_all(G* gw) const {
        const unsigned grid = (unsigned)std::min(p->T * p->C, 8192);
        wbp::class_reduce_kernel<G><<<grid, wbp::kThreads, 0, s>>>(p->wpart, p->wpart_per, p->groups_cn,
                                                                   p->graph->nblk, p->tiles_cn, p->cblk_ptr,
                                                                   p->cblk, p->C, p->T, gw);
        return cudaGetLastError();
    }
};

template <class Fn>
ldpc_status dispatch(ldpc_wbp* p, cudaStream_t s, Fn&& fn) {
    if (p->graph->kind == 1) {
        if (p->fp64) return fn(Runner<double, QcDev>{p, p->graph->qc, s});
        return fn(Runner<float, QcDev>{p, p->graph->qc, s});
    }
    if (p->fp64) return fn(Runner<double, CsrDev>{p, p->graph->csr, s});
    return fn(Runner<float, CsrDev>{p, p->graph->csr, s});
}

void release(ldpc_wbp* p) {
    for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
    p->ev.clear();
    if (p->s2) cudaStreamDestroy(p->s2);
    p->s2 = nullptr;
    if (p->tables) cudaFree(p->tables);
    if (p->buf) cudaFree(p->buf);
    p->tables = nullptr;
    p->buf = nullptr;
}

int grid_for(long long items, int sms) {
    const long long blocks = (items + wbp::kThreads - 1) / wbp::kThreads;
    return (int)std::max(1LL, std::min(blocks, (long long)sms * 16));
}

}  // namespace

namespace ldpcgb {
bool wbp_plan_classes(const ldpc_wbp* p, const ldpc_graph** graph, const int** cls, int* iters, int* classes) {
    if (!p) return false;
    *graph = p->graph;
    *cls = p->cls;
    *iters = p->T;
    *classes = p->C;
    return true;
}
}  // namespace ldpcgb

extern "C" {

ldpc_status ldpc_wbp_create(const ldpc_graph* graph, int32_t frames, int32_t iters, int32_t n_classes,
                            const int32_t* edge_class, int32_t checkpoint_every, int32_t fp64, ldpc_wbp** out) {
    if (!out) return LDPC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!graph || frames < 1 || iters < 1 || n_classes < 1 || !edge_class || checkpoint_every < 1 ||
        (fp64 != 0 && fp64 != 1))
        return LDPC_ERR_INVALID_ARG;
    if ((long long)frames * graph->E > (1LL << 36) || (long long)frames * graph->m > (1LL << 40))
        return LDPC_ERR_INVALID_ARG;
    const int Z = graph->Z;
    const long long nkeys = graph->kind == 1 ? graph->nblk : graph->E;
    for (long long i = 0; i < nkeys; ++i)
        if (edge_class[i] < 0 || edge_class[i] >= n_classes) return LDPC_ERR_INVALID_ARG;
    // per-class message slots (class order, then ascending slot)
    std::vector<int> cnt((size_t)n_classes + 1, 0);
    for (long long i = 0; i < nkeys; ++i) cnt[edge_class[i] + 1] += graph->kind == 1 ? Z : 1;
    for (int c = 0; c < n_classes; ++c) cnt[c + 1] += cnt[c];
    std::vector<int> slots((size_t)std::max<long long>(graph->E, 1));
    std::vector<int> fill(cnt.begin(), cnt.end() - 1);
    for (long long i = 0; i < nkeys; ++i) {
        const int c = edge_class[i];
        if (graph->kind == 1) {
            for (int p = 0; p < Z; ++p) slots[fill[c]++] = (int)(i * Z + p);
        } else {
            slots[fill[c]++] = (int)i;
        }
    }
    ldpc_wbp* p = new (std::nothrow) ldpc_wbp();
    if (!p) return LDPC_ERR_OOM;
    p->graph = graph;
    p->device = graph->device;
    p->F = frames;
    p->T = iters;
    p->C = n_classes;
    p->every = std::min(checkpoint_every, iters);
    p->fp64 = fp64;
    p->m = graph->m;
    p->n = graph->n;
    p->E = graph->E;
    p->elem = fp64 ? sizeof(double) : sizeof(float);
    p->nckpt = (iters - 1) / p->every;
    p->nseg = p->every - 1;
    p->k0_last = ((iters + p->every - 1) / p->every - 1) * p->every;
    p->ntail = iters - 1 - p->k0_last;
    const int ntailbuf = std::max(p->ntail, p->nseg);  // the tail set also serves as a recompute set
    DeviceGuard guard;
    cudaError_t ce = guard.enter(p->device);
    int sms = 0;
    if (ce == cudaSuccess) ce = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
    // QC: the blocks of each class (class order, ascending block)
    std::vector<int> bptr((size_t)n_classes + 1, 0), blist((size_t)std::max<long long>(nkeys, 1));
    if (graph->kind == 1) {
        for (long long i = 0; i < nkeys; ++i) bptr[edge_class[i] + 1] += 1;
        for (int c = 0; c < n_classes; ++c) bptr[c + 1] += bptr[c];
        std::vector<int> bf(bptr.begin(), bptr.end() - 1);
        for (long long i = 0; i < nkeys; ++i) blist[bf[edge_class[i]]++] = (int)i;
    }
    const size_t tb_cls = align_up((size_t)nkeys * 4, 256), tb_ptr = align_up(((size_t)n_classes + 1) * 4, 256);
    const size_t tb_slot = align_up(slots.size() * 4, 256), tb_blist = align_up(blist.size() * 4, 256);
    if (ce == cudaSuccess) ce = cudaMalloc(&p->tables, tb_cls + 2 * tb_ptr + tb_slot + tb_blist);
    if (ce == cudaSuccess) {
        char* t = (char*)p->tables;
        ce = cudaMemcpy(t, edge_class, (size_t)nkeys * 4, cudaMemcpyHostToDevice);
        if (ce == cudaSuccess) ce = cudaMemcpy(t + tb_cls, cnt.data(), cnt.size() * 4, cudaMemcpyHostToDevice);
        if (ce == cudaSuccess)
            ce = cudaMemcpy(t + tb_cls + tb_ptr, slots.data(), slots.size() * 4, cudaMemcpyHostToDevice);
        if (ce == cudaSuccess)
            ce = cudaMemcpy(t + tb_cls + tb_ptr + tb_slot, bptr.data(), bptr.size() * 4, cudaMemcpyHostToDevice);
        if (ce == cudaSuccess)
            ce = cudaMemcpy(t + tb_cls + 2 * tb_ptr + tb_slot, blist.data(), blist.size() * 4,
                            cudaMemcpyHostToDevice);
        p->cls = (const int*)t;
        p->class_ptr = (const int*)(t + tb_cls);
        p->class_slot = (const int*)(t + tb_cls + tb_ptr);
        p->cblk_ptr = (const int*)(t + tb_cls + tb_ptr + tb_slot);
        p->cblk = (const int*)(t + tb_cls + 2 * tb_ptr + tb_slot);
    }
    // workspace: work c2v/APP, checkpoints, recompute segment, adjoint state, loss partials
    const bool qc = graph->kind == 1;
    p->x4 = qc && !fp64;
    p->F4 = (frames + 3) / 4;
    const long long sframes = p->x4 ? 4LL * p->F4 : frames;  // frames the state arrays hold
    const size_t sE = align_up((size_t)sframes * (size_t)graph->E * p->elem, 256);
    const size_t sN = align_up((size_t)sframes * (size_t)graph->n * p->elem, 256);
    p->loss_blocks = grid_for((long long)frames * graph->n, std::max(sms, 1));
    if (p->x4) {
        // check side: quad groups for about four waves of resident CTAs (4 per SM);
        // variable side: about 2048 (quad, variable) pairs per CTA
        const long long waves = 4LL * std::max(sms, 1) * 4;
        p->tiles_cn = (Z + wbp::kQcCnTile - 1) / wbp::kQcCnTile;
        const long long cn_items = (long long)p->F4 * graph->mb * p->tiles_cn;
        p->fpq_cn = (int)std::max(1LL, std::min<long long>(p->F4, (cn_items + waves - 1) / waves));
        p->groups_cn = (p->F4 + p->fpq_cn - 1) / p->fpq_cn;
        if ((long long)p->groups_cn * graph->mb * p->tiles_cn >= (1LL << 31)) {
            release(p);
            delete p;
            return LDPC_ERR_INVALID_ARG;
        }
        p->grid_qcn = std::min<long long>((long long)p->groups_cn * graph->mb * p->tiles_cn, 1LL << 24);
        p->fpq_vn = std::max(1, std::min(p->F4, 2048 / std::max(Z, 1)));
        p->grid_qvn = std::min<long long>((long long)((p->F4 + p->fpq_vn - 1) / p->fpq_vn) * graph->nb, 1LL << 24);
        p->grid_pack = grid_for((long long)p->F4 * (graph->n + graph->m), std::max(sms, 1));
    } else if (qc) {
        // frame groups sized for about four waves of resident CTAs (4 per SM)
        const long long waves = 4LL * std::max(sms, 1) * 4;
        p->tiles_cn = (Z + wbp::kQcCnTile - 1) / wbp::kQcCnTile;
        const long long cn_items = (long long)frames * graph->mb * p->tiles_cn;
        p->fpc_cn = (int)std::max(1LL, std::min<long long>(frames, (cn_items + waves - 1) / waves));
        p->groups_cn = (frames + p->fpc_cn - 1) / p->fpc_cn;
        p->grid_qcn = std::min<long long>((long long)p->groups_cn * graph->mb * p->tiles_cn, 1LL << 24);
        // variable side: about 4096 (frame, variable) pairs per CTA
        p->fpc_vn = std::max(1, std::min(frames, 4096 / std::max(Z, 1)));
        p->grid_qvn = std::min<long long>((long long)((frames + p->fpc_vn - 1) / p->fpc_vn) * graph->nb, 1LL << 24);
    }
    const size_t sP = qc ? 0 : sE;  // per-edge G * t (CSR plans only)
    p->wpart_per = qc ? (size_t)p->groups_cn * graph->nblk * p->tiles_cn : 0;
    const size_t sW = qc ? align_up((size_t)iters * p->wpart_per * sizeof(double), 256) : 0;
    // interleaved plans: Lch copy, syndrome bits, accumulated dloss/dLch
    const size_t s4n = p->x4 ? align_up((size_t)p->F4 * graph->n * 4 * sizeof(float), 256) : 0;
    const size_t s4m = p->x4 ? align_up((size_t)p->F4 * graph->m, 256) : 0;
    const size_t total = sE + sN + (size_t)p->nckpt * (sE + sN) + (size_t)(p->nseg + ntailbuf) * (sE + sN) + sE + sP + sW +
                         align_up((size_t)p->loss_blocks * sizeof(double), 256) + 2 * s4n + s4m;
    if (ce == cudaSuccess) ce = cudaMalloc(&p->buf, total);
    if (ce != cudaSuccess) {
        release(p);
        delete p;
        return cuda_status(ce);
    }
    char* b = (char*)p->buf;
    p->c2v_work = b; b += sE;
    p->app_work = b; b += sN;
    for (int i = 0; i < p->nckpt; ++i) { p->ck_c2v.push_back(b); b += sE; p->ck_app.push_back(b); b += sN; }
    for (int i = 0; i < p->nseg; ++i) { p->seg_c2v.push_back(b); b += sE; p->seg_app.push_back(b); b += sN; }
    for (int i = 0; i < ntailbuf; ++i) { p->tail_c2v.push_back(b); b += sE; p->tail_app.push_back(b); b += sN; }
    p->G = b; b += sE;
    p->pbuf = sP ? b : nullptr; b += sP;
    p->wpart = sW ? (double*)b : nullptr; b += sW;
    p->partial = (double*)b; b += align_up((size_t)p->loss_blocks * sizeof(double), 256);
    if (p->x4) {
        p->llr4 = (float*)b; b += s4n;
        p->grad4 = (float*)b; b += s4n;
        p->syn4 = (unsigned char*)b; b += s4m;
    }
    p->grid_cn = grid_for((long long)frames * graph->m, sms);
    p->grid_vn = grid_for((long long)frames * graph->n, sms);
    p->grid_w = std::min(n_classes, sms * 16);
    if (p->x4) {
        // the backward pass recomputes the next segment on a stream of its own while the current
        // segment's adjoint runs; without them it runs everything on the caller's stream
        const int segments = (iters + p->every - 1) / p->every;
        bool ok = cudaStreamCreateWithFlags(&p->s2, cudaStreamNonBlocking) == cudaSuccess;
        for (int i = 0; ok && i < 1 + 2 * segments; ++i) {
            cudaEvent_t e = nullptr;
            ok = cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
            if (ok) p->ev.push_back(e);
        }
        if (!ok) {
            for (cudaEvent_t e : p->ev) cudaEventDestroy(e);
            p->ev.clear();
            if (p->s2) cudaStreamDestroy(p->s2);
            p->s2 = nullptr;
            cudaGetLastError();
        }
    }
    *out = p;
    return LDPC_OK;
}

void ldpc_wbp_destroy(ldpc_wbp* p) {
    if (!p) return;
    DeviceGuard guard;
    guard.enter(p->device);
    release(p);
    delete p;
}

ldpc_status ldpc_wbp_forward(ldpc_wbp* p, const float* llr, const uint8_t* syndrome, const void* weights,
                             void* app_out, int32_t save_for_backward, void* cuda_stream) {
    NvtxRange nvtx("ldpc_wbp_forward");
    if (!p || !llr || !syndrome || !weights || !app_out) return LDPC_ERR_INVALID_ARG;
    DeviceGuard guard;
    LDPC_TRY(guard.enter(p->device));
    const bool save = save_for_backward != 0;
    ldpc_status st = dispatch(p, (cudaStream_t)cuda_stream, [&](auto r) {
        using T = std::remove_pointer_t<decltype(r.ck_c2v(0))>;
        return r.forward(llr, syndrome, (const T*)weights, (T*)app_out, save);
    });
    if (st == LDPC_OK && save) p->saved = true;
    return st;
}

ldpc_status ldpc_wbp_loss(ldpc_wbp* p, const void* app, const uint8_t* x, void* loss_out, void* grad_app,
                          void* cuda_stream) {
    NvtxRange nvtx("ldpc_wbp_loss");
    if (!p || !app || !x || !loss_out) return LDPC_ERR_INVALID_ARG;
    DeviceGuard guard;
    LDPC_TRY(guard.enter(p->device));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const long long total = (long long)p->F * p->n;
    const double scale = 1.0 / (double)total;
    if (p->fp64) {
        wbp::loss_kernel<double><<<p->loss_blocks, wbp::kThreads, 0, s>>>((const double*)app, x, total, scale,
                                                                          (double*)grad_app, p->partial);
        LDPC_TRY(cudaGetLastError());
        wbp::loss_final_kernel<double><<<1, wbp::kThreads, 0, s>>>(p->partial, p->loss_blocks, scale, (double*)loss_out);
    } else {
        wbp::loss_kernel<float><<<p->loss_blocks, wbp::kThreads, 0, s>>>((const float*)app, x, total, scale,
                                                                        (float*)grad_app, p->partial);
        LDPC_TRY(cudaGetLastError());
        wbp::loss_final_kernel<float><<<1, wbp::kThreads, 0, s>>>(p->partial, p->loss_blocks, scale, (float*)loss_out);
    }
    LDPC_TRY(cudaGetLastError());
    return LDPC_OK;
}

ldpc_status ldpc_wbp_backward(ldpc_wbp* p, const float* llr, const uint8_t* syndrome, const void* weights,
                              const void* grad_app, void* grad_weights, void* grad_llr, void* cuda_stream) {
    NvtxRange nvtx("ldpc_wbp_backward");
    if (!p || !llr || !syndrome || !weights || !grad_app || !grad_weights) return LDPC_ERR_INVALID_ARG;
    if ((p->nckpt > 0 || p->ntail > 0) && !p->saved) return LDPC_ERR_INVALID_ARG;
    DeviceGuard guard;
    LDPC_TRY(guard.enter(p->device));
    return dispatch(p, (cudaStream_t)cuda_stream, [&](auto r) {
        using T = std::remove_pointer_t<decltype(r.ck_c2v(0))>;
        return r.backward(llr, syndrome, (const T*)weights, (const T*)grad_app, (T*)grad_weights, (T*)grad_llr);
    });
}

ldpc_status ldpc_wbp_sgd_step(ldpc_wbp* p, void* weights, const void* grad, double lr, void* cuda_stream) {
    NvtxRange nvtx("ldpc_wbp_sgd_step");
    if (!p || !weights || !grad) return LDPC_ERR_INVALID_ARG;
    DeviceGuard guard;
    LDPC_TRY(guard.enter(p->device));
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int count = p->T * p->C;
    const int grid = std::max(1, std::min((count + 255) / 256, 1024));
    if (p->fp64)
        wbp::sgd_kernel<double><<<grid, 256, 0, s>>>((double*)weights, (const double*)grad, count, lr);
    else
        wbp::sgd_kernel<float><<<grid, 256, 0, s>>>((float*)weights, (const float*)grad, count, (float)lr);
    LDPC_TRY(cudaGetLastError());
    return LDPC_OK;
}

}  // extern "C"
