// Device code of weighted belief propagation: T unrolled flooding iterations
// of the sum-product decoder (paper, section "Early Termination": tanh/atanh
// check rule with the syndrome sign, a-posteriori values l_out) with one
// trainable weight per (iteration, edge class) scaling each check-to-variable
// message, a binary cross-entropy loss on the last iteration's soft output,
// and the hand-written adjoint (reverse-mode gradient) of the whole chain.
//
// Iteration k (1..T), edge e = (c, v), weights w_k:
//   u_e   = APP_v^(k-1) - c2v_e^(k-1)          (APP^(0) = Lch, c2v^(0) = 0)
//   a_e   = clamp(u_e, +-lmax)
//   t_e   = (1 - 2 s_c) * boxplus_{e' in N(c), e' != e} a_e'  (lmax at degree-1 checks)
//   c2v_e = w_k[class(e)] * t_e
//   APP_v = Lch_v + sum_{e in M(v)} c2v_e
//
// Adjoint of iteration k, given G_e = dloss/dc2v_e^(k):
//   dloss/dw_k[cl] = sum_{e in cl} G_e t_e                 (per-edge products, then a
//                                                          fixed-order reduction per class)
//   dt_e  = G_e w_k[class(e)]   (0 at degree-1 checks: their message is constant)
//   da_j  = (1 - 2 s_c) sum_{e != j} dt_e * d(a_j [+] B_ej)/da_j,  B_ej = boxplus of N(c) \ {e, j}
//   du_j  = da_j if |u_j| <= lmax else 0
//   dloss/dLch_v += S_v = sum_{e in M(v)} du_e;  G_e <- S_v - du_e  (= dloss/dc2v^(k-1))
//
// FP32: the boxplus derivative in the same r = exp(-|x|) domain as the check
// rule: d(a [+] B)/da = sgn(B) r_a (1 - r_B^2) / ((r_a + r_B)(1 + r_a r_B)),
// with r_B the r-domain combination of B's inputs (0 for an empty B, which
// gives the exact derivative 1 of a degree-2 check's copy).  FP64: the tanh
// form literally, (1 - tanh^2(a_j/2)) prod_{i != e,j} tanh(a_i/2) / (1 - P_e^2).
//
// Every kernel is one thread per (frame, check) or (frame, variable), with
// grid-stride loops; sums over a variable's edges run in ascending edge
// order and every reduction has a fixed order, so results are deterministic.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "cn_math.cuh"
#include "device_types.h"

namespace ldpcgb {
namespace wbp {

constexpr int kThreads = 256;

template <typename T>
struct Args {
    int F, m, n;
    long long E;
    T lmax;
    const float* llr;              // [F][n] channel LLRs
    const unsigned char* syn;      // [F][m] syndrome bytes (nonzero = 1)
    const T* w;                    // [C] weights of this iteration
    const int* cls;                // class of each key (QC: base block, CSR: edge)
    const T* c2v_prev;             // [F][E] c2v^(k-1), NULL in iteration 1
    const T* app_prev;             // [F][n] APP^(k-1), NULL in iteration 1 (then Lch)
    T* c2v_out;                    // [F][E] forward: c2v^(k)
    T* app_out;                    // [F][n] forward: APP^(k)
    T* G;                          // [F][E] adjoint state (see above)
    T* pbuf;                       // [F][E] per-edge G * t
    T* grad_llr;                   // [F][n] or NULL
    int vec;                       // QC variable side: 16-byte loads allowed (Z % 4 == 0, aligned buffers)
};

// ---- graph walks: check c -> (message slot, variable, class key) --------
struct QcCheck {
    int b0, d, t;
};
__device__ __forceinline__ QcCheck check_of(const QcDev& q, int c) {
    const int i = c / q.Z;
    QcCheck r;
    r.t = c - i * q.Z;
    r.b0 = __ldg(q.row_ptr + i);
    r.d = __ldg(q.row_ptr + i + 1) - r.b0;
    return r;
}
__device__ __forceinline__ void check_edge(const QcDev& q, const QcCheck& ck, int k, long long& slot, int& var,
                                           int& key) {
    const int b = ck.b0 + k;
    int p = ck.t + __ldg(q.blk_shift + b);
    if (p >= q.Z) p -= q.Z;
    slot = (long long)b * q.Z + p;
    var = __ldg(q.blk_col + b) * q.Z + p;
    key = b;
}
struct CsrCheck {
    int b0, d;
};
__device__ __forceinline__ CsrCheck check_of(const CsrDev& g, int c) {
    CsrCheck r;
    r.b0 = __ldg(g.row_ptr + c);
    r.d = __ldg(g.row_ptr + c + 1) - r.b0;
    return r;
}
__device__ __forceinline__ void check_edge(const CsrDev& g, const CsrCheck& ck, int k, long long& slot, int& var,
                                           int& key) {
    slot = ck.b0 + k;
    var = __ldg(g.col_idx + ck.b0 + k);
    key = ck.b0 + k;
}

// ---- variable v -> its message slots, ascending edge order --------------
struct VarWalk {
    int b0, d, p;
};
__device__ __forceinline__ VarWalk var_of(const QcDev& q, int v) {
    const int j = v / q.Z;
    VarWalk r;
    r.p = v - j * q.Z;
    r.b0 = __ldg(q.col_ptr + j);
    r.d = __ldg(q.col_ptr + j + 1) - r.b0;
    return r;
}
__device__ __forceinline__ long long var_slot(const QcDev& q, const VarWalk& vw, int k) {
    return (long long)__ldg(q.col_blk + vw.b0 + k) * q.Z + vw.p;
}
__device__ __forceinline__ VarWalk var_of(const CsrDev& g, int v) {
    VarWalk r;
    r.p = 0;
    r.b0 = __ldg(g.var_ptr + v);
    r.d = __ldg(g.var_ptr + v + 1) - r.b0;
    return r;
}
__device__ __forceinline__ long long var_slot(const CsrDev& g, const VarWalk& vw, int k) {
    return __ldg(g.var_edge + vw.b0 + k);
}

// ---- boxplus derivatives ------------------------------------------------
// d(a_j [+] B)/da_j for B = boxplus of inputs i not in {e, j}; FP32 r-domain.
template <int D>
__device__ __forceinline__ float dbox(const float (&r)[D], const bool (&ng)[D], int e, int j) {
    if constexpr (D == 2) return 1.0f;  // B is empty: a degree-2 check copies its other input
    float rb = 0.0f;
    bool neg = false;
    if constexpr (D == 3) {  // B is the one remaining input
        const int i = 3 - e - j;
        rb = r[i];
        neg = ng[i];
    } else {
#pragma unroll
        for (int i = 0; i < D; ++i) {
            if (i == e || i == j) continue;
            rb = rcomb(rb, r[i]);
            neg ^= ng[i];
        }
    }
    const float rj = r[j];
    const float val = __fdividef(rj * fmaf(-rb, rb, 1.0f), (rj + rb) * fmaf(rj, rb, 1.0f));
    return neg ? -val : val;
}
// FP64: the tanh form, as written.
template <int D>
__device__ __forceinline__ double dbox(const double (&th)[D], int e, int j) {
    double P = 1.0, rest = 1.0;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        if (i == e) continue;
        P *= th[i];
        if (i != j) rest *= th[i];
    }
    return (1.0 - th[j] * th[j]) * rest / (1.0 - P * P);
}

// ---- one check, compile-time degree D -----------------------------------
template <int D, bool BWD, typename T, class Code, class Ck>
__device__ __forceinline__ void check_d(const Args<T>& a, const Code& g, const Ck& ck, int f, int c) {
    long long slot[D];
    int var[D], key[D];
    T u[D], av[D], o[D];
    const size_t fe = (size_t)f * (size_t)a.E, fn = (size_t)f * (size_t)a.n;
#pragma unroll
    for (int k = 0; k < D; ++k) check_edge(g, ck, k, slot[k], var[k], key[k]);
#pragma unroll
    for (int k = 0; k < D; ++k) {
        u[k] = a.app_prev ? a.app_prev[fn + var[k]] - a.c2v_prev[fe + slot[k]] : (T)__ldg(a.llr + fn + var[k]);
        av[k] = clampm(u[k], a.lmax);
    }
    const unsigned sbit = __ldg(a.syn + (size_t)f * a.m + c) != 0 ? 1u : 0u;
    cn_core<D>(av, sbit, a.lmax, o);
    if constexpr (!BWD) {
#pragma unroll
        for (int k = 0; k < D; ++k) a.c2v_out[fe + slot[k]] = a.w[__ldg(a.cls + key[k])] * o[k];
    } else {
        T dt[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const T Gk = a.G[fe + slot[k]];
            a.pbuf[fe + slot[k]] = Gk * o[k];
            dt[k] = D == 1 ? T(0) : Gk * a.w[__ldg(a.cls + key[k])];
        }
        const T sg = sbit ? T(-1) : T(1);
        T da[D];
        if constexpr (D == 1) {
            da[0] = T(0);
        } else if constexpr (sizeof(T) == 4) {
            float r[D];
            bool ng[D];
#pragma unroll
            for (int k = 0; k < D; ++k) {
                r[k] = __expf(-fabsf(av[k]));
                ng[k] = av[k] < 0.0f;
            }
#pragma unroll
            for (int j = 0; j < D; ++j) {
                float s = 0.0f;
#pragma unroll
                for (int e = 0; e < D; ++e)
                    if (e != j) s = fmaf(dt[e], dbox<D>(r, ng, e, j), s);
                da[j] = sg * s;
            }
        } else {
            double th[D];
#pragma unroll
            for (int k = 0; k < D; ++k) th[k] = tanh(0.5 * av[k]);
#pragma unroll
            for (int j = 0; j < D; ++j) {
                double s = 0.0;
#pragma unroll
                for (int e = 0; e < D; ++e)
                    if (e != j) s += dt[e] * sg * dbox<D>(th, e, j);
                da[j] = s;
            }
        }
#pragma unroll
        for (int j = 0; j < D; ++j) a.G[fe + slot[j]] = absm(u[j]) <= a.lmax ? da[j] : T(0);
    }
}

// Degree > 6: the same with loops over local arrays (O(d^3) derivative).  With
// acc, the products G * t are added to acc[k] instead of being stored per edge.
template <bool BWD, typename T, class Code, class Ck>
__device__ __noinline__ void check_n(const Args<T>& a, const Code& g, const Ck& ck, int f, int c,
                                     double* acc = nullptr) {
    const int d = ck.d;
    long long slot[kMaxDeg];
    int key[kMaxDeg];
    T u[kMaxDeg], av[kMaxDeg], o[kMaxDeg];
    const size_t fe = (size_t)f * (size_t)a.E, fn = (size_t)f * (size_t)a.n;
    for (int k = 0; k < d; ++k) {
        int var;
        check_edge(g, ck, k, slot[k], var, key[k]);
        u[k] = a.app_prev ? a.app_prev[fn + var] - a.c2v_prev[fe + slot[k]] : (T)__ldg(a.llr + fn + var);
        av[k] = clampm(u[k], a.lmax);
    }
    const unsigned sbit = __ldg(a.syn + (size_t)f * a.m + c) != 0 ? 1u : 0u;
    cn_core_n(av, d, sbit, a.lmax, o);
    if constexpr (!BWD) {
        for (int k = 0; k < d; ++k) a.c2v_out[fe + slot[k]] = a.w[__ldg(a.cls + key[k])] * o[k];
    } else {
        T dt[kMaxDeg];
        for (int k = 0; k < d; ++k) {
            const T Gk = a.G[fe + slot[k]];
            if (acc)
                acc[k] += (double)(Gk * o[k]);
            else
                a.pbuf[fe + slot[k]] = Gk * o[k];
            dt[k] = Gk * a.w[__ldg(a.cls + key[k])];
        }
        const T sg = sbit ? T(-1) : T(1);
        for (int j = 0; j < d; ++j) {
            T s = T(0);
            for (int e = 0; e < d; ++e) {
                if (e == j) continue;
                T dv;
                if constexpr (sizeof(T) == 4) {
                    float rb = 0.0f;
                    bool neg = false;
                    for (int i = 0; i < d; ++i) {
                        if (i == e || i == j) continue;
                        rb = rcomb(rb, __expf(-fabsf(av[i])));
                        neg ^= av[i] < 0.0f;
                    }
                    const float rj = __expf(-fabsf(av[j]));
                    dv = __fdividef(rj * fmaf(-rb, rb, 1.0f), (rj + rb) * fmaf(rj, rb, 1.0f));
                    if (neg) dv = -dv;
                } else {
                    double P = 1.0, rest = 1.0;
                    for (int i = 0; i < d; ++i) {
                        if (i == e) continue;
                        const double ti = tanh(0.5 * av[i]);
                        P *= ti;
                        if (i != j) rest *= ti;
                    }
                    const double tj = tanh(0.5 * av[j]);
                    dv = (1.0 - tj * tj) * rest / (1.0 - P * P);
                }
                s += dt[e] * sg * dv;
            }
            o[j] = s;  // reuse o for da
        }
        for (int j = 0; j < d; ++j) a.G[fe + slot[j]] = absm(u[j]) <= a.lmax ? o[j] : T(0);
    }
}

// Check-node pass of iteration k over every (frame, check): forward (c2v^(k))
// or adjoint (du from G, and the per-edge products G * t).
template <bool BWD, typename T, class Code>
__global__ void __launch_bounds__(kThreads) cn_kernel(Args<T> a, Code g) {
    const long long total = (long long)a.F * a.m;
    for (long long id = (long long)blockIdx.x * kThreads + threadIdx.x; id < total;
         id += (long long)gridDim.x * kThreads) {
        const int f = (int)(id / a.m);
        const int c = (int)(id - (long long)f * a.m);
        const auto ck = check_of(g, c);
        switch (ck.d) {
            case 0: break;
            case 1: check_d<1, BWD>(a, g, ck, f, c); break;
            case 2: check_d<2, BWD>(a, g, ck, f, c); break;
            case 3: check_d<3, BWD>(a, g, ck, f, c); break;
            case 4: check_d<4, BWD>(a, g, ck, f, c); break;
            case 5: check_d<5, BWD>(a, g, ck, f, c); break;
            case 6: check_d<6, BWD>(a, g, ck, f, c); break;
            default: check_n<BWD>(a, g, ck, f, c); break;
        }
    }
}

// Variable-node pass, forward: APP^(k) = Lch + sum of c2v^(k) (ascending edge order).
template <typename T, class Code>
__global__ void __launch_bounds__(kThreads) vn_fwd_kernel(Args<T> a, Code g) {
    const long long total = (long long)a.F * a.n;
    for (long long id = (long long)blockIdx.x * kThreads + threadIdx.x; id < total;
         id += (long long)gridDim.x * kThreads) {
        const int f = (int)(id / a.n);
        const int v = (int)(id - (long long)f * a.n);
        const VarWalk vw = var_of(g, v);
        const T* c2v = a.c2v_out + (size_t)f * a.E;
        T s = (T)__ldg(a.llr + id);
        for (int k = 0; k < vw.d; ++k) s += c2v[var_slot(g, vw, k)];
        a.app_out[id] = s;
    }
}

// Variable-node pass, adjoint: S = sum of du over the variable's edges,
// dloss/dLch += S, and G_e = S - du_e (the gradient w.r.t. c2v^(k-1)).
template <typename T, class Code>
__global__ void __launch_bounds__(kThreads) vn_bwd_kernel(Args<T> a, Code g) {
    const long long total = (long long)a.F * a.n;
    for (long long id = (long long)blockIdx.x * kThreads + threadIdx.x; id < total;
         id += (long long)gridDim.x * kThreads) {
        const int f = (int)(id / a.n);
        const int v = (int)(id - (long long)f * a.n);
        const VarWalk vw = var_of(g, v);
        T* G = a.G + (size_t)f * a.E;
        T s = T(0);
        for (int k = 0; k < vw.d; ++k) s += G[var_slot(g, vw, k)];
        if (a.grad_llr) a.grad_llr[id] += s;
        for (int k = 0; k < vw.d; ++k) {
            const long long e = var_slot(g, vw, k);
            G[e] = s - G[e];
        }
    }
}

// Start of the adjoint: G_e = dloss/dAPP_v^(T) on every edge of v; dloss/dLch = the same.
template <typename T, class Code>
__global__ void __launch_bounds__(kThreads) seed_kernel(Args<T> a, Code g, const T* grad_app) {
    const long long total = (long long)a.F * a.n;
    for (long long id = (long long)blockIdx.x * kThreads + threadIdx.x; id < total;
         id += (long long)gridDim.x * kThreads) {
        const int f = (int)(id / a.n);
        const int v = (int)(id - (long long)f * a.n);
        const VarWalk vw = var_of(g, v);
        const T gv = grad_app[id];
        if (a.grad_llr) a.grad_llr[id] = gv;
        T* G = a.G + (size_t)f * a.E;
        for (int k = 0; k < vw.d; ++k) G[var_slot(g, vw, k)] = gv;
    }
}

// Fixed-order block sum of one double per thread (result in thread 0).
__device__ __forceinline__ double block_sum(double v, double* sm) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sm[warp] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sm[i];
    return s;
}

// dloss/dw_k[cl] = sum over frames and the class's message slots of G * t
// (one CTA per class, grid-stride over classes; FP64 accumulation, fixed order).
template <typename T>
__global__ void __launch_bounds__(kThreads) wgrad_kernel(const T* pbuf, int F, long long E, const int* class_ptr,
                                                         const int* class_slot, int C, T* gw) {
    __shared__ double sm[kThreads / 32];
    for (int c = blockIdx.x; c < C; c += gridDim.x) {
        const int lo = __ldg(class_ptr + c), cnt = __ldg(class_ptr + c + 1) - lo;
        const long long total = (long long)F * cnt;
        double acc = 0.0;
        for (long long i = threadIdx.x; i < total; i += kThreads) {
            const int f = (int)(i / cnt);
            const int q = (int)(i - (long long)f * cnt);
            acc += (double)pbuf[(size_t)f * E + __ldg(class_slot + lo + q)];
        }
        const double s = block_sum(acc, sm);
        if (threadIdx.x == 0) gw[c] = (T)s;
    }
}

// Binary cross-entropy of the soft output against the bits x, mean over all
// F*n bits: loss = scale * sum softplus(-(1 - 2x) APP), and its gradient
// dloss/dAPP = -(1 - 2x) sigmoid(-(1 - 2x) APP) * scale.  Per-CTA partial
// sums (FP64, fixed order); loss_final_kernel adds them in order.
__device__ __forceinline__ float softplus_t(float z) { return fmaxf(z, 0.0f) + log1pf(__expf(-fabsf(z))); }
__device__ __forceinline__ double softplus_t(double z) { return fmax(z, 0.0) + log1p(exp(-fabs(z))); }
__device__ __forceinline__ float sigmoid_t(float z) {
    const float e = __expf(-fabsf(z));
    return z >= 0.0f ? __fdividef(1.0f, 1.0f + e) : __fdividef(e, 1.0f + e);
}
__device__ __forceinline__ double sigmoid_t(double z) {
    const double e = exp(-fabs(z));
    return z >= 0.0 ? 1.0 / (1.0 + e) : e / (1.0 + e);
}

template <typename T>
__global__ void __launch_bounds__(kThreads) loss_kernel(const T* app, const unsigned char* x, long long total,
                                                        double scale, T* grad_app, double* partial) {
    __shared__ double sm[kThreads / 32];
    // each thread sums its elements in the plan's type and widens once: FP64
    // additions are scarce on this part, and the FP32 loss is a diagnostic (the
    // gradient below does not depend on it)
    T acc = T(0);
    for (long long id = (long long)blockIdx.x * kThreads + threadIdx.x; id < total;
         id += (long long)gridDim.x * kThreads) {
        const T sx = __ldg(x + id) ? T(-1) : T(1);
        const T z = -sx * app[id];
        acc += softplus_t(z);
        if (grad_app) grad_app[id] = -sx * sigmoid_t(z) * (T)scale;
    }
    const double s = block_sum((double)acc, sm);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// One CTA of kThreads: thread t adds partials t, t + kThreads, ... in order,
// then a fixed-order block sum.
template <typename T>
__global__ void __launch_bounds__(kThreads) loss_final_kernel(const double* partial, int count, double scale,
                                                              T* loss_out) {
    __shared__ double sm[kThreads / 32];
    double s = 0.0;
    for (int i = threadIdx.x; i < count; i += kThreads) s += partial[i];
    s = block_sum(s, sm);
    if (threadIdx.x == 0) *loss_out = (T)(s * scale);
}

// Plain gradient step on the weights: w -= lr * g.
template <typename T>
__global__ void sgd_kernel(T* w, const T* g, int count, T lr) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) w[i] -= lr * g[i];
}

// ---------------------------------------------------------------------------
// Quasi-cyclic kernels.  Work is split by base row (check side) or base
// column (variable side) and by groups of `fpc` consecutive frames: a CTA
// reads its row's or column's block table once and then streams through the
// group's frames, so the dependent table loads are paid once per fpc frames
// and every thread keeps a steady stream of independent loads in flight.
//
// Check side: a CTA covers kQcCnTile consecutive checks t of base row i (tile)
// for each frame of its group, one check per thread per frame; the latency of
// the gathers is hidden by many resident warps (see the launch bounds).
// In the adjoint it also sums G * t per block over its checks and frames (per
// thread in the plan's type, frames in ascending order, then a fixed-order
// FP64 block reduction) into wpart[(g * nblk + b) * tiles + tile], g the frame
// group; class_reduce_kernel adds those up per class.
//
// Variable side: the group's (frame, variable) pairs of base column j are
// walked four at a time per thread, as 16-byte vectors when a.vec is set
// (message blocks are stored unrotated, so a column's messages are
// contiguous; Z % 4 == 0 keeps four consecutive variables in one frame).
// ---------------------------------------------------------------------------
constexpr int kQcCnTile = kThreads;

// One frame's inputs to one check of degree D: x = APP^(k-1) (Lch in
// iteration 1), c = c2v^(k-1) (0 in iteration 1), G (adjoint) and the
// syndrome bit.  ia / im: the check's APP index and message slot in a frame.
template <int D, typename T>
struct CnIn {
    T x[D], c[D], G[D];
    unsigned sb;
};

template <int D, bool BWD, typename T>
__device__ __forceinline__ void qc_cn_load(const Args<T>& a, int f, const int (&ia)[D], const int (&im)[D],
                                           const unsigned char* syn_t, CnIn<D, T>& in) {
    // frame base pointers, then 32-bit offsets within the frame
    const size_t fe = (size_t)f * (size_t)a.E, fn = (size_t)f * (size_t)a.n;
    if (a.app_prev) {
        const T* xf = a.app_prev + fn;
        const T* cf = a.c2v_prev + fe;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            in.x[k] = xf[ia[k]];
            in.c[k] = cf[im[k]];
        }
    } else {
        const float* lf = a.llr + fn;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            in.x[k] = (T)__ldg(lf + ia[k]);
            in.c[k] = T(0);
        }
    }
    if constexpr (BWD) {
        const T* gf = a.G + fe;
#pragma unroll
        for (int k = 0; k < D; ++k) in.G[k] = gf[im[k]];
    }
    in.sb = __ldg(syn_t + (size_t)f * (size_t)a.m) != 0 ? 1u : 0u;
}

template <int D, bool BWD, typename T>
__device__ __forceinline__ void qc_cn_frame(const Args<T>& a, int f, const int (&im)[D], const T (&wk)[D],
                                            const CnIn<D, T>& in, T (&acc)[D]) {
    const size_t fe = (size_t)f * (size_t)a.E;
    T u[D], av[D], o[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        u[k] = in.x[k] - in.c[k];  // x - 0 == x exactly in iteration 1
        av[k] = clampm(u[k], a.lmax);
    }
    cn_core<D>(av, in.sb, a.lmax, o);
    if constexpr (!BWD) {
        T* of = a.c2v_out + fe;
#pragma unroll
        for (int k = 0; k < D; ++k) of[im[k]] = wk[k] * o[k];
    } else {
        T dt[D], da[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            acc[k] += in.G[k] * o[k];
            dt[k] = D == 1 ? T(0) : in.G[k] * wk[k];
        }
    const T sg = in.sb ? T(-1) : T(1);
        if constexpr (D == 1) {
            da[0] = T(0);
        } else if constexpr (sizeof(T) == 4) {
            float rr[D];
            bool ng[D];
#pragma unroll
            for (int k = 0; k < D; ++k) {
                rr[k] = __expf(-fabsf(av[k]));
                ng[k] = av[k] < 0.0f;
            }
#pragma unroll
            for (int j = 0; j < D; ++j) {
                float s = 0.0f;
#pragma unroll
                for (int e = 0; e < D; ++e)
                    if (e != j) s = fmaf(dt[e], dbox<D>(rr, ng, e, j), s);
                da[j] = sg * s;
            }
        } else {
            double th[D];
#pragma unroll
            for (int k = 0; k < D; ++k) th[k] = tanh(0.5 * av[k]);
#pragma unroll
            for (int j = 0; j < D; ++j) {
                double s = 0.0;
#pragma unroll
                for (int e = 0; e < D; ++e)
                    if (e != j) s += dt[e] * sg * dbox<D>(th, e, j);
                da[j] = s;
            }
        }
        T* gf = a.G + fe;
#pragma unroll
        for (int j = 0; j < D; ++j) gf[im[j]] = absm(u[j]) <= a.lmax ? da[j] : T(0);
    }
}

template <int D, bool BWD, typename T>
__device__ __forceinline__ void qc_cn_rows(const Args<T>& a, const QcDev& q, int g, int fpc, int i, int tile, int b0,
                                           double* wpart, int tiles, double* sm) {
    const int Z = q.Z;
    const int t = tile * kQcCnTile + (int)threadIdx.x;
    int ia[D], im[D];
    T wk[D], acc[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        int p = t + __ldg(q.blk_shift + b0 + k);
        if (p >= Z) p -= Z;
        ia[k] = __ldg(q.blk_col + b0 + k) * Z + p;
        im[k] = (b0 + k) * Z + p;
        wk[k] = a.w[__ldg(a.cls + b0 + k)];
        acc[k] = T(0);
    }
    const unsigned char* syn_t = a.syn + ((size_t)i * Z + t);  // frame 0's byte of check (i, t)
    const int f0 = g * fpc, f_end = min(a.F, f0 + fpc);
    if (t < Z && f0 < f_end) {
        // one frame at a time: with 5-8 resident CTAs per SM, loading frame
        // f + 1 ahead of frame f's arithmetic (more registers, more spills) was
        // slower; it paid only at 4 CTAs per SM
        CnIn<D, T> in;
        for (int f = f0; f < f_end; ++f) {
            qc_cn_load<D, BWD>(a, f, ia, im, syn_t, in);
            qc_cn_frame<D, BWD>(a, f, im, wk, in, acc);
        }
    }
    if constexpr (BWD) {
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const double s = block_sum((double)acc[k], sm);
            if (threadIdx.x == 0) wpart[((size_t)g * q.nblk + b0 + k) * tiles + tile] = s;
        }
    }
}

// Rows of weight > 4: each thread runs the generic check for its checks (a
// local copy of the arguments keeps the hot paths free of it).
template <bool BWD, typename T>
__device__ __noinline__ void qc_cn_rows_n(const Args<T> a, const QcDev q, int g, int fpc, int i, int tile, int b0,
                                          int d, double* wpart, int tiles, double* sm) {
    double acc[kMaxDeg];
    for (int k = 0; k < d; ++k) acc[k] = 0.0;
    const int f_end = min(a.F, (g + 1) * fpc);
    for (int f = g * fpc; f < f_end; ++f) {
        const int t = tile * kQcCnTile + (int)threadIdx.x;
        if (t >= q.Z) continue;
        QcCheck ck;
        ck.b0 = b0;
        ck.d = d;
        ck.t = t;
        check_n<BWD>(a, q, ck, f, i * q.Z + t, BWD ? acc : nullptr);
    }
    if constexpr (BWD) {
        for (int k = 0; k < d; ++k) {
            const double s = block_sum(acc[k], sm);
            if (threadIdx.x == 0) wpart[((size_t)g * q.nblk + b0 + k) * tiles + tile] = s;
        }
    }
}

// Occupancy over registers: these passes are bound by the latency of their
// gathers, so more resident warps pay more than spill-free code, up to the
// point where spill traffic (local loads wait like gathers) eats the gain.
// Measured on the n = 65536, 128-frame training step: 4 CTAs per SM for both
// passes (64 registers, adjoint loading one frame ahead) 5.80 ms; forward at
// 8 CTAs per SM (32 registers) with the adjoint at 6 (40 registers) 5.33 ms;
// adjoint one frame at a time at 5 (48 registers, 68 bytes of spills)
// 4.73 ms, at 6 (40 registers, 128 bytes) 5.21 ms, at 8 5.50 ms.  FP64 plans
// (the parity mode) keep 4 CTAs per SM.
template <bool BWD, typename T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? (BWD ? 5 : 8) : 4) qc_cn_kernel(Args<T> a, QcDev q, int tiles, int fpc, double* wpart) {
    __shared__ double sm[kThreads / 32];
    const int groups = (a.F + fpc - 1) / fpc;
    const long long total = (long long)groups * q.mb * tiles;
    for (long long blk = blockIdx.x; blk < total; blk += gridDim.x) {
        // row-major over (row, tile), frame groups innermost: CTAs that run
        // together share the row's table and read neighbouring frames
        // (32-bit division where the index fits: the 64-bit one is a long routine)
        int g, i, tile;
        if (total <= 0x7fffffffLL) {
            const int b = (int)blk, rt = b / groups;
            g = b - rt * groups;
            i = rt / tiles;
            tile = rt - i * tiles;
        } else {
            const long long rt = blk / groups;
            g = (int)(blk - rt * groups);
            i = (int)(rt / tiles);
            tile = (int)(rt - (long long)i * tiles);
        }
        const int b0 = __ldg(q.row_ptr + i), d = __ldg(q.row_ptr + i + 1) - b0;
        switch (d) {
            case 0: break;
            case 1: qc_cn_rows<1, BWD>(a, q, g, fpc, i, tile, b0, wpart, tiles, sm); break;
            case 2: qc_cn_rows<2, BWD>(a, q, g, fpc, i, tile, b0, wpart, tiles, sm); break;
            case 3: qc_cn_rows<3, BWD>(a, q, g, fpc, i, tile, b0, wpart, tiles, sm); break;
            case 4: qc_cn_rows<4, BWD>(a, q, g, fpc, i, tile, b0, wpart, tiles, sm); break;
            default: qc_cn_rows_n<BWD>(a, q, g, fpc, i, tile, b0, d, wpart, tiles, sm); break;
        }
    }
}

// Variable side.  MODE kVnFwd: APP = Lch + sum of c2v (ascending row order);
// kVnBwd: S = sum du, dloss/dLch += S, G = S - du; kVnSeed: G = dloss/dAPP on
// every edge, dloss/dLch = dloss/dAPP.
enum : int { kVnFwd = 0, kVnBwd = 1, kVnSeed = 2 };

template <int MODE, int DV, typename T>
__device__ __forceinline__ void qc_vn_one(const Args<T>& a, const QcDev& q, size_t fe, size_t vi, int p,
                                          const int (&blk)[DV > 0 ? DV : 1], int cb0, int dv, const T* grad_app) {
    constexpr bool kFixed = DV > 0;
    const int nd = kFixed ? DV : dv;
    auto slot = [&](int b) -> size_t {
        if constexpr (kFixed) return fe + (size_t)blk[b] * q.Z + p;
        else return fe + (size_t)__ldg(q.col_blk + cb0 + b) * q.Z + p;
    };
    if constexpr (MODE == kVnFwd) {
        T s = (T)__ldg(a.llr + vi);
        for (int b = 0; b < nd; ++b) s += a.c2v_out[slot(b)];
        a.app_out[vi] = s;
    } else if constexpr (MODE == kVnBwd) {
        T s = T(0);
        for (int b = 0; b < nd; ++b) s += a.G[slot(b)];
        if (a.grad_llr) a.grad_llr[vi] += s;
        for (int b = 0; b < nd; ++b) {
            T* gp = a.G + slot(b);
            *gp = s - *gp;
        }
    } else {
        const T gv = grad_app[vi];
        if (a.grad_llr) a.grad_llr[vi] = gv;
        for (int b = 0; b < nd; ++b) a.G[slot(b)] = gv;
    }
}

template <int MODE, int DV>
__device__ __forceinline__ void qc_vn_vec(const Args<float>& a, const QcDev& q, size_t fe, size_t vi, int p,
                                          const int (&blk)[DV], const float* grad_app) {
    size_t mb[DV];
#pragma unroll
    for (int b = 0; b < DV; ++b) mb[b] = fe + (size_t)blk[b] * q.Z + p;
    if constexpr (MODE == kVnFwd) {
        float4 s = __ldg(reinterpret_cast<const float4*>(a.llr + vi));
        float4 m[DV];
#pragma unroll
        for (int b = 0; b < DV; ++b) m[b] = *reinterpret_cast<const float4*>(a.c2v_out + mb[b]);
#pragma unroll
        for (int b = 0; b < DV; ++b) {
            s.x += m[b].x;
            s.y += m[b].y;
            s.z += m[b].z;
            s.w += m[b].w;
        }
        *reinterpret_cast<float4*>(a.app_out + vi) = s;
    } else if constexpr (MODE == kVnBwd) {
        float4 m[DV];
#pragma unroll
        for (int b = 0; b < DV; ++b) m[b] = *reinterpret_cast<const float4*>(a.G + mb[b]);
        float4 s = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
        for (int b = 0; b < DV; ++b) {
            s.x += m[b].x;
            s.y += m[b].y;
            s.z += m[b].z;
            s.w += m[b].w;
        }
        if (a.grad_llr) {
            float4* gl = reinterpret_cast<float4*>(a.grad_llr + vi);
            float4 v = *gl;
            v.x += s.x;
            v.y += s.y;
            v.z += s.z;
            v.w += s.w;
            *gl = v;
        }
#pragma unroll
        for (int b = 0; b < DV; ++b)
            *reinterpret_cast<float4*>(a.G + mb[b]) =
                make_float4(s.x - m[b].x, s.y - m[b].y, s.z - m[b].z, s.w - m[b].w);
    } else {
        const float4 gv = *reinterpret_cast<const float4*>(grad_app + vi);
        if (a.grad_llr) *reinterpret_cast<float4*>(a.grad_llr + vi) = gv;
#pragma unroll
        for (int b = 0; b < DV; ++b) *reinterpret_cast<float4*>(a.G + mb[b]) = gv;
    }
}

template <int MODE, int DV, typename T>
__device__ __forceinline__ void qc_vn_cols(const Args<T>& a, const QcDev& q, int g, int fpc, int j, int cb0, int dv,
                                           const T* grad_app) {
    const int Z = q.Z;
    int blk[DV > 0 ? DV : 1];
    if constexpr (DV > 0) {
#pragma unroll
        for (int b = 0; b < DV; ++b) blk[b] = __ldg(q.col_blk + cb0 + b);
    }
    const int f0 = g * fpc, nf = min(a.F, f0 + fpc) - f0;
    const int count = nf * Z;  // (frame, variable) pairs of the group in column j
    for (int idx = 4 * (int)threadIdx.x; idx < count; idx += 4 * kThreads) {
        const int fl = idx / Z, p = idx - fl * Z;
        const size_t fe = (size_t)(f0 + fl) * (size_t)a.E, fn = (size_t)(f0 + fl) * (size_t)a.n;
        const size_t vi = fn + (size_t)j * Z + p;
        if constexpr (sizeof(T) == 4 && DV > 0) {
            if (a.vec) {  // Z % 4 == 0: the four variables are p .. p + 3 of one frame
                qc_vn_vec<MODE, DV>(a, q, fe, vi, p, blk, grad_app);
                continue;
            }
        }
        for (int e = 0; e < 4 && idx + e < count; ++e) {
            const int fe2 = (idx + e) / Z, pe = (idx + e) - fe2 * Z;
            qc_vn_one<MODE, DV, T>(a, q, (size_t)(f0 + fe2) * (size_t)a.E,
                                   (size_t)(f0 + fe2) * (size_t)a.n + (size_t)j * Z + pe, pe, blk, cb0, dv, grad_app);
        }
    }
}

// 6 CTAs per SM (40 registers) for FP32: 5.29 -> 5.15 ms per training step at
// n = 65536 x 128 frames (8 per SM: 5.23 ms).
template <int MODE, typename T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 6 : 1) qc_vn_kernel(Args<T> a, QcDev q, int fpc, const T* grad_app) {
    const int groups = (a.F + fpc - 1) / fpc;
    const long long total = (long long)groups * q.nb;
    for (long long blk = blockIdx.x; blk < total; blk += gridDim.x) {
        const int g = (int)(blk % groups), j = (int)(blk / groups);
        const int cb0 = __ldg(q.col_ptr + j), dv = __ldg(q.col_ptr + j + 1) - cb0;
        switch (dv) {
            case 1: qc_vn_cols<MODE, 1, T>(a, q, g, fpc, j, cb0, 1, grad_app); break;
            case 2: qc_vn_cols<MODE, 2, T>(a, q, g, fpc, j, cb0, 2, grad_app); break;
            case 3: qc_vn_cols<MODE, 3, T>(a, q, g, fpc, j, cb0, 3, grad_app); break;
            case 4: qc_vn_cols<MODE, 4, T>(a, q, g, fpc, j, cb0, 4, grad_app); break;
            default: qc_vn_cols<MODE, 0, T>(a, q, g, fpc, j, cb0, dv, grad_app); break;
        }
    }
}

// dloss/dw_k[cl] = sum over the class's blocks b, the frame groups g and the
// tiles of wpart (one CTA per iteration and class, grid-stride, fixed order).
template <typename T>
__global__ void __launch_bounds__(kThreads) class_reduce_kernel(const double* wpart, size_t per, int groups,
                                                                int nblk, int tiles, const int* cblk_ptr,
                                                                const int* cblk, int C, int iters, T* gw) {
    // one CTA per (iteration, class); iteration it's partials start at wpart + it * per
    __shared__ double sm[kThreads / 32];
    for (int ic = blockIdx.x; ic < iters * C; ic += gridDim.x) {
        const int it = ic / C, c = ic - it * C;
        const double* wp = wpart + (size_t)it * per;
        const int lo = __ldg(cblk_ptr + c), nbk = __ldg(cblk_ptr + c + 1) - lo;
        const long long per_g = (long long)nbk * tiles;
        const long long total = (long long)groups * per_g;
        double acc = 0.0;
        for (long long i = threadIdx.x; i < total; i += kThreads) {
            const int g = (int)(i / per_g);
            const int r = (int)(i - (long long)g * per_g);
            const int bi = r / tiles, tile = r - bi * tiles;
            acc += wp[((size_t)g * nblk + __ldg(cblk + lo + bi)) * tiles + tile];
        }
        const double s = block_sum(acc, sm);
        if (threadIdx.x == 0) gw[(size_t)it * C + c] = (T)s;
    }
}

// ---------------------------------------------------------------------------
// Four-frame interleaved QC kernels (FP32 plans).  A plan's own state -- c2v,
// APP, their checkpoints, the adjoint state G, an interleaved copy of Lch and
// the accumulated dloss/dLch -- is stored by frame quads: element (f, e) at
// ((f / 4) * E + e) * 4 + f % 4.  A thread then moves the four frames of one
// message with one 16-byte access and one address computation.  The caller's
// buffers stay frame-major; pack4_kernel / unpack4_kernel convert at the
// plan's edges (frames past F are zero: they add exact zeros everywhere).
// Each frame's arithmetic, and every sum's order over blocks and frames, is
// the one of the frame-major kernels above.
// ---------------------------------------------------------------------------
struct Args4 {
    int F, F4, m, n;
    long long E;
    float lmax;
    const float4* llr4;            // [F4][n] interleaved Lch
    const unsigned char* syn4;     // [F4][m] bit f of byte (q, c): syndrome of frame 4q + f at check c
    const float* w;                // [C] weights of this iteration
    const int* cls;                // class of each base block
    const float4* c2v_prev;        // [F4][E] c2v^(k-1), NULL in iteration 1
    const float4* app_prev;        // [F4][n] APP^(k-1), NULL in iteration 1 (then Lch)
    float4* c2v_out;               // [F4][E]
    float4* app_out;               // [F4][n] (NULL: only app_rows)
    float* app_rows;               // [F][n] frame-major APP output of the last iteration, or NULL
    float4* G;                     // [F4][E]
    float4* grad4;                 // [F4][n] accumulated dloss/dLch, or NULL
    const float* grad_app;         // [F][n] frame-major dloss/dAPP (seed pass)
};

__device__ __forceinline__ float f4get(const float4& v, int f) {
    return f == 0 ? v.x : (f == 1 ? v.y : (f == 2 ? v.z : v.w));
}
__device__ __forceinline__ void f4set(float4& v, int f, float x) {
    if (f == 0) v.x = x;
    else if (f == 1) v.y = x;
    else if (f == 2) v.z = x;
    else v.w = x;
}

// Interleave the caller's Lch and syndrome bytes of every frame quad.
__global__ void __launch_bounds__(kThreads) pack4_kernel(const float* llr, const unsigned char* syn, int F, int F4,
                                                         int n, int m, float4* llr4, unsigned char* syn4) {
    const long long tn = (long long)F4 * n, tm = (long long)F4 * m;
    for (long long id = (long long)blockIdx.x * kThreads + threadIdx.x; id < tn + tm;
         id += (long long)gridDim.x * kThreads) {
        if (id < tn) {
            const int q = (int)(id / n), v = (int)(id - (long long)q * n);
            float4 x = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll
            for (int f = 0; f < 4; ++f)
                if (4 * q + f < F) f4set(x, f, __ldg(llr + (size_t)(4 * q + f) * n + v));
            llr4[id] = x;
        } else {
            const long long j = id - tn;
            const int q = (int)(j / m), c = (int)(j - (long long)q * m);
            unsigned b = 0;
#pragma unroll
            for (int f = 0; f < 4; ++f)
                if (4 * q + f < F && __ldg(syn + (size_t)(4 * q + f) * m + c) != 0) b |= 1u << f;
            syn4[j] = (unsigned char)b;
        }
    }
}

// Frame-major copy of an interleaved [F4][n] array (frames < F).
__global__ void __launch_bounds__(kThreads) unpack4_kernel(const float4* src, int F, int n, float* dst) {
    const long long total = (long long)F * n;
    for (long long id = (long long)blockIdx.x * kThreads + threadIdx.x; id < total;
         id += (long long)gridDim.x * kThreads) {
        const int f = (int)(id / n), v = (int)(id - (long long)f * n);
        dst[id] = f4get(src[(size_t)(f >> 2) * n + v], f & 3);
    }
}

// One check of degree D for the four frames of quad q: the frame-major
// kernel's per-frame arithmetic (qc_cn_frame), four times.
template <int D, bool BWD>
__device__ __forceinline__ void qc_cn4_quad(const Args4& a, int q, const int (&ia)[D], const int (&im)[D],
                                            const float (&wk)[D], int c_global, float (&acc)[D]) {
    const size_t qe = (size_t)q * (size_t)a.E, qn = (size_t)q * (size_t)a.n;
    float4 x[D], cv[D], G[D];
    if (a.app_prev) {
#pragma unroll
        for (int k = 0; k < D; ++k) {
            x[k] = a.app_prev[qn + ia[k]];
            cv[k] = a.c2v_prev[qe + im[k]];
        }
    } else {
#pragma unroll
        for (int k = 0; k < D; ++k) {
            x[k] = __ldg(a.llr4 + qn + ia[k]);
            cv[k] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
    }
    if constexpr (BWD) {
#pragma unroll
        for (int k = 0; k < D; ++k) G[k] = a.G[qe + im[k]];
    }
    const unsigned sb4 = __ldg(a.syn4 + (size_t)q * a.m + c_global);
    float4 out[D];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
        const unsigned sb = (sb4 >> f) & 1u;
        float u[D], av[D], o[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            u[k] = f4get(x[k], f) - f4get(cv[k], f);
            av[k] = clampm(u[k], a.lmax);
        }
        cn_core<D>(av, sb, a.lmax, o);
        if constexpr (!BWD) {
#pragma unroll
            for (int k = 0; k < D; ++k) f4set(out[k], f, wk[k] * o[k]);
        } else {
            float dt[D], da[D];
#pragma unroll
            for (int k = 0; k < D; ++k) {
                const float Gk = f4get(G[k], f);
                acc[k] += Gk * o[k];
                dt[k] = D == 1 ? 0.0f : Gk * wk[k];
            }
            const float sg = sb ? -1.0f : 1.0f;
            if constexpr (D == 1) {
                da[0] = 0.0f;
            } else {
                float rr[D];
                bool ng[D];
#pragma unroll
                for (int k = 0; k < D; ++k) {
                    rr[k] = __expf(-fabsf(av[k]));
                    ng[k] = av[k] < 0.0f;
                }
#pragma unroll
                for (int j = 0; j < D; ++j) {
                    float s = 0.0f;
#pragma unroll
                    for (int e = 0; e < D; ++e)
                        if (e != j) s = fmaf(dt[e], dbox<D>(rr, ng, e, j), s);
                    da[j] = sg * s;
                }
            }
#pragma unroll
            for (int j = 0; j < D; ++j) f4set(out[j], f, fabsf(u[j]) <= a.lmax ? da[j] : 0.0f);
        }
    }
    float4* dst = BWD ? a.G + qe : a.c2v_out + qe;
#pragma unroll
    for (int k = 0; k < D; ++k) dst[im[k]] = out[k];
}

// Rows of weight > 4: per frame of the quad, scalar loads from the
// interleaved arrays and the generic check (as check_n), FP64 sums of G * t.
template <bool BWD>
__device__ __noinline__ void qc_cn4_quad_n(const Args4 a, const QcDev q, int qd, int i, int t, int b0, int d,
                                           double* acc) {
    const int Z = q.Z;
    const size_t qe = (size_t)qd * (size_t)a.E, qn = (size_t)qd * (size_t)a.n;
    const float* xs = a.app_prev ? (const float*)a.app_prev : (const float*)a.llr4;
    const float* cs = (const float*)a.c2v_prev;
    float* gs = (float*)a.G;
    float* os = (float*)a.c2v_out;
    const unsigned sb4 = __ldg(a.syn4 + (size_t)qd * a.m + (size_t)i * Z + t);
    for (int f = 0; f < 4; ++f) {
        int slot[kMaxDeg];
        float u[kMaxDeg], av[kMaxDeg], o[kMaxDeg];
        for (int k = 0; k < d; ++k) {
            int p = t + __ldg(q.blk_shift + b0 + k);
            if (p >= Z) p -= Z;
            const size_t iv = qn + (size_t)__ldg(q.blk_col + b0 + k) * Z + p;
            slot[k] = (b0 + k) * Z + p;
            const float xv = xs[iv * 4 + f];
            const float cv = a.app_prev ? cs[(qe + slot[k]) * 4 + f] : 0.0f;
            u[k] = xv - cv;
            av[k] = clampm(u[k], a.lmax);
        }
        const unsigned sb = (sb4 >> f) & 1u;
        cn_core_n(av, d, sb, a.lmax, o);
        if constexpr (!BWD) {
            for (int k = 0; k < d; ++k) os[(qe + slot[k]) * 4 + f] = a.w[__ldg(a.cls + b0 + k)] * o[k];
        } else {
            float dt[kMaxDeg];
            for (int k = 0; k < d; ++k) {
                const float Gk = gs[(qe + slot[k]) * 4 + f];
                acc[k] += (double)(Gk * o[k]);
                dt[k] = Gk * a.w[__ldg(a.cls + b0 + k)];
            }
            const float sg = sb ? -1.0f : 1.0f;
            for (int j = 0; j < d; ++j) {
                float sum = 0.0f;
                for (int e = 0; e < d; ++e) {
                    if (e == j) continue;
                    float rb = 0.0f;
                    bool neg = false;
                    for (int r = 0; r < d; ++r) {
                        if (r == e || r == j) continue;
                        rb = rcomb(rb, __expf(-fabsf(av[r])));
                        neg ^= av[r] < 0.0f;
                    }
                    const float rj = __expf(-fabsf(av[j]));
                    float dv = __fdividef(rj * fmaf(-rb, rb, 1.0f), (rj + rb) * fmaf(rj, rb, 1.0f));
                    if (neg) dv = -dv;
                    sum += dt[e] * sg * dv;
                }
                o[j] = sum;  // reuse o for da
            }
            for (int j = 0; j < d; ++j) gs[(qe + slot[j]) * 4 + f] = fabsf(u[j]) <= a.lmax ? o[j] : 0.0f;
        }
    }
}

// Check tile of base row i for the quads of group g (one check per thread,
// quads in ascending order), and in the adjoint the tile's sums of G * t per
// block into wpart[(g * nblk + b) * tiles + tile] (fixed order).
template <int D, bool BWD>
__device__ __forceinline__ void qc_cn4_rows(const Args4& a, const QcDev& q, int g, int fpq, int i, int tile, int b0,
                                            double* wpart, int tiles, double* sm) {
    const int Z = q.Z;
    const int t = tile * kQcCnTile + (int)threadIdx.x;
    int ia[D], im[D];
    float wk[D], acc[D];
#pragma unroll
    for (int k = 0; k < D; ++k) {
        int p = t + __ldg(q.blk_shift + b0 + k);
        if (p >= Z) p -= Z;
        ia[k] = __ldg(q.blk_col + b0 + k) * Z + p;
        im[k] = (b0 + k) * Z + p;
        wk[k] = a.w[__ldg(a.cls + b0 + k)];
        acc[k] = 0.0f;
    }
    const int q0 = g * fpq, q_end = min(a.F4, q0 + fpq);
    if (t < Z)
        for (int qd = q0; qd < q_end; ++qd) qc_cn4_quad<D, BWD>(a, qd, ia, im, wk, i * Z + t, acc);
    if constexpr (BWD) {
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const double s = block_sum((double)acc[k], sm);
            if (threadIdx.x == 0) wpart[((size_t)g * q.nblk + b0 + k) * tiles + tile] = s;
        }
    }
}

template <bool BWD>
__device__ __noinline__ void qc_cn4_rows_n(const Args4 a, const QcDev q, int g, int fpq, int i, int tile, int b0,
                                           int d, double* wpart, int tiles, double* sm) {
    double acc[kMaxDeg];
    for (int k = 0; k < d; ++k) acc[k] = 0.0;
    const int t = tile * kQcCnTile + (int)threadIdx.x;
    const int q_end = min(a.F4, (g + 1) * fpq);
    if (t < q.Z)
        for (int qd = g * fpq; qd < q_end; ++qd) qc_cn4_quad_n<BWD>(a, q, qd, i, t, b0, d, acc);
    if constexpr (BWD) {
        for (int k = 0; k < d; ++k) {
            const double s = block_sum(acc[k], sm);
            if (threadIdx.x == 0) wpart[((size_t)g * q.nblk + b0 + k) * tiles + tile] = s;
        }
    }
}

// Each thread moves four frames per message, so fewer resident warps keep as
// many bytes in flight as the frame-major kernels at 5-8 CTAs per SM.
template <bool BWD>
__global__ void __launch_bounds__(kThreads, BWD ? 3 : 4) qc_cn4_kernel(Args4 a, QcDev q, int tiles, int fpq,
                                                                      double* wpart) {
    __shared__ double sm[kThreads / 32];
    const int groups = (a.F4 + fpq - 1) / fpq;
    const long long total = (long long)groups * q.mb * tiles;
    for (long long blk = blockIdx.x; blk < total; blk += gridDim.x) {
        const int b = (int)blk, rt = b / groups;  // the host keeps total below 2^31
        const int g = b - rt * groups;
        const int i = rt / tiles, tile = rt - i * tiles;
        const int b0 = __ldg(q.row_ptr + i), d = __ldg(q.row_ptr + i + 1) - b0;
        switch (d) {
            case 0: break;
            case 1: qc_cn4_rows<1, BWD>(a, q, g, fpq, i, tile, b0, wpart, tiles, sm); break;
            case 2: qc_cn4_rows<2, BWD>(a, q, g, fpq, i, tile, b0, wpart, tiles, sm); break;
            case 3: qc_cn4_rows<3, BWD>(a, q, g, fpq, i, tile, b0, wpart, tiles, sm); break;
            case 4: qc_cn4_rows<4, BWD>(a, q, g, fpq, i, tile, b0, wpart, tiles, sm); break;
            default: qc_cn4_rows_n<BWD>(a, q, g, fpq, i, tile, b0, d, wpart, tiles, sm); break;
        }
    }
}

// Variable side, interleaved: the (quad, variable) pairs of base column j for
// the quads of group g, one pair (four frames, 16-byte accesses) per thread.
// Modes as qc_vn_one: kVnFwd APP = Lch + sum of c2v (block order; the last
// iteration also writes the caller's frame-major rows), kVnBwd S = sum G,
// dloss/dLch += S, G = S - G; kVnSeed G = dloss/dAPP, dloss/dLch = dloss/dAPP.
template <int MODE, int DV>
__device__ __forceinline__ void qc_vn4_cols(const Args4& a, const QcDev& q, int g, int fpq, int j, int cb0, int dv) {
    constexpr bool kFixed = DV > 0;
    const int Z = q.Z;
    const int nd = kFixed ? DV : dv;
    int blk[kFixed ? DV : 1];
    if constexpr (kFixed) {
#pragma unroll
        for (int b = 0; b < DV; ++b) blk[b] = __ldg(q.col_blk + cb0 + b);
    }
    auto block_of = [&](int b) { if constexpr (kFixed) return blk[b]; else return __ldg(q.col_blk + cb0 + b); };
    const int q0 = g * fpq, nq = min(a.F4, q0 + fpq) - q0;
    const int count = nq * Z;
    for (int idx = (int)threadIdx.x; idx < count; idx += kThreads) {
        const int ql = idx / Z, p = idx - ql * Z;
        const int qd = q0 + ql;
        const size_t qe = (size_t)qd * (size_t)a.E;
        const size_t vi = (size_t)qd * (size_t)a.n + (size_t)j * Z + p;
        if constexpr (MODE == kVnFwd) {
            float4 sum = __ldg(a.llr4 + vi);
            if constexpr (kFixed) {
                float4 m[DV];
#pragma unroll
                for (int b = 0; b < DV; ++b) m[b] = a.c2v_out[qe + (size_t)blk[b] * Z + p];
#pragma unroll
                for (int b = 0; b < DV; ++b) {
                    sum.x += m[b].x;
                    sum.y += m[b].y;
                    sum.z += m[b].z;
                    sum.w += m[b].w;
                }
            } else {
                for (int b = 0; b < nd; ++b) {
                    const float4 m = a.c2v_out[qe + (size_t)block_of(b) * Z + p];
                    sum.x += m.x;
                    sum.y += m.y;
                    sum.z += m.z;
                    sum.w += m.w;
                }
            }
            if (a.app_out) a.app_out[vi] = sum;
            if (a.app_rows) {
                const size_t v = (size_t)j * Z + p;
#pragma unroll
                for (int f = 0; f < 4; ++f)
                    if (4 * qd + f < a.F) a.app_rows[(size_t)(4 * qd + f) * a.n + v] = f4get(sum, f);
            }
        } else if constexpr (MODE == kVnBwd) {
            float4 sum = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            float4 m[kFixed ? DV : 1];
            if constexpr (kFixed) {
#pragma unroll
                for (int b = 0; b < DV; ++b) m[b] = a.G[qe + (size_t)blk[b] * Z + p];
#pragma unroll
                for (int b = 0; b < DV; ++b) {
                    sum.x += m[b].x;
                    sum.y += m[b].y;
                    sum.z += m[b].z;
                    sum.w += m[b].w;
                }
            } else {
                for (int b = 0; b < nd; ++b) {
                    const float4 mb = a.G[qe + (size_t)block_of(b) * Z + p];
                    sum.x += mb.x;
                    sum.y += mb.y;
                    sum.z += mb.z;
                    sum.w += mb.w;
                }
            }
            if (a.grad4) {
                float4 gl = a.grad4[vi];
                gl.x += sum.x;
                gl.y += sum.y;
                gl.z += sum.z;
                gl.w += sum.w;
                a.grad4[vi] = gl;
            }
            for (int b = 0; b < nd; ++b) {
                float4* gp = a.G + qe + (size_t)block_of(b) * Z + p;
                const float4 old = kFixed ? m[kFixed ? b : 0] : *gp;
                *gp = make_float4(sum.x - old.x, sum.y - old.y, sum.z - old.z, sum.w - old.w);
            }
        } else {
            float4 gv = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            const size_t v = (size_t)j * Z + p;
#pragma unroll
            for (int f = 0; f < 4; ++f)
                if (4 * qd + f < a.F) f4set(gv, f, __ldg(a.grad_app + (size_t)(4 * qd + f) * a.n + v));
            if (a.grad4) a.grad4[vi] = gv;
            for (int b = 0; b < nd; ++b) a.G[qe + (size_t)block_of(b) * Z + p] = gv;
        }
    }
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, 6) qc_vn4_kernel(Args4 a, QcDev q, int fpq) {
    const int groups = (a.F4 + fpq - 1) / fpq;
    const long long total = (long long)groups * q.nb;
    for (long long blk = blockIdx.x; blk < total; blk += gridDim.x) {
        const int g = (int)(blk % groups), j = (int)(blk / groups);
        const int cb0 = __ldg(q.col_ptr + j), dv = __ldg(q.col_ptr + j + 1) - cb0;
        switch (dv) {
            case 1: qc_vn4_cols<MODE, 1>(a, q, g, fpq, j, cb0, 1); break;
            case 2: qc_vn4_cols<MODE, 2>(a, q, g, fpq, j, cb0, 2); break;
            case 3: qc_vn4_cols<MODE, 3>(a, q, g, fpq, j, cb0, 3); break;
            case 4: qc_vn4_cols<MODE, 4>(a, q, g, fpq, j, cb0, 4); break;
            default: qc_vn4_cols<MODE, 0>(a, q, g, fpq, j, cb0, dv); break;
        }
    }
}

}  // namespace wbp
}  // namespace ldpcgb
