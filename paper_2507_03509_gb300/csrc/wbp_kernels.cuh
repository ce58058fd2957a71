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
    float rb = 0.0f;
    bool neg = false;
#pragma unroll
    for (int i = 0; i < D; ++i) {
        if (i == e || i == j) continue;
        rb = rcomb(rb, r[i]);
        neg ^= ng[i];
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

// Degree > 6: the same with loops over local arrays (O(d^3) derivative).
template <bool BWD, typename T, class Code, class Ck>
__device__ __noinline__ void check_n(const Args<T>& a, const Code& g, const Ck& ck, int f, int c) {
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
    double acc = 0.0;
    for (long long id = (long long)blockIdx.x * kThreads + threadIdx.x; id < total;
         id += (long long)gridDim.x * kThreads) {
        const T sx = __ldg(x + id) ? T(-1) : T(1);
        const T z = -sx * app[id];
        acc += (double)softplus_t(z);
        if (grad_app) grad_app[id] = -sx * sigmoid_t(z) * (T)scale;
    }
    const double s = block_sum(acc, sm);
    if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

template <typename T>
__global__ void loss_final_kernel(const double* partial, int count, double scale, T* loss_out) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double s = 0.0;
        for (int i = 0; i < count; ++i) s += partial[i];
        *loss_out = (T)(s * scale);
    }
}

// Plain gradient step on the weights: w -= lr * g.
template <typename T>
__global__ void sgd_kernel(T* w, const T* g, int count, T lr) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x) w[i] -= lr * g[i];
}

}  // namespace wbp
}  // namespace ldpcgb
