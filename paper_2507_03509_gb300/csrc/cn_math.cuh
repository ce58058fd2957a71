// Check-node arithmetic shared by the decoder and the weighted-BP kernels:
// clamping helpers and the check-node cores (the sum-product check rule of
// the paper's section "Early Termination", with the syndrome sign).
#pragma once

#include <cuda_runtime.h>

namespace ldpcgb {

constexpr int kMaxDeg = 64;              // largest check degree supported

__device__ __forceinline__ float clampm(float x, float l) { return fminf(fmaxf(x, -l), l); }
__device__ __forceinline__ double clampm(double x, double l) { return fmin(fmax(x, -l), l); }
__device__ __forceinline__ float absm(float x) { return fabsf(x); }
__device__ __forceinline__ double absm(double x) { return fabs(x); }

// ---------------------------------------------------------------------------
// Check-node cores.  In: clamped v2c messages v[0..D).  Out: c2v messages
// c2v_k = (1 - 2 s) * prod_{j != k} sgn(v_j) * |v_0 [+] ... (skip k) ... [+] v_{D-1}|
// where [+] is the boxplus, 2 atanh(tanh(a/2) tanh(b/2)).
//
// FP32: signs and magnitudes are kept apart, so the rule is exactly odd in
// every input.  A magnitude x maps to r = exp(-x); boxplus of magnitudes is
// then r_a (+) r_b = (r_a + r_b) / (1 + r_a r_b) -- the tanh-product identity
// rewritten for 1 - tanh, which neither saturates nor cancels in FP32 -- and
// the result is -ln r.  Exclusive combinations come from prefix and suffix
// products (forward-backward); a degree-2 check copies the other message.
// FP64 (debug): the tanh/atanh rule literally, products by explicit loop.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float rcomb(float a, float b) {
    return __fdividef(a + b, fmaf(a, b, 1.0f));
}

template <int D>
__device__ __forceinline__ void cn_core(const float (&v)[D], unsigned sbit, float lmax,
                                        float (&out)[D]) {
    if constexpr (D == 1) {
        out[0] = sbit ? -lmax : lmax;
    } else {
        unsigned par = sbit;
        bool ng[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            ng[k] = v[k] < 0.0f;
            par ^= (unsigned)ng[k];
        }
        float mag[D];
        if constexpr (D == 2) {
            mag[0] = fabsf(v[1]);
            mag[1] = fabsf(v[0]);
        } else {
            float r[D], pre[D], suf[D];
#pragma unroll
            for (int k = 0; k < D; ++k) r[k] = __expf(-fabsf(v[k]));
            pre[0] = r[0];
#pragma unroll
            for (int k = 1; k < D - 1; ++k) pre[k] = rcomb(pre[k - 1], r[k]);
            suf[D - 1] = r[D - 1];
#pragma unroll
            for (int k = D - 2; k >= 1; --k) suf[k] = rcomb(r[k], suf[k + 1]);
#pragma unroll
            for (int k = 0; k < D; ++k) {
                float ex = (k == 0) ? suf[1] : (k == D - 1) ? pre[D - 2] : rcomb(pre[k - 1], suf[k + 1]);
                mag[k] = fminf(fmaxf(-__logf(ex), 0.0f), lmax);
            }
        }
#pragma unroll
        for (int k = 0; k < D; ++k) out[k] = (par ^ (unsigned)ng[k]) ? -mag[k] : mag[k];
    }
}

template <int D>
__device__ __forceinline__ void cn_core(const double (&v)[D], unsigned sbit, double lmax,
                                        double (&out)[D]) {
    double th[D];
#pragma unroll
    for (int k = 0; k < D; ++k) th[k] = tanh(0.5 * v[k]);
    const double sg = sbit ? -1.0 : 1.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        double prod = 1.0;
#pragma unroll
        for (int j = 0; j < D; ++j)
            if (j != k) prod *= th[j];
        out[k] = clampm(sg * 2.0 * atanh(prod), lmax);
    }
}

// Degree > 8: the same rules with loops over local arrays.
static __device__ __noinline__ void cn_core_n(const float* v, int d, unsigned sbit, float lmax, float* out) {
    float r[kMaxDeg], suf[kMaxDeg];
    unsigned par = sbit;
    for (int k = 0; k < d; ++k) {
        par ^= (unsigned)(v[k] < 0.0f);
        r[k] = __expf(-fabsf(v[k]));
    }
    suf[d - 1] = r[d - 1];
    for (int k = d - 2; k >= 1; --k) suf[k] = rcomb(r[k], suf[k + 1]);
    float pre = 0.0f;
    for (int k = 0; k < d; ++k) {
        float ex = (k == 0) ? suf[1] : (k == d - 1) ? pre : rcomb(pre, suf[k + 1]);
        float mag = fminf(fmaxf(-__logf(ex), 0.0f), lmax);
        out[k] = (par ^ (unsigned)(v[k] < 0.0f)) ? -mag : mag;
        pre = (k == 0) ? r[0] : rcomb(pre, r[k]);
    }
}

static __device__ __noinline__ void cn_core_n(const double* v, int d, unsigned sbit, double lmax, double* out) {
    double th[kMaxDeg];
    for (int k = 0; k < d; ++k) th[k] = tanh(0.5 * v[k]);
    const double sg = sbit ? -1.0 : 1.0;
    for (int k = 0; k < d; ++k) {
        double prod = 1.0;
        for (int j = 0; j < d; ++j)
            if (j != k) prod *= th[j];
        out[k] = clampm(sg * 2.0 * atanh(prod), lmax);
    }
}

}  // namespace ldpcgb
