// Device evaluation of the Lagrange basis on the p-division points (§2.1.1,
// eq. Lag1): g_i(t) = cinv_i * prod_{k != i} (t - tau_k).
#pragma once
#include "fmm_internal.cuh"

namespace fmm {

// all p weights g_i(t), by prefix/suffix products; p <= NMAX, g holds NMAX
template <typename real, int NMAX = FMM_MAXP>
__device__ __forceinline__ void lag_weights(const Coef<real> &C, int p, real t, real *g) {
    real d[NMAX];
#pragma unroll
    for (int k = 0; k < NMAX; k++) d[k] = (k < p) ? t - C.tau[k] : real(1);
    real pre = 1;
#pragma unroll
    for (int i = 0; i < NMAX; i++) {
        g[i] = pre;
        pre *= d[i];
    }
    real suf = 1;
#pragma unroll
    for (int i = NMAX - 1; i >= 0; i--) {
        if (i < p) {
            g[i] *= suf * C.cinv[i];
            suf *= d[i];
        } else {
            g[i] = 0;
        }
    }
}

// weights and their derivatives d g_i / dt (running value/derivative product)
template <typename real>
__device__ __forceinline__ void lag_weights_deriv(const Coef<real> &C, int p, real t, real *g,
                                                  real *dg) {
    real d[FMM_MAXP];
#pragma unroll
    for (int k = 0; k < FMM_MAXP; k++) d[k] = (k < p) ? t - C.tau[k] : real(1);
#pragma unroll
    for (int i = 0; i < FMM_MAXP; i++) {
        real v = 1, dv = 0;
#pragma unroll
        for (int k = 0; k < FMM_MAXP; k++) {
            if (k != i && k < p) {
                dv = dv * d[k] + v;
                v = v * d[k];
            }
        }
        g[i] = (i < p) ? v * C.cinv[i] : real(0);
        dg[i] = (i < p) ? dv * C.cinv[i] : real(0);
    }
}

// one weight and its derivative
template <typename real>
__device__ __forceinline__ void lag_one(const Coef<real> &C, int p, int i, real t, real &g,
                                        real &dg) {
    real v = 1, dv = 0;
#pragma unroll
    for (int k = 0; k < FMM_MAXP; k++) {
        if (k != i && k < p) {
            real d = t - C.tau[k];
            dv = dv * d + v;
            v = v * d;
        }
    }
    g = v * C.cinv[i];
    dg = dv * C.cinv[i];
}

}  // namespace fmm
