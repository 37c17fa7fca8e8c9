// setup_kernels.cuh -- once-per-medium and export kernels of the GLBM
// library (validation, coefficient packing, equilibrium initialisation, FP16
// rescaling, distribution export).  They run outside the time loop; the step
// path itself is in glbm_kernels.cuh, which this header builds on.

#pragma once

#include "glbm_kernels.cuh"

namespace {

// A1: validate the medium; *first_bad receives the lowest invalid index
// (left at INT_MAX when every node has eps in (0, 1] and K > 0 or +inf).
__global__ void k_validate(const double *__restrict__ eps, const double *__restrict__ K,
                           long long N, int *__restrict__ first_bad) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const double e = eps[n], k = K[n];
        const bool ok = (e > 0.0) && (e <= 1.0) && (k > 0.0);  // NaN fails every test
        if (!ok) atomicMin(first_bad, int(n));
    }
}

// Warm-start inputs: rho must be positive and finite, u finite.
__global__ void k_validate_state(const double *__restrict__ rho, const double *__restrict__ ux,
                                 const double *__restrict__ uy, long long N, int *__restrict__ first_bad) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        bool ok = true;
        if (rho) ok = ok && rho[n] > 0.0 && isfinite(rho[n]);
        if (ux) ok = ok && isfinite(ux[n]) && isfinite(uy[n]);
        if (!ok) atomicMin(first_bad, int(n));
    }
}

// A1: pack per-node coefficients (Eqs. 36-37) from FP64 eps, K.  FP32
// coefficients take alpha = eps nu / K in IEEE single precision on the
// rounded inputs (within 2 ulp of the rounded FP64 quotient): FP64 division
// is slow on this GPU and set_medium sits inside end-to-end runs.  The
// Forchheimer beta keeps FP64 (its Ergun form cubes eps); without the
// Forchheimer term it is zero.
template <typename R>
__global__ void k_pack(const double *__restrict__ eps, const double *__restrict__ K, long long N,
                       double nu, double feps_mode, R *__restrict__ alpha, R *__restrict__ epsv,
                       R *__restrict__ betav) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const double e = eps[n], k = K[n];
        if constexpr (std::is_same<R, float>::value) {
            const float ef = float(e);
            alpha[n] = __fdiv_rn(__fmul_rn(ef, float(nu)), float(k));
            epsv[n] = ef;
        } else {
            alpha[n] = e * nu / k;
            epsv[n] = e;
        }
        if (betav) {
            if (feps_mode == 0.0) {
                betav[n] = R(0);
            } else {
                const double fe = feps_mode > 0.0 ? feps_mode : 1.75 / sqrt(150.0 * e * e * e);
                betav[n] = R(e * fe / sqrt(k));
            }
        }
    }
}

// K4: distributions set to the porosity equilibrium f_eq(rho, u; eps)
// (Eq. 30), stored as deviations.  rho/ux/uy may be NULL.
template <typename T>
__global__ void k_init_eq(T *__restrict__ dst, long long plane, long long N,
                          const typename Store<T>::R *__restrict__ epsv, const double *__restrict__ rho,
                          const double *__restrict__ ux, const double *__restrict__ uy,
                          typename Store<T>::R scale) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const double r = rho ? rho[n] : 1.0;
        const double vx = ux ? ux[n] : 0.0, vy = uy ? uy[n] : 0.0;
        const double ie = 1.0 / double(epsv[n]);
        const double uu = vx * vx + vy * vy;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double eu = cx(i) * vx + cy(i) * vy;
            const double w = wgt<double>(i);
            const double gdev = w * (r - 1.0) + w * r * (3.0 * eu + 4.5 * ie * eu * eu - 1.5 * ie * uu);
            dst[i * plane + n] = Store<T>::st(typename Store<T>::R(gdev), scale);
        }
    }
}

// Largest |f_eq - w| over nodes and populations (for choosing the FP16
// scale before a warm start); float bits of a non-negative value order like
// the integers, so atomicMax on them is a float max.
__global__ void k_eq_max(long long N, const float *__restrict__ epsv, const double *__restrict__ rho,
                         const double *__restrict__ ux, const double *__restrict__ uy, int *__restrict__ out) {
    float m = 0.0f;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const double r = rho ? rho[n] : 1.0;
        const double vx = ux ? ux[n] : 0.0, vy = uy ? uy[n] : 0.0;
        const double ie = 1.0 / double(epsv[n]);
        const double uu = vx * vx + vy * vy;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const double eu = cx(i) * vx + cy(i) * vy;
            const double w = wgt<double>(i);
            const double gdev = w * (r - 1.0) + w * r * (3.0 * eu + 4.5 * ie * eu * eu - 1.5 * ie * uu);
            m = fmaxf(m, float(fabs(gdev)));
        }
    }
    atomicMax(out, __float_as_int(m));
}

// Multiply every stored value by a power of two (FP16 scale change).
template <typename T>
__global__ void k_rescale(T *__restrict__ buf, long long count, float factor) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < count;
         n += (long long)gridDim.x * blockDim.x)
        buf[n] = Store<T>::st(Store<T>::ld(buf[n], 1.0f) * factor, 1.0f);
}

// Export absolute distributions f_i = g_i + w_i in FP64.
template <typename T>
__global__ void k_export_f(const T *__restrict__ src, long long plane, long long N,
                           typename Store<T>::R inv_s, double *__restrict__ f) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int i = 0; i < 9; ++i)
            f[i * N + n] = double(Store<T>::ld(src[i * plane + n], inv_s)) + wgt<double>(i);
    }
}

}  // namespace
