// EM fit of a one-dimensional Gaussian mixture on the GPU (Sec. 2.2,
// Eqs. 20-24): the pore-size statistics that the paper splits into organic
// (OM) and inorganic (IOM) components before the DGM/GMS permeabilities are
// assigned.  FP64 throughout.  One iteration is two passes over the samples:
//   pass 1: E-step responsibilities w_j(i) (Eqs. 20-21, exponent with its
//           minus sign) and the sums behind Phi_j (Eq. 22), mu_j (Eq. 23) and
//           the log-likelihood;
//   pass 2: the same responsibilities again and sum_i w_j(i)(x_i - mu_j)^2
//           with the new mu_j (Eq. 24).
// Each pass writes fixed per-block partials that one block adds in a fixed
// order, so a fit is bit-for-bit reproducible.

#include "glbm.h"

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>

extern __attribute__((visibility("hidden"))) thread_local char g_create_err[512];

namespace {

constexpr int KMAX = 8;
constexpr int EM_THREADS = 256;

struct EmParams {
    int k;
    double phi[KMAX], mu[KMAX], var[KMAX];  // current estimate (E-step uses these)
    double mu_new[KMAX];                    // pass-1 result used by pass 2
};

__device__ __forceinline__ void responsibilities(double x, const EmParams &p, double (&w)[KMAX], double &den) {
    const double inv_sqrt_2pi = 0.39894228040143267794;
    den = 0.0;
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
        if (j >= p.k) break;
        const double d = x - p.mu[j];
        const double g = inv_sqrt_2pi / sqrt(p.var[j]) * exp(-0.5 * d * d / p.var[j]);
        w[j] = g * p.phi[j];
        den += w[j];
    }
    const double inv = 1.0 / den;
#pragma unroll
    for (int j = 0; j < KMAX; ++j)
        if (j < p.k) w[j] *= inv;
}

// Block sum of `cnt` doubles held per thread in v[]; thread 0 writes them.
template <int CNT>
__device__ __forceinline__ void block_sums(double (&v)[CNT], int cnt, double *__restrict__ out) {
    __shared__ double sh[EM_THREADS / 32][CNT];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
#pragma unroll
    for (int c = 0; c < CNT; ++c) {
        if (c >= cnt) break;
        double s = v[c];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
        if (lane == 0) sh[warp][c] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int c = 0; c < cnt; ++c) {
            double s = 0.0;
            for (int w = 0; w < EM_THREADS / 32; ++w) s += sh[w][c];
            out[c] = s;
        }
    }
}

// pass 1 partials per block: [sum w_j (k), sum w_j x (k), sum log den]
__global__ void __launch_bounds__(EM_THREADS)
k_em_pass1(const double *__restrict__ x, long long m, const EmParams *__restrict__ pp, double *__restrict__ part) {
    const EmParams p = *pp;
    double v[2 * KMAX + 1];
#pragma unroll
    for (int c = 0; c < 2 * KMAX + 1; ++c) v[c] = 0.0;
    for (long long i = blockIdx.x * (long long)EM_THREADS + threadIdx.x; i < m;
         i += (long long)gridDim.x * EM_THREADS) {
        double w[KMAX], den;
        const double xi = x[i];
        responsibilities(xi, p, w, den);
#pragma unroll
        for (int j = 0; j < KMAX; ++j)
            if (j < p.k) {
                v[j] += w[j];
                v[KMAX + j] += w[j] * xi;
            }
        v[2 * KMAX] += log(den);
    }
    block_sums<2 * KMAX + 1>(v, 2 * KMAX + 1, part + (long long)blockIdx.x * (2 * KMAX + 1));
}

// pass 2 partials per block: [sum w_j (x - mu_new_j)^2 (k)]
__global__ void __launch_bounds__(EM_THREADS)
k_em_pass2(const double *__restrict__ x, long long m, const EmParams *__restrict__ pp, double *__restrict__ part) {
    const EmParams p = *pp;
    double v[KMAX];
#pragma unroll
    for (int c = 0; c < KMAX; ++c) v[c] = 0.0;
    for (long long i = blockIdx.x * (long long)EM_THREADS + threadIdx.x; i < m;
         i += (long long)gridDim.x * EM_THREADS) {
        double w[KMAX], den;
        const double xi = x[i];
        responsibilities(xi, p, w, den);
#pragma unroll
        for (int j = 0; j < KMAX; ++j)
            if (j < p.k) {
                const double d = xi - p.mu_new[j];
                v[j] += w[j] * d * d;
            }
    }
    block_sums<KMAX>(v, KMAX, part + (long long)blockIdx.x * KMAX);
}

// Fixed-order totals of the block partials; pass 1 sets phi, mu_new and the
// log-likelihood, pass 2 the variances and moves mu_new into mu.
__global__ void k_em_finalize(const double *__restrict__ part, int nblocks, long long m, int pass,
                              EmParams *__restrict__ pp, double *__restrict__ sw_keep, double *__restrict__ ll) {
    if (threadIdx.x != 0) return;
    EmParams &p = *pp;
    if (pass == 1) {
        const int W = 2 * KMAX + 1;
        for (int j = 0; j < p.k; ++j) {
            double sw = 0.0, swx = 0.0;
            for (int b = 0; b < nblocks; ++b) {
                sw += part[(long long)b * W + j];
                swx += part[(long long)b * W + KMAX + j];
            }
            sw_keep[j] = sw;
            p.mu_new[j] = swx / sw;
        }
        double s = 0.0;
        for (int b = 0; b < nblocks; ++b) s += part[(long long)b * W + 2 * KMAX];
        *ll = s / double(m);
    } else {
        for (int j = 0; j < p.k; ++j) {
            double sd = 0.0;
            for (int b = 0; b < nblocks; ++b) sd += part[(long long)b * KMAX + j];
            p.phi[j] = sw_keep[j] / double(m);
            p.mu[j] = p.mu_new[j];
            p.var[j] = sd / sw_keep[j];
        }
    }
}

glbm_status emfail(glbm_status s, const char *fmt, const char *detail) {
    snprintf(g_create_err, 512, fmt, detail);
    return s;
}

}  // namespace

extern "C" glbm_status glbm_em_gmm1d(const double *x, long long m, int k, double *phi, double *mu, double *var,
                                     int max_iter, double tol, int *iters, double *loglik, int device_ptrs,
                                     void *stream) {
    if (iters) *iters = 0;
    if (!x || !phi || !mu || !var || m < 1 || k < 1 || k > KMAX || max_iter < 0 || !std::isfinite(tol))
        return emfail(GLBM_EINVAL, "em_gmm1d: %s", "need x, m >= 1, 1 <= k <= 8, phi/mu/var and max_iter >= 0");
    EmParams hp{};
    hp.k = k;
    double fsum = 0.0;
    for (int j = 0; j < k; ++j) {
        if (!(phi[j] > 0.0) || !(var[j] > 0.0) || !std::isfinite(mu[j]))
            return emfail(GLBM_EINVAL, "em_gmm1d: %s", "initial fractions and variances must be > 0");
        hp.phi[j] = phi[j];
        hp.mu[j] = mu[j];
        hp.var[j] = var[j];
        fsum += phi[j];
    }
    for (int j = 0; j < k; ++j) hp.phi[j] /= fsum;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nb = int(std::min<long long>((m + EM_THREADS - 1) / EM_THREADS, 152LL * 8));
    double *dx = nullptr, *part = nullptr, *sw = nullptr, *dll = nullptr;
    EmParams *dp = nullptr;
    cudaError_t e = cudaSuccess;
    if (!device_ptrs) {
        e = cudaMalloc(&dx, sizeof(double) * m);
        if (e == cudaSuccess) e = cudaMemcpyAsync(dx, x, sizeof(double) * m, cudaMemcpyHostToDevice, st);
    }
    if (e == cudaSuccess) e = cudaMalloc(&part, sizeof(double) * nb * (2 * KMAX + 1));
    if (e == cudaSuccess) e = cudaMalloc(&sw, sizeof(double) * KMAX);
    if (e == cudaSuccess) e = cudaMalloc(&dll, sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&dp, sizeof(EmParams));
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp, &hp, sizeof(EmParams), cudaMemcpyHostToDevice, st);
    const double *xs = device_ptrs ? x : dx;
    double prev = -INFINITY, ll = -INFINITY;
    int it = 0;
    for (; e == cudaSuccess && it < max_iter; ++it) {
        k_em_pass1<<<nb, EM_THREADS, 0, st>>>(xs, m, dp, part);
        k_em_finalize<<<1, 32, 0, st>>>(part, nb, m, 1, dp, sw, dll);
        k_em_pass2<<<nb, EM_THREADS, 0, st>>>(xs, m, dp, part);
        k_em_finalize<<<1, 32, 0, st>>>(part, nb, m, 2, dp, sw, dll);
        e = cudaGetLastError();
        if (e == cudaSuccess && tol > 0.0) {
            e = cudaMemcpyAsync(&ll, dll, sizeof(double), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e == cudaSuccess && std::fabs(ll - prev) < tol) {
                ++it;
                break;
            }
            prev = ll;
        }
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hp, dp, sizeof(EmParams), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&ll, dll, sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    void *ptrs[] = {dx, part, sw, dll, dp};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    if (e != cudaSuccess) return emfail(GLBM_ECUDA, "em_gmm1d: %s", cudaGetErrorString(e));
    bool finite = true;
    for (int j = 0; j < k; ++j) {
        phi[j] = hp.phi[j];
        mu[j] = hp.mu[j];
        var[j] = hp.var[j];
        finite = finite && std::isfinite(phi[j]) && std::isfinite(mu[j]) && std::isfinite(var[j]);
    }
    if (iters) *iters = it;
    if (loglik) *loglik = max_iter > 0 ? ll : NAN;
    // a component that collapses onto a single sample has zero variance and
    // the next E-step is undefined
    if (!finite) return emfail(GLBM_ENAN, "em_gmm1d: %s", "estimate not finite (a component collapsed)");
    return GLBM_OK;
}
