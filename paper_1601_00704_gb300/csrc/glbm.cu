// GB300 (sm_103a) implementation of the generalized lattice Boltzmann model
// (GLBM) time loop of Wang, Chen, Kang & Rahman, arXiv:1601.00704, Sec. 2.3.
//
// Hot path: one fused pull-stream + collide kernel per time step (Eq. 29 with
// Eqs. 27, 30-37) over a structure-of-arrays distribution layout, followed every
// chunk by a deterministic FP64 mean-velocity reduction that stays on the
// device.  The C ABI is declared in include/glbm.h.
//
// Design notes
//  * Distributions are stored as deviations g_i = f_i - w_i (rho0 = 1).  At
//    the Darcy velocities of shale media (u ~ 1e-9 lattice units) the
//    momentum signal sits ~8 decades below f_i ~ w_i; deviations keep it
//    inside FP32 (and FP16/BF16 with a power-of-two scale) precision.
//  * Layout: plane i (D2Q9 order below) holds g_i for node n = y*nx + x; the
//    plane stride is nx*ny rounded up to 64 elements, so every plane and, when
//    nx is a multiple of the vector width, every row starts 16-byte aligned.
//  * Each thread owns VEC consecutive nodes of one row (VEC*sizeof(T) = 16 B)
//    and moves them with 128-bit loads/stores.  Populations with e_x = +-1
//    need the x-1 / x+1 neighbour: it comes from the adjacent lane by a warp
//    shuffle; lanes 0/31 and the periodic row ends fetch one scalar.  A scalar
//    (VEC = 1) instantiation serves lattices whose nx is not a multiple of VEC.
//  * Per-node coefficients are packed once per medium (Eqs. 36-37):
//      alpha = eps*nu/K   (c0 = 1/2 + alpha/4, Darcy drag alpha*u),
//      eps, beta = eps*F_eps/sqrt(K)  (c1 = beta/2, only with Forchheimer).
//    Storing alpha rather than c0 keeps full relative precision of the drag
//    for nearly clear nodes, where 4*c0 - 2 would cancel.
//  * Halfway bounce-back walls at y = -1/2 and y = ny-1/2 and periodic x are
//    index arithmetic inside the kernel; no ghost layers, no extra bytes.
//  * The velocity solve (Eqs. 32-35) uses explicitly rounded intrinsics so
//    the velocity export kernel reproduces the step kernel's u bit for bit.

#include "glbm.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

namespace {

// ---------------------------------------------------------------------------
// D2Q9: e0=(0,0); e1..e4=(1,0),(0,1),(-1,0),(0,-1);
//       e5..e8=(1,1),(-1,1),(-1,-1),(1,-1); w = 4/9, 1/9 (x4), 1/36 (x4).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 3 || i == 6 || i == 7) ? -1 : 0);
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : ((i == 4 || i == 7 || i == 8) ? -1 : 0);
}
__host__ __device__ constexpr int opp(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
}
template <typename R>
__host__ __device__ constexpr R wgt(int i) {
    return i == 0 ? R(4) / R(9) : (i <= 4 ? R(1) / R(9) : R(1) / R(36));
}
static_assert(opp(1) == 3 && opp(2) == 4 && opp(3) == 1 && opp(4) == 2, "opp");
static_assert(opp(5) == 7 && opp(6) == 8 && opp(7) == 5 && opp(8) == 6, "opp");

// ---------------------------------------------------------------------------
// Explicitly rounded arithmetic (no FMA contraction differences between
// kernels that must agree bitwise).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ float rdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float rsqrt_(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ double rdiv(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ double rsqrt_(double a) { return __dsqrt_rn(a); }
// Reciprocals of rho ~ 1, 2*c0 >= 1 and eps in (0, 1]: the hardware
// approximation (within 1 ulp) is ample and a fraction of IEEE rcp's cost.
__device__ __forceinline__ float rrcp(float a) { return __fdividef(1.0f, a); }
__device__ __forceinline__ double rrcp(double a) { return __drcp_rn(a); }

// ---------------------------------------------------------------------------
// Storage formats.  R is the collision arithmetic type.
// ---------------------------------------------------------------------------
// Stochastic rounding: round |x| up with probability equal to the dropped
// fraction, using uniform random bits r; unbiased in expectation, so slow
// modes whose per-step change is below half an ulp do not freeze.
// FP16: stochastic in the normal range [2^-14, 65504]; values below it are
// rounded to nearest -- with the scale keeping the largest stored magnitude
// near 2^12 they lie 2^26 below it, where a biased last bit is immaterial --
// and overflow, inf and NaN convert as usual.
__device__ __forceinline__ __half f2h_sr(float x, uint32_t r) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t a = b & 0x7fffffffu;
    const uint32_t t = (b + (r & 0x1FFFu)) & ~0x1FFFu;  // drop 13 mantissa bits
    const bool normal = a - 0x38800000u < 0x477fe000u - 0x38800000u;
    return normal ? __float2half_rz(__uint_as_float(t)) : __float2half_rn(x);
}
__device__ __forceinline__ __nv_bfloat16 f2bf_sr(float x, uint32_t r) {
    const uint32_t b = __float_as_uint(x);
    const uint32_t t = (b + (r & 0xFFFFu)) & 0xFFFF0000u;  // drop 16 mantissa bits
    const bool finite = (b & 0x7f800000u) != 0x7f800000u;
    return finite ? __float2bfloat16_rz(__uint_as_float(t)) : __float2bfloat16_rn(x);
}

template <typename T> struct Store;
template <> struct Store<float> {
    using R = float;
    static constexpr bool kSmall = false;
    __device__ static float ld(float v, float) { return v; }
    __device__ static float st(float v, float) { return v; }
    __device__ static float st_sr(float v, float, uint32_t) { return v; }
};
template <> struct Store<double> {
    using R = double;
    static constexpr bool kSmall = false;
    __device__ static double ld(double v, double) { return v; }
    __device__ static double st(double v, double) { return v; }
    __device__ static double st_sr(double v, double, uint32_t) { return v; }
};
template <> struct Store<__half> {
    using R = float;
    static constexpr bool kSmall = true;
    __device__ static float ld(__half v, float inv_s) { return __half2float(v) * inv_s; }
    __device__ static __half st(float v, float s) { return __float2half_rn(v * s); }
    __device__ static __half st_sr(float v, float s, uint32_t r) { return f2h_sr(v * s, r); }
    static constexpr bool kScaled = true;
    // Two scaled values -> packed pair with hardware stochastic rounding
    // (cvt.rs): `lo` lands in the low half (lower address), `hi` in the high.
    __device__ static uint32_t pack_sr(float lo, float hi, uint32_t rbits) {
        uint32_t d;
        asm("cvt.rs.f16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
        return d;
    }
};
template <> struct Store<__nv_bfloat16> {
    using R = float;
    static constexpr bool kSmall = true;
    // BF16 has FP32's exponent range: stored unscaled (the scale is always 1)
    __device__ static float ld(__nv_bfloat16 v, float) { return __bfloat162float(v); }
    __device__ static __nv_bfloat16 st(float v, float) { return __float2bfloat16_rn(v); }
    __device__ static __nv_bfloat16 st_sr(float v, float, uint32_t r) { return f2bf_sr(v, r); }
    static constexpr bool kScaled = false;
    __device__ static uint32_t pack_sr(float lo, float hi, uint32_t rbits) {
        uint32_t d;
        asm("cvt.rs.bf16x2.f32 %0, %1, %2, %3;" : "=r"(d) : "f"(hi), "f"(lo), "r"(rbits));
        return d;
    }
};

// Nodes per thread: 16-byte vectors for 32/64-bit storage, 8-byte vectors
// (4 nodes) for 16-bit storage.
template <typename T>
constexpr int kVecOf = sizeof(T) == 2 ? 4 : int(16 / sizeof(T));

// Integer hash ("lowbias32" multiply-xorshift) for the stochastic rounding
// bits: one 32-bit word per (node, step, population pair).
__host__ __device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

template <typename R>
struct Phys {
    R omega;     // 1/tau
    R A;         // 1 - 1/(2 tau)
    R gx, gy;    // external force G
    R scale;     // storage scale S (stored = g*S); 1 for FP32/FP64
    R inv_scale; // 1/S
    uint32_t step_key;  // per-step key of the stochastic-rounding hash
    int sr;             // 16-bit storage: 1 = stochastic rounding, 0 = nearest
};

struct Geo {
    int nx, ny;
    long long plane;  // elements per population plane
    int bpr;          // blocks per row
};

// Vector moves of 8 bytes or a multiple of 16 bytes.
template <typename X, int N>
__device__ __forceinline__ void ld16(const X *__restrict__ p, X (&out)[N]) {
    constexpr int B = int(N * sizeof(X));
    static_assert(B == 8 || B % 16 == 0, "8-byte or 16-byte multiple");
    if constexpr (B == 8) {
        uint2 u = *reinterpret_cast<const uint2 *>(p);
        memcpy(&out[0], &u, 8);
    } else {
#pragma unroll
        for (int j = 0; j < B / 16; ++j) {
            uint4 u = reinterpret_cast<const uint4 *>(p)[j];
            memcpy(&out[j * (16 / sizeof(X))], &u, 16);
        }
    }
}
template <typename X, int N>
__device__ __forceinline__ void st16(X *__restrict__ p, const X (&in)[N]) {
    constexpr int B = int(N * sizeof(X));
    if constexpr (B == 8) {
        uint2 u;
        memcpy(&u, &in[0], 8);
        __stcs(reinterpret_cast<uint2 *>(p), u);
    } else {
#pragma unroll
        for (int j = 0; j < B / 16; ++j) {
            uint4 u;
            memcpy(&u, &in[j * (16 / sizeof(X))], 16);
            __stcs(reinterpret_cast<uint4 *>(p) + j, u);
        }
    }
}

// ---------------------------------------------------------------------------
// Per-node physics.
// ---------------------------------------------------------------------------

// Eqs. 32, 33, 35, 36, 37, 34: density deviation and the node velocity from
// the streamed deviations g[9].  Explicit rounding: see file header.
template <typename R, bool FORCH>
__device__ __forceinline__ void node_velocity(const R (&g)[9], R alpha, R eps, R beta,
                                              const Phys<R> &ph, R &drho, R &ux, R &uy) {
    drho = radd(radd(radd(g[0], radd(g[1], g[3])), radd(g[2], g[4])),
                radd(radd(g[5], g[7]), radd(g[6], g[8])));
    const R mx = radd(radd(rsub(g[1], g[3]), rsub(g[5], g[7])), rsub(g[8], g[6]));
    const R my = radd(radd(rsub(g[2], g[4]), rsub(g[5], g[7])), rsub(g[6], g[8]));
    const R rho = radd(R(1), drho);
    const R inv_rho = rrcp(rho);
    const R heps = rmul(R(0.5), eps);
    const R vx = rfma(mx, inv_rho, rmul(heps, ph.gx));
    const R vy = rfma(my, inv_rho, rmul(heps, ph.gy));
    const R c0 = rfma(R(0.25), alpha, R(0.5));
    R den;
    if (FORCH) {
        const R c1 = rmul(R(0.5), beta);
        const R vmag = rsqrt_(rfma(vx, vx, rmul(vy, vy)));
        den = radd(c0, rsqrt_(rfma(c1, vmag, rmul(c0, c0))));
    } else {
        den = rfma(R(0.5), alpha, R(1));  // 2*c0
    }
    const R inv_den = rrcp(den);
    ux = rmul(vx, inv_den);
    uy = rmul(vy, inv_den);
}

// Eq. 27 force, Eq. 30 equilibrium and Eq. 31 forcing (with the 1/eps on the
// u.F term, the mass-conserving reading), then the BGK update of Eq. 29,
// g* = g + (g_eq - g)/tau + F_i.
//
// Rounding: at Darcy velocities every deviation is dominated by its density
// carrier w_i (rho - 1), several decades above the velocity terms.  The update
// is therefore regrouped as
//     g* = w d + [ (1 - 1/tau)(g - w d) + w (even +- odd) ],   d = rho - 1,
// where the bracket holds only small terms (g - w d is exact when g ~ w d),
// so the carrier is rounded twice per population instead of at every term.
// Opposite directions share the even part of f_eq and F_i (terms in 1,
// (e.u)^2, (e.u)(e.F)) and flip the odd part (e.u, e.F).  g[] holds the
// streamed deviations on entry and the post-collision deviations on exit.
template <typename R, bool CARRIER>
__device__ __forceinline__ void collide_pair(R &gi, R &gj, R w, R wd, R eu, R eF, R k1, R om, R su, R a2,
                                             R rho3, R fb, R f3, R f9) {
    // even:  om [rho (9/(2 eps)(e.u)^2 - 3/(2 eps) u^2)] + rho A [9/eps (e.u)(e.F) - 3/eps u.F]
    // odd :  om [3 rho e.u] + rho A [3 e.F]
    const R ev = om * (a2 * eu * eu - su) + (fb + f9 * eu * eF);
    const R od = om * rho3 * eu + f3 * eF;
    if (CARRIER) {
        gi = wd + (k1 * (gi - wd) + w * (ev + od));
        gj = wd + (k1 * (gj - wd) + w * (ev - od));
    } else {
        // 16-bit storage: its own rounding dominates, use the shorter form
        // k1 g + om w d + w (even +- odd)
        const R b = om * wd;
        gi = k1 * gi + (b + w * (ev + od));
        gj = k1 * gj + (b + w * (ev - od));
    }
}

template <typename R, bool FORCH, bool CARRIER = true>
__device__ __forceinline__ void collide(R (&g)[9], R alpha, R eps, R beta,
                                        const Phys<R> &ph, R &ux, R &uy) {
    R drho;
    node_velocity<R, FORCH>(g, alpha, eps, beta, ph, drho, ux, uy);
    const R rho = R(1) + drho;
    R Fx = eps * ph.gx - alpha * ux;
    R Fy = eps * ph.gy - alpha * uy;
    if (FORCH) {
        const R bu = beta * sqrt(ux * ux + uy * uy);
        Fx -= bu * ux;
        Fy -= bu * uy;
    }
    const R ie = rrcp(eps);
    const R om = ph.omega, k1 = R(1) - ph.omega;
    const R rho3 = R(3) * rho;
    const R a2 = R(4.5) * ie * rho;
    const R su = R(1.5) * ie * rho * (ux * ux + uy * uy);
    const R rA = rho * ph.A;
    const R f3 = R(3) * rA;
    const R f9 = R(9) * ie * rA;
    const R fb = R(-3) * ie * rA * (ux * Fx + uy * Fy);
    const R w0 = wgt<R>(0), w1 = wgt<R>(1), w2 = wgt<R>(5);
    const R wd0 = w0 * drho, wd1 = w1 * drho, wd2 = w2 * drho;
    if (CARRIER) g[0] = wd0 + (k1 * (g[0] - wd0) + w0 * (fb - om * su));
    else g[0] = k1 * g[0] + (om * wd0 + w0 * (fb - om * su));
    collide_pair<R, CARRIER>(g[1], g[3], w1, wd1, ux, Fx, k1, om, su, a2, rho3, fb, f3, f9);
    collide_pair<R, CARRIER>(g[2], g[4], w1, wd1, uy, Fy, k1, om, su, a2, rho3, fb, f3, f9);
    collide_pair<R, CARRIER>(g[5], g[7], w2, wd2, ux + uy, Fx + Fy, k1, om, su, a2, rho3, fb, f3, f9);
    collide_pair<R, CARRIER>(g[6], g[8], w2, wd2, uy - ux, Fy - Fx, k1, om, su, a2, rho3, fb, f3, f9);
}

// ---------------------------------------------------------------------------
// Pull-streaming gather of VEC consecutive nodes (x0..x0+VEC-1, row y).
// Phase 1 issues every load of the thread (9 vectors + up to 6 edge scalars)
// before phase 2 consumes any, so all of them are in flight together.
// ---------------------------------------------------------------------------
template <typename T, int VEC, bool WALLS>
__device__ __forceinline__ void gather(const T *__restrict__ src, const Geo &geo, int x0, int y,
                                       bool active, int lane, typename Store<T>::R inv_s,
                                       typename Store<T>::R (&g)[VEC][9]) {
    using R = typename Store<T>::R;
    const int nx = geo.nx, ny = geo.ny;
    if constexpr (VEC == 1) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            int ys = y - cy(i);
            const T *p;
            if (ys < 0 || ys >= ny) {
                if (WALLS) {
                    // halfway bounce-back: the opposite population that left
                    // this node towards the wall returns reversed
                    p = src + (long long)opp(i) * geo.plane + (long long)y * nx + x0;
                    g[0][i] = active ? Store<T>::ld(*p, inv_s) : R(0);
                    continue;
                }
                ys = ys < 0 ? ys + ny : ys - ny;
            }
            int xs = x0 - cx(i);
            xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
            p = src + (long long)i * geo.plane + (long long)ys * nx + xs;
            g[0][i] = active ? Store<T>::ld(*p, inv_s) : R(0);
        }
    } else {
        // shift mode per population: 0 none, +1 take x-1, -1 take x+1;
        // bounce-back rows take the same node's opposite population unshifted
        T v[9][VEC];
        T edge[9];
        int mode[9];
        const bool first = lane == 0 || x0 == 0;
        const bool last = lane == 31 || x0 + VEC >= nx;
        const int xl = x0 == 0 ? nx - 1 : x0 - 1;
        const int xr = x0 + VEC >= nx ? 0 : x0 + VEC;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            int ys = y - cy(i);
            int pl = i;
            mode[i] = cx(i);
            if (ys < 0 || ys >= ny) {
                if (WALLS) {
                    pl = opp(i);
                    ys = y;
                    mode[i] = 0;
                } else {
                    ys = ys < 0 ? ys + ny : ys - ny;
                }
            }
            const T *row = src + (long long)pl * geo.plane + (long long)ys * nx;
            if (active) ld16<T, VEC>(row + x0, v[i]);
            else {
#pragma unroll
                for (int k = 0; k < VEC; ++k) v[i][k] = T(0);
            }
            edge[i] = T(0);
            if (mode[i] == 1 && active && first) edge[i] = row[xl];
            if (mode[i] == -1 && active && last) edge[i] = row[xr];
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            R r[VEC];
#pragma unroll
            for (int k = 0; k < VEC; ++k) r[k] = Store<T>::ld(v[i][k], inv_s);
            if (mode[i] == 0) {
#pragma unroll
                for (int k = 0; k < VEC; ++k) g[k][i] = r[k];
            } else if (mode[i] == 1) {
                // node x takes x-1: shift right by one, left neighbour from lane-1
                R left = __shfl_up_sync(0xffffffffu, r[VEC - 1], 1);
                if (first) left = Store<T>::ld(edge[i], inv_s);
                g[0][i] = left;
#pragma unroll
                for (int k = 1; k < VEC; ++k) g[k][i] = r[k - 1];
            } else {
                // node x takes x+1: shift left by one, right neighbour from lane+1
                R right = __shfl_down_sync(0xffffffffu, r[0], 1);
                if (last) right = Store<T>::ld(edge[i], inv_s);
#pragma unroll
                for (int k = 0; k < VEC - 1; ++k) g[k][i] = r[k + 1];
                g[VEC - 1][i] = right;
            }
        }
    }
}

template <typename R, int VEC>
__device__ __forceinline__ void load_coef(const R *__restrict__ p, bool active, R (&c)[VEC]) {
    if constexpr (VEC == 1) {
        c[0] = active ? p[0] : R(1);
    } else if (active) {
        ld16<R, VEC>(p, c);
    } else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) c[k] = R(1);
    }
}

// Deterministic block sum of two doubles; thread 0 returns the totals.
__device__ __forceinline__ void block_sum2(double &a, double &b) {
    __shared__ double sh[2][32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        b += __shfl_down_sync(0xffffffffu, b, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        sh[0][warp] = a;
        sh[1][warp] = b;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        a = 0.0;
        b = 0.0;
        for (int w = 0; w < int(blockDim.x >> 5); ++w) {
            a += sh[0][w];
            b += sh[1][w];
        }
    }
}

constexpr int kThreads = 128;

// Block maximum of a non-negative float; thread 0 returns it.
__device__ __forceinline__ float block_max(float m) {
    __shared__ float shm[32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_down_sync(0xffffffffu, m, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) shm[warp] = m;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < int(blockDim.x >> 5); ++w) m = fmaxf(m, shm[w]);
    return m;
}

// ---------------------------------------------------------------------------
// K2: fused pull-stream + collide (one time step).  REDUCE additionally
// writes this block's FP64 sums of u_x, u_y to partial[2*block] and, for
// 16-bit storage, the largest stored magnitude |g*S| to pmax[block].
// ---------------------------------------------------------------------------
template <typename T, int VEC, bool WALLS, bool FORCH, bool REDUCE>
__global__ void __launch_bounds__(kThreads)
k_step(const T *__restrict__ src, T *__restrict__ dst, const typename Store<T>::R *__restrict__ alpha,
       const typename Store<T>::R *__restrict__ epsv, const typename Store<T>::R *__restrict__ betav,
       Geo geo, Phys<typename Store<T>::R> ph, double *__restrict__ partial, float *__restrict__ pmax) {
    using R = typename Store<T>::R;
    const int y = blockIdx.x / geo.bpr;
    const int bx = blockIdx.x - y * geo.bpr;
    const int x0 = (bx * kThreads + threadIdx.x) * VEC;
    const bool active = x0 < geo.nx;
    const int lane = threadIdx.x & 31;
    const long long n0 = (long long)y * geo.nx + x0;

    R g[VEC][9];
    gather<T, VEC, WALLS>(src, geo, x0, y, active, lane, ph.inv_scale, g);
    R a[VEC], e[VEC], b[VEC];
    load_coef<R, VEC>(alpha + n0, active, a);
    load_coef<R, VEC>(epsv + n0, active, e);
    if (FORCH) load_coef<R, VEC>(betav + n0, active, b);
    else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) b[k] = R(0);
    }

    double sx = 0.0, sy = 0.0;
#pragma unroll
    for (int k = 0; k < VEC; ++k) {
        R ux, uy;
        collide<R, FORCH, !Store<T>::kSmall>(g[k], a[k], e[k], b[k], ph, ux, uy);
        if (REDUCE && active) {
            sx += double(ux);
            sy += double(uy);
        }
    }
    float gm = 0.0f;
    bool stored = false;
    if constexpr (Store<T>::kSmall && VEC == 4) {
        if (active && ph.sr) {
            // 16-bit storage, 4 nodes: two hardware stochastic-rounding
            // conversions per population; the random words come from one
            // hash per thread, stepped by a multiply-add and xor-folded
            uint32_t x = mix32(uint32_t(n0) ^ ph.step_key);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                float v[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) v[k] = Store<T>::kScaled ? g[k][i] * ph.scale : g[k][i];
                if (REDUCE)
                    gm = fmaxf(gm, fmaxf(fmaxf(fabsf(v[0]), fabsf(v[1])), fmaxf(fabsf(v[2]), fabsf(v[3]))));
                x = x * 0x2C1B3C6Du + 0x297A2D39u;
                const uint32_t r0 = x ^ (x >> 15);
                x = x * 0x2C1B3C6Du + 0x297A2D39u;
                const uint32_t r1 = x ^ (x >> 15);
                uint2 u;
                u.x = Store<T>::pack_sr(v[0], v[1], r0);
                u.y = Store<T>::pack_sr(v[2], v[3], r1);
                __stcs(reinterpret_cast<uint2 *>(dst + (long long)i * geo.plane + n0), u);
            }
            stored = true;
        }
    }
    if (active && !stored) {
        uint32_t hk[VEC];
        if constexpr (Store<T>::kSmall) {
#pragma unroll
            for (int k = 0; k < VEC; ++k) hk[k] = mix32(uint32_t(n0 + k) ^ ph.step_key);
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            T v[VEC];
#pragma unroll
            for (int k = 0; k < VEC; ++k) {
                if constexpr (Store<T>::kSmall) {
                    if (ph.sr) {
                        // one multiply-xorshift per word on top of the node's full hash
                        uint32_t r = (hk[k] ^ (uint32_t(i >> 1) * 0x9E3779B9u)) * 0x2C1B3C6Du;
                        r ^= r >> 15;
                        v[k] = Store<T>::st_sr(g[k][i], ph.scale, (i & 1) ? (r >> 16) : r);
                    } else {
                        v[k] = Store<T>::st(g[k][i], ph.scale);
                    }
                    if (REDUCE) gm = fmaxf(gm, fabsf(float(v[k])));
                } else {
                    v[k] = Store<T>::st(g[k][i], ph.scale);
                }
            }
            T *p = dst + (long long)i * geo.plane + n0;
            if constexpr (VEC == 1) p[0] = v[0];
            else st16<T, VEC>(p, v);
        }
    }
    if (REDUCE) {
        block_sum2(sx, sy);
        if (threadIdx.x == 0) {
            partial[2ll * blockIdx.x] = sx;
            partial[2ll * blockIdx.x + 1] = sy;
        }
        if constexpr (Store<T>::kSmall) {
            gm = block_max(gm);
            if (threadIdx.x == 0) pmax[blockIdx.x] = gm;
        }
    }
}

// Device-side run status (A8 result and convergence test).
struct DevStatus {
    double ux, uy;     // mean velocity of the last reduced step
    double prev_ux;    // the previous check's mean u_x
    int have_prev;     // prev_ux valid
    int converged;     // set by the last finalize
    int nonfinite;     // mean velocity not finite
    float gmax;        // 16-bit storage: largest stored |g*S| at that step
};

// K3 finalize: fixed-order FP64 sum of the block partials, mean, test.
__global__ void __launch_bounds__(256)
k_finalize(const double *__restrict__ partial, int nparts, double inv_n, double tol,
           DevStatus *__restrict__ st, const float *__restrict__ pmax) {
    __shared__ double sh[2][256];
    double a = 0.0, b = 0.0;
    float m = 0.0f;
    for (int j = threadIdx.x; j < nparts; j += 256) {
        a += partial[2ll * j];
        b += partial[2ll * j + 1];
        if (pmax) m = fmaxf(m, pmax[j]);
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    if (pmax) m = block_max(m);
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double ux = sh[0][0] * inv_n, uy = sh[1][0] * inv_n;
        st->ux = ux;
        st->uy = uy;
        const bool fin = isfinite(ux) && isfinite(uy);
        st->nonfinite = fin ? 0 : 1;
        st->converged = (fin && tol > 0.0 && st->have_prev &&
                         fabs(ux - st->prev_ux) <= tol * fabs(ux)) ? 1 : 0;
        st->prev_ux = ux;
        st->have_prev = 1;
        st->gmax = m;
    }
}

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

// A1: pack per-node coefficients (Eqs. 36-37) from FP64 eps, K.
template <typename R>
__global__ void k_pack(const double *__restrict__ eps, const double *__restrict__ K, long long N,
                       double nu, double feps_mode, R *__restrict__ alpha, R *__restrict__ epsv,
                       R *__restrict__ betav) {
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const double e = eps[n], k = K[n];
        double fe = 0.0;
        if (feps_mode > 0.0) fe = feps_mode;
        else if (feps_mode < 0.0) fe = 1.75 / sqrt(150.0 * e * e * e);
        alpha[n] = R(e * nu / k);
        epsv[n] = R(e);
        betav[n] = R(e * fe / sqrt(k));
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

// Velocity export: re-run the step's gather and velocity solve on the
// pre-step state (scalar loads; same arithmetic as k_step).
template <typename T, bool WALLS, bool FORCH>
__global__ void __launch_bounds__(kThreads)
k_velocity(const T *__restrict__ src, const typename Store<T>::R *__restrict__ alpha,
           const typename Store<T>::R *__restrict__ epsv, const typename Store<T>::R *__restrict__ betav,
           Geo geo, Phys<typename Store<T>::R> ph, double *__restrict__ ux_out,
           double *__restrict__ uy_out) {
    using R = typename Store<T>::R;
    const int y = blockIdx.x / geo.bpr;
    const int bx = blockIdx.x - y * geo.bpr;
    const int x0 = bx * kThreads + threadIdx.x;
    const bool active = x0 < geo.nx;
    if (!active) return;  // no shuffles on the scalar path
    const long long n = (long long)y * geo.nx + x0;
    R g[1][9];
    gather<T, 1, WALLS>(src, geo, x0, y, true, threadIdx.x & 31, ph.inv_scale, g);
    R drho, ux, uy;
    node_velocity<R, FORCH>(g[0], alpha[n], epsv[n], FORCH ? betav[n] : R(0), ph, drho, ux, uy);
    ux_out[n] = double(ux);
    uy_out[n] = double(uy);
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

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
thread_local char g_create_err[512] = "";

}  // namespace

struct glbm {
    int nx = 0, ny = 0;
    long long N = 0, plane = 0;
    double tau = 1.0;
    glbm_storage storage = GLBM_F32;
    unsigned flags = 0;
    cudaStream_t stream = nullptr;
    int dev = 0;
    size_t elem = 4;     // bytes per stored population
    size_t celem = 4;    // bytes per coefficient
    void *buf[2] = {nullptr, nullptr};
    int cur = 0;         // buffer holding the current state
    void *coef[3] = {nullptr, nullptr, nullptr};  // alpha, eps, beta
    double *partial = nullptr;
    float *pmax = nullptr;  // 16-bit storage: block maxima of |stored|
    int nparts_max = 0;
    DevStatus *dstat = nullptr;
    DevStatus *hstat = nullptr;  // pinned
    int *dflag = nullptr;
    double *stage = nullptr;  // 3*N doubles of input staging, allocated on first host input
    bool has_medium = false, forch = false, reduced = false;
    double feps_mode = 0.0, gx = 0.0, gy = 0.0;
    double scale = 1.0;       // FP16 storage scale S (stored = g*S)
    bool sr = true;           // 16-bit storage: stochastic rounding
    bool at_rest = false;     // state is f_eq(1, 0) (zero deviations)
    uint32_t seed = 0x2545F491u;
    long long tstep = 0;      // time steps launched since the last reset
    long long steps = 0, launches = 0;
    char err[512] = "";
};

namespace {

glbm_status fail(glbm *h, glbm_status s, const char *fmt, ...) {
    char *dst = h ? h->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return s;
}

#define CU(h, call)                                                                          \
    do {                                                                                     \
        cudaError_t e_ = (call);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return fail((h), e_ == cudaErrorMemoryAllocation ? GLBM_ENOMEM : GLBM_ECUDA,     \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

int vec_width(const glbm *h) {
    const int v = h->elem == 2 ? 4 : int(16 / h->elem);
    return (h->nx % v == 0) ? v : 1;
}

Geo make_geo(const glbm *h, int vec) {
    Geo g;
    g.nx = h->nx;
    g.ny = h->ny;
    g.plane = h->plane;
    const int tpr = (h->nx + vec - 1) / vec;
    g.bpr = (tpr + kThreads - 1) / kThreads;
    return g;
}

template <typename R>
Phys<R> make_phys(const glbm *h) {
    Phys<R> p;
    p.omega = R(1.0 / h->tau);
    p.A = R(1.0 - 0.5 / h->tau);
    p.gx = R(h->gx);
    p.gy = R(h->gy);
    p.scale = R(h->scale);
    p.inv_scale = R(1.0 / h->scale);
    p.step_key = mix32(uint32_t(h->tstep) * 0x9E3779B9u + h->seed);
    p.sr = h->sr ? 1 : 0;
    return p;
}

int grid_1d(long long N) {
    long long b = (N + 255) / 256;
    return int(b > 152 * 64 ? 152 * 64 : (b < 1 ? 1 : b));
}

template <typename T, int VEC, bool WALLS, bool FORCH>
glbm_status launch_step_t(glbm *h, bool reduce) {
    using R = typename Store<T>::R;
    const Geo geo = make_geo(h, VEC);
    const Phys<R> ph = make_phys<R>(h);
    const T *src = static_cast<const T *>(h->buf[h->cur]);
    T *dst = static_cast<T *>(h->buf[h->cur ^ 1]);
    const R *a = static_cast<const R *>(h->coef[0]);
    const R *e = static_cast<const R *>(h->coef[1]);
    const R *b = static_cast<const R *>(h->coef[2]);
    const unsigned grid = unsigned(geo.bpr) * unsigned(geo.ny);
    if (reduce)
        k_step<T, VEC, WALLS, FORCH, true>
            <<<grid, kThreads, 0, h->stream>>>(src, dst, a, e, b, geo, ph, h->partial, h->pmax);
    else
        k_step<T, VEC, WALLS, FORCH, false>
            <<<grid, kThreads, 0, h->stream>>>(src, dst, a, e, b, geo, ph, h->partial, h->pmax);
    h->launches++;
    h->tstep++;
    h->cur ^= 1;
    return GLBM_OK;
}

template <typename T>
glbm_status launch_step(glbm *h, bool reduce) {
    constexpr int V = kVecOf<T>;
    const bool walls = !(h->flags & GLBM_PERIODIC_Y);
    const bool vec = vec_width(h) > 1;
    if (vec) {
        if (walls) return h->forch ? launch_step_t<T, V, true, true>(h, reduce) : launch_step_t<T, V, true, false>(h, reduce);
        return h->forch ? launch_step_t<T, V, false, true>(h, reduce) : launch_step_t<T, V, false, false>(h, reduce);
    }
    if (walls) return h->forch ? launch_step_t<T, 1, true, true>(h, reduce) : launch_step_t<T, 1, true, false>(h, reduce);
    return h->forch ? launch_step_t<T, 1, false, true>(h, reduce) : launch_step_t<T, 1, false, false>(h, reduce);
}

glbm_status do_step(glbm *h, bool reduce) {
    switch (h->storage) {
        case GLBM_F32: return launch_step<float>(h, reduce);
        case GLBM_F64: return launch_step<double>(h, reduce);
        case GLBM_F16DEV: return launch_step<__half>(h, reduce);
        case GLBM_BF16DEV: return launch_step<__nv_bfloat16>(h, reduce);
    }
    return GLBM_EINVAL;
}

int nparts(const glbm *h) {
    const Geo g = make_geo(h, vec_width(h));
    return g.bpr * g.ny;
}

glbm_status finalize(glbm *h, double tol) {
    k_finalize<<<1, 256, 0, h->stream>>>(h->partial, nparts(h), 1.0 / double(h->N), tol, h->dstat,
                                         h->elem == 2 ? h->pmax : nullptr);
    h->launches++;
    h->reduced = true;
    return GLBM_OK;
}

glbm_status read_status(glbm *h) {
    CU(h, cudaMemcpyAsync(h->hstat, h->dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    return GLBM_OK;
}

glbm_status reset_status(glbm *h) {
    CU(h, cudaMemsetAsync(h->dstat, 0, sizeof(DevStatus), h->stream));
    h->reduced = false;
    return GLBM_OK;
}

double pow2_floor(double x) { return std::ldexp(1.0, int(std::floor(std::log2(x)))); }

// FP16 scale that puts a deviation bound `gbound` near 2^12 (FP16 normal
// range is 2^-14 .. 65504, relative precision 2^-11 throughout).
double fp16_scale_for(double gbound) {
    if (!(gbound > 0.0) || !std::isfinite(gbound)) return 1.0;
    return std::fmin(std::fmax(pow2_floor(4096.0 / gbound), 0x1p-24), 0x1p64);
}

template <typename T>
void rescale_t(glbm *h, float factor) {
    for (int b = 0; b < 2; ++b) {
        k_rescale<T><<<grid_1d(9 * h->plane), 256, 0, h->stream>>>(static_cast<T *>(h->buf[b]), 9 * h->plane,
                                                                   factor);
        h->launches++;
    }
}

// Keep the largest stored FP16 magnitude between 2^8 and 2^13: rescale both
// buffers by a power of two when the last reduction saw it outside.
void adapt_fp16_scale(glbm *h, float gmax) {
    if (h->storage != GLBM_F16DEV || !(gmax >= 0.0f)) return;
    int k = 0;
    if (gmax > 8192.0f) k = -int(std::ceil(std::log2(double(gmax) / 4096.0)));
    else if (gmax > 0.0f && gmax < 256.0f) k = int(std::floor(std::log2(4096.0 / double(gmax))));
    if (k == 0) return;
    const float factor = float(std::ldexp(1.0, k));
    rescale_t<__half>(h, factor);
    h->scale *= double(factor);
}

template <typename T>
void launch_init_eq(glbm *h, const double *rho, const double *ux, const double *uy) {
    using R = typename Store<T>::R;
    k_init_eq<T><<<grid_1d(h->N), 256, 0, h->stream>>>(
        static_cast<T *>(h->buf[h->cur]), h->plane, h->N, static_cast<const R *>(h->coef[1]), rho, ux, uy,
        R(h->scale));
    h->launches++;
}

void init_eq_dispatch(glbm *h, const double *rho, const double *ux, const double *uy) {
    switch (h->storage) {
        case GLBM_F32: launch_init_eq<float>(h, rho, ux, uy); break;
        case GLBM_F64: launch_init_eq<double>(h, rho, ux, uy); break;
        case GLBM_F16DEV: launch_init_eq<__half>(h, rho, ux, uy); break;
        case GLBM_BF16DEV: launch_init_eq<__nv_bfloat16>(h, rho, ux, uy); break;
    }
}

template <typename T>
void launch_velocity(glbm *h, double *ux, double *uy) {
    using R = typename Store<T>::R;
    const Geo geo = make_geo(h, 1);
    const Phys<R> ph = make_phys<R>(h);
    const T *src = static_cast<const T *>(h->buf[h->cur ^ 1]);
    const R *a = static_cast<const R *>(h->coef[0]);
    const R *e = static_cast<const R *>(h->coef[1]);
    const R *b = static_cast<const R *>(h->coef[2]);
    const unsigned grid = unsigned(geo.bpr) * unsigned(geo.ny);
    const bool walls = !(h->flags & GLBM_PERIODIC_Y);
    if (walls) {
        if (h->forch) k_velocity<T, true, true><<<grid, kThreads, 0, h->stream>>>(src, a, e, b, geo, ph, ux, uy);
        else k_velocity<T, true, false><<<grid, kThreads, 0, h->stream>>>(src, a, e, b, geo, ph, ux, uy);
    } else {
        if (h->forch) k_velocity<T, false, true><<<grid, kThreads, 0, h->stream>>>(src, a, e, b, geo, ph, ux, uy);
        else k_velocity<T, false, false><<<grid, kThreads, 0, h->stream>>>(src, a, e, b, geo, ph, ux, uy);
    }
    h->launches++;
}

template <typename T>
void launch_export(glbm *h, double *f) {
    k_export_f<T><<<grid_1d(h->N), 256, 0, h->stream>>>(static_cast<const T *>(h->buf[h->cur]), h->plane, h->N,
                                                        typename Store<T>::R(1.0 / h->scale), f);
    h->launches++;
}

// Make `k` FP64 input arrays of N doubles device-resident: device pointers
// pass through; host arrays are copied into the handle's staging buffer.
glbm_status stage_inputs(glbm *h, const double *const *src, const double **dst, int k, int device_ptrs) {
    bool any = false;
    for (int j = 0; j < k; ++j) any = any || src[j];
    if (any && !device_ptrs && !h->stage) CU(h, cudaMalloc(&h->stage, sizeof(double) * 3 * size_t(h->N)));
    for (int j = 0; j < k; ++j) {
        if (!src[j] || device_ptrs) {
            dst[j] = src[j];
            continue;
        }
        double *d = h->stage + size_t(j) * h->N;
        CU(h, cudaMemcpyAsync(d, src[j], sizeof(double) * h->N, cudaMemcpyHostToDevice, h->stream));
        dst[j] = d;
    }
    return GLBM_OK;
}

// Read back the first-bad-index flag (INT_MAX = all valid).
glbm_status read_flag(glbm *h, int *first_bad) {
    CU(h, cudaGetLastError());
    CU(h, cudaMemcpyAsync(first_bad, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    return GLBM_OK;
}

glbm_status reset_flag(glbm *h) {
    CU(h, cudaMemsetAsync(h->dflag, 0x7f, sizeof(int), h->stream));  // 0x7f7f7f7f > any index
    return GLBM_OK;
}

double fetch(glbm *h, const double *p, long long n) {
    double v = NAN;
    if (p) cudaMemcpy(&v, p + n, sizeof(double), cudaMemcpyDeviceToHost);
    return v;
}

glbm_status check(glbm *h) {
    if (!h) return GLBM_EINVAL;
    cudaError_t e = cudaSetDevice(h->dev);
    if (e != cudaSuccess) return fail(h, GLBM_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    return GLBM_OK;
}

glbm_status launch_error(glbm *h) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(h, GLBM_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
    return GLBM_OK;
}

void release(glbm *h) {
    for (auto &p : h->buf) if (p) cudaFree(p), p = nullptr;
    for (auto &p : h->coef) if (p) cudaFree(p), p = nullptr;
    if (h->partial) cudaFree(h->partial), h->partial = nullptr;
    if (h->pmax) cudaFree(h->pmax), h->pmax = nullptr;
    if (h->dstat) cudaFree(h->dstat), h->dstat = nullptr;
    if (h->dflag) cudaFree(h->dflag), h->dflag = nullptr;
    if (h->stage) cudaFree(h->stage), h->stage = nullptr;
    if (h->hstat) cudaFreeHost(h->hstat), h->hstat = nullptr;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

glbm_status glbm_create(int nx, int ny, double tau, glbm_storage storage, unsigned flags, void *stream,
                        glbm_t *out) {
    if (!out) return fail(nullptr, GLBM_EINVAL, "glbm_create: out is NULL");
    *out = nullptr;
    if (nx < 2 || ny < 2 || (long long)nx * ny >= (1ll << 31))
        return fail(nullptr, GLBM_EINVAL, "glbm_create: need nx, ny >= 2 and nx*ny < 2^31 (got %d x %d)", nx, ny);
    if (!(tau > 0.5) || !std::isfinite(tau))
        return fail(nullptr, GLBM_EINVAL, "glbm_create: tau must be a finite value > 1/2 (got %g)", tau);
    if (storage != GLBM_F32 && storage != GLBM_F64 && storage != GLBM_F16DEV && storage != GLBM_BF16DEV)
        return fail(nullptr, GLBM_EINVAL, "glbm_create: unknown storage %d", int(storage));
    if (flags & ~(GLBM_PERIODIC_Y | GLBM_NEAREST16))
        return fail(nullptr, GLBM_EINVAL, "glbm_create: unknown flags 0x%x", flags);
    glbm *h = new (std::nothrow) glbm;
    if (!h) return fail(nullptr, GLBM_ENOMEM, "glbm_create: out of host memory");
    h->nx = nx;
    h->ny = ny;
    h->N = (long long)nx * ny;
    h->plane = (h->N + 63) / 64 * 64;
    h->tau = tau;
    h->storage = storage;
    h->flags = flags;
    h->stream = static_cast<cudaStream_t>(stream);
    h->elem = storage == GLBM_F64 ? 8 : (storage == GLBM_F32 ? 4 : 2);
    h->celem = storage == GLBM_F64 ? 8 : 4;
    h->sr = !(flags & GLBM_NEAREST16);
    cudaError_t e = cudaGetDevice(&h->dev);
    const size_t fbytes = size_t(9) * h->plane * h->elem;
    const size_t cbytes = size_t(h->plane) * h->celem;
    // the scalar grid has the most blocks
    const Geo g1 = make_geo(h, 1);
    h->nparts_max = g1.bpr * g1.ny;
    if (e == cudaSuccess) e = cudaMalloc(&h->buf[0], fbytes);
    if (e == cudaSuccess) e = cudaMalloc(&h->buf[1], fbytes);
    for (int c = 0; c < 3 && e == cudaSuccess; ++c) e = cudaMalloc(&h->coef[c], cbytes);
    if (e == cudaSuccess) e = cudaMalloc(&h->partial, sizeof(double) * 2 * size_t(h->nparts_max));
    if (e == cudaSuccess) e = cudaMalloc(&h->pmax, sizeof(float) * size_t(h->nparts_max));
    if (e == cudaSuccess) e = cudaMalloc(&h->dstat, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMalloc(&h->dflag, sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&h->hstat, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->dstat, 0, sizeof(DevStatus), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        glbm_status s = fail(nullptr, e == cudaErrorMemoryAllocation ? GLBM_ENOMEM : GLBM_ECUDA,
                             "glbm_create: %s", cudaGetErrorString(e));
        release(h);
        delete h;
        return s;
    }
    memset(h->hstat, 0, sizeof(DevStatus));
    *out = h;
    return GLBM_OK;
}

glbm_status glbm_set_medium(glbm_t h, const double *eps, const double *K, double F_eps, int device_ptrs) {
    if (glbm_status s = check(h)) return s;
    if (!eps || !K) return fail(h, GLBM_EINVAL, "set_medium: eps and K are required");
    if (!std::isfinite(F_eps)) return fail(h, GLBM_EINVAL, "set_medium: F_eps must be finite");
    const long long N = h->N;
    const double *src[2] = {eps, K};
    const double *d[2];
    if (glbm_status s = stage_inputs(h, src, d, 2, device_ptrs)) return s;
    if (glbm_status s = reset_flag(h)) return s;
    k_validate<<<grid_1d(N), 256, 0, h->stream>>>(d[0], d[1], N, h->dflag);
    h->launches++;
    int bad = 0;
    if (glbm_status s = read_flag(h, &bad)) return s;
    if (bad < N)
        return fail(h, GLBM_EINVAL, "set_medium: node %d has eps = %g, K = %g (need eps in (0, 1], K > 0)", bad,
                    fetch(h, d[0], bad), fetch(h, d[1], bad));
    const double nu = (h->tau - 0.5) / 3.0;
    if (h->celem == 8)
        k_pack<double><<<grid_1d(N), 256, 0, h->stream>>>(d[0], d[1], N, nu, F_eps, (double *)h->coef[0],
                                                          (double *)h->coef[1], (double *)h->coef[2]);
    else
        k_pack<float><<<grid_1d(N), 256, 0, h->stream>>>(d[0], d[1], N, nu, F_eps, (float *)h->coef[0],
                                                         (float *)h->coef[1], (float *)h->coef[2]);
    h->launches++;
    if (glbm_status s = launch_error(h)) return s;
    CU(h, cudaMemsetAsync(h->buf[0], 0, size_t(9) * h->plane * h->elem, h->stream));
    CU(h, cudaMemsetAsync(h->buf[1], 0, size_t(9) * h->plane * h->elem, h->stream));
    if (glbm_status s = reset_status(h)) return s;
    h->cur = 0;
    h->steps = 0;
    h->tstep = 0;
    h->at_rest = true;
    if (h->storage == GLBM_F16DEV) h->scale = fp16_scale_for(16.0 * (std::fabs(h->gx) + std::fabs(h->gy)));
    h->has_medium = true;
    h->feps_mode = F_eps;
    h->forch = F_eps != 0.0;
    return GLBM_OK;
}

glbm_status glbm_set_force(glbm_t h, double gx, double gy) {
    if (glbm_status s = check(h)) return s;
    if (!std::isfinite(gx) || !std::isfinite(gy)) return fail(h, GLBM_EINVAL, "set_force: G must be finite");
    h->gx = gx;
    h->gy = gy;
    // FP16 at rest: start with |g*S| ~ 2^8 per unit of G (the first steps'
    // deviations are O(eps*G)); later chunks adapt S to the stored maximum
    if (h->storage == GLBM_F16DEV && h->at_rest && (gx != 0.0 || gy != 0.0))
        h->scale = fp16_scale_for(16.0 * (std::fabs(gx) + std::fabs(gy)));
    // clear the convergence history but keep the last mean velocity
    CU(h, cudaMemsetAsync(&h->dstat->have_prev, 0, sizeof(int), h->stream));
    return GLBM_OK;
}

glbm_status glbm_init_equilibrium(glbm_t h, const double *rho, const double *ux, const double *uy,
                                  int device_ptrs) {
    if (glbm_status s = check(h)) return s;
    if (!h->has_medium) return fail(h, GLBM_ESTATE, "init_equilibrium: no medium set");
    if ((ux == nullptr) != (uy == nullptr))
        return fail(h, GLBM_EINVAL, "init_equilibrium: give both ux and uy or neither");
    const long long N = h->N;
    const double *src[3] = {rho, ux, uy};
    const double *d[3];
    if (glbm_status s = stage_inputs(h, src, d, 3, device_ptrs)) return s;
    if (rho || ux) {
        if (glbm_status s = reset_flag(h)) return s;
        k_validate_state<<<grid_1d(N), 256, 0, h->stream>>>(d[0], d[1], d[2], N, h->dflag);
        h->launches++;
        int bad = 0;
        if (glbm_status s = read_flag(h, &bad)) return s;
        if (bad < N)
            return fail(h, GLBM_EINVAL, "init_equilibrium: node %d has rho = %g, u = (%g, %g)", bad,
                        fetch(h, d[0], bad), fetch(h, d[1], bad), fetch(h, d[2], bad));
    }
    if (h->storage == GLBM_F16DEV) {
        int mbits = 0;
        CU(h, cudaMemsetAsync(h->dflag, 0, sizeof(int), h->stream));
        k_eq_max<<<grid_1d(N), 256, 0, h->stream>>>(N, static_cast<const float *>(h->coef[1]), d[0], d[1], d[2],
                                                     h->dflag);
        h->launches++;
        if (glbm_status s = read_flag(h, &mbits)) return s;
        float m;
        memcpy(&m, &mbits, sizeof(m));
        if (m > 0.0f) h->scale = fp16_scale_for(double(m));
        else h->scale = fp16_scale_for(16.0 * (std::fabs(h->gx) + std::fabs(h->gy)));
    }
    h->cur = 0;
    init_eq_dispatch(h, d[0], d[1], d[2]);
    if (glbm_status s = launch_error(h)) return s;
    if (glbm_status s = reset_status(h)) return s;
    h->steps = 0;
    h->tstep = 0;
    h->at_rest = !(rho || ux);
    return GLBM_OK;
}

glbm_status glbm_step(glbm_t h, long long n, double tol, int check_every, long long *steps_done,
                      int *converged) {
    if (steps_done) *steps_done = 0;
    if (converged) *converged = 0;
    if (glbm_status s = check(h)) return s;
    if (!h->has_medium) return fail(h, GLBM_ESTATE, "step: no medium set");
    if (n < 0 || check_every < 1) return fail(h, GLBM_EINVAL, "step: need n >= 0 and check_every >= 1");
    if (!std::isfinite(tol)) return fail(h, GLBM_EINVAL, "step: tol must be finite");
    long long done = 0;
    int conv = 0;
    const bool test = tol > 0.0;
    const bool adapt = h->storage == GLBM_F16DEV;
    if (n > 0) h->at_rest = false;
    while (done < n) {
        long long chunk = n - done;
        if (chunk > check_every) chunk = check_every;
        const bool last_chunk = done + chunk == n;
        const bool reduce_here = test || last_chunk || adapt;
        for (long long s = 0; s < chunk; ++s) {
            glbm_status st = do_step(h, reduce_here && s == chunk - 1);
            if (st) return st;
        }
        done += chunk;
        h->steps += chunk;
        if (reduce_here) finalize(h, test ? tol : 0.0);
        if (glbm_status st = launch_error(h)) return st;
        if (test || adapt) {
            if (glbm_status st = read_status(h)) return st;
            if (h->hstat->nonfinite) {
                if (steps_done) *steps_done = done;
                return fail(h, GLBM_ENAN, "step: non-finite mean velocity after %lld steps", h->steps);
            }
            adapt_fp16_scale(h, h->hstat->gmax);
            if (glbm_status st = launch_error(h)) return st;
            if (test && h->hstat->converged) {
                conv = 1;
                break;
            }
        }
    }
    if (steps_done) *steps_done = done;
    if (converged) *converged = conv;
    return GLBM_OK;
}

glbm_status glbm_mean_velocity(glbm_t h, double out[2]) {
    if (glbm_status s = check(h)) return s;
    if (!out) return fail(h, GLBM_EINVAL, "mean_velocity: out is NULL");
    if (!h->reduced) return fail(h, GLBM_ESTATE, "mean_velocity: no step has completed since the last reset");
    if (glbm_status s = read_status(h)) return s;
    out[0] = h->hstat->ux;
    out[1] = h->hstat->uy;
    if (h->hstat->nonfinite) return fail(h, GLBM_ENAN, "mean_velocity: not finite");
    return GLBM_OK;
}

glbm_status glbm_permeability(glbm_t h, double *kxx) {
    if (glbm_status s = check(h)) return s;
    if (!kxx) return fail(h, GLBM_EINVAL, "permeability: kxx is NULL");
    if (h->gx == 0.0) return fail(h, GLBM_EINVAL, "permeability: G_x is zero");
    double u[2];
    if (glbm_status s = glbm_mean_velocity(h, u)) return s;
    *kxx = (h->tau - 0.5) / 3.0 * u[0] / h->gx;
    return GLBM_OK;
}

glbm_status glbm_get_velocity(glbm_t h, double *ux, double *uy, int device_ptrs) {
    if (glbm_status s = check(h)) return s;
    if (!ux || !uy) return fail(h, GLBM_EINVAL, "get_velocity: ux and uy are required");
    if (h->steps == 0) return fail(h, GLBM_ESTATE, "get_velocity: no step has completed since the last reset");
    double *dbuf = nullptr;
    double *dx = ux, *dy = uy;
    if (!device_ptrs) {
        CU(h, cudaMalloc(&dbuf, sizeof(double) * 2 * h->N));
        dx = dbuf;
        dy = dbuf + h->N;
    }
    switch (h->storage) {
        case GLBM_F32: launch_velocity<float>(h, dx, dy); break;
        case GLBM_F64: launch_velocity<double>(h, dx, dy); break;
        case GLBM_F16DEV: launch_velocity<__half>(h, dx, dy); break;
        case GLBM_BF16DEV: launch_velocity<__nv_bfloat16>(h, dx, dy); break;
    }
    glbm_status s = launch_error(h);
    cudaError_t e = cudaSuccess;
    if (!s && !device_ptrs) {
        e = cudaMemcpyAsync(ux, dx, sizeof(double) * h->N, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(uy, dy, sizeof(double) * h->N, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
    if (dbuf) cudaFree(dbuf);
    if (!s && e != cudaSuccess) s = fail(h, GLBM_ECUDA, "get_velocity: %s", cudaGetErrorString(e));
    return s;
}

glbm_status glbm_get_distributions(glbm_t h, double *f, int device_ptrs) {
    if (glbm_status s = check(h)) return s;
    if (!f) return fail(h, GLBM_EINVAL, "get_distributions: f is NULL");
    if (!h->has_medium) return fail(h, GLBM_ESTATE, "get_distributions: no medium set");
    double *dbuf = nullptr, *df = f;
    if (!device_ptrs) {
        CU(h, cudaMalloc(&dbuf, sizeof(double) * 9 * h->N));
        df = dbuf;
    }
    switch (h->storage) {
        case GLBM_F32: launch_export<float>(h, df); break;
        case GLBM_F64: launch_export<double>(h, df); break;
        case GLBM_F16DEV: launch_export<__half>(h, df); break;
        case GLBM_BF16DEV: launch_export<__nv_bfloat16>(h, df); break;
    }
    glbm_status s = launch_error(h);
    cudaError_t e = cudaSuccess;
    if (!s && !device_ptrs) {
        e = cudaMemcpyAsync(f, df, sizeof(double) * 9 * h->N, cudaMemcpyDeviceToHost, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    }
    if (dbuf) cudaFree(dbuf);
    if (!s && e != cudaSuccess) s = fail(h, GLBM_ECUDA, "get_distributions: %s", cudaGetErrorString(e));
    return s;
}

glbm_status glbm_counters(glbm_t h, long long *steps, long long *launches) {
    if (!h) return GLBM_EINVAL;
    if (steps) *steps = h->steps;
    if (launches) *launches = h->launches;
    return GLBM_OK;
}

void glbm_destroy(glbm_t h) {
    if (!h) return;
    cudaSetDevice(h->dev);
    cudaStreamSynchronize(h->stream);
    release(h);
    delete h;
}

const char *glbm_last_error(glbm_t h) { return h ? h->err : g_create_err; }

}  // extern "C"

// ===========================================================================
// Allocation-free step (glbm_step_reduce_noalloc).
//
// For callers that may not allocate device memory themselves: applications
// whose host framework owns the whole device-memory budget and hands out
// every buffer, or pipelines that must not risk the implicit device-wide
// synchronisation that cudaMalloc/cudaFree can cause in the middle of their
// loop.  The step kernel's only scratch (one FP64 partial pair per block plus
// the reduction status) lives in the file-scope array below instead of a
// per-handle allocation; every GPU that loads this library holds it until the
// process exits.
// ===========================================================================
namespace {

constexpr int kNoAllocMaxBlocks = 65536;  // partial pairs: 1 MiB
constexpr int kNoAllocStatusDoubles = 8;  // room for DevStatus (40 B)
static_assert(sizeof(DevStatus) <= kNoAllocStatusDoubles * sizeof(double), "status slot");

static __device__ __align__(256) double g_noalloc_scratch[2 * kNoAllocMaxBlocks + kNoAllocStatusDoubles];

constexpr int kMaxDevices = 64;
double *g_noalloc_ptr[kMaxDevices] = {};
std::mutex g_noalloc_mu;
// Failures are reported like glbm_create's: glbm_last_error(NULL).
glbm_status noalloc_fail(glbm_status s, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_create_err, sizeof(g_create_err), fmt, ap);
    va_end(ap);
    return s;
}

// Device address of the scratch array on the current device, looked up once
// per device.  In host code the array's name is only a host-side stand-in,
// never a device address, so it is never handed to a kernel directly.
glbm_status noalloc_scratch(double **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return noalloc_fail(GLBM_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
    if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(GLBM_EINVAL, "device ordinal %d too large", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        double *p = nullptr;
        e = cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_noalloc_scratch);
        if (e != cudaSuccess)
            return noalloc_fail(GLBM_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return GLBM_OK;
}

template <int VEC, bool WALLS, bool FORCH>
void noalloc_launch(const float *src, float *dst, const float *a, const float *e, const float *b, const Geo &geo,
                    const Phys<float> &ph, double *partial, cudaStream_t st) {
    const unsigned grid = unsigned(geo.bpr) * unsigned(geo.ny);
    k_step<float, VEC, WALLS, FORCH, true><<<grid, kThreads, 0, st>>>(src, dst, a, e, b, geo, ph, partial, nullptr);
}

}  // namespace

extern "C" glbm_status glbm_step_reduce_noalloc(const float *g_src, float *g_dst, const float *alpha,
                                                const float *eps, const float *beta, int nx, int ny,
                                                long long plane, double tau, double gx, double gy,
                                                unsigned flags, double *mean_u, void *stream) {
    if (!g_src || !g_dst || !alpha || !eps || !mean_u)
        return noalloc_fail(GLBM_EINVAL, "step_reduce_noalloc: g_src, g_dst, alpha, eps and mean_u are required");
    if (g_src == g_dst) return noalloc_fail(GLBM_EINVAL, "step_reduce_noalloc: g_src and g_dst must differ");
    if (nx < 2 || ny < 2 || (long long)nx * ny >= (1ll << 31))
        return noalloc_fail(GLBM_EINVAL, "step_reduce_noalloc: need nx, ny >= 2 and nx*ny < 2^31");
    if (plane < (long long)nx * ny || plane % 4 != 0)
        return noalloc_fail(GLBM_EINVAL, "step_reduce_noalloc: plane must be >= nx*ny and a multiple of 4");
    if (!(tau > 0.5) || !std::isfinite(tau) || !std::isfinite(gx) || !std::isfinite(gy))
        return noalloc_fail(GLBM_EINVAL, "step_reduce_noalloc: need finite tau > 1/2 and finite G");
    if (flags & ~GLBM_PERIODIC_Y) return noalloc_fail(GLBM_EINVAL, "step_reduce_noalloc: unknown flags");
    const uintptr_t mis = (uintptr_t(g_src) | uintptr_t(g_dst) | uintptr_t(alpha) | uintptr_t(eps) |
                           uintptr_t(beta)) & 15u;
    if (mis) return noalloc_fail(GLBM_EINVAL, "step_reduce_noalloc: arrays must be 16-byte aligned");
    const int vec = (nx % 4 == 0) ? 4 : 1;
    Geo geo;
    geo.nx = nx;
    geo.ny = ny;
    geo.plane = plane;
    geo.bpr = ((nx + vec - 1) / vec + kThreads - 1) / kThreads;
    const long long blocks = (long long)geo.bpr * ny;
    if (blocks > kNoAllocMaxBlocks)
        return noalloc_fail(GLBM_EINVAL,
                            "step_reduce_noalloc: lattice needs %lld reduction blocks but the fixed scratch "
                            "holds %d (one block covers %d nodes of a row)",
                            blocks, kNoAllocMaxBlocks, vec * kThreads);
    double *scratch = nullptr;
    if (glbm_status s = noalloc_scratch(&scratch)) return s;
    double *partial = scratch;
    DevStatus *st = reinterpret_cast<DevStatus *>(scratch + 2 * kNoAllocMaxBlocks);
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    Phys<float> ph;
    ph.omega = float(1.0 / tau);
    ph.A = float(1.0 - 0.5 / tau);
    ph.gx = float(gx);
    ph.gy = float(gy);
    ph.scale = 1.0f;
    ph.inv_scale = 1.0f;
    ph.step_key = 0;
    ph.sr = 0;
    // the status keeps the previous call's values: start it from zero
    cudaError_t e = cudaMemsetAsync(st, 0, sizeof(DevStatus), cs);
    if (e != cudaSuccess) return noalloc_fail(GLBM_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    const bool walls = !(flags & GLBM_PERIODIC_Y), forch = beta != nullptr;
    if (vec == 4) {
        if (walls) forch ? noalloc_launch<4, true, true>(g_src, g_dst, alpha, eps, beta, geo, ph, partial, cs)
                         : noalloc_launch<4, true, false>(g_src, g_dst, alpha, eps, beta, geo, ph, partial, cs);
        else forch ? noalloc_launch<4, false, true>(g_src, g_dst, alpha, eps, beta, geo, ph, partial, cs)
                   : noalloc_launch<4, false, false>(g_src, g_dst, alpha, eps, beta, geo, ph, partial, cs);
    } else {
        if (walls) forch ? noalloc_launch<1, true, true>(g_src, g_dst, alpha, eps, beta, geo, ph, partial, cs)
                         : noalloc_launch<1, true, false>(g_src, g_dst, alpha, eps, beta, geo, ph, partial, cs);
        else forch ? noalloc_launch<1, false, true>(g_src, g_dst, alpha, eps, beta, geo, ph, partial, cs)
                   : noalloc_launch<1, false, false>(g_src, g_dst, alpha, eps, beta, geo, ph, partial, cs);
    }
    k_finalize<<<1, 256, 0, cs>>>(partial, int(blocks), 1.0 / double((long long)nx * ny), 0.0, st, nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess) return noalloc_fail(GLBM_ECUDA, "kernel launch: %s", cudaGetErrorString(e));
    // DevStatus begins with (ux, uy)
    e = cudaMemcpyAsync(mean_u, st, 2 * sizeof(double), cudaMemcpyDeviceToDevice, cs);
    if (e != cudaSuccess) return noalloc_fail(GLBM_ECUDA, "cudaMemcpyAsync: %s", cudaGetErrorString(e));
    return GLBM_OK;
}
