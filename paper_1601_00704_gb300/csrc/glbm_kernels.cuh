// glbm_kernels.cuh -- shared by glbm.cu (single lattice) and batch.cu (many lattices).
// Device code of the GB300 (sm_103a) generalized lattice Boltzmann model
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
//  * step_body() is the whole per-thread time step; k_step (one lattice) and
//    k_batch_step (many lattices, batch.cu) only map blocks to rows.
//  * Kernels that run once per medium or per export (validation, coefficient
//    packing, equilibrium start, FP16 rescale, f export) are in
//    setup_kernels.cuh, so this file holds the time loop alone.

#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <type_traits>
#include <utility>

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
__device__ __forceinline__ float rrcp(float a) {
    float r;  // hardware approximate reciprocal (within 1 ulp); every argument here is >= 1/2
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
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
    // 16-bit storage inside a replayed CUDA graph: when `clock` is set the
    // kernel forms its key from the device step counter instead,
    // step_key = mix32((*clock + step_off) * 0x9E3779B9 + seed), the same
    // value the host forms for step *clock + step_off.
    const unsigned *clock = nullptr;
    uint32_t step_off = 0;
    uint32_t seed = 0;
};

// Stochastic-rounding key of time step t (host and device agree).
__host__ __device__ __forceinline__ uint32_t step_key_of(uint32_t t, uint32_t seed) {
    return mix32(t * 0x9E3779B9u + seed);
}

struct Geo {
    int nx, ny;
    long long plane;  // elements per population plane
    int bpr;          // blocks per row
};

// Vector moves of 8 bytes or a multiple of 16 bytes.  CG: load through L2
// only (ld.global.cg), for data that other blocks of the same launch wrote
// (the persistent batch kernel), which a non-coherent L1 line could hide.
template <typename X, int N, bool CG = false>
__device__ __forceinline__ void ld16(const X *__restrict__ p, X (&out)[N]) {
    constexpr int B = int(N * sizeof(X));
    static_assert(B == 8 || B % 16 == 0, "8-byte or 16-byte multiple");
    if constexpr (B == 8) {
        uint2 u = CG ? __ldcg(reinterpret_cast<const uint2 *>(p)) : *reinterpret_cast<const uint2 *>(p);
        memcpy(&out[0], &u, 8);
    } else {
#pragma unroll
        for (int j = 0; j < B / 16; ++j) {
            uint4 u = CG ? __ldcg(reinterpret_cast<const uint4 *>(p) + j) : reinterpret_cast<const uint4 *>(p)[j];
            memcpy(&out[j * (16 / sizeof(X))], &u, 16);
        }
    }
}
// One element, optionally through L2 only (see ld16).
template <bool CG, typename X>
__device__ __forceinline__ X ld1(const X *p) {
    if constexpr (CG) {
        if constexpr (sizeof(X) == 2) {
            const unsigned short u = __ldcg(reinterpret_cast<const unsigned short *>(p));
            X v;
            memcpy(&v, &u, 2);
            return v;
        } else {
            return __ldcg(p);
        }
    } else {
        return *p;
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
template <typename R>
__device__ __forceinline__ void collide_pair(R &gi, R &gj, R w, R wd, R eu, R eF, R k1, R om, R su, R a2,
                                             R rho3, R fb, R f3, R f9) {
    // even:  om [rho (9/(2 eps)(e.u)^2 - 3/(2 eps) u^2)] + rho A [9/eps (e.u)(e.F) - 3/eps u.F]
    // odd :  om [3 rho e.u] + rho A [3 e.F]
    const R ev = om * (a2 * eu * eu - su) + (fb + f9 * eu * eF);
    const R od = om * rho3 * eu + f3 * eF;
    gi = wd + (k1 * (gi - wd) + w * (ev + od));
    gj = wd + (k1 * (gj - wd) + w * (ev - od));
}

// Error-free sum of g[first..8] as hi + lo (Knuth's TwoSum per addition,
// explicitly rounded so nothing is reassociated or contracted).
template <typename R>
__device__ __forceinline__ void exact_sum(const R (&g)[9], int first, R &hi, R &lo) {
    hi = g[first];
    lo = R(0);
#pragma unroll
    for (int i = first + 1; i < 9; ++i) {
        const R s = radd(hi, g[i]);
        const R z = rsub(s, hi);
        const R e = radd(rsub(hi, rsub(s, z)), rsub(g[i], z));
        hi = s;
        lo = radd(lo, e);
    }
}

template <typename R, bool FORCH>
__device__ __forceinline__ void collide(R (&g)[9], R alpha, R eps, R beta,
                                        const Phys<R> &ph, R &ux, R &uy) {
    // Mass closure: the collision conserves each node's mass exactly
    // in arithmetic, but rounding the nine stored populations does not, and
    // the slow pressure mode integrates that per-node error over thousands of
    // steps.  The exact sum of the streamed populations is kept, and the rest
    // population is stored as the exact remainder after the eight moving ones
    // (one rounding per node instead of nine).
    R in_hi, in_lo;
    exact_sum<R>(g, 0, in_hi, in_lo);
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
    g[0] = wd0 + (k1 * (g[0] - wd0) + w0 * (fb - om * su));
    collide_pair<R>(g[1], g[3], w1, wd1, ux, Fx, k1, om, su, a2, rho3, fb, f3, f9);
    collide_pair<R>(g[2], g[4], w1, wd1, uy, Fy, k1, om, su, a2, rho3, fb, f3, f9);
    collide_pair<R>(g[5], g[7], w2, wd2, ux + uy, Fx + Fy, k1, om, su, a2, rho3, fb, f3, f9);
    collide_pair<R>(g[6], g[8], w2, wd2, uy - ux, Fy - Fx, k1, om, su, a2, rho3, fb, f3, f9);
    R out_hi, out_lo;
    exact_sum<R>(g, 1, out_hi, out_lo);
    g[0] = radd(rsub(in_hi, out_hi), rsub(in_lo, out_lo));
}

// The same update for 16-bit storage, whose own rounding (2^-8 / 2^-11)
// dwarfs any FP32 regrouping error: every population is k1 g + c_i with
//   c_i = w_i [om (rho-1) + om rho (3 e.u + 9/(2 eps)(e.u)^2 - 3/(2 eps) u^2)
//              + rho A (3 e.F + 9/eps (e.u)(e.F) - 3/eps u.F)],
// folded per weight class into c = C + e.u (P e.u + Q e.F) +- (T e.u + U e.F)
// (even part C + ..., odd part T e.u + U e.F); w_diagonal = w_axis / 4 and
// w_0 = 4 w_axis, so the other classes are exact power-of-two multiples.
template <typename R, bool FORCH>
__device__ __forceinline__ void collide_small(R (&g)[9], R alpha, R eps, R beta,
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
    const R om = ph.omega, k1 = R(1) - om;
    const R w1 = R(1.0 / 9.0);
    const R cA = R(3) * w1 * ph.A;    // 3 w A
    const R cO = R(1.5) * w1 * om;    // (3/2) w om
    const R ier = rrcp(eps) * rho;    // rho / eps
    const R uu = ux * ux + uy * uy, uF = ux * Fx + uy * Fy;
    const R C1 = (w1 * om) * drho - ier * (cA * uF + cO * uu);
    const R P1 = (R(3) * cO) * ier, Q1 = (R(3) * cA) * ier;
    const R T1 = (R(2) * cO) * rho, U1 = cA * rho;
    g[0] = k1 * g[0] + R(4) * C1;
    auto pair = [&](R &gi, R &gj, R eu, R eF, R s) {
        const R E = s * (C1 + eu * (P1 * eu + Q1 * eF));
        const R O = s * (T1 * eu + U1 * eF);
        gi = k1 * gi + (E + O);
        gj = k1 * gj + (E - O);
    };
    pair(g[1], g[3], ux, Fx, R(1));
    pair(g[2], g[4], uy, Fy, R(1));
    pair(g[5], g[7], ux + uy, Fx + Fy, R(0.25));
    pair(g[6], g[8], uy - ux, Fy - Fx, R(0.25));
}

// Per-node coefficients of VEC consecutive nodes.
template <typename R, int VEC>
__device__ __forceinline__ void load_coef(const R *__restrict__ p, R (&c)[VEC]) {
    if constexpr (VEC == 1) c[0] = p[0];
    else ld16<R, VEC>(p, c);
}

// ---------------------------------------------------------------------------
// Pull-streaming gather of VEC consecutive nodes (x0..x0+VEC-1, row y) and
// of their coefficients (alpha, eps and, with Forchheimer, beta at node n0).
// Phase 1 issues every load of the thread (9 vectors + up to 6 edge scalars +
// 2-3 coefficient vectors) before phase 2 consumes any, so all of them are in
// flight together.
// ---------------------------------------------------------------------------
// INTERIOR: 0 < y < ny-1, so no population crosses a wall or the periodic
// y boundary and every shift mode is a compile-time constant.  x0 must be a
// valid node (callers clamp idle threads to x0 = 0 and discard their result).
template <typename T, int VEC, bool WALLS, bool INTERIOR, bool FORCH, bool CG = false>
__device__ __forceinline__ void gather(const T *__restrict__ src, const Geo &geo, int x0, int y,
                                       int lane, typename Store<T>::R inv_s,
                                       const typename Store<T>::R *__restrict__ alpha,
                                       const typename Store<T>::R *__restrict__ epsv,
                                       const typename Store<T>::R *__restrict__ betav, long long n0,
                                       typename Store<T>::R (&g)[VEC][9], typename Store<T>::R (&a)[VEC],
                                       typename Store<T>::R (&e)[VEC], typename Store<T>::R (&b)[VEC]) {
    using R = typename Store<T>::R;
    const int nx = geo.nx, ny = geo.ny;
    load_coef<R, VEC>(alpha + n0, a);
    load_coef<R, VEC>(epsv + n0, e);
    if (FORCH) load_coef<R, VEC>(betav + n0, b);
    else {
#pragma unroll
        for (int k = 0; k < VEC; ++k) b[k] = R(0);
    }
    if constexpr (VEC == 1) {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            int ys = y - cy(i);
            const T *p;
            if (!INTERIOR && (ys < 0 || ys >= ny)) {
                if (WALLS) {
                    // halfway bounce-back: the opposite population that left
                    // this node towards the wall returns reversed
                    p = src + (long long)opp(i) * geo.plane + (long long)y * nx + x0;
                    g[0][i] = Store<T>::ld(ld1<CG>(p), inv_s);
                    continue;
                }
                ys = ys < 0 ? ys + ny : ys - ny;
            }
            int xs = x0 - cx(i);
            xs = xs < 0 ? xs + nx : (xs >= nx ? xs - nx : xs);
            p = src + (long long)i * geo.plane + (long long)ys * nx + xs;
            g[0][i] = Store<T>::ld(ld1<CG>(p), inv_s);
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
            if (!INTERIOR && (ys < 0 || ys >= ny)) {
                if (WALLS) {
                    pl = opp(i);
                    ys = y;
                    mode[i] = 0;
                } else {
                    ys = ys < 0 ? ys + ny : ys - ny;
                }
            }
            const T *row = src + (long long)pl * geo.plane + (long long)ys * nx;
            ld16<T, VEC, CG>(row + x0, v[i]);
            edge[i] = T(0);
            if (mode[i] == 1 && first) edge[i] = ld1<CG>(row + xl);
            if (mode[i] == -1 && last) edge[i] = ld1<CG>(row + xr);
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

// One time step for the VEC consecutive nodes x0.. of row y of one lattice
// (src/dst/coefficients point at that lattice's plane 0).  Adds this thread's
// FP64 velocity sums to sx, sy and, for 16-bit storage, the largest stored
// magnitude to gm.
template <typename T, int VEC, bool WALLS, bool FORCH, bool REDUCE, bool CG = false>
__device__ __forceinline__ void step_body(const T *__restrict__ src, T *__restrict__ dst,
                                          const typename Store<T>::R *__restrict__ alpha,
                                          const typename Store<T>::R *__restrict__ epsv,
                                          const typename Store<T>::R *__restrict__ betav, const Geo &geo,
                                          const Phys<typename Store<T>::R> &ph, int x0, int y, double &sx,
                                          double &sy, float &gm) {
    using R = typename Store<T>::R;
    const bool active = x0 < geo.nx;
    x0 = active ? x0 : 0;  // idle threads read node 0 of the row and store nothing
    const int lane = threadIdx.x & 31;
    const long long n0 = (long long)y * geo.nx + x0;

    R g[VEC][9], a[VEC], e[VEC], b[VEC];
    if (y > 0 && y < geo.ny - 1)
        gather<T, VEC, WALLS, true, FORCH, CG>(src, geo, x0, y, lane, ph.inv_scale, alpha, epsv, betav, n0, g, a, e,
                                               b);
    else
        gather<T, VEC, WALLS, false, FORCH, CG>(src, geo, x0, y, lane, ph.inv_scale, alpha, epsv, betav, n0, g, a, e,
                                                b);

#pragma unroll
    for (int k = 0; k < VEC; ++k) {
        R ux, uy;
        if constexpr (Store<T>::kSmall) collide_small<R, FORCH>(g[k], a[k], e[k], b[k], ph, ux, uy);
        else collide<R, FORCH>(g[k], a[k], e[k], b[k], ph, ux, uy);
        if (REDUCE && active) {
            sx += double(ux);
            sy += double(uy);
        }
    }
    bool stored = false;
    if constexpr (Store<T>::kSmall && VEC == 4) {
        if (active && ph.sr) {
            // 16-bit storage, 4 nodes: two hardware stochastic-rounding
            // conversions per population.  The random words are successive
            // states of a full-period LCG seeded by one hash per thread; each
            // state is a bijective image of the seed, hence uniform like it,
            // which is all that unbiased rounding needs.
            uint32_t x = mix32(uint32_t(n0) ^ ph.step_key);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                float v[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) v[k] = Store<T>::kScaled ? g[k][i] * ph.scale : g[k][i];
                if (REDUCE)
                    gm = fmaxf(gm, fmaxf(fmaxf(fabsf(v[0]), fabsf(v[1])), fmaxf(fabsf(v[2]), fabsf(v[3]))));
                x = x * 0x2C1B3C6Du + 0x297A2D39u;
                const uint32_t r0 = x;
                x = x * 0x2C1B3C6Du + 0x297A2D39u;
                const uint32_t r1 = x;
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
}

// ---------------------------------------------------------------------------
// K2: fused pull-stream + collide (one time step).  REDUCE additionally
// writes this block's FP64 sums of u_x, u_y to partial[2*block] and, for
// 16-bit storage, the largest stored magnitude |g*S| to pmax[block].
// ---------------------------------------------------------------------------
// Programmatic dependent launch.  A step kernel launched with programmatic
// stream serialisation may be scheduled while the previous kernel of the
// stream drains.  It waits here, before touching any global memory (reads of
// the previous step's output and writes into the buffer that step read), for
// that kernel to complete and flush; then it lets the next launch start
// placing its blocks, so launch latency and the last partial wave overlap.
// Without the launch attribute both instructions return at once.
__device__ __forceinline__ void pdl_enter() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Host: launch `kern` on `st`, with programmatic stream serialisation when
// `pdl` (callers pass it for non-default streams).
template <typename... P, typename... A>
inline cudaError_t launch_kernel(void (*kern)(P...), dim3 grid, dim3 block, cudaStream_t st, bool pdl,
                                 A &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = pdl ? at : nullptr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<A>(args)...);
}

// Grid: x = blocks of a row (geo.bpr), row y = blockIdx.y + kMaxGridY *
// blockIdx.z (step_grid).  Blocks of 128 threads resident per SM, fixed by
// measurement on GB300: FP32 and FP16 fit 64 registers (8 blocks, 32 warps);
// BF16 spills at 64 and runs faster at 72 (7 blocks); FP64 is left free.
constexpr int kMaxGridY = 65535;
inline dim3 step_grid(const Geo &g) {
    const int gy = g.ny < kMaxGridY ? g.ny : kMaxGridY;
    return dim3(unsigned(g.bpr), unsigned(gy), unsigned((g.ny + kMaxGridY - 1) / kMaxGridY));
}
template <typename T>
constexpr int kMinBlocks = sizeof(T) == 8 ? 1 : (std::is_same<T, __nv_bfloat16>::value ? 7 : 8);

template <typename T, int VEC, bool WALLS, bool FORCH, bool REDUCE>
__global__ void __launch_bounds__(kThreads, kMinBlocks<T>)
k_step(const T *__restrict__ src, T *__restrict__ dst, const typename Store<T>::R *__restrict__ alpha,
       const typename Store<T>::R *__restrict__ epsv, const typename Store<T>::R *__restrict__ betav,
       Geo geo, Phys<typename Store<T>::R> ph, double *__restrict__ partial, float *__restrict__ pmax) {
    pdl_enter();
    if constexpr (Store<T>::kSmall) {
        if (ph.clock) ph.step_key = step_key_of(*ph.clock + ph.step_off, ph.seed);
    }
    const int y = int(blockIdx.y) + kMaxGridY * int(blockIdx.z);
    if (y >= geo.ny) return;  // padding of the last z slice (whole block)
    const int bx = int(blockIdx.x);
    const int x0 = (bx * kThreads + threadIdx.x) * VEC;
    const long long blk = (long long)y * geo.bpr + bx;  // reduction slot, row-major
    double sx = 0.0, sy = 0.0;
    float gm = 0.0f;
    step_body<T, VEC, WALLS, FORCH, REDUCE>(src, dst, alpha, epsv, betav, geo, ph, x0, y, sx, sy, gm);
    if (REDUCE) {
        block_sum2(sx, sy);
        if (threadIdx.x == 0) {
            partial[2 * blk] = sx;
            partial[2 * blk + 1] = sy;
        }
        if constexpr (Store<T>::kSmall) {
            gm = block_max(gm);
            if (threadIdx.x == 0) pmax[blk] = gm;
        }
    }
}

// Device step counter of 16-bit storage (see Phys::clock): set to a value
// or advanced by a captured chunk's length, one thread, ordered on the
// stream after the chunk's last step kernel.
__global__ void k_clock(unsigned *__restrict__ clock, unsigned value, int add) {
    pdl_enter();
    *clock = add ? *clock + value : value;
}

// Device-side run status (A8 result and convergence test).
struct DevStatus {
    double ux, uy;     // mean velocity of the last reduced step
    double prev_ux;    // the previous check's mean u_x
    int have_prev;     // prev_ux valid
    int converged;     // set by the last finalize
    int nonfinite;     // mean velocity not finite
    float gmax;        // 16-bit storage: largest stored |g*S| at that step
    int streak;        // consecutive checks that passed the relative-change test
    int pad;
};

// K3 finalize: fixed-order FP64 sum of the block partials, mean, test.
// Converged once `patience` consecutive checks pass |Ux - Ux_prev| <=
// tol |Ux| (patience 1: the first pass).
__global__ void __launch_bounds__(256)
k_finalize(const double *__restrict__ partial, int nparts, double inv_n, double tol,
           DevStatus *__restrict__ st, const float *__restrict__ pmax, int patience = 1) {
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
        const bool pass = fin && tol > 0.0 && st->have_prev && fabs(ux - st->prev_ux) <= tol * fabs(ux);
        st->streak = pass ? st->streak + 1 : 0;
        st->converged = st->streak >= patience ? 1 : 0;
        st->prev_ux = ux;
        st->have_prev = 1;
        st->gmax = m;
    }
}

// Velocity export: re-run the step's gather and velocity solve on the
// pre-step state (scalar loads; same arithmetic as k_step).
template <typename T, bool WALLS, bool FORCH>
__global__ void __launch_bounds__(kThreads)
k_velocity(const T *__restrict__ src, const typename Store<T>::R *__restrict__ alpha,
           const typename Store<T>::R *__restrict__ epsv, const typename Store<T>::R *__restrict__ betav,
           Geo geo, Phys<typename Store<T>::R> ph, double *__restrict__ ux_out,
           double *__restrict__ uy_out, double *__restrict__ rho_out = nullptr) {
    using R = typename Store<T>::R;
    const int y = blockIdx.x / geo.bpr;
    const int bx = blockIdx.x - y * geo.bpr;
    const int x0 = bx * kThreads + threadIdx.x;
    const bool active = x0 < geo.nx;
    if (!active) return;  // no shuffles on the scalar path
    const long long n = (long long)y * geo.nx + x0;
    R g[1][9], a[1], e[1], b[1];
    gather<T, 1, WALLS, false, FORCH>(src, geo, x0, y, threadIdx.x & 31, ph.inv_scale, alpha, epsv, betav, n, g, a, e,
                                      b);
    R drho, ux, uy;
    node_velocity<R, FORCH>(g[0], a[0], e[0], b[0], ph, drho, ux, uy);
    ux_out[n] = double(ux);
    uy_out[n] = double(uy);
    if (rho_out) rho_out[n] = 1.0 + double(drho);
}

}  // namespace
