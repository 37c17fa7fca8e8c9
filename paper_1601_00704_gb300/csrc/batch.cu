// Batched lattices and the DGM/GMS apparent-permeability field builder.
//
// A batch holds many media of uneven size (e.g. a sweep over pressure,
// Langmuir parameters and organic content) and advances all media that have
// not converged yet with ONE kernel launch per time step.  Block b of a
// launch handles the row segment tiles[b] = (medium, y, bx); the per-thread
// step is the same step_body() as the single-lattice solver, so every medium
// evolves bit for bit as it would alone.  Chunks of steps are captured into
// CUDA graphs and replayed.  Each medium's mean velocity is reduced from its
// tiles' FP64 partials by one block per medium, in a fixed order; converged
// media leave the tile table at the next chunk boundary.  An autotuner times
// the candidate schedules (threads per block x tile order) on the batch.
//
// Storage formats: FP32 and BF16 (BF16 needs no per-medium scale); the
// Forchheimer-free model of Eq. 28 only.

#include "glbm.h"
#include "guard.h"
#include "trace.h"
#include "glbm_kernels.cuh"
#include "setup_kernels.cuh"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <numeric>
#include <vector>

extern __attribute__((visibility("hidden"))) thread_local char g_create_err[512];
__attribute__((visibility("hidden"))) bool glbm_injected_failure();

namespace {

struct BTile {
    int med, y, bx, pad;
};

struct BMed {
    long long off_f;  // element offset of the medium's plane 0 in the f buffers
    long long off_c;  // element offset in the coefficient planes
    long long plane;  // plane stride, elements
    int nx, ny, bpr;  // geometry; bpr = blocks per row for the current schedule
    int tile0, ntiles;
    int pad;
};

// Step key of the stochastic-rounding hash, kept on the device so that a
// replayed graph advances it: every block reads it, and the last block of the
// launch (atomic ticket, no waiting) increments it and resets the ticket.
struct StepClock {
    unsigned int step;
    unsigned int ticket;
    unsigned int seed;
    unsigned int pad;
};

// Resident blocks as for k_step, scaled from its 128-thread blocks.
template <typename T, int THREADS, bool WALLS, bool REDUCE>
__global__ void __launch_bounds__(THREADS, kMinBlocks<T> * 128 / THREADS)
k_batch_step(const T *__restrict__ src_all, T *__restrict__ dst_all,
             const typename Store<T>::R *__restrict__ alpha, const typename Store<T>::R *__restrict__ epsv,
             const BTile *__restrict__ tiles, const BMed *__restrict__ meds, Phys<typename Store<T>::R> ph,
             StepClock *__restrict__ clock, double *__restrict__ partial, float *__restrict__ pmax) {
    constexpr int VEC = kVecOf<T>;
    pdl_enter();
    const BTile t = tiles[blockIdx.x];
    const BMed m = meds[t.med];
    Geo geo;
    geo.nx = m.nx;
    geo.ny = m.ny;
    geo.plane = m.plane;
    geo.bpr = m.bpr;
    if (Store<T>::kSmall) ph.step_key = mix32(clock->step * 0x9E3779B9u + clock->seed);
    const int x0 = (t.bx * THREADS + threadIdx.x) * VEC;
    double sx = 0.0, sy = 0.0;
    float gm = 0.0f;
    step_body<T, VEC, WALLS, false, REDUCE>(src_all + m.off_f, dst_all + m.off_f, alpha + m.off_c,
                                            epsv + m.off_c, nullptr, geo, ph, x0, t.y, sx, sy, gm);
    if (REDUCE) {
        block_sum2(sx, sy);
        if (threadIdx.x == 0) {
            partial[2ll * blockIdx.x] = sx;
            partial[2ll * blockIdx.x + 1] = sy;
        }
    }
    if (Store<T>::kSmall) {
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (atomicAdd(&clock->ticket, 1u) == gridDim.x - 1) {
                clock->ticket = 0u;
                clock->step += 1u;
                __threadfence();
            }
        }
    }
}

// Grid-wide barrier of the persistent kernel (all blocks co-resident: the
// launch is cooperative).  Generation counting: the last block to arrive
// resets the count and bumps the generation; the others wait for the bump,
// at most kBarrierCycles (~1 s), after which they record a timeout in *err
// and give up.  Returns false once this block has given up.
struct GridBar {
    unsigned count;
    unsigned gen;
};
constexpr long long kBarrierCycles = 2ll << 30;

__device__ __forceinline__ bool grid_barrier(GridBar *bar, int *err) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned *gen = &bar->gen;
        const unsigned g = *gen;
        __threadfence();
        ok = 1;
        if (atomicAdd(&bar->count, 1u) == gridDim.x - 1) {
            bar->count = 0u;
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g) {
                if (clock64() - t0 > kBarrierCycles) {
                    atomicExch(err, 1);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Persistent variant of k_batch_step: one cooperative launch runs `nsteps`
// time steps of every tile, the blocks striding over the tile table and
// meeting at a grid barrier between steps.  Step s reads buffer
// (parity0 + s) & 1 and writes the other; the last step writes the per-tile
// partials.  Loads of the distributions go through L2 only (they were
// written by other blocks of this launch).  The stochastic-rounding key of
// step s is that of step clock->step + s, and the last block to finish
// advances clock->step by nsteps.
template <typename T, int THREADS, bool WALLS>
__global__ void __launch_bounds__(THREADS, kMinBlocks<T> * 128 / THREADS)
k_batch_persist(T *__restrict__ buf0, T *__restrict__ buf1, int parity0, int nsteps,
                const typename Store<T>::R *__restrict__ alpha, const typename Store<T>::R *__restrict__ epsv,
                const BTile *__restrict__ tiles, int ntiles, const BMed *__restrict__ meds,
                Phys<typename Store<T>::R> ph, StepClock *__restrict__ clock, double *__restrict__ partial,
                GridBar *__restrict__ bar, int *__restrict__ err) {
    constexpr int VEC = kVecOf<T>;
    const unsigned step0 = clock->step, seed = clock->seed;
    for (int s = 0; s < nsteps; ++s) {
        const bool last = s == nsteps - 1;
        const T *src = ((parity0 + s) & 1) ? buf1 : buf0;
        T *dst = ((parity0 + s) & 1) ? buf0 : buf1;
        if (Store<T>::kSmall) ph.step_key = step_key_of(step0 + unsigned(s), seed);
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
            const BTile tl = tiles[t];
            const BMed m = meds[tl.med];
            Geo geo;
            geo.nx = m.nx;
            geo.ny = m.ny;
            geo.plane = m.plane;
            geo.bpr = m.bpr;
            const int x0 = (tl.bx * THREADS + threadIdx.x) * VEC;
            double sx = 0.0, sy = 0.0;
            float gm = 0.0f;
            if (last) {
                step_body<T, VEC, WALLS, false, true, true>(src + m.off_f, dst + m.off_f, alpha + m.off_c,
                                                            epsv + m.off_c, nullptr, geo, ph, x0, tl.y, sx, sy, gm);
                block_sum2(sx, sy);
                if (threadIdx.x == 0) {
                    partial[2ll * t] = sx;
                    partial[2ll * t + 1] = sy;
                }
                __syncthreads();  // block_sum2's shared slots are reused by the next tile
            } else {
                step_body<T, VEC, WALLS, false, false, true>(src + m.off_f, dst + m.off_f, alpha + m.off_c,
                                                             epsv + m.off_c, nullptr, geo, ph, x0, tl.y, sx, sy,
                                                             gm);
            }
        }
        if (!grid_barrier(bar, err)) return;
    }
    if (threadIdx.x == 0 && blockIdx.x == 0) clock->step = step0 + unsigned(nsteps);
}

// Per-medium finalize: block j reduces active medium act[j] over its tiles.
__global__ void __launch_bounds__(256)
k_batch_finalize(const double *__restrict__ partial, const BMed *__restrict__ meds, const int *__restrict__ act,
                 double tol, DevStatus *__restrict__ st, int patience) {
    __shared__ double sh[2][256];
    const int m = act[blockIdx.x];
    const BMed md = meds[m];
    double a = 0.0, b = 0.0;
    for (int j = threadIdx.x; j < md.ntiles; j += 256) {
        a += partial[2ll * (md.tile0 + j)];
        b += partial[2ll * (md.tile0 + j) + 1];
    }
    sh[0][threadIdx.x] = a;
    sh[1][threadIdx.x] = b;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            sh[0][threadIdx.x] += sh[0][threadIdx.x + s];
            sh[1][threadIdx.x] += sh[1][threadIdx.x + s];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double inv_n = 1.0 / double((long long)md.nx * md.ny);
        const double ux = sh[0][0] * inv_n, uy = sh[1][0] * inv_n;
        DevStatus &s = st[m];
        s.ux = ux;
        s.uy = uy;
        const bool fin = isfinite(ux) && isfinite(uy);
        s.nonfinite = fin ? 0 : 1;
        const bool pass = fin && tol > 0.0 && s.have_prev && fabs(ux - s.prev_ux) <= tol * fabs(ux);
        s.streak = pass ? s.streak + 1 : 0;
        s.converged = s.streak >= patience ? 1 : 0;
        s.prev_ux = ux;
        s.have_prev = 1;
    }
}

// DGM/GMS apparent permeability per node (Eqs. 3, 4, 18, 19 with the ideal
// gas rho_g = P M / (R T)), simplified algebraically:
//   K_app = K0 + eta D_K / P [+ (eta R T / P)(1 - eps) q_sat b D_s / (1 + b P)]
// with K0 = eps d^2 / (32 tau), D_K = (4/3)(eps d / (4 tau)) sqrt(8 R T / (pi M)),
// d = 2 r; returned in lattice units K_app / dx^2.
__global__ void k_kapp(const double *__restrict__ r, const unsigned char *__restrict__ organic,
                       const double *__restrict__ eps, long long n, double P, double T, double M, double eta,
                       double tort, double qsat, double b, double Ds, double inv_dx2, double *__restrict__ K) {
    const double R_GAS = 8.314462618;
    const double vbar = sqrt(8.0 * R_GAS * T / (3.14159265358979323846 * M));
    const double surf = eta * R_GAS * T / P * qsat * b * Ds / (1.0 + b * P);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double d = 2.0 * r[i], e = eps[i];
        const double k0 = e * d * d / (32.0 * tort);
        const double dk = (4.0 / 3.0) * (e * d / (4.0 * tort)) * vbar;
        double k = k0 + eta * dk / P;
        if (organic[i]) k += (1.0 - e) * surf;
        K[i] = k * inv_dx2;
    }
}

__global__ void k_kapp_check(const double *__restrict__ r, const double *__restrict__ eps, long long n,
                             int *__restrict__ first_bad) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        if (!(r[i] > 0.0) || !isfinite(r[i]) || !(eps[i] > 0.0 && eps[i] < 1.0)) atomicMin(first_bad, int(i));
}

}  // namespace

struct glbm_batch {
    int count = 0;
    double tau = 1.0;
    glbm_storage storage = GLBM_F32;
    unsigned flags = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int dev = 0;
    size_t elem = 4;
    std::vector<BMed> med;
    std::vector<char> has_medium;
    std::vector<char> active;
    std::vector<int> parity_of;          // buffer of a stopped medium's state
    std::vector<long long> steps_of;     // steps of a stopped medium
    long long off_f_total = 0, off_c_total = 0, max_tiles = 0;
    void *buf[2] = {nullptr, nullptr};
    float *coef[2] = {nullptr, nullptr};  // alpha, eps
    BMed *dmed = nullptr;
    BTile *dtiles = nullptr;
    int *dact = nullptr;
    int ntiles = 0, nact = 0;
    double *partial = nullptr;
    DevStatus *dstat = nullptr, *hstat = nullptr;
    StepClock *dclock = nullptr;
    int *dflag = nullptr;
    double *stage = nullptr;
    glbm_guard::Table guards;  // every device buffer of the batch, with its guard zones
    long long stage_n = 0;
    int parity = 0;
    long long tstep = 0;
    bool reduced = false;
    double gx = 0.0, gy = 0.0;
    int threads = 128, order = 0;
    bool persistent = false;  // one cooperative launch per chunk (k_batch_persist)
    int patience = 1;         // consecutive passing checks for a medium to converge
    GridBar *dbar = nullptr;
    int *derr = nullptr;      // persistent kernel: grid-barrier timeout flag
    int nsm = 0;
    struct Graph {
        int parity, chunk, test;
        cudaGraphExec_t exec;
    };
    std::vector<Graph> graphs;
    long long launches = 0;
    char err[512] = "";
};

namespace {

glbm_status bfail(glbm_batch *h, glbm_status s, const char *fmt, ...) {
    char *dst = h ? h->err : g_create_err;
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(dst, 512, fmt, ap);
    va_end(ap);
    return s;
}

#define BCU(h, call)                                                                          \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return bfail((h), e_ == cudaErrorMemoryAllocation ? GLBM_ENOMEM : GLBM_ECUDA,     \
                         "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

int vec_of(const glbm_batch *h) { return h->elem == 2 ? 4 : 4; }

void drop_graphs(glbm_batch *h) {
    for (auto &g : h->graphs) cudaGraphExecDestroy(g.exec);
    h->graphs.clear();
}

// Build the tile table of the active media for the current schedule.
glbm_status build_table(glbm_batch *h) {
    const int vec = vec_of(h);
    std::vector<int> act;
    for (int m = 0; m < h->count; ++m)
        if (h->active[m]) act.push_back(m);
    if (h->order == 1)
        std::stable_sort(act.begin(), act.end(), [&](int a, int b) {
            return (long long)h->med[a].nx * h->med[a].ny > (long long)h->med[b].nx * h->med[b].ny;
        });
    std::vector<BTile> tiles;
    for (int m = 0; m < h->count; ++m) {
        BMed &md = h->med[m];
        md.bpr = ((md.nx + vec - 1) / vec + h->threads - 1) / h->threads;
        md.tile0 = 0;
        md.ntiles = 0;
    }
    if (h->order == 2) {
        // rows round-robin over the media: row r of every medium, then r+1
        std::vector<int> dummy;
        int maxny = 0;
        for (int m : act) maxny = std::max(maxny, h->med[m].ny);
        // tiles of one medium must stay contiguous for the finalize, so
        // interleave at the granularity of whole media sorted by row count
        // alternating large and small
        std::vector<int> s = act;
        std::stable_sort(s.begin(), s.end(), [&](int a, int b) { return h->med[a].ny > h->med[b].ny; });
        act.clear();
        for (size_t i = 0, j = s.size(); i < j;) {
            act.push_back(s[i++]);
            if (i < j) act.push_back(s[--j]);
        }
        (void)maxny;
        (void)dummy;
    }
    for (int m : act) {
        BMed &md = h->med[m];
        md.tile0 = int(tiles.size());
        for (int y = 0; y < md.ny; ++y)
            for (int bx = 0; bx < md.bpr; ++bx) tiles.push_back({m, y, bx, 0});
        md.ntiles = int(tiles.size()) - md.tile0;
    }
    h->ntiles = int(tiles.size());
    h->nact = int(act.size());
    if (h->ntiles > h->max_tiles) return bfail(h, GLBM_EINVAL, "batch: tile table overflow");
    if (h->ntiles) BCU(h, cudaMemcpyAsync(h->dtiles, tiles.data(), sizeof(BTile) * tiles.size(), cudaMemcpyHostToDevice, h->stream));
    if (h->nact) BCU(h, cudaMemcpyAsync(h->dact, act.data(), sizeof(int) * act.size(), cudaMemcpyHostToDevice, h->stream));
    BCU(h, cudaMemcpyAsync(h->dmed, h->med.data(), sizeof(BMed) * h->count, cudaMemcpyHostToDevice, h->stream));
    BCU(h, cudaStreamSynchronize(h->stream));  // host vectors go out of scope
    drop_graphs(h);
    return GLBM_OK;
}

template <typename T, int THREADS, bool WALLS>
cudaError_t launch_bstep_t(glbm_batch *h, bool reduce) {
    using R = typename Store<T>::R;
    Phys<R> ph;
    ph.omega = R(1.0 / h->tau);
    ph.A = R(1.0 - 0.5 / h->tau);
    ph.gx = R(h->gx);
    ph.gy = R(h->gy);
    ph.scale = R(1);
    ph.inv_scale = R(1);
    ph.step_key = 0;
    ph.sr = 1;
    const T *src = static_cast<const T *>(h->buf[h->parity]);
    T *dst = static_cast<T *>(h->buf[h->parity ^ 1]);
    if (glbm_injected_failure()) return cudaErrorLaunchFailure;  // test hook: nothing is launched
    cudaError_t e;
    if (reduce)
        e = launch_kernel(k_batch_step<T, THREADS, WALLS, true>, dim3(h->ntiles), dim3(THREADS), h->stream,
                          h->stream != nullptr, src, dst, h->coef[0], h->coef[1], h->dtiles, h->dmed, ph, h->dclock,
                          h->partial, nullptr);
    else
        e = launch_kernel(k_batch_step<T, THREADS, WALLS, false>, dim3(h->ntiles), dim3(THREADS), h->stream,
                          h->stream != nullptr, src, dst, h->coef[0], h->coef[1], h->dtiles, h->dmed, ph, h->dclock,
                          h->partial, nullptr);
    if (e != cudaSuccess) return e;
    h->launches++;
    h->parity ^= 1;
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_bstep_s(glbm_batch *h, bool reduce) {
    const bool walls = !(h->flags & GLBM_PERIODIC_Y);
    switch (h->threads) {
        case 64: return walls ? launch_bstep_t<T, 64, true>(h, reduce) : launch_bstep_t<T, 64, false>(h, reduce);
        case 256: return walls ? launch_bstep_t<T, 256, true>(h, reduce) : launch_bstep_t<T, 256, false>(h, reduce);
        default: return walls ? launch_bstep_t<T, 128, true>(h, reduce) : launch_bstep_t<T, 128, false>(h, reduce);
    }
}

cudaError_t launch_bstep(glbm_batch *h, bool reduce) {
    if (h->storage == GLBM_BF16DEV) return launch_bstep_s<__nv_bfloat16>(h, reduce);
    return launch_bstep_s<float>(h, reduce);
}

template <typename T, int THREADS, bool WALLS>
cudaError_t launch_persist_t(glbm_batch *h, int chunk) {
    using R = typename Store<T>::R;
    Phys<R> ph;
    ph.omega = R(1.0 / h->tau);
    ph.A = R(1.0 - 0.5 / h->tau);
    ph.gx = R(h->gx);
    ph.gy = R(h->gy);
    ph.scale = R(1);
    ph.inv_scale = R(1);
    ph.step_key = 0;
    ph.sr = 1;
    auto kern = k_batch_persist<T, THREADS, WALLS>;
    int per_sm = 0;
    if (cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, THREADS, 0)) return e;
    if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
    const int grid = int(std::min<long long>(h->ntiles, (long long)per_sm * h->nsm));
    if (glbm_injected_failure()) return cudaErrorLaunchFailure;  // test hook: nothing is launched
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(grid));
    cfg.blockDim = dim3(THREADS);
    cfg.stream = h->stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaError_t e = cudaLaunchKernelEx(&cfg, kern, static_cast<T *>(h->buf[0]), static_cast<T *>(h->buf[1]),
                                       h->parity, chunk, static_cast<const R *>(h->coef[0]),
                                       static_cast<const R *>(h->coef[1]), static_cast<const BTile *>(h->dtiles),
                                       h->ntiles, static_cast<const BMed *>(h->dmed), ph, h->dclock, h->partial,
                                       h->dbar, h->derr);
    if (e != cudaSuccess) return e;
    h->launches++;
    if (chunk % 2) h->parity ^= 1;
    return cudaSuccess;
}

template <typename T>
cudaError_t launch_persist_s(glbm_batch *h, int chunk) {
    const bool walls = !(h->flags & GLBM_PERIODIC_Y);
    switch (h->threads) {
        case 64: return walls ? launch_persist_t<T, 64, true>(h, chunk) : launch_persist_t<T, 64, false>(h, chunk);
        case 256: return walls ? launch_persist_t<T, 256, true>(h, chunk) : launch_persist_t<T, 256, false>(h, chunk);
        default: return walls ? launch_persist_t<T, 128, true>(h, chunk) : launch_persist_t<T, 128, false>(h, chunk);
    }
}

// Enqueue `chunk` steps (+ the per-medium reduction at the last one); the
// first failed launch stops it and is returned.
cudaError_t enqueue_chunk(glbm_batch *h, int chunk, double tol) {
    if (h->persistent) {
        const cudaError_t e = h->storage == GLBM_BF16DEV ? launch_persist_s<__nv_bfloat16>(h, chunk)
                                                         : launch_persist_s<float>(h, chunk);
        if (e != cudaSuccess) return e;
    } else {
        for (int s = 0; s < chunk; ++s)
            if (cudaError_t e = launch_bstep(h, s == chunk - 1)) return e;
    }
    if (glbm_injected_failure()) return cudaErrorLaunchFailure;
    k_batch_finalize<<<h->nact, 256, 0, h->stream>>>(h->partial, h->dmed, h->dact, tol, h->dstat, h->patience);
    if (cudaError_t e = cudaGetLastError()) return e;
    h->launches++;
    return cudaSuccess;
}

// Run one chunk, from a captured graph when the same (parity, length, test)
// chunk has been seen since the table last changed.  The persistent kernel
// is one launch per chunk already and runs uncaptured.
glbm_status run_chunk(glbm_batch *h, int chunk, double tol) {
    const int test = tol > 0.0;
    if (h->persistent) {
        const int p0 = h->parity;
        const long long l0 = h->launches;
        if (cudaError_t e = enqueue_chunk(h, chunk, tol)) {
            (void)cudaGetLastError();
            h->parity = p0;
            h->launches = l0;
            return bfail(h, GLBM_ECUDA, "batch: persistent step launch failed: %s%s", cudaGetErrorString(e),
                         e == cudaErrorLaunchFailure ? " (injected by the test hook)" : "");
        }
        return GLBM_OK;
    }
    for (auto &g : h->graphs) {
        if (g.parity == h->parity && g.chunk == chunk && g.test == test) {
            BCU(h, cudaGraphLaunch(g.exec, h->stream));
            h->launches += chunk + 1;
            if (chunk % 2) h->parity ^= 1;
            return GLBM_OK;
        }
    }
    // a failure while capturing ends the capture, discards it and leaves the
    // parity and launch count as they were (nothing has run)
    const int p0 = h->parity;
    const long long l0 = h->launches;
    cudaGraph_t graph = nullptr;
    BCU(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
    const cudaError_t el = enqueue_chunk(h, chunk, tol);
    cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
    cudaGraphExec_t exec = nullptr;
    glbm_status st = GLBM_OK;
    if (el != cudaSuccess)
        st = bfail(h, GLBM_ECUDA, "batch: step launch failed: %s%s", cudaGetErrorString(el),
                   el == cudaErrorLaunchFailure ? " (injected by the test hook)" : "");
    else if (e != cudaSuccess)
        st = bfail(h, GLBM_ECUDA, "batch: graph capture failed: %s", cudaGetErrorString(e));
    if (!st) {
        e = cudaGraphInstantiate(&exec, graph, 0);
        if (e != cudaSuccess) st = bfail(h, GLBM_ECUDA, "batch: graph instantiate failed: %s", cudaGetErrorString(e));
    }
    if (graph) cudaGraphDestroy(graph);
    if (st) {
        (void)cudaGetLastError();
        h->parity = p0;
        h->launches = l0;
        return st;
    }
    h->graphs.push_back({p0, chunk, test, exec});
    BCU(h, cudaGraphLaunch(exec, h->stream));
    return GLBM_OK;
}

glbm_status bcheck(glbm_batch *h) {
    if (!h) return GLBM_EINVAL;
    cudaError_t e = cudaSetDevice(h->dev);
    if (e != cudaSuccess) return bfail(h, GLBM_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
    return GLBM_OK;
}

void brelease(glbm_batch *h) {
    drop_graphs(h);
    for (auto &p : h->buf) glbm_guard::release(h->guards, p), p = nullptr;
    for (auto &p : h->coef) glbm_guard::release(h->guards, p), p = nullptr;
    void *ptrs[] = {h->dmed, h->dtiles, h->dact, h->partial, h->dstat, h->dclock, h->dflag, h->stage, h->dbar, h->derr};
    for (void *p : ptrs) glbm_guard::release(h->guards, p);
    h->dmed = nullptr;
    h->dtiles = nullptr;
    h->dact = nullptr;
    h->partial = nullptr;
    h->dstat = nullptr;
    h->dclock = nullptr;
    h->dflag = nullptr;
    h->stage = nullptr;
    h->dbar = nullptr;
    h->derr = nullptr;
    if (h->hstat) cudaFreeHost(h->hstat), h->hstat = nullptr;
    if (h->own_stream && h->stream) cudaStreamDestroy(h->stream), h->stream = nullptr;
}

glbm_status zero_state(glbm_batch *h) {
    BCU(h, cudaMemsetAsync(h->buf[0], 0, h->off_f_total * h->elem, h->stream));
    BCU(h, cudaMemsetAsync(h->buf[1], 0, h->off_f_total * h->elem, h->stream));
    BCU(h, cudaMemsetAsync(h->dstat, 0, sizeof(DevStatus) * h->count, h->stream));
    StepClock c{0u, 0u, 0x2545F491u, 0u};
    BCU(h, cudaMemcpyAsync(h->dclock, &c, sizeof(c), cudaMemcpyHostToDevice, h->stream));
    BCU(h, cudaStreamSynchronize(h->stream));
    for (int m = 0; m < h->count; ++m) {
        h->active[m] = 1;
        h->parity_of[m] = 0;
        h->steps_of[m] = 0;
    }
    h->parity = 0;
    h->tstep = 0;
    h->reduced = false;
    return build_table(h);
}

}  // namespace

extern "C" {

glbm_status glbm_batch_create(int count, const int *nx, const int *ny, double tau, glbm_storage storage,
                              unsigned flags, void *stream, glbm_batch_t *out) {
    if (!out) return bfail(nullptr, GLBM_EINVAL, "glbm_batch_create: out is NULL");
    *out = nullptr;
    if (count < 1 || !nx || !ny) return bfail(nullptr, GLBM_EINVAL, "glbm_batch_create: need count >= 1 and sizes");
    if (!(tau > 0.5) || !std::isfinite(tau)) return bfail(nullptr, GLBM_EINVAL, "glbm_batch_create: tau must be > 1/2");
    if (storage != GLBM_F32 && storage != GLBM_BF16DEV)
        return bfail(nullptr, GLBM_EINVAL, "glbm_batch_create: batches store GLBM_F32 or GLBM_BF16DEV");
    if (flags & ~GLBM_PERIODIC_Y) return bfail(nullptr, GLBM_EINVAL, "glbm_batch_create: unknown flags 0x%x", flags);
    for (int m = 0; m < count; ++m)
        if (nx[m] < 4 || ny[m] < 2 || nx[m] % 4 || (long long)nx[m] * ny[m] >= (1ll << 31))
            return bfail(nullptr, GLBM_EINVAL,
                         "glbm_batch_create: medium %d is %d x %d (need nx a multiple of 4, ny >= 2)", m, nx[m],
                         ny[m]);
    glbm_batch *h = new (std::nothrow) glbm_batch;
    if (!h) return bfail(nullptr, GLBM_ENOMEM, "glbm_batch_create: out of host memory");
    h->count = count;
    h->tau = tau;
    h->storage = storage;
    h->flags = flags;
    h->elem = storage == GLBM_F32 ? 4 : 2;
    h->med.resize(count);
    h->has_medium.assign(count, 0);
    h->active.assign(count, 1);
    h->parity_of.assign(count, 0);
    h->steps_of.assign(count, 0);
    long long offf = 0, offc = 0, maxt = 0, maxn = 0;
    for (int m = 0; m < count; ++m) {
        BMed &md = h->med[m];
        md.nx = nx[m];
        md.ny = ny[m];
        const long long N = (long long)nx[m] * ny[m];
        md.plane = (N + 63) / 64 * 64;
        md.off_f = offf;
        md.off_c = offc;
        offf += 9 * md.plane;
        offc += md.plane;
        maxt += (long long)((nx[m] / 4 + 63) / 64) * ny[m];  // 64 threads per block: most tiles
        maxn = std::max(maxn, N);
    }
    h->off_f_total = offf;
    h->off_c_total = offc;
    h->max_tiles = maxt;
    h->stage_n = maxn;
    cudaError_t e = cudaGetDevice(&h->dev);
    if (e == cudaSuccess && !stream) {
        e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
        h->own_stream = true;
    } else {
        h->stream = static_cast<cudaStream_t>(stream);
    }
    auto galloc = [h](auto **p, size_t bytes) {
        return glbm_guard::alloc(h->guards, reinterpret_cast<void **>(p), bytes, h->stream);
    };
    if (e == cudaSuccess) e = galloc(&h->buf[0], offf * h->elem);
    if (e == cudaSuccess) e = galloc(&h->buf[1], offf * h->elem);
    if (e == cudaSuccess) e = galloc(&h->coef[0], offc * sizeof(float));
    if (e == cudaSuccess) e = galloc(&h->coef[1], offc * sizeof(float));
    if (e == cudaSuccess) e = galloc(&h->dmed, sizeof(BMed) * count);
    if (e == cudaSuccess) e = galloc(&h->dtiles, sizeof(BTile) * maxt);
    if (e == cudaSuccess) e = galloc(&h->dact, sizeof(int) * count);
    if (e == cudaSuccess) e = galloc(&h->partial, sizeof(double) * 2 * maxt);
    if (e == cudaSuccess) e = galloc(&h->dstat, sizeof(DevStatus) * count);
    if (e == cudaSuccess) e = galloc(&h->dclock, sizeof(StepClock));
    if (e == cudaSuccess) e = galloc(&h->dflag, sizeof(int));
    if (e == cudaSuccess) e = galloc(&h->dbar, sizeof(GridBar));
    if (e == cudaSuccess) e = galloc(&h->derr, sizeof(int));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->dbar, 0, sizeof(GridBar), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->derr, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->dev);
    if (e == cudaSuccess) e = cudaMallocHost(&h->hstat, sizeof(DevStatus) * count);
    glbm_status s = GLBM_OK;
    if (e != cudaSuccess)
        s = bfail(nullptr, e == cudaErrorMemoryAllocation ? GLBM_ENOMEM : GLBM_ECUDA, "glbm_batch_create: %s",
                  cudaGetErrorString(e));
    if (!s) s = zero_state(h);
    if (s) {
        if (s != GLBM_OK && h->err[0]) snprintf(g_create_err, 512, "%s", h->err);
        brelease(h);
        delete h;
        return s;
    }
    *out = h;
    return GLBM_OK;
}

glbm_status glbm_batch_set_medium(glbm_batch_t h, int index, const double *eps, const double *K, int device_ptrs) {
    glbm_trace::Range trace_range("glbm_batch_set_medium");
    if (glbm_status s = bcheck(h)) return s;
    if (index < 0 || index >= h->count) return bfail(h, GLBM_EINVAL, "batch_set_medium: index %d out of range", index);
    if (!eps || !K) return bfail(h, GLBM_EINVAL, "batch_set_medium: eps and K are required");
    BMed &md = h->med[index];
    const long long N = (long long)md.nx * md.ny;
    const double *de = eps, *dk = K;
    if (!device_ptrs) {
        if (!h->stage)
            BCU(h, glbm_guard::alloc(h->guards, reinterpret_cast<void **>(&h->stage), sizeof(double) * 2 * h->stage_n,
                                     h->stream));
        BCU(h, cudaMemcpyAsync(h->stage, eps, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream));
        BCU(h, cudaMemcpyAsync(h->stage + h->stage_n, K, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream));
        de = h->stage;
        dk = h->stage + h->stage_n;
    }
    BCU(h, cudaMemsetAsync(h->dflag, 0x7f, sizeof(int), h->stream));
    const int g = int(std::min<long long>((N + 255) / 256, 152 * 64));
    k_validate<<<g, 256, 0, h->stream>>>(de, dk, N, h->dflag);
    int bad = 0;
    BCU(h, cudaGetLastError());
    BCU(h, cudaMemcpyAsync(&bad, h->dflag, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
    BCU(h, cudaStreamSynchronize(h->stream));
    if (bad < N) return bfail(h, GLBM_EINVAL, "batch_set_medium: medium %d node %d has eps outside (0, 1] or K not > 0", index, bad);
    const double nu = (h->tau - 0.5) / 3.0;
    // Forchheimer-free batches: no beta plane
    k_pack<float><<<g, 256, 0, h->stream>>>(de, dk, N, nu, 0.0, h->coef[0] + md.off_c, h->coef[1] + md.off_c,
                                            nullptr);
    h->launches += 2;
    BCU(h, cudaGetLastError());
    // rest state for this medium in both buffers
    BCU(h, cudaMemsetAsync(static_cast<char *>(h->buf[0]) + md.off_f * h->elem, 0, 9 * md.plane * h->elem, h->stream));
    BCU(h, cudaMemsetAsync(static_cast<char *>(h->buf[1]) + md.off_f * h->elem, 0, 9 * md.plane * h->elem, h->stream));
    BCU(h, cudaStreamSynchronize(h->stream));
    h->has_medium[index] = 1;
    return GLBM_OK;
}

glbm_status glbm_batch_set_force(glbm_batch_t h, double gx, double gy) {
    if (glbm_status s = bcheck(h)) return s;
    if (!std::isfinite(gx) || !std::isfinite(gy)) return bfail(h, GLBM_EINVAL, "batch_set_force: G must be finite");
    h->gx = gx;
    h->gy = gy;
    drop_graphs(h);  // the force is baked into captured launches
    for (int m = 0; m < h->count; ++m)
        BCU(h, cudaMemsetAsync(&h->dstat[m].have_prev, 0, sizeof(int), h->stream));
    return GLBM_OK;
}

glbm_status glbm_batch_reset(glbm_batch_t h) {
    if (glbm_status s = bcheck(h)) return s;
    return zero_state(h);
}

glbm_status glbm_batch_set_schedule(glbm_batch_t h, int threads, int order) {
    if (glbm_status s = bcheck(h)) return s;
    if ((threads != 64 && threads != 128 && threads != 256) || order < 0 || order > 2)
        return bfail(h, GLBM_EINVAL, "batch_set_schedule: threads in {64,128,256}, order in {0,1,2}");
    h->threads = threads;
    h->order = order;
    return build_table(h);
}

glbm_status glbm_batch_set_persistent(glbm_batch_t h, int on) {
    if (glbm_status s = bcheck(h)) return s;
    h->persistent = on != 0;
    drop_graphs(h);
    return GLBM_OK;
}

glbm_status glbm_batch_set_convergence(glbm_batch_t h, int patience) {
    if (glbm_status s = bcheck(h)) return s;
    if (patience < 1 || patience > 1000000)
        return bfail(h, GLBM_EINVAL, "batch_set_convergence: patience must be in [1, 1e6] (got %d)", patience);
    h->patience = patience;
    drop_graphs(h);  // the finalize is captured with it
    return GLBM_OK;
}

glbm_status glbm_batch_get_persistent(glbm_batch_t h, int *on) {
    if (!h || !on) return GLBM_EINVAL;
    *on = h->persistent ? 1 : 0;
    return GLBM_OK;
}

glbm_status glbm_batch_debug_guards(glbm_batch_t h, int poke, long long *damaged) {
    if (glbm_status s = bcheck(h)) return s;
    if (!damaged) return bfail(h, GLBM_EINVAL, "batch_debug_guards: damaged is required");
    BCU(h, glbm_guard::count_damage(h->guards, h->stream, poke, damaged));
    return GLBM_OK;
}

glbm_status glbm_batch_step(glbm_batch_t h, long long n, double tol, int check_every, long long *steps_done,
                            int *active_left) {
    glbm_trace::Range trace_range("glbm_batch_step");
    if (steps_done) *steps_done = 0;
    if (glbm_status s = bcheck(h)) return s;
    for (int m = 0; m < h->count; ++m)
        if (!h->has_medium[m]) return bfail(h, GLBM_ESTATE, "batch_step: medium %d has no medium set", m);
    if (n < 0 || check_every < 1 || !std::isfinite(tol)) return bfail(h, GLBM_EINVAL, "batch_step: bad arguments");
    long long done = 0;
    const bool test = tol > 0.0;
    while (done < n && h->nact > 0) {
        const int chunk = int(std::min<long long>(check_every, n - done));
        if (glbm_status s = run_chunk(h, chunk, test ? tol : 0.0)) return s;
        done += chunk;
        h->tstep += chunk;
        h->reduced = true;
        if (test) {
            BCU(h, cudaMemcpyAsync(h->hstat, h->dstat, sizeof(DevStatus) * h->count, cudaMemcpyDeviceToHost, h->stream));
            BCU(h, cudaStreamSynchronize(h->stream));
            bool changed = false;
            for (int m = 0; m < h->count; ++m) {
                if (!h->active[m]) continue;
                if (h->hstat[m].nonfinite)
                    return bfail(h, GLBM_ENAN, "batch_step: medium %d has a non-finite mean velocity", m);
                if (h->hstat[m].converged) {
                    h->active[m] = 0;
                    h->parity_of[m] = h->parity;
                    h->steps_of[m] = h->tstep;
                    changed = true;
                }
            }
            if (changed)
                if (glbm_status s = build_table(h)) return s;
        }
    }
    for (int m = 0; m < h->count; ++m)
        if (h->active[m]) {
            h->parity_of[m] = h->parity;
            h->steps_of[m] = h->tstep;
        }
    if (h->persistent) {
        int berr = 0;
        BCU(h, cudaMemcpyAsync(&berr, h->derr, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        BCU(h, cudaStreamSynchronize(h->stream));
        if (berr) {
            BCU(h, cudaMemsetAsync(h->derr, 0, sizeof(int), h->stream));
            BCU(h, cudaMemsetAsync(h->dbar, 0, sizeof(GridBar), h->stream));
            return bfail(h, GLBM_ECUDA, "batch_step: a grid barrier of the persistent kernel timed out");
        }
    }
    if (steps_done) *steps_done = done;
    if (active_left) *active_left = h->nact;
    BCU(h, cudaGetLastError());
    return GLBM_OK;
}

glbm_status glbm_batch_autotune(glbm_batch_t h, int trial_steps, int *threads, int *order) {
    if (glbm_status s = bcheck(h)) return s;
    if (trial_steps < 1) return bfail(h, GLBM_EINVAL, "batch_autotune: trial_steps must be >= 1");
    for (int m = 0; m < h->count; ++m)
        if (!h->has_medium[m]) return bfail(h, GLBM_ESTATE, "batch_autotune: medium %d has no medium set", m);
    cudaEvent_t e0, e1;
    BCU(h, cudaEventCreate(&e0));
    BCU(h, cudaEventCreate(&e1));
    float best = 1e30f;
    int bt = 128, bo = 0;
    bool bp = false;
    const int cand_t[3] = {64, 128, 256};
    for (int pers = 0; pers < 2; ++pers)
    for (int o = 0; o < 3; ++o)
        for (int t : cand_t) {
            h->threads = t;
            h->order = o;
            h->persistent = pers != 0;
            if (glbm_status s = build_table(h)) return s;
            if (glbm_status s = run_chunk(h, trial_steps, 0.0)) return s;  // capture + warm-up
            BCU(h, cudaEventRecord(e0, h->stream));
            if (glbm_status s = run_chunk(h, trial_steps, 0.0)) return s;
            if (glbm_status s = run_chunk(h, trial_steps, 0.0)) return s;
            BCU(h, cudaEventRecord(e1, h->stream));
            BCU(h, cudaEventSynchronize(e1));
            float ms = 0.0f;
            BCU(h, cudaEventElapsedTime(&ms, e0, e1));
            if (ms < best) {
                best = ms;
                bt = t;
                bo = o;
                bp = pers != 0;
            }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h->threads = bt;
    h->order = bo;
    h->persistent = bp;
    if (threads) *threads = bt;
    if (order) *order = bo;
    return zero_state(h);  // trials advanced the state: start again from rest
}

glbm_status glbm_batch_results(glbm_batch_t h, double *kxx, double *mean_u, long long *steps, int *converged) {
    if (glbm_status s = bcheck(h)) return s;
    if (!h->reduced) return bfail(h, GLBM_ESTATE, "batch_results: no step has completed since the last reset");
    BCU(h, cudaMemcpyAsync(h->hstat, h->dstat, sizeof(DevStatus) * h->count, cudaMemcpyDeviceToHost, h->stream));
    BCU(h, cudaStreamSynchronize(h->stream));
    const double nu = (h->tau - 0.5) / 3.0;
    for (int m = 0; m < h->count; ++m) {
        if (kxx) kxx[m] = h->gx != 0.0 ? nu * h->hstat[m].ux / h->gx : NAN;
        if (mean_u) {
            mean_u[2 * m] = h->hstat[m].ux;
            mean_u[2 * m + 1] = h->hstat[m].uy;
        }
        if (steps) steps[m] = h->steps_of[m];
        if (converged) converged[m] = h->active[m] ? 0 : 1;
    }
    return GLBM_OK;
}

glbm_status glbm_batch_get_distributions(glbm_batch_t h, int index, double *f, int device_ptrs) {
    if (glbm_status s = bcheck(h)) return s;
    if (index < 0 || index >= h->count || !f) return bfail(h, GLBM_EINVAL, "batch_get_distributions: bad arguments");
    const BMed &md = h->med[index];
    const long long N = (long long)md.nx * md.ny;
    const int par = h->active[index] ? h->parity : h->parity_of[index];
    double *df = f, *tmp = nullptr;
    if (!device_ptrs) {
        BCU(h, cudaMalloc(&tmp, sizeof(double) * 9 * N));
        df = tmp;
    }
    const int g = int(std::min<long long>((N + 255) / 256, 152 * 64));
    if (h->storage == GLBM_BF16DEV)
        k_export_f<__nv_bfloat16><<<g, 256, 0, h->stream>>>(
            static_cast<const __nv_bfloat16 *>(h->buf[par]) + md.off_f, md.plane, N, 1.0f, df);
    else
        k_export_f<float><<<g, 256, 0, h->stream>>>(static_cast<const float *>(h->buf[par]) + md.off_f, md.plane, N,
                                                    1.0f, df);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && !device_ptrs)
        e = cudaMemcpyAsync(f, df, sizeof(double) * 9 * N, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (tmp) cudaFree(tmp);
    if (e != cudaSuccess) return bfail(h, GLBM_ECUDA, "batch_get_distributions: %s", cudaGetErrorString(e));
    return GLBM_OK;
}

glbm_status glbm_batch_get_fields(glbm_batch_t h, int index, double *rho, double *ux, double *uy, int device_ptrs) {
    if (glbm_status s = bcheck(h)) return s;
    if (index < 0 || index >= h->count || !ux || !uy) return bfail(h, GLBM_EINVAL, "batch_get_fields: bad arguments");
    if (!h->reduced) return bfail(h, GLBM_ESTATE, "batch_get_fields: no step has completed since the last reset");
    const BMed &md = h->med[index];
    const long long N = (long long)md.nx * md.ny;
    // the last step of this medium read the other buffer
    const int cur = h->active[index] ? h->parity : h->parity_of[index];
    double *tmp = nullptr, *dr = rho, *dx = ux, *dy = uy;
    if (!device_ptrs) {
        BCU(h, cudaMalloc(&tmp, sizeof(double) * 3 * N));
        dr = rho ? tmp : nullptr;
        dx = tmp + N;
        dy = tmp + 2 * N;
    }
    Geo geo;
    geo.nx = md.nx;
    geo.ny = md.ny;
    geo.plane = md.plane;
    geo.bpr = (md.nx + kThreads - 1) / kThreads;
    Phys<float> ph;
    ph.omega = float(1.0 / h->tau);
    ph.A = float(1.0 - 0.5 / h->tau);
    ph.gx = float(h->gx);
    ph.gy = float(h->gy);
    ph.scale = 1.0f;
    ph.inv_scale = 1.0f;
    ph.step_key = 0;
    ph.sr = 1;
    const unsigned grid = unsigned(geo.bpr) * unsigned(geo.ny);
    const bool walls = !(h->flags & GLBM_PERIODIC_Y);
    const float *a = h->coef[0] + md.off_c, *e = h->coef[1] + md.off_c;
    if (h->storage == GLBM_BF16DEV) {
        const __nv_bfloat16 *src = static_cast<const __nv_bfloat16 *>(h->buf[cur ^ 1]) + md.off_f;
        if (walls) k_velocity<__nv_bfloat16, true, false><<<grid, kThreads, 0, h->stream>>>(src, a, e, nullptr, geo, ph, dx, dy, dr);
        else k_velocity<__nv_bfloat16, false, false><<<grid, kThreads, 0, h->stream>>>(src, a, e, nullptr, geo, ph, dx, dy, dr);
    } else {
        const float *src = static_cast<const float *>(h->buf[cur ^ 1]) + md.off_f;
        if (walls) k_velocity<float, true, false><<<grid, kThreads, 0, h->stream>>>(src, a, e, nullptr, geo, ph, dx, dy, dr);
        else k_velocity<float, false, false><<<grid, kThreads, 0, h->stream>>>(src, a, e, nullptr, geo, ph, dx, dy, dr);
    }
    cudaError_t err = cudaGetLastError();
    if (err == cudaSuccess && !device_ptrs) {
        if (rho) err = cudaMemcpyAsync(rho, dr, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream);
        if (err == cudaSuccess) err = cudaMemcpyAsync(ux, dx, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream);
        if (err == cudaSuccess) err = cudaMemcpyAsync(uy, dy, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream);
    }
    if (err == cudaSuccess) err = cudaStreamSynchronize(h->stream);
    if (tmp) cudaFree(tmp);
    if (err != cudaSuccess) return bfail(h, GLBM_ECUDA, "batch_get_fields: %s", cudaGetErrorString(err));
    return GLBM_OK;
}

glbm_status glbm_batch_info(glbm_batch_t h, int *threads, int *order, long long *launches, long long *nodes) {
    if (!h) return GLBM_EINVAL;
    if (threads) *threads = h->threads;
    if (order) *order = h->order;
    if (launches) *launches = h->launches;
    if (nodes) {
        long long n = 0;
        for (const BMed &md : h->med) n += (long long)md.nx * md.ny;
        *nodes = n;
    }
    return GLBM_OK;
}

void glbm_batch_destroy(glbm_batch_t h) {
    if (!h) return;
    cudaSetDevice(h->dev);
    if (h->stream) cudaStreamSynchronize(h->stream);
    brelease(h);
    delete h;
}

const char *glbm_batch_last_error(glbm_batch_t h) { return h ? h->err : g_create_err; }

glbm_status glbm_kapp_field(const double *r, const unsigned char *organic, const double *eps, long long n, double P,
                            double T, double M, double eta, double tort, double qsat, double b, double Ds, double dx,
                            double *K, int device_ptrs, void *stream) {
    if (!r || !organic || !eps || !K || n < 1)
        return bfail(nullptr, GLBM_EINVAL, "kapp_field: r, organic, eps, K and n >= 1 are required");
    const double sc[] = {P, T, M, eta, tort, dx};
    for (double v : sc)
        if (!(v > 0.0) || !std::isfinite(v))
            return bfail(nullptr, GLBM_EINVAL, "kapp_field: P, T, M, eta, tort and dx must be finite and > 0");
    if (!(qsat >= 0.0) || !(b >= 0.0) || !(Ds >= 0.0) || !std::isfinite(qsat + b + Ds))
        return bfail(nullptr, GLBM_EINVAL, "kapp_field: qsat, b and Ds must be finite and >= 0");
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const double *dr = r, *de = eps;
    const unsigned char *dorg = organic;
    double *dK = K;
    char *tmp = nullptr;
    int *flag = nullptr;
    auto cleanup = [&]() {
        if (tmp) cudaFree(tmp);
        if (flag) cudaFree(flag);
    };
    cudaError_t e = cudaMalloc(&flag, sizeof(int));
    if (e == cudaSuccess && !device_ptrs) {
        e = cudaMalloc(&tmp, size_t(n) * (3 * sizeof(double) + 1));
        if (e == cudaSuccess) {
            double *p = reinterpret_cast<double *>(tmp);
            dr = p;
            de = p + n;
            dK = p + 2 * n;
            dorg = reinterpret_cast<unsigned char *>(p + 3 * n);
            e = cudaMemcpyAsync(const_cast<double *>(dr), r, sizeof(double) * n, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(const_cast<double *>(de), eps, sizeof(double) * n, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(const_cast<unsigned char *>(dorg), organic, n, cudaMemcpyHostToDevice, st);
        }
    }
    int bad = 0x7f7f7f7f;
    const int g = int(std::min<long long>((n + 255) / 256, 152 * 64));
    if (e == cudaSuccess) e = cudaMemsetAsync(flag, 0x7f, sizeof(int), st);
    if (e == cudaSuccess) {
        k_kapp_check<<<g, 256, 0, st>>>(dr, de, n, flag);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&bad, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cleanup();
        return bfail(nullptr, GLBM_ECUDA, "kapp_field: %s", cudaGetErrorString(e));
    }
    if (bad < n) {
        cleanup();
        return bfail(nullptr, GLBM_EINVAL, "kapp_field: node %d has a radius <= 0 or eps outside (0, 1)", bad);
    }
    k_kapp<<<g, 256, 0, st>>>(dr, dorg, de, n, P, T, M, eta, tort, qsat, b, Ds, 1.0 / (dx * dx), dK);
    e = cudaGetLastError();
    if (e == cudaSuccess && !device_ptrs) e = cudaMemcpyAsync(K, dK, sizeof(double) * n, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cleanup();
    if (e != cudaSuccess) return bfail(nullptr, GLBM_ECUDA, "kapp_field: %s", cudaGetErrorString(e));
    return GLBM_OK;
}

double glbm_qsat_from_langmuir_volume(double qsat_b, double rho_b, double eps, double toc, double rho_ch4,
                                      double M_ch4) {
    const double den = (1.0 - eps) * toc * M_ch4;
    if (!(den > 0.0)) return NAN;
    return qsat_b * rho_b * rho_ch4 / den;
}

}  // extern "C"
