// Host side and C ABI of the single-lattice GB300 (sm_103a) solver of the
// generalized lattice Boltzmann model (GLBM) time loop of Wang, Chen, Kang &
// Rahman, arXiv:1601.00704, Sec. 2.3.  The kernels and their design notes
// are in glbm_kernels.cuh; the C ABI is declared in include/glbm.h.

#include "glbm.h"
#include "guard.h"
#include "trace.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <atomic>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "glbm_kernels.cuh"
#include "setup_kernels.cuh"

// ---------------------------------------------------------------------------
// Host side.
// ---------------------------------------------------------------------------
// Message buffer for failures without a handle (glbm_last_error(NULL)),
// shared with the other translation units of the library.
__attribute__((visibility("hidden"))) thread_local char g_create_err[512] = "";

// Host-side fault injection for tests of the error paths
// (glbm_debug_fail_launch): the launch that comes `g_fail_countdown`
// launches from now is refused with GLBM_ECUDA, as a failed launch would be,
// without calling CUDA.  Negative = off.  Shared with batch.cu.
namespace {
std::atomic<long long> g_fail_countdown{-1};
}
__attribute__((visibility("hidden"))) bool glbm_injected_failure() {
    long long c = g_fail_countdown.load();
    while (c >= 0) {
        if (g_fail_countdown.compare_exchange_weak(c, c - 1)) return c == 0;
    }
    return false;
}

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
    glbm_guard::Table guards; // every device buffer above, with its guard zones
    bool has_medium = false, forch = false, reduced = false;
    double feps_mode = 0.0, gx = 0.0, gy = 0.0;
    double scale = 1.0;       // FP16 storage scale S (stored = g*S)
    bool sr = true;           // 16-bit storage: stochastic rounding
    bool at_rest = false;     // state is f_eq(1, 0) (zero deviations)
    uint32_t seed = 0x2545F491u;
    int patience = 1;         // consecutive passing checks for convergence
    long long tstep = 0;      // time steps launched since the last reset
    long long steps = 0, launches = 0;
    // 16-bit storage: device copy of tstep, read by the step kernels of
    // replayed graphs for their stochastic-rounding key
    unsigned *dclock = nullptr;
    // chunks replayed from captured CUDA graphs (any storage, on a
    // non-legacy stream): key = (buffer parity at start, steps, reduce at
    // end, test, tol, FP16 scale)
    struct Graph {
        int parity;
        long long chunk;
        int reduce, test, patience;
        double tol, scale;
        cudaGraphExec_t exec;
    };
    Graph graphs[8];
    int ngraphs = 0;
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
    p.step_key = step_key_of(uint32_t(h->tstep), h->seed);
    p.sr = h->sr ? 1 : 0;
    p.seed = h->seed;
    return p;
}

bool injected_failure() { return glbm_injected_failure(); }

int grid_1d(long long N) {
    long long b = (N + 255) / 256;
    return int(b > 152 * 64 ? 152 * 64 : (b < 1 ? 1 : b));
}

// One step kernel.  `clock_off` >= 0 (16-bit storage inside a graph
// capture): the kernel takes its rounding key from the device step counter
// plus clock_off, so that replays of the graph draw fresh bits.
template <typename T, int VEC, bool WALLS, bool FORCH>
glbm_status launch_step_t(glbm *h, bool reduce, long long clock_off) {
    using R = typename Store<T>::R;
    const Geo geo = make_geo(h, VEC);
    Phys<R> ph = make_phys<R>(h);
    if (Store<T>::kSmall && clock_off >= 0) {
        ph.clock = h->dclock;
        ph.step_off = uint32_t(clock_off);
    }
    if (injected_failure()) return fail(h, GLBM_ECUDA, "step launch: injected failure (test hook)");
    const T *src = static_cast<const T *>(h->buf[h->cur]);
    T *dst = static_cast<T *>(h->buf[h->cur ^ 1]);
    const R *a = static_cast<const R *>(h->coef[0]);
    const R *e = static_cast<const R *>(h->coef[1]);
    const R *b = static_cast<const R *>(h->coef[2]);
    const dim3 grid = step_grid(geo);
    const bool pdl = h->stream != nullptr;
    cudaError_t err;
    if (reduce)
        err = launch_kernel(k_step<T, VEC, WALLS, FORCH, true>, grid, dim3(kThreads), h->stream, pdl, src, dst, a, e,
                            b, geo, ph, h->partial, h->pmax);
    else
        err = launch_kernel(k_step<T, VEC, WALLS, FORCH, false>, grid, dim3(kThreads), h->stream, pdl, src, dst, a,
                            e, b, geo, ph, h->partial, h->pmax);
    if (err != cudaSuccess) return fail(h, GLBM_ECUDA, "step launch: %s", cudaGetErrorString(err));
    h->launches++;
    h->tstep++;
    h->cur ^= 1;
    return GLBM_OK;
}

template <typename T>
glbm_status launch_step(glbm *h, bool reduce, long long co) {
    constexpr int V = kVecOf<T>;
    const bool walls = !(h->flags & GLBM_PERIODIC_Y);
    const bool vec = vec_width(h) > 1;
    if (vec) {
        if (walls) return h->forch ? launch_step_t<T, V, true, true>(h, reduce, co) : launch_step_t<T, V, true, false>(h, reduce, co);
        return h->forch ? launch_step_t<T, V, false, true>(h, reduce, co) : launch_step_t<T, V, false, false>(h, reduce, co);
    }
    if (walls) return h->forch ? launch_step_t<T, 1, true, true>(h, reduce, co) : launch_step_t<T, 1, true, false>(h, reduce, co);
    return h->forch ? launch_step_t<T, 1, false, true>(h, reduce, co) : launch_step_t<T, 1, false, false>(h, reduce, co);
}

glbm_status do_step(glbm *h, bool reduce, long long clock_off = -1) {
    switch (h->storage) {
        case GLBM_F32: return launch_step<float>(h, reduce, clock_off);
        case GLBM_F64: return launch_step<double>(h, reduce, clock_off);
        case GLBM_F16DEV: return launch_step<__half>(h, reduce, clock_off);
        case GLBM_BF16DEV: return launch_step<__nv_bfloat16>(h, reduce, clock_off);
    }
    return GLBM_EINVAL;
}

int nparts(const glbm *h) {
    const Geo g = make_geo(h, vec_width(h));
    return g.bpr * g.ny;
}

glbm_status finalize(glbm *h, double tol) {
    if (injected_failure()) return fail(h, GLBM_ECUDA, "finalize launch: injected failure (test hook)");
    k_finalize<<<1, 256, 0, h->stream>>>(h->partial, nparts(h), 1.0 / double(h->N), tol, h->dstat,
                                         h->elem == 2 ? h->pmax : nullptr, h->patience);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(h, GLBM_ECUDA, "finalize launch: %s", cudaGetErrorString(e));
    h->launches++;
    h->reduced = true;
    return GLBM_OK;
}

// 16-bit storage: set (add = 0) or advance (add = 1) the device step counter.
glbm_status clock_op(glbm *h, long long value, bool add) {
    if (h->elem != 2) return GLBM_OK;
    k_clock<<<1, 1, 0, h->stream>>>(h->dclock, unsigned(value), add ? 1 : 0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(h, GLBM_ECUDA, "clock launch: %s", cudaGetErrorString(e));
    h->launches++;
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

void drop_graphs(glbm *h) {
    for (int i = 0; i < h->ngraphs; ++i) cudaGraphExecDestroy(h->graphs[i].exec);
    h->ngraphs = 0;
}

bool graph_eligible(const glbm *h) { return h->stream != nullptr; }

// Enqueue one chunk (chunk steps, the last one reducing when `reduce`, then
// the finalize), directly or by replaying a captured graph of it.  A failure
// while capturing ends the capture, discards it and leaves the handle's
// buffer parity, step and launch counts as they were; nothing has run.
glbm_status run_chunk(glbm *h, long long chunk, bool reduce, double tol) {
    const int test = tol > 0.0;
    const bool small = h->elem == 2;
    if (graph_eligible(h) && chunk >= 4) {
        for (int i = 0; i < h->ngraphs; ++i) {
            const glbm::Graph &g = h->graphs[i];
            if (g.parity == h->cur && g.chunk == chunk && g.reduce == int(reduce) && g.test == test &&
                g.tol == tol && g.scale == h->scale && g.patience == h->patience) {
                CU(h, cudaGraphLaunch(g.exec, h->stream));
                h->launches += chunk + (reduce ? 1 : 0) + (small ? 1 : 0);
                h->tstep += chunk;
                if (chunk % 2) h->cur ^= 1;
                if (reduce) h->reduced = true;
                return GLBM_OK;
            }
        }
        if (h->ngraphs == 8) drop_graphs(h);
        const int p0 = h->cur;
        const long long t0 = h->tstep, l0 = h->launches;
        const bool r0 = h->reduced;
        cudaGraph_t graph = nullptr;
        CU(h, cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
        glbm_status st = GLBM_OK;
        for (long long s = 0; s < chunk && !st; ++s) st = do_step(h, reduce && s == chunk - 1, small ? s : -1);
        if (!st && reduce) st = finalize(h, tol);
        if (!st) st = clock_op(h, chunk, true);
        cudaError_t e = cudaStreamEndCapture(h->stream, &graph);
        cudaGraphExec_t exec = nullptr;
        if (!st && e != cudaSuccess)
            st = fail(h, GLBM_ECUDA, "step: graph capture failed: %s", cudaGetErrorString(e));
        if (!st) {
            e = cudaGraphInstantiate(&exec, graph, 0);
            if (e != cudaSuccess)
                st = fail(h, GLBM_ECUDA, "step: graph instantiate failed: %s", cudaGetErrorString(e));
        }
        if (graph) cudaGraphDestroy(graph);
        if (st) {
            (void)cudaGetLastError();  // drop the capture's error state
            h->cur = p0;
            h->tstep = t0;
            h->launches = l0;
            h->reduced = r0;
            return st;
        }
        h->graphs[h->ngraphs++] = {p0, chunk, int(reduce), test, h->patience, tol, h->scale, exec};
        CU(h, cudaGraphLaunch(exec, h->stream));
        return GLBM_OK;
    }
    for (long long s = 0; s < chunk; ++s)
        if (glbm_status st = do_step(h, reduce && s == chunk - 1)) return st;
    if (reduce)
        if (glbm_status st = finalize(h, tol)) return st;
    // keep the device step counter in step for later graph replays
    if (graph_eligible(h)) return clock_op(h, h->tstep, false);
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
    if (any && !device_ptrs && !h->stage)
        CU(h, glbm_guard::alloc(h->guards, reinterpret_cast<void **>(&h->stage), sizeof(double) * 3 * size_t(h->N),
                                h->stream));
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
    drop_graphs(h);
    glbm_guard::Table &g = h->guards;
    for (auto &p : h->buf) glbm_guard::release(g, p), p = nullptr;
    for (auto &p : h->coef) glbm_guard::release(g, p), p = nullptr;
    glbm_guard::release(g, h->partial), h->partial = nullptr;
    glbm_guard::release(g, h->pmax), h->pmax = nullptr;
    glbm_guard::release(g, h->dstat), h->dstat = nullptr;
    glbm_guard::release(g, h->dflag), h->dflag = nullptr;
    glbm_guard::release(g, h->dclock), h->dclock = nullptr;
    glbm_guard::release(g, h->stage), h->stage = nullptr;
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
    auto galloc = [h](auto **p, size_t bytes) {
        return glbm_guard::alloc(h->guards, reinterpret_cast<void **>(p), bytes, h->stream);
    };
    if (e == cudaSuccess) e = galloc(&h->buf[0], fbytes);
    if (e == cudaSuccess) e = galloc(&h->buf[1], fbytes);
    for (int c = 0; c < 3 && e == cudaSuccess; ++c) e = galloc(&h->coef[c], cbytes);
    if (e == cudaSuccess) e = galloc(&h->partial, sizeof(double) * 2 * size_t(h->nparts_max));
    if (e == cudaSuccess) e = galloc(&h->pmax, sizeof(float) * size_t(h->nparts_max));
    if (e == cudaSuccess) e = galloc(&h->dstat, sizeof(DevStatus));
    if (e == cudaSuccess) e = galloc(&h->dflag, sizeof(int));
    if (e == cudaSuccess) e = galloc(&h->dclock, sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMallocHost(&h->hstat, sizeof(DevStatus));
    if (e == cudaSuccess) e = cudaMemsetAsync(h->dstat, 0, sizeof(DevStatus), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->dclock, 0, sizeof(unsigned), h->stream);
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
    glbm_trace::Range trace_range("glbm_set_medium");
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
    CU(h, cudaMemsetAsync(h->dclock, 0, sizeof(unsigned), h->stream));
    if (h->forch != (F_eps != 0.0)) drop_graphs(h);  // another kernel instantiation
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
    drop_graphs(h);  // G is baked into captured launches
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
    glbm_trace::Range trace_range("glbm_init_equilibrium");
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
    CU(h, cudaMemsetAsync(h->dclock, 0, sizeof(unsigned), h->stream));
    h->steps = 0;
    h->tstep = 0;
    h->at_rest = !(rho || ux);
    return GLBM_OK;
}

glbm_status glbm_step(glbm_t h, long long n, double tol, int check_every, long long *steps_done,
                      int *converged) {
    glbm_trace::Range trace_range("glbm_step");
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
        if (glbm_status st = run_chunk(h, chunk, reduce_here, test ? tol : 0.0)) return st;
        done += chunk;
        h->steps += chunk;
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

glbm_status glbm_set_convergence(glbm_t h, int patience) {
    if (glbm_status s = check(h)) return s;
    if (patience < 1 || patience > 1000000)
        return fail(h, GLBM_EINVAL, "set_convergence: patience must be in [1, 1e6] (got %d)", patience);
    h->patience = patience;
    return GLBM_OK;
}

glbm_status glbm_mean_velocity(glbm_t h, double out[2]) {
    glbm_trace::Range trace_range("glbm_mean_velocity");
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
    glbm_trace::Range trace_range("glbm_permeability");
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

// ---------------------------------------------------------------------------
// Checkpoint / resume.  File layout (native byte order): a fixed header
// (CkptHeader), then the current distributions as 9 planes of N stored
// elements (no padding), then the coefficient planes alpha, eps and, with
// Forchheimer, beta (N elements each).  An FNV-1a 64 checksum of everything
// after the header guards against truncated or altered files.
// ---------------------------------------------------------------------------
}  // extern "C"

namespace {

struct CkptHeader {
    char magic[8];  // "GLBMCKP1"
    unsigned version;
    int nx, ny, storage;
    unsigned flags;
    int forch, at_rest, reduced, sr;
    double tau, feps_mode, gx, gy, scale;
    unsigned seed;
    int patience;
    long long tstep, steps;
    DevStatus status;
    unsigned long long checksum;
};

constexpr unsigned kCkptVersion = 1;

void fnv1a(unsigned long long &h, const void *p, size_t n) {
    const unsigned char *b = static_cast<const unsigned char *>(p);
    for (size_t i = 0; i < n; ++i) {
        h ^= b[i];
        h *= 1099511628211ull;
    }
}

struct File {
    FILE *f = nullptr;
    ~File() {
        if (f) fclose(f);
    }
};

}  // namespace

extern "C" {

glbm_status glbm_debug_guards(glbm_t h, int poke, long long *damaged) {
    if (glbm_status s = check(h)) return s;
    if (!damaged) return fail(h, GLBM_EINVAL, "debug_guards: damaged is required");
    CU(h, glbm_guard::count_damage(h->guards, h->stream, poke, damaged));
    return GLBM_OK;
}

glbm_status glbm_save(glbm_t h, const char *path) {
    glbm_trace::Range trace_range("glbm_save");
    if (glbm_status s = check(h)) return s;
    if (!path) return fail(h, GLBM_EINVAL, "save: path is NULL");
    if (!h->has_medium) return fail(h, GLBM_ESTATE, "save: no medium set");
    const size_t N = size_t(h->N);
    const size_t fb = 9 * N * h->elem, cb = N * h->celem;
    const int ncoef = h->forch ? 3 : 2;
    std::vector<unsigned char> buf(fb + ncoef * cb);
    CkptHeader hd;
    memset(&hd, 0, sizeof(hd));
    memcpy(hd.magic, "GLBMCKP1", 8);
    hd.version = kCkptVersion;
    hd.nx = h->nx;
    hd.ny = h->ny;
    hd.storage = int(h->storage);
    hd.flags = h->flags;
    hd.forch = h->forch;
    hd.at_rest = h->at_rest;
    hd.reduced = h->reduced;
    hd.sr = h->sr;
    hd.tau = h->tau;
    hd.feps_mode = h->feps_mode;
    hd.gx = h->gx;
    hd.gy = h->gy;
    hd.scale = h->scale;
    hd.seed = h->seed;
    hd.patience = h->patience;
    hd.tstep = h->tstep;
    hd.steps = h->steps;
    CU(h, cudaMemcpy2DAsync(buf.data(), N * h->elem, h->buf[h->cur], size_t(h->plane) * h->elem, N * h->elem, 9,
                            cudaMemcpyDeviceToHost, h->stream));
    for (int c = 0; c < ncoef; ++c)
        CU(h, cudaMemcpyAsync(buf.data() + fb + c * cb, h->coef[c], cb, cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaMemcpyAsync(&hd.status, h->dstat, sizeof(DevStatus), cudaMemcpyDeviceToHost, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));
    hd.checksum = 14695981039346656037ull;
    fnv1a(hd.checksum, buf.data(), buf.size());
    File f;
    f.f = fopen(path, "wb");
    if (!f.f) return fail(h, GLBM_EINVAL, "save: cannot open %s for writing", path);
    if (fwrite(&hd, sizeof(hd), 1, f.f) != 1 || fwrite(buf.data(), 1, buf.size(), f.f) != buf.size() ||
        fflush(f.f) != 0)
        return fail(h, GLBM_EINVAL, "save: writing %s failed", path);
    return GLBM_OK;
}

glbm_status glbm_load(glbm_t h, const char *path) {
    glbm_trace::Range trace_range("glbm_load");
    if (glbm_status s = check(h)) return s;
    if (!path) return fail(h, GLBM_EINVAL, "load: path is NULL");
    File f;
    f.f = fopen(path, "rb");
    if (!f.f) return fail(h, GLBM_EINVAL, "load: cannot open %s", path);
    CkptHeader hd;
    if (fread(&hd, sizeof(hd), 1, f.f) != 1 || memcmp(hd.magic, "GLBMCKP1", 8) != 0 ||
        hd.version != kCkptVersion)
        return fail(h, GLBM_EINVAL, "load: %s is not a checkpoint of this library version", path);
    if (hd.nx != h->nx || hd.ny != h->ny || hd.storage != int(h->storage) || hd.flags != h->flags ||
        hd.tau != h->tau)
        return fail(h, GLBM_EINVAL,
                    "load: checkpoint is %d x %d, storage %d, flags 0x%x, tau %g; handle is %d x %d, storage %d, "
                    "flags 0x%x, tau %g",
                    hd.nx, hd.ny, hd.storage, hd.flags, hd.tau, h->nx, h->ny, int(h->storage), h->flags, h->tau);
    const size_t N = size_t(h->N);
    const size_t fb = 9 * N * h->elem, cb = N * h->celem;
    const int ncoef = hd.forch ? 3 : 2;
    std::vector<unsigned char> buf(fb + ncoef * cb);
    if (fread(buf.data(), 1, buf.size(), f.f) != buf.size())
        return fail(h, GLBM_EINVAL, "load: %s is truncated", path);
    unsigned long long sum = 14695981039346656037ull;
    fnv1a(sum, buf.data(), buf.size());
    if (sum != hd.checksum) return fail(h, GLBM_EINVAL, "load: checksum mismatch in %s", path);
    // the other buffer's padding and contents are never read before written
    CU(h, cudaMemcpy2DAsync(h->buf[0], size_t(h->plane) * h->elem, buf.data(), N * h->elem, N * h->elem, 9,
                            cudaMemcpyHostToDevice, h->stream));
    for (int c = 0; c < ncoef; ++c)
        CU(h, cudaMemcpyAsync(h->coef[c], buf.data() + fb + c * cb, cb, cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaMemcpyAsync(h->dstat, &hd.status, sizeof(DevStatus), cudaMemcpyHostToDevice, h->stream));
    const unsigned clock = unsigned(hd.tstep);
    CU(h, cudaMemcpyAsync(h->dclock, &clock, sizeof(unsigned), cudaMemcpyHostToDevice, h->stream));
    CU(h, cudaStreamSynchronize(h->stream));  // host staging goes out of scope
    if (bool(hd.forch) != h->forch) drop_graphs(h);
    if (hd.gx != h->gx || hd.gy != h->gy || hd.scale != h->scale) drop_graphs(h);
    h->cur = 0;
    h->forch = hd.forch;
    h->feps_mode = hd.feps_mode;
    h->at_rest = hd.at_rest;
    h->reduced = hd.reduced;
    h->sr = hd.sr;
    h->gx = hd.gx;
    h->gy = hd.gy;
    h->scale = hd.scale;
    h->seed = hd.seed;
    h->patience = hd.patience >= 1 ? hd.patience : 1;
    h->tstep = hd.tstep;
    h->steps = hd.steps;
    h->has_medium = true;
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

void glbm_debug_fail_launch(long long after) { g_fail_countdown.store(after < 0 ? -1 : after); }

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

bool ranges_overlap(const void *a, size_t na, const void *b, size_t nb) {
    if (!a || !b || !na || !nb) return false;
    const uintptr_t x = uintptr_t(a), y = uintptr_t(b);
    return x < y + nb && y < x + na;
}

template <int VEC, bool WALLS, bool FORCH>
void noalloc_launch(const float *src, float *dst, const float *a, const float *e, const float *b, const Geo &geo,
                    const Phys<float> &ph, double *partial, cudaStream_t st) {
    k_step<float, VEC, WALLS, FORCH, true><<<step_grid(geo), kThreads, 0, st>>>(src, dst, a, e, b, geo, ph, partial, nullptr);
}

}  // namespace

extern "C" glbm_status glbm_step_reduce_noalloc(const float *g_src, float *g_dst, const float *alpha,
                                                const float *eps, const float *beta, int nx, int ny,
                                                long long plane, double tau, double gx, double gy,
                                                unsigned flags, double *mean_u, void *stream) {
    if (!g_src || !g_dst || !alpha || !eps || !mean_u)
        return noalloc_fail(GLBM_EINVAL, "step_reduce_noalloc: g_src, g_dst, alpha, eps and mean_u are required");
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
    // The pull-stream reads g_src while the step writes g_dst: any overlap
    // between the buffer written and a buffer read gives wrong results.
    const size_t fbytes = size_t(9) * size_t(plane) * sizeof(float);
    const size_t cbytes = size_t(nx) * size_t(ny) * sizeof(float);
    struct Range {
        const void *p;
        size_t n;
        const char *name;
    };
    const Range reads[] = {{g_src, fbytes, "g_src"}, {alpha, cbytes, "alpha"}, {eps, cbytes, "eps"},
                           {beta, beta ? cbytes : 0, "beta"}};
    const Range writes[] = {{g_dst, fbytes, "g_dst"}, {mean_u, 2 * sizeof(double), "mean_u"}};
    for (const Range &w : writes)
        for (const Range &r : reads)
            if (ranges_overlap(w.p, w.n, r.p, r.n))
                return noalloc_fail(GLBM_EINVAL, "step_reduce_noalloc: %s overlaps %s", w.name, r.name);
    if (ranges_overlap(g_dst, fbytes, mean_u, 2 * sizeof(double)))
        return noalloc_fail(GLBM_EINVAL, "step_reduce_noalloc: mean_u overlaps g_dst");
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
