// Tensor-core (tcgen05) convolution for the warm-start network's inference
// on GB300 (sm_103a), plus the NHWC layout kernels around it.
//
// The network (a U-Net of 3x3 convolutions) is the library's own addition;
// the paper has no surrogate.  Its FP32 SIMT kernels (nn.cu) serve as the
// reference; this file runs the same convolutions on the 5th generation
// tensor cores (the training step's weight gradient is in nn_tc_train.cu).
// Three kernels, chosen per layer by glbm_nn_tc_conv:
//  * the tile kernel (below): any shape;
//  * the band kernel: 3x3 layers with 32 or 64 output channels, weights
//    resident in shared memory, each band's halo loaded once;
//  * the streaming kernel: the same layers where one CTA per image strip
//    gets a long segment of rows; it walks down the strip and keeps a ring
//    of output rows in tensor memory, so each input row is loaded and
//    multiplied once.
// The tile kernel:
//
//  * activations NHWC in BF16 (pixel stride = the buffer's channel count);
//    weights BF16 [tap][cout][cin]; FP32 accumulation in tensor memory;
//  * implicit GEMM: M = 128 output pixels (a tw x th tile of one image),
//    N = cout (16..256), K = taps x 32-channel chunks; per K step one TMA
//    load of the shifted pixel tile (hardware zero fill outside the image is
//    the convolution's zero padding) and one of the weight slice, both with
//    the 64-byte swizzle that the MMA's shared-memory descriptors read;
//  * the input channels may come from two tensors (c0 channels of x0, then
//    c1 of x1): the decoder's skip concatenation is never materialised;
//  * one CTA per output tile (two tiles stacked in y, sharing every weight
//    slice, when cout <= 64) with a 3-stage TMA ring (short, so that 4-6
//    CTAs share an SM and hide each other's latency; a grid that leaves
//    SMs empty takes a deeper ring instead): warp 0 issues TMA,
//    warp 1 issues tcgen05.mma
//    into a TMEM accumulator, warps 2-5 read it back (tcgen05.ld), add the
//    bias, apply ReLU and store BF16 NHWC (or FP32 NCHW for the head);
//  * every wait on an mbarrier is bounded: on timeout the CTA records a
//    code in *err, stops waiting, frees its TMEM and returns.

#include "tc_common.cuh"

__attribute__((visibility("hidden"))) int g_tc_starve = 0;
// 0 = choose per layer, 1 = tile kernel only (and the per-tap weight
// gradient), 2 = as 0 with the tile kernel's ring never deepened, 3 = band
// kernel never stacked, 4 = band kernel stacked but never streaming, 5 =
// streaming wherever it applies, however short its segments
// (glbm_nn_tc_set_variant).
__attribute__((visibility("hidden"))) int g_tc_variant = 0;

namespace {

struct TcConvArgs {
    int n, h, w, taps, nchunk0, nchunk, cout, tw, th;
    int starve;  // test hook: stage number + 1 the first CTA leaves unloaded
    uint32_t tmem_cols;  // MT accumulators of acc_cols columns
    uint32_t acc_cols;
    const float *bias;
    void *y;
    long long ys;  // output pixel stride (elements), NHWC output
    int relu, f32_nchw, cout_store;
    int *err;
};

// MT output tiles per CTA, stacked in y (tile t covers rows y0 + t th ..):
// they share every weight slice and accumulate into MT TMEM accumulators.
// S: depth of the TMA ring.
template <int MT, int S>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_tc_conv(const __grid_constant__ CUtensorMap mapA0, const __grid_constant__ CUtensorMap mapA1,
          const __grid_constant__ CUtensorMap mapB, const TcConvArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int stage_b = a.cout * TC_KC * 2;
    uint8_t *sA = smem;
    uint8_t *sB = smem + S * MT * TC_STAGE_A;
    __shared__ __align__(8) uint64_t full[S], empty[S], done;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int x0 = blockIdx.x * a.tw, y0 = blockIdx.y * (MT * a.th), img = blockIdx.z;
    const int iters = a.taps * a.nchunk;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(&tmem_base, a.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            const uint32_t bytes = uint32_t(MT * a.tw * a.th * TC_KC * 2 + stage_b);
            int i = 0;
            for (; i < iters; ++i) {
                const int s = i % S, use = i / S;
                if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1, &abort_flag, a.err, 1)) break;
                const int tap = i / a.nchunk, ch = i - tap * a.nchunk;
                const int dy = a.taps == 9 ? tap / 3 - 1 : 0, dx = a.taps == 9 ? tap % 3 - 1 : 0;
                mbar_expect_tx(&full[s], bytes);
                if (a.starve == i + 1 && blockIdx.x + blockIdx.y + blockIdx.z == 0) continue;
#pragma unroll
                for (int t = 0; t < MT; ++t) {
                    uint8_t *dst = sA + (s * MT + t) * TC_STAGE_A;
                    const int yt = y0 + t * a.th + dy;
                    if (ch < a.nchunk0)
                        tma_load_4d(dst, &mapA0, &full[s], ch * TC_KC, x0 + dx, yt, img);
                    else
                        tma_load_4d(dst, &mapA1, &full[s], (ch - a.nchunk0) * TC_KC, x0 + dx, yt, img);
                }
                tma_load_3d(sB + s * stage_b, &mapB, &full[s], ch * TC_KC, 0, tap);
            }
            drain_ring(full, S, i);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(a.cout);
            for (int i = 0; i < iters; ++i) {
                const int s = i % S, use = i / S;
                if (!mbar_wait(&full[s], use & 1, &abort_flag, a.err, 2)) break;
                tc_fence_after();
                const uint64_t bd = sdesc_k64(sB + s * stage_b);
#pragma unroll
                for (int t = 0; t < MT; ++t) {
                    const uint64_t ad = sdesc_k64(sA + (s * MT + t) * TC_STAGE_A);
#pragma unroll
                    for (int kk = 0; kk < TC_KC / 16; ++kk)  // K = 16 per MMA: 32 bytes along the row
                        umma_bf16(tmem + uint32_t(t) * a.acc_cols, ad + uint64_t((kk * 32) >> 4),
                                  bd + uint64_t((kk * 32) >> 4), idesc, (i > 0 || kk > 0) ? 1u : 0u);
                }
                umma_commit(&empty[s]);
            }
            umma_commit(&done);  // after a timeout too: the wait below retires every MMA issued
            mbar_drain(&done, 0);
        }
    } else {
        const int q = warp & 3;  // TMEM lanes 32q..32q+31 belong to this warp
        // after a timeout the MMA warp still commits `done` (to retire its MMAs):
        // the accumulator is then not a result
        const bool have = mbar_wait(&done, 0, &abort_flag, a.err, 3) && !abort_flag;
        tc_fence_after();
        for (int t = 0; t < MT && have; ++t) {
            const int m = q * 32 + lane;
            const int px = x0 + m % a.tw, py = y0 + t * a.th + m / a.tw;
            const bool ok = m < a.tw * a.th && px < a.w && py < a.h;
            const long long pix = ((long long)img * a.h + py) * a.w + px;
            for (int c = 0; c < a.cout; c += 16) {
                float v[16];
                tmem_ld16(tmem + uint32_t(t) * a.acc_cols + (uint32_t(q * 32) << 16) + uint32_t(c), v);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    v[j] += a.bias[c + j];
                    if (a.relu) v[j] = fmaxf(v[j], 0.0f);
                }
                if (!ok) continue;
                if (a.f32_nchw) {
                    float *yo = static_cast<float *>(a.y);
                    const long long hw = (long long)a.h * a.w;
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (c + j < a.cout_store)
                            yo[((long long)img * a.cout_store + c + j) * hw + (long long)py * a.w + px] = v[j];
                } else {
                    uint32_t pk[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        __nv_bfloat162 b2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                        pk[j] = *reinterpret_cast<uint32_t *>(&b2);
                    }
                    uint4 *dst = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(a.y) + pix * a.ys + c);
                    dst[0] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                    dst[1] = make_uint4(pk[4], pk[5], pk[6], pk[7]);
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, a.tmem_cols);
    }
}

// ---- Band variant for the shallow layers ------------------------------------
// With 32-96 input and 32-64 output channels a 128-pixel tile is only a few
// hundred tensor-core cycles, and the tile kernel above re-reads every input
// pixel nine times (one shifted tile per tap) through L2.  This persistent
// variant keeps all weight slices resident in shared memory and works on
// bands of R output rows x 128 pixels: per 32-channel chunk it loads the
// band's halo, rows y0-1 .. y0+R of pixels x0-1 .. x0+128, ONCE, in the
// unswizzled K-major layout
//     [8-channel block][halo row][halo pixel][8 channels = 16 bytes],
// where the A operand of output row r and tap (dy, dx) is a view starting
// ((r+1+dy) * 130 + 1+dx) * 16 bytes in: core matrices of 8 pixels are 128 B
// apart along M (SBO) and 8-channel blocks one block stride apart along K
// (LBO).  Each band accumulates R rows into one of two TMEM buffers, so the
// epilogue of one band overlaps the MMAs of the next.  The halo arrives by
// TMA, one box of 8 channels x 130 pixels x (R + 2) rows per 8-channel block
// (zero fill outside the image is the padding).  With 32 output channels the
// three vertical taps are stacked along N: one MMA of 96 columns per halo
// row, horizontal tap and 16 channels feeds three output rows' accumulator
// slots at once (each band first clears its slots with MMAs of an all-zero
// A operand and accumulate = 0).
// Roles: warp 0 issues TMA, warp 3 the MMAs, warps 4-7 run the epilogue
// (warps 1-2 idle: the TMEM lane quarters fix the epilogue to warps whose
// index is 0-3 mod 4); every wait is bounded.
constexpr int BAND_PX = TC_M + 2;   // halo pixels per row
constexpr int BAND_THREADS = 256;

struct BandArgs {
    int n, h, w, nchunk0, nchunk, cout, R, stages;
    int starve;  // test hook: stage number + 1 the first CTA leaves unloaded
    int nbx, nby;
    long long nbands;
    uint32_t blk_stride;   // bytes between 8-channel blocks of a stage (LBO)
    uint32_t stage_bytes;  // 4 blocks
    uint32_t tx_bytes;     // bytes the 4 TMA loads of a stage deliver
    uint32_t wtile;        // bytes of one weight slice (cout rows x 64 B)
    uint32_t acc_row;      // TMEM columns per output row (power of two >= cout)
    uint32_t acc_cols;     // TMEM columns of one accumulator buffer (R * acc_row)
    uint32_t tmem_cols;
    const __nv_bfloat16 *x0, *x1;  // NHWC inputs with c0 / c1 channels per pixel
    int c0, c1;
    int stack;  // 1: the three dy taps stacked along N (see k_tc_conv_band)
    const float *bias;
    void *y;               // BF16 NHWC output, or NULL (only the fused outputs below)
    long long ys;
    int relu;
    int *err;
    // fused outputs: the 2x2 average of the BF16 output (BF16 NHWC, h/2 x
    // w/2, cout channels; 32 or 64 output channels), and (32 output
    // channels, stacked) a 1x1 head of head_out <= 4 channels (BF16 weights
    // [head_out][32], FP32 bias) on the BF16-rounded output, written FP32 NCHW
    __nv_bfloat16 *pool_y;
    const __nv_bfloat16 *head_w;
    const float *head_b;
    float *head_y;
    int head_out;
};

// Two groups of 32 consecutive FP32 columns of this thread's TMEM lane,
// both loads in flight before one wait (the values are outputs of the same
// statement, so nothing reads them early).
__device__ __forceinline__ void tmem_ld32x2(uint32_t ta, uint32_t tb, float (&v0)[32], float (&v1)[32]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%64];\n"
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%32, %33, %34, %35, %36, %37, %38, %39, %40, %41, %42, %43, %44, %45, %46, %47, %48, %49, %50, %51, %52, %53, %54, %55, %56, %57, %58, %59, %60, %61, %62, %63}, [%65];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=f"(v0[0]), "=f"(v0[1]), "=f"(v0[2]), "=f"(v0[3]), "=f"(v0[4]), "=f"(v0[5]), "=f"(v0[6]), "=f"(v0[7]), "=f"(v0[8]), "=f"(v0[9]), "=f"(v0[10]), "=f"(v0[11]), "=f"(v0[12]), "=f"(v0[13]), "=f"(v0[14]), "=f"(v0[15]), "=f"(v0[16]), "=f"(v0[17]), "=f"(v0[18]), "=f"(v0[19]), "=f"(v0[20]), "=f"(v0[21]), "=f"(v0[22]), "=f"(v0[23]), "=f"(v0[24]), "=f"(v0[25]), "=f"(v0[26]), "=f"(v0[27]), "=f"(v0[28]), "=f"(v0[29]), "=f"(v0[30]), "=f"(v0[31]), "=f"(v1[0]), "=f"(v1[1]), "=f"(v1[2]), "=f"(v1[3]), "=f"(v1[4]), "=f"(v1[5]), "=f"(v1[6]), "=f"(v1[7]), "=f"(v1[8]), "=f"(v1[9]), "=f"(v1[10]), "=f"(v1[11]), "=f"(v1[12]), "=f"(v1[13]), "=f"(v1[14]), "=f"(v1[15]), "=f"(v1[16]), "=f"(v1[17]), "=f"(v1[18]), "=f"(v1[19]), "=f"(v1[20]), "=f"(v1[21]), "=f"(v1[22]), "=f"(v1[23]), "=f"(v1[24]), "=f"(v1[25]), "=f"(v1[26]), "=f"(v1[27]), "=f"(v1[28]), "=f"(v1[29]), "=f"(v1[30]), "=f"(v1[31])
        : "r"(ta), "r"(tb)
        : "memory");
}

// Shared-memory descriptor of an unswizzled K-major operand: core matrices
// (8 rows x 16 B) `sbo` bytes apart along M/N and `lbo` bytes apart along K.
__device__ __forceinline__ uint64_t sdesc_nosw(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return uint64_t((addr >> 4) & 0x3FFFu) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) |
           (uint64_t((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

__global__ void __launch_bounds__(BAND_THREADS, 1)
k_tc_conv_band(const __grid_constant__ CUtensorMap mapA0, const __grid_constant__ CUtensorMap mapA1,
               const __grid_constant__ CUtensorMap mapB, const BandArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int ntile_w = 9 * a.nchunk;
    uint8_t *sW = smem;
    uint8_t *sA = smem + size_t(ntile_w) * a.wtile;
    constexpr int SMAX = 3;
    __shared__ __align__(8) uint64_t full[SMAX], empty[SMAX], wfull, accfull[2], accempty[2], drainbar;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    __shared__ float sbias[64];
    __shared__ float shead[4 * 32], shead_b[4];

    // an all-zero A operand (128 rows x 16 K, unswizzled): MMAs with it and
    // accumulate = 0 clear the stacked accumulator slots of a band
    __shared__ __align__(128) uint8_t szero[4096];

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = a.stages;
    if (threadIdx.x < a.cout) sbias[threadIdx.x] = a.bias[threadIdx.x];
    if (a.head_y && threadIdx.x < a.head_out * 32) shead[threadIdx.x] = __bfloat162float(a.head_w[threadIdx.x]);
    if (a.head_y && threadIdx.x < a.head_out) shead_b[threadIdx.x] = a.head_b[threadIdx.x];
    for (int j = threadIdx.x; j < 4096 / 16; j += blockDim.x) reinterpret_cast<uint4 *>(szero)[j] = make_uint4(0, 0, 0, 0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&wfull, 1);
        mbar_init(&drainbar, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&accfull[b], 1);
            mbar_init(&accempty[b], 4);  // one arrival per epilogue warp
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 3) tmem_alloc(&tmem_base, a.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            mbar_expect_tx(&wfull, uint32_t(ntile_w) * a.wtile);
            for (int tap = 0; tap < 9; ++tap)
                for (int ch = 0; ch < a.nchunk; ++ch)
                    tma_load_3d(sW + size_t(a.stack ? ((ch * 3 + tap % 3) * 3 + (2 - tap / 3)) : (tap * a.nchunk + ch)) *
                                         a.wtile,
                                &mapB, &wfull, ch * TC_KC, 0, tap);
            long long i = 0;
            bool go = true;
            for (long long band = blockIdx.x; band < a.nbands && go; band += gridDim.x) {
                const int bx = int(band % a.nbx);
                const long long rest = band / a.nbx;
                const int by = int(rest % a.nby), img = int(rest / a.nby);
                const int x0 = bx * TC_M, y0 = by * a.R;
                for (int ch = 0; ch < a.nchunk; ++ch, ++i) {
                    const int s = int(i % S);
                    const long long use = i / S;
                    if (use > 0 && !mbar_wait(&empty[s], uint32_t(use - 1) & 1u, &abort_flag, a.err, 11)) {
                        go = false;
                        break;
                    }
                    mbar_expect_tx(&full[s], a.tx_bytes);
                    if (a.starve == i + 1 && blockIdx.x == 0) continue;
                    uint8_t *dst = sA + size_t(s) * a.stage_bytes;
                    const bool first = ch < a.nchunk0;
                    const int c0 = (first ? ch : ch - a.nchunk0) * TC_KC;
#pragma unroll
                    for (int blk = 0; blk < 4; ++blk)
                        tma_load_4d(dst + blk * a.blk_stride, first ? &mapA0 : &mapA1, &full[s], c0 + blk * 8,
                                    x0 - 1, y0 - 1, img);
                }
            }
            mbar_drain(&wfull, 0);
            drain_ring(full, S, i);
        }
    } else if (warp == 3) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16(a.stack ? 3 * a.cout : a.cout);
            bool ok = mbar_wait(&wfull, 0, &abort_flag, a.err, 12);
            tc_fence_after();
            long long i = 0, t = 0;
            for (long long band = blockIdx.x; band < a.nbands && ok; band += gridDim.x, ++t) {
                const int ab = int(t & 1);
                const long long use_ab = t >> 1;
                if (use_ab > 0 && !mbar_wait(&accempty[ab], uint32_t(use_ab - 1) & 1u, &abort_flag, a.err, 13)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t acc = tmem + uint32_t(ab) * a.acc_cols;
                if (a.stack) {
                    // clear the band's slots: zero A times any finite B, accumulate = 0,
                    // windows of 3 cout columns covering [0, acc_cols)
                    const uint64_t z = sdesc_nosw(smem_u32(szero), 2048u, 128u);
                    const uint64_t bw = sdesc_k64(sW);
                    const uint32_t n3 = uint32_t(3 * a.cout);
                    for (uint32_t c0 = 0;; c0 += n3) {
                        const uint32_t c = c0 + n3 > a.acc_cols ? a.acc_cols - n3 : c0;
                        umma_bf16(acc + c, z, bw, idesc, 0u);
                        if (c0 + n3 >= a.acc_cols) break;
                    }
                }
                for (int ch = 0; ch < a.nchunk; ++ch, ++i) {
                    const int s = int(i % S);
                    if (!mbar_wait(&full[s], uint32_t(i / S) & 1u, &abort_flag, a.err, 14)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t base = smem_u32(sA + size_t(s) * a.stage_bytes);
                    if (a.stack) {
                        // N = 3 cout: B stacks the weights of dy = +1, 0, -1 for one dx, so
                        // one MMA on halo row i adds to output rows i-2, i-1, i, whose
                        // accumulator slots (row + 2) are contiguous: D = acc + i cout.
                        const uint64_t a0 = sdesc_nosw(base, a.blk_stride, 128u);
                        const uint64_t b0 = sdesc_k64(sW + size_t(ch * 9) * a.wtile);
                        const uint32_t bstep = (3 * a.wtile) >> 4, kstep = (2 * a.blk_stride) >> 4;
                        for (int hr = 0; hr < a.R + 2; ++hr) {
                            const uint32_t d = acc + uint32_t(hr * a.cout);
                            const uint64_t arow = a0 + uint64_t(hr * BAND_PX);  // 16-byte units
#pragma unroll
                            for (int dxi = 0; dxi < 3; ++dxi)
#pragma unroll
                                for (int kk = 0; kk < 2; ++kk)
                                    umma_bf16(d, arow + uint64_t(dxi + kk * kstep),
                                              b0 + uint64_t(dxi * bstep + kk * 2), idesc, 1u);
                        }
                        umma_commit(&empty[s]);
                        continue;
                    }
                    for (int tap = 0; tap < 9; ++tap) {
                        const int dy = tap / 3 - 1, dx = tap % 3 - 1;
                        const uint64_t bd = sdesc_k64(sW + size_t(tap * a.nchunk + ch) * a.wtile);
                        for (int r = 0; r < a.R; ++r) {
                            const uint32_t pix = uint32_t((r + 1 + dy) * BAND_PX + 1 + dx) * 16u;
#pragma unroll
                            for (int kk = 0; kk < 2; ++kk) {
                                const uint64_t ad = sdesc_nosw(base + pix + uint32_t(2 * kk) * a.blk_stride,
                                                               a.blk_stride, 128u);
                                umma_bf16(acc + uint32_t(r) * a.acc_row, ad, bd + uint64_t((kk * 32) >> 4), idesc,
                                          (ch > 0 || tap > 0 || kk > 0) ? 1u : 0u);
                            }
                        }
                    }
                    umma_commit(&empty[s]);
                }
                if (!ok) break;
                umma_commit(&accfull[ab]);
            }
            umma_commit(&drainbar);  // retire every MMA issued, also after a timeout
            mbar_drain(&drainbar, 0);
        }
    } else if (warp >= 4) {
        // Epilogue: per output row one TMEM load of the pixel's channels (32
        // columns per load, one wait), bias, ReLU, BF16, 16-byte stores.
        const int q = warp & 3;  // TMEM lanes 32q..32q+31 belong to this warp
        long long t = 0;
        for (long long band = blockIdx.x; band < a.nbands; band += gridDim.x, ++t) {
            const int ab = int(t & 1);
            if (!mbar_wait(&accfull[ab], uint32_t(t >> 1) & 1u, &abort_flag, a.err, 15)) break;
            tc_fence_after();
            const int bx = int(band % a.nbx);
            const long long rest = band / a.nbx;
            const int by = int(rest % a.nby), img = int(rest / a.nby);
            const int px = bx * TC_M + q * 32 + lane;
            // two 32-column groups per TMEM wait: two rows of 32 channels, or
            // one row of 64; with pooling always the same 32 channels of two
            // rows 2k, 2k + 1 (R is even)
            const uint32_t lanes = uint32_t(q * 32) << 16;
            const uint32_t buf = tmem + uint32_t(ab) * a.acc_cols + lanes;
            const int first_slot = a.stack ? 2 : 0;
            const int ncg = a.cout / 32;
            const int ngroups = a.R * ncg;
            for (int g = 0; g < ngroups; g += 2) {
                float v[2][32];
                int rr[2], cc0[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    if (a.pool_y) {
                        rr[u] = (g / 2 / ncg) * 2 + u;
                        cc0[u] = (g / 2 % ncg) * 32;
                    } else {
                        const int gg = g + u < ngroups ? g + u : g;  // an odd last group loads twice
                        rr[u] = gg / ncg;
                        cc0[u] = (gg % ncg) * 32;
                    }
                }
                tmem_ld32x2(buf + uint32_t(rr[0] + first_slot) * a.acc_row + uint32_t(cc0[0]),
                            buf + uint32_t(rr[1] + first_slot) * a.acc_row + uint32_t(cc0[1]), v[0], v[1]);
                // bias, ReLU, BF16 rounding (the fused outputs start from the
                // rounded values, as the separate kernels would read them)
#pragma unroll
                for (int u = 0; u < 2; ++u)
#pragma unroll
                    for (int cc = 0; cc < 32; ++cc) {
                        float x = v[u][cc] + sbias[cc0[u] + cc];
                        if (a.relu) x = fmaxf(x, 0.0f);
                        v[u][cc] = __bfloat162float(__float2bfloat16_rn(x));
                    }
                const bool colok = px < a.w;
                if (a.y) {
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        if (g + u >= ngroups) break;
                        const int py = by * a.R + rr[u];
                        if (!colok || py >= a.h) continue;
                        uint4 *dst = reinterpret_cast<uint4 *>(static_cast<__nv_bfloat16 *>(a.y) +
                                                               (((long long)img * a.h + py) * a.w + px) * a.ys + cc0[u]);
#pragma unroll
                        for (int j4 = 0; j4 < 4; ++j4) {
                            uint32_t pk[4];
#pragma unroll
                            for (int j = 0; j < 4; ++j) {
                                __nv_bfloat162 b2 = __floats2bfloat162_rn(v[u][j4 * 8 + 2 * j], v[u][j4 * 8 + 2 * j + 1]);
                                pk[j] = *reinterpret_cast<uint32_t *>(&b2);
                            }
                            dst[j4] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
                        }
                    }
                }
                if (a.head_y) {
                    // 1x1 head on this pixel's 32 channels, per row of the pair
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        if (g + u >= ngroups) break;
                        const int py = by * a.R + rr[u];
                        for (int k = 0; k < a.head_out; ++k) {
                            float acc_h = 0.0f;
#pragma unroll
                            for (int cc = 0; cc < 32; ++cc) acc_h = fmaf(v[u][cc], shead[k * 32 + cc], acc_h);
                            if (colok && py < a.h)
                                a.head_y[(((long long)img * a.head_out + k) * a.h + py) * a.w + px] = acc_h + shead_b[k];
                        }
                    }
                }
                if (a.pool_y) {
                    // rows rr[0], rr[0] + 1 (even) of the pair and pixels px, px ^ 1 (lanes
                    // lane, lane ^ 1): FP32 ((a + b) + (d + e)) / 4, rounded to BF16
                    const int pyo = (by * a.R + rr[0]) >> 1;
                    const bool wr = (lane & 1) == 0 && colok && pyo < (a.h >> 1);
                    uint32_t pk[16];
#pragma unroll
                    for (int cc = 0; cc < 32; cc += 2) {
                        float s2[2];
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const float mine_top = v[0][cc + e], mine_bot = v[1][cc + e];
                            const float nb_top = __shfl_xor_sync(0xffffffffu, mine_top, 1);
                            const float nb_bot = __shfl_xor_sync(0xffffffffu, mine_bot, 1);
                            s2[e] = 0.25f * ((mine_top + nb_top) + (mine_bot + nb_bot));
                        }
                        __nv_bfloat162 b2 = __floats2bfloat162_rn(s2[0], s2[1]);
                        pk[cc / 2] = *reinterpret_cast<uint32_t *>(&b2);
                    }
                    if (wr) {
                        uint4 *dst = reinterpret_cast<uint4 *>(
                            a.pool_y + (((long long)img * (a.h >> 1) + pyo) * (a.w >> 1) + (px >> 1)) * a.cout +
                            cc0[0]);
#pragma unroll
                        for (int j4 = 0; j4 < 4; ++j4)
                            dst[j4] = make_uint4(pk[4 * j4], pk[4 * j4 + 1], pk[4 * j4 + 2], pk[4 * j4 + 3]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&accempty[ab])) : "memory");
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 3) {
        tc_fence_after();
        tmem_dealloc(tmem, a.tmem_cols);
    }
}

// ---- Streaming variant for 32 and 64 output channels --------------------------
// The band kernel above clears and drains its accumulator per band of R = 4
// rows: the stacked MMA of each of the band's R + 2 halo rows also feeds the
// two rows above and below the band, 1.5x the MMAs the outputs need, and the
// MMA and epilogue warps hand each band's two TMEM buffers back and forth.
// Here each CTA owns one 128-pixel strip of one image and a segment of L
// output rows and walks down it input row by input row.  TMEM holds a ring
// of 16 row slots of 32 columns: input row r adds, in one MMA of N = 96 per
// horizontal tap and 16 channels, to the slots of output rows r - 1, r and
// r + 1 (B stacks the weights of dy = +1, 0, -1), so every input row is
// multiplied once; output row r - 1 is then complete.  Rows are handed to the
// epilogue in pairs (8 pair slots in flight), so the MMA warp runs several
// row pairs ahead of the epilogue.  Where the three slots of a row wrap the
// ring (slots 14, 15, 0 or 15, 0, 1) the row takes two MMAs of the same
// shape (an MMA of another N in between stalls the tensor pipe): one on
// slots 13-15 and one on slots 0-2, their B windows shifted over zero tiles
// so that each adds only its part.  The weights of one (chunk, dx) sit as
// [0 0 W(+1) W(0) W(-1) 0 0] in shared memory, neighbours sharing their
// zero tiles.
// With 64 output channels the ring has 8 slots of 64 columns.  Where the
// stacked weights with their zero tiles fit in shared memory (STK), each
// input row takes one N = 192 MMA per tap and K step as above; otherwise
// three N = 64 MMAs, one per output row (no stacking, so no ring wrap inside
// an MMA).  A single thread issues MMAs no faster than about one per 46
// cycles whatever their size, so fewer, larger MMAs win.  Groups of two
// input rows leave the epilogue two groups of slack in the 4 pair slots.
// Where the weights do not fit in shared memory (wstream), each stage brings
// the nine weight tiles of its chunk along with its input rows (stacked: in
// the 17-tile layout with its zero tiles; else four-row groups, so that each
// weight tile serves four rows per load).  With up2 the epilogue writes the
// output 2x nearest-upsampled by TMA stores from a staged row pair.
// Roles: warp 0 TMA (G input rows of one 32-channel chunk per stage: boxes
// of G rows, as tall as the band kernel's, keep the TMA engine streaming),
// warp 1 MMA and TMEM, warps 4-7 epilogue (one per lane quarter); every wait
// is bounded.
constexpr int ST_THREADS = 256;
constexpr int ST_SLOTS = 16;
constexpr int ST_PAIRS = ST_SLOTS / 2;
constexpr int ST_SMAX = 12;

struct StreamArgs {
    int n, h, w, nchunk0, nchunk, nbx, nseg, L, stages;
    int starve;  // test hook: stage number + 1 the first CTA leaves unloaded
    int nblk;              // 8-channel blocks per chunk: 4, or 2 for a 16-channel input
    uint32_t blk_stride;   // bytes between the 8-channel blocks of a stage (LBO)
    uint32_t stage_bytes;  // 4 blocks
    uint32_t tx_bytes;     // bytes the 4 TMA loads of a stage deliver
    uint32_t wtile;        // bytes of one weight slice (32 rows x 64 B)
    const float *bias;
    void *y;  // BF16 NHWC output, or NULL (only the fused outputs)
    long long ys;
    int relu;
    int *err;
    __nv_bfloat16 *pool_y;  // as in BandArgs
    const __nv_bfloat16 *head_w;
    const float *head_b;
    float *head_y;
    int head_out;
    // 1: the output goes 2x nearest-upsampled to y by TMA stores (mapY0 /
    // mapY1: even / odd output columns) from a staged row pair; y unused
    int up2;
    int ystages;             // staged row pairs: 2 (double buffered) or 1
    uint32_t stage_y_bytes;  // one staged row: 128 pixels x COUT BF16
    // 1: no resident weights; a stage = input rows (wofs bytes) + the nine
    // weight tiles of its chunk
    int wstream;
    uint32_t wofs;
};

template <int G, int COUT, bool STK>
__global__ void __launch_bounds__(ST_THREADS, 1)
k_tc_conv_stream(const __grid_constant__ CUtensorMap mapA0, const __grid_constant__ CUtensorMap mapA1,
                 const __grid_constant__ CUtensorMap mapB, const __grid_constant__ CUtensorMap mapY0,
                 const __grid_constant__ CUtensorMap mapY1, const StreamArgs a) {
    constexpr bool STACK = STK;  // dy taps stacked along N (N = 3 COUT)
    constexpr int NS = 512 / COUT;      // TMEM row slots
    constexpr int NP = NS / 2;          // row pair slots
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    const int ntile_w = 9 * a.nchunk;
    const int nslot_w = a.wstream ? 0 : (STACK ? 15 * a.nchunk + 2 : ntile_w);  // stacked: with zero tiles
    uint8_t *sW = smem;
    uint8_t *sA = smem + size_t(nslot_w) * a.wtile;
    // up2: two buffers of a staged row pair after the stages
    uint8_t *sY = sA + size_t(a.stages) * a.stage_bytes;
    __shared__ int s_bad;  // up2: an epilogue wait gave up (all four warps leave together)
    __shared__ __align__(8) uint64_t full[ST_SMAX], empty[ST_SMAX], wfull, pfull[ST_PAIRS], pempty[ST_PAIRS], drainbar;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    __shared__ __align__(16) float sbias[COUT];
    __shared__ __align__(16) float shead[4 * 32];
    __shared__ float shead_b[4];
    __shared__ __align__(128) uint8_t szero[4096];  // all-zero A (128 rows x 16 K, unswizzled)

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int S = a.stages;
    const int seg = int(blockIdx.x % unsigned(a.nseg));
    const int rest = int(blockIdx.x / unsigned(a.nseg));
    const int bx = rest % a.nbx, img = rest / a.nbx;
    const int ya = seg * a.L;
    const int Lseg = min(a.L, a.h - ya);
    // input rows ya - 1 .. ya + Lseg (local index ir = 0 .. Lseg + 1), G per
    // group; output row j (row ya - 2 + j, slot j mod NS) takes input rows
    // j - 2 .. j, so row pair P (j = 2P, 2P + 1) is complete after the group
    // holding input row 2P + 1; pair 0 (rows above the segment) is never
    // stored, pairs 1 .. npairs are
    constexpr int hg = G / 2;
    const int ngroups = (Lseg + 2 + G - 1) / G;
    const int npairs = (Lseg + 1) / 2;
    if (threadIdx.x < COUT) sbias[threadIdx.x] = a.bias[threadIdx.x];
    // head weights, zero for the outputs beyond head_out (computed, never stored)
    if (threadIdx.x < 4 * 32)
        shead[threadIdx.x] =
            a.head_y && threadIdx.x < a.head_out * 32 ? __bfloat162float(a.head_w[threadIdx.x]) : 0.0f;
    if (a.head_y && threadIdx.x < a.head_out) shead_b[threadIdx.x] = a.head_b[threadIdx.x];
    for (int j = threadIdx.x; j < 4096 / 16; j += blockDim.x) reinterpret_cast<uint4 *>(szero)[j] = make_uint4(0, 0, 0, 0);
    if (STACK) {
        // the zero tiles: 0, 1 and 5 + 5k, 6 + 5k around (chunk, dx) group k,
        // in the resident weights or, with wstream, in every stage's 17 tiles
        const int per = int(a.wtile / 16);
        const int nw = a.wstream ? 17 : nslot_w;
        for (int st = 0; st < (a.wstream ? a.stages : 1); ++st) {
            uint4 *wz = reinterpret_cast<uint4 *>(a.wstream ? sA + size_t(st) * a.stage_bytes + a.wofs : sW);
            for (int j = threadIdx.x; j < nw * per; j += blockDim.x) {
                const int t = j / per;
                if (t < 2 || (t - 2) % 5 >= 3) wz[j] = make_uint4(0, 0, 0, 0);
            }
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&wfull, 1);
        mbar_init(&drainbar, 1);
        for (int p = 0; p < NP; ++p) {
            mbar_init(&pfull[p], 1);
            mbar_init(&pempty[p], 4);  // the four lane-quarter epilogue warps
        }
        abort_flag = 0;
        s_bad = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(&tmem_base, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const int x0 = bx * TC_M;

    if (warp == 0) {
        if (lane == 0) {
            if (!a.wstream) {
                mbar_expect_tx(&wfull, uint32_t(ntile_w) * a.wtile);
                for (int tap = 0; tap < 9; ++tap)
                    for (int ch = 0; ch < a.nchunk; ++ch)
                        tma_load_3d(
                            sW + size_t(STACK ? 2 + 5 * (ch * 3 + tap % 3) + (2 - tap / 3) : tap * a.nchunk + ch) *
                                     a.wtile,
                            &mapB, &wfull, ch * TC_KC, 0, tap);
            }
            long long i = 0;
            bool go = true;
            for (int g = 0; g < ngroups && go; ++g)
                for (int ch = 0; ch < a.nchunk; ++ch, ++i) {
                    const int s = int(i % S);
                    const long long use = i / S;
                    if (use > 0 && !mbar_wait_idle(&empty[s], uint32_t(use - 1) & 1u, &abort_flag, a.err, 21)) {
                        go = false;
                        break;
                    }
                    mbar_expect_tx(&full[s], a.tx_bytes);
                    if (a.starve == i + 1 && blockIdx.x == 0) continue;
                    uint8_t *dst = sA + size_t(s) * a.stage_bytes;
                    const bool first = ch < a.nchunk0;
                    const int c0 = (first ? ch : ch - a.nchunk0) * TC_KC;
                    for (int blk = 0; blk < a.nblk; ++blk)
                        tma_load_4d(dst + blk * a.blk_stride, first ? &mapA0 : &mapA1, &full[s], c0 + blk * 8,
                                    x0 - 1, ya - 1 + G * g, img);
                    if (a.wstream)
                        for (int tap = 0; tap < 9; ++tap)
                            tma_load_3d(dst + a.wofs +
                                            size_t(STACK ? 2 + 5 * (tap % 3) + (2 - tap / 3) : tap) * a.wtile,
                                        &mapB, &full[s], ch * TC_KC, 0, tap);
                }
            if (!a.wstream) mbar_drain(&wfull, 0);
            drain_ring(full, S, i);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA shapes: the main N (3 COUT stacked, else COUT) and the clearing
            // of a row pair's two slots
            const uint32_t idN = idesc_bf16(STACK ? 3 * COUT : COUT), idZ = idesc_bf16(STACK ? 2 * COUT : COUT);
            bool ok = a.wstream || mbar_wait(&wfull, 0, &abort_flag, a.err, 22);
            tc_fence_after();
            const uint64_t zdesc = sdesc_nosw(smem_u32(szero), 2048u, 128u);
            const uint64_t wdesc = sdesc_k64(sW);
            const uint32_t wt16 = a.wtile >> 4, kstep = (2 * a.blk_stride) >> 4;
            const int kks = a.nblk / 2;  // K steps of 16 channels per chunk
            const uint32_t d13 = uint32_t((NS - 3) * COUT);
            long long i = 0;
            for (int g = 0; g < ngroups && ok; ++g) {
                // pairs hg g + 1 .. hg g + hg enter their slots: wait until the
                // epilogue has drained each one's last stored occupant, then
                // clear them
                for (int pn = hg * g + 1; pn <= hg * g + hg && ok; ++pn) {
                    const int ps = pn % NP, prev = pn - NP;
                    if (prev >= 1 && prev <= npairs &&
                        !mbar_wait(&pempty[ps], uint32_t((prev - 1) / NP) & 1u, &abort_flag, a.err, 23)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    if (STACK) {
                        umma_bf16(tmem + uint32_t(2 * ps * COUT), zdesc, zdesc, idZ, 0u);
                    } else {
                        umma_bf16(tmem + uint32_t(2 * ps * COUT), zdesc, zdesc, idZ, 0u);
                        umma_bf16(tmem + uint32_t((2 * ps + 1) * COUT), zdesc, zdesc, idZ, 0u);
                    }
                }
                for (int ch = 0; ch < a.nchunk && ok; ++ch, ++i) {
                    const int s = int(i % S);
                    if (!mbar_wait(&full[s], uint32_t(i / S) & 1u, &abort_flag, a.err, 24)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t a0 = sdesc_nosw(smem_u32(sA + size_t(s) * a.stage_bytes), a.blk_stride, 128u);
                    if (!STACK) {
                        // input row G g + ri adds W(dy) to output row G g + ri + 1 - dy; the
                        // weight tile of (tap, chunk) is resident or in this stage
                        const uint64_t wbase = a.wstream ? sdesc_k64(sA + size_t(s) * a.stage_bytes + a.wofs) : wdesc;
#pragma unroll 1
                        for (int ri = 0; ri < G; ++ri) {
                            const uint64_t arow = a0 + uint64_t(ri * BAND_PX);  // 16-byte units
#pragma unroll
                            for (int o = 0; o < 3; ++o) {
                                const uint32_t d = tmem + uint32_t(((G * g + ri + o) % NS) * COUT);
#pragma unroll
                                for (int dxi = 0; dxi < 3; ++dxi) {
                                    const int tap = (2 - o) * 3 + dxi;
                                    const uint64_t bt =
                                        wbase + uint64_t(a.wstream ? tap : tap * a.nchunk + ch) * wt16;
#pragma unroll
                                    for (int kk = 0; kk < 2; ++kk)
                                        if (kk < kks)
                                            umma_bf16(d, arow + uint64_t(dxi + kk * kstep), bt + uint64_t(kk * 2),
                                                      idN, 1u);
                                }
                            }
                        }
                        umma_commit(&empty[s]);
                        continue;
                    }
                    // B of (chunk, dx) group k starts at tile 2 + 5k: [W(+1) W(0) W(-1)];
                    // with wstream the stage holds this chunk's 17 tiles
                    const uint64_t b0 = a.wstream
                                            ? sdesc_k64(sA + size_t(s) * a.stage_bytes + a.wofs) + uint64_t(2 * wt16)
                                            : sdesc_k64(sW) + uint64_t((2 + 15 * ch) * wt16);
#pragma unroll 1
                    for (int ri = 0; ri < G; ++ri) {
                        // input row G g + ri feeds the slots of rows G g + ri .. + 2
                        const int s0 = (G * g + ri) % NS;
                        const uint64_t arow = a0 + uint64_t(ri * BAND_PX);  // 16-byte units
                        if (s0 <= NS - 3) {
                            const uint32_t d0 = tmem + uint32_t(s0 * COUT);
#pragma unroll
                            for (int dxi = 0; dxi < 3; ++dxi)
#pragma unroll
                                for (int kk = 0; kk < 2; ++kk)
                                    if (kk < kks)
                                        umma_bf16(d0, arow + uint64_t(dxi + kk * kstep),
                                                  b0 + uint64_t(5 * dxi * wt16 + kk * 2), idN, 1u);
                        } else {
                            // slots 13-15 take B shifted by 1 (s0 = 14: [0 W(+1) W(0)]) or
                            // 2 (s0 = 15: [0 0 W(+1)]) tiles; slots 0-2 the rest, shifted
                            // the other way ([W(-1) 0 0] or [W(0) W(-1) 0])
                            const uint32_t sh = uint32_t(s0 - (NS - 3));  // 1 or 2
#pragma unroll
                            for (int dxi = 0; dxi < 3; ++dxi)
#pragma unroll
                                for (int kk = 0; kk < 2; ++kk) {
                                    if (kk >= kks) break;
                                    const uint64_t ad = arow + uint64_t(dxi + kk * kstep);
                                    const uint64_t bk = b0 + uint64_t(5 * dxi * wt16 + kk * 2);
                                    umma_bf16(tmem + d13, ad, bk - uint64_t(sh * wt16), idN, 1u);
                                    umma_bf16(tmem, ad, bk + uint64_t((3 - sh) * wt16), idN, 1u);
                                }
                        }
                    }
                    umma_commit(&empty[s]);
                }
                for (int pc = hg * g; pc < hg * g + hg && ok; ++pc)
                    if (pc >= 1 && pc <= npairs) umma_commit(&pfull[pc % NP]);
            }
            umma_commit(&drainbar);  // retire every MMA issued, also after a timeout
            mbar_drain(&drainbar, 0);
        }
    } else if (warp >= 4) {
        const int q = warp & 3;  // TMEM lanes 32q..32q+31 belong to this warp
        const int px = x0 + q * 32 + lane;
        const bool colok = px < a.w;
        const uint32_t lanes = uint32_t(q * 32) << 16;
        const float4 *sb4 = reinterpret_cast<const float4 *>(sbias);
        for (int P = 1; P <= npairs; ++P) {
            const int ps = P % NP;
            const bool got = mbar_wait_idle(&pfull[ps], uint32_t((P - 1) / NP) & 1u, &abort_flag, a.err, 25);
            uint8_t *stg = sY + size_t(a.ystages == 2 ? (P & 1) : 0) * 2 * a.stage_y_bytes;
            if (a.up2) {
                // the four warps agree before the named barriers below, so that a
                // wait that gave up can never leave a warp waiting at one of them
                if (!got) s_bad = 1;
                // the stores issued from this buffer (two pairs ago, or the last
                // pair's with one buffer) have read it
                if (warp == 4 && lane == 0) {
                    if (a.ystages == 2)
                        bulk_wait_read1();
                    else
                        bulk_wait_read0();
                }
                asm volatile("bar.sync 1, 128;" ::: "memory");
                const int bad = s_bad;
                asm volatile("bar.sync 1, 128;" ::: "memory");
                if (bad) break;
            } else if (!got) {
                break;
            }
            tc_fence_after();
            const int r0 = 2 * P - 2;  // segment row of the pair's first row
#pragma unroll 1
            for (int cg = 0; cg < COUT / 32; ++cg) {
                // 32 channels of both rows of the pair
                float v[2][32];
                tmem_ld32x2(tmem + lanes + uint32_t(2 * ps * COUT + cg * 32),
                            tmem + lanes + uint32_t((2 * ps + 1) * COUT + cg * 32), v[0], v[1]);
                uint32_t pk[2][16];
#pragma unroll
                for (int j4 = 0; j4 < 8; ++j4) {
                    const float4 b4 = sb4[cg * 8 + j4];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        float x0v = v[u][4 * j4] + b4.x, x1v = v[u][4 * j4 + 1] + b4.y;
                        float x2v = v[u][4 * j4 + 2] + b4.z, x3v = v[u][4 * j4 + 3] + b4.w;
                        if (a.relu) {
                            x0v = fmaxf(x0v, 0.0f);
                            x1v = fmaxf(x1v, 0.0f);
                            x2v = fmaxf(x2v, 0.0f);
                            x3v = fmaxf(x3v, 0.0f);
                        }
                        __nv_bfloat162 b0 = __floats2bfloat162_rn(x0v, x1v), b1 = __floats2bfloat162_rn(x2v, x3v);
                        pk[u][2 * j4] = *reinterpret_cast<uint32_t *>(&b0);
                        pk[u][2 * j4 + 1] = *reinterpret_cast<uint32_t *>(&b1);
                    }
                }
                if (a.up2) {
                    // staged row u: [128 pixels][COUT channels]
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        uint4 *dst = reinterpret_cast<uint4 *>(stg + size_t(u) * a.stage_y_bytes +
                                                               size_t(q * 32 + lane) * COUT * 2 + cg * 64);
#pragma unroll
                        for (int j4 = 0; j4 < 4; ++j4)
                            dst[j4] = make_uint4(pk[u][4 * j4], pk[u][4 * j4 + 1], pk[u][4 * j4 + 2], pk[u][4 * j4 + 3]);
                    }
                } else if (a.y && colok) {
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        if (r0 + u >= Lseg) break;
                        uint4 *dst = reinterpret_cast<uint4 *>(
                            static_cast<__nv_bfloat16 *>(a.y) + (((long long)img * a.h + ya + r0 + u) * a.w + px) * a.ys +
                            cg * 32);
#pragma unroll
                        for (int j4 = 0; j4 < 4; ++j4)
                            dst[j4] = make_uint4(pk[u][4 * j4], pk[u][4 * j4 + 1], pk[u][4 * j4 + 2], pk[u][4 * j4 + 3]);
                    }
                }
                if (a.pool_y || (COUT == 32 && a.head_y)) {
                    // the fused outputs start from the BF16-rounded values
#pragma unroll
                    for (int u = 0; u < 2; ++u)
#pragma unroll
                        for (int j = 0; j < 16; ++j) {
                            const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&pk[u][j]));
                            v[u][2 * j] = f.x;
                            v[u][2 * j + 1] = f.y;
                        }
                }
                if (COUT == 32 && a.head_y) {
                    // all (up to 4) head outputs in one pass: four independent FMA
                    // chains, each in channel order, weights read as float4
                    const float4 *sh4 = reinterpret_cast<const float4 *>(shead);
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        if (r0 + u >= Lseg) break;
                        float acc_h[4] = {0.0f, 0.0f, 0.0f, 0.0f};
#pragma unroll
                        for (int j4 = 0; j4 < 8; ++j4)
#pragma unroll
                            for (int kh = 0; kh < 4; ++kh) {
                                const float4 wv = sh4[kh * 8 + j4];
                                acc_h[kh] = fmaf(v[u][4 * j4], wv.x, acc_h[kh]);
                                acc_h[kh] = fmaf(v[u][4 * j4 + 1], wv.y, acc_h[kh]);
                                acc_h[kh] = fmaf(v[u][4 * j4 + 2], wv.z, acc_h[kh]);
                                acc_h[kh] = fmaf(v[u][4 * j4 + 3], wv.w, acc_h[kh]);
                            }
#pragma unroll
                        for (int kh = 0; kh < 4; ++kh)
                            if (kh < a.head_out && colok)
                                a.head_y[(((long long)img * a.head_out + kh) * a.h + ya + r0 + u) * a.w + px] =
                                    acc_h[kh] + shead_b[kh];
                    }
                }
                if (a.pool_y) {
                    // rows r0, r0 + 1 (ya and r0 even) and pixels px, px ^ 1 (lanes
                    // lane, lane ^ 1): the even lane pools channels 0-15 and the odd
                    // one 16-31, each receiving that half of the other pixel (16
                    // shuffles per row instead of 32); FP32 ((a + b) + (d + e)) / 4,
                    // rounded to BF16 (addition commutes: the same bits whichever
                    // lane adds)
                    const int odd = lane & 1;
                    const bool wr = colok && r0 + 1 < Lseg;
                    uint32_t pp[8];
#pragma unroll
                    for (int cj = 0; cj < 16; cj += 2) {
                        float s2[2];
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            const int c = cj + e;
                            const float mine_top = odd ? v[0][16 + c] : v[0][c];
                            const float mine_bot = odd ? v[1][16 + c] : v[1][c];
                            const float give_top = odd ? v[0][c] : v[0][16 + c];
                            const float give_bot = odd ? v[1][c] : v[1][16 + c];
                            const float nb_top = __shfl_xor_sync(0xffffffffu, give_top, 1);
                            const float nb_bot = __shfl_xor_sync(0xffffffffu, give_bot, 1);
                            s2[e] = 0.25f * ((mine_top + nb_top) + (mine_bot + nb_bot));
                        }
                        __nv_bfloat162 b2 = __floats2bfloat162_rn(s2[0], s2[1]);
                        pp[cj / 2] = *reinterpret_cast<uint32_t *>(&b2);
                    }
                    if (wr) {
                        const int pyo = (ya + r0) >> 1;
                        uint4 *dst = reinterpret_cast<uint4 *>(
                            a.pool_y + (((long long)img * (a.h >> 1) + pyo) * (a.w >> 1) + (px >> 1)) * COUT + cg * 32 +
                            odd * 16);
                        dst[0] = make_uint4(pp[0], pp[1], pp[2], pp[3]);
                        dst[1] = make_uint4(pp[4], pp[5], pp[6], pp[7]);
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&pempty[ps])) : "memory");
            if (a.up2) {
                // the staged pair -> output rows 2y, 2y + 1, even and odd columns
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                asm volatile("bar.sync 1, 128;" ::: "memory");
                if (warp == 4 && lane == 0) {
                    for (int u = 0; u < 2 && r0 + u < Lseg; ++u) {
                        const int yo = (img * a.h + ya + r0 + u) * 2;
#pragma unroll
                        for (int e = 0; e < 2; ++e) {
                            tma_store_3d(&mapY0, stg + size_t(u) * a.stage_y_bytes, 0, x0, yo + e);
                            tma_store_3d(&mapY1, stg + size_t(u) * a.stage_y_bytes, 0, x0, yo + e);
                        }
                    }
                    bulk_commit();
                }
            }
        }
        if (a.up2 && warp == 4 && lane == 0) bulk_wait_all();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
}

// ---- NHWC layout kernels (memory-bound, grid-stride) --------------------------
// One thread per pixel: coalesced reads of each input plane, cp/8 16-byte
// stores of the pixel's padded channel vector.
__global__ void k_nchw_to_nhwc(const float *__restrict__ x, int n, int c, int h, int w, uint4 *__restrict__ y,
                               int cp) {
    const long long hw = (long long)h * w, total = (long long)n * hw;
    for (long long pix = blockIdx.x * (long long)blockDim.x + threadIdx.x; pix < total;
         pix += (long long)gridDim.x * blockDim.x) {
        const long long img = pix / hw, p = pix - img * hw;
        for (int c0 = 0; c0 < cp; c0 += 8) {
            uint32_t pk[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int a = c0 + 2 * j, b = a + 1;
                const float va = a < c ? x[(img * c + a) * hw + p] : 0.0f;
                const float vb = b < c ? x[(img * c + b) * hw + p] : 0.0f;
                __nv_bfloat162 t = __floats2bfloat162_rn(va, vb);
                pk[j] = *reinterpret_cast<uint32_t *>(&t);
            }
            y[pix * (cp / 8) + c0 / 8] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
    }
}

// 3x3 patches (zero outside the image) as channels: y[pixel][ci * 9 + t] =
// x[ci][py + dy][px + dx] with t = 3 (dy + 1) + (dx + 1), the same order as
// the FP32 weights [cout][cin][3][3] flattened, so a 3x3 convolution of x is
// the 1x1 convolution of y with those weights read as [cout][9 cin]; the
// channels from 9c up to cp are zero.  One thread per output pixel.
__global__ void k_im2col3_nhwc(const float *__restrict__ x, int n, int c, int h, int w, uint4 *__restrict__ y,
                               int cp) {
    const long long hw = (long long)h * w, total = (long long)n * hw;
    for (long long pix = blockIdx.x * (long long)blockDim.x + threadIdx.x; pix < total;
         pix += (long long)gridDim.x * blockDim.x) {
        const long long img = pix / hw, p = pix - img * hw;
        const int py = int(p / w), px = int(p - (long long)py * w);
        for (int c0 = 0; c0 < cp; c0 += 8) {
            float v[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int k = c0 + j, ci = k / 9, t = k - 9 * ci;
                const int yy = py + t / 3 - 1, xx = px + t % 3 - 1;
                v[j] = (ci < c && yy >= 0 && yy < h && xx >= 0 && xx < w)
                           ? x[(img * c + ci) * hw + (long long)yy * w + xx]
                           : 0.0f;
            }
            uint32_t pk[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                __nv_bfloat162 t2 = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
                pk[j] = *reinterpret_cast<uint32_t *>(&t2);
            }
            y[pix * (cp / 8) + c0 / 8] = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
    }
}

// 2x2 average, FP32 arithmetic, two channels per thread.
__global__ void k_pool2_nhwc(const __nv_bfloat162 *__restrict__ x, int n, int c2, int h, int w,
                             __nv_bfloat162 *__restrict__ y) {
    const int ho = h / 2, wo = w / 2;
    const long long total = (long long)n * ho * wo * c2;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = int(i % c2);
        long long p = i / c2;
        const int xo = int(p % wo);
        p /= wo;
        const int yo = int(p % ho);
        const long long img = p / ho;
        const long long base = ((img * h + 2 * yo) * w + 2 * xo) * c2 + ch;
        const float2 a = __bfloat1622float2(x[base]), b = __bfloat1622float2(x[base + c2]);
        const float2 d = __bfloat1622float2(x[base + (long long)w * c2]),
                     e = __bfloat1622float2(x[base + (long long)w * c2 + c2]);
        y[i] = __floats2bfloat162_rn(0.25f * ((a.x + b.x) + (d.x + e.x)), 0.25f * ((a.y + b.y) + (d.y + e.y)));
    }
}

// Nearest 2x upsampling (h, w = input size), 16 bytes per thread.
__global__ void k_up2_nhwc(const uint4 *__restrict__ x, int n, int c8, int h, int w, uint4 *__restrict__ y) {
    const int ho = 2 * h, wo = 2 * w;
    const long long total = (long long)n * ho * wo * c8;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = int(i % c8);
        long long p = i / c8;
        const int xo = int(p % wo);
        p /= wo;
        const int yo = int(p % ho);
        const long long img = p / ho;
        y[i] = x[((img * h + yo / 2) * w + xo / 2) * c8 + ch];
    }
}

// FP32 [cout][cin][k][k] -> BF16 [k*k][cout_pad][cin_pad], zero padded.
__global__ void k_pack_w_tc(const float *__restrict__ w, int cout, int cin, int k, int cout_pad, int cin_pad,
                            __nv_bfloat16 *__restrict__ wt) {
    const long long total = (long long)k * k * cout_pad * cin_pad;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int ci = int(i % cin_pad);
        const int co = int((i / cin_pad) % cout_pad);
        const int tap = int(i / ((long long)cin_pad * cout_pad));
        float v = 0.0f;
        if (ci < cin && co < cout) v = w[((long long)co * cin + ci) * k * k + tap];
        wt[i] = __float2bfloat16_rn(v);
    }
}

// Network input of one medium (features of the warm start): channel 0
// (eps - 0.05) / 0.05, channel 1 (log10 K + 2) / 2, channel 2 the constant
// log10|G| + 6 (passed in).  FP32 arithmetic on the rounded inputs (the
// features are FP32 and feed a BF16 network; FP64 is slow on this GPU).
__global__ void k_warm_features(const double *__restrict__ eps, const double *__restrict__ K, long long np,
                                float g6, float *__restrict__ x) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < np;
         i += (long long)gridDim.x * blockDim.x) {
        x[i] = (float(eps[i]) - 0.05f) * 20.0f;
        x[np + i] = (log10f(float(K[i])) + 2.0f) * 0.5f;
        x[2 * np + i] = g6;
    }
}

// Network output -> warm-start fields: rho = 1 + y0 (G s), u = (y K) (G/nu)
// (the network predicts the density deviation over G s and the velocity over
// the local Darcy scale K G / nu), FP64, rounded in the written order with
// the two scalar factors formed once on the host.
__global__ void k_warm_decode(const float *__restrict__ y, const double *__restrict__ K, long long np, double gs,
                              double g_nu, double *__restrict__ rho, double *__restrict__ ux,
                              double *__restrict__ uy) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < np;
         i += (long long)gridDim.x * blockDim.x) {
        const double k = K[i];
        rho[i] = __dadd_rn(1.0, __dmul_rn(double(y[i]), gs));
        ux[i] = __dmul_rn(__dmul_rn(double(y[np + i]), k), g_nu);
        uy[i] = __dmul_rn(__dmul_rn(double(y[2 * np + i]), k), g_nu);
    }
}

// NHWC BF16 activations: dims (channels, w, h, n), box (32, tw, th, 1).
bool map_act(CUtensorMap *m, const void *ptr, int c, int w, int h, int n, int tw, int th) {
    const cuuint64_t dims[4] = {cuuint64_t(c), cuuint64_t(w), cuuint64_t(h), cuuint64_t(n)};
    const cuuint64_t strides[3] = {cuuint64_t(c) * 2, cuuint64_t(c) * 2 * w, cuuint64_t(c) * 2 * w * h};
    const cuuint32_t box[4] = {TC_KC, cuuint32_t(tw), cuuint32_t(th), 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(ptr), dims, strides, box, es,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// NHWC BF16 activations for the band kernel: dims (channels, w, h, n), box
// (8 channels, 130 pixels, R + 2 rows, 1), no swizzle.
bool map_act_band(CUtensorMap *m, const void *ptr, int c, int w, int h, int n, int R) {
    const cuuint64_t dims[4] = {cuuint64_t(c), cuuint64_t(w), cuuint64_t(h), cuuint64_t(n)};
    const cuuint64_t strides[3] = {cuuint64_t(c) * 2, cuuint64_t(c) * 2 * w, cuuint64_t(c) * 2 * w * h};
    const cuuint32_t box[4] = {8, cuuint32_t(BAND_PX), cuuint32_t(R + 2), 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(ptr), dims, strides, box, es,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// dynamic shared memory budget: the 227 KB opt-in limit less room for the
// kernels' static shared memory
constexpr size_t kSmemLimit = 226 * 1024;
constexpr size_t kBandMaxWeights = 80 * 1024;  // larger weight sets: tile kernel
// 32-channel K chunks of c input channels (a last partial chunk of 16: the
// loads fill its missing channels with zeros)
inline int kchunks(int c) { return (c + TC_KC - 1) / TC_KC; }

// Band kernel plan for a layer: rows per band and ring stages, or false when
// the layer does not fit it (3x3, BF16 output, rows of >= 128 pixels,
// cout <= 64, resident weights and two or more stages in shared memory).
bool band_plan(int k, int f32_nchw, int w, int cin, int cout, int h, int *R, int *stages, size_t *smem,
               int *stack) {
    if (k != 3 || f32_nchw || w < TC_M || cout > 64 || cout % 32) return false;
    const size_t wbytes = size_t(9) * kchunks(cin) * cout * TC_KC * 2;
    if (wbytes > kBandMaxWeights) return false;
    int row = 32;
    while (row < cout) row <<= 1;
    // 32 output channels: stack the three dy taps (N = 96); two buffers of
    // R + 4 row slots x 32 columns fill 512 columns at R = 4
    *stack = (cout == 32 && g_tc_variant != 3) ? 1 : 0;
    int r = *stack ? 4 : 256 / row;  // two accumulator buffers fill at most 512 columns
    if (r > 8) r = 8;
    if (r > h) r = h;
    for (; r >= 1; --r) {
        const size_t blk = (size_t(r + 2) * BAND_PX * 16 + 127) / 128 * 128;
        const size_t stage = 4 * blk;
        for (int st = 3; st >= 2; --st) {
            const size_t total = 1024 + wbytes + st * stage;
            if (total <= kSmemLimit) {
                *R = r;
                *stages = st;
                *smem = total;
                return true;
            }
        }
    }
    return false;
}

glbm_status launch_band(const void *x0, int c0, const void *x1, int c1, int n, int h, int w, const CUtensorMap &mB,
                        const float *bias, int cout, void *y, long long ys, int relu, int *err, cudaStream_t st,
                        int R, int stages, size_t smem, int stack, void *pool_y = nullptr,
                        const void *head_w = nullptr, const float *head_b = nullptr, float *head_y = nullptr,
                        int head_out = 0) {
    CUtensorMap mA0, mA1;
    if (!map_act_band(&mA0, x0, c0, w, h, n, R) ||
        !map_act_band(&mA1, c1 > 0 ? x1 : x0, c1 > 0 ? c1 : c0, w, h, n, R))
        return tcfail(GLBM_EINVAL, "nn_tc_conv: band activation tensor map rejected");
    BandArgs a;
    a.starve = take_starve();
    a.x0 = static_cast<const __nv_bfloat16 *>(x0);
    a.x1 = static_cast<const __nv_bfloat16 *>(c1 > 0 ? x1 : x0);
    a.c0 = c0;
    a.c1 = c1 > 0 ? c1 : c0;
    a.n = n;
    a.h = h;
    a.w = w;
    a.nchunk0 = kchunks(c0);
    a.nchunk = a.nchunk0 + c1 / TC_KC;
    a.cout = cout;
    a.R = R;
    a.stages = stages;
    a.nbx = (w + TC_M - 1) / TC_M;
    a.nby = (h + R - 1) / R;
    a.nbands = (long long)n * a.nby * a.nbx;
    a.blk_stride = uint32_t((size_t(R + 2) * BAND_PX * 16 + 127) / 128 * 128);
    a.stage_bytes = 4 * a.blk_stride;
    a.tx_bytes = uint32_t(4 * (R + 2) * BAND_PX * 16);
    a.wtile = uint32_t(cout * TC_KC * 2);
    a.stack = stack;
    a.pool_y = static_cast<__nv_bfloat16 *>(pool_y);
    a.head_w = static_cast<const __nv_bfloat16 *>(head_w);
    a.head_b = head_b;
    a.head_y = head_y;
    a.head_out = head_out;
    a.acc_row = 32;
    while (a.acc_row < uint32_t(cout)) a.acc_row <<= 1;
    // stacked: row slots -2 .. R + 1, exactly cout columns apart
    a.acc_cols = stack ? uint32_t(R + 4) * uint32_t(cout) : uint32_t(R) * a.acc_row;
    if (stack) a.acc_row = uint32_t(cout);
    a.tmem_cols = 32;
    while (a.tmem_cols < 2 * a.acc_cols) a.tmem_cols <<= 1;
    a.bias = bias;
    a.y = y;
    a.ys = ys;
    a.relu = relu ? 1 : 0;
    a.err = err;
    if (a.tmem_cols > 512) return tcfail(GLBM_EINVAL, "nn_tc_conv: band accumulators exceed tensor memory");
    cudaError_t e = cudaFuncSetAttribute(k_tc_conv_band, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return tccuda(e, "nn_tc_conv: shared memory attribute (band)");
    int dev = 0, nsm = 0;
    e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return tccuda(e, "nn_tc_conv: device query");
    const long long grid = a.nbands < nsm ? a.nbands : nsm;
    k_tc_conv_band<<<unsigned(grid), BAND_THREADS, smem, st>>>(mA0, mA1, mB, a);
    e = cudaGetLastError();
    return e == cudaSuccess ? GLBM_OK : tccuda(e, "nn_tc_conv launch (band)");
}

// Streaming plan for a 3x3 layer with 32 output channels: one CTA per
// (image, 128-pixel strip, segment of L output rows), at most one CTA per SM;
// false where the segments would be short (the band kernel's edge overhead
// is then no worse) or the weights and two stages do not fit.
struct StreamPlan {
    int L, nseg, G, stages;
    bool stack;          // dy taps stacked along N (weights with zero tiles)
    int ystages;         // up2: staged row pairs (2, or 1 where two do not fit)
    size_t smem;
    bool wstream;        // weights travel with each stage (too many to keep resident)
    uint32_t wofs;       // wstream: byte offset of the weight tiles in a stage
    size_t stage_bytes;
};

bool stream_plan(int w, int h, int n, int cin, int cout, int nsm, StreamPlan *p, bool up2 = false) {
    if (w < TC_M || g_tc_variant == 1 || g_tc_variant == 3 || g_tc_variant == 4) return false;
    if (cout != 32 && cout != 64) return false;
    const bool resident = size_t(9) * kchunks(cin) * TC_KC * cout * 2 <= kBandMaxWeights;
    // 32 output channels: resident weights only (the stacked tiles with
    // their zero tiles); 64: resident, or nine tiles per stage
    if (!resident && cout == 32) return false;
    // stacked tiles with their zero tiles; 64 output channels stack where
    // those fit with two stages of two rows (and with up2 two staged row
    // pairs: a single staging buffer serialises the stores with the
    // epilogue and cost more than stacking saved, d1b 116 -> 133 us), else
    // the plain tiles; weights carried in each stage stack too (17 tiles per
    // stage)
    const size_t wstack = size_t(15 * kchunks(cin) + 2) * cout * TC_KC * 2;
    const size_t stage2 = 4 * ((size_t(2) * BAND_PX * 16 + 127) / 128 * 128);
    const size_t pair_y = size_t(2) * TC_M * cout * 2;
    const int ystages = up2 ? 2 : 0;
    const bool stack = cout == 32 || !resident || 1024 + wstack + ystages * pair_y + 2 * stage2 <= 221 * 1024;
    const size_t staged = size_t(ystages) * pair_y;
    const size_t wbytes = !resident ? 0 : stack ? wstack : size_t(9) * kchunks(cin) * cout * TC_KC * 2;
    // the 227 KB per block less this kernel's ~5 KB of static shared memory
    constexpr size_t kStreamSmemLimit = 221 * 1024;
    const long long units = (long long)n * ((w + TC_M - 1) / TC_M);
    if (units > nsm) return false;
    int segs = int(nsm / units);
    int l = (h + segs - 1) / segs;
    l += l & 1;  // even: row pairs never straddle two segments
    if (l < (g_tc_variant == 5 ? 2 : 16)) return false;
    p->L = l;
    p->nseg = (h + l - 1) / l;
    p->wstream = !resident;
    p->stack = stack;
    p->ystages = ystages;
    // the tallest group that leaves three stages: 6, 4 or 2 rows with 32
    // output channels; 2 rows with 64 (the 4 pair slots need two groups of
    // slack), 4 when each stage carries the weights (amortised over 4 rows)
    const int g0 = cout == 32 ? 6 : (resident || stack ? 2 : 4);
    for (int g = g0; g >= 2; g -= 2) {
        const size_t blk = (size_t(g) * BAND_PX * 16 + 127) / 128 * 128;
        const size_t arows = resident ? 4 * blk : (4 * blk + 1023) / 1024 * 1024;
        const size_t stage = arows + (resident ? 0 : size_t(stack ? 17 : 9) * cout * TC_KC * 2);
        if (1024 + wbytes + staged + 2 * stage > kStreamSmemLimit) continue;
        const size_t room = kStreamSmemLimit - 1024 - wbytes - staged;
        int st = int(room / stage);
        if (st > ST_SMAX) st = ST_SMAX;
        if (st < (g > 2 ? 3 : 2)) continue;
        p->G = g;
        p->stages = st;
        p->wofs = uint32_t(arows);
        p->stage_bytes = stage;
        p->smem = 1024 + wbytes + staged + size_t(st) * stage;
        return true;
    }
    return false;
}

glbm_status launch_stream(const void *x0, int c0, const void *x1, int c1, int n, int h, int w, const CUtensorMap &mB,
                          const float *bias, int cout, void *y, long long ys, int relu, int *err, cudaStream_t st,
                          const StreamPlan &pl, void *pool_y = nullptr, const void *head_w = nullptr,
                          const float *head_b = nullptr, float *head_y = nullptr, int head_out = 0,
                          bool up2 = false) {
    const int L = pl.L, nseg = pl.nseg, G = pl.G, stages = pl.stages;
    const size_t smem = pl.smem;
    CUtensorMap mA0, mA1, mY0, mY1;
    if (up2) {
        // y (n, 2h, 2w, ys): output column 2j + e of full row r is element
        // (c, j, r) of map e, whose pixel stride is two pixels
        for (int e = 0; e < 2; ++e) {
            const cuuint64_t dims[3] = {cuuint64_t(cout), cuuint64_t(w), cuuint64_t(2) * h * n};
            const cuuint64_t strides[2] = {cuuint64_t(ys) * 2 * 2, cuuint64_t(ys) * 2 * 2 * w};
            const cuuint32_t box[3] = {cuuint32_t(cout), cuuint32_t(TC_M), 1};
            const cuuint32_t es[3] = {1, 1, 1};
            if (encode_fn()(e ? &mY1 : &mY0, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                            static_cast<__nv_bfloat16 *>(y) + e * ys, dims, strides, box, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
                return tcfail(GLBM_EINVAL, "nn_tc_conv_up2: output tensor map rejected");
        }
    }
    if (!map_act_band(&mA0, x0, c0, w, h, n, G - 2) ||
        !map_act_band(&mA1, c1 > 0 ? x1 : x0, c1 > 0 ? c1 : c0, w, h, n, G - 2))
        return tcfail(GLBM_EINVAL, "nn_tc_conv: streaming activation tensor map rejected");
    StreamArgs a;
    a.starve = take_starve();
    a.n = n;
    a.h = h;
    a.w = w;
    a.nchunk0 = kchunks(c0);
    a.nchunk = a.nchunk0 + c1 / TC_KC;
    // 16 input channels: two 8-channel blocks and one K step per tap
    a.nblk = c0 % TC_KC ? 2 : 4;
    a.nbx = (w + TC_M - 1) / TC_M;
    a.nseg = nseg;
    a.L = L;
    a.stages = stages;
    a.blk_stride = uint32_t((size_t(G) * BAND_PX * 16 + 127) / 128 * 128);
    a.wtile = uint32_t(cout * TC_KC * 2);
    a.wstream = pl.wstream ? 1 : 0;
    a.wofs = pl.wofs;
    a.stage_bytes = uint32_t(pl.stage_bytes);
    a.tx_bytes = uint32_t(a.nblk * G * BAND_PX * 16) + (pl.wstream ? 9 * a.wtile : 0u);
    a.bias = bias;
    a.y = y;
    a.ys = ys;
    a.relu = relu ? 1 : 0;
    a.err = err;
    a.pool_y = static_cast<__nv_bfloat16 *>(pool_y);
    a.head_w = static_cast<const __nv_bfloat16 *>(head_w);
    a.head_b = head_b;
    a.head_y = head_y;
    a.head_out = head_out;
    a.up2 = up2 ? 1 : 0;
    a.ystages = pl.ystages;
    a.stage_y_bytes = uint32_t(TC_M * cout * 2);
    if (up2) a.y = nullptr;
    if (!up2) {
        mY0 = mA0;  // unused
        mY1 = mA0;
    }
    const auto kern =
        cout == 64 ? (pl.stack ? (G == 4 ? k_tc_conv_stream<4, 64, true> : k_tc_conv_stream<2, 64, true>)
                               : (G == 4 ? k_tc_conv_stream<4, 64, false> : k_tc_conv_stream<2, 64, false>))
                   : (G == 6 ? k_tc_conv_stream<6, 32, true>
                             : (G == 4 ? k_tc_conv_stream<4, 32, true> : k_tc_conv_stream<2, 32, true>));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return tccuda(e, "nn_tc_conv: shared memory attribute (streaming)");
    const unsigned grid = unsigned((long long)n * a.nbx * nseg);
    kern<<<grid, ST_THREADS, smem, st>>>(mA0, mA1, mB, mY0, mY1, a);
    e = cudaGetLastError();
    return e == cudaSuccess ? GLBM_OK : tccuda(e, "nn_tc_conv launch (streaming)");
}

int sm_count(int *nsm) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(nsm, cudaDevAttrMultiProcessorCount, dev);
    return e == cudaSuccess ? 0 : 1;
}

}  // namespace

extern "C" void glbm_nn_tc_debug_starve(int stage) { g_tc_starve = stage > 0 ? stage : 0; }

extern "C" void glbm_nn_tc_set_variant(int variant) { g_tc_variant = (variant >= 0 && variant <= 5) ? variant : 0; }

extern "C" glbm_status glbm_nn_tc_conv(const void *x0, int c0, const void *x1, int c1, int n, int h, int w, int k,
                                       const void *wt, const float *bias, int cout, void *y, long long ys, int relu,
                                       int f32_nchw, int cout_store, int *err, void *stream) {
    if (!x0 || !wt || !bias || !y || !err || (c1 > 0 && !x1))
        return tcfail(GLBM_EINVAL, "nn_tc_conv: x0, wt, bias, y, err (and x1 when c1 > 0) are required");
    if (n < 1 || h < 1 || w < 1 || (k != 1 && k != 3))
        return tcfail(GLBM_EINVAL, "nn_tc_conv: need n, h, w >= 1 and k = 1 or 3");
    if (c0 < 16 || c0 % 16 || c1 < 0 || c1 % TC_KC || (c0 % TC_KC && c1))
        return tcfail(GLBM_EINVAL, "nn_tc_conv: input channel counts must be multiples of 32 (c0 may be 16, "
                                   "or any multiple of 16 when c1 = 0)");
    if (cout < 16 || cout > 256 || cout % 16)
        return tcfail(GLBM_EINVAL, "nn_tc_conv: cout must be a multiple of 16 in [16, 256]");
    if (f32_nchw ? (cout_store < 1 || cout_store > cout) : (ys < cout || ys % 8))
        return tcfail(GLBM_EINVAL, "nn_tc_conv: need 1 <= cout_store <= cout (FP32 NCHW output) or a pixel "
                                   "stride ys >= cout, multiple of 8 (BF16 NHWC output)");
    const uintptr_t mis = (uintptr_t(x0) | uintptr_t(x1) | uintptr_t(wt) | uintptr_t(y)) & 15u;
    if (mis) return tcfail(GLBM_EINVAL, "nn_tc_conv: arrays must be 16-byte aligned");
    if (!encode_fn()) return tcfail(GLBM_ECUDA, "nn_tc_conv: cuTensorMapEncodeTiled is not available");
    const int tw = w < TC_M ? w : TC_M;
    const int th = TC_M / tw;
    // two tiles per CTA for narrow outputs (cout <= 64): shared weight slices,
    // more tiles in flight per SM where the layer is latency-bound
    const int mt = cout <= 64 ? 2 : 1;
    const long long gy = (h + th * mt - 1) / (th * mt);
    if (gy > 65535 || n > 65535) return tcfail(GLBM_EINVAL, "nn_tc_conv: image too tall or batch too large");

    CUtensorMap mA0, mA1, mB;
    if (!map_act(&mA0, x0, c0, w, h, n, tw, th) || !map_act(&mA1, c1 > 0 ? x1 : x0, c1 > 0 ? c1 : c0, w, h, n, tw, th))
        return tcfail(GLBM_EINVAL, "nn_tc_conv: activation tensor map rejected");
    const int cin = c0 + c1, taps = k * k;
    {
        const cuuint64_t dims[3] = {cuuint64_t(cin), cuuint64_t(cout), cuuint64_t(taps)};
        const cuuint64_t strides[2] = {cuuint64_t(cin) * 2, cuuint64_t(cin) * 2 * cout};
        const cuuint32_t box[3] = {TC_KC, cuuint32_t(cout), 1};
        const cuuint32_t es[3] = {1, 1, 1};
        if (encode_fn()(&mB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(wt), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return tcfail(GLBM_EINVAL, "nn_tc_conv: weight tensor map rejected");
    }
    int nsm = 0;
    if (sm_count(&nsm)) return tcfail(GLBM_ECUDA, "nn_tc_conv: device query failed");
    int R = 0, stages = 0;
    size_t bsmem = 0;
    int stack = 0;
    StreamPlan pl;
    if (k == 3 && !f32_nchw && stream_plan(w, h, n, cin, cout, nsm, &pl))
        return launch_stream(x0, c0, x1, c1, n, h, w, mB, bias, cout, y, ys, relu, err,
                             static_cast<cudaStream_t>(stream), pl);
    if (g_tc_variant != 1 && band_plan(k, f32_nchw, w, cin, cout, h, &R, &stages, &bsmem, &stack))
        return launch_band(x0, c0, x1, c1, n, h, w, mB, bias, cout, y, ys, relu, err,
                           static_cast<cudaStream_t>(stream), R, stages, bsmem, stack);
    TcConvArgs a;
    a.starve = take_starve();
    a.n = n;
    a.h = h;
    a.w = w;
    a.taps = taps;
    a.nchunk0 = kchunks(c0);
    a.nchunk = a.nchunk0 + c1 / TC_KC;
    a.cout = cout;
    a.tw = tw;
    a.th = th;
    a.acc_cols = 32;
    while (a.acc_cols < uint32_t(cout)) a.acc_cols <<= 1;
    a.tmem_cols = a.acc_cols * uint32_t(mt);
    a.bias = bias;
    a.y = y;
    a.ys = ys;
    a.relu = relu ? 1 : 0;
    a.f32_nchw = f32_nchw ? 1 : 0;
    a.cout_store = f32_nchw ? cout_store : cout;
    a.err = err;
    const dim3 grid(unsigned((w + tw - 1) / tw), unsigned(gy), unsigned(n));
    // a grid of at most one CTA per SM cannot hide latency behind other
    // CTAs: it keeps more loads in flight with a deep ring instead
    const bool deep = g_tc_variant != 2 && (long long)grid.x * grid.y * grid.z <= nsm;
    const int ring = deep ? TC_STAGES_DEEP : TC_STAGES;
    const size_t smem = 1024 + size_t(ring) * (size_t(mt) * TC_STAGE_A + size_t(cout) * TC_KC * 2);
    const auto kern = mt == 2 ? (deep ? k_tc_conv<2, TC_STAGES_DEEP> : k_tc_conv<2, TC_STAGES>)
                              : (deep ? k_tc_conv<1, TC_STAGES_DEEP> : k_tc_conv<1, TC_STAGES>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return tccuda(e, "nn_tc_conv: shared memory attribute");
    kern<<<grid, TC_THREADS, smem, static_cast<cudaStream_t>(stream)>>>(mA0, mA1, mB, a);
    e = cudaGetLastError();
    return e == cudaSuccess ? GLBM_OK : tccuda(e, "nn_tc_conv launch");
}

extern "C" glbm_status glbm_nn_tc_conv_fused(const void *x0, int c0, const void *x1, int c1, int n, int h, int w,
                                             const void *wt, const float *bias, int cout, void *y, long long ys,
                                             int relu, void *pool_y, const void *head_w, const float *head_b,
                                             int head_out, float *head_y, int *err, void *stream) {
    if (!x0 || !wt || !bias || !err || (c1 > 0 && !x1) || (!y && !pool_y && !head_y))
        return tcfail(GLBM_EINVAL, "nn_tc_conv_fused: x0, wt, bias, err and at least one output are required");
    if (n < 1 || h < 1 || w < 1 || c0 < 16 || c0 % 16 || c1 < 0 || c1 % TC_KC || (c0 % TC_KC && c1) ||
        (cout != 32 && cout != 64))
        return tcfail(GLBM_EINVAL,
                      "nn_tc_conv_fused: needs 32 or 64 output channels and input channels in multiples of 32 "
                      "(c0 may be a multiple of 16 when c1 = 0)");
    if (cout != 32 && head_y) return tcfail(GLBM_EINVAL, "nn_tc_conv_fused: the fused head needs 32 output channels");
    if (y && (ys < cout || ys % 8)) return tcfail(GLBM_EINVAL, "nn_tc_conv_fused: bad output pixel stride");
    if (pool_y && (h % 2 || w % 2)) return tcfail(GLBM_EINVAL, "nn_tc_conv_fused: pooling needs even h and w");
    if (head_y && (!head_w || !head_b || head_out < 1 || head_out > 4))
        return tcfail(GLBM_EINVAL, "nn_tc_conv_fused: the head needs weights, bias and 1..4 outputs");
    const uintptr_t mis = (uintptr_t(x0) | uintptr_t(x1) | uintptr_t(wt) | uintptr_t(y) | uintptr_t(pool_y)) & 15u;
    if (mis) return tcfail(GLBM_EINVAL, "nn_tc_conv_fused: arrays must be 16-byte aligned");
    if (!encode_fn()) return tcfail(GLBM_ECUDA, "nn_tc_conv_fused: cuTensorMapEncodeTiled is not available");
    const int cin = c0 + c1;
    int R = 0, stages = 0, stack = 0, nsm = 0;
    size_t smem = 0;
    if (sm_count(&nsm)) return tcfail(GLBM_ECUDA, "nn_tc_conv_fused: device query failed");
    StreamPlan pl;
    const bool streaming = stream_plan(w, h, n, cin, cout, nsm, &pl);
    if (!streaming && (!band_plan(3, 0, w, cin, cout, h, &R, &stages, &smem, &stack) || (cout == 32 && !stack)))
        return tcfail(GLBM_EINVAL, "nn_tc_conv_fused: the layer does not fit the band kernel");
    if (!streaming && pool_y && R % 2) --R;  // pooling pairs the rows of a band (fewer rows need less memory)
    if (!streaming && R < 2 && pool_y)
        return tcfail(GLBM_EINVAL, "nn_tc_conv_fused: pooling needs bands of two rows or more");
    CUtensorMap mB;
    {
        const cuuint64_t dims[3] = {cuuint64_t(cin), cuuint64_t(cout), 9};
        const cuuint64_t strides[2] = {cuuint64_t(cin) * 2, cuuint64_t(cin) * 2 * cout};
        const cuuint32_t box[3] = {TC_KC, cuuint32_t(cout), 1};
        const cuuint32_t es[3] = {1, 1, 1};
        if (encode_fn()(&mB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(wt), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return tcfail(GLBM_EINVAL, "nn_tc_conv_fused: weight tensor map rejected");
    }
    if (streaming)
        return launch_stream(x0, c0, x1, c1, n, h, w, mB, bias, cout, y, ys, relu, err,
                             static_cast<cudaStream_t>(stream), pl, pool_y, head_w, head_b, head_y, head_out);
    return launch_band(x0, c0, x1, c1, n, h, w, mB, bias, cout, y, ys, relu, err, static_cast<cudaStream_t>(stream),
                       R, stages, smem, stack, pool_y, head_w, head_b, head_y, head_out);
}

extern "C" glbm_status glbm_nn_tc_conv_up2(const void *x0, int c0, const void *x1, int c1, int n, int h, int w,
                                           const void *wt, const float *bias, int cout, void *y, long long ys,
                                           int relu, int *err, void *stream) {
    if (!x0 || !wt || !bias || !y || !err || (c1 > 0 && !x1))
        return tcfail(GLBM_EINVAL, "nn_tc_conv_up2: x0, wt, bias, y, err (and x1 when c1 > 0) are required");
    if (n < 1 || h < 1 || w < 1 || c0 < 16 || c0 % 16 || c1 < 0 || c1 % TC_KC || (c0 % TC_KC && c1) ||
        (cout != 32 && cout != 64) || ys < cout || ys % 8)
        return tcfail(GLBM_EINVAL, "nn_tc_conv_up2: needs 32 or 64 output channels, input channels as in "
                                   "glbm_nn_tc_conv and a pixel stride ys >= cout, a multiple of 8");
    const uintptr_t mis = (uintptr_t(x0) | uintptr_t(x1) | uintptr_t(wt) | uintptr_t(y)) & 15u;
    if (mis) return tcfail(GLBM_EINVAL, "nn_tc_conv_up2: arrays must be 16-byte aligned");
    if (!encode_fn()) return tcfail(GLBM_ECUDA, "nn_tc_conv_up2: cuTensorMapEncodeTiled is not available");
    const int cin = c0 + c1;
    int nsm = 0;
    if (sm_count(&nsm)) return tcfail(GLBM_ECUDA, "nn_tc_conv_up2: device query failed");
    StreamPlan pl;
    if (!stream_plan(w, h, n, cin, cout, nsm, &pl, true))
        return tcfail(GLBM_EINVAL, "nn_tc_conv_up2: the layer does not fit the streaming kernel");
    CUtensorMap mB;
    {
        const cuuint64_t dims[3] = {cuuint64_t(cin), cuuint64_t(cout), 9};
        const cuuint64_t strides[2] = {cuuint64_t(cin) * 2, cuuint64_t(cin) * 2 * cout};
        const cuuint32_t box[3] = {TC_KC, cuuint32_t(cout), 1};
        const cuuint32_t es[3] = {1, 1, 1};
        if (encode_fn()(&mB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(wt), dims, strides, box, es,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return tcfail(GLBM_EINVAL, "nn_tc_conv_up2: weight tensor map rejected");
    }
    return launch_stream(x0, c0, x1, c1, n, h, w, mB, bias, cout, y, ys, relu, err, static_cast<cudaStream_t>(stream),
                         pl, nullptr, nullptr, nullptr, nullptr, 0, true);
}

extern "C" glbm_status glbm_nn_tc_pack_weights(const float *wf, int cout, int cin, int k, int cout_pad,
                                               int cin_pad, void *wt, void *stream) {
    if (!wf || !wt || cout < 1 || cin < 1 || (k != 1 && k != 3) || cout_pad < cout || cin_pad < cin)
        return tcfail(GLBM_EINVAL, "nn_tc_pack_weights: invalid sizes or pointers");
    const long long total = (long long)k * k * cout_pad * cin_pad;
    k_pack_w_tc<<<grid_for(total), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        wf, cout, cin, k, cout_pad, cin_pad, static_cast<__nv_bfloat16 *>(wt));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GLBM_OK : tccuda(e, "nn_tc_pack_weights launch");
}

extern "C" glbm_status glbm_nn_nchw_to_nhwc(const float *x, int n, int c, int h, int w, void *y, int c_pad,
                                            void *stream) {
    if (!x || !y || n < 1 || c < 1 || h < 1 || w < 1 || c_pad < c || c_pad % 8 || (uintptr_t(y) & 15u))
        return tcfail(GLBM_EINVAL, "nn_nchw_to_nhwc: need c_pad >= c, a multiple of 8, and 16-byte aligned y");
    const long long total = (long long)n * h * w;
    k_nchw_to_nhwc<<<grid_for(total), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, n, c, h, w,
                                                                                   static_cast<uint4 *>(y), c_pad);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GLBM_OK : tccuda(e, "nn_nchw_to_nhwc launch");
}

extern "C" glbm_status glbm_nn_im2col3_nhwc(const float *x, int n, int c, int h, int w, void *y, int c_pad,
                                            void *stream) {
    if (!x || !y || n < 1 || c < 1 || h < 1 || w < 1 || c_pad < 9 * c || c_pad % 8 || (uintptr_t(y) & 15u))
        return tcfail(GLBM_EINVAL, "nn_im2col3_nhwc: need c_pad >= 9 c, a multiple of 8, and 16-byte aligned y");
    const long long total = (long long)n * h * w;
    k_im2col3_nhwc<<<grid_for(total), 256, 0, static_cast<cudaStream_t>(stream)>>>(x, n, c, h, w,
                                                                                   static_cast<uint4 *>(y), c_pad);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GLBM_OK : tccuda(e, "nn_im2col3_nhwc launch");
}

extern "C" glbm_status glbm_nn_pool2_nhwc(const void *x, int n, int c, int h, int w, void *y, void *stream) {
    if (!x || !y || n < 1 || c < 2 || c % 2 || h < 2 || w < 2 || h % 2 || w % 2 ||
        ((uintptr_t(x) | uintptr_t(y)) & 3u))
        return tcfail(GLBM_EINVAL, "nn_pool2_nhwc: need even c, h, w and 4-byte aligned arrays");
    const long long total = (long long)n * (h / 2) * (w / 2) * (c / 2);
    k_pool2_nhwc<<<grid_for(total), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const __nv_bfloat162 *>(x), n, c / 2, h, w, static_cast<__nv_bfloat162 *>(y));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GLBM_OK : tccuda(e, "nn_pool2_nhwc launch");
}

extern "C" glbm_status glbm_nn_upsample2_nhwc(const void *x, int n, int c, int h, int w, void *y, void *stream) {
    if (!x || !y || n < 1 || c < 8 || c % 8 || h < 1 || w < 1 || ((uintptr_t(x) | uintptr_t(y)) & 15u))
        return tcfail(GLBM_EINVAL, "nn_upsample2_nhwc: need c a multiple of 8 and 16-byte aligned arrays");
    const long long total = (long long)n * (2 * h) * (2 * w) * (c / 8);
    k_up2_nhwc<<<grid_for(total), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        static_cast<const uint4 *>(x), n, c / 8, h, w, static_cast<uint4 *>(y));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GLBM_OK : tccuda(e, "nn_upsample2_nhwc launch");
}

extern "C" glbm_status glbm_nn_warm_features(const double *eps, const double *K, long long npix, double G, float *x,
                                             void *stream) {
    if (!eps || !K || !x || npix < 1 || !(G != 0.0) || !std::isfinite(G))
        return tcfail(GLBM_EINVAL, "nn_warm_features: need eps, K, x, npix >= 1 and finite G != 0");
    k_warm_features<<<grid_for(npix), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        eps, K, npix, float(log10(fabs(G)) + 6.0), x);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GLBM_OK : tccuda(e, "nn_warm_features launch");
}

extern "C" glbm_status glbm_nn_warm_decode(const float *y, const double *K, long long npix, double G, double nu,
                                           double rho_scale, double *rho, double *ux, double *uy, void *stream) {
    if (!y || !K || !rho || !ux || !uy || npix < 1 || !(nu > 0.0))
        return tcfail(GLBM_EINVAL, "nn_warm_decode: need y, K, rho, ux, uy, npix >= 1 and nu > 0");
    k_warm_decode<<<grid_for(npix), 256, 0, static_cast<cudaStream_t>(stream)>>>(y, K, npix, G * rho_scale,
                                                                                  G / nu, rho, ux, uy);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GLBM_OK : tccuda(e, "nn_warm_decode launch");
}
