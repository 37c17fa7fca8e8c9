// Tensor-core (tcgen05, sm_103a) training kernels of the warm-start network:
// the convolution weight gradient, the flipped/transposed weight packing
// that turns the input gradient into a forward convolution on the tensor
// cores (nn_tc.cu), and the bias gradient.  The paper has no surrogate; the
// network is this library's own addition (see nn.cu for its FP32 kernels).
//
// Weight gradient of a k x k convolution (zero padding k/2):
//     dW[o][c][tap] = sum over images and pixels p of dy[p][o] * x[p + s(tap)][c]
// with s(tap) = (ky - k/2, kx - k/2).  As a GEMM:
//     D[m][o] = sum_p A[m][p] * B[o][p],   m = (tap, c), o = output channel,
// where row m of A is channel c of the input shifted by s(tap).  Both
// operands come straight from the BF16 NHWC activations: a TMA box of 32
// channels x 32 pixels of one row lands as 32 rows of 64 bytes (64-byte
// swizzle), i.e. 32 consecutive channels per pixel -- an MN-major operand
// whose 64-byte atoms (32 channels x 8 pixels) are 512 B apart along K
// (pixels, SBO) and one box (2 KB) apart along M or N (LBO).  M = 128 rows =
// four (tap, 32-channel chunk) boxes, each loaded at its own shift (TMA's
// zero fill outside the image is the padding); N = the output channels (a
// multiple of 32, one box per 32).  FP32 accumulation in TMEM.
//
// Each CTA takes one M tile and a contiguous range of image rows (split-K);
// its partial sums are added to dW with FP32 atomics (so the summation order,
// and the last bits of dW, vary from run to run).  Roles: warp 0 issues TMA,
// warp 1 issues the MMAs and commits, warps 2-5 read the accumulator; every
// wait is bounded as in nn_tc.cu.
//
// That per-tap form (k_tc_wgrad) serves 1x1 layers and variant 1.  3x3
// layers run in the band form (k_tc_wgrad_band, below), which puts the taps
// into the MMA's M and N instead: three consecutive input rows along M, three
// one-pixel shifts of a dy row along N, all nine taps in one MMA, each input
// and dy row loaded once per band.

#include "tc_common.cuh"

#include <algorithm>

namespace {

constexpr int WG_KP = 32;        // pixels per K step (one box row of 32 pixels)
constexpr int WG_STAGES = 4;
constexpr int WG_THREADS = 192;
constexpr int WG_BOX = WG_KP * 64;  // bytes of one 32-channel x 32-pixel box

struct WgradArgs {
    int starve;                  // test hook: stage number + 1 the first CTA leaves unloaded
    int n, h, w, k, nchunk, nf;  // nf = k*k*nchunk (tap, chunk) boxes
    int cin, cout, cy;           // real input / output channels, dy channels (multiple of 32)
    int rows_per_cta;            // split-K: image rows (over n*h) per CTA
    int xsteps;                  // 32-pixel steps per row
    uint32_t stage_bytes, tx_a, tmem_cols;
    float *dw;
    int *err;
};

// MN-major operand with 64-byte swizzle: atoms of 32 elements x 8 rows,
// `lbo` bytes apart along M/N, 8-row groups `sbo` bytes apart along K.
__device__ __forceinline__ uint64_t sdesc_mn64(const void *tile, uint32_t lbo, uint32_t sbo) {
    const uint64_t a = smem_u32(tile);
    return ((a >> 4) & 0x3FFFull) | (uint64_t((lbo >> 4) & 0x3FFFu) << 16) | (uint64_t((sbo >> 4) & 0x3FFFu) << 32) |
           (1ull << 46) | (4ull << 61);
}
// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both
// MN-major (bits 15, 16), N/8 in bits 17-22, M/16 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16_mn(int m, int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | (uint32_t(n >> 3) << 17) |
           (uint32_t(m >> 4) << 24);
}

__global__ void __launch_bounds__(WG_THREADS, 1)
k_tc_wgrad(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapDY, const WgradArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[WG_STAGES], empty[WG_STAGES], done;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int mtile = blockIdx.x;
    const long long row0 = (long long)blockIdx.y * a.rows_per_cta;
    long long row1 = row0 + a.rows_per_cta;
    if (row1 > (long long)a.n * a.h) row1 = (long long)a.n * a.h;
    const int iters = row1 > row0 ? int((row1 - row0) * a.xsteps) : 0;
    const int nb = a.cy / 32;  // dy boxes (N atoms)

    if (threadIdx.x == 0) {
        for (int s = 0; s < WG_STAGES; ++s) {
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
            int i = 0;
            for (; i < iters; ++i) {
                const int s = i % WG_STAGES, use = i / WG_STAGES;
                if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1, &abort_flag, a.err, 21)) break;
                const long long row = row0 + i / a.xsteps;
                const int img = int(row / a.h), y = int(row % a.h);
                const int x0 = (i % a.xsteps) * WG_KP;
                uint8_t *st = smem + size_t(s) * a.stage_bytes;
                int nload = 0;
                for (int j = 0; j < 4; ++j) nload += (mtile * 4 + j < a.nf) ? 1 : 0;
                mbar_expect_tx(&full[s], uint32_t(nload + nb) * WG_BOX);
                if (a.starve == i + 1 && blockIdx.x + blockIdx.y == 0) continue;
                for (int j = 0; j < 4; ++j) {
                    const int f = mtile * 4 + j;
                    if (f >= a.nf) break;
                    const int tap = f / a.nchunk, ch = f - tap * a.nchunk;
                    const int dy = a.k == 3 ? tap / 3 - 1 : 0, dx = a.k == 3 ? tap % 3 - 1 : 0;
                    tma_load_4d(st + j * WG_BOX, &mapX, &full[s], ch * 32, x0 + dx, y + dy, img);
                }
                for (int b = 0; b < nb; ++b) tma_load_4d(st + (4 + b) * WG_BOX, &mapDY, &full[s], b * 32, x0, y, img);
            }
            drain_ring(full, WG_STAGES, i);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_mn(128, a.cy);
            for (int i = 0; i < iters; ++i) {
                const int s = i % WG_STAGES, use = i / WG_STAGES;
                if (!mbar_wait(&full[s], use & 1, &abort_flag, a.err, 22)) break;
                tc_fence_after();
                uint8_t *st = smem + size_t(s) * a.stage_bytes;
#pragma unroll
                for (int kk = 0; kk < WG_KP / 16; ++kk) {  // K = 16 pixels per MMA: two 8-pixel groups
                    const uint64_t ad = sdesc_mn64(st + kk * 1024, WG_BOX, 512);
                    const uint64_t bd = sdesc_mn64(st + 4 * WG_BOX + kk * 1024, WG_BOX, 512);
                    umma_bf16(tmem, ad, bd, idesc, (i > 0 || kk > 0) ? 1u : 0u);
                }
                umma_commit(&empty[s]);
            }
            umma_commit(&done);  // after a timeout too: the wait below retires every MMA issued
            mbar_drain(&done, 0);
        }
    } else if (iters > 0) {
        const int q = warp & 3;  // TMEM lanes 32q..: box q of this M tile
        const int f = mtile * 4 + q;
        // after a timeout the MMA warp still commits `done` (to retire its MMAs):
        // the accumulator is then not a result
        const bool have = mbar_wait(&done, 0, &abort_flag, a.err, 23) && !abort_flag;
        tc_fence_after();
        const int tap = f / a.nchunk, ch = f - tap * a.nchunk;
        const int c = ch * 32 + lane;
        const bool ok = have && f < a.nf && c < a.cin;
        const int kk2 = a.k * a.k;
        for (int o = 0; o < a.cy && have; o += 16) {
            float v[16];
            tmem_ld16(tmem + uint32_t(o) + (uint32_t(q * 32) << 16), v);
            if (!ok) continue;
#pragma unroll
            for (int j = 0; j < 16; ++j)
                if (o + j < a.cout) atomicAdd(&a.dw[((long long)(o + j) * a.cin + c) * kk2 + tap], v[j]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, a.tmem_cols);
    }
}

// 3x3 weight gradient with every tap in one MMA ("band form").  For the
// output-gradient row y and pixels x0 .. x0 + kp - 1 of one image,
//     D[(r, c)][(j, o)] += sum_k x[y + r - 1][x0 + k][c] * dy[y][x0 + k - 1 + j][o]
// is the (ky, kx) = (r, 2 - j) tap of dW for r, j in {0, 1, 2}: the pixel
// p = (y, x0 + k - 1 + j) of dy meets x at p + (r - 1, 1 - j).  Summed over
// every x0 and y this counts each product of the tap exactly once (outside
// the image TMA's zero fill supplies the padding on either side).
//   A: rows y - 1, y, y + 1 of one 32-channel chunk of x, consecutive row
//      boxes of a band (M = 128: the fourth 32-row atom reads the next row,
//      and its TMEM lanes are never read);
//   B: one dy row box of kp + 2 pixels (x0 - 1 ..), read as three atoms 64 B
//      (one pixel) apart -- N = 96 per 32-channel output chunk.  Each pixel
//      is a 64-byte row of the 64-byte-swizzled box, so a pixel shift is a
//      shift of whole swizzle rows, and the swizzle is a function of the
//      address the MMA computes.
// A work unit is a band of R dy rows (and the R + 2 x rows they meet) of
// one kp-pixel strip of one image, loaded once per stage.  Each CTA owns a
// group of input and output chunks and a contiguous range of units.
constexpr int WB_MAX_STAGES = 4;

struct WgradBandArgs {
    int starve;                    // test hook, as in WgradArgs
    int n, h, w;
    int nchunk, nobt;              // 32-channel chunks of x and of dy
    int nxc, nob, ngx;             // chunks per CTA (x, dy); x groups (grid.x = ngx * dy groups)
    int cin, cout;
    int kp, R, xsteps, ybands;     // kp pixels per strip, R dy rows per band
    long long units;               // n * ybands * xsteps
    int units_per_cta, stages;
    uint32_t xrow, dyrow;          // bytes of an x row box (kp pixels) and of a dy row slot (kp + 2 pixels, 512-aligned)
    uint32_t dy_off, stage_bytes, tmem_cols;
    int vec;                       // cin % 4 == 0 and dw 16-byte aligned: vector reductions
    float *dw;
    int *err;
};

__global__ void __launch_bounds__(WG_THREADS, 2)
k_tc_wgrad_band(const __grid_constant__ CUtensorMap mapX, const __grid_constant__ CUtensorMap mapDY,
                const WgradBandArgs a) {
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    __shared__ __align__(8) uint64_t full[WB_MAX_STAGES], empty[WB_MAX_STAGES], done;
    __shared__ uint32_t tmem_base;
    __shared__ volatile int abort_flag;
    __shared__ volatile int s_bad;  // the epilogue warps' joint verdict on the accumulator
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int xg = blockIdx.x % a.ngx, og = blockIdx.x / a.ngx;
    const int cx0 = xg * a.nxc, co0 = og * a.nob;
    const int nx = min(a.nxc, a.nchunk - cx0), no = min(a.nob, a.nobt - co0);
    const long long u0 = (long long)blockIdx.y * a.units_per_cta;
    long long u1 = u0 + a.units_per_cta;
    if (u1 > a.units) u1 = a.units;
    const int iters = u1 > u0 ? int(u1 - u0) : 0;
    const int S = a.stages;
    const uint32_t xblk = uint32_t(a.R + 2) * a.xrow, dyblk = uint32_t(a.R) * a.dyrow;

    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        abort_flag = 0;
        s_bad = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) tmem_alloc(&tmem_base, a.tmem_cols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            int i = 0;
            for (; i < iters; ++i) {
                const int s = i % S, use = i / S;
                if (use > 0 && !mbar_wait(&empty[s], (use - 1) & 1, &abort_flag, a.err, 21)) break;
                const long long u = u0 + i;
                const int x0 = int(u % a.xsteps) * a.kp;
                const long long band = u / a.xsteps;
                const int img = int(band / a.ybands), yb = int(band % a.ybands) * a.R;
                uint8_t *st = smem + size_t(s) * a.stage_bytes;
                mbar_expect_tx(&full[s], uint32_t(nx) * uint32_t(a.R + 2) * uint32_t(a.kp * 64) +
                                             uint32_t(no) * uint32_t(a.R) * uint32_t((a.kp + 2) * 64));
                if (a.starve == i + 1 && blockIdx.x + blockIdx.y == 0) continue;
                for (int xi = 0; xi < nx; ++xi)
                    for (int t = 0; t < a.R + 2; ++t)
                        tma_load_4d(st + xi * xblk + t * a.xrow, &mapX, &full[s], (cx0 + xi) * 32, x0, yb - 1 + t, img);
                for (int ob = 0; ob < no; ++ob)
                    for (int t = 0; t < a.R; ++t)
                        tma_load_4d(st + a.dy_off + ob * dyblk + t * a.dyrow, &mapDY, &full[s], (co0 + ob) * 32, x0 - 1,
                                    yb + t, img);
            }
            drain_ring(full, S, i);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_mn(128, 96);
            for (int i = 0; i < iters; ++i) {
                const int s = i % S, use = i / S;
                if (!mbar_wait(&full[s], use & 1, &abort_flag, a.err, 22)) break;
                tc_fence_after();
                uint8_t *st = smem + size_t(s) * a.stage_bytes;
                for (int t = 0; t < a.R; ++t)
                    for (int kk = 0; kk < a.kp / 16; ++kk)  // K = 16 pixels per MMA
                        for (int ob = 0; ob < no; ++ob) {
                            const uint64_t bd = sdesc_mn64(st + a.dy_off + ob * dyblk + t * a.dyrow + kk * 1024, 64, 512);
                            for (int xi = 0; xi < nx; ++xi) {
                                const uint64_t ad = sdesc_mn64(st + xi * xblk + t * a.xrow + kk * 1024, a.xrow, 512);
                                umma_bf16(tmem + uint32_t(xi * a.nob + ob) * 96u, ad, bd, idesc,
                                          (i > 0 || t > 0 || kk > 0) ? 1u : 0u);
                            }
                        }
                umma_commit(&empty[s]);
            }
            umma_commit(&done);  // after a timeout too: the wait below retires every MMA issued
            mbar_drain(&done, 0);
        }
    } else if (iters > 0) {
        // warps 2-5 (TMEM lanes 32r..: x row y + r - 1, i.e. ky = r; r = 3 holds no
        // tap).  Per (x chunk, dy chunk) the three tap rows are gathered in the
        // idle stage memory as [o][c][tap] -- 32 contiguous runs of up to 288
        // floats of dW -- and added with 16-byte reductions.
        const int r = warp & 3;
        const bool have = mbar_wait_idle(&done, 0, &abort_flag, a.err, 23) && !abort_flag;
        if (!have && lane == 0) s_bad = 1;
        tc_fence_after();
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (!s_bad) {
            float *T = reinterpret_cast<float *>(smem);
            const int et = threadIdx.x - 64;
            for (int xi = 0; xi < nx; ++xi) {
                const int c0 = (cx0 + xi) * 32, len = min(32, a.cin - c0) * 9;
                for (int ob = 0; ob < no; ++ob) {
                    if (r < 3) {
                        for (int col = 0; col < 96; col += 16) {
                            float v[16];
                            tmem_ld16(tmem + uint32_t(xi * a.nob + ob) * 96u + uint32_t(col) + (uint32_t(r * 32) << 16), v);
                            const int tap = 3 * r + 2 - col / 32, o0 = col % 32;
#pragma unroll
                            for (int q = 0; q < 16; ++q) T[((o0 + q) * 32 + lane) * 9 + tap] = v[q];
                        }
                    }
                    asm volatile("bar.sync 1, 128;" ::: "memory");
                    const int obase = (co0 + ob) * 32, nov = min(32, a.cout - obase);
                    float *dst = a.dw + ((long long)obase * a.cin + c0) * 9;
                    const long long ostride = (long long)a.cin * 9;
                    if (a.vec) {  // cin % 4 == 0 and dw 16-byte aligned: every run starts on 16 bytes
                        const int nq = len / 4;
                        for (int idx = et; idx < nov * nq; idx += 128) {
                            const int o = idx / nq, qd = idx - o * nq;
                            const float4 s4 = *reinterpret_cast<const float4 *>(T + o * 288 + qd * 4);
                            asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(
                                             dst + o * ostride + qd * 4),
                                         "f"(s4.x), "f"(s4.y), "f"(s4.z), "f"(s4.w)
                                         : "memory");
                        }
                    } else {
                        for (int idx = et; idx < nov * len; idx += 128) {
                            const int o = idx / len, i = idx - o * len;
                            atomicAdd(dst + o * ostride + i, T[o * 288 + i]);
                        }
                    }
                    asm volatile("bar.sync 1, 128;" ::: "memory");
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

// Weights of the input-gradient convolution: the forward weights flipped in
// space and with input and output channels swapped,
// wt[tap][c (cin_pad)][o (cout_pad)] = W[o][c][k*k - 1 - tap], BF16, zero padded.
__global__ void k_pack_w_flip(const float *__restrict__ w, int cout, int cin, int k, int c_begin, int c_pad,
                              int cout_pad, __nv_bfloat16 *__restrict__ wt) {
    const long long total = (long long)k * k * c_pad * cout_pad;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int o = int(i % cout_pad);
        const int c = c_begin + int((i / cout_pad) % c_pad);
        const int tap = int(i / ((long long)cout_pad * c_pad));
        float v = 0.0f;
        if (o < cout && c < cin) v = w[((long long)o * cin + c) * k * k + (k * k - 1 - tap)];
        wt[i] = __float2bfloat16_rn(v);
    }
}

// db[c] += sum over images and pixels of dy (FP32 NCHW, sample stride dybs):
// block (c, part) sums a slice of each of channel c's planes in FP32 (float4
// loads where the plane allows them), the block's warps reduce by shuffles,
// then one atomic per block.  FP32 throughout: FP64 arithmetic is slow on
// this GPU, and each thread's share is a few hundred values.
__global__ void k_bias_grad(const float *__restrict__ dy, long long dybs, int n, long long hw, float *__restrict__ db) {
    const int c = blockIdx.x;
    const long long stride = (long long)gridDim.y * blockDim.x;
    const long long t0 = (long long)blockIdx.y * blockDim.x + threadIdx.x;
    float s = 0.0f;
    for (int img = 0; img < n; ++img) {
        const float *plane = dy + img * dybs + (long long)c * hw;
        if ((hw & 3) == 0 && (reinterpret_cast<uintptr_t>(plane) & 15) == 0) {
            const float4 *p4 = reinterpret_cast<const float4 *>(plane);
            for (long long i = t0; i < hw / 4; i += stride) {
                const float4 v = p4[i];
                s += (v.x + v.y) + (v.z + v.w);
            }
        } else {
            for (long long i = t0; i < hw; i += stride) s += plane[i];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ float sh[32];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (threadIdx.x == 0) atomicAdd(&db[c], v);
    }
}

// NHWC BF16 activations as an MN-major operand: dims (channels, w, h, n),
// box (32 channels, kp pixels, 1, 1), 64-byte swizzle.
bool map_wgrad(CUtensorMap *m, const void *ptr, int c, int w, int h, int n, int kp = WG_KP) {
    const cuuint64_t dims[4] = {cuuint64_t(c), cuuint64_t(w), cuuint64_t(h), cuuint64_t(n)};
    const cuuint64_t strides[3] = {cuuint64_t(c) * 2, cuuint64_t(c) * 2 * w, cuuint64_t(c) * 2 * w * h};
    const cuuint32_t box[4] = {32, cuuint32_t(kp), 1, 1};
    const cuuint32_t es[4] = {1, 1, 1, 1};
    return encode_fn()(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(ptr), dims, strides, box, es,
                       CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                       CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// The band form (k_tc_wgrad_band) of a 3x3 weight gradient: chunk groups
// whose accumulators (96 columns per x chunk and dy chunk) fit 256 TMEM
// columns and whose stages fit ~100 KB of shared memory, so that two CTAs
// share an SM, and about two CTAs per SM.
glbm_status launch_wgrad_band(const void *x, int cx, int cin, const void *dy, int cy, int cout, int n, int h, int w,
                              float *dw, int *err, cudaStream_t stream) {
    const int kp = w <= 16 ? 16 : WG_KP;
    CUtensorMap mX, mDY;
    if (!map_wgrad(&mX, x, cx, w, h, n, kp) || !map_wgrad(&mDY, dy, cy, w, h, n, kp + 2))
        return tcfail(GLBM_EINVAL, "nn_tc_conv_wgrad: tensor map rejected");
    WgradBandArgs a;
    a.starve = take_starve();
    a.n = n;
    a.h = h;
    a.w = w;
    a.nchunk = cx / 32;
    a.nobt = cy / 32;
    a.nob = a.nobt >= 2 ? 2 : 1;
    a.nxc = a.nob == 1 && a.nchunk >= 2 ? 2 : 1;
    a.ngx = (a.nchunk + a.nxc - 1) / a.nxc;
    const int ngo = (a.nobt + a.nob - 1) / a.nob;
    a.cin = cin;
    a.cout = cout;
    a.kp = kp;
    a.xrow = uint32_t(kp) * 64;
    a.dyrow = (uint32_t(kp + 2) * 64 + 511) & ~511u;
    // the tallest band (8, 4, 2 or 1 rows, at most h) of which two stages fit the budget
    const uint32_t budget = 105u * 1024u;
    for (a.R = 8; a.R > 1; a.R >>= 1) {
        const uint32_t st = uint32_t(a.nxc) * uint32_t(a.R + 2) * a.xrow + uint32_t(a.nob) * uint32_t(a.R) * a.dyrow;
        if (a.R <= h && 2 * st <= budget) break;
    }
    a.xsteps = (w + kp - 1) / kp;
    a.ybands = (h + a.R - 1) / a.R;
    a.units = (long long)n * a.ybands * a.xsteps;
    a.dy_off = uint32_t(a.nxc) * uint32_t(a.R + 2) * a.xrow;
    a.stage_bytes = a.dy_off + uint32_t(a.nob) * uint32_t(a.R) * a.dyrow;
    a.stages = int(budget / a.stage_bytes);
    if (a.stages > WB_MAX_STAGES) a.stages = WB_MAX_STAGES;
    if (a.stages < 2) a.stages = 2;
    a.tmem_cols = 32;
    while (a.tmem_cols < uint32_t(96 * a.nob * a.nxc)) a.tmem_cols <<= 1;
    a.vec = (cin % 4 == 0 && (reinterpret_cast<uintptr_t>(dw) & 15u) == 0) ? 1 : 0;
    a.dw = dw;
    a.err = err;
    const int groups = a.ngx * ngo;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return tccuda(e, "nn_tc_conv_wgrad: device query");
    long long splits = (2LL * nsm + groups - 1) / groups;
    if (splits > a.units) splits = a.units;
    if (splits < 1) splits = 1;
    if (splits > 65535) splits = 65535;
    a.units_per_cta = int((a.units + splits - 1) / splits);
    splits = (a.units + a.units_per_cta - 1) / a.units_per_cta;
    // the stages also hold the epilogue's 32 x 32 x 9 FP32 gather
    const size_t smem = 1024 + std::max(size_t(a.stages) * a.stage_bytes, size_t(32 * 32 * 9 * 4));
    e = cudaFuncSetAttribute(k_tc_wgrad_band, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return tccuda(e, "nn_tc_conv_wgrad: shared memory attribute");
    k_tc_wgrad_band<<<dim3(unsigned(groups), unsigned(splits)), WG_THREADS, smem, stream>>>(mX, mDY, a);
    e = cudaGetLastError();
    return e == cudaSuccess ? GLBM_OK : tccuda(e, "nn_tc_conv_wgrad launch");
}

}  // namespace

extern "C" glbm_status glbm_nn_tc_conv_wgrad(const void *x, int cx, int cin, const void *dy, int cy, int cout,
                                             int n, int h, int w, int k, float *dw, int *err, void *stream) {
    if (!x || !dy || !dw || !err) return tcfail(GLBM_EINVAL, "nn_tc_conv_wgrad: x, dy, dw and err are required");
    if (n < 1 || h < 1 || w < 1 || (k != 1 && k != 3))
        return tcfail(GLBM_EINVAL, "nn_tc_conv_wgrad: need n, h, w >= 1 and k = 1 or 3");
    if (cx < 32 || cx % 32 || cin < 1 || cin > cx || cy < 32 || cy % 32 || cy > 256 || cout < 1 || cout > cy)
        return tcfail(GLBM_EINVAL, "nn_tc_conv_wgrad: need cx, cy multiples of 32 (cy <= 256), 1 <= cin <= cx, "
                                   "1 <= cout <= cy");
    if ((uintptr_t(x) | uintptr_t(dy)) & 15u) return tcfail(GLBM_EINVAL, "nn_tc_conv_wgrad: arrays must be 16-byte aligned");
    if (!encode_fn()) return tcfail(GLBM_ECUDA, "nn_tc_conv_wgrad: cuTensorMapEncodeTiled is not available");
    if (k == 3 && g_tc_variant != 1)
        return launch_wgrad_band(x, cx, cin, dy, cy, cout, n, h, w, dw, err, static_cast<cudaStream_t>(stream));
    CUtensorMap mX, mDY;
    if (!map_wgrad(&mX, x, cx, w, h, n) || !map_wgrad(&mDY, dy, cy, w, h, n))
        return tcfail(GLBM_EINVAL, "nn_tc_conv_wgrad: tensor map rejected");
    WgradArgs a;
    a.starve = take_starve();
    a.n = n;
    a.h = h;
    a.w = w;
    a.k = k;
    a.nchunk = cx / 32;
    a.nf = k * k * a.nchunk;
    a.cin = cin;
    a.cout = cout;
    a.cy = cy;
    a.xsteps = (w + WG_KP - 1) / WG_KP;
    a.stage_bytes = uint32_t((4 + cy / 32) * WG_BOX);
    a.tx_a = 4 * WG_BOX;
    a.tmem_cols = 32;
    while (a.tmem_cols < uint32_t(cy)) a.tmem_cols <<= 1;
    a.dw = dw;
    a.err = err;
    const int mtiles = (a.nf + 3) / 4;
    int dev = 0, nsm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return tccuda(e, "nn_tc_conv_wgrad: device query");
    // split the n*h rows so that about 2 CTAs per SM run, each >= 4 rows
    const long long rows = (long long)n * h;
    long long splits = (2LL * nsm + mtiles - 1) / mtiles;
    if (splits > rows / 4) splits = rows / 4;
    if (splits < 1) splits = 1;
    if (splits > 65535) splits = 65535;
    a.rows_per_cta = int((rows + splits - 1) / splits);
    splits = (rows + a.rows_per_cta - 1) / a.rows_per_cta;
    const size_t smem = 1024 + size_t(WG_STAGES) * a.stage_bytes;
    e = cudaFuncSetAttribute(k_tc_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return tccuda(e, "nn_tc_conv_wgrad: shared memory attribute");
    k_tc_wgrad<<<dim3(unsigned(mtiles), unsigned(splits)), WG_THREADS, smem, static_cast<cudaStream_t>(stream)>>>(
        mX, mDY, a);
    e = cudaGetLastError();
    return e == cudaSuccess ? GLBM_OK : tccuda(e, "nn_tc_conv_wgrad launch");
}

extern "C" glbm_status glbm_nn_tc_pack_weights_flip(const float *wf, int cout, int cin, int k, int c_begin,
                                                    int c_pad, int cout_pad, void *wt, void *stream) {
    if (!wf || !wt || cout < 1 || cin < 1 || (k != 1 && k != 3) || c_begin < 0 || c_begin >= cin || c_pad < 1 ||
        cout_pad < cout)
        return tcfail(GLBM_EINVAL, "nn_tc_pack_weights_flip: invalid sizes or pointers");
    const long long total = (long long)k * k * c_pad * cout_pad;
    k_pack_w_flip<<<grid_for(total), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        wf, cout, cin, k, c_begin, c_pad, cout_pad, static_cast<__nv_bfloat16 *>(wt));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GLBM_OK : tccuda(e, "nn_tc_pack_weights_flip launch");
}

extern "C" glbm_status glbm_nn_bias_grad(const float *dy, long long dybs, int c, int n, int h, int w, float *db,
                                         void *stream) {
    if (!dy || !db || c < 1 || n < 1 || h < 1 || w < 1 || dybs < (long long)c * h * w)
        return tcfail(GLBM_EINVAL, "nn_bias_grad: invalid sizes or pointers");
    const long long hw = (long long)h * w;
    // about 64 values per thread, and enough blocks for every SM
    long long parts = ((long long)n * hw + 256 * 64 - 1) / (256 * 64);
    if (parts > 1024) parts = 1024;
    if (parts < 1) parts = 1;
    k_bias_grad<<<dim3(unsigned(c), unsigned(parts)), 256, 0, static_cast<cudaStream_t>(stream)>>>(dy, dybs, n, hw, db);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? GLBM_OK : tccuda(e, "nn_bias_grad launch");
}
