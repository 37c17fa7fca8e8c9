// Convolutional-network kernels for the learned warm start of the GLBM
// (a U-Net that maps the medium to the steady density deviation and
// velocity, trained on the solver's own solutions).  The paper has no
// surrogate; it is this library's addition for cutting time to
// permeability.  FP32 SIMT kernels, NCHW tensors; every tensor argument is
// (pointer, per-sample stride in floats) so that a layer can read or write
// a channel slice of a larger buffer (U-Net skip concatenation) in place.
//
//   conv k x k (k = 1 or 3, zero padding k/2): forward (+bias, +ReLU),
//     backward-data (as a forward convolution with flipped, transposed
//     weights), backward-weight and bias (block partials, atomically added)
//   2x2 average pool and 2x nearest upsample, forward and backward
//   channel-slice copy / accumulate, ReLU backward
//   per-channel weighted MSE loss + gradient, Adam update

#include "glbm.h"

#include <cuda_runtime.h>

#include <cstdint>

#include <cstdio>

namespace {

constexpr int TILE = 16;   // output tile is TILE x TILE pixels
constexpr int COT = 16;    // output channels per block
constexpr int CIT = 8;     // input channels staged per iteration

// y[n][co] = b[co] + sum_{ci,ky,kx} w[co][ci][ky][kx] x[n][ci][h+ky-P][w+kx-P]
template <int K, bool RELU>
__global__ void __launch_bounds__(TILE *TILE)
k_conv_fwd(const float *__restrict__ x, long long xbs, int cin, float *__restrict__ y, long long ybs, int cout,
           int H, int W, const float *__restrict__ wt, const float *__restrict__ bias) {
    constexpr int P = K / 2;
    constexpr int S = TILE + K - 1;
    __shared__ float sx[CIT][S][S];
    __shared__ float sw[COT][CIT][K * K];
    const int tilesx = (W + TILE - 1) / TILE;
    const int tx = threadIdx.x % TILE, ty = threadIdx.x / TILE;
    const int ox = (blockIdx.x % tilesx) * TILE, oy = (blockIdx.x / tilesx) * TILE;
    const int co0 = blockIdx.y * COT;
    const int n = blockIdx.z;
    const float *xn = x + n * xbs;
    float acc[COT];
#pragma unroll
    for (int j = 0; j < COT; ++j) acc[j] = 0.0f;
    for (int c0 = 0; c0 < cin; c0 += CIT) {
        for (int i = threadIdx.x; i < CIT * S * S; i += TILE * TILE) {
            const int c = i / (S * S), r = (i / S) % S, q = i % S;
            const int gy = oy + r - P, gx = ox + q - P;
            float v = 0.0f;
            if (c0 + c < cin && gy >= 0 && gy < H && gx >= 0 && gx < W) v = xn[(long long)(c0 + c) * H * W + gy * W + gx];
            sx[c][r][q] = v;
        }
        for (int i = threadIdx.x; i < COT * CIT * K * K; i += TILE * TILE) {
            const int j = i / (CIT * K * K), c = (i / (K * K)) % CIT, t = i % (K * K);
            float v = 0.0f;
            if (co0 + j < cout && c0 + c < cin) v = wt[((long long)(co0 + j) * cin + c0 + c) * K * K + t];
            sw[j][c][t] = v;
        }
        __syncthreads();
#pragma unroll
        for (int c = 0; c < CIT; ++c)
#pragma unroll
            for (int t = 0; t < K * K; ++t) {
                const float v = sx[c][ty + t / K][tx + t % K];
#pragma unroll
                for (int j = 0; j < COT; ++j) acc[j] = fmaf(sw[j][c][t], v, acc[j]);
            }
        __syncthreads();
    }
    const int gy = oy + ty, gx = ox + tx;
    if (gy < H && gx < W) {
#pragma unroll
        for (int j = 0; j < COT; ++j) {
            if (co0 + j >= cout) break;
            float v = acc[j] + (bias ? bias[co0 + j] : 0.0f);
            if (RELU) v = fmaxf(v, 0.0f);
            y[n * ybs + (long long)(co0 + j) * H * W + gy * W + gx] = v;
        }
    }
}

// wt2[ci][co][K-1-ky][K-1-kx] = wt[co][ci][ky][kx]
__global__ void k_flip_transpose(const float *__restrict__ wt, float *__restrict__ wt2, int cout, int cin, int K) {
    const long long total = (long long)cout * cin * K * K;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int t = int(i % (K * K));
        const long long oc = i / (K * K);
        const int ci = int(oc % cin), co = int(oc / cin);
        const int ky = t / K, kx = t % K;
        wt2[((long long)ci * cout + co) * K * K + (K - 1 - ky) * K + (K - 1 - kx)] = wt[i];
    }
}

// dw[co][ci][t] += sum_{n,pix} dy[n][co][pix] x[n][ci][pix + shift(t)]; db[co] += sum dy
// Block: COT output x 16 input channels, one TILE x TILE pixel tile of one
// sample; thread (j, c) = (threadIdx.x / 16, threadIdx.x % 16) owns K*K taps.
template <int K>
__global__ void __launch_bounds__(256)
k_conv_bwd_w(const float *__restrict__ x, long long xbs, int cin, const float *__restrict__ dy, long long dybs,
             int cout, int H, int W, float *__restrict__ dw, float *__restrict__ db) {
    constexpr int P = K / 2;
    constexpr int S = TILE + K - 1;
    constexpr int CI = 16;
    __shared__ float sx[CI][S][S];
    __shared__ float sd[COT][TILE * TILE];
    const int tilesx = (W + TILE - 1) / TILE;
    const int ox = (blockIdx.x % tilesx) * TILE, oy = (blockIdx.x / tilesx) * TILE;
    const int nci = (cin + CI - 1) / CI;
    const int co0 = (blockIdx.y / nci) * COT, ci0 = (blockIdx.y % nci) * CI;
    const int n = blockIdx.z;
    for (int i = threadIdx.x; i < CI * S * S; i += 256) {
        const int c = i / (S * S), r = (i / S) % S, q = i % S;
        const int gy = oy + r - P, gx = ox + q - P;
        float v = 0.0f;
        if (ci0 + c < cin && gy >= 0 && gy < H && gx >= 0 && gx < W)
            v = x[n * xbs + (long long)(ci0 + c) * H * W + gy * W + gx];
        sx[c][r][q] = v;
    }
    for (int i = threadIdx.x; i < COT * TILE * TILE; i += 256) {
        const int j = i / (TILE * TILE), p = i % (TILE * TILE);
        const int gy = oy + p / TILE, gx = ox + p % TILE;
        float v = 0.0f;
        if (co0 + j < cout && gy < H && gx < W) v = dy[n * dybs + (long long)(co0 + j) * H * W + gy * W + gx];
        sd[j][p] = v;
    }
    __syncthreads();
    const int j = threadIdx.x / CI, c = threadIdx.x % CI;
    float acc[K * K];
#pragma unroll
    for (int t = 0; t < K * K; ++t) acc[t] = 0.0f;
    for (int p = 0; p < TILE * TILE; ++p) {
        const float d = sd[j][p];
        const int py = p / TILE, px = p % TILE;
#pragma unroll
        for (int t = 0; t < K * K; ++t) acc[t] = fmaf(d, sx[c][py + t / K][px + t % K], acc[t]);
    }
    if (co0 + j < cout && ci0 + c < cin) {
#pragma unroll
        for (int t = 0; t < K * K; ++t) atomicAdd(&dw[((long long)(co0 + j) * cin + ci0 + c) * K * K + t], acc[t]);
    }
    if (db && ci0 == 0 && threadIdx.x < COT && co0 + threadIdx.x < cout) {
        float s = 0.0f;
        for (int p = 0; p < TILE * TILE; ++p) s += sd[threadIdx.x][p];
        atomicAdd(&db[co0 + threadIdx.x], s);
    }
}

// The element-wise kernels below run on a grid whose z index walks the
// (sample, channel) planes, so that no thread divides a flat 64-bit index:
// planes whose pixels are contiguous (ReLU mask, channel copies) are walked
// in float4 runs where sizes and addresses allow; the resampling kernels
// (pooling, upsampling) give each thread one pixel of a 32 x 8 tile.
constexpr int kPlaneBlock = 256;

__device__ __forceinline__ bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// dy = 0 where y <= 0 (and where y is NaN), plane by plane
__global__ void k_relu_bwd(const float *__restrict__ y, long long ybs, float *__restrict__ dy, long long dybs,
                           int c, long long hw, int n) {
    for (long long q = blockIdx.z; q < (long long)n * c; q += gridDim.z) {
        const long long s = q / c, ch = q - s * c;
        const float *yp = y + s * ybs + ch * hw;
        float *dp = dy + s * dybs + ch * hw;
        const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
        if ((hw & 3) == 0 && aligned16(yp) && aligned16(dp)) {
            const float4 *y4 = reinterpret_cast<const float4 *>(yp);
            float4 *d4 = reinterpret_cast<float4 *>(dp);
            for (long long i = t0; i < hw / 4; i += st) {
                const float4 a = y4[i];
                float4 g = d4[i];
                g.x = a.x > 0.0f ? g.x : 0.0f;
                g.y = a.y > 0.0f ? g.y : 0.0f;
                g.z = a.z > 0.0f ? g.z : 0.0f;
                g.w = a.w > 0.0f ? g.w : 0.0f;
                d4[i] = g;
            }
        } else {
            for (long long i = t0; i < hw; i += st)
                if (!(yp[i] > 0.0f)) dp[i] = 0.0f;
        }
    }
}

// dst[n][0:c] (=|+=) src[n][0:c], plane by plane
__global__ void k_copy_ch(const float *__restrict__ src, long long sbs, float *__restrict__ dst, long long dbs, int c,
                          long long hw, int n, int accumulate) {
    for (long long q = blockIdx.z; q < (long long)n * c; q += gridDim.z) {
        const long long s = q / c, ch = q - s * c;
        const float *sp = src + s * sbs + ch * hw;
        float *dp = dst + s * dbs + ch * hw;
        const long long t0 = blockIdx.x * (long long)blockDim.x + threadIdx.x, st = (long long)gridDim.x * blockDim.x;
        if ((hw & 3) == 0 && aligned16(sp) && aligned16(dp)) {
            const float4 *s4 = reinterpret_cast<const float4 *>(sp);
            float4 *d4 = reinterpret_cast<float4 *>(dp);
            for (long long i = t0; i < hw / 4; i += st) {
                float4 v = s4[i];
                if (accumulate) {
                    const float4 o = d4[i];
                    v.x += o.x;
                    v.y += o.y;
                    v.z += o.z;
                    v.w += o.w;
                }
                d4[i] = v;
            }
        } else {
            for (long long i = t0; i < hw; i += st) {
                const float v = sp[i];
                if (accumulate) dp[i] += v;
                else dp[i] = v;
            }
        }
    }
}

// y (H/2 x W/2) = mean of 2x2 blocks of x (H x W); one output pixel per thread
__global__ void k_pool_fwd(const float *__restrict__ x, long long xbs, float *__restrict__ y, long long ybs, int c,
                           int H, int W, int n) {
    const int h2 = H / 2, w2 = W / 2;
    const int xx = blockIdx.x * blockDim.x + threadIdx.x, yy = blockIdx.y * blockDim.y + threadIdx.y;
    if (xx >= w2 || yy >= h2) return;
    for (long long q = blockIdx.z; q < (long long)n * c; q += gridDim.z) {
        const long long s = q / c, ch = q - s * c;
        const float *b = x + s * xbs + ch * H * W + (long long)(2 * yy) * W + 2 * xx;
        y[s * ybs + ch * h2 * w2 + (long long)yy * w2 + xx] = 0.25f * ((b[0] + b[1]) + (b[W] + b[W + 1]));
    }
}

// dx (H x W) (=|+=) dy (H/2 x W/2) / 4 spread over each 2x2 block
__global__ void k_pool_bwd(const float *__restrict__ dy, long long dybs, float *__restrict__ dx, long long dxbs, int c,
                           int H, int W, int n, int accumulate) {
    const int xx = blockIdx.x * blockDim.x + threadIdx.x, yy = blockIdx.y * blockDim.y + threadIdx.y;
    if (xx >= W || yy >= H) return;
    for (long long q = blockIdx.z; q < (long long)n * c; q += gridDim.z) {
        const long long s = q / c, ch = q - s * c;
        const float v = 0.25f * dy[s * dybs + ch * (H / 2) * (W / 2) + (long long)(yy / 2) * (W / 2) + xx / 2];
        float *o = dx + s * dxbs + ch * H * W + (long long)yy * W + xx;
        if (accumulate) *o += v;
        else *o = v;
    }
}

// y (2H x 2W) = nearest upsample of x (H x W)
__global__ void k_up_fwd(const float *__restrict__ x, long long xbs, float *__restrict__ y, long long ybs, int c, int H,
                         int W, int n) {
    const int H2 = 2 * H, W2 = 2 * W;
    const int xx = blockIdx.x * blockDim.x + threadIdx.x, yy = blockIdx.y * blockDim.y + threadIdx.y;
    if (xx >= W2 || yy >= H2) return;
    for (long long q = blockIdx.z; q < (long long)n * c; q += gridDim.z) {
        const long long s = q / c, ch = q - s * c;
        y[s * ybs + ch * H2 * W2 + (long long)yy * W2 + xx] = x[s * xbs + ch * H * W + (long long)(yy / 2) * W + xx / 2];
    }
}

// dx (H x W) = sum over each 2x2 block of dy (2H x 2W)
__global__ void k_up_bwd(const float *__restrict__ dy, long long dybs, float *__restrict__ dx, long long dxbs, int c,
                         int H, int W, int n) {
    const int W2 = 2 * W;
    const int xx = blockIdx.x * blockDim.x + threadIdx.x, yy = blockIdx.y * blockDim.y + threadIdx.y;
    if (xx >= W || yy >= H) return;
    for (long long q = blockIdx.z; q < (long long)n * c; q += gridDim.z) {
        const long long s = q / c, ch = q - s * c;
        const float *b = dy + s * dybs + ch * 4 * H * W + (long long)(2 * yy) * W2 + 2 * xx;
        dx[s * dxbs + ch * H * W + (long long)yy * W + xx] = (b[0] + b[1]) + (b[W2] + b[W2 + 1]);
    }
}

// loss = sum_c cw[c] * mean_{n,pix} (pred - target)^2 ; grad = d loss / d pred
__global__ void k_mse(const float *__restrict__ pred, const float *__restrict__ target, const float *__restrict__ cw,
                      int c, long long hw, int n, float *__restrict__ grad, double *__restrict__ loss) {
    __shared__ double sh[256];
    const long long per = (long long)c * hw, total = per * n;
    double s = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int ch = int((i % per) / hw);
        const float d = pred[i] - target[i];
        const float wgt = cw[ch] / float(hw * n);
        if (grad) grad[i] = 2.0f * wgt * d;
        s += double(wgt) * double(d) * double(d);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int k = 128; k > 0; k >>= 1) {
        if (threadIdx.x < k) sh[threadIdx.x] += sh[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0 && loss) atomicAdd(loss, sh[0]);
}

__global__ void k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, long long count, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
         i += (long long)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// Grids of the plane kernels: blocks of kPlaneBlock threads along each
// (sample, channel) plane of `units` work items, planes along z.  About
// kPlaneBlocks blocks in all: each block walks several planes, so that short
// planes do not turn into one short-lived block per plane.
constexpr long long kPlaneBlocks = 4096;
unsigned plane_z(long long per_plane_blocks, long long planes) {
    long long z = (kPlaneBlocks + per_plane_blocks - 1) / per_plane_blocks;
    z = z < 1 ? 1 : z;
    z = z > planes ? planes : z;
    return unsigned(z > 65535 ? 65535 : z);
}
dim3 plane_grid(long long units, long long planes) {
    long long gx = (units + kPlaneBlock - 1) / kPlaneBlock;
    gx = gx < 1 ? 1 : (gx > 4096 ? 4096 : gx);
    return dim3(unsigned(gx), 1, plane_z(gx, planes));
}
// ... and of the resampling kernels: 32 x 8 pixel tiles of the output plane.
const dim3 kTile(32, 8);
dim3 tile_grid(int w, int h, long long planes) {
    const long long gx = (w + 31) / 32, gy = (h + 7) / 8;
    return dim3(unsigned(gx), unsigned(gy), plane_z(gx * gy, planes));
}

int grid_for(long long total) {
    long long b = (total + 255) / 256;
    return int(b < 1 ? 1 : (b > 152 * 32 ? 152 * 32 : b));
}

glbm_status launch_status() {
    return cudaGetLastError() == cudaSuccess ? GLBM_OK : GLBM_ECUDA;
}

template <int K>
void conv_fwd_k(const float *x, long long xbs, int cin, float *y, long long ybs, int cout, int n, int h, int w,
                const float *wt, const float *b, int relu, cudaStream_t st) {
    dim3 grid(((w + TILE - 1) / TILE) * ((h + TILE - 1) / TILE), (cout + COT - 1) / COT, n);
    if (relu) k_conv_fwd<K, true><<<grid, TILE * TILE, 0, st>>>(x, xbs, cin, y, ybs, cout, h, w, wt, b);
    else k_conv_fwd<K, false><<<grid, TILE * TILE, 0, st>>>(x, xbs, cin, y, ybs, cout, h, w, wt, b);
}

bool bad_dims(int cin, int cout, int n, int h, int w, int k) {
    return cin < 1 || cout < 1 || n < 1 || h < 1 || w < 1 || (k != 1 && k != 3) || n > 65535 ||
           (long long)((cout + COT - 1) / COT) * ((cin + 15) / 16) > 65535;
}

}  // namespace

extern "C" {

glbm_status glbm_nn_conv_fwd(const float *x, long long xbs, int cin, float *y, long long ybs, int cout, int n, int h,
                             int w, int ksize, const float *wt, const float *bias, int relu, void *stream) {
    if (!x || !y || !wt || bad_dims(cin, cout, n, h, w, ksize)) return GLBM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (ksize == 3) conv_fwd_k<3>(x, xbs, cin, y, ybs, cout, n, h, w, wt, bias, relu, st);
    else conv_fwd_k<1>(x, xbs, cin, y, ybs, cout, n, h, w, wt, bias, relu, st);
    return launch_status();
}

glbm_status glbm_nn_conv_bwd_data(const float *dy, long long dybs, int cout, float *dx, long long dxbs, int cin, int n,
                                  int h, int w, int ksize, const float *wt, float *wt_scratch, void *stream) {
    if (!dy || !dx || !wt || !wt_scratch || bad_dims(cin, cout, n, h, w, ksize)) return GLBM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long nw = (long long)cout * cin * ksize * ksize;
    k_flip_transpose<<<grid_for(nw), 256, 0, st>>>(wt, wt_scratch, cout, cin, ksize);
    if (ksize == 3) conv_fwd_k<3>(dy, dybs, cout, dx, dxbs, cin, n, h, w, wt_scratch, nullptr, 0, st);
    else conv_fwd_k<1>(dy, dybs, cout, dx, dxbs, cin, n, h, w, wt_scratch, nullptr, 0, st);
    return launch_status();
}

glbm_status glbm_nn_conv_bwd_weight(const float *x, long long xbs, int cin, const float *dy, long long dybs, int cout,
                                    int n, int h, int w, int ksize, float *dw, float *db, void *stream) {
    if (!x || !dy || !dw || bad_dims(cin, cout, n, h, w, ksize)) return GLBM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    dim3 grid(((w + TILE - 1) / TILE) * ((h + TILE - 1) / TILE), ((cout + COT - 1) / COT) * ((cin + 15) / 16), n);
    if (ksize == 3) k_conv_bwd_w<3><<<grid, 256, 0, st>>>(x, xbs, cin, dy, dybs, cout, h, w, dw, db);
    else k_conv_bwd_w<1><<<grid, 256, 0, st>>>(x, xbs, cin, dy, dybs, cout, h, w, dw, db);
    return launch_status();
}

glbm_status glbm_nn_relu_bwd(const float *y, long long ybs, float *dy, long long dybs, int c, int n, int h, int w,
                             void *stream) {
    if (!y || !dy || c < 1 || n < 1 || h < 1 || w < 1) return GLBM_EINVAL;
    const long long hw = (long long)h * w;
    k_relu_bwd<<<plane_grid((hw + 3) / 4, (long long)n * c), kPlaneBlock, 0, static_cast<cudaStream_t>(stream)>>>(
        y, ybs, dy, dybs, c, hw, n);
    return launch_status();
}

glbm_status glbm_nn_copy_channels(const float *src, long long sbs, float *dst, long long dbs, int c, int n, int h,
                                  int w, int accumulate, void *stream) {
    if (!src || !dst || c < 1 || n < 1 || h < 1 || w < 1) return GLBM_EINVAL;
    const long long hw = (long long)h * w;
    k_copy_ch<<<plane_grid((hw + 3) / 4, (long long)n * c), kPlaneBlock, 0, static_cast<cudaStream_t>(stream)>>>(src, sbs, dst, dbs, c, hw, n,
                                                                                    accumulate);
    return launch_status();
}

glbm_status glbm_nn_pool2(const float *x, long long xbs, float *y, long long ybs, int c, int n, int h, int w,
                          int backward, int accumulate, void *stream) {
    if (!x || !y || c < 1 || n < 1 || h < 2 || w < 2 || h % 2 || w % 2) return GLBM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // forward: x (h x w) -> y (h/2 x w/2); backward: x = dy (h/2 x w/2) -> y = dx (h x w)
    const long long planes = (long long)n * c;
    if (!backward) k_pool_fwd<<<tile_grid(w / 2, h / 2, planes), kTile, 0, st>>>(x, xbs, y, ybs, c, h, w, n);
    else k_pool_bwd<<<tile_grid(w, h, planes), kTile, 0, st>>>(x, xbs, y, ybs, c, h, w, n, accumulate);
    return launch_status();
}

glbm_status glbm_nn_upsample2(const float *x, long long xbs, float *y, long long ybs, int c, int n, int h, int w,
                              int backward, void *stream) {
    if (!x || !y || c < 1 || n < 1 || h < 1 || w < 1) return GLBM_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // forward: x (h x w) -> y (2h x 2w); backward: x = dy (2h x 2w) -> y = dx (h x w)
    const long long planes = (long long)n * c;
    if (!backward) k_up_fwd<<<tile_grid(2 * w, 2 * h, planes), kTile, 0, st>>>(x, xbs, y, ybs, c, h, w, n);
    else k_up_bwd<<<tile_grid(w, h, planes), kTile, 0, st>>>(x, xbs, y, ybs, c, h, w, n);
    return launch_status();
}

glbm_status glbm_nn_mse(const float *pred, const float *target, const float *channel_weight, int c, int n, int h,
                        int w, float *grad, double *loss, void *stream) {
    if (!pred || !target || !channel_weight || c < 1 || n < 1) return GLBM_EINVAL;
    const long long hw = (long long)h * w;
    k_mse<<<grid_for(c * hw * n), 256, 0, static_cast<cudaStream_t>(stream)>>>(pred, target, channel_weight, c, hw, n,
                                                                               grad, loss);
    return launch_status();
}

glbm_status glbm_nn_adam(float *p, const float *g, float *m, float *v, long long count, float lr, float beta1,
                         float beta2, float eps, int t, void *stream) {
    if (!p || !g || !m || !v || count < 1 || t < 1) return GLBM_EINVAL;
    const float c1 = 1.0f - powf(beta1, float(t)), c2 = 1.0f - powf(beta2, float(t));
    k_adam<<<grid_for(count), 256, 0, static_cast<cudaStream_t>(stream)>>>(p, g, m, v, count, lr, beta1, beta2, eps,
                                                                           c1, c2);
    return launch_status();
}

}  // extern "C"
