// Guard zones around a handle's device buffers: memory safety evidence where
// no sanitizer runs.  Each buffer is allocated with kGuard extra bytes on
// either side, filled with kGuardByte; count_damage() reads them back and
// counts the bytes that no longer hold it -- 0 unless a kernel (or a copy)
// wrote outside its buffer.  The pointer handed out is raw + kGuard, so the
// buffers keep cudaMalloc's alignment (kGuard is a multiple of 256).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <cstring>
#include <vector>

namespace glbm_guard {

constexpr size_t kGuard = 4096;
constexpr unsigned char kGuardByte = 0xA5;
constexpr int kMaxBuffers = 24;

struct Table {
    char *raw[kMaxBuffers] = {};
    size_t bytes[kMaxBuffers] = {};
    int n = 0;
};

// cudaMalloc of `bytes` with both guard zones filled (on `stream`).
inline cudaError_t alloc(Table &t, void **p, size_t bytes, cudaStream_t stream) {
    *p = nullptr;
    if (t.n >= kMaxBuffers) return cudaErrorMemoryAllocation;
    char *raw = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&raw), bytes + 2 * kGuard);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(raw, kGuardByte, kGuard, stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(raw + kGuard + bytes, kGuardByte, kGuard, stream);
    if (e != cudaSuccess) {
        cudaFree(raw);
        return e;
    }
    t.raw[t.n] = raw;
    t.bytes[t.n] = bytes;
    ++t.n;
    *p = raw + kGuard;
    return cudaSuccess;
}

// Frees a buffer from alloc() (and forgets it); a pointer it did not hand
// out is freed as it is.
inline void release(Table &t, void *p) {
    if (!p) return;
    for (int i = 0; i < t.n; ++i)
        if (t.raw[i] + kGuard == static_cast<char *>(p)) {
            cudaFree(t.raw[i]);
            t.raw[i] = t.raw[t.n - 1];
            t.bytes[i] = t.bytes[t.n - 1];
            --t.n;
            return;
        }
    cudaFree(p);
}

// Guard bytes that no longer hold kGuardByte, over every live buffer.  With
// poke != 0 one byte of the first buffer's trailing guard is overwritten
// first (a check that the count sees it) and restored afterwards.  Waits for
// `stream`.
inline cudaError_t count_damage(const Table &t, cudaStream_t stream, int poke, long long *damaged) {
    *damaged = 0;
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e == cudaSuccess && poke && t.n > 0) e = cudaMemset(t.raw[0] + kGuard + t.bytes[0], 0, 1);
    std::vector<unsigned char> h(2 * kGuard);
    for (int i = 0; i < t.n && e == cudaSuccess; ++i) {
        e = cudaMemcpy(h.data(), t.raw[i], kGuard, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(h.data() + kGuard, t.raw[i] + kGuard + t.bytes[i], kGuard,
                                             cudaMemcpyDeviceToHost);
        for (size_t j = 0; j < h.size() && e == cudaSuccess; ++j) *damaged += h[j] != kGuardByte;
    }
    if (poke && t.n > 0) {
        const cudaError_t r = cudaMemset(t.raw[0] + kGuard + t.bytes[0], kGuardByte, 1);
        if (e == cudaSuccess) e = r;
    }
    return e;
}

}  // namespace glbm_guard
