// common.cuh -- shared host/device plumbing of the CUDA library (no counting arithmetic).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstddef>
#include <vector>

#include "tc.h"

namespace tcg {

constexpr int kWarp = 32;
constexpr unsigned kFull = 0xFFFFFFFFu;

// ------------------------------------------------------------------ device status word
// One per handle / batch.  The first error code written wins; `detail` carries an index
// (e.g. the first out-of-range input position).
struct DevStatus {
    int code;
    int pad;
    long long detail;
};

__device__ __forceinline__ void set_error(DevStatus* st, int code, long long detail) {
    if (atomicCAS(&st->code, 0, code) == 0) st->detail = detail;
}

// ------------------------------------------------------------------ warp helpers
__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ unsigned lanemask_le() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_le;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        T w = __shfl_xor_sync(kFull, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// inclusive prefix sum over the 32 lanes
template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T v, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T w = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += w;
    }
    return v;
}

// ------------------------------------------------------------------ host helpers
#define TC_CUDA_TRY(expr)                                  \
    do {                                                   \
        cudaError_t _e = (expr);                           \
        if (_e != cudaSuccess) {                           \
            (void)cudaGetLastError();                      \
            return (_e == cudaErrorMemoryAllocation)       \
                       ? TC_ERR_OOM                        \
                       : TC_ERR_CUDA;                      \
        }                                                  \
    } while (0)

#define TC_TRY(expr)                    \
    do {                                \
        tc_status _s = (expr);          \
        if (_s != TC_OK) return _s;     \
    } while (0)

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Device allocation through the caller's hooks or cudaMallocAsync.  Tracks the bytes it
// holds so a build can respect its budget.
struct Allocator {
    tc_alloc_fn alloc = nullptr;
    tc_release_fn release = nullptr;
    void* ctx = nullptr;
    int64_t budget = 0;      // 0 = no limit
    int64_t held = 0;        // bytes currently held through this allocator
    int64_t peak = 0;

    tc_status get(void** p, size_t bytes, cudaStream_t s) {
        *p = nullptr;
        if (bytes == 0) bytes = 16;
        bytes = align_up(bytes, 256);
        if (budget > 0 && held + (int64_t)bytes > budget) return TC_ERR_BUDGET;
        if (alloc) {
            *p = alloc(ctx, bytes, (tc_stream_t)s);
            if (!*p) return TC_ERR_OOM;
        } else {
            cudaError_t e = cudaMallocAsync(p, bytes, s);
            if (e != cudaSuccess) {
                (void)cudaGetLastError();
                *p = nullptr;
                return e == cudaErrorMemoryAllocation ? TC_ERR_OOM : TC_ERR_CUDA;
            }
        }
        held += (int64_t)bytes;
        if (held > peak) peak = held;
        return TC_OK;
    }
    void put(void* p, size_t bytes, cudaStream_t s) {
        if (!p) return;
        if (bytes == 0) bytes = 16;
        bytes = align_up(bytes, 256);
        if (release) release(ctx, p, (tc_stream_t)s);
        else (void)cudaFreeAsync(p, s);
        held -= (int64_t)bytes;
    }
};

// A device buffer owned by an Allocator (RAII within one host call).
template <typename T>
struct DevBuf {
    T* ptr = nullptr;
    size_t count = 0;
    Allocator* al = nullptr;
    cudaStream_t s = nullptr;
    tc_status alloc(Allocator* a, size_t n, cudaStream_t st) {
        release();
        al = a;
        s = st;
        count = n;
        void* p = nullptr;
        tc_status r = a->get(&p, n * sizeof(T), st);
        ptr = (T*)p;
        if (r != TC_OK) count = 0;
        return r;
    }
    void release() {
        if (ptr && al) al->put(ptr, count * sizeof(T), s);
        ptr = nullptr;
        count = 0;
    }
    T* detach() {
        T* p = ptr;
        ptr = nullptr;
        count = 0;
        return p;
    }
    ~DevBuf() { release(); }
};

int num_sms();

// Host-side count of kernel launches made by this library (tc_kernel_launches).
void note_launch(int k = 1);

// Keep the device's default stream-ordered pool from returning freed memory to the
// driver at every synchronisation (once per device, this process only).
void retain_pool_memory();

}  // namespace tcg
