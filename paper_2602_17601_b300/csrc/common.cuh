// Shared helpers of the GNN-MPC CUDA library: error state, bounded grid
// barrier, workspace carving.  Internal header (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/gm.h"

namespace gmi {

// ---------------------------------------------------------------- errors
void set_error(const char* fmt, ...);
void clear_error();

#define GM_CHECK_ARG(cond, ...)                 \
    do {                                        \
        if (!(cond)) {                          \
            ::gmi::set_error(__VA_ARGS__);      \
            return GM_ERR_INVALID_ARG;          \
        }                                       \
    } while (0)

#define GM_CUDA_TRY(expr)                                                          \
    do {                                                                           \
        cudaError_t _e = (expr);                                                   \
        if (_e != cudaSuccess) {                                                   \
            ::gmi::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(_e), \
                             __FILE__, __LINE__);                                  \
            return GM_ERR_CUDA;                                                    \
        }                                                                          \
    } while (0)

// Every kernel launch of the library is followed by GM_LAUNCH_CHECK, which also
// counts it (gm_launch_count).
void count_launch();

#define GM_LAUNCH_CHECK()                                                           \
    do {                                                                            \
        ::gmi::count_launch();                                                      \
        cudaError_t _e = cudaGetLastError();                                        \
        if (_e != cudaSuccess) {                                                    \
            ::gmi::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(_e), \
                             __FILE__, __LINE__);                                   \
            return GM_ERR_CUDA;                                                     \
        }                                                                           \
    } while (0)

#define GM_TRY(expr)                     \
    do {                                 \
        gm_status _s = (expr);           \
        if (_s != GM_OK) return _s;      \
    } while (0)

static inline int cdiv(long long a, long long b) { return (int)((a + b - 1) / b); }

// ---------------------------------------------------------------- device status word
// Kernels that can give up (a bounded wait) or detect a numeric failure OR a
// gm_status code into this word; the host reads it into gm_stats.
struct DevStatus {
    int code;
};

__device__ __forceinline__ void dev_fail(int* status, int code) { atomicOr(status, 1 << code); }

// Maxima of residuals that keep a NaN (fmax drops it, which would let a NaN
// iterate pass a convergence test).
__device__ __forceinline__ float nmaxf(float a, float b) {
    return (a != a || b != b) ? __int_as_float(0x7fc00000) : fmaxf(a, b);
}
__device__ __forceinline__ double nmax(double a, double b) {
    return (a != a || b != b) ? __longlong_as_double(0x7ff8000000000000LL) : fmax(a, b);
}

// ---------------------------------------------------------------- grid barrier
// A monotone arrival counter: barrier number `phase` (1, 2, ...) completes when
// counter >= phase * nblocks.  The counter is zeroed by the host before the
// launch.  Every wait is bounded: after max_spins polls the block records
// GM_ERR_TIMEOUT and returns false, and the caller leaves the kernel.  All
// blocks of the grid must be co-resident (cooperative launch).
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool grid_barrier(unsigned* counter, unsigned nblocks, unsigned phase,
                                             long long max_spins, int* status) {
    __syncthreads();
    __shared__ int s_ok;
    if (threadIdx.x == 0) {
        __threadfence();
        atomicAdd(counter, 1u);
        unsigned target = phase * nblocks;
        long long spins = 0;
        int ok = 1;
        while (ld_acquire(counter) < target) {
            if (++spins > max_spins) {
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        if (!ok) dev_fail(status, GM_ERR_TIMEOUT);
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// ---------------------------------------------------------------- workspace carving
struct Carver {
    char* base = nullptr;   // nullptr: size-only pass
    size_t off = 0;
    template <class T>
    T* take(size_t count) {
        off = (off + 255) & ~size_t(255);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
};

}  // namespace gmi
