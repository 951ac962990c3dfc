// Unit-rate microbenchmarks for the roofline denominators of the raster
// kernels: the special-function unit's base-2 exponential (one per fragment
// in both passes), FP32 fused multiply-add in its scalar and packed
// two-lane forms, and float reductions into global memory in the backward's
// pattern (12 lanes of a warp adding into one 64-byte gradient row). They
// are measurement helpers, not part of the training path: every loop has a
// fixed trip count, every address is inside the caller's buffer.
#include <cuda_runtime.h>

#include "lgs_internal.cuh"

namespace lgs {
namespace {

constexpr int kPeakThreads = 256;
constexpr int kPeakUnroll = 32;

__device__ __forceinline__ float peak_ex2(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// One dependent chain per thread, x <- 2^x - 1.5, which stays in [-1, 0.5]
// (up to the approximation's rounding) from any start in [-1, 1] and
// converges to the fixed point -1; full occupancy hides the chain's latency.
__global__ void __launch_bounds__(kPeakThreads) k_peak_ex2(float *__restrict__ out, int iters) {
    float x = 0.002f * (float)(threadIdx.x & 255) - 0.25f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kPeakUnroll; ++u) x = peak_ex2(x) - 1.5f;
    }
    out[(int64_t)blockIdx.x * kPeakThreads + threadIdx.x] = x;
}

// One dependent chain per thread, so that the compiler cannot pair
// independent scalar operations into the packed form: scalar x <- x a + b,
// or the same on both lanes of a float2 with the packed instruction.
template <bool PACKED>
__global__ void __launch_bounds__(kPeakThreads) k_peak_ffma(float *__restrict__ out, int iters) {
    const float a = 0.9990234375f, b = 1.0e-3f;
    if constexpr (PACKED) {
        float2 x = make_float2(0.001f * (float)threadIdx.x, 0.5f);
        const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kPeakUnroll; ++u) x = __ffma2_rn(x, a2, b2);
        }
        out[(int64_t)blockIdx.x * kPeakThreads + threadIdx.x] = x.x + x.y;
    } else {
        float x = 0.001f * (float)threadIdx.x;
        for (int i = 0; i < iters; ++i) {
#pragma unroll
            for (int u = 0; u < kPeakUnroll; ++u) x = __fmaf_rn(x, a, b);
        }
        out[(int64_t)blockIdx.x * kPeakThreads + threadIdx.x] = x;
    }
}

// Each warp, iters times: a row drawn by a hash of (warp, iteration) from
// [0, n_rows), lanes 0..11 each add 1 to one float of it (a reduction with
// no returned value, as the backward's gradient atomics).
__global__ void __launch_bounds__(kPeakThreads) k_peak_red(float *__restrict__ rows,
                                                           uint64_t n_rows, int iters) {
    const int lane = threadIdx.x & 31;
    const uint32_t gw = (uint32_t)((blockIdx.x * kPeakThreads + threadIdx.x) >> 5);
    uint32_t h = gw * 2654435761u + 0x9e3779b9u;
    for (int i = 0; i < iters; ++i) {
        h ^= h >> 15;
        h *= 2246822519u;
        h ^= h >> 13;
        const uint64_t row = ((uint64_t)h * n_rows) >> 32;  // < n_rows
        if (lane < 12) atomicAdd(rows + 16 * row + lane, 1.0f);
        h += 0x6d2b79f5u;
    }
}

lgs_status peak_args(int blocks, int iters) {
    return blocks > 0 && blocks <= (1 << 20) && iters > 0 ? LGS_OK : LGS_ERR_INVALID_ARG;
}

}  // namespace

lgs_status peak_ex2(float *out, int blocks, int iters, cudaStream_t s) {
    if (!out || peak_args(blocks, iters) != LGS_OK) return LGS_ERR_INVALID_ARG;
    k_peak_ex2<<<blocks, kPeakThreads, 0, s>>>(out, iters);
    count_launch();
    return check_launch();
}

lgs_status peak_ffma(float *out, int blocks, int iters, int packed, cudaStream_t s) {
    if (!out || peak_args(blocks, iters) != LGS_OK) return LGS_ERR_INVALID_ARG;
    if (packed)
        k_peak_ffma<true><<<blocks, kPeakThreads, 0, s>>>(out, iters);
    else
        k_peak_ffma<false><<<blocks, kPeakThreads, 0, s>>>(out, iters);
    count_launch();
    return check_launch();
}

lgs_status peak_red(float *rows, int64_t n_rows, int blocks, int iters, cudaStream_t s) {
    if (!rows || n_rows <= 0 || n_rows > 0x7fffffffLL || !aligned16(rows) ||
        peak_args(blocks, iters) != LGS_OK)
        return LGS_ERR_INVALID_ARG;
    k_peak_red<<<blocks, kPeakThreads, 0, s>>>(rows, (uint64_t)n_rows, iters);
    count_launch();
    return check_launch();
}

}  // namespace lgs
