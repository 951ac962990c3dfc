// Stable LSD radix sort of (key, u32 value) pairs and an exclusive scan,
// both with the element count read on the device, so that they can sit in a
// captured CUDA graph behind kernels that produce the count.
//
// Radix sort, one 8-bit digit per pass, reduce-then-scan:
//   upsweep   - a fixed grid of G CTAs, CTA b owns a contiguous run of
//               4096-item tiles and counts its digits;
//   scan      - one block per digit scans that digit's row of the [256][G]
//               counts (its start within the digit for each CTA) and
//               records the digit's total;
//   downsweep - each CTA scans the 256 digit totals into digit starts,
//               walks its tiles in order, ranks the items of a
//               tile stably with a warp multisplit (peer masks from
//               per-bit ballots), stages them
//               in shared memory in local digit order and writes them out
//               at its running per-digit offsets.
// A CTA handles its tiles in input order and ranks are stable inside a
// tile, so every pass is stable.
#include <cuda_runtime.h>

#include "lgs_internal.cuh"

namespace lgs {

namespace {

constexpr int kSortThreads = 512;
constexpr int kSortWarps = kSortThreads / kWarp;
constexpr int kItemsPerThread = 8;
constexpr int kTile = kSortThreads * kItemsPerThread;  // 4096
constexpr int kRadix = 256;

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ int64_t read_count(int64_t n_max, const int64_t *d_n64,
                                              const int32_t *d_n32) {
    int64_t n = n_max;
    if (d_n64) n = *d_n64;
    else if (d_n32) n = *d_n32;
    return n < n_max ? n : n_max;
}

// Lanes of `act` whose 8-bit digit equals this lane's, from one ballot per
// digit bit (every lane of `act` must call it). Cheaper than match.any, which
// runs on the address-divergence pipe and saturates it here.
__device__ __forceinline__ uint32_t digit_peers(uint32_t act, int d) {
    uint32_t peers = act;
#pragma unroll
    for (int b = 0; b < 8; ++b) {
        const bool bit = (d >> b) & 1;
        const uint32_t m = __ballot_sync(act, bit);
        peers &= bit ? m : ~m;
    }
    return peers;
}

template <typename K>
__device__ __forceinline__ int digit_of(K key, int shift) {
    return (int)((key >> shift) & (K)(kRadix - 1));
}

// Exclusive scan of one value per thread over the whole block (blockDim.x a
// multiple of 32, <= 1024). Returns the exclusive prefix; *total receives the
// block sum. smem holds 33 slots: 32 warp prefixes and the total (slot 32,
// kept apart so that a 32-warp block does not overwrite warp 31's prefix).
__device__ uint64_t block_exclusive_scan(uint64_t x, uint64_t *smem /* [33] */, uint64_t *total) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint64_t inc = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint64_t y = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += y;
    }
    if (lane == 31) smem[wid] = inc;
    __syncthreads();
    const int nw = blockDim.x >> 5;
    if (wid == 0) {
        uint64_t w = lane < nw ? smem[lane] : 0;
        uint64_t winc = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint64_t y = __shfl_up_sync(0xffffffffu, winc, o);
            if (lane >= o) winc += y;
        }
        if (lane < nw) smem[lane] = winc - w;
        if (lane == nw - 1) smem[32] = winc;
    }
    __syncthreads();
    uint64_t r = smem[wid] + inc - x;
    if (total) *total = smem[32];
    __syncthreads();
    return r;
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_radix_upsweep(const K *__restrict__ keys,
                                                               int64_t n_max, const int64_t *d_n64,
                                                               const int32_t *d_n32, int shift,
                                                               uint32_t *__restrict__ counts) {
    __shared__ uint32_t s_cnt[kSortWarps][kRadix];
    const int G = gridDim.x, b = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) (&s_cnt[0][0])[i] = 0;
    __syncthreads();
    const int64_t n = read_count(n_max, d_n64, d_n32);
    const int64_t tiles = (n + kTile - 1) / kTile;
    const int64_t t0 = tiles * b / G, t1 = tiles * (b + 1) / G;
    const int64_t lo = t0 * kTile, hi = min(t1 * kTile, n);
    for (int64_t base = lo; base < hi; base += kSortThreads) {
        const int64_t i = base + threadIdx.x;
        const bool ok = i < hi;
        const int d = ok ? digit_of(keys[i], shift) : -1;
        const uint32_t act = __ballot_sync(0xffffffffu, ok);
        if (ok) {
            const uint32_t peers = digit_peers(act, d);
            if (lane == __ffs(peers) - 1) s_cnt[wid][d] += __popc(peers);
        }
        __syncwarp();
    }
    __syncthreads();
    for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
        uint32_t s = 0;
        for (int w = 0; w < kSortWarps; ++w) s += s_cnt[w][d];
        counts[(int64_t)d * G + b] = s;
    }
}

// Per digit d (one block each): exclusive scan of counts[d][0..G) in place,
// and totals[d] = the row's sum. The digits' bases are scanned by each
// downsweep CTA from the 256 totals.
__global__ void __launch_bounds__(1024) k_scan_digit_rows(uint32_t *counts, int G,
                                                         uint32_t *totals) {
    __shared__ uint64_t s_tmp[33];
    uint32_t *row = counts + (int64_t)blockIdx.x * G;
    uint64_t carry = 0;
    for (int base = 0; base < G; base += blockDim.x) {
        const int i = base + threadIdx.x;
        const uint32_t x = i < G ? row[i] : 0u;
        uint64_t tot;
        const uint64_t ex = block_exclusive_scan(x, s_tmp, &tot);
        if (i < G) row[i] = (uint32_t)(carry + ex);
        carry += tot;
    }
    if (threadIdx.x == 0) totals[blockIdx.x] = (uint32_t)carry;
}

template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_radix_downsweep(
    const K *__restrict__ keys_in, const uint32_t *__restrict__ vals_in, K *__restrict__ keys_out,
    uint32_t *__restrict__ vals_out, const uint32_t *__restrict__ offsets,
    const uint32_t *__restrict__ totals, int64_t n_max, const int64_t *d_n64, const int32_t *d_n32,
    int shift) {
    __shared__ uint32_t s_wcnt[kSortWarps][kRadix];
    __shared__ uint32_t s_run[kRadix];
    __shared__ uint32_t s_start[kRadix];
    __shared__ uint32_t s_tcnt[kRadix];
    __shared__ uint64_t s_scan[33];
    // staging of one tile in local digit order (dynamic: above the 48 KB
    // static limit for 64-bit keys)
    extern __shared__ __align__(16) unsigned char s_dyn[];
    K *s_keys = reinterpret_cast<K *>(s_dyn);
    uint32_t *s_vals = reinterpret_cast<uint32_t *>(s_dyn + sizeof(K) * kTile);

    const int G = gridDim.x, b = blockIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t n = read_count(n_max, d_n64, d_n32);
    const int64_t tiles = (n + kTile - 1) / kTile;
    const int64_t t0 = tiles * b / G, t1 = tiles * (b + 1) / G;
    {
        // global start of each digit, then of this CTA's share of it
        const uint64_t tot = threadIdx.x < kRadix ? totals[threadIdx.x] : 0u;
        const uint64_t base = block_exclusive_scan(tot, s_scan, nullptr);
        if (threadIdx.x < kRadix)
            s_run[threadIdx.x] = (uint32_t)base + offsets[(int64_t)threadIdx.x * G + b];
    }
    const uint32_t lt = lanemask_lt();

    for (int64_t tile = t0; tile < t1; ++tile) {
        const int64_t base = tile * kTile;
        for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) (&s_wcnt[0][0])[i] = 0;
        __syncthreads();
        K key[kItemsPerThread];
        uint32_t val[kItemsPerThread], rank[kItemsPerThread];
        int dig[kItemsPerThread];
#pragma unroll
        for (int j = 0; j < kItemsPerThread; ++j) {
            const int64_t idx = base + wid * (kWarp * kItemsPerThread) + j * kWarp + lane;
            const bool ok = idx < n;
            key[j] = ok ? keys_in[idx] : (K)0;
            val[j] = ok ? vals_in[idx] : 0u;
            dig[j] = ok ? digit_of(key[j], shift) : -1;
        }
#pragma unroll
        for (int j = 0; j < kItemsPerThread; ++j) {
            const int d = dig[j];
            const uint32_t act = __ballot_sync(0xffffffffu, d >= 0);
            if (d >= 0) {
                const uint32_t peers = digit_peers(act, d);
                const uint32_t before = s_wcnt[wid][d];
                rank[j] = before + __popc(peers & lt);
                __syncwarp(peers);
                if (lane == __ffs(peers) - 1) s_wcnt[wid][d] = before + __popc(peers);
            }
            __syncwarp();
        }
        __syncthreads();
        // per digit: exclusive scan over warps, then over digits
        uint32_t tcnt = 0;
        if (threadIdx.x < kRadix) {
            const int d = threadIdx.x;
            for (int w = 0; w < kSortWarps; ++w) {
                const uint32_t c = s_wcnt[w][d];
                s_wcnt[w][d] = tcnt;
                tcnt += c;
            }
        }
        // block scan over the first 256 threads (all threads take part)
        const uint64_t st = block_exclusive_scan(threadIdx.x < kRadix ? tcnt : 0u, s_scan, nullptr);
        if (threadIdx.x < kRadix) {
            s_start[threadIdx.x] = (uint32_t)st;
            s_tcnt[threadIdx.x] = tcnt;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < kItemsPerThread; ++j) {
            if (dig[j] >= 0) {
                const uint32_t pos = s_start[dig[j]] + s_wcnt[wid][dig[j]] + rank[j];
                s_keys[pos] = key[j];
                s_vals[pos] = val[j];
            }
        }
        __syncthreads();
        const int ntile = (int)min((int64_t)kTile, n - base);
        for (int i = threadIdx.x; i < ntile; i += kSortThreads) {
            const K k = s_keys[i];
            const int d = digit_of(k, shift);
            const uint32_t o = s_run[d] + (uint32_t)i - s_start[d];
            keys_out[o] = k;
            vals_out[o] = s_vals[i];
        }
        __syncthreads();
        if (threadIdx.x < kRadix) s_run[threadIdx.x] += s_tcnt[threadIdx.x];
        __syncthreads();
    }
}

int sort_grid() { return num_sms() * 2; }

template <typename K>
lgs_status radix_sort_impl(K *keys[2], uint32_t *vals[2], int64_t n_max, const int64_t *d_n64,
                           const int32_t *d_n32, int bits, void *scratch, int *out_buf,
                           cudaStream_t s) {
    if (n_max <= 0) {
        *out_buf = 0;
        return LGS_OK;
    }
    if (n_max > 0xffffffffLL) return LGS_ERR_INVALID_ARG;
    const int G = sort_grid();
    uint32_t *counts = static_cast<uint32_t *>(scratch);
    uint32_t *totals = counts + (size_t)kRadix * G;
    const size_t dyn = (sizeof(K) + sizeof(uint32_t)) * kTile;
    static bool attr_set = false;
    if (!attr_set) {
        cudaFuncSetAttribute(k_radix_downsweep<K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)dyn);
        attr_set = true;
    }
    int cur = 0;
    const int passes = radix_passes(bits);
    for (int p = 0; p < passes; ++p) {
        const int shift = p * 8;
        count_launch();
        k_radix_upsweep<K><<<G, kSortThreads, 0, s>>>(keys[cur], n_max, d_n64, d_n32, shift, counts);
        count_launch();
        k_scan_digit_rows<<<kRadix, (G + 31) / 32 * 32 < 1024 ? (G + 31) / 32 * 32 : 1024, 0, s>>>(
            counts, G, totals);
        count_launch();
        k_radix_downsweep<K><<<G, kSortThreads, dyn, s>>>(keys[cur], vals[cur], keys[cur ^ 1],
                                                       vals[cur ^ 1], counts, totals, n_max, d_n64,
                                                       d_n32, shift);
        cur ^= 1;
    }
    *out_buf = cur;
    return check_launch();
}

// ---------------------------------------------------------------------------
// exclusive scan u32 -> u64 with a device count
// ---------------------------------------------------------------------------
constexpr int kScanThreads = 512;
constexpr int kScanBlocks = 256;

__global__ void __launch_bounds__(kScanThreads) k_scan_reduce(const uint32_t *__restrict__ in,
                                                             int64_t n_max, const int32_t *d_n32,
                                                             uint64_t *__restrict__ partial) {
    __shared__ uint64_t s_tmp[33];
    const int64_t n = read_count(n_max, nullptr, d_n32);
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = per * blockIdx.x, hi = min(lo + per, n);
    uint64_t s = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += kScanThreads) s += in[i];
    uint64_t tot;
    block_exclusive_scan(s, s_tmp, &tot);
    if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_partials(uint64_t *partial, int nb,
                                                               int64_t *d_total) {
    __shared__ uint64_t s_tmp[33];
    uint64_t x = threadIdx.x < nb ? partial[threadIdx.x] : 0;
    uint64_t tot;
    uint64_t ex = block_exclusive_scan(x, s_tmp, &tot);
    if (threadIdx.x < nb) partial[threadIdx.x] = ex;
    if (threadIdx.x == 0 && d_total) *d_total = (int64_t)tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const uint32_t *__restrict__ in,
                                                            uint64_t *__restrict__ out,
                                                            int64_t n_max, const int32_t *d_n32,
                                                            const uint64_t *__restrict__ partial) {
    __shared__ uint64_t s_tmp[33];
    const int64_t n = read_count(n_max, nullptr, d_n32);
    const int64_t per = (n + gridDim.x - 1) / gridDim.x;
    const int64_t lo = per * blockIdx.x, hi = min(lo + per, n);
    uint64_t carry = partial[blockIdx.x];
    for (int64_t base = lo; base < hi; base += kScanThreads) {
        const int64_t i = base + threadIdx.x;
        const uint32_t x = i < hi ? in[i] : 0u;
        uint64_t tot;
        const uint64_t ex = block_exclusive_scan(x, s_tmp, &tot);
        if (i < hi) out[i] = carry + ex;
        carry += tot;
    }
}

}  // namespace

int radix_passes(int bits) { return bits <= 0 ? 1 : (bits + 7) / 8; }

size_t radix_hist_bytes() { return (size_t)kRadix * (sort_grid() + 1) * sizeof(uint32_t); }

size_t radix_sort_workspace(int64_t n, int key_bytes) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    return 2 * al((size_t)n * key_bytes) + 2 * al((size_t)n * 4) + al(radix_hist_bytes());
}

lgs_status radix_sort_u16(uint16_t *keys[2], uint32_t *vals[2], int64_t n_max, const int64_t *d_n64,
                          const int32_t *d_n32, int bits, void *scratch, int *out_buf,
                          cudaStream_t s) {
    if (bits > 16) return LGS_ERR_INVALID_ARG;
    return radix_sort_impl<uint16_t>(keys, vals, n_max, d_n64, d_n32, bits, scratch, out_buf, s);
}
lgs_status radix_sort_u32(uint32_t *keys[2], uint32_t *vals[2], int64_t n_max, const int64_t *d_n64,
                          const int32_t *d_n32, int bits, void *scratch, int *out_buf,
                          cudaStream_t s) {
    if (bits > 32) return LGS_ERR_INVALID_ARG;
    return radix_sort_impl<uint32_t>(keys, vals, n_max, d_n64, d_n32, bits, scratch, out_buf, s);
}
lgs_status radix_sort_u64(uint64_t *keys[2], uint32_t *vals[2], int64_t n_max, const int64_t *d_n64,
                          const int32_t *d_n32, int bits, void *scratch, int *out_buf,
                          cudaStream_t s) {
    if (bits > 64) return LGS_ERR_INVALID_ARG;
    return radix_sort_impl<uint64_t>(keys, vals, n_max, d_n64, d_n32, bits, scratch, out_buf, s);
}

size_t scan_scratch_bytes() { return kScanBlocks * sizeof(uint64_t); }

lgs_status exclusive_scan_u32_to_u64(const uint32_t *in, uint64_t *out, int64_t n_max,
                                     const int32_t *d_n32, int64_t *d_total, void *scratch,
                                     cudaStream_t s) {
    uint64_t *partial = static_cast<uint64_t *>(scratch);
    count_launch();
    k_scan_reduce<<<kScanBlocks, kScanThreads, 0, s>>>(in, n_max, d_n32, partial);
    count_launch();
    k_scan_partials<<<1, kScanThreads, 0, s>>>(partial, kScanBlocks, d_total);
    count_launch();
    k_scan_apply<<<kScanBlocks, kScanThreads, 0, s>>>(in, out, n_max, d_n32, partial);
    return check_launch();
}

}  // namespace lgs
