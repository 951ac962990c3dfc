// Stable LSD radix sort of (key, value) pairs (u32 or u64 values) and an
// exclusive scan,
// both with the element count read on the device, so that they can sit in a
// captured CUDA graph behind kernels that produce the count.
//
// Radix sort, one 8-bit digit per pass, "onesweep" with decoupled look-back:
//   histogram - one read of the keys counts the digits of every pass (and
//               clears the first pass's tile status; each pass clears the
//               next one's);
//   per pass  - CTAs take 4096-item tiles in launch order from an atomic
//               counter, rank each tile's items stably with a warp
//               multisplit (peer masks from per-bit ballots), publish the
//               tile's per-digit counts, and obtain the exclusive prefix of
//               each digit over earlier tiles by looking back at their
//               published counts (a tile that has its own prefix publishes
//               it, so look-backs stop early); then the tile is staged in
//               shared memory in local digit order and written out.
// A tile only waits on tiles handed out before it, whose CTAs are resident
// or finished, so the look-back always progresses; it is still bounded, and
// a wait that gives up is counted (lgs_get_wait_timeouts) instead of hanging.
// Output positions depend on tile indices only, and ranks are stable inside
// a tile, so every pass is stable.
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

constexpr uint32_t kFlagAgg = 1u << 30;   // tile's own counts published
constexpr uint32_t kFlagPre = 2u << 30;   // inclusive prefix over tiles <= t published
constexpr uint32_t kCountMask = (1u << 30) - 1u;
constexpr int kMaxPasses = 8;

__device__ unsigned int g_sort_wait_timeouts;
// polls of an unpublished predecessor before a look-back gives up
__device__ uint32_t g_sort_spin_limit = kDefaultSpinLimit;

// Digit counts of every pass in one read of the keys (hist zeroed).
// Also clears the tile status words and the tile counter of the first pass.
template <typename K>
__global__ void __launch_bounds__(kSortThreads) k_digit_hist(const K *__restrict__ keys,
                                                            int64_t n_max, const int64_t *d_n64,
                                                            const int32_t *d_n32, int passes,
                                                            uint32_t *__restrict__ hist,
                                                            uint32_t *__restrict__ status0,
                                                            uint32_t *__restrict__ counter0) {
    __shared__ uint32_t s_h[kMaxPasses][kRadix];
    for (int i = threadIdx.x; i < kMaxPasses * kRadix; i += kSortThreads) (&s_h[0][0])[i] = 0;
    __syncthreads();
    const int64_t n = read_count(n_max, d_n64, d_n32);
    const int64_t words = (n + kTile - 1) / kTile * kRadix;
    for (int64_t i = blockIdx.x * (int64_t)kSortThreads + threadIdx.x; i < words;
         i += (int64_t)gridDim.x * kSortThreads)
        status0[i] = 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) *counter0 = 0u;
    for (int64_t i = blockIdx.x * (int64_t)kSortThreads + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * kSortThreads) {
        const K k = keys[i];
        for (int p = 0; p < passes; ++p) atomicAdd(&s_h[p][digit_of(k, 8 * p)], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadix; i += kSortThreads) {
        const uint32_t c = (&s_h[0][0])[i];
        if (c) atomicAdd(hist + i, c);
    }
}

template <typename K, typename V>
__global__ void __launch_bounds__(kSortThreads, 2) k_onesweep(
    const K *__restrict__ keys_in, const V *__restrict__ vals_in, K *__restrict__ keys_out,
    V *__restrict__ vals_out, const uint32_t *__restrict__ hist, uint32_t *status,
    uint32_t *counter, uint32_t *next_status, uint32_t *next_counter, int64_t n_max,
    const int64_t *d_n64, const int32_t *d_n32, int shift) {
    __shared__ uint32_t s_wcnt[kSortWarps][kRadix];
    __shared__ uint32_t s_gstart[kRadix];
    __shared__ uint32_t s_start[kRadix];
    __shared__ uint32_t s_base[kRadix];
    __shared__ uint64_t s_scan[33];
    __shared__ uint32_t s_tile;
    extern __shared__ __align__(16) unsigned char s_dyn[];
    V *s_vals = reinterpret_cast<V *>(s_dyn);
    K *s_keys = reinterpret_cast<K *>(s_dyn + sizeof(V) * kTile);

    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t n = read_count(n_max, d_n64, d_n32);
    const int64_t tiles = (n + kTile - 1) / kTile;
    if (next_status) {
        // the next pass's status words (its region was last used by the
        // previous pass, which has finished)
        for (int64_t i = blockIdx.x * (int64_t)kSortThreads + threadIdx.x; i < tiles * kRadix;
             i += (int64_t)gridDim.x * kSortThreads)
            next_status[i] = 0u;
        if (blockIdx.x == 0 && threadIdx.x == 0) *next_counter = 0u;
    }
    {
        // global start of each digit
        const uint64_t h = threadIdx.x < kRadix ? hist[threadIdx.x] : 0u;
        const uint64_t st = block_exclusive_scan(h, s_scan, nullptr);
        if (threadIdx.x < kRadix) s_gstart[threadIdx.x] = (uint32_t)st;
    }
    const uint32_t lt = lanemask_lt();
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
        for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) (&s_wcnt[0][0])[i] = 0;
        __syncthreads();
        const int64_t tile = s_tile;
        if (tile >= tiles) break;
        const int64_t base = tile * kTile;
        K key[kItemsPerThread];
        V val[kItemsPerThread];
        uint32_t rank[kItemsPerThread];
        int dig[kItemsPerThread];
#pragma unroll
        for (int j = 0; j < kItemsPerThread; ++j) {
            const int64_t idx = base + wid * (kWarp * kItemsPerThread) + j * kWarp + lane;
            const bool ok = idx < n;
            key[j] = ok ? keys_in[idx] : (K)0;
            val[j] = ok ? vals_in[idx] : (V)0;
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
        // per digit: exclusive scan over warps (the tile's count in tcnt)
        uint32_t tcnt = 0;
        if (threadIdx.x < kRadix) {
            const int d = threadIdx.x;
            for (int w = 0; w < kSortWarps; ++w) {
                const uint32_t c = s_wcnt[w][d];
                s_wcnt[w][d] = tcnt;
                tcnt += c;
            }
        }
        const uint64_t st = block_exclusive_scan(threadIdx.x < kRadix ? tcnt : 0u, s_scan, nullptr);
        if (threadIdx.x < kRadix) {
            const int d = threadIdx.x;
            s_start[d] = (uint32_t)st;
            volatile uint32_t *mine = status + tile * kRadix + d;
            uint32_t excl = 0;
            if (tile == 0) {
                *mine = kFlagPre | tcnt;
            } else {
                *mine = kFlagAgg | tcnt;
                int64_t k = tile - 1;
                uint32_t spins = 0;
                for (;;) {
                    const uint32_t w = *(volatile const uint32_t *)(status + k * kRadix + d);
                    const uint32_t fl = w & ~kCountMask;
                    if (fl == 0u) {
                        if (++spins > g_sort_spin_limit) {
                            atomicAdd(&g_sort_wait_timeouts, 1u);
                            break;
                        }
                        __nanosleep(32);
                        continue;
                    }
                    excl += w & kCountMask;
                    if (fl == kFlagPre || k == 0) break;
                    --k;
                }
                *mine = kFlagPre | ((excl + tcnt) & kCountMask);
            }
            s_base[d] = s_gstart[d] + excl;
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
            const uint32_t o = s_base[d] + (uint32_t)i - s_start[d];
            if (LGS_DCHECK((int64_t)o < n, kSiteSortScatter)) {
                keys_out[o] = k;
                vals_out[o] = s_vals[i];
            }
        }
        __syncthreads();
    }
}

int64_t sort_tiles(int64_t n_max) { return (n_max + kTile - 1) / kTile; }

template <typename K, typename V>
lgs_status radix_sort_impl(K *keys[2], V *vals[2], int64_t n_max, const int64_t *d_n64,
                           const int32_t *d_n32, int bits, void *scratch, int *out_buf,
                           cudaStream_t s) {
    if (n_max <= 0) {
        *out_buf = 0;
        return LGS_OK;
    }
    if (n_max > (int64_t)kCountMask) return LGS_ERR_INVALID_ARG;
    const int passes = radix_passes(bits);
    if (passes > kMaxPasses) return LGS_ERR_INVALID_ARG;
    // scratch: digit counts [kMaxPasses][256], two tile counters, and two
    // status regions [tiles][256] used by alternate passes, so that each pass
    // clears the region of the next one
    const int64_t tmax = sort_tiles(n_max);
    uint32_t *hist = static_cast<uint32_t *>(scratch);
    uint32_t *counter[2] = {hist + kMaxPasses * kRadix, hist + kMaxPasses * kRadix + 32};
    uint32_t *status[2] = {hist + kMaxPasses * kRadix + 64,
                           hist + kMaxPasses * kRadix + 64 + tmax * kRadix};
    const size_t dyn = (sizeof(K) + sizeof(V)) * kTile;
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        cudaFuncSetAttribute(k_onesweep<K, V>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)dyn);
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_onesweep<K, V>, kSortThreads, dyn);
    const int64_t cap = (int64_t)num_sms() * (per_sm > 0 ? per_sm : 1);
    const unsigned grid = (unsigned)(tmax < cap ? tmax : cap);
    cudaMemsetAsync(hist, 0, sizeof(uint32_t) * kRadix * passes, s);
    count_launch();
    k_digit_hist<K><<<grid_for(n_max, kSortThreads, 4), kSortThreads, 0, s>>>(
        keys[0], n_max, d_n64, d_n32, passes, hist, status[0], counter[0]);
    int cur = 0;
    for (int p = 0; p < passes; ++p) {
        const int q = p & 1;
        const bool more = p + 1 < passes;
        count_launch();
        k_onesweep<K, V><<<grid, kSortThreads, dyn, s>>>(
            keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], hist + p * kRadix, status[q],
            counter[q], more ? status[q ^ 1] : nullptr, more ? counter[q ^ 1] : nullptr, n_max,
            d_n64, d_n32, p * 8);
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

size_t radix_hist_bytes(int64_t n_max) {
    return sizeof(uint32_t) * ((size_t)kMaxPasses * kRadix + 64 +
                               2 * (size_t)sort_tiles(n_max > 0 ? n_max : 1) * kRadix);
}

DEBUG_TU(sort)

lgs_status sort_set_spin_limit(uint32_t spins) {
    if (cudaMemcpyToSymbol(g_sort_spin_limit, &spins, sizeof(spins)) != cudaSuccess) {
        set_cuda_error(cudaGetLastError());
        return LGS_ERR_CUDA;
    }
    return LGS_OK;
}

lgs_status sort_wait_timeouts(uint32_t *count) {
    unsigned int h = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&h, g_sort_wait_timeouts, sizeof(h)) != cudaSuccess ||
        cudaMemcpyToSymbol(g_sort_wait_timeouts, &zero, sizeof(zero)) != cudaSuccess) {
        set_cuda_error(cudaGetLastError());
        return LGS_ERR_CUDA;
    }
    *count = h;
    return h ? LGS_ERR_TIMEOUT : LGS_OK;
}

size_t radix_sort_workspace(int64_t n, int key_bytes) {
    auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
    return 2 * al((size_t)n * key_bytes) + 2 * al((size_t)n * 4) + al(radix_hist_bytes(n));
}

lgs_status radix_sort_u16_v64(uint16_t *keys[2], uint64_t *vals[2], int64_t n_max,
                              const int64_t *d_n64, const int32_t *d_n32, int bits, void *scratch,
                              int *out_buf, cudaStream_t s) {
    if (bits > 16) return LGS_ERR_INVALID_ARG;
    return radix_sort_impl<uint16_t, uint64_t>(keys, vals, n_max, d_n64, d_n32, bits, scratch,
                                               out_buf, s);
}
lgs_status radix_sort_u32(uint32_t *keys[2], uint32_t *vals[2], int64_t n_max, const int64_t *d_n64,
                          const int32_t *d_n32, int bits, void *scratch, int *out_buf,
                          cudaStream_t s) {
    if (bits > 32) return LGS_ERR_INVALID_ARG;
    return radix_sort_impl<uint32_t, uint32_t>(keys, vals, n_max, d_n64, d_n32, bits, scratch,
                                               out_buf, s);
}
lgs_status radix_sort_u64(uint64_t *keys[2], uint32_t *vals[2], int64_t n_max, const int64_t *d_n64,
                          const int32_t *d_n32, int bits, void *scratch, int *out_buf,
                          cudaStream_t s) {
    if (bits > 64) return LGS_ERR_INVALID_ARG;
    return radix_sort_impl<uint64_t, uint32_t>(keys, vals, n_max, d_n64, d_n32, bits, scratch,
                                               out_buf, s);
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
