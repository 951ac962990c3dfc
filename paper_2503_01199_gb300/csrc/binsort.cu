// Tile binning (Sec. 3.1: tile-based rasterisation; Eq. 1: per-tile depth
// order s(i)).
//
// Instead of one sort of 64-bit (tile, depth) keys over all P pairs, the
// splats are first sorted by depth (V 32-bit keys), the pairs are emitted in
// that order, and a stable sort by the tile id alone (ceil(log2 #tiles)
// bits, usually two 8-bit passes of 16-bit keys) groups them per tile. The
// result is identical to the stable (tile, depth) sort: within a tile the
// pairs keep depth order, and equal depths keep increasing splat index.
#include <cuda_runtime.h>

#include "lgs_internal.cuh"

namespace lgs {

__device__ unsigned long long g_overflow_needed = 0;

namespace {

constexpr int kThreads = 256;

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

int tile_bits(int ntiles) {
    int b = 1;
    while ((1ll << b) < ntiles) ++b;
    return b;
}

struct Layout {
    uint32_t *dkeys[2], *dvals[2];
    uint32_t *cnt;
    uint64_t *off;
    uint16_t *tkeys[2];
    uint32_t *tvals_ws;
    void *hist, *scan;
    size_t bytes;
};

Layout layout(void *base, int64_t maxV, int64_t cap) {
    Layout L;
    unsigned char *w = static_cast<unsigned char *>(base);
    auto take = [&](size_t n) {
        unsigned char *p = w;
        w += al256(n);
        return p;
    };
    L.dkeys[0] = reinterpret_cast<uint32_t *>(take((size_t)maxV * 4));
    L.dkeys[1] = reinterpret_cast<uint32_t *>(take((size_t)maxV * 4));
    L.dvals[0] = reinterpret_cast<uint32_t *>(take((size_t)maxV * 4));
    L.dvals[1] = reinterpret_cast<uint32_t *>(take((size_t)maxV * 4));
    L.cnt = reinterpret_cast<uint32_t *>(take((size_t)maxV * 4));
    L.off = reinterpret_cast<uint64_t *>(take((size_t)maxV * 8));
    L.tkeys[0] = reinterpret_cast<uint16_t *>(take((size_t)cap * 2));
    L.tkeys[1] = reinterpret_cast<uint16_t *>(take((size_t)cap * 2));
    L.tvals_ws = reinterpret_cast<uint32_t *>(take((size_t)cap * 4));
    L.hist = take(radix_hist_bytes());
    L.scan = take(scan_scratch_bytes());
    L.bytes = (size_t)(w - static_cast<unsigned char *>(base));
    return L;
}

__global__ void __launch_bounds__(kThreads) k_depth_keys(const float *__restrict__ depth,
                                                        const int32_t *__restrict__ radius,
                                                        int64_t maxV, const int32_t *d_V,
                                                        uint32_t *__restrict__ keys,
                                                        uint32_t *__restrict__ vals) {
    const int64_t V = load_count(d_V, maxV);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < V;
         j += (int64_t)gridDim.x * blockDim.x) {
        // depth > znear > 0, so the float bits order like the values; culled
        // splats go last
        keys[j] = radius[j] > 0 ? __float_as_uint(depth[j]) : 0xffffffffu;
        vals[j] = (uint32_t)j;
    }
}

__global__ void __launch_bounds__(kThreads) k_tile_counts(const float *__restrict__ rec,
                                                         const int32_t *__restrict__ radius,
                                                         const uint32_t *__restrict__ order,
                                                         int64_t maxV, const int32_t *d_V, int tw,
                                                         int th, int gx, int gy,
                                                         uint32_t *__restrict__ cnt) {
    const int64_t V = load_count(d_V, maxV);
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < V;
         r += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t g = order[r];
        uint32_t c = 0;
        const int rad = radius[g];
        if (rad > 0) {
            const float2 uv = *reinterpret_cast<const float2 *>(rec + 12 * (int64_t)g);
            const int4 rc = tile_rect(uv.x, uv.y, (float)rad, tw, th, gx, gy);
            if (rc.z > rc.x && rc.w > rc.y) c = (uint32_t)((rc.z - rc.x) * (rc.w - rc.y));
        }
        cnt[r] = c;
    }
}

__global__ void k_check_capacity(const int64_t *d_P, int64_t cap) {
    const int64_t P = *d_P;
    if (P > cap) atomicMax(&g_overflow_needed, (unsigned long long)P);
}

// Emit the pairs of 32 consecutive depth-ordered splats per warp, with the
// warp writing consecutive output positions together.
__global__ void __launch_bounds__(kThreads) k_duplicate(const float *__restrict__ rec,
                                                       const int32_t *__restrict__ radius,
                                                       const uint32_t *__restrict__ order,
                                                       const uint64_t *__restrict__ off,
                                                       int64_t maxV, const int32_t *d_V, int tw,
                                                       int th, int gx, int gy, int64_t cap,
                                                       uint16_t *__restrict__ tkeys,
                                                       uint32_t *__restrict__ tvals) {
    const int64_t V = load_count(d_V, maxV);
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = ((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5) * 32; base < V;
         base += nwarps * 32) {
        const int64_t r = base + lane;
        uint32_t g = 0;
        int4 rc = make_int4(0, 0, 0, 0);
        uint64_t o = 0;
        int c = 0;
        if (r < V) {
            g = order[r];
            o = off[r];
            const int rad = radius[g];
            if (rad > 0) {
                const float2 uv = *reinterpret_cast<const float2 *>(rec + 12 * (int64_t)g);
                rc = tile_rect(uv.x, uv.y, (float)rad, tw, th, gx, gy);
                if (rc.z > rc.x && rc.w > rc.y) c = (rc.z - rc.x) * (rc.w - rc.y);
            }
        }
        // warp-cooperative expansion of positions [o_first, o_last): lane ends
        // are non-decreasing (lanes past V get +inf), so the owner of a
        // position is the number of lanes whose end is <= it
        const uint64_t my_end = r < V ? o + (uint64_t)c : ~0ull;
        uint64_t o_last = r < V ? my_end : 0ull;
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) {
            const uint64_t y = __shfl_xor_sync(0xffffffffu, o_last, sh);
            o_last = y > o_last ? y : o_last;
        }
        const uint64_t o_first = __shfl_sync(0xffffffffu, o, 0);
        for (uint64_t p0 = o_first; p0 < o_last; p0 += 32) {
            const uint64_t p = p0 + lane;
            int lo = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                const uint64_t e = __shfl_sync(0xffffffffu, my_end, lo + step - 1);
                if (p >= e) lo += step;
            }
            const int src = lo < 31 ? lo : 31;
            const int sx0 = __shfl_sync(0xffffffffu, rc.x, src);
            const int sy0 = __shfl_sync(0xffffffffu, rc.y, src);
            const int sx1 = __shfl_sync(0xffffffffu, rc.z, src);
            const uint64_t so = __shfl_sync(0xffffffffu, o, src);
            const uint32_t sg = __shfl_sync(0xffffffffu, g, src);
            if (p < o_last && p < (uint64_t)cap) {
                const int w = sx1 - sx0;
                const int k = (int)(p - so);
                const int ty = sy0 + k / w, tx = sx0 + k % w;
                tkeys[p] = (uint16_t)(ty * gx + tx);
                tvals[p] = sg;
            }
        }
    }
}

__global__ void __launch_bounds__(kThreads) k_tile_ranges(const uint16_t *__restrict__ keys,
                                                         const int64_t *d_P, int64_t cap,
                                                         uint32_t *__restrict__ ranges) {
    const int64_t P = min(*d_P, cap);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        if (i == 0 || keys[i - 1] != k) ranges[2 * k] = (uint32_t)i;
        if (i == P - 1 || keys[i + 1] != k) ranges[2 * k + 1] = (uint32_t)(i + 1);
    }
}

}  // namespace

size_t bin_sort_workspace_size(int64_t maxV, int64_t cap, int ntiles) {
    (void)ntiles;
    return layout(nullptr, maxV, cap).bytes + 256;
}

lgs_status bin_sort(const lgs_splats *sp, const int32_t *d_V, int64_t maxV, const lgs_camera *cam,
                    int tw, int th, uint32_t *vals, int64_t cap, int64_t *d_P, uint32_t *ranges,
                    void *ws, cudaStream_t s) {
    const int gx = (int)ceil_div(cam->width, tw), gy = (int)ceil_div(cam->height, th);
    const int ntiles = gx * gy;
    if (ntiles > 65536) return LGS_ERR_INVALID_ARG;
    Layout L = layout(ws, maxV, cap);
    // 1. depth sort of the splats
    count_launch();
    k_depth_keys<<<grid_for(maxV, kThreads), kThreads, 0, s>>>(sp->depth, sp->radius, maxV, d_V,
                                                              L.dkeys[0], L.dvals[0]);
    lgs_status st = check_launch();
    if (st != LGS_OK) return st;
    int ob = 0;
    st = radix_sort_u32(L.dkeys, L.dvals, maxV, nullptr, d_V, 32, L.hist, &ob, s);
    if (st != LGS_OK) return st;
    const uint32_t *order = L.dvals[ob];
    // 2. pairs per splat in depth order, offsets, total
    count_launch();
    k_tile_counts<<<grid_for(maxV, kThreads), kThreads, 0, s>>>(sp->rec, sp->radius, order, maxV,
                                                               d_V, tw, th, gx, gy, L.cnt);
    st = exclusive_scan_u32_to_u64(L.cnt, L.off, maxV, d_V, d_P, L.scan, s);
    if (st != LGS_OK) return st;
    count_launch();
    k_check_capacity<<<1, 1, 0, s>>>(d_P, cap);
    // 3. emit pairs; pick the start buffer so the last pass lands in `vals`
    const int bits = tile_bits(ntiles);
    const int passes = radix_passes(bits);
    uint32_t *tv[2];
    if (passes % 2 == 0) { tv[0] = vals; tv[1] = L.tvals_ws; }
    else { tv[0] = L.tvals_ws; tv[1] = vals; }
    count_launch();
    k_duplicate<<<grid_for(maxV, kThreads), kThreads, 0, s>>>(sp->rec, sp->radius, order, L.off,
                                                             maxV, d_V, tw, th, gx, gy, cap,
                                                             L.tkeys[0], tv[0]);
    st = check_launch();
    if (st != LGS_OK) return st;
    // 4. stable sort by tile id
    st = radix_sort_u16(L.tkeys, tv, cap, d_P, nullptr, bits, L.hist, &ob, s);
    if (st != LGS_OK) return st;
    // 5. ranges
    cudaMemsetAsync(ranges, 0, (size_t)ntiles * 2 * sizeof(uint32_t), s);
    count_launch();
    k_tile_ranges<<<grid_for(cap, kThreads), kThreads, 0, s>>>(L.tkeys[ob], d_P, cap, ranges);
    return check_launch();
}

lgs_status get_overflow(int64_t *needed) {
    unsigned long long v = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&v, g_overflow_needed, sizeof(v));
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return LGS_ERR_CUDA;
    }
    if (needed) *needed = (int64_t)v;
    if (v) {
        unsigned long long z = 0;
        cudaMemcpyToSymbol(g_overflow_needed, &z, sizeof(z));
        return LGS_ERR_CAPACITY;
    }
    return LGS_OK;
}

}  // namespace lgs
