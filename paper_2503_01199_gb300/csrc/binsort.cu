// Tile binning (Sec. 3.1: tile-based rasterisation; Eq. 1: per-tile depth
// order s(i)), with the tile-level culling of App. A.1: tiles of a splat's
// rectangle where no pixel centre can reach alpha >= 1/255 are not listed.
//
// Result: for every tile, the splats listed in it in increasing depth, equal
// depths in increasing splat index -- the order of a stable sort of the key
// (tile << 32 | depth bits) -- as vals[ranges[t].x .. ranges[t].y).
//
// Two levels instead of one sort over all (tile, splat) pairs:
//   1. the splats are sorted by depth (32-bit keys);
//   2. each splat is binned into the super-tiles (8 x 4 tiles) its rectangle
//      meets, in depth order, and the (super-tile, splat) items are sorted
//      stably by super-tile (one 8-bit pass for up to 256 super-tiles);
//   3. each super-tile's items, in chunks of 1024, get a 32-bit mask of the
//      tiles they are listed in (rectangle and culling test per tile); one
//      ballot per tile per warp gives every item its rank among the earlier
//      items of the chunk listed in the same tile, so each tile's list is
//      written in depth order without sorting the pairs themselves.
// Tiles' lists are laid out super-tile by super-tile, tile by tile.
#include <cuda_runtime.h>

#include "lgs_internal.cuh"

namespace lgs {

__device__ unsigned long long g_overflow_needed = 0;

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kSX = 8, kSY = 4;   // super-tile = 8 x 4 tiles, one bit per tile
constexpr int kChunk = 1024;      // items of one super-tile per expansion chunk

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

int bits_for(int n) {
    int b = 1;
    while ((1ll << b) < n) ++b;
    return b;
}

struct Geo {
    int tw, th, gx, gy, sgx, sgy, ns;
};

Geo make_geo(const lgs_camera *cam, int tw, int th) {
    Geo g;
    g.tw = tw;
    g.th = th;
    g.gx = (int)ceil_div(cam->width, tw);
    g.gy = (int)ceil_div(cam->height, th);
    g.sgx = (int)ceil_div(g.gx, kSX);
    g.sgy = (int)ceil_div(g.gy, kSY);
    g.ns = g.sgx * g.sgy;
    return g;
}

int64_t max_chunks(int ns, int64_t cap) { return ns + ceil_div(cap, kChunk); }

struct Layout {
    uint32_t *dkeys[2], *dvals[2];
    uint32_t *scnt;
    uint64_t *soff;
    uint16_t *skeys[2];
    uint32_t *svals[2];
    uint32_t *masks;
    uint32_t *seg;        // [ns][2]
    uint32_t *cbase;      // [ns + 1]
    uint32_t *ccount;     // [max_chunks][32]
    uint32_t *tstart;     // [ns * 32]
    uint32_t *ttotal;     // [ns * 32]
    int64_t *d_psup;
    void *hist, *scan;
    size_t bytes;
};

Layout layout(void *base, int64_t maxV, int64_t cap, int ns) {
    Layout L;
    unsigned char *w = static_cast<unsigned char *>(base);
    auto take = [&](size_t n) {
        unsigned char *p = w;
        w += al256(n);
        return p;
    };
    for (int k = 0; k < 2; ++k) L.dkeys[k] = reinterpret_cast<uint32_t *>(take((size_t)maxV * 4));
    for (int k = 0; k < 2; ++k) L.dvals[k] = reinterpret_cast<uint32_t *>(take((size_t)maxV * 4));
    L.scnt = reinterpret_cast<uint32_t *>(take((size_t)maxV * 4));
    L.soff = reinterpret_cast<uint64_t *>(take((size_t)maxV * 8));
    for (int k = 0; k < 2; ++k) L.skeys[k] = reinterpret_cast<uint16_t *>(take((size_t)cap * 2));
    for (int k = 0; k < 2; ++k) L.svals[k] = reinterpret_cast<uint32_t *>(take((size_t)cap * 4));
    L.masks = reinterpret_cast<uint32_t *>(take((size_t)cap * 4));
    L.seg = reinterpret_cast<uint32_t *>(take((size_t)ns * 8));
    L.cbase = reinterpret_cast<uint32_t *>(take((size_t)(ns + 1) * 4));
    L.ccount = reinterpret_cast<uint32_t *>(take((size_t)max_chunks(ns, cap) * 32 * 4));
    L.tstart = reinterpret_cast<uint32_t *>(take((size_t)ns * 32 * 4));
    L.ttotal = reinterpret_cast<uint32_t *>(take((size_t)ns * 32 * 4));
    L.d_psup = reinterpret_cast<int64_t *>(take(8));
    L.hist = take(radix_hist_bytes(maxV > cap ? maxV : cap));
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

struct SplatGeom {
    int4 rc;        // tile rectangle (empty: culled)
    float u, v, A, B, C, rA, rC, tau;
};

__device__ __forceinline__ SplatGeom splat_geom(const float *__restrict__ rec,
                                                const int32_t *__restrict__ radius, uint32_t g,
                                                const Geo &G) {
    SplatGeom s;
    s.rc = make_int4(0, 0, 0, 0);
    s.u = s.v = s.A = s.B = s.C = s.rA = s.rC = s.tau = 0.f;
    const int rad = radius[g];
    if (rad > 0) {
        const float4 *p = reinterpret_cast<const float4 *>(rec + 12 * (int64_t)g);
        const float4 a = p[0];
        s.u = a.x; s.v = a.y; s.A = a.z; s.B = a.w;
        s.C = p[1].x;
        s.tau = p[2].y;
        s.rA = __frcp_rn(s.A);
        s.rC = __frcp_rn(s.C);
        s.rc = tile_rect(a.x, a.y, (float)rad, G.tw, G.th, G.gx, G.gy);
        if (s.rc.z <= s.rc.x || s.rc.w <= s.rc.y) s.rc = make_int4(0, 0, 0, 0);
    }
    return s;
}

// Stage 2: the super-tiles of each splat (depth order r), one thread per
// splat. A super-tile is kept when the box of pixel centres of the
// rectangle's tiles inside it passes the culling test with tau widened once
// more by 1e-3 (1 + |tau|), so that it never drops a super-tile holding a
// tile the per-tile test keeps.
template <bool kEmit>
__global__ void __launch_bounds__(kThreads) k_super_walk(const float *__restrict__ rec,
                                                        const int32_t *__restrict__ radius,
                                                        const uint32_t *__restrict__ order,
                                                        int64_t maxV, const int32_t *d_V, Geo G,
                                                        int cull, uint32_t *__restrict__ cnt,
                                                        const uint64_t *__restrict__ off,
                                                        int64_t cap, uint16_t *__restrict__ skeys,
                                                        uint32_t *__restrict__ svals) {
    const int64_t V = load_count(d_V, maxV);
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < V;
         r += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t g = order[r];
        const SplatGeom sg = splat_geom(rec, radius, g, G);
        uint64_t o = kEmit ? off[r] : 0ull;
        uint32_t n = 0;
        if (sg.rc.z > sg.rc.x) {
            const int sx0 = sg.rc.x / kSX, sx1 = (sg.rc.z - 1) / kSX + 1;
            const int sy0 = sg.rc.y / kSY, sy1 = (sg.rc.w - 1) / kSY + 1;
            const float tw_ = __fmaf_rn(1e-3f, 1.0f + fabsf(sg.tau), sg.tau);
            for (int sy = sy0; sy < sy1; ++sy)
                for (int sx = sx0; sx < sx1; ++sx) {
                    bool keep = true;
                    if (cull) {
                        const int tx0 = max(sg.rc.x, sx * kSX), tx1 = min(sg.rc.z, sx * kSX + kSX);
                        const int ty0 = max(sg.rc.y, sy * kSY), ty1 = min(sg.rc.w, sy * kSY + kSY);
                        keep = box_reachable(sg.u, sg.v, sg.A, sg.B, sg.C, sg.rA, sg.rC, tw_,
                                             (float)(tx0 * G.tw) + 0.5f, (float)(tx1 * G.tw) - 0.5f,
                                             (float)(ty0 * G.th) + 0.5f, (float)(ty1 * G.th) - 0.5f);
                    }
                    if (!keep) continue;
                    if (kEmit) {
                        if (o < (uint64_t)cap) {
                            skeys[o] = (uint16_t)(sy * G.sgx + sx);
                            svals[o] = g;
                        }
                        ++o;
                    } else {
                        ++n;
                    }
                }
        }
        if (!kEmit) cnt[r] = n;
    }
}

__global__ void k_check_super_capacity(const int64_t *d_psup, int64_t cap) {
    if (*d_psup > cap) atomicMax(&g_overflow_needed, (unsigned long long)*d_psup);
}

// Item range [start, end) of every super-tile in the sorted items.
__global__ void __launch_bounds__(kThreads) k_seg_ranges(const uint16_t *__restrict__ keys,
                                                        const int64_t *d_psup, int64_t cap,
                                                        uint32_t *__restrict__ seg) {
    const int64_t P = min(*d_psup, cap);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < P;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = keys[i];
        if (i == 0 || keys[i - 1] != k) seg[2 * k] = (uint32_t)i;
        if (i == P - 1 || keys[i + 1] != k) seg[2 * k + 1] = (uint32_t)(i + 1);
    }
}

// Chunks of every super-tile: cbase[s] = first chunk of s, cbase[ns] = total.
__global__ void __launch_bounds__(1024) k_chunk_plan(const uint32_t *__restrict__ seg, int ns,
                                                    uint32_t *__restrict__ cbase) {
    __shared__ uint32_t s_sum[1024];
    const int per = (ns + 1023) / 1024;
    const int s0 = threadIdx.x * per;
    uint32_t tot = 0;
    for (int s = s0; s < min(ns, s0 + per); ++s)
        tot += (seg[2 * s + 1] - seg[2 * s] + kChunk - 1) / kChunk;
    s_sum[threadIdx.x] = tot;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const uint32_t x = threadIdx.x >= o ? s_sum[threadIdx.x - o] : 0u;
        __syncthreads();
        s_sum[threadIdx.x] += x;
        __syncthreads();
    }
    uint32_t run = s_sum[threadIdx.x] - tot;
    for (int s = s0; s < min(ns, s0 + per); ++s) {
        cbase[s] = run;
        run += (seg[2 * s + 1] - seg[2 * s] + kChunk - 1) / kChunk;
    }
    if (threadIdx.x == 1023) cbase[ns] = s_sum[1023];
}

// super-tile of chunk k: the last s with cbase[s] <= k
__device__ __forceinline__ int chunk_super(const uint32_t *__restrict__ cbase, int ns, uint32_t k) {
    int lo = 0, hi = ns - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cbase[mid] <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Stage 3a: tile mask of every item (the tiles of its rectangle inside its
// super-tile that pass the per-tile culling test) and per-chunk counts per
// tile. One CTA per chunk.
__global__ void __launch_bounds__(kThreads) k_chunk_masks(const float *__restrict__ rec,
                                                         const int32_t *__restrict__ radius,
                                                         const uint32_t *__restrict__ svals,
                                                         const uint32_t *__restrict__ seg,
                                                         const uint32_t *__restrict__ cbase, Geo G,
                                                         int cull, uint32_t *__restrict__ masks,
                                                         uint32_t *__restrict__ ccount) {
    __shared__ uint32_t s_cnt[kWarps][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t K = cbase[G.ns];
    for (uint32_t k = blockIdx.x; k < K; k += gridDim.x) {
        const int s = chunk_super(cbase, G.ns, k);
        const uint32_t a = seg[2 * s] + (k - cbase[s]) * kChunk;
        const uint32_t b = min(a + (uint32_t)kChunk, seg[2 * s + 1]);
        const int sx = s % G.sgx, sy = s / G.sgx;
        uint32_t my = 0;  // this warp's count for tile `lane`
        for (uint32_t i0 = a; i0 < b; i0 += kThreads) {
            const uint32_t i = i0 + threadIdx.x;
            uint32_t mask = 0;
            if (i < b) {
                const SplatGeom sg = splat_geom(rec, radius, svals[i], G);
                const int tx0 = max(sg.rc.x, sx * kSX), tx1 = min(sg.rc.z, sx * kSX + kSX);
                const int ty0 = max(sg.rc.y, sy * kSY), ty1 = min(sg.rc.w, sy * kSY + kSY);
                const RowCull rcl = row_cull(sg.u, sg.v, sg.A, sg.B, sg.C, sg.rA, sg.rC, sg.tau);
                for (int ty = ty0; ty < ty1; ++ty) {
                    const uint32_t rowbit = (uint32_t)(ty - sy * kSY) * kSX - sx * kSX;
                    if (!cull) {
                        for (int tx = tx0; tx < tx1; ++tx) mask |= 1u << (rowbit + tx);
                    } else if (rcl.degenerate) {
                        for (int tx = tx0; tx < tx1; ++tx)
                            if (tile_reachable(sg.u, sg.v, sg.A, sg.B, sg.C, sg.rA, sg.rC, sg.tau,
                                               tx, ty, G.tw, G.th))
                                mask |= 1u << (rowbit + tx);
                    } else {
                        float L, U;
                        if (!row_interval(rcl, ty, G.th, L, U)) continue;
                        for (int tx = tx0; tx < tx1; ++tx)
                            if (tile_in_row(rcl, tx, G.tw, L, U)) mask |= 1u << (rowbit + tx);
                    }
                }
                masks[i] = mask;
            }
#pragma unroll
            for (int l = 0; l < 32; ++l) {
                const uint32_t m = __ballot_sync(0xffffffffu, (mask >> l) & 1u);
                if (lane == l) my += __popc(m);
            }
        }
        s_cnt[wid][lane] = my;
        __syncthreads();
        if (threadIdx.x < 32) {
            uint32_t t = 0;
            for (int w = 0; w < kWarps; ++w) t += s_cnt[w][threadIdx.x];
            ccount[(size_t)k * 32 + threadIdx.x] = t;
        }
        __syncthreads();
    }
}

// Stage 3b: per super-tile and tile, exclusive offsets of the chunks (in
// place) and the tile's total. One warp per super-tile, lane = tile.
__global__ void __launch_bounds__(kThreads) k_chunk_offsets(uint32_t *__restrict__ ccount,
                                                           const uint32_t *__restrict__ cbase,
                                                           int ns, uint32_t *__restrict__ ttotal) {
    const int lane = threadIdx.x & 31;
    for (int s = (blockIdx.x * kThreads + threadIdx.x) >> 5; s < ns;
         s += (gridDim.x * kThreads) >> 5) {
        uint32_t run = 0;
        for (uint32_t k = cbase[s]; k < cbase[s + 1]; ++k) {
            const uint32_t c = ccount[(size_t)k * 32 + lane];
            ccount[(size_t)k * 32 + lane] = run;
            run += c;
        }
        ttotal[s * 32 + lane] = run;
    }
}

// Stage 3c: tile starts (exclusive scan over super-tiles, then tiles), the
// ranges of every tile and the pair total. One CTA.
__global__ void __launch_bounds__(1024) k_tile_starts(const uint32_t *__restrict__ ttotal, Geo G,
                                                     uint32_t *__restrict__ tstart,
                                                     uint32_t *__restrict__ ranges, int64_t *d_P,
                                                     int64_t cap) {
    __shared__ uint64_t s_sum[1024];
    const int n = G.ns * 32;
    const int per = (n + 1023) / 1024;
    const int i0 = threadIdx.x * per;
    uint64_t tot = 0;
    for (int i = i0; i < min(n, i0 + per); ++i) tot += ttotal[i];
    s_sum[threadIdx.x] = tot;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const uint64_t x = threadIdx.x >= o ? s_sum[threadIdx.x - o] : 0ull;
        __syncthreads();
        s_sum[threadIdx.x] += x;
        __syncthreads();
    }
    uint64_t run = s_sum[threadIdx.x] - tot;
    for (int i = i0; i < min(n, i0 + per); ++i) {
        tstart[i] = (uint32_t)min(run, (uint64_t)cap);
        const int s = i >> 5, l = i & 31;
        const int tx = (s % G.sgx) * kSX + (l % kSX), ty = (s / G.sgx) * kSY + (l / kSX);
        if (tx < G.gx && ty < G.gy) {
            const int t = ty * G.gx + tx;
            ranges[2 * t] = (uint32_t)min(run, (uint64_t)cap);
            ranges[2 * t + 1] = (uint32_t)min(run + ttotal[i], (uint64_t)cap);
        }
        run += ttotal[i];
    }
    if (threadIdx.x == 1023) {
        *d_P = (int64_t)s_sum[1023];
        if ((int64_t)s_sum[1023] > cap) atomicMax(&g_overflow_needed, s_sum[1023]);
    }
}

// Stage 3d: write every item's pairs. Rank of an item in a tile = chunk
// offset + items of earlier passes + earlier warps + earlier lanes listed in
// that tile (from one ballot per tile per warp).
__global__ void __launch_bounds__(kThreads) k_chunk_emit(const uint32_t *__restrict__ svals,
                                                        const uint32_t *__restrict__ masks,
                                                        const uint32_t *__restrict__ seg,
                                                        const uint32_t *__restrict__ cbase,
                                                        const uint32_t *__restrict__ ccount,
                                                        const uint32_t *__restrict__ tstart, Geo G,
                                                        int64_t cap, uint32_t *__restrict__ vals) {
    __shared__ uint32_t s_bal[kWarps][32];
    __shared__ uint32_t s_wpre[kWarps][32];
    __shared__ uint32_t s_base[32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t K = cbase[G.ns];
    for (uint32_t k = blockIdx.x; k < K; k += gridDim.x) {
        const int s = chunk_super(cbase, G.ns, k);
        const uint32_t a = seg[2 * s] + (k - cbase[s]) * kChunk;
        const uint32_t b = min(a + (uint32_t)kChunk, seg[2 * s + 1]);
        if (threadIdx.x < 32)
            s_base[threadIdx.x] = tstart[s * 32 + threadIdx.x] + ccount[(size_t)k * 32 + threadIdx.x];
        __syncthreads();
        for (uint32_t i0 = a; i0 < b; i0 += kThreads) {
            const uint32_t i = i0 + threadIdx.x;
            const uint32_t mask = i < b ? masks[i] : 0u;
            const uint32_t g = i < b ? svals[i] : 0u;
            uint32_t mycnt = 0;
#pragma unroll
            for (int l = 0; l < 32; ++l) {
                const uint32_t m = __ballot_sync(0xffffffffu, (mask >> l) & 1u);
                if (lane == l) {
                    s_bal[wid][l] = m;
                    mycnt = __popc(m);
                }
            }
            s_wpre[wid][lane] = mycnt;
            __syncthreads();
            // exclusive prefix over warps for tile `threadIdx.x`; the pass
            // total stays in `tot` of threads 0..31
            uint32_t tot = 0;
            if (threadIdx.x < 32) {
                for (int w = 0; w < kWarps; ++w) {
                    const uint32_t c = s_wpre[w][threadIdx.x];
                    s_wpre[w][threadIdx.x] = tot;
                    tot += c;
                }
            }
            __syncthreads();
            uint32_t mm = mask;
            while (mm) {
                const int l = __ffs(mm) - 1;
                mm &= mm - 1;
                const uint64_t pos = (uint64_t)s_base[l] + s_wpre[wid][l] + __popc(s_bal[wid][l] & lt);
                if (pos < (uint64_t)cap) vals[pos] = g;
            }
            __syncthreads();
            if (threadIdx.x < 32) s_base[threadIdx.x] += tot;
            __syncthreads();
        }
    }
}

}  // namespace

size_t bin_sort_workspace_size(int64_t maxV, int64_t cap, int ntiles) {
    // super-tiles of a grid of ntiles tiles: at most ntiles (one per tile in
    // the degenerate one-row or one-column grid)
    const int ns = ntiles > 0 ? ntiles : 65536;
    return layout(nullptr, maxV, cap, ns).bytes + 256;
}

lgs_status bin_sort(const lgs_splats *sp, const int32_t *d_V, int64_t maxV, const lgs_camera *cam,
                    int tw, int th, int cull, uint32_t *vals, int64_t cap, int64_t *d_P,
                    uint32_t *ranges, void *ws, size_t ws_bytes, cudaStream_t s) {
    const Geo G = make_geo(cam, tw, th);
    const int ntiles = G.gx * G.gy;
    if (ntiles > 65536 || G.ns > 65536) return LGS_ERR_INVALID_ARG;
    Layout L = layout(ws, maxV, cap, G.ns);
    if (L.bytes > ws_bytes) return LGS_ERR_INVALID_ARG;
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
    // 2. (super-tile, splat) items in depth order, then grouped by super-tile
    const unsigned gw = grid_for(maxV, kThreads);
    count_launch();
    k_super_walk<false><<<gw, kThreads, 0, s>>>(sp->rec, sp->radius, order, maxV, d_V, G, cull,
                                               L.scnt, nullptr, 0, nullptr, nullptr);
    st = exclusive_scan_u32_to_u64(L.scnt, L.soff, maxV, d_V, L.d_psup, L.scan, s);
    if (st != LGS_OK) return st;
    count_launch();
    k_check_super_capacity<<<1, 1, 0, s>>>(L.d_psup, cap);
    count_launch();
    k_super_walk<true><<<gw, kThreads, 0, s>>>(sp->rec, sp->radius, order, maxV, d_V, G, cull,
                                              nullptr, L.soff, cap, L.skeys[0], L.svals[0]);
    st = check_launch();
    if (st != LGS_OK) return st;
    st = radix_sort_u16(L.skeys, L.svals, cap, L.d_psup, nullptr, bits_for(G.ns), L.hist, &ob, s);
    if (st != LGS_OK) return st;
    const uint16_t *skeys = L.skeys[ob];
    const uint32_t *svals = L.svals[ob];
    cudaMemsetAsync(L.seg, 0, (size_t)G.ns * 8, s);
    count_launch();
    k_seg_ranges<<<grid_for(cap, kThreads), kThreads, 0, s>>>(skeys, L.d_psup, cap, L.seg);
    count_launch();
    k_chunk_plan<<<1, 1024, 0, s>>>(L.seg, G.ns, L.cbase);
    // 3. masks, chunk counts, offsets, tile starts, pairs
    const int64_t mc = max_chunks(G.ns, cap), cap_blocks = (int64_t)num_sms() * 16;
    const unsigned gc = (unsigned)(mc < cap_blocks ? mc : cap_blocks);
    count_launch();
    k_chunk_masks<<<gc, kThreads, 0, s>>>(sp->rec, sp->radius, svals, L.seg, L.cbase, G, cull,
                                         L.masks, L.ccount);
    count_launch();
    k_chunk_offsets<<<(unsigned)ceil_div((int64_t)G.ns * 32, kThreads), kThreads, 0, s>>>(
        L.ccount, L.cbase, G.ns, L.ttotal);
    count_launch();
    k_tile_starts<<<1, 1024, 0, s>>>(L.ttotal, G, L.tstart, ranges, d_P, cap);
    count_launch();
    k_chunk_emit<<<gc, kThreads, 0, s>>>(svals, L.masks, L.seg, L.cbase, L.ccount, L.tstart, G, cap,
                                        vals);
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
