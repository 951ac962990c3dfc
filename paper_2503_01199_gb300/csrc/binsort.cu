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
//   2. each splat, in depth order, finds the tiles it is listed in (its
//      rectangle and, per tile row, the interval kept by the culling test)
//      and emits one item per super-tile (8 x 4 tiles) holding any of them,
//      with a 32-bit mask of those tiles; the items are sorted stably by
//      super-tile (one 8-bit pass for up to 256 super-tiles);
//   3. each super-tile's items are taken in chunks of 1024; a warp-wide bit
//      transpose of 32 items' masks gives every tile's ballot, hence the
//      counts per chunk and tile and every item's rank among the earlier
//      items listed in the same tile, so each tile's list is written in
//      depth order without sorting the pairs themselves.
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
    uint64_t *gstatus;    // look-back status per group of 32 splats
    uint32_t *gcounter;   // next group id (follows gstatus)
    size_t gstatus_bytes; // both, cleared before stage 2
    uint16_t *skeys[2];
    uint64_t *svals[2];   // tile mask << 32 | splat
    uint32_t *seg;        // [ns][2]
    uint32_t *cbase;      // [ns + 1]
    uint4 *ctab;          // [max_chunks]: super-tile, first item, end item
    uint32_t *ccount;     // [max_chunks][32]
    uint32_t *tstart;     // [ns * 32]
    uint32_t *ttotal;     // [ns * 32]
    int64_t *d_psup;
    void *hist;
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
    L.gstatus_bytes = (size_t)ceil_div(maxV > 0 ? maxV : 1, 32) * 8 + 8;
    L.gstatus = reinterpret_cast<uint64_t *>(take(L.gstatus_bytes));
    L.gcounter = reinterpret_cast<uint32_t *>(reinterpret_cast<unsigned char *>(L.gstatus) +
                                              L.gstatus_bytes - 8);
    for (int k = 0; k < 2; ++k) L.skeys[k] = reinterpret_cast<uint16_t *>(take((size_t)cap * 2));
    for (int k = 0; k < 2; ++k) L.svals[k] = reinterpret_cast<uint64_t *>(take((size_t)cap * 8));
    L.seg = reinterpret_cast<uint32_t *>(take((size_t)ns * 8));
    L.cbase = reinterpret_cast<uint32_t *>(take((size_t)(ns + 1) * 4));
    L.ctab = reinterpret_cast<uint4 *>(take((size_t)max_chunks(ns, cap) * 16));
    L.ccount = reinterpret_cast<uint32_t *>(take((size_t)max_chunks(ns, cap) * 32 * 4));
    L.tstart = reinterpret_cast<uint32_t *>(take((size_t)ns * 32 * 4));
    L.ttotal = reinterpret_cast<uint32_t *>(take((size_t)ns * 32 * 4));
    L.d_psup = reinterpret_cast<int64_t *>(take(8));
    L.hist = take(radix_hist_bytes(maxV > cap ? maxV : cap));
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
    // the record is read whatever the radius (row g < V is in bounds), so
    // both loads are in flight together; a culled splat's is unused
    const int rad = radius[g];
    const float4 *p = reinterpret_cast<const float4 *>(rec + 12 * (int64_t)g);
    const float4 a = p[0];
    const float c = p[1].x, tau = p[2].y;
    if (rad > 0) {
        s.u = a.x; s.v = a.y; s.A = a.z; s.B = a.w;
        s.C = c;
        s.tau = tau;
        s.rA = __frcp_rn(s.A);
        s.rC = __frcp_rn(s.C);
        s.rc = tile_rect(a.x, a.y, (float)rad, G.tw, G.th, G.gx, G.gy);
        if (s.rc.z <= s.rc.x || s.rc.w <= s.rc.y) s.rc = make_int4(0, 0, 0, 0);
    }
    return s;
}

// Tiles [a, b] of a tile row (a > b: none) that the row form of the culling
// test keeps, within the rectangle's columns [x0, x1): the test
// u - xh(tx) <= U only gets truer as tx grows and u - xl(tx) >= L only
// falser (correctly rounded differences are monotone), so the kept tiles
// form one interval, found from an estimate (rtw = 1 / tw) and a few exact
// tests -- the same operations as the row form's per-tile condition.
__device__ __forceinline__ bool right_ok(float u, int tx, int tw, float U) {
    const float xh = __fadd_rn((float)(tx * tw + tw), -0.5f);
    return __fsub_rn(u, xh) <= U;
}
__device__ __forceinline__ bool left_ok(float u, int tx, int tw, float L) {
    const float xl = __fadd_rn((float)(tx * tw), 0.5f);
    return __fsub_rn(u, xl) >= L;
}
__device__ __forceinline__ void row_span(float u, int x0, int x1, int tw, float rtw, float L,
                                         float U, int &a, int &b) {
    int t1 = (int)fminf(fmaxf(ceilf((u - U + 0.5f) * rtw - 1.0f), (float)x0), (float)x1);
    while (t1 > x0 && right_ok(u, t1 - 1, tw, U)) --t1;
    while (t1 < x1 && !right_ok(u, t1, tw, U)) ++t1;
    int t2 = (int)fminf(fmaxf(floorf((u - L - 0.5f) * rtw), (float)(x0 - 1)), (float)(x1 - 1));
    while (t2 < x1 - 1 && left_ok(u, t2 + 1, tw, L)) ++t2;
    while (t2 >= x0 && !left_ok(u, t2, tw, L)) --t2;
    a = t1;
    b = t2;
}

constexpr uint32_t kEmptySpan = 1u;  // packed span (a, b) = (1, 0)
constexpr int kSpanCap = 512;        // row spans per warp held in shared memory

// Packed kept span (a | b << 16) of tile row ty of a splat with rectangle
// columns [x0, x1): with the row test, the tiles whose offsets meet the
// row's interval; without it, the whole rectangle row.
__device__ __forceinline__ uint32_t row_span_of(const RowCull &q, int x0, int x1, int ty,
                                                bool row_test, const Geo &G, float rtw) {
    int a = x0, b = x1 - 1;
    if (row_test) {
        a = 1;
        b = 0;
        float L, U;
        if (row_interval(q, ty, G.th, L, U)) row_span(q.u, x0, x1, G.tw, rtw, L, U, a, b);
    }
    return a <= b ? ((uint32_t)a | ((uint32_t)b << 16)) : kEmptySpan;
}

// Calls f(super-tile id, 32-bit tile mask) for every super-tile in which the
// splat is listed in at least one tile, in row-major super-tile order, from
// the kept span of every tile row of its rectangle (span_of(k) for row
// rc.y + k). With per_tile (degenerate conic under culling) the spans are
// the rectangle's and each tile takes the box test.
template <class S, class F>
__device__ __forceinline__ void for_each_super(const int4 rc, S &&span_of, bool per_tile,
                                               const SplatGeom &sg, const Geo &G, F &&f) {
    if (rc.z <= rc.x || rc.w <= rc.y) return;
    for (int sy = rc.y / kSY; sy <= (rc.w - 1) / kSY; ++sy) {
        int a[kSY], b[kSY];
        int amin = rc.z, bmax = rc.x - 1;
#pragma unroll
        for (int k = 0; k < kSY; ++k) {
            const int ty = sy * kSY + k;
            const uint32_t w = (ty >= rc.y && ty < rc.w) ? span_of(ty - rc.y) : kEmptySpan;
            a[k] = (int)(w & 0xffffu);
            b[k] = (int)(w >> 16);
            if (a[k] <= b[k]) {
                amin = min(amin, a[k]);
                bmax = max(bmax, b[k]);
            }
        }
        if (bmax < amin) continue;
        for (int sx = amin / kSX; sx <= bmax / kSX; ++sx) {
            uint32_t mask = 0;
#pragma unroll
            for (int k = 0; k < kSY; ++k) {
                const int lo = max(a[k], sx * kSX), hi = min(b[k], sx * kSX + kSX - 1);
                if (lo <= hi) mask |= ((2u << (hi - lo)) - 1u) << (lo - sx * kSX + k * kSX);
            }
            if (per_tile) {
                uint32_t kept = 0;
                for (uint32_t m = mask; m; m &= m - 1) {
                    const int bit = __ffs(m) - 1;
                    if (tile_reachable(sg.u, sg.v, sg.A, sg.B, sg.C, sg.rA, sg.rC, sg.tau,
                                       sx * kSX + bit % kSX, sy * kSY + bit / kSX, G.tw, G.th))
                        kept |= 1u << bit;
                }
                mask = kept;
            }
            if (mask) f(sy * G.sgx + sx, mask);
        }
    }
}

// Number of super-tiles holding at least one of the splat's tiles: per
// super-tile row, the super-columns covered by the union of its (up to 4)
// tile rows' spans. Exact unless the box test refines tiles (per_tile).
template <class S>
__device__ __forceinline__ uint32_t super_count(const int4 rc, S &&span_of) {
    if (rc.z <= rc.x || rc.w <= rc.y) return 0u;
    uint32_t n = 0;
    for (int sy = rc.y / kSY; sy <= (rc.w - 1) / kSY; ++sy) {
        int a[kSY], b[kSY];
        int amin = rc.z, bmax = rc.x - 1;
#pragma unroll
        for (int k = 0; k < kSY; ++k) {
            const int ty = sy * kSY + k;
            const uint32_t w = (ty >= rc.y && ty < rc.w) ? span_of(ty - rc.y) : kEmptySpan;
            a[k] = (int)(w & 0xffffu);
            b[k] = (int)(w >> 16);
            if (a[k] <= b[k]) {
                amin = min(amin, a[k]);
                bmax = max(bmax, b[k]);
            }
        }
        if (bmax < amin) continue;
        const int base = amin / kSX, last = bmax / kSX;
        if (last - base < 32) {
            uint32_t m = 0;
#pragma unroll
            for (int k = 0; k < kSY; ++k)
                if (a[k] <= b[k]) {
                    const int p = a[k] / kSX - base, q = b[k] / kSX - base;
                    m |= ((2u << (q - p)) - 1u) << p;
                }
            n += __popc(m);
        } else {
            for (int sx = base; sx <= last; ++sx) {
                bool hit = false;
#pragma unroll
                for (int k = 0; k < kSY; ++k)
                    hit |= a[k] <= b[k] && a[k] / kSX <= sx && sx <= b[k] / kSX;
                n += hit ? 1u : 0u;
            }
        }
    }
    return n;
}

// Look-back status of a group of 32 splats: flag in the top two bits, the
// group's item count (AGG) or the inclusive item count of groups <= it (PRE).
constexpr uint64_t kGrpAgg = 1ull << 62, kGrpPre = 2ull << 62, kGrpVal = (1ull << 62) - 1ull;
constexpr int kItemCap = 384;  // items per warp staged in shared memory

__device__ unsigned int g_bin_wait_timeouts;
// polls of an unpublished predecessor group before the look-back gives up
__device__ uint32_t g_bin_spin_limit = kDefaultSpinLimit;

__device__ __forceinline__ uint64_t warp_sum_u64(uint64_t x) {
#pragma unroll
    for (int d = 16; d; d >>= 1) x += __shfl_xor_sync(0xffffffffu, x, d);
    return x;
}

// Lane owning position p of a warp's concatenated per-lane runs: the
// number of lanes whose inclusive end `incl` is <= p (32 if p is past the
// last run).
__device__ __forceinline__ int run_owner(uint32_t incl, uint32_t p) {
    int j = 0;
#pragma unroll
    for (int st = 16; st; st >>= 1)
        if (__shfl_sync(0xffffffffu, incl, j + st - 1) <= p) j += st;
    return j;
}

// Stage 2: the (super-tile, splat) items in depth order, written as
// (super-tile id, mask << 32 | splat). Each warp takes the next group of 32
// consecutive splats (group ids from an atomic counter, so a group only
// waits on groups already being processed):
//   - the tile rows of the group's rectangles are spread evenly over the
//     lanes (a row's owner found by a binary search over the warp's
//     inclusive row counts, its test parameters read from shared memory)
//     and each row's kept span goes to shared memory; a group with more
//     rows than fit computes each splat's rows in its own lane instead;
//   - each lane counts its items from the spans, the group's item offset
//     comes from a decoupled look-back over earlier groups (32 predecessors
//     per step, bounded wait), the items are assembled in shared memory in
//     output order and copied out with coalesced stores (written directly
//     when they do not fit).
__global__ void __launch_bounds__(kThreads) k_super_items(
    const float *__restrict__ rec, const int32_t *__restrict__ radius,
    const uint32_t *__restrict__ order, int64_t maxV, const int32_t *d_V, Geo G, int cull,
    uint32_t *counter, uint64_t *status, int64_t cap, uint16_t *__restrict__ skeys,
    uint64_t *__restrict__ svals, int64_t *d_psup) {
    __shared__ uint32_t s_span[kWarps][kSpanCap];
    __shared__ uint32_t s_imask[kWarps][kItemCap];
    __shared__ uint16_t s_isid[kWarps][kItemCap];
    __shared__ float4 s_par[kWarps][32][3];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t V = load_count(d_V, maxV);
    const int64_t groups = (V + 31) / 32;
    const float rtw = div_by_size(1.0f, G.tw), rth = div_by_size(1.0f, G.th);
    if (groups == 0 && blockIdx.x == 0 && threadIdx.x == 0) *d_psup = 0;
    for (;;) {
        uint32_t gid = 0;
        if (lane == 0) gid = atomicAdd(counter, 1u);
        gid = __shfl_sync(0xffffffffu, gid, 0);
        if ((int64_t)gid >= groups) break;
        const int64_t r = (int64_t)gid * 32 + lane;
        const bool ok = r < V;
        const uint32_t g = ok ? order[r] : 0u;
        SplatGeom sg{};
        if (ok) sg = splat_geom(rec, radius, g, G);
        const int4 rc = sg.rc;
        const RowCull rcl = row_cull(sg.u, sg.v, sg.A, sg.B, sg.C, sg.rA, sg.rC, sg.tau);
        const bool per_tile = cull && rcl.degenerate;
        const bool row_test = cull && !rcl.degenerate;
        // with the row test, only the rows [ry0, ry1) that pass its first
        // condition (v - yh <= e_y and v - yl >= -e_y, monotone in the row)
        // can keep a tile; the others are empty without computing them
        int ry0 = rc.y, ry1 = rc.w;
        if (row_test && rc.w > rc.y) {
            if (!(rcl.tau >= 0.0f)) {
                ry1 = ry0;
            } else {
                int a, b;
                row_span(rcl.v, rc.y, rc.w, G.th, rth, -rcl.ey, rcl.ey, a, b);
                ry0 = a;
                ry1 = max(a, b + 1);
            }
        }
        const uint32_t n = (uint32_t)(ry1 - ry0);
        uint32_t incl = n;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += y;
        }
        const uint32_t T = __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t first = incl - n;
        const bool staged = T <= (uint32_t)kSpanCap;
        if (staged) {
            s_par[wid][lane][0] = make_float4(rcl.u, rcl.v, rcl.A, rcl.B);
            s_par[wid][lane][1] = make_float4(rcl.tau, rcl.det, rcl.ey, rcl.dyU);
            s_par[wid][lane][2] = make_float4(__int_as_float(rc.x), __int_as_float(rc.z),
                                              __int_as_float(ry0),
                                              __int_as_float((int)(first << 1) | (row_test ? 1 : 0)));
            __syncwarp();
            for (uint32_t c = 0; c < T; c += 32) {
                const uint32_t p = c + lane;
                const int j = run_owner(incl, p);
                if (p < T) {
                    const float4 P0 = s_par[wid][j][0], P1 = s_par[wid][j][1], P2 = s_par[wid][j][2];
                    RowCull q;
                    q.u = P0.x; q.v = P0.y; q.A = P0.z; q.B = P0.w;
                    q.tau = P1.x; q.det = P1.y; q.ey = P1.z; q.dyU = P1.w;
                    q.C = q.rA = q.rC = 0.0f;
                    q.degenerate = false;
                    const int fl = __float_as_int(P2.w);
                    const int ty = __float_as_int(P2.z) + (int)(p - ((uint32_t)fl >> 1));
                    s_span[wid][p] = row_span_of(q, __float_as_int(P2.x), __float_as_int(P2.y), ty,
                                                 (fl & 1) != 0, G, rtw);
                }
            }
            __syncwarp();
        }
        auto span_of = [&](int k) -> uint32_t {
            const int ty = rc.y + k;
            if (ty < ry0 || ty >= ry1) return kEmptySpan;
            return staged ? s_span[wid][first + (ty - ry0)]
                          : row_span_of(rcl, rc.x, rc.z, ty, row_test, G, rtw);
        };
        uint32_t items;
        if (per_tile) {
            items = 0;
            for_each_super(rc, span_of, true, sg, G, [&](int, uint32_t) { ++items; });
        } else {
            items = super_count(rc, span_of);
        }
        uint32_t iincl = items;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, iincl, d);
            if (lane >= d) iincl += y;
        }
        const uint32_t agg = __shfl_sync(0xffffffffu, iincl, 31);
        volatile uint64_t *vs = status;
        if (lane == 0) vs[gid] = (gid == 0 ? kGrpPre : kGrpAgg) | agg;
        // assemble the group's items in output order while predecessors finish
        const bool istaged = agg <= (uint32_t)kItemCap;
        if (istaged) {
            uint32_t e = iincl - items;
            for_each_super(rc, span_of, per_tile, sg, G, [&](int sid, uint32_t mask) {
                s_imask[wid][e] = mask;
                s_isid[wid][e] = (uint16_t)sid;
                ++e;
            });
            __syncwarp();
        }
        uint64_t excl = 0;
        if (gid > 0) {
            int64_t k = (int64_t)gid - 1;
            uint32_t spins = 0;
            for (;;) {
                const int64_t idx = k - lane;
                uint64_t w = kGrpPre;  // before group 0: a prefix of 0
                if (idx >= 0) w = vs[idx];
                const uint32_t fl = (uint32_t)(w >> 62);
                const uint32_t pre = __ballot_sync(0xffffffffu, fl == 2u);
                const uint32_t wait = __ballot_sync(0xffffffffu, fl == 0u);
                const int stop = pre ? __ffs(pre) - 1 : 31;
                const uint32_t need = stop == 31 ? 0xffffffffu : ((2u << stop) - 1u);
                if (wait & need) {
                    if (++spins > g_bin_spin_limit) {
                        if (lane == 0) atomicAdd(&g_bin_wait_timeouts, 1u);
                        break;
                    }
                    __nanosleep(32);
                    continue;
                }
                excl += warp_sum_u64(lane <= stop ? (w & kGrpVal) : 0ull);
                if (pre) break;
                k -= 32;
            }
            if (lane == 0) vs[gid] = kGrpPre | ((excl + agg) & kGrpVal);
        }
        if ((int64_t)gid == groups - 1 && lane == 31) *d_psup = (int64_t)(excl + agg);
        if (istaged) {
            for (uint32_t c = 0; c < agg; c += 32) {
                const uint32_t e = c + lane;
                const int j = run_owner(iincl, e);
                const uint32_t gj = __shfl_sync(0xffffffffu, g, j < 32 ? j : 31);
                const uint64_t o = excl + e;
                if (e < agg && o < (uint64_t)cap) {
                    skeys[o] = s_isid[wid][e];
                    svals[o] = ((uint64_t)s_imask[wid][e] << 32) | gj;
                }
            }
        } else {
            uint64_t o = excl + iincl - items;
            for_each_super(rc, span_of, per_tile, sg, G, [&](int sid, uint32_t mask) {
                if (o < (uint64_t)cap) {
                    skeys[o] = (uint16_t)sid;
                    svals[o] = ((uint64_t)mask << 32) | g;
                }
                ++o;
            });
        }
        __syncwarp();
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

// Chunks of every super-tile: cbase[s] = first chunk of s, cbase[ns] = total,
// and ctab[k] = (super-tile, first item, end item) of every chunk k.
// With `hist` (the item count of every super-tile, when one sort pass
// covers all super-tile ids) the item ranges seg are derived here as well.
__global__ void __launch_bounds__(1024) k_chunk_plan(const uint32_t *__restrict__ hist,
                                                    uint32_t *__restrict__ seg, int ns,
                                                    uint32_t *__restrict__ cbase,
                                                    uint4 *__restrict__ ctab) {
    __shared__ uint64_t s_sum[1024];
    const int per = (ns + 1023) / 1024;
    const int s0 = threadIdx.x * per;
    auto items = [&](int s) { return hist ? hist[s] : seg[2 * s + 1] - seg[2 * s]; };
    // items in the high word, chunks in the low word: one scan for both
    uint64_t tot = 0;
    for (int s = s0; s < min(ns, s0 + per); ++s) {
        const uint32_t c = items(s);
        tot += ((uint64_t)c << 32) | ((c + kChunk - 1) / kChunk);
    }
    s_sum[threadIdx.x] = tot;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const uint64_t x = threadIdx.x >= o ? s_sum[threadIdx.x - o] : 0ull;
        __syncthreads();
        s_sum[threadIdx.x] += x;
        __syncthreads();
    }
    uint64_t run = s_sum[threadIdx.x] - tot;
    for (int s = s0; s < min(ns, s0 + per); ++s) {
        const uint32_t c = items(s);
        cbase[s] = (uint32_t)run;
        const uint32_t a = hist ? (uint32_t)(run >> 32) : seg[2 * s];
        if (hist) {
            seg[2 * s] = a;
            seg[2 * s + 1] = a + c;
        }
        for (uint32_t q = 0; q * kChunk < c; ++q) {
            const uint32_t i0 = q * kChunk;
            ctab[(uint32_t)run + q] =
                make_uint4((uint32_t)s, a + i0, a + i0 + min(c - i0, (uint32_t)kChunk), 0u);
        }
        run += ((uint64_t)c << 32) | ((c + kChunk - 1) / kChunk);
    }
    if (threadIdx.x == 1023) cbase[ns] = (uint32_t)s_sum[1023];
}

// 32 x 32 bit transpose across a warp: bit i of lane l's result is bit l of
// lane i's x (lane l receives the ballot of bit l). Five butterfly stages;
// stage j exchanges the off-diagonal j x j blocks between lanes l and l ^ j.
__device__ __forceinline__ uint32_t warp_transpose(uint32_t x, int lane) {
    constexpr uint32_t lo[5] = {0x0000ffffu, 0x00ff00ffu, 0x0f0f0f0fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int st = 0; st < 5; ++st) {
        const int j = 16 >> st;
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
        x = (lane & j) ? ((x & ~lo[st]) | ((y >> j) & lo[st]))
                       : ((x & lo[st]) | ((y << j) & ~lo[st]));
    }
    return x;
}

// Stage 3a: per chunk of 1024 items of one super-tile, the number of items
// listed in each of its 32 tiles. One CTA per chunk.
__global__ void __launch_bounds__(kThreads) k_chunk_counts(const uint64_t *__restrict__ svals,
                                                          const uint4 *__restrict__ ctab,
                                                          const uint32_t *__restrict__ cbase, Geo G,
                                                          uint32_t *__restrict__ ccount) {
    __shared__ uint32_t s_cnt[kWarps][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t K = cbase[G.ns];
    for (uint32_t k = blockIdx.x; k < K; k += gridDim.x) {
        const uint4 ck = ctab[k];
        const uint32_t a = ck.y, b = ck.z;
        uint32_t my = 0;  // this warp's count for tile `lane`
        for (uint32_t i = a + threadIdx.x; i - threadIdx.x < b; i += kThreads) {
            const uint32_t mask = i < b ? (uint32_t)(svals[i] >> 32) : 0u;
            my += __popc(warp_transpose(mask, lane));
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
// place) and the tile's total. One CTA per super-tile, lane = tile: each
// warp scans a contiguous range of the super-tile's chunks, then the warps'
// totals are scanned and added.
__global__ void __launch_bounds__(kThreads) k_chunk_offsets(uint32_t *__restrict__ ccount,
                                                           const uint32_t *__restrict__ cbase,
                                                           int ns, uint32_t *__restrict__ ttotal) {
    __shared__ uint32_t s_w[kWarps][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int s = blockIdx.x; s < ns; s += gridDim.x) {
        const uint32_t k0 = cbase[s], k1 = cbase[s + 1];
        const uint32_t per = (k1 - k0 + kWarps - 1) / kWarps;
        const uint32_t a = min(k0 + wid * per, k1), b = min(a + per, k1);
        uint32_t run = 0;
        for (uint32_t k = a; k < b; ++k) run += ccount[(size_t)k * 32 + lane];
        s_w[wid][lane] = run;
        __syncthreads();
        uint32_t base = 0;
        for (int w = 0; w < wid; ++w) base += s_w[w][lane];
        if (wid == kWarps - 1) ttotal[s * 32 + lane] = base + run;
        for (uint32_t k = a; k < b; ++k) {
            const uint32_t c = ccount[(size_t)k * 32 + lane];
            ccount[(size_t)k * 32 + lane] = base;
            base += c;
        }
        __syncthreads();
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

// Stage 3d: write every item's pairs. Each warp takes 128 consecutive items
// of the chunk (4 rounds of 32); the bit transpose of a round's masks gives
// lane t the round's items listed in tile t, so lane t writes tile t's
// entries itself, in item order, at: the chunk's start in the tile + items
// of earlier warps + items of earlier rounds. The entries go to a
// tile-major buffer in shared memory, copied out tile by tile with
// consecutive lanes storing consecutive addresses; a chunk with more pairs
// than the buffer holds is written directly.
constexpr int kStage = 6144;  // pairs of one chunk staged in shared memory (twice the
                              // typical chunk, small enough for 8 CTAs per SM)

__global__ void __launch_bounds__(kThreads) k_chunk_emit(const uint64_t *__restrict__ svals,
                                                        const uint4 *__restrict__ ctab,
                                                        const uint32_t *__restrict__ cbase,
                                                        const uint32_t *__restrict__ ccount,
                                                        const uint32_t *__restrict__ tstart, Geo G,
                                                        int64_t cap, uint32_t *__restrict__ vals) {
    constexpr int kRounds = kChunk / kThreads;
    constexpr int kPerWarp = kChunk / kWarps;
    __shared__ uint32_t s_w[kWarps][32];
    __shared__ uint32_t s_start[32], s_off[33];
    __shared__ uint32_t s_pairs[kStage];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t K = cbase[G.ns];
    for (uint32_t k = blockIdx.x; k < K; k += gridDim.x) {
        const uint4 ck = ctab[k];
        const int s = (int)ck.x;
        const uint32_t a = ck.y, b = ck.z;
        const uint32_t w0 = a + wid * kPerWarp;
        // the chunk's start in every tile, loaded while the items arrive
        uint32_t start = 0;
        if (threadIdx.x < 32) start = tstart[s * 32 + lane] + ccount[(size_t)k * 32 + lane];
        uint32_t g[kRounds], tw[kRounds];  // tw: the round's items listed in tile `lane`
        uint32_t cnt = 0;
#pragma unroll
        for (int j = 0; j < kRounds; ++j) {
            const uint32_t i = w0 + j * 32 + lane;
            const uint64_t v = i < b ? svals[i] : 0ull;
            g[j] = (uint32_t)v;
            tw[j] = warp_transpose((uint32_t)(v >> 32), lane);
            cnt += __popc(tw[j]);
        }
        s_w[wid][lane] = cnt;
        __syncthreads();
        if (threadIdx.x < 32) {
            // per tile: earlier warps' items, the chunk's total, and the
            // tile's place in the staging buffer
            uint32_t run = 0;
            for (int w = 0; w < kWarps; ++w) {
                const uint32_t c = s_w[w][lane];
                s_w[w][lane] = run;
                run += c;
            }
            uint32_t incl = run;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            s_start[lane] = start;
            s_off[lane] = incl - run;
            if (lane == 31) s_off[32] = incl;
        }
        __syncthreads();
        const bool staged = s_off[32] <= (uint32_t)kStage;
        // next entry of tile `lane`: in the buffer, or its position in vals
        uint64_t pos = (uint64_t)s_w[wid][lane] + (staged ? s_off[lane] : s_start[lane]);
#pragma unroll
        for (int j = 0; j < kRounds; ++j) {
            const int n = __reduce_max_sync(0xffffffffu, (unsigned)__popc(tw[j]));
            uint32_t t = tw[j];
            for (int r = 0; r < n; ++r) {
                const int i = t ? __ffs(t) - 1 : 0;
                const uint32_t gi = __shfl_sync(0xffffffffu, g[j], i);
                if (t) {
                    if (staged)
                        s_pairs[pos] = gi;
                    else if (pos < (uint64_t)cap)
                        vals[pos] = gi;
                    ++pos;
                    t &= t - 1u;
                }
            }
        }
        __syncthreads();
        if (staged) {
            for (int l = wid; l < 32; l += kWarps) {
                const uint32_t o = s_off[l], n = s_off[l + 1] - o;
                const uint64_t base = s_start[l];
                for (uint32_t e = lane; e < n; e += 32)
                    if (base + e < (uint64_t)cap) vals[base + e] = s_pairs[o + e];
            }
        }
        __syncthreads();
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
    // row spans hold tile columns in 16 bits
    if (ntiles > 65536 || G.ns > 65536 || G.gx > 65535) return LGS_ERR_INVALID_ARG;
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
    cudaMemsetAsync(L.gstatus, 0, L.gstatus_bytes, s);
    count_launch();
    k_super_items<<<grid_for(maxV, kThreads, 8), kThreads, 0, s>>>(
        sp->rec, sp->radius, order, maxV, d_V, G, cull, L.gcounter, L.gstatus, cap, L.skeys[0],
        L.svals[0], L.d_psup);
    count_launch();
    k_check_super_capacity<<<1, 1, 0, s>>>(L.d_psup, cap);
    st = check_launch();
    if (st != LGS_OK) return st;
    const int sbits = bits_for(G.ns);
    st = radix_sort_u16_v64(L.skeys, L.svals, cap, L.d_psup, nullptr, sbits, L.hist, &ob, s);
    if (st != LGS_OK) return st;
    const uint64_t *svals = L.svals[ob];
    const uint32_t *hist = nullptr;
    if (radix_passes(sbits) == 1) {
        // one pass: its digit counts are the item counts of the super-tiles
        hist = static_cast<const uint32_t *>(L.hist);
    } else {
        cudaMemsetAsync(L.seg, 0, (size_t)G.ns * 8, s);
        count_launch();
        k_seg_ranges<<<grid_for(cap, kThreads), kThreads, 0, s>>>(L.skeys[ob], L.d_psup, cap,
                                                                  L.seg);
    }
    count_launch();
    k_chunk_plan<<<1, 1024, 0, s>>>(hist, L.seg, G.ns, L.cbase, L.ctab);
    // 3. masks, chunk counts, offsets, tile starts, pairs
    const int64_t mc = max_chunks(G.ns, cap), cap_blocks = (int64_t)num_sms() * 16;
    const unsigned gc = (unsigned)(mc < cap_blocks ? mc : cap_blocks);
    count_launch();
    k_chunk_counts<<<gc, kThreads, 0, s>>>(svals, L.ctab, L.cbase, G, L.ccount);
    count_launch();
    k_chunk_offsets<<<(unsigned)G.ns, kThreads, 0, s>>>(L.ccount, L.cbase, G.ns, L.ttotal);
    count_launch();
    k_tile_starts<<<1, 1024, 0, s>>>(L.ttotal, G, L.tstart, ranges, d_P, cap);
    count_launch();
    k_chunk_emit<<<gc, kThreads, 0, s>>>(svals, L.ctab, L.cbase, L.ccount, L.tstart, G, cap,
                                        vals);
    return check_launch();
}

namespace {

// The 64-bit sort key (tile << 32 | depth bits) of every pair of a finished
// binning, one CTA per tile over its range of vals. A pair whose splat
// index is not below `rows` gets the key of a pair at infinite depth.
__global__ void __launch_bounds__(kThreads) k_bin_keys(const float *__restrict__ depth,
                                                      const uint32_t *__restrict__ vals,
                                                      const uint32_t *__restrict__ ranges,
                                                      int64_t rows, uint64_t *__restrict__ keys) {
    const uint32_t t = blockIdx.x;
    const uint32_t r0 = ranges[2 * t], r1 = ranges[2 * t + 1];
    for (uint32_t p = r0 + threadIdx.x; p < r1; p += kThreads) {
        const uint32_t v = vals[p];
        const uint32_t d = (int64_t)v < rows ? __float_as_uint(depth[v]) : 0x7f800000u;
        keys[p] = ((uint64_t)t << 32) | d;
    }
}

}  // namespace

lgs_status bin_keys(const float *depth, const uint32_t *vals, const uint32_t *ranges, int ntiles,
                    int64_t rows, uint64_t *keys, cudaStream_t s) {
    count_launch();
    k_bin_keys<<<(unsigned)ntiles, kThreads, 0, s>>>(depth, vals, ranges, rows, keys);
    return check_launch();
}

lgs_status bin_set_spin_limit(uint32_t spins) {
    if (cudaMemcpyToSymbol(g_bin_spin_limit, &spins, sizeof(spins)) != cudaSuccess) {
        set_cuda_error(cudaGetLastError());
        return LGS_ERR_CUDA;
    }
    return LGS_OK;
}

lgs_status bin_wait_timeouts(uint32_t *count) {
    unsigned int h = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&h, g_bin_wait_timeouts, sizeof(h)) != cudaSuccess ||
        cudaMemcpyToSymbol(g_bin_wait_timeouts, &zero, sizeof(zero)) != cudaSuccess) {
        set_cuda_error(cudaGetLastError());
        return LGS_ERR_CUDA;
    }
    *count = h;
    return h ? LGS_ERR_TIMEOUT : LGS_OK;
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
