// Internal declarations shared by the CUDA translation units of liblgs.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "lgs.h"

namespace lgs {

constexpr int kWarp = 32;

// Last CUDA error seen by a launch (for lgs_last_cuda_error()).
void set_cuda_error(cudaError_t e);

// Check the launch just made; map failures to LGS_ERR_CUDA.
lgs_status check_launch();

// Count one kernel launch of this library (reported by lgs_kernel_launches()).
void count_launch();

inline cudaStream_t as_stream(lgs_stream s) { return reinterpret_cast<cudaStream_t>(s); }

inline bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Number of SMs of the current device (cached per device).
int num_sms();

inline int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

// Grid for a grid-stride loop over `n` items with `threads` per block.
inline unsigned grid_for(int64_t n, int threads, int per_sm = 8) {
    int64_t blocks = ceil_div(n > 0 ? n : 1, threads);
    int64_t cap = (int64_t)num_sms() * per_sm;
    return (unsigned)(blocks < cap ? blocks : cap);
}

// ---------------------------------------------------------------------------
// Bounds checks of the debug build (compiled with -DLGS_DEBUG). LGS_DCHECK
// (cond, site) is true when cond holds; when it does not, the first failure
// of the translation unit is recorded in its error word as
// (site << 32) | source line, and the caller skips the access it guards.
// Release builds compile it to `true`. Each translation unit has its own
// word (the library is built without relocatable device code); DEBUG_TU
// defines the host function that reads and clears it.
// ---------------------------------------------------------------------------
enum DebugSite : uint32_t {
    kSiteRasterSplat = 1,   // splat index of a tile list < splat rows
    kSiteRasterRow = 2,     // gradient row < grad_acc rows
    kSiteSortScatter = 3,   // radix sort output position < key count
    kSiteGatherPerm = 4,    // Morton gather source row < rows
    kSitePreMap = 5,        // preprocess compaction-map row < rows
    kSiteAdamMap = 6,       // backward / Adam compaction-map row < rows
    kSiteDensifyRow = 7,    // densification source row / moments map row < rows
};

#ifdef LGS_DEBUG
namespace {
__device__ unsigned long long g_debug_error;
__device__ __forceinline__ bool dcheck(bool ok, uint32_t site, uint32_t line) {
    if (!ok) atomicCAS(&g_debug_error, 0ull, ((unsigned long long)site << 32) | line);
    return ok;
}
}  // namespace
#define LGS_DCHECK(cond, site) ::lgs::dcheck((cond), (site), __LINE__)
#define DEBUG_TU(name)                                                                      \
    lgs_status debug_error_##name(uint64_t *code) {                                        \
        unsigned long long h = 0, zero = 0;                                                 \
        if (cudaMemcpyFromSymbol(&h, g_debug_error, sizeof(h)) != cudaSuccess ||           \
            cudaMemcpyToSymbol(g_debug_error, &zero, sizeof(zero)) != cudaSuccess) {       \
            set_cuda_error(cudaGetLastError());                                            \
            return LGS_ERR_CUDA;                                                           \
        }                                                                                   \
        *code = h;                                                                          \
        return LGS_OK;                                                                      \
    }
#else
#define LGS_DCHECK(cond, site) true
#define DEBUG_TU(name)                                                                      \
    lgs_status debug_error_##name(uint64_t *code) {                                        \
        *code = 0;                                                                          \
        return LGS_OK;                                                                      \
    }
#endif
lgs_status debug_error_raster(uint64_t *code);
lgs_status debug_error_sort(uint64_t *code);
lgs_status debug_error_ccc(uint64_t *code);
lgs_status debug_error_preprocess(uint64_t *code);
lgs_status debug_error_densify(uint64_t *code);

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int load_count(const int32_t *d_count, int64_t fallback) {
    return d_count ? *d_count : (int)fallback;
}

// Order-preserving map of floats to unsigned ints (for atomic min / max).
__device__ __forceinline__ uint32_t float_to_ordered(float f) {
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ordered_to_float(uint32_t b) {
    return __uint_as_float((b & 0x80000000u) ? (b & 0x7fffffffu) : ~b);
}

// x / t correctly rounded; for a power-of-two t, x times the exact 1 / t,
// which rounds the same real number once and so gives the same float.
__device__ __forceinline__ float div_by_size(float x, int t) {
    if ((t & (t - 1)) == 0) return __fmul_rn(x, __int_as_float((127 - (__ffs(t) - 1)) << 23));
    return __fdiv_rn(x, (float)t);
}

// Tile rectangle of a splat: tiles whose pixel square meets
// [u - r, u + r] x [v - r, v + r], end-exclusive, clamped to the grid.
// Single precision with explicit rounding so that every caller (and any
// reference) obtains the same integers.
__device__ __forceinline__ int4 tile_rect(float u, float v, float r, int tw, int th, int gx,
                                          int gy) {
    float x0 = floorf(div_by_size(__fsub_rn(u, r), tw));
    float x1 = __fadd_rn(floorf(div_by_size(__fadd_rn(u, r), tw)), 1.0f);
    float y0 = floorf(div_by_size(__fsub_rn(v, r), th));
    float y1 = __fadd_rn(floorf(div_by_size(__fadd_rn(v, r), th)), 1.0f);
    x0 = fminf(fmaxf(x0, 0.0f), (float)gx);
    x1 = fminf(fmaxf(x1, 0.0f), (float)gx);
    y0 = fminf(fmaxf(y0, 0.0f), (float)gy);
    y1 = fminf(fmaxf(y1, 0.0f), (float)gy);
    return make_int4((int)x0, (int)y0, (int)x1, (int)y1);
}

// A*dx^2 + 2*B*dx*dy + C*dy^2 with a fixed rounding order.
__device__ __forceinline__ float quad_form(float A, float B, float C, float dx, float dy) {
    const float t1 = __fmul_rn(__fmul_rn(A, dx), dx);
    const float t2 = __fmul_rn(__fmul_rn(__fmul_rn(B, dx), dy), 2.0f);
    const float t3 = __fmul_rn(__fmul_rn(C, dy), dy);
    return __fadd_rn(__fadd_rn(t1, t2), t3);
}

// Whether a box of pixel centres [xl, xh] x [yl, yh] can receive a
// contribution from a splat: the minimum of the conic's quadratic form
// q(d) = d^T [[A, B], [B, C]] d over the box (d = splat centre - pixel
// centre) is at most tau, where tau bounds q at alpha = 1/255
// (alpha = o exp(-q / 2)). The minimum is at most 0 if the box holds the
// centre (0 for a definite form, so a negative tau lists nothing), else it
// lies on an edge at the clamped one-dimensional minimiser
// (-B dx / C on an edge of constant dx; rA = 1/A and rC = 1/C, correctly
// rounded). Single precision, explicit rounding.
__device__ __forceinline__ bool box_reachable(float u, float v, float A, float B, float C,
                                              float rA, float rC, float tau, float xl, float xh,
                                              float yl, float yh) {
    const float ax = __fsub_rn(u, xh), bx = __fsub_rn(u, xl);
    const float ay = __fsub_rn(v, yh), by = __fsub_rn(v, yl);
    if (ax <= 0.0f && bx >= 0.0f && ay <= 0.0f && by >= 0.0f && tau >= 0.0f) return true;
    float d, q;
    d = fminf(fmaxf(-__fmul_rn(__fmul_rn(B, ax), rC), ay), by);
    q = quad_form(A, B, C, ax, d);
    d = fminf(fmaxf(-__fmul_rn(__fmul_rn(B, bx), rC), ay), by);
    q = fminf(q, quad_form(A, B, C, bx, d));
    d = fminf(fmaxf(-__fmul_rn(__fmul_rn(B, ay), rA), ax), bx);
    q = fminf(q, quad_form(A, B, C, d, ay));
    d = fminf(fmaxf(-__fmul_rn(__fmul_rn(B, by), rA), ax), bx);
    q = fminf(q, quad_form(A, B, C, d, by));
    return q <= tau;
}

// The same test for tile (tx, ty): its pixel centres span
// [tx tw + 0.5, tx tw + tw - 0.5] x [ty th + 0.5, ty th + th - 0.5].
__device__ __forceinline__ bool tile_reachable(float u, float v, float A, float B, float C,
                                               float rA, float rC, float tau, int tx, int ty,
                                               int tw, int th) {
    const float xl = __fadd_rn((float)(tx * tw), 0.5f), xh = __fadd_rn((float)(tx * tw + tw), -0.5f);
    const float yl = __fadd_rn((float)(ty * th), 0.5f), yh = __fadd_rn((float)(ty * th + th), -0.5f);
    return box_reachable(u, v, A, B, C, rA, rC, tau, xl, xh, yl, yh);
}

// Row form of the same test. Within a tile row (pixel-centre offsets
// d_y = v - y in [ay, by]) the ellipse q(d) <= tau covers one interval
// [L, U] of d_x = u - x: U is the largest d_x on the ellipse, reached at
// d_y = -B e_x / C (e_x = sqrt(tau C / det), det = AC - B^2) or, when that
// lies outside the slab, at the slab edge nearest to it, where the ellipse's
// quadratic in d_x gives U = (sqrt(A tau - det d_y^2) - B d_y) / A; L
// likewise with the signs flipped. A tile of the row is reachable when its
// offsets [u - xh, u - xl] meet [L, U] (u - xh <= U and u - xl >= L, the
// differences correctly rounded). Exact in real arithmetic, the same
// decision as the box minimum; evaluated with explicitly rounded single
// precision operations (no contraction), so every binning kernel takes the
// same decision. It agrees with the exact minimum wherever that is not
// within a few roundings of tau.
struct RowCull {
    float u, v, A, B, C, rA, rC, tau, det, ey, dyU;
    bool degenerate;  // det <= 0 after rounding: the box test decides
};

__device__ __forceinline__ RowCull row_cull(float u, float v, float A, float B, float C, float rA,
                                            float rC, float tau) {
    RowCull r;
    r.u = u; r.v = v; r.A = A; r.B = B; r.C = C; r.rA = rA; r.rC = rC; r.tau = tau;
    r.det = __fsub_rn(__fmul_rn(A, C), __fmul_rn(B, B));
    r.degenerate = !(r.det > 0.0f);
    const float ex = __fsqrt_rn(__fdiv_rn(__fmul_rn(tau, C), r.det));
    r.ey = __fsqrt_rn(__fdiv_rn(__fmul_rn(tau, A), r.det));
    r.dyU = -__fdiv_rn(__fmul_rn(B, ex), C);
    return r;
}

// [L, U] for the slab of pixel-centre rows [yl, yh]; false if the slab
// misses the ellipse.
__device__ __forceinline__ bool slab_interval(const RowCull &r, float yl, float yh, float &L,
                                              float &U) {
    if (!(r.tau >= 0.0f)) return false;
    const float ay = __fsub_rn(r.v, yh), by = __fsub_rn(r.v, yl);
    if (ay > r.ey || by < -r.ey) return false;
    const float At = __fmul_rn(r.A, r.tau);
    float d = fminf(fmaxf(r.dyU, ay), by);
    float D = fmaxf(__fsub_rn(At, __fmul_rn(r.det, __fmul_rn(d, d))), 0.0f);
    U = __fdiv_rn(__fsub_rn(__fsqrt_rn(D), __fmul_rn(r.B, d)), r.A);
    d = fminf(fmaxf(-r.dyU, ay), by);
    D = fmaxf(__fsub_rn(At, __fmul_rn(r.det, __fmul_rn(d, d))), 0.0f);
    L = __fdiv_rn(-__fadd_rn(__fsqrt_rn(D), __fmul_rn(r.B, d)), r.A);
    return true;
}

// [L, U] for tile row ty (pixel-centre rows ty th + 0.5 .. ty th + th - 0.5).
__device__ __forceinline__ bool row_interval(const RowCull &r, int ty, int th, float &L, float &U) {
    const float yl = __fadd_rn((float)(ty * th), 0.5f), yh = __fadd_rn((float)(ty * th + th), -0.5f);
    return slab_interval(r, yl, yh, L, U);
}

// ---------------------------------------------------------------------------
// host-side building blocks implemented in sort.cu
// ---------------------------------------------------------------------------

// Workspace bytes for a stable LSD radix sort of up to n (key, u32 value)
// pairs with `key_bytes`-byte keys (ping-pong buffers plus histograms).
size_t radix_sort_workspace(int64_t n, int key_bytes);

// Stable LSD radix sort of (key, value) pairs over the low `bits` bits of
// the key. The count is *d_n (device; NULL means n_max). The pairs start in
// (keys[0], vals[0]); keys[1] / vals[1] are the alternate buffers. Returns
// the index (0 or 1) of the buffers holding the result in *out_buf.
// `scratch` holds the digit histograms and the tiles' look-back status
// (radix_hist_bytes(n_max)); after the sort, u32 word 256 p + d of it is
// the number of keys whose digit in pass p (bits 8p..8p+7) is d. Bounded
// look-back waits that give up are counted; sort_wait_timeouts() reads and
// clears the count.
size_t radix_hist_bytes(int64_t n_max);
lgs_status sort_wait_timeouts(uint32_t *count);
// Polls of an unpublished predecessor after which the look-backs of the
// radix sort and of the binning give up (counted, see above); the default
// is kDefaultSpinLimit. A look-back that gives up takes the partial prefix
// it has summed, which is never larger than the true one, so every output
// position it computes stays below the true one and inside the output.
constexpr uint32_t kDefaultSpinLimit = 1u << 22;
lgs_status sort_set_spin_limit(uint32_t spins);
lgs_status bin_set_spin_limit(uint32_t spins);
// The same count for the binning's look-back over groups of splats.
lgs_status bin_wait_timeouts(uint32_t *count);
// 16-bit keys carry 64-bit values.
lgs_status radix_sort_u16_v64(uint16_t *keys[2], uint64_t *vals[2], int64_t n_max,
                              const int64_t *d_n64, const int32_t *d_n32, int bits, void *scratch,
                              int *out_buf, cudaStream_t s);
lgs_status radix_sort_u32(uint32_t *keys[2], uint32_t *vals[2], int64_t n_max, const int64_t *d_n64,
                          const int32_t *d_n32, int bits, void *scratch, int *out_buf,
                          cudaStream_t s);
lgs_status radix_sort_u64(uint64_t *keys[2], uint32_t *vals[2], int64_t n_max, const int64_t *d_n64,
                          const int32_t *d_n32, int bits, void *scratch, int *out_buf,
                          cudaStream_t s);

// Number of passes the sort makes for `bits` key bits.
int radix_passes(int bits);

// Exclusive scan of n_max u32 values (count *d_n32 if given) into 64-bit
// offsets; *d_total receives the sum. `scratch` of scan_scratch_bytes().
size_t scan_scratch_bytes();
lgs_status exclusive_scan_u32_to_u64(const uint32_t *in, uint64_t *out, int64_t n_max,
                                     const int32_t *d_n32, int64_t *d_total, void *scratch,
                                     cudaStream_t s);

}  // namespace lgs
