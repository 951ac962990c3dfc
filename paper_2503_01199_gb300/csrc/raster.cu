// Tile rasteriser, forward (Eq. 1-2, Alg. 1) and backward (Eq. 3, App. A.1
// Eq. 4-6) with the opacity-gradient moments of Sec. 3.3.
//
// A tile is 16 x 16 pixels in four 8 x 8 quadrants. The tile's sorted
// splats are staged through shared memory 128 at a time. While staging, each
// thread tests its splats against the four quadrants with the test the
// binning uses per tile (the minimum of the exponent's quadratic form over
// the quadrant's pixel centres against tau, in its row form: one x interval
// per 8-row slab), so that each quadrant walks only the splats that can
// reach it.
// One CTA of 4 warps per tile; warp w owns quadrant w and each lane a
// horizontal pair of pixels of it, in both passes.
// In the backward each lane first sums a splat's per-pixel terms over its
// two pixels (App. A.1's thread-local sum), the warp reduces the 12 sums
// (9 gradients, S, M and the fragment count) through a transpose in shared
// memory (value i ends on lanes 2i, 2i + 1) and one lane per value issues
// one atomic: one atomic per value per splat and quadrant
// (App. A.1 Eq. 5-6, the tile's reduction split over its four quadrant
// warps). The per-pixel exponent moments are summed as sum qq, sum dx qq and
// sum dx^2 qq over the lane's row (dy is the same for both pixels), which
// gives the five conic and centre sums with dy applied once per splat.
// The backward evaluates its two pixels with packed two-lane FP32
// operations (one instruction for the pair, each lane rounded as the scalar
// operation), from a staged splat that holds each value twice; the forward
// keeps scalar operations, which measured faster there (a lane leaves its
// splat loop when both its pixels have ended).
//
// The exponent is evaluated in base 2: power log2(e) = dx (a dx + b dy) +
// c dy^2 with a = -A log2(e) / 2, b = -B log2(e), c = -C log2(e) / 2, so that
// G is one ex2 per pixel, with explicitly rounded FP32 operations in one
// helper shared by both passes, pixel by pixel: the backward re-derives
// exactly the alphas the forward composited. In the mixed-precision variants
// the Gaussian value G, o G and alpha of a pair of pixels are one FP16x2 or
// BF16x2 value; the exponent (conic), transmittance, colour accumulators and
// gradient sums stay FP32.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lgs_internal.cuh"

namespace lgs {

namespace {

constexpr int kTile = 16;
constexpr int kFwdThreads = 128;  // four warps per tile, one per quadrant
constexpr int kBwdThreads = 128;
constexpr int kBatch = 128;       // splats staged per round, one per thread
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;
constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;

// A splat staged for the forward: 3 x 16 bytes, read with three vector loads.
struct __align__(16) SplatS {
    float u, v, a, b, c, o;  // centre, exponent coefficients (base 2), opacity
    float r, g, bl;          // colour
    uint32_t oh;             // o as a 16-bit pair (mixed precision only)
    uint32_t id;             // splat index (gradient row)
    float pad;
};

// A splat staged for the backward: 5 x 16 bytes. A lane works on two
// pixels at once in packed two-lane FP32 arithmetic (one instruction for both pixels, each
// lane rounded as the scalar operation), so every value it combines with a
// pixel pair is stored twice: a vector load then leaves the pair in a
// register pair.
struct __align__(16) SplatP {
    float2 u, v;     // centre
    float2 a, b, c;  // exponent coefficients (base 2)
    float2 o;        // opacity
    float2 r, g, bl; // colour
    uint32_t oh;     // o as a 16-bit pair (mixed precision only)
    uint32_t id;     // splat index (gradient row)
};

__device__ __forceinline__ float2 dup(float x) { return make_float2(x, x); }

struct RCam {
    int W, H, gx, ntiles;
    float bg[3];
    int64_t splat_rows, grad_rows;  // bounds the debug build checks indices against
};

// PREC = blend precision (LGS_FP32 / LGS_MIXED_FP16 / LGS_MIXED_BF16),
// optionally | LGS_WARP_REDUCE_INT for the backward's warp sums.
constexpr int kDetFlag = 64;  // internal: fixed-point accumulation (deterministic backward)
constexpr int blend_of(int prec) { return prec & 3; }
constexpr bool int_reduce(int prec) { return (prec & LGS_WARP_REDUCE_INT) != 0; }
constexpr bool det_of(int prec) { return (prec & kDetFlag) != 0; }

template <int PREC>
__device__ __forceinline__ uint32_t pack_pair(float x) {
    if constexpr (blend_of(PREC) == LGS_MIXED_FP16) {
        const __half2 h = __float2half2_rn(x);
        return *reinterpret_cast<const uint32_t *>(&h);
    } else if constexpr (blend_of(PREC) == LGS_MIXED_BF16) {
        const __nv_bfloat162 h = __float2bfloat162_rn(x);
        return *reinterpret_cast<const uint32_t *>(&h);
    } else {
        return 0u;
    }
}

__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Approximate square root for the quadrant test: x * rsqrt(x), 0 for
// x <= 0, and finite (about 1.8e19) for an infinite x.
__device__ __forceinline__ float sqrt_approx(float x) {
    x = fminf(x, 3.0e38f);
    return x > 0.0f ? x * rsqrtf(x) : 0.0f;
}

// Loads splat j into s and returns the 4-bit mask of the tile quadrants
// (bit 2 qr + qc: quadrant x0 + 8 qc, y0 + 8 qr) it may reach. The mask
// only saves work: a quadrant left out must have alpha < 1/255 at every
// pixel, so the test may be loose but never tight. It is the row form of
// the tile test (per quadrant row, the x interval [L, U] of the ellipse
// q <= tau) in approximate arithmetic (reciprocals and square roots by the
// special-function unit), with slack far above that arithmetic's error: the
// y extent and the interval are widened by 2e-3 of the ellipse's extent plus
// 1e-2 pixel. A conic that is not positive definite reaches every quadrant.
// The staged values of record j (x = u, v, A, B; y = C, o, r, g; z = b, tau):
// the conic scaled to base 2, o also as a 16-bit pair, the row index.
template <int PREC>
__device__ __forceinline__ void fill_splat(SplatS &s, float4 x, float4 y, float2 z, uint32_t j) {
    SplatS t;
    t.u = x.x;
    t.v = x.y;
    t.a = __fmul_rn(x.z, -0.5f * kLog2e);
    t.b = __fmul_rn(x.w, -kLog2e);
    t.c = __fmul_rn(y.x, -0.5f * kLog2e);
    t.o = y.y;
    t.r = y.z;
    t.g = y.w;
    t.bl = z.x;
    t.oh = pack_pair<PREC>(y.y);
    t.id = j;
    t.pad = 0.0f;
    s = t;
}

template <int PREC>
__device__ __forceinline__ void fill_splat(SplatP &s, float4 x, float4 y, float2 z, uint32_t j) {
    SplatP t;
    t.u = dup(x.x);
    t.v = dup(x.y);
    t.a = dup(__fmul_rn(x.z, -0.5f * kLog2e));
    t.b = dup(__fmul_rn(x.w, -kLog2e));
    t.c = dup(__fmul_rn(y.x, -0.5f * kLog2e));
    t.o = dup(y.y);
    t.r = dup(y.z);
    t.g = dup(y.w);
    t.bl = dup(z.x);
    t.oh = pack_pair<PREC>(y.y);
    t.id = j;
    s = t;
}

template <int PREC, class S>
__device__ __forceinline__ uint32_t stage(const float *__restrict__ rec, uint32_t j,
                                          int64_t nrows, float x0, float y0, S &s) {
    if (!LGS_DCHECK((int64_t)j < nrows, kSiteRasterSplat)) {
        fill_splat<PREC>(s, make_float4(0.f, 0.f, 0.f, 0.f), make_float4(0.f, 0.f, 0.f, 0.f),
                         make_float2(0.f, 0.f), 0u);
        return 0u;  // reaches no quadrant
    }
    const float4 *p = reinterpret_cast<const float4 *>(rec + 12 * (int64_t)j);
    const float4 x = __ldg(p), y = __ldg(p + 1);
    const float2 z = __ldg(reinterpret_cast<const float2 *>(rec + 12 * (int64_t)j + 8));
    fill_splat<PREC>(s, x, y, z, j);
    const float A = x.z, B = x.w, C = y.x, tau = z.y;
    if (!(tau >= 0.0f)) return 0u;
    const float det = A * C - B * B;
    if (!(det > 0.0f) || !(A > 0.0f) || !(C > 0.0f)) return 0xfu;
    const float rdet = __fdividef(1.0f, det), rA = __fdividef(1.0f, A);
    const float ex = sqrt_approx(tau * C * rdet), ey = sqrt_approx(tau * A * rdet);
    const float dyU = -B * ex * __fdividef(1.0f, C);
    const float sy = 2e-3f * ey + 1e-2f, sx = 2e-3f * ex + 1e-2f;
    const float At = A * tau;
    uint32_t m = 0;
#pragma unroll
    for (int qr = 0; qr < 2; ++qr) {
        const float yl = y0 + 8.0f * qr;
        const float ay = x.y - (yl + 7.0f), by = x.y - yl;
        if (ay > ey + sy || by < -(ey + sy)) continue;
        float d = fminf(fmaxf(dyU, ay), by);
        const float U = (sqrt_approx(At - det * d * d) - B * d) * rA + sx;
        d = fminf(fmaxf(-dyU, ay), by);
        const float L = -(sqrt_approx(At - det * d * d) + B * d) * rA - sx;
#pragma unroll
        for (int qc = 0; qc < 2; ++qc) {
            const float xl = x0 + 8.0f * qc;
            if (x.x - (xl + 7.0f) <= U && x.x - xl >= L) m |= 1u << (2 * qr + qc);
        }
    }
    return m;
}

// Exponent (base 2) at two horizontally adjacent pixel centres fx, fx + 1
// of a row whose terms b dy and c dy^2 are given.
__device__ __forceinline__ void power2(const SplatS &s, float fx, float bdy, float cdy2,
                                       float &dx0, float &dx1, float &p0, float &p1) {
    dx0 = __fsub_rn(s.u, fx);
    dx1 = __fsub_rn(s.u, __fadd_rn(fx, 1.0f));
    p0 = __fmaf_rn(dx0, __fmaf_rn(s.a, dx0, bdy), cdy2);
    p1 = __fmaf_rn(dx1, __fmaf_rn(s.a, dx1, bdy), cdy2);
}

// b dy and c dy^2 of the row at fy; dy = v - fy.
__device__ __forceinline__ void row_terms(const SplatS &s, float fy, float &dy, float &bdy,
                                          float &cdy2) {
    dy = __fsub_rn(s.v, fy);
    bdy = __fmul_rn(s.b, dy);
    cdy2 = __fmul_rn(__fmul_rn(s.c, dy), dy);
}

// G = 2^p, alpha = min(0.99, o G) and whether the clamp is active, for a
// pixel pair (elementwise: a pixel's values do not depend on its partner).
template <int PREC>
__device__ __forceinline__ void blend2(const SplatS &s, float p0, float p1, float &G0, float &G1,
                                       float &a0, float &a1, bool &cl0, bool &cl1) {
    if constexpr (blend_of(PREC) == LGS_FP32) {
        G0 = ex2(p0);
        G1 = ex2(p1);
        const float q0 = s.o * G0, q1 = s.o * G1;
        a0 = fminf(kAlphaMax, q0);
        a1 = fminf(kAlphaMax, q1);
        cl0 = q0 >= kAlphaMax;
        cl1 = q1 >= kAlphaMax;
    } else if constexpr (blend_of(PREC) == LGS_MIXED_FP16) {
        const __half2 g = h2exp2(__floats2half2_rn(p0, p1));
        const __half2 q = __hmul2(*reinterpret_cast<const __half2 *>(&s.oh), g);
        const __half2 cap = __float2half2_rn(kAlphaMax);
        const float2 Gf = __half22float2(g), af = __half22float2(__hmin2(q, cap));
        const __half2 ge = __hge2(q, cap);
        G0 = Gf.x;
        G1 = Gf.y;
        a0 = af.x;
        a1 = af.y;
        cl0 = __low2float(ge) != 0.0f;
        cl1 = __high2float(ge) != 0.0f;
    } else {
        const __nv_bfloat162 g = h2exp2(__floats2bfloat162_rn(p0, p1));
        const __nv_bfloat162 q = __hmul2(*reinterpret_cast<const __nv_bfloat162 *>(&s.oh), g);
        const __nv_bfloat162 cap = __float2bfloat162_rn(kAlphaMax);
        const float2 Gf = __bfloat1622float2(g), af = __bfloat1622float2(__hmin2(q, cap));
        const __nv_bfloat162 ge = __hge2(q, cap);
        G0 = Gf.x;
        G1 = Gf.y;
        a0 = af.x;
        a1 = af.y;
        cl0 = __low2float(ge) != 0.0f;
        cl1 = __high2float(ge) != 0.0f;
    }
}

// The backward's packed form of row_terms + power2: pixel centres
// (fx, fy) and (fx + 1, fy) given as nfx = (-fx, -(fx + 1)) and
// nfy = (-fy, -fy), so that the differences are packed additions:
// dy = v - fy (both lanes), dx = (u - fx, u - fx - 1), and the exponent
// p = dx (a dx + b dy) + c dy^2 at both pixels. Each lane performs the
// forward's scalar operation with the same rounding, so the backward
// re-derives exactly the exponents, and hence the alphas, the forward
// composited.
__device__ __forceinline__ void power_pair(const SplatP &s, float2 nfx, float2 nfy, float2 &dy,
                                           float2 &dx, float2 &p) {
    dy = __fadd2_rn(s.v, nfy);
    const float2 bdy = __fmul2_rn(s.b, dy);
    const float2 cdy2 = __fmul2_rn(__fmul2_rn(s.c, dy), dy);
    dx = __fadd2_rn(s.u, nfx);
    p = __ffma2_rn(dx, __ffma2_rn(s.a, dx, bdy), cdy2);
}

// The packed form of blend2 (the same operations per lane).
template <int PREC>
__device__ __forceinline__ void blend_pair(const SplatP &s, float2 p, float2 &G, float2 &al,
                                           bool &cl0, bool &cl1) {
    if constexpr (blend_of(PREC) == LGS_FP32) {
        G = make_float2(ex2(p.x), ex2(p.y));
        const float2 q = __fmul2_rn(s.o, G);
        al = make_float2(fminf(kAlphaMax, q.x), fminf(kAlphaMax, q.y));
        cl0 = q.x >= kAlphaMax;
        cl1 = q.y >= kAlphaMax;
    } else if constexpr (blend_of(PREC) == LGS_MIXED_FP16) {
        const __half2 g = h2exp2(__floats2half2_rn(p.x, p.y));
        const __half2 q = __hmul2(*reinterpret_cast<const __half2 *>(&s.oh), g);
        const __half2 cap = __float2half2_rn(kAlphaMax);
        const __half2 ge = __hge2(q, cap);
        G = __half22float2(g);
        al = __half22float2(__hmin2(q, cap));
        cl0 = __low2float(ge) != 0.0f;
        cl1 = __high2float(ge) != 0.0f;
    } else {
        const __nv_bfloat162 g = h2exp2(__floats2bfloat162_rn(p.x, p.y));
        const __nv_bfloat162 q = __hmul2(*reinterpret_cast<const __nv_bfloat162 *>(&s.oh), g);
        const __nv_bfloat162 cap = __float2bfloat162_rn(kAlphaMax);
        const __nv_bfloat162 ge = __hge2(q, cap);
        G = __bfloat1622float2(g);
        al = __bfloat1622float2(__hmin2(q, cap));
        cl0 = __low2float(ge) != 0.0f;
        cl1 = __high2float(ge) != 0.0f;
    }
}

template <class S>
struct RasterSmemT {
    S sp[kBatch];
    uint8_t fl[kBatch];
    int maxlast;
};
using RasterSmem = RasterSmemT<SplatS>;   // forward
using RasterSmemP = RasterSmemT<SplatP>;  // backward

// One tile of the forward pass, by the whole CTA (kFwdThreads): warp w
// owns quadrant w (x0 + 8 (w & 1), y0 + 8 (w >> 1)), lane l the pixels
// (2 (l & 3), l >> 2) and its right neighbour in it.
template <int PREC>
__device__ __forceinline__ void fwd_tile(const float *__restrict__ rec,
                                         const uint32_t *__restrict__ vals,
                                         const uint32_t *__restrict__ ranges, const RCam &K,
                                         int tile, float *__restrict__ image,
                                         float *__restrict__ finalT, int32_t *__restrict__ last,
                                         RasterSmem &sm) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tx = tile % K.gx, ty = tile / K.gx;
    const int x = tx * kTile + 8 * (w & 1) + 2 * (lane & 3), y = ty * kTile + 8 * (w >> 1) + (lane >> 2);
    const float fx = (float)x + 0.5f, fy = (float)y + 0.5f;
    const float tx0 = (float)(tx * kTile) + 0.5f, ty0 = (float)(ty * kTile) + 0.5f;
    const uint32_t r0 = ranges[2 * tile], r1 = ranges[2 * tile + 1];
    float T[2] = {1.0f, 1.0f}, cr[2] = {0.f, 0.f}, cg[2] = {0.f, 0.f}, cb[2] = {0.f, 0.f};
    int32_t lst[2] = {0, 0};
    uint32_t live = (x < K.W && y < K.H ? 1u : 0u) | (x + 1 < K.W && y < K.H ? 2u : 0u);
    for (uint32_t b0 = r0; b0 < r1; b0 += kBatch) {
        if (__syncthreads_count(live != 0) == 0) break;
        const uint32_t idx = b0 + threadIdx.x;
        if (idx < r1)
            sm.fl[threadIdx.x] = (uint8_t)stage<PREC>(rec, vals[idx], K.splat_rows, tx0, ty0, sm.sp[threadIdx.x]);
        __syncthreads();
        const int cnt = (int)min((uint32_t)kBatch, r1 - b0);
#pragma unroll 1
        for (int q = 0; q < kBatch / 32; ++q) {
            const int t = 32 * q + lane;
            uint32_t m = __ballot_sync(0xffffffffu, t < cnt && ((sm.fl[t] >> w) & 1u));
            while (m && live) {
                const int k = 32 * q + __ffs(m) - 1;
                m &= m - 1;
                const SplatS s = sm.sp[k];
                float dy, bdy, cdy2, dx0, dx1, p0, p1, G0, G1, a0, a1;
                bool c0, c1;
                row_terms(s, fy, dy, bdy, cdy2);
                power2(s, fx, bdy, cdy2, dx0, dx1, p0, p1);
                blend2<PREC>(s, p0, p1, G0, G1, a0, a1, c0, c1);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float a = h ? a1 : a0;
                    if (((live >> h) & 1u) && a >= kAlphaMin) {
                        const float Tn = T[h] * (1.0f - a);
                        if (Tn < kTMin) {
                            live &= ~(1u << h);
                        } else {
                            const float wgt = a * T[h];
                            cr[h] = fmaf(s.r, wgt, cr[h]);
                            cg[h] = fmaf(s.g, wgt, cg[h]);
                            cb[h] = fmaf(s.bl, wgt, cb[h]);
                            T[h] = Tn;
                            lst[h] = (int32_t)(b0 - r0) + k + 1;
                        }
                    }
                }
            }
        }
    }
    const int64_t hw = (int64_t)K.W * K.H;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        if (x + h < K.W && y < K.H) {
            const int64_t p = (int64_t)y * K.W + x + h;
            image[p] = cr[h] + T[h] * K.bg[0];
            image[hw + p] = cg[h] + T[h] * K.bg[1];
            image[2 * hw + p] = cb[h] + T[h] * K.bg[2];
            finalT[p] = T[h];
            last[p] = lst[h];
        }
    }
}

template <int PREC>
__global__ void __launch_bounds__(kFwdThreads) k_raster_fwd(const float *__restrict__ rec,
                                                            const uint32_t *__restrict__ vals,
                                                            const uint32_t *__restrict__ ranges,
                                                            RCam K, float *__restrict__ image,
                                                            float *__restrict__ finalT,
                                                            int32_t *__restrict__ last) {
    __shared__ RasterSmem sm;
    fwd_tile<PREC>(rec, vals, ranges, K, blockIdx.x, image, finalT, last, sm);
}

// Warp sums of 12 values through a transpose in shared memory: every lane
// stores its 12 values as column `lane` of a 12 x 32 block (rows padded to
// kRedStride floats, so that the 128-bit row reads below take no bank
// conflict), then lane 2i + h (i < 12) adds the 16 entries of row i in
// columns [16 h, 16 h + 16) in a fixed tree (packed two-lane additions down
// to two partial sums, then one addition) and one shuffle joins the two
// halves: lanes 2i and 2i + 1 both return the warp sum of value i, lanes
// 24..31 return 0. 12 stores, 4 loads, 9 additions and one shuffle in
// place of a butterfly's 13 shuffles and their selects; the order of the
// additions is fixed, so the result does not depend on timing.
constexpr int kRedValues = 12;
constexpr int kRedStride = 36;
__device__ __forceinline__ float warp_sum12(const float v[kRedValues], float *buf, int lane) {
#pragma unroll
    for (int i = 0; i < kRedValues; ++i) buf[i * kRedStride + lane] = v[i];
    __syncwarp();
    float r = 0.0f;
    if (lane < 2 * kRedValues) {
        const float4 *src =
            reinterpret_cast<const float4 *>(buf + (lane >> 1) * kRedStride + 16 * (lane & 1));
        const float4 p = src[0], q = src[1], t = src[2], u = src[3];
        const float2 a = __fadd2_rn(__fadd2_rn(make_float2(p.x, p.y), make_float2(p.z, p.w)),
                                    __fadd2_rn(make_float2(q.x, q.y), make_float2(q.z, q.w)));
        const float2 b = __fadd2_rn(__fadd2_rn(make_float2(t.x, t.y), make_float2(t.z, t.w)),
                                    __fadd2_rn(make_float2(u.x, u.y), make_float2(u.z, u.w)));
        const float2 c = __fadd2_rn(a, b);
        r = c.x + c.y;
    }
    r += __shfl_xor_sync(0xffffffffu, r, 1);
    __syncwarp();  // the block is reused by the warp's next splat
    return r;
}

// Warp sum by the integer warp reduction of Sec. 3.1: the largest exponent
// (warp max), every value scaled to an integer aligned to it (26 bits, so
// that 32 of them cannot overflow 32 bits), an exact integer warp sum: the
// sum is tot 2^(emax - 152) (0 when emax < 26, every |x| < 2^-100).
// Truncation costs at most 2^-25 of the largest term per lane; the sum does
// not depend on the order of the lanes.
__device__ __forceinline__ void warp_sum_int(float x, int &tot, uint32_t &emax) {
    const uint32_t e = (__float_as_uint(x) >> 23) & 0xffu;
    emax = __reduce_max_sync(0xffffffffu, e);
    tot = 0;
    if (emax < 26u) return;
    const float up = __uint_as_float((279u - emax) << 23);  // 2^(152 - emax)
    tot = __reduce_add_sync(0xffffffffu, __float2int_rz(x * up));
}

__device__ __forceinline__ float int_sum_value(int tot, uint32_t emax) {
    return emax < 26u ? 0.0f : (float)tot * __uint_as_float((emax - 25u) << 23);  // 2^(emax - 152)
}

// ---------------------------------------------------------------------------
// Order-independent accumulation (lgs_raster_bwd_deterministic). Every
// contribution M 2^k (M a signed integer: a float's significand, or the
// integer warp sum of Sec. 3.1's reduction with its exponent) is added as
// the 96-bit two's-complement integer N = M 2^(k + 64), i.e. in units of
// 2^-64, split into two limbs: bits 0-31 summed in an unsigned 64-bit word
// (2^32 contributions cannot overflow it) and bits 32-95 summed modulo 2^64
// in a second word. Integer addition commutes, so the limbs, and the value
// they make, do not depend on the order in which tiles and quadrants add to
// a splat. A contribution whose N would need more than 94 bits
// (|value| >= 2^30) is counted in g_det_overflow and left out; bits below
// 2^-64 are truncated toward zero (at most 2^-64 per contribution).
// ---------------------------------------------------------------------------
constexpr int kDetValues = 10;  // du dv dA dB dC do dr dg db S (M = do; C is an integer)
constexpr int kDetLimbs = 2;

__device__ unsigned int g_det_overflow;

__device__ __forceinline__ void fixed_add(unsigned long long *acc, long long M, int k) {
    if (M == 0) return;
    const bool neg = M < 0;
    const uint64_t mag = neg ? (uint64_t)(-M) : (uint64_t)M;
    const int sh = k + 64;
    uint64_t lo, hi;  // N = hi 2^32 + lo, lo < 2^32
    if (sh >= 0) {
        if (64 - __clzll((long long)mag) + sh > 94) {
            atomicAdd(&g_det_overflow, 1u);
            return;
        }
        // mag 2^sh: low 32 bits and the rest (at most 62 bits)
        if (sh >= 32) {
            lo = 0;
            hi = mag << (sh - 32);
        } else {
            lo = (mag << sh) & 0xffffffffull;
            hi = sh ? (mag >> (32 - sh)) : (mag >> 32);
        }
    } else {
        if (sh <= -64) return;
        const uint64_t t = mag >> (-sh);
        if (t == 0) return;
        lo = t & 0xffffffffull;
        hi = t >> 32;
    }
    if (neg) {  // -(hi 2^32 + lo) = hi' 2^32 + lo' with lo' in [0, 2^32)
        if (lo) {
            lo = (1ull << 32) - lo;
            hi = ~hi;  // -(hi + 1)
        } else {
            hi = ~hi + 1ull;
        }
    }
    atomicAdd(acc, (unsigned long long)lo);
    atomicAdd(acc + 1, (unsigned long long)hi);
}

// A float x = M 2^k exactly (M its signed significand).
__device__ __forceinline__ void fixed_add_float(unsigned long long *acc, float x) {
    const uint32_t b = __float_as_uint(x);
    const int E = (int)((b >> 23) & 0xffu);
    if (E == 255) {
        atomicAdd(&g_det_overflow, 1u);
        return;
    }
    const long long m = E ? (long long)((b & 0x7fffffu) | 0x800000u) : (long long)(b & 0x7fffffu);
    fixed_add(acc, (b >> 31) ? -m : m, (E ? E : 1) - 150);
}

// Rows of grad_acc from the limbs: for every row j < rows, value v of the
// kDetValues is (limb0 + limb1 2^32) 2^-64 taken as a signed 96-bit integer
// (limb1 modulo 2^64 carries the sign), rounded to double (the magnitude's
// two 64-bit halves converted separately) and then to float; M = do.
__global__ void __launch_bounds__(256) k_det_finalize(const unsigned long long *__restrict__ acc,
                                                     int64_t rows, float *__restrict__ gacc) {
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < rows;
         j += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long *a = acc + (size_t)j * (kDetValues * kDetLimbs);
        float *row = gacc + 16 * j;
#pragma unroll
        for (int v = 0; v < kDetValues; ++v) {
            const uint64_t l0 = a[kDetLimbs * v], l1 = a[kDetLimbs * v + 1];
            // 128-bit N = l0 + l1 2^32 with l1 sign-extended
            uint64_t lo = l0 + (l1 << 32);
            uint64_t hi = (uint64_t)((int64_t)l1 >> 32) + (lo < l0 ? 1ull : 0ull);
            const bool neg = (int64_t)hi < 0;
            if (neg) {
                lo = ~lo + 1ull;
                hi = ~hi + (lo == 0ull ? 1ull : 0ull);
            }
            const double d = ((double)hi * 18446744073709551616.0 + (double)lo) * 0x1p-64;
            row[v] = (float)(neg ? -d : d);
        }
        row[10] = row[5];
    }
}

// One tile of the backward pass, by the whole CTA (kBwdThreads): warp w
// owns quadrant w, lane l the pixel pair (2 (l & 3), l >> 2) of it, as in
// the forward.
template <int PREC>
__device__ __forceinline__ void bwd_tile(const float *__restrict__ rec,
                                         const uint32_t *__restrict__ vals,
                                         const uint32_t *__restrict__ ranges, const RCam &K,
                                         int tile, const float *__restrict__ finalT,
                                         const int32_t *__restrict__ last,
                                         const float *__restrict__ dLdI, float *__restrict__ gacc,
                                         unsigned long long *__restrict__ det, RasterSmemP &sm,
                                         float *red_buf) {
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tx = tile % K.gx, ty = tile / K.gx;
    const int x = tx * kTile + 8 * (w & 1) + 2 * (lane & 3), y = ty * kTile + 8 * (w >> 1) + (lane >> 2);
    const float fx = (float)x + 0.5f, fy = (float)y + 0.5f;
    const float tx0 = (float)(tx * kTile) + 0.5f, ty0 = (float)(ty * kTile) + 0.5f;
    const uint32_t r0 = ranges[2 * tile];
    const int64_t hw = (int64_t)K.W * K.H;
    // per pixel: transmittance (recovered back to front), dL/dI, T_final bg.dL/dI,
    // and acc.dL/dI with acc the colour composited behind the current splat
    float T[2], g0[2], g1[2], g2[2], bgT[2], accg[2];
    int32_t lst[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        T[h] = 1.0f;
        g0[h] = g1[h] = g2[h] = 0.0f;
        lst[h] = 0;
        if (x + h < K.W && y < K.H) {
            const int64_t p = (int64_t)y * K.W + x + h;
            T[h] = finalT[p];
            lst[h] = last[p];
            g0[h] = dLdI[p];
            g1[h] = dLdI[hw + p];
            g2[h] = dLdI[2 * hw + p];
        }
        bgT[h] = T[h] * (K.bg[0] * g0[h] + K.bg[1] * g1[h] + K.bg[2] * g2[h]);
        accg[h] = 0.0f;
    }
    // the same per-pixel state as pixel pairs for the packed arithmetic
    float2 T2 = make_float2(T[0], T[1]), acc = make_float2(accg[0], accg[1]);
    const float2 gI0 = make_float2(g0[0], g0[1]), gI1 = make_float2(g1[0], g1[1]),
                 gI2 = make_float2(g2[0], g2[1]), nbgT = make_float2(-bgT[0], -bgT[1]);
    const float2 nfx = make_float2(-fx, -__fadd_rn(fx, 1.0f)), nfy = dup(-fy);
    const float2 one = dup(1.0f), neg1 = dup(-1.0f);
    const int32_t wmax = __reduce_max_sync(0xffffffffu, max(lst[0], lst[1]));
    if (threadIdx.x == 0) sm.maxlast = 0;
    __syncthreads();
    if (lane == 0) atomicMax(&sm.maxlast, wmax);
    __syncthreads();
    const int maxlast = sm.maxlast;
    const int vi = lane < 2 * kRedValues ? lane >> 1 : -1;
    float *const wred = red_buf + w * (kRedValues * kRedStride);
    // positions maxlast-1 .. 0 of the tile list, 128 at a time from the back
    for (int end = maxlast; end > 0; end -= kBatch) {
        const int cnt = min(kBatch, end);
        __syncthreads();
        if ((int)threadIdx.x < cnt)
            sm.fl[threadIdx.x] =
                (uint8_t)stage<PREC>(rec, vals[r0 + end - 1 - threadIdx.x], K.splat_rows, tx0, ty0,
                                     sm.sp[threadIdx.x]);
        __syncthreads();
#pragma unroll 1
        for (int q = 0; q < kBatch / 32; ++q) {
            const int t = 32 * q + lane;
            uint32_t m = __ballot_sync(0xffffffffu, t < cnt && end - 1 - t < wmax &&
                                                        ((sm.fl[t] >> w) & 1u));
            while (m) {
                const int k = 32 * q + __ffs(m) - 1;
                m &= m - 1;
                const int pos = end - 1 - k;
                const SplatP &s = sm.sp[k];
                float2 dy, dx, p, G, al;
                bool cl0, cl1;
                power_pair(s, nfx, nfy, dy, dx, p);
                blend_pair<PREC>(s, p, G, al, cl0, cl1);
                // pixel h takes part when the splat is before its last
                // composited one and alpha >= 1/255 (m0, m1); its opacity
                // and exponent terms also need the clamp off. A pixel that
                // does not take part keeps T and acc exactly (factor 1,
                // weight 0) and adds zeros to every sum.
                const bool m0 = pos < lst[0] && al.x >= kAlphaMin;
                const bool m1 = pos < lst[1] && al.y >= kAlphaMin;
                if (!__any_sync(0xffffffffu, m0 || m1)) continue;  // no pixel of the warp takes part
                const float2 oma = __ffma2_rn(al, neg1, one);  // 1 - alpha
                const float2 rom = make_float2(m0 ? __fdividef(1.0f, oma.x) : 1.0f,
                                               m1 ? __fdividef(1.0f, oma.y) : 1.0f);
                const float2 Tk = __fmul2_rn(T2, rom);  // T before the splat
                // dd = colour . dL/dI - acc (acc: the colour behind the splat)
                float2 dd = __fmul2_rn(s.r, gI0);
                dd = __ffma2_rn(s.g, gI1, dd);
                dd = __ffma2_rn(s.bl, gI2, dd);
                dd = __ffma2_rn(acc, neg1, dd);
                const float2 dLda = __ffma2_rn(Tk, dd, __fmul2_rn(nbgT, rom));
                const float2 alm = make_float2(m0 ? al.x : 0.0f, m1 ? al.y : 0.0f);
                const float2 dLdam = make_float2(m0 && !cl0 ? dLda.x : 0.0f,
                                                 m1 && !cl1 ? dLda.y : 0.0f);
                const float2 wT = __fmul2_rn(alm, Tk);
                const float2 pr = __fmul2_rn(wT, gI0), pg = __fmul2_rn(wT, gI1),
                             pb = __fmul2_rn(wT, gI2);
                const float2 dLdo = __fmul2_rn(G, dLdam), qq = __fmul2_rn(al, dLdam);
                const float2 s2 = __fmul2_rn(dLdo, dLdo), qx = __fmul2_rn(dx, qq);
                const float2 qxx = __fmul2_rn(dx, qx);
                // lane sums over its pixels: colour, opacity, opacity moment,
                // and Q0 = sum qq, Q1 = sum dx qq, Q2 = sum dx^2 qq, qq = dL/dpower
                const float gr = pr.x + pr.y, gg = pg.x + pg.y, gb = pb.x + pb.y;
                const float dO = dLdo.x + dLdo.y, S = s2.x + s2.y;
                const float Q0 = qq.x + qq.y, Q1 = qx.x + qx.y, Q2 = qxx.x + qxx.y;
                const float n = (float)((m0 ? 1 : 0) + (m1 ? 1 : 0));
                acc = __ffma2_rn(alm, dd, acc);
                T2 = Tk;
                // with a, b, c in base 2: -(A sx + B sy) = ln2 (2 a sx + b sy),
                // likewise for v; sx = Q1, sy = dy Q0, sxx = Q2, sxy = dy Q1,
                // syy = dy^2 Q0. Then dL/do, dL/dcolour, S, M (= dL/do) and
                // the fragment count (exact in FP32).
                const float dys = dy.x, dyQ0 = dys * Q0;
                const float sa = s.a.x, sb = s.b.x, sc = s.c.x;
                float v[kRedValues];
                v[0] = kLn2 * (2.0f * sa * Q1 + sb * dyQ0);
                v[1] = kLn2 * (sb * Q1 + 2.0f * sc * dyQ0);
                v[2] = -0.5f * Q2;
                v[3] = -dys * Q1;
                v[4] = -0.5f * dys * dyQ0;
                v[5] = dO;
                v[6] = gr;
                v[7] = gg;
                v[8] = gb;
                v[9] = S;
                v[10] = dO;
                v[11] = n;
                if (!LGS_DCHECK((int64_t)s.id < K.grad_rows, kSiteRasterRow)) continue;
                float *row = gacc + 16 * (int64_t)s.id;
                unsigned long long *drow = det + (size_t)s.id * (kDetValues * kDetLimbs);
                if constexpr (int_reduce(PREC)) {
                    const int mi = lane >> 1;
                    int mt = 0;
                    uint32_t me = 0;
#pragma unroll
                    for (int i = 0; i < 10; ++i) {
                        int t;
                        uint32_t e;
                        warp_sum_int(v[i], t, e);
                        if (mi == i || (i == 5 && mi == 10)) {  // M = the opacity sum
                            mt = t;
                            me = e;
                        }
                    }
                    const uint32_t cnt_w = __reduce_add_sync(0xffffffffu, (uint32_t)n);
                    if ((lane & 1) == 0) {
                        if (mi < 11) {
                            if constexpr (det_of(PREC)) {
                                if (mi < kDetValues && me >= 26u)
                                    fixed_add(drow + kDetLimbs * mi, (long long)mt, (int)me - 152);
                            } else {
                                atomicAdd(row + mi, int_sum_value(mt, me));
                            }
                        } else if (mi == 11) {
                            atomicAdd(reinterpret_cast<unsigned int *>(row + 11), cnt_w);
                        }
                    }
                } else {
                    const float red = warp_sum12(v, wred, lane);
                    if ((lane & 1) == 0 && vi >= 0) {
                        if (vi == 11)
                            atomicAdd(reinterpret_cast<unsigned int *>(row + 11), (unsigned int)red);
                        else if constexpr (det_of(PREC)) {
                            if (vi < kDetValues) fixed_add_float(drow + kDetLimbs * vi, red);
                        } else {
                            atomicAdd(row + vi, red);
                        }
                    }
                }
            }
        }
    }
}

template <int PREC>
__global__ void __launch_bounds__(kBwdThreads) k_raster_bwd(
    const float *__restrict__ rec, const uint32_t *__restrict__ vals,
    const uint32_t *__restrict__ ranges, RCam K, const float *__restrict__ finalT,
    const int32_t *__restrict__ last, const float *__restrict__ dLdI, float *__restrict__ gacc,
    unsigned long long *__restrict__ det) {
    __shared__ RasterSmemP sm;
    __shared__ __align__(16) float red[(kBwdThreads / 32) * kRedValues * kRedStride];
    bwd_tile<PREC>(rec, vals, ranges, K, blockIdx.x, finalT, last, dLdI, gacc, det, sm, red);
}

// ---------------------------------------------------------------------------
// Batched views: persistent CTAs take tiles of all views from one atomic
// counter (tiles numbered view by view from each view's tile_offset).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int view_of(const lgs_view *views, int n_views, uint32_t t) {
    int v = 0;
    while (v + 1 < n_views && views[v + 1].tile_offset <= t) ++v;
    return v;
}

__device__ __forceinline__ RCam view_rcam(const lgs_view &V) {
    RCam K;
    K.W = V.width;
    K.H = V.height;
    K.gx = (V.width + kTile - 1) / kTile;
    K.ntiles = K.gx * ((V.height + kTile - 1) / kTile);
    K.bg[0] = V.bg[0];
    K.bg[1] = V.bg[1];
    K.bg[2] = V.bg[2];
    K.splat_rows = K.grad_rows = INT64_MAX;  // a view carries no row counts
    return K;
}

template <int PREC>
__global__ void __launch_bounds__(kFwdThreads) k_raster_fwd_batch(const lgs_view *__restrict__ views,
                                                             int n_views, uint32_t total_tiles,
                                                             uint32_t *counter) {
    __shared__ RasterSmem sm;
    __shared__ uint32_t s_tile;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t t = s_tile;
        if (t >= total_tiles) break;
        const int v = view_of(views, n_views, t);
        const lgs_view &V = views[v];
        const RCam K = view_rcam(V);
        fwd_tile<PREC>(V.rec, V.vals, V.tile_ranges, K, (int)(t - V.tile_offset), V.image,
                       V.final_T, V.last_contrib, sm);
        __syncthreads();
    }
}

template <int PREC>
__global__ void __launch_bounds__(kBwdThreads) k_raster_bwd_batch(const lgs_view *__restrict__ views,
                                                             int n_views, uint32_t total_tiles,
                                                             uint32_t *counter) {
    __shared__ RasterSmemP sm;
    __shared__ __align__(16) float red[(kBwdThreads / 32) * kRedValues * kRedStride];
    __shared__ uint32_t s_tile;
    for (;;) {
        if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1u);
        __syncthreads();
        const uint32_t t = s_tile;
        if (t >= total_tiles) break;
        const int v = view_of(views, n_views, t);
        const lgs_view &V = views[v];
        const RCam K = view_rcam(V);
        bwd_tile<PREC>(V.rec, V.vals, V.tile_ranges, K, (int)(t - V.tile_offset), V.final_T,
                       V.last_contrib, V.dL_dimage, V.grad_acc, nullptr, sm, red);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_loss_l1(const float *__restrict__ img,
                                                const float *__restrict__ tgt, int64_t n,
                                                float *__restrict__ g, float *loss) {
    float s = 0.f;
    const float inv = 1.0f / (float)n;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float d = img[i] - tgt[i];
        s += fabsf(d);
        g[i] = d > 0.f ? inv : (d < 0.f ? -inv : 0.f);
    }
    // block sum, then one atomic per block
    __shared__ float s_part[8];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < 8 ? s_part[threadIdx.x] : 0.f;
        for (int o = 4; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (threadIdx.x == 0) atomicAdd(loss, s * inv);
    }
}

__global__ void __launch_bounds__(256) k_variance(const float *__restrict__ gacc,
                                                 const uint32_t *__restrict__ map,
                                                 const int32_t *d_V, int64_t max_rows,
                                                 float *__restrict__ out) {
    const int64_t V = load_count(d_V, max_rows);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < V;
         j += (int64_t)gridDim.x * blockDim.x) {
        const float S = gacc[16 * j + 9], M = gacc[16 * j + 10];
        const uint32_t C = reinterpret_cast<const uint32_t *>(gacc)[16 * j + 11];
        out[map ? map[j] : j] = C ? S - M * M / (float)C : 0.f;
    }
}

RCam make_rcam(const lgs_camera *c, int tw, int th, int64_t splat_rows, int64_t grad_rows) {
    RCam k;
    k.splat_rows = splat_rows;
    k.grad_rows = grad_rows;
    k.W = c->width;
    k.H = c->height;
    k.gx = (int)ceil_div(c->width, tw);
    k.ntiles = k.gx * (int)ceil_div(c->height, th);
    k.bg[0] = c->bg[0]; k.bg[1] = c->bg[1]; k.bg[2] = c->bg[2];
    return k;
}

}  // namespace

DEBUG_TU(raster)

lgs_status raster_fwd(const lgs_splats *sp, const uint32_t *vals, const uint32_t *ranges,
                      const lgs_camera *cam, int tw, int th, int precision, float *image,
                      float *finalT, int32_t *last, cudaStream_t s) {
    if (tw != kTile || th != kTile) return LGS_ERR_INVALID_ARG;
    const RCam K = make_rcam(cam, tw, th, sp->capacity, INT64_MAX);
    const unsigned grid = (unsigned)K.ntiles;
    count_launch();
    switch (precision) {
        case LGS_FP32:
            k_raster_fwd<LGS_FP32><<<grid, kFwdThreads, 0, s>>>(sp->rec, vals, ranges, K, image, finalT, last);
            break;
        case LGS_MIXED_FP16:
            k_raster_fwd<LGS_MIXED_FP16><<<grid, kFwdThreads, 0, s>>>(sp->rec, vals, ranges, K, image, finalT, last);
            break;
        case LGS_MIXED_BF16:
            k_raster_fwd<LGS_MIXED_BF16><<<grid, kFwdThreads, 0, s>>>(sp->rec, vals, ranges, K, image, finalT, last);
            break;
        default:
            return LGS_ERR_INVALID_ARG;
    }
    return check_launch();
}

lgs_status raster_bwd(const lgs_splats *sp, const uint32_t *vals, const uint32_t *ranges,
                      const lgs_camera *cam, int tw, int th, int precision, const float *finalT,
                      const int32_t *last, const float *dLdI, float *gacc, int64_t max_splats,
                      int accumulate, cudaStream_t s) {
    if (tw != kTile || th != kTile) return LGS_ERR_INVALID_ARG;
    if ((precision & ~LGS_WARP_REDUCE_INT) < LGS_FP32 || (precision & ~LGS_WARP_REDUCE_INT) > LGS_MIXED_BF16)
        return LGS_ERR_INVALID_ARG;
    if (!accumulate) cudaMemsetAsync(gacc, 0, (size_t)max_splats * 16 * sizeof(float), s);
    const RCam K = make_rcam(cam, tw, th, sp->capacity, max_splats);
    const unsigned grid = (unsigned)K.ntiles;
    count_launch();
#define LGS_RBW(P) k_raster_bwd<P><<<grid, kBwdThreads, 0, s>>>(sp->rec, vals, ranges, K, finalT, last, dLdI, gacc, nullptr)
    switch (precision) {
        case LGS_FP32: LGS_RBW(LGS_FP32); break;
        case LGS_MIXED_FP16: LGS_RBW(LGS_MIXED_FP16); break;
        case LGS_MIXED_BF16: LGS_RBW(LGS_MIXED_BF16); break;
        case LGS_FP32 | LGS_WARP_REDUCE_INT: LGS_RBW(LGS_FP32 | LGS_WARP_REDUCE_INT); break;
        case LGS_MIXED_FP16 | LGS_WARP_REDUCE_INT: LGS_RBW(LGS_MIXED_FP16 | LGS_WARP_REDUCE_INT); break;
        default: LGS_RBW(LGS_MIXED_BF16 | LGS_WARP_REDUCE_INT); break;
    }
#undef LGS_RBW
    return check_launch();
}

size_t raster_bwd_det_workspace_size(int64_t max_splats) {
    return (size_t)(max_splats > 0 ? max_splats : 0) * kDetValues * kDetLimbs *
           sizeof(unsigned long long);
}

lgs_status raster_bwd_det(const lgs_splats *sp, const uint32_t *vals, const uint32_t *ranges,
                          const lgs_camera *cam, int tw, int th, int precision, const float *finalT,
                          const int32_t *last, const float *dLdI, float *gacc, int64_t max_splats,
                          void *ws, size_t ws_bytes, cudaStream_t s) {
    if (tw != kTile || th != kTile) return LGS_ERR_INVALID_ARG;
    if ((precision & ~LGS_WARP_REDUCE_INT) < LGS_FP32 || (precision & ~LGS_WARP_REDUCE_INT) > LGS_MIXED_BF16)
        return LGS_ERR_INVALID_ARG;
    const size_t need = raster_bwd_det_workspace_size(max_splats);
    if (ws_bytes < need || (need && !ws)) return LGS_ERR_INVALID_ARG;
    unsigned long long *det = static_cast<unsigned long long *>(ws);
    cudaMemsetAsync(gacc, 0, (size_t)max_splats * 16 * sizeof(float), s);
    cudaMemsetAsync(det, 0, need, s);
    const RCam K = make_rcam(cam, tw, th, sp->capacity, max_splats);
    const unsigned grid = (unsigned)K.ntiles;
    count_launch();
#define LGS_RBD(P) k_raster_bwd<(P) | kDetFlag><<<grid, kBwdThreads, 0, s>>>(sp->rec, vals, ranges, K, finalT, last, dLdI, gacc, det)
    switch (precision) {
        case LGS_FP32: LGS_RBD(LGS_FP32); break;
        case LGS_MIXED_FP16: LGS_RBD(LGS_MIXED_FP16); break;
        case LGS_MIXED_BF16: LGS_RBD(LGS_MIXED_BF16); break;
        case LGS_FP32 | LGS_WARP_REDUCE_INT: LGS_RBD(LGS_FP32 | LGS_WARP_REDUCE_INT); break;
        case LGS_MIXED_FP16 | LGS_WARP_REDUCE_INT: LGS_RBD(LGS_MIXED_FP16 | LGS_WARP_REDUCE_INT); break;
        default: LGS_RBD(LGS_MIXED_BF16 | LGS_WARP_REDUCE_INT); break;
    }
#undef LGS_RBD
    lgs_status st = check_launch();
    if (st != LGS_OK) return st;
    if (max_splats > 0) {
        count_launch();
        k_det_finalize<<<grid_for(max_splats, 256), 256, 0, s>>>(det, max_splats, gacc);
        st = check_launch();
    }
    return st;
}

lgs_status det_overflow(uint32_t *count) {
    unsigned int h = 0, zero = 0;
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpyFromSymbol(&h, g_det_overflow, sizeof(h)) != cudaSuccess ||
        cudaMemcpyToSymbol(g_det_overflow, &zero, sizeof(zero)) != cudaSuccess) {
        set_cuda_error(cudaGetLastError());
        return LGS_ERR_CUDA;
    }
    *count = h;
    return h ? LGS_ERR_CAPACITY : LGS_OK;
}

lgs_status raster_batch(const lgs_view *views, int n_views, uint32_t total_tiles, int precision,
                        uint32_t *counter, int backward, cudaStream_t s) {
    cudaMemsetAsync(counter, 0, sizeof(uint32_t), s);
    int per_sm = 0;
    if (backward)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_raster_bwd_batch<LGS_FP32>, kBwdThreads, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_raster_fwd_batch<LGS_FP32>, kFwdThreads, 0);
    const int64_t cap = (int64_t)num_sms() * (per_sm > 0 ? per_sm : 1);
    const unsigned grid = (unsigned)(total_tiles < cap ? total_tiles : cap);
    if (grid == 0) return LGS_OK;
    count_launch();
#define LGS_RB(P) do { if (backward) k_raster_bwd_batch<P><<<grid, kBwdThreads, 0, s>>>(views, n_views, total_tiles, counter); \
                       else k_raster_fwd_batch<blend_of(P)><<<grid, kFwdThreads, 0, s>>>(views, n_views, total_tiles, counter); } while (0)
    switch (precision) {
        case LGS_MIXED_FP16: LGS_RB(LGS_MIXED_FP16); break;
        case LGS_MIXED_BF16: LGS_RB(LGS_MIXED_BF16); break;
        case LGS_FP32 | LGS_WARP_REDUCE_INT: LGS_RB(LGS_FP32 | LGS_WARP_REDUCE_INT); break;
        case LGS_MIXED_FP16 | LGS_WARP_REDUCE_INT: LGS_RB(LGS_MIXED_FP16 | LGS_WARP_REDUCE_INT); break;
        case LGS_MIXED_BF16 | LGS_WARP_REDUCE_INT: LGS_RB(LGS_MIXED_BF16 | LGS_WARP_REDUCE_INT); break;
        default: LGS_RB(LGS_FP32); break;
    }
#undef LGS_RB
    return check_launch();
}

lgs_status loss_l1(const float *img, const float *tgt, int64_t n, float *g, float *loss,
                   cudaStream_t s) {
    cudaMemsetAsync(loss, 0, sizeof(float), s);
    count_launch();
    k_loss_l1<<<grid_for(n, 256, 4), 256, 0, s>>>(img, tgt, n, g, loss);
    return check_launch();
}

lgs_status opacity_variance(const float *gacc, const uint32_t *map, const int32_t *d_V,
                            int64_t max_rows, float *out, cudaStream_t s) {
    count_launch();
    k_variance<<<grid_for(max_rows, 256), 256, 0, s>>>(gacc, map, d_V, max_rows, out);
    return check_launch();
}

}  // namespace lgs
