// Tile rasteriser, forward (Eq. 1-2, Alg. 1) and backward (Eq. 3, App. A.1
// Eq. 4-6) with the opacity-gradient moments of Sec. 3.3.
//
// One CTA of 4 warps per 16 x 16 tile; warp w owns the 8 x 8 quadrant w of
// the tile and every thread a horizontal pair of pixels. The tile's sorted
// splats are staged through shared memory 128 at a time (one per thread).
// While staging, each thread tests its splat against the four quadrants
// with the test the binning uses per tile (the minimum of the exponent's
// quadratic form over the quadrant's pixel centres against tau, in its row
// form: one x interval per 8-row slab), so each warp walks only the splats
// that can reach its quadrant.
// In the backward each thread first sums a splat's per-pixel terms over its
// two pixels, the warp reduces the 12 sums with a reduce-scatter butterfly
// (16 shuffles; value i ends on lanes 2i, 2i + 1) and lanes 0, 2, .., 22
// issue one atomic each (App. A.1 Eq. 5-6: one atomic per value per warp).
//
// The exponent is power = dx (a dx + b dy) + c dy^2 with a = -A/2, b = -B,
// c = -C/2, evaluated with explicitly rounded FP32 operations in one helper
// shared by both passes, so the backward re-derives exactly the alphas the
// forward composited. In the mixed-precision variants the Gaussian value G,
// o G and alpha are computed for the pixel pair as one FP16x2 or BF16x2
// value; the exponent (conic), transmittance, colour accumulators and
// gradient sums stay FP32.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lgs_internal.cuh"

namespace lgs {

namespace {

constexpr int kTile = 16;
constexpr int kBatch = 128;  // threads per CTA = splats staged per round
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

struct SplatS {
    float u, v, a, b, c, o, r, g, bl;
    uint32_t oh;  // o as a 16-bit pair (mixed precision only)
};

struct RCam {
    int W, H, gx, ntiles;
    float bg[3];
};

// PREC = blend precision (LGS_FP32 / LGS_MIXED_FP16 / LGS_MIXED_BF16),
// optionally | LGS_WARP_REDUCE_INT for the backward's warp sums.
constexpr int blend_of(int prec) { return prec & 3; }
constexpr bool int_reduce(int prec) { return (prec & LGS_WARP_REDUCE_INT) != 0; }

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

// Approximate square root for the quadrant test: x * rsqrt(x), 0 for
// x <= 0, and finite (about 1.8e19) for an infinite x.
__device__ __forceinline__ float sqrt_approx(float x) {
    x = fminf(x, 3.0e38f);
    return x > 0.0f ? x * rsqrtf(x) : 0.0f;
}

// Loads splat j into s and returns the 4-bit mask of the tile quadrants
// (bit w: quadrant x0 + 8 (w & 1), y0 + 8 (w >> 1)) it may reach. The mask
// only saves work: a quadrant left out must have alpha < 1/255 at every
// pixel, so the test may be loose but never tight. It is the row form of
// the tile test (per quadrant row, the x interval [L, U] of the ellipse
// q <= tau) in approximate arithmetic (reciprocals and square roots by the
// special-function unit), with slack far above that arithmetic's error: the
// y extent and the interval are widened by 2e-3 of the ellipse's extent plus
// 1e-2 pixel. A conic that is not positive definite reaches every quadrant.
template <int PREC>
__device__ __forceinline__ uint32_t stage(const float *__restrict__ rec, uint32_t j, float x0,
                                          float y0, SplatS &s) {
    const float4 *p = reinterpret_cast<const float4 *>(rec + 12 * (int64_t)j);
    const float4 x = __ldg(p), y = __ldg(p + 1);
    const float2 z = __ldg(reinterpret_cast<const float2 *>(rec + 12 * (int64_t)j + 8));
    s.u = x.x;
    s.v = x.y;
    s.a = -0.5f * x.z;
    s.b = -x.w;
    s.c = -0.5f * y.x;
    s.o = y.y;
    s.r = y.z;
    s.g = y.w;
    s.bl = z.x;
    s.oh = pack_pair<PREC>(y.y);
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

// Exponent at two horizontally adjacent pixels of one row.
__device__ __forceinline__ void power2(const SplatS &s, float fx, float fy, float &p0,
                                       float &p1) {
    const float dx0 = __fsub_rn(s.u, fx), dx1 = __fsub_rn(s.u, __fadd_rn(fx, 1.0f));
    const float dy = __fsub_rn(s.v, fy);
    const float bdy = __fmul_rn(s.b, dy), cdy2 = __fmul_rn(__fmul_rn(s.c, dy), dy);
    p0 = __fmaf_rn(dx0, __fmaf_rn(s.a, dx0, bdy), cdy2);
    p1 = __fmaf_rn(dx1, __fmaf_rn(s.a, dx1, bdy), cdy2);
}

// G = exp(power), alpha = min(0.99, o G) and whether the clamp is active,
// for a pixel pair.
template <int PREC>
__device__ __forceinline__ void blend2(const SplatS &s, float p0, float p1, float &G0, float &G1,
                                       float &a0, float &a1, bool &cl0, bool &cl1) {
    if constexpr (blend_of(PREC) == LGS_FP32) {
        G0 = __expf(p0);
        G1 = __expf(p1);
        const float q0 = s.o * G0, q1 = s.o * G1;
        a0 = fminf(kAlphaMax, q0);
        a1 = fminf(kAlphaMax, q1);
        cl0 = q0 >= kAlphaMax;
        cl1 = q1 >= kAlphaMax;
    } else if constexpr (blend_of(PREC) == LGS_MIXED_FP16) {
        const __half2 G = h2exp(__floats2half2_rn(p0, p1));
        const __half2 q = __hmul2(*reinterpret_cast<const __half2 *>(&s.oh), G);
        const __half2 cap = __float2half2_rn(kAlphaMax);
        const float2 Gf = __half22float2(G), af = __half22float2(__hmin2(q, cap));
        const __half2 ge = __hge2(q, cap);
        G0 = Gf.x;
        G1 = Gf.y;
        a0 = af.x;
        a1 = af.y;
        cl0 = __low2float(ge) != 0.0f;
        cl1 = __high2float(ge) != 0.0f;
    } else {
        const __nv_bfloat162 G = h2exp(__floats2bfloat162_rn(p0, p1));
        const __nv_bfloat162 q = __hmul2(*reinterpret_cast<const __nv_bfloat162 *>(&s.oh), G);
        const __nv_bfloat162 cap = __float2bfloat162_rn(kAlphaMax);
        const float2 Gf = __bfloat1622float2(G), af = __bfloat1622float2(__hmin2(q, cap));
        const __nv_bfloat162 ge = __hge2(q, cap);
        G0 = Gf.x;
        G1 = Gf.y;
        a0 = af.x;
        a1 = af.y;
        cl0 = __low2float(ge) != 0.0f;
        cl1 = __high2float(ge) != 0.0f;
    }
}

// One tile of the forward pass, by the whole CTA.
template <int PREC>
__device__ __forceinline__ void fwd_tile(const float *__restrict__ rec,
                                         const uint32_t *__restrict__ vals,
                                         const uint32_t *__restrict__ ranges, const RCam &K,
                                         int tile, float *__restrict__ image,
                                         float *__restrict__ finalT, int32_t *__restrict__ last,
                                         SplatS *s_sp, uint8_t *s_fl) {
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
        if (idx < r1) s_fl[threadIdx.x] = (uint8_t)stage<PREC>(rec, vals[idx], tx0, ty0, s_sp[threadIdx.x]);
        __syncthreads();
        const int cnt = (int)min((uint32_t)kBatch, r1 - b0);
#pragma unroll 1
        for (int q = 0; q < kBatch / 32; ++q) {
            const int t = 32 * q + lane;
            uint32_t m = __ballot_sync(0xffffffffu, t < cnt && ((s_fl[t] >> w) & 1u));
            while (m && live) {
                const int k = 32 * q + __ffs(m) - 1;
                m &= m - 1;
                const SplatS s = s_sp[k];
                float p0, p1, G0, G1, a0, a1;
                bool c0, c1;
                power2(s, fx, fy, p0, p1);
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
        __syncthreads();
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
__global__ void __launch_bounds__(kBatch) k_raster_fwd(const float *__restrict__ rec,
                                                     const uint32_t *__restrict__ vals,
                                                     const uint32_t *__restrict__ ranges, RCam K,
                                                     float *__restrict__ image,
                                                     float *__restrict__ finalT,
                                                     int32_t *__restrict__ last) {
    __shared__ SplatS s_sp[kBatch];
    __shared__ uint8_t s_fl[kBatch];
    fwd_tile<PREC>(rec, vals, ranges, K, blockIdx.x, image, finalT, last, s_sp, s_fl);
}

// Reduce-scatter of 10 values across the warp in 12 shuffles (halving the
// vector at every butterfly stage, odd lengths padded with a zero): on
// return, the two lanes 2i, 2i + 1 hold the warp sum of value
// scatter10_index(2i), or a padding zero when that index is negative.
__device__ __forceinline__ float warp_reduce_scatter10(const float v[10], int lane) {
    float w[6], x[4], y[2];
    {
        const bool up = lane & 16;  // 10 -> 5
#pragma unroll
        for (int i = 0; i < 5; ++i) {
            const float send = up ? v[i] : v[i + 5];
            const float keep = up ? v[i + 5] : v[i];
            w[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
        }
        w[5] = 0.0f;
    }
    {
        const bool up = lane & 8;  // 5 (+1) -> 3
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const float send = up ? w[i] : w[i + 3];
            const float keep = up ? w[i + 3] : w[i];
            x[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
        }
        x[3] = 0.0f;
    }
    {
        const bool up = lane & 4;  // 3 (+1) -> 2
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const float send = up ? x[i] : x[i + 2];
            const float keep = up ? x[i + 2] : x[i];
            y[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
        }
    }
    const bool up = lane & 2;  // 2 -> 1
    const float z = (up ? y[1] : y[0]) + __shfl_xor_sync(0xffffffffu, up ? y[0] : y[1], 2);
    return z + __shfl_xor_sync(0xffffffffu, z, 1);
}

// The value index warp_reduce_scatter10 leaves in `lane`: 5 b4 + 3 b3 +
// 2 b2 + b1 (b_k = bit k of the lane) when that slot holds a value, else -1.
__device__ __forceinline__ int scatter10_index(int lane) {
    const int b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1;
    const int loc = 2 * ((lane >> 2) & 1) + ((lane >> 1) & 1);
    return loc < (b3 ? 2 : 3) ? 5 * b4 + 3 * b3 + loc : -1;
}

// Warp sum by the integer warp reduction of Sec. 3.1: the largest exponent
// (warp max), every value scaled to an integer aligned to it (26 bits, so
// that 32 of them cannot overflow 32 bits), an exact integer warp sum, and
// the float result rebuilt. Truncation costs at most 2^-25 of the largest
// term per lane; the sum does not depend on the order of the lanes.
__device__ __forceinline__ float warp_sum_int(float x) {
    const uint32_t e = (__float_as_uint(x) >> 23) & 0xffu;
    const uint32_t emax = __reduce_max_sync(0xffffffffu, e);
    if (emax < 26u) return 0.0f;  // every |x| < 2^-100
    const float up = __uint_as_float((279u - emax) << 23);  // 2^(152 - emax)
    const int q = __float2int_rz(x * up);
    const int tot = __reduce_add_sync(0xffffffffu, q);
    return (float)tot * __uint_as_float((emax - 25u) << 23);  // 2^(emax - 152)
}

// One tile of the backward pass, by the whole CTA.
template <int PREC>
__device__ __forceinline__ void bwd_tile(const float *__restrict__ rec,
                                         const uint32_t *__restrict__ vals,
                                         const uint32_t *__restrict__ ranges, const RCam &K,
                                         int tile, const float *__restrict__ finalT,
                                         const int32_t *__restrict__ last,
                                         const float *__restrict__ dLdI, float *__restrict__ gacc,
                                         SplatS *s_sp, uint32_t *s_id, uint8_t *s_fl,
                                         int &s_maxlast) {
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
    const int32_t wmax = __reduce_max_sync(0xffffffffu, max(lst[0], lst[1]));
    if (threadIdx.x == 0) s_maxlast = 0;
    __syncthreads();
    if (lane == 0) atomicMax(&s_maxlast, wmax);
    __syncthreads();
    const int maxlast = s_maxlast;
    // positions maxlast-1 .. 0 of the tile list, 128 at a time from the back
    for (int end = maxlast; end > 0; end -= kBatch) {
        const int cnt = min(kBatch, end);
        __syncthreads();
        if ((int)threadIdx.x < cnt) {
            const uint32_t j = vals[r0 + end - 1 - threadIdx.x];
            s_id[threadIdx.x] = j;
            s_fl[threadIdx.x] = (uint8_t)stage<PREC>(rec, j, tx0, ty0, s_sp[threadIdx.x]);
        }
        __syncthreads();
#pragma unroll 1
        for (int q = 0; q < kBatch / 32; ++q) {
            const int t = 32 * q + lane;
            uint32_t m = __ballot_sync(0xffffffffu, t < cnt && end - 1 - t < wmax &&
                                                        ((s_fl[t] >> w) & 1u));
            while (m) {
                const int k = 32 * q + __ffs(m) - 1;
                m &= m - 1;
                const int pos = end - 1 - k;
                const SplatS s = s_sp[k];
                float v[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) v[i] = 0.f;
                float p0, p1, G0, G1, a0, a1;
                bool c0, c1;
                power2(s, fx, fy, p0, p1);
                blend2<PREC>(s, p0, p1, G0, G1, a0, a1, c0, c1);
                float gr = 0.f, gg = 0.f, gb = 0.f, sx = 0.f, sy = 0.f, sxx = 0.f, sxy = 0.f,
                      syy = 0.f, dO = 0.f, S = 0.f;
                uint32_t n = 0;
                const float dy = __fsub_rn(s.v, fy);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float a = h ? a1 : a0;
                    if (pos < lst[h] && a >= kAlphaMin) {
                        const float G = h ? G1 : G0;
                        const bool clamped = h ? c1 : c0;
                        const float rom = __fdividef(1.0f, 1.0f - a);
                        const float Tk = T[h] * rom;
                        const float dd = s.r * g0[h] + s.g * g1[h] + s.bl * g2[h] - accg[h];
                        const float dLda = Tk * dd - bgT[h] * rom;
                        const float wT = a * Tk;
                        gr = fmaf(wT, g0[h], gr);
                        gg = fmaf(wT, g1[h], gg);
                        gb = fmaf(wT, g2[h], gb);
                        if (!clamped) {
                            const float dx = __fsub_rn(s.u, __fadd_rn(fx, (float)h));
                            const float dLdo = G * dLda, qq = a * dLda;
                            dO += dLdo;
                            S = fmaf(dLdo, dLdo, S);
                            const float qx = dx * qq, qy = dy * qq;
                            sx += qx;
                            sy += qy;
                            sxx = fmaf(dx, qx, sxx);
                            sxy = fmaf(dy, qx, sxy);
                            syy = fmaf(dy, qy, syy);
                        }
                        ++n;
                        accg[h] = fmaf(a, dd, accg[h]);
                        T[h] = Tk;
                    }
                }
                if (__any_sync(0xffffffffu, n != 0u)) {
                    // -(A sx + B sy), -(B sx + C sy), -sxx/2, -sxy, -syy/2 with
                    // A = -2a, B = -b, C = -2c; then dL/do, dL/dcolour, S. The
                    // row's M (slot 10) is the same sum as dL/do, C (11) the
                    // integer count of contributing pixels.
                    float v[10];
                    v[0] = 2.0f * s.a * sx + s.b * sy;
                    v[1] = s.b * sx + 2.0f * s.c * sy;
                    v[2] = -0.5f * sxx;
                    v[3] = -sxy;
                    v[4] = -0.5f * syy;
                    v[5] = dO;
                    v[6] = gr;
                    v[7] = gg;
                    v[8] = gb;
                    v[9] = S;
                    const uint32_t cnt = __reduce_add_sync(0xffffffffu, n);
                    float *row = gacc + 16 * (int64_t)s_id[k];
                    if constexpr (int_reduce(PREC)) {
                        const int vi = lane >> 1;
                        float mine = 0.f;
#pragma unroll
                        for (int i = 0; i < 10; ++i) {
                            const float t = warp_sum_int(v[i]);
                            if (vi == i || (i == 5 && vi == 10)) mine = t;  // M = the opacity sum
                        }
                        if ((lane & 1) == 0) {
                            if (vi < 11)
                                atomicAdd(row + vi, mine);
                            else if (vi == 11)
                                atomicAdd(reinterpret_cast<unsigned int *>(row + 11), cnt);
                        }
                    } else {
                        const float red = warp_reduce_scatter10(v, lane);
                        if ((lane & 1) == 0) {
                            const int vi = scatter10_index(lane);
                            if (vi >= 0) {
                                atomicAdd(row + vi, red);
                                if (vi == 5) atomicAdd(row + 10, red);
                            } else if (lane == 12) {
                                atomicAdd(reinterpret_cast<unsigned int *>(row + 11), cnt);
                            }
                        }
                    }
                }
            }
        }
    }
}

template <int PREC>
__global__ void __launch_bounds__(kBatch) k_raster_bwd(
    const float *__restrict__ rec, const uint32_t *__restrict__ vals,
    const uint32_t *__restrict__ ranges, RCam K, const float *__restrict__ finalT,
    const int32_t *__restrict__ last, const float *__restrict__ dLdI, float *__restrict__ gacc) {
    __shared__ SplatS s_sp[kBatch];
    __shared__ uint32_t s_id[kBatch];
    __shared__ uint8_t s_fl[kBatch];
    __shared__ int s_maxlast;
    bwd_tile<PREC>(rec, vals, ranges, K, blockIdx.x, finalT, last, dLdI, gacc, s_sp, s_id, s_fl,
                   s_maxlast);
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
    return K;
}

template <int PREC>
__global__ void __launch_bounds__(kBatch) k_raster_fwd_batch(const lgs_view *__restrict__ views,
                                                           int n_views, uint32_t total_tiles,
                                                           uint32_t *counter) {
    __shared__ SplatS s_sp[kBatch];
    __shared__ uint8_t s_fl[kBatch];
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
                       V.final_T, V.last_contrib, s_sp, s_fl);
        __syncthreads();
    }
}

template <int PREC>
__global__ void __launch_bounds__(kBatch) k_raster_bwd_batch(const lgs_view *__restrict__ views,
                                                           int n_views, uint32_t total_tiles,
                                                           uint32_t *counter) {
    __shared__ SplatS s_sp[kBatch];
    __shared__ uint32_t s_id[kBatch];
    __shared__ uint8_t s_fl[kBatch];
    __shared__ int s_maxlast;
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
                       V.last_contrib, V.dL_dimage, V.grad_acc, s_sp, s_id, s_fl, s_maxlast);
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

RCam make_rcam(const lgs_camera *c, int tw, int th) {
    RCam k;
    k.W = c->width;
    k.H = c->height;
    k.gx = (int)ceil_div(c->width, tw);
    k.ntiles = k.gx * (int)ceil_div(c->height, th);
    k.bg[0] = c->bg[0]; k.bg[1] = c->bg[1]; k.bg[2] = c->bg[2];
    return k;
}

}  // namespace

lgs_status raster_fwd(const lgs_splats *sp, const uint32_t *vals, const uint32_t *ranges,
                      const lgs_camera *cam, int tw, int th, int precision, float *image,
                      float *finalT, int32_t *last, cudaStream_t s) {
    if (tw != kTile || th != kTile) return LGS_ERR_INVALID_ARG;
    const RCam K = make_rcam(cam, tw, th);
    const unsigned grid = (unsigned)K.ntiles;
    count_launch();
    switch (precision) {
        case LGS_FP32:
            k_raster_fwd<LGS_FP32><<<grid, kBatch, 0, s>>>(sp->rec, vals, ranges, K, image, finalT, last);
            break;
        case LGS_MIXED_FP16:
            k_raster_fwd<LGS_MIXED_FP16><<<grid, kBatch, 0, s>>>(sp->rec, vals, ranges, K, image, finalT, last);
            break;
        case LGS_MIXED_BF16:
            k_raster_fwd<LGS_MIXED_BF16><<<grid, kBatch, 0, s>>>(sp->rec, vals, ranges, K, image, finalT, last);
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
    const RCam K = make_rcam(cam, tw, th);
    const unsigned grid = (unsigned)K.ntiles;
    count_launch();
#define LGS_RBW(P) k_raster_bwd<P><<<grid, kBatch, 0, s>>>(sp->rec, vals, ranges, K, finalT, last, dLdI, gacc)
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

lgs_status raster_batch(const lgs_view *views, int n_views, uint32_t total_tiles, int precision,
                        uint32_t *counter, int backward, cudaStream_t s) {
    cudaMemsetAsync(counter, 0, sizeof(uint32_t), s);
    int per_sm = 0;
    if (backward)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_raster_bwd_batch<LGS_FP32>, kBatch, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_raster_fwd_batch<LGS_FP32>, kBatch, 0);
    const int64_t cap = (int64_t)num_sms() * (per_sm > 0 ? per_sm : 1);
    const unsigned grid = (unsigned)(total_tiles < cap ? total_tiles : cap);
    if (grid == 0) return LGS_OK;
    count_launch();
#define LGS_RB(P) do { if (backward) k_raster_bwd_batch<P><<<grid, kBatch, 0, s>>>(views, n_views, total_tiles, counter); \
                       else k_raster_fwd_batch<blend_of(P)><<<grid, kBatch, 0, s>>>(views, n_views, total_tiles, counter); } while (0)
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
