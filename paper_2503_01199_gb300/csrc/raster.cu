// Tile rasteriser, forward (Eq. 1-2, Alg. 1) and backward (Eq. 3, App. A.1
// Eq. 4-6) with the opacity-gradient moments of Sec. 3.3.
//
// One CTA per 16 x 16 tile, one pixel per thread. The tile's sorted splats
// are staged through shared memory in batches of 256 (one per thread). In
// the backward each warp reduces the per-pixel terms of a splat across its
// 32 pixels with a reduce-scatter butterfly (16 shuffles for 11 values,
// ending with value i on lanes 2i, 2i+1), and lanes 0, 2, .., 20 issue one
// atomic each: 11 adjacent floats of the splat's 64-byte gradient row.
#include <cuda_runtime.h>

#include "lgs_internal.cuh"

namespace lgs {

namespace {

constexpr int kTileW = 16, kTileH = 16;
constexpr int kBlock = kTileW * kTileH;
constexpr float kAlphaMin = 1.0f / 255.0f;
constexpr float kAlphaMax = 0.99f;
constexpr float kTMin = 1e-4f;

struct SplatS {
    float u, v, A, B, C, o, r, g, b;
};

struct RCam {
    int W, H, gx;
    float bg[3];
};

__device__ __forceinline__ void load_splat(const float *__restrict__ rec, uint32_t j, SplatS &s) {
    const float4 *p = reinterpret_cast<const float4 *>(rec + 12 * (int64_t)j);
    const float4 a = p[0], b = p[1];
    const float c = rec[12 * (int64_t)j + 8];
    s.u = a.x; s.v = a.y; s.A = a.z; s.B = a.w;
    s.C = b.x; s.o = b.y; s.r = b.z; s.g = b.w; s.b = c;
}

__global__ void __launch_bounds__(kBlock) k_raster_fwd(const float *__restrict__ rec,
                                                      const uint32_t *__restrict__ vals,
                                                      const uint32_t *__restrict__ ranges, RCam K,
                                                      float *__restrict__ image,
                                                      float *__restrict__ finalT,
                                                      int32_t *__restrict__ last) {
    __shared__ SplatS s_sp[kBlock];
    const int tile = blockIdx.x;
    const int tx = tile % K.gx, ty = tile / K.gx;
    const int px = tx * kTileW + (threadIdx.x % kTileW), py = ty * kTileH + (threadIdx.x / kTileW);
    const bool inside = px < K.W && py < K.H;
    const float pxc = px + 0.5f, pyc = py + 0.5f;
    const uint32_t r0 = ranges[2 * tile], r1 = ranges[2 * tile + 1];
    float T = 1.0f, cr = 0.f, cg = 0.f, cb = 0.f;
    int32_t lst = 0;
    bool done = !inside;
    for (uint32_t b0 = r0; b0 < r1; b0 += kBlock) {
        if (__syncthreads_count(done) == kBlock) break;
        const uint32_t idx = b0 + threadIdx.x;
        if (idx < r1) load_splat(rec, vals[idx], s_sp[threadIdx.x]);
        __syncthreads();
        const int cnt = min((uint32_t)kBlock, r1 - b0);
        for (int k = 0; k < cnt && !done; ++k) {
            const SplatS &s = s_sp[k];
            const float dx = s.u - pxc, dy = s.v - pyc;
            const float power = -0.5f * (s.A * dx * dx + s.C * dy * dy) - s.B * dx * dy;
            const float alpha = fminf(kAlphaMax, s.o * __expf(power));
            if (alpha < kAlphaMin) continue;
            const float Tn = T * (1.0f - alpha);
            if (Tn < kTMin) {
                done = true;
                break;
            }
            const float w = alpha * T;
            cr += s.r * w;
            cg += s.g * w;
            cb += s.b * w;
            T = Tn;
            lst = (int32_t)(b0 - r0) + k + 1;
        }
    }
    if (inside) {
        const int64_t p = (int64_t)py * K.W + px, hw = (int64_t)K.W * K.H;
        image[p] = cr + T * K.bg[0];
        image[hw + p] = cg + T * K.bg[1];
        image[2 * hw + p] = cb + T * K.bg[2];
        finalT[p] = T;
        last[p] = lst;
    }
}

// Reduce-scatter of 16 values across the warp: on return v[0] of lanes 2i
// and 2i + 1 holds the warp sum of input value i.
__device__ __forceinline__ float warp_reduce_scatter16(float v[16], int lane) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const bool up = lane & 16;
        const float send = up ? v[i] : v[i + 8];
        const float keep = up ? v[i + 8] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const bool up = lane & 8;
        const float send = up ? v[i] : v[i + 4];
        const float keep = up ? v[i + 4] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
    }
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const bool up = lane & 4;
        const float send = up ? v[i] : v[i + 2];
        const float keep = up ? v[i + 2] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
    }
    {
        const bool up = lane & 2;
        const float send = up ? v[0] : v[1];
        const float keep = up ? v[1] : v[0];
        v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 1);
}

__global__ void __launch_bounds__(kBlock) k_raster_bwd(
    const float *__restrict__ rec, const uint32_t *__restrict__ vals,
    const uint32_t *__restrict__ ranges, RCam K, const float *__restrict__ finalT,
    const int32_t *__restrict__ last, const float *__restrict__ dLdI, float *__restrict__ gacc) {
    __shared__ SplatS s_sp[kBlock];
    __shared__ uint32_t s_id[kBlock];
    __shared__ int s_maxlast;
    const int tile = blockIdx.x;
    const int tx = tile % K.gx, ty = tile / K.gx;
    const int lane = threadIdx.x & 31;
    const int px = tx * kTileW + (threadIdx.x % kTileW), py = ty * kTileH + (threadIdx.x / kTileW);
    const bool inside = px < K.W && py < K.H;
    const float pxc = px + 0.5f, pyc = py + 0.5f;
    const uint32_t r0 = ranges[2 * tile];
    const int64_t p = (int64_t)py * K.W + px, hw = (int64_t)K.W * K.H;
    float T = 1.0f, gI[3] = {0.f, 0.f, 0.f};
    int lst = 0;
    if (inside) {
        T = finalT[p];
        lst = last[p];
        gI[0] = dLdI[p];
        gI[1] = dLdI[hw + p];
        gI[2] = dLdI[2 * hw + p];
    }
    const float Tf = T;
    const float bgdot = K.bg[0] * gI[0] + K.bg[1] * gI[1] + K.bg[2] * gI[2];
    if (threadIdx.x == 0) s_maxlast = 0;
    __syncthreads();
    atomicMax(&s_maxlast, lst);
    __syncthreads();
    const int maxlast = s_maxlast;
    float acc[3] = {0.f, 0.f, 0.f}, pa = 0.f, prgb[3] = {0.f, 0.f, 0.f};
    // positions maxlast-1 .. 0 of the tile list, in batches from the back
    for (int end = maxlast; end > 0; end -= kBlock) {
        const int cnt = min(kBlock, end);
        __syncthreads();
        if (threadIdx.x < cnt) {
            const uint32_t j = vals[r0 + end - 1 - threadIdx.x];
            s_id[threadIdx.x] = j;
            load_splat(rec, j, s_sp[threadIdx.x]);
        }
        __syncthreads();
        for (int k = 0; k < cnt; ++k) {
            const int pos = end - 1 - k;
            const SplatS &s = s_sp[k];
            float v[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = 0.f;
            uint32_t contrib = 0;
            if (pos < lst) {
                const float dx = s.u - pxc, dy = s.v - pyc;
                const float power = -0.5f * (s.A * dx * dx + s.C * dy * dy) - s.B * dx * dy;
                const float G = __expf(power);
                const float oG = s.o * G;
                const float alpha = fminf(kAlphaMax, oG);
                if (alpha >= kAlphaMin) {
                    contrib = 1;
                    const float om = 1.0f - alpha;
                    const float Tk = T / om;
                    // colour behind this splat, normalised by the transmittance after it
                    acc[0] = pa * prgb[0] + (1.f - pa) * acc[0];
                    acc[1] = pa * prgb[1] + (1.f - pa) * acc[1];
                    acc[2] = pa * prgb[2] + (1.f - pa) * acc[2];
                    const float dLda = Tk * ((s.r - acc[0]) * gI[0] + (s.g - acc[1]) * gI[1] +
                                             (s.b - acc[2]) * gI[2]) -
                                       Tf * bgdot / om;
                    const float wT = alpha * Tk;
                    v[6] = wT * gI[0];
                    v[7] = wT * gI[1];
                    v[8] = wT * gI[2];
                    if (oG < kAlphaMax) {
                        const float dLdo = G * dLda;
                        const float dLdp = alpha * dLda;
                        v[0] = -(s.A * dx + s.B * dy) * dLdp;
                        v[1] = -(s.B * dx + s.C * dy) * dLdp;
                        v[2] = -0.5f * dx * dx * dLdp;
                        v[3] = -dx * dy * dLdp;
                        v[4] = -0.5f * dy * dy * dLdp;
                        v[5] = dLdo;
                        v[9] = dLdo * dLdo;
                        v[10] = dLdo;
                    }
                    T = Tk;
                    pa = alpha;
                    prgb[0] = s.r; prgb[1] = s.g; prgb[2] = s.b;
                }
            }
            if (__any_sync(0xffffffffu, contrib)) {
                const float red = warp_reduce_scatter16(v, lane);
                const uint32_t c = __reduce_add_sync(0xffffffffu, contrib);
                float *row = gacc + 16 * (int64_t)s_id[k];
                const int vi = lane >> 1;
                if ((lane & 1) == 0 && vi < 11) atomicAdd(row + vi, red);
                if (lane == 1) atomicAdd(reinterpret_cast<unsigned int *>(row + 11), c);
            }
        }
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
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, s * inv);
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

RCam make_rcam(const lgs_camera *c, int tw) {
    RCam k;
    k.W = c->width;
    k.H = c->height;
    k.gx = (int)ceil_div(c->width, tw);
    k.bg[0] = c->bg[0]; k.bg[1] = c->bg[1]; k.bg[2] = c->bg[2];
    return k;
}

}  // namespace

lgs_status raster_fwd(const lgs_splats *sp, const uint32_t *vals, const uint32_t *ranges,
                      const lgs_camera *cam, int tw, int th, float *image, float *finalT,
                      int32_t *last, cudaStream_t s) {
    if (tw != kTileW || th != kTileH) return LGS_ERR_INVALID_ARG;
    const RCam K = make_rcam(cam, tw);
    const int ntiles = K.gx * (int)ceil_div(cam->height, th);
    count_launch();
    k_raster_fwd<<<ntiles, kBlock, 0, s>>>(sp->rec, vals, ranges, K, image, finalT, last);
    return check_launch();
}

lgs_status raster_bwd(const lgs_splats *sp, const uint32_t *vals, const uint32_t *ranges,
                      const lgs_camera *cam, int tw, int th, const float *finalT,
                      const int32_t *last, const float *dLdI, float *gacc, int64_t max_splats,
                      int accumulate, cudaStream_t s) {
    if (tw != kTileW || th != kTileH) return LGS_ERR_INVALID_ARG;
    if (!accumulate) cudaMemsetAsync(gacc, 0, (size_t)max_splats * 16 * sizeof(float), s);
    const RCam K = make_rcam(cam, tw);
    const int ntiles = K.gx * (int)ceil_div(cam->height, th);
    count_launch();
    k_raster_bwd<<<ntiles, kBlock, 0, s>>>(sp->rec, vals, ranges, K, finalT, last, dLdI, gacc);
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
