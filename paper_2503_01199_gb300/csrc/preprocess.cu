// Preprocess (3D Gaussian -> projected splat, Sec. 3) and its backward, plus
// the fused backward + Adam step on visible rows (Sec. 3.2.3).
//
// One thread per compacted Gaussian j; row = map[j]. Parameter planes are
// read with unit stride across the warp: a visible cluster is a run of
// consecutive rows, so reads through the map stay coalesced.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lgs_internal.cuh"

namespace lgs {

namespace {

constexpr int kThreads = 128;
constexpr float kLowPass = 0.3f;
constexpr float kClampFov = 1.3f;

// ---------------------------------------------------------------------------
// real spherical harmonics up to degree 3 as Cartesian polynomials on the
// unit sphere: Y_l^{+-m} = sqrt2 K_l^m (-1)^m P_l^(m)(z) {Re, Im}(x + i y)^m,
// K_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!), P_l^(m) the m-th derivative of
// the Legendre polynomial. Constants are evaluated at compile time.
// ---------------------------------------------------------------------------
constexpr double c_sqrt(double x) {
    double r = x > 1.0 ? x : 1.0;
    for (int i = 0; i < 64; ++i) r = 0.5 * (r + x / r);
    return r;
}
constexpr double c_fact(int k) { return k <= 1 ? 1.0 : k * c_fact(k - 1); }
constexpr double c_pi = 3.14159265358979323846;
constexpr double shK(int l, int m) {
    return c_sqrt((2.0 * l + 1.0) / (4.0 * c_pi) * c_fact(l - m) / c_fact(l + m));
}
constexpr double c_sqrt2 = c_sqrt(2.0);

constexpr float Y0 = (float)shK(0, 0);
constexpr float Y1 = (float)shK(1, 0);                   // = sqrt2 K_1^1
constexpr float Y20 = (float)shK(2, 0);                  // (3z^2 - 1)/2
constexpr float Y21 = (float)(-3.0 * c_sqrt2 * shK(2, 1));  // z {x, y}
constexpr float Y22 = (float)(3.0 * c_sqrt2 * shK(2, 2));   // {x^2 - y^2, 2xy}
constexpr float Y30 = (float)shK(3, 0);                  // (5z^3 - 3z)/2
constexpr float Y31 = (float)(-0.5 * c_sqrt2 * shK(3, 1));  // (15z^2 - 3) {x, y}
constexpr float Y32 = (float)(15.0 * c_sqrt2 * shK(3, 2));  // z {x^2 - y^2, 2xy}
constexpr float Y33 = (float)(-15.0 * c_sqrt2 * shK(3, 3)); // {x^3 - 3xy^2, 3x^2 y - y^3}

__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float *Y) {
    Y[0] = Y0;
    if (deg < 1) return;
    Y[1] = -Y1 * y;
    Y[2] = Y1 * z;
    Y[3] = -Y1 * x;
    if (deg < 2) return;
    const float xx = x * x, yy = y * y, zz = z * z, xy = x * y;
    Y[4] = Y22 * 2.0f * xy;
    Y[5] = Y21 * z * y;
    Y[6] = Y20 * 0.5f * (3.0f * zz - 1.0f);
    Y[7] = Y21 * z * x;
    Y[8] = Y22 * (xx - yy);
    if (deg < 3) return;
    Y[9] = Y33 * (3.0f * xx * y - yy * y);
    Y[10] = Y32 * z * 2.0f * xy;
    Y[11] = Y31 * (15.0f * zz - 3.0f) * y;
    Y[12] = Y30 * 0.5f * (5.0f * zz * z - 3.0f * z);
    Y[13] = Y31 * (15.0f * zz - 3.0f) * x;
    Y[14] = Y32 * z * (xx - yy);
    Y[15] = Y33 * (xx * x - 3.0f * x * yy);
}

// g += sum_k w_k grad Y_k  (gradient of the polynomial extension)
__device__ __forceinline__ void sh_basis_grad(int deg, float x, float y, float z, const float *w,
                                              float &gx, float &gy, float &gz) {
    if (deg < 1) return;
    gy += -Y1 * w[1];
    gz += Y1 * w[2];
    gx += -Y1 * w[3];
    if (deg < 2) return;
    gx += Y22 * 2.0f * y * w[4];
    gy += Y22 * 2.0f * x * w[4];
    gy += Y21 * z * w[5];
    gz += Y21 * y * w[5];
    gz += Y20 * 3.0f * z * w[6];
    gx += Y21 * z * w[7];
    gz += Y21 * x * w[7];
    gx += Y22 * 2.0f * x * w[8];
    gy += -Y22 * 2.0f * y * w[8];
    if (deg < 3) return;
    const float xx = x * x, yy = y * y, zz = z * z;
    gx += Y33 * 6.0f * x * y * w[9];
    gy += Y33 * (3.0f * xx - 3.0f * yy) * w[9];
    gx += Y32 * 2.0f * y * z * w[10];
    gy += Y32 * 2.0f * x * z * w[10];
    gz += Y32 * 2.0f * x * y * w[10];
    gy += Y31 * (15.0f * zz - 3.0f) * w[11];
    gz += Y31 * 30.0f * y * z * w[11];
    gz += Y30 * 0.5f * (15.0f * zz - 3.0f) * w[12];
    gx += Y31 * (15.0f * zz - 3.0f) * w[13];
    gz += Y31 * 30.0f * x * z * w[13];
    gx += Y32 * 2.0f * x * z * w[14];
    gy += -Y32 * 2.0f * y * z * w[14];
    gz += Y32 * (xx - yy) * w[14];
    gx += Y33 * (3.0f * xx - 3.0f * yy) * w[15];
    gy += -Y33 * 6.0f * x * y * w[15];
}

// The terms of sh_basis_grad for coefficient k alone (same expressions, so
// summing k = 1.. in order adds the same terms in the same order).
__device__ __forceinline__ void sh_grad_single(int k, float x, float y, float z, float w,
                                               float &gx, float &gy, float &gz) {
    switch (k) {
        case 0: break;
        case 1: gy += -Y1 * w; break;
        case 2: gz += Y1 * w; break;
        case 3: gx += -Y1 * w; break;
        case 4: gx += Y22 * 2.0f * y * w; gy += Y22 * 2.0f * x * w; break;
        case 5: gy += Y21 * z * w; gz += Y21 * y * w; break;
        case 6: gz += Y20 * 3.0f * z * w; break;
        case 7: gx += Y21 * z * w; gz += Y21 * x * w; break;
        case 8: gx += Y22 * 2.0f * x * w; gy += -Y22 * 2.0f * y * w; break;
        case 9: {
            const float xx = x * x, yy = y * y;
            gx += Y33 * 6.0f * x * y * w;
            gy += Y33 * (3.0f * xx - 3.0f * yy) * w;
            break;
        }
        case 10:
            gx += Y32 * 2.0f * y * z * w;
            gy += Y32 * 2.0f * x * z * w;
            gz += Y32 * 2.0f * x * y * w;
            break;
        case 11: {
            const float zz = z * z;
            gy += Y31 * (15.0f * zz - 3.0f) * w;
            gz += Y31 * 30.0f * y * z * w;
            break;
        }
        case 12: {
            const float zz = z * z;
            gz += Y30 * 0.5f * (15.0f * zz - 3.0f) * w;
            break;
        }
        case 13: {
            const float zz = z * z;
            gx += Y31 * (15.0f * zz - 3.0f) * w;
            gz += Y31 * 30.0f * x * z * w;
            break;
        }
        case 14: {
            const float xx = x * x, yy = y * y;
            gx += Y32 * 2.0f * x * z * w;
            gy += -Y32 * 2.0f * y * z * w;
            gz += Y32 * (xx - yy) * w;
            break;
        }
        default: {
            const float xx = x * x, yy = y * y;
            gx += Y33 * (3.0f * xx - 3.0f * yy) * w;
            gy += -Y33 * 6.0f * x * y * w;
            break;
        }
    }
}

// Everything the forward computes for one Gaussian, kept for the backward.
struct Fwd {
    bool culled;
    float px, py, pz;        // camera-space centre
    float s[3];              // scales
    float qn[4], qinv;       // unit quaternion, 1/|q|
    float Rq[9];             // rotation of q
    float Sg[6];             // 3D covariance xx xy xz yy yz zz
    float tx, ty;            // clamped centre used by J
    int clx, cly;
    float Tm[6];             // J R_cam (2 x 3)
    float a, b, c;           // projected covariance incl. low-pass
    float det, A, B, C;      // inverse (conic)
    float u, v;
    int radius;
    float dir[3], dinv;      // view direction and 1/|p - centre|
    float logit;
};

struct Cam {
    float R[9], t[3], fx, fy, cx, cy, znear, cc[3], limx, limy;
    int W, H, tw, th, gx, gy;
    const float *pose;  // optional device pose (R row-major, t) read at run time
};

// Replaces R, t and the camera centre by the device-resident pose, if any.
__device__ __forceinline__ void resolve_pose(Cam &K) {
    if (!K.pose) return;
#pragma unroll
    for (int i = 0; i < 9; ++i) K.R[i] = __ldg(K.pose + i);
#pragma unroll
    for (int i = 0; i < 3; ++i) K.t[i] = __ldg(K.pose + 9 + i);
#pragma unroll
    for (int i = 0; i < 3; ++i)
        K.cc[i] = -(K.R[i] * K.t[0] + K.R[3 + i] * K.t[1] + K.R[6 + i] * K.t[2]);
}

Cam make_cam(const lgs_camera *c, int tw, int th) {
    Cam k;
    for (int i = 0; i < 9; ++i) k.R[i] = c->R[i];
    for (int i = 0; i < 3; ++i) k.t[i] = c->t[i];
    k.fx = c->fx; k.fy = c->fy; k.cx = c->cx; k.cy = c->cy; k.znear = c->znear;
    for (int i = 0; i < 3; ++i)
        k.cc[i] = -(c->R[i] * c->t[0] + c->R[3 + i] * c->t[1] + c->R[6 + i] * c->t[2]);
    k.limx = kClampFov * c->width / (2.0f * c->fx);
    k.limy = kClampFov * c->height / (2.0f * c->fy);
    k.W = c->width; k.H = c->height; k.tw = tw; k.th = th;
    k.gx = (int)ceil_div(c->width, tw);
    k.gy = (int)ceil_div(c->height, th);
    k.pose = c->d_pose;
    return k;
}

// View direction from the camera centre to the Gaussian centre and the
// inverse distance, with explicitly rounded operations so that the forward
// and the backward derive the same bits (the colour clamp depends on it). A
// centre at the camera centre gets dir 0.
__device__ __forceinline__ void view_dir(const Cam &K, float mx, float my, float mz, float *dir,
                                         float &dinv) {
    const float dx = __fsub_rn(mx, K.cc[0]), dy = __fsub_rn(my, K.cc[1]),
                dz = __fsub_rn(mz, K.cc[2]);
    const float d2 = __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
    dinv = d2 > 0.0f ? __frcp_rn(__fsqrt_rn(d2)) : 0.0f;
    dir[0] = __fmul_rn(dx, dinv);
    dir[1] = __fmul_rn(dy, dinv);
    dir[2] = __fmul_rn(dz, dinv);
}

// Geometry of one Gaussian (planes 0..10): camera-space centre, 3D and 2D
// covariance, conic, screen centre, radius and tile-rectangle cull, view
// direction. Returns false when the Gaussian is culled.
__device__ __forceinline__ bool geom_forward(const Cam &K, const float *__restrict__ P,
                                             int64_t stride, int64_t row, Fwd &f) {
    const float mx = P[0 * stride + row], my = P[1 * stride + row], mz = P[2 * stride + row];
    f.px = K.R[0] * mx + K.R[1] * my + K.R[2] * mz + K.t[0];
    f.py = K.R[3] * mx + K.R[4] * my + K.R[5] * mz + K.t[1];
    f.pz = K.R[6] * mx + K.R[7] * my + K.R[8] * mz + K.t[2];
    f.culled = !(f.pz > K.znear);
    if (f.culled) return false;
#pragma unroll
    for (int k = 0; k < 3; ++k) f.s[k] = expf(P[(3 + k) * stride + row]);
    float q0 = P[6 * stride + row], q1 = P[7 * stride + row], q2 = P[8 * stride + row],
          q3 = P[9 * stride + row];
    f.logit = P[10 * stride + row];
    const float qlen = sqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
    f.qinv = 1.0f / qlen;
    q0 *= f.qinv; q1 *= f.qinv; q2 *= f.qinv; q3 *= f.qinv;
    f.qn[0] = q0; f.qn[1] = q1; f.qn[2] = q2; f.qn[3] = q3;
    float *R = f.Rq;
    R[0] = 1.f - 2.f * (q2 * q2 + q3 * q3); R[1] = 2.f * (q1 * q2 - q0 * q3); R[2] = 2.f * (q1 * q3 + q0 * q2);
    R[3] = 2.f * (q1 * q2 + q0 * q3); R[4] = 1.f - 2.f * (q1 * q1 + q3 * q3); R[5] = 2.f * (q2 * q3 - q0 * q1);
    R[6] = 2.f * (q1 * q3 - q0 * q2); R[7] = 2.f * (q2 * q3 + q0 * q1); R[8] = 1.f - 2.f * (q1 * q1 + q2 * q2);
    // Sigma = sum_k s_k^2 r_k r_k^T with r_k the columns of Rq
    const float s0 = f.s[0] * f.s[0], s1 = f.s[1] * f.s[1], s2 = f.s[2] * f.s[2];
    f.Sg[0] = R[0] * R[0] * s0 + R[1] * R[1] * s1 + R[2] * R[2] * s2;
    f.Sg[1] = R[0] * R[3] * s0 + R[1] * R[4] * s1 + R[2] * R[5] * s2;
    f.Sg[2] = R[0] * R[6] * s0 + R[1] * R[7] * s1 + R[2] * R[8] * s2;
    f.Sg[3] = R[3] * R[3] * s0 + R[4] * R[4] * s1 + R[5] * R[5] * s2;
    f.Sg[4] = R[3] * R[6] * s0 + R[4] * R[7] * s1 + R[5] * R[8] * s2;
    f.Sg[5] = R[6] * R[6] * s0 + R[7] * R[7] * s1 + R[8] * R[8] * s2;
    // EWA Jacobian at the clamped centre
    const float z = f.pz, iz = 1.0f / z;
    const float xz = f.px * iz, yz = f.py * iz;
    f.clx = xz < -K.limx ? -1 : (xz > K.limx ? 1 : 0);
    f.cly = yz < -K.limy ? -1 : (yz > K.limy ? 1 : 0);
    f.tx = f.clx ? f.clx * K.limx * z : f.px;
    f.ty = f.cly ? f.cly * K.limy * z : f.py;
    const float j00 = K.fx * iz, j02 = -K.fx * f.tx * iz * iz;
    const float j11 = K.fy * iz, j12 = -K.fy * f.ty * iz * iz;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        f.Tm[k] = j00 * K.R[k] + j02 * K.R[6 + k];
        f.Tm[3 + k] = j11 * K.R[3 + k] + j12 * K.R[6 + k];
    }
    // S2 = Tm Sigma Tm^T
    const float *S = f.Sg;
    float w0[3], w1[3];  // Sigma Tm^T columns
    w0[0] = S[0] * f.Tm[0] + S[1] * f.Tm[1] + S[2] * f.Tm[2];
    w0[1] = S[1] * f.Tm[0] + S[3] * f.Tm[1] + S[4] * f.Tm[2];
    w0[2] = S[2] * f.Tm[0] + S[4] * f.Tm[1] + S[5] * f.Tm[2];
    w1[0] = S[0] * f.Tm[3] + S[1] * f.Tm[4] + S[2] * f.Tm[5];
    w1[1] = S[1] * f.Tm[3] + S[3] * f.Tm[4] + S[4] * f.Tm[5];
    w1[2] = S[2] * f.Tm[3] + S[4] * f.Tm[4] + S[5] * f.Tm[5];
    f.a = f.Tm[0] * w0[0] + f.Tm[1] * w0[1] + f.Tm[2] * w0[2] + kLowPass;
    f.b = f.Tm[3] * w0[0] + f.Tm[4] * w0[1] + f.Tm[5] * w0[2];
    f.c = f.Tm[3] * w1[0] + f.Tm[4] * w1[1] + f.Tm[5] * w1[2] + kLowPass;
    f.det = f.a * f.c - f.b * f.b;
    if (!(f.det > 0.0f)) { f.culled = true; return false; }
    const float idet = 1.0f / f.det;
    f.A = f.c * idet;
    f.B = -f.b * idet;
    f.C = f.a * idet;
    f.u = K.fx * f.px * iz + K.cx;
    f.v = K.fy * f.py * iz + K.cy;
    const float mid = 0.5f * (f.a + f.c);
    const float lam = mid + sqrtf(fmaxf(0.1f, mid * mid - f.det));
    f.radius = (int)ceilf(3.0f * sqrtf(lam));
    const int4 rc = tile_rect(f.u, f.v, (float)f.radius, K.tw, K.th, K.gx, K.gy);
    if (rc.z <= rc.x || rc.w <= rc.y) { f.culled = true; return false; }
    view_dir(K, mx, my, mz, f.dir, f.dinv);
    return true;
}

// raw colour (before the clamp at 0): 0.5 + sum_k c_k Y_k
template <int DEG>
__device__ __forceinline__ void color_forward(const float *__restrict__ P, int64_t stride,
                                              int64_t row, const float *Y, float *raw) {
    constexpr int KK = (DEG + 1) * (DEG + 1);
    raw[0] = raw[1] = raw[2] = 0.5f;
#pragma unroll
    for (int k = 0; k < KK; ++k)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch)
            raw[ch] = __fmaf_rn(P[(11 + 3 * k + ch) * stride + row], Y[k], raw[ch]);
}

// the same sum with the coefficients stored as 16-bit planes
template <int DEG, int SHT>
__device__ __forceinline__ void color_forward16(const uint16_t *__restrict__ sh, int64_t stride,
                                                int64_t row, const float *Y, float *raw) {
    constexpr int KK = (DEG + 1) * (DEG + 1);
    raw[0] = raw[1] = raw[2] = 0.5f;
#pragma unroll
    for (int k = 0; k < KK; ++k)
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            const uint16_t b = __ldg(sh + (3 * k + ch) * stride + row);
            const float c = SHT == LGS_SH_BF16 ? __uint_as_float((uint32_t)b << 16)
                                               : __half2float(__ushort_as_half(b));
            raw[ch] = __fmaf_rn(c, Y[k], raw[ch]);
        }
}

template <int DEG, int SHT>
__global__ void __launch_bounds__(kThreads) k_preprocess(const float *__restrict__ P,
                                                        const uint16_t *__restrict__ sh16,
                                                        int64_t stride,
                                                        int64_t n, const uint32_t *__restrict__ map,
                                                        const int32_t *d_V, Cam K,
                                                        float *__restrict__ rec,
                                                        float *__restrict__ depth,
                                                        int32_t *__restrict__ radius) {
    resolve_pose(K);
    const int64_t V = load_count(d_V, n);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < V;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = map ? map[j] : j;
        Fwd f;
        float4 *r4 = reinterpret_cast<float4 *>(rec + 12 * j);
        if (!LGS_DCHECK(row < n, kSitePreMap) || !geom_forward(K, P, stride, row, f)) {
            r4[0] = make_float4(0.f, 0.f, 0.f, 0.f);
            r4[1] = make_float4(0.f, 0.f, 0.f, 0.f);
            r4[2] = make_float4(0.f, 0.f, 0.f, 0.f);
            depth[j] = 0.0f;
            radius[j] = 0;
            continue;
        }
        float Y[16], raw[3];
        sh_basis(DEG, f.dir[0], f.dir[1], f.dir[2], Y);
        if (SHT == LGS_SH_F32)
            color_forward<DEG>(P, stride, row, Y, raw);
        else
            color_forward16<DEG, SHT>(sh16, stride, row, Y, raw);
        const float o = 1.0f / (1.0f + expf(-f.logit));
        // tau: the largest q = d^T conic d at which alpha = o exp(-q/2) can
        // still reach 1/255, widened by 1e-3 (1 + |tau|), far above the
        // rounding of the kernels' alpha and of the tile test
        const float t = 2.0f * logf(255.0f * o);
        const float tau = t > -1e30f ? t + 1e-3f * (1.0f + fabsf(t)) : -INFINITY;
        r4[0] = make_float4(f.u, f.v, f.A, f.B);
        r4[1] = make_float4(f.C, o, fmaxf(raw[0], 0.f), fmaxf(raw[1], 0.f));
        r4[2] = make_float4(fmaxf(raw[2], 0.f), tau, 0.f, 0.f);
        depth[j] = f.pz;
        radius[j] = f.radius;
    }
}

// ---------------------------------------------------------------------------
// backward: the gradient of every parameter plane of one Gaussian, handed to
// `sink(k, g)` as soon as it is known (planes in the order of lgs.h). The
// colour part streams over the SH planes; nothing is kept in local arrays.
// ---------------------------------------------------------------------------
// Geometric part of the backward: gradients of planes 3..10 to sink(k, g)
// and the geometric part of the centre's gradient (through u, v and the
// projection) to gm; the colour's dependence on the centre through the view
// direction is added by the caller.
template <typename Sink>
__device__ __forceinline__ void geom_backward(const Cam &K, const Fwd &f,
                                              const float *__restrict__ g16, Sink &sink,
                                              float *gm) {
    const float4 ga = reinterpret_cast<const float4 *>(g16)[0];
    const float2 gb2 = reinterpret_cast<const float2 *>(g16)[2];
    const float gu = ga.x, gv = ga.y, gA = ga.z, gB = ga.w, gC = gb2.x, go = gb2.y;
    // ---- opacity: o = sigmoid(logit)
    {
        const float o = 1.0f / (1.0f + expf(-f.logit));
        sink(10, go * o * (1.f - o));
    }
    // ---- conic -> projected covariance: dS2 = -Q dQ Q, B used twice
    const float hB = 0.5f * gB;
    const float t00 = f.A * gA + f.B * hB, t01 = f.A * hB + f.B * gC;
    const float t10 = f.B * gA + f.C * hB, t11 = f.B * hB + f.C * gC;
    const float s00 = -(t00 * f.A + t01 * f.B);
    const float s01 = -(t00 * f.B + t01 * f.C);
    const float s11 = -(t10 * f.B + t11 * f.C);
    // ---- S2 = Tm Sigma Tm^T:  dSigma = Tm^T dS2 Tm,  dTm = 2 dS2 Tm Sigma
    const float *T = f.Tm;
    float gS[6];  // symmetric: xx xy xz yy yz zz (full-matrix gradient entries)
    {
        float M0[3], M1[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            M0[k] = s00 * T[k] + s01 * T[3 + k];
            M1[k] = s01 * T[k] + s11 * T[3 + k];
        }
        gS[0] = T[0] * M0[0] + T[3] * M1[0];
        gS[1] = T[0] * M0[1] + T[3] * M1[1];
        gS[2] = T[0] * M0[2] + T[3] * M1[2];
        gS[3] = T[1] * M0[1] + T[4] * M1[1];
        gS[4] = T[1] * M0[2] + T[4] * M1[2];
        gS[5] = T[2] * M0[2] + T[5] * M1[2];
    }
    float gT[6];
    {
        const float *S = f.Sg;
        float U0[3], U1[3];  // Tm Sigma
        U0[0] = T[0] * S[0] + T[1] * S[1] + T[2] * S[2];
        U0[1] = T[0] * S[1] + T[1] * S[3] + T[2] * S[4];
        U0[2] = T[0] * S[2] + T[1] * S[4] + T[2] * S[5];
        U1[0] = T[3] * S[0] + T[4] * S[1] + T[5] * S[2];
        U1[1] = T[3] * S[1] + T[4] * S[3] + T[5] * S[4];
        U1[2] = T[3] * S[2] + T[4] * S[4] + T[5] * S[5];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            gT[k] = 2.f * (s00 * U0[k] + s01 * U1[k]);
            gT[3 + k] = 2.f * (s01 * U0[k] + s11 * U1[k]);
        }
    }
    // ---- Tm = J R_cam:  dJ = dTm R_cam^T (only J00, J02, J11, J12 are free)
    const float gJ00 = gT[0] * K.R[0] + gT[1] * K.R[1] + gT[2] * K.R[2];
    const float gJ02 = gT[0] * K.R[6] + gT[1] * K.R[7] + gT[2] * K.R[8];
    const float gJ11 = gT[3] * K.R[3] + gT[4] * K.R[4] + gT[5] * K.R[5];
    const float gJ12 = gT[3] * K.R[6] + gT[4] * K.R[7] + gT[5] * K.R[8];
    const float z = f.pz, iz = 1.f / z, iz2 = iz * iz, iz3 = iz2 * iz;
    float gpx = 0.f, gpy = 0.f, gpz = 0.f;
    gpz += -K.fx * iz2 * gJ00 - K.fy * iz2 * gJ11;
    gpz += 2.f * K.fx * f.tx * iz3 * gJ02 + 2.f * K.fy * f.ty * iz3 * gJ12;
    const float gtx = -K.fx * iz2 * gJ02, gty = -K.fy * iz2 * gJ12;
    if (f.clx) gpz += gtx * f.clx * K.limx; else gpx += gtx;
    if (f.cly) gpz += gty * f.cly * K.limy; else gpy += gty;
    // ---- u, v
    gpx += gu * K.fx * iz;
    gpy += gv * K.fy * iz;
    gpz += -(gu * K.fx * f.px + gv * K.fy * f.py) * iz2;
    // ---- camera transform: the geometric part of the centre's gradient
#pragma unroll
    for (int k = 0; k < 3; ++k) gm[k] = K.R[k] * gpx + K.R[3 + k] * gpy + K.R[6 + k] * gpz;
    // ---- Sigma = sum_k s_k^2 r_k r_k^T with G the full symmetric gradient:
    // d/dlog s_k = 2 s_k^2 r_k^T G r_k, d/dr_k = 2 s_k^2 G r_k
    {
        const float G00 = gS[0], G11 = gS[3], G22 = gS[5];
        const float G01 = gS[1], G02 = gS[2], G12 = gS[4];
        float gR[9];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float r0 = f.Rq[k], r1 = f.Rq[3 + k], r2 = f.Rq[6 + k];
            const float Gr0 = G00 * r0 + G01 * r1 + G02 * r2;
            const float Gr1 = G01 * r0 + G11 * r1 + G12 * r2;
            const float Gr2 = G02 * r0 + G12 * r1 + G22 * r2;
            const float s2 = f.s[k] * f.s[k];
            sink(3 + k, 2.f * s2 * (r0 * Gr0 + r1 * Gr1 + r2 * Gr2));
            gR[k] = 2.f * s2 * Gr0;
            gR[3 + k] = 2.f * s2 * Gr1;
            gR[6 + k] = 2.f * s2 * Gr2;
        }
        // Rq(q): derivative of each entry w.r.t. (w, x, y, z) of the unit q
        const float w = f.qn[0], x = f.qn[1], y = f.qn[2], zq = f.qn[3];
        float gq[4];
        gq[0] = 2.f * (-zq * gR[1] + y * gR[2] + zq * gR[3] - x * gR[5] - y * gR[6] + x * gR[7]);
        gq[1] = 2.f * (y * gR[1] + zq * gR[2] + y * gR[3] - 2.f * x * gR[4] - w * gR[5] +
                       zq * gR[6] + w * gR[7] - 2.f * x * gR[8]);
        gq[2] = 2.f * (-2.f * y * gR[0] + x * gR[1] + w * gR[2] + x * gR[3] + zq * gR[5] -
                       w * gR[6] + zq * gR[7] - 2.f * y * gR[8]);
        gq[3] = 2.f * (-2.f * zq * gR[0] - w * gR[1] + x * gR[2] + w * gR[3] - 2.f * zq * gR[4] +
                       y * gR[5] + x * gR[6] + y * gR[7]);
        const float dq = gq[0] * w + gq[1] * x + gq[2] * y + gq[3] * zq;
#pragma unroll
        for (int k = 0; k < 4; ++k) sink(6 + k, (gq[k] - f.qn[k] * dq) * f.qinv);
    }
}

template <int DEG, typename Sink>
__device__ __forceinline__ bool backward(const Cam &K, const float *__restrict__ P, int64_t stride,
                                         int64_t row, const float *__restrict__ g16, Sink &sink,
                                         float *dir_out = nullptr, float *grgb_out = nullptr) {
    constexpr int KK = (DEG + 1) * (DEG + 1);
    Fwd f;
    if (!geom_forward(K, P, stride, row, f)) {
#pragma unroll
        for (int k = 0; k < 11 + 3 * KK; ++k) sink(k, 0.0f);
        if (dir_out) dir_out[0] = dir_out[1] = dir_out[2] = 0.0f;
        if (grgb_out) grgb_out[0] = grgb_out[1] = grgb_out[2] = 0.0f;
        return false;
    }
    float gm[3];
    geom_backward(K, f, g16, sink, gm);
    // ---- colour: clamp test, SH coefficients (streamed) and view direction
    const float4 gb = reinterpret_cast<const float4 *>(g16)[1];
    const float gcb = g16[8];
    float Y[16], raw[3];
    sh_basis(DEG, f.dir[0], f.dir[1], f.dir[2], Y);
    color_forward<DEG>(P, stride, row, Y, raw);
    const float grgb[3] = {raw[0] > 0.f ? gb.z : 0.f, raw[1] > 0.f ? gb.w : 0.f,
                           raw[2] > 0.f ? gcb : 0.f};
    if (dir_out) {
        dir_out[0] = f.dir[0];
        dir_out[1] = f.dir[1];
        dir_out[2] = f.dir[2];
    }
    if (grgb_out) {
        grgb_out[0] = grgb[0];
        grgb_out[1] = grgb[1];
        grgb_out[2] = grgb[2];
    }
    float wk[16];
#pragma unroll
    for (int k = 0; k < KK; ++k) {
        float w = 0.f;
#pragma unroll
        for (int ch = 0; ch < 3; ++ch) {
            w += grgb[ch] * P[(11 + 3 * k + ch) * stride + row];
            sink(11 + 3 * k + ch, grgb[ch] * Y[k]);
        }
        wk[k] = w;
    }
    float gdx = 0.f, gdy = 0.f, gdz = 0.f;
    sh_basis_grad(DEG, f.dir[0], f.dir[1], f.dir[2], wk, gdx, gdy, gdz);
    const float dd = gdx * f.dir[0] + gdy * f.dir[1] + gdz * f.dir[2];
    sink(0, gm[0] + (gdx - f.dir[0] * dd) * f.dinv);
    sink(1, gm[1] + (gdy - f.dir[1] * dd) * f.dinv);
    sink(2, gm[2] + (gdz - f.dir[2] * dd) * f.dinv);
    return true;
}

struct AdamArgs {
    float lr[64];
    float b1, b2, eps, c1, c2;  // c1 = 1 / (1 - b1^t), c2 = 1 / (1 - b2^t)
};

// One Adam step; the quotient uses the fast reciprocal (2 ulp), far inside
// the FP32 tolerance of the update.
__device__ __forceinline__ void adam_update(float &p, float &m, float &v, float g, float lr,
                                            const AdamArgs &a) {
    m = a.b1 * m + (1.f - a.b1) * g;
    v = a.b2 * v + (1.f - a.b2) * g * g;
    p -= lr * __fdividef(m * a.c1, sqrtf(v * a.c2) + a.eps);
}

struct GradSink {
    float *__restrict__ out;
    int64_t stride, row;
    bool add;
    __device__ __forceinline__ void operator()(int k, float g) {
        float &o = out[k * stride + row];
        o = add ? o + g : g;
    }
};

template <int DEG>
__global__ void __launch_bounds__(kThreads) k_preprocess_bwd(const float *__restrict__ P,
                                                            int64_t stride, int64_t n,
                                                            const uint32_t *__restrict__ map,
                                                            const int32_t *d_V, Cam K,
                                                            const float *__restrict__ gacc,
                                                            float *__restrict__ gout,
                                                            int accumulate) {
    const int64_t V = load_count(d_V, n);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < V;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = map ? map[j] : j;
        if (!LGS_DCHECK(row < n, kSitePreMap)) continue;
        GradSink sink{gout, stride, row, accumulate != 0};
        backward<DEG>(K, P, stride, row, gacc + 16 * j, sink);
    }
}

// Fused backward + Adam over the visible Gaussians, in chunks of 256.
// Part A (one thread per Gaussian): the whole backward; Adam on the planes
// 0..10 (centre, scales, rotation, opacity) as their gradients are known.
// The SH planes' gradients are (colour gradient masked by the clamp) x
// Y_k(view direction); part A hands the masked colour gradient and the view
// direction to part B through shared memory.
// Part B (same thread, coefficient by coefficient): Adam on the three planes
// of each SH coefficient; a warp streams 32 consecutive rows of one plane.
struct GeomSink {
    float *__restrict__ P;
    float *__restrict__ M;
    float *__restrict__ V;
    int64_t stride, row;
    const AdamArgs *a;
    __device__ __forceinline__ void operator()(int k, float g) {
        if (k < 11) {
            const int64_t i = k * stride + row;
            float p = P[i], m = M[i], v = V[i];
            adam_update(p, m, v, g, a->lr[k], *a);
            P[i] = p;
            M[i] = m;
            V[i] = v;
        }
    }
};

// Y_k alone (k uniform across the CTA in part B), same expressions as sh_basis.
__device__ __forceinline__ float sh_single(int k, float x, float y, float z) {
    switch (k) {
        case 0: return Y0;
        case 1: return -Y1 * y;
        case 2: return Y1 * z;
        case 3: return -Y1 * x;
        case 4: return Y22 * 2.0f * (x * y);
        case 5: return Y21 * z * y;
        case 6: return Y20 * 0.5f * (3.0f * (z * z) - 1.0f);
        case 7: return Y21 * z * x;
        case 8: return Y22 * ((x * x) - (y * y));
        case 9: return Y33 * (3.0f * (x * x) * y - (y * y) * y);
        case 10: return Y32 * z * 2.0f * (x * y);
        case 11: return Y31 * (15.0f * (z * z) - 3.0f) * y;
        case 12: return Y30 * 0.5f * (5.0f * (z * z) * z - 3.0f * z);
        case 13: return Y31 * (15.0f * (z * z) - 3.0f) * x;
        case 14: return Y32 * z * ((x * x) - (y * y));
        default: return Y33 * ((x * x) * x - 3.0f * x * (y * y));
    }
}

// Asynchronous 4-byte global -> shared copy (cp.async), its commit and wait.
__device__ __forceinline__ void cp_async4(float *smem, const float *gmem) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// The densification metric of Sec. 3.3 (a8) from a gradient row: slots 9,
// 10, 11 hold S, M and the fragment count C; C Var = S - M^2 / C (0 when
// C = 0), the expression lgs_opacity_variance evaluates, so both give the
// same bits. Lets the fused step write the metric from the row it reads.
__device__ __forceinline__ float row_metric(const float *g16) {
    const float S = g16[9], M = g16[10];
    const uint32_t C = reinterpret_cast<const uint32_t *>(g16)[11];
    return C ? S - M * M / (float)C : 0.f;
}

// A CTA runs part A for its chunk, then part B; CTAs in different phases
// overlap part A's arithmetic with part B's memory traffic. Part B keeps
// kStages coefficients' loads in flight through shared memory (cp.async),
// so its memory parallelism does not cost registers; every thread reads
// back only what it copied itself. Bounded to four CTAs per SM (64
// registers).
constexpr int kStages = 4;

template <int DEG>
__global__ void __launch_bounds__(256, 4) k_bwd_adam_fused(
    float *__restrict__ P, float *__restrict__ Mo, float *__restrict__ Vo, int64_t stride,
    int64_t n, const uint32_t *__restrict__ map, const int32_t *d_V, Cam K,
    const float *__restrict__ gacc, AdamArgs a, float *__restrict__ metric) {
    constexpr int KK = (DEG + 1) * (DEG + 1);
    __shared__ float s_g[3][256], s_d[3][256];
    __shared__ int64_t s_row[256];
    __shared__ float s_buf[kStages][9][256];  // p, m, v of the 3 channels
    const int tid = threadIdx.x;
    const int64_t V = load_count(d_V, n);
    for (int64_t c0 = (int64_t)blockIdx.x * 256; c0 < V; c0 += (int64_t)gridDim.x * 256) {
        const int64_t j = c0 + tid;
        if (j < V) {
            const int64_t row = map ? map[j] : j;
            s_row[tid] = -1;  // a row the debug build rejects is not updated
            if (LGS_DCHECK(row < n, kSitePreMap)) {
                if (metric) metric[row] = row_metric(gacc + 16 * j);
                GeomSink sink{P, Mo, Vo, stride, row, &a};
                float dir[3], grgb[3];
                backward<DEG>(K, P, stride, row, gacc + 16 * j, sink, dir, grgb);
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    s_g[c][tid] = grgb[c];
                    s_d[c][tid] = dir[c];
                }
                s_row[tid] = row;
            }
        }
        __syncthreads();
        if (j < V && s_row[tid] >= 0) {
            const int64_t row = s_row[tid];
            const float gr[3] = {s_g[0][tid], s_g[1][tid], s_g[2][tid]};
            const float dx = s_d[0][tid], dy = s_d[1][tid], dz = s_d[2][tid];
            auto issue = [&](int k) {
                if (k < KK) {
                    const int64_t at = (11 + 3 * k) * stride + row;
                    float(*b)[256] = s_buf[k % kStages];
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) {
                        cp_async4(&b[ch][tid], P + at + ch * stride);
                        cp_async4(&b[3 + ch][tid], Mo + at + ch * stride);
                        cp_async4(&b[6 + ch][tid], Vo + at + ch * stride);
                    }
                }
                cp_async_commit();  // empty past the last coefficient
            };
#pragma unroll
            for (int k = 0; k < kStages - 1; ++k) issue(k);
#pragma unroll 1
            for (int k = 0; k < KK; ++k) {
                issue(k + kStages - 1);
                cp_async_wait<kStages - 1>();  // coefficient k has landed
                const float(*b)[256] = s_buf[k % kStages];
                const float yk = sh_single(k, dx, dy, dz);
                const int64_t at = (11 + 3 * k) * stride + row;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    float p = b[ch][tid], m = b[3 + ch][tid], v = b[6 + ch][tid];
                    adam_update(p, m, v, gr[ch] * yk, a.lr[11 + 3 * k + ch], a);
                    P[at + ch * stride] = p;
                    Mo[at + ch * stride] = m;
                    Vo[at + ch * stride] = v;
                }
            }
            cp_async_wait<0>();
        }
        __syncthreads();
    }
}

// The same step when the splat records of the forward are at hand (rec,
// 12 floats per compacted row, colours at 6..8, clamped at 0). Part A takes
// the colour clamp from the stored colours (stored > 0 exactly when the raw
// colour is > 0, both sides computing it the same way), so it reads no SH
// plane: it runs the geometric backward, applies Adam to planes 3..10 and
// hands the masked colour gradient, the view direction, 1 / distance and the
// centre's geometric gradient to part B. Part B streams the SH coefficients
// once: Adam on each, while summing the view direction's gradient
// sum_k (sum_ch grgb_ch c_k,ch) grad Y_k from the coefficients as read; it
// then completes the centre's gradient and applies Adam to planes 0..2.
constexpr int kStagesRec = 3;

// FP32 x rounded to nearest even in the 16-bit colour storage type.
__device__ __forceinline__ uint16_t round16(float x, int sh_dtype) {
    return sh_dtype == LGS_SH_BF16 ? __bfloat16_as_ushort(__float2bfloat16_rn(x))
                                   : __half_as_ushort(__float2half_rn(x));
}

// With sh16 (16-bit colour planes of type sh_dtype, the planes' stride), every
// colour coefficient the Adam step updates is also written there, rounded,
// so that a forward that reads the 16-bit planes sees the updated values.
template <int DEG>
__global__ void __launch_bounds__(256, 4) k_bwd_adam_rec(
    float *__restrict__ P, float *__restrict__ Mo, float *__restrict__ Vo, int64_t stride,
    int64_t n, const uint32_t *__restrict__ map, const int32_t *d_V, Cam K,
    const float *__restrict__ gacc, const float *__restrict__ rec, AdamArgs a,
    uint16_t *__restrict__ sh16, int sh_dtype, float *__restrict__ metric) {
    constexpr int KK = (DEG + 1) * (DEG + 1);
    __shared__ float s_g[3][256], s_d[3][256], s_c[4][256];  // s_c: centre gradient, 1 / dist
    __shared__ int64_t s_row[256];
    __shared__ float s_buf[kStagesRec][9][256];
    __shared__ float s_cen[9][256];
    const int tid = threadIdx.x;
    const int64_t V = load_count(d_V, n);
    for (int64_t c0 = (int64_t)blockIdx.x * 256; c0 < V; c0 += (int64_t)gridDim.x * 256) {
        const int64_t j = c0 + tid;
        if (j < V) {
            const int64_t row = map ? map[j] : j;
            s_row[tid] = -1;  // a row the debug build rejects is not updated
            if (LGS_DCHECK(row < n, kSitePreMap)) {
                if (metric) metric[row] = row_metric(gacc + 16 * j);
                GeomSink sink{P, Mo, Vo, stride, row, &a};
                Fwd f;
                float gm[3] = {0.f, 0.f, 0.f}, grgb[3] = {0.f, 0.f, 0.f}, dir[3] = {0.f, 0.f, 0.f};
                float dinv = 0.f;
                if (geom_forward(K, P, stride, row, f)) {
                    const float *g16 = gacc + 16 * j;
                    geom_backward(K, f, g16, sink, gm);
                    const float4 gb = reinterpret_cast<const float4 *>(g16)[1];
                    const float gcb = g16[8];
                    const float4 cr = reinterpret_cast<const float4 *>(rec + 12 * j)[1];
                    const float cb = rec[12 * j + 8];
                    grgb[0] = cr.z > 0.f ? gb.z : 0.f;
                    grgb[1] = cr.w > 0.f ? gb.w : 0.f;
                    grgb[2] = cb > 0.f ? gcb : 0.f;
                    dir[0] = f.dir[0];
                    dir[1] = f.dir[1];
                    dir[2] = f.dir[2];
                    dinv = f.dinv;
                } else {
#pragma unroll
                    for (int k = 3; k < 11; ++k) sink(k, 0.0f);
                }
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    s_g[c][tid] = grgb[c];
                    s_d[c][tid] = dir[c];
                    s_c[c][tid] = gm[c];
                }
                s_c[3][tid] = dinv;
                s_row[tid] = row;
            }
        }
        __syncthreads();
        if (j < V && s_row[tid] >= 0) {
            const int64_t row = s_row[tid];
            const float gr[3] = {s_g[0][tid], s_g[1][tid], s_g[2][tid]};
            const float dx = s_d[0][tid], dy = s_d[1][tid], dz = s_d[2][tid];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                cp_async4(&s_cen[c][tid], P + c * stride + row);
                cp_async4(&s_cen[3 + c][tid], Mo + c * stride + row);
                cp_async4(&s_cen[6 + c][tid], Vo + c * stride + row);
            }
            cp_async_commit();
            auto issue = [&](int k) {
                if (k < KK) {
                    const int64_t at = (11 + 3 * k) * stride + row;
                    float(*b)[256] = s_buf[k % kStagesRec];
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) {
                        cp_async4(&b[ch][tid], P + at + ch * stride);
                        cp_async4(&b[3 + ch][tid], Mo + at + ch * stride);
                        cp_async4(&b[6 + ch][tid], Vo + at + ch * stride);
                    }
                }
                cp_async_commit();  // empty past the last coefficient
            };
#pragma unroll
            for (int k = 0; k < kStagesRec - 1; ++k) issue(k);
            float gdx = 0.f, gdy = 0.f, gdz = 0.f;
#pragma unroll 1
            for (int k = 0; k < KK; ++k) {
                issue(k + kStagesRec - 1);
                cp_async_wait<kStagesRec - 1>();  // coefficient k has landed
                const float(*b)[256] = s_buf[k % kStagesRec];
                const float yk = sh_single(k, dx, dy, dz);
                const int64_t at = (11 + 3 * k) * stride + row;
                float w = 0.f;
#pragma unroll
                for (int ch = 0; ch < 3; ++ch) {
                    float p = b[ch][tid], m = b[3 + ch][tid], v = b[6 + ch][tid];
                    w += gr[ch] * p;
                    adam_update(p, m, v, gr[ch] * yk, a.lr[11 + 3 * k + ch], a);
                    P[at + ch * stride] = p;
                    Mo[at + ch * stride] = m;
                    Vo[at + ch * stride] = v;
                    if (sh16) sh16[(3 * k + ch) * stride + row] = round16(p, sh_dtype);
                }
                sh_grad_single(k, dx, dy, dz, w, gdx, gdy, gdz);
            }
            cp_async_wait<0>();
            const float dinv = s_c[3][tid];
            const float dd = gdx * dx + gdy * dy + gdz * dz;
            const float gc[3] = {s_c[0][tid] + (gdx - dx * dd) * dinv,
                                 s_c[1][tid] + (gdy - dy * dd) * dinv,
                                 s_c[2][tid] + (gdz - dz * dd) * dinv};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float p = s_cen[c][tid], m = s_cen[3 + c][tid], v = s_cen[6 + c][tid];
                adam_update(p, m, v, gc[c], a.lr[c], a);
                P[c * stride + row] = p;
                Mo[c * stride + row] = m;
                Vo[c * stride + row] = v;
            }
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(256) k_adam(float *__restrict__ P, const float *__restrict__ G,
                                             float *__restrict__ Mo, float *__restrict__ Vo,
                                             int64_t stride, int n_planes,
                                             const uint32_t *__restrict__ map, const int32_t *d_V,
                                             int64_t max_rows, AdamArgs a) {
    const int64_t V = load_count(d_V, max_rows);
    const int64_t total = V * n_planes;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int k = (int)(t / V);
        const int64_t j = t - (int64_t)k * V;
        const int64_t row = map ? map[j] : j;
        if (!LGS_DCHECK(row < max_rows, kSiteAdamMap)) continue;
        const int64_t i = k * stride + row;
        float p = P[i], m = Mo[i], v = Vo[i];
        adam_update(p, m, v, G[i], a.lr[k], a);
        P[i] = p;
        Mo[i] = m;
        Vo[i] = v;
    }
}

AdamArgs make_adam(const float *lr, int np, float b1, float b2, float eps, int step) {
    AdamArgs a;
    for (int k = 0; k < 64; ++k) a.lr[k] = k < np ? lr[k] : 0.f;
    a.b1 = b1; a.b2 = b2; a.eps = eps;
    a.c1 = (float)(1.0 / (1.0 - __builtin_pow((double)b1, step)));
    a.c2 = (float)(1.0 / (1.0 - __builtin_pow((double)b2, step)));
    return a;
}

// dst[k][i] = src[k][i] rounded to the 16-bit type, rows i < n of n_planes.
__global__ void __launch_bounds__(256) k_round_planes(const float *__restrict__ src,
                                                     int64_t src_stride,
                                                     uint16_t *__restrict__ dst,
                                                     int64_t dst_stride, int n_planes, int64_t n,
                                                     int dtype) {
    const int64_t total = (int64_t)n_planes * n;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = t / n, i = t - k * n;
        dst[k * dst_stride + i] = round16(src[k * src_stride + i], dtype);
    }
}

}  // namespace

DEBUG_TU(preprocess)

lgs_status round_planes(const float *src, int64_t src_stride, void *dst, int64_t dst_stride,
                        int n_planes, int64_t n, int dtype, cudaStream_t s) {
    count_launch();
    k_round_planes<<<grid_for((int64_t)n_planes * n, 256, 16), 256, 0, s>>>(
        src, src_stride, static_cast<uint16_t *>(dst), dst_stride, n_planes, n, dtype);
    return check_launch();
}

lgs_status preprocess(const lgs_gaussians *g, const uint32_t *map, const int32_t *d_V,
                      const lgs_camera *cam, int tw, int th, const lgs_splats *out,
                      cudaStream_t s) {
    const Cam K = make_cam(cam, tw, th);
    const unsigned grid = grid_for(g->n, kThreads, 16);
    const uint16_t *sh = static_cast<const uint16_t *>(g->sh16);
#define LGS_PRE(D, T) k_preprocess<D, T><<<grid, kThreads, 0, s>>>(g->data, sh, g->stride, g->n, map, d_V, K, out->rec, out->depth, out->radius)
#define LGS_PRE_T(D)                                                       \
    switch (g->sh_dtype) {                                                 \
    case LGS_SH_BF16: LGS_PRE(D, LGS_SH_BF16); break;                      \
    case LGS_SH_F16: LGS_PRE(D, LGS_SH_F16); break;                        \
    default: LGS_PRE(D, LGS_SH_F32); break;                                \
    }
    count_launch();
    switch (g->sh_degree) {
    case 0: LGS_PRE_T(0); break;
    case 1: LGS_PRE_T(1); break;
    case 2: LGS_PRE_T(2); break;
    default: LGS_PRE_T(3); break;
    }
#undef LGS_PRE_T
#undef LGS_PRE
    return check_launch();
}

lgs_status preprocess_bwd(const lgs_gaussians *g, const uint32_t *map, const int32_t *d_V,
                          const lgs_camera *cam, const float *gacc, float *gout, int accumulate,
                          cudaStream_t s) {
    const Cam K = make_cam(cam, 16, 16);
    const unsigned grid = grid_for(g->n, kThreads, 16);
    switch (g->sh_degree) {
    case 0: count_launch(); k_preprocess_bwd<0><<<grid, kThreads, 0, s>>>(g->data, g->stride, g->n, map, d_V, K, gacc, gout, accumulate); break;
    case 1: count_launch(); k_preprocess_bwd<1><<<grid, kThreads, 0, s>>>(g->data, g->stride, g->n, map, d_V, K, gacc, gout, accumulate); break;
    case 2: count_launch(); k_preprocess_bwd<2><<<grid, kThreads, 0, s>>>(g->data, g->stride, g->n, map, d_V, K, gacc, gout, accumulate); break;
    default: count_launch(); k_preprocess_bwd<3><<<grid, kThreads, 0, s>>>(g->data, g->stride, g->n, map, d_V, K, gacc, gout, accumulate); break;
    }
    return check_launch();
}

lgs_status preprocess_bwd_adam(const lgs_gaussians *g, float *m, float *v, const uint32_t *map,
                               const int32_t *d_V, const lgs_camera *cam, const float *rec,
                               float *gacc, const float *lr, float b1, float b2, float eps,
                               int step, float *metric, cudaStream_t s) {
    const Cam K = make_cam(cam, 16, 16);
    const AdamArgs a = make_adam(lr, LGS_NUM_PLANES(g->sh_degree), b1, b2, eps, step);
    const unsigned gf = grid_for(g->n, 256, 8);
    count_launch();
    if (rec) {
        uint16_t *sh16 = g->sh_dtype != LGS_SH_F32
                             ? static_cast<uint16_t *>(const_cast<void *>(g->sh16)) : nullptr;
        const int st = g->sh_dtype;
        switch (g->sh_degree) {
        case 0: k_bwd_adam_rec<0><<<gf, 256, 0, s>>>(g->data, m, v, g->stride, g->n, map, d_V, K, gacc, rec, a, sh16, st, metric); break;
        case 1: k_bwd_adam_rec<1><<<gf, 256, 0, s>>>(g->data, m, v, g->stride, g->n, map, d_V, K, gacc, rec, a, sh16, st, metric); break;
        case 2: k_bwd_adam_rec<2><<<gf, 256, 0, s>>>(g->data, m, v, g->stride, g->n, map, d_V, K, gacc, rec, a, sh16, st, metric); break;
        default: k_bwd_adam_rec<3><<<gf, 256, 0, s>>>(g->data, m, v, g->stride, g->n, map, d_V, K, gacc, rec, a, sh16, st, metric); break;
        }
        return check_launch();
    }
    switch (g->sh_degree) {
    case 0: k_bwd_adam_fused<0><<<gf, 256, 0, s>>>(g->data, m, v, g->stride, g->n, map, d_V, K, gacc, a, metric); break;
    case 1: k_bwd_adam_fused<1><<<gf, 256, 0, s>>>(g->data, m, v, g->stride, g->n, map, d_V, K, gacc, a, metric); break;
    case 2: k_bwd_adam_fused<2><<<gf, 256, 0, s>>>(g->data, m, v, g->stride, g->n, map, d_V, K, gacc, a, metric); break;
    default: k_bwd_adam_fused<3><<<gf, 256, 0, s>>>(g->data, m, v, g->stride, g->n, map, d_V, K, gacc, a, metric); break;
    }
    return check_launch();
}

lgs_status adam_step(float *p, const float *grad, float *m, float *v, int64_t stride, int np,
                     const float *lr, float b1, float b2, float eps, int step, const uint32_t *map,
                     const int32_t *d_V, int64_t max_rows, cudaStream_t s) {
    const AdamArgs a = make_adam(lr, np, b1, b2, eps, step);
    count_launch();
    k_adam<<<grid_for(max_rows * np, 256, 16), 256, 0, s>>>(p, grad, m, v, stride, np, map, d_V,
                                                           max_rows, a);
    return check_launch();
}

}  // namespace lgs
