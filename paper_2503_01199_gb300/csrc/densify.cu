// Densification by the opacity-gradient variance, opacity decay and the
// moments summed over views (Sec. 3.3).
//
// Selection: the K Gaussians with the largest positive C Var, ties by
// index: a stable radix sort of (complemented order-preserving key, index)
// pairs; non-candidates get the largest key and sort last. Clone / split
// follow the 3DGS mechanics the paper inherits: a selected Gaussian whose
// largest scale exceeds the threshold is replaced by a sample p + R(q)(s z)
// and another sample is appended, both with scales s / 1.6; otherwise an
// exact copy is appended. Appended and split rows start with zero Adam
// moments. One thread per selected Gaussian: rows read and written by
// different threads never overlap (selected rows are distinct and appended
// rows lie beyond n).
#include <cuda_runtime.h>

#include "lgs_internal.cuh"

namespace lgs {

namespace {

constexpr int kThreads = 256;
constexpr float kLn16 = 0.47000363f;  // ln 1.6
constexpr float kLn2 = 0.69314718f;   // ln 2

__global__ void __launch_bounds__(kThreads) k_select_keys(const float *__restrict__ metric,
                                                         int64_t n, uint32_t *__restrict__ keys,
                                                         uint32_t *__restrict__ vals,
                                                         uint32_t *__restrict__ d_cand) {
    uint32_t c = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float x = metric[i];
        const bool cand = x > 0.0f;
        keys[i] = cand ? ~float_to_ordered(x) : 0xffffffffu;
        vals[i] = (uint32_t)i;
        c += cand;
    }
    c = __reduce_add_sync(0xffffffffu, c);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(d_cand, c);
}

__global__ void __launch_bounds__(kThreads) k_densify_apply(
    float *__restrict__ P, float *__restrict__ Mo, float *__restrict__ Vo, int64_t stride,
    int np, int64_t n, int64_t K, float split_scale, const float *__restrict__ normals,
    const uint32_t *__restrict__ order, const uint32_t *__restrict__ d_cand,
    uint32_t *__restrict__ selected, int64_t *__restrict__ d_n_out) {
    const int64_t kk = min(K, (int64_t)*d_cand);
    if (blockIdx.x == 0 && threadIdx.x == 0) *d_n_out = n + kk;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < kk;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = order[r], j = n + r;
        if (!LGS_DCHECK(i < n, kSiteDensifyRow)) continue;
        if (selected) selected[r] = (uint32_t)i;
        float ls[3], s[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            ls[a] = P[(3 + a) * stride + i];
            s[a] = expf(ls[a]);
        }
        const float smax = fmaxf(s[0], fmaxf(s[1], s[2]));
        for (int pl = 0; pl < np; ++pl) {
            P[pl * stride + j] = P[pl * stride + i];
            Mo[pl * stride + j] = 0.0f;
            Vo[pl * stride + j] = 0.0f;
        }
        if (smax > split_scale) {
            float q0 = P[6 * stride + i], q1 = P[7 * stride + i], q2 = P[8 * stride + i],
                  q3 = P[9 * stride + i];
            const float qi = 1.0f / sqrtf(q0 * q0 + q1 * q1 + q2 * q2 + q3 * q3);
            q0 *= qi; q1 *= qi; q2 *= qi; q3 *= qi;
            const float R[9] = {1.f - 2.f * (q2 * q2 + q3 * q3), 2.f * (q1 * q2 - q0 * q3),
                                2.f * (q1 * q3 + q0 * q2),        2.f * (q1 * q2 + q0 * q3),
                                1.f - 2.f * (q1 * q1 + q3 * q3), 2.f * (q2 * q3 - q0 * q1),
                                2.f * (q1 * q3 - q0 * q2),        2.f * (q2 * q3 + q0 * q1),
                                1.f - 2.f * (q1 * q1 + q2 * q2)};
            const float p[3] = {P[i], P[stride + i], P[2 * stride + i]};
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const float *z = normals + 6 * r + 3 * h;
                const int64_t row = h == 0 ? i : j;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    float x = p[a];
#pragma unroll
                    for (int b = 0; b < 3; ++b) x += R[3 * a + b] * (s[b] * z[b]);
                    P[a * stride + row] = x;
                    P[(3 + a) * stride + row] = ls[a] - kLn16;
                }
            }
            for (int pl = 0; pl < np; ++pl) {
                Mo[pl * stride + i] = 0.0f;
                Vo[pl * stride + i] = 0.0f;
            }
        }
    }
}

// sigmoid(l') = sigmoid(l) / 2, in the form that stays finite for any l:
// l' = -log1p(2 e^-l) for l > 0, l - ln 2 - log1p(e^l / 2) otherwise.
__global__ void __launch_bounds__(kThreads) k_opacity_decay(float *__restrict__ logit, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const float l = logit[i];
        logit[i] = l > 0.0f ? -log1pf(2.0f * expf(-l)) : l - kLn2 - log1pf(0.5f * expf(l));
    }
}

__global__ void __launch_bounds__(kThreads) k_moments_accumulate(
    const float *__restrict__ gacc, const uint32_t *__restrict__ map, const int32_t *d_V,
    int64_t max_rows, float *__restrict__ S, float *__restrict__ M, uint32_t *__restrict__ C) {
    const int64_t V = load_count(d_V, max_rows);
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < V;
         j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = map ? map[j] : j;
        if (!LGS_DCHECK(row < max_rows, kSiteDensifyRow)) continue;
        const float4 t = reinterpret_cast<const float4 *>(gacc + 16 * j)[2];
        S[row] += t.y;
        M[row] += t.z;
        C[row] += __float_as_uint(t.w);
    }
}

__global__ void __launch_bounds__(kThreads) k_moments_metric(const float *__restrict__ S,
                                                            const float *__restrict__ M,
                                                            const uint32_t *__restrict__ C,
                                                            int64_t n, float *__restrict__ out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t c = C[i];
        out[i] = c ? S[i] - M[i] * M[i] / (float)c : 0.0f;
    }
}

}  // namespace

size_t densify_workspace_size(int64_t n) {
    return radix_sort_workspace(n, 4) + 256;
}

lgs_status densify(const lgs_gaussians *g, float *m, float *v, const float *metric, int64_t K,
                   float split_scale, const float *normals, int64_t *d_n_out,
                   uint32_t *selected, void *ws, size_t ws_bytes, cudaStream_t s) {
    const int64_t n = g->n;
    unsigned char *w = static_cast<unsigned char *>(ws);
    auto take = [&](size_t b) {
        unsigned char *p = w;
        w += (b + 255) & ~(size_t)255;
        return p;
    };
    uint32_t *keys[2], *vals[2];
    for (int k = 0; k < 2; ++k) keys[k] = reinterpret_cast<uint32_t *>(take((size_t)n * 4));
    for (int k = 0; k < 2; ++k) vals[k] = reinterpret_cast<uint32_t *>(take((size_t)n * 4));
    uint32_t *d_cand = reinterpret_cast<uint32_t *>(take(4));
    void *hist = take(radix_hist_bytes(n));
    if ((size_t)(w - static_cast<unsigned char *>(ws)) > ws_bytes) return LGS_ERR_INVALID_ARG;
    cudaMemsetAsync(d_cand, 0, 4, s);
    count_launch();
    k_select_keys<<<grid_for(n, kThreads), kThreads, 0, s>>>(metric, n, keys[0], vals[0], d_cand);
    lgs_status st = check_launch();
    if (st != LGS_OK) return st;
    int ob = 0;
    st = radix_sort_u32(keys, vals, n, nullptr, nullptr, 32, hist, &ob, s);
    if (st != LGS_OK) return st;
    count_launch();
    k_densify_apply<<<grid_for(K > 0 ? K : 1, kThreads), kThreads, 0, s>>>(
        g->data, m, v, g->stride, LGS_NUM_PLANES(g->sh_degree), n, K, split_scale, normals,
        vals[ob], d_cand, selected, d_n_out);
    return check_launch();
}

lgs_status opacity_decay(const lgs_gaussians *g, cudaStream_t s) {
    count_launch();
    k_opacity_decay<<<grid_for(g->n, kThreads), kThreads, 0, s>>>(g->data + 10 * g->stride, g->n);
    return check_launch();
}

lgs_status moments_accumulate(const float *gacc, const uint32_t *map, const int32_t *d_V,
                              int64_t max_rows, float *S, float *M, uint32_t *C, cudaStream_t s) {
    count_launch();
    k_moments_accumulate<<<grid_for(max_rows, kThreads), kThreads, 0, s>>>(gacc, map, d_V,
                                                                          max_rows, S, M, C);
    return check_launch();
}

lgs_status moments_metric(const float *S, const float *M, const uint32_t *C, int64_t n,
                          float *metric, cudaStream_t s) {
    count_launch();
    k_moments_metric<<<grid_for(n, kThreads), kThreads, 0, s>>>(S, M, C, n, metric);
    return check_launch();
}

DEBUG_TU(densify)

}  // namespace lgs
