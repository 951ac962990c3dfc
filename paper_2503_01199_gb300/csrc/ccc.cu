// Morton re-sort (Sec. 3.2.1) and Cluster-Cull-Compact (Sec. 3.2.2).
#include <cuda_runtime.h>

#include <mutex>

#include "lgs_internal.cuh"

namespace lgs {

namespace {

constexpr int kThreads = 256;

// ---------------------------------------------------------------------------
// Morton codes
// ---------------------------------------------------------------------------
__global__ void k_bbox_init(uint32_t *bb) {
    if (threadIdx.x < 3) bb[threadIdx.x] = 0xffffffffu;      // min (ordered)
    else if (threadIdx.x < 6) bb[threadIdx.x] = 0u;          // max (ordered)
}

// Bounding box of the centres (planes 0..2) as order-preserving uints.
__global__ void __launch_bounds__(kThreads) k_bbox(const float *__restrict__ src, int64_t n,
                                                  int64_t stride, uint32_t *bb) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float x = src[k * stride + i];
            lo[k] = fminf(lo[k], x);
            hi[k] = fmaxf(hi[k], x);
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
            hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            atomicMin(bb + k, float_to_ordered(lo[k]));
            atomicMax(bb + 3 + k, float_to_ordered(hi[k]));
        }
    }
}

// Spread the low 21 bits of x to every third bit of a 64-bit word.
__device__ __forceinline__ uint64_t spread3(uint32_t x) {
    uint64_t r = 0;
#pragma unroll
    for (int k = 0; k < 21; ++k) r |= (uint64_t)((x >> k) & 1u) << (3 * k);
    return r;
}

__global__ void __launch_bounds__(kThreads) k_morton(const float *__restrict__ src, int64_t n,
                                                    int64_t stride, const uint32_t *bb,
                                                    uint64_t *__restrict__ codes,
                                                    uint32_t *__restrict__ idx) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t q[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float lo = ordered_to_float(bb[k]), hi = ordered_to_float(bb[3 + k]);
        const float ext = __fsub_rn(hi, lo);
        float t = ext > 0.0f ? __fdiv_rn(__fsub_rn(src[k * stride + i], lo), ext) : 0.0f;
        t = fminf(fmaxf(t, 0.0f), 1.0f);
        q[k] = (uint32_t)floorf(__fmul_rn(t, 2097151.0f));
    }
    codes[i] = spread3(q[0]) | (spread3(q[1]) << 1) | (spread3(q[2]) << 2);
    idx[i] = (uint32_t)i;
}

// dst[k][i] = src[k][perm[i]] for every plane.
__global__ void __launch_bounds__(kThreads) k_gather_planes(const float *__restrict__ src,
                                                           int64_t src_stride,
                                                           float *__restrict__ dst,
                                                           int64_t dst_stride, int n_planes,
                                                           const uint32_t *__restrict__ perm,
                                                           int64_t n_max, const int32_t *d_n) {
    const int64_t n = d_n ? min((int64_t)*d_n, n_max) : n_max;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = perm[i];
        if (!LGS_DCHECK(r < n_max, kSiteGatherPerm)) continue;
        for (int k = 0; k < n_planes; ++k) dst[k * dst_stride + i] = src[k * src_stride + r];
    }
}

// ---------------------------------------------------------------------------
// cluster AABB + frustum test: one warp per cluster
// ---------------------------------------------------------------------------
struct Planes {
    float n[5][3];
    float d[5];
};

// World-space frustum planes from camera-space ones: n_world = R^T n_cam,
// d_world = n_cam . t + d_cam.
__host__ __device__ inline Planes world_planes(const float cn[5][3], const float cd[5],
                                               const float *R, const float *t) {
    Planes pl;
    for (int q = 0; q < 5; ++q) {
        for (int j = 0; j < 3; ++j)
            pl.n[q][j] = R[j] * cn[q][0] + R[3 + j] * cn[q][1] + R[6 + j] * cn[q][2];
        pl.d[q] = cn[q][0] * t[0] + cn[q][1] * t[1] + cn[q][2] * t[2] + cd[q];
    }
    return pl;
}

struct CamPlanes {
    float cn[5][3];
    float cd[5];
};

__global__ void __launch_bounds__(kThreads) k_cluster_cull(const float *__restrict__ p,
                                                          int64_t n, int64_t stride, int cs,
                                                          Planes pl, CamPlanes cp,
                                                          const float *__restrict__ pose,
                                                          float *aabb_out,
                                                          uint32_t *__restrict__ vis) {
    if (pose) {  // pose read at run time (graph replay with new cameras)
        float R[9], t[3];
        for (int i = 0; i < 9; ++i) R[i] = __ldg(pose + i);
        for (int i = 0; i < 3; ++i) t[i] = __ldg(pose + 9 + i);
        pl = world_planes(cp.cn, cp.cd, R, t);
    }
    const int64_t ncl = (n + cs - 1) / cs;
    const int lane = threadIdx.x & 31;
    for (int64_t c = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; c < ncl;
         c += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
        const int64_t r0 = c * cs, r1 = min(r0 + cs, n);
#pragma unroll 4
        for (int64_t r = r0 + lane; r < r1; r += 32) {
            const float e = 3.0f * fmaxf(expf(p[3 * stride + r]),
                                         fmaxf(expf(p[4 * stride + r]), expf(p[5 * stride + r])));
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float x = p[k * stride + r];
                lo[k] = fminf(lo[k], x - e);
                hi[k] = fmaxf(hi[k], x + e);
            }
        }
#pragma unroll
        for (int k = 0; k < 3; ++k)
            for (int o = 16; o > 0; o >>= 1) {
                lo[k] = fminf(lo[k], __shfl_xor_sync(0xffffffffu, lo[k], o));
                hi[k] = fmaxf(hi[k], __shfl_xor_sync(0xffffffffu, hi[k], o));
            }
        if (lane == 0) {
            bool v = true;
#pragma unroll
            for (int q = 0; q < 5; ++q) {
                float s = pl.d[q];
#pragma unroll
                for (int k = 0; k < 3; ++k) s += pl.n[q][k] * (pl.n[q][k] >= 0.0f ? hi[k] : lo[k]);
                v = v && (s >= 0.0f);
            }
            vis[c] = v ? 1u : 0u;
            if (aabb_out) {
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    aabb_out[6 * c + k] = lo[k];
                    aabb_out[6 * c + 3 + k] = hi[k];
                }
            }
        }
    }
}

// V = rows of visible clusters: all clusters are full except possibly the
// last, which is also last in the compacted order when it is visible.
__global__ void k_num_visible(const uint32_t *vis, const int64_t *d_nvis, int64_t n, int cs,
                              int32_t *d_V) {
    const int64_t ncl = (n + cs - 1) / cs;
    const int64_t nv = *d_nvis;
    int64_t V = nv * cs;
    if (ncl > 0 && vis[ncl - 1]) V -= ncl * cs - n;
    *d_V = (int32_t)V;
}

__global__ void __launch_bounds__(kThreads) k_compact_map(const uint32_t *__restrict__ vis,
                                                         const uint64_t *__restrict__ off,
                                                         int64_t n, int cs,
                                                         uint32_t *__restrict__ map) {
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = r / cs;
        if (vis[c]) map[(int64_t)off[c] * cs + (r - c * cs)] = (uint32_t)r;
    }
}

size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

}  // namespace

// ---------------------------------------------------------------------------
// a1
// ---------------------------------------------------------------------------
size_t morton_workspace_size(int64_t n) {
    // keys[2] (u64), vals[2] (u32), histograms, bbox
    return radix_sort_workspace(n, 8) + al256(64);
}

lgs_status morton_reorder(const float *src, float *dst, int64_t n, int64_t stride, int n_planes,
                          uint64_t *codes_out, uint32_t *perm_out, void *ws, cudaStream_t s) {
    unsigned char *w = static_cast<unsigned char *>(ws);
    uint64_t *keys[2];
    uint32_t *vals[2];
    keys[0] = reinterpret_cast<uint64_t *>(w); w += al256((size_t)n * 8);
    keys[1] = reinterpret_cast<uint64_t *>(w); w += al256((size_t)n * 8);
    vals[0] = reinterpret_cast<uint32_t *>(w); w += al256((size_t)n * 4);
    vals[1] = reinterpret_cast<uint32_t *>(w); w += al256((size_t)n * 4);
    void *hist = w; w += al256(radix_hist_bytes(n));
    uint32_t *bb = reinterpret_cast<uint32_t *>(w);
    count_launch();
    k_bbox_init<<<1, 32, 0, s>>>(bb);
    count_launch();
    k_bbox<<<grid_for(n, kThreads), kThreads, 0, s>>>(src, n, stride, bb);
    count_launch();
    k_morton<<<(unsigned)ceil_div(n, kThreads), kThreads, 0, s>>>(src, n, stride, bb, keys[0],
                                                                  vals[0]);
    lgs_status st = check_launch();
    if (st != LGS_OK) return st;
    int ob = 0;
    st = radix_sort_u64(keys, vals, n, nullptr, nullptr, 63, hist, &ob, s);
    if (st != LGS_OK) return st;
    count_launch();
    k_gather_planes<<<grid_for(n, kThreads), kThreads, 0, s>>>(src, stride, dst, stride, n_planes,
                                                              vals[ob], n, nullptr);
    if (codes_out)
        cudaMemcpyAsync(codes_out, keys[ob], (size_t)n * 8, cudaMemcpyDeviceToDevice, s);
    if (perm_out)
        cudaMemcpyAsync(perm_out, vals[ob], (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
    return check_launch();
}

// ---------------------------------------------------------------------------
// a2
// ---------------------------------------------------------------------------
DEBUG_TU(ccc)

size_t ccc_workspace_size(int64_t n, int cs) {
    const int64_t ncl = ceil_div(n, cs);
    return al256((size_t)ncl * 4) + al256((size_t)ncl * 8) + al256(8) + al256(scan_scratch_bytes());
}

lgs_status cluster_cull_compact(const lgs_gaussians *g, const lgs_camera *cam, int cs,
                                float *aabb_out, uint32_t *vis_out, uint32_t *map,
                                int32_t *d_V, void *ws, cudaStream_t s) {
    const int64_t n = g->n, ncl = ceil_div(n, cs);
    unsigned char *w = static_cast<unsigned char *>(ws);
    uint32_t *vis = reinterpret_cast<uint32_t *>(w); w += al256((size_t)ncl * 4);
    uint64_t *off = reinterpret_cast<uint64_t *>(w); w += al256((size_t)ncl * 8);
    int64_t *d_nvis = reinterpret_cast<int64_t *>(w); w += al256(8);
    void *scan_ws = w;
    // frustum planes n . x + d >= 0 (inside), camera space -> world space
    const float limx = 1.3f * cam->width / (2.0f * cam->fx);
    const float limy = 1.3f * cam->height / (2.0f * cam->fy);
    const CamPlanes cp = {{{0, 0, 1}, {-1, 0, limx}, {1, 0, limx}, {0, -1, limy}, {0, 1, limy}},
                          {-cam->znear, 0, 0, 0, 0}};
    const Planes pl = world_planes(cp.cn, cp.cd, cam->R, cam->t);
    const unsigned gcl = grid_for(ncl * 32, kThreads);
    count_launch();
    k_cluster_cull<<<gcl, kThreads, 0, s>>>(g->data, n, g->stride, cs, pl, cp, cam->d_pose,
                                            aabb_out, vis);
    lgs_status st = check_launch();
    if (st != LGS_OK) return st;
    st = exclusive_scan_u32_to_u64(vis, off, ncl, nullptr, d_nvis, scan_ws, s);
    if (st != LGS_OK) return st;
    count_launch();
    k_num_visible<<<1, 1, 0, s>>>(vis, d_nvis, n, cs, d_V);
    count_launch();
    k_compact_map<<<grid_for(n, kThreads), kThreads, 0, s>>>(vis, off, n, cs, map);
    if (vis_out) cudaMemcpyAsync(vis_out, vis, (size_t)ncl * 4, cudaMemcpyDeviceToDevice, s);
    return check_launch();
}

lgs_status compact_gather(const float *src, int64_t src_stride, float *dst, int64_t dst_stride,
                          int n_planes, const uint32_t *map, const int32_t *d_V, int64_t max_rows,
                          cudaStream_t s) {
    count_launch();
    k_gather_planes<<<grid_for(max_rows, kThreads), kThreads, 0, s>>>(
        src, src_stride, dst, dst_stride, n_planes, map, max_rows, d_V);
    return check_launch();
}

}  // namespace lgs

namespace lgs {

// ---------------------------------------------------------------------------
// lgs_cluster_cull_compact_noalloc: the same cull and compaction, with its
// scratch in a fixed device array instead of a caller workspace
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kNoallocMaxClusters = LGS_NOALLOC_MAX_CLUSTERS;
// ccc_workspace_size() for the largest cluster count: flags, offsets, count, scan
constexpr size_t kNoallocBytes = ((kNoallocMaxClusters * 4 + 255) / 256) * 256 +
                                 ((kNoallocMaxClusters * 8 + 255) / 256) * 256 + 256 + 4096;

// One copy per device that loads the library; kept until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocBytes];

std::mutex g_noalloc_mutex;
void *g_noalloc_ptr[64] = {nullptr};

// Device address of g_noalloc_scratch on the current device (looked up once
// per device and kept for the life of the process; in host code the symbol
// itself is not a device address). A device reset would leave the kept
// address stale; the entry point's contract excludes calls across one.
lgs_status noalloc_scratch(void **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return LGS_ERR_CUDA;
    }
    if (dev < 0 || dev >= 64) return LGS_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            set_cuda_error(e);
            return LGS_ERR_CUDA;
        }
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return LGS_OK;
}

}  // namespace

lgs_status cluster_cull_compact_noalloc(const lgs_gaussians *g, const lgs_camera *cam, int cs,
                                        float *aabb_out, uint32_t *vis_out, uint32_t *map,
                                        int32_t *d_V, cudaStream_t s) {
    if (ceil_div(g->n, cs) > kNoallocMaxClusters) return LGS_ERR_TOO_LARGE;
    if (ccc_workspace_size(g->n, cs) > kNoallocBytes) return LGS_ERR_TOO_LARGE;
    void *ws = nullptr;
    lgs_status st = noalloc_scratch(&ws);
    if (st != LGS_OK) return st;
    // every byte of the scratch that this call reads is written earlier in
    // the same call (flags, scan partials, offsets, count): nothing to clear
    return cluster_cull_compact(g, cam, cs, aabb_out, vis_out, map, d_V, ws, s);
}

}  // namespace lgs
