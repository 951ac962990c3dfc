// extern "C" entry points of liblgs (declared in include/lgs.h): argument
// checks, then the kernels of the other translation units.
#include <cuda_runtime.h>

#include <atomic>
#include <cstdio>

#include "lgs_internal.cuh"

namespace lgs {

// implemented in the other translation units
size_t morton_workspace_size(int64_t n);
lgs_status morton_reorder(const float *src, float *dst, int64_t n, int64_t stride, int n_planes,
                          uint64_t *codes_out, uint32_t *perm_out, void *ws, cudaStream_t s);
size_t ccc_workspace_size(int64_t n, int cs);
lgs_status cluster_cull_compact(const lgs_gaussians *g, const lgs_camera *cam, int cs,
                                float *aabb_out, uint32_t *vis_out, uint32_t *map, int32_t *d_V,
                                void *ws, cudaStream_t s);
lgs_status compact_gather(const float *src, int64_t src_stride, float *dst, int64_t dst_stride,
                          int n_planes, const uint32_t *map, const int32_t *d_V, int64_t max_rows,
                          cudaStream_t s);
lgs_status cluster_cull_compact_noalloc(const lgs_gaussians *g, const lgs_camera *cam, int cs,
                                        float *aabb_out, uint32_t *vis_out, uint32_t *map,
                                        int32_t *d_V, cudaStream_t s);
lgs_status preprocess(const lgs_gaussians *g, const uint32_t *map, const int32_t *d_V,
                      const lgs_camera *cam, int tw, int th, const lgs_splats *out, cudaStream_t s);
lgs_status preprocess_bwd(const lgs_gaussians *g, const uint32_t *map, const int32_t *d_V,
                          const lgs_camera *cam, const float *gacc, float *gout, int accumulate,
                          cudaStream_t s);
lgs_status preprocess_bwd_adam(const lgs_gaussians *g, float *m, float *v, const uint32_t *map,
                               const int32_t *d_V, const lgs_camera *cam, const float *rec,
                               float *gacc, const float *lr, float b1, float b2, float eps,
                               int step, float *metric, cudaStream_t s);
lgs_status round_planes(const float *src, int64_t src_stride, void *dst, int64_t dst_stride,
                        int n_planes, int64_t n, int dtype, cudaStream_t s);
lgs_status adam_step(float *p, const float *grad, float *m, float *v, int64_t stride, int np,
                     const float *lr, float b1, float b2, float eps, int step, const uint32_t *map,
                     const int32_t *d_V, int64_t max_rows, cudaStream_t s);
size_t bin_sort_workspace_size(int64_t maxV, int64_t cap, int ntiles);
lgs_status bin_sort(const lgs_splats *sp, const int32_t *d_V, int64_t maxV, const lgs_camera *cam,
                    int tw, int th, int cull, uint32_t *vals, int64_t cap, int64_t *d_P,
                    uint32_t *ranges, void *ws, size_t ws_bytes, cudaStream_t s);
lgs_status get_overflow(int64_t *needed);
lgs_status bin_keys(const float *depth, const uint32_t *vals, const uint32_t *ranges, int ntiles,
                    int64_t rows, uint64_t *keys, cudaStream_t s);
lgs_status raster_fwd(const lgs_splats *sp, const uint32_t *vals, const uint32_t *ranges,
                      const lgs_camera *cam, int tw, int th, int precision, float *image,
                      float *finalT, int32_t *last, cudaStream_t s);
lgs_status raster_bwd(const lgs_splats *sp, const uint32_t *vals, const uint32_t *ranges,
                      const lgs_camera *cam, int tw, int th, int precision, const float *finalT,
                      const int32_t *last, const float *dLdI, float *gacc, int64_t max_splats,
                      int accumulate, cudaStream_t s);
size_t raster_bwd_det_workspace_size(int64_t max_splats);
lgs_status raster_bwd_det(const lgs_splats *sp, const uint32_t *vals, const uint32_t *ranges,
                          const lgs_camera *cam, int tw, int th, int precision, const float *finalT,
                          const int32_t *last, const float *dLdI, float *gacc, int64_t max_splats,
                          void *ws, size_t ws_bytes, cudaStream_t s);
lgs_status det_overflow(uint32_t *count);
lgs_status loss_l1(const float *img, const float *tgt, int64_t n, float *g, float *loss,
                   cudaStream_t s);
lgs_status raster_batch(const lgs_view *views, int n_views, uint32_t total_tiles, int precision,
                        uint32_t *counter, int backward, cudaStream_t s);
size_t densify_workspace_size(int64_t n);
lgs_status densify(const lgs_gaussians *g, float *m, float *v, const float *metric, int64_t K,
                   float split_scale, const float *normals, int64_t *d_n_out,
                   uint32_t *selected, void *ws, size_t ws_bytes, cudaStream_t s);
lgs_status opacity_decay(const lgs_gaussians *g, cudaStream_t s);
lgs_status moments_accumulate(const float *gacc, const uint32_t *map, const int32_t *d_V,
                              int64_t max_rows, float *S, float *M, uint32_t *C, cudaStream_t s);
lgs_status moments_metric(const float *S, const float *M, const uint32_t *C, int64_t n,
                          float *metric, cudaStream_t s);
lgs_status opacity_variance(const float *gacc, const uint32_t *map, const int32_t *d_V,
                            int64_t max_rows, float *out, cudaStream_t s);
lgs_status peak_ex2(float *out, int blocks, int iters, cudaStream_t s);
lgs_status peak_ffma(float *out, int blocks, int iters, int packed, cudaStream_t s);
lgs_status peak_red(float *rows, int64_t n_rows, int blocks, int iters, cudaStream_t s);

namespace {
thread_local int32_t t_last_error = 0;
int g_sms[64] = {0};
std::atomic<uint64_t> g_launches{0};
}  // namespace

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_cuda_error(cudaError_t e) { t_last_error = (int32_t)e; }

lgs_status check_launch() {
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_cuda_error(e);
        return LGS_ERR_CUDA;
    }
    return LGS_OK;
}

int num_sms() {
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!g_sms[dev]) {
        int n = 0;
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        g_sms[dev] = n > 0 ? n : 1;
    }
    return g_sms[dev];
}

}  // namespace lgs

using namespace lgs;

namespace {

bool bad_camera(const lgs_camera *c) {
    return !c || c->width <= 0 || c->height <= 0 || !(c->fx > 0.f) || !(c->fy > 0.f) ||
           !(c->znear > 0.f);
}

bool bad_gaussians(const lgs_gaussians *g) {
    return !g || !g->data || g->n < 0 || g->n > 0x7fffffffLL || g->stride < g->n ||
           (g->stride & 3) || g->sh_degree < 0 || g->sh_degree > 3 || !aligned16(g->data) ||
           g->sh_dtype < LGS_SH_F32 || g->sh_dtype > LGS_SH_F16 ||
           (g->sh_dtype != LGS_SH_F32 && (!g->sh16 || !aligned16(g->sh16)));
}

// calls that update or differentiate the parameters need FP32 colour planes
// and the pose given on the host
bool training_only(const lgs_gaussians *g, const lgs_camera *c) {
    return g->sh_dtype != LGS_SH_F32 || c->d_pose != nullptr;
}

bool bad_splats(const lgs_splats *s, int64_t rows) {
    return !s || !s->rec || !s->depth || !s->radius || s->capacity < rows || !aligned16(s->rec);
}

bool bad_tiles(const lgs_camera *c, int tw, int th) {
    if (tw <= 0 || th <= 0) return true;
    const int64_t n = ceil_div(c->width, tw) * ceil_div(c->height, th);
    return n > 65536;
}

}  // namespace

extern "C" {

const char *lgs_version(void) { return "lgs 0.1 (sm_103a)"; }

int32_t lgs_last_cuda_error(void) { return t_last_error; }

uint64_t lgs_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

size_t lgs_morton_workspace_size(int64_t n) { return morton_workspace_size(n < 0 ? 0 : n); }

lgs_status lgs_morton_reorder(const float *src, float *dst, int64_t n, int64_t stride,
                              int32_t n_planes, uint64_t *codes_out, uint32_t *perm_out,
                              void *workspace, size_t workspace_bytes, lgs_stream stream) {
    if (!src || !dst || n <= 0 || n > 0x7fffffffLL || stride < n || (stride & 3) || n_planes < 3 ||
        !aligned16(src) || !aligned16(dst) || src == dst || !workspace ||
        workspace_bytes < morton_workspace_size(n))
        return LGS_ERR_INVALID_ARG;
    return morton_reorder(src, dst, n, stride, n_planes, codes_out, perm_out, workspace,
                          as_stream(stream));
}

size_t lgs_ccc_workspace_size(int64_t n, int32_t cluster_size) {
    return cluster_size > 0 ? ccc_workspace_size(n < 0 ? 0 : n, cluster_size) : 0;
}

lgs_status lgs_cluster_cull_compact(const lgs_gaussians *g, const lgs_camera *cam,
                                    int32_t cluster_size, float *aabb_out,
                                    uint32_t *cluster_visible_out, uint32_t *map_out,
                                    int32_t *d_num_visible, void *workspace,
                                    size_t workspace_bytes, lgs_stream stream) {
    if (bad_gaussians(g) || bad_camera(cam) || cluster_size <= 0 || !map_out || !d_num_visible ||
        g->n == 0 || !workspace || workspace_bytes < ccc_workspace_size(g->n, cluster_size))
        return LGS_ERR_INVALID_ARG;
    return cluster_cull_compact(g, cam, cluster_size, aabb_out, cluster_visible_out, map_out,
                                d_num_visible, workspace, as_stream(stream));
}

lgs_status lgs_cluster_cull_compact_noalloc(const lgs_gaussians *g, const lgs_camera *cam,
                                            int32_t cluster_size, float *aabb_out,
                                            uint32_t *cluster_visible_out, uint32_t *map_out,
                                            int32_t *d_num_visible, lgs_stream stream) {
    if (bad_gaussians(g) || bad_camera(cam) || cluster_size <= 0 || !map_out || !d_num_visible ||
        g->n == 0)
        return LGS_ERR_INVALID_ARG;
    return cluster_cull_compact_noalloc(g, cam, cluster_size, aabb_out, cluster_visible_out,
                                        map_out, d_num_visible, as_stream(stream));
}

lgs_status lgs_compact_gather(const float *src, int64_t src_stride, float *dst,
                              int64_t dst_stride, int32_t n_planes, const uint32_t *map,
                              const int32_t *d_num_visible, int64_t max_rows,
                              lgs_stream stream) {
    if (!src || !dst || !map || n_planes <= 0 || max_rows < 0 || src_stride <= 0 ||
        dst_stride < max_rows)
        return LGS_ERR_INVALID_ARG;
    return compact_gather(src, src_stride, dst, dst_stride, n_planes, map, d_num_visible, max_rows,
                          as_stream(stream));
}

lgs_status lgs_preprocess(const lgs_gaussians *g, const uint32_t *map,
                          const int32_t *d_num_visible, const lgs_camera *cam, int32_t tile_w,
                          int32_t tile_h, const lgs_splats *out, lgs_stream stream) {
    if (bad_gaussians(g) || bad_camera(cam) || bad_splats(out, g ? g->n : 0) ||
        bad_tiles(cam, tile_w, tile_h))
        return LGS_ERR_INVALID_ARG;
    if (g->n == 0) return LGS_OK;
    return preprocess(g, map, d_num_visible, cam, tile_w, tile_h, out, as_stream(stream));
}

size_t lgs_bin_sort_workspace_size(int64_t max_splats, int64_t pair_capacity, int32_t n_tiles) {
    if (max_splats < 0 || pair_capacity < 0) return 0;
    return bin_sort_workspace_size(max_splats, pair_capacity, n_tiles);
}

lgs_status lgs_bin_sort(const lgs_splats *sp, const int32_t *d_num_visible, int64_t max_splats,
                        const lgs_camera *cam, int32_t tile_w, int32_t tile_h, int32_t tile_cull,
                        uint32_t *vals, int64_t pair_capacity, int64_t *d_num_pairs,
                        uint32_t *tile_ranges, void *workspace, size_t workspace_bytes,
                        lgs_stream stream) {
    if (bad_camera(cam) || bad_splats(sp, max_splats) || bad_tiles(cam, tile_w, tile_h) ||
        (tile_cull != 0 && tile_cull != 1) ||
        !vals || !d_num_pairs || !tile_ranges || max_splats <= 0 || max_splats > 0x7fffffffLL ||
        pair_capacity <= 0 || pair_capacity > 0xffffffffLL || !workspace)
        return LGS_ERR_INVALID_ARG;
    const int ntiles = (int)(ceil_div(cam->width, tile_w) * ceil_div(cam->height, tile_h));
    if (workspace_bytes < bin_sort_workspace_size(max_splats, pair_capacity, ntiles))
        return LGS_ERR_INVALID_ARG;
    return bin_sort(sp, d_num_visible, max_splats, cam, tile_w, tile_h, tile_cull, vals,
                    pair_capacity, d_num_pairs, tile_ranges, workspace, workspace_bytes,
                    as_stream(stream));
}

lgs_status lgs_bin_keys(const lgs_splats *sp, const uint32_t *vals, const uint32_t *tile_ranges,
                        int32_t n_tiles, uint64_t *keys, lgs_stream stream) {
    if (!sp || !sp->depth || sp->capacity <= 0 || !vals || !tile_ranges || !keys ||
        n_tiles <= 0 || n_tiles > 65536)
        return LGS_ERR_INVALID_ARG;
    return bin_keys(sp->depth, vals, tile_ranges, n_tiles, sp->capacity, keys,
                    as_stream(stream));
}

lgs_status lgs_get_overflow(int64_t *needed) { return get_overflow(needed); }

int32_t lgs_debug_build(void) {
#ifdef LGS_DEBUG
    return 1;
#else
    return 0;
#endif
}

lgs_status lgs_get_debug_error(uint64_t *code) {
    if (!code) return LGS_ERR_INVALID_ARG;
    *code = 0;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        set_cuda_error(cudaGetLastError());
        return LGS_ERR_CUDA;
    }
    lgs_status (*const readers[])(uint64_t *) = {debug_error_raster, debug_error_sort,
                                                 debug_error_ccc, debug_error_preprocess,
                                                 debug_error_densify};
    for (auto rd : readers) {
        uint64_t c = 0;
        const lgs_status st = rd(&c);
        if (st != LGS_OK) return st;
        if (c && !*code) *code = c;
    }
    return *code ? LGS_ERR_BOUNDS : LGS_OK;
}

lgs_status lgs_set_wait_limit(uint32_t spins) {
    if (cudaDeviceSynchronize() != cudaSuccess) {
        set_cuda_error(cudaGetLastError());
        return LGS_ERR_CUDA;
    }
    const lgs_status a = sort_set_spin_limit(spins);
    return a != LGS_OK ? a : bin_set_spin_limit(spins);
}

lgs_status lgs_get_wait_timeouts(uint32_t *count) {
    if (!count) return LGS_ERR_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        set_cuda_error(cudaGetLastError());
        return LGS_ERR_CUDA;
    }
    uint32_t a = 0, b = 0;
    const lgs_status sa = sort_wait_timeouts(&a);
    const lgs_status sb = bin_wait_timeouts(&b);
    *count = a + b;
    if (sa == LGS_ERR_CUDA || sb == LGS_ERR_CUDA) return LGS_ERR_CUDA;
    return *count ? LGS_ERR_TIMEOUT : LGS_OK;
}

lgs_status lgs_raster_fwd(const lgs_splats *sp, const uint32_t *vals,
                          const uint32_t *tile_ranges, const lgs_camera *cam, int32_t tile_w,
                          int32_t tile_h, int32_t precision, float *image, float *final_T,
                          int32_t *last_contrib, lgs_stream stream) {
    if (bad_camera(cam) || bad_splats(sp, 0) || !vals || !tile_ranges || !image || !final_T ||
        !last_contrib || bad_tiles(cam, tile_w, tile_h) ||
        (precision & ~LGS_WARP_REDUCE_INT) < LGS_FP32 ||
        (precision & ~LGS_WARP_REDUCE_INT) > LGS_MIXED_BF16)
        return LGS_ERR_INVALID_ARG;
    return raster_fwd(sp, vals, tile_ranges, cam, tile_w, tile_h,
                      precision & ~LGS_WARP_REDUCE_INT, image, final_T, last_contrib,
                      as_stream(stream));
}

lgs_status lgs_raster_fwd_batch(const lgs_view *d_views, int32_t n_views, uint32_t total_tiles,
                                int32_t precision, uint32_t *d_counter, lgs_stream stream) {
    precision &= ~LGS_WARP_REDUCE_INT;
    if (!d_views || n_views < 1 || n_views > 1024 || !d_counter || precision < LGS_FP32 ||
        precision > LGS_MIXED_BF16)
        return LGS_ERR_INVALID_ARG;
    return raster_batch(d_views, n_views, total_tiles, precision, d_counter, 0, as_stream(stream));
}

lgs_status lgs_raster_bwd_batch(const lgs_view *d_views, int32_t n_views, uint32_t total_tiles,
                                int32_t precision, uint32_t *d_counter, lgs_stream stream) {
    if (!d_views || n_views < 1 || n_views > 1024 || !d_counter ||
        (precision & ~LGS_WARP_REDUCE_INT) < LGS_FP32 ||
        (precision & ~LGS_WARP_REDUCE_INT) > LGS_MIXED_BF16)
        return LGS_ERR_INVALID_ARG;
    return raster_batch(d_views, n_views, total_tiles, precision, d_counter, 1, as_stream(stream));
}

lgs_status lgs_loss_l1(const float *image, const float *target, int64_t n, float *dL_dimage,
                       float *d_loss, lgs_stream stream) {
    if (!image || !target || !dL_dimage || !d_loss || n <= 0) return LGS_ERR_INVALID_ARG;
    return loss_l1(image, target, n, dL_dimage, d_loss, as_stream(stream));
}

lgs_status lgs_raster_bwd(const lgs_splats *sp, const uint32_t *vals,
                          const uint32_t *tile_ranges, const lgs_camera *cam, int32_t tile_w,
                          int32_t tile_h, int32_t precision, const float *final_T,
                          const int32_t *last_contrib, const float *dL_dimage, float *grad_acc,
                          int64_t max_splats, int32_t accumulate, lgs_stream stream) {
    if (bad_camera(cam) || bad_splats(sp, 0) || !vals || !tile_ranges || !final_T ||
        !last_contrib || !dL_dimage || !grad_acc || !aligned16(grad_acc) || max_splats < 0 ||
        bad_tiles(cam, tile_w, tile_h) || (precision & ~LGS_WARP_REDUCE_INT) < LGS_FP32 ||
        (precision & ~LGS_WARP_REDUCE_INT) > LGS_MIXED_BF16)
        return LGS_ERR_INVALID_ARG;
    return raster_bwd(sp, vals, tile_ranges, cam, tile_w, tile_h, precision, final_T,
                      last_contrib, dL_dimage, grad_acc, max_splats, accumulate,
                      as_stream(stream));
}

size_t lgs_raster_bwd_det_workspace_size(int64_t max_splats) {
    return raster_bwd_det_workspace_size(max_splats);
}

lgs_status lgs_raster_bwd_deterministic(const lgs_splats *sp, const uint32_t *vals,
                                        const uint32_t *tile_ranges, const lgs_camera *cam,
                                        int32_t tile_w, int32_t tile_h, int32_t precision,
                                        const float *final_T, const int32_t *last_contrib,
                                        const float *dL_dimage, float *grad_acc,
                                        int64_t max_splats, void *workspace,
                                        size_t workspace_bytes, lgs_stream stream) {
    if (bad_camera(cam) || bad_splats(sp, 0) || !vals || !tile_ranges || !final_T ||
        !last_contrib || !dL_dimage || !grad_acc || !aligned16(grad_acc) || max_splats < 0 ||
        !aligned16(workspace) || bad_tiles(cam, tile_w, tile_h) ||
        (precision & ~LGS_WARP_REDUCE_INT) < LGS_FP32 ||
        (precision & ~LGS_WARP_REDUCE_INT) > LGS_MIXED_BF16)
        return LGS_ERR_INVALID_ARG;
    return raster_bwd_det(sp, vals, tile_ranges, cam, tile_w, tile_h, precision, final_T,
                          last_contrib, dL_dimage, grad_acc, max_splats, workspace,
                          workspace_bytes, as_stream(stream));
}

lgs_status lgs_get_det_overflow(uint32_t *count) {
    if (!count) return LGS_ERR_INVALID_ARG;
    return det_overflow(count);
}

lgs_status lgs_opacity_variance(const float *grad_acc, const uint32_t *map,
                                const int32_t *d_num_visible, int64_t max_rows, float *metric,
                                lgs_stream stream) {
    if (!grad_acc || !metric || max_rows < 0) return LGS_ERR_INVALID_ARG;
    return opacity_variance(grad_acc, map, d_num_visible, max_rows, metric, as_stream(stream));
}

lgs_status lgs_preprocess_bwd(const lgs_gaussians *g, const uint32_t *map,
                              const int32_t *d_num_visible, const lgs_camera *cam,
                              const float *grad_acc, float *grad_planes, int32_t accumulate,
                              lgs_stream stream) {
    if (bad_gaussians(g) || bad_camera(cam) || !grad_acc || !grad_planes || !aligned16(grad_acc) ||
        training_only(g, cam))
        return LGS_ERR_INVALID_ARG;
    if (g->n == 0) return LGS_OK;
    return preprocess_bwd(g, map, d_num_visible, cam, grad_acc, grad_planes, accumulate,
                          as_stream(stream));
}

lgs_status lgs_adam_step(float *params, const float *grads, float *m, float *v, int64_t stride,
                         int32_t n_planes, const float *lr, float beta1, float beta2, float eps,
                         int32_t step, const uint32_t *map, const int32_t *d_num_visible,
                         int64_t max_rows, lgs_stream stream) {
    if (!params || !grads || !m || !v || !lr || n_planes <= 0 || n_planes > 64 || step < 1 ||
        max_rows < 0 || stride < max_rows)
        return LGS_ERR_INVALID_ARG;
    if (max_rows == 0) return LGS_OK;
    return adam_step(params, grads, m, v, stride, n_planes, lr, beta1, beta2, eps, step, map,
                     d_num_visible, max_rows, as_stream(stream));
}

lgs_status lgs_preprocess_bwd_adam(const lgs_gaussians *g, float *m, float *v,
                                   const uint32_t *map, const int32_t *d_num_visible,
                                   const lgs_camera *cam, const lgs_splats *sp, float *grad_acc,
                                   const float *lr, float beta1, float beta2, float eps,
                                   int32_t step, float *metric, lgs_stream stream) {
    // 16-bit colour planes are accepted here as an extra output (the rounded
    // copy of the updated FP32 coefficients), with the splat records only
    if (bad_gaussians(g) || bad_camera(cam) || !m || !v || !grad_acc || !lr || step < 1 ||
        !aligned16(grad_acc) || !aligned16(m) || !aligned16(v) || cam->d_pose ||
        (g->sh_dtype != LGS_SH_F32 && !sp) || (sp && bad_splats(sp, g->n)))
        return LGS_ERR_INVALID_ARG;
    if (g->n == 0) return LGS_OK;
    return preprocess_bwd_adam(g, m, v, map, d_num_visible, cam, sp ? sp->rec : nullptr, grad_acc,
                               lr, beta1, beta2, eps, step, metric, as_stream(stream));
}

lgs_status lgs_round_planes(const float *src, int64_t src_stride, void *dst, int64_t dst_stride,
                            int32_t n_planes, int64_t n, int32_t dtype, lgs_stream stream) {
    if (!src || !dst || n_planes < 0 || n < 0 || src_stride < n || dst_stride < n ||
        (dtype != LGS_SH_BF16 && dtype != LGS_SH_F16))
        return LGS_ERR_INVALID_ARG;
    if (n_planes == 0 || n == 0) return LGS_OK;
    return round_planes(src, src_stride, dst, dst_stride, n_planes, n, dtype, as_stream(stream));
}

lgs_status lgs_moments_accumulate(const float *grad_acc, const uint32_t *map,
                                  const int32_t *d_num_visible, int64_t max_rows, float *S,
                                  float *M, uint32_t *C, lgs_stream stream) {
    if (!grad_acc || !aligned16(grad_acc) || !S || !M || !C || max_rows < 0)
        return LGS_ERR_INVALID_ARG;
    if (max_rows == 0) return LGS_OK;
    return moments_accumulate(grad_acc, map, d_num_visible, max_rows, S, M, C, as_stream(stream));
}

lgs_status lgs_moments_metric(const float *S, const float *M, const uint32_t *C, int64_t n,
                              float *metric, lgs_stream stream) {
    if (!S || !M || !C || !metric || n < 0) return LGS_ERR_INVALID_ARG;
    if (n == 0) return LGS_OK;
    return moments_metric(S, M, C, n, metric, as_stream(stream));
}

size_t lgs_densify_workspace_size(int64_t n) { return n < 0 ? 0 : densify_workspace_size(n); }

lgs_status lgs_densify(const lgs_gaussians *g, float *m, float *v, const float *metric,
                       int64_t max_new, float split_scale, const float *normals,
                       int64_t *d_n_out, uint32_t *selected_out, void *workspace,
                       size_t workspace_bytes, lgs_stream stream) {
    if (bad_gaussians(g) || g->sh_dtype != LGS_SH_F32 || !m || !v || !metric || !d_n_out ||
        max_new < 0 || (max_new > 0 && !normals) || g->stride < g->n + max_new || !workspace ||
        workspace_bytes < densify_workspace_size(g->n) || g->n + max_new > 0x7fffffffLL)
        return LGS_ERR_INVALID_ARG;
    return densify(g, m, v, metric, max_new, split_scale, normals, d_n_out, selected_out,
                   workspace, workspace_bytes, as_stream(stream));
}

lgs_status lgs_opacity_decay(const lgs_gaussians *g, lgs_stream stream) {
    if (bad_gaussians(g) || g->sh_dtype != LGS_SH_F32) return LGS_ERR_INVALID_ARG;
    if (g->n == 0) return LGS_OK;
    return opacity_decay(g, as_stream(stream));
}

lgs_status lgs_peak_ex2(float *out, int32_t blocks, int32_t iters, lgs_stream stream) {
    return peak_ex2(out, blocks, iters, as_stream(stream));
}

lgs_status lgs_peak_ffma(float *out, int32_t blocks, int32_t iters, int32_t packed,
                         lgs_stream stream) {
    return peak_ffma(out, blocks, iters, packed, as_stream(stream));
}

lgs_status lgs_peak_red(float *rows, int64_t n_rows, int32_t blocks, int32_t iters,
                        lgs_stream stream) {
    return peak_red(rows, n_rows, blocks, iters, as_stream(stream));
}

}  // extern "C"
