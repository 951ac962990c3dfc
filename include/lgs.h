/*
 * lgs.h -- C ABI of a GB300 (sm_103a) implementation of the training-step hot
 * path of LiteGS (arXiv 2503.01199): the tile-based differentiable Gaussian
 * rasterizer with its Cluster-Cull-Compact data path, per-Gaussian gradient
 * reduction, opacity-gradient variance statistic and sparse Adam update.
 *
 * Conventions for every call:
 *   - Pointers named d_* or documented as "device" are device pointers owned
 *     by the caller. The library never allocates, frees or retains them.
 *     Scratch memory comes from a caller-supplied workspace whose size is
 *     given by the matching *_workspace_size() query. Host structs (camera,
 *     Gaussian descriptor, splat descriptor) are read during the call only.
 *   - Float arrays must be 16-byte aligned; plane strides are in elements
 *     and must be multiples of 4.
 *   - Every call only enqueues work on `stream` (a cudaStream_t; 0 is the
 *     legacy default stream) and returns without synchronising, so a
 *     sequence of calls can be captured in a CUDA graph. Counts that are only
 *     known on the device (the number of visible Gaussians V, the number of
 *     tile/splat pairs P) stay on the device; kernels are sized by the host
 *     bound (n, capacity) and read the device count.
 *   - Return value: LGS_OK, LGS_ERR_INVALID_ARG (null or misaligned pointer,
 *     bad size, unsupported option; nothing was enqueued), LGS_ERR_CUDA (a
 *     launch failed; see lgs_last_cuda_error()), LGS_ERR_CAPACITY (only from
 *     lgs_get_overflow()).
 *
 * Gaussian parameters (Sec. 3: g_i = {p, Sigma, c, o}) are stored as planes
 * of float32, plane k of Gaussian i at data[k * stride + i]:
 *   0..2   centre p (world x, y, z)
 *   3..5   log of the per-axis scale (Sigma = R S S^T R^T, S = diag(exp(.)))
 *   6..9   rotation quaternion (w, x, y, z), any non-zero length
 *   10     opacity logit (o = sigmoid(logit))
 *   11..   colour coefficients c_i: SH coefficient k, channel ch at plane
 *          11 + 3k + ch, k < (sh_degree + 1)^2 (real SH, l-major, m = -l..l)
 * so a Gaussian has 11 + 3 (deg + 1)^2 planes: 14 at degree 0, 59 at 3.
 *
 * Projected splat record (Sec. 3: {x, y, Sigma^screen, c, o}), 12 floats per
 * visible Gaussian j, 48-byte aligned rows of `rec`:
 *   rec[12 j + 0..9] = u, v, A, B, C, o, r, g, b, tau
 * where (u, v) is the screen centre in pixels, (A, B, C) the inverse 2D
 * covariance [[A, B], [B, C]] used in the exponent of Eq. 2, o the opacity,
 * (r, g, b) the colour and tau the largest value of the exponent's quadratic
 * form d^T [[A, B], [B, C]] d at which alpha = o exp(-q/2) can reach 1/255:
 * tau = 2 ln(255 o) widened by 1e-3 (1 + |tau|). Slots 10..11 are reserved.
 * depth[j] is the camera-space z, radius[j] the integer screen radius
 * (0 = culled).
 *
 * Pixel (x, y) is sampled at its centre (x + 0.5, y + 0.5). Images are
 * planar float32 [3][height][width].
 */
#ifndef LGS_H
#define LGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t lgs_status;
#define LGS_OK 0
#define LGS_ERR_INVALID_ARG 1
#define LGS_ERR_CAPACITY 2
#define LGS_ERR_CUDA 3
#define LGS_ERR_TIMEOUT 4
#define LGS_ERR_TOO_LARGE 5 /* size beyond a fixed maximum of this library */
#define LGS_ERR_BOUNDS 6    /* a bounds check of the debug build failed */

typedef void *lgs_stream; /* cudaStream_t */

/* Number of parameter planes of a Gaussian of the given SH degree. */
#define LGS_NUM_PLANES(deg) (11 + 3 * ((deg) + 1) * ((deg) + 1))
#define LGS_MAX_PLANES 59
#define LGS_SPLAT_FLOATS 12
#define LGS_GRAD_FLOATS 16

/* Pinhole camera. R is the row-major world-to-camera rotation, t the
 * translation (camera = R world + t); the camera looks along +z. */
typedef struct lgs_camera {
    float R[9];
    float t[3];
    float fx, fy, cx, cy;
    int32_t width, height;
    float znear; /* Gaussians with camera z <= znear are culled */
    float bg[3]; /* background colour composited behind the last splat */
    /* Optional device pointer to 12 floats (R row-major, then t). When not
     * NULL, lgs_cluster_cull_compact and lgs_preprocess read the pose from
     * it when their kernels run instead of R and t above, so a captured CUDA
     * graph can be replayed for new poses (resolution and intrinsics stay
     * those of the capture). The backward calls reject it. */
    const float *d_pose;
} lgs_camera;

/* Gaussian parameter planes (see above). Device memory. */
typedef struct lgs_gaussians {
    float *data;
    int64_t n;      /* number of Gaussians */
    int64_t stride; /* plane stride in floats, >= n, multiple of 4 */
    int32_t sh_degree; /* 0..3 */
    /* Storage of the colour coefficients: LGS_SH_F32 (planes 11.. of data)
     * or LGS_SH_BF16 / LGS_SH_F16: 16-bit planes at sh16 + k * stride,
     * k = 3 coefficient + channel (planes 0..10 stay float32 in data).
     * 16-bit storage is for rendering (lgs_cluster_cull_compact,
     * lgs_preprocess) and for the fused lgs_preprocess_bwd_adam, which keeps
     * FP32 masters in data and writes the rounded copy; the other backward
     * and optimizer calls reject it. */
    int32_t sh_dtype;
    const void *sh16;
} lgs_gaussians;

#define LGS_SH_F32 0
#define LGS_SH_BF16 1
#define LGS_SH_F16 2

/* Projected splats, indexed by compacted index j < V. Device memory. */
typedef struct lgs_splats {
    float *rec;       /* [capacity][12] */
    float *depth;     /* [capacity]     */
    int32_t *radius;  /* [capacity]     */
    int64_t capacity; /* rows available; must be >= the V it is used with */
} lgs_splats;

/* Library version string and the CUDA error of the last failed launch. */
const char *lgs_version(void);
int32_t lgs_last_cuda_error(void);

/* Number of kernels this library has launched in this process (all
 * devices, all threads); for accounting, e.g. launches per training step. */
uint64_t lgs_kernel_launches(void);

/* ------------------------------------------------------------------------
 * a1. Morton re-sort (Sec. 3.2.1). Computes the 64-bit Morton code of every
 * centre (planes 0..2 of src): centres normalised to [0,1]^3 by their
 * bounding box (a degenerate axis maps to 0), scaled by 2^21 - 1 and
 * truncated in single precision, bits interleaved x, y, z from the least
 * significant bit (the paper's printed shifts 2k, 2k+1, 2k+2 are read as
 * 3k, 3k+1, 3k+2). Sorts the codes stably (ties keep the input order) and
 * gathers all n_planes planes of src into dst in that order:
 *   dst[k * stride + i] = src[k * stride + perm[i]].
 * src and dst must not overlap; plane count may include optimiser moments
 * stored as further planes with the same stride.
 * Outputs (device, nullable): codes_out[i] = sorted code, perm_out[i] = row
 * of src that landed in row i.
 * ---------------------------------------------------------------------- */
size_t lgs_morton_workspace_size(int64_t n);
lgs_status lgs_morton_reorder(const float *src, float *dst, int64_t n, int64_t stride,
                              int32_t n_planes, uint64_t *codes_out, uint32_t *perm_out,
                              void *workspace, size_t workspace_bytes, lgs_stream stream);

/* ------------------------------------------------------------------------
 * a2. Cluster-Cull-Compact (Sec. 3.2.2, App. A.3 figure). Rows are grouped
 * into clusters of cluster_size consecutive rows (the last may be partial).
 * Each cluster's axis-aligned box bounds its centres widened by 3 x the
 * largest scale of each Gaussian; a cluster is culled when its box lies
 * entirely outside one of five planes: the near plane z = znear and the four
 * side planes through the camera centre at 1.3 x the half field of view
 * (the paper names view-frustum culling of cluster AABBs; the planes and the
 * widening are this library's reading). Visible clusters are compacted in
 * increasing order: map[j] is the row of compacted index j, and
 * *d_num_visible = V, the total rows of visible clusters.
 * Outputs (device): map [n] (rows >= V undefined), d_num_visible [1];
 * optional aabb [ceil(n / cluster_size)][6] (min xyz, max xyz) and
 * cluster_visible [ceil(n / cluster_size)] (0/1).
 * The paper copies visible rows into a contiguous buffer; here the map is
 * the compaction (kernels read cluster-contiguous rows through it), and
 * lgs_compact_gather() performs the physical copy when one is wanted.
 * ---------------------------------------------------------------------- */
size_t lgs_ccc_workspace_size(int64_t n, int32_t cluster_size);
lgs_status lgs_cluster_cull_compact(const lgs_gaussians *g, const lgs_camera *cam,
                                    int32_t cluster_size, float *aabb_out,
                                    uint32_t *cluster_visible_out, uint32_t *map_out,
                                    int32_t *d_num_visible, void *workspace,
                                    size_t workspace_bytes, lgs_stream stream);

/* Allocation-free variant of lgs_cluster_cull_compact (the paper has no
 * counterpart; it is an interface addition of this library).
 * Some callers cannot call cudaMalloc or hand out a workspace: code that runs
 * inside another framework's memory pool and must not allocate outside it,
 * code that must not synchronise the device (cudaMalloc and cudaFree can),
 * and plugin or render-loop hosts that forbid allocation at frame time. This
 * entry point takes the same inputs and writes the same outputs as
 * lgs_cluster_cull_compact, but its scratch lives in a fixed array of
 * device memory inside the library (about 770 KB; every GPU that loads the
 * library holds it until the process exits). It calls no cudaMalloc, no
 * cudaFree and no allocating library routine.
 *   - Limit: ceil(n / cluster_size) <= LGS_NOALLOC_MAX_CLUSTERS (8,388,608
 *     Gaussians at 128 per cluster); larger inputs return LGS_ERR_TOO_LARGE
 *     and enqueue nothing.
 *   - The first call on a device looks up the array's device address (once
 *     per device, with that device current) and keeps it for the life of the
 *     process. Make that first call before any stream capture. Calls must
 *     not cross a device reset (cudaDeviceReset, or anything else that
 *     destroys and re-creates the device's primary context): the kept
 *     address would then be stale.
 *   - All calls share the one array, which keeps the last call's contents
 *     (nothing in it needs to start at zero). Calls that overlap on the GPU,
 *     e.g. on two streams without ordering between them, race on it: order
 *     them on one stream or with events. */
#define LGS_NOALLOC_MAX_CLUSTERS 65536
lgs_status lgs_cluster_cull_compact_noalloc(const lgs_gaussians *g, const lgs_camera *cam,
                                            int32_t cluster_size, float *aabb_out,
                                            uint32_t *cluster_visible_out, uint32_t *map_out,
                                            int32_t *d_num_visible, lgs_stream stream);

/* dst[k * dst_stride + j] = src[k * src_stride + map[j]] for j < V (device). */
lgs_status lgs_compact_gather(const float *src, int64_t src_stride, float *dst,
                              int64_t dst_stride, int32_t n_planes, const uint32_t *map,
                              const int32_t *d_num_visible, int64_t max_rows,
                              lgs_stream stream);

/* ------------------------------------------------------------------------
 * a3. Preprocess (Sec. 3: the projected primitive {x, y, Sigma^screen, c,
 * o}; the paper inherits the projection from 3DGS). For compacted index
 * j < V, row i = map[j] (map NULL: i = j, d_num_visible NULL: V = g->n):
 *   camera-space centre t = R p + T; culled if t.z <= znear;
 *   Sigma = R(q) diag(exp(2 s)) R(q)^T;
 *   J = [[fx/z, 0, -fx x'/z^2], [0, fy/z, -fy y'/z^2]] with x', y' the
 *   centre clamped to 1.3 x the half field of view;
 *   Sigma2D = J R Sigma R^T J^T + 0.3 I; (A, B, C) = inverse of Sigma2D;
 *   (u, v) = (fx x/z + cx, fy y/z + cy);
 *   radius = ceil(3 sqrt(lambda_max)), lambda_max = m + sqrt(max(0.1, m^2 - det)),
 *   m = trace/2; culled (radius 0) if its tile rectangle is empty;
 *   colour = max(0, sum_k c_k Y_k(dir) + 0.5), dir = (p - camera centre)/|.|;
 *   o = sigmoid(logit).
 * Writes out->rec, out->depth, out->radius rows j < V.
 * ---------------------------------------------------------------------- */
lgs_status lgs_preprocess(const lgs_gaussians *g, const uint32_t *map,
                          const int32_t *d_num_visible, const lgs_camera *cam, int32_t tile_w,
                          int32_t tile_h, const lgs_splats *out, lgs_stream stream);

/* ------------------------------------------------------------------------
 * a4. Tile binning and sort (Sec. 3.1 "tile-based method"; Eq. 1 requires
 * each tile's splats in depth order s(i)). A splat is listed in every tile
 * whose pixel square meets [u - r, u + r] x [v - r, v + r]:
 *   x0 = floor((u - r) / tile_w), x1 = floor((u + r) / tile_w) + 1 (same in
 *   y), clamped to the tile grid, computed in single precision.
 * With tile_cull = 1 (the tile-level culling of App. A.1) a tile of that
 * rectangle is listed only if the minimum of d^T [[A, B], [B, C]] d over the
 * box of its pixel centres (d = splat centre - pixel centre) is <= tau: the
 * other tiles cannot receive a contribution (alpha < 1/255 at every pixel),
 * so images, transmittances and gradients are the same as with
 * tile_cull = 0; only list positions change. Both tests are single
 * precision with explicit rounding.
 * Each tile's list is in increasing depth; equal depths keep increasing
 * compacted index (a stable sort of the key (tile << 32 | depth bits)).
 * Outputs (device): vals[P] = compacted splat index of each pair, grouped by
 * tile (the tiles' groups are laid out in an order of the library's
 * choosing); tile_ranges[2 t], [2 t + 1] = begin, end of tile t's list in
 * vals (row-major tile id t = ty * grid_w + tx); *d_num_pairs = P.
 * If P > pair_capacity only the first pair_capacity pairs are written, the
 * device overflow flag is raised and lgs_get_overflow() reports the size
 * needed; the image is then incomplete. The workspace sized by
 * pair_capacity also holds one item per (super-tile of 8 x 4 tiles, splat
 * listed in one of its tiles), never more than P; a count above
 * pair_capacity overflows the same way. The tile grid may have at most
 * 65536 tiles and 65535 columns (LGS_ERR_INVALID_ARG otherwise).
 * ---------------------------------------------------------------------- */
/* n_tiles: the tile count of the largest image the workspace will serve. */
size_t lgs_bin_sort_workspace_size(int64_t max_splats, int64_t pair_capacity, int32_t n_tiles);
lgs_status lgs_bin_sort(const lgs_splats *sp, const int32_t *d_num_visible, int64_t max_splats,
                        const lgs_camera *cam, int32_t tile_w, int32_t tile_h, int32_t tile_cull,
                        uint32_t *vals, int64_t pair_capacity, int64_t *d_num_pairs,
                        uint32_t *tile_ranges, void *workspace, size_t workspace_bytes,
                        lgs_stream stream);

/* The 64-bit sort keys of a finished binning, for callers that want them
 * beside vals: keys[p] = (t << 32) | bits of depth[vals[p]] (the float's
 * bits; depths are positive, so the bits order as the depths) for every pair
 * p of every tile t < n_tiles, in tile_ranges' layout. Within a tile's
 * range the keys do not decrease. sp: the splats the binning read (depth,
 * capacity); vals, tile_ranges: its outputs (device); keys: device, one per
 * pair. A splat index >= sp->capacity gets the key of an infinite depth.
 * LGS_ERR_INVALID_ARG for a null pointer or n_tiles outside 1..65536. */
lgs_status lgs_bin_keys(const lgs_splats *sp, const uint32_t *vals, const uint32_t *tile_ranges,
                        int32_t n_tiles, uint64_t *keys, lgs_stream stream);

/* Synchronises the device, returns LGS_ERR_CAPACITY and the largest pair
 * count seen if some lgs_bin_sort overflowed since the last query (and
 * clears the flag), else LGS_OK with *needed = 0. */
lgs_status lgs_get_overflow(int64_t *needed);

/* Synchronises the device; *count receives the number of bounded device-side
 * waits that gave up since the last query (the radix sorts' look-back over
 * earlier tiles and the binning's look-back over earlier groups of splats; a
 * wait that gives up leaves that result wrong instead of hanging), and the
 * count is cleared. Returns LGS_ERR_TIMEOUT if it was
 * non-zero, else LGS_OK. */
lgs_status lgs_get_wait_timeouts(uint32_t *count);

/* Synchronises the device and sets how many times a bounded device wait
 * polls a predecessor that has not published before it gives up (default
 * LGS_DEFAULT_WAIT_LIMIT; 0 gives up at the first such poll). It exists to
 * exercise the give-up path in tests: a wait that gives up takes the
 * partial prefix it has summed, never larger than the true one, so every
 * position computed from it stays inside its output (the result is wrong
 * and lgs_get_wait_timeouts reports it) and nothing hangs. No paper
 * counterpart. */
#define LGS_DEFAULT_WAIT_LIMIT 4194304u
lgs_status lgs_set_wait_limit(uint32_t spins);

/* The bounds-checked debug build (liblgs_debug.so, compiled with
 * -DLGS_DEBUG; no paper counterpart). Its kernels check the indices they
 * take from their inputs before using them: splat indices of the tile
 * lists against the splat rows (lgs_splats.capacity) in the raster calls,
 * gradient rows against max_splats in the backward, the radix sort's
 * scatter positions against the key count, the Morton gather's source rows
 * and the compaction-map rows of the preprocess, its backward, the fused
 * backward + Adam and the plain Adam step against the row count, and the
 * densification's source rows and moment rows. A failed check skips the
 * access and records its site and source line; the binning writes only
 * behind its capacity guards and is not checked. lgs_debug_build()
 * returns 1 in that build, 0 in the release build.
 * lgs_get_debug_error() synchronises the device; *code = (site << 32) |
 * line of the first failed check since the last query (0: none), cleared
 * on read; LGS_ERR_BOUNDS if one failed, else LGS_OK (always LGS_OK in the
 * release build, whose kernels carry no checks). Sites: 1 tile-list splat
 * index, 2 gradient row, 3 sort scatter, 4 gather row, 5 preprocess map
 * row (also of the fused backward + Adam), 6 Adam map row, 7 densification
 * row. */
int32_t lgs_debug_build(void);
lgs_status lgs_get_debug_error(uint64_t *code);

/* Arithmetic of the per-pixel blend in lgs_raster_fwd / lgs_raster_bwd.
 * LGS_FP32: everything in FP32. LGS_MIXED_FP16 / LGS_MIXED_BF16 (the
 * mixed-precision raster of Sec. 3.1, with BF16 as a second 16-bit type):
 * the Gaussian value G = exp(power), o G and alpha are computed in 16 bits
 * for pairs of pixels; the exponent's quadratic form (from the FP32 inverse
 * covariance), transmittance, colour accumulation and every gradient sum stay
 * FP32. A backward must use the precision of the forward whose final_T and
 * last_contrib it reads. */
#define LGS_FP32 0
#define LGS_MIXED_FP16 1
#define LGS_MIXED_BF16 2
/* OR-ed into the precision of lgs_raster_bwd / lgs_raster_bwd_batch: each
 * warp sums its gradient terms by the integer warp reduction of Sec. 3.1
 * (warp max of the exponents, values aligned to it as 26-bit integers, an
 * exact integer warp sum, the float rebuilt): the per-warp sum does not
 * depend on lane order; each term loses at most 2^-25 of the warp's largest
 * term. The forward calls ignore it. */
#define LGS_WARP_REDUCE_INT 16

/* ------------------------------------------------------------------------
 * a5. Forward rasterisation (Eq. 1-2, Alg. 1). Per pixel, front to back
 * over its tile's list: alpha = min(0.99, o exp(-0.5 (A dx^2 + C dy^2) -
 * B dx dy)) with (dx, dy) = (u, v) - pixel centre; alpha < 1/255 is skipped;
 * if T (1 - alpha) < 1e-4 the pixel stops without this splat; otherwise
 * colour += c alpha T and T *= 1 - alpha. image = colour + T bg.
 * Outputs (device): image [3][H][W]; final_T [H][W]; last_contrib [H][W] =
 * 1 + position within the tile list of the last composited splat (0: none).
 * tile_w x tile_h must be 16 x 16. precision: LGS_FP32, LGS_MIXED_FP16 or
 * LGS_MIXED_BF16.
 * ---------------------------------------------------------------------- */
lgs_status lgs_raster_fwd(const lgs_splats *sp, const uint32_t *vals,
                          const uint32_t *tile_ranges, const lgs_camera *cam, int32_t tile_w,
                          int32_t tile_h, int32_t precision, float *image, float *final_T,
                          int32_t *last_contrib, lgs_stream stream);

/* ------------------------------------------------------------------------
 * Batched views (a5 / a7 for several cameras in one launch). One persistent
 * kernel takes the tiles of all views from a shared counter, so views of
 * different sizes fill the GPU together. The table of views lives in
 * DEVICE memory (it is read by the kernels; its contents may stay fixed
 * across replays of a captured graph). Tiles are numbered view after view:
 * view v owns tiles tile_offset[v] .. tile_offset[v] + tiles(v) - 1, with
 * tile_offset increasing and tile_offset[0] = 0; total_tiles is the sum.
 * Each view is rendered exactly as lgs_raster_fwd / lgs_raster_bwd render
 * it alone (16 x 16 tiles); the backward always adds into grad_acc, which
 * the caller zeroes. counter: one device uint32 of scratch (zeroed by the
 * call). n_views <= 1024.
 * ---------------------------------------------------------------------- */
typedef struct lgs_view {
    const float *rec;             /* splat records of this view (lgs_splats.rec) */
    const uint32_t *vals;         /* tile lists of this view (lgs_bin_sort) */
    const uint32_t *tile_ranges;  /* [tiles][2] (lgs_bin_sort) */
    float *image;                 /* forward out: [3][height][width] */
    float *final_T;               /* forward out, backward in: [height][width] */
    int32_t *last_contrib;        /* forward out, backward in: [height][width] */
    const float *dL_dimage;       /* backward in: [3][height][width] */
    float *grad_acc;              /* backward: rows added as by lgs_raster_bwd */
    int32_t width, height;
    uint32_t tile_offset;
    float bg[3];
} lgs_view;

lgs_status lgs_raster_fwd_batch(const lgs_view *d_views, int32_t n_views, uint32_t total_tiles,
                                int32_t precision, uint32_t *d_counter, lgs_stream stream);
lgs_status lgs_raster_bwd_batch(const lgs_view *d_views, int32_t n_views, uint32_t total_tiles,
                                int32_t precision, uint32_t *d_counter, lgs_stream stream);

/* ------------------------------------------------------------------------
 * a6. L1 photometric loss (the paper does not state its loss; this is the
 * L1 term of 3DGS): loss = mean |image - target| over n values,
 * dL_dimage = sign(image - target) / n (sign(0) = 0). *d_loss (device) is
 * overwritten.
 * ---------------------------------------------------------------------- */
lgs_status lgs_loss_l1(const float *image, const float *target, int64_t n, float *dL_dimage,
                       float *d_loss, lgs_stream stream);

/* ------------------------------------------------------------------------
 * a7. Backward rasterisation with per-Gaussian reduction (Eq. 3; App. A.1
 * Eq. 4-6) and opacity-gradient moments (Sec. 3.3). Per pixel the included
 * splats are revisited back to front from last_contrib, the transmittance
 * recovered as T / (1 - alpha) from final_T, and
 *   dL/dc = alpha T dL/dI,
 *   dL/dalpha = T (c - acc) . dL/dI - T_final bg . dL/dI / (1 - alpha),
 * acc = colour composited behind. Per splat the per-pixel terms are summed
 * over each 8 x 8 quadrant of the tile (a warp's reduction) before one
 * atomic add per value: up to four atomics per value per tile.
 * grad_acc (device) [max_splats][16] floats, row j:
 *   0 du, 1 dv, 2 dA, 3 dB, 4 dC, 5 do (activated opacity), 6..8 dr dg db,
 *   9 S = sum of (dL/do per pixel)^2, 10 M = sum of dL/do per pixel,
 *   11 C = count of included fragments as uint32, 12..15 zero.
 * accumulate = 0 zeroes rows j < max_splats first; 1 adds to them.
 * precision must be the one the forward used, optionally with
 * LGS_WARP_REDUCE_INT.
 * ---------------------------------------------------------------------- */
lgs_status lgs_raster_bwd(const lgs_splats *sp, const uint32_t *vals,
                          const uint32_t *tile_ranges, const lgs_camera *cam, int32_t tile_w,
                          int32_t tile_h, int32_t precision, const float *final_T,
                          const int32_t *last_contrib, const float *dL_dimage, float *grad_acc,
                          int64_t max_splats, int32_t accumulate, lgs_stream stream);

/* ------------------------------------------------------------------------
 * a7, bit-reproducible (the accumulation of Sec. 3.1's integer warp
 * reduction carried through to the gradient rows). The same gradients and
 * moments as lgs_raster_bwd, but every (quadrant, splat) contribution is
 * added to its splat as an integer in units of 2^-64 (96-bit two's
 * complement, kept as two 64-bit limbs in the workspace) instead of by a
 * float atomic, so the result does not depend on the order in which the
 * GPU's warps add to a row: two calls on the same inputs give identical
 * bits. With LGS_WARP_REDUCE_INT the warp's exact integer sum is added as
 * it is, so the only error beyond the per-fragment FP32 arithmetic is the
 * integer reduction's truncation (at most 2^-25 of the warp's largest term
 * per lane), at most 2^-64 per contribution below the unit, and the final
 * rounding of each value to FP32.
 * grad_acc rows j < max_splats are OVERWRITTEN (no accumulate option); the
 * row layout is lgs_raster_bwd's. workspace (device, 16-byte aligned, any
 * contents) of lgs_raster_bwd_det_workspace_size(max_splats) bytes =
 * 160 bytes per row. A contribution of magnitude >= 2^30 is left out and
 * counted (lgs_get_det_overflow). Errors: LGS_ERR_INVALID_ARG for the
 * arguments lgs_raster_bwd rejects or a workspace that is too small.
 * ---------------------------------------------------------------------- */
size_t lgs_raster_bwd_det_workspace_size(int64_t max_splats);
lgs_status lgs_raster_bwd_deterministic(const lgs_splats *sp, const uint32_t *vals,
                                        const uint32_t *tile_ranges, const lgs_camera *cam,
                                        int32_t tile_w, int32_t tile_h, int32_t precision,
                                        const float *final_T, const int32_t *last_contrib,
                                        const float *dL_dimage, float *grad_acc,
                                        int64_t max_splats, void *workspace,
                                        size_t workspace_bytes, lgs_stream stream);
/* Synchronises the device; *count receives the number of contributions
 * lgs_raster_bwd_deterministic left out as out of range since the last
 * query, and the count is cleared. LGS_ERR_CAPACITY if non-zero. */
lgs_status lgs_get_det_overflow(uint32_t *count);

/* ------------------------------------------------------------------------
 * a8. Densification metric (Sec. 3.3): C Var = S - M^2 / C (0 if C = 0) for
 * compacted j < V, written to metric[map[j]] (map NULL: metric[j]).
 * ---------------------------------------------------------------------- */
lgs_status lgs_opacity_variance(const float *grad_acc, const uint32_t *map,
                                const int32_t *d_num_visible, int64_t max_rows, float *metric,
                                lgs_stream stream);

/* ------------------------------------------------------------------------
 * a9. Preprocess backward: the chain rule through a3 from grad_acc rows
 * 0..8 to the parameter planes. For j < V, writes (accumulate = 0) or adds
 * to (accumulate = 1, e.g. summing the views of a batch) plane k, row map[j]
 * of grad_planes (stride g->stride, LGS_NUM_PLANES(deg) planes); other rows
 * are not touched. Every clamp passes zero gradient while active.
 * ---------------------------------------------------------------------- */
lgs_status lgs_preprocess_bwd(const lgs_gaussians *g, const uint32_t *map,
                              const int32_t *d_num_visible, const lgs_camera *cam,
                              const float *grad_acc, float *grad_planes, int32_t accumulate,
                              lgs_stream stream);

/* ------------------------------------------------------------------------
 * a10. Adam on visible rows only (Sec. 3.2.3: sparse update at cluster
 * granularity on contiguous blocks). For j < V, row i = map[j], plane k:
 *   m = b1 m + (1 - b1) g;  v = b2 v + (1 - b2) g^2;
 *   p -= lr[k] (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * lr is a host array of n_planes (<= 64) learning rates. Rows of culled
 * clusters are not touched.
 * ---------------------------------------------------------------------- */
lgs_status lgs_adam_step(float *params, const float *grads, float *m, float *v, int64_t stride,
                         int32_t n_planes, const float *lr, float beta1, float beta2, float eps,
                         int32_t step, const uint32_t *map, const int32_t *d_num_visible,
                         int64_t max_rows, lgs_stream stream);

/* a9 + a10 without a gradient buffer: each parameter's gradient is applied
 * by Adam as soon as it is computed. m and v are planes with the stride of g;
 * g->data is updated in place. Same results as lgs_preprocess_bwd followed by
 * lgs_adam_step up to rounding. grad_acc is read only.
 * sp (may be NULL): the splat records lgs_preprocess wrote for this camera
 * from these parameters (rows j < V read, capacity >= g->n). With them the colour clamp
 * is taken from the stored colours instead of recomputing the colours, so
 * the SH planes are read once; without them the colours are recomputed.
 * 16-bit colour (the mixed-precision variant that keeps SH in FP16 / BF16
 * for the forward): with g->sh_dtype LGS_SH_BF16 / LGS_SH_F16, g->data still
 * holds all num_planes FP32 planes, which are the Adam masters, and every
 * colour coefficient the step updates is also written, rounded to nearest
 * even, to the 16-bit plane at g->sh16 (an output here); sp is then
 * required. A forward on the same g (lgs_preprocess) reads the 16-bit
 * planes.
 * metric (device, may be NULL): when given, the call also writes the a8
 * densification metric C Var = S - M^2 / C (0 if C = 0) of every row
 * map[j], j < V, from grad_acc's S, M and C, bit for bit what
 * lgs_opacity_variance writes, so that a step needs no separate a8 launch. */
lgs_status lgs_preprocess_bwd_adam(const lgs_gaussians *g, float *m, float *v,
                                   const uint32_t *map, const int32_t *d_num_visible,
                                   const lgs_camera *cam, const lgs_splats *sp, float *grad_acc,
                                   const float *lr, float beta1, float beta2, float eps,
                                   int32_t step, float *metric, lgs_stream stream);

/* dst[k][i] = src[k][i] rounded to nearest even in dtype (LGS_SH_BF16 or
 * LGS_SH_F16), planes k < n_planes, rows i < n; src float32 planes of stride
 * src_stride, dst 16-bit planes of stride dst_stride (device). The 16-bit
 * colour copy of FP32 colour planes (e.g. after a Morton re-sort). */
lgs_status lgs_round_planes(const float *src, int64_t src_stride, void *dst, int64_t dst_stride,
                            int32_t n_planes, int64_t n, int32_t dtype, lgs_stream stream);

/* ------------------------------------------------------------------------
 * Densification (Sec. 3.3; the step after a8 that consumes its metric).
 *
 * lgs_moments_accumulate adds one view's moments to per-Gaussian sums over
 * the views of an interval (S, M float, C uint32, indexed by row; the
 * caller zeroes them at the start of the interval):
 *   S[map[j]] += grad_acc[j].S, M[map[j]] += grad_acc[j].M, C[...] += .C.
 * lgs_moments_metric: metric[i] = S - M^2 / C (0 if C = 0), i < n.
 *
 * lgs_densify: candidates are Gaussians with metric > 0; the max_new with
 * the largest metric are selected (ties: lower index first). A selected
 * Gaussian whose largest scale exp(log-scale) exceeds split_scale is split
 * (the readings of the 3DGS mechanics the paper inherits): two samples
 * p + R(q) (s * z), z from `normals` (device, [max_new][2][3] standard
 * normal values, drawn by the caller), both with log-scales - ln 1.6; the
 * first replaces the original row, the second is appended. Otherwise an
 * exact copy is appended. Appended and split rows get zero m and v.
 * g->data, m and v must have room for g->n + max_new rows (stride). The
 * new count n + added is written to *d_n_out (device); selected_out
 * (device, optional, [max_new]) receives the selected rows in order.
 * Workspace: lgs_densify_workspace_size(g->n).
 *
 * lgs_opacity_decay halves every activated opacity in place:
 * sigmoid(logit') = sigmoid(logit) / 2, rows < g->n.
 * ---------------------------------------------------------------------- */
lgs_status lgs_moments_accumulate(const float *grad_acc, const uint32_t *map,
                                  const int32_t *d_num_visible, int64_t max_rows, float *S,
                                  float *M, uint32_t *C, lgs_stream stream);
lgs_status lgs_moments_metric(const float *S, const float *M, const uint32_t *C, int64_t n,
                              float *metric, lgs_stream stream);
size_t lgs_densify_workspace_size(int64_t n);
lgs_status lgs_densify(const lgs_gaussians *g, float *m, float *v, const float *metric,
                       int64_t max_new, float split_scale, const float *normals,
                       int64_t *d_n_out, uint32_t *selected_out, void *workspace,
                       size_t workspace_bytes, lgs_stream stream);
lgs_status lgs_opacity_decay(const lgs_gaussians *g, lgs_stream stream);

/* ----------------------------------------------------------------------
 * Unit-rate microbenchmarks (measurement helpers, not part of the training
 * path): the denominators of the raster kernels' rooflines, measured on the
 * device they run on. The caller times each call (CUDA events on `stream`)
 * and divides the operation count below by the time. Each kernel runs
 * `blocks` CTAs of 256 threads (1 <= blocks <= 2^20; a multiple of the SM
 * count times 8 fills every SM); iters >= 1; every loop has a fixed trip
 * count, so a call cannot hang.
 *
 * lgs_peak_ex2: each thread a dependent chain of 32 * iters base-2
 * exponentials on the special-function unit (ex2.approx, as in the raster),
 * x <- 2^x - 1.5: blocks * 256 * 32 * iters exponentials. out: device,
 * blocks * 256 floats (the chains' ends, so that the work is kept).
 *
 * lgs_peak_ffma: each thread a dependent chain of 32 * iters fused
 * multiply-adds, scalar FP32 (packed = 0: blocks * 256 * 32 * iters FMAs)
 * or the packed two-lane FP32 form on a float2 (packed = 1: twice as many
 * FMAs in as many instructions). out as above.
 *
 * lgs_peak_red: each warp, iters times, draws a row in [0, n_rows) by a
 * hash and its lanes 0..11 add 1.0f to floats 0..11 of that 16-float row
 * with float reductions into global memory (the backward's pattern:
 * 12 values of one 64-byte gradient row per warp instruction):
 * blocks * 8 * 12 * iters reductions. rows: device, 16-byte aligned,
 * n_rows * 16 floats (1 <= n_rows < 2^31), contents incremented.
 * Errors: LGS_ERR_INVALID_ARG for a null buffer or an argument out of range
 * (nothing enqueued), LGS_ERR_CUDA if the launch fails.
 * ---------------------------------------------------------------------- */
lgs_status lgs_peak_ex2(float *out, int32_t blocks, int32_t iters, lgs_stream stream);
lgs_status lgs_peak_ffma(float *out, int32_t blocks, int32_t iters, int32_t packed,
                         lgs_stream stream);
lgs_status lgs_peak_red(float *rows, int64_t n_rows, int32_t blocks, int32_t iters,
                        lgs_stream stream);

#ifdef __cplusplus
}
#endif
#endif /* LGS_H */
