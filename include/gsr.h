/*
 * gsr.h -- C ABI of the GB300 differentiable Gaussian-splat rasterizer.
 *
 * The library renders depth-sorted 3D Gaussian splats and back-propagates
 * per-pixel image gradients to per-splat parameter gradients, following
 * "Efficient Differentiable Hardware Rasterization for 3D Gaussian Splatting"
 * (arXiv 2505.18764).  Pipeline per view:
 *
 *   gs_project          per-splat EWA projection, SH colour, culling, depth key
 *                       (Sec. 2.1.1 Eq. 1, Sec. 2.1.2)
 *   gs_sort             global stable depth sort (Onesweep radix sort, Sec. 4.1)
 *   gs_raster_forward   quad-coverage binning + front-to-back alpha blending
 *                       with the 1/255 floor and T-culling (Eq. 2, Sec. 2.1.4)
 *   gs_raster_backward  front-to-back gradient recurrence (Eq. 5-7, Procedure 1),
 *                       per-splat reduction (Sec. 3.2, Procedure 2) and the chain
 *                       rule back to the 3D parameters
 *   gs_render_batch     a list of forward / forward+backward requests
 *                       (gs_render_batch_graph: the same as one CUDA graph)
 *   gs_zero_touched_gradients  zeroes the gradient rows the last view's backward
 *                       added to (a training step's reset, proportional to V)
 *
 * Conventions
 *   - Every array pointer is CUDA device memory owned by the caller, row-major,
 *     float32 unless stated.  Host pointers are marked "host".
 *   - Calls are asynchronous on `stream` (a cudaStream_t) and never allocate
 *     device memory: scratch lives in a caller-allocated workspace
 *     (gs_workspace_size / gs_workspace_init).  One workspace serves one stream
 *     at a time.  gs_render_batch_graph keeps one executable CUDA graph per
 *     workspace, and gs_render_batch a second stream and two events per
 *     workspace (gs_graph_release frees them).
 *   - Parameters are activated values: scales > 0, opacities in [0, 1],
 *     quaternions (w, x, y, z) normalised inside, SH coefficients [N][K][3]
 *     with K = (sh_degree + 1)^2, real orthonormal basis with the
 *     Condon-Shortley phase, index l*l + l + m.
 *   - Return value: GS_OK or a negative GS_ERR_*; gs_last_error() gives a
 *     message (per calling thread).  Conditions found on the device (pair
 *     capacity exceeded, a bounded wait that gave up) are recorded in the
 *     workspace's status word and reported by gs_check_status.
 */
#ifndef GSR_H_
#define GSR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; 0 is the legacy default stream. */
typedef struct CUstream_st* gs_stream_t;

enum {
  GS_OK = 0,
  GS_ERR_INVALID_ARG = -1, /* bad pointer, size, or a size beyond the workspace's capacity */
  GS_ERR_CAPACITY = -2,    /* more (splat, block) pairs than the workspace holds */
  GS_ERR_TIMEOUT = -3,     /* a device-side bounded wait (sort / scan look-back) gave up */
  GS_ERR_CUDA = -4         /* a CUDA runtime call failed */
};

/* Saved per-pixel state format (Sec. 3.3): colour C (3) and transmittance T. */
enum {
  GS_STATE_FP32 = 0,    /* float4  (r, g, b, T), 16 B / pixel */
  GS_STATE_FP16 = 1,    /* half4   (r, g, b, T),  8 B / pixel */
  GS_STATE_UNORM16 = 2, /* ushort4 (r, g, b, T),  8 B / pixel, colours saturated to [0, 1] */
  GS_STATE_UNORM8 = 3   /* uchar4  (r, g, b, T),  4 B / pixel, colours saturated to [0, 1] */
};

/* Per-splat gradient reduction in the backward raster (Sec. 3.2).  The raster
 * kernels give each warp a footprint of 64 pixels (8x8, two per lane) or, in
 * blocks with long splat lists, 32 (8x4) or 16 (4x4). */
enum {
  GS_REDUCE_WARP = 0,    /* summed over the warp first (in batches through shared memory): one
                            set of vector atomics per (splat, footprint) */
  GS_REDUCE_NAIVE = 1,   /* one vector-atomic triple per lane that has a fragment (a lane's two
                            pixels of an 8x8 footprint are added first) */
  GS_REDUCE_FRAGMENT = 2 /* one vector-atomic triple per fragment, every pixel its own (the
                            paper's 1x baseline of Sec. 4.3); front to back only */
};

/* Order in which the backward raster visits a pixel's fragments (Sec. 3.1.2).
 * Front to back (the paper's choice, Eq. 5-7) carries T forward from 1 and C'
 * from the stored colour.  Back to front starts at the pixel's last fragment
 * and recovers T_i = T_{i+1} / (1 - alpha_i) from the stored final
 * transmittance, accumulating the colour behind each fragment (Eq. 4): exact in
 * FP32 state, but a reduced-precision final T (unorm8 above all) corrupts every
 * recovered T, which is why the paper traverses front to back. */
enum { GS_BWD_FRONT_TO_BACK = 0, GS_BWD_BACK_TO_FRONT = 1 };

enum { GS_MODE_FORWARD = 0, GS_MODE_FORWARD_BACKWARD = 1 };
enum { GS_LOSS_NONE = 0, GS_LOSS_L1 = 1, GS_LOSS_L2 = 2 };

/* Pinhole camera.  viewmat: row-major 3x4 world->camera [R | t], OpenCV axes
 * (x right, y down, z forward).  Pixel (x, y) has its centre at (x+0.5, y+0.5);
 * mu_2D = (fx tx/tz + cx, fy ty/tz + cy).  Splats with tz <= znear are culled. */
typedef struct gs_camera {
  float viewmat[12];
  float campos[3];
  float fx, fy, cx, cy;
  int32_t width, height;
  float znear;
} gs_camera;

#define GS_SPLIT_THRESHOLD_DEFAULT 1536
#define GS_REDUCE_THRESHOLD_DEFAULT 16

typedef struct gs_raster_opts {
  int32_t state_format;     /* GS_STATE_* */
  int32_t reduce_mode;      /* GS_REDUCE_* */
  int32_t reduce_threshold; /* X of Sec. 3.2.4: a splat met by fewer than X lanes of a warp is
                               added by those lanes directly; 0 = default
                               (GS_REDUCE_THRESHOLD_DEFAULT), 1 = always reduce first */
  int32_t sh_degree;        /* 0..3 */
  float t_cull;             /* skip fragment i iff T_i < t_cull (Procedure 1); 0 disables */
  int32_t split_threshold;  /* a block whose splat list has at least this many entries is walked
                               by eight warps (8x4 pixels, one per lane) instead of four (8x8,
                               two per lane), from 8x this many by sixteen half-warps (4x4);
                               0 = default (GS_SPLIT_THRESHOLD_DEFAULT).  Results do not depend
                               on it. */
  int32_t backward_order;   /* GS_BWD_* */
  int32_t chunked;          /* memory-efficiency mode (1): the view is binned and rasterized in
                               chunks of the depth order whose pairs fit the pair capacity (at
                               least twice the block count), each pixel carrying its state from
                               one chunk to the next; only through gs_raster_forward and
                               gs_raster_backward, front to back.  Fixed at gs_workspace_init. */
  int64_t pair_capacity;    /* (splat, 16x16 block) pairs the workspace holds; 0 = 16 per splat */
} gs_raster_opts;

/* Host-side descriptor of a caller-allocated device workspace.  Filled by
 * gs_workspace_init; gs_project binds it to a scene size and camera. */
typedef struct gs_workspace {
  void* base;      /* device memory, >= gs_workspace_size bytes, 256-B aligned */
  size_t bytes;
  int32_t n_cap, width_cap, height_cap, chunked;   /* chunked: opts->chunked at init */
  int64_t pair_cap;
  /* bound by gs_project (read by the later calls) */
  int32_t n, width, height, sh_degree;
  int32_t state_format, clamp01, pair_passes, n_chunks;   /* n_chunks: of the last forward */
  uint64_t layout[24]; /* byte offsets of the internal arrays */
} gs_workspace;

/* Scene and request for gs_render_batch. */
typedef struct gs_scene_ref {
  const float* means;     /* [n][3] */
  const float* scales;    /* [n][3] */
  const float* quats;     /* [n][4] */
  const float* opacities; /* [n]    */
  const float* sh;        /* [n][K][3] */
  int32_t n;
  int32_t sh_degree;
} gs_scene_ref;

typedef struct gs_request {
  gs_scene_ref scene;
  gs_camera camera;
  gs_raster_opts opts;
  int32_t mode;          /* GS_MODE_* */
  int32_t loss_kind;     /* GS_LOSS_*: with NONE, dL_dimage is an input */
  float* image;          /* [H][W][3] out, may be null */
  void* state;           /* [H][W] pixels of the state format, out */
  uint32_t* last;        /* [H][W] depth rank of the last fragment, 0xFFFFFFFF if none */
  uint32_t* n_contrib;   /* [H][W] fragment count, may be null */
  const float* target;   /* [H][W][3], used with L1 / L2 */
  float* dL_dimage;      /* [H][W][3]: written by L1 / L2, read otherwise */
  double* loss;          /* one double, written by L1 / L2 (summed over pixels and channels) */
  float* d_means;        /* gradients, accumulated (+=) */
  float* d_scales;
  float* d_quats;
  float* d_opacities;
  float* d_sh;
  int32_t zero_touched;  /* forward+backward, for training loops that reset the gradients between
                            views: 0 = gradients are added to d_* (the default); 1 = first zero
                            the rows the workspace's last depth order touched
                            (gs_zero_touched_gradients), then add; 2 = d_* end up holding this
                            view's gradient alone: the rows the last store-mode request on this
                            workspace wrote are zeroed (the workspace keeps their ids), then the
                            rows of this view's splats with a gradient are written.  If a
                            backward that adds ran in between, every row the last depth order
                            held and every visible splat's row is zeroed or written instead.
                            2 needs d_* to hold zeros or the previous request's gradients of the
                            same scene on this workspace, and saves the reset pass and the read
                            of the rows */
  int32_t pad0;
  double* loss_host;     /* may be null: the loss is also copied to this pinned host double at
                            the end of the request (inside the batch's CUDA graph) */
} gs_request;

/* Bytes of device workspace for scenes of up to n_cap splats and images of up
 * to width_cap x height_cap pixels.  opts->pair_capacity sets the (splat,
 * block) pair capacity.  Host pointers in, host size out. */
int gs_workspace_size(int32_t n_cap, int32_t width_cap, int32_t height_cap,
                      const gs_raster_opts* opts, size_t* bytes);

/* Lays the workspace out in `device_base` (caller-owned, >= bytes) and clears
 * its header and look-back words asynchronously on `stream`; use the workspace
 * on that stream (or after it).  `ws` is a host struct the caller owns;
 * nothing is allocated. */
int gs_workspace_init(gs_workspace* ws, void* device_base, size_t bytes, int32_t n_cap,
                      int32_t width_cap, int32_t height_cap, const gs_raster_opts* opts,
                      gs_stream_t stream);

/* Per-splat projection (Sec. 2.1.2): t = W mu + w, cull if tz <= znear,
 * Sigma_2D = J W R S S^T R^T W^T J^T + 0.3 I, conic = Sigma_2D^-1,
 * colour = max(0, sum_k sh_k Y_k(normalize(mu - campos)) + 0.5) (and <= 1 for
 * the unorm formats, Sec. 3.3), opacity floor o >= 1/255, and the screen-space
 * bounding box of the alpha >= 1/255 ellipse (the quad of Sec. 1).  Writes
 * the projected records, depth keys and the visible count into `ws`. */
int gs_project(gs_workspace* ws, const float* means, const float* scales, const float* quats,
               const float* opacities, const float* sh, int32_t n, const gs_camera* cam,
               const gs_raster_opts* opts, gs_stream_t stream);

/* Stable ascending sort of the visible splats by camera depth (FP32 bits of
 * tz), ties by splat index; the count is read on the device (Sec. 4.1). */
int gs_sort(gs_workspace* ws, gs_stream_t stream);

/* Bins every visible splat into the 16x16 pixel blocks its quad covers (in
 * depth order), then blends front to back per pixel (Eq. 2): alpha =
 * min(0.99, o exp(power)), fragments with alpha < 1/255 or T_i < t_cull
 * skipped.  Outputs: image [H][W][3] (may be null), state [H][W] in
 * opts->state_format, last [H][W] (depth rank of the last fragment, or
 * 0xFFFFFFFF), n_contrib [H][W] (may be null). */
int gs_raster_forward(gs_workspace* ws, const gs_camera* cam, const gs_raster_opts* opts,
                      float* image, void* state, uint32_t* last, uint32_t* n_contrib,
                      gs_stream_t stream);

/* The two halves of gs_raster_forward, callable separately (e.g. to time the
 * rasterization apart from binning, as the paper's Table "tab:perf" splits
 * "rasterization" from "overall"):
 *   gs_bin           (splat, block) pairs of every visible splat's quad, sorted
 *                    by block with depth order kept inside each block, and the
 *                    per-block ranges (the quad rasterization step, Sec. 1);
 *   gs_blend_forward front-to-back blending of each block's list (Eq. 2).
 * Same arguments and outputs as gs_raster_forward. */
int gs_bin(gs_workspace* ws, const gs_camera* cam, const gs_raster_opts* opts, gs_stream_t stream);
int gs_blend_forward(gs_workspace* ws, const gs_camera* cam, const gs_raster_opts* opts,
                     float* image, void* state, uint32_t* last, uint32_t* n_contrib,
                     gs_stream_t stream);

/* Backward pass.  Re-traverses the forward's lists front to back with
 * (C'_1, T_1) = (stored C, 1) and the recurrences of Eq. 5 and Eq. 6, takes
 * dL/dc_i and dL/dalpha_i from Eq. 3 and Eq. 7 (Procedure 1), reduces them per
 * splat (opts->reduce_mode, Sec. 3.2) and applies the chain rule to the 3D
 * parameters.  Gradients are ADDED to d_* (callers zero them), so several views
 * can accumulate.  Must follow gs_raster_forward on the same workspace, scene,
 * camera and opts.  dL_dimage [H][W][3]. */
int gs_raster_backward(gs_workspace* ws, const float* means, const float* scales,
                       const float* quats, const float* opacities, const float* sh, int32_t n,
                       const gs_camera* cam, const gs_raster_opts* opts, const void* state,
                       const uint32_t* last, const float* dL_dimage, float* d_means,
                       float* d_scales, float* d_quats, float* d_opacities, float* d_sh,
                       gs_stream_t stream);

/* The two halves of gs_raster_backward:
 *   gs_blend_backward   per-pixel gradients of Procedure 1 (Eq. 3, 5-7) reduced
 *                       per splat (Sec. 3.2) into the workspace's per-splat
 *                       2D accumulators (mu_2D, conic, colour, opacity);
 *   gs_project_backward chain rule from those to the 3D parameters (added to
 *                       d_*).  Same arguments as gs_raster_backward. */
int gs_blend_backward(gs_workspace* ws, const gs_camera* cam, const gs_raster_opts* opts,
                      const void* state, const uint32_t* last, const float* dL_dimage,
                      gs_stream_t stream);
int gs_project_backward(gs_workspace* ws, const float* means, const float* scales,
                        const float* quats, const float* opacities, const float* sh, int32_t n,
                        const gs_camera* cam, const gs_raster_opts* opts, float* d_means,
                        float* d_scales, float* d_quats, float* d_opacities, float* d_sh,
                        gs_stream_t stream);

/* Zeroes the gradient rows (d_means, d_scales, d_quats, d_opacities, d_sh, the
 * layouts of gs_raster_backward) of the splats the last gs_sort on ws ordered,
 * i.e. the visible splats of the last projection: the only rows a backward on
 * that view adds to.  Buffers that were all zero before that backward are all
 * zero again afterwards, at a cost proportional to the visible splats instead
 * of all n (a training step over one view zeroes ~20% of the rows).  The count
 * is read on the device.  Call it before the next gs_sort on ws (which
 * replaces the order); rows of other splats are left as they are.  n must be
 * the n of the last gs_project.  Sizes follow gs_project's sh_degree. */
int gs_zero_touched_gradients(gs_workspace* ws, int32_t n, float* d_means, float* d_scales,
                              float* d_quats, float* d_opacities, float* d_sh,
                              gs_stream_t stream);

/* Depth slabs (Sec. 2.1.2: front-to-back blending is associative over
 * contiguous runs of the depth order).  After gs_project and gs_sort, slab k of
 * n_slabs is the run of depth ranks [k V / n_slabs, (k + 1) V / n_slabs) of
 * the V visible splats (V is read on the device).  gs_raster_forward_slab bins
 * and blends that run alone, each pixel starting from T = 1, and writes its
 * colour C_k (image, may be null), state (C_k, T_k) in opts->state_format,
 * last rank (a global depth rank) and fragment count (may be null).  T-culling
 * (opts->t_cull) uses the slab's own transmittance, so slabs composite to the
 * single-pass image exactly when t_cull = 0.  The whole view's pairs may
 * exceed the workspace's pair capacity as long as one slab's fit (else the
 * device status reads GS_ERR_CAPACITY).  Not with the memory-efficiency mode.
 * Slabs can be rendered on different GPUs, each with a replica of the scene:
 * the exchange is one gather of the states, then gs_slab_composite. */
int gs_raster_forward_slab(gs_workspace* ws, const gs_camera* cam, const gs_raster_opts* opts,
                           int32_t slab, int32_t n_slabs, float* image, void* state,
                           uint32_t* last, uint32_t* n_contrib, gs_stream_t stream);

/* "Over" composite of n_slabs slab states laid out one after another,
 * states[k][npix] in state_format (16, 8, 8 or 4 bytes per pixel, the format's
 * layout): image [npix][3] = C_0 + T_0 (C_1 + T_1 (C_2 + ...)), trans [npix] =
 * T_0 T_1 ..., and for the backward of each slab t_front [n_slabs][npix] =
 * T_0 ... T_{k-1} and behind [n_slabs][npix][3] = the composite of the slabs
 * after k (0 for the last).  Any output may be null.  Device pointers. */
int gs_slab_composite(const void* states, int32_t state_format, int32_t n_slabs, int64_t npix,
                      float* image, float* trans, float* t_front, float* behind,
                      gs_stream_t stream);

/* Backward of slab k (after gs_raster_forward_slab of that slab on ws, same
 * scene, camera and opts): Procedure 1 over the slab's fragments with the
 * image gradient dL_dimage [H][W][3] scaled by t_front (slab k's [H][W] of
 * gs_slab_composite; null = 1) and C' starting from the slab's colour plus T_k
 * times behind (slab k's [H][W][3]; null = 0), then the chain rule; gradients
 * are ADDED to d_*, so the slabs' calls sum to the single-pass gradient (at
 * t_cull = 0).  Arguments otherwise as gs_raster_backward. */
int gs_raster_backward_slab(gs_workspace* ws, const float* means, const float* scales,
                            const float* quats, const float* opacities, const float* sh,
                            int32_t n, const gs_camera* cam, const gs_raster_opts* opts,
                            int32_t slab, int32_t n_slabs, const void* state, const uint32_t* last,
                            const float* t_front, const float* behind, const float* dL_dimage,
                            float* d_means, float* d_scales, float* d_quats, float* d_opacities,
                            float* d_sh, gs_stream_t stream);

/* Summed image loss over n_values floats: L1 = sum |image - target| (dL/dimage =
 * sign) or L2 = sum (image - target)^2 (dL/dimage = 2 (image - target)).
 * Writes dL_dimage (may be null) and *loss (one device double). */
int gs_loss(const float* image, const float* target, int64_t n_values, int32_t kind,
            float* dL_dimage, double* loss, gs_stream_t stream);

/* Runs the requests in order on one stream with one workspace (sized for the
 * largest).  Forward: project, sort, raster.  Forward+backward adds the loss
 * (if any) and the backward pass. */
int gs_render_batch(const gs_request* reqs, int32_t n, gs_workspace* ws, gs_stream_t stream);

/* gs_render_batch through a CUDA graph: the requests' ~20 launches per request
 * are captured from `stream` into a graph and launched as one, without the
 * gaps between dependent launches.  The executable graph is kept per workspace
 * and updated in place when the next call has the same launch structure (new
 * pointers, camera or counts are fine); otherwise it is rebuilt.  Same results
 * and errors as gs_render_batch.  A request in the memory-efficiency mode
 * (which reads its chunk count on the host), a legacy default stream (NULL,
 * which cannot be captured) or a stream already being captured makes the call
 * run as gs_render_batch.  Not thread-safe for one workspace (neither is any
 * call on a workspace). */
int gs_render_batch_graph(const gs_request* reqs, int32_t n, gs_workspace* ws,
                          gs_stream_t stream);

/* Frees the executable graph gs_render_batch_graph keeps for ws (if any), and
 * the second stream and two events gs_render_batch creates for ws on first use
 * (it runs the backward's item ordering on that stream beside the loss).  Call
 * before freeing a workspace's memory that will not be used again. */
int gs_graph_release(gs_workspace* ws);

/* Sorting memory of a workspace (the paper's memory table, Sec. 4.5, counts
 * it apart): *depth_sort = the depth keys, the key/value ping-pong buffers and
 * the radix passes' look-back words; *pair_sort = the (block, rank) pair
 * buffers sized by the pair capacity.  Host outputs. */
int gs_workspace_sort_bytes(const gs_workspace* ws, size_t* depth_sort, size_t* pair_sort);

/* Synchronises `stream` and returns the device status recorded in `ws`
 * (GS_OK, GS_ERR_CAPACITY or GS_ERR_TIMEOUT). */
int gs_check_status(gs_workspace* ws, gs_stream_t stream);

/* Message of the calling thread's last error ("" if none).  Host string. */
const char* gs_last_error(void);

/* Introspection for tests and metrics.  gs_read_counters synchronises `stream`
 * and writes (host) out[0] = visible splats V, out[1] = (splat, block) pairs P
 * of the splats' block boxes, out[2] = device status, out[3] = 16x16 blocks of
 * the bound camera, out[4] = pairs the view needs (above out[1] when the pair
 * capacity was exceeded), out[5] = live pairs (those whose block the splat's
 * ellipse reaches: the sorted pair arrays hold these).  out holds 6. */
int gs_read_counters(gs_workspace* ws, int64_t* out, gs_stream_t stream);

/* Measurement helper, not part of the paper's method: the FP32 FMA rate of the
 * current GPU in TFLOP/s (the ceiling of the FP32-bound raster kernels), from
 * one launch of `iters` rounds of independent FMAs on every resident thread,
 * timed with CUDA events on `stream`.  Synchronises `stream`; writes *tflops
 * (host). */
int gs_fp32_fma_rate(int32_t iters, double* tflops, gs_stream_t stream);

/* Copies an internal array of `ws` into caller device memory `dst` (`bytes`):
 * GS_ARRAY_SORTED_IDS u32 [V], GS_ARRAY_DEPTH_KEYS u32 [n] (0xFFFFFFFF = culled),
 * GS_ARRAY_RECORDS float [n][12] (mu_x, mu_y, i11, k, i22, tau, mu_x_lo, mu_y_lo,
 * r, g, b, o: the screen centre mu + mu_lo as a float-float pair, the inverse
 * Cholesky factor of Sigma_2D scaled so that (i11 dx)^2 + (i22 (dy - k dx))^2 =
 * -log2(e) * power, and tau = log2(255 o)),
 * GS_ARRAY_PAIR_BLOCKS u32 [live pairs], GS_ARRAY_PAIR_RANKS u32 [live pairs]
 * (sorted by block, depth order within a block),
 * GS_ARRAY_RANGES u32 [blocks][2], GS_ARRAY_GRAD2D float [V][12] (per depth
 * rank: the backward's unscaled accumulators), GS_ARRAY_BOXES u32 [V][2] (per
 * depth rank: first block x | y << 16, box width | height << 16 in blocks). */
enum {
  GS_ARRAY_SORTED_IDS = 0,
  GS_ARRAY_DEPTH_KEYS = 1,
  GS_ARRAY_RECORDS = 2,
  GS_ARRAY_PAIR_BLOCKS = 3,
  GS_ARRAY_PAIR_RANKS = 4,
  GS_ARRAY_RANGES = 5,
  GS_ARRAY_GRAD2D = 6,
  GS_ARRAY_BOXES = 7
};
int gs_copy_array(gs_workspace* ws, int32_t which, void* dst, size_t bytes, gs_stream_t stream);

/* Stable LSD radix sort of n (u32 key, u32 value) pairs on key bits
 * [0, key_bits), using the workspace's depth-sort buffers (n <= ws->n_cap).
 * keys_in/vals_in are read; the result goes to keys_out/vals_out (device,
 * caller-owned, n entries; must not alias the inputs).  keys must be below
 * 2^key_bits rounded up to whole bytes.  Uses the workspace's scratch and header, so it
 * invalidates a view bound by gs_project.  Standalone use of the sort of Sec. 4.1. */
int gs_sort_pairs(gs_workspace* ws, const uint32_t* keys_in, const uint32_t* vals_in,
                  uint32_t* keys_out, uint32_t* vals_out, int32_t n, int32_t key_bits,
                  gs_stream_t stream);

/* Allocation-free pair sort.  The paper has no counterpart: this entry point
 * exists for callers that cannot provide device memory at the point of the
 * call, such as a host application or plugin interface that owns every device
 * allocation and hands the library only its inputs and outputs, or a
 * long-running service that fixes its HBM budget at start-up and forbids
 * allocations afterwards.  It performs the same stable LSD radix sort as
 * gs_sort_pairs (same arguments and results, keys below 2^key_bits rounded up
 * to whole bytes, outputs must not alias inputs) but keeps its scratch in one
 * fixed array inside the library: every GPU that loads the library holds
 * about 4.3 MB for it until the process exits, and n may not exceed
 * GS_SORT_NOALLOC_MAX_PAIRS (larger n returns GS_ERR_INVALID_ARG with a
 * message).  It calls no allocator.  The array is used on the current device:
 * keys_in must be memory of that device (else GS_ERR_INVALID_ARG).  Every call
 * looks the array's address up again; the first call on each device (and the
 * first after cudaDeviceReset moved the array) zeroes it on `stream` before
 * sorting, so make that first call before any stream capture.  All calls on a
 * device share the array, and it keeps the last call's contents: calls that
 * overlap on the GPU (on different streams, or from different threads) race
 * and corrupt each other; order them on one stream or serialise them.  A wait
 * on the device that gave up (GS_ERR_TIMEOUT, a wrong result) is reported by
 * gs_sort_pairs_noalloc_status, not by the call itself. */
#define GS_SORT_NOALLOC_MAX_PAIRS 262144
int gs_sort_pairs_noalloc(const uint32_t* keys_in, const uint32_t* vals_in, uint32_t* keys_out,
                          uint32_t* vals_out, int32_t n, int32_t key_bits, gs_stream_t stream);

/* Device status of the last gs_sort_pairs_noalloc on the current device:
 * synchronises `stream` (the stream of that call) and returns GS_OK, or
 * GS_ERR_TIMEOUT when one of its look-back waits gave up (its output is then
 * wrong).  The next gs_sort_pairs_noalloc on the device clears the status, so
 * read it before that call.  Allocates nothing; GS_OK before any call. */
int gs_sort_pairs_noalloc_status(gs_stream_t stream);

/* Self-test of the bounded device waits (a testing aid, not part of the
 * paper's method).  Runs the first radix pass of gs_sort_pairs (ws != NULL,
 * n <= ws->n_cap) or of gs_sort_pairs_noalloc (ws == NULL, n <=
 * GS_SORT_NOALLOC_MAX_PAIRS) on n > 2048 keys (at least two tiles) with tile 0
 * withheld: no CTA ever publishes tile 0's look-back word, so every wait on it
 * gives up after `spin_limit` polls (1 .. 2^22; ~1e4 polls take a few
 * milliseconds).  The pass then finishes with a wrong result written inside
 * keys_out / vals_out (n entries each) and records GS_ERR_TIMEOUT, which
 * gs_check_status(ws) or gs_sort_pairs_noalloc_status returns; the kernel
 * returns and the CUDA context stays usable. */
int gs_test_stalled_sort(gs_workspace* ws, const uint32_t* keys_in, const uint32_t* vals_in,
                         uint32_t* keys_out, uint32_t* vals_out, int32_t n, uint32_t spin_limit,
                         gs_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* GSR_H_ */
