/*
 * dgs.h -- C ABI of libdgs, a batched 3D Gaussian Splatting RGB + depth renderer for many
 * parallel environments on one GB300 (sm_103a).
 *
 * What is rendered (DISCOVERSE, Sec. III-A "Renderer", Sec. III-B "Asset Formatting",
 * Sec. III-C "Sensor"): each environment holds a background Gaussian node plus interactive
 * nodes (objects, robot links) whose Gaussians move rigidly with the node's pose; the
 * renderer is the native tile-based 3DGS pipeline (EWA splatting, spherical-harmonics colour,
 * depth sorting, front-to-back alpha-blending) and produces RGB and depth by
 * alpha-compositing the colour and the camera-space z of the Gaussians.
 *
 * Conventions (fixed readings; every numeric constant is a field of dgs_options):
 *   - Poses are row-major 3x4 [R|t] FP32 matrices.  node poses are world_from_node, camera
 *     extrinsics cam_from_world.  Cameras are pinhole, OpenCV axes (x right, y down, z
 *     forward); pixel (x, y) samples the point (x + 1/2, y + 1/2); u = fx*tx/tz + cx.
 *   - Quaternions are (w, x, y, z), need not be unit (normalised inside).  Scales are natural
 *     logs of the per-axis standard deviations.  Opacity = sigmoid(logit).
 *   - Colour = max(0, sum_k sh[k] Y_k(d) + 1/2) with the real SH basis (Condon-Shortley
 *     phase, k = l^2 + l + m, degree <= 3) and d the unit direction from the camera centre to
 *     the Gaussian, expressed in the node frame.
 *   - A Gaussian touches a pixel iff d^T conic d <= q_max (default 9, the 3-sigma ellipse);
 *     alpha = min(alpha_max, opacity*exp(-q/2)); alpha < alpha_min is skipped; compositing
 *     stops, without the current Gaussian, once T*(1-alpha) < t_min.
 *     RGB = sum w_i rgb_i + bg*T_final, depth = sum w_i z_i (not normalised), alpha = 1 - T.
 *   - Depth order and near-plane cull use the FP32 key z32 = the camera-space z of the
 *     Gaussian's centre, faithfully rounded: within one unit in the last place of the exact
 *     value for the FP32 inputs (camera_from_node is composed, and applied to the mean, with
 *     compensated sums); the projected centre is computed from the camera-space point rounded
 *     the same way.  Equal keys are ordered by global id = (sum of sizes of the preceding nodes
 *     in the node array) + index in the node.  Keys beyond 2^28 units of 2^(floor(log2
 *     z_near) - 23) above 2^floor(log2 z_near) compare equal.
 *
 * Memory: every array pointer marked DEVICE is a CUDA device pointer owned by the caller
 * and must stay valid until the work queued on `stream` has finished.  Arrays marked HOST are
 * read during the call only.  The library owns only the workspace inside a context.
 * Errors: every call returns a dgs_status; nothing throws across the ABI.  Argument
 * validation failures return synchronously and queue no work.  dgs_last_error() describes
 * the most recent failure of a context.  A context is not thread-safe: one host thread at a
 * time.
 */
#ifndef DGS_H
#define DGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DGS_ABI_VERSION 1

typedef enum dgs_status {
    DGS_OK = 0,
    DGS_ERR_INVALID_ARG = 1, /* bad shape, null pointer, bad enum, non-finite or non-rigid pose */
    DGS_ERR_CUDA = 2,        /* a CUDA runtime call failed; see dgs_last_error */
    DGS_ERR_OOM = 3,         /* workspace allocation failed */
    DGS_ERR_CAPACITY = 4,    /* a batch exceeds a hard limit (2^30 tile pairs per view group) */
    DGS_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up (results are invalid) */
    DGS_ERR_UNSUPPORTED = 6  /* the call is not available for these arguments */
} dgs_status;

typedef enum dgs_dtype { DGS_F32 = 0, DGS_BF16 = 1, DGS_F16 = 2 } dgs_dtype;

typedef enum dgs_mode {
    DGS_MODE_PLAIN = 0,   /* every view runs its own projection/binning/sort/composite sequence */
    DGS_MODE_BATCHED = 1, /* all views of a call share one sequence; attributes read once per group */
    DGS_MODE_GRAPH = 2    /* batched, replayed as one captured CUDA graph (see dgs_render) */
} dgs_mode;

/* One scene node: structure-of-arrays Gaussians in the node's own frame. */
typedef struct dgs_node {
    const float* mean;          /* DEVICE [n,3] FP32 */
    const void* log_scale;      /* DEVICE [n,3] of `dtype` */
    const void* quat;           /* DEVICE [n,4] of `dtype`, (w,x,y,z) */
    const float* opacity_logit; /* DEVICE [n] FP32 */
    const void* sh;             /* DEVICE [n,(sh_degree+1)^2,3] of `dtype`, coefficient-major */
    int64_t n;                  /* number of Gaussians, >= 0 */
    int32_t sh_degree;          /* 0..3 */
    int32_t dtype;              /* dgs_dtype of log_scale, quat and sh */
} dgs_node;

/* Pinhole camera.  width, height >= 1. */
typedef struct dgs_camera {
    float fx, fy, cx, cy;
    int32_t width, height;
    float cam_from_world[12];   /* row-major [R|t] */
} dgs_camera;

typedef struct dgs_options {
    int32_t mode;               /* dgs_mode, default DGS_MODE_BATCHED */
    int32_t tile_w, tile_h;     /* tile shape: w a multiple of 8, h of 4, w*h in {64,128,256}; 16x16 */
    int32_t exact_tile_test;    /* 1 = bin a Gaussian only to tiles its ellipse reaches (default) */
    float z_near;               /* default 0.01; must be > 0 */
    float lowpass;              /* screen-space dilation added to the 2D covariance, default 0.3 px^2 */
    float alpha_min;            /* default 1/255 */
    float alpha_max;            /* default 0.99 */
    float t_min;                /* default 1e-4 */
    float q_max;                /* default 9 */
    float guard;                /* Jacobian clamp: |tx/tz| <= guard * (W/2)/fx, default 1.3 */
    float bg[3];                /* background colour, default 0 */
    int32_t profile;            /* 1 = time each kernel class with CUDA events (dgs_kernel_times);
                                   2 = also count compositor work (dgs_stats), slower */
    int32_t views_per_group;    /* batched mode: max views per group; 0 = automatic: a batch with at
                                   least 2^22 tile pairs (bound) runs as two view groups on two
                                   streams, one group's binning overlapping the other's compositing;
                                   more groups only where the 2^30-pair or the 2^24-tile limit of a
                                   group needs them */
    int32_t spin_limit_us;      /* limit of every bounded device-side wait (the sort's look-back), in
                                   microseconds, 0 = 1 s; a wait that runs out ends the call with
                                   DGS_ERR_TIMEOUT (outputs invalid, the context stays usable) */
    int32_t check_binning;      /* 1 = eager renders read each view group's tile lists back and check
                                   them on the host before compositing: tiles non-decreasing and below
                                   the group's tile count, sub-tile masks within the tile, the ranges
                                   covering every pair once, and each tile's run in depth order (equal
                                   depths by instance number); a violation ends the call with
                                   DGS_ERR_CUDA and a description.  Slow: for tests and debugging */
    int32_t test_fault;         /* fault injection for tests, 0 = none.  1: the first digit pass of the
                                   depth sort leaves the look-back status of its second partition
                                   unpublished, so the waits behind it run out (DGS_ERR_TIMEOUT after
                                   about spin_limit_us per wave of resident blocks); 2: with
                                   check_binning, the host copy of the first view group's tile keys is
                                   corrupted (two adjacent pairs of different tiles exchanged) before
                                   the check, which must then report it; 3 (DGS_DEBUG builds only,
                                   DGS_ERR_INVALID_ARG otherwise): the compositors of an eager render
                                   or backward are told that every view group holds half the records
                                   it does, so the bounds check on tile-list entries fails
                                   (DGS_ERR_CUDA naming the check) while every access it lets
                                   through stays inside the records written; 4: not a fault -- the
                                   depth sort takes each instance's view from a separate array even
                                   where it fits in the instance numbers' high bits (the form of
                                   view groups too large for that), with identical results */
    int32_t keep_lists;         /* 1 = a render of at most two view groups -- eager, or a graph
                                   replay (not the call that captures) -- keeps its tile lists,
                                   records and device tables on the context, and a
                                   dgs_render_backward of the same batch differentiates them instead
                                   of binning again (stats.path = DGS_PATH_KEPT_LISTS).
                                   "The same batch": equal node descriptors, env -> node table, node
                                   pose pointer, cameras, per-env camera counts and pixel offsets, and
                                   no call that stages a batch (dgs_render, dgs_render_backward
                                   without a match, dgs_autotune, dgs_workspace_query_batch) nor
                                   dgs_set_options on the context in between; otherwise the backward
                                   bins again as without the option.  The caller must leave the
                                   device data the render read (attributes and poses) unchanged
                                   until that backward, as with any state saved for a backward.
                                   Default 0 */
} dgs_options;

typedef struct dgs_ctx dgs_ctx;

/* Per-call statistics of the most recent dgs_render (or dgs_render_backward) on a context. */
typedef struct dgs_stats {
    int64_t n_views;
    int64_t n_pixels;
    int64_t n_instances;        /* (Gaussian, view) pairs considered */
    int64_t n_visible;          /* instances emitted: those the count pass's conservative cull keeps (the
                                   few that the exact projection then rejects carry no tile pairs) */
    int64_t n_pairs;            /* (instance, tile) pairs sorted */
    int32_t n_groups;           /* view groups (batched) or views (plain) */
    int32_t key_bits;           /* significant sort-key bits of the largest group */
    /* compositor work, counted only when dgs_options.profile = 2: */
    int64_t px_evaluated;       /* (pixel, Gaussian) evaluations performed (warp lanes x records) */
    int64_t px_reached;         /* pairs inside the 3-sigma ellipse reached before termination */
    int64_t px_composited;      /* pairs composited */
    int32_t path;               /* dgs_path: how the call ran */
    int32_t graph_captures;     /* graphs captured by this context so far */
    int64_t bwd_reductions;     /* dgs_render_backward with profile = 2: global atomic adds of the
                                   compositing adjoint's per-instance partials */
} dgs_stats;

/* dgs_stats.path */
typedef enum dgs_path {
    DGS_PATH_EAGER = 0,         /* launched kernel by kernel (with one mid-call readback) */
    DGS_PATH_GRAPH = 1,         /* replayed the captured graph */
    DGS_PATH_CAPTURED = 2,      /* ran eagerly, then captured a graph for the next calls */
    DGS_PATH_REGROWN = 3,       /* a replay overflowed its capacity: ran eagerly and recaptured */
    DGS_PATH_KEPT_LISTS = 4     /* dgs_render_backward used the lists its forward kept (keep_lists) */
} dgs_path;

/* Kernel classes timed when dgs_options.profile = 1 (milliseconds, summed over the call). */
typedef enum dgs_kernel_class {
    DGS_K_SETUP = 0, DGS_K_COUNT = 1, DGS_K_SCAN = 2, DGS_K_EMIT = 3, DGS_K_SORT = 4,
    DGS_K_RANGES = 5, DGS_K_COMPOSITE = 6,
    DGS_K_BACKWARD = 7,         /* dgs_render_backward's compositing adjoint (per-instance partials) */
    DGS_K_GRAPH = 8,            /* a whole graph replay (DGS_MODE_GRAPH) */
    DGS_K_AUGMENT = 9,          /* dgs_augment_rgb's pass */
    DGS_K_LIDAR = 10,           /* dgs_lidar_trace (setup + trace) */
    DGS_K_MESH = 11,            /* dgs_mesh_to_gaussians */
    DGS_K_TSDF = 12,            /* dgs_tsdf_integrate */
    DGS_K_BACKWARD_PROJECT = 13, /* dgs_render_backward's projection, colour and pose adjoint */
    DGS_K_COUNT_CLASSES = 14
} dgs_kernel_class;

/* Fills *opt with the defaults listed above. */
void dgs_default_options(dgs_options* opt);

/* Creates a context on the current CUDA device.  Allocates no device memory yet.
 * Returns DGS_ERR_INVALID_ARG for a null `out` or invalid options. */
int dgs_context_create(dgs_ctx** out, const dgs_options* opt);

/* Replaces the options of a context (validated as for dgs_context_create; DGS_ERR_INVALID_ARG
 * keeps the old ones).  A captured graph (DGS_MODE_GRAPH) is dropped: the next render captures
 * anew.  The workspace is kept. */
int dgs_set_options(dgs_ctx* ctx, const dgs_options* opt);

/* Frees the context and its workspace (synchronises the device first).  Null is a no-op. */
int dgs_context_destroy(dgs_ctx* ctx);

/* Message of the most recent failure on `ctx` ("" if none); valid until the next call. */
const char* dgs_last_error(const dgs_ctx* ctx);

/* Bytes of device workspace currently held by the context (every buffer of every call made on it,
 * with the 25 % growth slack its allocations keep).  For the need of a given batch see
 * dgs_workspace_query_batch. */
int dgs_workspace_query(const dgs_ctx* ctx, size_t* bytes);

/*
 * Device workspace a dgs_render of this batch needs (Sec. III-A: the per-view projection records,
 * sort keys and tile lists scale with the visible instances and their tile pairs, which depend
 * on the poses and cameras, so they cannot be sized from the shapes alone).  Validates the batch
 * like dgs_render (arguments as there; no outputs needed), runs its setup, count and scan
 * kernels on `stream` (allocating the tables they need in the context, as a render would),
 * reads the totals back and writes to *bytes the sum of the count tables and of the tile lists of
 * its view groups (two list sets when the batch runs as two or more groups), without allocating
 * the lists.  The adjoint needs 40 bytes per visible instance of its largest view group on top.
 * Synchronises `stream`.
 */
int dgs_workspace_query_batch(dgs_ctx* ctx, const dgs_node* nodes, int32_t n_nodes, const int32_t* env_node_ids,
                              int32_t n_envs, int32_t max_nodes, const float* node_poses, const dgs_camera* cams,
                              const int32_t* cams_per_env, int32_t max_cams, const int64_t* view_pixel_offset,
                              size_t* bytes, void* stream);

/*
 * Renders every view of a batch of environments (Sec. III-A: tile-based splatting of RGB;
 * Sec. III-C: depth composited the same way; Sec. III-B: nodes at per-env rigid poses).
 *
 *   nodes[n_nodes]                HOST array of node descriptors (attribute arrays DEVICE).
 *   env_node_ids[n_envs*max_nodes] HOST, node drawn in slot j of env e, -1 = empty; a node id
 *                                 appears at most once per env.
 *   node_poses[n_envs*max_nodes*12] DEVICE, world_from_node of slot j of env e (FP32).
 *   cams[n_envs*max_cams]         HOST, camera c of env e (only c < cams_per_env[e] are read).
 *   cams_per_env[n_envs]          HOST, 0..max_cams.
 *   View v enumerates (e, c) env-major.  Outputs are flat over views: view v occupies pixels
 *   [off_v, off_v + W_v*H_v) in row-major order, off_v = view_pixel_offset[v] (HOST [V]) or,
 *   if view_pixel_offset is NULL, the sum of the sizes of the preceding views.
 *   out_rgb   DEVICE FP32 [total_pixels,3] (interleaved RGB), required.
 *   out_depth DEVICE FP32 [total_pixels], required.
 *   out_alpha DEVICE FP32 [total_pixels] or NULL.
 *   stream    a cudaStream_t (NULL = legacy default stream).
 *
 * Work is queued on `stream`.  The call reads per-view counts back once (one stream
 * synchronisation) to size the workspace, and synchronises again before returning so that
 * device-side error flags (invalid pose, timeout, capacity) are reported in the return code.
 *
 * DGS_MODE_GRAPH: the first call renders as above and then captures the whole sequence
 * (setup ... composite) as a CUDA graph sized for 1.25x the instance and tile-pair totals it
 * saw; its kernels read the live totals on the device, so a replay needs no readback until
 * the final synchronisation.  Later calls whose batch has the same structure -- the same
 * views, resolutions, node sizes, storage types and env node tables, the same node_poses and
 * output pointers, and a workspace that has not moved -- upload the host tables (camera
 * poses, intrinsics and node attribute pointers may change) and replay the graph.  Node poses
 * are read from node_poses at replay time.  If a replay finds more instances or pairs than its
 * capacity, its kernels skip their work, the call renders again eagerly (correct outputs) and
 * recaptures with larger capacities; dgs_stats.path says which happened.  The graph keeps the
 * one or two view groups of the render it was captured from (two groups run on two streams,
 * see views_per_group); a batch that needs more groups is not captured and runs eagerly.
 */
int dgs_render(dgs_ctx* ctx, const dgs_node* nodes, int32_t n_nodes,
               const int32_t* env_node_ids, int32_t n_envs, int32_t max_nodes,
               const float* node_poses,
               const dgs_camera* cams, const int32_t* cams_per_env, int32_t max_cams,
               float* out_rgb, float* out_depth, float* out_alpha,
               const int64_t* view_pixel_offset, void* stream);

/* Gradient buffers of one node (all DEVICE FP32, laid out like the node's attributes).  The
 * backward pass ADDS into them; a null pointer skips that attribute. */
typedef struct dgs_node_grads {
    float* mean;                /* [n,3] */
    float* log_scale;           /* [n,3] */
    float* quat;                /* [n,4] */
    float* opacity_logit;       /* [n]   */
    float* sh;                  /* [n,(sh_degree+1)^2,3] */
} dgs_node_grads;

/*
 * Adjoint of dgs_render (Sec. IV: the 3DGS assets are fitted by gradient descent on rendered
 * images and depth).  For L = sum grad_rgb . RGB + sum grad_depth . D, adds dL/d(attribute)
 * to the node gradient buffers and dL/d(world_from_node) (3x4, row-major) to grad_poses.
 *
 *   The scene arguments (nodes ... view_pixel_offset) must be those of the forward call.
 *   out_rgb, out_depth   DEVICE, the forward's outputs (used instead of stored per-pixel state).
 *   grad_rgb             DEVICE [total_pixels,3]; grad_depth DEVICE [total_pixels] or NULL.
 *   grads                HOST [n_nodes] of buffers (entries' pointers may be NULL), or NULL.
 *   grad_poses           DEVICE [n_envs*max_nodes*12] or NULL.
 *
 * The per-tile sorted lists are recomputed (same kernels and decisions as the forward), every
 * pixel is replayed front to back, and per-instance partials are chained through projection,
 * colour and pose.  Decisions are taken exactly as in the forward pass; gradients of clamped
 * quantities (alpha at alpha_max, colour at 0, the Jacobian guard) are zero.  Accumulation
 * uses FP32 atomics, so results may differ in the last bits between calls.
 */
int dgs_render_backward(dgs_ctx* ctx, const dgs_node* nodes, int32_t n_nodes,
                        const int32_t* env_node_ids, int32_t n_envs, int32_t max_nodes,
                        const float* node_poses,
                        const dgs_camera* cams, const int32_t* cams_per_env, int32_t max_cams,
                        const float* out_rgb, const float* out_depth,
                        const float* grad_rgb, const float* grad_depth,
                        const dgs_node_grads* grads, float* grad_poses,
                        const int64_t* view_pixel_offset, void* stream);

/*
 * se(3) gradient of node poses (Sec. III-B: interactive nodes move rigidly with poses from
 * physics; Sec. IV: the scene's parameters are fitted by gradient descent).  For each pose
 * T = [R | t] (world_from_node, row-major 3x4) and its gradient G = dL/dT (3x4, as written to
 * dgs_render_backward's grad_poses), writes the gradient of L with respect to the twist
 * xi = (rho, phi) of a left perturbation T' = exp(xi^) T at xi = 0:
 *   dL/drho = G_t,   dL/dphi = (A_21 - A_12, A_02 - A_20, A_10 - A_01),  A = G_R R^T + G_t t^T.
 *
 *   poses       DEVICE FP32 [n,12]
 *   grad_poses  DEVICE FP32 [n,12]
 *   out_twist   DEVICE FP32 [n,6] (rho then phi), overwritten
 * Queued on `stream` without synchronising; needs no context.  Returns DGS_ERR_INVALID_ARG for
 * n < 0 or a null pointer with n > 0, DGS_ERR_CUDA if the launch fails.
 */
int dgs_pose_twist_grad(const float* poses, const float* grad_poses, int64_t n, float* out_twist, void* stream);

/* Statistics of the most recent successful dgs_render on ctx. */
int dgs_last_stats(const dgs_ctx* ctx, dgs_stats* out);

/* Per-kernel-class device time (ms) of the most recent call with profile = 1 (dgs_render,
 * dgs_render_backward, dgs_augment_rgb, dgs_lidar_trace, dgs_mesh_to_gaussians or
 * dgs_tsdf_integrate);
 * ms[DGS_K_COUNT_CLASSES]. */
int dgs_kernel_times(const dgs_ctx* ctx, float* ms);

/* Launches of library kernels queued by the most recent call (a graph replay counts the
 * kernel nodes it runs). */
int64_t dgs_last_launches(const dgs_ctx* ctx);

/*
 * How this library was built: DGS_BUILD_DEBUG is set in a debug build (compiled with
 * -DDGS_DEBUG: libdgs_debug.so next to libdgs.so).  Its kernels check every index they take
 * from another kernel's output before using it -- record numbers from the scans, depth-sorted
 * instance numbers, sort scatter destinations, tile-list entries, Gaussian ids of the adjoint --
 * and a failed check skips the access and ends the call with DGS_ERR_CUDA and a description
 * (dgs_last_error) of the check, its index and its bound.  Results are otherwise bit-identical
 * to the release build's.  Needs no GPU.
 */
#define DGS_BUILD_DEBUG 1
int32_t dgs_build_flags(void);

/*
 * Storage order for a node (asset formatting, Sec. III-B: assets are converted once into the
 * renderer's format).  Writes to perm[n] (HOST) the permutation that lists the node's
 * Gaussians along a Z-order (Morton) curve of their means, mean[n,3] (HOST, FP32): 21 bits
 * per axis over the node's bounding box, one cell size for all axes, ties and non-finite means
 * (placed last) in index order.  The caller stores every attribute array permuted by it,
 * a'[i] = a[perm[i]], once at load time; global ids then follow the new order.  The renderer
 * culls each run of 32 consecutive Gaussians per view with one bounding-sphere test, which
 * rejects work only for spatially compact runs: the order changes speed, not the image
 * (except the id tie-break between Gaussians with bit-equal depth keys in one pixel).
 * Returns DGS_ERR_INVALID_ARG for n < 0 or null pointers with n > 0.  No GPU is used.
 */
int dgs_spatial_order(const float* mean, int64_t n, int64_t* perm);

/* Result of dgs_autotune: the candidates timed and the one chosen. */
#define DGS_TUNE_MAX 16
typedef struct dgs_tune_result {
    int32_t n;                        /* candidates timed */
    int32_t best;                     /* index of the fastest */
    int32_t tile_w[DGS_TUNE_MAX];
    int32_t tile_h[DGS_TUNE_MAX];
    float ms[DGS_TUNE_MAX];           /* mean milliseconds per dgs_render call */
} dgs_tune_result;

/*
 * Picks the compositing tile shape for a batch by timing it (Sec. III-A's rasterizer works on
 * screen tiles; their shape changes speed, never the image).  Renders the batch (arguments as
 * for dgs_render) with each candidate tile shape: one untimed call (in DGS_MODE_GRAPH that
 * call captures), then `reps` timed calls (CUDA events on `stream` around the calls, host
 * staging included).  Sets the context's tile shape to the fastest, renders once more with it
 * (so the outputs, and in graph mode the captured graph, belong to the chosen shape) and
 * fills *out.  All candidates produce the same image; only the binning granularity changes.
 *
 *   candidates  HOST [n_candidates][2] (tile_w, tile_h) pairs, each valid for dgs_options;
 *               NULL = 16x16, 32x8, 8x32, 16x8, 8x8.
 *   reps        timed calls per candidate, 1..1000.
 *
 * Returns DGS_ERR_INVALID_ARG for a bad candidate list (nothing rendered) and the first
 * failing render's status otherwise (the context keeps its previous tile shape).
 */
int dgs_autotune(dgs_ctx* ctx, const dgs_node* nodes, int32_t n_nodes,
                 const int32_t* env_node_ids, int32_t n_envs, int32_t max_nodes,
                 const float* node_poses,
                 const dgs_camera* cams, const int32_t* cams_per_env, int32_t max_cams,
                 float* out_rgb, float* out_depth, float* out_alpha,
                 const int64_t* view_pixel_offset,
                 const int32_t* candidates, int32_t n_candidates, int32_t reps,
                 dgs_tune_result* out, void* stream);

/*
 * Image randomisation of rendered frames (Sec. IV: policies are trained on rendered images
 * that are blended with crops of Internet videos, jittered in HSV space and given a random
 * gamma).  One parameter set per view, drawn by the caller.  Per pixel (x, y) of a view, with
 * c its composited RGB (background included):
 *   c0 = clamp(c, 0, 1)
 *   c1 = (1 - overlay_beta) c0 + overlay_beta o,   o = overlay[overlay_frame,
 *        (overlay_y + y) mod overlay_h, (overlay_x + x) mod overlay_w] / 255  (crop with wrap-around;
 *        not read when overlay_beta = 0)
 *   (H, S, V) = hexcone HSV of c1 (H in turns; H = 0 for a grey, S = 0 for black)
 *   c2 = RGB of (frac(H + hue_shift), min(1, S sat_scale), min(1, V val_scale))
 *   out = c2 ^ gamma  (0 ^ gamma = 0; gamma = 1 leaves c2 unchanged)
 * Depth and alpha are not randomised.  FP32 arithmetic: the two divisions of the HSV conversion
 * are approximate (2 ulp), a chroma max - min <= 1e-30 counts as grey, and the power is
 * 2^(gamma log2 c2) with the hardware's approximate base-2 logarithm and exponential.
 */
typedef struct dgs_augment {
    float hue_shift;            /* turns added to the hue, any finite value (1 = 360 degrees) */
    float sat_scale;            /* >= 0, finite */
    float val_scale;            /* >= 0, finite */
    float gamma;                /* > 0, finite */
    float overlay_beta;         /* weight of the overlay in the blend, in [0, 1] */
    int32_t overlay_frame;      /* 0 .. n_frames-1 */
    int32_t overlay_x;          /* crop origin in the frame: 0 .. overlay_w-1 */
    int32_t overlay_y;          /* 0 .. overlay_h-1 */
} dgs_augment;                  /* 32 bytes */

/*
 * Sec. IV randomisation, set per context.  Sets (or clears) the randomisation that every
 * later dgs_render / dgs_autotune call on ctx applies to its RGB output, fused into the
 * compositing kernel (the un-randomised colour is never written).
 *
 *   aug[n_views]   HOST, one record per view in dgs_render's view order; copied (the caller may
 *                  free it on return).  aug = NULL or n_views = 0 clears the randomisation.
 *   overlay        DEVICE uint8 [n_frames, overlay_h, overlay_w, 3] (row-major, interleaved RGB),
 *                  the clip whose crops are blended in; it must stay valid and unchanged while
 *                  calls that read it run.  May be NULL only if every overlay_beta is 0.
 *   n_frames, overlay_w, overlay_h  >= 1 and <= 32768 each when overlay is set.
 *
 * A render whose batch does not have exactly n_views views fails with DGS_ERR_INVALID_ARG.
 * dgs_render_backward fails with DGS_ERR_UNSUPPORTED while a randomisation is set (its
 * out_rgb must be the un-randomised forward output).  In DGS_MODE_GRAPH the records are
 * uploaded with the other host tables on every call; a new overlay pointer or shape, or
 * turning the randomisation on or off, recaptures.  Returns DGS_ERR_INVALID_ARG (and keeps the
 * previous setting) for a parameter outside the ranges above.  dgs_render_noalloc never
 * randomises.
 */
int dgs_set_augment(dgs_ctx* ctx, const dgs_augment* aug, int32_t n_views, const uint8_t* overlay,
                    int32_t n_frames, int32_t overlay_w, int32_t overlay_h);

/*
 * Sec. IV randomisation as a separate pass.  Applies the randomisation set on ctx to an
 * existing RGB image batch, in place, as a separate kernel (the same per-pixel arithmetic as
 * the fused path, so the result is bitwise that of dgs_render with the randomisation set).
 *
 *   rgb                  DEVICE FP32 [total_pixels,3], read and overwritten.
 *   view_size[n_views*2] HOST (width, height) of each view, 1..32768.
 *   view_pixel_offset    HOST [n_views] first pixel of each view, or NULL (views packed in order).
 *   n_views              must equal the n_views of dgs_set_augment (>= 1).
 *
 * Work is queued on `stream` and the call returns without synchronising (with dgs_options.profile
 * set it synchronises to read its kernel time); the host tables are staged in the context (the
 * caller's arrays may be freed on return).  Returns
 * DGS_ERR_INVALID_ARG when no randomisation is set or an argument is out of range.
 */
int dgs_augment_rgb(dgs_ctx* ctx, float* rgb, const int32_t* view_size, const int64_t* view_pixel_offset,
                    int32_t n_views, void* stream);

/*
 * LiDAR by Gaussian ray tracing (Sec. III-C: LiDAR is simulated by native ray tracing of the
 * scene's Gaussians, accelerated by a BVH).  For a ray o + t d (|d| = 1, t in metres) and a
 * Gaussian with mean mu and whitening M = diag(1/s) R^T in its node's frame (o, d moved there
 * with the node's pose): o' = M (o - mu), d' = M d; the response peaks at
 * t* = -(o'.d') / (d'.d') with Mahalanobis distance q* = |o' x d'|^2 / (d'.d').  A Gaussian is
 * hit iff q* <= q_max and r_min <= t* <= r_max; alpha = min(alpha_max, opacity exp(-q* / 2)),
 * skipped when < alpha_min.  Hits composite front to back in (t*, global id) order, stopping
 * (without the current hit) once T (1 - alpha) < t_min: D = sum T alpha t* (not normalised),
 * A = 1 - T_final.  The return's range is D / A.  q_max, alpha_min, alpha_max and t_min are the
 * context's options.  FP32 arithmetic.
 */
typedef struct dgs_lidar {
    int32_t env;                /* the env whose nodes the sensor sees */
    float world_from_sensor[12]; /* row-major [R|t], R orthonormal within 1e-4 */
} dgs_lidar;                    /* 52 bytes */

/*
 * Sec. III-C (BVH-accelerated ray tracing).  Builds the ray-tracing structures of the nodes
 * on the context: per Gaussian a 64-byte record
 * (mean, opacity, whitening matrix) and per node an implicit binary BVH over leaves of 8
 * consecutive Gaussians in storage order (store nodes in dgs_spatial_order for compact
 * leaves), boxes of the q_max ellipsoids in the node's frame.  Reads the nodes' mean,
 * log_scale, quat and opacity_logit (DEVICE, any dgs_dtype); replaces any earlier build.  Call
 * it again whenever those attributes change.  Synchronises `stream`.  Returns
 * DGS_ERR_INVALID_ARG for the node errors dgs_render reports.
 */
int dgs_lidar_build(dgs_ctx* ctx, const dgs_node* nodes, int32_t n_nodes, void* stream);

/*
 * Sec. III-C LiDAR returns.  Traces n_sensors x n_dirs rays: ray (s, j) starts at sensor s's origin along
 * R_s dirs[j] (normalised).
 *   nodes, n_nodes                the nodes of the last dgs_lidar_build (same sizes and attribute
 *                                 pointers; else DGS_ERR_INVALID_ARG)
 *   env_node_ids, n_envs, max_nodes, node_poses   as for dgs_render (node_poses DEVICE)
 *   sensors[n_sensors]            HOST
 *   dirs[n_dirs*3]                DEVICE FP32 sensor-frame directions (non-zero)
 *   r_min, r_max                  range window, 0 <= r_min < r_max, finite
 *   out_d, out_a                  DEVICE FP32 [n_sensors*n_dirs], sensor-major (sensors, dirs and the
 *                                 outputs may be NULL when n_sensors = 0: nothing is traced)
 * Work is queued on `stream`; the call synchronises it before returning (device-side pose
 * validation is reported as DGS_ERR_INVALID_ARG).  Rays (s, j) .. (s, j + 31) are traced together
 * as one packet: order dirs so that every 32 consecutive directions are neighbours (e.g. tiles of
 * 4 channels x 8 azimuths) — the result does not depend on the order, the speed does.
 */
int dgs_lidar_trace(dgs_ctx* ctx, const dgs_node* nodes, int32_t n_nodes,
                    const int32_t* env_node_ids, int32_t n_envs, int32_t max_nodes, const float* node_poses,
                    const dgs_lidar* sensors, int32_t n_sensors, const float* dirs, int32_t n_dirs,
                    float r_min, float r_max, float* out_d, float* out_a, void* stream);

/*
 * Mesh -> Gaussian transfer (Sec. III-B, Mesh-Gaussian Transfer: interactive nodes reconstructed
 * as textured meshes become Gaussian nodes).  Writes one Gaussian per facet, in the node layout
 * of dgs_node (FP32): mean = the facet's barycentre; rotation with columns (t1, t2, n),
 * n = normalised (v1 - v0) x (v2 - v0), t1 = normalised v1 - v0, t2 = n x t1 (identity for a
 * facet of zero area); log_scale = (log s, log s, log(flatten s)) with s the mean
 * barycentre-to-vertex distance (at least 1e-12); opacity_logit as given; SH degree-0
 * coefficient (c - 1/2) / Y_00 with c the mean of the facet's vertex colours (zero without
 * colours) and higher-degree coefficients zero.
 *
 *   vertices[n_vertices*3]       DEVICE FP32
 *   faces[n_faces*3]             DEVICE int32 vertex indices
 *   vertex_colors                DEVICE FP32 [n_vertices*3] in [0,1], or NULL
 *   flatten                      normal-to-tangent scale ratio, (0, 1]
 *   sh_degree                    0..3: out_sh holds (sh_degree+1)^2 coefficients per facet
 *   out_mean [F*3], out_log_scale [F*3], out_quat [F*4] (16-byte aligned), out_opacity_logit [F],
 *   out_sh [F*(sh_degree+1)^2*3]  DEVICE FP32
 * Synchronises `stream`; a face index outside [0, n_vertices) gives DGS_ERR_INVALID_ARG (that
 * facet's outputs are the identity-frame defaults).
 */
int dgs_mesh_to_gaussians(dgs_ctx* ctx, const float* vertices, int64_t n_vertices, const int32_t* faces,
                          int64_t n_faces, const float* vertex_colors, float flatten, float opacity_logit,
                          int32_t sh_degree, float* out_mean, float* out_log_scale, float* out_quat,
                          float* out_opacity_logit, float* out_sh, void* stream);

/*
 * Depth -> TSDF fusion (Sec. III-B: a Gaussian node is converted back to a mesh by rendering
 * multi-view depth maps and fusing them into a truncated signed distance field; decimation is
 * not part of the library).  Updates a voxel field in place, view by view in the given order.
 * Voxel (i, j, k) (x fastest) has centre origin + (i + 1/2, j + 1/2, k + 1/2) * voxel.  Per view:
 * x_c = cam_from_world p; skip if z_c <= 0; (u, v) = (fx x_c / z_c + cx, fy y_c / z_c + cy), the
 * pixel (floor u, floor v), skipped outside the image; the depth is D / A (the renderer's
 * unnormalised depth over its coverage), valid where A >= min_alpha; sdf = D / A - z_c, skipped
 * when sdf < -trunc; f = min(1, sdf / trunc); F <- (W F + f) / (W + 1); W <- min(W + 1, max_weight).
 * FP32 (approximate reciprocal in the projection and the normalisation).
 *
 *   tsdf, weight             DEVICE FP32 [nz*ny*nx] (start from F = 0, W = 0)
 *   nx, ny, nz               >= 1, nx*ny*nz < 2^31
 *   origin[3]                HOST, world coordinates of the grid's corner
 *   voxel, trunc, max_weight > 0, finite; min_alpha in (0, 1]
 *   cams[n_views]            HOST (intrinsics, resolution and cam_from_world of each view)
 *   depth, alpha             DEVICE FP32, flat over views like dgs_render's out_depth/out_alpha
 *   view_pixel_offset        HOST [n_views] or NULL (views packed in order)
 * Work is queued on `stream` without synchronising (with dgs_options.profile set the call
 * synchronises to read its kernel time); the host tables are staged in the context.
 */
int dgs_tsdf_integrate(dgs_ctx* ctx, float* tsdf, float* weight, int32_t nx, int32_t ny, int32_t nz,
                       const float* origin, float voxel, float trunc, float max_weight, float min_alpha,
                       const dgs_camera* cams, int32_t n_views, const float* depth, const float* alpha,
                       const int64_t* view_pixel_offset, void* stream);

/*
 * dgs_render_noalloc -- dgs_render for callers that must not allocate GPU memory.  The paper
 * has no counterpart: this is a deployment variant of the same batched render.
 *
 * Some callers cannot call cudaMalloc: a program whose device memory is owned by another
 * framework's caching allocator, a control loop that cannot take the device-wide
 * synchronisation that cudaMalloc/cudaFree may cause in the middle of a step, or code certified
 * to allocate nothing after start-up.  This call allocates no device or pinned host memory:
 * its workspace is a fixed 64 MiB array compiled into the library, present on every device
 * that loads it until the process exits.
 *
 *   opt       options (NULL = defaults); mode and profile are ignored, the batched sequence runs
 *             as a single view group.
 *   the other arguments are those of dgs_render (caller-owned inputs and outputs).
 *
 * Returns DGS_ERR_CAPACITY, before its second phase is queued, when the batch's tables,
 * projected records or tile pairs do not fit in the 64 MiB; DGS_ERR_INVALID_ARG for the cases
 * dgs_render rejects; no error message is recorded (there is no context).  The first call on a
 * device resolves the array's device address (cudaGetSymbolAddress) with that device current;
 * make it before any stream capture begins.  All calls on a device share the array and leave
 * their contents in it; each call clears what must start at zero.  Calls whose GPU work
 * overlaps (other streams or host threads) race on the array: serialise them.  The call reads
 * counts back once and synchronises `stream` before returning.
 */
int dgs_render_noalloc(const dgs_options* opt, const dgs_node* nodes, int32_t n_nodes,
                       const int32_t* env_node_ids, int32_t n_envs, int32_t max_nodes,
                       const float* node_poses,
                       const dgs_camera* cams, const int32_t* cams_per_env, int32_t max_cams,
                       float* out_rgb, float* out_depth, float* out_alpha,
                       const int64_t* view_pixel_offset, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* DGS_H */
