/*
 * gs.h -- C ABI of the B300-native batched 3D Gaussian Splatting renderer.
 *
 * The library renders, for a batch of cameras (one per simulated robot), every
 * camera's view of its scene of 3D Gaussians and returns colour and expected
 * depth. This is the renderer the paper drops into its vectorised simulator
 * (Sec. 3.2 "3D Gaussian Splatting as a Drop-in Renderer"), with depth as a
 * by-product of the same compositing pass (Sec. 3.3, Fig. 4), rendering many
 * robots over many scenes on one GPU (Sec. 3.3: 4,096 environments over 128
 * scenes at 640x480). The rasteriser itself is the 3DGS method the paper cites
 * (Sec. 2.3): EWA projection with a 0.3 px dilation, SH colour, 3-sigma tile
 * culling, 16x16 tiles, per-tile order by (depth, Gaussian index), front-to-back
 * compositing with alpha = min(0.99, o exp(-d^T Sigma'^-1 d / 2)), alpha < 1/255
 * skipped, and a pixel stops before its transmittance would fall below 1e-4.
 *
 * Conventions (all calls):
 *  - Pointers are plain host or device addresses as stated per argument; no
 *    framework types cross this boundary. `stream` is a cudaStream_t passed as
 *    void* (NULL = the legacy default stream).
 *  - Every call returns a gs_status; nothing throws. On failure the outputs of
 *    that call are unspecified and gs_last_error() holds a one-line reason.
 *  - A context belongs to one device and one host thread at a time.
 *  - Cameras: `viewmats` are row-major 4x4 world->camera matrices (OpenCV axes:
 *    x right, y down, z forward); `intrinsics` are (fx, fy, cx, cy) in pixels;
 *    pixel (i, j) has its centre at (i + 0.5, j + 0.5).
 *  - Outputs: rgb is [n][H][W][3] float32, depth [n][H][W] float32 (expected
 *    depth sum_i w_i z_i of the camera-space depths, not normalised, 0 where
 *    nothing is drawn), final_T [n][H][W] float32 (the transmittance left).
 */
#ifndef GS_B300_H
#define GS_B300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum gs_status {
    GS_OK = 0,
    GS_ERR_INVALID_ARG = 1, /* bad pointer, size, id or configuration */
    GS_ERR_CUDA = 2,        /* a CUDA runtime call failed (message in gs_last_error) */
    GS_ERR_OOM = 3,         /* device or pinned host allocation failed */
    GS_ERR_CAPACITY = 4,    /* a request exceeds a fixed limit of the library */
    GS_ERR_TIMEOUT = 5,     /* a bounded device-side wait gave up */
    GS_ERR_NOT_FOUND = 6    /* unknown scene id */
} gs_status;

typedef enum gs_dtype { GS_F32 = 0, GS_F16 = 1, GS_BF16 = 2 } gs_dtype;
typedef enum gs_memory { GS_MEM_HOST = 0, GS_MEM_DEVICE = 1 } gs_memory;

/* Rendering constants and resource limits. gs_config_default() fills the
 * rasteriser's standard constants; the oracle uses the same values. */
typedef struct gs_config {
    float near_plane;      /* cull Gaussians whose camera-space z <= this (0.2) */
    float dilation;        /* added to the 2D covariance diagonal, px^2 (0.3) */
    float guard_band;      /* Jacobian clamp: x/z limited to guard*(W/2)/fx around the
                              principal point (1.3) */
    float sigma_cull;      /* footprint radius in standard deviations (3) */
    float alpha_min;       /* a pair with alpha below this is skipped (1/255) */
    float alpha_max;       /* alpha is clamped to this (0.99) */
    float T_min;           /* a pixel stops before T would fall below this (1e-4) */
    float background[3];   /* added as T * background to rgb (0, 0, 0) */
    int32_t max_chunk_cameras; /* cameras rendered per internal chunk (2048) */
    int32_t camera_group;  /* cameras of one scene that share one Gaussian load in the
                              projection kernels (128, at most 128) */
    int32_t count_pairs;   /* 1: the compositing kernel also counts evaluated pairs
                              (a slower variant of the kernel) */
    int32_t time_stages;   /* 1: record CUDA events around every stage on the render
                              stream; gs_get_stats reports the per-stage device time */
    int32_t pixels_per_thread; /* compositing layout: 2, 4 or 8 pixels per thread (8) */
    int32_t tiles_per_block;   /* compositing blocks: 1 = one block per 16x16 tile, 4 = one
                                  block per 2x2 quad of tiles sharing the list scan and the
                                  record staging (1; quads only with 8 pixels per thread,
                                  other layouts use one tile per block) */
    int64_t workspace_survivors; /* surviving (camera, Gaussian) pairs per chunk the
                                    workspace starts with (0: a third of the Gaussians a
                                    chunk sees); it grows when a render needs more */
    int32_t sync_errors;   /* 0: render calls only enqueue work; a chunk that does not
                              fit the workspace is reported later (sticky, see
                              gs_render_batch). 1: each render call waits for its
                              status and renders such chunks again at once (0) */
    int32_t comp_batch;    /* records staged per compositing batch with 8 pixels per
                              thread: 32, 64, 96 or 128 (32; 0 = 32) */
    int32_t persistent;    /* 1: binning and compositing of a chunk run as one persistent
                              launch pulling (camera, stage) work items from a device
                              queue (8 pixels per thread, one tile per block, no pair
                              counting, images of at most 128 64x64-pixel super-tiles;
                              other calls use separate launches). Its stage time is
                              reported as compositing. (0) */
    int32_t depth_prefix;  /* progressive depth order (8 pixels per thread, one tile per
                              block, separate launches, no pair counting): compositing
                              stops reading a tile's list once every pixel has stopped,
                              almost always within the nearest few per cent of a
                              camera's survivors, so a first phase orders and bins only
                              each camera's nearest ranks (at least this many, rounded
                              up to whole depth buckets; 0: 4,096, or 1/128 of the
                              camera's survivors when more), tiles that still have
                              live pixels there
                              save their state, and a second phase orders and bins the
                              rest of those tiles' cameras only and resumes them. The
                              images are the same as with the whole order. -1: the
                              whole order in one phase. (0) */
} gs_config;

/* A scene: n Gaussians stored as structure of arrays.
 * mean [3][n] (x row, y row, z row), log_scale [3][n], quat [4][n] (w, x, y, z;
 * normalised by the renderer), logit_opacity [n], sh [K][3][n] with
 * K = (sh_degree+1)^2 (coefficient-major, l-major with m = -l..l, then the
 * channel, then the Gaussian; real SH basis with the Condon-Shortley phase).
 * geometry_dtype applies to mean, log_scale and quat; appearance_dtype to
 * logit_opacity and sh. memory says whether all five pointers are host or
 * device addresses. */
typedef struct gs_scene_desc {
    int64_t n;
    int32_t sh_degree;        /* 0..3 */
    int32_t geometry_dtype;   /* gs_dtype */
    int32_t appearance_dtype; /* gs_dtype */
    int32_t memory;           /* gs_memory */
    const void *mean;
    const void *log_scale;
    const void *quat;
    const void *logit_opacity;
    const void *sh;
} gs_scene_desc;

/* Counters of the last render call. */
typedef struct gs_stats {
    int64_t n_cameras;
    int64_t survivors;       /* sum over cameras of Gaussians that survive culling */
    int64_t intersections;   /* sum over cameras of (survivor, covered tile) pairs */
    int64_t pairs_evaluated; /* (pixel, Gaussian) pairs whose alpha was computed before
                                the pixel stopped; only with count_pairs */
    int64_t pairs_alpha;     /* of those, pairs with alpha >= alpha_min; count_pairs */
    int32_t n_chunks;
    float ms_project;        /* per-stage device time summed over chunks, time_stages */
    float ms_sort;
    float ms_bin;
    float ms_composite;
    float ms_total;
    int32_t reserved0;
    int64_t warp_iters;       /* compositing (warp, Gaussian) iterations of warps with live
                                 pixels; only with count_pairs */
    int64_t warp_iters_box;   /* of those, Gaussians whose alpha box meets the warp's rows */
    int64_t warp_iters_blend; /* of those, Gaussians some lane of the warp blends */
    int64_t sort_windows_listed; /* depth-order windows left to the one-block sort in global
                                    memory (over 2,048 keys, over 512 buckets, or a bin of
                                    more than 32 keys) */
    int64_t sort_equal_runs;  /* runs of equal depth keys the window pass listed for ordering
                                 by caller index */
    int64_t sort_long_runs;   /* runs of more than 32 equal keys (one block each) */
    int64_t depth_second_phase_cameras; /* cameras the progressive order's second phase
                                           ordered further (depth_prefix) */
    int64_t depth_resumed_tiles; /* tiles it composited past their camera's first phase */
} gs_stats;

typedef struct gs_context gs_context;
typedef struct gs_graph gs_graph;

/* Library ABI version (changes when a struct layout or signature changes). */
int32_t gs_abi_version(void);

/* Human-readable name of a status code (static string). */
const char *gs_status_string(gs_status s);

/* Fill *out with the default constants and limits. */
gs_status gs_config_default(gs_config *out);

/* Create a context on CUDA device `device` (cfg NULL = defaults). The context
 * owns scene storage and the render workspace. *out is NULL on failure. */
gs_status gs_context_create(const gs_config *cfg, int32_t device, gs_context **out);

/* Replace a context's launch parameters (chunk size, camera group, compositing
 * layout and batch, counting, stage timing, sync_errors) after waiting for its
 * last render call; the rasteriser constants (near plane ... background) must
 * equal the context's. Scenes and workspace are kept. A service of the library
 * (used by its autotuner); the paper has no counterpart. Errors: INVALID_ARG. */
gs_status gs_context_set_config(gs_context *ctx, const gs_config *cfg);

/* Free a context and everything it owns (NULL is a no-op). Waits for its work. */
void gs_context_destroy(gs_context *ctx);

/* Last error message of this context (never NULL; "" after success). */
const char *gs_last_error(gs_context *ctx);

/* Copy a scene into the context (the caller keeps ownership of its arrays).
 * A scene is one of the paper's reconstructed environments as 3D Gaussians
 * (Sec. 3.1-3.2: mean, scale, rotation, opacity, SH colour per Gaussian). The
 * copy is done before the call returns; the library stores the Gaussians in a
 * spatial (Morton) order of their means and keeps each one's index in the
 * caller's arrays, which is the index the renderer orders equal depths by and
 * the inspection calls report. *scene_id stays valid until gs_scene_destroy.
 * Temporary device memory of about the scene's size is used during the call.
 * Errors: INVALID_ARG (n < 0, degree or dtype out of range, NULL pointer with
 * n > 0), OOM, CUDA. */
gs_status gs_scene_create(gs_context *ctx, const gs_scene_desc *desc, int32_t *scene_id);

/* Release a scene's storage. Errors: NOT_FOUND. */
gs_status gs_scene_destroy(gs_context *ctx, int32_t scene_id);

/* Render n_cams cameras of size width x height: the batched renderer of the
 * simulator, one camera per robot, RGB and expected depth from the same
 * compositing pass (Sec. 3.2 "3D Gaussian Splatting as a Drop-in Renderer";
 * Sec. 3.3 and Fig. 4 for depth; Sec. 3.3: 4,096 environments at 640x480).
 *   scene_ids   HOST   [n_cams] scene of each camera (the library groups cameras
 *                      by scene so one Gaussian load serves many cameras)
 *   viewmats    DEVICE [n_cams][16] float32, row-major world->camera
 *   intrinsics  DEVICE [n_cams][4]  float32 (fx, fy, cx, cy)
 *   rgb         DEVICE [n_cams][height][width][3] float32, written
 *   depth       DEVICE [n_cams][height][width] float32, written
 *   final_T     DEVICE [n_cams][height][width] float32 or NULL
 * Work is enqueued on `stream` and, with the default sync_errors = 0, the call
 * returns without waiting for it (it waits only when the workspace has to
 * grow, or for a staging buffer that a call two calls back still copies
 * from). The exception is a call whose chunks see more Gaussians than any call
 * before on this context: it sizes the workspace, so it waits for its status
 * and renders an overflowed chunk again before it returns. Calls on one
 * context run in call order even on different streams.
 * A chunk of cameras whose survivors exceed the workspace is not rendered;
 * the device records it in a sticky status word and a later render call,
 * gs_sync or gs_get_stats returns GS_ERR_CAPACITY (once); the images of that
 * call are then not valid, the workspace has grown to the size recorded, and
 * rendering again succeeds. With sync_errors = 1 the call instead waits for
 * its status and renders such chunks again before it returns.
 * Output buffers must not overlap the inputs. n_cams == 0 is a no-op.
 * Errors: INVALID_ARG, NOT_FOUND, CAPACITY (more than 65536 16x16 tiles per camera),
 * OOM, CUDA. */
gs_status gs_render_batch(gs_context *ctx, int32_t n_cams, const int32_t *scene_ids,
                          const float *viewmats, const float *intrinsics, int32_t width,
                          int32_t height, float *rgb, float *depth, float *final_T,
                          void *stream);

/* gs_render_batch with a size per camera (a batch may mix resolutions; many
 * robots over scenes of uneven size, Sec. 3.3: 4,096 environments over 128
 * scenes).
 *   widths, heights  HOST [n_cams] camera sizes (each as in gs_render_batch)
 *   pixel_offsets    HOST [n_cams] index of camera i's first pixel in the packed
 *                    outputs: camera i writes rgb[3 * (off_i + y * W_i + x) + ch],
 *                    depth[off_i + y * W_i + x], final_T likewise; the images must
 *                    not overlap
 * Other arguments and errors as gs_render_batch. */
gs_status gs_render_batch_v(gs_context *ctx, int32_t n_cams, const int32_t *scene_ids,
                            const float *viewmats, const float *intrinsics,
                            const int32_t *widths, const int32_t *heights,
                            const int64_t *pixel_offsets, float *rgb, float *depth,
                            float *final_T, void *stream);

/* Motion blur as the paper simulates it (Sec. 3.3, Fig. 9): `samples` frames
 * whose camera centres are moved along the camera's velocity, by
 * velocity * shutter * (j/(samples-1) - 1/2) for frame j (orientation kept),
 * rendered and blended with equal weights 1/samples into one image per camera
 * (rgb, depth and final_T alike). samples = 1 is a plain render.
 *   velocities  DEVICE [n_cams][3] float32, world-frame camera velocity (m/s)
 *   shutter     exposure time in seconds (>= 0); samples in 1..64
 * Other arguments and errors as gs_render_batch (outputs must not alias the
 * inputs; the frames are accumulated in rgb / depth / final_T). */
gs_status gs_render_motion_blur(gs_context *ctx, int32_t n_cams, const int32_t *scene_ids,
                                const float *viewmats, const float *intrinsics,
                                const float *velocities, float shutter, int32_t samples,
                                int32_t width, int32_t height, float *rgb, float *depth,
                                float *final_T, void *stream);

/* Record the render of a fixed batch of cameras (arguments as gs_render_batch_v,
 * no stream) into a CUDA graph (the paper's vectorised simulator renders the
 * same batch of environment cameras every camera step, Sec. 3.3). The call renders the batch once (which sizes the
 * workspace; the graph keeps 1.25x headroom over the survivors it saw), then
 * captures the whole kernel sequence -- projection, sort, binning, compositing
 * for every chunk, with no host round trip inside -- into one graph. Later
 * launches read the cameras from and write the images to the same device
 * addresses: update viewmats / intrinsics in place between launches. A graph
 * uses its context's workspace: renders on that context (eager or other
 * graphs) must not overlap its launches, and an eager render that has to grow
 * the workspace invalidates it (gs_graph_launch then returns INVALID_ARG). */
gs_status gs_graph_create(gs_context *ctx, int32_t n_cams, const int32_t *scene_ids,
                          const float *viewmats, const float *intrinsics,
                          const int32_t *widths, const int32_t *heights,
                          const int64_t *pixel_offsets, float *rgb, float *depth,
                          float *final_T, gs_graph **out);

/* Enqueue one replay of the graph on `stream` (no host synchronisation). */
gs_status gs_graph_launch(gs_graph *g, void *stream);

/* Wait for `stream` and report whether the last replay fitted the workspace:
 * GS_ERR_CAPACITY when cameras moved so that a chunk had more survivors than
 * the workspace holds (that chunk's images are not written); render eagerly
 * once and create the graph again. */
gs_status gs_graph_check(gs_graph *g, void *stream);

/* Free the graph (NULL is a no-op). */
void gs_graph_destroy(gs_graph *g);

/* Same as gs_render_batch (Sec. 3.2) with every array in HOST memory, for a
 * host-side consumer of the frames: the call copies the
 * cameras to the device, renders into context-owned device buffers in parts of
 * at most min(max_chunk_cameras, 128) cameras and copies each part back on a
 * second stream while the next part renders (pinned host buffers make the copies asynchronous DMA).
 * Returns after the outputs are in host memory. */
gs_status gs_render_batch_host(gs_context *ctx, int32_t n_cams, const int32_t *scene_ids,
                               const float *viewmats, const float *intrinsics, int32_t width,
                               int32_t height, float *rgb, float *depth, float *final_T,
                               void *stream);

/* Counters (and stage times with time_stages) of the last render call (a
 * service of the library; the paper reports whole-simulator throughput only).
 * Waits for the last render call's work. Returns GS_ERR_CAPACITY (after
 * filling *out) when a render call of this context had a chunk that did not
 * fit the workspace and that has not been reported yet (see gs_render_batch);
 * the report clears it. */
gs_status gs_get_stats(gs_context *ctx, gs_stats *out);

/* Wait for `stream` and the context's last render call, then report a pending
 * device-detected error of an earlier asynchronous render call (as
 * gs_get_stats does; GS_OK if there is none). The paper has no counterpart:
 * it is the completion point of the asynchronous render calls. */
gs_status gs_sync(gs_context *ctx, void *stream);

/* Test of the persistent launch's bounded waits (see gs_config.persistent; the
 * paper has no counterpart): renders one camera (arguments as gs_render_batch,
 * viewmat / intrinsics in DEVICE memory) through the persistent binning +
 * compositing launch with the camera's tiles made to wait for one binning item
 * more than exists, and a bound of 4,096 polls. The waits give up, the tiles
 * are left unwritten, and the call returns GS_ERR_TIMEOUT after waiting for
 * `stream`; the context stays usable (the next render is complete). Any other
 * status means the bounded wait did not behave as documented. */
gs_status gs_render_timeout_probe(gs_context *ctx, int32_t scene_id, const float *viewmat,
                                  const float *intrinsics, int32_t width, int32_t height,
                                  float *rgb, float *depth, void *stream);

/* Test hook of the progressive depth order (gs_config.depth_prefix): the list of
 * saved tile states a chunk's first phase fills holds at most `tiles` entries on
 * later render calls (0: the default, a sixteenth of the chunk's tiles, at least
 * 1,024). Tiles past it are rendered again from rank 0 by the second phase, with
 * the same images. Returns GS_ERR_INVALID_ARG for a NULL context or tiles < 0. */
gs_status gs_set_resume_capacity(gs_context *ctx, int32_t tiles);

/* ---------------------------------------------------------------------------
 * Inspection entry points (used by the test suite). Each runs the hot-path
 * kernels for ONE camera (viewmat / intrinsics in DEVICE memory) and copies an
 * intermediate result to HOST buffers. They synchronise `stream`.
 * ------------------------------------------------------------------------- */

/* Projected records of the camera's surviving Gaussians, in Gaussian-index
 * order. rec: HOST [cap][12] float32 = (u, v, z, opacity, A, B, C, r, red,
 * green, blue, 0) with (A, B, C) the conic (inverse 2D covariance entries
 * [[A, B], [B, C]]) and r the footprint radius in pixels; gidx: HOST [cap]
 * Gaussian indices; rect: HOST [cap][4] tile rect (x0, x1, y0, y1, inclusive).
 * *n_out receives the survivor count; CAPACITY if it exceeds cap (nothing is
 * copied then). */
gs_status gs_debug_project(gs_context *ctx, int32_t scene_id, const float *viewmat,
                           const float *intrinsics, int32_t width, int32_t height, float *rec,
                           int32_t *gidx, int32_t *rect, int64_t cap, int64_t *n_out,
                           void *stream);

/* Per-tile Gaussian lists of the camera in compositing order (depth, index).
 * tile_off: HOST [ntiles+1] list offsets (ntiles = ceil(W/16) * ceil(H/16),
 * tiles row-major); gidx: HOST [cap] Gaussian indices. *n_out receives the
 * number of entries; CAPACITY if it exceeds cap (tile_off is still filled). */
gs_status gs_debug_tile_lists(gs_context *ctx, int32_t scene_id, const float *viewmat,
                              const float *intrinsics, int32_t width, int32_t height,
                              int64_t *tile_off, int32_t *gidx, int64_t cap, int64_t *n_out,
                              void *stream);

/* A segmented sort on caller data (no counterpart in the paper: the library's
 * stable radix sort, with which scene set-up orders the Morton codes of the
 * means; the render's depth order has kernels of its own): within each segment
 * [seg_start[s], seg_start[s] + seg_count[s]) of keys/vals, a stable ascending
 * sort of the uint32 keys, vals moved with their keys, in place.
 * keys, vals: DEVICE [n] uint32; seg_start, seg_count: DEVICE [n_seg] int64,
 * segments must not overlap and lie within [0, n) (else GS_ERR_INVALID_ARG).
 * The call reads the segment table to the host (it waits on `stream` for it);
 * its scratch (2 n uint32 and the tile tables) belongs to the context but not
 * to the render workspace, so a render still running on another stream is not
 * disturbed. */
gs_status gs_sort_segments(gs_context *ctx, uint32_t *keys, uint32_t *vals, int64_t n,
                           const int64_t *seg_start, const int64_t *seg_count, int32_t n_seg,
                           void *stream);

/* The segmented sort of gs_sort_segments for callers that cannot allocate
 * GPU memory (code inside a graph or stream region it does not own, plugins of
 * a host application that owns every device allocation, loops that forbid
 * allocation after start-up). The paper has no counterpart: this is a service
 * of this library. It takes no context and allocates nothing: its scratch
 * (temporary keys and values, tile table, histograms) is one file-scope device
 * array of about 22 MB that every GPU loading this library holds until the
 * process exits.
 *   keys, vals  DEVICE [n] uint32, sorted in place within each segment
 *               (stable, ascending keys; vals move with their keys)
 *   seg_start, seg_count  DEVICE [n_seg] int64; a segment outside [0, n) is
 *               treated as empty; segments must not overlap
 * Limits: n <= 2,097,152 keys and n_seg <= 4,096 segments, else
 * GS_ERR_CAPACITY with nothing done. The first call on a device looks up the
 * array's device address (a CUDA runtime query): make it before any stream
 * capture. The address is kept for the life of the process: a cudaDeviceReset of
 * that device after the first call is not supported. All calls share the array
 * and it keeps the last call's contents,
 * so calls that may overlap on the GPU (other streams or host threads) race
 * and must be serialised by the caller. Work is enqueued on `stream`. */
gs_status gs_sort_segments_noalloc(uint32_t *keys, uint32_t *vals, int64_t n,
                                   const int64_t *seg_start, const int64_t *seg_count,
                                   int32_t n_seg, void *stream);

/* ---- Measurement ----
 * Arithmetic-rate microbenchmarks for the renderer's roofline (the paper has
 * no counterpart: it reports whole-simulator throughput only). The compositing
 * pass is bound by FP32 arithmetic and the SFU exponential, and the device's
 * rates for these are measured rather than derived from unit counts.
 *   kind    0 = scalar FP32 FMA, 1 = packed FP32x2 FMA, 2 = ex2.approx.ftz.f32
 *   blocks  grid size (256 threads each; a multiple of the SM count fills the GPU)
 *   iters   rounds per thread (each round: 8 x 16 operations per thread)
 *   sink    DEVICE float32 [blocks], never written in practice (keeps the work)
 *   ops     HOST, receives the work of the launch: flops (2 per FMA) for kinds
 *           0 and 1, exponentials for kind 2
 * Enqueues one kernel on `stream` and returns; time it with events on that
 * stream. Errors: INVALID_ARG, CUDA (launch failure). */
gs_status gs_microbench(int32_t kind, int32_t blocks, int32_t iters, float *sink, int64_t *ops,
                        void *stream);

/* ---- Learned 4x upsampler ----
 * The paper renders every robot camera at 640x480 (Sec. 3.2) and has no
 * upsampler; this is a service of this library: a small residual CNN that
 * turns a render at a quarter of the resolution (e.g. 160x120, intrinsics / 4)
 * into the full-resolution image, trained on pairs the renderer produces.
 *   x0  = [rgb - 1/2, S (rgb - box3(rgb))]   6 channels, S = 32
 *   h_l = relu(conv3x3(h_{l-1}))           l = 1..5, 32 channels
 *   z   = conv3x3(h_5)                      48 channels
 *   out = bilinear4(rgb) + pixel_shuffle4(z) / S
 * box3 is the 3x3 mean (indices clamped); the detail channels and the 1/S
 * scale keep the small differences between a render and its bilinear
 * upsampling well above BF16's relative precision.
 * conv3x3 is cross-correlation with zero padding 1; pixel_shuffle4 sends
 * channel 16 c + 4 dy + dx of LR pixel (y, x) to colour c of HR pixel
 * (4 y + dy, 4 x + dx); bilinear4 uses half-pixel centres (HR pixel centre
 * i + 1/2 at LR coordinate (i + 1/2) / 4) with edge clamp. Weights and
 * activations are BF16 on the tensor cores with FP32 accumulation; master
 * weights, the loss and Adam are FP32.
 * Parameters: one flat FP32 array, per layer weights [c_out][c_in][3][3] then
 * biases [c_out], layers (c_out, c_in) = (32, 6), (32, 32) x 4, (48, 32):
 * gs_upsampler_param_count() = 52,624 values. A new upsampler has all
 * parameters zero (it then computes plain bilinear upsampling). */
typedef struct gs_upsampler gs_upsampler;

int64_t gs_upsampler_param_count(void);

/* Creates an upsampler on `device`. GS_ERR_INVALID_ARG for a bad device,
 * GS_ERR_OOM / GS_ERR_CUDA when its ~1.5 MB of parameter state cannot be set up. */
gs_status gs_upsampler_create(int32_t device, gs_upsampler **out);
void gs_upsampler_destroy(gs_upsampler *u);
const char *gs_upsampler_last_error(gs_upsampler *u);

/* HOST arrays of exactly gs_upsampler_param_count() floats. set_params also
 * clears the Adam moments and step count; all three synchronise the device. */
gs_status gs_upsampler_set_params(gs_upsampler *u, const float *host_params, int64_t n);
gs_status gs_upsampler_get_params(gs_upsampler *u, float *host_params, int64_t n);
/* Gradient of the last gs_upsample_grad call, same layout as the parameters. */
gs_status gs_upsampler_get_grads(gs_upsampler *u, float *host_grads, int64_t n);

/* Inference: n frames of h x w.
 *   lr_rgb    DEVICE [n][h][w][3] f32     lr_depth  DEVICE [n][h][w] f32 or NULL
 *   hr_rgb    DEVICE [n][4h][4w][3] f32   hr_depth  DEVICE [n][4h][4w] f32 or NULL
 * (depth is upsampled bilinearly; both depth pointers NULL or both set).
 * Enqueued on `stream`; the workspace (<= ~1 GB, frames in groups) grows with
 * cudaMalloc on first use. Sizes: n >= 0, 1 <= h, w <= 65535. */
gs_status gs_upsample_forward(gs_upsampler *u, int32_t n, int32_t h, int32_t w,
                              const float *lr_rgb, const float *lr_depth, float *hr_rgb,
                              float *hr_depth, void *stream);

/* Kernels of gs_upsample_forward and of gs_upsample_grad (forward, backward-data
 * and weight-gradient passes): the 5th-generation tensor cores (tcgen05.mma with
 * tensor-memory accumulators; the default) or warp-level mma.sync. Both compute
 * the same network with BF16 operands and FP32 accumulation. */
enum { GS_UPSAMPLE_TCGEN05 = 0, GS_UPSAMPLE_MMA_SYNC = 1 };
gs_status gs_upsampler_set_backend(gs_upsampler *u, int32_t backend);

/* Waits for `stream` and reports whether a tensor-core convolution enqueued
 * on it gave up waiting for its MMAs (GS_ERR_TIMEOUT; that call's outputs are
 * incomplete). Clears the flag. */
gs_status gs_upsample_check(gs_upsampler *u, void *stream);

/* Test hook for the failure path of the tensor-core kernels (no counterpart in
 * the paper): enqueues a hidden-layer convolution and a last-layer
 * (upsampling) convolution on a small internal input, in each of which the
 * first accumulator-ready signal per block is deliberately never sent, with
 * waits that give up after 4,096 polls. Every block then records the time-out,
 * waits for its own loads and MMAs and frees its tensor memory; the next
 * gs_upsample_check returns GS_ERR_TIMEOUT and the upsampler stays usable. No
 * GPU fault is involved. */
gs_status gs_upsample_timeout_probe(gs_upsampler *u, void *stream);

/* Training pass: forward on lr_rgb, loss = mean over HR pixels and channels of
 * (out - hr_target)^2, and the gradient of the loss with respect to every
 * parameter into the upsampler's gradient buffer (replacing the previous one).
 *   lr_rgb DEVICE [n][h][w][3], hr_target DEVICE [n][4h][4w][3] f32;
 *   loss   DEVICE 1 f32 (overwritten with the loss) or NULL.
 * The workspace holds every layer's activations (~0.8 KB per LR pixel). */
gs_status gs_upsample_grad(gs_upsampler *u, int32_t n, int32_t h, int32_t w, const float *lr_rgb,
                           const float *hr_target, float *loss, void *stream);

/* One Adam step (Kingma & Ba, bias-corrected) with the current gradient. */
gs_status gs_upsample_adam(gs_upsampler *u, float lr, float beta1, float beta2, float eps,
                           void *stream);

/* The upsampled render path in one call: renders every camera at a quarter of
 * the resolution (width / 4 x height / 4 with intrinsics / 4) and runs the
 * upsampler to width x height, RGB from the network and depth bilinear. The
 * batch is processed in parts of max_chunk_cameras cameras; the upsampler runs
 * part k on a stream of its own while part k + 1 renders. Arguments as
 * gs_render_batch (full-resolution intrinsics, outputs [n][height][width]...),
 * width and height multiples of 4; `up` must live on the context's device.
 * The work is ordered on `stream`: when it completes, the outputs are written.
 * The paper renders at full resolution; this path is a service of the library
 * (gs_upsampler_*) for callers that accept the upsampler's error. */
gs_status gs_render_batch_upsampled(gs_context *ctx, gs_upsampler *up, int32_t n_cams,
                                    const int32_t *scene_ids, const float *viewmats,
                                    const float *intrinsics, int32_t width, int32_t height,
                                    float *rgb, float *depth, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* GS_B300_H */
