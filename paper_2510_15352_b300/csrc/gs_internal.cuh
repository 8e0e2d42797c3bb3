// gs_internal.cuh -- data layouts and launchers shared by the kernel files of
// the batched 3DGS renderer (sm_103a). Nothing here is part of the C ABI.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace gsk {

constexpr int TILE = 16;            // tile edge in pixels
constexpr int MAX_GROUP = 128;      // cameras sharing one Gaussian load
constexpr int PROJ_THREADS = 256;   // Gaussians per projection block (8 mask words)
constexpr int BIN_THREADS = 256;    // threads per binning block
constexpr int BIN_RANKS = 1024;     // depth ranks per binning block (4 per thread) ...
constexpr int BIN_RANKS_SMALL = 256;  // ... or 1 per thread when the bitmap words of
                                      // 1,024 ranks of every super-tile exceed
constexpr int BIN_SMEM_MAX = 200 * 1024;  // this much shared memory
constexpr int MAX_TILES = 65536;    // tiles per camera (binning smem: 2 B per tile)
constexpr int COMP_BATCH = 64;      // Gaussian records staged per compositing sub-batch by
                                    // the 2- and 4-pixel and quad layouts
constexpr int COMP_BATCH_DEFAULT = 32;  // the configuration's batch for 8 px per thread
                                        // (32 / 64 / 96 / 128 selectable)

enum : int { DT_F32 = 0, DT_F16 = 1, DT_BF16 = 2 };

// Projection constants of a render call.
struct ProjParams {
    float near_plane, dilation, guard, sigma;
};

// Compositing constants of a render call.
struct CompParams {
    float log2_alpha_min;  // log2(alpha_min): alpha test done on log2(o e^power)
    float alpha_max, T_min;
    float log2_alpha_cap;  // log2(alpha_max) less a slack: for p + its float32 margin
                           // below it, 2^p < alpha_max (the cap can be left out)
    float bg[3];
    float out_w;           // outputs are out_w * value ...
    int accumulate;        // ... added to the existing outputs when non-zero
};

// A scene resident in device memory (structure of arrays, see gs.h).
// The Gaussians are stored in the library's spatial order (k_scene.cu): orig[p]
// is the caller's index of the Gaussian at position p; bounds holds two float4
// per group of 32 positions (min of the means and the largest squared scale;
// max of the means and a finite flag).
struct SceneDev {
    const void *mean, *log_scale, *quat, *logit, *sh;
    const int *orig;
    const float4 *bounds;
    // one row per Gaussian, for the records of the progressive order (read at
    // random positions): geo_rows 4 float4 = (mean, log2 o), M = R(q) S by rows
    // (M0..M3, M4..M7, M8), computed as the projection passes compute them;
    // sh_rows 48 coefficients of the appearance type, channel-major ([ch][16],
    // zero past the degree)
    const float4 *geo_rows;
    const void *sh_rows;
    const int *pos_of;  // pos_of[i]: the stored position of the caller's Gaussian i
    long long n;
    int deg, geo_dtype, app_dtype, pad;
};

// One camera of a chunk (a "slot"); offsets index the chunk's workspace arrays.
struct CamInfo {
    int user;        // index into viewmats / intrinsics / outputs
    int scene;       // index into the scene table
    int W, H;
    int TX, TY;
    int tile_off;    // first tile of this camera in the chunk's tile numbering
    int count;       // surviving Gaussians (after the scan)
    long long mask_off;  // first survival-mask word
    long long seg_off;   // first survivor slot
    long long bm_off;    // first super-tile bitmap word
    int nw;          // bitmap words per super-tile row = ceil(count / 32)
    int pad;
    long long pix_off;   // first pixel of this camera in the packed outputs
};

// Cameras of one scene that share a projection block's Gaussian loads.
struct Group {
    int scene, slot0, ncam, pad;
    long long n;
};

// A survivor's record, written by the projection pass in slot order
// (Gaussian-index order within the camera), in the form the compositing pass
// reads, with the constants folded so that p = a'dx^2 + b'dx dy + c'dy^2 + log2 o
// is log2(o e^power):
//   a: u, v, hx, hy      (hx, hy: half extents of the box around the region
//                         alpha >= alpha_min, widened past float32 rounding;
//                         negative when o < alpha_min)
//   b: a' = -log2(e)/2 A, b' = -log2(e) B, c' = -log2(e)/2 C, log2(o)
//   c: red, green, blue, z
//   d: x0 | x1 << 16, y0 | y1 << 16 (tile rect), Gaussian index, radius (bits)
// Layout in memory: blocks of 32 slots (2 KB), each holding the (a, b) pairs of
// its 32 slots, then their c, then their d. A warp writing consecutive slots
// writes each field as one contiguous run (coalesced stores), and a reader
// finds a and b of a slot in one 32-byte sector. (Plain 64-byte records in
// slot order made the projection's strided stores the bottleneck of its L1
// traffic; one array per field made the compositing pass touch three lines
// per record.) The render writes a, b and c only (the rect also goes to its own
// array); d is written for the debug entry points.
struct __align__(16) SlotRec {
    float4 a, b, c;
    uint4 d;
};
// float4 index of field a, b, c, d of slot s
__host__ __device__ inline long long rec_a(long long s) { return 4 * (s & ~31LL) + 2 * (s & 31); }
__host__ __device__ inline long long rec_b(long long s) { return rec_a(s) + 1; }
__host__ __device__ inline long long rec_c(long long s) { return 4 * (s & ~31LL) + 64 + (s & 31); }
__host__ __device__ inline long long rec_d(long long s) { return 4 * (s & ~31LL) + 96 + (s & 31); }
inline size_t rec_bytes(long long slots) { return (size_t)((slots + 31) / 32) * 32 * sizeof(SlotRec); }

constexpr int STILE = 4;  // tiles per super-tile edge (64 x 64 pixels)
constexpr int SORT_TILE_KEYS = 2048;  // keys per sort tile
constexpr int GS_STATUS_CAPACITY = 1; // device status word: a chunk exceeded the workspace

// ---- launchers (each defined in its kernel file) ----

// Projection constants of the chunk's cameras (cam_proj_bytes() each, in slot
// order), read by both projection passes.
size_t cam_proj_bytes();
cudaError_t launch_cam_setup(const CamInfo *cams, int m, const float *viewmats, const float *intr,
                             ProjParams P, void *camtab, cudaStream_t s);
cudaError_t launch_project_mask(const Group *groups, int n_groups, int max_blocks_x,
                                const SceneDev *scenes, const CamInfo *cams, const void *camtab,
                                ProjParams P, uint32_t *masks, cudaStream_t s);

cudaError_t launch_scan_masks(const CamInfo *cams, const SceneDev *scenes, int n_slots,
                              const uint32_t *masks, uint32_t *woff, int *counts,
                              cudaStream_t s);

cudaError_t launch_project_write(const Group *groups, int n_groups, int max_blocks_x,
                                 const SceneDev *scenes, const CamInfo *cams, const void *camtab,
                                 ProjParams P,
                                 const uint32_t *masks, const uint32_t *woff, float4 *rec, int rec_d,
                                 uint2 *srect, uint32_t *keys, uint32_t *oidx,
                                 float ln_alpha_min, const int *status, int max_deg,
                                 cudaStream_t s);
// The progressive order's projection output (instead of launch_project_write):
// per survivor slot only the depth key and the Gaussian's caller index; the
// records of the ranks the render reads are computed later by launch_bin_rec.
cudaError_t launch_project_keys(const Group *groups, int n_groups, int max_blocks_x,
                                const SceneDev *scenes, const CamInfo *cams, const void *camtab,
                                ProjParams P, const uint32_t *masks, const uint32_t *woff,
                                uint32_t *keys, uint32_t *oidx, const int *status, cudaStream_t s);

// Scene set-up (k_scene.cu): Morton codes of the means (box: 6 words of
// scratch) with idx = 0..n-1, to be sorted as (code, idx); a gather of `rows`
// attribute rows of n elements by perm; the projection-block bounds.
cudaError_t launch_scene_morton(const void *mean, int dtype, long long n, unsigned *box,
                                uint32_t *code, uint32_t *idx, cudaStream_t s);
cudaError_t launch_gather_rows(const void *src, void *dst, int elem_bytes, const uint32_t *perm,
                               long long n, int rows, cudaStream_t s);
// A stored scene's geo_rows / sh_rows (see SceneDev) from its attribute arrays,
// and pos_of, the inverse of orig.
cudaError_t launch_scene_rows(const SceneDev &s, float4 *geo_rows, void *sh_rows, int *pos_of,
                              cudaStream_t st);
long long scene_blocks(long long n);
cudaError_t launch_block_bounds(const void *mean, const void *log_scale, int dtype, long long n,
                                float4 *bounds, cudaStream_t s);

// Segmented sort: tile_start[n_seg + 1] is the prefix of sort_tiles_for(count)
// over the segments; hist needs 256 uint32 per tile. n_tiles blocks are
// launched; with n_tiles_dev != NULL the kernels loop over the device total
// *n_tiles_dev (grid-stride), else over n_tiles. With index_vals the input
// values are not read: value i of a segment is i (the projection's slots).
int sort_tiles_for(long long count);
cudaError_t launch_sort_segments(uint32_t *keys, uint32_t *vals, uint32_t *tmp_keys,
                                 uint32_t *tmp_vals, const long long *seg_start,
                                 const long long *seg_count, const int *tile_start, int n_seg,
                                 int n_tiles, uint32_t *hist, cudaStream_t s,
                                 const int *n_tiles_dev = nullptr, bool index_vals = false);

// One sort tile of a segmented sort: the segment's first key, the tile's
// first key within the segment, its key count, the segment's count and index
// (a direct lookup for the sort kernels, whose blocks would otherwise search
// the segment table first).
struct SortTile {
    long long seg_base;
    int t0, nk;
    int seg_n;  // keys of the whole segment
    int seg;    // the segment's index
};

// The render's depth order (k_depth.cu): every segment (camera) of keys (z bits
// minus the near plane's bits, slot order) sorted by (key, oidx[seg_base +
// slot]); the slots in that order end in sv. sk, keys and vals are scratch
// (sk and sv hold at least 4 elements past the chunk's survivors: the window
// pass copies 16-byte pieces). tiles / tile_start: the chunk's SortTile table
// and per-segment tile prefix (tile_start[m] the total, on the device);
// seg_start: the segments' first positions. Work buffers: count
// (DEPTH_BUCKETS uint32 per segment), win (SORT_TILE_KEYS / DEPTH_WINDOW
// entries of depth_window_bytes() per sort tile), big (big_cap entries of
// depth_big_bytes()), eq (eq_cap entries of depth_eq_bytes()), runs (run_cap
// entries of tie_run_bytes()), counters (3 ints, zeroed by the call). grid:
// blocks of the per-tile kernels. Chunk positions must stay below 2^32.
size_t depth_window_bytes();
size_t depth_big_bytes();
size_t depth_eq_bytes();
size_t tie_run_bytes();
constexpr int DEPTH_BUCKETS = 2048;  // per camera
constexpr int DEPTH_WINDOW = 1024;   // window stride (SORT_TILE_KEYS / 2)

// Progressive depth order. Compositing reads only the nearest few per cent of
// a camera's depth ranks before every pixel of a tile has stopped, so the first
// phase orders (and the binning pass bins) only each camera's ranks [0, pos):
// the buckets before `bucket`, which are the windows before `win1`. pos is the
// first bucket start at or past prefix ranks rounded up to whole windows
// (prefix: DEPTH_PREFIX_MIN, or count / DEPTH_PREFIX_DIV when larger, or the
// configured number; the whole segment when the order is not progressive).
// Measured: on the 640x480, 1M-Gaussian workload cuts at 2,048 and 4,096 ranks
// are as fast (1,024: more cameras need the second phase; 8,192 and an eighth
// of the survivors: more first-phase work is never read); on the 32-scene
// mixed batch, whose sparser scenes need deeper lists, 4,096 is 5 % faster than
// 2,048 (788 instead of 1,806 of 4,096 cameras need the second phase).
// A tile that still has live pixels at its camera's cut saves its compositing
// state and flags the camera; the second phase orders and bins the rest of the
// flagged cameras only and resumes those tiles.
struct DepthCut {
    int pos;     // first rank of the second phase (count when there is none)
    int bucket;  // its bucket (DEPTH_BUCKETS when there is none)
    int win1;    // windows of the first phase
    int count;   // the segment's keys
};
constexpr int DEPTH_PREFIX_MIN = 4096;
constexpr int DEPTH_PREFIX_DIV = 128;

// The work items of one phase per chunk (k_plan.cu, k_phase_map), an int
// array of phase_map_ints(m): [0] segments listed, [1..3] window items, binning
// blocks and sort tiles in all; then per kind (windows, binning blocks, sort
// tiles) the exclusive prefix of the listed segments' items and the first item
// of each. Item v of a kind is base[k] + v - pre[k] for the last k with
// pre[k] <= v.
inline size_t phase_map_ints(int m) { return 4 + 6 * (size_t)(m + 1); }
__device__ __forceinline__ int phase_item(const int *__restrict__ map, int m, int kind, int v) {
    const int *pre = map + 4 + 2 * kind * (m + 1), *base = pre + (m + 1);
    int lo = 0, hi = map[0] - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= v)
            lo = mid;
        else
            hi = mid - 1;
    }
    return base[lo] + v - pre[lo];
}
enum : int { MAP_WINDOWS = 0, MAP_BINS = 1, MAP_TILES = 2 };

// Phase maps: phase 1 lists every segment (its first-phase windows and binning
// blocks, all its sort tiles); phase 2 the segments whose flag is set (their
// remaining windows and binning blocks, all their sort tiles) and adds the
// listed segments and the tiles that reached their cut (rn[0]) to stats[0] /
// stats[1].
cudaError_t launch_phase_map(int phase, int m, const DepthCut *cut, const int *flag,
                             const int *tile_start, const int *blkpre, int bin_ranks, int *map,
                             const int *rn, unsigned long long *stats, cudaStream_t s);

// The first phase of the depth order: every segment (camera) of keys (z bits
// minus the near plane's bits, slot order) cut (cut, from prefix: < 0 the whole
// segment, 0 the default, > 0 that many ranks) and its first-phase ranks
// sorted by (key, oidx[seg_base + slot]); the slots in that order end in sv.
// map: the chunk's phase map, written here (phase 1). keys are read only; sk
// and the one-block sort's scratch scr_k / scr_v (the chunk's survivors each)
// are overwritten (sk and sv hold at least 4 elements past the chunk's
// survivors: the window pass copies 16-byte pieces); scratch other than keys
// keeps the keys for the second phase. tiles / tile_start: the chunk's SortTile
// table and per-segment tile prefix (tile_start[m] the total, on the device);
// seg_start: the segments' first positions; blkpre / bin_ranks: the binning
// blocks (for the map). Work buffers: count (DEPTH_BUCKETS uint32 per segment),
// win (SORT_TILE_KEYS / DEPTH_WINDOW entries of depth_window_bytes() per sort
// tile), big (big_cap entries of depth_big_bytes()), eq (eq_cap entries of
// depth_eq_bytes()), runs (run_cap entries of tie_run_bytes()), counters (3
// ints, zeroed by the call). grid: blocks of the per-tile kernels. Chunk
// positions must stay below 2^32.
cudaError_t launch_depth_order(uint32_t *keys, uint32_t *vals, uint32_t *sk, uint32_t *sv,
                               const uint32_t *oidx, const SortTile *tiles, const int *tile_start,
                               const long long *seg_start, int m, int grid, uint32_t *count,
                               void *win, void *big, long long big_cap, void *eq, long long eq_cap,
                               void *runs, long long run_cap, int *counters, DepthCut *cut,
                               int prefix, const int *blkpre, int bin_ranks, int *map,
                               uint32_t *scr_k, uint32_t *scr_v, cudaStream_t s);
// The second phase: the flagged segments' ranks [pos, count) (map: the phase-2
// map, written before). Same buffers as the first phase (whose scratch must not
// have been keys); counters: 3 more ints.
cudaError_t launch_depth_finish(const uint32_t *keys, uint32_t *scr_k, uint32_t *scr_v,
                                uint32_t *sk, uint32_t *sv, const uint32_t *oidx,
                                const SortTile *tiles, const long long *seg_start, int m, int grid,
                                uint32_t *count, void *win, void *big, long long big_cap, void *eq,
                                long long eq_cap, void *runs, long long run_cap, int *counters,
                                const DepthCut *cut, const int *map, cudaStream_t s);

// Motion-blur sub-frame poses (see k_blur.cu): out[j * n + i] for j < k.
// Intrinsics scaled by 1/f (see k_blur.cu).
cudaError_t launch_scale_intrinsics(const float *in, int n, float f, float *out, cudaStream_t s);

cudaError_t launch_blur_poses(const float *vm, const float *vel, int n, int k, float shutter,
                              float *out, cudaStream_t s);

// Device-side sizing of a chunk (see k_plan.cu).
cudaError_t launch_plan(CamInfo *cams, const int *counts, int m, int bin_ranks, long long cap_survivors,
                        int *blkpre, int *sorttiles, long long *segstart, long long *segcount,
                        SortTile *stiles, int2 *bintab, int *status, long long *need,
                        unsigned long long *survivors, unsigned long long *sticky,
                        cudaStream_t s);

// Super-tile bitmaps (one row of ceil(count/32) words per 64x64-pixel
// super-tile) and the rank-ordered tile rects.
// n_blocks blocks are launched; they loop over the device total blk_prefix[n_slots].
// bin_ranks: ranks per block, BIN_RANKS or BIN_RANKS_SMALL (the plan kernel's
// blocks must use the same value).
int bin_ranks_for(int n_super);
// phase 0: all ranks of every block; 1 / 2: the blocks of the phase map (map),
// the ranks before each camera's cut / all ranks (pairs counted from the cut).
cudaError_t launch_bin(const CamInfo *cams, const int *blk_prefix, const int2 *bintab, int n_slots,
                       int n_blocks,
                       int n_super, int bin_ranks, const uint2 *srect, const uint32_t *vals,
                       uint2 *rrect, uint32_t *bitmap, unsigned long long *n_isect,
                       const DepthCut *cut, int phase, const int *map, cudaStream_t s);
// The binning blocks of a phase map (phase 1 / 2, as launch_bin) that also
// compute each binned rank's record (the projection passes' arithmetic, from
// the scene rows of its Gaussian pos_of[oidx[seg_off + slot]]) into rec at the
// rank's position, and its rect.
cudaError_t launch_bin_rec(const CamInfo *cams, const int2 *bintab, int n_slots, int n_blocks,
                           int n_super, int bin_ranks, const SceneDev *scenes, const void *camtab,
                           ProjParams P, float ln_alpha_min, const uint32_t *oidx,
                           const uint32_t *vals, float4 *rec, uint2 *rrect, uint32_t *bitmap,
                           unsigned long long *n_isect, const DepthCut *cut, int phase,
                           const int *map, cudaStream_t s);

// Binning and compositing of a chunk in one persistent launch (k_composite.cu):
// 8 pixels per thread, binning items of BIN_RANKS_SMALL ranks (the plan must
// use that), cameras of at most persistent_max_super() super-tiles. head and
// bin_done ([n_slots] ints) must be zero at launch; a wait that gives up after
// wait_limit polls sets sticky[1] |= 2. grid = persistent_grid(comp_batch).
int persistent_max_super();
int persistent_grid(int comp_batch);
cudaError_t launch_bin_composite(const CamInfo *cams, const int *tile_prefix, int n_slots,
                                 int per_cam, int n_tiles, const float4 *rec, const uint32_t *vals,
                                 uint2 *rrect, CompParams C, float *rgb, float *depth,
                                 float *final_T, int comp_batch, const int *status,
                                 const int *blk_prefix, const int2 *bintab, const uint2 *srect,
                                 uint32_t *bitmap, unsigned long long *n_isect, int *head,
                                 int *bin_done, int wait_limit, int extra_need,
                                 unsigned long long *sticky, int grid, cudaStream_t s);

// tiles_per_block 1: one block per tile, pixels_per_thread 2, 4 or 8 (blocks of
// 128, 64 or 32 threads); tiles_per_block 4: one block of 4 warps per 2 x 2 quad
// of tiles (8 pixels per thread). tile_prefix / n_tiles count the blocks: tiles
// or quads per camera.
// The second phase's compositing work of a chunk (see DepthCut): a tile that
// still has live pixels when it reaches its camera's cut saves its state and
// flags the camera; when the saved list is full it is listed to be rendered
// again from rank 0 instead.
struct Resume {
    int *flag;       // [m] 1: the camera has tiles past its cut (zero before the first phase)
    int *n;          // [2] saved tiles, tiles to render again (zero before the first phase)
    int2 *saved;     // [cap] (camera, tile) of saved states
    float4 *state;   // [cap][12][32]: per lane its pixels' T, colour and depth sums and
                     // alpha thresholds
    int2 *again;     // [again_cap] (camera, tile) rendered again from rank 0
    int cap, again_cap;
};
constexpr int RESUME_STATE_F4 = 12 * 32;  // float4 of one saved tile state

// cut / R: the progressive order's first phase (8 pixels per thread, one tile
// per block, no counting only; R == nullptr: the whole order).
cudaError_t launch_composite(const CamInfo *cams, const int *tile_prefix, int n_slots,
                             int per_cam, int n_tiles, const float4 *rec, const uint32_t *vals,
                             const uint2 *rrect, const uint32_t *bitmap, CompParams C,
                             float *rgb, float *depth, float *final_T,
                             unsigned long long *stats, bool collect, int pixels_per_thread,
                             int tiles_per_block, int comp_batch, const int *status,
                             const DepthCut *cut, const Resume *R, cudaStream_t s);
// The second phase's compositing: the saved tiles resumed at their camera's cut,
// then the listed tiles rendered from rank 0 (8 pixels per thread, grid blocks).
cudaError_t launch_composite_resume(const CamInfo *cams, const float4 *rec, const uint32_t *vals,
                                    const uint2 *rrect, const uint32_t *bitmap, CompParams C,
                                    float *rgb, float *depth, float *final_T, int comp_batch,
                                    const int *status, const DepthCut *cut, const Resume &R,
                                    int grid, cudaStream_t s);

}  // namespace gsk
