// gs_api.cu -- the C ABI (include/gs.h): contexts, scenes and the batched
// render orchestration around the sm_103a kernels.
//
// A render call groups cameras by scene (so the projection kernel reads each
// Gaussian once per group of up to 32 cameras), splits them into chunks, and
// runs per chunk, in one stream:
//   project_mask -> scan_masks -> [read survivor counts] -> project_write
//   -> sort_segments -> bin -> composite
// The one host read per chunk sizes the workspace exactly (survivor slots,
// depth-rank records, tile bitmaps) and the grids of the later kernels.
// Workspace buffers grow on demand and are reused across calls.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "gs.h"
#include "gs_internal.cuh"

using namespace gsk;

namespace {

// Device statistics words: [0] evaluated pairs, [1] pairs with alpha >=
// alpha_min, [2] intersections, [3..5] warp iterations (all, box, blend), [6]
// survivors, [7] cameras of the progressive order's second phase, [8] tiles it
// resumed.
constexpr int N_STATS = 9;
// Stage events per chunk: project | first-phase depth order | binning |
// compositing | second-phase depth order | binning | compositing.
constexpr int EV_PER_CHUNK = 8;

// Blocks of the second phase's compositing launch: one resident wave of
// one-warp blocks (it loops over the resumed tiles).
int resume_grid() {
    static int grid[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (grid[dev] == 0) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
        grid[dev] = std::max(sms, 1) * 18;
    }
    return grid[dev];
}

struct DevBuf {
    void *p = nullptr;
    size_t cap = 0;
};

struct SceneSlot {
    bool live = false;
    void *storage = nullptr;
    SceneDev dev{};
};

struct PinBuf {
    void *p = nullptr;
    size_t cap = 0;
};

size_t dtype_size(int dt) { return dt == GS_F32 ? 4 : 2; }

float __uint_as_float_host(uint32_t u) {
    float f;
    memcpy(&f, &u, 4);
    return f;
}

}  // namespace

struct gs_context {
    gs_config cfg{};
    int device = 0;
    std::vector<SceneSlot> scenes;
    DevBuf d_scenes;
    // chunk workspace
    DevBuf masks, woff, counts, rec, keys, vals, tkeys, tvals, rrect, srect, bitmap;
    DevBuf tables, blkpre, segstart, segcount, stats, status, sorttiles, sorttab, bintab, camtab;
    DevBuf seg_tk, seg_tv, seg_tiles, seg_hist;  // gs_sort_segments' own scratch
    DevBuf oidx;  // per survivor slot: the Gaussian's caller index (depth tie-break)
    DevBuf dcount, dwin, dbig, deq;  // depth order: bucket counts, windows, listed windows / runs
    DevBuf ties, nruns;  // long runs of equal depth keys (list); per chunk 6 list counts
    // the progressive depth order: per camera its cut, the two phase maps, the
    // second phase's counts and camera flags, saved tile states, tiles to render again
    DevBuf dcut, pmap, prog, rsaved, rstate, ragain;
    long long cap_survivors = 0;  // survivors per chunk the workspace holds
    long long last_chunk_survivors = 0;  // largest chunk of the last render
    int workspace_gen = 0;        // bumped when a chunk-workspace buffer is reallocated
    // host-API staging
    DevBuf h_vm, h_in, h_rgb, h_depth, h_T;
    DevBuf blur_vm;  // motion-blur sub-frame poses
    PinBuf pin[2];
    gs_stats last{};
    bool stats_pending = false;
    std::string err;
    std::vector<cudaEvent_t> ev;  // time_stages: EV_PER_CHUNK events per chunk of the last call
    cudaStream_t copy_stream = nullptr;       // host entry point: device-to-host copies
    std::vector<cudaEvent_t> part_done;       // host / upsampled entry points: one event per part
    cudaStream_t up_stream = nullptr;         // upsampled entry point: the upsampler's stream
    cudaEvent_t up_done = nullptr;
    DevBuf lr_in, lr_rgb, lr_depth;           // upsampled entry point: quarter-resolution frames
    int ev_used = 0;              // chunks whose events the last call recorded
    // asynchronous calls: a sticky device word ([0] largest chunk need seen, [1]
    // a chunk did not fit), read back into pinned memory after every call and
    // looked at by a later call, gs_sync or gs_get_stats
    DevBuf sticky;
    PinBuf sticky_h;
    cudaEvent_t sticky_ev = nullptr;
    bool sticky_pending = false;
    PinBuf tab_pin[2];            // pinned staging of the per-call tables, two in turn
    cudaEvent_t tab_ev[2] = {nullptr, nullptr};  // after each one's last copy
    int tab_next = 0;
    cudaEvent_t done_ev = nullptr;  // end of the last render call's work (orders streams)
    bool done_valid = false;
    long long proven_gauss = 0;   // largest per-chunk Gaussian count a waited-for call rendered
    DevBuf pq;                    // persistent launch: queue head + per-camera binning counts
    int pgrid[4] = {0, 0, 0, 0};  // its resident grid, per compositing batch (32/64/96/128)
    int probe_extra = 0;          // timeout probe: camera 0 waits for items that never come
    int probe_limit = 0;          // timeout probe: polls before giving up (0: the default)
    int resume_cap = 0;           // saved tile states a chunk may hold (0: the workspace's)
};

struct gs_graph {
    gs_context *ctx = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    DevBuf tables;  // this graph's copy of the static per-camera tables
    int gen = 0;    // the context's workspace generation at capture
    int n_chunks = 0;
};

namespace {

gs_status fail(gs_context *ctx, gs_status s, const char *fmt, ...) {
    if (ctx) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof(buf), fmt, ap);
        va_end(ap);
        ctx->err = buf;
    }
    return s;
}

#define CKC(call)                                                                          \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(ctx, e_ == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA,   \
                        "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

#define CKS(expr)                        \
    do {                                 \
        gs_status s_ = (expr);           \
        if (s_ != GS_OK) return s_;      \
    } while (0)

// Grow a device buffer to at least `bytes` (contents are not preserved).
// Growth waits for the device so no queued kernel still uses the old memory.
gs_status grow(gs_context *ctx, DevBuf &b, size_t bytes) {
    if (bytes <= b.cap) return GS_OK;
    CKC(cudaDeviceSynchronize());
    if (b.p) CKC(cudaFree(b.p));
    b.p = nullptr;
    b.cap = 0;
    const size_t want = std::max<size_t>(bytes + bytes / 4, 256);
    CKC(cudaMalloc(&b.p, want));
    b.cap = want;
    return GS_OK;
}

gs_status grow_pinned(gs_context *ctx, PinBuf &b, size_t bytes) {
    if (bytes <= b.cap) return GS_OK;
    CKC(cudaDeviceSynchronize());
    if (b.p) CKC(cudaFreeHost(b.p));
    b.p = nullptr;
    b.cap = 0;
    const size_t want = std::max<size_t>(bytes + bytes / 4, 4096);
    CKC(cudaMallocHost(&b.p, want));
    b.cap = want;
    return GS_OK;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

gs_status sync_scene_table(gs_context *ctx) {
    std::vector<SceneDev> t(ctx->scenes.size());
    for (size_t i = 0; i < t.size(); ++i) t[i] = ctx->scenes[i].dev;
    if (t.empty()) return GS_OK;
    CKS(grow(ctx, ctx->d_scenes, t.size() * sizeof(SceneDev)));
    CKC(cudaMemcpy(ctx->d_scenes.p, t.data(), t.size() * sizeof(SceneDev), cudaMemcpyHostToDevice));
    return GS_OK;
}

enum Stage { UPTO_PROJECT = 0, UPTO_BIN = 1, UPTO_ALL = 2 };

struct RenderArgs {
    int n;
    const int32_t *scene_ids;  // host
    const float *vm, *in;      // device
    int W, H;                  // every camera's size when Ws == NULL
    const int32_t *Ws, *Hs;    // host per-camera sizes, or NULL
    const int64_t *pix_off;    // host per-camera first output pixel, or NULL (i * W * H)
    float *rgb, *depth, *T;    // device
    cudaStream_t st;
    Stage upto;
    float out_w = 1.0f;        // outputs = out_w * value (+ existing outputs if accumulate)
    int accumulate = 0;
    bool force_sync = false;   // wait for the status and re-render overflowed chunks here
    int cam_w(int i) const { return Ws ? Ws[i] : W; }
    int cam_h(int i) const { return Hs ? Hs[i] : H; }
    long long cam_pix(int i) const { return pix_off ? pix_off[i] : (long long)i * W * H; }
};

// Static per-call tables (host side), built once per call and uploaded in one copy.
struct ChunkPlan {
    int c0, m;            // first camera (in scene order) and cameras of the chunk
    int g0, n_groups;     // groups of the chunk in the group table
    int max_bx;           // projection blocks (x) for the largest scene of the chunk
    int tiles_total;      // compositing blocks of the chunk (tiles or 2x2 quads)
    int per_cam;          // compositing blocks of every camera when all are equal, else 0
    int max_sup;          // largest super-tile count of a camera of the chunk
    long long mask_words; // survival-mask words of the chunk
    long long n_gauss;    // sum over cameras of their scene sizes
    int sort_grid, bin_grid;
    int bin_ranks;        // depth ranks per binning block (from max_sup)
    int max_deg;          // largest SH degree of the chunk's scenes
    bool persistent;      // binning + compositing in one persistent launch
};

struct Plan {
    std::vector<ChunkPlan> chunks;
    int max_tiles = 0;               // compositing blocks of the largest chunk
    std::vector<CamInfo> cams;       // static fields, all chunks (chunk k at chunks[k].c0)
    std::vector<Group> groups;
    std::vector<int> tilepre;        // per chunk m + 1 entries, at c0 + k
    long long max_mask_words = 0, max_gauss = 0;
    int max_m = 0, max_sup = 1;
    size_t table_bytes = 0, off_groups = 0, off_tilepre = 0;
};

void build_plan(gs_context *ctx, const RenderArgs &a, Plan &P) {
    const gs_config &cfg = ctx->cfg;
    const int chunk_max = std::max(1, cfg.max_chunk_cameras);
    const int gmax = std::min(MAX_GROUP, std::max(1, cfg.camera_group));
    std::vector<int> order(a.n);
    for (int i = 0; i < a.n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return a.scene_ids[x] < a.scene_ids[y]; });
    P.cams.resize(a.n);
    P.tilepre.resize(a.n + (a.n + chunk_max - 1) / chunk_max + 1);
    int tp = 0;
    for (int c0 = 0; c0 < a.n; c0 += chunk_max) {
        ChunkPlan ch{};
        ch.c0 = c0;
        ch.m = std::min(chunk_max, a.n - c0);
        ch.g0 = (int)P.groups.size();
        long long sort_up = 0, bin_up = 0;
        for (int s = 0; s < ch.m; ++s) {
            const int user = order[c0 + s];
            const int sid = a.scene_ids[user];
            const SceneDev &sd = ctx->scenes[sid].dev;
            CamInfo &ci = P.cams[c0 + s];
            memset(&ci, 0, sizeof(ci));
            ci.user = user;
            ci.scene = sid;
            ci.W = a.cam_w(user);
            ci.H = a.cam_h(user);
            ci.TX = (ci.W + TILE - 1) / TILE;
            ci.TY = (ci.H + TILE - 1) / TILE;
            ci.pix_off = a.cam_pix(user);
            ci.tile_off = ch.tiles_total;
            P.tilepre[tp + s] = ch.tiles_total;
            // compositing blocks of this camera: tiles, or 2 x 2 quads of tiles
            const int blocks = cfg.tiles_per_block == 4 ? ((ci.TX + 1) / 2) * ((ci.TY + 1) / 2)
                                                        : ci.TX * ci.TY;
            ch.tiles_total += blocks;
            ch.per_cam = s == 0 ? blocks : (ch.per_cam == blocks ? blocks : 0);
            ch.max_sup = std::max(ch.max_sup,
                                  ((ci.TX + STILE - 1) / STILE) * ((ci.TY + STILE - 1) / STILE));
            ch.max_deg = std::max(ch.max_deg, sd.deg);
            ci.mask_off = ch.mask_words;
            ch.mask_words += (sd.n + 31) / 32;
            ch.n_gauss += sd.n;
            sort_up += (sd.n + SORT_TILE_KEYS - 1) / SORT_TILE_KEYS;
            bin_up += (sd.n + BIN_RANKS_SMALL - 1) / BIN_RANKS_SMALL;  // bound for either size
            const bool new_group = ch.n_groups == 0 || P.groups.back().scene != sid ||
                                   P.groups.back().ncam == gmax;
            if (new_group) {
                Group g{};
                g.scene = sid;
                g.slot0 = s;
                g.n = sd.n;
                P.groups.push_back(g);
                ch.n_groups++;
                ch.max_bx = std::max<long long>(ch.max_bx, (sd.n + PROJ_THREADS - 1) / PROJ_THREADS);
            }
            P.groups.back().ncam++;
        }
        P.tilepre[tp + ch.m] = ch.tiles_total;
        tp += ch.m + 1;
        ch.sort_grid = (int)std::max<long long>(1, std::min<long long>(sort_up, 32 * 1184));
        ch.persistent = cfg.persistent && cfg.pixels_per_thread == 8 && cfg.tiles_per_block == 1 &&
                        !cfg.count_pairs && ch.max_sup <= persistent_max_super();
        ch.bin_ranks = ch.persistent ? BIN_RANKS_SMALL : bin_ranks_for(ch.max_sup);
        if (ch.bin_ranks == BIN_RANKS) bin_up = (bin_up + 3) / 4;
        ch.bin_grid = (int)std::max<long long>(1, std::min<long long>(bin_up, 32 * 1184));
        P.max_mask_words = std::max(P.max_mask_words, ch.mask_words);
        P.max_gauss = std::max(P.max_gauss, ch.n_gauss);
        P.max_m = std::max(P.max_m, ch.m);
        P.max_sup = std::max(P.max_sup, ch.max_sup);
        P.max_tiles = std::max(P.max_tiles, ch.tiles_total);
        P.chunks.push_back(ch);
    }
    P.off_groups = align_up(P.cams.size() * sizeof(CamInfo), 256);
    P.off_tilepre = P.off_groups + align_up(std::max<size_t>(P.groups.size(), 1) * sizeof(Group), 256);
    P.table_bytes = P.off_tilepre + align_up(P.tilepre.size() * sizeof(int), 256);
}

// Workspace for a chunk of up to max_m cameras and cap_S survivors.
gs_status size_workspace(gs_context *ctx, const Plan &P) {
    const long long S = std::max<long long>(ctx->cap_survivors, 1);
    const size_t Sx = (size_t)S;
    const int m = std::max(P.max_m, 1);
    // a captured graph holds these addresses: any reallocation invalidates it
    DevBuf *held[] = {&ctx->masks,    &ctx->woff,     &ctx->counts,    &ctx->camtab, &ctx->rec,
                      &ctx->srect,    &ctx->rrect,    &ctx->keys,      &ctx->vals,   &ctx->tkeys,
                      &ctx->tvals,    &ctx->bitmap,   &ctx->dcount,    &ctx->sorttab,
                      &ctx->bintab,   &ctx->dwin,     &ctx->dbig,      &ctx->deq,
                      &ctx->blkpre,
                      &ctx->sorttiles,
                      &ctx->segstart, &ctx->segcount, &ctx->stats,     &ctx->status,
                      &ctx->oidx,     &ctx->ties,     &ctx->nruns,    &ctx->pq,
                      &ctx->dcut,     &ctx->pmap,     &ctx->prog,     &ctx->rsaved,
                      &ctx->rstate,   &ctx->ragain};
    // (compared by capacity: a reallocation may return the freed address)
    size_t before[sizeof(held) / sizeof(held[0])];
    for (size_t i = 0; i < sizeof(held) / sizeof(held[0]); ++i) before[i] = held[i]->cap;
    CKS(grow(ctx, ctx->masks, (size_t)std::max<long long>(P.max_mask_words, 1) * 4));
    CKS(grow(ctx, ctx->woff, (size_t)std::max<long long>(P.max_mask_words, 1) * 4));
    CKS(grow(ctx, ctx->counts, (size_t)m * sizeof(int)));
    CKS(grow(ctx, ctx->camtab, (size_t)m * cam_proj_bytes()));
    CKS(grow(ctx, ctx->rec, rec_bytes(S)));
    CKS(grow(ctx, ctx->srect, Sx * sizeof(uint2)));
    CKS(grow(ctx, ctx->rrect, Sx * sizeof(uint2)));
    // (+4 elements: the depth order's window pass copies 16-byte pieces, up to
    // 3 elements past a window's end)
    CKS(grow(ctx, ctx->keys, Sx * 4));
    CKS(grow(ctx, ctx->vals, (Sx + 4) * 4));
    CKS(grow(ctx, ctx->tkeys, (Sx + 4) * 4));
    CKS(grow(ctx, ctx->tvals, (Sx + 4) * 4));
    CKS(grow(ctx, ctx->oidx, Sx * 4));
    CKS(grow(ctx, ctx->ties, (Sx / 33 + 2) * tie_run_bytes()));
    CKS(grow(ctx, ctx->nruns, 6 * (P.chunks.size() + 1) * sizeof(int)));
    CKS(grow(ctx, ctx->pq, (size_t)(m + 2) * sizeof(int)));
    // bounds implied by S: bitmap words <= max_sup * (S/32 + m), sort tiles <= S/2048 + m
    CKS(grow(ctx, ctx->bitmap, (size_t)P.max_sup * (Sx / 32 + m + 1) * 4));
    const size_t sort_tiles = Sx / SORT_TILE_KEYS + m + 1;
    CKS(grow(ctx, ctx->sorttab, sort_tiles * sizeof(SortTile)));
    CKS(grow(ctx, ctx->dcount, (size_t)m * DEPTH_BUCKETS * 4));
    const size_t windows = sort_tiles * (SORT_TILE_KEYS / DEPTH_WINDOW);
    CKS(grow(ctx, ctx->dwin, windows * depth_window_bytes()));
    CKS(grow(ctx, ctx->dbig, windows * depth_big_bytes()));
    // runs of equal depth keys: about one per 500 survivors on the full-size
    // workloads; a window orders its runs itself when the list is full
    CKS(grow(ctx, ctx->deq, (Sx / 64 + 64) * depth_eq_bytes()));
    CKS(grow(ctx, ctx->bintab, (Sx / BIN_RANKS_SMALL + m + 1) * sizeof(int2)));
    CKS(grow(ctx, ctx->blkpre, (size_t)(m + 1) * sizeof(int)));
    CKS(grow(ctx, ctx->sorttiles, (size_t)(m + 1) * sizeof(int)));
    CKS(grow(ctx, ctx->segstart, (size_t)m * sizeof(long long)));
    CKS(grow(ctx, ctx->segcount, (size_t)m * sizeof(long long)));
    CKS(grow(ctx, ctx->stats, N_STATS * sizeof(unsigned long long)));
    CKS(grow(ctx, ctx->dcut, (size_t)m * sizeof(DepthCut)));
    CKS(grow(ctx, ctx->pmap, 2 * phase_map_ints(m) * sizeof(int)));
    CKS(grow(ctx, ctx->prog, (size_t)(m + 2) * sizeof(int)));
    // saved tile states: a sixteenth of the largest chunk's tiles (more tiles than
    // that reaching their camera's cut are rendered again from rank 0 instead)
    const size_t tiles = (size_t)std::max(P.max_tiles, 1);
    const size_t rcap = std::max<size_t>(1024, tiles / 16);
    CKS(grow(ctx, ctx->rsaved, rcap * sizeof(int2)));
    CKS(grow(ctx, ctx->rstate, rcap * RESUME_STATE_F4 * sizeof(float4)));
    CKS(grow(ctx, ctx->ragain, tiles * sizeof(int2)));
    CKS(grow(ctx, ctx->status, (P.chunks.size() + 2) * sizeof(long long)));
    for (size_t i = 0; i < sizeof(held) / sizeof(held[0]); ++i)
        if (held[i]->cap != before[i]) {
            ctx->workspace_gen++;
            break;
        }
    return GS_OK;
}

// Enqueue the whole render on `st` (no host synchronisation). `tab` holds the
// uploaded static tables of P. With events != NULL, EV_PER_CHUNK events per
// chunk are recorded around the stages.
gs_status enqueue_render(gs_context *ctx, const RenderArgs &a, const Plan &P, char *tab,
                         cudaStream_t st, cudaEvent_t *events,
                         const std::vector<char> *only = nullptr) {
    const gs_config &cfg = ctx->cfg;
    const ProjParams PP{cfg.near_plane, cfg.dilation, cfg.guard_band, cfg.sigma_cull};
    const CompParams C{std::log2(cfg.alpha_min),
                       cfg.alpha_max,
                       cfg.T_min,
                       std::log2(cfg.alpha_max) - 2e-3f,
                       {cfg.background[0], cfg.background[1], cfg.background[2]},
                       a.out_w,
                       a.accumulate};
    CamInfo *cams_all = (CamInfo *)tab;
    Group *groups_all = (Group *)(tab + P.off_groups);
    int *tilepre_all = (int *)(tab + P.off_tilepre);
    long long *need = (long long *)ctx->status.p;               // [0]: largest chunk
    int *status_all = (int *)((long long *)ctx->status.p + 1);  // [k]: chunk k overflowed
    unsigned long long *stats = (unsigned long long *)ctx->stats.p;
    // records: the render writes fields a, b, c; the debug stages also d
    float4 *recs = (float4 *)ctx->rec.p;
    const int with_d = a.upto != UPTO_ALL;
    int tp = 0;
    for (size_t k = 0; k < P.chunks.size(); ++k) {
        const ChunkPlan &ch = P.chunks[k];
        CamInfo *cams = cams_all + ch.c0;
        const Group *groups = groups_all + ch.g0;
        const int *tilepre = tilepre_all + tp;
        int *status = status_all + k;
        tp += ch.m + 1;
        if (only && !(*only)[k]) continue;
        cudaEvent_t *E = events ? events + EV_PER_CHUNK * k : nullptr;
        // the progressive depth order (see DepthCut) with the separate launches of
        // the 8-pixel, one-tile layout; the whole order otherwise
        const bool prog = cfg.depth_prefix >= 0 && a.upto == UPTO_ALL && !ch.persistent &&
                          cfg.pixels_per_thread == 8 && cfg.tiles_per_block == 1 &&
                          !cfg.count_pairs;
        DepthCut *cut = (DepthCut *)ctx->dcut.p;
        int *map1 = (int *)ctx->pmap.p, *map2 = map1 + phase_map_ints(ch.m);
        int *prog_n = (int *)ctx->prog.p;  // [2] counts, then [m] flags
        // the one-block sort's scratch: the slot-order rects' array (unused by the
        // progressive order), so that the keys stay for its second phase
        const size_t n_slots_ws = ctx->srect.cap / sizeof(uint2);
        uint32_t *scr_k = prog ? (uint32_t *)ctx->srect.p : (uint32_t *)ctx->keys.p;
        uint32_t *scr_v = prog ? (uint32_t *)ctx->srect.p + n_slots_ws : (uint32_t *)ctx->vals.p;
        const float ln_amin = std::log(cfg.alpha_min);
        Resume R{prog_n + 2, prog_n, (int2 *)ctx->rsaved.p, (float4 *)ctx->rstate.p,
                 (int2 *)ctx->ragain.p,
                 (int)std::min(ctx->rsaved.cap / sizeof(int2),
                               ctx->rstate.cap / (RESUME_STATE_F4 * sizeof(float4))),
                 (int)(ctx->ragain.cap / sizeof(int2))};
        if (ctx->resume_cap > 0) R.cap = std::min(R.cap, ctx->resume_cap);
        if (E) CKC(cudaEventRecord(E[0], st));
        CKC(launch_cam_setup(cams, ch.m, a.vm, a.in, PP, ctx->camtab.p, st));
        CKC(launch_project_mask(groups, ch.n_groups, ch.max_bx, (const SceneDev *)ctx->d_scenes.p,
                                cams, ctx->camtab.p, PP, (uint32_t *)ctx->masks.p, st));
        CKC(launch_scan_masks(cams, (const SceneDev *)ctx->d_scenes.p, ch.m,
                              (const uint32_t *)ctx->masks.p, (uint32_t *)ctx->woff.p,
                              (int *)ctx->counts.p, st));
        CKC(launch_plan(cams, (const int *)ctx->counts.p, ch.m, ch.bin_ranks, ctx->cap_survivors,
                        (int *)ctx->blkpre.p, (int *)ctx->sorttiles.p, (long long *)ctx->segstart.p,
                        (long long *)ctx->segcount.p, (SortTile *)ctx->sorttab.p,
                        (int2 *)ctx->bintab.p, status, need, stats + 6,
                        (unsigned long long *)ctx->sticky.p, st));
        if (prog)  // keys only: the records of the ranks read come from the binning pass
            CKC(launch_project_keys(groups, ch.n_groups, ch.max_bx,
                                    (const SceneDev *)ctx->d_scenes.p, cams, ctx->camtab.p, PP,
                                    (const uint32_t *)ctx->masks.p, (const uint32_t *)ctx->woff.p,
                                    (uint32_t *)ctx->keys.p, (uint32_t *)ctx->oidx.p, status, st));
        else
            CKC(launch_project_write(groups, ch.n_groups, ch.max_bx,
                                     (const SceneDev *)ctx->d_scenes.p, cams, ctx->camtab.p, PP,
                                     (const uint32_t *)ctx->masks.p, (const uint32_t *)ctx->woff.p,
                                     recs, with_d, (uint2 *)ctx->srect.p, (uint32_t *)ctx->keys.p,
                                     (uint32_t *)ctx->oidx.p, std::log(cfg.alpha_min), status,
                                     ch.max_deg, st));
        if (E) CKC(cudaEventRecord(E[1], st));
        if (a.upto == UPTO_PROJECT) break;
        // every camera's survivors in (depth, caller index) order, into tkeys / tvals
        CKC(launch_depth_order((uint32_t *)ctx->keys.p, (uint32_t *)ctx->vals.p,
                               (uint32_t *)ctx->tkeys.p, (uint32_t *)ctx->tvals.p,
                               (const uint32_t *)ctx->oidx.p, (const SortTile *)ctx->sorttab.p,
                               (const int *)ctx->sorttiles.p, (const long long *)ctx->segstart.p,
                               ch.m, ch.sort_grid, (uint32_t *)ctx->dcount.p, ctx->dwin.p,
                               ctx->dbig.p, (long long)(ctx->dbig.cap / depth_big_bytes()),
                               ctx->deq.p, (long long)(ctx->deq.cap / depth_eq_bytes()),
                               ctx->ties.p, (long long)(ctx->ties.cap / tie_run_bytes()),
                               (int *)ctx->nruns.p + 6 * k, cut, prog ? cfg.depth_prefix : -1,
                               (const int *)ctx->blkpre.p, ch.bin_ranks, map1, scr_k, scr_v, st));
        if (E) CKC(cudaEventRecord(E[2], st));
        const bool persist = ch.persistent && a.upto == UPTO_ALL;
        if (prog)
            CKC(launch_bin_rec(cams, (const int2 *)ctx->bintab.p, ch.m, ch.bin_grid, ch.max_sup,
                               ch.bin_ranks, (const SceneDev *)ctx->d_scenes.p, ctx->camtab.p, PP,
                               ln_amin, (const uint32_t *)ctx->oidx.p,
                               (const uint32_t *)ctx->tvals.p, recs, (uint2 *)ctx->rrect.p,
                               (uint32_t *)ctx->bitmap.p, stats + 2, cut, 1, map1, st));
        else if (!persist)
            CKC(launch_bin(cams, (const int *)ctx->blkpre.p, (const int2 *)ctx->bintab.p, ch.m,
                           ch.bin_grid, ch.max_sup,
                           ch.bin_ranks, (const uint2 *)ctx->srect.p, (const uint32_t *)ctx->tvals.p,
                           (uint2 *)ctx->rrect.p, (uint32_t *)ctx->bitmap.p, stats + 2, cut, 0,
                           map1, st));
        if (E) CKC(cudaEventRecord(E[3], st));
        if (a.upto == UPTO_BIN) break;
        if (persist) {
            // binning and compositing in one persistent launch (its time counts as
            // compositing): queue head and per-camera binning counts start at zero
            const int ci = cfg.comp_batch == 32 ? 0 : cfg.comp_batch == 96 ? 2
                         : cfg.comp_batch == 128 ? 3 : 1;
            if (ctx->pgrid[ci] <= 0) ctx->pgrid[ci] = persistent_grid(cfg.comp_batch);
            if (ctx->pgrid[ci] <= 0) return fail(ctx, GS_ERR_CUDA, "persistent grid size query failed");
            int *pq = (int *)ctx->pq.p;
            CKC(cudaMemsetAsync(pq, 0, (size_t)(ch.m + 1) * sizeof(int), st));
            CKC(launch_bin_composite(cams, tilepre, ch.m, ch.per_cam, ch.tiles_total, recs,
                                     (const uint32_t *)ctx->tvals.p, (uint2 *)ctx->rrect.p, C,
                                     a.rgb, a.depth, a.T, cfg.comp_batch, status,
                                     (const int *)ctx->blkpre.p, (const int2 *)ctx->bintab.p,
                                     (const uint2 *)ctx->srect.p, (uint32_t *)ctx->bitmap.p,
                                     stats + 2, pq, pq + 1,
                                     ctx->probe_limit > 0 ? ctx->probe_limit : (1 << 18),
                                     ctx->probe_extra, (unsigned long long *)ctx->sticky.p,
                                     ctx->pgrid[ci], st));
        } else {
            if (prog) CKC(cudaMemsetAsync(prog_n, 0, (size_t)(ch.m + 2) * sizeof(int), st));
            CKC(launch_composite(cams, tilepre, ch.m, ch.per_cam, ch.tiles_total, recs,
                                 (const uint32_t *)ctx->tvals.p, (const uint2 *)ctx->rrect.p,
                                 (const uint32_t *)ctx->bitmap.p, C, a.rgb, a.depth, a.T, stats,
                                 cfg.count_pairs != 0, cfg.pixels_per_thread, cfg.tiles_per_block,
                                 cfg.comp_batch, status, cut, prog ? &R : nullptr, st));
        }
        if (E) CKC(cudaEventRecord(E[4], st));
        if (prog) {
            // the second phase: the flagged cameras' remaining ranks, their tiles resumed
            CKC(launch_phase_map(2, ch.m, cut, R.flag, (const int *)ctx->sorttiles.p,
                                 (const int *)ctx->blkpre.p, ch.bin_ranks, map2, R.n, stats + 7, st));
            CKC(launch_depth_finish((const uint32_t *)ctx->keys.p, scr_k, scr_v,
                                    (uint32_t *)ctx->tkeys.p, (uint32_t *)ctx->tvals.p,
                                    (const uint32_t *)ctx->oidx.p, (const SortTile *)ctx->sorttab.p,
                                    (const long long *)ctx->segstart.p, ch.m, ch.sort_grid,
                                    (uint32_t *)ctx->dcount.p, ctx->dwin.p, ctx->dbig.p,
                                    (long long)(ctx->dbig.cap / depth_big_bytes()), ctx->deq.p,
                                    (long long)(ctx->deq.cap / depth_eq_bytes()), ctx->ties.p,
                                    (long long)(ctx->ties.cap / tie_run_bytes()),
                                    (int *)ctx->nruns.p + 6 * k + 3, cut, map2, st));
            if (E) CKC(cudaEventRecord(E[5], st));
            // (the flagged cameras only: usually little or no work, one wave of
            // resident blocks looping over the phase map)
            CKC(launch_bin_rec(cams, (const int2 *)ctx->bintab.p, ch.m, ch.bin_grid, ch.max_sup,
                               ch.bin_ranks, (const SceneDev *)ctx->d_scenes.p, ctx->camtab.p, PP,
                               ln_amin, (const uint32_t *)ctx->oidx.p,
                               (const uint32_t *)ctx->tvals.p, recs, (uint2 *)ctx->rrect.p,
                               (uint32_t *)ctx->bitmap.p, stats + 2, cut, 2, map2, st));
            if (E) CKC(cudaEventRecord(E[6], st));
            CKC(launch_composite_resume(cams, recs, (const uint32_t *)ctx->tvals.p,
                                        (const uint2 *)ctx->rrect.p, (const uint32_t *)ctx->bitmap.p,
                                        C, a.rgb, a.depth, a.T, cfg.comp_batch, status, cut, R,
                                        resume_grid(), st));
        } else if (E) {
            CKC(cudaEventRecord(E[5], st));
            CKC(cudaEventRecord(E[6], st));
        }
        if (E) CKC(cudaEventRecord(E[7], st));
    }
    return GS_OK;
}

gs_status upload_tables(gs_context *ctx, const Plan &P, DevBuf &dst, cudaStream_t st) {
    CKS(grow_pinned(ctx, ctx->pin[0], P.table_bytes));
    CKS(grow(ctx, dst, P.table_bytes));
    char *h = (char *)ctx->pin[0].p;
    memcpy(h, P.cams.data(), P.cams.size() * sizeof(CamInfo));
    if (!P.groups.empty()) memcpy(h + P.off_groups, P.groups.data(), P.groups.size() * sizeof(Group));
    memcpy(h + P.off_tilepre, P.tilepre.data(), P.tilepre.size() * sizeof(int));
    CKC(cudaMemcpyAsync(dst.p, h, P.table_bytes, cudaMemcpyHostToDevice, st));
    return GS_OK;
}

// The per-call tables through one of two pinned staging buffers in turn: a
// buffer is refilled only after its previous copy has run, so an asynchronous
// call never overwrites tables a queued copy still reads.
gs_status upload_tables_ring(gs_context *ctx, const Plan &P, cudaStream_t st) {
    const int i = ctx->tab_next;
    ctx->tab_next ^= 1;
    if (!ctx->tab_ev[i]) CKC(cudaEventCreateWithFlags(&ctx->tab_ev[i], cudaEventDisableTiming));
    CKC(cudaEventSynchronize(ctx->tab_ev[i]));
    CKS(grow_pinned(ctx, ctx->tab_pin[i], P.table_bytes));
    CKS(grow(ctx, ctx->tables, P.table_bytes));
    char *h = (char *)ctx->tab_pin[i].p;
    memcpy(h, P.cams.data(), P.cams.size() * sizeof(CamInfo));
    if (!P.groups.empty()) memcpy(h + P.off_groups, P.groups.data(), P.groups.size() * sizeof(Group));
    memcpy(h + P.off_tilepre, P.tilepre.data(), P.tilepre.size() * sizeof(int));
    CKC(cudaMemcpyAsync(ctx->tables.p, h, P.table_bytes, cudaMemcpyHostToDevice, st));
    CKC(cudaEventRecord(ctx->tab_ev[i], st));
    return GS_OK;
}

// The sticky status of earlier calls, from its last read-back (waiting for it
// only when `wait`). The workspace plan grows to the largest chunk seen; a
// chunk that did not fit is reported once (GS_ERR_CAPACITY) and the device
// flag cleared on `st`.
gs_status poll_sticky(gs_context *ctx, bool wait, cudaStream_t st) {
    if (!ctx->sticky_pending) return GS_OK;
    if (wait) {
        CKC(cudaEventSynchronize(ctx->sticky_ev));
    } else {
        const cudaError_t q = cudaEventQuery(ctx->sticky_ev);
        if (q == cudaErrorNotReady) return GS_OK;
        CKC(q);
    }
    ctx->sticky_pending = false;
    const unsigned long long *h = (const unsigned long long *)ctx->sticky_h.p;
    const long long need = (long long)h[0];
    ctx->last_chunk_survivors = std::max(ctx->last_chunk_survivors, need);
    if (h[1] & 2ull) {  // a persistent launch's bounded wait gave up
        CKC(cudaMemsetAsync((unsigned long long *)ctx->sticky.p + 1, 0, 8, st));
        if (h[1] & 1ull)
            ctx->cap_survivors = std::max(ctx->cap_survivors, need + need / 8 + 1024);
        return fail(ctx, GS_ERR_TIMEOUT,
                    "a render call's persistent binning + compositing launch gave up waiting "
                    "for a camera's binning: some of its tiles are not written");
    }
    if (h[1]) {
        ctx->cap_survivors = std::max(ctx->cap_survivors, need + need / 8 + 1024);
        CKC(cudaMemsetAsync((unsigned long long *)ctx->sticky.p + 1, 0, 8, st));
        return fail(ctx, GS_ERR_CAPACITY,
                    "an earlier render call had a chunk of %lld survivors, more than the "
                    "workspace held: its images are not valid (the workspace has grown; render "
                    "again)",
                    need);
    }
    return GS_OK;
}

gs_status render_impl(gs_context *ctx, const RenderArgs &a) {
    Plan P;
    build_plan(ctx, a, P);
    if (ctx->cap_survivors <= 0)  // configured, else a third of the Gaussians a chunk sees
        ctx->cap_survivors = ctx->cfg.workspace_survivors > 0
                                 ? ctx->cfg.workspace_survivors
                                 : std::max<long long>(1 << 20, P.max_gauss / 3);
    const bool timing = ctx->cfg.time_stages != 0;
    if (timing)
        while (ctx->ev.size() < EV_PER_CHUNK * P.chunks.size()) {
            cudaEvent_t e;
            CKC(cudaEventCreate(&e));
            ctx->ev.push_back(e);
        }
    if (!ctx->sticky.p) {
        CKS(grow(ctx, ctx->sticky, 2 * sizeof(unsigned long long)));
        CKC(cudaMemset(ctx->sticky.p, 0, 2 * sizeof(unsigned long long)));
        CKS(grow_pinned(ctx, ctx->sticky_h, 2 * sizeof(unsigned long long)));
        CKC(cudaEventCreateWithFlags(&ctx->sticky_ev, cudaEventDisableTiming));
        CKC(cudaEventCreateWithFlags(&ctx->done_ev, cudaEventDisableTiming));
    }
    // an error an earlier asynchronous call left is reported by this one
    CKS(poll_sticky(ctx, false, a.st));
    if (ctx->done_valid) CKC(cudaStreamWaitEvent(a.st, ctx->done_ev, 0));  // calls in order
    const size_t status_bytes = sizeof(long long) + P.chunks.size() * sizeof(int);
    // A call whose chunks see more Gaussians than any call before on this context
    // waits for its status and re-renders in place: it sizes the workspace. Later
    // calls of that size only enqueue.
    const bool sync = ctx->cfg.sync_errors != 0 || a.force_sync || P.max_gauss > ctx->proven_gauss;
    std::vector<char> redo;
    for (int attempt = 0; attempt < 2; ++attempt) {
        CKS(size_workspace(ctx, P));
        CKS(upload_tables_ring(ctx, P, a.st));
        if (attempt == 0) CKC(cudaMemsetAsync(ctx->stats.p, 0, N_STATS * sizeof(unsigned long long), a.st));
        CKC(cudaMemsetAsync(ctx->status.p, 0, status_bytes, a.st));
        // the second pass renders only the chunks that overflowed (the others are
        // final, and may have been accumulated into the outputs)
        CKS(enqueue_render(ctx, a, P, (char *)ctx->tables.p, a.st,
                           timing && attempt == 0 ? ctx->ev.data() : nullptr,
                           attempt ? &redo : nullptr));
        if (!sync) {
            // no host wait: the sticky word is read back for a later call
            CKC(cudaMemcpyAsync(ctx->sticky_h.p, ctx->sticky.p, 2 * sizeof(unsigned long long),
                                cudaMemcpyDeviceToHost, a.st));
            CKC(cudaEventRecord(ctx->sticky_ev, a.st));
            ctx->sticky_pending = true;
            break;
        }
        CKS(grow_pinned(ctx, ctx->pin[1], status_bytes + 64));
        char *hs = (char *)ctx->pin[1].p;
        CKC(cudaMemcpyAsync(hs, ctx->status.p, status_bytes, cudaMemcpyDeviceToHost, a.st));
        CKC(cudaStreamSynchronize(a.st));
        const long long need = *(long long *)hs;
        const int *st = (const int *)(hs + sizeof(long long));
        ctx->last_chunk_survivors = std::max(attempt ? ctx->last_chunk_survivors : 0LL, need);
        redo.assign(P.chunks.size(), 0);
        bool any = false;
        for (size_t k = 0; k < P.chunks.size(); ++k)
            if (st[k]) redo[k] = 1, any = true;
        if (!any) break;
        if (attempt == 1)
            return fail(ctx, GS_ERR_CAPACITY, "workspace overflow after resizing (%lld survivors)",
                        need);
        ctx->cap_survivors = need + need / 8 + 1024;  // exact need plus headroom; render again
        // re-rendered here: not an error for a later call
        CKC(cudaMemsetAsync((unsigned long long *)ctx->sticky.p + 1, 0, 8, a.st));
    }
    if (sync) {  // this call's persistent waits: read the sticky word now
        CKS(grow_pinned(ctx, ctx->pin[1], 64));
        unsigned long long *hs = (unsigned long long *)ctx->pin[1].p;
        CKC(cudaMemcpyAsync(hs, ctx->sticky.p, 2 * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, a.st));
        CKC(cudaStreamSynchronize(a.st));
        if (hs[1] & 2ull) {
            CKC(cudaMemsetAsync((unsigned long long *)ctx->sticky.p + 1, 0, 8, a.st));
            CKC(cudaEventRecord(ctx->done_ev, a.st));
            ctx->done_valid = true;
            return fail(ctx, GS_ERR_TIMEOUT,
                        "the persistent binning + compositing launch gave up waiting for a "
                        "camera's binning: some of its tiles are not written");
        }
    }
    CKC(cudaEventRecord(ctx->done_ev, a.st));
    ctx->done_valid = true;
    if (sync) ctx->proven_gauss = std::max(ctx->proven_gauss, P.max_gauss);
    gs_stats stt{};
    stt.n_cameras = a.n;
    stt.n_chunks = (int)P.chunks.size();
    ctx->last = stt;
    ctx->ev_used = timing ? (int)P.chunks.size() : 0;
    ctx->stats_pending = true;
    return GS_OK;
}

gs_status validate(gs_context *ctx, int n, const int32_t *scene_ids, const void *vm,
                   const void *in, int W, int H, const void *rgb, const void *depth,
                   bool need_out) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    if (n < 0) return fail(ctx, GS_ERR_INVALID_ARG, "n_cams < 0");
    if (n == 0) return GS_OK;
    if (!scene_ids || !vm || !in) return fail(ctx, GS_ERR_INVALID_ARG, "NULL camera array");
    if (need_out && (!rgb || !depth)) return fail(ctx, GS_ERR_INVALID_ARG, "NULL output array");
    if (W < 1 || H < 1 || W > 65535 || H > 65535)
        return fail(ctx, GS_ERR_INVALID_ARG, "image size %dx%d out of range", W, H);
    const long long tiles = (long long)((W + 15) / 16) * ((H + 15) / 16);
    if (tiles > MAX_TILES)
        return fail(ctx, GS_ERR_CAPACITY, "%lld tiles per camera > %d", tiles, MAX_TILES);
    (void)tiles;
    for (int i = 0; i < n; ++i) {
        const int s = scene_ids[i];
        if (s < 0 || s >= (int)ctx->scenes.size() || !ctx->scenes[s].live)
            return fail(ctx, GS_ERR_NOT_FOUND, "camera %d: unknown scene id %d", i, s);
    }
    return GS_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI

extern "C" {

int32_t gs_abi_version(void) { return 6; }

const char *gs_status_string(gs_status s) {
    switch (s) {
        case GS_OK: return "ok";
        case GS_ERR_INVALID_ARG: return "invalid argument";
        case GS_ERR_CUDA: return "CUDA error";
        case GS_ERR_OOM: return "out of memory";
        case GS_ERR_CAPACITY: return "capacity exceeded";
        case GS_ERR_TIMEOUT: return "device wait timed out";
        case GS_ERR_NOT_FOUND: return "not found";
    }
    return "unknown status";
}

gs_status gs_config_default(gs_config *out) {
    if (!out) return GS_ERR_INVALID_ARG;
    memset(out, 0, sizeof(*out));
    out->near_plane = 0.2f;
    out->dilation = 0.3f;
    out->guard_band = 1.3f;
    out->sigma_cull = 3.0f;
    out->alpha_min = 1.0f / 255.0f;
    out->alpha_max = 0.99f;
    out->T_min = 1e-4f;
    out->max_chunk_cameras = 2048;
    out->camera_group = 128;
    out->count_pairs = 0;
    out->time_stages = 0;
    out->pixels_per_thread = 8;
    out->tiles_per_block = 1;
    out->comp_batch = COMP_BATCH_DEFAULT;
    out->sync_errors = 0;
    out->depth_prefix = 0;
    return GS_OK;
}

// Checks a configuration and fills its defaults (0 fields that mean a default).
static bool check_config(gs_config &c) {
    if (!(c.near_plane > 0.0f) || !(c.dilation >= 0.0f) || !(c.sigma_cull > 0.0f) ||
        !(c.alpha_min > 0.0f) || !(c.alpha_max > 0.0f && c.alpha_max < 1.0f) ||
        !(c.T_min > 0.0f && c.T_min < 1.0f) || c.max_chunk_cameras < 1 || c.camera_group < 1 ||
        c.camera_group > MAX_GROUP || !(c.guard_band >= 1.0f) || c.workspace_survivors < 0 ||
        (c.pixels_per_thread != 2 && c.pixels_per_thread != 4 && c.pixels_per_thread != 8) ||
        (c.tiles_per_block != 0 && c.tiles_per_block != 1 && c.tiles_per_block != 4) ||
        (c.comp_batch != 0 && c.comp_batch != 32 && c.comp_batch != 64 && c.comp_batch != 96 &&
         c.comp_batch != 128) ||
        (c.sync_errors != 0 && c.sync_errors != 1) || (c.persistent != 0 && c.persistent != 1) ||
        c.depth_prefix < -1)
        return false;
    // 0 (a zero-initialised config) means 1; quads use 8 pixels per thread
    if (c.tiles_per_block == 0 || c.pixels_per_thread != 8) c.tiles_per_block = 1;
    if (c.comp_batch == 0) c.comp_batch = COMP_BATCH_DEFAULT;
    return true;
}

gs_status gs_context_create(const gs_config *cfg, int32_t device, gs_context **out) {
    if (!out) return GS_ERR_INVALID_ARG;
    *out = nullptr;
    gs_config c;
    if (cfg)
        c = *cfg;
    else
        gs_config_default(&c);
    if (!check_config(c)) return GS_ERR_INVALID_ARG;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
        return GS_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return GS_ERR_CUDA;
    gs_context *ctx = new gs_context();
    ctx->cfg = c;
    ctx->device = device;
    *out = ctx;
    return GS_OK;
}

gs_status gs_context_set_config(gs_context *ctx, const gs_config *cfg) {
    if (!ctx || !cfg) return GS_ERR_INVALID_ARG;
    gs_config c = *cfg;
    if (!check_config(c)) return fail(ctx, GS_ERR_INVALID_ARG, "invalid configuration");
    const gs_config &o = ctx->cfg;
    if (c.near_plane != o.near_plane || c.dilation != o.dilation || c.guard_band != o.guard_band ||
        c.sigma_cull != o.sigma_cull || c.alpha_min != o.alpha_min || c.alpha_max != o.alpha_max ||
        c.T_min != o.T_min || c.background[0] != o.background[0] ||
        c.background[1] != o.background[1] || c.background[2] != o.background[2])
        return fail(ctx, GS_ERR_INVALID_ARG, "the rasteriser constants of a context are fixed");
    CKC(cudaSetDevice(ctx->device));
    if (ctx->done_valid) CKC(cudaEventSynchronize(ctx->done_ev));
    ctx->cfg = c;
    return GS_OK;
}

void gs_context_destroy(gs_context *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto &s : ctx->scenes)
        if (s.storage) cudaFree(s.storage);
    DevBuf *bufs[] = {&ctx->d_scenes, &ctx->masks, &ctx->woff,    &ctx->counts,  &ctx->rec,
                      &ctx->keys,     &ctx->vals,  &ctx->tkeys,   &ctx->tvals,   &ctx->rrect, &ctx->srect,
                      &ctx->bitmap,   &ctx->tables, &ctx->status, &ctx->blkpre,
                      &ctx->segstart, &ctx->segcount, &ctx->stats, &ctx->h_vm,   &ctx->h_in,
                      &ctx->sorttiles, &ctx->seg_tk, &ctx->seg_tv, &ctx->seg_tiles, &ctx->seg_hist,
                      &ctx->sorttab, &ctx->bintab, &ctx->camtab, &ctx->blur_vm,
                      &ctx->oidx,     &ctx->dcount, &ctx->dwin,   &ctx->dbig,    &ctx->deq,
                      &ctx->ties,
                      &ctx->nruns,    &ctx->pq,
                      &ctx->dcut,     &ctx->pmap,   &ctx->prog,   &ctx->rsaved,  &ctx->rstate,
                      &ctx->ragain,
                      &ctx->h_rgb,    &ctx->h_depth, &ctx->h_T};
    for (DevBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    for (auto &p : ctx->pin)
        if (p.p) cudaFreeHost(p.p);
    for (auto &p : ctx->tab_pin)
        if (p.p) cudaFreeHost(p.p);
    if (ctx->sticky_h.p) cudaFreeHost(ctx->sticky_h.p);
    if (ctx->sticky.p) cudaFree(ctx->sticky.p);
    for (auto &e : ctx->tab_ev)
        if (e) cudaEventDestroy(e);
    if (ctx->sticky_ev) cudaEventDestroy(ctx->sticky_ev);
    if (ctx->done_ev) cudaEventDestroy(ctx->done_ev);
    for (auto &e : ctx->ev) cudaEventDestroy(e);
    for (auto &e : ctx->part_done) cudaEventDestroy(e);
    if (ctx->copy_stream) cudaStreamDestroy(ctx->copy_stream);
    if (ctx->up_stream) cudaStreamDestroy(ctx->up_stream);
    if (ctx->up_done) cudaEventDestroy(ctx->up_done);
    for (DevBuf *b : {&ctx->lr_in, &ctx->lr_rgb, &ctx->lr_depth})
        if (b->p) cudaFree(b->p);
    delete ctx;
}

const char *gs_last_error(gs_context *ctx) { return ctx ? ctx->err.c_str() : "NULL context"; }

gs_status gs_scene_create(gs_context *ctx, const gs_scene_desc *d, int32_t *scene_id) {
    if (!ctx || !d || !scene_id) return fail(ctx, GS_ERR_INVALID_ARG, "NULL argument");
    ctx->err.clear();
    if (d->n < 0 || d->n > (1LL << 31) - 1)
        return fail(ctx, GS_ERR_INVALID_ARG, "scene size %lld out of range", (long long)d->n);
    if (d->sh_degree < 0 || d->sh_degree > 3)
        return fail(ctx, GS_ERR_INVALID_ARG, "sh_degree %d not in 0..3", d->sh_degree);
    for (int dt : {d->geometry_dtype, d->appearance_dtype})
        if (dt < GS_F32 || dt > GS_BF16) return fail(ctx, GS_ERR_INVALID_ARG, "bad dtype %d", dt);
    if (d->memory != GS_MEM_HOST && d->memory != GS_MEM_DEVICE)
        return fail(ctx, GS_ERR_INVALID_ARG, "bad memory kind %d", d->memory);
    if (d->n > 0 && (!d->mean || !d->log_scale || !d->quat || !d->logit_opacity || !d->sh))
        return fail(ctx, GS_ERR_INVALID_ARG, "NULL attribute pointer");
    CKC(cudaSetDevice(ctx->device));
    const long long n = d->n;
    const int K = (d->sh_degree + 1) * (d->sh_degree + 1);
    const size_t gs = dtype_size(d->geometry_dtype), as = dtype_size(d->appearance_dtype);
    const size_t sz[5] = {3 * n * gs, 3 * n * gs, 4 * n * gs, n * as, (size_t)K * 3 * n * as};
    const size_t esz[5] = {gs, gs, gs, as, as};
    const int rows[5] = {3, 3, 4, 1, 3 * K};
    const void *src[5] = {d->mean, d->log_scale, d->quat, d->logit_opacity, d->sh};
    size_t total = 0, offs[5];
    for (int i = 0; i < 5; ++i) {
        offs[i] = total;
        total += align_up(sz[i], 256);
    }
    const long long nblk = scene_blocks(n);
    const size_t off_orig = total;
    total += align_up((size_t)n * 4, 256);
    const size_t off_bounds = total;
    total += align_up((size_t)nblk * 2 * sizeof(float4), 256);
    // rows per Gaussian for the progressive order's records (see SceneDev)
    const size_t off_geo_rows = total;
    total += align_up((size_t)n * 4 * sizeof(float4), 256);
    const size_t off_sh_rows = total;
    total += align_up((size_t)n * 48 * as, 256);
    const size_t off_pos_of = total;
    total += align_up((size_t)n * 4, 256);
    SceneSlot slot;
    slot.live = true;
    if (n > 0) {
        cudaError_t e = cudaMalloc(&slot.storage, total);
        if (e != cudaSuccess)
            return fail(ctx, GS_ERR_OOM, "scene storage (%zu bytes): %s", total, cudaGetErrorString(e));
        // The caller's arrays go to a temporary buffer first; the scene is stored
        // in Morton order of the means (see k_scene.cu), orig[p] = caller index.
        const long long nt = sort_tiles_for(n);
        const size_t off_raw = 0, raw_bytes = offs[4] + align_up(sz[4], 256);
        const size_t off_code = raw_bytes, u32n = align_up((size_t)n * 4, 256);
        const size_t off_idx = off_code + u32n, off_tk = off_idx + u32n, off_tv = off_tk + u32n;
        const size_t off_hist = off_tv + u32n, hist_bytes = align_up((size_t)nt * 256 * 4, 256);
        const size_t off_meta = off_hist + hist_bytes, tmp_bytes = off_meta + 256;
        void *tmp = nullptr;
        e = cudaMalloc(&tmp, tmp_bytes);
        if (e != cudaSuccess) {
            cudaFree(slot.storage);
            return fail(ctx, GS_ERR_OOM, "scene set-up (%zu bytes): %s", tmp_bytes,
                        cudaGetErrorString(e));
        }
        char *t = (char *)tmp;
        char *st = (char *)slot.storage;
        long long *segs = (long long *)(t + off_meta);         // [0] start, [1] count
        int *tstart = (int *)(t + off_meta + 16);              // [0] 0, [1] tiles
        unsigned *box = (unsigned *)(t + off_meta + 32);       // 6 words
        uint32_t *code = (uint32_t *)(t + off_code), *idx = (uint32_t *)(t + off_idx);
        const long long meta_ll[2] = {0, n};
        const int meta_i[2] = {0, (int)nt};
        for (int i = 0; i < 5 && e == cudaSuccess; ++i)
            if (sz[i])
                e = cudaMemcpy(t + off_raw + offs[i], src[i], sz[i],
                               d->memory == GS_MEM_HOST ? cudaMemcpyHostToDevice
                                                        : cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(segs, meta_ll, sizeof(meta_ll), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(tstart, meta_i, sizeof(meta_i), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = launch_scene_morton(t + off_raw + offs[0], d->geometry_dtype, n, box, code, idx,
                                    nullptr);
        if (e == cudaSuccess)
            e = launch_sort_segments(code, idx, (uint32_t *)(t + off_tk), (uint32_t *)(t + off_tv),
                                     segs, segs + 1, tstart, 1, (int)nt,
                                     (uint32_t *)(t + off_hist), nullptr);
        for (int i = 0; i < 5 && e == cudaSuccess; ++i)
            e = launch_gather_rows(t + off_raw + offs[i], st + offs[i], (int)esz[i], idx, n,
                                   rows[i], nullptr);
        if (e == cudaSuccess)
            e = cudaMemcpy(st + off_orig, idx, (size_t)n * 4, cudaMemcpyDeviceToDevice);
        if (e == cudaSuccess)
            e = launch_block_bounds(st + offs[0], st + offs[1], d->geometry_dtype, n,
                                    (float4 *)(st + off_bounds), nullptr);
        if (e == cudaSuccess) {
            SceneDev sd{};
            sd.mean = st + offs[0];
            sd.log_scale = st + offs[1];
            sd.quat = st + offs[2];
            sd.logit = st + offs[3];
            sd.sh = st + offs[4];
            sd.n = n;
            sd.deg = d->sh_degree;
            sd.geo_dtype = d->geometry_dtype;
            sd.app_dtype = d->appearance_dtype;
            sd.orig = (const int *)(st + off_orig);
            e = launch_scene_rows(sd, (float4 *)(st + off_geo_rows), st + off_sh_rows,
                                  (int *)(st + off_pos_of), nullptr);
        }
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        cudaFree(tmp);
        if (e != cudaSuccess) {
            cudaFree(slot.storage);
            return fail(ctx, GS_ERR_CUDA, "scene set-up: %s", cudaGetErrorString(e));
        }
    }
    char *b = (char *)slot.storage;
    slot.dev.mean = b + offs[0];
    slot.dev.log_scale = b + offs[1];
    slot.dev.quat = b + offs[2];
    slot.dev.logit = b + offs[3];
    slot.dev.sh = b + offs[4];
    slot.dev.orig = (const int *)(b + off_orig);
    slot.dev.bounds = (const float4 *)(b + off_bounds);
    slot.dev.geo_rows = (const float4 *)(b + off_geo_rows);
    slot.dev.sh_rows = b + off_sh_rows;
    slot.dev.pos_of = (const int *)(b + off_pos_of);
    slot.dev.n = n;
    slot.dev.deg = d->sh_degree;
    slot.dev.geo_dtype = d->geometry_dtype;
    slot.dev.app_dtype = d->appearance_dtype;
    int id = -1;
    for (size_t i = 0; i < ctx->scenes.size(); ++i)
        if (!ctx->scenes[i].live) {
            id = (int)i;
            break;
        }
    if (id < 0) {
        id = (int)ctx->scenes.size();
        ctx->scenes.push_back(slot);
    } else {
        ctx->scenes[id] = slot;
    }
    gs_status s = sync_scene_table(ctx);
    if (s != GS_OK) return s;
    *scene_id = id;
    return GS_OK;
}

gs_status gs_scene_destroy(gs_context *ctx, int32_t scene_id) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    if (scene_id < 0 || scene_id >= (int)ctx->scenes.size() || !ctx->scenes[scene_id].live)
        return fail(ctx, GS_ERR_NOT_FOUND, "unknown scene id %d", scene_id);
    CKC(cudaSetDevice(ctx->device));
    CKC(cudaDeviceSynchronize());
    SceneSlot &s = ctx->scenes[scene_id];
    if (s.storage) CKC(cudaFree(s.storage));
    s = SceneSlot();
    return sync_scene_table(ctx);
}

gs_status gs_render_batch(gs_context *ctx, int32_t n_cams, const int32_t *scene_ids,
                          const float *viewmats, const float *intrinsics, int32_t width,
                          int32_t height, float *rgb, float *depth, float *final_T,
                          void *stream) {
    CKS(validate(ctx, n_cams, scene_ids, viewmats, intrinsics, width, height, rgb, depth, true));
    ctx->err.clear();
    if (n_cams == 0) return GS_OK;
    CKC(cudaSetDevice(ctx->device));
    RenderArgs a{n_cams, scene_ids, viewmats, intrinsics, width, height, nullptr, nullptr,
                 nullptr, rgb, depth, final_T, (cudaStream_t)stream, UPTO_ALL};
    return render_impl(ctx, a);
}

gs_status gs_render_batch_v(gs_context *ctx, int32_t n_cams, const int32_t *scene_ids,
                            const float *viewmats, const float *intrinsics, const int32_t *widths,
                            const int32_t *heights, const int64_t *pixel_offsets, float *rgb,
                            float *depth, float *final_T, void *stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    if (n_cams > 0 && (!widths || !heights || !pixel_offsets))
        return fail(ctx, GS_ERR_INVALID_ARG, "NULL per-camera size or offset array");
    for (int i = 0; i < n_cams; ++i) {
        CKS(validate(ctx, 1, scene_ids + i, viewmats, intrinsics, widths[i], heights[i], rgb,
                     depth, true));
        if (pixel_offsets[i] < 0) return fail(ctx, GS_ERR_INVALID_ARG, "negative pixel offset");
    }
    CKS(validate(ctx, n_cams, scene_ids, viewmats, intrinsics, 1, 1, rgb, depth, true));
    ctx->err.clear();
    if (n_cams == 0) return GS_OK;
    CKC(cudaSetDevice(ctx->device));
    RenderArgs a{n_cams, scene_ids, viewmats, intrinsics, 0,
                 0,      widths,    heights,  pixel_offsets, rgb,
                 depth,  final_T,   (cudaStream_t)stream, UPTO_ALL};
    return render_impl(ctx, a);
}

gs_status gs_render_motion_blur(gs_context *ctx, int32_t n_cams, const int32_t *scene_ids,
                                const float *viewmats, const float *intrinsics,
                                const float *velocities, float shutter, int32_t samples,
                                int32_t width, int32_t height, float *rgb, float *depth,
                                float *final_T, void *stream) {
    CKS(validate(ctx, n_cams, scene_ids, viewmats, intrinsics, width, height, rgb, depth, true));
    if (samples < 1 || samples > 64)
        return fail(ctx, GS_ERR_INVALID_ARG, "samples %d not in 1..64", samples);
    if (!(shutter >= 0.0f)) return fail(ctx, GS_ERR_INVALID_ARG, "negative shutter time");
    if (n_cams > 0 && !velocities) return fail(ctx, GS_ERR_INVALID_ARG, "NULL velocities");
    ctx->err.clear();
    if (n_cams == 0) return GS_OK;
    CKC(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    CKS(grow(ctx, ctx->blur_vm, (size_t)n_cams * samples * 16 * sizeof(float)));
    CKC(launch_blur_poses(viewmats, velocities, n_cams, samples, shutter, (float *)ctx->blur_vm.p,
                          st));
    for (int j = 0; j < samples; ++j) {
        RenderArgs a{n_cams,  scene_ids, (const float *)ctx->blur_vm.p + (size_t)j * n_cams * 16,
                     intrinsics, width, height, nullptr, nullptr, nullptr, rgb, depth, final_T, st,
                     UPTO_ALL};
        a.out_w = 1.0f / (float)samples;
        a.accumulate = j > 0;
        CKS(render_impl(ctx, a));
    }
    return GS_OK;
}

gs_status gs_graph_create(gs_context *ctx, int32_t n_cams, const int32_t *scene_ids,
                          const float *viewmats, const float *intrinsics, const int32_t *widths,
                          const int32_t *heights, const int64_t *pixel_offsets, float *rgb,
                          float *depth, float *final_T, gs_graph **out) {
    if (!ctx || !out) return GS_ERR_INVALID_ARG;
    *out = nullptr;
    if (n_cams < 1) return fail(ctx, GS_ERR_INVALID_ARG, "a graph needs at least one camera");
    // size everything with one eager render of the same cameras (waiting for its
    // status, so the survivors of its largest chunk are known)
    if (!widths || !heights || !pixel_offsets)
        return fail(ctx, GS_ERR_INVALID_ARG, "NULL per-camera size or offset array");
    for (int i = 0; i < n_cams; ++i) {
        CKS(validate(ctx, 1, scene_ids + i, viewmats, intrinsics, widths[i], heights[i], rgb,
                     depth, true));
        if (pixel_offsets[i] < 0) return fail(ctx, GS_ERR_INVALID_ARG, "negative pixel offset");
    }
    ctx->err.clear();
    CKC(cudaSetDevice(ctx->device));
    RenderArgs a{n_cams, scene_ids, viewmats, intrinsics, 0,
                 0,      widths,    heights,  pixel_offsets, rgb,
                 depth,  final_T,   nullptr,  UPTO_ALL};
    a.force_sync = true;
    CKS(render_impl(ctx, a));
    CKC(cudaDeviceSynchronize());
    a.force_sync = false;
    Plan P;
    build_plan(ctx, a, P);
    // headroom for cameras that move between launches: 1.25x the largest chunk seen
    const long long want = ctx->last_chunk_survivors + ctx->last_chunk_survivors / 4 + 4096;
    if (want > ctx->cap_survivors) ctx->cap_survivors = want;
    CKS(size_workspace(ctx, P));
    gs_graph *g = new gs_graph();
    g->ctx = ctx;
    cudaStream_t cs = nullptr;
    gs_status rc = GS_OK;
    do {
        if (upload_tables(ctx, P, g->tables, nullptr) != GS_OK) { rc = GS_ERR_CUDA; break; }
        if (cudaDeviceSynchronize() != cudaSuccess) { rc = GS_ERR_CUDA; break; }
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
            rc = GS_ERR_CUDA;
            break;
        }
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            rc = GS_ERR_CUDA;
            break;
        }
        RenderArgs ac = a;
        ac.st = cs;
        gs_status e1 = GS_OK;
        if (cudaMemsetAsync(ctx->stats.p, 0, N_STATS * sizeof(unsigned long long), cs) != cudaSuccess ||
            cudaMemsetAsync(ctx->status.p, 0, sizeof(long long) + P.chunks.size() * sizeof(int),
                            cs) != cudaSuccess)
            e1 = GS_ERR_CUDA;
        if (e1 == GS_OK) e1 = enqueue_render(ctx, ac, P, (char *)g->tables.p, cs, nullptr);
        const cudaError_t e2 = cudaStreamEndCapture(cs, &g->graph);
        if (e1 != GS_OK || e2 != cudaSuccess) {
            rc = e1 != GS_OK ? e1 : GS_ERR_CUDA;
            if (e2 != cudaSuccess) fail(ctx, rc, "graph capture: %s", cudaGetErrorString(e2));
            break;
        }
        const cudaError_t e3 = cudaGraphInstantiate(&g->exec, g->graph, 0);
        if (e3 != cudaSuccess) {
            rc = fail(ctx, GS_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e3));
            break;
        }
    } while (0);
    if (cs) cudaStreamDestroy(cs);
    if (rc != GS_OK) {
        gs_graph_destroy(g);
        return rc;
    }
    g->gen = ctx->workspace_gen;
    g->n_chunks = (int)P.chunks.size();
    ctx->stats_pending = false;
    *out = g;
    return GS_OK;
}

gs_status gs_graph_launch(gs_graph *g, void *stream) {
    if (!g || !g->exec) return GS_ERR_INVALID_ARG;
    gs_context *ctx = g->ctx;
    if (g->gen != ctx->workspace_gen)
        return fail(ctx, GS_ERR_INVALID_ARG,
                    "the context's workspace was reallocated after capture: create the graph again");
    CKC(cudaSetDevice(ctx->device));
    CKC(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
    return GS_OK;
}

gs_status gs_graph_check(gs_graph *g, void *stream) {
    if (!g) return GS_ERR_INVALID_ARG;
    gs_context *ctx = g->ctx;
    CKC(cudaSetDevice(ctx->device));
    CKC(cudaStreamSynchronize((cudaStream_t)stream));
    std::vector<char> h(sizeof(long long) + g->n_chunks * sizeof(int));
    CKC(cudaMemcpy(h.data(), ctx->status.p, h.size(), cudaMemcpyDeviceToHost));
    const int *st = (const int *)(h.data() + sizeof(long long));
    if (ctx->sticky.p) {
        unsigned long long sk[2];
        CKC(cudaMemcpy(sk, ctx->sticky.p, sizeof(sk), cudaMemcpyDeviceToHost));
        if (sk[1] & 2ull) {
            CKC(cudaMemset((unsigned long long *)ctx->sticky.p + 1, 0, sizeof(unsigned long long)));
            return fail(ctx, GS_ERR_TIMEOUT,
                        "a graph launch's persistent binning + compositing gave up waiting");
        }
    }
    for (int k = 0; k < g->n_chunks; ++k)
        if (st[k]) {
            // reported here, not again by a later call
            if (ctx->sticky.p)
                CKC(cudaMemset((unsigned long long *)ctx->sticky.p + 1, 0, sizeof(unsigned long long)));
            return fail(ctx, GS_ERR_CAPACITY,
                        "a graph launch exceeded the workspace (%lld survivors in a chunk): "
                        "render eagerly once and create the graph again",
                        *(const long long *)h.data());
        }
    return GS_OK;
}

void gs_graph_destroy(gs_graph *g) {
    if (!g) return;
    if (g->ctx) cudaSetDevice(g->ctx->device);
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->tables.p) cudaFree(g->tables.p);
    delete g;
}

gs_status gs_render_batch_host(gs_context *ctx, int32_t n_cams, const int32_t *scene_ids,
                               const float *viewmats, const float *intrinsics, int32_t width,
                               int32_t height, float *rgb, float *depth, float *final_T,
                               void *stream) {
    CKS(validate(ctx, n_cams, scene_ids, viewmats, intrinsics, width, height, rgb, depth, true));
    ctx->err.clear();
    if (n_cams == 0) return GS_OK;
    CKC(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const size_t px = (size_t)n_cams * width * height;
    CKS(grow(ctx, ctx->h_vm, (size_t)n_cams * 16 * 4));
    CKS(grow(ctx, ctx->h_in, (size_t)n_cams * 4 * 4));
    CKS(grow(ctx, ctx->h_rgb, px * 3 * 4));
    CKS(grow(ctx, ctx->h_depth, px * 4));
    if (final_T) CKS(grow(ctx, ctx->h_T, px * 4));
    CKC(cudaMemcpyAsync(ctx->h_vm.p, viewmats, (size_t)n_cams * 16 * 4, cudaMemcpyHostToDevice, st));
    CKC(cudaMemcpyAsync(ctx->h_in.p, intrinsics, (size_t)n_cams * 4 * 4, cudaMemcpyHostToDevice, st));
    // The batch is rendered in parts (at most one chunk, at most 128 cameras);
    // the copies of part k back to the host run on a second stream while part
    // k + 1 renders, so only the last part's copy is not hidden.
    if (!ctx->copy_stream)
        CKC(cudaStreamCreateWithFlags(&ctx->copy_stream, cudaStreamNonBlocking));
    const int part = std::max(1, std::min(ctx->cfg.max_chunk_cameras, 128));
    const int n_parts = (n_cams + part - 1) / part;
    while ((int)ctx->part_done.size() < n_parts) {
        cudaEvent_t e;
        CKC(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->part_done.push_back(e);
    }
    const size_t fpx = (size_t)width * height;  // pixels per frame
    for (int k = 0; k < n_parts; ++k) {
        const int c0 = k * part, m = std::min(part, n_cams - c0);
        const size_t p0 = (size_t)c0 * fpx, pm = (size_t)m * fpx;
        RenderArgs a{m,
                     scene_ids + c0,
                     (const float *)ctx->h_vm.p + 16LL * c0,
                     (const float *)ctx->h_in.p + 4LL * c0,
                     width,
                     height,
                     nullptr,
                     nullptr,
                     nullptr,
                     (float *)ctx->h_rgb.p + 3 * p0,
                     (float *)ctx->h_depth.p + p0,
                     final_T ? (float *)ctx->h_T.p + p0 : nullptr,
                     st,
                     UPTO_ALL};
        a.force_sync = true;  // a part is copied out only once it is complete
        gs_status rs = render_impl(ctx, a);
        if (rs != GS_OK) {
            cudaStreamSynchronize(ctx->copy_stream);
            return rs;
        }
        CKC(cudaEventRecord(ctx->part_done[k], st));
        cudaStream_t cs = ctx->copy_stream;
        CKC(cudaStreamWaitEvent(cs, ctx->part_done[k], 0));
        CKC(cudaMemcpyAsync(rgb + 3 * p0, (float *)ctx->h_rgb.p + 3 * p0, pm * 3 * 4,
                            cudaMemcpyDeviceToHost, cs));
        CKC(cudaMemcpyAsync(depth + p0, (float *)ctx->h_depth.p + p0, pm * 4, cudaMemcpyDeviceToHost,
                            cs));
        if (final_T)
            CKC(cudaMemcpyAsync(final_T + p0, (float *)ctx->h_T.p + p0, pm * 4,
                                cudaMemcpyDeviceToHost, cs));
    }
    CKC(cudaStreamSynchronize(ctx->copy_stream));
    CKC(cudaStreamSynchronize(st));
    return GS_OK;
}

gs_status gs_render_batch_upsampled(gs_context *ctx, gs_upsampler *up, int32_t n_cams,
                                    const int32_t *scene_ids, const float *viewmats,
                                    const float *intrinsics, int32_t width, int32_t height,
                                    float *rgb, float *depth, void *stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    if (!up) return fail(ctx, GS_ERR_INVALID_ARG, "NULL upsampler");
    if (width % 4 || height % 4)
        return fail(ctx, GS_ERR_INVALID_ARG, "width and height must be multiples of 4");
    CKS(validate(ctx, n_cams, scene_ids, viewmats, intrinsics, width, height, rgb, depth, true));
    ctx->err.clear();
    if (n_cams == 0) return GS_OK;
    CKC(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    const int w = width / 4, h = height / 4;
    const size_t lpx = (size_t)w * h;
    CKS(grow(ctx, ctx->lr_in, (size_t)n_cams * 4 * sizeof(float)));
    CKS(grow(ctx, ctx->lr_rgb, (size_t)n_cams * lpx * 3 * sizeof(float)));
    CKS(grow(ctx, ctx->lr_depth, (size_t)n_cams * lpx * sizeof(float)));
    if (!ctx->up_stream) CKC(cudaStreamCreateWithFlags(&ctx->up_stream, cudaStreamNonBlocking));
    if (!ctx->up_done) CKC(cudaEventCreateWithFlags(&ctx->up_done, cudaEventDisableTiming));
    CKC(gsk::launch_scale_intrinsics(intrinsics, n_cams, 4.0f, (float *)ctx->lr_in.p, st));
    // Parts of one chunk: the upsampler works on part k on its own stream while
    // part k + 1 renders.
    const int part = std::max(1, ctx->cfg.max_chunk_cameras);
    const int n_parts = (n_cams + part - 1) / part;
    while ((int)ctx->part_done.size() < n_parts) {
        cudaEvent_t e;
        CKC(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        ctx->part_done.push_back(e);
    }
    CKC(cudaEventRecord(ctx->up_done, ctx->up_stream));
    CKC(cudaStreamWaitEvent(st, ctx->up_done, 0));  // earlier upsampling of these buffers done
    for (int k = 0; k < n_parts; ++k) {
        const int c0 = k * part, m = std::min(part, n_cams - c0);
        float *lr = (float *)ctx->lr_rgb.p + (size_t)c0 * lpx * 3;
        float *ld = (float *)ctx->lr_depth.p + (size_t)c0 * lpx;
        RenderArgs a{m,  scene_ids + c0, viewmats + 16LL * c0, (const float *)ctx->lr_in.p + 4LL * c0,
                     w,  h,  nullptr, nullptr, nullptr, lr, ld, nullptr, st, UPTO_ALL};
        a.force_sync = true;  // the upsampler reads a part only once it is complete
        CKS(render_impl(ctx, a));
        CKC(cudaEventRecord(ctx->part_done[k], st));
        CKC(cudaStreamWaitEvent(ctx->up_stream, ctx->part_done[k], 0));
        const gs_status us = gs_upsample_forward(up, m, h, w, lr, ld, rgb + (size_t)c0 * lpx * 48,
                                                 depth + (size_t)c0 * lpx * 16, ctx->up_stream);
        if (us != GS_OK) return fail(ctx, us, "upsampler: %s", gs_upsampler_last_error(up));
    }
    // the caller's stream continues after the last upsampling
    CKC(cudaEventRecord(ctx->up_done, ctx->up_stream));
    CKC(cudaStreamWaitEvent(st, ctx->up_done, 0));
    return GS_OK;
}

gs_status gs_sync(gs_context *ctx, void *stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    CKC(cudaSetDevice(ctx->device));
    CKC(cudaStreamSynchronize((cudaStream_t)stream));
    if (ctx->done_valid) CKC(cudaEventSynchronize(ctx->done_ev));
    return poll_sticky(ctx, true, (cudaStream_t)stream);
}

gs_status gs_render_timeout_probe(gs_context *ctx, int32_t scene_id, const float *viewmat,
                                  const float *intrinsics, int32_t width, int32_t height,
                                  float *rgb, float *depth, void *stream) {
    CKS(validate(ctx, 1, &scene_id, viewmat, intrinsics, width, height, rgb, depth, true));
    ctx->err.clear();
    CKC(cudaSetDevice(ctx->device));
    const gs_config saved = ctx->cfg;
    ctx->cfg.persistent = 1;
    ctx->cfg.pixels_per_thread = 8;
    ctx->cfg.tiles_per_block = 1;
    ctx->cfg.count_pairs = 0;
    ctx->probe_extra = 1;     // camera 0's tiles wait for a binning item that never comes
    ctx->probe_limit = 4096;  // and give up after 4,096 polls
    RenderArgs a{1,   &scene_id, viewmat, intrinsics, width,  height,
                 nullptr, nullptr, nullptr, rgb, depth, nullptr, (cudaStream_t)stream, UPTO_ALL};
    a.force_sync = true;
    const gs_status r = render_impl(ctx, a);
    ctx->cfg = saved;
    ctx->probe_extra = 0;
    ctx->probe_limit = 0;
    return r;
}

gs_status gs_set_resume_capacity(gs_context *ctx, int32_t tiles) {
    if (!ctx || tiles < 0) return GS_ERR_INVALID_ARG;
    ctx->resume_cap = tiles;
    return GS_OK;
}

gs_status gs_get_stats(gs_context *ctx, gs_stats *out) {
    if (!ctx || !out) return GS_ERR_INVALID_ARG;
    CKC(cudaSetDevice(ctx->device));
    if (ctx->done_valid) CKC(cudaEventSynchronize(ctx->done_ev));  // the last call is complete
    if (ctx->stats_pending && ctx->stats.p) {
        unsigned long long h[N_STATS];
        CKC(cudaMemcpy(h, ctx->stats.p, sizeof(h), cudaMemcpyDeviceToHost));
        ctx->last.pairs_evaluated = (int64_t)h[0];
        ctx->last.pairs_alpha = (int64_t)h[1];
        ctx->last.intersections = (int64_t)h[2];
        ctx->last.warp_iters = (int64_t)h[3];
        ctx->last.warp_iters_box = (int64_t)h[4];
        ctx->last.warp_iters_blend = (int64_t)h[5];
        ctx->last.survivors = (int64_t)h[6];
        ctx->last.depth_second_phase_cameras = (int64_t)h[7];
        ctx->last.depth_resumed_tiles = (int64_t)h[8];
        // the depth order's lists, per chunk and phase: long runs, listed windows,
        // equal runs
        const int nc = ctx->last.n_chunks;
        if (nc > 0 && ctx->nruns.p && ctx->nruns.cap >= 6 * (size_t)nc * sizeof(int)) {
            std::vector<int> cnt(6 * (size_t)nc);
            CKC(cudaMemcpy(cnt.data(), ctx->nruns.p, cnt.size() * sizeof(int), cudaMemcpyDeviceToHost));
            for (int c = 0; c < 2 * nc; ++c) {
                ctx->last.sort_long_runs += cnt[3 * c];
                ctx->last.sort_windows_listed += cnt[3 * c + 1];
                ctx->last.sort_equal_runs += cnt[3 * c + 2];
            }
        }
        // stages: project, depth order (both phases), binning (both), compositing (both)
        float ms[4] = {0, 0, 0, 0};
        const int stage_of[EV_PER_CHUNK - 1] = {0, 1, 2, 3, 1, 2, 3};
        for (int c = 0; c < ctx->ev_used; ++c) {
            cudaEvent_t *E = &ctx->ev[EV_PER_CHUNK * c];
            CKC(cudaEventSynchronize(E[EV_PER_CHUNK - 1]));
            for (int k = 0; k < EV_PER_CHUNK - 1; ++k) {
                float t = 0;
                CKC(cudaEventElapsedTime(&t, E[k], E[k + 1]));
                ms[stage_of[k]] += t;
            }
        }
        ctx->last.ms_project = ms[0];
        ctx->last.ms_sort = ms[1];
        ctx->last.ms_bin = ms[2];
        ctx->last.ms_composite = ms[3];
        ctx->last.ms_total = ms[0] + ms[1] + ms[2] + ms[3];
        ctx->stats_pending = false;
    }
    *out = ctx->last;
    return poll_sticky(ctx, true, nullptr);  // a chunk of an earlier call did not fit
}

// The first S records of the last render (all four fields) to the host.
static gs_status copy_records(gs_context *ctx, long long S, std::vector<SlotRec> &out) {
    if (S == 0) return GS_OK;
    std::vector<float4> raw(rec_bytes(S) / sizeof(float4));
    CKC(cudaMemcpy(raw.data(), ctx->rec.p, rec_bytes(S), cudaMemcpyDeviceToHost));
    for (long long i = 0; i < S; ++i) {
        uint4 d;
        memcpy(&d, &raw[rec_d(i)], sizeof(d));
        out[i] = SlotRec{raw[rec_a(i)], raw[rec_b(i)], raw[rec_c(i)], d};
    }
    return GS_OK;
}

gs_status gs_debug_project(gs_context *ctx, int32_t scene_id, const float *viewmat,
                           const float *intrinsics, int32_t width, int32_t height, float *rec,
                           int32_t *gidx, int32_t *rect, int64_t cap, int64_t *n_out,
                           void *stream) {
    CKS(validate(ctx, 1, &scene_id, viewmat, intrinsics, width, height, nullptr, nullptr, false));
    if (!n_out || cap < 0 || (cap > 0 && (!rec || !gidx || !rect)))
        return fail(ctx, GS_ERR_INVALID_ARG, "bad output buffers");
    ctx->err.clear();
    CKC(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    RenderArgs a{1,       &scene_id, viewmat, intrinsics, width, height, nullptr, nullptr,
                 nullptr, nullptr,   nullptr, nullptr,    st,    UPTO_PROJECT};
    a.force_sync = true;
    CKS(render_impl(ctx, a));
    CKC(cudaStreamSynchronize(st));
    gs_stats tmp;
    CKS(gs_get_stats(ctx, &tmp));
    const long long S = ctx->last.survivors;
    *n_out = S;
    if (S > cap) return fail(ctx, GS_ERR_CAPACITY, "%lld survivors > cap %lld", S, (long long)cap);
    std::vector<SlotRec> h((size_t)S);
    CKS(copy_records(ctx, S, h));
    // slots follow the storage order; report in the caller's Gaussian-index order
    std::vector<long long> order((size_t)S);
    for (long long i = 0; i < S; ++i) order[i] = i;
    std::sort(order.begin(), order.end(),
              [&](long long x, long long y) { return h[x].d.z < h[y].d.z; });
    const float L2E = 1.4426950408889634f;
    for (long long i = 0; i < S; ++i) {
        const SlotRec &R = h[order[i]];
        // undo the folding of the compositing constants (see SlotRec)
        const float v[12] = {R.a.x,
                             R.a.y,
                             R.c.w,
                             std::exp2(R.b.w),
                             R.b.x / (-0.5f * L2E),
                             R.b.y / (-L2E),
                             R.b.z / (-0.5f * L2E),
                             __uint_as_float_host(R.d.w),
                             R.c.x,
                             R.c.y,
                             R.c.z,
                             0.0f};
        memcpy(rec + 12 * i, v, sizeof(v));
        gidx[i] = (int32_t)R.d.z;
        rect[4 * i + 0] = (int32_t)(R.d.x & 0xffffu);
        rect[4 * i + 1] = (int32_t)(R.d.x >> 16);
        rect[4 * i + 2] = (int32_t)(R.d.y & 0xffffu);
        rect[4 * i + 3] = (int32_t)(R.d.y >> 16);
    }
    return GS_OK;
}

gs_status gs_debug_tile_lists(gs_context *ctx, int32_t scene_id, const float *viewmat,
                              const float *intrinsics, int32_t width, int32_t height,
                              int64_t *tile_off, int32_t *gidx, int64_t cap, int64_t *n_out,
                              void *stream) {
    CKS(validate(ctx, 1, &scene_id, viewmat, intrinsics, width, height, nullptr, nullptr, false));
    if (!n_out || !tile_off || cap < 0 || (cap > 0 && !gidx))
        return fail(ctx, GS_ERR_INVALID_ARG, "bad output buffers");
    ctx->err.clear();
    CKC(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    RenderArgs a{1,       &scene_id, viewmat, intrinsics, width, height, nullptr, nullptr,
                 nullptr, nullptr,   nullptr, nullptr,    st,    UPTO_BIN};
    a.force_sync = true;
    CKS(render_impl(ctx, a));
    CKC(cudaStreamSynchronize(st));
    gs_stats tmp;
    CKS(gs_get_stats(ctx, &tmp));
    const long long S = ctx->last.survivors;
    const int TX = (width + 15) / 16, TY = (height + 15) / 16, tiles = TX * TY;
    const int SX = (TX + STILE - 1) / STILE, SY = (TY + STILE - 1) / STILE;
    const int nw = (int)((S + 31) / 32);
    std::vector<SlotRec> rec((size_t)S);
    std::vector<uint32_t> vals((size_t)S), bm((size_t)SX * SY * nw);
    std::vector<uint2> rr((size_t)S);
    if (S) {
        CKS(copy_records(ctx, S, rec));
        CKC(cudaMemcpy(vals.data(), ctx->tvals.p, S * 4, cudaMemcpyDeviceToHost));
        CKC(cudaMemcpy(rr.data(), ctx->rrect.p, S * sizeof(uint2), cudaMemcpyDeviceToHost));
        CKC(cudaMemcpy(bm.data(), ctx->bitmap.p, bm.size() * 4, cudaMemcpyDeviceToHost));
    }
    // the compositing pass's reading of a tile's list: set bits of its
    // super-tile's row in order, kept when the rank-ordered rect holds the tile
    long long k = 0;
    tile_off[0] = 0;
    for (int t = 0; t < tiles; ++t) {
        const int tx = t % TX, ty = t / TX;
        const uint32_t *row = bm.data() + (size_t)((ty / STILE) * SX + tx / STILE) * nw;
        for (int w = 0; w < nw; ++w) {
            uint32_t word = row[w];
            while (word) {
                const int b = __builtin_ctz(word);
                word &= word - 1u;
                const size_t r = (size_t)w * 32 + b;
                const uint2 q = rr[r];
                if (tx < (int)(q.x & 0xffffu) || tx > (int)(q.x >> 16) ||
                    ty < (int)(q.y & 0xffffu) || ty > (int)(q.y >> 16))
                    continue;
                if (k < cap) gidx[k] = (int32_t)rec[vals[r]].d.z;
                ++k;
            }
        }
        tile_off[t + 1] = k;
    }
    *n_out = k;
    if (k > cap) return fail(ctx, GS_ERR_CAPACITY, "%lld entries > cap %lld", k, (long long)cap);
    return GS_OK;
}

gs_status gs_sort_segments(gs_context *ctx, uint32_t *keys, uint32_t *vals, int64_t n,
                           const int64_t *seg_start, const int64_t *seg_count, int32_t n_seg,
                           void *stream) {
    if (!ctx) return GS_ERR_INVALID_ARG;
    if (n < 0 || n_seg < 0) return fail(ctx, GS_ERR_INVALID_ARG, "negative size");
    if (n_seg == 0) return GS_OK;
    if (!keys || !vals || !seg_start || !seg_count)
        return fail(ctx, GS_ERR_INVALID_ARG, "NULL argument");
    ctx->err.clear();
    CKC(cudaSetDevice(ctx->device));
    cudaStream_t st = (cudaStream_t)stream;
    // the tile table is built on the host from the segment lengths
    std::vector<int64_t> hs(n_seg), hc(n_seg);
    CKC(cudaMemcpyAsync(hs.data(), seg_start, n_seg * 8, cudaMemcpyDeviceToHost, st));
    CKC(cudaMemcpyAsync(hc.data(), seg_count, n_seg * 8, cudaMemcpyDeviceToHost, st));
    CKC(cudaStreamSynchronize(st));
    std::vector<int> tiles(n_seg + 1);
    int nt = 0;
    for (int i = 0; i < n_seg; ++i) {
        if (hc[i] < 0 || hs[i] < 0 || hs[i] + hc[i] > n)
            return fail(ctx, GS_ERR_INVALID_ARG, "segment %d out of range", i);
        tiles[i] = nt;
        nt += sort_tiles_for(hc[i]);
    }
    tiles[n_seg] = nt;
    // scratch of its own: a render may still be running on the workspace
    CKS(grow(ctx, ctx->seg_tk, (size_t)std::max<int64_t>(n, 1) * 4));
    CKS(grow(ctx, ctx->seg_tv, (size_t)std::max<int64_t>(n, 1) * 4));
    CKS(grow(ctx, ctx->seg_tiles, tiles.size() * sizeof(int)));
    CKS(grow(ctx, ctx->seg_hist, (size_t)std::max(nt, 1) * 256 * 4));
    CKC(cudaMemcpyAsync(ctx->seg_tiles.p, tiles.data(), tiles.size() * sizeof(int),
                        cudaMemcpyHostToDevice, st));
    CKC(launch_sort_segments(keys, vals, (uint32_t *)ctx->seg_tk.p, (uint32_t *)ctx->seg_tv.p,
                             (const long long *)seg_start, (const long long *)seg_count,
                             (const int *)ctx->seg_tiles.p, n_seg, nt,
                             (uint32_t *)ctx->seg_hist.p, st));
    CKC(cudaStreamSynchronize(st));  // the host tile table must outlive the copy
    return GS_OK;
}

}  // extern "C"
