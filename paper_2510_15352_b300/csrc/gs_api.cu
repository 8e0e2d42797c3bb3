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
    DevBuf cams, groups, blkpre, tilepre, segstart, segcount, stats, sorttiles, sorthist;
    // host-API staging
    DevBuf h_vm, h_in, h_rgb, h_depth, h_T;
    PinBuf pin[2];
    gs_stats last{};
    bool stats_pending = false;
    std::string err;
    std::vector<cudaEvent_t> ev;  // time_stages: 5 events per chunk of the last call
    int ev_used = 0;              // chunks whose events the last call recorded
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
    int cam_w(int i) const { return Ws ? Ws[i] : W; }
    int cam_h(int i) const { return Hs ? Hs[i] : H; }
    long long cam_pix(int i) const { return pix_off ? pix_off[i] : (long long)i * W * H; }
};

// Pinned staging layout of one chunk.
struct Staging {
    CamInfo *cams;
    Group *groups;
    int *blkpre, *tilepre, *counts, *sorttiles;
    long long *segstart, *segcount;
};

gs_status render_impl(gs_context *ctx, const RenderArgs &a) {
    const gs_config &cfg = ctx->cfg;
    const int chunk_max = std::max(1, cfg.max_chunk_cameras);
    const int gmax = std::min(MAX_GROUP, std::max(1, cfg.camera_group));
    const ProjParams P{cfg.near_plane, cfg.dilation, cfg.guard_band, cfg.sigma_cull};
    const CompParams C{std::log2(cfg.alpha_min), cfg.alpha_max, cfg.T_min,
                       {cfg.background[0], cfg.background[1], cfg.background[2]}};
    const bool timing = cfg.time_stages != 0;

    // cameras grouped by scene (stable), then chunked
    std::vector<int> order(a.n);
    for (int i = 0; i < a.n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return a.scene_ids[x] < a.scene_ids[y]; });

    gs_stats st{};
    st.n_cameras = a.n;
    CKS(grow(ctx, ctx->stats, 8 * sizeof(unsigned long long)));
    CKC(cudaMemsetAsync(ctx->stats.p, 0, 8 * sizeof(unsigned long long), a.st));
    const size_t stage_bytes =
        align_up((size_t)chunk_max * sizeof(CamInfo), 256) + align_up((size_t)chunk_max * sizeof(Group), 256) +
        4 * align_up((size_t)(chunk_max + 1) * sizeof(int), 256) +
        2 * align_up((size_t)chunk_max * sizeof(long long), 256);
    for (int k = 0; k < 2; ++k) CKS(grow_pinned(ctx, ctx->pin[k], stage_bytes));
    CKS(grow(ctx, ctx->cams, (size_t)chunk_max * sizeof(CamInfo)));
    CKS(grow(ctx, ctx->groups, (size_t)chunk_max * sizeof(Group)));
    CKS(grow(ctx, ctx->blkpre, (size_t)(chunk_max + 1) * sizeof(int)));
    CKS(grow(ctx, ctx->tilepre, (size_t)(chunk_max + 1) * sizeof(int)));
    CKS(grow(ctx, ctx->segstart, (size_t)chunk_max * sizeof(long long)));
    CKS(grow(ctx, ctx->segcount, (size_t)chunk_max * sizeof(long long)));
    CKS(grow(ctx, ctx->counts, (size_t)chunk_max * sizeof(int)));
    CKS(grow(ctx, ctx->sorttiles, (size_t)(chunk_max + 1) * sizeof(int)));
    const int n_chunks = (a.n + chunk_max - 1) / chunk_max;
    if (timing)
        while ((int)ctx->ev.size() < 5 * n_chunks) {
            cudaEvent_t e;
            CKC(cudaEventCreate(&e));
            ctx->ev.push_back(e);
        }
    ctx->ev_used = 0;

    int chunk_id = 0;
    for (int c0 = 0; c0 < a.n; c0 += chunk_max, ++chunk_id) {
        const int m = std::min(chunk_max, a.n - c0);
        // pinned staging for this chunk
        char *base = (char *)ctx->pin[chunk_id & 1].p;
        Staging S;
        size_t off = 0;
        S.cams = (CamInfo *)(base + off);
        off += align_up((size_t)chunk_max * sizeof(CamInfo), 256);
        S.groups = (Group *)(base + off);
        off += align_up((size_t)chunk_max * sizeof(Group), 256);
        S.blkpre = (int *)(base + off);
        off += align_up((size_t)(chunk_max + 1) * sizeof(int), 256);
        S.tilepre = (int *)(base + off);
        off += align_up((size_t)(chunk_max + 1) * sizeof(int), 256);
        S.counts = (int *)(base + off);
        off += align_up((size_t)(chunk_max + 1) * sizeof(int), 256);
        S.sorttiles = (int *)(base + off);
        off += align_up((size_t)(chunk_max + 1) * sizeof(int), 256);
        S.segstart = (long long *)(base + off);
        off += align_up((size_t)chunk_max * sizeof(long long), 256);
        S.segcount = (long long *)(base + off);

        long long mask_words = 0;
        int n_groups = 0, max_bx = 0, tiles_total = 0, max_sup = 1;
        for (int s = 0; s < m; ++s) {
            const int user = order[c0 + s];
            const int sid = a.scene_ids[user];
            const SceneDev &sd = ctx->scenes[sid].dev;
            CamInfo &ci = S.cams[s];
            memset(&ci, 0, sizeof(ci));
            ci.user = user;
            ci.scene = sid;
            ci.W = a.cam_w(user);
            ci.H = a.cam_h(user);
            ci.TX = (ci.W + TILE - 1) / TILE;
            ci.TY = (ci.H + TILE - 1) / TILE;
            ci.pix_off = a.cam_pix(user);
            ci.tile_off = tiles_total;
            S.tilepre[s] = tiles_total;
            tiles_total += ci.TX * ci.TY;
            max_sup = std::max(max_sup, ((ci.TX + STILE - 1) / STILE) * ((ci.TY + STILE - 1) / STILE));
            ci.mask_off = mask_words;
            mask_words += (sd.n + 31) / 32;
            const bool new_group = s == 0 || S.groups[n_groups - 1].scene != sid ||
                                   S.groups[n_groups - 1].ncam == gmax;
            if (new_group) {
                Group &g = S.groups[n_groups++];
                g.scene = sid;
                g.slot0 = s;
                g.ncam = 0;
                g.pad = 0;
                g.n = sd.n;
                max_bx = std::max<long long>(max_bx, (sd.n + PROJ_THREADS - 1) / PROJ_THREADS);
            }
            S.groups[n_groups - 1].ncam++;
        }
        CKS(grow(ctx, ctx->masks, (size_t)std::max<long long>(mask_words, 1) * 4));
        CKS(grow(ctx, ctx->woff, (size_t)std::max<long long>(mask_words, 1) * 4));
        CKC(cudaMemcpyAsync(ctx->cams.p, S.cams, m * sizeof(CamInfo), cudaMemcpyHostToDevice, a.st));
        CKC(cudaMemcpyAsync(ctx->groups.p, S.groups, n_groups * sizeof(Group),
                            cudaMemcpyHostToDevice, a.st));
        cudaEvent_t *E = timing ? &ctx->ev[5 * chunk_id] : nullptr;
        if (timing) CKC(cudaEventRecord(E[0], a.st));
        CKC(launch_project_mask((const Group *)ctx->groups.p, n_groups, max_bx,
                                (const SceneDev *)ctx->d_scenes.p, (const CamInfo *)ctx->cams.p,
                                a.vm, a.in, P, (uint32_t *)ctx->masks.p, a.st));
        CKC(launch_scan_masks((const CamInfo *)ctx->cams.p, (const SceneDev *)ctx->d_scenes.p, m,
                              (const uint32_t *)ctx->masks.p, (uint32_t *)ctx->woff.p,
                              (int *)ctx->counts.p, a.st));
        CKC(cudaMemcpyAsync(S.counts, ctx->counts.p, m * sizeof(int), cudaMemcpyDeviceToHost, a.st));
        CKC(cudaStreamSynchronize(a.st));

        // exact sizes of this chunk
        long long S_total = 0, bm_words = 0;
        int blocks = 0, sort_tiles = 0;
        for (int s = 0; s < m; ++s) {
            CamInfo &ci = S.cams[s];
            ci.count = S.counts[s];
            ci.seg_off = S_total;
            ci.nw = (ci.count + 31) / 32;
            ci.bm_off = bm_words;
            S_total += ci.count;
            bm_words += (long long)((ci.TX + STILE - 1) / STILE) * ((ci.TY + STILE - 1) / STILE) * ci.nw;
            S.blkpre[s] = blocks;
            blocks += (ci.count + BIN_RANKS - 1) / BIN_RANKS;
            S.segstart[s] = ci.seg_off;
            S.segcount[s] = ci.count;
            S.sorttiles[s] = sort_tiles;
            sort_tiles += sort_tiles_for(ci.count);
        }
        S.sorttiles[m] = sort_tiles;
        S.blkpre[m] = blocks;
        S.tilepre[m] = tiles_total;
        st.survivors += S_total;
        const size_t Sx = (size_t)std::max<long long>(S_total, 1);
        CKS(grow(ctx, ctx->rec, Sx * sizeof(SlotRec)));
        CKS(grow(ctx, ctx->keys, Sx * 4));
        CKS(grow(ctx, ctx->vals, Sx * 4));
        CKS(grow(ctx, ctx->tkeys, Sx * 4));
        CKS(grow(ctx, ctx->tvals, Sx * 4));
        CKS(grow(ctx, ctx->rrect, Sx * sizeof(uint2)));
        CKS(grow(ctx, ctx->srect, Sx * sizeof(uint2)));
        CKS(grow(ctx, ctx->bitmap, (size_t)std::max<long long>(bm_words, 1) * 4));
        CKS(grow(ctx, ctx->sorthist, (size_t)std::max(sort_tiles, 1) * 256 * 4));
        CKC(cudaMemcpyAsync(ctx->cams.p, S.cams, m * sizeof(CamInfo), cudaMemcpyHostToDevice, a.st));
        CKC(cudaMemcpyAsync(ctx->blkpre.p, S.blkpre, (m + 1) * sizeof(int), cudaMemcpyHostToDevice, a.st));
        CKC(cudaMemcpyAsync(ctx->tilepre.p, S.tilepre, (m + 1) * sizeof(int), cudaMemcpyHostToDevice, a.st));
        CKC(cudaMemcpyAsync(ctx->segstart.p, S.segstart, m * sizeof(long long), cudaMemcpyHostToDevice, a.st));
        CKC(cudaMemcpyAsync(ctx->segcount.p, S.segcount, m * sizeof(long long), cudaMemcpyHostToDevice, a.st));
        CKC(cudaMemcpyAsync(ctx->sorttiles.p, S.sorttiles, (m + 1) * sizeof(int), cudaMemcpyHostToDevice, a.st));
        CKC(launch_project_write((const Group *)ctx->groups.p, n_groups, max_bx,
                                 (const SceneDev *)ctx->d_scenes.p, (const CamInfo *)ctx->cams.p,
                                 a.vm, a.in, P, (const uint32_t *)ctx->masks.p,
                                 (const uint32_t *)ctx->woff.p, (SlotRec *)ctx->rec.p,
                                 (uint2 *)ctx->srect.p, (uint32_t *)ctx->keys.p,
                                 (uint32_t *)ctx->vals.p, std::log(cfg.alpha_min), a.st));
        if (timing) CKC(cudaEventRecord(E[1], a.st));
        if (a.upto == UPTO_PROJECT) break;
        CKC(launch_sort_segments((uint32_t *)ctx->keys.p, (uint32_t *)ctx->vals.p,
                                 (uint32_t *)ctx->tkeys.p, (uint32_t *)ctx->tvals.p,
                                 (const long long *)ctx->segstart.p,
                                 (const long long *)ctx->segcount.p, (const int *)ctx->sorttiles.p,
                                 m, sort_tiles, (uint32_t *)ctx->sorthist.p, a.st));
        if (timing) CKC(cudaEventRecord(E[2], a.st));
        CKC(launch_bin((const CamInfo *)ctx->cams.p, (const int *)ctx->blkpre.p, m, blocks, max_sup,
                       (const uint2 *)ctx->srect.p, (const uint32_t *)ctx->vals.p,
                       (uint2 *)ctx->rrect.p, (uint32_t *)ctx->bitmap.p,
                       (unsigned long long *)ctx->stats.p + 2, a.st));
        if (timing) CKC(cudaEventRecord(E[3], a.st));
        if (a.upto == UPTO_BIN) break;
        CKC(launch_composite((const CamInfo *)ctx->cams.p, (const int *)ctx->tilepre.p, m, tiles_total,
                             (const SlotRec *)ctx->rec.p, (const uint32_t *)ctx->vals.p,
                             (const uint2 *)ctx->rrect.p, (const uint32_t *)ctx->bitmap.p, C, a.rgb,
                             a.depth, a.T, (unsigned long long *)ctx->stats.p,
                             cfg.count_pairs != 0, cfg.pixels_per_thread, a.st));
        if (timing) {
            CKC(cudaEventRecord(E[4], a.st));
            ctx->ev_used = chunk_id + 1;
        }
    }
    st.n_chunks = chunk_id;
    ctx->last = st;
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

int32_t gs_abi_version(void) { return 2; }

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
    out->max_chunk_cameras = 256;
    out->camera_group = 32;
    out->count_pairs = 0;
    out->time_stages = 0;
    out->pixels_per_thread = 8;
    return GS_OK;
}

gs_status gs_context_create(const gs_config *cfg, int32_t device, gs_context **out) {
    if (!out) return GS_ERR_INVALID_ARG;
    *out = nullptr;
    gs_config c;
    if (cfg)
        c = *cfg;
    else
        gs_config_default(&c);
    if (!(c.near_plane > 0.0f) || !(c.dilation >= 0.0f) || !(c.sigma_cull > 0.0f) ||
        !(c.alpha_min > 0.0f) || !(c.alpha_max > 0.0f && c.alpha_max < 1.0f) ||
        !(c.T_min > 0.0f && c.T_min < 1.0f) || c.max_chunk_cameras < 1 || c.camera_group < 1 ||
        c.camera_group > MAX_GROUP || !(c.guard_band >= 1.0f) ||
        (c.pixels_per_thread != 2 && c.pixels_per_thread != 4 && c.pixels_per_thread != 8))
        return GS_ERR_INVALID_ARG;
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

void gs_context_destroy(gs_context *ctx) {
    if (!ctx) return;
    cudaSetDevice(ctx->device);
    cudaDeviceSynchronize();
    for (auto &s : ctx->scenes)
        if (s.storage) cudaFree(s.storage);
    DevBuf *bufs[] = {&ctx->d_scenes, &ctx->masks, &ctx->woff,    &ctx->counts,  &ctx->rec,
                      &ctx->keys,     &ctx->vals,  &ctx->tkeys,   &ctx->tvals,   &ctx->rrect, &ctx->srect,
                      &ctx->bitmap,   &ctx->cams,  &ctx->groups,  &ctx->blkpre,  &ctx->tilepre,
                      &ctx->segstart, &ctx->segcount, &ctx->stats, &ctx->h_vm,   &ctx->h_in,
                      &ctx->sorttiles, &ctx->sorthist,
                      &ctx->h_rgb,    &ctx->h_depth, &ctx->h_T};
    for (DevBuf *b : bufs)
        if (b->p) cudaFree(b->p);
    for (auto &p : ctx->pin)
        if (p.p) cudaFreeHost(p.p);
    for (auto &e : ctx->ev) cudaEventDestroy(e);
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
    const void *src[5] = {d->mean, d->log_scale, d->quat, d->logit_opacity, d->sh};
    size_t total = 0, offs[5];
    for (int i = 0; i < 5; ++i) {
        offs[i] = total;
        total += align_up(sz[i], 256);
    }
    SceneSlot slot;
    slot.live = true;
    if (total > 0) {
        cudaError_t e = cudaMalloc(&slot.storage, total);
        if (e != cudaSuccess)
            return fail(ctx, GS_ERR_OOM, "scene storage (%zu bytes): %s", total, cudaGetErrorString(e));
        for (int i = 0; i < 5; ++i)
            if (sz[i]) {
                e = cudaMemcpy((char *)slot.storage + offs[i], src[i], sz[i],
                               d->memory == GS_MEM_HOST ? cudaMemcpyHostToDevice
                                                        : cudaMemcpyDeviceToDevice);
                if (e != cudaSuccess) {
                    cudaFree(slot.storage);
                    return fail(ctx, GS_ERR_CUDA, "scene copy: %s", cudaGetErrorString(e));
                }
            }
    }
    char *b = (char *)slot.storage;
    slot.dev.mean = b + offs[0];
    slot.dev.log_scale = b + offs[1];
    slot.dev.quat = b + offs[2];
    slot.dev.logit = b + offs[3];
    slot.dev.sh = b + offs[4];
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
    RenderArgs a{n_cams,
                 scene_ids,
                 (const float *)ctx->h_vm.p,
                 (const float *)ctx->h_in.p,
                 width,
                 height,
                 nullptr,
                 nullptr,
                 nullptr,
                 (float *)ctx->h_rgb.p,
                 (float *)ctx->h_depth.p,
                 final_T ? (float *)ctx->h_T.p : nullptr,
                 st,
                 UPTO_ALL};
    CKS(render_impl(ctx, a));
    CKC(cudaMemcpyAsync(rgb, ctx->h_rgb.p, px * 3 * 4, cudaMemcpyDeviceToHost, st));
    CKC(cudaMemcpyAsync(depth, ctx->h_depth.p, px * 4, cudaMemcpyDeviceToHost, st));
    if (final_T) CKC(cudaMemcpyAsync(final_T, ctx->h_T.p, px * 4, cudaMemcpyDeviceToHost, st));
    CKC(cudaStreamSynchronize(st));
    return GS_OK;
}

gs_status gs_get_stats(gs_context *ctx, gs_stats *out) {
    if (!ctx || !out) return GS_ERR_INVALID_ARG;
    if (ctx->stats_pending && ctx->stats.p) {
        CKC(cudaSetDevice(ctx->device));
        unsigned long long h[8];
        CKC(cudaMemcpy(h, ctx->stats.p, sizeof(h), cudaMemcpyDeviceToHost));
        ctx->last.pairs_evaluated = (int64_t)h[0];
        ctx->last.pairs_alpha = (int64_t)h[1];
        ctx->last.intersections = (int64_t)h[2];
        ctx->last.warp_iters = (int64_t)h[3];
        ctx->last.warp_iters_box = (int64_t)h[4];
        ctx->last.warp_iters_blend = (int64_t)h[5];
        float ms[4] = {0, 0, 0, 0};
        for (int c = 0; c < ctx->ev_used; ++c) {
            cudaEvent_t *E = &ctx->ev[5 * c];
            CKC(cudaEventSynchronize(E[4]));
            for (int k = 0; k < 4; ++k) {
                float t = 0;
                CKC(cudaEventElapsedTime(&t, E[k], E[k + 1]));
                ms[k] += t;
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
    CKS(render_impl(ctx, a));
    CKC(cudaStreamSynchronize(st));
    const long long S = ctx->last.survivors;
    *n_out = S;
    if (S > cap) return fail(ctx, GS_ERR_CAPACITY, "%lld survivors > cap %lld", S, (long long)cap);
    std::vector<SlotRec> h((size_t)S);
    if (S) CKC(cudaMemcpy(h.data(), ctx->rec.p, S * sizeof(SlotRec), cudaMemcpyDeviceToHost));
    const float L2E = 1.4426950408889634f;
    for (long long i = 0; i < S; ++i) {
        const SlotRec &R = h[i];
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
    CKS(render_impl(ctx, a));
    CKC(cudaStreamSynchronize(st));
    const long long S = ctx->last.survivors;
    const int TX = (width + 15) / 16, TY = (height + 15) / 16, tiles = TX * TY;
    const int SX = (TX + STILE - 1) / STILE, SY = (TY + STILE - 1) / STILE;
    const int nw = (int)((S + 31) / 32);
    std::vector<SlotRec> rec((size_t)S);
    std::vector<uint32_t> vals((size_t)S), bm((size_t)SX * SY * nw);
    std::vector<uint2> rr((size_t)S);
    if (S) {
        CKC(cudaMemcpy(rec.data(), ctx->rec.p, S * sizeof(SlotRec), cudaMemcpyDeviceToHost));
        CKC(cudaMemcpy(vals.data(), ctx->vals.p, S * 4, cudaMemcpyDeviceToHost));
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
    CKS(grow(ctx, ctx->tkeys, (size_t)std::max<int64_t>(n, 1) * 4));
    CKS(grow(ctx, ctx->tvals, (size_t)std::max<int64_t>(n, 1) * 4));
    CKS(grow(ctx, ctx->sorttiles, tiles.size() * sizeof(int)));
    CKS(grow(ctx, ctx->sorthist, (size_t)std::max(nt, 1) * 256 * 4));
    CKC(cudaMemcpyAsync(ctx->sorttiles.p, tiles.data(), tiles.size() * sizeof(int),
                        cudaMemcpyHostToDevice, st));
    CKC(launch_sort_segments(keys, vals, (uint32_t *)ctx->tkeys.p, (uint32_t *)ctx->tvals.p,
                             (const long long *)seg_start, (const long long *)seg_count,
                             (const int *)ctx->sorttiles.p, n_seg, nt,
                             (uint32_t *)ctx->sorthist.p, st));
    CKC(cudaStreamSynchronize(st));  // the host tile table must outlive the copy
    return GS_OK;
}

}  // extern "C"
