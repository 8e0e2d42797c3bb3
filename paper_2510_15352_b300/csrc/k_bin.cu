// k_bin.cu -- binning of depth-sorted survivors: the last, most significant
// digit (the tile) of the (camera, tile, depth, index) order of the 3DGS
// renderer (Sec. 3.2 of the paper uses that renderer), applied as a stable
// counting sort in bitmap form.
//
// Representation: camera c has S_c survivors in depth-rank order. Each
// 64x64-pixel super-tile (4x4 tiles) owns a bitmap row of ceil(S_c/32) words;
// bit r is set when the tile rect of the survivor of rank r meets the
// super-tile. Next to it, rrect[r] holds that survivor's exact tile rect. A
// tile's list -- every survivor whose rect holds the tile, in (depth, index)
// order -- is the set bits of its super-tile's row, read in increasing order,
// whose rect holds the tile. No per-intersection key, global scan or second
// sort is needed, and every bitmap word is written once.
//
// A block takes 1,024 consecutive ranks of one camera (4 per thread, their
// slot and rect loads issued together): it builds the 32 words of that rank
// column for every super-tile of the camera in shared memory, then writes them
// out as 128-byte segments. In shared memory the words are word-major with an
// odd row pitch (P >= number of super-tiles): the lanes of a warp set bits of
// one word in the super-tiles their rects meet, which then fall in different
// banks, and the write-out reads 32 words of one super-tile from 32 banks.
#include "bin_core.cuh"
#include "proj_core.cuh"

namespace gsk {

namespace {

// phase 0: every binning block of the chunk, all ranks; phase 1 / 2: the
// blocks of the phase map, the ranks before the camera's cut / all ranks (the
// second phase counts pairs from the cut on).
template <int RPT>  // ranks per thread
__global__ void __launch_bounds__(BIN_THREADS)
    k_bin(const CamInfo *__restrict__ cams, const int *__restrict__ blk_prefix,
          const int2 *__restrict__ bintab, int n_slots,
          const uint2 *__restrict__ srect, const uint32_t *__restrict__ vals,
          uint2 *__restrict__ rrect, uint32_t *__restrict__ bitmap,
          unsigned long long *__restrict__ n_isect, const DepthCut *__restrict__ cut, int phase,
          const int *__restrict__ map) {
    extern __shared__ uint32_t sbm[];  // [ranks / 32][P]
    const int nblk = phase == 0 ? blk_prefix[n_slots] : map[2];
    for (int bv = blockIdx.x; bv < nblk; bv += gridDim.x) {
        const int blk = phase == 0 ? bv : phase_item(map, n_slots, MAP_BINS, bv);
        const int2 bt = bintab[blk];  // (camera, first rank) of this binning block
        const CamInfo ci = cams[bt.x];
        const int lim = phase == 1 ? min(ci.count, cut[bt.x].pos) : ci.count;
        const int from = phase == 2 ? cut[bt.x].pos : 0;
        bin_item<BIN_THREADS, RPT>(sbm, ci, bt.y, lim, from, srect, vals, rrect, bitmap, n_isect);
    }
}

// The record and rect of rank r's survivor (Gaussian g of scene sc, camera
// constants cam), as the projection's write pass makes them: the same
// projection, the SH colour from the coefficient row in quads of four with the
// even and odd terms on the two lanes of a packed accumulator, the alpha box.
// The record goes to position at (rank order) of rec.
template <typename A>
__device__ __forceinline__ uint2 rank_record(const CamProj &cam, const SceneDev &sc, long long g,
                                             const ProjParams &P, float ln_alpha_min,
                                             float4 *__restrict__ rec, long long at) {
    constexpr float LOG2E_ = 1.4426950408889634f;
    const float4 g0 = sc.geo_rows[4 * g], g1 = sc.geo_rows[4 * g + 1];
    const float4 g2 = sc.geo_rows[4 * g + 2], g3 = sc.geo_rows[4 * g + 3];
    GaussGeo G;
    G.mx = g0.x;
    G.my = g0.y;
    G.mz = g0.z;
    G.M[0] = g1.x; G.M[1] = g1.y; G.M[2] = g1.z; G.M[3] = g1.w;
    G.M[4] = g2.x; G.M[5] = g2.y; G.M[6] = g2.z; G.M[7] = g2.w;
    G.M[8] = g3.x;
    G.smax2 = 0.0f;  // (the culling bound only)
    const float log2o = g0.w;
    Proj pr;
    project<false>(cam, G, P, pr);
    // SH colour: view direction, basis, then per channel the quads of the row
    float dx, dy, dz;
    sh_dir(cam.cpos, G.mx, G.my, G.mz, dx, dy, dz);
    float Y[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) Y[k] = 0.0f;
    sh_basis(3, dx, dy, dz, Y);
    const A *row = reinterpret_cast<const A *>(sc.sh_rows) + 48 * g;
    float rgb[3];
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float2 acc = make_float2(0.5f, 0.0f);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            float w[4];
            if constexpr (std::is_same<A, float>::value) {
                const float4 v = reinterpret_cast<const float4 *>(row)[4 * ch + j];
                w[0] = v.x; w[1] = v.y; w[2] = v.z; w[3] = v.w;
            } else {
                const uint2 v = reinterpret_cast<const uint2 *>(row)[4 * ch + j];
                A h[4];
                memcpy(h, &v, sizeof(v));
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    if constexpr (std::is_same<A, __half>::value)
                        w[e] = __half2float(h[e]);
                    else
                        w[e] = __bfloat162float(h[e]);
                }
            }
            acc = __ffma2_rn(make_float2(w[0], w[1]), make_float2(Y[4 * j], Y[4 * j + 1]), acc);
            acc = __ffma2_rn(make_float2(w[2], w[3]), make_float2(Y[4 * j + 2], Y[4 * j + 3]), acc);
        }
        rgb[ch] = fmaxf(__fadd_rn(acc.x, acc.y), 0.0f);
    }
    const float q = 2.0f * fmaf(log2o, 0.6931471805599453f, -ln_alpha_min);
    float hx = -1e30f, hy = -1e30f;
    if (q >= 0.0f) {
        hx = fmaf(1.002f, sqrt_a(__fmul_rn(q, pr.sa)), 0.02f);
        hy = fmaf(1.002f, sqrt_a(__fmul_rn(q, pr.sc)), 0.02f);
    }
    rec[rec_a(at)] = make_float4(pr.u, pr.v, hx, hy);
    rec[rec_b(at)] = make_float4(__fmul_rn(-0.5f * LOG2E_, pr.A), __fmul_rn(-LOG2E_, pr.B),
                     __fmul_rn(-0.5f * LOG2E_, pr.C), log2o);
    rec[rec_c(at)] = make_float4(rgb[0], rgb[1], rgb[2], pr.z);
    return make_uint2((uint32_t)pr.x0 | ((uint32_t)pr.x1 << 16),
                      (uint32_t)pr.y0 | ((uint32_t)pr.y1 << 16));
}

// The blocks of a phase map (as k_bin), with each binned rank's record and rect
// computed here (rank_record, for the block's scene's appearance type: one
// camera, so one scene, per block) instead of gathered by slot.
template <int RPT>
__global__ void __launch_bounds__(BIN_THREADS)
    k_bin_rec(const CamInfo *__restrict__ cams, const int2 *__restrict__ bintab, int n_slots,
              const SceneDev *__restrict__ scenes, const CamProj *__restrict__ camtab, ProjParams P,
              float ln_alpha_min, const uint32_t *__restrict__ oidx,
              const uint32_t *__restrict__ vals, float4 *__restrict__ rec,
              uint2 *__restrict__ rrect, uint32_t *__restrict__ bitmap,
              unsigned long long *__restrict__ n_isect, const DepthCut *__restrict__ cut,
              int phase, const int *__restrict__ map) {
    constexpr int NTH = BIN_THREADS, RANKS = RPT * NTH, WORDS = RANKS / 32;
    extern __shared__ uint32_t sbm[];  // [ranks / 32][P]
    __shared__ CamProj scam;
    const int nblk = map[2];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int bv = blockIdx.x; bv < nblk; bv += gridDim.x) {
        const int2 bt = bintab[phase_item(map, n_slots, MAP_BINS, bv)];
        const CamInfo ci = cams[bt.x];
        const int r0 = bt.y;
        const int lim = phase == 1 ? min(ci.count, cut[bt.x].pos) : ci.count;
        const int from = phase == 2 ? cut[bt.x].pos : 0;
        const SceneDev sc = scenes[ci.scene];
        const int SX = (ci.TX + STILE - 1) / STILE, SY = (ci.TY + STILE - 1) / STILE;
        const int nsup = SX * SY, Pp = nsup | 1;
        if (tid < 7) reinterpret_cast<float4 *>(&scam)[tid] = reinterpret_cast<const float4 *>(&camtab[bt.x])[tid];
        for (int i = tid; i < Pp * WORDS; i += NTH) sbm[i] = 0u;
        // the Gaussians of the thread's ranks, each step's loads issued together
        // (slot, caller index, position: three dependent gathers, not twelve)
        uint32_t gi[RPT];
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            const int r = r0 + j * NTH + tid;
            gi[j] = r < lim ? vals[ci.seg_off + r] : 0u;
        }
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            const int r = r0 + j * NTH + tid;
            gi[j] = r < lim ? oidx[ci.seg_off + gi[j]] : 0u;
        }
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            const int r = r0 + j * NTH + tid;
            gi[j] = r < lim ? (uint32_t)sc.pos_of[gi[j]] : 0u;
        }
        __syncthreads();  // sbm cleared, scam loaded
        unsigned long long area = 0;
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            const int r = r0 + j * NTH + tid;
            if (r >= lim) continue;
            const long long g = gi[j];
            const long long at = ci.seg_off + r;
            const uint2 d =
                sc.app_dtype == DT_F32 ? rank_record<float>(scam, sc, g, P, ln_alpha_min, rec, at)
                : sc.app_dtype == DT_F16
                    ? rank_record<__half>(scam, sc, g, P, ln_alpha_min, rec, at)
                    : rank_record<__nv_bfloat16>(scam, sc, g, P, ln_alpha_min, rec, at);
            rrect[ci.seg_off + r] = d;
            const int x0 = (int)(d.x & 0xffffu), x1 = (int)(d.x >> 16);
            const int y0 = (int)(d.y & 0xffffu), y1 = (int)(d.y >> 16);
            if (x1 >= x0 && y1 >= y0) {
                if (r >= from) area += (unsigned long long)(x1 - x0 + 1) * (y1 - y0 + 1);
                const uint32_t bit = 1u << lane;
                const int word = j * (NTH / 32) + warp;
                for (int sy = y0 / STILE; sy <= y1 / STILE; ++sy)
                    for (int sx = x0 / STILE; sx <= x1 / STILE; ++sx)
                        atomicOr(&sbm[word * Pp + sy * SX + sx], bit);
            }
        }
        __syncthreads();
        const int w0 = r0 >> 5;
        const int nwb = min(WORDS, ci.nw - w0);
        for (int i = tid; i < nsup * WORDS; i += NTH) {
            const int st = i / WORDS, k = i - st * WORDS;
            if (k < nwb) bitmap[ci.bm_off + (long long)st * ci.nw + w0 + k] = sbm[k * Pp + st];
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) area += __shfl_down_sync(0xffffffffu, area, o);
        if (lane == 0 && area) atomicAdd(n_isect, area);
        __syncthreads();  // sbm and scam are rewritten by the block's next item
    }
}

}  // namespace

cudaError_t launch_bin_rec(const CamInfo *cams, const int2 *bintab, int n_slots, int n_blocks,
                           int n_super, int bin_ranks, const SceneDev *scenes, const void *camtab,
                           ProjParams P, float ln_alpha_min, const uint32_t *oidx,
                           const uint32_t *vals, float4 *rec, uint2 *rrect, uint32_t *bitmap,
                           unsigned long long *n_isect, const DepthCut *cut, int phase,
                           const int *map, cudaStream_t s) {
    if (n_blocks == 0) return cudaSuccess;
    const size_t smem = (size_t)(n_super | 1) * (bin_ranks / 32) * sizeof(uint32_t);
    const CamProj *ct = (const CamProj *)camtab;
#define GS_BINREC(RPT)                                                                           \
    do {                                                                                         \
        auto kern = k_bin_rec<RPT>;                                                              \
        if (smem > 48 * 1024) {                                                                  \
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                                 (int)smem);                                     \
            if (e != cudaSuccess) return e;                                                      \
        }                                                                                        \
        if (phase == 2) { /* one wave of resident blocks: a second wave would double the time */ \
            int occ = 0, dev = 0, sms = 0;                                                       \
            cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, BIN_THREADS, \
                                                                          smem);                 \
            if (e == cudaSuccess) e = cudaGetDevice(&dev);                                       \
            if (e == cudaSuccess)                                                                \
                e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);           \
            if (e != cudaSuccess) return e;                                                      \
            n_blocks = std::min(n_blocks, std::max(occ * sms, 1));                               \
        }                                                                                        \
        kern<<<n_blocks, BIN_THREADS, smem, s>>>(cams, bintab, n_slots, scenes, ct, P,           \
                                                 ln_alpha_min, oidx, vals, rec, rrect, bitmap,   \
                                                 n_isect, cut, phase, map);                      \
    } while (0)
    if (bin_ranks == BIN_RANKS)
        GS_BINREC(BIN_RANKS / BIN_THREADS);
    else
        GS_BINREC(BIN_RANKS_SMALL / BIN_THREADS);
#undef GS_BINREC
    return cudaGetLastError();
}

int bin_ranks_for(int n_super) {
    return (size_t)(n_super | 1) * (BIN_RANKS / 32) * sizeof(uint32_t) <= (size_t)BIN_SMEM_MAX
               ? BIN_RANKS
               : BIN_RANKS_SMALL;
}

cudaError_t launch_bin(const CamInfo *cams, const int *blk_prefix, const int2 *bintab, int n_slots,
                       int n_blocks,
                       int n_super, int bin_ranks, const uint2 *srect, const uint32_t *vals,
                       uint2 *rrect, uint32_t *bitmap, unsigned long long *n_isect,
                       const DepthCut *cut, int phase, const int *map, cudaStream_t s) {
    if (n_blocks == 0) return cudaSuccess;
    const size_t smem = (size_t)(n_super | 1) * (bin_ranks / 32) * sizeof(uint32_t);
    auto kern = bin_ranks == BIN_RANKS ? k_bin<BIN_RANKS / BIN_THREADS>
                                       : k_bin<BIN_RANKS_SMALL / BIN_THREADS>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    kern<<<n_blocks, BIN_THREADS, smem, s>>>(cams, blk_prefix, bintab, n_slots, srect, vals, rrect, bitmap,
                                             n_isect, cut, phase, map);
    return cudaGetLastError();
}

}  // namespace gsk
