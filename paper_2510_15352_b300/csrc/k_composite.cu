// k_composite.cu -- per-tile front-to-back alpha compositing of RGB and
// expected depth (the 3DGS rendering step the paper uses as its renderer,
// Sec. 3.2; depth comes out of the same pass, Sec. 3.3 / Fig. 4).
//
// One block per (camera, 16x16 tile); PPT pixels per thread in one row
// (columns c, c + 16/PPT, ...), so the per-Gaussian row terms (dy, c'dy^2 +
// log2 o, b'dy) are shared by the thread's pixels. A warp covers 2*PPT rows.
//
// The tile's list is its bitmap row (bit r = the survivor of depth rank r
// covers the tile). Each round reads one bitmap word per thread, turns the
// set bits into a rank list in shared memory (block prefix of popcounts),
// then stages the records of up to 128 ranks at a time in shared memory and
// composites them. Per pixel and Gaussian:
//   p = a'dx^2 + b'dx dy + c'dy^2 + log2(o) = log2(o e^power)
//   p < log2(alpha_min): skip;  alpha = min(alpha_max, 2^p)
//   T' = T (1 - alpha); T' < T_min: the pixel stops (this Gaussian not added)
//   C += alpha T rgb, D += alpha T z, T = T'.
// Instruction economy (the kernel is issue-bound): a warp skips a Gaussian
// whose alpha >= alpha_min box misses the warp's pixel rows (uniform branch;
// the box is widened past float32 rounding, so the skip never changes a
// result), the blend runs only when some lane passes the alpha test (warp
// vote), and a warp whose pixels have all stopped skips the batch. The block
// stops reading its list once every pixel has stopped. No tensor cores: this
// is not a dense contraction.
#include "gs_internal.cuh"

namespace gsk {

namespace {

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int PPT, bool STATS>
__global__ void __launch_bounds__(256 / PPT)
    k_composite(const CamInfo *__restrict__ cams, const int *__restrict__ tile_prefix,
                int n_slots, const CRec *__restrict__ crec, const uint32_t *__restrict__ bitmap,
                CompParams P, float *__restrict__ rgb, float *__restrict__ depth,
                float *__restrict__ finalT, unsigned long long *__restrict__ stats) {
    constexpr int NT = 256 / PPT;    // threads per block
    constexpr int CPR = 16 / PPT;    // threads per pixel row
    constexpr int RPW = 32 / CPR;    // pixel rows per warp
    constexpr int NWARP = NT / 32;
    __shared__ float4 s0[COMP_BATCH], s1[COMP_BATCH], s2[COMP_BATCH];
    __shared__ uint32_t slist[NT * 32];
    __shared__ uint32_t wsum[NWARP];

    int lo = 0, hi = n_slots - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tile_prefix[mid] <= (int)blockIdx.x)
            lo = mid;
        else
            hi = mid - 1;
    }
    const CamInfo ci = cams[lo];
    const int t = (int)blockIdx.x - tile_prefix[lo];
    const int tx = t % ci.TX, ty = t / ci.TX;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int y = ty * TILE + tid / CPR;
    const float py = y + 0.5f;
    float px[PPT], T[PPT], cr[PPT], cg[PPT], cb[PPT], cd[PPT];
    bool done[PPT], in[PPT];
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int x = tx * TILE + tid % CPR + k * CPR;
        px[k] = x + 0.5f;
        in[k] = x < ci.W && y < ci.H;
        done[k] = !in[k];
        T[k] = 1.0f;
        cr[k] = cg[k] = cb[k] = cd[k] = 0.0f;
    }
    // pixel-centre box of this warp's rows
    const float wx0 = tx * TILE + 0.5f, wx1 = tx * TILE + TILE - 0.5f;
    const float wy0 = ty * TILE + warp * RPW + 0.5f, wy1 = wy0 + (RPW - 1);
    unsigned long long ev = 0, al = 0;

    const uint32_t *bm = bitmap + ci.bm_off + (long long)t * ci.nw;
    const CRec *recs = crec + ci.seg_off;
    for (int wb = 0; wb < ci.nw; wb += NT) {
        bool mine_done = true;
#pragma unroll
        for (int k = 0; k < PPT; ++k) mine_done = mine_done && done[k];
        if (!__syncthreads_or(!mine_done)) break;
        const int w = wb + tid;
        uint32_t word = w < ci.nw ? bm[w] : 0u;
        const uint32_t c = __popc(word);
        uint32_t incl = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += v;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        uint32_t before = 0, total = 0;
#pragma unroll
        for (int k = 0; k < NWARP; ++k) {
            const uint32_t v = wsum[k];
            before += k < warp ? v : 0u;
            total += v;
        }
        uint32_t pos = before + incl - c;
        while (word) {
            const int bit = __ffs(word) - 1;
            slist[pos++] = (uint32_t)w * 32u + (uint32_t)bit;
            word &= word - 1u;
        }
        __syncthreads();
        for (uint32_t j0 = 0; j0 < total; j0 += COMP_BATCH) {
            const int nb = (int)min((uint32_t)COMP_BATCH, total - j0);
            for (int q = tid; q < nb; q += NT) {
                const CRec R = recs[slist[j0 + q]];
                s0[q] = R.a;
                s1[q] = R.b;
                s2[q] = R.c;
            }
            __syncthreads();
            bool live = false;
#pragma unroll
            for (int k = 0; k < PPT; ++k) live = live || !done[k];
            if (__any_sync(0xffffffffu, live)) {
                for (int j = 0; j < nb; ++j) {
                    const float4 g0 = s0[j];  // u, v, hx, hy
                    if (STATS) {
#pragma unroll
                        for (int k = 0; k < PPT; ++k) ev += done[k] ? 0u : 1u;
                    }
                    if (g0.x + g0.z < wx0 || g0.x - g0.z > wx1 || g0.y + g0.w < wy0 ||
                        g0.y - g0.w > wy1)
                        continue;  // warp-uniform: no pixel of these rows can pass
                    const float4 g1 = s1[j];  // a', b', c', log2 o
                    const float dy = py - g0.y;
                    const float base = fmaf(g1.z * dy, dy, g1.w);
                    const float bdy = g1.y * dy;
                    float p[PPT];
                    bool any = false;
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        const float dx = px[k] - g0.x;
                        p[k] = fmaf(fmaf(g1.x, dx, bdy), dx, base);
                        any = any || (!done[k] && p[k] >= P.log2_alpha_min);
                    }
                    if (!__any_sync(0xffffffffu, any)) continue;
                    const float4 g2 = s2[j];  // red, green, blue, z
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        if (done[k] || p[k] < P.log2_alpha_min) continue;
                        if (STATS) al++;
                        const float alpha = fminf(P.alpha_max, ex2_approx(p[k]));
                        const float Tn = T[k] * (1.0f - alpha);
                        if (Tn < P.T_min) {
                            done[k] = true;
                            continue;
                        }
                        const float wgt = alpha * T[k];
                        cr[k] = fmaf(wgt, g2.x, cr[k]);
                        cg[k] = fmaf(wgt, g2.y, cg[k]);
                        cb[k] = fmaf(wgt, g2.z, cb[k]);
                        cd[k] = fmaf(wgt, g2.w, cd[k]);
                        T[k] = Tn;
                    }
                }
            }
            bool mine_done2 = true;
#pragma unroll
            for (int k = 0; k < PPT; ++k) mine_done2 = mine_done2 && done[k];
            if (!__syncthreads_or(!mine_done2)) goto finished;
        }
    }
finished:
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        if (!in[k]) continue;
        const int x = tx * TILE + tid % CPR + k * CPR;
        const long long pix = ((long long)ci.user * ci.H + y) * ci.W + x;
        rgb[3 * pix + 0] = fmaf(T[k], P.bg[0], cr[k]);
        rgb[3 * pix + 1] = fmaf(T[k], P.bg[1], cg[k]);
        rgb[3 * pix + 2] = fmaf(T[k], P.bg[2], cb[k]);
        depth[pix] = cd[k];
        if (finalT) finalT[pix] = T[k];
    }
    if (STATS) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            ev += __shfl_down_sync(0xffffffffu, ev, d);
            al += __shfl_down_sync(0xffffffffu, al, d);
        }
        if (lane == 0) {
            atomicAdd(&stats[0], ev);
            atomicAdd(&stats[1], al);
        }
    }
}

template <int PPT>
cudaError_t launch_ppt(const CamInfo *cams, const int *tile_prefix, int n_slots, int n_tiles,
                       const CRec *crec, const uint32_t *bitmap, CompParams C, float *rgb,
                       float *depth, float *final_T, unsigned long long *stats, bool collect,
                       cudaStream_t s) {
    if (collect)
        k_composite<PPT, true><<<n_tiles, 256 / PPT, 0, s>>>(cams, tile_prefix, n_slots, crec,
                                                             bitmap, C, rgb, depth, final_T, stats);
    else
        k_composite<PPT, false><<<n_tiles, 256 / PPT, 0, s>>>(cams, tile_prefix, n_slots, crec,
                                                              bitmap, C, rgb, depth, final_T, stats);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_composite(const CamInfo *cams, const int *tile_prefix, int n_slots,
                             int n_tiles, const CRec *crec, const uint32_t *bitmap,
                             CompParams C, float *rgb, float *depth, float *final_T,
                             unsigned long long *stats, bool collect, int pixels_per_thread,
                             cudaStream_t s) {
    if (n_tiles == 0) return cudaSuccess;
    if (pixels_per_thread == 4)
        return launch_ppt<4>(cams, tile_prefix, n_slots, n_tiles, crec, bitmap, C, rgb, depth,
                             final_T, stats, collect, s);
    return launch_ppt<2>(cams, tile_prefix, n_slots, n_tiles, crec, bitmap, C, rgb, depth,
                         final_T, stats, collect, s);
}

}  // namespace gsk
