// bin_core.cuh -- the body of one binning item (see k_bin.cu): NTH threads
// take RPT consecutive depth ranks each (NTH * RPT ranks from r0 of camera
// ci; ranks at or past lim are left out: their bits are zero), build the rank
// column's words of every super-tile row in shared memory (sbm: [NTH * RPT /
// 32][P] words, P = super-tiles | 1), write the rank-ordered rects and the
// words out, and add the item's (survivor, tile) pairs of ranks at or past
// from to *n_isect. Used by the binning kernel (256 threads per item) and by the
// persistent binning + compositing kernel (one warp per item).
#pragma once

#include "gs_internal.cuh"

namespace gsk {

template <int NTH, int RPT>
__device__ __forceinline__ void bin_item(uint32_t *sbm, const CamInfo &ci, int r0, int lim, int from,
                                         const uint2 *__restrict__ srect,
                                         const uint32_t *__restrict__ vals,
                                         uint2 *__restrict__ rrect, uint32_t *__restrict__ bitmap,
                                         unsigned long long *__restrict__ n_isect) {
    constexpr int RANKS = RPT * NTH, WORDS = RANKS / 32;
    const int SX = (ci.TX + STILE - 1) / STILE, SY = (ci.TY + STILE - 1) / STILE;
    const int nsup = SX * SY;
    const int P = nsup | 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < P * WORDS; i += NTH) sbm[i] = 0u;
    // rank r0 + j * NTH + tid: word j * (NTH / 32) + warp, bit lane
    uint32_t slot[RPT];
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const int r = r0 + j * NTH + tid;
        slot[j] = r < lim ? vals[ci.seg_off + r] : 0u;
    }
    uint2 d[RPT];
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const int r = r0 + j * NTH + tid;
        d[j] = r < lim ? srect[ci.seg_off + slot[j]] : make_uint2(1u, 1u);  // empty rect
    }
    __syncthreads();  // sbm cleared
    unsigned long long area = 0;
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const int r = r0 + j * NTH + tid;
        if (r >= lim) continue;
        rrect[ci.seg_off + r] = d[j];
        const int x0 = (int)(d[j].x & 0xffffu), x1 = (int)(d[j].x >> 16);
        const int y0 = (int)(d[j].y & 0xffffu), y1 = (int)(d[j].y >> 16);
        if (x1 >= x0 && y1 >= y0) {
            if (r >= from) area += (unsigned long long)(x1 - x0 + 1) * (y1 - y0 + 1);
            const uint32_t bit = 1u << lane;
            const int word = j * (NTH / 32) + warp;
            for (int sy = y0 / STILE; sy <= y1 / STILE; ++sy)
                for (int sx = x0 / STILE; sx <= x1 / STILE; ++sx)
                    atomicOr(&sbm[word * P + sy * SX + sx], bit);
        }
    }
    __syncthreads();
    const int w0 = r0 >> 5;
    const int nwb = min(WORDS, ci.nw - w0);
    for (int i = tid; i < nsup * WORDS; i += NTH) {
        const int st = i / WORDS, k = i - st * WORDS;
        if (k < nwb) bitmap[ci.bm_off + (long long)st * ci.nw + w0 + k] = sbm[k * P + st];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) area += __shfl_down_sync(0xffffffffu, area, o);
    if (lane == 0 && area) atomicAdd(n_isect, area);
    __syncthreads();  // sbm is cleared by the next item of this block
}

}  // namespace gsk
