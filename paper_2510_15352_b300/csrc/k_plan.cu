// k_plan.cu -- device-side sizing of one chunk, so that a render needs no host
// round trip between its kernels (and can be captured in a CUDA graph).
//
// From the per-camera survivor counts it writes each camera's survivor slot
// offset, bitmap words and offsets, the prefix tables of the binning blocks and
// of the sort tiles, the segment table of the sort and one SortTile entry per
// sort tile. When the chunk's
// survivors exceed the workspace, it records the size needed, raises the status
// word (and the context's sticky word, kept across calls until the host reports
// it) and plans an empty chunk (every count 0), so the later kernels do
// nothing and the host can grow the workspace and render again.
#include "gs_internal.cuh"

namespace gsk {

namespace {

constexpr int PT = 1024;

template <typename T>
__device__ __forceinline__ T block_excl_scan(T v, T &total, T *wsum) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const T t = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += t;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    T before = 0;
    total = 0;
    for (int w = 0; w < PT / 32; ++w) {
        const T x = wsum[w];
        before += w < warp ? x : (T)0;
        total += x;
    }
    __syncthreads();
    return before + incl - v;
}

__global__ void __launch_bounds__(PT)
    k_plan(CamInfo *__restrict__ cams, const int *__restrict__ counts, int m,
           int bin_ranks, long long cap_survivors, int *__restrict__ blkpre,
           int *__restrict__ sorttiles,
           long long *__restrict__ segstart, long long *__restrict__ segcount,
           int *__restrict__ status,
           long long *__restrict__ need,
           unsigned long long *__restrict__ survivors,
           unsigned long long *__restrict__ sticky) {
    __shared__ long long ws64[PT / 32];
    __shared__ int ws32[PT / 32];
    __shared__ long long carry_s, carry_bm;
    __shared__ int carry_bb, carry_st, overflow;
    const int tid = threadIdx.x;
    // 1. is the chunk's survivor total within the workspace?
    long long part = 0;
    for (int i = tid; i < m; i += PT) part += counts[i];
    long long tot;
    block_excl_scan<long long>(part, tot, ws64);
    if (tid == 0) {
        overflow = tot > cap_survivors;
        atomicMax((unsigned long long *)need, (unsigned long long)tot);  // largest chunk
        if (sticky) atomicMax(sticky, (unsigned long long)tot);  // kept across calls
        if (overflow) {
            *status = GS_STATUS_CAPACITY;
            if (sticky) atomicOr(sticky + 1, 1ull);  // reported by a later call or gs_sync
        } else
            atomicAdd(survivors, (unsigned long long)tot);
        carry_s = carry_bm = 0;
        carry_bb = carry_st = 0;
    }
    __syncthreads();
    // 2. offsets (all zero-sized when the chunk does not fit)
    for (int b = 0; b < m; b += PT) {
        const int i = b + tid;
        long long c = 0, bmw = 0;
        int bb = 0, st = 0, nw = 0;
        if (i < m && !overflow) {
            const CamInfo ci = cams[i];
            c = counts[i];
            nw = (int)((c + 31) / 32);
            const int nsup = ((ci.TX + STILE - 1) / STILE) * ((ci.TY + STILE - 1) / STILE);
            bmw = (long long)nsup * nw;
            bb = (int)((c + bin_ranks - 1) / bin_ranks);
            st = (int)((c + SORT_TILE_KEYS - 1) / SORT_TILE_KEYS);
        }
        long long t_s, t_bm;
        int t_bb, t_st;
        const long long off_s = block_excl_scan<long long>(c, t_s, ws64) + carry_s;
        const long long off_bm = block_excl_scan<long long>(bmw, t_bm, ws64) + carry_bm;
        const int off_bb = block_excl_scan<int>(bb, t_bb, ws32) + carry_bb;
        const int off_st = block_excl_scan<int>(st, t_st, ws32) + carry_st;
        if (i < m) {
            cams[i].count = (int)c;
            cams[i].seg_off = off_s;
            cams[i].nw = nw;
            cams[i].bm_off = off_bm;
            blkpre[i] = off_bb;
            sorttiles[i] = off_st;
            segstart[i] = off_s;
            segcount[i] = c;
        }
        __syncthreads();
        if (tid == 0) {
            carry_s += t_s;
            carry_bm += t_bm;
            carry_bb += t_bb;
            carry_st += t_st;
        }
        __syncthreads();
    }
    if (tid == 0) {
        blkpre[m] = carry_bb;
        sorttiles[m] = carry_st;
    }
}

// The binning blocks' (camera, first rank) and the sort tiles' entries of the
// chunk, one thread per entry over the whole grid (k_plan's single block wrote
// the per-camera prefixes): an entry's camera is the last whose prefix is at
// most the entry's index (cameras without blocks share the next one's prefix).
__device__ __forceinline__ int owner(const int *__restrict__ pre, int m, int g) {
    int lo = 0, hi = m - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (pre[mid] <= g)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__global__ void k_plan_tables(int m, int bin_ranks, const int *__restrict__ blkpre,
                              const int *__restrict__ sorttiles,
                              const long long *__restrict__ segstart,
                              const long long *__restrict__ segcount, SortTile *__restrict__ stiles,
                              int2 *__restrict__ bintab) {
    const int nbb = blkpre[m], nst = sorttiles[m];
    const int stride = gridDim.x * blockDim.x;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < nbb; g += stride) {
        const int c = owner(blkpre, m, g);
        bintab[g] = make_int2(c, (g - blkpre[c]) * bin_ranks);
    }
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < nst; g += stride) {
        const int c = owner(sorttiles, m, g);
        const int t0 = (g - sorttiles[c]) * SORT_TILE_KEYS;
        const long long cnt = segcount[c];
        stiles[g] = SortTile{segstart[c], t0, (int)min((long long)SORT_TILE_KEYS, cnt - t0),
                             (int)cnt, c};
    }
}

// The work items of one phase of the progressive depth order (DepthCut): one
// block, the chunk's segments PT at a time. Phase 1 lists every segment: its
// first-phase windows (win1), its binning blocks up to the cut (all of them
// when there is no second phase) and all its sort tiles. Phase 2 lists the
// segments whose flag is set: their windows from win1 on, their binning blocks
// from the one holding the cut on (that block bins its ranks below the cut
// again, with the same result) and all their sort tiles.
__global__ void __launch_bounds__(PT)
    k_phase_map(int phase, int m, const DepthCut *__restrict__ cut, const int *__restrict__ flag,
                const int *__restrict__ tile_start, const int *__restrict__ blkpre, int bin_ranks,
                int *__restrict__ map, const int *__restrict__ rn,
                unsigned long long *__restrict__ stats) {
    constexpr int WPS = SORT_TILE_KEYS / DEPTH_WINDOW;  // window items per sort tile
    __shared__ int ws32[PT / 32];
    __shared__ int carry[4];  // listed segments, windows, binning blocks, sort tiles
    const int tid = threadIdx.x;
    const int M1 = m + 1;
    int *pre_w = map + 4, *base_w = pre_w + M1;
    int *pre_b = base_w + M1, *base_b = pre_b + M1;
    int *pre_t = base_b + M1, *base_t = pre_t + M1;
    if (tid < 4) carry[tid] = 0;
    __syncthreads();
    for (int b = 0; b < m; b += PT) {
        const int i = b + tid;
        int in = 0, nw = 0, nb = 0, nt = 0, bw = 0, bb = 0, bt = 0;
        if (i < m) {
            const DepthCut X = cut[i];
            const int t0 = tile_start[i], t1 = tile_start[i + 1];
            const int k0 = blkpre[i], k1 = blkpre[i + 1];
            if (phase == 1) {
                in = 1;
                bw = WPS * t0;
                nw = X.win1;
                bb = k0;
                nb = min(k1 - k0, (X.pos + bin_ranks - 1) / bin_ranks);
                if (X.pos >= X.count) nb = k1 - k0;
            } else if (flag[i] && X.pos < X.count) {
                in = 1;
                bw = WPS * t0 + X.win1;
                nw = WPS * (t1 - t0) - X.win1;
                bb = k0 + X.pos / bin_ranks;
                nb = k1 - bb;
            }
            bt = t0;
            nt = in ? t1 - t0 : 0;
        }
        int t_in, t_w, t_b, t_t;
        const int o_in = block_excl_scan<int>(in, t_in, ws32) + carry[0];
        const int o_w = block_excl_scan<int>(nw, t_w, ws32) + carry[1];
        const int o_b = block_excl_scan<int>(nb, t_b, ws32) + carry[2];
        const int o_t = block_excl_scan<int>(nt, t_t, ws32) + carry[3];
        if (in) {
            pre_w[o_in] = o_w;
            base_w[o_in] = bw;
            pre_b[o_in] = o_b;
            base_b[o_in] = bb;
            pre_t[o_in] = o_t;
            base_t[o_in] = bt;
        }
        __syncthreads();
        if (tid == 0) {
            carry[0] += t_in;
            carry[1] += t_w;
            carry[2] += t_b;
            carry[3] += t_t;
        }
        __syncthreads();
    }
    if (tid == 0) {
        const int n = carry[0];
        map[0] = n;
        map[1] = carry[1];
        map[2] = carry[2];
        map[3] = carry[3];
        pre_w[n] = carry[1];
        pre_b[n] = carry[2];
        pre_t[n] = carry[3];
        if (phase == 2 && stats) {
            atomicAdd(&stats[0], (unsigned long long)n);
            atomicAdd(&stats[1], (unsigned long long)rn[0]);  // tiles that reached their cut
        }
    }
}

}  // namespace

cudaError_t launch_phase_map(int phase, int m, const DepthCut *cut, const int *flag,
                             const int *tile_start, const int *blkpre, int bin_ranks, int *map,
                             const int *rn, unsigned long long *stats, cudaStream_t s) {
    if (m <= 0) return cudaSuccess;
    k_phase_map<<<1, PT, 0, s>>>(phase, m, cut, flag, tile_start, blkpre, bin_ranks, map, rn, stats);
    return cudaGetLastError();
}

cudaError_t launch_plan(CamInfo *cams, const int *counts, int m, int bin_ranks,
                        long long cap_survivors, int *blkpre, int *sorttiles, long long *segstart,
                        long long *segcount, SortTile *stiles, int2 *bintab, int *status,
                        long long *need, unsigned long long *survivors,
                        unsigned long long *sticky, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    k_plan<<<1, PT, 0, s>>>(cams, counts, m, bin_ranks, cap_survivors, blkpre, sorttiles, segstart,
                            segcount, status, need, survivors, sticky);
    k_plan_tables<<<4 * 148, 256, 0, s>>>(m, bin_ranks, blkpre, sorttiles, segstart, segcount,
                                          stiles, bintab);
    return cudaGetLastError();
}

}  // namespace gsk
