// k_sort.cu -- segmented, stable LSD radix sort of uint32 keys with uint32
// values: the (camera, depth, index) part of the renderer's sort order.
//
// Each camera's survivors form one segment, written in Gaussian-index order by
// the projection pass; a stable sort on the depth key (float bits of z, which
// are monotone for z > 0) then orders every segment by (depth, index), the
// order in which the 3DGS renderer composites a tile (Sec. 3.2 of the paper
// uses that renderer). The tile is the last, most significant digit of the
// full key; the binning pass applies it as a stable counting sort.
//
// One block per segment, four 8-bit passes ping-ponging between the caller's
// buffers and scratch. A pass whose digit is the same for every key of the
// segment is skipped. Stability inside a pass: the block handles tiles of 4096
// keys in order; warp w takes keys [w*256, w*256+256) of the tile in rounds of
// 32, and a key's rank among equal digits before it is
//   (equal digits in earlier warps of the tile) + (earlier rounds of its warp)
//   + (lower lanes of its round, from __match_any_sync).
#include "gs_internal.cuh"

namespace gsk {

namespace {

constexpr int NW = SORT_THREADS / 32;          // warps per block
constexpr int TILE_KEYS = SORT_THREADS * SORT_IPT;

__global__ void __launch_bounds__(SORT_THREADS)
    k_sort_segments(uint32_t *__restrict__ keys, uint32_t *__restrict__ vals,
                    uint32_t *__restrict__ tkeys, uint32_t *__restrict__ tvals,
                    const long long *__restrict__ seg_start, const long long *__restrict__ seg_count) {
    const long long base = seg_start[blockIdx.x];
    const long long n = seg_count[blockIdx.x];
    if (n <= 1) return;
    __shared__ uint32_t hist[4][256];
    __shared__ uint32_t wcnt[NW][256];
    __shared__ uint32_t dbase[256];
    __shared__ uint32_t ttot[256];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < 4 * 256; i += SORT_THREADS) (&hist[0][0])[i] = 0;
    __syncthreads();
    for (long long i = tid; i < n; i += SORT_THREADS) {
        const uint32_t k = keys[base + i];
        atomicAdd(&hist[0][k & 255u], 1u);
        atomicAdd(&hist[1][(k >> 8) & 255u], 1u);
        atomicAdd(&hist[2][(k >> 16) & 255u], 1u);
        atomicAdd(&hist[3][k >> 24], 1u);
    }
    __syncthreads();

    uint32_t *sk = keys + base, *sv = vals + base;
    uint32_t *dk = tkeys + base, *dv = tvals + base;
    const uint32_t lt = (1u << lane) - 1u;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 8 * pass;
        // skip a pass whose digit is constant over the segment
        __shared__ int trivial;
        if (tid == 0) trivial = 0;
        __syncthreads();
        if (tid < 256 && (long long)hist[pass][tid] == n) trivial = 1;
        __syncthreads();
        const int skip = trivial;
        __syncthreads();  // every thread has read the flag before it is reset
        if (skip) continue;
        // exclusive scan of the digit histogram (one warp, 8 digits per lane)
        if (warp == 0) {
            uint32_t loc[8], s = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                loc[j] = s;
                s += hist[pass][lane * 8 + j];
            }
            uint32_t incl = s;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += t;
            }
            const uint32_t ex = incl - s;
#pragma unroll
            for (int j = 0; j < 8; ++j) dbase[lane * 8 + j] = ex + loc[j];
        }
        __syncthreads();
        for (long long t0 = 0; t0 < n; t0 += TILE_KEYS) {
#pragma unroll
            for (int j = 0; j < 8; ++j) wcnt[warp][lane * 8 + j] = 0;
            __syncwarp();
            uint32_t kr[SORT_IPT], vr[SORT_IPT], rk[SORT_IPT];
            // all loads of the warp's sub-tile first, so they are in flight together
#pragma unroll
            for (int r = 0; r < SORT_IPT; ++r) {
                const long long i = t0 + (long long)warp * (32 * SORT_IPT) + r * 32 + lane;
                kr[r] = i < n ? sk[i] : 0u;
                vr[r] = i < n ? sv[i] : 0u;
            }
#pragma unroll
            for (int r = 0; r < SORT_IPT; ++r) {
                const long long i = t0 + (long long)warp * (32 * SORT_IPT) + r * 32 + lane;
                const bool ok = i < n;
                const uint32_t k = kr[r];
                const uint32_t d = (k >> shift) & 255u;
                const uint32_t peers = __match_any_sync(0xffffffffu, ok ? d : 256u + lane);
                const uint32_t before = wcnt[warp][d & 255u];
                rk[r] = ok ? before + __popc(peers & lt) : 0xffffffffu;
                __syncwarp();
                if (ok && (__ffs(peers) - 1) == lane) wcnt[warp][d] = before + __popc(peers);
                __syncwarp();
            }
            __syncthreads();
            if (tid < 256) {
                uint32_t run = 0;
#pragma unroll
                for (int w = 0; w < NW; ++w) {
                    const uint32_t c = wcnt[w][tid];
                    wcnt[w][tid] = run;
                    run += c;
                }
                ttot[tid] = run;
            }
            __syncthreads();
#pragma unroll
            for (int r = 0; r < SORT_IPT; ++r) {
                if (rk[r] != 0xffffffffu) {
                    const uint32_t d = (kr[r] >> shift) & 255u;
                    const uint32_t pos = dbase[d] + wcnt[warp][d] + rk[r];
                    dk[pos] = kr[r];
                    dv[pos] = vr[r];
                }
            }
            __syncthreads();
            if (tid < 256) dbase[tid] += ttot[tid];
            __syncthreads();
        }
        uint32_t *t;
        t = sk; sk = dk; dk = t;
        t = sv; sv = dv; dv = t;
    }
    // the sorted data must end in the caller's buffers
    if (sk != keys + base) {
        for (long long i = tid; i < n; i += SORT_THREADS) {
            keys[base + i] = sk[i];
            vals[base + i] = sv[i];
        }
    }
}

}  // namespace

cudaError_t launch_sort_segments(uint32_t *keys, uint32_t *vals, uint32_t *tmp_keys,
                                 uint32_t *tmp_vals, const long long *seg_start,
                                 const long long *seg_count, int n_seg, cudaStream_t s) {
    if (n_seg == 0) return cudaSuccess;
    k_sort_segments<<<n_seg, SORT_THREADS, 0, s>>>(keys, vals, tmp_keys, tmp_vals, seg_start,
                                                   seg_count);
    return cudaGetLastError();
}

}  // namespace gsk
