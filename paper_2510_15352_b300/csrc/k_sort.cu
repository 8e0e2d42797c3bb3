// k_sort.cu -- segmented, stable LSD radix sort of uint32 keys with uint32
// values (gs_sort_segments, the scene set-up's Morton order). The render's
// depth order has its own kernels (k_depth.cu).
//
// Four 8-bit passes, ping-ponging between the caller's buffers and scratch.
// Every segment is cut into tiles of 2048 keys and each pass runs three
// kernels over all tiles of all segments at once:
//   k_sort_hist    -- digit histogram of every tile;
//   k_sort_offsets -- per segment: where each (tile, digit) run starts
//                     (digits in order, tiles in order within a digit);
//   k_sort_scatter -- stable rank of each key among equal digits of its tile;
//                     the tile is put in sorted order in shared memory, then
//                     written out run by run (coalesced) at segment start +
//                     run start + rank.
// A block finds its tile's segment base, offset and key count by searching the
// segment table.
// Stable rank inside a tile: warp w takes keys [256 w, 256 w + 256) in rounds
// of 32; a key's rank is (equal digits in earlier warps) + (equal digits in
// earlier rounds of its warp) + (equal digits in lower lanes of its round,
// from eight ballots over the digit bits).
#include <algorithm>

#include "gs_internal.cuh"

namespace gsk {

namespace {

constexpr int ST = 256;         // threads per sort block
constexpr int SIPT = 8;         // keys per thread
constexpr int TK = ST * SIPT;   // keys per tile
constexpr int SNW = ST / 32;    // warps per block

__device__ __forceinline__ int find_seg(const int *__restrict__ tile_start, int n_seg, int tile) {
    int lo = 0, hi = n_seg - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tile_start[mid] <= tile)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

// Where tile `tile` lies, from the segment table.
__device__ __forceinline__ SortTile tile_of(const long long *__restrict__ seg_start,
                                            const long long *__restrict__ seg_count,
                                            const int *__restrict__ tile_start, int n_seg, int tile) {
    const int s = find_seg(tile_start, n_seg, tile);
    const int t0 = (tile - tile_start[s]) * TK;
    return SortTile{seg_start[s], t0, (int)min((long long)TK, seg_count[s] - t0),
                    (int)seg_count[s], s};
}

// Digit histogram of every tile: BITS-bit digit at `shift`.
template <int BITS>
__global__ void __launch_bounds__(ST)
    k_sort_hist(const uint32_t *__restrict__ keys, const long long *__restrict__ seg_start,
                const long long *__restrict__ seg_count, const int *__restrict__ tile_start,
                int n_seg, int shift, uint32_t *__restrict__ hist, const int *__restrict__ nt_dev,
                int nt_host) {
    constexpr int ND = 1 << BITS;
    __shared__ uint32_t h[ND];
    const int nt = nt_dev ? *nt_dev : nt_host;
    for (int tile = blockIdx.x; tile < nt; tile += gridDim.x) {
    const SortTile T = tile_of(seg_start, seg_count, tile_start, n_seg, tile);
    const uint32_t *k = keys + T.seg_base + T.t0;
    for (int d = threadIdx.x; d < ND; d += ST) h[d] = 0;
    uint32_t kv[SIPT];
#pragma unroll
    for (int r = 0; r < SIPT; ++r) {
        const int j = r * ST + threadIdx.x;
        kv[r] = j < T.nk ? k[j] : 0u;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < SIPT; ++r)
        if (r * ST + (int)threadIdx.x < T.nk) atomicAdd(&h[(kv[r] >> shift) & (ND - 1)], 1u);
    __syncthreads();
    for (int d = threadIdx.x; d < ND; d += ST) hist[(long long)tile * ND + d] = h[d];
    __syncthreads();  // h is cleared for the next tile of this block
    }
}

// One block of ND threads per segment; thread d owns digit d. In place:
// hist[tile][d] becomes the offset (within the segment) of the run of digit d
// of that tile.
template <int BITS>
__global__ void __launch_bounds__(1 << BITS, 1024 >> BITS)  // 64 registers: 4 blocks per SM
    k_sort_offsets(const int *__restrict__ tile_start, uint32_t *__restrict__ hist) {
    constexpr int ND = 1 << BITS, NWD = ND / 32;
    const int s = blockIdx.x, d = threadIdx.x, lane = d & 31, warp = d >> 5;
    const int t0 = tile_start[s], t1 = tile_start[s + 1];
    uint32_t run_d = 0;
    // 16 independent loads in flight, then the running sum over them
    for (int tb = t0; tb < t1; tb += 16) {
        uint32_t c[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) c[k] = tb + k < t1 ? hist[(long long)(tb + k) * ND + d] : 0u;
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            if (tb + k < t1) hist[(long long)(tb + k) * ND + d] = run_d;
            run_d += c[k];
        }
    }
    // exclusive scan of the digit totals
    __shared__ uint32_t ws[NWD];
    uint32_t incl = run_d;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    uint32_t before = 0;
#pragma unroll
    for (int w = 0; w < NWD; ++w) before += w < warp ? ws[w] : 0u;
    const uint32_t base = before + incl - run_d;
    for (int tb = t0; tb < t1; tb += 16) {
        uint32_t c[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) c[k] = tb + k < t1 ? hist[(long long)(tb + k) * ND + d] : 0u;
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (tb + k < t1) hist[(long long)(tb + k) * ND + d] = c[k] + base;
    }
}

// Five resident blocks per SM: the scatter waits on its loads more than it
// computes, and the extra block hides more of that.
template <int BITS>
__global__ void __launch_bounds__(ST, 5)
    k_sort_scatter(const uint32_t *__restrict__ sk, const uint32_t *__restrict__ sv,
                   uint32_t *__restrict__ dk, uint32_t *__restrict__ dv,
                   const long long *__restrict__ seg_start, const long long *__restrict__ seg_count,
                   const int *__restrict__ tile_start, int n_seg, int shift,
                   const uint32_t *__restrict__ offs, const int *__restrict__ nt_dev, int nt_host,
                   int index_vals) {
    constexpr int ND = 1 << BITS, DPT = ND / ST;  // digits per thread (1 or 2)
    static_assert(ND % ST == 0, "digits are a multiple of the block size");
    __shared__ uint32_t wcnt[SNW][ND];
    __shared__ uint32_t tdig[ND];   // where each digit starts in the tile's sorted order
    __shared__ uint32_t tmove[ND];  // run start in the segment minus tdig (>= 0)
    __shared__ uint32_t dsum[SNW];
    __shared__ uint32_t skey[TK], sval[TK];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nt = nt_dev ? *nt_dev : nt_host;
    for (int tile = blockIdx.x; tile < nt; tile += gridDim.x) {
    const SortTile T = tile_of(seg_start, seg_count, tile_start, n_seg, tile);
    const long long base = T.seg_base;
    const long long t0 = T.t0;
    const long long i0 = t0 + (long long)warp * (32 * SIPT);
    const long long n = t0 + T.nk;  // keys of the segment up to the end of this tile
    const int nk = T.nk;            // keys in this tile
    uint32_t toff[DPT];  // where the tile's run of digit q * ST + tid starts in the segment
#pragma unroll
    for (int q = 0; q < DPT; ++q) toff[q] = offs[(long long)tile * ND + q * ST + tid];
    for (int j = lane; j < ND; j += 32) wcnt[warp][j] = 0;
    uint32_t kr[SIPT], vr[SIPT], rk[SIPT];
#pragma unroll
    for (int r = 0; r < SIPT; ++r) {
        const long long i = i0 + r * 32 + lane;
        kr[r] = i < n ? sk[base + i] : 0u;
        // index_vals: the values are the positions in the segment (not read)
        vr[r] = i < n ? (index_vals ? (uint32_t)i : sv[base + i]) : 0u;
    }
    __syncwarp();
    const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
    for (int r = 0; r < SIPT; ++r) {
        const bool ok = i0 + r * 32 + lane < n;
        const uint32_t d = (kr[r] >> shift) & (ND - 1);
        // lanes whose digit differs from this lane's in some bit: per bit, the
        // ballot XOR this lane's bit spread over 32 bits (0 - bit)
        uint32_t differ = ~__ballot_sync(0xffffffffu, ok);
#pragma unroll
        for (int b = 0; b < BITS; ++b) {
            const uint32_t t = (d >> b) & 1u;
            const uint32_t bal = __ballot_sync(0xffffffffu, t);
            differ |= bal ^ (0u - t);
        }
        const uint32_t peers = ~differ;
        const uint32_t below = peers & lt;
        const uint32_t before = wcnt[warp][d];
        rk[r] = before + __popc(below);
        __syncwarp();
        if (ok && below == 0u) wcnt[warp][d] = before + __popc(peers);  // lowest peer lane
        __syncwarp();
    }
    __syncthreads();
    // per digit (thread tid owns digits tid and tid + ST): exclusive prefix over
    // warps, and the digit's total for the tile
    uint32_t tot[DPT];
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        uint32_t run_d = 0;
#pragma unroll
        for (int w = 0; w < SNW; ++w) {
            const uint32_t c = wcnt[w][q * ST + tid];
            wcnt[w][q * ST + tid] = run_d;
            run_d += c;
        }
        tot[q] = run_d;
    }
    // exclusive prefix of the digit totals over digits: where each digit's keys
    // start in the tile's sorted order (digits q * ST + tid, in order of q then tid)
    uint32_t carry = 0;
#pragma unroll
    for (int q = 0; q < DPT; ++q) {
        uint32_t incl = tot[q];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) dsum[warp] = incl;
        __syncthreads();
        uint32_t before = 0, all = 0;
#pragma unroll
        for (int w = 0; w < SNW; ++w) {
            before += w < warp ? dsum[w] : 0u;
            all += dsum[w];
        }
        const uint32_t td = carry + before + incl - tot[q];
        tdig[q * ST + tid] = td;
        tmove[q * ST + tid] = toff[q] - td;
        carry += all;
        __syncthreads();
    }
    // the tile in sorted order in shared memory ...
#pragma unroll
    for (int r = 0; r < SIPT; ++r) {
        if (i0 + r * 32 + lane < n) {
            const uint32_t d = (kr[r] >> shift) & (ND - 1);
            const uint32_t pos = tdig[d] + wcnt[warp][d] + rk[r];
            skey[pos] = kr[r];
            sval[pos] = vr[r];
        }
    }
    __syncthreads();
    // ... then written out in that order: consecutive threads write
    // consecutive addresses within each digit's run
    for (int p = tid; p < nk; p += ST) {
        const uint32_t key = skey[p];
        const uint32_t d = (key >> shift) & (ND - 1);
        const long long at = base + tmove[d] + p;
        dk[at] = key;
        dv[at] = sval[p];
    }
    __syncthreads();  // shared arrays are rebuilt for the next tile of this block
    }
}

template <int BITS>
void sort_pass(const uint32_t *sk, const uint32_t *sv, uint32_t *dk, uint32_t *dv,
               const long long *seg_start, const long long *seg_count, const int *tile_start,
               int n_seg, int n_tiles, int shift, uint32_t *hist, cudaStream_t s,
               const int *n_tiles_dev, bool index_vals) {
    k_sort_hist<BITS><<<n_tiles, ST, 0, s>>>(sk, seg_start, seg_count, tile_start, n_seg, shift,
                                             hist, n_tiles_dev, n_tiles);
    k_sort_offsets<BITS><<<n_seg, 1 << BITS, 0, s>>>(tile_start, hist);
    k_sort_scatter<BITS><<<n_tiles, ST, 0, s>>>(sk, sv, dk, dv, seg_start, seg_count, tile_start,
                                                n_seg, shift, hist, n_tiles_dev, n_tiles,
                                                index_vals);
}

}  // namespace

int sort_tiles_for(long long count) { return (int)((count + TK - 1) / TK); }

cudaError_t launch_sort_segments(uint32_t *keys, uint32_t *vals, uint32_t *tmp_keys,
                                 uint32_t *tmp_vals, const long long *seg_start,
                                 const long long *seg_count, const int *tile_start, int n_seg,
                                 int n_tiles, uint32_t *hist, cudaStream_t s,
                                 const int *n_tiles_dev, bool index_vals) {
    if (n_seg == 0 || n_tiles == 0) return cudaSuccess;
    uint32_t *src_k = keys, *src_v = vals, *dst_k = tmp_keys, *dst_v = tmp_vals;
    for (int pass = 0; pass < 4; ++pass) {
        sort_pass<8>(src_k, src_v, dst_k, dst_v, seg_start, seg_count, tile_start, n_seg, n_tiles,
                     8 * pass, hist, s, n_tiles_dev, index_vals && pass == 0);
        uint32_t *t;
        t = src_k; src_k = dst_k; dst_k = t;
        t = src_v; src_v = dst_v; dst_v = t;
    }
    // four passes: the sorted data is back in keys / vals
    return cudaGetLastError();
}

}  // namespace gsk
