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
#include "gs_internal.cuh"

namespace gsk {

namespace {

template <int RPT>  // ranks per thread
__global__ void __launch_bounds__(BIN_THREADS)
    k_bin(const CamInfo *__restrict__ cams, const int *__restrict__ blk_prefix,
          const int2 *__restrict__ bintab, int n_slots,
          const uint2 *__restrict__ srect, const uint32_t *__restrict__ vals,
          uint2 *__restrict__ rrect, uint32_t *__restrict__ bitmap,
          unsigned long long *__restrict__ n_isect) {
    constexpr int BIN_RANKS = RPT * BIN_THREADS, BIN_WORDS = BIN_RANKS / 32;
    extern __shared__ uint32_t sbm[];  // [BIN_WORDS][P]
    const int nblk = blk_prefix[n_slots];
    for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    const int2 bt = bintab[blk];  // (camera, first rank) of this binning block
    const CamInfo ci = cams[bt.x];
    const int r0 = bt.y;
    const int SX = (ci.TX + STILE - 1) / STILE, SY = (ci.TY + STILE - 1) / STILE;
    const int nsup = SX * SY;
    const int P = nsup | 1;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < P * BIN_WORDS; i += BIN_THREADS) sbm[i] = 0u;
    // rank r0 + j * BIN_THREADS + tid: word j * (BIN_THREADS / 32) + warp, bit lane
    uint32_t slot[RPT];
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const int r = r0 + j * BIN_THREADS + tid;
        slot[j] = r < ci.count ? vals[ci.seg_off + r] : 0u;
    }
    uint2 d[RPT];
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const int r = r0 + j * BIN_THREADS + tid;
        d[j] = r < ci.count ? srect[ci.seg_off + slot[j]] : make_uint2(1u, 1u);  // empty rect
    }
    __syncthreads();  // sbm cleared
    unsigned long long area = 0;
#pragma unroll
    for (int j = 0; j < RPT; ++j) {
        const int r = r0 + j * BIN_THREADS + tid;
        if (r >= ci.count) continue;
        rrect[ci.seg_off + r] = d[j];
        const int x0 = (int)(d[j].x & 0xffffu), x1 = (int)(d[j].x >> 16);
        const int y0 = (int)(d[j].y & 0xffffu), y1 = (int)(d[j].y >> 16);
        if (x1 >= x0 && y1 >= y0) {
            area += (unsigned long long)(x1 - x0 + 1) * (y1 - y0 + 1);
            const uint32_t bit = 1u << lane;
            const int word = j * (BIN_THREADS / 32) + warp;
            for (int sy = y0 / STILE; sy <= y1 / STILE; ++sy)
                for (int sx = x0 / STILE; sx <= x1 / STILE; ++sx)
                    atomicOr(&sbm[word * P + sy * SX + sx], bit);
        }
    }
    __syncthreads();
    const int w0 = r0 >> 5;
    const int nwb = min(BIN_WORDS, ci.nw - w0);
    for (int i = tid; i < nsup * BIN_WORDS; i += BIN_THREADS) {
        const int st = i / BIN_WORDS, k = i - st * BIN_WORDS;
        if (k < nwb) bitmap[ci.bm_off + (long long)st * ci.nw + w0 + k] = sbm[k * P + st];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) area += __shfl_down_sync(0xffffffffu, area, o);
    if (lane == 0 && area) atomicAdd(n_isect, area);
    __syncthreads();  // sbm is cleared for the next block of ranks
    }
}

}  // namespace

int bin_ranks_for(int n_super) {
    return (size_t)(n_super | 1) * (BIN_RANKS / 32) * sizeof(uint32_t) <= (size_t)BIN_SMEM_MAX
               ? BIN_RANKS
               : BIN_RANKS_SMALL;
}

cudaError_t launch_bin(const CamInfo *cams, const int *blk_prefix, const int2 *bintab, int n_slots,
                       int n_blocks,
                       int n_super, int bin_ranks, const uint2 *srect, const uint32_t *vals,
                       uint2 *rrect, uint32_t *bitmap, unsigned long long *n_isect,
                       cudaStream_t s) {
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
                                             n_isect);
    return cudaGetLastError();
}

}  // namespace gsk
