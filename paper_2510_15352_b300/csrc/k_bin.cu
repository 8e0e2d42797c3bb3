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
