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
// A block takes 256 consecutive ranks of one camera: it builds the 8 words of
// that rank column for every super-tile of the camera in shared memory, then
// writes them out as 32-byte segments.
#include "gs_internal.cuh"

namespace gsk {

namespace {

__global__ void __launch_bounds__(BIN_RANKS)
    k_bin(const CamInfo *__restrict__ cams, const int *__restrict__ blk_prefix, int n_slots,
          const uint2 *__restrict__ srect, const uint32_t *__restrict__ vals,
          uint2 *__restrict__ rrect, uint32_t *__restrict__ bitmap,
          unsigned long long *__restrict__ n_isect) {
    extern __shared__ uint32_t sbm[];  // [super-tiles][BIN_WORDS]
    const int nblk = blk_prefix[n_slots];
    for (int blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
    int lo = 0, hi = n_slots - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (blk_prefix[mid] <= blk)
            lo = mid;
        else
            hi = mid - 1;
    }
    const CamInfo ci = cams[lo];
    const int r0 = (blk - blk_prefix[lo]) * BIN_RANKS;
    const int SX = (ci.TX + STILE - 1) / STILE, SY = (ci.TY + STILE - 1) / STILE;
    const int nsup = SX * SY;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int i = tid; i < nsup * BIN_WORDS; i += BIN_RANKS) sbm[i] = 0u;
    __syncthreads();
    const int r = r0 + tid;
    unsigned long long area = 0;
    if (r < ci.count) {
        const uint32_t slot = vals[ci.seg_off + r];
        const uint2 d = srect[ci.seg_off + slot];
        rrect[ci.seg_off + r] = d;
        const int x0 = (int)(d.x & 0xffffu), x1 = (int)(d.x >> 16);
        const int y0 = (int)(d.y & 0xffffu), y1 = (int)(d.y >> 16);
        if (x1 >= x0 && y1 >= y0) {
            area = (unsigned long long)(x1 - x0 + 1) * (y1 - y0 + 1);
            const uint32_t bit = 1u << lane;
            for (int sy = y0 / STILE; sy <= y1 / STILE; ++sy)
                for (int sx = x0 / STILE; sx <= x1 / STILE; ++sx)
                    atomicOr(&sbm[(sy * SX + sx) * BIN_WORDS + warp], bit);
        }
    }
    __syncthreads();
    const int w0 = r0 >> 5;
    const int nwb = min(BIN_WORDS, ci.nw - w0);
    for (int i = tid; i < nsup * BIN_WORDS; i += BIN_RANKS) {
        const int st = i / BIN_WORDS, k = i - st * BIN_WORDS;
        if (k < nwb) bitmap[ci.bm_off + (long long)st * ci.nw + w0 + k] = sbm[i];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) area += __shfl_down_sync(0xffffffffu, area, o);
    if (lane == 0 && area) atomicAdd(n_isect, area);
    __syncthreads();  // sbm is cleared for the next block of ranks
    }
}

}  // namespace

cudaError_t launch_bin(const CamInfo *cams, const int *blk_prefix, int n_slots, int n_blocks,
                       int n_super, const uint2 *srect, const uint32_t *vals, uint2 *rrect,
                       uint32_t *bitmap, unsigned long long *n_isect, cudaStream_t s) {
    if (n_blocks == 0) return cudaSuccess;
    const size_t smem = (size_t)n_super * BIN_WORDS * sizeof(uint32_t);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k_bin, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    k_bin<<<n_blocks, BIN_RANKS, smem, s>>>(cams, blk_prefix, n_slots, srect, vals, rrect, bitmap,
                                            n_isect);
    return cudaGetLastError();
}

}  // namespace gsk
