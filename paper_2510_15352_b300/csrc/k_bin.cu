// k_bin.cu -- tile binning of depth-sorted survivors: the stable counting sort
// on the tile digit that completes the (camera, tile, depth, index) order of
// the 3DGS renderer (Sec. 3.2 of the paper uses that renderer).
//
// Representation: for camera c with S_c survivors in depth-rank order, tile t
// owns a bitmap row of ceil(S_c/32) words; bit r is set when the survivor of
// rank r covers the tile. Reading a row's set bits in increasing order yields
// exactly the tile's list in (depth, index) order, so no per-intersection key,
// global scan or second sort is needed, and every word is written once.
//
// A block takes 256 consecutive ranks of one camera: it builds the 8 words of
// that rank column for every tile of the camera in shared memory (32 B per
// tile), then writes them out as 32-byte segments. The same pass copies each
// survivor's record into rank order with the compositing constants folded in.
#include "gs_internal.cuh"

namespace gsk {

namespace {

constexpr float LOG2E = 1.4426950408889634f;

__global__ void __launch_bounds__(BIN_RANKS)
    k_bin(const CamInfo *__restrict__ cams, const int *__restrict__ blk_prefix, int n_slots,
          const SlotRec *__restrict__ rec, const uint32_t *__restrict__ vals,
          CRec *__restrict__ crec, uint32_t *__restrict__ bitmap,
          unsigned long long *__restrict__ n_isect, float ln_alpha_min) {
    extern __shared__ uint32_t sbm[];  // [tiles][BIN_WORDS]
    int lo = 0, hi = n_slots - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (blk_prefix[mid] <= (int)blockIdx.x)
            lo = mid;
        else
            hi = mid - 1;
    }
    const CamInfo ci = cams[lo];
    const int r0 = ((int)blockIdx.x - blk_prefix[lo]) * BIN_RANKS;
    const int tiles = ci.TX * ci.TY;
    const int tid = threadIdx.x;
    for (int i = tid; i < tiles * BIN_WORDS; i += BIN_RANKS) sbm[i] = 0u;
    __syncthreads();
    const int r = r0 + tid;
    const int lane = tid & 31, warp = tid >> 5;
    int x0 = 0, y0 = 0, w = 0;
    uint32_t a = 0;
    if (r < ci.count) {
        const uint32_t slot = vals[ci.seg_off + r];
        const SlotRec R = rec[ci.seg_off + slot];
        // box of the alpha >= alpha_min region d^T Sigma'^-1 d <= q = 2 ln(o / alpha_min):
        // half extents sqrt(q Sigma'_00), sqrt(q Sigma'_11), widened so that float32
        // rounding of the per-pixel test can never pass a pixel outside it
        const float q = 2.0f * (logf(R.a.w) - ln_alpha_min);
        float hx = -1e30f, hy = -1e30f;
        if (q >= 0.0f) {
            hx = fmaf(1.001f, sqrtf(q * R.c.w), 0.01f);
            hy = fmaf(1.001f, sqrtf(q * __uint_as_float(R.d.w)), 0.01f);
        }
        CRec C;
        C.a = make_float4(R.a.x, R.a.y, hx, hy);
        C.b = make_float4(-0.5f * LOG2E * R.b.x, -LOG2E * R.b.y, -0.5f * LOG2E * R.b.z,
                          log2f(R.a.w));
        C.c = make_float4(R.c.x, R.c.y, R.c.z, R.a.z);
        crec[ci.seg_off + r] = C;
        x0 = (int)(R.d.x & 0xffffu);
        const int x1 = (int)(R.d.x >> 16);
        y0 = (int)(R.d.y & 0xffffu);
        const int y1 = (int)(R.d.y >> 16);
        if (x1 >= x0 && y1 >= y0) {
            w = x1 - x0 + 1;
            a = (uint32_t)(w * (y1 - y0 + 1));
        }
    }
    // Load-balanced expansion of the warp's 32 rects into (rank, tile) pairs:
    // pair e belongs to the first lane whose inclusive area prefix exceeds e.
    uint32_t incl = a;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += v;
    }
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    for (uint32_t b = 0; b < total; b += 32) {
        const uint32_t e = b + lane;
        int l = 0;
#pragma unroll
        for (int st = 16; st > 0; st >>= 1) {
            const uint32_t v = __shfl_sync(0xffffffffu, incl, l + st - 1);
            if (v <= e) l += st;
        }
        const uint32_t oi = __shfl_sync(0xffffffffu, incl, l);
        const uint32_t oa = __shfl_sync(0xffffffffu, a, l);
        const int ox = __shfl_sync(0xffffffffu, x0, l);
        const int oy = __shfl_sync(0xffffffffu, y0, l);
        const int ow = __shfl_sync(0xffffffffu, w, l);
        if (e < total) {
            const int local = (int)(e - (oi - oa));
            const int dy = local / ow;
            const int tx = ox + (local - dy * ow), ty = oy + dy;
            atomicOr(&sbm[(ty * ci.TX + tx) * BIN_WORDS + warp], 1u << l);
        }
    }
    unsigned long long area = (lane == 0) ? total : 0ull;
    __syncthreads();
    const int w0 = r0 >> 5;
    const int nwb = min(BIN_WORDS, ci.nw - w0);
    for (int i = tid; i < tiles * BIN_WORDS; i += BIN_RANKS) {
        const int t = i / BIN_WORDS, k = i - t * BIN_WORDS;
        if (k < nwb) bitmap[ci.bm_off + (long long)t * ci.nw + w0 + k] = sbm[i];
    }
    if (area) atomicAdd(n_isect, area);
}

}  // namespace

cudaError_t launch_bin(const CamInfo *cams, const int *blk_prefix, int n_slots, int n_blocks,
                       int max_tiles, const SlotRec *rec, const uint32_t *vals, CRec *crec,
                       uint32_t *bitmap, unsigned long long *n_isect, float ln_alpha_min,
                       cudaStream_t s) {
    if (n_blocks == 0) return cudaSuccess;
    const size_t smem = (size_t)max_tiles * BIN_WORDS * sizeof(uint32_t);
    cudaError_t e = cudaFuncSetAttribute(k_bin, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_bin<<<n_blocks, BIN_RANKS, smem, s>>>(cams, blk_prefix, n_slots, rec, vals, crec, bitmap,
                                            n_isect, ln_alpha_min);
    return cudaGetLastError();
}

}  // namespace gsk
