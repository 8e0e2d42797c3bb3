// k_composite.cu -- per-tile front-to-back alpha compositing of RGB and
// expected depth (the 3DGS rendering step the paper uses as its renderer,
// Sec. 3.2; depth comes out of the same pass, Sec. 3.3 / Fig. 4).
//
// One block per (camera, 16x16 tile), 128 threads, two pixels per thread in
// the same row (columns c and c+8), so the per-Gaussian row terms (dy, c'dy^2,
// b'dy) are shared by both pixels and each staged record is read from shared
// memory once per two pixels. A warp covers 4 rows x 16 columns.
//
// The tile's list is its bitmap row (bit r = the survivor of depth rank r
// covers the tile). Each round reads 128 bitmap words (4096 ranks), turns the
// set bits into a rank list in shared memory (block-wide prefix of popcounts),
// then stages the records of 128 ranks at a time in shared memory and
// composites them. Per pixel and Gaussian:
//   p = a'dx^2 + b'dx dy + c'dy^2 + log2(o) = log2(o e^power)
//   p < log2(alpha_min): skip;  alpha = min(alpha_max, 2^p)
//   T' = T (1 - alpha); T' < T_min: the pixel stops (this Gaussian not added)
//   C += alpha T rgb, D += alpha T z, T = T'.
// A warp whose pixels have all stopped skips the arithmetic (warp vote); the
// block stops reading its list once every pixel has stopped (block vote).
// No tensor cores: this is not a dense contraction.
#include "gs_internal.cuh"

namespace gsk {

namespace {

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

struct PixState {
    float T, r, g, b, d;
    bool done;
    uint32_t ev, al;
};

template <bool STATS>
__device__ __forceinline__ void blend(PixState &s, float px, const float4 &g0, float bdy,
                                      float base, const float4 &g1, const float4 &g2,
                                      const CompParams &P) {
    if (s.done) return;
    const float dx = px - g0.x;
    const float p = fmaf(fmaf(g0.z, dx, bdy), dx, base);
    if (STATS) s.ev++;
    if (p < P.log2_alpha_min) return;
    if (STATS) s.al++;
    const float alpha = fminf(P.alpha_max, ex2_approx(p));
    const float Tn = s.T * (1.0f - alpha);
    if (Tn < P.T_min) {
        s.done = true;
        return;
    }
    const float w = alpha * s.T;
    s.r = fmaf(w, g2.x, s.r);
    s.g = fmaf(w, g2.y, s.g);
    s.b = fmaf(w, g2.z, s.b);
    s.d = fmaf(w, g1.z, s.d);
    s.T = Tn;
}

template <bool STATS>
__global__ void __launch_bounds__(COMP_THREADS)
    k_composite(const CamInfo *__restrict__ cams, const int *__restrict__ tile_prefix,
                int n_slots, const CRec *__restrict__ crec, const uint32_t *__restrict__ bitmap,
                CompParams P, float *__restrict__ rgb, float *__restrict__ depth,
                float *__restrict__ finalT, unsigned long long *__restrict__ stats) {
    __shared__ float4 s0[COMP_BATCH], s1[COMP_BATCH], s2[COMP_BATCH];
    __shared__ uint32_t slist[COMP_WORDS * 32];
    __shared__ uint32_t wsum[COMP_THREADS / 32];

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
    const int xa = tx * TILE + (tid & 7), xb = xa + 8, y = ty * TILE + (tid >> 3);
    const float pxa = xa + 0.5f, pxb = xb + 0.5f, py = y + 0.5f;
    const bool ina = xa < ci.W && y < ci.H, inb = xb < ci.W && y < ci.H;
    PixState A = {1.0f, 0.0f, 0.0f, 0.0f, 0.0f, !ina, 0u, 0u};
    PixState B = {1.0f, 0.0f, 0.0f, 0.0f, 0.0f, !inb, 0u, 0u};

    const uint32_t *bm = bitmap + ci.bm_off + (long long)t * ci.nw;
    const CRec *cr = crec + ci.seg_off;
    for (int wb = 0; wb < ci.nw; wb += COMP_WORDS) {
        if (!__syncthreads_or(!(A.done && B.done))) break;
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
        for (int k = 0; k < COMP_THREADS / 32; ++k) {
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
            if (tid < nb) {
                const CRec R = cr[slist[j0 + tid]];
                s0[tid] = R.a;
                s1[tid] = R.b;
                s2[tid] = R.c;
            }
            __syncthreads();
            if (__any_sync(0xffffffffu, !(A.done && B.done))) {
                for (int j = 0; j < nb; ++j) {
                    const float4 g0 = s0[j], g1 = s1[j], g2 = s2[j];
                    const float dy = py - g0.y;
                    const float base = fmaf(g1.x * dy, dy, g1.y);
                    const float bdy = g0.w * dy;
                    blend<STATS>(A, pxa, g0, bdy, base, g1, g2, P);
                    blend<STATS>(B, pxb, g0, bdy, base, g1, g2, P);
                }
            }
            if (!__syncthreads_or(!(A.done && B.done))) goto finished;
        }
    }
finished:
    const long long img = (long long)ci.user * ci.H;
    if (ina) {
        const long long p = (img + y) * ci.W + xa;
        rgb[3 * p + 0] = fmaf(A.T, P.bg[0], A.r);
        rgb[3 * p + 1] = fmaf(A.T, P.bg[1], A.g);
        rgb[3 * p + 2] = fmaf(A.T, P.bg[2], A.b);
        depth[p] = A.d;
        if (finalT) finalT[p] = A.T;
    }
    if (inb) {
        const long long p = (img + y) * ci.W + xb;
        rgb[3 * p + 0] = fmaf(B.T, P.bg[0], B.r);
        rgb[3 * p + 1] = fmaf(B.T, P.bg[1], B.g);
        rgb[3 * p + 2] = fmaf(B.T, P.bg[2], B.b);
        depth[p] = B.d;
        if (finalT) finalT[p] = B.T;
    }
    if (STATS) {
        unsigned long long ev = (unsigned long long)A.ev + B.ev, al = (unsigned long long)A.al + B.al;
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

}  // namespace

cudaError_t launch_composite(const CamInfo *cams, const int *tile_prefix, int n_slots,
                             int n_tiles, const CRec *crec, const uint32_t *bitmap,
                             CompParams C, float *rgb, float *depth, float *final_T,
                             unsigned long long *stats, bool collect, cudaStream_t s) {
    if (n_tiles == 0) return cudaSuccess;
    if (collect)
        k_composite<true><<<n_tiles, COMP_THREADS, 0, s>>>(cams, tile_prefix, n_slots, crec,
                                                           bitmap, C, rgb, depth, final_T, stats);
    else
        k_composite<false><<<n_tiles, COMP_THREADS, 0, s>>>(cams, tile_prefix, n_slots, crec,
                                                            bitmap, C, rgb, depth, final_T, stats);
    return cudaGetLastError();
}

}  // namespace gsk
