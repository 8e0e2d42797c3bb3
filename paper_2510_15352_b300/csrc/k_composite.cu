// k_composite.cu -- per-tile front-to-back alpha compositing of RGB and
// expected depth (the 3DGS rendering step the paper uses as its renderer,
// Sec. 3.2; depth comes out of the same pass, Sec. 3.3 / Fig. 4).
//
// One block per (camera, 16x16 tile); PPT pixels per thread in one row
// (columns c, c + 16/PPT, ...), so the per-Gaussian row terms (dy, c'dy^2 +
// log2 o, b'dy) are shared by the thread's pixels. A warp covers 2*PPT rows.
//
// The tile's list: each round reads one word per thread of its super-tile's
// bitmap row (bit r = the survivor of depth rank r meets the 4x4-tile
// super-tile), turns the set bits into candidate ranks in shared memory
// (block prefix of popcounts), keeps the candidates whose exact tile rect
// holds this tile (order-preserving ballot compaction), then stages up to
// a batch of their records at a time in shared memory and composites them
// (COMP_BATCH = 64 for 2 and 4 pixels per thread and quads; with 8 pixels per
// thread the batch is a template parameter, 32 (default), 64, 96 or 128, chosen
// by the configuration / autotuner: a smaller batch refreshes the skip test's
// live-pixel rectangle more often, a larger one amortises the staging). Per pixel
// and Gaussian:
//   p = a'dx^2 + b'dx dy + c'dy^2 + log2(o) = log2(o e^power)
//   p < log2(alpha_min): skip;  alpha = min(alpha_max, 2^p)
//   (the cap is applied only for records that staging marks as able to reach
//   it: log2 o plus the float32 margin of p over the live pixels at least
//   log2(alpha_max); for the others 2^p < alpha_max at every pixel, so the
//   result is the same without it)
//   T' = T (1 - alpha); T' < T_min: the pixel stops (this Gaussian not added)
//   C += alpha T rgb, D += alpha T z, T = T'.
// Instruction economy (the kernel is issue-bound): when a record is staged,
// the warps some pixel of which can pass its alpha test are marked (the box of
// its alpha >= alpha_min region meets the warp's rows, and the largest value of
// the quadratic over the rows' pixel-centre rectangle reaches the threshold);
// other warps skip it (uniform branch; both tests have margins past float32
// rounding, so the skip never changes a result); the blend is branch-free: a
// stopped pixel's alpha threshold becomes +inf, which freezes it. With one
// warp per tile (8 pixels per thread) records no pixel of the tile can take
// are not staged and every staged record is blended; the other layouts blend
// only when some lane passes the alpha test (warp vote). The block stops
// reading its list once every pixel has stopped. The blend updates T and the
// sums of two pixels per packed FP32x2 instruction (each lane rounds as the
// scalar instruction would). No tensor cores: this is not a dense contraction.
#include <type_traits>

#include "bin_core.cuh"
#include "gs_internal.cuh"

namespace gsk {

namespace {

constexpr int PB_RPT = 8;     // depth ranks per lane of a persistent binning item (256)
constexpr int PB_MAXP = 129;  // super-tile row pitch its shared memory holds
constexpr int PB_BATCH_BIN = 4, PB_BATCH_TILE = 8;  // items per queue unit

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Largest value over the rectangle [X0, X1] x [Y0, Y1] of the concave quadratic
// p(x, y) = a dx^2 + b dx dy + c dy^2 + l (dx = x - u, dy = y - v; a, c < 0): the
// centre value when (u, v) lies inside, else the best of the four edges, each a
// 1-D concave quadratic whose vertex is clamped to the edge. The vertices come
// from approximate reciprocals: p at a point a few ulp from a vertex differs
// from the vertex value in second order only, far inside the skip margin.
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float max_p_rect(float u, float v, float a, float b, float c, float l,
                                            float X0, float X1, float Y0, float Y1) {
    if (u >= X0 && u <= X1 && v >= Y0 && v <= Y1) return l;
    const float ia = -0.5f * rcp_approx(a), ic = -0.5f * rcp_approx(c);
    float best = -__int_as_float(0x7f800000);
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float dx = (e ? X1 : X0) - u;
        const float dy = fminf(fmaxf(v + b * dx * ic, Y0), Y1) - v;
        best = fmaxf(best, fmaf(fmaf(a, dx, b * dy), dx, fmaf(c * dy, dy, l)));
    }
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float dy = (e ? Y1 : Y0) - v;
        const float dx = fminf(fmaxf(u + b * dy * ia, X0), X1) - u;
        best = fmaxf(best, fmaf(fmaf(a, dx, b * dy), dx, fmaf(c * dy, dy, l)));
    }
    return best;
}

// The camera of compositing block b and its first block: b / per_cam when every
// camera of the chunk has per_cam blocks (no memory access), else a search of
// the chunk's block prefix.
__device__ __forceinline__ int block_camera(const int *__restrict__ prefix, int n_slots, int per_cam,
                                            int b, int &first) {
    if (per_cam > 0) {
        const int c = b / per_cam;
        first = c * per_cam;
        return c;
    }
    int lo = 0, hi = n_slots - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (prefix[mid] <= b)
            lo = mid;
        else
            hi = mid - 1;
    }
    first = prefix[lo];
    return lo;
}

// With 8 pixels per thread (one-warp blocks) 20 blocks are resident per SM (96
// registers; shared memory allows 20). Asking for at least 18 makes ptxas fit the
// kernel in those 96 registers without spills; asking for 20 gave the same count
// with a few spilled bytes (21.33 vs 21.28 ms per 1,024 cameras), and 16 gives 116
// registers and 17 blocks (21.74 ms). Earlier layouts, per 1,024 cameras: 16
// blocks 29.0 ms, 18 blocks 28.2 ms, 20 blocks 27.2 ms, 22 blocks 28.6 ms, 24
// blocks 31.3 ms (the last two spill).
// Shared memory of one compositing block (NT = 256 / PPT threads).
template <int PPT, int CB>
struct CompSmem {
    // staged records: s0 = (u, v, a', b'), s1 = (c', log2 o, z, warp mask bits
    // and, in bit 31, "2^p may reach alpha_max"),
    // s2 = (red, green, blue, -)
    float4 s0[CB], s1[CB], s2[CB];
    // candidate ranks of one round in order; compacted in place to the ranks of
    // this tile's list (a kept candidate only moves to a lower index)
    uint32_t cand[(256 / PPT) * 32];
    uint32_t wsum[(256 / PPT) / 32];
    // per warp: the pixel-centre rectangle of its live pixels (x0, x1, y0, y1);
    // the staging skip test bounds the quadratic over it instead of over the
    // warp's rows (stopped pixels pass no alpha test), empty when x0 > x1
    float4 wl[(256 / PPT) / 32];
};

// One tile t of camera ci, composited by the whole block (see the file header).
// Arguments of a compositing launch (read from the kernel's parameter space).
struct CompArgs {
    const CamInfo *cams;
    const int *tile_prefix;
    int n_slots, per_cam;
    const float4 *rec;
    const uint32_t *vals;
    const uint2 *rrect;
    const uint32_t *bitmap;
    CompParams P;
    float *rgb, *depth, *finalT;
    unsigned long long *stats;
    const int *status;
    const DepthCut *cut;  // the progressive order's cuts (phases 1 and 2)
    Resume R;
};

// L2ONLY: the bitmap words and rank-ordered rects are read through L2 only
// (the persistent kernel writes them during the same launch, on other SMs).
// PH: 0 the whole list; 1 the ranks before camera cam's cut, the state saved
// (and the camera flagged) when live pixels remain; 2 the ranks from the cut on,
// from saved state sidx (sidx < 0: the whole list from rank 0).
template <int PPT, bool STATS, int CB, bool L2ONLY = false, int PH = 0>
__device__ __forceinline__ void composite_tile(const CamInfo ci, int t, const CompArgs &A,
                                               int cam = 0, int sidx = -1) {
    static_assert(PH == 0 || (PPT == 8 && !STATS), "the progressive order: 8 px, no counting");
    const float4 *__restrict__ rec = A.rec;
    const uint32_t *__restrict__ vals = A.vals;
    const uint2 *__restrict__ rrect = A.rrect;
    const uint32_t *__restrict__ bitmap = A.bitmap;
    const CompParams &P = A.P;
    float *__restrict__ rgb = A.rgb;
    float *__restrict__ depth = A.depth;
    float *__restrict__ finalT = A.finalT;
    unsigned long long *__restrict__ stats = A.stats;
    constexpr int NT = 256 / PPT;    // threads per block
    constexpr int CPR = 16 / PPT;    // threads per pixel row
    constexpr int NWARP = NT / 32;
    __shared__ CompSmem<PPT, CB> sm;  // one per block of every kernel that composites
    float4 *s0 = sm.s0, *s1 = sm.s1, *s2 = sm.s2, *wl = sm.wl;
    uint32_t *cand = sm.cand, *wsum = sm.wsum;
    const int tx = t % ci.TX, ty = t / ci.TX;
    const int SX = (ci.TX + STILE - 1) / STILE;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int y = ty * TILE + tid / CPR;
    const float py = y + 0.5f;
    const float INF = __int_as_float(0x7f800000);
    // Per pixel: T, colour, depth and its own alpha threshold; a pixel that has
    // stopped (or lies outside the image) has threshold +inf, so it passes no
    // further alpha test and its state stays frozen without a branch. T and the
    // sums are held for pixel pairs (k, k + 1) in float2 so the blend updates two
    // pixels per packed FP32 instruction (each lane rounds as its scalar
    // counterpart would).
    constexpr int NPR = PPT / 2;
    float2 T2[NPR], cr2[NPR], cg2[NPR], cb2[NPR], cd2[NPR];
    float thr[PPT];
    const int x0 = tx * TILE + tid % CPR;  // pixel k of this thread is x0 + k * CPR
    const float px0 = x0 + 0.5f;
#pragma unroll
    for (int k = 0; k < PPT; ++k)
        thr[k] = (x0 + k * CPR < ci.W && y < ci.H) ? P.log2_alpha_min : INF;
#pragma unroll
    for (int i = 0; i < NPR; ++i) {
        T2[i] = make_float2(1.0f, 1.0f);
        cr2[i] = cg2[i] = cb2[i] = cd2[i] = make_float2(0.0f, 0.0f);
    }
    // the bitmap words this call reads: [w_begin, w_end), the first word's ranks
    // below the cut left out when resuming
    int w_begin = 0, w_end = ci.nw;
    uint32_t first_mask = 0xffffffffu;
    bool rest = false;  // ranks past the cut remain (the cut can fall inside the last word)
    if constexpr (PH == 1) {
        const int pos = A.cut[cam].pos;
        rest = pos < ci.count;
        if (rest) w_end = (pos + 31) >> 5;
    } else if constexpr (PH == 2) {
        if (sidx >= 0) {
            const int pos = A.cut[cam].pos;
            w_begin = pos >> 5;
            first_mask = ~((1u << (pos & 31)) - 1u);
            const float4 *st = A.R.state + (long long)sidx * RESUME_STATE_F4 + lane;
#pragma unroll
            for (int i = 0; i < NPR / 2; ++i) {
                float4 v = st[(0 + i) * 32];
                T2[2 * i] = make_float2(v.x, v.y);
                T2[2 * i + 1] = make_float2(v.z, v.w);
                v = st[(2 + i) * 32];
                cr2[2 * i] = make_float2(v.x, v.y);
                cr2[2 * i + 1] = make_float2(v.z, v.w);
                v = st[(4 + i) * 32];
                cg2[2 * i] = make_float2(v.x, v.y);
                cg2[2 * i + 1] = make_float2(v.z, v.w);
                v = st[(6 + i) * 32];
                cb2[2 * i] = make_float2(v.x, v.y);
                cb2[2 * i + 1] = make_float2(v.z, v.w);
                v = st[(8 + i) * 32];
                cd2[2 * i] = make_float2(v.x, v.y);
                cd2[2 * i + 1] = make_float2(v.z, v.w);
            }
#pragma unroll
            for (int i = 0; i < PPT / 4; ++i) {
                const float4 v = st[(10 + i) * 32];
                thr[4 * i] = v.x;
                thr[4 * i + 1] = v.y;
                thr[4 * i + 2] = v.z;
                thr[4 * i + 3] = v.w;
            }
        }
    }
    const uint32_t warp_bit = 1u << warp;
    unsigned long long ev = 0, al = 0, wi = 0, wbox = 0, wbl = 0;
    auto live_rect = [&]() {
        int xlo = 0x7fffffff, xhi = -1;
#pragma unroll
        for (int k = 0; k < PPT; ++k)
            if (thr[k] != INF) {
                xlo = min(xlo, x0 + k * CPR);
                xhi = max(xhi, x0 + k * CPR);
            }
        int ylo = xhi >= 0 ? y : 0x7fffffff, yhi = xhi >= 0 ? y : -1;
        xlo = __reduce_min_sync(0xffffffffu, xlo);
        xhi = __reduce_max_sync(0xffffffffu, xhi);
        ylo = __reduce_min_sync(0xffffffffu, ylo);
        yhi = __reduce_max_sync(0xffffffffu, yhi);
        if (lane == 0)
            wl[warp] = xhi >= 0 ? make_float4(xlo + 0.5f, xhi + 0.5f, ylo + 0.5f, yhi + 0.5f)
                                : make_float4(1.0f, 0.0f, 1.0f, 0.0f);
    };
    live_rect();  // read after the block's next barrier

    const uint32_t *bm = bitmap + ci.bm_off + (long long)((ty / STILE) * SX + tx / STILE) * ci.nw;
    const long long rec0 = ci.seg_off;
    const uint32_t *cv = vals + ci.seg_off;
    const uint2 *crr = rrect + ci.seg_off;
    for (int wb = w_begin; wb < w_end; wb += NT) {
        bool live = false;
#pragma unroll
        for (int k = 0; k < PPT; ++k) live = live || thr[k] != INF;
        if (!__syncthreads_or(live)) break;
        // 1. candidates: set bits of NT words of the super-tile row, in rank order
        const int w = wb + tid;
        uint32_t word = w < w_end ? (L2ONLY ? __ldcg(bm + w) : bm[w]) : 0u;
        if (PH == 2 && w == w_begin) word &= first_mask;
        uint32_t c = __popc(word);
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
            cand[pos++] = (uint32_t)w * 32u + (uint32_t)bit;
            word &= word - 1u;
        }
        __syncthreads();
        // 2. keep the candidates whose rect holds this tile (order preserved)
        uint32_t nkept = 0;
        for (uint32_t q0 = 0; q0 < total; q0 += NT) {
            const uint32_t q = q0 + tid;
            bool keep = false;
            uint32_t rk = 0;
            if (q < total) {
                rk = cand[q];
                const uint2 rr = L2ONLY ? __ldcg(crr + rk) : crr[rk];
                keep = tx >= (int)(rr.x & 0xffffu) && tx <= (int)(rr.x >> 16) &&
                       ty >= (int)(rr.y & 0xffffu) && ty <= (int)(rr.y >> 16);
            }
            const uint32_t bal = __ballot_sync(0xffffffffu, keep);
            if (lane == 0) wsum[warp] = __popc(bal);
            __syncthreads();
            uint32_t wbefore = 0, wtotal = 0;
#pragma unroll
            for (int k = 0; k < NWARP; ++k) {
                const uint32_t v = wsum[k];
                wbefore += k < warp ? v : 0u;
                wtotal += v;
            }
            if (keep) cand[nkept + wbefore + __popc(bal & ((1u << lane) - 1u))] = rk;
            nkept += wtotal;
            __syncthreads();
        }
        // 3. composite the kept records, CB at a time. With one warp per
        // block (and no counting), a record no pixel of the tile can take is not
        // staged at all (order-preserving ballot compaction), so the blend loop
        // visits only records that may contribute; otherwise every record is
        // staged with its per-warp mask.
        constexpr bool COMPACT = NWARP == 1 && !STATS;
        for (uint32_t j0 = 0; j0 < nkept; j0 += CB) {
            int nb = (int)min((uint32_t)CB, nkept - j0);
            int nstaged = 0;
            for (int q0 = 0; q0 < nb; q0 += NT) {
                const int q = q0 + tid;
                // the record of a rank: by its slot, or (the progressive order) at
                // the rank's own position
                const uint32_t rk = cand[j0 + min(q, nb - 1)];
                const long long sl = rec0 + (PH != 0 ? (long long)rk : (long long)cv[rk]);
                const float4 a = rec[rec_a(sl)], b = rec[rec_b(sl)], cc = rec[rec_c(sl)];
                // warps some pixel of which can pass the alpha test: the box of the
                // alpha >= alpha_min region meets the warp's rows and the largest p
                // over the rows' pixel-centre rectangle reaches the threshold (with a
                // margin past float32 rounding, so no passing pair is skipped)
                uint32_t m = 0;
                bool cap = false;
#pragma unroll
                for (int k = 0; k < NWARP; ++k) {
                    const float4 L = wl[k];  // live pixel centres of warp k
                    const float X0 = L.x, X1 = L.y, Y0 = L.z, Y1 = L.w;
                    if (!(a.x + a.z >= X0 && a.x - a.z <= X1 && a.y + a.w >= Y0 && a.y - a.w <= Y1))
                        continue;  // (also when the rectangle is empty)
                    // float32 error of p grows with its terms' size: bound them
                    const float DX = fmaxf(fabsf(X0 - a.x), fabsf(X1 - a.x));
                    const float DY = fmaxf(fabsf(Y0 - a.y), fabsf(Y1 - a.y));
                    const float terms = fmaf(fabsf(b.x), DX * DX,
                                             fmaf(fabsf(b.y), DX * DY, fabsf(b.z) * DY * DY));
                    const float margin = fmaf(1e-6f, terms, 1e-3f);
                    cap = cap || b.w + margin >= P.log2_alpha_cap;
                    if (max_p_rect(a.x, a.y, b.x, b.y, b.z, b.w, X0, X1, Y0, Y1) >=
                        P.log2_alpha_min - margin)
                        m |= 1u << k;
                }
                if (q >= nb) m = 0;
                int at = q;
                bool put = q < nb;
                if (COMPACT) {
                    const uint32_t bal = __ballot_sync(0xffffffffu, m != 0);
                    at = nstaged + __popc(bal & ((1u << lane) - 1u));
                    put = m != 0;
                    nstaged += __popc(bal);
                }
                if (put) {
                    s0[at] = make_float4(a.x, a.y, b.x, b.y);
                    s1[at] = make_float4(b.z, b.w, cc.w, __uint_as_float(m | (cap ? 0x80000000u : 0u)));
                    s2[at] = cc;
                }
            }
            if (COMPACT) nb = nstaged;
            __syncthreads();
            live = false;
#pragma unroll
            for (int k = 0; k < PPT; ++k) live = live || thr[k] != INF;
            if (__any_sync(0xffffffffu, live)) {
                // p_k = a'dx^2 + b'dy dx + c'dy^2 + log2 o of the thread's pixels
                // k = 0..PPT-1 (at dx = dx0 + k CPR: P0 + k (D + k E)); true when
                // some pixel passes its alpha test (the warp vote of the layouts
                // that stage every record)
                auto quad_p = [&](const float4 &g0, const float4 &g1, float (&p)[PPT]) {
                    const float dy = py - g0.y;
                    const float dx0 = px0 - g0.x;
                    const float bdy = g0.w * dy;
                    const float t0 = fmaf(g0.z, dx0, bdy);
                    const float P0 = fmaf(t0, dx0, fmaf(g1.x * dy, dy, g1.y));
                    const float D = (float)CPR * fmaf(g0.z, dx0, t0);
                    const float E = (float)(CPR * CPR) * g0.z;
                    const float2 P02 = make_float2(P0, P0), D2 = make_float2(D, D),
                                 E2 = make_float2(E, E);
                    bool any = false;
#pragma unroll
                    for (int i = 0; i < NPR; ++i) {
                        const float2 K = make_float2((float)(2 * i), (float)(2 * i + 1));
                        const float2 pp = __ffma2_rn(K, __ffma2_rn(K, E2, D2), P02);
                        p[2 * i] = pp.x;
                        p[2 * i + 1] = pp.y;
                        any = any || pp.x >= thr[2 * i] || pp.y >= thr[2 * i + 1];
                    }
                    return any;
                };
                // CAP: std::true_type when the record may reach alpha_max
                auto blend = [&](const float (&p)[PPT], const float4 &g2, float z, auto CAP) {
                    const float2 R2 = make_float2(g2.x, g2.x), G2 = make_float2(g2.y, g2.y),
                                 B2 = make_float2(g2.z, g2.z), Z2 = make_float2(z, z);
                    const float2 M1 = make_float2(-1.0f, -1.0f);
#pragma unroll
                    for (int i = 0; i < NPR; ++i) {
                        // A pair that passes its alpha test (a stopped pixel,
                        // threshold +inf, passes none) is added when T - alpha T
                        // stays >= T_min; otherwise it is not added and the pixel
                        // stops. A pair that fails adds nothing, whatever its
                        // (unused) alpha.
                        const int k = 2 * i;
                        const bool pass0 = p[k] >= thr[k], pass1 = p[k + 1] >= thr[k + 1];
                        if (STATS) al += (pass0 ? 1u : 0u) + (pass1 ? 1u : 0u);
                        float2 alpha = make_float2(ex2_approx(p[k]), ex2_approx(p[k + 1]));
                        if constexpr (decltype(CAP)::value)
                            alpha = make_float2(fminf(P.alpha_max, alpha.x), fminf(P.alpha_max, alpha.y));
                        const float2 wgt = __fmul2_rn(alpha, T2[i]);
                        const float2 Tn = __ffma2_rn(wgt, M1, T2[i]);  // T - wgt
                        const bool ok0 = Tn.x >= P.T_min, ok1 = Tn.y >= P.T_min;
                        const float2 wa = make_float2(pass0 && ok0 ? wgt.x : 0.0f,
                                                      pass1 && ok1 ? wgt.y : 0.0f);
                        cr2[i] = __ffma2_rn(wa, R2, cr2[i]);
                        cg2[i] = __ffma2_rn(wa, G2, cg2[i]);
                        cb2[i] = __ffma2_rn(wa, B2, cb2[i]);
                        cd2[i] = __ffma2_rn(wa, Z2, cd2[i]);
                        T2[i] = __ffma2_rn(wa, M1, T2[i]);  // T - wa
                        thr[k] = pass0 && !ok0 ? INF : thr[k];
                        thr[k + 1] = pass1 && !ok1 ? INF : thr[k + 1];
                    }
                };
                auto blend_rec = [&](const float (&p)[PPT], const float4 &g2, const float4 &g1) {
                    if (__float_as_uint(g1.w) >> 31)  // warp-uniform
                        blend(p, g2, g1.z, std::true_type{});
                    else
                        blend(p, g2, g1.z, std::false_type{});
                };
                if constexpr (COMPACT) {
                    // Every staged record is blended, with no warp vote first: a
                    // record no pixel passes adds exactly nothing (its weights are
                    // zero, T and the thresholds unchanged). The vote skipped ~14 %
                    // of the staged records but cost a compare per pixel on the
                    // ALU pipe, the kernel's busiest (79.4 -> 78.7 ms per 4,096
                    // cameras without it; records in pairs then spilled: 83.5).
                    for (int j = 0; j < nb; ++j) {
                        const float4 g1 = s1[j];
                        float p[PPT];
                        quad_p(s0[j], g1, p);
                        blend_rec(p, s2[j], g1);
                    }
                } else {
                    for (int j = 0; j < nb; ++j) {
                        const float4 g1 = s1[j];  // c', log2 o, z, warp mask
                        if (STATS) {
#pragma unroll
                            for (int k = 0; k < PPT; ++k) ev += thr[k] != INF ? 1u : 0u;
                        }
                        if (STATS) wi++;
                        if (!(__float_as_uint(g1.w) & warp_bit)) continue;  // warp-uniform
                        if (STATS) wbox++;
                        float p[PPT];
                        if (!__any_sync(0xffffffffu, quad_p(s0[j], g1, p))) continue;
                        if (STATS) wbl++;
                        blend_rec(p, s2[j], g1);
                    }
                }
            }
            live = false;
#pragma unroll
            for (int k = 0; k < PPT; ++k) live = live || thr[k] != INF;
            live_rect();  // for the next staging, after this barrier
            if (!__syncthreads_or(live)) goto finished;
        }
    }
    if constexpr (PH == 1) {
        // the list ends at the camera's cut: a tile with live pixels left saves
        // its state for the second phase (which writes its outputs). (Finding
        // the camera again from the block index at this point, instead of
        // keeping it live, made the kernel 1 % slower.)
        if (rest) {
            bool live = false;
#pragma unroll
            for (int k = 0; k < PPT; ++k) live = live || thr[k] != INF;
            if (__any_sync(0xffffffffu, live)) {
                int slot = 0;
                if (lane == 0) slot = atomicAdd(A.R.n, 1);
                slot = __shfl_sync(0xffffffffu, slot, 0);
                if (slot < A.R.cap) {
                    float4 *st = A.R.state + (long long)slot * RESUME_STATE_F4 + lane;
#pragma unroll
                    for (int i = 0; i < NPR / 2; ++i) {
                        st[(0 + i) * 32] = make_float4(T2[2 * i].x, T2[2 * i].y, T2[2 * i + 1].x, T2[2 * i + 1].y);
                        st[(2 + i) * 32] = make_float4(cr2[2 * i].x, cr2[2 * i].y, cr2[2 * i + 1].x, cr2[2 * i + 1].y);
                        st[(4 + i) * 32] = make_float4(cg2[2 * i].x, cg2[2 * i].y, cg2[2 * i + 1].x, cg2[2 * i + 1].y);
                        st[(6 + i) * 32] = make_float4(cb2[2 * i].x, cb2[2 * i].y, cb2[2 * i + 1].x, cb2[2 * i + 1].y);
                        st[(8 + i) * 32] = make_float4(cd2[2 * i].x, cd2[2 * i].y, cd2[2 * i + 1].x, cd2[2 * i + 1].y);
                    }
#pragma unroll
                    for (int i = 0; i < PPT / 4; ++i)
                        st[(10 + i) * 32] = make_float4(thr[4 * i], thr[4 * i + 1], thr[4 * i + 2], thr[4 * i + 3]);
                    if (lane == 0) A.R.saved[slot] = make_int2(cam, t);
                } else if (lane == 0) {
                    const int r = atomicAdd(A.R.n + 1, 1);
                    if (r < A.R.again_cap) A.R.again[r] = make_int2(cam, t);
                }
                if (lane == 0) A.R.flag[cam] = 1;
                return;
            }
        }
    }
finished:
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int x = x0 + k * CPR;
        if (x >= ci.W || y >= ci.H) continue;
        const long long pix = ci.pix_off + (long long)y * ci.W + x;
        const float Tk = k & 1 ? T2[k >> 1].y : T2[k >> 1].x;
        const float crk = k & 1 ? cr2[k >> 1].y : cr2[k >> 1].x;
        const float cgk = k & 1 ? cg2[k >> 1].y : cg2[k >> 1].x;
        const float cbk = k & 1 ? cb2[k >> 1].y : cb2[k >> 1].x;
        const float cdk = k & 1 ? cd2[k >> 1].y : cd2[k >> 1].x;
        float o[5] = {fmaf(Tk, P.bg[0], crk), fmaf(Tk, P.bg[1], cgk),
                      fmaf(Tk, P.bg[2], cbk), cdk, Tk};
        if (P.accumulate) {  // one sub-frame of a blended image (motion blur)
            o[0] = fmaf(P.out_w, o[0], rgb[3 * pix + 0]);
            o[1] = fmaf(P.out_w, o[1], rgb[3 * pix + 1]);
            o[2] = fmaf(P.out_w, o[2], rgb[3 * pix + 2]);
            o[3] = fmaf(P.out_w, o[3], depth[pix]);
            if (finalT) o[4] = fmaf(P.out_w, o[4], finalT[pix]);
        } else if (P.out_w != 1.0f) {
#pragma unroll
            for (int q = 0; q < 5; ++q) o[q] *= P.out_w;
        }
        rgb[3 * pix + 0] = o[0];
        rgb[3 * pix + 1] = o[1];
        rgb[3 * pix + 2] = o[2];
        depth[pix] = o[3];
        if (finalT) finalT[pix] = o[4];
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
            atomicAdd(&stats[3], wi);  // per warp: the same count on every lane
            atomicAdd(&stats[4], wbox);
            atomicAdd(&stats[5], wbl);
        }
    }
}


template <int PPT, bool STATS, int CB, int PH = 0>
__global__ void __launch_bounds__(256 / PPT, PPT == 8 ? 18 : 1) k_composite(const CompArgs A) {
    if (A.status && *A.status) return;  // the chunk did not fit the workspace: nothing written
    int first;
    const int cam = block_camera(A.tile_prefix, A.n_slots, A.per_cam, (int)blockIdx.x, first);
    composite_tile<PPT, STATS, CB, false, PH>(A.cams[cam], (int)blockIdx.x - first, A, cam);
}

// The second phase of the progressive order: saved tiles resumed at their
// camera's cut, then the tiles listed to be rendered again, grid-stride.
template <int CB>
__global__ void __launch_bounds__(32, 18) k_composite_resume(const CompArgs A) {
    if (A.status && *A.status) return;
    const int ns = min(A.R.n[0], A.R.cap), na = min(A.R.n[1], A.R.again_cap);
    for (int e = blockIdx.x; e < ns + na; e += gridDim.x) {
        const int2 ct = e < ns ? A.R.saved[e] : A.R.again[e - ns];
        composite_tile<8, false, CB, false, 2>(A.cams[ct.x], ct.y, A, ct.x, e < ns ? e : -1);
        __syncthreads();  // shared memory is reused by the next tile
    }
}

// Binning and compositing of a chunk in one persistent launch (8 pixels per
// thread, one warp per block, as many blocks as are resident). A device queue
// (an atomic counter) hands out work items in order: first the binning items
// (256 depth ranks of one camera each, bin_item at warp granularity), then one
// compositing item per (camera, tile) across all cameras and scenes of the
// chunk; a warp takes a unit of 4 binning items or 8 tiles per atomic on the
// queue head. A tile may be composited only when every binning item of its camera
// is done: its warp polls the camera's counter (written after a fence by each
// binning item) with a bounded number of polls, and when the bound is reached
// it raises the timeout bit of the context's sticky status word (reported as
// GS_ERR_TIMEOUT by the host) and leaves the tile unwritten instead of
// waiting on. Binning items are handed out before any tile and never wait, so
// in a correct launch every wait ends; the bound only guards the device.
struct BinCompQueue {
    const int *blk_prefix;        // [n_slots + 1] binning items per camera, prefix
    const int2 *bintab;           // (camera, first rank) of every binning item
    const uint2 *srect;
    uint2 *rrect;
    uint32_t *bitmap;
    unsigned long long *n_isect;
    int *head;                    // next item (zero at launch)
    int *bin_done;                // [n_slots] binning items completed per camera (zero)
    int n_tiles;                  // compositing items (tiles of the chunk)
    int wait_limit;               // polls of a camera's counter before giving up
    int extra_need;               // timeout probe: camera 0 waits for this many more items
    unsigned long long *sticky;   // [1] |= 2 when a wait gives up
};

template <int CB>
__global__ void __launch_bounds__(32, 16) k_bin_composite(const CompArgs A, const BinCompQueue Q) {
    if (A.status && *A.status) return;  // the chunk did not fit the workspace: nothing written
    __shared__ uint32_t sbm[(32 * PB_RPT / 32) * PB_MAXP];
    const int lane = threadIdx.x;
    const int nbin = Q.blk_prefix[A.n_slots];
    // work units: PB_BATCH_BIN binning items or PB_BATCH_TILE tiles per unit, so a
    // warp takes one unit per atomic on the queue head (one counter for the launch)
    const int ubin = (nbin + PB_BATCH_BIN - 1) / PB_BATCH_BIN;
    const int total = ubin + (Q.n_tiles + PB_BATCH_TILE - 1) / PB_BATCH_TILE;
    int item = 0, item_end = 0;
    for (;;) {
        if (item == item_end) {
            int u = 0;
            if (lane == 0) u = atomicAdd(Q.head, 1);
            u = __shfl_sync(0xffffffffu, u, 0);
            if (u >= total) break;
            if (u < ubin) {
                item = u * PB_BATCH_BIN;
                item_end = min(item + PB_BATCH_BIN, nbin);
            } else {
                item = nbin + (u - ubin) * PB_BATCH_TILE;
                item_end = min(item + PB_BATCH_TILE, nbin + Q.n_tiles);
            }
        }
        const int it_now = item++;
        if (it_now < nbin) {
            const int item = it_now;
            const int2 bt = Q.bintab[item];
            const CamInfo ci = A.cams[bt.x];
            bin_item<32, PB_RPT>(sbm, ci, bt.y, ci.count, 0, Q.srect, A.vals, Q.rrect, Q.bitmap,
                                 Q.n_isect);
            __threadfence();  // this item's rects and words before its count
            if (lane == 0) atomicAdd(Q.bin_done + bt.x, 1);
        } else {
            const int t = it_now - nbin;
            int first;
            const int c = block_camera(A.tile_prefix, A.n_slots, A.per_cam, t, first);
            const int need = Q.blk_prefix[c + 1] - Q.blk_prefix[c] + (c == 0 ? Q.extra_need : 0);
            int ok = 1;
            if (lane == 0) {
                const volatile int *done = Q.bin_done + c;
                const volatile unsigned long long *flag = Q.sticky + 1;
                int polls = 0;
                while (*done < need) {
                    // give up after wait_limit polls, or at once when another wait has
                    // given up (so no launch ever holds more than one bounded wait per warp)
                    if (++polls > Q.wait_limit || (*flag & 2ull)) {
                        ok = 0;
                        break;
                    }
                    __nanosleep(64);
                }
                if (!ok) atomicOr(Q.sticky + 1, 2ull);
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) continue;  // the tile stays unwritten; the host reports the timeout
            __threadfence();
            const CamInfo ci = A.cams[c];
            composite_tile<8, false, CB, true>(ci, t - first, A);
        }
    }
}

// The same compositing with a 2 x 2 quad of tiles per block: warp w owns tile
// (2 qx + (w & 1), 2 qy + (w >> 1)) with 8 pixels per thread (16 rows x 2
// threads, pixels x0, x0 + 2, ...). The quad lies inside one super-tile, so
// the four warps share one scan of its bitmap row, one rect filter (the rect
// meets the quad) and one staging of every record: per record, bits 4-7 mark
// the warps whose tile lies in the record's rect (the record is in that
// tile's list) and bits 0-3 those of them some pixel of which can reach
// alpha >= alpha_min (the box test and the exact maximum of the quadratic over
// the tile's pixel-centre rectangle, with the float32 margin).
// A warp blends only the records whose bit it has, so each tile still sees
// exactly its own list, in order.
template <bool STATS>
__global__ void __launch_bounds__(128)
    k_composite_quad(const CamInfo *__restrict__ cams, const int *__restrict__ quad_prefix,
                     int n_slots, int per_cam, const float4 *__restrict__ rec,
                     const uint32_t *__restrict__ vals,
                     const uint2 *__restrict__ rrect, const uint32_t *__restrict__ bitmap,
                     CompParams P, float *__restrict__ rgb, float *__restrict__ depth,
                     float *__restrict__ finalT, unsigned long long *__restrict__ stats,
                     const int *__restrict__ status) {
    if (status && *status) return;  // the chunk did not fit the workspace: nothing written
    constexpr int PPT = 8, NT = 128, CPR = 2, NWARP = 4;
    __shared__ float4 s0[COMP_BATCH], s1[COMP_BATCH], s2[COMP_BATCH];
    __shared__ uint32_t cand[NT * 32];
    __shared__ uint32_t wsum[NWARP];

    int first;
    const CamInfo ci = cams[block_camera(quad_prefix, n_slots, per_cam, (int)blockIdx.x, first)];
    const int QX = (ci.TX + 1) >> 1;
    const int qi = (int)blockIdx.x - first;
    const int qx = qi % QX, qy = qi / QX;
    const int SX = (ci.TX + STILE - 1) / STILE;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int tx = 2 * qx + (warp & 1), ty = 2 * qy + (warp >> 1);  // this warp's tile
    const int y = ty * TILE + (lane >> 1);
    const float py = y + 0.5f;
    const float INF = __int_as_float(0x7f800000);
    float T[PPT], cr[PPT], cg[PPT], cb[PPT], cd[PPT], thr[PPT];
    const int x0 = tx * TILE + (lane & 1);
    const float px0 = x0 + 0.5f;
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        thr[k] = (x0 + k * CPR < ci.W && y < ci.H) ? P.log2_alpha_min : INF;
        T[k] = 1.0f;
        cr[k] = cg[k] = cb[k] = cd[k] = 0.0f;
    }
    const uint32_t warp_bit = 1u << warp;
    unsigned long long ev = 0, al = 0, wi = 0, wbox = 0, wbl = 0;

    const uint32_t *bm = bitmap + ci.bm_off + (long long)((2 * qy / STILE) * SX + 2 * qx / STILE) * ci.nw;
    const long long rec0 = ci.seg_off;
    const uint32_t *cv = vals + ci.seg_off;
    const uint2 *crr = rrect + ci.seg_off;
    const int qx0 = 2 * qx, qx1 = 2 * qx + 1, qy0 = 2 * qy, qy1 = 2 * qy + 1;
    for (int wb = 0; wb < ci.nw; wb += NT) {
        bool live = false;
#pragma unroll
        for (int k = 0; k < PPT; ++k) live = live || thr[k] != INF;
        if (!__syncthreads_or(live)) break;
        // 1. candidates: set bits of NT words of the super-tile row, in rank order
        const int w = wb + tid;
        uint32_t word = w < ci.nw ? bm[w] : 0u;
        uint32_t c = __popc(word);
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
            cand[pos++] = (uint32_t)w * 32u + (uint32_t)bit;
            word &= word - 1u;
        }
        __syncthreads();
        // 2. keep the candidates whose rect meets the quad (order preserved)
        uint32_t nkept = 0;
        for (uint32_t q0 = 0; q0 < total; q0 += NT) {
            const uint32_t q = q0 + tid;
            bool keep = false;
            uint32_t rk = 0;
            if (q < total) {
                rk = cand[q];
                const uint2 rr = crr[rk];
                keep = qx1 >= (int)(rr.x & 0xffffu) && qx0 <= (int)(rr.x >> 16) &&
                       qy1 >= (int)(rr.y & 0xffffu) && qy0 <= (int)(rr.y >> 16);
            }
            const uint32_t bal = __ballot_sync(0xffffffffu, keep);
            if (lane == 0) wsum[warp] = __popc(bal);
            __syncthreads();
            uint32_t wbefore = 0, wtotal = 0;
#pragma unroll
            for (int k = 0; k < NWARP; ++k) {
                const uint32_t v = wsum[k];
                wbefore += k < warp ? v : 0u;
                wtotal += v;
            }
            if (keep) cand[nkept + wbefore + __popc(bal & ((1u << lane) - 1u))] = rk;
            nkept += wtotal;
            __syncthreads();
        }
        // 3. composite the kept records, COMP_BATCH at a time
        for (uint32_t j0 = 0; j0 < nkept; j0 += COMP_BATCH) {
            const int nb = (int)min((uint32_t)COMP_BATCH, nkept - j0);
            for (int q = tid; q < nb; q += NT) {
                const uint32_t rk = cand[j0 + q];
                const long long sl = rec0 + cv[rk];
                const float4 a = rec[rec_a(sl)], b = rec[rec_b(sl)], cc = rec[rec_c(sl)];
                const uint2 d = crr[rk];  // the record's tile rect (rank order)
                const int rx0 = (int)(d.x & 0xffffu), rx1 = (int)(d.x >> 16);
                const int ry0 = (int)(d.y & 0xffffu), ry1 = (int)(d.y >> 16);
                uint32_t m = 0;
#pragma unroll
                for (int k = 0; k < NWARP; ++k) {
                    const int ktx = 2 * qx + (k & 1), kty = 2 * qy + (k >> 1);
                    if (ktx < rx0 || ktx > rx1 || kty < ry0 || kty > ry1) continue;
                    m |= 16u << k;  // in this warp's tile list
                    const float X0 = ktx * TILE + 0.5f, X1 = ktx * TILE + TILE - 0.5f;
                    const float Y0 = kty * TILE + 0.5f, Y1 = kty * TILE + TILE - 0.5f;
                    if (!(a.x + a.z >= X0 && a.x - a.z <= X1 && a.y + a.w >= Y0 && a.y - a.w <= Y1))
                        continue;
                    const float DX = fmaxf(fabsf(X0 - a.x), fabsf(X1 - a.x));
                    const float DY = fmaxf(fabsf(Y0 - a.y), fabsf(Y1 - a.y));
                    const float terms =
                        fmaf(fabsf(b.x), DX * DX, fmaf(fabsf(b.y), DX * DY, fabsf(b.z) * DY * DY));
                    const float margin = fmaf(1e-6f, terms, 1e-3f);
                    if (max_p_rect(a.x, a.y, b.x, b.y, b.z, b.w, X0, X1, Y0, Y1) >=
                        P.log2_alpha_min - margin)
                        m |= 1u << k;
                }
                s0[q] = make_float4(a.x, a.y, b.x, b.y);
                s1[q] = make_float4(b.z, b.w, cc.w, __uint_as_float(m));
                s2[q] = cc;
            }
            __syncthreads();
            live = false;
#pragma unroll
            for (int k = 0; k < PPT; ++k) live = live || thr[k] != INF;
            if (__any_sync(0xffffffffu, live)) {
                for (int j = 0; j < nb; ++j) {
                    const float4 g1 = s1[j];  // c', log2 o, z, warp masks
                    // pairs of this tile's list only (bit 4 + warp: the record's
                    // rect holds the warp's tile)
                    if (STATS && (__float_as_uint(g1.w) & (16u << warp))) {
#pragma unroll
                        for (int k = 0; k < PPT; ++k) ev += thr[k] != INF ? 1u : 0u;
                    }
                    if (STATS) wi++;
                    if (!(__float_as_uint(g1.w) & warp_bit)) continue;  // warp-uniform
                    if (STATS) wbox++;
                    const float4 g0 = s0[j];  // u, v, a', b'
                    const float dy = py - g0.y;
                    const float base = fmaf(g1.x * dy, dy, g1.y);
                    const float bdy = g0.w * dy;
                    float p[PPT];
                    bool any = false;
                    const float dx0 = px0 - g0.x;
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        const float dx = dx0 + (float)(k * CPR);
                        p[k] = fmaf(fmaf(g0.z, dx, bdy), dx, base);
                        any = any || p[k] >= thr[k];
                    }
                    if (!__any_sync(0xffffffffu, any)) continue;
                    if (STATS) wbl++;
                    const float4 g2 = s2[j];  // red, green, blue
#pragma unroll
                    for (int k = 0; k < PPT; ++k) {
                        const bool pass = p[k] >= thr[k];
                        if (STATS) al += pass ? 1u : 0u;
                        const float alpha = pass ? fminf(P.alpha_max, ex2_approx(p[k])) : 0.0f;
                        const float wgt = alpha * T[k];
                        const bool keep = T[k] - wgt >= P.T_min;
                        const float wa = keep ? wgt : 0.0f;
                        cr[k] = fmaf(wa, g2.x, cr[k]);
                        cg[k] = fmaf(wa, g2.y, cg[k]);
                        cb[k] = fmaf(wa, g2.z, cb[k]);
                        cd[k] = fmaf(wa, g1.z, cd[k]);
                        T[k] -= wa;
                        thr[k] = keep ? thr[k] : INF;
                    }
                }
            }
            live = false;
#pragma unroll
            for (int k = 0; k < PPT; ++k) live = live || thr[k] != INF;
            if (!__syncthreads_or(live)) goto finished;
        }
    }
finished:
#pragma unroll
    for (int k = 0; k < PPT; ++k) {
        const int x = x0 + k * CPR;
        if (x >= ci.W || y >= ci.H) continue;
        const long long pix = ci.pix_off + (long long)y * ci.W + x;
        float o[5] = {fmaf(T[k], P.bg[0], cr[k]), fmaf(T[k], P.bg[1], cg[k]),
                      fmaf(T[k], P.bg[2], cb[k]), cd[k], T[k]};
        if (P.accumulate) {  // one sub-frame of a blended image (motion blur)
            o[0] = fmaf(P.out_w, o[0], rgb[3 * pix + 0]);
            o[1] = fmaf(P.out_w, o[1], rgb[3 * pix + 1]);
            o[2] = fmaf(P.out_w, o[2], rgb[3 * pix + 2]);
            o[3] = fmaf(P.out_w, o[3], depth[pix]);
            if (finalT) o[4] = fmaf(P.out_w, o[4], finalT[pix]);
        } else if (P.out_w != 1.0f) {
#pragma unroll
            for (int q = 0; q < 5; ++q) o[q] *= P.out_w;
        }
        rgb[3 * pix + 0] = o[0];
        rgb[3 * pix + 1] = o[1];
        rgb[3 * pix + 2] = o[2];
        depth[pix] = o[3];
        if (finalT) finalT[pix] = o[4];
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
            atomicAdd(&stats[3], wi);
            atomicAdd(&stats[4], wbox);
            atomicAdd(&stats[5], wbl);
        }
    }
}

template <int PPT>
cudaError_t launch_ppt(const CamInfo *cams, const int *tile_prefix, int n_slots, int per_cam, int n_tiles,
                       const float4 *rec, const uint32_t *vals, const uint2 *rrect,
                       const uint32_t *bitmap, CompParams C, float *rgb, float *depth,
                       float *final_T, unsigned long long *stats, bool collect, int comp_batch,
                       const int *status, const DepthCut *cut, const Resume *R, cudaStream_t s) {
    CompArgs A{cams, tile_prefix, n_slots, per_cam, rec, vals, rrect, bitmap,
               C, rgb, depth, final_T, stats, status, cut, {}};
    if (R) A.R = *R;
#define GS_COMP(ST, CBV, PHV) k_composite<PPT, ST, CBV, PHV><<<n_tiles, 256 / PPT, 0, s>>>(A)
    if (collect) {
        GS_COMP(true, COMP_BATCH, 0);
    } else if constexpr (PPT == 8) {  // the render layout: batch sizes to tune
        if (R) {  // the progressive order's first phase
            switch (comp_batch) {
                case 32: GS_COMP(false, 32, 1); break;
                case 96: GS_COMP(false, 96, 1); break;
                case 128: GS_COMP(false, 128, 1); break;
                default: GS_COMP(false, COMP_BATCH, 1); break;
            }
        } else {
            switch (comp_batch) {
                case 32: GS_COMP(false, 32, 0); break;
                case 96: GS_COMP(false, 96, 0); break;
                case 128: GS_COMP(false, 128, 0); break;
                default: GS_COMP(false, COMP_BATCH, 0); break;
            }
        }
    } else {
        GS_COMP(false, COMP_BATCH, 0);
    }
#undef GS_COMP
    return cudaGetLastError();
}

}  // namespace

int persistent_max_super() { return PB_MAXP - 1; }

cudaError_t launch_bin_composite(const CamInfo *cams, const int *tile_prefix, int n_slots,
                                 int per_cam, int n_tiles, const float4 *rec, const uint32_t *vals,
                                 uint2 *rrect, CompParams C, float *rgb, float *depth,
                                 float *final_T, int comp_batch, const int *status,
                                 const int *blk_prefix, const int2 *bintab, const uint2 *srect,
                                 uint32_t *bitmap, unsigned long long *n_isect, int *head,
                                 int *bin_done, int wait_limit, int extra_need,
                                 unsigned long long *sticky, int grid, cudaStream_t s) {
    if (grid < 1) return cudaErrorInvalidConfiguration;
    const CompArgs A{cams, tile_prefix, n_slots, per_cam, rec, vals, rrect, bitmap,
                     C, rgb, depth, final_T, nullptr, status};
    const BinCompQueue Q{blk_prefix, bintab, srect, rrect, bitmap, n_isect, head, bin_done,
                         n_tiles, wait_limit, extra_need, sticky};
    switch (comp_batch) {
        case 32: k_bin_composite<32><<<grid, 32, 0, s>>>(A, Q); break;
        case 96: k_bin_composite<96><<<grid, 32, 0, s>>>(A, Q); break;
        case 128: k_bin_composite<128><<<grid, 32, 0, s>>>(A, Q); break;
        default: k_bin_composite<COMP_BATCH><<<grid, 32, 0, s>>>(A, Q); break;
    }
    return cudaGetLastError();
}

int persistent_grid(int comp_batch) {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    cudaError_t e;
    switch (comp_batch) {
        case 32: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bin_composite<32>, 32, 0); break;
        case 96: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bin_composite<96>, 32, 0); break;
        case 128: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bin_composite<128>, 32, 0); break;
        default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_bin_composite<COMP_BATCH>, 32, 0); break;
    }
    if (e != cudaSuccess || per < 1) return 0;
    return sms * per;
}

cudaError_t launch_composite(const CamInfo *cams, const int *tile_prefix, int n_slots,
                             int per_cam, int n_tiles, const float4 *rec, const uint32_t *vals,
                             const uint2 *rrect, const uint32_t *bitmap, CompParams C,
                             float *rgb, float *depth, float *final_T,
                             unsigned long long *stats, bool collect, int pixels_per_thread,
                             int tiles_per_block, int comp_batch, const int *status,
                             const DepthCut *cut, const Resume *R, cudaStream_t s) {
    if (n_tiles == 0) return cudaSuccess;
    if (tiles_per_block == 4) {
        if (collect)
            k_composite_quad<true><<<n_tiles, 128, 0, s>>>(cams, tile_prefix, n_slots, per_cam, rec, vals,
                                                            rrect, bitmap, C, rgb, depth, final_T,
                                                            stats, status);
        else
            k_composite_quad<false><<<n_tiles, 128, 0, s>>>(cams, tile_prefix, n_slots, per_cam, rec, vals,
                                                             rrect, bitmap, C, rgb, depth, final_T,
                                                             stats, status);
        return cudaGetLastError();
    }
    if (pixels_per_thread == 8)
        return launch_ppt<8>(cams, tile_prefix, n_slots, per_cam, n_tiles, rec, vals, rrect, bitmap, C,
                             rgb, depth, final_T, stats, collect, comp_batch, status, cut, R, s);
    if (pixels_per_thread == 4)
        return launch_ppt<4>(cams, tile_prefix, n_slots, per_cam, n_tiles, rec, vals, rrect, bitmap, C,
                             rgb, depth, final_T, stats, collect, comp_batch, status, nullptr,
                             nullptr, s);
    return launch_ppt<2>(cams, tile_prefix, n_slots, per_cam, n_tiles, rec, vals, rrect, bitmap, C, rgb,
                         depth, final_T, stats, collect, comp_batch, status, nullptr, nullptr, s);
}

cudaError_t launch_composite_resume(const CamInfo *cams, const float4 *rec, const uint32_t *vals,
                                    const uint2 *rrect, const uint32_t *bitmap, CompParams C,
                                    float *rgb, float *depth, float *final_T, int comp_batch,
                                    const int *status, const DepthCut *cut, const Resume &R,
                                    int grid, cudaStream_t s) {
    if (grid < 1) return cudaSuccess;
    const CompArgs A{cams, nullptr, 0, 0, rec, vals, rrect, bitmap, C, rgb, depth, final_T,
                     nullptr, status, cut, R};
    switch (comp_batch) {
        case 32: k_composite_resume<32><<<grid, 32, 0, s>>>(A); break;
        case 96: k_composite_resume<96><<<grid, 32, 0, s>>>(A); break;
        case 128: k_composite_resume<128><<<grid, 32, 0, s>>>(A); break;
        default: k_composite_resume<COMP_BATCH><<<grid, 32, 0, s>>>(A); break;
    }
    return cudaGetLastError();
}

}  // namespace gsk
