// k_project.cu -- projection, SH colour and culling of Gaussians for a batch of
// cameras (the EWA splatting step of the 3DGS renderer the paper uses, Sec. 3.2).
//
// Layout of the work: a block holds 256 consecutive (stored) Gaussians of one
// scene and loops over a group of up to 64 cameras of that scene, so each
// Gaussian's attributes are read from HBM once per camera group instead of once
// per camera. Attribute loads are structure-of-arrays: consecutive threads read
// consecutive addresses of each attribute row. Scenes are stored in spatial
// (Morton) order (k_scene.cu), so a warp's 32 Gaussians are close together and
// most such groups are, for a given camera, entirely outside the view or
// entirely inside it; the mask pass tests the group's box first and the
// Gaussians one by one only when the box straddles the view's edges.
//
// Two passes keep the survivor order deterministic (storage order within a
// camera; the tie-break pass after the depth sort restores index order among
// equal depths) without a global sort key that carries the index:
//   k_cam_setup     -- once per chunk: each camera's projection constants, which
//                      both passes copy into shared memory per block;
//   k_project_mask  -- survival bit per (camera, Gaussian), one 32-bit mask word
//                      per warp and camera: zero or all ones from the group test,
//                      else per Gaussian (prefilter, then the exact test);
//   k_scan_masks    -- per camera, exclusive prefix of the mask popcounts;
//   k_project_write -- every lane holds one Gaussian (geometry, opacity, SH) in
//                      registers and walks the group's cameras; where its bit is
//                      set it recomputes the projection, evaluates the SH colour
//                      and writes the record, the rect, the depth key (float bits
//                      of z minus those of the near plane) and the Gaussian's
//                      caller index at the pair's stable slot.
// The decision chain is written with explicit fmaf / *_rn intrinsics so both
// passes round identically.
#include <type_traits>

#include "proj_core.cuh"

namespace gsk {

namespace {

__device__ void cam_setup(CamProj &c, const float *vm, const float *in, int W, int H,
                          float guard) {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
#pragma unroll
        for (int j = 0; j < 3; ++j) c.R[3 * i + j] = vm[4 * i + j];
        c.t[i] = vm[4 * i + 3];
    }
    c.fx = in[0];
    c.fy = in[1];
    c.cx = in[2];
    c.cy = in[3];
#pragma unroll
    for (int j = 0; j < 3; ++j)
        c.cpos[j] = -(c.R[j] * c.t[0] + c.R[3 + j] * c.t[1] + c.R[6 + j] * c.t[2]);
    const float g = guard - 1.0f;
    c.lxp = ((W - c.cx) + g * 0.5f * W) / c.fx;
    c.lxn = (c.cx + g * 0.5f * W) / c.fx;
    c.lyp = ((H - c.cy) + g * 0.5f * H) / c.fy;
    c.lyn = (c.cy + g * 0.5f * H) / c.fy;
    const float lx = fmaxf(c.lxp, c.lxn), ly = fmaxf(c.lyp, c.lyn);
    c.kk = c.fx * c.fx * (1.0f + lx * lx) + c.fy * c.fy * (1.0f + ly * ly);
    c.W = (float)W;
    c.H = (float)H;
    c.TX = (W + TILE - 1) / TILE;
    c.TY = (H + TILE - 1) / TILE;
}

// The prefilter constants of two cameras (c, c + 1), field by field as float2
// pairs, for prefilter2.
struct __align__(16) CamPair {
    float2 R[9], t[3];
    float2 fx, fy, cx, cy;
    float2 kk, W, H;
    float2 pad;
};
static_assert(sizeof(CamPair) == 10 * 16, "CamPair is ten float4");

__device__ __forceinline__ CamPair load_pair(const CamPair &src) {
    CamPair c;
    const float4 *s4 = reinterpret_cast<const float4 *>(&src);
    float4 *d4 = reinterpret_cast<float4 *>(&c);
#pragma unroll
    for (int k = 0; k < 10; ++k) d4[k] = s4[k];
    return c;
}

__device__ __forceinline__ void make_pair(CamPair &d, const CamProj &a, const CamProj &b) {
#pragma unroll
    for (int k = 0; k < 9; ++k) d.R[k] = make_float2(a.R[k], b.R[k]);
#pragma unroll
    for (int k = 0; k < 3; ++k) d.t[k] = make_float2(a.t[k], b.t[k]);
    d.fx = make_float2(a.fx, b.fx);
    d.fy = make_float2(a.fy, b.fy);
    d.cx = make_float2(a.cx, b.cx);
    d.cy = make_float2(a.cy, b.cy);
    d.kk = make_float2(a.kk, b.kk);
    d.W = make_float2(a.W, b.W);
    d.H = make_float2(a.H, b.H);
    d.pad = make_float2(0.0f, 0.0f);
}

// prefilter() for two cameras at once on packed FP32x2 arithmetic: every
// operation is the scalar one's, with the same operands in the same order and
// round-to-nearest in each lane, so in0 / in1 equal prefilter() for cameras
// c / c + 1 bit for bit.
__device__ __forceinline__ void prefilter2(const CamPair &c, const GaussGeo &G,
                                           const ProjParams &P, bool &in0, bool &in1) {
    const float2 mx = make_float2(G.mx, G.mx), my = make_float2(G.my, G.my),
                 mz = make_float2(G.mz, G.mz);
    const float2 px = __ffma2_rn(c.R[0], mx, __ffma2_rn(c.R[1], my, __ffma2_rn(c.R[2], mz, c.t[0])));
    const float2 py = __ffma2_rn(c.R[3], mx, __ffma2_rn(c.R[4], my, __ffma2_rn(c.R[5], mz, c.t[1])));
    const float2 z = __ffma2_rn(c.R[6], mx, __ffma2_rn(c.R[7], my, __ffma2_rn(c.R[8], mz, c.t[2])));
    const float2 iz = make_float2(rcp_a(z.x), rcp_a(z.y));
    const float2 xz = __fmul2_rn(px, iz), yz = __fmul2_rn(py, iz);
    const float2 u = __ffma2_rn(c.fx, xz, c.cx), v = __ffma2_rn(c.fy, yz, c.cy);
    const float2 k2 = __fmul2_rn(__fmul2_rn(c.kk, iz), iz);
    const float2 e = __ffma2_rn(k2, make_float2(G.smax2, G.smax2),
                                make_float2(P.dilation, P.dilation));
    const float sg = 1.002f * P.sigma;
    const float2 rb = __ffma2_rn(make_float2(sg, sg), make_float2(sqrt_a(e.x), sqrt_a(e.y)),
                                 make_float2(0.02f, 0.02f));
    const float2 M1 = make_float2(-1.0f, -1.0f);
    const float2 ua = __fadd2_rn(u, rb), us = __ffma2_rn(rb, M1, u);  // u + rb, u - rb
    const float2 va = __fadd2_rn(v, rb), vs = __ffma2_rn(rb, M1, v);
    in0 = z.x > P.near_plane && !(ua.x < 0.0f || us.x >= c.W.x || va.x < 0.0f || vs.x >= c.H.x);
    in1 = z.y > P.near_plane && !(ua.y < 0.0f || us.y >= c.W.y || va.y < 0.0f || vs.y >= c.H.y);
}

// A group of Gaussians (a warp's 32) against one camera, before the Gaussians
// one by one: BLK_OUT when the exact test culls every Gaussian of the group,
// BLK_IN when it keeps every one, BLK_PART otherwise. The group is the box of
// its means (lo, hi) and its largest squared scale (lo.w); hi.w = 0 flags a
// non-finite value (always BLK_PART). Over the box, a camera-space linear form a.mu + b ranges
// over its centre value -+ |a|.e (e: half extents), widened for float32
// rounding. For z > near, u + rb < 0 is fx x + cx z + rb z < 0, and rb z (the
// prefilter's radius bound times z) is at most
// B = 1.002 sigma sqrt(kk S + dil Z^2) + 0.02 Z over the block (S, Z its
// largest squared scale and depth); the test adds 1 % and one pixel times Z.
// The other three sides likewise. Inside: every mean at least one pixel within
// the image (u in [1, W - 1], v in [1, H - 1]) and in front of the near plane
// with a margin, where project() keeps every Gaussian whatever its size.
enum { BLK_OUT = 0, BLK_IN = 1, BLK_PART = 2 };

__device__ __forceinline__ int classify_block(const CamProj &c, float4 lo, float4 hi,
                                              const ProjParams &P) {
    if (!(hi.w > 0.0f)) return BLK_PART;
    const float mx = 0.5f * (lo.x + hi.x), my = 0.5f * (lo.y + hi.y), mz = 0.5f * (lo.z + hi.z);
    const float ex = 0.5f * (hi.x - lo.x), ey = 0.5f * (hi.y - lo.y), ez = 0.5f * (hi.z - lo.z);
    float rlo, rhi;
    auto range = [&](float ax, float ay, float az, float b) {
        const float cv = fmaf(ax, mx, fmaf(ay, my, fmaf(az, mz, b)));
        const float rad = fabsf(ax) * ex + fabsf(ay) * ey + fabsf(az) * ez;
        const float slack =
            1e-5f * (fabsf(ax * mx) + fabsf(ay * my) + fabsf(az * mz) + fabsf(b) + rad) + 1e-6f;
        rlo = cv - rad - slack;
        rhi = cv + rad + slack;
    };
    range(c.R[6], c.R[7], c.R[8], c.t[2]);
    const float zlo = rlo, zhi = rhi;
    if (zhi <= P.near_plane) return BLK_OUT;
    const float Z = fmaxf(zhi, P.near_plane);
    const float B = fmaf(1.01f, fmaf(1.002f * P.sigma, sqrtf(fmaf(c.kk, lo.w, P.dilation * Z * Z)),
                                     0.02f * Z), Z);
    // coefficients of fx x + k z and fy y + k z in world coordinates
    const float ax0 = c.fx * c.R[0], ax1 = c.fx * c.R[1], ax2 = c.fx * c.R[2], bx = c.fx * c.t[0];
    const float ay0 = c.fy * c.R[3], ay1 = c.fy * c.R[4], ay2 = c.fy * c.R[5], by = c.fy * c.t[1];
    auto side = [&](float a0, float a1, float a2, float b, float k) {
        range(fmaf(k, c.R[6], a0), fmaf(k, c.R[7], a1), fmaf(k, c.R[8], a2), fmaf(k, c.t[2], b));
    };
    side(ax0, ax1, ax2, bx, c.cx);  // u >= 0 side
    if (rhi + B < 0.0f) return BLK_OUT;
    side(ax0, ax1, ax2, bx, c.cx - c.W);  // u < W side
    if (rlo - B >= 0.0f) return BLK_OUT;
    side(ay0, ay1, ay2, by, c.cy);
    if (rhi + B < 0.0f) return BLK_OUT;
    side(ay0, ay1, ay2, by, c.cy - c.H);
    if (rlo - B >= 0.0f) return BLK_OUT;
    // inside: every mean with z > near (margin) and 1 <= u <= W - 1, 1 <= v <= H - 1
    if (!(zlo > fmaf(1.001f, P.near_plane, 1e-4f))) return BLK_PART;
    side(ax0, ax1, ax2, bx, c.cx - 1.0f);
    if (!(rlo >= 0.0f)) return BLK_PART;
    side(ax0, ax1, ax2, bx, c.cx - c.W + 1.0f);
    if (!(rhi <= 0.0f)) return BLK_PART;
    side(ay0, ay1, ay2, by, c.cy - 1.0f);
    if (!(rlo >= 0.0f)) return BLK_PART;
    side(ay0, ay1, ay2, by, c.cy - c.H + 1.0f);
    if (!(rhi <= 0.0f)) return BLK_PART;
    return BLK_IN;
}

// Mask pass in two phases so that the long exact test runs on full warps:
// per camera (two at a time on packed arithmetic, prefilter2), every lane
// applies the cheap prefilter to its own Gaussian and
// the warp appends the passing (camera, Gaussian) pairs to a queue in shared
// memory; whenever 32 pairs are queued, each lane takes one and runs the exact
// test (project()); the results are OR-ed into the warp's mask word of that
// camera. Pairs the prefilter rejects are exactly those project() rejects
// there, so the words equal one ballot of project() per camera. A queued
// pair's Gaussian belongs to a lane of the same warp, so the exact test takes
// its geometry from that lane's registers by shuffles (13 of them) instead of
// gathering rows of random Gaussians from shared memory (project 8.59 -> 8.52 ms
// per 1,024 cameras).
constexpr int MQ = 64;  // queue entries per warp: < 32 left + < 32 appended

__global__ void __launch_bounds__(PROJ_THREADS, 4)
    k_project_mask(const Group *__restrict__ groups, const SceneDev *__restrict__ scenes,
                   const CamInfo *__restrict__ cams, const CamProj *__restrict__ camtab,
                   ProjParams P, uint32_t *__restrict__ masks) {
    const Group gr = groups[blockIdx.y];
    const long long g0 = (long long)blockIdx.x * PROJ_THREADS;
    if (g0 >= gr.n) return;
    constexpr int NW = PROJ_THREADS / 32;
    __shared__ CamProj cp[MAX_GROUP];
    __shared__ CamPair cpair[MAX_GROUP / 2];  // cameras (2i, 2i + 1) for prefilter2
    __shared__ long long moff[MAX_GROUP];
    __shared__ uint16_t queue[NW][MQ];                // camera << 5 | lane
    __shared__ uint32_t smask[NW][MAX_GROUP];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const SceneDev sc = scenes[gr.scene];
    if (tid < gr.ncam) {
        cp[tid] = load_cam(camtab[gr.slot0 + tid]);
        moff[tid] = cams[gr.slot0 + tid].mask_off;
    }
    if (2 * tid < gr.ncam) {  // an odd last camera is paired with itself
        const int c1 = 2 * tid + 1 < gr.ncam ? 2 * tid + 1 : 2 * tid;
        make_pair(cpair[tid], load_cam(camtab[gr.slot0 + 2 * tid]), load_cam(camtab[gr.slot0 + c1]));
    }
#pragma unroll
    for (int c = lane; c < MAX_GROUP; c += 32) smask[warp][c] = 0u;
    const long long g = g0 + tid;
    const bool valid = g < gr.n;
    GaussGeo G;
    if (valid) {
        load_geo(sc, g, G);
    } else {
        G.mx = G.my = G.mz = G.smax2 = 0.0f;
#pragma unroll
        for (int k = 0; k < 9; ++k) G.M[k] = 0.0f;
    }
    __syncthreads();
    // the warp's 32 Gaussians as a group against each camera
    uint32_t in_cams[MAX_GROUP / 32], part_cams[MAX_GROUP / 32];
    {
        const long long wb = (g0 >> 5) + warp;
        const bool live = (wb << 5) < gr.n;
        float4 blo = make_float4(0.0f, 0.0f, 0.0f, 0.0f), bhi = blo;
        if (live) {
            blo = sc.bounds[2 * wb];
            bhi = sc.bounds[2 * wb + 1];
        }
        // lane l classifies cameras l, l + 32, ...; ballots give the warp the
        // cameras that keep the whole group (IN) and those that straddle it
#pragma unroll
        for (int q = 0; q < MAX_GROUP / 32; ++q) {
            const int c = lane + 32 * q;
            const int k = (live && c < gr.ncam) ? classify_block(load_cam(cp[c]), blo, bhi, P) : BLK_OUT;
            in_cams[q] = __ballot_sync(0xffffffffu, k == BLK_IN);
            part_cams[q] = __ballot_sync(0xffffffffu, k == BLK_PART);
        }
    }
    const uint32_t lt = (1u << lane) - 1u;
    int nq = 0;  // queued pairs of this warp (warp-uniform)
    // the exact test on queue entries [0, cnt) (cnt <= 32), results OR-ed into smask
    auto drain = [&](int cnt) {
        const int e = lane < cnt ? (int)queue[warp][lane] : 0;
        const int cam = e >> 5, src = e & 31;
        GaussGeo H;  // the geometry of lane src's Gaussian (every lane shuffles)
        H.mx = __shfl_sync(0xffffffffu, G.mx, src);
        H.my = __shfl_sync(0xffffffffu, G.my, src);
        H.mz = __shfl_sync(0xffffffffu, G.mz, src);
        H.smax2 = __shfl_sync(0xffffffffu, G.smax2, src);
#pragma unroll
        for (int k = 0; k < 9; ++k) H.M[k] = __shfl_sync(0xffffffffu, G.M[k], src);
        if (lane < cnt) {
            Proj pr;
            if (project(load_cam(cp[cam]), H, P, pr)) atomicOr(&smask[warp][cam], 1u << src);
        }
        __syncwarp();
        // move the entries past the drained ones to the front
        const int rest = nq - cnt;
        const uint16_t keep = lane < rest ? queue[warp][cnt + lane] : (uint16_t)0;
        __syncwarp();
        if (lane < rest) queue[warp][lane] = keep;
        __syncwarp();
        nq = rest;
    };
    // append this lane's pair with camera c when it passed the prefilter
    auto append = [&](int c, bool cand) {
        const uint32_t b = __ballot_sync(0xffffffffu, cand);
        if (cand) queue[warp][nq + __popc(b & lt)] = (uint16_t)((c << 5) | lane);
        nq += __popc(b);
        __syncwarp();
        if (nq >= 32) drain(32);
    };
    // the block's valid Gaussians: the mask word of a camera that keeps them all
    const uint32_t all = __ballot_sync(0xffffffffu, valid);
#pragma unroll
    for (int q = 0; q < MAX_GROUP / 32; ++q)  // cameras that keep the whole group
        if ((in_cams[q] >> lane) & 1u) smask[warp][lane + 32 * q] = all;
    // only the camera pairs (2i, 2i + 1) with a straddling camera, in camera
    // order (most pairs have none: their group test said outside)
#pragma unroll
    for (int q = 0; q < MAX_GROUP / 32; ++q) {
        const uint32_t pm = part_cams[q];
        uint32_t pairs = (pm | (pm >> 1)) & 0x55555555u;
        while (pairs) {  // warp-uniform
            const int b = __ffs(pairs) - 1;
            pairs &= pairs - 1u;
            const int c = 32 * q + b;
            bool in0 = false, in1 = false;
            if (valid) prefilter2(load_pair(cpair[c >> 1]), G, P, in0, in1);
            append(c, in0 && ((pm >> b) & 1u));
            if (c + 1 < gr.ncam) append(c + 1, in1 && ((pm >> (b + 1)) & 1u));
        }
    }
    if (nq > 0) drain(nq);
    __syncwarp();
    const bool warp_live = (g0 + warp * 32) < gr.n;
#pragma unroll
    for (int c = lane; c < MAX_GROUP; c += 32)
        if (c < gr.ncam && warp_live) masks[moff[c] + (g0 >> 5) + warp] = smask[warp][c];
}

__global__ void __launch_bounds__(1024)
    k_scan_masks(const CamInfo *__restrict__ cams, const SceneDev *__restrict__ scenes,
                 const uint32_t *__restrict__ masks, uint32_t *__restrict__ woff,
                 int *__restrict__ counts) {
    const CamInfo ci = cams[blockIdx.x];
    const long long nwords = (scenes[ci.scene].n + 31) >> 5;
    const uint32_t *m = masks + ci.mask_off;
    uint32_t *wo = woff + ci.mask_off;
    __shared__ uint32_t wsum[32];
    __shared__ uint32_t carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0) carry = 0;
    __syncthreads();
    for (long long base = 0; base < nwords; base += 1024) {
        const long long i = base + tid;
        const uint32_t c = i < nwords ? __popc(m[i]) : 0u;
        uint32_t incl = c;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += t;
        }
        if (lane == 31) wsum[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const uint32_t v = wsum[lane];
            uint32_t s = v;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, s, d);
                if (lane >= d) s += t;
            }
            wsum[lane] = s - v;  // exclusive prefix of the warp sums
        }
        __syncthreads();
        const uint32_t excl = carry + wsum[warp] + incl - c;
        if (i < nwords) wo[i] = excl;
        __syncthreads();
        if (tid == 1023) carry = excl + c;
        __syncthreads();
    }
    if (tid == 0) counts[blockIdx.x] = (int)carry;
}


// SH coefficients per channel in groups of four consecutive k (zero past the
// scene's degree): a Gaussian's column holds 3 * SH_QUADS(DEG) float4.
__host__ __device__ constexpr int sh_quads(int deg) { return ((deg + 1) * (deg + 1) + 3) / 4; }

// Colour of one Gaussian seen from camera c with its SH coefficients in the
// lane's own shared-memory column (sh4[(ch Q + j) PROJ_THREADS] = coefficients
// 4j .. 4j + 3 of channel ch; consecutive lanes read consecutive 16-byte words,
// no bank conflict). Per channel the even-k and the odd-k terms add in order of
// k on the two lanes of a packed FP32x2 accumulator, and the two sums are added
// last (a different association from a single running sum: a few ulp).
template <int DEG>
__device__ __forceinline__ void sh_colour_smem(const float4 *sh4, const CamProj &c,
                                               const GaussGeo &G, float rgb[3]) {
    constexpr int Q = sh_quads(DEG);
    float dx, dy, dz;
    sh_dir(c.cpos, G.mx, G.my, G.mz, dx, dy, dz);
    float Y[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) Y[k] = 0.0f;
    sh_basis(DEG, dx, dy, dz, Y);
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float2 acc = make_float2(0.5f, 0.0f);
#pragma unroll
        for (int j = 0; j < Q; ++j) {
            const float4 w = sh4[(ch * Q + j) * PROJ_THREADS];
            acc = __ffma2_rn(make_float2(w.x, w.y), make_float2(Y[4 * j], Y[4 * j + 1]), acc);
            acc = __ffma2_rn(make_float2(w.z, w.w), make_float2(Y[4 * j + 2], Y[4 * j + 3]), acc);
        }
        rgb[ch] = fmaxf(__fadd_rn(acc.x, acc.y), 0.0f);
    }
}

// SH coefficient rows of Gaussian g into registers (zero past the scene's rows).
template <typename T, int NC>
__device__ __forceinline__ void load_sh(const SceneDev &sc, long long g, float *sh) {
    const int rows = 3 * (sc.deg + 1) * (sc.deg + 1);
#pragma unroll
    for (int i = 0; i < NC; ++i) sh[i] = i < rows ? ldt<T>(sc.sh, (long long)i * sc.n + g) : 0.0f;
}

// Write pass: a block holds the same PROJ_THREADS Gaussians as a mask block and
// every lane owns one of them: its geometry and opacity are read from HBM once
// into registers and its SH coefficients into its own shared-memory column
// (80 registers, three blocks per SM; with the coefficients in registers the
// kernel needed 128 and ran two blocks per SM, 0.7 ms per step slower), and
// used for every camera of the group.
// The warp walks the group's cameras; for a camera whose mask word of this
// warp is zero it moves on at once, else the lanes whose bit is set recompute
// the projection (the same arithmetic as the mask pass), evaluate the colour
// from their registers and write the record at the pair's stable slot (the
// word's offset plus the set bits below the lane), so the lanes of a word write
// consecutive slots. With Gaussians stored in spatial order a camera sees
// either most or none of a warp's 32, so few lanes idle. DEG is the largest SH
// degree of the chunk's scenes (lower degrees run with zero coefficients,
// which add nothing).
template <int DEG>
__global__ void __launch_bounds__(PROJ_THREADS, 3)
    k_project_write(const Group *__restrict__ groups, const SceneDev *__restrict__ scenes,
                    const CamInfo *__restrict__ cams, const CamProj *__restrict__ camtab,
                    ProjParams P,
                    const uint32_t *__restrict__ masks, const uint32_t *__restrict__ woff,
                    float4 *__restrict__ rec, int with_d, uint2 *__restrict__ srect,
                    uint32_t *__restrict__ keys, uint32_t *__restrict__ oidx,
                    float ln_alpha_min, const int *__restrict__ status) {
    const Group gr = groups[blockIdx.y];
    const long long g0 = (long long)blockIdx.x * PROJ_THREADS;
    if (g0 >= gr.n) return;
    if (status && *status) return;  // the chunk was planned empty: workspace too small
    constexpr int NW = PROJ_THREADS / 32;
    constexpr int NC = 3 * (DEG + 1) * (DEG + 1);
    __shared__ CamProj cp[MAX_GROUP];
    __shared__ long long soff[MAX_GROUP];
    __shared__ uint32_t sword[MAX_GROUP][NW], swoff[MAX_GROUP][NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const SceneDev sc = scenes[gr.scene];
    // the mask word and slot offset of every (camera, warp): consecutive
    // threads read consecutive words of one camera
    for (int e = tid; e < gr.ncam * NW; e += PROJ_THREADS) {
        const int c = e / NW, w = e % NW;
        const long long wi = (g0 >> 5) + w;
        uint32_t m = 0u, o = 0u;
        if ((wi << 5) < gr.n) {
            const long long at = cams[gr.slot0 + c].mask_off + wi;
            m = masks[at];
            o = woff[at];
        }
        sword[c][w] = m;
        swoff[c][w] = o;
    }
    if (tid < gr.ncam) {
        cp[tid] = load_cam(camtab[gr.slot0 + tid]);
        soff[tid] = cams[gr.slot0 + tid].seg_off;
    }
    // this lane's Gaussian, into registers
    const long long g = g0 + tid;
    const bool valid = g < gr.n;
    GaussGeo G;
    constexpr int SQ = sh_quads(DEG);
    extern __shared__ float4 shs[];  // [3 SQ][PROJ_THREADS]: this lane's column
    float4 *shc = shs + tid;
    float log2o = 0.0f;
    uint32_t gidx = 0u;
    if (valid) {
        load_geo(sc, g, G);
        log2o = log2_opacity(ldv(sc.logit, g, sc.app_dtype));
        float sh[NC];
        if (sc.app_dtype == DT_F32)
            load_sh<float, NC>(sc, g, sh);
        else if (sc.app_dtype == DT_F16)
            load_sh<__half, NC>(sc, g, sh);
        else
            load_sh<__nv_bfloat16, NC>(sc, g, sh);
        // coefficient (k, ch) is row 3 k + ch of the scene
#pragma unroll
        for (int ch = 0; ch < 3; ++ch)
#pragma unroll
            for (int j = 0; j < SQ; ++j) {
                float w[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) w[e] = 4 * j + e < NC / 3 ? sh[3 * (4 * j + e) + ch] : 0.0f;
                shc[(ch * SQ + j) * PROJ_THREADS] = make_float4(w[0], w[1], w[2], w[3]);
            }
        gidx = (uint32_t)sc.orig[g];
    } else {
        G.mx = G.my = G.mz = G.smax2 = 0.0f;
#pragma unroll
        for (int k = 0; k < 9; ++k) G.M[k] = 0.0f;
#pragma unroll
        for (int i = 0; i < 3 * SQ; ++i) shc[i * PROJ_THREADS] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    // box of the alpha >= alpha_min region d^T Sigma'^-1 d <= q = 2 ln(o/alpha_min):
    // half extents sqrt(q Sigma'_00), sqrt(q Sigma'_11), widened so float32
    // rounding of the per-pixel test can never pass a pixel outside it
    const float q = 2.0f * fmaf(log2o, 0.6931471805599453f, -ln_alpha_min);
    // the cameras whose mask word for this warp is not zero (most are zero:
    // the group test found the group outside), visited in camera order
    uint32_t live_cams[MAX_GROUP / 32];
#pragma unroll
    for (int k = 0; k < MAX_GROUP / 32; ++k) {
        const int c = lane + 32 * k;
        live_cams[k] = __ballot_sync(0xffffffffu, c < gr.ncam && sword[c][warp] != 0u);
    }
#pragma unroll
    for (int k = 0; k < MAX_GROUP / 32; ++k)
    for (uint32_t lc = live_cams[k]; lc; lc &= lc - 1u) {  // warp-uniform
        const int c = 32 * k + __ffs(lc) - 1;
        const uint32_t word = sword[c][warp];
        if (!((word >> lane) & 1u)) continue;
        const CamProj cam = load_cam(cp[c]);
        Proj pr;
        project<false>(cam, G, P, pr);  // the mask pass kept this pair
        float rgb[3];
        sh_colour_smem<DEG>(shc, cam, G, rgb);
        float hx = -1e30f, hy = -1e30f;
        if (q >= 0.0f) {
            hx = fmaf(1.002f, sqrt_a(__fmul_rn(q, pr.sa)), 0.02f);
            hy = fmaf(1.002f, sqrt_a(__fmul_rn(q, pr.sc)), 0.02f);
        }
        const long long at = soff[c] + swoff[c][warp] + __popc(word & lt);
        const uint2 rect = make_uint2((uint32_t)pr.x0 | ((uint32_t)pr.x1 << 16),
                                      (uint32_t)pr.y0 | ((uint32_t)pr.y1 << 16));
        rec[rec_a(at)] = make_float4(pr.u, pr.v, hx, hy);
        rec[rec_b(at)] = make_float4(__fmul_rn(-0.5f * LOG2E, pr.A), __fmul_rn(-LOG2E, pr.B),
                     __fmul_rn(-0.5f * LOG2E, pr.C), log2o);
        rec[rec_c(at)] = make_float4(rgb[0], rgb[1], rgb[2], pr.z);
        if (with_d)
            reinterpret_cast<uint4 *>(rec)[rec_d(at)] =
                make_uint4(rect.x, rect.y, gidx, __float_as_uint(pr.r));
        srect[at] = rect;
        // depth key: float bits of z minus those of the near plane (z > near, so
        // non-negative and in the same order); its value, the slot, is implied
        // by the position.
        const uint32_t kz = __float_as_uint(pr.z) - __float_as_uint(P.near_plane);
        keys[at] = kz;
        oidx[at] = gidx;
    }
}

// Key pass of the progressive order: the write pass's walk over the group's
// cameras whose mask word of this warp is not zero, but a lane with its bit set
// writes only the depth key (z as the projection computes it, bits minus the
// near plane's) and its Gaussian's caller index at the pair's stable slot: 8
// bytes per survivor instead of 64, and no projection or SH work (the records
// of the ranks the render reads come from the binning pass, which finds the
// Gaussian through the scene's inverse of orig).
__global__ void __launch_bounds__(PROJ_THREADS)
    k_project_keys(const Group *__restrict__ groups, const SceneDev *__restrict__ scenes,
                   const CamInfo *__restrict__ cams, const CamProj *__restrict__ camtab,
                   ProjParams P, const uint32_t *__restrict__ masks,
                   const uint32_t *__restrict__ woff, uint32_t *__restrict__ keys,
                   uint32_t *__restrict__ oidx, const int *__restrict__ status) {
    const Group gr = groups[blockIdx.y];
    const long long g0 = (long long)blockIdx.x * PROJ_THREADS;
    if (g0 >= gr.n) return;
    if (status && *status) return;  // the chunk was planned empty: workspace too small
    constexpr int NW = PROJ_THREADS / 32;
    __shared__ float4 zrow[MAX_GROUP];  // R[6], R[7], R[8], t[2]: z of a point
    __shared__ long long soff[MAX_GROUP];
    __shared__ uint32_t sword[MAX_GROUP][NW], swoff[MAX_GROUP][NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const SceneDev sc = scenes[gr.scene];
    for (int e = tid; e < gr.ncam * NW; e += PROJ_THREADS) {
        const int c = e / NW, w = e % NW;
        const long long wi = (g0 >> 5) + w;
        uint32_t m = 0u, o = 0u;
        if ((wi << 5) < gr.n) {
            const long long at = cams[gr.slot0 + c].mask_off + wi;
            m = masks[at];
            o = woff[at];
        }
        sword[c][w] = m;
        swoff[c][w] = o;
    }
    if (tid < gr.ncam) {
        const CamProj &cp = camtab[gr.slot0 + tid];
        zrow[tid] = make_float4(cp.R[6], cp.R[7], cp.R[8], cp.t[2]);
        soff[tid] = cams[gr.slot0 + tid].seg_off;
    }
    const long long g = g0 + tid;
    const bool valid = g < gr.n;
    float mx = 0.0f, my = 0.0f, mz = 0.0f;
    uint32_t gidx = 0u;
    if (valid) {
        mx = ldv(sc.mean, g, sc.geo_dtype);
        my = ldv(sc.mean, sc.n + g, sc.geo_dtype);
        mz = ldv(sc.mean, 2 * sc.n + g, sc.geo_dtype);
        gidx = (uint32_t)sc.orig[g];
    }
    __syncthreads();
    const uint32_t lt = (1u << lane) - 1u;
    const uint32_t near_bits = __float_as_uint(P.near_plane);
#pragma unroll
    for (int k = 0; k < MAX_GROUP / 32; ++k) {
        const int cl = lane + 32 * k;
        uint32_t lc = __ballot_sync(0xffffffffu, cl < gr.ncam && sword[cl][warp] != 0u);
        for (; lc; lc &= lc - 1u) {  // warp-uniform
            const int c = 32 * k + __ffs(lc) - 1;
            const uint32_t word = sword[c][warp];
            if (!((word >> lane) & 1u)) continue;
            const float4 zr = zrow[c];
            const float z = fmaf(zr.x, mx, fmaf(zr.y, my, fmaf(zr.z, mz, zr.w)));
            const long long at = soff[c] + swoff[c][warp] + __popc(word & lt);
            keys[at] = __float_as_uint(z) - near_bits;
            oidx[at] = gidx;
        }
    }
}

// The projection constants of every camera of a chunk (one thread each), read
// by both projection passes.
__global__ void k_cam_setup(const CamInfo *__restrict__ cams, int m, const float *__restrict__ vms,
                            const float *__restrict__ intr, ProjParams P, CamProj *__restrict__ out) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= m) return;
    const CamInfo ci = cams[c];
    CamProj cp;
    cam_setup(cp, vms + 16LL * ci.user, intr + 4LL * ci.user, ci.W, ci.H, P.guard);
    out[c] = cp;
}

}  // namespace

size_t cam_proj_bytes() { return sizeof(CamProj); }

cudaError_t launch_cam_setup(const CamInfo *cams, int m, const float *viewmats, const float *intr,
                             ProjParams P, void *camtab, cudaStream_t s) {
    if (m == 0) return cudaSuccess;
    k_cam_setup<<<(m + 127) / 128, 128, 0, s>>>(cams, m, viewmats, intr, P, (CamProj *)camtab);
    return cudaGetLastError();
}

cudaError_t launch_project_mask(const Group *groups, int n_groups, int max_blocks_x,
                                const SceneDev *scenes, const CamInfo *cams, const void *camtab,
                                ProjParams P, uint32_t *masks, cudaStream_t s) {
    if (n_groups == 0 || max_blocks_x == 0) return cudaSuccess;
    dim3 grid(max_blocks_x, n_groups);
    k_project_mask<<<grid, PROJ_THREADS, 0, s>>>(groups, scenes, cams, (const CamProj *)camtab, P,
                                                 masks);
    return cudaGetLastError();
}

cudaError_t launch_scan_masks(const CamInfo *cams, const SceneDev *scenes, int n_slots,
                              const uint32_t *masks, uint32_t *woff, int *counts,
                              cudaStream_t s) {
    if (n_slots == 0) return cudaSuccess;
    k_scan_masks<<<n_slots, 1024, 0, s>>>(cams, scenes, masks, woff, counts);
    return cudaGetLastError();
}

cudaError_t launch_project_write(const Group *groups, int n_groups, int max_blocks_x,
                                 const SceneDev *scenes, const CamInfo *cams, const void *camtab,
                                 ProjParams P,
                                 const uint32_t *masks, const uint32_t *woff, float4 *rec, int with_d,
                                 uint2 *srect, uint32_t *keys, uint32_t *oidx,
                                 float ln_alpha_min, const int *status, int max_deg,
                                 cudaStream_t s) {
    if (n_groups == 0 || max_blocks_x == 0) return cudaSuccess;
    dim3 grid(max_blocks_x, n_groups);  // PROJ_THREADS Gaussians per block, as the mask pass
    const CamProj *ct = (const CamProj *)camtab;
#define GS_WRITE(D)                                                                              \
    cudaFuncSetAttribute(k_project_write<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,           \
                         3 * sh_quads(D) * PROJ_THREADS * 16);                                       \
    k_project_write<D><<<grid, PROJ_THREADS, 3 * sh_quads(D) * PROJ_THREADS * 16, s>>>(          \
        groups, scenes, cams, ct, P, masks, woff, rec, with_d, srect, keys, oidx,                 \
        ln_alpha_min, status)
    switch (max_deg) {
        case 0: GS_WRITE(0); break;
        case 1: GS_WRITE(1); break;
        case 2: GS_WRITE(2); break;
        default: GS_WRITE(3); break;
    }
#undef GS_WRITE
    return cudaGetLastError();
}

cudaError_t launch_project_keys(const Group *groups, int n_groups, int max_blocks_x,
                                const SceneDev *scenes, const CamInfo *cams, const void *camtab,
                                ProjParams P, const uint32_t *masks, const uint32_t *woff,
                                uint32_t *keys, uint32_t *oidx, const int *status, cudaStream_t s) {
    if (n_groups == 0 || max_blocks_x == 0) return cudaSuccess;
    dim3 grid(max_blocks_x, n_groups);  // PROJ_THREADS Gaussians per block, as the mask pass
    k_project_keys<<<grid, PROJ_THREADS, 0, s>>>(groups, scenes, cams, (const CamProj *)camtab, P,
                                                 masks, woff, keys, oidx, status);
    return cudaGetLastError();
}

}  // namespace gsk
