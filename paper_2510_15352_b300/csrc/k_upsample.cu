// k_upsample.cu -- the learned 4x upsampler's kernels on the BF16 tensor cores
// (warp-level mma.sync m16n8k16, FP32 accumulation).
//
// Network (a residual CNN on the 160x120 render of a camera): the input is
// x0 = [rgb - 1/2, S (rgb - box3(rgb))] (box3: 3x3 mean, edge clamp; S = 32),
// then five 3x3 convolutions of 32 channels with ReLU, a 3x3 convolution to
// 48 channels, pixel shuffle x4 (channel 16 c + 4 dy + dx -> colour c at
// offset (dy, dx)) scaled by 1/S and added to the bilinear x4 upsampling of
// rgb (half-pixel centres, edge clamp). The detail channels and the 1/S scale
// keep the ~1e-3 differences between a render and its bilinear upsampling far
// above BF16's relative precision. Activations are NHWC BF16; weights are BF16
// copies of FP32 master weights.
//
// A convolution is an implicit GEMM over a tile of 8 x 16 output pixels: the
// input tile with its one-pixel halo and all nine taps of the weights sit in
// shared memory, and for tap (u, v) the A operand of output row r is input row
// r + u shifted by v -- a pointer offset, no im2col buffer. Warp w owns output
// rows 2w and 2w + 1 (two m16 tiles) and all output channels (n8 tiles).
// Shared-memory rows are padded by 16 bytes so that the fragment loads of the
// eight row groups of a warp fall in distinct banks.
//
// The same kernel runs the backward data pass (the gradient with respect to a
// layer's input is the convolution of the output gradient with the flipped,
// transposed weights), gated by the ReLU derivative of the layer below. The
// weight gradient is a reduction over pixels: one warp per tap, ldmatrix.trans
// fragments straight from the NHWC tiles, FP32 partial sums per block, one
// atomic add per weight per block at the end.
#include <algorithm>

#include "gs_internal.cuh"

namespace gsk {

namespace {

constexpr int UT_W = 16, UT_H = 8;            // output tile of a convolution block
constexpr int UH_W = UT_W + 2, UH_H = UT_H + 2;  // input tile with halo
constexpr int CONV_THREADS = 128;             // 4 warps x 2 tile rows
constexpr int WGRAD_THREADS = 288;            // one warp per tap
constexpr float DETAIL_S = 32.0f;             // scale of the detail channels and 1/S of the output

typedef __nv_bfloat16 bf16;

__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void ldsm_x4_trans(uint32_t (&r)[4], const void *p) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(a));
}

__device__ __forceinline__ uint32_t lds32(const bf16 *p) { return *(const uint32_t *)p; }

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *(uint32_t *)&v;
}

// Bilinear x4 source of an output coordinate (half-pixel centres, clamped).
__device__ __forceinline__ void bl_src(int o, int n, int &i0, int &i1, float &f) {
    float s = (o + 0.5f) * 0.25f - 0.5f;
    s = fminf(fmaxf(s, 0.0f), (float)(n - 1));
    i0 = (int)s;
    i1 = min(i0 + 1, n - 1);
    f = s - (float)i0;
}

// Loads the input tile (with halo, zero outside the image) and the weights.
template <int CIN, int COUT>
__device__ __forceinline__ void load_conv_tiles(const bf16 *__restrict__ x, int h, int w,
                                                const bf16 *__restrict__ wt, bf16 *xs, bf16 *ws,
                                                int img, int by, int bx) {
    constexpr int SX = CIN + 8, C8 = CIN / 8;
    for (int i = threadIdx.x; i < 9 * COUT * C8; i += blockDim.x) {
        const int row = i / C8, c8 = i - row * C8;
        *(uint4 *)(ws + row * SX + c8 * 8) = *(const uint4 *)(wt + (long long)row * CIN + c8 * 8);
    }
    for (int i = threadIdx.x; i < UH_H * UH_W * C8; i += blockDim.x) {
        const int p = i / C8, c8 = i - p * C8;
        const int yy = by - 1 + p / UH_W, xx = bx - 1 + p % UH_W;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (yy >= 0 && yy < h && xx >= 0 && xx < w)
            v = *(const uint4 *)(x + (((long long)img * h + yy) * w + xx) * CIN + c8 * 8);
        *(uint4 *)(xs + p * SX + c8 * 8) = v;
    }
}

// acc[mi][j] += sum over taps and input channels for output rows 2 warp + mi.
template <int CIN, int COUT>
__device__ __forceinline__ void conv_mma(const bf16 *xs, const bf16 *ws,
                                         float (&acc)[2][COUT / 8][4]) {
    constexpr int SX = CIN + 8, NT = COUT / 8;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
        const int u = tap / 3, v = tap - 3 * (tap / 3);
#pragma unroll
        for (int ks = 0; ks < CIN / 16; ++ks) {
            uint32_t b[NT][2];
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const bf16 *wp = ws + (tap * COUT + 8 * j + g) * SX + 16 * ks + 2 * t;
                b[j][0] = lds32(wp);
                b[j][1] = lds32(wp + 8);
            }
#pragma unroll
            for (int mi = 0; mi < 2; ++mi) {
                const int r = 2 * warp + mi;
                const bf16 *ap = xs + ((r + u) * UH_W + v + g) * SX + 16 * ks + 2 * t;
                uint32_t a[4];
                a[0] = lds32(ap);
                a[1] = lds32(ap + 8 * SX);
                a[2] = lds32(ap + 8);
                a[3] = lds32(ap + 8 * SX + 8);
#pragma unroll
                for (int j = 0; j < NT; ++j) mma16816(acc[mi][j], a, b[j][0], b[j][1]);
            }
        }
    }
}

// Epilogues of the convolution kernel.
enum : int {
    EPI_RELU = 0,    // out bf16 = relu(acc + bias)
    EPI_LINEAR = 1,  // out f32 = acc + bias (last layer, kept for the loss)
    EPI_GATE = 2,    // out bf16 = acc * (gate > 0)   (backward data pass)
};

template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(CONV_THREADS)
    k_conv(const bf16 *__restrict__ x, int h, int w, const bf16 *__restrict__ wt,
           const float *__restrict__ bias, const bf16 *__restrict__ gate, void *__restrict__ out) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int SX = CIN + 8, NT = COUT / 8;
    bf16 *xs = (bf16 *)smem;
    bf16 *ws = xs + UH_H * UH_W * SX;
    const int img = blockIdx.z, by = blockIdx.y * UT_H, bx = blockIdx.x * UT_W;
    load_conv_tiles<CIN, COUT>(x, h, w, wt, xs, ws, img, by, bx);
    __syncthreads();
    float acc[2][NT][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[mi][j][q] = 0.0f;
    conv_mma<CIN, COUT>(xs, ws, acc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi) {
        const int yy = by + 2 * warp + mi;
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int xx = bx + g + 8 * half;
            if (yy >= h || xx >= w) continue;
            const long long pix = ((long long)img * h + yy) * w + xx;
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const int co = 8 * j + 2 * t;
                float v0 = acc[mi][j][2 * half], v1 = acc[mi][j][2 * half + 1];
                if (EPI == EPI_RELU) {
                    v0 = fmaxf(v0 + bias[co], 0.0f);
                    v1 = fmaxf(v1 + bias[co + 1], 0.0f);
                    *(uint32_t *)((bf16 *)out + pix * COUT + co) = pack_bf16(v0, v1);
                } else if (EPI == EPI_LINEAR) {
                    *(float2 *)((float *)out + pix * COUT + co) =
                        make_float2(v0 + bias[co], v1 + bias[co + 1]);
                } else {
                    const __nv_bfloat162 gv = *(const __nv_bfloat162 *)(gate + pix * COUT + co);
                    v0 = __bfloat162float(gv.x) > 0.0f ? v0 : 0.0f;
                    v1 = __bfloat162float(gv.y) > 0.0f ? v1 : 0.0f;
                    *(uint32_t *)((bf16 *)out + pix * COUT + co) = pack_bf16(v0, v1);
                }
            }
        }
    }
}

// Last layer for inference: z = conv(h5) + bias (48 channels), then
// out[4y + dy][4x + dx][c] = bilinear(rgb)[..][c] + z[16 c + 4 dy + dx] / S, written
// as whole HR rows of the tile (coalesced).
template <int CIN>
__global__ void __launch_bounds__(CONV_THREADS)
    k_conv_upsample(const bf16 *__restrict__ x, int h, int w, const bf16 *__restrict__ wt,
                    const float *__restrict__ bias, const float *__restrict__ rgb,
                    float *__restrict__ out) {
    constexpr int COUT = 48, SX = CIN + 8, NT = COUT / 8, ZS = COUT + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    bf16 *xs = (bf16 *)smem;
    bf16 *ws = xs + UH_H * UH_W * SX;
    float *zs = (float *)smem;  // reuses xs / ws after the MMAs
    float *ls = (float *)(smem + (size_t)(UH_H * UH_W + 9 * COUT) * SX * sizeof(bf16));
    const int img = blockIdx.z, by = blockIdx.y * UT_H, bx = blockIdx.x * UT_W;
    load_conv_tiles<CIN, COUT>(x, h, w, wt, xs, ws, img, by, bx);
    // the LR colours of the tile and its halo, edge-clamped
    for (int i = threadIdx.x; i < UH_H * UH_W; i += blockDim.x) {
        const int yy = min(max(by - 1 + i / UH_W, 0), h - 1);
        const int xx = min(max(bx - 1 + i % UH_W, 0), w - 1);
        const float *src = rgb + (((long long)img * h + yy) * w + xx) * 3;
        ls[3 * i + 0] = src[0];
        ls[3 * i + 1] = src[1];
        ls[3 * i + 2] = src[2];
    }
    __syncthreads();
    float acc[2][NT][4];
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[mi][j][q] = 0.0f;
    conv_mma<CIN, COUT>(xs, ws, acc);
    __syncthreads();  // xs / ws are dead: zs overlays them
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int p = (2 * warp + mi) * UT_W + g + 8 * half;
#pragma unroll
            for (int j = 0; j < NT; ++j) {
                const int co = 8 * j + 2 * t;
                zs[p * ZS + co] = acc[mi][j][2 * half] + bias[co];
                zs[p * ZS + co + 1] = acc[mi][j][2 * half + 1] + bias[co + 1];
            }
        }
    __syncthreads();
    const int H4 = 4 * h, W4 = 4 * w;
    constexpr int ROWF = 4 * UT_W * 3;  // floats per HR row of the tile
    for (int i = threadIdx.x; i < 4 * UT_H * ROWF; i += blockDim.x) {
        const int row = i / ROWF, e = i - row * ROWF;
        const int X = e / 3, c = e - 3 * X;
        const int HY = 4 * by + row, HX = 4 * bx + X;
        if (HY >= H4 || HX >= W4) continue;
        int y0, y1, x0, x1;
        float fy, fx;
        bl_src(HY, h, y0, y1, fy);
        bl_src(HX, w, x0, x1, fx);
        y0 -= by - 1; y1 -= by - 1; x0 -= bx - 1; x1 -= bx - 1;
        const float top = fmaf(fx, ls[3 * (y0 * UH_W + x1) + c] - ls[3 * (y0 * UH_W + x0) + c],
                               ls[3 * (y0 * UH_W + x0) + c]);
        const float bot = fmaf(fx, ls[3 * (y1 * UH_W + x1) + c] - ls[3 * (y1 * UH_W + x0) + c],
                               ls[3 * (y1 * UH_W + x0) + c]);
        const float bl = fmaf(fy, bot - top, top);
        const int p = (row >> 2) * UT_W + (X >> 2);
        const float z = zs[p * ZS + 16 * c + 4 * (row & 3) + (X & 3)];
        out[(((long long)img * H4 + HY) * W4 + HX) * 3 + c] = fmaf(z, 1.0f / DETAIL_S, bl);
    }
}

// Weight and bias gradients of one convolution: gW[co][ci][tap] += sum_p dz[p][co]
// x[p + off(tap)][ci], gb[co] += sum_p dz[p][co]. Warp w handles tap w over
// the block's pixel tiles; the K dimension of a step is one tile row (16 pixels).
template <int CIN, int COUT>
__global__ void __launch_bounds__(WGRAD_THREADS)
    k_wgrad(const bf16 *__restrict__ x, const bf16 *__restrict__ dz, int n, int h, int w,
            float *__restrict__ gW, float *__restrict__ gb, int cin_real) {
    constexpr int SX = CIN + 8, SD = COUT + 8, MT = COUT / 16, NT = CIN / 8;
    extern __shared__ __align__(16) unsigned char smem[];
    bf16 *xs = (bf16 *)smem;
    bf16 *ds = xs + UH_H * UH_W * SX;
    const int tid = threadIdx.x, lane = tid & 31, tap = tid >> 5;
    const int u = tap / 3, v = tap - 3 * (tap / 3);
    const int tx = (w + UT_W - 1) / UT_W, ty = (h + UT_H - 1) / UT_H;
    const long long n_tiles = (long long)tx * ty * n;
    float acc[MT][NT][4];
#pragma unroll
    for (int mi = 0; mi < MT; ++mi)
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[mi][j][q] = 0.0f;
    float bacc = 0.0f;
    // ldmatrix row addresses (per lane): A = dz^T (rows = pixels k, 8-channel
    // column blocks m), B = x (rows = pixels k, 8-channel column blocks n)
    const int a_k = (lane & 7) + ((lane >> 4) << 3), a_m = ((lane >> 3) & 1) * 8;
    const int b_k = (lane & 7) + (((lane >> 3) & 1) << 3), b_n = (lane >> 4) * 8;
    for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int img = (int)(tile / ((long long)tx * ty));
        const int rem = (int)(tile - (long long)img * tx * ty);
        const int by = (rem / tx) * UT_H, bx = (rem % tx) * UT_W;
        constexpr int C8 = CIN / 8, D8 = COUT / 8;
        for (int i = tid; i < UH_H * UH_W * C8; i += blockDim.x) {
            const int p = i / C8, c8 = i - p * C8;
            const int yy = by - 1 + p / UH_W, xx = bx - 1 + p % UH_W;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (yy >= 0 && yy < h && xx >= 0 && xx < w)
                val = *(const uint4 *)(x + (((long long)img * h + yy) * w + xx) * CIN + c8 * 8);
            *(uint4 *)(xs + p * SX + c8 * 8) = val;
        }
        for (int i = tid; i < UT_H * UT_W * D8; i += blockDim.x) {
            const int p = i / D8, c8 = i - p * D8;
            const int yy = by + p / UT_W, xx = bx + p % UT_W;
            uint4 val = make_uint4(0u, 0u, 0u, 0u);
            if (yy < h && xx < w)
                val = *(const uint4 *)(dz + (((long long)img * h + yy) * w + xx) * COUT + c8 * 8);
            *(uint4 *)(ds + p * SD + c8 * 8) = val;
        }
        __syncthreads();
        if (tid < COUT)
            for (int p = 0; p < UT_H * UT_W; ++p) bacc += __bfloat162float(ds[p * SD + tid]);
#pragma unroll 2
        for (int r = 0; r < UT_H; ++r) {
            uint32_t af[MT][4];
#pragma unroll
            for (int mi = 0; mi < MT; ++mi)
                ldsm_x4_trans(af[mi], ds + (r * UT_W + a_k) * SD + 16 * mi + a_m);
#pragma unroll
            for (int jj = 0; jj < NT / 2; ++jj) {
                uint32_t bf[4];
                ldsm_x4_trans(bf, xs + ((r + u) * UH_W + b_k + v) * SX + 16 * jj + b_n);
#pragma unroll
                for (int mi = 0; mi < MT; ++mi) {
                    mma16816(acc[mi][2 * jj], af[mi], bf[0], bf[1]);
                    mma16816(acc[mi][2 * jj + 1], af[mi], bf[2], bf[3]);
                }
            }
        }
        __syncthreads();
    }
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int mi = 0; mi < MT; ++mi)
#pragma unroll
        for (int j = 0; j < NT; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int co = 16 * mi + g + 8 * (q >> 1), ci = 8 * j + 2 * t + (q & 1);
                if (ci < cin_real) atomicAdd(&gW[((long long)co * cin_real + ci) * 9 + tap], acc[mi][j][q]);
            }
    if (tid < COUT) atomicAdd(&gb[tid], bacc);
}

// x0 = [rgb - 1/2, S (rgb - box3(rgb))] in BF16, channels 6..15 zero. One
// block row per image row (blockIdx.x = img * h + y).
__global__ void k_prep_input(const float *__restrict__ rgb, int h, int w, bf16 *__restrict__ x0) {
    const int y = blockIdx.x % h;
    const long long rowp = (long long)blockIdx.x * w;  // first pixel of this row
    const float *row_img = rgb + (rowp - (long long)y * w) * 3;  // first pixel of the image
    for (int x = threadIdx.x; x < w; x += blockDim.x) {
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
#pragma unroll
        for (int du = -1; du <= 1; ++du) {
            const int yy = min(max(y + du, 0), h - 1);
#pragma unroll
            for (int dv = -1; dv <= 1; ++dv) {
                const int xx = min(max(x + dv, 0), w - 1);
                const float *q = row_img + ((long long)yy * w + xx) * 3;
                s0 += q[0];
                s1 += q[1];
                s2 += q[2];
            }
        }
        const long long p = rowp + x;
        const float r = rgb[3 * p], g = rgb[3 * p + 1], b = rgb[3 * p + 2];
        uint4 lo, hi = make_uint4(0u, 0u, 0u, 0u);
        lo.x = pack_bf16(r - 0.5f, g - 0.5f);
        lo.y = pack_bf16(b - 0.5f, DETAIL_S * (r - s0 / 9.0f));
        lo.z = pack_bf16(DETAIL_S * (g - s1 / 9.0f), DETAIL_S * (b - s2 / 9.0f));
        lo.w = 0u;
        *(uint4 *)(x0 + 16 * p) = lo;
        *(uint4 *)(x0 + 16 * p + 8) = hi;
    }
}

// The same input for the tensor-core inference path, as one plane of the 8
// stored channels ([n][h][w][8]; channels 8-15 of the padded input are zero
// and are not stored: that kernel keeps them zero in shared memory).
__global__ void k_prep_input_plane(const float *__restrict__ rgb, int h, int w, bf16 *__restrict__ x0) {
    const int y = blockIdx.x % h;
    const long long rowp = (long long)blockIdx.x * w;
    const float *row_img = rgb + (rowp - (long long)y * w) * 3;
    for (int x = threadIdx.x; x < w; x += blockDim.x) {
        float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
#pragma unroll
        for (int du = -1; du <= 1; ++du) {
            const int yy = min(max(y + du, 0), h - 1);
#pragma unroll
            for (int dv = -1; dv <= 1; ++dv) {
                const int xx = min(max(x + dv, 0), w - 1);
                const float *q = row_img + ((long long)yy * w + xx) * 3;
                s0 += q[0];
                s1 += q[1];
                s2 += q[2];
            }
        }
        const long long p = rowp + x;
        const float r = rgb[3 * p], g = rgb[3 * p + 1], b = rgb[3 * p + 2];
        uint4 lo;
        lo.x = pack_bf16(r - 0.5f, g - 0.5f);
        lo.y = pack_bf16(b - 0.5f, DETAIL_S * (r - s0 / 9.0f));
        lo.z = pack_bf16(DETAIL_S * (g - s1 / 9.0f), DETAIL_S * (b - s2 / 9.0f));
        lo.w = 0u;
        *(uint4 *)(x0 + 8 * p) = lo;
    }
}

// Loss of the training pass: out = bilinear(rgb) + shuffle(z) / S; per LR pixel
// and channel, dz = 2 (out - target) / (count S) (BF16) and sum (out - target)^2 / count.
__global__ void __launch_bounds__(256)
    k_upsample_loss(const float *__restrict__ z, const float *__restrict__ rgb,
                    const float *__restrict__ target, int n, int h, int w,
                    bf16 *__restrict__ dz, float *__restrict__ loss) {
    const long long total = (long long)n * h * w * 48;
    const int H4 = 4 * h, W4 = 4 * w;
    const float inv = 1.0f / (float)((double)n * H4 * W4 * 3);
    float part = 0.0f;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long p = i / 48;
        const int ch = (int)(i - p * 48);
        const int img = (int)(p / ((long long)h * w));
        const int rem = (int)(p - (long long)img * h * w);
        const int y = rem / w, xx = rem - y * w;
        const int c = ch >> 4, dy = (ch >> 2) & 3, dx = ch & 3;
        const int HY = 4 * y + dy, HX = 4 * xx + dx;
        int y0, y1, x0, x1;
        float fy, fx;
        bl_src(HY, h, y0, y1, fy);
        bl_src(HX, w, x0, x1, fx);
        const float *base = rgb + (long long)img * h * w * 3;
        const float a00 = base[(y0 * w + x0) * 3 + c], a01 = base[(y0 * w + x1) * 3 + c];
        const float a10 = base[(y1 * w + x0) * 3 + c], a11 = base[(y1 * w + x1) * 3 + c];
        const float top = fmaf(fx, a01 - a00, a00), bot = fmaf(fx, a11 - a10, a10);
        const float o = fmaf(z[i], 1.0f / DETAIL_S, fmaf(fy, bot - top, top));
        const float d = o - target[(((long long)img * H4 + HY) * W4 + HX) * 3 + c];
        dz[i] = __float2bfloat16_rn(2.0f * d * inv * (1.0f / DETAIL_S));
        part = fmaf(d * d, inv, part);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) part += __shfl_down_sync(0xffffffffu, part, o);
    if ((threadIdx.x & 31) == 0) atomicAdd(loss, part);
}

// Bilinear x4 of a single-channel image (the depth of the upsampled path).
// One block per HR row (blockIdx.x = img * 4h + HY).
__global__ void k_bilinear1(const float *__restrict__ src, int h, int w, float *__restrict__ dst) {
    const int H4 = 4 * h, W4 = 4 * w;
    const int img = blockIdx.x / H4, HY = blockIdx.x - img * H4;
    int y0, y1;
    float fy;
    bl_src(HY, h, y0, y1, fy);
    const float *b = src + (long long)img * h * w;
    float *o = dst + (long long)blockIdx.x * W4;
    for (int HX = threadIdx.x; HX < W4; HX += blockDim.x) {
        int x0, x1;
        float fx;
        bl_src(HX, w, x0, x1, fx);
        const float top = fmaf(fx, b[y0 * w + x1] - b[y0 * w + x0], b[y0 * w + x0]);
        const float bot = fmaf(fx, b[y1 * w + x1] - b[y1 * w + x0], b[y1 * w + x0]);
        o[HX] = fmaf(fy, bot - top, top);
    }
}

// Writes one weight, as BF16, into the four layouts the kernels read:
// wf[tap][co][cin_pad] (warp-level MMA, forward), wd[8 - tap][ci][co] (warp-level
// MMA, backward data pass), wt[tap][cin_pad / 8][co][8] (tcgen05 K-major B
// operand, forward) and wdt[8 - tap][co / 8][ci][8] (tcgen05, backward data).
__device__ __forceinline__ void store_weight(float val, int i, int co, int ci, int cin_pad,
                                             bf16 *wf, bf16 *wd, bf16 *wt, bf16 *wdt) {
    const int o = i / (ci * 9), rem = i - o * ci * 9, c = rem / 9, tap = rem - 9 * c;
    const bf16 b = __float2bfloat16_rn(val);
    wf[((long long)tap * co + o) * cin_pad + c] = b;
    if (wd) wd[((long long)(8 - tap) * ci + c) * co + o] = b;
    if (wt) wt[(((long long)tap * (cin_pad / 8) + c / 8) * co + o) * 8 + (c & 7)] = b;
    if (wdt) wdt[(((long long)(8 - tap) * (co / 8) + o / 8) * ci + c) * 8 + (o & 7)] = b;
}

// Adam on one layer's FP32 master weights [co][ci][3][3] and biases [co]
// (flat: weights then biases), refreshing the BF16 copies.
__global__ void k_adam(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, int co, int ci, int cin_pad, float lr,
                       float b1, float b2, float eps, float c1, float c2, bf16 *__restrict__ wf,
                       bf16 *__restrict__ wd, bf16 *__restrict__ wt, bf16 *__restrict__ wdt) {
    const int nW = co * ci * 9, total = nW + co;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = fmaf(b1, m[i], (1.0f - b1) * gi);
        const float vi = fmaf(b2, v[i], (1.0f - b2) * gi * gi);
        m[i] = mi;
        v[i] = vi;
        const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
        p[i] = pi;
        if (i < nW) store_weight(pi, i, co, ci, cin_pad, wf, wd, wt, wdt);
    }
}

// BF16 copies of one layer's weights without an update (after a parameter upload).
__global__ void k_weights_bf16(const float *__restrict__ p, int co, int ci, int cin_pad,
                               bf16 *__restrict__ wf, bf16 *__restrict__ wd,
                               bf16 *__restrict__ wt, bf16 *__restrict__ wdt) {
    const int nW = co * ci * 9;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nW; i += gridDim.x * blockDim.x)
        store_weight(p[i], i, co, ci, cin_pad, wf, wd, wt, wdt);
}

template <int CIN, int COUT>
constexpr size_t conv_smem() {
    return (size_t)(UH_H * UH_W + 9 * COUT) * (CIN + 8) * sizeof(bf16);
}

template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int CIN, int COUT, int EPI>
cudaError_t run_conv(const bf16 *x, int n, int h, int w, const bf16 *wt, const float *bias,
                     const bf16 *gate, void *out, cudaStream_t s) {
    constexpr size_t smem = conv_smem<CIN, COUT>();
    cudaError_t e = allow_smem(k_conv<CIN, COUT, EPI>, smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((w + UT_W - 1) / UT_W, (h + UT_H - 1) / UT_H, n);
    k_conv<CIN, COUT, EPI><<<grid, CONV_THREADS, smem, s>>>(x, h, w, wt, bias, gate, out);
    return cudaGetLastError();
}

template <int CIN, int COUT>
cudaError_t run_wgrad(const bf16 *x, const bf16 *dz, int n, int h, int w, float *gW, float *gb,
                      int cin_real, int n_sm, cudaStream_t s) {
    constexpr size_t smem = (size_t)(UH_H * UH_W * (CIN + 8) + UT_H * UT_W * (COUT + 8)) * 2;
    cudaError_t e = allow_smem(k_wgrad<CIN, COUT>, smem);
    if (e != cudaSuccess) return e;
    const long long tiles =
        (long long)((w + UT_W - 1) / UT_W) * ((h + UT_H - 1) / UT_H) * n;
    const int grid = (int)std::min<long long>(tiles, 2LL * n_sm);
    k_wgrad<CIN, COUT><<<grid, WGRAD_THREADS, smem, s>>>(x, dz, n, h, w, gW, gb, cin_real);
    return cudaGetLastError();
}

}  // namespace

// ---- launchers ----

cudaError_t up_prep_input(const float *rgb, int n, int h, int w, __nv_bfloat16 *x0,
                          cudaStream_t s) {
    if ((long long)n * h == 0) return cudaSuccess;
    k_prep_input<<<n * h, std::min(256, (w + 31) / 32 * 32), 0, s>>>(rgb, h, w, x0);
    return cudaGetLastError();
}

cudaError_t up_prep_input_plane(const float *rgb, int n, int h, int w, __nv_bfloat16 *x0,
                                cudaStream_t s) {
    if ((long long)n * h == 0) return cudaSuccess;
    k_prep_input_plane<<<n * h, std::min(256, (w + 31) / 32 * 32), 0, s>>>(rgb, h, w, x0);
    return cudaGetLastError();
}

cudaError_t up_conv_forward(int layer, const __nv_bfloat16 *x, int n, int h, int w,
                            const __nv_bfloat16 *wt, const float *bias, void *out,
                            cudaStream_t s) {
    if (layer == 0) return run_conv<16, 32, EPI_RELU>(x, n, h, w, wt, bias, nullptr, out, s);
    if (layer < 5) return run_conv<32, 32, EPI_RELU>(x, n, h, w, wt, bias, nullptr, out, s);
    return run_conv<32, 48, EPI_LINEAR>(x, n, h, w, wt, bias, nullptr, out, s);
}

cudaError_t up_conv_upsample(const __nv_bfloat16 *x, int n, int h, int w,
                             const __nv_bfloat16 *wt, const float *bias, const float *rgb,
                             float *out, cudaStream_t s) {
    constexpr size_t smem = conv_smem<32, 48>() + UH_H * UH_W * 3 * sizeof(float);
    static_assert((size_t)UT_H * UT_W * 49 * sizeof(float) <= conv_smem<32, 48>(),
                  "the z tile must fit over the input and weight tiles");
    cudaError_t e = allow_smem(k_conv_upsample<32>, smem);
    if (e != cudaSuccess) return e;
    const dim3 grid((w + UT_W - 1) / UT_W, (h + UT_H - 1) / UT_H, n);
    k_conv_upsample<32><<<grid, CONV_THREADS, smem, s>>>(x, h, w, wt, bias, rgb, out);
    return cudaGetLastError();
}

// Gradient with respect to the input of layer `layer` (1..5), gated by relu' of
// that input: dx = conv(dz, wd) * (act > 0).
cudaError_t up_conv_dgrad(int layer, const __nv_bfloat16 *dz, int n, int h, int w,
                          const __nv_bfloat16 *wd, const __nv_bfloat16 *act,
                          __nv_bfloat16 *dx, cudaStream_t s) {
    if (layer == 5) return run_conv<48, 32, EPI_GATE>(dz, n, h, w, wd, nullptr, act, dx, s);
    return run_conv<32, 32, EPI_GATE>(dz, n, h, w, wd, nullptr, act, dx, s);
}

cudaError_t up_wgrad(int layer, const __nv_bfloat16 *x, const __nv_bfloat16 *dz, int n, int h,
                     int w, float *gW, float *gb, int n_sm, cudaStream_t s) {
    if (layer == 0) return run_wgrad<16, 32>(x, dz, n, h, w, gW, gb, 6, n_sm, s);
    if (layer < 5) return run_wgrad<32, 32>(x, dz, n, h, w, gW, gb, 32, n_sm, s);
    return run_wgrad<32, 48>(x, dz, n, h, w, gW, gb, 32, n_sm, s);
}

cudaError_t up_loss(const float *z, const float *rgb, const float *target, int n, int h, int w,
                    __nv_bfloat16 *dz, float *loss, cudaStream_t s) {
    const long long total = (long long)n * h * w * 48;
    if (total == 0) return cudaSuccess;
    const int grid = (int)std::min<long long>((total + 255) / 256, 148LL * 16);
    k_upsample_loss<<<grid, 256, 0, s>>>(z, rgb, target, n, h, w, dz, loss);
    return cudaGetLastError();
}

cudaError_t up_bilinear1(const float *src, int n, int h, int w, float *dst, cudaStream_t s) {
    if ((long long)n * h == 0) return cudaSuccess;
    k_bilinear1<<<n * 4 * h, std::min(256, (4 * w + 31) / 32 * 32), 0, s>>>(src, h, w, dst);
    return cudaGetLastError();
}

cudaError_t up_adam(float *p, float *m, float *v, const float *g, int co, int ci, int cin_pad,
                    float lr, float b1, float b2, float eps, float c1, float c2,
                    __nv_bfloat16 *wf, __nv_bfloat16 *wd, __nv_bfloat16 *wt, __nv_bfloat16 *wdt,
                    cudaStream_t s) {
    const int total = co * ci * 9 + co;
    k_adam<<<(total + 255) / 256, 256, 0, s>>>(p, m, v, g, co, ci, cin_pad, lr, b1, b2, eps, c1,
                                                c2, wf, wd, wt, wdt);
    return cudaGetLastError();
}

cudaError_t up_weights_bf16(const float *p, int co, int ci, int cin_pad, __nv_bfloat16 *wf,
                            __nv_bfloat16 *wd, __nv_bfloat16 *wt, __nv_bfloat16 *wdt,
                            cudaStream_t s) {
    const int nW = co * ci * 9;
    k_weights_bf16<<<(nW + 255) / 256, 256, 0, s>>>(p, co, ci, cin_pad, wf, wd, wt, wdt);
    return cudaGetLastError();
}

}  // namespace gsk
