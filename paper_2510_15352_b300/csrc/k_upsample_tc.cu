// k_upsample_tc.cu -- the upsampler's inference convolutions on the 5th-generation
// tensor cores: tcgen05.mma (kind::f16, BF16 operands from shared memory, FP32
// accumulators in tensor memory), one elected thread issuing, tcgen05.ld epilogue.
//
// Implicit GEMM with shifted shared-memory views. A block owns an output tile
// of 14 x 16 pixels and stores the input tile (one-pixel halo) as 18-pixel-wide
// padded rows in "planes" of 8 channels: byte (c8 * P_IN + pos) * 16 holds
// channels 8 c8 .. 8 c8 + 7 of padded position pos = row * 18 + col. The MMA's
// M dimension runs over 128 consecutive padded positions, so for tap (u, v) the
// A operand is the same planes read from position 18 u + v onwards: a start
// address, no im2col copy. In the no-swizzle K-major layout a core matrix is 8
// consecutive positions x 16 bytes (128 contiguous bytes); the stride between
// 8-position groups (M direction) is 128 bytes and between channel planes (K
// direction) P_IN * 16 bytes. Outputs at padded columns 16, 17 (and past row
// 13) are computed and dropped: 224 of the 256 positions per tile are kept.
// Weights are staged once per block as [tap][c8][c_out][8] (K-major B).
//
// Blocks are persistent: weights and the tensor-memory accumulator (2 M-tiles
// x N columns) are set up once, then each block walks its tiles: load the input
// tile, one thread issues 9 taps x CIN/16 x 2 MMAs and commits them to an
// mbarrier, every warp reads its 32 TMEM lanes (tcgen05.ld 32x32b) and writes
// the epilogue. Every mbarrier wait is bounded; on time-out the block records
// the error in the status word and leaves, releasing its tensor memory.
#include <algorithm>

#include "gs_internal.cuh"

namespace gsk {

namespace {

typedef __nv_bfloat16 bf16;

constexpr int TC_TH = 14, TC_TW = 16;       // output tile
constexpr int TC_PW = TC_TW + 2;            // padded row width
constexpr int TC_ROWS_IN = TC_TH + 3;       // input rows staged (halo + overrun of the last M-tile)
constexpr int TC_PIN = 312;                 // staged positions: >= 17 * 18 = 306, multiple of 8
constexpr int TC_THREADS = 128;
constexpr int TC_MT = 2;                    // M-tiles of 128 positions per tile
constexpr float TC_DETAIL_S = 32.0f;
constexpr long long TC_SPIN_LIMIT = 1LL << 22;

static_assert(TC_MT * 128 >= TC_TH * TC_PW, "the M-tiles cover every output row");
static_assert(TC_MT * 128 - 1 + 2 * TC_PW + 2 < TC_PIN, "taps stay inside the staged rows");
static_assert(TC_ROWS_IN * TC_PW <= TC_PIN, "staged rows fit");

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor, no swizzle (tcgen05 format: start >> 4 in
// bits 0-13, leading-dimension byte offset >> 4 in bits 16-29, stride-dimension
// byte offset >> 4 in bits 32-45, fixed 0b001 in bits 46-48, swizzle mode 0).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
           ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: D = F32 (bits 4-5 = 1), A = B = BF16
// (bits 7-9 = 1, bits 10-12 = 1), both K-major, N >> 3 in bits 17-22, M >> 4 in
// bits 24-28.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(mbar)
        : "memory");
}

__device__ __forceinline__ void fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// Bounded wait for phase `parity` of an mbarrier; false on time-out.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (long long i = 0; i < TC_SPIN_LIMIT; ++i) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(ok)
            : "r"(mbar), "r"(parity)
            : "memory");
        if (ok) return true;
    }
    return false;
}

// 32 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ uint32_t pack2(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *(uint32_t *)&v;
}

__device__ __forceinline__ void bl_src(int o, int n, int &i0, int &i1, float &f) {
    float s = (o + 0.5f) * 0.25f - 0.5f;
    s = fminf(fmaxf(s, 0.0f), (float)(n - 1));
    i0 = (int)s;
    i1 = min(i0 + 1, n - 1);
    f = s - (float)i0;
}

// TMEM columns between the accumulators of the two M-tiles (32-aligned), and
// the allocation (a power of two >= 32).
template <int COUT>
__host__ __device__ constexpr int tmem_stride() {
    return COUT <= 32 ? 32 : 64;
}
template <int COUT>
__host__ __device__ constexpr int tmem_cols() {
    return TC_MT * tmem_stride<COUT>() <= 64 ? 64 : 128;
}

enum : int { TC_EPI_RELU = 0, TC_EPI_UPSAMPLE = 1 };

template <int CIN, int COUT, int EPI>
struct TcSmem {
    static constexpr size_t in_bytes = (size_t)(CIN / 8) * TC_PIN * 16;
    static constexpr size_t w_bytes = (size_t)9 * CIN * COUT * 2;
    static constexpr size_t z_bytes = EPI == TC_EPI_UPSAMPLE ? (size_t)TC_TH * TC_TW * (COUT + 1) * 4 : 0;
    static constexpr size_t l_bytes = EPI == TC_EPI_UPSAMPLE ? (size_t)(TC_TH + 2) * TC_PW * 3 * 4 : 0;
    static constexpr size_t off_w = in_bytes;
    static constexpr size_t off_z = off_w + w_bytes;
    static constexpr size_t off_l = off_z + z_bytes;
    static constexpr size_t off_bias = off_l + l_bytes;
    static constexpr size_t off_bar = off_bias + COUT * 4;
    static constexpr size_t total = off_bar + 16;
};

template <int CIN, int COUT, int EPI>
__global__ void __launch_bounds__(TC_THREADS)
    k_conv_tc(const bf16 *__restrict__ x, int n, int h, int w, const bf16 *__restrict__ wt,
              const float *__restrict__ bias, void *__restrict__ out,
              const float *__restrict__ rgb, int *__restrict__ status) {
    using L = TcSmem<CIN, COUT, EPI>;
    constexpr int NCOL = tmem_cols<COUT>(), CST = tmem_stride<COUT>();
    constexpr uint32_t IDESC = idesc_bf16(128, COUT);
    extern __shared__ __align__(128) unsigned char smem[];
    unsigned char *xs = smem;
    unsigned char *ws = smem + L::off_w;
    float *bs = (float *)(smem + L::off_bias);
    uint64_t *bar = (uint64_t *)(smem + L::off_bar);
    uint32_t *tslot = (uint32_t *)(smem + L::off_bar + 8);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    // weights (already in [tap][c8][co][8] order) and biases, once per block
    for (int i = tid; i < (int)(L::w_bytes / 16); i += TC_THREADS)
        ((uint4 *)ws)[i] = ((const uint4 *)wt)[i];
    for (int i = tid; i < COUT; i += TC_THREADS) bs[i] = bias[i];
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(bar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                         smem_u32(tslot)),
                     "r"(NCOL));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tmem = *tslot;

    const int tx = (w + TC_TW - 1) / TC_TW, ty = (h + TC_TH - 1) / TC_TH;
    const long long n_tiles = (long long)tx * ty * n;
    uint32_t phase = 0;
    bool failed = false;
    for (long long tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int img = (int)(tile / ((long long)tx * ty));
        const int rem = (int)(tile - (long long)img * tx * ty);
        const int by = (rem / tx) * TC_TH, bx = (rem % tx) * TC_TW;
        // input tile, zero outside the image and past the staged rows
        constexpr int C8 = CIN / 8;
        for (int i = tid; i < TC_PIN * C8; i += TC_THREADS) {
            const int c8 = i / TC_PIN, pos = i - c8 * TC_PIN;
            const int yy = by - 1 + pos / TC_PW, xx = bx - 1 + pos % TC_PW;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (pos < TC_ROWS_IN * TC_PW && yy >= 0 && yy < h && xx >= 0 && xx < w)
                v = *(const uint4 *)(x + (((long long)img * h + yy) * w + xx) * CIN + c8 * 8);
            *(uint4 *)(xs + (size_t)i * 16) = v;
        }
        if (EPI == TC_EPI_UPSAMPLE) {
            float *ls = (float *)(smem + L::off_l);
            for (int i = tid; i < (TC_TH + 2) * TC_PW; i += TC_THREADS) {
                const int yy = min(max(by - 1 + i / TC_PW, 0), h - 1);
                const int xx = min(max(bx - 1 + i % TC_PW, 0), w - 1);
                const float *src = rgb + (((long long)img * h + yy) * w + xx) * 3;
                ls[3 * i] = src[0];
                ls[3 * i + 1] = src[1];
                ls[3 * i + 2] = src[2];
            }
        }
        // generic-proxy stores -> visible to the tensor core's async proxy
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        fence_before();
        __syncthreads();
        fence_after();
        if (tid == 0) {
            const uint32_t xa = smem_u32(xs), wa = smem_u32(ws);
#pragma unroll 1
            for (int m = 0; m < TC_MT; ++m) {
#pragma unroll 1
                for (int tap = 0; tap < 9; ++tap) {
                    const int off = (tap / 3) * TC_PW + tap % 3;
#pragma unroll
                    for (int ks = 0; ks < CIN / 16; ++ks) {
                        const uint64_t a = sdesc(xa + (uint32_t)((2 * ks * TC_PIN + m * 128 + off) * 16),
                                                 TC_PIN * 16, 128);
                        const uint64_t b = sdesc(wa + (uint32_t)((tap * C8 + 2 * ks) * COUT * 16),
                                                 COUT * 16, 128);
                        mma_bf16(tmem + (uint32_t)(m * CST), a, b, IDESC, (tap | ks) ? 1u : 0u);
                    }
                }
            }
            mma_commit(smem_u32(bar));
        }
        __syncwarp();
        const bool ok = mbar_wait(smem_u32(bar), phase);
        phase ^= 1u;
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        fence_after();
        // epilogue: warp w owns TMEM lanes 32 w .. 32 w + 31 of each M-tile
#pragma unroll 1
        for (int m = 0; m < TC_MT; ++m) {
            const int p = m * 128 + warp * 32 + lane;
            const int row = p / TC_PW, col = p - row * TC_PW;
            const int yy = by + row, xx = bx + col;
            const bool valid = row < TC_TH && col < TC_TW && yy < h && xx < w;
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(m * CST);
            if (EPI == TC_EPI_RELU) {
                float v[32];
                tmem_ld32(taddr, v);
                if (valid) {
                    uint4 *dst = (uint4 *)((bf16 *)out + (((long long)img * h + yy) * w + xx) * COUT);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        uint4 o;
                        o.x = pack2(fmaxf(v[8 * q + 0] + bs[8 * q + 0], 0.f), fmaxf(v[8 * q + 1] + bs[8 * q + 1], 0.f));
                        o.y = pack2(fmaxf(v[8 * q + 2] + bs[8 * q + 2], 0.f), fmaxf(v[8 * q + 3] + bs[8 * q + 3], 0.f));
                        o.z = pack2(fmaxf(v[8 * q + 4] + bs[8 * q + 4], 0.f), fmaxf(v[8 * q + 5] + bs[8 * q + 5], 0.f));
                        o.w = pack2(fmaxf(v[8 * q + 6] + bs[8 * q + 6], 0.f), fmaxf(v[8 * q + 7] + bs[8 * q + 7], 0.f));
                        dst[q] = o;
                    }
                }
            } else {
                float *zs = (float *)(smem + L::off_z);
                float v[32], v2[16];
                tmem_ld32(taddr, v);
                tmem_ld16(taddr + 32, v2);
                if (row < TC_TH && col < TC_TW) {
                    float *zp = zs + (row * TC_TW + col) * (COUT + 1);
#pragma unroll
                    for (int c = 0; c < 32; ++c) zp[c] = v[c] + bs[c];
#pragma unroll
                    for (int c = 0; c < 16; ++c) zp[32 + c] = v2[c] + bs[32 + c];
                }
            }
        }
        if (EPI == TC_EPI_UPSAMPLE) {
            __syncthreads();
            const float *zs = (const float *)(smem + L::off_z);
            const float *ls = (const float *)(smem + L::off_l);
            const int H4 = 4 * h, W4 = 4 * w;
            constexpr int ROWF = 4 * TC_TW * 3;
            float *o = (float *)out;
            for (int i = tid; i < 4 * TC_TH * ROWF; i += TC_THREADS) {
                const int r = i / ROWF, e = i - r * ROWF;
                const int X = e / 3, c = e - 3 * X;
                const int HY = 4 * by + r, HX = 4 * bx + X;
                if (HY >= H4 || HX >= W4) continue;
                int y0, y1, x0, x1;
                float fy, fx;
                bl_src(HY, h, y0, y1, fy);
                bl_src(HX, w, x0, x1, fx);
                y0 -= by - 1; y1 -= by - 1; x0 -= bx - 1; x1 -= bx - 1;
                const float a00 = ls[3 * (y0 * TC_PW + x0) + c], a01 = ls[3 * (y0 * TC_PW + x1) + c];
                const float a10 = ls[3 * (y1 * TC_PW + x0) + c], a11 = ls[3 * (y1 * TC_PW + x1) + c];
                const float top = fmaf(fx, a01 - a00, a00), bot = fmaf(fx, a11 - a10, a10);
                const float z = zs[((r >> 2) * TC_TW + (X >> 2)) * (COUT + 1) + 16 * c + 4 * (r & 3) + (X & 3)];
                o[(((long long)img * H4 + HY) * W4 + HX) * 3 + c] = fmaf(z, 1.0f / TC_DETAIL_S, fmaf(fy, bot - top, top));
            }
        }
        // TMEM and the staged tiles are reused by the next tile
        fence_before();
        __syncthreads();
        fence_after();
    }
    if (failed && tid == 0) atomicOr(status, 1);
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(NCOL));
}

template <int CIN, int COUT, int EPI>
cudaError_t run_tc(const bf16 *x, int n, int h, int w, const bf16 *wt, const float *bias,
                   void *out, const float *rgb, int *status, int n_sm, cudaStream_t s) {
    using L = TcSmem<CIN, COUT, EPI>;
    auto kern = k_conv_tc<CIN, COUT, EPI>;
    // One block per SM with the largest shared-memory request, so that every
    // operand read the descriptors describe stays inside the block's
    // allocation whatever the tile position.
    const int per_sm = 1;
    const size_t smem = (size_t)227 * 1024;
    static_assert(L::total <= (size_t)227 * 1024, "tile fits shared memory");
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const long long tiles = (long long)((w + TC_TW - 1) / TC_TW) * ((h + TC_TH - 1) / TC_TH) * n;
    if (tiles == 0) return cudaSuccess;
    const int grid = (int)std::min<long long>(tiles, (long long)per_sm * n_sm);
    kern<<<grid, TC_THREADS, smem, s>>>(x, n, h, w, wt, bias, out, rgb, status);
    return cudaGetLastError();
}

}  // namespace

// Forward convolution of layer `layer` on the tensor cores. Layers 0-4 write
// relu(conv + bias) as BF16 NHWC; layer 5 writes the upsampled image
// bilinear4(rgb) + shuffle4(conv + bias) / S (FP32, [n][4h][4w][3]).
cudaError_t up_conv_tc(int layer, const __nv_bfloat16 *x, int n, int h, int w,
                       const __nv_bfloat16 *wt, const float *bias, void *out, const float *rgb,
                       int *status, int n_sm, cudaStream_t s) {
    if (layer == 0)
        return run_tc<16, 32, TC_EPI_RELU>(x, n, h, w, wt, bias, out, nullptr, status, n_sm, s);
    if (layer < 5)
        return run_tc<32, 32, TC_EPI_RELU>(x, n, h, w, wt, bias, out, nullptr, status, n_sm, s);
    return run_tc<32, 48, TC_EPI_UPSAMPLE>(x, n, h, w, wt, bias, out, rgb, status, n_sm, s);
}

}  // namespace gsk
