// k_scene.cu -- spatial order of a scene's Gaussians, set up once at upload,
// and the bounds of the projection blocks.
//
// The projection's mask pass tests each warp's 32 consecutive Gaussians as a
// group against each camera before the Gaussians themselves: a group entirely
// outside the view culls all of them, a group entirely inside keeps all of
// them, and only the groups in between are tested Gaussian by Gaussian. That pays only when a block's Gaussians are close together in
// space, so the library stores a scene in Morton (Z-curve) order of the means:
// 10 bits per axis of the means' bounding box, a stable radix sort of the
// 30-bit codes, then a gather of every attribute row. orig[p] keeps the
// caller's index of the Gaussian stored at position p; the renderer orders
// equal depths by it and the inspection entry points report it.
//
// Rows per Gaussian (k_scene_rows): the progressive depth order computes the
// records of the ranks it renders after the depth order, at scattered
// positions, so each Gaussian also gets its geometry as the projection passes
// derive it (mean, log2 opacity, M = R(q) S: 64 bytes) and its SH coefficients
// channel-major in one row (load_geo and the opacity expression of
// proj_core.cuh, so the records are those the projection's write pass makes).
#include <algorithm>
#include <type_traits>

#include "proj_core.cuh"

namespace gsk {

namespace {

// float <-> unsigned with the same order (for atomic min / max)
__device__ __forceinline__ unsigned ord_of(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float float_of(unsigned o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

template <typename T>
__device__ __forceinline__ float ld(const void *p, long long i) {
    if constexpr (sizeof(T) == 4)
        return reinterpret_cast<const float *>(p)[i];
    else if constexpr (std::is_same<T, __half>::value)
        return __half2float(reinterpret_cast<const __half *>(p)[i]);
    else
        return __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(p)[i]);
}

__global__ void k_box_init(unsigned *box) {
    if (threadIdx.x < 6) box[threadIdx.x] = threadIdx.x < 3 ? 0xffffffffu : 0u;
}

// box[0..2] = ordered min of x, y, z over the finite means; box[3..5] = max
template <typename T>
__global__ void k_bbox(const void *mean, long long n, unsigned *box) {
    unsigned lo[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu}, hi[3] = {0u, 0u, 0u};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float v = ld<T>(mean, a * n + i);
            if (isfinite(v)) {
                lo[a] = min(lo[a], ord_of(v));
                hi[a] = max(hi[a], ord_of(v));
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) {
            lo[a] = min(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], d));
            hi[a] = max(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], d));
        }
        if ((threadIdx.x & 31) == 0) {
            atomicMin(box + a, lo[a]);
            atomicMax(box + 3 + a, hi[a]);
        }
    }
}

__device__ __forceinline__ uint32_t spread10(uint32_t x) {  // bit k -> bit 3k
    x &= 0x3ffu;
    x = (x | (x << 16)) & 0x030000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

template <typename T>
__global__ void k_morton(const void *mean, long long n, const unsigned *box, uint32_t *code,
                         uint32_t *idx) {
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float lo = float_of(box[a]), hi = float_of(box[3 + a]);
        const float v = ld<T>(mean, a * n + i);
        const float span = hi - lo;
        float t = span > 0.0f ? (v - lo) / span * 1024.0f : 0.0f;
        if (!(t >= 0.0f)) t = 0.0f;  // also NaN
        q[a] = (uint32_t)fminf(t, 1023.0f);
    }
    code[i] = spread10(q[0]) | (spread10(q[1]) << 1) | (spread10(q[2]) << 2);
    idx[i] = (uint32_t)i;
}

// dst[r n + p] = src[r n + perm[p]] for rows r < rows; element size 2 or 4 bytes
template <typename E>
__global__ void k_gather_rows(const E *__restrict__ src, E *__restrict__ dst,
                              const uint32_t *__restrict__ perm, long long n, int rows) {
    for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
         p += (long long)gridDim.x * blockDim.x) {
        const long long s = perm[p];
        for (int r = 0; r < rows; ++r) dst[r * n + p] = src[r * n + s];
    }
}

// Per group of 32 stored Gaussians (one warp of the projection): bounds[2b] =
// (min x, y, z of the means, largest squared scale), bounds[2b + 1] = (max x,
// y, z, 1 if every mean and scale of the group is finite else 0). The squared
// scale is computed exactly as the projection computes it (expf of the stored
// log-scale).
template <typename T>
__global__ void __launch_bounds__(256)
    k_block_bounds(const void *mean, const void *log_scale, long long n, float4 *bounds) {
    const long long g = blockIdx.x * 256LL + threadIdx.x;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    float s2 = 0.0f;
    int finite = 1;
    if (g < n) {
        float sm = 0.0f;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float v = ld<T>(mean, a * n + g);
            lo[a] = hi[a] = v;
            const float s = expf(ld<T>(log_scale, a * n + g));
            sm = fmaxf(sm, s);
            finite &= isfinite(v) && isfinite(s);
        }
        s2 = sm * sm;
        finite &= isfinite(s2);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], d));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], d));
        }
        s2 = fmaxf(s2, __shfl_xor_sync(0xffffffffu, s2, d));
        finite &= __shfl_xor_sync(0xffffffffu, finite, d);
    }
    const long long wb = g >> 5;
    if ((threadIdx.x & 31) == 0 && (wb << 5) < n) {
        bounds[2 * wb] = make_float4(lo[0], lo[1], lo[2], s2);
        bounds[2 * wb + 1] = make_float4(hi[0], hi[1], hi[2], (float)finite);
    }
}

template <typename F>
void by_dtype(int dt, F &&f) {
    if (dt == DT_F32)
        f(float{});
    else if (dt == DT_F16)
        f(__half{});
    else
        f(__nv_bfloat16{});
}

// One thread per Gaussian: its geometry row (4 float4) and SH row (48
// elements of the appearance type, raw bits; zero past the degree).
template <typename A>
__global__ void k_scene_rows(const SceneDev s, float4 *__restrict__ geo, A *__restrict__ shr,
                             int *__restrict__ pos_of) {
    const int K = (s.deg + 1) * (s.deg + 1);
    const A *sh = reinterpret_cast<const A *>(s.sh);
    for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < s.n;
         g += (long long)gridDim.x * blockDim.x) {
        GaussGeo G;
        load_geo(s, g, G);
        const float log2o = log2_opacity(ldv(s.logit, g, s.app_dtype));
        pos_of[s.orig[g]] = (int)g;
        geo[4 * g + 0] = make_float4(G.mx, G.my, G.mz, log2o);
        geo[4 * g + 1] = make_float4(G.M[0], G.M[1], G.M[2], G.M[3]);
        geo[4 * g + 2] = make_float4(G.M[4], G.M[5], G.M[6], G.M[7]);
        geo[4 * g + 3] = make_float4(G.M[8], 0.0f, 0.0f, 0.0f);
        for (int ch = 0; ch < 3; ++ch)
            for (int k = 0; k < 16; ++k)
                shr[48 * g + 16 * ch + k] = k < K ? sh[(long long)(3 * k + ch) * s.n + g] : A(0);
    }
}

}  // namespace

cudaError_t launch_scene_rows(const SceneDev &s, float4 *geo_rows, void *sh_rows, int *pos_of,
                              cudaStream_t st) {
    if (s.n <= 0) return cudaSuccess;
    const int grid = (int)std::min<long long>((s.n + 255) / 256, 148 * 16);
    if (s.app_dtype == DT_F32)
        k_scene_rows<uint32_t><<<grid, 256, 0, st>>>(s, geo_rows, (uint32_t *)sh_rows, pos_of);
    else
        k_scene_rows<uint16_t><<<grid, 256, 0, st>>>(s, geo_rows, (uint16_t *)sh_rows, pos_of);
    return cudaGetLastError();
}

cudaError_t launch_scene_morton(const void *mean, int dtype, long long n, unsigned *box,
                                uint32_t *code, uint32_t *idx, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_box_init<<<1, 32, 0, s>>>(box);
    const int grid = (int)std::min<long long>((n + 255) / 256, 148LL * 8);
    by_dtype(dtype, [&](auto tag) {
        using T = decltype(tag);
        k_bbox<T><<<grid, 256, 0, s>>>(mean, n, box);
        k_morton<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(mean, n, box, code, idx);
    });
    return cudaGetLastError();
}

cudaError_t launch_gather_rows(const void *src, void *dst, int elem_bytes, const uint32_t *perm,
                               long long n, int rows, cudaStream_t s) {
    if (n == 0 || rows == 0) return cudaSuccess;
    const int grid = (int)std::min<long long>((n + 255) / 256, 148LL * 16);
    if (elem_bytes == 4)
        k_gather_rows<uint32_t><<<grid, 256, 0, s>>>((const uint32_t *)src, (uint32_t *)dst, perm,
                                                     n, rows);
    else
        k_gather_rows<uint16_t><<<grid, 256, 0, s>>>((const uint16_t *)src, (uint16_t *)dst, perm,
                                                     n, rows);
    return cudaGetLastError();
}

long long scene_blocks(long long n) { return (n + 31) / 32; }

cudaError_t launch_block_bounds(const void *mean, const void *log_scale, int dtype, long long n,
                                float4 *bounds, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    by_dtype(dtype, [&](auto tag) {
        using T = decltype(tag);
        k_block_bounds<T><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(mean, log_scale, n, bounds);
    });
    return cudaGetLastError();
}

}  // namespace gsk
