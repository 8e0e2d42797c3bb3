// proj_core.cuh -- the per (camera, Gaussian) projection arithmetic shared by
// the projection passes (k_project.cu) and the record pass of the progressive
// depth order (k_bin.cu): camera constants, a Gaussian's geometry, the EWA
// projection with its culling tests, the real SH basis. Every caller runs the
// same instructions, so a record is the same bit for bit whichever pass
// computes it.
#pragma once

#include <type_traits>

#include "gs_internal.cuh"

namespace gsk {

namespace {

// 28 words = 7 float4 (loaded as such from shared memory)
struct __align__(16) CamProj {
    float R[9], t[3];
    float fx, fy, cx, cy;
    float lxp, lxn, lyp, lyn;  // guard-band limits of x/z and y/z
    float cpos[3];             // camera centre in world coordinates
    float kk;                  // bound of z^2 |J|_F^2 over the guard band
    float W, H;
    int TX, TY;
};
static_assert(sizeof(CamProj) == 7 * 16, "CamProj is seven float4");

__device__ __forceinline__ CamProj load_cam(const CamProj &src) {
    CamProj c;
    const float4 *s4 = reinterpret_cast<const float4 *>(&src);
    float4 *d4 = reinterpret_cast<float4 *>(&c);
#pragma unroll
    for (int k = 0; k < 7; ++k) d4[k] = s4[k];
    return c;
}

struct GaussGeo {
    float mx, my, mz;
    float M[9];   // R(q) diag(exp(log_scale)), row-major
    float smax2;  // largest scale squared (largest eigenvalue of Sigma)
};

struct Proj {
    float u, v, z, A, B, C, r;
    float sa, sc;  // 2D covariance diagonal (with the dilation)
    int x0, x1, y0, y1;
};

// Hardware approximations (PTX rcp/sqrt .approx): a few ulp, far inside the
// parity tolerances. Both projection passes run these same instructions.
__device__ __forceinline__ float rcp_a(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float sqrt_a(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_a(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2_a(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float ldv(const void *p, long long i, int dt) {
    if (dt == DT_F32) return __ldg(reinterpret_cast<const float *>(p) + i);
    if (dt == DT_F16) return __half2float(reinterpret_cast<const __half *>(p)[i]);
    return __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(p)[i]);
}

template <typename T>
__device__ __forceinline__ float ldt(const void *p, long long i) {
    if constexpr (sizeof(T) == 4)
        return __ldg(reinterpret_cast<const float *>(p) + i);
    else if constexpr (std::is_same<T, __half>::value)
        return __half2float(__ldg(reinterpret_cast<const __half *>(p) + i));
    else
        return __bfloat162float(__ldg(reinterpret_cast<const __nv_bfloat16 *>(p) + i));
}

// Mean and M = R(q) S of Gaussian g (quaternion normalised here), attributes of type T.
template <typename T>
__device__ __forceinline__ void load_geo_t(const SceneDev &s, long long g, GaussGeo &G) {
    const long long n = s.n;
    G.mx = ldt<T>(s.mean, g);
    G.my = ldt<T>(s.mean, n + g);
    G.mz = ldt<T>(s.mean, 2 * n + g);
    const float sx = expf(ldt<T>(s.log_scale, g));
    const float sy = expf(ldt<T>(s.log_scale, n + g));
    const float sz = expf(ldt<T>(s.log_scale, 2 * n + g));
    const float sm = fmaxf(sx, fmaxf(sy, sz));
    G.smax2 = __fmul_rn(sm, sm);
    float w = ldt<T>(s.quat, g), x = ldt<T>(s.quat, n + g);
    float y = ldt<T>(s.quat, 2 * n + g), z = ldt<T>(s.quat, 3 * n + g);
    // (explicit roundings: the compiler may not fuse these differently in the
    // kernels that compute a Gaussian's geometry)
    const float qq = fmaf(w, w, fmaf(x, x, fmaf(y, y, __fmul_rn(z, z))));
    if (qq > 0.0f) {
        const float inv = __fdiv_rn(1.0f, __fsqrt_rn(qq));
        w = __fmul_rn(w, inv);
        x = __fmul_rn(x, inv);
        y = __fmul_rn(y, inv);
        z = __fmul_rn(z, inv);
    } else {
        w = 1.0f;
        x = y = z = 0.0f;
    }
    const float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
    const float xy = __fmul_rn(x, y), xz = __fmul_rn(x, z), yz = __fmul_rn(y, z);
    const float wx = __fmul_rn(w, x), wy = __fmul_rn(w, y), wz = __fmul_rn(w, z);
    G.M[0] = __fmul_rn(fmaf(-2.0f, __fadd_rn(yy, zz), 1.0f), sx);
    G.M[1] = __fmul_rn(__fmul_rn(2.0f, __fsub_rn(xy, wz)), sy);
    G.M[2] = __fmul_rn(__fmul_rn(2.0f, __fadd_rn(xz, wy)), sz);
    G.M[3] = __fmul_rn(__fmul_rn(2.0f, __fadd_rn(xy, wz)), sx);
    G.M[4] = __fmul_rn(fmaf(-2.0f, __fadd_rn(xx, zz), 1.0f), sy);
    G.M[5] = __fmul_rn(__fmul_rn(2.0f, __fsub_rn(yz, wx)), sz);
    G.M[6] = __fmul_rn(__fmul_rn(2.0f, __fsub_rn(xz, wy)), sx);
    G.M[7] = __fmul_rn(__fmul_rn(2.0f, __fadd_rn(yz, wx)), sy);
    G.M[8] = __fmul_rn(fmaf(-2.0f, __fadd_rn(xx, yy), 1.0f), sz);
}

// The storage type is uniform per scene: one branch, then loads of a fixed type.
__device__ __forceinline__ void load_geo(const SceneDev &s, long long g, GaussGeo &G) {
    if (s.geo_dtype == DT_F32)
        load_geo_t<float>(s, g, G);
    else if (s.geo_dtype == DT_F16)
        load_geo_t<__half>(s, g, G);
    else
        load_geo_t<__nv_bfloat16>(s, g, G);
}

// The cheap first part of project(): near plane and the cull with a bound of
// the radius. lambda_max(Sigma') <= |J|_F^2 s_max^2 + dil and |J|_F^2 <= kk / z^2
// over the guard band; the 1.002 and +0.02 px margins keep rb above the float32
// radius, so this culls only what the exact test culls. project() calls it, so
// a pair it rejects is exactly a pair project() rejects here.
__device__ __forceinline__ bool prefilter(const CamProj &c, const GaussGeo &G, const ProjParams &P,
                                          float &z, float &iz, float &xz, float &yz, float &u,
                                          float &v) {
    const float px = fmaf(c.R[0], G.mx, fmaf(c.R[1], G.my, fmaf(c.R[2], G.mz, c.t[0])));
    const float py = fmaf(c.R[3], G.mx, fmaf(c.R[4], G.my, fmaf(c.R[5], G.mz, c.t[1])));
    z = fmaf(c.R[6], G.mx, fmaf(c.R[7], G.my, fmaf(c.R[8], G.mz, c.t[2])));
    if (!(z > P.near_plane)) return false;
    iz = rcp_a(z);
    xz = __fmul_rn(px, iz);
    yz = __fmul_rn(py, iz);
    u = fmaf(c.fx, xz, c.cx);
    v = fmaf(c.fy, yz, c.cy);
    const float rb = fmaf(1.002f * P.sigma, sqrt_a(fmaf(c.kk * iz * iz, G.smax2, P.dilation)), 0.02f);
    return !(u + rb < 0.0f || u - rb >= c.W || v + rb < 0.0f || v - rb >= c.H);
}

// CULL = false: the values of a pair known to survive (the write pass), without
// the radius bound and the cull tests; every value is computed by the same
// operations as with CULL = true, so it is the same bit for bit.
template <bool CULL = true>
__device__ __forceinline__ bool project(const CamProj &c, const GaussGeo &G,
                                        const ProjParams &P, Proj &o) {
    float z, iz, xz, yz, u, v;
    if (CULL) {
        const bool pre = prefilter(c, G, P, z, iz, xz, yz, u, v);
        o.z = z;
        if (!pre) return false;
    } else {
        const float px = fmaf(c.R[0], G.mx, fmaf(c.R[1], G.my, fmaf(c.R[2], G.mz, c.t[0])));
        const float py = fmaf(c.R[3], G.mx, fmaf(c.R[4], G.my, fmaf(c.R[5], G.mz, c.t[1])));
        z = fmaf(c.R[6], G.mx, fmaf(c.R[7], G.my, fmaf(c.R[8], G.mz, c.t[2])));
        iz = rcp_a(z);
        xz = __fmul_rn(px, iz);
        yz = __fmul_rn(py, iz);
        u = fmaf(c.fx, xz, c.cx);
        v = fmaf(c.fy, yz, c.cy);
        o.z = z;
    }
    const float xc = fminf(fmaxf(xz, -c.lxn), c.lxp);
    const float yc = fminf(fmaxf(yz, -c.lyn), c.lyp);
    const float j00 = __fmul_rn(c.fx, iz), j02 = -__fmul_rn(__fmul_rn(c.fx, xc), iz);
    const float j11 = __fmul_rn(c.fy, iz), j12 = -__fmul_rn(__fmul_rn(c.fy, yc), iz);
    float T0[3], T1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        T0[k] = fmaf(j00, c.R[k], __fmul_rn(j02, c.R[6 + k]));
        T1[k] = fmaf(j11, c.R[3 + k], __fmul_rn(j12, c.R[6 + k]));
    }
    float g0[3], g1[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        g0[k] = fmaf(T0[0], G.M[k], fmaf(T0[1], G.M[3 + k], __fmul_rn(T0[2], G.M[6 + k])));
        g1[k] = fmaf(T1[0], G.M[k], fmaf(T1[1], G.M[3 + k], __fmul_rn(T1[2], G.M[6 + k])));
    }
    const float s00 = fmaf(g0[0], g0[0], fmaf(g0[1], g0[1], __fmul_rn(g0[2], g0[2])));
    const float s11 = fmaf(g1[0], g1[0], fmaf(g1[1], g1[1], __fmul_rn(g1[2], g1[2])));
    const float s01 = fmaf(g0[0], g1[0], fmaf(g0[1], g1[1], __fmul_rn(g0[2], g1[2])));
    const float dil = P.dilation;
    const float a = __fadd_rn(s00, dil), cc = __fadd_rn(s11, dil), b = s01;
    const float hd = __fmul_rn(0.5f, __fsub_rn(a, cc));
    const float lmax = fmaf(0.5f, __fadd_rn(a, cc), sqrt_a(fmaf(hd, hd, __fmul_rn(b, b))));
    const float r = __fmul_rn(P.sigma, sqrt_a(lmax));
    if (CULL && (!(__fadd_rn(u, r) >= 0.0f) || !(__fsub_rn(u, r) < c.W) ||
                 !(__fadd_rn(v, r) >= 0.0f) || !(__fsub_rn(v, r) < c.H)))
        return false;
    o.x0 = (int)fmaxf(floorf(__fmul_rn(__fsub_rn(u, r), 0.0625f)), 0.0f);
    o.x1 = (int)fminf(floorf(__fmul_rn(__fadd_rn(u, r), 0.0625f)), (float)(c.TX - 1));
    o.y0 = (int)fmaxf(floorf(__fmul_rn(__fsub_rn(v, r), 0.0625f)), 0.0f);
    o.y1 = (int)fminf(floorf(__fmul_rn(__fadd_rn(v, r), 0.0625f)), (float)(c.TY - 1));
    // conic: only the write pass uses it
    const float e0 = fmaf(g0[1], g1[2], -__fmul_rn(g0[2], g1[1]));
    const float e1 = fmaf(g0[2], g1[0], -__fmul_rn(g0[0], g1[2]));
    const float e2 = fmaf(g0[0], g1[1], -__fmul_rn(g0[1], g1[0]));
    const float det = fmaf(dil, __fadd_rn(__fadd_rn(s00, s11), dil),
                           fmaf(e0, e0, fmaf(e1, e1, __fmul_rn(e2, e2))));
    const float idet = rcp_a(det);
    o.A = cc * idet;
    o.B = -b * idet;
    o.C = a * idet;
    o.sa = a;
    o.sc = cc;
    o.u = u;
    o.v = v;
    o.r = r;
    return true;
}

// Real SH basis (Condon-Shortley phase), l-major with m = -l..l, constants
// written as their closed forms sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!) times the
// factors of the Cartesian polynomials.
// (Explicit roundings throughout: every degree and every kernel evaluates
// these terms with the same instructions.)
__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float *Y) {
    Y[0] = 0.28209479177387814f;  // 1/(2 sqrt(pi))
    if (deg >= 1) {
        const float c1 = 0.4886025119029199f;  // sqrt(3/(4 pi))
        Y[1] = __fmul_rn(-c1, y);
        Y[2] = __fmul_rn(c1, z);
        Y[3] = __fmul_rn(-c1, x);
    }
    if (deg >= 2) {
        const float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
        const float c2 = 1.0925484305920792f;                                // sqrt(15/(4 pi))
        Y[4] = __fmul_rn(__fmul_rn(c2, x), y);
        Y[5] = __fmul_rn(__fmul_rn(-c2, y), z);
        Y[6] = __fmul_rn(0.31539156525252005f, fmaf(3.0f, zz, -1.0f));    // sqrt(5/(16 pi))
        Y[7] = __fmul_rn(__fmul_rn(-c2, x), z);
        Y[8] = __fmul_rn(0.5462742152960396f, __fsub_rn(xx, yy));         // sqrt(15/(16 pi))
        if (deg >= 3) {
            const float c9 = 0.5900435899266435f, c11 = 0.4570457994644658f;
            Y[9] = __fmul_rn(__fmul_rn(-c9, y), fmaf(3.0f, xx, -yy));      // sqrt(35/(32 pi))
            Y[10] = __fmul_rn(__fmul_rn(__fmul_rn(2.890611442640554f, x), y), z);  // sqrt(105/(4 pi))
            Y[11] = __fmul_rn(__fmul_rn(-c11, y), fmaf(5.0f, zz, -1.0f));  // sqrt(21/(32 pi))
            Y[12] = __fmul_rn(__fmul_rn(0.3731763325901154f, z), fmaf(5.0f, zz, -3.0f));  // sqrt(7/(16 pi))
            Y[13] = __fmul_rn(__fmul_rn(-c11, x), fmaf(5.0f, zz, -1.0f));
            Y[14] = __fmul_rn(__fmul_rn(1.445305721320277f, z), __fsub_rn(xx, yy));  // sqrt(105/(16 pi))
            Y[15] = __fmul_rn(__fmul_rn(-c9, x), fmaf(-3.0f, yy, xx));
        }
    }
}

// The unit view direction from camera centre cpos to the mean (z axis when they
// coincide), with explicit roundings.
__device__ __forceinline__ void sh_dir(const float *cpos, float mx, float my, float mz, float &dx,
                                       float &dy, float &dz) {
    dx = __fsub_rn(mx, cpos[0]);
    dy = __fsub_rn(my, cpos[1]);
    dz = __fsub_rn(mz, cpos[2]);
    const float dd = fmaf(dx, dx, fmaf(dy, dy, __fmul_rn(dz, dz)));
    if (dd > 0.0f) {
        const float inv = rsqrt_a(dd);
        dx = __fmul_rn(dx, inv);
        dy = __fmul_rn(dy, inv);
        dz = __fmul_rn(dz, inv);
    } else {
        dx = 0.0f;
        dy = 0.0f;
        dz = 1.0f;
    }
}

// log2 of a Gaussian's opacity sigmoid(logit), with explicit roundings.
__device__ __forceinline__ float log2_opacity(float logit) {
    return lg2_a(__fdiv_rn(1.0f, __fadd_rn(1.0f, expf(-logit))));
}

constexpr float LOG2E = 1.4426950408889634f;

}  // namespace

}  // namespace gsk
