// k_blur.cu -- camera arrays derived on the device: poses for motion blur and
// intrinsics at a reduced resolution. The paper simulates blur by
// rendering a few frames offset along the camera's velocity and blending them
// into one image (Sec. 3.3, Fig. 9). Sub-frame j of k has its centre moved by
// v * shutter * (j/(k-1) - 1/2); the orientation is kept, so only the
// translation column changes: t_j = t - R d_j.
#include "gs_internal.cuh"

namespace gsk {

namespace {

__global__ void k_blur_poses(const float *__restrict__ vm, const float *__restrict__ vel, int n,
                             int k, float shutter, float *__restrict__ out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= n * k) return;
    const int j = idx / n, i = idx - j * n;
    const float frac = k > 1 ? (float)j / (float)(k - 1) - 0.5f : 0.0f;
    const float d0 = vel[3 * i] * shutter * frac, d1 = vel[3 * i + 1] * shutter * frac,
                d2 = vel[3 * i + 2] * shutter * frac;
    const float *a = vm + 16LL * i;
    float *o = out + 16LL * idx;
#pragma unroll
    for (int e = 0; e < 16; ++e) o[e] = a[e];
#pragma unroll
    for (int r = 0; r < 3; ++r)
        o[4 * r + 3] = a[4 * r + 3] - (a[4 * r] * d0 + a[4 * r + 1] * d1 + a[4 * r + 2] * d2);
}

// Intrinsics of the same cameras at 1/f of the resolution: (fx, fy, cx, cy) / f
// (pixel centres (i + 1/2) map to (i + 1/2) / f).
__global__ void k_scale_intrinsics(const float *__restrict__ in, int n, float f,
                                   float *__restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < 4 * n) out[i] = in[i] / f;
}

}  // namespace

cudaError_t launch_scale_intrinsics(const float *in, int n, float f, float *out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_scale_intrinsics<<<(4 * n + 255) / 256, 256, 0, s>>>(in, n, f, out);
    return cudaGetLastError();
}

cudaError_t launch_blur_poses(const float *vm, const float *vel, int n, int k, float shutter,
                              float *out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const int total = n * k;
    k_blur_poses<<<(total + 255) / 256, 256, 0, s>>>(vm, vel, n, k, shutter, out);
    return cudaGetLastError();
}

}  // namespace gsk
