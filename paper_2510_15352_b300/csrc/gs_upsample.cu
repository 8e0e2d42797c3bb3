// gs_upsample.cu -- C ABI of the learned 4x upsampler (inference, gradients,
// Adam), on the kernels of k_upsample.cu.
//
// Parameters are one flat FP32 array, layer by layer: weights [c_out][c_in][3][3]
// then biases [c_out], for the layers (c_out, c_in) = (32, 6), 4 x (32, 32),
// (48, 32) -- 52,624 values. The library keeps them as FP32 masters plus BF16
// copies in the layouts the convolution kernels read.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "gs.h"
#include "gs_internal.cuh"

namespace gsk {
cudaError_t up_prep_input(const float *rgb, int n, int h, int w, __nv_bfloat16 *x0,
                          cudaStream_t s);
cudaError_t up_conv_forward(int layer, const __nv_bfloat16 *x, int n, int h, int w,
                            const __nv_bfloat16 *wt, const float *bias, void *out,
                            cudaStream_t s);
cudaError_t up_conv_upsample(const __nv_bfloat16 *x, int n, int h, int w,
                             const __nv_bfloat16 *wt, const float *bias, const float *rgb,
                             float *out, cudaStream_t s);
cudaError_t up_conv_dgrad(int layer, const __nv_bfloat16 *dz, int n, int h, int w,
                          const __nv_bfloat16 *wd, const __nv_bfloat16 *act,
                          __nv_bfloat16 *dx, cudaStream_t s);
cudaError_t up_wgrad(int layer, const __nv_bfloat16 *x, const __nv_bfloat16 *dz, int n, int h,
                     int w, float *gW, float *gb, int n_sm, cudaStream_t s);
cudaError_t up_wgrad_tc(int layer, const __nv_bfloat16 *x, const __nv_bfloat16 *dz, int n, int h,
                        int w, float *gW, float *gb, int *status, int n_sm, cudaStream_t s);
cudaError_t up_loss(const float *z, const float *rgb, const float *target, int n, int h, int w,
                    __nv_bfloat16 *dz, float *loss, cudaStream_t s);
cudaError_t up_bilinear1(const float *src, int n, int h, int w, float *dst, cudaStream_t s);
cudaError_t up_adam(float *p, float *m, float *v, const float *g, int co, int ci, int cin_pad,
                    float lr, float b1, float b2, float eps, float c1, float c2,
                    __nv_bfloat16 *wf, __nv_bfloat16 *wd, __nv_bfloat16 *wt, __nv_bfloat16 *wdt,
                    cudaStream_t s);
cudaError_t up_weights_bf16(const float *p, int co, int ci, int cin_pad, __nv_bfloat16 *wf,
                            __nv_bfloat16 *wd, __nv_bfloat16 *wt, __nv_bfloat16 *wdt,
                            cudaStream_t s);
cudaError_t up_conv_tc_linear(const __nv_bfloat16 *x, int n, int h, int w,
                              const __nv_bfloat16 *wt, const float *bias, float *z, int *status,
                              int n_sm, cudaStream_t s);
cudaError_t up_conv_tc_timeout_probe(const __nv_bfloat16 *x, int n, int h, int w,
                                     const __nv_bfloat16 *wt, const float *bias, __nv_bfloat16 *out,
                                     int *status, int n_sm, long long spin_limit, cudaStream_t s);
cudaError_t up_conv_tc_timeout_probe_up(const __nv_bfloat16 *x, int n, int h, int w,
                                        const __nv_bfloat16 *wt, const float *bias,
                                        const float *rgb, const float *lr_depth, float *hr,
                                        float *hr_depth, int *status, int n_sm,
                                        long long spin_limit, cudaStream_t s);
cudaError_t up_dgrad_tc(int layer, const __nv_bfloat16 *dz, int n, int h, int w,
                        const __nv_bfloat16 *wdt, const __nv_bfloat16 *act, __nv_bfloat16 *dx,
                        int *status, int n_sm, cudaStream_t s);
cudaError_t up_conv_tc(int layer, const __nv_bfloat16 *x, int n, int h, int w,
                       const __nv_bfloat16 *wt, const float *bias, void *out, const float *rgb,
                       const float *lr_depth, float *hr_depth, int *status, int n_sm,
                       cudaStream_t s);
cudaError_t up_conv_tc_planar(int layer, const __nv_bfloat16 *x, int n, int h, int w,
                              const __nv_bfloat16 *wt, const float *bias, void *out,
                              const float *rgb, const float *lr_depth, float *hr_depth,
                              int *status, int n_sm, cudaStream_t s);
cudaError_t up_prep_input_plane(const float *rgb, int n, int h, int w, __nv_bfloat16 *x0,
                                cudaStream_t s);
}  // namespace gsk

namespace {

using bf16 = __nv_bfloat16;
constexpr int NL = 6;
constexpr int L_CO[NL] = {32, 32, 32, 32, 32, 48};
constexpr int L_CI[NL] = {6, 32, 32, 32, 32, 32};
constexpr int L_CIP[NL] = {16, 32, 32, 32, 32, 32};  // input channels as stored (padded)

constexpr long long layer_size(int l) { return (long long)L_CO[l] * L_CI[l] * 9 + L_CO[l]; }
long long layer_off(int l) {
    long long o = 0;
    for (int i = 0; i < l; ++i) o += layer_size(i);
    return o;
}
constexpr long long N_PARAMS = 1760 + 4 * 9248 + 13872;

// Inference works on frames in groups whose activations fit this budget.
constexpr size_t INFER_BYTES = size_t(1) << 30;

struct Buf {
    void *p = nullptr;
    size_t cap = 0;
};

}  // namespace

struct gs_upsampler {
    int device = 0, n_sm = 148;
    float *params = nullptr, *grads = nullptr, *m = nullptr, *v = nullptr;
    bf16 *wf[NL] = {}, *wd[NL] = {}, *wt[NL] = {}, *wdt[NL] = {};
    bf16 *wblock = nullptr;
    int *status = nullptr;  // device: set when a tensor-core kernel timed out
    int backend = GS_UPSAMPLE_TCGEN05;
    long long steps = 0;
    Buf work;
    std::string err;
};

namespace {

gs_status fail(gs_upsampler *u, gs_status s, const std::string &msg) {
    if (u) u->err = msg;
    return s;
}

gs_status cuda_fail(gs_upsampler *u, cudaError_t e, const char *what) {
    return fail(u, e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

cudaError_t grow(Buf &b, size_t bytes) {
    if (b.cap >= bytes) return cudaSuccess;
    if (b.p) cudaFree(b.p);
    b.p = nullptr;
    b.cap = 0;
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e == cudaSuccess) b.cap = bytes;
    return e;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

cudaError_t refresh_bf16(gs_upsampler *u, cudaStream_t s) {
    for (int l = 0; l < NL; ++l) {
        cudaError_t e = gsk::up_weights_bf16(u->params + layer_off(l), L_CO[l], L_CI[l], L_CIP[l],
                                             u->wf[l], l > 0 ? u->wd[l] : nullptr, u->wt[l],
                                             l > 0 ? u->wdt[l] : nullptr, s);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

}  // namespace

extern "C" {

int64_t gs_upsampler_param_count(void) { return N_PARAMS; }

gs_status gs_upsampler_create(int32_t device, gs_upsampler **out) {
    if (!out) return GS_ERR_INVALID_ARG;
    *out = nullptr;
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev)
        return GS_ERR_INVALID_ARG;
    DeviceGuard dg(device);
    gs_upsampler *u = new gs_upsampler();
    u->device = device;
    cudaDeviceGetAttribute(&u->n_sm, cudaDevAttrMultiProcessorCount, device);
    size_t wbytes = 0;
    for (int l = 0; l < NL; ++l)
        wbytes += 4 * align256((size_t)9 * L_CO[l] * std::max(L_CIP[l], L_CI[l]) * sizeof(bf16));
    wbytes += 256;  // status word
    cudaError_t e = cudaMalloc(&u->params, 4 * N_PARAMS * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&u->wblock, wbytes);
    if (e != cudaSuccess) {
        cudaFree(u->params);
        delete u;
        return e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA;
    }
    u->grads = u->params + N_PARAMS;
    u->m = u->grads + N_PARAMS;
    u->v = u->m + N_PARAMS;
    cudaMemset(u->params, 0, 4 * N_PARAMS * sizeof(float));
    cudaMemset(u->wblock, 0, wbytes);  // also the zero padding of layer 0's inputs
    char *w = (char *)u->wblock;
    for (int l = 0; l < NL; ++l) {
        const size_t sz = align256((size_t)9 * L_CO[l] * std::max(L_CIP[l], L_CI[l]) * sizeof(bf16));
        u->wf[l] = (bf16 *)w;
        u->wd[l] = (bf16 *)(w + sz);
        u->wt[l] = (bf16 *)(w + 2 * sz);
        u->wdt[l] = (bf16 *)(w + 3 * sz);
        w += 4 * sz;
    }
    u->status = (int *)w;
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(u->params);
        cudaFree(u->wblock);
        delete u;
        return GS_ERR_CUDA;
    }
    *out = u;
    return GS_OK;
}

void gs_upsampler_destroy(gs_upsampler *u) {
    if (!u) return;
    DeviceGuard dg(u->device);
    cudaFree(u->params);
    cudaFree(u->wblock);
    if (u->work.p) cudaFree(u->work.p);
    delete u;
}

const char *gs_upsampler_last_error(gs_upsampler *u) { return u ? u->err.c_str() : ""; }

gs_status gs_upsampler_set_params(gs_upsampler *u, const float *host_params, int64_t n) {
    if (!u || !host_params || n != N_PARAMS) return fail(u, GS_ERR_INVALID_ARG, "set_params: bad arguments");
    DeviceGuard dg(u->device);
    cudaError_t e = cudaMemcpy(u->params, host_params, N_PARAMS * sizeof(float), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(u->m, 0, 2 * N_PARAMS * sizeof(float));
    if (e == cudaSuccess) e = refresh_bf16(u, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(u, e, "set_params");
    u->steps = 0;
    return GS_OK;
}

gs_status gs_upsampler_get_params(gs_upsampler *u, float *host_params, int64_t n) {
    if (!u || !host_params || n != N_PARAMS) return fail(u, GS_ERR_INVALID_ARG, "get_params: bad arguments");
    DeviceGuard dg(u->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpy(host_params, u->params, N_PARAMS * sizeof(float), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? GS_OK : cuda_fail(u, e, "get_params");
}

gs_status gs_upsampler_get_grads(gs_upsampler *u, float *host_grads, int64_t n) {
    if (!u || !host_grads || n != N_PARAMS) return fail(u, GS_ERR_INVALID_ARG, "get_grads: bad arguments");
    DeviceGuard dg(u->device);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess)
        e = cudaMemcpy(host_grads, u->grads, N_PARAMS * sizeof(float), cudaMemcpyDeviceToHost);
    return e == cudaSuccess ? GS_OK : cuda_fail(u, e, "get_grads");
}

gs_status gs_upsample_forward(gs_upsampler *u, int32_t n, int32_t h, int32_t w,
                              const float *lr_rgb, const float *lr_depth, float *hr_rgb,
                              float *hr_depth, void *stream) {
    if (!u) return GS_ERR_INVALID_ARG;
    if (n < 0 || h <= 0 || w <= 0 || h > 65535 || w > 65535)
        return fail(u, GS_ERR_INVALID_ARG, "upsample_forward: bad sizes");
    if (n == 0) return GS_OK;
    if (!lr_rgb || !hr_rgb || (lr_depth == nullptr) != (hr_depth == nullptr))
        return fail(u, GS_ERR_INVALID_ARG, "upsample_forward: null pointer");
    DeviceGuard dg(u->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t px = (size_t)h * w;
    const size_t per_frame = align256(px * 16 * 2) + 2 * align256(px * 32 * 2);
    const int group = (int)std::max<size_t>(1, std::min<size_t>(n, INFER_BYTES / per_frame));
    cudaError_t e = grow(u->work, per_frame * group);
    if (e != cudaSuccess) return cuda_fail(u, e, "upsample_forward: workspace");
    char *base = (char *)u->work.p;
    bf16 *x0 = (bf16 *)base;
    bf16 *a = (bf16 *)(base + align256(px * 16 * 2) * group);
    bf16 *b = (bf16 *)((char *)a + align256(px * 32 * 2) * group);
    const bool tc = u->backend == GS_UPSAMPLE_TCGEN05;
    for (int f0 = 0; f0 < n; f0 += group) {
        const int m = std::min(group, n - f0);
        const float *rgb = lr_rgb + (size_t)f0 * px * 3;
        float *hr = hr_rgb + (size_t)f0 * px * 48;
        // tensor cores: planar activations (one stored input plane); mma.sync: NHWC
        e = tc ? gsk::up_prep_input_plane(rgb, m, h, w, x0, s) : gsk::up_prep_input(rgb, m, h, w, x0, s);
        const bf16 *in = x0;
        for (int l = 0; l < NL && e == cudaSuccess; ++l) {
            const float *bias = u->params + layer_off(l) + (long long)L_CO[l] * L_CI[l] * 9;
            bf16 *dst = (in == a) ? b : a;
            const float *ldep = lr_depth ? lr_depth + (size_t)f0 * px : nullptr;
            float *hdep = hr_depth ? hr_depth + (size_t)f0 * px * 16 : nullptr;
            if (tc)
                e = gsk::up_conv_tc_planar(l, in, m, h, w, u->wt[l], bias,
                                           l < NL - 1 ? (void *)dst : (void *)hr, rgb, ldep, hdep,
                                           u->status, u->n_sm, s);
            else if (l < NL - 1)
                e = gsk::up_conv_forward(l, in, m, h, w, u->wf[l], bias, dst, s);
            else
                e = gsk::up_conv_upsample(in, m, h, w, u->wf[l], bias, rgb, hr, s);
            in = dst;
        }
        // the tensor-core path writes the depth in its last layer
        if (e == cudaSuccess && lr_depth && !tc)
            e = gsk::up_bilinear1(lr_depth + (size_t)f0 * px, m, h, w, hr_depth + (size_t)f0 * px * 16, s);
        if (e != cudaSuccess) return cuda_fail(u, e, "upsample_forward");
    }
    return GS_OK;
}

gs_status gs_upsampler_set_backend(gs_upsampler *u, int32_t backend) {
    if (!u || (backend != GS_UPSAMPLE_TCGEN05 && backend != GS_UPSAMPLE_MMA_SYNC))
        return fail(u, GS_ERR_INVALID_ARG, "set_backend: unknown backend");
    u->backend = backend;
    return GS_OK;
}

gs_status gs_upsample_timeout_probe(gs_upsampler *u, void *stream) {
    if (!u) return GS_ERR_INVALID_ARG;
    DeviceGuard dg(u->device);
    cudaStream_t s = (cudaStream_t)stream;
    const int n = 4, h = 28, w = 32;  // 16 tiles: several blocks
    const size_t px = (size_t)n * h * w;
    const size_t act = align256(px * 32 * sizeof(bf16)), lr = align256(px * 4 * sizeof(float));
    const size_t hr = align256(px * 16 * 4 * sizeof(float));
    cudaError_t e = grow(u->work, 2 * act + lr + hr);
    if (e != cudaSuccess) return cuda_fail(u, e, "timeout_probe: workspace");
    char *base = (char *)u->work.p;
    bf16 *x = (bf16 *)base, *y = (bf16 *)(base + act);
    float *rgb = (float *)(base + 2 * act), *dep = rgb + px * 3;
    float *hrgb = (float *)(base + 2 * act + lr), *hdep = hrgb + px * 16 * 3;
    e = cudaMemsetAsync(base, 0, 2 * act + lr, s);
    if (e == cudaSuccess)  // a hidden layer
        e = gsk::up_conv_tc_timeout_probe(x, n, h, w, u->wt[1], u->params + layer_off(1) + 32 * 32 * 9,
                                          y, u->status, u->n_sm, 1 << 12, s);
    if (e == cudaSuccess)  // the last layer
        e = gsk::up_conv_tc_timeout_probe_up(x, n, h, w, u->wt[5],
                                             u->params + layer_off(5) + (long long)48 * 32 * 9, rgb, dep,
                                             hrgb, hdep, u->status, u->n_sm, 1 << 12, s);
    return e == cudaSuccess ? GS_OK : cuda_fail(u, e, "timeout_probe");
}

gs_status gs_upsample_check(gs_upsampler *u, void *stream) {
    if (!u) return GS_ERR_INVALID_ARG;
    DeviceGuard dg(u->device);
    cudaStream_t s = (cudaStream_t)stream;
    int st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, u->status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(u, e, "upsample_check");
    if (st) {
        cudaMemsetAsync(u->status, 0, sizeof(int), s);
        cudaStreamSynchronize(s);
        return fail(u, GS_ERR_TIMEOUT, "a tensor-core convolution timed out waiting for its MMAs");
    }
    return GS_OK;
}

gs_status gs_upsample_grad(gs_upsampler *u, int32_t n, int32_t h, int32_t w, const float *lr_rgb,
                           const float *hr_target, float *loss, void *stream) {
    if (!u) return GS_ERR_INVALID_ARG;
    if (n <= 0 || h <= 0 || w <= 0 || h > 65535 || w > 65535)
        return fail(u, GS_ERR_INVALID_ARG, "upsample_grad: bad sizes");
    if (!lr_rgb || !hr_target) return fail(u, GS_ERR_INVALID_ARG, "upsample_grad: null pointer");
    DeviceGuard dg(u->device);
    cudaStream_t s = (cudaStream_t)stream;
    const size_t px = (size_t)n * h * w;
    const size_t s16 = align256(px * 16 * 2), s32 = align256(px * 32 * 2),
                 s48 = align256(px * 48 * 2), sz = align256(px * 48 * 4);
    const size_t bytes = s16 + 5 * s32 + sz + s48 + 2 * s32 + 256;
    cudaError_t e = grow(u->work, bytes);
    if (e != cudaSuccess) return cuda_fail(u, e, "upsample_grad: workspace");
    char *p = (char *)u->work.p;
    bf16 *act[6];
    act[0] = (bf16 *)p;
    p += s16;
    for (int l = 1; l < 6; ++l, p += s32) act[l] = (bf16 *)p;
    float *z = (float *)p;
    p += sz;
    bf16 *dz6 = (bf16 *)p;
    p += s48;
    bf16 *dzA = (bf16 *)p, *dzB = (bf16 *)(p + s32);
    p += 2 * s32;
    float *lacc = loss ? loss : (float *)p;
    e = cudaMemsetAsync(u->grads, 0, N_PARAMS * sizeof(float), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(lacc, 0, sizeof(float), s);
    if (e == cudaSuccess) e = gsk::up_prep_input(lr_rgb, n, h, w, act[0], s);
    const bool tc = u->backend == GS_UPSAMPLE_TCGEN05;
    for (int l = 0; l < 6 && e == cudaSuccess; ++l) {
        const float *bias = u->params + layer_off(l) + (long long)L_CO[l] * L_CI[l] * 9;
        if (tc && l < 5)
            e = gsk::up_conv_tc(l, act[l], n, h, w, u->wt[l], bias, act[l + 1], nullptr, nullptr,
                                nullptr, u->status, u->n_sm, s);
        else if (tc)
            e = gsk::up_conv_tc_linear(act[l], n, h, w, u->wt[l], bias, z, u->status, u->n_sm, s);
        else
            e = gsk::up_conv_forward(l, act[l], n, h, w, u->wf[l], bias,
                                     l < 5 ? (void *)act[l + 1] : (void *)z, s);
    }
    if (e == cudaSuccess) e = gsk::up_loss(z, lr_rgb, hr_target, n, h, w, dz6, lacc, s);
    const bf16 *dz = dz6;
    for (int l = 5; l >= 0 && e == cudaSuccess; --l) {
        float *gW = u->grads + layer_off(l);
        float *gb = gW + (long long)L_CO[l] * L_CI[l] * 9;
        e = tc ? gsk::up_wgrad_tc(l, act[l], dz, n, h, w, gW, gb, u->status, u->n_sm, s)
               : gsk::up_wgrad(l, act[l], dz, n, h, w, gW, gb, u->n_sm, s);
        if (e == cudaSuccess && l > 0) {
            bf16 *dst = (dz == dzA) ? dzB : dzA;
            e = tc ? gsk::up_dgrad_tc(l, dz, n, h, w, u->wdt[l], act[l], dst, u->status, u->n_sm, s)
                   : gsk::up_conv_dgrad(l, dz, n, h, w, u->wd[l], act[l], dst, s);
            dz = dst;
        }
    }
    return e == cudaSuccess ? GS_OK : cuda_fail(u, e, "upsample_grad");
}

gs_status gs_upsample_adam(gs_upsampler *u, float lr, float beta1, float beta2, float eps,
                           void *stream) {
    if (!u) return GS_ERR_INVALID_ARG;
    if (!(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) ||
        !(eps > 0.0f))
        return fail(u, GS_ERR_INVALID_ARG, "upsample_adam: bad hyper-parameters");
    DeviceGuard dg(u->device);
    cudaStream_t s = (cudaStream_t)stream;
    u->steps += 1;
    const float c1 = (float)(1.0 - std::pow((double)beta1, (double)u->steps));
    const float c2 = (float)(1.0 - std::pow((double)beta2, (double)u->steps));
    for (int l = 0; l < NL; ++l) {
        const long long o = layer_off(l);
        cudaError_t e = gsk::up_adam(u->params + o, u->m + o, u->v + o, u->grads + o, L_CO[l], L_CI[l],
                                     L_CIP[l], lr, beta1, beta2, eps, c1, c2, u->wf[l],
                                     l > 0 ? u->wd[l] : nullptr, u->wt[l],
                                     l > 0 ? u->wdt[l] : nullptr, s);
        if (e != cudaSuccess) return cuda_fail(u, e, "upsample_adam");
    }
    return GS_OK;
}

}  // extern "C"
