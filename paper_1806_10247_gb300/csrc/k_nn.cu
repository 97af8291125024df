// Kernels of the learned warm start: a small 3D convolutional network trained
// and evaluated on the GPU (forward, backward, loss, Adam).  Activations are
// FP32 in [batch][channel][D][H][W] layout; weights are read either as FP32 or
// as BF16 (the trained network's storage form), always accumulated in FP32.
// The paper has no counterpart: this supports the warm start of the LB
// iteration, which alone decides the converged field.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>

#include "../../include/lbm.h"

namespace {

constexpr int kT = 256;
thread_local std::string g_nn_error;

int nn_fail(int code, const char *fmt, ...)
{
    char buf[256];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_nn_error = buf;
    return code;
}

struct Shape {
    int n, ci, co, d, h, w;  // batch, channels in/out, spatial extents
    int kd, kh, kw;          // kernel extents (odd)
    int dd, dh, dw;          // dilations
    __host__ __device__ long long in_count() const { return (long long)n * ci * d * h * w; }
    __host__ __device__ long long out_count() const { return (long long)n * co * d * h * w; }
};

__device__ __forceinline__ float wload(const void *w, int bf16, long long i)
{
    if (bf16) return __bfloat162float(reinterpret_cast<const __nv_bfloat16 *>(w)[i]);
    return reinterpret_cast<const float *>(w)[i];
}

// y[n,o,p] = b[o] + sum_{i,tap} w[o,i,tap] x[n,i,p + shift(tap)], zero padding.
__global__ void __launch_bounds__(kT)
k_conv_fwd(const float *__restrict__ x, const void *__restrict__ w, int bf16, const float *__restrict__ b,
           float *__restrict__ y, Shape s, int act)
{
    const long long idx = (long long)blockIdx.x * kT + threadIdx.x;
    if (idx >= s.out_count()) return;
    const int v = idx % s.w;
    long long r = idx / s.w;
    const int hh = r % s.h;
    r /= s.h;
    const int dd = r % s.d;
    r /= s.d;
    const int o = r % s.co;
    const int n = (int)(r / s.co);
    float acc = b[o];
    const int taps = s.kd * s.kh * s.kw;
    for (int i = 0; i < s.ci; i++) {
        const float *xi = x + ((long long)n * s.ci + i) * s.d * s.h * s.w;
        const long long wbase = ((long long)o * s.ci + i) * taps;
        for (int a = 0; a < s.kd; a++) {
            const int zd = dd + s.dd * (a - (s.kd - 1) / 2);
            if (zd < 0 || zd >= s.d) continue;
            for (int c = 0; c < s.kh; c++) {
                const int zh = hh + s.dh * (c - (s.kh - 1) / 2);
                if (zh < 0 || zh >= s.h) continue;
                for (int e = 0; e < s.kw; e++) {
                    const int zw = v + s.dw * (e - (s.kw - 1) / 2);
                    if (zw < 0 || zw >= s.w) continue;
                    acc = fmaf(wload(w, bf16, wbase + (a * s.kh + c) * s.kw + e), xi[((long long)zd * s.h + zh) * s.w + zw],
                               acc);
                }
            }
        }
    }
    y[idx] = act == 1 ? tanhf(acc) : acc;
}

// gx[n,i,p] = sum_{o,tap} w[o,i,tap] gy[n,o,p - shift(tap)]  (transposed convolution).
__global__ void __launch_bounds__(kT)
k_conv_bwd_in(const float *__restrict__ gy, const void *__restrict__ w, int bf16, float *__restrict__ gx, Shape s)
{
    const long long idx = (long long)blockIdx.x * kT + threadIdx.x;
    if (idx >= s.in_count()) return;
    const int v = idx % s.w;
    long long r = idx / s.w;
    const int hh = r % s.h;
    r /= s.h;
    const int dd = r % s.d;
    r /= s.d;
    const int i = r % s.ci;
    const int n = (int)(r / s.ci);
    const int taps = s.kd * s.kh * s.kw;
    float acc = 0.0f;
    for (int o = 0; o < s.co; o++) {
        const float *go = gy + ((long long)n * s.co + o) * s.d * s.h * s.w;
        const long long wbase = ((long long)o * s.ci + i) * taps;
        for (int a = 0; a < s.kd; a++) {
            const int zd = dd - s.dd * (a - (s.kd - 1) / 2);
            if (zd < 0 || zd >= s.d) continue;
            for (int c = 0; c < s.kh; c++) {
                const int zh = hh - s.dh * (c - (s.kh - 1) / 2);
                if (zh < 0 || zh >= s.h) continue;
                for (int e = 0; e < s.kw; e++) {
                    const int zw = v - s.dw * (e - (s.kw - 1) / 2);
                    if (zw < 0 || zw >= s.w) continue;
                    acc = fmaf(wload(w, bf16, wbase + (a * s.kh + c) * s.kw + e), go[((long long)zd * s.h + zh) * s.w + zw],
                               acc);
                }
            }
        }
    }
    gx[idx] = acc;
}

__device__ __forceinline__ float block_sum(float v)
{
    __shared__ float sh[kT / 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    v = threadIdx.x < kT / 32 ? sh[threadIdx.x] : 0.0f;
    if (warp == 0)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;  // valid in thread 0
}

// One block per weight (o, i, tap) and, after those, one per bias o:
// gw = sum_{n,p} gy[n,o,p] x[n,i,p + shift(tap)],  gb = sum_{n,p} gy[n,o,p].
// Fixed summation order: deterministic.
__global__ void __launch_bounds__(kT)
k_conv_bwd_w(const float *__restrict__ x, const float *__restrict__ gy, float *__restrict__ gw, float *__restrict__ gb,
             Shape s)
{
    const int taps = s.kd * s.kh * s.kw;
    const long long nweights = (long long)s.co * s.ci * taps;
    const long long bid = blockIdx.x;
    const long long sp = (long long)s.d * s.h * s.w;
    float acc = 0.0f;
    if (bid < nweights) {
        const int tap = bid % taps;
        const int i = (bid / taps) % s.ci;
        const int o = (int)(bid / ((long long)taps * s.ci));
        const int e = tap % s.kw, c = (tap / s.kw) % s.kh, a = tap / (s.kw * s.kh);
        const int sd = s.dd * (a - (s.kd - 1) / 2), sh = s.dh * (c - (s.kh - 1) / 2), sw = s.dw * (e - (s.kw - 1) / 2);
        for (long long q = threadIdx.x; q < (long long)s.n * sp; q += kT) {
            const int n = (int)(q / sp);
            const long long p = q % sp;
            const int v = p % s.w, hh = (p / s.w) % s.h, dd = (int)(p / ((long long)s.w * s.h));
            const int zd = dd + sd, zh = hh + sh, zw = v + sw;
            if (zd < 0 || zd >= s.d || zh < 0 || zh >= s.h || zw < 0 || zw >= s.w) continue;
            acc = fmaf(gy[((long long)n * s.co + o) * sp + p],
                       x[((long long)n * s.ci + i) * sp + ((long long)zd * s.h + zh) * s.w + zw], acc);
        }
        acc = block_sum(acc);
        if (threadIdx.x == 0) gw[bid] = acc;
    } else {
        const int o = (int)(bid - nweights);
        for (long long q = threadIdx.x; q < (long long)s.n * sp; q += kT) {
            const int n = (int)(q / sp);
            acc += gy[((long long)n * s.co + o) * sp + q % sp];
        }
        acc = block_sum(acc);
        if (threadIdx.x == 0) gb[o] = acc;
    }
}

__global__ void __launch_bounds__(kT) k_tanh_bwd(float *__restrict__ g, const float *__restrict__ y, long long count)
{
    const long long i = (long long)blockIdx.x * kT + threadIdx.x;
    if (i < count) g[i] *= 1.0f - y[i] * y[i];
}

// g = 2 (y - t) / count and loss = mean((y - t)^2), one block (fixed order).
__global__ void __launch_bounds__(1024)
k_mse(const float *__restrict__ y, const float *__restrict__ t, float *__restrict__ g, long long count,
      double *__restrict__ loss)
{
    __shared__ double sh[32];
    double acc = 0.0;
    const float scale = 2.0f / (float)count;
    for (long long i = threadIdx.x; i < count; i += 1024) {
        const float d = y[i] - t[i];
        g[i] = scale * d;
        acc += (double)d * (double)d;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        acc = sh[threadIdx.x];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
        if (threadIdx.x == 0) *loss = acc / (double)count;
    }
}

// Adam (bias-corrected) on FP32 master weights; also refreshes the BF16 copy.
__global__ void __launch_bounds__(kT)
k_adam(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
       __nv_bfloat16 *__restrict__ pb, long long count, float lr, float b1, float b2, float eps, float c1, float c2)
{
    const long long i = (long long)blockIdx.x * kT + threadIdx.x;
    if (i >= count) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    p[i] = pi;
    if (pb) pb[i] = __float2bfloat16_rn(pi);
}

__global__ void __launch_bounds__(kT) k_to_bf16(const float *__restrict__ p, __nv_bfloat16 *__restrict__ pb, long long count)
{
    const long long i = (long long)blockIdx.x * kT + threadIdx.x;
    if (i < count) pb[i] = __float2bfloat16_rn(p[i]);
}

int check_shape(const int *sp, const int *k, const int *dil, int n, int ci, int co, Shape &s)
{
    if (!sp || !k || !dil) return nn_fail(LBM_EINVAL, "shape, kernel and dilation are required");
    if (n < 1 || ci < 1 || co < 1) return nn_fail(LBM_EINVAL, "batch and channel counts must be >= 1");
    for (int d = 0; d < 3; d++) {
        if (sp[d] < 1) return nn_fail(LBM_EINVAL, "spatial extents must be >= 1");
        if (k[d] < 1 || (k[d] & 1) == 0) return nn_fail(LBM_EINVAL, "kernel extents must be odd");
        if (dil[d] < 1) return nn_fail(LBM_EINVAL, "dilations must be >= 1");
    }
    s = Shape{n, ci, co, sp[0], sp[1], sp[2], k[0], k[1], k[2], dil[0], dil[1], dil[2]};
    if (s.in_count() > (1LL << 40) || s.out_count() > (1LL << 40)) return nn_fail(LBM_EINVAL, "tensor too large");
    return LBM_OK;
}

int launched(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return nn_fail(LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return LBM_OK;
}

unsigned grid_of(long long count, int block) { return (unsigned)((count + block - 1) / block); }

}  // namespace

extern "C" {

const char *lbm_nn_last_error(void) { return g_nn_error.c_str(); }

int lbm_nn_conv3d_forward(const float *x, const void *w, int w_bf16, const float *b, float *y, int n, int ci, int co,
                          const int dhw[3], const int k[3], const int dil[3], int act, void *stream)
{
    Shape s;
    int rc = check_shape(dhw, k, dil, n, ci, co, s);
    if (rc != LBM_OK) return rc;
    if (!x || !w || !b || !y) return nn_fail(LBM_EINVAL, "conv3d_forward: NULL pointer");
    if (act != 0 && act != 1) return nn_fail(LBM_EINVAL, "conv3d_forward: act must be 0 or 1");
    k_conv_fwd<<<grid_of(s.out_count(), kT), kT, 0, (cudaStream_t)stream>>>(x, w, w_bf16, b, y, s, act);
    return launched("conv3d_forward");
}

int lbm_nn_conv3d_backward(const float *x, const void *w, int w_bf16, const float *gy, float *gx, float *gw, float *gb,
                           int n, int ci, int co, const int dhw[3], const int k[3], const int dil[3], void *stream)
{
    Shape s;
    int rc = check_shape(dhw, k, dil, n, ci, co, s);
    if (rc != LBM_OK) return rc;
    if (!x || !w || !gy || !gw || !gb) return nn_fail(LBM_EINVAL, "conv3d_backward: NULL pointer");
    cudaStream_t st = (cudaStream_t)stream;
    if (gx) {
        k_conv_bwd_in<<<grid_of(s.in_count(), kT), kT, 0, st>>>(gy, w, w_bf16, gx, s);
        rc = launched("conv3d_backward(input)");
        if (rc != LBM_OK) return rc;
    }
    const long long blocks = (long long)co * ci * s.kd * s.kh * s.kw + co;
    k_conv_bwd_w<<<(unsigned)blocks, kT, 0, st>>>(x, gy, gw, gb, s);
    return launched("conv3d_backward(weights)");
}

int lbm_nn_tanh_backward(float *g, const float *y, long long count, void *stream)
{
    if (!g || !y || count < 0) return nn_fail(LBM_EINVAL, "tanh_backward: bad arguments");
    if (count == 0) return LBM_OK;
    k_tanh_bwd<<<grid_of(count, kT), kT, 0, (cudaStream_t)stream>>>(g, y, count);
    return launched("tanh_backward");
}

int lbm_nn_mse(const float *y, const float *t, float *g, long long count, double *loss, void *stream)
{
    if (!y || !t || !g || !loss || count < 1) return nn_fail(LBM_EINVAL, "mse: bad arguments");
    k_mse<<<1, 1024, 0, (cudaStream_t)stream>>>(y, t, g, count, loss);
    return launched("mse");
}

int lbm_nn_adam(float *p, const float *g, float *m, float *v, void *p_bf16, long long count, double lr, double b1,
                double b2, double eps, long long step, void *stream)
{
    if (!p || !g || !m || !v || count < 0 || step < 1) return nn_fail(LBM_EINVAL, "adam: bad arguments");
    if (count == 0) return LBM_OK;
    const float c1 = (float)(1.0 - pow(b1, (double)step)), c2 = (float)(1.0 - pow(b2, (double)step));
    k_adam<<<grid_of(count, kT), kT, 0, (cudaStream_t)stream>>>(p, g, m, v, (__nv_bfloat16 *)p_bf16, count, (float)lr,
                                                                 (float)b1, (float)b2, (float)eps, c1, c2);
    return launched("adam");
}

int lbm_nn_to_bf16(const float *p, void *p_bf16, long long count, void *stream)
{
    if (!p || !p_bf16 || count < 0) return nn_fail(LBM_EINVAL, "to_bf16: bad arguments");
    if (count == 0) return LBM_OK;
    k_to_bf16<<<grid_of(count, kT), kT, 0, (cudaStream_t)stream>>>(p, (__nv_bfloat16 *)p_bf16, count);
    return launched("to_bf16");
}

}  // extern "C"
