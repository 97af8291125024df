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
#include <mutex>
#include <string>

#include "../../include/lbm.h"
#include "k_nn_tc.cuh"

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

int launched(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return nn_fail(LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return LBM_OK;
}

unsigned grid_of(long long count, int block) { return (unsigned)((count + block - 1) / block); }

// ------------------------------------------------ tensor-core convolutions ---
// With BF16 weights (the trained network's storage form) the convolutions run
// as implicit GEMMs on the tensor cores (tcgen05, BF16 operands, FP32
// accumulation in tensor memory): activations and incoming gradients are
// rounded to BF16 as they are staged, every product is exact and the sums are
// FP32.  Tiles: kM = 128 pixels (or weight rows) by up to kMaxKp padded K
// values and kMaxNp padded output channels; one thread stages one row.

// Bit 0 set when a tensor-core wait ran out (read and cleared by lbm_nn_tc_status).
__device__ int g_tc_status;

int round16(int v) { return (v + 15) / 16 * 16; }

enum TcMode { TC_FWD = 0, TC_BWD_IN = 1 };

// TC_FWD:    y[n,o,p] = act(b[o] + sum_{i,tap} w[o,i,tap] x[n,i,p + shift(tap)])
//            rows: pixels of y; K = (i, tap); N = o.
// TC_BWD_IN: gx[n,i,p] = sum_{o,tap} w[o,i,tap] gy[n,o,p - shift(tap)]
//            rows: pixels of x; K = (o, tap); N = i.
template <int MODE>
__global__ void __launch_bounds__(nntc::kM)
k_tc_conv(const float *__restrict__ in, const __nv_bfloat16 *__restrict__ w, const float *__restrict__ b,
          float *__restrict__ out, Shape s, int act, int Kp, int Np)
{
    using namespace nntc;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t tmem_base;
    unsigned char *As = smem;
    unsigned char *Bs = smem + kM * Kp * 2;
    const int tid = threadIdx.x;
    const int taps = s.kd * s.kh * s.kw;
    const int cin = MODE == TC_FWD ? s.ci : s.co;    // channels of the gathered operand
    const int cout = MODE == TC_FWD ? s.co : s.ci;   // channels of the result
    const int K = cin * taps;
    const int sgn = MODE == TC_FWD ? 1 : -1;
    const long long sp = (long long)s.d * s.h * s.w, npix = (long long)s.n * sp;
    const long long m = (long long)blockIdx.x * kM + tid;
    const uint32_t ncols = tmem_cols(Np);
    if (tid < 32) tmem_alloc(smem_u32(&tmem_base), ncols);
    if (tid == 0) mbar_init(smem_u32(&mbar));
    const bool valid = m < npix;
    int n_ = 0, pd = 0, ph = 0, pw = 0;
    long long p = 0;
    if (valid) {
        n_ = (int)(m / sp);
        p = m % sp;
        pw = (int)(p % s.w);
        ph = (int)((p / s.w) % s.h);
        pd = (int)(p / ((long long)s.w * s.h));
    }
    for (int k = 0; k < Kp; k++) {
        float v = 0.f;
        if (valid && k < K) {
            const int c = k / taps, tap = k - c * taps;
            const int e = tap % s.kw, f = (tap / s.kw) % s.kh, a = tap / (s.kw * s.kh);
            const int zd = pd + sgn * s.dd * (a - (s.kd - 1) / 2);
            const int zh = ph + sgn * s.dh * (f - (s.kh - 1) / 2);
            const int zw = pw + sgn * s.dw * (e - (s.kw - 1) / 2);
            if (zd >= 0 && zd < s.d && zh >= 0 && zh < s.h && zw >= 0 && zw < s.w)
                v = in[((long long)n_ * cin + c) * sp + ((long long)zd * s.h + zh) * s.w + zw];
        }
        *reinterpret_cast<__nv_bfloat16 *>(As + core_off(tid, k, kM)) = __float2bfloat16_rn(v);
    }
    for (int idx = tid; idx < Np * Kp; idx += kM) {
        const int r = idx / Kp, k = idx - r * Kp;  // r: output channel, k: (input channel, tap)
        __nv_bfloat16 v = __float2bfloat16_rn(0.f);
        if (r < cout && k < K) {
            const int c = k / taps, tap = k - c * taps;
            v = MODE == TC_FWD ? w[((long long)r * s.ci + c) * taps + tap] : w[((long long)c * s.ci + r) * taps + tap];
        }
        *reinterpret_cast<__nv_bfloat16 *>(Bs + core_off(r, k, Np)) = v;
    }
    fence_smem_to_async();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_base;
    if (tid == 0) {
        issue_tile(tmem, smem_u32(As), smem_u32(Bs), Kp, Np, false);
        mma_commit(smem_u32(&mbar));
    }
    const bool ok = __syncthreads_and(mbar_wait_bounded(smem_u32(&mbar), 0));
    fence_after_sync();
    if (ok) {
        for (int c0 = 0; c0 < Np; c0 += 16) {
            float v[16];
            tmem_load16(tmem + ((uint32_t)(32 * (tid >> 5)) << 16) + (uint32_t)c0, v);
            if (valid) {
#pragma unroll
                for (int j = 0; j < 16; j++) {
                    const int o = c0 + j;
                    if (o < cout) {
                        float r = v[j];
                        if (MODE == TC_FWD) {
                            r += b[o];
                            if (act == 1) r = tanhf(r);
                        }
                        out[((long long)n_ * cout + o) * sp + p] = r;
                    }
                }
            }
        }
    } else {
        if (tid == 0) atomicOr(&g_tc_status, 1);
        mbar_wait_bounded(smem_u32(&mbar), 0);  // the MMAs end before their accumulators are freed
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (tid < 32) tmem_dealloc(tmem, ncols);
}

// Weight gradient, partial sums: block (g, t) accumulates, over the 128-pixel
// chunks c = g, g + G, ..., the rows r = 128 t .. 128 t + 127 of
// part[g][r][o] = sum_p x[n,i,p + shift(tap)] gy[n,o,p], r = i * taps + tap
// (rows: weight entries; K: pixels; N: o).  k_tc_reduce_w adds the G partial
// sums in a fixed order.
__global__ void __launch_bounds__(nntc::kM)
k_tc_conv_bwd_w(const float *__restrict__ x, const float *__restrict__ gy, float *__restrict__ part, Shape s, int G,
                int Mp, int Np)
{
    using namespace nntc;
    extern __shared__ __align__(1024) unsigned char smem[];
    __shared__ __align__(8) unsigned long long mbar;
    __shared__ uint32_t tmem_base;
    unsigned char *As = smem;
    unsigned char *Bs = smem + kM * kM * 2;
    const int tid = threadIdx.x;
    const int taps = s.kd * s.kh * s.kw, Kw = s.ci * taps;
    const long long sp = (long long)s.d * s.h * s.w, npix = (long long)s.n * sp;
    const long long nchunks = (npix + kM - 1) / kM;
    const int g = blockIdx.x, row0 = blockIdx.y * kM;
    const uint32_t ncols = tmem_cols(Np);
    if (tid < 32) tmem_alloc(smem_u32(&tmem_base), ncols);
    if (tid == 0) mbar_init(smem_u32(&mbar));
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = tmem_base;
    bool ok = true;
    int round = 0;
    for (long long c = g; c < nchunks && ok; c += G, round++) {
        // this thread stages pixel j = tid of the chunk: column j of A and of B
        const long long q = c * kM + tid;
        const bool valid = q < npix;
        int n_ = 0, pd = 0, ph = 0, pw = 0;
        long long p = 0;
        if (valid) {
            n_ = (int)(q / sp);
            p = q % sp;
            pw = (int)(p % s.w);
            ph = (int)((p / s.w) % s.h);
            pd = (int)(p / ((long long)s.w * s.h));
        }
        for (int rr = 0; rr < kM; rr++) {
            const int r = row0 + rr;
            float v = 0.f;
            if (valid && r < Kw) {
                const int i = r / taps, tap = r - i * taps;
                const int e = tap % s.kw, f = (tap / s.kw) % s.kh, a = tap / (s.kw * s.kh);
                const int zd = pd + s.dd * (a - (s.kd - 1) / 2);
                const int zh = ph + s.dh * (f - (s.kh - 1) / 2);
                const int zw = pw + s.dw * (e - (s.kw - 1) / 2);
                if (zd >= 0 && zd < s.d && zh >= 0 && zh < s.h && zw >= 0 && zw < s.w)
                    v = x[((long long)n_ * s.ci + i) * sp + ((long long)zd * s.h + zh) * s.w + zw];
            }
            *reinterpret_cast<__nv_bfloat16 *>(As + core_off(rr, tid, kM)) = __float2bfloat16_rn(v);
        }
        for (int o = 0; o < Np; o++) {
            const float v = (valid && o < s.co) ? gy[((long long)n_ * s.co + o) * sp + p] : 0.f;
            *reinterpret_cast<__nv_bfloat16 *>(Bs + core_off(o, tid, Np)) = __float2bfloat16_rn(v);
        }
        fence_smem_to_async();
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
        if (tid == 0) {
            issue_tile(tmem, smem_u32(As), smem_u32(Bs), kM, Np, round > 0);
            mma_commit(smem_u32(&mbar));
        }
        // the next chunk overwrites the operands: wait for this chunk's MMAs
        ok = __syncthreads_and(mbar_wait_bounded(smem_u32(&mbar), (uint32_t)(round & 1)));
        fence_after_sync();
    }
    if (ok) {
        const int r = row0 + tid;
        for (int c0 = 0; c0 < Np; c0 += 16) {
            float v[16];
            tmem_load16(tmem + ((uint32_t)(32 * (tid >> 5)) << 16) + (uint32_t)c0, v);
#pragma unroll
            for (int j = 0; j < 16; j++) part[((long long)g * Mp + r) * Np + c0 + j] = round > 0 ? v[j] : 0.f;
        }
    } else {
        if (tid == 0) atomicOr(&g_tc_status, 1);
        mbar_wait_bounded(smem_u32(&mbar), (uint32_t)((round - 1) & 1));
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (tid < 32) tmem_dealloc(tmem, ncols);
}

// gw[o][i][tap] = sum_{g = 0..G-1} part[g][i * taps + tap][o], in order of g.
__global__ void __launch_bounds__(kT)
k_tc_reduce_w(const float *__restrict__ part, float *__restrict__ gw, int co, int Kw, int G, int Mp, int Np)
{
    const int idx = blockIdx.x * kT + threadIdx.x;
    if (idx >= co * Kw) return;
    const int o = idx / Kw, r = idx - o * Kw;
    float acc = 0.f;
    for (int g = 0; g < G; g++) acc += part[((long long)g * Mp + r) * Np + o];
    gw[idx] = acc;
}

// gb[o] = sum_{n,p} gy[n,o,p] (one block per channel, fixed order).
__global__ void __launch_bounds__(kT) k_bias_grad(const float *__restrict__ gy, float *__restrict__ gb, Shape s)
{
    const long long sp = (long long)s.d * s.h * s.w;
    const int o = blockIdx.x;
    float acc = 0.0f;
    for (long long q = threadIdx.x; q < (long long)s.n * sp; q += kT) {
        const int n = (int)(q / sp);
        acc += gy[((long long)n * s.co + o) * sp + q % sp];
    }
    acc = block_sum(acc);
    if (threadIdx.x == 0) gb[o] = acc;
}

// Partial-sum workspace of the weight gradient, one per device, grown on
// demand (cudaMalloc only when a larger one is needed).
std::mutex g_ws_mu;
float *g_ws[64] = {};
size_t g_ws_cap[64] = {};

float *tc_workspace(size_t floats)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(g_ws_mu);
    if (g_ws_cap[dev] < floats) {
        if (g_ws[dev]) cudaFree(g_ws[dev]);
        g_ws[dev] = nullptr;
        g_ws_cap[dev] = 0;
        if (cudaMalloc(&g_ws[dev], floats * sizeof(float)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        g_ws_cap[dev] = floats;
    }
    return g_ws[dev];
}

bool tc_fits(int kdim, int ndim) { return round16(kdim) <= nntc::kMaxKp && round16(ndim) <= nntc::kMaxNp; }

template <int MODE>
int tc_conv_launch(const float *in, const void *w, const float *b, float *out, const Shape &s, int act,
                   cudaStream_t st, const char *what)
{
    const int taps = s.kd * s.kh * s.kw;
    const int K = (MODE == TC_FWD ? s.ci : s.co) * taps, Np = round16(MODE == TC_FWD ? s.co : s.ci);
    const int Kp = round16(K);
    const size_t smem = (size_t)(nntc::kM + Np) * Kp * 2 + nntc::kSlack;
    cudaError_t e = cudaFuncSetAttribute(k_tc_conv<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return nn_fail(LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    const long long npix = (long long)s.n * s.d * s.h * s.w;
    k_tc_conv<MODE><<<(unsigned)((npix + nntc::kM - 1) / nntc::kM), nntc::kM, smem, st>>>(
        in, reinterpret_cast<const __nv_bfloat16 *>(w), b, out, s, act, Kp, Np);
    return launched(what);
}

int tc_conv_bwd_w_launch(const float *x, const float *gy, float *gw, const Shape &s, cudaStream_t st)
{
    const int taps = s.kd * s.kh * s.kw, Kw = s.ci * taps;
    const int Mp = (Kw + nntc::kM - 1) / nntc::kM * nntc::kM, Np = round16(s.co);
    const long long npix = (long long)s.n * s.d * s.h * s.w;
    const long long nchunks = (npix + nntc::kM - 1) / nntc::kM;
    const int G = (int)(nchunks < 128 ? nchunks : 128);
    float *part = tc_workspace((size_t)G * Mp * Np);
    if (!part) return nn_fail(LBM_ENOMEM, "conv3d_backward: tensor-core workspace");
    const size_t smem = (size_t)(nntc::kM + Np) * nntc::kM * 2 + nntc::kSlack;
    cudaError_t e = cudaFuncSetAttribute(k_tc_conv_bwd_w, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return nn_fail(LBM_ECUDA, "conv3d_backward(weights): %s", cudaGetErrorString(e));
    k_tc_conv_bwd_w<<<dim3((unsigned)G, (unsigned)(Mp / nntc::kM)), nntc::kM, smem, st>>>(x, gy, part, s, G, Mp, Np);
    int rc = launched("conv3d_backward(weights)");
    if (rc != LBM_OK) return rc;
    k_tc_reduce_w<<<grid_of((long long)s.co * Kw, kT), kT, 0, st>>>(part, gw, s.co, Kw, G, Mp, Np);
    return launched("conv3d_backward(weight reduction)");
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

}  // namespace

extern "C" {

const char *lbm_nn_last_error(void) { return g_nn_error.c_str(); }

int lbm_nn_tc_status(int *status)
{
    if (!status) return nn_fail(LBM_EINVAL, "tc_status: status is NULL");
    int v = 0, zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(&v, g_tc_status, sizeof v);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tc_status, &zero, sizeof zero);
    if (e != cudaSuccess) return nn_fail(LBM_ECUDA, "tc_status: %s", cudaGetErrorString(e));
    *status = v;
    return LBM_OK;
}

int lbm_nn_conv3d_forward(const float *x, const void *w, int w_bf16, const float *b, float *y, int n, int ci, int co,
                          const int dhw[3], const int k[3], const int dil[3], int act, void *stream)
{
    Shape s;
    int rc = check_shape(dhw, k, dil, n, ci, co, s);
    if (rc != LBM_OK) return rc;
    if (!x || !w || !b || !y) return nn_fail(LBM_EINVAL, "conv3d_forward: NULL pointer");
    if (act != 0 && act != 1) return nn_fail(LBM_EINVAL, "conv3d_forward: act must be 0 or 1");
    if (w_bf16 && tc_fits(ci * s.kd * s.kh * s.kw, co))
        return tc_conv_launch<TC_FWD>(x, w, b, y, s, act, (cudaStream_t)stream, "conv3d_forward");
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
    const int taps = s.kd * s.kh * s.kw;
    if (gx) {
        if (w_bf16 && tc_fits(co * taps, ci)) {
            rc = tc_conv_launch<TC_BWD_IN>(gy, w, nullptr, gx, s, 0, st, "conv3d_backward(input)");
        } else {
            k_conv_bwd_in<<<grid_of(s.in_count(), kT), kT, 0, st>>>(gy, w, w_bf16, gx, s);
            rc = launched("conv3d_backward(input)");
        }
        if (rc != LBM_OK) return rc;
    }
    if (w_bf16 && ci * taps <= nntc::kMaxKp && round16(co) <= nntc::kMaxNp) {
        rc = tc_conv_bwd_w_launch(x, gy, gw, s, st);
        if (rc != LBM_OK) return rc;
        k_bias_grad<<<(unsigned)co, kT, 0, st>>>(gy, gb, s);
        return launched("conv3d_backward(bias)");
    }
    const long long blocks = (long long)co * ci * taps + co;
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
