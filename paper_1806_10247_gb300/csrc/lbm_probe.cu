// Device facts and an FP64 throughput probe, for the roofline of the FP64
// step kernels.  The paper has no counterpart: on this GPU the FP64 step
// kernels are bound by the FP64 unit, not by memory, so their roofline needs
// the FP64 instruction rate the unit actually sustains, measured on the
// device that runs them.
//
// The probe kernel runs 8 or 16 independent dependency chains per thread of
// one FP64 operation (FMA, add or multiply).  The second and third operands
// are read from constant memory, as the step kernels read their rates and
// weights: with every operand in a register the unit issued at 1.68 per
// clock per SM on the GB300 (three 64-bit register reads per instruction),
// with constant operands at 2.0, the unit's rate.  The compiler can neither
// fold nor reorder the chains; the loop (unrolled four times) keeps its
// bookkeeping on the integer pipes, so the count of FP64 instructions issued
// is exactly blocks * threads * iters * chains.
#include <cuda_runtime.h>

#include <string>

#include "../../include/lbm.h"

namespace {

thread_local std::string g_probe_error;

int probe_fail(int code, const char *what, cudaError_t e)
{
    g_probe_error = std::string(what) + (e != cudaSuccess ? std::string(": ") + cudaGetErrorString(e) : "");
    return code;
}

// x -> x a + b stays near 1; x + b grows by 1e-9 per step; x a decays by
// 1e-9 per step: every chain stays finite and away from subnormals
__constant__ double c_a = 1.0 - 1e-9, c_b = 1e-9;

template <int OP, int kChains>
__global__ void k_fp64_rate(long long iters, double *sink)
{
    // block 0 times its own run in SM cycles and in nanoseconds: the ratio is
    // the SM clock the probe ran at (the rate itself is timed by the caller)
    long long c0 = 0, t0 = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        c0 = clock64();
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    }
    double x[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) x[k] = 1.0 + 1e-3 * (threadIdx.x + k);
#pragma unroll 4
    for (long long it = 0; it < iters; it++) {
#pragma unroll
        for (int k = 0; k < kChains; k++) {
            if (OP == 0) x[k] = fma(x[k], c_a, c_b);
            else if (OP == 1) x[k] = x[k] + c_b;
            else x[k] = x[k] * c_a;
        }
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += x[k];
    // Never true for these operands; keeps the chains live.
    if (s == -1.0) sink[2] = s;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        long long t1;
        asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
        sink[0] = (double)(clock64() - c0);
        sink[1] = (double)(t1 - t0);
    }
}

template <int CH>
void launch_rate(int op, int blocks, int threads, long long iters, double *sink, cudaStream_t s)
{
    if (op == 0) k_fp64_rate<0, CH><<<blocks, threads, 0, s>>>(iters, sink);
    else if (op == 1) k_fp64_rate<1, CH><<<blocks, threads, 0, s>>>(iters, sink);
    else k_fp64_rate<2, CH><<<blocks, threads, 0, s>>>(iters, sink);
}

}  // namespace

extern "C" {

const char *lbm_probe_last_error(void) { return g_probe_error.c_str(); }

int lbm_device_info(int device, long long info[8])
{
    if (!info) return probe_fail(LBM_EINVAL, "lbm_device_info: info is NULL", cudaSuccess);
    const cudaDeviceAttr attrs[8] = {cudaDevAttrMultiProcessorCount, cudaDevAttrClockRate,
                                     cudaDevAttrMemoryClockRate,      cudaDevAttrGlobalMemoryBusWidth,
                                     cudaDevAttrL2CacheSize,          cudaDevAttrComputeCapabilityMajor,
                                     cudaDevAttrComputeCapabilityMinor, cudaDevAttrMaxThreadsPerMultiProcessor};
    for (int k = 0; k < 8; k++) {
        int v = 0;
        const cudaError_t e = cudaDeviceGetAttribute(&v, attrs[k], device);
        if (e != cudaSuccess) return probe_fail(LBM_ECUDA, "lbm_device_info: cudaDeviceGetAttribute", e);
        info[k] = v;
    }
    return LBM_OK;
}

int lbm_probe_fp64(int op, int chains, int blocks, int threads, long long iters, double *sink, void *stream)
{
    if (op < 0 || op > 2 || (chains != 8 && chains != 16) || blocks < 1 || threads < 32 || threads > 1024 ||
        threads % 32 || iters < 1 || !sink)
        return probe_fail(LBM_EINVAL, "lbm_probe_fp64: bad arguments", cudaSuccess);
    cudaStream_t s = (cudaStream_t)stream;
    if (chains == 8) launch_rate<8>(op, blocks, threads, iters, sink, s);
    else launch_rate<16>(op, blocks, threads, iters, sink, s);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return probe_fail(LBM_ECUDA, "lbm_probe_fp64: launch", e);
    return LBM_OK;
}

}  // extern "C"
