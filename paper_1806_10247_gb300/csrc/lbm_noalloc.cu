// lbm_reduce_sums_noalloc: the mass / momentum reduction of lbm_reduce without
// any device allocation.
//
// lbm_reduce needs device scratch for its per-block partial sums (allocated at
// lbm_create) and lazily allocates a velocity snapshot on its first call.  Some
// callers cannot allocate at the moment they want these sums: code whose
// device memory is owned by another allocator (for example a PyTorch process
// whose caching allocator already holds the free HBM, where a raw cudaMalloc
// can fail even though memory is nominally available), and monitoring code
// inside a running time loop that must not call cudaMalloc / cudaFree because
// those calls can synchronise the whole device and stall every other stream.
// This entry point serves them: its scratch is a fixed, file-scope device
// array, so it calls no cudaMalloc, cudaFree or allocating library routine.
#include <cuda_runtime.h>

#include <mutex>

#include "lbm_ctx.h"

namespace {

// Partial sums of at most kMaxBlocks blocks plus the final result, 8 doubles
// each: (1216 + 1) * 8 * 8 B = 77,888 B held by every GPU that loads the
// library, until the process exits.  1216 = 152 SMs x 8 resident blocks is the
// largest grid the reduction ever uses (it loops over nodes), so no lattice
// exceeds it.
constexpr int kMaxBlocks = lbmk::kReduceMaxBlocks;
static_assert(kMaxBlocks == 1216, "the header's stated scratch size (1217 x 8 doubles) follows this cap");
constexpr int kSlots = 8;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_reduce_scratch[(kMaxBlocks + 1) * kSlots];

std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_reduce_scratch on `device`, looked up once per device
// with that device current.  In host code the name g_reduce_scratch is only a
// host-side stand-in and must never be passed to a kernel.
int scratch_on(lbm_ctx *c, int device, double **out)
{
    if (device < 0 || device >= kMaxDevices)
        return lbmc::fail(c, LBM_EINVAL, "lbm_reduce_sums_noalloc: device %d out of range", device);
    std::lock_guard<std::mutex> lock(g_mu);
    if (g_scratch_ptr[device] == nullptr) {
        int prev = 0;
        cudaError_t e = cudaGetDevice(&prev);
        if (e == cudaSuccess && prev != device) e = cudaSetDevice(device);
        double *p = nullptr;
        if (e == cudaSuccess) e = cudaGetSymbolAddress((void **)&p, g_reduce_scratch);
        if (prev != device) cudaSetDevice(prev);
        if (e != cudaSuccess) return lbmc::cuda_fail(c, e, "lbm_reduce_sums_noalloc: cudaGetSymbolAddress");
        g_scratch_ptr[device] = p;
    }
    *out = g_scratch_ptr[device];
    return LBM_OK;
}

}  // namespace

extern "C" int lbm_reduce_sums_noalloc(lbm_ctx *c, double out[4])
{
    using namespace lbmc;
    if (!c) return LBM_EINVAL;
    c->err.clear();
    if (!c->initialised) return fail(c, LBM_ESTATE, "lbm_reduce_sums_noalloc: populations not initialised");
    if (!out) return fail(c, LBM_EINVAL, "lbm_reduce_sums_noalloc: out is NULL");
    const int nb = lbmk::reduce_blocks(c->g);
    if (nb > kMaxBlocks)
        return fail(c, LBM_EINVAL, "lbm_reduce_sums_noalloc: %d partial blocks exceed the scratch limit of %d",
                    nb, kMaxBlocks);
    double *scratch = nullptr;
    int rc = scratch_on(c, c->device, &scratch);
    if (rc != LBM_OK) return rc;
    // a local-reference context is read through its FP32 deviations, whose
    // buffer an earlier read or write of the state must have allocated
    if (c->lref_every && !c->lref_dev)
        return fail(c, LBM_ESTATE, "lbm_reduce_sums_noalloc: a context stored at a local reference needs one "
                                   "allocating read of its state (e.g. lbm_reduce) first");
    LrefView view(c, true);
    if (view.rc != LBM_OK) return view.rc;
    // Every partial slot that the final pass reads is written by its block
    // first, and the result slot is written by the final pass, so nothing has
    // to be cleared between calls.
    double apre, apost;
    envelope_pair(c, c->t, apre, apost);
    lbmk::LaunchArgs a = launch_args(c, c->A, nullptr, apre, apost);
    double *result = scratch + (size_t)kMaxBlocks * kSlots;
    LBM_CK(lbmk::reduce_sums(c->lattice, a, scratch, nb, result), "lbm_reduce_sums_noalloc: kernels");
    c->launches += 2;
    double r[kSlots];
    LBM_CK(cudaMemcpyAsync(r, result, sizeof r, cudaMemcpyDeviceToHost, c->stream), "lbm_reduce_sums_noalloc: copy");
    LBM_CK(cudaStreamSynchronize(c->stream), "lbm_reduce_sums_noalloc");
    for (int k = 0; k < 4; k++) out[k] = r[k];
    if (r[5] != 0.0)
        return fail(c, LBM_EUNSTABLE, "lbm_reduce_sums_noalloc: non-finite or non-positive density/scalar");
    return LBM_OK;
}
