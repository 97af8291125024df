// Batched stepping (include/lbm.h, lbm_batch_*): many independent lattices of
// one kind advanced by one kernel launch per time step.
//
// Per call the host writes a descriptor per lattice (geometry, buffers,
// fields, collision coefficients) and the envelope pairs of every step into a
// pinned staging slot, copies them to the device asynchronously and launches
// one batched kernel per step.  Two slots alternate, so a call only waits for
// the copy issued two calls earlier.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <string>
#include <vector>

#include "lbm_ctx.h"

using namespace lbmk;

struct lbm_batch {
    std::vector<lbm_ctx *> ctx;
    int lattice = 0;
    cudaStream_t stream = nullptr;
    int count = 0;
    int nblocks = 0;
    int *d_first = nullptr;
    BatchItem *d_items[2] = {nullptr, nullptr};
    BatchItem *h_items[2] = {nullptr, nullptr};
    double2 *d_pairs[2] = {nullptr, nullptr};
    double2 *h_pairs[2] = {nullptr, nullptr};
    size_t pairs_cap[2] = {0, 0};  // double2 entries per slot
    cudaEvent_t ev[2] = {nullptr, nullptr};
    int slot = 0;
    long long launches = 0;
    std::string err;
};

namespace {

thread_local std::string g_batch_create_error;

int bfail(lbm_batch *b, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (b) b->err = buf;
    else g_batch_create_error = buf;
    return code;
}

#define BCK(call, what)                                                                         \
    do {                                                                                        \
        cudaError_t e_ = (call);                                                                \
        if (e_ != cudaSuccess) return bfail(b, LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e_)); \
    } while (0)

// Second value of a step's envelope pair as the batched kernels expect it:
// D2Q9 (a_pre + a_post)/12, D2Q5 (a_pre + a_post)/10, D3Q27 a_post -- the same
// expressions as the single-lattice launchers, so both paths agree bit for bit.
double pair_second(int lattice, double apre, double apost)
{
    if (lattice == LBM_D2Q9) return (apre + apost) / 12.0;
    if (lattice == LBM_D2Q5_CDE) return (apre + apost) / 10.0;
    return apost;
}

int grow_pairs(lbm_batch *b, int s, size_t need)
{
    if (need <= b->pairs_cap[s]) return LBM_OK;
    size_t cap = std::max(need, 2 * b->pairs_cap[s]);
    BCK(cudaStreamSynchronize(b->stream), "lbm_batch_step: sync before growing");
    cudaFreeHost(b->h_pairs[s]);
    cudaFree(b->d_pairs[s]);
    b->h_pairs[s] = nullptr;
    b->d_pairs[s] = nullptr;
    b->pairs_cap[s] = 0;
    BCK(cudaMallocHost(&b->h_pairs[s], cap * sizeof(double2)), "cudaMallocHost(pairs)");
    BCK(cudaMalloc(&b->d_pairs[s], cap * sizeof(double2)), "cudaMalloc(pairs)");
    b->pairs_cap[s] = cap;
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_batch_create(lbm_batch **out, lbm_ctx *const *ctxs, int count)
{
    g_batch_create_error.clear();
    if (!out) return bfail(nullptr, LBM_EINVAL, "lbm_batch_create: out is NULL");
    *out = nullptr;
    if (!ctxs || count < 1) return bfail(nullptr, LBM_EINVAL, "lbm_batch_create: need at least one context");
    for (int i = 0; i < count; i++) {
        if (!ctxs[i]) return bfail(nullptr, LBM_EINVAL, "lbm_batch_create: context %d is NULL", i);
        if (ctxs[i]->lattice != ctxs[0]->lattice || ctxs[i]->storage != ctxs[0]->storage)
            return bfail(nullptr, LBM_EINVAL, "lbm_batch_create: contexts differ in lattice or storage");
        if (ctxs[i]->stream != ctxs[0]->stream || ctxs[i]->device != ctxs[0]->device)
            return bfail(nullptr, LBM_EINVAL, "lbm_batch_create: contexts differ in stream or device");
        for (int j = 0; j < i; j++)
            if (ctxs[j] == ctxs[i]) return bfail(nullptr, LBM_EINVAL, "lbm_batch_create: context %d repeated", i);
    }
    lbm_batch *b = new (std::nothrow) lbm_batch();
    if (!b) return bfail(nullptr, LBM_ENOMEM, "lbm_batch_create: out of host memory");
    b->ctx.assign(ctxs, ctxs + count);
    b->lattice = ctxs[0]->lattice;
    b->stream = ctxs[0]->stream;
    b->count = count;
    std::vector<int> first(count);
    long long nb = 0;
    for (int i = 0; i < count; i++) {
        first[i] = (int)nb;
        nb += batch_blocks(ctxs[i]->g);
    }
    if (nb > 2147483647LL) {
        delete b;
        return bfail(nullptr, LBM_EINVAL, "lbm_batch_create: more than 2^31-1 blocks");
    }
    b->nblocks = (int)nb;
    cudaError_t e = cudaMalloc(&b->d_first, count * sizeof(int));
    for (int s = 0; s < 2 && e == cudaSuccess; s++) {
        e = cudaMalloc(&b->d_items[s], count * sizeof(BatchItem));
        if (e == cudaSuccess) e = cudaMallocHost(&b->h_items[s], count * sizeof(BatchItem));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev[s], cudaEventDisableTiming);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_first, first.data(), count * sizeof(int), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        int code = e == cudaErrorMemoryAllocation ? LBM_ENOMEM : LBM_ECUDA;
        bfail(nullptr, code, "lbm_batch_create: %s", cudaGetErrorString(e));
        cudaGetLastError();
        lbm_batch_destroy(b);
        return code;
    }
    *out = b;
    return LBM_OK;
}

void lbm_batch_destroy(lbm_batch *b)
{
    if (!b) return;
    cudaStreamSynchronize(b->stream);
    cudaFree(b->d_first);
    for (int s = 0; s < 2; s++) {
        cudaFree(b->d_items[s]);
        cudaFreeHost(b->h_items[s]);
        cudaFree(b->d_pairs[s]);
        cudaFreeHost(b->h_pairs[s]);
        if (b->ev[s]) cudaEventDestroy(b->ev[s]);
    }
    delete b;
}

const char *lbm_batch_last_error(const lbm_batch *b)
{
    return b ? b->err.c_str() : g_batch_create_error.c_str();
}

int lbm_batch_step(lbm_batch *b, long n)
{
    if (!b) return LBM_EINVAL;
    b->err.clear();
    if (n < 0) return bfail(b, LBM_EINVAL, "lbm_batch_step: n < 0");
    if (n == 0) return LBM_OK;
    if (n > 2147483647L / b->count) return bfail(b, LBM_EINVAL, "lbm_batch_step: n too large");
    for (int i = 0; i < b->count; i++) {
        const lbm_ctx *c = b->ctx[i];
        if (!c->initialised) return bfail(b, LBM_ESTATE, "lbm_batch_step: context %d not initialised", i);
        if (!lbmc::envelope_covers(c, c->t, n))
            return bfail(b, LBM_EINVAL, "lbm_batch_step: context %d steps outside its envelope table", i);
    }
    const int s = b->slot;
    b->slot ^= 1;
    // The staging slot was last read by the copy recorded two calls ago.
    BCK(cudaEventSynchronize(b->ev[s]), "lbm_batch_step: wait for staging slot");
    int rc = grow_pairs(b, s, (size_t)n * b->count);
    if (rc != LBM_OK) return rc;
    for (int i = 0; i < b->count; i++) {
        const lbm_ctx *c = b->ctx[i];
        BatchItem &it = b->h_items[s][i];
        it = BatchItem{};
        it.g = c->g;
        it.buf[0] = c->A;
        it.buf[1] = c->B;
        it.parity = 0;
        it.fkind = c->force.kind;
        it.F = c->force.d;
        it.vkind = c->vel.kind;
        it.V = c->vel.d;
        batch_coef(c->lattice, c->omega, it);
        for (long k = 0; k < n; k++) {
            double apre, apost;
            lbmc::envelope_pair(c, c->t + k, apre, apost);
            b->h_pairs[s][(size_t)k * b->count + i] = make_double2(apre, pair_second(b->lattice, apre, apost));
        }
    }
    BCK(cudaMemcpyAsync(b->d_items[s], b->h_items[s], b->count * sizeof(BatchItem), cudaMemcpyHostToDevice,
                        b->stream),
        "lbm_batch_step: copy descriptors");
    BCK(cudaMemcpyAsync(b->d_pairs[s], b->h_pairs[s], (size_t)n * b->count * sizeof(double2),
                        cudaMemcpyHostToDevice, b->stream),
        "lbm_batch_step: copy envelope pairs");
    BCK(cudaEventRecord(b->ev[s], b->stream), "lbm_batch_step: record");
    for (long k = 0; k < n; k++) {
        cudaError_t e = batch_step(b->lattice, b->d_items[s], b->d_first, b->count, b->nblocks, b->d_pairs[s],
                                   (int)k, b->stream);
        if (e != cudaSuccess) return bfail(b, LBM_ECUDA, "lbm_batch_step: kernel: %s", cudaGetErrorString(e));
        b->launches++;
    }
    for (int i = 0; i < b->count; i++) {
        lbm_ctx *c = b->ctx[i];
        if (n & 1) std::swap(c->A, c->B);
        c->t += n;
    }
    return LBM_OK;
}

int lbm_batch_launch_count(const lbm_batch *b, long long *count)
{
    if (!b || !count) return LBM_EINVAL;
    *count = b->launches;
    return LBM_OK;
}

}  // extern "C"
