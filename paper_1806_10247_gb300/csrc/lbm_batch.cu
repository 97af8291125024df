// Batched stepping (include/lbm.h, lbm_batch_*): many independent lattices of
// one kind advanced by one kernel launch per time step.
//
// The device keeps one descriptor per lattice (geometry, both population
// buffers, fields, collision coefficients); it is re-sent only when a member
// changed (its version counter moved, or its buffers are no longer in
// lockstep with the others).  The buffer parity of a step is a launch
// argument.  The envelope pairs of a step travel in the launch arguments for
// batches of up to kInlinePairs lattices; larger batches copy a per-call
// table through one of two alternating pinned staging slots.
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
    BatchItem *d_items = nullptr;      // descriptors on the device
    BatchItem *h_items = nullptr;      // pinned staging of the descriptors
    cudaEvent_t ev_items = nullptr;    // recorded after the last descriptor copy
    bool items_valid = false;
    std::vector<long long> item_version;
    std::vector<double *> item_buf0;   // buf[0] of each uploaded descriptor
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
// expressions as the single-lattice launchers.
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
    b->item_version.assign(count, -1);
    b->item_buf0.assign(count, nullptr);
    cudaError_t e = cudaMalloc(&b->d_first, count * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_items, count * sizeof(BatchItem));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_items, count * sizeof(BatchItem));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_items, cudaEventDisableTiming);
    for (int s = 0; s < 2 && e == cudaSuccess; s++) e = cudaEventCreateWithFlags(&b->ev[s], cudaEventDisableTiming);
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
    cudaFree(b->d_items);
    cudaFreeHost(b->h_items);
    if (b->ev_items) cudaEventDestroy(b->ev_items);
    for (int s = 0; s < 2; s++) {
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
    // Descriptors: reuse the device copy while every member is unchanged and
    // all members sit on the same buffer parity relative to it.
    int parity = 0;
    bool reuse = b->items_valid;
    for (int i = 0; i < b->count && reuse; i++) {
        const lbm_ctx *c = b->ctx[i];
        const int p = c->A == b->item_buf0[i] ? 0 : 1;
        if (c->version != b->item_version[i] || (i == 0 ? false : p != parity)) reuse = false;
        if (i == 0) parity = p;
    }
    if (!reuse) {
        BCK(cudaEventSynchronize(b->ev_items), "lbm_batch_step: wait for descriptor staging");
        for (int i = 0; i < b->count; i++) {
            const lbm_ctx *c = b->ctx[i];
            BatchItem &it = b->h_items[i];
            it = BatchItem{};
            it.g = c->g;
            it.rho_ref = c->rho_ref;
            it.buf[0] = c->A;
            it.buf[1] = c->B;
            it.parity = 0;
            it.fkind = c->force.kind;
            it.F = c->force.d;
            it.vkind = c->vel.kind;
            it.V = c->vel.d;
            batch_coef(c->lattice, c->omega, it);
            for (int k = 0; k < 16; k++) it.fcoef[k] = (float)it.coef[k];
            it.fcoef[16] = (float)(it.coef[4] + (2.0 / 3.0) * it.coef[7]);
            it.frho_ref = (float)it.rho_ref;
            b->item_version[i] = c->version;
            b->item_buf0[i] = c->A;
        }
        BCK(cudaMemcpyAsync(b->d_items, b->h_items, b->count * sizeof(BatchItem), cudaMemcpyHostToDevice,
                            b->stream),
            "lbm_batch_step: copy descriptors");
        BCK(cudaEventRecord(b->ev_items, b->stream), "lbm_batch_step: record");
        b->items_valid = true;
        parity = 0;
    }
    BatchLaunch L{};
    L.items = b->d_items;
    L.first = b->d_first;
    L.count = b->count;
    const bool inline_pairs = b->count <= kInlinePairs;
    if (!inline_pairs) {
        const int s = b->slot;
        b->slot ^= 1;
        // The staging slot was last read by the copy recorded two calls ago.
        BCK(cudaEventSynchronize(b->ev[s]), "lbm_batch_step: wait for staging slot");
        int rc = grow_pairs(b, s, (size_t)n * b->count);
        if (rc != LBM_OK) return rc;
        const bool fp32 = b->ctx[0]->storage != LBM_FP64;
        float2 *hf = reinterpret_cast<float2 *>(b->h_pairs[s]);  // FP32 pairs reuse the staging memory
        for (int i = 0; i < b->count; i++) {
            const lbm_ctx *c = b->ctx[i];
            for (long k = 0; k < n; k++) {
                double apre, apost;
                lbmc::envelope_pair(c, c->t + k, apre, apost);
                const double second = pair_second(b->lattice, apre, apost);
                if (fp32) hf[(size_t)k * b->count + i] = make_float2((float)apre, (float)second);
                else b->h_pairs[s][(size_t)k * b->count + i] = make_double2(apre, second);
            }
        }
        BCK(cudaMemcpyAsync(b->d_pairs[s], b->h_pairs[s], (size_t)n * b->count * sizeof(double2),
                            cudaMemcpyHostToDevice, b->stream),
            "lbm_batch_step: copy envelope pairs");
        BCK(cudaEventRecord(b->ev[s], b->stream), "lbm_batch_step: record");
        if (fp32) L.pairsf = reinterpret_cast<const float2 *>(b->d_pairs[s]);
        else L.pairs = b->d_pairs[s];
    }
    for (long k = 0; k < n; k++) {
        L.k = (int)k;
        L.parity = (parity + (int)k) & 1;
        if (inline_pairs)
            for (int i = 0; i < b->count; i++) {
                double apre, apost;
                lbmc::envelope_pair(b->ctx[i], b->ctx[i]->t + k, apre, apost);
                const double second = pair_second(b->lattice, apre, apost);
                L.inl[i] = make_double2(apre, second);
                L.inlf[i] = make_float2((float)apre, (float)second);
            }
        const int storage = b->ctx[0]->storage;
        cudaError_t e = storage == LBM_FP64 ? batch_step(b->lattice, L, b->nblocks, b->stream)
                                            : rp_batch_step(b->lattice, storage, L, b->nblocks, b->stream);
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
