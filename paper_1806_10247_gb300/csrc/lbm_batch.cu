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
//
// Tiling (reduced-precision batches): the nodes of every member are cut into
// tiles of 128, 256 or 512 nodes (one thread per node); a launch either gives
// each tile its own block or runs a persistent grid (as many blocks as are
// resident on the GPU at once) whose blocks take contiguous runs of tiles.
// lbm_batch_autotune times every combination on the batch itself and keeps the
// fastest.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <new>
#include <string>
#include <vector>

#include "lbm_ctx.h"

using namespace lbmk;

// Asynchronous packed readbacks use their slots in turn (host destination,
// device staging, a_pre staging, events), so up to three can be in flight.
constexpr int kReadbackSlots = 3;

struct lbm_batch {
    std::vector<lbm_ctx *> ctx;
    int lattice = 0;
    cudaStream_t stream = nullptr;
    int count = 0;
    // tile sizes kTiles[j]: first tile of each member (device) and the tile count
    int *d_first[3] = {nullptr, nullptr, nullptr};
    long long ntiles[3] = {0, 0, 0};
    int tile_idx = 1;                  // index into kTiles of the tiling in use
    bool persistent = false;
    int resident[3] = {0, 0, 0};       // resident blocks on the GPU per tile size (0 = not queried)
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
    long long graph_replays = 0;
    // CUDA-graph replay of graph_steps steps (0 = off)
    int graph_steps = 0;
    cudaGraphExec_t gexec = nullptr;
    int gparity = -1;                  // descriptor parity the graph was captured for
    cudaStream_t gstream = nullptr;    // private stream used only to capture
    double2 *h_gpairs = nullptr;       // pinned envelope pairs of one replay (double2 or float2)
    double2 *d_gpairs = nullptr;
    bool gpairs_filled = false;        // constant envelopes: pairs written once
    cudaEvent_t ev_graph = nullptr;    // recorded after each replay
    // packed moments (lbm_batch_moments_packed)
    long long total_nodes = 0;
    long long *d_off = nullptr;        // first node of each member in the packed output
    double *h_apre = nullptr;          // pinned a_pre of each member, and its device copy
    double *d_apre = nullptr;
    cudaEvent_t ev_apre = nullptr;     // recorded after the a_pre copy
    double *d_mom = nullptr;           // device staging of the packed output (host destinations)
    // asynchronous packed readback (where = 2 / 3): two slots used in turn,
    // kernel (and, for 2, copies) on a private stream so that they overlap
    // the next steps
    double *d_momq[kReadbackSlots] = {};
    cudaStream_t cstream = nullptr;
    cudaEvent_t ev_copied[kReadbackSlots] = {};  // slot copied out (recorded on the copy stream)
    cudaEvent_t ev_host[kReadbackSlots] = {};    // the fields of slot k are in host memory
    // where >= 2 readbacks run their kernel on the copy stream, after the
    // state it reads (ev_state on the batch stream) and overlapping the next
    // step; ev_read[k] marks that slot k's kernel has read the populations
    // (each member keeps it as a reader entry of the buffer it read)
    cudaEvent_t ev_read[kReadbackSlots] = {};
    bool read_recorded[kReadbackSlots] = {};
    cudaEvent_t ev_state = nullptr;
    double *h_apreq[kReadbackSlots] = {};  // pinned a_pre of each member, per slot
    double *d_apreq[kReadbackSlots] = {};
    int qslot = 0;   // slot of the next readback (the slots are used in turn)
    bool copies_pending = false;
    std::string err;
};

namespace {

constexpr int kTiles[3] = {128, 256, 512};

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
// D2Q9 (a_pre + a_post)/12, D2Q5 (a_pre + a_post)/10, D3Q27 and D3Q15 a_post --
// the same expressions as the single-lattice launchers.
double pair_second(int lattice, double apre, double apost)
{
    if (lattice == LBM_D2Q9) return (apre + apost) / 12.0;
    if (lattice == LBM_D2Q5_CDE) return (apre + apost) / 10.0;
    return apost;
}

// First value of an FP64 pair: a_pre, halved for D2Q5 (its step takes
// g_0 + (a_pre/2) S; halving is exact, so a kernel that needs a_pre itself
// doubles it back exactly).  Reduced-precision pairs carry a_pre.
double pair_first(int lattice, double apre) { return lattice == LBM_D2Q5_CDE ? 0.5 * apre : apre; }

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

// Is e one of this batch's readback events?
bool is_own_reader(const lbm_batch *b, cudaEvent_t e)
{
    for (int k = 0; k < kReadbackSlots; k++)
        if (e == b->ev_read[k]) return true;
    return false;
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
        if (ctxs[i]->sround)
            return bfail(nullptr, LBM_EINVAL, "lbm_batch_create: context %d rounds stochastically (single-lattice "
                                              "steps only)", i);
        if (ctxs[i]->lref_every)
            return bfail(nullptr, LBM_EINVAL, "lbm_batch_create: context %d stores at a local reference "
                                              "(single-lattice steps only)", i);
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
    std::vector<int> first[3];
    for (int j = 0; j < 3; j++) {
        first[j].resize(count);
        long long nt = 0;
        for (int i = 0; i < count; i++) {
            first[j][i] = (int)std::min(nt, 2147483647LL);
            nt += (ctxs[i]->g.N + kTiles[j] - 1) / kTiles[j];
        }
        b->ntiles[j] = nt;
    }
    if (b->ntiles[0] > 2147483647LL) {
        delete b;
        return bfail(nullptr, LBM_EINVAL, "lbm_batch_create: more than 2^31-1 tiles of 128 nodes");
    }
    b->item_version.assign(count, -1);
    b->item_buf0.assign(count, nullptr);
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < 3 && e == cudaSuccess; j++) e = cudaMalloc(&b->d_first[j], count * sizeof(int));
    std::vector<long long> off(count);
    for (int i = 0; i < count; i++) {
        off[i] = b->total_nodes;
        b->total_nodes += ctxs[i]->g.N;
    }
    if (e == cudaSuccess) e = cudaMalloc(&b->d_off, count * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_apre, count * sizeof(double));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_apre, count * sizeof(double));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_apre, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_off, off.data(), count * sizeof(long long), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_items, count * sizeof(BatchItem));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_items, count * sizeof(BatchItem));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_items, cudaEventDisableTiming);
    for (int s = 0; s < 2 && e == cudaSuccess; s++) e = cudaEventCreateWithFlags(&b->ev[s], cudaEventDisableTiming);
    for (int j = 0; j < 3 && e == cudaSuccess; j++)
        e = cudaMemcpyAsync(b->d_first[j], first[j].data(), count * sizeof(int), cudaMemcpyHostToDevice, b->stream);
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
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->gstream) cudaStreamDestroy(b->gstream);
    if (b->ev_graph) cudaEventDestroy(b->ev_graph);
    cudaFreeHost(b->h_gpairs);
    cudaFree(b->d_gpairs);
    for (int j = 0; j < 3; j++) cudaFree(b->d_first[j]);
    cudaFree(b->d_off);
    cudaFree(b->d_apre);
    cudaFreeHost(b->h_apre);
    cudaFree(b->d_mom);
    if (b->cstream) cudaStreamSynchronize(b->cstream);
    // the readbacks are done: the members forget this batch's reader events
    for (lbm_ctx *c : b->ctx)
        for (int k = 0; k < 2; k++)
            if (c->rd_buf[k] && is_own_reader(b, c->rd_ev[k])) {
                c->rd_buf[k] = nullptr;
                c->rd_ev[k] = nullptr;
            }
    for (int k = 0; k < kReadbackSlots; k++) {
        cudaFree(b->d_momq[k]);
        cudaFree(b->d_apreq[k]);
        cudaFreeHost(b->h_apreq[k]);
        if (b->ev_copied[k]) cudaEventDestroy(b->ev_copied[k]);
        if (b->ev_read[k]) cudaEventDestroy(b->ev_read[k]);
    }
    if (b->ev_state) cudaEventDestroy(b->ev_state);
    if (b->cstream) cudaStreamDestroy(b->cstream);
    if (b->ev_apre) cudaEventDestroy(b->ev_apre);
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

namespace {

bool has_envelope(const lbm_batch *b)
{
    for (const lbm_ctx *c : b->ctx)
        if (c->env || !c->env_tab.empty()) return true;
    return false;
}

// Make the device descriptors current; returns the buffer parity of the
// current state relative to them (0 or 1) through *parity.
// Before work on the batch stream writes the members' population buffers
// (each member's second buffer, or both when `both`), make the stream wait for
// the readbacks that may still read them (the members' reader entries; one
// wait per distinct event).
int wait_member_readers(lbm_batch *b, bool both)
{
    std::vector<cudaEvent_t> evs;
    for (lbm_ctx *c : b->ctx)
        for (int k = 0; k < 2; k++) {
            if (!c->rd_buf[k] || (!both && c->rd_buf[k] != c->B)) continue;
            if (std::find(evs.begin(), evs.end(), c->rd_ev[k]) == evs.end()) evs.push_back(c->rd_ev[k]);
            c->rd_buf[k] = nullptr;
            c->rd_ev[k] = nullptr;
        }
    for (cudaEvent_t e : evs) BCK(cudaStreamWaitEvent(b->stream, e, 0), "wait for a readback of the populations");
    return LBM_OK;
}

int refresh_descriptors(lbm_batch *b, int *parity)
{
    int p0 = 0;
    bool reuse = b->items_valid;
    for (int i = 0; i < b->count && reuse; i++) {
        const lbm_ctx *c = b->ctx[i];
        const int p = c->A == b->item_buf0[i] ? 0 : 1;
        if (c->version != b->item_version[i] || (i > 0 && p != p0)) reuse = false;
        if (i == 0) p0 = p;
    }
    if (reuse) {
        *parity = p0;
        return LBM_OK;
    }
    if (b->gexec) {
        // a captured graph may hold the old descriptors by value: capture again
        BCK(cudaStreamSynchronize(b->stream), "lbm_batch_step: sync before dropping the graph");
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    BCK(cudaEventSynchronize(b->ev_items), "lbm_batch_step: wait for descriptor staging");
    // readback kernels on the copy stream read the descriptors too
    for (int k = 0; k < kReadbackSlots; k++)
        if (b->read_recorded[k])
            BCK(cudaStreamWaitEvent(b->stream, b->ev_read[k], 0), "lbm_batch_step: wait for a readback");
    for (int i = 0; i < b->count; i++)
        if (b->ctx[i]->lref_every || b->ctx[i]->sround)
            return bfail(b, LBM_EINVAL, "lbm_batch_step: member %d now rounds stochastically or stores at a local "
                                        "reference (single-lattice steps only)", i);
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
        if (c->lattice == LBM_D2Q5_CDE && c->storage != LBM_FP64 && it.vkind != FK_GENERAL) {
            // what one step adds to the member's reference: M g_ref - g_ref
            double cr[5];
            d2q5_reference_change(c->omega, it.vkind == FK_CONST ? it.V.cval[0] : 0.0,
                                  it.vkind == FK_CONST ? it.V.cval[1] : 0.0, c->gref, cr);
            for (int k = 0; k < 5; k++) it.fref[k] = (float)cr[k];
        }
        it.variant = batch_variant(c->lattice, c->omega, it.fkind, it.F);
        if (c->storage != LBM_FP64) it.variant &= 1;  // the reduced-precision kernels have no force-along-x form
        b->item_version[i] = c->version;
        b->item_buf0[i] = c->A;
    }
    BCK(cudaMemcpyAsync(b->d_items, b->h_items, b->count * sizeof(BatchItem), cudaMemcpyHostToDevice, b->stream),
        "lbm_batch_step: copy descriptors");
    BCK(cudaEventRecord(b->ev_items, b->stream), "lbm_batch_step: record");
    b->items_valid = true;
    *parity = 0;
    return LBM_OK;
}

bool reduced_precision(const lbm_batch *b) { return b->ctx[0]->storage != LBM_FP64; }

int resident_for(lbm_batch *b, int tile_idx)
{
    if (b->resident[tile_idx] == 0)
        b->resident[tile_idx] = reduced_precision(b)
                                    ? rp_batch_resident(b->lattice, b->ctx[0]->storage, kTiles[tile_idx])
                                    : batch_resident(b->lattice, kTiles[tile_idx]);
    return b->resident[tile_idx];
}

// One batched launch with the given tiling: fills in the tile map of L.
cudaError_t launch_tiled(lbm_batch *b, BatchLaunch L, int tile_idx, bool persistent, cudaStream_t s)
{
    const int nt = (int)b->ntiles[tile_idx];
    int grid = nt;
    L.first = b->d_first[tile_idx];
    L.ntiles = nt;
    L.persist = 0;
    L.single = 0;
    if (b->count == 1) {
        // one member: its descriptor goes in the launch arguments
        L.single = 1;
        L.one = b->h_items[0];
        persistent = false;
    }
    if (persistent) {
        const int r = resident_for(b, tile_idx);
        if (r > 0 && r < nt) {  // one resident grid; runs of nt / r tiles
            L.persist = 1;
            grid = r;
        }
    }
    if (!reduced_precision(b)) return batch_step(b->lattice, L, grid, kTiles[tile_idx], s);
    return rp_batch_step(b->lattice, b->ctx[0]->storage, L, grid, kTiles[tile_idx], s);
}

cudaError_t launch_one(lbm_batch *b, const BatchLaunch &L, cudaStream_t s)
{
    return launch_tiled(b, L, b->tile_idx, b->persistent, s);
}

// Envelope pairs of steps t_i .. t_i + k - 1 of every member into dst (double2
// for FP64 batches, float2 otherwise), [k][count].
void fill_pairs(const lbm_batch *b, void *dst, long k)
{
    const bool fp32 = b->ctx[0]->storage != LBM_FP64;
    for (int i = 0; i < b->count; i++) {
        const lbm_ctx *c = b->ctx[i];
        for (long s = 0; s < k; s++) {
            double apre, apost;
            lbmc::envelope_pair(c, c->t + s, apre, apost);
            const double second = pair_second(b->lattice, apre, apost);
            const size_t at = (size_t)s * b->count + i;
            if (fp32) reinterpret_cast<float2 *>(dst)[at] = make_float2((float)apre, (float)second);
            else reinterpret_cast<double2 *>(dst)[at] = make_double2(pair_first(b->lattice, apre), second);
        }
    }
}

// Envelope pairs of the members' next n steps into a device table (through
// one of the two alternating pinned staging slots), referenced by L.
int stage_pairs(lbm_batch *b, BatchLaunch &L, long n)
{
    const int s = b->slot;
    b->slot ^= 1;
    // The staging slot was last read by the copy recorded two calls ago.
    BCK(cudaEventSynchronize(b->ev[s]), "lbm_batch_step: wait for staging slot");
    int rc = grow_pairs(b, s, (size_t)n * b->count);
    if (rc != LBM_OK) return rc;
    fill_pairs(b, b->h_pairs[s], n);
    const bool fp32 = reduced_precision(b);
    const size_t esz = fp32 ? sizeof(float2) : sizeof(double2);
    BCK(cudaMemcpyAsync(b->d_pairs[s], b->h_pairs[s], (size_t)n * b->count * esz, cudaMemcpyHostToDevice,
                        b->stream),
        "lbm_batch_step: copy envelope pairs");
    BCK(cudaEventRecord(b->ev[s], b->stream), "lbm_batch_step: record");
    if (fp32) L.pairsf = reinterpret_cast<const float2 *>(b->d_pairs[s]);
    else L.pairs = b->d_pairs[s];
    return LBM_OK;
}

// Envelope pairs of step t_i + k of every member into the launch arguments.
void inline_pairs_of_step(const lbm_batch *b, BatchLaunch &L, long k)
{
    for (int i = 0; i < b->count; i++) {
        double apre, apost;
        lbmc::envelope_pair(b->ctx[i], b->ctx[i]->t + k, apre, apost);
        const double second = pair_second(b->lattice, apre, apost);
        L.inl[i] = make_double2(pair_first(b->lattice, apre), second);
        L.inlf[i] = make_float2((float)apre, (float)second);
    }
}

int check_members(lbm_batch *b, long n, const char *what)
{
    for (int i = 0; i < b->count; i++) {
        const lbm_ctx *c = b->ctx[i];
        if (!c->initialised) return bfail(b, LBM_ESTATE, "%s: context %d not initialised", what, i);
        if (!lbmc::envelope_covers(c, c->t, n))
            return bfail(b, LBM_EINVAL, "%s: context %d steps outside its envelope table", what, i);
    }
    return LBM_OK;
}

void drop_graph(lbm_batch *b)
{
    if (b->gexec) {
        cudaStreamSynchronize(b->stream);
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
}

// Capture graph_steps batched launches (after one copy of their envelope
// pairs from pinned memory) for descriptor parity `parity`.
int capture_graph(lbm_batch *b, int parity)
{
    if (b->gexec) {
        cudaGraphExecDestroy(b->gexec);
        b->gexec = nullptr;
    }
    const size_t bytes = (size_t)b->graph_steps * b->count * sizeof(double2);
    if (!b->gstream) BCK(cudaStreamCreateWithFlags(&b->gstream, cudaStreamNonBlocking), "graph stream");
    if (!b->ev_graph) BCK(cudaEventCreateWithFlags(&b->ev_graph, cudaEventDisableTiming), "graph event");
    if (!b->h_gpairs) {
        BCK(cudaMallocHost(&b->h_gpairs, bytes), "cudaMallocHost(graph pairs)");
        BCK(cudaMalloc(&b->d_gpairs, bytes), "cudaMalloc(graph pairs)");
    }
    b->gpairs_filled = false;
    BCK(cudaStreamBeginCapture(b->gstream, cudaStreamCaptureModeThreadLocal), "begin capture");
    cudaError_t e = cudaMemcpyAsync(b->d_gpairs, b->h_gpairs, bytes, cudaMemcpyHostToDevice, b->gstream);
    const bool fp32 = b->ctx[0]->storage != LBM_FP64;
    for (int k = 0; k < b->graph_steps && e == cudaSuccess; k++) {
        BatchLaunch L{};
        L.items = b->d_items;
        L.count = b->count;
        L.k = k;
        L.parity = (parity + k) & 1;
        if (fp32) L.pairsf = reinterpret_cast<const float2 *>(b->d_gpairs);
        else L.pairs = b->d_gpairs;
        e = launch_one(b, L, b->gstream);
    }
    cudaGraph_t graph = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(b->gstream, &graph);
    if (e == cudaSuccess) e = e2;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        b->gexec = nullptr;
        return bfail(b, LBM_ECUDA, "lbm_batch_step: graph capture: %s", cudaGetErrorString(e));
    }
    b->gparity = parity;
    return LBM_OK;
}


// Stream, events and staging of the asynchronous readbacks (on first use).
int ensure_readback(lbm_batch *b)
{
    if (b->cstream) return LBM_OK;
    BCK(cudaStreamCreateWithFlags(&b->cstream, cudaStreamNonBlocking), "copy stream");
    BCK(cudaEventCreateWithFlags(&b->ev_state, cudaEventDisableTiming), "event");
    for (int k = 0; k < kReadbackSlots; k++) {
        BCK(cudaEventCreateWithFlags(&b->ev_copied[k], cudaEventDisableTiming), "event");
        BCK(cudaEventCreateWithFlags(&b->ev_read[k], cudaEventDisableTiming), "event");
        BCK(cudaHostAlloc(&b->h_apreq[k], b->count * sizeof(double), cudaHostAllocDefault), "cudaHostAlloc(a_pre)");
        BCK(cudaMalloc(&b->d_apreq[k], b->count * sizeof(double)), "cudaMalloc(a_pre)");
    }
    return LBM_OK;
}

// Device addresses of host outputs that the device can address (pinned by
// cudaHostAlloc, or registered as mapped); refuses anything else.
int mapped_outputs(lbm_batch *b, double *rho, double *u, double **drho, double **du, const char *what)
{
    const bool scalar = b->lattice == LBM_D2Q5_CDE;
    double *outs[2] = {rho, u};
    double *devs[2] = {nullptr, nullptr};
    for (int k = 0; k < (scalar ? 1 : 2); k++) {
        cudaPointerAttributes pa{};
        const cudaError_t e = cudaPointerGetAttributes(&pa, outs[k]);
        if (e != cudaSuccess || pa.type != cudaMemoryTypeHost || !pa.devicePointer) {
            cudaGetLastError();
            return bfail(b, LBM_EINVAL, "%s: where = 3 needs host memory mapped into the device's address space", what);
        }
        devs[k] = static_cast<double *>(pa.devicePointer);
    }
    *drho = devs[0];
    *du = devs[1];
    return LBM_OK;
}

// where = 2 / 3 of lbm_batch_moments_packed: the moments kernel runs on the
// copy stream after the state it reads (so it overlaps the next step on the
// batch stream), then either copies the fields out of a device slot (2) or has
// written them straight into mapped host memory (3).
int packed_readback_async(lbm_batch *b, double *rho, double *u, int where, int half, int parity, size_t nrho,
                          size_t nu)
{
    const bool scalar = b->lattice == LBM_D2Q5_CDE;
    int rc = ensure_readback(b);
    if (rc != LBM_OK) return rc;
    double *drho = nullptr, *du = nullptr;
    if (where == 3) {
        rc = mapped_outputs(b, rho, u, &drho, &du, "lbm_batch_moments_packed");
        if (rc != LBM_OK) return rc;
    } else if (!b->d_momq[0]) {
        for (int k = 0; k < kReadbackSlots; k++)
            BCK(cudaMalloc(&b->d_momq[k], (nrho + nu) * sizeof(double)), "cudaMalloc(packed moments)");
    }
    const int slot = b->qslot;
    b->qslot = (b->qslot + 1) % kReadbackSlots;
    // a_pre of each member: in the launch arguments for small batches, else
    // through the slot's pinned staging, which the slot's previous readback
    // must have finished with
    const bool inl = b->count <= kInlinePairs;
    if (!inl && b->ev_host[slot])
        BCK(cudaEventSynchronize(b->ev_host[slot]), "lbm_batch_moments_packed: wait for the slot");
    if (where == 2) {
        drho = b->d_momq[slot];
        du = b->d_momq[slot] + nrho;
    }
    BatchMoments M{};
    for (int i = 0; i < b->count; i++) {
        double apre, apost;
        lbmc::envelope_pair(b->ctx[i], b->ctx[i]->t, apre, apost);
        if (inl) M.apre_inl[i] = apre;
        else b->h_apreq[slot][i] = apre;
    }
    // order after the state on the batch stream; a member buffer already read
    // by another batch's pending readback keeps that reader too (this copy
    // stream waits for it, so the new reader event implies the old one)
    BCK(cudaEventRecord(b->ev_state, b->stream), "lbm_batch_moments_packed: record");
    BCK(cudaStreamWaitEvent(b->cstream, b->ev_state, 0), "lbm_batch_moments_packed: wait");
    std::vector<cudaEvent_t> foreign;
    for (lbm_ctx *c : b->ctx)
        for (int k = 0; k < 2; k++)
            if (c->rd_buf[k] == c->A && !is_own_reader(b, c->rd_ev[k]) &&
                std::find(foreign.begin(), foreign.end(), c->rd_ev[k]) == foreign.end())
                foreign.push_back(c->rd_ev[k]);
    for (cudaEvent_t e : foreign) BCK(cudaStreamWaitEvent(b->cstream, e, 0), "lbm_batch_moments_packed: wait");
    if (!inl)
        BCK(cudaMemcpyAsync(b->d_apreq[slot], b->h_apreq[slot], b->count * sizeof(double), cudaMemcpyHostToDevice,
                            b->cstream),
            "lbm_batch_moments_packed: copy a_pre");
    M.items = b->d_items;
    M.first = b->d_first[1];
    M.count = b->count;
    M.parity = parity;
    M.half = half;
    M.apre = inl ? nullptr : b->d_apreq[slot];
    M.off = b->d_off;
    M.rho = drho;
    M.u = du;
    BCK(batch_moments(b->lattice, b->ctx[0]->storage, M, (int)b->ntiles[1], b->cstream),
        "lbm_batch_moments_packed: kernel");
    b->launches++;
    BCK(cudaEventRecord(b->ev_read[slot], b->cstream), "lbm_batch_moments_packed: record");
    b->read_recorded[slot] = true;
    for (lbm_ctx *c : b->ctx) {
        // one entry per buffer: the one already naming c->A, else a free one
        const int k = c->rd_buf[0] == c->A ? 0 : (c->rd_buf[1] == c->A ? 1 : (c->rd_buf[0] ? 1 : 0));
        c->rd_buf[k] = c->A;
        c->rd_ev[k] = b->ev_read[slot];
    }
    if (where == 2) {
        BCK(cudaMemcpyAsync(rho, drho, nrho * sizeof(double), cudaMemcpyDeviceToHost, b->cstream),
            "lbm_batch_moments_packed: copy rho");
        if (!scalar)
            BCK(cudaMemcpyAsync(u, du, nu * sizeof(double), cudaMemcpyDeviceToHost, b->cstream),
                "lbm_batch_moments_packed: copy u");
        BCK(cudaEventRecord(b->ev_copied[slot], b->cstream), "lbm_batch_moments_packed: record");
        b->ev_host[slot] = b->ev_copied[slot];
    } else {
        b->ev_host[slot] = b->ev_read[slot];
    }
    b->copies_pending = true;
    return LBM_OK;
}

}  // namespace

int lbm_batch_step(lbm_batch *b, long n)
{
    lbmc::NvtxRange nvtx_("lbm_batch_step");
    if (!b) return LBM_EINVAL;
    b->err.clear();
    if (n < 0) return bfail(b, LBM_EINVAL, "lbm_batch_step: n < 0");
    if (n == 0) return LBM_OK;
    if (n > 2147483647L / b->count) return bfail(b, LBM_EINVAL, "lbm_batch_step: n too large");
    int rc = check_members(b, n, "lbm_batch_step");
    if (rc != LBM_OK) return rc;
    // one step writes each member's second buffer only (a readback of the
    // current state may go on meanwhile); more steps write both
    rc = wait_member_readers(b, n > 1);
    if (rc != LBM_OK) return rc;
    int parity = 0;
    rc = refresh_descriptors(b, &parity);
    if (rc != LBM_OK) return rc;

    // Whole graph replays first (graph_steps is even: parity is unchanged).
    if (b->graph_steps > 0 && n >= b->graph_steps) {
        if (!b->gexec || b->gparity != parity) {
            rc = capture_graph(b, parity);
            if (rc != LBM_OK) return rc;
        }
        const bool env = has_envelope(b);
        while (n >= b->graph_steps) {
            if (env || !b->gpairs_filled) {
                // the previous replay's copy has read the pinned pairs by the time it completes
                BCK(cudaEventSynchronize(b->ev_graph), "lbm_batch_step: wait for the previous replay");
                fill_pairs(b, b->h_gpairs, b->graph_steps);
                b->gpairs_filled = true;
            }
            BCK(cudaGraphLaunch(b->gexec, b->stream), "lbm_batch_step: graph launch");
            BCK(cudaEventRecord(b->ev_graph, b->stream), "lbm_batch_step: record");
            b->launches += b->graph_steps;
            b->graph_replays++;
            for (lbm_ctx *c : b->ctx) c->t += b->graph_steps;
            n -= b->graph_steps;
        }
        if (n == 0) return LBM_OK;
    }

    if (b->count == 1) {
        // One member outside graph replays: its own single-lattice step kernel
        // (launch arguments by value, no descriptor), counted by the member.
        rc = lbm_step(b->ctx[0], n);
        if (rc != LBM_OK) return bfail(b, rc, "lbm_batch_step: %s", lbm_last_error(b->ctx[0]));
        return LBM_OK;
    }
    BatchLaunch L{};
    L.items = b->d_items;
    L.count = b->count;
    const bool inline_pairs = b->count <= kInlinePairs;
    if (!inline_pairs) {
        rc = stage_pairs(b, L, n);
        if (rc != LBM_OK) return rc;
    }
    for (long k = 0; k < n; k++) {
        L.k = (int)k;
        L.parity = (parity + (int)k) & 1;
        if (inline_pairs) inline_pairs_of_step(b, L, k);
        cudaError_t e = launch_one(b, L, b->stream);
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

int lbm_batch_set_graph(lbm_batch *b, int steps_per_graph)
{
    if (!b) return LBM_EINVAL;
    b->err.clear();
    if (steps_per_graph < 0 || (steps_per_graph & 1))
        return bfail(b, LBM_EINVAL, "lbm_batch_set_graph: steps per graph must be 0 or a positive even number");
    if (steps_per_graph != b->graph_steps) {
        if (b->gexec) {
            cudaStreamSynchronize(b->stream);
            cudaGraphExecDestroy(b->gexec);
            b->gexec = nullptr;
        }
        cudaFreeHost(b->h_gpairs);
        cudaFree(b->d_gpairs);
        b->h_gpairs = nullptr;
        b->d_gpairs = nullptr;
        b->graph_steps = steps_per_graph;
    }
    return LBM_OK;
}

int lbm_batch_set_tiling(lbm_batch *b, int tile, int persistent)
{
    if (!b) return LBM_EINVAL;
    b->err.clear();
    int j = -1;
    for (int k = 0; k < 3; k++)
        if (kTiles[k] == tile) j = k;
    if (j < 0 || (persistent != 0 && persistent != 1))
        return bfail(b, LBM_EINVAL, "lbm_batch_set_tiling: tile must be 128, 256 or 512 and persistent 0 or 1");
    if (j != b->tile_idx || (persistent != 0) != b->persistent) {
        drop_graph(b);
        b->tile_idx = j;
        b->persistent = persistent != 0;
    }
    return LBM_OK;
}

int lbm_batch_get_tiling(lbm_batch *b, int *tile, int *persistent, int *grid)
{
    if (!b) return LBM_EINVAL;
    b->err.clear();
    if (tile) *tile = kTiles[b->tile_idx];
    if (persistent) *persistent = b->persistent ? 1 : 0;
    if (grid) {
        long long g = b->ntiles[b->tile_idx];
        if (b->persistent && b->count > 1) {
            const long long r = resident_for(b, b->tile_idx);
            if (r > 0 && r < g) g = r;
        }
        *grid = (int)g;
    }
    return LBM_OK;
}

int lbm_batch_autotune(lbm_batch *b, int trial_steps, double *best_us, double *all_us)
{
    lbmc::NvtxRange nvtx_("lbm_batch_autotune");
    if (!b) return LBM_EINVAL;
    b->err.clear();
    if (trial_steps < 1 || trial_steps > 1000)
        return bfail(b, LBM_EINVAL, "lbm_batch_autotune: trial_steps must be in [1, 1000]");
    int rc = check_members(b, 1, "lbm_batch_autotune");
    if (rc != LBM_OK) return rc;
    rc = wait_member_readers(b, true);
    if (rc != LBM_OK) return rc;
    int parity = 0;
    rc = refresh_descriptors(b, &parity);
    if (rc != LBM_OK) return rc;
    // Trial launches keep the buffer parity: every one reads the current state
    // and overwrites the other buffer, which holds nothing until the next step.
    BatchLaunch L{};
    L.items = b->d_items;
    L.count = b->count;
    L.k = 0;
    L.parity = parity;
    if (b->count <= kInlinePairs) inline_pairs_of_step(b, L, 0);
    else if ((rc = stage_pairs(b, L, 1)) != LBM_OK) return rc;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BCK(cudaEventCreate(&e0), "lbm_batch_autotune: event");
    cudaError_t e = cudaEventCreate(&e1);
    if (all_us)
        for (int k = 0; k < 6; k++) all_us[k] = -1.0;
    float best = -1.0f;
    int best_j = b->tile_idx;
    bool best_p = b->persistent;
    for (int j = 0; j < 3 && e == cudaSuccess; j++)
        for (int p = 0; p < 2 && e == cudaSuccess; p++) {
            e = launch_tiled(b, L, j, p != 0, b->stream);  // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(e0, b->stream);
            for (int r = 0; r < trial_steps && e == cudaSuccess; r++) e = launch_tiled(b, L, j, p != 0, b->stream);
            if (e == cudaSuccess) e = cudaEventRecord(e1, b->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            b->launches += trial_steps + 1;
            if (e == cudaSuccess && all_us) all_us[2 * j + p] = 1000.0 * ms / trial_steps;
            if (e == cudaSuccess && (best < 0.0f || ms < best)) {
                best = ms;
                best_j = j;
                best_p = p != 0;
            }
        }
    cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) return bfail(b, LBM_ECUDA, "lbm_batch_autotune: %s", cudaGetErrorString(e));
    if (best_j != b->tile_idx || best_p != b->persistent) {
        drop_graph(b);
        b->tile_idx = best_j;
        b->persistent = best_p;
    }
    if (best_us) *best_us = 1000.0 * best / trial_steps;
    return LBM_OK;
}

int lbm_batch_moments(lbm_batch *b, double *const *rho, double *const *u, int where, int half_forced)
{
    if (!b) return LBM_EINVAL;
    b->err.clear();
    if (!rho) return bfail(b, LBM_EINVAL, "lbm_batch_moments: rho is NULL");
    if (where != 0 && where != 1) return bfail(b, LBM_EINVAL, "lbm_batch_moments: where must be 0 or 1");
    const bool scalar = b->lattice == LBM_D2Q5_CDE;
    for (int i = 0; i < b->count; i++) {
        if (!b->ctx[i]->initialised)
            return bfail(b, LBM_ESTATE, "lbm_batch_moments: context %d not initialised", i);
        if (!rho[i] || (!scalar && (!u || !u[i])))
            return bfail(b, LBM_EINVAL, "lbm_batch_moments: NULL output for context %d", i);
    }
    // Every member's fields are formed into its scratch buffer (the second
    // population buffer, or the staging buffer of a reduced-precision context)
    // and copied out on the shared stream; one synchronisation at the end.
    if (where == 0) {
        const int rc = wait_member_readers(b, false);
        if (rc != LBM_OK) return rc;
    }
    for (int i = 0; i < b->count; i++) {
        lbm_ctx *c = b->ctx[i];
        double apre, apost;
        lbmc::envelope_pair(c, c->t, apre, apost);
        LaunchArgs a = lbmc::launch_args(c, c->A, nullptr, apre, apost);
        const size_t N = (size_t)c->g.N;
        double *drho = rho[i], *du = scalar ? nullptr : u[i];
        if (where == 0) {
            double *st = c->B;
            if (c->storage != LBM_FP64) {
                int rc = lbmc::ensure_stage(c);
                if (rc != LBM_OK) return bfail(b, rc, "lbm_batch_moments: %s", c->err.c_str());
                st = c->stage;
            }
            drho = st;
            du = st + N;
        }
        BCK(moments(c->lattice, a, drho, du, half_forced ? 1 : 0), "lbm_batch_moments: moments kernel");
        c->launches++;
        if (where == 0) {
            BCK(cudaMemcpyAsync(rho[i], drho, N * sizeof(double), cudaMemcpyDeviceToHost, b->stream),
                "lbm_batch_moments: copy rho");
            if (!scalar)
                BCK(cudaMemcpyAsync(u[i], du, (size_t)c->dim * N * sizeof(double), cudaMemcpyDeviceToHost, b->stream),
                    "lbm_batch_moments: copy u");
        }
    }
    if (where == 0) BCK(cudaStreamSynchronize(b->stream), "lbm_batch_moments");
    return LBM_OK;
}

int lbm_batch_moments_packed(lbm_batch *b, double *rho, double *u, int where, int half_forced)
{
    lbmc::NvtxRange nvtx_("lbm_batch_moments_packed");
    if (!b) return LBM_EINVAL;
    b->err.clear();
    const bool scalar = b->lattice == LBM_D2Q5_CDE;
    if (!rho || (!scalar && !u)) return bfail(b, LBM_EINVAL, "lbm_batch_moments_packed: NULL output");
    if (where < 0 || where > 3) return bfail(b, LBM_EINVAL, "lbm_batch_moments_packed: where must be 0, 1, 2 or 3");
    for (int i = 0; i < b->count; i++)
        if (!b->ctx[i]->initialised)
            return bfail(b, LBM_ESTATE, "lbm_batch_moments_packed: context %d not initialised", i);
    int parity = 0;
    int rc = refresh_descriptors(b, &parity);
    if (rc != LBM_OK) return rc;
    const int dim = b->ctx[0]->dim;
    const size_t nrho = (size_t)b->total_nodes, nu = scalar ? 0 : (size_t)dim * b->total_nodes;
    double *drho = rho, *du = u;
    if (where == 0) {
        if (!b->d_mom) BCK(cudaMalloc(&b->d_mom, (nrho + nu) * sizeof(double)), "cudaMalloc(packed moments)");
        drho = b->d_mom;
        du = b->d_mom + nrho;
    } else if (where >= 2) {
        return packed_readback_async(b, rho, u, where, half_forced ? 1 : 0, parity, nrho, nu);
    }
    // a_pre of each member's current step: in the launch arguments for small
    // batches, else through pinned staging (the previous copy has read it by ev_apre)
    BatchMoments M{};
    const bool inl = b->count <= kInlinePairs;
    if (!inl) BCK(cudaEventSynchronize(b->ev_apre), "lbm_batch_moments_packed: wait for the previous copy");
    for (int i = 0; i < b->count; i++) {
        double apre, apost;
        lbmc::envelope_pair(b->ctx[i], b->ctx[i]->t, apre, apost);
        if (inl) M.apre_inl[i] = apre;
        else b->h_apre[i] = apre;
    }
    if (!inl) {
        BCK(cudaMemcpyAsync(b->d_apre, b->h_apre, b->count * sizeof(double), cudaMemcpyHostToDevice, b->stream),
            "lbm_batch_moments_packed: copy a_pre");
        BCK(cudaEventRecord(b->ev_apre, b->stream), "lbm_batch_moments_packed: record");
    }
    M.items = b->d_items;
    M.first = b->d_first[1];
    M.count = b->count;
    M.parity = parity;
    M.half = half_forced ? 1 : 0;
    M.apre = inl ? nullptr : b->d_apre;
    M.off = b->d_off;
    M.rho = drho;
    M.u = du;
    BCK(batch_moments(b->lattice, b->ctx[0]->storage, M, (int)b->ntiles[1], b->stream),
        "lbm_batch_moments_packed: kernel");
    b->launches++;
    if (where == 0) {
        BCK(cudaMemcpyAsync(rho, drho, nrho * sizeof(double), cudaMemcpyDeviceToHost, b->stream),
            "lbm_batch_moments_packed: copy rho");
        if (!scalar)
            BCK(cudaMemcpyAsync(u, du, nu * sizeof(double), cudaMemcpyDeviceToHost, b->stream),
                "lbm_batch_moments_packed: copy u");
        BCK(cudaStreamSynchronize(b->stream), "lbm_batch_moments_packed");
    }
    return LBM_OK;
}

int lbm_batch_step_read(lbm_batch *b, double *rho, double *u, int where, int half_forced)
{
    lbmc::NvtxRange nvtx_("lbm_batch_step_read");
    if (!b) return LBM_EINVAL;
    b->err.clear();
    const bool scalar = b->lattice == LBM_D2Q5_CDE;
    if (!rho || (!scalar && !u)) return bfail(b, LBM_EINVAL, "lbm_batch_step_read: NULL output");
    if (where != 1 && where != 3) return bfail(b, LBM_EINVAL, "lbm_batch_step_read: where must be 1 or 3");
    if (reduced_precision(b)) return bfail(b, LBM_EINVAL, "lbm_batch_step_read: FP64 batches only");
    int rc = check_members(b, 1, "lbm_batch_step_read");
    if (rc != LBM_OK) return rc;
    rc = wait_member_readers(b, false);
    if (rc != LBM_OK) return rc;
    rc = ensure_readback(b);
    if (rc != LBM_OK) return rc;
    double *drho = rho, *du = u;
    if (where == 3) {
        rc = mapped_outputs(b, rho, u, &drho, &du, "lbm_batch_step_read");
        if (rc != LBM_OK) return rc;
    }
    int parity = 0;
    rc = refresh_descriptors(b, &parity);
    if (rc != LBM_OK) return rc;
    BatchLaunch L{};
    L.items = b->d_items;
    L.count = b->count;
    L.k = 0;
    L.parity = parity;
    if (b->count <= kInlinePairs) inline_pairs_of_step(b, L, 0);
    else if ((rc = stage_pairs(b, L, 1)) != LBM_OK) return rc;
    L.mrho = drho;
    L.mu = scalar ? nullptr : du;
    L.moff = b->d_off;
    L.mhalf = half_forced ? 1 : 0;
    // the batched kernel even for a single member (the single-lattice kernel has no fused readback)
    const cudaError_t e = launch_one(b, L, b->stream);
    if (e != cudaSuccess) return bfail(b, LBM_ECUDA, "lbm_batch_step_read: kernel: %s", cudaGetErrorString(e));
    b->launches++;
    for (int i = 0; i < b->count; i++) {
        lbm_ctx *c = b->ctx[i];
        std::swap(c->A, c->B);
        c->t += 1;
    }
    const int slot = b->qslot;
    b->qslot = (b->qslot + 1) % kReadbackSlots;
    BCK(cudaEventRecord(b->ev_read[slot], b->stream), "lbm_batch_step_read: record");
    b->ev_host[slot] = b->ev_read[slot];
    b->copies_pending = true;
    return LBM_OK;
}

int lbm_batch_wait_moments(lbm_batch *b, int keep)
{
    if (!b) return LBM_EINVAL;
    b->err.clear();
    if (keep < 0 || keep >= kReadbackSlots)
        return bfail(b, LBM_EINVAL, "lbm_batch_wait_moments: keep must be 0, 1 or 2");
    if (!b->copies_pending) return LBM_OK;
    // the slots are used in turn: qslot is the oldest, qslot - 1 the latest;
    // wait for all but the `keep` most recent readbacks
    for (int age = kReadbackSlots - 1; age >= keep; age--) {
        const int slot = (b->qslot + kReadbackSlots - 1 - age) % kReadbackSlots;
        if (b->ev_host[slot]) BCK(cudaEventSynchronize(b->ev_host[slot]), "lbm_batch_wait_moments");
    }
    if (keep == 0) b->copies_pending = false;
    return LBM_OK;
}

int lbm_batch_graph_replays(const lbm_batch *b, long long *count)
{
    if (!b || !count) return LBM_EINVAL;
    *count = b->graph_replays;
    return LBM_OK;
}

int lbm_batch_launch_count(const lbm_batch *b, long long *count)
{
    if (!b || !count) return LBM_EINVAL;
    *count = b->launches;
    return LBM_OK;
}

}  // extern "C"
