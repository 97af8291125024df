// C ABI of the library (declared in include/lbm.h): context management,
// argument validation, field uploads, the host step loop with the force /
// source envelope, and the data movement entry points.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <limits>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "lbm_ctx.h"

using namespace lbmk;

namespace {

thread_local std::string g_create_error;

}  // namespace

namespace lbmc {

int fail(lbm_ctx *c, int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    else g_create_error = buf;
    return code;
}

int cuda_fail(lbm_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, LBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int wait_readers(lbm_ctx *c, const void *buf)
{
    for (int k = 0; k < 2; k++) {
        if (!c->rd_buf[k] || (buf && c->rd_buf[k] != buf)) continue;
        const cudaError_t e = cudaStreamWaitEvent(c->stream, c->rd_ev[k], 0);
        if (e != cudaSuccess) return cuda_fail(c, e, "wait for a readback of the populations");
        c->rd_buf[k] = nullptr;
        c->rd_ev[k] = nullptr;
    }
    return LBM_OK;
}

#define CK(call, what) LBM_CK(call, what)

int lattice_q(int lattice)
{
    return lattice == LBM_D2Q9 ? 9 : lattice == LBM_D3Q27 ? 27 : lattice == LBM_D2Q5_CDE ? 5 : lattice == LBM_D3Q15 ? 15 : 0;
}
int lattice_dim(int lattice) { return (lattice == LBM_D3Q27 || lattice == LBM_D3Q15) ? 3 : 2; }

// Relaxation rates that a lattice uses (the others are ignored).
bool omega_used(int lattice, int k)
{
    if (lattice == LBM_D2Q9) return k >= 3 && k <= 8;
    if (lattice == LBM_D2Q5_CDE) return k >= 1 && k <= 4;
    if (lattice == LBM_D3Q15) return k >= 1 && k <= 4;
    return k >= 1 && k <= 6;
}

void envelope_pair(const lbm_ctx *c, long t, double &apre, double &apost)
{
    double a0, ah, a1;
    const double tt = (double)t;
    if (!c->env_tab.empty()) {
        // table entries at half-integer times; lbm_step checks the range first
        long k = (long)((tt - c->env_t0) * 2.0);
        const long last = (long)c->env_tab.size() - 1;
        if (k < 0) k = 0;
        if (k + 2 > last) k = last - 2;
        a0 = c->env_tab[k];
        ah = c->env_tab[k + 1];
        a1 = c->env_tab[k + 2];
    } else if (c->env) {
        a0 = c->env(tt, c->env_user);
        ah = c->env(tt + 0.5, c->env_user);
        a1 = c->env(tt + 1.0, c->env_user);
    } else {
        apre = apost = 1.0;
        return;
    }
    apre = 0.5 * (a0 + ah);
    apost = 0.5 * (ah + a1);
}

// Whether the envelope can be evaluated for steps t .. t+n-1 (and the moments at t+n).
bool envelope_covers(const lbm_ctx *c, long t, long n)
{
    if (c->env_tab.empty()) return true;
    const double first = c->env_t0, last = c->env_t0 + 0.5 * (double)(c->env_tab.size() - 1);
    return (double)t >= first && (double)(t + n) + 1.0 <= last;
}

LaunchArgs launch_args(const lbm_ctx *c, const double *fin, double *fout, double apre, double apost)
{
    LaunchArgs a{};
    a.g = c->g;
    a.fin = fin;
    a.fout = fout;
    a.fkind = c->force.kind;
    a.F = c->force.d;
    a.vkind = c->vel.kind;
    a.V = c->vel.d;
    a.apre = apre;
    a.apost = apost;
    for (int k = 0; k < 9; k++) a.omega[k] = c->omega[k];
    a.stream = c->stream;
    a.storage = c->storage;
    a.rho_ref = c->rho_ref;
    a.sround = c->sround;
    a.srkey = sr_step_key(c->sr_seed, c->t);
    for (int k = 0; k < 5; k++) a.gref[k] = c->gref[k];
    return a;
}

lbmk::Ref5 ref5(const lbm_ctx *c)
{
    lbmk::Ref5 r;
    for (int k = 0; k < 5; k++) r.v[k] = c->gref[k];
    return r;
}

lbmk::Lref lref_of(const lbm_ctx *c)
{
    lbmk::Lref L{};
    L.ref = c->lref_ref;
    L.scale = c->lref_aux;
    // D2Q5: the Eq. 39 equilibrium per unit scalar at the uniform velocity
    double ux = 0.0, uy = 0.0;
    if (c->vel.kind == FK_CONST) {
        ux = c->vel.d.cval[0];
        uy = c->vel.d.cval[1];
    }
    const double t = 1.0 / 3.0;
    L.q5[0] = (float)(t - ux * ux - uy * uy);
    L.q5[1] = (float)(0.5 * (t + ux * ux + ux));
    L.q5[2] = (float)(0.5 * (t + uy * uy + uy));
    L.q5[3] = (float)(0.5 * (t + ux * ux - ux));
    L.q5[4] = (float)(0.5 * (t + uy * uy - uy));
    return L;
}

int lref_decode_state(lbm_ctx *c)
{
    if (!c->lref_dev)
        CK(cudaMalloc(&c->lref_dev, (size_t)c->q * c->g.Np * sizeof(float)), "cudaMalloc(local reference FP32 state)");
    CK(lref_decode(c->lattice, c->storage, c->g, lref_of(c), c->A, c->lref_dev, c->stream), "decode kernel");
    c->launches++;
    return LBM_OK;
}

int lref_rebuild_state(lbm_ctx *c, const lbmk::Lref &old)
{
    const int rc = wait_readers(c, c->A);
    if (rc != LBM_OK) return rc;
    lbmk::Lref nw = lref_of(c);
    nw.ref = c->lref_ref2;
    nw.scale = c->lref_aux2;
    CK(lref_rebuild(c->lattice, c->storage, c->g, old, nw, c->lref_aux + 2, c->A, c->stream), "rebuild kernels");
    c->launches += 3;
    std::swap(c->lref_ref, c->lref_ref2);
    std::swap(c->lref_aux, c->lref_aux2);
    return LBM_OK;
}

int lref_encode_state(lbm_ctx *c)
{
    const int rc = wait_readers(c, c->A);
    if (rc != LBM_OK) return rc;
    CK(lref_rebase(c->lattice, c->storage, c->g, lref_of(c), c->lref_aux + 2, c->lref_dev, c->A, c->stream),
       "rebase kernels");
    c->launches += 3;
    return LBM_OK;
}

LrefView::LrefView(lbm_ctx *cc, bool decode) : c(cc)
{
    if (!c->lref_every) return;
    if (decode && c->initialised) {
        rc = lref_decode_state(c);
    } else if (!c->lref_dev) {
        const cudaError_t e = cudaMalloc(&c->lref_dev, (size_t)c->q * c->g.Np * sizeof(float));
        if (e != cudaSuccess) rc = cuda_fail(c, e, "cudaMalloc(local reference FP32 state)");
    }
    if (rc != LBM_OK) return;
    A0 = c->A;
    st0 = c->storage;
    el0 = c->elem;
    c->A = reinterpret_cast<double *>(c->lref_dev);
    c->storage = LBM_FP32_DEV;
    c->elem = 4;
    on = true;
}

void LrefView::restore()
{
    if (!on) return;
    c->A = A0;
    c->storage = st0;
    c->elem = el0;
    on = false;
}

// Back to the plain 16-bit deviations (reference 0, sigma 1).
// old: the encoding the state is in (its q5 may differ from the current velocity's).
static int lref_off(lbm_ctx *c, const lbmk::Lref &old)
{
    lbmk::Lref plain = lref_of(c);
    plain.ref = c->lref_ref2;
    plain.scale = c->lref_aux2;
    CK(lref_reset(c->lattice, c->g, plain, c->stream), "lref reset");
    if (c->initialised) {
        const int rc = wait_readers(c, c->A);
        if (rc != LBM_OK) return rc;
        CK(lref_reencode(c->lattice, c->storage, c->g, old, plain, c->A, c->stream), "re-encode kernel");
        c->launches++;
    }
    std::swap(c->lref_ref, c->lref_ref2);
    std::swap(c->lref_aux, c->lref_aux2);
    c->lref_every = 0;
    c->lref_since = 0;
    c->version++;
    CK(cudaStreamSynchronize(c->stream), "lref off");
    return LBM_OK;
}

// D2Q5 reference populations for reduced-precision storage: the equilibrium
// at (rho_ref, u) for a periodic lattice whose advecting velocity u is
// uniform (the step maps it to itself: the stored deviations then carry the
// scalar's variation only); else the rest state w rho_ref (a wall reflects a
// population into the opposite slot, and a field velocity has no single
// equilibrium).  The D2Q5 equilibrium of Eq. 39: g_0 = rho (1/3 - ux^2 -
// uy^2), g_{+-x} = rho (1/3 + ux^2 +- ux) / 2, g_{+-y} likewise.
void choose_d2q5_reference(lbm_ctx *c)
{
    const double r = c->rho_ref;
    const bool periodic = !c->g.wall[0] && !c->g.wall[1];
    if (periodic && c->vel.kind != FK_GENERAL) {
        const double ux = c->vel.kind == FK_CONST ? c->vel.d.cval[0] : 0.0;
        const double uy = c->vel.kind == FK_CONST ? c->vel.d.cval[1] : 0.0;
        c->gref[0] = r * ((1.0 / 3.0) - ux * ux - uy * uy);
        c->gref[1] = 0.5 * r * ((1.0 / 3.0) + ux * ux + ux);
        c->gref[3] = 0.5 * r * ((1.0 / 3.0) + ux * ux - ux);
        c->gref[2] = 0.5 * r * ((1.0 / 3.0) + uy * uy + uy);
        c->gref[4] = 0.5 * r * ((1.0 / 3.0) + uy * uy - uy);
    } else {
        c->gref[0] = r / 3.0;
        for (int k = 1; k < 5; k++) c->gref[k] = r / 6.0;
    }
}

// Key of step t's stochastic-rounding bits: the seed, mixed (SplitMix64
// output function, see k_rp.cu), XOR the step counter shifted above the
// node and chunk bits of the per-node counter (node < 2^31, chunk < 8), so
// that every (step < 2^30, node, chunk) has its own counter.
unsigned long long sr_step_key(unsigned long long seed, long t)
{
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    return z ^ ((unsigned long long)t << 34);
}

// Reduced-precision contexts: FP64 staging of q*N doubles for host I/O.
int ensure_stage(lbm_ctx *c)
{
    if (c->stage) return LBM_OK;
    cudaError_t e = cudaMalloc(&c->stage, (size_t)c->q * c->g.N * sizeof(double));
    if (e != cudaSuccess) {
        c->stage = nullptr;
        return cuda_fail(c, e, "cudaMalloc(staging)");
    }
    return LBM_OK;
}

}  // namespace lbmc

using namespace lbmc;

namespace {

// Upload a shape with `ncomp` components into `out` (replacing any previous one).
int upload_field(lbm_ctx *c, const lbm_field *f, int ncomp, DeviceField &out, const char *what)
{
    if (f == nullptr || f->kind == LBM_FIELD_NONE) {
        if (out.dev) cudaFree(out.dev);
        if (out.fdev) cudaFree(out.fdev);
        out = DeviceField{};
        return LBM_OK;
    }
    if (f->data == nullptr) return fail(c, LBM_EINVAL, "%s: data is NULL", what);
    const int n[3] = {c->g.nx, c->g.ny, c->g.nz};
    DeviceField nf;
    size_t count = 0;
    if (f->kind == LBM_FIELD_SEPARABLE) {
        for (int d = 0; d < 3; d++)
            if (!(f->len[d] == 1 || f->len[d] == n[d]))
                return fail(c, LBM_EINVAL, "%s: table length %d on axis %d must be 1 or %d", what, f->len[d], d, n[d]);
        const size_t per = (size_t)f->len[0] + f->len[1] + f->len[2];
        count = per * ncomp;
        if (f->len[0] == 1 && f->len[1] == 1 && f->len[2] == 1) {
            // Constant shape: the kernels take the per-component product as a scalar.
            nf.kind = FK_CONST;
            for (int cc = 0; cc < ncomp; cc++) {
                const double *t = f->data + cc * per;
                nf.d.cval[cc] = (t[0] * t[1]) * t[2];
                nf.d.fcval[cc] = (float)nf.d.cval[cc];
            }
            if (out.dev) cudaFree(out.dev);
            if (out.fdev) cudaFree(out.fdev);
            out = nf;
            return LBM_OK;
        }
        nf.d.sep = 1;
        nf.d.cstride = (long long)per;
        for (int d = 0; d < 3; d++) nf.d.len[d] = f->len[d];
        // Components whose product is identically zero, and axes whose table
        // is exactly 1.0 for every other component, are skipped by the kernels.
        nf.d.zmask = 0;
        for (int cc = 0; cc < ncomp; cc++) {
            const double *t = f->data + cc * per;
            for (int d = 0, off = 0; d < 3; off += f->len[d], d++) {
                bool allzero = true;
                for (int k = 0; k < f->len[d]; k++) allzero = allzero && t[off + k] == 0.0;
                if (allzero) nf.d.zmask |= 1 << cc;
            }
        }
        nf.d.axes = 0;
        for (int d = 0, off = 0; d < 3; off += f->len[d], d++) {
            bool one = f->len[d] == 1;
            for (int cc = 0; cc < ncomp && one; cc++)
                if (!((nf.d.zmask >> cc) & 1)) one = f->data[cc * per + off] == 1.0;
            if (!one) nf.d.axes |= 1 << d;
        }
    } else if (f->kind == LBM_FIELD_FULL || f->kind == LBM_FIELD_FULL_DEVICE) {
        count = (size_t)c->g.N * ncomp;
        nf.d.sep = 0;
        nf.d.cstride = c->g.N;
        if (f->kind == LBM_FIELD_FULL_DEVICE) {
            cudaPointerAttributes at{};
            const cudaError_t ea = cudaPointerGetAttributes(&at, f->data);
            if (ea != cudaSuccess) {
                cudaGetLastError();
                return fail(c, LBM_EINVAL, "%s: data is not a device pointer", what);
            }
            if (!((at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == c->device))
                return fail(c, LBM_EINVAL, "%s: data is not device memory of the context's device %d", what,
                            c->device);
        }
    } else {
        return fail(c, LBM_EINVAL, "%s: unknown field kind %d", what, f->kind);
    }
    nf.kind = FK_GENERAL;
    // Reuse the previous device buffer when it is large enough (a shape that is
    // re-uploaded every step costs one copy, no allocation).
    const bool want_f = c->storage != LBM_FP64;
    const bool reuse = out.dev != nullptr && out.cap >= count && (!want_f || out.fdev != nullptr);
    if (reuse) {
        nf.dev = out.dev;
        nf.fdev = out.fdev;
        nf.cap = out.cap;
    } else {
        CK(cudaMalloc(&nf.dev, count * sizeof(double)), "cudaMalloc(field)");
        if (want_f) {
            cudaError_t ef = cudaMalloc(&nf.fdev, count * sizeof(float));
            if (ef != cudaSuccess) {
                cudaFree(nf.dev);
                return cuda_fail(c, ef, "cudaMalloc(field, FP32 copy)");
            }
        }
        nf.cap = count;
    }
    // A reused buffer may still be read by a readback queued on another
    // stream (the half-forced fields read the force): the copy waits for it.
    if (reuse) {
        const int rc = wait_readers(c, nullptr);
        if (rc != LBM_OK) return rc;
    }
    cudaError_t e = cudaSuccess;
    if (f->kind == LBM_FIELD_FULL_DEVICE) {
        // Device field: copied (and converted for reduced-precision storage)
        // on the context's stream, in order with the steps before and after;
        // nothing synchronises.
        e = cudaMemcpyAsync(nf.dev, f->data, count * sizeof(double), cudaMemcpyDeviceToDevice, c->stream);
        if (e == cudaSuccess && want_f) {
            e = lbmk::to_float(nf.dev, nf.fdev, (long long)count, c->stream);
            c->launches++;
        }
    } else {
        // The copies are complete before returning: the caller may reuse its buffer.
        e = cudaMemcpyAsync(nf.dev, f->data, count * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        std::vector<float> fcopy;
        if (e == cudaSuccess && want_f) {
            fcopy.assign(f->data, f->data + count);
            e = cudaMemcpyAsync(nf.fdev, fcopy.data(), count * sizeof(float), cudaMemcpyHostToDevice, c->stream);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    }
    if (e != cudaSuccess) {
        if (!reuse) {
            cudaFree(nf.dev);
            cudaFree(nf.fdev);
        }
        return cuda_fail(c, e, "upload field");
    }
    nf.d.data = nf.dev;
    nf.d.fdata = nf.fdev;
    if (!reuse) {
        if (out.dev) cudaFree(out.dev);
        if (out.fdev) cudaFree(out.fdev);
    }
    out = nf;
    return LBM_OK;
}

}  // namespace

extern "C" {

int lbm_create(lbm_ctx **out, int lattice, int nx, int ny, int nz, const lbm_relax *relax,
               const lbm_boundary *bc, int storage, void *stream)
{
    g_create_error.clear();
    if (out == nullptr) return fail(nullptr, LBM_EINVAL, "lbm_create: out is NULL");
    *out = nullptr;
    const int q = lattice_q(lattice);
    if (q == 0) return fail(nullptr, LBM_EINVAL, "lbm_create: unknown lattice %d", lattice);
    if (storage < LBM_FP64 || storage > LBM_BF16_DEV)
        return fail(nullptr, LBM_EINVAL, "lbm_create: unsupported storage %d", storage);
    if (lattice == LBM_D3Q15 && storage != LBM_FP64)
        return fail(nullptr, LBM_EINVAL, "lbm_create: D3Q15 supports FP64 storage only");
    if (nx < 1 || ny < 1 || nz < 1) return fail(nullptr, LBM_EINVAL, "lbm_create: extents must be >= 1");
    if (lattice_dim(lattice) == 2 && nz != 1) return fail(nullptr, LBM_EINVAL, "lbm_create: nz must be 1 for a 2D lattice");
    const long long N = (long long)nx * ny * nz;
    if (N > LBM_MAX_NODES) return fail(nullptr, LBM_EINVAL, "lbm_create: %lld nodes, more than LBM_MAX_NODES", N);
    if (relax == nullptr) return fail(nullptr, LBM_EINVAL, "lbm_create: relax is NULL");
    for (int k = 0; k < 9; k++)
        if (omega_used(lattice, k) && !(relax->omega[k] > 0.0 && relax->omega[k] < 2.0))
            return fail(nullptr, LBM_EINVAL, "lbm_create: omega[%d] = %g outside (0, 2)", k, relax->omega[k]);
    int wall[3] = {0, 0, 0};
    if (bc)
        for (int d = 0; d < 3; d++) {
            if (bc->axis[d] != LBM_PERIODIC && bc->axis[d] != LBM_BOUNCE_BACK)
                return fail(nullptr, LBM_EINVAL, "lbm_create: boundary kind %d on axis %d", bc->axis[d], d);
            wall[d] = bc->axis[d] == LBM_BOUNCE_BACK;
        }
    if (lattice_dim(lattice) == 2 && wall[2]) return fail(nullptr, LBM_EINVAL, "lbm_create: walls on z for a 2D lattice");

    lbm_ctx *c = new (std::nothrow) lbm_ctx();
    if (!c) return fail(nullptr, LBM_ENOMEM, "lbm_create: out of host memory");
    c->lattice = lattice;
    c->q = q;
    c->dim = lattice_dim(lattice);
    c->storage = storage;
    c->elem = storage == LBM_FP64 ? 8 : (storage == LBM_FP32_DEV ? 4 : 2);
    c->g.nx = nx;
    c->g.ny = ny;
    c->g.nz = nz;
    c->g.N = (int)N;
    c->g.Np = (N + 127) / 128 * 128;  // every plane starts 256-byte aligned for any element size
    for (int d = 0; d < 3; d++) c->g.wall[d] = wall[d];
    lbmk::div_magic(nx, c->g.mx, c->g.lx);
    lbmk::div_magic(ny, c->g.my, c->g.ly);
    for (int k = 0; k < 9; k++) c->omega[k] = relax->omega[k];
    c->stream = (cudaStream_t)stream;
    cudaGetDevice(&c->device);
    const size_t bytes = (size_t)q * c->g.Np * c->elem;
    cudaError_t e = cudaMalloc(&c->A, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&c->B, bytes);
    if (e == cudaSuccess) e = cudaMalloc(&c->partials, (size_t)reduce_blocks(c->g) * 8 * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&c->red_out, 8 * sizeof(double));
    if (e != cudaSuccess) {
        int code = (e == cudaErrorMemoryAllocation) ? LBM_ENOMEM : LBM_ECUDA;
        fail(nullptr, code, "lbm_create: cudaMalloc of %zu bytes: %s", bytes, cudaGetErrorString(e));
        cudaGetLastError();
        lbm_destroy(c);
        return code;
    }
    *out = c;
    return LBM_OK;
}

void lbm_destroy(lbm_ctx *c)
{
    if (!c) return;
    for (int k = 0; k < 2; k++)
        if (c->rd_buf[k]) cudaEventSynchronize(c->rd_ev[k]);
    if (c->stream || c->A) cudaStreamSynchronize(c->stream);
    cudaFree(c->A);
    cudaFree(c->B);
    cudaFree(c->snap);
    cudaFree(c->partials);
    cudaFree(c->red_out);
    cudaFree(c->force.dev);
    cudaFree(c->vel.dev);
    cudaFree(c->force.fdev);
    cudaFree(c->vel.fdev);
    cudaFree(c->stage);
    cudaFree(c->lref_ref);
    cudaFree(c->lref_aux);
    cudaFree(c->lref_dev);
    cudaFree(c->lref_ref2);
    cudaFree(c->lref_aux2);
    delete c;
}

const char *lbm_last_error(const lbm_ctx *c)
{
    return c ? c->err.c_str() : g_create_error.c_str();
}

int lbm_init_equilibrium(lbm_ctx *c, double rho0, const double u0[3], const double *rho, const double *u)
{
    if (!c) return LBM_EINVAL;
    c->err.clear();
    if (c->lattice != LBM_D2Q5_CDE && rho == nullptr && !(rho0 > 0.0))
        return fail(c, LBM_EINVAL, "lbm_init_equilibrium: rho0 must be positive");
    {
        const int rc = wait_readers(c, nullptr);
        if (rc != LBM_OK) return rc;
    }
    LrefView view(c, false);  // local reference: the FP32 fill, then the encoding
    double uu[3] = {0.0, 0.0, 0.0};
    if (u0)
        for (int d = 0; d < c->dim; d++) uu[d] = u0[d];
    const size_t N = (size_t)c->g.N;
    double *drho = nullptr, *du = nullptr;
    // Per-node inputs are staged in A (q*Np >= (1+dim)*N doubles); the
    // equilibrium goes to B and the scatter then overwrites A.
    if ((rho || u) && c->storage != LBM_FP64) {
        int rc = ensure_stage(c);
        if (rc != LBM_OK) return rc;
    }
    if (rho || u) {
        double *stage = c->storage == LBM_FP64 ? c->A : c->stage;
        if (rho) {
            drho = stage;
            CK(cudaMemcpyAsync(drho, rho, N * sizeof(double), cudaMemcpyHostToDevice, c->stream), "upload rho");
            stage += N;
        }
        if (u) {
            du = stage;
            CK(cudaMemcpyAsync(du, u, (size_t)c->dim * N * sizeof(double), cudaMemcpyHostToDevice, c->stream),
               "upload u");
        }
    }
    if (c->storage == LBM_FP64) {
        CK(equilibrium(c->lattice, c->g, rho0, uu, drho, du, c->B, c->stream), "equilibrium kernel");
        CK(scatter_to_stored(c->lattice, c->g, c->B, c->A, c->stream), "scatter kernel");
        c->launches += 2;
    } else {
        c->rho_ref = rho0 > 0.0 ? rho0 : 1.0;
        if (c->lattice == LBM_D2Q5_CDE) choose_d2q5_reference(c);
        CK(rp_init_equilibrium(c->lattice, c->storage, c->g, c->rho_ref, ref5(c), rho0, uu, drho, du, c->A,
                               c->stream),
           "equilibrium kernel");
        c->launches += 1;
    }
    view.restore();
    if (c->lref_every) {
        const int rc = lref_encode_state(c);
        if (rc != LBM_OK) return rc;
        c->lref_since = 0;
    }
    CK(cudaStreamSynchronize(c->stream), "lbm_init_equilibrium");
    c->t = 0;
    c->initialised = true;
    c->have_snap = false;
    c->version++;
    return LBM_OK;
}

int lbm_set_force(lbm_ctx *c, const lbm_field *shape)
{
    if (!c) return LBM_EINVAL;
    c->err.clear();
    c->version++;
    if (c->lattice == LBM_D2Q5_CDE) return fail(c, LBM_EINVAL, "lbm_set_force: scalar lattice (use lbm_set_source)");
    return upload_field(c, shape, c->dim, c->force, "lbm_set_force");
}

int lbm_set_source(lbm_ctx *c, const lbm_field *shape)
{
    if (!c) return LBM_EINVAL;
    c->err.clear();
    c->version++;
    if (c->lattice != LBM_D2Q5_CDE) return fail(c, LBM_EINVAL, "lbm_set_source: flow lattice (use lbm_set_force)");
    return upload_field(c, shape, 1, c->force, "lbm_set_source");
}

int lbm_set_velocity(lbm_ctx *c, const lbm_field *u)
{
    if (!c) return LBM_EINVAL;
    c->err.clear();
    c->version++;
    if (c->lattice != LBM_D2Q5_CDE) return fail(c, LBM_EINVAL, "lbm_set_velocity: only for the scalar lattice");
    // the encoding depends on the uniform velocity: the state's, before the change
    const lbmk::Lref old_enc = lref_of(c);
    int rc = upload_field(c, u, 2, c->vel, "lbm_set_velocity");
    if (rc != LBM_OK) return rc;
    if (c->lref_every) {
        if (c->vel.kind == FK_GENERAL) {
            // a velocity field ends the local-reference encoding: plain deviations
            rc = lref_off(c, old_enc);
            if (rc != LBM_OK) return rc;
        } else {
            if (c->initialised) {
                rc = lref_rebuild_state(c, old_enc);
                if (rc != LBM_OK) return rc;
                c->lref_since = 0;
            }
            CK(cudaStreamSynchronize(c->stream), "lbm_set_velocity");
            return LBM_OK;
        }
    }
    if (c->storage == LBM_FP64 || !c->initialised || c->vel.kind != FK_GENERAL) return rc;
    // A velocity field needs the rest-state reference: re-express the stored
    // deviations (gather with the old reference, scatter with the new one).
    double rest[5] = {c->rho_ref / 3.0, c->rho_ref / 6.0, c->rho_ref / 6.0, c->rho_ref / 6.0, c->rho_ref / 6.0};
    bool same = true;
    for (int k = 0; k < 5; k++) same = same && c->gref[k] == rest[k];
    if (same) return LBM_OK;
    rc = ensure_stage(c);
    if (rc != LBM_OK) return rc;
    rc = wait_readers(c, nullptr);
    if (rc != LBM_OK) return rc;
    CK(rp_gather(c->lattice, c->storage, c->g, c->rho_ref, ref5(c), c->A, c->stage, c->stream), "gather kernel");
    for (int k = 0; k < 5; k++) c->gref[k] = rest[k];
    CK(rp_scatter(c->lattice, c->storage, c->g, c->rho_ref, ref5(c), c->stage, c->A, c->stream), "scatter kernel");
    c->launches += 2;
    c->version++;
    CK(cudaStreamSynchronize(c->stream), "lbm_set_velocity");
    return LBM_OK;
}

int lbm_set_envelope(lbm_ctx *c, lbm_envelope_fn fn, void *user)
{
    if (!c) return LBM_EINVAL;
    c->env = fn;
    c->env_user = user;
    c->env_tab.clear();
    return LBM_OK;
}

int lbm_set_envelope_table(lbm_ctx *c, const double *a, long count, double t0)
{
    if (!c) return LBM_EINVAL;
    c->err.clear();
    if (a == nullptr && count == 0) {
        c->env_tab.clear();
        return LBM_OK;
    }
    if (a == nullptr || count < 3) return fail(c, LBM_EINVAL, "lbm_set_envelope_table: need at least 3 values");
    c->env_tab.assign(a, a + count);
    c->env_t0 = t0;
    c->env = nullptr;
    c->env_user = nullptr;
    return LBM_OK;
}

int lbm_set_stochastic_rounding(lbm_ctx *c, int on, unsigned long long seed)
{
    if (!c) return LBM_EINVAL;
    c->err.clear();
    if (c->storage != LBM_FP16_DEV && c->storage != LBM_BF16_DEV)
        return fail(c, LBM_EINVAL, "lbm_set_stochastic_rounding: only for FP16 / BF16 deviation storage");
    c->sround = on ? 1 : 0;
    c->sr_seed = seed;
    c->version++;
    return LBM_OK;
}

int lbm_set_local_reference(lbm_ctx *c, int every)
{
    if (!c) return LBM_EINVAL;
    c->err.clear();
    if (c->storage != LBM_FP16_DEV && c->storage != LBM_BF16_DEV)
        return fail(c, LBM_EINVAL, "lbm_set_local_reference: only for FP16 / BF16 deviation storage");
    if (c->lattice != LBM_D2Q9 && c->lattice != LBM_D2Q5_CDE)
        return fail(c, LBM_EINVAL, "lbm_set_local_reference: D2Q9 and D2Q5 lattices only");
    if (every < 0) return fail(c, LBM_EINVAL, "lbm_set_local_reference: every < 0");
    if (every > 0 && c->lattice == LBM_D2Q5_CDE && c->vel.kind == FK_GENERAL)
        return fail(c, LBM_EINVAL, "lbm_set_local_reference: the scalar lattice needs a uniform advecting velocity");
    {
        const int rc = wait_readers(c, nullptr);
        if (rc != LBM_OK) return rc;
    }
    if (every == 0) return c->lref_every ? lref_off(c, lref_of(c)) : LBM_OK;
    if (!c->lref_every) {
        const int nref = c->lattice == LBM_D2Q9 ? 3 : 1;
        // sigma, 1 / sigma, the rebuild's largest |d - e| per block of 256 nodes
        const size_t np = (size_t)c->g.Np, naux = 2 + ((size_t)c->g.N + 255) / 256;
        if (!c->lref_ref) CK(cudaMalloc(&c->lref_ref, nref * np * sizeof(float)), "cudaMalloc(local reference)");
        if (!c->lref_ref2) CK(cudaMalloc(&c->lref_ref2, nref * np * sizeof(float)), "cudaMalloc(local reference)");
        if (!c->lref_aux) CK(cudaMalloc(&c->lref_aux, naux * sizeof(float)), "cudaMalloc(local reference scale)");
        if (!c->lref_aux2) CK(cudaMalloc(&c->lref_aux2, naux * sizeof(float)), "cudaMalloc(local reference scale)");
        // the plain deviations are this encoding at reference 0 and sigma 1
        CK(lref_reset(c->lattice, c->g, lref_of(c), c->stream), "lref reset");
        c->lref_every = every;
        if (c->initialised) {
            const int rc = lref_rebuild_state(c, lref_of(c));
            if (rc != LBM_OK) {
                c->lref_every = 0;
                return rc;
            }
        }
    }
    c->lref_every = every;
    c->lref_since = 0;
    c->version++;
    CK(cudaStreamSynchronize(c->stream), "lbm_set_local_reference");
    return LBM_OK;
}

int lbm_step(lbm_ctx *c, long n)
{
    NvtxRange nvtx_("lbm_step");
    if (!c) return LBM_EINVAL;
    c->err.clear();
    if (n < 0) return fail(c, LBM_EINVAL, "lbm_step: n < 0");
    if (!c->initialised) return fail(c, LBM_ESTATE, "lbm_step: populations not initialised");
    if (!envelope_covers(c, c->t, n))
        return fail(c, LBM_EINVAL, "lbm_step: steps %ld..%ld are outside the envelope table", c->t, c->t + n);
    if (n == 0) return LBM_OK;
    {
        // one step writes the second buffer only; more steps write both
        const int rc = wait_readers(c, n == 1 ? c->B : nullptr);
        if (rc != LBM_OK) return rc;
    }
    if (n >= 2 && n <= 2147483647L && c->lattice == LBM_D2Q9 && !c->env && c->env_tab.empty() && !c->sround &&
        !c->lref_every) {
        // a small lattice with a constant force: all n steps in one cluster launch
        double *out = (n & 1) ? c->B : c->A;
        LaunchArgs a = launch_args(c, c->A, out, 1.0, 1.0);
        cudaError_t e = c->storage == LBM_FP64 ? d2q9_cluster_steps(a, (int)n) : rp_cluster_steps9(a, (int)n);
        if (e == cudaSuccess) {
            c->launches++;
            if (n & 1) {
                double *tmp = c->A;
                c->A = c->B;
                c->B = tmp;
            }
            c->t += n;
            return LBM_OK;
        }
        // Not supported here (too large), or a cluster launch the device
        // refuses: clear the launch error and take single-step launches.
        if (e != cudaErrorNotSupported) cudaGetLastError();
    }
    for (long k = 0; k < n; k++) {
        double apre, apost;
        envelope_pair(c, c->t, apre, apost);
        LaunchArgs a = launch_args(c, c->A, c->B, apre, apost);
        cudaError_t e;
        if (c->lref_every) {
            e = lref_step(c->lattice, a, lref_of(c));
        } else if (c->storage != LBM_FP64) {
            e = rp_step(c->lattice, a);
        } else {
            switch (c->lattice) {
            case LBM_D2Q9: e = d2q9_step(a); break;
            case LBM_D2Q5_CDE: e = d2q5_step(a); break;
            case LBM_D3Q15: e = d3q15_step(a); break;
            default: e = d3q27_step(a); break;
            }
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "step kernel");
        c->launches++;
        double *tmp = c->A;
        c->A = c->B;
        c->B = tmp;
        c->t++;
        if (c->lref_every && ++c->lref_since >= c->lref_every) {
            // rebuild the local reference from the state, in place
            const int rc = lref_rebuild_state(c, lref_of(c));
            if (rc != LBM_OK) return rc;
            c->lref_since = 0;
        }
    }
    return LBM_OK;
}

int lbm_moments(lbm_ctx *c, double *rho, double *u, int where, int half_forced)
{
    NvtxRange nvtx_("lbm_moments");
    if (!c) return LBM_EINVAL;
    c->err.clear();
    if (!c->initialised) return fail(c, LBM_ESTATE, "lbm_moments: populations not initialised");
    if (rho == nullptr || (c->lattice != LBM_D2Q5_CDE && u == nullptr))
        return fail(c, LBM_EINVAL, "lbm_moments: NULL output");
    if (where != 0 && where != 1) return fail(c, LBM_EINVAL, "lbm_moments: where must be 0 or 1");
    LrefView view(c, true);
    if (view.rc != LBM_OK) return view.rc;
    double apre, apost;
    envelope_pair(c, c->t, apre, apost);
    LaunchArgs a = launch_args(c, c->A, nullptr, apre, apost);
    const size_t N = (size_t)c->g.N;
    double *drho = rho, *du = u;
    if (where == 0) {  // stage through the scratch buffer B (FP64) or the staging buffer
        double *st = c->B;
        if (c->storage != LBM_FP64) {
            int rc = ensure_stage(c);
            if (rc != LBM_OK) return rc;
            st = c->stage;
        } else {
            const int rc = wait_readers(c, c->B);
            if (rc != LBM_OK) return rc;
        }
        drho = st;
        du = st + N;
    }
    CK(moments(c->lattice, a, drho, du, half_forced ? 1 : 0), "moments kernel");
    c->launches++;
    if (where == 0) {
        CK(cudaMemcpyAsync(rho, drho, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy rho");
        if (c->lattice != LBM_D2Q5_CDE)
            CK(cudaMemcpyAsync(u, du, (size_t)c->dim * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
               "copy u");
        CK(cudaStreamSynchronize(c->stream), "lbm_moments");
    }
    return LBM_OK;
}

int lbm_debug_poison(lbm_ctx *c)
{
    if (!c) return LBM_EINVAL;
    c->err.clear();
    const int rc = wait_readers(c, c->B);
    if (rc != LBM_OK) return rc;
    // all-ones bytes are a NaN in every storage type (FP64, FP32, FP16, BF16)
    CK(cudaMemsetAsync(c->B, 0xFF, (size_t)c->q * c->g.Np * c->elem, c->stream), "poison");
    return LBM_OK;
}

int lbm_strain_rate(lbm_ctx *c, double rho0, double *S, int where)
{
    if (!c) return LBM_EINVAL;
    c->err.clear();
    if (c->lattice == LBM_D2Q5_CDE) return fail(c, LBM_EINVAL, "lbm_strain_rate: flow lattices only");
    if (!c->initialised) return fail(c, LBM_ESTATE, "lbm_strain_rate: populations not initialised");
    if (S == nullptr) return fail(c, LBM_EINVAL, "lbm_strain_rate: NULL output");
    if (where != 0 && where != 1) return fail(c, LBM_EINVAL, "lbm_strain_rate: where must be 0 or 1");
    if (!(rho0 > 0.0)) return fail(c, LBM_EINVAL, "lbm_strain_rate: rho0 must be positive");
    LrefView view(c, true);
    if (view.rc != LBM_OK) return view.rc;
    double apre, apost;
    envelope_pair(c, c->t, apre, apost);
    LaunchArgs a = launch_args(c, c->A, nullptr, apre, apost);
    const size_t N = (size_t)c->g.N;
    const int ncomp = c->dim == 2 ? 3 : 6;
    double *dst = S;
    if (where == 0) {
        const int rw = wait_readers(c, c->B);
        if (rw != LBM_OK) return rw;
        dst = c->B;
        if (c->storage != LBM_FP64) {
            int rc = ensure_stage(c);
            if (rc != LBM_OK) return rc;
            dst = c->stage;
        }
    }
    CK(strain_rate(c->lattice, a, rho0, dst), "strain-rate kernel");
    c->launches++;
    if (where == 0) {
        CK(cudaMemcpyAsync(S, dst, ncomp * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "copy strain");
        CK(cudaStreamSynchronize(c->stream), "lbm_strain_rate");
    }
    return LBM_OK;
}

int lbm_set_source_from_strain(lbm_ctx *scalar, lbm_ctx *flow, double rho0, double coef)
{
    if (!scalar || !flow) return LBM_EINVAL;
    lbm_ctx *c = scalar;  // errors are reported on the scalar context
    c->err.clear();
    if (scalar->lattice != LBM_D2Q5_CDE || flow->lattice == LBM_D2Q5_CDE)
        return fail(scalar, LBM_EINVAL, "lbm_set_source_from_strain: needs a scalar and a flow lattice");
    if (scalar->g.nx != flow->g.nx || scalar->g.ny != flow->g.ny || scalar->g.nz != flow->g.nz)
        return fail(scalar, LBM_EINVAL, "lbm_set_source_from_strain: grids differ");
    if (scalar->stream != flow->stream || scalar->device != flow->device)
        return fail(scalar, LBM_EINVAL, "lbm_set_source_from_strain: lattices on different streams or devices");
    if (!flow->initialised) return fail(scalar, LBM_ESTATE, "lbm_set_source_from_strain: flow not initialised");
    if (!(rho0 > 0.0)) return fail(scalar, LBM_EINVAL, "lbm_set_source_from_strain: rho0 must be positive");
    LrefView fview(flow, true);
    if (fview.rc != LBM_OK) return fail(scalar, fview.rc, "lbm_set_source_from_strain: %s", flow->err.c_str());
    const size_t N = (size_t)scalar->g.N;
    DeviceField &out = scalar->force;
    const bool want_f = scalar->storage != LBM_FP64;
    if (!(out.kind == FK_GENERAL && out.dev && out.cap >= N && !out.d.sep && (!want_f || out.fdev))) {
        DeviceField nf;
        CK(cudaMalloc(&nf.dev, N * sizeof(double)), "cudaMalloc(source field)");
        if (want_f) {
            cudaError_t ef = cudaMalloc(&nf.fdev, N * sizeof(float));
            if (ef != cudaSuccess) {
                cudaFree(nf.dev);
                return cuda_fail(scalar, ef, "cudaMalloc(source field, FP32 copy)");
            }
        }
        nf.cap = N;
        nf.kind = FK_GENERAL;
        nf.d.sep = 0;
        nf.d.cstride = (long long)N;
        nf.d.data = nf.dev;
        nf.d.fdata = nf.fdev;
        CK(cudaStreamSynchronize(scalar->stream), "lbm_set_source_from_strain: sync");
        if (out.dev) cudaFree(out.dev);
        if (out.fdev) cudaFree(out.fdev);
        out = nf;
    }
    // the flow's strain into its own scratch buffer, then coef * S:S into the source field
    double apre, apost;
    envelope_pair(flow, flow->t, apre, apost);
    LaunchArgs a = launch_args(flow, flow->A, nullptr, apre, apost);
    double *tmp = flow->B;
    if (flow->storage == LBM_FP64) {
        const int rw = wait_readers(flow, flow->B);
        if (rw != LBM_OK) return fail(scalar, rw, "lbm_set_source_from_strain: %s", flow->err.c_str());
    }
    if (flow->storage != LBM_FP64) {
        int rc = ensure_stage(flow);
        if (rc != LBM_OK) return fail(scalar, rc, "lbm_set_source_from_strain: %s", flow->err.c_str());
        tmp = flow->stage;
    }
    cudaError_t e = strain_rate(flow->lattice, a, rho0, tmp);
    if (e == cudaSuccess) e = viscous_source((int)N, flow->dim, tmp, coef, out.dev, out.fdev, scalar->stream);
    if (e != cudaSuccess) return cuda_fail(scalar, e, "lbm_set_source_from_strain kernels");
    flow->launches++;
    scalar->launches++;
    scalar->version++;
    return LBM_OK;
}

int lbm_reduce(lbm_ctx *c, double out[5])
{
    NvtxRange nvtx_("lbm_reduce");
    if (!c) return LBM_EINVAL;
    c->err.clear();
    if (!c->initialised) return fail(c, LBM_ESTATE, "lbm_reduce: populations not initialised");
    if (!out) return fail(c, LBM_EINVAL, "lbm_reduce: out is NULL");
    LrefView view(c, true);
    if (view.rc != LBM_OK) return view.rc;
    if (!c->snap) {
        const int ncomp = c->lattice == LBM_D2Q5_CDE ? 1 : c->dim;
        CK(cudaMalloc(&c->snap, (size_t)ncomp * c->g.N * sizeof(double)), "cudaMalloc(snapshot)");
        c->have_snap = false;
    }
    double apre, apost;
    envelope_pair(c, c->t, apre, apost);
    LaunchArgs a = launch_args(c, c->A, nullptr, apre, apost);
    const int nb = reduce_blocks(c->g);
    CK(reduce(c->lattice, a, c->snap, c->have_snap ? 1 : 0, c->partials, nb, c->red_out), "reduce kernels");
    c->launches += 2;
    double r[8];
    CK(cudaMemcpyAsync(r, c->red_out, sizeof r, cudaMemcpyDeviceToHost, c->stream), "copy reduction");
    CK(cudaStreamSynchronize(c->stream), "lbm_reduce");
    out[0] = r[0];
    out[1] = r[1];
    out[2] = r[2];
    out[3] = r[3];
    out[4] = c->have_snap ? r[4] : std::numeric_limits<double>::infinity();
    c->have_snap = true;
    if (r[5] != 0.0) return fail(c, LBM_EUNSTABLE, "lbm_reduce: non-finite or non-positive density/scalar");
    return LBM_OK;
}

int lbm_l2_error(lbm_ctx *c, const double *ref, int where, int field, int half_forced, double out[3])
{
    NvtxRange nvtx_("lbm_l2_error");
    if (!c) return LBM_EINVAL;
    c->err.clear();
    if (!c->initialised) return fail(c, LBM_ESTATE, "lbm_l2_error: populations not initialised");
    if (!ref || !out) return fail(c, LBM_EINVAL, "lbm_l2_error: NULL argument");
    if (where != 0 && where != 1) return fail(c, LBM_EINVAL, "lbm_l2_error: where must be 0 or 1");
    const bool scalar = c->lattice == LBM_D2Q5_CDE;
    if (field != 0 && (field != 1 || scalar))
        return fail(c, LBM_EINVAL, "lbm_l2_error: field must be 0 (rho or phi) or 1 (u, flow lattices)");
    LrefView view(c, true);
    if (view.rc != LBM_OK) return view.rc;
    const size_t N = (size_t)c->g.N;
    const size_t n = field == 0 ? N : (size_t)c->dim * N;
    // The field (and a host reference) go to the scratch buffer B (FP64) or the
    // staging buffer: rho at [0, N), u at [N, (1 + dim) N), ref after them;
    // (1 + 2 dim) N <= q N doubles for every lattice.
    double *st = c->B;
    if (c->storage != LBM_FP64) {
        const int rc = ensure_stage(c);
        if (rc != LBM_OK) return rc;
        st = c->stage;
    } else {
        const int rc = wait_readers(c, c->B);
        if (rc != LBM_OK) return rc;
    }
    double apre, apost;
    envelope_pair(c, c->t, apre, apost);
    LaunchArgs a = launch_args(c, c->A, nullptr, apre, apost);
    CK(moments(c->lattice, a, st, st + N, half_forced ? 1 : 0), "moments kernel");
    const double *dref = ref;
    if (where == 0) {
        double *r = st + (size_t)(1 + c->dim) * N;
        CK(cudaMemcpyAsync(r, ref, n * sizeof(double), cudaMemcpyHostToDevice, c->stream), "copy reference");
        dref = r;
    }
    const int nb = reduce_blocks(c->g);
    CK(l2_terms(field == 0 ? st : st + N, dref, (long long)n, c->partials, nb, c->red_out, c->stream), "l2 kernels");
    c->launches += 3;
    double r[8];
    CK(cudaMemcpyAsync(r, c->red_out, sizeof r, cudaMemcpyDeviceToHost, c->stream), "copy l2 terms");
    CK(cudaStreamSynchronize(c->stream), "lbm_l2_error");
    out[0] = r[0];
    out[1] = r[1];
    out[2] = r[1] > 0.0 ? std::sqrt(r[0] / r[1]) : (r[0] > 0.0 ? std::numeric_limits<double>::infinity() : 0.0);
    return LBM_OK;
}

int lbm_get_populations(lbm_ctx *c, double *dst, size_t count, int where, long *step_out)
{
    if (!c) return LBM_EINVAL;
    c->err.clear();
    if (!c->initialised) return fail(c, LBM_ESTATE, "lbm_get_populations: populations not initialised");
    if (!dst || count != (size_t)c->q * c->g.N) return fail(c, LBM_EINVAL, "lbm_get_populations: count must be q*N");
    LrefView view(c, true);
    if (view.rc != LBM_OK) return view.rc;
    if (step_out) *step_out = c->t;
    const size_t N = (size_t)c->g.N;
    const cudaMemcpyKind kind = where ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (c->storage != LBM_FP64) {
        double *plain = where ? dst : nullptr;
        if (!plain) {
            int rc = ensure_stage(c);
            if (rc != LBM_OK) return rc;
            plain = c->stage;
        }
        CK(rp_gather(c->lattice, c->storage, c->g, c->rho_ref, ref5(c), c->A, plain, c->stream), "gather kernel");
        c->launches++;
        if (!where) {
            CK(cudaMemcpyAsync(dst, plain, (size_t)c->q * N * sizeof(double), kind, c->stream), "copy populations");
            CK(cudaStreamSynchronize(c->stream), "lbm_get_populations");
        }
        return LBM_OK;
    }
    {
        const int rc = wait_readers(c, c->B);
        if (rc != LBM_OK) return rc;
    }
    CK(gather_from_stored(c->lattice, c->g, c->A, c->B, c->stream), "gather kernel");
    c->launches++;
    CK(cudaMemcpy2DAsync(dst, N * sizeof(double), c->B, (size_t)c->g.Np * sizeof(double), N * sizeof(double),
                         (size_t)c->q, kind, c->stream),
       "copy populations");
    if (!where) CK(cudaStreamSynchronize(c->stream), "lbm_get_populations");
    return LBM_OK;
}

int lbm_set_populations(lbm_ctx *c, const double *src, size_t count, int where, long step)
{
    if (!c) return LBM_EINVAL;
    c->err.clear();
    if (!src || count != (size_t)c->q * c->g.N) return fail(c, LBM_EINVAL, "lbm_set_populations: count must be q*N");
    if (step < 0) return fail(c, LBM_EINVAL, "lbm_set_populations: step < 0");
    {
        const int rc = wait_readers(c, nullptr);
        if (rc != LBM_OK) return rc;
    }
    const size_t N = (size_t)c->g.N;
    const cudaMemcpyKind kind = where ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (c->storage != LBM_FP64) {
        LrefView view(c, false);  // local reference: the FP32 scatter, then the encoding
        const double *plain = where ? src : nullptr;
        if (!plain) {
            int rc = ensure_stage(c);
            if (rc != LBM_OK) return rc;
            CK(cudaMemcpyAsync(c->stage, src, (size_t)c->q * N * sizeof(double), kind, c->stream), "copy populations");
            plain = c->stage;
        }
        CK(rp_scatter(c->lattice, c->storage, c->g, c->rho_ref, ref5(c), plain, c->A, c->stream), "scatter kernel");
        c->launches++;
        view.restore();
        if (c->lref_every) {
            const int rc = lref_encode_state(c);
            if (rc != LBM_OK) return rc;
            c->lref_since = 0;
        }
        CK(cudaStreamSynchronize(c->stream), "lbm_set_populations");
        c->t = step;
        c->initialised = true;
        c->have_snap = false;
        c->version++;
        return LBM_OK;
    }
    CK(cudaMemcpy2DAsync(c->B, (size_t)c->g.Np * sizeof(double), src, N * sizeof(double), N * sizeof(double),
                         (size_t)c->q, kind, c->stream),
       "copy populations");
    CK(scatter_to_stored(c->lattice, c->g, c->B, c->A, c->stream), "scatter kernel");
    c->launches++;
    CK(cudaStreamSynchronize(c->stream), "lbm_set_populations");
    c->t = step;
    c->initialised = true;
    c->have_snap = false;
    c->version++;
    return LBM_OK;
}

int lbm_get_step(const lbm_ctx *c, long *step)
{
    if (!c || !step) return LBM_EINVAL;
    *step = c->t;
    return LBM_OK;
}

int lbm_sync(lbm_ctx *c)
{
    if (!c) return LBM_EINVAL;
    CK(cudaStreamSynchronize(c->stream), "lbm_sync");
    return LBM_OK;
}

int lbm_launch_count(const lbm_ctx *c, long long *count)
{
    if (!c || !count) return LBM_EINVAL;
    *count = c->launches;
    return LBM_OK;
}

}  // extern "C"
