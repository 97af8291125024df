// Internal definition of the library context (shared by the C ABI files).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_internal.h"

namespace lbmc {

struct DeviceField {
    int kind = lbmk::FK_NONE;  // FieldKind seen by the kernels
    double *dev = nullptr;
    float *fdev = nullptr;     // FP32 copy for reduced-precision contexts
    size_t cap = 0;            // values allocated at dev (and fdev)
    lbmk::FieldDev d{};
};

}  // namespace lbmc

struct lbm_ctx {
    int lattice = 0, q = 0, dim = 0, storage = 0;
    int elem = 8;         // bytes per stored population value
    double rho_ref = 1.0; // reduced-precision storage: reference of the deviations
    int sround = 0;       // 16-bit storage: stochastic rounding of the stored deviations
    unsigned long long sr_seed = 0;
    // 16-bit D2Q9 / D2Q5 storage at a per-node reference (lbmk::Lref): steps
    // between rebuilds of the reference (0: off, the plain deviations), steps
    // since the last one, the reference [1 or 3][Np], {sigma, 1 / sigma, the
    // rebuild's largest |d - e| per block}, and q*Np floats of FP32 deviations (every read
    // or write of the state goes through them; the step's rebuilds do not)
    int lref_every = 0;
    int lref_since = 0;
    float *lref_ref = nullptr;
    float *lref_aux = nullptr;
    float *lref_dev = nullptr;  // allocated at the first read or write of the state
    // the rebuild's target (swapped with lref_ref / lref_aux after each)
    float *lref_ref2 = nullptr;
    float *lref_aux2 = nullptr;
    // D2Q5 reduced-precision storage: reference populations of the deviations
    // (lbmk::Ref5; set at lbm_init_equilibrium)
    double gref[5] = {0, 0, 0, 0, 0};
    double *stage = nullptr;  // reduced-precision storage: q*N doubles for host I/O (lazy)
    int device = 0;       // CUDA device that was current at lbm_create
    lbmk::Geom g{};
    double omega[9] = {0};
    cudaStream_t stream = nullptr;
    double *A = nullptr;  // stored populations of the current state (element type per storage)
    double *B = nullptr;  // next state / scratch
    lbmc::DeviceField force;  // force (flow) or source (scalar)
    lbmc::DeviceField vel;    // advecting velocity (scalar)
    lbm_envelope_fn env = nullptr;
    void *env_user = nullptr;
    std::vector<double> env_tab;  // a(env_t0 + k/2), k = 0..size-1 (used when non-empty)
    double env_t0 = 0.0;
    long t = 0;
    bool initialised = false;
    double *snap = nullptr;
    bool have_snap = false;
    double *partials = nullptr;
    double *red_out = nullptr;
    long long launches = 0;
    long long version = 0;  // bumped by every change a batch descriptor depends on
    // Readback kernels queued on another stream (a batch's copy stream) that
    // may still read a population buffer: entry k says that buffer rd_buf[k]
    // is read until event rd_ev[k] completes.  Work on this context's stream
    // that writes a buffer waits for its entry first (lbmc::wait_readers).
    const void *rd_buf[2] = {nullptr, nullptr};
    cudaEvent_t rd_ev[2] = {nullptr, nullptr};
    std::string err;
};

#include <nvtx3/nvToolsExt.h>

namespace lbmc {

// NVTX range for the duration of a scope (no cost unless a profiler attaches).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Record a failure on c (or, for c == NULL, the process-wide lbm_create error)
// and return code.
int fail(lbm_ctx *c, int code, const char *fmt, ...);
int cuda_fail(lbm_ctx *c, cudaError_t e, const char *what);
// Envelope averages (a_pre, a_post) of step t (trapezoid rule of Sec. 6.3).
void envelope_pair(const lbm_ctx *c, long t, double &apre, double &apost);
bool envelope_covers(const lbm_ctx *c, long t, long n);
// Reduced-precision contexts: allocate the FP64 host-I/O staging buffer on first use.
int ensure_stage(lbm_ctx *c);
// Before work on c's stream writes population buffer `buf` (nullptr: either
// buffer), make the stream wait for the readbacks that may still read it.
int wait_readers(lbm_ctx *c, const void *buf);
// The D2Q5 reference populations of c as a kernel argument.
lbmk::Ref5 ref5(const lbm_ctx *c);
// Key of step t's stochastic-rounding bits (seed mixed, step in the high bits).
unsigned long long sr_step_key(unsigned long long seed, long t);
// The local-reference encoding of a 16-bit context (lbmk::Lref).
lbmk::Lref lref_of(const lbm_ctx *c);
// Local-reference contexts: the state decoded to FP32 deviations (lref_dev),
// and rebuilt from them (new reference and sigma, stored values into A).
int lref_decode_state(lbm_ctx *c);
int lref_encode_state(lbm_ctx *c);
// The rebuild in place (new reference and sigma from the stored state, no
// FP32 copy); `old` describes the encoding the state is in (its q5 may
// differ from the context's current velocity's).
int lref_rebuild_state(lbm_ctx *c, const lbmk::Lref &old);
// For the length of a scope a local-reference context looks like an FP32
// deviation context whose stored buffer is lref_dev (decoded on entry when
// `decode`), so that the FP32 read and write paths serve it; a write path
// then calls lref_encode_state after restore().
struct LrefView {
    lbm_ctx *c;
    double *A0 = nullptr;
    int st0 = 0, el0 = 0;
    bool on = false;
    int rc = 0;
    LrefView(lbm_ctx *cc, bool decode);
    void restore();
    ~LrefView() { restore(); }
    LrefView(const LrefView &) = delete;
    LrefView &operator=(const LrefView &) = delete;
};
// Launch arguments of the context's kernels.
lbmk::LaunchArgs launch_args(const lbm_ctx *c, const double *fin, double *fout, double apre, double apost);

}  // namespace lbmc

#define LBM_CK(call, what)                                            \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return lbmc::cuda_fail(c, e_, what);   \
    } while (0)
