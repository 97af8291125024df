// Host-side interface between the C ABI (lbm_capi.cu) and the per-lattice
// kernel launchers (k_d2q9.cu, k_d2q5.cu, k_d3q27.cu, k_common.cu).
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbmk {

// Host: a force of kind `fkind` has identically zero components 1 .. dim-1
// (along x only), so that a step kernel may leave their terms out.
inline bool force_x_only(int fkind, const FieldDev &F, int dim)
{
    bool zero = true;
    for (int c = 1; c < dim; c++) {
        if (fkind == FK_CONST) zero = zero && F.cval[c] == 0.0;
        else if (fkind == FK_GENERAL) zero = zero && F.sep && ((F.zmask >> c) & 1);
        else zero = false;
    }
    return zero;
}

// Everything one launch of a step / moments / reduction kernel needs.
struct LaunchArgs {
    Geom g;
    const double *fin;   // stored populations (the state from which f(t) is pulled)
    double *fout;        // step: new stored populations
    int fkind;           // FieldKind of the force (flow) or source (scalar)
    FieldDev F;
    int vkind;           // scalar lattice: FieldKind of the advecting velocity
    FieldDev V;
    double apre, apost;  // envelope averages of the two half steps
    double omega[9];
    cudaStream_t stream;
    int storage;         // 0 FP64 populations; 1/2/3 FP32/FP16/BF16 deviations f - w rho_ref
    double rho_ref;      // reference density/scalar of the deviations
    int sround;          // 16-bit storage: round the stored deviations stochastically
    unsigned long long srkey;  // ... with random bits keyed by this step key
    double gref[5];      // D2Q5, reduced precision: reference populations of the deviations
};

// D2Q5 reduced-precision storage keeps deviations d = g - g_ref from a
// uniform reference g_ref (sum g_ref = rho_ref): the rest state w rho_ref, or,
// on a periodic lattice with a uniform advecting velocity, the equilibrium at
// (rho_ref, u), which the step leaves unchanged, so the deviations carry the
// scalar's signal alone instead of the background's advection term.
struct Ref5 {
    double v[5];
};

// The source-free D2Q5 step matrix M of a uniform advecting velocity (Eqs. 41
// and 48 applied to the unit vectors; row-major), and C(g) - g = M g - g for
// a uniform state g (what one step adds to a uniform reference).
void d2q5_step_matrix(const double omega[9], double ux, double uy, double M[25]);
void d2q5_reference_change(const double omega[9], double ux, double uy, const double g[5], double out[5]);

// Reduced-precision storage (deviations from the rest state w * rho_ref):
// fused equilibrium fill into the stored layout, conversions between f(t) as
// dense [q][N] doubles and the stored layout, and the step kernel.
// gref: the D2Q5 reference (ignored by the other lattices, whose reference is w rho_ref).
cudaError_t rp_init_equilibrium(int lattice, int storage, const Geom &g, double rho_ref, const Ref5 &gref,
                                double rho0, const double *u0, const double *rho, const double *u, void *stored,
                                cudaStream_t s);
cudaError_t rp_scatter(int lattice, int storage, const Geom &g, double rho_ref, const Ref5 &gref,
                       const double *plain, void *stored, cudaStream_t s);
cudaError_t rp_gather(int lattice, int storage, const Geom &g, double rho_ref, const Ref5 &gref, const void *stored,
                      double *plain, cudaStream_t s);
cudaError_t rp_step(int lattice, const LaunchArgs &a);

// Relaxation rates are validated on the host; omega_high_one records whether
// every rate of order >= 3 equals 1 (enables the reduced collision).

// One lattice of a batch (lbm_batch_step): everything a batched step kernel
// needs for it.  Step k of a launch sequence reads buf[(parity + k) & 1] and
// writes buf[(parity + k + 1) & 1]; its envelope pair is pairs[k * count + item].
struct BatchItem {
    Geom g;
    double *buf[2];     // population buffers (element type given by the batch's storage)
    double rho_ref;     // reduced-precision storage: reference of the deviations
    int parity;
    int fkind, vkind;
    FieldDev F, V;
    double coef[16];  // lattice-specific collision coefficients (filled by batch_coef)
    float fcoef[20];  // FP32 copies for the reduced-precision kernels (FP64 runs at 1/64 rate);
                      // D2Q5: [16] holds P3 + (2/3) S3 of the uniform-velocity form
    float frho_ref;
    int variant;      // collision variant of this member (batch_variant)
    float fref[5];    // D2Q5 reduced precision, uniform velocity: M g_ref - g_ref, added after the collision
    double mat[25];   // D2Q5 with a uniform advecting velocity, FP64: step matrix M (row-major)
};

// Host: fill item.coef from the relaxation rates (and, for the scalar lattice
// with a uniform advecting velocity, that velocity).
void batch_coef(int lattice, const double omega[9], BatchItem &item);

// Arguments of one batched launch (passed by value as a __grid_constant__
// kernel parameter).  Item i of step k uses buf[(items[i].parity + parity) & 1]
// as input and its envelope pair pairs[k * count + i], or inl[i] when pairs is
// NULL (batches of at most kInlinePairs lattices: no per-step copy).
constexpr int kInlinePairs = 32;
struct BatchLaunch {
    const BatchItem *items;
    const int *first;  // first tile of each item (ascending, first[0] = 0)
    int count;
    // The launch covers ntiles tiles of the kernel's tile size; with
    // persist = 1 (persistent grid of G blocks) block b takes tiles
    // [b ntiles / G, (b + 1) ntiles / G), else tile b.
    int ntiles;
    int persist;
    // single = 1: the batch has one member, whose descriptor travels here in
    // the launch arguments (read from the constant bank, nothing staged).
    int single;
    BatchItem one;
    int k;
    int parity;
    const double2 *pairs;
    double2 inl[kInlinePairs];
    // reduced-precision kernels read the same pairs in FP32
    const float2 *pairsf;
    float2 inlf[kInlinePairs];
    // Fused readback (FP64 kernels, lbm_batch_step_read): when mrho is not
    // NULL every node also writes the packed fields of the state its step
    // starts from, member i at moff[i] (the layout of lbm_batch_moments_packed).
    double *mrho;
    double *mu;
    const long long *moff;
    int mhalf;
};

// Packed fields of every member of a batch (one launch, tiles of 256 nodes).
struct BatchMoments {
    const BatchItem *items;
    const int *first;        // first 256-node tile of each member
    int count;
    int parity;              // buffer parity of the current state relative to the descriptors
    int half;                // add the pre-collision half force / source
    const double *apre;      // a_pre of each member's current step (device), or NULL:
    double apre_inl[kInlinePairs];  // ... then here (batches of at most kInlinePairs members)
    const long long *off;    // first node of each member in the packed output
    double *rho;             // [sum N_i]
    double *u;               // [sum dim N_i], member i's [dim][N_i] block at dim * off_i
};
cudaError_t batch_moments(int lattice, int storage, const BatchMoments &M, int nblocks, cudaStream_t s);

// One launch advancing every item of a batch by one step (FP64 storage);
// tile = nodes per tile = threads per block: 128, 256 or 512.
cudaError_t batch_step(int lattice, const BatchLaunch &L, int nblocks, int tile, cudaStream_t s);
// Blocks of the FP64 batch kernel resident on the whole GPU at once.
int batch_resident(int lattice, int tile);
// Collision variant of a batch member (BatchItem::variant): bit 0 set when
// the higher-order rates are 1 (D3Q27 omega_3..omega_6, D2Q9 omega_6..omega_8),
// bit 1 set as well when the force acts along x only (force_x_only) -- the
// same choices the single-lattice launch makes.
int batch_variant(int lattice, const double omega[9], int fkind, const FieldDev &F);
// tile = nodes per tile = threads per block: 128, 256 or 512.
cudaError_t rp_batch_step(int lattice, int storage, const BatchLaunch &L, int nblocks, int tile, cudaStream_t s);
// Blocks of the reduced-precision batch kernel resident on the whole GPU at once.
int rp_batch_resident(int lattice, int storage, int tile);

// Strain-rate tensor of the current state (flow lattices): out [ncomp][N],
// ncomp = 3 (2D: xx, yy, xy) or 6 (3D: xx, yy, zz, xy, xz, yz).
cudaError_t strain_rate(int lattice, const LaunchArgs &a, double rho0, double *out);
// out[i] = round-to-nearest FP32 of in[i], i < n (FP32 copies of device fields).
cudaError_t to_float(const double *in, float *out, long long n, cudaStream_t s);
// out[i] = coef * S:S from strain components S [ncomp][N]; fout (may be NULL) its FP32 copy.
cudaError_t viscous_source(int N, int dim, const double *S, double coef, double *out, float *fout, cudaStream_t s);

// One fused stream + collide step (pull form): fin -> fout.
cudaError_t d2q9_step(const LaunchArgs &a);
cudaError_t d2q5_step(const LaunchArgs &a);
cudaError_t d3q15_step(const LaunchArgs &a);
// D2Q9, FP64, constant envelope: nsteps steps of a small lattice in one
// launch (one thread-block cluster holding the state in its shared memory);
// cudaErrorNotSupported when the lattice is too large.  fin -> fout after
// nsteps steps (fout may equal fin).
cudaError_t d2q9_cluster_steps(const LaunchArgs &a, int nsteps);
// The same for reduced-precision storage (deviations kept in the storage type).
cudaError_t rp_cluster_steps9(const LaunchArgs &a, int nsteps);
cudaError_t d3q27_step(const LaunchArgs &a);

// Moments of the current state: rho[N] and u[dim][N] (flow) or phi[N] (scalar);
// half = 1 adds the pre-collision half force / source.
cudaError_t moments(int lattice, const LaunchArgs &a, double *rho, double *u, int half);

// Per-block partial reductions (see lbm_reduce) into partials[nblocks][8],
// updating the snapshot; then a single-block pass writes out[8].
cudaError_t reduce(int lattice, const LaunchArgs &a, double *snap, int have_snap, double *partials,
                   int nblocks, double *out);
// Largest grid of the reductions (152 SMs x 8 resident blocks); they loop
// over the nodes, so no lattice needs more.  reduce_blocks never exceeds it,
// and fixed scratch arrays of partial sums are sized by it.
constexpr int kReduceMaxBlocks = 1216;
int reduce_blocks(const Geom &g);
// Terms of the l2 error of Eq. sca over n values: out[0] = sum (q - ref)^2,
// out[1] = sum ref^2 (per-block partials[nblocks][8], then one block; out[8]).
cudaError_t l2_terms(const double *q, const double *ref, long long n, double *partials, int nblocks, double *out,
                     cudaStream_t s);
// Mass / momentum / instability-flag sums only (no snapshot): partials[nblocks][8], out[8].
cudaError_t reduce_sums(int lattice, const LaunchArgs &a, double *partials, int nblocks, double *out);

// Equilibrium populations at (rho, u) in plain [q][Np] layout into dst.
// rho/u may be NULL (uniform rho0/u0).
cudaError_t equilibrium(int lattice, const Geom &g, double rho0, const double *u0, const double *rho,
                        const double *u, double *dst, cudaStream_t s);

// Conversions between f(t) in plain [q][Np] layout and the stored layout
// (stored = inverse stream of f(t); f(t) = pull of stored).
cudaError_t scatter_to_stored(int lattice, const Geom &g, const double *plain, double *stored,
                              cudaStream_t s);
cudaError_t gather_from_stored(int lattice, const Geom &g, const double *stored, double *plain,
                               cudaStream_t s);

// 16-bit storage at a per-node reference (k_rp.cu): stored s = sigma (d - e),
// e the deviation of a low-order equilibrium at the node's reference.
struct Lref {
    float *ref;    // device [1 or 3][Np]: dphi (D2Q5), or drho, jx, jy (D2Q9)
    float *scale;  // device [2]: sigma (a power of two), 1 / sigma
    float q5[5];   // D2Q5: the equilibrium per unit scalar at the uniform velocity
};
// One step of a D2Q9 or D2Q5 (uniform velocity) lattice in this encoding.
cudaError_t lref_step(int lattice, const LaunchArgs &a, const Lref &L);
// Stored values -> FP32 deviations (the FP32 forms' stored layout).
cudaError_t lref_decode(int lattice, int storage, const Geom &g, const Lref &L, const void *stored, float *dev,
                        cudaStream_t s);
// The plain 16-bit deviations as this encoding (reference 0, every sigma 1).
cudaError_t lref_reset(int lattice, const Geom &g, const Lref &L, cudaStream_t s);
// FP32 deviations -> stored values at the current reference and sigma.
cudaError_t lref_encode(int lattice, int storage, const Geom &g, const Lref &L, const float *dev, void *stored,
                        cudaStream_t s);
// The rebuild in place, without an FP32 copy: a new reference (the node's
// own moments) into Lnew.ref and sigma into Lnew.scale, and every stored value
// decoded at Lold and stored at Lnew (Lnew.q5 may differ from Lold.q5);
// bmax: ceil(N / 256) floats of scratch.  Lnew's buffers differ from Lold's.
cudaError_t lref_rebuild(int lattice, int storage, const Geom &g, const Lref &Lold, const Lref &Lnew, float *bmax,
                         void *stored, cudaStream_t s);
// Every stored value decoded at Lold and stored at Lnew, in place (no new reference).
cudaError_t lref_reencode(int lattice, int storage, const Geom &g, const Lref &Lold, const Lref &Lnew, void *stored,
                          cudaStream_t s);
// A new reference and sigma from FP32 deviations, and the stored values at
// them; bmax: ceil(N / 256) floats of scratch.
cudaError_t lref_rebase(int lattice, int storage, const Geom &g, const Lref &L, float *bmax, const float *dev,
                        void *stored, cudaStream_t s);

}  // namespace lbmk
