/*
 * lbm.h — C ABI of the GB300 (sm_103a) cascaded lattice Boltzmann library.
 *
 * The library advances lattices with the cascaded (central-moment) lattice
 * Boltzmann method and the symmetrized (Strang) operator-split force and
 * source steps of arXiv:1806.10247:
 *
 *   one time step  f(t+1) = S F^1/2 C F^1/2 f(t)          (Sec. 3, Eq. 14)
 *   scalar step    g(t+1) = S R^1/2 C R^1/2 g(t)          (Sec. 5, Eq. StrangLBMCDE)
 *
 * on three lattices: D2Q9 flow (Sec. 4), D2Q5 passive scalar with a source
 * (Sec. 5) and D3Q27 flow (the extension of the 3D method of Appendix A to
 * D3Q27, by the generic central-moment procedure).  Every step runs on the
 * GPU in hand-written CUDA kernels; there is no CPU path.
 *
 * Conventions for every entry point:
 *  - Return value: an lbm_status code.  Nothing is thrown across the ABI.
 *    After a failure lbm_last_error(ctx) describes it (a string owned by the
 *    context, valid until the next call on that context).
 *  - Ownership: the library owns the population buffers of a context.  Caller
 *    pointers are read or written only during the call and never retained;
 *    fields passed to lbm_set_force / lbm_set_source / lbm_set_velocity are
 *    copied into library memory (a device field in stream order on the
 *    context's stream, see LBM_FIELD_FULL_DEVICE).
 *  - Streams: all device work of a context is issued on the CUDA stream given
 *    to lbm_create (NULL = the legacy default stream).  Calls that return
 *    data to host memory synchronise that stream before returning.  A context
 *    is not thread-safe.
 *  - Node order: node (x, y, z) has index i = x + nx*(y + ny*z); population
 *    arrays are [q][N] (structure of arrays), N = nx*ny*nz.
 *  - Velocity order: D2Q9 as in Sec. 4 Eq. 15; D2Q5 as in Sec. 5 Eq. 34;
 *    D3Q27: alpha = (ex+1) + 3*(ey+1) + 9*(ez+1).
 *  - Lattice units: dx = dt = 1, c_s^2 = 1/3.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_ABI_VERSION 2

/* Largest lattice of one context: 2^31 - 2^16 nodes (e.g. 65536 x 32767). */
#define LBM_MAX_NODES 2147418112LL

typedef struct lbm_ctx lbm_ctx;

/* Lattices. */
#define LBM_D2Q9 1     /* flow, Sec. 4 */
#define LBM_D3Q27 2    /* flow, Appendix A extended to D3Q27 */
#define LBM_D2Q5_CDE 3 /* passive scalar with source, Sec. 5 */
#define LBM_D3Q15 4    /* flow, Appendix A (Eqs. a1, 2A, 6A-13A); FP64 storage only */

/* Population storage / arithmetic.
 *   LBM_FP64     : populations in FP64, FP64 arithmetic (the reference form).
 *   LBM_FP32_DEV : deviations d = f - w * rho_ref from the rest state stored
 *   LBM_FP16_DEV   in FP32 / FP16 / BF16, all moment arithmetic in FP32
 *   LBM_BF16_DEV   (rest-state moments folded in analytically); moments,
 *                  reductions and population I/O stay FP64.  rho_ref is the
 *                  rho0 given to lbm_init_equilibrium (1 if not positive). */
#define LBM_FP64 0
#define LBM_FP32_DEV 1
#define LBM_FP16_DEV 2
#define LBM_BF16_DEV 3

/* Status codes. */
#define LBM_OK 0
#define LBM_EINVAL -1   /* invalid argument; nothing was changed */
#define LBM_ENOMEM -2   /* device allocation failed */
#define LBM_ECUDA -3    /* a CUDA call failed (message in lbm_last_error) */
#define LBM_EUNSTABLE -4 /* a density/scalar is non-finite or (flow) not positive */
#define LBM_ESTATE -6   /* call out of order (e.g. stepping before initialisation) */

/* Boundary kinds, one per axis. */
#define LBM_PERIODIC 0
#define LBM_BOUNCE_BACK 1 /* stationary halfway bounce-back walls at -1/2 and n-1/2 (Sec. 6.1) */

typedef struct {
    int axis[3]; /* x, y, z: LBM_PERIODIC or LBM_BOUNCE_BACK */
} lbm_boundary;

/* Relaxation rates, all in (0, 2).
 *   D2Q9  : omega[3..8] = omega_3 .. omega_8 of Sec. 4 Eq. 23 (omega_4 = omega_5
 *           = 1/tau gives nu = (tau - 1/2)/3; the paper uses omega_3 = omega_6 =
 *           omega_7 = omega_8 = 1, Sec. 6).
 *   D2Q5  : omega[1..4] = omega_1^phi .. omega_4^phi of Sec. 5 Eq. 41 (omega_1 =
 *           omega_2 = 1/tau_phi gives D = (tau_phi - 1/2)/3).
 *   D3Q27 : omega[1] trace of the second-order central moments (bulk),
 *           omega[2] their deviatoric and off-diagonal parts (shear, 1/tau),
 *           omega[3..6] every central moment of order 3..6.
 *   D3Q15 : rates of Appendix A Eq. 6A: omega[1] = omega_9 (trace, bulk),
 *           omega[2] = omega_4 .. omega_8 (shear, 1/tau), omega[3] = omega_10 ..
 *           omega_13 (third order), omega[4] = omega_14 (fourth order).
 *           Readings of the appendix built in: omega_9 relaxes the trace
 *           towards rho; the populations are exactly f + K g (the printed
 *           f^p_12 has the sign of g_13 flipped); the fourth-order target is
 *           the product of the post-collision kappa_xx and kappa_yy over rho.
 * Entries not listed for a lattice are ignored. */
typedef struct {
    double omega[9];
} lbm_relax;

/* A force (flow) or source (scalar) shape P, or the advecting velocity of the
 * scalar lattice.  Per component c:
 *   LBM_FIELD_SEPARABLE: P_c(x,y,z) = (px_c[x] * py_c[y]) * pz_c[z], evaluated
 *     in that order; data holds, for each component in turn, px_c (len[0]
 *     values), py_c (len[1]), pz_c (len[2]); a length of 1 means constant
 *     along that axis, otherwise it must equal the axis extent.
 *   LBM_FIELD_FULL: data holds P[c][N] in node order.
 *   LBM_FIELD_FULL_DEVICE: as LBM_FIELD_FULL, but data is DEVICE memory of
 *     the context's device (e.g. a field another kernel produced, such as a
 *     coupled flow's).  It is copied device to device on the context's
 *     stream, in stream order with the steps queued before and after the
 *     call, and nothing synchronises: the caller keeps data unchanged until
 *     the context's stream has passed the call (e.g. lbm_sync, or its own
 *     later work on that stream).  A pointer that is not device memory of
 *     the context's device gives LBM_EINVAL.
 * For the other kinds data is a host pointer; the values are copied before
 * the call returns. */
#define LBM_FIELD_NONE 0
#define LBM_FIELD_SEPARABLE 1
#define LBM_FIELD_FULL 2
#define LBM_FIELD_FULL_DEVICE 3

typedef struct {
    int kind;
    int len[3];
    const double *data;
} lbm_field;

/* Time envelope a(t) of the force or source: F(x, t) = a(t) P(x).  Each step
 * t -> t+1 uses a_pre = (a(t) + a(t+1/2))/2 in the pre-collision half step and
 * a_post = (a(t+1/2) + a(t+1))/2 in the post-collision half step (trapezoid
 * rule of Sec. 6.3).  Evaluated on the host, three times per step. */
typedef double (*lbm_envelope_fn)(double t, void *user);

/* Create a context.  Allocates two population buffers of q*N values (8, 4 or
 * 2 bytes each by `storage`) on the current CUDA device (N = nx*ny*nz; nz must
 * be 1 for the 2D lattices).
 * `stream` is a cudaStream_t (NULL = legacy default stream).
 * At most LBM_MAX_NODES nodes: node indices are 32-bit in the kernels, and
 * this bound keeps every thread's index, rounded up to a whole block, below
 * 2^31 (component offsets of [dim][N] and [q][N] arrays are 64-bit).
 * Errors: LBM_EINVAL (unknown lattice or storage, extent < 1, more than
 * LBM_MAX_NODES nodes, omega outside (0,2), bad boundary kind), LBM_ENOMEM,
 * LBM_ECUDA.  *out is NULL on error. */
int lbm_create(lbm_ctx **out, int lattice, int nx, int ny, int nz, const lbm_relax *relax,
               const lbm_boundary *bc, int storage, void *stream);

/* Release all device memory of a context (synchronises its stream).  NULL is a no-op. */
void lbm_destroy(lbm_ctx *ctx);

/* Message describing the last failure on ctx ("" if none); for ctx == NULL,
 * the last failure of lbm_create in this process. */
const char *lbm_last_error(const lbm_ctx *ctx);

/* Fill the populations with the equilibrium whose central moments are those of
 * Sec. 4 Eq. 20 (flow) or Sec. 5 Eq. 39 (scalar) — the product of 1D
 * Maxwellian profiles — and set the step counter to 0.
 *   rho    : host [N] density (flow) or scalar phi (D2Q5); NULL = rho0 everywhere
 *   u      : host [dim][N] velocity; NULL = u0 everywhere.  For D2Q5 this is
 *            the velocity of the equilibrium (normally the advecting velocity).
 * Errors: LBM_EINVAL (rho0 <= 0 for flow), LBM_ECUDA. */
int lbm_init_equilibrium(lbm_ctx *ctx, double rho0, const double u0[3], const double *rho,
                         const double *u);

/* Body force shape of a flow lattice (Sec. 3 Eq. 13; Sec. 4 Eqs. 25-31); dim
 * components.  kind LBM_FIELD_NONE removes the force.  The force enters the
 * pre-collision half step as u = (sum f e + a_pre P / 2)/rho (Eq. 25) and the
 * post-collision change of the first moment as (a_pre + a_post) P / 2
 * (Eqs. 27-31).  Errors: LBM_EINVAL (scalar lattice, bad lengths), LBM_ECUDA. */
int lbm_set_force(lbm_ctx *ctx, const lbm_field *shape);

/* Source shape of the scalar lattice (Sec. 5 Eqs. 43-47); one component.
 * phi = sum g + a_pre S / 2 enters the collision (Eq. 43) and the zeroth
 * moment changes by (a_pre + a_post) S / 2 (Eqs. 44-47).
 * Errors: LBM_EINVAL (flow lattice, bad lengths), LBM_ECUDA. */
int lbm_set_source(lbm_ctx *ctx, const lbm_field *shape);

/* Advecting velocity u(x) of the scalar lattice (Sec. 5 Eq. 33), two
 * components, constant in time.  Default: zero.
 * Errors: LBM_EINVAL (flow lattice), LBM_ECUDA. */
int lbm_set_velocity(lbm_ctx *ctx, const lbm_field *u);

/* Time envelope of the force or source as a host callback (NULL fn = a(t) = 1).
 * Replaces any envelope table. */
int lbm_set_envelope(lbm_ctx *ctx, lbm_envelope_fn fn, void *user);

/* Time envelope as a table of count >= 3 samples a[k] = a(t0 + k/2) (copied),
 * used instead of a callback; steps outside the table fail with LBM_EINVAL
 * (stepping from t needs samples up to t + n + 1).  count = 0 with a = NULL
 * removes the table.  Same trapezoid averages as lbm_set_envelope. */
int lbm_set_envelope_table(lbm_ctx *ctx, const double *a, long count, double t0);

/* Rounding of the stored deviations of a 16-bit storage context (LBM_FP16_DEV,
 * LBM_BF16_DEV): on = 0 rounds to nearest (the default); on = 1 rounds
 * stochastically: each stored value goes to the representable neighbour
 * further from zero with probability equal to its distance from the one
 * nearer to zero, in units of the step between them, so that it equals the
 * FP32 result on average and increments smaller than the storage step are not
 * lost on average (the paper has no counterpart: this addresses the force and
 * source increments of Eqs. 25/31 and 43/47 that 16-bit storage cannot
 * resolve).  The random bits come from a counter-based generator (the
 * SplitMix64 output function, Steele, Lea and Flood, OOPSLA 2014) keyed by
 * `seed`, the step counter, the node and the population, so a run is
 * reproducible for a given seed.  Applies to lbm_step (one launch per step;
 * the one-launch cluster form of small D2Q9 lattices is not used while it is
 * on); a context with it on cannot join a batch.
 * Errors: LBM_EINVAL (storage not 16-bit). */
int lbm_set_stochastic_rounding(lbm_ctx *ctx, int on, unsigned long long seed);

/* Storage of a 16-bit D2Q9 or D2Q5 context at a per-node reference (the
 * paper has no counterpart: this keeps the Strang-split force and source
 * increments of Eqs. 25/31 and 43/47, which a 16-bit deviation from the
 * fixed rest state of a few 1e-4 cannot resolve).  Each node keeps a
 * reference in FP32 -- D2Q9: the deviation of rho and j; D2Q5: the deviation
 * of phi -- and the stored 16-bit value of population a is
 * sigma (d_a - e_a): d_a the deviation the FP32 forms store (f_a - w_a rho_ref,
 * or g_a - g_ref,a), e_a that of an equilibrium at the reference (D2Q9:
 * w_a (drho + 3 c + 4.5 c^2 - 1.5 |j|^2), c = e_a . j, second order in j at
 * unit density; D2Q5: the Eq. 39 equilibrium per unit scalar at the uniform
 * advecting velocity, times dphi), and sigma a power of two per lattice that
 * puts the largest |d - e| in [8, 16) (FP16 then holds values 4096 times
 * larger).  A step pulls d = s / sigma + e of the source node and collides
 * exactly as the FP32 deviation form; every `every` steps of lbm_step the
 * reference and sigma are rebuilt from the state (the node's own moments), so
 * the 16-bit values hold only the non-equilibrium part and the change since
 * (the rebuild runs in place: two passes over the stored values).  Reads and
 * writes of the state (moments, reductions, populations, init) go through
 * FP32 deviations.
 * Memory: 2 x (1 or 3) floats per node on top of the 16-bit state (two
 * references), and q floats per node from the first read or write of the
 * state on.
 *   every : steps between rebuilds (>= 1), or 0 to return to the plain
 *           16-bit deviations (the state is converted either way).
 * A D2Q5 context needs a uniform advecting velocity (setting a velocity field
 * returns it to the plain deviations); stochastic rounding applies as set; a
 * context stored this way cannot join a batch.  Between rebuilds the stored
 * values must stay within the 16-bit range (FP16: 65504; see above); a
 * rebuild interval short against the flow's time
 * scales keeps them there, and an overflow shows as a non-finite density in
 * lbm_reduce.
 * Errors: LBM_EINVAL (storage not 16-bit, lattice not D2Q9 / D2Q5, every < 0,
 * a D2Q5 velocity field), LBM_ENOMEM, LBM_ECUDA. */
int lbm_set_local_reference(lbm_ctx *ctx, int every);

/* Advance n >= 0 time steps (n = 0 is a no-op).  Each step is one fused
 * kernel launch: stream (Eq. 22b / 40b, pull form, with periodic wrap or
 * halfway bounce-back), moments (Eq. 24 / 42), pre-collision half force or
 * source (Eq. 25 / 43), cascaded collision (Eq. 23 / 41 / generic D3Q27),
 * post-collision half step (Eq. 31 / 47) and the post-collision populations
 * (Eq. 32 / 48).  Exception: a small D2Q9 lattice (up to ~5000 nodes, any
 * storage) with a constant force envelope takes all n >= 2 steps in ONE launch of a
 * thread-block cluster that holds the state in its distributed shared memory
 * (same per-node arithmetic, one cluster barrier per step; counted as one
 * launch).  Asynchronous on the context's stream.
 * Errors: LBM_ESTATE (not initialised), LBM_EINVAL (n < 0), LBM_ECUDA. */
int lbm_step(lbm_ctx *ctx, long n);

/* Macroscopic fields of the current state f(t):
 *   flow : rho[N] = sum f (Eq. 24 / step (vi)); u[dim][N] = (sum f e + h a_pre P/2)/rho
 *   D2Q5 : rho[N] receives phi = sum g + h a_pre S/2 (Eqs. 42-43); u unused (may be NULL)
 * with h = 1 if half_forced, else 0 (u^o and phi^o).  Rounding: the sums in a
 * fixed grouping per lattice; j + a_pre P/2 rounded once; u = that times the
 * correctly rounded 1/rho (each product rounded), so u is within two units in
 * the last place of the exact quotient.  Every FP64 readback
 * (lbm_batch_moments, lbm_batch_moments_packed, lbm_batch_step_read) returns
 * these same bits.  where = 0: host pointers (the call synchronises);
 * where = 1: device pointers (asynchronous).
 * Errors: LBM_ESTATE, LBM_EINVAL (NULL output), LBM_ECUDA. */
int lbm_moments(lbm_ctx *ctx, double *rho, double *u, int where, int half_forced);

/* Debug aid: fill the context's second population buffer (the destination
 * of the next step) with NaN.  Every node of every plane is written by a
 * step, so after it the state holds no NaN; a node a kernel failed to write
 * would keep the NaN and make lbm_reduce return LBM_EUNSTABLE.  Asynchronous.
 * Errors: LBM_EINVAL, LBM_ECUDA. */
int lbm_debug_poison(lbm_ctx *ctx);

/* Strain-rate tensor of the current state (flow lattices) from the
 * non-equilibrium second moments, Sec. 6.6: with Pi_ab = sum f e_a e_b -
 * rho u_a u_b - rho c_s^2 delta_ab about the half-forced velocity of lbm_moments,
 *   S_ab = -(3 omega_s / (2 rho0)) Pi_ab   (a != b; the formula of Sec. 6.6)
 *   S_aa = -(3 / (2 rho0)) (omega_d D_a + omega_b T / dim),
 * T = sum_a Pi_aa, D_a = Pi_aa - T / dim.  Rates: D2Q9 omega_s = omega[5],
 * omega_d = omega[4], omega_b = omega[3]; D3Q27 and D3Q15 omega_s = omega_d =
 * omega[2], omega_b = omega[1].  S receives [ncomp][N]: 2D xx, yy, xy; 3D xx,
 * yy, zz, xy, xz, yz.  where = 0 host (synchronises), 1 device.  rho0 is the
 * reference density of the formula (> 0).  Errors: LBM_EINVAL (scalar lattice,
 * NULL output, rho0 <= 0), LBM_ESTATE, LBM_ECUDA. */
int lbm_strain_rate(lbm_ctx *ctx, double rho0, double *S, int where);

/* Viscous-heating source of a scalar lattice from a flow lattice on the same
 * grid and stream (Sec. 6.6, S_r = (2 nu / C_v) S:S): sets the scalar's source
 * shape to the full field coef * S:S of the flow's current state (computed on
 * the device, S as in lbm_strain_rate; coef = 2 nu / C_v).  The envelope of
 * the scalar still multiplies it.  Asynchronous on the shared stream.
 * Errors: LBM_EINVAL (wrong lattice kinds, grids, streams or devices; rho0
 * <= 0), LBM_ESTATE (flow not initialised), LBM_ENOMEM, LBM_ECUDA; the
 * message is on the scalar context. */
int lbm_set_source_from_strain(lbm_ctx *scalar, lbm_ctx *flow, double rho0, double coef);

/* Global sums over the lattice, computed on the GPU in FP64 with a fixed
 * (deterministic) reduction order:
 *   out[0] = sum rho (flow) or sum phi^o (scalar)
 *   out[1..3] = sum of sum_alpha f e (flow; zeros for the scalar lattice)
 *   out[4] = max over nodes and components of |u(t) - u(t_prev)| (flow, half
 *            forced velocity) or |phi(t) - phi(t_prev)| (scalar), where t_prev is
 *            the state at the previous lbm_reduce call; +inf on the first call.
 * out is a host array of 5 doubles; the call synchronises.
 * Errors: LBM_EUNSTABLE (some density/scalar non-finite or, for flow, <= 0;
 * out is still written), LBM_ESTATE, LBM_ECUDA. */
int lbm_reduce(lbm_ctx *ctx, double out[5]);

/* Discrete relative l2 error of a macroscopic field against a reference,
 * Eq. sca (Sec. 6.1, grid convergence study): sqrt(sum (q - q_ref)^2 /
 * sum q_ref^2), the sums running over every node (and every component).
 * q is the field lbm_moments returns with the same half_forced flag:
 *   field 0: rho (flow) or phi (scalar), ref holds N doubles;
 *   field 1: u (flow lattices only), ref holds dim*N doubles laid out [dim][N].
 * ref is host memory (where = 0; copied in during the call) or device memory
 * (where = 1), read only during the call.  Computed on the GPU in FP64 with a
 * fixed reduction order (the same state and reference give the same bits):
 *   out[0] = sum (q - q_ref)^2, out[1] = sum q_ref^2,
 *   out[2] = sqrt(out[0] / out[1]); +inf when out[1] = 0 < out[0], 0 when both are 0.
 * Uses the context's scratch buffer; synchronises the context's stream.
 * Errors: LBM_EINVAL (NULL ref/out, where or field out of range, field 1 on
 * the scalar lattice), LBM_ESTATE, LBM_ENOMEM, LBM_ECUDA. */
int lbm_l2_error(lbm_ctx *ctx, const double *ref, int where, int field, int half_forced, double out[3]);

/* The sums out[0..3] of lbm_reduce (mass, then momentum) without allocating
 * any device memory.  The paper has no counterpart: this exists for callers
 * that cannot allocate when they want the sums, e.g. a process whose device
 * memory is held by another allocator (a raw cudaMalloc may then fail) or a
 * time loop that must not call cudaMalloc/cudaFree because they can
 * synchronise the device.  The partial sums live in a fixed device array of
 * 1217 x 8 doubles (77,888 bytes) inside the library, reserved on every GPU
 * that loads it until the process exits; a lattice whose reduction would need
 * more than 1216 partial blocks is rejected with LBM_EINVAL (the reduction
 * never uses more, so in practice none is).  The first call on a device looks
 * up that array's device address (no allocation); make that first call before
 * any stream capture.  All calls, from every context on a device, share the
 * array: calls whose kernels overlap on the GPU race and may return wrong
 * sums, so serialise them (e.g. one stream).  Nothing in the array needs
 * clearing between calls.  Synchronises the context's stream; out is a host
 * array of 4 doubles.  Does not touch lbm_reduce's max-change snapshot.  A
 * context stored at a local reference (lbm_set_local_reference) is read
 * through its FP32 working copy, which the first other read or write of its
 * state allocates: before that, LBM_ESTATE.
 * Errors: LBM_ESTATE, LBM_EINVAL, LBM_EUNSTABLE (out still written), LBM_ECUDA. */
int lbm_reduce_sums_noalloc(lbm_ctx *ctx, double out[4]);

/* Copy the populations f(t) (the state after the streaming step of step t,
 * as [q][N] doubles) to dst.  count must equal q*N.  where: 0 host (the
 * call synchronises), 1 device (asynchronous on the context's stream).
 * step_out (may be NULL) receives t, the step counter of the state copied
 * (in lattice units the time equals the step count).
 * Errors: LBM_ESTATE, LBM_EINVAL (count), LBM_ECUDA. */
int lbm_get_populations(lbm_ctx *ctx, double *dst, size_t count, int where, long *step_out);

/* Replace the populations by src ([q][N] doubles, count = q*N) and set the
 * step counter to `step` (checkpoint restore).  where: 0 host, 1 device.
 * Errors: LBM_EINVAL, LBM_ECUDA. */
int lbm_set_populations(lbm_ctx *ctx, const double *src, size_t count, int where, long step);

/* Current step counter t. */
int lbm_get_step(const lbm_ctx *ctx, long *step);

/* Block until all work issued on the context's stream is done. */
int lbm_sync(lbm_ctx *ctx);

/* Number of kernel launches issued by this context since its creation
 * (every step, initialisation, moments, reduction and copy kernel counts). */
int lbm_launch_count(const lbm_ctx *ctx, long long *count);

/* ---- Batches: many lattices, one kernel launch per time step ------------
 *
 * A batch groups contexts of the same lattice and storage that share one
 * stream and device (e.g. the members of a parameter sweep).  lbm_batch_step
 * advances all of them together: each time step is a single kernel launch
 * over the blocks of every member, each member keeping its own geometry,
 * relaxation rates, force/source/velocity shape, envelope and step counter.
 * The arithmetic is that of lbm_step on each member; results agree with it to
 * FP64 rounding (the two kernels may fuse multiply-adds differently).  The
 * batch keeps pointers to the contexts (they must outlive it) and owns only
 * its own descriptor buffers. */
typedef struct lbm_batch lbm_batch;

/* Errors: LBM_EINVAL (count < 1, NULL or repeated context, members differing
 * in lattice, storage, stream or device, a member with stochastic rounding
 * on), LBM_ENOMEM, LBM_ECUDA. */
int lbm_batch_create(lbm_batch **out, lbm_ctx *const *ctxs, int count);

/* Advance every member by n >= 0 steps (asynchronous on the members' stream).
 * Errors: LBM_ESTATE (a member not initialised), LBM_EINVAL (n < 0, envelope
 * table too short), LBM_ECUDA. */
int lbm_batch_step(lbm_batch *b, long n);

/* Kernel launches issued so far: one per step of lbm_batch_step (whether
 * launched directly or as a node of a replayed graph) plus the trial launches
 * of lbm_batch_autotune.  A batch of one member steps outside graph replays
 * with the member's own single-lattice kernel; those launches are counted by
 * the member (lbm_launch_count), not here. */
int lbm_batch_launch_count(const lbm_batch *b, long long *count);

/* Tiling of the batched launch.  The nodes of every member are cut into tiles
 * of `tile` nodes (128, 256 or 512; one thread per node, `tile` threads per
 * block), numbered member after member.  persistent = 0: one block per tile;
 * persistent = 1: a grid of as many blocks as the GPU holds resident at once,
 * each block taking a contiguous run of tiles, the runs differing in length
 * by at most one tile (a block reloads a member's descriptor only when its
 * run crosses into the next member; the FP64 scalar-lattice kernel also
 * loads each tile's operands while it computes the previous tile).  Default
 * 256 / 0.  The arithmetic per node does not depend on the tiling (up to the
 * compiler's multiply-add contraction in the different kernel instances).
 * A change drops a captured graph.  Errors: LBM_EINVAL. */
int lbm_batch_set_tiling(lbm_batch *b, int tile, int persistent);

/* Current tiling and the grid (blocks) a launch uses with it.  Any output
 * pointer may be NULL.  Errors: LBM_EINVAL (b NULL). */
int lbm_batch_get_tiling(lbm_batch *b, int *tile, int *persistent, int *grid);

/* Autotuner: runs every tiling the batch accepts for trial_steps launches
 * (after one warm-up launch each), timed with CUDA events on the batch's
 * stream, and keeps the fastest (ties: the first tried).  The trials leave
 * the members' state, step counters and envelope position unchanged: each
 * reads the current populations and writes only the second buffer, which the
 * next step overwrites anyway.  *best_us (if not NULL) receives the fastest
 * average time per launch in microseconds; all_us (if not NULL, 6 entries)
 * the average of every tiling, at index 2 * j + persistent for the tile sizes
 * j = 0, 1, 2 (128, 256, 512 nodes), -1 for tilings not tried.  Blocks the
 * host until the trials finish.  Errors: LBM_EINVAL (trial_steps outside
 * [1, 1000]), LBM_ESTATE (a member not initialised), LBM_ECUDA. */
int lbm_batch_autotune(lbm_batch *b, int trial_steps, double *best_us, double *all_us);

/* Replay steps as CUDA graphs of `steps_per_graph` launches each (a positive
 * even number; 0 turns graphs off, the default).  lbm_batch_step(b, n) then
 * issues n / steps_per_graph graph replays followed by ordinary launches for
 * the remainder.  Each graph copies that replay's envelope pairs from pinned
 * host memory and runs the batched step steps_per_graph times; it is captured
 * on first use (on a private stream) and again when the members' buffer
 * parity changes.  With a time-dependent envelope the host waits for the
 * previous replay before refilling the pinned pairs.  Errors: LBM_EINVAL. */
int lbm_batch_set_graph(lbm_batch *b, int steps_per_graph);

/* Macroscopic fields of every member (as lbm_moments, Eqs. 24-25 / 42-43):
 * rho[i] (and, for flow lattices, u[i] as [dim][N]) receive member i's
 * fields.  where = 0: host pointers; all members' kernels and copies are
 * queued on the batch's stream and the call synchronises once at the end
 * (pinned host buffers make the copies asynchronous DMA).  where = 1: device
 * pointers, asynchronous.  Each member's second population buffer (or its
 * staging buffer) holds the fields on the way out.  Errors: LBM_EINVAL (NULL
 * output), LBM_ESTATE, LBM_ECUDA. */
int lbm_batch_moments(lbm_batch *b, double *const *rho, double *const *u, int where, int half_forced);

/* The same fields for every member in one kernel launch, packed member after
 * member in the batch's order: rho receives N_0 + N_1 + ... values (phi for the
 * scalar lattice); u (flow lattices) receives member i's [dim][N_i] block
 * starting at dim * (N_0 + ... + N_{i-1}).  where = 0: host pointers (two
 * copies and one synchronisation in all); where = 1: device pointers,
 * asynchronous; where = 2: host pointers (pinned memory for a true overlap),
 * asynchronous: the kernel runs on the batch's stream into one of two
 * staging slots and the copies run on a private copy stream, so that they
 * overlap the steps queued after this call; the host buffers are valid after
 * lbm_batch_wait_moments.  where = 3: host pointers into memory the device
 * can address (pinned by cudaHostAlloc / cudaMallocHost, or registered with
 * cudaHostRegisterMapped): the kernel writes the fields straight into host
 * memory (over NVLink-C2C on a Grace system), with no staging copy;
 * asynchronous, valid after lbm_batch_wait_moments.  Errors: LBM_EINVAL (NULL
 * output; for where = 3 also a pointer the device cannot address, e.g.
 * pageable memory), LBM_ESTATE, LBM_ENOMEM, LBM_ECUDA. */
int lbm_batch_moments_packed(lbm_batch *b, double *rho, double *u, int where, int half_forced);

/* One time step of every member (as lbm_batch_step(b, 1)) whose kernel also
 * writes the packed fields of the state the step STARTS from — the fields
 * lbm_batch_moments_packed(b, ..., half_forced) would have returned just
 * before this call, bit for bit, in the same packed layout.  The step pulls
 * exactly the populations those fields are sums of, so the readback costs the
 * step a few operations per node and no separate kernel.  FP64 batches only.
 * where = 1: device pointers; where = 3: host memory mapped into the device's
 * address space (written over the host link).  Asynchronous on the batch's
 * stream; the outputs are complete after lbm_batch_wait_moments (the call
 * takes one of the three readback slots like where = 2 / 3 readbacks) or a
 * synchronisation of the stream.  The state after the last call is read with
 * lbm_batch_moments_packed.  Errors: LBM_EINVAL (NULL output, where not 1 or
 * 3, reduced-precision batch, unmapped host memory), LBM_ESTATE, LBM_ECUDA. */
int lbm_batch_step_read(lbm_batch *b, double *rho, double *u, int where, int half_forced);

/* Wait for the asynchronous readbacks (where = 2 or 3, and lbm_batch_step_read), of which up to three
 * are in flight (the library uses three slots in turn): keep = 0 waits for
 * all of them, keep = 1 or 2 for all but the `keep` most recent ones (the
 * caller's host buffers then rotate among keep + 1 or more destinations; the
 * fields of the older readbacks are in host memory while the latest ones are
 * still on their way).  Errors: LBM_EINVAL (keep outside 0..2), LBM_ECUDA. */
int lbm_batch_wait_moments(lbm_batch *b, int keep);

/* Graph replays issued so far. */
int lbm_batch_graph_replays(const lbm_batch *b, long long *count);

/* Message of the last failure on b (NULL: the last lbm_batch_create failure). */
const char *lbm_batch_last_error(const lbm_batch *b);

/* Free the batch (synchronises its stream); the member contexts stay valid. */
void lbm_batch_destroy(lbm_batch *b);

/* ---- Device facts and the FP64 throughput probe ---------------------------
 *
 * The paper has no counterpart.  On this GPU the FP64 step kernels are bound
 * by the FP64 unit rather than by memory, so their roofline is stated
 * against the FP64 instruction rate measured on the device that runs them. */

/* Message of the last failure of lbm_device_info / lbm_probe_fp64 (per thread). */
const char *lbm_probe_last_error(void);

/* Attributes of CUDA device `device` into info[8]: [0] SM count, [1] maximum
 * SM clock (kHz), [2] memory clock (kHz), [3] memory bus width (bits), [4] L2
 * size (bytes), [5] compute capability major, [6] minor, [7] maximum resident
 * threads per SM.  Errors: LBM_EINVAL (info NULL), LBM_ECUDA (bad device). */
int lbm_device_info(int device, long long info[8]);

/* Queue (on `stream`, a cudaStream_t; NULL = default) a kernel of `blocks` x
 * `threads` threads, each running `chains` (8 or 16) independent dependency
 * chains of `iters` FP64 operations of one kind: op 0 fused multiply-add,
 * 1 add, 2 multiply.  It issues exactly blocks * threads * iters * chains
 * FP64 instructions.  sink (three device doubles, owned by the caller)
 * receives sink[0] = the SM clock cycles and sink[1] = the nanoseconds of
 * block 0's run: its SM clock in MHz is sink[0] / sink[1] * 1000 (the run
 * of one block is not the launch's when more blocks are launched than the
 * GPU holds resident).  sink[2] is never written in practice.  The caller
 * times the launch (e.g. CUDA events on the stream) for the rate.  Nothing
 * synchronises.
 * Errors: LBM_EINVAL (op outside 0..2, chains not 8 or 16, blocks < 1,
 * threads not a multiple of 32 in [32, 1024], iters < 1, sink NULL),
 * LBM_ECUDA (launch failure). */
int lbm_probe_fp64(int op, int chains, int blocks, int threads, long long iters, double *sink, void *stream);

/* ---- Learned warm start: network kernels ---------------------------------
 *
 * The paper has no counterpart.  These kernels train and evaluate the small 3D
 * convolutional surrogate that predicts an initial velocity field for the LB
 * iteration (which alone decides the converged result).  All pointers are
 * device pointers; tensors are FP32 in [batch][channel][D][H][W] layout;
 * weights [Co][Ci][KD][KH][KW] are read as FP32 (w_bf16 = 0) or BF16
 * (w_bf16 = 1) and accumulated in FP32; kernels are odd, padding is "same"
 * (zero outside), dilation per axis.  Work is queued on `stream` (a
 * cudaStream_t, NULL = default); nothing synchronises.  Errors: LBM_EINVAL
 * (bad sizes or NULL pointers), LBM_ECUDA; message in lbm_nn_last_error(). */
const char *lbm_nn_last_error(void);

/* Tensor cores: with BF16 weights (w_bf16 = 1), a convolution whose padded
 * shapes fit one tile (input channels x kernel taps <= 512 and output
 * channels <= 64 for the forward pass; output channels x taps <= 512 and
 * input channels <= 64 for the input gradient; input channels x taps <= 512
 * and output channels <= 64 for the weight gradient) runs as an implicit
 * GEMM on the tensor cores (tcgen05, 128-pixel tiles): the activations and
 * incoming gradients are rounded to BF16 as they are staged, each product is
 * exact and the sums are FP32; the weight gradient adds per-block partial
 * sums in a fixed order (deterministic).  Other shapes, and FP32 weights,
 * take CUDA-core kernels with FP32 operands. */

/* Status of the tensor-core kernels since the last call: *status = 1 if a
 * kernel's wait for its tensor-core work gave up after 2 s (its outputs are
 * then not written), else 0; the flag is cleared.  Synchronises the device.
 * Errors: LBM_EINVAL (status NULL), LBM_ECUDA. */
int lbm_nn_tc_status(int *status);

/* y = act(conv(x, w) + b); act 0 = identity, 1 = tanh. */
int lbm_nn_conv3d_forward(const float *x, const void *w, int w_bf16, const float *b, float *y, int n, int ci, int co,
                          const int dhw[3], const int k[3], const int dil[3], int act, void *stream);

/* Gradients of sum(gy * conv(x, w)): gx (skipped if NULL), gw, gb (sums over
 * batch and space in a fixed order). */
int lbm_nn_conv3d_backward(const float *x, const void *w, int w_bf16, const float *gy, float *gx, float *gw, float *gb,
                           int n, int ci, int co, const int dhw[3], const int k[3], const int dil[3], void *stream);

/* g *= 1 - y^2 (y = tanh output), in place. */
int lbm_nn_tanh_backward(float *g, const float *y, long long count, void *stream);

/* Mean squared error: g = 2 (y - t)/count, *loss (device double) = mean((y-t)^2). */
int lbm_nn_mse(const float *y, const float *t, float *g, long long count, double *loss, void *stream);

/* One bias-corrected Adam step on FP32 weights p (moments m, v); also writes
 * the BF16 copy p_bf16 if not NULL.  step >= 1. */
int lbm_nn_adam(float *p, const float *g, float *m, float *v, void *p_bf16, long long count, double lr, double b1,
                double b2, double eps, long long step, void *stream);

/* p_bf16 = round-to-nearest BF16 of p. */
int lbm_nn_to_bf16(const float *p, void *p_bf16, long long count, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
