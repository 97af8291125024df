/*
 * Plain FP64 CPU oracle of the cascaded lattice Boltzmann step with
 * Strang-split forcing (flow) and Strang-split sources (passive scalar),
 * arXiv:1806.10247.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link
 * or call this code: it is used by the tests, by the smoke check and by the
 * CPU-baseline leg of the benchmark.  It shares no code with the CUDA path.
 *
 * Populations are stored structure-of-arrays, f[q][z][y][x], x fastest.
 * The state held between steps is the pre-collision population set f(t)
 * (the result of the streaming step, Eq. 22b / Eq. 40b).
 *
 * Velocity orderings:
 *   D2Q9  : the paper's order (Sec. 4, Eq. 15).
 *   D2Q5  : the paper's order (Sec. 5, Eq. 34).
 *   D3Q27 : alpha = (ex+1) + 3 (ey+1) + 9 (ez+1)  (the paper gives no D3Q27 order).
 *   D3Q15 : the paper's order (Appendix A, Eq. a1).
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ORC_D2Q9  1
#define ORC_D3Q27 2
#define ORC_D2Q5  3
#define ORC_D3Q15 4

typedef struct {
    int lattice;            /* ORC_D2Q9 / ORC_D3Q27 / ORC_D2Q5 / ORC_D3Q15 */
    int n[3];               /* nx, ny, nz (nz = 1 for the 2D lattices) */
    int wall[3];            /* per axis: 0 periodic, 1 halfway bounce-back walls at both ends */
    /* Relaxation parameters.
     *   D2Q9 : omega[3..8] = omega_3..omega_8 of Eq. 23.
     *   D2Q5 : omega[1..4] = omega_1^phi..omega_4^phi of Eq. 41.
     *   D3Q27: omega[1] trace (bulk), omega[2] deviatoric and off-diagonal second
     *          order (shear), omega[3..6] all central moments of order 3..6.
     *   D3Q15: omega[1] = omega_9 (trace), omega[2] = omega_4..omega_8 (shear),
     *          omega[3] = omega_10..omega_13 (third order), omega[4] = omega_14
     *          (fourth order), numbered as in Eq. 6A. */
    double omega[9];
    int generic;            /* D2Q9 only: 1 = generic central-moment procedure instead of Eqs. 23/32 */
    int as_printed;         /* D2Q5: 1 = Eq. 41 with the u^2 phi signs exactly as printed.
                             * D3Q15: 1 = g_9 of Eq. 6A without its missing rho term and
                             * the printed sign of g_13 in f^p_12 (Appendix A). */
} orc_params;

/* Number of velocities of a lattice (9, 27, 5, 15), 0 if unknown. */
/* Set the thread count of the node loops (n > 0); returns the count in use. */
int orc_set_threads(int n);
int orc_q(int lattice);
/* Spatial dimension of a lattice (2 or 3). */
int orc_dim(int lattice);
/* Velocity components e[alpha][3] of a lattice, written into e (q*3 ints). */
int orc_velocities(int lattice, int *e);

/* Equilibrium populations whose central moments are those of Eq. 20 (flow) or
 * Eq. 39 (scalar) at the given density/scalar and velocity field.
 *   rho : [N] density (flow) or scalar phi (D2Q5)
 *   u   : [3][N] velocity (for D2Q5: the advecting velocity)
 *   f   : [q][N] output */
int orc_equilibrium(const orc_params *p, const double *rho, const double *u, double *f);

/* Advance f by nsteps time steps.
 *   f      : [q][N] in/out, pre-collision populations
 *   work   : [q][N] scratch (post-collision populations)
 *   P      : flow: [dim][N] force shape; D2Q5: [N] source shape; NULL = no force/source
 *   a      : [2*nsteps] envelope values (a_pre, a_post) per step; the force at
 *            node x in the pre-collision half step is a_pre*P(x) and in the post-
 *            collision half step a_post*P(x).  NULL = 1,1 each step.
 *   uadv   : D2Q5 only: [2][N] advecting velocity
 * Returns 0, or -1 on invalid parameters. */
int orc_run(const orc_params *p, double *f, double *work, long nsteps,
            const double *P, const double *a, const double *uadv);

/* Macroscopic fields of f (Eq. 24 / Eq. 42).
 *   flow : rho[N] = sum f; u[dim][N] = (sum f e + a_pre*P/2)/rho
 *   D2Q5 : rho[N] = phi = sum g + a_pre*P/2;   u unused
 * P may be NULL (no force/source); a_pre is then ignored. */
int orc_moments(const orc_params *p, const double *f, const double *P, double a_pre,
                double *rho, double *u);

/* Strain-rate tensor from the non-equilibrium second moments (Sec. 6.6):
 * Pi_ab = sum f e_a e_b - rho u_a u_b - rho c_s^2 delta_ab about the half-forced
 * velocity u of Eq. 25 / 8A (the a_pre * P / 2 term as in orc_moments), and
 *   S_ab = -(3 omega_s / (2 rho0)) Pi_ab            (a != b; the formula of Sec. 6.6)
 *   S_aa = -(3 / (2 rho0)) (omega_d D_a + omega_b T / dim)
 * with T = sum_a Pi_aa, D_a = Pi_aa - T / dim (trace and deviatoric parts relax
 * with their own rates: D2Q9 omega_d = omega_4, omega_s = omega_5, omega_b =
 * omega_3; D3Q27 and D3Q15 omega_d = omega_s = omega[2], omega_b = omega[1]).
 * Output S[ncomp][N]: 2D xx, yy, xy; 3D xx, yy, zz, xy, xz, yz.  Flow lattices only. */
int orc_strain_rate(const orc_params *p, const double *f, const double *P, double a_pre, double rho0, double *S);

/* One collision (no streaming) of a single node's populations, for the unit
 * tests: fin[q] -> fout[q], with pre/post force (or source) values and, for
 * D2Q5, the advecting velocity.  Fpre/Fpost have dim entries (flow) or 1 (D2Q5). */
int orc_collide_node(const orc_params *p, const double *fin, const double *Fpre,
                     const double *Fpost, const double *uadv, double *fout);

/* Same collision through the generic central-moment procedure (tensor-product
 * lattices D2Q9 and D3Q27 only). */
int orc_collide_node_generic(const orc_params *p, const double *fin, const double *Fpre,
                             const double *Fpost, double *fout);

/* ---- Context API -----------------------------------------------------------
 * The oracle behind the same calls as the library's C ABI (lbm_* there,
 * lbmref_* here), with host pointers only: a context owns f(t) and steps it
 * with orc_run.  Status codes mirror the library's; fields are full node
 * arrays (expand a separable shape first).  Relaxation rates as in
 * orc_params.omega; wall[d] = 1 puts halfway bounce-back walls on axis d. */
#define LBMREF_OK 0
#define LBMREF_EINVAL -1
#define LBMREF_ENOMEM -2
#define LBMREF_EUNSTABLE -4
#define LBMREF_ESTATE -6

typedef struct lbmref_ctx lbmref_ctx;
typedef double (*lbmref_envelope_fn)(double t, void *user);

int lbmref_create(lbmref_ctx **out, int lattice, int nx, int ny, int nz, const double omega[9],
                  const int wall[3]);
void lbmref_destroy(lbmref_ctx *c);
/* f = equilibrium at (rho, u): host rho [N] (NULL = rho0), u [dim][N] (NULL = u0);
 * step counter to 0. */
int lbmref_init_equilibrium(lbmref_ctx *c, double rho0, const double u0[3], const double *rho, const double *u);
/* Force shape [dim][N] (flow) / source shape [N] (D2Q5) / advecting velocity
 * [2][N] (D2Q5); copied; NULL removes it (zero velocity). */
int lbmref_set_force(lbmref_ctx *c, const double *P);
int lbmref_set_source(lbmref_ctx *c, const double *S);
int lbmref_set_velocity(lbmref_ctx *c, const double *u);
/* Envelope a(t) (NULL = 1); each step uses the trapezoid averages of Sec. 6.3. */
int lbmref_set_envelope(lbmref_ctx *c, lbmref_envelope_fn fn, void *user);
int lbmref_step(lbmref_ctx *c, long n);
/* rho [N] (phi for D2Q5) and u [dim][N] of f(t); half_forced as in orc_moments. */
int lbmref_moments(lbmref_ctx *c, double *rho, double *u, int half_forced);
/* out[0] = sum rho (sum phi^o), out[1..3] = sum of sum f e (flow), out[4] = max
 * |u - u_prev| (|phi - phi_prev|) since the previous call, +inf on the first;
 * LBMREF_EUNSTABLE if a density is non-finite or (flow) not positive. */
int lbmref_reduce(lbmref_ctx *c, double out[5]);
/* Discrete relative l2 error of Eq. sca (Sec. 6.1) of a field of f(t) against
 * a reference: field 0 = rho (phi for D2Q5), ref [N]; field 1 = u (flow),
 * ref [dim][N]; half_forced as in lbmref_moments.  out[0] = sum over every
 * node and component of (q - q_ref)^2, out[1] = sum q_ref^2, out[2] =
 * sqrt(out[0] / out[1]) (+inf when out[1] = 0 < out[0], 0 when both are 0). */
int lbmref_l2_error(lbmref_ctx *c, const double *ref, int field, int half_forced, double out[3]);
int lbmref_get_populations(const lbmref_ctx *c, double *dst, size_t count);
int lbmref_set_populations(lbmref_ctx *c, const double *src, size_t count, long step);
int lbmref_get_step(const lbmref_ctx *c, long *step);

#ifdef __cplusplus
}
#endif
#endif
