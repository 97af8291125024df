/*
 * Plain FP64 CPU oracle of the cascaded lattice Boltzmann method with the
 * symmetrized (Strang) operator-split force and source steps of
 * arXiv:1806.10247.
 *
 * TEST INFRASTRUCTURE ONLY: used by the tests, the smoke check and the CPU
 * baseline of the benchmark.  The product (CUDA) path never includes, links
 * or calls it, and the two share no code.
 *
 * Everything here is written for clarity, not speed: explicit loops over
 * nodes and velocities, the paper's formulas spelled out term by term, a
 * Gauss-Jordan inverse for the moment matrices.  Compile with
 * -ffp-contract=off so that the results do not depend on whether the host
 * compiler fuses multiply-adds.
 *
 * Readings of the paper that this file takes (each named where it is used):
 *  - Eq. 41 (D2Q5 collision) is printed with "+(ux^2+uy^2) phi" in h3 and
 *    "+(ux^2-uy^2) phi" in h4.  Expanding the central moments of Eq. 37 gives
 *    a minus sign for both; with the printed sign the equilibrium is not a
 *    fixed point of the collision.  The default here is the minus sign; the
 *    flag `as_printed` selects the printed sign (used only to show the defect).
 *  - Eq. 45 writes <K_beta|1> for the D2Q5 basis; it is read as <L_beta|1>.
 *  - Time-dependent forces/sources: the pre-collision half step uses the
 *    trapezoid average a_pre = (a(t)+a(t+1/2))/2 and the post-collision half
 *    step a_post = (a(t+1/2)+a(t+1))/2 (Sec. 6.3, where the printed argument of
 *    the second cosine is garbled).  The first moment therefore changes by
 *    (F_pre+F_post)/2 per step, which reduces to Eq. 27 for constant F.
 *  - D3Q27: the paper states the 3D method for D3Q15 only (Appendix A) and
 *    says it extends to D3Q27.  D3Q27 here is the generic central-moment
 *    procedure of orc_collide_node_generic (raw moments -> half force on the
 *    first moments -> central moments -> relaxation to the Maxwellian central
 *    moments -> raw moments -> populations), plus the post-collision force
 *    along K_1 = e_x, e_y, e_z normalised by sum_alpha e_alpha,x^2 = 18, the
 *    analogue of Eqs. 29-31 and Eq. 12A-13A.  The same procedure applied to
 *    D2Q9 reproduces Eqs. 23, 31, 32, which the tests check.
 *  - D3Q15 (Appendix A) follows Eq. 6A, Eq. 8A, Eq. 13A and the printed f^p
 *    expansion, with three corrections (the flag `as_printed` restores the
 *    first two, used only to show the defects):
 *    (i) g_9 relaxes the trace of the central second moments towards its
 *        equilibrium rho (3 c_s^2 rho); the printed bracket lacks that rho,
 *        so the rest state would not be a fixed point;
 *    (ii) the printed f^p_12 carries -g_13, but K_13 = e_x e_y e_z is +1 for
 *        e_12 = (-1, 1, -1); +g_13 is used (the populations are K g);
 *    (iii) the fourth-order bracket of g_14 contains an undefined product
 *        "kappa~_xx kappa~_yy" of the dimension rho^2; it is read as the
 *        product of the post-collision second central moments divided by rho,
 *        so that at omega = 1 kappa_xxyy relaxes to kappa~_xx kappa~_yy / rho
 *        (= c_s^4 rho at equilibrium).
 *    With time-dependent forces g_1..g_3 = (F_pre + F_post)/20 (Eq. 12A: the
 *    first-moment change is 10 g_1, and it must equal (F_pre + F_post)/2).
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define MAXQ 27

/* ------------------------------------------------------------------------ */
/* Lattices                                                                  */
/* ------------------------------------------------------------------------ */

/* D2Q9 particle velocities, Sec. 4 Eq. 15. */
static const int D2Q9_E[9][3] = {
    {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0},
    {1, 1, 0}, {-1, 1, 0}, {-1, -1, 0}, {1, -1, 0}};

/* D2Q5 particle velocities, Sec. 5 Eq. 34. */
static const int D2Q5_E[5][3] = {
    {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {0, -1, 0}};

/* D3Q15 particle velocities, Appendix A Eq. a1 (columns of |e_x>, |e_y>, |e_z>). */
static const int D3Q15_E[15][3] = {
    {0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 1}, {-1, 1, 1}, {1, -1, 1}, {-1, -1, 1}, {1, 1, -1}, {-1, 1, -1}, {1, -1, -1}, {-1, -1, -1}};

/* Monomials e_x^a e_y^b e_z^c whose moments span the D3Q15 population space:
 * the moments behind K_0..K_14 of Eq. 2A (1; e; the second-order products;
 * e_x e_y^2, e_x^2 e_y, e_x^2 e_z, e_x e_y e_z; e_x^2 e_y^2). */
static const int D3Q15_X[15][3] = {
    {0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {1, 1, 0}, {1, 0, 1}, {0, 1, 1},
    {2, 0, 0}, {0, 2, 0}, {0, 0, 2}, {1, 2, 0}, {2, 1, 0}, {2, 0, 1}, {1, 1, 1}, {2, 2, 0}};

/* Thread count of the OpenMP loops over nodes (timing only: the result of a
 * step does not depend on it, every node being computed independently). */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

int orc_q(int lattice)
{
    switch (lattice) {
    case ORC_D2Q9: return 9;
    case ORC_D3Q27: return 27;
    case ORC_D2Q5: return 5;
    case ORC_D3Q15: return 15;
    default: return 0;
    }
}

int orc_dim(int lattice)
{
    switch (lattice) {
    case ORC_D2Q9: return 2;
    case ORC_D3Q27: return 3;
    case ORC_D2Q5: return 2;
    case ORC_D3Q15: return 3;
    default: return 0;
    }
}

int orc_velocities(int lattice, int *e)
{
    int q = orc_q(lattice);
    if (q == 0) return -1;
    for (int a = 0; a < q; a++) {
        for (int d = 0; d < 3; d++) {
            if (lattice == ORC_D2Q9) e[3 * a + d] = D2Q9_E[a][d];
            else if (lattice == ORC_D2Q5) e[3 * a + d] = D2Q5_E[a][d];
            else if (lattice == ORC_D3Q15) e[3 * a + d] = D3Q15_E[a][d];
        }
        if (lattice == ORC_D3Q27) {
            e[3 * a + 0] = a % 3 - 1;
            e[3 * a + 1] = (a / 3) % 3 - 1;
            e[3 * a + 2] = a / 9 - 1;
        }
    }
    return 0;
}

/* Moment basis of a lattice: monomials e_x^a e_y^b e_z^c.
 * D2Q9: a,b in {0,1,2} (index a + 3b); D3Q27: a,b,c in {0,1,2} (a + 3b + 9c);
 * D2Q5: 1, e_x, e_y, e_x^2, e_y^2 (the monomials behind L_0..L_4 of Eq. 35);
 * D3Q15: D3Q15_X. */
typedef struct {
    int q;
    int e[MAXQ][3];
    int ex[MAXQ][3];        /* exponents of moment k */
    double M[MAXQ][MAXQ];   /* M[k][alpha] = prod_d e_d^ex_d */
    double Minv[MAXQ][MAXQ];
    int opp[MAXQ];          /* index of -e_alpha */
} basis;

static double ipow(double x, int n)
{
    double r = 1.0;
    for (int i = 0; i < n; i++) r *= x;
    return r;
}

/* Gauss-Jordan inverse with partial pivoting of an n x n matrix. */
static int invert(int n, double A[MAXQ][MAXQ], double Ainv[MAXQ][MAXQ])
{
    double W[MAXQ][2 * MAXQ];
    for (int i = 0; i < n; i++)
        for (int j = 0; j < 2 * n; j++)
            W[i][j] = (j < n) ? A[i][j] : (j - n == i ? 1.0 : 0.0);
    for (int c = 0; c < n; c++) {
        int piv = c;
        for (int r = c + 1; r < n; r++)
            if (fabs(W[r][c]) > fabs(W[piv][c])) piv = r;
        if (W[piv][c] == 0.0) return -1;
        if (piv != c)
            for (int j = 0; j < 2 * n; j++) {
                double t = W[c][j]; W[c][j] = W[piv][j]; W[piv][j] = t;
            }
        double d = W[c][c];
        for (int j = 0; j < 2 * n; j++) W[c][j] /= d;
        for (int r = 0; r < n; r++) {
            if (r == c || W[r][c] == 0.0) continue;
            double s = W[r][c];
            for (int j = 0; j < 2 * n; j++) W[r][j] -= s * W[c][j];
        }
    }
    for (int i = 0; i < n; i++)
        for (int j = 0; j < n; j++) Ainv[i][j] = W[i][n + j];
    return 0;
}

static int basis_build(int lattice, basis *B)
{
    int e[3 * MAXQ];
    memset(B, 0, sizeof(*B));
    B->q = orc_q(lattice);
    if (B->q == 0) return -1;
    orc_velocities(lattice, e);
    for (int a = 0; a < B->q; a++)
        for (int d = 0; d < 3; d++) B->e[a][d] = e[3 * a + d];
    for (int k = 0; k < B->q; k++) {
        if (lattice == ORC_D2Q5) {
            static const int X5[5][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {2, 0, 0}, {0, 2, 0}};
            for (int d = 0; d < 3; d++) B->ex[k][d] = X5[k][d];
        } else if (lattice == ORC_D3Q15) {
            for (int d = 0; d < 3; d++) B->ex[k][d] = D3Q15_X[k][d];
        } else {
            B->ex[k][0] = k % 3;
            B->ex[k][1] = (k / 3) % 3;
            B->ex[k][2] = k / 9;
        }
    }
    for (int k = 0; k < B->q; k++)
        for (int a = 0; a < B->q; a++)
            B->M[k][a] = ipow(B->e[a][0], B->ex[k][0]) * ipow(B->e[a][1], B->ex[k][1]) *
                         ipow(B->e[a][2], B->ex[k][2]);
    for (int a = 0; a < B->q; a++)
        for (int b = 0; b < B->q; b++)
            if (B->e[b][0] == -B->e[a][0] && B->e[b][1] == -B->e[a][1] && B->e[b][2] == -B->e[a][2])
                B->opp[a] = b;
    return invert(B->q, B->M, B->Minv);
}

/* Index of the moment with exponents (a,b,c), -1 if not in the basis. */
static int mindex(const basis *B, int a, int b, int c)
{
    if (B->q == 27) return a + 3 * b + 9 * c;
    if (B->q == 9) return c == 0 ? a + 3 * b : -1;
    for (int k = 0; k < B->q; k++)
        if (B->ex[k][0] == a && B->ex[k][1] == b && B->ex[k][2] == c) return k;
    return -1;
}

static double binom(int n, int k)
{
    static const double C[3][3] = {{1, 0, 0}, {1, 1, 0}, {1, 2, 1}};
    return C[n][k];
}

/* Moments about velocity s of a moment vector given about the origin:
 * out_abc = sum_{i<=a, j<=b, l<=c} C(a,i) C(b,j) C(c,l) (-s_x)^(a-i) (-s_y)^(b-j)
 *           (-s_z)^(c-l) in_ijl.
 * With s = u this turns raw moments into central moments (Eq. 19 vs Eq. 21);
 * with s = -u it turns central moments back into raw moments. */
static void shift_moments(const basis *B, const double *in, const double s[3], double *out)
{
    for (int k = 0; k < B->q; k++) {
        int a = B->ex[k][0], b = B->ex[k][1], c = B->ex[k][2];
        double acc = 0.0;
        for (int i = 0; i <= a; i++)
            for (int j = 0; j <= b; j++)
                for (int l = 0; l <= c; l++) {
                    int kk = mindex(B, i, j, l);
                    if (kk < 0) continue; /* D2Q5, D3Q15: the lower monomials are all present */
                    acc += binom(a, i) * binom(b, j) * binom(c, l) * ipow(-s[0], a - i) *
                           ipow(-s[1], b - j) * ipow(-s[2], c - l) * in[kk];
                }
        out[k] = acc;
    }
}

/* Central-moment equilibria of Eq. 20 (D2Q9) / Eq. 39 (D2Q5), and their
 * Maxwellian continuation for D3Q27 and D3Q15: rho * prod_d (c_s^2 if exponent
 * 2, 1 if 0, 0 if odd) with c_s^2 = 1/3.  For D3Q15 these are the central
 * moments that the collision of Eq. 6A reaches at omega = 1 (with the
 * readings above), so the equilibrium built from them is the image of an
 * omega = 1 collision. */
static double central_eq(const basis *B, int k, double rho)
{
    double v = rho;
    for (int d = 0; d < 3; d++) {
        if (B->ex[k][d] == 1) return 0.0;
        if (B->ex[k][d] == 2) v *= 1.0 / 3.0;
    }
    return v;
}

/* ------------------------------------------------------------------------ */
/* Collision: D2Q9 as printed in the paper (Sec. 4)                          */
/* ------------------------------------------------------------------------ */

static void collide_d2q9_paper(const double *om, const double f[9], const double Fpre[2],
                               const double Fpost[2], double fp[9])
{
    const double ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
    const double ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};

    /* Step (vi) of the algorithm / Eq. 24: density and output momentum. */
    double rho = 0.0, jx = 0.0, jy = 0.0;
    for (int a = 0; a < 9; a++) {
        rho += f[a];
        jx += f[a] * ex[a];
        jy += f[a] * ey[a];
    }
    /* Step (i) / Eq. 25: pre-collision half force step. */
    double ux = (jx + Fpre[0] / 2.0) / rho;
    double uy = (jy + Fpre[1] / 2.0) / rho;

    /* Raw moments, Eq. 21. */
    double kxx = 0, kyy = 0, kxy = 0, kxxy = 0, kxyy = 0, kxxyy = 0;
    for (int a = 0; a < 9; a++) {
        kxx += f[a] * ex[a] * ex[a];
        kyy += f[a] * ey[a] * ey[a];
        kxy += f[a] * ex[a] * ey[a];
        kxxy += f[a] * ex[a] * ex[a] * ey[a];
        kxyy += f[a] * ex[a] * ey[a] * ey[a];
        kxxyy += f[a] * ex[a] * ex[a] * ey[a] * ey[a];
    }

    /* Step (ii) / Eq. 23: cascaded change of moments. */
    double w3 = om[3], w4 = om[4], w5 = om[5], w6 = om[6], w7 = om[7], w8 = om[8];
    double g3 = w3 / 12.0 * (2.0 / 3.0 * rho + rho * (ux * ux + uy * uy) - (kxx + kyy));
    double g4 = w4 / 4.0 * (rho * (ux * ux - uy * uy) - (kxx - kyy));
    double g5 = w5 / 4.0 * (rho * ux * uy - kxy);
    double g6 = w6 / 4.0 * (2.0 * rho * ux * ux * uy + kxxy - 2.0 * ux * kxy - uy * kxx)
                - 0.5 * uy * (3.0 * g3 + g4) - 2.0 * ux * g5;
    double g7 = w7 / 4.0 * (2.0 * rho * ux * uy * uy + kxyy - 2.0 * uy * kxy - ux * kyy)
                - 0.5 * ux * (3.0 * g3 - g4) - 2.0 * uy * g5;
    double g8 = w8 / 4.0 * (1.0 / 9.0 * rho + 3.0 * rho * ux * ux * uy * uy
                            - (kxxyy - 2.0 * ux * kxyy - 2.0 * uy * kxxy + ux * ux * kyy
                               + uy * uy * kxx + 4.0 * ux * uy * kxy))
                - 2.0 * g3 - 0.5 * uy * uy * (3.0 * g3 + g4) - 0.5 * ux * ux * (3.0 * g3 - g4)
                - 4.0 * ux * uy * g5 - 2.0 * uy * g6 - 2.0 * ux * g7;

    /* Step (iii) / Eqs. 27-31: mass and momentum are collision invariants
     * (g0 = 0); the post-collision half force step sets the first-moment change
     * so that rho u^p = rho u^o + (F_pre + F_post)/2, i.e. 6 g1 = (F_pre+F_post)/2. */
    double g0 = 0.0;
    double g1 = (Fpre[0] + Fpost[0]) / 2.0 / 6.0;
    double g2 = (Fpre[1] + Fpost[1]) / 2.0 / 6.0;

    /* Step (iv) / Eq. 32: post-collision populations f + K g. */
    fp[0] = f[0] + (g0 - 4.0 * (g3 - g8));
    fp[1] = f[1] + (g0 + g1 - g3 + g4 + 2.0 * (g7 - g8));
    fp[2] = f[2] + (g0 + g2 - g3 - g4 + 2.0 * (g6 - g8));
    fp[3] = f[3] + (g0 - g1 - g3 + g4 - 2.0 * (g7 + g8));
    fp[4] = f[4] + (g0 - g2 - g3 - g4 - 2.0 * (g6 + g8));
    fp[5] = f[5] + (g0 + g1 + g2 + 2.0 * g3 + g5 - g6 - g7 + g8);
    fp[6] = f[6] + (g0 - g1 + g2 + 2.0 * g3 - g5 - g6 + g7 + g8);
    fp[7] = f[7] + (g0 - g1 - g2 + 2.0 * g3 + g5 + g6 + g7 + g8);
    fp[8] = f[8] + (g0 + g1 - g2 + 2.0 * g3 - g5 + g6 - g7 + g8);
}

/* ------------------------------------------------------------------------ */
/* Collision: D2Q5 passive scalar with source (Sec. 5)                       */
/* ------------------------------------------------------------------------ */

static void collide_d2q5_paper(const double *om, int as_printed, const double g[5], double Spre,
                               double Spost, double ux, double uy, double gp[5])
{
    const double ex[5] = {0, 1, 0, -1, 0};
    const double ey[5] = {0, 0, 1, 0, -1};
    const double cs2 = 1.0 / 3.0;

    /* Eq. 42: output scalar. */
    double phio = 0.0;
    for (int a = 0; a < 5; a++) phio += g[a];
    /* Eq. 43: pre-collision half source step. */
    double phi = phio + Spre / 2.0;

    /* Raw moments, Eq. 38. */
    double kx = 0, ky = 0, kxx = 0, kyy = 0;
    for (int a = 0; a < 5; a++) {
        kx += g[a] * ex[a];
        ky += g[a] * ey[a];
        kxx += g[a] * ex[a] * ex[a];
        kyy += g[a] * ey[a] * ey[a];
    }

    /* Eq. 41 (minus sign on the u^2 phi terms unless as_printed). */
    double sg = as_printed ? 1.0 : -1.0;
    double h1 = om[1] / 2.0 * (phi * ux - kx);
    double h2 = om[2] / 2.0 * (phi * uy - ky);
    double h3 = om[3] / 4.0 * (2.0 * cs2 * phi - (kxx + kyy) + 2.0 * (ux * kx + uy * ky)
                               + sg * (ux * ux + uy * uy) * phi)
                + ux * h1 + uy * h2;
    double h4 = om[4] / 4.0 * (-(kxx - kyy) + 2.0 * (ux * kx - uy * ky)
                               + sg * (ux * ux - uy * uy) * phi)
                + ux * h1 - uy * h2;

    /* Eqs. 44-47 (with <L_beta|1>): phi^p = phi^o + (S_pre+S_post)/2 = phi^o + 5 h0. */
    double h0 = (Spre + Spost) / 2.0 / 5.0;

    /* Eq. 48. */
    gp[0] = g[0] + (h0 - 4.0 * h3);
    gp[1] = g[1] + (h0 + h1 + h3 + h4);
    gp[2] = g[2] + (h0 + h2 + h3 - h4);
    gp[3] = g[3] + (h0 - h1 + h3 + h4);
    gp[4] = g[4] + (h0 - h2 + h3 - h4);
}

/* ------------------------------------------------------------------------ */
/* Collision: D3Q15 (Appendix A)                                             */
/* ------------------------------------------------------------------------ */

static void collide_d3q15_paper(const double *om, int as_printed, const double f[15], const double Fpre[3],
                                const double Fpost[3], double fp[15])
{
    /* Rates of Eq. 6A from the grouped parameters. */
    const double w4 = om[2], w5 = om[2], w6 = om[2], w7 = om[2], w8 = om[2];
    const double w9 = om[1];
    const double w10 = om[3], w11 = om[3], w12 = om[3], w13 = om[3];
    const double w14 = om[4];

    /* Density and output momentum (Eq. 7A); raw moments (Eq. g8). */
    double rho = 0, jx = 0, jy = 0, jz = 0;
    double kxx = 0, kyy = 0, kzz = 0, kxy = 0, kxz = 0, kyz = 0;
    double kxyy = 0, kxxy = 0, kxxz = 0, kxyz = 0, kxxyy = 0;
    for (int a = 0; a < 15; a++) {
        const double ex = D3Q15_E[a][0], ey = D3Q15_E[a][1], ez = D3Q15_E[a][2];
        rho += f[a];
        jx += f[a] * ex;
        jy += f[a] * ey;
        jz += f[a] * ez;
        kxx += f[a] * ex * ex;
        kyy += f[a] * ey * ey;
        kzz += f[a] * ez * ez;
        kxy += f[a] * ex * ey;
        kxz += f[a] * ex * ez;
        kyz += f[a] * ey * ez;
        kxyy += f[a] * ex * ey * ey;
        kxxy += f[a] * ex * ex * ey;
        kxxz += f[a] * ex * ex * ez;
        kxyz += f[a] * ex * ey * ez;
        kxxyy += f[a] * ex * ex * ey * ey;
    }
    /* Pre-collision half force step (Eq. 8A). */
    const double ux = (jx + Fpre[0] / 2.0) / rho;
    const double uy = (jy + Fpre[1] / 2.0) / rho;
    const double uz = (jz + Fpre[2] / 2.0) / rho;

    /* Cascaded change of moments, Eq. 6A (corrections (i) and (iii), see the
     * file header). */
    const double g4 = w4 / 8.0 * (-kxy + rho * ux * uy);
    const double g5 = w5 / 8.0 * (-kxz + rho * ux * uz);
    const double g6 = w6 / 8.0 * (-kyz + rho * uy * uz);
    const double g7 = w7 / 4.0 * (-(kxx - kyy) + rho * (ux * ux - uy * uy));
    const double g8 = w8 / 12.0 * (-(kxx + kyy - 2.0 * kzz) + rho * (ux * ux + uy * uy - 2.0 * uz * uz));
    const double trace_eq = as_printed ? 0.0 : rho;
    const double g9 = w9 / 18.0 * (trace_eq - (kxx + kyy + kzz) + rho * (ux * ux + uy * uy + uz * uz));
    const double g10 = w10 / 16.0 * (-kxyy + 2.0 * uy * kxy + ux * kyy - 2.0 * rho * ux * uy * uy)
                       + uy * g4 + ux / 8.0 * (-g7 + g8 + 3.0 * g9);
    const double g11 = w11 / 16.0 * (-kxxy + 2.0 * ux * kxy + uy * kxx - 2.0 * rho * ux * ux * uy)
                       + ux * g4 + uy / 8.0 * (g7 + g8 + 3.0 * g9);
    const double g12 = w12 / 16.0 * (-kxxz + 2.0 * ux * kxz + uz * kxx - 2.0 * rho * ux * ux * uz)
                       + ux * g5 + uz / 8.0 * (g7 + g8 + 3.0 * g9);
    const double g13 = w13 / 8.0 * (-kxyz + ux * kyz + uy * kxz + uz * kxy - 2.0 * rho * ux * uy * uz)
                       + uz * g4 + uy * g5 + ux * g6;
    /* Post-collision second central moments: the pre-collision central
     * moments about u plus the changes K_7, K_8, K_9 make to them (K_4..K_6
     * leave the diagonal ones unchanged): xx gains 2 g7 + 2 g8 + 6 g9, yy
     * gains -2 g7 + 2 g8 + 6 g9. */
    const double cxx = kxx - rho * ux * ux, cyy = kyy - rho * uy * uy;
    const double cxx_post = cxx + 2.0 * g7 + 2.0 * g8 + 6.0 * g9;
    const double cyy_post = cyy - 2.0 * g7 + 2.0 * g8 + 6.0 * g9;
    const double g14 = w14 / 16.0 * (-kxxyy + 2.0 * ux * kxyy + 2.0 * uy * kxxy - ux * ux * kyy - uy * uy * kxx
                                     - 4.0 * ux * uy * kxy + cxx_post * cyy_post / rho
                                     + 3.0 * rho * ux * ux * uy * uy)
                       - 2.0 * ux * uy * g4 + (ux * ux - uy * uy) / 8.0 * g7 - (ux * ux + uy * uy) / 8.0 * g8
                       + (3.0 / 8.0 * (-ux * ux - uy * uy) - 0.5) * g9 + 2.0 * ux * g10 + 2.0 * uy * g11;

    /* Mass is conserved (g0 = 0); the first-moment change 10 g_d equals the
     * mean force of the two half steps (Eqs. 10A-13A). */
    const double g0 = 0.0;
    const double g1 = (Fpre[0] + Fpost[0]) / 2.0 / 10.0;
    const double g2 = (Fpre[1] + Fpost[1]) / 2.0 / 10.0;
    const double g3 = (Fpre[2] + Fpost[2]) / 2.0 / 10.0;

    /* Post-collision populations (the expansion of f + K g ending Appendix A;
     * correction (ii) in f^p_12). */
    const double s12 = as_printed ? -1.0 : 1.0;
    fp[0] = f[0] + (g0 - 2.0 * g9 + 32.0 * g14);
    fp[1] = f[1] + (g0 + g1 + g7 + g8 - g9 - 8.0 * g10 - 8.0 * g14);
    fp[2] = f[2] + (g0 - g1 + g7 + g8 - g9 + 8.0 * g10 - 8.0 * g14);
    fp[3] = f[3] + (g0 + g2 - g7 + g8 - g9 - 8.0 * g11 - 8.0 * g14);
    fp[4] = f[4] + (g0 - g2 - g7 + g8 - g9 + 8.0 * g11 - 8.0 * g14);
    fp[5] = f[5] + (g0 + g3 - 2.0 * g8 - g9 - 8.0 * g12 - 8.0 * g14);
    fp[6] = f[6] + (g0 - g3 - 2.0 * g8 - g9 + 8.0 * g12 - 8.0 * g14);
    fp[7] = f[7] + (g0 + g1 + g2 + g3 + g4 + g5 + g6 + g9 + 2.0 * g10 + 2.0 * g11 + 2.0 * g12 + g13 + 2.0 * g14);
    fp[8] = f[8] + (g0 - g1 + g2 + g3 - g4 - g5 + g6 + g9 - 2.0 * g10 + 2.0 * g11 + 2.0 * g12 - g13 + 2.0 * g14);
    fp[9] = f[9] + (g0 + g1 - g2 + g3 - g4 + g5 - g6 + g9 + 2.0 * g10 - 2.0 * g11 + 2.0 * g12 - g13 + 2.0 * g14);
    fp[10] = f[10] + (g0 - g1 - g2 + g3 + g4 - g5 - g6 + g9 - 2.0 * g10 - 2.0 * g11 + 2.0 * g12 + g13 + 2.0 * g14);
    fp[11] = f[11] + (g0 + g1 + g2 - g3 + g4 - g5 - g6 + g9 + 2.0 * g10 + 2.0 * g11 - 2.0 * g12 - g13 + 2.0 * g14);
    fp[12] = f[12] + (g0 - g1 + g2 - g3 - g4 + g5 - g6 + g9 - 2.0 * g10 + 2.0 * g11 - 2.0 * g12 + s12 * g13
                      + 2.0 * g14);
    fp[13] = f[13] + (g0 + g1 - g2 - g3 - g4 - g5 + g6 + g9 + 2.0 * g10 - 2.0 * g11 - 2.0 * g12 + g13 + 2.0 * g14);
    fp[14] = f[14] + (g0 - g1 - g2 - g3 + g4 + g5 + g6 + g9 - 2.0 * g10 - 2.0 * g11 - 2.0 * g12 - g13 + 2.0 * g14);
}

/* ------------------------------------------------------------------------ */
/* Collision: generic central-moment procedure (D2Q9, D3Q27)                 */
/* ------------------------------------------------------------------------ */

/* Relaxation of central moments kappa (first-order entries zero after the
 * pre-collision half force), in place.
 * D2Q9 (rates numbered as in Eq. 23): trace kxx+kyy with omega_3 towards
 *   2 c_s^2 rho, kxx-kyy with omega_4 and kxy with omega_5 towards 0, kxxy with
 *   omega_6, kxyy with omega_7 towards 0, kxxyy with omega_8 towards c_s^4 rho.
 * D3Q27: trace with omega[1] towards 3 c_s^2 rho; kxx-kyy, kxx-kzz, kxy, kxz,
 *   kyz with omega[2] towards 0; every central moment of order n = 3..6 with
 *   omega[n] towards its Maxwellian value. */
static void relax_central(int lattice, const basis *B, const double *om, double rho, double *kap)
{
    double out[MAXQ];
    memcpy(out, kap, sizeof(double) * B->q);
    if (lattice == ORC_D2Q9) {
        int i20 = mindex(B, 2, 0, 0), i02 = mindex(B, 0, 2, 0), i11 = mindex(B, 1, 1, 0);
        int i21 = mindex(B, 2, 1, 0), i12 = mindex(B, 1, 2, 0), i22 = mindex(B, 2, 2, 0);
        double T = kap[i20] + kap[i02], D = kap[i20] - kap[i02];
        double Ts = T + om[3] * (2.0 / 3.0 * rho - T);
        double Ds = D + om[4] * (0.0 - D);
        out[i20] = (Ts + Ds) / 2.0;
        out[i02] = (Ts - Ds) / 2.0;
        out[i11] = kap[i11] + om[5] * (0.0 - kap[i11]);
        out[i21] = kap[i21] + om[6] * (0.0 - kap[i21]);
        out[i12] = kap[i12] + om[7] * (0.0 - kap[i12]);
        out[i22] = kap[i22] + om[8] * (central_eq(B, i22, rho) - kap[i22]);
    } else {
        int i200 = mindex(B, 2, 0, 0), i020 = mindex(B, 0, 2, 0), i002 = mindex(B, 0, 0, 2);
        double T = kap[i200] + kap[i020] + kap[i002];
        double D1 = kap[i200] - kap[i020], D2 = kap[i200] - kap[i002];
        double Ts = T + om[1] * (rho - T);
        double D1s = D1 + om[2] * (0.0 - D1), D2s = D2 + om[2] * (0.0 - D2);
        out[i200] = (Ts + D1s + D2s) / 3.0;
        out[i020] = out[i200] - D1s;
        out[i002] = out[i200] - D2s;
        for (int k = 0; k < B->q; k++) {
            int n = B->ex[k][0] + B->ex[k][1] + B->ex[k][2];
            int diag2 = (n == 2) && (B->ex[k][0] == 2 || B->ex[k][1] == 2 || B->ex[k][2] == 2);
            if (n == 2 && !diag2) out[k] = kap[k] + om[2] * (0.0 - kap[k]);
            if (n >= 3) out[k] = kap[k] + om[n] * (central_eq(B, k, rho) - kap[k]);
        }
    }
    memcpy(kap, out, sizeof(double) * B->q);
}

static void collide_generic(int lattice, const basis *B, const double *om, const double *f,
                            const double *Fpre, const double *Fpost, double *fp)
{
    int q = B->q, dim = orc_dim(lattice);
    double m[MAXQ], kap[MAXQ], mstar[MAXQ], dm[MAXQ];
    /* Raw moments (Eq. 21 and its 3D analogue). */
    for (int k = 0; k < q; k++) {
        m[k] = 0.0;
        for (int a = 0; a < q; a++) m[k] += B->M[k][a] * f[a];
    }
    /* Pre-collision half force on the first moments (Eq. 25 / Eq. 8A). */
    int i1[3] = {mindex(B, 1, 0, 0), mindex(B, 0, 1, 0), mindex(B, 0, 0, 1)};
    for (int d = 0; d < dim; d++) m[i1[d]] += Fpre[d] / 2.0;
    double rho = m[mindex(B, 0, 0, 0)];
    double u[3] = {0, 0, 0};
    for (int d = 0; d < dim; d++) u[d] = m[i1[d]] / rho;
    /* Central moments (Eq. 19), relaxation, back to raw moments. */
    shift_moments(B, m, u, kap);
    relax_central(lattice, B, om, rho, kap);
    double mu[3] = {-u[0], -u[1], -u[2]};
    shift_moments(B, kap, mu, mstar);
    /* Collision change in population space (mass and momentum unchanged). */
    for (int k = 0; k < q; k++) dm[k] = mstar[k] - m[k];
    for (int d = 0; d < dim; d++) dm[i1[d]] = 0.0;
    dm[mindex(B, 0, 0, 0)] = 0.0;
    /* Post-collision half force along K_1 = e (Eqs. 29-31 / 12A-13A). */
    double norm = 0.0;
    for (int a = 0; a < q; a++) norm += (double)(B->e[a][0] * B->e[a][0]);
    for (int a = 0; a < q; a++) {
        double df = 0.0;
        for (int k = 0; k < q; k++) df += B->Minv[a][k] * dm[k];
        double fe = 0.0;
        for (int d = 0; d < dim; d++) fe += (Fpre[d] + Fpost[d]) / 2.0 / norm * B->e[a][d];
        fp[a] = f[a] + df + fe;
    }
}

/* ------------------------------------------------------------------------ */
/* Public entry points                                                       */
/* ------------------------------------------------------------------------ */

static int check_params(const orc_params *p)
{
    int q = orc_q(p->lattice);
    if (q == 0) return -1;
    for (int d = 0; d < 3; d++)
        if (p->n[d] < 1) return -1;
    if (orc_dim(p->lattice) == 2 && p->n[2] != 1) return -1;
    return 0;
}

int orc_collide_node(const orc_params *p, const double *fin, const double *Fpre,
                     const double *Fpost, const double *uadv, double *fout)
{
    if (check_params(p)) return -1;
    if (p->lattice == ORC_D2Q9 && !p->generic) {
        collide_d2q9_paper(p->omega, fin, Fpre, Fpost, fout);
        return 0;
    }
    if (p->lattice == ORC_D2Q5) {
        if (!uadv) return -1; /* the scalar's collision needs the advecting velocity */
        collide_d2q5_paper(p->omega, p->as_printed, fin, Fpre[0], Fpost[0], uadv[0], uadv[1], fout);
        return 0;
    }
    if (p->lattice == ORC_D3Q15) {
        collide_d3q15_paper(p->omega, p->as_printed, fin, Fpre, Fpost, fout);
        return 0;
    }
    return orc_collide_node_generic(p, fin, Fpre, Fpost, fout);
}

int orc_collide_node_generic(const orc_params *p, const double *fin, const double *Fpre,
                             const double *Fpost, double *fout)
{
    basis B;
    if (p->lattice == ORC_D2Q5 || p->lattice == ORC_D3Q15) return -1;
    if (basis_build(p->lattice, &B)) return -1;
    collide_generic(p->lattice, &B, p->omega, fin, Fpre, Fpost, fout);
    return 0;
}

int orc_equilibrium(const orc_params *p, const double *rho, const double *u, double *f)
{
    basis B;
    if (check_params(p) || basis_build(p->lattice, &B)) return -1;
    long N = (long)p->n[0] * p->n[1] * p->n[2];
    int dim = orc_dim(p->lattice);
    for (long i = 0; i < N; i++) {
        double kap[MAXQ], m[MAXQ], mu[3] = {0, 0, 0};
        for (int d = 0; d < dim; d++) mu[d] = -u[d * N + i];
        for (int k = 0; k < B.q; k++) kap[k] = central_eq(&B, k, rho[i]);
        shift_moments(&B, kap, mu, m);
        for (int a = 0; a < B.q; a++) {
            double acc = 0.0;
            for (int k = 0; k < B.q; k++) acc += B.Minv[a][k] * m[k];
            f[a * N + i] = acc;
        }
    }
    return 0;
}

/* Streaming, Eq. 22b / Eq. 40b: f_alpha(x) = f^p_alpha(x - e_alpha).  On an
 * axis with walls, a source node outside the domain means the population has
 * hit the wall half way between the nodes and comes back reversed
 * (stationary halfway bounce-back, Sec. 6.1): f_alpha(x) = f^p_opp(alpha)(x). */
static void stream(const orc_params *p, const basis *B, const double *fp, double *f)
{
    long nx = p->n[0], ny = p->n[1], nz = p->n[2], N = nx * ny * nz;
    for (int a = 0; a < B->q; a++) {
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (N >= 16384)
#endif
        for (long i = 0; i < N; i++) {
            long x = i % nx, y = (i / nx) % ny, z = i / (nx * ny);
            long s[3] = {x - B->e[a][0], y - B->e[a][1], z - B->e[a][2]};
            long n[3] = {nx, ny, nz};
            int outside = 0;
            for (int d = 0; d < 3; d++) {
                if (s[d] < 0 || s[d] >= n[d]) {
                    if (p->wall[d]) outside = 1;
                    else s[d] = (s[d] + n[d]) % n[d];
                }
            }
            if (outside) f[a * N + i] = fp[B->opp[a] * N + i];
            else f[a * N + i] = fp[a * N + s[0] + nx * (s[1] + ny * s[2])];
        }
    }
}

int orc_run(const orc_params *p, double *f, double *work, long nsteps, const double *P,
            const double *a, const double *uadv)
{
    basis B;
    if (check_params(p) || basis_build(p->lattice, &B)) return -1;
    if (p->lattice == ORC_D2Q5 && uadv == NULL) return -1;
    long N = (long)p->n[0] * p->n[1] * p->n[2];
    int q = B.q, dim = orc_dim(p->lattice);
    int ncomp = (p->lattice == ORC_D2Q5) ? 1 : dim;
    for (long t = 0; t < nsteps; t++) {
        double apre = a ? a[2 * t] : 1.0, apost = a ? a[2 * t + 1] : 1.0;
        /* Collision with the two half force/source steps at every node. */
#ifdef _OPENMP
#pragma omp parallel for schedule(static) if (N >= 16384)
#endif
        for (long i = 0; i < N; i++) {
            double fin[MAXQ], fout[MAXQ], Fpre[3] = {0, 0, 0}, Fpost[3] = {0, 0, 0};
            for (int k = 0; k < q; k++) fin[k] = f[k * N + i];
            if (P)
                for (int d = 0; d < ncomp; d++) {
                    Fpre[d] = apre * P[d * N + i];
                    Fpost[d] = apost * P[d * N + i];
                }
            if (p->lattice == ORC_D2Q9 && !p->generic)
                collide_d2q9_paper(p->omega, fin, Fpre, Fpost, fout);
            else if (p->lattice == ORC_D2Q5)
                collide_d2q5_paper(p->omega, p->as_printed, fin, Fpre[0], Fpost[0], uadv[i],
                                   uadv[N + i], fout);
            else if (p->lattice == ORC_D3Q15)
                collide_d3q15_paper(p->omega, p->as_printed, fin, Fpre, Fpost, fout);
            else
                collide_generic(p->lattice, &B, p->omega, fin, Fpre, Fpost, fout);
            for (int k = 0; k < q; k++) work[k * N + i] = fout[k];
        }
        /* Streaming. */
        stream(p, &B, work, f);
    }
    return 0;
}

int orc_moments(const orc_params *p, const double *f, const double *P, double a_pre, double *rho,
                double *u)
{
    basis B;
    if (check_params(p) || basis_build(p->lattice, &B)) return -1;
    long N = (long)p->n[0] * p->n[1] * p->n[2];
    int dim = orc_dim(p->lattice);
    for (long i = 0; i < N; i++) {
        double r = 0.0, j[3] = {0, 0, 0};
        for (int a = 0; a < B.q; a++) {
            r += f[a * N + i];
            for (int d = 0; d < dim; d++) j[d] += f[a * N + i] * B.e[a][d];
        }
        if (p->lattice == ORC_D2Q5) {
            /* Eq. 42 plus the pre-collision half source of Eq. 43. */
            rho[i] = P ? r + a_pre * P[i] / 2.0 : r;
        } else {
            /* Eq. 24 plus the pre-collision half force of Eq. 25. */
            rho[i] = r;
            for (int d = 0; d < dim; d++)
                u[d * N + i] = (P ? j[d] + a_pre * P[d * N + i] / 2.0 : j[d]) / r;
        }
    }
    return 0;
}

int orc_strain_rate(const orc_params *p, const double *f, const double *P, double a_pre, double rho0, double *S)
{
    basis B;
    if (check_params(p) || basis_build(p->lattice, &B) || p->lattice == ORC_D2Q5) return -1;
    long N = (long)p->n[0] * p->n[1] * p->n[2];
    int dim = orc_dim(p->lattice);
    double ws, wd, wb;
    if (p->lattice == ORC_D2Q9) {
        ws = p->omega[5];
        wd = p->omega[4];
        wb = p->omega[3];
    } else {
        ws = p->omega[2];
        wd = p->omega[2];
        wb = p->omega[1];
    }
    const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};
    const int ncomp = dim == 2 ? 3 : 6;
    for (long i = 0; i < N; i++) {
        double rho = 0.0, j[3] = {0, 0, 0}, m2[3][3] = {{0}};
        for (int a = 0; a < B.q; a++) {
            const double fa = f[a * N + i];
            rho += fa;
            for (int d = 0; d < dim; d++) {
                j[d] += fa * B.e[a][d];
                for (int e = 0; e < dim; e++) m2[d][e] += fa * B.e[a][d] * B.e[a][e];
            }
        }
        double u[3] = {0, 0, 0};
        for (int d = 0; d < dim; d++) u[d] = (P ? j[d] + a_pre * P[d * N + i] / 2.0 : j[d]) / rho;
        double Pi[3][3];
        for (int d = 0; d < dim; d++)
            for (int e = 0; e < dim; e++)
                Pi[d][e] = m2[d][e] - rho * u[d] * u[e] - (d == e ? rho / 3.0 : 0.0);
        double T = 0.0;
        for (int d = 0; d < dim; d++) T += Pi[d][d];
        for (int c = 0; c < ncomp; c++) {
            int a, b;
            if (dim == 2) {
                a = c == 2 ? 0 : c;
                b = c == 2 ? 1 : c;
            } else {
                a = pa[c];
                b = pb[c];
            }
            double v;
            if (a != b) v = -1.5 * ws / rho0 * Pi[a][b];
            else v = -1.5 / rho0 * (wd * (Pi[a][a] - T / dim) + wb * T / dim);
            S[c * N + i] = v;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Context API (lbmref_*): the oracle behind the same calls as the library   */
/* ------------------------------------------------------------------------ */

struct lbmref_ctx {
    orc_params p;
    long N;
    int q, dim;
    double *f, *work;  /* f(t), [q][N]; scratch */
    double *P;         /* force shape [dim][N] or source shape [N]; NULL = none */
    double *uadv;      /* D2Q5 advecting velocity [2][N] (zero by default) */
    double *uprev;     /* velocity (flow) or scalar (D2Q5) at the previous lbmref_reduce */
    int have_prev, initialised;
    lbmref_envelope_fn env;
    void *user;
    long step;
};

static double env_at(const lbmref_ctx *c, double t) { return c->env ? c->env(t, c->user) : 1.0; }

int lbmref_create(lbmref_ctx **out, int lattice, int nx, int ny, int nz, const double omega[9],
                  const int wall[3])
{
    if (!out) return LBMREF_EINVAL;
    *out = NULL;
    if (orc_q(lattice) == 0 || nx < 1 || ny < 1 || nz < 1 || !omega) return LBMREF_EINVAL;
    if (orc_dim(lattice) == 2 && nz != 1) return LBMREF_EINVAL;
    const int n[3] = {nx, ny, nz};
    for (int d = 0; d < 3; d++) {
        const int w = wall ? wall[d] : 0;
        if (w != 0 && w != 1) return LBMREF_EINVAL;
        if (w && (n[d] < 2 || (orc_dim(lattice) == 2 && d == 2))) return LBMREF_EINVAL;
    }
    for (int k = 0; k < 9; k++)
        if (!(omega[k] >= 0.0 && omega[k] < 2.0)) return LBMREF_EINVAL;
    lbmref_ctx *c = (lbmref_ctx *)calloc(1, sizeof(lbmref_ctx));
    if (!c) return LBMREF_ENOMEM;
    c->p.lattice = lattice;
    for (int d = 0; d < 3; d++) {
        c->p.n[d] = n[d];
        c->p.wall[d] = wall ? wall[d] : 0;
    }
    for (int k = 0; k < 9; k++) c->p.omega[k] = omega[k];
    c->N = (long)nx * ny * nz;
    c->q = orc_q(lattice);
    c->dim = orc_dim(lattice);
    c->f = (double *)calloc((size_t)c->q * c->N, sizeof(double));
    c->work = (double *)calloc((size_t)c->q * c->N, sizeof(double));
    c->uprev = (double *)calloc((size_t)3 * c->N, sizeof(double));
    if (lattice == ORC_D2Q5) c->uadv = (double *)calloc((size_t)2 * c->N, sizeof(double));
    if (!c->f || !c->work || !c->uprev || (lattice == ORC_D2Q5 && !c->uadv)) {
        lbmref_destroy(c);
        return LBMREF_ENOMEM;
    }
    *out = c;
    return LBMREF_OK;
}

void lbmref_destroy(lbmref_ctx *c)
{
    if (!c) return;
    free(c->f);
    free(c->work);
    free(c->P);
    free(c->uadv);
    free(c->uprev);
    free(c);
}

int lbmref_init_equilibrium(lbmref_ctx *c, double rho0, const double u0[3], const double *rho, const double *u)
{
    if (!c || (c->p.lattice != ORC_D2Q5 && !rho && !(rho0 > 0.0))) return LBMREF_EINVAL;
    const long N = c->N;
    double *r = (double *)malloc((size_t)N * sizeof(double));
    double *v = (double *)malloc((size_t)3 * N * sizeof(double));
    if (!r || !v) {
        free(r);
        free(v);
        return LBMREF_ENOMEM;
    }
    for (long i = 0; i < N; i++) r[i] = rho ? rho[i] : rho0;
    for (int d = 0; d < c->dim; d++)
        for (long i = 0; i < N; i++) v[d * N + i] = u ? u[d * N + i] : (u0 ? u0[d] : 0.0);
    const int rc = orc_equilibrium(&c->p, r, v, c->f);
    free(r);
    free(v);
    if (rc) return LBMREF_EINVAL;
    c->step = 0;
    c->have_prev = 0;
    c->initialised = 1;
    return LBMREF_OK;
}

static int set_shape(lbmref_ctx *c, const double *S, int ncomp)
{
    if (!S) {
        free(c->P);
        c->P = NULL;
        return LBMREF_OK;
    }
    double *P = (double *)malloc((size_t)ncomp * c->N * sizeof(double));
    if (!P) return LBMREF_ENOMEM;
    memcpy(P, S, (size_t)ncomp * c->N * sizeof(double));
    free(c->P);
    c->P = P;
    return LBMREF_OK;
}

int lbmref_set_force(lbmref_ctx *c, const double *P)
{
    if (!c || c->p.lattice == ORC_D2Q5) return LBMREF_EINVAL;
    return set_shape(c, P, c->dim);
}

int lbmref_set_source(lbmref_ctx *c, const double *S)
{
    if (!c || c->p.lattice != ORC_D2Q5) return LBMREF_EINVAL;
    return set_shape(c, S, 1);
}

int lbmref_set_velocity(lbmref_ctx *c, const double *u)
{
    if (!c || c->p.lattice != ORC_D2Q5) return LBMREF_EINVAL;
    if (u) memcpy(c->uadv, u, (size_t)2 * c->N * sizeof(double));
    else memset(c->uadv, 0, (size_t)2 * c->N * sizeof(double));
    return LBMREF_OK;
}

int lbmref_set_envelope(lbmref_ctx *c, lbmref_envelope_fn fn, void *user)
{
    if (!c) return LBMREF_EINVAL;
    c->env = fn;
    c->user = user;
    return LBMREF_OK;
}

/* Trapezoid averages of the envelope over the two half steps (Sec. 6.3):
 * a_pre = (a(t) + a(t+1/2))/2, a_post = (a(t+1/2) + a(t+1))/2. */
int lbmref_step(lbmref_ctx *c, long n)
{
    if (!c || n < 0) return LBMREF_EINVAL;
    if (!c->initialised) return LBMREF_ESTATE;
    if (n == 0) return LBMREF_OK;
    double *a = (double *)malloc((size_t)2 * n * sizeof(double));
    if (!a) return LBMREF_ENOMEM;
    for (long k = 0; k < n; k++) {
        const double t = (double)(c->step + k);
        const double a0 = env_at(c, t), ah = env_at(c, t + 0.5), a1 = env_at(c, t + 1.0);
        a[2 * k] = 0.5 * (a0 + ah);
        a[2 * k + 1] = 0.5 * (ah + a1);
    }
    const int rc = orc_run(&c->p, c->f, c->work, n, c->P, a, c->uadv);
    free(a);
    if (rc) return LBMREF_EINVAL;
    c->step += n;
    return LBMREF_OK;
}

static double a_pre_now(const lbmref_ctx *c)
{
    const double t = (double)c->step;
    return 0.5 * (env_at(c, t) + env_at(c, t + 0.5));
}

int lbmref_moments(lbmref_ctx *c, double *rho, double *u, int half_forced)
{
    if (!c || !rho || (c->p.lattice != ORC_D2Q5 && !u)) return LBMREF_EINVAL;
    if (!c->initialised) return LBMREF_ESTATE;
    double *uu = u;
    if (!uu) {
        uu = (double *)malloc((size_t)c->dim * c->N * sizeof(double));
        if (!uu) return LBMREF_ENOMEM;
    }
    const int rc = orc_moments(&c->p, c->f, half_forced ? c->P : NULL, a_pre_now(c), rho, uu);
    if (uu != u) free(uu);
    return rc ? LBMREF_EINVAL : LBMREF_OK;
}

int lbmref_reduce(lbmref_ctx *c, double out[5])
{
    if (!c || !out) return LBMREF_EINVAL;
    if (!c->initialised) return LBMREF_ESTATE;
    const long N = c->N;
    const int flow = c->p.lattice != ORC_D2Q5;
    double *rho = (double *)malloc((size_t)N * sizeof(double));
    double *u = (double *)malloc((size_t)c->dim * N * sizeof(double));
    if (!rho || !u) {
        free(rho);
        free(u);
        return LBMREF_ENOMEM;
    }
    orc_moments(&c->p, c->f, c->P, a_pre_now(c), rho, u);
    int ev[MAXQ * 3];
    orc_velocities(c->p.lattice, ev);
    double mass = 0.0, mom[3] = {0.0, 0.0, 0.0}, du = 0.0;
    int unstable = 0;
    for (long i = 0; i < N; i++) {
        /* mass sum f (phi^o for the scalar) and momentum sum f e (flow), Eq. 24 / 42 */
        double r = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int a = 0; a < c->q; a++) {
            r += c->f[a * N + i];
            if (flow)
                for (int d = 0; d < c->dim; d++) j[d] += c->f[a * N + i] * ev[3 * a + d];
        }
        mass += r;
        for (int d = 0; d < 3; d++) mom[d] += j[d];
        if (!isfinite(rho[i]) || (flow && !(rho[i] > 0.0))) unstable = 1;
        if (flow) {
            for (int d = 0; d < c->dim; d++) {
                const double v = u[d * N + i];
                if (c->have_prev) du = fmax(du, fabs(v - c->uprev[d * N + i]));
                c->uprev[d * N + i] = v;
            }
        } else {
            if (c->have_prev) du = fmax(du, fabs(rho[i] - c->uprev[i]));
            c->uprev[i] = rho[i];
        }
    }
    free(rho);
    free(u);
    out[0] = mass;
    out[1] = mom[0];
    out[2] = mom[1];
    out[3] = mom[2];
    out[4] = c->have_prev ? du : INFINITY;
    c->have_prev = 1;
    return unstable ? LBMREF_EUNSTABLE : LBMREF_OK;
}

int lbmref_l2_error(lbmref_ctx *c, const double *ref, int field, int half_forced, double out[3])
{
    if (!c || !ref || !out) return LBMREF_EINVAL;
    const int flow = c->p.lattice != ORC_D2Q5;
    if (field != 0 && !(field == 1 && flow)) return LBMREF_EINVAL;
    if (!c->initialised) return LBMREF_ESTATE;
    const long N = c->N;
    double *rho = (double *)malloc((size_t)N * sizeof(double));
    double *u = (double *)malloc((size_t)c->dim * N * sizeof(double));
    if (!rho || !u) {
        free(rho);
        free(u);
        return LBMREF_ENOMEM;
    }
    orc_moments(&c->p, c->f, half_forced ? c->P : NULL, a_pre_now(c), rho, u);
    /* Eq. sca: the computed field u_c against the reference u_a, summed over
       the flow domain (every node; every component of a vector field) */
    const double *uc = field == 0 ? rho : u;
    const long n = field == 0 ? N : (long)c->dim * N;
    double num = 0.0, den = 0.0;
    for (long k = 0; k < n; k++) {
        num += (uc[k] - ref[k]) * (uc[k] - ref[k]);
        den += ref[k] * ref[k];
    }
    free(rho);
    free(u);
    out[0] = num;
    out[1] = den;
    out[2] = den > 0.0 ? sqrt(num / den) : (num > 0.0 ? INFINITY : 0.0);
    return LBMREF_OK;
}

int lbmref_get_populations(const lbmref_ctx *c, double *dst, size_t count)
{
    if (!c || !dst || count != (size_t)c->q * (size_t)c->N) return LBMREF_EINVAL;
    if (!c->initialised) return LBMREF_ESTATE;
    memcpy(dst, c->f, count * sizeof(double));
    return LBMREF_OK;
}

int lbmref_set_populations(lbmref_ctx *c, const double *src, size_t count, long step)
{
    if (!c || !src || count != (size_t)c->q * (size_t)c->N || step < 0) return LBMREF_EINVAL;
    memcpy(c->f, src, count * sizeof(double));
    c->step = step;
    c->have_prev = 0;
    c->initialised = 1;
    return LBMREF_OK;
}

int lbmref_get_step(const lbmref_ctx *c, long *step)
{
    if (!c || !step) return LBMREF_EINVAL;
    *step = c->step;
    return LBMREF_OK;
}
