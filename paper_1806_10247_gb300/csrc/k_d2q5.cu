// D2Q5 cascaded LB step for a passive scalar with a Strang-split source
// (arXiv:1806.10247 Sec. 5), FP64, one thread per node, pull form: stream
// (Eq. 40b), output scalar (Eq. 42), pre-collision half source (Eq. 43),
// cascaded collision (Eq. 41), post-collision half source (Eqs. 44-47) and
// g^p = g + L h (Eq. 48).
//
// Eq. 41 is used with a minus sign on its (ux^2 + uy^2) phi and
// (ux^2 - uy^2) phi terms: expanding the central moments of Eq. 37 gives
// that sign, and only with it is the equilibrium of Eq. 39 a fixed point of
// the collision (the printed plus sign is a typesetting slip).
#include "lbm_internal.h"
#include "lbm_lattices.cuh"
#include "lbm_tiles.cuh"

namespace lbmk {
namespace {

constexpr int kBlock = 256;

struct Rates5 {
    double c1, c2, c3, c4;  // omega_1/2, omega_2/2, omega_3/4, omega_4/4
};

//   S   : pre-collision source a_pre S(x) (Eq. 43)
//   H0  : zeroth-moment coefficient h_0 = (S_pre + S_post)/10 (Eqs. 44-47)
//   ux, uy : advecting velocity at the node
__device__ __forceinline__ void collide(double (&g)[5], double S, double H0, double ux, double uy,
                                        const Rates5 &w)
{
    // Raw moments, Eq. 38.
    const double kx = g[1] - g[3], ky = g[2] - g[4];
    const double kxx = g[1] + g[3], kyy = g[2] + g[4];
    const double phio = g[0] + (kxx + kyy);  // Eq. 42
    const double phi = fma(0.5, S, phio);    // Eq. 43

    // Eq. 41 (sign-corrected u^2 phi terms).
    const double h1 = w.c1 * (phi * ux - kx);
    const double h2 = w.c2 * (phi * uy - ky);
    const double h3 = w.c3 * ((2.0 / 3.0) * phi - (kxx + kyy) + 2.0 * (ux * kx + uy * ky)
                              - (ux * ux + uy * uy) * phi)
                      + ux * h1 + uy * h2;
    const double h4 = w.c4 * (-(kxx - kyy) + 2.0 * (ux * kx - uy * ky) - (ux * ux - uy * uy) * phi)
                      + ux * h1 - uy * h2;

    // Eq. 48.
    const double c = H0 + h3;
    g[0] += H0 - 4.0 * h3;
    g[1] += c + h1 + h4;
    g[2] += c + h2 - h4;
    g[3] += c - h1 + h4;
    g[4] += c - h2 - h4;
}

// With a uniform advecting velocity, Eq. 41 is linear in (phi, kx, ky,
// kxx + kyy, kxx - kyy) with coefficients fixed for the whole launch (Coef5,
// formed on the host; the reduced-precision kernels use them directly).
struct Coef5 {
    double A1, c1, A2, c2;      // h1 = A1 phi - c1 kx,  h2 = A2 phi - c2 ky
    double P3, X3, Y3, S3;      // h3 = P3 phi + X3 kx + Y3 ky + S3 (kxx + kyy)
    double P4, X4, Y4, D4;      // h4 = P4 phi + X4 kx + Y4 ky + D4 (kxx - kyy)
};

Coef5 make_coef(const Rates5 &w, double ux, double uy)
{
    Coef5 k;
    const double ux2 = ux * ux, uy2 = uy * uy;
    k.A1 = w.c1 * ux;
    k.c1 = w.c1;
    k.A2 = w.c2 * uy;
    k.c2 = w.c2;
    // h3 = c3[(2/3) phi - S + 2(ux kx + uy ky) - (ux^2 + uy^2) phi] + ux h1 + uy h2
    k.P3 = w.c3 * ((2.0 / 3.0) - ux2 - uy2) + w.c1 * ux2 + w.c2 * uy2;
    k.X3 = ux * (2.0 * w.c3 - w.c1);
    k.Y3 = uy * (2.0 * w.c3 - w.c2);
    k.S3 = -w.c3;
    // h4 = c4[-D + 2(ux kx - uy ky) - (ux^2 - uy^2) phi] + ux h1 - uy h2
    k.P4 = -w.c4 * (ux2 - uy2) + w.c1 * ux2 - w.c2 * uy2;
    k.X4 = ux * (2.0 * w.c4 - w.c1);
    k.Y4 = uy * (w.c2 - 2.0 * w.c4);
    k.D4 = -w.c4;
    return k;
}


// With a uniform advecting velocity the whole step is linear in the pulled
// populations: writing g0* = g0 + S_pre/2 (phi of Eq. 43 enters only through
// g0 + S_pre/2), g'_a = sum_b M_ab g*_b + H0 for a = 1..4 and
// g'_0 = sum_b M_0b g*_b + H0 - S_pre/2, with H0 = (S_pre + S_post)/10
// (Eqs. 44-48).  M is formed once per launch on the host by applying Eqs. 41
// and 48 to the unit vectors; a node takes rows 1..4 (20 multiply-adds) and
// the rest population from the zeroth moment (collide_mat).
struct Mat5 {
    double m[25];
};

Mat5 make_mat(const Coef5 &k)
{
    Mat5 M;
    for (int b = 0; b < 5; b++) {
        double g[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        g[b] = 1.0;
        const double kx = g[1] - g[3], ky = g[2] - g[4];
        const double Sg = (g[1] + g[3]) + (g[2] + g[4]), Dg = (g[1] + g[3]) - (g[2] + g[4]);
        const double phi = g[0] + Sg;
        const double h1 = k.A1 * phi - k.c1 * kx;
        const double h2 = k.A2 * phi - k.c2 * ky;
        const double h3 = k.P3 * phi + k.X3 * kx + k.Y3 * ky + k.S3 * Sg;
        const double h4 = k.P4 * phi + k.X4 * kx + k.Y4 * ky + k.D4 * Dg;
        const double out[5] = {g[0] - 4.0 * h3, g[1] + h3 + h1 + h4, g[2] + h3 + h2 - h4, g[3] + h3 - h1 + h4,
                               g[4] + h3 - h2 - h4};
        for (int a = 0; a < 5; a++) M.m[5 * a + b] = out[a];
    }
    return M;
}

//   ahalf = a_pre / 2;  hsum = (a_pre + a_post)/10;  P = source shape at the node (0 without one)
// Rows 1..4 of the step matrix give g'_1..g'_4; the rest population comes
// from the zeroth moment instead of row 0: sum_a g'_a = sum_a g_a + (S_pre +
// S_post)/2 = sum_a g_a + 5 H0 (Eqs. 44-48), so g'_0 is that total minus the
// other four.  The matrix entries are rounded on the host, so their column
// sums differ from 1 by ~1e-16; taken through row 0 that would change the
// total scalar by the same amount every step (1e-12 after ~10^4 steps).
// phi0 receives the zeroth moment of the pulled populations, summed as
// zeroth_first sums it (for a fused readback).
template <bool SRC>
__device__ __forceinline__ void collide_mat(double (&g)[5], double P, double ahalf, double hsum, const double *M,
                                            double &phi0)
{
    phi0 = (((g[0] + g[1]) + g[2]) + g[3]) + g[4];
    double gs[5] = {g[0], g[1], g[2], g[3], g[4]};
    double h = 0.0;
    if (SRC) {
        gs[0] = fma(ahalf, P, g[0]);
        h = hsum * P;
    }
#pragma unroll
    for (int a = 1; a < 5; a++) {
        double acc = SRC ? fma(M[5 * a], gs[0], h) : M[5 * a] * gs[0];
#pragma unroll
        for (int b = 1; b < 5; b++) acc = fma(M[5 * a + b], gs[b], acc);
        g[a] = acc;
    }
    const double total = SRC ? fma(5.0, h, phi0) : phi0;
    g[0] = total - ((g[1] + g[2]) + (g[3] + g[4]));
}

template <int SK>
__global__ void __launch_bounds__(kBlock)
k_step_mat(const __grid_constant__ Planes<double, 5> P, Geom g, FieldDev S, double ahalf, double hsum, Mat5 M)
{
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    int x, y;
    node_xy(g, i, x, y);
    double f[5], phi0;
    load_pulled<LD2Q5>(P, g, x, y, 0, i, f);
    if (SK != FK_NONE) collide_mat<true>(f, field_value(S, SK, 0, x, y, 0, i), ahalf, hsum, M.m, phi0);
    else collide_mat<false>(f, 0.0, ahalf, hsum, M.m, phi0);
#pragma unroll
    for (int a = 0; a < 5; a++) P.out[a][i] = f[a];
}


template <int SK, int VK>
__global__ void __launch_bounds__(kBlock)
k_step(const __grid_constant__ Planes<double, 5> P, Geom g, FieldDev S, FieldDev V, double apre, double hsum,
       Rates5 w)
{
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    int x, y;
    node_xy(g, i, x, y);
    double f[5];
    load_pulled<LD2Q5>(P, g, x, y, 0, i, f);
    double Spre = 0.0, H0 = 0.0;
    if (SK != FK_NONE) {
        const double P = field_value(S, SK, 0, x, y, 0, i);
        Spre = apre * P;
        H0 = hsum * P;
    }
    double ux = 0.0, uy = 0.0;
    if (VK != FK_NONE) {
        ux = field_value(V, VK, 0, x, y, 0, i);
        uy = field_value(V, VK, 1, x, y, 0, i);
    }
    collide(f, Spre, H0, ux, uy, w);
#pragma unroll
    for (int a = 0; a < 5; a++) P.out[a][i] = f[a];
}

template <int SK>
void launch_v(const LaunchArgs &a, int grid, double hsum, const Rates5 &w)
{
    if (a.vkind != FK_GENERAL) {
        const double ux = a.vkind == FK_CONST ? a.V.cval[0] : 0.0;
        const double uy = a.vkind == FK_CONST ? a.V.cval[1] : 0.0;
        k_step_mat<SK><<<grid, kBlock, 0, a.stream>>>(make_planes<double, 5>(a.fin, a.fout, a.g.Np), a.g, a.F,
                                                       0.5 * a.apre, hsum, make_mat(make_coef(w, ux, uy)));
        return;
    }
    k_step<SK, FK_GENERAL><<<grid, kBlock, 0, a.stream>>>(make_planes<double, 5>(a.fin, a.fout, a.g.Np), a.g, a.F,
                                                          a.V, a.apre, hsum, w);
}

// Batched form; FP64 pairs hold (a_pre/2, (a_pre + a_post)/10) per step and
// item (a_pre is halved on the host: one multiply fewer per node).
// coef[0..11] = Coef5 of a uniform advecting velocity, coef[12..15] = Rates5,
// mat = the step matrix of a uniform advecting velocity.
// One node of a batched launch (member `it`, node i; B staged in shared memory).
__device__ __forceinline__ void batch_node(const BatchItem &B, const BatchLaunch &L, int it, int i)
{
    const Geom &g = B.g;
    const int p = B.parity + L.parity;
    const double *fin = B.buf[p & 1];
    double *fout = B.buf[(p + 1) & 1];
    const double2 ap = L.pairs ? L.pairs[(size_t)L.k * L.count + it] : L.inl[it];
    int x, y;
    node_xy(g, i, x, y);
    double f[5];
    load_pulled<LD2Q5>(fin, g, x, y, 0, i, f);
    if (B.vkind != FK_GENERAL) {
        const bool src = B.fkind != FK_NONE;
        const double P = src ? field_value(B.F, B.fkind, 0, x, y, 0, i) : 0.0;
        double phi0;
        if (src) collide_mat<true>(f, P, ap.x, ap.y, B.mat, phi0);
        else collide_mat<false>(f, 0.0, 0.0, 0.0, B.mat, phi0);
        if (L.mrho) {
            // fused readback of f(t)'s scalar from the step's own zeroth
            // moment: phi0 + (a_pre/2) P, the bits store_fields forms
            const double jd[3] = {0.0, 0.0, 0.0};
            put_fields<LD2Q5>(L.mhalf && src ? __dadd_rn(phi0, __dmul_rn(ap.x, P)) : phi0, jd, 0.0, i, g.N,
                              __ldg(L.moff + it), L.mrho, L.mu);
        }
    } else {
        if (L.mrho) fused_fields<LD2Q5>(B, L, it, i, x, y, 0, f, 2.0 * ap.x);
        double Spre = 0.0, H0 = 0.0;
        if (B.fkind != FK_NONE) {
            const double P = field_value(B.F, B.fkind, 0, x, y, 0, i);
            Spre = (2.0 * ap.x) * P;
            H0 = ap.y * P;
        }
        const Rates5 w{B.coef[12], B.coef[13], B.coef[14], B.coef[15]};
        const double ux = field_value(B.V, FK_GENERAL, 0, x, y, 0, i);
        const double uy = field_value(B.V, FK_GENERAL, 1, x, y, 0, i);
        collide(f, Spre, H0, ux, uy, w);
    }
#pragma unroll
    for (int a = 0; a < 5; a++) fout[a * g.Np + i] = f[a];
}

template <int TB, int MODE>
__global__ void __launch_bounds__(TB)
k_batch(const __grid_constant__ BatchLaunch L)
{
    batch_tiles<TB, MODE>(L, [](const BatchItem &B, const BatchLaunch &L2, int it, int i) { batch_node(B, L2, it, i); });
}

}  // namespace

void d2q5_batch_coef(const double omega[9], BatchItem &item)
{
    const Rates5 w{omega[1] / 2.0, omega[2] / 2.0, omega[3] / 4.0, omega[4] / 4.0};
    const double ux = item.vkind == FK_CONST ? item.V.cval[0] : 0.0;
    const double uy = item.vkind == FK_CONST ? item.V.cval[1] : 0.0;
    const Coef5 c = make_coef(w, ux, uy);
    const double v[16] = {c.A1, c.c1, c.A2, c.c2, c.P3, c.X3, c.Y3, c.S3,
                          c.P4, c.X4, c.Y4, c.D4, w.c1, w.c2, w.c3, w.c4};
    for (int k = 0; k < 16; k++) item.coef[k] = v[k];
    const Mat5 M = make_mat(c);
    for (int k = 0; k < 25; k++) item.mat[k] = M.m[k];
}

cudaError_t d2q5_batch_step(const BatchLaunch &L, int nblocks, int tile, cudaStream_t s)
{
    LBM_TILED_LAUNCH(k_batch, L, nblocks, tile, s);
}

int d2q5_batch_resident(int tile)
{
    LBM_TILED_RESIDENT(k_batch, tile);
}

cudaError_t d2q5_step(const LaunchArgs &a)
{
    Rates5 w{a.omega[1] / 2.0, a.omega[2] / 2.0, a.omega[3] / 4.0, a.omega[4] / 4.0};
    const double hsum = (a.apre + a.apost) / 10.0;
    const int grid = (a.g.N + kBlock - 1) / kBlock;
    switch (a.fkind) {
    case FK_NONE: launch_v<FK_NONE>(a, grid, hsum, w); break;
    case FK_CONST: launch_v<FK_CONST>(a, grid, hsum, w); break;
    default: launch_v<FK_GENERAL>(a, grid, hsum, w); break;
    }
    return cudaGetLastError();
}

}  // namespace lbmk
