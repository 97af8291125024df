// D3Q15 fused stream + collide step, FP64: the 3D cascaded method of
// Appendix A with the symmetrized operator-split force.
//
// Per node: pull the 15 populations (Eq. 22b with halfway bounce-back or
// periodic wrap), raw moments of Eq. g8 (the corner populations through an
// 8-point sign transform), the pre-collision half force of Eq. 8A, the
// cascaded changes g_4..g_14 of Eq. 6A, the force change g_1..g_3 of
// Eq. 13A and the populations f + K g (Eq. 2A), again through the sign
// transform on the corners.  Three readings of the appendix are built in:
// the trace bracket of g_9 relaxes towards its equilibrium rho (as printed
// the rest state would not be a fixed point); the populations are K g
// exactly (the printed f^p_12 has the sign of g_13 flipped); the product in
// the fourth-order bracket of g_14 is that of the post-collision second
// central moments kappa_xx, kappa_yy divided by rho.  With a time-dependent
// force the first moments change by (F_pre + F_post)/2, i.e.
// g_1..3 = (F_pre + F_post)/20.
#include "lbm_d3q15.cuh"
#include "lbm_internal.h"
#include "lbm_lattices.cuh"
#include "lbm_tiles.cuh"

namespace lbmk {
namespace {

constexpr int kBlock = 256;

// omega_4..omega_8 (shear), omega_9 (trace), omega_10..omega_13, omega_14
struct Rates15 {
    double s, b, t, q;
};

// Moments the collision forms on the way (for a fused readback): rho and the
// un-forced j, grouped as zeroth_first<LD3Q15> groups them, the half-forced
// j of Eq. 8A and 1/rho (__drcp_rn).
struct Mom15 {
    double rho, j[3], jf[3], rinv;
};

// F = a_pre P (Eq. 8A), Fq = a_post P (second half step).
__device__ __forceinline__ void collide(double (&f)[15], const double (&F)[3], const double (&Fq)[3],
                                        const Rates15 &w, Mom15 &mo)
{
    // Axis pairs and the corner sign transform: S_{ijk} = sum_c s_x^i s_y^j s_z^k f_c.
    const double axs = f[1] + f[2], axd = f[1] - f[2];
    const double ays = f[3] + f[4], ayd = f[3] - f[4];
    const double azs = f[5] + f[6], azd = f[5] - f[6];
    const double A1 = f[7] + f[8], B1 = f[7] - f[8];      // y+, z+
    const double A2 = f[9] + f[10], B2 = f[9] - f[10];    // y-, z+
    const double A3 = f[11] + f[12], B3 = f[11] - f[12];  // y+, z-
    const double A4 = f[13] + f[14], B4 = f[13] - f[14];  // y-, z-
    const double P1 = A1 + A2, Q1 = A1 - A2, P2 = A3 + A4, Q2 = A3 - A4;
    const double R1 = B1 + B2, T1 = B1 - B2, R2 = B3 + B4, T2 = B3 - B4;
    const double S = P1 + P2, Sz = P1 - P2, Sy = Q1 + Q2, Syz = Q1 - Q2;
    const double Sx = R1 + R2, Sxz = R1 - R2, Sxy = T1 + T2, Sxyz = T1 - T2;

    // Raw moments (Eq. g8): on D3Q15 every cubic and quartic monomial of the
    // basis lives on the corners only.
    const double rho = f[0] + axs + ays + azs + S;
    const double kxx = axs + S, kyy = ays + S, kzz = azs + S;
    const double kxy = Sxy, kxz = Sxz, kyz = Syz;
    const double kxyy = Sx, kxxy = Sy, kxxz = Sz, kxyz = Sxyz, kxxyy = S;

    // Eq. 8A: half-forced momentum J = rho u.
    const double jx0 = axd + Sx, jy0 = ayd + Sy, jz0 = azd + Sz;
    const double Jx = fma(0.5, F[0], jx0), Jy = fma(0.5, F[1], jy0), Jz = fma(0.5, F[2], jz0);
    const double ir = __drcp_rn(rho);
    mo = Mom15{rho, {jx0, jy0, jz0}, {Jx, Jy, Jz}, ir};
    const double ux = Jx * ir, uy = Jy * ir, uz = Jz * ir;

    // Eq. 6A.  Second order: central moments about u.
    const double cxx = kxx - Jx * ux, cyy = kyy - Jy * uy, czz = kzz - Jz * uz;
    const double g4 = -0.125 * w.s * (kxy - Jx * uy);
    const double g5 = -0.125 * w.s * (kxz - Jx * uz);
    const double g6 = -0.125 * w.s * (kyz - Jy * uz);
    const double g7 = -0.25 * w.s * (cxx - cyy);
    const double g8 = -(w.s / 12.0) * (cxx + cyy - 2.0 * czz);
    const double g9 = (w.b / 18.0) * (rho - (cxx + cyy + czz));
    const double h3 = g7 + g8 + 3.0 * g9;  // the combination the cubic cascades share
    const double g10 = 0.0625 * w.t * (-kxyy + 2.0 * uy * kxy + ux * kyy - 2.0 * Jx * uy * uy) + uy * g4 +
                       0.125 * ux * (h3 - 2.0 * g7);
    const double g11 = 0.0625 * w.t * (-kxxy + 2.0 * ux * kxy + uy * kxx - 2.0 * Jx * ux * uy) + ux * g4 +
                       0.125 * uy * h3;
    const double g12 = 0.0625 * w.t * (-kxxz + 2.0 * ux * kxz + uz * kxx - 2.0 * Jx * ux * uz) + ux * g5 +
                       0.125 * uz * h3;
    const double g13 = 0.125 * w.t * (-kxyz + ux * kyz + uy * kxz + uz * kxy - 2.0 * Jx * uy * uz) + uz * g4 +
                       uy * g5 + ux * g6;
    // post-collision kappa_xx, kappa_yy (the changes of K_7, K_8, K_9 to them)
    const double cxx_p = cxx + 2.0 * (g7 + g8) + 6.0 * g9;
    const double cyy_p = cyy + 2.0 * (g8 - g7) + 6.0 * g9;
    const double ux2 = ux * ux, uy2 = uy * uy;
    const double g14 = 0.0625 * w.q *
                           (-kxxyy + 2.0 * ux * kxyy + 2.0 * uy * kxxy - ux2 * kyy - uy2 * kxx -
                            4.0 * ux * uy * kxy + cxx_p * cyy_p * ir + 3.0 * Jx * ux * uy2) -
                       2.0 * ux * uy * g4 + 0.125 * (ux2 - uy2) * g7 - 0.125 * (ux2 + uy2) * g8 -
                       (0.375 * (ux2 + uy2) + 0.5) * g9 + 2.0 * ux * g10 + 2.0 * uy * g11;

    // Eq. 13A with the two half steps.
    const double g1 = 0.05 * (F[0] + Fq[0]), g2 = 0.05 * (F[1] + Fq[1]), g3 = 0.05 * (F[2] + Fq[2]);

    // f + K g.  Rest and axes:
    f[0] += 32.0 * g14 - 2.0 * g9;
    const double bx = g7 + g8 - g9 - 8.0 * g14, ox = g1 - 8.0 * g10;
    const double by = g8 - g7 - g9 - 8.0 * g14, oy = g2 - 8.0 * g11;
    const double bz = -2.0 * g8 - g9 - 8.0 * g14, oz = g3 - 8.0 * g12;
    f[1] += bx + ox;
    f[2] += bx - ox;
    f[3] += by + oy;
    f[4] += by - oy;
    f[5] += bz + oz;
    f[6] += bz - oz;
    // corners: c0 + s_x cx + s_y cy + s_z cz + s_x s_y g4 + s_x s_z g5 + s_y s_z g6 + s_x s_y s_z g13
    const double c0 = g9 + 2.0 * g14, cx = g1 + 2.0 * g10, cy = g2 + 2.0 * g11, cz = g3 + 2.0 * g12;
    const double U0 = c0 + cz, Ux = cx + g5, Uy = cy + g6, Uxy = g4 + g13;  // z = +1
    const double V0 = c0 - cz, Vx = cx - g5, Vy = cy - g6, Vxy = g4 - g13;  // z = -1
    const double a0 = U0 + Uy, ax = Ux + Uxy, b0 = U0 - Uy, bxx = Ux - Uxy;
    const double c0m = V0 + Vy, cxm = Vx + Vxy, d0 = V0 - Vy, dx = Vx - Vxy;
    f[7] += a0 + ax;
    f[8] += a0 - ax;
    f[9] += b0 + bxx;
    f[10] += b0 - bxx;
    f[11] += c0m + cxm;
    f[12] += c0m - cxm;
    f[13] += d0 + dx;
    f[14] += d0 - dx;
}

template <int FK>
__global__ void __launch_bounds__(kBlock)
k_step(const __grid_constant__ Planes<double, 15> P, Geom g, FieldDev Fd, double apre, double apost, Rates15 w)
{
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    double f[15];
    load_pulled<LD3Q15>(P, g, x, y, z, i, f);
    double F[3] = {0.0, 0.0, 0.0}, Fq[3] = {0.0, 0.0, 0.0};
    if (FK != FK_NONE) {
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const double P = field_value(Fd, FK, d, x, y, z, i);
            F[d] = apre * P;
            Fq[d] = apost * P;
        }
    }
    Mom15 mo;
    collide(f, F, Fq, w, mo);
#pragma unroll
    for (int a = 0; a < 15; a++) P.out[a][i] = f[a];
}

// Batched form; pairs hold (a_pre, a_post) per step and item.
// One node of a batched launch (member `it`, node i; B staged in shared memory).
__device__ __forceinline__ void batch_node(const BatchItem &B, const BatchLaunch &L, int it, int i)
{
    const Geom &g = B.g;
    const int p = B.parity + L.parity;
    const double *fin = B.buf[p & 1];
    double *fout = B.buf[(p + 1) & 1];
    const double2 ap = L.pairs ? L.pairs[(size_t)L.k * L.count + it] : L.inl[it];
    int x, y, z;
    node_xyz(g, i, x, y, z);
    double f[15];
    load_pulled<LD3Q15>(fin, g, x, y, z, i, f);
    double F[3] = {0.0, 0.0, 0.0}, Fq[3] = {0.0, 0.0, 0.0};
    if (B.fkind != FK_NONE) {
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const double P = field_value(B.F, B.fkind, d, x, y, z, i);
            F[d] = ap.x * P;
            Fq[d] = ap.y * P;
        }
    }
    const Rates15 w{B.coef[0], B.coef[1], B.coef[2], B.coef[3]};
    Mom15 mo;
    collide(f, F, Fq, w, mo);
    if (L.mrho) {
        // fused readback of f(t)'s fields from the collision's own moments;
        // the same bits as store_fields (F = a_pre P)
        const bool forced = L.mhalf && B.fkind != FK_NONE;
        const double jd[3] = {forced ? mo.jf[0] : mo.j[0], forced ? mo.jf[1] : mo.j[1], forced ? mo.jf[2] : mo.j[2]};
        put_fields<LD3Q15>(mo.rho, jd, mo.rinv, i, g.N, __ldg(L.moff + it), L.mrho, L.mu);
    }
#pragma unroll
    for (int a = 0; a < 15; a++) fout[a * g.Np + i] = f[a];
}

template <int TB, int MODE>
__global__ void __launch_bounds__(TB)
k_batch(const __grid_constant__ BatchLaunch L)
{
    batch_tiles<TB, MODE>(L, [](const BatchItem &B, const BatchLaunch &L2, int it, int i) { batch_node(B, L2, it, i); });
}

}  // namespace

void d3q15_batch_coef(const double omega[9], BatchItem &item)
{
    item.coef[0] = omega[2];
    item.coef[1] = omega[1];
    item.coef[2] = omega[3];
    item.coef[3] = omega[4];
}

cudaError_t d3q15_batch_step(const BatchLaunch &L, int nblocks, int tile, cudaStream_t s)
{
    LBM_TILED_LAUNCH(k_batch, L, nblocks, tile, s);
}

int d3q15_batch_resident(int tile)
{
    LBM_TILED_RESIDENT(k_batch, tile);
}

cudaError_t d3q15_step(const LaunchArgs &a)
{
    const Rates15 w{a.omega[2], a.omega[1], a.omega[3], a.omega[4]};
    const int grid = (a.g.N + kBlock - 1) / kBlock;
    const Planes<double, 15> P = make_planes<double, 15>(a.fin, a.fout, a.g.Np);
    switch (a.fkind) {
    case FK_NONE: k_step<FK_NONE><<<grid, kBlock, 0, a.stream>>>(P, a.g, a.F, a.apre, a.apost, w); break;
    case FK_CONST: k_step<FK_CONST><<<grid, kBlock, 0, a.stream>>>(P, a.g, a.F, a.apre, a.apost, w); break;
    default: k_step<FK_GENERAL><<<grid, kBlock, 0, a.stream>>>(P, a.g, a.F, a.apre, a.apost, w); break;
    }
    return cudaGetLastError();
}

}  // namespace lbmk
