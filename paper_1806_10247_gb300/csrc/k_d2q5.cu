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

template <int SK, int VK>
__global__ void __launch_bounds__(kBlock)
k_step(const double *__restrict__ fin, double *__restrict__ fout, Geom g, FieldDev S, FieldDev V,
       double apre, double hsum, Rates5 w)
{
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    const int x = i % g.nx, y = i / g.nx;
    double f[5];
    load_pulled<LD2Q5>(fin, g, x, y, 0, i, f);
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
    for (int a = 0; a < 5; a++) fout[a * g.Np + i] = f[a];
}

template <int SK>
void launch_v(const LaunchArgs &a, int grid, double hsum, const Rates5 &w)
{
    switch (a.vkind) {
    case FK_NONE: k_step<SK, FK_NONE><<<grid, kBlock, 0, a.stream>>>(a.fin, a.fout, a.g, a.F, a.V, a.apre, hsum, w); break;
    case FK_CONST: k_step<SK, FK_CONST><<<grid, kBlock, 0, a.stream>>>(a.fin, a.fout, a.g, a.F, a.V, a.apre, hsum, w); break;
    default: k_step<SK, FK_GENERAL><<<grid, kBlock, 0, a.stream>>>(a.fin, a.fout, a.g, a.F, a.V, a.apre, hsum, w); break;
    }
}

}  // namespace

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
