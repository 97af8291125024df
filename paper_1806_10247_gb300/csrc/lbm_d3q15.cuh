// D3Q15 velocity set (Appendix A, Eq. a1) as compile-time traits, and its
// equilibrium populations.
#pragma once

#include "lbm_device.cuh"

namespace lbmk {

// 0 rest; 1 +x, 2 -x, 3 +y, 4 -y, 5 +z, 6 -z; 7..14 the corners
// (+,+,+), (-,+,+), (+,-,+), (-,-,+), (+,+,-), (-,+,-), (+,-,-), (-,-,-):
// x alternates fastest, then y, then z.  The opposite of corner a is 21 - a.
struct LD3Q15 {
    static constexpr int Q = 15, DIM = 3, ID = 4;
    __host__ __device__ static constexpr int ex(int a)
    {
        return a >= 7 ? ((a & 1) ? 1 : -1) : (a == 1 ? 1 : (a == 2 ? -1 : 0));
    }
    __host__ __device__ static constexpr int ey(int a)
    {
        return a >= 7 ? ((((a - 7) >> 1) & 1) ? -1 : 1) : (a == 3 ? 1 : (a == 4 ? -1 : 0));
    }
    __host__ __device__ static constexpr int ez(int a)
    {
        return a >= 7 ? (a <= 10 ? 1 : -1) : (a == 5 ? 1 : (a == 6 ? -1 : 0));
    }
    __host__ __device__ static constexpr int opp(int a) { return a == 0 ? 0 : (a >= 7 ? 21 - a : ((a & 1) ? a + 1 : a - 1)); }
    // rest-state populations per unit density (2/9, 1/9, 1/72)
    __host__ __device__ static constexpr double w(int a) { return a == 0 ? 2.0 / 9.0 : (a <= 6 ? 1.0 / 9.0 : 1.0 / 72.0); }
};

// Equilibrium population a at (rho, u): the populations whose moments of the
// fifteen monomials 1, e_x, e_y, e_z, e_x e_y, e_x e_z, e_y e_z, e_x^2, e_y^2,
// e_z^2, e_x e_y^2, e_x^2 e_y, e_x^2 e_z, e_x e_y e_z, e_x^2 e_y^2 (a basis of
// the D3Q15 population space, the moments behind K_0..K_14 of Eq. 2A) are
// those of a Maxwellian with c_s^2 = 1/3: the raw moment of e_x^a e_y^b e_z^c
// is rho * M(a, u_x) M(b, u_y) M(c, u_z) with M(0) = 1, M(1) = u, M(2) = 1/3 + u^2.
// Every moment but e_x^2 e_y^2 and the three cubic ones lives on the axes as
// well as the corners; solving the two groups separately gives the closed form.
__device__ __forceinline__ double d3q15_equilibrium(double r, double ux, double uy, double uz, int a)
{
    const double Mx = 1.0 / 3.0 + ux * ux, My = 1.0 / 3.0 + uy * uy, Mz = 1.0 / 3.0 + uz * uz;
    // corner sums sum_c s_x^i s_y^j s_z^k f_c, fixed by the moments that vanish on the axes
    const double S = r * Mx * My;
    if (a == 0) return r * (1.0 - Mx - My - Mz) + 2.0 * S;
    if (a <= 2) return 0.5 * ((r * Mx - S) + (double)LD3Q15::ex(a) * (r * ux - r * ux * My));
    if (a <= 4) return 0.5 * ((r * My - S) + (double)LD3Q15::ey(a) * (r * uy - r * uy * Mx));
    if (a <= 6) return 0.5 * ((r * Mz - S) + (double)LD3Q15::ez(a) * (r * uz - r * uz * Mx));
    const double sx = LD3Q15::ex(a), sy = LD3Q15::ey(a), sz = LD3Q15::ez(a);
    return 0.125 * (S + sx * (r * ux * My) + sy * (r * uy * Mx) + sz * (r * uz * Mx) + sx * sy * (r * ux * uy) +
                    sx * sz * (r * ux * uz) + sy * sz * (r * uy * uz) + sx * sy * sz * (r * ux * uy * uz));
}

}  // namespace lbmk
