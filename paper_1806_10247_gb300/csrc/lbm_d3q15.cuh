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

// Zeroth and first moments grouped as the D3Q15 collision forms them: the
// axis pairs f_+ +/- f_-, then the corner sign transform (pairs along x, then
// along y, then along z), so that the collision's own rho and j are these
// bits (m0 = (((f_0 + ax) + ay) + az) + corners, j_d = axis difference +
// corner sum).  Declared as a specialization of zeroth_first.
template <class L>
__device__ __forceinline__ void zeroth_first(const double (&f)[L::Q], double &m0, double (&j)[3]);
template <>
__device__ __forceinline__ void zeroth_first<LD3Q15>(const double (&f)[15], double &m0, double (&j)[3])
{
    const double A1 = f[7] + f[8], B1 = f[7] - f[8], A2 = f[9] + f[10], B2 = f[9] - f[10];
    const double A3 = f[11] + f[12], B3 = f[11] - f[12], A4 = f[13] + f[14], B4 = f[13] - f[14];
    const double P1 = A1 + A2, Q1 = A1 - A2, P2 = A3 + A4, Q2 = A3 - A4;
    const double R1 = B1 + B2, R2 = B3 + B4;
    m0 = (((f[0] + (f[1] + f[2])) + (f[3] + f[4])) + (f[5] + f[6])) + (P1 + P2);
    j[0] = (f[1] - f[2]) + (R1 + R2);
    j[1] = (f[3] - f[4]) + (Q1 + Q2);
    j[2] = (f[5] - f[6]) + (P1 - P2);
}

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
