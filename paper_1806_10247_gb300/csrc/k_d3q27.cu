// D3Q27 cascaded (central-moment) LB step with Strang-split body force, FP64,
// one thread per node, pull form.  arXiv:1806.10247 states the 3D method for
// D3Q15 (Appendix A) and notes that it extends to D3Q27; this is that
// extension by the generic central-moment procedure:
//
//   raw moments m_abc (a,b,c in {0,1,2})  ->  pre-collision half force on the
//   first moments (Eq. 8A analogue: m_100 += F_pre/2, ...)  ->  central moments
//   about u = m_1/rho  ->  relaxation (trace with omega_bulk towards rho,
//   deviatoric and off-diagonal second order with omega_shear towards 0, every
//   moment of order n = 3..6 with omega_n towards its Maxwellian value)  ->
//   raw moments  ->  post-collision force along K_1 = e (Eqs. 12A-13A
//   analogue, g_1 = (F_pre + F_post)/2 / 18 since sum_alpha e_x^2 = 18)  ->
//   populations.
//
// The transforms are factorised along the axes (three passes of nine 1D
// transforms on the moment orders 0, 1, 2 of the velocities -1, 0, +1), so a
// node costs ~400 FP64 operations instead of the ~1500 of dense 27 x 27
// transforms.  Moment index k = a + 3 b + 9 c matches the velocity index
// alpha = (ex+1) + 3 (ey+1) + 9 (ez+1) position by position.
#include <utility>

#include "lbm_internal.h"
#include "lbm_lattices.cuh"
#include "lbm_tiles.cuh"

namespace lbmk {
namespace {

constexpr int kBlock = 256;

struct Rates27 {
    double wb, ws, w3, w4, w5, w6;
};

// Populations at velocities -1, 0, +1 -> raw moments of order 0, 1, 2.
__device__ __forceinline__ void raw_fwd(double &a, double &b, double &c)
{
    const double s = c + a, d = c - a;
    a = s + b;
    b = d;
    c = s;
}
// Raw moments -> central moments about u (binomial shift, one axis).
__device__ __forceinline__ void shift_fwd(double m0, double &m1, double &m2, double u)
{
    const double k1 = fma(-u, m0, m1);
    m2 = fma(-u, m1 + k1, m2);
    m1 = k1;
}

// The way back runs on HALVED moments: every axis on which a moment has order
// 1 or 2 contributes a factor 1/2 (m~_abc = m_abc / 2^(#nonzero orders)).  The
// inverse 1D transform of a halved triple (m0, m1/2, m2/2) is then
// f_-1 = m2/2 - m1/2, f_0 = m0 - m2, f_+1 = m2/2 + m1/2: three operations per
// line instead of four, and the factors cost nothing where they land on
// constants (relaxation rates, equilibrium values, force coefficients).
//
// Halved raw moments of order 0, 1, 2 -> populations at -1, 0, +1.
__device__ __forceinline__ void raw_bwd_h(double &m0, double &m1, double &m2)
{
    const double fm = m2 - m1, fp = m2 + m1, f0 = fma(-2.0, m2, m0);
    m0 = fm;
    m1 = f0;
    m2 = fp;
}
// Halved central moments about u -> halved raw moments (one axis; uh = u / 2):
// m1 = k1 + u k0 and m2 = k2 + 2 u k1 + u^2 k0 with the halves carried along.
__device__ __forceinline__ void shift_bwd_h(double k0, double &k1, double &k2, double u, double uh)
{
    const double m1 = fma(uh, k0, k1);
    k2 = fma(u, k1 + m1, k2);
    k1 = m1;
}

// Apply a 1D operation to the nine triples along axis `ax` (0 x, 1 y, 2 z).
template <int AX, class Op>
__device__ __forceinline__ void along(double (&m)[27], Op op)
{
    constexpr int st = AX == 0 ? 1 : (AX == 1 ? 3 : 9);
#pragma unroll
    for (int t = 0; t < 9; t++) {
        // base index of the t-th line along AX
        const int p = AX == 0 ? 3 * t : (AX == 1 ? (t % 3) + 9 * (t / 3) : t);
        op(m[p], m[p + st], m[p + 2 * st]);
    }
}

// The back-shift with a compile-time zero pattern: bit k of Z set means m[k]
// is exactly 0 on entry (the unit-rates collision leaves 16 of the 27 halved
// central moments at 0).  An operation with a known-zero operand is left out
// and its value taken as is: fma(a, 0, x) = x, fma(a, x, 0) = a x, x + 0 = x
// (equal to the full operation up to the sign of a zero result).  Z = 0 is
// shift_bwd_h on every line.
template <int AX>
__host__ __device__ constexpr int line_base(int t)
{
    return AX == 0 ? 3 * t : (AX == 1 ? (t % 3) + 9 * (t / 3) : t);
}
template <int AX>
__host__ __device__ constexpr int line_stride()
{
    return AX == 0 ? 1 : (AX == 1 ? 3 : 9);
}

// Zero pattern after shift_bwd_h along AX: on a line (k0, k1, k2), the new k1
// is 0 when k0 and k1 are, the new k2 when all three are.
template <int AX>
__host__ __device__ constexpr unsigned shift_zeros(unsigned z)
{
    unsigned r = z;
    for (int t = 0; t < 9; t++) {
        const int p0 = line_base<AX>(t), p1 = p0 + line_stride<AX>(), p2 = p0 + 2 * line_stride<AX>();
        const bool z01 = ((z >> p0) & 1u) && ((z >> p1) & 1u), z012 = z01 && ((z >> p2) & 1u);
        r = (r & ~(1u << p1) & ~(1u << p2)) | (z01 ? 1u << p1 : 0u) | (z012 ? 1u << p2 : 0u);
    }
    return r;
}

template <unsigned Z, int AX, int T>
__device__ __forceinline__ void shift_line(double (&m)[27], double u, double uh)
{
    constexpr int p0 = line_base<AX>(T), p1 = p0 + line_stride<AX>(), p2 = p0 + 2 * line_stride<AX>();
    constexpr bool z0 = (Z >> p0) & 1u, z1 = (Z >> p1) & 1u, z2 = (Z >> p2) & 1u;
    if constexpr (z0 && z1) {
        return;  // m1 = 0, and k2 keeps its value
    } else {
        double m1;
        if constexpr (z0) m1 = m[p1];
        else if constexpr (z1) m1 = uh * m[p0];
        else m1 = fma(uh, m[p0], m[p1]);
        double s;
        if constexpr (z1) s = m1;
        else s = m[p1] + m1;
        if constexpr (z2) m[p2] = u * s;
        else m[p2] = fma(u, s, m[p2]);
        m[p1] = m1;
    }
}

template <unsigned Z, int AX, int... T>
__device__ __forceinline__ void shift_lines(double (&m)[27], double u, double uh, std::integer_sequence<int, T...>)
{
    (shift_line<Z, AX, T>(m, u, uh), ...);
}

// Halved post-collision central moments about u -> populations: back-shift,
// the post-collision force in moment space, inverse raw transform.  Z: the
// moments known to be exactly 0 on entry (see shift_line).  XO: the force has
// no y and z components (their terms, additions of 0, are left out).
template <unsigned Z, bool XO>
__device__ __forceinline__ void finish(double (&m)[27], double ux, double uy, double uz, const double (&F)[3],
                                       const double (&Fq)[3])
{
    const double hx = 0.5 * ux, hy = 0.5 * uy, hz = 0.5 * uz;
    constexpr unsigned Zy = shift_zeros<0>(Z), Zz = shift_zeros<1>(Zy);
    shift_lines<Z, 0>(m, ux, hx, std::make_integer_sequence<int, 9>{});
    shift_lines<Zy, 1>(m, uy, hy, std::make_integer_sequence<int, 9>{});
    shift_lines<Zz, 2>(m, uz, hz, std::make_integer_sequence<int, 9>{});

    // K_1 g_1 in moment space, g = (F_pre + F_post) / 36: e_x changes m_100 by
    // 18 g, m_120 and m_102 by 12 g, m_122 by 8 g (halved: 9 g, 3 g, 3 g, g).
    // m_100 = rho u already carries F_pre / 2 (the pre-collision shift), so
    // only F_post / 2 is added to it.
    {
        const double sx = F[0] + Fq[0];
        m[1] = fma(0.25, Fq[0], m[1]);
        m[7] = fma(sx, 1.0 / 12.0, m[7]); m[19] = fma(sx, 1.0 / 12.0, m[19]); m[25] = fma(sx, 1.0 / 36.0, m[25]);
        if constexpr (!XO) {
            const double sy = F[1] + Fq[1], sz = F[2] + Fq[2];
            m[3] = fma(0.25, Fq[1], m[3]);
            m[9] = fma(0.25, Fq[2], m[9]);
            m[5] = fma(sy, 1.0 / 12.0, m[5]); m[21] = fma(sy, 1.0 / 12.0, m[21]); m[23] = fma(sy, 1.0 / 36.0, m[23]);
            m[11] = fma(sz, 1.0 / 12.0, m[11]); m[15] = fma(sz, 1.0 / 12.0, m[15]); m[17] = fma(sz, 1.0 / 36.0, m[17]);
        }
    }

    along<2>(m, [](double &a, double &b, double &c) { raw_bwd_h(a, b, c); });
    along<1>(m, [](double &a, double &b, double &c) { raw_bwd_h(a, b, c); });
    along<0>(m, [](double &a, double &b, double &c) { raw_bwd_h(a, b, c); });
}

// Moments a collision forms on the way (for a fused readback): rho and the
// un-forced j of the pulled populations, grouped as zeroth_first<LD3Q27>
// groups them, the half-forced j and 1/rho (__drcp_rn).
struct Mom27 {
    double rho, j[3], jf[3], rinv;
};

// F: pre-collision force a_pre P; Fq: post-collision force a_post P; XO: the
// force has no y and z components.
template <bool XO = false>
__device__ __forceinline__ void collide(double (&m)[27], const double (&F)[3], const double (&Fq)[3],
                                        const Rates27 &w, Mom27 &mo)
{
    along<0>(m, [](double &a, double &b, double &c) { raw_fwd(a, b, c); });
    along<1>(m, [](double &a, double &b, double &c) { raw_fwd(a, b, c); });
    along<2>(m, [](double &a, double &b, double &c) { raw_fwd(a, b, c); });

    // Pre-collision half force on the first moments; velocity u = m_1 / rho.
    mo.j[0] = m[1];
    mo.j[1] = m[3];
    mo.j[2] = m[9];
    m[1] = fma(0.5, F[0], m[1]);
    if constexpr (!XO) {
        m[3] = fma(0.5, F[1], m[3]);
        m[9] = fma(0.5, F[2], m[9]);
    }
    const double rho = m[0];
    const double rinv = __drcp_rn(rho);
    mo.rho = rho;
    mo.jf[0] = m[1];
    mo.jf[1] = m[3];
    mo.jf[2] = m[9];
    mo.rinv = rinv;
    const double ux = m[1] * rinv, uy = m[3] * rinv, uz = m[9] * rinv;

    along<0>(m, [ux](double &a, double &b, double &c) { shift_fwd(a, b, c, ux); });
    along<1>(m, [uy](double &a, double &b, double &c) { shift_fwd(a, b, c, uy); });
    along<2>(m, [uz](double &a, double &b, double &c) { shift_fwd(a, b, c, uz); });

    // Relaxation of the central moments; the results are written halved.
    {
        const double T = m[2] + m[6] + m[18];
        const double D1 = m[2] - m[6], D2 = m[2] - m[18];
        const double Ts = fma(w.wb, rho - T, T);
        const double rs = 1.0 - w.ws;
        const double rh = 0.5 * rs, rq = 0.25 * rs;
        const double D1h = rh * D1, D2h = rh * D2;  // halved relaxed deviatoric parts
        const double kxx = fma(Ts, 1.0 / 6.0, (D1h + D2h) * (1.0 / 3.0));
        m[2] = kxx;
        m[6] = kxx - D1h;
        m[18] = kxx - D2h;
        m[4] *= rq;   // 110
        m[10] *= rq;  // 101
        m[12] *= rq;  // 011
        m[1] = 0.0;   // first central moments vanish after the half force
        m[3] = 0.0;
        m[9] = 0.0;
        const double r3 = 1.0 - w.w3, r4 = 1.0 - w.w4, r5 = 1.0 - w.w5;
        const double r3q = 0.25 * r3, r3e = 0.125 * r3;
        m[5] *= r3q; m[7] *= r3q; m[11] *= r3q; m[15] *= r3q; m[19] *= r3q; m[21] *= r3q; m[13] *= r3e;
        // m~_220 = (1 - w4) m_220 / 4 + w4 (rho / 9) / 4
        const double r4q = 0.25 * r4, e4 = (w.w4 * (1.0 / 36.0)) * rho;
        m[8] = fma(r4q, m[8], e4);
        m[20] = fma(r4q, m[20], e4);
        m[24] = fma(r4q, m[24], e4);
        const double r4e = 0.125 * r4, r5e = 0.125 * r5;
        m[14] *= r4e; m[16] *= r4e; m[22] *= r4e;
        m[17] *= r5e; m[23] *= r5e; m[25] *= r5e;
        m[26] = fma(0.125 * (1.0 - w.w6), m[26], (w.w6 * (1.0 / 216.0)) * rho);
    }

    finish<0u, XO>(m, ux, uy, uz, F, Fq);
}

// Halved central moments the unit-rates collision leaves exactly 0: all but
// 000, 200, 020, 002, 110, 101, 011, 220, 202, 022, 222 (index a + 3b + 9c).
constexpr unsigned kNonZeroW1 = (1u << 0) | (1u << 2) | (1u << 6) | (1u << 18) | (1u << 4) | (1u << 10) | (1u << 12) |
                                (1u << 8) | (1u << 20) | (1u << 24) | (1u << 26);
constexpr unsigned kZeroW1 = ((1u << 27) - 1u) & ~kNonZeroW1;

// The same collision when omega_3 = omega_4 = omega_5 = omega_6 = 1 (the
// paper's choice for the higher moments, Sec. 6): every central moment of
// order 3..6 lands exactly on its Maxwellian value, so only the raw moments of
// order <= 2 are formed (partial transforms) and the forward shift reduces to
// the six second-order central moments.
template <bool XO = false>
__device__ __forceinline__ void collide_w1(double (&m)[27], const double (&F)[3], const double (&Fq)[3],
                                           const Rates27 &w, Mom27 &mo)
{
    along<0>(m, [](double &a, double &b, double &c) { raw_fwd(a, b, c); });
    // Line (b, c) along x holds M0, M1, M2 at m[3b + 9c + 0..2]; e_y = b - 1, e_z = c - 1.
    double Y0[3], Y1[3], Y2[3], X0[3], X1[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const double s = m[9 * c + 6] + m[9 * c], d = m[9 * c + 6] - m[9 * c];
        Y0[c] = s + m[9 * c + 3];
        Y1[c] = d;
        Y2[c] = s;
        X0[c] = (m[9 * c + 7] + m[9 * c + 1]) + m[9 * c + 4];
        X1[c] = m[9 * c + 7] - m[9 * c + 1];
    }
    const double rho = (Y0[2] + Y0[0]) + Y0[1];
    double jz = Y0[2] - Y0[0];
    const double kzz = Y0[2] + Y0[0];
    double jy = (Y1[2] + Y1[0]) + Y1[1];
    const double kyz = Y1[2] - Y1[0];
    const double kyy = (Y2[2] + Y2[0]) + Y2[1];
    double jx = (X0[2] + X0[0]) + X0[1];
    const double kxz = X0[2] - X0[0];
    const double kxy = (X1[2] + X1[0]) + X1[1];
    const double kxx = ((m[2] + m[5]) + (m[8] + m[11])) + ((m[14] + m[17]) + (m[20] + m[23])) + m[26];

    mo.j[0] = jx;
    mo.j[1] = jy;
    mo.j[2] = jz;
    jx = fma(0.5, F[0], jx);
    if constexpr (!XO) {
        jy = fma(0.5, F[1], jy);
        jz = fma(0.5, F[2], jz);
    }
    const double rinv = __drcp_rn(rho);
    mo.rho = rho;
    mo.jf[0] = jx;
    mo.jf[1] = jy;
    mo.jf[2] = jz;
    mo.rinv = rinv;
    const double ux = jx * rinv, uy = jy * rinv, uz = jz * rinv;

    // Second-order central moments (the first ones vanish) and their relaxation.
    const double cxx = fma(-jx, ux, kxx), cyy = fma(-jy, uy, kyy), czz = fma(-jz, uz, kzz);
    const double T = cxx + cyy + czz;
    const double D1 = cxx - cyy, D2 = cxx - czz;
    const double Ts = fma(w.wb, rho - T, T);
    const double rs = 1.0 - w.ws;
    const double rh = 0.5 * rs, rq = 0.25 * rs;
    const double D1h = rh * D1, D2h = rh * D2;
    const double sxx = fma(Ts, 1.0 / 6.0, (D1h + D2h) * (1.0 / 3.0));
    // halved post-collision central moments (orders 3..6 at their Maxwellian values)
#pragma unroll
    for (int k = 0; k < 27; k++) m[k] = 0.0;
    m[0] = rho;
    m[2] = sxx;
    m[6] = sxx - D1h;
    m[18] = sxx - D2h;
    m[4] = rq * fma(-jx, uy, kxy);
    m[10] = rq * fma(-jx, uz, kxz);
    m[12] = rq * fma(-jy, uz, kyz);
    const double e4 = rho * (1.0 / 36.0);
    m[8] = e4;
    m[20] = e4;
    m[24] = e4;
    m[26] = rho * (1.0 / 216.0);
    finish<kZeroW1, XO>(m, ux, uy, uz, F, Fq);
}

// XO: the force has no y and z components (checked on the host).
template <int FK, bool W1, bool XO>
__global__ void __launch_bounds__(kBlock)
k_step(const __grid_constant__ Planes<double, 27> P, Geom g, FieldDev Fd, double apre, double apost, Rates27 w)
{
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    double m[27];
    load_pulled<LD3Q27>(P, g, x, y, z, i, m);
    double F[3] = {0.0, 0.0, 0.0}, Fq[3] = {0.0, 0.0, 0.0};
    if (FK != FK_NONE) {
#pragma unroll
        for (int d = 0; d < (XO ? 1 : 3); d++) {
            const double P = field_value(Fd, FK, d, x, y, z, i);
            F[d] = apre * P;
            Fq[d] = apost * P;
        }
    }
    Mom27 mo;
    if (W1) collide_w1<XO>(m, F, Fq, w, mo);
    else collide<XO>(m, F, Fq, w, mo);
#pragma unroll
    for (int a = 0; a < 27; a++) P.out[a][i] = m[a];
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
    double m[27];
    load_pulled<LD3Q27>(fin, g, x, y, z, i, m);
    double F[3] = {0.0, 0.0, 0.0}, Fq[3] = {0.0, 0.0, 0.0};
    if (B.fkind != FK_NONE) {
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const double P = field_value(B.F, B.fkind, d, x, y, z, i);
            F[d] = ap.x * P;
            Fq[d] = ap.y * P;
        }
    }
    const Rates27 w{B.coef[0], B.coef[1], B.coef[2], B.coef[3], B.coef[4], B.coef[5]};
    Mom27 mo;
    if (B.variant == 3) collide_w1<true>(m, F, Fq, w, mo);  // uniform over the member
    else if (B.variant == 1) collide_w1<false>(m, F, Fq, w, mo);
    else collide(m, F, Fq, w, mo);
    if (L.mrho) {
        // fused readback of f(t)'s fields from the collision's own moments;
        // the same bits as store_fields (F = a_pre P, so fma(0.5, F, j) is
        // j + (a_pre P)/2 rounded once)
        const bool forced = L.mhalf && B.fkind != FK_NONE;
        const double jd[3] = {forced ? mo.jf[0] : mo.j[0], forced ? mo.jf[1] : mo.j[1], forced ? mo.jf[2] : mo.j[2]};
        put_fields<LD3Q27>(mo.rho, jd, mo.rinv, i, g.N, __ldg(L.moff + it), L.mrho, L.mu);
    }
#pragma unroll
    for (int a = 0; a < 27; a++) fout[a * g.Np + i] = m[a];
}

template <int TB, int MODE>
__global__ void __launch_bounds__(TB) k_batch(const __grid_constant__ BatchLaunch L)
{
    batch_tiles<TB, MODE>(L, [](const BatchItem &B, const BatchLaunch &L2, int it, int i) { batch_node(B, L2, it, i); });
}

bool high_rates_one(const double *om) { return om[3] == 1.0 && om[4] == 1.0 && om[5] == 1.0 && om[6] == 1.0; }

}  // namespace

// coef[0..5] = omega[1..6]
void d3q27_batch_coef(const double omega[9], BatchItem &item)
{
    for (int k = 0; k < 6; k++) item.coef[k] = omega[k + 1];
}

cudaError_t d3q27_batch_step(const BatchLaunch &L, int nblocks, int tile, cudaStream_t s)
{
    LBM_TILED_LAUNCH(k_batch, L, nblocks, tile, s);
}

int d3q27_batch_resident(int tile)
{
    LBM_TILED_RESIDENT(k_batch, tile);
}

bool d3q27_high_rates_one(const double omega[9]) { return high_rates_one(omega); }

cudaError_t d3q27_step(const LaunchArgs &a)
{
    Rates27 w{a.omega[1], a.omega[2], a.omega[3], a.omega[4], a.omega[5], a.omega[6]};
    const int grid = (a.g.N + kBlock - 1) / kBlock;
    const bool w1 = high_rates_one(a.omega);
    const Planes<double, 27> P = make_planes<double, 27>(a.fin, a.fout, a.g.Np);
    const bool xo = force_x_only(a.fkind, a.F, 3);
    switch (a.fkind) {
    case FK_NONE:
        if (w1) k_step<FK_NONE, true, false><<<grid, kBlock, 0, a.stream>>>(P, a.g, a.F, a.apre, a.apost, w);
        else k_step<FK_NONE, false, false><<<grid, kBlock, 0, a.stream>>>(P, a.g, a.F, a.apre, a.apost, w);
        break;
    case FK_CONST:
        if (w1 && xo) k_step<FK_CONST, true, true><<<grid, kBlock, 0, a.stream>>>(P, a.g, a.F, a.apre, a.apost, w);
        else if (w1) k_step<FK_CONST, true, false><<<grid, kBlock, 0, a.stream>>>(P, a.g, a.F, a.apre, a.apost, w);
        else k_step<FK_CONST, false, false><<<grid, kBlock, 0, a.stream>>>(P, a.g, a.F, a.apre, a.apost, w);
        break;
    default:
        if (w1 && xo) k_step<FK_GENERAL, true, true><<<grid, kBlock, 0, a.stream>>>(P, a.g, a.F, a.apre, a.apost, w);
        else if (w1) k_step<FK_GENERAL, true, false><<<grid, kBlock, 0, a.stream>>>(P, a.g, a.F, a.apre, a.apost, w);
        else k_step<FK_GENERAL, false, false><<<grid, kBlock, 0, a.stream>>>(P, a.g, a.F, a.apre, a.apost, w);
        break;
    }
    return cudaGetLastError();
}

}  // namespace lbmk
