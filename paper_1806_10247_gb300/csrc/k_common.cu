// Lattice-generic kernels: equilibrium fill, conversion between f(t) and the
// stored (inverse-streamed) layout, macroscopic moments and deterministic
// FP64 reductions.
#include "lbm_d3q15.cuh"
#include "lbm_internal.h"
#include "lbm_lattices.cuh"

namespace lbmk {
namespace {

constexpr int kBlock = 256;

int grid_for(long long n, int block = kBlock) { return (int)((n + block - 1) / block); }

// 1D Maxwellian profile with c_s^2 = 1/3 on the velocities -1, 0, +1: the
// unique populations whose moments of order 0, 1, 2 are 1, u, 1/3 + u^2.
__device__ __forceinline__ double maxwell1d(int e, double u)
{
    double s = (1.0 / 3.0) + u * u;
    if (e == 0) return 1.0 - s;
    return 0.5 * (s + (double)e * u);
}

// Deviation moments of a node in double: dm0 = sum d, j = sum d e.
template <class L, class T>
__device__ __forceinline__ void dev_moments(const T *__restrict__ fin, const Geom &g, int x, int y, int z, int i,
                                            double &dm0, double (&j)[3])
{
    float d[L::Q];
    load_pulled_dev<L, T>(fin, g, x, y, z, i, d);
    double dd[L::Q];
#pragma unroll
    for (int a = 0; a < L::Q; a++) dd[a] = (double)d[a];
    zeroth_first<L>(dd, dm0, j);
}

// Equilibrium populations whose central moments are Eq. 20 (flow; the
// product of 1D profiles, which reproduces c_s^2 rho per squared direction;
// for D3Q15 the populations with the Maxwellian moments of its fifteen basis
// monomials) or Eq. 39 (D2Q5 scalar: moments phi, phi u, phi (1/3 + u^2)).
template <class L>
__global__ void __launch_bounds__(kBlock)
k_equilibrium(Geom g, double rho0, double u0x, double u0y, double u0z, const double *__restrict__ rho,
              const double *__restrict__ u, double *__restrict__ dst)
{
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    double r = rho ? rho[i] : rho0;
    double ux = u ? u[i] : u0x;
    double uy = u ? u[(long long)g.N + i] : u0y;
    double uz = (u && L::DIM == 3) ? u[2LL * g.N + i] : u0z;
#pragma unroll
    for (int a = 0; a < L::Q; a++) {
        double v;
        if (L::Q == 15) {
            v = d3q15_equilibrium(r, ux, uy, uz, a);
        } else if (L::Q == 5) {
            const int ex = L::ex(a), ey = L::ey(a);
            if (ex == 0 && ey == 0) v = r * ((1.0 / 3.0) - ux * ux - uy * uy);
            else if (ex != 0) v = 0.5 * r * ((1.0 / 3.0) + ux * ux + (double)ex * ux);
            else v = 0.5 * r * ((1.0 / 3.0) + uy * uy + (double)ey * uy);
        } else {
            v = r * maxwell1d(L::ex(a), ux) * maxwell1d(L::ey(a), uy);
            if (L::DIM == 3) v *= maxwell1d(L::ez(a), uz);
        }
        dst[a * g.Np + i] = v;
    }
}

// stored_a(x - e_a) = f_a(x)  (or stored_opp(a)(x) = f_a(x) beyond a wall):
// the inverse of the pull, so that pulling the stored layout returns f.
template <class L>
__global__ void __launch_bounds__(kBlock)
k_scatter(Geom g, const double *__restrict__ plain, double *__restrict__ stored)
{
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
#pragma unroll
    for (int a = 0; a < L::Q; a++) {
        bool opp;
        int off = pull_off(g, x, y, z, L::ex(a), L::ey(a), L::ez(a), opp);
        stored[(opp ? L::opp(a) : a) * g.Np + off] = plain[a * g.Np + i];
    }
}

template <class L>
__global__ void __launch_bounds__(kBlock)
k_gather(Geom g, const double *__restrict__ stored, double *__restrict__ plain)
{
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    double f[L::Q];
    load_pulled<L>(stored, g, x, y, z, i, f);
#pragma unroll
    for (int a = 0; a < L::Q; a++) plain[a * g.Np + i] = f[a];
}

// Macroscopic fields of f(t): Eq. 24 plus h * Eq. 25 (flow), Eq. 42 plus
// h * Eq. 43 (scalar).  Outputs are dense [N] / [dim][N] arrays.
template <class L>
__global__ void __launch_bounds__(kBlock)
k_moments(Geom g, const double *__restrict__ fin, int fkind, FieldDev F, double apre, int half,
          double *__restrict__ rho, double *__restrict__ u)
{
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    double f[L::Q];
    load_pulled<L>(fin, g, x, y, z, i, f);
    double m0, j[3];
    zeroth_first<L>(f, m0, j);
    store_fields<L>(m0, j, half && fkind != FK_NONE, apre, F, fkind, x, y, z, i, g.N, 0, rho, u);
}

// Reduction slots.
enum { R_MASS = 0, R_JX, R_JY, R_JZ, R_DU, R_BAD, R_SLOTS = 8 };

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Reduces v[R_SLOTS] over the block (sums, except max for R_DU and R_BAD);
// thread 0 writes the result.  Fixed order: deterministic for a fixed grid.
__device__ void block_reduce_store(double (&v)[R_SLOTS], double *out)
{
    __shared__ double sh[kBlock / 32][R_SLOTS];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int s = 0; s < R_SLOTS; s++) v[s] = (s == R_DU || s == R_BAD) ? warp_max(v[s]) : warp_sum(v[s]);
    if (lane == 0)
#pragma unroll
        for (int s = 0; s < R_SLOTS; s++) sh[warp][s] = v[s];
    __syncthreads();
    if (warp == 0) {
#pragma unroll
        for (int s = 0; s < R_SLOTS; s++) {
            double w = lane < kBlock / 32 ? sh[lane][s] : 0.0;
            v[s] = (s == R_DU || s == R_BAD) ? warp_max(w) : warp_sum(w);
        }
        if (lane == 0)
#pragma unroll
            for (int s = 0; s < R_SLOTS; s++) out[s] = v[s];
    }
}

// Per-block partial sums of rho (or phi^o) and momentum, the largest change
// of the half-forced velocity (or scalar) since the snapshot (the snapshot is
// then overwritten), and a flag for non-finite or non-positive densities.
template <class L>
__global__ void __launch_bounds__(kBlock)
k_reduce_partial(Geom g, const double *__restrict__ fin, int fkind, FieldDev F, double apre,
                 double *__restrict__ snap, int have_snap, double *__restrict__ partials)
{
    double v[R_SLOTS] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long n = blockIdx.x * (long long)kBlock + threadIdx.x; n < g.N; n += (long long)gridDim.x * kBlock) {
        const int i = (int)n;
        int x, y, z;
        node_xyz(g, i, x, y, z);
        double f[L::Q];
        load_pulled<L>(fin, g, x, y, z, i, f);
        double m0, j[3];
        zeroth_first<L>(f, m0, j);
        v[R_MASS] += m0;
        bool bad = !isfinite(m0) || (L::Q != 5 && !(m0 > 0.0));
        if (L::Q == 5) {
            double phi = fkind != FK_NONE ? m0 + 0.5 * (apre * field_value(F, fkind, 0, x, y, z, i)) : m0;
            if (have_snap) v[R_DU] = fmax(v[R_DU], fabs(phi - snap[i]));
            snap[i] = phi;
        } else {
#pragma unroll
            for (int d = 0; d < L::DIM; d++) {
                v[R_JX + d] += j[d];
                double jd = fkind != FK_NONE ? j[d] + 0.5 * (apre * field_value(F, fkind, d, x, y, z, i)) : j[d];
                double ud = jd / m0;
                bad = bad || !isfinite(ud);
                if (have_snap) v[R_DU] = fmax(v[R_DU], fabs(ud - snap[(long long)d * g.N + i]));
                snap[(long long)d * g.N + i] = ud;
            }
        }
        if (bad) v[R_BAD] = 1.0;
    }
    block_reduce_store(v, partials + (size_t)blockIdx.x * R_SLOTS);
}

// Same partial sums without the velocity snapshot (mass, momentum and the
// instability flag only); writes nothing but its partials slot.
template <class L>
__global__ void __launch_bounds__(kBlock)
k_reduce_partial_sums(Geom g, const double *__restrict__ fin, double *__restrict__ partials)
{
    double v[R_SLOTS] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long n = blockIdx.x * (long long)kBlock + threadIdx.x; n < g.N; n += (long long)gridDim.x * kBlock) {
        const int i = (int)n;
        int x, y, z;
        node_xyz(g, i, x, y, z);
        double f[L::Q];
        load_pulled<L>(fin, g, x, y, z, i, f);
        double m0, j[3];
        zeroth_first<L>(f, m0, j);
        v[R_MASS] += m0;
        bool bad = !isfinite(m0) || (L::Q != 5 && !(m0 > 0.0));
        if (L::Q != 5)
#pragma unroll
            for (int d = 0; d < L::DIM; d++) v[R_JX + d] += j[d];
        if (bad) v[R_BAD] = 1.0;
    }
    block_reduce_store(v, partials + (size_t)blockIdx.x * R_SLOTS);
}

template <class L, class T>
__global__ void __launch_bounds__(kBlock)
k_reduce_partial_rp(Geom g, const T *__restrict__ fin, double rho_ref, int fkind, FieldDev F, double apre,
                    double *__restrict__ snap, int have_snap, int with_snap, double *__restrict__ partials)
{
    double v[R_SLOTS] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long n = blockIdx.x * (long long)kBlock + threadIdx.x; n < g.N; n += (long long)gridDim.x * kBlock) {
        const int i = (int)n;
        int x, y, z;
        node_xyz(g, i, x, y, z);
        double dm0, j[3];
        dev_moments<L, T>(fin, g, x, y, z, i, dm0, j);
        const double m0 = rho_ref + dm0;
        v[R_MASS] += m0;
        bool bad = !isfinite(m0) || (L::Q != 5 && !(m0 > 0.0));
        if (L::Q == 5) {
            if (with_snap) {
                double phi = fkind != FK_NONE ? m0 + 0.5 * (apre * field_value(F, fkind, 0, x, y, z, i)) : m0;
                if (have_snap) v[R_DU] = fmax(v[R_DU], fabs(phi - snap[i]));
                snap[i] = phi;
            }
        } else {
#pragma unroll
            for (int d = 0; d < L::DIM; d++) {
                v[R_JX + d] += j[d];
                if (with_snap) {
                    double jd = fkind != FK_NONE ? j[d] + 0.5 * (apre * field_value(F, fkind, d, x, y, z, i)) : j[d];
                    double ud = jd / m0;
                    bad = bad || !isfinite(ud);
                    if (have_snap) v[R_DU] = fmax(v[R_DU], fabs(ud - snap[(long long)d * g.N + i]));
                    snap[(long long)d * g.N + i] = ud;
                }
            }
        }
        if (bad) v[R_BAD] = 1.0;
    }
    block_reduce_store(v, partials + (size_t)blockIdx.x * R_SLOTS);
}

__global__ void __launch_bounds__(kBlock) k_reduce_final(const double *__restrict__ partials, int nblocks,
                                                         double *__restrict__ out)
{
    double v[R_SLOTS] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblocks; b += kBlock)
#pragma unroll
        for (int s = 0; s < R_SLOTS; s++) {
            double p = partials[(size_t)b * R_SLOTS + s];
            v[s] = (s == R_DU || s == R_BAD) ? fmax(v[s], p) : v[s] + p;
        }
    block_reduce_store(v, out);
}

// Discrete l2 error terms of Eq. sca: per-block sums of (q - q_ref)^2 (slot 0)
// and q_ref^2 (slot 1) over n values, grid-stride, fixed order.
__global__ void __launch_bounds__(kBlock)
k_l2_partial(const double *__restrict__ q, const double *__restrict__ ref, long long n, double *__restrict__ partials)
{
    double v[R_SLOTS] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (long long k = blockIdx.x * (long long)kBlock + threadIdx.x; k < n; k += (long long)gridDim.x * kBlock) {
        const double r = ref[k], d = q[k] - r;
        v[0] = fma(d, d, v[0]);
        v[1] = fma(r, r, v[1]);
    }
    block_reduce_store(v, partials + (size_t)blockIdx.x * R_SLOTS);
}

// ---- reduced-precision storage: deviations d = f - w rho_ref in type T ----
// (D2Q5: d = g - g_ref, the reference populations of the context.)

template <class L>
__device__ __forceinline__ double ref_pop(int a, double rho_ref, const Ref5 &R)
{
    if constexpr (L::Q == 5) return R.v[a];
    else return L::w(a) * rho_ref;
}

template <class L, class T>
__global__ void __launch_bounds__(kBlock)
k_init_rp(Geom g, double rho_ref, Ref5 R, double rho0, double u0x, double u0y, double u0z,
          const double *__restrict__ rho, const double *__restrict__ u, T *__restrict__ stored)
{
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    double r = rho ? rho[i] : rho0;
    double ux = u ? u[i] : u0x;
    double uy = u ? u[(long long)g.N + i] : u0y;
    double uz = (u && L::DIM == 3) ? u[2LL * g.N + i] : u0z;
#pragma unroll
    for (int a = 0; a < L::Q; a++) {
        double v;
        if (L::Q == 15) {
            v = d3q15_equilibrium(r, ux, uy, uz, a);
        } else if (L::Q == 5) {
            const int ex = L::ex(a), ey = L::ey(a);
            if (ex == 0 && ey == 0) v = r * ((1.0 / 3.0) - ux * ux - uy * uy);
            else if (ex != 0) v = 0.5 * r * ((1.0 / 3.0) + ux * ux + (double)ex * ux);
            else v = 0.5 * r * ((1.0 / 3.0) + uy * uy + (double)ey * uy);
        } else {
            v = r * maxwell1d(L::ex(a), ux) * maxwell1d(L::ey(a), uy);
            if (L::DIM == 3) v *= maxwell1d(L::ez(a), uz);
        }
        bool opp;
        int off = pull_off(g, x, y, z, L::ex(a), L::ey(a), L::ez(a), opp);
        const int slot = opp ? L::opp(a) : a;
        stored[slot * g.Np + off] = Dev<T>::to_store((float)(v - ref_pop<L>(slot, rho_ref, R)));
    }
}

template <class L, class T>
__global__ void __launch_bounds__(kBlock)
k_scatter_rp(Geom g, double rho_ref, Ref5 R, const double *__restrict__ plain, T *__restrict__ stored)
{
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
#pragma unroll
    for (int a = 0; a < L::Q; a++) {
        bool opp;
        int off = pull_off(g, x, y, z, L::ex(a), L::ey(a), L::ez(a), opp);
        const int slot = opp ? L::opp(a) : a;
        const double v = plain[(size_t)a * g.N + i] - ref_pop<L>(slot, rho_ref, R);
        stored[slot * g.Np + off] = Dev<T>::to_store((float)v);
    }
}

template <class L, class T>
__global__ void __launch_bounds__(kBlock)
k_gather_rp(Geom g, double rho_ref, Ref5 R, const T *__restrict__ stored, double *__restrict__ plain)
{
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    float d[L::Q];
    load_pulled_dev<L, T>(stored, g, x, y, z, i, d);
    // a population pulled from beyond a wall comes from the opposite slot,
    // whose reference it carries (the D2Q5 equilibrium reference is used on
    // periodic lattices only, and w(opp a) = w(a))
#pragma unroll
    for (int a = 0; a < L::Q; a++) plain[(size_t)a * g.N + i] = ref_pop<L>(a, rho_ref, R) + (double)d[a];
}

template <class L, class T>
__global__ void __launch_bounds__(kBlock)
k_moments_rp(Geom g, const T *__restrict__ fin, double rho_ref, int fkind, FieldDev F, double apre, int half,
             double *__restrict__ rho, double *__restrict__ u)
{
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    double dm0, j[3];
    dev_moments<L, T>(fin, g, x, y, z, i, dm0, j);
    const double m0 = rho_ref + dm0;
    store_fields<L>(m0, j, half && fkind != FK_NONE, apre, F, fkind, x, y, z, i, g.N, 0, rho, u);
}

// Strain rate from the non-equilibrium second moments (Sec. 6.6): with
// Pi = sum f e e - rho u u - rho c_s^2 I about the half-forced u,
// S_ab = -(3 ws / (2 rho0)) Pi_ab (a != b) and, splitting the diagonal into
// trace T and deviatoric parts D_a = Pi_aa - T/dim,
// S_aa = -(3 / (2 rho0)) (wd D_a + wb T/dim).  Order: xx, yy, (zz,) xy, (xz, yz).
struct StrainRates {
    double ws, wd, wb;
};

template <class L>
__device__ __forceinline__ void strain_node(const double (&f)[L::Q], const double (&Fh)[3], double rho0,
                                            const StrainRates &r, double *__restrict__ out, long long N, int i)
{
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0}, m[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int a = 0; a < L::Q; a++) {
        const double ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
        rho += f[a];
        j[0] += ex * f[a];
        j[1] += ey * f[a];
        j[2] += ez * f[a];
        m[0] += ex * ex * f[a];
        m[1] += ey * ey * f[a];
        m[2] += ez * ez * f[a];
        m[3] += ex * ey * f[a];
        m[4] += ex * ez * f[a];
        m[5] += ey * ez * f[a];
    }
    const double ux = (j[0] + Fh[0]) / rho, uy = (j[1] + Fh[1]) / rho, uz = (j[2] + Fh[2]) / rho;
    const double c = rho / 3.0;
    const double pxx = m[0] - rho * ux * ux - c, pyy = m[1] - rho * uy * uy - c;
    const double pxy = m[3] - rho * ux * uy;
    const double k = -1.5 / rho0;
    if (L::DIM == 2) {
        const double T = pxx + pyy;
        out[i] = k * (r.wd * (pxx - 0.5 * T) + r.wb * 0.5 * T);
        out[N + i] = k * (r.wd * (pyy - 0.5 * T) + r.wb * 0.5 * T);
        out[2 * N + i] = k * r.ws * pxy;
    } else {
        const double pzz = m[2] - rho * uz * uz - c;
        const double pxz = m[4] - rho * ux * uz, pyz = m[5] - rho * uy * uz;
        const double T = pxx + pyy + pzz;
        out[i] = k * (r.wd * (pxx - T / 3.0) + r.wb * T / 3.0);
        out[N + i] = k * (r.wd * (pyy - T / 3.0) + r.wb * T / 3.0);
        out[2 * N + i] = k * (r.wd * (pzz - T / 3.0) + r.wb * T / 3.0);
        out[3 * N + i] = k * r.ws * pxy;
        out[4 * N + i] = k * r.ws * pxz;
        out[5 * N + i] = k * r.ws * pyz;
    }
}

template <class L>
__global__ void __launch_bounds__(kBlock)
k_strain(Geom g, const double *__restrict__ fin, int fkind, FieldDev F, double apre, double rho0, StrainRates r,
         double *__restrict__ out)
{
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    double f[L::Q];
    load_pulled<L>(fin, g, x, y, z, i, f);
    double Fh[3] = {0.0, 0.0, 0.0};
    if (fkind != FK_NONE)
        for (int d = 0; d < L::DIM; d++) Fh[d] = 0.5 * (apre * field_value(F, fkind, d, x, y, z, i));
    strain_node<L>(f, Fh, rho0, r, out, g.N, i);
}

template <class L, class T>
__global__ void __launch_bounds__(kBlock)
k_strain_rp(Geom g, const T *__restrict__ fin, double rho_ref, int fkind, FieldDev F, double apre, double rho0,
            StrainRates r, double *__restrict__ out)
{
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    float d[L::Q];
    load_pulled_dev<L, T>(fin, g, x, y, z, i, d);
    double f[L::Q];
#pragma unroll
    for (int a = 0; a < L::Q; a++) f[a] = L::w(a) * rho_ref + (double)d[a];
    double Fh[3] = {0.0, 0.0, 0.0};
    if (fkind != FK_NONE)
        for (int dd = 0; dd < L::DIM; dd++) Fh[dd] = 0.5 * (apre * field_value(F, fkind, dd, x, y, z, i));
    strain_node<L>(f, Fh, rho0, r, out, g.N, i);
}

// Viscous heating source coef * S:S (Sec. 6.6, S_r = (2 nu / C_v) S:S) from the
// strain components; written as a full source field (FP64 and FP32 copy).
__global__ void __launch_bounds__(kBlock)
k_viscous_source(int n, int dim, const double *__restrict__ S, double coef, double *__restrict__ out,
                 float *__restrict__ fout)
{
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= n) return;
    const long long N = n;  // component stride: 64-bit offsets
    double v;
    if (dim == 2) {
        const double a = S[i], b = S[N + i], c = S[2 * N + i];
        v = a * a + b * b + 2.0 * c * c;
    } else {
        double d2 = 0.0, o2 = 0.0;
        for (int k = 0; k < 3; k++) d2 += S[k * N + i] * S[k * N + i];
        for (int k = 3; k < 6; k++) o2 += S[k * N + i] * S[k * N + i];
        v = d2 + 2.0 * o2;
    }
    out[i] = coef * v;
    if (fout) fout[i] = (float)(coef * v);
}

template <class Fn>
cudaError_t by_storage(int storage, Fn &&fn)
{
    switch (storage) {
    case 1: return fn(float{});
    case 2: return fn(__half{});
    case 3: return fn(__nv_bfloat16{});
    default: return cudaErrorInvalidValue;
    }
}

// Lattices with reduced-precision storage.
template <class Fn>
cudaError_t by_lattice(int lattice, Fn &&fn)
{
    switch (lattice) {
    case LD2Q9::ID: return fn(LD2Q9{});
    case LD2Q5::ID: return fn(LD2Q5{});
    case LD3Q27::ID: return fn(LD3Q27{});
    default: return cudaErrorInvalidValue;
    }
}

// Every lattice (FP64 storage).
template <class Fn>
cudaError_t by_lattice64(int lattice, Fn &&fn)
{
    if (lattice == LD3Q15::ID) return fn(LD3Q15{});
    return by_lattice(lattice, fn);
}

}  // namespace

cudaError_t equilibrium(int lattice, const Geom &g, double rho0, const double *u0, const double *rho,
                        const double *u, double *dst, cudaStream_t s)
{
    return by_lattice64(lattice, [&](auto L) {
        using LT = decltype(L);
        k_equilibrium<LT><<<grid_for(g.N), kBlock, 0, s>>>(g, rho0, u0[0], u0[1], u0[2], rho, u, dst);
        return cudaGetLastError();
    });
}

cudaError_t scatter_to_stored(int lattice, const Geom &g, const double *plain, double *stored,
                              cudaStream_t s)
{
    return by_lattice64(lattice, [&](auto L) {
        using LT = decltype(L);
        k_scatter<LT><<<grid_for(g.N), kBlock, 0, s>>>(g, plain, stored);
        return cudaGetLastError();
    });
}

cudaError_t gather_from_stored(int lattice, const Geom &g, const double *stored, double *plain,
                               cudaStream_t s)
{
    return by_lattice64(lattice, [&](auto L) {
        using LT = decltype(L);
        k_gather<LT><<<grid_for(g.N), kBlock, 0, s>>>(g, stored, plain);
        return cudaGetLastError();
    });
}

cudaError_t moments(int lattice, const LaunchArgs &a, double *rho, double *u, int half)
{
    if (a.storage != 0)
        return by_lattice(lattice, [&](auto L) {
            using LT = decltype(L);
            return by_storage(a.storage, [&](auto T) {
                using TT = decltype(T);
                k_moments_rp<LT, TT><<<grid_for(a.g.N), kBlock, 0, a.stream>>>(
                    a.g, reinterpret_cast<const TT *>(a.fin), a.rho_ref, a.fkind, a.F, a.apre, half, rho, u);
                return cudaGetLastError();
            });
        });
    return by_lattice64(lattice, [&](auto L) {
        using LT = decltype(L);
        k_moments<LT><<<grid_for(a.g.N), kBlock, 0, a.stream>>>(a.g, a.fin, a.fkind, a.F, a.apre, half,
                                                                rho, u);
        return cudaGetLastError();
    });
}

cudaError_t strain_rate(int lattice, const LaunchArgs &a, double rho0, double *out)
{
    StrainRates r;
    if (lattice == LD2Q9::ID) r = StrainRates{a.omega[5], a.omega[4], a.omega[3]};
    else r = StrainRates{a.omega[2], a.omega[2], a.omega[1]};
    if (lattice == LD2Q5::ID) return cudaErrorInvalidValue;
    if (a.storage != 0)
        return by_lattice(lattice, [&](auto L) {
            using LT = decltype(L);
            if (LT::Q == 5) return cudaErrorInvalidValue;
            return by_storage(a.storage, [&](auto T) {
                using TT = decltype(T);
                k_strain_rp<LT, TT><<<grid_for(a.g.N), kBlock, 0, a.stream>>>(
                    a.g, reinterpret_cast<const TT *>(a.fin), a.rho_ref, a.fkind, a.F, a.apre, rho0, r, out);
                return cudaGetLastError();
            });
        });
    return by_lattice64(lattice, [&](auto L) {
        using LT = decltype(L);
        if (LT::Q == 5) return cudaErrorInvalidValue;
        k_strain<LT><<<grid_for(a.g.N), kBlock, 0, a.stream>>>(a.g, a.fin, a.fkind, a.F, a.apre, rho0, r, out);
        return cudaGetLastError();
    });
}

__global__ void __launch_bounds__(kBlock) k_to_float(const double *__restrict__ in, float *__restrict__ out, long long n)
{
    const long long i = (long long)blockIdx.x * kBlock + threadIdx.x;
    if (i < n) out[i] = __double2float_rn(in[i]);
}

cudaError_t to_float(const double *in, float *out, long long n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    k_to_float<<<(unsigned)((n + kBlock - 1) / kBlock), kBlock, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t viscous_source(int N, int dim, const double *S, double coef, double *out, float *fout, cudaStream_t s)
{
    k_viscous_source<<<grid_for(N), kBlock, 0, s>>>(N, dim, S, coef, out, fout);
    return cudaGetLastError();
}

int reduce_blocks(const Geom &g)
{
    long long b = (g.N + kBlock - 1) / kBlock;
    return (int)(b < kReduceMaxBlocks ? (b < 1 ? 1 : b) : kReduceMaxBlocks);
}

cudaError_t l2_terms(const double *q, const double *ref, long long n, double *partials, int nblocks, double *out,
                     cudaStream_t s)
{
    k_l2_partial<<<nblocks, kBlock, 0, s>>>(q, ref, n, partials);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_final<<<1, kBlock, 0, s>>>(partials, nblocks, out);
    return cudaGetLastError();
}

cudaError_t reduce(int lattice, const LaunchArgs &a, double *snap, int have_snap, double *partials,
                   int nblocks, double *out)
{
    if (a.storage != 0)
        return by_lattice(lattice, [&](auto L) {
            using LT = decltype(L);
            return by_storage(a.storage, [&](auto T) {
                using TT = decltype(T);
                k_reduce_partial_rp<LT, TT><<<nblocks, kBlock, 0, a.stream>>>(
                    a.g, reinterpret_cast<const TT *>(a.fin), a.rho_ref, a.fkind, a.F, a.apre, snap, have_snap, 1,
                    partials);
                cudaError_t e = cudaGetLastError();
                if (e != cudaSuccess) return e;
                k_reduce_final<<<1, kBlock, 0, a.stream>>>(partials, nblocks, out);
                return cudaGetLastError();
            });
        });
    return by_lattice64(lattice, [&](auto L) {
        using LT = decltype(L);
        k_reduce_partial<LT><<<nblocks, kBlock, 0, a.stream>>>(a.g, a.fin, a.fkind, a.F, a.apre, snap,
                                                              have_snap, partials);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_reduce_final<<<1, kBlock, 0, a.stream>>>(partials, nblocks, out);
        return cudaGetLastError();
    });
}

cudaError_t rp_init_equilibrium(int lattice, int storage, const Geom &g, double rho_ref, const Ref5 &gref,
                                double rho0, const double *u0, const double *rho, const double *u, void *stored,
                                cudaStream_t s)
{
    return by_lattice(lattice, [&](auto L) {
        using LT = decltype(L);
        return by_storage(storage, [&](auto T) {
            using TT = decltype(T);
            k_init_rp<LT, TT><<<grid_for(g.N), kBlock, 0, s>>>(g, rho_ref, gref, rho0, u0[0], u0[1], u0[2], rho, u,
                                                              reinterpret_cast<TT *>(stored));
            return cudaGetLastError();
        });
    });
}

cudaError_t rp_scatter(int lattice, int storage, const Geom &g, double rho_ref, const Ref5 &gref,
                       const double *plain, void *stored, cudaStream_t s)
{
    return by_lattice(lattice, [&](auto L) {
        using LT = decltype(L);
        return by_storage(storage, [&](auto T) {
            using TT = decltype(T);
            k_scatter_rp<LT, TT><<<grid_for(g.N), kBlock, 0, s>>>(g, rho_ref, gref, plain,
                                                                 reinterpret_cast<TT *>(stored));
            return cudaGetLastError();
        });
    });
}

cudaError_t rp_gather(int lattice, int storage, const Geom &g, double rho_ref, const Ref5 &gref, const void *stored,
                      double *plain, cudaStream_t s)
{
    return by_lattice(lattice, [&](auto L) {
        using LT = decltype(L);
        return by_storage(storage, [&](auto T) {
            using TT = decltype(T);
            k_gather_rp<LT, TT><<<grid_for(g.N), kBlock, 0, s>>>(g, rho_ref, gref,
                                                                reinterpret_cast<const TT *>(stored), plain);
            return cudaGetLastError();
        });
    });
}

void d2q9_batch_coef(const double omega[9], BatchItem &item);
void d2q5_batch_coef(const double omega[9], BatchItem &item);
void d3q27_batch_coef(const double omega[9], BatchItem &item);
void d3q15_batch_coef(const double omega[9], BatchItem &item);
cudaError_t d2q9_batch_step(const BatchLaunch &, int, int, cudaStream_t);
cudaError_t d2q5_batch_step(const BatchLaunch &, int, int, cudaStream_t);
cudaError_t d3q27_batch_step(const BatchLaunch &, int, int, cudaStream_t);
cudaError_t d3q15_batch_step(const BatchLaunch &, int, int, cudaStream_t);
int d2q9_batch_resident(int);
int d2q5_batch_resident(int);
int d3q27_batch_resident(int);
int d3q15_batch_resident(int);

void batch_coef(int lattice, const double omega[9], BatchItem &item)
{
    if (lattice == LD2Q9::ID) d2q9_batch_coef(omega, item);
    else if (lattice == LD2Q5::ID) d2q5_batch_coef(omega, item);
    else if (lattice == LD3Q15::ID) d3q15_batch_coef(omega, item);
    else d3q27_batch_coef(omega, item);
}

cudaError_t batch_step(int lattice, const BatchLaunch &L, int nblocks, int tile, cudaStream_t s)
{
    if (lattice == LD2Q9::ID) return d2q9_batch_step(L, nblocks, tile, s);
    if (lattice == LD2Q5::ID) return d2q5_batch_step(L, nblocks, tile, s);
    if (lattice == LD3Q15::ID) return d3q15_batch_step(L, nblocks, tile, s);
    return d3q27_batch_step(L, nblocks, tile, s);
}

bool d3q27_high_rates_one(const double omega[9]);
bool d2q9_high_rates_one(const double omega[9]);

int batch_variant(int lattice, const double omega[9], int fkind, const FieldDev &F)
{
    int w1 = 0, dim = 2;
    if (lattice == LD3Q27::ID) {
        w1 = d3q27_high_rates_one(omega) ? 1 : 0;
        dim = 3;
    } else if (lattice == LD2Q9::ID) {
        w1 = d2q9_high_rates_one(omega) ? 1 : 0;
    }
    return w1 && force_x_only(fkind, F, dim) ? 3 : w1;
}

int batch_resident(int lattice, int tile)
{
    if (lattice == LD2Q9::ID) return d2q9_batch_resident(tile);
    if (lattice == LD2Q5::ID) return d2q5_batch_resident(tile);
    if (lattice == LD3Q15::ID) return d3q15_batch_resident(tile);
    return d3q27_batch_resident(tile);
}


cudaError_t reduce_sums(int lattice, const LaunchArgs &a, double *partials, int nblocks, double *out)
{
    if (a.storage != 0)
        return by_lattice(lattice, [&](auto L) {
            using LT = decltype(L);
            return by_storage(a.storage, [&](auto T) {
                using TT = decltype(T);
                k_reduce_partial_rp<LT, TT><<<nblocks, kBlock, 0, a.stream>>>(
                    a.g, reinterpret_cast<const TT *>(a.fin), a.rho_ref, a.fkind, a.F, a.apre, nullptr, 0, 0,
                    partials);
                cudaError_t e = cudaGetLastError();
                if (e != cudaSuccess) return e;
                k_reduce_final<<<1, kBlock, 0, a.stream>>>(partials, nblocks, out);
                return cudaGetLastError();
            });
        });
    return by_lattice64(lattice, [&](auto L) {
        using LT = decltype(L);
        k_reduce_partial_sums<LT><<<nblocks, kBlock, 0, a.stream>>>(a.g, a.fin, partials);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        k_reduce_final<<<1, kBlock, 0, a.stream>>>(partials, nblocks, out);
        return cudaGetLastError();
    });
}

}  // namespace lbmk
