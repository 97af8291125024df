// Velocity sets as compile-time traits, and the per-node helpers that every
// kernel of a lattice shares: pulling the streamed populations of a node and
// the zeroth/first moments.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "lbm_device.cuh"

namespace lbmk {

// D2Q9, Sec. 4 Eq. 15: 0 rest, 1 +x, 2 +y, 3 -x, 4 -y, 5 (+,+), 6 (-,+), 7 (-,-), 8 (+,-).
struct LD2Q9 {
    static constexpr int Q = 9, DIM = 2, ID = 1;
    __host__ __device__ static constexpr int ex(int a) { return (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0); }
    __host__ __device__ static constexpr int ey(int a) { return (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0); }
    __host__ __device__ static constexpr int ez(int) { return 0; }
    __host__ __device__ static constexpr int opp(int a) { return a == 0 ? 0 : (a <= 4 ? ((a + 1) % 4) + 1 : ((a - 3) % 4) + 5); }
    // rest-state populations per unit density (4/9, 1/9, 1/36)
    __host__ __device__ static constexpr double w(int a) { return a == 0 ? 4.0 / 9.0 : (a <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }
};

// D2Q5, Sec. 5 Eq. 34: 0 rest, 1 +x, 2 +y, 3 -x, 4 -y.
struct LD2Q5 {
    static constexpr int Q = 5, DIM = 2, ID = 3;
    __host__ __device__ static constexpr int ex(int a) { return a == 1 ? 1 : (a == 3 ? -1 : 0); }
    __host__ __device__ static constexpr int ey(int a) { return a == 2 ? 1 : (a == 4 ? -1 : 0); }
    __host__ __device__ static constexpr int ez(int) { return 0; }
    __host__ __device__ static constexpr int opp(int a) { return a == 0 ? 0 : ((a + 1) % 4) + 1; }
    // rest-state populations per unit scalar (1/3, 1/6): moments 1, 0, 1/3
    __host__ __device__ static constexpr double w(int a) { return a == 0 ? 1.0 / 3.0 : 1.0 / 6.0; }
};

// D3Q27 in tensor order: a = (ex+1) + 3 (ey+1) + 9 (ez+1); the opposite of a is 26 - a.
struct LD3Q27 {
    static constexpr int Q = 27, DIM = 3, ID = 2;
    __host__ __device__ static constexpr int ex(int a) { return a % 3 - 1; }
    __host__ __device__ static constexpr int ey(int a) { return (a / 3) % 3 - 1; }
    __host__ __device__ static constexpr int ez(int a) { return a / 9 - 1; }
    __host__ __device__ static constexpr int opp(int a) { return 26 - a; }
    // rest-state populations per unit density: product of (1/6, 2/3, 1/6) per axis
    __host__ __device__ static constexpr double w1(int e) { return e == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
    __host__ __device__ static constexpr double w(int a) { return w1(ex(a)) * w1(ey(a)) * w1(ez(a)); }
};

// Source offset of the pull f_a(x) = f^p_a(x - e_a) (Eq. 22b / Eq. 40b) with
// periodic wrap, or the node itself with opp = true when x - e_a lies beyond a
// halfway bounce-back wall (the population comes back reversed).
__device__ __forceinline__ int pull_off(const Geom &g, int x, int y, int z, int ex, int ey, int ez,
                                        bool &opp)
{
    int sx = x - ex, sy = y - ey, sz = z - ez;
    opp = false;
    if (ex != 0 && (sx < 0 || sx >= g.nx)) {
        if (g.wall[0]) opp = true;
        else sx = (sx < 0) ? sx + g.nx : sx - g.nx;
    }
    if (ey != 0 && (sy < 0 || sy >= g.ny)) {
        if (g.wall[1]) opp = true;
        else sy = (sy < 0) ? sy + g.ny : sy - g.ny;
    }
    if (ez != 0 && (sz < 0 || sz >= g.nz)) {
        if (g.wall[2]) opp = true;
        else sz = (sz < 0) ? sz + g.nz : sz - g.nz;
    }
    if (opp) return x + g.nx * (y + g.ny * z);
    return sx + g.nx * (sy + g.ny * sz);
}

// Pulled populations of node i = (x, y, z): get(p, k) returns the stored
// value of plane p at node k.  A node that has no wall beside it takes every
// population along its wrapped periodic offset (no per-population test, so a
// warp whose nodes straddle a periodic edge does not diverge); a node next to
// a wall tests each population with pull_off.
template <class L, class V, class Get>
__device__ __forceinline__ void pull_node(const Geom &g, int x, int y, int z, int i, V (&f)[L::Q], Get get)
{
    const bool wall_x = g.wall[0] && (x == 0 || x == g.nx - 1);
    const bool wall_y = g.wall[1] && (y == 0 || y == g.ny - 1);
    const bool wall_z = L::DIM == 3 && g.wall[2] && (z == 0 || z == g.nz - 1);
    if (!(wall_x || wall_y || wall_z)) {
        // offset of the source node for e = +1 (coordinate - 1) and e = -1
        // (coordinate + 1) along each axis, wrapped
        const int sy = g.nx;
        const int xm = x == 0 ? g.nx - 1 : -1, xp = x == g.nx - 1 ? 1 - g.nx : 1;
        const int ym = y == 0 ? (g.ny - 1) * sy : -sy, yp = y == g.ny - 1 ? (1 - g.ny) * sy : sy;
        int zm = 0, zp = 0;
        if (L::DIM == 3) {
            const int sz = g.nx * g.ny;
            zm = z == 0 ? (g.nz - 1) * sz : -sz;
            zp = z == g.nz - 1 ? (1 - g.nz) * sz : sz;
        }
#pragma unroll
        for (int a = 0; a < L::Q; a++) {
            const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
            const int row = i + (ey == 1 ? ym : (ey == -1 ? yp : 0)) + (ez == 1 ? zm : (ez == -1 ? zp : 0));
            f[a] = get(a, row + (ex == 1 ? xm : (ex == -1 ? xp : 0)));
        }
        return;
    }
#pragma unroll
    for (int a = 0; a < L::Q; a++) {
        const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
        if (ex == 0 && ey == 0 && ez == 0) {
            f[a] = get(a, i);
        } else {
            bool opp;
            const int off = pull_off(g, x, y, z, ex, ey, ez, opp);
            f[a] = get(opp ? L::opp(a) : a, off);
        }
    }
}

template <class L>
__device__ __forceinline__ void load_pulled(const double *__restrict__ fin, const Geom &g, int x, int y,
                                            int z, int i, double (&f)[L::Q])
{
    pull_node<L>(g, x, y, z, i, f, [&](int p, int k) { return __ldg(fin + p * g.Np + k); });
}

// Base pointers of the Q population planes of a step's source and
// destination buffers, passed in the launch arguments: a kernel then
// addresses plane a of node k with one multiply-add on a parameter instead of
// forming the 64-bit product a * Np per access.
template <class T, int Q>
struct Planes {
    const T *in[Q];
    T *out[Q];
};

template <class T, int Q>
inline Planes<T, Q> make_planes(const void *fin, void *fout, long long Np)
{
    Planes<T, Q> P;
    for (int a = 0; a < Q; a++) {
        P.in[a] = static_cast<const T *>(fin) + a * Np;
        P.out[a] = static_cast<T *>(fout) + a * Np;
    }
    return P;
}

// Reduced-precision storage: conversions of a stored deviation to/from float.
template <class T> struct Dev;
template <> struct Dev<float> {
    __device__ static float get(const float *p) { return __ldg(p); }
    __device__ static float to_store(float v) { return v; }
};
// 16-bit values are loaded as plain unsigned shorts (a native read-only load
// the compiler can schedule freely) and reinterpreted.
template <> struct Dev<__half> {
    __device__ static float get(const __half *p)
    {
        return __half2float(__ushort_as_half(__ldg(reinterpret_cast<const unsigned short *>(p))));
    }
    __device__ static __half to_store(float v) { return __float2half_rn(v); }
};
template <> struct Dev<__nv_bfloat16> {
    __device__ static float get(const __nv_bfloat16 *p)
    {
        return __bfloat162float(__ushort_as_bfloat16(__ldg(reinterpret_cast<const unsigned short *>(p))));
    }
    __device__ static __nv_bfloat16 to_store(float v) { return __float2bfloat16_rn(v); }
};

// Pulled deviations of a node (as float) from stored planes of type T.
template <class L, class T>
__device__ __forceinline__ void load_pulled_dev(const T *__restrict__ fin, const Geom &g, int x, int y, int z,
                                                int i, float (&d)[L::Q])
{
    pull_node<L>(g, x, y, z, i, d, [&](int p, int k) { return Dev<T>::get(fin + p * g.Np + k); });
}

// The same pulls through a plane table in the launch arguments.
template <class L>
__device__ __forceinline__ void load_pulled(const Planes<double, L::Q> &P, const Geom &g, int x, int y, int z,
                                            int i, double (&f)[L::Q])
{
    pull_node<L>(g, x, y, z, i, f, [&](int p, int k) { return __ldg(P.in[p] + k); });
}
template <class L, class T>
__device__ __forceinline__ void load_pulled_dev(const Planes<T, L::Q> &P, const Geom &g, int x, int y, int z,
                                                int i, float (&d)[L::Q])
{
    pull_node<L>(g, x, y, z, i, d, [&](int p, int k) { return Dev<T>::get(P.in[p] + k); });
}

// Zeroth and first moments of a node's populations (summed in velocity order).
template <class L>
__device__ __forceinline__ void zeroth_first(const double (&f)[L::Q], double &m0, double (&j)[3])
{
    m0 = f[0];
    j[0] = j[1] = j[2] = 0.0;
#pragma unroll
    for (int a = 0; a < L::Q; a++) {
        if (a > 0) m0 += f[a];
        if (L::ex(a) == 1) j[0] += f[a];
        if (L::ex(a) == -1) j[0] -= f[a];
        if (L::ey(a) == 1) j[1] += f[a];
        if (L::ey(a) == -1) j[1] -= f[a];
        if (L::ez(a) == 1) j[2] += f[a];
        if (L::ez(a) == -1) j[2] -= f[a];
    }
}

// D2Q9: the same sums grouped as the collision groups them (x-moments of the
// rows e_y = 0, +1, -1 first), so that a step kernel's own rho and j are
// these bits and a fused readback can store them without summing again.
template <>
__device__ __forceinline__ void zeroth_first<LD2Q9>(const double (&f)[9], double &m0, double (&j)[3])
{
    const double s0 = f[1] + f[3], s1 = f[5] + f[6], s2 = f[8] + f[7];
    const double B0 = f[2] + s1, C0 = f[4] + s2;
    m0 = (f[0] + s0) + (B0 + C0);
    j[0] = (f[1] - f[3]) + ((f[5] - f[6]) + (f[8] - f[7]));
    j[1] = B0 - C0;
    j[2] = 0.0;
}

// D3Q27: grouped as the factorised collision forms them — the 1D transform
// (f_+ + f_-) + f_0 and f_+ - f_- along x on every line, then along y, then
// along z — so that the collision's own rho and j are these bits.
template <>
__device__ __forceinline__ void zeroth_first<LD3Q27>(const double (&f)[27], double &m0, double (&j)[3])
{
    double Y0[3], Y1[3], XY[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        double X0[3], X1[3];
#pragma unroll
        for (int b = 0; b < 3; b++) {
            const int k = 3 * b + 9 * c;  // velocities (-1, 0, +1) along x at k, k + 1, k + 2
            X0[b] = (f[k + 2] + f[k]) + f[k + 1];
            X1[b] = f[k + 2] - f[k];
        }
        Y0[c] = (X0[2] + X0[0]) + X0[1];
        Y1[c] = X0[2] - X0[0];
        XY[c] = (X1[2] + X1[0]) + X1[1];
    }
    m0 = (Y0[2] + Y0[0]) + Y0[1];
    j[0] = (XY[2] + XY[0]) + XY[1];
    j[1] = (Y1[2] + Y1[0]) + Y1[1];
    j[2] = Y0[2] - Y0[0];
}

// Stores the packed fields of a node: rho (phi for the scalar lattice) at
// rho[off + i] and u_d = jd_d (1/rho) at u[dim * off + d * N + i], with rinv =
// the correctly rounded 1/rho (__drcp_rn) and the product rounded on its own.
template <class L>
__device__ __forceinline__ void put_fields(double m0, const double (&jd)[3], double rinv, int i, int N, long long off,
                                           double *rho, double *u)
{
    rho[off + i] = m0;
    if (L::Q == 5) return;
#pragma unroll
    for (int d = 0; d < L::DIM; d++) u[L::DIM * off + (long long)d * N + i] = __dmul_rn(jd[d], rinv);
}

// The packed fields of a node from its zeroth and first moments, as every
// readback writes them: rho (phi for the scalar lattice) at rho[off + i],
// velocity component d at u[dim * off + d * N + i]; with `forced` the
// pre-collision half force / source a_pre P / 2 is included (Eq. 25 / 43).
// Rounded operation by operation (no contraction), so that every kernel that
// forms them gives the same bits.  A step kernel that has rho, the half-forced
// j and 1/rho at hand stores them with put_fields instead: j + (a_pre P)/2
// rounded once equals fma(0.5, a_pre P, j), and phi + (a_pre/2) P equals
// phi + (a_pre P)/2 (halving is exact for products in the normal range).
template <class L>
__device__ __forceinline__ void store_fields(double m0, const double (&j)[3], bool forced, double apre, const FieldDev &F,
                                             int fkind, int x, int y, int z, int i, int N, long long off, double *rho,
                                             double *u)
{
    if (L::Q == 5) {
        rho[off + i] = forced ? __dadd_rn(m0, __dmul_rn(0.5, __dmul_rn(apre, field_value(F, fkind, 0, x, y, z, i)))) : m0;
        return;
    }
    double jd[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int d = 0; d < L::DIM; d++)
        jd[d] = forced ? __dadd_rn(j[d], __dmul_rn(0.5, __dmul_rn(apre, field_value(F, fkind, d, x, y, z, i)))) : j[d];
    put_fields<L>(m0, jd, __drcp_rn(m0), i, N, off, rho, u);
}

// Copy an object into shared memory cooperatively (word by word); the caller
// synchronises.  Used to give every thread of a block one copy of its batch
// descriptor without repeated global loads.
template <class Obj>
__device__ __forceinline__ void stage_to_shared(Obj &dst, const Obj &src)
{
    static_assert(sizeof(Obj) % 4 == 0, "word copy");
    const unsigned *s = reinterpret_cast<const unsigned *>(&src);
    unsigned *d = reinterpret_cast<unsigned *>(&dst);
    for (int k = threadIdx.x; k < (int)(sizeof(Obj) / 4); k += blockDim.x) d[k] = __ldg(s + k);
}

// Item of a batched launch that owns this block: the last i with
// first_block[i] <= blockIdx.x (first_block ascending, first_block[0] = 0).
__device__ __forceinline__ int batch_find(const int *__restrict__ first_block, int count)
{
    const int b = blockIdx.x;
    int lo = 0, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(first_block + mid) <= b) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Coordinates of node i = x + nx (y + ny z).
__device__ __forceinline__ void node_xyz(const Geom &g, int i, int &x, int &y, int &z)
{
    const int r = div_invariant(i, g.mx, g.lx);
    x = i - r * g.nx;
    z = div_invariant(r, g.my, g.ly);
    y = r - z * g.ny;
}

// Coordinates of node i = x + nx y of a 2D lattice.
__device__ __forceinline__ void node_xy(const Geom &g, int i, int &x, int &y)
{
    y = div_invariant(i, g.mx, g.lx);
    x = i - y * g.nx;
}

}  // namespace lbmk
