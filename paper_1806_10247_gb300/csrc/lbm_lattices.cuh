// Velocity sets as compile-time traits, and the per-node helpers that every
// kernel of a lattice shares: pulling the streamed populations of a node and
// the zeroth/first moments.
#pragma once

#include "lbm_device.cuh"

namespace lbmk {

// D2Q9, Sec. 4 Eq. 15: 0 rest, 1 +x, 2 +y, 3 -x, 4 -y, 5 (+,+), 6 (-,+), 7 (-,-), 8 (+,-).
struct LD2Q9 {
    static constexpr int Q = 9, DIM = 2, ID = 1;
    __host__ __device__ static constexpr int ex(int a) { return (a == 1 || a == 5 || a == 8) ? 1 : ((a == 3 || a == 6 || a == 7) ? -1 : 0); }
    __host__ __device__ static constexpr int ey(int a) { return (a == 2 || a == 5 || a == 6) ? 1 : ((a == 4 || a == 7 || a == 8) ? -1 : 0); }
    __host__ __device__ static constexpr int ez(int) { return 0; }
    __host__ __device__ static constexpr int opp(int a) { return a == 0 ? 0 : (a <= 4 ? ((a + 1) % 4) + 1 : ((a - 3) % 4) + 5); }
};

// D2Q5, Sec. 5 Eq. 34: 0 rest, 1 +x, 2 +y, 3 -x, 4 -y.
struct LD2Q5 {
    static constexpr int Q = 5, DIM = 2, ID = 3;
    __host__ __device__ static constexpr int ex(int a) { return a == 1 ? 1 : (a == 3 ? -1 : 0); }
    __host__ __device__ static constexpr int ey(int a) { return a == 2 ? 1 : (a == 4 ? -1 : 0); }
    __host__ __device__ static constexpr int ez(int) { return 0; }
    __host__ __device__ static constexpr int opp(int a) { return a == 0 ? 0 : ((a + 1) % 4) + 1; }
};

// D3Q27 in tensor order: a = (ex+1) + 3 (ey+1) + 9 (ez+1); the opposite of a is 26 - a.
struct LD3Q27 {
    static constexpr int Q = 27, DIM = 3, ID = 2;
    __host__ __device__ static constexpr int ex(int a) { return a % 3 - 1; }
    __host__ __device__ static constexpr int ey(int a) { return (a / 3) % 3 - 1; }
    __host__ __device__ static constexpr int ez(int a) { return a / 9 - 1; }
    __host__ __device__ static constexpr int opp(int a) { return 26 - a; }
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

template <class L>
__device__ __forceinline__ void load_pulled(const double *__restrict__ fin, const Geom &g, int x, int y,
                                            int z, int i, double (&f)[L::Q])
{
#pragma unroll
    for (int a = 0; a < L::Q; a++) {
        const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
        if (ex == 0 && ey == 0 && ez == 0) {
            f[a] = __ldg(fin + a * g.Np + i);
        } else {
            bool opp;
            int off = pull_off(g, x, y, z, ex, ey, ez, opp);
            f[a] = __ldg(fin + (opp ? L::opp(a) : a) * g.Np + off);
        }
    }
}

// Zeroth and first moments of a node's populations.
template <class L>
__device__ __forceinline__ void zeroth_first(const double (&f)[L::Q], double &m0, double (&j)[3])
{
    m0 = 0.0;
    j[0] = j[1] = j[2] = 0.0;
#pragma unroll
    for (int a = 0; a < L::Q; a++) {
        m0 += f[a];
        if (L::ex(a) == 1) j[0] += f[a];
        if (L::ex(a) == -1) j[0] -= f[a];
        if (L::ey(a) == 1) j[1] += f[a];
        if (L::ey(a) == -1) j[1] -= f[a];
        if (L::ez(a) == 1) j[2] += f[a];
        if (L::ez(a) == -1) j[2] -= f[a];
    }
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

__device__ __forceinline__ void node_xyz(const Geom &g, int i, int &x, int &y, int &z)
{
    x = i % g.nx;
    int r = i / g.nx;
    y = r % g.ny;
    z = r / g.ny;
}

}  // namespace lbmk
