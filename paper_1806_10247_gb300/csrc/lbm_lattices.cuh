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

// A node none of whose pull sources leaves the domain: every population comes
// from the fixed offset -(ex + nx ey + nx ny ez), no wrap or wall test needed.
__device__ __forceinline__ bool interior(const Geom &g, int x, int y, int z)
{
    return x > 0 && x < g.nx - 1 && y > 0 && y < g.ny - 1 && (g.nz == 1 || (z > 0 && z < g.nz - 1));
}

template <class L>
__device__ __forceinline__ void load_pulled(const double *__restrict__ fin, const Geom &g, int x, int y,
                                            int z, int i, double (&f)[L::Q])
{
    if (interior(g, x, y, z)) {
        const int sy = g.nx, sz = g.nx * g.ny;
#pragma unroll
        for (int a = 0; a < L::Q; a++)
            f[a] = __ldg(fin + a * g.Np + i - (L::ex(a) + L::ey(a) * sy + L::ez(a) * sz));
        return;
    }
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
    if (interior(g, x, y, z)) {
        const int sy = g.nx, sz = g.nx * g.ny;
#pragma unroll
        for (int a = 0; a < L::Q; a++)
            d[a] = Dev<T>::get(fin + a * g.Np + i - (L::ex(a) + L::ey(a) * sy + L::ez(a) * sz));
        return;
    }
#pragma unroll
    for (int a = 0; a < L::Q; a++) {
        const int ex = L::ex(a), ey = L::ey(a), ez = L::ez(a);
        if (ex == 0 && ey == 0 && ez == 0) {
            d[a] = Dev<T>::get(fin + a * g.Np + i);
        } else {
            bool opp;
            int off = pull_off(g, x, y, z, ex, ey, ez, opp);
            d[a] = Dev<T>::get(fin + (opp ? L::opp(a) : a) * g.Np + off);
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

__device__ __forceinline__ void node_xyz(const Geom &g, int i, int &x, int &y, int &z)
{
    x = i % g.nx;
    int r = i / g.nx;
    y = r % g.ny;
    z = r / g.ny;
}

}  // namespace lbmk
