// Reduced-precision form of the three lattice steps: populations stored as
// deviations d_a = f_a - w_a rho_ref from the rest state (FP32, FP16 or BF16),
// every moment computed in FP32 from the deviations.  The rest state's own
// moments are folded in analytically, so no O(1) quantities are ever
// subtracted in FP32; only the non-equilibrium signal is carried.  The
// arithmetic is the same method as the FP64 kernels (Eqs. 23/25/31/32 for
// D2Q9, Eqs. 41-48 for D2Q5, the generic central-moment procedure for D3Q27),
// rearranged around the rest state.
#include <cooperative_groups.h>

#include <algorithm>

#include "lbm_internal.h"
#include "lbm_lattices.cuh"
#include "lbm_tiles.cuh"

namespace lbmk {
namespace {

constexpr int kBlock = 256;

// Two nodes' values in one register pair: every operation on them is one
// packed FP32 instruction (add / multiply / fused multiply-add on f32x2, sm_100
// and later), each half rounded exactly as the scalar operation would be.  The
// 16-bit steps at unit higher rates run two x-neighbouring nodes per thread in
// this form (D3Q27: fewer instructions per node; D2Q9 / D2Q5: twice the bytes
// of loads in flight per thread).
struct f2 {
    float2 v;
    __device__ __forceinline__ f2() {}
    __device__ __forceinline__ f2(float s) : v(make_float2(s, s)) {}
    __device__ __forceinline__ f2(float a, float b) : v(make_float2(a, b)) {}
    __device__ __forceinline__ explicit f2(float2 x) : v(x) {}
};
__device__ __forceinline__ f2 operator+(f2 a, f2 b) { return f2(__fadd2_rn(a.v, b.v)); }
__device__ __forceinline__ f2 operator*(f2 a, f2 b) { return f2(__fmul2_rn(a.v, b.v)); }
// a - b as a + b * (-1): exact negation, one rounding, one instruction
__device__ __forceinline__ f2 operator-(f2 a, f2 b) { return f2(__ffma2_rn(b.v, make_float2(-1.f, -1.f), a.v)); }
__device__ __forceinline__ f2 operator-(f2 a) { return f2(__fmul2_rn(a.v, make_float2(-1.f, -1.f))); }
__device__ __forceinline__ f2 vfma(f2 a, f2 b, f2 c) { return f2(__ffma2_rn(a.v, b.v, c.v)); }
__device__ __forceinline__ float vfma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ f2 vrcp(f2 a) { return f2(__frcp_rn(a.v.x), __frcp_rn(a.v.y)); }
__device__ __forceinline__ float vrcp(float a) { return __frcp_rn(a); }

// ------------------------------------------------------ stochastic rounding ---
// Counter-based random bits: the output function of SplitMix64 (Steele, Lea
// and Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014),
// a bijective mix of a 64-bit counter.
__device__ __forceinline__ unsigned long long mix64(unsigned long long z)
{
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// 16-bit random numbers for the populations of node i in a step with key
// `key` (the seed mixed with the step counter on the host): population a
// takes bits 16 (a % 4) .. of mix64 of a counter distinct for every node
// i < 2^31 and chunk a / 4 < 8 of the step.
struct SRBits {
    unsigned long long key;
    int i;
    unsigned long long word;
    int chunk;
    __device__ __forceinline__ SRBits(unsigned long long k, int node) : key(k), i(node), word(0), chunk(-1) {}
    __device__ __forceinline__ unsigned get(int a)
    {
        if ((a >> 2) != chunk) {
            chunk = a >> 2;
            word = mix64(key ^ (((unsigned long long)(unsigned)i << 3) | (unsigned)chunk));
        }
        return (unsigned)(word >> (16 * (a & 3))) & 0xffffu;
    }
};

// Rounding of a deviation to the storage type: to nearest, or (SR)
// stochastically with a 16-bit random r16 -- to the neighbour further from
// zero with probability equal to the distance from the nearer-to-zero
// neighbour in units of the step between the two, so that the stored value is
// the input on average.
template <class T> struct Round;
template <> struct Round<float> {
    __device__ static float sr(float v, unsigned) { return v; }
};
template <> struct Round<__half> {
    __device__ static __half sr(float v, unsigned r16)
    {
        const __half lo = __float2half_rz(v);
        const float flo = __half2float(lo);
        if (flo == v) return lo;
        // one step further from zero (the same sign bit, magnitude + 1)
        const __half hi = __ushort_as_half((unsigned short)(__half_as_ushort(lo) + 1u));
        const float step = __half2float(hi) - flo;  // a power of two: exact, and so is its reciprocal
        const float p = (v - flo) * __frcp_rn(step);
        return (float)r16 * (1.0f / 65536.0f) < p ? hi : lo;
    }
};
template <> struct Round<__nv_bfloat16> {
    __device__ static __nv_bfloat16 sr(float v, unsigned r16)
    {
        // BF16 keeps the upper 16 bits of the FP32 pattern: adding a uniform
        // 16-bit integer to the dropped bits before truncating rounds up
        // with probability (dropped bits) / 2^16
        unsigned b = __float_as_uint(v);
        if ((b & 0x7f800000u) != 0x7f800000u) b += r16;
        return __ushort_as_bfloat16((unsigned short)(b >> 16));
    }
};
template <class T, bool SR>
__device__ __forceinline__ T store_dev(float v, SRBits &rb, int a)
{
    if constexpr (SR) return Round<T>::sr(v, rb.get(a));
    else return Dev<T>::to_store(v);
}

// ------------------------------------------------------------------ D2Q9 ---

struct Rates9f {
    float c3, c4, c5, c6, c7, c8;  // omega_3/12, omega_4/4, ..., omega_8/4
};

//   Fx, Fy : a_pre P (Eq. 25);  Gx, Gy : (F_pre + F_post)/12 (Eq. 31)
__device__ __forceinline__ void collide9(float (&d)[9], float rref, float Fx, float Fy, float Gx, float Gy,
                                         const Rates9f &w)
{
    // Raw moments of the deviations (Eq. 21 minus the rest state's moments:
    // the rest state has rho_ref, zero odd moments, rho_ref/3 per squared
    // direction and rho_ref/9 for xxyy).
    const float s0 = d[1] + d[3], d0 = d[1] - d[3];
    const float s1 = d[5] + d[6], d1 = d[5] - d[6];
    const float s2 = d[8] + d[7], d2 = d[8] - d[7];
    const float A0 = d[0] + s0, B0 = d[2] + s1, C0 = d[4] + s2;
    const float drho = A0 + (B0 + C0), jy = B0 - C0, myy = B0 + C0;
    const float jx = d0 + (d1 + d2), mxy = d1 - d2, mxyy = d1 + d2;
    const float mxx = s0 + (s1 + s2), mxxy = s1 - s2, mxxyy = s1 + s2;
    const float rho = rref + drho;
    const float rinv = __frcp_rn(rho);
    const float ux = fmaf(0.5f, Fx, jx) * rinv;  // Eq. 25
    const float uy = fmaf(0.5f, Fy, jy) * rinv;
    const float ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;
    const float r3 = rref * (1.0f / 3.0f);

    // Eq. 23 with the rest moments substituted.
    const float g3 = w.c3 * ((2.0f / 3.0f) * drho + rho * (ux2 + uy2) - (mxx + myy));
    const float g4 = w.c4 * (rho * (ux2 - uy2) - (mxx - myy));
    const float g5 = w.c5 * (rho * uxy - mxy);
    const float p34 = 3.0f * g3 + g4, m34 = 3.0f * g3 - g4;
    const float g6 = w.c6 * (2.0f * rho * ux2 * uy + mxxy - 2.0f * ux * mxy - uy * (r3 + mxx))
                     - 0.5f * uy * p34 - 2.0f * ux * g5;
    const float g7 = w.c7 * (2.0f * rho * ux * uy2 + mxyy - 2.0f * uy * mxy - ux * (r3 + myy))
                     - 0.5f * ux * m34 - 2.0f * uy * g5;
    const float g8 = w.c8 * ((1.0f / 9.0f) * drho + 3.0f * rho * ux2 * uy2
                             - (mxxyy - 2.0f * ux * mxyy - 2.0f * uy * mxxy + ux2 * (r3 + myy)
                                + uy2 * (r3 + mxx) + 4.0f * uxy * mxy))
                     - 2.0f * g3 - 0.5f * uy2 * p34 - 0.5f * ux2 * m34 - 4.0f * uxy * g5
                     - 2.0f * uy * g6 - 2.0f * ux * g7;

    // Eq. 32 (the rest state cancels: d^p = d + K g).
    const float ax = g4 - g3, ay = -g3 - g4, c = 2.0f * g3 + g8;
    d[0] += -4.0f * (g3 - g8);
    d[1] += Gx + ax + 2.0f * (g7 - g8);
    d[2] += Gy + ay + 2.0f * (g6 - g8);
    d[3] += -Gx + ax - 2.0f * (g7 + g8);
    d[4] += -Gy + ay - 2.0f * (g6 + g8);
    d[5] += c + (Gx + Gy) + (g5 - g6 - g7);
    d[6] += c + (Gy - Gx) + (-g5 - g6 + g7);
    d[7] += c - (Gx + Gy) + (g5 + g6 + g7);
    d[8] += c + (Gx - Gy) + (-g5 + g6 - g7);
}

// The same step when omega_6 = omega_7 = omega_8 = 1, as the FP64 kernel's
// collide_w1: the post-collision deviations follow from drho, u and the three
// relaxed second-order central moments, through the halved back-shift and
// inverse transform.  The transform is linear and maps the rest state's
// central moments about u, rho_ref prod(1, -u, 1/3 + u^2), to w rho_ref, so
// it is applied to the DEVIATIONS of the post-collision central moments from
// those: first order rho_ref u (the total is 0), second order the relaxed
// moments minus rho_ref (1/3 + u^2) (resp. rho_ref u_x u_y), third order
// rho_ref (1/3 + u_x^2) u_y (the total is 0), fourth order
// drho / 9 - rho_ref (u_x^2 / 3 + u_y^2 / 3 + u_x^2 u_y^2).  No O(1)
// quantity is subtracted.  The first raw moments come back as j itself, not
// as rho (j / rho): in FP32 that round trip would change the momentum by the
// same rounding every step of a steady flow, and the error would add up.
template <class V>
__device__ __forceinline__ void collide9_w1(V (&d)[9], float rref, V Fx, V Fy, V Gx, V Gy, const Rates9f &w)
{
    const V s0 = d[1] + d[3], d0 = d[1] - d[3];
    const V s1 = d[5] + d[6], d1 = d[5] - d[6];
    const V s2 = d[8] + d[7], d2 = d[8] - d[7];
    const V B0 = d[2] + s1, C0 = d[4] + s2;
    const V drho = (d[0] + s0) + (B0 + C0);
    const V jx = vfma(V(0.5f), Fx, d0 + (d1 + d2)), jy = vfma(V(0.5f), Fy, B0 - C0);  // Eq. 25
    const V mxx = s0 + (s1 + s2), myy = B0 + C0, mxy = d1 - d2;  // deviations: m_xx - rho_ref / 3 etc.
    const V rho = V(rref) + drho;
    const V rinv = vrcp(rho);
    const V ux = jx * rinv, uy = jy * rinv;
    const V ux2 = ux * ux, uy2 = uy * uy;

    // second-order central moments minus rho_ref / 3 (xx, yy), relaxed; then
    // their deviations from the rest state's, halved
    const V cxx = vfma(-jx, ux, mxx), cyy = vfma(-jy, uy, myy), cxy = vfma(-jx, uy, mxy);
    const V T = cxx + cyy, D = cxx - cyy;
    const V Tq = vfma(V(3.0f * w.c3), vfma(V(2.0f / 3.0f), drho, -T), V(0.25f) * T);
    const V Dq = V(0.25f - w.c4) * D;
    const float rh = 0.5f * rref, rq = 0.25f * rref;
    const V kxx = vfma(V(-rh), ux2, Tq + Dq), kyy = vfma(V(-rh), uy2, Tq - Dq);
    const V kxy = vfma(V(-rq), ux * uy, V(0.25f - w.c5) * cxy);
    // halved first central moments of the deviations, j - u drho (= rho_ref u)
    const V k10 = V(0.5f) * vfma(-ux, drho, jx), k01 = V(0.5f) * vfma(-uy, drho, jy);
    const V k21 = V(rq) * vfma(ux, ux, V(1.0f / 3.0f)) * uy, k12 = V(rq) * ux * vfma(uy, uy, V(1.0f / 3.0f));
    const V k22 = vfma(V(1.0f / 36.0f), drho, V(-rq) * (vfma(ux2 + uy2, V(1.0f / 3.0f), ux2 * uy2)));

    // back-shift along x of the lines of y-order 0, 1, 2, then along y
    const V hx = V(0.5f) * ux, hy = V(0.5f) * uy;
    const V M10 = V(0.5f) * jx, M20 = vfma(ux, k10 + M10, kxx);  // m_10 = j_x exactly
    const V M01 = k01, M11 = vfma(hx, k01, kxy), M21 = vfma(ux, kxy + M11, k21);
    const V M02 = kyy, M12 = vfma(hx, kyy, k12), M22 = vfma(ux, k12 + M12, k22);
    const V N00 = drho, N01 = V(0.5f) * jy, N02 = vfma(uy, M01 + N01, M02);  // m_01 = j_y exactly
    V N10 = M10, N11 = vfma(hy, M10, M11), N12 = vfma(uy, M11 + N11, M12);
    const V N20 = M20;
    V N21 = vfma(hy, M20, M21);
    const V N22 = vfma(uy, M21 + N21, M22);
    const V N01f = vfma(V(3.0f), Gy, vfma(V(-0.25f), Fy, N01));  // post-collision force (Eq. 31), halved
    N10 = vfma(V(3.0f), Gx, vfma(V(-0.25f), Fx, N10));
    N12 = N12 + Gx;
    N21 = N21 + Gy;
    const V P0m = N02 - N01f, P00 = vfma(V(-2.0f), N02, N00), P0p = N02 + N01f;
    const V P1m = N12 - N11, P10 = vfma(V(-2.0f), N12, N10), P1p = N12 + N11;
    const V P2m = N22 - N21, P20 = vfma(V(-2.0f), N22, N20), P2p = N22 + N21;
    d[0] = vfma(V(-2.0f), P20, P00);
    d[1] = P20 + P10;
    d[3] = P20 - P10;
    d[2] = vfma(V(-2.0f), P2p, P0p);
    d[5] = P2p + P1p;
    d[6] = P2p - P1p;
    d[4] = vfma(V(-2.0f), P2m, P0m);
    d[8] = P2m + P1m;
    d[7] = P2m - P1m;
}

template <class T, int FK, bool W1, bool SR = false>
__global__ void __launch_bounds__(kBlock)
k_step9(const __grid_constant__ Planes<T, 9> P, Geom g, FieldDev F, float apre, float gsum, Rates9f w, float rref,
        unsigned long long srkey)
{
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    int x, y;
    node_xy(g, i, x, y);
    float d[9];
    load_pulled_dev<LD2Q9, T>(P, g, x, y, 0, i, d);
    float Fx = 0.f, Fy = 0.f, Gx = 0.f, Gy = 0.f;
    if (FK != FK_NONE) {
        const float Px = field_value_f(F, FK, 0, x, y, 0, i), Py = field_value_f(F, FK, 1, x, y, 0, i);
        Fx = apre * Px;
        Fy = apre * Py;
        Gx = gsum * Px;
        Gy = gsum * Py;
    }
    if (W1) collide9_w1(d, rref, Fx, Fy, Gx, Gy, w);
    else collide9(d, rref, Fx, Fy, Gx, Gy, w);
    SRBits rb(srkey, i);
#pragma unroll
    for (int a = 0; a < 9; a++) P.out[a][i] = store_dev<T, SR>(d[a], rb, a);
}

// Many steps per launch for a small D2Q9 lattice (the FP32 / 16-bit form of
// the FP64 cluster kernel): the stored deviations of block b's nodes live in
// its shared memory (as the storage type, so every step rounds exactly as a
// single-step launch does); pulls from other blocks read their shared memory
// through the cluster; one cluster barrier per step.
namespace cg = cooperative_groups;
constexpr int kClusterThreads = 384;

template <class T, int FK, bool W1>
__global__ void __launch_bounds__(kClusterThreads)
k_cluster9(const T *__restrict__ fin, T *__restrict__ fout, Geom g, FieldDev F, float apre, float gsum, Rates9f w,
           float rref, int P, int nsteps)
{
    extern __shared__ __align__(16) unsigned char smraw[];
    T *sm = reinterpret_cast<T *>(smraw);  // [2][9][P]
    cg::cluster_group cl = cg::this_cluster();
    const int b = (int)cl.block_rank();
    const int l = threadIdx.x;
    const int i = b * P + l;
    const bool own = l < P && i < g.N;
    if (own)
#pragma unroll
        for (int a = 0; a < 9; a++) sm[a * P + l] = fin[a * g.Np + i];
    const int x = own ? i % g.nx : 0, y = own ? i / g.nx : 0;
    float Fx = 0.f, Fy = 0.f, Gx = 0.f, Gy = 0.f;
    if (FK != FK_NONE && own) {
        const float Px = field_value_f(F, FK, 0, x, y, 0, i), Py = field_value_f(F, FK, 1, x, y, 0, i);
        Fx = apre * Px;
        Fy = apre * Py;
        Gx = gsum * Px;
        Gy = gsum * Py;
    }
    int src_blk[9], src_off[9];
    if (own) {
#pragma unroll
        for (int a = 0; a < 9; a++) {
            bool opp = false;
            const int j = pull_off(g, x, y, 0, LD2Q9::ex(a), LD2Q9::ey(a), 0, opp);
            const int aa = opp ? LD2Q9::opp(a) : a;
            src_blk[a] = j / P;
            src_off[a] = aa * P + (j - (j / P) * P);
        }
    }
    cl.sync();
    int cur = 0;
    for (int k = 0; k < nsteps; k++) {
        if (own) {
            float d[9];
#pragma unroll
            for (int a = 0; a < 9; a++) {
                const T *base = cl.map_shared_rank(sm + cur * 9 * P, src_blk[a]);
                d[a] = (float)base[src_off[a]];
            }
            if (W1) collide9_w1(d, rref, Fx, Fy, Gx, Gy, w);
            else collide9(d, rref, Fx, Fy, Gx, Gy, w);
            T *nxt = sm + (cur ^ 1) * 9 * P;
#pragma unroll
            for (int a = 0; a < 9; a++) nxt[a * P + l] = Dev<T>::to_store(d[a]);
        }
        cur ^= 1;
        cl.sync();
    }
    if (own)
#pragma unroll
        for (int a = 0; a < 9; a++) fout[a * g.Np + i] = sm[cur * 9 * P + a * P + l];
}

template <class T, bool W1>
cudaError_t cluster9_launch(cudaLaunchConfig_t &cfg, int C, const LaunchArgs &a, const T *fin, T *fout, float apre,
                            float gsum, const Rates9f &w, float rref, int P, int nsteps)
{
    switch (a.fkind) {
    case FK_NONE:
        if (C > 8) cudaFuncSetAttribute(k_cluster9<T, FK_NONE, W1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        return cudaLaunchKernelEx(&cfg, k_cluster9<T, FK_NONE, W1>, fin, fout, a.g, a.F, apre, gsum, w, rref, P,
                                  nsteps);
    case FK_CONST:
        if (C > 8) cudaFuncSetAttribute(k_cluster9<T, FK_CONST, W1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        return cudaLaunchKernelEx(&cfg, k_cluster9<T, FK_CONST, W1>, fin, fout, a.g, a.F, apre, gsum, w, rref, P,
                                  nsteps);
    default:
        if (C > 8)
            cudaFuncSetAttribute(k_cluster9<T, FK_GENERAL, W1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        return cudaLaunchKernelEx(&cfg, k_cluster9<T, FK_GENERAL, W1>, fin, fout, a.g, a.F, apre, gsum, w, rref, P,
                                  nsteps);
    }
}

template <class T>
cudaError_t cluster9_t(const LaunchArgs &a, int nsteps)
{
    const int C = a.g.N >= 16 * 8 ? 16 : (a.g.N + 7) / 8;
    const int P = (a.g.N + C - 1) / C;
    const int threads = (P + 31) / 32 * 32;
    const size_t smem = (size_t)2 * 9 * P * sizeof(T);
    if (threads > kClusterThreads || smem > 48 * 1024) return cudaErrorNotSupported;
    const Rates9f w{(float)(a.omega[3] / 12.0), (float)(a.omega[4] / 4.0), (float)(a.omega[5] / 4.0),
                    (float)(a.omega[6] / 4.0), (float)(a.omega[7] / 4.0), (float)(a.omega[8] / 4.0)};
    const float gsum = (float)((a.apre + a.apost) / 12.0), apre = (float)a.apre, rref = (float)a.rho_ref;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(C);
    cfg.blockDim = dim3(threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = a.stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const T *fin = reinterpret_cast<const T *>(a.fin);
    T *fout = reinterpret_cast<T *>(a.fout);
    return (a.omega[6] == 1.0 && a.omega[7] == 1.0 && a.omega[8] == 1.0)
               ? cluster9_launch<T, true>(cfg, C, a, fin, fout, apre, gsum, w, rref, P, nsteps)
               : cluster9_launch<T, false>(cfg, C, a, fin, fout, apre, gsum, w, rref, P, nsteps);
}

// ------------------------------------------------------------------ D2Q5 ---

struct Rates5f {
    float c1, c2, c3, c4;  // omega_1/2 .. omega_4/4
};

// General advecting velocity.  S: a_pre S(x); H0: (S_pre + S_post)/10.
__device__ __forceinline__ void collide5(float (&d)[5], float rref, float S, float H0, float ux, float uy,
                                         const Rates5f &w)
{
    const float kx = d[1] - d[3], ky = d[2] - d[4];
    const float mxx = d[1] + d[3], myy = d[2] + d[4];  // minus the rest values rref/3
    const float dphi = fmaf(0.5f, S, d[0] + (mxx + myy));  // Eqs. 42-43, minus rref
    const float phi = rref + dphi;
    const float h1 = w.c1 * (phi * ux - kx);
    const float h2 = w.c2 * (phi * uy - ky);
    const float h3 = w.c3 * ((2.0f / 3.0f) * dphi - (mxx + myy) + 2.0f * (ux * kx + uy * ky)
                             - (ux * ux + uy * uy) * phi)
                     + ux * h1 + uy * h2;
    const float h4 = w.c4 * (-(mxx - myy) + 2.0f * (ux * kx - uy * ky) - (ux * ux - uy * uy) * phi)
                     + ux * h1 - uy * h2;
    const float c = H0 + h3;  // Eq. 48
    d[0] += H0 - 4.0f * h3;
    d[1] += c + h1 + h4;
    d[2] += c + h2 - h4;
    d[3] += c - h1 + h4;
    d[4] += c - h2 - h4;
}

// Uniform advecting velocity: launch-constant coefficients (see the FP64
// kernel) with the rest-state terms split off: h3 = Q3 rref + P3 dphi + ...,
// h4 = P4 rref + P4 dphi + ..., h1 = A1 rref + A1 dphi - c1 kx.
struct Coef5f {
    float A1, c1, A2, c2, P3, X3, Y3, S3, P4, X4, Y4, D4, Q3;
};

template <class V>
__device__ __forceinline__ void collide5u(V (&d)[5], float rref, V S, V H0, const Coef5f &k)
{
    const V kx = d[1] - d[3], ky = d[2] - d[4];
    const V mxx = d[1] + d[3], myy = d[2] + d[4];
    const V Sg = mxx + myy, Dg = mxx - myy;
    const V dphi = vfma(V(0.5f), S, d[0] + Sg);
    const V phi = V(rref) + dphi;
    const V h1 = vfma(V(k.A1), phi, V(-k.c1) * kx);
    const V h2 = vfma(V(k.A2), phi, V(-k.c2) * ky);
    const V h3 = vfma(V(k.Q3), V(rref), vfma(V(k.P3), dphi, vfma(V(k.X3), kx, vfma(V(k.Y3), ky, V(k.S3) * Sg))));
    const V h4 = vfma(V(k.P4), phi, vfma(V(k.X4), kx, vfma(V(k.Y4), ky, V(k.D4) * Dg)));
    const V c = H0 + h3;
    const V e1 = c + h4, e2 = c - h4;
    d[0] = d[0] + vfma(V(-4.0f), h3, H0);
    d[1] = d[1] + (e1 + h1);
    d[2] = d[2] + (e2 + h2);
    d[3] = d[3] + (e1 - h1);
    d[4] = d[4] + (e2 - h2);
}

// Coefficients of a uniform velocity (double on the host, then float).
Coef5f make_coef5f(const double omega[9], double ux, double uy)
{
    const double c1 = omega[1] / 2.0, c2 = omega[2] / 2.0, c3 = omega[3] / 4.0, c4 = omega[4] / 4.0;
    const double ux2 = ux * ux, uy2 = uy * uy;
    Coef5f k;
    k.A1 = (float)(c1 * ux);
    k.c1 = (float)c1;
    k.A2 = (float)(c2 * uy);
    k.c2 = (float)c2;
    const double P3 = c3 * ((2.0 / 3.0) - ux2 - uy2) + c1 * ux2 + c2 * uy2;
    k.P3 = (float)P3;
    k.X3 = (float)(ux * (2.0 * c3 - c1));
    k.Y3 = (float)(uy * (2.0 * c3 - c2));
    k.S3 = (float)(-c3);
    k.Q3 = (float)(-c3 * (ux2 + uy2) + c1 * ux2 + c2 * uy2);  // P3 - (2/3) c3: small, O(u^2)
    k.P4 = (float)(-c4 * (ux2 - uy2) + c1 * ux2 - c2 * uy2);
    k.X4 = (float)(ux * (2.0 * c4 - c1));
    k.Y4 = (float)(uy * (c2 - 2.0 * c4));
    k.D4 = (float)(-c4);
    return k;
}

// Deviations from the reference; a uniform velocity takes the linear step of
// the deviations (collide5u with no rest-state terms) plus the constant cref =
// M g_ref - g_ref (zero for the equilibrium reference of a periodic lattice).
struct Ref5f {
    float v[5];
};

template <class T, int SK, bool UNIFORM, bool SR = false>
__global__ void __launch_bounds__(kBlock)
k_step5(const __grid_constant__ Planes<T, 5> P, Geom g, FieldDev S, FieldDev V, float apre, float hsum, Rates5f w,
        Coef5f k, float rref, Ref5f cref, unsigned long long srkey)
{
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    int x, y;
    node_xy(g, i, x, y);
    float d[5];
    load_pulled_dev<LD2Q5, T>(P, g, x, y, 0, i, d);
    float Sp = 0.f, H0 = 0.f;
    if (SK != FK_NONE) {
        const float Ps = field_value_f(S, SK, 0, x, y, 0, i);
        Sp = apre * Ps;
        H0 = hsum * Ps;
    }
    if (UNIFORM) {
        collide5u(d, 0.0f, Sp, H0, k);
#pragma unroll
        for (int a = 0; a < 5; a++) d[a] += cref.v[a];
    } else {
        const float ux = field_value_f(V, FK_GENERAL, 0, x, y, 0, i);
        const float uy = field_value_f(V, FK_GENERAL, 1, x, y, 0, i);
        collide5(d, rref, Sp, H0, ux, uy, w);
    }
    SRBits rb(srkey, i);
#pragma unroll
    for (int a = 0; a < 5; a++) P.out[a][i] = store_dev<T, SR>(d[a], rb, a);
}

// ----------------------------------------------------------------- D3Q27 ---

struct Rates27f {
    float wb, ws, w3, w4, w5, w6;
};

template <class V>
__device__ __forceinline__ void raw_fwd(V &a, V &b, V &c)
{
    const V s = c + a, dd = c - a;
    a = s + b;
    b = dd;
    c = s;
}
// The way back runs on HALVED moments (each axis on which a moment has order 1
// or 2 contributes a factor 1/2), as in the FP64 kernel: the inverse 1D
// transform of (m0, m1/2, m2/2) is f_-1 = m2/2 - m1/2, f_0 = m0 - m2,
// f_+1 = m2/2 + m1/2, three operations per line instead of four.
template <class V>
__device__ __forceinline__ void raw_bwd_h(V &m0, V &m1, V &m2)
{
    const V fm = m2 - m1, fp = m2 + m1, f0 = vfma(V(-2.0f), m2, m0);
    m0 = fm;
    m1 = f0;
    m2 = fp;
}
__device__ __forceinline__ void shift_fwd(float m0, float &m1, float &m2, float u)
{
    const float k1 = fmaf(-u, m0, m1);
    m2 = fmaf(-u, m1 + k1, m2);
    m1 = k1;
}
// Halved central moments about u -> halved raw moments (one axis; uh = u / 2).
template <class V>
__device__ __forceinline__ void shift_bwd_h(V k0, V &k1, V &k2, V u, V uh)
{
    const V m1 = vfma(uh, k0, k1);
    k2 = vfma(u, k1 + m1, k2);
    k1 = m1;
}
template <int AX, class V, class Op>
__device__ __forceinline__ void along(V (&m)[27], Op op)
{
    constexpr int st = AX == 0 ? 1 : (AX == 1 ? 3 : 9);
#pragma unroll
    for (int t = 0; t < 9; t++) {
        const int p = AX == 0 ? 3 * t : (AX == 1 ? (t % 3) + 9 * (t / 3) : t);
        op(m[p], m[p + st], m[p + 2 * st]);
    }
}

// Halved post-collision central moments of the deviations about u ->
// deviations: back-shift, post-collision force in moment space (K_1 g_1 with
// g = (F_pre + F_post) / 36; m_100 already carries F_pre / 2), inverse raw
// transform.
// XO: the force has no y and z components (their terms, additions of 0, are left out).
template <class V, bool XO = false>
__device__ __forceinline__ void finish27(V (&m)[27], V ux, V uy, V uz, const V (&F)[3], const V (&Fq)[3])
{
    const V hx = V(0.5f) * ux, hy = V(0.5f) * uy, hz = V(0.5f) * uz;
    along<0>(m, [ux, hx](V &a, V &b, V &c) { shift_bwd_h(a, b, c, ux, hx); });
    along<1>(m, [uy, hy](V &a, V &b, V &c) { shift_bwd_h(a, b, c, uy, hy); });
    along<2>(m, [uz, hz](V &a, V &b, V &c) { shift_bwd_h(a, b, c, uz, hz); });

    {
        const V c4 = V(0.25f), c12 = V(1.0f / 12.0f), c36 = V(1.0f / 36.0f);
        const V sx = F[0] + Fq[0];
        m[1] = vfma(c4, Fq[0], m[1]);
        m[7] = vfma(sx, c12, m[7]); m[19] = vfma(sx, c12, m[19]); m[25] = vfma(sx, c36, m[25]);
        if constexpr (!XO) {
            const V sy = F[1] + Fq[1], sz = F[2] + Fq[2];
            m[3] = vfma(c4, Fq[1], m[3]);
            m[9] = vfma(c4, Fq[2], m[9]);
            m[5] = vfma(sy, c12, m[5]); m[21] = vfma(sy, c12, m[21]); m[23] = vfma(sy, c36, m[23]);
            m[11] = vfma(sz, c12, m[11]); m[15] = vfma(sz, c12, m[15]); m[17] = vfma(sz, c36, m[17]);
        }
    }

    along<2>(m, [](V &a, V &b, V &c) { raw_bwd_h(a, b, c); });
    along<1>(m, [](V &a, V &b, V &c) { raw_bwd_h(a, b, c); });
    along<0>(m, [](V &a, V &b, V &c) { raw_bwd_h(a, b, c); });
}

// Halving factor of moment k = a + 3b + 9c: 2^-(number of nonzero a, b, c).
__host__ __device__ constexpr float halving(int k)
{
    return ((k % 3) ? 0.5f : 1.0f) * (((k / 3) % 3) ? 0.5f : 1.0f) * ((k / 9) ? 0.5f : 1.0f);
}

// Deviation target of the central moment k = a + 3b + 9c of order n >= 3: its
// Maxwellian value minus the rest state's central moment about u, times the
// factor h that dr = h drho and rr = h rref carry (h = halving(k)).
template <class V>
__device__ __forceinline__ V high_target(int k, V dr, V nrr, V ux, V uy, V uz)
{
    // nrr = -rr: the rest state's part enters with a minus sign
    const V ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    const int a = k % 3, b = (k / 3) % 3, c = k / 9;
    const int n = a + b + c;
    const V third = V(1.0f / 3.0f);
    const V hx[3] = {V(1.0f), -ux, third + ux2};
    const V hy[3] = {V(1.0f), -uy, third + uy2};
    const V hz[3] = {V(1.0f), -uz, third + uz2};
    if (a == 1 || b == 1 || c == 1) {  // equilibrium 0: -rr hx hy hz (factors 1 left out)
        V p = V(1.0f);
        bool have = false;
        if (a) { p = hx[a]; have = true; }
        if (b) { p = have ? p * hy[b] : hy[b]; have = true; }
        if (c) { p = have ? p * hz[c] : hz[c]; }
        return nrr * p;
    }
    if (n == 4) {
        const V p = (a == 2 && b == 2) ? ux2 + uy2 : ((a == 2) ? ux2 + uz2 : uy2 + uz2);
        const V q = (a == 2 && b == 2) ? ux2 * uy2 : ((a == 2) ? ux2 * uz2 : uy2 * uz2);
        return vfma(nrr, vfma(p, third, q), dr * V(1.0f / 9.0f));
    }
    return vfma(nrr,
                vfma(ux2 + uy2 + uz2, V(1.0f / 9.0f), (ux2 * uy2 + ux2 * uz2 + uy2 * uz2) * third) + ux2 * uy2 * uz2,
                dr * V(1.0f / 27.0f));
}

// Deviation form of the generic central-moment collision: m holds the raw
// moments of the deviations (index a + 3b + 9c); the rest state's central
// moments about u, rref * prod(1, -u, 1/3 + u^2), are folded in analytically.
__device__ __forceinline__ void collide27(float (&m)[27], float rref, const float (&F)[3], const float (&Fq)[3],
                                          const Rates27f &w)
{
    along<0>(m, [](float &a, float &b, float &c) { raw_fwd(a, b, c); });
    along<1>(m, [](float &a, float &b, float &c) { raw_fwd(a, b, c); });
    along<2>(m, [](float &a, float &b, float &c) { raw_fwd(a, b, c); });

    m[1] = fmaf(0.5f, F[0], m[1]);  // pre-collision half force (rest state has no momentum)
    m[3] = fmaf(0.5f, F[1], m[3]);
    m[9] = fmaf(0.5f, F[2], m[9]);
    const float drho = m[0];
    const float rho = rref + drho;
    const float rinv = __frcp_rn(rho);
    const float ux = m[1] * rinv, uy = m[3] * rinv, uz = m[9] * rinv;

    along<0>(m, [ux](float &a, float &b, float &c) { shift_fwd(a, b, c, ux); });
    along<1>(m, [uy](float &a, float &b, float &c) { shift_fwd(a, b, c, uy); });
    along<2>(m, [uz](float &a, float &b, float &c) { shift_fwd(a, b, c, uz); });

    const float ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;
    {
        // second order: trace towards rho, deviatoric and off-diagonal towards
        // 0; results halved
        const float Tn = m[2] + m[6] + m[18];
        const float Ts = fmaf(w.wb, drho - rref * (ux2 + uy2 + uz2) - Tn, Tn);
        const float D1 = m[2] - m[6], D2 = m[2] - m[18];
        const float rs = 1.0f - w.ws;
        const float rh = 0.5f * rs, rq = 0.25f * rs, wh = 0.5f * w.ws * rref, wq = 0.25f * w.ws * rref;
        const float D1h = rh * D1 - wh * (ux2 - uy2);
        const float D2h = rh * D2 - wh * (ux2 - uz2);
        const float kxx = fmaf(Ts, 1.0f / 6.0f, (D1h + D2h) * (1.0f / 3.0f));
        m[2] = kxx;
        m[6] = kxx - D1h;
        m[18] = kxx - D2h;
        m[4] = rq * m[4] - wq * (ux * uy);
        m[10] = rq * m[10] - wq * (ux * uz);
        m[12] = rq * m[12] - wq * (uy * uz);
        m[1] *= 0.5f;
        m[3] *= 0.5f;
        m[9] *= 0.5f;
        // orders 3..6 towards the Maxwellian central moments:
        // h (m + om (t - m)) = h (1 - om) m + om (h t)
        const float d4 = 0.25f * drho, r4 = -0.25f * rref, d8 = 0.125f * drho, r8 = -0.125f * rref;
#pragma unroll
        for (int k = 0; k < 27; k++) {
            const int n = k % 3 + (k / 3) % 3 + k / 9;
            if (n < 3) continue;
            const float om = n == 3 ? w.w3 : (n == 4 ? w.w4 : (n == 5 ? w.w5 : w.w6));
            const bool quarter = halving(k) == 0.25f;
            const float t = high_target(k, quarter ? d4 : d8, quarter ? r4 : r8, ux, uy, uz);
            m[k] = fmaf(halving(k) * (1.0f - om), m[k], om * t);
        }
    }

    finish27(m, ux, uy, uz, F, Fq);
}

// The same collision when omega_3 = omega_4 = omega_5 = omega_6 = 1: the
// central moments of orders 3..6 land on their targets, so only the raw
// moments of order <= 2 are formed and the forward shift reduces to the
// first- and second-order central moments.  V = float (one node) or f2 (two
// nodes, packed); rref is the launch's reference density.
template <class V, bool XO = false>
__device__ __forceinline__ void collide27_w1(V (&m)[27], float rref, const V (&F)[3], const V (&Fq)[3],
                                             const Rates27f &w)
{
    along<0>(m, [](V &a, V &b, V &c) { raw_fwd(a, b, c); });
    // Line (b, c) along x holds M0, M1, M2 at m[3b + 9c + 0..2]; e_y = b - 1, e_z = c - 1.
    V Y0[3], Y1[3], Y2[3], X0[3], X1[3];
#pragma unroll
    for (int c = 0; c < 3; c++) {
        const V s = m[9 * c + 6] + m[9 * c], d = m[9 * c + 6] - m[9 * c];
        Y0[c] = s + m[9 * c + 3];
        Y1[c] = d;
        Y2[c] = s;
        X0[c] = (m[9 * c + 7] + m[9 * c + 1]) + m[9 * c + 4];
        X1[c] = m[9 * c + 7] - m[9 * c + 1];
    }
    const V half = V(0.5f);
    const V drho = (Y0[2] + Y0[0]) + Y0[1];
    const V jz = XO ? Y0[2] - Y0[0] : vfma(half, F[2], Y0[2] - Y0[0]);
    const V kzz = Y0[2] + Y0[0];
    const V jy = XO ? (Y1[2] + Y1[0]) + Y1[1] : vfma(half, F[1], (Y1[2] + Y1[0]) + Y1[1]);
    const V kyz = Y1[2] - Y1[0];
    const V kyy = (Y2[2] + Y2[0]) + Y2[1];
    const V jx = vfma(half, F[0], (X0[2] + X0[0]) + X0[1]);
    const V kxz = X0[2] - X0[0];
    const V kxy = (X1[2] + X1[0]) + X1[1];
    const V kxx = ((m[2] + m[5]) + (m[8] + m[11])) + ((m[14] + m[17]) + (m[20] + m[23])) + m[26];

    const V rho = V(rref) + drho;
    const V rinv = vrcp(rho);
    const V ux = jx * rinv, uy = jy * rinv, uz = jz * rinv;
    const V nux = -ux, nuy = -uy, nuz = -uz;
    const V ux2 = ux * ux, uy2 = uy * uy, uz2 = uz * uz;

    // first-order central moments of the deviations (k1 = m1 - u m0)
    const V k100 = vfma(nux, drho, jx), k010 = vfma(nuy, drho, jy), k001 = vfma(nuz, drho, jz);
    // second-order central moments (k2 = m2 - u (m1 + k1); mixed: k_ab = m_ab - u_a m_b - u_b k_a)
    const V cxx = vfma(nux, jx + k100, kxx), cyy = vfma(nuy, jy + k010, kyy), czz = vfma(nuz, jz + k001, kzz);
    const V cxy = vfma(nuy, k100, vfma(nux, jy, kxy));
    const V cxz = vfma(nuz, k100, vfma(nux, jz, kxz));
    const V cyz = vfma(nuz, k010, vfma(nuy, jz, kyz));

    // relaxed central moments, halved; the rest state's second central
    // moments about u are rref (1/3 + u_a^2) and rref u_a u_b
    const V Tn = cxx + cyy + czz;
    const V Ts = vfma(V(w.wb), vfma(V(-rref), ux2 + uy2 + uz2, drho) - Tn, Tn);
    const V D1 = cxx - cyy, D2 = cxx - czz;
    const float rs = 1.0f - w.ws;
    const V rh = V(0.5f * rs), rq = V(0.25f * rs), nwh = V(-0.5f * w.ws * rref), nwq = V(-0.25f * w.ws * rref);
    const V D1h = vfma(nwh, ux2 - uy2, rh * D1);
    const V D2h = vfma(nwh, ux2 - uz2, rh * D2);
    const V sxx = vfma(Ts, V(1.0f / 6.0f), (D1h + D2h) * V(1.0f / 3.0f));
    const V d4 = V(0.25f) * drho, nr4 = V(-0.25f * rref), d8 = V(0.125f) * drho, nr8 = V(-0.125f * rref);
#pragma unroll
    for (int k = 0; k < 27; k++) {
        const int n = k % 3 + (k / 3) % 3 + k / 9;
        const bool quarter = halving(k) == 0.25f;
        if (n >= 3) m[k] = high_target(k, quarter ? d4 : d8, quarter ? nr4 : nr8, ux, uy, uz);
    }
    m[0] = drho;
    m[1] = half * k100;
    m[3] = half * k010;
    m[9] = half * k001;
    m[2] = sxx;
    m[6] = sxx - D1h;
    m[18] = sxx - D2h;
    m[4] = vfma(nwq, ux * uy, rq * cxy);
    m[10] = vfma(nwq, ux * uz, rq * cxz);
    m[12] = vfma(nwq, uy * uz, rq * cyz);
    finish27<V, XO>(m, ux, uy, uz, F, Fq);
}

// 4 resident blocks per SM (<= 64 registers): the reduced-precision D3Q27
// step is memory-bound, so occupancy to cover load latency matters more than
// registers.
template <class T, int FK, bool W1, bool SR = false>
__global__ void __launch_bounds__(kBlock, 4)
k_step27(const __grid_constant__ Planes<T, 27> P, Geom g, FieldDev Fd, float apre, float apost, Rates27f w,
         float rref, unsigned long long srkey)
{
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    float m[27];
    load_pulled_dev<LD3Q27, T>(P, g, x, y, z, i, m);
    float F[3] = {0.f, 0.f, 0.f}, Fq[3] = {0.f, 0.f, 0.f};
    if (FK != FK_NONE) {
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const float Pd = field_value_f(Fd, FK, d, x, y, z, i);
            F[d] = apre * Pd;
            Fq[d] = apost * Pd;
        }
    }
    if (W1) collide27_w1(m, rref, F, Fq, w);
    else collide27(m, rref, F, Fq, w);
    SRBits rb(srkey, i);
#pragma unroll
    for (int a = 0; a < 27; a++) P.out[a][i] = store_dev<T, SR>(m[a], rb, a);
}

// 16-bit storage, unit higher rates: two x-neighbouring nodes (x even, x + 1)
// per thread, every moment operation one packed f32x2 instruction for both.
// The 16-bit step moves half the bytes of the FP32 one but issues as many
// instructions per node, so one node per thread is bound by instruction
// issue; the pair halves the arithmetic instructions, shares each plane's
// address between the two nodes, loads the populations with e_x = 0 of both
// nodes as one 32-bit word and stores every plane's two values as one 32-bit
// word.  Needs nx even (the pair never straddles a row); the launcher checks.
template <class T> struct Pair16;
template <> struct Pair16<__half> {
    // two stored values (low half: the lower address) as an FP32 pair, and back
    __device__ static f2 from_bits(unsigned u)
    {
        __half2 h;
        memcpy(&h, &u, sizeof h);
        return f2(__half22float2(h));
    }
    __device__ static unsigned to_bits(const f2 &v)
    {
        const __half2 h = __float22half2_rn(v.v);
        unsigned u;
        memcpy(&u, &h, sizeof u);
        return u;
    }
    __device__ static unsigned raw_bits(__half a, __half b)
    {
        return (unsigned)__half_as_ushort(a) | ((unsigned)__half_as_ushort(b) << 16);
    }
    __device__ static f2 get2(const __half *p) { return from_bits(__ldg(reinterpret_cast<const unsigned *>(p))); }
    __device__ static void put2(__half *p, const f2 &v) { *reinterpret_cast<unsigned *>(p) = to_bits(v); }
    __device__ static void put2raw(__half *p, __half a, __half b) { *reinterpret_cast<unsigned *>(p) = raw_bits(a, b); }
};
template <> struct Pair16<__nv_bfloat16> {
    __device__ static f2 from_bits(unsigned u)
    {
        __nv_bfloat162 h;
        memcpy(&h, &u, sizeof h);
        return f2(__bfloat1622float2(h));
    }
    __device__ static unsigned to_bits(const f2 &v)
    {
        const __nv_bfloat162 h = __float22bfloat162_rn(v.v);
        unsigned u;
        memcpy(&u, &h, sizeof u);
        return u;
    }
    __device__ static unsigned raw_bits(__nv_bfloat16 a, __nv_bfloat16 b)
    {
        return (unsigned)__bfloat16_as_ushort(a) | ((unsigned)__bfloat16_as_ushort(b) << 16);
    }
    __device__ static f2 get2(const __nv_bfloat16 *p)
    {
        return from_bits(__ldg(reinterpret_cast<const unsigned *>(p)));
    }
    __device__ static void put2(__nv_bfloat16 *p, const f2 &v) { *reinterpret_cast<unsigned *>(p) = to_bits(v); }
    __device__ static void put2raw(__nv_bfloat16 *p, __nv_bfloat16 a, __nv_bfloat16 b)
    {
        *reinterpret_cast<unsigned *>(p) = raw_bits(a, b);
    }
};

// Four consecutive stored 16-bit values (8-byte aligned) as FP32.
template <class T>
__device__ __forceinline__ void get4(const T *p, float (&w)[4])
{
    const uint2 u = __ldg(reinterpret_cast<const uint2 *>(p));
    const f2 lo = Pair16<T>::from_bits(u.x), hi = Pair16<T>::from_bits(u.y);
    w[0] = lo.v.x;
    w[1] = lo.v.y;
    w[2] = hi.v.x;
    w[3] = hi.v.y;
}

// The FP32 shape of component c at the K consecutive nodes (x0 + j, y) of one
// row of a 2D lattice (z = 0), i0 the node index of (x0, y): each value formed
// as field_value_f forms it, (px * py) * pz, with py and pz loaded once.
template <int K>
__device__ __forceinline__ void field_row_f(const FieldDev &F, int kind, int c, int x0, int y, int i0,
                                            float (&v)[K])
{
    if (kind == FK_CONST) {
#pragma unroll
        for (int j = 0; j < K; j++) v[j] = F.fcval[c];
        return;
    }
    if ((F.zmask >> c) & 1) {
#pragma unroll
        for (int j = 0; j < K; j++) v[j] = 0.0f;
        return;
    }
    const float *t = F.fdata + c * F.cstride;
    if (!F.sep) {
#pragma unroll
        for (int j = 0; j < K; j++) v[j] = __ldg(t + i0 + j);
        return;
    }
    const bool ax = F.axes & 1, ay = F.axes & 2, az = F.axes & 4;
    const float py = ay ? __ldg(t + F.len[0] + (F.len[1] > 1 ? y : 0)) : 1.0f;
    const float pz = az ? __ldg(t + F.len[0] + F.len[1]) : 1.0f;
#pragma unroll
    for (int j = 0; j < K; j++) {
        float w = 1.0f;
        bool have = false;
        if (ax) {
            w = __ldg(t + (F.len[0] > 1 ? x0 + j : 0));
            have = true;
        }
        if (ay) {
            w = have ? w * py : py;
            have = true;
        }
        if (az) w = have ? w * pz : pz;
        v[j] = w;
    }
}

// Pulled deviations of a 2D node pair (i0 = node (x, y), x even; i0 + 1), as
// pull_pair27 below: wrapped offsets along y, along x node 0's e_x = +1 source
// wraps at x = 0 and node 1's e_x = -1 source at x + 1 = nx - 1; the e_x = 0
// values of both nodes are one aligned 32-bit word.  A pair next to a wall
// takes the general per-node pull.
template <class L, class T>
__device__ __forceinline__ void pull_pair2d(const Planes<T, L::Q> &P, const Geom &g, int x, int y, int i0,
                                            f2 (&d)[L::Q])
{
    const bool wall_x = g.wall[0] && (x == 0 || x + 1 == g.nx - 1);
    const bool wall_y = g.wall[1] && (y == 0 || y == g.ny - 1);
    if (!(wall_x || wall_y)) {
        const int sy = g.nx;
        const int ym = y == 0 ? (g.ny - 1) * sy : -sy, yp = y == g.ny - 1 ? (1 - g.ny) * sy : sy;
        const int xm0 = x == 0 ? g.nx - 1 : -1;
        const int xp1 = x + 1 == g.nx - 1 ? 2 - g.nx : 2;
#pragma unroll
        for (int a = 0; a < L::Q; a++) {
            const int ex = L::ex(a), ey = L::ey(a);
            const T *pl = P.in[a] + i0 + (ey == 1 ? ym : (ey == -1 ? yp : 0));
            if (ex == 0) d[a] = Pair16<T>::get2(pl);
            else if (ex == 1) d[a] = f2(Dev<T>::get(pl + xm0), Dev<T>::get(pl));
            else d[a] = f2(Dev<T>::get(pl + 1), Dev<T>::get(pl + xp1));
        }
        return;
    }
    float d0[L::Q], d1[L::Q];
    load_pulled_dev<L, T>(P, g, x, y, 0, i0, d0);
    load_pulled_dev<L, T>(P, g, x + 1, y, 0, i0 + 1, d1);
#pragma unroll
    for (int a = 0; a < L::Q; a++) d[a] = f2(d0[a], d1[a]);
}

// Store a 16-bit node pair's deviations (rounded to nearest, or stochastically
// with each node's own bits).
template <class T, bool SR, int Q>
__device__ __forceinline__ void store_pair(T *const (&out)[Q], int i0, const f2 (&m)[Q], unsigned long long srkey)
{
    if constexpr (SR) {
        SRBits r0(srkey, i0), r1(srkey, i0 + 1);
#pragma unroll
        for (int a = 0; a < Q; a++) {
            const T lo = Round<T>::sr(m[a].v.x, r0.get(a)), hi = Round<T>::sr(m[a].v.y, r1.get(a));
            Pair16<T>::put2raw(out[a] + i0, lo, hi);
        }
    } else {
#pragma unroll
        for (int a = 0; a < Q; a++) Pair16<T>::put2(out[a] + i0, m[a]);
    }
}

// 16-bit D2Q9 storage, unit higher rates: two x-neighbouring nodes per thread
// in packed FP32x2 arithmetic (nx even; the launcher checks).  One node per
// thread keeps only 9 two-byte loads in flight per thread; the pair doubles
// that and halves the arithmetic instructions.
template <class T, int FK, bool SR = false>
__global__ void __launch_bounds__(kBlock)
k_step9x2(const __grid_constant__ Planes<T, 9> P, Geom g, FieldDev F, float apre, float gsum, Rates9f w, float rref,
          unsigned long long srkey)
{
    const int t = blockIdx.x * kBlock + threadIdx.x;
    if (t >= (g.N >> 1)) return;
    const int i0 = 2 * t;
    int x, y;
    node_xy(g, i0, x, y);
    f2 d[9];
    pull_pair2d<LD2Q9, T>(P, g, x, y, i0, d);
    f2 Fx(0.f), Fy(0.f), Gx(0.f), Gy(0.f);
    if (FK != FK_NONE) {
        float px[2], py[2];
        field_row_f<2>(F, FK, 0, x, y, i0, px);
        field_row_f<2>(F, FK, 1, x, y, i0, py);
        const f2 Px(px[0], px[1]), Py(py[0], py[1]);
        Fx = f2(apre) * Px;
        Fy = f2(apre) * Py;
        Gx = f2(gsum) * Px;
        Gy = f2(gsum) * Py;
    }
    collide9_w1<f2>(d, rref, Fx, Fy, Gx, Gy, w);
    store_pair<T, SR, 9>(P.out, i0, d, srkey);
}

// 16-bit D2Q5 storage, uniform advecting velocity: two x-neighbouring nodes
// per thread in packed FP32x2 arithmetic (nx even), the linear step of the
// deviations plus cref as the one-node kernel does.
template <class T, int SK, bool SR = false>
__global__ void __launch_bounds__(kBlock)
k_step5x2(const __grid_constant__ Planes<T, 5> P, Geom g, FieldDev S, float apre, float hsum, Coef5f k, Ref5f cref,
          unsigned long long srkey)
{
    const int t = blockIdx.x * kBlock + threadIdx.x;
    if (t >= (g.N >> 1)) return;
    const int i0 = 2 * t;
    int x, y;
    node_xy(g, i0, x, y);
    f2 d[5];
    pull_pair2d<LD2Q5, T>(P, g, x, y, i0, d);
    f2 Sp(0.f), H0(0.f);
    if (SK != FK_NONE) {
        float ps[2];
        field_row_f<2>(S, SK, 0, x, y, i0, ps);
        Sp = f2(apre) * f2(ps[0], ps[1]);
        H0 = f2(hsum) * f2(ps[0], ps[1]);
    }
    collide5u<f2>(d, 0.0f, Sp, H0, k);
#pragma unroll
    for (int a = 0; a < 5; a++) d[a] = d[a] + f2(cref.v[a]);
    store_pair<T, SR, 5>(P.out, i0, d, srkey);
}

// Pulled deviations of four consecutive nodes of a 2D row (i0 = node (x0, y),
// x0 a multiple of 4; nodes x0, x0 + 1 in dA, x0 + 2, x0 + 3 in dB).  Every
// plane is one aligned 64-bit load of the four values at the source row; a
// plane with e_x = +1 adds the value at x0 - 1, one with e_x = -1 the value at
// x0 + 4 (both wrapped).  Next to a wall: the general per-node pull.
template <class L, class T>
__device__ __forceinline__ void pull_quad2d(const Planes<T, L::Q> &P, const Geom &g, int x0, int y, int i0,
                                            f2 (&dA)[L::Q], f2 (&dB)[L::Q])
{
    const bool wall_x = g.wall[0] && (x0 == 0 || x0 + 3 == g.nx - 1);
    const bool wall_y = g.wall[1] && (y == 0 || y == g.ny - 1);
    if (!(wall_x || wall_y)) {
        const int sy = g.nx;
        const int ym = y == 0 ? (g.ny - 1) * sy : -sy, yp = y == g.ny - 1 ? (1 - g.ny) * sy : sy;
        const int xm = x0 == 0 ? g.nx - 1 : -1;       // node x0 - 1, wrapped
        const int xp = x0 + 4 == g.nx ? 4 - g.nx : 4;  // node x0 + 4, wrapped
#pragma unroll
        for (int a = 0; a < L::Q; a++) {
            const int ex = L::ex(a), ey = L::ey(a);
            const T *pl = P.in[a] + i0 + (ey == 1 ? ym : (ey == -1 ? yp : 0));
            float w[4];
            get4<T>(pl, w);
            if (ex == 0) {
                dA[a] = f2(w[0], w[1]);
                dB[a] = f2(w[2], w[3]);
            } else if (ex == 1) {
                dA[a] = f2(Dev<T>::get(pl + xm), w[0]);
                dB[a] = f2(w[1], w[2]);
            } else {
                dA[a] = f2(w[1], w[2]);
                dB[a] = f2(w[3], Dev<T>::get(pl + xp));
            }
        }
        return;
    }
    float d0[L::Q], d1[L::Q], d2[L::Q], d3[L::Q];
    load_pulled_dev<L, T>(P, g, x0, y, 0, i0, d0);
    load_pulled_dev<L, T>(P, g, x0 + 1, y, 0, i0 + 1, d1);
    load_pulled_dev<L, T>(P, g, x0 + 2, y, 0, i0 + 2, d2);
    load_pulled_dev<L, T>(P, g, x0 + 3, y, 0, i0 + 3, d3);
#pragma unroll
    for (int a = 0; a < L::Q; a++) {
        dA[a] = f2(d0[a], d1[a]);
        dB[a] = f2(d2[a], d3[a]);
    }
}

// Store four consecutive nodes' deviations as one 64-bit word per plane.
template <class T, bool SR, int Q>
__device__ __forceinline__ void store_quad(T *const (&out)[Q], int i0, const f2 (&A)[Q], const f2 (&B)[Q],
                                           unsigned long long srkey)
{
    if constexpr (SR) {
        SRBits r0(srkey, i0), r1(srkey, i0 + 1), r2(srkey, i0 + 2), r3(srkey, i0 + 3);
#pragma unroll
        for (int a = 0; a < Q; a++) {
            const unsigned lo = Pair16<T>::raw_bits(Round<T>::sr(A[a].v.x, r0.get(a)), Round<T>::sr(A[a].v.y, r1.get(a)));
            const unsigned hi = Pair16<T>::raw_bits(Round<T>::sr(B[a].v.x, r2.get(a)), Round<T>::sr(B[a].v.y, r3.get(a)));
            *reinterpret_cast<uint2 *>(out[a] + i0) = make_uint2(lo, hi);
        }
    } else {
#pragma unroll
        for (int a = 0; a < Q; a++)
            *reinterpret_cast<uint2 *>(out[a] + i0) = make_uint2(Pair16<T>::to_bits(A[a]), Pair16<T>::to_bits(B[a]));
    }
}

// 16-bit D2Q9 (unit higher rates) and D2Q5 (uniform velocity) storage, four
// consecutive nodes of a row per thread (nx a multiple of 4; the launchers
// check): two packed pairs, the plane addresses and the y / z factors of the
// force or source shared by the four, 64-bit loads and stores.  One or two
// nodes per thread spend most of their instructions on addressing.
template <class T, int FK, bool SR = false>
__global__ void __launch_bounds__(kBlock)
k_step9x4(const __grid_constant__ Planes<T, 9> P, Geom g, FieldDev F, float apre, float gsum, Rates9f w, float rref,
          unsigned long long srkey)
{
    const int t = blockIdx.x * kBlock + threadIdx.x;
    if (t >= (g.N >> 2)) return;
    const int i0 = 4 * t;
    int x0, y;
    node_xy(g, i0, x0, y);
    f2 dA[9], dB[9];
    pull_quad2d<LD2Q9, T>(P, g, x0, y, i0, dA, dB);
    f2 FxA(0.f), FyA(0.f), GxA(0.f), GyA(0.f), FxB(0.f), FyB(0.f), GxB(0.f), GyB(0.f);
    if (FK != FK_NONE) {
        float px[4], py[4];
        field_row_f<4>(F, FK, 0, x0, y, i0, px);
        field_row_f<4>(F, FK, 1, x0, y, i0, py);
        const f2 PxA(px[0], px[1]), PyA(py[0], py[1]), PxB(px[2], px[3]), PyB(py[2], py[3]);
        FxA = f2(apre) * PxA;
        FyA = f2(apre) * PyA;
        GxA = f2(gsum) * PxA;
        GyA = f2(gsum) * PyA;
        FxB = f2(apre) * PxB;
        FyB = f2(apre) * PyB;
        GxB = f2(gsum) * PxB;
        GyB = f2(gsum) * PyB;
    }
    collide9_w1<f2>(dA, rref, FxA, FyA, GxA, GyA, w);
    collide9_w1<f2>(dB, rref, FxB, FyB, GxB, GyB, w);
    store_quad<T, SR, 9>(P.out, i0, dA, dB, srkey);
}

template <class T, int SK, bool SR = false>
__global__ void __launch_bounds__(kBlock)
k_step5x4(const __grid_constant__ Planes<T, 5> P, Geom g, FieldDev S, float apre, float hsum, Coef5f k, Ref5f cref,
          unsigned long long srkey)
{
    const int t = blockIdx.x * kBlock + threadIdx.x;
    if (t >= (g.N >> 2)) return;
    const int i0 = 4 * t;
    int x0, y;
    node_xy(g, i0, x0, y);
    f2 dA[5], dB[5];
    pull_quad2d<LD2Q5, T>(P, g, x0, y, i0, dA, dB);
    f2 SpA(0.f), H0A(0.f), SpB(0.f), H0B(0.f);
    if (SK != FK_NONE) {
        float ps[4];
        field_row_f<4>(S, SK, 0, x0, y, i0, ps);
        const f2 PA(ps[0], ps[1]), PB(ps[2], ps[3]);
        SpA = f2(apre) * PA;
        H0A = f2(hsum) * PA;
        SpB = f2(apre) * PB;
        H0B = f2(hsum) * PB;
    }
    collide5u<f2>(dA, 0.0f, SpA, H0A, k);
    collide5u<f2>(dB, 0.0f, SpB, H0B, k);
#pragma unroll
    for (int a = 0; a < 5; a++) {
        dA[a] = dA[a] + f2(cref.v[a]);
        dB[a] = dB[a] + f2(cref.v[a]);
    }
    store_quad<T, SR, 5>(P.out, i0, dA, dB, srkey);
}

// Pulled deviations of the node pair (i0 = node (x, y, z), x even; i0 + 1).
template <class T>
__device__ __forceinline__ void pull_pair27(const Planes<T, 27> &P, const Geom &g, int x, int y, int z, int i0,
                                            f2 (&m)[27])
{
    const bool wall_x = g.wall[0] && (x == 0 || x + 1 == g.nx - 1);
    const bool wall_y = g.wall[1] && (y == 0 || y == g.ny - 1);
    const bool wall_z = g.wall[2] && (z == 0 || z == g.nz - 1);
    if (!(wall_x || wall_y || wall_z)) {
        // wrapped source offsets along y and z (as pull_node), and along x:
        // e_x = +1 takes x - 1 (node 0 wraps at x = 0; node 1's source is
        // node 0's position), e_x = -1 takes x + 1 (node 0's source is node
        // 1's position; node 1 wraps at x + 1 = nx - 1)
        const int sy = g.nx, sz = g.nx * g.ny;
        const int ym = y == 0 ? (g.ny - 1) * sy : -sy, yp = y == g.ny - 1 ? (1 - g.ny) * sy : sy;
        const int zm = z == 0 ? (g.nz - 1) * sz : -sz, zp = z == g.nz - 1 ? (1 - g.nz) * sz : sz;
        const int xm0 = x == 0 ? g.nx - 1 : -1;
        const int xp1 = x + 1 == g.nx - 1 ? 2 - g.nx : 2;
#pragma unroll
        for (int a = 0; a < 27; a++) {
            const int ex = LD3Q27::ex(a), ey = LD3Q27::ey(a), ez = LD3Q27::ez(a);
            const T *pl = P.in[a] + i0 + (ey == 1 ? ym : (ey == -1 ? yp : 0)) + (ez == 1 ? zm : (ez == -1 ? zp : 0));
            if (ex == 0) m[a] = Pair16<T>::get2(pl);  // both nodes' values, one aligned word
            else if (ex == 1) m[a] = f2(Dev<T>::get(pl + xm0), Dev<T>::get(pl));
            else m[a] = f2(Dev<T>::get(pl + 1), Dev<T>::get(pl + xp1));
        }
        return;
    }
    float d0[27], d1[27];
    load_pulled_dev<LD3Q27, T>(P, g, x, y, z, i0, d0);
    load_pulled_dev<LD3Q27, T>(P, g, x + 1, y, z, i0 + 1, d1);
#pragma unroll
    for (int a = 0; a < 27; a++) m[a] = f2(d0[a], d1[a]);
}

constexpr int kBlockPair = 128;
// Blocks of the pair kernel resident per SM (bounds its registers): 6 x 128
// threads at <= 80 registers keep 1536 nodes' loads in flight per SM; 4
// blocks (120 registers, no spills) ran at 0.69 of HBM on the 512^3 FP16 grid,
// 5 at 0.75, 6 at 0.79 (a few spilled registers cost less than the loads the
// extra blocks keep in flight).
#ifndef LBM_PAIR_MIN_BLOCKS
#define LBM_PAIR_MIN_BLOCKS 6
#endif

// XO: the force acts along x only (checked on the host).
template <class T, int FK, bool SR = false, bool XO = false>
__global__ void __launch_bounds__(kBlockPair, LBM_PAIR_MIN_BLOCKS)
k_step27x2(const __grid_constant__ Planes<T, 27> P, Geom g, FieldDev Fd, float apre, float apost, Rates27f w,
           float rref, unsigned long long srkey)
{
    const int t = blockIdx.x * kBlockPair + threadIdx.x;
    if (t >= (g.N >> 1)) return;
    const int i0 = 2 * t;
    int x, y, z;
    node_xyz(g, i0, x, y, z);
    f2 m[27];
    pull_pair27<T>(P, g, x, y, z, i0, m);
    f2 F[3] = {f2(0.f), f2(0.f), f2(0.f)}, Fq[3] = {f2(0.f), f2(0.f), f2(0.f)};
    if (FK != FK_NONE) {
#pragma unroll
        for (int d = 0; d < (XO ? 1 : 3); d++) {
            const f2 Pd(field_value_f(Fd, FK, d, x, y, z, i0), field_value_f(Fd, FK, d, x + 1, y, z, i0 + 1));
            F[d] = f2(apre) * Pd;
            Fq[d] = f2(apost) * Pd;
        }
    }
    collide27_w1<f2, XO>(m, rref, F, Fq, w);
    store_pair<T, SR, 27>(P.out, i0, m, srkey);
}

// --------------------------------------------------------------- batched ---
// (tile loop: lbm_tiles.cuh)

// A batched node in two phases: fetch issues the node's global loads (pulled
// populations, envelope pair, force or source and velocity values) before
// finish does any arithmetic and the stores.
struct In9 {
    float d[9];
    float Px, Py;  // force shape at the node (0 without a force)
    float2 ap;     // (a_pre, (a_pre + a_post)/12)
    int i;
};

template <class T>
__device__ __forceinline__ void fetch9(const BatchItem &B, const BatchLaunch &L, int it, int i, In9 &s)
{
    const Geom &g = B.g;
    s.i = i;
    if (i >= g.N) return;
    const T *fin = reinterpret_cast<const T *>(B.buf[(B.parity + L.parity) & 1]);
    s.ap = L.pairsf ? L.pairsf[(size_t)L.k * L.count + it] : L.inlf[it];
    int x, y;
    node_xy(g, i, x, y);
    load_pulled_dev<LD2Q9, T>(fin, g, x, y, 0, i, s.d);
    s.Px = s.Py = 0.f;
    if (B.fkind != FK_NONE) {
        s.Px = field_value_f(B.F, B.fkind, 0, x, y, 0, i);
        s.Py = field_value_f(B.F, B.fkind, 1, x, y, 0, i);
    }
}

template <class T>
__device__ __forceinline__ void finish9(const BatchItem &B, const BatchLaunch &L, int it, In9 &s)
{
    const Geom &g = B.g;
    const int i = s.i;
    if (i >= g.N) return;
    T *fout = reinterpret_cast<T *>(B.buf[(B.parity + L.parity + 1) & 1]);
    float Fx = 0.f, Fy = 0.f, Gx = 0.f, Gy = 0.f;
    if (B.fkind != FK_NONE) {
        Fx = s.ap.x * s.Px;
        Fy = s.ap.x * s.Py;
        Gx = s.ap.y * s.Px;
        Gy = s.ap.y * s.Py;
    }
    const Rates9f w{B.fcoef[0], B.fcoef[1], B.fcoef[2], B.fcoef[3], B.fcoef[4], B.fcoef[5]};
    if (B.variant == 1) collide9_w1(s.d, B.frho_ref, Fx, Fy, Gx, Gy, w);  // uniform over the member
    else collide9(s.d, B.frho_ref, Fx, Fy, Gx, Gy, w);
#pragma unroll
    for (int a = 0; a < 9; a++) fout[a * g.Np + i] = Dev<T>::to_store(s.d[a]);
}

template <class T>
__device__ __forceinline__ void node9(const BatchItem &B, const BatchLaunch &L, int it, int i)
{
    In9 s;
    fetch9<T>(B, L, it, i, s);
    finish9<T>(B, L, it, s);
}

// D2Q5 items carry Coef5 (double) in coef[0..11] and the rates in coef[12..15].
struct In5 {
    float d[5];
    float P;        // source shape at the node (0 without a source)
    float ux, uy;   // advecting velocity (members with a velocity field)
    float2 ap;      // (a_pre, (a_pre + a_post)/10)
    int i;
};

template <class T>
__device__ __forceinline__ void fetch5(const BatchItem &B, const BatchLaunch &L, int it, int i, In5 &s)
{
    const Geom &g = B.g;
    s.i = i;
    if (i >= g.N) return;
    const T *fin = reinterpret_cast<const T *>(B.buf[(B.parity + L.parity) & 1]);
    s.ap = L.pairsf ? L.pairsf[(size_t)L.k * L.count + it] : L.inlf[it];
    int x, y;
    node_xy(g, i, x, y);
    load_pulled_dev<LD2Q5, T>(fin, g, x, y, 0, i, s.d);
    s.P = B.fkind != FK_NONE ? field_value_f(B.F, B.fkind, 0, x, y, 0, i) : 0.f;
    if (B.vkind == FK_GENERAL) {
        s.ux = field_value_f(B.V, FK_GENERAL, 0, x, y, 0, i);
        s.uy = field_value_f(B.V, FK_GENERAL, 1, x, y, 0, i);
    }
}

template <class T>
__device__ __forceinline__ void finish5(const BatchItem &B, const BatchLaunch &L, int it, In5 &s)
{
    const Geom &g = B.g;
    const int i = s.i;
    if (i >= g.N) return;
    T *fout = reinterpret_cast<T *>(B.buf[(B.parity + L.parity + 1) & 1]);
    float (&d)[5] = s.d;
    float Sp = 0.f, H0 = 0.f;
    if (B.fkind != FK_NONE) {
        Sp = s.ap.x * s.P;
        H0 = s.ap.y * s.P;
    }
    const float rref = B.frho_ref;
    if (B.vkind != FK_GENERAL) {
        Coef5f k;
        k.A1 = B.fcoef[0]; k.c1 = B.fcoef[1]; k.A2 = B.fcoef[2]; k.c2 = B.fcoef[3];
        k.P3 = B.fcoef[4]; k.X3 = B.fcoef[5]; k.Y3 = B.fcoef[6]; k.S3 = B.fcoef[7];
        k.P4 = B.fcoef[8]; k.X4 = B.fcoef[9]; k.Y4 = B.fcoef[10]; k.D4 = B.fcoef[11];
        k.Q3 = B.fcoef[16];
        collide5u(d, 0.0f, Sp, H0, k);
#pragma unroll
        for (int a = 0; a < 5; a++) d[a] += B.fref[a];
    } else {
        const Rates5f w{B.fcoef[12], B.fcoef[13], B.fcoef[14], B.fcoef[15]};
        collide5(d, rref, Sp, H0, s.ux, s.uy, w);
    }
#pragma unroll
    for (int a = 0; a < 5; a++) fout[a * g.Np + i] = Dev<T>::to_store(d[a]);
}

template <class T>
__device__ __forceinline__ void node5(const BatchItem &B, const BatchLaunch &L, int it, int i)
{
    In5 s;
    fetch5<T>(B, L, it, i, s);
    finish5<T>(B, L, it, s);
}

template <class T>
__device__ __forceinline__ void node27(const BatchItem &B, const BatchLaunch &L, int it, int i)
{
    const Geom &g = B.g;
    const int p = B.parity + L.parity;
    const T *fin = reinterpret_cast<const T *>(B.buf[p & 1]);
    T *fout = reinterpret_cast<T *>(B.buf[(p + 1) & 1]);
    const float2 ap = L.pairsf ? L.pairsf[(size_t)L.k * L.count + it] : L.inlf[it];
    int x, y, z;
    node_xyz(g, i, x, y, z);
    float m[27];
    load_pulled_dev<LD3Q27, T>(fin, g, x, y, z, i, m);
    float F[3] = {0.f, 0.f, 0.f}, Fq[3] = {0.f, 0.f, 0.f};
    if (B.fkind != FK_NONE) {
#pragma unroll
        for (int d = 0; d < 3; d++) {
            const float P = field_value_f(B.F, B.fkind, d, x, y, z, i);
            F[d] = ap.x * P;
            Fq[d] = ap.y * P;
        }
    }
    const Rates27f w{B.fcoef[0], B.fcoef[1], B.fcoef[2], B.fcoef[3], B.fcoef[4], B.fcoef[5]};
    if (B.variant == 1) collide27_w1(m, B.frho_ref, F, Fq, w);  // uniform over the block's tile
    else collide27(m, B.frho_ref, F, Fq, w);
#pragma unroll
    for (int a = 0; a < 27; a++) fout[a * g.Np + i] = Dev<T>::to_store(m[a]);
}

template <class T, int TB, int MODE>
__global__ void __launch_bounds__(TB) k_batch9(const __grid_constant__ BatchLaunch L)
{
    batch_tiles<TB, MODE>(L, [](const BatchItem &B, const BatchLaunch &L2, int it, int i) { node9<T>(B, L2, it, i); });
}

template <class T, int TB, int MODE>
__global__ void __launch_bounds__(TB) k_batch5(const __grid_constant__ BatchLaunch L)
{
    batch_tiles<TB, MODE>(L, [](const BatchItem &B, const BatchLaunch &L2, int it, int i) { node5<T>(B, L2, it, i); });
}

// 1024 / TB blocks per SM keep the D3Q27 kernel at <= 64 registers.
template <class T, int TB, int MODE>
__global__ void __launch_bounds__(TB, 1024 / TB) k_batch27(const __grid_constant__ BatchLaunch L)
{
    batch_tiles<TB, MODE>(L, [](const BatchItem &B, const BatchLaunch &L2, int it, int i) { node27<T>(B, L2, it, i); });
}


template <class T, bool W1, bool SR>
void step9_launch(const Planes<T, 9> &fin, const LaunchArgs &a, int grid, float apre, float gsum, const Rates9f &w,
                  float rref, cudaStream_t s)
{
    const unsigned long long k = a.srkey;
    if constexpr (sizeof(T) == 2 && W1) {
        if (a.g.nx % 4 == 0) {
            // four consecutive nodes of a row per thread
            const int qgrid = (a.g.N / 4 + kBlock - 1) / kBlock;
            if (a.fkind == FK_NONE)
                k_step9x4<T, FK_NONE, SR><<<qgrid, kBlock, 0, s>>>(fin, a.g, a.F, apre, gsum, w, rref, k);
            else if (a.fkind == FK_CONST)
                k_step9x4<T, FK_CONST, SR><<<qgrid, kBlock, 0, s>>>(fin, a.g, a.F, apre, gsum, w, rref, k);
            else k_step9x4<T, FK_GENERAL, SR><<<qgrid, kBlock, 0, s>>>(fin, a.g, a.F, apre, gsum, w, rref, k);
            return;
        }
        if (a.g.nx % 2 == 0) {
            // two x-neighbouring nodes per thread, packed FP32x2 arithmetic
            const int pgrid = (a.g.N / 2 + kBlock - 1) / kBlock;
            if (a.fkind == FK_NONE)
                k_step9x2<T, FK_NONE, SR><<<pgrid, kBlock, 0, s>>>(fin, a.g, a.F, apre, gsum, w, rref, k);
            else if (a.fkind == FK_CONST)
                k_step9x2<T, FK_CONST, SR><<<pgrid, kBlock, 0, s>>>(fin, a.g, a.F, apre, gsum, w, rref, k);
            else k_step9x2<T, FK_GENERAL, SR><<<pgrid, kBlock, 0, s>>>(fin, a.g, a.F, apre, gsum, w, rref, k);
            return;
        }
    }
    if (a.fkind == FK_NONE) k_step9<T, FK_NONE, W1, SR><<<grid, kBlock, 0, s>>>(fin, a.g, a.F, apre, gsum, w, rref, k);
    else if (a.fkind == FK_CONST)
        k_step9<T, FK_CONST, W1, SR><<<grid, kBlock, 0, s>>>(fin, a.g, a.F, apre, gsum, w, rref, k);
    else k_step9<T, FK_GENERAL, W1, SR><<<grid, kBlock, 0, s>>>(fin, a.g, a.F, apre, gsum, w, rref, k);
}

template <class T, int SK, bool SR>
void step5_launch(const Planes<T, 5> &fin, const LaunchArgs &a, int grid, float apre, float hsum, const Rates5f &w,
                  const Coef5f &k, float rref, const Ref5f &cref, bool uni, cudaStream_t s)
{
    if constexpr (sizeof(T) == 2) {
        if (uni && a.g.nx % 4 == 0) {
            // four consecutive nodes of a row per thread
            const int qgrid = (a.g.N / 4 + kBlock - 1) / kBlock;
            k_step5x4<T, SK, SR><<<qgrid, kBlock, 0, s>>>(fin, a.g, a.F, apre, hsum, k, cref, a.srkey);
            return;
        }
        if (uni && a.g.nx % 2 == 0) {
            // two x-neighbouring nodes per thread, packed FP32x2 arithmetic
            const int pgrid = (a.g.N / 2 + kBlock - 1) / kBlock;
            k_step5x2<T, SK, SR><<<pgrid, kBlock, 0, s>>>(fin, a.g, a.F, apre, hsum, k, cref, a.srkey);
            return;
        }
    }
    if (uni)
        k_step5<T, SK, true, SR><<<grid, kBlock, 0, s>>>(fin, a.g, a.F, a.V, apre, hsum, w, k, rref, cref, a.srkey);
    else
        k_step5<T, SK, false, SR><<<grid, kBlock, 0, s>>>(fin, a.g, a.F, a.V, apre, hsum, w, k, rref, cref, a.srkey);
}

template <class T, int FK, bool SR>
void step27_launch(const Planes<T, 27> &fin, const LaunchArgs &a, float ap, float aq, const Rates27f &w, float rref,
                   bool w1, cudaStream_t s)
{
    if constexpr (sizeof(T) == 2) {
        if (w1 && a.g.nx % 2 == 0) {
            // two x-neighbouring nodes per thread, packed FP32x2 arithmetic
            const int pgrid = (a.g.N / 2 + kBlockPair - 1) / kBlockPair;
            if (FK != FK_NONE && force_x_only(FK, a.F, 3))
                k_step27x2<T, FK, SR, true><<<pgrid, kBlockPair, 0, s>>>(fin, a.g, a.F, ap, aq, w, rref, a.srkey);
            else
                k_step27x2<T, FK, SR, false><<<pgrid, kBlockPair, 0, s>>>(fin, a.g, a.F, ap, aq, w, rref, a.srkey);
            return;
        }
    }
    const int grid = (a.g.N + kBlock - 1) / kBlock;
    if (w1) k_step27<T, FK, true, SR><<<grid, kBlock, 0, s>>>(fin, a.g, a.F, ap, aq, w, rref, a.srkey);
    else k_step27<T, FK, false, SR><<<grid, kBlock, 0, s>>>(fin, a.g, a.F, ap, aq, w, rref, a.srkey);
}

template <class T, bool SR>
cudaError_t step_ts(int lattice, const LaunchArgs &a)
{
    const int grid = (a.g.N + kBlock - 1) / kBlock;
    const float rref = (float)a.rho_ref;
    const cudaStream_t s = a.stream;
    if (lattice == LD2Q9::ID) {
        const Planes<T, 9> fin = make_planes<T, 9>(a.fin, a.fout, a.g.Np);
        const Rates9f w{(float)(a.omega[3] / 12.0), (float)(a.omega[4] / 4.0), (float)(a.omega[5] / 4.0),
                        (float)(a.omega[6] / 4.0), (float)(a.omega[7] / 4.0), (float)(a.omega[8] / 4.0)};
        const float gsum = (float)((a.apre + a.apost) / 12.0), apre = (float)a.apre;
        const bool w1 = a.omega[6] == 1.0 && a.omega[7] == 1.0 && a.omega[8] == 1.0;
        if (w1) step9_launch<T, true, SR>(fin, a, grid, apre, gsum, w, rref, s);
        else step9_launch<T, false, SR>(fin, a, grid, apre, gsum, w, rref, s);
    } else if (lattice == LD2Q5::ID) {
        const Rates5f w{(float)(a.omega[1] / 2.0), (float)(a.omega[2] / 2.0), (float)(a.omega[3] / 4.0),
                        (float)(a.omega[4] / 4.0)};
        const double ux = a.vkind == FK_CONST ? a.V.cval[0] : 0.0, uy = a.vkind == FK_CONST ? a.V.cval[1] : 0.0;
        const Coef5f k = make_coef5f(a.omega, ux, uy);
        const float hsum = (float)((a.apre + a.apost) / 10.0), apre = (float)a.apre;
        const bool uni = a.vkind != FK_GENERAL;
        Ref5f cref{};
        if (uni) {
            double c[5];
            d2q5_reference_change(a.omega, ux, uy, a.gref, c);
            for (int q = 0; q < 5; q++) cref.v[q] = (float)c[q];
        }
        const Planes<T, 5> fin = make_planes<T, 5>(a.fin, a.fout, a.g.Np);
        if (a.fkind == FK_NONE) step5_launch<T, FK_NONE, SR>(fin, a, grid, apre, hsum, w, k, rref, cref, uni, s);
        else if (a.fkind == FK_CONST)
            step5_launch<T, FK_CONST, SR>(fin, a, grid, apre, hsum, w, k, rref, cref, uni, s);
        else step5_launch<T, FK_GENERAL, SR>(fin, a, grid, apre, hsum, w, k, rref, cref, uni, s);
    } else {
        const Rates27f w{(float)a.omega[1], (float)a.omega[2], (float)a.omega[3],
                         (float)a.omega[4], (float)a.omega[5], (float)a.omega[6]};
        const bool w1 = a.omega[3] == 1.0 && a.omega[4] == 1.0 && a.omega[5] == 1.0 && a.omega[6] == 1.0;
        const float ap = (float)a.apre, aq = (float)a.apost;
        const Planes<T, 27> fin = make_planes<T, 27>(a.fin, a.fout, a.g.Np);
        if (a.fkind == FK_NONE) step27_launch<T, FK_NONE, SR>(fin, a, ap, aq, w, rref, w1, s);
        else if (a.fkind == FK_CONST) step27_launch<T, FK_CONST, SR>(fin, a, ap, aq, w, rref, w1, s);
        else step27_launch<T, FK_GENERAL, SR>(fin, a, ap, aq, w, rref, w1, s);
    }
    return cudaGetLastError();
}

// Stochastic rounding is a 16-bit storage option (FP32 rounding is taken to
// nearest always).
template <class T>
cudaError_t step_t(int lattice, const LaunchArgs &a)
{
    if constexpr (sizeof(T) == 2) {
        if (a.sround) return step_ts<T, true>(lattice, a);
    }
    return step_ts<T, false>(lattice, a);
}

template <class T, int TB, int M>
cudaError_t batch_tbm(int lattice, const BatchLaunch &L, int nblocks, cudaStream_t s)
{
    if (lattice == LD2Q9::ID) k_batch9<T, TB, M><<<nblocks, TB, 0, s>>>(L);
    else if (lattice == LD2Q5::ID) k_batch5<T, TB, M><<<nblocks, TB, 0, s>>>(L);
    else k_batch27<T, TB, M><<<nblocks, TB, 0, s>>>(L);
    return cudaGetLastError();
}

template <class T, int TB>
cudaError_t batch_tb(int lattice, const BatchLaunch &L, int nblocks, cudaStream_t s)
{
    const int m = tile_mode(L);
    if (m == TILE_SINGLE) return batch_tbm<T, TB, TILE_SINGLE>(lattice, L, nblocks, s);
    if (m == TILE_PERSIST) return batch_tbm<T, TB, TILE_PERSIST>(lattice, L, nblocks, s);
    return batch_tbm<T, TB, TILE_ONE>(lattice, L, nblocks, s);
}

template <class T>
cudaError_t batch_t(int lattice, const BatchLaunch &L, int nblocks, int tile, cudaStream_t s)
{
    switch (tile) {
    case 128: return batch_tb<T, 128>(lattice, L, nblocks, s);
    case 256: return batch_tb<T, 256>(lattice, L, nblocks, s);
    case 512: return batch_tb<T, 512>(lattice, L, nblocks, s);
    default: return cudaErrorInvalidValue;
    }
}

template <class T, int TB>
int resident_tb(int lattice)
{
    if (lattice == LD2Q9::ID) return resident_blocks(k_batch9<T, TB, TILE_PERSIST>, TB);
    if (lattice == LD2Q5::ID) return resident_blocks(k_batch5<T, TB, TILE_PERSIST>, TB);
    return resident_blocks(k_batch27<T, TB, TILE_PERSIST>, TB);
}

template <class T>
int resident_t(int lattice, int tile)
{
    switch (tile) {
    case 128: return resident_tb<T, 128>(lattice);
    case 256: return resident_tb<T, 256>(lattice);
    case 512: return resident_tb<T, 512>(lattice);
    default: return 0;
    }
}

struct LrefK {
    const float *ref;    // [1 or 3][Np]: dphi, or drho, jx, jy
    const float *scale;  // [2]: sigma, 1 / sigma
    long long Np;
    float q5[5];
};

// ------------------------------------------------ local-reference encoding ---
// 16-bit storage at a per-node reference.  A 16-bit deviation from the fixed
// reference state of a few 1e-4 has a step of ~1e-7 (FP16) or ~1e-6 (BF16),
// the size of one step's force or source increment, so increments are lost.
// Here the stored value is s_a(x) = sigma (d_a(x) - e_a(x)): d the deviation of
// the FP32 forms, e_a(x) the deviation of a low-order equilibrium at the
// node's reference -- D2Q9: e_a = w_a (drho + 3 e_a . j + second-order terms);
// D2Q5 at a uniform velocity u: e_a = q_a dphi, q the equilibrium per unit
// scalar at u (Eq. 39) -- which holds the node's zeroth and first moments in
// FP32, and sigma a power of two per lattice that brings the lattice's
// largest |d - e| to [8, 16) (FP16 then holds values 4096 times larger).  A
// step pulls d = s / sigma + e (e of the source node), collides in FP32
// exactly as the deviation kernels do and stores sigma (d - e) of its own
// node.  The reference is rebuilt from the state every few steps (rebase), so
// s holds only the non-equilibrium part and the change since the last rebase.
// (A per-node sigma, up to 2^8 times the lattice's, was tried: it overflowed
// FP16 in start-up transients next to walls and was no more accurate.)

// e_a from a node's reference values r0 (drho or dphi), r1, r2 (j, D2Q9 only).
// D2Q9: w_a (drho + 3 c + 4.5 c^2 - 1.5 |j|^2), c = e_a . j -- the equilibrium
// to second order in j at unit density, whose zeroth and first moments are
// drho and j.
template <class L>
__device__ __forceinline__ float lref_e_of(const LrefK &R, int a, float r0, float r1, float r2)
{
    if constexpr (L::Q == 9) {
        const float c = fmaf((float)LD2Q9::ex(a), r1, (float)LD2Q9::ey(a) * r2);
        const float q = fmaf(4.5f * c, c, -1.5f * fmaf(r1, r1, r2 * r2));
        return (float)LD2Q9::w(a) * fmaf(3.0f, c, r0 + q);
    } else {
        return R.q5[a] * r0;
    }
}
template <class L>
__device__ __forceinline__ float lref_e(const LrefK &R, int a, int k)
{
    const float r0 = __ldg(R.ref + k);
    float r1 = 0.f, r2 = 0.f;
    if constexpr (L::Q == 9) {
        r1 = __ldg(R.ref + R.Np + k);
        r2 = __ldg(R.ref + 2 * R.Np + k);
    }
    return lref_e_of<L>(R, a, r0, r1, r2);
}

// the stored value s of population a at node k, decoded: s / sigma + e_a(k)
template <class L, class T>
__device__ __forceinline__ float lref_dec(const LrefK &R, const T *plane, int a, int k, float sinv)
{
    return fmaf(Dev<T>::get(plane + k), sinv, lref_e<L>(R, a, k));
}
// the value to store for deviation d of population a at node k
template <class L>
__device__ __forceinline__ float lref_enc(const LrefK &R, float d, int a, int k, float sig)
{
    return (d - lref_e<L>(R, a, k)) * sig;
}

template <class T, int FK, bool W1, bool SR>
__global__ void __launch_bounds__(kBlock)
k_lref_step9(const __grid_constant__ Planes<T, 9> P, Geom g, FieldDev F, float apre, float gsum, Rates9f w, float rref,
             LrefK R, unsigned long long srkey)
{
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    int x, y;
    node_xy(g, i, x, y);
    const float sig = __ldg(R.scale), sinv = __ldg(R.scale + 1);
    float d[9];
    pull_node<LD2Q9>(g, x, y, 0, i, d, [&](int p, int k) { return lref_dec<LD2Q9, T>(R, P.in[p], p, k, sinv); });
    float Fx = 0.f, Fy = 0.f, Gx = 0.f, Gy = 0.f;
    if (FK != FK_NONE) {
        const float Px = field_value_f(F, FK, 0, x, y, 0, i), Py = field_value_f(F, FK, 1, x, y, 0, i);
        Fx = apre * Px;
        Fy = apre * Py;
        Gx = gsum * Px;
        Gy = gsum * Py;
    }
    if (W1) collide9_w1(d, rref, Fx, Fy, Gx, Gy, w);
    else collide9(d, rref, Fx, Fy, Gx, Gy, w);
    SRBits rb(srkey, i);
#pragma unroll
    for (int a = 0; a < 9; a++) P.out[a][i] = store_dev<T, SR>(lref_enc<LD2Q9>(R, d[a], a, i, sig), rb, a);
}

template <class T, int SK, bool SR>
__global__ void __launch_bounds__(kBlock)
k_lref_step5(const __grid_constant__ Planes<T, 5> P, Geom g, FieldDev S, float apre, float hsum, Coef5f k, Ref5f cref,
             LrefK R, unsigned long long srkey)
{
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    int x, y;
    node_xy(g, i, x, y);
    const float sig = __ldg(R.scale), sinv = __ldg(R.scale + 1);
    float d[5];
    pull_node<LD2Q5>(g, x, y, 0, i, d, [&](int p, int kk) { return lref_dec<LD2Q5, T>(R, P.in[p], p, kk, sinv); });
    float Sp = 0.f, H0 = 0.f;
    if (SK != FK_NONE) {
        const float Ps = field_value_f(S, SK, 0, x, y, 0, i);
        Sp = apre * Ps;
        H0 = hsum * Ps;
    }
    collide5u(d, 0.0f, Sp, H0, k);
    SRBits rb(srkey, i);
#pragma unroll
    for (int a = 0; a < 5; a++) P.out[a][i] = store_dev<T, SR>(lref_enc<LD2Q5>(R, d[a] + cref.v[a], a, i, sig), rb, a);
}

// Four consecutive nodes of a row per thread (nx a multiple of 4), as the
// plain 16-bit row kernels: every population plane and every reference plane
// of a source row is one aligned 64-bit (populations) or 128-bit (reference)
// load, plus the values at x0 - 1 and x0 + 4; e of a source node is formed
// once per row position, in packed pairs, with the same operations as
// lref_e_of (so decode and encode agree to the bit).  Next to a wall: the
// general per-node pull.
template <int NR>
struct RowRef {
    float r[NR][6];  // [plane][x0 - 1 .. x0 + 4] of one source row
};
template <int NR>
struct OwnRef {
    float r[NR][4];  // [plane][x0 .. x0 + 3]: the four nodes' own reference
};
template <int NR>
__device__ __forceinline__ void load_rowref(const LrefK &R, int base, int xm, int xp, RowRef<NR> &Rr)
{
#pragma unroll
    for (int p = 0; p < NR; p++) {
        const float *b = R.ref + p * R.Np + base;
        const float4 v = __ldg(reinterpret_cast<const float4 *>(b));
        Rr.r[p][0] = __ldg(b + xm);
        Rr.r[p][1] = v.x;
        Rr.r[p][2] = v.y;
        Rr.r[p][3] = v.z;
        Rr.r[p][4] = v.w;
        Rr.r[p][5] = __ldg(b + xp);
    }
}
// e_a from the reference values of two positions (packed), the same
// operations as lref_e_of
template <class L>
__device__ __forceinline__ f2 lref_e2v(const LrefK &R, int a, f2 r0, f2 r1, f2 r2)
{
    if constexpr (L::Q == 9) {
        const f2 c = vfma(f2((float)LD2Q9::ex(a)), r1, f2((float)LD2Q9::ey(a)) * r2);
        const f2 q = vfma(f2(4.5f) * c, c, f2(-1.5f) * vfma(r1, r1, r2 * r2));
        return f2((float)LD2Q9::w(a)) * vfma(f2(3.0f), c, r0 + q);
    } else {
        return f2(R.q5[a]) * r0;
    }
}
template <class L, int NR>
__device__ __forceinline__ f2 lref_e2(const LrefK &R, const RowRef<NR> &Rr, int a, int k)
{
    const f2 r0(Rr.r[0][k], Rr.r[0][k + 1]);
    if constexpr (NR == 3)
        return lref_e2v<L>(R, a, r0, f2(Rr.r[1][k], Rr.r[1][k + 1]), f2(Rr.r[2][k], Rr.r[2][k + 1]));
    else
        return lref_e2v<L>(R, a, r0, f2(0.f), f2(0.f));
}
// The pulled and decoded deviations of four consecutive nodes (see above);
// source row by source row, so that one row's reference is live at a time;
// the centre row's reference is kept for the encode.
template <class L, class T>
__device__ __forceinline__ void lref_pull_quad(const Planes<T, L::Q> &P, const Geom &g, const LrefK &R, int x0, int y,
                                               int i0, float sinv, f2 (&dA)[L::Q], f2 (&dB)[L::Q],
                                               OwnRef<(L::Q == 9 ? 3 : 1)> &Own, bool &interior)
{
    constexpr int NR = L::Q == 9 ? 3 : 1;
    const bool wall_x = g.wall[0] && (x0 == 0 || x0 + 3 == g.nx - 1);
    const bool wall_y = g.wall[1] && (y == 0 || y == g.ny - 1);
    interior = !(wall_x || wall_y);
    if (interior) {
        const int sy = g.nx;
        const int ym = y == 0 ? (g.ny - 1) * sy : -sy, yp = y == g.ny - 1 ? (1 - g.ny) * sy : sy;
        const int xm = x0 == 0 ? g.nx - 1 : -1;
        const int xp = x0 + 4 == g.nx ? 4 - g.nx : 4;
        const f2 si(sinv);
        const int roffs[3] = {ym, 0, yp};  // source rows of e_y = +1, 0, -1
        // the stored pair values of population a (pulled from row offset roff)
        auto pulled = [&](int a, int roff, f2 &sA, f2 &sB) {
            const int ex = L::ex(a);
            const T *pl = P.in[a] + i0 + roff;
            float wv[4];
            get4<T>(pl, wv);
            if (ex == 0) {
                sA = f2(wv[0], wv[1]);
                sB = f2(wv[2], wv[3]);
            } else if (ex == 1) {
                sA = f2(Dev<T>::get(pl + xm), wv[0]);
                sB = f2(wv[1], wv[2]);
            } else {
                sA = f2(wv[1], wv[2]);
                sB = f2(wv[3], Dev<T>::get(pl + xp));
            }
        };
        if constexpr (NR == 1) {
            // one reference plane: every row's reference loaded first, populations in order
            RowRef<NR> Rr[3];
#pragma unroll
            for (int r = 0; r < 3; r++) load_rowref<NR>(R, i0 + roffs[r], xm, xp, Rr[r]);
#pragma unroll
            for (int j = 0; j < 4; j++) Own.r[0][j] = Rr[1].r[0][j + 1];
#pragma unroll
            for (int a = 0; a < L::Q; a++) {
                const int ex = L::ex(a), r = 1 - L::ey(a);
                f2 sA, sB;
                pulled(a, roffs[r], sA, sB);
                // source positions of nodes x0 + j: row index 1 + j - e_x (0 = x0 - 1)
                dA[a] = vfma(sA, si, lref_e2<L, NR>(R, Rr[r], a, 1 - ex));
                dB[a] = vfma(sB, si, lref_e2<L, NR>(R, Rr[r], a, 3 - ex));
            }
        } else {
            // three reference planes: one source row at a time (fewer registers)
#pragma unroll
            for (int r = 0; r < 3; r++) {
                RowRef<NR> Rr;
                load_rowref<NR>(R, i0 + roffs[r], xm, xp, Rr);
                if (r == 1)
#pragma unroll
                    for (int p = 0; p < NR; p++)
#pragma unroll
                        for (int j = 0; j < 4; j++) Own.r[p][j] = Rr.r[p][j + 1];
#pragma unroll
                for (int a = 0; a < L::Q; a++) {
                    if (L::ey(a) != 1 - r) continue;
                    const int ex = L::ex(a);
                    f2 sA, sB;
                    pulled(a, roffs[r], sA, sB);
                    dA[a] = vfma(sA, si, lref_e2<L, NR>(R, Rr, a, 1 - ex));
                    dB[a] = vfma(sB, si, lref_e2<L, NR>(R, Rr, a, 3 - ex));
                }
            }
        }
        return;
    }
    float d[4][L::Q];
#pragma unroll
    for (int j = 0; j < 4; j++)
        pull_node<L>(g, x0 + j, y, 0, i0 + j, d[j],
                     [&](int p, int k) { return lref_dec<L, T>(R, P.in[p], p, k, sinv); });
#pragma unroll
    for (int a = 0; a < L::Q; a++) {
        dA[a] = f2(d[0][a], d[1][a]);
        dB[a] = f2(d[2][a], d[3][a]);
    }
}
// sigma (d - e) of the four nodes themselves, in place
template <class L, class T>
__device__ __forceinline__ void lref_encode_quad(const LrefK &R, const OwnRef<(L::Q == 9 ? 3 : 1)> &Own,
                                                 bool interior, int i0, float sig, f2 (&dA)[L::Q], f2 (&dB)[L::Q])
{
    constexpr int NR = L::Q == 9 ? 3 : 1;
    const f2 sg(sig);
#pragma unroll
    for (int a = 0; a < L::Q; a++) {
        f2 eA, eB;
        if (interior) {
            const f2 z(0.f);
            eA = lref_e2v<L>(R, a, f2(Own.r[0][0], Own.r[0][1]), NR == 3 ? f2(Own.r[1 % NR][0], Own.r[1 % NR][1]) : z,
                             NR == 3 ? f2(Own.r[2 % NR][0], Own.r[2 % NR][1]) : z);
            eB = lref_e2v<L>(R, a, f2(Own.r[0][2], Own.r[0][3]), NR == 3 ? f2(Own.r[1 % NR][2], Own.r[1 % NR][3]) : z,
                             NR == 3 ? f2(Own.r[2 % NR][2], Own.r[2 % NR][3]) : z);
        } else {
            eA = f2(lref_e<L>(R, a, i0), lref_e<L>(R, a, i0 + 1));
            eB = f2(lref_e<L>(R, a, i0 + 2), lref_e<L>(R, a, i0 + 3));
        }
        dA[a] = (dA[a] - eA) * sg;
        dB[a] = (dB[a] - eB) * sg;
    }
}

#ifndef LBM_LREF9X4_MIN_BLOCKS
#define LBM_LREF9X4_MIN_BLOCKS 1
#endif
template <class T, int FK, bool SR>
__global__ void __launch_bounds__(kBlock, LBM_LREF9X4_MIN_BLOCKS)
k_lref_step9x4(const __grid_constant__ Planes<T, 9> P, Geom g, FieldDev F, float apre, float gsum, Rates9f w,
               float rref, LrefK R, unsigned long long srkey)
{
    const int t = blockIdx.x * kBlock + threadIdx.x;
    if (t >= (g.N >> 2)) return;
    const int i0 = 4 * t;
    int x0, y;
    node_xy(g, i0, x0, y);
    const float sig = __ldg(R.scale), sinv = __ldg(R.scale + 1);
    f2 dA[9], dB[9];
    OwnRef<3> Own;
    bool interior;
    lref_pull_quad<LD2Q9, T>(P, g, R, x0, y, i0, sinv, dA, dB, Own, interior);
    f2 FxA(0.f), FyA(0.f), GxA(0.f), GyA(0.f), FxB(0.f), FyB(0.f), GxB(0.f), GyB(0.f);
    if (FK != FK_NONE) {
        float px[4], py[4];
        field_row_f<4>(F, FK, 0, x0, y, i0, px);
        field_row_f<4>(F, FK, 1, x0, y, i0, py);
        const f2 PxA(px[0], px[1]), PyA(py[0], py[1]), PxB(px[2], px[3]), PyB(py[2], py[3]);
        FxA = f2(apre) * PxA;
        FyA = f2(apre) * PyA;
        GxA = f2(gsum) * PxA;
        GyA = f2(gsum) * PyA;
        FxB = f2(apre) * PxB;
        FyB = f2(apre) * PyB;
        GxB = f2(gsum) * PxB;
        GyB = f2(gsum) * PyB;
    }
    collide9_w1<f2>(dA, rref, FxA, FyA, GxA, GyA, w);
    collide9_w1<f2>(dB, rref, FxB, FyB, GxB, GyB, w);
    lref_encode_quad<LD2Q9, T>(R, Own, interior, i0, sig, dA, dB);
    store_quad<T, SR, 9>(P.out, i0, dA, dB, srkey);
}

template <class T, int SK, bool SR>
__global__ void __launch_bounds__(kBlock)
k_lref_step5x4(const __grid_constant__ Planes<T, 5> P, Geom g, FieldDev S, float apre, float hsum, Coef5f k,
               Ref5f cref, LrefK R, unsigned long long srkey)
{
    const int t = blockIdx.x * kBlock + threadIdx.x;
    if (t >= (g.N >> 2)) return;
    const int i0 = 4 * t;
    int x0, y;
    node_xy(g, i0, x0, y);
    const float sig = __ldg(R.scale), sinv = __ldg(R.scale + 1);
    f2 dA[5], dB[5];
    OwnRef<1> Own;
    bool interior;
    lref_pull_quad<LD2Q5, T>(P, g, R, x0, y, i0, sinv, dA, dB, Own, interior);
    f2 SpA(0.f), H0A(0.f), SpB(0.f), H0B(0.f);
    if (SK != FK_NONE) {
        float ps[4];
        field_row_f<4>(S, SK, 0, x0, y, i0, ps);
        const f2 PA(ps[0], ps[1]), PB(ps[2], ps[3]);
        SpA = f2(apre) * PA;
        H0A = f2(hsum) * PA;
        SpB = f2(apre) * PB;
        H0B = f2(hsum) * PB;
    }
    collide5u<f2>(dA, 0.0f, SpA, H0A, k);
    collide5u<f2>(dB, 0.0f, SpB, H0B, k);
#pragma unroll
    for (int a = 0; a < 5; a++) {
        dA[a] = dA[a] + f2(cref.v[a]);
        dB[a] = dB[a] + f2(cref.v[a]);
    }
    lref_encode_quad<LD2Q5, T>(R, Own, interior, i0, sig, dA, dB);
    store_quad<T, SR, 5>(P.out, i0, dA, dB, srkey);
}

// Stored (s, reference, sigma) -> FP32 deviations d, both in the stored [q][Np] layout.
template <class L, class T>
__global__ void __launch_bounds__(kBlock)
k_lref_decode(const T *__restrict__ st, Geom g, LrefK R, float *__restrict__ dev)
{
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    const float sinv = __ldg(R.scale + 1);
#pragma unroll
    for (int a = 0; a < L::Q; a++) dev[a * g.Np + i] = lref_dec<L, T>(R, st + a * g.Np, a, i, sinv);
}

// The block's largest m into bmax[blockIdx.x].
__device__ __forceinline__ void block_max_to(float m, float *bmax)
{
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float wm[kBlock / 32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = 0.0f;
        for (int k = 0; k < kBlock / 32; k++) b = fmaxf(b, wm[k]);
        bmax[blockIdx.x] = b;
    }
}

// New reference from FP32 deviations (the node's own zeroth and first
// moments: then e has the same moments as d) and each block's largest |d - e|.
template <class L>
__global__ void __launch_bounds__(kBlock)
k_lref_reference(const float *__restrict__ dev, Geom g, LrefK R, float *__restrict__ ref, float *__restrict__ bmax)
{
    const int i = blockIdx.x * kBlock + threadIdx.x;
    float m = 0.0f;
    if (i < g.N) {
        float d[L::Q];
        float r0 = 0.f, r1 = 0.f, r2 = 0.f;
#pragma unroll
        for (int a = 0; a < L::Q; a++) {
            d[a] = dev[a * g.Np + i];
            r0 += d[a];
            if constexpr (L::Q == 9) {
                r1 += (float)L::ex(a) * d[a];
                r2 += (float)L::ey(a) * d[a];
            }
        }
        ref[i] = r0;
        if constexpr (L::Q == 9) {
            ref[g.Np + i] = r1;
            ref[2 * g.Np + i] = r2;
        }
#pragma unroll
        for (int a = 0; a < L::Q; a++) m = fmaxf(m, fabsf(d[a] - lref_e_of<L>(R, a, r0, r1, r2)));
    }
    block_max_to(m, bmax);
}

__device__ __forceinline__ float plain_val(const __half *p) { return __half2float(*p); }
__device__ __forceinline__ float plain_val(const __nv_bfloat16 *p) { return __bfloat162float(*p); }

// The rebuild without an FP32 copy of the state, in two passes over the
// stored values: the new reference (the node's own moments of its decoded
// deviations, into the second reference buffer) with the per-block largest
// |d - e_new|, then, once sigma_new is known, every value decoded at the old
// reference and sigma and stored at the new ones, in place (each thread
// touches its own node only).  Old and new may differ in q5 too (a D2Q5
// velocity change).
template <class L, class T>
__global__ void __launch_bounds__(kBlock)
k_lref_newref(const T *__restrict__ st, Geom g, LrefK Ro, LrefK Rn, float *__restrict__ ref_new,
              float *__restrict__ bmax)
{
    const float sinv = __ldg(Ro.scale + 1);
    const int i = blockIdx.x * kBlock + threadIdx.x;
    float m = 0.0f;
    if (i < g.N) {
        float d[L::Q];
        float r0 = 0.f, r1 = 0.f, r2 = 0.f;
#pragma unroll
        for (int a = 0; a < L::Q; a++) {
            d[a] = lref_dec<L, T>(Ro, st + a * g.Np, a, i, sinv);
            r0 += d[a];
            if constexpr (L::Q == 9) {
                r1 += (float)L::ex(a) * d[a];
                r2 += (float)L::ey(a) * d[a];
            }
        }
        ref_new[i] = r0;
        if constexpr (L::Q == 9) {
            ref_new[g.Np + i] = r1;
            ref_new[2 * g.Np + i] = r2;
        }
#pragma unroll
        for (int a = 0; a < L::Q; a++) m = fmaxf(m, fabsf(d[a] - lref_e_of<L>(Rn, a, r0, r1, r2)));
    }
    block_max_to(m, bmax);
}

template <class L, class T>
__global__ void __launch_bounds__(kBlock)
k_lref_reencode(T *__restrict__ st, Geom g, LrefK Ro, LrefK Rn)
{
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    const float sinv = __ldg(Ro.scale + 1), sig = __ldg(Rn.scale);
#pragma unroll
    for (int a = 0; a < L::Q; a++) {
        // plain loads: this kernel writes the values it reads
        const float sv = plain_val(st + a * g.Np + i);
        const float d = fmaf(sv, sinv, lref_e<L>(Ro, a, i));
        st[a * g.Np + i] = Dev<T>::to_store(lref_enc<L>(Rn, d, a, i, sig));
    }
}

// sigma = 2^k with the lattice's largest |d - e| (the largest of the nb block
// maxima) times sigma in [8, 16) (k clamped to [-30, 30]; 1 for an exactly
// uniform state).
constexpr int kScaleThreads = 1024;
__global__ void __launch_bounds__(kScaleThreads) k_lref_scale(const float *__restrict__ bmax, int nb,
                                                              float *__restrict__ scale)
{
    float m = 0.0f;
    for (int k = threadIdx.x; k < nb; k += kScaleThreads) m = fmaxf(m, bmax[k]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    __shared__ float wm[kScaleThreads / 32];
    if ((threadIdx.x & 31) == 0) wm[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 0; k < kScaleThreads / 32; k++) m = fmaxf(m, wm[k]);
        int e = 0;
        int k = 0;
        if (m > 0.0f && isfinite(m)) {
            frexpf(m, &e);  // m in [2^(e-1), 2^e)
            k = min(30, max(-30, 4 - e));
        }
        scale[0] = ldexpf(1.0f, k);
        scale[1] = ldexpf(1.0f, -k);
    }
}

// FP32 deviations -> stored s = sigma (d - e), rounded to nearest.
template <class L, class T>
__global__ void __launch_bounds__(kBlock)
k_lref_encode(const float *__restrict__ dev, Geom g, LrefK R, T *__restrict__ st)
{
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    const float sig = __ldg(R.scale);
#pragma unroll
    for (int a = 0; a < L::Q; a++)
        st[a * g.Np + i] = Dev<T>::to_store(lref_enc<L>(R, dev[a * g.Np + i], a, i, sig));
}

// The plain 16-bit deviations as this encoding: reference 0, sigma 1.
template <class L>
__global__ void __launch_bounds__(kBlock) k_lref_reset(Geom g, float *__restrict__ ref, float *__restrict__ scale)
{
    const int i = blockIdx.x * kBlock + threadIdx.x;
    if (i == 0) {
        scale[0] = 1.0f;
        scale[1] = 1.0f;
    }
    if (i >= g.N) return;
#pragma unroll
    for (int p = 0; p < (L::Q == 9 ? 3 : 1); p++) ref[p * g.Np + i] = 0.0f;
}

template <class T, bool SR>
cudaError_t lref_step_ts(int lattice, const LaunchArgs &a, const LrefK &R)
{
    const int grid = (a.g.N + kBlock - 1) / kBlock;
    const float rref = (float)a.rho_ref;
    const cudaStream_t s = a.stream;
    const unsigned long long key = a.srkey;
    if (lattice == LD2Q9::ID) {
        const Planes<T, 9> P = make_planes<T, 9>(a.fin, a.fout, a.g.Np);
        const Rates9f w{(float)(a.omega[3] / 12.0), (float)(a.omega[4] / 4.0), (float)(a.omega[5] / 4.0),
                        (float)(a.omega[6] / 4.0), (float)(a.omega[7] / 4.0), (float)(a.omega[8] / 4.0)};
        const float gsum = (float)((a.apre + a.apost) / 12.0), apre = (float)a.apre;
        const bool w1 = a.omega[6] == 1.0 && a.omega[7] == 1.0 && a.omega[8] == 1.0;
#define LREF9(FKV, W1V) k_lref_step9<T, FKV, W1V, SR><<<grid, kBlock, 0, s>>>(P, a.g, a.F, apre, gsum, w, rref, R, key)
#define LREF9X4(FKV) k_lref_step9x4<T, FKV, SR><<<qgrid, kBlock, 0, s>>>(P, a.g, a.F, apre, gsum, w, rref, R, key)
        const int qgrid = (a.g.N / 4 + kBlock - 1) / kBlock;
        if (w1 && a.g.nx % 4 == 0) {
            if (a.fkind == FK_NONE) LREF9X4(FK_NONE);
            else if (a.fkind == FK_CONST) LREF9X4(FK_CONST);
            else LREF9X4(FK_GENERAL);
        } else if (w1) {
            if (a.fkind == FK_NONE) LREF9(FK_NONE, true);
            else if (a.fkind == FK_CONST) LREF9(FK_CONST, true);
            else LREF9(FK_GENERAL, true);
        } else {
            if (a.fkind == FK_NONE) LREF9(FK_NONE, false);
            else if (a.fkind == FK_CONST) LREF9(FK_CONST, false);
            else LREF9(FK_GENERAL, false);
        }
#undef LREF9
#undef LREF9X4
    } else if (lattice == LD2Q5::ID) {
        if (a.vkind == FK_GENERAL) return cudaErrorInvalidValue;
        const double ux = a.vkind == FK_CONST ? a.V.cval[0] : 0.0, uy = a.vkind == FK_CONST ? a.V.cval[1] : 0.0;
        const Coef5f k = make_coef5f(a.omega, ux, uy);
        const float hsum = (float)((a.apre + a.apost) / 10.0), apre = (float)a.apre;
        Ref5f cref{};
        double c[5];
        d2q5_reference_change(a.omega, ux, uy, a.gref, c);
        for (int q = 0; q < 5; q++) cref.v[q] = (float)c[q];
        const Planes<T, 5> P = make_planes<T, 5>(a.fin, a.fout, a.g.Np);
        if (a.g.nx % 4 == 0) {
            const int qgrid = (a.g.N / 4 + kBlock - 1) / kBlock;
            if (a.fkind == FK_NONE)
                k_lref_step5x4<T, FK_NONE, SR><<<qgrid, kBlock, 0, s>>>(P, a.g, a.F, apre, hsum, k, cref, R, key);
            else if (a.fkind == FK_CONST)
                k_lref_step5x4<T, FK_CONST, SR><<<qgrid, kBlock, 0, s>>>(P, a.g, a.F, apre, hsum, k, cref, R, key);
            else k_lref_step5x4<T, FK_GENERAL, SR><<<qgrid, kBlock, 0, s>>>(P, a.g, a.F, apre, hsum, k, cref, R, key);
        } else if (a.fkind == FK_NONE)
            k_lref_step5<T, FK_NONE, SR><<<grid, kBlock, 0, s>>>(P, a.g, a.F, apre, hsum, k, cref, R, key);
        else if (a.fkind == FK_CONST)
            k_lref_step5<T, FK_CONST, SR><<<grid, kBlock, 0, s>>>(P, a.g, a.F, apre, hsum, k, cref, R, key);
        else k_lref_step5<T, FK_GENERAL, SR><<<grid, kBlock, 0, s>>>(P, a.g, a.F, apre, hsum, k, cref, R, key);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

LrefK lref_k(const Lref &L, const Geom &g)
{
    LrefK R;
    R.ref = L.ref;
    R.scale = L.scale;
    R.Np = g.Np;
    for (int q = 0; q < 5; q++) R.q5[q] = L.q5[q];
    return R;
}

template <class T>
cudaError_t lref_codec_t(int lattice, int encode, const Geom &g, const LrefK &R, float *ref, const void *stored_in,
                         void *stored_out, const float *dev_in, float *dev_out, cudaStream_t s)
{
    // encode: 0 decode, otherwise encode at the current reference and sigma
    const int grid = (g.N + kBlock - 1) / kBlock;
    if (lattice == LD2Q9::ID) {
        if (encode) k_lref_encode<LD2Q9, T><<<grid, kBlock, 0, s>>>(dev_in, g, R, static_cast<T *>(stored_out));
        else k_lref_decode<LD2Q9, T><<<grid, kBlock, 0, s>>>(static_cast<const T *>(stored_in), g, R, dev_out);
    } else if (lattice == LD2Q5::ID) {
        if (encode) k_lref_encode<LD2Q5, T><<<grid, kBlock, 0, s>>>(dev_in, g, R, static_cast<T *>(stored_out));
        else k_lref_decode<LD2Q5, T><<<grid, kBlock, 0, s>>>(static_cast<const T *>(stored_in), g, R, dev_out);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

void d2q5_batch_coef(const double omega[9], BatchItem &item);

void d2q5_step_matrix(const double omega[9], double ux, double uy, double M[25])
{
    BatchItem it{};
    it.vkind = FK_CONST;
    it.V.cval[0] = ux;
    it.V.cval[1] = uy;
    d2q5_batch_coef(omega, it);
    for (int k = 0; k < 25; k++) M[k] = it.mat[k];
}

void d2q5_reference_change(const double omega[9], double ux, double uy, const double g[5], double out[5])
{
    double M[25];
    d2q5_step_matrix(omega, ux, uy, M);
    for (int a = 0; a < 5; a++) {
        double acc = 0.0;
        for (int b = 0; b < 5; b++) acc += M[5 * a + b] * g[b];
        out[a] = acc - g[a];
    }
}

cudaError_t rp_step(int lattice, const LaunchArgs &a)
{
    switch (a.storage) {
    case 1: return step_t<float>(lattice, a);
    case 2: return step_t<__half>(lattice, a);
    case 3: return step_t<__nv_bfloat16>(lattice, a);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t rp_cluster_steps9(const LaunchArgs &a, int nsteps)
{
    switch (a.storage) {
    case 1: return cluster9_t<float>(a, nsteps);
    case 2: return cluster9_t<__half>(a, nsteps);
    case 3: return cluster9_t<__nv_bfloat16>(a, nsteps);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t rp_batch_step(int lattice, int storage, const BatchLaunch &L, int nblocks, int tile, cudaStream_t s)
{
    switch (storage) {
    case 1: return batch_t<float>(lattice, L, nblocks, tile, s);
    case 2: return batch_t<__half>(lattice, L, nblocks, tile, s);
    case 3: return batch_t<__nv_bfloat16>(lattice, L, nblocks, tile, s);
    default: return cudaErrorInvalidValue;
    }
}

int rp_batch_resident(int lattice, int storage, int tile)
{
    switch (storage) {
    case 1: return resident_t<float>(lattice, tile);
    case 2: return resident_t<__half>(lattice, tile);
    case 3: return resident_t<__nv_bfloat16>(lattice, tile);
    default: return 0;
    }
}

cudaError_t lref_step(int lattice, const LaunchArgs &a, const Lref &L)
{
    const LrefK R = lref_k(L, a.g);
    if (a.storage == 2) return a.sround ? lref_step_ts<__half, true>(lattice, a, R) : lref_step_ts<__half, false>(lattice, a, R);
    if (a.storage == 3)
        return a.sround ? lref_step_ts<__nv_bfloat16, true>(lattice, a, R) : lref_step_ts<__nv_bfloat16, false>(lattice, a, R);
    return cudaErrorInvalidValue;
}

cudaError_t lref_decode(int lattice, int storage, const Geom &g, const Lref &L, const void *stored, float *dev,
                        cudaStream_t s)
{
    const LrefK R = lref_k(L, g);
    if (storage == 2) return lref_codec_t<__half>(lattice, 0, g, R, L.ref, stored, nullptr, nullptr, dev, s);
    if (storage == 3) return lref_codec_t<__nv_bfloat16>(lattice, 0, g, R, L.ref, stored, nullptr, nullptr, dev, s);
    return cudaErrorInvalidValue;
}

cudaError_t lref_encode(int lattice, int storage, const Geom &g, const Lref &L, const float *dev, void *stored,
                        cudaStream_t s)
{
    const LrefK R = lref_k(L, g);
    if (storage == 2) return lref_codec_t<__half>(lattice, 1, g, R, L.ref, nullptr, stored, dev, nullptr, s);
    if (storage == 3) return lref_codec_t<__nv_bfloat16>(lattice, 1, g, R, L.ref, nullptr, stored, dev, nullptr, s);
    return cudaErrorInvalidValue;
}

cudaError_t lref_reset(int lattice, const Geom &g, const Lref &L, cudaStream_t s)
{
    const int grid = std::max(1, (g.N + kBlock - 1) / kBlock);
    if (lattice == LD2Q9::ID) k_lref_reset<LD2Q9><<<grid, kBlock, 0, s>>>(g, L.ref, L.scale);
    else if (lattice == LD2Q5::ID) k_lref_reset<LD2Q5><<<grid, kBlock, 0, s>>>(g, L.ref, L.scale);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

template <class T>
cudaError_t lref_rebuild_t(int lattice, const Geom &g, const LrefK &Ro, const LrefK &Rn, float *ref_new,
                           float *scale_new, float *bmax, void *stored, cudaStream_t s)
{
    const int grid = (g.N + kBlock - 1) / kBlock;
    T *st = static_cast<T *>(stored);
    if (lattice == LD2Q9::ID) {
        k_lref_newref<LD2Q9, T><<<grid, kBlock, 0, s>>>(st, g, Ro, Rn, ref_new, bmax);
        k_lref_scale<<<1, kScaleThreads, 0, s>>>(bmax, grid, scale_new);
        k_lref_reencode<LD2Q9, T><<<grid, kBlock, 0, s>>>(st, g, Ro, Rn);
    } else if (lattice == LD2Q5::ID) {
        k_lref_newref<LD2Q5, T><<<grid, kBlock, 0, s>>>(st, g, Ro, Rn, ref_new, bmax);
        k_lref_scale<<<1, kScaleThreads, 0, s>>>(bmax, grid, scale_new);
        k_lref_reencode<LD2Q5, T><<<grid, kBlock, 0, s>>>(st, g, Ro, Rn);
    } else {
        return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

cudaError_t lref_reencode(int lattice, int storage, const Geom &g, const Lref &Lold, const Lref &Lnew, void *stored,
                          cudaStream_t s)
{
    const LrefK Ro = lref_k(Lold, g), Rn = lref_k(Lnew, g);
    const int grid = (g.N + kBlock - 1) / kBlock;
    if (lattice == LD2Q9::ID && storage == 2)
        k_lref_reencode<LD2Q9, __half><<<grid, kBlock, 0, s>>>(static_cast<__half *>(stored), g, Ro, Rn);
    else if (lattice == LD2Q9::ID && storage == 3)
        k_lref_reencode<LD2Q9, __nv_bfloat16><<<grid, kBlock, 0, s>>>(static_cast<__nv_bfloat16 *>(stored), g, Ro, Rn);
    else if (lattice == LD2Q5::ID && storage == 2)
        k_lref_reencode<LD2Q5, __half><<<grid, kBlock, 0, s>>>(static_cast<__half *>(stored), g, Ro, Rn);
    else if (lattice == LD2Q5::ID && storage == 3)
        k_lref_reencode<LD2Q5, __nv_bfloat16><<<grid, kBlock, 0, s>>>(static_cast<__nv_bfloat16 *>(stored), g, Ro, Rn);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t lref_rebuild(int lattice, int storage, const Geom &g, const Lref &Lold, const Lref &Lnew, float *bmax,
                         void *stored, cudaStream_t s)
{
    const LrefK Ro = lref_k(Lold, g), Rn = lref_k(Lnew, g);
    if (storage == 2) return lref_rebuild_t<__half>(lattice, g, Ro, Rn, Lnew.ref, Lnew.scale, bmax, stored, s);
    if (storage == 3) return lref_rebuild_t<__nv_bfloat16>(lattice, g, Ro, Rn, Lnew.ref, Lnew.scale, bmax, stored, s);
    return cudaErrorInvalidValue;
}

cudaError_t lref_rebase(int lattice, int storage, const Geom &g, const Lref &L, float *bmax, const float *dev,
                        void *stored, cudaStream_t s)
{
    if (lattice != LD2Q9::ID && lattice != LD2Q5::ID) return cudaErrorInvalidValue;
    const LrefK R = lref_k(L, g);
    const int grid = (g.N + kBlock - 1) / kBlock;
    if (lattice == LD2Q9::ID) k_lref_reference<LD2Q9><<<grid, kBlock, 0, s>>>(dev, g, R, L.ref, bmax);
    else k_lref_reference<LD2Q5><<<grid, kBlock, 0, s>>>(dev, g, R, L.ref, bmax);
    k_lref_scale<<<1, kScaleThreads, 0, s>>>(bmax, grid, L.scale);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (storage == 2) return lref_codec_t<__half>(lattice, 2, g, R, L.ref, nullptr, stored, dev, nullptr, s);
    if (storage == 3) return lref_codec_t<__nv_bfloat16>(lattice, 2, g, R, L.ref, nullptr, stored, dev, nullptr, s);
    return cudaErrorInvalidValue;
}

}  // namespace lbmk
