// D2Q9 cascaded LB step with Strang-split body force (arXiv:1806.10247 Sec. 4),
// FP64, one thread per node, pull form: each launch streams f^p(t-1) into
// f(t) (Eq. 22b, periodic wrap or halfway bounce-back), then applies the
// pre-collision half force (Eq. 25), the cascaded collision (Eq. 23), the
// post-collision half force (Eq. 31) and writes f^p(t) = f + K g (Eq. 32).
#include <cooperative_groups.h>

#include "lbm_internal.h"
#include "lbm_lattices.cuh"
#include "lbm_tiles.cuh"

namespace lbmk {
namespace {

constexpr int kBlock = 256;

struct Rates9 {
    double c3, c4, c5, c6, c7, c8;  // omega_3/12, omega_4/4, omega_5/4, omega_6/4, omega_7/4, omega_8/4
};

// Moments a collision forms on the way (for a fused readback): rho and the
// un-forced j of the pulled populations, summed as zeroth_first<LD2Q9> sums
// them, the half-forced j of Eq. 25 and 1/rho (__drcp_rn).
struct Mom9 {
    double rho, jx, jy, jfx, jfy, rinv;
};

// Post-collision populations of one node, in place.
//   Fx, Fy : pre-collision force a_pre P (Eq. 25)
//   Gx, Gy : first-moment coefficients g_1, g_2 = (F_pre + F_post)/12 (Eqs. 27-31)
__device__ __forceinline__ void collide(double (&f)[9], double Fx, double Fy, double Gx, double Gy,
                                        const Rates9 &w, Mom9 &mo)
{
    // Raw moments (Eq. 21) by 1D passes: x-moments of the three rows ey = 0,
    // +1, -1, then y-moments of those.
    const double s0 = f[1] + f[3], d0 = f[1] - f[3];  // row ey = 0
    const double s1 = f[5] + f[6], d1 = f[5] - f[6];  // row ey = +1
    const double s2 = f[8] + f[7], d2 = f[8] - f[7];  // row ey = -1
    const double A0 = f[0] + s0, B0 = f[2] + s1, C0 = f[4] + s2;
    const double rho = A0 + (B0 + C0), jy = B0 - C0, myy = B0 + C0;
    const double jx = d0 + (d1 + d2), mxy = d1 - d2, mxyy = d1 + d2;
    const double mxx = s0 + (s1 + s2), mxxy = s1 - s2, mxxyy = s1 + s2;

    // Eq. 25: velocity after the pre-collision half force step.
    const double rinv = __drcp_rn(rho);
    const double jfx = fma(0.5, Fx, jx), jfy = fma(0.5, Fy, jy);
    const double ux = jfx * rinv;
    const double uy = jfy * rinv;
    mo = Mom9{rho, jx, jy, jfx, jfy, rinv};
    const double ux2 = ux * ux, uy2 = uy * uy, uxy = ux * uy;

    // Eq. 23: cascaded change of moments.
    const double g3 = w.c3 * ((2.0 / 3.0) * rho + rho * (ux2 + uy2) - (mxx + myy));
    const double g4 = w.c4 * (rho * (ux2 - uy2) - (mxx - myy));
    const double g5 = w.c5 * (rho * uxy - mxy);
    const double p34 = 3.0 * g3 + g4, m34 = 3.0 * g3 - g4;
    const double g6 = w.c6 * (2.0 * rho * ux2 * uy + mxxy - 2.0 * ux * mxy - uy * mxx)
                      - 0.5 * uy * p34 - 2.0 * ux * g5;
    const double g7 = w.c7 * (2.0 * rho * ux * uy2 + mxyy - 2.0 * uy * mxy - ux * myy)
                      - 0.5 * ux * m34 - 2.0 * uy * g5;
    const double g8 = w.c8 * ((1.0 / 9.0) * rho + 3.0 * rho * ux2 * uy2
                              - (mxxyy - 2.0 * ux * mxyy - 2.0 * uy * mxxy + ux2 * myy + uy2 * mxx
                                 + 4.0 * uxy * mxy))
                      - 2.0 * g3 - 0.5 * uy2 * p34 - 0.5 * ux2 * m34 - 4.0 * uxy * g5
                      - 2.0 * uy * g6 - 2.0 * ux * g7;

    // Eq. 32 with g_0 = 0 and g_1, g_2 from Eq. 31.
    const double ax = g4 - g3, ay = -g3 - g4, c = 2.0 * g3 + g8;
    f[0] += -4.0 * (g3 - g8);
    f[1] += Gx + ax + 2.0 * (g7 - g8);
    f[2] += Gy + ay + 2.0 * (g6 - g8);
    f[3] += -Gx + ax - 2.0 * (g7 + g8);
    f[4] += -Gy + ay - 2.0 * (g6 + g8);
    f[5] += c + (Gx + Gy) + (g5 - g6 - g7);
    f[6] += c + (Gy - Gx) + (-g5 - g6 + g7);
    f[7] += c - (Gx + Gy) + (g5 + g6 + g7);
    f[8] += c + (Gx - Gy) + (-g5 + g6 - g7);
}

// The same step when omega_6 = omega_7 = omega_8 = 1 (the paper's choice for
// the higher moments, Sec. 6).  Eq. 23 is the relaxation of the central
// moments (trace towards 2 rho / 3 with omega_3, xx - yy and xy towards 0
// with omega_4, omega_5, each higher one towards its equilibrium value with
// its own rate); at unit rates the third- and fourth-order central moments
// land on 0 and rho / 9, so the post-collision populations follow from rho,
// u and the three relaxed second-order central moments.  They are built by
// the factorised back-shift and inverse transform on HALVED moments (each
// axis on which a moment has order 1 or 2 contributes a factor 1/2, so that
// the inverse 1D transform of (m0, m1/2, m2/2) is m2/2 - m1/2, m0 - m2,
// m2/2 + m1/2), with the post-collision force K_1 g_1, K_2 g_2 of Eq. 31
// added to the raw moments: e_x changes m_10 by 6 g_1 (of which F_pre / 2 is
// already in j) and m_12 by 4 g_1.  The first raw moments are carried as j
// itself (not rebuilt as rho (j / rho)), so the step transports momentum
// without a rounding of its own.  About 80 FP64 operations instead of 132.
// XO: the force has no y component (its terms, additions of 0, are left out).
template <bool XO = false>
__device__ __forceinline__ void collide_w1(double (&f)[9], double Fx, double Fy, double Gx, double Gy,
                                           const Rates9 &w, Mom9 &mo)
{
    // raw moments of order <= 2 per axis (Eq. 21)
    const double s0 = f[1] + f[3], d0 = f[1] - f[3];  // row ey = 0
    const double s1 = f[5] + f[6], d1 = f[5] - f[6];  // row ey = +1
    const double s2 = f[8] + f[7], d2 = f[8] - f[7];  // row ey = -1
    const double B0 = f[2] + s1, C0 = f[4] + s2;
    const double rho = (f[0] + s0) + (B0 + C0);
    const double jx0 = d0 + (d1 + d2), jy0 = B0 - C0;
    const double jx = fma(0.5, Fx, jx0), jy = XO ? jy0 : fma(0.5, Fy, jy0);  // Eq. 25
    const double mxx = s0 + (s1 + s2), myy = B0 + C0, mxy = d1 - d2;
    const double rinv = __drcp_rn(rho);
    const double ux = jx * rinv, uy = jy * rinv;
    mo = Mom9{rho, jx0, jy0, jx, jy, rinv};

    // second-order central moments, relaxed and halved (xx, yy by 1/2 ... of
    // the trace and difference: k_xx = (T + D) / 2 halved is (T + D) / 4)
    const double cxx = fma(-jx, ux, mxx), cyy = fma(-jy, uy, myy), cxy = fma(-jx, uy, mxy);
    const double T = cxx + cyy, D = cxx - cyy;
    const double Tq = fma(3.0 * w.c3, fma(2.0 / 3.0, rho, -T), 0.25 * T);  // (T + omega_3 (2 rho/3 - T)) / 4
    const double Dq = (0.25 - w.c4) * D;                                      // (1 - omega_4) D / 4
    const double kxx = Tq + Dq, kyy = Tq - Dq, kxy = (0.25 - w.c5) * cxy;    // kxy: (1 - omega_5) k_xy / 4
    const double k22 = rho * (1.0 / 36.0);                                    // rho / 9, quartered

    // back-shift along x of the lines of y-order 0, 1, 2: (rho, 0, kxx), (0, kxy, 0), (kyy, 0, k22)
    const double hx = 0.5 * ux, hy = 0.5 * uy;
    const double M10 = 0.5 * jx, M20 = fma(ux, M10, kxx);  // m_10 = rho u_x = j_x
    const double M11 = kxy, M21 = (kxy + kxy) * ux;
    const double M12 = hx * kyy, M22 = fma(ux, M12, k22);
    // back-shift along y of the lines of x-order 0, 1, 2
    double N00 = rho, N01 = 0.5 * jy, N02 = fma(uy, N01, kyy);  // m_01 = j_y
    double N10 = M10, N11 = fma(hy, M10, M11), N12 = fma(uy, M11 + N11, M12);
    double N20 = M20, N21 = fma(hy, M20, M21), N22 = fma(uy, M21 + N21, M22);
    // post-collision force (Eq. 31), halved: m_10 gains F_post / 2 = 6 Gx - Fx / 2, m_12 gains 4 Gx
    N10 = fma(3.0, Gx, fma(-0.25, Fx, N10));
    N12 += Gx;
    if constexpr (!XO) {
        N01 = fma(3.0, Gy, fma(-0.25, Fy, N01));
        N21 += Gy;
    }
    // inverse transform along y, then along x
    const double P0m = N02 - N01, P00 = fma(-2.0, N02, N00), P0p = N02 + N01;  // x-order 0; e_y = -1, 0, +1
    const double P1m = N12 - N11, P10 = fma(-2.0, N12, N10), P1p = N12 + N11;
    const double P2m = N22 - N21, P20 = fma(-2.0, N22, N20), P2p = N22 + N21;
    f[0] = fma(-2.0, P20, P00);
    f[1] = P20 + P10;
    f[3] = P20 - P10;
    f[2] = fma(-2.0, P2p, P0p);
    f[5] = P2p + P1p;
    f[6] = P2p - P1p;
    f[4] = fma(-2.0, P2m, P0m);
    f[8] = P2m + P1m;
    f[7] = P2m - P1m;
}

// XO (unit higher rates only): the force has no y component (checked on the host).
template <int FK, bool W1, bool XO>
__global__ void __launch_bounds__(kBlock)
k_step(const __grid_constant__ Planes<double, 9> P, Geom g, FieldDev F, double apre, double gsum, Rates9 w)
{
    int i = blockIdx.x * kBlock + threadIdx.x;
    if (i >= g.N) return;
    int x, y;
    node_xy(g, i, x, y);
    double f[9];
    load_pulled<LD2Q9>(P, g, x, y, 0, i, f);
    double Fx = 0.0, Fy = 0.0, Gx = 0.0, Gy = 0.0;
    if (FK != FK_NONE) {
        const double Px = field_value(F, FK, 0, x, y, 0, i);
        Fx = apre * Px;
        Gx = gsum * Px;
        if (!XO) {
            const double Py = field_value(F, FK, 1, x, y, 0, i);
            Fy = apre * Py;
            Gy = gsum * Py;
        }
    }
    Mom9 mo;
    if (W1) collide_w1<XO>(f, Fx, Fy, Gx, Gy, w, mo);
    else collide(f, Fx, Fy, Gx, Gy, w, mo);
#pragma unroll
    for (int a = 0; a < 9; a++) P.out[a][i] = f[a];
}

// ------------------------------------------------------------------------
// Many steps per launch for a small lattice (e.g. the 3 x 33 channel): the
// whole state lives in the distributed shared memory of one thread-block
// cluster.  Block b of the cluster owns nodes [b P, (b + 1) P) and keeps
// their post-collision populations twice (current and next step) in its
// shared memory; a pull from a node of another block reads that block's
// shared memory directly.  One cluster barrier per step separates the
// writes of a step from the reads of the next.  The per-node arithmetic is
// `collide` above, so the result equals n single-step launches up to the
// compiler's multiply-add contraction.
namespace cg = cooperative_groups;

constexpr int kClusterThreads = 384;  // >= 32-rounded 341, the largest block (48 KB of shared memory)

template <int FK, bool W1>
__global__ void __launch_bounds__(kClusterThreads)
k_cluster_steps(const double *__restrict__ fin, double *__restrict__ fout, Geom g, FieldDev F, double apre,
                double gsum, Rates9 w, int P, int nsteps)
{
    extern __shared__ double sm[];  // [2][9][P]
    cg::cluster_group cl = cg::this_cluster();
    const int b = (int)cl.block_rank();
    const int l = threadIdx.x;
    const int i = b * P + l;
    const bool own = l < P && i < g.N;
    if (own)
#pragma unroll
        for (int a = 0; a < 9; a++) sm[a * P + l] = fin[a * g.Np + i];
    const int x = own ? i % g.nx : 0, y = own ? i / g.nx : 0;
    double Fx = 0.0, Fy = 0.0, Gx = 0.0, Gy = 0.0;
    if (FK != FK_NONE && own) {
        const double Px = field_value(F, FK, 0, x, y, 0, i), Py = field_value(F, FK, 1, x, y, 0, i);
        Fx = apre * Px;
        Fy = apre * Py;
        Gx = gsum * Px;
        Gy = gsum * Py;
    }
    // pull sources of this node: owner block, offset inside its buffer
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
            double f[9];
#pragma unroll
            for (int a = 0; a < 9; a++) {
                const double *base = cl.map_shared_rank(sm + cur * 9 * P, src_blk[a]);
                f[a] = base[src_off[a]];
            }
            Mom9 mo;
            if (W1) collide_w1(f, Fx, Fy, Gx, Gy, w, mo);
            else collide(f, Fx, Fy, Gx, Gy, w, mo);
            double *nxt = sm + (cur ^ 1) * 9 * P;
#pragma unroll
            for (int a = 0; a < 9; a++) nxt[a * P + l] = f[a];
        }
        cur ^= 1;
        cl.sync();
    }
    if (own)
#pragma unroll
        for (int a = 0; a < 9; a++) fout[a * g.Np + i] = sm[cur * 9 * P + a * P + l];
}

// Batched form: one launch for every lattice of a batch; pairs hold
// (a_pre, (a_pre + a_post)/12) per step and item.
// One node of a batched launch (member `it`, node i; B staged in shared memory).
__device__ __forceinline__ void batch_node(const BatchItem &B, const BatchLaunch &L, int it, int i)
{
    const Geom &g = B.g;
    const int p = B.parity + L.parity;
    const double *fin = B.buf[p & 1];
    double *fout = B.buf[(p + 1) & 1];
    const double2 ap = L.pairs ? L.pairs[(size_t)L.k * L.count + it] : L.inl[it];
    int x, y;
    node_xy(g, i, x, y);
    double f[9];
    load_pulled<LD2Q9>(fin, g, x, y, 0, i, f);
    double Fx = 0.0, Fy = 0.0, Gx = 0.0, Gy = 0.0;
    const int fk = B.fkind;
    if (fk != FK_NONE) {
        const double Px = field_value(B.F, fk, 0, x, y, 0, i), Py = field_value(B.F, fk, 1, x, y, 0, i);
        Fx = ap.x * Px;
        Fy = ap.x * Py;
        Gx = ap.y * Px;
        Gy = ap.y * Py;
    }
    const Rates9 w{B.coef[0], B.coef[1], B.coef[2], B.coef[3], B.coef[4], B.coef[5]};
    Mom9 mo;
    if (B.variant == 3) collide_w1<true>(f, Fx, Fy, Gx, Gy, w, mo);  // uniform over the member
    else if (B.variant == 1) collide_w1<false>(f, Fx, Fy, Gx, Gy, w, mo);
    else collide(f, Fx, Fy, Gx, Gy, w, mo);
    if (L.mrho) {
        // fused readback of f(t)'s fields from the collision's own moments;
        // the same bits as store_fields (Fx = a_pre P, so fma(0.5, Fx, j) is
        // j + (a_pre P)/2 rounded once)
        const bool forced = L.mhalf && fk != FK_NONE;
        const double jd[3] = {forced ? mo.jfx : mo.jx, forced ? mo.jfy : mo.jy, 0.0};
        put_fields<LD2Q9>(mo.rho, jd, mo.rinv, i, g.N, __ldg(L.moff + it), L.mrho, L.mu);
    }
#pragma unroll
    for (int a = 0; a < 9; a++) fout[a * g.Np + i] = f[a];
}

template <int TB, int MODE>
__global__ void __launch_bounds__(TB)
k_batch(const __grid_constant__ BatchLaunch L)
{
    batch_tiles<TB, MODE>(L, [](const BatchItem &B, const BatchLaunch &L2, int it, int i) { batch_node(B, L2, it, i); });
}

template <bool W1>
cudaError_t cluster_launch(cudaLaunchConfig_t &cfg, int C, const LaunchArgs &a, double gsum, const Rates9 &w, int P,
                           int nsteps)
{
    switch (a.fkind) {
    case FK_NONE:
        if (C > 8) cudaFuncSetAttribute(k_cluster_steps<FK_NONE, W1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        return cudaLaunchKernelEx(&cfg, k_cluster_steps<FK_NONE, W1>, a.fin, a.fout, a.g, a.F, a.apre, gsum, w, P,
                                  nsteps);
    case FK_CONST:
        if (C > 8) cudaFuncSetAttribute(k_cluster_steps<FK_CONST, W1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        return cudaLaunchKernelEx(&cfg, k_cluster_steps<FK_CONST, W1>, a.fin, a.fout, a.g, a.F, a.apre, gsum, w, P,
                                  nsteps);
    default:
        if (C > 8)
            cudaFuncSetAttribute(k_cluster_steps<FK_GENERAL, W1>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        return cudaLaunchKernelEx(&cfg, k_cluster_steps<FK_GENERAL, W1>, a.fin, a.fout, a.g, a.F, a.apre, gsum, w,
                                  P, nsteps);
    }
}

template <bool W1>
void step_launch(const LaunchArgs &a, int grid, double gsum, const Rates9 &w)
{
    const Planes<double, 9> P = make_planes<double, 9>(a.fin, a.fout, a.g.Np);
    const bool xo = W1 && force_x_only(a.fkind, a.F, 2);
    switch (a.fkind) {
    case FK_NONE: k_step<FK_NONE, W1, false><<<grid, kBlock, 0, a.stream>>>(P, a.g, a.F, a.apre, gsum, w); break;
    case FK_CONST:
        if (xo) k_step<FK_CONST, W1, W1><<<grid, kBlock, 0, a.stream>>>(P, a.g, a.F, a.apre, gsum, w);
        else k_step<FK_CONST, W1, false><<<grid, kBlock, 0, a.stream>>>(P, a.g, a.F, a.apre, gsum, w);
        break;
    default:
        if (xo) k_step<FK_GENERAL, W1, W1><<<grid, kBlock, 0, a.stream>>>(P, a.g, a.F, a.apre, gsum, w);
        else k_step<FK_GENERAL, W1, false><<<grid, kBlock, 0, a.stream>>>(P, a.g, a.F, a.apre, gsum, w);
        break;
    }
}

}  // namespace

// omega_6 = omega_7 = omega_8 = 1: the step takes collide_w1.
bool d2q9_high_rates_one(const double omega[9])
{
    return omega[6] == 1.0 && omega[7] == 1.0 && omega[8] == 1.0;
}

void d2q9_batch_coef(const double omega[9], BatchItem &item)
{
    const double c[6] = {omega[3] / 12.0, omega[4] / 4.0, omega[5] / 4.0,
                         omega[6] / 4.0, omega[7] / 4.0, omega[8] / 4.0};
    for (int k = 0; k < 6; k++) item.coef[k] = c[k];
}

cudaError_t d2q9_batch_step(const BatchLaunch &L, int nblocks, int tile, cudaStream_t s)
{
    LBM_TILED_LAUNCH(k_batch, L, nblocks, tile, s);
}

int d2q9_batch_resident(int tile)
{
    LBM_TILED_RESIDENT(k_batch, tile);
}

// Cluster form for small lattices with a constant envelope; returns
// cudaErrorNotSupported when the lattice does not fit (the caller then steps
// with single launches).
cudaError_t d2q9_cluster_steps(const LaunchArgs &a, int nsteps)
{
    // about 8 nodes per block (the FP64 work of a step spread over up to 16 SMs)
    const int C = a.g.N >= 16 * 8 ? 16 : (a.g.N + 7) / 8;
    const int P = (a.g.N + C - 1) / C;
    const int threads = (P + 31) / 32 * 32;
    const size_t smem = (size_t)2 * 9 * P * sizeof(double);
    if (threads > kClusterThreads || smem > 48 * 1024) return cudaErrorNotSupported;
    Rates9 w{a.omega[3] / 12.0, a.omega[4] / 4.0, a.omega[5] / 4.0,
             a.omega[6] / 4.0, a.omega[7] / 4.0, a.omega[8] / 4.0};
    const double gsum = (a.apre + a.apost) / 12.0;
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
    return d2q9_high_rates_one(a.omega) ? cluster_launch<true>(cfg, C, a, gsum, w, P, nsteps)
                                        : cluster_launch<false>(cfg, C, a, gsum, w, P, nsteps);
}

cudaError_t d2q9_step(const LaunchArgs &a)
{
    Rates9 w{a.omega[3] / 12.0, a.omega[4] / 4.0, a.omega[5] / 4.0,
             a.omega[6] / 4.0, a.omega[7] / 4.0, a.omega[8] / 4.0};
    const double gsum = (a.apre + a.apost) / 12.0;
    const int grid = (a.g.N + kBlock - 1) / kBlock;
    if (d2q9_high_rates_one(a.omega)) step_launch<true>(a, grid, gsum, w);
    else step_launch<false>(a, grid, gsum, w);
    return cudaGetLastError();
}

}  // namespace lbmk
