// Device-side building blocks shared by the lattice kernels: grid geometry
// and evaluation of force / source / velocity shapes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace lbmk {

// Lattice geometry.  Populations are stored as planes of Np doubles (Np = N
// rounded up to a multiple of 32, so that every plane starts on a 256-byte
// boundary); node (x, y, z) sits at offset x + nx*(y + ny*z) in each plane.
struct Geom {
    int nx, ny, nz;
    int N;          // nodes (validated < 2^31 on the host)
    long long Np;   // plane stride in doubles
    int wall[3];    // 1 = halfway bounce-back walls on that axis, 0 = periodic
    // n / nx and n / ny for 0 <= n < 2^31 by multiply-high (see div_invariant)
    unsigned mx, my;
    int lx, ly;
};

// Quotient n / d of 0 <= n < 2^31 by an invariant divisor 1 <= d < 2^31,
// after Granlund and Montgomery, "Division by invariant integers using
// multiplication" (PLDI 1994), round-up method: with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, n / d = (umulhi(m, n) + n) >> l.  The sum
// stays below 2^32 because umulhi(m, n) < n < 2^31.
__device__ __forceinline__ int div_invariant(int n, unsigned m, int l)
{
    return (int)((__umulhi(m, (unsigned)n) + (unsigned)n) >> l);
}

// The (m, l) pair of div_invariant for divisor d (host side).
inline void div_magic(int d, unsigned &m, int &l)
{
    l = 0;
    while ((1LL << l) < (long long)d) l++;
    m = (unsigned)(((unsigned long long)((1LL << l) - d) << 32) / (unsigned long long)d + 1ULL);
}

// Kinds of a force / source / velocity shape as seen by a kernel.
enum FieldKind { FK_NONE = 0, FK_CONST = 1, FK_GENERAL = 2 };

// A shape on the device.  CONST: per-component values in cval.  GENERAL:
// either separable tables (sep = 1: for component c, px at data + c*cstride,
// then py, then pz, with lengths len[0..2], 1 meaning constant on that axis)
// or a full field (sep = 0: data[c*cstride + node]).
// zmask: bit c set = component c is identically zero.  axes (separable only):
// bit d set = the axis-d table takes part in the product; a table that is the
// single value 1.0 for every non-zero component is left out (multiplying by
// 1.0 is exact, so the value is unchanged).
struct FieldDev {
    const double *data;
    const float *fdata;  // FP32 copy of data (reduced-precision contexts only)
    long long cstride;
    int len[3];
    int sep;
    int zmask;
    int axes;
    double cval[3];
    float fcval[3];
};

__device__ __forceinline__ double field_value(const FieldDev &F, int kind, int c, int x, int y, int z,
                                              int node)
{
    if (kind == FK_CONST) return F.cval[c];
    if ((F.zmask >> c) & 1) return 0.0;
    const double *t = F.data + c * F.cstride;
    if (!F.sep) return __ldg(t + node);
    // (px * py) * pz, the documented evaluation order, skipping exact-1 tables
    double v = 1.0;
    bool have = false;
    if (F.axes & 1) {
        v = __ldg(t + (F.len[0] > 1 ? x : 0));
        have = true;
    }
    if (F.axes & 2) {
        const double py = __ldg(t + F.len[0] + (F.len[1] > 1 ? y : 0));
        v = have ? v * py : py;
        have = true;
    }
    if (F.axes & 4) {
        const double pz = __ldg(t + F.len[0] + F.len[1] + (F.len[2] > 1 ? z : 0));
        v = have ? v * pz : pz;
    }
    return v;
}

// The same shape evaluated in FP32 from the FP32 copy (reduced-precision
// kernels keep FP64 out of their inner loop: FP64 runs at 1/64 rate here).
__device__ __forceinline__ float field_value_f(const FieldDev &F, int kind, int c, int x, int y, int z,
                                               int node)
{
    if (kind == FK_CONST) return F.fcval[c];
    if ((F.zmask >> c) & 1) return 0.0f;
    const float *t = F.fdata + c * F.cstride;
    if (!F.sep) return __ldg(t + node);
    float v = 1.0f;
    bool have = false;
    if (F.axes & 1) {
        v = __ldg(t + (F.len[0] > 1 ? x : 0));
        have = true;
    }
    if (F.axes & 2) {
        const float py = __ldg(t + F.len[0] + (F.len[1] > 1 ? y : 0));
        v = have ? v * py : py;
        have = true;
    }
    if (F.axes & 4) {
        const float pz = __ldg(t + F.len[0] + F.len[1] + (F.len[2] > 1 ? z : 0));
        v = have ? v * pz : pz;
    }
    return v;
}

}  // namespace lbmk
