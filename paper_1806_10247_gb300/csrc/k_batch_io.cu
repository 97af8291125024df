// Macroscopic fields of every member of a batch in one launch (Eq. 24 / 42,
// plus the pre-collision half force / source of Eq. 25 / 43 when asked),
// written packed member after member: rho (or phi) of member i at
// rho[off_i .. off_i + N_i), its velocity as a [dim][N_i] block at
// u[dim * off_i ...].  One tile of 256 nodes per block; the member's
// descriptor is staged in shared memory as in the step kernels.
#include "lbm_d3q15.cuh"
#include "lbm_internal.h"
#include "lbm_lattices.cuh"
#include "lbm_tiles.cuh"

namespace lbmk {
namespace {

constexpr int kTile = 256;

template <class L, class T>
__device__ __forceinline__ void member_moments(const BatchItem &B, const BatchMoments &M, int it, int i)
{
    const Geom &g = B.g;
    int x, y, z;
    node_xyz(g, i, x, y, z);
    const int p = (B.parity + M.parity) & 1;
    double m0, j[3];
    if constexpr (sizeof(T) == 8) {
        double f[L::Q];
        load_pulled<L>(reinterpret_cast<const double *>(B.buf[p]), g, x, y, z, i, f);
        zeroth_first<L>(f, m0, j);
    } else {
        float d[L::Q];
        load_pulled_dev<L, T>(reinterpret_cast<const T *>(B.buf[p]), g, x, y, z, i, d);
        double dd[L::Q];
#pragma unroll
        for (int a = 0; a < L::Q; a++) dd[a] = (double)d[a];
        zeroth_first<L>(dd, m0, j);
        m0 += B.rho_ref;  // the rest state carries no momentum
    }
    const bool forced = M.half && B.fkind != FK_NONE;
    const double apre = M.apre ? __ldg(M.apre + it) : M.apre_inl[it];
    store_fields<L>(m0, j, forced, apre, B.F, B.fkind, x, y, z, i, g.N, __ldg(M.off + it), M.rho, M.u);
}

template <class L, class T>
__global__ void __launch_bounds__(kTile) k_batch_moments(const __grid_constant__ BatchMoments M)
{
    __shared__ BatchItem B;
    const int tile = blockIdx.x;
    const int it = tile_item(M.first, M.count, tile, -1);
    stage_to_shared(B, M.items[it]);
    __syncthreads();
    const int i = (tile - __ldg(M.first + it)) * kTile + (int)threadIdx.x;
    if (i < B.g.N) member_moments<L, T>(B, M, it, i);
}

template <class L>
cudaError_t launch_l(const BatchMoments &M, int storage, int nblocks, cudaStream_t s)
{
    switch (storage) {
    case 0: k_batch_moments<L, double><<<nblocks, kTile, 0, s>>>(M); break;
    case 1: k_batch_moments<L, float><<<nblocks, kTile, 0, s>>>(M); break;
    case 2: k_batch_moments<L, __half><<<nblocks, kTile, 0, s>>>(M); break;
    case 3: k_batch_moments<L, __nv_bfloat16><<<nblocks, kTile, 0, s>>>(M); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t batch_moments(int lattice, int storage, const BatchMoments &M, int nblocks, cudaStream_t s)
{
    switch (lattice) {
    case LD2Q9::ID: return launch_l<LD2Q9>(M, storage, nblocks, s);
    case LD2Q5::ID: return launch_l<LD2Q5>(M, storage, nblocks, s);
    case LD3Q27::ID: return launch_l<LD3Q27>(M, storage, nblocks, s);
    case LD3Q15::ID: return launch_l<LD3Q15>(M, 0, nblocks, s);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace lbmk
