// Tile loop of the batched launches.  A batched launch covers the tiles of
// every member lattice (TB nodes per tile, TB threads per block, tiles
// numbered member after member; first[i] is member i's first tile).  Either
// each block takes one tile, or (persistent grid, L.persist = 1) each block
// takes a contiguous run of tiles, the runs of the grid's blocks differing by
// at most one tile, so that consecutive tiles mostly belong to the same
// member and its descriptor is staged into shared memory once per run.
#pragma once

#include <cuda_runtime.h>

#include "lbm_internal.h"
#include "lbm_lattices.cuh"

namespace lbmk {

// Member owning tile `tile`: `cur` if it still does (tiles ascend within a
// block), else a binary search for the last i with first[i] <= tile.
__device__ __forceinline__ int tile_item(const int *__restrict__ first, int count, int tile, int cur)
{
    if (cur >= 0 && (cur + 1 == count || tile < __ldg(first + cur + 1))) return cur;
    int lo = cur < 0 ? 0 : cur, hi = count - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(first + mid) <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Kernel forms: one tile per block, persistent (a run of tiles per block),
// single member (descriptor in the launch arguments, one tile per block).
enum { TILE_ONE = 0, TILE_PERSIST = 1, TILE_SINGLE = 2 };

// Run [t0, t1) of this block of a persistent grid: the ntiles tiles split
// evenly over the grid's blocks.
__device__ __forceinline__ void persist_run(const BatchLaunch &L, int &t0, int &t1)
{
    const long long nt = L.ntiles, G = gridDim.x, b = blockIdx.x;
    t0 = (int)(b * nt / G);
    t1 = (int)((b + 1) * nt / G);
}

// Runs node(B, L, member, node index) for every node of the block's tiles,
// with B the member's descriptor (staged in shared memory, or the launch
// argument copy for a single member).
template <int TB, int MODE, class Node>
__device__ __forceinline__ void batch_tiles(const BatchLaunch &L, Node node)
{
    if (MODE == TILE_SINGLE) {
        const int i = blockIdx.x * TB + (int)threadIdx.x;
        if (i < L.one.g.N) node(L.one, L, 0, i);
        return;
    }
    __shared__ BatchItem B;
    if (MODE == TILE_ONE) {
        const int tile = blockIdx.x;
        const int it = tile_item(L.first, L.count, tile, -1);
        stage_to_shared(B, L.items[it]);
        __syncthreads();
        const int i = (tile - __ldg(L.first + it)) * TB + (int)threadIdx.x;
        if (i < B.g.N) node(B, L, it, i);
        return;
    }
    int t0, t1;
    persist_run(L, t0, t1);
    int cur = -1;
    for (int tile = t0; tile < t1; tile++) {
        const int it = tile_item(L.first, L.count, tile, cur);
        if (it != cur) {  // block-uniform
            if (cur >= 0) __syncthreads();
            stage_to_shared(B, L.items[it]);
            __syncthreads();
            cur = it;
        }
        const int i = (tile - __ldg(L.first + it)) * TB + (int)threadIdx.x;
        if (i < B.g.N) node(B, L, it, i);
    }
}

// Fused readback of an FP64 batched step: the packed fields of the state the
// step starts from, formed from the node's pulled populations f(t) exactly as
// the packed readback kernel forms them.
template <class L>
__device__ __forceinline__ void fused_fields(const BatchItem &B, const BatchLaunch &Ln, int it, int i, int x, int y, int z,
                                             const double (&f)[L::Q], double apre)
{
    double m0, j[3];
    zeroth_first<L>(f, m0, j);
    store_fields<L>(m0, j, Ln.mhalf && B.fkind != FK_NONE, apre, B.F, B.fkind, x, y, z, i, B.g.N, __ldg(Ln.moff + it),
                    Ln.mrho, Ln.mu);
}

// Blocks of `kernel` (launched with tb threads) resident on the current GPU at once.
template <class K>
int resident_blocks(K kernel, int tb)
{
    int per_sm = 0, dev = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, tb, 0);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return per_sm * sms;
}

// Form of a launch from its arguments.
inline int tile_mode(const BatchLaunch &L) { return L.single ? TILE_SINGLE : (L.persist ? TILE_PERSIST : TILE_ONE); }

// Launch of a batched kernel template K<TB, MODE> for tile sizes 128, 256, 512.
#define LBM_TILED_LAUNCH(KERNEL, L, nblocks, tile, s)                                              \
    do {                                                                                           \
        const int m_ = tile_mode(L);                                                               \
        switch (tile) {                                                                            \
        case 128: if (m_ == TILE_SINGLE) KERNEL<128, TILE_SINGLE><<<(nblocks), 128, 0, (s)>>>(L);   \
                  else if (m_ == TILE_PERSIST) KERNEL<128, TILE_PERSIST><<<(nblocks), 128, 0, (s)>>>(L); \
                  else KERNEL<128, TILE_ONE><<<(nblocks), 128, 0, (s)>>>(L); break;                 \
        case 256: if (m_ == TILE_SINGLE) KERNEL<256, TILE_SINGLE><<<(nblocks), 256, 0, (s)>>>(L);   \
                  else if (m_ == TILE_PERSIST) KERNEL<256, TILE_PERSIST><<<(nblocks), 256, 0, (s)>>>(L); \
                  else KERNEL<256, TILE_ONE><<<(nblocks), 256, 0, (s)>>>(L); break;                 \
        case 512: if (m_ == TILE_SINGLE) KERNEL<512, TILE_SINGLE><<<(nblocks), 512, 0, (s)>>>(L);   \
                  else if (m_ == TILE_PERSIST) KERNEL<512, TILE_PERSIST><<<(nblocks), 512, 0, (s)>>>(L); \
                  else KERNEL<512, TILE_ONE><<<(nblocks), 512, 0, (s)>>>(L); break;                 \
        default: return cudaErrorInvalidValue;                                                     \
        }                                                                                          \
        return cudaGetLastError();                                                                 \
    } while (0)

// Resident blocks of the persistent form (the grid a persistent launch uses).
#define LBM_TILED_RESIDENT(KERNEL, tile)                                                           \
    do {                                                                                           \
        switch (tile) {                                                                            \
        case 128: return resident_blocks(KERNEL<128, TILE_PERSIST>, 128);                          \
        case 256: return resident_blocks(KERNEL<256, TILE_PERSIST>, 256);                          \
        case 512: return resident_blocks(KERNEL<512, TILE_PERSIST>, 512);                          \
        default: return 0;                                                                         \
        }                                                                                          \
    } while (0)

}  // namespace lbmk
