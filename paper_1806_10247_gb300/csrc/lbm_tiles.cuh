// Tile loop of the batched launches.  A batched launch covers the tiles of
// every member lattice (TB nodes per tile, TB threads per block, tiles
// numbered member after member; first[i] is member i's first tile).  Either
// each block takes one tile, or (persistent grid, L.chunk > 0) each block
// takes a contiguous run of L.chunk tiles, so that consecutive tiles mostly
// belong to the same member and its descriptor is staged into shared memory
// once per run.
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

// Runs node(B, L, member, node index) for every node of the block's tiles,
// with B the member's descriptor staged in shared memory.  PERSIST selects
// the persistent form (L.chunk > 0: a run of tiles per block); the one-tile
// form has no loop, so that it costs no registers.
template <int TB, bool PERSIST, class Node>
__device__ __forceinline__ void batch_tiles(const BatchLaunch &L, Node node)
{
    __shared__ BatchItem B;
    if (!PERSIST) {
        const int tile = blockIdx.x;
        const int it = tile_item(L.first, L.count, tile, -1);
        stage_to_shared(B, L.items[it]);
        __syncthreads();
        const int i = (tile - __ldg(L.first + it)) * TB + (int)threadIdx.x;
        if (i < B.g.N) node(B, L, it, i);
        return;
    }
    const int t0 = blockIdx.x * L.chunk;
    const int t1 = min(t0 + L.chunk, L.ntiles);
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

// Launch of a batched kernel template K<TB, PERSIST> for tile sizes 128,
// 256, 512; the persistent form when L.chunk > 0.
#define LBM_TILED_LAUNCH(KERNEL, L, nblocks, tile, s)                                              \
    do {                                                                                           \
        const bool p_ = (L).chunk > 0;                                                             \
        switch (tile) {                                                                            \
        case 128: if (p_) KERNEL<128, true><<<(nblocks), 128, 0, (s)>>>(L);                         \
                  else KERNEL<128, false><<<(nblocks), 128, 0, (s)>>>(L); break;                    \
        case 256: if (p_) KERNEL<256, true><<<(nblocks), 256, 0, (s)>>>(L);                         \
                  else KERNEL<256, false><<<(nblocks), 256, 0, (s)>>>(L); break;                    \
        case 512: if (p_) KERNEL<512, true><<<(nblocks), 512, 0, (s)>>>(L);                         \
                  else KERNEL<512, false><<<(nblocks), 512, 0, (s)>>>(L); break;                    \
        default: return cudaErrorInvalidValue;                                                     \
        }                                                                                          \
        return cudaGetLastError();                                                                 \
    } while (0)

// Resident blocks of the persistent form (the grid a persistent launch uses).
#define LBM_TILED_RESIDENT(KERNEL, tile)                                                           \
    do {                                                                                           \
        switch (tile) {                                                                            \
        case 128: return resident_blocks(KERNEL<128, true>, 128);                                  \
        case 256: return resident_blocks(KERNEL<256, true>, 256);                                  \
        case 512: return resident_blocks(KERNEL<512, true>, 512);                                  \
        default: return 0;                                                                         \
        }                                                                                          \
    } while (0)

}  // namespace lbmk
