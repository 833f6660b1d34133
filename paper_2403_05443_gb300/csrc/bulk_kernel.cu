// Bulk lattice kernel: pull streaming and BGK collision with Guo forcing
// (Eq. 3-4) on every node of every box, the hot loop of the method.
//
// A node's 19 populations are read once and written once (2*19*s bytes).  One
// thread owns 4 consecutive x nodes: each direction is one 16-byte load of
// the source row (8 bytes for 16-bit storage) and the +-1 shift in x comes from
// the neighbouring lane by a warp shuffle, with a scalar load at warp and row
// ends that also wraps x periodically.  No shared memory and no barrier: the
// block finds its box in a table and starts loading at once.
//
// Wall links (solid planes y = 0 and y = ny-1 moving with u_w) are handled
// here: they are static and row-uniform.  Nodes next to a particle's surface
// (the redo mask of this step) are left to the boundary kernel, which writes
// them concurrently; a thread tests its row against the cubes of its box's
// particles, a few integer compares per particle.
//
// This standalone launch (two 256-thread blocks per SM walking the tiles with
// a grid stride) serves the first collision and the per-kernel profile; the
// time steps themselves run the same tile function inside the persistent step
// kernel (step_kernel.cu).
#include "bulk_tile.cuh"

namespace lbsph {

template <class St, bool FIRST>
__global__ void __launch_bounds__(KBLOCK, 2) bulk_kernel(const BulkParams P, int tiles)
{
    // warp-sized units of 32 quads, strided over all warps of the grid
    constexpr int WPB = KBLOCK / 32;
    const int lane = threadIdx.x & 31;
    const int units = tiles * WPB;
    for (int u = blockIdx.x * WPB + (threadIdx.x >> 5); u < units; u += gridDim.x * WPB)
        bulk_tile<St, FIRST>(P, u / WPB, (u % WPB) * 32 + lane);
}

// two blocks per SM of the current device (queried on every launch: a process
// may drive devices of different sizes; the grid-stride loop covers every unit
// whatever the grid)
static int bulk_grid(int tiles)
{
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        nsm < 1)
        nsm = 1;
    const int g = 2 * nsm;
    return tiles < g ? tiles : g;
}

template <class St>
static cudaError_t launch_bulk_t(const BulkParams& p, int tiles, cudaStream_t s)
{
    const int g = bulk_grid(tiles);
    if (p.first) bulk_kernel<St, true><<<g, KBLOCK, 0, s>>>(p, tiles);
    else bulk_kernel<St, false><<<g, KBLOCK, 0, s>>>(p, tiles);
    return cudaGetLastError();
}

cudaError_t launch_bulk(const BulkParams& p, int precision, int blocks, cudaStream_t s)
{
    if (precision == 1) return launch_bulk_t<StF16>(p, blocks, s);
    if (precision == 2) return launch_bulk_t<StBF16>(p, blocks, s);
    if (precision == 3) return launch_bulk_t<StF32G>(p, blocks, s);   // FP32, the paper's collision
    return launch_bulk_t<StF32>(p, blocks, s);
}

}  // namespace lbsph
