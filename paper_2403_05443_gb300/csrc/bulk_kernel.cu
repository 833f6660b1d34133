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
// The grid is persistent: each block (256 threads, half an SM's registers)
// walks 256-quad tiles with a grid stride.  It has FREE_SLOTS blocks fewer
// than two per SM, so that about FREE_SLOTS half-SMs stay free for the
// particle kernels that run concurrently on the particle streams.
#include "lattice_common.cuh"

namespace lbsph {

template <class St, bool FIRST>
__device__ __forceinline__ void bulk_tile(const BulkParams& P, int tile)
{
    const int tix = threadIdx.x;
    using T = typename St::T;
    const int bi = __ldg(P.blk_box + tile);
    const BoxDev& B = P.boxes[bi];
    const int nx = B.nx, ny = B.ny, nz = B.nz, nxq = B.nxq;
    const long long N = B.N;
    long long q = (long long)(tile - B.block_begin) * KBLOCK + tix;
    const bool valid = q < B.nq;
    if (!valid) q = B.nq - 1;
    const int xq = (int)(q % nxq);
    const long long row = q / nxq;
    const int y = (int)(row % ny), z = (int)(row / ny);
    const int lane = tix & 31;
    const T* A = reinterpret_cast<const T*>(P.src) + B.off;
    T* D = reinterpret_cast<T*>(P.dst) + B.off;
    const float inv = B.inv_scale;
    const long long own = row * nx + 4 * xq;

    long long rofs[3][3];  // element offsets of the source rows (y + dy, z + dz), wrapped
    {
        const int yy[3] = {y == 0 ? ny - 1 : y - 1, y, y == ny - 1 ? 0 : y + 1};
        const int zz[3] = {z == 0 ? nz - 1 : z - 1, z, z == nz - 1 ? 0 : z + 1};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) rofs[a][b] = ((long long)zz[b] * ny + yy[a]) * nx;
    }
    const bool left_ld = (lane == 0) || (xq == 0);
    const bool right_ld = (lane == 31) || (xq == nxq - 1);

    float4 v[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (FIRST) {
            v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
            continue;
        }
        const T* rp = A + (long long)i * N + rofs[1 - cy_of(i)][1 - cz_of(i)];
        float4 t = St::ld4(rp + 4 * xq, inv);
        if (cx_of(i) == 1) {            // source x - 1
            float l = __shfl_up_sync(0xffffffffu, t.w, 1);
            if (left_ld) l = St::ld1(rp + (xq == 0 ? nx - 1 : 4 * xq - 1), inv);
            t = make_float4(l, t.x, t.y, t.z);
        } else if (cx_of(i) == -1) {    // source x + 1
            float r = __shfl_down_sync(0xffffffffu, t.x, 1);
            if (right_ld) r = St::ld1(rp + (xq == nxq - 1 ? 0 : 4 * xq + 4), inv);
            t = make_float4(t.y, t.z, t.w, r);
        }
        v[i] = t;
    }

    const BoxDyn dyn = P.box_dyn[bi];
    const bool wallrow = B.walls && (y == 0 || y == ny - 1);
    if (!FIRST && B.walls && (y == 1 || y == ny - 2)) {
        // link bounce-back on a moving wall (Eq. fb with u_b = u_w)
        const int cyw = (y == 1) ? 1 : -1;
        const float* uw = (y == 1) ? B.uw_lo : B.uw_hi;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            if (cy_of(i) != cyw) continue;
            const float ubc = cx_of(i) * uw[0] + cy_of(i) * uw[1] + cz_of(i) * uw[2];
            const float add = 6.0f * w_of(i) * B.rho0f * ubc;
            const float4 o = St::ld4(A + (long long)opp_of(i) * N + own, inv);
            v[i] = make_float4(o.x + add, o.y + add, o.z + add, o.w + add);
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float f[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i] = comp(v[i], k);
        collide19(f, B.omega, B.rho0f, dyn.g[0], dyn.g[1], dyn.g[2], dyn.eps);
#pragma unroll
        for (int i = 0; i < Q; ++i) set_comp(v[i], k, wallrow ? 0.0f : f[i]);
    }
    // nodes of this quad that the boundary kernel writes
    unsigned skip = 0;
    for (int j = 0; j < B.pcnt; ++j) {
        const NeedHdr h = P.need_hdr[B.pbeg + j];
        int dz = z - h.ow[2];
        if (dz < 0) dz += nz;
        if (dz >= h.S) continue;
        int dy = y - h.ow[1];
        if (dy < 0) dy += ny;
        if (dy >= h.S) continue;
        int dx = 4 * xq - h.ow[0];
        if (dx < 0) dx += nx;
        if (dx >= h.S && dx + 3 < nx) continue;
        const uint64_t w = P.need[(size_t)(B.pbeg + j) * (MAXS * MAXS) + dz * h.S + dy];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int mx = dx + k < nx ? dx + k : dx + k - nx;
            if (mx < h.S && ((w >> mx) & 1ull)) skip |= 1u << k;
        }
    }
    if (valid) {
        T* dp = D + own;
        if (!skip) {
#pragma unroll
            for (int i = 0; i < Q; ++i) St::st4(dp + (long long)i * N, v[i], B.scale);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if ((skip >> k) & 1u) continue;
#pragma unroll
                for (int i = 0; i < Q; ++i) St::st1(dp + (long long)i * N + k, comp(v[i], k), B.scale);
            }
        }
    }
}

#ifndef LBSPH_FREE_SLOTS
#define LBSPH_FREE_SLOTS 32
#endif
constexpr int FREE_SLOTS = LBSPH_FREE_SLOTS;   // half-SMs left to the particle kernels

template <class St, bool FIRST>
__global__ void __launch_bounds__(KBLOCK, 2) bulk_kernel(const BulkParams P, int tiles)
{
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) bulk_tile<St, FIRST>(P, tile);
}

static int bulk_grid(int tiles)
{
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            nsm = 1;
    }
    const int g = nsm > FREE_SLOTS ? 2 * nsm - FREE_SLOTS : 2 * nsm;
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
    return launch_bulk_t<StF32>(p, blocks, s);
}

}  // namespace lbsph
