// Persistent step kernel: many iterations of the method in one cooperative
// launch, so that no step pays kernel launches, stream hand-offs or a cold
// instruction cache on the SMs that take the particle work.
//
// Each iteration (two 256-thread blocks per SM, all resident by the
// cooperative launch):
//   - particle items, gx + 1 per particle, on fixed blocks ranked by SM, so
//     that they fill whole SMs (no bulk traffic next to them while they run)
//     and the same SMs keep their code cached from step to step: gx boundary
//     chunks of step t (the
//     nodes next to the particle's surface, boundary_block.cuh) and the
//     auxiliary block of step t-1 (drag matrix and inverse of the solve of
//     step t); the last of the particle's items to finish goes on with its
//     critical block (force, implicit solve, pose, new occupancy, redo masks
//     and box terms of step t+1);
//   - bulk work (bulk_tile.cuh), every other node of every box, taken by
//     every warp from a counter in units of 32 quads (128 nodes), so that the
//     warps of a block load and compute out of step with each other; the next
//     unit is fetched while one runs.
// A grid barrier ends the iteration: after it the lattice of step t, the box
// terms and the redo masks of step t+1 are complete.  The auxiliary block of
// the last iteration runs first in the next launch: a launch ends at its last
// barrier, and the barrier, work and item counters are zero again then, so
// launches follow each other with no reset in between.
//
// Cross-block data are read through L2 (ld.global.cg, see lattice_common.cuh).
// Every wait is bounded: a barrier that waits longer than SPIN_LIMIT polls
// sets ST_TIMEOUT in the status word, and every block leaves the kernel at the
// next barrier it reaches.
#include "boundary_block.cuh"
#include "bulk_tile.cuh"
#include "particle_blocks.cuh"

namespace lbsph {

constexpr int SYNC_BAR = 0;          // barrier arrivals
constexpr int SYNC_GEN = 1;          // barrier generation
constexpr int SYNC_WORK = 2;         // work counter of the current iteration
constexpr int SYNC_PART = 4;         // + p: items of particle p done in this iteration
constexpr int MAX_GRID = 4096;
constexpr long long SPIN_LIMIT = 1ll << 24;   // polls of about 100 ns: under 2 s

struct StepParams {
    BulkParams bulk[2];              // by buffer parity of the iteration
    BndParams bnd[2];
    PParams part[2];
    unsigned* sync;                  // SYNC_PART + np words, zero at launch (and again at exit), then the blocks' SM ids
    unsigned* status;
    int np, gx, tiles, iters, cur0;
    int fetch;                       // bulk units per counter fetch (1, 2, 4, 8)
    const double* io_ft;             // per iteration np * 6 doubles of F_ext, T_ext (or null)
    double* io_rec;                  // per iteration np * RECD doubles of records (or null)
};

__device__ __forceinline__ bool grid_barrier(const StepParams& SP)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = SP.sync + SYNC_GEN;
        const unsigned g = *gen;
        __threadfence();
        if (atomicAdd(SP.sync + SYNC_BAR, 1u) == gridDim.x - 1) {
            // last to arrive: reset the counters of the next iteration, then release
            SP.sync[SYNC_BAR] = 0;
            SP.sync[SYNC_WORK] = 0;
            __threadfence();
            atomicExch(SP.sync + SYNC_GEN, g + 1);
        } else {
            long long n = 0;
            while (*gen == g) {
                if (++n > SPIN_LIMIT) {
                    atomicOr(SP.status, ST_TIMEOUT);
                    break;
                }
                __nanosleep(100);
            }
        }
        __threadfence();
        s_ok = (*reinterpret_cast<volatile unsigned*>(SP.status) & ST_TIMEOUT) == 0;
    }
    __syncthreads();
    return s_ok != 0;
}

// The cluster of particle p for this iteration: the particles reachable from p
// through the partner lists (symmetric) that the critical blocks of the last
// iteration wrote.  A particle's boundary blocks read its partners' maps and
// add to their accumulators, so no critical block of a cluster may start before
// every item of the cluster is done.  Returns the lowest index (the cluster's
// counter) and the members as a mask over the box's particles (at most MAXPB
// when any particle has partners).  One thread.
__device__ __forceinline__ int cluster_of(const PartK* pk, int p, unsigned long long& members, int& size)
{
    const int nnb0 = __ldcg(&pk[p].nnb);
    if (nnb0 == 0) {
        members = 0;
        size = 1;
        return p;
    }
    const int pbeg = __ldcg(&pk[p].pbeg);
    unsigned long long seen = 1ull << (p - pbeg), todo = seen;
    while (todo) {
        const int j = __ffsll((long long)todo) - 1;
        todo &= todo - 1;
        const int q = pbeg + j;
        const int n = min(__ldcg(&pk[q].nnb), MAXNB);
        for (int k = 0; k < n; ++k) {
            const int r = __ldcg(&pk[q].nb[k]) - pbeg;
            if (r < 0 || r >= MAXPB) continue;
            const unsigned long long bit = 1ull << r;
            if (!(seen & bit)) { seen |= bit; todo |= bit; }
        }
    }
    members = seen;
    size = __popcll(seen);
    return pbeg + __ffsll((long long)seen) - 1;
}

template <class St>
__global__ void __launch_bounds__(KBLOCK, 2) step_kernel(const __grid_constant__ StepParams SP)
{
    __shared__ int s_last, s_rank, s_root;
    __shared__ unsigned long long s_members;
    const int tid = threadIdx.x;
    const int gx = SP.gx;
    const int npart = SP.np * (gx + 1);
    // a context whose barrier timed out before keeps its counters as they were
    // left: do no work (the status word already reports the timeout)
    if (__ldcg(SP.status) & ST_TIMEOUT) return;
    // ---- rank of this block by (SM, block index): particle items go to whole SMs
    unsigned* blk_sm = SP.sync + SYNC_PART + SP.np;
    if (tid == 0) {
        unsigned smid;
        asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
        blk_sm[blockIdx.x] = smid;
        s_rank = 0;
    }
    if (!grid_barrier(SP)) return;
    {
        const unsigned mine = __ldcg(blk_sm + blockIdx.x);
        int before = 0;
        for (int b = tid; b < (int)gridDim.x; b += KBLOCK) {
            const unsigned o = __ldcg(blk_sm + b);
            before += (o < mine) || (o == mine && b < (int)blockIdx.x);
        }
        if (before) atomicAdd(&s_rank, before);
    }
    __syncthreads();
    const int prank = s_rank;
    for (int it = 0; it < SP.iters; ++it) {
        const int cur = (SP.cur0 + it) & 1;
        const BulkParams& BP = SP.bulk[cur];
        const BndParams& NP = SP.bnd[cur];
        const PParams& PP = SP.part[cur];
        // ---- particle items
        for (int item = prank; item < npart; item += gridDim.x) {
            const int p = item / (gx + 1), c = item % (gx + 1);
            if (c < gx) boundary_block<St, false>(NP, p, c);
            else aux_block(PP, p);                 // a no-op if it already ran for this pose
            __threadfence();
            __syncthreads();
            if (tid == 0) {
                // the last item of the particle's cluster runs the cluster's
                // critical blocks (a single particle: its own), in index order
                unsigned long long mem;
                int size;
                const int root = cluster_of(PP.pk, p, mem, size);
                s_root = root;
                s_members = mem;
                s_last = atomicAdd(SP.sync + SYNC_PART + root, 1u) == (unsigned)(size * (gx + 1) - 1);
            }
            __syncthreads();
            if (s_last) {
                __threadfence();
                const int root = s_root;
                if (tid == 0) SP.sync[SYNC_PART + root] = 0;
                unsigned long long mem = s_members;
                const int pbeg = root - (mem ? __ffsll((long long)mem) - 1 : 0);
                int q = root;
                do {
                    if (mem) {
                        q = pbeg + __ffsll((long long)mem) - 1;
                        mem &= mem - 1;
                    }
                    const size_t io = (size_t)it * SP.np + q;
                    crit_block(PP, q, SP.io_ft ? SP.io_ft + io * 6 : nullptr,
                               SP.io_rec ? SP.io_rec + io * RECD : nullptr);
                    __syncthreads();
                } while (mem);
            }
            __syncthreads();
        }
        // ---- bulk work in warp-sized units (32 quads of a tile), SP.fetch
        // consecutive units per fetch from the counter: no block barrier, each
        // warp moves on as soon as its stores are issued; the next fetch is
        // issued before the current units run
        {
            const int lane = tid & 31;
            const int units = SP.tiles * (KBLOCK / 32);
            const int fetch = SP.fetch;
            int u = 0;
            if (lane == 0) u = (int)atomicAdd(SP.sync + SYNC_WORK, 1u) * fetch;
            u = __shfl_sync(0xffffffffu, u, 0);
            while (u < units) {
                int nu = 0;
                if (lane == 0) nu = (int)atomicAdd(SP.sync + SYNC_WORK, 1u) * fetch;
                const int end = min(u + fetch, units);
                for (int v = u; v < end; ++v) bulk_tile<St, false>(BP, v >> 3, ((v & 7) << 5) + lane);
                u = __shfl_sync(0xffffffffu, nu, 0);
            }
        }
        if (!grid_barrier(SP)) return;
    }
    // the auxiliary blocks of the last iteration run as the first items of the
    // next launch (or before the next separate-kernel iteration or getter)
}

template <class St>
static cudaError_t launch_step_t(const StepParams& sp, size_t smem, cudaStream_t s)
{
    // co-resident blocks for this device and dynamic shared memory size (one
    // cheap occupancy query per launch: a process may drive several devices)
    cudaError_t e;
    if (smem > 0) {        // static + dynamic may pass the 48 KB default: always opt in
        e = cudaFuncSetAttribute(step_kernel<St>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    int dev = 0, nsm = 0, occ = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, step_kernel<St>, KBLOCK, smem)) != cudaSuccess) return e;
    if (occ < 1) return cudaErrorCooperativeLaunchTooLarge;
    const int grid = occ * nsm < MAX_GRID ? occ * nsm : MAX_GRID;
    void* args[] = {const_cast<StepParams*>(&sp)};
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(step_kernel<St>), dim3(grid), dim3(KBLOCK), args,
                                       smem, s);
}

cudaError_t launch_step(const BulkParams bulk[2], const BndParams bnd[2], const PParams part[2], unsigned* sync,
                        unsigned* status, int np, int gx, int tiles, int iters, int cur0, int precision, int fetch,
                        const double* io_ft, double* io_rec, cudaStream_t s)
{
    StepParams sp;
    sp.io_ft = io_ft;
    sp.io_rec = io_rec;
    for (int c = 0; c < 2; ++c) { sp.bulk[c] = bulk[c]; sp.bnd[c] = bnd[c]; sp.part[c] = part[c]; }
    sp.sync = sync; sp.status = status;
    sp.np = np; sp.gx = gx; sp.fetch = fetch < 1 ? 1 : fetch; sp.tiles = tiles; sp.iters = iters; sp.cur0 = cur0;
    const int smax = bnd[0].smax;
    const size_t maps = 2ull * smax * smax * sizeof(uint64_t);
    const size_t smem = np > 0 ? maps + (size_t)bnd[0].list_cap * sizeof(unsigned) : 0;
    if (precision == 1) return launch_step_t<StF16>(sp, smem, s);
    if (precision == 2) return launch_step_t<StBF16>(sp, smem, s);
    if (precision == 3) return launch_step_t<StF32G>(sp, smem, s);   // FP32, the paper's collision
    return launch_step_t<StF32>(sp, smem, s);
}

}  // namespace lbsph
