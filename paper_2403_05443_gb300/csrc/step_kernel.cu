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
// barrier, with the arrival and item counters at zero, so launches follow each
// other with no reset in between.  The iterations take their bulk units from
// two counters in turn (by barrier generation), each cleared by block 0 while
// the other one is in use.
//
// Cross-block data are read through L2 (ld.global.cg, see lattice_common.cuh).
// Every wait is bounded: a barrier that waits longer than SPIN_LIMIT polls
// sets ST_TIMEOUT in the status word and the abort flag, and every block
// leaves the kernel at the barrier it waits at or at the next one it reaches.
#include "boundary_block.cuh"
#include "bulk_tile.cuh"
#include "particle_blocks.cuh"

namespace lbsph {

constexpr int SYNC_BAR = 0;          // barrier arrivals (zero between barriers)
constexpr int SYNC_GEN = 2;          // barrier generation (counts up, wraps), 8-byte aligned with
constexpr int SYNC_ABORT = 3;        //   the abort flag: nonzero once a wait ran out
constexpr int SYNC_WORK = 4;         // + (generation & 1): bulk units taken in the iteration of that generation
constexpr int SYNC_PART = SYNC_HDR;  // + p: items of particle p done in this iteration
constexpr int MAX_GRID = 4096;
constexpr long long SPIN_LIMIT = 1ll << 22;   // polls (an L2 read, then a 64 ns sleep): a few seconds

struct StepParams {
    BulkParams bulk[2];              // by buffer parity of the iteration
    BndParams bnd[2];
    PParams part[2];
    unsigned* sync;                  // SYNC_PART + np words (the arrival and item counters zero at launch and
                                     // again at exit), then the blocks' SM ids
    unsigned* status;
    int np, gx, tiles, iters, cur0;
    int fetch;                       // bulk units per counter fetch (1, 2, 4, 8), single units at the end
    const double* io_ft;             // per iteration np * 6 doubles of F_ext, T_ext (or null)
    double* io_rec;                  // per iteration np * RECD doubles of records (or null)
};

// Grid barrier.  Each block counts the generations itself (s_gen, read once
// at kernel entry), so a barrier costs one arrival atomic and the polls of the
// generation word: the last block to arrive clears the arrival counter and
// publishes the next generation; the others poll the generation together with
// the abort flag (one 8-byte load), which a block whose wait ran out sets
// after setting ST_TIMEOUT, so that every other block leaves at the barrier it
// waits at or at its next one.
__device__ __forceinline__ bool grid_barrier(const StepParams& SP, unsigned& s_gen)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        const unsigned g = s_gen;
        bool ok = true;
        __threadfence();
        if (atomicAdd(SP.sync + SYNC_BAR, 1u) == gridDim.x - 1) {
            // last to arrive: clear the arrivals, then release the next generation
            SP.sync[SYNC_BAR] = 0;
            __threadfence();
            *reinterpret_cast<volatile unsigned*>(SP.sync + SYNC_GEN) = g + 1;
        } else {
            const volatile unsigned long long* ga = reinterpret_cast<const volatile unsigned long long*>(SP.sync + SYNC_GEN);
            long long n = 0;
            for (;;) {
                const unsigned long long v = *ga;
                if ((unsigned)(v >> 32) != 0u) { ok = false; break; }
                if ((unsigned)v != g) break;
                if (++n > SPIN_LIMIT) {
                    atomicOr(SP.status, ST_TIMEOUT);
                    atomicExch(SP.sync + SYNC_ABORT, 1u);
                    ok = false;
                    break;
                }
                if (n > 64) __nanosleep(64);
            }
            __threadfence();
        }
        s_gen = g + 1;
        s_ok = ok;
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
    __shared__ unsigned s_gen;
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
        // the generation before this launch's first barrier (no block can pass
        // that barrier before every block has read it)
        s_gen = *reinterpret_cast<volatile unsigned*>(SP.sync + SYNC_GEN);
        // the work counter of the first iteration was the last launch's last
        // one: clear it (the launches on a stream do not overlap)
        if (blockIdx.x == 0) SP.sync[SYNC_WORK + ((s_gen + 1) & 1)] = 0;
    }
    if (!grid_barrier(SP, s_gen)) return;
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
    const int nwarps = (int)gridDim.x * (KBLOCK / 32);
    for (int it = 0; it < SP.iters; ++it) {
        const int cur = (SP.cur0 + it) & 1;
        const BulkParams& BP = SP.bulk[cur];
        const BndParams& NP = SP.bnd[cur];
        const PParams& PP = SP.part[cur];
        const unsigned gen = s_gen;
        unsigned* work = SP.sync + SYNC_WORK + (gen & 1);
        // the other work counter (the last iteration's) for the next iteration
        if (blockIdx.x == 0 && tid == 0) SP.sync[SYNC_WORK + ((gen + 1) & 1)] = 0;
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
        // ---- bulk work in warp-sized units (32 quads of a tile): SP.fetch
        // consecutive units per fetch from the counter while more than two
        // rounds of such fetches remain, then single units, so that the last
        // units to finish are short; no block barrier, each warp moves on as
        // soon as its stores are issued; the next fetch is issued before the
        // current units run
        {
            const int lane = tid & 31;
            const int units = SP.tiles * (KBLOCK / 32);
            const int fetch = SP.fetch;
            const int coarse_end = units - 2 * nwarps * fetch;
            int u = 0, nf = fetch;
            if (lane == 0) u = (int)atomicAdd(work, (unsigned)fetch);
            u = __shfl_sync(0xffffffffu, u, 0);
            while (u < units) {
                const int end = min(u + nf, units);
                nf = u + nf < coarse_end ? fetch : 1;
                int nu = 0;
                if (lane == 0) nu = (int)atomicAdd(work, (unsigned)nf);
                for (int v = u; v < end; ++v) bulk_tile<St, false>(BP, v >> 3, ((v & 7) << 5) + lane);
                u = __shfl_sync(0xffffffffu, nu, 0);
            }
        }
        if (!grid_barrier(SP, s_gen)) return;
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
