// Particle kernels, one CTA per particle.
//
// particle_crit (between the boundary kernel of iteration t and the bulk kernel
// of t+1, on the critical path), all FP64 work in one warp, one component per
// lane:
//   - F0, T0 of the links of map t (Eq. F0, Eq. T0): the boundary kernel's
//     fixed-point sums about the cube origin, moved to the centre, plus the
//     geometric and squirmer-slip parts prepared by the auxiliary kernel;
//   - the impulse of the nodes covered / uncovered by the last remap;
//   - the implicit solve of Eq. Fdiscrete / Eq. Tdiscrete as a product with the
//     inverse prepared by the auxiliary kernel, and the split of Eq. Fsplit /
//     Eq. Tsplit;
//   - Eq. posupdate and Eq. qnplus0-1;
//   - the occupancy map of the new pose (Eq. ellipsoidsurface): an FP32 test
//     settles every node whose value is farther than 1e-4 from 1, the rest use
//     the exact FP64 test in the fixed operation order the CPU oracle also uses;
//   - the box's uniform body force and mass return for the next collision.
// An FP64 instruction occupies the FP64 pipe of its SM quarter for about 64
// cycles on this part whatever the number of active lanes, so the chain is
// written to issue few FP64 instructions, each across lanes.
//
// particle_aux (after particle_crit of t, concurrent with the bulk kernel):
// link moments of the new map, drag matrices, the inverse for the next solve,
// the fixed parts of F0 and T0, and the list of nodes the boundary kernel must
// redo.
#include <cmath>

#include "../../include/lbsph.h"
#include "particle_blocks.cuh"

namespace lbsph {

__global__ void __launch_bounds__(CBLOCK) particle_crit_kernel(const __grid_constant__ PParams P)
{
    if (blockIdx.x < P.np) crit_block(P, blockIdx.x);
}

__global__ void __launch_bounds__(ABLOCK) particle_aux_kernel(const __grid_constant__ PParams P)
{
    if (blockIdx.x < P.np) aux_block(P, blockIdx.x);
}

// Boundary links of one particle's current map, compacted in (row, direction,
// x) order: a block-wide count, an exclusive scan, then the writes.
__global__ void __launch_bounds__(PBLOCK) links_kernel(const PartDev* pd, const PartK* pk, const uint64_t* rows_all,
                                                      const BoxDev* boxes, int p, int* out, int cap,
                                                      int* count)
{
    const PartDev& S = pd[p];
    const BoxDev& B = boxes[S.box];
    const int nnb = pk[p].nnb;
    const int Lb[3] = {B.nx, B.ny, B.nz};
    const uint64_t* rows = rows_all + ((long long)p * 2 + S.slot) * (MAXS * MAXS);
    const int Sd = S.S;
    const uint64_t maskS = Sd >= 64 ? ~0ull : ((1ull << Sd) - 1ull);
    const int items = Sd * Sd * 18;
    const int per = (items + PBLOCK - 1) / PBLOCK;
    const int i0 = threadIdx.x * per, i1 = min(items, i0 + per);
    __shared__ int s_cnt[PBLOCK];
    for (int pass = 0; pass < 2; ++pass) {
        int base = 0;
        if (pass == 1) {
            base = s_cnt[threadIdx.x];
        }
        int cnt = 0;
        for (int it = i0; it < i1; ++it) {
            const int r = it / 18, b = 1 + it % 18;
            const int my = r % Sd, mz = r / Sd;
            const int Yu = S.o[1] + my;
            if (B.walls && (Yu <= 0 || Yu >= B.ny - 1)) continue;
            const int ny2 = my + cy_of(b), nz2 = mz + cz_of(b);
            if (ny2 < 0 || ny2 >= Sd || nz2 < 0 || nz2 >= Sd) continue;
            const uint64_t nb = rows[nz2 * Sd + ny2];
            const int cbx = cx_of(b);
            const uint64_t sh = cbx == 1 ? (nb >> 1) : (cbx == -1 ? (nb << 1) : nb);
            uint64_t L = ~rows[r] & sh & maskS;
            // a node solid in a partner is no fluid end of a link
            if (L && nnb > 0) L &= ~partner_row_mask(pd, pk, rows_all, p, S.o, nnb, Lb, my, mz, maskS);
            while (L) {
                const int mx = __ffsll((long long)L) - 1;
                L &= L - 1;
                if (pass == 1) {
                    const int k = base + cnt;
                    if (k < cap) {
                        const int X = wrapi(S.o[0] + mx, B.nx), Y = wrapi(Yu, B.ny), Z = wrapi(S.o[2] + mz, B.nz);
                        out[2 * k] = (Z * B.ny + Y) * B.nx + X;
                        out[2 * k + 1] = b;
                    }
                }
                ++cnt;
            }
        }
        if (pass == 0) {
            s_cnt[threadIdx.x] = cnt;
            __syncthreads();
            if (threadIdx.x == 0) {
                int run = 0;
                for (int t = 0; t < PBLOCK; ++t) { const int c = s_cnt[t]; s_cnt[t] = run; run += c; }
                *count = run;
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// Boundary links of one spheroid without any allocation (lb_links_noalloc).
//
// The occupancy bitmap and the link counter live in this file-scope scratch,
// shared by every call on a device and kept from one call to the next; each
// call clears the part it uses first.  Calls that overlap on the GPU race on it.
constexpr int NOALLOC_WORDS = MAXS * MAXS;                  // 32 KiB of bitmap rows
static __device__ __align__(256) uint64_t g_noalloc_scratch[NOALLOC_WORDS + 32];

struct NoallocArgs {
    double semi[3], q[4], x[3];
    int nx, ny, nz, walls, S, h, cap;
    int* pairs;
    int* count;
};

__global__ void __launch_bounds__(PBLOCK) links_noalloc_kernel(const NoallocArgs a, uint64_t* scratch)
{
    uint64_t* rows = scratch;
    int* cnt = reinterpret_cast<int*>(scratch + NOALLOC_WORDS);
    const int tid = threadIdx.x, Sd = a.S;
    __shared__ double s_A[9], s_xc[3];
    __shared__ float s_e[3][3], s_inv[3], s_ro[3];
    __shared__ int s_o[3];
    for (int r = tid; r < Sd * Sd; r += PBLOCK) rows[r] = 0ull;
    if (tid == 0) {
        *cnt = 0;
        double e[3][3];
        canon_shape(a.semi, a.q, s_A, e);
        for (int k = 0; k < 3; ++k) {
            s_o[k] = (int)floor(a.x[k]) - a.h;
            s_xc[k] = a.x[k];
            s_ro[k] = (float)((double)s_o[k] - a.x[k]);
            s_inv[k] = (float)(1.0 / (a.semi[k] * a.semi[k]));
            for (int j = 0; j < 3; ++j) s_e[k][j] = (float)e[k][j];
        }
    }
    __syncthreads();
    const bool py = !a.walls;
    // occupancy: FP32 test away from the surface, exact FP64 test near it
    for (int n = tid; n < Sd * Sd * Sd; n += PBLOCK) {
        const int mx = n % Sd, my = (n / Sd) % Sd, mz = n / (Sd * Sd);
        const float dx = s_ro[0] + mx, dy = s_ro[1] + my, dz = s_ro[2] + mz;
        float v = 0.0f;
        for (int m = 0; m < 3; ++m) {
            const float t = s_e[m][0] * dx + s_e[m][1] * dy + s_e[m][2] * dz;
            v += t * t * s_inv[m];
        }
        bool solid;
        if (fabsf(v - 1.0f) > 1e-4f) {
            solid = v < 1.0f;
        } else {
            solid = canon_value(s_A, s_xc, wrapi(s_o[0] + mx, a.nx), wrapi(s_o[1] + my, a.ny), wrapi(s_o[2] + mz, a.nz),
                                a.nx, a.ny, a.nz, py) <= 1.0;
        }
        const int Yu = s_o[1] + my;
        if (solid && !(a.walls && (Yu <= 0 || Yu >= a.ny - 1)))
            atomicOr(reinterpret_cast<unsigned long long*>(rows + mz * Sd + my), 1ull << mx);
    }
    __syncthreads();
    // links (x fluid, x + c_b solid), written as (node index, direction) pairs
    const uint64_t maskS = Sd >= 64 ? ~0ull : ((1ull << Sd) - 1ull);
    for (int it = tid; it < Sd * Sd * 18; it += PBLOCK) {
        const int r = it / 18, b = 1 + it % 18;
        const int my = r % Sd, mz = r / Sd;
        const int Yu = s_o[1] + my;
        if (a.walls && (Yu <= 0 || Yu >= a.ny - 1)) continue;
        const int ny2 = my + cy_of(b), nz2 = mz + cz_of(b);
        if (ny2 < 0 || ny2 >= Sd || nz2 < 0 || nz2 >= Sd) continue;
        const uint64_t nb = rows[nz2 * Sd + ny2];
        const uint64_t sh = cx_of(b) == 1 ? (nb >> 1) : (cx_of(b) == -1 ? (nb << 1) : nb);
        uint64_t L = ~rows[r] & sh & maskS;
        while (L) {
            const int mx = __ffsll((long long)L) - 1;
            L &= L - 1;
            const int k = atomicAdd(cnt, 1);
            if (k < a.cap) {
                const int X = wrapi(s_o[0] + mx, a.nx), Y = wrapi(Yu, a.ny), Z = wrapi(s_o[2] + mz, a.nz);
                a.pairs[2 * k] = (Z * a.ny + Y) * a.nx + X;
                a.pairs[2 * k + 1] = b;
            }
        }
    }
    __syncthreads();
    if (tid == 0) *a.count = *cnt;
}

}  // namespace lbsph

extern "C" lb_status lb_links_noalloc(const double* semi, const double* q, const double* x, int32_t nx, int32_t ny,
                                      int32_t nz, int32_t walls, int32_t* pairs_dev, int32_t cap, int32_t* count_dev,
                                      void* stream)
{
    using namespace lbsph;
    if (!semi || !q || !x || !pairs_dev || !count_dev || cap < 0) return LB_EINVAL;
    if (nx < 4 || ny < 4 || nz < 4 || (walls && ny < 5)) return LB_EINVAL;
    const double qn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (std::fabs(qn - 1.0) > 1e-6) return LB_EINVAL;
    double m = 0.0;
    for (int k = 0; k < 3; ++k) {
        if (!(semi[k] > 0.0)) return LB_EINVAL;
        m = std::fmax(m, semi[k]);
    }
    NoallocArgs a{};
    a.h = (int)std::ceil(m) + CUBE_MARGIN;
    a.S = 2 * a.h + 2;
    if (a.S > MAXS || a.S > nx || a.S > nz || (!walls && a.S > ny)) return LB_ECAPACITY;
    for (int k = 0; k < 3; ++k) { a.semi[k] = semi[k]; a.x[k] = x[k]; }
    for (int k = 0; k < 4; ++k) a.q[k] = q[k] / qn;
    a.nx = nx; a.ny = ny; a.nz = nz; a.walls = walls; a.cap = cap;
    a.pairs = pairs_dev;
    a.count = count_dev;
    // Device address of the scratch array in the current device's context.
    // Host code cannot use the array's name as an address, and the address
    // belongs to the context: it is looked up on every call (a table lookup in
    // the runtime, no allocation and no synchronisation) rather than kept, so
    // that a context destroyed and created again (cudaDeviceReset) never
    // leaves a stale address behind.
    void* scratch = nullptr;
    if (cudaGetSymbolAddress(&scratch, g_noalloc_scratch) != cudaSuccess || !scratch) {
        cudaGetLastError();
        return LB_ECUDA;
    }
    links_noalloc_kernel<<<1, PBLOCK, 0, static_cast<cudaStream_t>(stream)>>>(a, static_cast<uint64_t*>(scratch));
    return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ECUDA;
}

namespace lbsph {

cudaError_t launch_particles(const PParams& p, cudaStream_t s)
{
    if (p.np <= 0) return cudaSuccess;
    const size_t smem = 2ull * p.smax * p.smax * sizeof(uint64_t);
    if (smem > 0) {        // static + dynamic may pass the 48 KB default: always opt in
        const cudaError_t e = cudaFuncSetAttribute(particle_crit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    particle_crit_kernel<<<p.np, CBLOCK, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_particles_aux(const PParams& p, cudaStream_t s)
{
    if (p.np <= 0) return cudaSuccess;
    const size_t smem = 2ull * p.smax * p.smax * sizeof(uint64_t);     // the new map, the partners' solids
    if (smem > 0) {        // static + dynamic may pass the 48 KB default: always opt in
        const cudaError_t e = cudaFuncSetAttribute(particle_aux_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    particle_aux_kernel<<<p.np, ABLOCK, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_links(const PartDev* pd, const PartK* pk, const uint64_t* rows, const BoxDev* boxes, int p, int* out,
                         int cap, int* count, cudaStream_t s)
{
    links_kernel<<<1, PBLOCK, 0, s>>>(pd, pk, rows, boxes, p, out, cap, count);
    return cudaGetLastError();
}

}  // namespace lbsph
