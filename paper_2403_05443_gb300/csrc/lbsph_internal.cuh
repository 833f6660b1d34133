// Internal definitions shared by the CUDA translation units of liblbsph.
//
// One iteration t of the paper's Appendix is four kernels on three streams:
//   main stream
//     bulk      every node except those next to a particle's surface: pull
//               streaming + BGK/Guo collision, wall links inline (the only
//               kernel that moves the whole lattice: 2*19*s bytes/node);
//   particle stream (runs while the bulk kernel streams the lattice)
//     boundary  the nodes next to a particle's old or new surface, with link
//               bounce-back (Eq. fb, Eq. ub), the remap of covered / uncovered
//               nodes and the momentum-exchange sums of the new links, written
//               straight into the lattice (the bulk kernel skips them);
//     particle  (critical) force, implicit solve with the inverse prepared by
//               the auxiliary kernel, pose and quaternion update, the new
//               occupancy map, the nodes both lattice kernels split at t+1 and
//               the box's uniform forces for the next step;
//   auxiliary stream (overlaps the next boundary kernel)
//     particle  (auxiliary) integer link sums of the new map, drag matrices (Eq.
//               drag1-drag4), the inverse of the next implicit solve and the
//               geometric parts of F0 / T0.
//
// Data layout in HBM (one allocation per buffer, every box back to back):
//   distributions  two buffers (ping-pong), each box b holds 19 planes of
//                  N_b = nx*ny*nz stored deviations f_i - w_i rho0, plane i at
//                  box_off + i*N_b, x fastest (SoA), so a warp reads one row of
//                  a plane with 16-byte loads (4 nodes per thread).
//   occupancy      per particle a ring of two bitmaps over its bounding cube
//                  (side S <= 64): one 64-bit word per (y, z) row, bit x set
//                  when the node is inside the particle (Eq. ellipsoidsurface).
//                  Boundary links are implicit: (x fluid, x + c_b solid).
//   redo masks     per particle and buffer parity, the nodes the boundary
//                  kernel takes over at one step: one 64-bit word per row of
//                  the particle's current cube, with the cube in a NeedHdr.
//   particle state PartDev (FP64, owned by the particle kernels) and PartK (the
//                  FP32 snapshot the lattice kernels read).
//   accumulators   per particle NACC int64 fixed-point sums filled by the
//                  boundary kernel with integer atomics (order independent, so
//                  every run is bitwise reproducible) and drained by the
//                  critical particle kernel.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace lbsph {

constexpr int Q = 19;
constexpr int MAXS = 64;            // largest bounding-cube side (one 64-bit word per row)
constexpr int RECD = 25;            // doubles per particle record (LB_RECORD_DOUBLES of the C ABI)
constexpr int KBLOCK = 256;         // threads per block of the lattice kernel
constexpr int PBLOCK = 512;         // threads per block of the links read-back kernels
constexpr int ABLOCK = 256;         // threads per block of the auxiliary particle kernel
constexpr int MAXC = 4;             // particles a lattice tile may touch (field read-back)
constexpr int BBLOCK = 256;         // threads per block of the boundary kernel
constexpr int CBLOCK = 256;         // threads per block of the critical particle kernel
constexpr int MAXAMB = 512;         // near-surface nodes settled by the exact FP64 test per step
constexpr int SYNC_HDR = 8;          // step kernel: barrier and work-counter words before the per-particle item counters
constexpr int MAXNB = 8;            // partners of a particle: others whose bounding cubes come within reach
constexpr int MAXPB = 64;           // particles of one box when any of them has partners (cluster masks)
constexpr int RINGD = 10;           // doubles per particle and step parity in the pose ring: x, U, q

// accumulator layout (int64 per particle); d = fixed-point f* of a link (x, b),
// m = cube-local position of x
constexpr int ACC_F = 0;            // sum over links of c_b d                [3]
constexpr int ACC_T = 3;            // sum over links of m x (c_b d)          [3]
constexpr int ACC_COV = 6;          // n, sum drho, J[3], sum m x j [3]
constexpr int ACC_UNC = 14;         // n, sum m [3], sum m m^T [6: xx xy xz yy yz zz]
constexpr int NACC = 24;
constexpr float FIXF = 70368744177664.0f;    // 2^46: |deviation| * 63 * 2^46 * links stays < 2^63
constexpr double FIXD = 70368744177664.0;

// status bits of the device status word
constexpr unsigned ST_NAN = 1u;
constexpr unsigned ST_CAPACITY = 2u;
constexpr unsigned ST_OVERLAP = 4u;
constexpr unsigned ST_TIMEOUT = 8u;  // a grid barrier of the step kernel gave up waiting

// cube margin: h = ceil(max semi-axis) + CUBE_MARGIN, side S = 2h + 2, so the
// solid nodes of this step and of the last one, grown by one link, stay inside
// the cube while a particle moves less than one node per step
constexpr int CUBE_MARGIN = 2;

// ---------------------------------------------------------------------------
// D3Q19, this library's order: rest, 6 faces in +/- pairs, 12 edges in +/- pairs.
// opp(i) = i + 1 for odd i, i - 1 for even i > 0.
__host__ __device__ constexpr int cx_of(int i)
{
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy_of(int i)
{
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz_of(int i)
{
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr int opp_of(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
__host__ __device__ constexpr float w_of(int i)
{
    return i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
}
__host__ __device__ constexpr double wd_of(int i)
{
    return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// ---------------------------------------------------------------------------
struct BoxDev {
    int nx, ny, nz, nxq;            // nxq = nx / 4 quads per row
    long long N;                    // nodes
    long long nq;                   // quads
    long long off;                  // element offset of plane 0 in a distribution buffer
    int block_begin, nblocks;       // lattice-kernel blocks of this box
    float omega;                    // 1 / tau
    float rho0f;
    double rho0;
    double body[3];
    int counter;                    // counter body force on
    int walls;
    float uw_lo[3], uw_hi[3];
    int pbeg, pcnt;                 // particles of this box
    long long nwall;                // wall nodes (2 nx nz when walls)
    float scale, inv_scale;         // 16-bit storage scale (1 for FP32 / BF16)
    double lub_cut, mu;             // lubrication cut-off gap (0: none), dynamic viscosity rho0 (tau - 1/2) / 3
    unsigned dq_m, dy_m;            // q / nxq and row / ny as __umulhi(n, m) >> s (div_magic)
    int dq_s, dy_s;
    int rowwarp;                    // 1: nxq divides 32, every row lies within one warp's 32 quads
};

// Division by a box constant d without a divide: n / d == (n m / 2^32) >> s
// for 0 <= n < 2^31, with l = ceil(log2 d), m = ceil(2^(31+l) / d) and
// s = l - 1 (m < 2^32).  m exceeds 2^(31+l) / d by less than 1, so n m / 2^(31+l)
// exceeds n / d by less than n / 2^(31+l) < 1 / d, which cannot reach the next
// integer (the fraction of n / d is at most 1 - 1/d).  d = 1 gives s = -1.
inline void magic_div(unsigned d, unsigned& m, int& s)
{
    if (d <= 1) {
        m = 0;
        s = -1;
        return;
    }
    int l = 0;
    while ((1ull << l) < d) ++l;
    const unsigned long long num = 1ull << (31 + l);
    m = (unsigned)((num + d - 1) / d);
    s = l - 1;
}

// n / d for 0 <= n < 2^31 with the multiplier and shift of magic_div (s < 0: d = 1)
__host__ __device__ __forceinline__ int div_magic(int n, unsigned m, int s)
{
#ifdef __CUDA_ARCH__
    return s < 0 ? n : (int)(__umulhi((unsigned)n, m) >> s);
#else
    return s < 0 ? n : (int)((((unsigned long long)(unsigned)n * m) >> 32) >> s);
#endif
}

// FP32 snapshot of one particle for the lattice kernels, written by the
// critical particle kernel of iteration t for the kernels of iteration t+1.
struct PartK {
    const uint64_t* rows_old;       // occupancy of the pose at t   (map t)
    const uint64_t* rows_new;       // occupancy of the pose at t+1 (map t+1)
    int ow_old[3], ow_new[3];       // cube origins wrapped into the box
    int oy_new;                     // y of the new cube origin, not wrapped (wall rows)
    int S;                          // cube side
    int box;
    float ro_old[3];                // origin(t) - x_c(t)     (r = ro + m [+ c/2])
    float ro_new[3];                // origin(t+1) - x_c(t+1)
    float U[3], W[3];               // U(t+1), Omega(t+1)
    float e_old[3];                 // body x axis at t (squirmer slip)
    float a, b, eps2, B1, B2;       // squirmer parameters
    int squirmer;
    int nsolid;                     // solid nodes of map t+1
    double dm_return;               // mass put back at the next collision
    double Fext[3];
    // the particle's box (constant, set with the particles), so that no kernel
    // of the particle chain needs a second dependent load
    long long N, off, nwall;
    double rho0;
    int nx, ny, nz, walls;
    float omega, rho0f, scale, inv_scale;
    float uw_lo[3], uw_hi[3];
    float body[3];
    int counter;                    // counter body force on
    int pbeg, pcnt;                 // particles of the box
    double lub_cut, mu;             // the box's lubrication cut-off and viscosity
    // partners: the other particles of the box whose bounding cubes come within
    // reach of this one's (symmetric); their boundary nodes, links, covered and
    // uncovered nodes interleave with this particle's
    int nnb;
    int nb[MAXNB];
};

// cube of a particle's redo mask: origin wrapped into the box, side
struct NeedHdr {
    int ow[3];
    int S;
};

// uniform per-box terms of the next collision: body force g and mass return eps
struct BoxDyn {
    float g[3];
    float eps;
};

// Full FP64 state of one particle, read and written by the particle kernels only.
struct PartDev {
    double semi[3], M, Ib[3], density, B1, B2;
    double Fext[3], Text[3];        // adjacent: lb_set_external copies the six together
    double x[3], q[4], U[3], W[3];  // at time t (before the critical kernel of t)
    double inv_semi2[3];            // 1 / semi^2, rounded as the exact inside test rounds it
    // prepared by the auxiliary kernel of t-1 for the critical kernel of t
    double Icur[9];                 // lab-frame inertia at q(t) (Eq. Irot)
    double zeta[36];                // drag matrix of links(t) (Eq. drag1-drag4)
    double Ainv[36];                // inverse of the matrix of Eq. Fdiscrete / Eq. Tdiscrete
    double F0g[3], T0g[3];          // parts of F0, T0 fixed by links(t) alone (Eq. F0, Eq. T0)
    double phi[3];                  // cube origin of map t - x_c(t)
    int o[3];                       // cube origin (unwrapped) of map t
    int o_prev[3];                  // cube origin of map t-1
    int S, h, box, slot;            // slot: ring slot holding map t
    long long step;
    double rec[RECD];               // F0, T0, F, T, U, Omega, x, q of the last iteration
    long long aux_step;             // value of `step` the auxiliary block last ran for (-1: none)
    long long lsum[27];             // the auxiliary block's integer link sums of its map
    long long lsum_step;            // value of `step` they belong to (-1: none)
    int nsolid, pad;
};

static_assert(sizeof(PartDev) % 8 == 0, "PartDev is copied as 8-byte words");
static_assert(sizeof(PartK) % 4 == 0, "PartK is copied as 4-byte words");

struct KParams {
    const BoxDev* boxes;
    int nbox;
    const PartK* pk;
    const void* src;                // distributions of iteration t-1 (post-collision)
    unsigned* status;
    // outputs (one box)
    float* out_f;                   // [19][N] or nullptr
    int out_dev;                    // 1: out_f holds deviations, 0: full f
    float* out_rho;                 // [N] rho - rho0 or nullptr
    float* out_u;                   // [3][N] or nullptr
    int* out_solid;                 // [N] or nullptr
    int only_box;                   // box index (the grid covers that box only)
    int nopull;                     // before the first collision: f = w rho0, no streaming
};

struct PParams {
    PartDev* pd;
    PartK* pk;
    long long* acc;                 // np * NACC
    uint64_t* rows;                 // np * 2 * MAXS*MAXS words
    const BoxDev* boxes;
    BoxDyn* box_dyn;                // per box, for the next collision (slot of the next iteration)
    BoxDyn* pdyn;                   // the same per particle (the boundary kernel's copy)
    int* box_done;                  // per box arrival counters (boxes with several particles)
    NeedHdr* need_hdr;              // per particle: redo mask of the next step (written)
    uint64_t* need;                 // per particle MAXS*MAXS words (written)
    unsigned* status;
    double* ring;                   // [np][2][RINGD]: x, U, q at time t in slot t & 1 (partners read it)
    int np;
    int init;                       // 1: build maps / moments only (no solve, no pose update)
    int didt_mode;
    int smax;                       // largest cube side of the context (sizes dynamic shared memory)
};

struct BulkParams {
    const BoxDev* boxes;
    const int* blk_box;             // box of every bulk block
    const BoxDyn* box_dyn;
    const NeedHdr* need_hdr;        // per particle: the nodes left to the boundary kernel
    const uint64_t* need;           // per particle MAXS*MAXS words
    const void* src;
    void* dst;
    int first;                      // 1: first collision of the run (rest state, no streaming)
};

struct BndParams {
    const BoxDyn* pdyn;             // per particle: the box's uniform terms of this collision
    const PartK* pk;
    long long* acc;                 // np * NACC
    const uint64_t* rows;           // np * 2 * MAXS*MAXS words (both ring slots)
    const uint64_t* need;           // per particle MAXS*MAXS words: the nodes to redo
    const NeedHdr* need_hdr;        // per particle: the cube of its redo mask (partners' nodes)
    unsigned* status;
    const void* src;
    void* dst;                      // the lattice buffer of this step (written directly)
    int list_cap;                   // node list entries per block (shared memory)
    int first;
    int smax;                       // largest cube side (sizes dynamic shared memory)
    int gx;                         // blocks per particle; block c takes cube rows c, c + gx, ...
};

inline int rows_stride() { return MAXS * MAXS; }

}  // namespace lbsph
