// D3Q27 path: the 27-velocity lattice the paper compares D3Q19 with
// (Sec. III.A), for periodic boxes holding at most one passive spheroid each,
// FP32 deviation storage, BGK or the paper's ghost-mode collision, with Guo
// forcing (q27.cu):
//   lattice   pull streaming of the last post-collision field with mid-link
//             bounce-back on the old surface (Eq. fb, Eq. ub), the remap of
//             covered / uncovered nodes to the new map (Appendix step 8), the
//             collision (Appendix step 1) and the integer momentum-exchange
//             sums of the new links (Eq. F0, T0); one pass over every node, or
//             (after the first step) a near pass over the nodes of each
//             particle's old and new cubes and a bulk pass over all others;
//   particle  one block per particle: F0, T0 and the remap terms, the
//             implicit solve (Eq. Fdiscrete, Tdiscrete), the pose update
//             (Eq. posupdate, qnplus0-1), the new occupancy map (Eq.
//             ellipsoidsurface, exact FP64 test near the surface) and the drag
//             matrix of its links (Eq. drag1-4), and the box's uniform terms of
//             the next collision.
// The iteration is the oracle's Appendix order turned by half a step: a
// lattice pass does the streaming, bounce-back and remap of iteration t-1 and
// the collision of iteration t, so the particle solve sits between two lattice
// passes and every population is read and written once per step.  The near
// pass and the particle kernel run on their own stream beside the bulk pass.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "lbsph_internal.cuh"

namespace lbsph {
namespace q27 {

constexpr int Q27 = 27;

// this library's D3Q27 order: the 19 directions of D3Q19 in their order, then
// the eight corners in +/- pairs (19 +++, 20 ---, 21 ++-, 22 --+, 23 +-+,
// 24 -+-, 25 -++, 26 +--); opp(i) = i + 1 for odd i, i - 1 for even i > 0
__host__ __device__ constexpr int cx27(int i)
{
    return i < 19 ? ((i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
                     : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0)
                  : ((i == 19 || i == 21 || i == 23 || i == 26) ? 1 : -1);
}
__host__ __device__ constexpr int cy27(int i)
{
    return i < 19 ? ((i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
                     : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0)
                  : ((i == 19 || i == 21 || i == 24 || i == 25) ? 1 : -1);
}
__host__ __device__ constexpr int cz27(int i)
{
    return i < 19 ? ((i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
                     : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0)
                  : ((i == 19 || i == 22 || i == 23 || i == 25) ? 1 : -1);
}
__host__ __device__ constexpr int opp27(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }
// weights for |c|^2 = 0, 1, 2, 3 (c_s^2 = 1/3)
__host__ __device__ constexpr double wd27(int i)
{
    return i == 0 ? 8.0 / 27.0 : (i <= 6 ? 2.0 / 27.0 : (i <= 18 ? 1.0 / 54.0 : 1.0 / 216.0));
}
__host__ __device__ constexpr float w27(int i) { return (float)wd27(i); }

// per box, constant
struct Box27 {
    int nx, ny, nz, counter;
    long long N, off;               // nodes; element offset of plane 0 in a distribution buffer
    int block_begin, nblocks;       // lattice-kernel blocks of this box
    float omega, rho0f;
    double rho0, body[3];
    int p;                          // the box's particle, or -1
    unsigned dx_m, dy_m;            // n / nx and n / ny as __umulhi(n, m) >> s (div_magic)
    int dx_s, dy_s;
    int pad;
};

// per box, written by the particle kernel for the next lattice pass (or by
// the host for a box without a particle)
struct Dyn27 {
    float g[3], eps;                // uniform force and mass return of the next collision
    int active;                     // 1: the box holds a particle
    int S;                          // cube side (rows of 64-bit words, S <= 64)
    int slot_old, slot_new;         // bitmap slots of the map the bounce-back uses and of the new map
    int o_old[3], o_new[3];         // cube origins wrapped into the box
    float U[3], W[3];               // velocities of the last solve (bounce-back and uncovered nodes)
    float phi_old[3], phi_new[3];   // cube origin - particle centre, old and new pose
    int uo[3], E[3];                // the box that holds both cubes: wrapped origin and extents
};

// per particle, FP64, read and written by the particle kernel only
struct Part27 {
    double semi[3], M, Ib[3], Fext[3], Text[3];
    double x[3], q[4], U[3], W[3];  // at time t
    double Iprev[9];                // lab inertia of the last solve (finite-difference rate)
    double inv2[3];                 // 1 / semi^2, rounded as the exact inside test rounds it
    float band;                     // FP32 decides a node farther than this from the surface value 1
    float fpad;
    double zeta[36];                // drag matrix of the links of the current map (Eq. drag1-4)
    double F0g[3], T0g[3];          // 2 rho0 sum w_b c_b and 2 rho0 sum w_b r_b x c_b over those links
    double phi[3];                  // cube origin - x of the current map
    double dP[3], dL[3], dm;        // terms of the last remap (dm: its mass, returned at the next collision)
    double rec[25];                 // F0, T0, F, T, U, Omega, x, q of the last iteration
    int o[3];                       // unwrapped cube origin of the current map
    int S, h, slot, nsolid, box;
    int pad;
};

// lattice pass modes: every node; every node outside the particles' cube
// unions (bulk); the nodes of the cube unions only (near: block b takes
// particle b / nbpp)
enum { LAT_ALL = 0, LAT_BULK = 1, LAT_NEAR = 2 };

struct LatParams27 {
    const Box27* boxes;
    const Dyn27* dyn;
    const Part27* pd;               // LAT_NEAR: the box of each particle
    const int* blk_box;             // box of every lattice block
    const uint64_t* rows;           // [np][2][64*64] occupancy bitmaps
    long long* acc;                 // [np][24] integer link and remap sums
    const float* src;               // post-collision deviations of t-1 (first: the initial field)
    float* dst;
    int first;                      // 1: collide the stored field, no streaming
    int mode;                       // LAT_ALL, LAT_BULK or LAT_NEAR
    int nbpp;                       // LAT_NEAR: blocks per particle (covering (S + 1)^3 nodes)
    int ghost;                      // 1: the paper's ghost-mode collision, 0: BGK
};

struct PartParams27 {
    Part27* pd;
    Dyn27* dyn;
    const Box27* boxes;
    uint64_t* rows;
    long long* acc;
    unsigned* status;
    int init;                       // 1: map, drag matrix and box terms of the current pose only
    int didt_mode;
};

struct FieldParams27 {
    const Box27* boxes;
    const Dyn27* dyn;
    const uint64_t* rows;
    const float* src;
    int box, nopull, out_dev;
    float* out_f;                   // [27][N] or null
    float* out_rho;                 // [N] rho - rho0 or null
    float* out_u;                   // [3][N] or null
    int* out_solid;                 // [N] or null
};

cudaError_t launch_lattice27(const LatParams27& p, int blocks, cudaStream_t s);
cudaError_t launch_bulk27(const LatParams27& p, int blocks, cudaStream_t s);   // LAT_BULK only
cudaError_t launch_particles27(const PartParams27& p, int np, cudaStream_t s);
cudaError_t launch_fields27(const FieldParams27& p, int blocks, cudaStream_t s);
cudaError_t launch_refresh27(const Part27* pd, const Box27* boxes, Dyn27* dyn, int np, cudaStream_t s);
cudaError_t launch_links27(const Part27* pd, const Box27* boxes, const uint64_t* rows, int p, int* out, int cap,
                           int* count, cudaStream_t s);

}  // namespace q27
}  // namespace lbsph
