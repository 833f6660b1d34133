// Boundary kernel: the nodes next to a particle's surface, redone after the
// bulk kernel with the particle coupling of Sec. II.B and the remap of the
// Appendix (step 8):
//   - streaming with mid-link bounce-back where the source was solid at t-1:
//     f_i(x) = f*_{-i}(x) + 6 w_i rho0 (u_b . c_i), u_b = U + Omega x r_b (+ u_s),
//     r_b = x - c_i/2 - x_c (Eq. fb, Eq. ub, Eq. ubsquirmer);
//   - a node uncovered by the move starts from f_eq(rho0, U + Omega x r);
//   - a node covered by the move hands its mass and momentum to the particle;
//   - after the collision, the momentum-exchange sums of the new links (x fluid,
//     x + c_b solid) for Eq. F0 and Eq. T0.  Only two vectors per particle are
//     needed: sum c_b f*_b and sum m x c_b f*_b (m the node's cube-local
//     position; the torque arm's -c_b/2 drops out of c_b x c_b and the cube
//     origin is added by the particle kernel).
// Sums are kept per thread, reduced per warp, and go as int64 fixed point to
// the particle's accumulators (integer atomics: order independent).  The nodes
// are the ones the bulk kernel of this step skips (the redo mask written by
// the critical particle kernel of the step before), so this kernel writes them
// straight into the lattice while the bulk kernel streams the rest.
//
// Grid (blocks per particle, particles).  Block c of a particle takes the
// cube rows c, c + gx, c + 2 gx, ... and compacts the nodes of their redo
// words into a shared list.  Everything a block needs is fetched in one round
// of independent loads: the snapshot, both ring slots of the occupancy map,
// the redo words of its rows and the box terms of this collision.
#include "boundary_block.cuh"

namespace lbsph {

template <class St, bool FIRST>
__global__ void __launch_bounds__(BBLOCK, 2) boundary_kernel(const __grid_constant__ BndParams P)
{
    boundary_block<St, FIRST>(P, blockIdx.y, blockIdx.x);
}

template <class St>
static cudaError_t launch_bnd_t(const BndParams& p, dim3 grid, size_t smem, cudaStream_t s)
{
    if (smem > 0) {        // static + dynamic may pass the 48 KB default: always opt in
        cudaError_t e = cudaFuncSetAttribute(boundary_kernel<St, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(boundary_kernel<St, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (p.first) boundary_kernel<St, true><<<grid, BBLOCK, smem, s>>>(p);
    else boundary_kernel<St, false><<<grid, BBLOCK, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_boundary(const BndParams& p, int precision, int np, cudaStream_t s)
{
    if (np <= 0) return cudaSuccess;
    const dim3 grid(p.gx, np);
    const size_t smem = 2ull * p.smax * p.smax * sizeof(uint64_t) + (size_t)p.list_cap * sizeof(unsigned);
    if (precision == 1) return launch_bnd_t<StF16>(p, grid, smem, s);
    if (precision == 2) return launch_bnd_t<StBF16>(p, grid, smem, s);
    if (precision == 3) return launch_bnd_t<StF32G>(p, grid, smem, s);   // FP32, the paper's collision
    return launch_bnd_t<StF32>(p, grid, smem, s);
}

}  // namespace lbsph
