// Boundary kernel: the nodes next to a particle's surface, redone after the
// bulk kernel with the particle coupling of Sec. II.B and the remap of the
// Appendix (step 8):
//   - streaming with mid-link bounce-back where the source was solid at t-1:
//     f_i(x) = f*_{-i}(x) + 6 w_i rho0 (u_b . c_i), u_b = U + Omega x r_b (+ u_s),
//     r_b = x - c_i/2 - x_c (Eq. fb, Eq. ub, Eq. ubsquirmer);
//   - a node uncovered by the move starts from f_eq(rho0, U + Omega x r);
//   - a node covered by the move hands its mass and momentum to the particle;
//   - after the collision, the momentum-exchange sums sum f*_b and sum f*_b m of
//     the new links (x fluid, x + c_b solid) per direction b (Eq. F0, Eq. T0).
// Sums go to block-level shared accumulators and then, as int64 fixed point,
// to the particle's accumulators (integer atomics: order independent).
//
// One thread per listed node; grid (ceil(capacity / 128), particles): blocks
// past a particle's list length exit at once.
#include "lattice_common.cuh"

namespace lbsph {

__device__ __forceinline__ bool bit_at(const uint64_t* rows, int S, const int ow[3], int X, int Y, int Z, int nx,
                                       int ny, int nz, int& mx, int& my, int& mz)
{
    mx = wrapd(X - ow[0], nx);
    my = wrapd(Y - ow[1], ny);
    mz = wrapd(Z - ow[2], nz);
    if (mx >= S || my >= S || mz >= S) return false;
    return (rows[mz * S + my] >> mx) & 1ull;
}

__device__ __forceinline__ void acc_add(long long* a, long long v)
{
    if (v != 0) atomicAdd(reinterpret_cast<unsigned long long*>(a), static_cast<unsigned long long>(v));
}

template <class St, bool FIRST>
__global__ void __launch_bounds__(BBLOCK) boundary_kernel(const BndParams P)
{
    using T = typename St::T;
    const int p = blockIdx.y;
    const PartK& K = P.pk[p];
    const int count = *K.list_count;
    const int e = blockIdx.x * BBLOCK + threadIdx.x;
    if (blockIdx.x * BBLOCK >= count) return;       // whole block past the list
    __shared__ long long s_acc[NACC];
    for (int j = threadIdx.x; j < NACC; j += BBLOCK) s_acc[j] = 0;
    __syncthreads();

    const BoxDev& B = P.boxes[K.box];
    const int nx = B.nx, ny = B.ny, nz = B.nz;
    const long long N = B.N;
    const T* A = reinterpret_cast<const T*>(P.src) + B.off;
    T* D = reinterpret_cast<T*>(P.dst) + B.off;
    const float inv = B.inv_scale, rho0 = B.rho0f;
    const int S = K.S;

    if (e < count) {
        const unsigned code = K.list[e];
        const int mx = code & 0xff, my = (code >> 8) & 0xff, mz = (code >> 16) & 0xff;
        const int X = wrapd(K.ow_new[0] + mx, nx), Y = wrapd(K.ow_new[1] + my, ny), Z = wrapd(K.ow_new[2] + mz, nz);
        const long long own = ((long long)Z * ny + Y) * nx + X;
        const bool wallrow = B.walls && (Y == 0 || Y == ny - 1);
        const bool sol_new = (K.rows_new[mz * S + my] >> mx) & 1ull;
        int ox, oy, oz;
        const bool sol_old = !FIRST && bit_at(K.rows_old, S, K.ow_old, X, Y, Z, nx, ny, nz, ox, oy, oz);
        const float ex[3] = {K.e_old[0], K.e_old[1], K.e_old[2]};
        float f[Q];
        bool write = !wallrow;
        if (wallrow || (sol_new && (sol_old || FIRST))) {
            write = false;                          // solid before and after: untouched
        } else if (sol_old) {
            // uncovered: f = f_eq(rho0, U + Omega x r) with r = x - x_c(t)
            const float rx = K.ro_new[0] + mx, ry = K.ro_new[1] + my, rz = K.ro_new[2] + mz;
            const float ux = K.U[0] + (K.W[1] * rz - K.W[2] * ry);
            const float uy = K.U[1] + (K.W[2] * rx - K.W[0] * rz);
            const float uz = K.U[2] + (K.W[0] * ry - K.W[1] * rx);
            const float uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const float cu = cx_of(i) * ux + cy_of(i) * uy + cz_of(i) * uz;
                f[i] = w_of(i) * rho0 * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu);
            }
            long long* a = s_acc + ACC_UNC;
            acc_add(a + 0, 1);
            acc_add(a + 1, mx); acc_add(a + 2, my); acc_add(a + 3, mz);
            acc_add(a + 4, mx * mx); acc_add(a + 5, mx * my); acc_add(a + 6, mx * mz);
            acc_add(a + 7, my * my); acc_add(a + 8, my * mz); acc_add(a + 9, mz * mz);
        } else {
            // fluid at t-1: pull, with bounce-back from solid sources and walls
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if (FIRST) { f[i] = 0.0f; continue; }
                const int Xs = wrapd(X - cx_of(i), nx), Ys = Y - cy_of(i), Zs = wrapd(Z - cz_of(i), nz);
                if (i > 0 && B.walls && (Ys == 0 || Ys == ny - 1)) {
                    const float* uw = (Ys == 0) ? B.uw_lo : B.uw_hi;
                    const float ubc = cx_of(i) * uw[0] + cy_of(i) * uw[1] + cz_of(i) * uw[2];
                    f[i] = St::ld1(A + (long long)opp_of(i) * N + own, inv) + 6.0f * w_of(i) * rho0 * ubc;
                    continue;
                }
                const int Ysw = wrapd(Ys, ny);
                int sx, sy, sz;
                if (i > 0 && bit_at(K.rows_old, S, K.ow_old, Xs, Ysw, Zs, nx, ny, nz, sx, sy, sz)) {
                    const float rx = K.ro_old[0] + sx + 0.5f * cx_of(i);
                    const float ry = K.ro_old[1] + sy + 0.5f * cy_of(i);
                    const float rz = K.ro_old[2] + sz + 0.5f * cz_of(i);
                    float ux = K.U[0] + (K.W[1] * rz - K.W[2] * ry);
                    float uy = K.U[1] + (K.W[2] * rx - K.W[0] * rz);
                    float uz = K.U[2] + (K.W[0] * ry - K.W[1] * rx);
                    if (K.squirmer) {
                        float qx, qy, qz;
                        squirmer_slip(ex, K.a, K.eps2, K.B1, K.B2, rx, ry, rz, qx, qy, qz);
                        ux += qx; uy += qy; uz += qz;
                    }
                    const float ubc = cx_of(i) * ux + cy_of(i) * uy + cz_of(i) * uz;
                    f[i] = St::ld1(A + (long long)opp_of(i) * N + own, inv) + 6.0f * w_of(i) * rho0 * ubc;
                } else {
                    f[i] = St::ld1(A + (long long)i * N + ((long long)Zs * ny + Ysw) * nx + Xs, inv);
                }
            }
            if (sol_new) {
                // covered: mass and momentum go to the particle's next solve
                write = false;
                float drho = 0.f;
#pragma unroll
                for (int i = 0; i < Q; ++i) drho += f[i];
                const float jx = (f[1] - f[2]) + (f[7] - f[8]) + (f[9] - f[10]) + (f[11] - f[12]) + (f[13] - f[14]);
                const float jy = (f[3] - f[4]) + (f[7] - f[8]) - (f[9] - f[10]) + (f[15] - f[16]) + (f[17] - f[18]);
                const float jz = (f[5] - f[6]) + (f[11] - f[12]) - (f[13] - f[14]) + (f[15] - f[16]) - (f[17] - f[18]);
                const long long Jx = fixp(jx), Jy = fixp(jy), Jz = fixp(jz);
                long long* a = s_acc + ACC_COV;
                acc_add(a + 0, 1);
                acc_add(a + 1, fixp(drho));
                acc_add(a + 2, Jx); acc_add(a + 3, Jy); acc_add(a + 4, Jz);
                acc_add(a + 5, my * Jz - mz * Jy);
                acc_add(a + 6, mz * Jx - mx * Jz);
                acc_add(a + 7, mx * Jy - my * Jx);
            }
        }
        if (write) {
            const BoxDyn dyn = P.box_dyn[K.box];
            collide19(f, B.omega, rho0, dyn.g[0], dyn.g[1], dyn.g[2], dyn.eps);
#pragma unroll
            for (int i = 0; i < Q; ++i) St::st1(D + (long long)i * N + own, f[i], B.scale);
            // momentum-exchange sums of the links (x, b) of the new map, with f*(t)
#pragma unroll
            for (int b = 1; b < Q; ++b) {
                const int m2x = mx + cx_of(b), m2y = my + cy_of(b), m2z = mz + cz_of(b);
                if (m2x < 0 || m2x >= S || m2y < 0 || m2y >= S || m2z < 0 || m2z >= S) continue;
                if (!((K.rows_new[m2z * S + m2y] >> m2x) & 1ull)) continue;
                const long long d = fixp(f[b]);
                long long* a = s_acc + ACC_LINK + 4 * b;
                acc_add(a + 0, d);
                acc_add(a + 1, d * mx);
                acc_add(a + 2, d * my);
                acc_add(a + 3, d * mz);
            }
        } else if (sol_new && !wallrow) {
            // a solid node keeps finite contents: zero it (never read as a source)
#pragma unroll
            for (int i = 0; i < Q; ++i) St::st1(D + (long long)i * N + own, 0.0f, B.scale);
        }
    }
    __syncthreads();
    for (int j = threadIdx.x; j < NACC; j += BBLOCK) {
        const long long v = s_acc[j];
        if (v != 0) atomicAdd(reinterpret_cast<unsigned long long*>(K.acc + j), static_cast<unsigned long long>(v));
    }
}

template <class St>
static cudaError_t launch_bnd_t(const BndParams& p, dim3 grid, cudaStream_t s)
{
    if (p.first) boundary_kernel<St, true><<<grid, BBLOCK, 0, s>>>(p);
    else boundary_kernel<St, false><<<grid, BBLOCK, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_boundary(const BndParams& p, int precision, int list_cap, int np, cudaStream_t s)
{
    if (np <= 0) return cudaSuccess;
    const dim3 grid((list_cap + BBLOCK - 1) / BBLOCK, np);
    if (precision == 1) return launch_bnd_t<StF16>(p, grid, s);
    if (precision == 2) return launch_bnd_t<StBF16>(p, grid, s);
    return launch_bnd_t<StF32>(p, grid, s);
}

}  // namespace lbsph
