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
// to the particle's accumulators (integer atomics: order independent).  The
// node values go to a side buffer; the scatter kernel writes them into the
// lattice after the bulk kernel, so this kernel (and the particle kernels after
// it) can run while the bulk kernel streams the lattice.
//
// One thread per listed node; grid (ceil(capacity / 128), particles): blocks
// past a particle's list length exit at once.
#include "lattice_common.cuh"

namespace lbsph {

__device__ __forceinline__ void acc_add(long long* a, long long v)
{
    if (v != 0) atomicAdd(reinterpret_cast<unsigned long long*>(a), static_cast<unsigned long long>(v));
}

__device__ __forceinline__ long long warp_sum(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += (long long)__shfl_xor_sync(0xffffffffu, (unsigned long long)v, o);
    return v;
}

template <class St, bool FIRST>
__global__ void __launch_bounds__(BBLOCK) boundary_kernel(const BndParams P)
{
    using T = typename St::T;
    const int p = blockIdx.y;
    const int count = *P.pk[p].list_count;
    // the scatter kernel reads this count: the auxiliary kernel rewrites list_count meanwhile
    if (blockIdx.x == 0 && threadIdx.x == 0) *P.pk[p].side_count = count;
    if (blockIdx.x * BBLOCK >= count) return;       // whole block past the list
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int e = blockIdx.x * BBLOCK + tid;

    extern __shared__ uint64_t s_bits[];            // new map, then old map in new-cube coordinates
    __shared__ PartK K;
    __shared__ long long s_acc[NACC];
    __shared__ long long s_part[BBLOCK / 32][Q][4];
    {
        const unsigned* src = reinterpret_cast<const unsigned*>(P.pk + p);
        unsigned* dst = reinterpret_cast<unsigned*>(&K);
        for (int j = tid; j < (int)(sizeof(PartK) / 4); j += BBLOCK) dst[j] = src[j];
        for (int j = tid; j < NACC; j += BBLOCK) s_acc[j] = 0;
    }
    __syncthreads();
    const int S = K.S;
    uint64_t* s_new = s_bits;
    uint64_t* s_old = s_bits + S * S;
    const BoxDev& B = P.boxes[K.box];
    const int nx = B.nx, ny = B.ny, nz = B.nz;
    int d[3];                                       // o_new - o_old (cube origins)
    {
        // old map in new-cube coordinates: new-local m is old-local m - d
        for (int k = 0; k < 3; ++k) {
            const int L = k == 0 ? nx : (k == 1 ? ny : nz);
            int v = K.ow_new[k] - K.ow_old[k];
            if (v > L / 2) v -= L;
            if (v < -L / 2) v += L;
            d[k] = FIRST ? 0 : v;
        }
        const uint64_t maskS = S >= 64 ? ~0ull : ((1ull << S) - 1ull);
        for (int r = tid; r < S * S; r += BBLOCK) {
            s_new[r] = K.rows_new[r];
            const int my = r % S + d[1], mz = r / S + d[2];
            uint64_t w = 0;
            if (my >= 0 && my < S && mz >= 0 && mz < S) {
                w = K.rows_old[mz * S + my];
                w = d[0] == 1 ? (w >> 1) : (d[0] == -1 ? (w << 1) : w);
                w &= maskS;
            }
            s_old[r] = w;
        }
    }
    __syncthreads();

    const long long N = B.N;
    const T* A = reinterpret_cast<const T*>(P.src) + B.off;
    const float inv = B.inv_scale, rho0 = B.rho0f;
    unsigned lmask = 0;                             // directions b with a new link (x, b)
    float f[Q];
    int mx = 0, my = 0, mz = 0;
    if (e < count) {
        const unsigned code = K.list[e];
        mx = code & 0xff; my = (code >> 8) & 0xff; mz = (code >> 16) & 0xff;
        const int X = wrapd(K.ow_new[0] + mx, nx), Y = wrapd(K.ow_new[1] + my, ny), Z = wrapd(K.ow_new[2] + mz, nz);
        const long long own = ((long long)Z * ny + Y) * nx + X;
        const bool wallrow = B.walls && (Y == 0 || Y == ny - 1);
        auto bit = [&](const uint64_t* rows, int ax, int ay, int az) -> bool {
            if (ax < 0 || ax >= S || ay < 0 || ay >= S || az < 0 || az >= S) return false;
            return (rows[az * S + ay] >> ax) & 1ull;
        };
        const bool sol_new = bit(s_new, mx, my, mz);
        const bool sol_old = !FIRST && bit(s_old, mx, my, mz);
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
        } else if (FIRST) {
#pragma unroll
            for (int i = 0; i < Q; ++i) f[i] = 0.0f;
        } else {
            // fluid at t-1: decide every source first, then issue the 19 loads together
            unsigned bb = 0, wl = 0;
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                const int Ys = Y - cy_of(i);
                if (B.walls && (Ys == 0 || Ys == ny - 1)) wl |= 1u << i;
                else if (bit(s_old, mx - cx_of(i), my - cy_of(i), mz - cz_of(i))) bb |= 1u << i;
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const bool back = ((bb | wl) >> i) & 1u;
                const long long src = back ? (long long)opp_of(i) * N + own
                                           : (long long)i * N + ((long long)wrapd(Z - cz_of(i), nz) * ny + wrapd(Y - cy_of(i), ny)) * nx +
                                                 wrapd(X - cx_of(i), nx);
                f[i] = St::ld1(A + src, inv);
            }
            // mid-link bounce-back terms: + 6 w_i rho0 (u_b . c_i) (Eq. fb, Eq. ub, Eq. ubsquirmer)
            const float ex[3] = {K.e_old[0], K.e_old[1], K.e_old[2]};
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                if (!(((bb | wl) >> i) & 1u)) continue;
                float ubc;
                if ((wl >> i) & 1u) {
                    const float* uw = (Y - cy_of(i) == 0) ? B.uw_lo : B.uw_hi;
                    ubc = cx_of(i) * uw[0] + cy_of(i) * uw[1] + cz_of(i) * uw[2];
                } else {
                    // r_b = x - c_i/2 - x_c(t-1) = ro_old + d + m - c_i/2
                    const float px = K.ro_old[0] + (float)(d[0] + mx) - 0.5f * cx_of(i);
                    const float py = K.ro_old[1] + (float)(d[1] + my) - 0.5f * cy_of(i);
                    const float pz = K.ro_old[2] + (float)(d[2] + mz) - 0.5f * cz_of(i);
                    float ux = K.U[0] + (K.W[1] * pz - K.W[2] * py);
                    float uy = K.U[1] + (K.W[2] * px - K.W[0] * pz);
                    float uz = K.U[2] + (K.W[0] * py - K.W[1] * px);
                    if (K.squirmer) {
                        float qx, qy, qz;
                        squirmer_slip(ex, K.a, K.eps2, K.B1, K.B2, px, py, pz, qx, qy, qz);
                        ux += qx; uy += qy; uz += qz;
                    }
                    ubc = cx_of(i) * ux + cy_of(i) * uy + cz_of(i) * uz;
                }
                f[i] += 6.0f * w_of(i) * rho0 * ubc;
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
            float* sv = K.side_val + (long long)e * Q;
#pragma unroll
            for (int i = 0; i < Q; ++i) sv[i] = f[i];
            K.side_idx[e] = (int)own;
#pragma unroll
            for (int b = 1; b < Q; ++b)
                if (bit(s_new, mx + cx_of(b), my + cy_of(b), mz + cz_of(b))) lmask |= 1u << b;
        } else if (sol_new && !wallrow) {
            K.side_idx[e] = -2 - (int)own;          // solid now: zero it (never read as a source)
        } else {
            K.side_idx[e] = -1;
        }
    }
    // momentum-exchange sums of the new links (x, b), with f*(t): per direction,
    // a warp reduction over the lanes that have that link, then per warp to shared
    const unsigned wmask = __reduce_or_sync(0xffffffffu, lmask);
#pragma unroll
    for (int b = 1; b < Q; ++b) {
        if (!((wmask >> b) & 1u)) {
            if (lane == 0) { s_part[warp][b][0] = s_part[warp][b][1] = s_part[warp][b][2] = s_part[warp][b][3] = 0; }
            continue;
        }
        const long long d = ((lmask >> b) & 1u) ? fixp(f[b]) : 0ll;
        const long long v0 = warp_sum(d), v1 = warp_sum(d * mx), v2 = warp_sum(d * my), v3 = warp_sum(d * mz);
        if (lane == 0) { s_part[warp][b][0] = v0; s_part[warp][b][1] = v1; s_part[warp][b][2] = v2; s_part[warp][b][3] = v3; }
    }
    __syncthreads();
    for (int j = tid; j < NACC; j += BBLOCK) {
        long long v = s_acc[j];
        if (j >= 4 && j < ACC_COV) {
            const int b = j / 4, k = j % 4;
#pragma unroll
            for (int w = 0; w < BBLOCK / 32; ++w) v += s_part[w][b][k];
        }
        if (v != 0) atomicAdd(reinterpret_cast<unsigned long long*>(K.acc + j), static_cast<unsigned long long>(v));
    }
}

// Writes the boundary kernel's node values into the lattice buffer of
// iteration t (after the bulk kernel has written its provisional values).
template <class St>
__global__ void __launch_bounds__(BBLOCK) scatter_kernel(const BndParams P)
{
    using T = typename St::T;
    const int p = blockIdx.y;
    const PartK& K = P.pk[p];
    const int count = *K.side_count;
    const int e = blockIdx.x * BBLOCK + threadIdx.x;
    if (e >= count) return;
    const BoxDev& B = P.boxes[K.box];
    T* D = reinterpret_cast<T*>(P.dst) + B.off;
    const int idx = K.side_idx[e];
    if (idx == -1) return;
    const long long N = B.N;
    if (idx >= 0) {
        const float* sv = K.side_val + (long long)e * Q;
#pragma unroll
        for (int i = 0; i < Q; ++i) St::st1(D + (long long)i * N + idx, sv[i], B.scale);
    } else {
        const long long own = -2 - idx;
#pragma unroll
        for (int i = 0; i < Q; ++i) St::st1(D + (long long)i * N + own, 0.0f, B.scale);
    }
}

template <class St>
static cudaError_t launch_scatter_t(const BndParams& p, dim3 grid, cudaStream_t s)
{
    scatter_kernel<St><<<grid, BBLOCK, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const BndParams& p, int precision, int list_cap, int np, cudaStream_t s)
{
    if (np <= 0) return cudaSuccess;
    const dim3 grid((list_cap + BBLOCK - 1) / BBLOCK, np);
    if (precision == 1) return launch_scatter_t<StF16>(p, grid, s);
    if (precision == 2) return launch_scatter_t<StBF16>(p, grid, s);
    return launch_scatter_t<StF32>(p, grid, s);
}

template <class St>
static cudaError_t launch_bnd_t(const BndParams& p, dim3 grid, size_t smem, cudaStream_t s)
{
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(boundary_kernel<St, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(boundary_kernel<St, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (p.first) boundary_kernel<St, true><<<grid, BBLOCK, smem, s>>>(p);
    else boundary_kernel<St, false><<<grid, BBLOCK, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_boundary(const BndParams& p, int precision, int list_cap, int np, cudaStream_t s)
{
    if (np <= 0) return cudaSuccess;
    const dim3 grid((list_cap + BBLOCK - 1) / BBLOCK, np);
    const size_t smem = 2ull * p.smax * p.smax * sizeof(uint64_t);
    if (precision == 1) return launch_bnd_t<StF16>(p, grid, smem, s);
    if (precision == 2) return launch_bnd_t<StBF16>(p, grid, smem, s);
    return launch_bnd_t<StF32>(p, grid, smem, s);
}

}  // namespace lbsph
