// D3Q27 lattice and particle kernels (see q27.cuh for the method and the
// order of an iteration).
#include "particle_blocks.cuh"   // the exact FP64 inside test (canon_shape, canon_value)
#include "q27.cuh"

namespace lbsph {
namespace q27 {

constexpr int LBLOCK = 256;          // threads per lattice block (one node each)
constexpr int PBLK = 512;            // threads per particle block
constexpr int RW = MAXS * MAXS;      // words per bitmap slot

__device__ __forceinline__ int wrapc(int a, int L) { return a < 0 ? a + L : (a >= L ? a - L : a); }

// local coordinate of box coordinate X in a cube of side S at wrapped origin o
// along an axis of length L; returns false outside the cube
__device__ __forceinline__ bool cube_local(int X, int o, int L, int S, int& m)
{
    m = X - o;
    if (m < 0) m += L;
    return m < S;
}

__device__ __forceinline__ bool bit_at(const uint64_t* map, int S, int mx, int my, int mz)
{
    if (mx < 0 || my < 0 || mz < 0 || mx >= S || my >= S || mz >= S) return false;
    return (__ldg(map + mz * S + my) >> mx) & 1ull;
}

// The 3 x 3 x 3 neighbourhood of cube cell (mx, my, mz), 0 <= m < S, of a map of
// side S as one mask: bit (dx + 1) + 3 (dy + 1) + 9 (dz + 1) is the cell
// (mx + dx, my + dy, mz + dz), 0 outside the cube (rows hold no bits at S and
// beyond).  Nine row loads instead of a bounds-checked load per direction.
__device__ __forceinline__ unsigned nbhd27(const uint64_t* map, int S, int mx, int my, int mz)
{
    unsigned nb = 0;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy) {
            const int y = my + dy, z = mz + dz;
            if (y < 0 || z < 0 || y >= S || z >= S) continue;
            const uint64_t w = __ldg(map + z * S + y);
            // bits mx - 1, mx, mx + 1 of the row
            const unsigned t = mx > 0 ? (unsigned)((w >> (mx - 1)) & 7ull) : (unsigned)((w << 1) & 6ull);
            nb |= t << (3 * (dy + 1) + 9 * (dz + 1));
        }
    return nb;
}

// bit of the neighbour at offset c in a mask of nbhd27
__device__ __forceinline__ bool nb_bit(unsigned nb, int cx, int cy, int cz)
{
    return (nb >> (13 + cx + 3 * cy + 9 * cz)) & 1u;
}

enum { K_FLUID = 0, K_SOLID = 1, K_COVERED = 2, K_UNCOVERED = 3 };

// Pre-collision deviations d = f - w rho0 of node (X, Y, Z) at the start of
// iteration t, from the post-collision field A of t - 1: pull streaming, with
// mid-link bounce-back where the source is inside the old surface (Eq. fb,
// Eq. ub: f_i(x) = f*_{opp i}(x) + 6 w_i rho0 (u_b . c_i), u_b = U + W x r_b,
// r_b = x - c_i/2 - x_c(t-1)), then the remap to the new map (Appendix step 8):
// a covered node keeps its pulled values for the particle's sums (its stored
// values become 0), an uncovered node gets f_eq(rho0, U + W x r) with
// r = x - x_c(t).  mn: the node's local coordinates in the new cube (when
// inside it).  nopull: the stored field is taken as it is (before the first
// collision).
__device__ __forceinline__ int pre_collision(const Box27& B, const Dyn27& K, const uint64_t* rows, const float* A,
                                             int X, int Y, int Z, int node, bool nopull, float (&d)[Q27],
                                             int (&mn)[3], bool& in_new, unsigned& nb_new)
{
    const int nx = B.nx, ny = B.ny, nz = B.nz, N = (int)B.N;
    int mo[3] = {0, 0, 0};
    bool in_old = false;
    in_new = false;
    bool sol_old = false, sol_new = false;
    unsigned nb_old = 0u;
    nb_new = 0u;
    if (K.active) {
        const int S = K.S;
        const uint64_t* map_old = rows + (size_t)K.slot_old * RW;
        const uint64_t* map_new = rows + (size_t)K.slot_new * RW;
        in_old = cube_local(X, K.o_old[0], nx, S, mo[0]) && cube_local(Y, K.o_old[1], ny, S, mo[1]) &&
                 cube_local(Z, K.o_old[2], nz, S, mo[2]);
        in_new = cube_local(X, K.o_new[0], nx, S, mn[0]) && cube_local(Y, K.o_new[1], ny, S, mn[1]) &&
                 cube_local(Z, K.o_new[2], nz, S, mn[2]);
        nb_old = in_old ? nbhd27(map_old, S, mo[0], mo[1], mo[2]) : 0u;
        nb_new = in_new ? nbhd27(map_new, S, mn[0], mn[1], mn[2]) : 0u;
        sol_old = nb_bit(nb_old, 0, 0, 0);
        sol_new = nb_bit(nb_new, 0, 0, 0);
    }
    if (nopull) {
#pragma unroll
        for (int i = 0; i < Q27; ++i) d[i] = sol_new ? 0.0f : __ldg(A + (i * N + node));
        return sol_new ? K_SOLID : K_FLUID;
    }
    if (sol_old && sol_new) {
#pragma unroll
        for (int i = 0; i < Q27; ++i) d[i] = 0.0f;
        return K_SOLID;
    }
    if (sol_old) {
        // uncovered: f_eq(rho0, u) with u the body's velocity at the node
        const float rx = K.phi_new[0] + mn[0], ry = K.phi_new[1] + mn[1], rz = K.phi_new[2] + mn[2];
        const float ux = K.U[0] + (K.W[1] * rz - K.W[2] * ry);
        const float uy = K.U[1] + (K.W[2] * rx - K.W[0] * rz);
        const float uz = K.U[2] + (K.W[0] * ry - K.W[1] * rx);
        const float uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
        for (int i = 0; i < Q27; ++i) {
            const float cu = cx27(i) * ux + cy27(i) * uy + cz27(i) * uz;
            d[i] = w27(i) * B.rho0f * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu);
        }
        return K_UNCOVERED;
    }
    // fluid at t - 1: pull, bouncing back from the old surface.  The source
    // x - c_i is node + ox[c_x] + oy[c_y] + oz[c_z], each offset wrapped at the
    // box faces (index 0: c = -1, 2: c = +1).
    const int nxy = nx * ny;
    const int ox[3] = {X == nx - 1 ? 1 - nx : 1, 0, X == 0 ? nx - 1 : -1};
    const int oy[3] = {Y == ny - 1 ? nx - nxy : nx, 0, Y == 0 ? nxy - nx : -nx};
    const int oz[3] = {Z == nz - 1 ? nxy - N : nxy, 0, Z == 0 ? N - nxy : -nxy};
    if (!in_old) {
#pragma unroll
        for (int i = 0; i < Q27; ++i)
            d[i] = __ldg(A + (i * N + node + ox[cx27(i) + 1] + oy[cy27(i) + 1] + oz[cz27(i) + 1]));
        return sol_new ? K_COVERED : K_FLUID;
    }
#pragma unroll
    for (int i = 0; i < Q27; ++i) {
        const int cx = cx27(i), cy = cy27(i), cz = cz27(i);
        const bool back = i > 0 && nb_bit(nb_old, -cx, -cy, -cz);
        if (back) {
            const float px = K.phi_old[0] + mo[0] - 0.5f * cx;
            const float py = K.phi_old[1] + mo[1] - 0.5f * cy;
            const float pz = K.phi_old[2] + mo[2] - 0.5f * cz;
            const float ux = K.U[0] + (K.W[1] * pz - K.W[2] * py);
            const float uy = K.U[1] + (K.W[2] * px - K.W[0] * pz);
            const float uz = K.U[2] + (K.W[0] * py - K.W[1] * px);
            const float ubc = cx * ux + cy * uy + cz * uz;
            d[i] = __ldg(A + (opp27(i) * N + node)) + 6.0f * w27(i) * B.rho0f * ubc;
        } else {
            d[i] = __ldg(A + (i * N + node + ox[cx + 1] + oy[cy + 1] + oz[cz + 1]));
        }
    }
    return sol_new ? K_COVERED : K_FLUID;
}

// BGK (Eq. 3-4) with Guo forcing on deviations, mass return eps added first
// as w_i eps to every population.
//
// GHOST: the collision of the paper's simulations (Sec. II.A: one relaxation
// time for the non-conserved hydrodynamic modes, the non-hydrodynamic ones
// relaxed at once).  Of f - f_eq only the projection on the hydrodynamic
// Hermite modes survives, relaxed by 1 - omega:
//   d_i' = deq_i + (1 - omega) w_i [3 c_i.j_neq + 4.5 (c_i c_i - I/3) : Pi_neq] + S_i,
// j_neq = j - rho u = -g/2 (u carries the half-force shift) and
// Pi_neq = sum_i c_i c_i d_i - drho/3 I - rho u u (the rest state w rho0
// contributes rho0/3 I, the equilibrium rho/3 I + rho u u).  The 17 modes of
// D3Q27 beyond these ten leave at equilibrium.  At omega = 1 it is BGK.
template <bool GHOST>
__device__ __forceinline__ void collide27(float (&d)[Q27], float omega, float rho0, const float g[3], float eps)
{
    // moments, per pair of opposite directions (2m+1, 2m+2), c_{2m+2} = -c_{2m+1}:
    // the sum sm enters drho and the second moments, the difference df the momentum
    float sm[13], df[13];
    d[0] += w27(0) * eps;
    float drho = d[0], jx = 0.0f, jy = 0.0f, jz = 0.0f;
    float pxx = 0.0f, pyy = 0.0f, pzz = 0.0f, pxy = 0.0f, pxz = 0.0f, pyz = 0.0f;
#pragma unroll
    for (int m = 0; m < 13; ++m) {
        const int i = 2 * m + 1;
        const float we = w27(i) * eps;
        sm[m] = (d[i] + we) + (d[i + 1] + we);
        df[m] = (d[i] + we) - (d[i + 1] + we);
        const int cx = cx27(i), cy = cy27(i), cz = cz27(i);
        drho += sm[m];
        if (cx) jx += cx * df[m];
        if (cy) jy += cy * df[m];
        if (cz) jz += cz * df[m];
        if constexpr (GHOST) {
            if (cx) pxx += sm[m];
            if (cy) pyy += sm[m];
            if (cz) pzz += sm[m];
            if (cx * cy) pxy += (cx * cy) * sm[m];
            if (cx * cz) pxz += (cx * cz) * sm[m];
            if (cy * cz) pyz += (cy * cz) * sm[m];
        }
    }
    const float rho = rho0 + drho;
    const float ir = 1.0f / rho;
    const float ux = (jx + 0.5f * g[0]) * ir, uy = (jy + 0.5f * g[1]) * ir, uz = (jz + 0.5f * g[2]) * ir;
    const float uu = ux * ux + uy * uy + uz * uz, ug = ux * g[0] + uy * g[1] + uz * g[2];
    const float cf = 1.0f - 0.5f * omega, om1 = 1.0f - omega;
    // even part of the equilibrium about rho0 w (without the w factor)
    const float e0 = drho - 1.5f * rho * uu;
    if constexpr (GHOST) {
        // d_i' = deq_i + (1 - omega) w_i [3 c_i.j_neq + 4.5 (c_i c_i - I/3) : Pi_neq] + S_i;
        // per pair the odd part is 3 w rho cu + 1.5 w cg whatever omega (j_neq = -g/2)
        const float iso = -drho * (1.0f / 3.0f);
        const float nxx = pxx + iso - rho * ux * ux, nyy = pyy + iso - rho * uy * uy, nzz = pzz + iso - rho * uz * uz;
        const float nxy = pxy - rho * ux * uy, nxz = pxz - rho * ux * uz, nyz = pyz - rho * uy * uz;
        const float tr3 = (nxx + nyy + nzz) * (1.0f / 3.0f);
        d[0] = w27(0) * (e0 - om1 * 4.5f * tr3 - cf * 3.0f * ug);
#pragma unroll
        for (int m = 0; m < 13; ++m) {
            const int i = 2 * m + 1;
            const int cx = cx27(i), cy = cy27(i), cz = cz27(i);
            const float cu = cx * ux + cy * uy + cz * uz;
            const float cg = cx * g[0] + cy * g[1] + cz * g[2];
            float qp = -tr3;
            if (cx) qp += nxx;
            if (cy) qp += nyy;
            if (cz) qp += nzz;
            if (cx * cy) qp += (2 * cx * cy) * nxy;
            if (cx * cz) qp += (2 * cx * cz) * nxz;
            if (cy * cz) qp += (2 * cy * cz) * nyz;
            const float E = w27(i) * (e0 + 4.5f * rho * cu * cu + om1 * 4.5f * qp + cf * (9.0f * cu * cg - 3.0f * ug));
            const float O = w27(i) * (3.0f * rho * cu + 1.5f * cg);
            d[i] = E + O;
            d[i + 1] = E - O;
        }
    } else {
        // d_i' = (1 - omega) d_i + omega deq_i + S_i, even and odd parts per pair
        d[0] = om1 * d[0] + w27(0) * (omega * e0 - cf * 3.0f * ug);
#pragma unroll
        for (int m = 0; m < 13; ++m) {
            const int i = 2 * m + 1;
            const int cx = cx27(i), cy = cy27(i), cz = cz27(i);
            const float cu = cx * ux + cy * uy + cz * uz;
            const float cg = cx * g[0] + cy * g[1] + cz * g[2];
            const float E = w27(i) * (omega * (e0 + 4.5f * rho * cu * cu) + cf * (9.0f * cu * cg - 3.0f * ug));
            const float O = w27(i) * (omega * 3.0f * rho * cu + cf * 3.0f * cg);
            const float a = om1 * (0.5f * sm[m]), b = om1 * (0.5f * df[m]);
            d[i] = (a + b) + E + O;
            d[i + 1] = (a - b) + E - O;
        }
    }
}

__device__ __forceinline__ long long wsum(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += (long long)__shfl_xor_sync(0xffffffffu, (unsigned long long)v, o);
    return v;
}

__device__ __forceinline__ void acc_add(long long* a, long long v)
{
    if (v != 0) atomicAdd(reinterpret_cast<unsigned long long*>(a), static_cast<unsigned long long>(v));
}

// ---------------------------------------------------------------------------
// One lattice pass over every node of every box (one node per thread).
template <bool GHOST>
__global__ void __launch_bounds__(LBLOCK, 3) lattice27_kernel(const __grid_constant__ LatParams27 P)
{
    __shared__ Box27 sB;
    __shared__ Dyn27 sK;
    const int bi = P.mode == LAT_NEAR ? __ldg(&P.pd[blockIdx.x / P.nbpp].box) : __ldg(P.blk_box + blockIdx.x);
    if (threadIdx.x < sizeof(Box27) / 4)
        reinterpret_cast<int*>(&sB)[threadIdx.x] = __ldg(reinterpret_cast<const int*>(P.boxes + bi) + threadIdx.x);
    else if (threadIdx.x >= 64 && threadIdx.x < 64 + sizeof(Dyn27) / 4)
        reinterpret_cast<int*>(&sK)[threadIdx.x - 64] =
            __ldg(reinterpret_cast<const int*>(P.dyn + bi) + (threadIdx.x - 64));
    __syncthreads();
    const Box27& B = sB;
    const Dyn27& K = sK;
    bool valid, skip = false;
    int nd, X, Y, Z;
    if (P.mode == LAT_NEAR) {
        // the nodes of the box that holds the particle's old and new cubes
        const int l = (blockIdx.x % P.nbpp) * LBLOCK + threadIdx.x;
        const int e0 = K.E[0], e1 = K.E[1];
        valid = l < e0 * e1 * K.E[2];
        const int ll = valid ? l : 0;
        const int mz = ll / (e0 * e1), my = (ll / e0) % e1, mx = ll % e0;
        X = wrapc(K.uo[0] + mx, B.nx);
        Y = wrapc(K.uo[1] + my, B.ny);
        Z = wrapc(K.uo[2] + mz, B.nz);
        nd = (Z * B.ny + Y) * B.nx + X;
    } else {
        const int node = (blockIdx.x - B.block_begin) * LBLOCK + threadIdx.x;
        valid = node < (int)B.N;
        nd = valid ? node : (int)B.N - 1;
        const int row = div_magic(nd, B.dx_m, B.dx_s);
        X = nd - row * B.nx;
        Z = div_magic(row, B.dy_m, B.dy_s);
        Y = row - Z * B.ny;
        if (P.mode == LAT_BULK && K.active) {
            // nodes of the cube union are left to the near pass
            int m;
            if (cube_local(X, K.uo[0], B.nx, K.E[0], m) && cube_local(Y, K.uo[1], B.ny, K.E[1], m) &&
                cube_local(Z, K.uo[2], B.nz, K.E[2], m))
                skip = true;
        }
    }
    const int node = nd;
    const float* A = P.src + B.off;
    float* D = P.dst + B.off;
    const uint64_t* rows = K.active ? P.rows + (size_t)B.p * 2 * RW : nullptr;
    float d[Q27];
    int mn[3] = {0, 0, 0};
    bool in_new = false;
    unsigned nb_new = 0u;
    // a skipped node reads nothing: its cube's maps may be rewritten meanwhile
    // by the particle kernel beside this pass
    if (skip) valid = false;
    int kind = K_SOLID;
    if (skip) {
#pragma unroll
        for (int i = 0; i < Q27; ++i) d[i] = 0.0f;
    } else {
        kind = pre_collision(B, K, rows, A, X, Y, Z, nd, P.first != 0, d, mn, in_new, nb_new);
    }
    // integer sums for the particle: links of the new map, covered and uncovered nodes
    long long aF[3] = {0, 0, 0}, aT[3] = {0, 0, 0};
    if (valid && kind == K_COVERED) {
        long long* acc = P.acc + (size_t)B.p * NACC;
        float sr = 0.0f, j[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
        for (int i = 0; i < Q27; ++i) {
            sr += d[i];
            j[0] += cx27(i) * d[i];
            j[1] += cy27(i) * d[i];
            j[2] += cz27(i) * d[i];
        }
        const long long J[3] = {fixp(j[0]), fixp(j[1]), fixp(j[2])};
        acc_add(acc + ACC_COV, 1);
        acc_add(acc + ACC_COV + 1, fixp(sr));
        for (int k = 0; k < 3; ++k) acc_add(acc + ACC_COV + 2 + k, J[k]);
        acc_add(acc + ACC_COV + 5, mn[1] * J[2] - mn[2] * J[1]);
        acc_add(acc + ACC_COV + 6, mn[2] * J[0] - mn[0] * J[2]);
        acc_add(acc + ACC_COV + 7, mn[0] * J[1] - mn[1] * J[0]);
    } else if (valid && kind == K_UNCOVERED) {
        long long* acc = P.acc + (size_t)B.p * NACC;
        const long long m0 = mn[0], m1 = mn[1], m2 = mn[2];
        const long long uv[10] = {1, m0, m1, m2, m0 * m0, m0 * m1, m0 * m2, m1 * m1, m1 * m2, m2 * m2};
        for (int e = 0; e < 10; ++e) acc_add(acc + ACC_UNC + e, uv[e]);
    }
    if (kind == K_FLUID || kind == K_UNCOVERED) {
        const float g[3] = {K.g[0], K.g[1], K.g[2]};
        collide27<GHOST>(d, B.omega, B.rho0f, g, K.eps);
        if (in_new && valid) {
#pragma unroll
            for (int b = 1; b < Q27; ++b) {
                const int cx = cx27(b), cy = cy27(b), cz = cz27(b);
                if (!nb_bit(nb_new, cx, cy, cz)) continue;
                const long long a = fixp(2.0f * d[b]);
                const long long gx = cx * a, gy = cy * a, gz = cz * a;
                aF[0] += gx; aF[1] += gy; aF[2] += gz;
                aT[0] += mn[1] * gz - mn[2] * gy;
                aT[1] += mn[2] * gx - mn[0] * gz;
                aT[2] += mn[0] * gy - mn[1] * gx;
            }
        }
    } else {
#pragma unroll
        for (int i = 0; i < Q27; ++i) d[i] = 0.0f;
    }
    if (valid) {
#pragma unroll
        for (int i = 0; i < Q27; ++i) D[(size_t)i * B.N + node] = d[i];
    }
    // link sums: warp totals, one atomic per nonzero total
    const bool any = __any_sync(0xffffffffu, (aF[0] | aF[1] | aF[2] | aT[0] | aT[1] | aT[2]) != 0);
    if (any) {
        long long* acc = P.acc + (size_t)(B.p >= 0 ? B.p : 0) * NACC;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const long long f = wsum(aF[k]), t = wsum(aT[k]);
            if ((threadIdx.x & 31) == 0 && B.p >= 0) {
                acc_add(acc + ACC_F + k, f);
                acc_add(acc + ACC_T + k, t);
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Bulk pass (LAT_BULK): every node outside the particles' cube unions takes the
// plain pull of the last post-collision field and the collision, exactly as in
// lattice27_kernel (outside both cubes no source is solid and no node changes
// sides), without the bounce-back, remap and link-sum code: fewer registers and
// instructions per node, so more warps and more loads in flight per SM.
#ifndef BULK27_MINB
#define BULK27_MINB 3
#endif
template <bool GHOST>
__global__ void __launch_bounds__(LBLOCK, BULK27_MINB) bulk27_kernel(const __grid_constant__ LatParams27 P)
{
    __shared__ Box27 sB;
    __shared__ Dyn27 sK;
    const int bi = __ldg(P.blk_box + blockIdx.x);
    if (threadIdx.x < sizeof(Box27) / 4)
        reinterpret_cast<int*>(&sB)[threadIdx.x] = __ldg(reinterpret_cast<const int*>(P.boxes + bi) + threadIdx.x);
    else if (threadIdx.x >= 64 && threadIdx.x < 64 + sizeof(Dyn27) / 4)
        reinterpret_cast<int*>(&sK)[threadIdx.x - 64] =
            __ldg(reinterpret_cast<const int*>(P.dyn + bi) + (threadIdx.x - 64));
    __syncthreads();
    const Box27& B = sB;
    const Dyn27& K = sK;
    const int node = (blockIdx.x - B.block_begin) * LBLOCK + threadIdx.x;
    if (node >= (int)B.N) return;
    const int row = div_magic(node, B.dx_m, B.dx_s);
    const int X = node - row * B.nx;
    const int Z = div_magic(row, B.dy_m, B.dy_s);
    const int Y = row - Z * B.ny;
    if (K.active) {
        int m;
        if (cube_local(X, K.uo[0], B.nx, K.E[0], m) && cube_local(Y, K.uo[1], B.ny, K.E[1], m) &&
            cube_local(Z, K.uo[2], B.nz, K.E[2], m))
            return;                                // a node of the near pass
    }
    const int nx = B.nx, ny = B.ny, nz = B.nz, N = (int)B.N;
    const int nxy = nx * ny;
    const int ox[3] = {X == nx - 1 ? 1 - nx : 1, 0, X == 0 ? nx - 1 : -1};
    const int oy[3] = {Y == ny - 1 ? nx - nxy : nx, 0, Y == 0 ? nxy - nx : -nx};
    const int oz[3] = {Z == nz - 1 ? nxy - N : nxy, 0, Z == 0 ? N - nxy : -nxy};
    const float* A = P.src + B.off;
    float* D = P.dst + B.off;
    float d[Q27];
#pragma unroll
    for (int i = 0; i < Q27; ++i) d[i] = __ldg(A + (i * N + node + ox[cx27(i) + 1] + oy[cy27(i) + 1] + oz[cz27(i) + 1]));
    const float g[3] = {K.g[0], K.g[1], K.g[2]};
    collide27<GHOST>(d, B.omega, B.rho0f, g, K.eps);
#pragma unroll
    for (int i = 0; i < Q27; ++i) D[(size_t)i * B.N + node] = d[i];
}

// ---------------------------------------------------------------------------
// Rigid-body algebra in FP64 (one thread)
__device__ __forceinline__ void qmul27(const double a[4], const double b[4], double o[4])
{
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

// q' = qt q, qt the rotation by the angle |W| about W (Eq. qnplus0-1; no
// rotation for W = 0)
// For |W| < 0.01 (a step's rotation, always in practice) cos(n/2) and
// sin(n/2)/n come from their Taylor series in n^2, 1 - n^2/8 + n^4/384 and
// 1/2 - n^2/48 + n^4/3840: the next terms (n^6/46080, n^6/645120) lie below
// the FP64 rounding of the results, and no square root or trigonometric
// function is evaluated.
__device__ __forceinline__ void qstep27(const double q[4], const double W[3], double o[4])
{
    const double n2 = W[0] * W[0] + W[1] * W[1] + W[2] * W[2];
    double t[4] = {1.0, 0.0, 0.0, 0.0};
    if (n2 < 1e-4) {
        const double s = 0.5 - n2 * (1.0 / 48.0 - n2 * (1.0 / 3840.0));
        t[0] = 1.0 - n2 * (0.125 - n2 * (1.0 / 384.0));
        t[1] = s * W[0]; t[2] = s * W[1]; t[3] = s * W[2];
    } else {
        const double n = sqrt(n2);
        const double s = sin(0.5 * n) / n;
        t[0] = cos(0.5 * n);
        t[1] = s * W[0]; t[2] = s * W[1]; t[3] = s * W[2];
    }
    qmul27(t, q, o);
}

// lab-frame inertia R diag(Ib) R^T (Eq. Irot), R the rotation of unit q
__device__ __forceinline__ void inertia27(const double q[4], const double Ib[3], double I[9])
{
    const double R[9] = {1.0 - 2.0 * (q[2] * q[2] + q[3] * q[3]), 2.0 * (q[1] * q[2] - q[0] * q[3]),
                         2.0 * (q[1] * q[3] + q[0] * q[2]),       2.0 * (q[1] * q[2] + q[0] * q[3]),
                         1.0 - 2.0 * (q[1] * q[1] + q[3] * q[3]), 2.0 * (q[2] * q[3] - q[0] * q[1]),
                         2.0 * (q[1] * q[3] - q[0] * q[2]),       2.0 * (q[2] * q[3] + q[0] * q[1]),
                         1.0 - 2.0 * (q[1] * q[1] + q[2] * q[2])};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            I[i * 3 + j] = R[i * 3] * Ib[0] * R[j * 3] + R[i * 3 + 1] * Ib[1] * R[j * 3 + 1] +
                           R[i * 3 + 2] * Ib[2] * R[j * 3 + 2];
}

// dI/dt = [W]x I - I [W]x (Eq. Irotdiff)
__device__ __forceinline__ void inertia_rate27(const double I[9], const double W[3], double dI[9])
{
    const double X[9] = {0.0, -W[2], W[1], W[2], 0.0, -W[0], -W[1], W[0], 0.0};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += X[i * 3 + k] * I[k * 3 + j] - I[i * 3 + k] * X[k * 3 + j];
            dI[i * 3 + j] = s;
        }
}

__device__ __forceinline__ void cross27(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// The parts of the solve of Eq. Fdiscrete / Eq. Tdiscrete for particle D,
// spread over the block: q27_sums (one thread) turns the integer sums of the
// last lattice pass into F0, T0 and the remap terms; the inertia and its rate
// come from another warp at the same time; a warp solves the 6 x 6 system
// (q27_solve6); six threads form F and T; three threads move the centre and
// another the orientation, and a warp writes the record.
__device__ void q27_sums(const PartParams27& P, Part27* D, const Box27& B, int p, double F0[3], double T0[3])
{
    long long* acc = P.acc + (size_t)p * NACC;
    double a[NACC];
    for (int e = 0; e < NACC; ++e) {
        a[e] = (double)acc[e];
        acc[e] = 0;
    }
    const double rho0 = B.rho0;
    double Fd[3], Tm[3], J[3], MJ[3], Sm[3], phi[3];
    for (int k = 0; k < 3; ++k) {
        Fd[k] = a[ACC_F + k] / FIXD;
        Tm[k] = a[ACC_T + k] / FIXD;
        J[k] = a[ACC_COV + 2 + k] / FIXD;
        MJ[k] = a[ACC_COV + 5 + k] / FIXD;
        Sm[k] = a[ACC_UNC + 1 + k];
        phi[k] = D->phi[k];
    }
    // Eq. F0 / Eq. T0 over the links of the current map: r_b x c_b = (phi + m) x c_b
    double pF[3];
    cross27(phi, Fd, pF);
    for (int k = 0; k < 3; ++k) {
        F0[k] = Fd[k] + D->F0g[k];
        T0[k] = pF[k] + Tm[k] + D->T0g[k];
    }
    // remap terms (Appendix step 8): covered nodes give their momentum and its
    // moment about x_c; uncovered ones take rho0 (U + W x r), r = phi + m
    const double nc = a[ACC_COV], nu = a[ACC_UNC];
    if (nc == 0.0 && nu == 0.0) {              // most steps: no node changed sides
        for (int k = 0; k < 3; ++k) D->dP[k] = D->dL[k] = 0.0;
        D->dm = 0.0;
        return;
    }
    const double Smm[9] = {a[ACC_UNC + 4], a[ACC_UNC + 5], a[ACC_UNC + 6], a[ACC_UNC + 5], a[ACC_UNC + 7],
                           a[ACC_UNC + 8], a[ACC_UNC + 6], a[ACC_UNC + 8], a[ACC_UNC + 9]};
    double Sr[3], Srr[9];
    for (int i = 0; i < 3; ++i) Sr[i] = nu * phi[i] + Sm[i];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) Srr[i * 3 + j] = nu * phi[i] * phi[j] + phi[i] * Sm[j] + Sm[i] * phi[j] + Smm[i * 3 + j];
    const double tr = Srr[0] + Srr[4] + Srr[8];
    double WxSr[3], pJ[3], SrxU[3];
    cross27(D->W, Sr, WxSr);
    cross27(phi, J, pJ);
    cross27(Sr, D->U, SrxU);
    for (int k = 0; k < 3; ++k) {
        D->dP[k] = J[k] - rho0 * (nu * D->U[k] + WxSr[k]);
        const double SrrW = Srr[k * 3] * D->W[0] + Srr[k * 3 + 1] * D->W[1] + Srr[k * 3 + 2] * D->W[2];
        D->dL[k] = pJ[k] + MJ[k] - rho0 * (SrxU[k] + D->W[k] * tr - SrrW);
    }
    D->dm = nc * rho0 + a[ACC_COV + 1] / FIXD - nu * rho0;
}

// Gauss-Jordan with partial pivoting on one warp in FP32: lane j < 12 holds
// column j of [A | I] (rows 0..5); on return lanes 6..11 hold the columns of
// A^-1.  The pivot is chosen by lane k and broadcast, so every lane takes the
// same row exchanges; false (on every lane) if a pivot vanishes.
__device__ __forceinline__ bool gj_inv6_warp_f32(float (&col)[6], int lane)
{
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        int piv = k;
        if (lane == k) {
            float best = fabsf(col[k]);
#pragma unroll
            for (int i = k + 1; i < 6; ++i)
                if (fabsf(col[i]) > best) { best = fabsf(col[i]); piv = i; }
        }
        piv = __shfl_sync(0xffffffffu, piv, k);
        float rowk = col[k], rowp = col[k];
#pragma unroll
        for (int i = k + 1; i < 6; ++i)
            if (i == piv) rowp = col[i];
#pragma unroll
        for (int i = k + 1; i < 6; ++i)
            if (i == piv) col[i] = rowk;
        col[k] = rowp;
        const float pv = __shfl_sync(0xffffffffu, col[k], k);
        ok = ok && (pv != 0.0f);
        col[k] *= 1.0f / pv;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            if (i == k) continue;
            const float fi = __shfl_sync(0xffffffffu, col[i], k);
            col[i] -= fi * col[k];
        }
    }
    return ok;
}

// x = A^-1 rhs for the 6 x 6 system of Eq. Fdiscrete / Eq. Tdiscrete on one
// warp: the inverse in FP32, then iterative refinement, x += A^-1 (rhs - A x)
// with the residual in FP64.  Each step multiplies the error by about cond(A)
// times the FP32 rounding; three steps bring it to FP64 rounding for these
// systems (mass, inertia and drag matrices: cond(A) of order 10-10^3).  Only
// the residuals are FP64, so the chain of dependent FP64 operations is short;
// measured beside the bulk pass the solve still takes about as long as a
// Gauss-Jordan elimination in FP64 (about 15 us; with the pivot loop rolled up,
// a fifth of the code, 17.5 us), so its time is the latency of its dependent
// chain, not arithmetic or instruction fetch.  s_Ai: 36 floats of scratch.
// Writes x6 (lanes 0..5); false if a pivot vanishes.
__device__ bool q27_solve6(const double* A6, const double* rhs, double* x6, float* s_Ai, int lane)
{
    float col[6];
#pragma unroll
    for (int i = 0; i < 6; ++i)
        col[i] = lane < 6 ? (float)A6[i * 6 + lane] : (lane - 6 == i ? 1.0f : 0.0f);
    const bool ok = gj_inv6_warp_f32(col, lane);
    if (lane >= 6 && lane < 12)
#pragma unroll
        for (int i = 0; i < 6; ++i) s_Ai[i * 6 + lane - 6] = col[i];
    __syncwarp();
    const int i = lane < 6 ? lane : 0;
    double a[6];
    float ai[6];
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        a[j] = A6[i * 6 + j];
        ai[j] = s_Ai[i * 6 + j];
    }
    const double b = rhs[i];
    float xf = 0.0f;
#pragma unroll
    for (int j = 0; j < 6; ++j) xf += ai[j] * (float)rhs[j];
    double x = xf;
    for (int it = 0; it < 3; ++it) {
        double r0 = b, r1 = 0.0;
#pragma unroll
        for (int j = 0; j < 6; j += 2) {
            r0 -= a[j] * __shfl_sync(0xffffffffu, x, j);
            r1 -= a[j + 1] * __shfl_sync(0xffffffffu, x, j + 1);
        }
        const float r = (float)(r0 + r1);
        float d = 0.0f;
#pragma unroll
        for (int j = 0; j < 6; ++j) d += ai[j] * __shfl_sync(0xffffffffu, r, j);
        x += (double)d;
    }
    if (lane < 6) x6[lane] = x;
    __syncwarp();
    return ok;
}

// ---------------------------------------------------------------------------
// Particle kernel: one block of 512 threads per particle, the particle's state
// staged in shared memory and written back at the end.  Step mode: the solve
// and pose update of the last lattice pass's iteration, then for the new pose
// the occupancy map (Eq. ellipsoidsurface), built in shared memory one cube row
// per thread: along a row the inside value is the quadratic a x^2 + b x + c,
// evaluated in FP32 and decided there outside a band around 1 (its FP32 error
// stays far below the band inside the cube); the nodes inside the band are
// collected and then tested by the exact FP64 test in the oracle's operation
// order, one node per thread, so the map is bit-identical to the oracle's.
// The links (x fluid, x + c_b solid) of each row and direction are a bit mask;
// their drag matrix and the geometric parts of F0 / T0 (Eq. drag1-4, Eq. F0,
// Eq. T0) come from exact integer sums per direction (link count, sum of m,
// sum of m m^T over the cube coordinates m of the fluid ends), combined once
// in FP64 with p = phi + m, r_b x c_b = p x c_b.  Init mode: the map and its
// terms for the current pose.
constexpr int NCAND = 512;                       // nodes of the FP32 band tested exactly after the row pass
__global__ void __launch_bounds__(PBLK, 1) particle27_kernel(const __grid_constant__ PartParams27 P)
{
    constexpr int NSUM = 10;                     // per direction: n, sum m (3), sum m m^T (6)
    constexpr int NG = PBLK / (Q27 - 1);         // row groups of the link sums (one direction per thread)
    const int p = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    Part27* G = P.pd + p;
    __shared__ Part27 sD;
    __shared__ Box27 sB;
    __shared__ uint64_t s_map[MAXS * MAXS];
    __shared__ int s_sum[Q27][NSUM];
    __shared__ double s_con[Q27][42];            // per direction: drag matrix (36), F0g (3), T0g (3)
    __shared__ double s_A[9], s_E[9], s_x[3], s_phi[3];
    __shared__ float s_A32[9], s_d0[3];
    __shared__ int s_o[3], s_ow[3], s_S, s_slot, s_ok, s_nsol, s_ncand;
    __shared__ float s_band;
    __shared__ int s_cand[NCAND];
    static_assert(sizeof(Part27) % 8 == 0 && sizeof(Box27) % 4 == 0, "staged as words");
    {
        const int bi = __ldg(&G->box);
        for (int k = tid; k < (int)(sizeof(Part27) / 8); k += PBLK)
            reinterpret_cast<unsigned long long*>(&sD)[k] = reinterpret_cast<const unsigned long long*>(G)[k];
        if (tid >= 256 && tid < 256 + (int)(sizeof(Box27) / 4))
            reinterpret_cast<int*>(&sB)[tid - 256] = __ldg(reinterpret_cast<const int*>(P.boxes + bi) + (tid - 256));
    }
    __syncthreads();
    Part27* D = &sD;
    const Box27& B = sB;
    if (!P.init) {
        __shared__ double s_F0[3], s_T0[3], s_In[9], s_dI[9], s_A6[36], s_rhs[6], s_x6[6], s_FT[6], s_xn[3], s_qn[4];
        __shared__ float s_Ai[36];
        __shared__ int s_solved;
        if (tid == 0) {
            q27_sums(P, D, B, p, s_F0, s_T0);
        } else if (tid == 32) {
            inertia27(D->q, D->Ib, s_In);
            if (P.didt_mode == 1) {
                for (int k = 0; k < 9; ++k) s_dI[k] = s_In[k] - D->Iprev[k];
            } else {
                inertia_rate27(s_In, D->W, s_dI);
            }
        }
        __syncthreads();
        if (tid < 36) {
            // A = zeta + diag(M) + (I + dI) in the rotational block
            const int i = tid / 6, j = tid % 6;
            double a = D->zeta[tid];
            if (i == j && i < 3) a += D->M;
            if (i >= 3 && j >= 3) a += s_In[(i - 3) * 3 + j - 3] + s_dI[(i - 3) * 3 + j - 3];
            s_A6[tid] = a;
        } else if (tid >= 64 && tid < 70) {
            // rhs = (M U + F0 + F_ext + dP, I W + T0 + T_ext + dL)
            const int k = tid - 64;
            if (k < 3) {
                s_rhs[k] = D->M * D->U[k] + s_F0[k] + D->Fext[k] + D->dP[k];
            } else {
                const int m = k - 3;
                s_rhs[k] = s_In[m * 3] * D->W[0] + s_In[m * 3 + 1] * D->W[1] + s_In[m * 3 + 2] * D->W[2] + s_T0[m] +
                           D->Text[m] + D->dL[m];
            }
        }
        __syncthreads();
        if (tid < 32) {
            const bool ok = q27_solve6(s_A6, s_rhs, s_x6, s_Ai, tid);
            if (tid == 0) s_solved = ok;
        }
        __syncthreads();
        if (P.didt_mode == 2 && s_solved) {
            // corrector: I(t+1) of the orientation the first solution predicts
            if (tid == 0) {
                double Wm[3], qp[4], Ip[9];
                for (int k = 0; k < 3; ++k) Wm[k] = 0.5 * (D->W[k] + s_x6[k + 3]);
                qstep27(D->q, Wm, qp);
                inertia27(qp, D->Ib, Ip);
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) s_A6[(i + 3) * 6 + j + 3] = D->zeta[(i + 3) * 6 + j + 3] + Ip[i * 3 + j];
            }
            __syncthreads();
            if (tid < 32) {
                const bool ok = q27_solve6(s_A6, s_rhs, s_x6, s_Ai, tid);
                if (tid == 0) s_solved = ok;
            }
            __syncthreads();
        }
        // F = F0 - zeta_F (U', W'), T = T0 - zeta_T (U', W'), one component per
        // thread; the new centre (Eq. posupdate) on three threads and the new
        // orientation (Eq. qnplus0-1, mean angular velocity of the step) on another
        if (tid < 6) {
            double z = 0.0;
            for (int j = 0; j < 6; ++j) z += D->zeta[tid * 6 + j] * s_x6[j];
            s_FT[tid] = (tid < 3 ? s_F0[tid] : s_T0[tid - 3]) - z;
        } else if (tid >= 32 && tid < 35) {
            const int k = tid - 32;
            s_xn[k] = D->x[k] + 0.5 * (D->U[k] + s_x6[k]);
        } else if (tid == 64) {
            double Wm[3];
            for (int k = 0; k < 3; ++k) Wm[k] = 0.5 * (D->W[k] + s_x6[k + 3]);
            qstep27(D->q, Wm, s_qn);
        }
        __syncthreads();
        if (s_solved) {
            // the new state, and the record F0, T0, F, T, U, W, x, q (finite or ST_NAN)
            if (tid < 9) {
                D->Iprev[tid] = s_In[tid];
                if (tid < 3) {
                    D->x[tid] = s_xn[tid];
                    D->U[tid] = s_x6[tid];
                    D->W[tid] = s_x6[tid + 3];
                }
                if (tid < 4) D->q[tid] = s_qn[tid];
            } else if (warp == 1) {
                double v = 0.0;
                if (lane < 3) v = s_F0[lane];
                else if (lane < 6) v = s_T0[lane - 3];
                else if (lane < 12) v = s_FT[lane - 6];
                else if (lane < 18) v = s_x6[lane - 12];
                else if (lane < 21) v = s_xn[lane - 18];
                else if (lane < 25) v = s_qn[lane - 21];
                if (lane < 25) D->rec[lane] = v;
                if (!__all_sync(0xffffffffu, lane >= 25 || isfinite(v)) && lane == 0) atomicOr(P.status, ST_NAN);
            }
        } else if (tid == 0) {
            atomicOr(P.status, ST_NAN);
        }
        __syncthreads();
    }
    // the cube of the new pose (origin floor(x) - h, side S = 2h + 2), one axis
    // per thread; the exact inside-test matrix of the new orientation on another
    // warp (lanes 0..8)
    if (tid < 3) {
        const int k = tid;
        const int L = k == 0 ? B.nx : (k == 1 ? B.ny : B.nz);
        const int o = (int)floor(D->x[k]) - D->h;
        s_o[k] = o;
        s_ow[k] = ((o % L) + L) % L;
        s_phi[k] = (double)o - D->x[k];
        s_d0[k] = (float)s_phi[k];                 // d = X - x_c at cube coordinate 0
        s_x[k] = D->x[k];
        if (k == 0) {
            s_ok = 1;
            if (!P.init) {
                if (__ldcg(P.status) & ST_NAN) s_ok = 0;
            }
            s_S = D->S;
            s_slot = P.init ? 0 : 1 - D->slot;
            s_nsol = 0;
            s_ncand = 0;
            s_band = D->band;                      // the FP32 decision band of the map (set on the host)
        }
    } else if (warp == 1) {
        canon_shape_warp(D->inv2, D->q, s_E, s_A, lane);
        if (lane < 9) s_A32[lane] = (float)s_A[lane];
    } else if (P.init && tid == 64) {
        inertia27(D->q, D->Ib, D->Iprev);          // I(t - 1) = I(t) before the first step
    }
    for (int k = tid; k < Q27 * NSUM; k += PBLK) (&s_sum[0][0])[k] = 0;
    __syncthreads();
    if (!s_ok) {
        for (int k = tid; k < (int)(sizeof(Part27) / 8); k += PBLK)
            reinterpret_cast<unsigned long long*>(G)[k] = reinterpret_cast<const unsigned long long*>(&sD)[k];
        return;
    }
    const int S = s_S;
    const uint64_t full = S == 64 ? ~0ull : ((1ull << S) - 1ull);
    // ---- occupancy of the new pose: FP32 outside the band, band nodes listed
    for (int r = tid; r < S * S; r += PBLK) {
        const int my = r % S, mz = r / S;
        const float dy = s_d0[1] + (float)my, dz = s_d0[2] + (float)mz;
        const float qa = s_A32[0], qb = 2.0f * (s_A32[1] * dy + s_A32[2] * dz);
        const float qc = s_A32[4] * dy * dy + 2.0f * s_A32[5] * dy * dz + s_A32[8] * dz * dz;
        const float band = s_band;
        uint64_t w = 0;
        for (int mx = 0; mx < S; ++mx) {
            const float dx = s_d0[0] + (float)mx;
            const float v = (qa * dx + qb) * dx + qc;
            if (fabsf(v - 1.0f) > band) {
                if (v < 1.0f) w |= 1ull << mx;
            } else {
                const int c = atomicAdd(&s_ncand, 1);
                if (c < NCAND) {
                    s_cand[c] = (mz << 16) | (my << 8) | mx;
                } else {
                    const int X = wrapc(s_ow[0] + mx, B.nx), Y = wrapc(s_ow[1] + my, B.ny),
                              Z = wrapc(s_ow[2] + mz, B.nz);
                    if (canon_value(s_A, s_x, X, Y, Z, B.nx, B.ny, B.nz, true) <= 1.0) w |= 1ull << mx;
                }
            }
        }
        s_map[r] = w;
    }
    __syncthreads();
    {
        const int nc = min(s_ncand, NCAND);
        for (int c = tid; c < nc; c += PBLK) {
            const int code = s_cand[c];
            const int mx = code & 0xff, my = (code >> 8) & 0xff, mz = code >> 16;
            const int X = wrapc(s_ow[0] + mx, B.nx), Y = wrapc(s_ow[1] + my, B.ny), Z = wrapc(s_ow[2] + mz, B.nz);
            if (canon_value(s_A, s_x, X, Y, Z, B.nx, B.ny, B.nz, true) <= 1.0)
                atomicOr(reinterpret_cast<unsigned long long*>(&s_map[mz * S + my]), 1ull << mx);
        }
    }
    __syncthreads();
    // ---- solid nodes; the map into its global slot (the lattice kernel and the
    // read-back use it); links of the new map summed per direction in integers:
    // thread t takes direction 1 + t % 26 over the rows g, g + NG, ... (g = t / 26);
    // the sums of x and x^2 over a row's link bits come from popcounts of the
    // masks of bit positions whose bit p is set (x = sum_p 2^p [bit p of x])
    {
        uint64_t* map = P.rows + ((size_t)p * 2 + s_slot) * RW;
        int ns = 0;
        for (int r = tid; r < S * S; r += PBLK) {
            const uint64_t w = s_map[r];
            map[r] = w;
            ns += __popcll(w);
        }
        ns = __reduce_add_sync(0xffffffffu, ns);
        if (lane == 0 && ns) atomicAdd(&s_nsol, ns);
    }
    {
        const int b = 1 + tid % (Q27 - 1), g = tid / (Q27 - 1);
        if (g < NG) {
            int t[NSUM];
#pragma unroll
            for (int k = 0; k < NSUM; ++k) t[k] = 0;
            const int cx = cx27(b), cy = cy27(b), cz = cz27(b);
            const uint64_t M[6] = {0xAAAAAAAAAAAAAAAAull, 0xCCCCCCCCCCCCCCCCull, 0xF0F0F0F0F0F0F0F0ull,
                                   0xFF00FF00FF00FF00ull, 0xFFFF0000FFFF0000ull, 0xFFFFFFFF00000000ull};
            int my = g % S, mz = g / S;
            for (int r = g; r < S * S; r += NG) {
                const int ny_ = my + cy, nz_ = mz + cz;
                if (ny_ >= 0 && nz_ >= 0 && ny_ < S && nz_ < S) {
                    const uint64_t nb = s_map[nz_ * S + ny_];
                    const uint64_t sol = cx == 1 ? (nb >> 1) : (cx == -1 ? (nb << 1) : nb);
                    uint64_t L = ~s_map[r] & sol & full;
                    if (L) {
                        const int n = __popcll(L);
                        int sx = 0, sxx = 0;
                        if (n <= 4) {
                            // a few links: their positions one by one
                            while (L) {
                                const int x = __ffsll((long long)L) - 1;
                                L &= L - 1;
                                sx += x;
                                sxx += x * x;
                            }
                        } else {
                            int pc[6];
#pragma unroll
                            for (int q = 0; q < 6; ++q) {
                                pc[q] = __popcll(L & M[q]);
                                sx += pc[q] << q;
                                sxx += pc[q] << (2 * q);
                            }
#pragma unroll
                            for (int q = 0; q < 6; ++q)
#pragma unroll
                                for (int q2 = q + 1; q2 < 6; ++q2) sxx += __popcll(L & M[q] & M[q2]) << (q + q2 + 1);
                        }
                        t[0] += n; t[1] += sx; t[2] += n * my; t[3] += n * mz; t[4] += sxx;
                        t[5] += sx * my; t[6] += sx * mz; t[7] += n * my * my; t[8] += n * my * mz; t[9] += n * mz * mz;
                    }
                }
                my += NG;
                while (my >= S) { my -= S; ++mz; }
            }
#pragma unroll
            for (int k = 0; k < NSUM; ++k)
                if (t[k]) atomicAdd(&s_sum[b][k], t[k]);
        }
    }
    __syncthreads();
    // each direction's share of the drag matrix and of F0g / T0g: thread b the
    // translational and mixed blocks, thread 32 + b (another warp) the
    // rotational block
    if ((tid >= 1 && tid < Q27) || (tid >= 33 && tid < 32 + Q27)) {
        const int b = tid & 31;
        const bool rot = tid >= 32;
        const double rho0 = B.rho0;
        const double* phi = s_phi;
        double* out = s_con[b];
        const int* t = s_sum[b];
        const double n = t[0];
        const double c[3] = {(double)cx27(b), (double)cy27(b), (double)cz27(b)};
        const double Sm[3] = {(double)t[1], (double)t[2], (double)t[3]};
        // p x c = K p, K = -[c]x, p = phi + m over the direction's links
        const double K[9] = {0.0, c[2], -c[1], -c[2], 0.0, c[0], c[1], -c[0], 0.0};
        const double wz = 6.0 * rho0 * wd27(b);        // 2 rho0 w_b / c_s^2
        if (!rot) {
            double Pb[3], KP[3];
            for (int i = 0; i < 3; ++i) Pb[i] = n * phi[i] + Sm[i];
            for (int i = 0; i < 3; ++i) KP[i] = K[i * 3] * Pb[0] + K[i * 3 + 1] * Pb[1] + K[i * 3 + 2] * Pb[2];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    out[i * 6 + j] = wz * n * c[i] * c[j];
                    out[i * 6 + j + 3] = wz * c[i] * KP[j];
                    out[(i + 3) * 6 + j] = wz * KP[i] * c[j];
                }
            for (int i = 0; i < 3; ++i) {
                out[36 + i] = 2.0 * rho0 * wd27(b) * n * c[i];
                out[39 + i] = 2.0 * rho0 * wd27(b) * KP[i];
            }
        } else {
            const double Qm[9] = {(double)t[4], (double)t[5], (double)t[6], (double)t[5], (double)t[7],
                                  (double)t[8], (double)t[6], (double)t[8], (double)t[9]};
            double PP[9], KPP[9];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    PP[i * 3 + j] = n * phi[i] * phi[j] + phi[i] * Sm[j] + Sm[i] * phi[j] + Qm[i * 3 + j];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    KPP[i * 3 + j] = K[i * 3] * PP[j] + K[i * 3 + 1] * PP[3 + j] + K[i * 3 + 2] * PP[6 + j];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j)
                    out[(i + 3) * 6 + j + 3] =
                        wz * (KPP[i * 3] * K[j * 3] + KPP[i * 3 + 1] * K[j * 3 + 1] + KPP[i * 3 + 2] * K[j * 3 + 2]);
        }
    }
    __syncthreads();
    // every entry summed over the 26 directions: a warp per entry, lane l the
    // direction l + 1, a shuffle tree (five dependent additions)
    for (int e = warp; e < 42; e += PBLK / 32) {
        double v = lane < Q27 - 1 ? s_con[lane + 1][e] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0) {
            if (e < 36) D->zeta[e] = v;
            else if (e < 39) D->F0g[e - 36] = v;
            else D->T0g[e - 39] = v;
        }
    }
    __syncthreads();
    // the new state, one thread per axis (thread 0 also the scalars)
    if (tid < 3) {
        const int i = tid;
        const int ns = s_nsol;
        Dyn27& Y = P.dyn[D->box];
        // the map the next pass bounces back from is the current one
        const int Lk = i == 0 ? B.nx : (i == 1 ? B.ny : B.nz);
        Y.phi_old[i] = P.init ? (float)s_phi[i] : (float)D->phi[i];
        Y.o_old[i] = P.init ? s_ow[i] : ((D->o[i] % Lk) + Lk) % Lk;
        // the box that holds both cubes (the near pass covers its nodes)
        const int lo = P.init ? s_o[i] : min(D->o[i], s_o[i]);
        const int hi = (P.init ? s_o[i] : max(D->o[i], s_o[i])) + S;
        Y.E[i] = min(hi - lo, Lk);
        Y.uo[i] = ((lo % Lk) + Lk) % Lk;
        if (!P.init && abs(s_o[i] - D->o[i]) > 1) atomicOr(P.status, ST_CAPACITY);
        Y.phi_new[i] = (float)s_phi[i];
        Y.o_new[i] = s_ow[i];
        Y.U[i] = (float)D->U[i];
        Y.W[i] = (float)D->W[i];
        // uniform terms of the next collision: body force (with the counter
        // force on the fluid nodes of the new map) and the mass of this remap,
        // returned over every fluid node
        const double inf = 1.0 / (double)(B.N - ns);
        Y.g[i] = (float)(B.body[i] - (B.counter ? D->Fext[i] * inf : 0.0));
        if (i == 0) {
            Y.slot_old = P.init ? s_slot : D->slot;
            Y.slot_new = s_slot;
            Y.S = S;
            Y.active = 1;
            Y.eps = P.init ? 0.0f : (float)(D->dm * inf);
        }
    }
    __syncthreads();
    if (tid < 3) {
        D->phi[tid] = s_phi[tid];
        D->o[tid] = s_o[tid];
        if (tid == 0) {
            D->slot = s_slot;
            D->nsolid = s_nsol;
        }
    }
    __syncthreads();
    for (int k = tid; k < (int)(sizeof(Part27) / 8); k += PBLK)
        reinterpret_cast<unsigned long long*>(G)[k] = reinterpret_cast<const unsigned long long*>(&sD)[k];
}

// ---------------------------------------------------------------------------
// Read-back of one box: the pre-collision populations of the current time
// (the first half of a lattice pass: pull, bounce-back, remap), their
// density and velocity (u = (sum f c + g/2) / rho, g of the next collision),
// and the occupancy.  Solid nodes read 0.
__global__ void __launch_bounds__(LBLOCK) fields27_kernel(const __grid_constant__ FieldParams27 P)
{
    const Box27 B = P.boxes[P.box];
    const Dyn27 K = P.dyn[P.box];
    const int node = blockIdx.x * LBLOCK + threadIdx.x;
    if (node >= (int)B.N) return;
    const int X = node % B.nx, Y = (node / B.nx) % B.ny, Z = node / (B.nx * B.ny);
    const uint64_t* rows = K.active ? P.rows + (size_t)B.p * 2 * RW : nullptr;
    float d[Q27];
    int mn[3] = {0, 0, 0};
    bool in_new = false;
    unsigned nb_new = 0;
    const int kind = pre_collision(B, K, rows, P.src + B.off, X, Y, Z, node, P.nopull != 0, d, mn, in_new, nb_new);
    const bool solid = kind == K_SOLID || kind == K_COVERED;
    float drho = 0.0f, j[3] = {0.0f, 0.0f, 0.0f};
#pragma unroll
    for (int i = 0; i < Q27; ++i) {
        const float v = solid ? 0.0f : d[i];
        if (P.out_f) P.out_f[(size_t)i * B.N + node] = solid ? 0.0f : (P.out_dev ? v : v + w27(i) * B.rho0f);
        drho += v;
        j[0] += cx27(i) * v;
        j[1] += cy27(i) * v;
        j[2] += cz27(i) * v;
    }
    if (P.out_rho) P.out_rho[node] = solid ? 0.0f : drho;
    if (P.out_u)
        for (int k = 0; k < 3; ++k) P.out_u[(size_t)k * B.N + node] = solid ? 0.0f : (j[k] + 0.5f * K.g[k]) / (B.rho0f + drho);
    if (P.out_solid) P.out_solid[node] = solid ? 1 : 0;
}

// Boundary links of particle p's current map: pairs (node index in its box,
// direction b) for every fluid node x with x + c_b solid
__global__ void links27_kernel(const Part27* pd, const Box27* boxes, const uint64_t* rows, int p, int* out, int cap,
                               int* count)
{
    const Part27& D = pd[p];
    const Box27 B = boxes[D.box];
    const int S = D.S;
    const uint64_t* map = rows + ((size_t)p * 2 + D.slot) * RW;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= S * S) return;
    const int my = r % S, mz = r / S;
    const int L[3] = {B.nx, B.ny, B.nz};
    int ow[3];
    for (int k = 0; k < 3; ++k) ow[k] = ((D.o[k] % L[k]) + L[k]) % L[k];
    const uint64_t own = map[r];
    for (int mx = 0; mx < S; ++mx) {
        if ((own >> mx) & 1ull) continue;
        for (int b = 1; b < Q27; ++b) {
            const int ax = mx + cx27(b), ay = my + cy27(b), az = mz + cz27(b);
            if (ax < 0 || ay < 0 || az < 0 || ax >= S || ay >= S || az >= S) continue;
            if (!((map[az * S + ay] >> ax) & 1ull)) continue;
            const int X = wrapc(ow[0] + mx, B.nx), Y = wrapc(ow[1] + my, B.ny), Z = wrapc(ow[2] + mz, B.nz);
            const int k = atomicAdd(count, 1);
            if (k < cap) {
                out[2 * k] = (Z * B.ny + Y) * B.nx + X;
                out[2 * k + 1] = b;
            }
        }
    }
}

// after new external forces: the counter force of the next collision,
// -F_ext / N_fluid on the fluid nodes of the current map (one thread per particle)
__global__ void refresh27_kernel(const Part27* pd, const Box27* boxes, Dyn27* dyn, int np)
{
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= np) return;
    const Part27& D = pd[p];
    const Box27& B = boxes[D.box];
    const double nf = (double)(B.N - D.nsolid);
    for (int i = 0; i < 3; ++i) dyn[D.box].g[i] = (float)(B.body[i] - (B.counter ? D.Fext[i] / nf : 0.0));
}

cudaError_t launch_refresh27(const Part27* pd, const Box27* boxes, Dyn27* dyn, int np, cudaStream_t s)
{
    if (np <= 0) return cudaSuccess;
    refresh27_kernel<<<(np + 127) / 128, 128, 0, s>>>(pd, boxes, dyn, np);
    return cudaGetLastError();
}

cudaError_t launch_lattice27(const LatParams27& p, int blocks, cudaStream_t s)
{
    if (p.ghost)
        lattice27_kernel<true><<<blocks, LBLOCK, 0, s>>>(p);
    else
        lattice27_kernel<false><<<blocks, LBLOCK, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_bulk27(const LatParams27& p, int blocks, cudaStream_t s)
{
    if (p.ghost)
        bulk27_kernel<true><<<blocks, LBLOCK, 0, s>>>(p);
    else
        bulk27_kernel<false><<<blocks, LBLOCK, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_particles27(const PartParams27& p, int np, cudaStream_t s)
{
    if (np <= 0) return cudaSuccess;
    particle27_kernel<<<np, PBLK, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_fields27(const FieldParams27& p, int blocks, cudaStream_t s)
{
    fields27_kernel<<<blocks, LBLOCK, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_links27(const Part27* pd, const Box27* boxes, const uint64_t* rows, int p, int* out, int cap,
                           int* count, cudaStream_t s)
{
    // one thread per cube row (at most 64 x 64)
    links27_kernel<<<(MAXS * MAXS + 255) / 256, 256, 0, s>>>(pd, boxes, rows, p, out, cap, count);
    return cudaGetLastError();
}

}  // namespace q27
}  // namespace lbsph
