// Field read-back kernel (lb_get_fields): the pre-collision state of every
// node of one box at the start of iteration t, i.e. the second half of
// iteration t-1 of the paper's Appendix (step 2 streaming, step 6 bounce-back
// with U(t), Omega(t), the remap of step 8) without the collision, with
// density and velocity moments.  Every decision is taken per node from the
// occupancy maps, in a layout independent of the bulk + boundary kernels that
// advance the simulation, so the read-back also cross-checks them.
//
// Thread mapping: one thread per 4 consecutive x nodes ("quad"), 256 threads
// per block, blocks in x-fastest order over the box.  Each direction is read
// with one 16-byte load of the source row; the +-1 shift in x comes from the
// neighbouring lane by a warp shuffle (a scalar load at warp and row ends,
// which also wraps x periodically).  Threads whose nodes (grown by one) touch
// a particle's bounding cube or a wall test them against the occupancy
// bitmaps (old map for the streaming sources, new map for the node itself).
#include "lattice_common.cuh"

namespace lbsph {

// one cached particle for a tile
struct CandK {
    const uint64_t* rows_old;
    const uint64_t* rows_new;
    int ow_old[3], ow_new[3];
    int S, gidx;
    float ro_old[3], ro_new[3], U[3], W[3], e_old[3];
    float a, b, eps2, B1, B2;
    int squirmer;
};

// Is lattice node (X, Y, Z) (wrapped into the box) a solid node of one of the
// cached particles?  old selects map t-1 (streaming sources) or map t.
__device__ __forceinline__ int lookup(const CandK* cs, int nc, bool old, int X, int Y, int Z, int nx,
                                      int ny, int nz, int& mx, int& my, int& mz)
{
    for (int c = 0; c < nc; ++c) {
        const int* ow = old ? cs[c].ow_old : cs[c].ow_new;
        const int S = cs[c].S;
        const int ax = wrapd(X - ow[0], nx);
        if (ax >= S) continue;
        const int ay = wrapd(Y - ow[1], ny);
        if (ay >= S) continue;
        const int az = wrapd(Z - ow[2], nz);
        if (az >= S) continue;
        const uint64_t* rows = old ? cs[c].rows_old : cs[c].rows_new;
        if ((rows[az * S + ay] >> ax) & 1ull) {
            mx = ax; my = ay; mz = az;
            return c;
        }
    }
    return -1;
}

// Occupancy of the 6 nodes x = X0-1 .. X0+4 of row (Y, Z) (wrapped) in one
// particle's bitmap, as bits 0..5.
__device__ __forceinline__ unsigned window6(const uint64_t* rows, int S, const int ow[3], int X0, int Y, int Z,
                                            int nx, int ny, int nz)
{
    const int ay = wrapd(Y - ow[1], ny);
    if (ay >= S) return 0u;
    const int az = wrapd(Z - ow[2], nz);
    if (az >= S) return 0u;
    const uint64_t word = rows[az * S + ay];
    if (!word) return 0u;
    unsigned m = 0u;
#pragma unroll
    for (int j = 0; j < 6; ++j) {
        const int X = wrapd(X0 - 1 + j, nx);
        const int ax = wrapd(X - ow[0], nx);
        if (ax < S) m |= (unsigned)((word >> ax) & 1ull) << j;
    }
    return m;
}

__device__ __forceinline__ void slip_f32(const CandK& c, float rx, float ry, float rz, float& sx,
                                         float& sy, float& sz)
{
    squirmer_slip(c.e_old, c.a, c.eps2, c.B1, c.B2, rx, ry, rz, sx, sy, sz);
}

// Does the range [lo, hi] of a periodic axis of length L meet [ow, ow+S-1] (mod L)?
__device__ __forceinline__ bool hits(int lo, int hi, int ow, int S, int L)
{
    if (hi - lo + 1 >= L) return true;
    int d = (lo - ow) % L;
    if (d < 0) d += L;
    if (d < S) return true;
    return (hi - lo) >= (L - d);
}

// ---------------------------------------------------------------------------
template <class St>
__global__ void __launch_bounds__(KBLOCK) fields_kernel(const KParams P)
{
    using T = typename St::T;
    __shared__ CandK s_c[MAXC];
    __shared__ int s_nc;
    __shared__ float s_g[3];

    // ---- box of this block
    const int bi = P.only_box;
    const int blk = blockIdx.x + P.boxes[bi].block_begin;
    const BoxDev& B = P.boxes[bi];
    const int nx = B.nx, ny = B.ny, nz = B.nz, nxq = B.nxq;
    const long long N = B.N;
    const long long q0 = (long long)(blk - B.block_begin) * KBLOCK;
    const long long qlast = min(q0 + KBLOCK, B.nq) - 1;

    // ---- particles near the tile, box forces (warp 0)
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        const long long r0 = q0 / nxq, r1 = qlast / nxq;
        const int z0 = (int)(r0 / ny), y0 = (int)(r0 % ny), z1 = (int)(r1 / ny), y1 = (int)(r1 % ny);
        int ylo, yhi;
        if (z0 == z1) { ylo = y0 - 1; yhi = y1 + 1; } else { ylo = -1; yhi = ny; }
        const int zlo = z0 - 1, zhi = z1 + 1;
        int nc = 0;
        double fx = 0.0, fy = 0.0, fz = 0.0;
        long long nsol = 0;
        for (int base = 0; base < B.pcnt; base += 32) {
            const int pi = base + lane;
            bool hit = false;
            if (pi < B.pcnt) {
                const PartK& k = P.pk[B.pbeg + pi];
                hit = (hits(ylo, yhi, k.ow_old[1], k.S, ny) && hits(zlo, zhi, k.ow_old[2], k.S, nz)) ||
                      (hits(ylo, yhi, k.ow_new[1], k.S, ny) && hits(zlo, zhi, k.ow_new[2], k.S, nz));
                fx += k.Fext[0]; fy += k.Fext[1]; fz += k.Fext[2];
                nsol += k.nsolid;
            }
            unsigned m = __ballot_sync(0xffffffffu, hit);
            while (m) {
                const int l = __ffs(m) - 1;
                m &= m - 1;
                if (lane == 0) {
                    if (nc < MAXC) {
                        const PartK& k = P.pk[B.pbeg + base + l];
                        CandK& c = s_c[nc];
                        c.rows_old = k.rows_old; c.rows_new = k.rows_new;
                        for (int a = 0; a < 3; ++a) {
                            c.ow_old[a] = k.ow_old[a]; c.ow_new[a] = k.ow_new[a];
                            c.ro_old[a] = k.ro_old[a]; c.ro_new[a] = k.ro_new[a];
                            c.U[a] = k.U[a]; c.W[a] = k.W[a]; c.e_old[a] = k.e_old[a];
                        }
                        c.S = k.S; c.gidx = B.pbeg + base + l;
                        c.a = k.a; c.b = k.b; c.eps2 = k.eps2; c.B1 = k.B1; c.B2 = k.B2;
                        c.squirmer = k.squirmer;
                    } else {
                        atomicOr(P.status, ST_CAPACITY);
                    }
                }
                ++nc;
            }
        }
        for (int o = 16; o > 0; o >>= 1) {
            fx += __shfl_xor_sync(0xffffffffu, fx, o);
            fy += __shfl_xor_sync(0xffffffffu, fy, o);
            fz += __shfl_xor_sync(0xffffffffu, fz, o);
            nsol += __shfl_xor_sync(0xffffffffu, nsol, o);
        }
        if (lane == 0) {
            const double nf = (double)(N - B.nwall - nsol);
            double g[3] = {B.body[0], B.body[1], B.body[2]};
            if (B.counter && nf > 0) { g[0] -= fx / nf; g[1] -= fy / nf; g[2] -= fz / nf; }
            s_g[0] = (float)g[0]; s_g[1] = (float)g[1]; s_g[2] = (float)g[2];
            s_nc = nc < MAXC ? nc : MAXC;
        }
    }
    __syncthreads();
    const int nc = s_nc;
    const float gx = s_g[0], gy = s_g[1], gz = s_g[2];

    // ---- this thread's quad
    long long q = q0 + threadIdx.x;
    const bool valid = q < B.nq;
    if (!valid) q = B.nq - 1;
    const int xq = (int)(q % nxq);
    const long long row = q / nxq;
    const int y = (int)(row % ny), z = (int)(row / ny);
    const int lane = threadIdx.x & 31;
    const T* A = reinterpret_cast<const T*>(P.src) + B.off;
    const float inv = B.inv_scale;
    const unsigned long long pol = l2_evict_normal();

    long long rofs[3][3];  // element offset of source rows (y + dy, z + dz), wrapped
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

    // ---- pull (stream): v[i] = f*_i(x - c_i) for the 4 nodes
    const bool first = P.nopull != 0;
    float4 v[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (first) {
            // before the first collision: the initial distributions in place
            v[i] = St::ld4(A + (long long)i * N + rofs[1][1] + 4 * xq, inv, pol);
            continue;
        }
        const T* rp = A + (long long)i * N + rofs[1 - cy_of(i)][1 - cz_of(i)];
        float4 t = St::ld4(rp + 4 * xq, inv, pol);
        if (cx_of(i) == 1) {           // source x - 1
            float l = __shfl_up_sync(0xffffffffu, t.w, 1);
            if (left_ld) l = St::ld1(rp + (xq == 0 ? nx - 1 : 4 * xq - 1), inv, pol);
            t = make_float4(l, t.x, t.y, t.z);
        } else if (cx_of(i) == -1) {   // source x + 1
            float r = __shfl_down_sync(0xffffffffu, t.x, 1);
            if (right_ld) r = St::ld1(rp + (xq == nxq - 1 ? 0 : 4 * xq + 4), inv, pol);
            t = make_float4(t.y, t.z, t.w, r);
        }
        v[i] = t;
    }

    // ---- only threads whose nodes (grown by one) touch a particle cube or a
    // wall test nodes; they read the neighbourhood occupancy as 6-bit windows
    // of the 9 rows (y + dy, z + dz)
    bool near = B.walls && (y <= 1 || y >= ny - 2);
    for (int c = 0; c < nc; ++c) {
        const CandK& C = s_c[c];
        near = near ||
               (hits(y - 1, y + 1, C.ow_old[1], C.S, ny) && hits(z - 1, z + 1, C.ow_old[2], C.S, nz) &&
                hits(4 * xq - 1, 4 * xq + 4, C.ow_old[0], C.S, nx)) ||
               (hits(y - 1, y + 1, C.ow_new[1], C.S, ny) && hits(z - 1, z + 1, C.ow_new[2], C.S, nz) &&
                hits(4 * xq - 1, 4 * xq + 4, C.ow_new[0], C.S, nx));
    }
    const long long own = row * nx + 4 * xq;
    const float rho0 = B.rho0f;
    float rho_out[4], u_out[4][3];
    int solid_out[4];
    unsigned so[3][3], sn[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) { so[a][b] = 0u; sn[a][b] = 0u; }
    if (near) {
        for (int c = 0; c < nc; ++c) {
            const CandK& C = s_c[c];
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const int Y = wrapd(y + a - 1, ny), Z = wrapd(z + b - 1, nz);
                    if (!first) so[a][b] |= window6(C.rows_old, C.S, C.ow_old, 4 * xq, Y, Z, nx, ny, nz);
                    sn[a][b] |= window6(C.rows_new, C.S, C.ow_new, 4 * xq, Y, Z, nx, ny, nz);
                }
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int X = 4 * xq + k;
        bool skip = !valid;
        rho_out[k] = 0.f; u_out[k][0] = u_out[k][1] = u_out[k][2] = 0.f;
        solid_out[k] = 0;
        float f[Q];
        const bool wallrow = B.walls && (y == 0 || y == ny - 1);
        const bool sol_old = !wallrow && ((so[1][1] >> (k + 1)) & 1u);
        const bool sol_new = !wallrow && ((sn[1][1] >> (k + 1)) & 1u);
        int mx, my, mz;
        if (wallrow) {
            skip = true;
            solid_out[k] = -1;
        } else if (sol_new && (sol_old || first)) {
            skip = true;                         // solid before and after
            const int c = lookup(s_c, nc, false, X, y, z, nx, ny, nz, mx, my, mz);
            solid_out[k] = c >= 0 ? s_c[c].gidx - B.pbeg + 1 : 0;
        } else if (sol_old) {
            // uncovered: f = f_eq(rho0, U + Omega x r) (remap, step 8)
            const int c0 = lookup(s_c, nc, true, X, y, z, nx, ny, nz, mx, my, mz);
            const CandK& c = s_c[c0 < 0 ? 0 : c0];
            const int ax = wrapd(X - c.ow_new[0], nx), ay = wrapd(y - c.ow_new[1], ny), az = wrapd(z - c.ow_new[2], nz);
            const float rx = c.ro_new[0] + ax, ry = c.ro_new[1] + ay, rz = c.ro_new[2] + az;
            const float ux = c.U[0] + (c.W[1] * rz - c.W[2] * ry);
            const float uy = c.U[1] + (c.W[2] * rx - c.W[0] * rz);
            const float uz = c.U[2] + (c.W[0] * ry - c.W[1] * rx);
            const float uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                const float cu = cx_of(i) * ux + cy_of(i) * uy + cz_of(i) * uz;
                f[i] = w_of(i) * rho0 * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu);
            }
        } else {
            // fluid at t-1: pulled populations, bounce-back where the source was solid
#pragma unroll
            for (int i = 0; i < Q; ++i) f[i] = comp(v[i], k);
            if (!first && near) {
#pragma unroll
                for (int i = 1; i < Q; ++i) {
                    const int Ys = y - cy_of(i);
                    if (B.walls && (Ys == 0 || Ys == ny - 1)) {
                        const float* uw = (Ys == 0) ? B.uw_lo : B.uw_hi;
                        const float ubc = cx_of(i) * uw[0] + cy_of(i) * uw[1] + cz_of(i) * uw[2];
                        f[i] = St::ld1(A + (long long)opp_of(i) * N + own + k, inv, pol) + 6.0f * w_of(i) * rho0 * ubc;
                        continue;
                    }
                    if (!((so[1 - cy_of(i)][1 - cz_of(i)] >> (k + 1 - cx_of(i))) & 1u)) continue;
                    int sx, sy, sz;
                    const int c = lookup(s_c, nc, true, wrapd(X - cx_of(i), nx), wrapd(Ys, ny),
                                         wrapd(z - cz_of(i), nz), nx, ny, nz, sx, sy, sz);
                    if (c < 0) continue;
                    const CandK& C = s_c[c];
                    const float rx = C.ro_old[0] + sx + 0.5f * cx_of(i);
                    const float ry = C.ro_old[1] + sy + 0.5f * cy_of(i);
                    const float rz = C.ro_old[2] + sz + 0.5f * cz_of(i);
                    float ux = C.U[0] + (C.W[1] * rz - C.W[2] * ry);
                    float uy = C.U[1] + (C.W[2] * rx - C.W[0] * rz);
                    float uz = C.U[2] + (C.W[0] * ry - C.W[1] * rx);
                    if (C.squirmer) {
                        float qx, qy, qz;
                        slip_f32(C, rx, ry, rz, qx, qy, qz);
                        ux += qx; uy += qy; uz += qz;
                    }
                    const float ubc = cx_of(i) * ux + cy_of(i) * uy + cz_of(i) * uz;
                    f[i] = St::ld1(A + (long long)opp_of(i) * N + own + k, inv, pol) + 6.0f * w_of(i) * rho0 * ubc;
                }
            }
            if (sol_new) {
                // covered: its mass and momentum go to the particle (remap, step 8)
                skip = true;
                const int c = lookup(s_c, nc, false, X, y, z, nx, ny, nz, mx, my, mz);
                solid_out[k] = c >= 0 ? s_c[c].gidx - B.pbeg + 1 : 0;
            }
        }
        if (skip) {
#pragma unroll
            for (int i = 0; i < Q; ++i) set_comp(v[i], k, 0.0f);
            continue;
        }
        float drho = 0.f;
#pragma unroll
        for (int i = 0; i < Q; ++i) drho += f[i];
        const float jx = (f[1] - f[2]) + (f[7] - f[8]) + (f[9] - f[10]) + (f[11] - f[12]) + (f[13] - f[14]);
        const float jy = (f[3] - f[4]) + (f[7] - f[8]) - (f[9] - f[10]) + (f[15] - f[16]) + (f[17] - f[18]);
        const float jz = (f[5] - f[6]) + (f[11] - f[12]) - (f[13] - f[14]) + (f[15] - f[16]) - (f[17] - f[18]);
        const float ir = 1.0f / (rho0 + drho);
        rho_out[k] = drho;
        u_out[k][0] = (jx + 0.5f * gx) * ir;
        u_out[k][1] = (jy + 0.5f * gy) * ir;
        u_out[k][2] = (jz + 0.5f * gz) * ir;
#pragma unroll
        for (int i = 0; i < Q; ++i) set_comp(v[i], k, P.out_dev ? f[i] : f[i] + w_of(i) * rho0);
    }

    if (valid) {
        if (P.out_f) {
#pragma unroll
            for (int i = 0; i < Q; ++i)
                *reinterpret_cast<float4*>(P.out_f + (long long)i * N + own) = v[i];
        }
        if (P.out_rho) *reinterpret_cast<float4*>(P.out_rho + own) = make_float4(rho_out[0], rho_out[1], rho_out[2], rho_out[3]);
        if (P.out_u) {
#pragma unroll
            for (int a = 0; a < 3; ++a)
                *reinterpret_cast<float4*>(P.out_u + (long long)a * N + own) =
                    make_float4(u_out[0][a], u_out[1][a], u_out[2][a], u_out[3][a]);
        }
        if (P.out_solid) *reinterpret_cast<int4*>(P.out_solid + own) = make_int4(solid_out[0], solid_out[1], solid_out[2], solid_out[3]);
    }
}

// ---------------------------------------------------------------------------
// Field read-back: pre-collision populations at the start of iteration t
// (streaming, bounce-back and remap fix-ups of t-1 without a collision), every
// tile tested against the particles' occupancy maps.
template <class St>
static cudaError_t launch_mode(const KParams& p, int blocks, cudaStream_t s)
{
    fields_kernel<St><<<blocks, KBLOCK, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_fields(const KParams& p, int precision, int blocks, cudaStream_t s)
{
    if (precision == 1) return launch_mode<StF16>(p, blocks, s);
    if (precision == 2) return launch_mode<StBF16>(p, blocks, s);
    return launch_mode<StF32>(p, blocks, s);
}

}  // namespace lbsph
