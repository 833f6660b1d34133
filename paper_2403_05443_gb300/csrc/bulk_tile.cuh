// One 256-quad tile of the bulk lattice kernel (see bulk_kernel.cu), shared by
// the bulk kernel and the persistent step kernel.
#pragma once

#include "lattice_common.cuh"

namespace lbsph {

// quad tix (0..255) of tile `tile`; the 32 quads of a warp are consecutive
template <class St, bool FIRST>
__device__ __forceinline__ void bulk_tile(const BulkParams& P, int tile, int tix)
{
    using T = typename St::T;
    const int bi = __ldg(P.blk_box + tile);
    const BoxDev& B = P.boxes[bi];
    const int nx = B.nx, ny = B.ny, nz = B.nz, nxq = B.nxq;
    // every offset within a box fits in 32 bits: 19 N < 2^31 (checked at lb_create)
    const int N = (int)B.N;
    int q = (tile - B.block_begin) * KBLOCK + tix;
    const bool valid = q < (int)B.nq;
    if (!valid) q = (int)B.nq - 1;
    const int row = div_magic(q, B.dq_m, B.dq_s);
    const int xq = q - row * nxq;
    const int z = div_magic(row, B.dy_m, B.dy_s);
    const int y = row - z * ny;
    const int lane = tix & 31;
    const T* A = reinterpret_cast<const T*>(P.src) + B.off;
    T* D = reinterpret_cast<T*>(P.dst) + B.off;
    const int own = row * nx + 4 * xq;
    const unsigned long long pol_first = l2_evict_first();

    int rofs[3][3];  // element offsets of the source rows (y + dy, z + dz), wrapped
    {
        const int yy[3] = {y == 0 ? ny - 1 : y - 1, y, y == ny - 1 ? 0 : y + 1};
        const int zz[3] = {z == 0 ? nz - 1 : z - 1, z, z == nz - 1 ? 0 : z + 1};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) rofs[a][b] = (zz[b] * ny + yy[a]) * nx;
    }
    float4 v[Q];
    if (FIRST) {
        // first collision: the initial distributions of the node itself
        // (rest, or a field set by lb_init_fluid), no streaming
#pragma unroll
        for (int i = 0; i < Q; ++i) v[i] = St::ld4r(A + (i * N + own), pol_first);
    } else if (B.rowwarp) {
        // every row lies within this warp's 32 quads (nxq divides 32 and
        // the unit starts a row): the periodic wrap in x is a shuffle too
        const int srcl = xq == 0 ? lane + nxq - 1 : lane - 1;
        const int srcr = xq == nxq - 1 ? lane - nxq + 1 : lane + 1;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            float4 t = St::ld4r(A + (i * N + rofs[1 - cy_of(i)][1 - cz_of(i)] + 4 * xq), pol_first);
            if (cx_of(i) == 1) t = make_float4(__shfl_sync(0xffffffffu, t.w, srcl), t.x, t.y, t.z);
            else if (cx_of(i) == -1) t = make_float4(t.y, t.z, t.w, __shfl_sync(0xffffffffu, t.x, srcr));
            v[i] = t;
        }
    } else {
        const bool left_ld = (lane == 0) || (xq == 0);
        const bool right_ld = (lane == 31) || (xq == nxq - 1);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const T* rp = A + (i * N + rofs[1 - cy_of(i)][1 - cz_of(i)]);
            float4 t = St::ld4r(rp + 4 * xq, pol_first);
            if (cx_of(i) == 1) {            // source x - 1
                float l = __shfl_up_sync(0xffffffffu, t.w, 1);
                if (left_ld) l = St::ld1r(rp + (xq == 0 ? nx - 1 : 4 * xq - 1), pol_first);
                t = make_float4(l, t.x, t.y, t.z);
            } else if (cx_of(i) == -1) {    // source x + 1
                float r = __shfl_down_sync(0xffffffffu, t.x, 1);
                if (right_ld) r = St::ld1r(rp + (xq == nxq - 1 ? 0 : 4 * xq + 4), pol_first);
                t = make_float4(t.y, t.z, t.w, r);
            }
            v[i] = t;
        }
    }

    const BoxDyn dyn = ldcg_dyn(P.box_dyn + bi);
    const bool wallrow = B.walls && (y == 0 || y == ny - 1);
    if (!FIRST && B.walls && (y == 1 || y == ny - 2)) {
        // link bounce-back on a moving wall (Eq. fb with u_b = u_w)
        const int cyw = (y == 1) ? 1 : -1;
        const float* uw = (y == 1) ? B.uw_lo : B.uw_hi;
#pragma unroll
        for (int i = 1; i < Q; ++i) {
            if (cy_of(i) != cyw) continue;
            const float ubc = cx_of(i) * uw[0] + cy_of(i) * uw[1] + cz_of(i) * uw[2];
            float add = 6.0f * w_of(i) * B.rho0f * ubc;
            if (St::SCALED) add *= B.scale;
            const float4 o = St::ld4r(A + (opp_of(i) * N + own), pol_first);
            v[i] = make_float4(o.x + add, o.y + add, o.z + add, o.w + add);
        }
    }
    ColliderT<St::SCALED, St::GHOST> C;
    C.init(B.omega, B.rho0f, dyn.g[0], dyn.g[1], dyn.g[2], dyn.eps, B.scale, B.inv_scale);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float f[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i] = comp(v[i], k);
        C.apply(f);
#pragma unroll
        for (int i = 0; i < Q; ++i) set_comp(v[i], k, f[i]);
    }
    // nodes of this quad that the boundary kernel writes
    unsigned skip = 0;
    for (int j = 0; j < B.pcnt; ++j) {
        const NeedHdr h = ldcg_hdr(P.need_hdr + B.pbeg + j);
        int dz = z - h.ow[2];
        if (dz < 0) dz += nz;
        int dy = y - h.ow[1];
        if (dy < 0) dy += ny;
        int dx = 4 * xq - h.ow[0];
        if (dx < 0) dx += nx;
        // within two nodes of the cube, cyclically (a cache hint only)
        if (dz >= h.S || dy >= h.S) continue;
        if (dx >= h.S && dx + 3 < nx) continue;
        const uint64_t w = __ldcg(P.need + (size_t)(B.pbeg + j) * (MAXS * MAXS) + dz * h.S + dy);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int mx = dx + k < nx ? dx + k : dx + k - nx;
            if (mx < h.S && ((w >> mx) & 1ull)) skip |= 1u << k;
        }
    }
    // the solid wall planes keep the zeros they were created with
    if (valid && !wallrow) {
        T* dp = D + own;
        const unsigned long long pol = pol_first;
        if (!skip) {
#pragma unroll
            for (int i = 0; i < Q; ++i) St::st4r(dp + i * N, v[i], pol);
        } else {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if ((skip >> k) & 1u) continue;
#pragma unroll
                for (int i = 0; i < Q; ++i) St::st1r(dp + (i * N + k), comp(v[i], k), pol);
            }
        }
    }
}

}  // namespace lbsph
