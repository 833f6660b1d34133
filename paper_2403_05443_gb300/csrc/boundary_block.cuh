// Boundary block (see boundary_kernel.cu for the method), shared by the
// boundary kernel and the persistent step kernel.
#pragma once

#include <type_traits>

#include "lattice_common.cuh"

namespace lbsph {

// round(f * 2^46) toward zero, from the IEEE 754 fields with integer
// instructions (exact for |f| >= 2^-23, off by less than 2^-46 below; 64-bit
// float-to-integer conversions run at the slow FP64 rate on this part)
__device__ __forceinline__ long long fixq(float f)
{
    const unsigned u = __float_as_uint(f);
    const int ex = (int)((u >> 23) & 0xffu);
    const long long m = (long long)((u & 0x7fffffu) | 0x800000u);
    const int sh = ex - 104;                    // f * 2^46 = m * 2^(ex - 127 - 23 + 46)
    long long v;
    if (ex == 0 || sh <= -24) v = 0;            // zero, subnormal, or |f| < 2^-46
    else if (sh >= 0) v = m << (sh > 38 ? 38 : sh);   // saturates for |f| >= 2^16 (no deviation is)
    else v = m >> (-sh);
    return (u >> 31) ? -v : v;
}

__device__ __forceinline__ long long warp_sum(long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += (long long)__shfl_xor_sync(0xffffffffu, (unsigned long long)v, o);
    return v;
}

// block c (of P.gx) of particle p; BBLOCK threads
template <class St, bool FIRST>
__device__ __forceinline__ void boundary_block(const BndParams& P, int p, int c)
{
    using T = typename St::T;
    constexpr int NW = BBLOCK / 32;
    const int gx = P.gx;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int cap = P.list_cap, smax = P.smax;

    extern __shared__ uint64_t s_bits[];            // ring slots 0 and 1 (smax*smax rows each), then the node list
    unsigned* s_list = reinterpret_cast<unsigned*>(s_bits + 2 * smax * smax);
    __shared__ PartK K;
    __shared__ long long s_red[NW][ACC_COV];        // per-warp link sums
    __shared__ long long s_rare[NACC - ACC_COV];    // covered / uncovered nodes (rare: shared atomics)
    __shared__ int s_wsum[NW];
    __shared__ PartK s_pk[MAXNB];                   // partners' snapshots (particles whose cubes reach this one's)
    __shared__ NeedHdr s_ph[MAXNB];

    // ---- one round of independent loads
    const BoxDyn dyn = ldcg_dyn(P.pdyn + p);
    const int rrow = c + gx * tid;                  // this thread's cube row
    uint64_t need = rrow < smax * smax ? __ldcg(P.need + (size_t)p * (MAXS * MAXS) + rrow) : 0ull;
    {
        ldcg_copy(&K, P.pk + p, tid, BBLOCK);
        if (tid < NACC - ACC_COV) s_rare[tid] = 0;
        const uint64_t* r0 = P.rows + (size_t)p * 2 * (MAXS * MAXS);
        const int n = smax * smax;
#pragma unroll 4
        for (int r = tid; r < n; r += BBLOCK) {
            s_bits[r] = __ldcg(r0 + r);
            s_bits[n + r] = __ldcg(r0 + MAXS * MAXS + r);
        }
    }
    __syncthreads();

    // partners: their snapshots and redo-mask cubes (the critical blocks of a
    // partner run only after this block: the cluster's items come first)
    const int nnb = min(K.nnb, MAXNB);
    if (nnb > 0) {
        for (int j = 0; j < nnb; ++j) ldcg_copy(&s_pk[j], P.pk + K.nb[j], tid, BBLOCK);
        if (tid < nnb) s_ph[tid] = ldcg_hdr(P.need_hdr + K.nb[tid]);
        __syncthreads();
    }
    const int S = K.S;
    const uint64_t* slot1 = P.rows + ((size_t)p * 2 + 1) * (MAXS * MAXS);
    const uint64_t* s_new = s_bits + (K.rows_new == slot1 ? smax * smax : 0);
    const uint64_t* s_old = s_bits + (K.rows_old == slot1 ? smax * smax : 0);
    const int nx = K.nx, ny = K.ny, nz = K.nz;
    const bool walls = K.walls != 0;
    int dsh[3];                                     // o_new - o_old: old-local = new-local + dsh
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int L = k == 0 ? nx : (k == 1 ? ny : nz);
        int v = K.ow_new[k] - K.ow_old[k];
        if (v > L / 2) v -= L;
        if (v < -L / 2) v += L;
        dsh[k] = FIRST ? 0 : v;
    }
    auto bit_new = [&](int ax, int ay, int az) -> bool {
        if (ax < 0 || ax >= S || ay < 0 || ay >= S || az < 0 || az >= S) return false;
        return (s_new[az * S + ay] >> ax) & 1ull;
    };
    auto bit_old = [&](int ax, int ay, int az) -> bool {
        ax += dsh[0]; ay += dsh[1]; az += dsh[2];
        if (ax < 0 || ax >= S || ay < 0 || ay >= S || az < 0 || az >= S) return false;
        return (s_old[az * S + ay] >> ax) & 1ull;
    };
    // a node (X, Y, Z in the box) in partner j's new or old cube: its local coordinates
    auto ploc = [&](int j, bool nw, int X_, int Y_, int Z_, int& lx, int& ly, int& lz) -> bool {
        const int* ow = nw ? s_pk[j].ow_new : s_pk[j].ow_old;
        lx = X_ - ow[0]; if (lx < 0) lx += nx;
        ly = Y_ - ow[1]; if (ly < 0) ly += ny;
        lz = Z_ - ow[2]; if (lz < 0) lz += nz;
        const int Sq = s_pk[j].S;
        return lx < Sq && ly < Sq && lz < Sq;
    };
    auto pbit = [&](int j, bool nw, int X_, int Y_, int Z_) -> bool {
        int lx, ly, lz;
        if (!ploc(j, nw, X_, Y_, Z_, lx, ly, lz)) return false;
        const uint64_t* rw = nw ? s_pk[j].rows_new : s_pk[j].rows_old;
        return (__ldcg(rw + lz * s_pk[j].S + ly) >> lx) & 1ull;
    };
    // integer sums that belong to partner j (global atomics: rare)
    auto padd = [&](int j, int e, long long v) {
        if (v != 0) atomicAdd(reinterpret_cast<unsigned long long*>(P.acc + (size_t)K.nb[j] * NACC + e),
                              static_cast<unsigned long long>(v));
    };
    // ---- this block's rows: the nodes to redo, compacted into shared memory
    {
        if (rrow >= S * S) need = 0;
        // block-wide exclusive scan of the row counts
        const int cnt = __popcll(need);
        int inc = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, inc, o);
            if (lane >= o) inc += v;
        }
        if (lane == 31) s_wsum[warp] = inc;
        __syncthreads();
        int base = inc - cnt;
        for (int w = 0; w < warp; ++w) base += s_wsum[w];
        const int my = rrow % S, mz = rrow / S;
        for (int k = 0; need; ++k) {
            const int mx = __ffsll((long long)need) - 1;
            need &= need - 1;
            if (base + k < cap) s_list[base + k] = (unsigned)((mz << 16) | (my << 8) | mx);
        }
    }
    __syncthreads();
    int total = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) total += s_wsum[w];
    if (tid == 0 && total > cap) atomicOr(P.status, ST_CAPACITY);
    const int count = min(total, cap);

    const long long N = K.N;
    const T* A = reinterpret_cast<const T*>(P.src) + K.off;
    const float inv = K.inv_scale, rho0 = K.rho0f, scale = K.scale;
    const unsigned long long pol = l2_evict_normal();
    T* D = reinterpret_cast<T*>(P.dst) + K.off;

    // ---- this block's nodes, two warps per node: the even warp of a pair takes
    // the rest population and the directions 1..10, the odd warp 11..18 (each
    // warp's path stays uniform and each thread's dependent chain is about half
    // as long); the node's moments (and, for the ghost-mode collision, its second
    // moments) are added up through shared memory, in one order on both warps, so
    // that both take identical decisions and values.  Per-thread link sums.
    long long aF[3] = {0, 0, 0}, aT[3] = {0, 0, 0};
    auto rare_add = [&](int j, long long v) {
        if (v != 0) atomicAdd(reinterpret_cast<unsigned long long*>(&s_rare[j - ACC_COV]), (unsigned long long)v);
    };
    constexpr int NX = St::GHOST ? 10 : 4;         // exchanged partial moments per node
    __shared__ float s_xch[NW / 2][2][NX][32];
    const int wpair = warp >> 1;
    const int rounds = (count + (BBLOCK / 2) - 1) / (BBLOCK / 2);

    auto node_round = [&](auto Hc, int rnd) {
        constexpr int H = decltype(Hc)::value;
        auto mine = [](int i) { return H == 0 ? i <= 10 : i >= 11; };
        const int e = rnd * (BBLOCK / 2) + wpair * 32 + lane;
        bool act = e < count;
        int mx = 0, my = 0, mz = 0, X = 0, Y = 0, Z = 0;
        long long own = 0;
        bool wallrow = false, sol_new = false, sol_old = false;
        int pn = -1, po = -1;
        if (act) {
            const unsigned code = s_list[e];
            mx = code & 0xff; my = (code >> 8) & 0xff; mz = (code >> 16) & 0xff;
            X = wrapd(K.ow_new[0] + mx, nx); Y = wrapd(K.ow_new[1] + my, ny); Z = wrapd(K.ow_new[2] + mz, nz);
            own = ((long long)Z * ny + Y) * nx + X;
            wallrow = walls && (Y == 0 || Y == ny - 1);
            sol_new = bit_new(mx, my, mz);
            sol_old = !FIRST && bit_old(mx, my, mz);
            // partners: a node in the redo masks of two particles is done once, by
            // the one of lower index; a partner may hold it now (pn) or before (po)
            if (nnb > 0) {
                bool dup = false;
                for (int j = 0; j < nnb; ++j) {
                    if (K.nb[j] < p) {
                        const NeedHdr& h = s_ph[j];
                        int lx = X - h.ow[0], ly = Y - h.ow[1], lz = Z - h.ow[2];
                        if (lx < 0) lx += nx;
                        if (ly < 0) ly += ny;
                        if (lz < 0) lz += nz;
                        if (lx < h.S && ly < h.S && lz < h.S &&
                            ((__ldcg(P.need + (size_t)K.nb[j] * (MAXS * MAXS) + lz * h.S + ly) >> lx) & 1ull))
                            dup = true;
                    }
                    if (pbit(j, true, X, Y, Z)) pn = j;
                    if (!FIRST && pbit(j, false, X, Y, Z)) po = j;
                }
                if (dup) act = false;
            }
        }
        const bool solN = sol_new || pn >= 0, solO = sol_old || po >= 0;
        // 0 nothing, 1 solid before and after (untouched), 2 uncovered, 3 first
        // collision, 4 fluid before (pull with bounce-back; covered if solid now)
        const int kind = !act ? 0 : ((wallrow || (solN && (solO || FIRST))) ? 1 : (solO ? 2 : (FIRST ? 3 : 4)));
        float f[Q];
#pragma unroll
        for (int i = 0; i < Q; ++i) f[i] = 0.0f;
        if (kind == 2) {
            // uncovered: f = f_eq(rho0, U + Omega x r) with r = x - x_c(t+1) of the
            // body that held it, whose sums get its cube coordinates m
            int m0 = mx, m1 = my, m2 = mz;
            const PartK& Ko = sol_old ? K : s_pk[po];
            if (!sol_old) ploc(po, true, X, Y, Z, m0, m1, m2);
            const float rx = Ko.ro_new[0] + m0, ry = Ko.ro_new[1] + m1, rz = Ko.ro_new[2] + m2;
            const float ux = Ko.U[0] + (Ko.W[1] * rz - Ko.W[2] * ry);
            const float uy = Ko.U[1] + (Ko.W[2] * rx - Ko.W[0] * rz);
            const float uz = Ko.U[2] + (Ko.W[0] * ry - Ko.W[1] * rx);
            const float uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if (!mine(i)) continue;
                const float cu = cx_of(i) * ux + cy_of(i) * uy + cz_of(i) * uz;
                f[i] = w_of(i) * rho0 * (3.0f * cu + 4.5f * cu * cu - 1.5f * uu);
            }
            if (H == 0) {
                const long long uv[10] = {1, m0, m1, m2, m0 * m0, m0 * m1, m0 * m2, m1 * m1, m1 * m2, m2 * m2};
                for (int e2 = 0; e2 < 10; ++e2) {
                    if (sol_old) rare_add(ACC_UNC + e2, uv[e2]);
                    else padd(po, ACC_UNC + e2, uv[e2]);
                }
            }
        } else if (kind == 3) {
            // first collision: the node's initial distributions, no streaming
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if (mine(i)) f[i] = St::ld1(A + ((long long)i * N + own), inv, pol);
        } else if (kind == 4) {
            // fluid at t-1: decide every source first, then issue the loads together
            unsigned bb = 0, wl = 0, pb = 0;        // own, wall and partner bounce-back
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                if (!mine(i)) continue;
                const int Ys = Y - cy_of(i);
                if (walls && (Ys == 0 || Ys == ny - 1)) wl |= 1u << i;
                else if (bit_old(mx - cx_of(i), my - cy_of(i), mz - cz_of(i))) bb |= 1u << i;
            }
            if (nnb > 0) {
                for (int i = 1; i < Q; ++i) {
                    if (!mine(i) || (((bb | wl) >> i) & 1u)) continue;
                    const int Xs = wrapd(X - cx_of(i), nx), Ys = wrapd(Y - cy_of(i), ny), Zs = wrapd(Z - cz_of(i), nz);
                    for (int j = 0; j < nnb; ++j)
                        if (pbit(j, false, Xs, Ys, Zs)) pb |= 1u << i;
                }
                bb |= pb;
            }
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if (!mine(i)) continue;
                const bool back = ((bb | wl) >> i) & 1u;
                const long long src = back ? (long long)opp_of(i) * N + own
                                           : (long long)i * N + ((long long)wrapd(Z - cz_of(i), nz) * ny + wrapd(Y - cy_of(i), ny)) * nx +
                                                 wrapd(X - cx_of(i), nx);
                f[i] = St::ld1(A + src, inv, pol);
            }
            // mid-link bounce-back terms: + 6 w_i rho0 (u_b . c_i) (Eq. fb, Eq. ub, Eq. ubsquirmer)
            const float ex[3] = {K.e_old[0], K.e_old[1], K.e_old[2]};
#pragma unroll
            for (int i = 1; i < Q; ++i) {
                if (!mine(i) || !(((bb | wl) >> i) & 1u)) continue;
                float ubc;
                if ((wl >> i) & 1u) {
                    const float* uw = (Y - cy_of(i) == 0) ? K.uw_lo : K.uw_hi;
                    ubc = cx_of(i) * uw[0] + cy_of(i) * uw[1] + cz_of(i) * uw[2];
                } else if ((pb >> i) & 1u) {
                    // a partner's surface: its velocity at r_b = x - c_i/2 - x_c(t) of that body
                    const int Xs = wrapd(X - cx_of(i), nx), Ys = wrapd(Y - cy_of(i), ny), Zs = wrapd(Z - cz_of(i), nz);
                    int j = 0;
                    while (j < nnb - 1 && !pbit(j, false, Xs, Ys, Zs)) ++j;
                    const PartK& Kq = s_pk[j];
                    int l0, l1, l2;
                    ploc(j, false, X, Y, Z, l0, l1, l2);
                    const float px = Kq.ro_old[0] + (float)l0 - 0.5f * cx_of(i);
                    const float py = Kq.ro_old[1] + (float)l1 - 0.5f * cy_of(i);
                    const float pz = Kq.ro_old[2] + (float)l2 - 0.5f * cz_of(i);
                    float ux = Kq.U[0] + (Kq.W[1] * pz - Kq.W[2] * py);
                    float uy = Kq.U[1] + (Kq.W[2] * px - Kq.W[0] * pz);
                    float uz = Kq.U[2] + (Kq.W[0] * py - Kq.W[1] * px);
                    if (Kq.squirmer) {
                        float qx, qy, qz;
                        squirmer_slip(Kq.e_old, Kq.a, Kq.eps2, Kq.B1, Kq.B2, px, py, pz, qx, qy, qz);
                        ux += qx; uy += qy; uz += qz;
                    }
                    ubc = cx_of(i) * ux + cy_of(i) * uy + cz_of(i) * uz;
                } else {
                    // r_b = x - c_i/2 - x_c(t-1) = ro_old + dsh + m - c_i/2
                    const float px = K.ro_old[0] + (float)(dsh[0] + mx) - 0.5f * cx_of(i);
                    const float py = K.ro_old[1] + (float)(dsh[1] + my) - 0.5f * cy_of(i);
                    const float pz = K.ro_old[2] + (float)(dsh[2] + mz) - 0.5f * cz_of(i);
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
        }
        // ---- the node's moments: this warp's part and the partner warp's
        float tot[NX];
        {
            float part[NX];
#pragma unroll
            for (int k = 0; k < NX; ++k) part[k] = 0.0f;
#pragma unroll
            for (int i = 0; i < Q; ++i) {
                if (!mine(i)) continue;
                const int cx = cx_of(i), cy = cy_of(i), cz = cz_of(i);
                part[0] += f[i];
                if (cx) part[1] += cx * f[i];
                if (cy) part[2] += cy * f[i];
                if (cz) part[3] += cz * f[i];
                if constexpr (NX > 4) {
                    if (cx) part[4] += f[i];
                    if (cy) part[5] += f[i];
                    if (cz) part[6] += f[i];
                    if (cx * cy) part[7] += (cx * cy) * f[i];
                    if (cx * cz) part[8] += (cx * cz) * f[i];
                    if (cy * cz) part[9] += (cy * cz) * f[i];
                }
            }
#pragma unroll
            for (int k = 0; k < NX; ++k) s_xch[wpair][H][k][lane] = part[k];
            asm volatile("bar.sync %0, %1;" ::"r"(1 + wpair), "r"(64) : "memory");
#pragma unroll
            for (int k = 0; k < NX; ++k) tot[k] = s_xch[wpair][0][k][lane] + s_xch[wpair][1][k][lane];
            asm volatile("bar.sync %0, %1;" ::"r"(1 + wpair), "r"(64) : "memory");
        }
        bool write = kind == 2 || kind == 3 || (kind == 4 && !solN);
        if (kind == 4 && solN && H == 0) {
            // covered: mass and momentum go to the next solve of the body that
            // holds the node now
            const long long Jx = fixq(tot[1]), Jy = fixq(tot[2]), Jz = fixq(tot[3]);
            int m0 = mx, m1 = my, m2 = mz;
            if (!sol_new) ploc(pn, true, X, Y, Z, m0, m1, m2);
            const long long cv[8] = {1, fixq(tot[0]), Jx, Jy, Jz, m1 * Jz - m2 * Jy, m2 * Jx - m0 * Jz,
                                     m0 * Jy - m1 * Jx};
            for (int e2 = 0; e2 < 8; ++e2) {
                if (sol_new) rare_add(ACC_COV + e2, cv[e2]);
                else padd(pn, ACC_COV + e2, cv[e2]);
            }
        }
        if (write) {
            collide_half<St::GHOST, H>(f, tot, K.omega, rho0, dyn.g[0], dyn.g[1], dyn.g[2], dyn.eps);
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if (mine(i)) St::st1(D + (long long)i * N + own, f[i], scale, pol);
            // momentum-exchange sums of the new links (x, b), with f*(t)
            long long fx = 0, fy = 0, fz = 0;
            bool any = false;
#pragma unroll
            for (int b = 1; b < Q; ++b) {
                if (!mine(b) || !bit_new(mx + cx_of(b), my + cy_of(b), mz + cz_of(b))) continue;
                const long long d = fixq(f[b]);
                any = true;
                if (cx_of(b) == 1) fx += d; else if (cx_of(b) == -1) fx -= d;
                if (cy_of(b) == 1) fy += d; else if (cy_of(b) == -1) fy -= d;
                if (cz_of(b) == 1) fz += d; else if (cz_of(b) == -1) fz -= d;
            }
            if (any) {
                aF[0] += fx; aF[1] += fy; aF[2] += fz;
                aT[0] += my * fz - mz * fy;
                aT[1] += mz * fx - mx * fz;
                aT[2] += mx * fy - my * fx;
            }
            // links to partners' surfaces: their sums, about their cube origins
            if (nnb > 0) {
                for (int b = 1; b < Q; ++b) {
                    if (!mine(b)) continue;
                    const int Xb = wrapd(X + cx_of(b), nx), Yb = wrapd(Y + cy_of(b), ny), Zb = wrapd(Z + cz_of(b), nz);
                    for (int j = 0; j < nnb; ++j) {
                        if (!pbit(j, true, Xb, Yb, Zb)) continue;
                        int l0, l1, l2;
                        ploc(j, true, X, Y, Z, l0, l1, l2);
                        const long long d = fixq(f[b]);
                        const long long gx_ = cx_of(b) * d, gy_ = cy_of(b) * d, gz_ = cz_of(b) * d;
                        padd(j, ACC_F, gx_); padd(j, ACC_F + 1, gy_); padd(j, ACC_F + 2, gz_);
                        padd(j, ACC_T, l1 * gz_ - l2 * gy_);
                        padd(j, ACC_T + 1, l2 * gx_ - l0 * gz_);
                        padd(j, ACC_T + 2, l0 * gy_ - l1 * gx_);
                    }
                }
            }
        } else if (act && solN && !wallrow) {
            // solid now: zero it (never read as a source)
#pragma unroll
            for (int i = 0; i < Q; ++i)
                if (mine(i)) St::st1(D + (long long)i * N + own, 0.0f, scale, pol);
        }
    };
    for (int rnd = 0; rnd < rounds; ++rnd) {
        if (warp & 1) node_round(std::integral_constant<int, 1>{}, rnd);
        else node_round(std::integral_constant<int, 0>{}, rnd);
    }

    // ---- per-warp link sums into shared memory, then one atomic per nonzero sum
    if (__any_sync(0xffffffffu, (aF[0] | aF[1] | aF[2] | aT[0] | aT[1] | aT[2]) != 0)) {
#pragma unroll
        for (int k = 0; k < 3; ++k) { aF[k] = warp_sum(aF[k]); aT[k] = warp_sum(aT[k]); }
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k) { s_red[warp][ACC_F + k] = aF[k]; s_red[warp][ACC_T + k] = aT[k]; }
    }
    __syncthreads();
    if (tid < NACC) {
        long long v = 0;
        if (tid < ACC_COV) {
#pragma unroll
            for (int w = 0; w < NW; ++w) v += s_red[w][tid];
        } else {
            v = s_rare[tid - ACC_COV];
        }
        if (v != 0) atomicAdd(reinterpret_cast<unsigned long long*>(P.acc + (size_t)p * NACC + tid), static_cast<unsigned long long>(v));
    }
}

}  // namespace lbsph
