// Critical and auxiliary particle blocks (see particle_kernel.cu for the
// method), shared by the particle kernels and the persistent step kernel.
#pragma once

#include "lattice_common.cuh"

namespace lbsph {

// ---- exact FP64 inside test (no contraction: explicit round-to-nearest ops)
__device__ inline void canon_rotate(const double q[4], const double s[3], double o[3])
{
    const double a = __dsub_rn(__dmul_rn(2.0, __dmul_rn(q[0], q[0])), 1.0);
    const double qs = __dadd_rn(__dadd_rn(__dmul_rn(q[1], s[0]), __dmul_rn(q[2], s[1])), __dmul_rn(q[3], s[2]));
    const double cx = __dsub_rn(__dmul_rn(q[2], s[2]), __dmul_rn(q[3], s[1]));
    const double cy = __dsub_rn(__dmul_rn(q[3], s[0]), __dmul_rn(q[1], s[2]));
    const double cz = __dsub_rn(__dmul_rn(q[1], s[1]), __dmul_rn(q[2], s[0]));
    const double tqs = __dmul_rn(2.0, qs), tq0 = __dmul_rn(2.0, q[0]);
    o[0] = __dadd_rn(__dadd_rn(__dmul_rn(a, s[0]), __dmul_rn(tqs, q[1])), __dmul_rn(tq0, cx));
    o[1] = __dadd_rn(__dadd_rn(__dmul_rn(a, s[1]), __dmul_rn(tqs, q[2])), __dmul_rn(tq0, cy));
    o[2] = __dadd_rn(__dadd_rn(__dmul_rn(a, s[2]), __dmul_rn(tqs, q[3])), __dmul_rn(tq0, cz));
}

__device__ inline void canon_shape(const double semi[3], const double q[4], double A[9], double e[3][3])
{
    double inv[3];
    for (int m = 0; m < 3; ++m) {
        double u[3] = {0.0, 0.0, 0.0};
        u[m] = 1.0;
        canon_rotate(q, u, e[m]);
        inv[m] = __ddiv_rn(1.0, __dmul_rn(semi[m], semi[m]));
    }
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k)
            A[j * 3 + k] = __dadd_rn(__dadd_rn(__dmul_rn(__dmul_rn(e[0][j], e[0][k]), inv[0]),
                                               __dmul_rn(__dmul_rn(e[1][j], e[1][k]), inv[1])),
                                     __dmul_rn(__dmul_rn(e[2][j], e[2][k]), inv[2]));
}

__device__ __forceinline__ double canon_minimage(double d, int L, bool periodic)
{
    if (!periodic) return d;
    const double Ld = (double)L;
    // |d| <= L/2 - 1 puts d/L + 0.5 inside (0, 1) whatever the rounding, so the
    // shift below is exactly zero and d comes back unchanged
    if (fabs(d) <= 0.5 * Ld - 1.0) return d;
    return __dsub_rn(d, __dmul_rn(Ld, floor(__dadd_rn(__ddiv_rn(d, Ld), 0.5))));
}

__device__ inline double canon_value(const double A[9], const double xc[3], int X, int Y, int Z, int nx, int ny,
                              int nz, bool py)
{
    double d[3];
    d[0] = canon_minimage(__dsub_rn((double)X, xc[0]), nx, true);
    d[1] = canon_minimage(__dsub_rn((double)Y, xc[1]), ny, py);
    d[2] = canon_minimage(__dsub_rn((double)Z, xc[2]), nz, true);
    double Ad[3];
    for (int j = 0; j < 3; ++j)
        Ad[j] = __dadd_rn(__dadd_rn(__dmul_rn(A[j * 3 + 0], d[0]), __dmul_rn(A[j * 3 + 1], d[1])),
                          __dmul_rn(A[j * 3 + 2], d[2]));
    return __dadd_rn(__dadd_rn(__dmul_rn(d[0], Ad[0]), __dmul_rn(d[1], Ad[1])), __dmul_rn(d[2], Ad[2]));
}

__device__ __forceinline__ int wrapi(int a, int L) { a %= L; return a < 0 ? a + L : a; }

__device__ __forceinline__ unsigned long long abs_bits(double x)
{
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

// Minimum image of a displacement along a periodic axis of length L.
__device__ __forceinline__ double min_image_d(double d, int L, bool periodic)
{
    return periodic ? d - (double)L * floor(d / (double)L + 0.5) : d;
}

// Centre-to-surface distance of an ellipsoid along the unit vector n:
// (n^T A n)^(-1/2), A = R diag(1/s^2) R^T (Eq. ellipsoidsurface), i.e. the body
// components of n, (R^T n)_m, weighted by 1/s_m^2.
__device__ __forceinline__ double radius_along(const double* q, const double* semi, const double n[3])
{
    const double q0 = q[0], q1 = q[1], q2 = q[2], q3 = q[3];
    const double R[3][3] = {{1.0 - 2.0 * (q2 * q2 + q3 * q3), 2.0 * (q1 * q2 - q0 * q3), 2.0 * (q1 * q3 + q0 * q2)},
                            {2.0 * (q1 * q2 + q0 * q3), 1.0 - 2.0 * (q1 * q1 + q3 * q3), 2.0 * (q2 * q3 - q0 * q1)},
                            {2.0 * (q1 * q3 - q0 * q2), 2.0 * (q2 * q3 + q0 * q1), 1.0 - 2.0 * (q1 * q1 + q2 * q2)}};
    double v = 0.0;
#pragma unroll
    for (int m = 0; m < 3; ++m) {
        const double b = R[0][m] * n[0] + R[1][m] * n[1] + R[2][m] * n[2];
        v += b * b / (semi[m] * semi[m]);
    }
    return 1.0 / sqrt(v);
}

// Lubrication correction on body `lo` from body `hi` (the opposite acts on hi):
// with d the minimum image of x_hi - x_lo, n = d/|d|, radii R = (n^T A n)^(-1/2)
// of both bodies along n and the gap h = |d| - R_lo - R_hi along the line of
// centres, below the cut-off h_c the squeeze force of two spheres of those radii
// that the lattice does not resolve, -6 pi mu R_e^2 (1/h - 1/h_c) (n.(U_lo -
// U_hi)) n, R_e = R_lo R_hi / (R_lo + R_hi), h >= 0.1, the coefficient at most
// the reduced mass (an explicit update stays stable).  Velocities and
// orientations of time t; ring entries x[3], U[3], q[4].
constexpr double LUB_H_MIN = 0.1;
__device__ __forceinline__ void lubrication_pair(const double* rlo, const double* semi_lo, double M_lo,
                                                 const double* rhi, const double* semi_hi, double M_hi,
                                                 const int L[3], const bool per[3], double mu, double h_cut,
                                                 double f[3])
{
    double d[3], n[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) d[k] = min_image_d(rhi[k] - rlo[k], L[k], per[k]);
    const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
#pragma unroll
    for (int k = 0; k < 3; ++k) n[k] = d[k] / r;
    const double Rl = radius_along(rlo + 6, semi_lo, n), Rh = radius_along(rhi + 6, semi_hi, n);
    const double h = r - Rl - Rh;
    f[0] = f[1] = f[2] = 0.0;
    if (!(h < h_cut)) return;
    const double hh = h > LUB_H_MIN ? h : LUB_H_MIN;
    const double Re = Rl * Rh / (Rl + Rh);
    double k = 6.0 * M_PI * mu * Re * Re * (1.0 / hh - 1.0 / h_cut);
    const double kmax = M_lo * M_hi / (M_lo + M_hi);
    if (k > kmax) k = kmax;
    const double vn = n[0] * (rlo[3] - rhi[3]) + n[1] * (rlo[4] - rhi[4]) + n[2] * (rlo[5] - rhi[5]);
#pragma unroll
    for (int c = 0; c < 3; ++c) f[c] = -k * vn * n[c];
}

// Component jq of q' = qt(Wm) q (Eq. qnplus0-1, rotation by the mean angular
// velocity Wm over one step), for a warp whose lanes all hold Wm and q.
__device__ __forceinline__ double quat_step_component(const double Wm[3], const double* q, int jq)
{
    const double th2 = Wm[0] * Wm[0] + Wm[1] * Wm[1] + Wm[2] * Wm[2];
    double qt[4];
    if (th2 < 1e-4) {
        // cos(th/2) and sin(th/2)/th by their Taylor series (th < 0.01: error < 1e-20)
        const double x2 = 0.25 * th2;
        const double c = 1.0 - x2 * (0.5 - x2 * (1.0 / 24.0 - x2 * (1.0 / 720.0)));
        const double sc = 0.5 * (1.0 - x2 * (1.0 / 6.0 - x2 * (1.0 / 120.0 - x2 * (1.0 / 5040.0))));
        qt[0] = c; qt[1] = sc * Wm[0]; qt[2] = sc * Wm[1]; qt[3] = sc * Wm[2];
    } else {
        const double th = sqrt(th2);
        double sn, cs;
        sincos(0.5 * th, &sn, &cs);
        sn /= th;
        qt[0] = cs; qt[1] = sn * Wm[0]; qt[2] = sn * Wm[1]; qt[3] = sn * Wm[2];
    }
    // sum_m +-qt_m q_(m xor jq), the sign applied by flipping the sign bit
    constexpr unsigned NEG = (1u << 1) | (1u << 2) | (1u << 3) | (1u << 7) | (1u << 9) | (1u << 14);
    double qn = 0.0;
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const unsigned long long sgn = (unsigned long long)((NEG >> (jq * 4 + m)) & 1u) << 63;
        const double qs = __longlong_as_double(__double_as_longlong(qt[m]) ^ (long long)sgn);
        qn = fma(qs, q[m ^ jq], qn);
    }
    return qn;
}

// The same component of q' = qt(Wm) q written as q + (qt - 1) q, for the
// small rotations of a step (|Wm| < 0.01): the increment's entries
// (cos(th/2) - 1, sin(th/2)/th Wm) are formed in FP32 from their Taylor series
// (each is of the order of the angle turned or its square, so their FP32
// rounding lies far below the FP64 rounding of q) and applied in FP64: four
// FP64 multiply-adds instead of the whole step in FP64.  Larger rotations take
// quat_step_component.  Lane k < 3 of the warp holds Wm[k] in wk; every lane
// gets the component jq.
__device__ __forceinline__ double quat_step_component_small(float wk, const double* q, int jq)
{
    const float w0 = __shfl_sync(0xffffffffu, wk, 0), w1 = __shfl_sync(0xffffffffu, wk, 1),
                w2 = __shfl_sync(0xffffffffu, wk, 2);
    const float x2 = 0.25f * (w0 * w0 + w1 * w1 + w2 * w2);
    const float cm1 = -x2 * (0.5f - x2 * (1.0f / 24.0f - x2 * (1.0f / 720.0f)));
    const float sc = 0.5f * (1.0f - x2 * (1.0f / 6.0f - x2 * (1.0f / 120.0f - x2 * (1.0f / 5040.0f))));
    const float dt[4] = {cm1, sc * w0, sc * w1, sc * w2};
    constexpr unsigned NEG = (1u << 1) | (1u << 2) | (1u << 3) | (1u << 7) | (1u << 9) | (1u << 14);
    double qn = q[jq];
#pragma unroll
    for (int m = 0; m < 4; ++m) {
        const float ds = ((NEG >> (jq * 4 + m)) & 1u) ? -dt[m] : dt[m];
        qn = fma((double)ds, q[m ^ jq], qn);
    }
    return qn;
}

// Solution of the 6x6 system A x = b by Gauss-Jordan elimination with partial
// pivoting, one warp: lane j < 6 holds column j of A, lane 6 holds b (col[i] =
// row i); on return lane 6 holds x.  Returns false if a pivot vanishes.
__device__ __forceinline__ bool gj_solve6_warp(double col[6], int lane)
{
    bool ok = true;
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        int piv = k;
        if (lane == k) {
            unsigned long long best = abs_bits(col[k]);
#pragma unroll
            for (int i = k + 1; i < 6; ++i) {
                const unsigned long long bi = abs_bits(col[i]);
                if (bi > best) { best = bi; piv = i; }
            }
        }
        piv = __shfl_sync(0xffffffffu, piv, k);
        double rowk = col[k], rowp = col[k];
#pragma unroll
        for (int i = k + 1; i < 6; ++i)
            if (i == piv) rowp = col[i];
#pragma unroll
        for (int i = k + 1; i < 6; ++i)
            if (i == piv) col[i] = rowk;
        col[k] = rowp;
        const double pv = __shfl_sync(0xffffffffu, col[k], k);
        ok = ok && (pv != 0.0);
        col[k] *= 1.0 / pv;
#pragma unroll
        for (int i = 0; i < 6; ++i) {
            if (i == k) continue;
            const double fi = __shfl_sync(0xffffffffu, col[i], k);
            col[i] -= fi * col[k];
        }
    }
    return ok;
}

__device__ __forceinline__ long long warp_sum_ll(long long v)
{
    for (int o = 16; o > 0; o >>= 1) v += (long long)__shfl_xor_sync(0xffffffffu, (unsigned long long)v, o);
    return v;
}

// ---------------------------------------------------------------------------
// The exact inside-test matrix A = sum_m e_m e_m^T / semi_m^2 of canon_shape,
// spread over lanes 0..8 of one warp (same operations, same order per entry).
__device__ inline void canon_shape_warp(const double inv[3], const double q[4], double* s_E, double* s_A, int lane)
{
    if (lane < 3) {
        const double u[3] = {lane == 0 ? 1.0 : 0.0, lane == 1 ? 1.0 : 0.0, lane == 2 ? 1.0 : 0.0};
        double o[3];
        canon_rotate(q, u, o);
        s_E[lane * 3 + 0] = o[0]; s_E[lane * 3 + 1] = o[1]; s_E[lane * 3 + 2] = o[2];
    }
    __syncwarp();
    if (lane < 9) {
        const int j = lane / 3, k = lane % 3;
        s_A[lane] = __dadd_rn(__dadd_rn(__dmul_rn(__dmul_rn(s_E[j], s_E[k]), inv[0]),
                                        __dmul_rn(__dmul_rn(s_E[3 + j], s_E[3 + k]), inv[1])),
                              __dmul_rn(__dmul_rn(s_E[6 + j], s_E[6 + k]), inv[2]));
    }
    __syncwarp();
}

// ---------------------------------------------------------------------------
// particle p; CBLOCK threads
// io_ft (6 doubles: F_ext, T_ext) replaces the particle's external force and
// torque for this step and from then on; io_rec (25 doubles) receives its
// record after the step.  Either may be null.  Both may be pinned host memory
// that the GPU reads and writes directly.
__device__ __forceinline__ void crit_block(const PParams& P, int p, const double* io_ft = nullptr,
                                           double* io_rec = nullptr)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ PartDev S;
    __shared__ PartK K;
    __shared__ long long s_acc[NACC];
    extern __shared__ uint64_t s_maps[];            // both ring slots of the occupancy map, smax*smax rows each
    __shared__ double s_E[9], s_A[9], s_xc[3], s_dm;
    __shared__ float s_e[3][3], s_inv[3], s_ro[3];
    __shared__ double s_x6[6], s_ft0[6];             // the solution and F0, T0 (force and torque records)
    __shared__ int s_o[3], s_nsolid, s_namb;
    __shared__ int s_ext[4];                        // rows solid now or before: y min, max, z min, max (new cube)
    __shared__ int s_amb[MAXAMB];
    __shared__ double s_FL[3], s_fpair[MAXPB][3];   // lubrication: total and per other particle of the box
    __shared__ int s_nnb, s_nbl[MAXNB];

    // ---- stage the state, the snapshot (so that every field not updated
    // below carries over) and this step's accumulators; clear the accumulators
    {
        ldcg_copy(&S, P.pd + p, tid, CBLOCK);
        ldcg_copy(&K, P.pk + p, tid, CBLOCK);
        long long* acc = P.acc + (long long)p * NACC;
        for (int e = tid; e < NACC; e += CBLOCK) {
            s_acc[e] = __ldcg(acc + e);
            acc[e] = 0;
        }
        const uint64_t* r0 = P.rows + (size_t)p * 2 * (MAXS * MAXS);
        const int n = P.smax * P.smax;
        for (int r = tid; r < n; r += CBLOCK) {
            s_maps[r] = __ldcg(r0 + r);
            s_maps[n + r] = __ldcg(r0 + MAXS * MAXS + r);
        }
        if (tid == 0) {
            s_nsolid = 0; s_namb = 0; s_dm = 0.0;
            s_ext[0] = s_ext[2] = 1 << 20;
            s_ext[1] = s_ext[3] = -(1 << 20);
        }
    }
    __syncthreads();
    if (io_ft) {
        if (tid < 3) S.Fext[tid] = io_ft[tid];
        else if (tid < 6) S.Text[tid - 3] = io_ft[tid];
        __syncthreads();
    }
    // ---- partners for the next iteration and the lubrication forces of this
    // one, from the poses of time t in the ring (slot t & 1, which no crit
    // block writes during this iteration): the same inputs on both sides of
    // every pair, so the partner relation is symmetric and the pair forces are
    // exactly opposite; warp 1, while warp 0 prepares the solve
    if (tid == 0) { s_FL[0] = s_FL[1] = s_FL[2] = 0.0; s_nnb = 0; }
    __syncthreads();
    if (!P.init && K.pcnt > 1 && warp == 1) {
        const int t = (int)(S.step & 1);
        const int Lb[3] = {K.nx, K.ny, K.nz};
        const bool per[3] = {true, !K.walls, true};
        const bool lub = K.lub_cut > 0.0;
        for (int j0 = 0; j0 < K.pcnt; j0 += 32) {
            const int j = j0 + lane;
            const int q = K.pbeg + j;
            bool near = false;
            double fp[3] = {0.0, 0.0, 0.0};
            if (j < K.pcnt && q != p) {
                const int lo = min(p, q), hi = max(p, q);
                double rl[RINGD], rh[RINGD];
                for (int e = 0; e < RINGD; ++e) {
                    rl[e] = __ldcg(P.ring + ((size_t)lo * 2 + t) * RINGD + e);
                    rh[e] = __ldcg(P.ring + ((size_t)hi * 2 + t) * RINGD + e);
                }
                const double reach = 0.5 * (double)(P.pd[lo].S + P.pd[hi].S) + 3.0;
                near = true;
                for (int k = 0; k < 3; ++k)
                    near = near && fabs(min_image_d(rh[k] - rl[k], Lb[k], per[k])) < reach;
                if (near && lub) {
                    double f[3];
                    lubrication_pair(rl, P.pd[lo].semi, P.pd[lo].M, rh, P.pd[hi].semi, P.pd[hi].M, Lb, per, K.mu,
                                     K.lub_cut, f);
                    const double sg = (p == lo) ? 1.0 : -1.0;
                    for (int c = 0; c < 3; ++c) fp[c] = sg * f[c];
                }
            }
            if (j < MAXPB)
                for (int c = 0; c < 3; ++c) s_fpair[j][c] = fp[c];
            const unsigned bal = __ballot_sync(0xffffffffu, near);
            if (near) {
                const int slot = s_nnb + __popc(bal & ((1u << lane) - 1u));
                if (slot < MAXNB) s_nbl[slot] = q;
            }
            __syncwarp();
            if (lane == 0) s_nnb += __popc(bal);
            __syncwarp();
        }
        if (lane < 3 && lub) {
            double a = 0.0;
            for (int j = 0; j < K.pcnt && j < MAXPB; ++j) a += s_fpair[j][lane];    // in index order
            s_FL[lane] = a;
        }
    }
    __syncthreads();
    const int slot_new = P.init ? 0 : (S.slot ^ 1);
    uint64_t* s_rows = s_maps + slot_new * P.smax * P.smax;          // map t+1, built below
    const uint64_t* s_old = s_maps + (P.init ? slot_new : S.slot) * P.smax * P.smax;   // map t
    const int nx = K.nx, ny = K.ny, nz = K.nz;
    const bool py = !K.walls;
    const int Sd = S.S;

    // ---- warp 0: force, solve, pose (lane k < 3: x/F component k, 3 <= lane < 6: torque component lane-3)
    if (warp == 0 && !P.init) {
        const double rho0 = K.rho0;
        const double inv_fix = 1.0 / FIXD;
        const int k = lane % 3, k1 = (k + 1) % 3, k2 = (k + 2) % 3;
        const bool isT = lane >= 3;
        // F0, T0 (Eq. F0, Eq. T0): this step's link sums about the cube origin,
        // moved to the centre (phi x F for the torque), plus the parts the links
        // alone fix; one branch-free expression for force and torque lanes
        const double phi1 = isT ? S.phi[k1] : 0.0, phi2 = isT ? S.phi[k2] : 0.0;
        const double a0 = (double)s_acc[isT ? ACC_T + k : ACC_F + k];
        const double pxD = phi1 * (double)s_acc[ACC_F + k2] - phi2 * (double)s_acc[ACC_F + k1];
        const double ft0 = 2.0 * ((pxD + a0) * inv_fix) + (isT ? S.T0g[k] : S.F0g[k]);
        // impulse of the nodes covered / uncovered by the last remap (Appendix, step 8)
        double dpl = 0.0;
        const long long ncv = s_acc[ACC_COV], nun = s_acc[ACC_UNC];
        if (ncv != 0 || nun != 0) {
            const double* phi = S.phi;
            const double Jk1 = (double)s_acc[ACC_COV + 2 + k1] * inv_fix, Jk2 = (double)s_acc[ACC_COV + 2 + k2] * inv_fix;
            dpl = isT ? (phi[k1] * Jk2 - phi[k2] * Jk1) + (double)s_acc[ACC_COV + 5 + k] * inv_fix
                      : (double)s_acc[ACC_COV + 2 + k] * inv_fix;
            double dm = (double)ncv * rho0 + (double)s_acc[ACC_COV + 1] * inv_fix;
            if (nun > 0) {
                const double nu = (double)nun;
                const double SM[3] = {(double)s_acc[ACC_UNC + 1], (double)s_acc[ACC_UNC + 2], (double)s_acc[ACC_UNC + 3]};
                double Sr[3];
                for (int a = 0; a < 3; ++a) Sr[a] = nu * phi[a] + SM[a];
                if (!isT) {
                    dpl -= rho0 * (nu * S.U[k] + (S.W[k1] * Sr[k2] - S.W[k2] * Sr[k1]));
                } else {
                    const int ui[3][3] = {{4, 5, 6}, {5, 7, 8}, {6, 8, 9}};
                    auto RR = [&](int i, int j) {
                        return nu * phi[i] * phi[j] + phi[i] * SM[j] + SM[i] * phi[j] + (double)s_acc[ACC_UNC + ui[i][j]];
                    };
                    const double tr = RR(0, 0) + RR(1, 1) + RR(2, 2);
                    const double RRW = RR(k, 0) * S.W[0] + RR(k, 1) * S.W[1] + RR(k, 2) * S.W[2];
                    const double SxU = Sr[k1] * S.U[k2] - Sr[k2] * S.U[k1];
                    dpl -= rho0 * (SxU + S.W[k] * tr - RRW);
                }
                dm -= nu * rho0;
            }
            if (lane == 0) s_dm = dm;
        }
        // right-hand side of Eq. Fdiscrete / Eq. Tdiscrete (dt = 1), times the
        // inverse the auxiliary kernel prepared from zeta, M, I and dI/dt
        double rhs;
        {
            // force lanes: M U_k; torque lanes: (I Omega)_k
            const double m0 = isT ? S.Icur[k * 3] : S.M, v0 = isT ? S.W[0] : S.U[k];
            const double m1 = isT ? S.Icur[k * 3 + 1] : 0.0, m2 = isT ? S.Icur[k * 3 + 2] : 0.0;
            rhs = m0 * v0 + m1 * S.W[1] + m2 * S.W[2] + ft0 + (isT ? S.Text[k] : S.Fext[k] + s_FL[k]) + dpl;
        }
        const int row = lane < 6 ? lane : 5;
        double x6 = 0.0;
#pragma unroll
        for (int j = 0; j < 6; ++j) x6 += S.Ainv[row * 6 + j] * __shfl_sync(0xffffffffu, rhs, j);
        if (P.didt_mode == 2) {
            // predictor-corrector for I(t+1): the solution above (I(t+1) ~ I(t) +
            // dI/dt) predicts Omega(t+1), hence the orientation q_p by Eq.
            // qnplus0-1 with the mean angular velocity; the system is solved
            // again with I(t+1) = R(q_p) I_body R(q_p)^T (Eq. Irot)
            double Wp[3], qp[4];
#pragma unroll
            for (int a = 0; a < 3; ++a) Wp[a] = 0.5 * (S.W[a] + __shfl_sync(0xffffffffu, x6, 3 + a));
            const double qpl = quat_step_component(Wp, S.q, lane & 3);
#pragma unroll
            for (int m = 0; m < 4; ++m) qp[m] = __shfl_sync(0xffffffffu, qpl, m);
            double R[3][3];
            R[0][0] = 1.0 - 2.0 * (qp[2] * qp[2] + qp[3] * qp[3]);
            R[1][1] = 1.0 - 2.0 * (qp[1] * qp[1] + qp[3] * qp[3]);
            R[2][2] = 1.0 - 2.0 * (qp[1] * qp[1] + qp[2] * qp[2]);
            R[0][1] = 2.0 * (qp[1] * qp[2] - qp[0] * qp[3]);
            R[1][0] = 2.0 * (qp[1] * qp[2] + qp[0] * qp[3]);
            R[0][2] = 2.0 * (qp[1] * qp[3] + qp[0] * qp[2]);
            R[2][0] = 2.0 * (qp[1] * qp[3] - qp[0] * qp[2]);
            R[1][2] = 2.0 * (qp[2] * qp[3] - qp[0] * qp[1]);
            R[2][1] = 2.0 * (qp[2] * qp[3] + qp[0] * qp[1]);
            // lane j < 6: column j of the corrected matrix; lane 6: the right-hand side
            double col[6];
            const int jc = lane < 7 ? lane : 6;
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                const double b = __shfl_sync(0xffffffffu, rhs, i);
                double v = 0.0;
                if (jc < 6) {
                    v = S.zeta[i * 6 + jc];
                    if (i == jc && i < 3) v += S.M;
                    if (i >= 3 && jc >= 3) {
                        const int a = i - 3, c = jc - 3;
                        v += R[a][0] * S.Ib[0] * R[c][0] + R[a][1] * S.Ib[1] * R[c][1] + R[a][2] * S.Ib[2] * R[c][2];
                    }
                } else {
                    v = b;
                }
                col[i] = v;
            }
            if (!gj_solve6_warp(col, lane) && lane == 0) atomicOr(P.status, ST_NAN);
            double xr = 0.0;
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                const double v = __shfl_sync(0xffffffffu, col[i], 6);
                if (row == i) xr = v;
            }
            x6 = xr;
        }
        // the solution to every lane; x6 and ft0 kept for the force and torque
        // records, which are formed after the new pose is out
        double xs[6];
#pragma unroll
        for (int j = 0; j < 6; ++j) xs[j] = __shfl_sync(0xffffffffu, x6, j);
        if (lane < 6) { s_x6[lane] = x6; s_ft0[lane] = ft0; }
        // Eq. posupdate, Eq. qnplus0-1: rotation by Omega_mid = (Omega + Omega') / 2
        // (lane k < 3 forms component k)
        const double wmk = 0.5 * (S.W[k] + xs[3 + k]);
        const float wkf = (float)wmk;
        double qn;
        const float th2 = __shfl_sync(0xffffffffu, wkf, 0) * __shfl_sync(0xffffffffu, wkf, 0) +
                          __shfl_sync(0xffffffffu, wkf, 1) * __shfl_sync(0xffffffffu, wkf, 1) +
                          __shfl_sync(0xffffffffu, wkf, 2) * __shfl_sync(0xffffffffu, wkf, 2);
        if (th2 < 1e-4f) {
            qn = quat_step_component_small(wkf, S.q, lane & 3);
        } else {
            double Wm[3];
            for (int a = 0; a < 3; ++a) Wm[a] = __shfl_sync(0xffffffffu, wmk, a);
            qn = quat_step_component(Wm, S.q, lane & 3);
        }
        // body x axis at t (the squirmer's axis for the next bounce-back):
        // R_k0 = base + 2 (qa qb + s qc qd)
        const double* q = S.q;
        const double qa = q[k == 0 ? 2 : 1], qb = q[k == 0 ? 2 : (k == 1 ? 2 : 3)];
        const double qc = q[k == 0 ? 3 : 0], qd = q[k == 0 ? 3 : (k == 1 ? 3 : 2)];
        const double xk = S.x[k], Uk = S.U[k], phik = S.phi[k];
        const int ok = S.o[k];
        const double xn = xk + 0.5 * (Uk + xs[k]);
        __syncwarp();
        if (lane < 3) {
            const int L = k == 0 ? nx : (k == 1 ? ny : nz);
            S.x[k] = xn;
            S.U[k] = xs[k];
            S.W[k] = xs[3 + k];
            S.o_prev[k] = ok;
            K.ow_old[k] = wrapi(ok, L);
            K.ro_old[k] = (float)phik;
            const double t2 = fma(k == 2 ? -qc : qc, qd, qa * qb);
            K.e_old[k] = (float)fma(k == 0 ? -2.0 : 2.0, t2, k == 0 ? 1.0 : 0.0);
            S.rec[12 + k] = xs[k]; S.rec[15 + k] = xs[3 + k]; S.rec[18 + k] = xn;
        }
        if (lane < 4) { S.q[lane] = qn; S.rec[21 + lane] = qn; }
        if (lane == 0) {
            K.rows_old = P.rows + ((long long)p * 2 + S.slot) * (MAXS * MAXS);
            K.dm_return = s_dm;
        }
    } else if (warp == 0 && lane == 0) {
        // initial pose: no remap before, nothing to return
        for (int k = 0; k < 3; ++k) {
            S.rec[12 + k] = S.U[k]; S.rec[15 + k] = S.W[k]; S.rec[18 + k] = S.x[k];
            S.rec[k] = S.rec[3 + k] = S.rec[6 + k] = S.rec[9 + k] = 0.0;
            S.inv_semi2[k] = __ddiv_rn(1.0, __dmul_rn(S.semi[k], S.semi[k]));
        }
        for (int k = 0; k < 4; ++k) S.rec[21 + k] = S.q[k];
        K.dm_return = 0.0;
    }
    __syncwarp();

    // ---- the new pose: cube origin and FP32 data of the inside test (warp 0)
    if (warp == 0) {
        if (lane < 3) {
            const int o = (int)floor(S.x[lane]) - S.h;
            const float ro = (float)((double)o - S.x[lane]);
            s_o[lane] = o;
            s_xc[lane] = S.x[lane];
            s_ro[lane] = ro;
            s_inv[lane] = (float)S.inv_semi2[lane];
            // the snapshot's new pose and velocities, one component per lane
            K.ow_new[lane] = wrapi(o, lane == 0 ? nx : (lane == 1 ? ny : nz));
            K.ro_new[lane] = ro;
            K.U[lane] = (float)S.U[lane];
            K.W[lane] = (float)S.W[lane];
            K.Fext[lane] = S.Fext[lane];
            if (lane == 1) K.oy_new = o;
        } else if (lane == 3) {
            const double* q = S.q;
            const float qf[4] = {(float)q[0], (float)q[1], (float)q[2], (float)q[3]};
            // body axes e_m = R(q) u_m in FP32 (the FP32 test only needs ~1e-6)
            const float Rf[9] = {1.f - 2.f * (qf[2] * qf[2] + qf[3] * qf[3]), 2.f * (qf[1] * qf[2] - qf[0] * qf[3]),
                                 2.f * (qf[1] * qf[3] + qf[0] * qf[2]), 2.f * (qf[1] * qf[2] + qf[0] * qf[3]),
                                 1.f - 2.f * (qf[1] * qf[1] + qf[3] * qf[3]), 2.f * (qf[2] * qf[3] - qf[0] * qf[1]),
                                 2.f * (qf[1] * qf[3] - qf[0] * qf[2]), 2.f * (qf[2] * qf[3] + qf[0] * qf[1]),
                                 1.f - 2.f * (qf[1] * qf[1] + qf[2] * qf[2])};
            for (int m = 0; m < 3; ++m)
                for (int j = 0; j < 3; ++j) s_e[m][j] = Rf[j * 3 + m];
        }
    }
    __syncthreads();

    // ---- warp 0: the shape matrix of the exact test (FP64, needed only if a
    // node turns out ambiguous, formed while the other warps build the map) and
    // the force and torque records; warps 1..: occupancy of the new pose, one
    // row per thread, FP32 test per node, near-surface nodes listed for the
    // exact test.
    const uint64_t maskS = Sd >= 64 ? ~0ull : ((1ull << Sd) - 1ull);
    if (warp == 0) {
        canon_shape_warp(S.inv_semi2, S.q, s_E, s_A, lane);
        if (!P.init) {
            // F = F0 - zeta_FU U' - zeta_FOmega Omega' (Eq. Fsplit) + the
            // lubrication force, T likewise (Eq. Tsplit)
            const int row = lane < 6 ? lane : 5;
            double ft = s_ft0[row] + (row < 3 ? s_FL[row] : 0.0);
#pragma unroll
            for (int j = 0; j < 6; ++j) ft -= S.zeta[row * 6 + j] * s_x6[j];
            if (lane < 6) {
                S.rec[lane] = s_ft0[lane];
                S.rec[6 + lane] = ft;
            }
            __syncwarp();
            if (lane < 25) {
                // exponent all ones: Inf or NaN
                const unsigned long long b = (unsigned long long)__double_as_longlong(S.rec[lane]);
                if (((b >> 52) & 0x7ff) == 0x7ff) atomicOr(P.status, ST_NAN);
            }
        }
    } else {
        // Along a row the value v(dx) = a dx^2 + 2 b dx + c is a convex quadratic,
        // so the row's solid nodes form one interval between its roots.  Nodes at
        // least one node from both roots have |v - 1| >= a >= 1/29^2, far above
        // both the FP32 rounding of v and the 1e-4 band of the exact test, and are
        // set from the interval; the nodes within 1.5 of a root (or within 3 of the
        // vertex when the interval is shorter than 4 nodes) take the node-by-node
        // test, which is the whole decision: the map is the one a test of every
        // node gives.  v = sum_m (e_m . d / s_m)^2 with the body axes scaled by
        // 1 / s_m: a sum of three nonnegative squares, each at most v, so its FP32
        // rounding stays a few units of 1e-7 near the surface.
        float es[3][3];
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            const float sm = sqrtf(s_inv[m]);
#pragma unroll
            for (int c = 0; c < 3; ++c) es[m][c] = s_e[m][c] * sm;
        }
        const float ro0 = s_ro[0], ro1 = s_ro[1], ro2 = s_ro[2];
        const float qa = es[0][0] * es[0][0] + es[1][0] * es[1][0] + es[2][0] * es[2][0];
        // With every semi-axis at least one node (1 / s_m^2 <= 1) and cube sides
        // of at most 64 nodes the FP32 rounding of the row minimum
        // v_min = 1 - disc / a stays below 1e-3, so a row with v_min > 1.01 has no
        // solid node and needs no test, and the FP32 roots are within 0.1 node of
        // the exact ones, so nodes half a node from both have |v - 1| >= 1.7 a
        // and the root bands can be one node wide; otherwise the wide bands.
        const bool narrow = fmaxf(s_inv[0], fmaxf(s_inv[1], s_inv[2])) <= 1.0f;
        const float wb = narrow ? 0.5f : 1.5f;
        const int dsh1 = P.init ? 0 : s_o[1] - S.o[1], dsh2 = P.init ? 0 : s_o[2] - S.o[2];
        int ey0 = 1 << 20, ey1 = -(1 << 20), ez0 = 1 << 20, ez1 = -(1 << 20);   // rows solid now or before
        for (int base = (warp - 1) * 32; base < Sd * Sd; base += CBLOCK - 32) {
            const int r = base + lane;
            if (r < Sd * Sd) {
                const int my = r % Sd, mz = r / Sd;
                const float dy = ro1 + my, dz = ro2 + mz;
                const float t0 = es[0][1] * dy + es[0][2] * dz;
                const float t1 = es[1][1] * dy + es[1][2] * dz;
                const float t2 = es[2][1] * dy + es[2][2] * dz;
                const float qb = es[0][0] * t0 + es[1][0] * t1 + es[2][0] * t2;
                const float qc = t0 * t0 + t1 * t1 + t2 * t2;
                const float disc = qb * qb - qa * (qc - 1.0f);
                const float xv = __fdividef(-qb, qa) - ro0;     // the vertex, in cube nodes
                uint64_t word = 0;
                bool touched = false;
                // node ranges of the node-by-node test: around the vertex, or around each root
                float bl0 = 0.0f, bl1 = 0.0f;
                int nbands = 0;
                if (narrow && disc < -0.01f * qa) {
                    nbands = 0;                         // v > 1.01 along the whole row
                } else if (disc < 4.0f * qa * qa) {
                    bl0 = xv - 3.0f;
                    bl1 = xv + 3.0f;
                    nbands = 1;
                } else {
                    const float hw = __fdividef(disc * rsqrtf(disc), qa);   // half-width of the interval, >= 2
                    const float x1 = xv - hw, x2 = xv + hw;
                    const int i0 = max(0, (int)ceilf(x1 + wb)), i1 = min(Sd - 1, (int)floorf(x2 - wb));
                    if (i1 >= i0) {
                        const uint64_t hiMask = i1 >= 63 ? ~0ull : ((1ull << (i1 + 1)) - 1ull);
                        word = hiMask & ~((1ull << i0) - 1ull) & maskS;
                    }
                    bl0 = x1 - wb;
                    bl1 = x2 - wb;
                    nbands = 2;
                }
#pragma unroll
                for (int b = 0; b < 2; ++b) {
                    if (b >= nbands) break;
                    const float lo = b == 0 ? bl0 : bl1, hi = nbands == 1 ? bl1 : lo + 2.0f * wb;
                    const int m0 = max(0, (int)ceilf(lo)), m1 = min(Sd - 1, (int)floorf(hi));
                    for (int mx = m0; mx <= m1; ++mx) {
                        // evaluated from dx directly, not accumulated, so rounding does not grow along the row
                        const float dx = ro0 + mx;
                        const float u0 = es[0][0] * dx + t0;
                        const float u1 = es[1][0] * dx + t1;
                        const float u2 = es[2][0] * dx + t2;
                        const float v = u0 * u0 + u1 * u1 + u2 * u2;
                        const uint64_t bit = 1ull << mx;
                        if (fabsf(v - 1.0f) > 1e-4f) {
                            word = v < 1.0f ? (word | bit) : (word & ~bit);
                        } else {
                            word &= ~bit;
                            touched = true;
                            const int slot = atomicAdd(&s_namb, 1);
                            if (slot < MAXAMB) s_amb[slot] = (mz << 16) | (my << 8) | mx;
                        }
                    }
                }
                s_rows[r] = word;
                if (word != 0 || touched) {
                    ey0 = min(ey0, my); ey1 = max(ey1, my);
                    ez0 = min(ez0, mz); ez1 = max(ez1, mz);
                }
                // row r of the old map, in the new cube's rows
                if (!P.init && s_old[r] != 0) {
                    const int oy = my - dsh1, oz = mz - dsh2;
                    ey0 = min(ey0, oy); ey1 = max(ey1, oy);
                    ez0 = min(ez0, oz); ez1 = max(ez1, oz);
                }
            }
        }
        ey0 = __reduce_min_sync(0xffffffffu, ey0);
        ey1 = __reduce_max_sync(0xffffffffu, ey1);
        ez0 = __reduce_min_sync(0xffffffffu, ez0);
        ez1 = __reduce_max_sync(0xffffffffu, ez1);
        if (lane == 0 && ey0 <= ey1) {
            atomicMin(&s_ext[0], ey0); atomicMax(&s_ext[1], ey1);
            atomicMin(&s_ext[2], ez0); atomicMax(&s_ext[3], ez1);
        }
    }
    __syncthreads();
    const int namb = s_namb;
    if (namb > 0) {
        // exact FP64 test in the oracle's operation order, only for listed nodes
        if (tid == 0 && namb > MAXAMB) atomicOr(P.status, ST_CAPACITY);
        for (int a = tid; a < min(namb, MAXAMB); a += CBLOCK) {
            const int code = s_amb[a];
            const int mx = code & 0xff, my = (code >> 8) & 0xff, mz = (code >> 16) & 0xff;
            const int Xw = wrapi(s_o[0] + mx, nx), Yw = wrapi(s_o[1] + my, ny), Zw = wrapi(s_o[2] + mz, nz);
            if (canon_value(s_A, s_xc, Xw, Yw, Zw, nx, ny, nz, py) <= 1.0)
                atomicOr(reinterpret_cast<unsigned long long*>(&s_rows[mz * Sd + my]), 1ull << mx);
        }
        __syncthreads();
    }
    // ---- publish the map, count solid nodes, reject walls inside the particle
    uint64_t* rows_new = P.rows + ((long long)p * 2 + slot_new) * (MAXS * MAXS);
    {
        int ns = 0;
        for (int r = tid; r < Sd * Sd; r += CBLOCK) {
            uint64_t word = s_rows[r];
            const int Yu = s_o[1] + r % Sd;
            if (!py && (Yu <= 0 || Yu >= ny - 1) && word) {
                atomicOr(P.status, ST_OVERLAP);
                word = 0;
                s_rows[r] = 0;
            }
            rows_new[r] = word;
            ns += __popcll(word);
        }
        ns = __reduce_add_sync(0xffffffffu, ns);
        if (lane == 0 && ns) atomicAdd(&s_nsolid, ns);
    }
    __syncthreads();
    // ---- redo mask of step t+1 in the new cube: nodes fluid now with a solid
    // neighbour now or before, or solid before (uncovered), and nodes covered now;
    // the bulk kernel of t+1 skips them and the boundary kernel writes them
    {
        int dsh[3];                                 // new origin - old origin: old-local = new-local + dsh
        for (int k = 0; k < 3; ++k) dsh[k] = P.init ? 0 : s_o[k] - S.o[k];
        if (tid == 0 && (abs(dsh[0]) > 1 || abs(dsh[1]) > 1 || abs(dsh[2]) > 1)) atomicOr(P.status, ST_CAPACITY);
        auto row_old = [&](int ay, int az) -> uint64_t {
            ay += dsh[1]; az += dsh[2];
            if (ay < 0 || ay >= Sd || az < 0 || az >= Sd) return 0ull;
            const uint64_t w = s_old[az * Sd + ay];
            return (dsh[0] == 1 ? (w >> 1) : (dsh[0] == -1 ? (w << 1) : w)) & maskS;
        };
        uint64_t* need = P.need + (size_t)p * (MAXS * MAXS);
        // solid now or before, row (ay, az) of the new cube
        auto uni = [&](int ay, int az) -> uint64_t {
            if (ay < 0 || ay >= Sd || az < 0 || az >= Sd) return 0ull;
            return s_rows[az * Sd + ay] | row_old(ay, az);
        };
        auto s3 = [](uint64_t w) { return w | (w << 1) | (w >> 1); };
        // rows more than one row from every row solid now or before have no
        // solid neighbour: nothing to redo there
        const int ry0 = s_ext[0] - 1, ry1 = s_ext[1] + 1, rz0 = s_ext[2] - 1, rz1 = s_ext[3] + 1;
        for (int r = tid; r < Sd * Sd; r += CBLOCK) {
            const int my = r % Sd, mz = r / Sd;
            const int Yu = s_o[1] + my;
            uint64_t nd = 0;
            if ((py || (Yu > 0 && Yu < ny - 1)) && my >= ry0 && my <= ry1 && mz >= rz0 && mz <= rz1) {
                // the D3Q19 neighbourhood by rows: this row shifted by one node
                // either way, the four face-adjacent rows shifted by -1, 0, +1,
                // the four diagonal rows unshifted
                const uint64_t u0 = uni(my, mz);
                const uint64_t dil = (u0 << 1) | (u0 >> 1) | s3(uni(my - 1, mz)) | s3(uni(my + 1, mz)) |
                                     s3(uni(my, mz - 1)) | s3(uni(my, mz + 1)) | uni(my - 1, mz - 1) |
                                     uni(my + 1, mz - 1) | uni(my - 1, mz + 1) | uni(my + 1, mz + 1);
                const uint64_t nw = s_rows[r], od = row_old(my, mz);
                nd = (((dil | od) & ~nw) | (nw & ~od)) & maskS;
            }
            need[r] = nd;
        }
        if (tid == 0) {
            NeedHdr h;
            for (int k = 0; k < 3; ++k) h.ow[k] = K.ow_new[k];
            h.S = Sd;
            P.need_hdr[p] = h;
        }
    }
    if (tid == 0) {
        K.rows_new = rows_new;
        K.S = Sd;
        K.nsolid = s_nsolid;
        if (P.init) {
            K.rows_old = rows_new;
            for (int k = 0; k < 3; ++k) {
                K.ow_old[k] = K.ow_new[k];
                K.ro_old[k] = K.ro_new[k];
                K.e_old[k] = s_e[0][k];
                S.o_prev[k] = s_o[k];
            }
        }
        S.slot = slot_new;
        for (int k = 0; k < 3; ++k) S.o[k] = s_o[k];
        S.nsolid = s_nsolid;
        if (!P.init) S.step += 1;
        if (!P.init && K.pcnt > 1) {
            K.nnb = min(s_nnb, MAXNB);
            for (int j = 0; j < K.nnb; ++j) K.nb[j] = s_nbl[j];
            if (s_nnb > MAXNB) atomicOr(P.status, ST_CAPACITY);
        }
        if (Sd > nx || Sd > nz || (py && Sd > ny)) atomicOr(P.status, ST_CAPACITY);
    }
    __syncthreads();
    // ---- write back
    {
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(&S);
        unsigned long long* dst = reinterpret_cast<unsigned long long*>(P.pd + p);
        for (int e = tid; e < (int)(sizeof(PartDev) / 8); e += CBLOCK) dst[e] = src[e];
        const unsigned* ks = reinterpret_cast<const unsigned*>(&K);
        unsigned* kd = reinterpret_cast<unsigned*>(P.pk + p);
        for (int e = tid; e < (int)(sizeof(PartK) / 4); e += CBLOCK) kd[e] = ks[e];
        if (io_rec)
            for (int e = tid; e < RECD; e += CBLOCK) io_rec[e] = S.rec[e];
        // the pose of time t+1 for the partners of the next iteration
        if (!P.init && tid < RINGD)
            P.ring[((size_t)p * 2 + (S.step & 1)) * RINGD + tid] =
                tid < 3 ? S.x[tid] : (tid < 6 ? S.U[tid - 3] : S.q[tid - 6]);
    }
    // ---- the box's uniform terms of the next collision: body force with the
    // counter force over the fluid nodes, and the mass put back
    auto box_terms = [&](double fx, double fy, double fz, double dm, long long ns) {
        const float nf = (float)(K.N - K.nwall - ns);
        const float inf = nf > 0.0f ? 1.0f / nf : 0.0f;
        BoxDyn d;
        d.g[0] = K.body[0] - (K.counter ? (float)fx * inf : 0.0f);
        d.g[1] = K.body[1] - (K.counter ? (float)fy * inf : 0.0f);
        d.g[2] = K.body[2] - (K.counter ? (float)fz * inf : 0.0f);
        d.eps = (float)dm * inf;
        return d;
    };
    if (K.pcnt == 1) {
        // the only particle of its box: no other block to wait for
        if (tid == 0) {
            const BoxDyn d = box_terms(K.Fext[0], K.Fext[1], K.Fext[2], K.dm_return, K.nsolid);
            P.box_dyn[K.box] = d;
            P.pdyn[p] = d;
        }
        return;
    }
    // several particles: the last block of the box sums them
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const int prev = atomicAdd(P.box_done + K.box, 1);
        if (prev == K.pcnt - 1) {
            __threadfence();
            double fx = 0, fy = 0, fz = 0, dm = 0;
            long long ns = 0;
            for (int i = 0; i < K.pcnt; ++i) {
                const volatile PartK& k = P.pk[K.pbeg + i];
                fx += k.Fext[0]; fy += k.Fext[1]; fz += k.Fext[2];
                dm += k.dm_return;
                ns += k.nsolid;
            }
            const BoxDyn d = box_terms(fx, fy, fz, dm, ns);
            P.box_dyn[K.box] = d;
            for (int i = 0; i < K.pcnt; ++i) P.pdyn[K.pbeg + i] = d;
            P.box_done[K.box] = 0;
        }
    }
}

// ---------------------------------------------------------------------------
// D3Q19 velocity components packed two bits per direction (value + 1), so that
// a rolled loop over directions stays small in the instruction cache
__host__ __device__ constexpr unsigned long long pack_c(int comp)
{
    unsigned long long v = 0;
    for (int b = 0; b < Q; ++b) v |= (unsigned long long)((comp == 0 ? cx_of(b) : (comp == 1 ? cy_of(b) : cz_of(b))) + 1) << (2 * b);
    return v;
}
__device__ __forceinline__ int c_of(unsigned long long packed, int b) { return (int)((packed >> (2 * b)) & 3ull) - 1; }

// Auxiliary particle kernel, after the critical one of iteration t and before
// the critical one of t+1: everything the next solve needs that depends only
// on the new pose and map.
//   - the drag matrix (Eq. drag1-drag4).  Per link g = (c_b, r_b x c_b) and
//     zeta = sum_b (2 rho0 w_b / c_s^2) g g^T.  With r_b = phi + m (phi = cube
//     origin - x_c; the -c_b/2 drops out of r_b x c_b) g = T g0, g0 = (c_b,
//     m x c_b), T = [[1, 0], [phi x, 1]], so zeta = T zeta0 T^T where zeta0 =
//     (rho0 / 6) sum_links 36 w_b g0 g0^T is an exact integer sum.  Along a
//     cube row y, z are fixed and m x c_b = alpha + beta x, so a row adds its
//     link count n, sum x and sum x^2 per direction;
//   - the same integer sums give the geometric parts of F0 and T0 (Eq. F0,
//     Eq. T0); squirmer links add their slip (Eq. ubsquirmer) one by one;
//   - the lab-frame inertia and its rate at t+1 (Eq. Irot, Eq. Irotdiff, or
//     the finite difference), and the inverse of the implicit-solve matrix
//     [[M + zeta_FU, zeta_FOmega], [zeta_TU, I + dI/dt + zeta_TOmega]] by
//     Gauss-Jordan elimination with partial pivoting, one column per lane.
constexpr int NSUM = 27;            // zeta0: FU 6, FOmega 9, TOmega 6; sum w n c 3; sum w m x c 3
// particle p; ABLOCK threads
// Nodes of row (my, mz) of particle p's current cube that are solid in a
// partner's current map (after the critical blocks of the last iteration),
// as bits of that row.
__device__ __forceinline__ uint64_t partner_row_mask(const PartDev* pd, const PartK* pk, const uint64_t* rows, int p,
                                                     const int o[3], int nnb, const int L[3], int my, int mz,
                                                     uint64_t maskS)
{
    uint64_t pm = 0;
    for (int j = 0; j < nnb; ++j) {
        const int q = __ldcg(&pk[p].nb[j]);
        const PartDev& Gq = pd[q];
        const int Sq = Gq.S;
        int dd[3];
        for (int k = 0; k < 3; ++k) {
            int v = (Gq.o[k] - o[k]) % L[k];
            if (v < -L[k] / 2) v += L[k];
            if (v >= (L[k] + 1) / 2) v -= L[k];
            dd[k] = v;                              // partner origin - this origin
        }
        const int qy = my - dd[1], qz = mz - dd[2];
        if (qy < 0 || qy >= Sq || qz < 0 || qz >= Sq || dd[0] <= -64 || dd[0] >= 64) continue;
        const uint64_t w = __ldcg(rows + ((long long)q * 2 + Gq.slot) * (MAXS * MAXS) + qz * Sq + qy);
        pm |= dd[0] >= 0 ? (w << dd[0]) : (w >> -dd[0]);
    }
    return pm & maskS;
}

static __device__ __noinline__ void aux_block(const PParams& P, int p)
{
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    PartDev& G = P.pd[p];
    extern __shared__ uint64_t s_new[];
    __shared__ PartDev S;
    __shared__ long long s_sum[NSUM], s_slip[6];
    __shared__ double s_R[9], s_I[9], s_dI[9], s_P[36], s_Z[36];
    __shared__ float s_ro[3], s_ex[3];
    {
        ldcg_copy(&S, P.pd + p, tid, ABLOCK);
        if (tid < NSUM) s_sum[tid] = 0;
        if (tid >= 32 && tid < 38) s_slip[tid - 32] = 0;
    }
    __syncthreads();
    // once per pose: a second call for the same step leaves everything as it is
    // (the finite-difference dI/dt would otherwise see I(t+1) twice)
    if (S.aux_step == S.step) return;
    if (tid == 0) G.aux_step = S.step;
    const BoxDev& B = P.boxes[S.box];
    const int ny = B.ny;
    const bool walls = B.walls != 0;
    const double rho0 = B.rho0;
    const int Sd = S.S;
    const uint64_t maskS = Sd >= 64 ? ~0ull : ((1ull << Sd) - 1ull);
    if (tid < 3) {
        const double ph = (double)S.o[tid] - S.x[tid];
        G.phi[tid] = ph;
        s_ro[tid] = (float)ph;
    }
    if (warp == 1 && lane < 9) {
        // rotation matrix at t+1 (body -> lab)
        const double* q = S.q;
        const int i = lane / 3, j = lane % 3;
        double r;
        if (i == j) {
            const double a = q[1 + (i + 1) % 3], bq = q[1 + (i + 2) % 3];
            r = 1.0 - 2.0 * (a * a + bq * bq);
        } else {
            const int kk = 3 - i - j;
            const double sgn = ((j - i + 3) % 3 == 1) ? -1.0 : 1.0;
            r = 2.0 * (q[1 + i] * q[1 + j] + sgn * q[0] * q[1 + kk]);
        }
        s_R[lane] = r;
        if (j == 0) s_ex[i] = (float)r;
    }
    {
        const uint64_t* rn = P.rows + ((long long)p * 2 + S.slot) * (MAXS * MAXS);
        for (int r = tid; r < Sd * Sd; r += ABLOCK) s_new[r] = __ldcg(rn + r);
    }
    // nodes solid in a partner's new map, in this cube's rows (its links and
    // the drag matrices count fluid nodes only); a node solid in both maps
    // means the bodies overlap
    uint64_t* s_pm = s_new + P.smax * P.smax;
    const int nnb = __ldcg(&P.pk[p].nnb);
    if (nnb > 0) {
        const int Lb[3] = {B.nx, B.ny, B.nz};
        for (int r = tid; r < Sd * Sd; r += ABLOCK)
            s_pm[r] = partner_row_mask(P.pd, P.pk, P.rows, p, S.o, nnb, Lb, r % Sd, r / Sd, maskS);
    }
    __syncthreads();
    if (nnb > 0)
        for (int r = tid; r < Sd * Sd; r += ABLOCK)
            if (s_new[r] & s_pm[r]) atomicOr(P.status, ST_OVERLAP);
    // the integer link sums depend on the map alone: when the new map is the
    // last one, on the same cube (no partner, sums of the last pose kept),
    // they are taken over instead of summed again; a particle covers or
    // uncovers a node only every few tens of steps at these speeds
    __shared__ int s_same;
    if (tid == 0)
        s_same = nnb == 0 && S.lsum_step == S.step - 1 && S.o[0] == S.o_prev[0] && S.o[1] == S.o_prev[1] &&
                 S.o[2] == S.o_prev[2];
    __syncthreads();
    if (s_same) {
        const uint64_t* ro = P.rows + ((long long)p * 2 + (S.slot ^ 1)) * (MAXS * MAXS);
        bool diff = false;
        for (int r = tid; r < Sd * Sd; r += ABLOCK) diff = diff || (__ldcg(ro + r) != s_new[r]);
        if (__syncthreads_or(diff) && tid == 0) s_same = 0;
        __syncthreads();
    }

    // ---- integer link sums of the new map, one cube row per thread; the
    // direction loop is unrolled so that every c_b is a constant and the 27
    // sums stay in registers
    const bool squirmer = (S.B1 != 0.0 || S.B2 != 0.0);
    if (s_same) {
        if (tid < NSUM) s_sum[tid] = S.lsum[tid];
    } else {
        int fu0 = 0, fu1 = 0, fu2 = 0, fu3 = 0, fu4 = 0, fu5 = 0;                 // FU: xx xy xz yy yz zz
        int fo[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};                                   // FOmega[i][j]
        int to0 = 0, to1 = 0, to2 = 0, to3 = 0, to4 = 0, to5 = 0;                 // TOmega: xx xy xz yy yz zz
        int g0 = 0, g1 = 0, g2 = 0, gm0 = 0, gm1 = 0, gm2 = 0;                    // sum w n c, sum w m x c
        for (int r = tid; r < Sd * Sd; r += ABLOCK) {
            const int my = r % Sd, mz = r / Sd;
            const int Yu = S.o[1] + my;
            if (walls && (Yu <= 0 || Yu >= ny - 1)) continue;
            const uint64_t fluid = ~s_new[r] & (nnb > 0 ? ~s_pm[r] : ~0ull) & maskS;
#pragma unroll
            for (int b = 1; b < Q; ++b) {
                const int cx = cx_of(b), cy = cy_of(b), cz = cz_of(b);
                const int ay = my + cy, az = mz + cz;
                if (ay < 0 || ay >= Sd || az < 0 || az >= Sd) continue;
                const uint64_t nb = s_new[az * Sd + ay];
                uint64_t L = fluid & (cx == 1 ? (nb >> 1) : (cx == -1 ? (nb << 1) : nb));
                if (!L) continue;
                const int kw = b <= 6 ? 2 : 1;               // 36 w_b
                const int n = __popcll(L);
                int sx = 0, sxx = 0;
                while (L) {
                    const int mx = __ffsll((long long)L) - 1;
                    L &= L - 1;
                    sx += mx;
                    sxx += mx * mx;
                }
                // m x c = alpha + beta x along the row
                const int a0 = my * cz - mz * cy, a1 = mz * cx, a2 = -my * cx;
                const int b1 = -cz, b2 = cy;
                const int v0 = a0 * n, v1 = a1 * n + b1 * sx, v2 = a2 * n + b2 * sx;
                fu0 += kw * n * cx * cx; fu1 += kw * n * cx * cy; fu2 += kw * n * cx * cz;
                fu3 += kw * n * cy * cy; fu4 += kw * n * cy * cz; fu5 += kw * n * cz * cz;
                fo[0] += kw * cx * v0; fo[1] += kw * cx * v1; fo[2] += kw * cx * v2;
                fo[3] += kw * cy * v0; fo[4] += kw * cy * v1; fo[5] += kw * cy * v2;
                fo[6] += kw * cz * v0; fo[7] += kw * cz * v1; fo[8] += kw * cz * v2;
                to0 += kw * a0 * a0 * n;
                to1 += kw * (a0 * a1 * n + a0 * b1 * sx);
                to2 += kw * (a0 * a2 * n + a0 * b2 * sx);
                to3 += kw * (a1 * a1 * n + 2 * a1 * b1 * sx + b1 * b1 * sxx);
                to4 += kw * (a1 * a2 * n + (a1 * b2 + a2 * b1) * sx + b1 * b2 * sxx);
                to5 += kw * (a2 * a2 * n + 2 * a2 * b2 * sx + b2 * b2 * sxx);
                g0 += kw * n * cx; g1 += kw * n * cy; g2 += kw * n * cz;
                gm0 += kw * v0; gm1 += kw * v1; gm2 += kw * v2;
            }
        }
        const int acc[NSUM] = {fu0, fu1, fu2, fu3, fu4, fu5, fo[0], fo[1], fo[2], fo[3], fo[4], fo[5], fo[6], fo[7], fo[8],
                               to0, to1, to2, to3, to4, to5, g0, g1, g2, gm0, gm1, gm2};
#pragma unroll
        for (int k = 0; k < NSUM; ++k) {
            const long long v = (k >= 15 && k < 21) ? warp_sum_ll(acc[k]) : (long long)__reduce_add_sync(0xffffffffu, acc[k]);
            if (lane == 0 && v) atomicAdd(reinterpret_cast<unsigned long long*>(&s_sum[k]), (unsigned long long)v);
        }
        __syncthreads();
        if (tid < NSUM) G.lsum[tid] = s_sum[tid];
    }
    if (tid == 0) G.lsum_step = S.step;
    if (squirmer) {
        // squirmer slip (Eq. ubsquirmer) at every link: sum w s c and sum w s (m x c)
        constexpr unsigned long long PX = pack_c(0), PY = pack_c(1), PZ = pack_c(2);
        long long sl[6] = {0, 0, 0, 0, 0, 0};
        const float sa = (float)S.semi[0];
        const float seps2 = (float)fmax(0.0, 1.0 - (S.semi[1] * S.semi[1]) / (S.semi[0] * S.semi[0]));
        const float sB1 = (float)S.B1, sB2 = (float)S.B2;
        for (int r = tid; r < Sd * Sd; r += ABLOCK) {
            const int my = r % Sd, mz = r / Sd;
            const int Yu = S.o[1] + my;
            if (walls && (Yu <= 0 || Yu >= ny - 1)) continue;
            const uint64_t fluid = ~s_new[r] & (nnb > 0 ? ~s_pm[r] : ~0ull) & maskS;
#pragma unroll 1
            for (int b = 1; b < Q; ++b) {
                const int cx = c_of(PX, b), cy = c_of(PY, b), cz = c_of(PZ, b);
                const int ay = my + cy, az = mz + cz;
                if (ay < 0 || ay >= Sd || az < 0 || az >= Sd) continue;
                const uint64_t nb = s_new[az * Sd + ay];
                uint64_t L = fluid & (cx == 1 ? (nb >> 1) : (cx == -1 ? (nb << 1) : nb));
                const int kw = b <= 6 ? 2 : 1;
                while (L) {
                    const int mx = __ffsll((long long)L) - 1;
                    L &= L - 1;
                    const float rx = s_ro[0] + mx + 0.5f * cx, ry = s_ro[1] + my + 0.5f * cy, rz = s_ro[2] + mz + 0.5f * cz;
                    float ux, uy, uz;
                    squirmer_slip(s_ex, sa, seps2, sB1, sB2, rx, ry, rz, ux, uy, uz);
                    const long long sv = kw * __float2ll_rn((ux * cx + uy * cy + uz * cz) * FIXF);
                    sl[0] += sv * cx; sl[1] += sv * cy; sl[2] += sv * cz;
                    sl[3] += sv * (my * cz - mz * cy); sl[4] += sv * (mz * cx - mx * cz); sl[5] += sv * (mx * cy - my * cx);
                }
            }
        }
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const long long v = warp_sum_ll(sl[k]);
            if (lane == 0 && v) atomicAdd(reinterpret_cast<unsigned long long*>(&s_slip[k]), (unsigned long long)v);
        }
    }
    if (warp == 2 && lane < 9) {
        // lab-frame inertia at t+1 (Eq. Irot): I = R diag(I_body) R^T
        const int i = lane / 3, j = lane % 3;
        s_I[lane] = s_R[i * 3] * S.Ib[0] * s_R[j * 3] + s_R[i * 3 + 1] * S.Ib[1] * s_R[j * 3 + 1] +
                    s_R[i * 3 + 2] * S.Ib[2] * s_R[j * 3 + 2];
    }
    __syncthreads();

    // ---- P = T zeta0, the inertia rate, the fixed parts of F0 and T0
    double phi[3];
    for (int a = 0; a < 3; ++a) phi[a] = (double)S.o[a] - S.x[a];
    auto z0 = [&](int i, int j) -> double {        // zeta0 / (rho0 / 6) from the packed sums
        constexpr int sym[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
        if (i < 3 && j < 3) return (double)s_sum[sym[i][j]];
        if (i < 3) return (double)s_sum[6 + i * 3 + (j - 3)];
        if (j < 3) return (double)s_sum[6 + j * 3 + (i - 3)];
        return (double)s_sum[15 + sym[i - 3][j - 3]];
    };
    if (tid < 36) {
        // rows 3..5 of P gain [phi x] times rows 0..2
        const int i = tid / 6, j = tid % 6;
        double v = z0(i, j);
        if (i >= 3) {
            const int a = i - 3, a1 = (a + 1) % 3, a2 = (a + 2) % 3;
            v += -phi[a2] * z0(a1, j) + phi[a1] * z0(a2, j);
        }
        s_P[tid] = v;
    } else if (warp == 2 && lane < 9) {
        // its rate (Eq. Irotdiff): [Omega]x I - I [Omega]x, or the finite difference
        const int i = lane / 3, j = lane % 3;
        if (P.didt_mode != 1) {
            const double* W = S.W;
            const double Wk[9] = {0, -W[2], W[1], W[2], 0, -W[0], -W[1], W[0], 0};
            s_dI[lane] = Wk[i * 3] * s_I[j] + Wk[i * 3 + 1] * s_I[3 + j] + Wk[i * 3 + 2] * s_I[6 + j] -
                         (s_I[i * 3] * Wk[j] + s_I[i * 3 + 1] * Wk[3 + j] + s_I[i * 3 + 2] * Wk[6 + j]);
        } else {
            s_dI[lane] = P.init ? 0.0 : s_I[lane] - S.Icur[lane];
        }
    } else if (warp == 3 && lane < 6) {
        // F0, T0 parts fixed by the links: 2 rho0 sum w_b c_b (geometric) and the
        // squirmer slip, about the centre (Eq. F0, Eq. T0)
        const double inv_fix = 1.0 / FIXD;
        constexpr double i36 = 1.0 / 36.0;
        const double fix36 = inv_fix * i36;
        const int k = lane % 3, k1 = (k + 1) % 3, k2 = (k + 2) % 3;
        const long long* Gs = s_sum + 21;     // [0..2] sum w n c, [3..5] sum w m x c
        if (lane < 3) {
            G.F0g[k] = 2.0 * rho0 * ((double)Gs[k] * i36) - 6.0 * rho0 * ((double)s_slip[k] * fix36);
        } else {
            const double pxG = (phi[k1] * (double)Gs[k2] - phi[k2] * (double)Gs[k1]) * i36;
            const double pxS = (phi[k1] * (double)s_slip[k2] - phi[k2] * (double)s_slip[k1]) * fix36;
            G.T0g[k] = 2.0 * rho0 * (pxG + (double)Gs[3 + k] * i36) - 6.0 * rho0 * (pxS + (double)s_slip[3 + k] * fix36);
        }
    }
    __syncthreads();
    // ---- zeta = (rho0 / 6) P T^T
    if (tid < 36) {
        // columns 3..5 gain P times [phi x]^T
        const int i = tid / 6, j = tid % 6;
        double v = s_P[tid];
        if (j >= 3) {
            const int b = j - 3, b1 = (b + 1) % 3, b2 = (b + 2) % 3;
            v += -phi[b2] * s_P[i * 6 + b1] + phi[b1] * s_P[i * 6 + b2];
        }
        v *= rho0 * (1.0 / 6.0);
        s_Z[tid] = v;
        G.zeta[tid] = v;
    }
    __syncthreads();
    // ---- inverse of the solve matrix A = [[M + zeta_FU, zeta_FOmega], [zeta_TU, I + dI/dt + zeta_TOmega]]:
    // an FP32 inverse X0 by 3 x 3 blocks, then two Newton-Schulz steps in FP64,
    // X <- X + X (I - A X), each of which squares the relative error of X (about
    // 1e-7 times the condition number after FP32), so that X carries FP64
    // accuracy.  FP64 instructions issue at a small fraction of the FP32 rate on
    // this GPU, one warp at a time per scheduler, so the FP64 part is only the
    // two 6-term products per step, one entry of A^-1 per thread.
    __shared__ double s_Af[36], s_X[36], s_Ei[36];
    __shared__ float s_f[36];
    __shared__ int s_bad;
    if (tid < 36) {
        const int i = tid / 6, j = tid % 6;
        double a = s_Z[tid];
        if (i < 3 && i == j) a += S.M;
        if (i >= 3 && j >= 3) a += s_I[(i - 3) * 3 + (j - 3)] + s_dI[(i - 3) * 3 + (j - 3)];
        s_Af[tid] = a;
    }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    if (warp == 0) {
        // FP32, by blocks: A = [[P, B], [C, D]] (each 3 x 3), X = P^-1 B,
        // Y = C P^-1, the Schur complement S = D - C X,
        //   A^-1 = [[P^-1 + X S^-1 Y, -X S^-1], [-S^-1 Y, S^-1]];
        // P (M I + the drag's translation block) and S are symmetric positive
        // definite up to the small dI/dt, so their inverses by cofactors need no
        // pivoting.  Lane e < 9 holds entry (e / 3, e % 3) of each block.
        float* sP = s_f;                            // P^-1 [0, 9), X [9, 18), Y [18, 27), S^-1 [27, 36)
        const int e = lane < 9 ? lane : 8, r = e / 3, c = e % 3;
        const int r1 = (r + 1) % 3, r2 = (r + 2) % 3, c1 = (c + 1) % 3, c2 = (c + 2) % 3;
        auto Af = [&](int a, int b) { return (float)s_Af[a * 6 + b]; };
        const float cofP = Af(c1, r1) * Af(c2, r2) - Af(c1, r2) * Af(c2, r1);
        float detP = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) detP += Af(0, k) * __shfl_sync(0xffffffffu, cofP, k * 3);
        const float Pi = cofP / detP;
        if (lane < 9) sP[e] = Pi;
        __syncwarp();
        float x = 0.0f, y = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            x += sP[r * 3 + k] * Af(k, 3 + c);
            y += Af(3 + r, k) * sP[k * 3 + c];
        }
        if (lane < 9) { sP[9 + e] = x; sP[18 + e] = y; }
        __syncwarp();
        float sv = Af(3 + r, 3 + c);
#pragma unroll
        for (int k = 0; k < 3; ++k) sv -= Af(3 + r, k) * sP[9 + k * 3 + c];
        if (lane < 9) sP[27 + e] = sv;
        __syncwarp();
        const float* Sm = sP + 27;
        const float cofS = Sm[c1 * 3 + r1] * Sm[c2 * 3 + r2] - Sm[c1 * 3 + r2] * Sm[c2 * 3 + r1];
        float detS = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) detS += Sm[k] * __shfl_sync(0xffffffffu, cofS, k * 3);
        const float Si = cofS / detS;
        __syncwarp();
        if (lane < 9) sP[27 + e] = Si;
        __syncwarp();
        float sy = 0.0f, xs = 0.0f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            sy += sP[27 + r * 3 + k] * sP[18 + k * 3 + c];
            xs += sP[9 + r * 3 + k] * sP[27 + k * 3 + c];
        }
        __syncwarp();
        if (lane < 9) sP[18 + e] = sy;
        __syncwarp();
        float tl = Pi;
#pragma unroll
        for (int k = 0; k < 3; ++k) tl += sP[9 + r * 3 + k] * sP[18 + k * 3 + c];
        if (lane < 9) {
            s_X[r * 6 + c] = tl;
            s_X[r * 6 + 3 + c] = -xs;
            s_X[(3 + r) * 6 + c] = -sy;
            s_X[(3 + r) * 6 + 3 + c] = Si;
            if (!(detP != 0.0f && detS != 0.0f && isfinite(tl) && isfinite(xs) && isfinite(sy) && isfinite(Si)))
                s_bad = 1;
        }
    } else if (warp == 1 && lane < 9) {
        G.Icur[lane] = s_I[lane];
    }
    __syncthreads();
    const int ri = tid / 6, ci = tid % 6;
#pragma unroll 1
    for (int step = 0; step < 2; ++step) {
        if (tid < 36) {                             // I - A X
            double v = ri == ci ? 1.0 : 0.0;
#pragma unroll
            for (int k = 0; k < 6; ++k) v = fma(-s_Af[ri * 6 + k], s_X[k * 6 + ci], v);
            s_Ei[tid] = v;
        }
        __syncthreads();
        double xn = 0.0;
        if (tid < 36) {                             // X + X (I - A X)
            xn = s_X[tid];
#pragma unroll
            for (int k = 0; k < 6; ++k) xn = fma(s_X[ri * 6 + k], s_Ei[k * 6 + ci], xn);
        }
        __syncthreads();
        if (tid < 36) s_X[tid] = xn;
        __syncthreads();
    }
    if (tid < 36) {
        G.Ainv[tid] = s_X[tid];
        if ((tid == 0 && s_bad) || !isfinite(s_X[tid])) atomicOr(P.status, ST_NAN);
    }
}

}  // namespace lbsph
