// Particle kernels, one CTA per particle.
//
// particle_crit (between the boundary kernel of iteration t and the bulk kernel
// of t+1, on the critical path):
//   - F0, T0 of the links of map t (Eq. F0, Eq. T0) from the boundary kernel's
//     fixed-point sums, reduced over the 18 directions in exact integer
//     arithmetic, then combined with the geometric and squirmer-slip parts;
//   - the impulse of the nodes covered / uncovered by the last remap;
//   - lab-frame inertia I = R I_body R^T and dI/dt = [Omega]x I - I [Omega]x
//     (Eq. Irot, Eq. Irotdiff in closed form), or the finite difference;
//   - the implicit solve of Eq. Fdiscrete / Eq. Tdiscrete by Gauss-Jordan
//     elimination with partial pivoting, one column per lane;
//   - Eq. posupdate and Eq. qnplus0-1;
//   - the occupancy map of the new pose (Eq. ellipsoidsurface): an FP32 test
//     settles every node whose value is farther than 1e-4 from 1, the rest use
//     the exact FP64 test in the fixed operation order the CPU oracle also uses;
//   - the last CTA of a box writes the box's uniform body force and mass return
//     for the next collision.
// FP64 throughput is low on this part, so FP64 work is spread over lanes and
// kept to the few operations that need it.
//
// particle_aux (concurrent with the bulk kernel of t+1): integer link moments
// of the new map, the drag matrices of Eq. drag1-drag4 from them, the
// squirmer-slip sums, and the list of nodes the boundary kernel must redo.
#include <cmath>
#include <mutex>

#include "../../include/lbsph.h"
#include "lattice_common.cuh"

namespace lbsph {

// ---- exact FP64 inside test (no contraction: explicit round-to-nearest ops)
__device__ void canon_rotate(const double q[4], const double s[3], double o[3])
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

__device__ void canon_shape(const double semi[3], const double q[4], double A[9], double e[3][3])
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
    return __dsub_rn(d, __dmul_rn(Ld, floor(__dadd_rn(__ddiv_rn(d, Ld), 0.5))));
}

__device__ double canon_value(const double A[9], const double xc[3], int X, int Y, int Z, int nx, int ny,
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

// ---- small FP64 helpers (thread 0)
__device__ __forceinline__ void cross(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ void quat_mul(const double a[4], const double b[4], double o[4])
{
    o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
    o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
    o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
    o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

// rotation matrix of a unit quaternion (body -> lab)
__device__ void rot_matrix(const double q[4], double R[9])
{
    const double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
}

__device__ __forceinline__ int wrapi(int a, int L) { a %= L; return a < 0 ? a + L : a; }

// per-direction part of the 6x6 drag matrix (Eq. drag1-drag4) from the integer
// link moments of direction b, phi = cube origin - x_c
__device__ void drag_terms(int b, const int lm[10], const double phi[3], double rho0, double Z[36])
{
    for (int k = 0; k < 36; ++k) Z[k] = 0.0;
    const double n = lm[0];
    if (n == 0.0) return;
    const double w = wd_of(b) * 6.0 * rho0;             // 2 rho0 w_b / c_s^2
    const double c[3] = {(double)cx_of(b), (double)cy_of(b), (double)cz_of(b)};
    const double M1[3] = {(double)lm[1], (double)lm[2], (double)lm[3]};
    const double M2[9] = {(double)lm[4], (double)lm[5], (double)lm[6], (double)lm[5], (double)lm[7],
                          (double)lm[8], (double)lm[6], (double)lm[8], (double)lm[9]};
    double A1[3], A2[9], v[3];
    for (int i = 0; i < 3; ++i) A1[i] = n * phi[i] + M1[i];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) A2[i * 3 + j] = n * phi[i] * phi[j] + phi[i] * M1[j] + M1[i] * phi[j] + M2[i * 3 + j];
    cross(A1, c, v);                                   // sum over links of r_b x c_b
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            Z[i * 6 + j] = w * n * c[i] * c[j];                  // zeta_FU
            Z[i * 6 + 3 + j] = w * c[i] * v[j];                  // zeta_FOmega
            Z[(3 + i) * 6 + j] = w * v[i] * c[j];                // zeta_TU
        }
    // zeta_TOmega = sum (r x c)(r x c)^T = K A2 K^T, K a = c x a
    const double K[9] = {0, -c[2], c[1], c[2], 0, -c[0], -c[1], c[0], 0};
    double KA[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            KA[i * 3 + j] = K[i * 3] * A2[j] + K[i * 3 + 1] * A2[3 + j] + K[i * 3 + 2] * A2[6 + j];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            Z[(3 + i) * 6 + 3 + j] = w * (KA[i * 3] * K[j * 3] + KA[i * 3 + 1] * K[j * 3 + 1] + KA[i * 3 + 2] * K[j * 3 + 2]);
}

__device__ __forceinline__ unsigned long long abs_bits(double x)
{
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

__device__ __forceinline__ long long shfl_ll(long long v, int src)
{
    return (long long)__shfl_sync(0xffffffffu, (unsigned long long)v, src);
}

__device__ __forceinline__ long long warp_sum_ll(long long v)
{
    for (int o = 16; o > 0; o >>= 1) v += (long long)__shfl_xor_sync(0xffffffffu, (unsigned long long)v, o);
    return v;
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(CBLOCK) particle_crit_kernel(const PParams P)
{
    const int p = blockIdx.x;
    if (p >= P.np) return;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    __shared__ PartDev S;
    __shared__ PartK K;
    __shared__ long long s_acc[NACC];
    __shared__ uint64_t s_rows[MAXS * MAXS];
    __shared__ long long s_isum[18];          // integer force sums
    __shared__ long long s_iterm[Q][18];      // per-direction terms of those sums
    __shared__ double s_F0[3], s_T0[3], s_dP[3], s_dL[3], s_dm;
    __shared__ double s_R[9], s_I[9], s_dI[9], s_x6[6];
    __shared__ float s_e[3][3], s_inv[3], s_ro[3];
    __shared__ int s_o[3], s_nsolid, s_namb;
    __shared__ int s_amb[MAXAMB];
    __shared__ double s_A[9], s_xc[3];

    // ---- stage the state, the lattice snapshot (so that every field not
    // updated below, e.g. buffer pointers, carries over) and this step's
    // accumulators; clear the accumulators
    {
        const unsigned long long* src = reinterpret_cast<const unsigned long long*>(P.pd + p);
        unsigned long long* dst = reinterpret_cast<unsigned long long*>(&S);
        for (int e = tid; e < (int)(sizeof(PartDev) / 8); e += CBLOCK) dst[e] = src[e];
        const unsigned* ks = reinterpret_cast<const unsigned*>(P.pk + p);
        unsigned* kd = reinterpret_cast<unsigned*>(&K);
        for (int e = tid; e < (int)(sizeof(PartK) / 4); e += CBLOCK) kd[e] = ks[e];
        long long* acc = P.acc + (long long)p * NACC;
        for (int e = tid; e < NACC; e += CBLOCK) {
            s_acc[e] = acc[e];
            acc[e] = 0;
        }
        if (tid == 0) { s_nsolid = 0; s_namb = 0; }
    }
    __syncthreads();
    const BoxDev& B = P.boxes[S.box];
    const int nx = B.nx, ny = B.ny, nz = B.nz;
    const bool py = !B.walls;
    const int Sd = S.S;
    const double rho0 = B.rho0;

    if (!P.init) {
        // ---- integer sums over directions: lane b of warp 0 writes direction b's terms
        if (warp == 0 && lane >= 1 && lane < Q) {
            const int b = lane;
            const int c[3] = {cx_of(b), cy_of(b), cz_of(b)};
            const int kw = (b <= 6) ? 2 : 1;                 // 36 w_b
            const long long D = s_acc[ACC_LINK + 4 * b];
            const long long E[3] = {s_acc[ACC_LINK + 4 * b + 1], s_acc[ACC_LINK + 4 * b + 2], s_acc[ACC_LINK + 4 * b + 3]};
            const long long n = S.lm[b][0];
            const long long M1[3] = {S.lm[b][1], S.lm[b][2], S.lm[b][3]};
            const long long sl = S.slip[b][0];
            const long long sm[3] = {S.slip[b][1], S.slip[b][2], S.slip[b][3]};
            long long* t = s_iterm[b];
            for (int k = 0; k < 3; ++k) {
                const int k1 = (k + 1) % 3, k2 = (k + 2) % 3;
                t[k] = D * c[k];                                     // sum D c
                t[3 + k] = E[k1] * c[k2] - E[k2] * c[k1];            // sum E x c
                t[6 + k] = kw * n * c[k];                            // 36 sum w n c
                t[9 + k] = kw * (M1[k1] * c[k2] - M1[k2] * c[k1]);   // 36 sum w M1 x c
                t[12 + k] = kw * sl * c[k];                          // 36 sum w s c
                t[15 + k] = kw * (sm[k1] * c[k2] - sm[k2] * c[k1]);  // 36 sum w (s m) x c
            }
        }
        // ---- rotation matrix at t (warp 1)
        if (warp == 1 && lane < 9) {
            const double* q = S.q;
            const int i = lane / 3, j = lane % 3;
            double r;
            if (i == j) {
                const double a = q[1 + (i + 1) % 3], bq = q[1 + (i + 2) % 3];
                r = 1.0 - 2.0 * (a * a + bq * bq);
            } else {
                // off-diagonal of R: 2 (q_i q_j -/+ q0 q_k)
                const int k = 3 - i - j;
                const double sgn = ((j - i + 3) % 3 == 1) ? -1.0 : 1.0;
                r = 2.0 * (q[1 + i] * q[1 + j] + sgn * q[0] * q[1 + k]);
            }
            s_R[lane] = r;
        }
        __syncthreads();
        if (tid < 18) {
            long long a = 0;
            for (int b = 1; b < Q; ++b) a += s_iterm[b][tid];
            s_isum[tid] = a;
        }
        __syncthreads();
        const double inv_fix = 1.0 / FIXD;
        if (warp == 0 && lane < 6) {
            // F0 (lanes 0-2), T0 (lanes 3-5) (Eq. F0, Eq. T0) with the geometric and slip parts
            const int k = lane % 3, k1 = (k + 1) % 3, k2 = (k + 2) % 3;
            constexpr double i36 = 1.0 / 36.0;
            const double fix36 = inv_fix * i36;
            if (lane < 3) {
                s_F0[k] = 2.0 * ((double)s_isum[k] * inv_fix) + 2.0 * rho0 * ((double)s_isum[6 + k] * i36) -
                          6.0 * rho0 * ((double)s_isum[12 + k] * fix36);
            } else {
                const double phi1 = (double)S.o[k1] - S.x[k1], phi2 = (double)S.o[k2] - S.x[k2];
                const double pxD = (phi1 * (double)s_isum[k2] - phi2 * (double)s_isum[k1]) * inv_fix;
                const double pxG = (phi1 * (double)s_isum[6 + k2] - phi2 * (double)s_isum[6 + k1]) * i36;
                const double pxS = (phi1 * (double)s_isum[12 + k2] - phi2 * (double)s_isum[12 + k1]) * fix36;
                s_T0[k] = 2.0 * (pxD + (double)s_isum[3 + k] * inv_fix) + 2.0 * rho0 * (pxG + (double)s_isum[9 + k] * i36) -
                          6.0 * rho0 * (pxS + (double)s_isum[15 + k] * fix36);
            }
        } else if (warp == 1 && lane < 9) {
            // lab-frame inertia (Eq. Irot): I = R diag(I_body) R^T
            const int i = lane / 3, j = lane % 3;
            s_I[lane] = s_R[i * 3] * S.Ib[0] * s_R[j * 3] + s_R[i * 3 + 1] * S.Ib[1] * s_R[j * 3 + 1] +
                        s_R[i * 3 + 2] * S.Ib[2] * s_R[j * 3 + 2];
        } else if (warp == 2 && lane == 0 && s_acc[ACC_COV] == 0 && s_acc[ACC_UNC] == 0) {
            for (int k = 0; k < 3; ++k) { s_dP[k] = 0.0; s_dL[k] = 0.0; }   // no node changed
            s_dm = 0.0;
        } else if (warp == 2 && lane == 0) {
            // impulse of the nodes covered / uncovered by the last remap
            double phi[3];
            for (int a = 0; a < 3; ++a) phi[a] = (double)S.o[a] - S.x[a];
            const double ncov = (double)s_acc[ACC_COV];
            double J[3], MJ[3], pxj[3], dP[3], dL[3];
            for (int k = 0; k < 3; ++k) {
                J[k] = (double)s_acc[ACC_COV + 2 + k] * inv_fix;
                MJ[k] = (double)s_acc[ACC_COV + 5 + k] * inv_fix;
            }
            cross(phi, J, pxj);
            for (int k = 0; k < 3; ++k) { dP[k] = J[k]; dL[k] = pxj[k] + MJ[k]; }
            double dm = ncov * rho0 + (double)s_acc[ACC_COV + 1] * inv_fix;
            const double nu = (double)s_acc[ACC_UNC];
            if (nu > 0) {
                const double SM[3] = {(double)s_acc[ACC_UNC + 1], (double)s_acc[ACC_UNC + 2], (double)s_acc[ACC_UNC + 3]};
                const double SMM[9] = {(double)s_acc[ACC_UNC + 4], (double)s_acc[ACC_UNC + 5], (double)s_acc[ACC_UNC + 6],
                                       (double)s_acc[ACC_UNC + 5], (double)s_acc[ACC_UNC + 7], (double)s_acc[ACC_UNC + 8],
                                       (double)s_acc[ACC_UNC + 6], (double)s_acc[ACC_UNC + 8], (double)s_acc[ACC_UNC + 9]};
                double Sr[3], RR[9], WxS[3], SxU[3], RRW[3];
                for (int i = 0; i < 3; ++i) Sr[i] = nu * phi[i] + SM[i];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) RR[i * 3 + j] = nu * phi[i] * phi[j] + phi[i] * SM[j] + SM[i] * phi[j] + SMM[i * 3 + j];
                cross(S.W, Sr, WxS);
                cross(Sr, S.U, SxU);
                const double tr = RR[0] + RR[4] + RR[8];
                for (int i = 0; i < 3; ++i) RRW[i] = RR[i * 3] * S.W[0] + RR[i * 3 + 1] * S.W[1] + RR[i * 3 + 2] * S.W[2];
                for (int k = 0; k < 3; ++k) {
                    dP[k] -= rho0 * (nu * S.U[k] + WxS[k]);
                    dL[k] -= rho0 * (SxU[k] + S.W[k] * tr - RRW[k]);
                }
                dm -= nu * rho0;
            }
            for (int k = 0; k < 3; ++k) { s_dP[k] = dP[k]; s_dL[k] = dL[k]; }
            s_dm = dm;
        }
        __syncthreads();
        if (warp == 1 && lane < 9) {
            // its rate (Eq. Irotdiff): [Omega]x I - I [Omega]x, or the finite difference
            const int i = lane / 3, j = lane % 3;
            if (P.didt_mode == 0) {
                const double* W = S.W;
                const double Wk[9] = {0, -W[2], W[1], W[2], 0, -W[0], -W[1], W[0], 0};
                s_dI[lane] = Wk[i * 3] * s_I[j] + Wk[i * 3 + 1] * s_I[3 + j] + Wk[i * 3 + 2] * s_I[6 + j] -
                             (s_I[i * 3] * Wk[j] + s_I[i * 3 + 1] * Wk[3 + j] + s_I[i * 3 + 2] * Wk[6 + j]);
            } else {
                s_dI[lane] = s_I[lane] - S.Iprev[lane];
            }
        }
        __syncthreads();
        if (warp == 0) {
            // ---- Eq. Fdiscrete / Eq. Tdiscrete (dt = 1): Gauss-Jordan, column j on lane j
            double col[6];
            const int j = lane < 7 ? lane : 6;
#pragma unroll
            for (int i = 0; i < 6; ++i) {
                double v;
                if (j < 6) {
                    v = S.zeta[i * 6 + j];
                    if (i == j && i < 3) v += S.M;
                    if (i >= 3 && j >= 3) v += s_I[(i - 3) * 3 + (j - 3)] + s_dI[(i - 3) * 3 + (j - 3)];
                } else if (i < 3) {
                    v = S.M * S.U[i] + s_F0[i] + S.Fext[i] + s_dP[i];
                } else {
                    const int k = i - 3;
                    v = s_I[k * 3] * S.W[0] + s_I[k * 3 + 1] * S.W[1] + s_I[k * 3 + 2] * S.W[2] + s_T0[k] + S.Text[k] + s_dL[k];
                }
                col[i] = v;
            }
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
            if (lane == 6) {
                for (int i = 0; i < 6; ++i) s_x6[i] = col[i];
            }
            if (lane == 0 && !ok) atomicOr(P.status, ST_NAN);
        }
        __syncthreads();
        if (warp == 0 && lane < 6) {
            // F = F0 - zeta_FU U' - zeta_FOmega Omega' (Eq. Fsplit), T likewise (Eq. Tsplit)
            const int k = lane;
            double sres = (k < 3) ? s_F0[k] : s_T0[k - 3];
            for (int j = 0; j < 6; ++j) sres -= S.zeta[k * 6 + j] * s_x6[j];
            S.rec[6 + k] = sres;       // F (k < 3) then T (k >= 3): rec[6..11]
        } else if (warp == 1 && lane == 0) {
            // ---- Eq. posupdate, Eq. qnplus0-1
            double Un[3], Wn[3], Wm[3], qt[4], qn[4];
            for (int k = 0; k < 3; ++k) { Un[k] = s_x6[k]; Wn[k] = s_x6[3 + k]; }
            for (int k = 0; k < 3; ++k) {
                K.ow_old[k] = wrapi(S.o[k], k == 0 ? nx : (k == 1 ? ny : nz));
                K.ro_old[k] = (float)((double)S.o[k] - S.x[k]);
                K.e_old[k] = (float)s_R[k * 3 + 0];
                S.x[k] += 0.5 * (S.U[k] + Un[k]);
                Wm[k] = 0.5 * (S.W[k] + Wn[k]);
            }
            const double th2 = Wm[0] * Wm[0] + Wm[1] * Wm[1] + Wm[2] * Wm[2];
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
            quat_mul(qt, S.q, qn);
            for (int k = 0; k < 4; ++k) S.q[k] = qn[k];
            for (int k = 0; k < 3; ++k) { S.U[k] = Un[k]; S.W[k] = Wn[k]; }
            for (int k = 0; k < 3; ++k) {
                S.rec[k] = s_F0[k]; S.rec[3 + k] = s_T0[k];
                S.rec[12 + k] = Un[k]; S.rec[15 + k] = Wn[k]; S.rec[18 + k] = S.x[k];
            }
            for (int k = 0; k < 4; ++k) S.rec[21 + k] = S.q[k];
            K.rows_old = P.rows + ((long long)p * 2 + S.slot) * (MAXS * MAXS);
            K.dm_return = s_dm;
            for (int k = 0; k < 3; ++k) S.o_prev[k] = S.o[k];
        } else if (warp == 2 && lane < 9) {
            S.Iprev[lane] = s_I[lane];
        }
        __syncthreads();
        if (tid < 25) {
            // exponent all ones: Inf or NaN
            const unsigned long long b = (unsigned long long)__double_as_longlong(S.rec[tid]);
            if (((b >> 52) & 0x7ff) == 0x7ff) atomicOr(P.status, ST_NAN);
        }
    } else if (tid == 0) {
        // initial pose: no remap before, nothing to return
        for (int k = 0; k < 3; ++k) {
            S.rec[12 + k] = S.U[k]; S.rec[15 + k] = S.W[k]; S.rec[18 + k] = S.x[k];
            S.rec[k] = S.rec[3 + k] = S.rec[6 + k] = S.rec[9 + k] = 0.0;
        }
        for (int k = 0; k < 4; ++k) S.rec[21 + k] = S.q[k];
        double R[9];
        rot_matrix(S.q, R);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                S.Iprev[i * 3 + j] = R[i * 3] * S.Ib[0] * R[j * 3] + R[i * 3 + 1] * S.Ib[1] * R[j * 3 + 1] +
                                     R[i * 3 + 2] * S.Ib[2] * R[j * 3 + 2];
        K.dm_return = 0.0;
    }
    __syncthreads();

    // ---- the new pose: cube origin and FP32 data of the inside test
    if (tid == 0) {
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
        for (int k = 0; k < 3; ++k) {
            const int o = (int)floor(S.x[k]) - S.h;
            s_o[k] = o;
            s_xc[k] = S.x[k];
            s_ro[k] = (float)((double)o - S.x[k]);
            s_inv[k] = (float)(1.0 / (S.semi[k] * S.semi[k]));
        }
    }
    __syncthreads();

    // ---- occupancy of the new pose: one row per thread, FP32 test per node
    // (the three projections e_m . d grow by e_m.x per node along the row),
    // near-surface nodes listed for the exact test
    for (int r = tid; r < Sd * Sd; r += CBLOCK) {
        const int my = r % Sd, mz = r / Sd;
        const float dy = s_ro[1] + my, dz = s_ro[2] + mz;
        float t0 = s_e[0][0] * s_ro[0] + s_e[0][1] * dy + s_e[0][2] * dz;
        float t1 = s_e[1][0] * s_ro[0] + s_e[1][1] * dy + s_e[1][2] * dz;
        float t2 = s_e[2][0] * s_ro[0] + s_e[2][1] * dy + s_e[2][2] * dz;
        uint64_t word = 0;
        for (int mx = 0; mx < Sd; ++mx) {
            const float dx = s_ro[0] + mx;
            // evaluated from dx directly, not accumulated, so rounding does not grow along the row
            const float u0 = s_e[0][0] * dx + (t0 - s_e[0][0] * s_ro[0]);
            const float u1 = s_e[1][0] * dx + (t1 - s_e[1][0] * s_ro[0]);
            const float u2 = s_e[2][0] * dx + (t2 - s_e[2][0] * s_ro[0]);
            const float v = u0 * u0 * s_inv[0] + u1 * u1 * s_inv[1] + u2 * u2 * s_inv[2];
            if (fabsf(v - 1.0f) > 1e-4f) {
                if (v < 1.0f) word |= 1ull << mx;
            } else {
                const int slot = atomicAdd(&s_namb, 1);
                if (slot < MAXAMB) s_amb[slot] = (mz << 16) | (my << 8) | mx;
            }
        }
        s_rows[r] = word;
    }
    __syncthreads();
    const int namb = s_namb;
    if (namb > 0) {
        // exact FP64 test in the oracle's operation order, only for listed nodes
        if (tid == 0) {
            double e[3][3];
            canon_shape(S.semi, S.q, s_A, e);
            if (namb > MAXAMB) atomicOr(P.status, ST_CAPACITY);
        }
        __syncthreads();
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
    const int slot_new = P.init ? 0 : (S.slot ^ 1);
    uint64_t* rows_new = P.rows + ((long long)p * 2 + slot_new) * (MAXS * MAXS);
    for (int r = tid; r < Sd * Sd; r += CBLOCK) {
        uint64_t word = s_rows[r];
        const int Yu = s_o[1] + r % Sd;
        if (B.walls && (Yu <= 0 || Yu >= ny - 1) && word) {
            atomicOr(P.status, ST_OVERLAP);
            word = 0;
        }
        rows_new[r] = word;
        if (word) atomicAdd(&s_nsolid, __popcll(word));
    }
    __syncthreads();
    if (tid == 0) {
        K.rows_new = rows_new;
        for (int k = 0; k < 3; ++k) {
            K.ow_new[k] = wrapi(s_o[k], k == 0 ? nx : (k == 1 ? ny : nz));
            K.ro_new[k] = s_ro[k];
            K.U[k] = (float)S.U[k];
            K.W[k] = (float)S.W[k];
            K.Fext[k] = S.Fext[k];
        }
        K.S = Sd;
        K.box = S.box;
        K.acc = P.acc + (long long)p * NACC;
        K.squirmer = (S.B1 != 0.0 || S.B2 != 0.0) ? 1 : 0;
        K.a = (float)S.semi[0];
        K.b = (float)S.semi[1];
        K.eps2 = (float)fmax(0.0, 1.0 - (S.semi[1] * S.semi[1]) / (S.semi[0] * S.semi[0]));
        K.B1 = (float)S.B1;
        K.B2 = (float)S.B2;
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
    }
    // ---- the last CTA of a box sets the box's uniform terms of the next collision
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        const int prev = atomicAdd(P.box_done + S.box, 1);
        if (prev == B.pcnt - 1) {
            __threadfence();
            double fx = 0, fy = 0, fz = 0, dm = 0;
            long long ns = 0;
            for (int i = 0; i < B.pcnt; ++i) {
                const volatile PartK& k = P.pk[B.pbeg + i];
                fx += k.Fext[0]; fy += k.Fext[1]; fz += k.Fext[2];
                dm += k.dm_return;
                ns += k.nsolid;
            }
            const float nf = (float)(B.N - B.nwall - ns);
            const float inf = nf > 0.0f ? 1.0f / nf : 0.0f;
            BoxDyn d;
            d.g[0] = (float)B.body[0] - (B.counter ? (float)fx * inf : 0.0f);
            d.g[1] = (float)B.body[1] - (B.counter ? (float)fy * inf : 0.0f);
            d.g[2] = (float)B.body[2] - (B.counter ? (float)fz * inf : 0.0f);
            d.eps = (float)dm * inf;
            P.box_dyn[S.box] = d;
            P.box_done[S.box] = 0;
        }
    }
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(PBLOCK) particle_aux_kernel(const PParams P)
{
    const int p = blockIdx.x;
    if (p >= P.np) return;
    const int tid = threadIdx.x;
    PartDev& S = P.pd[p];
    const BoxDev& B = P.boxes[S.box];
    const int nx = B.nx, ny = B.ny, nz = B.nz;
    const int Sd = S.S;
    extern __shared__ uint64_t s_dyn[];
    uint64_t* s_new = s_dyn;
    uint64_t* s_old = s_dyn + P.smax * P.smax;
    __shared__ int s_lm[Q][10], s_count;
    __shared__ unsigned long long s_slip[Q][4];
    __shared__ double s_dir[Q][36];
    __shared__ int s_o[3], s_d[3];
    __shared__ float s_ro[3], s_ex[3];
    if (tid == 0) {
        for (int k = 0; k < 3; ++k) {
            s_o[k] = S.o[k];
            s_d[k] = S.o[k] - S.o_prev[k];                 // new origin - old origin, in {-1, 0, 1}
            s_ro[k] = (float)((double)S.o[k] - S.x[k]);
        }
        double R[9];
        rot_matrix(S.q, R);
        for (int k = 0; k < 3; ++k) s_ex[k] = (float)R[k * 3];
        s_count = 0;
        if (abs(s_d[0]) > 1 || abs(s_d[1]) > 1 || abs(s_d[2]) > 1) atomicOr(P.status, ST_CAPACITY);
    }
    for (int e = tid; e < Q * 10; e += PBLOCK) (&s_lm[0][0])[e] = 0;
    for (int e = tid; e < Q * 4; e += PBLOCK) (&s_slip[0][0])[e] = 0ull;
    __syncthreads();
    const uint64_t* rn = P.rows + ((long long)p * 2 + S.slot) * (MAXS * MAXS);
    const uint64_t* ro = P.rows + ((long long)p * 2 + (P.init ? S.slot : (S.slot ^ 1))) * (MAXS * MAXS);
    const uint64_t maskS = Sd >= 64 ? ~0ull : ((1ull << Sd) - 1ull);
    for (int r = tid; r < Sd * Sd; r += PBLOCK) {
        s_new[r] = rn[r];
        // old map in new cube coordinates: new-local m is old-local m + d
        const int my = r % Sd + (P.init ? 0 : s_d[1]), mz = r / Sd + (P.init ? 0 : s_d[2]);
        uint64_t w = 0;
        if (my >= 0 && my < Sd && mz >= 0 && mz < Sd) {
            w = ro[mz * Sd + my];
            const int dx = P.init ? 0 : s_d[0];
            w = dx == 1 ? (w >> 1) : (dx == -1 ? (w << 1) : w);
            w &= maskS;
        }
        s_old[r] = w;
    }
    __syncthreads();

    // ---- link moments of the new map, squirmer slip sums
    const bool squirmer = (S.B1 != 0.0 || S.B2 != 0.0);
    const float sa = (float)S.semi[0];
    const float seps2 = (float)fmax(0.0, 1.0 - (S.semi[1] * S.semi[1]) / (S.semi[0] * S.semi[0]));
    const float sB1 = (float)S.B1, sB2 = (float)S.B2;
    constexpr int NE = (PBLOCK / 18) * 18;
    if (tid < NE) {
        const int b = 1 + (int)(tid % 18);
        const int cbx = cx_of(b), cby = cy_of(b), cbz = cz_of(b);
        int mom[10] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
        long long sl[4] = {0, 0, 0, 0};
        for (int r = tid / 18; r < Sd * Sd; r += NE / 18) {
            const int my = r % Sd, mz = r / Sd;
            const int Yu = s_o[1] + my;
            if (B.walls && (Yu <= 0 || Yu >= ny - 1)) continue;
            const int ny2 = my + cby, nz2 = mz + cbz;
            if (ny2 < 0 || ny2 >= Sd || nz2 < 0 || nz2 >= Sd) continue;
            const uint64_t nb = s_new[nz2 * Sd + ny2];
            const uint64_t sh = cbx == 1 ? (nb >> 1) : (cbx == -1 ? (nb << 1) : nb);
            uint64_t L = ~s_new[r] & sh & maskS;
            while (L) {
                const int mx = __ffsll((long long)L) - 1;
                L &= L - 1;
                mom[0] += 1;
                mom[1] += mx; mom[2] += my; mom[3] += mz;
                mom[4] += mx * mx; mom[5] += mx * my; mom[6] += mx * mz;
                mom[7] += my * my; mom[8] += my * mz; mom[9] += mz * mz;
                if (squirmer) {
                    const float rx = s_ro[0] + mx + 0.5f * cbx, ry = s_ro[1] + my + 0.5f * cby, rz = s_ro[2] + mz + 0.5f * cbz;
                    float ux, uy, uz;
                    squirmer_slip(s_ex, sa, seps2, sB1, sB2, rx, ry, rz, ux, uy, uz);
                    const long long sv = __float2ll_rn((ux * cbx + uy * cby + uz * cbz) * FIXF);
                    sl[0] += sv; sl[1] += sv * mx; sl[2] += sv * my; sl[3] += sv * mz;
                }
            }
        }
        for (int k = 0; k < 10; ++k)
            if (mom[k]) atomicAdd(&s_lm[b][k], mom[k]);
        for (int k = 0; k < 4; ++k)
            if (sl[k]) atomicAdd(&s_slip[b][k], (unsigned long long)sl[k]);
    }

    // ---- nodes the boundary kernel redoes: fluid now with a solid neighbour now
    // or before (or solid before), and nodes covered now
    for (int r = tid; r < Sd * Sd; r += PBLOCK) {
        const int my = r % Sd, mz = r / Sd;
        const int Yu = s_o[1] + my;
        if (B.walls && (Yu <= 0 || Yu >= ny - 1)) continue;
        uint64_t dil = 0;
#pragma unroll
        for (int b = 1; b < Q; ++b) {
            const int ny2 = my + cy_of(b), nz2 = mz + cz_of(b);
            if (ny2 < 0 || ny2 >= Sd || nz2 < 0 || nz2 >= Sd) continue;
            const uint64_t nb = s_new[nz2 * Sd + ny2] | s_old[nz2 * Sd + ny2];
            dil |= cx_of(b) == 1 ? (nb >> 1) : (cx_of(b) == -1 ? (nb << 1) : nb);
        }
        const uint64_t nw = s_new[r], od = s_old[r];
        uint64_t need = (((dil | od) & ~nw) | (nw & ~od)) & maskS;
        const int n = __popcll(need);
        if (!n) continue;
        const int base = atomicAdd(&s_count, n);
        int k = 0;
        while (need) {
            const int mx = __ffsll((long long)need) - 1;
            need &= need - 1;
            if (base + k < P.pk[p].list_cap) P.pk[p].list[base + k] = (unsigned)((mz << 16) | (my << 8) | mx);
            ++k;
        }
    }
    __syncthreads();

    // ---- drag matrix of the new links: per direction, then summed
    if (tid >= 1 && tid < Q) {
        double phi[3];
        for (int k = 0; k < 3; ++k) phi[k] = (double)S.o[k] - S.x[k];
        drag_terms(tid, s_lm[tid], phi, B.rho0, s_dir[tid]);
    }
    __syncthreads();
    if (tid < 36) {
        double a = 0.0;
        for (int b = 1; b < Q; ++b) a += s_dir[b][tid];
        S.zeta[tid] = a;
    }
    if (tid >= 64 && tid < 64 + Q) {
        const int b = tid - 64;
        for (int k = 0; k < 10; ++k) S.lm[b][k] = s_lm[b][k];
        for (int k = 0; k < 4; ++k) S.slip[b][k] = (long long)s_slip[b][k];
    }
    if (tid == 96) {
        const int n = s_count;
        if (n > P.pk[p].list_cap) atomicOr(P.status, ST_CAPACITY);
        *P.pk[p].list_count = n < P.pk[p].list_cap ? n : P.pk[p].list_cap;
    }
}

// Boundary links of one particle's current map, compacted in (row, direction,
// x) order: a block-wide count, an exclusive scan, then the writes.
__global__ void __launch_bounds__(PBLOCK) links_kernel(const PartDev* pd, const uint64_t* rows_all,
                                                      const BoxDev* boxes, int p, int* out, int cap,
                                                      int* count)
{
    const PartDev& S = pd[p];
    const BoxDev& B = boxes[S.box];
    const uint64_t* rows = rows_all + ((long long)p * 2 + S.slot) * (MAXS * MAXS);
    const int Sd = S.S;
    const uint64_t maskS = Sd >= 64 ? ~0ull : ((1ull << Sd) - 1ull);
    const int items = Sd * Sd * 18;
    const int per = (items + PBLOCK - 1) / PBLOCK;
    const int i0 = threadIdx.x * per, i1 = min(items, i0 + per);
    __shared__ int s_cnt[PBLOCK];
    for (int pass = 0; pass < 2; ++pass) {
        int base = 0;
        if (pass == 1) {
            base = s_cnt[threadIdx.x];
        }
        int cnt = 0;
        for (int it = i0; it < i1; ++it) {
            const int r = it / 18, b = 1 + it % 18;
            const int my = r % Sd, mz = r / Sd;
            const int Yu = S.o[1] + my;
            if (B.walls && (Yu <= 0 || Yu >= B.ny - 1)) continue;
            const int ny2 = my + cy_of(b), nz2 = mz + cz_of(b);
            if (ny2 < 0 || ny2 >= Sd || nz2 < 0 || nz2 >= Sd) continue;
            const uint64_t nb = rows[nz2 * Sd + ny2];
            const int cbx = cx_of(b);
            const uint64_t sh = cbx == 1 ? (nb >> 1) : (cbx == -1 ? (nb << 1) : nb);
            uint64_t L = ~rows[r] & sh & maskS;
            while (L) {
                const int mx = __ffsll((long long)L) - 1;
                L &= L - 1;
                if (pass == 1) {
                    const int k = base + cnt;
                    if (k < cap) {
                        const int X = wrapi(S.o[0] + mx, B.nx), Y = wrapi(Yu, B.ny), Z = wrapi(S.o[2] + mz, B.nz);
                        out[2 * k] = (Z * B.ny + Y) * B.nx + X;
                        out[2 * k + 1] = b;
                    }
                }
                ++cnt;
            }
        }
        if (pass == 0) {
            s_cnt[threadIdx.x] = cnt;
            __syncthreads();
            if (threadIdx.x == 0) {
                int run = 0;
                for (int t = 0; t < PBLOCK; ++t) { const int c = s_cnt[t]; s_cnt[t] = run; run += c; }
                *count = run;
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------------------
// Boundary links of one spheroid without any allocation (lb_links_noalloc).
//
// The occupancy bitmap and the link counter live in this file-scope scratch,
// shared by every call on a device and kept from one call to the next; each
// call clears the part it uses first.  Calls that overlap on the GPU race on it.
constexpr int NOALLOC_WORDS = MAXS * MAXS;                  // 32 KiB of bitmap rows
static __device__ __align__(256) uint64_t g_noalloc_scratch[NOALLOC_WORDS + 32];

struct NoallocArgs {
    double semi[3], q[4], x[3];
    int nx, ny, nz, walls, S, h, cap;
    int* pairs;
    int* count;
};

__global__ void __launch_bounds__(PBLOCK) links_noalloc_kernel(const NoallocArgs a, uint64_t* scratch)
{
    uint64_t* rows = scratch;
    int* cnt = reinterpret_cast<int*>(scratch + NOALLOC_WORDS);
    const int tid = threadIdx.x, Sd = a.S;
    __shared__ double s_A[9], s_xc[3];
    __shared__ float s_e[3][3], s_inv[3], s_ro[3];
    __shared__ int s_o[3];
    for (int r = tid; r < Sd * Sd; r += PBLOCK) rows[r] = 0ull;
    if (tid == 0) {
        *cnt = 0;
        double e[3][3];
        canon_shape(a.semi, a.q, s_A, e);
        for (int k = 0; k < 3; ++k) {
            s_o[k] = (int)floor(a.x[k]) - a.h;
            s_xc[k] = a.x[k];
            s_ro[k] = (float)((double)s_o[k] - a.x[k]);
            s_inv[k] = (float)(1.0 / (a.semi[k] * a.semi[k]));
            for (int j = 0; j < 3; ++j) s_e[k][j] = (float)e[k][j];
        }
    }
    __syncthreads();
    const bool py = !a.walls;
    // occupancy: FP32 test away from the surface, exact FP64 test near it
    for (int n = tid; n < Sd * Sd * Sd; n += PBLOCK) {
        const int mx = n % Sd, my = (n / Sd) % Sd, mz = n / (Sd * Sd);
        const float dx = s_ro[0] + mx, dy = s_ro[1] + my, dz = s_ro[2] + mz;
        float v = 0.0f;
        for (int m = 0; m < 3; ++m) {
            const float t = s_e[m][0] * dx + s_e[m][1] * dy + s_e[m][2] * dz;
            v += t * t * s_inv[m];
        }
        bool solid;
        if (fabsf(v - 1.0f) > 1e-4f) {
            solid = v < 1.0f;
        } else {
            solid = canon_value(s_A, s_xc, wrapi(s_o[0] + mx, a.nx), wrapi(s_o[1] + my, a.ny), wrapi(s_o[2] + mz, a.nz),
                                a.nx, a.ny, a.nz, py) <= 1.0;
        }
        const int Yu = s_o[1] + my;
        if (solid && !(a.walls && (Yu <= 0 || Yu >= a.ny - 1)))
            atomicOr(reinterpret_cast<unsigned long long*>(rows + mz * Sd + my), 1ull << mx);
    }
    __syncthreads();
    // links (x fluid, x + c_b solid), written as (node index, direction) pairs
    const uint64_t maskS = Sd >= 64 ? ~0ull : ((1ull << Sd) - 1ull);
    for (int it = tid; it < Sd * Sd * 18; it += PBLOCK) {
        const int r = it / 18, b = 1 + it % 18;
        const int my = r % Sd, mz = r / Sd;
        const int Yu = s_o[1] + my;
        if (a.walls && (Yu <= 0 || Yu >= a.ny - 1)) continue;
        const int ny2 = my + cy_of(b), nz2 = mz + cz_of(b);
        if (ny2 < 0 || ny2 >= Sd || nz2 < 0 || nz2 >= Sd) continue;
        const uint64_t nb = rows[nz2 * Sd + ny2];
        const uint64_t sh = cx_of(b) == 1 ? (nb >> 1) : (cx_of(b) == -1 ? (nb << 1) : nb);
        uint64_t L = ~rows[r] & sh & maskS;
        while (L) {
            const int mx = __ffsll((long long)L) - 1;
            L &= L - 1;
            const int k = atomicAdd(cnt, 1);
            if (k < a.cap) {
                const int X = wrapi(s_o[0] + mx, a.nx), Y = wrapi(Yu, a.ny), Z = wrapi(s_o[2] + mz, a.nz);
                a.pairs[2 * k] = (Z * a.ny + Y) * a.nx + X;
                a.pairs[2 * k + 1] = b;
            }
        }
    }
    __syncthreads();
    if (tid == 0) *a.count = *cnt;
}

}  // namespace lbsph

// Device address of the scratch array, looked up once per device (host code
// cannot use the array's name as an address).
static std::mutex g_noalloc_mutex;
static void* g_noalloc_ptr[256];

extern "C" lb_status lb_links_noalloc(const double* semi, const double* q, const double* x, int32_t nx, int32_t ny,
                                      int32_t nz, int32_t walls, int32_t* pairs_dev, int32_t cap, int32_t* count_dev,
                                      void* stream)
{
    using namespace lbsph;
    if (!semi || !q || !x || !pairs_dev || !count_dev || cap < 0) return LB_EINVAL;
    if (nx < 4 || ny < 4 || nz < 4 || (walls && ny < 5)) return LB_EINVAL;
    const double qn = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    if (std::fabs(qn - 1.0) > 1e-6) return LB_EINVAL;
    double m = 0.0;
    for (int k = 0; k < 3; ++k) {
        if (!(semi[k] > 0.0)) return LB_EINVAL;
        m = std::fmax(m, semi[k]);
    }
    NoallocArgs a{};
    a.h = (int)std::ceil(m) + CUBE_MARGIN;
    a.S = 2 * a.h + 2;
    if (a.S > MAXS || a.S > nx || a.S > nz || (!walls && a.S > ny)) return LB_ECAPACITY;
    for (int k = 0; k < 3; ++k) { a.semi[k] = semi[k]; a.x[k] = x[k]; }
    for (int k = 0; k < 4; ++k) a.q[k] = q[k] / qn;
    a.nx = nx; a.ny = ny; a.nz = nz; a.walls = walls; a.cap = cap;
    a.pairs = pairs_dev;
    a.count = count_dev;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return LB_ECUDA;
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
                cudaGetLastError();
                return LB_ECUDA;
            }
            g_noalloc_ptr[dev] = p;
        }
        scratch = g_noalloc_ptr[dev];
    }
    links_noalloc_kernel<<<1, PBLOCK, 0, static_cast<cudaStream_t>(stream)>>>(a, static_cast<uint64_t*>(scratch));
    return cudaGetLastError() == cudaSuccess ? LB_OK : LB_ECUDA;
}

namespace lbsph {

cudaError_t launch_particles(const PParams& p, cudaStream_t s)
{
    if (p.np <= 0) return cudaSuccess;
    particle_crit_kernel<<<p.np, CBLOCK, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_particles_aux(const PParams& p, cudaStream_t s)
{
    if (p.np <= 0) return cudaSuccess;
    const size_t smem = 2ull * p.smax * p.smax * sizeof(uint64_t);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(particle_aux_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    particle_aux_kernel<<<p.np, PBLOCK, smem, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_links(const PartDev* pd, const uint64_t* rows, const BoxDev* boxes, int p, int* out,
                         int cap, int* count, cudaStream_t s)
{
    links_kernel<<<1, PBLOCK, 0, s>>>(pd, rows, boxes, p, out, cap, count);
    return cudaGetLastError();
}

}  // namespace lbsph
