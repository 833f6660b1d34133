/*
 * FP64 CPU oracle: lattice Boltzmann D3Q19 (or D3Q27) fluid coupled to rigid spheroids
 * by link bounce-back and an implicit velocity / quaternion update.
 *
 * TEST INFRASTRUCTURE ONLY (tests/, __graft_entry__.smoke(), bench.py's
 * cpu_baseline leg).  Plain, slow, double precision, no blocking or fusion:
 * one function per step of the paper's Appendix, called in the Appendix
 * order by orc_step().  Compile with -ffp-contract=off so that the inside
 * test (Eq. ellipsoidsurface) is evaluated with exactly the stated operation
 * order.
 *
 * Readings of points the paper leaves open:
 *   - lattice: D3Q19 textbook set, weights 1/3, 1/18, 1/36, c_s^2 = 1/3 (Sec. II.A);
 *     compiled with -DORC_D3Q27 (liboracle27.so): the D3Q27 set the paper compares it
 *     with (Sec. III.A), all c in {-1,0,1}^3, weights 8/27, 2/27, 1/54, 1/216 for
 *     |c|^2 = 0, 1, 2, 3, the same c_s^2 = 1/3; every step below is written for
 *     either set;
 *   - collision: BGK with the quadratic equilibrium of Eq. 4 (Sec. II.A);
 *   - body force: Guo forcing, u = (sum f c + g/2)/rho, applied on fluid nodes;
 *     with counter_force the fluid gets g = -sum(F_ext)/N_fluid;
 *   - rho_0 in the bounce-back term is the box's mean density rho0 (Eq. fb);
 *   - inside test: solid iff (x-x_c)^T A (x-x_c) <= 1 with minimum image,
 *     A = sum_m e_m e_m^T / s_m^2, e_m the rotated body axes (Eq. ellipsoidsurface,
 *     Eq. vectrotn), evaluated in the fixed order of orc_inside_value();
 *   - r_b = x_b - x_c with x_b = x + c_b/2, minimum image (Eq. ub);
 *   - external force and torque enter the right-hand sides of Eq. Fdiscrete /
 *     Eq. Tdiscrete;
 *   - dI/dt at time t uses qdot = Omega(t) q(t)/2 (Eq. qevolution); the
 *     optional predictor-corrector (didt_mode 2) re-solves with I(t+1) of the
 *     orientation the first solve predicts;
 *   - the initial quaternion is divided by its norm, sqrt of the sum of the
 *     squares of q0..q3 taken in that order (Eq. vectrotn assumes |q| = 1);
 *   - covered / uncovered nodes at the remap (Appendix step 8): a covered node's
 *     momentum and angular momentum go to the particle's next solve; an
 *     uncovered node gets f_eq(rho0, U + Omega x r) and that momentum is taken
 *     from the particle; the net fluid mass removed by the remap of iteration t is
 *     returned at the collision of iteration t+2, spread over every fluid node as
 *     w_i dm / N_fluid (no momentum, so no kick on the particle);
 *   - squirmer slip u_s (Eq. squirmer) evaluated at x_b in body coordinates and
 *     added to u_b (Eq. ubsquirmer); its bounce-back term is velocity independent
 *     and so belongs to F_0 / T_0.
 */
#include "lb_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#ifdef ORC_D3Q27
#define Q 27
#define QMAXC2 3
#else
#define Q 19
#define QMAXC2 2
#endif

/* ------------------------------------------------------------------------- */
/* Lattice: D3Q19 enumerated as all c in {-1,0,1}^3 with |c|^2 <= 2, z slowest
 * (D3Q27: every c in {-1,0,1}^3, same order). */
static int C[Q][3];
static double Wt[Q];
static int OPP[Q];
static int lattice_ready = 0;

static void lattice_init(void)
{
    if (lattice_ready) return;
    int n = 0;
    for (int cz = -1; cz <= 1; ++cz)
        for (int cy = -1; cy <= 1; ++cy)
            for (int cx = -1; cx <= 1; ++cx) {
                int m = cx * cx + cy * cy + cz * cz;
                if (m > QMAXC2) continue;
                C[n][0] = cx; C[n][1] = cy; C[n][2] = cz;
#ifdef ORC_D3Q27
                Wt[n] = (m == 0) ? 8.0 / 27.0 : (m == 1) ? 2.0 / 27.0 : (m == 2) ? 1.0 / 54.0 : 1.0 / 216.0;
#else
                Wt[n] = (m == 0) ? 1.0 / 3.0 : (m == 1) ? 1.0 / 18.0 : 1.0 / 36.0;
#endif
                ++n;
            }
    for (int i = 0; i < Q; ++i)
        for (int j = 0; j < Q; ++j)
            if (C[j][0] == -C[i][0] && C[j][1] == -C[i][1] && C[j][2] == -C[i][2]) OPP[i] = j;
    lattice_ready = 1;
}

int orc_q(void) { return Q; }

void orc_lattice(int c[][3], double w[])
{
    lattice_init();
    memcpy(c, C, sizeof(C));
    memcpy(w, Wt, sizeof(Wt));
}

/* ------------------------------------------------------------------------- */
typedef struct {
    double semi[3], x[3], q[4], U[3], Om[3];
    double density, F_ext[3], T_ext[3], B1, B2;
    double M, Ibody[3];
    int nlink, caplink;
    int* link_node;
    int* link_dir;
    double zeta[6][6];
    double dP[3], dL[3], dm;     /* pending terms from the last remap     */
    double dm_return;            /* mass of the remap before, returned at the next collision */
    double Iprev[9];
    double F0[3], T0[3], F[3], T[3];
    double FL[3];                /* lubrication force of this iteration (part of F) */
} part_t;

struct orc_sim {
    int nx, ny, nz, N;
    double tau, rho0, gbody[3];
    int counter, walls, didt_mode, collision;
    double lub_cut;
    double uw_lo[3], uw_hi[3];
    double *f, *fpost, *fnext;
    int *owner, *owner_new;
    int* nb;                     /* nb[n*Q + i] = index of node x + c_i (periodic addressing) */
    unsigned* linkmask;          /* per node: bit b set if x + c_b is a particle node */
    int np;
    part_t* P;
    long t;
    int nthreads;
    int nfluid;
};

static inline int node_index(const orc_sim* s, int x, int y, int z)
{
    return (z * s->ny + y) * s->nx + x;
}
static inline int wrap(int a, int L) { a %= L; return a < 0 ? a + L : a; }

static void node_coords(const orc_sim* s, int n, int X[3])
{
    X[0] = n % s->nx;
    X[1] = (n / s->nx) % s->ny;
    X[2] = n / (s->nx * s->ny);
}

/* neighbour x + c_i with periodic addressing on every axis; walls are solid
 * nodes of the owner map, so they stop any crossing in y. */
static int neighbour_of(const orc_sim* s, int n, int i)
{
    int X[3];
    node_coords(s, n, X);
    return node_index(s, wrap(X[0] + C[i][0], s->nx), wrap(X[1] + C[i][1], s->ny),
                      wrap(X[2] + C[i][2], s->nz));
}

static inline int neighbour(const orc_sim* s, int n, int i) { return s->nb[(size_t)n * Q + i]; }

/* minimum image of a displacement along one axis (periodic axes only) */
static double min_image(double d, int L, int periodic)
{
    if (!periodic) return d;
    return d - (double)L * floor(d / (double)L + 0.5);
}

static void cross3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* ------------------------------------------------------------------------- */
/* Quaternion algebra (Sec. II.C).  Hamilton product. */
void orc_quat_mul(const double a[4], const double b[4], double o[4])
{
    double r0 = a[0] * b[0] - (a[1] * b[1] + a[2] * b[2] + a[3] * b[3]);
    double v[3], c[3];
    cross3(a + 1, b + 1, c);
    for (int k = 0; k < 3; ++k) v[k] = a[0] * b[k + 1] + b[0] * a[k + 1] + c[k];
    o[0] = r0; o[1] = v[0]; o[2] = v[1]; o[3] = v[2];
}

/* Eq. vectrotn: s' = (2 q0^2 - 1) s + 2 (q.s) q + 2 q0 q x s, in this order. */
void orc_rotate(const double q[4], const double s[3], double o[3])
{
    double a = 2.0 * (q[0] * q[0]) - 1.0;
    double qs = (q[1] * s[0] + q[2] * s[1]) + q[3] * s[2];
    double cx = q[2] * s[2] - q[3] * s[1];
    double cy = q[3] * s[0] - q[1] * s[2];
    double cz = q[1] * s[1] - q[2] * s[0];
    double tqs = 2.0 * qs, tq0 = 2.0 * q[0];
    o[0] = (a * s[0] + tqs * q[1]) + tq0 * cx;
    o[1] = (a * s[1] + tqs * q[2]) + tq0 * cy;
    o[2] = (a * s[2] + tqs * q[3]) + tq0 * cz;
}

/* Apply p -> a p b to every column p of a 4x4 matrix (columns are quaternions). */
static void quat_cols(const double a[4], const double M[4][4], const double b[4], double O[4][4])
{
    for (int j = 0; j < 4; ++j) {
        double col[4], t[4], r[4];
        for (int i = 0; i < 4; ++i) col[i] = M[i][j];
        orc_quat_mul(a, col, t);
        orc_quat_mul(t, b, r);
        for (int i = 0; i < 4; ++i) O[i][j] = r[i];
    }
}

static void transpose4(const double M[4][4], double O[4][4])
{
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) O[j][i] = M[i][j];
}

/* (a (b I c)^T d)^T for the pure-quaternion inertia matrix I (Eq. Irot form) */
static void irot_form(const double a[4], const double b[4], const double c[4], const double d[4],
                      const double I4[4][4], double O[4][4])
{
    double X[4][4], XT[4][4], Y[4][4];
    quat_cols(b, I4, c, X);
    transpose4(X, XT);
    quat_cols(a, XT, d, Y);
    transpose4(Y, O);
}

static void pure_inertia(const double Ib[3], double I4[4][4])
{
    memset(I4, 0, sizeof(double) * 16);
    I4[1][1] = Ib[0]; I4[2][2] = Ib[1]; I4[3][3] = Ib[2];
}

static void conj4(const double q[4], double o[4])
{
    o[0] = q[0]; o[1] = -q[1]; o[2] = -q[2]; o[3] = -q[3];
}

/* Eq. Irot: I' = (q (q I q^-1)^T q^-1)^T, lab-frame inertia from q. */
void orc_inertia_lab(const double q[4], const double Ib[3], double out[9])
{
    double I4[4][4], qi[4], O[4][4];
    pure_inertia(Ib, I4);
    conj4(q, qi);
    irot_form(q, q, qi, qi, I4, O);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) out[i * 3 + j] = O[i + 1][j + 1];
}

/* Eq. Irotdiff with qdot from Eq. qevolution (qdot = Omega q / 2, Omega pure).
 * For a unit quaternion d(q^-1)/dt = conj(qdot). */
void orc_inertia_rate(const double q[4], const double Om[3], const double Ib[3], double out[9])
{
    double I4[4][4], qi[4], qd[4], qdi[4], Omq[4] = {0.0, Om[0], Om[1], Om[2]};
    double T1[4][4], T2[4][4], T3[4][4], T4[4][4];
    pure_inertia(Ib, I4);
    conj4(q, qi);
    orc_quat_mul(Omq, q, qd);
    for (int k = 0; k < 4; ++k) qd[k] *= 0.5;
    conj4(qd, qdi);
    irot_form(qd, q, qi, qi, I4, T1);
    irot_form(q, qd, qi, qi, I4, T2);
    irot_form(q, q, qdi, qi, I4, T3);
    irot_form(q, q, qi, qdi, I4, T4);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            out[i * 3 + j] = T1[i + 1][j + 1] + T2[i + 1][j + 1] + T3[i + 1][j + 1] + T4[i + 1][j + 1];
}

/* Eq. qnplus0 / qnplus1: q(t+dt) = [cos(|W|/2), sin(|W|/2) W/|W|] q(t), dt = 1. */
void orc_quat_step(const double q[4], const double W[3], double out[4])
{
    double n = sqrt(W[0] * W[0] + W[1] * W[1] + W[2] * W[2]);
    double qt[4];
    if (n < 1e-300) {
        qt[0] = 1.0; qt[1] = qt[2] = qt[3] = 0.0;
    } else {
        double sn = sin(0.5 * n) / n;
        qt[0] = cos(0.5 * n); qt[1] = sn * W[0]; qt[2] = sn * W[1]; qt[3] = sn * W[2];
    }
    orc_quat_mul(qt, q, out);
}

/* Gaussian elimination with partial pivoting (Sec. II.C, "solved using the
 * Gaussian elimination method").  A is row-major n x n.  Returns 0 on success. */
int orc_gauss_solve(int n, const double* A, const double* b, double* x)
{
    double M[8][9];
    if (n > 8) return -1;
    for (int i = 0; i < n; ++i) {
        for (int j = 0; j < n; ++j) M[i][j] = A[i * n + j];
        M[i][n] = b[i];
    }
    for (int k = 0; k < n; ++k) {
        int piv = k;
        for (int i = k + 1; i < n; ++i)
            if (fabs(M[i][k]) > fabs(M[piv][k])) piv = i;
        if (M[piv][k] == 0.0) return -2;
        if (piv != k)
            for (int j = 0; j <= n; ++j) { double t = M[k][j]; M[k][j] = M[piv][j]; M[piv][j] = t; }
        for (int i = k + 1; i < n; ++i) {
            double l = M[i][k] / M[k][k];
            for (int j = k; j <= n; ++j) M[i][j] -= l * M[k][j];
        }
    }
    for (int i = n - 1; i >= 0; --i) {
        double s = M[i][n];
        for (int j = i + 1; j < n; ++j) s -= M[i][j] * x[j];
        x[i] = s / M[i][i];
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Eq. ellipsoidsurface: value of (x - x_c)^T A (x - x_c) at lattice node X.
 * A = sum_m e_m e_m^T / s_m^2 with e_m the body axes rotated by Eq. vectrotn.
 * Fixed evaluation order; a node is solid iff the value is <= 1. */
static void shape_matrix(const double semi[3], const double q[4], double A[3][3])
{
    double e[3][3], inv[3];
    for (int m = 0; m < 3; ++m) {
        double u[3] = {0.0, 0.0, 0.0};
        u[m] = 1.0;
        orc_rotate(q, u, e[m]);
        inv[m] = 1.0 / (semi[m] * semi[m]);
    }
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k)
            A[j][k] = ((e[0][j] * e[0][k]) * inv[0] + (e[1][j] * e[1][k]) * inv[1]) +
                      (e[2][j] * e[2][k]) * inv[2];
}

static double quad_form(const double A[3][3], const double d[3])
{
    double Ad[3];
    for (int j = 0; j < 3; ++j) Ad[j] = (A[j][0] * d[0] + A[j][1] * d[1]) + A[j][2] * d[2];
    return (d[0] * Ad[0] + d[1] * Ad[1]) + d[2] * Ad[2];
}

double orc_inside_value(const double semi[3], const double q[4], const double xc[3],
                        const int X[3], const int L[3], const int periodic[3])
{
    double A[3][3], d[3];
    shape_matrix(semi, q, A);
    for (int k = 0; k < 3; ++k) d[k] = min_image((double)X[k] - xc[k], L[k], periodic[k]);
    return quad_form(A, d);
}

/* ------------------------------------------------------------------------- */
/* Eq. 4: quadratic equilibrium. */
static double feq_i(int i, double rho, const double u[3])
{
    double cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return rho * Wt[i] * (1.0 + 3.0 * cu + 4.5 * cu * cu - 1.5 * uu);
}

void orc_feq(double rho, const double u[3], double out[])
{
    lattice_init();
    for (int i = 0; i < Q; ++i) out[i] = feq_i(i, rho, u);
}

/* Eq. squirmer with the surface tangent s and spheroidal coordinate zeta of
 * Sec. III.D, evaluated at r = x_b - x_c in body coordinates; e = body x axis. */
void orc_squirmer_slip(const double semi[3], const double q[4], double B1, double B2,
                       const double r[3], double out[3])
{
    double ex[3] = {1.0, 0.0, 0.0}, e[3], rp[3];
    out[0] = out[1] = out[2] = 0.0;
    if (B1 == 0.0 && B2 == 0.0) return;
    orc_rotate(q, ex, e);
    double a = semi[0], b = semi[1];
    double zr = r[0] * e[0] + r[1] * e[1] + r[2] * e[2];
    for (int k = 0; k < 3; ++k) rp[k] = r[k] - zr * e[k];
    double rho = sqrt(rp[0] * rp[0] + rp[1] * rp[1] + rp[2] * rp[2]);
    if (rho < 1e-12) return;
    double z = zr > a ? a : (zr < -a ? -a : zr);
    double eps2 = 1.0 - (b * b) / (a * a);
    if (eps2 < 0.0) eps2 = 0.0;
    double eps = sqrt(eps2);
    double den = sqrt(a * a - eps2 * z * z);
    double s_e = -sqrt(a * a - z * z) / den;       /* coefficient of e      */
    double s_p = sqrt(1.0 - eps2) * z / den;       /* coefficient of e_perp */
    double zeta;
    if (eps < 1e-8) {
        zeta = zr / a;
    } else {
        double d1 = sqrt(rho * rho + (zr + a * eps) * (zr + a * eps));
        double d2 = sqrt(rho * rho + (zr - a * eps) * (zr - a * eps));
        zeta = (d1 - d2) / (2.0 * a * eps);
    }
    /* s.e = s_e since e_perp is orthogonal to e */
    double amp = -(B1 + B2 * zeta) * s_e;
    for (int k = 0; k < 3; ++k) out[k] = amp * (s_e * e[k] + s_p * rp[k] / rho);
}

/* ------------------------------------------------------------------------- */
static int periodic_axis(const orc_sim* s, int k) { return !(k == 1 && s->walls); }

static void body_force(const orc_sim* s, double g[3])
{
    for (int k = 0; k < 3; ++k) g[k] = s->gbody[k];
    if (s->counter && s->nfluid > 0) {
        for (int p = 0; p < s->np; ++p)
            for (int k = 0; k < 3; ++k) g[k] -= s->P[p].F_ext[k] / (double)s->nfluid;
    }
}

/* Appendix step 1: BGK collision (Eq. 3-4) with Guo forcing on every fluid node.
 * Before it, the mass removed by an earlier remap is put back uniformly:
 * f_i += w_i eps, eps = sum_p dm_return / N_fluid.
 *
 * collision == 1, the scheme the paper's simulations use (Sec. II.A: one
 * relaxation time for the non-conserved hydrodynamic modes, instantaneous
 * relaxation of the non-hydrodynamic ones): of the non-equilibrium part
 * f_i - feq_i only its projection on the hydrodynamic Hermite modes survives
 * the collision, relaxed by (1 - 1/tau); every other (ghost) mode is set to its
 * equilibrium value:
 *   f*_i = feq_i + (1 - 1/tau) w_i [c_i . j_neq / c_s^2
 *                                   + (c_i c_i - c_s^2 I) : Pi_neq / (2 c_s^4)] + S_i,
 * j_neq = sum_i c_i (f_i - feq_i) (= -g/2 with the half-force velocity),
 * Pi_neq = sum_i c_i c_i (f_i - feq_i), S_i the same Guo source (its moments
 * are of first and second order only).  Mass, momentum (+ g) and the relaxed
 * stress are those of BGK; at tau = 1 the two are the same. */
static void collide(orc_sim* s, const double g[3])
{
    const double tau = s->tau;
    double dm = 0.0;
    for (int p = 0; p < s->np; ++p) dm += s->P[p].dm_return;
    const double eps = s->nfluid > 0 ? dm / (double)s->nfluid : 0.0;
#pragma omp parallel for num_threads(s->nthreads) schedule(static)
    for (int n = 0; n < s->N; ++n) {
        if (s->owner[n] != 0) continue;
        double* f = s->f + (size_t)n * Q;
        if (eps != 0.0)
            for (int i = 0; i < Q; ++i) f[i] += Wt[i] * eps;
        double* fo = s->fpost + (size_t)n * Q;
        double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q; ++i) {
            rho += f[i];
            for (int k = 0; k < 3; ++k) m[k] += f[i] * C[i][k];
        }
        double u[3];
        for (int k = 0; k < 3; ++k) u[k] = (m[k] + 0.5 * g[k]) / rho;
        double Pn[3][3] = {{0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}, {0.0, 0.0, 0.0}}, jn[3] = {0.0, 0.0, 0.0};
        if (s->collision == 1)
            for (int i = 0; i < Q; ++i) {
                const double d = f[i] - feq_i(i, rho, u);
                for (int a = 0; a < 3; ++a) {
                    jn[a] += C[i][a] * d;
                    for (int b = 0; b < 3; ++b) Pn[a][b] += C[i][a] * C[i][b] * d;
                }
            }
        for (int i = 0; i < Q; ++i) {
            double cu = C[i][0] * u[0] + C[i][1] * u[1] + C[i][2] * u[2];
            double cg = C[i][0] * g[0] + C[i][1] * g[1] + C[i][2] * g[2];
            double ug = u[0] * g[0] + u[1] * g[1] + u[2] * g[2];
            double S = (1.0 - 0.5 / tau) * Wt[i] * (3.0 * (cg - ug) + 9.0 * cu * cg);
            if (s->collision == 1) {
                double QP = 0.0;        /* (c c - c_s^2 I) : Pi_neq */
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) QP += (C[i][a] * C[i][b] - (a == b ? 1.0 / 3.0 : 0.0)) * Pn[a][b];
                const double cj = C[i][0] * jn[0] + C[i][1] * jn[1] + C[i][2] * jn[2];
                fo[i] = feq_i(i, rho, u) + (1.0 - 1.0 / tau) * Wt[i] * (3.0 * cj + 4.5 * QP) + S;
            } else {
                fo[i] = f[i] - (f[i] - feq_i(i, rho, u)) / tau + S;
            }
        }
    }
}

/* Appendix step 2: stream from every fluid node to every fluid neighbour. */
static void stream(orc_sim* s)
{
    memset(s->fnext, 0, sizeof(double) * (size_t)s->N * Q);
#pragma omp parallel for num_threads(s->nthreads) schedule(static)
    for (int n = 0; n < s->N; ++n) {
        if (s->owner[n] != 0) continue;
        for (int i = 0; i < Q; ++i) {
            int m = neighbour(s, n, i);
            if (s->owner[m] == 0) s->fnext[(size_t)m * Q + i] = s->fpost[(size_t)n * Q + i];
        }
    }
}

/* r_b = x + c_b/2 - x_c, minimum image (Eq. ub). */
static void link_r(const orc_sim* s, const part_t* P, int node, int b, double r[3])
{
    int X[3], L[3] = {s->nx, s->ny, s->nz};
    node_coords(s, node, X);
    for (int k = 0; k < 3; ++k)
        r[k] = min_image(((double)X[k] + 0.5 * C[b][k]) - P->x[k], L[k], periodic_axis(s, k));
}

/* Appendix step 3: velocity-independent force and torque, Eq. F0 / Eq. T0,
 * from post-collision populations on the links, plus the squirmer slip term,
 * which is velocity independent as well. */
static void force0(orc_sim* s, part_t* P)
{
    for (int k = 0; k < 3; ++k) P->F0[k] = P->T0[k] = 0.0;
    for (int l = 0; l < P->nlink; ++l) {
        int n = P->link_node[l], b = P->link_dir[l];
        double r[3], us[3], cb[3] = {C[b][0], C[b][1], C[b][2]}, rxc[3];
        link_r(s, P, n, b, r);
        orc_squirmer_slip(P->semi, P->q, P->B1, P->B2, r, us);
        double usc = us[0] * cb[0] + us[1] * cb[1] + us[2] * cb[2];
        double a = 2.0 * s->fpost[(size_t)n * Q + b] - 6.0 * Wt[b] * s->rho0 * usc;
        cross3(r, cb, rxc);
        for (int k = 0; k < 3; ++k) {
            P->F0[k] += a * cb[k];
            P->T0[k] += a * rxc[k];
        }
    }
}

/* Lubrication correction (the Nguyen-Ladd correction the paper's method builds
 * on, Sec. II.B; the paper itself does not use it).  Readings:
 *   - gap and radii along the line of centres: n = d/|d|, d = minimum image of
 *     x_q - x_p; R(n) = (n^T A n)^(-1/2) is the body's centre-to-surface
 *     distance along n (A of Eq. ellipsoidsurface); h = |d| - R_p(n) - R_q(-n);
 *   - below the cut-off gap h_c the lattice no longer resolves the gap, and the
 *     missing normal squeeze force of two spheres of radii R_p, R_q is added:
 *     F_p = -6 pi mu R^2 (1/h - 1/h_c) (n . (U_p - U_q)) n, R = R_p R_q/(R_p + R_q),
 *     F_q = -F_p (no torque: the force acts along the line of centres);
 *   - h is clamped at H_MIN = 0.1 and the velocities are those of time t, so
 *     the force is explicit and exactly antisymmetric (combined momentum is
 *     conserved); its coefficient is capped at the reduced mass M_p M_q /
 *     (M_p + M_q), which stops the normal relative motion within one step
 *     (the largest coefficient an explicit update keeps stable). */
#define LUB_H_MIN 0.1

void orc_lubrication_pair(const double semi_p[3], const double q_p[4], const double x_p[3], const double U_p[3],
                          double M_p, const double semi_q[3], const double q_q[4], const double x_q[3],
                          const double U_q[3], double M_q, const int L[3], const int periodic[3], double mu,
                          double h_cut, double force_p[3], double* gap)
{
    double d[3], n[3], Ap[3][3], Aq[3][3];
    for (int k = 0; k < 3; ++k) d[k] = min_image(x_q[k] - x_p[k], L[k], periodic[k]);
    const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    force_p[0] = force_p[1] = force_p[2] = 0.0;
    for (int k = 0; k < 3; ++k) n[k] = d[k] / r;
    shape_matrix(semi_p, q_p, Ap);
    shape_matrix(semi_q, q_q, Aq);
    const double Rp = 1.0 / sqrt(quad_form(Ap, n)), Rq = 1.0 / sqrt(quad_form(Aq, n));
    const double h = r - Rp - Rq;
    *gap = h;
    if (!(h < h_cut)) return;
    const double hh = h > LUB_H_MIN ? h : LUB_H_MIN;
    const double R = Rp * Rq / (Rp + Rq);
    double k = 6.0 * M_PI * mu * R * R * (1.0 / hh - 1.0 / h_cut);
    const double kmax = M_p * M_q / (M_p + M_q);
    if (k > kmax) k = kmax;
    const double vn = n[0] * (U_p[0] - U_q[0]) + n[1] * (U_p[1] - U_q[1]) + n[2] * (U_p[2] - U_q[2]);
    for (int c = 0; c < 3; ++c) force_p[c] = -k * vn * n[c];
}

/* Lubrication forces of every pair of particles at time t (zero when off). */
static void lubrication(orc_sim* s)
{
    int L[3] = {s->nx, s->ny, s->nz}, per[3];
    for (int k = 0; k < 3; ++k) per[k] = periodic_axis(s, k);
    for (int p = 0; p < s->np; ++p) s->P[p].FL[0] = s->P[p].FL[1] = s->P[p].FL[2] = 0.0;
    if (!(s->lub_cut > 0.0)) return;
    const double mu = s->rho0 * (s->tau - 0.5) / 3.0;
    for (int p = 0; p < s->np; ++p)
        for (int q = p + 1; q < s->np; ++q) {
            part_t *A = s->P + p, *B = s->P + q;
            double f[3], h;
            orc_lubrication_pair(A->semi, A->q, A->x, A->U, A->M, B->semi, B->q, B->x, B->U, B->M, L, per, mu,
                                 s->lub_cut, f, &h);
            for (int k = 0; k < 3; ++k) { A->FL[k] += f[k]; B->FL[k] -= f[k]; }
        }
}

/* Appendix steps 4-5 for one body: inertia (Eq. Irot) and the implicit solve of
 * Eq. Fdiscrete / Eq. Tdiscrete (dt = 1) for U(t+1), Omega(t+1), given the drag
 * matrix zeta and the velocity-independent forces rF = F0 + F_ext + dP,
 * rT = T0 + T_ext + dL.  The rotational equation needs I(t+1):
 *   mode 0: I(t) + dI/dt, dI/dt of Eq. Irotdiff at time t;
 *   mode 1: I(t) + (I(t) - I(t-1)) (finite difference, Iprev = I(t-1));
 *   mode 2: predictor-corrector (Sec. II.D names it as the refinement of the
 *           Eq. Irotdiff step): the mode-0 solution predicts Omega(t+1), hence
 *           the orientation q_p = qnplus(q, (Omega(t) + Omega_p)/2) of
 *           Eq. qnplus0-1, and the system is solved again with
 *           I(t+1) = I(q_p) of Eq. Irot.
 * The right-hand side is the same in every mode: M U(t) + rF and
 * I(t) Omega(t) + rT.  Returns 0, or 1 if a pivot vanishes. */
static int solve_body(double M, const double Ib[3], const double q[4], const double U[3], const double Om[3],
                      const double zeta[6][6], const double rF[3], const double rT[3], const double Iprev[9],
                      int mode, double Unew[3], double Wnew[3], double Inow[9])
{
    double dI[9], A[36], rhs[6], x6[6];
    orc_inertia_lab(q, Ib, Inow);
    if (mode == 1) {
        for (int k = 0; k < 9; ++k) dI[k] = Inow[k] - Iprev[k];
    } else {
        orc_inertia_rate(q, Om, Ib, dI);
    }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) A[i * 6 + j] = zeta[i][j];
    for (int k = 0; k < 3; ++k) A[k * 6 + k] += M;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) A[(i + 3) * 6 + (j + 3)] += Inow[i * 3 + j] + dI[i * 3 + j];
    for (int k = 0; k < 3; ++k) {
        rhs[k] = M * U[k] + rF[k];
        double IW = Inow[k * 3 + 0] * Om[0] + Inow[k * 3 + 1] * Om[1] + Inow[k * 3 + 2] * Om[2];
        rhs[k + 3] = IW + rT[k];
    }
    if (orc_gauss_solve(6, A, rhs, x6) != 0) return 1;
    if (mode == 2) {
        /* corrector: I(t+1) from the predicted orientation */
        double Wm[3], qp[4], Ip[9];
        for (int k = 0; k < 3; ++k) Wm[k] = 0.5 * (Om[k] + x6[k + 3]);
        orc_quat_step(q, Wm, qp);
        orc_inertia_lab(qp, Ib, Ip);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) A[(i + 3) * 6 + (j + 3)] = zeta[i + 3][j + 3] + Ip[i * 3 + j];
        if (orc_gauss_solve(6, A, rhs, x6) != 0) return 1;
    }
    for (int k = 0; k < 3; ++k) { Unew[k] = x6[k]; Wnew[k] = x6[k + 3]; }
    return 0;
}

int orc_rigid_solve(double M, const double Ib[3], const double q[4], const double U[3], const double Om[3],
                    const double zeta36[36], const double rF[3], const double rT[3], const double Iprev[9], int mode,
                    double Unew[3], double Wnew[3])
{
    double Z[6][6], Inow[9];
    memcpy(Z, zeta36, sizeof(Z));
    return solve_body(M, Ib, q, U, Om, Z, rF, rT, Iprev, mode, Unew, Wnew, Inow);
}

/* Appendix steps 4-5 for particle P, then F and T of Eq. Fsplit / Eq. Tsplit. */
static int solve_velocities(orc_sim* s, part_t* P, double Unew[3], double Wnew[3], double Inow[9])
{
    double rF[3], rT[3];
    for (int k = 0; k < 3; ++k) {
        rF[k] = P->F0[k] + P->FL[k] + P->F_ext[k] + P->dP[k];
        rT[k] = P->T0[k] + P->T_ext[k] + P->dL[k];
    }
    if (solve_body(P->M, P->Ibody, P->q, P->U, P->Om, P->zeta, rF, rT, P->Iprev, s->didt_mode, Unew, Wnew, Inow))
        return 1;
    for (int k = 0; k < 3; ++k) {
        double zu = 0.0, zw = 0.0, tu = 0.0, tw = 0.0;
        for (int j = 0; j < 3; ++j) {
            zu += P->zeta[k][j] * Unew[j];
            zw += P->zeta[k][j + 3] * Wnew[j];
            tu += P->zeta[k + 3][j] * Unew[j];
            tw += P->zeta[k + 3][j + 3] * Wnew[j];
        }
        P->F[k] = P->F0[k] - zu - zw + P->FL[k];
        P->T[k] = P->T0[k] - tu - tw;
    }
    return 0;
}

/* Appendix step 6: mid-link bounce-back with u_b = U + Omega x r_b (+ u_s),
 * Eq. fb / Eq. ub / Eq. ubsquirmer, using the new velocities; walls likewise
 * with their own velocity. */
static void bounce_back(orc_sim* s)
{
    for (int p = 0; p < s->np; ++p) {
        part_t* P = s->P + p;
        for (int l = 0; l < P->nlink; ++l) {
            int n = P->link_node[l], b = P->link_dir[l];
            double r[3], us[3], wr[3], ub[3];
            link_r(s, P, n, b, r);
            orc_squirmer_slip(P->semi, P->q, P->B1, P->B2, r, us);
            cross3(P->Om, r, wr);
            for (int k = 0; k < 3; ++k) ub[k] = P->U[k] + wr[k] + us[k];
            double ubc = ub[0] * C[b][0] + ub[1] * C[b][1] + ub[2] * C[b][2];
            s->fnext[(size_t)n * Q + OPP[b]] =
                s->fpost[(size_t)n * Q + b] - 6.0 * Wt[b] * s->rho0 * ubc;
        }
    }
    if (!s->walls) return;
    for (int n = 0; n < s->N; ++n) {
        if (s->owner[n] != 0) continue;
        for (int b = 0; b < Q; ++b) {
            int m = neighbour(s, n, b);
            if (s->owner[m] != -1) continue;
            int X[3];
            node_coords(s, m, X);
            const double* uw = (X[1] == 0) ? s->uw_lo : s->uw_hi;
            double ubc = uw[0] * C[b][0] + uw[1] * C[b][1] + uw[2] * C[b][2];
            s->fnext[(size_t)n * Q + OPP[b]] = s->fpost[(size_t)n * Q + b] - 6.0 * Wt[b] * s->rho0 * ubc;
        }
    }
}

/* Appendix step 8 (map part): owner of every node from Eq. ellipsoidsurface.
 * Returns nonzero if two particles, or a particle and a wall, claim a node. */
static int build_owner(orc_sim* s, int* owner)
{
    int L[3] = {s->nx, s->ny, s->nz}, per[3];
    int bad = 0;
    double A[64][3][3];
    int npa = s->np < 64 ? s->np : 64;
    for (int k = 0; k < 3; ++k) per[k] = periodic_axis(s, k);
    for (int p = 0; p < npa; ++p) shape_matrix(s->P[p].semi, s->P[p].q, A[p]);
#pragma omp parallel for num_threads(s->nthreads) schedule(static) reduction(| : bad)
    for (int n = 0; n < s->N; ++n) {
        int X[3];
        node_coords(s, n, X);
        int o = 0;
        if (s->walls && (X[1] == 0 || X[1] == s->ny - 1)) o = -1;
        for (int p = 0; p < s->np; ++p) {
            double d[3], v;
            for (int k = 0; k < 3; ++k) d[k] = min_image((double)X[k] - s->P[p].x[k], L[k], per[k]);
            if (p < 64) {
                v = quad_form(A[p], d);
            } else {
                v = orc_inside_value(s->P[p].semi, s->P[p].q, s->P[p].x, X, L, per);
            }
            if (v <= 1.0) {
                if (o != 0) bad = 1;
                o = p + 1;
            }
        }
        owner[n] = o;
    }
    return bad;
}

/* Appendix step 8 (re-initialisation part): covered and uncovered nodes. */
static void remap(orc_sim* s)
{
    int L[3] = {s->nx, s->ny, s->nz};
    for (int p = 0; p < s->np; ++p) {
        part_t* P = s->P + p;
        for (int k = 0; k < 3; ++k) P->dP[k] = P->dL[k] = 0.0;
        P->dm_return = P->dm;
        P->dm = 0.0;
    }
    for (int n = 0; n < s->N; ++n) {
        int o = s->owner[n], w = s->owner_new[n];
        if (o == w) continue;
        int X[3];
        node_coords(s, n, X);
        if (o == 0 && w > 0) {                 /* covered by particle w-1 */
            part_t* P = s->P + (w - 1);
            double* f = s->fnext + (size_t)n * Q;
            double rho = 0.0, j[3] = {0.0, 0.0, 0.0}, r[3], rxj[3];
            for (int i = 0; i < Q; ++i) {
                rho += f[i];
                for (int k = 0; k < 3; ++k) j[k] += f[i] * C[i][k];
            }
            for (int k = 0; k < 3; ++k) r[k] = min_image((double)X[k] - P->x[k], L[k], periodic_axis(s, k));
            cross3(r, j, rxj);
            for (int k = 0; k < 3; ++k) { P->dP[k] += j[k]; P->dL[k] += rxj[k]; }
            P->dm += rho;
            for (int i = 0; i < Q; ++i) f[i] = 0.0;
        } else if (o > 0 && w == 0) {          /* uncovered, was particle o-1 */
            part_t* P = s->P + (o - 1);
            double r[3], wr[3], ub[3], rxj[3], j[3];
            for (int k = 0; k < 3; ++k) r[k] = min_image((double)X[k] - P->x[k], L[k], periodic_axis(s, k));
            cross3(P->Om, r, wr);
            for (int k = 0; k < 3; ++k) ub[k] = P->U[k] + wr[k];
            for (int i = 0; i < Q; ++i) s->fnext[(size_t)n * Q + i] = feq_i(i, s->rho0, ub);
            for (int k = 0; k < 3; ++k) j[k] = s->rho0 * ub[k];
            cross3(r, j, rxj);
            for (int k = 0; k < 3; ++k) { P->dP[k] -= j[k]; P->dL[k] -= rxj[k]; }
            P->dm -= s->rho0;
        }
    }
}

/* Appendix step 9: boundary links of each particle and Eq. drag1 - Eq. drag4. */
static void links_and_drag(orc_sim* s)
{
#pragma omp parallel for num_threads(s->nthreads) schedule(static)
    for (int n = 0; n < s->N; ++n) {
        unsigned m = 0;
        if (s->owner[n] == 0)
            for (int b = 0; b < Q; ++b)
                if (s->owner[neighbour(s, n, b)] > 0) m |= 1u << b;
        s->linkmask[n] = m;
    }
    for (int p = 0; p < s->np; ++p) s->P[p].nlink = 0;
    for (int n = 0; n < s->N; ++n) {                 /* node order, then direction order */
        unsigned m = s->linkmask[n];
        for (int b = 0; m && b < Q; ++b) {
            if (!(m & (1u << b))) continue;
            part_t* P = s->P + (s->owner[neighbour(s, n, b)] - 1);
            if (P->nlink == P->caplink) {
                P->caplink = P->caplink ? 2 * P->caplink : 1024;
                P->link_node = (int*)realloc(P->link_node, sizeof(int) * P->caplink);
                P->link_dir = (int*)realloc(P->link_dir, sizeof(int) * P->caplink);
            }
            P->link_node[P->nlink] = n;
            P->link_dir[P->nlink] = b;
            P->nlink++;
        }
    }
    for (int p = 0; p < s->np; ++p) {
        part_t* P = s->P + p;
        double pref = 2.0 * s->rho0 / (1.0 / 3.0);
        memset(P->zeta, 0, sizeof(P->zeta));
        for (int l = 0; l < P->nlink; ++l) {
            int b = P->link_dir[l];
            double r[3], cb[3] = {C[b][0], C[b][1], C[b][2]}, rxc[3], v[6];
            link_r(s, P, P->link_node[l], b, r);
            cross3(r, cb, rxc);
            for (int k = 0; k < 3; ++k) { v[k] = cb[k]; v[k + 3] = rxc[k]; }
            for (int i = 0; i < 6; ++i)
                for (int j = 0; j < 6; ++j) P->zeta[i][j] += pref * Wt[b] * v[i] * v[j];
        }
    }
    int nf = 0;
    for (int n = 0; n < s->N; ++n) nf += (s->owner[n] == 0);
    s->nfluid = nf;
}

/* ------------------------------------------------------------------------- */
orc_sim* orc_create(const orc_box* box, const orc_particle* parts, int np, int nthreads)
{
    lattice_init();
    if (box->nx < 2 || box->ny < 2 || box->nz < 2 || !(box->tau > 0.5) || np < 0) return NULL;
    orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
    s->nx = box->nx; s->ny = box->ny; s->nz = box->nz;
    s->N = s->nx * s->ny * s->nz;
    s->tau = box->tau; s->rho0 = box->rho0;
    for (int k = 0; k < 3; ++k) {
        s->gbody[k] = box->body_force[k];
        s->uw_lo[k] = box->wall_u_lo[k];
        s->uw_hi[k] = box->wall_u_hi[k];
    }
    s->counter = box->counter_force; s->walls = box->walls; s->didt_mode = box->didt_mode;
    s->lub_cut = box->lub_cut;
    s->collision = box->collision;
    s->nthreads = nthreads > 0 ? nthreads : 1;
    size_t nf = (size_t)s->N * Q;
    s->f = (double*)calloc(nf, sizeof(double));
    s->fpost = (double*)calloc(nf, sizeof(double));
    s->fnext = (double*)calloc(nf, sizeof(double));
    s->owner = (int*)calloc(s->N, sizeof(int));
    s->owner_new = (int*)calloc(s->N, sizeof(int));
    s->nb = (int*)malloc(sizeof(int) * nf);
    s->linkmask = (unsigned*)calloc(s->N, sizeof(unsigned));
    for (int n = 0; n < s->N; ++n)
        for (int i = 0; i < Q; ++i) s->nb[(size_t)n * Q + i] = neighbour_of(s, n, i);
    s->np = np;
    s->P = (part_t*)calloc(np > 0 ? np : 1, sizeof(part_t));
    for (int p = 0; p < np; ++p) {
        part_t* P = s->P + p;
        const orc_particle* I = parts + p;
        memcpy(P->semi, I->semi, sizeof(P->semi));
        memcpy(P->x, I->x, sizeof(P->x));
        {   /* Eq. vectrotn needs a unit quaternion: q is normalised on input */
            const double qn = sqrt(I->q[0] * I->q[0] + I->q[1] * I->q[1] + I->q[2] * I->q[2] + I->q[3] * I->q[3]);
            for (int k = 0; k < 4; ++k) P->q[k] = I->q[k] / qn;
        }
        memcpy(P->U, I->U, sizeof(P->U));
        memcpy(P->Om, I->Om, sizeof(P->Om));
        memcpy(P->F_ext, I->F_ext, sizeof(P->F_ext));
        memcpy(P->T_ext, I->T_ext, sizeof(P->T_ext));
        P->density = I->density; P->B1 = I->B1; P->B2 = I->B2;
        double a = P->semi[0], b = P->semi[1], c = P->semi[2];
        P->M = P->density * 4.0 / 3.0 * M_PI * a * b * c;        /* continuum volume */
        P->Ibody[0] = P->M * (b * b + c * c) / 5.0;                /* Sec. II.D */
        P->Ibody[1] = P->M * (a * a + c * c) / 5.0;
        P->Ibody[2] = P->M * (a * a + b * b) / 5.0;
        orc_inertia_lab(P->q, P->Ibody, P->Iprev);
    }
    if (build_owner(s, s->owner)) { orc_destroy(s); return NULL; }
    for (int n = 0; n < s->N; ++n)
        if (s->owner[n] == 0)
            for (int i = 0; i < Q; ++i) s->f[(size_t)n * Q + i] = Wt[i] * s->rho0;  /* quiescent */
    links_and_drag(s);
    return s;
}

void orc_destroy(orc_sim* s)
{
    if (!s) return;
    for (int p = 0; p < s->np; ++p) { free(s->P[p].link_node); free(s->P[p].link_dir); }
    free(s->P); free(s->f); free(s->fpost); free(s->fnext); free(s->owner); free(s->owner_new);
    free(s->nb); free(s->linkmask);
    free(s);
}

long orc_time(const orc_sim* s) { return s->t; }

/* One iteration t -> t+1 in the order of the paper's Appendix. */
static int step_once(orc_sim* s)
{
    double g[3], Un[64][3], Wn[64][3], In[64][9], Umean[64][3], Wmean[64][3];
    if (s->np > 64) return 3;
    body_force(s, g);
    collide(s, g);                                               /* step 1 */
    stream(s);                                                   /* step 2 */
    for (int p = 0; p < s->np; ++p) force0(s, s->P + p);         /* step 3 */
    lubrication(s);                                              /* (f1) pair forces at t */
    for (int p = 0; p < s->np; ++p)                              /* steps 4-5 */
        if (solve_velocities(s, s->P + p, Un[p], Wn[p], In[p])) return 1;
    for (int p = 0; p < s->np; ++p) {
        part_t* P = s->P + p;
        for (int k = 0; k < 3; ++k) {
            Umean[p][k] = 0.5 * (P->U[k] + Un[p][k]);            /* Eq. posupdate */
            Wmean[p][k] = 0.5 * (P->Om[k] + Wn[p][k]);           /* mean angular velocity */
        }
        memcpy(P->Iprev, In[p], sizeof(P->Iprev));
        memcpy(P->U, Un[p], sizeof(P->U));
        memcpy(P->Om, Wn[p], sizeof(P->Om));
    }
    bounce_back(s);                          /* step 6: new U, Omega; x_c, q still at t */
    for (int p = 0; p < s->np; ++p) {        /* step 7: Eq. posupdate, Eq. qnplus0-1 */
        part_t* P = s->P + p;
        double qn[4];
        for (int k = 0; k < 3; ++k) P->x[k] += Umean[p][k];
        orc_quat_step(P->q, Wmean[p], qn);
        memcpy(P->q, qn, sizeof(qn));
    }
    if (build_owner(s, s->owner_new)) return 2;                  /* step 8 */
    remap(s);
    int* t = s->owner; s->owner = s->owner_new; s->owner_new = t;
    links_and_drag(s);                                           /* step 9 */
    double* tf = s->f; s->f = s->fnext; s->fnext = tf;
    s->t++;
    return 0;
}

int orc_step(orc_sim* s, int nsteps)
{
    for (int k = 0; k < nsteps; ++k) {
        int e = step_once(s);
        if (e) return e;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
void orc_get_f(const orc_sim* s, double* out)
{
    memcpy(out, s->f, sizeof(double) * (size_t)s->N * Q);
}

void orc_set_f(orc_sim* s, const double* in)
{
    memcpy(s->f, in, sizeof(double) * (size_t)s->N * Q);
    for (int n = 0; n < s->N; ++n)
        if (s->owner[n] != 0)
            for (int i = 0; i < Q; ++i) s->f[(size_t)n * Q + i] = 0.0;
}

void orc_get_moments(const orc_sim* s, double* rho, double* u)
{
    double g[3];
    body_force(s, g);
    for (int n = 0; n < s->N; ++n) {
        const double* f = s->f + (size_t)n * Q;
        if (s->owner[n] != 0) {
            rho[n] = 0.0;
            u[3 * n] = u[3 * n + 1] = u[3 * n + 2] = 0.0;
            continue;
        }
        double r = 0.0, m[3] = {0.0, 0.0, 0.0};
        for (int i = 0; i < Q; ++i) {
            r += f[i];
            for (int k = 0; k < 3; ++k) m[k] += f[i] * C[i][k];
        }
        rho[n] = r;
        for (int k = 0; k < 3; ++k) u[3 * n + k] = (m[k] + 0.5 * g[k]) / r;
    }
}

void orc_get_owner(const orc_sim* s, int* owner) { memcpy(owner, s->owner, sizeof(int) * s->N); }

double orc_total_fluid_mass(const orc_sim* s)
{
    double m = 0.0;
    for (size_t k = 0; k < (size_t)s->N * Q; ++k) m += s->f[k];
    return m;
}

void orc_total_fluid_momentum(const orc_sim* s, double out[3])
{
    out[0] = out[1] = out[2] = 0.0;
    for (int n = 0; n < s->N; ++n)
        for (int i = 0; i < Q; ++i)
            for (int k = 0; k < 3; ++k) out[k] += s->f[(size_t)n * Q + i] * C[i][k];
}

void orc_get_particle(const orc_sim* s, int p, double* out)
{
    const part_t* P = s->P + p;
    memcpy(out + 0, P->F0, 3 * sizeof(double));
    memcpy(out + 3, P->T0, 3 * sizeof(double));
    memcpy(out + 6, P->F, 3 * sizeof(double));
    memcpy(out + 9, P->T, 3 * sizeof(double));
    memcpy(out + 12, P->U, 3 * sizeof(double));
    memcpy(out + 15, P->Om, 3 * sizeof(double));
    memcpy(out + 18, P->x, 3 * sizeof(double));
    memcpy(out + 21, P->q, 4 * sizeof(double));
}

void orc_get_pending(const orc_sim* s, int p, double* out8)
{
    const part_t* P = s->P + p;
    memcpy(out8, P->dP, 3 * sizeof(double));
    memcpy(out8 + 3, P->dL, 3 * sizeof(double));
    out8[6] = P->dm;
    out8[7] = P->dm_return;
}

void orc_get_zeta(const orc_sim* s, int p, double* out36)
{
    memcpy(out36, s->P[p].zeta, 36 * sizeof(double));
}

int orc_get_links(const orc_sim* s, int p, int* node, int* cvec, int cap)
{
    const part_t* P = s->P + p;
    int n = P->nlink < cap ? P->nlink : cap;
    for (int l = 0; l < n; ++l) {
        node[l] = P->link_node[l];
        for (int k = 0; k < 3; ++k) cvec[3 * l + k] = C[P->link_dir[l]][k];
    }
    return P->nlink;
}

double orc_mass(const orc_sim* s, int p) { return s->P[p].M; }
