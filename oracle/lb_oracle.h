/*
 * FP64 CPU oracle for the lattice Boltzmann method for rigid spheroids
 * (Thampi, Stratford, Henrich, "Simulating dynamics of ellipsoidal particles
 * using lattice Boltzmann method").
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py may load this library.  It shares no code,
 * header, table or constant with the CUDA library: it has its own lattice
 * table (enumerated here in a different order), its own structs and its own
 * arithmetic.  It follows the paper's Appendix (algorithmic steps 1-10) in
 * that order, one function per step, in double precision.
 *
 * Parity status per function is stated in lb_oracle.c beside each function.
 */
#ifndef LB_ORACLE_H
#define LB_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_sim orc_sim;

/* Box description.  Walls (when walls != 0) are the solid planes y = 0 and
 * y = ny-1 moving with wall_u_lo / wall_u_hi; x and z stay periodic. */
typedef struct {
    int nx, ny, nz;
    double tau, rho0;
    double body_force[3];   /* uniform force density on every fluid node */
    int counter_force;      /* 1: fluid also gets -sum(F_ext)/N_fluid      */
    int walls;
    double wall_u_lo[3], wall_u_hi[3];
    int didt_mode;          /* 0: analytic Eq. Irotdiff, 1: finite difference, 2: predictor-corrector */
    double lub_cut;         /* lubrication correction below this gap (0: none)  */
    int collision;          /* 0: BGK; 1: the paper's ghost-mode scheme (stress modes relax with tau,
                               non-hydrodynamic modes to equilibrium at once) */
} orc_box;

typedef struct {
    double semi[3];         /* a (body x), b (body y), c (body z) */
    double x[3];
    double q[4];            /* (q0, q1, q2, q3), unit, body -> lab */
    double U[3], Om[3];
    double density;         /* particle mass density; M = density*4/3*pi*abc */
    double F_ext[3], T_ext[3];
    double B1, B2;          /* squirmer modes, 0 for a passive particle */
} orc_particle;

/* lifecycle */
orc_sim* orc_create(const orc_box* box, const orc_particle* parts, int np, int nthreads);
void     orc_destroy(orc_sim* s);
int      orc_step(orc_sim* s, int nsteps);          /* 0 ok, nonzero error code */
long     orc_time(const orc_sim* s);

/* lattice (oracle order): Q = 19 velocities, or 27 in the library built with
 * -DORC_D3Q27 (liboracle27.so); c has Q rows of 3, w Q entries */
int  orc_q(void);
void orc_lattice(int c[][3], double w[]);

/* fields.  f is node-major: f[node*Q + i], node = (z*ny + y)*nx + x,
 * oracle direction order.  Values are pre-collision f(x, t) at the start of
 * the current iteration; solid nodes read 0. */
void orc_get_f(const orc_sim* s, double* out);
void orc_set_f(orc_sim* s, const double* in);
/* rho and u = (sum f c + g/2)/rho per node (0 on solid nodes). */
void orc_get_moments(const orc_sim* s, double* rho, double* u /* N*3 */);
void orc_get_owner(const orc_sim* s, int* owner /* 0 fluid, -1 wall, p+1 */);
double orc_total_fluid_mass(const orc_sim* s);
void orc_total_fluid_momentum(const orc_sim* s, double out[3]);

/* particles: out[25] = F0[3], T0[3], F[3], T[3], U[3], Om[3], x[3], q[4] */
void orc_get_particle(const orc_sim* s, int p, double* out);
/* pending remap terms: dP[3], dL[3] (next solve), dm (last remap), dm_return
 * (remap before, put back at the next collision) */
void orc_get_pending(const orc_sim* s, int p, double* out8);
void orc_get_zeta(const orc_sim* s, int p, double* out36);
int  orc_get_links(const orc_sim* s, int p, int* node, int* cvec /* 3 per link */, int cap);
double orc_mass(const orc_sim* s, int p);

/* single pieces, for the pins */
void orc_feq(double rho, const double u[3], double out[] /* Q */);
void orc_quat_mul(const double a[4], const double b[4], double out[4]);
void orc_rotate(const double q[4], const double s[3], double out[3]);
void orc_inertia_lab(const double q[4], const double Ibody[3], double out[9]);
void orc_inertia_rate(const double q[4], const double Om[3], const double Ibody[3], double out[9]);
void orc_quat_step(const double q[4], const double Om_mean[3], double out[4]);
int  orc_gauss_solve(int n, const double* A, const double* b, double* x);
/* Lubrication correction between two bodies (positions, velocities and
 * orientations at time t): force on body p (the opposite acts on q) and the
 * gap h along the line of centres.  L/periodic: box edges for the minimum image. */
void orc_lubrication_pair(const double semi_p[3], const double q_p[4], const double x_p[3], const double U_p[3],
                          double M_p, const double semi_q[3], const double q_q[4], const double x_q[3],
                          const double U_q[3], double M_q, const int L[3], const int periodic[3], double mu,
                          double h_cut, double force_p[3], double* gap);
/* Steps 4-5 for one body with a given drag matrix (row-major 6x6) and
 * velocity-independent forces rF, rT; Iprev = I(t-1) (mode 1 only). */
int  orc_rigid_solve(double M, const double Ib[3], const double q[4], const double U[3], const double Om[3],
                     const double zeta36[36], const double rF[3], const double rT[3], const double Iprev[9],
                     int mode, double Unew[3], double Wnew[3]);
double orc_inside_value(const double semi[3], const double q[4], const double xc[3],
                        const int X[3], const int L[3], const int periodic[3]);
void orc_squirmer_slip(const double semi[3], const double q[4], double B1, double B2,
                       const double r[3], double out[3]);

#ifdef __cplusplus
}
#endif
#endif
