/*
 * psm_oracle.h -- plain FP64 CPU oracle of the LBM-PSM hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
 * leg of bench.py may load this library.  It shares no code, header, table or
 * constant with the CUDA path; it is written directly from the paper
 * (Kemmler et al., "Efficiency and scalability of fully-resolved fluid-particle
 * simulations on heterogeneous CPU-GPU architectures"):
 *   Sec. 2.1  D3Q19 LBM: Eq. 1 (collide), Eq. 2 (stream), Eq. 3 (SRT),
 *             Eq. 5 (incompressible equilibrium), Eqs. 6-7 (moments with the
 *             half-force shift), Eq. 8 (forcing operator)
 *   Sec. 2.2  DEM: Eq. 12 (normal spring-dashpot), Eqs. 15-16 (velocity Verlet)
 *   Sec. 2.3  PSM: Eq. 17-19 (modified collision, solid operator), Eq. 20
 *             (surface velocity), Eqs. 21-22 (hydrodynamic force and torque)
 *   Sec. 2.3.2 particle mapping: Eqs. 25-27 (linear approximation of the
 *             overlap fraction) and the sub-division sampling it is compared to.
 * Readings of points the paper leaves open are listed at the top of
 * psm_oracle.c; each one is a documented constant of the project.
 *
 * Lattice ordering (a project constant shared only through documentation):
 *   q:  0      1      2      3      4      5      6
 *   c: (0,0,0)(1,0,0)(-1,0,0)(0,1,0)(0,-1,0)(0,0,1)(0,0,-1)
 *   q:  7        8         9        10       11       12
 *   c: (1,1,0) (-1,-1,0) (1,-1,0) (-1,1,0) (1,0,1) (-1,0,-1)
 *   q:  13       14       15       16        17       18
 *   c: (1,0,-1)(-1,0,1) (0,1,1) (0,-1,-1) (0,1,-1) (0,-1,1)
 *   opposite(q) = q+1 for odd q, q-1 for even q > 0.
 * PDF arrays are f[q][z][y][x] (x fastest), N = nx*ny*nz cells, cell centre of
 * (x,y,z) at (x+1/2, y+1/2, z+1/2).  The stored state between steps is the
 * post-collision field f~ (pull streaming reads it at the start of the next
 * step).
 */
#ifndef PSM_ORACLE_H
#define PSM_ORACLE_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int nx, ny, nz;
  int wall[6];        /* faces -x,+x,-y,+y,-z,+z: 0 = periodic, 1 =
                         stationary halfway bounce-back wall, 2 = velocity
                         inflow (bc_velocity), 3 = pressure outflow
                         (bc_density); 2 and 3 on the z faces only.  Both
                         faces of one axis are periodic or neither is. */
  double tau;         /* relaxation time (tau_plus for TRT) */
  int relax;          /* 0 = SRT (Eq. 3), 1 = TRT */
  double magic;       /* TRT magic parameter Lambda */
  double fbody[3];    /* fluid body-force density */
  int weighting;      /* 0: B = eps; 1: B = eps(tau-1/2)/((1-eps)+(tau-1/2)) */
  int eps_mode;       /* 0: n^3 sub-division sampling, 1: linear approximation
                         (Eqs. 25-27), 2: MLP surrogate with 8^3 fallback */
  int eps_n;          /* samples per axis for eps_mode 0 */
  double gravity[3];  /* gravitational acceleration on particles */
  double kn;          /* normal contact stiffness */
  double restitution; /* normal coefficient of restitution */
  int subcycles;      /* DEM sub-steps per LBM step */
  int dem;            /* 1: integrate free particles; 0: particles never move */
  double bc_velocity[3]; /* fluid velocity of an inflow face */
  double bc_density;     /* fluid density of an outflow face */
  double kt_ratio;       /* tangential contact (Eqs. 13-14): k_t = kt_ratio k_n,
                            d_t = kt_ratio d_n; 0 = normal contacts only */
} or_config;

typedef struct or_ctx or_ctx;

or_ctx* or_create(const or_config* cfg);
void or_destroy(or_ctx* c);
/* 0 on success, negative on invalid input */
int or_set_particles(or_ctx* c, int n, const double* x, const double* r,
                     const double* u, const double* om, const double* rho_p,
                     const unsigned char* fixed);
/* MLP weights (row-major, W1: 32x4, W2: 32x32, W3: 1x32), FP64 */
int or_set_mlp(or_ctx* c, const double* W1, const double* b1, const double* W2,
               const double* b2, const double* W3, const double* b3);
void or_set_pdfs(or_ctx* c, const double* f);
void or_get_pdfs(const or_ctx* c, double* f);
/* Mapping of the current particle positions (Sec. 2.3.2). Returns 0, or -2
 * when a cell lies within reach of more than two particles. */
int or_map(or_ctx* c);
/* Per-cell slots of the last mapping: pid = -1 for an empty slot. */
void or_get_slots(const or_ctx* c, int* pid0, double* B0, int* pid1, double* B1);
/* Host threads of the step's loops (default 1).  The mapping's overlap
 * fractions, the cells of the collision and the particles of the DEM are
 * split over the threads; every sum keeps the single-thread order (slots in
 * particle-index order, forces in cell order), so the results do not depend
 * on the thread count.  Without OpenMP the oracle runs on one thread. */
void or_set_threads(or_ctx* c, int threads);
/* n full time steps: mapping, PSM stream-collide, force/torque, DEM. */
int or_step(or_ctx* c, int n);
/* Only the DEM sub-cycles of n time steps, hydrodynamic force held fixed. */
int or_dem_only(or_ctx* c, int n);
void or_get_force_torque(const or_ctx* c, double* F, double* T);
void or_set_hydro(or_ctx* c, const double* F, const double* T);
void or_get_particles(const or_ctx* c, double* x, double* u, double* om);
/* contact force and torque on every particle (fixed ones included) at the
 * last DEM sub-step */
void or_get_contact(const or_ctx* c, double* F, double* T);
/* rho and U (component-major, 3*N) of the streamed field, Eqs. 6-7 */
void or_macroscopic(const or_ctx* c, double* rho, double* u);
/* sums over the stored field: mass and momentum */
double or_mass(const or_ctx* c);
void or_momentum(const or_ctx* c, double* P);
/* fluid force density used in the last step (body force + counter force) */
void or_last_fext(const or_ctx* c, double* fext);
double or_last_fluid_volume(const or_ctx* c);

/* stand-alone mapping pieces (Sec. 2.3.2) */
double or_Va(double r);
double or_eps_linear(double dist, double r);
/* sub-division sampling of the cell whose centre is at offset d from the
 * sphere centre; returns the count of the n^3 sample points inside */
long or_eps_supersample_count(double dx, double dy, double dz, double r, int n);
double or_nt_weight(double eps, double tau);
void or_supersample_batch(long m, const double* d, const double* r, int n, long* count);
void or_eps_linear_batch(long m, const double* dist, const double* r, double* eps);

#ifdef __cplusplus
}
#endif
#endif
