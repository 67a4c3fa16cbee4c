/*
 * psm_oracle.c -- plain FP64 CPU oracle of the LBM-PSM hot path.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by tests/, by the smoke check and by the
 * CPU-baseline leg of bench.py; never by the product path.  Plain loops in the
 * order the paper gives them (Fig. "implementation", Sec. 3): mapping ->
 * stream + PSM collide -> force/torque -> DEM sub-cycles.  No blocking, no
 * fusion beyond what the equations state.  Compile with -ffp-contract=off.
 *
 * Readings of points the paper leaves open (documented project constants):
 *  A  Eq. 8 is printed without the (1 - dt/(2 tau)) prefactor although Eq. 7
 *     shifts U by f_ext/2.  The forcing term here carries the Guo prefactor:
 *     (1 - 1/(2 tau)) for SRT; for TRT its symmetric part gets (1 - w+/2) and
 *     its antisymmetric part (1 - w-/2).  With it the momentum a cell gains
 *     per step equals f_ext exactly (pinned by the momentum budget and by the
 *     Poiseuille amplitude).
 *  B  B(eps): weighting 0 is B = eps (paper text, Sec. 2.3); weighting 1 is
 *     the Noble-Torczynski form B = eps(tau-1/2)/((1-eps)+(tau-1/2)).
 *  C  "If B > 1 it is normalised to 1" (Sec. 2.3): every B_i is divided by
 *     sum_i B_i and B is set to 1.
 *  D  U_f keeps the full +f_ext/2 shift in every cell, covered or not (Eq. 7).
 *  E  The solid operator is exactly Eq. 19.
 *  F  A sample point exactly on the sphere surface counts as inside (<=).
 *  G  n^3 sampling uses sub-cell centres (a+1/2)/n - 1/2, a = 0..n-1.
 *  H  Walls sit on the domain faces; all cells are fluid cells; halfway
 *     bounce-back f_q(x) = f~_qbar(x) for a link that leaves the domain.
 *  V  Open faces of the fluidized bed (Sec. 4.1 names a velocity inflow at
 *     the bottom and a pressure outflow at the top, without formulas), on the
 *     z faces: an inflow face is a wall moving with the inflow velocity U_b,
 *     f_q(x) = f~_qbar(x) + 6 w_q (c_q . U_b) (bounce-back of a moving wall,
 *     rho_0 = 1), which lets exactly U_b,z cross each face cell per step; an
 *     outflow face holds the density rho_b by anti-bounce-back,
 *     f_q(x) = -f~_qbar(x) + 2 w_q (rho_b + 9/2 (c_q . u_b)^2 - 3/2 u_b . u_b),
 *     with u_b = sum_p f~_p(x) c_p the cell's own velocity after the last
 *     collision.  A link that also crosses a side wall is bounced back.  For
 *     particles the open faces are walls (Sec. 4.1: planes keep the particles
 *     in the box), and the counter force of reading J is not applied: the
 *     fluid is not a closed periodic system.
 *  I  MLP mode: the network is used for a partial cell within reach of one
 *     particle and not next to a wall face; every other partial cell uses
 *     8^3 sampling.  The network predicts the correction to the linear
 *     approximation of Eqs. 25-27: eps = clamp(eps_lin + MLP(x), 0, 1), with
 *     x = (|d/r| components sorted in decreasing order, r) -- the offset in
 *     the orientation fixed by the cube's symmetries (eps does not change
 *     under sign flips and permutations of the offset components).
 *  J  Gravity: a free particle feels (m - V) g (buoyancy with rho_f = 1).
 *     The fluid gets the uniform counter force density
 *     -sum_free (m_i - V_i) g / V_fluid, V_fluid = sum_x (1 - B(x)), applied
 *     through the (1-B) F_q term, so no net momentum enters a periodic box.
 *  K  Normal contact (Eq. 12): n_ij points from j to i and the spring term
 *     is written to be repulsive.  Damping from the restitution coefficient:
 *     d_n = -2 ln(e) sqrt(m_eff k_n)/sqrt(pi^2+ln^2 e) with
 *     m_eff = m_i m_j/(m_i+m_j) (m_i for a wall).
 *  W  Tangential contact between particles (Eqs. 13-14; the paper gives no
 *     coefficients): k_t = kt_ratio k_n and d_t = kt_ratio d_n.  With
 *     kt_ratio = 2/7 the tangential oscillator of two solid spheres (its
 *     effective mass is 2/7 m_eff) has the normal one's frequency and damping
 *     ratio.  The contact point is x_cp = x_i - (r_i - delta_n/2) n_ij; U^cp is
 *     the relative velocity of the two surfaces there, U_t its tangential
 *     part.  The history delta_t of a pair (Eq. 14) is kept while the pair is
 *     in contact: each sub-step it is projected onto the current tangent
 *     plane and advanced by dt_p U_t; it is dropped when the contact ends.
 *     F_t = -k_t delta_t - d_t U_t acts on i, -F_t on j, with the torques
 *     (x_cp - x_p) x F_t (Eq. 11).  No Coulomb limit (none is printed).
 *     Wall contacts stay normal only (Eqs. 11-13 sum over particle pairs).
 *  L  DEM sub-cycles use dt_p = 1/subcycles; the hydrodynamic force and torque
 *     of the LBM step are held constant over them; F_old starts as the
 *     external force when particles are set.
 *  S  "Reach" of a particle = cells whose centre is closer than r + sqrt(3)/2
 *     to the sphere centre.  A cell within reach of a particle holds a slot
 *     for it (its B may be 0); more than two slots per cell is an error.
 *     Slots are filled in particle-index order.  The offset d = x_cell - x_p
 *     is ((double)i + 0.5) - x_p with the integer i shifted by a multiple of
 *     the box length to the nearest image.
 */
#include "psm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q 19

/* D3Q19 velocities and weights (Sec. 2.1; weights of Qian et al.) */
static const int CX[Q] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int CY[Q] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int CZ[Q] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
static double W[Q];

static int opposite(int q) {
  if (q == 0) return 0;
  return (q % 2 == 1) ? q + 1 : q - 1;
}

static void init_weights(void) {
  W[0] = 1.0 / 3.0;
  for (int q = 1; q <= 6; ++q) W[q] = 1.0 / 18.0;
  for (int q = 7; q < Q; ++q) W[q] = 1.0 / 36.0;
}

struct or_ctx {
  or_config cfg;
  long N;
  double* f;      /* stored post-collision field f~ */
  double* fnew;
  /* mapping: two slots per cell */
  int* pid0;
  int* pid1;
  double* B0;
  double* B1;
  /* particles */
  int np;
  double *x, *r, *u, *om, *m, *I, *vol;
  unsigned char* fixed;
  double *Fh, *Th;       /* hydrodynamic force / torque of the last step */
  double *Fold, *Told;   /* total force / torque of the last DEM sub-step */
  /* MLP */
  int have_mlp;
  double W1[32 * 4], b1[32], W2[32 * 32], b2[32], W3[32], b3;
  /* last step */
  double fext_last[3];
  double vfluid_last;
  /* host threads of the loops (or_set_threads) */
  int threads;
  /* tangential contact history (reading W): per particle the partners in
   * contact at the last sub-step, ascending, with their delta_t */
  int* hcnt;
  int* hcap;
  int** hj;
  double** hd;
  double *Fcol, *Tcol;  /* contact force and torque of the last sub-step */
  /* per covered cell and slot, the force and torque contributions of the
   * last collision in cell order (z, y, x, slot), summed per particle after
   * the cell loop */
  long* plane_off;   /* first covered cell of each z-plane */
  double* contrib;   /* 12 values per covered cell: F, T of slot 0, then slot 1 */
  long contrib_cap;
};

or_ctx* or_create(const or_config* cfg) {
  init_weights();
  if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1) return NULL;
  for (int f = 0; f < 6; ++f) {
    if (cfg->wall[f] < 0 || cfg->wall[f] > 3) return NULL;
    if (cfg->wall[f] >= 2 && f < 4) return NULL; /* open faces on z only */
  }
  for (int a = 0; a < 3; ++a)
    if ((cfg->wall[2 * a] != 0) != (cfg->wall[2 * a + 1] != 0)) return NULL;
  if (!(cfg->tau > 0.5)) return NULL;
  or_ctx* c = (or_ctx*)calloc(1, sizeof(or_ctx));
  c->cfg = *cfg;
  c->N = (long)cfg->nx * cfg->ny * cfg->nz;
  c->f = (double*)malloc(sizeof(double) * Q * c->N);
  c->fnew = (double*)malloc(sizeof(double) * Q * c->N);
  c->pid0 = (int*)malloc(sizeof(int) * c->N);
  c->pid1 = (int*)malloc(sizeof(int) * c->N);
  c->B0 = (double*)malloc(sizeof(double) * c->N);
  c->B1 = (double*)malloc(sizeof(double) * c->N);
  /* initial state: equilibrium at rest, f_q = w_q (Eq. 5 with rho=1, U=0) */
  for (int q = 0; q < Q; ++q)
    for (long i = 0; i < c->N; ++i) c->f[q * c->N + i] = W[q];
  for (long i = 0; i < c->N; ++i) {
    c->pid0[i] = -1; c->pid1[i] = -1; c->B0[i] = 0.0; c->B1[i] = 0.0;
  }
  c->vfluid_last = (double)c->N;
  for (int a = 0; a < 3; ++a) c->fext_last[a] = cfg->fbody[a];
  c->threads = 1;
  c->plane_off = (long*)malloc(sizeof(long) * ((size_t)cfg->nz + 1));
  return c;
}

void or_set_threads(or_ctx* c, int threads) { c->threads = threads < 1 ? 1 : threads; }

static void free_particles(or_ctx* c) {
  for (int i = 0; i < c->np; ++i) {
    if (c->hj) free(c->hj[i]);
    if (c->hd) free(c->hd[i]);
  }
  free(c->hcnt); free(c->hcap); free(c->hj); free(c->hd); free(c->Fcol); free(c->Tcol);
  c->hcnt = c->hcap = NULL; c->hj = NULL; c->hd = NULL; c->Fcol = c->Tcol = NULL;
  free(c->x); free(c->r); free(c->u); free(c->om); free(c->m); free(c->I);
  free(c->vol); free(c->fixed); free(c->Fh); free(c->Th); free(c->Fold); free(c->Told);
  c->x = c->r = c->u = c->om = c->m = c->I = c->vol = NULL;
  c->Fh = c->Th = c->Fold = c->Told = NULL;
  c->fixed = NULL;
  c->np = 0;
}

void or_destroy(or_ctx* c) {
  if (!c) return;
  free(c->f); free(c->fnew); free(c->pid0); free(c->pid1); free(c->B0); free(c->B1);
  free(c->plane_off); free(c->contrib);
  free_particles(c);
  free(c);
}

static const double PI = 3.14159265358979323846;

int or_set_particles(or_ctx* c, int n, const double* x, const double* r,
                     const double* u, const double* om, const double* rho_p,
                     const unsigned char* fixed) {
  if (n < 0) return -1;
  free_particles(c);
  c->np = n;
  size_t s3 = sizeof(double) * 3 * (size_t)(n > 0 ? n : 1);
  size_t s1 = sizeof(double) * (size_t)(n > 0 ? n : 1);
  c->x = (double*)malloc(s3); c->u = (double*)malloc(s3); c->om = (double*)malloc(s3);
  c->Fh = (double*)calloc(1, s3); c->Th = (double*)calloc(1, s3);
  c->Fold = (double*)calloc(1, s3); c->Told = (double*)calloc(1, s3);
  c->r = (double*)malloc(s1); c->m = (double*)malloc(s1); c->I = (double*)malloc(s1);
  c->vol = (double*)malloc(s1);
  c->fixed = (unsigned char*)calloc(1, (size_t)(n > 0 ? n : 1));
  size_t n1 = (size_t)(n > 0 ? n : 1);
  c->hcnt = (int*)calloc(n1, sizeof(int));
  c->hcap = (int*)calloc(n1, sizeof(int));
  c->hj = (int**)calloc(n1, sizeof(int*));
  c->hd = (double**)calloc(n1, sizeof(double*));
  c->Fcol = (double*)calloc(1, s3);
  c->Tcol = (double*)calloc(1, s3);
  for (int i = 0; i < n; ++i) {
    if (!(r[i] > 0.0) || !(rho_p[i] > 0.0)) return -1;
    for (int a = 0; a < 3; ++a) {
      c->x[3 * i + a] = x[3 * i + a];
      c->u[3 * i + a] = u[3 * i + a];
      c->om[3 * i + a] = om[3 * i + a];
    }
    c->r[i] = r[i];
    c->vol[i] = 4.0 / 3.0 * PI * r[i] * r[i] * r[i];
    c->m[i] = rho_p[i] * c->vol[i];
    c->I[i] = 0.4 * c->m[i] * r[i] * r[i];
    c->fixed[i] = fixed ? fixed[i] : 0;
    /* reading L: F_old starts as the external (buoyancy-corrected) force */
    for (int a = 0; a < 3; ++a)
      c->Fold[3 * i + a] = c->fixed[i] ? 0.0 : (c->m[i] - c->vol[i]) * c->cfg.gravity[a];
  }
  return 0;
}

int or_set_mlp(or_ctx* c, const double* W1, const double* b1, const double* W2,
               const double* b2, const double* W3, const double* b3) {
  memcpy(c->W1, W1, sizeof(double) * 32 * 4);
  memcpy(c->b1, b1, sizeof(double) * 32);
  memcpy(c->W2, W2, sizeof(double) * 32 * 32);
  memcpy(c->b2, b2, sizeof(double) * 32);
  memcpy(c->W3, W3, sizeof(double) * 32);
  c->b3 = b3[0];
  c->have_mlp = 1;
  return 0;
}

void or_set_pdfs(or_ctx* c, const double* f) { memcpy(c->f, f, sizeof(double) * Q * c->N); }
void or_get_pdfs(const or_ctx* c, double* f) { memcpy(f, c->f, sizeof(double) * Q * c->N); }

/* ---------------------------------------------------------------- mapping */

/* Eq. 27: V_a = integral of sqrt(r^2-x^2-y^2) over the unit square centred on
 * the axis (the closed form printed in Sec. 2.3.2). */
double or_Va(double r) {
  double r2 = r * r;
  double s = sqrt(r2 - 0.5);
  return (1.0 / 12.0 - r2) * atan((0.5 * s) / (0.5 - r2)) + s / 3.0 +
         (r2 - 1.0 / 12.0) * atan(0.5 / s) - 4.0 / 3.0 * r2 * r * atan(0.25 / (r * s));
}

/* Eqs. 25-26: eps = -D + f(r), f(r) = V_a - r + 1/2, D = dist - r, clamped to
 * [0, 1] (an overlap exists only for eps in (0, 1]). */
double or_eps_linear(double dist, double r) {
  double D = dist - r;
  double fr = or_Va(r) - r + 0.5;
  double e = -D + fr;
  if (e < 0.0) e = 0.0;
  if (e > 1.0) e = 1.0;
  return e;
}

/* Sub-division sampling (reading G, F): count sample points p of the cell with
 * |p - x_p|^2 <= r^2, p - x_p = d + s, s_a = (a + 1/2)/n - 1/2. */
long or_eps_supersample_count(double dx, double dy, double dz, double r, int n) {
  long count = 0;
  double r2 = r * r;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b)
      for (int k = 0; k < n; ++k) {
        double sx = (a + 0.5) / n - 0.5;
        double sy = (b + 0.5) / n - 0.5;
        double sz = (k + 0.5) / n - 0.5;
        double px = dx + sx, py = dy + sy, pz = dz + sz;
        double d2 = px * px + py * py + pz * pz;
        if (d2 <= r2) ++count;
      }
  return count;
}

/* Weighting of Noble and Torczynski (reading B) */
double or_nt_weight(double eps, double tau) {
  return eps * (tau - 0.5) / ((1.0 - eps) + (tau - 0.5));
}

/* linear approximation for a batch of distances and radii */
void or_eps_linear_batch(long m, const double* dist, const double* r, double* eps) {
  for (long i = 0; i < m; ++i) eps[i] = or_eps_linear(dist[i], r[i]);
}

/* labels for a batch of offsets: count of n^3 samples inside, per row */
void or_supersample_batch(long m, const double* d, const double* r, int n, long* count) {
  for (long i = 0; i < m; ++i)
    count[i] = or_eps_supersample_count(d[3 * i + 0], d[3 * i + 1], d[3 * i + 2], r[i], n);
}

static const double HALF_SQRT3 = 0.86602540378443864676; /* sqrt(3)/2 */

static double mlp_eval(const or_ctx* c, const double in[4]) {
  double h1[32], h2[32];
  for (int j = 0; j < 32; ++j) {
    double s = c->b1[j];
    for (int k = 0; k < 4; ++k) s += c->W1[j * 4 + k] * in[k];
    h1[j] = s > 0.0 ? s : 0.0;
  }
  for (int j = 0; j < 32; ++j) {
    double s = c->b2[j];
    for (int k = 0; k < 32; ++k) s += c->W2[j * 32 + k] * h1[k];
    h2[j] = s > 0.0 ? s : 0.0;
  }
  double o = c->b3;
  for (int k = 0; k < 32; ++k) o += c->W3[k] * h2[k];
  return o;
}

/* overlap fraction of one cell for one particle at offset d (dist = |d|) */
static double cell_eps(const or_ctx* c, double dx, double dy, double dz, double r,
                       int single, int next_to_wall) {
  double d2 = dx * dx + dy * dy + dz * dz;
  double dist = sqrt(d2);
  int mode = c->cfg.eps_mode;
  if (mode == 1) return or_eps_linear(dist, r);
  /* cells fully inside or outside need no sampling: every sample point lies
   * within sqrt(3)/2 of the cell centre */
  double rin = r - HALF_SQRT3;
  if (rin > 0.0 && d2 <= rin * rin) return 1.0;
  double rout = r + HALF_SQRT3;
  if (d2 >= rout * rout) return 0.0;
  if (mode == 2 && c->have_mlp && single && !next_to_wall) {
    double a[3] = {fabs(dx / r), fabs(dy / r), fabs(dz / r)};
    /* sort in decreasing order */
    for (int i = 0; i < 2; ++i)
      for (int j = i + 1; j < 3; ++j)
        if (a[j] > a[i]) { double t = a[i]; a[i] = a[j]; a[j] = t; }
    double in[4] = {a[0], a[1], a[2], r};
    double e = or_eps_linear(dist, r) + mlp_eval(c, in);
    if (e < 0.0) e = 0.0;
    if (e > 1.0) e = 1.0;
    return e;
  }
  int n = (mode == 0) ? c->cfg.eps_n : 8;
  long cnt = or_eps_supersample_count(dx, dy, dz, r, n);
  return (double)cnt / ((double)n * n * n);
}

static long cell_index(const or_ctx* c, int x, int y, int z) {
  return (long)x + (long)c->cfg.nx * ((long)y + (long)c->cfg.ny * z);
}

/* nearest-image integer coordinate of the cell along one axis (reading S) */
static int nearest_image(int i, double xp, int n, int periodic) {
  if (!periodic) return i;
  double d = (i + 0.5) - xp;
  if (d > 0.5 * n) return i - n;
  if (d < -0.5 * n) return i + n;
  return i;
}

/* The cells within reach of particle p (reading S), in the order of its box
 * of cells (z, y, x): their indices and nearest-image offsets d = x_cell - x_p
 * (3 per cell).  Returns -1 when the box is wider than a periodic axis. */
static int reach_list(const or_ctx* c, int p, const int dims[3], const int per[3],
                      long** cells_out, double** offs_out, int* count_out) {
  double r = c->r[p];
  int lo[3], hi[3];
  long box = 1;
  *cells_out = NULL; *offs_out = NULL; *count_out = 0;
  for (int a = 0; a < 3; ++a) {
    double xp = c->x[3 * p + a];
    lo[a] = (int)floor(xp - r - 1.0);
    hi[a] = (int)floor(xp + r + 1.0);
    if (per[a] && hi[a] - lo[a] + 1 > dims[a]) return -1;
    if (!per[a]) {
      if (lo[a] < 0) lo[a] = 0;
      if (hi[a] > dims[a] - 1) hi[a] = dims[a] - 1;
    }
    box *= (hi[a] >= lo[a]) ? (long)(hi[a] - lo[a] + 1) : 0;
  }
  long* cells = (long*)malloc(sizeof(long) * (size_t)(box > 0 ? box : 1));
  double* offs = (double*)malloc(sizeof(double) * 3 * (size_t)(box > 0 ? box : 1));
  int n = 0;
  double reach = r + HALF_SQRT3;
  for (int kz = lo[2]; kz <= hi[2]; ++kz)
    for (int ky = lo[1]; ky <= hi[1]; ++ky)
      for (int kx = lo[0]; kx <= hi[0]; ++kx) {
        int ix = ((kx % dims[0]) + dims[0]) % dims[0];
        int iy = ((ky % dims[1]) + dims[1]) % dims[1];
        int iz = ((kz % dims[2]) + dims[2]) % dims[2];
        int ux = nearest_image(ix, c->x[3 * p + 0], dims[0], per[0]);
        int uy = nearest_image(iy, c->x[3 * p + 1], dims[1], per[1]);
        int uz = nearest_image(iz, c->x[3 * p + 2], dims[2], per[2]);
        double dx = (ux + 0.5) - c->x[3 * p + 0];
        double dy = (uy + 0.5) - c->x[3 * p + 1];
        double dz = (uz + 0.5) - c->x[3 * p + 2];
        double d2 = dx * dx + dy * dy + dz * dz;
        if (!(d2 < reach * reach)) continue;
        cells[n] = cell_index(c, ix, iy, iz);
        offs[3 * n + 0] = dx; offs[3 * n + 1] = dy; offs[3 * n + 2] = dz;
        ++n;
      }
  *cells_out = cells; *offs_out = offs; *count_out = n;
  return 0;
}

int or_map(or_ctx* c) {
  const or_config* g = &c->cfg;
  int dims[3] = {g->nx, g->ny, g->nz};
  int per[3] = {!g->wall[0], !g->wall[2], !g->wall[4]};
  int np = c->np;
  int status = 0, bad = 0;
  for (long i = 0; i < c->N; ++i) {
    c->pid0[i] = -1; c->pid1[i] = -1; c->B0[i] = 0.0; c->B1[i] = 0.0;
  }
  int* nreach = (int*)calloc((size_t)c->N, sizeof(int));
  long** cells = (long**)calloc((size_t)(np > 0 ? np : 1), sizeof(long*));
  double** offs = (double**)calloc((size_t)(np > 0 ? np : 1), sizeof(double*));
  double** Bs = (double**)calloc((size_t)(np > 0 ? np : 1), sizeof(double*));
  int* cnt = (int*)calloc((size_t)(np > 0 ? np : 1), sizeof(int));
  /* pass 1: the cells each particle reaches, and how many particles reach
   * each cell (for the MLP fallback rule; integer counts, so the order of
   * the increments does not matter) */
#pragma omp parallel for schedule(dynamic, 4) num_threads(c->threads) reduction(| : bad)
  for (int p = 0; p < np; ++p) {
    bad |= reach_list(c, p, dims, per, &cells[p], &offs[p], &cnt[p]) != 0;
    for (int k = 0; k < cnt[p]; ++k) {
#pragma omp atomic
      nreach[cells[p][k]] += 1;
    }
  }
  if (!bad) {
    /* pass 2: overlap fraction and weight of every (particle, cell) pair
     * (Sec. 2.3.2; reading B) */
#pragma omp parallel for schedule(dynamic, 4) num_threads(c->threads)
    for (int p = 0; p < np; ++p) {
      Bs[p] = (double*)malloc(sizeof(double) * (size_t)(cnt[p] > 0 ? cnt[p] : 1));
      for (int k = 0; k < cnt[p]; ++k) {
        long cell = cells[p][k];
        int ix = (int)(cell % g->nx);
        int iy = (int)((cell / g->nx) % g->ny);
        int iz = (int)(cell / ((long)g->nx * g->ny));
        int next_to_wall = (g->wall[0] && (ix == 0 || ix == dims[0] - 1)) ||
                           (g->wall[2] && (iy == 0 || iy == dims[1] - 1)) ||
                           (g->wall[4] && (iz == 0 || iz == dims[2] - 1));
        const double* d = &offs[p][3 * k];
        double eps = cell_eps(c, d[0], d[1], d[2], c->r[p], nreach[cell] == 1, next_to_wall);
        Bs[p][k] = (g->weighting == 1) ? or_nt_weight(eps, g->tau) : eps;
      }
    }
    /* slots filled in particle-index order (reading S) */
    for (int p = 0; p < np; ++p)
      for (int k = 0; k < cnt[p]; ++k) {
        long cell = cells[p][k];
        if (c->pid0[cell] < 0) {
          c->pid0[cell] = p; c->B0[cell] = Bs[p][k];
        } else if (c->pid1[cell] < 0) {
          c->pid1[cell] = p; c->B1[cell] = Bs[p][k];
        } else {
          status = -2;
        }
      }
  }
  for (int p = 0; p < np; ++p) { free(cells[p]); free(offs[p]); free(Bs[p]); }
  free(cells); free(offs); free(Bs); free(cnt); free(nreach);
  return bad ? -1 : status;
}

void or_get_slots(const or_ctx* c, int* pid0, double* B0, int* pid1, double* B1) {
  memcpy(pid0, c->pid0, sizeof(int) * c->N);
  memcpy(pid1, c->pid1, sizeof(int) * c->N);
  memcpy(B0, c->B0, sizeof(double) * c->N);
  memcpy(B1, c->B1, sizeof(double) * c->N);
}

/* ------------------------------------------------------- LBM + PSM step */

/* Eq. 5, incompressible equilibrium (He and Luo), rho_0 = 1, c_s^2 = 1/3 */
static double feq(int q, double rho, const double U[3]) {
  double cu = CX[q] * U[0] + CY[q] * U[1] + CZ[q] * U[2];
  double uu = U[0] * U[0] + U[1] * U[1] + U[2] * U[2];
  return W[q] * (rho + (3.0 * cu + 4.5 * cu * cu - 1.5 * uu));
}

/* bare forcing term of Eq. 8 (Delta t = 1), without the prefactor of reading A */
static double force_term(int q, const double U[3], const double fe[3]) {
  double c[3] = {CX[q], CY[q], CZ[q]};
  double cu = c[0] * U[0] + c[1] * U[1] + c[2] * U[2];
  double s = 0.0;
  for (int a = 0; a < 3; ++a) s += ((c[a] - U[a]) * 3.0 + cu * c[a] * 9.0) * fe[a];
  return W[q] * s;
}

/* nearest-image offset of a cell centre from particle p (reading S) */
static void cell_offset(const or_ctx* c, int p, int x, int y, int z, double d[3]) {
  const or_config* g = &c->cfg;
  int ux = nearest_image(x, c->x[3 * p + 0], g->nx, !g->wall[0]);
  int uy = nearest_image(y, c->x[3 * p + 1], g->ny, !g->wall[2]);
  int uz = nearest_image(z, c->x[3 * p + 2], g->nz, !g->wall[4]);
  d[0] = (ux + 0.5) - c->x[3 * p + 0];
  d[1] = (uy + 0.5) - c->x[3 * p + 1];
  d[2] = (uz + 0.5) - c->x[3 * p + 2];
}

/* pull streaming of direction q into cell (x,y,z): Eq. 2 read backwards, with
 * periodic wrap, halfway bounce-back (reading H) and the open faces of
 * reading V */
static double pull(const or_ctx* c, const double* src, int q, int x, int y, int z) {
  const or_config* g = &c->cfg;
  int sx = x - CX[q], sy = y - CY[q], sz = z - CZ[q];
  int side = 0; /* face type the link leaves through: 1 wall, 2 inflow, 3 outflow */
  if (sx < 0 || sx >= g->nx) { if (g->wall[0]) side = 1; else sx = (sx + g->nx) % g->nx; }
  if (sy < 0 || sy >= g->ny) { if (g->wall[2]) side = 1; else sy = (sy + g->ny) % g->ny; }
  if (sz < 0 || sz >= g->nz) {
    int t = g->wall[sz < 0 ? 4 : 5];
    if (!t) sz = (sz + g->nz) % g->nz;
    else if (side != 1) side = t;
  }
  long cell = cell_index(c, x, y, z);
  int qb = opposite(q);
  if (side == 0) return src[q * c->N + cell_index(c, sx, sy, sz)];
  if (side == 1) return src[qb * c->N + cell];
  if (side == 2) {
    const double* U = g->bc_velocity;
    return src[qb * c->N + cell] + 6.0 * W[q] * (CX[q] * U[0] + CY[q] * U[1] + CZ[q] * U[2]);
  }
  double ub[3] = {0.0, 0.0, 0.0};
  for (int p = 0; p < Q; ++p) {
    double fp = src[p * c->N + cell];
    ub[0] += fp * CX[p]; ub[1] += fp * CY[p]; ub[2] += fp * CZ[p];
  }
  double cu = CX[q] * ub[0] + CY[q] * ub[1] + CZ[q] * ub[2];
  double uu = ub[0] * ub[0] + ub[1] * ub[1] + ub[2] * ub[2];
  return -src[qb * c->N + cell] + 2.0 * W[q] * (g->bc_density + 4.5 * cu * cu - 1.5 * uu);
}

static void fluid_force_density(or_ctx* c, double fe[3]) {
  /* reading J: counter force for the buoyancy-corrected gravity on free
   * particles, spread over the fluid volume of the current mapping */
  double vfluid = 0.0;
  for (long i = 0; i < c->N; ++i) {
    double B = c->B0[i] + c->B1[i];
    if (B > 1.0) B = 1.0;
    vfluid += 1.0 - B;
  }
  double G[3] = {0.0, 0.0, 0.0};
  int open = 0;
  for (int f = 0; f < 6; ++f) open |= c->cfg.wall[f] >= 2;
  if (c->cfg.dem && !open) {
    for (int p = 0; p < c->np; ++p) {
      if (c->fixed[p]) continue;
      for (int a = 0; a < 3; ++a) G[a] += (c->m[p] - c->vol[p]) * c->cfg.gravity[a];
    }
  }
  for (int a = 0; a < 3; ++a)
    fe[a] = c->cfg.fbody[a] - (vfluid > 0.0 ? G[a] / vfluid : 0.0);
  c->vfluid_last = vfluid;
}

static void psm_collide_stream(or_ctx* c) {
  const or_config* g = &c->cfg;
  double tau_p = g->tau;
  double tau_m = (g->relax == 1) ? 0.5 + g->magic / (g->tau - 0.5) : g->tau;
  double fe[3];
  fluid_force_density(c, fe);
  for (int a = 0; a < 3; ++a) c->fext_last[a] = fe[a];
  for (int p = 0; p < c->np; ++p)
    for (int a = 0; a < 3; ++a) { c->Fh[3 * p + a] = 0.0; c->Th[3 * p + a] = 0.0; }
  /* a place for the force and torque contributions of every covered cell,
   * numbered in cell order from the first covered cell of its z-plane */
  long ncov = 0;
  for (int z = 0; z < g->nz; ++z) {
    c->plane_off[z] = ncov;
    for (long i = (long)z * g->nx * g->ny; i < (long)(z + 1) * g->nx * g->ny; ++i)
      if (c->pid0[i] >= 0) ++ncov;
  }
  c->plane_off[g->nz] = ncov;
  if (ncov > c->contrib_cap) {
    free(c->contrib);
    c->contrib = (double*)malloc(sizeof(double) * 12 * (size_t)ncov);
    c->contrib_cap = ncov;
  }

  /* the cells of one z-plane are visited in order by one thread */
#pragma omp parallel for schedule(dynamic, 1) num_threads(c->threads)
  for (int z = 0; z < g->nz; ++z) {
    long icov = c->plane_off[z];
    for (int y = 0; y < g->ny; ++y)
      for (int x = 0; x < g->nx; ++x) {
        long cell = cell_index(c, x, y, z);
        double f[Q];
        for (int q = 0; q < Q; ++q) f[q] = pull(c, c->f, q, x, y, z);
        /* Eqs. 6-7 */
        double rho = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int q = 0; q < Q; ++q) {
          rho += f[q];
          j[0] += f[q] * CX[q]; j[1] += f[q] * CY[q]; j[2] += f[q] * CZ[q];
        }
        double U[3];
        for (int a = 0; a < 3; ++a) U[a] = j[a] + 0.5 * fe[a];
        double fq_eq[Q], Cf[Q], Fq[Q], Fbare[Q];
        for (int q = 0; q < Q; ++q) fq_eq[q] = feq(q, rho, U);
        for (int q = 0; q < Q; ++q) Fbare[q] = force_term(q, U, fe);
        if (g->relax == 0) {
          /* Eq. 3 and Eq. 8 with the prefactor of reading A */
          for (int q = 0; q < Q; ++q) {
            Cf[q] = (fq_eq[q] - f[q]) / tau_p;
            Fq[q] = (1.0 - 1.0 / (2.0 * tau_p)) * Fbare[q];
          }
        } else {
          /* TRT: relax symmetric and antisymmetric parts separately */
          for (int q = 0; q < Q; ++q) {
            int qb = opposite(q);
            double fp = 0.5 * (f[q] + f[qb]), fm = 0.5 * (f[q] - f[qb]);
            double ep = 0.5 * (fq_eq[q] + fq_eq[qb]), em = 0.5 * (fq_eq[q] - fq_eq[qb]);
            Cf[q] = -(fp - ep) / tau_p - (fm - em) / tau_m;
            double Fp = 0.5 * (Fbare[q] + Fbare[qb]), Fm = 0.5 * (Fbare[q] - Fbare[qb]);
            Fq[q] = (1.0 - 1.0 / (2.0 * tau_p)) * Fp + (1.0 - 1.0 / (2.0 * tau_m)) * Fm;
          }
        }
        /* PSM weights and normalisation (Sec. 2.3, reading C) */
        int pid[2] = {c->pid0[cell], c->pid1[cell]};
        double Bi[2] = {c->B0[cell], c->B1[cell]};
        double B = Bi[0] + Bi[1];
        if (B > 1.0) {
          Bi[0] = Bi[0] / B;
          Bi[1] = Bi[1] / B;
          B = 1.0;
        }
        double Cs[2][Q];
        double dvec[2][3];
        for (int s = 0; s < 2; ++s) {
          if (pid[s] < 0) continue;
          int p = pid[s];
          cell_offset(c, p, x, y, z, dvec[s]);
          /* Eq. 20: particle velocity at the cell centre */
          double Up[3];
          const double* om = &c->om[3 * p];
          double* d = dvec[s];
          Up[0] = c->u[3 * p + 0] + (om[1] * d[2] - om[2] * d[1]);
          Up[1] = c->u[3 * p + 1] + (om[2] * d[0] - om[0] * d[2]);
          Up[2] = c->u[3 * p + 2] + (om[0] * d[1] - om[1] * d[0]);
          /* Eq. 19: solid collision operator */
          for (int q = 0; q < Q; ++q) {
            int qb = opposite(q);
            Cs[s][q] = (f[qb] - fq_eq[qb]) - (f[q] - feq(q, rho, Up));
          }
        }
        /* Eq. 17 with Eq. 18 */
        for (int q = 0; q < Q; ++q) {
          double sol = 0.0;
          for (int s = 0; s < 2; ++s)
            if (pid[s] >= 0) sol += Bi[s] * Cs[s][q];
          c->fnew[q * c->N + cell] = f[q] + (1.0 - B) * Cf[q] + sol + (1.0 - B) * Fq[q];
        }
        /* Eqs. 21-22 with dx = dt = 1: this cell's contribution per slot */
        for (int s = 0; s < 2; ++s) {
          if (pid[s] < 0) continue;
          double S[3] = {0.0, 0.0, 0.0};
          for (int q = 0; q < Q; ++q) {
            int qb = opposite(q);
            S[0] += Cs[s][q] * CX[qb];
            S[1] += Cs[s][q] * CY[qb];
            S[2] += Cs[s][q] * CZ[qb];
          }
          double* d = dvec[s];
          double* o = &c->contrib[12 * icov + 6 * s];
          o[0] = Bi[s] * S[0];
          o[1] = Bi[s] * S[1];
          o[2] = Bi[s] * S[2];
          o[3] = d[1] * o[2] - d[2] * o[1];
          o[4] = d[2] * o[0] - d[0] * o[2];
          o[5] = d[0] * o[1] - d[1] * o[0];
        }
        if (pid[0] >= 0) ++icov;
      }
  }
  /* per-particle sums in cell order (z, y, x), slot 0 before slot 1 */
  long icov = 0;
  for (long cell = 0; cell < c->N; ++cell) {
    if (c->pid0[cell] < 0) continue;
    int pid[2] = {c->pid0[cell], c->pid1[cell]};
    for (int s = 0; s < 2; ++s) {
      if (pid[s] < 0) continue;
      const double* o = &c->contrib[12 * icov + 6 * s];
      for (int a = 0; a < 3; ++a) {
        c->Fh[3 * pid[s] + a] += o[a];
        c->Th[3 * pid[s] + a] += o[3 + a];
      }
    }
    ++icov;
  }
  double* t = c->f;
  c->f = c->fnew;
  c->fnew = t;
}

/* ------------------------------------------------------------------ DEM */

static double damping(double meff, double kn, double e) {
  double le = log(e);
  return -2.0 * le * sqrt(meff * kn) / sqrt(PI * PI + le * le);
}

static void dem_substeps(or_ctx* c) {
  const or_config* g = &c->cfg;
  int np = c->np;
  if (!g->dem || np == 0) return;
  double dims[3] = {g->nx, g->ny, g->nz};
  int per[3] = {!g->wall[0], !g->wall[2], !g->wall[4]};
  double dt = 1.0 / g->subcycles;
  for (int sc = 0; sc < g->subcycles; ++sc) {
    /* Eq. 15: position update with the old force */
#pragma omp parallel for num_threads(c->threads)
    for (int i = 0; i < np; ++i) {
      if (c->fixed[i]) continue;
      for (int a = 0; a < 3; ++a) {
        double xn = c->x[3 * i + a] + dt * c->u[3 * i + a] +
                    dt * dt * c->Fold[3 * i + a] / (2.0 * c->m[i]);
        if (per[a]) {
          if (xn >= dims[a]) xn -= dims[a];
          else if (xn < 0.0) xn += dims[a];
        }
        c->x[3 * i + a] = xn;
      }
    }
    /* Eq. 12 (and Eqs. 13-14, reading W): spring-dashpot contacts, pairs in
     * ascending j, then walls */
#pragma omp parallel for schedule(dynamic, 16) num_threads(c->threads)
    for (int i = 0; i < np; ++i) {
      double F[3] = {0.0, 0.0, 0.0}, T[3] = {0.0, 0.0, 0.0};
      int nold = c->hcnt[i], po = 0, nnew = 0, cap = nold + 8;
      int* nj = (int*)malloc(sizeof(int) * (size_t)cap);
      double* nd = (double*)malloc(sizeof(double) * 3 * (size_t)cap);
      for (int jj = 0; jj < np; ++jj) {
        if (jj == i) continue;
        double d[3];
        for (int a = 0; a < 3; ++a) {
          double v = c->x[3 * i + a] - c->x[3 * jj + a];
          if (per[a]) {
            if (v > 0.5 * dims[a]) v -= dims[a];
            else if (v < -0.5 * dims[a]) v += dims[a];
          }
          d[a] = v;
        }
        double dist2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        double rs = c->r[i] + c->r[jj];
        if (!(dist2 < rs * rs)) continue;
        double dist = sqrt(dist2);
        double delta = rs - dist;
        double n[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
        double vrel[3] = {c->u[3 * i + 0] - c->u[3 * jj + 0], c->u[3 * i + 1] - c->u[3 * jj + 1],
                          c->u[3 * i + 2] - c->u[3 * jj + 2]};
        double vn = vrel[0] * n[0] + vrel[1] * n[1] + vrel[2] * n[2];
        double meff = c->m[i] * c->m[jj] / (c->m[i] + c->m[jj]);
        double dn = damping(meff, g->kn, g->restitution);
        for (int a = 0; a < 3; ++a) F[a] += g->kn * delta * n[a] - dn * vn * n[a];
        if (!(g->kt_ratio > 0.0)) continue;
        /* Eq. 13 at the contact point: arms from the centres, relative
         * velocity of the surfaces, its tangential part */
        double ai = -(c->r[i] - 0.5 * delta), aj = c->r[jj] - 0.5 * delta;
        double Ai[3] = {ai * n[0], ai * n[1], ai * n[2]};
        double Aj[3] = {aj * n[0], aj * n[1], aj * n[2]};
        const double* wi = &c->om[3 * i];
        const double* wj = &c->om[3 * jj];
        double Ucp[3] = {
            (c->u[3 * i + 0] + (wi[1] * Ai[2] - wi[2] * Ai[1])) -
                (c->u[3 * jj + 0] + (wj[1] * Aj[2] - wj[2] * Aj[1])),
            (c->u[3 * i + 1] + (wi[2] * Ai[0] - wi[0] * Ai[2])) -
                (c->u[3 * jj + 1] + (wj[2] * Aj[0] - wj[0] * Aj[2])),
            (c->u[3 * i + 2] + (wi[0] * Ai[1] - wi[1] * Ai[0])) -
                (c->u[3 * jj + 2] + (wj[0] * Aj[1] - wj[1] * Aj[0]))};
        double un = Ucp[0] * n[0] + Ucp[1] * n[1] + Ucp[2] * n[2];
        double Ut[3] = {Ucp[0] - un * n[0], Ucp[1] - un * n[1], Ucp[2] - un * n[2]};
        /* Eq. 14: the pair's history, projected onto the current tangent
         * plane and advanced by this sub-step */
        double h[3] = {0.0, 0.0, 0.0};
        while (po < nold && c->hj[i][po] < jj) ++po;
        if (po < nold && c->hj[i][po] == jj)
          for (int a = 0; a < 3; ++a) h[a] = c->hd[i][3 * po + a];
        double hn = h[0] * n[0] + h[1] * n[1] + h[2] * n[2];
        for (int a = 0; a < 3; ++a) h[a] = (h[a] - hn * n[a]) + dt * Ut[a];
        double kt = g->kt_ratio * g->kn, dtg = g->kt_ratio * dn;
        double Ft[3] = {-kt * h[0] - dtg * Ut[0], -kt * h[1] - dtg * Ut[1],
                        -kt * h[2] - dtg * Ut[2]};
        for (int a = 0; a < 3; ++a) F[a] += Ft[a];
        T[0] += Ai[1] * Ft[2] - Ai[2] * Ft[1];
        T[1] += Ai[2] * Ft[0] - Ai[0] * Ft[2];
        T[2] += Ai[0] * Ft[1] - Ai[1] * Ft[0];
        if (nnew == cap) {
          cap *= 2;
          nj = (int*)realloc(nj, sizeof(int) * (size_t)cap);
          nd = (double*)realloc(nd, sizeof(double) * 3 * (size_t)cap);
        }
        nj[nnew] = jj;
        for (int a = 0; a < 3; ++a) nd[3 * nnew + a] = h[a];
        ++nnew;
      }
      free(c->hj[i]); free(c->hd[i]);
      c->hj[i] = nj; c->hd[i] = nd; c->hcnt[i] = nnew; c->hcap[i] = cap;
      for (int a = 0; a < 3; ++a) {
        if (per[a]) continue;
        for (int side = 0; side < 2; ++side) {
          double delta = side == 0 ? c->r[i] - c->x[3 * i + a]
                                   : c->x[3 * i + a] + c->r[i] - dims[a];
          if (!(delta > 0.0)) continue;
          double nn = side == 0 ? 1.0 : -1.0;
          double vn = c->u[3 * i + a] * nn;
          double dn = damping(c->m[i], g->kn, g->restitution);
          F[a] += g->kn * delta * nn - dn * vn * nn;
        }
      }
      for (int a = 0; a < 3; ++a) {
        c->Fcol[3 * i + a] = F[a];
        c->Tcol[3 * i + a] = T[a];
      }
    }
    /* total force (Eq. 9 without lubrication) and Eq. 16 */
#pragma omp parallel for num_threads(c->threads)
    for (int i = 0; i < np; ++i) {
      if (c->fixed[i]) continue;
      for (int a = 0; a < 3; ++a) {
        double Fn = c->Fh[3 * i + a] + c->Fcol[3 * i + a] + (c->m[i] - c->vol[i]) * g->gravity[a];
        double Tn = c->Th[3 * i + a] + c->Tcol[3 * i + a];
        c->u[3 * i + a] += dt * (c->Fold[3 * i + a] + Fn) / (2.0 * c->m[i]);
        c->om[3 * i + a] += dt * (c->Told[3 * i + a] + Tn) / (2.0 * c->I[i]);
        c->Fold[3 * i + a] = Fn;
        c->Told[3 * i + a] = Tn;
      }
    }
  }
}

int or_step(or_ctx* c, int n) {
  for (int s = 0; s < n; ++s) {
    int st = or_map(c);
    if (st != 0) return st;
    psm_collide_stream(c);
    dem_substeps(c);
  }
  return 0;
}

int or_dem_only(or_ctx* c, int n) {
  for (int s = 0; s < n; ++s) dem_substeps(c);
  return 0;
}

void or_get_force_torque(const or_ctx* c, double* F, double* T) {
  memcpy(F, c->Fh, sizeof(double) * 3 * c->np);
  memcpy(T, c->Th, sizeof(double) * 3 * c->np);
}

void or_get_contact(const or_ctx* c, double* F, double* T) {
  memcpy(F, c->Fcol, sizeof(double) * 3 * c->np);
  memcpy(T, c->Tcol, sizeof(double) * 3 * c->np);
}

void or_set_hydro(or_ctx* c, const double* F, const double* T) {
  memcpy(c->Fh, F, sizeof(double) * 3 * c->np);
  memcpy(c->Th, T, sizeof(double) * 3 * c->np);
}

void or_get_particles(const or_ctx* c, double* x, double* u, double* om) {
  memcpy(x, c->x, sizeof(double) * 3 * c->np);
  memcpy(u, c->u, sizeof(double) * 3 * c->np);
  memcpy(om, c->om, sizeof(double) * 3 * c->np);
}

void or_macroscopic(const or_ctx* c, double* rho, double* u) {
  const or_config* g = &c->cfg;
  for (int z = 0; z < g->nz; ++z)
    for (int y = 0; y < g->ny; ++y)
      for (int x = 0; x < g->nx; ++x) {
        long cell = cell_index(c, x, y, z);
        double r = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int q = 0; q < Q; ++q) {
          double fq = pull(c, c->f, q, x, y, z);
          r += fq;
          j[0] += fq * CX[q]; j[1] += fq * CY[q]; j[2] += fq * CZ[q];
        }
        rho[cell] = r;
        for (int a = 0; a < 3; ++a) u[a * c->N + cell] = j[a] + 0.5 * c->fext_last[a];
      }
}

double or_mass(const or_ctx* c) {
  double m = 0.0;
  for (long i = 0; i < c->N; ++i)
    for (int q = 0; q < Q; ++q) m += c->f[q * c->N + i];
  return m;
}

void or_momentum(const or_ctx* c, double* P) {
  P[0] = P[1] = P[2] = 0.0;
  for (long i = 0; i < c->N; ++i)
    for (int q = 0; q < Q; ++q) {
      double fq = c->f[q * c->N + i];
      P[0] += fq * CX[q]; P[1] += fq * CY[q]; P[2] += fq * CZ[q];
    }
}

void or_last_fext(const or_ctx* c, double* fe) {
  for (int a = 0; a < 3; ++a) fe[a] = c->fext_last[a];
}

double or_last_fluid_volume(const or_ctx* c) { return c->vfluid_last; }
