/*
 * psm.h -- C ABI of the GB300 LBM-PSM engine (fully resolved fluid-particle
 * coupling with the Partially Saturated Cells Method).
 *
 * The engine computes, per time step, the hot path of Kemmler et al.,
 * "Efficiency and scalability of fully-resolved fluid-particle simulations on
 * heterogeneous CPU-GPU architectures":
 *   (a) particle mapping: per-cell solid fraction B_i of spherical particles
 *       (Sec. 2.3.2: linear approximation, Eqs. 25-27; sub-division sampling;
 *       or a learned surrogate with a sampling fallback),
 *   (b) the PSM collision (Sec. 2.3, Eqs. 17-19) blending the SRT (Eq. 3) or
 *       TRT fluid relaxation with the solid operator, driven by the particle
 *       surface velocity of Eq. 20, fused with D3Q19 streaming (Eq. 2) and the
 *       forcing operator (Eq. 8),
 *   (c) the per-particle reduction of hydrodynamic force and torque
 *       (Eqs. 21-22),
 * followed by the DEM sub-cycles of Sec. 2.2 (linear spring-dashpot, Eq. 12;
 * velocity Verlet, Eqs. 15-16) on the device, so particle state stays in GPU
 * memory between steps.
 *
 * Conventions
 *  - Units are lattice units (dx = dt = 1, rho_0 = 1).  Cell (x,y,z) has its
 *    centre at (x+1/2, y+1/2, z+1/2); the domain is [0,nx)x[0,ny)x[0,nz).
 *  - D3Q19 ordering: q = 0 rest; q = 1..18 in opposite pairs (q, q+1) for odd
 *    q, with c_1 = (1,0,0), c_3 = (0,1,0), c_5 = (0,0,1), c_7 = (1,1,0),
 *    c_9 = (1,-1,0), c_11 = (1,0,1), c_13 = (1,0,-1), c_15 = (0,1,1),
 *    c_17 = (0,1,-1) and c_{q+1} = -c_q.
 *  - Host arrays of PDFs are f[q][z][y][x] (x fastest, nx*ny*nz cells per q);
 *    vector fields are component-major u[a][z][y][x]; particle vectors are
 *    n x 3 row-major.
 *  - Every pointer argument of the functions below is a HOST pointer owned by
 *    the caller; every call copies.  The context owns all device memory,
 *    allocated through psm_options.alloc (cudaMalloc when NULL).
 *  - All device work is queued on psm_options.stream (a cudaStream_t; NULL is
 *    the legacy default stream).  Functions that return data synchronise that
 *    stream only.
 *  - Every function returns a status and never aborts.  Errors detected on
 *    the device (slot overflow, non-finite force) are returned by the next
 *    psm_step / psm_get_* call; the context then refuses further steps with
 *    PSM_ERR_STATE until psm_set_pdfs or psm_set_particles is called.
 *  - A context must not be used from two host threads at once.
 */
#ifndef PSM_H
#define PSM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct psm_ctx psm_ctx;

typedef enum {
  PSM_OK = 0,
  PSM_ERR_ARG = 1,           /* invalid argument; nothing was changed */
  PSM_ERR_CUDA = 2,          /* a CUDA call failed; see psm_last_error */
  PSM_ERR_OOM = 3,           /* the allocator returned NULL */
  PSM_ERR_SLOT_OVERFLOW = 4, /* a cell lies within reach of > 2 particles */
  PSM_ERR_NONFINITE = 5,     /* a hydrodynamic force or a check sum is NaN/Inf */
  PSM_ERR_TIMEOUT = 6,       /* reserved: a bounded device wait gave up */
  PSM_ERR_STATE = 7          /* call not allowed in the current state */
} psm_status;

/* Domain: nx, ny, nz cells.  wall[f] sets the type of face f (order
 * -x,+x,-y,+y,-z,+z; boundaries sit on the domain faces, all cells are fluid
 * cells): PSM_FACE_PERIODIC, PSM_FACE_WALL (stationary halfway bounce-back),
 * and on the z faces only the open faces of the fluidized bed (Sec. 4.1: a
 * velocity inflow at the bottom, a pressure outflow at the top):
 * PSM_FACE_INFLOW, bounce-back of a wall moving with
 * psm_options.bc_velocity, f_q = f~_qbar + 6 w_q c_q.U_b, which lets exactly
 * U_b,z of mass through each face cell per step; PSM_FACE_OUTFLOW,
 * anti-bounce-back to psm_options.bc_density,
 * f_q = -f~_qbar + 2 w_q (rho_b + 9/2 (c_q.u_b)^2 - 3/2 u_b.u_b), u_b the
 * cell's own velocity after the last collision.  A link that also crosses a
 * side wall is bounced back.  Both faces of an axis are periodic or neither
 * is.  Particles see every non-periodic face as a wall plane; with an open
 * face the fluid gets no counter force for the particles' weight.  Open faces
 * need pull streaming (PSM_AA gives PSM_ERR_ARG). */
enum { PSM_FACE_PERIODIC = 0, PSM_FACE_WALL = 1, PSM_FACE_INFLOW = 2, PSM_FACE_OUTFLOW = 3 };
typedef struct {
  int nx, ny, nz;
  int wall[6];
} psm_grid;

typedef enum { PSM_SRT = 0, PSM_TRT = 1 } psm_relax;

enum { PSM_FP64 = 0,       /* PDFs stored and collided in FP64 */
       PSM_FP32_DEV = 1,   /* PDFs stored as FP32 deviations f_q - w_q,
                              collided in FP32; forces and checks in FP64 */
       PSM_FP64_DF = 2 };  /* PDFs stored as deviations in double-float form
                              (a pair of FP32 values hi + lo, 8 bytes, a
                              48-bit significand) and collided in double-float
                              arithmetic on the FP32 pipes; mapping, forces,
                              DEM and checks in FP64 */
enum { PSM_PULL = 0,       /* two buffers, pull streaming */
       PSM_AA = 1 };       /* one buffer, AA-pattern in-place streaming */
enum { PSM_EPS_SUPERSAMPLE = 0, /* eps from eps_n^3 sub-cell sample points */
       PSM_EPS_LINEAR = 1,      /* linear approximation, Eqs. 25-27 */
       PSM_EPS_MLP = 2 };       /* learned surrogate; 8^3 sampling for cells
                                   within reach of two particles or next to a
                                   wall face */
enum { PSM_W_EPS = 0,      /* B = eps (Sec. 2.3) */
       PSM_W_NT = 1 };     /* B = eps (tau-1/2) / ((1-eps) + (tau-1/2)),
                              Noble and Torczynski (cited in Sec. 2.3) */

typedef struct {
  double magic;          /* TRT magic parameter Lambda (default 3/16) */
  int precision;         /* PSM_FP64 | PSM_FP32_DEV | PSM_FP64_DF */
  int streaming;         /* PSM_PULL | PSM_AA */
  int eps_mode;          /* PSM_EPS_* */
  int eps_n;             /* samples per axis for PSM_EPS_SUPERSAMPLE (1..16); with
                            PSM_EPS_MLP the fallback always samples 8^3 points,
                            and eps_n = 8 lets the batched 8^3 count pass take
                            the shared cells (same results, faster) */
  int weighting;         /* PSM_W_EPS | PSM_W_NT */
  double body_force[3];  /* fluid body-force density f_ext */
  double gravity[3];     /* acceleration of free particles; a free particle
                            feels (m - V) g and the fluid a uniform counter
                            force so that a periodic box gains no momentum */
  double k_n;            /* normal contact stiffness (Eq. 12) */
  double restitution;    /* normal restitution coefficient, (0, 1] */
  int dem_subcycles;     /* DEM sub-steps per LBM step (default 10) */
  int dem;               /* 1: integrate free particles on the device */
  int deterministic;     /* must be 1: the force/torque reduction sums each
                            particle's cells in a fixed order (bitwise
                            reproducible run to run); any other value is
                            refused with PSM_ERR_ARG (no atomic reduction
                            is built) */
  int use_graphs;        /* 1: replay captured CUDA graphs for steps */
  void* stream;          /* cudaStream_t to queue all work on */
  void* (*alloc)(size_t bytes, void* user); /* device allocator or NULL */
  void (*free)(void* ptr, void* user);      /* matching release or NULL */
  void* alloc_user;                         /* passed to alloc/free */
  double bc_velocity[3]; /* fluid velocity of a PSM_FACE_INFLOW face */
  double bc_density;     /* fluid density of a PSM_FACE_OUTFLOW face (default 1) */
  double kt_ratio;       /* tangential contact between spheres (Eqs. 13-14):
                            k_t = kt_ratio k_n, d_t = kt_ratio d_n, with the
                            accumulated tangential displacement kept per pair
                            while in contact; 0 = normal contacts only
                            (default 2/7) */
} psm_options;

/* Fills *o with the defaults: Lambda = 3/16, FP64, pull, 4^3 sampling, NT
 * weighting, no forces, k_n = 1e3, e = 0.9, 10 sub-cycles, DEM on,
 * deterministic reduction, graphs on, default stream, cudaMalloc. */
void psm_default_options(psm_options* o);

/* Creates a context for the grid, relaxation time tau (> 1/2; tau_plus for
 * TRT) and relaxation model.  The fluid starts at rest, f_q = w_q.  On success
 * *out receives the context; on failure *out is NULL. */
psm_status psm_create(const psm_grid* grid, double tau, psm_relax relax,
                      const psm_options* opt, psm_ctx** out);

/* Replaces the particle set: n spheres with centres x (n*3), radii r,
 * velocities u (n*3), angular velocities omega (n*3), density ratios
 * density (particle/fluid), and fixed[i] != 0 for particles that never move
 * (fixed may be NULL: all free).  Positions along periodic axes are wrapped
 * into the box.  A particle must fit twice across a periodic box
 * (2 r + 3 <= n along that axis).  The next step re-maps the particles. */
psm_status psm_set_particles(psm_ctx* ctx, int n, const double* x, const double* r,
                             const double* u, const double* omega,
                             const double* density, const unsigned char* fixed);

/* Overwrites the centres, velocities and angular velocities (n*3 each, n as
 * set) of the current particles from host arrays, keeping radii, densities
 * and forces; the next step re-maps.  This is the per-step host->device
 * particle transfer of a hybrid CPU-GPU loop (Sec. 3.1.1). */
psm_status psm_update_particles(psm_ctx* ctx, const double* x, const double* u,
                                const double* omega);

/* Advances nsteps time steps: mapping (when particles moved or were set),
 * PSM stream-collide, force/torque reduction, DEM sub-cycles. */
psm_status psm_step(psm_ctx* ctx, int nsteps);

/* Advances nsteps time steps with the particle dynamics on the host cores,
 * the coupling the paper runs (Sec. 3.2): per step the device maps, collides
 * and reduces the forces (as psm_step), the hydrodynamic force and torque are
 * copied to the host, one DEM step (Eqs. 12, 15-16, the context's
 * sub-cycles) runs on up to `threads` host threads (<= 0 or more than the
 * hardware threads: all hardware threads; at most one thread per 256
 * particles),
 * and the particle state (centres, velocities, angular velocities and the
 * last sub-step's total force and torque) is copied back.  The DEM arithmetic
 * is the device's, operation for operation, so the state equals psm_step's.
 * *host_ms (may be NULL) receives the wall-clock milliseconds of the host
 * phase summed over the steps (from the end of the device part: force copy,
 * DEM, state copy).  Needs a context
 * created with the DEM on (PSM_ERR_ARG otherwise); without free particles it
 * is psm_step.  A particle that moves more than half the partner-list skin
 * within a step gives PSM_ERR_STATE.  The device status word is read with
 * each step's force copy: an error of the device part (slot overflow,
 * non-finite force) ends the loop at that step, before the host DEM uses the
 * forces, and is returned as psm_step would.  PSM_ERR_OOM when host memory
 * for the particle state runs out.  Every error leaves the context in its
 * error state. */
psm_status psm_step_host_dem(psm_ctx* ctx, int nsteps, int threads, double* host_ms);

/* One LBM step of particle dynamics on the host cores for n spheres, without
 * a context (for a caller that owns its fluid solver): the DEM of
 * psm_step_host_dem (Eqs. 12-16) with `subcycles` sub-steps of 1/subcycles,
 * stiffness k_n, restitution in (0, 1], tangential ratio kt_ratio (>= 0, see
 * psm_options), gravity[3], the grid's box (an axis whose faces are not
 * periodic has wall planes; both faces of an axis are periodic or neither
 * is).  In/out (host arrays, n*3): x, u, omega and F_old,
 * T_old (the total force and torque of the last sub-step; a new particle
 * starts with F_old = (m - V) gravity, T_old = 0), and the tangential
 * contact history: hist_count (n), hist_partner (n*64, each particle's
 * partners in contact in ascending order) and hist_delta (n*64*3, their
 * accumulated tangential displacement); a new particle starts with
 * hist_count = 0.  In: F_hyd, T_hyd (n*3,
 * held over the sub-steps), r, density (n), fixed (n, may be NULL).  Mass,
 * volume and inertia follow psm_set_particles (fluid density 1).  threads
 * as for psm_step_host_dem.  Returns PSM_ERR_ARG for invalid arguments
 * (nothing changed), PSM_ERR_STATE when a particle moved more than half the
 * partner-list skin (1 cell) within the step (the arrays then hold the
 * advanced state, which may have missed a contact) or when a particle
 * touched more than 64 partners, PSM_ERR_OOM when host
 * memory for the step ran out (the arrays may then be partly advanced).  A
 * worker thread that cannot be started makes the step run on fewer threads
 * with the same result; nothing is thrown.  Needs no GPU. */
psm_status psm_dem_step_host(const psm_grid* grid, double k_n, double restitution,
                             double kt_ratio, int subcycles, const double* gravity, int n,
                             double* x, double* u, double* omega, double* F_old, double* T_old,
                             int* hist_count, int* hist_partner, double* hist_delta,
                             const double* F_hyd, const double* T_hyd, const double* r,
                             const double* density, const unsigned char* fixed, int threads);

/* Hydrodynamic force and torque of Eqs. 21-22 from the last step (n*3 each). */
psm_status psm_get_force_torque(psm_ctx* ctx, double* F, double* T);

/* rho (N) and U (3*N, component-major) of the streamed PDFs: Eqs. 6-7 with
 * the fluid force density of the last step. */
psm_status psm_get_macroscopic(psm_ctx* ctx, double* rho, double* u);

/* Current particle centres, velocities and angular velocities (n*3 each). */
psm_status psm_get_particles(psm_ctx* ctx, double* x, double* u, double* omega);

/* The post-collision PDFs f~ of the last step (before streaming), 19*N FP64,
 * in the canonical layout above, whatever the storage precision/pattern. */
psm_status psm_get_pdfs(psm_ctx* ctx, double* f);

/* The same for a box of bx*by*bz cells with origin (x0, y0, z0): 19*bx*by*bz
 * FP64 values, layout f[q][z][y][x] over the box.  Along a periodic axis the
 * box wraps around (origin in [-n, 2n)); along an axis with walls it must lie
 * inside the grid.  PSM_ERR_ARG otherwise. */
psm_status psm_get_pdfs_box(psm_ctx* ctx, int x0, int y0, int z0, int bx, int by, int bz,
                            double* f);

/* Fluid force density applied in the last step (3 values): the body force
 * plus, with gravity and free particles, the counter force
 * -sum_i (m_i - V_i) g / V_fluid that keeps the periodic system from
 * accelerating (buoyancy-corrected gravity, Sec. 2.2), and V_fluid =
 * sum_x (1 - B) from the mapping it used (vfluid may be NULL). */
psm_status psm_get_fluid_force(psm_ctx* ctx, double* f, double* vfluid);

/* Replaces the PDF field (canonical layout, 19*N FP64) and clears a device
 * error state. */
psm_status psm_set_pdfs(psm_ctx* ctx, const double* f);

/* Mapping of the current particles as dense per-cell slots (N each): slot 0
 * holds the lower particle index; pid = -1 marks an empty slot; B is the
 * weight after the B > 1 normalisation of Sec. 2.3.  Maps first if needed. */
psm_status psm_get_slots(psm_ctx* ctx, int* pid0, double* B0, int* pid1, double* B1);

/* Per-slot hydrodynamic forces of the last step (Eq. 21: B_i times the
 * momentum the solid operator of slot i takes from the cell), with the
 * mapping they belong to (the last step's, not remapped for particles moved
 * since), as dense per-cell arrays: pid0, pid1 (N each, -1 for an empty
 * slot) and F0, F1 (3*N each, component-minor: F0[3 c + a]), converted to
 * FP64 from the form's precision, zero for an empty slot.  The per-particle
 * sums of these, with the torque arms of Eq. 22 taken from the particle
 * positions the mapping used, are what psm_get_force_torque returns; the
 * call lets a caller check that reduction. */
psm_status psm_get_slot_forces(psm_ctx* ctx, int* pid0, int* pid1, double* F0, double* F1);

/* FP64 sums over the stored PDFs: mass sum_x sum_q f_q and momentum
 * sum_x sum_q f_q c_q (3 values); fixed summation order. */
psm_status psm_check(psm_ctx* ctx, double* mass, double* momentum);

/* Surrogate network for PSM_EPS_MLP: 4 -> 32 (ReLU) -> 32 (ReLU) -> 1.  Its
 * inputs are x = (|d/r| components in decreasing order, r), d the offset of
 * the cell centre from the sphere centre (eps is invariant under sign flips
 * and permutations of d), and it predicts the correction to the linear
 * approximation of Eqs. 25-27: eps = clamp(eps_lin(|d|, r) + MLP(x), 0, 1).
 * params is the packed FP32 vector [W1 (32x4), b1 (32), W2 (32x32), b2 (32),
 * W3 (32), b3 (1)], row-major, PSM_MLP_PARAMS floats.  Inference runs the
 * hidden layer on the tensor cores with BF16 operands and FP32 accumulation. */
#define PSM_MLP_PARAMS 1249
psm_status psm_set_mlp(psm_ctx* ctx, const float* params);
psm_status psm_get_mlp(psm_ctx* ctx, float* params);

/* Trains the surrogate on the device with the engine's own forward/backward
 * and Adam kernels: nsamples samples of the SplitMix64 training recipe
 * (stream seed), labelled by 8^3 sub-division sampling (target: label minus
 * the linear approximation), minibatches of batch samples, epochs passes,
 * learning rate lr decaying exponentially to 3% of lr over the run.  Starts
 * from the current parameters.  loss_out (may be NULL) receives the mean
 * squared error of the final parameters over the training set. */
psm_status psm_train_surrogate(psm_ctx* ctx, long nsamples, unsigned long long seed,
                               int epochs, int batch, float lr, float* loss_out);

/* Kernel-level entry points of the surrogate (used to check them):
 * training samples i = first .. first+count-1 of stream seed: network inputs
 * X (count*4) and 8^3 labels eps (count); loss and gradient (PSM_MLP_PARAMS
 * floats) of the mean squared error of params on (X, t); raw network output
 * of the inference kernel for inputs X (before the linear approximation is
 * added and the result clamped): layer 1 in FP32, layer 2 on the tensor cores
 * (tcgen05.mma, BF16 operands, FP32 accumulation), layer 3 in FP32 — the
 * kernel the mapping runs in PSM_EPS_MLP mode. */
psm_status psm_mlp_samples(psm_ctx* ctx, unsigned long long seed, long first, long count,
                           float* X, float* eps);
psm_status psm_mlp_loss_grad(psm_ctx* ctx, const float* params, long m, const float* X,
                             const float* t, float* loss, float* grad);
psm_status psm_mlp_infer(psm_ctx* ctx, const float* params, long m, const float* X,
                         float* eps);

/* Event timings (ms) of the kernel classes, summed over the psm_step calls
 * since timing was enabled: out[0] mapping, out[1] PSM stream-collide,
 * out[2] force/torque reduction, out[3] DEM, out[4] steps timed.  With timing
 * on, steps are launched without graphs and bracketed by CUDA events on the
 * context's stream (no host synchronisation inside psm_step). */
psm_status psm_set_timing(psm_ctx* ctx, int enable);
psm_status psm_get_timings(psm_ctx* ctx, double* out5);

/* Kernel launches queued by the last psm_step call (all of this library's
 * kernels, graph nodes included). */
long psm_last_launch_count(const psm_ctx* ctx);

/* Mass and momentum of a PDF field that the caller already holds on the
 * device, computed without allocating any device memory.  The paper has no
 * counterpart to this call; it is here for callers that cannot allocate when
 * they want the check: a code that gives out all device memory from its own
 * fixed pool, a monitoring hook inside another solver's time loop where
 * cudaMalloc/cudaFree would synchronise the device and stall its streams, or
 * a run whose memory budget is fully committed.  psm_check gives the same
 * sums but allocates.
 *   f       device pointer, canonical FP64 layout f[q][cell] (19 * ncells)
 *   ncells  1 .. PSM_NOALLOC_MAX_CELLS; larger fields give PSM_ERR_ARG
 *   sums    device pointer to 4 doubles: mass, momentum x, y, z (written)
 *   stream  cudaStream_t the two kernels are queued on (NULL: legacy default)
 * Returns PSM_OK once the work is queued (nothing is synchronised),
 * PSM_ERR_ARG for NULL pointers or sizes out of range, PSM_ERR_CUDA if the
 * set-up or a launch fails.  The block partials live in one 128 KiB array in
 * device memory that the library declares at file scope: every GPU that
 * loads the library holds it until the process exits, and all calls on a
 * GPU share it, so calls whose work overlaps on the GPU (unordered streams)
 * race; order them on one stream.  The first call in each CUDA context of a
 * device (with that device current) looks up the array's device address:
 * the first call on the device, and again the first call after a
 * cudaDeviceReset or after another context was made current there, since the
 * library's device code is then loaded anew.  Make such a first call before
 * any stream capture. */
#define PSM_NOALLOC_MAX_CELLS (4096LL * 65536LL)
psm_status psm_field_sums_noalloc(const double* f, long long ncells, double* sums,
                                  void* stream);

/* Checkpoint and restart of the time stepper (the loop of Sec. 3 and its
 * Fig. "implementation"; the paper itself describes no checkpoint format).
 * psm_save writes, to the file at path, everything a later step depends on:
 * the PDF field in the storage form of ctx (its own values, not canonical
 * FP64: a resumed run continues bit for bit), the per-particle state (x, u,
 * omega, r, mass, inertia, volume, f(r), fixed flags, the last hydrodynamic
 * force and torque, the DEM force history) and the surrogate's parameters
 * when set.  psm_load reads such a file into ctx, which must have been
 * created with the same grid, walls, precision, streaming pattern,
 * relaxation, tau, magic parameter and DEM setting (PSM_ERR_ARG otherwise,
 * and for a missing, foreign or truncated file, ctx unchanged in that case);
 * derived state (slots, neighbour lists, step constants) is rebuilt on the
 * next step, and an error state is cleared.  Both synchronise the stream of
 * ctx.  The file is in the native byte order (little-endian on x86-64 and
 * aarch64). */
psm_status psm_save(psm_ctx* ctx, const char* path);
psm_status psm_load(psm_ctx* ctx, const char* path);
/* Diagnostic of failure detection (the paper has no counterpart): runs each
 * bounded device wait of the engine (the staged collision kernel's mbarrier
 * wait, the surrogate inference's wait on the tensor-core commit, the DEM
 * grid barrier) against a barrier that nothing completes, with a limit of
 * limit_ns (0..1e9) instead of the production 1 s.  Each must give up and
 * raise the timeout bit of the device status word; returns PSM_ERR_STATE if
 * one did not, PSM_OK otherwise, leaving the bit set so that the next
 * psm_step or psm_get_* reports PSM_ERR_TIMEOUT (and the context enters its
 * error state until psm_set_pdfs or psm_load).  No wait that can hang is
 * involved: every one is bounded by the global timer. */
psm_status psm_selftest_waits(psm_ctx* ctx, long long limit_ns);

/* Number of particles of ctx (after psm_set_particles or psm_load). */
psm_status psm_get_particle_count(const psm_ctx* ctx, int* n);

/* Human-readable description of the last error of ctx (never NULL). */
const char* psm_last_error(const psm_ctx* ctx);

/* Releases every device buffer of ctx through the free callback. */
void psm_destroy(psm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif
