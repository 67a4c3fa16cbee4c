// psm_internal.cuh -- device data layout and kernel launchers of the engine.
//
// Layout in HBM (one GPU):
//   PDFs      T* buf[q * ncell + cell], cell = x + nxp*(y + ny*z), x padded to
//             nxp = a multiple of 32 so that one warp covers 32 cells of one
//             x-row and one 32-bit coverage word.  Values are deviations
//             delta_q = f_q - w_q (FP64 or FP32).  Pull streaming keeps two
//             buffers; the AA pattern keeps one.
//   Coverage  mask[word] (bit = cell within reach of some particle), base[word]
//             = exclusive prefix count of set bits: the covered cells, in cell
//             order, index the slot table.
//   Slots     per covered cell: int2 pid (slot 0 < slot 1, -1 = empty), B as
//             T2 (after the B > 1 normalisation), cnt (particles in reach),
//             and the per-slot hydrodynamic contribution Fc[6] (T) written by
//             the collision kernel for the fixed-order force reduction.
//   Particles FP64 SoA on the device (x, u, omega, r, m, I, F_hyd, T_hyd,
//             F_old, T_old, fixed); the FP32 path reads float copies.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "df.cuh"

namespace psm {

constexpr int Q = 19;

// storage and arithmetic of the PDFs: FP64; FP32 deviations; double-float
// pairs (FP32 hi + lo, 8 bytes per value, arithmetic on the FP32 pipes)
enum : int { PREC_FP64 = 0, PREC_FP32 = 1, PREC_DF = 2 };

// Status bits raised on the device
enum : unsigned {
  ST_SLOT_OVERFLOW = 1u,
  ST_NONFINITE = 2u,
  ST_CONTACT_OVERFLOW = 4u,
  ST_TIMEOUT = 8u,   // a bounded device wait gave up
  ST_DEM_SKIN = 16u, // a particle moved more than half the neighbour-list skin in one step
};

// unsigned division by an invariant d for 0 <= n < 2^32 (Granlund and
// Montgomery, PLDI 1994, Sec. 4): with l = ceil(log2 d) and
// m = floor(2^32 (2^l - d) / d) + 1, t = mulhi(m, n) gives
// n / d = (t + ((n - t) >> min(l, 1))) >> max(l - 1, 0).
struct FastDiv {
  unsigned m;
  int s1, s2;
#ifdef __CUDACC__
  __device__ __forceinline__ unsigned div(unsigned n) const {
    const unsigned t = __umulhi(n, m);
    return (t + ((n - t) >> s1)) >> s2;
  }
#endif
};
__host__ __device__ inline FastDiv make_fastdiv(unsigned d) {
  int l = 0;
  while ((1ull << l) < d) ++l;
  FastDiv f;
  f.m = (unsigned)((((1ull << 32) * ((1ull << l) - d)) / d) + 1);
  f.s1 = l < 1 ? l : 1;
  f.s2 = l > 1 ? l - 1 : 0;
  return f;
}

// face types (the values of PSM_FACE_* in include/psm.h)
enum { FACE_PERIODIC = 0, FACE_WALL = 1, FACE_INFLOW = 2, FACE_OUTFLOW = 3 };

// constants of the open z faces: per direction 6 w_q c_q.U_b of a velocity
// inflow, and rho_b - 1 of a pressure outflow
struct OpenBC {
  double in[19];
  double rho1;
};

struct Grid {
  int nx, ny, nz, nxp;
  int wall[3];          // 1 = both faces of that axis are not periodic
  int zface[2];         // face types of -z and +z (PSM_FACE_*; open faces on z only)
  int wpr;              // warps (coverage words) per x-row = nxp / 32
  long long ncell;      // nxp * ny * nz (< 2^31)
  long long nwords;     // ncell / 32
  FastDiv div_wpr, div_ny;
};

// Constants of one time step, computed on the device after the mapping
// collision coefficients of one step in the storage precision: Eqs. 3-8
// with the Guo prefactors (1 - omega/2) on the forcing, grouped so that the
// relaxation of a pair is a chain of fused multiply-adds, and packed in
// groups of four for 16-byte loads.  Class c = 0 holds the face pairs
// (w = 1/18), c = 1 the edge pairs (w = 1/36).
enum {
  CC_HF = 0,      // f_ext / 2 (3 values), the velocity shift of Eq. 7
  CC_NWP = 3,     // -omega+
  CC_F = 4,       // f_ext (3 values)
  CC_WPW0 = 7,    // omega+ w_0
  CC_H = 8,       // forcing, symmetric part / (U . f_ext): rest, faces, edges
  CC_MHWP = 11,   // -omega+/2
  CC_WPW = 12,    // omega+ w_c (2 values)
  CC_MHWM = 14    // -omega-/2
};
template <typename T>
struct alignas(16) CollideCoef {
  T head[16];
  // per pair k: symmetric forcing / (c_k . U), antisymmetric forcing,
  // 9/2 omega+ w_c, 3 omega- w_c
  T pair[9][4];
  // for cells without particles, where a pair's update is written as
  // d_q' = S_k + A_k: 1 - omega+, (1 - omega+)/2, (1 - omega-)/2, 0
  T tail[4];
};

struct StepConst {
  double fext[3];       // fluid force density (body force + counter force)
  double vfluid;        // sum over cells of (1 - B)
  double sumB;          // sum over cells of min(B, 1), accumulated by the mapping
  double ncells;        // nx * ny * nz
  CollideCoef<double> d;
  CollideCoef<float> f;
  CollideCoef<df> x;
};

struct Particles {
  int n;
  double* x;      // n*3
  double* u;      // n*3
  double* om;     // n*3
  double* r;      // n
  double* m;      // n
  double* I;      // n
  double* vol;    // n
  double* fr;     // n, f(r) of Eq. 26 for the linear approximation
  unsigned char* fixed;  // n
  double* Fh;     // n*3 hydrodynamic force of the last step
  double* Th;     // n*3
  double* Fold;   // n*3 total force of the last DEM sub-step
  double* Told;   // n*3
  double* Fc;     // n*3 contact force scratch
  float* xf;      // n*4 float copies for the FP32 collision
  float* uf;      // n*4
  float* omf;     // n*4
  double* x2;     // second buffers of the DEM sub-steps
  double* u2;
  float* xf2;
  double* om2;
  // tangential contact history (Eqs. 13-14), two buffers: per particle the
  // partners in contact at the last sub-step (ascending, at most DEM list
  // capacity K) and their accumulated tangential displacement delta_t
  int* hcnt[2];   // n
  int* hj[2];     // n*K
  double* hd[2];  // n*K*3
};

struct Slots {
  int* cell;      // padded cell index of each entry
  int2* pid;
  int* cnt;       // particles in reach of entry e: 2-bit field e % 16 of word e / 16
  void* Fc;       // slot s's force of entry e at T[3 (s cap + e)]
  // slot s's record of entry e at T[4 (s cap + e)]: the particle's surface
  // velocity at the cell centre (Eq. 20) and the slot's normalised weight
  // B_i, negated in slot 0 when the cell has a second particle
  void* V;
  long long cap;
};

struct Coverage {
  uint32_t* mask;
  int* base;
  // FP64 records only (else nullptr): bit = covered cell with one particle
  // and B = 1 (every sample inside), written by the finish pass
  uint32_t* full;
  // bit = cell in reach of two or more particles (the mark pass sets it when
  // its coverage bit was already set): a cell without it takes slot 0 with no
  // claim, and in surrogate mode it is the network's if partial
  uint32_t* dup;
  int* blocksum;
  int* ncov;      // device scalar
  long long nblocks;
};

struct MapParams {
  Grid g;
  Particles p;
  Coverage cov;
  Slots s;
  int fp32;             // slot records and forces in FP32 (1), else FP64 or double-float
  int dfrec;            // slot records and forces as double-float pairs (the df form)
  int eps_mode, eps_n, weighting;
  double tau;
  unsigned* status;
  StepConst* sc;
  double G[3];          // sum over free particles of (m - V) g
  double fbody[3];
  double omega_p, omega_m;
  const double* wtab;   // B of each sampled count c = 0..n^3 (n^3 < 513), or NULL;
                        // their FP32 roundings follow at (const float*)(wtab + 513)
  const float* mlp;     // FP32 parameters (PSM_MLP_PARAMS)
  double* partials;     // >= MAP_PARTIALS doubles of scratch
  // surrogate worklist (eps mode 2): network inputs, linear approximation,
  // 2 * slot entry + slot, item count (at most mlp_cap items)
  // 8^3 sampling: each particle's cells that need sampling, listed by the
  // fill pass at the particle's list range (FP32 offset of the cell centre
  // and the cell's box index; 2 * slot entry + slot, as unsigned) and their
  // number per particle; counted by a pass of their own
  float4* wl_X;
  int* wl_work;
  int* wl_cnt;
  float* mlp_X;
  float* mlp_lin;
  int* mlp_work;
  int* mlp_count;
  long long mlp_cap;
  void* boxes;          // per particle: its box of cells and FP64 set-up (map_box_bytes() each)
  // per-particle lists of covered slot entries (box order) for the
  // fixed-order force/torque reduction
  const long long* list_off;   // n+1 offsets
  int* list;
  int* list_cnt;
  // surrogate mode: per particle, its partial cells for the network (in
  // reach, not inside by the margin, not next to a wall face), counted by the
  // mark pass; the fill pass reserves that many worklist items
  int* list_net;
};
constexpr int MAP_PARTIALS = 152 * 32;

struct LbmParams {
  Grid g;
  const void* src;      // T*
  void* dst;            // T*
  const void* srcq[19]; // per-direction planes (filled by the launcher)
  void* dstq[19];
  const uint32_t* mask; // nullptr when there are no particles
  const int* base;
  const uint32_t* full; // Coverage::full (FP64 records), or nullptr
  void* slot_Fc;        // Slots::Fc
  const void* slot_V;   // Slots::V
  long long slot_cap;   // entries allocated
  const StepConst* sc;
  double omega_p, omega_m;
  OpenBC bc;            // open z faces
  unsigned* status;     // device status word (ST_* bits)
  // staged kernel (stages > 0): tiles of tile_rows x-rows, `stages` tiles in
  // flight per block, `blocks` persistent blocks with `smem` bytes each
  int tile_rows, ntiles, stages, blocks;
  size_t smem;
  // one-cell-per-thread FP32 pull kernel: each block prefetches into L2 the
  // source spans of the block pf_ahead places later (0: no prefetch)
  int pf_ahead;
};

struct LbmPlan {
  int tile_rows, ntiles, stages, blocks;
  size_t smem;
  int pf_ahead;
};

// ---- launchers (stream-ordered; return the number of kernel launches) ----
int lbm_configure();  // kernel attributes; call once before launching (returns != 0 on error)
// staged-kernel plan for a grid (stages = 0: use the one-cell-per-thread kernel)
int lbm_plan(const Grid& g, int prec, int aa, LbmPlan* plan);
int launch_lbm(const LbmParams& P, int prec, int mode, cudaStream_t s);
// a box of cells, origin (x0, y0, z0) (non-negative, taken modulo the grid) and
// extent (bx, by, bz); output layout [q][z][y][x] over the box
struct BoxSel {
  int x0, y0, z0, bx, by, bz;
};
int launch_to_canonical(const Grid& g, const void* buf, int prec, int aa_parity, int aa,
                        const BoxSel& B, double* out, cudaStream_t s);
int launch_from_canonical(const Grid& g, const double* in, void* buf, int prec, int aa,
                          cudaStream_t s);
int launch_macroscopic(const Grid& g, const double* f, const StepConst* sc, const OpenBC& bc,
                       double* rho,
                       double* u, cudaStream_t s);
int launch_sums(const Grid& g, const double* f, double* partials, int nparts, double* out4,
                cudaStream_t s);
int launch_step_const(MapParams P, cudaStream_t s);

int launch_map(MapParams P, cudaStream_t s);                   // full mapping
size_t map_box_bytes();                                        // bytes per particle of MapParams::boxes
int launch_force_reduce(MapParams P, cudaStream_t s);
// table of B for the n^3 + 1 sampled counts (n^3 < 513); returns launches
int launch_weight_table(int n, double tau, int weighting, double* out, cudaStream_t s);          // fixed-order F/T
int launch_force_reduce_atomic_finish(MapParams P, cudaStream_t s);
int launch_pack_particles(Particles p, cudaStream_t s);
int launch_wrap_particles(const Grid& g, Particles p, cudaStream_t s);
int launch_slot_forces_to_dense(MapParams P, int* pid0, int* pid1, double* F0, double* F1,
                                cudaStream_t s);
int launch_slots_to_dense(MapParams P, int* pid0, double* B0, int* pid1, double* B1,
                          cudaStream_t s);

struct DemParams {
  Grid g;
  Particles p;
  double kn, log_e, dt;
  double kt_ratio;    // tangential contact: k_t = kt_ratio k_n, d_t = kt_ratio d_n (0: off)
  double gravity[3];
  unsigned* status;
  int nc[3];          // bins per axis (edge >= largest diameter + skin)
  float h[3];         // bin edges
  float skin;         // neighbour-list margin beyond contact
  int K;              // neighbour-list capacity per particle
  int nbins;
  int* bin_count;     // nbins
  int* bin_start;     // nbins
  int* bin_cursor;    // nbins
  int* bin_items;     // n, particle indices grouped by bin
  int* pbin;          // n, bin of each particle
  int* nbr;           // n*K, candidate partners in ascending order
  int* nbr_cnt;       // n
  float4* xbuild;     // n, positions when the lists were built
  unsigned* bar;      // [0] barrier arrivals, [1] barrier generation, [2] lists valid
                      // (0: rebuild), [3] particles with a non-empty list
  int max_blocks;     // blocks that can be resident at once (cooperative launch)
};
int dem_max_blocks();
// diagnostics of the bounded device waits (each raises ST_TIMEOUT in *status
// after limit_ns): the staged collision's mbarrier wait, the surrogate
// inference's mbarrier wait, the DEM grid barrier (bar: 4 words of scratch)
int launch_wait_selftest_lbm(unsigned* status, unsigned long long limit_ns, cudaStream_t s);
int launch_wait_selftest_mlp(unsigned* status, unsigned long long limit_ns, cudaStream_t s);
int launch_wait_selftest_dem(unsigned* bar, unsigned* status, unsigned long long limit_ns,
                             cudaStream_t s);
int launch_dem_step(DemParams P, int subcycles, cudaStream_t s);

// MLP
int launch_mlp_samples(unsigned long long seed, long long first, long long count, float* X,
                       float* eps, float* resid, cudaStream_t s);
int launch_mlp_loss_grad(const float* params, long long m, const float* X, const float* t,
                         float* grad_partials, int nblocks, float* grad, float* loss,
                         cudaStream_t s);
int launch_adam(float* params, const float* grad, float* mstate, float* vstate, int step,
                float lr, cudaStream_t s);
// where the network's outputs go: raw outputs (eps != NULL), or, in the
// mapping, B of each worklist item's slot record
struct InferSink {
  float* eps;          // raw outputs, or NULL
  void* V;             // Slots::V
  const float* lin;    // linear approximation (Eqs. 25-27) per item
  const int* work;     // item -> 2 * slot entry + slot
  long long cap;       // slot entries allocated
  int fp32, dfrec, nt; // record precision (FP32, double-float, else FP64); weighting
  double tau;
};
int launch_mlp_infer(const float* params, long long m, const int* m_dev, long long cap,
                     const float* X, const InferSink& out, unsigned* status, cudaStream_t s);
int mlp_grad_blocks(long long m);
int mlp_configure();  // inference grid from the device's occupancy; call once (returns != 0 on error)

}  // namespace psm
