// psm_capi.cu -- the engine behind include/psm.h: device buffers, the order of
// the kernels within one time step, CUDA-graph replay, error and status
// handling.  Host arithmetic that feeds the device (particle volume, mass,
// inertia, f(r) of Eq. 26) is compiled with -ffp-contract=off.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/psm.h"
#include "psm_internal.cuh"
#include "host_dem.h"

namespace psm {
int launch_map_mlp(MapParams P, cudaStream_t s);
}

using namespace psm;

struct Alloc {
  void* ptr;
};

// DEM neighbour lists: margin beyond contact (lattice units; a particle may
// move up to half of it within one LBM step) and capacity per particle
constexpr float kDemSkin = 1.0f;
constexpr int kDemListCap = 64;

struct psm_ctx {
  psm_options opt{};
  Grid g{};
  OpenBC bc{};         // constants of the open z faces
  bool open = false;   // an inflow or outflow face exists
  double tau = 0.6, omega_p = 0, omega_m = 0;
  int relax = 0, fp32 = 0, aa = 0;
  int prec = PREC_FP64;  // PDF storage and collision arithmetic (PREC_*)
  LbmPlan plan{};       // staged collision kernel (plan.stages = 0: not used)
  cudaStream_t stream = nullptr;
  cudaStream_t capture = nullptr;
  std::vector<void*> allocs;
  void* buf[2] = {nullptr, nullptr};
  int cur = 0;        // pull: buffer holding f~ of the last step
  int parity = 0;     // AA: 0 = buffer holds streamed PDFs (next step even)
  Coverage cov{};
  Slots slots{};
  StepConst* sc = nullptr;
  unsigned* status = nullptr;
  double* partials = nullptr;
  Particles p{};
  std::vector<void*> palloc;  // particle-sized allocations
  bool any_free = false;
  bool need_map = false;
  bool need_pack = false;
  double G[3] = {0, 0, 0};
  double log_e = 0;
  int dem_nc[3] = {1, 1, 1};   // DEM bins per axis
  float dem_h[3] = {1, 1, 1};
  int dem_nbins = 1;
  int* dem_bins = nullptr;       // count, start, cursor (3 * dem_nbins)
  int* dem_items = nullptr;      // bin_items, pbin, nbr_cnt (3 * n)
  int* dem_nbr = nullptr;        // n * kDemListCap
  float4* dem_xbuild = nullptr;  // n
  double* wtab = nullptr;        // B of the sampled counts (eps_n^3 < 513)
  bool have_wtab = false;
  unsigned* dem_bar = nullptr;   // grid barrier of the DEM step kernel
  int dem_blocks = 0;            // resident blocks of the DEM step kernel
  float* mlp = nullptr;   // FP32 parameters on the device
  bool have_mlp = false;
  float4* wl_X = nullptr;  // 8^3 sampling worklist (per list entry)
  int* wl_work = nullptr;
  int* wl_cnt = nullptr;     // its length per particle
  float* mlp_X = nullptr; // MLP worklist inputs (float4 per slot)
  float* mlp_lin = nullptr;  // linear approximation per worklist item
  int* mlp_work = nullptr;   // entry index per worklist item
  int* mlp_count = nullptr;
  long long mlp_cap = 0;
  long long* list_off = nullptr;  // per-particle entry lists (force reduction)
  int* list = nullptr;
  int* list_cnt = nullptr;
  int* list_net = nullptr;   // surrogate mode: the network's cells per particle
  void* boxes = nullptr;     // per-particle box of cells (mapping set-up)
  bool error_state = false;
  std::string err;
  // graphs: [buffer or parity][with mapping]
  // [state][with mapping][DEM on the device]
  cudaGraphExec_t graph[2][2][2] = {};
  long graph_launches[2][2][2] = {};
  long launches = 0;
  bool timing = false;
  static constexpr int kTimedRing = 64;   // steps whose events are in flight
  std::vector<cudaEvent_t> tev;           // 5 events per ring slot
  int tpending = 0;                       // recorded, not yet accumulated
  cudaEvent_t* ev = nullptr;              // events of the step being enqueued
  double t_ms[5] = {0, 0, 0, 0, 0};
};

namespace {

// NVTX range over a scope of host work (a tracing tool shows the engine's
// calls and, outside graph replay, the phases each step enqueues)
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

psm_status fail(psm_ctx* c, psm_status st, const std::string& msg) {
  if (c) c->err = msg;
  return st;
}

#define CK(call)                                                                         \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(c, PSM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
  } while (0)

void* dalloc(psm_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  void* p = nullptr;
  if (c->opt.alloc) {
    p = c->opt.alloc(bytes, c->opt.alloc_user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  return p;
}

void dfree(psm_ctx* c, void* p) {
  if (!p) return;
  if (c->opt.free) c->opt.free(p, c->opt.alloc_user);
  else if (!c->opt.alloc) cudaFree(p);
}

template <typename T>
T* alloc_n(psm_ctx* c, size_t n, std::vector<void*>& owner) {
  void* p = dalloc(c, sizeof(T) * n);
  owner.push_back(p);  // NULL too: callers scan `owner` for failed allocations
  return static_cast<T*>(p);
}

void free_graphs(psm_ctx* c) {
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j)
      for (int k = 0; k < 2; ++k)
        if (c->graph[i][j][k]) {
          cudaGraphExecDestroy(c->graph[i][j][k]);
          c->graph[i][j][k] = nullptr;
        }
}

void free_particles(psm_ctx* c) {
  for (void* q : c->palloc) dfree(c, q);
  c->palloc.clear();
  c->p = Particles{};
  c->slots = Slots{};
  c->wl_X = nullptr;
  c->wl_work = nullptr;
  c->wl_cnt = nullptr;
  c->mlp_X = nullptr;
  c->mlp_lin = nullptr;
  c->mlp_work = nullptr;
  c->mlp_cap = 0;
  c->list_off = nullptr;
  c->list = nullptr;
  c->dem_bins = nullptr;
  c->dem_items = nullptr;
  c->dem_nbr = nullptr;
  c->dem_xbuild = nullptr;
  c->list_cnt = nullptr;
  c->list_net = nullptr;
  c->boxes = nullptr;
}

MapParams map_params(psm_ctx* c) {
  MapParams P{};
  P.g = c->g;
  P.p = c->p;
  P.cov = c->cov;
  P.s = c->slots;
  P.fp32 = c->fp32;
  P.dfrec = c->prec == PREC_DF;
  P.eps_mode = c->opt.eps_mode;
  P.eps_n = c->opt.eps_n;
  P.weighting = c->opt.weighting;
  P.tau = c->tau;
  P.status = c->status;
  P.sc = c->sc;
  for (int a = 0; a < 3; ++a) {
    // no counter force for the particles' weight when the fluid has open faces
    P.G[a] = c->open ? 0.0 : c->G[a];
    P.fbody[a] = c->opt.body_force[a];
  }
  P.omega_p = c->omega_p;
  P.omega_m = c->omega_m;
  P.mlp = c->have_mlp ? c->mlp : nullptr;
  P.wtab = c->have_wtab ? c->wtab : nullptr;
  P.partials = c->partials;
  P.wl_X = c->wl_X;
  P.wl_work = c->wl_work;
  P.wl_cnt = c->wl_cnt;
  P.mlp_X = c->mlp_X;
  P.mlp_lin = c->mlp_lin;
  P.mlp_cap = c->mlp_cap;
  P.mlp_work = c->mlp_work;
  P.mlp_count = c->mlp_count;
  P.list_off = c->list_off;
  P.list = c->list;
  P.list_cnt = c->list_cnt;
  P.list_net = c->list_net;
  P.boxes = c->boxes;
  return P;
}

// Eq. 27 and Eq. 26: f(r) = V_a(r) - r + 1/2 (same closed form as printed)
double jones_fr(double r) {
  double r2 = r * r;
  double s = std::sqrt(r2 - 0.5);
  double Va = (1.0 / 12.0 - r2) * std::atan((0.5 * s) / (0.5 - r2)) + s / 3.0 +
              (r2 - 1.0 / 12.0) * std::atan(0.5 / s) -
              4.0 / 3.0 * r2 * r * std::atan(0.25 / (r * s));
  return Va - r + 0.5;
}

// Kernels of one time step, in the order of the paper's Fig. "implementation":
// mapping (when needed), stream + PSM collide, force/torque reduction, DEM
// (unless the host runs it: dem = false).
int enqueue_step(psm_ctx* c, bool with_map, cudaStream_t s, bool dem = true) {
  int n = 0;
  MapParams MP = map_params(c);
  if (c->timing) cudaEventRecord(c->ev[0], s);
  if (with_map) {
    NvtxRange r("psm mapping");
    if (c->opt.eps_mode == PSM_EPS_MLP) n += launch_map_mlp(MP, s);
    else n += launch_map(MP, s);
    n += launch_step_const(MP, s);
  }
  if (c->fp32 && c->p.n > 0 && (with_map || c->any_free)) n += launch_pack_particles(c->p, s);
  if (c->timing) cudaEventRecord(c->ev[1], s);
  LbmParams L{};
  L.g = c->g;
  int mode = 0;
  if (c->aa) {
    L.src = c->buf[0];
    L.dst = c->buf[0];
    mode = c->parity == 0 ? 1 : 2;
  } else {
    L.src = c->buf[c->cur];
    L.dst = c->buf[1 - c->cur];
  }
  if (c->p.n > 0) {
    L.mask = c->cov.mask;
    L.base = c->cov.base;
    L.full = c->cov.full;
    L.slot_Fc = c->slots.Fc;
    L.slot_V = c->slots.V;
    L.slot_cap = c->slots.cap;
  }
  L.sc = c->sc;
  L.omega_p = c->omega_p;
  L.omega_m = c->omega_m;
  L.bc = c->bc;
  L.status = c->status;
  L.tile_rows = c->plan.tile_rows;
  L.ntiles = c->plan.ntiles;
  L.stages = c->plan.stages;
  L.blocks = c->plan.blocks;
  L.smem = c->plan.smem;
  L.pf_ahead = c->plan.pf_ahead;
  {
    NvtxRange r("psm stream-collide");
    n += launch_lbm(L, c->prec, mode, s);
  }
  if (c->timing) cudaEventRecord(c->ev[2], s);
  if (c->p.n > 0) {
    NvtxRange r("psm force-reduce");
    n += launch_force_reduce(MP, s);
  }
  if (c->timing) cudaEventRecord(c->ev[3], s);
  if (dem && c->any_free) {
    NvtxRange r("psm dem");
    DemParams D{};
    D.g = c->g;
    D.p = c->p;
    D.kn = c->opt.k_n;
    D.kt_ratio = c->opt.kt_ratio;
    D.log_e = c->log_e;
    D.dt = 1.0 / c->opt.dem_subcycles;
    for (int a = 0; a < 3; ++a) {
      D.gravity[a] = c->opt.gravity[a];
      D.nc[a] = c->dem_nc[a];
      D.h[a] = c->dem_h[a];
    }
    D.status = c->status;
    D.skin = kDemSkin;
    D.K = kDemListCap;
    D.nbins = c->dem_nbins;
    D.bin_count = c->dem_bins;
    D.bin_start = c->dem_bins + c->dem_nbins;
    D.bin_cursor = c->dem_bins + 2 * c->dem_nbins;
    D.bin_items = c->dem_items;
    D.pbin = c->dem_items + c->p.n;
    D.nbr_cnt = c->dem_items + 2 * c->p.n;
    D.nbr = c->dem_nbr;
    D.xbuild = c->dem_xbuild;
    D.bar = c->dem_bar;
    D.max_blocks = c->dem_blocks;
    n += launch_dem_step(D, c->opt.dem_subcycles, s);
  }
  if (c->timing) cudaEventRecord(c->ev[4], s);
  return n;
}

// adds the event intervals of the pending timed steps to t_ms
cudaError_t flush_timing(psm_ctx* c) {
  for (int k = 0; k < c->tpending; ++k) {
    cudaEvent_t* e = &c->tev[5 * k];
    cudaError_t err = cudaEventSynchronize(e[4]);
    if (err != cudaSuccess) return err;
    for (int i = 0; i < 4; ++i) {
      float ms = 0;
      cudaEventElapsedTime(&ms, e[i], e[i + 1]);
      c->t_ms[i] += ms;
    }
    c->t_ms[4] += 1;
  }
  c->tpending = 0;
  return cudaSuccess;
}

void advance_state(psm_ctx* c) {
  if (c->aa) c->parity ^= 1;
  else c->cur ^= 1;
}

int state_index(const psm_ctx* c) { return c->aa ? c->parity : c->cur; }

psm_status ensure_mapped(psm_ctx* c) {
  if (!c->need_map) return PSM_OK;
  MapParams MP = map_params(c);
  if (c->opt.eps_mode == PSM_EPS_MLP) launch_map_mlp(MP, c->stream);
  else launch_map(MP, c->stream);
  launch_step_const(MP, c->stream);
  if (c->fp32 && c->p.n > 0) launch_pack_particles(c->p, c->stream);
  CK(cudaGetLastError());
  c->need_map = c->any_free;
  return PSM_OK;
}

psm_status read_status(psm_ctx* c) {
  unsigned st = 0;
  CK(cudaMemcpyAsync(&st, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (st) {
    CK(cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream));
    c->error_state = true;
    if (st & ST_SLOT_OVERFLOW)
      return fail(c, PSM_ERR_SLOT_OVERFLOW, "a cell lies within reach of more than two particles");
    if (st & ST_NONFINITE) return fail(c, PSM_ERR_NONFINITE, "non-finite hydrodynamic force");
    if (st & ST_CONTACT_OVERFLOW)
      return fail(c, PSM_ERR_STATE, "more DEM neighbours than the list holds");
    if (st & ST_DEM_SKIN)
      return fail(c, PSM_ERR_STATE,
                  "a particle moved more than half the DEM neighbour-list skin in one step");
    if (st & ST_TIMEOUT)
      return fail(c, PSM_ERR_TIMEOUT, "a bounded wait in the collision kernel gave up");
    return fail(c, PSM_ERR_STATE, "device status " + std::to_string(st));
  }
  return PSM_OK;
}

psm_status canonical(psm_ctx* c, double** out, const BoxSel* box = nullptr) {
  const BoxSel B = box ? *box : BoxSel{0, 0, 0, c->g.nx, c->g.ny, c->g.nz};
  const size_t N = (size_t)B.bx * B.by * B.bz;
  double* f = static_cast<double*>(dalloc(c, sizeof(double) * Q * N));
  if (!f) return fail(c, PSM_ERR_OOM, "allocator returned NULL");
  launch_to_canonical(c->g, c->aa ? c->buf[0] : c->buf[c->cur], c->prec, c->parity, c->aa, B, f,
                      c->stream);
  *out = f;
  CK(cudaGetLastError());
  return PSM_OK;
}

}  // namespace

// ---- checkpoint: the state of the time stepper, exactly.  Layout (native
// byte order, little-endian on the supported hosts): a header of int64
// fields, then the PDF storage as stored (the form's own values), the
// per-particle arrays, the surrogate's parameters when set.
namespace {
constexpr char kCkptMagic[8] = {'P', 'S', 'M', 'C', 'K', 'P', 'T', '2'};
enum {
  CK_NX, CK_NY, CK_NZ, CK_WX, CK_WY, CK_WZ, CK_PREC, CK_AA, CK_RELAX, CK_PARITY, CK_N,
  CK_MLP, CK_DEM, CK_FIELDS
};
// the z faces in the header: 0 periodic, 1 walls, and with an open face
// 1 + 4 * type(-z) + 16 * type(+z)
long long z_code(const Grid& g) {
  if (!g.wall[2]) return 0;
  if (g.zface[0] < FACE_INFLOW && g.zface[1] < FACE_INFLOW) return 1;
  return 1 + 4LL * g.zface[0] + 16LL * g.zface[1];
}
struct CkptHeader {
  char magic[8];
  long long v[CK_FIELDS];
  double tau, omega_m, G[3];
};

bool write_all(FILE* f, const void* p, size_t bytes) {
  return bytes == 0 || fwrite(p, 1, bytes, f) == bytes;
}
bool read_all(FILE* f, void* p, size_t bytes) {
  return bytes == 0 || fread(p, 1, bytes, f) == bytes;
}

// the per-particle device arrays of a checkpoint, in file order, with their
// element counts (multiples of n) and sizes
struct CkptArray {
  void* dev;
  size_t per, esz;
};
std::vector<CkptArray> ckpt_arrays(psm_ctx* c) {
  Particles& P = c->p;
  return {{P.x, 3, 8},  {P.u, 3, 8},   {P.om, 3, 8},   {P.r, 1, 8},    {P.m, 1, 8},
          {P.I, 1, 8},  {P.vol, 1, 8}, {P.fr, 1, 8},   {P.fixed, 1, 1}, {P.Fh, 3, 8},
          {P.Th, 3, 8}, {P.Fold, 3, 8}, {P.Told, 3, 8}, {P.hcnt[0], 1, 4},
          {P.hj[0], kDemListCap, 4}, {P.hd[0], 3 * kDemListCap, 8}};
}
}  // namespace

extern "C" {

void psm_default_options(psm_options* o) {
  std::memset(o, 0, sizeof(*o));
  o->magic = 3.0 / 16.0;
  o->precision = PSM_FP64;
  o->streaming = PSM_PULL;
  o->eps_mode = PSM_EPS_SUPERSAMPLE;
  o->eps_n = 4;
  o->weighting = PSM_W_NT;
  o->k_n = 1e3;
  o->restitution = 0.9;
  o->dem_subcycles = 10;
  o->dem = 1;
  o->deterministic = 1;
  o->use_graphs = 1;
  o->bc_density = 1.0;
  o->kt_ratio = 2.0 / 7.0;
}

psm_status psm_create(const psm_grid* grid, double tau, psm_relax relax, const psm_options* opt,
                      psm_ctx** out) {
  if (!out) return PSM_ERR_ARG;
  *out = nullptr;
  if (!grid || !opt) return PSM_ERR_ARG;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return PSM_ERR_ARG;
  static_assert(FACE_INFLOW == PSM_FACE_INFLOW && FACE_OUTFLOW == PSM_FACE_OUTFLOW &&
                    FACE_WALL == PSM_FACE_WALL && FACE_PERIODIC == PSM_FACE_PERIODIC,
                "face types");
  bool open = false;
  for (int f = 0; f < 6; ++f) {
    if (grid->wall[f] < PSM_FACE_PERIODIC || grid->wall[f] > PSM_FACE_OUTFLOW) return PSM_ERR_ARG;
    if (grid->wall[f] >= PSM_FACE_INFLOW) {
      if (f < 4) return PSM_ERR_ARG;  // open faces on the z faces only
      open = true;
    }
  }
  for (int a = 0; a < 3; ++a)
    if ((grid->wall[2 * a] != 0) != (grid->wall[2 * a + 1] != 0)) return PSM_ERR_ARG;
  if (open && opt->streaming != PSM_PULL) return PSM_ERR_ARG;
  if (open && !(opt->bc_density > 0.0 && std::isfinite(opt->bc_density))) return PSM_ERR_ARG;
  for (int a = 0; a < 3; ++a)
    if (!std::isfinite(opt->bc_velocity[a])) return PSM_ERR_ARG;
  if (!(tau > 0.5) || !std::isfinite(tau)) return PSM_ERR_ARG;
  if (relax != PSM_SRT && relax != PSM_TRT) return PSM_ERR_ARG;
  if (opt->precision != PSM_FP64 && opt->precision != PSM_FP32_DEV &&
      opt->precision != PSM_FP64_DF)
    return PSM_ERR_ARG;
  if (opt->streaming != PSM_PULL && opt->streaming != PSM_AA) return PSM_ERR_ARG;
  // only the fixed-order reduction is built: results are bitwise reproducible
  if (opt->deterministic != 1) return PSM_ERR_ARG;
  if (opt->eps_mode < 0 || opt->eps_mode > 2) return PSM_ERR_ARG;
  if (opt->eps_n < 1 || opt->eps_n > 16) return PSM_ERR_ARG;
  if (opt->weighting != PSM_W_EPS && opt->weighting != PSM_W_NT) return PSM_ERR_ARG;
  if (relax == PSM_TRT && !(opt->magic > 0.0)) return PSM_ERR_ARG;
  if (opt->dem && (opt->dem_subcycles < 1 || !(opt->k_n > 0) || !(opt->restitution > 0) ||
                   opt->restitution > 1.0 || !(opt->kt_ratio >= 0.0) ||
                   !std::isfinite(opt->kt_ratio)))
    return PSM_ERR_ARG;
  const long long nxp = ((grid->nx + 31) / 32) * 32LL;
  const long long ncell = nxp * grid->ny * grid->nz;
  if (ncell >= (1LL << 31)) return PSM_ERR_ARG;

  psm_ctx* c = new psm_ctx();
  c->opt = *opt;
  c->tau = tau;
  c->relax = relax;
  c->fp32 = opt->precision == PSM_FP32_DEV;
  c->prec = opt->precision == PSM_FP32_DEV ? PREC_FP32
            : opt->precision == PSM_FP64_DF ? PREC_DF
                                             : PREC_FP64;
  c->aa = opt->streaming == PSM_AA;
  c->stream = static_cast<cudaStream_t>(opt->stream);
  c->omega_p = 1.0 / tau;
  c->omega_m = relax == PSM_TRT ? 1.0 / (0.5 + opt->magic / (tau - 0.5)) : c->omega_p;
  c->log_e = opt->restitution > 0 ? std::log(opt->restitution) : 0.0;
  Grid& g = c->g;
  g.nx = grid->nx;
  g.ny = grid->ny;
  g.nz = grid->nz;
  g.nxp = (int)nxp;
  for (int a = 0; a < 3; ++a) g.wall[a] = grid->wall[2 * a] ? 1 : 0;
  g.zface[0] = grid->wall[4];
  g.zface[1] = grid->wall[5];
  c->open = open;
  {
    // open faces: 6 w_q c_q.U_b per direction (inflow), rho_b - 1 (outflow)
    static const int cq[19][3] = {{0, 0, 0},  {1, 0, 0},   {-1, 0, 0}, {0, 1, 0},  {0, -1, 0},
                                  {0, 0, 1},  {0, 0, -1},  {1, 1, 0},  {-1, -1, 0}, {1, -1, 0},
                                  {-1, 1, 0}, {1, 0, 1},   {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
                                  {0, 1, 1},  {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
    for (int q = 0; q < Q; ++q) {
      const double w = q == 0 ? 1.0 / 3.0 : (q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
      const double* U = opt->bc_velocity;
      c->bc.in[q] = 6.0 * w * (cq[q][0] * U[0] + cq[q][1] * U[1] + cq[q][2] * U[2]);
    }
    c->bc.rho1 = opt->bc_density - 1.0;
  }
  g.wpr = (int)(nxp / 32);
  g.ncell = ncell;
  g.nwords = ncell / 32;
  g.div_wpr = make_fastdiv((unsigned)g.wpr);
  g.div_ny = make_fastdiv((unsigned)g.ny);

  auto bail = [&](psm_status st, const char* msg) {
    psm_status r = st;
    c->err = msg;
    psm_destroy(c);
    return r;
  };
  const size_t esz = c->fp32 ? sizeof(float) : sizeof(double);
  const int nbuf = c->aa ? 1 : 2;
  for (int b = 0; b < nbuf; ++b) {
    c->buf[b] = alloc_n<unsigned char>(c, esz * Q * (size_t)ncell, c->allocs);
    if (!c->buf[b]) return bail(PSM_ERR_OOM, "allocator returned NULL for the PDF field");
  }
  c->cov.mask = alloc_n<uint32_t>(c, (size_t)g.nwords, c->allocs);
  c->cov.base = alloc_n<int>(c, (size_t)g.nwords, c->allocs);
  c->cov.dup = alloc_n<uint32_t>(c, (size_t)g.nwords, c->allocs);
  if (c->prec == PREC_FP64) {
    c->cov.full = alloc_n<uint32_t>(c, (size_t)g.nwords, c->allocs);
    if (!c->cov.full) return bail(PSM_ERR_OOM, "allocator returned NULL");
  }
  c->cov.nblocks = (g.nwords + 1023) / 1024;
  c->cov.blocksum = alloc_n<int>(c, (size_t)c->cov.nblocks, c->allocs);
  c->cov.ncov = alloc_n<int>(c, 1, c->allocs);
  c->sc = alloc_n<StepConst>(c, 1, c->allocs);
  c->status = alloc_n<unsigned>(c, 1, c->allocs);
  c->partials = alloc_n<double>(c, MAP_PARTIALS * 4, c->allocs);
  c->mlp = alloc_n<float>(c, PSM_MLP_PARAMS, c->allocs);
  c->mlp_count = alloc_n<int>(c, 1, c->allocs);
  c->dem_bar = alloc_n<unsigned>(c, 4, c->allocs);
  // 513 doubles, 513 floats, 513 double-float pairs
  c->wtab = alloc_n<double>(c, 513 + 257 + 513, c->allocs);
  if (!c->cov.mask || !c->cov.base || !c->cov.dup || !c->cov.blocksum || !c->cov.ncov || !c->sc ||
      !c->status || !c->partials || !c->mlp || !c->mlp_count || !c->dem_bar || !c->wtab)
    return bail(PSM_ERR_OOM, "allocator returned NULL");
  cudaStream_t s = c->stream;
  bool ok = true;
  for (int b = 0; b < nbuf; ++b)
    ok = ok && cudaMemsetAsync(c->buf[b], 0, esz * Q * (size_t)ncell, s) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->cov.mask, 0, sizeof(uint32_t) * g.nwords, s) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->cov.dup, 0, sizeof(uint32_t) * g.nwords, s) == cudaSuccess;
  if (c->cov.full)
    ok = ok && cudaMemsetAsync(c->cov.full, 0, sizeof(uint32_t) * g.nwords, s) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->status, 0, sizeof(unsigned), s) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->dem_bar, 0, 4 * sizeof(unsigned), s) == cudaSuccess;
  ok = ok && cudaMemsetAsync(c->cov.ncov, 0, sizeof(int), s) == cudaSuccess;
  StepConst h{};
  h.ncells = (double)g.nx * g.ny * g.nz;
  h.vfluid = h.ncells;
  ok = ok && cudaMemcpyAsync(c->sc, &h, sizeof(h), cudaMemcpyHostToDevice, s) == cudaSuccess;
  ok = ok && cudaStreamSynchronize(s) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    return bail(PSM_ERR_CUDA, "initialisation of device buffers failed");
  }
  if (lbm_configure() != 0) {
    cudaGetLastError();
    return bail(PSM_ERR_CUDA, "could not set the shared-memory size of the collision kernel");
  }
  if (mlp_configure() != 0) {
    cudaGetLastError();
    return bail(PSM_ERR_CUDA, "occupancy query of the inference kernel failed");
  }
  c->dem_blocks = dem_max_blocks();
  if (c->dem_blocks <= 0) {
    cudaGetLastError();
    return bail(PSM_ERR_CUDA, "occupancy query of the DEM kernel failed");
  }
  if (lbm_plan(g, c->prec, c->aa, &c->plan) != 0) {
    cudaGetLastError();
    return bail(PSM_ERR_CUDA, "occupancy query of the collision kernel failed");
  }
  launch_step_const(map_params(c), s);
  c->have_wtab = launch_weight_table(c->opt.eps_n, c->tau, c->opt.weighting, c->wtab, s) > 0;
  if (cudaStreamCreateWithFlags(&c->capture, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return bail(PSM_ERR_CUDA, "cudaStreamCreate failed");
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return bail(PSM_ERR_CUDA, "initialisation kernel failed");
  }
  *out = c;
  return PSM_OK;
}

// volume, mass and moment of inertia of a sphere (fluid density 1)
static void sphere_constants(double r, double density, double* vol, double* m, double* I) {
  const double PI = 3.14159265358979323846;
  *vol = 4.0 / 3.0 * PI * r * r * r;
  *m = density * *vol;
  *I = 0.4 * *m * r * r;
}

psm_status psm_set_particles(psm_ctx* c, int n, const double* x, const double* r,
                             const double* u, const double* omega, const double* density,
                             const unsigned char* fixed) {
  if (!c) return PSM_ERR_ARG;
  if (n < 0) return fail(c, PSM_ERR_ARG, "negative particle count");
  if (n > 0 && (!x || !r || !u || !omega || !density))
    return fail(c, PSM_ERR_ARG, "NULL particle array");
  const int dims[3] = {c->g.nx, c->g.ny, c->g.nz};
  std::vector<double> hx(3 * (size_t)n), vol(n), m(n), I(n), fr(n), Fold(3 * (size_t)n, 0.0);
  std::vector<unsigned char> fx(n, 0);
  double G[3] = {0, 0, 0};
  bool any_free = false;
  const double PI = 3.14159265358979323846;
  long long cap = 0;
  // cells within reach of a sphere: their unit cubes lie in the ball of
  // radius r + sqrt(3), so at most 4/3 pi (r + sqrt(3))^3 of them
  std::vector<long long> loff(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    if (!(r[i] > 0.0) || !std::isfinite(r[i]) || !(density[i] > 0.0))
      return fail(c, PSM_ERR_ARG, "radius and density must be positive");
    for (int a = 0; a < 3; ++a) {
      double v = x[3 * i + a];
      if (!std::isfinite(v) || !std::isfinite(u[3 * i + a]) || !std::isfinite(omega[3 * i + a]))
        return fail(c, PSM_ERR_ARG, "non-finite particle state");
      if (!c->g.wall[a]) {
        if (2.0 * r[i] + 4.0 > dims[a])
          return fail(c, PSM_ERR_ARG, "particle too large for the periodic box");
        v = std::fmod(v, (double)dims[a]);
        if (v < 0) v += dims[a];
      }
      hx[3 * i + a] = v;
    }
    sphere_constants(r[i], density[i], &vol[i], &m[i], &I[i]);
    fr[i] = r[i] * r[i] > 0.5 ? jones_fr(r[i]) : 0.5;
    fx[i] = fixed ? (fixed[i] ? 1 : 0) : 0;
    if (!fx[i] && c->opt.dem) {
      any_free = true;
      for (int a = 0; a < 3; ++a) {
        Fold[3 * i + a] = (m[i] - vol[i]) * c->opt.gravity[a];
        G[a] += (m[i] - vol[i]) * c->opt.gravity[a];
      }
    }
    const double R = r[i] + std::sqrt(3.0);
    const long long ci = (long long)(4.0 / 3.0 * PI * R * R * R) + 1;
    cap += ci;
    loff[i + 1] = loff[i] + ci;
  }
  // DEM bins: edge >= the largest diameter plus the skin, at least three
  // bins along an axis or a single one, at most max(4096, 8 n) bins
  double rmax = 0.0;
  for (int i = 0; i < n; ++i) rmax = r[i] > rmax ? r[i] : rmax;
  int nc[3];
  for (int a = 0; a < 3; ++a) {
    nc[a] = (int)std::floor(dims[a] / (2.0 * rmax + kDemSkin + 0.01));
    if (nc[a] < 3) nc[a] = 1;
  }
  const long long bin_cap = std::max(4096LL, 8LL * n);
  while ((long long)nc[0] * nc[1] * nc[2] > bin_cap) {
    const int a = nc[0] >= nc[1] && nc[0] >= nc[2] ? 0 : (nc[1] >= nc[2] ? 1 : 2);
    nc[a] = nc[a] / 2 < 3 ? 1 : nc[a] / 2;
  }
  for (int a = 0; a < 3; ++a) {
    c->dem_nc[a] = nc[a];
    c->dem_h[a] = (float)((double)dims[a] / nc[a]);
  }
  c->dem_nbins = nc[0] * nc[1] * nc[2];
  const long long list_total = cap > 0 ? cap : 1;
  if (cap > c->g.ncell) cap = c->g.ncell;
  free_graphs(c);
  free_particles(c);
  Particles& P = c->p;
  const size_t n1 = n > 0 ? n : 1, n3 = 3 * n1, n4 = 4 * n1;
  P.n = n;
  P.x = alloc_n<double>(c, n3, c->palloc);
  P.u = alloc_n<double>(c, n3, c->palloc);
  P.om = alloc_n<double>(c, n3, c->palloc);
  P.r = alloc_n<double>(c, n1, c->palloc);
  P.m = alloc_n<double>(c, n1, c->palloc);
  P.I = alloc_n<double>(c, n1, c->palloc);
  P.vol = alloc_n<double>(c, n1, c->palloc);
  P.fr = alloc_n<double>(c, n1, c->palloc);
  P.fixed = alloc_n<unsigned char>(c, n1, c->palloc);
  P.Fh = alloc_n<double>(c, n3, c->palloc);
  P.Th = alloc_n<double>(c, n3, c->palloc);
  P.Fold = alloc_n<double>(c, n3, c->palloc);
  P.Told = alloc_n<double>(c, n3, c->palloc);
  P.Fc = alloc_n<double>(c, n3, c->palloc);
  P.xf = alloc_n<float>(c, n4, c->palloc);
  P.uf = alloc_n<float>(c, n4, c->palloc);
  P.omf = alloc_n<float>(c, n4, c->palloc);
  P.x2 = alloc_n<double>(c, n3, c->palloc);
  P.u2 = alloc_n<double>(c, n3, c->palloc);
  P.xf2 = alloc_n<float>(c, n4, c->palloc);
  P.om2 = alloc_n<double>(c, n3, c->palloc);
  for (int b = 0; b < 2; ++b) {
    P.hcnt[b] = alloc_n<int>(c, n1, c->palloc);
    P.hj[b] = alloc_n<int>(c, n1 * kDemListCap, c->palloc);
    P.hd[b] = alloc_n<double>(c, n1 * kDemListCap * 3, c->palloc);
  }
  Slots& S = c->slots;
  const size_t cp = cap > 0 ? (size_t)cap : 1;
  S.cap = (long long)cp;
  S.cell = alloc_n<int>(c, cp, c->palloc);
  S.pid = alloc_n<int2>(c, cp, c->palloc);
  S.cnt = alloc_n<int>(c, cp, c->palloc);
  S.Fc = alloc_n<unsigned char>(c, cp * 6 * (c->fp32 ? 4 : 8), c->palloc);
  S.V = alloc_n<unsigned char>(c, cp * 8 * (c->fp32 ? 4 : 8), c->palloc);
  c->list_off = alloc_n<long long>(c, (size_t)n + 1, c->palloc);
  c->list = alloc_n<int>(c, (size_t)list_total, c->palloc);
  c->list_cnt = alloc_n<int>(c, n1, c->palloc);
  c->boxes = alloc_n<unsigned char>(c, n1 * map_box_bytes(), c->palloc);
  c->dem_bins = alloc_n<int>(c, 3 * (size_t)c->dem_nbins, c->palloc);
  c->dem_items = alloc_n<int>(c, 3 * n1, c->palloc);
  c->dem_nbr = alloc_n<int>(c, n1 * kDemListCap, c->palloc);
  c->dem_xbuild = alloc_n<float4>(c, n1, c->palloc);
  // the 8^3 count pass's worklist: 8^3 sampling, and the surrogate's shared
  // cells (its fallback samples 8^3 points)
  if ((c->opt.eps_mode == PSM_EPS_SUPERSAMPLE || c->opt.eps_mode == PSM_EPS_MLP) &&
      c->opt.eps_n == 8) {
    c->wl_X = alloc_n<float4>(c, (size_t)list_total, c->palloc);
    c->wl_work = alloc_n<int>(c, (size_t)list_total, c->palloc);
    c->wl_cnt = alloc_n<int>(c, n1, c->palloc);
  }
  if (c->opt.eps_mode == PSM_EPS_MLP) {
    c->mlp_cap = (long long)cp;
    c->mlp_X = alloc_n<float>(c, 4 * cp, c->palloc);
    c->mlp_lin = alloc_n<float>(c, cp, c->palloc);
    c->mlp_work = alloc_n<int>(c, cp, c->palloc);
    c->list_net = alloc_n<int>(c, n1, c->palloc);
  }
  for (void* q : c->palloc)
    if (!q) {
      free_particles(c);
      return fail(c, PSM_ERR_OOM, "allocator returned NULL for particle buffers");
    }
  cudaStream_t s = c->stream;
  const size_t b3 = sizeof(double) * 3 * n, b1 = sizeof(double) * n;
  if (n > 0) {
    CK(cudaMemcpyAsync(P.x, hx.data(), b3, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(P.u, u, b3, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(P.om, omega, b3, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(P.r, r, b1, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(P.m, m.data(), b1, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(P.I, I.data(), b1, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(P.vol, vol.data(), b1, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(P.fr, fr.data(), b1, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(P.fixed, fx.data(), n, cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(P.Fold, Fold.data(), b3, cudaMemcpyHostToDevice, s));
    CK(cudaMemsetAsync(P.Told, 0, b3, s));
    CK(cudaMemsetAsync(P.Fh, 0, b3, s));
    CK(cudaMemsetAsync(P.Th, 0, b3, s));
    CK(cudaMemsetAsync(P.Fc, 0, b3, s));
    // new particles: no tangential contact history
    CK(cudaMemsetAsync(P.hcnt[0], 0, sizeof(int) * n, s));
    CK(cudaMemsetAsync(P.hcnt[1], 0, sizeof(int) * n, s));
  }
  CK(cudaMemcpyAsync(c->list_off, loff.data(), sizeof(long long) * (n + 1),
                     cudaMemcpyHostToDevice, s));
  for (int a = 0; a < 3; ++a) c->G[a] = G[a];
  c->any_free = any_free;
  c->need_map = true;
  c->error_state = false;
  CK(cudaMemsetAsync(c->status, 0, sizeof(unsigned), s));
  CK(cudaMemsetAsync(c->dem_bar, 0, 4 * sizeof(unsigned), s));
  CK(cudaStreamSynchronize(s));
  return PSM_OK;
}

// Queues one step (as a captured graph, or launch by launch when timing);
// dem = false leaves out the DEM kernel.
static psm_status launch_one_step(psm_ctx* c, bool dem) {
  const bool graphs = c->opt.use_graphs && !c->timing;
  const bool with_map = c->need_map;
  const int si = state_index(c), mi = with_map ? 1 : 0, di = dem ? 1 : 0;
  if (graphs) {
    cudaGraphExec_t& ge = c->graph[si][mi][di];
    if (!ge) {
      cudaGraph_t gr = nullptr;
      CK(cudaStreamBeginCapture(c->capture, cudaStreamCaptureModeThreadLocal));
      const int nl = enqueue_step(c, with_map, c->capture, dem);
      cudaError_t e1 = cudaStreamEndCapture(c->capture, &gr);
      if (e1 != cudaSuccess) return fail(c, PSM_ERR_CUDA, cudaGetErrorString(e1));
      cudaError_t e2 = cudaGraphInstantiate(&ge, gr, 0);
      cudaGraphDestroy(gr);
      if (e2 != cudaSuccess) {
        ge = nullptr;
        return fail(c, PSM_ERR_CUDA, cudaGetErrorString(e2));
      }
      c->graph_launches[si][mi][di] = nl;
    }
    CK(cudaGraphLaunch(ge, c->stream));
    c->launches += c->graph_launches[si][mi][di];
  } else {
    if (c->timing) {
      if (c->tpending == psm_ctx::kTimedRing) CK(flush_timing(c));
      c->ev = &c->tev[5 * c->tpending];
      ++c->tpending;
    }
    c->launches += enqueue_step(c, with_map, c->stream, dem);
  }
  CK(cudaGetLastError());
  if (with_map) c->need_map = c->any_free;
  advance_state(c);
  return PSM_OK;
}

psm_status psm_step(psm_ctx* c, int nsteps) {
  if (!c) return PSM_ERR_ARG;
  NvtxRange range("psm_step");
  if (nsteps < 0) return fail(c, PSM_ERR_ARG, "negative step count");
  if (c->error_state) return fail(c, PSM_ERR_STATE, "context is in an error state");
  c->launches = 0;
  for (int k = 0; k < nsteps; ++k) {
    const psm_status st = launch_one_step(c, true);
    if (st != PSM_OK) return st;
  }
  return read_status(c);
}

// host threads for the DEM: the request, at most the hardware threads (all
// of them for a request <= 0)
static int host_threads(int requested) {
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  return requested <= 0 || requested > hw ? hw : requested;
}

// The paper's coupling (Sec. 3.2): the LBM part of each step on the device,
// the particle dynamics on the host cores, the hydrodynamic forces sent to
// the host and the particle state sent back every step.
psm_status psm_step_host_dem(psm_ctx* c, int nsteps, int threads, double* host_ms) {
  if (!c) return PSM_ERR_ARG;
  NvtxRange range("psm_step_host_dem");
  if (host_ms) *host_ms = 0.0;
  if (nsteps < 0) return fail(c, PSM_ERR_ARG, "negative step count");
  if (c->error_state) return fail(c, PSM_ERR_STATE, "context is in an error state");
  if (!c->opt.dem) return fail(c, PSM_ERR_ARG, "the context was created without the DEM");
  c->launches = 0;
  const int n = c->p.n;
  if (n == 0 || !c->any_free) return psm_step(c, nsteps);
  threads = host_threads(threads);
  // host copy of the particle state and constants (the device copy stays the
  // reference: it is rewritten after every step)
  const size_t b3 = sizeof(double) * 3 * n, b1 = sizeof(double) * n;
  std::vector<double> x, u, om, Fo, To, Fh, Th, r, m, I, vol, hd;
  std::vector<unsigned char> fixed;
  std::vector<int> hc, hj;
  try {
    for (auto* v : {&x, &u, &om, &Fo, &To, &Fh, &Th}) v->resize(3 * (size_t)n);
    for (auto* v : {&r, &m, &I, &vol}) v->resize((size_t)n);
    fixed.resize((size_t)n);
    hc.resize((size_t)n);
    hj.resize((size_t)n * kDemListCap);
    hd.resize((size_t)n * kDemListCap * 3);
  } catch (...) {
    return fail(c, PSM_ERR_OOM, "host memory for the particle state");
  }
  static_assert(kDemListCap == kHostDemHistCap, "history layout");
  CK(cudaMemcpyAsync(x.data(), c->p.x, b3, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(u.data(), c->p.u, b3, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(om.data(), c->p.om, b3, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(Fo.data(), c->p.Fold, b3, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(To.data(), c->p.Told, b3, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(r.data(), c->p.r, b1, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(m.data(), c->p.m, b1, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(I.data(), c->p.I, b1, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(vol.data(), c->p.vol, b1, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(fixed.data(), c->p.fixed, n, cudaMemcpyDeviceToHost, c->stream));
  // the tangential contact history continues on the host (and comes back at
  // the end, for a later device step)
  const size_t bh = sizeof(int) * (size_t)n * kDemListCap;
  CK(cudaMemcpyAsync(hc.data(), c->p.hcnt[0], sizeof(int) * n, cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaMemcpyAsync(hj.data(), c->p.hj[0], bh, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(hd.data(), c->p.hd[0], 6 * bh, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  HostDemParams HP{};
  HP.dims[0] = c->g.nx;
  HP.dims[1] = c->g.ny;
  HP.dims[2] = c->g.nz;
  for (int a = 0; a < 3; ++a) {
    HP.wall[a] = c->g.wall[a];
    HP.gravity[a] = c->opt.gravity[a];
  }
  HP.kn = c->opt.k_n;
  HP.kt_ratio = c->opt.kt_ratio;
  HP.log_e = c->log_e;
  HP.dt = 1.0 / c->opt.dem_subcycles;
  HP.skin = kDemSkin;
  HP.subcycles = c->opt.dem_subcycles;
  HostDemState HS{n,         x.data(),   u.data(),  om.data(),   Fo.data(),
                  To.data(), Fh.data(),  Th.data(), r.data(),    m.data(),
                  I.data(),  vol.data(), fixed.data(), hc.data(), hj.data(), hd.data()};
  for (int k = 0; k < nsteps; ++k) {
    psm_status st = launch_one_step(c, false);
    if (st != PSM_OK) return st;
    CK(cudaStreamSynchronize(c->stream));  // the device part of the step is done
    const auto t0 = std::chrono::steady_clock::now();
    unsigned dev_status = 0;
    CK(cudaMemcpyAsync(Fh.data(), c->p.Fh, b3, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(Th.data(), c->p.Th, b3, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&dev_status, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    // an error of the device part (a non-finite force, a slot overflow) stops
    // the loop before the host DEM integrates with it
    if (dev_status) return read_status(c);
    const int moved = host_dem_step(HP, HS, threads);
    if (moved < 0) {
      c->error_state = true;
      return fail(c, PSM_ERR_OOM, "host memory for the DEM step");
    }
    CK(cudaMemcpyAsync(c->p.x, x.data(), b3, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->p.u, u.data(), b3, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->p.om, om.data(), b3, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->p.Fold, Fo.data(), b3, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->p.Told, To.data(), b3, cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemsetAsync(c->dem_bar + 2, 0, sizeof(unsigned), c->stream));  // device lists stale
    // the host buffers are reused by the next step's copies: wait for these
    CK(cudaStreamSynchronize(c->stream));
    const auto t2 = std::chrono::steady_clock::now();
    if (host_ms) *host_ms += std::chrono::duration<double, std::milli>(t2 - t0).count();
    c->need_map = true;
    if (moved) {
      c->error_state = true;
      return fail(c, PSM_ERR_STATE,
                  "a particle moved more than half the DEM neighbour-list skin in one step, "
                  "or touched more partners than the contact history holds");
    }
  }
  CK(cudaMemcpyAsync(c->p.hcnt[0], hc.data(), sizeof(int) * n, cudaMemcpyHostToDevice,
                     c->stream));
  CK(cudaMemcpyAsync(c->p.hj[0], hj.data(), bh, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->p.hd[0], hd.data(), 6 * bh, cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return read_status(c);
}

psm_status psm_dem_step_host(const psm_grid* grid, double k_n, double restitution,
                             double kt_ratio, int subcycles, const double* gravity, int n,
                             double* x, double* u, double* omega, double* F_old, double* T_old,
                             int* hist_count, int* hist_partner, double* hist_delta,
                             const double* F_hyd, const double* T_hyd, const double* r,
                             const double* density, const unsigned char* fixed, int threads) {
  if (!grid || !gravity || n < 0 || subcycles < 1 || !(k_n > 0.0) || !(restitution > 0.0) ||
      !(restitution <= 1.0) || !(kt_ratio >= 0.0) || !std::isfinite(kt_ratio))
    return PSM_ERR_ARG;
  if (n == 0) return PSM_OK;
  if (!x || !u || !omega || !F_old || !T_old || !F_hyd || !T_hyd || !r || !density)
    return PSM_ERR_ARG;
  if (!hist_count || !hist_partner || !hist_delta) return PSM_ERR_ARG;
  const int dims[3] = {grid->nx, grid->ny, grid->nz};
  HostDemParams HP{};
  for (int a = 0; a < 3; ++a) {
    if (dims[a] < 1) return PSM_ERR_ARG;
    HP.dims[a] = dims[a];
    if ((grid->wall[2 * a] != 0) != (grid->wall[2 * a + 1] != 0)) return PSM_ERR_ARG;
    HP.wall[a] = grid->wall[2 * a] ? 1 : 0;
    HP.gravity[a] = gravity[a];
  }
  HP.kn = k_n;
  HP.kt_ratio = kt_ratio;
  HP.log_e = std::log(restitution);
  HP.dt = 1.0 / subcycles;
  HP.skin = kDemSkin;
  HP.subcycles = subcycles;
  std::vector<double> vol, m, I;
  std::vector<unsigned char> fx;
  try {
    vol.resize(n);
    m.resize(n);
    I.resize(n);
    fx.resize(n);
  } catch (...) {
    return PSM_ERR_OOM;
  }
  for (int i = 0; i < n; ++i) {
    if (!(r[i] > 0.0) || !(density[i] > 0.0)) return PSM_ERR_ARG;
    sphere_constants(r[i], density[i], &vol[i], &m[i], &I[i]);
    fx[i] = fixed && fixed[i] ? 1 : 0;
  }
  threads = host_threads(threads);
  HostDemState HS{n,      x,      u,        omega,    F_old,     T_old,
                  F_hyd,  T_hyd,  r,        m.data(), I.data(),  vol.data(),
                  fx.data(), hist_count, hist_partner, hist_delta};
  const int st = host_dem_step(HP, HS, threads);
  return st < 0 ? PSM_ERR_OOM : (st ? PSM_ERR_STATE : PSM_OK);
}

psm_status psm_get_force_torque(psm_ctx* c, double* F, double* T) {
  if (!c || (c->p.n > 0 && (!F || !T))) return PSM_ERR_ARG;
  if (c->p.n == 0) return PSM_OK;
  const size_t b3 = sizeof(double) * 3 * c->p.n;
  CK(cudaMemcpyAsync(F, c->p.Fh, b3, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(T, c->p.Th, b3, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PSM_OK;
}

psm_status psm_get_particles(psm_ctx* c, double* x, double* u, double* om) {
  if (!c || (c->p.n > 0 && (!x || !u || !om))) return PSM_ERR_ARG;
  if (c->p.n == 0) return PSM_OK;
  const size_t b3 = sizeof(double) * 3 * c->p.n;
  CK(cudaMemcpyAsync(x, c->p.x, b3, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(u, c->p.u, b3, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(om, c->p.om, b3, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PSM_OK;
}

psm_status psm_get_pdfs(psm_ctx* c, double* f) {
  if (!c || !f) return PSM_ERR_ARG;
  double* d = nullptr;
  psm_status st = canonical(c, &d);
  if (st != PSM_OK) return st;
  const size_t N = (size_t)c->g.nx * c->g.ny * c->g.nz;
  cudaError_t e = cudaMemcpyAsync(f, d, sizeof(double) * Q * N, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  dfree(c, d);
  if (e != cudaSuccess) return fail(c, PSM_ERR_CUDA, cudaGetErrorString(e));
  return PSM_OK;
}

psm_status psm_get_pdfs_box(psm_ctx* c, int x0, int y0, int z0, int bx, int by, int bz,
                            double* f) {
  if (!c || !f) return PSM_ERR_ARG;
  const int n[3] = {c->g.nx, c->g.ny, c->g.nz};
  const int o[3] = {x0, y0, z0}, b[3] = {bx, by, bz};
  for (int a = 0; a < 3; ++a) {
    if (b[a] < 1 || b[a] > n[a]) return fail(c, PSM_ERR_ARG, "box extent outside 1..n");
    if (c->g.wall[a] ? (o[a] < 0 || o[a] + b[a] > n[a]) : (o[a] < -n[a] || o[a] >= 2 * n[a]))
      return fail(c, PSM_ERR_ARG, "box origin outside the grid");
  }
  BoxSel B{(x0 + n[0]) % n[0], (y0 + n[1]) % n[1], (z0 + n[2]) % n[2], bx, by, bz};
  double* d = nullptr;
  psm_status st = canonical(c, &d, &B);
  if (st != PSM_OK) return st;
  const size_t N = (size_t)bx * by * bz;
  cudaError_t e = cudaMemcpyAsync(f, d, sizeof(double) * Q * N, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  dfree(c, d);
  if (e != cudaSuccess) return fail(c, PSM_ERR_CUDA, cudaGetErrorString(e));
  return PSM_OK;
}

psm_status psm_get_fluid_force(psm_ctx* c, double* f, double* vfluid) {
  if (!c || !f) return PSM_ERR_ARG;
  StepConst h;
  CK(cudaMemcpyAsync(&h, c->sc, sizeof(StepConst), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int a = 0; a < 3; ++a) f[a] = h.fext[a];
  if (vfluid) *vfluid = h.vfluid;
  return PSM_OK;
}

psm_status psm_set_pdfs(psm_ctx* c, const double* f) {
  if (!c || !f) return PSM_ERR_ARG;
  const size_t N = (size_t)c->g.nx * c->g.ny * c->g.nz;
  double* d = static_cast<double*>(dalloc(c, sizeof(double) * Q * N));
  if (!d) return fail(c, PSM_ERR_OOM, "allocator returned NULL");
  cudaError_t e = cudaMemcpyAsync(d, f, sizeof(double) * Q * N, cudaMemcpyHostToDevice, c->stream);
  void* target = c->aa ? c->buf[0] : c->buf[c->cur];
  if (e == cudaSuccess) {
    launch_from_canonical(c->g, d, target, c->prec, c->aa, c->stream);
    e = cudaStreamSynchronize(c->stream);
  }
  dfree(c, d);
  if (e != cudaSuccess) return fail(c, PSM_ERR_CUDA, cudaGetErrorString(e));
  c->parity = 0;
  c->error_state = false;
  return PSM_OK;
}

psm_status psm_get_macroscopic(psm_ctx* c, double* rho, double* u) {
  if (!c || !rho || !u) return PSM_ERR_ARG;
  const size_t N = (size_t)c->g.nx * c->g.ny * c->g.nz;
  double* f = nullptr;
  psm_status st = canonical(c, &f);
  if (st != PSM_OK) return st;
  double* ru = static_cast<double*>(dalloc(c, sizeof(double) * 4 * N));
  if (!ru) {
    dfree(c, f);
    return fail(c, PSM_ERR_OOM, "allocator returned NULL");
  }
  launch_macroscopic(c->g, f, c->sc, c->bc, ru, ru + N, c->stream);
  cudaError_t e = cudaMemcpyAsync(rho, ru, sizeof(double) * N, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(u, ru + N, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  dfree(c, f);
  dfree(c, ru);
  if (e != cudaSuccess) return fail(c, PSM_ERR_CUDA, cudaGetErrorString(e));
  return PSM_OK;
}

psm_status psm_get_slot_forces(psm_ctx* c, int* pid0, int* pid1, double* F0, double* F1) {
  if (!c || !pid0 || !pid1 || !F0 || !F1) return PSM_ERR_ARG;
  const size_t N = (size_t)c->g.nx * c->g.ny * c->g.nz;
  if (c->p.n == 0) {
    for (size_t i = 0; i < N; ++i) pid0[i] = pid1[i] = -1;
    std::memset(F0, 0, sizeof(double) * 3 * N);
    std::memset(F1, 0, sizeof(double) * 3 * N);
    return PSM_OK;
  }
  psm_status st = read_status(c);
  if (st != PSM_OK) return st;
  double* d = static_cast<double*>(dalloc(c, sizeof(double) * 7 * N));
  if (!d) return fail(c, PSM_ERR_OOM, "allocator returned NULL");
  int* dp0 = reinterpret_cast<int*>(d + 6 * N);
  int* dp1 = dp0 + N;
  launch_slot_forces_to_dense(map_params(c), dp0, dp1, d, d + 3 * N, c->stream);
  cudaError_t e = cudaMemcpyAsync(F0, d, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost,
                                  c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(F1, d + 3 * N, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost,
                        c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pid0, dp0, 4 * N, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pid1, dp1, 4 * N, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  dfree(c, d);
  if (e != cudaSuccess) return fail(c, PSM_ERR_CUDA, cudaGetErrorString(e));
  return PSM_OK;
}

psm_status psm_get_slots(psm_ctx* c, int* pid0, double* B0, int* pid1, double* B1) {
  if (!c || !pid0 || !B0 || !pid1 || !B1) return PSM_ERR_ARG;
  const size_t N = (size_t)c->g.nx * c->g.ny * c->g.nz;
  if (c->p.n == 0) {
    for (size_t i = 0; i < N; ++i) {
      pid0[i] = pid1[i] = -1;
      B0[i] = B1[i] = 0.0;
    }
    return PSM_OK;
  }
  psm_status st = ensure_mapped(c);
  if (st != PSM_OK) return st;
  st = read_status(c);
  if (st != PSM_OK) return st;
  unsigned char* d = static_cast<unsigned char*>(dalloc(c, N * 24));
  if (!d) return fail(c, PSM_ERR_OOM, "allocator returned NULL");
  int* dp0 = reinterpret_cast<int*>(d);
  int* dp1 = dp0 + N;
  double* db0 = reinterpret_cast<double*>(d + 8 * N);
  double* db1 = db0 + N;
  launch_slots_to_dense(map_params(c), dp0, db0, dp1, db1, c->stream);
  cudaError_t e = cudaMemcpyAsync(pid0, dp0, 4 * N, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(pid1, dp1, 4 * N, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B0, db0, 8 * N, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(B1, db1, 8 * N, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  dfree(c, d);
  if (e != cudaSuccess) return fail(c, PSM_ERR_CUDA, cudaGetErrorString(e));
  return PSM_OK;
}

psm_status psm_check(psm_ctx* c, double* mass, double* momentum) {
  if (!c || !mass || !momentum) return PSM_ERR_ARG;
  double* f = nullptr;
  psm_status st = canonical(c, &f);
  if (st != PSM_OK) return st;
  double out[4];
  launch_sums(c->g, f, c->partials, 1024, c->partials + 4 * 1024, c->stream);
  cudaError_t e = cudaMemcpyAsync(out, c->partials + 4 * 1024, sizeof(out),
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  dfree(c, f);
  if (e != cudaSuccess) return fail(c, PSM_ERR_CUDA, cudaGetErrorString(e));
  *mass = out[0];
  for (int a = 0; a < 3; ++a) momentum[a] = out[1 + a];
  if (!std::isfinite(out[0])) return fail(c, PSM_ERR_NONFINITE, "non-finite mass");
  return PSM_OK;
}

psm_status psm_set_mlp(psm_ctx* c, const float* params) {
  if (!c || !params) return PSM_ERR_ARG;
  CK(cudaMemcpyAsync(c->mlp, params, sizeof(float) * PSM_MLP_PARAMS, cudaMemcpyHostToDevice,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->have_mlp = true;
  c->need_map = c->need_map || c->p.n > 0;
  free_graphs(c);
  return PSM_OK;
}

psm_status psm_get_mlp(psm_ctx* c, float* params) {
  if (!c || !params) return PSM_ERR_ARG;
  if (!c->have_mlp) return fail(c, PSM_ERR_STATE, "no surrogate parameters set");
  CK(cudaMemcpyAsync(params, c->mlp, sizeof(float) * PSM_MLP_PARAMS, cudaMemcpyDeviceToHost,
                     c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PSM_OK;
}

psm_status psm_mlp_samples(psm_ctx* c, unsigned long long seed, long first, long count,
                           float* X, float* eps) {
  if (!c || !X || !eps || first < 0 || count < 0) return PSM_ERR_ARG;
  if (count == 0) return PSM_OK;
  float* d = static_cast<float*>(dalloc(c, sizeof(float) * 5 * count));
  if (!d) return fail(c, PSM_ERR_OOM, "allocator returned NULL");
  launch_mlp_samples(seed, first, count, d, d + 4 * count, nullptr, c->stream);
  cudaError_t e = cudaMemcpyAsync(X, d, sizeof(float) * 4 * count, cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(eps, d + 4 * count, sizeof(float) * count, cudaMemcpyDeviceToHost,
                        c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  dfree(c, d);
  if (e != cudaSuccess) return fail(c, PSM_ERR_CUDA, cudaGetErrorString(e));
  return PSM_OK;
}

psm_status psm_mlp_loss_grad(psm_ctx* c, const float* params, long m, const float* X,
                             const float* t, float* loss, float* grad) {
  if (!c || !params || !X || !t || !loss || !grad || m <= 0) return PSM_ERR_ARG;
  const int nb = mlp_grad_blocks(m);
  const size_t floats = PSM_MLP_PARAMS * 2 + 1 + 5 * (size_t)m + (size_t)nb * (PSM_MLP_PARAMS + 1);
  float* d = static_cast<float*>(dalloc(c, sizeof(float) * floats));
  if (!d) return fail(c, PSM_ERR_OOM, "allocator returned NULL");
  float* dp = d;
  float* dg = dp + PSM_MLP_PARAMS;
  float* dl = dg + PSM_MLP_PARAMS;
  float* dX = dl + 1;
  float* dt = dX + 4 * m;
  float* part = dt + m;
  cudaError_t e = cudaMemcpyAsync(dp, params, sizeof(float) * PSM_MLP_PARAMS,
                                  cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dX, X, sizeof(float) * 4 * m, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dt, t, sizeof(float) * m, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) {
    launch_mlp_loss_grad(dp, m, dX, dt, part, nb, dg, dl, c->stream);
    e = cudaMemcpyAsync(grad, dg, sizeof(float) * PSM_MLP_PARAMS, cudaMemcpyDeviceToHost, c->stream);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(loss, dl, sizeof(float), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  dfree(c, d);
  if (e != cudaSuccess) return fail(c, PSM_ERR_CUDA, cudaGetErrorString(e));
  return PSM_OK;
}

psm_status psm_mlp_infer(psm_ctx* c, const float* params, long m, const float* X, float* eps) {
  if (!c || !params || !X || !eps || m < 0) return PSM_ERR_ARG;
  if (m == 0) return PSM_OK;
  float* d = static_cast<float*>(dalloc(c, sizeof(float) * (PSM_MLP_PARAMS + 5 * (size_t)m + 4)));
  if (!d) return fail(c, PSM_ERR_OOM, "allocator returned NULL");
  float* dp = d;
  float* dX = d + ((PSM_MLP_PARAMS + 3) / 4) * 4;  // float4-aligned
  float* de = dX + 4 * m;
  cudaError_t e = cudaMemcpyAsync(dp, params, sizeof(float) * PSM_MLP_PARAMS,
                                  cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dX, X, sizeof(float) * 4 * m, cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess) {
    InferSink out{};
    out.eps = de;
    launch_mlp_infer(dp, m, nullptr, m, dX, out, c->status, c->stream);
    e = cudaMemcpyAsync(eps, de, sizeof(float) * m, cudaMemcpyDeviceToHost, c->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  dfree(c, d);
  if (e != cudaSuccess) return fail(c, PSM_ERR_CUDA, cudaGetErrorString(e));
  return PSM_OK;
}

psm_status psm_train_surrogate(psm_ctx* c, long nsamples, unsigned long long seed, int epochs,
                               int batch, float lr, float* loss_out) {
  if (!c || nsamples <= 0 || epochs < 1 || batch < 1 || !(lr > 0)) return PSM_ERR_ARG;
  if (!c->have_mlp) return fail(c, PSM_ERR_STATE, "set initial surrogate parameters first");
  const int nb = mlp_grad_blocks(batch);
  const size_t floats = 6 * (size_t)nsamples + 3 * PSM_MLP_PARAMS + 1 +
                        (size_t)nb * (PSM_MLP_PARAMS + 1);
  float* d = static_cast<float*>(dalloc(c, sizeof(float) * floats));
  if (!d) return fail(c, PSM_ERR_OOM, "allocator returned NULL");
  float* X = d;
  float* T = X + 4 * nsamples;   // residual targets: label - eps_lin
  float* L = T + nsamples;       // labels (unused by the optimiser)
  float* g = L + nsamples;
  float* ms = g + PSM_MLP_PARAMS;
  float* vs = ms + PSM_MLP_PARAMS;
  float* dl = vs + PSM_MLP_PARAMS;
  float* part = dl + 1;
  cudaStream_t s = c->stream;
  launch_mlp_samples(seed, 0, nsamples, X, L, T, s);
  cudaMemsetAsync(ms, 0, sizeof(float) * 2 * PSM_MLP_PARAMS, s);
  int step = 0;
  double last = 0.0;
  const long per_epoch = (nsamples + batch - 1) / batch;
  const double total = (double)per_epoch * epochs;
  for (int ep = 0; ep < epochs; ++ep) {
    for (long b0 = 0; b0 < nsamples; b0 += batch) {
      const long mb = nsamples - b0 < batch ? nsamples - b0 : batch;
      launch_mlp_loss_grad(c->mlp, mb, X + 4 * b0, T + b0, part, mlp_grad_blocks(mb), g, dl, s);
      // learning rate decays exponentially to 3% of lr over the run
      const float lr_t = (float)(lr * std::pow(0.03, (double)step / total));
      launch_adam(c->mlp, g, ms, vs, ++step, lr_t, s);
    }
  }
  // loss of the final parameters over the whole sample set, in minibatches
  double acc = 0.0;
  for (long b0 = 0; b0 < nsamples; b0 += batch) {
    const long mb = nsamples - b0 < batch ? nsamples - b0 : batch;
    launch_mlp_loss_grad(c->mlp, mb, X + 4 * b0, T + b0, part, mlp_grad_blocks(mb), g, dl, s);
    float hl = 0;
    cudaMemcpyAsync(&hl, dl, sizeof(float), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) break;
    acc += (double)hl * mb;
  }
  last = acc / nsamples;
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  dfree(c, d);
  if (e != cudaSuccess) return fail(c, PSM_ERR_CUDA, cudaGetErrorString(e));
  if (loss_out) *loss_out = (float)last;
  c->need_map = c->need_map || c->p.n > 0;
  free_graphs(c);
  return PSM_OK;
}

psm_status psm_set_timing(psm_ctx* c, int enable) {
  if (!c) return PSM_ERR_ARG;
  if (enable && c->tev.empty()) {
    c->tev.resize(5 * psm_ctx::kTimedRing);
    for (auto& e : c->tev) CK(cudaEventCreate(&e));
  }
  CK(flush_timing(c));
  c->timing = enable != 0;
  for (int i = 0; i < 5; ++i) c->t_ms[i] = 0;
  return PSM_OK;
}

psm_status psm_get_timings(psm_ctx* c, double* out5) {
  if (!c || !out5) return PSM_ERR_ARG;
  CK(flush_timing(c));
  for (int i = 0; i < 5; ++i) out5[i] = c->t_ms[i];
  return PSM_OK;
}

psm_status psm_update_particles(psm_ctx* c, const double* x, const double* u, const double* om) {
  if (!c) return PSM_ERR_ARG;
  const int n = c->p.n;
  if (n == 0) return PSM_OK;
  if (!x || !u || !om) return fail(c, PSM_ERR_ARG, "NULL particle array");
  const size_t b3 = sizeof(double) * 3 * n;
  CK(cudaMemcpyAsync(c->p.x, x, b3, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->p.u, u, b3, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->p.om, om, b3, cudaMemcpyHostToDevice, c->stream));
  launch_wrap_particles(c->g, c->p, c->stream);
  CK(cudaMemsetAsync(c->dem_bar + 2, 0, sizeof(unsigned), c->stream));  // new DEM lists
  CK(cudaGetLastError());
  c->need_map = true;
  return PSM_OK;
}


// checkpoint of the stepper state (layout above)
psm_status psm_save(psm_ctx* c, const char* path) {
  if (!c || !path) return PSM_ERR_ARG;
  NvtxRange range("psm_save");
  CK(cudaStreamSynchronize(c->stream));
  const int n = c->p.n;
  CkptHeader h{};
  std::memcpy(h.magic, kCkptMagic, 8);
  const long long v[CK_FIELDS] = {c->g.nx, c->g.ny, c->g.nz, c->g.wall[0], c->g.wall[1],
                                  z_code(c->g), c->prec, c->aa, c->relax,
                                  c->aa ? c->parity : 0, n, c->have_mlp ? 1 : 0,
                                  c->opt.dem ? 1 : 0};
  std::memcpy(h.v, v, sizeof(v));
  h.tau = c->tau;
  h.omega_m = c->omega_m;
  for (int a = 0; a < 3; ++a) h.G[a] = c->G[a];
  const size_t esz = c->prec == PREC_FP32 ? 4 : 8;
  const size_t pdf_bytes = esz * Q * (size_t)c->g.ncell;
  std::vector<unsigned char> host(pdf_bytes);
  const void* field = c->aa ? c->buf[0] : c->buf[c->cur];
  CK(cudaMemcpy(host.data(), field, pdf_bytes, cudaMemcpyDeviceToHost));
  FILE* f = std::fopen(path, "wb");
  if (!f) return fail(c, PSM_ERR_ARG, std::string("cannot open for writing: ") + path);
  bool ok = write_all(f, &h, sizeof(h)) && write_all(f, host.data(), pdf_bytes);
  for (const CkptArray& a : ckpt_arrays(c)) {
    if (!ok || n == 0) break;
    const size_t bytes = a.per * a.esz * (size_t)n;
    std::vector<unsigned char> buf(bytes);
    if (cudaMemcpy(buf.data(), a.dev, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
      std::fclose(f);
      return fail(c, PSM_ERR_CUDA, "reading the particle state");
    }
    ok = write_all(f, buf.data(), bytes);
  }
  if (ok && c->have_mlp) {
    std::vector<float> prm(PSM_MLP_PARAMS);
    if (cudaMemcpy(prm.data(), c->mlp, sizeof(float) * PSM_MLP_PARAMS,
                   cudaMemcpyDeviceToHost) != cudaSuccess) {
      std::fclose(f);
      return fail(c, PSM_ERR_CUDA, "reading the surrogate parameters");
    }
    ok = write_all(f, prm.data(), sizeof(float) * PSM_MLP_PARAMS);
  }
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return fail(c, PSM_ERR_ARG, std::string("short write: ") + path);
  return PSM_OK;
}

psm_status psm_load(psm_ctx* c, const char* path) {
  if (!c || !path) return PSM_ERR_ARG;
  NvtxRange range("psm_load");
  FILE* f = std::fopen(path, "rb");
  if (!f) return fail(c, PSM_ERR_ARG, std::string("cannot open: ") + path);
  auto bad = [&](const std::string& msg) {
    std::fclose(f);
    return fail(c, PSM_ERR_ARG, msg);
  };
  CkptHeader h{};
  if (!read_all(f, &h, sizeof(h)) || std::memcmp(h.magic, kCkptMagic, 8) != 0)
    return bad("not a checkpoint of this engine");
  const long long want[CK_N] = {c->g.nx, c->g.ny, c->g.nz, c->g.wall[0], c->g.wall[1],
                                z_code(c->g), c->prec, c->aa, c->relax};
  for (int i = 0; i < CK_PARITY; ++i)
    if (h.v[i] != want[i]) return bad("checkpoint of another grid, storage form or relaxation");
  if (h.tau != c->tau || h.omega_m != c->omega_m || (h.v[CK_DEM] != 0) != (c->opt.dem != 0))
    return bad("checkpoint of another tau, magic parameter or DEM setting");
  const long long n = h.v[CK_N];
  if (n < 0 || n > (1LL << 30)) return bad("bad particle count");
  const size_t esz = c->prec == PREC_FP32 ? 4 : 8;
  const size_t pdf_bytes = esz * Q * (size_t)c->g.ncell;
  std::vector<unsigned char> field(pdf_bytes);
  if (!read_all(f, field.data(), pdf_bytes)) return bad("truncated checkpoint (PDFs)");
  // particle arrays in file order
  std::vector<double> x(3 * n), u(3 * n), om(3 * n), r(n), m(n), I(n), vol(n), fr(n);
  std::vector<unsigned char> fixed(n);
  std::vector<double> Fh(3 * n), Th(3 * n), Fold(3 * n), Told(3 * n);
  std::vector<int> hc(n), hj(n * kDemListCap);
  std::vector<double> hd(n * kDemListCap * 3);
  void* hosts[] = {x.data(),  u.data(),    om.data(),   r.data(),    m.data(),  I.data(),
                   vol.data(), fr.data(),  fixed.data(), Fh.data(),  Th.data(), Fold.data(),
                   Told.data(), hc.data(), hj.data(),   hd.data()};
  const size_t per[] = {3, 3, 3, 1, 1, 1, 1, 1, 1, 3, 3, 3, 3, 1, kDemListCap, 3 * kDemListCap};
  const size_t es[] = {8, 8, 8, 8, 8, 8, 8, 8, 1, 8, 8, 8, 8, 4, 4, 8};
  constexpr int kArrays = 16;
  for (int i = 0; i < kArrays && n > 0; ++i)
    if (!read_all(f, hosts[i], per[i] * es[i] * (size_t)n))
      return bad("truncated checkpoint (particles)");
  std::vector<float> prm;
  if (h.v[CK_MLP]) {
    prm.resize(PSM_MLP_PARAMS);
    if (!read_all(f, prm.data(), sizeof(float) * PSM_MLP_PARAMS))
      return bad("truncated checkpoint (surrogate)");
  }
  std::fclose(f);
  // particles through the regular path (buffers, lists, bins), then their
  // saved derived values and force history over the recomputed ones
  std::vector<double> dens(n);
  for (long long i = 0; i < n; ++i) dens[i] = m[i] / vol[i];
  psm_status st = psm_set_particles(c, (int)n, x.data(), r.data(), u.data(), om.data(),
                                    dens.data(), fixed.data());
  if (st != PSM_OK) return st;
  const std::vector<CkptArray> arrs = ckpt_arrays(c);
  // m, I, vol, fr, fixed, Fh, Th, Fold, Told, contact history
  for (int i = 4; i < kArrays && n > 0; ++i)
    CK(cudaMemcpyAsync(arrs[i].dev, hosts[i], per[i] * es[i] * (size_t)n,
                       cudaMemcpyHostToDevice, c->stream));
  for (int a = 0; a < 3; ++a) c->G[a] = h.G[a];
  if (!prm.empty()) {
    st = psm_set_mlp(c, prm.data());
    if (st != PSM_OK) return st;
  }
  c->cur = 0;
  c->parity = c->aa ? (int)h.v[CK_PARITY] : 0;
  CK(cudaMemcpyAsync(c->buf[0], field.data(), pdf_bytes, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->need_map = true;
  c->error_state = false;
  return PSM_OK;
}

psm_status psm_selftest_waits(psm_ctx* c, long long limit_ns) {
  if (!c || limit_ns < 0 || limit_ns > 1000000000LL) return PSM_ERR_ARG;
  const unsigned long long ns = (unsigned long long)limit_ns;
  CK(cudaStreamSynchronize(c->stream));
  unsigned st = 0;
  const int which[3] = {0, 1, 2};
  for (int w : which) {
    CK(cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream));
    if (w == 0) launch_wait_selftest_lbm(c->status, ns, c->stream);
    else if (w == 1) launch_wait_selftest_mlp(c->status, ns, c->stream);
    else launch_wait_selftest_dem(c->dem_bar, c->status, ns, c->stream);
    CK(cudaGetLastError());
    unsigned one = 0;
    CK(cudaMemcpyAsync(&one, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (!(one & ST_TIMEOUT)) {
      CK(cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream));
      CK(cudaStreamSynchronize(c->stream));
      return fail(c, PSM_ERR_STATE, "a bounded wait did not give up");
    }
    st |= one;
  }
  // the status word keeps ST_TIMEOUT: the next call reports PSM_ERR_TIMEOUT
  CK(cudaMemsetAsync(c->dem_bar, 0, 4 * sizeof(unsigned), c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return PSM_OK;
}

psm_status psm_get_particle_count(const psm_ctx* c, int* n) {
  if (!c || !n) return PSM_ERR_ARG;
  *n = c->p.n;
  return PSM_OK;
}

long psm_last_launch_count(const psm_ctx* c) { return c ? c->launches : 0; }

const char* psm_last_error(const psm_ctx* c) {
  if (!c) return "null context";
  return c->err.c_str();
}

void psm_destroy(psm_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  free_graphs(c);
  free_particles(c);
  for (void* q : c->allocs) dfree(c, q);
  c->allocs.clear();
  for (auto& e : c->tev)
    if (e) cudaEventDestroy(e);
  if (c->capture) cudaStreamDestroy(c->capture);
  delete c;
}

}  // extern "C"
