// dem_kernels.cu -- particle dynamics on the device (paper Sec. 2.2, Sec. 3.2):
// velocity Verlet (Eqs. 15-16) with sub-cycling, linear spring-dashpot normal
// contacts between spheres and with wall faces (Eq. 12), tangential
// spring-dashpot contacts with history between spheres (Eqs. 13-14), and
// positions, velocities and angular velocities double-buffered over the
// sub-steps; buoyancy-corrected
// gravity and the hydrodynamic force/torque of the last LBM step held fixed
// over the sub-steps.
//
// The particles are binned (bin edge >= largest diameter + skin) and each
// particle gets the list of partners within contact distance plus the skin,
// in ascending index order.  The lists are rebuilt at the start of a step
// once a particle has moved more than a quarter of the skin since they were
// built (or the host changed the particles); a particle that moves more than
// half the skin could miss a contact: the sub-steps check the displacement
// and set ST_DEM_SKIN.  A list longer than its capacity sets
// ST_CONTACT_OVERFLOW.  When every list is empty no contact can occur within
// the step and each particle runs its sub-steps alone.
//
// Per sub-step one launch, one thread per particle: positions of the current
// sub-step are read, contacts are summed over the list in ascending j (FP32
// prefilter -- float positions differ from FP64 by far less than the 1e-2
// margin -- then the exact FP64 contact), then the walls -x,+x,-y,+y,-z,+z,
// with plain IEEE FP64 operations (this file is compiled with -fmad=false),
// so the sums are bitwise reproducible; then the velocity update and the next
// sub-step's positions (Eqs. 15-16 with dt/(2m), dt/(2I) formed once per
// sub-step: equal to the quotients up to rounding).  FP64 runs at 1/64 of the FP32 rate here, so each
// FP64 instruction works on 32 particles and the blocks (32 threads) spread
// over many SMs.
#include "psm_internal.cuh"

namespace psm {
namespace {

constexpr double PI = 3.14159265358979323846;

__device__ __forceinline__ double damping(double meff, double kn, double le) {
  return -2.0 * le * sqrt(meff * kn) / sqrt(PI * PI + le * le);
}

__device__ void dem_position(const DemParams& P, int i) {
  const double dims[3] = {(double)P.g.nx, (double)P.g.ny, (double)P.g.nz};
  if (!P.p.fixed[i]) {
    const double dt = P.dt;
    const double h2m = dt * dt / (2.0 * P.p.m[i]);
    for (int a = 0; a < 3; ++a) {
      double xn = P.p.x[3 * i + a] + dt * P.p.u[3 * i + a] + h2m * P.p.Fold[3 * i + a];
      if (!P.g.wall[a]) {
        if (xn >= dims[a]) xn -= dims[a];
        else if (xn < 0.0) xn += dims[a];
      }
      P.p.x[3 * i + a] = xn;
    }
  }
  for (int a = 0; a < 3; ++a) P.p.xf[4 * i + a] = (float)P.p.x[3 * i + a];
  P.p.xf[4 * i + 3] = (float)P.p.r[i];
}

// Tangential history of particle i: its entries in buffer b (partners in
// ascending order), read by a moving cursor while the new entries of the
// sub-step are written to buffer 1 - b.
struct HistCursor {
  const int* oj;
  const double* od;
  int nold, po;
  int* nj;
  double* nd;
  int nnew;
};

// exact FP64 contact of i with j (j != i); adds to F (and, with the
// tangential model, the tangential force to F and its torque to T) when in
// contact.  X, U, W are the positions, velocities and angular velocities of
// the current sub-step.  Eqs. 12-14 with the readings of the oracle: contact
// point x_i - (r_i - delta/2) n, history projected onto the current tangent
// plane and advanced by dt U_t, F_t = -k_t delta_t - d_t U_t.
__device__ __noinline__ void pair_contact(const DemParams& P, const double* X,
                                             const double* U, const double* W, int i, int j,
                                             double* F, double* T, HistCursor& H) {
  const double dims[3] = {(double)P.g.nx, (double)P.g.ny, (double)P.g.nz};
  double d[3];
  for (int a = 0; a < 3; ++a) {
    double v = X[3 * i + a] - X[3 * j + a];
    if (!P.g.wall[a]) {
      if (v > 0.5 * dims[a]) v -= dims[a];
      else if (v < -0.5 * dims[a]) v += dims[a];
    }
    d[a] = v;
  }
  const double dist2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
  const double rs = P.p.r[i] + P.p.r[j];
  if (!(dist2 < rs * rs)) return;
  const double dist = sqrt(dist2);
  const double delta = rs - dist;
  const double n[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
  const double vrel[3] = {U[3 * i] - U[3 * j], U[3 * i + 1] - U[3 * j + 1],
                          U[3 * i + 2] - U[3 * j + 2]};
  const double vn = vrel[0] * n[0] + vrel[1] * n[1] + vrel[2] * n[2];
  const double meff = P.p.m[i] * P.p.m[j] / (P.p.m[i] + P.p.m[j]);
  const double dn = damping(meff, P.kn, P.log_e);
  for (int a = 0; a < 3; ++a) F[a] += P.kn * delta * n[a] - dn * vn * n[a];
  if (!(P.kt_ratio > 0.0)) return;
  const double ai = -(P.p.r[i] - 0.5 * delta), aj = P.p.r[j] - 0.5 * delta;
  const double Ai[3] = {ai * n[0], ai * n[1], ai * n[2]};
  const double Aj[3] = {aj * n[0], aj * n[1], aj * n[2]};
  const double* wi = W + 3 * i;
  const double* wj = W + 3 * j;
  const double Ucp[3] = {
      (U[3 * i + 0] + (wi[1] * Ai[2] - wi[2] * Ai[1])) -
          (U[3 * j + 0] + (wj[1] * Aj[2] - wj[2] * Aj[1])),
      (U[3 * i + 1] + (wi[2] * Ai[0] - wi[0] * Ai[2])) -
          (U[3 * j + 1] + (wj[2] * Aj[0] - wj[0] * Aj[2])),
      (U[3 * i + 2] + (wi[0] * Ai[1] - wi[1] * Ai[0])) -
          (U[3 * j + 2] + (wj[0] * Aj[1] - wj[1] * Aj[0]))};
  const double un = Ucp[0] * n[0] + Ucp[1] * n[1] + Ucp[2] * n[2];
  const double Ut[3] = {Ucp[0] - un * n[0], Ucp[1] - un * n[1], Ucp[2] - un * n[2]};
  double h[3] = {0.0, 0.0, 0.0};
  while (H.po < H.nold && H.oj[H.po] < j) ++H.po;
  if (H.po < H.nold && H.oj[H.po] == j)
    for (int a = 0; a < 3; ++a) h[a] = H.od[3 * H.po + a];
  const double hn = h[0] * n[0] + h[1] * n[1] + h[2] * n[2];
  for (int a = 0; a < 3; ++a) h[a] = (h[a] - hn * n[a]) + P.dt * Ut[a];
  const double kt = P.kt_ratio * P.kn, dtg = P.kt_ratio * dn;
  const double Ft[3] = {-kt * h[0] - dtg * Ut[0], -kt * h[1] - dtg * Ut[1],
                        -kt * h[2] - dtg * Ut[2]};
  for (int a = 0; a < 3; ++a) F[a] += Ft[a];
  T[0] += Ai[1] * Ft[2] - Ai[2] * Ft[1];
  T[1] += Ai[2] * Ft[0] - Ai[0] * Ft[2];
  T[2] += Ai[0] * Ft[1] - Ai[1] * Ft[0];
  // the list of partners holds every particle in contact: at most K entries
  H.nj[H.nnew] = j;
  for (int a = 0; a < 3; ++a) H.nd[3 * H.nnew + a] = h[a];
  ++H.nnew;
}

__device__ __forceinline__ void wall_contacts(const DemParams& P, const double* X,
                                              const double* U, int i, double* F) {
  const double dims[3] = {(double)P.g.nx, (double)P.g.ny, (double)P.g.nz};
  for (int a = 0; a < 3; ++a) {
    if (!P.g.wall[a]) continue;
    for (int side = 0; side < 2; ++side) {
      const double delta = side == 0 ? P.p.r[i] - X[3 * i + a]
                                     : X[3 * i + a] + P.p.r[i] - dims[a];
      if (!(delta > 0.0)) continue;
      const double nn = side == 0 ? 1.0 : -1.0;
      const double vn = U[3 * i + a] * nn;
      const double dn = damping(P.p.m[i], P.kn, P.log_e);
      F[a] += P.kn * delta * nn - dn * vn * nn;
    }
  }
}

// ---- neighbour lists, once per LBM step
__device__ __forceinline__ int bin_of(const DemParams& P, float x, int a) {
  int b = (int)(x / P.h[a]);
  return b < 0 ? 0 : (b >= P.nc[a] ? P.nc[a] - 1 : b);
}

__device__ void dem_bin(const DemParams& P, int i) {
  const float x = (float)P.p.x[3 * i], y = (float)P.p.x[3 * i + 1], z = (float)P.p.x[3 * i + 2];
  P.xbuild[i] = make_float4(x, y, z, (float)P.p.r[i]);
  const int b = bin_of(P, x, 0) + P.nc[0] * (bin_of(P, y, 1) + P.nc[1] * bin_of(P, z, 2));
  P.pbin[i] = b;
  atomicAdd(&P.bin_count[b], 1);
}

// exclusive scan of the bin counts by one block (part: blockDim ints of
// shared memory)
__device__ void dem_scan(const DemParams& P, int* part) {
  const int n = P.nbins, t = threadIdx.x, nt = blockDim.x;
  const int chunk = (n + nt - 1) / nt;
  const int lo = t * chunk, hi = min(n, lo + chunk);
  int s = 0;
  for (int b = lo; b < hi; ++b) s += P.bin_count[b];
  part[t] = s;
  __syncthreads();
  for (int off = 1; off < nt; off <<= 1) {
    const int v = t >= off ? part[t - off] : 0;
    __syncthreads();
    part[t] += v;
    __syncthreads();
  }
  int run = part[t] - s;
  for (int b = lo; b < hi; ++b) {
    P.bin_start[b] = run;
    P.bin_cursor[b] = run;
    run += P.bin_count[b];
  }
}

__device__ void dem_fill(const DemParams& P, int i) {
  P.bin_items[atomicAdd(&P.bin_cursor[P.pbin[i]], 1)] = i;
}

// the bins next to bin b along one axis (periodic wrap or none at walls)
__device__ __forceinline__ int axis_bins(const DemParams& P, int a, int b, int* out) {
  const int nc = P.nc[a];
  if (nc < 3) {
    for (int k = 0; k < nc; ++k) out[k] = k;
    return nc;
  }
  int m = 0;
  for (int o = -1; o <= 1; ++o) {
    int v = b + o;
    if (v < 0 || v >= nc) {
      if (P.g.wall[a]) continue;
      v = v < 0 ? v + nc : v - nc;
    }
    out[m++] = v;
  }
  return m;
}

__device__ __forceinline__ float min_image(float d, float dim, int periodic) {
  if (periodic) {
    if (d > 0.5f * dim) d -= dim;
    else if (d < -0.5f * dim) d += dim;
  }
  return d;
}

__device__ void dem_nbr(const DemParams& P, int i) {
  const float dims[3] = {(float)P.g.nx, (float)P.g.ny, (float)P.g.nz};
  const float4 xi = P.xbuild[i];
  const float xa[3] = {xi.x, xi.y, xi.z};
  int bx[3], by[3], bz[3];
  const int nbx = axis_bins(P, 0, bin_of(P, xi.x, 0), bx);
  const int nby = axis_bins(P, 1, bin_of(P, xi.y, 1), by);
  const int nbz = axis_bins(P, 2, bin_of(P, xi.z, 2), bz);
  int* L = P.nbr + (size_t)i * P.K;
  int cnt = 0;
  bool over = false;
  for (int c = 0; c < nbz; ++c)
    for (int bb = 0; bb < nby; ++bb)
      for (int aa = 0; aa < nbx; ++aa) {
        const int b = bx[aa] + P.nc[0] * (by[bb] + P.nc[1] * bz[c]);
        const int e = P.bin_start[b] + P.bin_count[b];
        for (int k = P.bin_start[b]; k < e; ++k) {
          const int j = P.bin_items[k];
          if (j == i) continue;
          const float4 xj = P.xbuild[j];
          const float xb[3] = {xj.x, xj.y, xj.z};
          float d2 = 0.0f;
          for (int a = 0; a < 3; ++a) {
            const float d = min_image(xa[a] - xb[a], dims[a], !P.g.wall[a]);
            d2 += d * d;
          }
          const float reach = xi.w + xj.w + P.skin;
          if (!(d2 < reach * reach)) continue;
          if (cnt == P.K) {
            over = true;
            continue;
          }
          // insertion keeps the list in ascending index order
          int pos = cnt++;
          while (pos > 0 && L[pos - 1] > j) {
            L[pos] = L[pos - 1];
            --pos;
          }
          L[pos] = j;
        }
      }
  P.nbr_cnt[i] = cnt;
  if (cnt > 0) atomicAdd(&P.bar[3], 1u);
  if (over) atomicOr(P.status, ST_CONTACT_OVERFLOW);
}

// One sub-step in one launch, one thread per particle: contacts over the
// neighbour list in ascending j (Eq. 12), velocity update (Eq. 16) and the
// positions of the next sub-step (Eq. 15).  Positions and velocities are
// double-buffered: every contact reads the current sub-step's state (Xc, Uc,
// XFc) while the new state goes to (Xn, Un, XFn).  On the last sub-step the
// positions are carried over.
constexpr int DEM_BATCH = 8;
__device__ void dem_substep(const DemParams& P, int i, const double* __restrict__ Xc,
                            const double* __restrict__ Uc, const double* __restrict__ Wc,
                            const float4* __restrict__ XFc, double* __restrict__ Xn,
                            double* __restrict__ Un, double* __restrict__ Wn,
                            float4* __restrict__ XFn, int hb, int last) {
  const float dims[3] = {(float)P.g.nx, (float)P.g.ny, (float)P.g.nz};
  const float4 xi = XFc[i];
  double F[3] = {0.0, 0.0, 0.0}, T[3] = {0.0, 0.0, 0.0};
  const int cnt = P.nbr_cnt[i];
  const int* L = P.nbr + (size_t)i * P.K;
  HistCursor H;
  H.oj = P.p.hj[hb] + (size_t)i * P.K;
  H.od = P.p.hd[hb] + (size_t)i * P.K * 3;
  H.nold = P.kt_ratio > 0.0 ? P.p.hcnt[hb][i] : 0;
  H.po = 0;
  H.nj = P.p.hj[1 - hb] + (size_t)i * P.K;
  H.nd = P.p.hd[1 - hb] + (size_t)i * P.K * 3;
  H.nnew = 0;
  for (int k0 = 0; k0 < cnt; k0 += DEM_BATCH) {
    // the batch's partners and positions are loaded before any is used
    int jj[DEM_BATCH];
    float4 xj[DEM_BATCH];
#pragma unroll
    for (int u = 0; u < DEM_BATCH; ++u) jj[u] = k0 + u < cnt ? L[k0 + u] : -1;
#pragma unroll
    for (int u = 0; u < DEM_BATCH; ++u) xj[u] = jj[u] >= 0 ? XFc[jj[u]] : xi;
#pragma unroll
    for (int u = 0; u < DEM_BATCH; ++u) {
      if (jj[u] < 0) continue;
      const float dx = min_image(xi.x - xj[u].x, dims[0], !P.g.wall[0]);
      const float dy = min_image(xi.y - xj[u].y, dims[1], !P.g.wall[1]);
      const float dz = min_image(xi.z - xj[u].z, dims[2], !P.g.wall[2]);
      const float rs = xi.w + xj[u].w + 1e-2f;
      if (dx * dx + dy * dy + dz * dz < rs * rs) pair_contact(P, Xc, Uc, Wc, i, jj[u], F, T, H);
    }
  }
  P.p.hcnt[1 - hb][i] = H.nnew;
  wall_contacts(P, Xc, Uc, i, F);
  const double dt = P.dt;
  const double ddims[3] = {(double)P.g.nx, (double)P.g.ny, (double)P.g.nz};
  double u[3], x[3], w[3];
  for (int a = 0; a < 3; ++a) {
    u[a] = Uc[3 * i + a];
    x[a] = Xc[3 * i + a];
    w[a] = Wc[3 * i + a];
  }
  if (!P.p.fixed[i]) {
    // FP64 division is a long instruction sequence here: the three
    // reciprocal factors once per sub-step
    const double hm = dt / (2.0 * P.p.m[i]), hI = dt / (2.0 * P.p.I[i]), h2m = dt * hm;
    for (int a = 0; a < 3; ++a) {
      const double Fn = P.p.Fh[3 * i + a] + F[a] + (P.p.m[i] - P.p.vol[i]) * P.gravity[a];
      const double Tn = P.p.Th[3 * i + a] + T[a];
      u[a] += hm * (P.p.Fold[3 * i + a] + Fn);
      w[a] += hI * (P.p.Told[3 * i + a] + Tn);
      P.p.Fold[3 * i + a] = Fn;
      P.p.Told[3 * i + a] = Tn;
    }
    if (!last) {
      for (int a = 0; a < 3; ++a) {
        double xn = x[a] + dt * u[a] + h2m * P.p.Fold[3 * i + a];
        if (!P.g.wall[a]) {
          if (xn >= ddims[a]) xn -= ddims[a];
          else if (xn < 0.0) xn += ddims[a];
        }
        x[a] = xn;
      }
    }
    // the lists stay valid while every particle moves less than skin / 2
    const float4 xb = P.xbuild[i];
    const float ex = min_image((float)x[0] - xb.x, dims[0], !P.g.wall[0]);
    const float ey = min_image((float)x[1] - xb.y, dims[1], !P.g.wall[1]);
    const float ez = min_image((float)x[2] - xb.z, dims[2], !P.g.wall[2]);
    const float e2 = ex * ex + ey * ey + ez * ez;
    if (e2 > 0.25f * P.skin * P.skin) atomicOr(P.status, ST_DEM_SKIN);
    if (last && e2 > 0.0625f * P.skin * P.skin) P.bar[2] = 0u;  // rebuild next step
  }
  for (int a = 0; a < 3; ++a) {
    Un[3 * i + a] = u[a];
    Xn[3 * i + a] = x[a];
    Wn[3 * i + a] = w[a];
  }
  XFn[i] = make_float4((float)x[0], (float)x[1], (float)x[2], xi.w);
}

// after an odd number of sub-steps the state is in the second buffers: back
// to the first ones (history included)
__device__ void dem_copy_back(const DemParams& P, int i, const double* __restrict__ X,
                              const double* __restrict__ U, const double* __restrict__ W,
                              const float4* __restrict__ XF) {
  for (int a = 0; a < 3; ++a) {
    P.p.x[3 * i + a] = X[3 * i + a];
    P.p.u[3 * i + a] = U[3 * i + a];
    P.p.om[3 * i + a] = W[3 * i + a];
  }
  reinterpret_cast<float4*>(P.p.xf)[i] = XF[i];
  const int c = P.p.hcnt[1][i];
  P.p.hcnt[0][i] = c;
  for (int k = 0; k < c; ++k) {
    P.p.hj[0][(size_t)i * P.K + k] = P.p.hj[1][(size_t)i * P.K + k];
    for (int a = 0; a < 3; ++a)
      P.p.hd[0][((size_t)i * P.K + k) * 3 + a] = P.p.hd[1][((size_t)i * P.K + k) * 3 + a];
  }
}

// ---- one DEM step in one launch: the phases above separated by a grid
// barrier (all blocks resident: cooperative launch).  The barrier's wait is
// bounded (1 s); a block that gives up sets ST_TIMEOUT and leaves.
constexpr int DEM_THREADS = 32;
constexpr unsigned long long kBarrierLimitNs = 1000000000ull;

__device__ __forceinline__ unsigned long long dem_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// sense by generation: the last block to arrive resets the count and bumps
// the generation the others wait on
__device__ bool grid_barrier(const DemParams& P, unsigned& gen,
                             unsigned long long limit_ns = kBarrierLimitNs) {
  __syncthreads();
  int ok = 1;
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(&P.bar[0], 1u) == gridDim.x - 1) {
      atomicExch(&P.bar[0], 0u);
      __threadfence();
      atomicAdd(&P.bar[1], 1u);
    } else {
      volatile unsigned* g = &P.bar[1];
      const unsigned long long t0 = dem_ns();
      while (*g == gen) {
        if (dem_ns() - t0 > limit_ns) {
          ok = 0;
          atomicOr(P.status, ST_TIMEOUT);
          break;
        }
      }
    }
    __threadfence();
  }
  ++gen;
  return __syncthreads_and(ok) != 0;
}

__global__ void __launch_bounds__(DEM_THREADS) dem_step_kernel(DemParams P, int subcycles) {
  __shared__ int part[DEM_THREADS];
  unsigned gen = *(volatile unsigned*)&P.bar[1];
  // lists are rebuilt when a particle has moved more than a quarter of the
  // skin since they were built, or the host changed the particles
  const bool rebuild = *(volatile unsigned*)&P.bar[2] == 0u;
  const int n = P.p.n;
  const int stride = gridDim.x * blockDim.x;
  const int i0 = blockIdx.x * blockDim.x + threadIdx.x;
  if (rebuild) {
    for (int b = i0; b < P.nbins; b += stride) P.bin_count[b] = 0;
    if (i0 == 0) P.bar[3] = 0u;
    if (!grid_barrier(P, gen)) return;
    for (int i = i0; i < n; i += stride) dem_bin(P, i);
    if (!grid_barrier(P, gen)) return;
    if (blockIdx.x == 0) dem_scan(P, part);
    if (!grid_barrier(P, gen)) return;
    for (int i = i0; i < n; i += stride) dem_fill(P, i);
    if (!grid_barrier(P, gen)) return;
    for (int i = i0; i < n; i += stride) dem_nbr(P, i);
    if (i0 == 0) P.bar[2] = 1u;  // every block read the flag before its first barrier
  }
  for (int i = i0; i < n; i += stride) dem_position(P, i);
  if (!grid_barrier(P, gen)) return;
  const double* X0 = P.p.x;
  const double* U0 = P.p.u;
  const double* W0 = P.p.om;
  const float4* XF0 = reinterpret_cast<const float4*>(P.p.xf);
  if (*(volatile unsigned*)&P.bar[3] == 0u) {
    // no particle has a partner within contact distance plus the skin: no
    // contact can occur this step, each particle's sub-steps need only its
    // own state (same arithmetic, no barriers)
    for (int i = i0; i < n; i += stride) {
      const double* Xc = X0;
      const double* Uc = U0;
      const double* Wc = W0;
      const float4* XFc = XF0;
      for (int sc = 0; sc < subcycles; ++sc) {
        const bool to2 = (sc % 2) == 0;
        double* Xn = to2 ? P.p.x2 : P.p.x;
        double* Un = to2 ? P.p.u2 : P.p.u;
        double* Wn = to2 ? P.p.om2 : P.p.om;
        float4* XFn = reinterpret_cast<float4*>(to2 ? P.p.xf2 : P.p.xf);
        dem_substep(P, i, Xc, Uc, Wc, XFc, Xn, Un, Wn, XFn, sc & 1, sc + 1 == subcycles);
        Xc = Xn;
        Uc = Un;
        Wc = Wn;
        XFc = XFn;
      }
      if (subcycles % 2 == 1) dem_copy_back(P, i, Xc, Uc, Wc, XFc);
    }
    return;
  }
  const double* Xc = X0;
  const double* Uc = U0;
  const double* Wc = W0;
  const float4* XFc = XF0;
  for (int sc = 0; sc < subcycles; ++sc) {
    const bool to2 = (sc % 2) == 0;
    double* Xn = to2 ? P.p.x2 : P.p.x;
    double* Un = to2 ? P.p.u2 : P.p.u;
    double* Wn = to2 ? P.p.om2 : P.p.om;
    float4* XFn = reinterpret_cast<float4*>(to2 ? P.p.xf2 : P.p.xf);
    for (int i = i0; i < n; i += stride)
      dem_substep(P, i, Xc, Uc, Wc, XFc, Xn, Un, Wn, XFn, sc & 1, sc + 1 == subcycles);
    if (!grid_barrier(P, gen)) return;
    Xc = Xn;
    Uc = Un;
    Wc = Wn;
    XFc = XFn;
  }
  if (subcycles % 2 == 1)
    for (int i = i0; i < n; i += stride) dem_copy_back(P, i, Xc, Uc, Wc, XFc);
}

}  // namespace

int dem_max_blocks() {
  int per_sm = 0, dev = 0, nsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dem_step_kernel, DEM_THREADS, 0) !=
          cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 0;
  return per_sm * nsm;
}

// diagnostic: the grid barrier of the DEM step, entered by one block with
// an arrival count that never completes, gives up after limit_ns and raises
// ST_TIMEOUT (bar: 4 words of scratch, left zero)
__global__ void barrier_selftest_kernel(unsigned* bar, unsigned* status,
                                        unsigned long long limit_ns) {
  DemParams P{};
  P.bar = bar;
  P.status = status;
  if (threadIdx.x == 0) {
    bar[0] = 1u;  // one arrival that no block made: the count never completes
    bar[1] = 0u;
    __threadfence();
  }
  unsigned gen = 0;
  grid_barrier(P, gen, limit_ns);
  __syncthreads();
  if (threadIdx.x == 0) {
    bar[0] = 0u;
    bar[1] = 0u;
  }
}

int launch_wait_selftest_dem(unsigned* bar, unsigned* status, unsigned long long limit_ns,
                             cudaStream_t s) {
  barrier_selftest_kernel<<<1, DEM_THREADS, 0, s>>>(bar, status, limit_ns);
  return 1;
}

int launch_dem_step(DemParams P, int subcycles, cudaStream_t s) {
  const int n = P.p.n;
  if (n == 0) return 0;
  int blocks = (n + DEM_THREADS - 1) / DEM_THREADS;
  if (blocks > P.max_blocks) blocks = P.max_blocks;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)blocks);
  cfg.blockDim = dim3(DEM_THREADS);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, dem_step_kernel, P, subcycles);
  return 1;
}

}  // namespace psm
