// dem_kernels.cu -- particle dynamics on the device (paper Sec. 2.2, Sec. 3.2):
// velocity Verlet (Eqs. 15-16) with sub-cycling, linear spring-dashpot normal
// contacts between spheres and with wall faces (Eq. 12), buoyancy-corrected
// gravity and the hydrodynamic force/torque of the last LBM step held fixed
// over the sub-steps.
//
// Per sub-step: positions (all particles), then contact forces (every
// particle reads the new positions and the old velocities of the others),
// then velocities.  Contacts of particle i are summed in ascending j, then the
// walls -x,+x,-y,+y,-z,+z, with plain IEEE FP64 operations (this file is
// compiled with -fmad=false), so the sums are bitwise reproducible.
//
// Per sub-step two launches: contacts (one warp per particle scanning all
// others with an FP32 prefilter -- float positions differ from FP64 by far
// less than the 1e-2 margin -- and evaluating candidates in FP64, ascending
// j), then the velocity update fused with the next sub-step's positions.
// FP64 runs at 1/58 of the FP32 rate here, so the per-particle FP64 work is
// spread over many SMs rather than run in one block.
#include "psm_internal.cuh"

namespace psm {
namespace {

constexpr double PI = 3.14159265358979323846;

__device__ __forceinline__ double damping(double meff, double kn, double le) {
  return -2.0 * le * sqrt(meff * kn) / sqrt(PI * PI + le * le);
}

__global__ void dem_position_kernel(DemParams P) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.p.n) return;
  const double dims[3] = {(double)P.g.nx, (double)P.g.ny, (double)P.g.nz};
  if (!P.p.fixed[i]) {
    const double dt = P.dt;
    for (int a = 0; a < 3; ++a) {
      double xn = P.p.x[3 * i + a] + dt * P.p.u[3 * i + a] +
                  dt * dt * P.p.Fold[3 * i + a] / (2.0 * P.p.m[i]);
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

// exact FP64 contact of i with j (j != i); adds to F when in contact.
// X and U are the positions and velocities of the current sub-step.
__device__ __forceinline__ void pair_contact(const DemParams& P, const double* X,
                                             const double* U, int i, int j, double* F) {
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

// One sub-step in one launch: one warp per particle scans all others with an
// FP32 prefilter, sums its contacts in ascending j (Eq. 12), updates its
// velocity (Eq. 16) and writes the positions of the next sub-step (Eq. 15).
// Positions and velocities are double-buffered: every contact reads the
// current sub-step's state (Xc, Uc, XFc) while the new state goes to
// (Xn, Un, XFn).  On the last sub-step the positions are carried over.
__global__ void dem_substep_kernel(DemParams P, const double* __restrict__ Xc,
                                   const double* __restrict__ Uc,
                                   const float4* __restrict__ XFc, double* __restrict__ Xn,
                                   double* __restrict__ Un, float4* __restrict__ XFn,
                                   int last) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= P.p.n) return;
  const float dims[3] = {(float)P.g.nx, (float)P.g.ny, (float)P.g.nz};
  const float4 xi = XFc[i];
  double F[3] = {0.0, 0.0, 0.0};
  const int n = P.p.n;
  for (int base = 0; base < n; base += 32) {
    const int j = base + lane;
    bool cand = false;
    if (j < n && j != i) {
      const float4 xj = XFc[j];
      float d[3] = {xi.x - xj.x, xi.y - xj.y, xi.z - xj.z};
      for (int a = 0; a < 3; ++a) {
        if (!P.g.wall[a]) {
          if (d[a] > 0.5f * dims[a]) d[a] -= dims[a];
          else if (d[a] < -0.5f * dims[a]) d[a] += dims[a];
        }
      }
      const float rs = xi.w + xj.w + 1e-2f;
      cand = d[0] * d[0] + d[1] * d[1] + d[2] * d[2] < rs * rs;
    }
    unsigned bits = __ballot_sync(0xffffffffu, cand);
    while (bits) {
      const int l = __ffs(bits) - 1;
      bits &= bits - 1;
      pair_contact(P, Xc, Uc, i, base + l, F);  // same values on all lanes
    }
  }
  if (lane != 0) return;
  wall_contacts(P, Xc, Uc, i, F);
  const double dt = P.dt;
  const double ddims[3] = {(double)P.g.nx, (double)P.g.ny, (double)P.g.nz};
  double u[3], x[3];
  for (int a = 0; a < 3; ++a) {
    u[a] = Uc[3 * i + a];
    x[a] = Xc[3 * i + a];
  }
  if (!P.p.fixed[i]) {
    for (int a = 0; a < 3; ++a) {
      const double Fn = P.p.Fh[3 * i + a] + F[a] + (P.p.m[i] - P.p.vol[i]) * P.gravity[a];
      const double Tn = P.p.Th[3 * i + a];
      u[a] += dt * (P.p.Fold[3 * i + a] + Fn) / (2.0 * P.p.m[i]);
      P.p.om[3 * i + a] += dt * (P.p.Told[3 * i + a] + Tn) / (2.0 * P.p.I[i]);
      P.p.Fold[3 * i + a] = Fn;
      P.p.Told[3 * i + a] = Tn;
    }
    if (!last) {
      for (int a = 0; a < 3; ++a) {
        double xn = x[a] + dt * u[a] + dt * dt * P.p.Fold[3 * i + a] / (2.0 * P.p.m[i]);
        if (!P.g.wall[a]) {
          if (xn >= ddims[a]) xn -= ddims[a];
          else if (xn < 0.0) xn += ddims[a];
        }
        x[a] = xn;
      }
    }
  }
  for (int a = 0; a < 3; ++a) {
    Un[3 * i + a] = u[a];
    Xn[3 * i + a] = x[a];
  }
  XFn[i] = make_float4((float)x[0], (float)x[1], (float)x[2], xi.w);
}

__global__ void dem_copy_back_kernel(DemParams P, const double* __restrict__ X,
                                     const double* __restrict__ U,
                                     const float4* __restrict__ XF) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P.p.n) return;
  for (int a = 0; a < 3; ++a) {
    P.p.x[3 * i + a] = X[3 * i + a];
    P.p.u[3 * i + a] = U[3 * i + a];
  }
  reinterpret_cast<float4*>(P.p.xf)[i] = XF[i];
}

}  // namespace

int launch_dem_step(DemParams P, int subcycles, cudaStream_t s) {
  const int n = P.p.n;
  if (n == 0) return 0;
  const int tb = 128;
  const unsigned gp = (n + tb - 1) / tb;
  const unsigned gw = (unsigned)(((long long)n * 32 + tb - 1) / tb);
  int launches = 0;
  dem_position_kernel<<<gp, tb, 0, s>>>(P);
  ++launches;
  const double* Xc = P.p.x;
  const double* Uc = P.p.u;
  const float4* XFc = reinterpret_cast<const float4*>(P.p.xf);
  for (int sc = 0; sc < subcycles; ++sc) {
    const bool to2 = (sc % 2) == 0;
    double* Xn = to2 ? P.p.x2 : P.p.x;
    double* Un = to2 ? P.p.u2 : P.p.u;
    float4* XFn = reinterpret_cast<float4*>(to2 ? P.p.xf2 : P.p.xf);
    dem_substep_kernel<<<gw, tb, 0, s>>>(P, Xc, Uc, XFc, Xn, Un, XFn, sc + 1 == subcycles);
    ++launches;
    Xc = Xn;
    Uc = Un;
    XFc = XFn;
  }
  if (subcycles % 2 == 1) {
    dem_copy_back_kernel<<<gp, tb, 0, s>>>(P, Xc, Uc, XFc);
    ++launches;
  }
  return launches;
}

}  // namespace psm
