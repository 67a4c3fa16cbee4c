// lbm_kernels.cu -- D3Q19 stream + PSM collide (paper Sec. 2.1 and 2.3), one
// thread per cell, one warp per 32 cells of an x-row and per coverage word.
//
// The collision is written in deviation form, delta_q = f_q - w_q, and in
// opposite pairs (q, qbar) = (2k+1, 2k+2) with velocity +-c_k:
//   s_k = delta_q + delta_qbar, a_k = delta_q - delta_qbar,
//   rho - 1 = delta_0 + sum_k s_k,  j = sum_k a_k c_k,  U = j + f_ext/2 (Eq. 7)
// The equilibrium of Eq. 5 splits into a symmetric part
//   E_s,k = w_k (rho - 1 - 3/2 U.U + 9/2 (c_k.U)^2)  and antisymmetric part
//   E_a,k = 3 w_k c_k.U.
// TRT relaxes (s_k/2 - E_s,k) with omega+ and (a_k/2 - E_a,k) with omega-;
// SRT (Eq. 3) is the case omega- = omega+.  The forcing term of Eq. 8 carries
// the Guo prefactor (1 - omega/2) per part.  PSM (Eq. 17): the fluid change is
// weighted by (1 - B) and each particle i adds B_i C^s_i (Eq. 19), whose
// symmetric part per pair is E_s(U_p) - E_s(U_f) and antisymmetric part
// E_a(U_f) + E_a(U_p) - a_k; its momentum gives the force of Eq. 21.
#include "psm_internal.cuh"

namespace psm {
namespace {

__host__ __device__ constexpr int ckx(int k) {
  return (k == 0 || k == 3 || k == 4 || k == 5 || k == 6) ? 1 : 0;
}
__host__ __device__ constexpr int cky(int k) {
  return (k == 1 || k == 3 || k == 7 || k == 8) ? 1 : (k == 4 ? -1 : 0);
}
__host__ __device__ constexpr int ckz(int k) {
  return (k == 2 || k == 5 || k == 7) ? 1 : ((k == 6 || k == 8) ? -1 : 0);
}
template <typename T>
__host__ __device__ constexpr T wk(int k) {
  return k < 3 ? T(1.0 / 18.0) : T(1.0 / 36.0);
}
template <typename T>
__host__ __device__ constexpr T w0() {
  return T(1.0 / 3.0);
}

// c_k . (x, y, z) for a compile-time k, written without multiplications by 0
// or 1 (IEEE rules keep 0 * x in the instruction stream)
template <typename T>
__device__ __forceinline__ T cdot(int k, T x, T y, T z) {
  switch (k) {
    case 0: return x;
    case 1: return y;
    case 2: return z;
    case 3: return x + y;
    case 4: return x - y;
    case 5: return x + z;
    case 6: return x - z;
    case 7: return y + z;
    default: return y - z;
  }
}

// lattice weight of direction q in the canonical ordering
__host__ __device__ inline double wq(int q) {
  return q == 0 ? 1.0 / 3.0 : (q <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// neighbours of one cell with periodic wrap and wall validity.  WALLS is a
// compile-time bitmask of the axes that may have walls (bit a for axis a);
// for the other axes every link is valid and no test is compiled.
template <int WALLS>
struct NbrT {
  int X[3], Y[3], Z[3];
  bool VX[3], VY[3], VZ[3];
  __device__ void init(int x, int y, int z, int nx, int ny, int nz, int pitch_x,
                       const int* wall) {
    X[1] = x;
    X[0] = x == 0 ? nx - 1 : x - 1;
    X[2] = x == nx - 1 ? 0 : x + 1;
    VX[1] = true;
    VX[0] = !(wall[0] && x == 0);
    VX[2] = !(wall[0] && x == nx - 1);
    int ym = y == 0 ? ny - 1 : y - 1, yp = y == ny - 1 ? 0 : y + 1;
    Y[0] = ym * pitch_x;
    Y[1] = y * pitch_x;
    Y[2] = yp * pitch_x;
    VY[1] = true;
    VY[0] = !(wall[1] && y == 0);
    VY[2] = !(wall[1] && y == ny - 1);
    int zm = z == 0 ? nz - 1 : z - 1, zp = z == nz - 1 ? 0 : z + 1;
    int plane = pitch_x * ny;
    Z[0] = zm * plane;
    Z[1] = z * plane;
    Z[2] = zp * plane;
    VZ[1] = true;
    VZ[0] = !(wall[2] && z == 0);
    VZ[2] = !(wall[2] && z == nz - 1);
  }
  __device__ __forceinline__ int idx(int ox, int oy, int oz) const {
    return X[ox + 1] + Y[oy + 1] + Z[oz + 1];
  }
  __device__ __forceinline__ bool ok(int ox, int oy, int oz) const {
    const bool okx = (ox == 0 || !(WALLS & 1)) ? true : VX[ox + 1];
    const bool oky = (oy == 0 || !(WALLS & 2)) ? true : VY[oy + 1];
    const bool okz = (oz == 0 || !(WALLS & 4)) ? true : VZ[oz + 1];
    return okx && oky && okz;
  }
};
using Nbr = NbrT<7>;

template <typename T>
struct Vec2;
template <>
struct Vec2<double> {
  using type = double2;
};
template <>
struct Vec2<float> {
  using type = float2;
};

template <typename T>
__device__ __forceinline__ T ld(const T* p) {
  return __ldg(p);
}

template <typename T>
__device__ __forceinline__ const CollideCoef<T>* coef_of(const StepConst* sc);
template <>
__device__ __forceinline__ const CollideCoef<double>* coef_of<double>(const StepConst* sc) {
  return &sc->d;
}
template <>
__device__ __forceinline__ const CollideCoef<float>* coef_of<float>(const StepConst* sc) {
  return &sc->f;
}

// particle data for the solid operator
template <typename T>
__device__ __forceinline__ void load_particle(const LbmParams& P, int p, T* xp, T* up, T* op);
template <>
__device__ __forceinline__ void load_particle<double>(const LbmParams& P, int p, double* xp,
                                                      double* up, double* op) {
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    xp[a] = __ldg(&P.px[3 * p + a]);
    up[a] = __ldg(&P.pu[3 * p + a]);
    op[a] = __ldg(&P.pom[3 * p + a]);
  }
}
template <>
__device__ __forceinline__ void load_particle<float>(const LbmParams& P, int p, float* xp,
                                                     float* up, float* op) {
  float4 a = __ldg(reinterpret_cast<const float4*>(P.pxf) + p);
  float4 b = __ldg(reinterpret_cast<const float4*>(P.puf) + p);
  float4 c = __ldg(reinterpret_cast<const float4*>(P.pomf) + p);
  xp[0] = a.x; xp[1] = a.y; xp[2] = a.z;
  up[0] = b.x; up[1] = b.y; up[2] = b.z;
  op[0] = c.x; op[1] = c.y; op[2] = c.z;
}

// nearest-image offset of the cell centre from the particle centre
template <typename T>
__device__ __forceinline__ T image_offset(int i, T xp, int n, bool periodic) {
  T d = (T(i) + T(0.5)) - xp;
  if (periodic) {
    if (d > T(0.5) * T(n)) d = (T(i - n) + T(0.5)) - xp;
    else if (d < -T(0.5) * T(n)) d = (T(i + n) + T(0.5)) - xp;
  }
  return d;
}

// Shared memory of one warp for the solid operator.  Work is split in
// "jobs" (one per covered cell and occupied slot, at most 32 per round) and
// "items" (job x direction pair, 9 per job) spread over all 32 lanes, so that
// the FP64 work of a warp with a few covered cells is not repeated by its
// idle lanes.  The owner lane of a job folds the item results into its PDFs
// and its force in a fixed order.
template <typename T>
struct SolidSmem {
  T cu[32][9];     // per lane: c_k . U_f of its cell
  T am[32][9];     // per lane: antisymmetric moments a_k of its cell
  T cv[32][9];     // per job: c_k . U_p
  T con[32][7];    // per job: alpha, beta, gamma for faces and edges, B_i
  T oq[32][9];     // per job and pair: change of f_q
  T ob[32][9];     // per job and pair: change of f_qbar
  T ba[32][9];     // per job and pair: B_i A_k (momentum exchange)
  int owner[32];
};
constexpr int LBM_THREADS = 256;

template <typename T>
size_t lbm_smem_bytes() {
  return sizeof(SolidSmem<T>) * (LBM_THREADS / 32);
}

// FP32 kernels are bandwidth bound and want resident warps (3 blocks per
// SM); FP64 kernels are FP64-pipe bound and keep their registers
template <typename T, int MODE, int WALLS>
__global__ void __launch_bounds__(LBM_THREADS, sizeof(T) == 4 ? 4 : 1) lbm_kernel(LbmParams P) {
  using T2 = typename Vec2<T>::type;
  extern __shared__ __align__(16) unsigned char lbm_smem[];
  const Grid& g = P.g;
  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (warp >= g.nwords) return;  // whole warps only
  const int row = (int)(warp / g.wpr);
  const int xr = (int)(warp - (long long)row * g.wpr) * 32 + lane;
  const bool live = xr < g.nx;   // padding lanes compute on a copy of a real cell
  const int x = live ? xr : g.nx - 1;
  const int y = row % g.ny;
  const int z = row / g.ny;
  const uint32_t m = P.mask ? __ldg(&P.mask[warp]) : 0u;

  NbrT<WALLS> nb;
  nb.init(x, y, z, g.nx, g.ny, g.nz, g.nxp, g.wall);
  const int cell = nb.idx(0, 0, 0);
  // per-direction base pointers live in the kernel parameters: one address
  // computation per access.  For the AA pattern source and destination are
  // the same array: every thread reads its whole set of locations before it
  // writes the same set.
#define SRC(q) static_cast<const T*>(P.srcq[q])
#define DST(q) static_cast<T*>(P.dstq[q])

  // ---- streaming (Eq. 2 read backwards; halfway bounce-back at walls)
  T d[Q];
  d[0] = ld(SRC(0) + cell);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int cx = ckx(k), cy = cky(k), cz = ckz(k);
    const int qa = 2 * k + 1, qb = 2 * k + 2;
    if (MODE == 0) {         // pull from the other buffer
      d[qa] = nb.ok(-cx, -cy, -cz) ? ld(SRC(qa) + nb.idx(-cx, -cy, -cz)) : ld(SRC(qb) + cell);
      d[qb] = nb.ok(cx, cy, cz) ? ld(SRC(qb) + nb.idx(cx, cy, cz)) : ld(SRC(qa) + cell);
    } else if (MODE == 1) {  // AA even: own cell
      d[qa] = ld(SRC(qa) + cell);
      d[qb] = ld(SRC(qb) + cell);
    } else {                 // AA odd: swapped slots of the neighbours
      d[qa] = nb.ok(-cx, -cy, -cz) ? ld(SRC(qb) + nb.idx(-cx, -cy, -cz)) : ld(SRC(qa) + cell);
      d[qb] = nb.ok(cx, cy, cz) ? ld(SRC(qa) + nb.idx(cx, cy, cz)) : ld(SRC(qb) + cell);
    }
  }

  // ---- coverage of this cell
  bool cov = live && ((m >> lane) & 1u);
  int e = 0;
  int2 pid = make_int2(-1, -1);
  T2 Bs;
  Bs.x = T(0);
  Bs.y = T(0);
  if (cov) {
    e = __ldg(&P.base[warp]) + __popc(m & ((1u << lane) - 1u));
    if (e < P.slot_cap) {
      pid = __ldg(&P.slot_pid[e]);
      Bs = __ldg(static_cast<const T2*>(P.slot_B) + e);
    } else {
      cov = false;
    }
  }
  T B = Bs.x + Bs.y;
  if (B > T(1)) B = T(1);
  const T omB = T(1) - B;

  // ---- moments (Eqs. 6-7)
  const CollideCoef<T>* cf = coef_of<T>(P.sc);
  T a[9], sk[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    sk[k] = d[2 * k + 1] + d[2 * k + 2];
    a[k] = d[2 * k + 1] - d[2 * k + 2];
  }
  // pairwise sums: rho - 1 = delta_0 + sum s_k, j = sum a_k c_k
  const T drho = ((d[0] + (sk[0] + sk[1])) + ((sk[2] + sk[3]) + (sk[4] + sk[5]))) +
                 ((sk[6] + sk[7]) + sk[8]);
  const T jx = ((a[0] + a[3]) + (a[4] + a[5])) + a[6];
  const T jy = ((a[1] + a[3]) - (a[4] - a[7])) + a[8];
  const T jz = ((a[2] + a[5]) - (a[6] - a[7])) - a[8];
  const T Ux = jx + __ldg(&cf->hf[0]);
  const T Uy = jy + __ldg(&cf->hf[1]);
  const T Uz = jz + __ldg(&cf->hf[2]);
  const T uu = Ux * Ux + Uy * Uy + Uz * Uz;
  const T Uf = Ux * __ldg(&cf->f[0]) + Uy * __ldg(&cf->f[1]) + Uz * __ldg(&cf->f[2]);
  const T base0 = drho - T(1.5) * uu;

  // ---- fluid relaxation + forcing, weighted by (1 - B).  Per pair:
  //   symmetric change  = -omega+/2 s_k + omega+ E_s,k + forcing
  //                     = -omega+/2 s_k + ((9/2 omega+ w) c.U + G_k) c.U + C_c
  //   antisymmetric     = -omega-/2 a_k + 3 omega- w c.U + F_k
  // with C_c = omega+ w base0 + H_c U.f once per class.
  {
    const T dl = __ldg(&cf->nwp) * d[0] + (__ldg(&cf->wpw0) * base0 + __ldg(&cf->H[0]) * Uf);
    d[0] += omB * dl;
  }
  const T C0 = __ldg(&cf->wpw[0]) * base0 + __ldg(&cf->H[1]) * Uf;
  const T C1 = __ldg(&cf->wpw[1]) * base0 + __ldg(&cf->H[2]) * Uf;
  const T mhwp = __ldg(&cf->mhwp), mhwm = __ldg(&cf->mhwm);
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int c = k < 3 ? 0 : 1;
    const T cu = cdot<T>(k, Ux, Uy, Uz);
    const T ds = mhwp * sk[k] + ((__ldg(&cf->A[c]) * cu + __ldg(&cf->Gs[k])) * cu + (c ? C1 : C0));
    const T da = mhwm * a[k] + (__ldg(&cf->D[c]) * cu + __ldg(&cf->Fa[k]));
    d[2 * k + 1] += omB * (ds + da);
    d[2 * k + 2] += omB * (ds - da);
  }

  // ---- solid operator of each overlapping particle (Eqs. 19-21).  In FP64
  // (1/58 of the FP32 rate here) the work is shared out over the lanes of the
  // warp; in FP32 each covered lane does its own cell.
  if (sizeof(T) == 4 && cov) {
#pragma unroll 1
    for (int sl = 0; sl < 2; ++sl) {
      const int p = sl ? pid.y : pid.x;
      if (p < 0) continue;
      const T Bi = sl ? Bs.y : Bs.x;
      T xp[3], up[3], op[3];
      load_particle<T>(P, p, xp, up, op);
      const T dx = image_offset<T>(x, xp[0], g.nx, !g.wall[0]);
      const T dy = image_offset<T>(y, xp[1], g.ny, !g.wall[1]);
      const T dz = image_offset<T>(z, xp[2], g.nz, !g.wall[2]);
      // Eq. 20: surface velocity at the cell centre
      const T Vx = up[0] + (op[1] * dz - op[2] * dy);
      const T Vy = up[1] + (op[2] * dx - op[0] * dz);
      const T Vz = up[2] + (op[0] * dy - op[1] * dx);
      const T dU2 = (Vx * Vx + Vy * Vy + Vz * Vz) - uu;
      d[0] += Bi * (T(-1.5) * w0<T>() * dU2);
      T ax = T(0), ay = T(0), az = T(0);
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const T w = wk<T>(k);
        const T cu = cdot<T>(k, Ux, Uy, Uz);
        const T cv = cdot<T>(k, Vx, Vy, Vz);
        const T Sv = cv + cu;
        const T BdS = (T(4.5) * w * Bi) * ((cv - cu) * Sv) + (T(-1.5) * w) * (Bi * dU2);
        const T BA = (T(3) * w * Bi) * Sv - Bi * a[k];
        d[2 * k + 1] += BdS + BA;
        d[2 * k + 2] += BdS - BA;
        if (ckx(k) > 0) ax += BA;
        if (cky(k) > 0) ay += BA;
        if (cky(k) < 0) ay -= BA;
        if (ckz(k) > 0) az += BA;
        if (ckz(k) < 0) az -= BA;
      }
      // Eq. 21: B_i sum_q C^s_q c_qbar = -2 sum_k B_i A_k c_k
      T* o = static_cast<T*>(P.slot_Fc) + 6LL * e + 3 * sl;
      o[0] = T(-2) * ax;
      o[1] = T(-2) * ay;
      o[2] = T(-2) * az;
    }
  }
  if (sizeof(T) == 8 && m != 0u) {
    SolidSmem<T>& S = reinterpret_cast<SolidSmem<T>*>(lbm_smem)[threadIdx.x >> 5];
    const bool has0 = cov && pid.x >= 0, has1 = cov && pid.y >= 0;
    const unsigned b0 = __ballot_sync(0xffffffffu, has0);
    const unsigned b1 = __ballot_sync(0xffffffffu, has1);
    const unsigned below = (1u << lane) - 1u;
    const int J0 = __popc(b0), J = J0 + __popc(b1);
    const int j0 = __popc(b0 & below), j1 = J0 + __popc(b1 & below);
    if (has0 || has1) {
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        S.cu[lane][k] = cdot<T>(k, Ux, Uy, Uz);
        S.am[lane][k] = a[k];
      }
    }
    for (int c0 = 0; c0 < J; c0 += 32) {
      // job set-up by the owner lanes: surface velocity (Eq. 20) and the
      // per-job constants of the item arithmetic
#pragma unroll
      for (int sl = 0; sl < 2; ++sl) {
        const bool has = sl ? has1 : has0;
        const int jj = (sl ? j1 : j0) - c0;
        if (has && jj >= 0 && jj < 32) {
          const int p = sl ? pid.y : pid.x;
          const T Bi = sl ? Bs.y : Bs.x;
          T xp[3], up[3], op[3];
          load_particle<T>(P, p, xp, up, op);
          const T dx = image_offset<T>(x, xp[0], g.nx, !g.wall[0]);
          const T dy = image_offset<T>(y, xp[1], g.ny, !g.wall[1]);
          const T dz = image_offset<T>(z, xp[2], g.nz, !g.wall[2]);
          const T Vx = up[0] + (op[1] * dz - op[2] * dy);
          const T Vy = up[1] + (op[2] * dx - op[0] * dz);
          const T Vz = up[2] + (op[0] * dy - op[1] * dx);
          const T dU2 = (Vx * Vx + Vy * Vy + Vz * Vz) - uu;
          d[0] += Bi * (T(-1.5) * w0<T>() * dU2);
#pragma unroll
          for (int k = 0; k < 9; ++k)
            S.cv[jj][k] = cdot<T>(k, Vx, Vy, Vz);
          const T BdU = Bi * dU2;
          S.con[jj][0] = (T(4.5) * wk<T>(0)) * Bi;
          S.con[jj][1] = (T(-1.5) * wk<T>(0)) * BdU;
          S.con[jj][2] = (T(3) * wk<T>(0)) * Bi;
          S.con[jj][3] = (T(4.5) * wk<T>(3)) * Bi;
          S.con[jj][4] = (T(-1.5) * wk<T>(3)) * BdU;
          S.con[jj][5] = (T(3) * wk<T>(3)) * Bi;
          S.con[jj][6] = Bi;
          S.owner[jj] = lane;
        }
      }
      __syncwarp();
      // items: job j, pair k.  C^s has symmetric part B_i w_k (9/2 (cv^2 -
      // cu^2) - 3/2 dU2) and antisymmetric part B_i (3 w_k (cu + cv) - a_k)
      const int nj = J - c0 < 32 ? J - c0 : 32;
      for (int t = lane; t < 9 * nj; t += 32) {
        const int j = t / 9, k = t - 9 * j;
        const int L = S.owner[j];
        const T cu = S.cu[L][k], cv = S.cv[j][k];
        const int cl = k < 3 ? 0 : 3;
        const T Dv = cv - cu, Sv = cv + cu;
        const T BdS = S.con[j][cl] * (Dv * Sv) + S.con[j][cl + 1];
        const T BA = S.con[j][cl + 2] * Sv - S.con[j][6] * S.am[L][k];
        S.oq[j][k] = BdS + BA;
        S.ob[j][k] = BdS - BA;
        S.ba[j][k] = BA;
      }
      __syncwarp();
      // owners fold the results in a fixed order; Eq. 21 per slot:
      // B_i sum_q C^s_q c_qbar = -2 sum_k B_i A_k c_k
#pragma unroll
      for (int sl = 0; sl < 2; ++sl) {
        const bool has = sl ? has1 : has0;
        const int jj = (sl ? j1 : j0) - c0;
        if (has && jj >= 0 && jj < 32) {
          T ax = T(0), ay = T(0), az = T(0);
#pragma unroll
          for (int k = 0; k < 9; ++k) {
            d[2 * k + 1] += S.oq[jj][k];
            d[2 * k + 2] += S.ob[jj][k];
            const T A = S.ba[jj][k];
            if (ckx(k) > 0) ax += A;
            if (cky(k) > 0) ay += A;
            if (cky(k) < 0) ay -= A;
            if (ckz(k) > 0) az += A;
            if (ckz(k) < 0) az -= A;
          }
          T* o = static_cast<T*>(P.slot_Fc) + 6LL * e + 3 * sl;
          o[0] = T(-2) * ax;
          o[1] = T(-2) * ay;
          o[2] = T(-2) * az;
        }
      }
      __syncwarp();
    }
  }
  if (!live) return;

  // ---- store
  DST(0)[cell] = d[0];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const int cx = ckx(k), cy = cky(k), cz = ckz(k);
    const int qa = 2 * k + 1, qb = 2 * k + 2;
    if (MODE == 0) {
      DST(qa)[cell] = d[qa];
      DST(qb)[cell] = d[qb];
    } else if (MODE == 1) {
      DST(qb)[cell] = d[qa];
      DST(qa)[cell] = d[qb];
    } else {
      if (nb.ok(cx, cy, cz)) DST(qa)[nb.idx(cx, cy, cz)] = d[qa];
      else DST(qb)[cell] = d[qa];
      if (nb.ok(-cx, -cy, -cz)) DST(qb)[nb.idx(-cx, -cy, -cz)] = d[qb];
      else DST(qa)[cell] = d[qb];
    }
  }
#undef SRC
#undef DST
}

// canonical FP64 f~ (unpadded, full f = w + delta) from the storage layout
template <typename T>
__global__ void to_canonical_kernel(Grid g, const T* __restrict__ buf, int aa, int parity,
                                    double* __restrict__ out) {
  const long long N = (long long)g.nx * g.ny * g.nz;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % g.nx);
    const int y = (int)((c / g.nx) % g.ny);
    const int z = (int)(c / ((long long)g.nx * g.ny));
    Nbr nb;
    nb.init(x, y, z, g.nx, g.ny, g.nz, g.nxp, g.wall);
    const int cell = nb.idx(0, 0, 0);
    const long long NC = g.ncell;
    out[c] = wq(0) + (double)buf[cell];
    for (int k = 0; k < 9; ++k) {
      const int cx = ckx(k), cy = cky(k), cz = ckz(k);
      const int qa = 2 * k + 1, qb = 2 * k + 2;
      long long ia, ib;
      if (!aa) {
        ia = qa * NC + cell;
        ib = qb * NC + cell;
      } else if (parity == 1) {
        ia = qb * NC + cell;
        ib = qa * NC + cell;
      } else {
        ia = nb.ok(cx, cy, cz) ? qa * NC + nb.idx(cx, cy, cz) : qb * NC + cell;
        ib = nb.ok(-cx, -cy, -cz) ? qb * NC + nb.idx(-cx, -cy, -cz) : qa * NC + cell;
      }
      out[qa * N + c] = wq(qa) + (double)buf[ia];
      out[qb * N + c] = wq(qb) + (double)buf[ib];
    }
  }
}

// storage layout from canonical f~; the AA buffer is written in the state
// "next step is even" (each cell holds its streamed PDFs)
template <typename T>
__global__ void from_canonical_kernel(Grid g, const double* __restrict__ in, int aa,
                                      T* __restrict__ buf) {
  const long long N = (long long)g.nx * g.ny * g.nz;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % g.nx);
    const int y = (int)((c / g.nx) % g.ny);
    const int z = (int)(c / ((long long)g.nx * g.ny));
    Nbr nc;  // neighbours in the unpadded canonical array
    nc.init(x, y, z, g.nx, g.ny, g.nz, g.nx, g.wall);
    const long long cell = (long long)x + (long long)g.nxp * (y + (long long)g.ny * z);
    const long long NC = g.ncell;
    buf[cell] = (T)(in[c] - wq(0));
    for (int k = 0; k < 9; ++k) {
      const int cx = ckx(k), cy = cky(k), cz = ckz(k);
      const int qa = 2 * k + 1, qb = 2 * k + 2;
      double va, vb;
      if (!aa) {
        va = in[qa * N + c];
        vb = in[qb * N + c];
      } else {
        va = nc.ok(-cx, -cy, -cz) ? in[qa * N + nc.idx(-cx, -cy, -cz)] : in[qb * N + c];
        vb = nc.ok(cx, cy, cz) ? in[qb * N + nc.idx(cx, cy, cz)] : in[qa * N + c];
      }
      buf[qa * NC + cell] = (T)(va - wq(qa));
      buf[qb * NC + cell] = (T)(vb - wq(qb));
    }
  }
}

// rho and U of the streamed canonical field (Eqs. 6-7)
__global__ void macroscopic_kernel(Grid g, const double* __restrict__ f, const StepConst* sc,
                                   double* __restrict__ rho, double* __restrict__ u) {
  const long long N = (long long)g.nx * g.ny * g.nz;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % g.nx);
    const int y = (int)((c / g.nx) % g.ny);
    const int z = (int)(c / ((long long)g.nx * g.ny));
    Nbr nc;
    nc.init(x, y, z, g.nx, g.ny, g.nz, g.nx, g.wall);
    double r = f[c], jx = 0.0, jy = 0.0, jz = 0.0;
    for (int k = 0; k < 9; ++k) {
      const int cx = ckx(k), cy = cky(k), cz = ckz(k);
      const int qa = 2 * k + 1, qb = 2 * k + 2;
      const double va = nc.ok(-cx, -cy, -cz) ? f[qa * N + nc.idx(-cx, -cy, -cz)] : f[qb * N + c];
      const double vb = nc.ok(cx, cy, cz) ? f[qb * N + nc.idx(cx, cy, cz)] : f[qa * N + c];
      r += va + vb;
      jx += (va - vb) * cx;
      jy += (va - vb) * cy;
      jz += (va - vb) * cz;
    }
    rho[c] = r;
    u[c] = jx + 0.5 * sc->fext[0];
    u[N + c] = jy + 0.5 * sc->fext[1];
    u[2 * N + c] = jz + 0.5 * sc->fext[2];
  }
}

// fixed-order sums of mass and momentum over the canonical field
constexpr int SUM_THREADS = 256;
__global__ void sums_partial_kernel(long long N, const double* __restrict__ f,
                                    double* __restrict__ partials) {
  __shared__ double sh[4][SUM_THREADS];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  const long long per = (N + gridDim.x - 1) / gridDim.x;
  const long long lo = per * blockIdx.x;
  const long long hi = lo + per < N ? lo + per : N;
  for (long long c = lo + threadIdx.x; c < hi; c += SUM_THREADS) {
    double r = f[c], jx = 0.0, jy = 0.0, jz = 0.0;
    for (int k = 0; k < 9; ++k) {
      const double va = f[(2 * k + 1) * N + c], vb = f[(2 * k + 2) * N + c];
      r += va + vb;
      jx += (va - vb) * ckx(k);
      jy += (va - vb) * cky(k);
      jz += (va - vb) * ckz(k);
    }
    acc[0] += r;
    acc[1] += jx;
    acc[2] += jy;
    acc[3] += jz;
  }
  for (int i = 0; i < 4; ++i) sh[i][threadIdx.x] = acc[i];
  __syncthreads();
  for (int s = SUM_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int i = 0; i < 4; ++i) sh[i][threadIdx.x] += sh[i][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int i = 0; i < 4; ++i) partials[4 * blockIdx.x + i] = sh[i][0];
}

__global__ void sums_final_kernel(int nparts, const double* __restrict__ partials,
                                  double* __restrict__ out) {
  if (threadIdx.x < 4) {
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += partials[4 * b + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

}  // namespace

template <typename T>
size_t lbm_dyn_smem() {
  return sizeof(T) == 8 ? lbm_smem_bytes<T>() : 0;
}

template <typename T, int W>
int configure_walls() {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  const int sm = (int)lbm_dyn_smem<T>();
  int bad = 0;
  bad |= cudaFuncSetAttribute(lbm_kernel<T, 0, W>, a, sm) != cudaSuccess;
  bad |= cudaFuncSetAttribute(lbm_kernel<T, 1, W>, a, sm) != cudaSuccess;
  bad |= cudaFuncSetAttribute(lbm_kernel<T, 2, W>, a, sm) != cudaSuccess;
  return bad;
}

int lbm_configure() {
  return configure_walls<float, 0>() | configure_walls<float, 1>() | configure_walls<float, 7>() |
         configure_walls<double, 0>() | configure_walls<double, 1>() |
         configure_walls<double, 7>();
}

template <typename T, int W>
void launch_lbm_t(const LbmParams& P, int mode, unsigned grid, cudaStream_t s) {
  const size_t sm = lbm_dyn_smem<T>();
  if (mode == 0) lbm_kernel<T, 0, W><<<grid, LBM_THREADS, sm, s>>>(P);
  else if (mode == 1) lbm_kernel<T, 1, W><<<grid, LBM_THREADS, sm, s>>>(P);
  else lbm_kernel<T, 2, W><<<grid, LBM_THREADS, sm, s>>>(P);
}

template <typename T>
void launch_lbm_w(const LbmParams& P, int mode, unsigned grid, cudaStream_t s) {
  const int w = P.g.wall[0] | (P.g.wall[1] << 1) | (P.g.wall[2] << 2);
  if (w == 0) launch_lbm_t<T, 0>(P, mode, grid, s);
  else if (w == 1) launch_lbm_t<T, 1>(P, mode, grid, s);
  else launch_lbm_t<T, 7>(P, mode, grid, s);
}

int launch_lbm(const LbmParams& P0, int fp32, int mode, cudaStream_t s) {
  LbmParams P = P0;
  const size_t esz = fp32 ? sizeof(float) : sizeof(double);
  for (int q = 0; q < Q; ++q) {
    P.srcq[q] = static_cast<const char*>(P.src) + esz * (size_t)q * P.g.ncell;
    P.dstq[q] = static_cast<char*>(P.dst) + esz * (size_t)q * P.g.ncell;
  }
  const long long threads = P.g.nwords * 32;
  const unsigned grid = (unsigned)((threads + LBM_THREADS - 1) / LBM_THREADS);
  if (fp32) launch_lbm_w<float>(P, mode, grid, s);
  else launch_lbm_w<double>(P, mode, grid, s);
  return 1;
}

static unsigned grid_for(long long n, int block) {
  long long b = (n + block - 1) / block;
  if (b > 152LL * 64) b = 152LL * 64;
  return (unsigned)(b > 0 ? b : 1);
}

int launch_to_canonical(const Grid& g, const void* buf, int fp32, int aa_parity, int aa,
                        double* out, cudaStream_t s) {
  const long long N = (long long)g.nx * g.ny * g.nz;
  if (fp32)
    to_canonical_kernel<float><<<grid_for(N, 256), 256, 0, s>>>(
        g, static_cast<const float*>(buf), aa, aa_parity, out);
  else
    to_canonical_kernel<double><<<grid_for(N, 256), 256, 0, s>>>(
        g, static_cast<const double*>(buf), aa, aa_parity, out);
  return 1;
}

int launch_from_canonical(const Grid& g, const double* in, void* buf, int fp32, int aa,
                             cudaStream_t s) {
  const long long N = (long long)g.nx * g.ny * g.nz;
  if (fp32)
    from_canonical_kernel<float><<<grid_for(N, 256), 256, 0, s>>>(g, in, aa,
                                                                  static_cast<float*>(buf));
  else
    from_canonical_kernel<double><<<grid_for(N, 256), 256, 0, s>>>(g, in, aa,
                                                                   static_cast<double*>(buf));
  return 1;
}

int launch_macroscopic(const Grid& g, const double* f, const StepConst* sc, double* rho,
                       double* u, cudaStream_t s) {
  const long long N = (long long)g.nx * g.ny * g.nz;
  macroscopic_kernel<<<grid_for(N, 256), 256, 0, s>>>(g, f, sc, rho, u);
  return 1;
}

int launch_sums(const Grid& g, const double* f, double* partials, int nparts, double* out4,
                cudaStream_t s) {
  const long long N = (long long)g.nx * g.ny * g.nz;
  sums_partial_kernel<<<nparts, SUM_THREADS, 0, s>>>(N, f, partials);
  sums_final_kernel<<<1, 32, 0, s>>>(nparts, partials, out4);
  return 2;
}

// per-step constants: fluid force density (body force and the counter force
// of the buoyancy-corrected gravity) and the forcing coefficients
template <typename T>
__device__ void fill_coef(CollideCoef<T>& c, const double* f, double wp, double wm) {
  const double gp = 1.0 - 0.5 * wp, gm = 1.0 - 0.5 * wm;
  for (int a = 0; a < 3; ++a) {
    c.hf[a] = (T)(0.5 * f[a]);
    c.f[a] = (T)f[a];
  }
  for (int k = 0; k < 9; ++k) {
    const double cfk = ckx(k) * f[0] + cky(k) * f[1] + ckz(k) * f[2];
    const double w = wk<double>(k);
    c.Gs[k] = (T)(gp * 9.0 * w * cfk);
    c.Fa[k] = (T)(gm * 3.0 * w * cfk);
  }
  c.H[0] = (T)(-3.0 * (1.0 / 3.0) * gp);
  c.H[1] = (T)(-3.0 * (1.0 / 18.0) * gp);
  c.H[2] = (T)(-3.0 * (1.0 / 36.0) * gp);
  c.nwp = (T)(-wp);
  c.mhwp = (T)(-0.5 * wp);
  c.mhwm = (T)(-0.5 * wm);
  c.wpw0 = (T)(wp * (1.0 / 3.0));
  for (int cl = 0; cl < 2; ++cl) {
    const double w = cl ? 1.0 / 36.0 : 1.0 / 18.0;
    c.wpw[cl] = (T)(wp * w);
    c.A[cl] = (T)(4.5 * w * wp);
    c.D[cl] = (T)(3.0 * w * wm);
  }
}

__global__ void step_const_kernel(MapParams P) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  StepConst* sc = P.sc;
  const double vf = sc->vfluid;
  double f[3];
  for (int a = 0; a < 3; ++a) {
    f[a] = P.fbody[a] - ((P.G[a] != 0.0 && vf > 0.0) ? P.G[a] / vf : 0.0);
    sc->fext[a] = f[a];
  }
  fill_coef<double>(sc->d, f, P.omega_p, P.omega_m);
  fill_coef<float>(sc->f, f, P.omega_p, P.omega_m);
}

int launch_step_const(MapParams P, cudaStream_t s) {
  step_const_kernel<<<1, 32, 0, s>>>(P);
  return 1;
}

}  // namespace psm
