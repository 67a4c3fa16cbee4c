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
#include "df.cuh"
#include "psm_internal.cuh"

namespace psm {
namespace {

// element traits: FP64 (the warp-shared solid operator, FP64-pipe bound), or
// a form that runs on the FP32 pipes (FP32 deviations, double-float pairs)
template <typename T>
constexpr bool kFP64 = false;
template <>
constexpr bool kFP64<double> = true;
template <typename T>
constexpr bool kDF = false;
template <>
constexpr bool kDF<df> = true;
// slot records and per-slot forces are stored in the form's own precision
// (FP32, FP64, double-float pairs)
__device__ __forceinline__ double as_double(double v) { return v; }
__device__ __forceinline__ double as_double(float v) { return (double)v; }
__device__ __forceinline__ double as_double(df v) { return to_double(v); }
template <typename T>
__device__ __forceinline__ T from_double(double v) {
  return (T)v;
}
template <>
__device__ __forceinline__ df from_double<df>(double v) {
  return df(v);
}
// sign flag and magnitude of a record's weight (slot 0's weight is negated
// when a second particle shares the cell)
__device__ __forceinline__ bool neg_flag(float v) { return signbit(v); }
__device__ __forceinline__ bool neg_flag(double v) { return signbit(v); }
__device__ __forceinline__ bool neg_flag(df v) { return signbit(v.hi); }
__device__ __forceinline__ float magnitude(float v) { return fabsf(v); }
__device__ __forceinline__ double magnitude(double v) { return fabs(v); }
__device__ __forceinline__ df magnitude(df v) { return signbit(v.hi) ? -v : v; }

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
__device__ __forceinline__ df ld(const df* p) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  return df(v.x, v.y);
}

// four consecutive coefficients (16-byte aligned) in 16-byte loads
__device__ __forceinline__ void ld4(const float* p, float* o) {
  const float4 v = __ldg(reinterpret_cast<const float4*>(p));
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ld4(const double* p, double* o) {
  const double2 u = __ldg(reinterpret_cast<const double2*>(p));
  const double2 v = __ldg(reinterpret_cast<const double2*>(p) + 1);
  o[0] = u.x; o[1] = u.y; o[2] = v.x; o[3] = v.y;
}
__device__ __forceinline__ void ld4(const df* p, df* o) {
  const float4 u = __ldg(reinterpret_cast<const float4*>(p));
  const float4 v = __ldg(reinterpret_cast<const float4*>(p) + 1);
  o[0] = df(u.x, u.y); o[1] = df(u.z, u.w); o[2] = df(v.x, v.y); o[3] = df(v.z, v.w);
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
template <>
__device__ __forceinline__ const CollideCoef<df>* coef_of<df>(const StepConst* sc) {
  return &sc->x;
}

// Shared memory of one warp for the FP64 solid operator.  Work is split in
// "jobs" (one per covered cell and occupied slot) and "items" (job x
// direction pair, 9 per job) spread over all 32 lanes, so that the FP64 work
// of a warp with a few covered cells is not repeated by its idle lanes.  The
// items add their results to a shared copy of the owner lane's PDFs, slot 0
// before slot 1.
template <typename T>
struct SolidSmem {
  T cu[32][9];     // per lane: c_k . U_f of its cell
  T am[32][9];     // per lane: antisymmetric moments a_k of its cell
  T dd[32][18];    // per lane: its PDFs 1..18 while the items add to them
  T cv[32][9];     // per job: c_k . U_p
  T con[32][7];    // per job: alpha, beta, gamma for faces and edges, B_i
  int owner[32];
};
constexpr int LBM_THREADS = 256;

template <typename T>
size_t lbm_smem_bytes() {
  return sizeof(SolidSmem<T>) * (LBM_THREADS / 32);
}

// Force of one slot on its particle (Eq. 21): B_i sum_q C^s_q c_qbar =
// -2 B_i sum_k A_k c_k over the pairs, with A_k = 3 w_k c_k.(U_f + U_p) - a_k.
// The lattice sum over the pairs, sum_k w_k c_k c_k^T = I/6, reduces it
// exactly to B_i ((U_f + U_p)/2 - j) (-2) = B_i (U_f - U_p - f_ext), since
// j = U_f - f_ext/2 (Eq. 7).
template <typename T>
__device__ __forceinline__ void slot_force(const LbmParams& P, int e, int sl, T Bi, T dux, T duy,
                                           T duz, const T* f) {
  T* o = static_cast<T*>(P.slot_Fc) + 3 * ((long long)sl * P.slot_cap + e);
  o[0] = Bi * (dux - f[0]);
  o[1] = Bi * (duy - f[1]);
  o[2] = Bi * (duz - f[2]);
}

// Coverage of one cell and its first slot record (m: coverage word of its
// warp, eb: slot of the word's first covered cell).  A slot record holds the
// particle's surface velocity at the cell centre (Eq. 20) and the weight B_i,
// both written by the mapping; the sign of slot 0's weight tells whether a
// second particle shares the cell.  Issued ahead of the PDF reads where the
// kernel can.
template <typename T>
struct SlotRec {
  bool cov;  // covered, and its record exists
  int e;     // slot index
  T r0[4];   // slot 0: surface velocity, signed weight
};
template <typename T>
__device__ __forceinline__ void load_slot_rec(const LbmParams& P, uint32_t m, int eb, int lane,
                                              bool live, SlotRec<T>& R) {
  R.cov = live && ((m >> lane) & 1u);
  R.e = 0;
#pragma unroll
  for (int i = 0; i < 4; ++i) R.r0[i] = T(0);
  if (R.cov) {
    R.e = eb + __popc(m & ((1u << lane) - 1u));
    if (R.e < P.slot_cap) ld4(static_cast<const T*>(P.slot_V) + 4LL * R.e, R.r0);
    else R.cov = false;
  }
}

// Collision of one cell (Eqs. 3-8 and 17-21) on the PDFs d gathered by the
// streaming step; the warp's 32 lanes hold the 32 cells of coverage word
// `word` (padding lanes compute on a copy of a real cell).  FP64 kernels
// pass the warp's SolidSmem.
// `pre` holds the cell's slot record when the kernel loaded it ahead (PRE),
// else the record is read here.
template <typename T, bool PRE>
__device__ __forceinline__ void psm_collide(const LbmParams& P, unsigned word, int lane, bool live,
                                            T* d, SolidSmem<T>* solid, uint32_t m, int eb,
                                            const SlotRec<T>* pre) {
  // ---- the cell's slots; the second one's record is read only when present
  bool cov, has1 = false;
  int e = 0;
  T r0[4] = {T(0), T(0), T(0), T(0)}, r1[4] = {T(0), T(0), T(0), T(0)};
  if constexpr (PRE) {
    cov = pre->cov;
    e = pre->e;
#pragma unroll
    for (int i = 0; i < 4; ++i) r0[i] = pre->r0[i];
  } else {
    cov = live && ((m >> lane) & 1u);
    if (cov) {
      e = eb + __popc(m & ((1u << lane) - 1u));
      if (e < P.slot_cap) ld4(static_cast<const T*>(P.slot_V) + 4LL * e, r0);
      else cov = false;
    }
  }
  if (cov) {
    has1 = neg_flag(r0[3]);
    r0[3] = magnitude(r0[3]);
    if (has1) ld4(static_cast<const T*>(P.slot_V) + 4LL * (P.slot_cap + e), r1);
  }
  T omB = T(1);  // 1 - B; the FP64 operations only where a lane is covered
  if (cov) {
    T B = r0[3] + r1[3];
    if (B > T(1)) B = T(1);
    omB = T(1) - B;
  }

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
  T h[16];
  ld4(cf->head, h);
  ld4(cf->head + 4, h + 4);
  ld4(cf->head + 8, h + 8);
  ld4(cf->head + 12, h + 12);
  const T Ux = jx + h[CC_HF];
  const T Uy = jy + h[CC_HF + 1];
  const T Uz = jz + h[CC_HF + 2];
  const T uu = Ux * Ux + Uy * Uy + Uz * Uz;
  const T Uf = Ux * h[CC_F] + Uy * h[CC_F + 1] + Uz * h[CC_F + 2];
  const T base0 = drho - T(1.5) * uu;

  // ---- fluid relaxation + forcing, weighted by (1 - B).  Per pair:
  //   symmetric change  = -omega+/2 s_k + omega+ E_s,k + forcing
  //                     = -omega+/2 s_k + ((9/2 omega+ w) c.U + G_k) c.U + C_c
  //   antisymmetric     = -omega-/2 a_k + 3 omega- w c.U + F_k
  // with C_c = omega+ w base0 + H_c U.f once per class.
  // the (1 - B) weight is a multiply-add in FP32/FP64; in double-float it is
  // a product of its own, skipped in warps without a covered cell
  const bool weighted = !kDF<T> || m != 0u;
  {
    const T dl = h[CC_NWP] * d[0] + (h[CC_WPW0] * base0 + h[CC_H] * Uf);
    if (kDF<T> && !weighted) d[0] += dl;
    else d[0] += omB * dl;
  }
  const T C0 = h[CC_WPW] * base0 + h[CC_H + 1] * Uf;
  const T C1 = h[CC_WPW + 1] * base0 + h[CC_H + 2] * Uf;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    T pk[4];
    ld4(cf->pair[k], pk);
    const T cu = cdot<T>(k, Ux, Uy, Uz);
    const T ds = h[CC_MHWP] * sk[k] + ((pk[2] * cu + pk[0]) * cu + (k < 3 ? C0 : C1));
    const T da = h[CC_MHWM] * a[k] + (pk[3] * cu + pk[1]);
    if (kDF<T> && !weighted) {
      d[2 * k + 1] += ds + da;
      d[2 * k + 2] += ds - da;
    } else {
      d[2 * k + 1] += omB * (ds + da);
      d[2 * k + 2] += omB * (ds - da);
    }
  }

  // ---- solid operator of each overlapping particle (Eqs. 19-21).  In FP64
  // (1/64 of the FP32 rate here) the work is shared out over the lanes of the
  // warp; in FP32 each covered lane does its own cell.
  if constexpr (!kFP64<T>) {
  if (cov) {
#pragma unroll 1
    for (int sl = 0; sl < 2; ++sl) {
      if (sl && !has1) continue;
      const T Vx = sl ? r1[0] : r0[0], Vy = sl ? r1[1] : r0[1], Vz = sl ? r1[2] : r0[2];
      const T Bi = sl ? r1[3] : r0[3];
      const T dU2 = (Vx * Vx + Vy * Vy + Vz * Vz) - uu;
      d[0] += Bi * (T(-1.5) * w0<T>() * dU2);
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
      }
      slot_force<T>(P, e, sl, Bi, Ux - Vx, Uy - Vy, Uz - Vz, h + CC_F);
    }
  }
  } else if (m != 0u) {
    SolidSmem<T>& S = *solid;
    const bool has0 = cov, hs1 = cov && has1;
    const unsigned b0 = __ballot_sync(0xffffffffu, has0);
    const unsigned b1 = __ballot_sync(0xffffffffu, hs1);
    const unsigned below = (1u << lane) - 1u;
    if (has0) {
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        S.cu[lane][k] = cdot<T>(k, Ux, Uy, Uz);
        S.am[lane][k] = a[k];
      }
#pragma unroll
      for (int q = 1; q < Q; ++q) S.dd[lane][q - 1] = d[q];
    }
    // the jobs of slot 0, then those of slot 1: within a pass each owner lane
    // has at most one job, so no two items of a pass update the same PDF
#pragma unroll
    for (int sl = 0; sl < 2; ++sl) {
      const unsigned bs = sl ? b1 : b0;
      if (bs == 0u) continue;
      const int Js = __popc(bs);
      if (sl ? hs1 : has0) {
        // job set-up by the owner lane: the per-job constants of the item
        // arithmetic and the slot's force (Eq. 21)
        const int jj = __popc(bs & below);
        const T Vx = sl ? r1[0] : r0[0], Vy = sl ? r1[1] : r0[1], Vz = sl ? r1[2] : r0[2];
        const T Bi = sl ? r1[3] : r0[3];
        const T dU2 = (Vx * Vx + Vy * Vy + Vz * Vz) - uu;
        d[0] += Bi * (T(-1.5) * w0<T>() * dU2);
#pragma unroll
        for (int k = 0; k < 9; ++k) S.cv[jj][k] = cdot<T>(k, Vx, Vy, Vz);
        const T BdU = Bi * dU2;
        S.con[jj][0] = (T(4.5) * wk<T>(0)) * Bi;
        S.con[jj][1] = (T(-1.5) * wk<T>(0)) * BdU;
        S.con[jj][2] = (T(3) * wk<T>(0)) * Bi;
        S.con[jj][3] = (T(4.5) * wk<T>(3)) * Bi;
        S.con[jj][4] = (T(-1.5) * wk<T>(3)) * BdU;
        S.con[jj][5] = (T(3) * wk<T>(3)) * Bi;
        S.con[jj][6] = Bi;
        S.owner[jj] = lane;
        slot_force<T>(P, e, sl, Bi, Ux - Vx, Uy - Vy, Uz - Vz, h + CC_F);
      }
      __syncwarp();
      // items: job j, pair k, added to the owner's PDFs.  C^s has symmetric
      // part B_i w_k (9/2 (cv^2 - cu^2) - 3/2 dU2) and antisymmetric part
      // B_i (3 w_k (cu + cv) - a_k)
      for (int t = lane; t < 9 * Js; t += 32) {
        const int j = t / 9, k = t - 9 * j;
        const int L = S.owner[j];
        const T cu = S.cu[L][k], cv = S.cv[j][k];
        const int cl = k < 3 ? 0 : 3;
        const T Dv = cv - cu, Sv = cv + cu;
        const T BdS = S.con[j][cl] * (Dv * Sv) + S.con[j][cl + 1];
        const T BA = S.con[j][cl + 2] * Sv - S.con[j][6] * S.am[L][k];
        S.dd[L][2 * k] += BdS + BA;
        S.dd[L][2 * k + 1] += BdS - BA;
      }
      __syncwarp();
    }
    if (has0) {
#pragma unroll
      for (int q = 1; q < Q; ++q) d[q] = S.dd[lane][q - 1];
    }
  }
  if constexpr (kDF<T>) {
    // stored pairs are canonical, so their low parts do not grow over steps
#pragma unroll
    for (int q = 0; q < Q; ++q) d[q] = renorm_fast(d[q]);
  }
}

// ---- open z faces (the velocity inflow and pressure outflow of the
// fluidized bed, Sec. 4.1): type of the open face a pulled link with source
// offset (ox, oy, oz) leaves through, or 0 (a link that also leaves through a
// side wall is bounced back)
template <int WALLS>
__device__ __forceinline__ int open_face(const Grid& g, const NbrT<WALLS>& nb, int ox, int oy,
                                         int oz) {
  if constexpr (!(WALLS & 4)) {
    return 0;
  } else {
    if (oz == 0 || nb.ok(0, 0, oz) || !nb.ok(ox, 0, 0) || !nb.ok(0, oy, 0)) return 0;
    const int t = g.zface[oz < 0 ? 0 : 1];
    return t >= FACE_INFLOW ? t : 0;
  }
}

// deviation of direction q pulled across an open face, from the bounced-back
// deviation bb: an inflow adds 6 w_q c_q.U_b (bounce-back of a moving wall);
// an outflow reverses it and adds 2 w_q (rho_b - 1 + 9/2 (c_q.u_b)^2 -
// 3/2 u_b.u_b) (anti-bounce-back), u_b the cell's own velocity after the last
// collision
template <typename T>
__device__ __forceinline__ T open_value(const OpenBC& bc, int type, int q, T bb, const T* ub) {
  if (type == FACE_INFLOW) return bb + from_double<T>(bc.in[q]);
  const int k = (q - 1) >> 1;
  const T cu = cdot<T>(k, ub[0], ub[1], ub[2]);
  const T uu = (ub[0] * ub[0] + ub[1] * ub[1]) + ub[2] * ub[2];
  const T e = (from_double<T>(bc.rho1) + from_double<T>(4.5) * (cu * cu)) -
              from_double<T>(1.5) * uu;
  return from_double<T>(2.0 * wq(q)) * e - bb;
}

// the cell's own velocity after the last collision, sum_q delta~_q c_q, from
// the source buffer of pull streaming
template <typename T>
__device__ __forceinline__ void own_velocity(const LbmParams& P, int cell, T* ub) {
  T a[9];
#pragma unroll
  for (int k = 0; k < 9; ++k)
    a[k] = ld(static_cast<const T*>(P.srcq[2 * k + 1]) + cell) -
           ld(static_cast<const T*>(P.srcq[2 * k + 2]) + cell);
  ub[0] = ((a[0] + a[3]) + (a[4] + a[5])) + a[6];
  ub[1] = ((a[1] + a[3]) - (a[4] - a[7])) + a[8];
  ub[2] = ((a[2] + a[5]) - (a[6] - a[7])) - a[8];
}

// whether the layer z of a pull step needs its cells' own velocity (an
// outflow face on its side)
__device__ __forceinline__ bool outflow_layer(const Grid& g, int z) {
  return (z == 0 && g.zface[0] == FACE_OUTFLOW) || (z == g.nz - 1 && g.zface[1] == FACE_OUTFLOW);
}

// pull streaming across open z faces: the links of a cell in the first or
// last layer that leave through an open face take the face's value, from the
// bounced-back deviation the pull loaded for them (d[q] of a link whose
// source is outside the grid).  Applied after all loads of the cell, so that
// the loads of every other cell stay unconditional selects.
template <typename T, int WALLS>
__device__ __forceinline__ void apply_open_faces(const LbmParams& P, const NbrT<WALLS>& nb, int z,
                                                 int cell, T* d) {
  if constexpr ((WALLS & 4) != 0) {
    const Grid& g = P.g;
    if (!((z == 0 && g.zface[0] >= FACE_INFLOW) || (z == g.nz - 1 && g.zface[1] >= FACE_INFLOW)))
      return;
    T ub[3] = {T(0), T(0), T(0)};
    if (outflow_layer(g, z)) own_velocity<T>(P, cell, ub);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int cx = ckx(k), cy = cky(k), cz = ckz(k);
      if (cz == 0) continue;
      const int qa = 2 * k + 1, qb = 2 * k + 2;
      if (!nb.ok(-cx, -cy, -cz)) {
        const int t = open_face<WALLS>(g, nb, -cx, -cy, -cz);
        if (t) d[qa] = open_value<T>(P.bc, t, qa, d[qa], ub);
      }
      if (!nb.ok(cx, cy, cz)) {
        const int t = open_face<WALLS>(g, nb, cx, cy, cz);
        if (t) d[qb] = open_value<T>(P.bc, t, qb, d[qb], ub);
      }
    }
  }
}

// store of the collided PDFs (pull: own cell of the other buffer; AA even:
// swapped slots of the own cell; AA odd: the neighbours' slots, or the own
// cell's opposite slot across a wall)
template <typename T, int MODE, int WALLS>
__device__ __forceinline__ void store_pdfs(const LbmParams& P, const NbrT<WALLS>& nb, int cell,
                                           const T* d) {
#define DST(q) static_cast<T*>(P.dstq[q])
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
#undef DST
}

// components of c_q in the canonical ordering (q = 2k+1: +c_k, q = 2k+2: -c_k)
__device__ __forceinline__ int qsign(int q) { return (q & 1) ? 1 : -1; }

__device__ __forceinline__ void prefetch_l2(const void* p, unsigned bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}

// L2 prefetch for the one-cell-per-thread kernel: lane q < 19 of the first
// warp requests the span of source array q that block `bn` will read, the
// block's 256 consecutive (padded) cells shifted by the streaming offset of
// that array (pull: back by c_q; AA even: none; AA odd: forward by c_q, the
// neighbours' swapped slots), widened to 16-byte boundaries and kept inside
// the array.  Spans across a periodic face point at the neighbouring row
// instead of the wrapped one: those few are only not prefetched.
template <typename T, int MODE>
__device__ __forceinline__ void prefetch_span(const LbmParams& P, unsigned bn, int q) {
  const Grid& g = P.g;
  long long off = 0;
  if (q > 0 && MODE != 1) {
    const int k = (q - 1) >> 1, sg = MODE == 0 ? qsign(q) : -qsign(q);
    off = sg * ((long long)ckx(k) + (long long)cky(k) * g.nxp +
                (long long)ckz(k) * g.nxp * g.ny);
  }
  constexpr long long per16 = 16 / sizeof(T);
  long long c0 = (long long)bn * LBM_THREADS - off;
  long long c1 = c0 + LBM_THREADS;
  c0 = c0 < 0 ? 0 : c0 & ~(per16 - 1);
  c1 = (c1 + per16 - 1) & ~(per16 - 1);
  if (c1 > g.ncell) c1 = g.ncell & ~(per16 - 1);
  if (c1 <= c0) return;
  prefetch_l2(static_cast<const T*>(P.srcq[q]) + c0, (unsigned)((c1 - c0) * sizeof(T)));
}

// FP32 kernels are bandwidth bound and want resident warps (4 blocks per
// SM); FP64 kernels are FP64-pipe bound and keep their registers
template <typename T, int MODE, int WALLS>
__global__ void __launch_bounds__(LBM_THREADS, kFP64<T> ? 1 : (sizeof(T) == 4 ? 4 : 2))
    lbm_kernel(LbmParams P) {
  extern __shared__ __align__(16) unsigned char lbm_smem[];
  const Grid& g = P.g;
  if constexpr (sizeof(T) == 4) {
    if (P.pf_ahead > 0 && threadIdx.x < Q && blockIdx.x + (unsigned)P.pf_ahead < gridDim.x)
      prefetch_span<T, MODE>(P, blockIdx.x + (unsigned)P.pf_ahead, (int)threadIdx.x);
  }
  // the grid has fewer than 2^31 cells: 32-bit indices throughout
  const unsigned warp = blockIdx.x * (LBM_THREADS / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (warp >= (unsigned)g.nwords) return;  // whole warps only
  const unsigned row = g.div_wpr.div(warp);
  const int xr = (int)(warp - row * (unsigned)g.wpr) * 32 + lane;
  const bool live = xr < g.nx;   // padding lanes compute on a copy of a real cell
  const int x = live ? xr : g.nx - 1;
  const int z = (int)g.div_ny.div(row);
  const int y = (int)row - z * g.ny;

  // coverage word and first slot: loaded ahead of the PDFs, the slot loads
  // of the collision depend on them
  const uint32_t m = P.mask ? __ldg(&P.mask[warp]) : 0u;
  const int eb = P.mask ? __ldg(&P.base[warp]) : 0;

  NbrT<WALLS> nb;
  nb.init(x, y, z, g.nx, g.ny, g.nz, g.nxp, g.wall);
  const int cell = nb.idx(0, 0, 0);
  // per-direction base pointers live in the kernel parameters: one address
  // computation per access.  For the AA pattern source and destination are
  // the same array: every thread reads its whole set of locations before it
  // writes the same set.
#define SRC(q) static_cast<const T*>(P.srcq[q])
  // ---- streaming (Eq. 2 read backwards; halfway bounce-back at walls, the
  // open faces' values across open z faces)
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

  if constexpr (MODE == 0) apply_open_faces<T, WALLS>(P, nb, z, cell, d);
#undef SRC
  psm_collide<T, false>(P, warp, lane, live, d,
                        reinterpret_cast<SolidSmem<T>*>(lbm_smem) + (threadIdx.x >> 5), m, eb,
                        nullptr);
  if (live) store_pdfs<T, MODE, WALLS>(P, nb, cell, d);
}

// ---- staged variant.  Whole x-rows are copied into shared memory by bulk
// copies (cp.async.bulk) that complete on mbarriers, in a ring of `stages`
// tiles per block; a tile is tile_rows consecutive x-rows.  One producer warp
// issues, per tile, the copy of each direction's source row (the row at
// (y, z) - c_q; the own row in the even AA step); eight consumer warps take
// the x-shift of a direction as an index offset within the staged row,
// collide, and store to global memory.  Links across a wall read the own
// cell from global memory.  The memory system thus sees the next tiles'
// loads while the current one is computed, independent of warp scheduling.
// Every wait is bounded (1 s); a wait that gives up sets ST_TIMEOUT, and the
// producer waits for its copies in flight before the block exits.
constexpr int BULK_CONSUMER_WARPS = 8;
constexpr int BULK_THREADS = 32 * (BULK_CONSUMER_WARPS + 1);
constexpr int BULK_MAX_STAGES = 8;
constexpr int BULK_BAR_BYTES = 16 * BULK_MAX_STAGES;  // full[] and empty[] barriers
constexpr unsigned long long kWaitLimitNs = 1000000000ull;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait until the phase with the given parity has completed, at most limit_ns
__device__ __noinline__ bool mbar_wait(unsigned long long* bar, unsigned parity,
                                       unsigned long long limit_ns = kWaitLimitNs) {
  if (mbar_test(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (mbar_test(bar, parity)) return true;
    if (global_ns() - t0 > limit_ns) return false;
  }
}

// diagnostic: the staged kernel's bounded wait on an mbarrier that nothing
// arrives on gives up after limit_ns and raises ST_TIMEOUT
__global__ void wait_selftest_kernel(unsigned* status, unsigned long long limit_ns) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (threadIdx.x == 0 && !mbar_wait(&bar, 0u, limit_ns)) atomicOr(status, ST_TIMEOUT);
}
__device__ __forceinline__ void bulk_copy_g2s(void* dst, const void* src, unsigned bytes,
                                              unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

template <typename T, int MODE, int WALLS>
__global__ void __launch_bounds__(BULK_THREADS, sizeof(T) == 4 ? 2 : 1)
    lbm_bulk_kernel(LbmParams P) {
  extern __shared__ __align__(128) unsigned char bulk_smem[];
  const Grid& g = P.g;
  unsigned long long* full = reinterpret_cast<unsigned long long*>(bulk_smem);
  unsigned long long* empty = full + BULK_MAX_STAGES;
  const int S = P.stages, TR = P.tile_rows, nxp = g.nxp;
  const int C = TR * nxp;  // elements per direction in a tile
  const size_t stage_elems = (size_t)Q * C;
  T* ring = reinterpret_cast<T*>(bulk_smem + BULK_BAR_BYTES);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nrows = g.ny * g.nz;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], BULK_CONSUMER_WARPS);
    }
    mbar_fence_init();
  }
  __syncthreads();

  if (warp == BULK_CONSUMER_WARPS) {
    // ---- producer
    int issued = 0;
    for (int tile = blockIdx.x; tile < P.ntiles; tile += gridDim.x) {
      const int s = issued % S;
      const unsigned ph = (unsigned)(issued / S) & 1u;
      if (issued >= S && !mbar_wait(&empty[s], ph ^ 1u)) {
        if (lane == 0) atomicOr(P.status, ST_TIMEOUT);
        break;
      }
      const int row0 = tile * TR;
      const int nr = min(TR, nrows - row0);
      if (lane == 0) mbar_expect_tx(&full[s], (unsigned)(Q * nr * nxp * sizeof(T)));
      __syncwarp();
      T* st = ring + s * stage_elems;
      for (int j = lane; j < Q * nr; j += 32) {
        const int q = j / nr, r = j - q * nr;
        const int row = row0 + r;
        const int z = (int)g.div_ny.div((unsigned)row);
        const int y = row - z * g.ny;
        int sy = y, sz = z, sq = q;
        if (MODE != 1 && q > 0) {
          const int k = (q - 1) >> 1, sg = qsign(q);
          sy -= sg * cky(k);
          sz -= sg * ckz(k);
          sy = sy < 0 ? sy + g.ny : (sy >= g.ny ? sy - g.ny : sy);
          sz = sz < 0 ? sz + g.nz : (sz >= g.nz ? sz - g.nz : sz);
          if (MODE == 2) sq = q + sg;  // AA odd: the opposite direction's array
        }
        const T* src = static_cast<const T*>(P.src) + (size_t)sq * g.ncell +
                       ((size_t)sz * g.ny + sy) * nxp;
        bulk_copy_g2s(st + ((size_t)q * TR + r) * nxp, src, (unsigned)(nxp * sizeof(T)),
                      &full[s]);
      }
      ++issued;
    }
    // no copy may land after the block has exited
    for (int j = issued - S < 0 ? 0 : issued - S; j < issued; ++j)
      if (!mbar_wait(&full[j % S], (unsigned)(j / S) & 1u)) {
        if (lane == 0) atomicOr(P.status, ST_TIMEOUT);
      }
    return;
  }

  // ---- consumers
  SolidSmem<T>* solid = reinterpret_cast<SolidSmem<T>*>(
                            bulk_smem + BULK_BAR_BYTES + S * stage_elems * sizeof(T)) + warp;
#define SRC(q) static_cast<const T*>(P.srcq[q])
  // FP32: the coverage word and first slot of a word are loaded one word
  // ahead (the slot records of the collision depend on them): the word a
  // warp takes next is w + 8 in the same tile, else its first word in the
  // block's next tile.  Word index of (tile, w): tile * TR * wpr + w.  FP64
  // loads them at the word.
  constexpr bool ahead = !kFP64<T>;
  const int tile_words = TR * g.wpr;
  auto words_in = [&](int t) { return min(TR, nrows - t * TR) * g.wpr; };
  uint32_t m_next = 0u;
  int eb_next = 0;
  if (ahead && P.mask && blockIdx.x < P.ntiles && warp < words_in(blockIdx.x)) {
    const unsigned w0 = (unsigned)(blockIdx.x * tile_words + warp);
    m_next = __ldg(&P.mask[w0]);
    eb_next = __ldg(&P.base[w0]);
  }
  int it = 0;
  for (int tile = blockIdx.x; tile < P.ntiles; tile += gridDim.x, ++it) {
    const int s = it % S;
    if (!mbar_wait(&full[s], (unsigned)(it / S) & 1u)) {
      if (lane == 0) atomicOr(P.status, ST_TIMEOUT);
      break;
    }
    const T* st = ring + s * stage_elems;
    const int row0 = tile * TR;
    const int nw = words_in(tile);  // coverage words of the tile
    for (int w = warp; w < nw; w += BULK_CONSUMER_WARPS) {
      const int r = (int)g.div_wpr.div((unsigned)w);
      const int wr = w - r * g.wpr;
      const int xr = wr * 32 + lane;
      const bool live = xr < g.nx;  // padding lanes compute on a copy of a real cell
      const int x = live ? xr : g.nx - 1;
      const int row = row0 + r;
      const unsigned word = (unsigned)(row * g.wpr + wr);
      const uint32_t m = ahead ? m_next : (P.mask ? __ldg(&P.mask[word]) : 0u);
      const int eb = ahead ? eb_next : (P.mask ? __ldg(&P.base[word]) : 0);
      // FP32: the record loads go out before the PDF reads; FP64 (bound by
      // its pipe, registers tight) reads them in the collision
      SlotRec<T> R;
      if constexpr (ahead) load_slot_rec<T>(P, m, eb, lane, live, R);
      if (ahead && P.mask) {
        int t2 = tile, w2 = w + BULK_CONSUMER_WARPS;
        if (w2 >= nw) {
          t2 = tile + gridDim.x;
          w2 = warp;
        }
        if (t2 < P.ntiles && w2 < words_in(t2)) {
          const unsigned wn = (unsigned)(t2 * tile_words + w2);
          m_next = __ldg(&P.mask[wn]);
          eb_next = __ldg(&P.base[wn]);
        }
      }
      const int z = (int)g.div_ny.div((unsigned)row);
      const int y = row - z * g.ny;
      NbrT<WALLS> nb;
      nb.init(x, y, z, g.nx, g.ny, g.nz, g.nxp, g.wall);
      const int cell = nb.idx(0, 0, 0);
      const int xm = x == 0 ? g.nx - 1 : x - 1, xq = x == g.nx - 1 ? 0 : x + 1;
      const T* sr = st + (size_t)r * nxp;  // direction q of this row at sr[q * C]
      T d[Q];
      d[0] = sr[x];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const int cx = ckx(k), cy = cky(k), cz = ckz(k);
        const int qa = 2 * k + 1, qb = 2 * k + 2;
        const int xa = cx > 0 ? xm : (cx < 0 ? xq : x);  // x - c_x
        const int xb = cx > 0 ? xq : (cx < 0 ? xm : x);  // x + c_x
        if (MODE == 0) {
          d[qa] = nb.ok(-cx, -cy, -cz) ? sr[qa * C + xa] : ld(SRC(qb) + cell);
          d[qb] = nb.ok(cx, cy, cz) ? sr[qb * C + xb] : ld(SRC(qa) + cell);
        } else if (MODE == 1) {
          d[qa] = sr[qa * C + x];
          d[qb] = sr[qb * C + x];
        } else {
          d[qa] = nb.ok(-cx, -cy, -cz) ? sr[qa * C + xa] : ld(SRC(qa) + cell);
          d[qb] = nb.ok(cx, cy, cz) ? sr[qb * C + xb] : ld(SRC(qb) + cell);
        }
      }
      if constexpr (MODE == 0) apply_open_faces<T, WALLS>(P, nb, z, cell, d);
      psm_collide<T, ahead>(P, word, lane, live, d, solid, m, eb, &R);
      if (live) store_pdfs<T, MODE, WALLS>(P, nb, cell, d);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
#undef SRC
}

// ---- FP64 collision on compacted warps.  FP64 runs at 1/64 of the FP32
// rate on GB300, so the FP64 kernel is bound by its count of FP64
// instructions.  Two things cost instructions on warps of 32 consecutive
// cells: a warp with a covered cell weights every lane's fluid change by
// (1 - B), and the solid operator of a few covered lanes keeps the whole warp
// busy.  So each tile's cells are listed in three groups (uncovered cells,
// covered cells, covered cells of one particle with B = 1) and warps take 32
// list entries at a time: a warp of uncovered cells runs the particle-free
// form, a warp of full cells the solid operator alone, any other warp every
// lane's own fluid change and solid operators; at most two warps per tile
// are mixed.
enum { CK_UNCOVERED = 0, CK_MIXED = 1, CK_FULL = 2 };

// the step's FP64 collision coefficients sit in shared memory (copied once
// per block): the same four values for every lane, read as two 16-byte
// broadcasts, which keeps them off the L1/texture path of the slot records
constexpr int F64_COEF_BYTES = 512;
static_assert(sizeof(CollideCoef<double>) <= F64_COEF_BYTES, "coefficient area");
__device__ __forceinline__ void lds4(const double* p, double* o) {
  const double2 u = reinterpret_cast<const double2*>(p)[0];
  const double2 v = reinterpret_cast<const double2*>(p)[1];
  o[0] = u.x; o[1] = u.y; o[2] = v.x; o[3] = v.y;
}

// FP64 collision of one cell (Eqs. 3-8 and 17-21).
// CK_UNCOVERED: all lanes of the warp are uncovered (B = 0); a pair's update
// is written as d_q' = S_k + A_k, d_qbar' = S_k - A_k with
// S_k = (1 - omega+)/2 s_k + X_k, A_k = (1 - omega-)/2 a_k + Y_k,
// X_k = (9/2 omega+ w c.U + G_k) c.U + C_c, Y_k = 3 omega- w c.U + F_k: seven
// FP64 operations per pair instead of nine.
// CK_FULL: every lane is a covered cell of one particle with B = 1; the fluid
// change vanishes and the solid operator (Eq. 19) swaps the pair and adds the
// difference of the equilibria: d_q' = d_qbar + (BdS + 3 w (cu + cv)),
// d_qbar' = d_q + (BdS - 3 w (cu + cv)), BdS = w (9/2 (cv^2 - cu^2) -
// 3/2 (V^2 - U^2)).
// CK_MIXED: a covered lane (cov, slot index e) reads its slot records,
// weights the fluid change by 1 - B and adds the solid operator of each of
// its slots (Eq. 19); an uncovered lane has B = 0.
// Covered lanes write their slots' forces (Eq. 21).

template <int KIND>
__device__ __forceinline__ void fp64_collide(const LbmParams& P, const CollideCoef<double>* cf,
                                             double* d, bool cov, int e) {
  using T = double;
  T a[9], sk[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    sk[k] = d[2 * k + 1] + d[2 * k + 2];
    a[k] = d[2 * k + 1] - d[2 * k + 2];
  }
  const T drho = ((d[0] + (sk[0] + sk[1])) + ((sk[2] + sk[3]) + (sk[4] + sk[5]))) +
                 ((sk[6] + sk[7]) + sk[8]);
  const T jx = ((a[0] + a[3]) + (a[4] + a[5])) + a[6];
  const T jy = ((a[1] + a[3]) - (a[4] - a[7])) + a[8];
  const T jz = ((a[2] + a[5]) - (a[6] - a[7])) - a[8];
  T h[16];
  lds4(cf->head, h);
  lds4(cf->head + 4, h + 4);
  lds4(cf->head + 8, h + 8);
  lds4(cf->head + 12, h + 12);
  const T Ux = jx + h[CC_HF];
  const T Uy = jy + h[CC_HF + 1];
  const T Uz = jz + h[CC_HF + 2];
  const T uu = Ux * Ux + Uy * Uy + Uz * Uz;
  const T Uf = Ux * h[CC_F] + Uy * h[CC_F + 1] + Uz * h[CC_F + 2];
  const T base0 = drho - T(1.5) * uu;
  const T C0 = h[CC_WPW] * base0 + h[CC_H + 1] * Uf;
  const T C1 = h[CC_WPW + 1] * base0 + h[CC_H + 2] * Uf;

  if constexpr (KIND == CK_UNCOVERED) {
    T tl[4];
    lds4(cf->tail, tl);
    d[0] = fma(tl[0], d[0], h[CC_WPW0] * base0 + h[CC_H] * Uf);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      T pk[4];
      lds4(cf->pair[k], pk);
      const T cu = cdot<T>(k, Ux, Uy, Uz);
      const T X = (pk[2] * cu + pk[0]) * cu + (k < 3 ? C0 : C1);
      const T Y = pk[3] * cu + pk[1];
      const T Sk = tl[1] * sk[k] + X;
      const T Ak = tl[2] * a[k] + Y;
      d[2 * k + 1] = Sk + Ak;
      d[2 * k + 2] = Sk - Ak;
    }
  } else if constexpr (KIND == CK_FULL) {
    T r0[4] = {T(0), T(0), T(0), T(0)};
    if (cov) ld4(static_cast<const T*>(P.slot_V) + 4LL * e, r0);
    const T Vx = r0[0], Vy = r0[1], Vz = r0[2];
    const T dU2 = (Vx * Vx + Vy * Vy + Vz * Vz) - uu;
    d[0] += (T(-1.5) * w0<T>()) * dU2;
    const T cd[2] = {(T(-1.5) * wk<T>(0)) * dU2, (T(-1.5) * wk<T>(3)) * dU2};
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const int cl = k < 3 ? 0 : 1;
      const T cu = cdot<T>(k, Ux, Uy, Uz);
      const T cv = cdot<T>(k, Vx, Vy, Vz);
      const T Sv = cv + cu;
      const T BdS = (T(4.5) * wk<T>(cl == 0 ? 0 : 3)) * ((cv - cu) * Sv) + cd[cl];
      const T t = (T(3) * wk<T>(cl == 0 ? 0 : 3)) * Sv;
      const T dq = d[2 * k + 1];
      d[2 * k + 1] = d[2 * k + 2] + (BdS + t);
      d[2 * k + 2] = dq + (BdS - t);
    }
    if (cov) slot_force<T>(P, e, 0, T(1), Ux - Vx, Uy - Vy, Uz - Vz, h + CC_F);
  } else {
    // the cell's slots; the second one's record is read only when present
    T r0[4] = {T(0), T(0), T(0), T(0)}, r1[4] = {T(0), T(0), T(0), T(0)};
    bool has1 = false;
    T omB = T(1);
    if (cov) {
      ld4(static_cast<const T*>(P.slot_V) + 4LL * e, r0);
      has1 = neg_flag(r0[3]);
      r0[3] = magnitude(r0[3]);
      if (has1) ld4(static_cast<const T*>(P.slot_V) + 4LL * (P.slot_cap + e), r1);
      T B = r0[3] + r1[3];
      if (B > T(1)) B = T(1);
      omB = T(1) - B;
    }
    // slot 0 (zero weight on an uncovered lane) joins the fluid update of each
    // pair: with the fluid change omB (ds +- da) and the solid operator's
    // symmetric part BdS = B_0 w (9/2 (cv^2 - cu^2) - 3/2 dU2) and
    // antisymmetric part B_0 (3 w (cu + cv) - a_k), the pair becomes
    // d_q' = SYM + ANT, d_qbar' = SYM - ANT with
    // SYM = (1/2 + omB hp) s_k + (omB X_k + BdS) and
    // ANT = (1/2 + omB hm - B_0) a_k + (omB Y_k + 3 w B_0 (cu + cv))
    const T Vx = r0[0], Vy = r0[1], Vz = r0[2], B0 = r0[3];
    const T dU2 = (Vx * Vx + Vy * Vy + Vz * Vz) - uu;
    const T BdU = B0 * dU2;
    {
      const T dl = h[CC_NWP] * d[0] + (h[CC_WPW0] * base0 + h[CC_H] * Uf);
      d[0] = (d[0] + omB * dl) + (T(-1.5) * w0<T>()) * BdU;
    }
    const T c45[2] = {(T(4.5) * wk<T>(0)) * B0, (T(4.5) * wk<T>(3)) * B0};
    const T c3[2] = {(T(3) * wk<T>(0)) * B0, (T(3) * wk<T>(3)) * B0};
    const T cd[2] = {(T(-1.5) * wk<T>(0)) * BdU, (T(-1.5) * wk<T>(3)) * BdU};
    const T as = omB * h[CC_MHWP] + T(0.5);
    const T aa = omB * h[CC_MHWM] + (T(0.5) - B0);
    // per class, with X_k = (9/2 omega+ w c.U + G_k) c.U + C_c and
    // Y_k = 3 omega- w c.U + F_k: SYM = as s_k + ((al cu + omB G_k) cu + ga
    // + c45 cv^2) with al = omB 9/2 omega+ w - c45, ga = omB C_c + cd, and
    // ANT = aa a_k + (de cu + (c3 cv + omB F_k)) with de = omB 3 omega- w + c3
    T al[2], ga[2], de[2];
#pragma unroll
    for (int cl = 0; cl < 2; ++cl) {
      T pc[4];
      lds4(cf->pair[cl == 0 ? 0 : 3], pc);
      al[cl] = omB * pc[2] - c45[cl];
      ga[cl] = omB * (cl == 0 ? C0 : C1) + cd[cl];
      de[cl] = omB * pc[3] + c3[cl];
    }
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      T pk[4];
      lds4(cf->pair[k], pk);
      const int cl = k < 3 ? 0 : 1;
      const T cu = cdot<T>(k, Ux, Uy, Uz);
      const T cv = cdot<T>(k, Vx, Vy, Vz);
      const T sy = (al[cl] * cu + omB * pk[0]) * cu + ga[cl];
      const T SYM = as * sk[k] + ((c45[cl] * cv) * cv + sy);
      const T ANT = aa * a[k] + (de[cl] * cu + (c3[cl] * cv + omB * pk[1]));
      d[2 * k + 1] = SYM + ANT;
      d[2 * k + 2] = SYM - ANT;
    }
    if (cov) slot_force<T>(P, e, 0, B0, Ux - Vx, Uy - Vy, Uz - Vz, h + CC_F);
    // slot 1 (a cell shared by two particles: rare), on its own
    if (__any_sync(0xffffffffu, has1) && has1) {
      const T Wx = r1[0], Wy = r1[1], Wz = r1[2], B1 = r1[3];
      const T eU2 = (Wx * Wx + Wy * Wy + Wz * Wz) - uu;
      const T BeU = B1 * eU2;
      d[0] += (T(-1.5) * w0<T>()) * BeU;
      const T e45[2] = {(T(4.5) * wk<T>(0)) * B1, (T(4.5) * wk<T>(3)) * B1};
      const T e3[2] = {(T(3) * wk<T>(0)) * B1, (T(3) * wk<T>(3)) * B1};
      const T ed[2] = {(T(-1.5) * wk<T>(0)) * BeU, (T(-1.5) * wk<T>(3)) * BeU};
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const int cl = k < 3 ? 0 : 1;
        const T cu = cdot<T>(k, Ux, Uy, Uz);
        const T cv = cdot<T>(k, Wx, Wy, Wz);
        const T Sv = cv + cu;
        const T BdS = e45[cl] * ((cv - cu) * Sv) + ed[cl];
        const T BA = e3[cl] * Sv - B1 * a[k];
        d[2 * k + 1] += BdS + BA;
        d[2 * k + 2] += BdS - BA;
      }
      slot_force<T>(P, e, 1, B1, Ux - Wx, Uy - Wy, Uz - Wz, h + CC_F);
    }
  }
}

// The producer warp lists the cells of a tile into the tile's stage: the
// live cells' positions (r << 16 | x) in three groups, each in cell order:
// uncovered cells, covered cells, and covered cells of one particle with
// B = 1 (the full mask), with each covered cell's slot index (-1 for an
// uncovered cell); hdr[0] = number of uncovered cells, hdr[1] = number of
// live cells, hdr[2] = index of the first cell of the third group.  Two
// warp-wide passes over the tile's coverage words (the group sizes, then the
// entries); the lanes load the words 32 at a time and the rounds take them by
// shuffles.
__device__ __forceinline__ void fp64_list_tile(const LbmParams& P, int tile, int nw,
                                               int* lst_cell, int* lst_slot, int* hdr,
                                               int lane) {
  const Grid& g = P.g;
  const size_t word0 = (size_t)tile * P.tile_rows * g.wpr;
  const unsigned below = (1u << lane) - 1u;
  int pu = 0, pc = 0, pf = 0, tot_u = 0, tot_c = 0;
  // two passes over the words (counts, then entries), 32 words at a time:
  // lane k loads word w0 + k and the rounds take them by shuffles, so each
  // round issues its loads together
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      pc = tot_u;  // the covered cells follow all uncovered ones
      pf = tot_u + tot_c;  // and the full ones follow them
      pu = 0;
    }
    for (int w0 = 0; w0 < nw; w0 += 32) {
      const int kmax = min(32, nw - w0);
      const bool own = P.mask && lane < kmax;
      const uint32_t m_l = own ? __ldg(&P.mask[word0 + w0 + lane]) : 0u;
      const uint32_t f_l = (own && P.full) ? __ldg(&P.full[word0 + w0 + lane]) : 0u;
      const int b_l = (own && pass == 1) ? __ldg(&P.base[word0 + w0 + lane]) : 0;
      for (int k = 0; k < kmax; ++k) {
        const int w = w0 + k;
        const int r = (int)g.div_wpr.div((unsigned)w);
        const int xr = (w - r * g.wpr) * 32 + lane;
        const bool live = xr < g.nx;
        const uint32_t m = __shfl_sync(0xffffffffu, m_l, k);
        const uint32_t fm = __shfl_sync(0xffffffffu, f_l, k) & m;
        const bool cv = live && ((m >> lane) & 1u);
        const bool fl = live && ((fm >> lane) & 1u);
        const unsigned bu = __ballot_sync(0xffffffffu, live && !cv);
        const unsigned bc = __ballot_sync(0xffffffffu, cv && !fl);
        const unsigned bf = __ballot_sync(0xffffffffu, fl);
        if (pass == 0) {
          pu += __popc(bu);
          pc += __popc(bc);
          continue;
        }
        const int base = __shfl_sync(0xffffffffu, b_l, k);
        if (live) {
          const int pos = fl   ? pf + __popc(bf & below)
                          : cv ? pc + __popc(bc & below)
                               : pu + __popc(bu & below);
          lst_cell[pos] = (r << 16) | xr;
          int e = -1;
          if (cv) {
            e = base + __popc(m & below);
            if (e >= P.slot_cap) e = -1;  // never the case: the mapping sized the slots
          }
          lst_slot[pos] = e;
        }
        pu += __popc(bu);
        pc += __popc(bc);
        pf += __popc(bf);
      }
    }
    if (pass == 0) {
      tot_u = pu;
      tot_c = pc;
    }
  }
  if (lane == 0) {
    hdr[0] = tot_u;
    hdr[1] = pf;  // after the second pass: every live cell
    hdr[2] = tot_u + tot_c;
  }
}

// Staged FP64 kernel with compacted warps: the producer warp and the ring of
// staged rows are those of lbm_bulk_kernel, and the producer also lists each
// tile's cells into the tile's stage (fp64_list_tile) before it arrives on
// the stage's full barrier (count 2: its expect-tx arrival and this one), so
// the consumers find the list with the data.  Consumer warps take 32 list
// entries at a time and need no barrier among themselves.
template <int MODE, int WALLS>
__global__ void __launch_bounds__(BULK_THREADS, 1) lbm_fp64_kernel(LbmParams P) {
  using T = double;
  extern __shared__ __align__(128) unsigned char bulk_smem[];
  const Grid& g = P.g;
  unsigned long long* full = reinterpret_cast<unsigned long long*>(bulk_smem);
  unsigned long long* empty = full + BULK_MAX_STAGES;
  const int S = P.stages, TR = P.tile_rows, nxp = g.nxp;
  const int C = TR * nxp;  // elements per direction in a tile
  const size_t stage_elems = (size_t)Q * C;
  // the barriers, the step's collision coefficients, the ring
  CollideCoef<double>* coef = reinterpret_cast<CollideCoef<double>*>(bulk_smem + BULK_BAR_BYTES);
  T* ring = reinterpret_cast<T*>(bulk_smem + BULK_BAR_BYTES + F64_COEF_BYTES);
  // per stage: header (2 ints, padded to 4), cells, slot indices
  int* lists = reinterpret_cast<int*>(ring + S * stage_elems);
  const size_t list_ints = 4 + 2 * (size_t)C;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nrows = g.ny * g.nz;
  {
    constexpr int NV = (int)(sizeof(CollideCoef<double>) / sizeof(double2));
    const double2* src = reinterpret_cast<const double2*>(&P.sc->d);
    for (int i = threadIdx.x; i < NV; i += blockDim.x) reinterpret_cast<double2*>(coef)[i] = src[i];
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 2);
      mbar_init(&empty[s], BULK_CONSUMER_WARPS);
    }
    mbar_fence_init();
  }
  __syncthreads();

  if (warp == BULK_CONSUMER_WARPS) {
    // ---- producer
    int issued = 0;
    for (int tile = blockIdx.x; tile < P.ntiles; tile += gridDim.x) {
      const int s = issued % S;
      const unsigned ph = (unsigned)(issued / S) & 1u;
      if (issued >= S && !mbar_wait(&empty[s], ph ^ 1u)) {
        if (lane == 0) atomicOr(P.status, ST_TIMEOUT);
        break;
      }
      const int row0 = tile * TR;
      const int nr = min(TR, nrows - row0);
      if (lane == 0) mbar_expect_tx(&full[s], (unsigned)(Q * nr * nxp * sizeof(T)));
      __syncwarp();
      T* st = ring + s * stage_elems;
      for (int j = lane; j < Q * nr; j += 32) {
        const int q = j / nr, r = j - q * nr;
        const int row = row0 + r;
        const int z = (int)g.div_ny.div((unsigned)row);
        const int y = row - z * g.ny;
        int sy = y, sz = z, sq = q;
        if (MODE != 1 && q > 0) {
          const int k = (q - 1) >> 1, sg = qsign(q);
          sy -= sg * cky(k);
          sz -= sg * ckz(k);
          sy = sy < 0 ? sy + g.ny : (sy >= g.ny ? sy - g.ny : sy);
          sz = sz < 0 ? sz + g.nz : (sz >= g.nz ? sz - g.nz : sz);
          if (MODE == 2) sq = q + sg;  // AA odd: the opposite direction's array
        }
        const T* src = static_cast<const T*>(P.src) + (size_t)sq * g.ncell +
                       ((size_t)sz * g.ny + sy) * nxp;
        bulk_copy_g2s(st + ((size_t)q * TR + r) * nxp, src, (unsigned)(nxp * sizeof(T)),
                      &full[s]);
      }
      int* ls = lists + s * list_ints;
      fp64_list_tile(P, tile, nr * g.wpr, ls + 4, ls + 4 + C, ls, lane);
      __threadfence_block();
      __syncwarp();
      if (lane == 0) mbar_arrive(&full[s]);  // release: the list is visible with the data
      ++issued;
    }
    // no copy may land after the block has exited
    for (int j = issued - S < 0 ? 0 : issued - S; j < issued; ++j)
      if (!mbar_wait(&full[j % S], (unsigned)(j / S) & 1u)) {
        if (lane == 0) atomicOr(P.status, ST_TIMEOUT);
      }
    return;
  }

  // ---- consumers
#define SRC(q) static_cast<const T*>(P.srcq[q])
  int it = 0;
  for (int tile = blockIdx.x; tile < P.ntiles; tile += gridDim.x, ++it) {
    const int s = it % S;
    if (!mbar_wait(&full[s], (unsigned)(it / S) & 1u)) {
      if (lane == 0) atomicOr(P.status, ST_TIMEOUT);
      break;
    }
    const T* st = ring + s * stage_elems;
    const int* ls = lists + s * list_ints;
    const int tot_u = ls[0], L = ls[1], full0 = ls[2];
    const int* lst_cell = ls + 4;
    const int* lst_slot = ls + 4 + C;
    const int row0 = tile * TR;
    const int nch = (L + 31) / 32;
    // the covered chunks come last in every tile: the chunk a warp starts
    // with turns by 3 from tile to tile (3 and 8 are coprime), so every
    // warp takes its share of them and none runs ahead of the ring
    const int ch0 = (warp + 3 * it) % BULK_CONSUMER_WARPS;
    for (int ch = ch0; ch < nch; ch += BULK_CONSUMER_WARPS) {
      const int i = ch * 32 + lane;
      const bool active = i < L;
      const int ent = lst_cell[active ? i : L - 1];
      const int e = active ? lst_slot[i] : -1;
      const int r = ent >> 16, x = ent & 0xffff;
      const int row = row0 + r;
      const int z = (int)g.div_ny.div((unsigned)row);
      const int y = row - z * g.ny;
      NbrT<WALLS> nb;
      nb.init(x, y, z, g.nx, g.ny, g.nz, g.nxp, g.wall);
      const int cell = nb.idx(0, 0, 0);
      const int xm = x == 0 ? g.nx - 1 : x - 1, xq = x == g.nx - 1 ? 0 : x + 1;
      const T* sr = st + (size_t)r * nxp;  // direction q of this row at sr[q * C]
      T d[Q];
      d[0] = sr[x];
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        const int cx = ckx(k), cy = cky(k), cz = ckz(k);
        const int qa = 2 * k + 1, qb = 2 * k + 2;
        const int xa = cx > 0 ? xm : (cx < 0 ? xq : x);  // x - c_x
        const int xb = cx > 0 ? xq : (cx < 0 ? xm : x);  // x + c_x
        if (MODE == 0) {
          d[qa] = nb.ok(-cx, -cy, -cz) ? sr[qa * C + xa] : ld(SRC(qb) + cell);
          d[qb] = nb.ok(cx, cy, cz) ? sr[qb * C + xb] : ld(SRC(qa) + cell);
        } else if (MODE == 1) {
          d[qa] = sr[qa * C + x];
          d[qb] = sr[qb * C + x];
        } else {
          d[qa] = nb.ok(-cx, -cy, -cz) ? sr[qa * C + xa] : ld(SRC(qa) + cell);
          d[qb] = nb.ok(cx, cy, cz) ? sr[qb * C + xb] : ld(SRC(qb) + cell);
        }
      }
      if constexpr (MODE == 0) apply_open_faces<T, WALLS>(P, nb, z, cell, d);
      if (ch * 32 + 32 <= tot_u) fp64_collide<CK_UNCOVERED>(P, coef, d, false, -1);
      else if (ch * 32 >= full0) fp64_collide<CK_FULL>(P, coef, d, e >= 0, e);
      else fp64_collide<CK_MIXED>(P, coef, d, e >= 0, e);
      if (active) store_pdfs<T, MODE, WALLS>(P, nb, cell, d);
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }
#undef SRC
}

// canonical FP64 f~ (unpadded, full f = w + delta) from the storage layout
template <typename T>
__global__ void to_canonical_kernel(Grid g, const T* __restrict__ buf, int aa, int parity,
                                    BoxSel B, double* __restrict__ out) {
  const long long N = (long long)B.bx * B.by * B.bz;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)((B.x0 + c % B.bx) % g.nx);
    const int y = (int)((B.y0 + (c / B.bx) % B.by) % g.ny);
    const int z = (int)((B.z0 + c / ((long long)B.bx * B.by)) % g.nz);
    Nbr nb;
    nb.init(x, y, z, g.nx, g.ny, g.nz, g.nxp, g.wall);
    const int cell = nb.idx(0, 0, 0);
    const long long NC = g.ncell;
    out[c] = wq(0) + as_double(buf[cell]);
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
      out[qa * N + c] = wq(qa) + as_double(buf[ia]);
      out[qb * N + c] = wq(qb) + as_double(buf[ib]);
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
    buf[cell] = from_double<T>(in[c] - wq(0));
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
      buf[qa * NC + cell] = from_double<T>(va - wq(qa));
      buf[qb * NC + cell] = from_double<T>(vb - wq(qb));
    }
  }
}

// rho and U of the streamed canonical field (Eqs. 6-7)
__global__ void macroscopic_kernel(Grid g, const double* __restrict__ f, const StepConst* sc,
                                   OpenBC bc, double* __restrict__ rho, double* __restrict__ u) {
  const long long N = (long long)g.nx * g.ny * g.nz;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(c % g.nx);
    const int y = (int)((c / g.nx) % g.ny);
    const int z = (int)(c / ((long long)g.nx * g.ny));
    Nbr nc;
    nc.init(x, y, z, g.nx, g.ny, g.nz, g.nx, g.wall);
    // the open faces' values, in deviations from the lattice weights
    double ub[3] = {0.0, 0.0, 0.0};
    if (outflow_layer(g, z)) {
      for (int k = 0; k < 9; ++k) {
        const double ak = f[(2 * k + 1) * N + c] - f[(2 * k + 2) * N + c];
        ub[0] += ak * ckx(k);
        ub[1] += ak * cky(k);
        ub[2] += ak * ckz(k);
      }
    }
    auto pulled = [&](int q, int qr, int ox, int oy, int oz) {
      if (nc.ok(ox, oy, oz)) return f[q * N + nc.idx(ox, oy, oz)];
      const double bb = f[qr * N + c];
      const int t = open_face<7>(g, nc, ox, oy, oz);
      return t ? wq(q) + open_value<double>(bc, t, q, bb - wq(qr), ub) : bb;
    };
    double r = f[c], jx = 0.0, jy = 0.0, jz = 0.0;
    for (int k = 0; k < 9; ++k) {
      const int cx = ckx(k), cy = cky(k), cz = ckz(k);
      const int qa = 2 * k + 1, qb = 2 * k + 2;
      const double va = pulled(qa, qb, -cx, -cy, -cz);
      const double vb = pulled(qb, qa, cx, cy, cz);
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
  return kFP64<T> ? lbm_smem_bytes<T>() : 0;
}

template <typename T, int W>
int configure_walls(int optin) {
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  const int sm = (int)lbm_dyn_smem<T>();
  int bad = 0;
  bad |= cudaFuncSetAttribute(lbm_kernel<T, 0, W>, a, sm) != cudaSuccess;
  bad |= cudaFuncSetAttribute(lbm_kernel<T, 1, W>, a, sm) != cudaSuccess;
  bad |= cudaFuncSetAttribute(lbm_kernel<T, 2, W>, a, sm) != cudaSuccess;
  if constexpr (!kFP64<T>) {  // FP64 stages through lbm_fp64_kernel
    bad |= cudaFuncSetAttribute(lbm_bulk_kernel<T, 0, W>, a, optin) != cudaSuccess;
    bad |= cudaFuncSetAttribute(lbm_bulk_kernel<T, 1, W>, a, optin) != cudaSuccess;
    bad |= cudaFuncSetAttribute(lbm_bulk_kernel<T, 2, W>, a, optin) != cudaSuccess;
  } else {
    bad |= cudaFuncSetAttribute(lbm_fp64_kernel<0, W>, a, optin) != cudaSuccess;
    bad |= cudaFuncSetAttribute(lbm_fp64_kernel<1, W>, a, optin) != cudaSuccess;
    bad |= cudaFuncSetAttribute(lbm_fp64_kernel<2, W>, a, optin) != cudaSuccess;
  }
  return bad;
}

static int smem_optin() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return 0;
  return v;
}

int lbm_configure() {
  const int o = smem_optin();
  if (o <= 0) return 1;
  return configure_walls<float, 0>(o) | configure_walls<float, 1>(o) |
         configure_walls<float, 7>(o) | configure_walls<double, 0>(o) |
         configure_walls<double, 1>(o) | configure_walls<double, 7>(o) |
         configure_walls<df, 0>(o) | configure_walls<df, 1>(o) | configure_walls<df, 7>(o);
}

// tiles of whole x-rows: 256 cells (tile_rows rows) when the padded row
// divides 256, else one row; as many stages as fit the per-block budget
// (FP32: two blocks per SM; FP64: one block next to the solid-operator
// scratch).  The staged kernel serves FP64 (FP64-pipe bound: it frees the
// warps from load latency) and the FP32 AA pattern; FP32 pull streaming runs
// faster on the one-cell-per-thread kernel, whose 32 resident warps per SM
// keep enough loads in flight.  Returns 0 and leaves plan.stages = 0 when
// the one-cell-per-thread kernel is to be used.
template <typename T, int W>
const void* bulk_fn() {
  if constexpr (kFP64<T>) return (const void*)lbm_fp64_kernel<0, W>;
  else return (const void*)lbm_bulk_kernel<T, 0, W>;
}
template <typename T>
const void* bulk_fn_w(int w) {
  return w == 0 ? bulk_fn<T, 0>() : (w == 1 ? bulk_fn<T, 1>() : bulk_fn<T, 7>());
}

template <typename T>
const void* cell_fn_w(int w) {
  if (w == 0) return reinterpret_cast<const void*>(lbm_kernel<T, 0, 0>);
  if (w == 1) return reinterpret_cast<const void*>(lbm_kernel<T, 0, 1>);
  return reinterpret_cast<const void*>(lbm_kernel<T, 0, 7>);
}

// Prefetch distance of the one-cell-per-thread kernel: half the number of
// its blocks resident at once, so the block that many places later starts
// about half a wave of the grid later.  Measured on GB300 (FP32 pull, channel
// 256x256x512 and settling box 512x512x1024): half and three quarters of a
// wave are best (87% of the measured copy bandwidth, from 75-78% without
// prefetch); a full wave loses 1-2%, two waves 10%.
template <typename T>
int cell_prefetch_ahead(const Grid& g, int* ahead) {
  const int w = g.wall[0] | (g.wall[1] << 1) | (g.wall[2] << 2);
  int per_sm = 0, dev = 0, nsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, cell_fn_w<T>(w), LBM_THREADS,
                                                    lbm_dyn_smem<T>()) != cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 1;
  *ahead = per_sm * nsm / 2;
  return 0;
}

int lbm_plan(const Grid& g, int prec, int aa, LbmPlan* plan) {
  *plan = LbmPlan{};
  const int fp32 = prec == PREC_FP32;
  if (fp32 && !aa) return cell_prefetch_ahead<float>(g, &plan->pf_ahead);
  // the double-float form is bound by the FP32 pipes: it takes the
  // one-cell-per-thread kernel (two blocks of eight warps per SM; the staged
  // kernel fits one block of nine warps next to its ring)
  // (and does not prefetch: on settle128 a prefetch half a wave ahead made
  // its collision 16% slower)
  if (prec == PREC_DF) return 0;
  const int optin = smem_optin();
  if (optin <= 0) return 1;
  const size_t esz = fp32 ? sizeof(float) : sizeof(double);
  const int TR = (g.nxp <= 256 && 256 % g.nxp == 0) ? 256 / g.nxp : 1;
  const size_t stage = (size_t)Q * TR * g.nxp * esz;
  // FP64 (compacted warps): per stage the tile's cell list and slot indices
  // with a 16-byte header
  const size_t list_stage = prec == PREC_FP64 ? (size_t)8 * TR * g.nxp + 16 : 0;
  const size_t extra = BULK_BAR_BYTES + (prec == PREC_FP64 ? F64_COEF_BYTES : 0);
  const size_t budget = prec == PREC_FP64 ? (size_t)optin : (size_t)100 * 1024;
  if (budget <= extra) return 0;
  size_t S = (budget - extra) / (stage + list_stage);
  if (S > BULK_MAX_STAGES) S = BULK_MAX_STAGES;
  if (S < 2) {
    if (extra + 2 * (stage + list_stage) > (size_t)optin) return 0;
    S = 2;
  }
  const size_t smem = extra + S * (stage + list_stage);
  const int w = g.wall[0] | (g.wall[1] << 1) | (g.wall[2] << 2);
  const void* fn = prec == PREC_FP32 ? bulk_fn_w<float>(w)
                   : prec == PREC_DF ? bulk_fn_w<df>(w)
                                     : bulk_fn_w<double>(w);
  int per_sm = 0, dev = 0, nsm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, BULK_THREADS, smem) !=
          cudaSuccess ||
      cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 1;
  if (per_sm < 1) return 0;
  const long long nrows = (long long)g.ny * g.nz;
  plan->tile_rows = TR;
  plan->ntiles = (int)((nrows + TR - 1) / TR);
  plan->stages = (int)S;
  plan->smem = smem;
  const long long blocks = (long long)nsm * per_sm;
  plan->blocks = (int)(blocks < plan->ntiles ? blocks : plan->ntiles);
  return 0;
}

template <typename T, int W>
void launch_lbm_t(const LbmParams& P, int mode, unsigned grid, cudaStream_t s) {
  if (P.stages > 0 && kFP64<T>) {
    const size_t sm = P.smem;
    if (mode == 0) lbm_fp64_kernel<0, W><<<P.blocks, BULK_THREADS, sm, s>>>(P);
    else if (mode == 1) lbm_fp64_kernel<1, W><<<P.blocks, BULK_THREADS, sm, s>>>(P);
    else lbm_fp64_kernel<2, W><<<P.blocks, BULK_THREADS, sm, s>>>(P);
    return;
  }
  if constexpr (!kFP64<T>) {
    if (P.stages > 0) {
      const size_t sm = P.smem;
      if (mode == 0) lbm_bulk_kernel<T, 0, W><<<P.blocks, BULK_THREADS, sm, s>>>(P);
      else if (mode == 1) lbm_bulk_kernel<T, 1, W><<<P.blocks, BULK_THREADS, sm, s>>>(P);
      else lbm_bulk_kernel<T, 2, W><<<P.blocks, BULK_THREADS, sm, s>>>(P);
      return;
    }
  }
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

int launch_lbm(const LbmParams& P0, int prec, int mode, cudaStream_t s) {
  LbmParams P = P0;
  const size_t esz = prec == PREC_FP32 ? sizeof(float) : sizeof(double);
  for (int q = 0; q < Q; ++q) {
    P.srcq[q] = static_cast<const char*>(P.src) + esz * (size_t)q * P.g.ncell;
    P.dstq[q] = static_cast<char*>(P.dst) + esz * (size_t)q * P.g.ncell;
  }
  const long long threads = P.g.nwords * 32;
  const unsigned grid = (unsigned)((threads + LBM_THREADS - 1) / LBM_THREADS);
  if (prec == PREC_FP32) launch_lbm_w<float>(P, mode, grid, s);
  else if (prec == PREC_DF) launch_lbm_w<df>(P, mode, grid, s);
  else launch_lbm_w<double>(P, mode, grid, s);
  return 1;
}

static unsigned grid_for(long long n, int block) {
  long long b = (n + block - 1) / block;
  if (b > 152LL * 64) b = 152LL * 64;
  return (unsigned)(b > 0 ? b : 1);
}

int launch_to_canonical(const Grid& g, const void* buf, int prec, int aa_parity, int aa,
                        const BoxSel& B, double* out, cudaStream_t s) {
  const long long N = (long long)B.bx * B.by * B.bz;
  if (prec == PREC_FP32)
    to_canonical_kernel<float><<<grid_for(N, 256), 256, 0, s>>>(
        g, static_cast<const float*>(buf), aa, aa_parity, B, out);
  else if (prec == PREC_DF)
    to_canonical_kernel<df><<<grid_for(N, 256), 256, 0, s>>>(g, static_cast<const df*>(buf), aa,
                                                              aa_parity, B, out);
  else
    to_canonical_kernel<double><<<grid_for(N, 256), 256, 0, s>>>(
        g, static_cast<const double*>(buf), aa, aa_parity, B, out);
  return 1;
}

int launch_from_canonical(const Grid& g, const double* in, void* buf, int prec, int aa,
                          cudaStream_t s) {
  const long long N = (long long)g.nx * g.ny * g.nz;
  if (prec == PREC_FP32)
    from_canonical_kernel<float><<<grid_for(N, 256), 256, 0, s>>>(g, in, aa,
                                                                  static_cast<float*>(buf));
  else if (prec == PREC_DF)
    from_canonical_kernel<df><<<grid_for(N, 256), 256, 0, s>>>(g, in, aa, static_cast<df*>(buf));
  else
    from_canonical_kernel<double><<<grid_for(N, 256), 256, 0, s>>>(g, in, aa,
                                                                   static_cast<double*>(buf));
  return 1;
}

int launch_macroscopic(const Grid& g, const double* f, const StepConst* sc, const OpenBC& bc,
                       double* rho, double* u, cudaStream_t s) {
  const long long N = (long long)g.nx * g.ny * g.nz;
  macroscopic_kernel<<<grid_for(N, 256), 256, 0, s>>>(g, f, sc, bc, rho, u);
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
    c.head[CC_HF + a] = (T)(0.5 * f[a]);
    c.head[CC_F + a] = (T)f[a];
  }
  c.head[CC_NWP] = (T)(-wp);
  c.head[CC_WPW0] = (T)(wp * (1.0 / 3.0));
  c.head[CC_H] = (T)(-3.0 * (1.0 / 3.0) * gp);
  c.head[CC_H + 1] = (T)(-3.0 * (1.0 / 18.0) * gp);
  c.head[CC_H + 2] = (T)(-3.0 * (1.0 / 36.0) * gp);
  c.head[CC_MHWP] = (T)(-0.5 * wp);
  c.head[CC_WPW] = (T)(wp * (1.0 / 18.0));
  c.head[CC_WPW + 1] = (T)(wp * (1.0 / 36.0));
  c.head[CC_MHWM] = (T)(-0.5 * wm);
  c.head[15] = (T)0;
  c.tail[0] = (T)(1.0 - wp);
  c.tail[1] = (T)(0.5 * (1.0 - wp));
  c.tail[2] = (T)(0.5 * (1.0 - wm));
  c.tail[3] = (T)0;
  for (int k = 0; k < 9; ++k) {
    const double cfk = ckx(k) * f[0] + cky(k) * f[1] + ckz(k) * f[2];
    const double w = wk<double>(k);
    c.pair[k][0] = (T)(gp * 9.0 * w * cfk);
    c.pair[k][1] = (T)(gm * 3.0 * w * cfk);
    c.pair[k][2] = (T)(4.5 * w * wp);
    c.pair[k][3] = (T)(3.0 * w * wm);
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
  if (P.dfrec) fill_coef<df>(sc->x, f, P.omega_p, P.omega_m);
}

int launch_wait_selftest_lbm(unsigned* status, unsigned long long limit_ns, cudaStream_t s) {
  wait_selftest_kernel<<<1, 32, 0, s>>>(status, limit_ns);
  return 1;
}

int launch_step_const(MapParams P, cudaStream_t s) {
  step_const_kernel<<<1, 32, 0, s>>>(P);
  return 1;
}

}  // namespace psm
