// map_kernels.cu -- particle mapping (paper Sec. 2.3.2, Sec. 3.1.1) and the
// fixed-order reduction of hydrodynamic force and torque (Eqs. 21-22).
//
// Mapping replaces the paper's CPU-built sub-block particle lists with a
// device-side, particle-centric scan:
//   1. mark   every cell within reach (centre closer than r + sqrt(3)/2) of a
//             particle sets its bit in the coverage mask;
//   2. scan   exclusive prefix count of the mask words gives each covered
//             cell its slot-table index, in cell order;
//   3. fill   each (particle, covered cell) pair claims one of the cell's two
//             slots and stores B_i = W(eps_i);
//   4. finish slots are ordered by particle index, MLP-mode cells get their
//             eps, and B > 1 is normalised (every B_i divided by the sum).
// Distances, sample points and reach tests use plain IEEE FP64 operations
// (no fused multiply-add: this file is compiled with -fmad=false) so the
// decisions they take are the ones the FP64 definition takes.
#include "psm_internal.cuh"
#include "geom.cuh"

namespace psm {
namespace {

constexpr double HALF_SQRT3 = kHalfSqrt3;
constexpr int MAP_THREADS = 128;

struct Box {
  int lo[3], n[3];
  long long count;
};

__device__ __forceinline__ Box particle_box(const Grid& g, double x0, double x1, double x2,
                                            double r) {
  Box b;
  const double xp[3] = {x0, x1, x2};
  const int dims[3] = {g.nx, g.ny, g.nz};
  for (int a = 0; a < 3; ++a) {
    int lo = (int)floor(xp[a] - r - 1.0);
    int hi = (int)floor(xp[a] + r + 1.0);
    if (g.wall[a]) {
      if (lo < 0) lo = 0;
      if (hi > dims[a] - 1) hi = dims[a] - 1;
    }
    b.lo[a] = lo;
    b.n[a] = hi >= lo ? hi - lo + 1 : 0;
  }
  b.count = (long long)b.n[0] * b.n[1] * b.n[2];
  return b;
}

__device__ __forceinline__ int wrap(int k, int n) {
  int i = k % n;
  return i < 0 ? i + n : i;
}

// nearest image of cell coordinate i relative to xp (integer shifted first)
__device__ __forceinline__ double image_d(int i, double xp, int n, int periodic) {
  double d = ((double)i + 0.5) - xp;
  if (periodic) {
    if (d > 0.5 * n) d = ((double)(i - n) + 0.5) - xp;
    else if (d < -0.5 * n) d = ((double)(i + n) + 0.5) - xp;
  }
  return d;
}

struct CellHit {
  int ix, iy, iz;
  double dx, dy, dz, d2;
};

__device__ __forceinline__ void box_cell(const Grid& g, const Box& b, long long t, double x0,
                                         double x1, double x2, CellHit& h) {
  const int kx = b.lo[0] + (int)(t % b.n[0]);
  const int ky = b.lo[1] + (int)((t / b.n[0]) % b.n[1]);
  const int kz = b.lo[2] + (int)(t / ((long long)b.n[0] * b.n[1]));
  h.ix = wrap(kx, g.nx);
  h.iy = wrap(ky, g.ny);
  h.iz = wrap(kz, g.nz);
  h.dx = image_d(h.ix, x0, g.nx, !g.wall[0]);
  h.dy = image_d(h.iy, x1, g.ny, !g.wall[1]);
  h.dz = image_d(h.iz, x2, g.nz, !g.wall[2]);
  h.d2 = h.dx * h.dx + h.dy * h.dy + h.dz * h.dz;
}

__device__ __forceinline__ bool in_reach(double d2, double r) {
  const double reach = r + HALF_SQRT3;
  return d2 < reach * reach;
}

__device__ __forceinline__ long long padded_cell(const Grid& g, int x, int y, int z) {
  return (long long)x + (long long)g.nxp * ((long long)y + (long long)g.ny * z);
}

__device__ __forceinline__ double weight(double eps, double tau, int nt) {
  if (!nt) return eps;
  return eps * (tau - 0.5) / ((1.0 - eps) + (tau - 0.5));
}

__global__ void mark_kernel(MapParams P) {
  const int p = blockIdx.x;
  const double x0 = P.p.x[3 * p], x1 = P.p.x[3 * p + 1], x2 = P.p.x[3 * p + 2];
  const double r = P.p.r[p];
  const Box b = particle_box(P.g, x0, x1, x2, r);
  for (long long t = threadIdx.x; t < b.count; t += blockDim.x) {
    CellHit h;
    box_cell(P.g, b, t, x0, x1, x2, h);
    if (!in_reach(h.d2, r)) continue;
    const long long cell = padded_cell(P.g, h.ix, h.iy, h.iz);
    atomicOr(&P.cov.mask[cell >> 5], 1u << (cell & 31));
  }
}

// ---- exclusive scan of the popcounts of the mask words
constexpr int SCAN_THREADS = 1024;

__device__ __forceinline__ int block_exclusive_scan(int v, int* total) {
  __shared__ int warp_sums[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int incl = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_sums[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    int s = lane < nw ? warp_sums[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += t;
    }
    if (lane < nw) warp_sums[lane] = s;  // inclusive over warps
  }
  __syncthreads();
  const int warp_off = wid ? warp_sums[wid - 1] : 0;
  *total = warp_sums[(blockDim.x >> 5) - 1];
  __syncthreads();
  return warp_off + incl - v;
}

__global__ void scan_words_kernel(Coverage cov, long long nwords) {
  const long long w = (long long)blockIdx.x * SCAN_THREADS + threadIdx.x;
  const int v = w < nwords ? __popc(cov.mask[w]) : 0;
  int total;
  const int ex = block_exclusive_scan(v, &total);
  if (w < nwords) cov.base[w] = ex;
  if (threadIdx.x == 0) cov.blocksum[blockIdx.x] = total;
}

__global__ void scan_blocks_kernel(Coverage cov, long long nblocks) {
  // one block: each thread scans a contiguous chunk, then the chunk totals
  const long long per = (nblocks + SCAN_THREADS - 1) / SCAN_THREADS;
  const long long lo = per * threadIdx.x;
  const long long hi = lo + per < nblocks ? lo + per : nblocks;
  int s = 0;
  for (long long i = lo; i < hi; ++i) s += cov.blocksum[i];
  int total;
  int run = block_exclusive_scan(s, &total);
  for (long long i = lo; i < hi; ++i) {
    const int v = cov.blocksum[i];
    cov.blocksum[i] = run;
    run += v;
  }
  if (threadIdx.x == 0) *cov.ncov = total;
}

__global__ void scan_add_kernel(Coverage cov, long long nwords) {
  const long long w = (long long)blockIdx.x * SCAN_THREADS + threadIdx.x;
  if (w < nwords) cov.base[w] += cov.blocksum[blockIdx.x];
}

__device__ __forceinline__ int slot_count(const MapParams& P) {
  const long long n = *P.cov.ncov;
  return (int)(n < P.s.cap ? n : P.s.cap);
}

__global__ void clear_slots_kernel(MapParams P) {
  const int n = slot_count(P);
  if (blockIdx.x == 0 && threadIdx.x == 0 && *P.cov.ncov > P.s.cap)
    atomicOr(P.status, ST_SLOT_OVERFLOW);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    P.s.pid[e] = make_int2(-1, -1);
    P.s.cnt[e] = 0;
    if (P.fp32) static_cast<float2*>(P.s.B)[e] = make_float2(0.f, 0.f);
    else static_cast<double2*>(P.s.B)[e] = make_double2(0.0, 0.0);
  }
}

__device__ __forceinline__ void store_B(const MapParams& P, long long e, int s, double B) {
  if (P.fp32) reinterpret_cast<float*>(static_cast<float2*>(P.s.B) + e)[s] = (float)B;
  else reinterpret_cast<double*>(static_cast<double2*>(P.s.B) + e)[s] = B;
}
__device__ __forceinline__ double load_B(const MapParams& P, long long e, int s) {
  if (P.fp32) return (double)reinterpret_cast<const float*>(static_cast<float2*>(P.s.B) + e)[s];
  return reinterpret_cast<const double*>(static_cast<double2*>(P.s.B) + e)[s];
}

__device__ __forceinline__ long long slot_index(const Coverage& cov, long long cell) {
  const long long w = cell >> 5;
  const uint32_t below = (1u << (cell & 31)) - 1u;
  return (long long)cov.base[w] + __popc(cov.mask[w] & below);
}

// eps of a cell for one particle; returns -1 for "resolve in the finish pass"
__device__ double cell_eps(const MapParams& P, const CellHit& h, double r, double fr) {
  const double rin = r - HALF_SQRT3;
  if (rin > 0.0 && h.d2 <= rin * rin) return 1.0;
  if (P.eps_mode == 1) {
    const double dist = sqrt(h.d2);
    const double D = dist - r;
    double e = -D + fr;
    if (e < 0.0) e = 0.0;
    if (e > 1.0) e = 1.0;
    return e;
  }
  if (P.eps_mode == 2) return -1.0;
  return (double)supersample_count(h.dx, h.dy, h.dz, r, P.eps_n) /
         ((double)P.eps_n * P.eps_n * P.eps_n);
}

__global__ void fill_kernel(MapParams P) {
  const int p = blockIdx.x;
  const double x0 = P.p.x[3 * p], x1 = P.p.x[3 * p + 1], x2 = P.p.x[3 * p + 2];
  const double r = P.p.r[p];
  const double fr = P.p.fr[p];
  const Box b = particle_box(P.g, x0, x1, x2, r);
  for (long long t = threadIdx.x; t < b.count; t += blockDim.x) {
    CellHit h;
    box_cell(P.g, b, t, x0, x1, x2, h);
    if (!in_reach(h.d2, r)) continue;
    const long long cell = padded_cell(P.g, h.ix, h.iy, h.iz);
    const long long e = slot_index(P.cov, cell);
    if (e >= P.s.cap) continue;
    const int s = atomicAdd(&P.s.cnt[e], 1);
    if (s >= 2) {
      atomicOr(P.status, ST_SLOT_OVERFLOW);
      continue;
    }
    P.s.cell[e] = (int)cell;
    reinterpret_cast<int*>(&P.s.pid[e])[s] = p;
    const double eps = cell_eps(P, h, r, fr);
    store_B(P, e, s, eps < 0.0 ? -1.0 : weight(eps, P.tau, P.weighting));
  }
}

// surrogate mode: a partial cell within reach of exactly one particle and not
// next to a wall face goes to the network's worklist (inputs d/r, r); the
// finish pass samples every other pending cell with 8^3 points
__global__ void classify_kernel(MapParams P) {
  const int n = slot_count(P);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    if (P.s.cnt[e] != 1) continue;
    const int2 pid = P.s.pid[e];
    if (pid.x < 0 || load_B(P, e, 0) >= 0.0) continue;
    const int cell = P.s.cell[e];
    const int x = cell % P.g.nxp;
    const int y = (cell / P.g.nxp) % P.g.ny;
    const int z = cell / (P.g.nxp * P.g.ny);
    const bool wall = (P.g.wall[0] && (x == 0 || x == P.g.nx - 1)) ||
                      (P.g.wall[1] && (y == 0 || y == P.g.ny - 1)) ||
                      (P.g.wall[2] && (z == 0 || z == P.g.nz - 1));
    if (wall) continue;
    const int p = pid.x;
    const double r = P.p.r[p];
    const double dx = image_d(x, P.p.x[3 * p], P.g.nx, !P.g.wall[0]);
    const double dy = image_d(y, P.p.x[3 * p + 1], P.g.ny, !P.g.wall[1]);
    const double dz = image_d(z, P.p.x[3 * p + 2], P.g.nz, !P.g.wall[2]);
    const int k = atomicAdd(P.mlp_count, 1);
    reinterpret_cast<float4*>(P.mlp_X)[k] =
        make_float4((float)(dx / r), (float)(dy / r), (float)(dz / r), (float)r);
    P.mlp_work[k] = e;
  }
}

__global__ void apply_mlp_kernel(MapParams P) {
  const int n = *P.mlp_count;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    const int e = P.mlp_work[k];
    store_B(P, e, 0, weight((double)P.mlp_eps[k], P.tau, P.weighting));
  }
}

__global__ void finish_kernel(MapParams P) {
  __shared__ double red[256];
  const int n = slot_count(P);
  double accB = 0.0;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    int2 pid = P.s.pid[e];
    double B0 = load_B(P, e, 0), B1 = load_B(P, e, 1);
    if (pid.y >= 0 && pid.y < pid.x) {
      const int t = pid.x; pid.x = pid.y; pid.y = t;
      const double tb = B0; B0 = B1; B1 = tb;
    }
    if (B0 < 0.0 || B1 < 0.0) {
      // cells left for the surrogate and not taken by it: 8^3 sampling
      const int cell = P.s.cell[e];
      const int x = cell % P.g.nxp;
      const int y = (cell / P.g.nxp) % P.g.ny;
      const int z = cell / (P.g.nxp * P.g.ny);
      for (int s = 0; s < 2; ++s) {
        const int p = s ? pid.y : pid.x;
        double& Bs = s ? B1 : B0;
        if (p < 0 || Bs >= 0.0) continue;
        const double r = P.p.r[p];
        const double dx = image_d(x, P.p.x[3 * p], P.g.nx, !P.g.wall[0]);
        const double dy = image_d(y, P.p.x[3 * p + 1], P.g.ny, !P.g.wall[1]);
        const double dz = image_d(z, P.p.x[3 * p + 2], P.g.nz, !P.g.wall[2]);
        const double eps = (double)supersample_count(dx, dy, dz, r, 8) / 512.0;
        Bs = weight(eps, P.tau, P.weighting);
      }
    }
    double B = B0 + B1;
    if (B > 1.0) {
      B0 = B0 / B;
      B1 = B1 / B;
      B = 1.0;
    }
    P.s.pid[e] = pid;
    store_B(P, e, 0, B0);
    store_B(P, e, 1, B1);
    accB += B;
  }
  red[threadIdx.x] = accB;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) P.partials[blockIdx.x] = red[0];
}

// fluid volume sum_x (1 - B) from the finish-pass partial sums, fixed order
__global__ void vfluid_kernel(MapParams P, int nparts) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < nparts; ++b) s += P.partials[b];
    P.sc->sumB = s;
    P.sc->vfluid = P.sc->ncells - s;
  }
}

// ---- fixed-order force and torque reduction, one block per particle
constexpr int RED_THREADS = 128;

template <typename T>
__global__ void force_reduce_kernel(MapParams P) {
  __shared__ double sh[6][RED_THREADS];
  const int p = blockIdx.x;
  const double x0 = P.p.x[3 * p], x1 = P.p.x[3 * p + 1], x2 = P.p.x[3 * p + 2];
  const double r = P.p.r[p];
  const Box b = particle_box(P.g, x0, x1, x2, r);
  const T* Fc = static_cast<const T*>(P.s.Fc);
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  for (long long t = threadIdx.x; t < b.count; t += RED_THREADS) {
    CellHit h;
    box_cell(P.g, b, t, x0, x1, x2, h);
    if (!in_reach(h.d2, r)) continue;
    const long long cell = padded_cell(P.g, h.ix, h.iy, h.iz);
    const long long e = slot_index(P.cov, cell);
    if (e >= P.s.cap) continue;
    const int2 pid = P.s.pid[e];
    const int s = pid.x == p ? 0 : (pid.y == p ? 1 : -1);
    if (s < 0) continue;
    const double f0 = (double)Fc[6 * e + 3 * s];
    const double f1 = (double)Fc[6 * e + 3 * s + 1];
    const double f2 = (double)Fc[6 * e + 3 * s + 2];
    acc[0] += f0;
    acc[1] += f1;
    acc[2] += f2;
    acc[3] += h.dy * f2 - h.dz * f1;
    acc[4] += h.dz * f0 - h.dx * f2;
    acc[5] += h.dx * f1 - h.dy * f0;
  }
  for (int i = 0; i < 6; ++i) sh[i][threadIdx.x] = acc[i];
  __syncthreads();
  for (int s = RED_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int i = 0; i < 6; ++i) sh[i][threadIdx.x] += sh[i][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    bool finite = true;
    for (int i = 0; i < 3; ++i) {
      P.p.Fh[3 * p + i] = sh[i][0];
      P.p.Th[3 * p + i] = sh[3 + i][0];
      finite = finite && isfinite(sh[i][0]) && isfinite(sh[3 + i][0]);
    }
    if (!finite) atomicOr(P.status, ST_NONFINITE);
  }
}

__global__ void pack_particles_kernel(Particles p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.n) return;
  for (int a = 0; a < 3; ++a) {
    p.xf[4 * i + a] = (float)p.x[3 * i + a];
    p.uf[4 * i + a] = (float)p.u[3 * i + a];
    p.omf[4 * i + a] = (float)p.om[3 * i + a];
  }
  p.xf[4 * i + 3] = (float)p.r[i];
  p.uf[4 * i + 3] = 0.f;
  p.omf[4 * i + 3] = 0.f;
}

// positions along periodic axes wrapped into the box (host-supplied states)
__global__ void wrap_particles_kernel(Grid g, Particles p) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= p.n) return;
  const int dims[3] = {g.nx, g.ny, g.nz};
  for (int a = 0; a < 3; ++a) {
    if (g.wall[a]) continue;
    double v = fmod(p.x[3 * i + a], (double)dims[a]);
    if (v < 0.0) v += dims[a];
    p.x[3 * i + a] = v;
  }
}

__global__ void dense_clear_kernel(long long N, int* pid0, double* B0, int* pid1, double* B1) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < N;
       c += (long long)gridDim.x * blockDim.x) {
    pid0[c] = -1;
    pid1[c] = -1;
    B0[c] = 0.0;
    B1[c] = 0.0;
  }
}

__global__ void dense_scatter_kernel(MapParams P, int* pid0, double* B0, int* pid1, double* B1) {
  const int n = slot_count(P);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int cell = P.s.cell[e];
    const int x = cell % P.g.nxp;
    const int y = (cell / P.g.nxp) % P.g.ny;
    const int z = cell / (P.g.nxp * P.g.ny);
    const long long c = (long long)x + (long long)P.g.nx * ((long long)y + (long long)P.g.ny * z);
    const int2 pid = P.s.pid[e];
    pid0[c] = pid.x;
    pid1[c] = pid.y;
    B0[c] = load_B(P, e, 0);
    B1[c] = load_B(P, e, 1);
  }
}

unsigned grid_cap(long long n, int block) {
  long long b = (n + block - 1) / block;
  if (b > 152LL * 32) b = 152LL * 32;
  return (unsigned)(b > 0 ? b : 1);
}

}  // namespace

int launch_map(MapParams P, cudaStream_t s) {
  int launches = 0;
  cudaMemsetAsync(P.cov.mask, 0, sizeof(uint32_t) * P.g.nwords, s);
  if (P.p.n > 0) {
    mark_kernel<<<P.p.n, MAP_THREADS, 0, s>>>(P);
    ++launches;
  }
  const unsigned nb = (unsigned)P.cov.nblocks;
  scan_words_kernel<<<nb, SCAN_THREADS, 0, s>>>(P.cov, P.g.nwords);
  scan_blocks_kernel<<<1, SCAN_THREADS, 0, s>>>(P.cov, P.cov.nblocks);
  scan_add_kernel<<<nb, SCAN_THREADS, 0, s>>>(P.cov, P.g.nwords);
  launches += 3;
  clear_slots_kernel<<<grid_cap(P.s.cap, 256), 256, 0, s>>>(P);
  ++launches;
  if (P.p.n > 0) {
    fill_kernel<<<P.p.n, MAP_THREADS, 0, s>>>(P);
    ++launches;
  }
  const unsigned nfin = grid_cap(P.s.cap, 256);
  finish_kernel<<<nfin, 256, 0, s>>>(P);
  vfluid_kernel<<<1, 32, 0, s>>>(P, (int)nfin);
  launches += 2;
  return launches;
}

int launch_mlp_infer_dev(const float* params, const int* count_dev, long long cap,
                         const float* X, float* eps, cudaStream_t s);

// mapping with the surrogate: as launch_map, with the network evaluated on the
// tensor cores for the worklist between the fill and finish passes
int launch_map_mlp(MapParams P, cudaStream_t s) {
  int launches = 0;
  cudaMemsetAsync(P.cov.mask, 0, sizeof(uint32_t) * P.g.nwords, s);
  cudaMemsetAsync(P.mlp_count, 0, sizeof(int), s);
  if (P.p.n > 0) {
    mark_kernel<<<P.p.n, MAP_THREADS, 0, s>>>(P);
    ++launches;
  }
  const unsigned nb = (unsigned)P.cov.nblocks;
  scan_words_kernel<<<nb, SCAN_THREADS, 0, s>>>(P.cov, P.g.nwords);
  scan_blocks_kernel<<<1, SCAN_THREADS, 0, s>>>(P.cov, P.cov.nblocks);
  scan_add_kernel<<<nb, SCAN_THREADS, 0, s>>>(P.cov, P.g.nwords);
  clear_slots_kernel<<<grid_cap(P.s.cap, 256), 256, 0, s>>>(P);
  launches += 4;
  if (P.p.n > 0) {
    fill_kernel<<<P.p.n, MAP_THREADS, 0, s>>>(P);
    ++launches;
  }
  if (P.mlp) {
    classify_kernel<<<grid_cap(P.s.cap, 256), 256, 0, s>>>(P);
    launches += launch_mlp_infer_dev(P.mlp, P.mlp_count, P.s.cap, P.mlp_X, P.mlp_eps, s);
    apply_mlp_kernel<<<grid_cap(P.s.cap, 256), 256, 0, s>>>(P);
    launches += 2;
  }
  const unsigned nfin = grid_cap(P.s.cap, 256);
  finish_kernel<<<nfin, 256, 0, s>>>(P);
  vfluid_kernel<<<1, 32, 0, s>>>(P, (int)nfin);
  launches += 2;
  return launches;
}

int launch_force_reduce(MapParams P, cudaStream_t s) {
  if (P.p.n == 0) return 0;
  if (P.fp32) force_reduce_kernel<float><<<P.p.n, RED_THREADS, 0, s>>>(P);
  else force_reduce_kernel<double><<<P.p.n, RED_THREADS, 0, s>>>(P);
  return 1;
}

int launch_pack_particles(Particles p, cudaStream_t s) {
  if (p.n == 0) return 0;
  pack_particles_kernel<<<(p.n + 127) / 128, 128, 0, s>>>(p);
  return 1;
}

int launch_wrap_particles(const Grid& g, Particles p, cudaStream_t s) {
  if (p.n == 0) return 0;
  wrap_particles_kernel<<<(p.n + 127) / 128, 128, 0, s>>>(g, p);
  return 1;
}

int launch_slots_to_dense(MapParams P, int* pid0, double* B0, int* pid1, double* B1,
                          cudaStream_t s) {
  const long long N = (long long)P.g.nx * P.g.ny * P.g.nz;
  dense_clear_kernel<<<grid_cap(N, 256), 256, 0, s>>>(N, pid0, B0, pid1, B1);
  dense_scatter_kernel<<<grid_cap(P.s.cap, 256), 256, 0, s>>>(P, pid0, B0, pid1, B1);
  return 2;
}

}  // namespace psm
