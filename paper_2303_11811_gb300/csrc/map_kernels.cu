// map_kernels.cu -- particle mapping (paper Sec. 2.3.2, Sec. 3.1.1) and the
// fixed-order reduction of hydrodynamic force and torque (Eqs. 21-22).
//
// Mapping replaces the paper's CPU-built sub-block particle lists with a
// device-side, particle-centric scan:
//   1. mark   every cell within reach (centre closer than r + sqrt(3)/2) of a
//             particle sets its bit in the coverage mask (and, when the bit
//             was set already, in the mask of shared cells);
//   2. scan   exclusive prefix count of the mask words gives each covered
//             cell its slot-table index, in cell order;
//   3. fill   each (particle, covered cell) pair takes one of the cell's two
//             slots (slot 0 when the cell is not shared, else a claim on a
//             counter), stores B_i = W(eps_i) and appends the entry to the
//             particle's list (box order, deterministic); with 8^3 sampling
//             the cells that need samples go to a per-particle worklist,
//             3b. count8 counts them, four cells per warp;
//   4. finish slots are ordered by particle index, MLP-mode and fallback cells
//             get their eps, and B > 1 is normalised (every B_i divided by
//             the sum); FP64 records: the mask of cells with one particle and
//             B = 1.
// Reach tests and sub-cell sampling take the FP64 definition's decisions: FP32
// with a certified band and FP64 inside the band (geom.cuh); this file is
// compiled with -fmad=false (fused multiply-adds only where written out).
#include "geom.cuh"
#include "psm_internal.cuh"

namespace psm {
namespace {

constexpr double HALF_SQRT3 = kHalfSqrt3;
constexpr int MAP_THREADS = 128;
// threads of a fill block (one block per particle) and blocks per SM: a
// block's phases wait on dependent global loads, so many small blocks keep
// more of them in flight (settle512: 64 threads map 6-7% faster than 256;
// 10 blocks per SM, 102 registers, 3% faster than 12 blocks at 85)
constexpr int FILL_THREADS = 64;
constexpr int FILL_MIN_BLOCKS = 10;
constexpr int RED_THREADS = 128;
constexpr int SCAN_THREADS = 1024;

struct Box {
  double rin2;        // (r - sqrt(3)/2)^2 when r > sqrt(3)/2, else -1
  float rin2f;
  int lo[3], n[3];
  int count;
  int ip[3];          // floor of the centre
  float fpf[3];       // centre minus its floor, rounded to FP32
  double xp[3];
  double r;
  double reach2;      // (r + sqrt(3)/2)^2 in FP64
  float reach2f, E;   // its FP32 value and the certified band of geom.cuh
  float r2f;          // (float)(r * r)
  bool has_in;        // rin2 >= 0: cells can lie inside by the margin
  // the n^3 = 8^3 samples lie within 7 sqrt(3)/16 < 0.76 of the cell centre:
  // (r -+ 0.76)^2 in FP32 (in8f < 0 when r <= 0.76), for counts of 512 and 0
  // taken without sampling
  float in8f, out8f;
  FastDiv div_n0, div_nxy;  // box index t -> (kx, ky, kz)
  FastDiv div_n1;           // box row r -> (ky, kz)
};

__device__ __forceinline__ Box particle_box(const Grid& g, const double* x, double r) {
  Box b;
  const int dims[3] = {g.nx, g.ny, g.nz};
  for (int a = 0; a < 3; ++a) {
    const double xp = x[a];
    int lo = (int)floor(xp - r - 1.0);
    int hi = (int)floor(xp + r + 1.0);
    if (g.wall[a]) {
      if (lo < 0) lo = 0;
      if (hi > dims[a] - 1) hi = dims[a] - 1;
    }
    b.lo[a] = lo;
    b.n[a] = hi >= lo ? hi - lo + 1 : 0;
    b.xp[a] = xp;
    const double fl = floor(xp);
    b.ip[a] = (int)fl;
    b.fpf[a] = (float)(xp - fl);
  }
  b.count = b.n[0] * b.n[1] * b.n[2];
  b.div_n0 = make_fastdiv((unsigned)(b.n[0] > 0 ? b.n[0] : 1));
  b.div_n1 = make_fastdiv((unsigned)(b.n[1] > 0 ? b.n[1] : 1));
  b.div_nxy = make_fastdiv((unsigned)(b.n[0] * b.n[1] > 0 ? b.n[0] * b.n[1] : 1));
  b.r = r;
  const double reach = r + HALF_SQRT3;
  b.reach2 = reach * reach;
  b.reach2f = (float)b.reach2;
  b.E = certified_band(r);
  b.r2f = (float)(r * r);
  const double rin = r - HALF_SQRT3;
  b.rin2 = rin > 0.0 ? rin * rin : -1.0;
  b.has_in = rin > 0.0;
  b.rin2f = (float)b.rin2;
  b.in8f = r > 0.76 ? (float)((r - 0.76) * (r - 0.76)) : -1.0f;
  b.out8f = (float)((r + 0.76) * (r + 0.76));
  return b;
}

// Every particle's box, one thread per particle: the FP64 set-up of the mark
// and fill passes (on GB300 a serial FP64 sequence in one thread of each
// block would hold the block at its first barrier)
__global__ void box_kernel(MapParams P) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < P.p.n) static_cast<Box*>(P.boxes)[p] = particle_box(P.g, P.p.x + 3 * p, P.p.r[p]);
}

// a particle's box into shared memory, copied by the block's threads
__device__ __forceinline__ void load_box(const MapParams& P, int p, Box* sb) {
  static_assert(sizeof(Box) % 4 == 0, "Box is copied as 32-bit words");
  constexpr int W = (int)(sizeof(Box) / 4);
  const int* src = reinterpret_cast<const int*>(static_cast<const Box*>(P.boxes) + p);
  for (int i = threadIdx.x; i < W; i += blockDim.x) reinterpret_cast<int*>(sb)[i] = src[i];
  __syncthreads();
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

// One cell of a particle's bounding box.  Box coordinates k are unwrapped
// around the centre and the box is narrower than half a periodic box, so
// ((double)k + 1/2) - x_p is the nearest-image offset.
struct CellHit {
  int ix, iy, iz;
  int kx, ky, kz;
  double dx, dy, dz, d2;
  float d2f;
  float dxf, dyf, dzf;  // FP32 roundings of dx, dy, dz
};

// box coordinates lie within one period of the grid (the box is narrower
// than half a periodic extent)
__device__ __forceinline__ int wrap1(int k, int n) { return k < 0 ? k + n : (k >= n ? k - n : k); }

__device__ __forceinline__ void box_coords(const Grid& g, const Box& b, int t, CellHit& h) {
  const int kz = (int)b.div_nxy.div((unsigned)t);
  const int rem = t - kz * (b.n[0] * b.n[1]);
  const int ky = (int)b.div_n0.div((unsigned)rem);
  h.kx = b.lo[0] + (rem - ky * b.n[0]);
  h.ky = b.lo[1] + ky;
  h.kz = b.lo[2] + kz;
  h.ix = wrap1(h.kx, g.nx);
  h.iy = wrap1(h.ky, g.ny);
  h.iz = wrap1(h.kz, g.nz);
}

// reach test of the FP64 definition, evaluated in FP32 outside the certified
// band (FP64 offsets only inside the band)
__device__ __forceinline__ bool reach_test(const Box& b, CellHit& h) {
  const float dxf = (float)(h.kx - b.ip[0]) + (0.5f - b.fpf[0]);
  const float dyf = (float)(h.ky - b.ip[1]) + (0.5f - b.fpf[1]);
  const float dzf = (float)(h.kz - b.ip[2]) + (0.5f - b.fpf[2]);
  const float d2f = dxf * dxf + dyf * dyf + dzf * dzf;
  h.d2f = d2f;
  if (d2f > b.reach2f + b.E) return false;
  if (d2f < b.reach2f - b.E) return true;
  const double dx = ((double)h.kx + 0.5) - b.xp[0];
  const double dy = ((double)h.ky + 0.5) - b.xp[1];
  const double dz = ((double)h.kz + 0.5) - b.xp[2];
  return dx * dx + dy * dy + dz * dz < b.reach2;
}

__device__ __forceinline__ long long padded_cell(const Grid& g, int x, int y, int z) {
  return (long long)x + (long long)g.nxp * ((long long)y + (long long)g.ny * z);
}

// padded cell index -> (x, y, z); nxp is a multiple of 32, so the row is the
// coverage word divided by the words per row
__device__ __forceinline__ void cell_xyz(const Grid& g, int cell, int& x, int& y, int& z) {
  const unsigned row = g.div_wpr.div((unsigned)cell >> 5);
  x = cell - (int)row * g.nxp;
  z = (int)g.div_ny.div(row);
  y = (int)row - z * g.ny;
}

// B(eps); for eps = 0 and eps = 1 the FP64 formula gives exactly 0 and 1
__device__ __forceinline__ double weight(double eps, double tau, int nt) {
  if (!nt || eps == 0.0 || eps == 1.0) return eps;
  return eps * (tau - 0.5) / ((1.0 - eps) + (tau - 0.5));
}

// the weight of slot s of entry e lives in the last component of its record
// (during the mapping: raw, -1 for "resolved in a later pass"; after the
// finish pass: normalised, slot 0's negated when the cell has a second
// particle)
__device__ __forceinline__ long long rec_w(const MapParams& P, long long e, int s) {
  return 4 * (s * P.s.cap + e) + 3;
}
__device__ __forceinline__ double load_B(const MapParams& P, long long e, int s) {
  if (P.fp32) return (double)static_cast<const float*>(P.s.V)[rec_w(P, e, s)];
  if (P.dfrec) return to_double(static_cast<const df*>(P.s.V)[rec_w(P, e, s)]);
  return static_cast<const double*>(P.s.V)[rec_w(P, e, s)];
}

__device__ __forceinline__ long long slot_index(const Coverage& cov, long long cell) {
  const long long w = cell >> 5;
  const uint32_t below = (1u << (cell & 31)) - 1u;
  return (long long)cov.base[w] + __popc(cov.mask[w] & below);
}

__device__ __forceinline__ int slot_count(const MapParams& P) {
  const long long n = *P.cov.ncov;
  return (int)(n < P.s.cap ? n : P.s.cap);
}

__device__ __forceinline__ void load_offsets(int n, double* s64, float* s32) {
  if (threadIdx.x < n) {
    s64[threadIdx.x] = sample_offset(threadIdx.x, n);
    s32[threadIdx.x] = (float)s64[threadIdx.x];
  }
  __syncthreads();
}

// reach test of box cell (kx, ky, kz) (box coordinates unwrapped), the FP64
// definition's decision (reach_test)
__device__ __forceinline__ bool in_reach(const Box& b, int kx, int ky, int kz) {
  CellHit h;
  h.kx = kx;
  h.ky = ky;
  h.kz = kz;
  return reach_test(b, h);
}

// inside by the margin (FP64 squared distance <= (r - sqrt(3)/2)^2, the
// decision of the fill pass's class test), in FP32 outside the certified band
__device__ __forceinline__ bool inside_margin(const Box& b, int kx, int ky, int kz) {
  const float dxf = (float)(kx - b.ip[0]) + (0.5f - b.fpf[0]);
  const float dyf = (float)(ky - b.ip[1]) + (0.5f - b.fpf[1]);
  const float dzf = (float)(kz - b.ip[2]) + (0.5f - b.fpf[2]);
  const float d2f = dxf * dxf + dyf * dyf + dzf * dzf;
  if (d2f < b.rin2f - b.E) return true;
  if (d2f > b.rin2f + b.E) return false;
  const double dx = ((double)kx + 0.5) - b.xp[0];
  const double dy = ((double)ky + 0.5) - b.xp[1];
  const double dz = ((double)kz + 0.5) - b.xp[2];
  return dx * dx + dy * dy + dz * dz <= b.rin2;
}

__device__ __forceinline__ bool wall_cell(const Grid& g, int ix, int iy, int iz) {
  return (g.wall[0] && (ix == 0 || ix == g.nx - 1)) || (g.wall[1] && (iy == 0 || iy == g.ny - 1)) ||
         (g.wall[2] && (iz == 0 || iz == g.nz - 1));
}

// surrogate mode: of the cells a..e of a box row (all in reach), those that
// go to the network: not inside by the margin and not next to a wall face.
// Like the cells in reach, the inside cells of a row form one run around
// the centre's column kc (the FP64 squared distance is unimodal along x).
__device__ int row_net(const Grid& g, const Box& b, int a, int e, int kc, int ky, int kz) {
  const int iy = wrap1(ky, g.ny), iz = wrap1(kz, g.nz);
  if ((g.wall[1] && (iy == 0 || iy == g.ny - 1)) || (g.wall[2] && (iz == 0 || iz == g.nz - 1)))
    return 0;
  int ai = 1, ei = 0;  // inside run (empty)
  if (b.has_in && inside_margin(b, kc, ky, kz)) {
    const float dyf = (float)(ky - b.ip[1]) + (0.5f - b.fpf[1]);
    const float dzf = (float)(kz - b.ip[2]) + (0.5f - b.fpf[2]);
    const float rem = b.rin2f - (dyf * dyf + dzf * dzf);
    const int w = (int)sqrtf(rem > 0.f ? rem : 0.f) + 1;
    ai = kc - w < a ? a : kc - w;
    while (ai < kc && !inside_margin(b, ai, ky, kz)) ++ai;
    while (ai > a && inside_margin(b, ai - 1, ky, kz)) --ai;
    ei = kc + w > e ? e : kc + w;
    while (ei > kc && !inside_margin(b, ei, ky, kz)) --ei;
    while (ei < e && inside_margin(b, ei + 1, ky, kz)) ++ei;
  }
  int net = (e - a + 1) - (ei >= ai ? ei - ai + 1 : 0);
  if (g.wall[0]) {  // along a wall axis box coordinates are not wrapped
    if (a <= 0 && 0 <= e && !(ai <= 0 && 0 <= ei)) --net;
    const int xl = g.nx - 1;
    if (xl > 0 && a <= xl && xl <= e && !(ai <= xl && xl <= ei)) --net;
  }
  return net;
}

// coverage bits of the cells x0..x1 (0 <= x0 <= x1 < nx) of the grid row
// whose first mask word is wb, one atomicOr per word; bits that were set
// already (a second particle) go to the mask of shared cells.  A run of at
// most 33 cells spans at most two words, whose atomics are both issued
// before either result is used.
__device__ __forceinline__ unsigned run_bits(int x0, int x1, int w) {
  const int b0 = x0 - 32 * w > 0 ? x0 - 32 * w : 0;
  const int b1 = x1 - 32 * w < 31 ? x1 - 32 * w : 31;
  const unsigned hi = b1 == 31 ? 0xffffffffu : (1u << (b1 + 1)) - 1u;
  return hi & ~((1u << b0) - 1u);
}
__device__ __forceinline__ void cover_run(const Coverage& cov, long long wb, int x0, int x1) {
  const int w0 = x0 >> 5, w1 = x1 >> 5;
  if (w1 - w0 <= 1) {
    const unsigned m0 = run_bits(x0, x1, w0);
    const unsigned m1 = w1 > w0 ? run_bits(x0, x1, w1) : 0u;
    const unsigned o0 = atomicOr(cov.mask + wb + w0, m0);
    const unsigned o1 = w1 > w0 ? atomicOr(cov.mask + wb + w1, m1) : 0u;
    if (o0 & m0) atomicOr(cov.dup + wb + w0, o0 & m0);
    if (o1 & m1) atomicOr(cov.dup + wb + w1, o1 & m1);
    return;
  }
  for (int w = w0; w <= w1; ++w) {
    const unsigned bits = run_bits(x0, x1, w);
    const unsigned old = atomicOr(cov.mask + wb + w, bits);
    if (old & bits) atomicOr(cov.dup + wb + w, old & bits);
  }
}

// the row pass serves boxes of at most MARK_MAX_ROWS rows (radius up to 14)
constexpr int MARK_MAX_ROWS = 1024;

// Cells in reach of one particle (one block per particle): the coverage bits
// (the mask of shared cells from the bits already set) and the particle's
// list of its cells in box order, as box indices t; the fill pass replaces
// them by slot indices.  Along an x-row of the box the FP64 squared distance
// is unimodal (IEEE rounding is monotone), so the row's cells in reach form
// one run: its ends are found with a few certified reach tests around the
// cell holding the centre.  One thread per row finds the run, the run
// lengths are scanned in row order, the same thread sets the run's bits with
// one atomicOr per mask word, and the list entries are written in list order
// (a thread per entry finds its row by bisection).  In surrogate mode the
// row's cells for the network are counted as well.  Very large boxes test
// every cell.
__global__ void __launch_bounds__(MAP_THREADS, 12) mark_kernel(MapParams P) {
  __shared__ int warp_tot[MAP_THREADS / 32];
  __shared__ int running, net_sum;
  __shared__ Box sbox;
  __shared__ int row_lo[MARK_MAX_ROWS], row_n[MARK_MAX_ROWS], row_off[MARK_MAX_ROWS];
  const int p = blockIdx.x;
  const long long loff = P.list_off[p];
  const int lcap = (int)(P.list_off[p + 1] - loff);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const bool count_net = P.list_net != nullptr;
  if (threadIdx.x == 0) {
    running = 0;
    net_sum = 0;
  }
  load_box(P, p, &sbox);  // ends with __syncthreads
  const Box b = sbox;
  const int rows = b.n[1] * b.n[2];
  int net = 0;
  if (rows <= MARK_MAX_ROWS) {
    // ---- runs of the rows
    const int kc = b.ip[0];  // the x cell holding the centre: the row's closest
    for (int r = threadIdx.x; r < rows; r += MAP_THREADS) {
      const int rz = (int)b.div_n1.div((unsigned)r);
      const int kz = b.lo[2] + rz;
      const int ky = b.lo[1] + (r - rz * b.n[1]);
      int lo = 0, cnt = 0;
      if (b.n[0] > 0 && in_reach(b, kc, ky, kz)) {
        const float dyf = (float)(ky - b.ip[1]) + (0.5f - b.fpf[1]);
        const float dzf = (float)(kz - b.ip[2]) + (0.5f - b.fpf[2]);
        const float rem = b.reach2f - (dyf * dyf + dzf * dzf);
        const int w = (int)sqrtf(rem > 0.f ? rem : 0.f) + 1;
        const int x0 = b.lo[0], x1 = b.lo[0] + b.n[0] - 1;
        int a = kc - w < x0 ? x0 : kc - w;
        while (a < kc && !in_reach(b, a, ky, kz)) ++a;
        while (a > x0 && in_reach(b, a - 1, ky, kz)) --a;
        int e = kc + w > x1 ? x1 : kc + w;
        while (e > kc && !in_reach(b, e, ky, kz)) --e;
        while (e < x1 && in_reach(b, e + 1, ky, kz)) ++e;
        lo = a - x0;
        cnt = e - a + 1;
        if (count_net) net += row_net(P.g, b, a, e, kc, ky, kz);
      }
      row_lo[r] = lo;
      row_n[r] = cnt;
    }
    __syncthreads();
    // ---- exclusive scan of the run lengths in row order: each thread sums a
    // contiguous chunk of rows, the chunk totals are scanned across the block
    const int per = (rows + MAP_THREADS - 1) / MAP_THREADS;
    const int r0 = threadIdx.x * per;
    int mine = 0;
    for (int r = r0; r < r0 + per && r < rows; ++r) mine += row_n[r];
    int incl = mine;
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    int base = 0, total = 0;
    for (int w = 0; w < MAP_THREADS / 32; ++w) {
      if (w < wid) base += warp_tot[w];
      total += warp_tot[w];
    }
    int off = base + incl - mine;
    for (int r = r0; r < r0 + per && r < rows; ++r) {
      row_off[r] = off;
      off += row_n[r];
    }
    __syncthreads();
    // ---- coverage bits: one thread per row, one atomicOr per mask word
    for (int r = threadIdx.x; r < rows; r += MAP_THREADS) {
      const int n = row_n[r];
      if (n == 0) continue;
      const int rz = (int)b.div_n1.div((unsigned)r);
      const int kz = b.lo[2] + rz;
      const int ky = b.lo[1] + (r - rz * b.n[1]);
      const long long wb = padded_cell(P.g, 0, wrap1(ky, P.g.ny), wrap1(kz, P.g.nz)) >> 5;
      // the run in grid x: box x is unwrapped and the run is shorter than
      // the period, so it wraps at most once
      const int xs = wrap1(b.lo[0] + row_lo[r], P.g.nx), xe = xs + n - 1;
      if (xe < P.g.nx) {
        cover_run(P.cov, wb, xs, xe);
      } else {
        cover_run(P.cov, wb, xs, P.g.nx - 1);
        cover_run(P.cov, wb, 0, xe - P.g.nx);
      }
    }
    // ---- list entries in list order (coalesced stores): entry pos belongs
    // to the last row whose offset is <= pos (that row is not empty)
    const int m = total < lcap ? total : lcap;
    for (int pos = threadIdx.x; pos < m; pos += MAP_THREADS) {
      int lo = 0, hi = rows - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (row_off[mid] <= pos) lo = mid;
        else hi = mid - 1;
      }
      P.list[loff + pos] = row_lo[lo] + b.n[0] * lo + (pos - row_off[lo]);
    }
    if (count_net) {
      net = __reduce_add_sync(0xffffffffu, net);
      if (lane == 0 && net) atomicAdd(&net_sum, net);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      P.list_cnt[p] = total < lcap ? total : lcap;
      if (total > lcap) atomicOr(P.status, ST_SLOT_OVERFLOW);
      if (count_net) P.list_net[p] = net_sum;
    }
    return;
  }
  // ---- very large boxes: every cell of the box
  for (int t0 = 0; t0 < b.count; t0 += MAP_THREADS) {
    const int t = t0 + threadIdx.x;
    CellHit h;
    bool in = false;
    if (t < b.count) {
      box_coords(P.g, b, t, h);
      in = reach_test(b, h);
    }
    if (count_net && in && !wall_cell(P.g, h.ix, h.iy, h.iz) &&
        !(b.has_in && inside_margin(b, h.kx, h.ky, h.kz)))
      ++net;
    const unsigned bal = __ballot_sync(0xffffffffu, in);
    if (lane == 0) warp_tot[wid] = __popc(bal);
    const long long cell = in ? padded_cell(P.g, h.ix, h.iy, h.iz) : 0;
    unsigned pend = bal;
    while (pend) {
      const int leader = __ffs(pend) - 1;
      const long long w0 = __shfl_sync(0xffffffffu, cell >> 5, leader);
      const bool mine = in && (cell >> 5) == w0;
      const unsigned bits = __reduce_or_sync(0xffffffffu, mine ? 1u << (cell & 31) : 0u);
      if (lane == leader) {
        const unsigned old = atomicOr(&P.cov.mask[w0], bits);
        if (old & bits) atomicOr(&P.cov.dup[w0], old & bits);
      }
      pend &= ~__ballot_sync(0xffffffffu, mine);
    }
    __syncthreads();
    int before = running, chunk = 0;
    for (int w = 0; w < MAP_THREADS / 32; ++w) {
      if (w < wid) before += warp_tot[w];
      chunk += warp_tot[w];
    }
    const int pos = before + __popc(bal & ((1u << lane) - 1u));
    if (in && pos < lcap) P.list[loff + pos] = t;
    __syncthreads();
    if (threadIdx.x == 0) running += chunk;
    __syncthreads();
  }
  if (count_net) {
    net = __reduce_add_sync(0xffffffffu, net);
    if (lane == 0 && net) atomicAdd(&net_sum, net);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    P.list_cnt[p] = running < lcap ? running : lcap;
    if (running > lcap) atomicOr(P.status, ST_SLOT_OVERFLOW);
    if (count_net) P.list_net[p] = net_sum;
  }
}

// ---- exclusive scan of the popcounts of the mask words
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

__global__ void clear_slots_kernel(MapParams P) {
  const int n = slot_count(P);
  if (blockIdx.x == 0 && threadIdx.x == 0 && *P.cov.ncov > P.s.cap)
    atomicOr(P.status, ST_SLOT_OVERFLOW);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    P.s.pid[e] = make_int2(-1, -1);
    if ((e & 15) == 0) P.s.cnt[e >> 4] = 0;  // 16 packed counters per word
  }
}

// sampled count of a cell for one particle (n^3 for a cell inside by the
// margin sqrt(3)/2, which the sampling would also give)
template <int NS>
__device__ int cell_count(const MapParams& P, const Box& b, const CellHit& h, const double* s64,
                          const float* s32) {
  const int n = P.eps_n;
  if (b.has_in) {
    if (h.d2f < b.rin2f - b.E) return n * n * n;
    if (h.d2f <= b.rin2f + b.E && h.dx * h.dx + h.dy * h.dy + h.dz * h.dz <= b.rin2)
      return n * n * n;
  }
  if (NS > 0)
    return supersample_count_n<(NS > 0 ? NS : 1)>(h.dx, h.dy, h.dz, b.r, h.dxf, h.dyf, h.dzf,
                                                  b.r2f, b.E);
  return supersample_count_fast(h.dx, h.dy, h.dz, b.r, n, s64, s32);
}

// eps of a cell for one particle; -1 means "resolved in a later pass".  The
// inside test d2 <= (r - sqrt(3)/2)^2 is taken in FP32 outside the band.
__device__ double cell_eps(const MapParams& P, const Box& b, const CellHit& h, double fr,
                           const double* s64, const float* s32) {
  const double r = b.r;
  if (b.rin2 >= 0.0) {
    if (h.d2f < b.rin2f - b.E) return 1.0;
    if (h.d2f <= b.rin2f + b.E && h.d2 <= b.rin2) return 1.0;
  }
  if (P.eps_mode == 1) {  // Eqs. 25-26
    const double dist = sqrt(h.d2);
    const double D = dist - r;
    double e = -D + fr;
    if (e < 0.0) e = 0.0;
    if (e > 1.0) e = 1.0;
    return e;
  }
  if (P.eps_mode == 2) return -1.0;
  const int n = P.eps_n;
  const int cnt = n == 4   ? supersample_count_n<4>(h.dx, h.dy, h.dz, r)
                  : n == 8 ? supersample_count_n<8>(h.dx, h.dy, h.dz, r)
                           : supersample_count_fast(h.dx, h.dy, h.dz, r, n, s64, s32);
  const int n3 = n * n * n;
  // count / n^3; for n^3 a power of two the product with the reciprocal is
  // the same IEEE result as the quotient
  if ((n3 & (n3 - 1)) == 0) return (double)cnt * (1.0 / (double)n3);
  return (double)cnt / (double)n3;
}

// eps of a sampled count: count / n^3; for n^3 a power of two the product
// with the reciprocal is the same IEEE result as the quotient
__device__ __forceinline__ double count_eps(int cnt, int n3) {
  if ((n3 & (n3 - 1)) == 0) return (double)cnt * (1.0 / (double)n3);
  return (double)cnt / (double)n3;
}

constexpr int WTAB = 513;  // B of every sampled count up to 8^3
constexpr int WTAB_DF = WTAB + 257;  // their double-float pairs (after the FP32 copy)
constexpr int FILL_AXIS = 64;  // box extent per axis with offset tables (r < 30)

// B of every sampled count (Eq. 16 of each eps = c / n^3), once per context
// (doubles at out[0..n3], their FP32 roundings after WTAB doubles, their
// double-float pairs after WTAB_DF doubles)
__global__ void wtab_kernel(int n3, double tau, int weighting, double* out) {
  float* outf = reinterpret_cast<float*>(out + WTAB);
  df* outd = reinterpret_cast<df*>(out + WTAB_DF);
  for (int c = threadIdx.x; c <= n3; c += blockDim.x) {
    const double B = weight(count_eps(c, n3), tau, weighting);
    out[c] = B;
    outf[c] = (float)B;
    outd[c] = df(B);
  }
}

// 8^3 sampled count of a cell for one sphere by a whole warp: every lane
// passes the same FP32 roundings of the offset d (dxf, dyf, dzf), of r^2
// (r2f) and the certified band E of geom.cuh; the FP64 offset and r^2 are
// taken from lane L.  Lane l takes the sample columns (a, b) = (l / 4,
// 2 (l % 4) + {0, 1}), 16 samples, with the certified FP32 test; if any lane
// has a sample inside the band, every lane recounts its samples with the FP64
// definition inside the band.  Same count as the FP64 definition.
__device__ int warp_count8(float dxf, float dyf, float dzf, float r2f, float E, int L, double dx,
                           double dy, double dz, double r2) {
  const int lane = threadIdx.x & 31;
  const float lo = r2f - E, hi = r2f + E;
  const int a = lane >> 2;
  const float px = dxf + (((float)a + 0.5f) * 0.125f - 0.5f);
  const float Xa = px * px;
  float Z[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float pz = dzf + (((float)c + 0.5f) * 0.125f - 0.5f);
    Z[c] = pz * pz;
  }
  float XY[2];
  int in = 0, maybe = 0;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const int bb = 2 * (lane & 3) + j;
    const float py = dyf + (((float)bb + 0.5f) * 0.125f - 0.5f);
    XY[j] = Xa + py * py;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float S = XY[j] + Z[c];
      in += S < lo;
      maybe += S <= hi;
    }
  }
  if (__any_sync(0xffffffffu, in != maybe)) {
    dx = __shfl_sync(0xffffffffu, dx, L);
    dy = __shfl_sync(0xffffffffu, dy, L);
    dz = __shfl_sync(0xffffffffu, dz, L);
    r2 = __shfl_sync(0xffffffffu, r2, L);
    in = 0;
    for (int j = 0; j < 2; ++j) {
      const int bb = 2 * (lane & 3) + j;
      for (int c = 0; c < 8; ++c) {
        const float S = XY[j] + Z[c];
        if (S < lo) ++in;
        else if (S <= hi && sample_inside_fp64(dx, dy, dz, sample_offset(a, 8),
                                               sample_offset(bb, 8), sample_offset(c, 8), r2))
          ++in;
      }
    }
  }
  return __reduce_add_sync(0xffffffffu, in);
}

// 8^3 sampled counts of up to four cells at once, eight lanes per cell: lane
// a = lane & 7 of group g = lane >> 3 takes the sample plane x = a (64
// samples) of the group's cell, with the FP32 roundings of its offset d (dxf,
// dyf, dzf), of r^2 (r2f) and the certified band E of geom.cuh.  Each sample's
// D = ((px^2 - r2f) + py^2) + pz^2 in FP32 lies within E of the FP64
// definition's S - r^2 (three squares off by at most 2^-21 (r + 2.5)^2 each,
// three sums by 2^-24 (r + 2.5)^2 each, r2f by 2^-24 r^2), so D < -E is
// inside and D > E outside.  Returns the group's count in every lane of the
// group (the samples certainly inside), whether this lane's plane has a
// sample in the band (|D| <= E) and whether any lane of the group has one;
// such samples are decided afterwards by plane_band8.
__device__ __forceinline__ int group_count8(float dxf, float dyf, float dzf, float r2f, float E,
                                            bool* lane_band, bool* band) {
  const unsigned all = 0xffffffffu;
  const int a = threadIdx.x & 7;
  const float px = dxf + (((float)a + 0.5f) * 0.125f - 0.5f);
  const float Xr = px * px - r2f;
  float Z[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const float pz = dzf + (((float)c + 0.5f) * 0.125f - 0.5f);
    Z[c] = pz * pz;
  }
  int in = 0;
  float mn = 3.0e38f;
#pragma unroll
  for (int bb = 0; bb < 8; ++bb) {
    const float py = dyf + (((float)bb + 0.5f) * 0.125f - 0.5f);
    const float XY = Xr + py * py;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const float D = XY + Z[c];
      in += D < -E;
      mn = fminf(mn, fabsf(D));
    }
  }
  const unsigned bm = __ballot_sync(all, mn <= E);
  *lane_band = mn <= E;
  *band = ((bm >> (threadIdx.x & 24)) & 0xffu) != 0u;
  in += __shfl_xor_sync(all, in, 4);
  in += __shfl_xor_sync(all, in, 2);
  in += __shfl_xor_sync(all, in, 1);
  return in;
}

// offsets of a box cell whose coordinates are set: FP64 offsets from the
// centre (cell_offsets64, or cell_offsets with fp64) and their FP32 roundings
// (from the per-block tables when the box fits them), FP32 squared distance
__device__ __forceinline__ void cell_offsets64(const Box& b, bool tables,
                                               const double (*toff)[FILL_AXIS], CellHit& h) {
  if (tables) {
    h.dx = toff[0][h.kx - b.lo[0]];
    h.dy = toff[1][h.ky - b.lo[1]];
    h.dz = toff[2][h.kz - b.lo[2]];
  } else {
    h.dx = ((double)h.kx + 0.5) - b.xp[0];
    h.dy = ((double)h.ky + 0.5) - b.xp[1];
    h.dz = ((double)h.kz + 0.5) - b.xp[2];
  }
}
__device__ __forceinline__ void cell_offsets(const Box& b, bool tables, bool fp64,
                                             const double (*toff)[FILL_AXIS],
                                             const float (*toff32)[FILL_AXIS], CellHit& h) {
  if (tables) {
    const int i0 = h.kx - b.lo[0], i1 = h.ky - b.lo[1], i2 = h.kz - b.lo[2];
    if (fp64) {
      h.dx = toff[0][i0];
      h.dy = toff[1][i1];
      h.dz = toff[2][i2];
    }
    h.dxf = toff32[0][i0];
    h.dyf = toff32[1][i1];
    h.dzf = toff32[2][i2];
  } else {
    h.dx = ((double)h.kx + 0.5) - b.xp[0];
    h.dy = ((double)h.ky + 0.5) - b.xp[1];
    h.dz = ((double)h.kz + 0.5) - b.xp[2];
    h.dxf = (float)h.dx;
    h.dyf = (float)h.dy;
    h.dzf = (float)h.dz;
  }
  // FP32 squared distance of the inside test (its band is certified for
  // the components rounded from FP64 as well as for the box-local form)
  h.d2f = h.dxf * h.dxf + h.dyf * h.dyf + h.dzf * h.dzf;
  h.d2 = -1.0;  // formed where a decision needs it
}

// surrogate mode (reading I): 1 = inside by the margin (eps = 1), 2 = a
// partial cell next to a wall face (8^3 sampling), 0 = any other partial
// cell (the network)
__device__ __forceinline__ int net_class(const Grid& g, const Box& b, const CellHit& h) {
  if (b.has_in) {
    if (h.d2f < b.rin2f - b.E) return 1;
    if (h.d2f <= b.rin2f + b.E && h.dx * h.dx + h.dy * h.dy + h.dz * h.dz <= b.rin2) return 1;
  }
  return wall_cell(g, h.ix, h.iy, h.iz) ? 2 : 0;
}

// Slots of one particle's cells (one block per particle, over the list the
// mark pass wrote): claims a slot per cell, writes B (Eq. 16, from a table
// of the n^3 + 1 sampled values when eps is a count), and the particle's
// surface velocity at the cell centre (Eq. 20); the list entry becomes the
// slot index (and, for the FP32 path, the float offset from the centre).
// record formats of the slot records the fill pass writes
enum { REC_FP64 = 0, REC_FP32 = 1, REC_DF = 2 };

template <int NS, int REC>
__global__ void __launch_bounds__(FILL_THREADS, FILL_MIN_BLOCKS) fill_kernel(MapParams P) {
  __shared__ double s64[16];
  __shared__ float s32[16];
  __shared__ Box sbox;
  // per-axis offsets (k + 1/2) - x_p of the box columns, FP64 and their FP32
  // roundings, formed once per block
  __shared__ double toff[3][FILL_AXIS];
  __shared__ float toff32[3][FILL_AXIS];
  __shared__ df toffd[3][FILL_AXIS];  // double-float records: offsets as pairs
  __shared__ df sud[6];               // and the particle's u, omega
  __shared__ float suf[6];            // u, omega rounded to FP32 (FP32 records)
  const int p = blockIdx.x;
  load_box(P, p, &sbox);
  const double fr = P.p.fr[p];
  const bool tab = P.eps_mode == 0 && P.wtab != nullptr;
  const double* wtab = P.wtab;
  load_offsets(P.eps_n, s64, s32);  // ends with __syncthreads
  const Box& b = sbox;  // read from shared memory (a register copy spills)
  const bool tables = b.n[0] <= FILL_AXIS && b.n[1] <= FILL_AXIS && b.n[2] <= FILL_AXIS;
  if (tables) {
    for (int t = threadIdx.x; t < 3 * FILL_AXIS; t += FILL_THREADS) {
      const int a = t / FILL_AXIS, k = t - a * FILL_AXIS;
      // the axis is a run-time index: read the shared copy (a local copy
      // indexed at run time would live on the stack)
      if (k < sbox.n[a]) {
        const double d = ((double)(sbox.lo[a] + k) + 0.5) - sbox.xp[a];
        toff[a][k] = d;
        toff32[a][k] = (float)d;
        if (REC == REC_DF) toffd[a][k] = df(d);
      }
    }
  }
  if (threadIdx.x < 6) {
    const double v = threadIdx.x < 3 ? P.p.u[3 * p + threadIdx.x] : P.p.om[3 * p + threadIdx.x - 3];
    suf[threadIdx.x] = (float)v;
    if (REC == REC_DF) sud[threadIdx.x] = df(v);
  }
  __syncthreads();
  const double u0 = P.p.u[3 * p], u1 = P.p.u[3 * p + 1], u2 = P.p.u[3 * p + 2];
  const double o0 = P.p.om[3 * p], o1 = P.p.om[3 * p + 1], o2 = P.p.om[3 * p + 2];
  const float uf0 = suf[0], uf1 = suf[1], uf2 = suf[2];
  const float of0 = suf[3], of1 = suf[4], of2 = suf[5];
  const float* wtabf = reinterpret_cast<const float*>(wtab + WTAB);  // FP32 copy
  const df* wtabd = reinterpret_cast<const df*>(wtab + WTAB_DF);      // double-float copy
  const float rf = (float)b.r, rinvf = 1.0f / rf, frf = (float)fr;  // surrogate inputs
  const long long loff = P.list_off[p];
  const int cnt = P.list_cnt[p];
  // surrogate mode: the block's network cells, its worklist range and next free index
  __shared__ int net_cnt, net_base, net_next;
  // 8^3 sampling (and, in surrogate mode, shared partial cells): next free
  // item of the particle's 8^3 worklist
  __shared__ int wl_next;
  if constexpr (NS == 8) {
    if (threadIdx.x == 0) wl_next = 0;
    __syncthreads();
  }
  if constexpr (NS < 0) {
    // the particle's network cells (counted by the mark pass) get one
    // worklist range, reserved with one atomic (a counter shared by every
    // block would serialise)
    if (threadIdx.x == 0) {
      wl_next = 0;
      net_cnt = P.list_net[p];
      net_base = net_cnt ? atomicAdd(P.mlp_count, net_cnt) : 0;
      net_next = net_base;
    }
    __syncthreads();
  }
  // 8^3 sampling iterates whole warps (the worklist is appended to warp by
  // warp; lanes past the list idle); the other modes give each thread its
  // own cells
  const int lane = threadIdx.x & 31;
  // software pipeline over a thread's rounds: the list entry two rounds
  // ahead and the coverage words (base, mask, shared mask) of the next
  // round's cell are loaded before this round's cell is filled
  const int kfirst = NS == 8 ? (threadIdx.x & ~31) + lane : threadIdx.x;
  // box index -> coordinates with the box's origin and divisors in registers
  const int blo0 = b.lo[0], blo1 = b.lo[1], blo2 = b.lo[2];
  const int bn0 = b.n[0], bn01 = b.n[0] * b.n[1];
  const FastDiv bd0 = b.div_n0, bdxy = b.div_nxy;
  // the FP32 records of the surrogate form need the FP64 offsets only for
  // decisions inside the certified band and for wall cells
  constexpr bool lazy64 = NS < 0 && REC == REC_FP32;
  // the cell of box index t (coordinates in q) and its coverage words
  auto words_of = [&](int t, CellHit& q, long long& c, int& wbase, uint32_t& wmask,
                      uint32_t& wdup) {
    const int kz = (int)bdxy.div((unsigned)t);
    const int rem = t - kz * bn01;
    const int ky = (int)bd0.div((unsigned)rem);
    q.kx = blo0 + (rem - ky * bn0);
    q.ky = blo1 + ky;
    q.kz = blo2 + kz;
    q.ix = wrap1(q.kx, P.g.nx);
    q.iy = wrap1(q.ky, P.g.ny);
    q.iz = wrap1(q.kz, P.g.nz);
    c = padded_cell(P.g, q.ix, q.iy, q.iz);
    const long long w = c >> 5;
    wbase = P.cov.base[w];
    wmask = P.cov.mask[w];
    wdup = P.cov.dup[w];
  };
  int tb_next = 0, tb_next2 = 0;  // list entries of the next two rounds
  CellHit hn;                      // the next round's cell: coordinates,
  long long cell_next = 0;         // padded index
  int nbase = 0;                   // and coverage words
  uint32_t nmask = 0u, ndup = 0u;
  hn.kx = hn.ky = hn.kz = hn.ix = hn.iy = hn.iz = 0;
  if (kfirst < cnt) {
    tb_next = P.list[loff + kfirst];
    words_of(tb_next, hn, cell_next, nbase, nmask, ndup);
  }
  if (kfirst + FILL_THREADS < cnt) tb_next2 = P.list[loff + kfirst + FILL_THREADS];
  for (int k0 = NS == 8 ? (threadIdx.x & ~31) : threadIdx.x; k0 < cnt; k0 += FILL_THREADS) {
    const int k = NS == 8 ? k0 + lane : k0;
    bool ok = NS == 8 ? k < cnt : true;
    const int tb = tb_next;  // box index of the cell (the list entry before the fill)
    CellHit h = hn;
    long long cell = cell_next;
    const int cbase = nbase;
    const uint32_t cmask = nmask, cdup = ndup;
    tb_next = tb_next2;
    tb_next2 = k + 2 * FILL_THREADS < cnt ? P.list[loff + k + 2 * FILL_THREADS] : 0;
    if (k + FILL_THREADS < cnt) words_of(tb_next, hn, cell_next, nbase, nmask, ndup);
    if constexpr (NS == 8) {  // lanes past the list still take part in the ballot
      h.dx = h.dy = h.dz = 0.0;
      h.dxf = h.dyf = h.dzf = 0.f;
    }
    long long e = 0;
    int s = 0;
    bool shared = false;  // a second particle in reach of the cell
    if (ok) {
      cell_offsets(b, tables, !lazy64, toff, toff32, h);
      const uint32_t bit = 1u << (cell & 31);
      e = (long long)cbase + __popc(cmask & (bit - 1u));
      shared = (cdup & bit) != 0u;
      if (e >= P.s.cap) {
        P.list[loff + k] = 0;  // the step reports the slot overflow
        ok = false;
      } else {
        P.list[loff + k] = (int)e;
        // a cell of this particle alone takes slot 0; a shared cell claims
        // its slot on a particle count (2-bit fields, 16 per word, so that
        // the counters of a whole mapping stay in L2 for these atomics)
        if (shared) {
          const int sh = 2 * (int)(e & 15);
          s = (int)((atomicAdd(reinterpret_cast<unsigned*>(P.s.cnt) + (e >> 4), 1u << sh) >>
                     sh) &
                    3u);
        }
        if (s >= 2) {
          atomicOr(P.status, ST_SLOT_OVERFLOW);
          ok = false;
        } else {
          P.s.cell[e] = (int)cell;
          reinterpret_cast<int*>(&P.s.pid[e])[s] = p;
        }
      }
    }
    // 8^3 sampling: a cell whose samples all lie inside (centre closer than
    // r - 0.76) counts 512 and one whose samples all lie outside (farther
    // than r + 0.76) counts 0 without sampling, both certified in FP32; the
    // other cells go to the particle's worklist (B stays -1 until the count
    // pass writes it; without a worklist the finish pass samples them)
    int count8 = 512;
    bool pending = false;
    if constexpr (NS == 8) {
      if (ok && tab) {
        pending = true;
        if (h.d2f < b.in8f - b.E) {
          pending = false;
        } else if (h.d2f > b.out8f + b.E) {
          pending = false;
          count8 = 0;
        }
      }
      const unsigned pm = __ballot_sync(0xffffffffu, pending);
      if (pm && P.wl_X) {
        int first = 0;
        if (lane == 0) first = atomicAdd(&wl_next, __popc(pm));
        first = __shfl_sync(0xffffffffu, first, 0);
        if (pending) {
          const long long k2 = loff + first + __popc(pm & ((1u << lane) - 1u));
          P.wl_X[k2] = make_float4(h.dxf, h.dyf, h.dzf, __int_as_float(tb));
          P.wl_work[k2] = (int)(unsigned)(2 * e + s);
        }
      }
    }
    if (!ok) continue;
    double B;
    float Bf = 0.f;
    int cidx = -1;      // sampled count when B comes from the table
    bool want = false;  // surrogate mode: the cell goes to the network's worklist
    bool pend8 = false;  // surrogate mode: a shared partial cell for the 8^3 count pass
    if constexpr (NS < 0) {
      // surrogate mode (reading I): inside by the margin -> 1; a partial
      // cell next to a wall face -> 8^3 sampling; any other partial cell ->
      // the network (B stays -1 until the inference writes it)
      if (lazy64 && b.has_in && h.d2f >= b.rin2f - b.E && h.d2f <= b.rin2f + b.E)
        cell_offsets64(b, tables, toff, h);  // the inside test's FP64 decision
      const int cls = net_class(P.g, b, h);
      if (cls == 1) {
        B = 1.0;
        Bf = 1.f;
      } else if (cls == 2) {
        if (lazy64) cell_offsets64(b, tables, toff, h);
        const int c = supersample_count_n<8>(h.dx, h.dy, h.dz, b.r, h.dxf, h.dyf, h.dzf, b.r2f,
                                             b.E);
        B = weight((double)c * (1.0 / 512.0), P.tau, P.weighting);
        Bf = (float)B;
      } else {
        // a cell shared with another particle stays pending: 8^3 sampling
        // in the count pass (its worklist), else in the finish pass
        B = -1.0;
        Bf = -1.f;
        want = !shared;
        pend8 = shared;
      }
    } else if (NS == 8 && pending) {
      B = -1.0;
      Bf = -1.f;
    } else if (tab) {
      const int c = NS == 8 ? count8 : cell_count<NS>(P, b, h, s64, s32);
      cidx = c;
      if (REC == REC_FP32) Bf = __ldg(&wtabf[c]);
      else B = __ldg(&wtab[c]);
    } else if (REC == REC_FP32 && P.eps_mode == 1) {
      // linear approximation (Eqs. 25-26) for FP32 records: the inside test
      // as the FP64 definition (certified band), eps and B in FP32 (the
      // record's own precision; FP64 square roots are slow on this GPU)
      bool inside = false;
      if (b.has_in) {
        if (h.d2f < b.rin2f - b.E) inside = true;
        else if (h.d2f <= b.rin2f + b.E && h.dx * h.dx + h.dy * h.dy + h.dz * h.dz <= b.rin2)
          inside = true;
      }
      float ef = 1.f;
      if (!inside) {
        ef = (rf - sqrtf(h.d2f)) + frf;
        ef = ef < 0.f ? 0.f : (ef > 1.f ? 1.f : ef);
      }
      Bf = ef;
      if (P.weighting && ef != 0.f && ef != 1.f) {
        const float tm = (float)(P.tau - 0.5);
        Bf = ef * tm / ((1.f - ef) + tm);
      }
    } else {
      h.d2 = h.dx * h.dx + h.dy * h.dy + h.dz * h.dz;
      const double eps = cell_eps(P, b, h, fr, s64, s32);
      B = eps < 0.0 ? -1.0 : weight(eps, P.tau, P.weighting);
      Bf = (float)B;
    }
    const long long rec = s * P.s.cap + e;  // slot s's record: velocity and B
    if (REC == REC_FP32) {
      // the FP32 collision takes the surface velocity in FP32
      const float fx = h.dxf, fy = h.dyf, fz = h.dzf;
      static_cast<float4*>(P.s.V)[rec] =
          make_float4(uf0 + (of1 * fz - of2 * fy), uf1 + (of2 * fx - of0 * fz),
                      uf2 + (of0 * fy - of1 * fx), Bf);
    } else if (REC == REC_DF) {
      // the double-float form: surface velocity (Eq. 20) in double-float from
      // the pairs of the offsets and of u, omega; B from the table's pairs
      df dx, dy, dz;
      if (tables) {
        dx = toffd[0][h.kx - b.lo[0]];
        dy = toffd[1][h.ky - b.lo[1]];
        dz = toffd[2][h.kz - b.lo[2]];
      } else {
        dx = df(h.dx);
        dy = df(h.dy);
        dz = df(h.dz);
      }
      const df v0 = sud[0] + (sud[4] * dz - sud[5] * dy);
      const df v1 = sud[1] + (sud[5] * dx - sud[3] * dz);
      const df v2 = sud[2] + (sud[3] * dy - sud[4] * dx);
      const df w = cidx >= 0 ? wtabd[cidx] : df(B);
      float4* R = static_cast<float4*>(P.s.V) + 2 * rec;
      R[0] = make_float4(v0.hi, v0.lo, v1.hi, v1.lo);
      R[1] = make_float4(v2.hi, v2.lo, w.hi, w.lo);
    } else {
      // Eq. 20 with one fused multiply-add per component (FP64 runs at 1/64
      // of the FP32 rate)
      const double v0 = u0 + __fma_rn(o1, h.dz, -(o2 * h.dy));
      const double v1 = u1 + __fma_rn(o2, h.dx, -(o0 * h.dz));
      const double v2 = u2 + __fma_rn(o0, h.dy, -(o1 * h.dx));
      double2* R = static_cast<double2*>(P.s.V) + 2 * rec;
      R[0] = make_double2(v0, v1);
      R[1] = make_double2(v2, B);
    }
    if constexpr (NS < 0) {
      // shared partial cells: the particle's 8^3 worklist (FP32 offset and
      // box index; 2 * entry + slot), counted by the count pass
      if (P.wl_X) {
        const unsigned grp8 = __activemask();
        const unsigned pm = __ballot_sync(grp8, pend8);
        if (pend8) {
          const int lane = threadIdx.x & 31;
          const int leader = __ffs(pm) - 1;
          int first = 0;
          if (lane == leader) first = atomicAdd(&wl_next, __popc(pm));
          first = __shfl_sync(pm, first, leader);
          const long long k2 = loff + first + __popc(pm & ((1u << lane) - 1u));
          P.wl_X[k2] = make_float4(h.dxf, h.dyf, h.dzf, __int_as_float(tb));
          P.wl_work[k2] = (int)(unsigned)(2 * e + s);
        }
      }
      // worklist append within the block's range, one shared-memory atomic
      // per group of converged lanes: the
      // network's inputs (|d/r| components in decreasing order, r), the
      // linear approximation of Eqs. 25-27, and 2 * entry + slot.  Items
      // beyond the particle's range or the worklist's capacity keep B = -1
      // (8^3 sampling later).
      const unsigned grp = __activemask();
      const unsigned wm = __ballot_sync(grp, want);
      if (want) {
        const int lane = threadIdx.x & 31;
        const int leader = __ffs(wm) - 1;
        int first = 0;
        if (lane == leader) first = atomicAdd(&net_next, __popc(wm));
        first = __shfl_sync(wm, first, leader);
        const long long k = (long long)first + __popc(wm & ((1u << lane) - 1u));
        if (k < (long long)net_base + net_cnt && k < P.mlp_cap) {
          float a0 = fabsf(h.dxf) * rinvf, a1 = fabsf(h.dyf) * rinvf, a2 = fabsf(h.dzf) * rinvf;
          float t;
          if (a1 > a0) { t = a0; a0 = a1; a1 = t; }
          if (a2 > a0) { t = a0; a0 = a2; a2 = t; }
          if (a2 > a1) { t = a1; a1 = a2; a2 = t; }
          reinterpret_cast<float4*>(P.mlp_X)[k] = make_float4(a0, a1, a2, rf);
          const float lin = (rf - sqrtf(h.d2f)) + frf;
          P.mlp_lin[k] = lin < 0.f ? 0.f : (lin > 1.f ? 1.f : lin);
          P.mlp_work[k] = (int)(2 * e + s);
        }
      }
    }
  }
  if constexpr (NS == 8 || NS < 0) {
    __syncthreads();
    if (threadIdx.x == 0 && P.wl_cnt) P.wl_cnt[p] = wl_next;
  }
  if constexpr (NS < 0) {
    // cells counted but not listed (slot overflow) leave empty items
    __syncthreads();
    const long long end = (long long)net_base + net_cnt;
    for (long long k = net_next + threadIdx.x; k < end && k < P.mlp_cap; k += FILL_THREADS) {
      reinterpret_cast<float4*>(P.mlp_X)[k] = make_float4(0.f, 0.f, 0.f, 0.f);
      P.mlp_lin[k] = 0.f;
      P.mlp_work[k] = -1;
    }
  }
}

// the samples of plane a of a cell that lie in the band (|D| <= E, the same
// FP32 D as group_count8), decided by the FP64 definition; the cell's FP64
// offset from its box index t (box coordinates unwrapped around the centre,
// ((double)k + 1/2) - x_p, as the fill pass forms it).  Returns the number
// of those inside.
__device__ int plane_band8(float dxf, float dyf, float dzf, float r2f, float E, int a, int t,
                           const Box& b) {
  const int nxy = b.n[0] * b.n[1];
  const int kz = (int)b.div_nxy.div((unsigned)t);
  const int rem = t - kz * nxy;
  const int ky = (int)b.div_n0.div((unsigned)rem);
  const int kx = rem - ky * b.n[0];
  const double dx = ((double)(b.lo[0] + kx) + 0.5) - b.xp[0];
  const double dy = ((double)(b.lo[1] + ky) + 0.5) - b.xp[1];
  const double dz = ((double)(b.lo[2] + kz) + 0.5) - b.xp[2];
  const double r2 = b.r * b.r;
  const float px = dxf + (((float)a + 0.5f) * 0.125f - 0.5f);
  const float Xr = px * px - r2f;
  int in = 0;
  for (int bb = 0; bb < 8; ++bb) {
    const float py = dyf + (((float)bb + 0.5f) * 0.125f - 0.5f);
    const float XY = Xr + py * py;
    for (int c = 0; c < 8; ++c) {
      const float pz = dzf + (((float)c + 0.5f) * 0.125f - 0.5f);
      const float D = XY + pz * pz;
      if (fabsf(D) <= E && sample_inside_fp64(dx, dy, dz, sample_offset(a, 8),
                                                sample_offset(bb, 8), sample_offset(c, 8), r2))
        ++in;
    }
  }
  return in;
}

// B of a count from the table into slot sl of entry e
template <int REC>
__device__ __forceinline__ void write_count_weight(const MapParams& P, unsigned e, unsigned sl,
                                                   int c) {
  const long long rec = (long long)sl * P.s.cap + e;
  if (REC == REC_FP32) {
    reinterpret_cast<float*>(P.s.V)[4 * rec + 3] =
        __ldg(reinterpret_cast<const float*>(P.wtab + WTAB) + c);
  } else if (REC == REC_DF) {
    const df w = reinterpret_cast<const df*>(P.wtab + WTAB_DF)[c];
    float* R = reinterpret_cast<float*>(P.s.V) + 8 * rec;
    R[6] = w.hi;
    R[7] = w.lo;
  } else {
    reinterpret_cast<double*>(P.s.V)[4 * rec + 3] = __ldg(P.wtab + c);
  }
}

// 8^3 counts of the cells the fill pass listed (one block per particle, four
// cells per warp and round, eight lanes per cell): B of each count from the
// table into the slot record's weight.  A cell with samples in the certified
// band (about one in eighty) is queued with its certain count, and after the
// rounds each queued plane is finished by one thread (plane_band8), so that
// the rounds never wait on the FP64 definition; cells beyond the queue keep
// the fill pass's B = -1 and the finish pass samples them.
constexpr int CQ_ITEMS = 128, CQ_PLANES = 256;
constexpr int COUNT_THREADS = 128;
template <int REC>
__global__ void __launch_bounds__(COUNT_THREADS, 6) count8_kernel(MapParams P) {
  __shared__ Box sbox;
  __shared__ int q_items, q_planes;
  __shared__ int q_item[CQ_ITEMS], q_cnt[CQ_ITEMS], q_plane[CQ_PLANES];
  const int p = blockIdx.x;
  const int n = P.wl_cnt[p];
  if (n == 0) return;  // the whole block
  if (threadIdx.x == 0) {
    q_items = 0;
    q_planes = 0;
  }
  load_box(P, p, &sbox);  // ends with __syncthreads
  const long long base = P.list_off[p];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, g = lane >> 3;
  const float r2f = sbox.r2f, E = sbox.E;
  // each round's items are loaded one round ahead
  constexpr int STEP = 4 * (COUNT_THREADS / 32);
  float4 Xn = make_float4(0.f, 0.f, 0.f, 0.f);
  unsigned wkn = 0u;
  if (4 * warp < n) {
    const long long it = base + (4 * warp + g < n ? 4 * warp + g : 4 * warp);
    Xn = P.wl_X[it];
    wkn = (unsigned)P.wl_work[it];
  }
  for (int i0 = 4 * warp; i0 < n; i0 += STEP) {  // warp-uniform
    const int i = i0 + g;
    const bool valid = i < n;
    const float4 X = Xn;
    const unsigned wk = wkn;
    if (i0 + STEP < n) {
      const int i2 = i0 + STEP + g;
      const long long it = base + (i2 < n ? i2 : i0 + STEP);
      Xn = P.wl_X[it];
      wkn = (unsigned)P.wl_work[it];
    }
    const unsigned e = wk >> 1, sl = wk & 1u;
    bool lane_band, band;
    const int c = group_count8(X.x, X.y, X.z, r2f, E, &lane_band, &band);
    if (valid && (lane & 7) == 0 && !band) write_count_weight<REC>(P, e, sl, c);
    if (__any_sync(0xffffffffu, valid && band)) {
      // queue the cell with its certain count, then its planes with band samples
      int j = -1;
      if (valid && band && (lane & 7) == 0) {
        j = atomicAdd(&q_items, 1);
        if (j < CQ_ITEMS) {
          q_item[j] = i;
          q_cnt[j] = c;
        }
      }
      j = __shfl_sync(0xffffffffu, j, lane & 24);
      __syncwarp();  // the leaders' entries before the planes' updates
      if (valid && band && lane_band && j >= 0 && j < CQ_ITEMS) {
        const int k = atomicAdd(&q_planes, 1);
        if (k < CQ_PLANES) q_plane[k] = (j << 3) | (lane & 7);
        else atomicOr(&q_cnt[j], (int)0x80000000);  // left to the finish pass
      }
    }
  }
  __syncthreads();
  const int np = min(q_planes, CQ_PLANES), ni = min(q_items, CQ_ITEMS);
  for (int k = threadIdx.x; k < np; k += COUNT_THREADS) {
    const int j = q_plane[k] >> 3, a = q_plane[k] & 7;
    const float4 X = P.wl_X[base + q_item[j]];
    const int add = plane_band8(X.x, X.y, X.z, r2f, E, a, __float_as_int(X.w), sbox);
    if (add) atomicAdd(&q_cnt[j], add);
  }
  __syncthreads();
  for (int j = threadIdx.x; j < ni; j += COUNT_THREADS) {
    const int cnt = q_cnt[j];
    if (cnt < 0) continue;  // a plane did not fit the queue: B stays -1
    const unsigned wk = (unsigned)P.wl_work[base + q_item[j]];
    write_count_weight<REC>(P, wk >> 1, wk & 1u, cnt);
  }
}

// one slot entry of the finish pass in the storage precision T: order the
// two slots by particle index, sample cells left pending with 8^3 points,
// normalise B > 1 (Sec. 2.3), flag a second particle in the sign of slot 0's
// weight; returns min(B, 1)
__device__ __forceinline__ void rec_load(const float* p, float* o) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void rec_load(const double* p, double* o) {
  const double2 u = reinterpret_cast<const double2*>(p)[0];
  const double2 v = reinterpret_cast<const double2*>(p)[1];
  o[0] = u.x; o[1] = u.y; o[2] = v.x; o[3] = v.y;
}
__device__ __forceinline__ void rec_store(float* p, const float* o) {
  *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
}
// double-float records: the finish pass only moves the velocity pairs (their
// 8 bytes travel as the bits of a double) and computes with the weight
__device__ __forceinline__ void rec_load(const df* p, double* o) {
  const double2 u = reinterpret_cast<const double2*>(p)[0];
  const float4 v = reinterpret_cast<const float4*>(p)[1];
  o[0] = u.x;
  o[1] = u.y;
  o[2] = __longlong_as_double((long long)(((unsigned long long)__float_as_uint(v.y) << 32) |
                                          __float_as_uint(v.x)));
  o[3] = to_double(df(v.z, v.w));
}
__device__ __forceinline__ void rec_store(df* p, const double* o) {
  const df w(o[3]);
  const unsigned long long b2 = (unsigned long long)__double_as_longlong(o[2]);
  reinterpret_cast<double2*>(p)[0] = make_double2(o[0], o[1]);
  reinterpret_cast<float4*>(p)[1] =
      make_float4(__uint_as_float((unsigned)b2), __uint_as_float((unsigned)(b2 >> 32)), w.hi,
                  w.lo);
}
__device__ __forceinline__ void rec_store(double* p, const double* o) {
  reinterpret_cast<double2*>(p)[0] = make_double2(o[0], o[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(o[2], o[3]);
}

// weights of the slots left pending (B < 0: cells of two particles in
// surrogate mode, worklist overflow, no network set) by 8^3 sampling, one
// warp-wide count per pending slot; pend/pend1: lanes with slot 0 / slot 1
// pending (every lane of the warp calls this together)
template <typename T>
struct WeightPair {
  T b0, b1;
};
// the FP64 set-up of one pending slot's count, in the lane that owns it
struct PendingPrep {
  double dx, dy, dz, r2;
  float f[5];  // FP32 roundings of dx, dy, dz, r^2 and the certified band
};
__device__ __forceinline__ PendingPrep pending_prep(const MapParams& P, int cell, int p) {
  PendingPrep q;
  int x, y, z;
  cell_xyz(P.g, cell, x, y, z);
  const double r = P.p.r[p];
  q.dx = image_d(x, P.p.x[3 * p], P.g.nx, !P.g.wall[0]);
  q.dy = image_d(y, P.p.x[3 * p + 1], P.g.ny, !P.g.wall[1]);
  q.dz = image_d(z, P.p.x[3 * p + 2], P.g.nz, !P.g.wall[2]);
  q.r2 = r * r;
  q.f[0] = (float)q.dx;
  q.f[1] = (float)q.dy;
  q.f[2] = (float)q.dz;
  q.f[3] = (float)q.r2;
  q.f[4] = certified_band(r);
  return q;
}

template <typename T>
__device__ __noinline__ WeightPair<T> pending_weights(const MapParams& P, int e, int2 pid,
                                                      unsigned pend, unsigned pend1, T B0, T B1) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  // every pending lane forms its FP64 set-up at once (an FP64 instruction
  // costs a warp the same for one lane as for 32)
  PendingPrep q0{}, q1{};
  const int cell = (((pend | pend1) >> lane) & 1u) ? P.s.cell[e] : 0;
  if ((pend >> lane) & 1u) q0 = pending_prep(P, cell, pid.x);
  if ((pend1 >> lane) & 1u) q1 = pending_prep(P, cell, pid.y);
  while (pend | pend1) {
    const bool s1 = pend == 0u;
    const int L = __ffs(s1 ? pend1 : pend) - 1;
    if (s1) pend1 &= pend1 - 1u; else pend &= pend - 1u;
    const PendingPrep& q = s1 ? q1 : q0;
    float f[5];
#pragma unroll
    for (int i = 0; i < 5; ++i) f[i] = __shfl_sync(full, q.f[i], L);
    const int cnt = warp_count8(f[0], f[1], f[2], f[3], f[4], L, q.dx, q.dy, q.dz, q.r2);
    if (lane == L) {
      // B of the count: from the context's table when it holds the 8^3 counts
      const bool tab8 = P.wtab != nullptr && P.eps_n == 8;
      const T B = tab8 ? (sizeof(T) == 4 ? (T)reinterpret_cast<const float*>(P.wtab + WTAB)[cnt]
                                         : (T)P.wtab[cnt])
                       : (T)weight((double)cnt * (1.0 / 512.0), P.tau, P.weighting);
      if (s1) B1 = B; else B0 = B;
    }
  }
  return WeightPair<T>{B0, B1};
}

// one slot entry of the finish pass in the storage precision T, taken by a
// whole warp (lanes with e >= n take part in the sampling only): order the two
// slots by particle index, sample the slots left pending (B < 0: cells of two
// particles in surrogate mode, worklist overflow, no network) with 8^3 points,
// normalise B > 1 (Sec. 2.3), flag a second particle in the sign of slot 0's
// weight; returns min(B, 1) (0 for lanes without an entry)
// pid and r0: the entry's particle pair and slot-0 record, loaded by the
// caller a round ahead
template <typename T, typename S>  // arithmetic in T, records stored as S
__device__ double finish_entry(const MapParams& P, int e, int n, int2 pid, const T* pre,
                               bool* full) {
  const bool live = e < n;
  T r0[4] = {pre[0], pre[1], pre[2], pre[3]}, r1[4] = {T(0), T(0), T(0), T(0)};
  S* V = static_cast<S*>(P.s.V);
  const long long e1 = P.s.cap + e;
  bool two = false;
  if (live) {
    two = pid.y >= 0;
    if (two) rec_load(V + 4 * e1, r1);
    if (two && pid.y < pid.x) {
      const int t = pid.x;
      pid.x = pid.y;
      pid.y = t;
      for (int a = 0; a < 4; ++a) {
        const T v = r0[a];
        r0[a] = r1[a];
        r1[a] = v;
      }
    }
  }
  // pending slots, one warp-wide count each (out of line: rare, and its
  // registers should not weigh on the common path)
  const unsigned pend = __ballot_sync(0xffffffffu, live && r0[3] < T(0));
  const unsigned pend1 = __ballot_sync(0xffffffffu, live && two && r1[3] < T(0));
  if (pend | pend1) {
    const WeightPair<T> w = pending_weights<T>(P, e, pid, pend, pend1, r0[3], r1[3]);
    r0[3] = w.b0;
    r1[3] = w.b1;
  }
  if (!live) return 0.0;
  T B = r0[3] + r1[3];
  if (B > T(1)) {
    r0[3] = r0[3] / B;
    r1[3] = r1[3] / B;
    B = T(1);
  }
  r0[3] = two ? -r0[3] : r0[3];
  // a cell of one particle whose weight was not pending is unchanged (its B
  // is at most 1 and keeps its sign): no store
  if (two || ((pend >> (threadIdx.x & 31)) & 1u)) rec_store(V + 4 * e, r0);
  if (two) {
    P.s.pid[e] = pid;
    rec_store(V + 4 * e1, r1);
  }
  *full = !two && r0[3] == T(1);
  return (double)B;
}

// the full-cell mask (one particle, B = 1: the FP64 collision takes these
// cells in warps of their own, where the fluid change vanishes): the warp's
// entries are consecutive slots, hence cells in increasing order; a
// segmented OR over lanes of the same mask word leaves one atomicOr per run
__device__ __forceinline__ void mark_full(const MapParams& P, int e, bool fl) {
  const unsigned all = 0xffffffffu;
  if (!__any_sync(all, fl)) return;
  const int lane = threadIdx.x & 31;
  const int cell = fl ? P.s.cell[e] : 0;
  const int w = fl ? cell >> 5 : -1;
  unsigned v = fl ? 1u << (cell & 31) : 0u;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const unsigned vu = __shfl_up_sync(all, v, off);
    const int wu = __shfl_up_sync(all, w, off);
    if (lane >= off && wu == w) v |= vu;
  }
  const int wn = __shfl_down_sync(all, w, 1);
  if (fl && (lane == 31 || wn != w)) atomicOr(P.cov.full + w, v);
}

// one instance per record format (REC_*), so that each carries only its own
// path's registers
template <int REC> struct RecTypes { using T = double; using S = double; };
template <> struct RecTypes<REC_FP32> { using T = float; using S = float; };
template <> struct RecTypes<REC_DF> { using T = double; using S = df; };

template <int REC>
__global__ void __launch_bounds__(256, 3) finish_kernel(MapParams P) {
  using T = typename RecTypes<REC>::T;
  using S = typename RecTypes<REC>::S;
  __shared__ double red[256];
  const int n = slot_count(P);
  const S* V = static_cast<const S*>(P.s.V);
  double accB = 0.0;
  // warp-uniform loop: every lane of a warp runs the same iterations; the
  // next round's particle pair and slot-0 record are loaded a round ahead
  const int stride = gridDim.x * blockDim.x;
  const int efirst = blockIdx.x * blockDim.x + threadIdx.x;
  int2 pid_n = make_int2(-1, -1);
  T rec_n[4] = {T(0), T(0), T(0), T(0)};
  if (efirst < n) {
    pid_n = P.s.pid[efirst];
    rec_load(V + 4 * (long long)efirst, rec_n);
  }
  for (int e0 = blockIdx.x * blockDim.x + (threadIdx.x & ~31); e0 < n; e0 += stride) {
    const int e = e0 + (threadIdx.x & 31);
    const int2 pid = pid_n;
    const T r0[4] = {rec_n[0], rec_n[1], rec_n[2], rec_n[3]};
    if (e + stride < n) {
      pid_n = P.s.pid[e + stride];
      rec_load(V + 4 * (long long)(e + stride), rec_n);
    }
    bool fl = false;
    accB += finish_entry<T, S>(P, e, n, pid, r0, &fl);
    if (REC == REC_FP64 && P.cov.full) mark_full(P, e, fl);
  }
  red[threadIdx.x] = accB;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) P.partials[blockIdx.x] = red[0];
}

// fluid volume sum_x (1 - B) from the finish-pass partial sums, fixed order:
// each thread sums a strided subset, then a tree (one block of 256)
__global__ void vfluid_kernel(MapParams P, int nparts) {
  __shared__ double red[256];
  double s = 0.0;
  for (int b = threadIdx.x; b < nparts; b += 256) s += P.partials[b];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = 128; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    P.sc->sumB = red[0];
    P.sc->vfluid = P.sc->ncells - red[0];
  }
}

// ---- fixed-order force and torque reduction over each particle's list
//
// The torque arm of a cell is its nearest-image offset from the centre,
// (k - i_p) + (1/2 - frac(x_p)) per axis: an integer part that varies per
// cell plus a fraction that is the same for every cell of the particle.  So
// T = sum (k - i_p) x F_c + (1/2 - frac) x F, and each entry costs the three
// force sums and two fused multiply-adds per torque component (FP64 runs at
// 1/64 of the FP32 rate on GB300).

// Sum of six values over the 32 lanes of a warp in a fixed order, halving the
// values each lane carries at the first levels: 8 additions per lane instead
// of 30.  Returns the total of value i in the lanes with (lane & 3) == 0 and
// lane >> 2 = 4 (i / 3) + (i % 3) (lanes whose index maps to 3 or 7 carry an
// empty slot).
__device__ __forceinline__ double warp_sum6(const double (&v)[6], int lane, int& which) {
  const bool b4 = (lane >> 4) & 1, b3 = (lane >> 3) & 1, b2 = (lane >> 2) & 1;
  double w[4];
#pragma unroll
  for (int i = 0; i < 3; ++i) {  // lanes 0-15 keep values 0-2, lanes 16-31 values 3-5
    const double keep = b4 ? v[i + 3] : v[i];
    const double send = b4 ? v[i] : v[i + 3];
    w[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  w[3] = 0.0;
  double u[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) {  // then pairs {0,1} / {2,3}
    const double keep = b3 ? w[i + 2] : w[i];
    const double send = b3 ? w[i] : w[i + 2];
    u[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  {
    const double keep = b2 ? u[1] : u[0];
    const double send = b2 ? u[0] : u[1];
    u[0] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  u[0] += __shfl_xor_sync(0xffffffffu, u[0], 2);
  u[0] += __shfl_xor_sync(0xffffffffu, u[0], 1);
  const int j = 2 * b3 + b2;
  which = j < 3 ? 3 * b4 + j : -1;
  return u[0];
}

// A thread's walk over a particle's list entries k = threadIdx.x,
// + RED_THREADS, ... with the list entries loaded two rounds ahead and the
// next round's particle pair and cell one round ahead (the same entries in
// the same order as a plain loop, so the sums are unchanged).
struct ListWalk {
  const MapParams& P;
  long long loff;
  int cnt;
  int e1, e2;  // list entries of the next two rounds
  int2 pid1;   // the next round's particle pair and padded cell
  int cell1;
  __device__ __forceinline__ ListWalk(const MapParams& P_, long long loff_, int cnt_)
      : P(P_), loff(loff_), cnt(cnt_), e1(0), e2(0), pid1(make_int2(-1, -1)), cell1(0) {
    const int k = threadIdx.x;
    if (k < cnt) {
      e1 = P.list[loff + k];
      pid1 = P.s.pid[e1];
      cell1 = P.s.cell[e1];
    }
    if (k + RED_THREADS < cnt) e2 = P.list[loff + k + RED_THREADS];
  }
  // entry k's slot entry, particle pair and cell; loads ahead for k + 1, k + 2 rounds
  __device__ __forceinline__ void next(int k, int& e, int2& pid, int& cell) {
    e = e1;
    pid = pid1;
    cell = cell1;
    e1 = e2;
    if (k + 2 * RED_THREADS < cnt) e2 = P.list[loff + k + 2 * RED_THREADS];
    if (k + RED_THREADS < cnt) {
      pid1 = P.s.pid[e1];
      cell1 = P.s.cell[e1];
    }
  }
};

template <typename T>
__global__ void __launch_bounds__(RED_THREADS) force_reduce_kernel(MapParams P) {
  __shared__ double sh[6][RED_THREADS / 32];
  __shared__ int sip[3];
  __shared__ double sfr[3];
  const int p = blockIdx.x;
  const T* Fc = static_cast<const T*>(P.s.Fc);
  const long long loff = P.list_off[p];
  const int cnt = P.list_cnt[p];
  if (threadIdx.x < 3) {  // centre = integer part + (1/2 - fraction), once per block
    const double xp = P.p.x[3 * p + threadIdx.x];
    const double fl = floor(xp);
    sip[threadIdx.x] = (int)fl;
    sfr[threadIdx.x] = 0.5 - (xp - fl);
  }
  __syncthreads();
  const int dims[3] = {P.g.nx, P.g.ny, P.g.nz};
  // F, then sum over cells of (k - i_p) x F_c
  double acc[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
  ListWalk walk(P, loff, cnt);
  for (int k = threadIdx.x; k < cnt; k += RED_THREADS) {
    int e, cell;
    int2 pid;
    walk.next(k, e, pid, cell);
    const int s = pid.x == p ? 0 : (pid.y == p ? 1 : -1);
    if (s < 0) continue;
    int c3[3];
    cell_xyz(P.g, cell, c3[0], c3[1], c3[2]);
    double kd[3];
    for (int a = 0; a < 3; ++a) {  // nearest image of the integer offset
      int k0 = c3[a] - sip[a];
      if (!P.g.wall[a]) {
        if (2 * k0 > dims[a]) k0 -= dims[a];
        else if (2 * k0 < -dims[a]) k0 += dims[a];
      }
      kd[a] = (double)k0;
    }
    const long long fo = 3 * (s * P.s.cap + e);
    const double f0 = (double)Fc[fo];
    const double f1 = (double)Fc[fo + 1];
    const double f2 = (double)Fc[fo + 2];
    acc[0] += f0;
    acc[1] += f1;
    acc[2] += f2;
    acc[3] = fma(-kd[2], f1, fma(kd[1], f2, acc[3]));
    acc[4] = fma(-kd[0], f2, fma(kd[2], f0, acc[4]));
    acc[5] = fma(-kd[1], f0, fma(kd[0], f1, acc[5]));
  }
  // fixed-order tree: within each warp by shuffles, then over the warps
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int which;
  const double ws = warp_sum6(acc, lane, which);
  if ((lane & 3) == 0 && which >= 0) sh[which][wid] = ws;
  __syncthreads();
  if (threadIdx.x < 6) {
    const int i = threadIdx.x;
    double t = sh[i][0];
    for (int w = 1; w < RED_THREADS / 32; ++w) t += sh[i][w];
    sh[i][0] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double F[3] = {sh[0][0], sh[1][0], sh[2][0]};
    const double Tq[3] = {sh[3][0] + (sfr[1] * F[2] - sfr[2] * F[1]),
                          sh[4][0] + (sfr[2] * F[0] - sfr[0] * F[2]),
                          sh[5][0] + (sfr[0] * F[1] - sfr[1] * F[0])};
    bool finite = true;
    for (int i = 0; i < 3; ++i) {
      P.p.Fh[3 * p + i] = F[i];
      P.p.Th[3 * p + i] = Tq[i];
      finite = finite && isfinite(F[i]) && isfinite(Tq[i]);
    }
    if (!finite) atomicOr(P.status, ST_NONFINITE);
  }
}

// FP32 path: per-slot contributions are FP32, and so are the torque arms
// (formed from the cell index and the centre's integer and fractional
// parts); every component is summed with an error-free two-sum (a float pair
// carrying about 48 bits), across the block by shuffles in a fixed order, and
// converted to FP64 once.  No FP64 arithmetic per entry: GB300 runs FP64 at
// 1/64 of the FP32 rate.
struct FloatPair {
  float hi, lo;
  __device__ __forceinline__ void add(float x) {
    const float t = hi + x;
    const float bb = t - hi;
    const float err = (hi - (t - bb)) + (x - bb);
    hi = t;
    lo += err;
  }
  // merges another pair: its high part through the two-sum, its low part
  // into the low word
  __device__ __forceinline__ void merge(const FloatPair& o) {
    add(o.hi);
    lo += o.lo;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

__global__ void __launch_bounds__(RED_THREADS) force_reduce_f32_kernel(MapParams P) {
  __shared__ FloatPair sh[6][RED_THREADS / 32];
  __shared__ int sip[3];
  __shared__ float sfp[3];
  const int p = blockIdx.x;
  const float* Fc = static_cast<const float*>(P.s.Fc);
  const long long loff = P.list_off[p];
  const int cnt = P.list_cnt[p];
  if (threadIdx.x < 3) {  // centre = floor + fraction, once per block in FP64
    const double xp = P.p.x[3 * p + threadIdx.x];
    const double fl = floor(xp);
    sip[threadIdx.x] = (int)fl;
    sfp[threadIdx.x] = (float)(xp - fl);
  }
  __syncthreads();
  const int dims[3] = {P.g.nx, P.g.ny, P.g.nz};
  FloatPair acc[6];
  for (int i = 0; i < 6; ++i) acc[i] = FloatPair{0.f, 0.f};
  ListWalk walk(P, loff, cnt);
  for (int k = threadIdx.x; k < cnt; k += RED_THREADS) {
    int e, cell;
    int2 pid;
    walk.next(k, e, pid, cell);
    // torque arm: the cell centre's nearest-image offset, in FP32 from the
    // integer and fractional parts of the centre
    int c3[3];
    cell_xyz(P.g, cell, c3[0], c3[1], c3[2]);
    float d3[3];
    for (int a = 0; a < 3; ++a) {
      int k0 = c3[a] - sip[a];
      if (!P.g.wall[a]) {
        if (2 * k0 > dims[a]) k0 -= dims[a];
        else if (2 * k0 < -dims[a]) k0 += dims[a];
      }
      d3[a] = (float)k0 + (0.5f - sfp[a]);
    }
    const float4 d = make_float4(d3[0], d3[1], d3[2], 0.f);
    const int s = pid.x == p ? 0 : (pid.y == p ? 1 : -1);
    if (s < 0) continue;
    const long long fo = 3 * (s * P.s.cap + e);
    const float f0 = Fc[fo];
    const float f1 = Fc[fo + 1];
    const float f2 = Fc[fo + 2];
    acc[0].add(f0);
    acc[1].add(f1);
    acc[2].add(f2);
    acc[3].add(d.y * f2 - d.z * f1);
    acc[4].add(d.z * f0 - d.x * f2);
    acc[5].add(d.x * f1 - d.y * f0);
  }
  // fixed-order tree of the pairs: within each warp by shuffles, then over
  // the warps; one conversion to FP64 per component at the end
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1)
    for (int i = 0; i < 6; ++i) {
      FloatPair q;
      q.hi = __shfl_down_sync(0xffffffffu, acc[i].hi, o);
      q.lo = __shfl_down_sync(0xffffffffu, acc[i].lo, o);
      acc[i].merge(q);
    }
  if (lane == 0)
    for (int i = 0; i < 6; ++i) sh[i][wid] = acc[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot[6];
    for (int i = 0; i < 6; ++i) {
      FloatPair t = sh[i][0];
      for (int w = 1; w < RED_THREADS / 32; ++w) t.merge(sh[i][w]);
      tot[i] = t.value();
    }
    bool finite = true;
    for (int i = 0; i < 3; ++i) {
      P.p.Fh[3 * p + i] = tot[i];
      P.p.Th[3 * p + i] = tot[3 + i];
      finite = finite && isfinite(tot[i]) && isfinite(tot[3 + i]);
    }
    if (!finite) atomicOr(P.status, ST_NONFINITE);
  }
}

// The same reduction for the double-float form: slot forces arrive as FP32
// pairs, torque arms are formed as (integer offset) + (1/2 - fraction of the
// centre) in double-float, products and sums in double-float on the FP32
// pipes (df.cuh), the same fixed-order tree, one conversion to FP64 per
// component at the end.
__global__ void __launch_bounds__(RED_THREADS) force_reduce_df_kernel(MapParams P) {
  __shared__ df sh[6][RED_THREADS / 32];
  __shared__ int sip[3];
  __shared__ df sfr[3];
  const int p = blockIdx.x;
  const df* Fc = static_cast<const df*>(P.s.Fc);
  const long long loff = P.list_off[p];
  const int cnt = P.list_cnt[p];
  if (threadIdx.x < 3) {  // centre = integer part + (1/2 - fraction), once per block
    const double xp = P.p.x[3 * p + threadIdx.x];
    const double fl = floor(xp);
    sip[threadIdx.x] = (int)fl;
    sfr[threadIdx.x] = df(0.5 - (xp - fl));
  }
  __syncthreads();
  const int dims[3] = {P.g.nx, P.g.ny, P.g.nz};
  df acc[6];
  for (int i = 0; i < 6; ++i) acc[i] = df(0.f, 0.f);
  ListWalk walk(P, loff, cnt);
  for (int k = threadIdx.x; k < cnt; k += RED_THREADS) {
    int e, cell;
    int2 pid;
    walk.next(k, e, pid, cell);
    const int s = pid.x == p ? 0 : (pid.y == p ? 1 : -1);
    if (s < 0) continue;
    int c3[3];
    cell_xyz(P.g, cell, c3[0], c3[1], c3[2]);
    df d3[3];
    for (int a = 0; a < 3; ++a) {
      int k0 = c3[a] - sip[a];
      if (!P.g.wall[a]) {
        if (2 * k0 > dims[a]) k0 -= dims[a];
        else if (2 * k0 < -dims[a]) k0 += dims[a];
      }
      d3[a] = df((float)k0, 0.f) + sfr[a];
    }
    const long long fo = 3 * (s * P.s.cap + e);
    const float2 u = reinterpret_cast<const float2*>(Fc)[fo];
    const float2 v = reinterpret_cast<const float2*>(Fc)[fo + 1];
    const float2 w = reinterpret_cast<const float2*>(Fc)[fo + 2];
    const df f0(u.x, u.y), f1(v.x, v.y), f2(w.x, w.y);
    acc[0] = renorm(acc[0] + f0);
    acc[1] = renorm(acc[1] + f1);
    acc[2] = renorm(acc[2] + f2);
    acc[3] = renorm(acc[3] + (d3[1] * f2 - d3[2] * f1));
    acc[4] = renorm(acc[4] + (d3[2] * f0 - d3[0] * f2));
    acc[5] = renorm(acc[5] + (d3[0] * f1 - d3[1] * f0));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1)
    for (int i = 0; i < 6; ++i) {
      const df q(__shfl_down_sync(0xffffffffu, acc[i].hi, o),
                 __shfl_down_sync(0xffffffffu, acc[i].lo, o));
      acc[i] = renorm(acc[i] + q);
    }
  if (lane == 0)
    for (int i = 0; i < 6; ++i) sh[i][wid] = acc[i];
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot[6];
    for (int i = 0; i < 6; ++i) {
      df t = sh[i][0];
      for (int w = 1; w < RED_THREADS / 32; ++w) t = renorm(t + sh[i][w]);
      tot[i] = to_double(t);
    }
    bool finite = true;
    for (int i = 0; i < 3; ++i) {
      P.p.Fh[3 * p + i] = tot[i];
      P.p.Th[3 * p + i] = tot[3 + i];
      finite = finite && isfinite(tot[i]) && isfinite(tot[3 + i]);
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
    int x, y, z;
    cell_xyz(P.g, P.s.cell[e], x, y, z);
    const long long c = (long long)x + (long long)P.g.nx * ((long long)y + (long long)P.g.ny * z);
    const int2 pid = P.s.pid[e];
    pid0[c] = pid.x;
    pid1[c] = pid.y;
    B0[c] = fabs(load_B(P, e, 0));
    B1[c] = pid.y >= 0 ? load_B(P, e, 1) : 0.0;
  }
}

// per-slot forces of the last collision (Eq. 21), in FP64, into dense
// per-cell arrays (3 per cell; zero where the slot is empty)
__global__ void dense_forces_kernel(MapParams P, int* pid0, int* pid1, double* F0, double* F1) {
  const int n = slot_count(P);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    int x, y, z;
    cell_xyz(P.g, P.s.cell[e], x, y, z);
    const long long c = (long long)x + (long long)P.g.nx * ((long long)y + (long long)P.g.ny * z);
    const int2 pid = P.s.pid[e];
    pid0[c] = pid.x;
    pid1[c] = pid.y;
    for (int sl = 0; sl < 2; ++sl) {
      if ((sl ? pid.y : pid.x) < 0) continue;
      const long long fo = 3 * ((long long)sl * P.s.cap + e);
      double* out = (sl ? F1 : F0) + 3 * c;
      for (int a = 0; a < 3; ++a) {
        if (P.fp32) out[a] = (double)static_cast<const float*>(P.s.Fc)[fo + a];
        else if (P.dfrec) out[a] = to_double(static_cast<const df*>(P.s.Fc)[fo + a]);
        else out[a] = static_cast<const double*>(P.s.Fc)[fo + a];
      }
    }
  }
}

unsigned grid_cap(long long n, int block) {
  long long b = (n + block - 1) / block;
  if (b > MAP_PARTIALS) b = MAP_PARTIALS;
  return (unsigned)(b > 0 ? b : 1);
}

template <int REC>
void launch_fill(const MapParams& P, bool mlp, cudaStream_t s) {
  if (mlp) fill_kernel<-1, REC><<<P.p.n, FILL_THREADS, 0, s>>>(P);
  else if (P.eps_mode == 0 && P.eps_n == 4) fill_kernel<4, REC><<<P.p.n, FILL_THREADS, 0, s>>>(P);
  else if (P.eps_mode == 0 && P.eps_n == 8) fill_kernel<8, REC><<<P.p.n, FILL_THREADS, 0, s>>>(P);
  else fill_kernel<0, REC><<<P.p.n, FILL_THREADS, 0, s>>>(P);
}

int map_common(MapParams P, cudaStream_t s, bool mlp) {
  int launches = 0;
  cudaMemsetAsync(P.cov.mask, 0, sizeof(uint32_t) * P.g.nwords, s);
  cudaMemsetAsync(P.cov.dup, 0, sizeof(uint32_t) * P.g.nwords, s);
  if (P.cov.full) cudaMemsetAsync(P.cov.full, 0, sizeof(uint32_t) * P.g.nwords, s);
  if (mlp) cudaMemsetAsync(P.mlp_count, 0, sizeof(int), s);
  if (P.p.n > 0) {
    box_kernel<<<(P.p.n + 127) / 128, 128, 0, s>>>(P);
    mark_kernel<<<P.p.n, MAP_THREADS, 0, s>>>(P);
    launches += 2;
  }
  const unsigned nb = (unsigned)P.cov.nblocks;
  scan_words_kernel<<<nb, SCAN_THREADS, 0, s>>>(P.cov, P.g.nwords);
  scan_blocks_kernel<<<1, SCAN_THREADS, 0, s>>>(P.cov, P.cov.nblocks);
  scan_add_kernel<<<nb, SCAN_THREADS, 0, s>>>(P.cov, P.g.nwords);
  clear_slots_kernel<<<grid_cap(P.s.cap, 256), 256, 0, s>>>(P);
  launches += 4;
  if (P.p.n > 0) {
    const int rec = P.fp32 ? REC_FP32 : (P.dfrec ? REC_DF : REC_FP64);
    if (rec == REC_FP32) launch_fill<REC_FP32>(P, mlp, s);
    else if (rec == REC_DF) launch_fill<REC_DF>(P, mlp, s);
    else launch_fill<REC_FP64>(P, mlp, s);
    ++launches;
    // the count pass: 8^3 sampling's worklist, or the surrogate's shared cells
    if ((mlp || P.eps_mode == 0) && P.eps_n == 8 && P.wtab && P.wl_X) {
      if (rec == REC_FP32) count8_kernel<REC_FP32><<<P.p.n, COUNT_THREADS, 0, s>>>(P);
      else if (rec == REC_DF) count8_kernel<REC_DF><<<P.p.n, COUNT_THREADS, 0, s>>>(P);
      else count8_kernel<REC_FP64><<<P.p.n, COUNT_THREADS, 0, s>>>(P);
      ++launches;
    }
  }
  return launches;
}

int map_finish(MapParams P, cudaStream_t s) {
  const unsigned nfin = grid_cap(P.s.cap, 256);
  if (P.fp32) finish_kernel<REC_FP32><<<nfin, 256, 0, s>>>(P);
  else if (P.dfrec) finish_kernel<REC_DF><<<nfin, 256, 0, s>>>(P);
  else finish_kernel<REC_FP64><<<nfin, 256, 0, s>>>(P);
  vfluid_kernel<<<1, 256, 0, s>>>(P, (int)nfin);
  return 2;
}

}  // namespace

int launch_map(MapParams P, cudaStream_t s) {
  return map_common(P, s, false) + map_finish(P, s);
}

// mapping with the surrogate: the fill pass lists the network's cells, the
// network runs on the tensor cores and writes their B, the finish pass
// samples what is left (cells of two particles, worklist overflow, no
// network set) with 8^3 points
int launch_map_mlp(MapParams P, cudaStream_t s) {
  int launches = map_common(P, s, true);
  if (P.mlp && P.mlp_cap > 0) {
    InferSink out{};
    out.V = P.s.V;
    out.lin = P.mlp_lin;
    out.work = P.mlp_work;
    out.cap = P.s.cap;
    out.fp32 = P.fp32;
    out.dfrec = P.dfrec;
    out.nt = P.weighting;
    out.tau = P.tau;
    launches += launch_mlp_infer(P.mlp, -1, P.mlp_count, P.mlp_cap, P.mlp_X, out, P.status, s);
  }
  return launches + map_finish(P, s);
}

size_t map_box_bytes() { return sizeof(Box); }

int launch_weight_table(int n, double tau, int weighting, double* out, cudaStream_t s) {
  const int n3 = n * n * n;
  if (n3 >= WTAB) return 0;
  wtab_kernel<<<1, 256, 0, s>>>(n3, tau, weighting, out);
  return 1;
}

int launch_force_reduce(MapParams P, cudaStream_t s) {
  if (P.p.n == 0) return 0;
  if (P.fp32) force_reduce_f32_kernel<<<P.p.n, RED_THREADS, 0, s>>>(P);
  else if (P.dfrec) force_reduce_df_kernel<<<P.p.n, RED_THREADS, 0, s>>>(P);
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

int launch_slot_forces_to_dense(MapParams P, int* pid0, int* pid1, double* F0, double* F1,
                                cudaStream_t s) {
  const long long N = (long long)P.g.nx * P.g.ny * P.g.nz;
  cudaMemsetAsync(pid0, 0xff, sizeof(int) * N, s);  // -1
  cudaMemsetAsync(pid1, 0xff, sizeof(int) * N, s);
  cudaMemsetAsync(F0, 0, sizeof(double) * 3 * N, s);
  cudaMemsetAsync(F1, 0, sizeof(double) * 3 * N, s);
  dense_forces_kernel<<<grid_cap(P.s.cap, 256), 256, 0, s>>>(P, pid0, pid1, F0, F1);
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
