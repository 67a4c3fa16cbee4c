// mlp_kernels.cu -- the learned eps surrogate: 4 -> 32 (ReLU) -> 32 (ReLU) -> 1.
// Inputs x = (|d/r| components in decreasing order, r), d = cell centre minus
// sphere centre: the offset in the orientation fixed by the cube's symmetries
// (eps is invariant under sign flips and permutations of d).  The network
// predicts the correction to the linear approximation of Sec. 2.3.2
// (Eqs. 25-27): eps = clamp(eps_lin(|d|, r) + MLP(x), 0, 1).  It replaces the
// sub-division sampling for partial cells within reach of one particle and
// away from walls; 8^3 sampling stays the fallback and gives the labels the
// network is trained on (target: label - eps_lin).
//
// Parameters (FP32, packed): W1 [0,128) 32x4 row-major, b1 [128,160),
// W2 [160,1184) 32x32, b2 [1184,1216), W3 [1216,1248), b3 [1248].
//
// Training samples: SplitMix64 counter stream (value k of stream s is the
// SplitMix64 output for state s + (k+1)*0x9E3779B97F4A7C15; a uniform double
// is its top 53 bits times 2^-53).  Sample i uses values 5i..5i+4:
//   r = 2 + 10 u0; v = (2u1-1, 2u2-1, 2u3-1); rho = (r - sqrt3/2) + sqrt3 u4;
//   d = v * (rho / |v|); label = (8^3 samples of the cell inside) / 512.
// Every step is an IEEE-rounded FP64 operation (compiled with -fmad=false).
//
// Training: one block per 128-sample tile computes forward and backward in
// FP32 and the tile's gradient as sums over its samples (no atomics); the
// tiles are reduced in a fixed order; Adam (Kingma and Ba, 2015) updates the
// FP32 master weights.
//
// Inference: tiles of 128 inputs per CTA; layer 1 (K = 4) in FP32, layer 2
// on the 5th-generation tensor cores (tcgen05.mma, BF16 operands from shared
// memory, FP32 accumulator in tensor memory), layer 3 (N = 1) in FP32 after
// tcgen05.ld; in the mapping the same kernel turns the outputs into B.
#include <cuda_bf16.h>

#include "geom.cuh"
#include "psm_internal.cuh"

namespace psm {
namespace {

constexpr int OFF_B1 = 128, OFF_W2 = 160, OFF_B2 = 1184, OFF_W3 = 1216, OFF_B3 = 1248;
constexpr int NPARAM = 1249;

__device__ __forceinline__ unsigned long long splitmix64(unsigned long long seed,
                                                         unsigned long long k) {
  unsigned long long z = seed + (k + 1ULL) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform01(unsigned long long seed, unsigned long long k) {
  return (double)(splitmix64(seed, k) >> 11) * 0x1.0p-53;
}

// f(r) = V_a(r) - r + 1/2 of Eqs. 26-27 (training targets only; the mapping
// takes f(r) computed on the host for each particle)
__device__ double linear_fr(double r) {
  const double r2 = r * r;
  const double s = sqrt(r2 - 0.5);
  const double Va = (1.0 / 12.0 - r2) * atan((0.5 * s) / (0.5 - r2)) + s / 3.0 +
                    (r2 - 1.0 / 12.0) * atan(0.5 / s) - 4.0 / 3.0 * r2 * r * atan(0.25 / (r * s));
  return Va - r + 0.5;
}

// inputs of the network for offset d and radius r
__device__ __forceinline__ float4 network_input(double dx, double dy, double dz, double r) {
  double a = fabs(dx / r), b = fabs(dy / r), c = fabs(dz / r), t;
  if (b > a) { t = a; a = b; b = t; }
  if (c > a) { t = a; a = c; c = t; }
  if (c > b) { t = b; b = c; c = t; }
  return make_float4((float)a, (float)b, (float)c, (float)r);
}

// resid (optional): label - eps_lin, the network's training target
__global__ void samples_kernel(unsigned long long seed, long long first, long long count,
                               float* __restrict__ X, float* __restrict__ eps,
                               float* __restrict__ resid) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < count;
       t += (long long)gridDim.x * blockDim.x) {
    const unsigned long long i = (unsigned long long)(first + t);
    double u[5];
    for (int j = 0; j < 5; ++j) u[j] = uniform01(seed, 5ULL * i + j);
    const double r = 2.0 + 10.0 * u[0];
    double v0 = 2.0 * u[1] - 1.0, v1 = 2.0 * u[2] - 1.0, v2 = 2.0 * u[3] - 1.0;
    double nv = sqrt(v0 * v0 + v1 * v1 + v2 * v2);
    if (nv == 0.0) {
      v0 = 1.0; v1 = 0.0; v2 = 0.0; nv = 1.0;
    }
    const double rho = (r - kHalfSqrt3) + 1.7320508075688772935 * u[4];
    const double tt = rho / nv;
    const double d0 = v0 * tt, d1 = v1 * tt, d2 = v2 * tt;
    const int cnt = supersample_count_n<8>(d0, d1, d2, r);
    reinterpret_cast<float4*>(X)[t] = network_input(d0, d1, d2, r);
    const double label = (double)cnt * (1.0 / 512.0);
    eps[t] = (float)label;
    if (resid) {
      const double dist = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
      double lin = -(dist - r) + linear_fr(r);
      lin = lin < 0.0 ? 0.0 : (lin > 1.0 ? 1.0 : lin);
      resid[t] = (float)(label - lin);
    }
  }
}

// ---- training: forward + backward of one tile of samples
constexpr int TILE = 128;
constexpr int ROW = 33;  // padded row of 32 activations (bank-conflict free)

struct TrainSmem {
  float p[NPARAM + 3];
  float x[TILE][4];
  float h1[TILE][ROW];
  float h2[TILE][ROW];
  float dh1[TILE][ROW];
  float dh2[TILE][ROW];
  float dy[TILE];
  float l2[TILE];
};

__global__ void __launch_bounds__(TILE) train_tile_kernel(const float* __restrict__ params,
                                                         long long m,
                                                         const float* __restrict__ X,
                                                         const float* __restrict__ t,
                                                         float* __restrict__ partials) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TrainSmem& S = *reinterpret_cast<TrainSmem*>(smem_raw);
  for (int i = threadIdx.x; i < NPARAM; i += TILE) S.p[i] = params[i];
  __syncthreads();
  const long long s = (long long)blockIdx.x * TILE + threadIdx.x;
  const int r = threadIdx.x;
  const float inv_m = 1.0f / (float)m;
  if (s < m) {
    float x[4];
    for (int k = 0; k < 4; ++k) x[k] = X[4 * s + k];
    float a1[32], h2v[32];
    for (int j = 0; j < 32; ++j) {
      float acc = S.p[OFF_B1 + j];
      for (int k = 0; k < 4; ++k) acc = fmaf(S.p[j * 4 + k], x[k], acc);
      a1[j] = acc;
      S.h1[r][j] = acc > 0.f ? acc : 0.f;
    }
    float y = S.p[OFF_B3];
    for (int j = 0; j < 32; ++j) {
      float acc = S.p[OFF_B2 + j];
      for (int k = 0; k < 32; ++k) acc = fmaf(S.p[OFF_W2 + j * 32 + k], S.h1[r][k], acc);
      h2v[j] = acc;  // pre-activation
      const float h = acc > 0.f ? acc : 0.f;
      S.h2[r][j] = h;
      y = fmaf(S.p[OFF_W3 + j], h, y);
    }
    const float res = y - t[s];
    const float dy = 2.0f * res * inv_m;
    S.dy[r] = dy;
    S.l2[r] = res * res;
    for (int j = 0; j < 32; ++j) S.dh2[r][j] = h2v[j] > 0.f ? dy * S.p[OFF_W3 + j] : 0.f;
    for (int k = 0; k < 32; ++k) {
      float acc = 0.f;
      for (int j = 0; j < 32; ++j) acc = fmaf(S.p[OFF_W2 + j * 32 + k], S.dh2[r][j], acc);
      S.dh1[r][k] = a1[k] > 0.f ? acc : 0.f;
    }
    for (int k = 0; k < 4; ++k) S.x[r][k] = x[k];
  } else {
    for (int j = 0; j < 32; ++j) {
      S.h1[r][j] = 0.f; S.h2[r][j] = 0.f; S.dh1[r][j] = 0.f; S.dh2[r][j] = 0.f;
    }
    for (int k = 0; k < 4; ++k) S.x[r][k] = 0.f;
    S.dy[r] = 0.f;
    S.l2[r] = 0.f;
  }
  __syncthreads();
  // gradient of this tile: sums over its samples in a fixed order
  float* out = partials + (long long)blockIdx.x * (NPARAM + 1);
  for (int e = threadIdx.x; e < NPARAM + 1; e += TILE) {
    float acc = 0.f;
    if (e < OFF_B1) {  // dW1[j][k]
      const int j = e / 4, k = e % 4;
      for (int q = 0; q < TILE; ++q) acc = fmaf(S.dh1[q][j], S.x[q][k], acc);
    } else if (e < OFF_W2) {  // db1
      const int j = e - OFF_B1;
      for (int q = 0; q < TILE; ++q) acc += S.dh1[q][j];
    } else if (e < OFF_B2) {  // dW2[j][k]
      const int j = (e - OFF_W2) / 32, k = (e - OFF_W2) % 32;
      for (int q = 0; q < TILE; ++q) acc = fmaf(S.dh2[q][j], S.h1[q][k], acc);
    } else if (e < OFF_W3) {  // db2
      const int j = e - OFF_B2;
      for (int q = 0; q < TILE; ++q) acc += S.dh2[q][j];
    } else if (e < OFF_B3) {  // dW3
      const int j = e - OFF_W3;
      for (int q = 0; q < TILE; ++q) acc = fmaf(S.dy[q], S.h2[q][j], acc);
    } else if (e == OFF_B3) {
      for (int q = 0; q < TILE; ++q) acc += S.dy[q];
    } else {  // loss numerator
      for (int q = 0; q < TILE; ++q) acc += S.l2[q];
    }
    out[e] = acc;
  }
}

__global__ void grad_reduce_kernel(const float* __restrict__ partials, int nblocks,
                                   float* __restrict__ grad, float* __restrict__ loss,
                                   float inv_m) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e > NPARAM) return;
  float acc = 0.f;
  for (int b = 0; b < nblocks; ++b) acc += partials[(long long)b * (NPARAM + 1) + e];
  if (e < NPARAM) grad[e] = acc;
  else if (loss) *loss = acc * inv_m;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g,
                            float* __restrict__ m, float* __restrict__ v, float bc1, float bc2,
                            float lr) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAM) return;
  const float gi = g[i];
  const float mi = 0.9f * m[i] + 0.1f * gi;
  const float vi = 0.999f * v[i] + 0.001f * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float mh = mi / bc1, vh = vi / bc2;
  p[i] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

// ---- inference on the 5th-generation tensor cores.  One CTA of 128
// threads takes two tiles of 128 inputs at a time: each thread computes its
// two rows' layer 1 in FP32 (each weight read once for both) and writes the
// ReLU activations as BF16 into shared memory in the K-major core-matrix
// layout (8 rows x 16 bytes per core matrix); one thread issues each tile's
// layer-2 product h1 (128 x 32) x W2^T (32 x 32) as two tcgen05.mma (K = 16
// each, BF16 operands) into its own FP32 accumulator in tensor memory (32
// columns each) and one commit for the four; after the commit arrives on the
// mbarrier each warp reads its 32 rows of each tile back with tcgen05.ld and
// finishes layer 3 (bias, ReLU, dot with W3) in FP32.  Waits are bounded: a wait that gives up sets
// ST_TIMEOUT, waits once more for the tensor core and frees its tensor memory.
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

constexpr int INF_M = 128;         // rows per tile: the MMA's M
constexpr int INF_THREADS = 128;   // thread t owns row t; warp w reads TMEM lanes 32w..32w+31
constexpr int INF_PER_SM = 6;      // resident CTAs per SM: the grid is one wave of them
constexpr unsigned INF_TMEM_COLS = 64;  // two FP32 accumulators of N = 32 columns
constexpr unsigned long long kInferWaitNs = 1000000000ull;
// instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N / 8 at
// bits 17-22, M / 16 at bits 24-28
constexpr uint32_t kInferIdesc =
    (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((unsigned)(INF_M >> 4) << 24);

struct InferSmem {
  alignas(128) unsigned char a[2][INF_M * 32 * 2];  // layer-1 activations of two tiles, BF16
  alignas(128) unsigned char b[32 * 32 * 2];     // W2 (N = 32 rows of K = 32), BF16
  float4 w1[32];
  float b1[32], b2[32], w3[32];
  float b3;
  unsigned tmem;
  unsigned long long bar;
};

// byte offset of the 16-byte chunk kc (elements 8kc..8kc+7) of row `row` in
// the K-major layout without swizzle: core matrices of 8 rows x 16 bytes, the
// K direction's four core matrices 128 bytes apart (leading byte offset),
// successive groups of 8 rows 512 bytes apart (stride byte offset)
__device__ __forceinline__ int kmajor_off(int row, int kc) {
  return (row >> 3) * 512 + kc * 128 + (row & 7) * 16;
}
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
// shared-memory matrix descriptor of tcgen05: start address >> 4 (bits 0-13),
// leading byte offset >> 4 (bits 16-29), stride byte offset >> 4 (bits
// 32-45), the fixed value 1 at bits 46-48, base offset 0, no swizzle
__device__ __forceinline__ uint64_t kmajor_desc(const void* p) {
  return (uint64_t)((smem_addr(p) & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)(512 >> 4) << 32) | (1ull << 46);
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ bool inf_mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __noinline__ bool inf_mbar_wait(unsigned long long* bar, unsigned parity,
                                           unsigned long long limit_ns = kInferWaitNs) {
  if (inf_mbar_test(bar, parity)) return true;
  unsigned long long t0, t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (;;) {
    for (int i = 0; i < 64; ++i)
      if (inf_mbar_test(bar, parity)) return true;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > limit_ns) return false;
  }
}

// diagnostic: the inference kernel's bounded wait on an mbarrier that no
// commit arrives on gives up after limit_ns and raises ST_TIMEOUT
__global__ void infer_wait_selftest_kernel(unsigned* status, unsigned long long limit_ns) {
  __shared__ __align__(8) unsigned long long bar;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && !inf_mbar_wait(&bar, 0u, limit_ns)) atomicOr(status, ST_TIMEOUT);
}
__device__ __forceinline__ void tc_mma_bf16(unsigned d_tmem, uint64_t adesc, uint64_t bdesc,
                                            int accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(kInferIdesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void tc_commit(unsigned long long* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(bar))
      : "memory");
}
// 32 consecutive accumulator columns of this warp's 32 TMEM lanes, one lane per thread
__device__ __forceinline__ void tc_ld32(unsigned taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// B(eps) of Eq. 16 in the storage precision of the slot records
__device__ __forceinline__ void apply_weight(const InferSink& o, long long rec, float epsf) {
  if (o.fp32) {
    float B = epsf;
    if (o.nt && epsf != 0.f && epsf != 1.f) {
      const float tm = (float)(o.tau - 0.5);
      B = epsf * tm / ((1.f - epsf) + tm);
    }
    static_cast<float*>(o.V)[4 * rec + 3] = B;
  } else {
    const double eps = (double)epsf;
    double B = eps;
    if (o.nt && eps != 0.0 && eps != 1.0) B = eps * (o.tau - 0.5) / ((1.0 - eps) + (o.tau - 0.5));
    if (o.dfrec) static_cast<df*>(o.V)[4 * rec + 3] = df(B);
    else static_cast<double*>(o.V)[4 * rec + 3] = B;
  }
}

// raw network outputs (o.eps != NULL) or, in the mapping, eps = clamp(linear
// approximation + output, 0, 1) and its weight B into the item's slot record
// when the cell is within reach of this particle only (cells shared by two
// particles keep B = -1 and are sampled by the finish pass).  count: number
// of inputs, read from *count_dev when count < 0, at most cap.
__global__ void __launch_bounds__(INF_THREADS, INF_PER_SM) infer_tc_kernel(
    const float* __restrict__ P, long long count, const int* __restrict__ count_dev,
    long long cap, const float4* __restrict__ X, InferSink o, unsigned* status) {
  __shared__ InferSmem S;
  const int tid = threadIdx.x, warp = tid >> 5;
  long long n = count >= 0 ? count : (long long)*count_dev;
  if (n > cap) n = cap;
  // W2 as the B operand (row j = output neuron, K = input neuron), the
  // other parameters in FP32
  for (int i = tid; i < 32 * 4; i += INF_THREADS) {
    const int j = i >> 2, kc = i & 3;
    const float* w = P + OFF_W2 + j * 32 + kc * 8;
    *reinterpret_cast<uint4*>(S.b + kmajor_off(j, kc)) =
        make_uint4(pack_bf16(w[0], w[1]), pack_bf16(w[2], w[3]), pack_bf16(w[4], w[5]),
                   pack_bf16(w[6], w[7]));
  }
  if (tid < 32) {
    S.w1[tid] = make_float4(P[4 * tid], P[4 * tid + 1], P[4 * tid + 2], P[4 * tid + 3]);
    S.b1[tid] = P[OFF_B1 + tid];
    S.b2[tid] = P[OFF_B2 + tid];
    S.w3[tid] = P[OFF_W3 + tid];
  }
  if (tid == 0) {
    S.b3 = P[OFF_B3];
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&S.bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_addr(&S.tmem)),
                 "r"(INF_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_async_smem();  // W2 was written by the generic proxy, the MMA reads it
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = S.tmem;
  // A operands of the two tiles, K = 0..15 and 16..31 (chunks 0-1 and 2-3)
  const uint64_t ad00 = kmajor_desc(S.a[0]), ad01 = kmajor_desc(S.a[0] + 256);
  const uint64_t ad10 = kmajor_desc(S.a[1]), ad11 = kmajor_desc(S.a[1] + 256);
  const uint64_t bd0 = kmajor_desc(S.b), bd1 = kmajor_desc(S.b + 256);
  unsigned phase = 0;
  bool in_flight = false;
  // software pipeline: a tile's inputs (and, in the mapping, its slot item
  // and linear approximation) are loaded while the previous tile computes
  auto load_row = [&](long long r, float4& xr, int& it, float& ln) {
    xr = make_float4(0.f, 0.f, 0.f, 0.f);
    it = -1;
    ln = 0.f;
    if (r < n) {
      xr = X[r];
      if (!o.eps) {
        it = o.work[r];
        ln = o.lin[r];
      }
    }
  };
  // each iteration takes two tiles (rows r and r + 128 of a pair): layer 1
  // reads each weight once for both rows, one commit covers both products
  // and the CTA meets at two barriers per 256 rows
  const long long npairs = (n + 2 * INF_M - 1) / (2 * INF_M);
  float4 x0, x1;
  int item0, item1;
  float lin0, lin1;
  load_row((long long)blockIdx.x * (2 * INF_M) + tid, x0, item0, lin0);
  load_row((long long)blockIdx.x * (2 * INF_M) + INF_M + tid, x1, item1, lin1);
  // layer 3 and B(eps) of one row from its accumulator columns
  auto finish_row = [&](const float* acc, long long row, int item, float lin) {
    float y = 0.f;
#pragma unroll
    for (int j = 0; j < 32; ++j) {
      const float v = acc[j] + S.b2[j];
      y = fmaf(S.w3[j], v > 0.f ? v : 0.f, y);
    }
    y += S.b3;
    if (row < n) {
      if (o.eps) {
        o.eps[row] = y;
      } else if (item >= 0) {  // item -1: an empty item (the fill pass lists
                               // only cells in reach of one particle)
        float eps = lin + y;
        eps = eps < 0.f ? 0.f : (eps > 1.f ? 1.f : eps);
        apply_weight(o, (item & 1) * o.cap + (item >> 1), eps);
      }
    }
  };
  for (long long pr = blockIdx.x; pr < npairs; pr += gridDim.x) {
    const long long row0 = pr * (2 * INF_M) + tid, row1 = row0 + INF_M;
    float4 xn0, xn1;
    int itemn0, itemn1;
    float linn0, linn1;
    const long long next = (pr + gridDim.x) * (2 * INF_M) + tid;
    load_row(next, xn0, itemn0, linn0);
    load_row(next + INF_M, xn1, itemn1, linn1);
    // layer 1 (FP32), ReLU, BF16 activations into the two A operands
#pragma unroll
    for (int kc = 0; kc < 4; ++kc) {
      uint32_t w0[4], w1[4];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        float v0[2], v1[2];
#pragma unroll
        for (int e = 0; e < 2; ++e) {
          const int j = 8 * kc + 2 * h + e;
          const float4 wj = S.w1[j];
          const float bj = S.b1[j];
          float a = fmaf(wj.x, x0.x, bj);
          a = fmaf(wj.y, x0.y, a);
          a = fmaf(wj.z, x0.z, a);
          a = fmaf(wj.w, x0.w, a);
          float b = fmaf(wj.x, x1.x, bj);
          b = fmaf(wj.y, x1.y, b);
          b = fmaf(wj.z, x1.z, b);
          b = fmaf(wj.w, x1.w, b);
          v0[e] = a > 0.f ? a : 0.f;
          v1[e] = b > 0.f ? b : 0.f;
        }
        w0[h] = pack_bf16(v0[0], v0[1]);
        w1[h] = pack_bf16(v1[0], v1[1]);
      }
      *reinterpret_cast<uint4*>(S.a[0] + kmajor_off(tid, kc)) =
          make_uint4(w0[0], w0[1], w0[2], w0[3]);
      *reinterpret_cast<uint4*>(S.a[1] + kmajor_off(tid, kc)) =
          make_uint4(w1[0], w1[1], w1[2], w1[3]);
    }
    fence_async_smem();
    __syncthreads();
    bool done = true;
    if (tid == 0) {
      tc_fence_after();
      tc_mma_bf16(tmem, ad00, bd0, 0);
      tc_mma_bf16(tmem, ad01, bd1, 1);
      tc_mma_bf16(tmem + 32u, ad10, bd0, 0);
      tc_mma_bf16(tmem + 32u, ad11, bd1, 1);
      tc_commit(&S.bar);
      done = inf_mbar_wait(&S.bar, phase);
    }
    in_flight = true;
    if (!__syncthreads_and(done)) {
      if (tid == 0) atomicOr(status, ST_TIMEOUT);
      break;
    }
    in_flight = false;
    phase ^= 1u;
    tc_fence_after();
    float acc[32];
    const unsigned lanes = (unsigned)(warp * 32) << 16;
    tc_ld32(tmem + lanes, acc);
    finish_row(acc, row0, item0, lin0);
    tc_ld32(tmem + lanes + 32u, acc);
    finish_row(acc, row1, item1, lin1);
    x0 = xn0;
    x1 = xn1;
    item0 = itemn0;
    item1 = itemn1;
    lin0 = linn0;
    lin1 = linn1;
    tc_fence_before();
    __syncthreads();  // the A tiles and the accumulators are free again
  }
  if (in_flight && tid == 0) inf_mbar_wait(&S.bar, phase);  // the MMA of a wait that gave up
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(INF_TMEM_COLS)
                 : "memory");
  }
}

}  // namespace

int launch_mlp_samples(unsigned long long seed, long long first, long long count, float* X,
                       float* eps, float* resid, cudaStream_t s) {
  if (count <= 0) return 0;
  long long blocks = (count + 255) / 256;
  if (blocks > 152 * 64) blocks = 152 * 64;
  samples_kernel<<<(unsigned)blocks, 256, 0, s>>>(seed, first, count, X, eps, resid);
  return 1;
}

int mlp_grad_blocks(long long m) { return (int)((m + TILE - 1) / TILE); }

int launch_mlp_loss_grad(const float* params, long long m, const float* X, const float* t,
                         float* grad_partials, int nblocks, float* grad, float* loss,
                         cudaStream_t s) {
  static bool configured = false;
  const int smem = (int)sizeof(TrainSmem);
  if (!configured) {
    cudaFuncSetAttribute(train_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    configured = true;
  }
  train_tile_kernel<<<nblocks, TILE, smem, s>>>(params, m, X, t, grad_partials);
  grad_reduce_kernel<<<(NPARAM + 1 + 255) / 256, 256, 0, s>>>(grad_partials, nblocks, grad,
                                                             loss, 1.0f / (float)m);
  return 2;
}

int launch_adam(float* params, const float* grad, float* mstate, float* vstate, int step,
                float lr, cudaStream_t s) {
  const float bc1 = 1.0f - powf(0.9f, (float)step);
  const float bc2 = 1.0f - powf(0.999f, (float)step);
  adam_kernel<<<(NPARAM + 255) / 256, 256, 0, s>>>(params, grad, mstate, vstate, bc1, bc2, lr);
  return 1;
}

int launch_wait_selftest_mlp(unsigned* status, unsigned long long limit_ns, cudaStream_t s) {
  infer_wait_selftest_kernel<<<1, 32, 0, s>>>(status, limit_ns);
  return 1;
}

// network outputs for m inputs (m_dev: count on the device, m < 0), at most
// cap; results to the sink
// resident inference CTAs on the device (all SMs), set by mlp_configure
static int g_infer_ctas = 0;

int mlp_configure() {
  // INF_PER_SM CTAs per SM (the launch bounds keep their registers within
  // the SM's file; 6 x 64 of the 512 tensor-memory columns) times the SMs;
  // shared memory for all of them (6 x 19 KB): the carveout's maximum.
  // (Eight CTAs of 64 registers spilled and measured 7% slower.)
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      sms <= 0 ||
      cudaFuncSetAttribute(infer_tc_kernel, cudaFuncAttributePreferredSharedMemoryCarveout,
                           (int)cudaSharedmemCarveoutMaxShared) != cudaSuccess)
    return 1;
  g_infer_ctas = sms * INF_PER_SM;
  return 0;
}

int launch_mlp_infer(const float* params, long long m, const int* m_dev, long long cap,
                     const float* X, const InferSink& out, unsigned* status, cudaStream_t s) {
  const long long rows = m >= 0 ? (m < cap ? m : cap) : cap;
  if (rows <= 0) return 0;
  // one wave of CTAs, each looping over tiles (a second, partial wave would
  // leave SMs idle)
  long long blocks = (rows + 2 * INF_M - 1) / (2 * INF_M);  // pairs of tiles
  const long long wave = g_infer_ctas > 0 ? g_infer_ctas : 152 * INF_PER_SM;
  if (blocks > wave) blocks = wave;
  infer_tc_kernel<<<(unsigned)blocks, INF_THREADS, 0, s>>>(
      params, m, m_dev, cap, reinterpret_cast<const float4*>(X), out, status);
  return 1;
}

}  // namespace psm
