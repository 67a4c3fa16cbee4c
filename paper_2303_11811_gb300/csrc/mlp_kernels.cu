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
// Inference: per warp, tiles of 16 inputs; layer 1 (K = 4) in FP32, layer 2
// on the tensor cores (mma.sync m16n8k16, BF16 operands, FP32 accumulation,
// the layer-1 accumulator fragments reused as the A operand), layer 3 (N = 1)
// as FP32 dot products reduced across the quad of lanes that holds a row.
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

// ---- inference
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ void mma_bf16(float* c, const uint32_t* a, const uint32_t* b) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
      "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// raw network outputs for inputs X; count: number of inputs, read from
// *count_dev when count < 0
__global__ void __launch_bounds__(128) infer_kernel(const float* __restrict__ P, long long count,
                                                   const int* __restrict__ count_dev,
                                                   const float4* __restrict__ X,
                                                   float* __restrict__ eps) {
  const long long n = count >= 0 ? count : (long long)*count_dev;
  const int lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  // layer-1 neurons this lane produces: j = 8c + 2t + {0,1}, c = 0..3
  float w1[8][4], b1[8];
  for (int c = 0; c < 4; ++c)
    for (int h = 0; h < 2; ++h) {
      const int j = 8 * c + 2 * t + h;
      for (int k = 0; k < 4; ++k) w1[2 * c + h][k] = P[j * 4 + k];
      b1[2 * c + h] = P[OFF_B1 + j];
    }
  // layer-2 B fragments: n-tile nt (outputs 8nt + g), k-step ks
  uint32_t bw[4][2][2];
  for (int nt = 0; nt < 4; ++nt)
    for (int ks = 0; ks < 2; ++ks) {
      const float* row = P + OFF_W2 + (8 * nt + g) * 32 + 16 * ks;
      bw[nt][ks][0] = pack_bf16(row[2 * t], row[2 * t + 1]);
      bw[nt][ks][1] = pack_bf16(row[8 + 2 * t], row[8 + 2 * t + 1]);
    }
  float b2[8], w3[8];
  for (int nt = 0; nt < 4; ++nt)
    for (int h = 0; h < 2; ++h) {
      b2[2 * nt + h] = P[OFF_B2 + 8 * nt + 2 * t + h];
      w3[2 * nt + h] = P[OFF_W3 + 8 * nt + 2 * t + h];
    }
  const float b3 = P[OFF_B3];

  const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  const long long ntiles = (n + 15) / 16;
  for (long long tile = warp; tile < ntiles; tile += nwarps) {
    const long long r0 = tile * 16 + g, r1 = r0 + 8;
    const float4 x0 = r0 < n ? X[r0] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 x1 = r1 < n ? X[r1] : make_float4(0.f, 0.f, 0.f, 0.f);
    // layer 1 in FP32, ReLU, packed as the A fragments of layer 2
    float h0[8], h1v[8];
    for (int i = 0; i < 8; ++i) {
      float a = b1[i], b = b1[i];
      a = fmaf(w1[i][0], x0.x, a); a = fmaf(w1[i][1], x0.y, a);
      a = fmaf(w1[i][2], x0.z, a); a = fmaf(w1[i][3], x0.w, a);
      b = fmaf(w1[i][0], x1.x, b); b = fmaf(w1[i][1], x1.y, b);
      b = fmaf(w1[i][2], x1.z, b); b = fmaf(w1[i][3], x1.w, b);
      h0[i] = a > 0.f ? a : 0.f;
      h1v[i] = b > 0.f ? b : 0.f;
    }
    uint32_t A[2][4];
    for (int ks = 0; ks < 2; ++ks) {
      // k = 16ks + 2t (+1) -> neuron index i = 2*(2ks) + h; k + 8 -> 2*(2ks+1) + h
      A[ks][0] = pack_bf16(h0[4 * ks + 0], h0[4 * ks + 1]);
      A[ks][1] = pack_bf16(h1v[4 * ks + 0], h1v[4 * ks + 1]);
      A[ks][2] = pack_bf16(h0[4 * ks + 2], h0[4 * ks + 3]);
      A[ks][3] = pack_bf16(h1v[4 * ks + 2], h1v[4 * ks + 3]);
    }
    float y0 = 0.f, y1 = 0.f;
    for (int nt = 0; nt < 4; ++nt) {
      float c[4] = {0.f, 0.f, 0.f, 0.f};
      mma_bf16(c, A[0], bw[nt][0]);
      mma_bf16(c, A[1], bw[nt][1]);
      for (int h = 0; h < 2; ++h) {
        const float v0 = c[h] + b2[2 * nt + h];
        const float v1 = c[2 + h] + b2[2 * nt + h];
        y0 = fmaf(w3[2 * nt + h], v0 > 0.f ? v0 : 0.f, y0);
        y1 = fmaf(w3[2 * nt + h], v1 > 0.f ? v1 : 0.f, y1);
      }
    }
    y0 += __shfl_xor_sync(0xffffffffu, y0, 1);
    y0 += __shfl_xor_sync(0xffffffffu, y0, 2);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 1);
    y1 += __shfl_xor_sync(0xffffffffu, y1, 2);
    if (t == 0) {
      if (r0 < n) eps[r0] = y0 + b3;
      if (r1 < n) eps[r1] = y1 + b3;
    }
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

int launch_mlp_infer(const float* params, long long m, const float* X, float* eps,
                     cudaStream_t s) {
  if (m <= 0) return 0;
  long long tiles = (m + 15) / 16;
  long long blocks = (tiles + 3) / 4;
  if (blocks > 152 * 16) blocks = 152 * 16;
  infer_kernel<<<(unsigned)blocks, 128, 0, s>>>(params, m, nullptr,
                                               reinterpret_cast<const float4*>(X), eps);
  return 1;
}

int launch_mlp_infer_dev(const float* params, const int* count_dev, long long cap,
                         const float* X, float* eps, cudaStream_t s) {
  long long tiles = (cap + 15) / 16;
  long long blocks = (tiles + 3) / 4;
  if (blocks > 152 * 16) blocks = 152 * 16;
  if (blocks < 1) blocks = 1;
  infer_kernel<<<(unsigned)blocks, 128, 0, s>>>(params, -1, count_dev,
                                               reinterpret_cast<const float4*>(X), eps);
  return 1;
}

}  // namespace psm
