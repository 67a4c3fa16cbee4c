// noalloc_sums.cu -- mass and momentum of a PDF field without any device
// allocation (psm_field_sums_noalloc in include/psm.h).
//
// psm_check sums through buffers the context allocates.  Some callers cannot
// allocate at the point where they want this check: a solver that hands out
// all device memory from its own fixed pool at start-up, a monitoring hook
// inside another code's time loop where cudaMalloc/cudaFree would synchronise
// the whole device and stall its other streams, or a run that has committed
// its memory budget so that a late allocation could fail.  This file gives
// them the same sums with the block partials kept in a file-scope device
// array instead of allocated memory.
//
// The array holds NOALLOC_MAX_PARTS x 4 doubles (128 KiB).  Every GPU that
// loads the library keeps it until the process exits, and all calls on one
// GPU share it: it keeps the last call's partials, and two calls whose work
// overlaps on the GPU (different streams, no ordering between them) race on
// it.  Each call writes every partial it reads before reading it, so nothing
// has to be cleared between calls.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/psm.h"

namespace {

constexpr int NOALLOC_MAX_PARTS = 4096;
constexpr long long NOALLOC_CELLS_PER_PART = 65536;
constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) double g_sum_partials[4 * NOALLOC_MAX_PARTS];

// device address of g_sum_partials per device, looked up once per device
std::mutex g_mutex;
double* g_partials_addr[NOALLOC_MAX_DEVICES] = {};

// velocity components of direction q in the D3Q19 order of include/psm.h
__device__ __forceinline__ void velocity(int q, int& cx, int& cy, int& cz) {
  const int k = (q - 1) >> 1;              // opposite pair of q >= 1
  const int sgn = (q & 1) ? 1 : -1;
  const int ax[9] = {1, 0, 0, 1, 1, 1, 1, 0, 0};
  const int ay[9] = {0, 1, 0, 1, -1, 0, 0, 1, 1};
  const int az[9] = {0, 0, 1, 0, 0, 1, -1, 1, -1};
  cx = sgn * ax[k];
  cy = sgn * ay[k];
  cz = sgn * az[k];
}

// one block per run of NOALLOC_CELLS_PER_PART cells: its four sums go to
// partials[4 * block + i] (mass, momentum x, y, z)
__global__ void __launch_bounds__(NOALLOC_THREADS)
sums_part_kernel(const double* __restrict__ f, long long ncells, double* partials) {
  __shared__ double sh[4][NOALLOC_THREADS];
  const long long lo = (long long)blockIdx.x * NOALLOC_CELLS_PER_PART;
  const long long hi = lo + NOALLOC_CELLS_PER_PART < ncells ? lo + NOALLOC_CELLS_PER_PART : ncells;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (long long c = lo + threadIdx.x; c < hi; c += NOALLOC_THREADS) {
    double m = f[c], jx = 0.0, jy = 0.0, jz = 0.0;
    for (int q = 1; q < 19; ++q) {
      const double v = f[(long long)q * ncells + c];
      int cx, cy, cz;
      velocity(q, cx, cy, cz);
      m += v;
      jx += cx * v;
      jy += cy * v;
      jz += cz * v;
    }
    acc[0] += m;
    acc[1] += jx;
    acc[2] += jy;
    acc[3] += jz;
  }
  for (int i = 0; i < 4; ++i) sh[i][threadIdx.x] = acc[i];
  __syncthreads();
  for (int s = NOALLOC_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int i = 0; i < 4; ++i) sh[i][threadIdx.x] += sh[i][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int i = 0; i < 4; ++i) partials[4 * blockIdx.x + i] = sh[i][0];
}

// fixed-order sum of the nparts partials into out[0..3]
__global__ void __launch_bounds__(NOALLOC_THREADS)
sums_final_kernel(const double* partials, int nparts, double* out) {
  __shared__ double sh[4][NOALLOC_THREADS];
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int b = threadIdx.x; b < nparts; b += NOALLOC_THREADS)
    for (int i = 0; i < 4; ++i) acc[i] += partials[4 * b + i];
  for (int i = 0; i < 4; ++i) sh[i][threadIdx.x] = acc[i];
  __syncthreads();
  for (int s = NOALLOC_THREADS / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s)
      for (int i = 0; i < 4; ++i) sh[i][threadIdx.x] += sh[i][threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int i = 0; i < 4; ++i) out[i] = sh[i][0];
}

}  // namespace

extern "C" psm_status psm_field_sums_noalloc(const double* f, long long ncells, double* sums,
                                              void* stream) {
  if (!f || !sums || ncells <= 0) return PSM_ERR_ARG;
  if (ncells > (long long)NOALLOC_MAX_PARTS * NOALLOC_CELLS_PER_PART) return PSM_ERR_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
    cudaGetLastError();
    return PSM_ERR_CUDA;
  }
  double* partials = nullptr;
  {
    // set-up on the first call on this device (the current one)
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_partials_addr[dev]) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_sum_partials) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return PSM_ERR_CUDA;
      }
      g_partials_addr[dev] = static_cast<double*>(ptr);
    }
    partials = g_partials_addr[dev];
  }
  const int nparts = (int)((ncells + NOALLOC_CELLS_PER_PART - 1) / NOALLOC_CELLS_PER_PART);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  sums_part_kernel<<<nparts, NOALLOC_THREADS, 0, s>>>(f, ncells, partials);
  sums_final_kernel<<<1, NOALLOC_THREADS, 0, s>>>(partials, nparts, sums);
  if (cudaGetLastError() != cudaSuccess) return PSM_ERR_CUDA;
  return PSM_OK;
}
