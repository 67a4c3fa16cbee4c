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
#include <cuda.h>  // CUcontext and CUresult types only; the functions come by entry point
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/psm.h"

namespace {

constexpr int NOALLOC_MAX_PARTS = 4096;
constexpr long long NOALLOC_CELLS_PER_PART = 65536;
constexpr int NOALLOC_THREADS = 256;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) double g_sum_partials[4 * NOALLOC_MAX_PARTS];

// Device address of g_sum_partials per device, looked up once per CUDA
// context: a cudaDeviceReset (or another context made current on the device)
// loads the module again, possibly at another address, so each cached
// address is kept with the id of the context it was looked up in (context
// ids are unique within a process) and looked up again when that changes.
struct PartialsAddr {
  unsigned long long ctx_id;
  double* addr;
};
std::mutex g_mutex;
PartialsAddr g_partials[NOALLOC_MAX_DEVICES] = {};

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;

// id of the context current on the calling thread (the runtime makes the
// device's primary context current if none is); false on failure
bool current_context_id(unsigned long long* id) {
  if (!g_ctx_get_current || !g_ctx_get_id) {
    void* f1 = nullptr;
    void* f2 = nullptr;
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) !=
            cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || !f1)
      return false;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) !=
            cudaSuccess ||
        q2 != cudaDriverEntryPointSuccess || !f2)
      return false;
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(f1);
    g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(f2);
  }
  CUcontext ctx = nullptr;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return false;
  if (!ctx) {
    // no context current on this thread yet: cudaSetDevice initialises the
    // device's primary context and makes it current (it allocates nothing)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess) return false;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
  }
  return g_ctx_get_id(ctx, id) == CUDA_SUCCESS;
}

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
    // set-up on the first call in each context of this device (the current one)
    std::lock_guard<std::mutex> lock(g_mutex);
    unsigned long long ctx_id = 0;
    if (!current_context_id(&ctx_id)) {
      cudaGetLastError();
      return PSM_ERR_CUDA;
    }
    if (!g_partials[dev].addr || g_partials[dev].ctx_id != ctx_id) {
      void* ptr = nullptr;
      if (cudaGetSymbolAddress(&ptr, g_sum_partials) != cudaSuccess || !ptr) {
        cudaGetLastError();
        return PSM_ERR_CUDA;
      }
      g_partials[dev].addr = static_cast<double*>(ptr);
      g_partials[dev].ctx_id = ctx_id;
    }
    partials = g_partials[dev].addr;
  }
  const int nparts = (int)((ncells + NOALLOC_CELLS_PER_PART - 1) / NOALLOC_CELLS_PER_PART);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  sums_part_kernel<<<nparts, NOALLOC_THREADS, 0, s>>>(f, ncells, partials);
  sums_final_kernel<<<1, NOALLOC_THREADS, 0, s>>>(partials, nparts, sums);
  if (cudaGetLastError() != cudaSuccess) return PSM_ERR_CUDA;
  return PSM_OK;
}
