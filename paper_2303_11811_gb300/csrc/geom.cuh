// geom.cuh -- sub-division sampling of a cell against a sphere (paper
// Sec. 2.3.2), shared by the mapping and the surrogate's training sampler.
//
// The definition is an FP64 computation: sample offsets
//   s_a = (a + 1/2)/n - 1/2,  p = d + s,  inside <=> ((p_x^2 + p_y^2) + p_z^2) <= r^2
// with every operation rounded in FP64 (files including this are compiled with
// -fmad=false).  FP64 runs at 1/64 of the FP32 rate on this GPU, so the count
// is evaluated in FP32 and a sample goes to the FP64 definition only when its
// FP32 value lies within a certified bound E of r^2:
//   |S_fp32 - S_fp64| <= 2^-19 (r + 2.5)^2 for |d| <= r + 2 (each of the three
//   squared terms is off by at most 2^-21 (r + 2.5)^2, the two sums by
//   2^-24 S each), |fl32(r^2) - r^2| <= 2^-24 r^2, so E = 2^-18 (r + 2.5)^2.
// Outside that band the FP32 decision equals the FP64 one, so the count is
// exactly the FP64 definition's.
#pragma once

namespace psm {

constexpr double kHalfSqrt3 = 0.86602540378443864676;

__device__ __forceinline__ double sample_offset(int a, int n) { return (a + 0.5) / n - 0.5; }

// FP64 definition for one sample point
__device__ __forceinline__ bool sample_inside_fp64(double dx, double dy, double dz, double sx,
                                                   double sy, double sz, double r2) {
  const double px = dx + sx, py = dy + sy, pz = dz + sz;
  return px * px + py * py + pz * pz <= r2;
}

__device__ __forceinline__ float certified_band(double r) {
  const float q = (float)r + 2.5f;
  return 3.8147e-6f * q * q;  // 2^-18 (r + 2.5)^2, rounded up
}

// count of the n^3 sample points inside; s64/s32 hold the n offsets
__device__ inline int supersample_count_fast(double dx, double dy, double dz, double r, int n,
                                             const double* s64, const float* s32) {
  const double r2 = r * r;
  const float r2f = (float)r2;
  const float E = certified_band(r);
  const float lo = r2f - E, hi = r2f + E;
  const float dxf = (float)dx, dyf = (float)dy, dzf = (float)dz;
  int count = 0;
  for (int a = 0; a < n; ++a) {
    const float px = dxf + s32[a];
    const float X = px * px;
    for (int b = 0; b < n; ++b) {
      const float py = dyf + s32[b];
      const float XY = X + py * py;
      for (int c = 0; c < n; ++c) {
        const float pz = dzf + s32[c];
        const float S = XY + pz * pz;
        if (S < lo) ++count;
        else if (S <= hi && sample_inside_fp64(dx, dy, dz, s64[a], s64[b], s64[c], r2)) ++count;
      }
    }
  }
  return count;
}

// the same count for a compile-time n (4 or 8): offsets are exact constants
// and the squared x, y, z terms of the sample rows are formed once.  The
// unrolled loop counts the samples certainly inside (S < lo) and those not
// certainly outside (S <= hi); when the counts agree no sample lies in the
// band, otherwise the cell is recounted with the FP64 test inside the band.
// dxf, dyf, dzf: the FP32 roundings of dx, dy, dz; r2f = (float)(r * r);
// E = certified_band(r) (callers with many cells of one sphere form them once)
template <int N>
__device__ inline int supersample_count_n(double dx, double dy, double dz, double r, float dxf,
                                          float dyf, float dzf, float r2f, float E) {
  const float lo = r2f - E, hi = r2f + E;
  float Y[N], Z[N];
#pragma unroll
  for (int a = 0; a < N; ++a) {
    const float s = (float)((a + 0.5) / N - 0.5);
    const float py = dyf + s, pz = dzf + s;
    Y[a] = py * py;
    Z[a] = pz * pz;
  }
  int in = 0, maybe = 0;
  // the x samples stay a loop for N = 8 (64 samples per pass): the fully
  // unrolled 512 samples overflow the instruction cache
#pragma unroll(N <= 4 ? N : 1)
  for (int a = 0; a < N; ++a) {
    // (a + 1/2)/N - 1/2 is exact in FP32 for N a power of two
    const float px = dxf + (((float)a + 0.5f) * (1.0f / N) - 0.5f);
    const float Xa = px * px;
#pragma unroll
    for (int b = 0; b < N; ++b) {
      const float XY = Xa + Y[b];
#pragma unroll
      for (int c = 0; c < N; ++c) {
        const float S = XY + Z[c];
        in += S < lo;
        maybe += S <= hi;
      }
    }
  }
  if (in == maybe) return in;
  double s64[N];
  float s32[N];
  for (int a = 0; a < N; ++a) {
    s64[a] = sample_offset(a, N);
    s32[a] = (float)s64[a];
  }
  return supersample_count_fast(dx, dy, dz, r, N, s64, s32);
}

template <int N>
__device__ inline int supersample_count_n(double dx, double dy, double dz, double r) {
  return supersample_count_n<N>(dx, dy, dz, r, (float)dx, (float)dy, (float)dz, (float)(r * r),
                                certified_band(r));
}

// FP64 definition, all samples (reference for small counts and tests)
__device__ inline int supersample_count(double dx, double dy, double dz, double r, int n) {
  const double r2 = r * r;
  int count = 0;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b)
      for (int c = 0; c < n; ++c)
        if (sample_inside_fp64(dx, dy, dz, sample_offset(a, n), sample_offset(b, n),
                               sample_offset(c, n), r2))
          ++count;
  return count;
}

}  // namespace psm
