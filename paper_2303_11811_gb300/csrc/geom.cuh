// geom.cuh -- sub-division sampling of a cell against a sphere (paper
// Sec. 2.3.2), shared by the mapping and the surrogate's training sampler.
// Plain IEEE FP64 operations; files including it are compiled with -fmad=false.
#pragma once

namespace psm {

constexpr double kHalfSqrt3 = 0.86602540378443864676;

// number of the n^3 sub-cell centres d + s, s_a = (a + 1/2)/n - 1/2, that lie
// inside the sphere of radius r centred at the origin (|p|^2 <= r^2)
__device__ inline int supersample_count(double dx, double dy, double dz, double r, int n) {
  const double r2 = r * r;
  int count = 0;
  for (int a = 0; a < n; ++a) {
    const double sx = (a + 0.5) / n - 0.5;
    const double px = dx + sx;
    const double X = px * px;
    for (int b = 0; b < n; ++b) {
      const double sy = (b + 0.5) / n - 0.5;
      const double py = dy + sy;
      const double XY = X + py * py;
      for (int c = 0; c < n; ++c) {
        const double sz = (c + 0.5) / n - 0.5;
        const double pz = dz + sz;
        if (XY + pz * pz <= r2) ++count;
      }
    }
  }
  return count;
}

}  // namespace psm
