// host_dem.h -- particle dynamics on the host cores: the coupling the paper
// runs (Sec. 3.2: the DEM on the CPU, with the hydrodynamic forces sent from
// the GPU and the particle state sent back every LBM step).  The engine's own
// step keeps the DEM on the device; this form exists to measure that split.
//
// The arithmetic is the device DEM's (dem_kernels.cu): velocity Verlet with
// sub-cycling (Eqs. 15-16), linear spring-dashpot normal contacts between
// spheres and with the wall faces (Eq. 12), tangential contacts with history
// between spheres (Eqs. 13-14), buoyancy-corrected gravity, the
// hydrodynamic force and torque held over the sub-steps; the same IEEE FP64
// operations in the same order (partners in ascending index, then the walls),
// so the two forms agree to the last bit.
#pragma once

namespace psm {

// partners per particle in the tangential contact history (the device DEM's
// neighbour-list capacity)
constexpr int kHostDemHistCap = 64;

struct HostDemParams {
  int dims[3];      // nx, ny, nz
  int wall[3];      // 1: walls on both faces of the axis, 0: periodic
  double kn;        // normal spring stiffness
  double kt_ratio;  // tangential contact: k_t = kt_ratio k_n, d_t = kt_ratio d_n (0: off)
  double log_e;     // ln(restitution)
  double dt;        // sub-step, 1 / subcycles
  double gravity[3];
  double skin;      // partner lists: contact distance plus this margin
  int subcycles;
};

// Particle state in host memory (n particles, vectors as n*3).  x, u, om,
// Fold and Told are read and advanced by one LBM step; Fh, Th (hydrodynamic
// force and torque of the step) and the constants are read only.
struct HostDemState {
  int n;
  double *x, *u, *om, *Fold, *Told;
  const double *Fh, *Th, *r, *m, *I, *vol;
  const unsigned char* fixed;
  // tangential contact history, read and advanced: per particle the count,
  // the partners (ascending, kHostDemHistCap per particle) and delta_t (3 each)
  int* hcnt;
  int* hj;
  double* hd;
};

// One LBM step of particle dynamics on up to `threads` host threads (at
// most one per 256 particles).
// Returns 0, 1 when a particle moved more than half the skin within the
// step (its partner list may then have missed a contact), or -1 when host
// memory for the step's buffers ran out (the state is then partly advanced).
// Throws nothing: a worker thread that cannot be started makes the step run
// on fewer threads, with the same result.
int host_dem_step(const HostDemParams& P, HostDemState& S, int threads);

}  // namespace psm
