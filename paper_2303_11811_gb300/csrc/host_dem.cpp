// host_dem.cpp -- particle dynamics of one LBM step on the host cores (see
// host_dem.h).  Threads own contiguous ranges of particles and meet at a
// spinning barrier between phases: position update, partner lists, then per
// sub-step the contacts of the current state (double-buffered positions and
// velocities) and the Verlet update.
#include "host_dem.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <thread>
#include <vector>

namespace psm {
namespace {

constexpr double PI = 3.14159265358979323846;

// damping coefficient of Eq. 12 from the restitution coefficient
double damping(double meff, double kn, double le) {
  return -2.0 * le * std::sqrt(meff * kn) / std::sqrt(PI * PI + le * le);
}

double min_image(double v, double dim, bool periodic) {
  if (periodic) {
    if (v > 0.5 * dim) v -= dim;
    else if (v < -0.5 * dim) v += dim;
  }
  return v;
}

// Spinning barrier that a failing thread can abort: wait() then returns
// false in every thread (those waiting and those arriving later), so no
// thread is left spinning for a partner that stopped.
class SpinBarrier {
 public:
  explicit SpinBarrier(int n) : n_(n) {}
  bool wait() {
    if (n_ == 1) return !aborted();
    const int g = gen_.load(std::memory_order_acquire);
    if (count_.fetch_add(1, std::memory_order_acq_rel) == n_ - 1) {
      count_.store(0, std::memory_order_relaxed);
      gen_.fetch_add(1, std::memory_order_acq_rel);
    } else {
      while (gen_.load(std::memory_order_acquire) == g) {
        if (aborted()) return false;
        std::this_thread::yield();
      }
    }
    return !aborted();
  }
  void abort() { abort_.store(true, std::memory_order_release); }
  bool aborted() const { return abort_.load(std::memory_order_acquire); }

 private:
  const int n_;
  std::atomic<int> count_{0};
  std::atomic<int> gen_{0};
  std::atomic<bool> abort_{false};
};

struct Step {
  const HostDemParams& P;
  HostDemState& S;
  double dims[3];
  bool periodic[3];
  std::vector<double> x2, u2, om2;     // second buffers of positions and velocities
  std::vector<int> hcnt2, hj2;         // second buffer of the contact history
  std::vector<double> hd2;
  std::vector<double> xb;              // positions the partner lists were built from
  std::vector<std::vector<int>> cand;  // partners within contact distance + skin
  int nc[3] = {1, 1, 1};
  double h[3] = {1.0, 1.0, 1.0};
  std::vector<int> bin_start, bin_items;
  std::atomic<int> moved{0};
  mutable std::atomic<int> overflow{0};  // a particle in contact with more than kHostDemHistCap others

  Step(const HostDemParams& p, HostDemState& s) : P(p), S(s) {
    for (int a = 0; a < 3; ++a) {
      dims[a] = (double)P.dims[a];
      periodic[a] = !P.wall[a];
    }
    x2.resize(3 * (size_t)S.n);
    u2.resize(3 * (size_t)S.n);
    om2.resize(3 * (size_t)S.n);
    hcnt2.resize((size_t)S.n);
    hj2.resize((size_t)S.n * kHostDemHistCap);
    hd2.resize((size_t)S.n * kHostDemHistCap * 3);
    xb.resize(3 * (size_t)S.n);
    cand.resize(S.n);
  }

  // positions at the start of the step from the last sub-step's velocity and
  // force (Eq. 15)
  void position(int i) {
    if (S.fixed[i]) return;
    const double dt = P.dt;
    const double h2m = dt * dt / (2.0 * S.m[i]);
    for (int a = 0; a < 3; ++a) {
      double xn = S.x[3 * i + a] + dt * S.u[3 * i + a] + h2m * S.Fold[3 * i + a];
      if (periodic[a]) {
        if (xn >= dims[a]) xn -= dims[a];
        else if (xn < 0.0) xn += dims[a];
      }
      S.x[3 * i + a] = xn;
    }
  }

  int bin_of(double v, int a) const {
    int b = (int)std::floor(v / h[a]);
    return b < 0 ? 0 : (b >= nc[a] ? nc[a] - 1 : b);
  }

  // counting sort of the particles into bins of edge >= largest diameter + skin
  void bins() {
    double rmax = 0.0;
    for (int i = 0; i < S.n; ++i) rmax = std::max(rmax, S.r[i]);
    for (int a = 0; a < 3; ++a) {
      nc[a] = std::max(1, (int)std::floor(dims[a] / (2.0 * rmax + P.skin)));
      h[a] = dims[a] / nc[a];
    }
    const int nb = nc[0] * nc[1] * nc[2];
    std::vector<int> pb(S.n);
    bin_start.assign(nb + 1, 0);
    for (int i = 0; i < S.n; ++i) {
      pb[i] = bin_of(S.x[3 * i], 0) +
              nc[0] * (bin_of(S.x[3 * i + 1], 1) + nc[1] * bin_of(S.x[3 * i + 2], 2));
      ++bin_start[pb[i] + 1];
    }
    for (int b = 0; b < nb; ++b) bin_start[b + 1] += bin_start[b];
    std::vector<int> cur(bin_start.begin(), bin_start.end() - 1);
    bin_items.resize(S.n);
    for (int i = 0; i < S.n; ++i) bin_items[cur[pb[i]]++] = i;
  }

  int axis_bins(int a, int b, int* out) const {
    if (nc[a] < 3) {
      for (int k = 0; k < nc[a]; ++k) out[k] = k;
      return nc[a];
    }
    int m = 0;
    for (int o = -1; o <= 1; ++o) {
      int v = b + o;
      if (v < 0 || v >= nc[a]) {
        if (!periodic[a]) continue;
        v = v < 0 ? v + nc[a] : v - nc[a];
      }
      out[m++] = v;
    }
    return m;
  }

  void partners(int i) {
    for (int a = 0; a < 3; ++a) xb[3 * i + a] = S.x[3 * i + a];
    int bx[3], by[3], bz[3];
    const int nbx = axis_bins(0, bin_of(S.x[3 * i], 0), bx);
    const int nby = axis_bins(1, bin_of(S.x[3 * i + 1], 1), by);
    const int nbz = axis_bins(2, bin_of(S.x[3 * i + 2], 2), bz);
    std::vector<int>& L = cand[i];
    L.clear();
    for (int c = 0; c < nbz; ++c)
      for (int bb = 0; bb < nby; ++bb)
        for (int aa = 0; aa < nbx; ++aa) {
          const int b = bx[aa] + nc[0] * (by[bb] + nc[1] * bz[c]);
          for (int k = bin_start[b]; k < bin_start[b + 1]; ++k) {
            const int j = bin_items[k];
            if (j == i) continue;
            double d2 = 0.0;
            for (int a = 0; a < 3; ++a) {
              const double d = min_image(S.x[3 * i + a] - S.x[3 * j + a], dims[a], periodic[a]);
              d2 += d * d;
            }
            const double reach = S.r[i] + S.r[j] + P.skin;
            if (d2 < reach * reach) L.push_back(j);
          }
        }
    std::sort(L.begin(), L.end());
  }

  // history buffer b of particle i: counts, partners, delta_t
  int* hc(int b) { return b ? hcnt2.data() : S.hcnt; }
  int* hjb(int b, int i) { return (b ? hj2.data() : S.hj) + (size_t)i * kHostDemHistCap; }
  double* hdb(int b, int i) {
    return (b ? hd2.data() : S.hd) + (size_t)i * kHostDemHistCap * 3;
  }

  struct Cursor {
    const int* oj;
    const double* od;
    int nold, po;
    int* nj;
    double* nd;
    int nnew;
  };

  // exact contact of i with j at the current state (Eq. 12, and Eqs. 13-14
  // with the device DEM's readings), added to F and T
  void pair_contact(const double* X, const double* U, const double* W, int i, int j, double* F,
                    double* T, Cursor& H) const {
    double d[3];
    for (int a = 0; a < 3; ++a) d[a] = min_image(X[3 * i + a] - X[3 * j + a], dims[a], periodic[a]);
    const double dist2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    const double rs = S.r[i] + S.r[j];
    if (!(dist2 < rs * rs)) return;
    const double dist = std::sqrt(dist2);
    const double delta = rs - dist;
    const double n[3] = {d[0] / dist, d[1] / dist, d[2] / dist};
    const double vrel[3] = {U[3 * i] - U[3 * j], U[3 * i + 1] - U[3 * j + 1],
                            U[3 * i + 2] - U[3 * j + 2]};
    const double vn = vrel[0] * n[0] + vrel[1] * n[1] + vrel[2] * n[2];
    const double meff = S.m[i] * S.m[j] / (S.m[i] + S.m[j]);
    const double dn = damping(meff, P.kn, P.log_e);
    for (int a = 0; a < 3; ++a) F[a] += P.kn * delta * n[a] - dn * vn * n[a];
    if (!(P.kt_ratio > 0.0)) return;
    const double ai = -(S.r[i] - 0.5 * delta), aj = S.r[j] - 0.5 * delta;
    const double Ai[3] = {ai * n[0], ai * n[1], ai * n[2]};
    const double Aj[3] = {aj * n[0], aj * n[1], aj * n[2]};
    const double* wi = W + 3 * i;
    const double* wj = W + 3 * j;
    const double Ucp[3] = {
        (U[3 * i + 0] + (wi[1] * Ai[2] - wi[2] * Ai[1])) -
            (U[3 * j + 0] + (wj[1] * Aj[2] - wj[2] * Aj[1])),
        (U[3 * i + 1] + (wi[2] * Ai[0] - wi[0] * Ai[2])) -
            (U[3 * j + 1] + (wj[2] * Aj[0] - wj[0] * Aj[2])),
        (U[3 * i + 2] + (wi[0] * Ai[1] - wi[1] * Ai[0])) -
            (U[3 * j + 2] + (wj[0] * Aj[1] - wj[1] * Aj[0]))};
    const double un = Ucp[0] * n[0] + Ucp[1] * n[1] + Ucp[2] * n[2];
    const double Ut[3] = {Ucp[0] - un * n[0], Ucp[1] - un * n[1], Ucp[2] - un * n[2]};
    double h[3] = {0.0, 0.0, 0.0};
    while (H.po < H.nold && H.oj[H.po] < j) ++H.po;
    if (H.po < H.nold && H.oj[H.po] == j)
      for (int a = 0; a < 3; ++a) h[a] = H.od[3 * H.po + a];
    const double hn = h[0] * n[0] + h[1] * n[1] + h[2] * n[2];
    for (int a = 0; a < 3; ++a) h[a] = (h[a] - hn * n[a]) + P.dt * Ut[a];
    const double kt = P.kt_ratio * P.kn, dtg = P.kt_ratio * dn;
    const double Ft[3] = {-kt * h[0] - dtg * Ut[0], -kt * h[1] - dtg * Ut[1],
                          -kt * h[2] - dtg * Ut[2]};
    for (int a = 0; a < 3; ++a) F[a] += Ft[a];
    T[0] += Ai[1] * Ft[2] - Ai[2] * Ft[1];
    T[1] += Ai[2] * Ft[0] - Ai[0] * Ft[2];
    T[2] += Ai[0] * Ft[1] - Ai[1] * Ft[0];
    if (H.nnew < kHostDemHistCap) {
      H.nj[H.nnew] = j;
      for (int a = 0; a < 3; ++a) H.nd[3 * H.nnew + a] = h[a];
      ++H.nnew;
    } else {
      overflow.store(1, std::memory_order_relaxed);
    }
  }

  void wall_contacts(const double* X, const double* U, int i, double* F) const {
    for (int a = 0; a < 3; ++a) {
      if (periodic[a]) continue;
      for (int side = 0; side < 2; ++side) {
        const double delta = side == 0 ? S.r[i] - X[3 * i + a] : X[3 * i + a] + S.r[i] - dims[a];
        if (!(delta > 0.0)) continue;
        const double nn = side == 0 ? 1.0 : -1.0;
        const double vn = U[3 * i + a] * nn;
        const double dn = damping(S.m[i], P.kn, P.log_e);
        F[a] += P.kn * delta * nn - dn * vn * nn;
      }
    }
  }

  // one sub-step of particle i: contacts at (Xc, Uc, Wc) with the history of
  // buffer hb, velocity and angular velocity (Eq. 16) and, except on the
  // last sub-step, the next positions (Eq. 15) into (Xn, Un, Wn), the
  // history into buffer 1 - hb
  void substep(int i, const double* Xc, const double* Uc, const double* Wc, double* Xn,
               double* Un, double* Wn, int hb, bool last) {
    double F[3] = {0.0, 0.0, 0.0}, T[3] = {0.0, 0.0, 0.0};
    Cursor H{hjb(hb, i), hdb(hb, i), P.kt_ratio > 0.0 ? hc(hb)[i] : 0, 0, hjb(1 - hb, i),
             hdb(1 - hb, i), 0};
    for (int j : cand[i]) pair_contact(Xc, Uc, Wc, i, j, F, T, H);
    hc(1 - hb)[i] = H.nnew;
    wall_contacts(Xc, Uc, i, F);
    const double dt = P.dt;
    double u[3], x[3], w[3];
    for (int a = 0; a < 3; ++a) {
      u[a] = Uc[3 * i + a];
      x[a] = Xc[3 * i + a];
      w[a] = Wc[3 * i + a];
    }
    if (!S.fixed[i]) {
      const double hm = dt / (2.0 * S.m[i]), hI = dt / (2.0 * S.I[i]), h2m = dt * hm;
      for (int a = 0; a < 3; ++a) {
        const double Fn = S.Fh[3 * i + a] + F[a] + (S.m[i] - S.vol[i]) * P.gravity[a];
        const double Tn = S.Th[3 * i + a] + T[a];
        u[a] += hm * (S.Fold[3 * i + a] + Fn);
        w[a] += hI * (S.Told[3 * i + a] + Tn);
        S.Fold[3 * i + a] = Fn;
        S.Told[3 * i + a] = Tn;
      }
      if (!last) {
        for (int a = 0; a < 3; ++a) {
          double xn = x[a] + dt * u[a] + h2m * S.Fold[3 * i + a];
          if (periodic[a]) {
            if (xn >= dims[a]) xn -= dims[a];
            else if (xn < 0.0) xn += dims[a];
          }
          x[a] = xn;
        }
      }
      double e2 = 0.0;
      for (int a = 0; a < 3; ++a) {
        const double e = min_image(x[a] - xb[3 * i + a], dims[a], periodic[a]);
        e2 += e * e;
      }
      if (e2 > 0.25 * P.skin * P.skin) moved.store(1, std::memory_order_relaxed);
    }
    for (int a = 0; a < 3; ++a) {
      Un[3 * i + a] = u[a];
      Xn[3 * i + a] = x[a];
      Wn[3 * i + a] = w[a];
    }
  }

  // the phases of one step for the particles of thread t; returns early
  // (leaving the step unfinished) when the barrier was aborted
  void phases(int t, int nt, SpinBarrier& bar) {
    const int lo = (int)((long long)S.n * t / nt), hi = (int)((long long)S.n * (t + 1) / nt);
    for (int i = lo; i < hi; ++i) position(i);
    if (!bar.wait()) return;
    if (t == 0) bins();
    if (!bar.wait()) return;
    for (int i = lo; i < hi; ++i) partners(i);
    if (!bar.wait()) return;
    const double* Xc = S.x;
    const double* Uc = S.u;
    const double* Wc = S.om;
    for (int sc = 0; sc < P.subcycles; ++sc) {
      double* Xn = (sc % 2 == 0) ? x2.data() : S.x;
      double* Un = (sc % 2 == 0) ? u2.data() : S.u;
      double* Wn = (sc % 2 == 0) ? om2.data() : S.om;
      for (int i = lo; i < hi; ++i)
        substep(i, Xc, Uc, Wc, Xn, Un, Wn, sc & 1, sc + 1 == P.subcycles);
      if (!bar.wait()) return;
      Xc = Xn;
      Uc = Un;
      Wc = Wn;
    }
    if (Xc != S.x)
      for (int i = lo; i < hi; ++i) {
        for (int a = 0; a < 3; ++a) {
          S.x[3 * i + a] = Xc[3 * i + a];
          S.u[3 * i + a] = Uc[3 * i + a];
          S.om[3 * i + a] = Wc[3 * i + a];
        }
        const int c = hcnt2[i];
        S.hcnt[i] = c;
        for (int k = 0; k < c; ++k) {
          S.hj[(size_t)i * kHostDemHistCap + k] = hj2[(size_t)i * kHostDemHistCap + k];
          for (int a = 0; a < 3; ++a)
            S.hd[((size_t)i * kHostDemHistCap + k) * 3 + a] =
                hd2[((size_t)i * kHostDemHistCap + k) * 3 + a];
        }
      }
  }

  // a thread's part of the step; an exception (an allocation in the bins or
  // partner lists) marks the step failed and releases the other threads
  void run(int t, int nt, SpinBarrier& bar) {
    try {
      phases(t, nt, bar);
    } catch (...) {
      failed.store(1, std::memory_order_relaxed);
      bar.abort();
    }
  }
  std::atomic<int> failed{0};
};

}  // namespace

namespace {

// Starts nt - 1 workers parked on a flag, so that a failure to start one of
// them (std::system_error) leaves the particle state untouched: the started
// workers are released with an abort and joined, and the step runs on the
// calling thread alone.  Returns the number of threads the step ran on.
int run_threads(Step& st, int nt) {
  if (nt > 1) {
    SpinBarrier bar(nt);
    std::atomic<int> go{0};  // 1: run, -1: give up
    std::vector<std::thread> pool;
    bool started = true;
    try {
      pool.reserve(nt - 1);
      for (int t = 1; t < nt; ++t)
        pool.emplace_back([&st, &bar, &go, t, nt] {
          int g;
          while ((g = go.load(std::memory_order_acquire)) == 0) std::this_thread::yield();
          if (g > 0) st.run(t, nt, bar);
        });
    } catch (...) {
      started = false;
    }
    go.store(started ? 1 : -1, std::memory_order_release);
    if (started) st.run(0, nt, bar);
    for (auto& th : pool) th.join();
    if (started) return nt;
  }
  SpinBarrier one(1);
  st.run(0, 1, one);
  return 1;
}

}  // namespace

int host_dem_step(const HostDemParams& P, HostDemState& S, int threads) {
  if (S.n <= 0) return 0;
  // a thread per 256 particles at most: below that, starting threads and
  // meeting at the 13 barriers of a step costs more than the work (400
  // spheres: 0.31 ms per step on one core, 0.79 ms on eight)
  int nt = threads < 1 ? 1 : threads;
  nt = std::min(nt, std::max(1, S.n / 256));
  try {
    Step st(P, S);
    run_threads(st, nt);
    if (st.failed.load()) return -1;
    return (st.moved.load() || st.overflow.load()) ? 1 : 0;
  } catch (...) {  // the step's own buffers could not be allocated
    return -1;
  }
}

}  // namespace psm
