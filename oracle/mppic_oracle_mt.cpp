// Multithreaded driver of the FP64 oracle, for the all-core CPU baseline of the benchmark.
//
// TEST INFRASTRUCTURE ONLY, like the oracle itself: nothing on the product path loads it.
// It includes mppic_oracle.cpp unchanged and runs the same per-parcel and per-node functions
// over OpenMP threads; it adds no blocking or fusion to the arithmetic. Each thread owns a
// fixed contiguous range of parcels (np * t / nt .. np * (t + 1) / nt) and its own node
// arrays for the deposits; the per-thread node arrays and partial sums are added in thread
// order, so a run is deterministic for a given thread count. Node passes (node fields, the
// gas iterations of implicit coupling) run serially, as in the oracle.

#include "mppic_oracle.cpp"

#include <omp.h>

namespace {

// Sums per-thread node arrays into `out` in thread order (parallel over nodes).
void reduce_nodes(const std::vector<std::vector<double>>& parts, std::vector<double>& out,
                  long n, int nt) {
  out.assign(n, 0.0);
#pragma omp parallel for num_threads(nt) schedule(static)
  for (long i = 0; i < n; ++i) {
    double s = 0.0;
    for (size_t t = 0; t < parts.size(); ++t) s += parts[t][i];
    out[i] = s;
  }
}

int step_once_mt(const orc_config& c, const Grid& G, const Params<double>& P, long np, double* x,
                 double* y, double* z, double* u, double* v, double* w, const double* d,
                 const double* om, const double* const U[3], const double* const GP[3], int nt,
                 double& dP, double& H) {
  auto lo = [&](int t) { return np * t / nt; };
  std::vector<std::vector<double>> part(nt), partB(nt);
  std::vector<double> Vs, eps_s, ug, tau, A, B;
  // deposit of the solids volume: each thread its parcel range
#pragma omp parallel num_threads(nt)
  {
    const int t = omp_get_thread_num();
    const long a = lo(t), b = lo(t + 1);
    deposit_volume(G, P, b - a, x + a, y + a, z + a, d + a, om + a, part[t]);
  }
  reduce_nodes(part, Vs, G.nnode, nt);
  node_fields(c, G, P, Vs, U, eps_s, ug, tau);
  // implicit coupling: the drag sums at the head of every gas iteration
  for (int m = 0; m < c.coupling_iters; ++m) {
#pragma omp parallel num_threads(nt)
    {
      const int t = omp_get_thread_num();
      const long a = lo(t), b = lo(t + 1);
      drag_sums(c, G, P, b - a, x + a, y + a, z + a, u + a, v + a, w + a, d + a, om + a, eps_s,
                ug, tau, GP, part[t], partB[t]);
    }
    reduce_nodes(part, A, G.nnode, nt);
    reduce_nodes(partB, B, 3 * G.nnode, nt);
    gas_update(c, G, P, eps_s, U, A, B, ug);
  }
  // the parcel update: per-thread drag sums and objective partials
  std::vector<double> dps(nt, 0.0), hns(nt, 0.0), vss(nt, 0.0);
  std::vector<int> sts(nt, 0);
#pragma omp parallel num_threads(nt)
  {
    const int t = omp_get_thread_num();
    part[t].assign(G.nnode, 0.0);
    partB[t].assign(3 * G.nnode, 0.0);
    sts[t] = push_parcels(c, G, P, lo(t), lo(t + 1), x, y, z, u, v, w, d, om, nullptr, GP, eps_s,
                          ug, tau, part[t], partB[t], dps[t], hns[t], vss[t]);
  }
  double dPsum = 0.0, Hnum = 0.0, Vsum = 0.0;
  int status = 0;
  for (int t = 0; t < nt; ++t) {
    dPsum += dps[t];
    Hnum += hns[t];
    Vsum += vss[t];
    if (sts[t]) status = sts[t];
  }
  dP = dPsum / (G.L[0] * G.L[1]);
  H = 2.0 * Hnum / Vsum;
  return status;
}

}  // namespace

extern "C" {

// nsteps coupling steps in place on nthreads threads (0 = all the OpenMP runtime offers);
// obj[2*nsteps] (may be NULL) receives per step (dP, H). Returns 0 or 4.
int orc_step_mt(const orc_config* c, long np, double* x, double* y, double* z, double* u,
                double* v, double* w, const double* d, const double* om, const double* Ux,
                const double* Uy, const double* Uz, int nsteps, double* obj, int nthreads) {
  Grid G(*c);
  Params<double> P{c->drag_mult, c->dscale, c->u_in};
  const double* U[3] = {Ux, Uy, Uz};
  const double* GP[3] = {nullptr, nullptr, nullptr};
  const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();
  int status = 0;
  for (int s = 0; s < nsteps; ++s) {
    double dP = 0.0, H = 0.0;
    int st = step_once_mt(*c, G, P, np, x, y, z, u, v, w, d, om, U, GP, nt, dP, H);
    if (st) status = st;
    if (obj) { obj[2 * s] = dP; obj[2 * s + 1] = H; }
  }
  return status;
}

// Threads the OpenMP runtime offers.
int orc_max_threads() { return omp_get_max_threads(); }

}  // extern "C"
