// Reverse-mode (adjoint) kernels of the MP-PIC coupling step, for gradients of the
// time-averaged bed pressure drop and bed height with respect to the drag multiplier C,
// the diameter scale s_d and the inflow velocity u_in.
//
// The forward step they differentiate is the one of mppic_device.cuh (Woo et al.,
// arXiv 2211.15605, Sec. 2.1: Eqs. 3-5 with Wen-Yu drag, trilinear deposit and
// interpolation, semi-implicit drag, specular walls). Each backward step reads the
// state S_n, recomputes that step's node fields and per-parcel quantities, and maps the
// adjoint of S_{n+1} to the adjoint of S_n:
//   k_adj_parcel : reverse of push, walls, drag, objectives and interpolation weights;
//                  scatters the adjoints of the interpolated fields to the nodes
//                  (interp^T, a deposit);
//   k_adj_node   : reverse of the node fields (Eq. 5 and u_g = U / eps_g), giving the
//                  adjoint of the deposited volume;
//   k_adj_deposit: reverse of the volume deposit (deposit^T, a gather).
// The state recomputation inside a checkpoint segment uses k_dep_simple and
// k_push_simple, which evaluate the same arithmetic one parcel per thread without a sort.
// Node adjoints are accumulated with FP64 atomics (their last bits depend on ordering).
#pragma once

#include "mppic_device.cuh"

namespace mppic {

// Per-parcel forward quantities of one step, recomputed in the adjoint kernels.
template <class T>
struct Fwd {
  Cell3<T> c;
  T w[3][2];            // trilinear factors
  Interp<T> I;
  T s[3], smag, eg, de, rem, D1, D, V, f;
  bool eg_free;         // eps_g = 1 - eps_s (not floored)
  bool laminar;         // Re_m < 1000 branch
  T inv_den, inv_esr;
  T u1[3];              // velocity after the drag update, before walls
  bool refl[3];
};

template <class T>
__device__ __forceinline__ void forward_parcel(const KParams<T>& p, const Fields<T>& F, T x, T y,
                                               T z, T u, T v, T w, T d, T om, Fwd<T>& r) {
  bin3(p, x, y, z, r.c);
  for (int a = 0; a < 3; ++a) { r.w[a][0] = T(1) - r.c.xi[a]; r.w[a][1] = r.c.xi[a]; }
  interp8(p, F, p.has_gp != 0, node_id(p, r.c.i, r.c.j, r.c.k), 1, p.nx + 1,
          (long long)(p.nx + 1) * (p.ny + 1), r.c.xi, r.I);
  const T up[3] = {u, v, w};
  for (int a = 0; a < 3; ++a) r.s[a] = r.I.ug[a] - up[a];
  const T egr = T(1) - r.I.es;
  r.eg_free = egr >= p.eg_min;
  r.eg = r.eg_free ? egr : p.eg_min;
  r.de = p.sd * d;
  r.smag = fsqrt(r.s[0] * r.s[0] + r.s[1] * r.s[1] + r.s[2] * r.s[2]);
  r.rem = r.eg * r.de * r.smag * p.kRe;
  const T inv_de = frcp(r.de);
  const T e165 = fpow(r.eg, T(-1.65));
  r.laminar = r.rem < T(1000);
  if (r.laminar)
    r.D1 = p.kD1u * (T(1) + T(0.15) * fpow(r.rem, T(0.687))) * e165 * frcp(r.eg) * (inv_de * inv_de);
  else
    r.D1 = p.kD2u * r.smag * e165 * inv_de;
  r.D = p.C * r.D1;
  r.V = om * (d * d * d) * p.vcoef;
  r.f = p.rho_p * r.V * r.D;
  r.inv_den = frcp(T(1) + p.dt * r.D);
  r.inv_esr = r.I.es > T(1e-12) ? frcp(r.I.es * p.rho_p) : T(0);
  const T pos[3] = {x, y, z};
  for (int a = 0; a < 3; ++a) {
    const T acc = r.D * r.I.ug[a] + p.g[a] - r.I.gp[a] * p.inv_rho_p - r.I.gt[a] * r.inv_esr;
    r.u1[a] = (up[a] + p.dt * acc) * r.inv_den;
    const T xn = pos[a] + p.dt * r.u1[a];
    r.refl[a] = xn < T(0) || xn > p.L[a];
  }
}

// Solids-volume deposit, one parcel per thread, exact fixed point (no sort needed).
template <class T>
__global__ void k_dep_simple(KParams<T> p, const T* __restrict__ x, const T* __restrict__ y,
                             const T* __restrict__ z, const T* __restrict__ d,
                             const T* __restrict__ om, long long np) {
  constexpr int W = Words<T>::n;
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= np) return;
  Cell3<T> c;
  bin3(p, x[q], y[q], z[q], c);
  const T dq = d[q];
  const T V = om[q] * (dq * dq * dq) * p.vcoef;
  T w[3][2];
  for (int a = 0; a < 3; ++a) { w[a][0] = T(1) - c.xi[a]; w[a][1] = c.xi[a]; }
  for (int cc = 0; cc < 2; ++cc)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        u64 fx[W];
        to_fixed(V * ((w[0][a] * w[1][b]) * w[2][cc]), p.mV, fx, p.errs);
        acc_add(p.acc + p.nbase + node_id(p, c.i + a, c.j + b, c.k + cc), p.nstride, fx);
      }
}

// One forward step, one parcel per thread, in place (used to recompute segment states).
template <class T>
__global__ void k_push_simple(KParams<T> p, T* x, T* y, T* z, T* u, T* v, T* w,
                              const T* __restrict__ d, const T* __restrict__ om, long long np) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= np) return;
  Fields<T> F;
  for (int f = 0; f < 5; ++f) F.f[f] = p.fld[f];
  for (int a = 0; a < 3; ++a) F.g[a] = p.gpf[a];
  Fwd<T> r;
  forward_parcel(p, F, x[q], y[q], z[q], u[q], v[q], w[q], d[q], om[q], r);
  T pos[3] = {x[q], y[q], z[q]};
  bool bad = false;
  for (int a = 0; a < 3; ++a) {
    T un = r.u1[a];
    T xn = pos[a] + p.dt * un;
    if (xn < T(0)) { xn = -xn; un = -p.e_wall * un; }
    else if (xn > p.L[a]) { xn = T(2) * p.L[a] - xn; un = -p.e_wall * un; }
    if (!(xn >= T(0) && xn <= p.L[a]) || !isfinite(un)) bad = true;
    pos[a] = xn;
    if (a == 0) u[q] = un; else if (a == 1) v[q] = un; else w[q] = un;
  }
  if (bad) atomicOr(p.errs, ERR_DOMAIN);
  x[q] = pos[0]; y[q] = pos[1]; z[q] = pos[2];
}

// sums[0] += sum V z, sums[1] += sum V (for the bed height of a state).
template <class T>
__global__ void k_height_sums(KParams<T> p, const T* __restrict__ z, const T* __restrict__ d,
                              const T* __restrict__ om, long long np, double* sums) {
  __shared__ double sh[2][256];
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double vz = 0, vv = 0;
  if (q < np) {
    const T dq = d[q];
    const double V = (double)(om[q] * (dq * dq * dq) * p.vcoef);
    vz = V * (double)z[q];
    vv = V;
  }
  sh[0][threadIdx.x] = vz;
  sh[1][threadIdx.x] = vv;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) { sh[0][threadIdx.x] += sh[0][threadIdx.x + o]; sh[1][threadIdx.x] += sh[1][threadIdx.x + o]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { atomicAdd(&sums[0], sh[0][0]); atomicAdd(&sums[1], sh[1][0]); }
}

struct AdjWeights {
  double a_dp;   // dL/d(dP_n) / area
  double a_h;    // dL/d(H_n)
};

// Node adjoint planes: 0 eps_s, 1-3 u_g, 4 tau (interp^T); 5 Vs (finalize^T output).
// theta[0..2] accumulate dL/dC, dL/ds_d, dL/du_in.
template <class T>
__global__ void k_adj_parcel(KParams<T> p, const T* __restrict__ x, const T* __restrict__ y,
                             const T* __restrict__ z, const T* __restrict__ u,
                             const T* __restrict__ v, const T* __restrict__ w,
                             const T* __restrict__ d, const T* __restrict__ om, long long np,
                             double* __restrict__ xb, double* __restrict__ ub,
                             double* __restrict__ Vb, double* __restrict__ nadj,
                             const double* __restrict__ hsum, AdjWeights aw,
                             double* __restrict__ theta) {
  __shared__ double sh[2][256];
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double cbar = 0, sdbar = 0;
  if (q < np) {
    Fields<T> F;
    for (int f = 0; f < 5; ++f) F.f[f] = p.fld[f];
    for (int a = 0; a < 3; ++a) F.g[a] = p.gpf[a];
    Fwd<T> r;
    const T X[3] = {x[q], y[q], z[q]};
    const T Uv[3] = {u[q], v[q], w[q]};
    const T dq = d[q];
    forward_parcel(p, F, X[0], X[1], X[2], Uv[0], Uv[1], Uv[2], dq, om[q], r);
    const double dt = (double)p.dt;
    double xbar[3], ubar[3], u1b[3], accb[3];
    double Db = 0;
    for (int a = 0; a < 3; ++a) {
      // walls: x = -x1 or 2L - x1, u = -e u1
      const double x2b = xb[a * np + q], u2b = ub[a * np + q];
      const double x1b = r.refl[a] ? -x2b : x2b;
      u1b[a] = (r.refl[a] ? -(double)p.e_wall : 1.0) * u2b;
      // x1 = x + dt u1
      xbar[a] = x1b;
      u1b[a] += dt * x1b;
      // u1 = (u + dt acc) / (1 + dt D)
      ubar[a] = u1b[a] * (double)r.inv_den;
      accb[a] = u1b[a] * dt * (double)r.inv_den;
      Db -= u1b[a] * dt * (double)r.u1[a] * (double)r.inv_den;
    }
    // acc = D u_g + g - grad p / rho_p - grad tau / (eps_s rho_p)
    double ugb[3], gtb[3], gpb[3], esb = 0;
    for (int a = 0; a < 3; ++a) {
      Db += accb[a] * (double)r.I.ug[a];
      ugb[a] = accb[a] * (double)r.D;
      gpb[a] = -accb[a] * (double)p.inv_rho_p;
      gtb[a] = -accb[a] * (double)r.inv_esr;
      esb += accb[a] * (double)r.I.gt[a] * (double)r.inv_esr * (double)r.inv_esr * (double)p.rho_p;
    }
    // objectives: dP_n = sum f s_z / area, H_n = 2 sum V z / sum V
    const double fb = aw.a_dp * (double)r.s[2];
    double sb[3] = {0, 0, aw.a_dp * (double)r.f};
    const double SV = hsum[1], Hn = 2.0 * hsum[0] / hsum[1];
    xbar[2] += aw.a_h * 2.0 * (double)r.V / SV;
    double Vbar = aw.a_h * (2.0 * (double)X[2] - Hn) / SV;
    // f = rho_p V D
    Vbar += fb * (double)p.rho_p * (double)r.D;
    Db += fb * (double)p.rho_p * (double)r.V;
    // D = C D1(rem, eps_g, d_e); rem = eps_g d_e |s| rho_g / mu
    cbar += Db * (double)r.D1;
    const double D1b = Db * (double)p.C;
    double remb = 0, egb, deb, smagb;
    const double D1 = r.D1, eg = r.eg, de = r.de, rem = r.rem;
    if (r.laminar) {
      const double P = 1.0 + 0.15 * pow(rem, 0.687);
      const double dPdrem = rem > 0 ? 0.15 * 0.687 * pow(rem, 0.687) / rem : 0.0;
      remb = D1b * D1 / P * dPdrem;
      egb = D1b * (-2.65 * D1 / eg) + remb * rem / eg;
      deb = D1b * (-2.0 * D1 / de) + remb * rem / de;
      smagb = remb * eg * de * (double)p.kRe;
    } else {
      egb = D1b * (-1.65 * D1 / eg);
      deb = D1b * (-D1 / de);
      smagb = r.smag > T(0) ? D1b * D1 / (double)r.smag : 0.0;
    }
    sdbar += deb * (double)dq;
    if (r.eg_free) esb -= egb;
    if (r.smag > T(0))
      for (int a = 0; a < 3; ++a) sb[a] += smagb * (double)r.s[a] / (double)r.smag;
    // s = u_g - u
    for (int a = 0; a < 3; ++a) { ugb[a] += sb[a]; ubar[a] -= sb[a]; }
    // V = w pi/6 (s_d d)^3 (the deposit^T part of Vbar is added by k_adj_deposit)
    Vb[q] = Vbar;
    // interpolation: node adjoints (interp^T) and the position dependence of the weights
    const double inv[3] = {(double)p.invh[0], (double)p.invh[1], (double)p.invh[2]};
    for (int cc = 0; cc < 2; ++cc)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
          const long long n = node_id(p, r.c.i + a, r.c.j + b, r.c.k + cc);
          const double wa = r.w[0][a], wb = r.w[1][b], wc = r.w[2][cc];
          const double sa = a ? inv[0] : -inv[0], sbb = b ? inv[1] : -inv[1], sc = cc ? inv[2] : -inv[2];
          const double Wq = wa * wb * wc;
          const double dW[3] = {sa * wb * wc, sbb * wa * wc, sc * wa * wb};
          atomicAdd(&nadj[0 * p.nnode + n], Wq * esb);
          for (int k2 = 0; k2 < 3; ++k2) atomicAdd(&nadj[(1 + k2) * p.nnode + n], Wq * ugb[k2]);
          atomicAdd(&nadj[4 * p.nnode + n], dW[0] * gtb[0] + dW[1] * gtb[1] + dW[2] * gtb[2]);
          // d/dx of the interpolated values through the weights
          const double es_n = (double)p.fld[0][n], tau_n = (double)p.fld[4][n];
          double lin = es_n * esb;
          for (int k2 = 0; k2 < 3; ++k2) lin += (double)p.fld[1 + k2][n] * ugb[k2];
          if (p.has_gp)
            for (int k2 = 0; k2 < 3; ++k2) lin += (double)p.gpf[k2][n] * gpb[k2];
          // second derivatives of the weight (mixed only): d2W/dx dy = sa sbb wc, etc.
          const double dxy = sa * sbb * wc, dxz = sa * sc * wb, dyz = sbb * sc * wa;
          xbar[0] += dW[0] * lin + tau_n * (dxy * gtb[1] + dxz * gtb[2]);
          xbar[1] += dW[1] * lin + tau_n * (dxy * gtb[0] + dyz * gtb[2]);
          xbar[2] += dW[2] * lin + tau_n * (dxz * gtb[0] + dyz * gtb[1]);
        }
    for (int a = 0; a < 3; ++a) { xb[a * np + q] = xbar[a]; ub[a * np + q] = ubar[a]; }
  }
  sh[0][threadIdx.x] = cbar;
  sh[1][threadIdx.x] = sdbar;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) { sh[0][threadIdx.x] += sh[0][threadIdx.x + o]; sh[1][threadIdx.x] += sh[1][threadIdx.x + o]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) { atomicAdd(&theta[0], sh[0][0]); atomicAdd(&theta[1], sh[1][0]); }
}

// Reverse of the node fields: from the adjoints of eps_s, u_g and tau at a node to the
// adjoint of its deposited volume (plane 5), and the u_in part of the gradient.
template <class T>
__global__ void k_adj_node(KParams<T> p, double* __restrict__ nadj, double* __restrict__ theta) {
  __shared__ double sh[256];
  const int nx1 = p.nx + 1, ny1 = p.ny + 1;
  long long nn = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double uinb = 0;
  if (nn < p.nnode) {
    const int n = (int)nn;
    const int i = n % nx1, j = (n / nx1) % ny1, k = n / (nx1 * ny1);
    double vn = p.vcell;
    if (i == 0 || i == p.nx) vn *= 0.5;
    if (j == 0 || j == p.ny) vn *= 0.5;
    if (k == 0 || k == p.nz) vn *= 0.5;
    const double es = (double)p.fld[0][n];
    double esb = nadj[0 * p.nnode + n];
    // tau = Ps es^beta / max(eps_cp - es, alpha (1 - es))
    const double Ps = p.Ps, beta = p.beta, ecp = p.eps_cp, al = p.alpha;
    const double d1 = ecp - es, d2 = al * (1.0 - es);
    const bool first = d1 >= d2;
    const double den = first ? d1 : d2;
    const double dden = first ? -1.0 : -al;
    const double tau = Ps * pow(es, beta) / den;
    const double dtau = (es > 0 ? Ps * beta * pow(es, beta - 1.0) / den : 0.0) - tau / den * dden;
    esb += nadj[4 * p.nnode + n] * dtau;
    // u_g = U / max(1 - es, eg_min)
    const double egr = 1.0 - es;
    const bool free = egr >= (double)p.eg_min;
    const double egc = free ? egr : (double)p.eg_min;
    if (free)
      for (int a = 0; a < 3; ++a) esb += nadj[(1 + a) * p.nnode + n] * (double)p.fld[1 + a][n] / egc;
    uinb = nadj[3 * p.nnode + n] / egc;
    nadj[5 * p.nnode + n] = esb / vn;
  }
  sh[threadIdx.x] = uinb;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(&theta[2], sh[0]);
}

// Reverse of the volume deposit (a gather): Vbar_p += sum W Vsbar, xbar += V sum dW Vsbar;
// then the s_d part of the gradient through V = w pi/6 (s_d d)^3.
template <class T>
__global__ void k_adj_deposit(KParams<T> p, const T* __restrict__ x, const T* __restrict__ y,
                              const T* __restrict__ z, const T* __restrict__ d,
                              const T* __restrict__ om, long long np, double* __restrict__ xb,
                              const double* __restrict__ Vb, const double* __restrict__ nadj,
                              double* __restrict__ theta) {
  __shared__ double sh[256];
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  double sdbar = 0;
  if (q < np) {
    Cell3<T> c;
    bin3(p, x[q], y[q], z[q], c);
    const T dq = d[q];
    const double V = (double)(om[q] * (dq * dq * dq) * p.vcoef);
    double Vbar = Vb[q];
    double xg[3] = {0, 0, 0};
    const double inv[3] = {(double)p.invh[0], (double)p.invh[1], (double)p.invh[2]};
    double w[3][2];
    for (int a = 0; a < 3; ++a) { w[a][0] = 1.0 - (double)c.xi[a]; w[a][1] = (double)c.xi[a]; }
    for (int cc = 0; cc < 2; ++cc)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
          const long long n = node_id(p, c.i + a, c.j + b, c.k + cc);
          const double g = nadj[5 * p.nnode + n];
          Vbar += w[0][a] * w[1][b] * w[2][cc] * g;
          xg[0] += (a ? inv[0] : -inv[0]) * w[1][b] * w[2][cc] * g;
          xg[1] += (b ? inv[1] : -inv[1]) * w[0][a] * w[2][cc] * g;
          xg[2] += (cc ? inv[2] : -inv[2]) * w[0][a] * w[1][b] * g;
        }
    for (int a = 0; a < 3; ++a) xb[a * np + q] += V * xg[a];
    sdbar = Vbar * 3.0 * V / (double)p.sd;
  }
  sh[threadIdx.x] = sdbar;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(&theta[1], sh[0]);
}

// Adjoint state re-ordering across a checkpoint boundary: inv[tag_next[j]] = j, then
// a_this[i] = a_next[inv[tag_this[i]]] for the 6 adjoint components.
__global__ void k_tag_inverse(const int* __restrict__ tag, long long np, int* __restrict__ inv) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q < np) inv[tag[q]] = (int)q;
}

__global__ void k_adj_reorder(const double* __restrict__ src, double* __restrict__ dst,
                              const int* __restrict__ tag_this, const int* __restrict__ inv_next,
                              long long np) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= np) return;
  const int j = inv_next[tag_this[q]];
  for (int c = 0; c < 6; ++c) dst[c * np + q] = src[c * np + j];
}

__global__ void k_iota(int* a, long long n) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q < n) a[q] = (int)q;
}

}  // namespace mppic
