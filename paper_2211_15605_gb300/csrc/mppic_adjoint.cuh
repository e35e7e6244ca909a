// Reverse-mode (adjoint) kernels of the MP-PIC coupling step, for gradients of the
// time-averaged bed pressure drop and bed height with respect to the drag multiplier C,
// the diameter scale s_d and the inflow velocity u_in.
//
// The forward step they differentiate is the one of mppic_device.cuh (Woo et al.,
// arXiv 2211.15605, Sec. 2.1: Eqs. 3-5 with Wen-Yu drag, trilinear deposit and
// interpolation, semi-implicit drag, specular walls). A checkpoint segment is first
// recomputed forward (k_dep_simple, k_finalize, k_push_simple: the same arithmetic one
// parcel per thread without a sort), keeping each state's node fields and height sums.
// Each backward step then maps the adjoint of S_{n+1} to the adjoint of S_n:
//   k_adj_parcel : reverse of push, walls, drag, objectives and of the position dependence
//                  of the interpolation weights; writes each parcel's adjoints of the
//                  interpolated fields (the sources of interp^T) and bounds on their sums;
//                  its last block turns the bounds into one power-of-two fixed-point
//                  multiplier per node plane;
//   k_adj_scatter: interp^T, a deposit of the sources to the nodes in exact fixed point;
//   k_adj_node   : reverse of the node fields (Eq. 5 and u_g = U / eps_g), giving the
//                  adjoint of the deposited volume;
//   k_adj_deposit: reverse of the volume deposit (deposit^T, a gather);
//                  its last block adds the step's gradient partials in a fixed order.
// The per-parcel arithmetic and the parcel adjoint state are in the form's type T (the
// FP32 form keeps GB300's narrow FP64 pipe out of the per-parcel work); sums across blocks
// are FP64. No floating-point atomics: node sums are integer, block sums are fixed trees,
// so the gradient is bitwise reproducible.
#pragma once

#include "mppic_device.cuh"

namespace mppic {

// Per-parcel forward quantities of one step, recomputed in the adjoint kernels.
template <class T>
struct Fwd {
  Cell3<T> c;
  T w[3][2];            // trilinear factors
  Interp<T> I;
  T s[3], smag, eg, de, rem, p687, D1, D, V, f;
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
  r.p687 = T(0);
  if (r.laminar) {
    r.p687 = fpow(r.rem, T(0.687));
    r.D1 = p.kD1u * (T(1) + T(0.15) * r.p687) * e165 * frcp(r.eg) * (inv_de * inv_de);
  } else {
    r.D1 = p.kD2u * r.smag * e165 * inv_de;
  }
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

// ----------------------------------------------------- deterministic sums --

// Block sums of N values per thread, in a fixed tree: the lanes of each warp by shuffles in
// the values' type R (the form's type: no FP64 per thread in the FP32 form), then the warps in
// order in FP64; part[k * stride + blockIdx.x] receives quantity k. Every thread of the block
// must call it.
template <class R, int N>
__device__ __forceinline__ void block_partials(R (&v)[N], double* __restrict__ part,
                                               long long stride) {
  __shared__ R sh[N][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < N; ++k)
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < N; ++k) sh[k][wid] = v[k];
  __syncthreads();
  if (threadIdx.x < N) {
    double s = 0.0;
    for (int w = 0; w < nw; ++w) s += (double)sh[threadIdx.x][w];
    part[threadIdx.x * stride + blockIdx.x] = s;
  }
}

// Sums of N rows of per-block partials by one block of ADJ_RED threads in a fixed order:
// thread t takes entries t, t + ADJ_RED, ... of every row, the lanes of each warp are added
// by shuffles, then the warps in order. Row k is part[rows[k] * stride + 0 .. n[k]); thread 0
// receives the sums.
constexpr int ADJ_RED = 256;
template <int N>
__device__ __forceinline__ void block_totals(const double* __restrict__ part, long long stride,
                                             const int (&rows)[N], const long long (&n)[N],
                                             double (&out)[N]) {
  __shared__ double sh[N][ADJ_RED / 32];
  double s[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    s[k] = 0.0;
    for (long long b = threadIdx.x; b < n[k]; b += ADJ_RED) s[k] += __ldcg(part + rows[k] * stride + b);
  }
#pragma unroll
  for (int k = 0; k < N; ++k)
    for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_down_sync(0xffffffffu, s[k], o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < N; ++k) sh[k][wid] = s[k];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int k = 0; k < N; ++k) {
      double t = 0.0;
      for (int w = 0; w < ADJ_RED / 32; ++w) t += sh[k][w];
      out[k] = t;
    }
}

// Rows of the per-block partial sums (part[row * stride + block]).
enum AdjPart {
  AP_VZ = 0, AP_V = 1,                     // height sums of a state (k_dep_simple)
  AP_C = 2, AP_SD = 3,                     // dL/dC, dL/ds_d from k_adj_parcel
  AP_S0 = 4,                               // AP_S0 + q: bound on the plane-q node sums
  AP_SD2 = 9,                              // dL/ds_d from k_adj_deposit
  AP_UIN = 10,                             // dL/du_in from k_adj_node
  AP_ROWS = 11
};

// After the block has written its partials: true in the block that finishes last (the
// counter is then reset for the next launch). That block reads every other block's
// partials; their sum is taken in a fixed order, so the result does not depend on which
// block is last.
__device__ __forceinline__ bool last_block(unsigned* cnt) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(cnt, 1u);
    last = (t == gridDim.x - 1);
    if (last) *cnt = 0u;
  }
  __syncthreads();
  if (last) __threadfence();
  return last;
}

// Fixed-point conversion with integer instructions only: the same value as to_fixed (round
// to nearest even), without the float-to-int64 conversion, which runs on the FP64 pipe (a
// narrow one on this GPU). |s| < 2^23 rounds through a 32-bit conversion; from 2^23 on, a
// float is an integer and its bits give the int64 directly.
__device__ __forceinline__ void to_fixed_alu(float v, float m, u64 (&w)[1], int* errs) {
  float s = v * m;
  if (!(fabsf(s) < 1.152921504606847e18f)) { atomicOr(errs, ERR_RANGE); s = 0.0f; }
  const int b = __float_as_int(s);
  const int e = ((b >> 23) & 0xff) - 127;
  long long r;
  if (e < 23) {
    r = (long long)__float2int_rn(s);
  } else {
    r = (long long)((b & 0x7fffff) | 0x800000) << (e - 23);
    if (b < 0) r = -r;
  }
  w[0] = (u64)r;
}
__device__ __forceinline__ void to_fixed_alu(double v, double m, u64 (&w)[2], int* errs) {
  to_fixed(v, m, w, errs);
}

// ------------------------------------------------------------ chunk tiles --
// The deposits of the reverse sweep are made by blocks over contiguous chunks of ADJ_CHUNK
// parcels. A saved state keeps the layout order of a sort (drifted by at most a checkpoint
// segment and a sort period), in which a brick's parcels are contiguous and bricks follow
// each other along x. So a block adds its corners to a shared node tile covering the brick
// of the chunk's first parcel and the next brick along x, widened by one cell on every side
// (integer shared atomics), and adds the tile's non-zero entries to the global planes at the
// end; corners outside the tile go to the global planes directly. Integer sums: the result
// does not depend on the split between tile and global adds.
constexpr int ADJ_THREADS = 256, ADJ_CHUNK = 512;
constexpr int CX = 2 * BX + 3, CY = BY + 3, CZ = BZ + 3;   // tile nodes per axis
constexpr int CN = CX * CY * CZ;

template <class T>
__device__ __forceinline__ void chunk_origin(const KParams<T>& p, T x, T y, T z, int (&o)[3]) {
  Cell3<T> c;
  bin3(p, x, y, z, c);
  o[0] = (c.i / BX) * BX - 1;
  o[1] = (c.j / BY) * BY - 1;
  o[2] = (c.k / BZ) * BZ - 1;
}

// Adds f (plane `pl`) at node (i, j, k): into the tile if it covers the node, else globally.
template <class T, int W>
__device__ __forceinline__ void tile_add(const KParams<T>& p, u64* tile, const int (&o)[3], int pl,
                                         int i, int j, int k, const u64 (&f)[W]) {
  const int li = i - o[0], lj = j - o[1], lk = k - o[2];
  if ((unsigned)li < (unsigned)CX && (unsigned)lj < (unsigned)CY && (unsigned)lk < (unsigned)CZ)
    acc_add(tile + (pl * W) * CN + li + CX * (lj + CY * lk), CN, f);
  else
    acc_add(p.acc + (long long)(pl * W) * p.nstride + p.nbase + node_id(p, i, j, k), p.nstride, f);
}

// The tile's non-zero entries of planes [0, NPL) into the global planes.
template <class T, int W, int NPL>
__device__ __forceinline__ void tile_flush(const KParams<T>& p, const u64* tile, const int (&o)[3]) {
  for (int e = threadIdx.x; e < CN; e += blockDim.x) {
    const int li = e % CX, lj = (e / CX) % CY, lk = e / (CX * CY);
#pragma unroll
    for (int pl = 0; pl < NPL; ++pl) {
      u64 f[W];
#pragma unroll
      for (int w = 0; w < W; ++w) f[w] = tile[(pl * W + w) * CN + e];
      bool nz = false;
#pragma unroll
      for (int w = 0; w < W; ++w) nz |= f[w] != 0ull;
      if (nz)
        acc_add(p.acc + (long long)(pl * W) * p.nstride + p.nbase +
                    node_id(p, o[0] + li, o[1] + lj, o[2] + lk),
                p.nstride, f);
    }
  }
}

// Solids-volume deposit of a saved state in exact fixed point (chunk tiles), and its height
// sums: hs[0] = sum V z, hs[1] = sum V, hs[2] = 1 / sum V (fixed-order block sums, taken by
// the last block).
template <class T>
__global__ void __launch_bounds__(ADJ_THREADS)
k_dep_simple(KParams<T> p, const T* __restrict__ x, const T* __restrict__ y,
             const T* __restrict__ z, const T* __restrict__ d, const T* __restrict__ om,
             long long np, double* __restrict__ part, long long pstride, unsigned* cnt,
             double* __restrict__ hs) {
  constexpr int W = Words<T>::n;
  __shared__ u64 tile[W * CN];
  __shared__ int org[3];
  const long long c0 = blockIdx.x * (long long)ADJ_CHUNK;
  const long long c1 = c0 + ADJ_CHUNK < np ? c0 + ADJ_CHUNK : np;
  if (threadIdx.x == 0) {
    int o[3];
    chunk_origin(p, x[c0], y[c0], z[c0], o);
    org[0] = o[0]; org[1] = o[1]; org[2] = o[2];
  }
  for (int e = threadIdx.x; e < W * CN; e += blockDim.x) tile[e] = 0ull;
  __syncthreads();
  const int o[3] = {org[0], org[1], org[2]};
  T hv[2] = {T(0), T(0)};
  for (long long q = c0 + threadIdx.x; q < c1; q += blockDim.x) {
    Cell3<T> c;
    const T zq = z[q];
    bin3(p, x[q], y[q], zq, c);
    const T dq = d[q];
    const T V = om[q] * (dq * dq * dq) * p.vcoef;
    hv[0] += V * zq;
    hv[1] += V;
    T w[3][2];
    for (int a = 0; a < 3; ++a) { w[a][0] = T(1) - c.xi[a]; w[a][1] = c.xi[a]; }
    for (int cc = 0; cc < 2; ++cc)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
          u64 fx[W];
          to_fixed_alu(V * ((w[0][a] * w[1][b]) * w[2][cc]), p.mV, fx, p.errs);
          tile_add<T, W>(p, tile, o, 0, c.i + a, c.j + b, c.k + cc, fx);
        }
  }
  __syncthreads();
  tile_flush<T, W, 1>(p, tile, o);
  block_partials<T, 2>(hv, part + AP_VZ * pstride, pstride);
  if (last_block(cnt)) {
    double t[2];
    block_totals<2>(part, pstride, {AP_VZ, AP_V}, {(long long)gridDim.x, (long long)gridDim.x}, t);
    if (threadIdx.x == 0) { hs[0] = t[0]; hs[1] = t[1]; hs[2] = t[1] > 0.0 ? 1.0 / t[1] : 0.0; }
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

struct AdjWeights {
  double a_dp;   // dL/d(dP_n) / area
  double a_h;    // dL/d(H_n)
};

// Fixed-point multipliers of the five node-adjoint planes (0 eps_s, 1-3 u_g, 4 tau) of one
// backward step.
template <class T>
struct AdjScale {
  T m[5];
  double inv_m[5];
};

// The multiplier of plane q, m_q = 2^(B - E_q) with S_q < 2^E_q the bound on the plane's
// sums of |contributions|, so that every node sum of the plane is below 2^B in magnitude
// (B = 59 for the one-word FP32 form, 123 for the two-word FP64 form) and the integer sums
// cannot overflow. m_q is clamped to T's normal range; to_fixed flags what still overflows.
template <class T>
__device__ __forceinline__ void plane_scale(double S, int q, AdjScale<T>* sc, int* errs) {
  constexpr int B = Words<T>::n == 1 ? 59 : 123;
  constexpr int ELO = Words<T>::n == 1 ? -126 : -1000, EHI = Words<T>::n == 1 ? 127 : 1000;
  int E = 0;
  if (S > 0.0 && S <= 1.7976931348623157e308) frexp(S, &E);
  else if (!(S == 0.0)) atomicOr(errs, ERR_RANGE);
  int e = B - E;
  e = e < ELO ? ELO : (e > EHI ? EHI : e);
  sc->m[q] = (T)ldexp(1.0, e);
  sc->inv_m[q] = ldexp(1.0, -e);
}

// Reverse of one parcel's step. xb, ub: the parcel adjoint state (3 x np each), mapped in
// place from S_{n+1} to S_n (the deposit^T part of x is added by k_adj_deposit); Vb: the
// adjoint of the parcel volume V (without the deposit^T part); src: the adjoints of the
// interpolated fields [7][np] (eps_s, u_g x3, grad tau x3); hs: the state's height sums.
// The height objective H = 2 sum V z / sum V does not change when every V is scaled alike
// (V = w pi/6 (s_d d)^3 scales so with s_d), so its V-adjoint terms sum to exactly zero in
// dL/ds_d and are left out; its position adjoint 2 V / sum V is kept. Block partials: dL/dC, dL/ds_d, and for every node plane q a bound on the sum
// of |contributions| of the block's parcels (sum |src_q|; for tau sum_a 2 |gtb_a| / h_a,
// since the weight gradients of one axis sum to 2 / h_a in magnitude over the 8 corners);
// the last block turns the bounds into the planes' fixed-point multipliers (sc).
template <class T>
__global__ void k_adj_parcel(KParams<T> p, const T* __restrict__ x, const T* __restrict__ y,
                             const T* __restrict__ z, const T* __restrict__ u,
                             const T* __restrict__ v, const T* __restrict__ w,
                             const T* __restrict__ d, const T* __restrict__ om, long long np,
                             T* __restrict__ xb, T* __restrict__ ub, T* __restrict__ Vb,
                             T* __restrict__ src, const double* __restrict__ hs, AdjWeights aw,
                             double* __restrict__ part, long long pstride, unsigned* cnt,
                             AdjScale<T>* __restrict__ sc) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  T red[7] = {T(0), T(0), T(0), T(0), T(0), T(0), T(0)};   // dL/dC, dL/ds_d, plane bounds 0..4
  if (q < np) {
    Fields<T> F;
    for (int f = 0; f < 5; ++f) F.f[f] = p.fld[f];
    for (int a = 0; a < 3; ++a) F.g[a] = p.gpf[a];
    Fwd<T> r;
    const T X[3] = {x[q], y[q], z[q]};
    const T Uv[3] = {u[q], v[q], w[q]};
    const T dq = d[q];
    forward_parcel(p, F, X[0], X[1], X[2], Uv[0], Uv[1], Uv[2], dq, om[q], r);
    const T dt = p.dt;
    T xbar[3], ubar[3], accb[3];
    T Db = T(0);
    for (int a = 0; a < 3; ++a) {
      // walls: x = -x1 or 2L - x1, u = -e u1
      const T x2b = xb[a * np + q], u2b = ub[a * np + q];
      const T x1b = r.refl[a] ? -x2b : x2b;
      T u1b = (r.refl[a] ? -p.e_wall : T(1)) * u2b;
      // x1 = x + dt u1
      xbar[a] = x1b;
      u1b += dt * x1b;
      // u1 = (u + dt acc) / (1 + dt D)
      ubar[a] = u1b * r.inv_den;
      accb[a] = ubar[a] * dt;
      Db -= accb[a] * r.u1[a];
    }
    // acc = D u_g + g - grad p / rho_p - grad tau / (eps_s rho_p)
    T ugb[3], gtb[3], gpb[3], esb = T(0);
    for (int a = 0; a < 3; ++a) {
      Db += accb[a] * r.I.ug[a];
      ugb[a] = accb[a] * r.D;
      gpb[a] = -accb[a] * p.inv_rho_p;
      gtb[a] = -accb[a] * r.inv_esr;
      esb += accb[a] * r.I.gt[a] * r.inv_esr * r.inv_esr * p.rho_p;
    }
    // objectives: dP_n = sum f s_z / area, H_n = 2 sum V z / sum V
    const T a_dp = (T)aw.a_dp, a_h = (T)aw.a_h;
    const T fb = a_dp * r.s[2];
    T sb[3] = {T(0), T(0), a_dp * r.f};
    xbar[2] += a_h * T(2) * r.V * (T)hs[2];
    // f = rho_p V D
    const T Vbar = fb * p.rho_p * r.D;
    Db += fb * p.rho_p * r.V;
    // D = C D1(rem, eps_g, d_e); rem = eps_g d_e |s| rho_g / mu
    red[0] = Db * r.D1;
    const T D1b = Db * p.C;
    T remb = T(0), egb, deb, smagb;
    const T D1 = r.D1, eg = r.eg, de = r.de, rem = r.rem;
    const T inv_eg = frcp(eg), inv_de = frcp(de);
    if (r.laminar) {
      const T P = T(1) + T(0.15) * r.p687;
      const T dPdrem = rem > T(0) ? T(0.15 * 0.687) * r.p687 * frcp(rem) : T(0);
      remb = D1b * D1 * frcp(P) * dPdrem;
      egb = (D1b * (T(-2.65) * D1) + remb * rem) * inv_eg;
      deb = (D1b * (T(-2) * D1) + remb * rem) * inv_de;
      smagb = remb * eg * de * p.kRe;
    } else {
      egb = D1b * (T(-1.65) * D1) * inv_eg;
      deb = -(D1b * D1) * inv_de;
      smagb = r.smag > T(0) ? D1b * D1 * frcp(r.smag) : T(0);
    }
    red[1] = deb * dq;
    if (r.eg_free) esb -= egb;
    if (r.smag > T(0)) {
      const T k = smagb * frcp(r.smag);
      for (int a = 0; a < 3; ++a) sb[a] += k * r.s[a];
    }
    // s = u_g - u
    for (int a = 0; a < 3; ++a) { ugb[a] += sb[a]; ubar[a] -= sb[a]; }
    // V = w pi/6 (s_d d)^3 (the deposit^T part of Vbar is added by k_adj_deposit)
    Vb[q] = Vbar;
    // the sources of interp^T, and bounds on the node sums they make
    src[0 * np + q] = esb;
    for (int a = 0; a < 3; ++a) { src[(1 + a) * np + q] = ugb[a]; src[(4 + a) * np + q] = gtb[a]; }
    red[2] = fabs(esb);
    for (int a = 0; a < 3; ++a) red[3 + a] = fabs(ugb[a]);
    red[6] = T(2) * (fabs(gtb[0]) * p.invh[0] + fabs(gtb[1]) * p.invh[1] + fabs(gtb[2]) * p.invh[2]);
    // the position dependence of the interpolation weights
    const T inv[3] = {p.invh[0], p.invh[1], p.invh[2]};
    for (int cc = 0; cc < 2; ++cc)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
          const long long n = node_id(p, r.c.i + a, r.c.j + b, r.c.k + cc);
          const T wa = r.w[0][a], wb = r.w[1][b], wc = r.w[2][cc];
          const T sa = a ? inv[0] : -inv[0], sbb = b ? inv[1] : -inv[1], sc = cc ? inv[2] : -inv[2];
          const T dW[3] = {sa * wb * wc, sbb * wa * wc, sc * wa * wb};
          const T es_n = p.fld[0][n], tau_n = p.fld[4][n];
          T lin = es_n * esb;
          for (int k2 = 0; k2 < 3; ++k2) lin += p.fld[1 + k2][n] * ugb[k2];
          if (p.has_gp)
            for (int k2 = 0; k2 < 3; ++k2) lin += p.gpf[k2][n] * gpb[k2];
          // second derivatives of the weight (mixed only): d2W/dx dy = sa sbb wc, etc.
          const T dxy = sa * sbb * wc, dxz = sa * sc * wb, dyz = sbb * sc * wa;
          xbar[0] += dW[0] * lin + tau_n * (dxy * gtb[1] + dxz * gtb[2]);
          xbar[1] += dW[1] * lin + tau_n * (dxy * gtb[0] + dyz * gtb[2]);
          xbar[2] += dW[2] * lin + tau_n * (dxz * gtb[0] + dyz * gtb[1]);
        }
    for (int a = 0; a < 3; ++a) { xb[a * np + q] = xbar[a]; ub[a * np + q] = ubar[a]; }
  }
  block_partials<T, 7>(red, part + AP_C * pstride, pstride);   // rows AP_C, AP_SD, AP_S0..AP_S0+4
  if (last_block(cnt)) {
    const long long g = gridDim.x;
    double S[5];
    block_totals<5>(part, pstride, {AP_S0, AP_S0 + 1, AP_S0 + 2, AP_S0 + 3, AP_S0 + 4}, {g, g, g, g, g}, S);
    if (threadIdx.x == 0)
      for (int k = 0; k < 5; ++k) plane_scale(S[k], k, sc, p.errs);
  }
}

// interp^T: each parcel's sources times its trilinear weights (planes 0-3) and weight
// gradients (plane 4), added to the node planes p.acc[q] in fixed point (chunk tiles;
// dynamic shared memory: 5 planes x W words x CN nodes).
template <class T>
__global__ void __launch_bounds__(ADJ_THREADS)
k_adj_scatter(KParams<T> p, const T* __restrict__ x, const T* __restrict__ y,
              const T* __restrict__ z, long long np, const T* __restrict__ src,
              const AdjScale<T>* __restrict__ scp) {
  constexpr int W = Words<T>::n;
  extern __shared__ u64 tile[];
  __shared__ int org[3];
  const long long c0 = blockIdx.x * (long long)ADJ_CHUNK;
  const long long c1 = c0 + ADJ_CHUNK < np ? c0 + ADJ_CHUNK : np;
  if (threadIdx.x == 0) {
    int o[3];
    chunk_origin(p, x[c0], y[c0], z[c0], o);
    org[0] = o[0]; org[1] = o[1]; org[2] = o[2];
  }
  for (int e = threadIdx.x; e < 5 * W * CN; e += blockDim.x) tile[e] = 0ull;
  __syncthreads();
  const int o[3] = {org[0], org[1], org[2]};
  const T m0 = scp->m[0], m1 = scp->m[1], m2 = scp->m[2], m3 = scp->m[3], m4 = scp->m[4];
  const T inv[3] = {p.invh[0], p.invh[1], p.invh[2]};
  for (long long q = c0 + threadIdx.x; q < c1; q += blockDim.x) {
    Cell3<T> c;
    bin3(p, x[q], y[q], z[q], c);
    T w[3][2];
    for (int a = 0; a < 3; ++a) { w[a][0] = T(1) - c.xi[a]; w[a][1] = c.xi[a]; }
    const T s0 = src[q], s1 = src[np + q], s2 = src[2 * np + q], s3 = src[3 * np + q];
    const T s4 = src[4 * np + q], s5 = src[5 * np + q], s6 = src[6 * np + q];
#pragma unroll
    for (int cc = 0; cc < 2; ++cc)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int a = 0; a < 2; ++a) {
          const T wa = w[0][a], wb = w[1][b], wc = w[2][cc];
          const T sa = a ? inv[0] : -inv[0], sbb = b ? inv[1] : -inv[1], sc = cc ? inv[2] : -inv[2];
          const T Wq = wa * wb * wc;
          auto put = [&](int k, T val, T mk) {
            u64 f[W];
            to_fixed_alu(val, mk, f, p.errs);
            tile_add<T, W>(p, tile, o, k, c.i + a, c.j + b, c.k + cc, f);
          };
          put(0, Wq * s0, m0);
          put(1, Wq * s1, m1);
          put(2, Wq * s2, m2);
          put(3, Wq * s3, m3);
          put(4, (sa * wb * wc) * s4 + (sbb * wa * wc) * s5 + (sc * wa * wb) * s6, m4);
        }
  }
  __syncthreads();
  tile_flush<T, W, 5>(p, tile, o);
}

// Reverse of the node fields: from the adjoints of eps_s, u_g and tau at a node (the fixed-
// point planes of k_adj_scatter) to the adjoint of its deposited volume, Vsb[n], and the
// u_in part of the gradient (block partials).
template <class T>
__global__ void k_adj_node(KParams<T> p, const AdjScale<T>* __restrict__ scp, double inv_vcell,
                           T* __restrict__ Vsb, double* __restrict__ part, long long pstride) {
  constexpr int W = Words<T>::n;
  const int nx1 = p.nx + 1, ny1 = p.ny + 1;
  long long nn = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  T red[1] = {T(0)};
  if (nn < p.nnode) {
    const int n = (int)nn;
    const int i = n % nx1, j = (n / nx1) % ny1, k = n / (nx1 * ny1);
    double nad[5];
    for (int q = 0; q < 5; ++q) {
      u64 f[W];
      for (int e = 0; e < W; ++e) f[e] = p.acc[(long long)(q * W + e) * p.nstride + p.nbase + n];
      nad[q] = from_fixed(f, scp->inv_m[q]);
    }
    // 1 / (node volume): boundary nodes own half (a quarter, an eighth) of a cell
    double inv_vn = inv_vcell;
    if (i == 0 || i == p.nx) inv_vn *= 2.0;
    if (j == 0 || j == p.ny) inv_vn *= 2.0;
    if (k == 0 || k == p.nz) inv_vn *= 2.0;
    const T es = p.fld[0][n];
    double esb = nad[0];
    // tau = Ps es^beta / max(eps_cp - es, alpha (1 - es))
    const T d1 = p.eps_cp - es, d2 = p.alpha * (T(1) - es);
    const bool first = d1 >= d2;
    const T inv_den = frcp(first ? d1 : d2);
    const T dden = first ? T(-1) : -p.alpha;
    const T tau = p.Ps * fpow(es, p.beta) * inv_den;
    const T dtau = (es > T(0) ? p.Ps * p.beta * fpow(es, p.beta - T(1)) * inv_den : T(0)) -
                   tau * inv_den * dden;
    esb += nad[4] * (double)dtau;
    // u_g = U / max(1 - es, eg_min)
    const T egr = T(1) - es;
    const bool free = egr >= p.eg_min;
    const T inv_egc = frcp(free ? egr : p.eg_min);
    if (free)
      for (int a = 0; a < 3; ++a) esb += nad[1 + a] * (double)(p.fld[1 + a][n] * inv_egc);
    red[0] = (T)(nad[3] * (double)inv_egc);
    Vsb[n] = (T)(esb * inv_vn);
  }
  block_partials<T, 1>(red, part + AP_UIN * pstride, pstride);
}

// Reverse of the volume deposit (a gather): Vbar_p += sum W Vsb, xbar += V sum dW Vsb;
// then the s_d part of the gradient through V = w pi/6 (s_d d)^3. The last block adds the
// step's gradient partials to theta[0..2] (dL/dC, dL/ds_d, dL/du_in) in a fixed order.
template <class T>
__global__ void k_adj_deposit(KParams<T> p, const T* __restrict__ x, const T* __restrict__ y,
                              const T* __restrict__ z, const T* __restrict__ d,
                              const T* __restrict__ om, long long np, T* __restrict__ xb,
                              const T* __restrict__ Vb, const T* __restrict__ Vsb,
                              double* __restrict__ part, long long pstride, long long nblk_node,
                              unsigned* cnt, double* __restrict__ theta) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  T red[1] = {T(0)};
  if (q < np) {
    Cell3<T> c;
    bin3(p, x[q], y[q], z[q], c);
    const T dq = d[q];
    const T V = om[q] * (dq * dq * dq) * p.vcoef;
    T Vg = T(0);
    T xg[3] = {T(0), T(0), T(0)};
    const T inv[3] = {p.invh[0], p.invh[1], p.invh[2]};
    T w[3][2];
    for (int a = 0; a < 3; ++a) { w[a][0] = T(1) - c.xi[a]; w[a][1] = c.xi[a]; }
    for (int cc = 0; cc < 2; ++cc)
      for (int b = 0; b < 2; ++b)
        for (int a = 0; a < 2; ++a) {
          const T g = Vsb[node_id(p, c.i + a, c.j + b, c.k + cc)];
          Vg += w[0][a] * w[1][b] * w[2][cc] * g;
          xg[0] += (a ? inv[0] : -inv[0]) * w[1][b] * w[2][cc] * g;
          xg[1] += (b ? inv[1] : -inv[1]) * w[0][a] * w[2][cc] * g;
          xg[2] += (cc ? inv[2] : -inv[2]) * w[0][a] * w[1][b] * g;
        }
    for (int a = 0; a < 3; ++a) xb[a * np + q] += V * xg[a];
    red[0] = (Vb[q] + Vg) * (T(3) * V / p.sd);
  }
  block_partials<T, 1>(red, part + AP_SD2 * pstride, pstride);
  if (last_block(cnt)) {
    const long long g = gridDim.x;
    double t[4];
    block_totals<4>(part, pstride, {AP_C, AP_SD, AP_SD2, AP_UIN}, {g, g, g, nblk_node}, t);
    if (threadIdx.x == 0) {
      theta[0] += t[0];
      theta[1] += t[1] + t[2];
      theta[2] += t[3];
    }
  }
}

// With no parcels: theta[2] += the step's dL/du_in (one block).
__global__ void k_adj_theta_nodes(const double* __restrict__ part, long long pstride,
                                  long long nblk_node, double* __restrict__ theta) {
  double t[1];
  block_totals<1>(part, pstride, {AP_UIN}, {nblk_node}, t);
  if (threadIdx.x == 0) theta[2] += t[0];
}

// Adjoint state re-ordering across a checkpoint boundary: inv[tag_next[j]] = j, then
// a_this[i] = a_next[inv[tag_this[i]]] for the 6 adjoint components.
__global__ void k_tag_inverse(const int* __restrict__ tag, long long np, int* __restrict__ inv) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q < np) inv[tag[q]] = (int)q;
}

template <class T>
__global__ void k_adj_reorder(const T* __restrict__ src, T* __restrict__ dst,
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
