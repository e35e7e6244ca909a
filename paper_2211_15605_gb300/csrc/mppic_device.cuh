// Device code of libmppic: the MP-PIC parcel-grid coupling step for sm_103a.
//
// Physics (Woo et al., arXiv 2211.15605, Sec. 2.1): parcel volume V = w V_particle,
// Eq. 3 (dx/dt = u), Eq. 4 (parcel momentum with pressure gradient, drag, gravity and
// the solids stress gradient), Eq. 5 (Snider stress), and the drag force F of Eq. 2
// deposited to the mesh. Drag is Wen-Yu, interpolation trilinear on the node grid,
// walls specular at the parcel centre, drag implicit and the rest explicit.
//
// Layout and determinism:
//  * Cells are grouped in bricks of 8x8x4; parcels are sorted by a brick-major key
//    (brick id * 256 + local cell id). One CTA of 256 threads owns one brick, one
//    thread one cell, one warp a group of 32 cells. Within a group the sorted parcels
//    are stored by level (the r-th parcel of every cell that has one, then level r+1),
//    so a warp reads each level as one contiguous run.
//  * A thread walks its own cell's parcels and sums their contributions at the cell's 8
//    corners in registers (solids volume, drag sums); the sums enter a shared node tile
//    once per brick in 8 corner phases, in a fixed order. Parcels off their sorted cell
//    (drift since the last sort, or moved this step) add exact fixed-point contributions.
//  * Global deposits are exact integer fixed point: int64 for the FP32 form, int128 (two
//    64-bit words with carry) for the FP64 form. Integer addition is associative, so the
//    global sums do not depend on thread scheduling or on the order bricks finish.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mppic {

constexpr int BX = 8, BY = 8, BZ = 4;            // brick of cells
constexpr int BCELLS = BX * BY * BZ;             // 256 = threads per brick CTA
constexpr int TX = BX + 1, TY = BY + 1, TZ = BZ + 1;
constexpr int TNODES = TX * TY * TZ;             // 405 nodes per brick tile
constexpr int NQ = 5;                            // Vs, A, Bx, By, Bz
constexpr int ERR_DOMAIN = 1, ERR_RANGE = 2, ERR_TIMEOUT = 4;
// drag closures (the drag_model field of the configuration)
constexpr int DRAG_WEN_YU = 0, DRAG_SYAMLAL_OBRIEN = 1, DRAG_GIDASPOW = 2, DRAG_GIDASPOW_BLEND = 3;
// cell kernel modes: the solids volume only; a full step; the drag sums only (a gas
// iteration of implicit coupling)
constexpr int MODE_VOLUME = 0, MODE_STEP = 1, MODE_DRAG = 2;

typedef unsigned long long u64;

// ------------------------------------------------------------ parameters --

template <class T>
struct KParams {
  int nx, ny, nz;
  int nbx, nby, nbz;
  long long nnode;
  long long nbricks;
  // position of this bed in concatenated batch arrays (a single bed: 0, 0, nnode)
  long long nbase;           // first node of the bed in the accumulator planes
  long long bbase;           // first brick of the bed in the global brick (key) numbering
  long long nstride;         // accumulator plane stride (nodes of all beds)
  double inv_d[3];           // fl64(1/h): binning multiplier
  float inv_f[3], inv_lo[3]; // FP32 split: inv_d ~= inv_f + inv_lo
  T invh[3];                 // 1/h in T (interpolant gradient)
  T L[3];
  double vcell;
  double inv_vcell;          // 1 / vcell
  float es_scale;            // FP32 form: cell volume fraction per fixed-point unit, inv_mV / vcell
  T rho_g, mu_g, g[3], gp[3], rho_p, Ps, beta, eps_cp, alpha, eg_min, e_wall, C, sd, dt;
  T vcoef;                   // pi/6 * s_d^3: V = w d^3 vcoef
  T inv_rho_p;               // 1 / rho_p
  T kRe;                     // rho_g / mu_g (Re_m = eps_g d |s| kRe)
  T kD1, kD2;                // C 18 mu / rho_p and C 0.33 rho_g / rho_p (drag prefactors)
  T kD1u, kD2u;              // the same without C
  T kE1, kE2;                // Ergun: C 150 mu / rho_p and C 1.75 rho_g / rho_p
  T kS1, kS2;                // Syamlal-O'Brien: C 3/4 rho_g / rho_p and mu / rho_g
  int drag_model;            // DRAG_WEN_YU, DRAG_SYAMLAL_OBRIEN, DRAG_GIDASPOW, DRAG_GIDASPOW_BLEND
  T mV, mA;                  // fixed-point multipliers (value * m = integer units), powers of
                             // two, so that a value's product with them is exact
  double inv_mV, inv_mA;
  T u_in;
  // node fields: 0 eps_s, 1-3 u_g, 4 tau; 5-7 grad p (caller arrays, used if has_gp)
  T* fld[5];
  const T* gpf[3];
  int has_gp;
  const T* U[3];
  u64* acc;                  // [NQ][words][nnode]
  int* errs;
  int* zr;                   // node-layer ranges: [0,1] touched by the last deposit, [2,3] last finalized
  const int* cstart;         // [nkeys+1]: first sorted parcel of each brick-major key
  const uint8_t* cellmap;    // [nbricks*256]: local cell of thread t of each brick (own
                             // order, or ranked by parcel count; chosen at the last sort)
  u64* bacc;                 // [nbricks][NQ][words][TNODES]: each brick's node tile of the
                             // last deposit that covered it, in fixed point
  int* bstamp;               // [nbricks]: deposit epoch that wrote the brick's tile
  int* epoch;                // the current deposit epoch (advanced after each node pass)
};

template <class T> struct Words;
template <> struct Words<float> { static constexpr int n = 1; };
template <> struct Words<double> { static constexpr int n = 2; };

// ---------------------------------------------------------------- binning --

// FP64 form: the formula itself, without contraction.
__device__ __forceinline__ void bin_axis(double x, double inv_d, float, float, int n, int& i,
                                         double& xi) {
  double t = __dmul_rn(x, inv_d);
  double f = floor(t);
  if (!(f >= 0.0)) f = 0.0;
  if (f > (double)(n - 1)) f = (double)(n - 1);
  i = (int)f;
  xi = __dsub_rn(t, f);
  xi = fmin(fmax(xi, 0.0), 1.0);
}

// FP32 form: the same integer result as the FP64 formula. r = fma(x, inv_lo, fma(x, inv_f, -i))
// (inv_f + inv_lo = 1/h to about 2^-48 relative) is the in-cell coordinate x/h - i to within
// 1.3e-7 absolute, whatever the size of i: the inner fused multiply-add rounds once a value
// below 2 in magnitude, the outer adds the low part of the product. So where 2.5e-7 <= r <=
// 1 - 2.5e-7 the FP64 formula's floor is i as well; within 2.5e-7 of a face the FP64 formula
// decides.
__device__ __forceinline__ void bin_axis(float x, double inv_d, float inv_f, float inv_lo, int n,
                                         int& i, float& xi) {
  float fl = floorf(__fmul_rn(x, inv_f));
  float r = __fmaf_rn(x, inv_lo, __fmaf_rn(x, inv_f, -fl));
  if (!(r >= 2.5e-7f && r <= 1.0f - 2.5e-7f)) {
    double f64 = floor(__dmul_rn((double)x, inv_d));
    if (!(f64 >= 0.0)) f64 = 0.0;
    if (f64 > (double)(n - 1)) f64 = (double)(n - 1);
    fl = (float)f64;
    r = __fmaf_rn(x, inv_lo, __fmaf_rn(x, inv_f, -fl));
  }
  if (!(fl >= 0.0f)) fl = 0.0f;
  if (fl > (float)(n - 1)) fl = (float)(n - 1);
  i = (int)fl;
  xi = fminf(fmaxf(r, 0.0f), 1.0f);
}

template <class T>
struct Cell3 {
  int i, j, k;
  T xi[3];
};

template <class T>
__device__ __forceinline__ void bin3(const KParams<T>& p, T x, T y, T z, Cell3<T>& c) {
  bin_axis(x, p.inv_d[0], p.inv_f[0], p.inv_lo[0], p.nx, c.i, c.xi[0]);
  bin_axis(y, p.inv_d[1], p.inv_f[1], p.inv_lo[1], p.ny, c.j, c.xi[1]);
  bin_axis(z, p.inv_d[2], p.inv_f[2], p.inv_lo[2], p.nz, c.k, c.xi[2]);
}

// In-cell coordinate of x on one axis if the binning formula puts x in cell ic there, with
// the same value bin_axis would give; false if it does not, or (FP32 form) if x is within
// the face margin where the FP64 formula must decide (the caller then uses bin_axis).
__device__ __forceinline__ bool xi_in_cell(double x, double inv_d, float, float, int ic, double& xi) {
  const double t = __dmul_rn(x, inv_d);
  const double d = __dsub_rn(t, (double)ic);
  if (!(d >= 0.0 && d < 1.0)) return false;
  xi = d;
  return true;
}
__device__ __forceinline__ bool xi_in_cell(float x, double, float inv_f, float inv_lo, int ic, float& xi) {
  const float r = __fmaf_rn(x, inv_lo, __fmaf_rn(x, inv_f, -(float)ic));
  if (!(r >= 2.5e-7f && r <= 1.0f - 2.5e-7f)) return false;
  xi = r;
  return true;
}

// Binning of (x, y, z) when cell (i, j, k) is the likely answer: the in-cell test on each
// axis, and the full formula only on the axes where it fails (where the test passes, the
// formula gives the same index and in-cell coordinate). Returns whether the cell is (i, j, k).
// FP64 form: the formula on all three axes once a test fails. Re-binning only the failing
// axes, the compiler computed the formula's FP64 products for every parcel and selected
// (12 more FP64 multiplies per parcel on the narrow FP64 pipe: the FP64 step 3% slower).
template <class T>
__device__ __forceinline__ bool bin3_expect(const KParams<T>& p, T x, T y, T z, int i, int j, int k,
                                            Cell3<T>& c) {
  if constexpr (sizeof(T) == 8) {
    if (xi_in_cell(x, p.inv_d[0], p.inv_f[0], p.inv_lo[0], i, c.xi[0]) &&
        xi_in_cell(y, p.inv_d[1], p.inv_f[1], p.inv_lo[1], j, c.xi[1]) &&
        xi_in_cell(z, p.inv_d[2], p.inv_f[2], p.inv_lo[2], k, c.xi[2])) {
      c.i = i; c.j = j; c.k = k;
      return true;
    }
    bin3(p, x, y, z, c);
    return c.i == i && c.j == j && c.k == k;
  }
  const bool ox = xi_in_cell(x, p.inv_d[0], p.inv_f[0], p.inv_lo[0], i, c.xi[0]);
  const bool oy = xi_in_cell(y, p.inv_d[1], p.inv_f[1], p.inv_lo[1], j, c.xi[1]);
  const bool oz = xi_in_cell(z, p.inv_d[2], p.inv_f[2], p.inv_lo[2], k, c.xi[2]);
  c.i = i; c.j = j; c.k = k;
  if (ox && oy && oz) return true;
  if (!ox) bin_axis(x, p.inv_d[0], p.inv_f[0], p.inv_lo[0], p.nx, c.i, c.xi[0]);
  if (!oy) bin_axis(y, p.inv_d[1], p.inv_f[1], p.inv_lo[1], p.ny, c.j, c.xi[1]);
  if (!oz) bin_axis(z, p.inv_d[2], p.inv_f[2], p.inv_lo[2], p.nz, c.k, c.xi[2]);
  return c.i == i && c.j == j && c.k == k;
}

template <class T>
__device__ __forceinline__ int cell_id(const KParams<T>& p, int i, int j, int k) {
  return i + p.nx * (j + p.ny * k);
}

template <class T>
__device__ __forceinline__ void decode_cell(const KParams<T>& p, int c, int& i, int& j, int& k) {
  i = c % p.nx;
  int r = c / p.nx;
  j = r % p.ny;
  k = r / p.ny;
}

// Cell (i,j,k) as bit fields of cb[0] and cb[1] bits for i and j (cb[0] < 0: the cell id,
// for a grid whose fields would not fit 31 bits). Unpacking is shifts, not divisions.
struct CellBits {
  int b0, b1;
};
template <class T>
__device__ __forceinline__ CellBits cell_bits(const KParams<T>& p) {
  auto bits = [](int n) { return n > 1 ? 32 - __clz(n - 1) : 0; };
  CellBits cb{bits(p.nx), bits(p.ny)};
  if (cb.b0 + cb.b1 + bits(p.nz) > 31) cb.b0 = -1;
  return cb;
}
template <class T>
__device__ __forceinline__ int pack_cell(const KParams<T>& p, CellBits cb, int i, int j, int k) {
  return cb.b0 >= 0 ? (i | (j << cb.b0) | (k << (cb.b0 + cb.b1))) : cell_id(p, i, j, k);
}
template <class T>
__device__ __forceinline__ void unpack_cell(const KParams<T>& p, CellBits cb, int c, int& i, int& j,
                                            int& k) {
  if (cb.b0 >= 0) {
    i = c & ((1 << cb.b0) - 1);
    j = (c >> cb.b0) & ((1 << cb.b1) - 1);
    k = c >> (cb.b0 + cb.b1);
  } else {
    decode_cell(p, c, i, j, k);
  }
}

// Brick-major sort key of cell (i,j,k).
template <class T>
__device__ __forceinline__ uint32_t brick_key(const KParams<T>& p, int i, int j, int k) {
  int bi = i / BX, bj = j / BY, bk = k / BZ;
  uint32_t b = (uint32_t)(bi + p.nbx * (bj + p.nby * bk));
  uint32_t l = (uint32_t)((i - bi * BX) + BX * ((j - bj * BY) + BY * (k - bk * BZ)));
  return b * BCELLS + l;
}

template <class T>
__device__ __forceinline__ long long node_id(const KParams<T>& p, int i, int j, int k) {
  return (long long)i + (long long)(p.nx + 1) * ((long long)j + (long long)(p.ny + 1) * k);
}

// ----------------------------------------------------------- fixed point --

// FP32 form: one signed 64-bit word. v*m is rounded once in FP32, then exactly to an
// integer. |v*m| >= 2^60 marks the accumulator out of range.
__device__ __forceinline__ void to_fixed(float v, float m, u64 (&w)[1], int* errs) {
  float s = v * m;
  if (!(fabsf(s) < 1.152921504606847e18f)) { atomicOr(errs, ERR_RANGE); s = 0.0f; }
  w[0] = (u64)__float2ll_rn(s);
}

// FP64 form: a signed 128-bit integer (lo, hi) equal to round(v*m), built from the bits
// of the double so that no FP64 arithmetic beyond the one product is needed.
__device__ __forceinline__ void to_fixed(double v, double m, u64 (&w)[2], int* errs) {
  double s = v * m;
  u64 bits = (u64)__double_as_longlong(s);
  int e = (int)((bits >> 52) & 0x7ff);
  u64 mant = (bits & 0xfffffffffffffull) | (1ull << 52);
  u64 lo = 0, hi = 0;
  if (e == 0x7ff) {
    atomicOr(errs, ERR_RANGE);
  } else if (e != 0) {
    int sh = e - 1075;                 // value = mant * 2^sh
    if (sh >= 0) {
      if (sh > 73) {
        atomicOr(errs, ERR_RANGE);
      } else if (sh >= 64) {
        hi = mant << (sh - 64);
      } else if (sh == 0) {
        lo = mant;
      } else {
        lo = mant << sh;
        hi = mant >> (64 - sh);
      }
    } else if (sh > -64) {
      int r = -sh;                     // round half away from zero
      lo = (mant + (1ull << (r - 1))) >> r;
    }
  }
  if (bits >> 63) {                    // negate
    lo = ~lo + 1ull;
    hi = ~hi + (lo == 0ull ? 1ull : 0ull);
  }
  w[0] = lo;
  w[1] = hi;
}

__device__ __forceinline__ double from_fixed(const u64 (&w)[1], double inv_m) {
  return (double)(long long)w[0] * inv_m;
}
__device__ __forceinline__ double from_fixed(const u64 (&w)[2], double inv_m) {
  // hi * 2^64 + lo with hi signed
  double v = (double)(long long)w[1] * 18446744073709551616.0 + (double)w[0];
  return v * inv_m;
}

// Atomic add of a fixed-point value (global or shared address).
__device__ __forceinline__ void acc_add(u64* base, long long stride, const u64 (&w)[1]) {
  if (w[0]) atomicAdd(base, w[0]);
}
__device__ __forceinline__ void acc_add(u64* base, long long stride, const u64 (&w)[2]) {
  if (w[0] | w[1]) {
    u64 old = atomicAdd(base, w[0]);
    u64 carry = (old + w[0] < old) ? 1ull : 0ull;
    u64 hi = w[1] + carry;
    if (hi) atomicAdd(base + stride, hi);
  }
}

template <class T> __device__ __forceinline__ T tmax(T a, T b) { return a >= b ? a : b; }

// ------------------------------------------------------------ node fields --

// Interpolation at one parcel from 8 corner nodes. Node n of corner (a,b,c) is
// base + a*sx + b*sy + c*sz in the arrays f[0..4] (and g[0..2] if non-null).
template <class T>
struct Interp {
  T es, ug[3], gp[3], gt[3];
};

template <class T>
struct Fields {
  const T* f[5];   // eps_s, u_g x/y/z, tau
  const T* g[3];   // grad p (used when has_g)
};

template <class T>
__device__ __forceinline__ void interp8(const KParams<T>& p, const Fields<T> F, bool has_g,
                                        long long base, long long sx, long long sy, long long sz,
                                        const T (&xi)[3], Interp<T>& r) {
  T w[3][2];
  for (int a = 0; a < 3; ++a) { w[a][0] = T(1) - xi[a]; w[a][1] = xi[a]; }
  r.es = 0;
  for (int a = 0; a < 3; ++a) { r.ug[a] = 0; r.gt[a] = 0; r.gp[a] = 0; }
#pragma unroll
  for (int c = 0; c < 2; ++c)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int a = 0; a < 2; ++a) {
        long long n = base + a * sx + b * sy + c * sz;
        T W = (w[0][a] * w[1][b]) * w[2][c];
        r.es += W * F.f[0][n];
        r.ug[0] += W * F.f[1][n];
        r.ug[1] += W * F.f[2][n];
        r.ug[2] += W * F.f[3][n];
        T tau = F.f[4][n];
        r.gt[0] += ((a ? p.invh[0] : -p.invh[0]) * (w[1][b] * w[2][c])) * tau;
        r.gt[1] += ((b ? p.invh[1] : -p.invh[1]) * (w[0][a] * w[2][c])) * tau;
        r.gt[2] += ((c ? p.invh[2] : -p.invh[2]) * (w[0][a] * w[1][b])) * tau;
        if (has_g) {
          r.gp[0] += W * F.g[0][n];
          r.gp[1] += W * F.g[1][n];
          r.gp[2] += W * F.g[2][n];
        }
      }
  if (!has_g) { r.gp[0] = p.gp[0]; r.gp[1] = p.gp[1]; r.gp[2] = p.gp[2]; }
}

__device__ __forceinline__ float tpow(float a, float b) { return powf(a, b); }
__device__ __forceinline__ double tpow(double a, double b) { return pow(a, b); }
__device__ __forceinline__ float tsqrt(float a) { return sqrtf(a); }
__device__ __forceinline__ double tsqrt(double a) { return sqrt(a); }

// Wen-Yu drag as an acceleration coefficient D: F_P / (eps_P rho_P) = D (u_g - u_P).
// Re_m = eps_g rho_g d |s| / mu; Cd = 24/Re_m (1 + 0.15 Re_m^0.687) below 1000, else 0.44;
// D = C (3/4) Cd rho_g |s| eps_g^-1.65 / (d rho_p), evaluated through Cd |s|.
template <class T>
__device__ __forceinline__ T wen_yu(const KParams<T>& p, T d, T es, const T (&s)[3]) {
  T eg = tmax(T(1) - es, p.eg_min);
  T de = p.sd * d;
  T smag = tsqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
  T rem = eg * p.rho_g * de * smag / p.mu_g;
  T cds;
  if (rem < T(1000))
    cds = T(24) * p.mu_g / (p.rho_g * de * eg) * (T(1) + T(0.15) * tpow(rem, T(0.687)));
  else
    cds = T(0.44) * smag;
  return p.C * T(0.75) * cds * p.rho_g * tpow(eg, T(-1.65)) / (de * p.rho_p);
}

// ---------------------------------------------------------------- kernels --

// a1: cell id of every parcel (exact FP64 binning formula).
template <class T>
__global__ void k_bin(KParams<T> p, const T* __restrict__ x, const T* __restrict__ y,
                      const T* __restrict__ z, int* __restrict__ cell, long long np) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= np) return;
  Cell3<T> c;
  bin3(p, x[q], y[q], z[q], c);
  cell[q] = cell_id(p, c.i, c.j, c.k);
}

// Sort keys (brick-major). The first radix pass takes the parcel index as the value.
template <class T>
__global__ void k_keys(KParams<T> p, const T* __restrict__ x, const T* __restrict__ y,
                       const T* __restrict__ z, uint32_t* __restrict__ key, long long np) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= np) return;
  Cell3<T> c;
  bin3(p, x[q], y[q], z[q], c);
  key[q] = brick_key(p, c.i, c.j, c.k);
}

// Permute the parcel arrays by the sorted order.
template <class T>
struct PArrays {
  T* a[8];        // x y z u v w d omega
  int* pid;       // caller's identity array (optional)
  int* tag;       // the handle's identity array while checkpointing (optional)
  const uint32_t* perm;   // (step kernel reads only) the parcel of layout position q is at
                          // index perm[q] of a[] (a sort that moved no values); else q
};

constexpr unsigned FULL = 0xffffffffu;

__host__ __device__ constexpr size_t rup(size_t x, size_t a) { return (x + a - 1) / a * a; }

__device__ __forceinline__ float fpow(float a, float b) { return __powf(a, b); }
__device__ __forceinline__ double fpow(double a, double b) { return pow(a, b); }
__device__ __forceinline__ float frcp(float a) { return __fdividef(1.0f, a); }
__device__ __forceinline__ double frcp(double a) { return 1.0 / a; }
__device__ __forceinline__ float fsqrt(float a) { return a > 0.0f ? a * rsqrtf(a) : 0.0f; }
__device__ __forceinline__ double fsqrt(double a) { return sqrt(a); }

// Wen-Yu drag as an acceleration coefficient (same closure as wen_yu, in the form
// D = C 18 mu (1 + 0.15 Re_m^0.687) eps_g^-2.65 / (d^2 rho_p) below Re_m = 1000 and
// D = C 0.33 rho_g |s| eps_g^-1.65 / (d rho_p) above).
template <class T>
__device__ __forceinline__ T wen_yu_fast(const KParams<T>& p, T d, T es, const T (&s)[3]) {
  T eg = tmax(T(1) - es, p.eg_min);
  T de = p.sd * d;
  T inv_de = frcp(de);
  T smag = fsqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
  T rem = eg * de * smag * p.kRe;
  T e165 = fpow(eg, T(-1.65));
  if (rem < T(1000))
    return p.kD1 * (T(1) + T(0.15) * fpow(rem, T(0.687))) * e165 * frcp(eg) * (inv_de * inv_de);
  return p.kD2 * smag * e165 * inv_de;
}

// The brick's node-field tile, in T units (VW = values per 16-byte vector: 4 floats or 2
// doubles), node-major planes so the 8 lanes of a quarter-warp (8 consecutive nodes along
// x) read 128 contiguous bytes:
//   [0, 4 TNODES)        eps_s, u_g[3] as 4/VW planes of VW-vectors;
//   with grad p (a node field): [4 TNODES, 8 TNODES) grad p[3] (and a pad) the same way,
//   then tau at [8 TNODES, 9 TNODES); without: tau at [4 TNODES, 5 TNODES).
template <class T> struct TileVec;
template <> struct TileVec<float> { static constexpr int n = 4; };
template <> struct TileVec<double> { static constexpr int n = 2; };
__host__ __device__ constexpr int tile_vals(bool gp) { return gp ? 9 : 5; }  // T values per node
__host__ __device__ constexpr int tau_off(bool gp) { return gp ? 8 * TNODES : 4 * TNODES; }

// Offset (in T) of field f of tile node tn (ta = tau_off of the tile's layout).
template <class T>
__device__ __forceinline__ int tile_off(int f, int tn, int ta) {
  constexpr int VW = TileVec<T>::n;
  if (f < 4) return VW * ((f / VW) * TNODES + tn) + f % VW;
  if (f == 4) return ta + tn;
  const int g = f - 5;
  return 4 * TNODES + VW * ((g / VW) * TNODES + tn) + g % VW;
}

__device__ __forceinline__ void tile_node(const float* t, int n, bool gpf, int ta, float (&v)[8]) {
  const float4 a = *reinterpret_cast<const float4*>(t + 4 * n);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
  v[4] = t[ta + n];
  if (gpf) {
    const float4 g = *reinterpret_cast<const float4*>(t + 4 * (TNODES + n));
    v[5] = g.x; v[6] = g.y; v[7] = g.z;
  }
}
__device__ __forceinline__ void tile_node(const double* t, int n, bool gpf, int ta, double (&v)[8]) {
  const double2 a0 = *reinterpret_cast<const double2*>(t + 2 * n);
  const double2 a1 = *reinterpret_cast<const double2*>(t + 2 * (TNODES + n));
  v[0] = a0.x; v[1] = a0.y; v[2] = a1.x; v[3] = a1.y;
  v[4] = t[ta + n];
  if (gpf) {
    const double2 g0 = *reinterpret_cast<const double2*>(t + 2 * (2 * TNODES + n));
    const double2 g1 = *reinterpret_cast<const double2*>(t + 2 * (3 * TNODES + n));
    v[5] = g0.x; v[6] = g0.y; v[7] = g1.x;
  }
}

// ------------------------------------------------------------ cell kernel --

// Threads of a cell-kernel CTA: thread t owns two cells of its brick, local cell t of the
// lower half and the cell of the upper half the brick's pair map gives it (set at each sort,
// pair_layout in mppic_sort.cuh), and walks the parcels of the first, then of the second.
constexpr int CT = BCELLS / 2;

// Shared memory of the cell kernels (sections 128-byte aligned), for a node-field tile with
// or without the grad p planes (gp):
//   fld  node-field tile (tile_vals(gp) values per node); after the parcel loop it holds the
//        objective partials [3][CT];
//   fx   [NQ][W][TNODES] u64: exact fixed-point sums (parcels off their sorted cell; in the
//        FP32 form also the exact volume of the cells' own parcels);
//   tile [NQ][TNODES] T: the node sums of the cells' own parcels (after the parcel loop);
//        during the loop, each warp's two queues of QCAP parcel records for the off-cell
//        deposits;
//   cbuf [NQ*8][CT] T and [CT] long long: the 40 corner sums (and exact volume) a thread's
//        first cell leaves when the thread moves on to its second.
template <class T>
struct CellSmem {
  static constexpr int W = Words<T>::n;
  __host__ __device__ static constexpr size_t fx(bool gp) { return rup(sizeof(T) * tile_vals(gp) * TNODES, 128); }
  __host__ __device__ static constexpr size_t tile(bool gp) { return rup(fx(gp) + sizeof(u64) * NQ * W * TNODES, 128); }
  // the warps' off-cell queues, two of QCAP records of 8 values per warp, share the tile
  static constexpr int QCAP = 32;
  static constexpr size_t tile_len = NQ * TNODES > 2 * QCAP * 8 * (CT / 32) ? NQ * TNODES : 2 * QCAP * 8 * (CT / 32);
  __host__ __device__ static constexpr size_t cbuf(bool gp) { return rup(tile(gp) + sizeof(T) * tile_len, 128); }
  __host__ __device__ static constexpr size_t vbuf(bool gp) { return cbuf(gp) + sizeof(T) * NQ * 8 * CT; }
  __host__ __device__ static constexpr size_t bytes(bool gp) { return vbuf(gp) + sizeof(long long) * CT; }
};
static_assert(sizeof(float) * 3 * CT <= sizeof(float) * 5 * TNODES, "objective partials fit the tile");

// Asynchronous copy of one parcel value into this thread's prefetch slot.
__device__ __forceinline__ void cp_async(float* dst, const float* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async(double* dst, const double* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// A parcel record of the off-cell queue: cell (pack_cell), in-cell coordinates, up to 4
// values, 8 values of T (the cell id's bits in the FP32 form, its value in the FP64 form).
__device__ __forceinline__ float cell_as_t(int c, float) { return __int_as_float(c); }
__device__ __forceinline__ double cell_as_t(int c, double) { return (double)c; }
__device__ __forceinline__ int cell_of_t(float v) { return __float_as_int(v); }
__device__ __forceinline__ int cell_of_t(double v) { return (int)v; }
__device__ __forceinline__ void store_rec(float* r, const float (&v)[8]) {
  reinterpret_cast<float4*>(r)[0] = make_float4(v[0], v[1], v[2], v[3]);
  reinterpret_cast<float4*>(r)[1] = make_float4(v[4], v[5], v[6], v[7]);
}
__device__ __forceinline__ void store_rec(double* r, const double (&v)[8]) {
#pragma unroll
  for (int h = 0; h < 4; ++h) reinterpret_cast<double2*>(r)[h] = make_double2(v[2 * h], v[2 * h + 1]);
}
__device__ __forceinline__ void load_rec(const float* r, float (&v)[8]) {
  const float4 a = reinterpret_cast<const float4*>(r)[0], b = reinterpret_cast<const float4*>(r)[1];
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void load_rec(const double* r, double (&v)[8]) {
#pragma unroll
  for (int h = 0; h < 4; ++h) {
    const double2 d = reinterpret_cast<const double2*>(r)[h];
    v[2 * h] = d.x; v[2 * h + 1] = d.y;
  }
}

// Off-cell deposits. Parcels that are not in their sorted cell add their contributions in
// exact fixed point: NV values at the 8 corners of cell `cell` (pack_cell) with in-cell
// coordinates x0..x2, starting at quantity q0 (0 = Vs, 1 = A, then Bx, By, Bz), into the
// brick's shared tile if the cell is in the brick (i0, j0, k0 = its first cell), else into
// the global accumulators. These are a few percent of the parcels, so the warp shares the
// work: the lanes with such a parcel queue a record of it (queue_offcell) in the warp's
// queue, and when the next records would not fit (and after the loop) the whole warp drains it
// (drain_offcell) in rounds of four records, lanes 8g..8g+7 taking the 8 corners of record
// 4r+g, instead of each lane running its 8 corners while the rest of the warp idles.
// Integer additions commute, so neither when a record is drained nor the rounds change any
// sum. EXACT (the solids volume of the FP32 form): the corner with the largest weight adds
// the parcel's volume in fixed point minus the other seven corners' values, so that the 8
// corners add up to exactly the parcel's volume (v0 * mV is exact: mV is a power of two).

// Appends a record for every lane in `pend` (a ballot; all 32 lanes call it) to the warp's
// queue wq (16-byte aligned records of 8 values) holding n records; returns the new count.
template <class T>
__device__ __forceinline__ int queue_offcell(T* wq, int n, unsigned pend, int cell, T x0, T x1, T x2,
                                             T v0, T v1, T v2, T v3) {
  const int lane = threadIdx.x & 31;
  if ((pend >> lane) & 1u) {
    const T rec[8] = {cell_as_t(cell, T(0)), x0, x1, x2, v0, v1, v2, v3};
    store_rec(wq + 8 * (n + __popc(pend & ((1u << lane) - 1u))), rec);
  }
  return n + __popc(pend);
}

// Deposits the warp's npend queued records (all 32 lanes call it, npend uniform) and empties
// the queue. A call, not inlined: the cell kernel's parcel loop runs it rarely, and its code
// inlined at each use made the loop's instructions miss in the instruction cache (the step
// kernel took 6% longer).
template <class T, int NV, bool EXACT = false>
__device__ __noinline__ void drain_offcell(const KParams<T>& p, u64* fx, int* kr, int i0, int j0,
                                              int k0, CellBits cb, int q0, const T* wq, int npend) {
  constexpr int W = Words<T>::n;
  const int lane = threadIdx.x & 31, g = lane >> 3, corner = lane & 7;
  const int a = corner & 1, b = (corner >> 1) & 1, c = corner >> 2;
  __syncwarp();                                  // the records are written
  for (int k = g; k - g < npend; k += 4) {
    const bool has = k < npend;
    T rec[8];
    load_rec(wq + 8 * (has ? k : 0), rec);
    int si, sj, sk;
    unpack_cell(p, cb, cell_of_t(rec[0]), si, sj, sk);
    const T y0 = rec[1], y1 = rec[2], y2 = rec[3];
    const T Wq = ((a ? y0 : T(1) - y0) * (b ? y1 : T(1) - y1)) * (c ? y2 : T(1) - y2);
    u64 fe[W] = {};
    if (EXACT) {                                 // all 32 lanes: the group sum of the others
      const int kst = (y0 >= T(0.5) ? 1 : 0) + (y1 >= T(0.5) ? 2 : 0) + (y2 >= T(0.5) ? 4 : 0);
      to_fixed(has ? rec[4] * Wq : T(0), p.mV, fe, p.errs);
      long long others = corner == kst ? 0ll : (long long)fe[0];
#pragma unroll
      for (int o = 1; o < 8; o <<= 1) others += __shfl_xor_sync(FULL, others, o);
      if (corner == kst) {
        u64 tot[W];
        to_fixed(has ? rec[4] : T(0), p.mV, tot, p.errs);
        fe[0] = (u64)((long long)tot[0] - others);
      }
    }
    if (has) {
      const int ti = si - i0, tj = sj - j0, tk = sk - k0;
      const bool in = ti >= 0 && ti < BX && tj >= 0 && tj < BY && tk >= 0 && tk < BZ;
      if (corner == 0) {                         // node layers deposited into (shared)
        atomicMin(kr, sk);
        atomicMax(kr + 1, sk + 1);
      }
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        const int qq = q0 + v;
        u64 f[W];
        if (EXACT) {
          f[0] = fe[0];
        } else {
          to_fixed(rec[4 + v] * Wq, qq == 0 ? p.mV : p.mA, f, p.errs);
        }
        if (in)
          acc_add(fx + (qq * W) * TNODES + (ti + a) + TX * ((tj + b) + TY * (tk + c)), TNODES, f);
        else
          acc_add(p.acc + (long long)(qq * W) * p.nstride + p.nbase + node_id(p, si + a, sj + b, sk + c),
                  p.nstride, f);
      }
    }
  }
  __syncwarp();                                  // the queue is refilled after this
}

// Trilinear corner weights W[a + 2b + 4c] of in-cell coordinates xi. FP64: 8 values. FP32:
// 4 pairs (corners 2k and 2k+1, which differ in the x factor), formed and used with the
// paired FP32 operations (each lane one rounded product or fused multiply-add, so the values
// equal the scalar ones).
template <class T> struct W8;
template <> struct W8<double> {
  double w[8];
  __device__ __forceinline__ double get(int q) const { return w[q]; }
};
template <> struct W8<float> {
  float2 w[4];
  __device__ __forceinline__ float get(int q) const { return (q & 1) ? w[q >> 1].y : w[q >> 1].x; }
};

// The weights and the y-z products yz[b + 2c] they are built from (also the weights of d/dx
// of the interpolant), and xi (the other two gradient weights are formed where they are used).
template <class T>
struct Weights {
  W8<T> W;
  T yz[4], xi[3];
};

__device__ __forceinline__ void corner_weights(const double (&xi)[3], W8<double>& W, double (&yz)[4]) {
  const double w0[2] = {1.0 - xi[0], xi[0]}, w1[2] = {1.0 - xi[1], xi[1]}, w2[2] = {1.0 - xi[2], xi[2]};
#pragma unroll
  for (int q = 0; q < 4; ++q) yz[q] = w1[q & 1] * w2[q >> 1];
#pragma unroll
  for (int q = 0; q < 8; ++q) W.w[q] = w0[q & 1] * yz[q >> 1];
}
__device__ __forceinline__ void corner_weights(const float (&xi)[3], W8<float>& W, float (&yz)[4]) {
  const float2 wx = make_float2(1.0f - xi[0], xi[0]), wy = make_float2(1.0f - xi[1], xi[1]);
  const float z0 = 1.0f - xi[2], z1 = xi[2];
  const float2 yz01 = __fmul2_rn(wy, make_float2(z0, z0));   // yz[0], yz[1]
  const float2 yz23 = __fmul2_rn(wy, make_float2(z1, z1));   // yz[2], yz[3]
  yz[0] = yz01.x; yz[1] = yz01.y; yz[2] = yz23.x; yz[3] = yz23.y;
#pragma unroll
  for (int k = 0; k < 4; ++k) W.w[k] = __fmul2_rn(wx, make_float2(yz[k], yz[k]));
}

template <class T>
__device__ __forceinline__ void all_weights(const T (&xi)[3], Weights<T>& r) {
  corner_weights(xi, r.W, r.yz);
  r.xi[0] = xi[0]; r.xi[1] = xi[1]; r.xi[2] = xi[2];
}

// The 40 per-cell register sums of the cell kernel: the solids volume and the drag sums A,
// Bx, By, Bz at the cell's 8 corners.
template <class T> struct CellSums;
template <> struct CellSums<double> {
  double v[NQ][8];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
      for (int k = 0; k < 8; ++k) v[q][k] = 0.0;
  }
  __device__ __forceinline__ void add_vol(double V, const W8<double>& W) {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[0][k] += V * W.w[k];
  }
  __device__ __forceinline__ void add_drag(double f, double fu0, double fu1, double fu2,
                                           const W8<double>& W) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      v[1][k] += f * W.w[k];
      v[2][k] += fu0 * W.w[k];
      v[3][k] += fu1 * W.w[k];
      v[4][k] += fu2 * W.w[k];
    }
  }
  __device__ __forceinline__ double get(int q, int k) const { return v[q][k]; }
  // quantities [Q0, Q1) into cb ([NQ*4][CT] double2, see cbuf_get) as thread t's
  template <int Q0, int Q1>
  __device__ __forceinline__ void store(double* cb, int t) const {
    double2* c2 = reinterpret_cast<double2*>(cb);
#pragma unroll
    for (int q = Q0; q < Q1; ++q)
#pragma unroll
      for (int h = 0; h < 4; ++h) c2[(q * 4 + h) * CT + t] = make_double2(v[q][2 * h], v[q][2 * h + 1]);
  }
};
template <> struct CellSums<float> {
  float2 v[NQ][4];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
      for (int k = 0; k < 4; ++k) v[q][k] = make_float2(0.0f, 0.0f);
  }
  __device__ __forceinline__ void add_vol(float V, const W8<float>& W) {
    const float2 s = make_float2(V, V);
#pragma unroll
    for (int k = 0; k < 4; ++k) v[0][k] = __ffma2_rn(s, W.w[k], v[0][k]);
  }
  __device__ __forceinline__ void add_drag(float f, float fu0, float fu1, float fu2,
                                           const W8<float>& W) {
    const float2 s1 = make_float2(f, f), s2 = make_float2(fu0, fu0), s3 = make_float2(fu1, fu1),
                 s4 = make_float2(fu2, fu2);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      v[1][k] = __ffma2_rn(s1, W.w[k], v[1][k]);
      v[2][k] = __ffma2_rn(s2, W.w[k], v[2][k]);
      v[3][k] = __ffma2_rn(s3, W.w[k], v[3][k]);
      v[4][k] = __ffma2_rn(s4, W.w[k], v[4][k]);
    }
  }
  __device__ __forceinline__ float get(int q, int k) const {
    return (k & 1) ? v[q][k >> 1].y : v[q][k >> 1].x;
  }
  // quantities [Q0, Q1) into cb ([NQ*2][CT] float4, see cbuf_get) as thread t's
  template <int Q0, int Q1>
  __device__ __forceinline__ void store(float* cb, int t) const {
    float4* c4 = reinterpret_cast<float4*>(cb);
#pragma unroll
    for (int q = Q0; q < Q1; ++q)
#pragma unroll
      for (int h = 0; h < 2; ++h)
        c4[(q * 2 + h) * CT + t] = make_float4(v[q][2 * h].x, v[q][2 * h].y, v[q][2 * h + 1].x, v[q][2 * h + 1].y);
  }
};

// Corner k of quantity q of the sums thread t left in cb (CellSums::store): vectors of VW
// corners, [NQ * 8 / VW][CT], so that the threads of a warp store and load contiguous vectors.
template <class T>
__device__ __forceinline__ T cbuf_get(const T* cb, int q, int k, int t) {
  constexpr int VW = TileVec<T>::n;
  return cb[((q * (8 / VW) + k / VW) * CT + t) * VW + k % VW];
}

// Interpolation at one parcel from the brick's node-field tile (corner (0,0,0) at tile node
// base) with precomputed weights. The gradient of the trilinear interpolant of tau is
// formed from differences across the cell faces: d/dx = (1/dx) sum_{b,c} (tau_1bc -
// tau_0bc) w_y,b w_z,c, and likewise for y and z.
template <class T>
__device__ __forceinline__ void interp_tile_w(const KParams<T>& p, const T* t, int base, int ta,
                                              const Weights<T>& w, Interp<T>& r) {
  T tau[8];
  r.es = 0;
  for (int a = 0; a < 3; ++a) { r.ug[a] = 0; r.gp[a] = 0; }
  const bool gpf = p.has_gp != 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    T v[8];
    tile_node(t, base + (q & 1) + TX * (((q >> 1) & 1) + TY * (q >> 2)), gpf, ta, v);
    const T Wq = w.W.get(q);
    r.es += Wq * v[0];
    r.ug[0] += Wq * v[1];
    r.ug[1] += Wq * v[2];
    r.ug[2] += Wq * v[3];
    tau[q] = v[4];
    if (gpf) {
      r.gp[0] += Wq * v[5];
      r.gp[1] += Wq * v[6];
      r.gp[2] += Wq * v[7];
    }
  }
  if (!gpf) { r.gp[0] = p.gp[0]; r.gp[1] = p.gp[1]; r.gp[2] = p.gp[2]; }
  T gx = 0, gy = 0, gz = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int u0 = q & 1, u1 = q >> 1;
    const T wx = u0 ? w.xi[0] : T(1) - w.xi[0];
    const T wy = u1 ? w.xi[1] : T(1) - w.xi[1];
    const T wz = u1 ? w.xi[2] : T(1) - w.xi[2];
    gx += (tau[1 + 2 * u0 + 4 * u1] - tau[2 * u0 + 4 * u1]) * w.yz[q];
    gy += (tau[u0 + 2 + 4 * u1] - tau[u0 + 4 * u1]) * (wx * wz);
    gz += (tau[u0 + 2 * u1 + 4] - tau[u0 + 2 * u1]) * (wx * wy);
  }
  r.gt[0] = gx * p.invh[0];
  r.gt[1] = gy * p.invh[1];
  r.gt[2] = gz * p.invh[2];
}

// The same interpolation in the FP32 form with paired operations: (eps_s, u_g,x) and
// (u_g,y, u_g,z) are summed as two pairs per corner, and the x and y components of the
// stress gradient as one pair (each lane one rounded operation: the scalar values).
__device__ __forceinline__ void interp_tile_w(const KParams<float>& p, const float* t, int base,
                                              int ta, const Weights<float>& w, Interp<float>& r) {
  float2 e0 = make_float2(0.0f, 0.0f), e1 = make_float2(0.0f, 0.0f), g01 = make_float2(0.0f, 0.0f);
  float g2 = 0.0f;
  float tau[8];
  const bool gpf = p.has_gp != 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int n = base + (q & 1) + TX * (((q >> 1) & 1) + TY * (q >> 2));
    const float4 a = *reinterpret_cast<const float4*>(t + 4 * n);
    const float Wq = w.W.get(q);
    const float2 W2 = make_float2(Wq, Wq);
    e0 = __ffma2_rn(W2, make_float2(a.x, a.y), e0);
    e1 = __ffma2_rn(W2, make_float2(a.z, a.w), e1);
    tau[q] = t[ta + n];
    if (gpf) {
      const float4 g = *reinterpret_cast<const float4*>(t + 4 * (TNODES + n));
      g01 = __ffma2_rn(W2, make_float2(g.x, g.y), g01);
      g2 += Wq * g.z;
    }
  }
  r.es = e0.x; r.ug[0] = e0.y; r.ug[1] = e1.x; r.ug[2] = e1.y;
  if (gpf) { r.gp[0] = g01.x; r.gp[1] = g01.y; r.gp[2] = g2; }
  else { r.gp[0] = p.gp[0]; r.gp[1] = p.gp[1]; r.gp[2] = p.gp[2]; }
  float2 gxy = make_float2(0.0f, 0.0f);
  float gz = 0.0f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int u0 = q & 1, u1 = q >> 1;
    const float wx = u0 ? w.xi[0] : 1.0f - w.xi[0];
    const float wy = u1 ? w.xi[1] : 1.0f - w.xi[1];
    const float wz = u1 ? w.xi[2] : 1.0f - w.xi[2];
    const float2 dxy = __fadd2_rn(make_float2(tau[1 + 2 * u0 + 4 * u1], tau[u0 + 2 + 4 * u1]),
                                  make_float2(-tau[2 * u0 + 4 * u1], -tau[u0 + 4 * u1]));
    gxy = __ffma2_rn(dxy, make_float2(w.yz[q], wx * wz), gxy);
    gz += (tau[u0 + 2 * u1 + 4] - tau[u0 + 2 * u1]) * (wx * wy);
  }
  const float2 gt = __fmul2_rn(gxy, make_float2(p.invh[0], p.invh[1]));
  r.gt[0] = gt.x;
  r.gt[1] = gt.y;
  r.gt[2] = gz * p.invh[2];
}

// Wen-Yu drag coefficient in the FP32 form: the two powers of the voidage share one log2.
__device__ __forceinline__ float wen_yu_step(const KParams<float>& p, float d, float es,
                                             const float (&s)[3]) {
  const float eg = fmaxf(1.0f - es, p.eg_min);
  const float de = p.sd * d;
  const float inv_de = __fdividef(1.0f, de);
  const float s2 = s[0] * s[0] + s[1] * s[1] + s[2] * s[2];
  const float smag = s2 > 0.0f ? s2 * rsqrtf(s2) : 0.0f;
  const float rem = eg * de * smag * p.kRe;
  const float lg = __log2f(eg);
  if (rem < 1000.0f)
    return p.kD1 * (1.0f + 0.15f * exp2f(0.687f * __log2f(rem))) * exp2f(-2.65f * lg) *
           (inv_de * inv_de);
  return p.kD2 * smag * exp2f(-1.65f * lg) * inv_de;
}
__device__ __forceinline__ double wen_yu_step(const KParams<double>& p, double d, double es,
                                              const double (&s)[3]) {
  return wen_yu_fast(p, d, es, s);
}

// Syamlal-O'Brien drag (the paper's closure, Sec. 2.1) as an acceleration coefficient:
// D = C 3/4 C_D eps_g rho_g |s| / (V_r^2 d rho_p) with Dallavalle's C_D at Re / V_r and the
// velocity ratio V_r of Re = rho_g d |s| / mu, A = eps_g^4.14 and B = 0.8 eps_g^1.28
// (eps_g <= 0.85) or eps_g^2.65, evaluated as
//   V_r = (A + t / (sqrt(r^2 + t) + r)) / 2,  r = 0.06 Re,  t = A^2 + 2r (2B - A)
// (no cancellation: t > 0 since A < 2B) and C_D |s| = (0.63 sqrt|s| + 4.8 sqrt(V_r mu /
// (rho_g d)))^2, finite at zero slip.
__device__ __forceinline__ float syamlal_obrien_step(const KParams<float>& p, float d, float es,
                                                     const float (&s)[3]) {
  const float eg = fmaxf(1.0f - es, p.eg_min);
  const float de = p.sd * d;
  const float inv_de = __fdividef(1.0f, de);
  const float s2 = s[0] * s[0] + s[1] * s[1] + s[2] * s[2];
  const float smag = s2 > 0.0f ? s2 * rsqrtf(s2) : 0.0f;
  const float r = 0.06f * (p.kRe * de * smag);
  const float lg = __log2f(eg);
  const float A = exp2f(4.14f * lg);
  const float B = eg <= 0.85f ? 0.8f * exp2f(1.28f * lg) : exp2f(2.65f * lg);
  const float t = A * A + 2.0f * r * (2.0f * B - A);
  const float vr = 0.5f * (A + __fdividef(t, sqrtf(r * r + t) + r));
  const float root = 0.63f * sqrtf(smag) + 4.8f * sqrtf(vr * p.kS2 * inv_de);
  return p.kS1 * root * root * eg * __fdividef(inv_de, vr * vr);
}
__device__ __forceinline__ double syamlal_obrien_step(const KParams<double>& p, double d, double es,
                                                      const double (&s)[3]) {
  const double eg = fmax(1.0 - es, p.eg_min);
  const double de = p.sd * d;
  const double smag = sqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
  const double r = 0.06 * (p.kRe * de * smag);
  const double A = pow(eg, 4.14);
  const double B = eg <= 0.85 ? 0.8 * pow(eg, 1.28) : pow(eg, 2.65);
  const double t = A * A + 2.0 * r * (2.0 * B - A);
  const double vr = 0.5 * (A + t / (sqrt(r * r + t) + r));
  const double root = 0.63 * sqrt(smag) + 4.8 * sqrt(vr * p.kS2 / de);
  return p.kS1 * root * root * eg / (vr * vr * de);
}

// Ergun's dense-bed drag as an acceleration coefficient: D = C (150 eps_s mu / (eps_g d^2) +
// 1.75 rho_g |s| / d) / rho_p, with eps_s = 1 - eps_g of the floored voidage.
template <class T>
__device__ __forceinline__ T ergun_step(const KParams<T>& p, T d, T es, const T (&s)[3]) {
  const T eg = tmax(T(1) - es, p.eg_min);
  const T inv_de = frcp(p.sd * d);
  const T smag = fsqrt(s[0] * s[0] + s[1] * s[1] + s[2] * s[2]);
  return p.kE1 * (T(1) - eg) * frcp(eg) * (inv_de * inv_de) + p.kE2 * smag * inv_de;
}

// Gidaspow drag: Ergun below a voidage of 0.8, Wen-Yu at and above it; the blend weights them
// with phi = atan(262.5 (0.2 - eps_s)) / pi + 1/2 (Wen-Yu weight), eps_s = 1 - floored eps_g.
__device__ __forceinline__ float tatan(float a) { return atanf(a); }
__device__ __forceinline__ double tatan(double a) { return atan(a); }
template <class T>
__device__ __forceinline__ T gidaspow_step(const KParams<T>& p, T d, T es, const T (&s)[3], bool blend) {
  const T eg = tmax(T(1) - es, p.eg_min);
  if (!blend) return eg < T(0.8) ? ergun_step(p, d, es, s) : wen_yu_step(p, d, es, s);
  const T phi = tatan(T(262.5) * (T(0.2) - (T(1) - eg))) * T(0.31830988618379067) + T(0.5);
  return (T(1) - phi) * ergun_step(p, d, es, s) + phi * wen_yu_step(p, d, es, s);
}

// The drag closure of the step kernels. DRAG = 0: Wen-Yu only (the fast path); DRAG = 1: the
// closure each bed's drag_model names.
template <class T, int DRAG>
__device__ __forceinline__ T drag_step(const KParams<T>& p, T d, T es, const T (&s)[3]) {
  if (DRAG == 0) return wen_yu_step(p, d, es, s);
  switch (p.drag_model) {
    case DRAG_SYAMLAL_OBRIEN: return syamlal_obrien_step(p, d, es, s);
    case DRAG_GIDASPOW: return gidaspow_step(p, d, es, s, false);
    case DRAG_GIDASPOW_BLEND: return gidaspow_step(p, d, es, s, true);
    default: return wen_yu_step(p, d, es, s);
  }
}

// Deterministic sum of three per-thread values over the CTA (NW warps): a fixed shuffle tree
// in each warp, then the warp partials in warp order.
template <int NW, class T>
__device__ void cta_sum3(T a, T b, T c, T* sm, double* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(FULL, a, o);
    b += __shfl_down_sync(FULL, b, o);
    c += __shfl_down_sync(FULL, c, o);
  }
  if (lane == 0) { sm[3 * warp] = a; sm[3 * warp + 1] = b; sm[3 * warp + 2] = c; }
  __syncthreads();
  if (threadIdx.x == 0) {
    T A = 0, B = 0, C = 0;
    for (int w = 0; w < NW; ++w) { A += sm[3 * w]; B += sm[3 * w + 1]; C += sm[3 * w + 2]; }
    out[0] = (double)A; out[1] = (double)B; out[2] = (double)C;
  }
}

// The cell kernel. One CTA of CT threads owns one brick (taken from a work counter:
// persistent grid). Thread t owns two cells of it: local cell t of the lower half and the
// upper-half cell of the brick's pair map (chosen at each sort so that the threads' parcel
// counts are even, pair_layout); it walks the parcels of the first cell, then those of the
// second. Warp w (threads 32w..32w+31) stores its threads' parcels by level (the r-th parcel
// of every thread that has one, in thread order), so the warp's r-th iteration reads and
// writes one contiguous run.
// MODE_VOLUME: deposit the solids volume of the current positions.
// MODE_STEP: one full step (interp from a shared node-field tile, drag, drag sums,
// objectives, push, walls, re-bin), depositing the solids volume of the new positions
// for the next step. src/dst may be the same arrays; if not, the read-only arrays are
// copied too. key_out (nullable) receives the sort key of every new position (the step
// before a sort, so the sort needs no key pass).
// MODE_DRAG: the drag sums A, B of the current state against the current node gas velocity,
// parcels unchanged (a gas iteration of implicit coupling).
// A thread sums the contributions of its current cell's parcels (old position for the drag
// sums, new position for the volume) at the cell's 8 corners in registers: up to 40 sums.
// When it moves on to its second cell it leaves the first cell's sums in shared memory;
// at the brick's end both cells' sums are added to a shared node tile in 8 corner phases
// (no two cells of a phase share a node, so plain adds in a fixed order are deterministic).
// In the FP32 form the thread also sums its parcels' volumes exactly in fixed point, per
// cell, and the corner with the largest sum takes that total minus the other seven, so the
// deposited volume of a cell is exactly the sum of its parcels' volumes. A parcel that is not
// in its sorted cell (it drifted since the last sort, or moved this step) adds its
// contributions in exact fixed point to a second shared tile (or, outside the brick, to the
// global accumulators). Both tiles go to the brick's slot in fixed point once per brick.
// Threads wait on each other only at the brick's start and end.
// DRAG: 0 Wen-Yu only, 1 the drag closure of each bed's drag_model.
// gp_tile: the node-field tile holds the grad p planes (some bed has a node field).
template <class T> struct CellOccupancy;
template <> struct CellOccupancy<float> { static constexpr int ctas = 3; };
template <> struct CellOccupancy<double> { static constexpr int ctas = 2; };

// BATCH: the parameters of each brick's bed come from `beds` (copied to shared memory when
// the bed changes); otherwise from p0, which the kernel reads in place from its constant
// parameter space (no copy, no per-use shared-memory load).
template <class T, int MODE, int DRAG, bool BATCH, bool PERM = false>
__global__ void __launch_bounds__(CT, CellOccupancy<T>::ctas)
k_cells(const __grid_constant__ KParams<T> p0, const KParams<T>* __restrict__ beds,
        const int* __restrict__ brick_bed, long long total_bricks,
        unsigned long long* __restrict__ work, PArrays<T> src, PArrays<T> dst,
        int* __restrict__ cell_out, uint32_t* __restrict__ key_out, double* __restrict__ obj_part,
        long long np, int gp_tile) {
  typedef CellSmem<T> S;
  constexpr int W = S::W;
  constexpr bool EXACT_V = W == 1 && MODE != MODE_DRAG;  // FP32 form: exact cell volume totals
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ KParams<T> sp;                        // parameters of the current brick's bed
  __shared__ long long s_brick;
  __shared__ int s_kr[2];                          // node layers deposited into by this brick
  __shared__ int s_wsum[CT / 32];                  // parcels of each warp's cells
  const bool gpl = gp_tile != 0;
  const int ta = tau_off(gpl);                     // tau plane of the node-field tile
  T* sf = reinterpret_cast<T*>(smem);              // node-field tile (planes)
  u64* fx = reinterpret_cast<u64*>(smem + S::fx(gpl));  // [NQ][W][TNODES] exact fixed point
  T* tile = reinterpret_cast<T*>(smem + S::tile(gpl));  // [NQ][TNODES] sums of the cells' own parcels
  T* cbuf = reinterpret_cast<T*>(smem + S::cbuf(gpl));  // sums of each thread's first cell
  long long* vbuf = reinterpret_cast<long long*>(smem + S::vbuf(gpl));
  T* red = sf;                                     // after the parcel loop: objective partials
  // the warp's off-cell queues (old position, new position): records of 8 values
  constexpr int QCAP = S::QCAP;
  T* q_old = tile + (threadIdx.x >> 5) * 2 * QCAP * 8;
  T* q_new = q_old + QCAP * 8;

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  const unsigned below = (1u << lane) - 1u;
  int cur_bed = -1;
  const bool copy_ro = src.a[0] != dst.a[0];
  // quantities this mode deposits: [q0, q1)
  constexpr int q0 = MODE == MODE_DRAG ? 1 : 0;
  constexpr int q1 = MODE == MODE_VOLUME ? 1 : NQ;
  const int epoch = *(BATCH ? beds[0].epoch : p0.epoch);

  // one brick, with its bed's parameters p
  auto brick = [&](const KParams<T>& p, const long long b) {
  const unsigned bu = (unsigned)(b - p.bbase);   // brick within its bed
  const int bi0 = (int)(bu % (unsigned)p.nbx) * BX;
  const int bj0 = (int)((bu / (unsigned)p.nbx) % (unsigned)p.nby) * BY;
  const int bk0 = (int)(bu / ((unsigned)p.nbx * (unsigned)p.nby)) * BZ;
  const CellBits cb = cell_bits(p);
  const long long kbase = b * BCELLS;
  if (p.cstart[kbase] == p.cstart[kbase + BCELLS]) {
    if (MODE == MODE_STEP && tid == 0) { obj_part[3 * b] = 0; obj_part[3 * b + 1] = 0; obj_part[3 * b + 2] = 0; }
    return;
  }

  // this thread's cells (the second from the pair map of the last sort) and their parcels
  const int lcB = p.cellmap[kbase + tid];
  const int nA = p.cstart[kbase + tid + 1] - p.cstart[kbase + tid];
  const int nB = p.cstart[kbase + lcB + 1] - p.cstart[kbase + lcB];
  const int n = nA + nB;
  {
    const int ws = __reduce_add_sync(FULL, n);
    if (lane == 0) s_wsum[warp] = ws;
  }
  for (int e = tid + q0 * W * TNODES; e < q1 * W * TNODES; e += CT) fx[e] = 0;
  if (tid == 0) { s_kr[0] = 1 << 30; s_kr[1] = -1; }
  if (MODE != MODE_VOLUME) {
    // asynchronous copies, all in flight at once; absent nodes and fields are zero. The drag
    // sums need only eps_s and u_g.
    constexpr int nf = MODE == MODE_DRAG ? 4 : 8;
    for (int tn = tid; tn < TNODES; tn += CT) {
      const int i = bi0 + tn % TX, j = bj0 + (tn / TX) % TY, k = bk0 + tn / (TX * TY);
      const bool in = i <= p.nx && j <= p.ny && k <= p.nz;
      const long long nid = in ? node_id(p, i, j, k) : 0;
#pragma unroll
      for (int f = 0; f < nf; ++f) {
        if (f >= 5 && !p.has_gp) continue;       // grad p planes are read only for a node field
        T* dstv = sf + tile_off<T>(f, tn, ta);
        if (in)
          cp_async(dstv, (f < 5 ? (const T*)p.fld[f] : p.gpf[f - 5]) + nid);
        else
          *dstv = T(0);
      }
    }
    cp_async_commit();
  }
  __syncthreads();                               // the warps' parcel counts are written

  // the cell whose parcels the thread walks (the first one with parcels), and sw: the level
  // at which it moves on to the second (-1: it does not)
  int lc = nA > 0 ? tid : lcB;
  const int sw = nA > 0 && nB > 0 ? nA : -1;
  int ci = bi0 + lc % BX, cj = bj0 + (lc / BX) % BY, ck = bk0 + lc / (BX * BY);
  const int nmax = __reduce_max_sync(FULL, n);
  int off = p.cstart[kbase];                     // the group's first parcel
  for (int w = 0; w < warp; ++w) off += s_wsum[w];
  CellSums<T> sums;
  sums.zero();
  long long vtot = 0;                            // EXACT_V: the current cell's volume, fixed point
  T o_dp = 0, o_hn = 0, o_vs = 0;
  int n_old = 0, n_new = 0;                      // records in the warp's off-cell queues
  auto drain_old = [&]() {
    if (MODE == MODE_VOLUME)
      drain_offcell<T, 1, EXACT_V>(p, fx, s_kr, bi0, bj0, bk0, cb, 0, q_old, n_old);
    else
      drain_offcell<T, 4>(p, fx, s_kr, bi0, bj0, bk0, cb, 1, q_old, n_old);
  };
  auto drain_new = [&]() { drain_offcell<T, 1, EXACT_V>(p, fx, s_kr, bi0, bj0, bk0, cb, 0, q_new, n_new); };

  // Level r+1's parcel values are loaded into registers (nv) while level r is processed, so
  // that their latency is covered by one iteration. PERM (a step or volume deposit after a
  // sort that wrote only the permutation): the values of layout position q are read from
  // index src.perm[q];
  // each level's load also fetches the next level's index, one iteration ahead of its use.
  int pf_off = off;                              // first position of the next level to load
  uint32_t pf_src = 0;                           // PERM: this thread's index in that level
  auto perm_at = [&](int lv, int base) -> uint32_t {
    const bool a = n > lv;
    const unsigned bl = __ballot_sync(FULL, a);
    return a ? __ldg(src.perm + base + __popc(bl & below)) : 0u;
  };
  T nv[8];
#pragma unroll
  for (int f = 0; f < 8; ++f) nv[f] = T(0);
  auto load_level = [&](int lv) {
    const bool a = n > lv;
    const unsigned bl = __ballot_sync(FULL, a);
    if (a) {
      const int q = pf_off + __popc(bl & below);
      const uint32_t sq = PERM ? pf_src : (uint32_t)q;
#pragma unroll
      for (int f = 0; f < 8; ++f)
        if (MODE != MODE_VOLUME || f < 3 || f >= 6) nv[f] = src.a[f][sq];
    }
    pf_off += __popc(bl);
    if (PERM && lv + 1 < nmax) pf_src = perm_at(lv + 1, pf_off);
  };
  // the first level's loads are in flight while the node-field tile completes
  if (MODE != MODE_VOLUME && PERM && nmax > 0) pf_src = perm_at(0, pf_off);
  if (MODE != MODE_VOLUME && nmax > 0) load_level(0);
  if (MODE != MODE_VOLUME) cp_async_wait<0>();
  __syncthreads();                               // the node-field tile is complete
  if constexpr (MODE == MODE_VOLUME) {
    // The volume deposit's work per level is short: one level of prefetch would leave the
    // loads' latency (after a sort, the permutation's index and then the values) exposed at
    // every level. Its loads are issued VG levels at a time: the group's indices, then its
    // values; then the group's levels are processed in order, as the step's loop does.
    constexpr int VG = 8;
    int ld_off = off;                            // first position of the next level to load
    for (int r0 = 0; r0 < nmax; r0 += VG) {
      uint32_t gq[VG];
      T gv[VG][5];                               // x y z d omega
#pragma unroll
      for (int u = 0; u < VG; ++u) {
        const bool a = n > r0 + u;
        const unsigned bl = __ballot_sync(FULL, a);
        const int q = ld_off + __popc(bl & below);
        gq[u] = a ? (PERM ? __ldg(src.perm + q) : (uint32_t)q) : 0u;
        ld_off += __popc(bl);
      }
#pragma unroll
      for (int u = 0; u < VG; ++u) {
        const bool a = n > r0 + u;
#pragma unroll
        for (int f = 0; f < 5; ++f) gv[u][f] = a ? src.a[f < 3 ? f : f + 3][gq[u]] : T(0);
      }
#pragma unroll
      for (int u = 0; u < VG; ++u) {
        const int r = r0 + u;
        if (r >= nmax) break;                    // uniform over the warp
        const bool act = n > r;
        const unsigned bal = __ballot_sync(FULL, act);
        if (r == sw) {           // the first cell is done: leave its sums, go on to the second
          sums.template store<q0, q1>(cbuf, tid);
          if (EXACT_V) vbuf[tid] = vtot;
          sums.zero();
          vtot = 0;
          lc = lcB;
          ci = bi0 + lc % BX; cj = bj0 + (lc / BX) % BY; ck = bk0 + lc / (BX * BY);
        }
        bool off_old = false;
        int co = 0;
        T xo[3] = {T(0), T(0), T(0)};
        T V = T(0);
        if (act) {
          const T d = gv[u][3], om = gv[u][4];
          Cell3<T> c;
          const bool own = bin3_expect(p, gv[u][0], gv[u][1], gv[u][2], ci, cj, ck, c);
          V = om * (d * d * d) * p.vcoef;
          if (own) {
            W8<T> Wq;
            T yz[4];
            corner_weights(c.xi, Wq, yz);
            sums.add_vol(V, Wq);
            if (EXACT_V) { u64 vf[W]; to_fixed(V, p.mV, vf, p.errs); vtot += (long long)vf[0]; }
          } else {
            off_old = true;
            co = pack_cell(p, cb, c.i, c.j, c.k);
            xo[0] = c.xi[0]; xo[1] = c.xi[1]; xo[2] = c.xi[2];
          }
        }
        const unsigned po = __ballot_sync(FULL, off_old);
        if (po) {
          if (n_old + __popc(po) > QCAP) { drain_old(); n_old = 0; }
          n_old = queue_offcell(q_old, n_old, po, co, xo[0], xo[1], xo[2], V, T(0), T(0), T(0));
        }
        off += __popc(bal);
      }
    }
  } else {
  for (int r = 0; r < nmax; ++r) {
    T cv[8];
#pragma unroll
    for (int f = 0; f < 8; ++f) cv[f] = nv[f];
    if (r + 1 < nmax) load_level(r + 1);
    const bool act = n > r;
    const unsigned bal = __ballot_sync(FULL, act);
    if (r == sw) {               // the first cell is done: leave its sums, go on to the second
      sums.template store<q0, q1>(cbuf, tid);
      if (EXACT_V) vbuf[tid] = vtot;
      sums.zero();
      vtot = 0;
      lc = lcB;
      ci = bi0 + lc % BX; cj = bj0 + (lc / BX) % BY; ck = bk0 + lc / (BX * BY);
    }
    // parcels off their sorted cell: recorded here, deposited by the whole warp below
    bool off_old = false, off_new = false;       // at the old position / the new one
    int co = 0, cno = 0;                         // their cell ids
    T xo[3] = {T(0), T(0), T(0)}, xno[3] = {T(0), T(0), T(0)};
    T V = T(0), fd[4] = {T(0), T(0), T(0), T(0)};
    if (act) {
      const int q = off + __popc(bal & below);
      const T x = cv[0], y = cv[1], z = cv[2];
      const T d = cv[6], om = cv[7];
      Cell3<T> c;
      const bool own = bin3_expect(p, x, y, z, ci, cj, ck, c);
      V = om * (d * d * d) * p.vcoef;
      if (!own) {
        co = pack_cell(p, cb, c.i, c.j, c.k);
        xo[0] = c.xi[0]; xo[1] = c.xi[1]; xo[2] = c.xi[2];
      }
      if (MODE == MODE_VOLUME) {
        if (own) {
          W8<T> Wq;
          T yz[4];
          corner_weights(c.xi, Wq, yz);
          sums.add_vol(V, Wq);
          if (EXACT_V) { u64 vf[W]; to_fixed(V, p.mV, vf, p.errs); vtot += (long long)vf[0]; }
        } else {
          off_old = true;
        }
      } else {
        const T u = cv[3], v = cv[4], w = cv[5];
        const int ti = c.i - bi0, tj = c.j - bj0, tk = c.k - bk0;
        const bool inb = ti >= 0 && ti < BX && tj >= 0 && tj < BY && tk >= 0 && tk < BZ;
        Weights<T> wt;
        all_weights(c.xi, wt);
        Interp<T> I;
        if (inb) {
          interp_tile_w(p, sf, ti + TX * (tj + TY * tk), ta, wt, I);
        } else {  // outside the brick (rare): from the global node arrays
          Fields<T> FG;
          for (int f = 0; f < 5; ++f) FG.f[f] = p.fld[f];
          for (int a = 0; a < 3; ++a) FG.g[a] = p.gpf[a];
          interp8(p, FG, p.has_gp != 0, node_id(p, c.i, c.j, c.k), 1, p.nx + 1,
                  (long long)(p.nx + 1) * (p.ny + 1), c.xi, I);
        }
        T up[3] = {u, v, w};
        const T s[3] = {I.ug[0] - u, I.ug[1] - v, I.ug[2] - w};
        const T D = drag_step<T, DRAG>(p, d, I.es, s);
        const T f = p.rho_p * V * D;
        // drag sums of the pre-push state, at the old position
        if (own) {
          sums.add_drag(f, f * u, f * v, f * w, wt.W);
        } else {
          off_old = true;
          fd[0] = f; fd[1] = f * u; fd[2] = f * v; fd[3] = f * w;
        }
        if (MODE == MODE_STEP) {
          o_dp += f * s[2];
          o_hn += V * z;
          o_vs += V;
          // semi-implicit push (Eq. 4 / (eps_P rho_P), drag implicit), Eq. 3, specular walls
          T pos[3] = {x, y, z};
          const T inv_den = frcp(T(1) + p.dt * D);
          const T inv_esr = I.es > T(1e-12) ? frcp(I.es * p.rho_p) : T(0);
          bool bad = false;
#pragma unroll
          for (int a = 0; a < 3; ++a) {
            const T acc = D * I.ug[a] + p.g[a] - I.gp[a] * p.inv_rho_p - I.gt[a] * inv_esr;
            T un = (up[a] + p.dt * acc) * inv_den;
            T xn = pos[a] + p.dt * un;
            if (xn < T(0)) { xn = -xn; un = -p.e_wall * un; }
            else if (xn > p.L[a]) { xn = T(2) * p.L[a] - xn; un = -p.e_wall * un; }
            // a non-finite velocity makes the position non-finite, which fails this test too
            if (!(xn >= T(0) && xn <= p.L[a])) bad = true;
            pos[a] = xn;
            up[a] = un;
          }
          if (bad) atomicOr(p.errs, ERR_DOMAIN);
          // solids volume of the new position, for the next step
          Cell3<T> cn;
          if (bin3_expect(p, pos[0], pos[1], pos[2], ci, cj, ck, cn)) {
            W8<T> Wq;
            T yz[4];
            corner_weights(cn.xi, Wq, yz);
            sums.add_vol(V, Wq);
            if (EXACT_V) { u64 vf[W]; to_fixed(V, p.mV, vf, p.errs); vtot += (long long)vf[0]; }
          } else {
            off_new = true;
            cno = pack_cell(p, cb, cn.i, cn.j, cn.k);
            xno[0] = cn.xi[0]; xno[1] = cn.xi[1]; xno[2] = cn.xi[2];
          }
          dst.a[0][q] = pos[0]; dst.a[1][q] = pos[1]; dst.a[2][q] = pos[2];
          dst.a[3][q] = up[0]; dst.a[4][q] = up[1]; dst.a[5][q] = up[2];
          if (copy_ro) {
            dst.a[6][q] = d; dst.a[7][q] = om;
            if (src.pid || src.tag) {
              const uint32_t sq = PERM ? __ldg(src.perm + q) : (uint32_t)q;
              if (src.pid) dst.pid[q] = src.pid[sq];
              if (src.tag) dst.tag[q] = src.tag[sq];
            }
          }
          if (cell_out) cell_out[q] = cell_id(p, cn.i, cn.j, cn.k);
          if (key_out) key_out[q] = (uint32_t)(p.bbase * BCELLS) + brick_key(p, cn.i, cn.j, cn.k);
        }
      }
    }
    {                            // queue the parcels off their cell (a full queue is drained first)
      const unsigned po = __ballot_sync(FULL, off_old);
      if (po) {
        if (n_old + __popc(po) > QCAP) { drain_old(); n_old = 0; }
        if (MODE == MODE_VOLUME)
          n_old = queue_offcell(q_old, n_old, po, co, xo[0], xo[1], xo[2], V, T(0), T(0), T(0));
        else
          n_old = queue_offcell(q_old, n_old, po, co, xo[0], xo[1], xo[2], fd[0], fd[1], fd[2], fd[3]);
      }
      const unsigned pn = MODE == MODE_STEP ? __ballot_sync(FULL, off_new) : 0u;
      if (pn) {
        if (n_new + __popc(pn) > QCAP) { drain_new(); n_new = 0; }
        n_new = queue_offcell(q_new, n_new, pn, cno, xno[0], xno[1], xno[2], V, T(0), T(0), T(0));
      }
    }
    off += __popc(bal);
  }
  }
  if (n_old) drain_old();
  if (n_new) drain_new();
  // ---- node layers of this brick's own-cell deposits (off-cell deposits recorded theirs
  // as they were made); merged into the global range below, for the next finalize
  const int ckA = bk0 + tid / (BX * BY), ckB = bk0 + lcB / (BX * BY);
  {
    const int lo = nA > 0 ? ckA : (nB > 0 ? ckB : (1 << 30));
    const int hi = nB > 0 ? ckB + 1 : (nA > 0 ? ckA + 1 : -1);
    const int klo = __reduce_min_sync(FULL, lo);
    const int khi = __reduce_max_sync(FULL, hi);
    if (lane == 0 && khi >= 0) { atomicMin(&s_kr[0], klo); atomicMax(&s_kr[1], khi); }
  }
  // the cell whose sums are in registers (lc, if the thread has parcels), the one left in
  // cbuf (the first, if the thread moved on)
  const bool has_reg = n > 0, has_buf = sw >= 0;
  // ---- FP32 volume: the 8 corner sums of each cell in fixed point, the largest replaced by
  // the cell's exact total minus the other seven
  long long vfx[8], vfb[8];
  if (EXACT_V) {
    long long sum7 = 0, sumb = 0;
    int kmax = 0, kmb = 0;
    T vmax = sums.get(0, 0), vmb = has_buf ? cbuf_get(cbuf, 0, 0, tid) : T(0);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      u64 f[W];
      to_fixed(sums.get(0, k), p.mV, f, p.errs);
      vfx[k] = (long long)f[0];
      sum7 += vfx[k];
      if (sums.get(0, k) > vmax) { vmax = sums.get(0, k); kmax = k; }
      const T bv = has_buf ? cbuf_get(cbuf, 0, k, tid) : T(0);
      to_fixed(bv, p.mV, f, p.errs);
      vfb[k] = (long long)f[0];
      sumb += vfb[k];
      if (bv > vmb) { vmb = bv; kmb = k; }
    }
    const long long vtb = has_buf ? vbuf[tid] : 0ll;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (k == kmax) vfx[k] += vtot - sum7;
      if (k == kmb) vfb[k] += vtb - sumb;
    }
  }
  // ---- the cells' sums into the tiles, one corner per phase: in a phase no two cells touch
  // the same node, so plain adds in a fixed order are deterministic (the off-cell atomics
  // into fx are complete: the loop is over).
  constexpr int qt = EXACT_V ? 1 : q0;           // first quantity summed in the float tile
  __syncthreads();
  for (int e = tid + qt * TNODES; e < q1 * TNODES; e += CT) tile[e] = T(0);
  const int tnR = lc % BX + TX * ((lc / BX) % BY + TY * (lc / (BX * BY)));
  const int tnA = tid % BX + TX * ((tid / BX) % BY + TY * (tid / (BX * BY)));
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    __syncthreads();
    const int ko = (k & 1) + TX * (((k >> 1) & 1) + TY * (k >> 2));
    if (has_reg) {
      const int tn = tnR + ko;
      if (EXACT_V) fx[tn] += (u64)vfx[k];
#pragma unroll
      for (int q = qt; q < q1; ++q) tile[q * TNODES + tn] += sums.get(q, k);
    }
    if (has_buf) {
      const int tn = tnA + ko;
      if (EXACT_V) fx[tn] += (u64)vfb[k];
#pragma unroll
      for (int q = qt; q < q1; ++q) tile[q * TNODES + tn] += cbuf_get(cbuf, q, k, tid);
    }
  }
  __syncthreads();
  if (tid == 0 && s_kr[1] >= 0) { atomicMin(&p.zr[0], s_kr[0]); atomicMax(&p.zr[1], s_kr[1]); }
  // ---- the tile in exact fixed point, plus the off-cell contributions, to the brick's slot
  // (plain stores; the node pass after the step adds the slots of the bricks that share a
  // node), stamped with this deposit's epoch
  {
    u64* slot = p.bacc + b * (long long)(NQ * W * TNODES);
    for (int e = tid + q0 * TNODES; e < q1 * TNODES; e += CT) {
      const int qq = e / TNODES, tn = e % TNODES;
      u64 f[W] = {};
      if (!(EXACT_V && qq == 0)) to_fixed(tile[e], qq == 0 ? p.mV : p.mA, f, p.errs);
      u64 carry = 0;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        const u64 g = fx[(qq * W + w) * TNODES + tn];
        const u64 s0 = f[w] + g;
        const u64 c1 = s0 < g ? 1ull : 0ull;
        f[w] = s0 + carry;
        carry = c1 + (f[w] < s0 ? 1ull : 0ull);
        slot[(qq * W + w) * TNODES + tn] = f[w];
      }
    }
    if (tid == 0) p.bstamp[b] = epoch;
  }
  if (MODE == MODE_STEP) cta_sum3<CT / 32>(o_dp, o_hn, o_vs, red, obj_part + 3 * b);
  };  // one brick

  // thread 0 takes the next brick from the work counter while the current one runs
  long long next = 0;
  if (tid == 0) next = (long long)atomicAdd(work, 1ull);
  for (long long iter = 0; iter <= total_bricks; ++iter) {
    __syncthreads();
    if (tid == 0) s_brick = next;
    __syncthreads();
    const long long b = s_brick;
    if (b >= total_bricks) break;
    if (tid == 0) next = (long long)atomicAdd(work, 1ull);
    if (BATCH) {
      const int bed = brick_bed[b];
      if (bed != cur_bed) {
        if (tid == 0) sp = beds[bed];
        cur_bed = bed;
        __syncthreads();
      }
      brick(sp, b);
    } else {
      brick(p0, b);
    }
  }  // persistent loop
}

// Fixed-point value of quantity q at node (i, j, k) of a bed: the global accumulator (the
// off-brick deposits) plus the tile slots of the bricks (at most 2 per axis) whose tile
// holds the node and that were written in deposit epoch ep.
template <class T>
__device__ __forceinline__ void node_sum(const KParams<T>& p, int ep, int q, long long n, int i,
                                         int j, int k, u64 (&f)[Words<T>::n]) {
  constexpr int W = Words<T>::n;
#pragma unroll
  for (int w = 0; w < W; ++w) f[w] = p.acc[(long long)(q * W + w) * p.nstride + p.nbase + n];
  const int bx1 = min(i / BX, p.nbx - 1), by1 = min(j / BY, p.nby - 1), bz1 = min(k / BZ, p.nbz - 1);
  const int bx0 = (i % BX == 0 && i > 0) ? i / BX - 1 : bx1;
  const int by0 = (j % BY == 0 && j > 0) ? j / BY - 1 : by1;
  const int bz0 = (k % BZ == 0 && k > 0) ? k / BZ - 1 : bz1;
  for (int bz = bz0; bz <= bz1; ++bz)
    for (int by = by0; by <= by1; ++by)
      for (int bx = bx0; bx <= bx1; ++bx) {
        const long long b = p.bbase + bx + (long long)p.nbx * (by + (long long)p.nby * bz);
        if (p.bstamp[b] != ep) continue;
        const int tn = (i - bx * BX) + TX * ((j - by * BY) + TY * (k - bz * BZ));
        const u64* slot = p.bacc + b * (long long)(NQ * W * TNODES);
        u64 carry = 0;
#pragma unroll
        for (int w = 0; w < W; ++w) {
          const u64 g = slot[(q * W + w) * TNODES + tn];
          const u64 s0 = f[w] + g;
          const u64 c1 = s0 < g ? 1ull : 0ull;
          f[w] = s0 + carry;
          carry = c1 + (f[w] < s0 ? 1ull : 0ull);
        }
      }
}

// a5: node fields from the deposited volume. Reads and clears the Vs accumulator and
// clears the drag-sum accumulators for the coming push. vs_out (nullable) receives Vs.
template <class T>
__device__ __forceinline__ void finalize_node(const KParams<T>& p, int ep, int n, int i, int j, int k,
                                              double* vs_out);

template <class T>
__global__ void k_finalize(KParams<T> p, double* __restrict__ vs_out, int full) {
  const int nx1 = p.nx + 1, ny1 = p.ny + 1;
  const int layer = nx1 * ny1;
  int klo = 0, khi = p.nz;
  if (!full) {               // layers deposited into now or at the previous finalize
    klo = max(0, min(p.zr[0], p.zr[2]));
    khi = min(p.nz, max(p.zr[1], p.zr[3]));
  }
  const int n0 = klo * layer, n1 = (khi + 1) * layer;
  const int ep = *p.epoch;
  for (int n = n0 + blockIdx.x * blockDim.x + threadIdx.x; n < n1; n += gridDim.x * blockDim.x)
    finalize_node(p, ep, n, n % nx1, (n / nx1) % ny1, n / layer, vs_out);
}

// Moves the deposit's layer range to "last finalized" and empties it for the next deposit,
// and advances the deposit epoch (the tile slots written so far are consumed).
__global__ void k_range_roll(int* zr, int* epoch) {
  zr[2] = zr[0];
  zr[3] = zr[1];
  zr[0] = 1 << 30;
  zr[1] = -1;
  *epoch += 1;
}

__global__ void k_epoch_next(int* epoch) { *epoch += 1; }

// After the last step of a call: the solids volume of the new positions and the drag sums
// A, B of the bricks' tile slots are added to the global accumulators (which then hold the
// step's complete sums, read by the volume and drag-sum outputs until the next call's deposit
// and node pass clear them). Layers of the last deposit only.
template <class T>
__global__ void k_drag_fold(KParams<T> p) {
  constexpr int W = Words<T>::n;
  const int nx1 = p.nx + 1, ny1 = p.ny + 1;
  const int layer = nx1 * ny1;
  const int klo = max(0, p.zr[0]), khi = min(p.nz, p.zr[1]);
  if (khi < klo) return;
  const int ep = *p.epoch;
  for (int n = klo * layer + blockIdx.x * blockDim.x + threadIdx.x; n < (khi + 1) * layer;
       n += gridDim.x * blockDim.x) {
    const int i = n % nx1, j = (n / nx1) % ny1, k = n / layer;
    for (int q = 0; q < NQ; ++q) {
      u64 f[W];
      node_sum(p, ep, q, n, i, j, k, f);
#pragma unroll
      for (int w = 0; w < W; ++w) p.acc[(long long)(q * W + w) * p.nstride + p.nbase + n] = f[w];
    }
  }
}

// The solids volume of the last step's new positions as doubles (after k_drag_fold).
template <class T>
__global__ void k_vol_out(KParams<T> p, double* __restrict__ Vs) {
  constexpr int W = Words<T>::n;
  long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= p.nnode) return;
  u64 fx[W];
  for (int w = 0; w < W; ++w) fx[w] = p.acc[(long long)w * p.nstride + n];
  if (W == 1 && (long long)fx[0] >= (1ll << 62)) atomicOr(p.errs, ERR_RANGE);
  Vs[n] = from_fixed(fx, p.inv_mV);
}

template <class T>
__device__ __forceinline__ void finalize_node(const KParams<T>& p, int ep, int n, int i, int j, int k,
                                              double* vs_out) {
  constexpr int W = Words<T>::n;
  u64 fx[W];
  node_sum(p, ep, 0, n, i, j, k, fx);
  if (W == 1 && (long long)fx[0] >= (1ll << 62)) atomicOr(p.errs, ERR_RANGE);
  for (int e = 0; e < NQ * W; ++e) p.acc[(long long)e * p.nstride + p.nbase + n] = 0;
  if (vs_out) vs_out[n] = from_fixed(fx, p.inv_mV);
  // the node's control volume is the cell volume halved once per boundary axis: eps_s is
  // Vs / V_n = Vs 2^nb / vcell, formed with a product (the FP32 form in FP32 from the integer:
  // the FP64 pipe is narrow on GB300, and a division per node made it this pass's bound)
  const int nb = (i == 0 || i == p.nx) + (j == 0 || j == p.ny) + (k == 0 || k == p.nz);
  T es;
  if (W == 1)
    es = (T)((float)(long long)fx[0] * (p.es_scale * (float)(1 << nb)));
  else
    es = (T)(from_fixed(fx, p.inv_mV) * (p.inv_vcell * (double)(1 << nb)));
  T eg = T(1) - es;
  T egc = tmax(eg, p.eg_min);
  const T iegc = T(1) / egc;
  T U0 = p.U[0] ? p.U[0][n] : T(0);
  T U1 = p.U[1] ? p.U[1][n] : T(0);
  T U2 = (p.U[2] ? p.U[2][n] : T(0)) + p.u_in;
  p.fld[0][n] = es;
  p.fld[1][n] = U0 * iegc;
  p.fld[2][n] = U1 * iegc;
  p.fld[3][n] = U2 * iegc;
  T den = tmax(p.eps_cp - es, p.alpha * (T(1) - es));
  p.fld[4][n] = p.Ps * tpow(es, p.beta) / den;
}

// Implicit coupling, one gas iteration at node (i, j, k) (Sec. 2.2.2, with the gas side
// reduced to the unsteady and interphase terms of Eq. 2, drag implicit): from the drag sums
// of the last drag deposit,
//   u_g' = (m u_g0 + B) / (m + A),   m = rho_g eps_g V_n / dt,
// eps_g the floored voidage of the node and u_g0 = U / eps_g the gas velocity of the step's
// start. Reads and clears the drag-sum accumulators; writes the node gas velocity. A node
// whose four drag sums are all zero (no parcel exchanges momentum there) keeps u_g0 as it is.
template <class T>
__device__ __forceinline__ void gas_update_node(const KParams<T>& p, int ep, int n, int i, int j,
                                                int k) {
  constexpr int W = Words<T>::n;
  double s[4];
  for (int q = 1; q < NQ; ++q) {
    u64 f[W];
    node_sum(p, ep, q, n, i, j, k, f);
    if (W == 1 && ((long long)f[0] >= (1ll << 62) || (long long)f[0] <= -(1ll << 62)))
      atomicOr(p.errs, ERR_RANGE);
    s[q - 1] = from_fixed(f, p.inv_mA);
    for (int w = 0; w < W; ++w) p.acc[(long long)(q * W + w) * p.nstride + p.nbase + n] = 0;
  }
  if (s[0] == 0.0 && s[1] == 0.0 && s[2] == 0.0 && s[3] == 0.0) return;
  double vn = p.vcell;
  if (i == 0 || i == p.nx) vn *= 0.5;
  if (j == 0 || j == p.ny) vn *= 0.5;
  if (k == 0 || k == p.nz) vn *= 0.5;
  const double egc = fmax(1.0 - (double)p.fld[0][n], (double)p.eg_min);
  const double m = (double)p.rho_g * egc * vn / (double)p.dt;
  for (int a = 0; a < 3; ++a) {
    double U = p.U[a] ? (double)p.U[a][n] : 0.0;
    if (a == 2) U += (double)p.u_in;
    p.fld[1 + a][n] = (T)((m * (U / egc) + s[1 + a]) / (m + s[0]));
  }
}

template <class T>
__global__ void k_gas_update(KParams<T> p) {
  const int nx1 = p.nx + 1, ny1 = p.ny + 1;
  const int layer = nx1 * ny1;
  const int klo = max(0, min(p.zr[0], p.zr[2])), khi = min(p.nz, max(p.zr[1], p.zr[3]));
  if (khi < klo) return;
  const int ep = *p.epoch;
  for (int n = klo * layer + blockIdx.x * blockDim.x + threadIdx.x; n < (khi + 1) * layer;
       n += gridDim.x * blockDim.x)
    gas_update_node(p, ep, n, n % nx1, (n / nx1) % ny1, n / layer);
}

// Drag sums of the last step as doubles.
template <class T>
__global__ void k_drag_out(KParams<T> p, double* A, double* Bx, double* By, double* Bz) {
  constexpr int W = Words<T>::n;
  long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= p.nnode) return;
  double* outs[4] = {A, Bx, By, Bz};
  for (int q = 1; q < NQ; ++q) {
    if (!outs[q - 1]) continue;
    u64 fx[W];
    for (int w = 0; w < W; ++w) fx[w] = p.acc[(long long)(q * W + w) * p.nstride + p.nbase + n];
    if (W == 1) {
      long long v = (long long)fx[0];
      if (v >= (1ll << 62) || v <= -(1ll << 62)) atomicOr(p.errs, ERR_RANGE);
    }
    outs[q - 1][n] = from_fixed(fx, p.inv_mA);
  }
}

// a6 as a standalone output: interpolate the node fields to every parcel.
template <class T>
__global__ void k_interp_out(KParams<T> p, const T* __restrict__ x, const T* __restrict__ y,
                             const T* __restrict__ z, T* __restrict__ out, long long np) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= np) return;
  Cell3<T> c;
  bin3(p, x[q], y[q], z[q], c);
  Fields<T> FG;
  for (int f = 0; f < 5; ++f) FG.f[f] = p.fld[f];
  for (int a = 0; a < 3; ++a) FG.g[a] = p.gpf[a];
  Interp<T> I;
  interp8(p, FG, p.has_gp != 0, node_id(p, c.i, c.j, c.k), 1, p.nx + 1,
          (long long)(p.nx + 1) * (p.ny + 1), c.xi, I);
  out[q] = I.es;
  for (int a = 0; a < 3; ++a) {
    out[(1 + a) * np + q] = I.ug[a];
    out[(4 + a) * np + q] = I.gp[a];
    out[(7 + a) * np + q] = I.gt[a];
  }
}

// Number of bricks holding at least one parcel in the current sorted order.
__global__ void k_count_bricks(const int* __restrict__ cstart, long long nbricks,
                               unsigned long long* __restrict__ count) {
  long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (b >= nbricks) return;
  if (cstart[(b + 1) * BCELLS] > cstart[b * BCELLS]) atomicAdd(count, 1ull);
}

// a10: deterministic reduction of the per-brick objective partials into (dP, H): OBJ_BLOCKS
// blocks each sum a fixed slice of bricks with a fixed tree; the last block to finish loads
// the slice partials at once and one thread sums them in order. obj[0] = dP = sum f s_z /
// area, obj[1] = H = 2 sum V z / sum V.
constexpr int OBJ_BLOCKS = 32, OBJ_THREADS = 256;
__global__ void k_obj_reduce(const double* __restrict__ part, long long nb, double area,
                             double* __restrict__ slices, unsigned* __restrict__ count,
                             double* __restrict__ obj) {
  static_assert(3 * OBJ_BLOCKS <= OBJ_THREADS, "one slice value per thread");
  __shared__ double s[3][OBJ_THREADS];
  __shared__ double sl[3 * OBJ_BLOCKS];
  __shared__ bool last;
  const int t = threadIdx.x;
  const long long per = (nb + gridDim.x - 1) / gridDim.x;
  const long long lo = blockIdx.x * per, hi = lo + per < nb ? lo + per : nb;
  double a = 0, b = 0, c = 0;
  for (long long i = lo + t; i < hi; i += OBJ_THREADS) {
    a += part[3 * i]; b += part[3 * i + 1]; c += part[3 * i + 2];
  }
  s[0][t] = a; s[1][t] = b; s[2][t] = c;
  __syncthreads();
  for (int off = OBJ_THREADS / 2; off > 0; off >>= 1) {
    if (t < off) { s[0][t] += s[0][t + off]; s[1][t] += s[1][t + off]; s[2][t] += s[2][t + off]; }
    __syncthreads();
  }
  if (t == 0) {
    slices[3 * blockIdx.x] = s[0][0];
    slices[3 * blockIdx.x + 1] = s[1][0];
    slices[3 * blockIdx.x + 2] = s[2][0];
    __threadfence();
    last = atomicAdd(count, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return;                             // uniform over the block
  __threadfence();                               // every slice is written
  if (t < 3 * (int)gridDim.x) sl[t] = __ldcg(slices + t);
  __syncthreads();
  if (t == 0) {                                  // in slice order
    double A = 0, B = 0, C = 0;
    for (unsigned k = 0; k < gridDim.x; ++k) { A += sl[3 * k]; B += sl[3 * k + 1]; C += sl[3 * k + 2]; }
    obj[0] = A / area;
    obj[1] = C > 0 ? 2.0 * B / C : 0.0;
    *count = 0;                                  // ready for the next launch
  }
}

// ---------------------------------------------------------------- batches --
// Several independent beds share one sort and one launch of each kernel: their parcels,
// nodes and bricks are concatenated; off arrays give each bed's first element.

__device__ __forceinline__ int find_bed(const long long* __restrict__ off, int nbeds, long long x) {
  int lo = 0, hi = nbeds;                        // largest b with off[b] <= x
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (off[mid] <= x) lo = mid; else hi = mid;
  }
  return lo;
}

template <class T>
__global__ void k_keys_b(const KParams<T>* __restrict__ beds, const long long* __restrict__ poff,
                         int nbeds, const T* __restrict__ x, const T* __restrict__ y,
                         const T* __restrict__ z, uint32_t* __restrict__ key, long long np) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= np) return;
  const KParams<T>& p = beds[find_bed(poff, nbeds, q)];
  Cell3<T> c;
  bin3(p, x[q], y[q], z[q], c);
  key[q] = (uint32_t)(p.bbase * BCELLS) + brick_key(p, c.i, c.j, c.k);
}

template <class T>
__global__ void k_bin_b(const KParams<T>* __restrict__ beds, const long long* __restrict__ poff,
                        int nbeds, const T* __restrict__ x, const T* __restrict__ y,
                        const T* __restrict__ z, int* __restrict__ cell, long long np) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= np) return;
  const KParams<T>& p = beds[find_bed(poff, nbeds, q)];
  Cell3<T> c;
  bin3(p, x[q], y[q], z[q], c);
  cell[q] = cell_id(p, c.i, c.j, c.k);
}

template <class T>
__global__ void k_finalize_b(const KParams<T>* __restrict__ beds, const long long* __restrict__ noff,
                             int nbeds, long long total) {
  const int ep = *beds[0].epoch;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const int bed = find_bed(noff, nbeds, g);
    const KParams<T>& p = beds[bed];
    const int n = (int)(g - noff[bed]);
    const int nx1 = p.nx + 1, ny1 = p.ny + 1;
    finalize_node(p, ep, n, n % nx1, (n / nx1) % ny1, n / (nx1 * ny1), (double*)nullptr);
  }
}

// k_drag_fold for a batch: every node of every bed.
template <class T>
__global__ void k_drag_fold_b(const KParams<T>* __restrict__ beds, const long long* __restrict__ noff,
                              int nbeds, long long total) {
  constexpr int W = Words<T>::n;
  const int ep = *beds[0].epoch;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const int bed = find_bed(noff, nbeds, g);
    const KParams<T>& p = beds[bed];
    const int n = (int)(g - noff[bed]);
    const int nx1 = p.nx + 1, ny1 = p.ny + 1;
    const int i = n % nx1, j = (n / nx1) % ny1, k = n / (nx1 * ny1);
    for (int q = 0; q < NQ; ++q) {
      u64 f[W];
      node_sum(p, ep, q, n, i, j, k, f);
#pragma unroll
      for (int w = 0; w < W; ++w) p.acc[(long long)(q * W + w) * p.nstride + p.nbase + n] = f[w];
    }
  }
}

// k_gas_update for a batch: every node of every bed.
template <class T>
__global__ void k_gas_update_b(const KParams<T>* __restrict__ beds, const long long* __restrict__ noff,
                               int nbeds, long long total) {
  const int ep = *beds[0].epoch;
  for (long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x; g < total;
       g += (long long)gridDim.x * blockDim.x) {
    const int bed = find_bed(noff, nbeds, g);
    const KParams<T>& p = beds[bed];
    const int n = (int)(g - noff[bed]);
    const int nx1 = p.nx + 1, ny1 = p.ny + 1;
    gas_update_node(p, ep, n, n % nx1, (n / nx1) % ny1, n / (nx1 * ny1));
  }
}

// Per-bed objectives: one CTA per bed sums the partials of its bricks in a fixed order.
// obj[2*bed] = dP, obj[2*bed+1] = H.
__global__ void k_obj_reduce_b(const double* __restrict__ part, const long long* __restrict__ boff,
                               const double* __restrict__ area, double* __restrict__ obj) {
  __shared__ double s[3][256];
  const int bed = blockIdx.x, t = threadIdx.x;
  double a = 0, b = 0, c = 0;
  for (long long i = boff[bed] + t; i < boff[bed + 1]; i += blockDim.x) {
    a += part[3 * i]; b += part[3 * i + 1]; c += part[3 * i + 2];
  }
  s[0][t] = a; s[1][t] = b; s[2][t] = c;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (t < off) { s[0][t] += s[0][t + off]; s[1][t] += s[1][t + off]; s[2][t] += s[2][t + off]; }
    __syncthreads();
  }
  if (t == 0) {
    obj[2 * bed] = s[0][0] / area[bed];
    obj[2 * bed + 1] = s[2][0] > 0 ? 2.0 * s[1][0] / s[2][0] : 0.0;
  }
}

}  // namespace mppic
