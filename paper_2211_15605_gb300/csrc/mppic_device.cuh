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
//    (brick id * 256 + local cell id). One CTA of 256 threads owns one brick.
//  * Deposits are exact integer fixed point: int64 for the FP32 form, int128 (two
//    64-bit words with carry) for the FP64 form. Integer addition is associative, so
//    every sum is independent of thread scheduling and of how far parcels drifted
//    since the last sort; the sorted order only makes the sums cheap.
//  * Inside a CTA, parcels are processed parcel-per-thread (coalesced loads, node
//    fields from a shared-memory tile), each parcel leaving a small record in shared
//    memory; then one thread per cell sums its records in registers in sorted order,
//    converts the 40 per-cell sums once to fixed point and adds them to a shared
//    node tile, which is flushed to the global accumulators once per brick.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mppic {

constexpr int BX = 8, BY = 8, BZ = 4;            // brick of cells
constexpr int BCELLS = BX * BY * BZ;             // 256 = threads per brick CTA
constexpr int TX = BX + 1, TY = BY + 1, TZ = BZ + 1;
constexpr int TNODES = TX * TY * TZ;             // 405 nodes per brick tile
constexpr int NQ = 5;                            // Vs, A, Bx, By, Bz
constexpr int ERR_DOMAIN = 1, ERR_RANGE = 2;

typedef unsigned long long u64;

// ------------------------------------------------------------ parameters --

template <class T>
struct KParams {
  int nx, ny, nz;
  int nbx, nby, nbz;
  long long nnode;
  long long nbricks;
  double inv_d[3];           // fl64(1/h): binning multiplier
  float inv_f[3], inv_lo[3]; // FP32 split: inv_d ~= inv_f + inv_lo
  T invh[3];                 // 1/h in T (interpolant gradient)
  T L[3];
  double vcell;
  T rho_g, mu_g, g[3], gp[3], rho_p, Ps, beta, eps_cp, alpha, eg_min, e_wall, C, sd, dt;
  T vcoef;                   // pi/6 * s_d^3: V = w d^3 vcoef
  T mV, mA;                  // fixed-point multipliers (value * m = integer units)
  double inv_mV, inv_mA;
  T u_in;
  // node fields: 0 eps_s, 1-3 u_g, 4 tau; 5-7 grad p (caller arrays, used if has_gp)
  T* fld[5];
  const T* gpf[3];
  int has_gp;
  const T* U[3];
  u64* acc;                  // [NQ][words][nnode]
  int* errs;
  const int* cstart;         // [nkeys+1]: first sorted parcel of each brick-major key
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

// FP32 form: the same integer result as the FP64 formula. The FP32 product is within
// 1.2e-7 |t| of the FP64 one, so away from a face its floor is the same; within
// 2.5e-7 |t| of a face the FP64 formula decides. The in-cell coordinate is computed
// with the product's exact rounding error and the low part of 1/h, so it does not lose
// the digits of i (about 1e-7 absolute instead of |t| * 6e-8).
__device__ __forceinline__ void bin_axis(float x, double inv_d, float inv_f, float inv_lo, int n,
                                         int& i, float& xi) {
  float t = __fmul_rn(x, inv_f);
  float fl = floorf(t);
  float r = __fsub_rn(t, fl);
  float tol = fabsf(t) * 2.5e-7f;
  if (!(r >= tol && r <= 1.0f - tol)) {
    double f64 = floor(__dmul_rn((double)x, inv_d));
    if (!(f64 >= 0.0)) f64 = 0.0;
    if (f64 > (double)(n - 1)) f64 = (double)(n - 1);
    fl = (float)f64;
  }
  if (!(fl >= 0.0f)) fl = 0.0f;
  if (fl > (float)(n - 1)) fl = (float)(n - 1);
  i = (int)fl;
  float lo = __fmaf_rn(x, inv_f, -t);
  xi = __fadd_rn(__fadd_rn(__fsub_rn(t, fl), lo), __fmul_rn(x, inv_lo));
  xi = fminf(fmaxf(xi, 0.0f), 1.0f);
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
__device__ __forceinline__ void interp8(const KParams<T>& p, const T* const* f, const T* const* g,
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
        r.es += W * f[0][n];
        r.ug[0] += W * f[1][n];
        r.ug[1] += W * f[2][n];
        r.ug[2] += W * f[3][n];
        T tau = f[4][n];
        r.gt[0] += ((a ? p.invh[0] : -p.invh[0]) * (w[1][b] * w[2][c])) * tau;
        r.gt[1] += ((b ? p.invh[1] : -p.invh[1]) * (w[0][a] * w[2][c])) * tau;
        r.gt[2] += ((c ? p.invh[2] : -p.invh[2]) * (w[0][a] * w[1][b])) * tau;
        if (g) {
          r.gp[0] += W * g[0][n];
          r.gp[1] += W * g[1][n];
          r.gp[2] += W * g[2][n];
        }
      }
  if (!g) { r.gp[0] = p.gp[0]; r.gp[1] = p.gp[1]; r.gp[2] = p.gp[2]; }
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

// Sort keys (brick-major) and identity values.
template <class T>
__global__ void k_keys(KParams<T> p, const T* __restrict__ x, const T* __restrict__ y,
                       const T* __restrict__ z, uint32_t* __restrict__ key,
                       uint32_t* __restrict__ val, long long np) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= np) return;
  Cell3<T> c;
  bin3(p, x[q], y[q], z[q], c);
  key[q] = brick_key(p, c.i, c.j, c.k);
  val[q] = (uint32_t)q;
}

// ------------------------------------------------------------ radix sort --
// Stable LSD radix sort of (key, value) by 8-bit digits: a per-tile digit histogram, a
// scan per digit across tiles, then a stable scatter in which each warp ranks its own
// contiguous segment with __match_any_sync.

constexpr int SORT_THREADS = 256;
constexpr int SORT_TILE = 4096;
constexpr int SORT_WARPS = SORT_THREADS / 32;
constexpr int SORT_SEG = SORT_TILE / SORT_WARPS;   // 512 keys per warp

__global__ void k_sort_hist(const uint32_t* __restrict__ key, long long n, int shift,
                            uint32_t* __restrict__ hist, int nblk) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  long long base = (long long)blockIdx.x * SORT_TILE;
  for (int it = 0; it < SORT_TILE / SORT_THREADS; ++it) {
    long long q = base + it * SORT_THREADS + threadIdx.x;
    if (q < n) atomicAdd(&h[(key[q] >> shift) & 255u], 1u);
  }
  __syncthreads();
  hist[(long long)threadIdx.x * nblk + blockIdx.x] = h[threadIdx.x];
}

// One CTA per digit: exclusive scan of that digit's per-tile counts, and its total.
__global__ void k_sort_scan(uint32_t* __restrict__ hist, int nblk, uint32_t* __restrict__ totals) {
  __shared__ uint32_t part[1024];
  uint32_t* row = hist + (long long)blockIdx.x * nblk;
  int per = (nblk + blockDim.x - 1) / blockDim.x;
  int lo = threadIdx.x * per, hi = min(nblk, lo + per);
  uint32_t s = 0;
  for (int i = lo; i < hi; ++i) s += row[i];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < blockDim.x; off <<= 1) {   // inclusive Hillis-Steele scan
    uint32_t t = threadIdx.x >= off ? part[threadIdx.x - off] : 0u;
    __syncthreads();
    part[threadIdx.x] += t;
    __syncthreads();
  }
  uint32_t run = threadIdx.x ? part[threadIdx.x - 1] : 0u;
  for (int i = lo; i < hi; ++i) {
    uint32_t c = row[i];
    row[i] = run;
    run += c;
  }
  if (threadIdx.x == blockDim.x - 1) totals[blockIdx.x] = part[threadIdx.x];
}

__global__ void k_sort_scatter(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
                               uint32_t* __restrict__ kout, uint32_t* __restrict__ vout,
                               long long n, int shift, const uint32_t* __restrict__ hist,
                               const uint32_t* __restrict__ totals, int nblk) {
  __shared__ uint32_t dbase[256];
  __shared__ uint32_t wcnt[SORT_WARPS][256];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  // digit base = exclusive scan of the digit totals + this tile's offset within the digit
  {
    __shared__ uint32_t tot[256];
    tot[tid] = totals[tid];
    __syncthreads();
    for (int off = 1; off < 256; off <<= 1) {
      uint32_t t = tid >= off ? tot[tid - off] : 0u;
      __syncthreads();
      tot[tid] += t;
      __syncthreads();
    }
    dbase[tid] = (tid ? tot[tid - 1] : 0u) + hist[(long long)tid * nblk + blockIdx.x];
  }
  for (int w = 0; w < SORT_WARPS; ++w) wcnt[w][tid] = 0;
  __syncthreads();
  const long long seg = (long long)blockIdx.x * SORT_TILE + (long long)warp * SORT_SEG;
  const unsigned lt = (1u << lane) - 1u;
  // count this warp's segment
  for (int c = 0; c < SORT_SEG; c += 32) {
    long long q = seg + c + lane;
    bool ok = q < n;
    unsigned act = __ballot_sync(0xffffffffu, ok);
    if (!act) break;
    if (ok) {
      uint32_t d = (kin[q] >> shift) & 255u;
      unsigned m = __match_any_sync(act, d);
      if ((m & lt) == 0) wcnt[warp][d] += __popc(m);
    }
    __syncwarp();
  }
  __syncthreads();
  // per-warp starting rank of each digit
  {
    uint32_t run = dbase[tid];
    for (int w = 0; w < SORT_WARPS; ++w) {
      uint32_t c = wcnt[w][tid];
      wcnt[w][tid] = run;
      run += c;
    }
  }
  __syncthreads();
  for (int c = 0; c < SORT_SEG; c += 32) {
    long long q = seg + c + lane;
    bool ok = q < n;
    unsigned act = __ballot_sync(0xffffffffu, ok);
    if (!act) break;
    uint32_t k = 0, d = 0;
    unsigned m = 0;
    uint32_t pos = 0;
    if (ok) {
      k = kin[q];
      d = (k >> shift) & 255u;
      m = __match_any_sync(act, d);
      pos = wcnt[warp][d] + __popc(m & lt);
    }
    __syncwarp();
    if (ok) {
      kout[pos] = k;
      vout[pos] = vin ? vin[q] : (uint32_t)q;
      if ((m & lt) == 0) wcnt[warp][d] += __popc(m);
    }
    __syncwarp();
  }
}

// First sorted position of each key k in [0, nkeys]: lower bound in the sorted keys.
__global__ void k_cell_starts(const uint32_t* __restrict__ skey, long long n, long long nkeys,
                              int* __restrict__ start) {
  long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (k > nkeys) return;
  long long lo = 0, hi = n;
  while (lo < hi) {
    long long mid = (lo + hi) >> 1;
    if ((long long)skey[mid] < k) lo = mid + 1; else hi = mid;
  }
  start[k] = (int)lo;
}

// Permute the parcel arrays by the sorted order.
template <class T>
struct PArrays {
  T* a[8];        // x y z u v w d omega
  int* pid;
};

template <class T>
__global__ void k_gather(PArrays<T> src, PArrays<T> dst, const uint32_t* __restrict__ perm,
                         long long np) {
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= np) return;
  uint32_t s = perm[q];
#pragma unroll
  for (int f = 0; f < 8; ++f) dst.a[f][q] = src.a[f][s];
  if (src.pid) dst.pid[q] = src.pid[s];
}

// ------------------------------------------------------------ brick CTA --

template <class T> struct Chunk;                          // parcels per CTA chunk
template <> struct Chunk<float> { static constexpr int n = 1024; };
template <> struct Chunk<double> { static constexpr int n = 384; };

// Shared-memory layout of the brick kernels.
template <class T>
struct BrickSmem {
  static constexpr int W = Words<T>::n;
  static constexpr int NC = Chunk<T>::n;
  // node fields tile: 5 fields (+3 grad p) x TNODES
  static constexpr size_t fld_bytes = sizeof(T) * 8 * TNODES;
  // fixed-point tile: NQ x W x TNODES words
  static constexpr size_t acc_bytes = sizeof(u64) * NQ * W * TNODES;
  // records: f, u[3], xi_old[3], V, xi_new[3] (11 T) + old and new cell (2 int)
  static constexpr size_t rec_bytes = NC * (11 * sizeof(T) + 2 * sizeof(int));
  static constexpr size_t bytes = fld_bytes + acc_bytes + rec_bytes;
};

// Adds the fixed-point contributions of one parcel (values q at the 8 corners of cell
// (i,j,k) with in-cell coordinates xi) to the shared tile where the node is inside the
// brick tile, else to the global accumulators. Used for parcels outside their sorted cell.
template <class T, int NV>
__device__ void scatter_parcel(const KParams<T>& p, u64* tile, int bi0, int bj0, int bk0, int i,
                               int j, int k, const T (&xi)[3], const T (&vals)[NV], int q0) {
  constexpr int W = Words<T>::n;
  T w[3][2];
  for (int a = 0; a < 3; ++a) { w[a][0] = T(1) - xi[a]; w[a][1] = xi[a]; }
  for (int c = 0; c < 2; ++c)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        T Wq = (w[0][a] * w[1][b]) * w[2][c];
        int ti = i + a - bi0, tj = j + b - bj0, tk = k + c - bk0;
        bool in_tile = ti >= 0 && ti < TX && tj >= 0 && tj < TY && tk >= 0 && tk < TZ;
        long long gn = node_id(p, i + a, j + b, k + c);
        int tn = ti + TX * (tj + TY * tk);
        for (int v = 0; v < NV; ++v) {
          int q = q0 + v;
          u64 fx[W];
          to_fixed(vals[v] * Wq, q == 0 ? p.mV : p.mA, fx, p.errs);
          if (in_tile)
            acc_add(tile + (q * W) * TNODES + tn, TNODES, fx);
          else
            acc_add(p.acc + (long long)(q * W) * p.nnode + gn, p.nnode, fx);
        }
      }
}

// Deterministic block reduction of three per-thread values in T, in thread order.
template <class T>
__device__ void block_sum3(T a, T b, T c, T* sm, double* out) {
  const int t = threadIdx.x;
  sm[t] = a; sm[BCELLS + t] = b; sm[2 * BCELLS + t] = c;
  __syncthreads();
  for (int off = BCELLS / 2; off > 0; off >>= 1) {
    if (t < off) {
      sm[t] += sm[t + off];
      sm[BCELLS + t] += sm[BCELLS + t + off];
      sm[2 * BCELLS + t] += sm[2 * BCELLS + t + off];
    }
    __syncthreads();
  }
  if (t == 0) { out[0] = (double)sm[0]; out[1] = (double)sm[BCELLS]; out[2] = (double)sm[2 * BCELLS]; }
}

// The brick kernel. MODE 0: deposit the solids volume of the current positions.
// MODE 1: one full step for the parcels of the brick (interp, drag, drag sums, objectives,
// push, walls, re-bin) with the solids volume of the new positions deposited for the next
// step. src/dst may be the same arrays; if not, the read-only arrays are copied too.
template <class T, int MODE>
__global__ void __launch_bounds__(BCELLS, 2)
k_brick(KParams<T> p, PArrays<T> src, PArrays<T> dst, int* __restrict__ cell_out,
        double* __restrict__ obj_part) {
  constexpr int W = Words<T>::n;
  constexpr int NC = Chunk<T>::n;
  extern __shared__ __align__(16) unsigned char smem[];
  T* sf = reinterpret_cast<T*>(smem);                                        // [8][TNODES]
  u64* tile = reinterpret_cast<u64*>(smem + BrickSmem<T>::fld_bytes);       // [NQ*W][TNODES]
  unsigned char* recb = smem + BrickSmem<T>::fld_bytes + BrickSmem<T>::acc_bytes;
  T* rf = reinterpret_cast<T*>(recb);            // f
  T* ru = rf + NC;                               // u_old [3][NC]
  T* rxo = ru + 3 * NC;                          // xi_old [3][NC]
  T* rV = rxo + 3 * NC;                          // V
  T* rxn = rV + NC;                              // xi_new [3][NC]
  int* rco = reinterpret_cast<int*>(rxn + 3 * NC);
  int* rcn = rco + NC;

  const int tid = threadIdx.x;
  const long long b = blockIdx.x;
  const int bi = (int)(b % p.nbx), bj = (int)((b / p.nbx) % p.nby), bk = (int)(b / ((long long)p.nbx * p.nby));
  const int bi0 = bi * BX, bj0 = bj * BY, bk0 = bk * BZ;
  const long long kbase = b * BCELLS;
  const int pstart = p.cstart[kbase], pend = p.cstart[kbase + BCELLS];

  if (pstart == pend) {
    if (MODE == 1 && tid == 0) { obj_part[3 * b] = 0; obj_part[3 * b + 1] = 0; obj_part[3 * b + 2] = 0; }
    return;
  }

  // this thread's cell in the brick
  const int li = tid % BX, lj = (tid / BX) % BY, lk = tid / (BX * BY);
  const int gi = bi0 + li, gj = bj0 + lj, gk = bk0 + lk;
  const bool cell_ok = gi < p.nx && gj < p.ny && gk < p.nz;
  const int mycell = cell_ok ? cell_id(p, gi, gj, gk) : -1;
  const int cs = p.cstart[kbase + tid], ce = p.cstart[kbase + tid + 1];
  const int tbase = li + TX * (lj + TY * lk);     // tile node of corner (0,0,0)

  // zero the accumulator tile; stage the node-field tile (MODE 1)
  for (int e = tid; e < NQ * W * TNODES; e += BCELLS) tile[e] = 0;
  if (MODE == 1) {
    const int nf = p.has_gp ? 8 : 5;
    for (int e = tid; e < nf * TNODES; e += BCELLS) {
      int f = e / TNODES, tn = e % TNODES;
      int ti = tn % TX, tj = (tn / TX) % TY, tk = tn / (TX * TY);
      int i = bi0 + ti, j = bj0 + tj, k = bk0 + tk;
      T v = 0;
      if (i <= p.nx && j <= p.ny && k <= p.nz) {
        long long n = node_id(p, i, j, k);
        v = f < 5 ? p.fld[f][n] : p.gpf[f - 5][n];
      }
      sf[e] = v;
    }
  }
  __syncthreads();

  const T* tf[5] = {sf, sf + TNODES, sf + 2 * TNODES, sf + 3 * TNODES, sf + 4 * TNODES};
  const T* tg[3] = {sf + 5 * TNODES, sf + 6 * TNODES, sf + 7 * TNODES};
  const long long sxg = 1, syg = p.nx + 1, szg = (long long)(p.nx + 1) * (p.ny + 1);
  T o_dp = 0, o_hn = 0, o_vs = 0;

  for (int c0 = pstart; c0 < pend; c0 += NC) {
    const int cn = min(NC, pend - c0);
    // ---- phase A: one parcel per thread
    for (int r = tid; r < cn; r += BCELLS) {
      const long long q = (long long)c0 + r;
      T x = src.a[0][q], y = src.a[1][q], z = src.a[2][q];
      T d = src.a[6][q], om = src.a[7][q];
      T V = om * (d * d * d) * p.vcoef;
      Cell3<T> c;
      bin3(p, x, y, z, c);
      const int oldcell = cell_id(p, c.i, c.j, c.k);
      if (MODE == 0) {
        rV[r] = V;
        rxn[r] = c.xi[0]; rxn[NC + r] = c.xi[1]; rxn[2 * NC + r] = c.xi[2];
        rcn[r] = oldcell;
        continue;
      }
      T u = src.a[3][q], v = src.a[4][q], w = src.a[5][q];
      // interpolation: from the tile if the cell is in this brick, else from global memory
      Interp<T> I;
      int ti = c.i - bi0, tj = c.j - bj0, tk = c.k - bk0;
      if (ti >= 0 && ti < BX && tj >= 0 && tj < BY && tk >= 0 && tk < BZ) {
        interp8(p, tf, p.has_gp ? tg : nullptr, ti + TX * (tj + TY * tk), 1, TX, TX * TY, c.xi, I);
      } else {
        const T* gf[5] = {p.fld[0], p.fld[1], p.fld[2], p.fld[3], p.fld[4]};
        interp8(p, gf, p.has_gp ? p.gpf : nullptr, node_id(p, c.i, c.j, c.k), sxg, syg, szg, c.xi, I);
      }
      T up[3] = {u, v, w};
      T s[3] = {I.ug[0] - u, I.ug[1] - v, I.ug[2] - w};
      T D = wen_yu(p, d, I.es, s);
      T f = p.rho_p * V * D;
      o_dp += f * s[2];
      o_hn += V * z;
      o_vs += V;
      rf[r] = f;
      ru[r] = u; ru[NC + r] = v; ru[2 * NC + r] = w;
      rxo[r] = c.xi[0]; rxo[NC + r] = c.xi[1]; rxo[2 * NC + r] = c.xi[2];
      rV[r] = V;
      rco[r] = oldcell;
      // semi-implicit push (Eq. 4 / (eps_P rho_P), drag implicit), Eq. 3, specular walls
      T pos[3] = {x, y, z};
      const T den = T(1) + p.dt * D;
      bool bad = false;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        T acc = D * I.ug[a] + p.g[a] - I.gp[a] / p.rho_p;
        if (I.es > T(1e-12)) acc = acc - I.gt[a] / (I.es * p.rho_p);
        T un = (up[a] + p.dt * acc) / den;
        T xn = pos[a] + p.dt * un;
        if (xn < T(0)) { xn = -xn; un = -p.e_wall * un; }
        else if (xn > p.L[a]) { xn = T(2) * p.L[a] - xn; un = -p.e_wall * un; }
        if (!(xn >= T(0) && xn <= p.L[a]) || !isfinite(un)) bad = true;
        pos[a] = xn;
        up[a] = un;
      }
      if (bad) atomicOr(p.errs, ERR_DOMAIN);
      Cell3<T> cnw;
      bin3(p, pos[0], pos[1], pos[2], cnw);
      const int newcell = cell_id(p, cnw.i, cnw.j, cnw.k);
      rxn[r] = cnw.xi[0]; rxn[NC + r] = cnw.xi[1]; rxn[2 * NC + r] = cnw.xi[2];
      rcn[r] = newcell;
      dst.a[0][q] = pos[0]; dst.a[1][q] = pos[1]; dst.a[2][q] = pos[2];
      dst.a[3][q] = up[0]; dst.a[4][q] = up[1]; dst.a[5][q] = up[2];
      if (src.a[0] != dst.a[0]) {
        dst.a[6][q] = d; dst.a[7][q] = om;
        if (src.pid) dst.pid[q] = src.pid[q];
      }
      if (cell_out) cell_out[q] = newcell;
    }
    __syncthreads();
    // ---- phase B: one thread per cell sums the records of its sorted range
    const int r0 = max(cs, c0) - c0, r1 = min(ce, c0 + cn) - c0;
    if (r0 < r1) {
      T aV[8], aA[8], aB[3][8];
#pragma unroll
      for (int q = 0; q < 8; ++q) { aV[q] = 0; aA[q] = 0; aB[0][q] = 0; aB[1][q] = 0; aB[2][q] = 0; }
      for (int r = r0; r < r1; ++r) {
        if (MODE == 1) {
          T xo[3] = {rxo[r], rxo[NC + r], rxo[2 * NC + r]};
          T fr = rf[r];
          T fu[3] = {fr * ru[r], fr * ru[NC + r], fr * ru[2 * NC + r]};
          int co = rco[r];
          if (co == mycell) {
            T w[3][2];
            for (int a = 0; a < 3; ++a) { w[a][0] = T(1) - xo[a]; w[a][1] = xo[a]; }
#pragma unroll
            for (int q = 0; q < 8; ++q) {
              T Wq = (w[0][q & 1] * w[1][(q >> 1) & 1]) * w[2][q >> 2];
              aA[q] += fr * Wq;
              aB[0][q] += fu[0] * Wq;
              aB[1][q] += fu[1] * Wq;
              aB[2][q] += fu[2] * Wq;
            }
          } else {
            int i, j, k;
            decode_cell(p, co, i, j, k);
            T vals[4] = {fr, fu[0], fu[1], fu[2]};
            scatter_parcel<T, 4>(p, tile, bi0, bj0, bk0, i, j, k, xo, vals, 1);
          }
        }
        T xn[3] = {rxn[r], rxn[NC + r], rxn[2 * NC + r]};
        T Vr = rV[r];
        int cnr = rcn[r];
        if (cnr == mycell) {
          T w[3][2];
          for (int a = 0; a < 3; ++a) { w[a][0] = T(1) - xn[a]; w[a][1] = xn[a]; }
#pragma unroll
          for (int q = 0; q < 8; ++q) aV[q] += Vr * ((w[0][q & 1] * w[1][(q >> 1) & 1]) * w[2][q >> 2]);
        } else {
          int i, j, k;
          decode_cell(p, cnr, i, j, k);
          T vals[1] = {Vr};
          scatter_parcel<T, 1>(p, tile, bi0, bj0, bk0, i, j, k, xn, vals, 0);
        }
      }
      // per-cell sums -> fixed point -> shared tile (corner order: no two threads of an
      // instruction touch the same node)
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int tn = tbase + (q & 1) + TX * (((q >> 1) & 1) + TY * (q >> 2));
        u64 fx[W];
        to_fixed(aV[q], p.mV, fx, p.errs);
        acc_add(tile + 0 * W * TNODES + tn, TNODES, fx);
        if (MODE == 1) {
          to_fixed(aA[q], p.mA, fx, p.errs);
          acc_add(tile + 1 * W * TNODES + tn, TNODES, fx);
          for (int a = 0; a < 3; ++a) {
            to_fixed(aB[a][q], p.mA, fx, p.errs);
            acc_add(tile + (2 + a) * W * TNODES + tn, TNODES, fx);
          }
        }
      }
    }
    __syncthreads();
  }
  // ---- flush the tile to the global accumulators
  const int nq = MODE == 1 ? NQ : 1;
  for (int e = tid; e < nq * TNODES; e += BCELLS) {
    int q = e / TNODES, tn = e % TNODES;
    int ti = tn % TX, tj = (tn / TX) % TY, tk = tn / (TX * TY);
    int i = bi0 + ti, j = bj0 + tj, k = bk0 + tk;
    if (i > p.nx || j > p.ny || k > p.nz) continue;
    u64 fx[W];
    for (int w = 0; w < W; ++w) fx[w] = tile[(q * W + w) * TNODES + tn];
    acc_add(p.acc + (long long)(q * W) * p.nnode + node_id(p, i, j, k), p.nnode, fx);
  }
  if (MODE == 1) {
    __syncthreads();
    block_sum3(o_dp, o_hn, o_vs, reinterpret_cast<T*>(recb), obj_part + 3 * b);
  }
}

// a5: node fields from the deposited volume. Reads and clears the Vs accumulator and
// clears the drag-sum accumulators for the coming push. vs_out (nullable) receives Vs.
template <class T>
__global__ void k_finalize(KParams<T> p, double* __restrict__ vs_out) {
  constexpr int W = Words<T>::n;
  long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= p.nnode) return;
  int i = (int)(n % (p.nx + 1));
  long long r = n / (p.nx + 1);
  int j = (int)(r % (p.ny + 1));
  int k = (int)(r / (p.ny + 1));
  u64 fx[W];
  for (int w = 0; w < W; ++w) { fx[w] = p.acc[(long long)w * p.nnode + n]; }
  if (W == 1 && (long long)fx[0] >= (1ll << 62)) atomicOr(p.errs, ERR_RANGE);
  double Vs = from_fixed(fx, p.inv_mV);
  for (int e = 0; e < NQ * W; ++e) p.acc[(long long)e * p.nnode + n] = 0;
  if (vs_out) vs_out[n] = Vs;
  double vn = p.vcell;
  if (i == 0 || i == p.nx) vn *= 0.5;
  if (j == 0 || j == p.ny) vn *= 0.5;
  if (k == 0 || k == p.nz) vn *= 0.5;
  T es = (T)(Vs / vn);
  T eg = T(1) - es;
  T egc = tmax(eg, p.eg_min);
  T U0 = p.U[0] ? p.U[0][n] : T(0);
  T U1 = p.U[1] ? p.U[1][n] : T(0);
  T U2 = (p.U[2] ? p.U[2][n] : T(0)) + p.u_in;
  p.fld[0][n] = es;
  p.fld[1][n] = U0 / egc;
  p.fld[2][n] = U1 / egc;
  p.fld[3][n] = U2 / egc;
  T den = tmax(p.eps_cp - es, p.alpha * (T(1) - es));
  p.fld[4][n] = p.Ps * tpow(es, p.beta) / den;
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
    for (int w = 0; w < W; ++w) fx[w] = p.acc[(long long)(q * W + w) * p.nnode + n];
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
  const T* gf[5] = {p.fld[0], p.fld[1], p.fld[2], p.fld[3], p.fld[4]};
  Interp<T> I;
  interp8(p, gf, p.has_gp ? p.gpf : nullptr, node_id(p, c.i, c.j, c.k), 1, p.nx + 1,
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

// a10: deterministic reduction of the per-brick objective partials into (dP, H).
__global__ void k_obj_reduce(const double* __restrict__ part, long long nb, double area,
                             double* __restrict__ obj) {
  __shared__ double s[3][1024];
  const int t = threadIdx.x;
  double a = 0, b = 0, c = 0;
  for (long long i = t; i < nb; i += blockDim.x) {
    a += part[3 * i]; b += part[3 * i + 1]; c += part[3 * i + 2];
  }
  s[0][t] = a; s[1][t] = b; s[2][t] = c;
  __syncthreads();
  for (int off = blockDim.x / 2; off > 0; off >>= 1) {
    if (t < off) { s[0][t] += s[0][t + off]; s[1][t] += s[1][t + off]; s[2][t] += s[2][t + off]; }
    __syncthreads();
  }
  if (t == 0) {
    obj[0] = s[0][0] / area;
    obj[1] = s[2][0] > 0 ? 2.0 * s[1][0] / s[2][0] : 0.0;
  }
}

}  // namespace mppic
