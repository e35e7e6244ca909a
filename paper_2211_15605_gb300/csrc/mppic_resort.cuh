// Local re-sort: the stable sort of the parcels by brick-major cell key (the sort by cell
// that precedes the deposit, this library's own step) when the parcels are already laid out
// by the previous sort, so that each brick's parcels occupy the range of sorted positions
// the cell starts give it. Between two sorts a parcel moves a fraction of a cell per step,
// so almost every parcel's new brick is its range's brick or one of that brick's 26
// neighbours. The sort then needs no global digit passes:
//
//   k_rs_hist     per source brick (its range of the current layout): how many of its
//                 parcels go to each of the 27 neighbour bricks (slots), per warp segment
//                 and in total; parcels going further ("far") are counted per destination;
//   k_rs_count    per destination brick: its parcel count (its neighbours' slot counts
//                 towards it, plus its far count), and the sum over each CTA's bricks;
//   k_rs_offsets  per destination brick: its first position (a scan over bricks), and
//                 where the run from each neighbour starts, the neighbours taken in
//                 ascending brick index (= ascending source position);
//   k_rs_scatter  per source brick: each parcel's (source index, cell byte) into its
//                 destination's bucket, stable within each run; far parcels at the end of
//                 the bucket, in any order;
//   k_rs_build    per destination brick: if far parcels arrived, sort the bucket by source
//                 index (LSD passes in the CTA); then a stable counting pass by cell gives
//                 the cell starts and the permutation, and level_layout moves the parcels
//                 (or, inside a step call, writes only the permutation, which the next
//                 step kernel reads its parcels through).
//
// The result is exactly the stable sort of the current order by key, whatever that order
// is (a bucket in source order, then a stable pass by cell); locality only decides the
// cost. All counts are integers and no result depends on the order of atomic operations.

namespace mppic {

constexpr int NSLOT = 27;          // neighbour slots (dx+1) + 3 (dy+1) + 9 (dz+1)
constexpr int RS_THREADS = 256;
constexpr int RS_CAP = 4096;       // bucket size up to which the brick sorts in shared memory

// Brick geometry: {first brick of the bed, bricks along x, y, z}, one entry per brick.
__device__ __forceinline__ void rs_coords(int4 g, long long b, int& x, int& y, int& z) {
  const int l = (int)(b - g.x);
  x = l % g.y;
  const int r = l / g.y;
  y = r % g.z;
  z = r / g.z;
}

// Slot of destination brick B seen from source brick (bx, by, bz) of bed geometry g, or -1
// if B is in another bed or more than one brick away along some axis.
__device__ __forceinline__ int rs_slot(int4 g, int bx, int by, int bz, long long B) {
  const long long l = B - g.x;
  if (l < 0 || l >= (long long)g.y * g.z * g.w) return -1;
  int x, y, z;
  rs_coords(g, B, x, y, z);
  const int dx = x - bx, dy = y - by, dz = z - bz;
  if (dx < -1 || dx > 1 || dy < -1 || dy > 1 || dz < -1 || dz > 1) return -1;
  return (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
}

// Source brick of destination B's slot s, or -1 if it lies outside B's bed.
__device__ __forceinline__ long long rs_source(int4 g, int x, int y, int z, int s) {
  const int sx = x - (s % 3 - 1), sy = y - ((s / 3) % 3 - 1), sz = z - (s / 9 - 1);
  if (sx < 0 || sx >= g.y || sy < 0 || sy >= g.z || sz < 0 || sz >= g.w) return -1;
  return (long long)g.x + sx + (long long)g.y * (sy + (long long)g.z * sz);
}

constexpr int RS_U = 4;           // keys in flight per thread in the per-brick passes
constexpr int RS_NW = RS_THREADS / 32;

// Exclusive scan of one int per thread over the CTA (RS_THREADS threads); *total gets the sum.
__device__ __forceinline__ int rs_block_scan(int v, int* wsum, int* total) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  int inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(FULL, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  int pre = 0, all = 0;
  for (int w = 0; w < RS_NW; ++w) {
    if (w < warp) pre += wsum[w];
    all += wsum[w];
  }
  __syncthreads();                               // wsum may be reused at once
  if (total) *total = all;
  return pre + inc - v;
}

// Warp w of a brick's CTA takes parcels [lo, hi) of the brick's n (a contiguous segment,
// a multiple of 32 long), in both the count and the scatter pass.
__device__ __forceinline__ void rs_segment(int n, int warp, int& lo, int& hi) {
  const int seg = ((n + RS_NW - 1) / RS_NW + 31) & ~31;
  lo = min(n, warp * seg);
  hi = min(n, warp * seg + seg);
}

// Per source brick: each warp counts its segment's parcels per slot (wcnt, [nbricks][NW][27]);
// cnt gets the brick's totals. Far parcels are counted per destination brick.
__global__ void __launch_bounds__(RS_THREADS)
k_rs_hist(const uint32_t* __restrict__ key, const int* __restrict__ cstart,
          const int4* __restrict__ bgeo, long long nbricks, uint32_t* __restrict__ cnt,
          uint32_t* __restrict__ wcnt, int* __restrict__ far_cnt) {
  __shared__ int s_w[RS_NW][32];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const unsigned below = (1u << lane) - 1u;
  for (long long b = blockIdx.x; b < nbricks; b += gridDim.x) {
    const int s0 = cstart[b * BCELLS], s1 = cstart[(b + 1) * BCELLS];
    if (s0 == s1) {                              // uniform over the CTA
      if (t < NSLOT) cnt[b * NSLOT + t] = 0u;
      continue;
    }
    const int4 g = bgeo[b];
    int bx, by, bz;
    rs_coords(g, b, bx, by, bz);
    int lo, hi;
    rs_segment(s1 - s0, warp, lo, hi);
    lo += s0;
    hi += s0;
    s_w[warp][lane] = 0;
    __syncwarp();
    for (int i0 = lo; i0 < hi; i0 += RS_U * 32) {
      uint32_t kk[RS_U];
#pragma unroll
      for (int j = 0; j < RS_U; ++j) {
        const int q = i0 + j * 32 + lane;
        kk[j] = q < hi ? key[q] : 0u;
      }
#pragma unroll
      for (int j = 0; j < RS_U; ++j) {
        const bool ok = i0 + j * 32 + lane < hi;
        const uint32_t B = kk[j] / BCELLS;
        const bool own = !ok || B == (uint32_t)b;
        if (__all_sync(FULL, own)) {             // the common case: no lane left the brick
          const unsigned bl = __ballot_sync(FULL, ok);
          if (lane == 0) s_w[warp][13] += __popc(bl);
          __syncwarp();
          continue;
        }
        const int slot = !ok ? -2 : (B == (uint32_t)b ? 13 : rs_slot(g, bx, by, bz, B));
        const unsigned m = match_bits<5>((unsigned)(slot + 2));
        if (slot >= 0) {
          if ((m & below) == 0) s_w[warp][slot] += __popc(m);
        } else if (slot == -1) {
          atomicAdd(&far_cnt[B], 1);
        }
        __syncwarp();
      }
    }
    if (lane < NSLOT) wcnt[(b * RS_NW + warp) * NSLOT + lane] = (uint32_t)s_w[warp][lane];
    __syncthreads();
    if (t < NSLOT) {
      uint32_t c = 0;
      for (int w = 0; w < RS_NW; ++w) c += (uint32_t)s_w[w][t];
      cnt[b * NSLOT + t] = c;
    }
    __syncthreads();                             // s_w is reset for the next brick
  }
}

// Bucket size of each destination brick, and the sum over each CTA's bricks.
__global__ void __launch_bounds__(RS_THREADS)
k_rs_count(const uint32_t* __restrict__ cnt, const int* __restrict__ far_cnt,
           const int4* __restrict__ bgeo, long long nbricks, int* __restrict__ bcount,
           int* __restrict__ part) {
  __shared__ int wsum[RS_NW];
  const long long B = blockIdx.x * (long long)RS_THREADS + threadIdx.x;
  int n = 0;
  if (B < nbricks) {
    const int4 g = bgeo[B];
    int x, y, z;
    rs_coords(g, B, x, y, z);
    n = far_cnt[B];
    for (int s = 0; s < NSLOT; ++s) {
      const long long b = rs_source(g, x, y, z, s);
      if (b >= 0) n += (int)cnt[b * NSLOT + s];
    }
    bcount[B] = n;
  }
  int total;
  rs_block_scan(n, wsum, &total);
  if (threadIdx.x == 0) part[blockIdx.x] = total;
}

// Bucket starts (the sums of the earlier CTAs' bricks, then a scan within the CTA) and the
// run offsets of each destination brick. Source b = B - d has index B - (dx + nbx (dy +
// nby dz)); over the valid neighbours, descending slot order is ascending source index.
__global__ void __launch_bounds__(RS_THREADS)
k_rs_offsets(const uint32_t* __restrict__ cnt, const int* __restrict__ bcount,
             const int* __restrict__ part, const int4* __restrict__ bgeo, long long nbricks,
             int* __restrict__ bstart, uint32_t* __restrict__ off, int* __restrict__ far_next,
             int* __restrict__ cstart_end) {
  __shared__ int wsum[RS_NW];
  const int t = threadIdx.x;
  int pre = 0;
  for (int i = t; i < (int)blockIdx.x; i += RS_THREADS) pre += part[i];
  int before;
  rs_block_scan(pre, wsum, &before);
  const long long B = blockIdx.x * (long long)RS_THREADS + t;
  const int c = B < nbricks ? bcount[B] : 0;
  const int e = rs_block_scan(c, wsum, nullptr);
  if (B >= nbricks) return;
  int run = before + e;
  bstart[B] = run;
  const int4 g = bgeo[B];
  int x, y, z;
  rs_coords(g, B, x, y, z);
  for (int s = NSLOT - 1; s >= 0; --s) {
    const long long b = rs_source(g, x, y, z, s);
    if (b < 0) continue;
    off[b * NSLOT + s] = (uint32_t)run;
    run += (int)cnt[b * NSLOT + s];
  }
  far_next[B] = run;                             // the far parcels follow the runs
  if (B == nbricks - 1) *cstart_end = before + e + c;
}

// Per source brick: warp w places its segment's parcels in order, from its first position
// in each run (the run offset plus the counts of the earlier warps' segments), so each run
// keeps source order.
__global__ void __launch_bounds__(RS_THREADS)
k_rs_scatter(const uint32_t* __restrict__ key, const int* __restrict__ cstart,
             const int4* __restrict__ bgeo, long long nbricks, const uint32_t* __restrict__ off,
             const uint32_t* __restrict__ wcnt, int* __restrict__ far_next,
             uint32_t* __restrict__ bsrc, uint8_t* __restrict__ bcell) {
  __shared__ int s_w[RS_NW][32];                 // per warp and slot: next position
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const unsigned below = (1u << lane) - 1u;
  for (long long b = blockIdx.x; b < nbricks; b += gridDim.x) {
    const int s0 = cstart[b * BCELLS], s1 = cstart[(b + 1) * BCELLS];
    if (s0 == s1) continue;                      // uniform over the CTA
    const int4 g = bgeo[b];
    int bx, by, bz;
    rs_coords(g, b, bx, by, bz);
    if (t < NSLOT) {
      int r = (int)off[b * NSLOT + t];
      for (int w = 0; w < RS_NW; ++w) {
        s_w[w][t] = r;
        r += (int)wcnt[(b * RS_NW + w) * NSLOT + t];
      }
    }
    __syncthreads();
    int lo, hi;
    rs_segment(s1 - s0, warp, lo, hi);
    lo += s0;
    hi += s0;
    for (int i0 = lo; i0 < hi; i0 += RS_U * 32) {
      uint32_t kk[RS_U];
#pragma unroll
      for (int j = 0; j < RS_U; ++j) {
        const int q = i0 + j * 32 + lane;
        kk[j] = q < hi ? key[q] : 0u;
      }
#pragma unroll
      for (int j = 0; j < RS_U; ++j) {
        const int q = i0 + j * 32 + lane;
        const bool ok = q < hi;
        const uint32_t B = kk[j] / BCELLS;
        const bool own = !ok || B == (uint32_t)b;
        if (__all_sync(FULL, own)) {             // the common case: the warp's run is contiguous
          const unsigned bl = __ballot_sync(FULL, ok);
          const int base = s_w[warp][13];
          if (ok) {
            const int pos = base + __popc(bl & below);
            bsrc[pos] = (uint32_t)q;
            bcell[pos] = (uint8_t)(kk[j] % BCELLS);
          }
          __syncwarp();
          if (lane == 0) s_w[warp][13] = base + __popc(bl);
          __syncwarp();
          continue;
        }
        const int slot = !ok ? -2 : (B == (uint32_t)b ? 13 : rs_slot(g, bx, by, bz, B));
        const unsigned m = match_bits<5>((unsigned)(slot + 2));
        if (slot >= -1) {
          const int pos = slot >= 0 ? s_w[warp][slot] + __popc(m & below) : atomicAdd(&far_next[B], 1);
          bsrc[pos] = (uint32_t)q;
          bcell[pos] = (uint8_t)(kk[j] % BCELLS);
        }
        __syncwarp();
        if (slot >= 0 && (m & below) == 0) s_w[warp][slot] += __popc(m);
        __syncwarp();
      }
    }
    __syncthreads();                             // s_w is rewritten for the next brick
  }
}

// One stable counting pass over n (source index, cell byte) pairs by a 256-way digit, by
// the whole CTA. Warp w takes a contiguous segment: it counts its pairs per digit; a prefix
// over digits and warps gives each warp's first position per digit; the warp then places
// its pairs in order, ranked within each 32 by match_bits.
struct RsPass {
  int w[RS_NW][256];             // per warp and digit: count, then next position
  int start[256];                // digit starts
  int wsum[RS_NW];
};

struct DigitOfSource {
  uint32_t base;
  int shift;
  static constexpr bool cell_only = false;
  __device__ int operator()(uint32_t s, uint8_t) const { return (int)(((s - base) >> shift) & 255u); }
};
struct DigitOfCell {
  static constexpr bool cell_only = true;
  __device__ int operator()(uint32_t, uint8_t c) const { return (int)c; }
};

template <class Dig>
__device__ void rs_pass(const uint32_t* in_s, const uint8_t* in_c, uint32_t* out_s,
                        uint8_t* out_c, int n, Dig dig, RsPass& ps) {
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const unsigned below = (1u << lane) - 1u;
  int lo, hi;
  rs_segment(n, warp, lo, hi);
  for (int d = lane; d < 256; d += 32) ps.w[warp][d] = 0;
  __syncwarp();
  for (int i0 = lo; i0 < hi; i0 += RS_U * 32) {  // count (order does not matter)
    int dd[RS_U];
#pragma unroll
    for (int j = 0; j < RS_U; ++j) {
      const int i = i0 + j * 32 + lane;
      dd[j] = -1;
      if (i < hi) dd[j] = Dig::cell_only ? dig(0u, in_c[i]) : dig(in_s[i], in_c[i]);
    }
#pragma unroll
    for (int j = 0; j < RS_U; ++j)               // integer counts: their order does not matter
      if (dd[j] >= 0) atomicAdd(&ps.w[warp][dd[j]], 1);
  }
  __syncthreads();
  {                                              // digit t: warps' offsets, then digit start
    int tot = 0;
#pragma unroll
    for (int w = 0; w < RS_NW; ++w) {
      const int h = ps.w[w][t];
      ps.w[w][t] = tot;
      tot += h;
    }
    const int st = rs_block_scan(tot, ps.wsum, nullptr);
    ps.start[t] = st;
#pragma unroll
    for (int w = 0; w < RS_NW; ++w) ps.w[w][t] += st;
  }
  __syncthreads();
  for (int i0 = lo; i0 < hi; i0 += RS_U * 32) {  // place, in order
    uint32_t ss[RS_U];
    uint8_t cc[RS_U];
#pragma unroll
    for (int j = 0; j < RS_U; ++j) {
      const int i = i0 + j * 32 + lane;
      ss[j] = i < hi ? in_s[i] : 0u;
      cc[j] = i < hi ? in_c[i] : (uint8_t)0;
    }
#pragma unroll
    for (int j = 0; j < RS_U; ++j) {
      const bool ok = i0 + j * 32 + lane < hi;
      const int d = ok ? dig(ss[j], cc[j]) : 0;
      // the lanes' digits are usually distinct (consecutive pairs of a level layout are
      // different cells): then each lane takes the digit's next position alone
      const unsigned m = match_bits<8>((unsigned)d) & __ballot_sync(FULL, ok);
      if (ok) {
        const int pos = ps.w[warp][d] + __popc(m & below);
        out_s[pos] = ss[j];
        if (out_c) out_c[pos] = cc[j];
      }
      __syncwarp();
      if (ok && (m & below) == 0) ps.w[warp][d] += __popc(m);
      __syncwarp();
    }
  }
  __syncthreads();
}

template <class T> struct RsOccupancy;
template <> struct RsOccupancy<float> { static constexpr int ctas = 4; };
template <> struct RsOccupancy<double> { static constexpr int ctas = 4; };

template <class T>
__global__ void __launch_bounds__(RS_THREADS, RsOccupancy<T>::ctas)
k_rs_build(PArrays<T> src, PArrays<T> dst, const int* __restrict__ bstart,
           const int* __restrict__ bcount, const int* __restrict__ far_cnt, uint32_t* bsrc,
           uint8_t* bcell, uint32_t* tsrc, uint8_t* tcell, int* __restrict__ cstart,
           uint8_t* __restrict__ cellmap, uint32_t* __restrict__ lperm) {
  __shared__ union {
    RsPass ps;
    LevelSmem ls;
  } u;
  __shared__ uint32_t s_perm[RS_CAP];
  __shared__ uint32_t s_src[RS_CAP];
  __shared__ uint8_t s_cell[RS_CAP];
  __shared__ int s_cs[BCELLS + 1];
  __shared__ uint32_t s_mn[RS_NW], s_mx[RS_NW];
  const long long B = blockIdx.x, k0 = B * BCELLS;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int bs = bstart[B], n = bcount[B];
  if (n == 0) {                                  // uniform: an empty brick
    cstart[k0 + t] = bs;
    if (t < CT) cellmap[k0 + t] = (uint8_t)(t + CT);   // the natural pair map
    return;
  }
  uint32_t* is = bsrc + bs;
  uint8_t* ic = bcell + bs;
  uint32_t* os = tsrc + bs;
  uint8_t* oc = tcell + bs;
  if (far_cnt[B] > 0) {          // far parcels sit unordered at the end: sort by source index
    uint32_t mn = 0xffffffffu, mx = 0u;
    for (int i = t; i < n; i += RS_THREADS) {
      const uint32_t v = is[i];
      mn = min(mn, v);
      mx = max(mx, v);
    }
    mn = __reduce_min_sync(FULL, mn);
    mx = __reduce_max_sync(FULL, mx);
    if (lane == 0) { s_mn[warp] = mn; s_mx[warp] = mx; }
    __syncthreads();
    mn = s_mn[0];
    mx = s_mx[0];
    for (int w = 1; w < RS_NW; ++w) { mn = min(mn, s_mn[w]); mx = max(mx, s_mx[w]); }
    const uint32_t span = mx - mn;
    const int passes = span ? (32 - __clz((int)span) + 7) / 8 : 0;
    for (int k = 0; k < passes; ++k) {
      rs_pass(is, ic, os, oc, n, DigitOfSource{mn, 8 * k}, u.ps);
      uint32_t* ts = is; is = os; os = ts;
      uint8_t* tc = ic; ic = oc; oc = tc;
    }
  }
  uint32_t* perm = os;                           // os: the buffer not holding the input
  if (n <= RS_CAP) {             // the whole bucket into shared memory, all loads in flight
    constexpr int PER = RS_CAP / RS_THREADS;
    uint32_t vs[PER];
    uint8_t vc[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int i = j * RS_THREADS + t;
      vs[j] = i < n ? is[i] : 0u;
      vc[j] = i < n ? ic[i] : (uint8_t)0;
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int i = j * RS_THREADS + t;
      if (i < n) {
        s_src[i] = vs[j];
        s_cell[i] = vc[j];
      }
    }
    __syncthreads();
    is = s_src;
    ic = s_cell;
    perm = s_perm;
  }
  rs_pass(is, ic, perm, nullptr, n, DigitOfCell{}, u.ps);
  const int cs = u.ps.start[t];
  __syncthreads();                               // u.ps is reused as u.ls
  s_cs[t] = cs;
  if (t == 0) s_cs[BCELLS] = n;
  cstart[k0 + t] = bs + cs;
  __syncthreads();
  level_layout<T>(src, dst, k0, bs, s_cs, perm, cellmap, u.ls, lperm);
}

}  // namespace mppic
