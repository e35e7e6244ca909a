// Sorting the parcels by brick-major cell key from an arbitrary order, before the deposit
// (the paper locates each parcel's cell with index arithmetic, Sec. 2.2.3; ordering the
// parcels by cell is this library's own step): a stable LSD radix sort of the keys
// with the parcel index as value, the first sorted position of each key, and the level
// layout of each brick's parcels that the cell kernel reads (level_layout, shared with the
// local re-sort in mppic_resort.cuh).

namespace mppic {

// The lanes of the warp whose v equals this lane's (what __match_any_sync(FULL, v) returns),
// from one ballot per bit of v, 0 <= v < 2^BITS. All 32 lanes must call it. Ballots run at
// full rate; a warp-wide match over up to 32 distinct values does not.
template <int BITS>
__device__ __forceinline__ unsigned match_bits(unsigned v) {
  unsigned m = 0xffffffffu;
#pragma unroll
  for (int i = 0; i < BITS; ++i) {
    const bool bit = (v >> i) & 1u;
    const unsigned bl = __ballot_sync(0xffffffffu, bit);
    m &= bit ? bl : ~bl;
  }
  return m;
}

// ------------------------------------------------------------ radix sort --
// Stable LSD radix sort of (key, value) by 8-bit digits: a per-tile digit histogram, a
// scan per digit across tiles, then a stable scatter in which each warp ranks its own
// contiguous segment with match_bits.

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

// Two forms of the stable scatter of one digit pass. Both rank each warp's segment with
// match_bits. k_sort_scatter_direct writes every key straight to its output
// position: best when a tile's keys mostly share a digit (the upper digits of nearly
// sorted keys). k_sort_scatter_reorder first places the tile in digit order in shared
// memory and writes it out in that order, so each digit's run lands on consecutive
// positions: best when a tile's keys spread over many digits (the lowest digit).
__global__ void __launch_bounds__(SORT_THREADS)
k_sort_scatter_direct(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
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
    const uint32_t d = ok ? (kin[q] >> shift) & 255u : 0u;
    const unsigned m = match_bits<8>(d) & act;
    if (ok && (m & lt) == 0) wcnt[warp][d] += __popc(m);
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
    const uint32_t k = ok ? kin[q] : 0u;
    const uint32_t d = (k >> shift) & 255u;
    const unsigned m = match_bits<8>(d) & act;
    uint32_t pos = 0;
    if (ok) pos = wcnt[warp][d] + __popc(m & lt);
    __syncwarp();
    if (ok) {
      kout[pos] = k;
      vout[pos] = vin ? vin[q] : (uint32_t)q;
      if ((m & lt) == 0) wcnt[warp][d] += __popc(m);
    }
    __syncwarp();
  }
}

__global__ void __launch_bounds__(SORT_THREADS)
k_sort_scatter_reorder(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin,
               uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, long long n, int shift,
               const uint32_t* __restrict__ hist, const uint32_t* __restrict__ totals, int nblk) {
  __shared__ uint32_t dbase[256];                // output start of each digit for this tile
  __shared__ uint32_t lbase[256];                // start of each digit in the tile's digit order
  __shared__ uint32_t wcnt[SORT_WARPS][256];
  __shared__ uint32_t sk[SORT_TILE], sv[SORT_TILE];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long tbase = (long long)blockIdx.x * SORT_TILE;
  const int tn = (int)(n - tbase < SORT_TILE ? n - tbase : SORT_TILE);
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
  const int seg = warp * SORT_SEG;
  const unsigned lt = (1u << lane) - 1u;
  // count this warp's segment
  for (int c = 0; c < SORT_SEG; c += 32) {
    const int r = seg + c + lane;
    const bool ok = r < tn;
    const unsigned act = __ballot_sync(0xffffffffu, ok);
    if (!act) break;
    const uint32_t d = ok ? (kin[tbase + r] >> shift) & 255u : 0u;
    const unsigned m = match_bits<8>(d) & act;
    if (ok && (m & lt) == 0) wcnt[warp][d] += __popc(m);
    __syncwarp();
  }
  __syncthreads();
  // per digit: each warp's offset within the digit, and the digit's start in the tile
  uint32_t cnt = 0;
  {
    uint32_t run = 0;
    for (int w = 0; w < SORT_WARPS; ++w) {
      const uint32_t c = wcnt[w][tid];
      wcnt[w][tid] = run;
      run += c;
    }
    cnt = run;
  }
  lbase[tid] = cnt;
  __syncthreads();
  for (int off = 1; off < 256; off <<= 1) {      // inclusive scan of the digit counts
    const uint32_t t = tid >= off ? lbase[tid - off] : 0u;
    __syncthreads();
    lbase[tid] += t;
    __syncthreads();
  }
  const uint32_t incl = lbase[tid];
  __syncthreads();
  lbase[tid] = incl - cnt;                       // exclusive
  __syncthreads();
  // place the tile in digit order (stable: warp order, then chunk order, then lane order)
  for (int c = 0; c < SORT_SEG; c += 32) {
    const int r = seg + c + lane;
    const bool ok = r < tn;
    const unsigned act = __ballot_sync(0xffffffffu, ok);
    if (!act) break;
    const uint32_t k = ok ? kin[tbase + r] : 0u;
    const uint32_t d = (k >> shift) & 255u;
    const unsigned m = match_bits<8>(d) & act;
    if (ok) {
      const uint32_t loc = lbase[d] + wcnt[warp][d] + __popc(m & lt);
      sk[loc] = k;
      sv[loc] = vin ? vin[tbase + r] : (uint32_t)(tbase + r);
    }
    __syncwarp();
    if (ok && (m & lt) == 0) wcnt[warp][d] += __popc(m);
    __syncwarp();
  }
  __syncthreads();
  // write out in digit order: each digit's run of the tile lands on consecutive positions
  for (int i = tid; i < tn; i += SORT_THREADS) {
    const uint32_t k = sk[i];
    const uint32_t d = (k >> shift) & 255u;
    const uint32_t pos = dbase[d] + (uint32_t)i - lbase[d];
    kout[pos] = k;
    vout[pos] = sv[i];
  }
}

// First sorted position of each key k in [0, nkeys], in two levels: k_brick_starts finds
// the first position of every brick's first key (b * 256, b in [0, nbricks]) by binary
// search; k_cell_starts then gives each brick one warp, which walks the brick's sorted
// keys once and writes the start of each of its 256 keys (a key with no parcels starts at
// the next key's first parcel).
__global__ void k_brick_starts(const uint32_t* __restrict__ skey, long long n, long long nbricks,
                               int* __restrict__ start) {
  const long long b = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (b > nbricks) return;
  const long long k = b * BCELLS;
  long long lo = 0, hi = n;
  while (lo < hi) {
    const long long mid = (lo + hi) >> 1;
    if ((long long)skey[mid] < k) lo = mid + 1; else hi = mid;
  }
  start[k] = (int)lo;
}

__global__ void k_cell_starts(const uint32_t* __restrict__ skey, long long nbricks,
                              int* __restrict__ start) {
  const long long b = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (b >= nbricks) return;                      // whole warps leave together
  const long long k0 = b * BCELLS;
  const int bs = start[k0], be = start[k0 + BCELLS];
  // keys (key[q-1], key[q]] start at q, for q in (bs, be); keys (k0, key[bs]] start at bs
  for (int q0 = bs; q0 < be; q0 += 32) {
    const int q = q0 + lane;
    if (q < be) {
      const long long k = skey[q];
      const long long prev = q == bs ? k0 : (long long)skey[q - 1];
      for (long long kk = prev + 1; kk <= k; ++kk) start[kk] = q;
    }
  }
  // keys after the brick's last parcel (all of them if the brick is empty) start at be
  const long long last = be > bs ? (long long)skey[be - 1] : k0;
  for (long long kk = last + 1 + lane; kk < k0 + BCELLS; kk += 32) start[kk] = be;
}

// ------------------------------------------------------------ level layout --


// The step kernel runs CT = 128 threads per brick: thread t walks the parcels of two
// cells, local cell t of the lower half of the brick and one cell of the upper half (the
// brick's pair map, cellmap[brick * 256 + t]), and a CTA's time follows its largest
// per-thread parcel count (its warps wait for each other at the brick's end). The natural
// pairing gives thread t cell t + 128, one half-brick above: the warp's cells then form two
// 8x4 blocks whose node-tile reads are conflict-free. Where the counts are uneven (a
// fluidised bed: bubbles and clusters), the lower-half cells ranked by count (descending,
// ties by cell index) take the upper-half cells ranked the other way (ascending, ties by
// cell index), so a heavy cell shares its thread with a light one. The choice is made per
// brick at each sort: the count pairing is taken if it lowers the largest per-thread count
// by more than a tenth (it is not tried where the natural pairing is already within a tenth
// of the mean). Within a warp the parcels are laid out by level: level r holds the r-th
// parcel of each thread's sequence (its first cell's parcels in sorted order, then its
// second cell's) for every thread whose sequence is longer than r, in thread order; the
// warp's r-th iteration then reads one contiguous run.
// level_layout chooses the pairing, records it in cellmap, and permutes the parcel arrays
// into the layout straight from the sorted order. Both sorts end in it: the full radix sort
// (k_level_gather) and the local re-sort (k_rs_build, in mppic_resort.cuh). It runs on
// BCELLS threads: thread t lays out the even levels (t < CT) or the odd levels (t >= CT) of
// the cell kernel's thread t mod CT.
struct LevelSmem {
  uint32_t sk[BCELLS];           // ranking keys: each half sorted on its own
  uint8_t pb[CT];                // upper-half cell of each thread under the count pairing
  int wa[BCELLS / 32];
  int mx[BCELLS / 32];
};

// Largest v over the CTA (BCELLS threads); ls.mx is reused, so callers sync between uses.
__device__ __forceinline__ int cta_max(int v, LevelSmem& ls) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = __reduce_max_sync(FULL, v);
  if (lane == 0) ls.mx[warp] = v;
  __syncthreads();
  int m = ls.mx[0];
  for (int w = 1; w < BCELLS / 32; ++w) m = max(m, ls.mx[w]);
  __syncthreads();
  return m;
}

// One CTA (BCELLS threads) lays out brick k0 / BCELLS: its parcels occupy sorted positions
// [bs, bs + cs[BCELLS]); cs (shared) holds each cell's first position relative to bs, and
// perm[i] the source index of relative sorted position i (shared or global). With lperm,
// only the source index of every layout position is written (lperm[q]); the values stay
// where they are and the next step kernel reads them through lperm.
template <class T>
__device__ __forceinline__ void level_layout(const PArrays<T>& src, const PArrays<T>& dst,
                                             long long k0, int bs, const int* cs,
                                             const uint32_t* perm, uint8_t* __restrict__ cellmap,
                                             LevelSmem& ls, uint32_t* __restrict__ lperm = nullptr) {
  const int t = threadIdx.x, lane = t & 31;
  const int u = t & (CT - 1), h = t / CT;        // the cell kernel's thread, level parity
  if (cs[BCELLS] == 0) {                         // an empty brick: the natural pairing
    if (t < CT) cellmap[k0 + t] = (uint8_t)(t + CT);
    return;
  }
  const int total = cs[BCELLS];
  const int nlo = cs[u + 1] - cs[u];
  const int nat = nlo + cs[u + CT + 1] - cs[u + CT];
  const int mx_nat = cta_max(nat, ls);
  int cB = u + CT;
  // the count pairing can lower the largest count to about the mean, ceil(total / CT)
  if (10 * ((total + CT - 1) / CT) < 9 * mx_nat) {  // uniform over the CTA
    const int cnt = min(cs[t + 1] - cs[t], 0xFFFFFF);
    ls.sk[t] = t < CT ? ((uint32_t)(0xFFFFFF - cnt) << 8) | (uint32_t)t
                      : ((uint32_t)cnt << 8) | (uint32_t)t;
    __syncthreads();
    // ascending bitonic sort of each half's unique keys (partners t ^ j stay in the half)
    for (int k = 2; k <= CT; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        const int ixj = t ^ j;
        if (ixj > t) {
          const uint32_t x = ls.sk[t], y = ls.sk[ixj];
          if ((x > y) == ((u & k) == 0)) { ls.sk[t] = y; ls.sk[ixj] = x; }
        }
        __syncthreads();
      }
    }
    if (t < CT) ls.pb[ls.sk[t] & 255u] = (uint8_t)(ls.sk[CT + t] & 255u);
    __syncthreads();
    const int pc = ls.pb[u];
    const int mx_cnt = cta_max(nlo + cs[pc + 1] - cs[pc], ls);
    if (10 * mx_cnt < 9 * mx_nat) cB = pc;
  }
  if (t < CT) cellmap[k0 + t] = (uint8_t)cB;
  const int a0 = cs[u], b0 = cs[cB];
  const int n = nlo + cs[cB + 1] - b0;           // this thread's sequence: a0.., then b0..
  const int ws = __reduce_add_sync(FULL, n);
  const int kw = (t >> 5) & (CT / 32 - 1);       // the cell kernel's warp
  if (t < CT && lane == 0) ls.wa[kw] = ws;
  __syncthreads();
  int off = bs;                                  // first parcel of this warp's group
  for (int w = 0; w < kw; ++w) off += ls.wa[w];
  const int nmax = __reduce_max_sync(FULL, n);
  const unsigned below = (1u << lane) - 1u;
  // L levels of this thread's parity per iteration (4 FP32, 2 FP64), all loads before the
  // stores; the ballots of both parities give the positions
  constexpr int L = sizeof(T) == 4 ? 4 : 2;
  for (int r = 0; r < nmax; r += 2 * L) {
    bool a[L];
    int q[L];
    uint32_t si[L];
    int acc = off;
#pragma unroll
    for (int l = 0; l < 2 * L; ++l) {
      const bool al = n > r + l;
      const unsigned bl = __ballot_sync(FULL, al);
      if ((l & 1) == h) {
        const int rl = r + l;
        a[l >> 1] = al;
        q[l >> 1] = acc + __popc(bl & below);
        si[l >> 1] = al ? perm[rl < nlo ? a0 + rl : b0 + (rl - nlo)] : 0u;
      }
      acc += __popc(bl);
    }
    off = acc;
    if (lperm) {                                 // uniform: the permutation only
#pragma unroll
      for (int l = 0; l < L; ++l)
        if (a[l]) lperm[q[l]] = si[l];
      continue;
    }
    T v[L][8];
    int ip[L], ig[L];
#pragma unroll
    for (int l = 0; l < L; ++l) {
      if (a[l]) {
#pragma unroll
        for (int f = 0; f < 8; ++f) v[l][f] = __ldg(src.a[f] + si[l]);
        if (src.pid) ip[l] = __ldg(src.pid + si[l]);
        if (src.tag) ig[l] = __ldg(src.tag + si[l]);
      }
    }
#pragma unroll
    for (int l = 0; l < L; ++l) {
      if (a[l]) {
#pragma unroll
        for (int f = 0; f < 8; ++f) dst.a[f][q[l]] = v[l][f];
        if (src.pid) dst.pid[q[l]] = ip[l];
        if (src.tag) dst.tag[q[l]] = ig[l];
      }
    }
  }
}

// The level layout after the full radix sort: perm maps each sorted position to its source
// index, start each key to its first sorted position. One CTA per brick.
template <class T>
__global__ void __launch_bounds__(BCELLS)
k_level_gather(PArrays<T> src, PArrays<T> dst, const uint32_t* __restrict__ perm,
               const int* __restrict__ start, uint8_t* __restrict__ cellmap) {
  __shared__ int s_cs[BCELLS + 1];
  __shared__ LevelSmem ls;
  const long long k0 = (long long)blockIdx.x * BCELLS;
  const int t = threadIdx.x;
  const int bs = start[k0];
  s_cs[t] = start[k0 + t] - bs;
  if (t == 0) s_cs[BCELLS] = start[k0 + BCELLS] - bs;
  __syncthreads();
  level_layout<T>(src, dst, k0, bs, s_cs, perm + bs, cellmap, ls);
}

// ---- math of the step: full precision in the FP64 form, CUDA's fast intrinsics in FP32.

}  // namespace mppic
