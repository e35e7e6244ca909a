// libmppic host side: the C ABI declared in include/mppic.h.
//
// The handle owns the scratch of the coupling step (sort buffers, the sorted copy of
// the parcel arrays, cell ranges, fixed-point node accumulators, node fields and the
// objective partials) and enqueues every kernel on one stream. Nothing here computes
// step arithmetic on the host: host code only validates arguments, sizes scratch and
// launches the kernels of mppic_device.cuh.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/mppic.h"
#include "mppic_adjoint.cuh"
#include "mppic_device.cuh"
#include "mppic_sort.cuh"
#include "mppic_resort.cuh"

using namespace mppic;

enum { PH_SORT = 0, PH_DEPOSIT = 1, PH_FINALIZE = 2, PH_STEP = 3, PH_REDUCE = 4, PH_OTHER = 5,
       PH_COUPLE = 6, NPHASE = 7 };

struct mppic_handle {
  mppic_config cfg;
  // batch of independent beds (nbeds == 1: a single bed, described by cfg)
  int nbeds = 1;
  std::vector<mppic_config> bed_cfg;
  std::vector<long long> poff, noff, boff;       // first parcel / node / brick of each bed
  long long* d_poff = nullptr;
  long long* d_noff = nullptr;
  long long* d_boff = nullptr;
  int* d_brick_bed = nullptr;
  double* d_area = nullptr;
  void* d_beds = nullptr;                        // KParams<T>[nbeds]
  std::vector<unsigned char> beds_host;          // last uploaded copy
  unsigned long long* wq = nullptr;              // persistent-kernel work counter
  int nsm = 0;
  int grid_factor = 0;                           // persistent CTAs per SM (0: resident maximum)
  // captured step sequence (mppic_step_graph) and the arguments it was captured for
  cudaGraphExec_t gexec = nullptr;
  std::vector<const void*> gkey;
  cudaStream_t cap_stream = nullptr;             // capture stream (the caller's may be the legacy one)
  cudaStream_t stream = nullptr;
  // side stream of a step call: the node pass runs there while a re-sort runs on `stream`,
  // and each step's objective reduction while the next step's node pass and sort run.
  // Forked and joined with events (no timing), so a captured call stays one graph.
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_fin = nullptr, ev_red = nullptr;
  int device = 0;
  int nx = 0, ny = 0, nz = 0, nbx = 0, nby = 0, nbz = 0;
  long long nnode = 0, nbricks = 0, nkeys = 0;
  int key_bits = 0;
  size_t tsize = 4;          // sizeof parcel scalar
  int words = 1;             // fixed-point words per accumulator
  // grid-sized scratch
  u64* acc = nullptr;        // [NQ][words][nnode]
  void* fld = nullptr;       // 5 x nnode T
  int* cstart = nullptr;     // nkeys + 1
  uint8_t* cellmap = nullptr;  // nbricks * 256: per brick, the upper-half cell of each cell-kernel thread (first CT entries)
  u64* bacc = nullptr;         // [nbricks][NQ][words][TNODES]: bricks' tile slots
  int* bstamp = nullptr;       // [nbricks]: deposit epoch of each slot
  int* epoch = nullptr;        // the current deposit epoch (device counter)
  double* obj_part = nullptr;  // 3 x nbricks
  double* obj_tmp = nullptr;   // 2 doubles (objectives when the caller passes none)
  double* obj_slices = nullptr;  // 3 x OBJ_BLOCKS slice partials of the objective reduction
  unsigned* obj_count = nullptr; // blocks of the objective reduction done (reset by the last)
  int* errs = nullptr;
  int* zr = nullptr;           // node-layer ranges of deposits (see k_finalize)
  // parcel-sized scratch
  long long cap = 0;
  uint32_t* keys[2] = {nullptr, nullptr};
  uint32_t* vals[2] = {nullptr, nullptr};
  uint32_t* hist = nullptr;
  uint32_t* totals = nullptr;
  uint8_t* bcell[2] = {nullptr, nullptr};  // local re-sort: cell bytes of the bucket and its copy
  // local re-sort, per brick (see mppic_resort.cuh)
  int4* bgeo = nullptr;        // {first brick of the bed, nbx, nby, nbz}
  uint32_t* rs_cnt = nullptr;  // [nbricks][27] parcels of the source brick per neighbour slot
  uint32_t* rs_off = nullptr;  // [nbricks][27] first bucket position of each run
  uint32_t* rs_wcnt = nullptr; // [nbricks][8][27] the same counts per warp segment
  int* rs_far = nullptr;       // parcels arriving from beyond the neighbours
  int* rs_far_next = nullptr;  // next free position of the far parcels
  int* rs_count = nullptr;     // bucket size
  int* rs_start = nullptr;     // bucket start
  int* rs_part = nullptr;      // bucket sizes summed over each CTA's bricks
  void* sorted[8] = {};
  int* sorted_pid = nullptr;
  bool sorted_pid_ok = false;
  // ordering state
  long long order_np = -1;   // parcel count the cell ranges were built for
  bool order_on_caller = false;
  long long step_counter = 0;
  // last gas seen by deposit (node grad p arrays are read by later pushes)
  mppic_gas gas{};
  // reverse mode: identity tags carried through sorts and the saved segment states
  int ckpt_every = 0;
  int* tag = nullptr;          // identity of the parcel at each caller position
  int* sorted_tag = nullptr;   // the same for the sorted copy
  uint32_t* lperm = nullptr;   // [cap] a re-sort inside a step call: source index of each position
  long long tag_cap = 0;
  std::vector<void*> ckpt;     // per checkpoint: 8 parcel arrays then the tags
  long long ckpt_np = 0;
  int last_nsteps = -1;
  // backward buffers
  void* adj = nullptr;         // 6 x np (form's type): adjoint of x, y, z, u, v, w
  void* adj_tmp = nullptr;     // 6 x np
  void* Vb = nullptr;          // np: adjoint of the parcel volume
  void* nadj = nullptr;        // nnode: adjoint of the deposited volume
  int* inv = nullptr;          // np
  void* work = nullptr;        // 8 x np parcel arrays of the segment being recomputed
  void* seg = nullptr;         // ckpt_every x 6 x np saved states
  void* adj_src = nullptr;     // 7 x np: per-parcel sources of interp^T
  void* fcache = nullptr;      // ckpt_every x 5 x nnode: node fields of the saved states
  double* hcache = nullptr;    // ckpt_every x 2: height sums of the saved states
  double* part = nullptr;      // AP_ROWS x part_stride: per-block partial sums
  long long part_stride = 0;
  void* adj_sc = nullptr;      // the step's fixed-point multipliers (AdjScale<T>)
  unsigned* adj_cnt = nullptr; // finished-block counter of the last-block reductions
  double* theta = nullptr;     // 3 gradient accumulators
  long long adj_np = 0;
  int seg_len = 0;
  // profiling: event pairs recorded around each phase while enabled
  bool prof = false;
  std::vector<cudaEvent_t> ev;         // start/stop pairs
  std::vector<int> ev_phase;
  size_t ev_used = 0;
  long long launches[NPHASE] = {};
  bool drag_any = false;       // a bed names a drag closure other than Wen-Yu
  long long total_launches = 0;
  char err[512] = {0};
};


static char g_create_err[512] = {0};

namespace {

mppic_status fail(mppic_handle* h, mppic_status s, const char* fmt, ...) {
  char* buf = h ? h->err : g_create_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, 512, fmt, ap);
  va_end(ap);
  return s;
}

// A failed runtime call is reported through the status; the runtime's last-error state is
// cleared so that the next launch check does not report it again.
#define CU(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      cudaGetLastError();                                                                 \
      return fail(h, e_ == cudaErrorMemoryAllocation ? MPPIC_ERR_OOM : MPPIC_ERR_CUDA,    \
                  "%s: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);   \
    }                                                                                     \
  } while (0)

#define LAUNCHED()                                                                        \
  do {                                                                                    \
    cudaError_t e_ = cudaGetLastError();                                                  \
    if (e_ != cudaSuccess)                                                                \
      return fail(h, MPPIC_ERR_CUDA, "kernel launch: %s (%s:%d)", cudaGetErrorString(e_), \
                  __FILE__, __LINE__);                                                    \
  } while (0)

inline unsigned blocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

// Records a CUDA event pair around one phase on the handle's stream (or the given one)
// while profiling is enabled, and counts the phase's kernel launches.
struct Phase {
  mppic_handle* h;
  int phase;
  cudaStream_t st;
  size_t slot = (size_t)-1;
  Phase(mppic_handle* h_, int ph, cudaStream_t s = nullptr) : h(h_), phase(ph), st(s ? s : h_->stream) {
    if (!h->prof) return;
    if (h->ev_used * 2 + 2 > h->ev.size()) {
      cudaEvent_t a, b;
      if (cudaEventCreate(&a) != cudaSuccess) return;
      if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
      h->ev.push_back(a);
      h->ev.push_back(b);
      h->ev_phase.push_back(ph);
    }
    slot = h->ev_used++;
    h->ev_phase[slot] = ph;
    cudaEventRecord(h->ev[2 * slot], st);
  }
  void launched(int n = 1) {
    if (!h->prof) return;
    h->launches[phase] += n;
    h->total_launches += n;
  }
  ~Phase() {
    if (slot != (size_t)-1) cudaEventRecord(h->ev[2 * slot + 1], st);
  }
};

// Fixed-point multipliers: powers of two, so that the product of a parcel value with them is
// exact. The solids volume counts 2^47..2^48 units per cell volume (FP32 form, int64) or
// 2^95..2^96 (FP64 form, int128); the drag sums 2^39..2^40 (2^87..2^88) units per
// rho_p x cell volume per second.
template <class T>
void fixed_units(const mppic_config& c, size_t tsize, T* mV, T* mA) {
  int ev = 0, ea = 0;
  std::frexp(c.dx * c.dy * c.dz, &ev);
  std::frexp(c.rho_p * c.dx * c.dy * c.dz, &ea);
  const int SV = tsize == 4 ? 48 : 96, SA = tsize == 4 ? 40 : 88;
  *mV = (T)std::ldexp(1.0, SV - ev);
  *mA = (T)std::ldexp(1.0, SA - ea);
}

template <class T>
KParams<T> make_params(const mppic_handle* h, const mppic_gas* gas) {
  const mppic_config& c = h->cfg;
  KParams<T> p;
  memset(&p, 0, sizeof(p));
  p.nx = c.nx; p.ny = c.ny; p.nz = c.nz;
  p.nbx = h->nbx; p.nby = h->nby; p.nbz = h->nbz;
  p.nnode = h->nnode;
  p.nbricks = h->nbricks;
  p.nbase = 0;
  p.bbase = 0;
  p.nstride = h->nnode;
  const double hs[3] = {c.dx, c.dy, c.dz};
  const int ns[3] = {c.nx, c.ny, c.nz};
  for (int a = 0; a < 3; ++a) {
    p.inv_d[a] = 1.0 / hs[a];
    p.inv_f[a] = (float)p.inv_d[a];
    p.inv_lo[a] = (float)(p.inv_d[a] - (double)p.inv_f[a]);
    p.invh[a] = (T)p.inv_d[a];
    p.L[a] = (T)(ns[a] * hs[a]);
    p.g[a] = (T)c.g[a];
    p.gp[a] = (T)c.gradp[a];
  }
  p.vcell = c.dx * c.dy * c.dz;
  p.rho_g = (T)c.rho_g; p.mu_g = (T)c.mu_g; p.rho_p = (T)c.rho_p;
  p.Ps = (T)c.Ps; p.beta = (T)c.beta; p.eps_cp = (T)c.eps_cp; p.alpha = (T)c.alpha;
  p.eg_min = (T)c.eps_g_min; p.e_wall = (T)c.e_wall; p.C = (T)c.drag_mult; p.sd = (T)c.dscale;
  p.dt = (T)c.dt; p.u_in = (T)c.u_in;
  p.vcoef = (T)(M_PI / 6.0 * c.dscale * c.dscale * c.dscale);
  p.inv_rho_p = (T)(1.0 / c.rho_p);
  p.kRe = (T)(c.rho_g / c.mu_g);
  p.kD1 = (T)(c.drag_mult * 18.0 * c.mu_g / c.rho_p);
  p.kD2 = (T)(c.drag_mult * 0.33 * c.rho_g / c.rho_p);
  p.kD1u = (T)(18.0 * c.mu_g / c.rho_p);
  p.kD2u = (T)(0.33 * c.rho_g / c.rho_p);
  p.kE1 = (T)(c.drag_mult * 150.0 * c.mu_g / c.rho_p);
  p.kE2 = (T)(c.drag_mult * 1.75 * c.rho_g / c.rho_p);
  p.kS1 = (T)(c.drag_mult * 0.75 * c.rho_g / c.rho_p);
  p.kS2 = (T)(c.mu_g / c.rho_g);
  p.drag_model = c.drag_model;
  fixed_units(c, sizeof(T), &p.mV, &p.mA);
  p.inv_vcell = 1.0 / p.vcell;
  p.es_scale = (float)(1.0 / (double)p.mV / p.vcell);
  p.inv_mV = 1.0 / (double)p.mV; p.inv_mA = 1.0 / (double)p.mA;
  T* f = static_cast<T*>(h->fld);
  for (int k = 0; k < 5; ++k) p.fld[k] = f + (long long)k * h->nnode;
  p.has_gp = 0;
  if (gas) {
    for (int a = 0; a < 3; ++a) p.U[a] = static_cast<const T*>(gas->U[a]);
    if (gas->gradp[0] && gas->gradp[1] && gas->gradp[2]) {
      p.has_gp = 1;
      for (int a = 0; a < 3; ++a) p.gpf[a] = static_cast<const T*>(gas->gradp[a]);
    }
  }
  p.acc = h->acc;
  p.errs = h->errs;
  p.zr = h->zr;
  p.cstart = h->cstart;
  p.cellmap = h->cellmap;
  p.bacc = h->bacc;
  p.bstamp = h->bstamp;
  p.epoch = h->epoch;
  return p;
}

// Per-bed parameters of a batch, uploaded when they change. Node-field and gas pointers
// point at each bed's slice of the concatenated node arrays.
template <class T>
mppic_status upload_beds(mppic_handle* h, const mppic_gas* gas, const KParams<T>** out) {
  *out = nullptr;
  if (h->nbeds == 1) return MPPIC_OK;
  std::vector<KParams<T>> v(h->nbeds);
  for (int b = 0; b < h->nbeds; ++b) {
    mppic_handle tmp;                       // only cfg/geometry/pointers are read by make_params
    tmp.cfg = h->bed_cfg[b];
    tmp.cfg.precision = h->cfg.precision;
    const mppic_config& c = tmp.cfg;
    tmp.nbx = (c.nx + BX - 1) / BX; tmp.nby = (c.ny + BY - 1) / BY; tmp.nbz = (c.nz + BZ - 1) / BZ;
    tmp.nnode = h->noff[b + 1] - h->noff[b];
    tmp.nbricks = h->boff[b + 1] - h->boff[b];
    tmp.fld = h->fld; tmp.acc = h->acc; tmp.errs = h->errs; tmp.cstart = h->cstart; tmp.cellmap = h->cellmap; tmp.zr = h->zr;
    tmp.bacc = h->bacc; tmp.bstamp = h->bstamp; tmp.epoch = h->epoch;
    KParams<T> p = make_params<T>(&tmp, nullptr);
    p.nbase = h->noff[b];
    p.bbase = h->boff[b];
    p.nstride = h->nnode;
    T* f = static_cast<T*>(h->fld);
    for (int k = 0; k < 5; ++k) p.fld[k] = f + (long long)k * h->nnode + h->noff[b];
    p.has_gp = 0;
    if (gas) {
      for (int a = 0; a < 3; ++a)
        p.U[a] = gas->U[a] ? static_cast<const T*>(gas->U[a]) + h->noff[b] : nullptr;
      if (gas->gradp[0] && gas->gradp[1] && gas->gradp[2]) {
        p.has_gp = 1;
        for (int a = 0; a < 3; ++a) p.gpf[a] = static_cast<const T*>(gas->gradp[a]) + h->noff[b];
      }
    }
    tmp.fld = nullptr; tmp.acc = nullptr; tmp.errs = nullptr; tmp.cstart = nullptr; tmp.cellmap = nullptr; tmp.zr = nullptr;
    tmp.bacc = nullptr; tmp.bstamp = nullptr; tmp.epoch = nullptr;
    v[b] = p;
  }
  const size_t bytes = sizeof(KParams<T>) * h->nbeds;
  if (!h->d_beds) CU(cudaMalloc(&h->d_beds, bytes));
  if (h->beds_host.size() != bytes || memcmp(h->beds_host.data(), v.data(), bytes) != 0) {
    h->beds_host.assign(reinterpret_cast<unsigned char*>(v.data()),
                        reinterpret_cast<unsigned char*>(v.data()) + bytes);
    CU(cudaMemcpyAsync(h->d_beds, h->beds_host.data(), bytes, cudaMemcpyHostToDevice, h->stream));
    CU(cudaStreamSynchronize(h->stream));
  }
  *out = static_cast<const KParams<T>*>(h->d_beds);
  return MPPIC_OK;
}

template <class T>
PArrays<T> caller_arrays(const mppic_parcels* pc, int* tag = nullptr) {
  PArrays<T> a;
  a.perm = nullptr;
  void* const src[8] = {pc->x, pc->y, pc->z, pc->u, pc->v, pc->w, pc->d, pc->omega};
  for (int f = 0; f < 8; ++f) a.a[f] = static_cast<T*>(src[f]);
  a.pid = pc->pid;
  a.tag = tag;
  return a;
}

template <class T>
PArrays<T> sorted_arrays(mppic_handle* h, bool with_pid, bool with_tag = false) {
  PArrays<T> a;
  a.perm = nullptr;
  for (int f = 0; f < 8; ++f) a.a[f] = static_cast<T*>(h->sorted[f]);
  a.pid = with_pid ? h->sorted_pid : nullptr;
  a.tag = with_tag ? h->sorted_tag : nullptr;
  return a;
}

mppic_status check_parcels(mppic_handle* h, const mppic_parcels* pc) {
  if (!pc) return fail(h, MPPIC_ERR_INVALID, "parcels is NULL");
  if (pc->np < 0 || pc->np > 0x7fffffffLL)
    return fail(h, MPPIC_ERR_INVALID, "np=%lld out of range [0, 2^31)", pc->np);
  if (pc->np > 0 && (!pc->x || !pc->y || !pc->z || !pc->u || !pc->v || !pc->w || !pc->d ||
                     !pc->omega))
    return fail(h, MPPIC_ERR_INVALID, "a parcel array is NULL");
  // the brick kernels bulk-copy the parcel arrays, which needs 16-byte aligned bases
  const void* arrays[8] = {pc->x, pc->y, pc->z, pc->u, pc->v, pc->w, pc->d, pc->omega};
  for (int f = 0; f < 8; ++f)
    if (((uintptr_t)arrays[f]) % 16 != 0)
      return fail(h, MPPIC_ERR_INVALID, "parcel array %d is not 16-byte aligned", f);
  return MPPIC_OK;
}

mppic_status ensure_capacity(mppic_handle* h, long long np, bool want_pid) {
  if (np <= h->cap && (!want_pid || h->sorted_pid)) return MPPIC_OK;
  long long cap = np > h->cap ? np : h->cap;
  if (cap > h->cap) {
    for (int i = 0; i < 2; ++i) {
      cudaFree(h->keys[i]); cudaFree(h->vals[i]); cudaFree(h->bcell[i]);
      h->keys[i] = h->vals[i] = nullptr;
      h->bcell[i] = nullptr;
    }
    cudaFree(h->hist); h->hist = nullptr;
    for (int f = 0; f < 8; ++f) { cudaFree(h->sorted[f]); h->sorted[f] = nullptr; }
    cudaFree(h->sorted_pid); h->sorted_pid = nullptr;
    cudaFree(h->lperm); h->lperm = nullptr;
    h->cap = 0;
    long long nblk = (cap + SORT_TILE - 1) / SORT_TILE;
    for (int i = 0; i < 2; ++i) {
      CU(cudaMalloc(&h->keys[i], sizeof(uint32_t) * cap));
      CU(cudaMalloc(&h->vals[i], sizeof(uint32_t) * cap));
      CU(cudaMalloc(&h->bcell[i], cap));
    }
    CU(cudaMalloc(&h->hist, sizeof(uint32_t) * 256 * (nblk > 0 ? nblk : 1)));
    for (int f = 0; f < 8; ++f) CU(cudaMalloc(&h->sorted[f], h->tsize * cap));
    CU(cudaMalloc(&h->lperm, sizeof(uint32_t) * cap));
    h->cap = cap;
  }
  if (want_pid && !h->sorted_pid) CU(cudaMalloc(&h->sorted_pid, sizeof(int) * h->cap));
  return MPPIC_OK;
}

// Sort the parcels currently in `cur` by brick-major cell key into the handle's sorted
// copy, and rebuild the cell ranges. Leaves the sorted copy as the parcel source.
template <class T>
mppic_status sort_into_scratch(mppic_handle* h, const mppic_parcels* pc, PArrays<T> cur,
                               bool keys_ready = false, bool local = false,
                               const mppic_gas* gas = nullptr, bool perm_only = false) {
  const long long np = pc->np;
  mppic_status s = ensure_capacity(h, np, pc->pid != nullptr);
  if (s) return s;
  KParams<T> p = make_params<T>(h, nullptr);
  const KParams<T>* beds = nullptr;
  // the sort reads no gas field; a step passes its own, so the per-bed parameters it uploads
  // are the ones the step uses next (an upload waits for the stream)
  s = upload_beds<T>(h, gas, &beds);
  if (s) return s;
  cudaStream_t st = h->stream;
  Phase ph(h, PH_SORT);
  if (np > 0) {
    if (!keys_ready) {          // else the last step kernel wrote them into keys[0]
      if (beds)
        k_keys_b<T><<<blocks(np, 256), 256, 0, st>>>(beds, h->d_poff, h->nbeds, cur.a[0],
                                                      cur.a[1], cur.a[2], h->keys[0], np);
      else
        k_keys<T><<<blocks(np, 256), 256, 0, st>>>(p, cur.a[0], cur.a[1], cur.a[2], h->keys[0], np);
      LAUNCHED();
    }
    if (local) {                // `cur` is laid out by the current cell starts
      const long long nb = h->nbricks;
      const unsigned gb = (unsigned)nb;            // one CTA per brick: empty ones exit at once
      CU(cudaMemsetAsync(h->rs_far, 0, sizeof(int) * nb, st));
      k_rs_hist<<<gb, RS_THREADS, 0, st>>>(h->keys[0], h->cstart, h->bgeo, nb, h->rs_cnt,
                                           h->rs_wcnt, h->rs_far);
      k_rs_count<<<blocks(nb, RS_THREADS), RS_THREADS, 0, st>>>(h->rs_cnt, h->rs_far, h->bgeo, nb,
                                                                h->rs_count, h->rs_part);
      k_rs_offsets<<<blocks(nb, RS_THREADS), RS_THREADS, 0, st>>>(
          h->rs_cnt, h->rs_count, h->rs_part, h->bgeo, nb, h->rs_start, h->rs_off,
          h->rs_far_next, h->cstart + h->nkeys);
      // the hist pass read the old brick ranges; the scatter reads them too, the build
      // rewrites them
      k_rs_scatter<<<gb, RS_THREADS, 0, st>>>(h->keys[0], h->cstart, h->bgeo, nb, h->rs_off,
                                              h->rs_wcnt, h->rs_far_next, h->keys[1], h->bcell[0]);
      k_rs_build<T><<<(unsigned)nb, RS_THREADS, 0, st>>>(
          cur, sorted_arrays<T>(h, cur.pid != nullptr, cur.tag != nullptr), h->rs_start,
          h->rs_count, h->rs_far, h->keys[1], h->bcell[0], h->vals[0], h->bcell[1], h->cstart,
          h->cellmap, perm_only ? h->lperm : nullptr);
      LAUNCHED();
      ph.launched(keys_ready ? 5 : 6);
      h->order_np = np;
      h->sorted_pid_ok = pc->pid != nullptr;
      return MPPIC_OK;
    }
    const int nblk = (int)((np + SORT_TILE - 1) / SORT_TILE);
    const int passes = (h->key_bits + 7) / 8;
    int src = 0;
    for (int ps = 0; ps < passes; ++ps) {
      const int shift = 8 * ps;
      k_sort_hist<<<nblk, SORT_THREADS, 0, st>>>(h->keys[src], np, shift, h->hist, nblk);
      k_sort_scan<<<256, 1024, 0, st>>>(h->hist, nblk, h->totals);
      if (ps == 0)                // values are the parcel indices; keys spread over digits
        k_sort_scatter_reorder<<<nblk, SORT_THREADS, 0, st>>>(h->keys[src], nullptr,
                                                              h->keys[1 - src], h->vals[1 - src],
                                                              np, shift, h->hist, h->totals, nblk);
      else
        k_sort_scatter_direct<<<nblk, SORT_THREADS, 0, st>>>(h->keys[src], h->vals[src],
                                                             h->keys[1 - src], h->vals[1 - src],
                                                             np, shift, h->hist, h->totals, nblk);
      LAUNCHED();
      ph.launched(3);
      src = 1 - src;
    }
    k_brick_starts<<<blocks(h->nbricks + 1, 256), 256, 0, st>>>(h->keys[src], np, h->nbricks,
                                                                 h->cstart);
    LAUNCHED();
    k_cell_starts<<<blocks(h->nbricks * 32, 256), 256, 0, st>>>(h->keys[src], h->nbricks, h->cstart);
    LAUNCHED();
    // the sorted copy, in the level layout of each group of 32 count-ranked cells
    k_level_gather<T><<<(unsigned)h->nbricks, BCELLS, 0, st>>>(
        cur, sorted_arrays<T>(h, cur.pid != nullptr, cur.tag != nullptr), h->vals[src], h->cstart,
        h->cellmap);
    ph.launched(keys_ready ? 3 : 4);
  } else {
    CU(cudaMemsetAsync(h->cstart, 0, sizeof(int) * (h->nkeys + 1), st));
  }
  LAUNCHED();
  h->order_np = np;
  h->sorted_pid_ok = pc->pid != nullptr;
  return MPPIC_OK;
}

// Node pass over the layers deposited into (all layers if full), then roll the ranges.
template <class T>
mppic_status launch_finalize(mppic_handle* h, const KParams<T>& p, double* vs_out, bool full,
                             const KParams<T>* beds = nullptr, cudaStream_t st = nullptr) {
  if (!st) st = h->stream;
  Phase ph(h, PH_FINALIZE, st);
  unsigned g = blocks(h->nnode, 256);
  if (g > 152u * 8u) g = 152u * 8u;
  if (beds) {                  // a batch: every node of every bed
    ph.launched(2);
    k_finalize_b<T><<<g, 256, 0, st>>>(beds, h->d_noff, h->nbeds, h->nnode);
    LAUNCHED();
    k_epoch_next<<<1, 1, 0, st>>>(h->epoch);
    LAUNCHED();
    return MPPIC_OK;
  }
  ph.launched(2);
  k_finalize<T><<<g, 256, 0, st>>>(p, vs_out, full ? 1 : 0);
  LAUNCHED();
  k_range_roll<<<1, 1, 0, st>>>(h->zr, h->epoch);
  LAUNCHED();
  return MPPIC_OK;
}

// After the last step of a call: the bricks' drag sums into the global accumulators (for
// the drag-sum output), then the next epoch.
template <class T>
mppic_status launch_drag_fold(mppic_handle* h, const KParams<T>& p, const KParams<T>* beds) {
  Phase ph(h, PH_FINALIZE);
  ph.launched(2);
  unsigned g = blocks(h->nnode, 256);
  if (g > 152u * 8u) g = 152u * 8u;
  if (beds)
    k_drag_fold_b<T><<<g, 256, 0, h->stream>>>(beds, h->d_noff, h->nbeds, h->nnode);
  else
    k_drag_fold<T><<<g, 256, 0, h->stream>>>(p);
  LAUNCHED();
  k_epoch_next<<<1, 1, 0, h->stream>>>(h->epoch);
  LAUNCHED();
  return MPPIC_OK;
}

// The Vs accumulator may still hold the deposit a previous push made for positions the
// caller has since replaced or advanced; a deposit of the current positions starts from zero.
mppic_status clear_volume_accumulator(mppic_handle* h) {
  CU(cudaMemsetAsync(h->acc, 0, sizeof(u64) * h->words * h->nnode, h->stream));
  return MPPIC_OK;
}

// One cell kernel instance: its shared-memory attribute (the larger layout, with the grad p
// planes) and its resident CTAs for each tile layout are set up once.
template <class T, int MODE, int DRAG, bool BATCH, bool PERM>
mppic_status cell_kernel_setup(mppic_handle* h, bool gp, int* resident) {
  static bool done = false;
  static int res[2] = {0, 0};
  if (!done) {
    CU(cudaFuncSetAttribute(k_cells<T, MODE, DRAG, BATCH, PERM>,
                            cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CellSmem<T>::bytes(true)));
    for (int g = 0; g < 2; ++g)
      CU(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&res[g], k_cells<T, MODE, DRAG, BATCH, PERM>, CT,
                                                       CellSmem<T>::bytes(g != 0)));
    done = true;
  }
  *resident = res[gp ? 1 : 0];
  return MPPIC_OK;
}

template <class T, int MODE, int DRAG, bool BATCH, bool PERM>
mppic_status launch_cells_b(mppic_handle* h, const KParams<T>& p, PArrays<T> src, PArrays<T> dst,
                            int* cell_out, long long np, const KParams<T>* beds, uint32_t* key_out) {
  // the node-field tile holds the grad p planes when the gas gives a node field (the same
  // for every bed of a batch)
  const bool gp = p.has_gp != 0;
  int resident = 0;
  mppic_status s = cell_kernel_setup<T, MODE, DRAG, BATCH, PERM>(h, gp, &resident);
  if (s) return s;
  if (h->nbricks == 0) return MPPIC_OK;
  // persistent grid: the CTAs that fit on the GPU at once (or grid_factor per SM)
  const int per_sm = h->grid_factor > 0 ? h->grid_factor : (resident > 0 ? resident : 1);
  long long grid = (long long)per_sm * (h->nsm > 0 ? h->nsm : 1);
  if (grid > h->nbricks) grid = h->nbricks;
  CU(cudaMemsetAsync(h->wq, 0, sizeof(unsigned long long), h->stream));
  Phase ph(h, MODE == MODE_VOLUME ? PH_DEPOSIT : MODE == MODE_STEP ? PH_STEP : PH_COUPLE);
  ph.launched();
  k_cells<T, MODE, DRAG, BATCH, PERM><<<(unsigned)grid, CT, CellSmem<T>::bytes(gp), h->stream>>>(
      p, beds, h->d_brick_bed, h->nbricks, h->wq, src, dst, cell_out, key_out, h->obj_part, np,
      gp ? 1 : 0);
  LAUNCHED();
  return MPPIC_OK;
}

// A batch (beds != NULL) takes the instance that reads each bed's parameters from `beds`;
// src.perm set (a step or volume deposit after a sort that wrote only the permutation) the
// instance that reads its parcels through it.
template <class T, int MODE, int DRAG>
mppic_status launch_cells_t(mppic_handle* h, const KParams<T>& p, PArrays<T> src, PArrays<T> dst,
                            int* cell_out, long long np, const KParams<T>* beds, uint32_t* key_out) {
  if constexpr (MODE != MODE_DRAG)
    if (src.perm)
      return beds ? launch_cells_b<T, MODE, DRAG, true, true>(h, p, src, dst, cell_out, np, beds, key_out)
                  : launch_cells_b<T, MODE, DRAG, false, true>(h, p, src, dst, cell_out, np, beds, key_out);
  return beds ? launch_cells_b<T, MODE, DRAG, true, false>(h, p, src, dst, cell_out, np, beds, key_out)
              : launch_cells_b<T, MODE, DRAG, false, false>(h, p, src, dst, cell_out, np, beds, key_out);
}

// mode: MODE_VOLUME, MODE_STEP or MODE_DRAG; the Wen-Yu-only instance unless a bed names
// another drag closure.
template <class T>
mppic_status launch_cells(mppic_handle* h, int mode, const KParams<T>& p, PArrays<T> src,
                          PArrays<T> dst, int* cell_out, long long np,
                          const KParams<T>* beds = nullptr, uint32_t* key_out = nullptr) {
  if (mode == MODE_VOLUME)
    return launch_cells_t<T, MODE_VOLUME, 0>(h, p, src, dst, cell_out, np, beds, key_out);
  if (mode == MODE_STEP)
    return h->drag_any ? launch_cells_t<T, MODE_STEP, 1>(h, p, src, dst, cell_out, np, beds, key_out)
                       : launch_cells_t<T, MODE_STEP, 0>(h, p, src, dst, cell_out, np, beds, key_out);
  return h->drag_any ? launch_cells_t<T, MODE_DRAG, 1>(h, p, src, dst, cell_out, np, beds, key_out)
                     : launch_cells_t<T, MODE_DRAG, 0>(h, p, src, dst, cell_out, np, beds, key_out);
}

// Implicit coupling, one gas iteration at the nodes from the last drag deposit, then the
// next epoch (the drag tile slots are consumed).
template <class T>
mppic_status launch_gas_update(mppic_handle* h, const KParams<T>& p, const KParams<T>* beds) {
  Phase ph(h, PH_COUPLE);
  ph.launched(2);
  unsigned g = blocks(h->nnode, 256);
  if (g > 152u * 8u) g = 152u * 8u;
  if (beds)
    k_gas_update_b<T><<<g, 256, 0, h->stream>>>(beds, h->d_noff, h->nbeds, h->nnode);
  else
    k_gas_update<T><<<g, 256, 0, h->stream>>>(p);
  LAUNCHED();
  k_epoch_next<<<1, 1, 0, h->stream>>>(h->epoch);
  LAUNCHED();
  return MPPIC_OK;
}

// Deposit the solids volume of the given parcels (order from the handle, sorting into the
// scratch copy if the caller's arrays carry no valid order) and form the node fields.
template <class T>
mppic_status deposit_impl(mppic_handle* h, const mppic_parcels* pc, const mppic_gas* gas,
                          double* vs_out, bool full) {
  PArrays<T> cur = caller_arrays<T>(pc);
  PArrays<T> src = cur;
  if (!h->order_on_caller || h->order_np != pc->np) {
    mppic_status s = sort_into_scratch<T>(h, pc, cur);
    if (s) return s;
    src = sorted_arrays<T>(h, pc->pid != nullptr);
    h->order_on_caller = false;
  }
  KParams<T> p = make_params<T>(h, gas);
  mppic_status s = clear_volume_accumulator(h);
  if (s) return s;
  s = launch_cells<T>(h, MODE_VOLUME, p, src, src, nullptr, pc->np);
  if (s) return s;
  s = launch_finalize<T>(h, p, vs_out, full);
  if (s) return s;
  if (gas) h->gas = *gas; else memset(&h->gas, 0, sizeof(h->gas));
  return MPPIC_OK;
}

// Identity tags and checkpoint storage for a step call with checkpointing.
mppic_status prepare_checkpoints(mppic_handle* h, long long np, int nsteps) {
  if (np > h->tag_cap) {
    cudaFree(h->tag); cudaFree(h->sorted_tag);
    h->tag = h->sorted_tag = nullptr;
    h->tag_cap = 0;
    CU(cudaMalloc(&h->tag, sizeof(int) * (np > 0 ? np : 1)));
    CU(cudaMalloc(&h->sorted_tag, sizeof(int) * (np > 0 ? np : 1)));
    h->tag_cap = np;
  }
  const int K = h->ckpt_every;
  const size_t need = (size_t)((nsteps + K - 1) / K > 0 ? (nsteps + K - 1) / K : 1);
  if (np != h->ckpt_np) {
    for (void* c : h->ckpt) cudaFree(c);
    h->ckpt.clear();
    h->ckpt_np = np;
  }
  while (h->ckpt.size() < need) {
    void* c = nullptr;
    CU(cudaMalloc(&c, (8 * h->tsize + sizeof(int)) * (size_t)(np > 0 ? np : 1)));
    h->ckpt.push_back(c);
  }
  if (np > 0) {
    k_iota<<<blocks(np, 256), 256, 0, h->stream>>>(h->tag, np);
    LAUNCHED();
  }
  return MPPIC_OK;
}

template <class T>
mppic_status save_checkpoint(mppic_handle* h, int idx, const PArrays<T>& src, long long np) {
  if (np == 0) return MPPIC_OK;
  char* c = static_cast<char*>(h->ckpt[idx]);
  for (int f = 0; f < 8; ++f)
    CU(cudaMemcpyAsync(c + (size_t)f * np * h->tsize, src.a[f], np * h->tsize,
                       cudaMemcpyDeviceToDevice, h->stream));
  CU(cudaMemcpyAsync(c + (size_t)8 * np * h->tsize, src.tag, np * sizeof(int),
                     cudaMemcpyDeviceToDevice, h->stream));
  return MPPIC_OK;
}

template <class T>
mppic_status step_impl(mppic_handle* h, mppic_parcels* pc, const mppic_gas* gas, int nsteps,
                       double* obj_out) {
  const long long np = pc->np;
  const bool ck = h->ckpt_every > 0;
  if (ck) {
    mppic_status s = prepare_checkpoints(h, np, nsteps);
    if (s) return s;
  }
  PArrays<T> dst = caller_arrays<T>(pc, ck ? h->tag : nullptr);
  PArrays<T> src = dst;
  const PArrays<T> caller = dst;
  const int every = h->cfg.sort_every;
  auto sort_due = [&](long long step) { return every > 0 && step % every == 0; };
  // A local re-sort (the arrays hold the layout of the handle's last sort) may leave the
  // values where they are and only write the permutation, which the step reads its parcels
  // through, writing them to the other buffer (the handle's copy, or the caller's arrays if
  // the values are in the copy); a step without a sort updates the values where they are,
  // and the copy's values go back to the caller's arrays once, after the last step. Taken
  // where no identity array travels with the parcels and no gas iteration reads them before
  // the step. A re-sort at the call's start does the same, and the call's volume deposit
  // then reads the parcels through its permutation, as the gathered path reads the moved
  // values: both group the parcels by their new cells, so their sums agree bit for bit.
  const bool perm_sort = !ck && !pc->pid && h->cfg.coupling_iters == 0;
  bool start_perm = false;
  if (!h->order_on_caller || h->order_np != np || sort_due(h->step_counter)) {
    const bool local = h->order_on_caller && h->order_np == np;
    if (local && perm_sort && nsteps > 0) {
      start_perm = true;
    } else {
      mppic_status s = sort_into_scratch<T>(h, pc, dst, false, local, gas);
      if (s) return s;
      src = sorted_arrays<T>(h, pc->pid != nullptr, ck);
    }
  }
  KParams<T> p = make_params<T>(h, gas);
  const KParams<T>* beds = nullptr;
  mppic_status s = upload_beds<T>(h, gas, &beds);
  if (s) return s;
  s = clear_volume_accumulator(h);
  if (s) return s;
  if (start_perm) {
    s = sort_into_scratch<T>(h, pc, caller, false, true, gas, true);
    if (s) return s;
    src.perm = h->lperm;
  }
  s = launch_cells<T>(h, MODE_VOLUME, p, src, src, nullptr, pc->np, beds);   // Vs of the current positions
  if (s) return s;
  const double area = h->cfg.nx * h->cfg.dx * h->cfg.ny * h->cfg.dy;
  const PArrays<T> copy = sorted_arrays<T>(h, false, false);
  bool in_copy = start_perm;                     // the values are (step 0: go) in the handle's copy
  bool red_pending = false;                      // a reduction on the side stream not yet joined
  for (int it = 0; it < nsteps; ++it) {
    dst = in_copy ? copy : caller;
    // A step with a re-sort: the node pass of the last step's deposits (it reads the deposit
    // accumulators and writes the node fields; the sort touches neither) runs on the side
    // stream meanwhile, and the step kernel waits for both.
    const bool sort_now = it > 0 && sort_due(h->step_counter + it);
    if (sort_now) {
      CU(cudaEventRecord(h->ev_fork, h->stream));
      CU(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
      s = launch_finalize<T>(h, p, nullptr, false, beds, h->side);
      if (s) return s;
      CU(cudaEventRecord(h->ev_fin, h->side));
    }
    if (sort_now) {
      if (perm_sort) {
        s = sort_into_scratch<T>(h, pc, src, true, true, gas, true);   // keys from the previous step
        if (s) return s;
        dst = in_copy ? caller : copy;
        in_copy = !in_copy;
        src.perm = h->lperm;
      } else {
        s = sort_into_scratch<T>(h, pc, caller, true, true, gas);    // keys from the previous step
        if (s) return s;
        src = sorted_arrays<T>(h, pc->pid != nullptr, ck);
      }
    }
    if (ck && it % h->ckpt_every == 0) {
      s = save_checkpoint<T>(h, it / h->ckpt_every, src, np);
      if (s) return s;
    }
    if (sort_now) {
      CU(cudaStreamWaitEvent(h->stream, h->ev_fin, 0));
    } else {
      s = launch_finalize<T>(h, p, nullptr, false, beds);
      if (s) return s;
    }
    // implicit coupling (Sec. 2.2.2): the drag sums again at the head of every gas
    // iteration, each followed by the iteration's node update of the gas velocity
    for (int m = 0; m < h->cfg.coupling_iters; ++m) {
      s = launch_cells<T>(h, MODE_DRAG, p, src, src, nullptr, np, beds);
      if (s) return s;
      s = launch_gas_update<T>(h, p, beds);
      if (s) return s;
    }
    // the step before a sort in this call writes the sort keys of the new positions
    uint32_t* key_out = it + 1 < nsteps && sort_due(h->step_counter + it + 1) ? h->keys[0] : nullptr;
    if (red_pending) {           // the step rewrites the per-brick objective partials
      CU(cudaStreamWaitEvent(h->stream, h->ev_red, 0));
      red_pending = false;
    }
    s = launch_cells<T>(h, MODE_STEP, p, src, dst, (it == nsteps - 1 && !beds) ? pc->cell : nullptr, np,
                        beds, key_out);
    if (s) return s;
    src = dst;
    {                            // the objectives on the side stream, while the next step's
      CU(cudaEventRecord(h->ev_fork, h->stream));   // node pass and sort run
      CU(cudaStreamWaitEvent(h->side, h->ev_fork, 0));
      Phase ph(h, PH_REDUCE, h->side);
      ph.launched();
      if (beds)
        k_obj_reduce_b<<<h->nbeds, 256, 0, h->side>>>(
            h->obj_part, h->d_boff, h->d_area, obj_out ? obj_out + 2LL * it * h->nbeds : h->obj_tmp);
      else
        k_obj_reduce<<<OBJ_BLOCKS, OBJ_THREADS, 0, h->side>>>(
            h->obj_part, h->nbricks, area, h->obj_slices, h->obj_count,
            obj_out ? obj_out + 2 * it : h->obj_tmp);
      LAUNCHED();
    }
    CU(cudaEventRecord(h->ev_red, h->side));
    red_pending = true;
  }
  if (red_pending) CU(cudaStreamWaitEvent(h->stream, h->ev_red, 0));   // joined: the call's
                                                                         // work is on `stream`
  if (in_copy && np > 0)                         // the last step wrote the handle's copy
    for (int f = 0; f < 8; ++f)
      CU(cudaMemcpyAsync(caller.a[f], h->sorted[f], h->tsize * np, cudaMemcpyDeviceToDevice, h->stream));
  dst = caller;
  if (nsteps > 0) {              // the last step's drag sums, complete, for the drag-sum output
    s = launch_drag_fold<T>(h, p, beds);
    if (s) return s;
  } else {                       // the call-start deposit's tile slots are not consumed
    k_epoch_next<<<1, 1, 0, h->stream>>>(h->epoch);
    LAUNCHED();
  }
  if ((nsteps == 0 || beds) && pc->cell && np > 0) {
    if (beds)
      k_bin_b<T><<<blocks(np, 256), 256, 0, h->stream>>>(beds, h->d_poff, h->nbeds, dst.a[0],
                                                          dst.a[1], dst.a[2], pc->cell, np);
    else
      k_bin<T><<<blocks(np, 256), 256, 0, h->stream>>>(p, dst.a[0], dst.a[1], dst.a[2], pc->cell, np);
    LAUNCHED();
  }
  h->order_on_caller = true;
  h->order_np = np;
  h->step_counter += nsteps;
  h->last_nsteps = ck ? nsteps : -1;
  if (gas) h->gas = *gas; else memset(&h->gas, 0, sizeof(h->gas));
  return MPPIC_OK;
}

// Reverse sweep over the last checkpointed mppic_step call (see mppic_backward).
// Per segment: the forward recompute of its states (keeping each state's node fields and
// height sums), then the reverse steps. Every sum is integer or a fixed tree: the gradient
// does not depend on the order in which threads run.
template <class T>
mppic_status backward_impl(mppic_handle* h, const double* dL, double* grad_out) {
  const long long np = h->ckpt_np;
  const int N = h->last_nsteps, K = h->ckpt_every;
  const size_t ts = h->tsize;
  const long long nnode = h->nnode;
  const unsigned gp = blocks(np > 0 ? np : 1, 256);
  const unsigned gc = blocks(np > 0 ? np : 1, ADJ_CHUNK);     // chunk-tile deposits
  const unsigned gn = blocks(nnode, 256);
  const long long pstride = gp > gn ? gp : gn;
  if (np > h->adj_np || h->seg_len < K || h->part_stride < pstride) {
    cudaFree(h->adj); cudaFree(h->adj_tmp); cudaFree(h->Vb); cudaFree(h->inv);
    cudaFree(h->work); cudaFree(h->seg); cudaFree(h->adj_src); cudaFree(h->fcache);
    cudaFree(h->hcache); cudaFree(h->part);
    h->adj = h->adj_tmp = h->Vb = nullptr;
    h->hcache = h->part = nullptr;
    h->inv = nullptr;
    h->work = h->seg = h->adj_src = h->fcache = nullptr;
    h->adj_np = 0; h->seg_len = 0; h->part_stride = 0;
    const size_t n1 = (size_t)(np > 0 ? np : 1);
    CU(cudaMalloc(&h->adj, ts * 6 * n1));
    CU(cudaMalloc(&h->adj_tmp, ts * 6 * n1));
    CU(cudaMalloc(&h->Vb, ts * n1));
    CU(cudaMalloc(&h->inv, sizeof(int) * n1));
    CU(cudaMalloc(&h->work, ts * 8 * n1));
    CU(cudaMalloc(&h->seg, ts * 6 * n1 * (size_t)K));
    CU(cudaMalloc(&h->adj_src, ts * 7 * n1));
    CU(cudaMalloc(&h->fcache, ts * 5 * (size_t)nnode * (size_t)K));
    CU(cudaMalloc(&h->hcache, sizeof(double) * 3 * (size_t)K));
    CU(cudaMalloc(&h->part, sizeof(double) * AP_ROWS * (size_t)pstride));
    h->adj_np = np; h->seg_len = K; h->part_stride = pstride;
  }
  if (!h->nadj) CU(cudaMalloc(&h->nadj, ts * nnode));
  if (!h->theta) CU(cudaMalloc(&h->theta, sizeof(double) * 3));
  if (!h->adj_sc) {
    CU(cudaMalloc(&h->adj_sc, sizeof(AdjScale<double>)));
    CU(cudaMemset(h->adj_sc, 0, sizeof(AdjScale<double>)));   // no parcels: zero planes
  }
  if (!h->adj_cnt) {
    CU(cudaMalloc(&h->adj_cnt, sizeof(unsigned)));
    CU(cudaMemset(h->adj_cnt, 0, sizeof(unsigned)));
  }
  {
    static bool attr = false;   // the scatter's tile exceeds the default 48 KB
    if (!attr) {
      CU(cudaFuncSetAttribute(k_adj_scatter<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)(5 * Words<T>::n * CN * sizeof(u64))));
      attr = true;
    }
  }
  cudaStream_t st = h->stream;
  CU(cudaMemsetAsync(h->theta, 0, sizeof(double) * 3, st));
  CU(cudaMemsetAsync(h->adj, 0, ts * 6 * (np > 0 ? np : 1), st));
  const KParams<T> p = make_params<T>(h, &h->gas);
  const double area = h->cfg.nx * h->cfg.dx * h->cfg.ny * h->cfg.dy;
  AdjWeights aw;
  aw.a_dp = dL[0] / N / area;
  aw.a_h = dL[1] / N;
  T* work = static_cast<T*>(h->work);
  T* wa[8];
  for (int f = 0; f < 8; ++f) wa[f] = work + (size_t)f * np;
  T* src = static_cast<T*>(h->adj_src);
  T* fc = static_cast<T*>(h->fcache);
  AdjScale<T>* sc = static_cast<AdjScale<T>*>(h->adj_sc);
  const size_t plane = sizeof(u64) * h->words * (size_t)nnode;   // one accumulator plane
  // the parameters of saved state t: its node fields in the cache
  auto at_state = [&](int t) {
    KParams<T> q = p;
    for (int f = 0; f < 5; ++f) q.fld[f] = fc + ((size_t)t * 5 + f) * nnode;
    return q;
  };
  const int nseg = (N + K - 1) / K;
  for (int sg = nseg - 1; sg >= 0; --sg) {
    const int s0 = sg * K, len = (N - s0) < K ? (N - s0) : K;
    const char* c = static_cast<const char*>(h->ckpt[sg]);
    if (np > 0) CU(cudaMemcpyAsync(work, c, ts * 8 * np, cudaMemcpyDeviceToDevice, st));
    if (sg < nseg - 1 && np > 0) {   // adjoint state from the next segment's parcel order
      const int* tag_next = reinterpret_cast<const int*>(static_cast<const char*>(h->ckpt[sg + 1]) + ts * 8 * np);
      const int* tag_this = reinterpret_cast<const int*>(c + ts * 8 * np);
      k_tag_inverse<<<gp, 256, 0, st>>>(tag_next, np, h->inv);
      k_adj_reorder<T><<<gp, 256, 0, st>>>(static_cast<T*>(h->adj), static_cast<T*>(h->adj_tmp),
                                           tag_this, h->inv, np);
      LAUNCHED();
      std::swap(h->adj, h->adj_tmp);
    }
    // recompute the segment's states S_s0 .. S_s0+len-1 with their node fields and heights
    T* seg = static_cast<T*>(h->seg);
    for (int t = 0; t < len; ++t) {
      if (np > 0)
        CU(cudaMemcpyAsync(seg + (size_t)t * 6 * np, work, ts * 6 * np, cudaMemcpyDeviceToDevice, st));
      const KParams<T> pt = at_state(t);
      CU(cudaMemsetAsync(h->acc, 0, plane, st));
      if (np > 0) {
        k_dep_simple<T><<<gc, ADJ_THREADS, 0, st>>>(pt, wa[0], wa[1], wa[2], wa[6], wa[7], np, h->part,
                                                    pstride, h->adj_cnt, h->hcache + 3 * t);
        LAUNCHED();
      } else {
        CU(cudaMemsetAsync(h->hcache + 3 * t, 0, sizeof(double) * 3, st));
      }
      mppic_status s = launch_finalize<T>(h, pt, nullptr, true);
      if (s) return s;
      if (t < len - 1 && np > 0) {
        k_push_simple<T><<<gp, 256, 0, st>>>(pt, wa[0], wa[1], wa[2], wa[3], wa[4], wa[5], wa[6],
                                             wa[7], np);
        LAUNCHED();
      }
    }
    // reverse sweep through the segment
    for (int t = len - 1; t >= 0; --t) {
      T* xs[6];
      for (int f = 0; f < 6; ++f) xs[f] = seg + ((size_t)t * 6 + f) * np;
      const KParams<T> pt = at_state(t);
      CU(cudaMemsetAsync(h->acc, 0, plane * NQ, st));
      if (np > 0) {
        k_adj_parcel<T><<<gp, 256, 0, st>>>(pt, xs[0], xs[1], xs[2], xs[3], xs[4], xs[5], wa[6], wa[7],
                                             np, static_cast<T*>(h->adj), static_cast<T*>(h->adj) + 3 * np,
                                             static_cast<T*>(h->Vb), src,
                                             h->hcache + 3 * t, aw, h->part, pstride, h->adj_cnt, sc);
        LAUNCHED();
        k_adj_scatter<T><<<gc, ADJ_THREADS, 5 * Words<T>::n * CN * sizeof(u64), st>>>(
            pt, xs[0], xs[1], xs[2], np, src, sc);
        LAUNCHED();
      }
      k_adj_node<T><<<gn, 256, 0, st>>>(pt, sc, 1.0 / p.vcell, static_cast<T*>(h->nadj), h->part,
                                        pstride);
      LAUNCHED();
      if (np > 0) {
        k_adj_deposit<T><<<gp, 256, 0, st>>>(pt, xs[0], xs[1], xs[2], wa[6], wa[7], np,
                                              static_cast<T*>(h->adj), static_cast<const T*>(h->Vb),
                                              static_cast<const T*>(h->nadj), h->part, pstride, gn,
                                              h->adj_cnt,
                                              h->theta);
      } else {
        k_adj_theta_nodes<<<1, ADJ_RED, 0, st>>>(h->part, pstride, gn, h->theta);
      }
      LAUNCHED();
    }
  }
  double th[3];
  CU(cudaMemcpyAsync(th, h->theta, sizeof(th), cudaMemcpyDeviceToHost, st));
  // the accumulators are left empty; the node arrays hold a recomputed state, so the next
  // call re-deposits and finalizes every layer
  CU(cudaMemsetAsync(h->acc, 0, plane * NQ, st));
  CU(cudaStreamSynchronize(st));
  for (int i = 0; i < 3; ++i) grad_out[i] = th[i];
  const int zr0[4] = {1 << 30, -1, 0, h->cfg.nz};
  CU(cudaMemcpy(h->zr, zr0, sizeof(zr0), cudaMemcpyHostToDevice));
  return MPPIC_OK;
}

template <class T>
mppic_status bin_impl(mppic_handle* h, mppic_parcels* pc, int do_sort) {
  const long long np = pc->np;
  PArrays<T> cur = caller_arrays<T>(pc);
  if (do_sort) {
    mppic_status s = sort_into_scratch<T>(h, pc, cur, false, h->order_on_caller && h->order_np == np);
    if (s) return s;
    if (np > 0) {
      for (int f = 0; f < 8; ++f)
        CU(cudaMemcpyAsync(cur.a[f], h->sorted[f], h->tsize * np, cudaMemcpyDeviceToDevice,
                           h->stream));
      if (pc->pid)
        CU(cudaMemcpyAsync(pc->pid, h->sorted_pid, sizeof(int) * np, cudaMemcpyDeviceToDevice,
                           h->stream));
    }
    h->order_on_caller = true;
  }
  if (np > 0 && pc->cell) {
    KParams<T> p = make_params<T>(h, nullptr);
    const KParams<T>* beds = nullptr;
    mppic_status s = upload_beds<T>(h, nullptr, &beds);
    if (s) return s;
    if (beds)
      k_bin_b<T><<<blocks(np, 256), 256, 0, h->stream>>>(beds, h->d_poff, h->nbeds, cur.a[0],
                                                          cur.a[1], cur.a[2], pc->cell, np);
    else
      k_bin<T><<<blocks(np, 256), 256, 0, h->stream>>>(p, cur.a[0], cur.a[1], cur.a[2], pc->cell, np);
    LAUNCHED();
  }
  return MPPIC_OK;
}

template <class T>
mppic_status interp_impl(mppic_handle* h, const mppic_parcels* pc, const mppic_gas* gas, void* out) {
  mppic_status s = deposit_impl<T>(h, pc, gas, nullptr, false);
  if (s) return s;
  if (pc->np > 0) {
    KParams<T> p = make_params<T>(h, gas);
    PArrays<T> cur = caller_arrays<T>(pc);
    k_interp_out<T><<<blocks(pc->np, 256), 256, 0, h->stream>>>(p, cur.a[0], cur.a[1], cur.a[2],
                                                                 static_cast<T*>(out), pc->np);
    LAUNCHED();
  }
  return MPPIC_OK;
}

template <class T>
mppic_status volume_impl(mppic_handle* h, double* Vs) {
  KParams<T> p = make_params<T>(h, nullptr);
  k_vol_out<T><<<blocks(h->nnode, 256), 256, 0, h->stream>>>(p, Vs);
  LAUNCHED();
  return MPPIC_OK;
}

template <class T>
mppic_status drag_impl(mppic_handle* h, double* A, double* Bx, double* By, double* Bz) {
  KParams<T> p = make_params<T>(h, nullptr);
  k_drag_out<T><<<blocks(h->nnode, 256), 256, 0, h->stream>>>(p, A, Bx, By, Bz);
  LAUNCHED();
  return MPPIC_OK;
}

// Everything a step call may do for the first time that is not allowed while a stream is
// being captured: scratch allocation, kernel attributes, per-bed parameter upload.
template <class T>
mppic_status prepare_capture(mppic_handle* h, const mppic_parcels* pc, const mppic_gas* gas) {
  mppic_status s = ensure_capacity(h, pc->np, pc->pid != nullptr);
  if (s) return s;
  const KParams<T>* beds = nullptr;
  s = upload_beds<T>(h, gas, &beds);
  if (s) return s;
  KParams<T> p = make_params<T>(h, gas);
  PArrays<T> none = caller_arrays<T>(pc);
  // one zero-parcel launch of each cell kernel sets its one-time attributes and occupancy
  const long long saved = h->nbricks;
  h->nbricks = 0;
  s = launch_cells<T>(h, MODE_VOLUME, p, none, none, nullptr, 0, beds);
  if (!s) s = launch_cells<T>(h, MODE_STEP, p, none, none, nullptr, 0, beds);
  if (!s) s = launch_cells<T>(h, MODE_DRAG, p, none, none, nullptr, 0, beds);
  PArrays<T> none_perm = none;                 // the instance that reads through a permutation
  none_perm.perm = reinterpret_cast<const uint32_t*>(h->cstart);
  if (!s) s = launch_cells<T>(h, MODE_STEP, p, none_perm, none, nullptr, 0, beds);
  h->nbricks = saved;
  if (s) return s;
  CU(cudaStreamSynchronize(h->stream));
  return MPPIC_OK;
}

int bits_for(long long n) {  // bits to represent values 0..n-1
  int b = 0;
  while ((1LL << b) < n) ++b;
  return b < 1 ? 1 : b;
}

}  // namespace

extern "C" {

static mppic_status check_config(const mppic_config* c, const char* what, int index) {
  mppic_handle* h = nullptr;
  if (c->nx < 1 || c->ny < 1 || c->nz < 1)
    return fail(h, MPPIC_ERR_INVALID, "%s %d: grid %dx%dx%d must be at least 1 cell per axis", what,
                index, c->nx, c->ny, c->nz);
  if (!(c->dx > 0 && c->dy > 0 && c->dz > 0 && c->dt > 0))
    return fail(h, MPPIC_ERR_INVALID, "%s %d: dx, dy, dz and dt must be positive", what, index);
  if (!(c->rho_p > 0 && c->rho_g > 0 && c->mu_g > 0))
    return fail(h, MPPIC_ERR_INVALID, "%s %d: densities and viscosity must be positive", what, index);
  if (!(c->dscale > 0)) return fail(h, MPPIC_ERR_INVALID, "%s %d: dscale must be positive", what, index);
  if (c->drag_model < MPPIC_DRAG_WEN_YU || c->drag_model > MPPIC_DRAG_GIDASPOW_BLEND)
    return fail(h, MPPIC_ERR_INVALID, "%s %d: unknown drag_model %d", what, index, c->drag_model);
  if (c->coupling_iters < 0 || c->coupling_iters > MPPIC_MAX_COUPLING_ITERS)
    return fail(h, MPPIC_ERR_INVALID, "%s %d: coupling_iters %d outside [0, %d]", what, index,
                c->coupling_iters, MPPIC_MAX_COUPLING_ITERS);
  return MPPIC_OK;
}

mppic_status mppic_create(const mppic_config* cfg, int nbeds, const long long* bed_parcel_offsets,
                          const mppic_config* per_bed, void* stream, mppic_handle** out) {
  mppic_handle* h = nullptr;
  if (!cfg || !out) return fail(h, MPPIC_ERR_INVALID, "cfg and out must not be NULL");
  *out = nullptr;
  if (nbeds < 1) return fail(h, MPPIC_ERR_INVALID, "nbeds must be >= 1");
  if (nbeds > 1 && (!bed_parcel_offsets || !per_bed))
    return fail(h, MPPIC_ERR_INVALID, "a batch needs bed_parcel_offsets and per_bed");
  if (cfg->precision != 32 && cfg->precision != 64)
    return fail(h, MPPIC_ERR_INVALID, "precision must be 32 or 64, got %d", cfg->precision);
  if (cfg->sort_every < 0) return fail(h, MPPIC_ERR_INVALID, "sort_every must be >= 0");
  if (cfg->coupling_iters < 0 || cfg->coupling_iters > MPPIC_MAX_COUPLING_ITERS)
    return fail(h, MPPIC_ERR_INVALID, "coupling_iters %d outside [0, %d]", cfg->coupling_iters,
                MPPIC_MAX_COUPLING_ITERS);
  std::vector<mppic_config> beds(nbeds);
  for (int b = 0; b < nbeds; ++b) {
    beds[b] = nbeds > 1 ? per_bed[b] : *cfg;
    mppic_status s = check_config(&beds[b], "bed", b);
    if (s) return s;
  }
  std::vector<long long> poff(nbeds + 1, 0), noff(nbeds + 1, 0), boff(nbeds + 1, 0);
  for (int b = 0; b < nbeds; ++b) {
    const mppic_config& c = beds[b];
    if (nbeds > 1) {
      poff[b + 1] = bed_parcel_offsets[b + 1];
      if (bed_parcel_offsets[0] != 0 || poff[b + 1] < bed_parcel_offsets[b])
        return fail(h, MPPIC_ERR_INVALID, "bed_parcel_offsets must start at 0 and not decrease");
    }
    noff[b + 1] = noff[b] + (long long)(c.nx + 1) * (c.ny + 1) * (c.nz + 1);
    boff[b + 1] = boff[b] + (long long)((c.nx + BX - 1) / BX) * ((c.ny + BY - 1) / BY) * ((c.nz + BZ - 1) / BZ);
  }
  const long long nnode = noff[nbeds], nbricks = boff[nbeds], nkeys = nbricks * BCELLS;
  if (nnode >= 0x7fffffffLL || nkeys >= 0x7fffffffLL || poff[nbeds] > 0x7fffffffLL)
    return fail(h, MPPIC_ERR_INVALID, "grid too large: node, key or parcel count overflows int32");
  h = new (std::nothrow) mppic_handle();
  if (!h) return fail(nullptr, MPPIC_ERR_OOM, "host allocation failed");
  h->cfg = beds[0];
  h->cfg.precision = cfg->precision;
  h->cfg.sort_every = cfg->sort_every;
  h->cfg.coupling_iters = cfg->coupling_iters;
  for (int b = 0; b < nbeds; ++b)
    if (beds[b].drag_model != MPPIC_DRAG_WEN_YU) h->drag_any = true;
  h->nbeds = nbeds;
  h->bed_cfg = beds;
  h->poff = poff; h->noff = noff; h->boff = boff;
  h->stream = static_cast<cudaStream_t>(stream);
  h->nx = h->cfg.nx; h->ny = h->cfg.ny; h->nz = h->cfg.nz;
  h->nbx = (h->nx + BX - 1) / BX; h->nby = (h->ny + BY - 1) / BY; h->nbz = (h->nz + BZ - 1) / BZ;
  h->nnode = nnode;
  h->nbricks = nbricks;
  h->nkeys = nkeys;
  h->key_bits = bits_for(nkeys);
  h->tsize = cfg->precision == 32 ? 4 : 8;
  h->words = cfg->precision == 32 ? 1 : 2;
  mppic_status s = MPPIC_OK;
  auto alloc = [&](void** ptr, size_t bytes) -> bool {
    cudaError_t e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
      s = fail(h, e == cudaErrorMemoryAllocation ? MPPIC_ERR_OOM : MPPIC_ERR_CUDA,
               "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
      return false;
    }
    return true;
  };
  if (cudaGetDevice(&h->device) != cudaSuccess) s = fail(h, MPPIC_ERR_CUDA, "no CUDA device");
  if (!s && (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
             cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
             cudaEventCreateWithFlags(&h->ev_fin, cudaEventDisableTiming) != cudaSuccess ||
             cudaEventCreateWithFlags(&h->ev_red, cudaEventDisableTiming) != cudaSuccess)) {
    cudaGetLastError();
    s = fail(h, MPPIC_ERR_CUDA, "cannot create the side stream and its events");
  }
  if (!s && cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess)
    s = fail(h, MPPIC_ERR_CUDA, "cannot read the SM count");
  if (!s && alloc((void**)&h->acc, sizeof(u64) * NQ * h->words * nnode) &&
      alloc(&h->fld, h->tsize * 5 * nnode) && alloc((void**)&h->cstart, sizeof(int) * (nkeys + 1)) &&
      alloc((void**)&h->obj_part, sizeof(double) * 3 * (nbricks > 0 ? nbricks : 1)) &&
      alloc((void**)&h->obj_tmp, sizeof(double) * 2 * nbeds) && alloc((void**)&h->errs, sizeof(int)) &&
      alloc((void**)&h->zr, sizeof(int) * 4) && alloc((void**)&h->wq, sizeof(unsigned long long)) &&
      alloc((void**)&h->totals, sizeof(uint32_t) * 256) &&
      alloc((void**)&h->cellmap, (size_t)BCELLS * (nbricks > 0 ? nbricks : 1)) &&
      alloc((void**)&h->bacc, sizeof(u64) * NQ * h->words * TNODES * (nbricks > 0 ? nbricks : 1)) &&
      alloc((void**)&h->bstamp, sizeof(int) * (nbricks > 0 ? nbricks : 1)) &&
      alloc((void**)&h->epoch, sizeof(int)) &&
      alloc((void**)&h->obj_slices, sizeof(double) * 3 * OBJ_BLOCKS) &&
      alloc((void**)&h->obj_count, sizeof(unsigned)) &&
      alloc((void**)&h->bgeo, sizeof(int4) * (nbricks > 0 ? nbricks : 1)) &&
      alloc((void**)&h->rs_cnt, sizeof(uint32_t) * NSLOT * (nbricks > 0 ? nbricks : 1)) &&
      alloc((void**)&h->rs_off, sizeof(uint32_t) * NSLOT * (nbricks > 0 ? nbricks : 1)) &&
      alloc((void**)&h->rs_wcnt, sizeof(uint32_t) * NSLOT * RS_NW * (nbricks > 0 ? nbricks : 1)) &&
      alloc((void**)&h->rs_far, sizeof(int) * (nbricks > 0 ? nbricks : 1)) &&
      alloc((void**)&h->rs_far_next, sizeof(int) * (nbricks > 0 ? nbricks : 1)) &&
      alloc((void**)&h->rs_count, sizeof(int) * (nbricks > 0 ? nbricks : 1)) &&
      alloc((void**)&h->rs_start, sizeof(int) * (nbricks > 0 ? nbricks : 1)) &&
      alloc((void**)&h->rs_part, sizeof(int) * (nbricks / RS_THREADS + 1))) {
    cudaError_t e = cudaMemsetAsync(h->acc, 0, sizeof(u64) * NQ * h->words * nnode, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->obj_count, 0, sizeof(unsigned), h->stream);
    // no tile slot is valid yet: stamps -1, epoch 0
    if (e == cudaSuccess) e = cudaMemsetAsync(h->bstamp, 0xff, sizeof(int) * (nbricks > 0 ? nbricks : 1), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->epoch, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) {                      // the natural pair map until the first sort
      std::vector<uint8_t> id((size_t)BCELLS * (nbricks > 0 ? nbricks : 1));
      for (size_t i = 0; i < id.size(); ++i) id[i] = (uint8_t)(i % BCELLS < CT ? i % BCELLS + CT : 0);
      e = cudaMemcpy(h->cellmap, id.data(), id.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && nbricks > 0) {       // brick geometry for the local re-sort
      std::vector<int4> geo((size_t)nbricks);
      for (int b = 0; b < nbeds; ++b) {
        const int nbx = (beds[b].nx + BX - 1) / BX, nby = (beds[b].ny + BY - 1) / BY,
                  nbz = (beds[b].nz + BZ - 1) / BZ;
        for (long long g = boff[b]; g < boff[b + 1]; ++g)
          geo[(size_t)g] = make_int4((int)boff[b], nbx, nby, nbz);
      }
      e = cudaMemcpy(h->bgeo, geo.data(), sizeof(int4) * geo.size(), cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(h->errs, 0, sizeof(int), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(h->fld, 0, h->tsize * 5 * nnode, h->stream);
    // no deposit yet; the first finalize covers every layer
    const int zr0[4] = {1 << 30, -1, 0, h->cfg.nz};
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->zr, zr0, sizeof(zr0), cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess && nbeds > 1) {
      std::vector<int> brick_bed(nbricks);
      std::vector<double> area(nbeds);
      for (int b = 0; b < nbeds; ++b) {
        for (long long g = boff[b]; g < boff[b + 1]; ++g) brick_bed[g] = b;
        area[b] = beds[b].nx * beds[b].dx * beds[b].ny * beds[b].dy;
      }
      if (!alloc((void**)&h->d_poff, sizeof(long long) * (nbeds + 1)) ||
          !alloc((void**)&h->d_noff, sizeof(long long) * (nbeds + 1)) ||
          !alloc((void**)&h->d_boff, sizeof(long long) * (nbeds + 1)) ||
          !alloc((void**)&h->d_brick_bed, sizeof(int) * (nbricks > 0 ? nbricks : 1)) ||
          !alloc((void**)&h->d_area, sizeof(double) * nbeds)) {
        e = cudaErrorMemoryAllocation;
      } else {
        e = cudaMemcpy(h->d_poff, poff.data(), sizeof(long long) * (nbeds + 1), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(h->d_noff, noff.data(), sizeof(long long) * (nbeds + 1), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(h->d_boff, boff.data(), sizeof(long long) * (nbeds + 1), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(h->d_brick_bed, brick_bed.data(), sizeof(int) * nbricks, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(h->d_area, area.data(), sizeof(double) * nbeds, cudaMemcpyHostToDevice);
      }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess && !s) s = fail(h, MPPIC_ERR_CUDA, "create: %s", cudaGetErrorString(e));
  }
  if (s) {
    snprintf(g_create_err, sizeof(g_create_err), "%s", h->err);
    mppic_destroy(h);
    return s;
  }
  *out = h;
  return MPPIC_OK;
}

mppic_status mppic_tune(mppic_handle* h, int grid_per_sm, int sort_every) {
  if (!h) return fail(h, MPPIC_ERR_INVALID, "handle is NULL");
  if (grid_per_sm < 0 || grid_per_sm > 64) return fail(h, MPPIC_ERR_INVALID, "grid_per_sm out of range");
  h->grid_factor = grid_per_sm;
  if (sort_every >= 0) h->cfg.sort_every = sort_every;
  if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; h->gkey.clear(); }
  return MPPIC_OK;
}

mppic_status mppic_bin(mppic_handle* h, mppic_parcels* parcels, int do_sort) {
  if (!h) return fail(h, MPPIC_ERR_INVALID, "handle is NULL");
  mppic_status s = check_parcels(h, parcels);
  if (s) return s;
  return h->cfg.precision == 32 ? bin_impl<float>(h, parcels, do_sort)
                                : bin_impl<double>(h, parcels, do_sort);
}

mppic_status mppic_deposit(mppic_handle* h, const mppic_parcels* parcels, const mppic_gas* gas,
                           double* Vs_out, void* fields_out) {
  if (!h) return fail(h, MPPIC_ERR_INVALID, "handle is NULL");
  if (h->nbeds > 1) return fail(h, MPPIC_ERR_INVALID, "mppic_deposit takes a single-bed handle");
  mppic_status s = check_parcels(h, parcels);
  if (s) return s;
  const bool full = Vs_out != nullptr || fields_out != nullptr;
  s = h->cfg.precision == 32 ? deposit_impl<float>(h, parcels, gas, Vs_out, full)
                             : deposit_impl<double>(h, parcels, gas, Vs_out, full);
  if (s) return s;
  if (fields_out)
    CU(cudaMemcpyAsync(fields_out, h->fld, h->tsize * 5 * h->nnode, cudaMemcpyDeviceToDevice,
                       h->stream));
  return MPPIC_OK;
}

mppic_status mppic_interp(mppic_handle* h, const mppic_parcels* parcels, const mppic_gas* gas,
                          void* out) {
  if (!h) return fail(h, MPPIC_ERR_INVALID, "handle is NULL");
  if (h->nbeds > 1) return fail(h, MPPIC_ERR_INVALID, "mppic_interp takes a single-bed handle");
  mppic_status s = check_parcels(h, parcels);
  if (s) return s;
  if (!out && parcels->np > 0) return fail(h, MPPIC_ERR_INVALID, "out is NULL");
  return h->cfg.precision == 32 ? interp_impl<float>(h, parcels, gas, out)
                                : interp_impl<double>(h, parcels, gas, out);
}

mppic_status mppic_step(mppic_handle* h, mppic_parcels* parcels, const mppic_gas* gas, int nsteps,
                        double* obj_out) {
  if (!h) return fail(h, MPPIC_ERR_INVALID, "handle is NULL");
  mppic_status s = check_parcels(h, parcels);
  if (s) return s;
  if (h->nbeds > 1 && parcels->np != h->poff[h->nbeds])
    return fail(h, MPPIC_ERR_INVALID, "np=%lld does not match the batch's %lld parcels", parcels->np,
                h->poff[h->nbeds]);
  if (nsteps < 0) return fail(h, MPPIC_ERR_INVALID, "nsteps must be >= 0");
  return h->cfg.precision == 32 ? step_impl<float>(h, parcels, gas, nsteps, obj_out)
                                : step_impl<double>(h, parcels, gas, nsteps, obj_out);
}

mppic_status mppic_step_graph(mppic_handle* h, mppic_parcels* parcels, const mppic_gas* gas,
                              int nsteps, double* obj_out) {
  if (!h) return fail(h, MPPIC_ERR_INVALID, "handle is NULL");
  mppic_status s = check_parcels(h, parcels);
  if (s) return s;
  if (nsteps < 1) return fail(h, MPPIC_ERR_INVALID, "nsteps must be >= 1");
  if (h->ckpt_every > 0) return fail(h, MPPIC_ERR_INVALID, "mppic_step_graph does not checkpoint");
  if (h->nbeds > 1 && parcels->np != h->poff[h->nbeds])
    return fail(h, MPPIC_ERR_INVALID, "np=%lld does not match the batch's %lld parcels", parcels->np,
                h->poff[h->nbeds]);
  std::vector<const void*> key = {parcels->x, parcels->y, parcels->z, parcels->u, parcels->v,
                                  parcels->w, parcels->d, parcels->omega, parcels->cell,
                                  parcels->pid, (const void*)(intptr_t)parcels->np,
                                  (const void*)(intptr_t)nsteps, obj_out};
  for (int a = 0; a < 3; ++a) {
    key.push_back(gas ? gas->U[a] : nullptr);
    key.push_back(gas ? gas->gradp[a] : nullptr);
  }
  if (!h->gexec || key != h->gkey) {
    if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; h->gkey.clear(); }
    s = h->cfg.precision == 32 ? prepare_capture<float>(h, parcels, gas)
                               : prepare_capture<double>(h, parcels, gas);
    if (s) return s;
    if (!h->cap_stream) CU(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
    const bool prof = h->prof;
    cudaStream_t user = h->stream;
    h->prof = false;
    h->stream = h->cap_stream;               // capture the sequence on the handle's own stream
    cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
      h->stream = user; h->prof = prof; cudaGetLastError();
      return fail(h, MPPIC_ERR_CUDA, "begin capture: %s", cudaGetErrorString(e));
    }
    s = h->cfg.precision == 32 ? step_impl<float>(h, parcels, gas, nsteps, obj_out)
                               : step_impl<double>(h, parcels, gas, nsteps, obj_out);
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(h->cap_stream, &graph);
    h->stream = user;
    h->prof = prof;
    if (e != cudaSuccess) cudaGetLastError();
    if (s) { if (graph) cudaGraphDestroy(graph); return s; }
    if (e != cudaSuccess) return fail(h, MPPIC_ERR_CUDA, "stream capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiate(&h->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      h->gexec = nullptr;
      cudaGetLastError();
      return fail(h, MPPIC_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    h->gkey = key;
  }
  CU(cudaGraphLaunch(h->gexec, h->stream));
  return MPPIC_OK;
}

mppic_status mppic_set_params(mppic_handle* h, double drag_mult, double dscale, double u_in) {
  if (!h) return fail(h, MPPIC_ERR_INVALID, "handle is NULL");
  if (h->nbeds > 1) return fail(h, MPPIC_ERR_INVALID, "mppic_set_params takes a single-bed handle");
  if (!(dscale > 0)) return fail(h, MPPIC_ERR_INVALID, "dscale must be positive");
  h->cfg.drag_mult = drag_mult;
  h->cfg.dscale = dscale;
  h->cfg.u_in = u_in;
  if (h->gexec) { cudaGraphExecDestroy(h->gexec); h->gexec = nullptr; h->gkey.clear(); }
  return MPPIC_OK;
}

mppic_status mppic_checkpoint(mppic_handle* h, int every) {
  if (!h) return fail(h, MPPIC_ERR_INVALID, "handle is NULL");
  if (h->nbeds > 1 && every != 0)
    return fail(h, MPPIC_ERR_INVALID, "checkpointing takes a single-bed handle");
  if (every < 0) return fail(h, MPPIC_ERR_INVALID, "every must be >= 0");
  if (every > 0 && (h->drag_any || h->cfg.coupling_iters > 0))
    return fail(h, MPPIC_ERR_INVALID,
                "reverse mode differentiates explicit coupling with Wen-Yu drag only");
  h->ckpt_every = every;
  h->last_nsteps = -1;
  return MPPIC_OK;
}

mppic_status mppic_backward(mppic_handle* h, const double* dL_d_dP_H, double* grad_out) {
  if (!h) return fail(h, MPPIC_ERR_INVALID, "handle is NULL");
  if (!dL_d_dP_H || !grad_out) return fail(h, MPPIC_ERR_INVALID, "dL and grad_out must not be NULL");
  if (h->ckpt_every <= 0 || h->last_nsteps <= 0)
    return fail(h, MPPIC_ERR_INVALID,
                "no checkpointed mppic_step call to differentiate (call mppic_checkpoint first)");
  return h->cfg.precision == 32 ? backward_impl<float>(h, dL_d_dP_H, grad_out)
                                : backward_impl<double>(h, dL_d_dP_H, grad_out);
}

mppic_status mppic_drag_sums(mppic_handle* h, double* A, double* Bx, double* By, double* Bz) {
  if (!h) return fail(h, MPPIC_ERR_INVALID, "handle is NULL");
  if (h->nbeds > 1) return fail(h, MPPIC_ERR_INVALID, "mppic_drag_sums takes a single-bed handle");
  return h->cfg.precision == 32 ? drag_impl<float>(h, A, Bx, By, Bz)
                                : drag_impl<double>(h, A, Bx, By, Bz);
}

mppic_status mppic_step_volume(mppic_handle* h, double* Vs_out) {
  if (!h) return fail(h, MPPIC_ERR_INVALID, "handle is NULL");
  if (h->nbeds > 1) return fail(h, MPPIC_ERR_INVALID, "mppic_step_volume takes a single-bed handle");
  if (!Vs_out) return fail(h, MPPIC_ERR_INVALID, "Vs_out is NULL");
  if (h->step_counter == 0) return fail(h, MPPIC_ERR_INVALID, "no mppic_step call yet");
  return h->cfg.precision == 32 ? volume_impl<float>(h, Vs_out) : volume_impl<double>(h, Vs_out);
}

mppic_status mppic_check(mppic_handle* h) {
  if (!h) return fail(h, MPPIC_ERR_INVALID, "handle is NULL");
  CU(cudaStreamSynchronize(h->stream));
  int flags = 0;
  CU(cudaMemcpy(&flags, h->errs, sizeof(int), cudaMemcpyDeviceToHost));
  CU(cudaMemset(h->errs, 0, sizeof(int)));
  if (flags & ERR_TIMEOUT) return fail(h, MPPIC_ERR_TIMEOUT, "a bounded device wait gave up");
  if (flags & ERR_RANGE) return fail(h, MPPIC_ERR_RANGE, "a fixed-point accumulator left its range");
  if (flags & ERR_DOMAIN)
    return fail(h, MPPIC_ERR_DOMAIN, "a parcel left the box after reflection or became non-finite");
  return MPPIC_OK;
}

mppic_status mppic_profile_enable(mppic_handle* h, int enable) {
  if (!h) return fail(h, MPPIC_ERR_INVALID, "handle is NULL");
  CU(cudaStreamSynchronize(h->stream));
  h->prof = enable != 0;
  h->ev_used = 0;
  for (int i = 0; i < NPHASE; ++i) h->launches[i] = 0;
  h->total_launches = 0;
  return MPPIC_OK;
}

mppic_status mppic_profile_read(mppic_handle* h, mppic_profile* out) {
  if (!h || !out) return fail(h, MPPIC_ERR_INVALID, "handle and out must not be NULL");
  CU(cudaStreamSynchronize(h->stream));
  memset(out, 0, sizeof(*out));
  for (size_t i = 0; i < h->ev_used; ++i) {
    float ms = 0;
    CU(cudaEventElapsedTime(&ms, h->ev[2 * i], h->ev[2 * i + 1]));
    out->ms[h->ev_phase[i]] += ms;
  }
  for (int i = 0; i < NPHASE; ++i) out->launches[i] = h->launches[i];
  out->total_launches = h->total_launches;
  out->parcels = h->order_np > 0 ? h->order_np : 0;
  if (h->nbricks > 0) {
    unsigned long long* cnt = nullptr;
    CU(cudaMalloc(&cnt, sizeof(unsigned long long)));
    CU(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), h->stream));
    k_count_bricks<<<blocks(h->nbricks, 256), 256, 0, h->stream>>>(h->cstart, h->nbricks, cnt);
    unsigned long long c = 0;
    cudaError_t e = cudaMemcpyAsync(&c, cnt, sizeof(c), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    cudaFree(cnt);
    if (e != cudaSuccess) return fail(h, MPPIC_ERR_CUDA, "profile read: %s", cudaGetErrorString(e));
    out->active_bricks = (long long)c;
  }
  return MPPIC_OK;
}

long long mppic_num_nodes(const mppic_handle* h) { return h ? h->nnode : 0; }

void mppic_destroy(mppic_handle* h) {
  if (!h) return;
  cudaFree(h->acc); cudaFree(h->fld); cudaFree(h->cstart); cudaFree(h->obj_part);
  cudaFree(h->obj_tmp); cudaFree(h->errs); cudaFree(h->zr); cudaFree(h->totals); cudaFree(h->hist);
  cudaFree(h->obj_slices); cudaFree(h->obj_count); cudaFree(h->cellmap);
  cudaFree(h->bacc); cudaFree(h->bstamp); cudaFree(h->epoch);
  for (int i = 0; i < 2; ++i) { cudaFree(h->keys[i]); cudaFree(h->vals[i]); cudaFree(h->bcell[i]); }
  cudaFree(h->bgeo); cudaFree(h->rs_cnt); cudaFree(h->rs_off); cudaFree(h->rs_wcnt); cudaFree(h->rs_far);
  cudaFree(h->rs_far_next); cudaFree(h->rs_count); cudaFree(h->rs_start); cudaFree(h->rs_part);
  for (int f = 0; f < 8; ++f) cudaFree(h->sorted[f]);
  cudaFree(h->sorted_pid);
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  cudaFree(h->tag); cudaFree(h->sorted_tag); cudaFree(h->lperm);
  for (void* c : h->ckpt) cudaFree(c);
  cudaFree(h->adj); cudaFree(h->adj_tmp); cudaFree(h->Vb); cudaFree(h->nadj); cudaFree(h->inv);
  cudaFree(h->work); cudaFree(h->seg); cudaFree(h->theta); cudaFree(h->adj_src);
  cudaFree(h->fcache); cudaFree(h->hcache); cudaFree(h->part); cudaFree(h->adj_sc);
  cudaFree(h->adj_cnt);
  cudaFree(h->d_poff); cudaFree(h->d_noff); cudaFree(h->d_boff); cudaFree(h->d_brick_bed);
  cudaFree(h->d_area); cudaFree(h->d_beds); cudaFree(h->wq);
  if (h->gexec) cudaGraphExecDestroy(h->gexec);
  if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_fin) cudaEventDestroy(h->ev_fin);
  if (h->ev_red) cudaEventDestroy(h->ev_red);
  delete h;
}

const char* mppic_last_error(const mppic_handle* h) { return h ? h->err : g_create_err; }

}  // extern "C"

// ------------------------------------------------------------------------------
// Allocation-free solids-volume deposit (mppic_deposit_static).
//
// Its scratch is a file-scope device array, so the entry point never calls cudaMalloc,
// cudaFree or an allocating library routine. Host code cannot use the array's name as a
// device address (it names a host-side shadow), so the device address is looked up with
// cudaGetSymbolAddress, with the device current, and passed to the kernels.

namespace {

constexpr int kStaticWords = 2;                       // FP64 form needs two words per node
static __device__ __align__(256) unsigned long long
    g_static_scratch[MPPIC_STATIC_MAX_NODES * kStaticWords + 32];  // + one slot for flags

constexpr int kMaxDevices = 64;
// The address looked up on each device, for calls made while a stream is being captured
// (a lookup is not made then). Atomic: host threads may call concurrently.
static std::atomic<void*> g_static_addr[kMaxDevices];

// Each parcel adds its 8 fixed-point corner contributions to the static accumulator. FP32
// form: the corner with the largest weight adds the parcel's exact volume minus the other
// seven, so that the corners add up to exactly the parcel's volume. A position outside the
// box or not finite, or a value out of the fixed-point range, sets a flag (the output is
// then NaN); such a parcel is clamped into the edge cells for its deposit.
template <class T>
__global__ void k_deposit_static(KParams<T> p, const T* __restrict__ x, const T* __restrict__ y,
                                 const T* __restrict__ z, const T* __restrict__ d,
                                 const T* __restrict__ om, long long np, u64* acc) {
  constexpr int W = Words<T>::n;
  long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (q >= np) return;
  const T pos[3] = {x[q], y[q], z[q]};
  for (int a = 0; a < 3; ++a)
    if (!(pos[a] >= T(0) && pos[a] <= p.L[a])) atomicOr(p.errs, ERR_DOMAIN);
  Cell3<T> c;
  bin3(p, pos[0], pos[1], pos[2], c);
  T dq = d[q];
  T V = om[q] * (dq * dq * dq) * p.vcoef;
  T w[3][2];
  for (int a = 0; a < 3; ++a) { w[a][0] = T(1) - c.xi[a]; w[a][1] = c.xi[a]; }
  const int kst = (c.xi[0] >= T(0.5) ? 1 : 0) + (c.xi[1] >= T(0.5) ? 2 : 0) + (c.xi[2] >= T(0.5) ? 4 : 0);
  long long rest = 0;
  if (W == 1) {
    u64 tot[W];
    to_fixed(V, p.mV, tot, p.errs);
    rest = (long long)tot[0];
  }
  for (int cc = 0; cc < 2; ++cc)
    for (int b = 0; b < 2; ++b)
      for (int a = 0; a < 2; ++a) {
        const int k = a + 2 * b + 4 * cc;
        if (W == 1 && k == kst) continue;
        u64 fx[W];
        to_fixed(V * ((w[0][a] * w[1][b]) * w[2][cc]), p.mV, fx, p.errs);
        if (W == 1) rest -= (long long)fx[0];
        acc_add(acc + node_id(p, c.i + a, c.j + b, c.k + cc), p.nnode, fx);  // single bed
      }
  if (W == 1) {
    u64 fx[W];
    fx[0] = (u64)rest;
    acc_add(acc + node_id(p, c.i + (kst & 1), c.j + ((kst >> 1) & 1), c.k + (kst >> 2)), p.nnode, fx);
  }
}

// The accumulator as doubles; every output is NaN if a parcel raised a flag.
template <class T>
__global__ void k_static_out(const u64* __restrict__ acc, const int* __restrict__ errs,
                             long long nnode, double inv_m, double* __restrict__ out) {
  constexpr int W = Words<T>::n;
  long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (n >= nnode) return;
  if (*errs) { out[n] = __longlong_as_double(0x7ff8000000000000ll); return; }
  u64 fx[W];
  for (int w = 0; w < W; ++w) fx[w] = acc[(long long)w * nnode + n];
  out[n] = from_fixed(fx, inv_m);
}

template <class T>
mppic_status deposit_static_impl(const mppic_config* c, const mppic_parcels* pc, double* Vs_out,
                                 cudaStream_t st, u64* base) {
  mppic_handle* h = nullptr;  // errors go to the creation message buffer
  KParams<T> p;
  memset(&p, 0, sizeof(p));
  p.nx = c->nx; p.ny = c->ny; p.nz = c->nz;
  p.nnode = (long long)(c->nx + 1) * (c->ny + 1) * (c->nz + 1);
  p.nstride = p.nnode;
  const double hs[3] = {c->dx, c->dy, c->dz};
  const int ns[3] = {c->nx, c->ny, c->nz};
  for (int a = 0; a < 3; ++a) {
    p.inv_d[a] = 1.0 / hs[a];
    p.inv_f[a] = (float)p.inv_d[a];
    p.inv_lo[a] = (float)(p.inv_d[a] - (double)p.inv_f[a]);
    p.L[a] = (T)(ns[a] * hs[a]);
  }
  p.vcoef = (T)(M_PI / 6.0 * c->dscale * c->dscale * c->dscale);
  fixed_units(*c, sizeof(T), &p.mV, &p.mA);
  u64* acc = base + 32;                         // the first 256 bytes hold the flag word
  p.errs = reinterpret_cast<int*>(base);
  CU(cudaMemsetAsync(base, 0, sizeof(u64) * (32 + (size_t)Words<T>::n * p.nnode), st));
  if (pc->np > 0) {
    k_deposit_static<T><<<blocks(pc->np, 256), 256, 0, st>>>(
        p, static_cast<const T*>(pc->x), static_cast<const T*>(pc->y),
        static_cast<const T*>(pc->z), static_cast<const T*>(pc->d),
        static_cast<const T*>(pc->omega), pc->np, acc);
    LAUNCHED();
  }
  k_static_out<T><<<blocks(p.nnode, 256), 256, 0, st>>>(acc, p.errs, p.nnode, 1.0 / (double)p.mV,
                                                       Vs_out);
  LAUNCHED();
  return MPPIC_OK;
}

}  // namespace

extern "C" mppic_status mppic_deposit_static(const mppic_config* cfg, const mppic_parcels* parcels,
                                             double* Vs_out, void* stream) {
  mppic_handle* h = nullptr;
  if (!cfg || !parcels || !Vs_out)
    return fail(h, MPPIC_ERR_INVALID, "cfg, parcels and Vs_out must not be NULL");
  if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1 || !(cfg->dx > 0 && cfg->dy > 0 && cfg->dz > 0))
    return fail(h, MPPIC_ERR_INVALID, "grid and spacing must be positive");
  if (!(cfg->dscale > 0)) return fail(h, MPPIC_ERR_INVALID, "dscale must be positive");
  if (cfg->precision != 32 && cfg->precision != 64)
    return fail(h, MPPIC_ERR_INVALID, "precision must be 32 or 64, got %d", cfg->precision);
  const long long nnode = (long long)(cfg->nx + 1) * (cfg->ny + 1) * (cfg->nz + 1);
  if (nnode > MPPIC_STATIC_MAX_NODES)
    return fail(h, MPPIC_ERR_INVALID,
                "mppic_deposit_static: %lld nodes exceed the static scratch limit of %d nodes",
                nnode, MPPIC_STATIC_MAX_NODES);
  if (parcels->np < 0 || parcels->np > 0x7fffffffLL)
    return fail(h, MPPIC_ERR_INVALID, "np=%lld out of range", parcels->np);
  if (parcels->np > 0 && (!parcels->x || !parcels->y || !parcels->z || !parcels->d || !parcels->omega))
    return fail(h, MPPIC_ERR_INVALID, "x, y, z, d and omega must not be NULL");
  int dev = 0;
  CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(h, MPPIC_ERR_INVALID, "device %d unsupported", dev);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // Outside stream capture the address is looked up on every call (cheap, allocates nothing),
  // so a device reset or a re-created context cannot leave a stale one; during capture the
  // last address looked up on this device is used.
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  CU(cudaStreamIsCapturing(st, &cap));
  void* addr = nullptr;
  if (cap == cudaStreamCaptureStatusNone) {
    CU(cudaGetSymbolAddress(&addr, g_static_scratch));
    g_static_addr[dev].store(addr);
  } else {
    addr = g_static_addr[dev].load();
    if (!addr)
      return fail(h, MPPIC_ERR_INVALID,
                  "mppic_deposit_static: make a first call on this device outside stream capture");
  }
  u64* base = static_cast<u64*>(addr);
  return cfg->precision == 32 ? deposit_static_impl<float>(cfg, parcels, Vs_out, st, base)
                              : deposit_static_impl<double>(cfg, parcels, Vs_out, st, base);
}
