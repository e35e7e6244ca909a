/*
 * mppic.h - C ABI of libmppic, the GB300 (sm_103a) MP-PIC parcel-grid coupling step.
 *
 * The library advances the parcel side of the multiphase particle-in-cell model of
 * Woo et al., "Development of an Equation-based Parallelization Method for Multiphase
 * Particle-in-Cell Simulations" (arXiv 2211.15605), Sec. 2.1:
 *   Eq. 3   dx_P/dt = u_P
 *   Eq. 4   eps_P rho_P du_P/dt = -eps_P grad p + F_P + eps_P rho_P g - grad tau_P
 *   Eq. 5   tau_P = p_s eps_P^beta / max[eps_CP - eps_P, alpha (1 - eps_P)]
 * with the parcel volume V = w * V_particle (Sec. 2.1) and the drag force F of Eq. 2
 * deposited back to the mesh (Sec. 2.1, explicit coupling of Sec. 2.2.2).
 * The gas is prescribed (no SIMPLE solve). Drag is Wen-Yu, Syamlal-O'Brien (the paper's
 * closure, Sec. 2.1), Gidaspow or the Gidaspow blend; interpolation is trilinear
 * cloud-in-cell on the node grid; walls reflect specularly at the parcel centre. Coupling is
 * explicit or implicit (Sec. 2.2.2: F once per step, or again at the head of every gas
 * iteration).
 *
 * Geometry: box [0, nx*dx] x [0, ny*dy] x [0, nz*dz]. Cells (i,j,k), 0 <= i < nx, with
 * row-major id i + nx*(j + ny*k). Nodes (i,j,k), 0 <= i <= nx, with index
 * i + (nx+1)*(j + (ny+1)*k). Node control volume = dx*dy*dz halved once per axis on
 * which the node lies on a boundary plane.
 *
 * Conventions for every call:
 *   - Array pointers are DEVICE pointers owned by the caller unless stated otherwise.
 *     Parcel and node arrays hold float (precision 32) or double (precision 64).
 *   - Calls are asynchronous on the stream given to mppic_create. A call returns after
 *     enqueuing its work; host-side argument errors are returned at once.
 *   - Errors detected on the device (a parcel still outside the box after reflection,
 *     a non-finite value, a fixed-point accumulator out of range) never trap: they set
 *     a flag that mppic_check() returns at the next synchronisation.
 *   - No exception crosses the ABI. mppic_last_error() describes the last failure.
 *   - The handle owns all scratch (sort buffers, fixed-point accumulators, node fields,
 *     objective partials); it is freed by mppic_destroy.
 */
#ifndef MPPIC_H
#define MPPIC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mppic_handle mppic_handle;

typedef enum {
  MPPIC_OK = 0,
  MPPIC_ERR_INVALID = 1,  /* bad argument or configuration (host check) */
  MPPIC_ERR_CUDA = 2,     /* a CUDA runtime call failed */
  MPPIC_ERR_OOM = 3,      /* device allocation failed */
  MPPIC_ERR_DOMAIN = 4,   /* a parcel left the box after reflection, or a value became non-finite */
  MPPIC_ERR_TIMEOUT = 5,  /* a bounded device wait gave up (reserved: the current kernels
                             have no spin-waits) */
  MPPIC_ERR_RANGE = 6     /* a fixed-point node accumulator exceeded its range */
} mppic_status;

/* Drag closures (mppic_config.drag_model), each as the acceleration coefficient D of
 * F_P / (eps_P rho_P) = D (u_G - u_P) with slip s = u_G - u_P, Re = rho_G d |s| / mu and the
 * voidage eps_g = max(1 - eps_P, eps_g_min):
 *   WEN_YU           D = C 3/4 Cd rho_G |s| eps_g^-1.65 / (d rho_P), Cd = 24/Re_m (1 + 0.15
 *                    Re_m^0.687) below Re_m = eps_g Re = 1000, else 0.44;
 *   SYAMLAL_OBRIEN   the paper's closure (Sec. 2.1): D = C 3/4 C_D eps_g rho_G |s| / (V_r^2 d
 *                    rho_P), Dallavalle's C_D = (0.63 + 4.8 sqrt(V_r / Re))^2, and the velocity
 *                    ratio V_r of A = eps_g^4.14, B = 0.8 eps_g^1.28 (eps_g <= 0.85) or
 *                    eps_g^2.65;
 *   GIDASPOW         Ergun, D = C (150 eps_s mu / (eps_g d^2) + 1.75 rho_G |s| / d) / rho_P with
 *                    eps_s = 1 - eps_g, below eps_g = 0.8; Wen-Yu at and above;
 *   GIDASPOW_BLEND   (1 - phi) Ergun + phi Wen-Yu, phi = atan(262.5 (0.2 - eps_s)) / pi + 1/2.
 * The paper names only Syamlal-O'Brien; the formulas are the published forms of the MFiX
 * theory guide that it defers to. */
#define MPPIC_DRAG_WEN_YU 0
#define MPPIC_DRAG_SYAMLAL_OBRIEN 1
#define MPPIC_DRAG_GIDASPOW 2
#define MPPIC_DRAG_GIDASPOW_BLEND 3

/* Largest number of gas iterations per step of implicit coupling. */
#define MPPIC_MAX_COUPLING_ITERS 64

/* Parameters of one bed. Paper symbols in brackets. */
typedef struct {
  int nx, ny, nz;        /* cells per axis */
  int precision;         /* 32: FP32 parcel state, interp, drag and push (deposits stay exact
                            fixed point); 64: FP64 throughout */
  double dx, dy, dz;     /* cell size [m] */
  double rho_g, mu_g;    /* gas density [rho_G], viscosity */
  double g[3];           /* gravity [g] */
  double gradp[3];       /* uniform pressure gradient [grad p], used when mppic_gas has none */
  double rho_p;          /* parcel material density [rho_P] */
  double Ps, beta, eps_cp, alpha; /* Eq. 5 [p_s, beta, eps_CP, alpha] */
  double eps_g_min;      /* voidage floor for u_g = U / eps_g and for the drag */
  double e_wall;         /* wall restitution of the specular reflection */
  double drag_mult;      /* C: multiplies the drag coefficient */
  double dscale;         /* s_d: multiplies every parcel diameter */
  double u_in;           /* added to the z superficial gas velocity at every node */
  double dt;             /* time step [s] */
  int sort_every;        /* mppic_step sorts parcels by cell every this many steps;
                            0 = only when the handle has no valid order */
  int drag_model;        /* MPPIC_DRAG_*; in a batch each bed has its own */
  int coupling_iters;    /* 0: explicit coupling (Sec. 2.2.2: the drag force F is deposited once
                            per step, from the state before the push); K in [1,
                            MPPIC_MAX_COUPLING_ITERS]: implicit coupling with K gas iterations
                            per step (see mppic_step); in a batch taken from cfg for all beds */
  int reserved;
} mppic_config;

/* Parcel state, structure of arrays, np entries each (caller-owned device memory).
 * x,y,z,u,v,w,d,omega are float or double per the precision. cell receives the row-major
 * cell id of each parcel's current position. Sorting permutes every array together;
 * pid (optional, may be NULL) lets the caller follow parcel identity through sorts.
 * The eight value arrays must start on 16-byte boundaries (as cudaMalloc and PyTorch
 * allocations do); calls with unaligned arrays return MPPIC_ERR_INVALID. */
typedef struct {
  void *x, *y, *z, *u, *v, *w, *d, *omega;
  int32_t *cell;
  int32_t *pid;
  long long np;
} mppic_parcels;

/* Prescribed gas at the nodes (caller-owned device arrays of (nx+1)(ny+1)(nz+1) values in
 * the parcel precision). U is the superficial velocity before u_in is added; a NULL
 * component is zero. gradp all NULL means the uniform gradient of the config. */
typedef struct {
  const void *U[3];
  const void *gradp[3];
} mppic_gas;

/* Create a handle for one bed (nbeds = 1; bed_parcel_offsets and per_bed may be NULL) or
 * for a batch of nbeds independent beds advanced together. Sec. 2.2.1: the paper passes the
 * model parameters to the solver once at initialisation and afterwards only the time step
 * crosses the boundary; here the parameters are fixed at creation (mppic_set_params and
 * mppic_tune change the few that a caller varies) and the step calls carry only device
 * pointers and a step count. For a batch:
 *   - per_bed (host, nbeds configs) gives each bed's grid and physics; precision and
 *     sort_every come from cfg;
 *   - bed_parcel_offsets (host, nbeds+1, starting at 0) gives each bed's parcel range in
 *     the one concatenated set of parcel arrays passed to mppic_bin / mppic_step;
 *   - node arrays (gas U / grad p) are concatenated in bed order, each bed's
 *     (nx+1)(ny+1)(nz+1) nodes after the previous bed's;
 *   - mppic_step's obj_out is [nsteps][nbeds][2];
 *   - mppic_deposit, mppic_interp, mppic_drag_sums and reverse mode take single-bed
 *     handles only.
 * All beds share one sort (keys are global brick, local cell; each bed's parcels keep their
 * range) and one persistent launch of each kernel per step. stream is a cudaStream_t
 * (NULL = legacy default stream). The handle binds to the current CUDA device. Returns
 * MPPIC_ERR_INVALID for sizes whose cell, node or key count overflows int32, non-positive
 * spacing, dt or dscale, or an unknown precision. */
mppic_status mppic_create(const mppic_config *cfg, int nbeds, const long long *bed_parcel_offsets,
                          const mppic_config *per_bed, void *stream, mppic_handle **out);

/* Step a1-a3 (binning; optional sort by cell). Sec. 2.2.3: the paper locates each parcel's
 * computation cell through rank-1 index tensors; Sec. 3.1: the hard conditionals near cell
 * faces and walls decide results bit by bit, so binning here is one exact formula that every
 * form shares. Writes parcels->cell from the positions with the exact FP64 formula
 * i = clamp(floor(fl64(x * fl64(1/dx))), 0, nx-1).
 * If do_sort != 0, sorts all parcel arrays by cell and records the cell ranges in the
 * handle. The order: cells are grouped in bricks of 8x8x4 (brick-major), each brick in eight
 * groups of 32 cells, taken in local cell order i + 8 (j + 8 k), or, where that saves more
 * than a quarter of the warp iterations (the sum over groups of the group's largest count),
 * ranked by parcel count (descending, ties by local cell index); within a group the parcels
 * are stored by level: the r-th parcel of every cell of the group that has more than r
 * parcels, in group order, then level r + 1. Within a cell parcels keep their previous
 * relative order (stable). parcels->cell is in the new order.
 * When the arrays hold the layout of the handle's last sort (as the last mppic_step or
 * mppic_bin left them), the sort starts from it and is local (each brick from its own range
 * and its 26 neighbours'); the result is the same stable order for any input order, only
 * the cost depends on it. */
mppic_status mppic_bin(mppic_handle *h, mppic_parcels *parcels, int do_sort);

/* Steps a4-a5: deposit the solids volume of every parcel (V = w pi (s_d d)^3 / 6, trilinear
 * weights) and form the node fields eps_s, u_g = U / max(1 - eps_s, eps_g_min) and tau
 * (Eq. 5), kept in the handle. Vs_out (device, double[nnode], may be NULL) receives the
 * deposited volume. fields_out (device, may be NULL) receives 5 arrays of nnode values in the
 * parcel precision, back to back: eps_s, u_g,x, u_g,y, u_g,z, tau. gas may be NULL (U = 0). */
mppic_status mppic_deposit(mppic_handle *h, const mppic_parcels *parcels, const mppic_gas *gas,
                           double *Vs_out, void *fields_out);

/* Steps a4-a6: deposit, node fields, then interpolation to every parcel (Sec. 3.1: the solids
 * fraction at a parcel is interpolated from the mesh with the same weights the deposit uses;
 * Eq. 4 needs grad p and grad tau at the parcel). out (device,
 * 10*np values in the parcel precision, back to back): eps_s, u_g[3], grad p[3],
 * grad tau[3] (the exact gradient of the trilinear interpolant of the node stresses). */
mppic_status mppic_interp(mppic_handle *h, const mppic_parcels *parcels, const mppic_gas *gas,
                          void *out);

/* Steps a1-a10 for nsteps coupling steps, in place. Each step deposits the solids volume,
 * forms the node fields, and per parcel interpolates, evaluates the drag closure and the
 * stress gradient, deposits the drag sums A = sum f W and B = sum f u W (f = rho_p V D),
 * pushes semi-implicitly (Eq. 4, drag implicit) with Eq. 3, reflects at the walls and
 * re-bins. obj_out (device, double[2*nsteps], may be NULL) receives per step the pressure
 * drop dP = sum_p f s_z / (Lx Ly) and the bed height H = 2 sum V z / sum V of the pre-push
 * state. Parcels are re-sorted every cfg.sort_every steps.
 * Implicit coupling (cfg.coupling_iters = K > 0; Sec. 2.2.2: the paper re-deposits F at the
 * head of every SIMPLE iteration): before the push, K gas iterations each deposit the drag
 * sums A, B of the parcels at rest against the current node gas velocity and then update it
 * at every node with the unsteady and interphase terms of Eq. 2, drag implicit:
 *   u_g' = (m u_g0 + B) / (m + A),  m = rho_G eps_g V_node / dt,  u_g0 = U / eps_g
 * (eps_g the floored voidage of the node, V_node its control volume); the push then uses the
 * last gas velocity and deposits the drag sums of the step. Without a gas solver this
 * update stands in for the SIMPLE iteration's momentum solve. */
mppic_status mppic_step(mppic_handle *h, mppic_parcels *parcels, const mppic_gas *gas,
                        int nsteps, double *obj_out);

/* Change the three differentiable parameters (drag multiplier C, diameter scale s_d, inflow
 * velocity u_in) of the handle's config for subsequent calls. dscale must be positive. The
 * paper has no counterpart (it varies the inlet velocity between runs, Sec. 3.2, but
 * differentiates nothing); s_d scales the particle diameter in V = w V_particle (Sec. 2.1). */
mppic_status mppic_set_params(mppic_handle *h, double drag_mult, double dscale, double u_in);

/* Reverse mode, part 1. The paper has no counterpart (see mppic_backward). With every > 0,
 * each following mppic_step call saves the parcel
 * state (in handle memory, 8 arrays and an identity tag per saved state) at its first step
 * and every `every` steps after, so that mppic_backward can differentiate that call.
 * every = 0 switches checkpointing off. */
mppic_status mppic_checkpoint(mppic_handle *h, int every);

/* Reverse mode, part 2. The paper has no counterpart: it differentiates nothing. This is the
 * differentiation form added to the method: the gradient of L = a <dP> + b <H> over the steps of the last
 * checkpointed mppic_step call, where <.> is the average over its steps of the objectives
 * that call returned, with respect to (drag multiplier C, diameter scale s_d, inflow
 * velocity u_in). dL_d_dP_H (host, 2 doubles) = (a, b); grad_out (host, 3 doubles) receives
 * (dL/dC, dL/ds_d, dL/du_in). Hand-written adjoints of the push, drag, walls, objectives,
 * interpolation (its transpose is a deposit) and deposit (its transpose is a gather); the
 * states between checkpoints are recomputed without sorting. Synchronous. Afterwards the
 * handle's node fields belong to a recomputed state; the next call recomputes them. */
mppic_status mppic_backward(mppic_handle *h, const double *dL_d_dP_H, double *grad_out);

/* The drag sums of the last step of the last mppic_step call, as doubles (device arrays of
 * nnode values; any may be NULL): A and B[3], from which a gas solver forms the interphase
 * force of Eq. 2 at each node, F_n = (A_n u_G,n - B_n) / V_node (Sec. 2.1: F is the parcel
 * force interpolated back to the mesh). */
mppic_status mppic_drag_sums(mppic_handle *h, double *A, double *Bx, double *By, double *Bz);

/* The solids volume the last mppic_step call deposited for the parcels' final positions
 * (step a4 inside the fused step: Vs_n = sum_p V_p W_pn, V = w pi (s_d d)^3 / 6, Sec. 2.1), as
 * doubles (device array of nnode values): the deposit the next step's node fields start from,
 * e.g. for a gas solver's voidage at the new time level. Valid until the next call that
 * deposits (mppic_step, mppic_deposit, mppic_interp); single-bed handles only. */
mppic_status mppic_step_volume(mppic_handle *h, double *Vs_out);

/* The paper has no counterpart (its TF graph reports no device errors). Synchronise the
 * handle's stream and return (and clear) any device-side error flag:
 * MPPIC_OK, MPPIC_ERR_DOMAIN or MPPIC_ERR_RANGE. */
mppic_status mppic_check(mppic_handle *h);

/* Per-phase timing of the handle's kernels, taken with CUDA events recorded on the
 * handle's stream around each launch while profiling is enabled. */
typedef struct {
  double ms[7];              /* accumulated milliseconds: sort, deposit, finalize, step (the
                                fused interp/drag/push/deposit kernel), reduce, other, couple
                                (the drag deposits and gas updates of implicit coupling) */
  long long launches[7];     /* kernel launches per phase */
  long long total_launches;  /* all kernels the handle launched while profiling */
  long long active_bricks;   /* bricks (8x8x4 cells) holding parcels at the last sort */
  long long parcels;         /* parcel count at the last sort */
} mppic_profile;

/* Enable (1) or disable (0) per-phase event timing and reset the counters. The paper has no
 * counterpart inside its solver; Sec. 4 reports computation times per SIMPLE iteration. */
mppic_status mppic_profile_enable(mppic_handle *h, int enable);

/* Synchronise the stream and return the counters accumulated since enabling (no counterpart
 * in the paper; see mppic_profile_enable). */
mppic_status mppic_profile_read(mppic_handle *h, mppic_profile *out);

/* Largest node count (nx+1)(ny+1)(nz+1) that mppic_deposit_static accepts. */
#define MPPIC_STATIC_MAX_NODES 524288

/* Solids-volume deposit that allocates nothing. The paper has no counterpart: this entry
 * point exists for callers that may not call cudaMalloc, such as a host simulation code
 * that hands the library a fixed device memory pool, or a solve phase in which a device
 * allocation (and the synchronisation it implies) is not allowed.
 *
 * It computes what mppic_deposit writes to Vs_out (Vs_n = sum_p V_p W_pn, as doubles),
 * without a handle: its fixed-point scratch is one static device array of
 * MPPIC_STATIC_MAX_NODES x 16 bytes (8 MiB) that every GPU which loads the library holds
 * until the process exits. Parcels need not be sorted.
 *   cfg      grid, spacing, dscale and precision of the bed (host pointer)
 *   parcels  device arrays x, y, z, d, omega of np entries (other fields are not read)
 *   Vs_out   device array of (nx+1)(ny+1)(nz+1) doubles, written
 *   stream   cudaStream_t the work is enqueued on (NULL = legacy default stream)
 * Returns MPPIC_ERR_INVALID, without enqueuing anything, if the node count exceeds
 * MPPIC_STATIC_MAX_NODES or the arguments are invalid. The first call on each device
 * looks up the device address of the static array (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture. Every call clears and reuses
 * the same array, so calls that overlap on the GPU (on different streams, or from several
 * threads) race and produce wrong sums; serialise them. */
mppic_status mppic_deposit_static(const mppic_config *cfg, const mppic_parcels *parcels,
                                  double *Vs_out, void *stream);

/* Launch tuning; the paper has no counterpart. The persistent step and deposit kernels use
 * grid_per_sm CTAs per SM
 * (0 = as many as fit at once, the default); sort_every >= 0 replaces the config's sort
 * period (< 0 keeps it). Results do not depend on grid_per_sm; the sort period changes
 * only the summation grouping (within the tolerances of the form). */
mppic_status mppic_tune(mppic_handle *h, int grid_per_sm, int sort_every);

/* mppic_step as one CUDA graph (Sec. 2.2.1: the paper builds one computational graph that
 * advances a complete time step and crosses the host boundary only with the time step; here
 * one graph advances nsteps steps). The first call with a given set of arguments (array
 * pointers, np, nsteps, obj_out, gas pointers) captures the whole nsteps-step sequence on
 * the handle's stream and launches it; later calls with the same arguments relaunch the
 * captured graph (one host call, no per-kernel launch cost). The captured sequence,
 * including where it sorts, is replayed as is, so nsteps should be a multiple of the sort
 * period. Changing parameters or tuning drops the graph. Not with checkpointing. */
mppic_status mppic_step_graph(mppic_handle *h, mppic_parcels *parcels, const mppic_gas *gas,
                              int nsteps, double *obj_out);

/* Node count (nx+1)(ny+1)(nz+1) of the handle's bed (all beds of a batch); no counterpart in
 * the paper. */
long long mppic_num_nodes(const mppic_handle *h);

/* Free the handle and everything it owns (no counterpart in the paper). */
void mppic_destroy(mppic_handle *h);

/* Human-readable description of the handle's last error; h may be NULL (creation errors). No
 * counterpart in the paper. */
const char *mppic_last_error(const mppic_handle *h);

#ifdef __cplusplus
}
#endif

#endif /* MPPIC_H */
