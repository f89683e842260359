/*
 * esbgk.h -- C ABI of the GB300 (sm_103a) library for the coupled IMEX
 * domain-decomposition method for the ES-BGK model (Caparello & Tenna,
 * arXiv 2512.03586).
 *
 * One context advances one 2-D problem: N_x x N_y cells, each either kinetic
 * (a discrete distribution f over N_v x N_v velocities) or fluid (Euler
 * conserved variables U = (rho, rho u_x, rho u_y, E)).  One step is
 * Algorithm 1 of the paper: regime update (Sec. 3.1.2), then the s stages of
 * an IMEX Runge-Kutta scheme (Eqs. RKEI1-RKEI2 for f, RKEuler for U) with the
 * coupling of Sec. 3.3 at every stage, then the final combination.
 *
 * Conventions (every function):
 *  - Return value: ESBGK_OK (0) or a negative esbgk_status.  Errors are sticky:
 *    after an error every call but esbgk_last_error/esbgk_destroy returns it
 *    until esbgk_set_state succeeds.
 *  - Host arrays are caller-owned, C-contiguous float64 (uint8 for flags),
 *    cell index c = j * N_x + i (j along y).  f is [c][v_y index][v_x index].
 *    They are copied in or out inside the call; calls that return data wait
 *    for the context's stream.
 *  - Device memory: the library allocates none.  The caller passes one device
 *    workspace of esbgk_workspace_bytes() bytes (e.g. a torch uint8 tensor)
 *    and keeps it alive until esbgk_destroy.
 *  - All device work goes to the caller's CUDA stream (cudaStream_t passed as
 *    void*; NULL = legacy default stream).  A context is not thread-safe, and
 *    the library keeps process-wide launch caches (occupancy per kernel and
 *    launch shape, the shared-memory limit) without a lock: calls from several
 *    host threads must be serialised by the caller, on one context or on many.
 *  - Velocity nodes (Sec. 3.2): v_k = -v_max + (k + 1/2) dv, dv = 2 v_max/N_v,
 *    quadrature weight dv^2 (midpoint rule).
 */
#ifndef ESBGK_H
#define ESBGK_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct esbgk_ctx esbgk_ctx;

typedef enum {
  ESBGK_OK = 0,
  ESBGK_E_ARG = -1,            /* invalid argument (sizes, tableau, dt, NULL)        */
  ESBGK_E_WORKSPACE = -2,      /* workspace too small or misaligned (< 256 B)        */
  ESBGK_E_CUDA = -3,           /* a CUDA runtime call failed; see esbgk_last_error   */
  ESBGK_E_NONREALIZABLE = -4,  /* rho <= 0, T <= 0, det(temperature tensor) <= 0 or a
                                  singular moment system in some cell                */
  ESBGK_E_TIMEOUT = -5,        /* a bounded device wait expired                     */
  ESBGK_E_STATE = -6,          /* call out of order (e.g. step before set_state)    */
  ESBGK_E_TOO_LARGE = -7       /* problem exceeds the fixed scratch of
                                  esbgk_kinetic_steps_noalloc                        */
} esbgk_status;

typedef enum { ESBGK_FP64 = 0, ESBGK_FP32 = 1, ESBGK_BF16 = 2 } esbgk_prec;
typedef enum { ESBGK_BC_PERIODIC = 0, ESBGK_BC_OUTFLOW = 1 } esbgk_bc;
typedef enum { ESBGK_SWITCH_FROZEN = 0, ESBGK_SWITCH_PLAIN = 1, ESBGK_SWITCH_LEARNED = 2 } esbgk_switch;
typedef enum { ESBGK_COUPLE_STAGE = 0, ESBGK_COUPLE_STEP = 1 } esbgk_coupling;
typedef enum { ESBGK_INTERFACE_OWN = 0, ESBGK_INTERFACE_CONSERVATIVE = 1 } esbgk_interface;
typedef enum { ESBGK_TAU_CONSTANT = 0, ESBGK_TAU_DENSITY = 1 } esbgk_tau_model;
typedef enum { ESBGK_SUMS_PLAIN = 0, ESBGK_SUMS_COMPENSATED = 1 } esbgk_moment_sums;

/* Cartesian grid of Sec. 3.2: N_x x N_y cells on [x0,x1] x [y0,y1]; two ghost
 * cells per side, periodic or outflow (copy of the edge cell). */
typedef struct {
  int32_t nx, ny;
  double x0, x1, y0, y1;
  int32_t bc_x, bc_y; /* esbgk_bc */
} esbgk_grid;

/* Velocity grid of Sec. 3.2: N_v points per direction on [-v_max, v_max],
 * 3 <= N_v <= 64.  The discrete Gaussian is corrected by a quadratic in the
 * velocity (1, xi_x, xi_y, xi_x^2, xi_x xi_y, xi_y^2); on two points per
 * direction xi^2 is a multiple of 1, the 6x6 moment system is singular, and
 * N_v = 2 is rejected (E_ARG; 0 workspace bytes). */
typedef struct {
  int32_t nv;
  double vmax;
} esbgk_vmesh;

/* Model and switch parameters.
 *  beta       ES-BGK parameter (Sec. 2): Pr = 1/(1 - beta), beta in [-1/2, 1).
 *  tau        collision rate nu = tau / eps(x) (tau constant).
 *  eta_factor eta = eta_factor * eps(x) in the criterion of Eq. crit:CompEuler.
 *  delta      threshold of Eq. eqKintoFluid1 (absolute L1 deviation).
 *  cweno_eps  epsilon of the CWENO3 nonlinear weights (Sec. 3.2).
 *  sw         esbgk_switch: FROZEN keeps the regime map, PLAIN applies
 *             Sec. 3.1.2 before every step, LEARNED applies Sec. 3.1.2 and
 *             adds the cells a trained network predicts kinetic for the
 *             next step (see "Learned regime switch" below).
 *  coupling   esbgk_coupling: STAGE couples at every stage (Algorithm 1),
 *             STEP only at step end (the LOC-hybrid of Sec. 3.5).
 *  prec       esbgk_prec of f storage and per-element arithmetic: FP64; FP32;
 *             BF16 storage with FP32 arithmetic.  Per-cell tensor solves,
 *             U and the totals are always FP64.
 *  interface_flux  esbgk_interface: OWN -- at a face between a kinetic and a
 *             fluid cell each cell uses its own model's flux (Sec. 3.6 states
 *             conservation but gives no interface flux; the totals then drift at the interfaces);
 *             CONSERVATIVE -- the fluid cell's Euler update takes, at that
 *             face, the moments (1, v, |v|^2/2) of the kinetic numerical flux
 *             the kinetic cell uses, so that mass, momentum and energy are
 *             conserved to rounding.  Zero-initialised structs get OWN.
 *  tau_model  esbgk_tau_model: CONSTANT -- nu = tau / eps(x); DENSITY -- the
 *             relaxation time scales with the density (Sec. 2 lets tau
 *             depend on the macroscopic moments): nu = tau rho / eps(x), rho
 *             of the cell's f* at each stage, and the criterion's viscosity
 *             and conductivity use tau rho.  Zero-initialised: CONSTANT.
 *  moment_sums  esbgk_moment_sums: how FP32 and BF16 storage sum the moments
 *             of f* over the velocity nodes in the stages (Sec. 2: the
 *             moments set the targets of the projected Gaussian, so their
 *             rounding enters the relaxation's mass balance).  PLAIN --
 *             paired per-lane partial sums and a butterfly over the lanes;
 *             COMPENSATED -- the per-lane runs go every 16 nodes into a
 *             Neumaier-compensated accumulator and the lanes are added with
 *             error-free two-sums (several times smaller mass drift; these
 *             stages run in kernels of their own and take about 14 % more
 *             time per step on an all-kinetic 256 x 256 x 48^2 problem).
 *             No effect in FP64 storage.
 *             Zero-initialised: PLAIN. */
typedef struct {
  double beta, tau, eta_factor, delta, cweno_eps;
  int32_t sw, coupling, prec, interface_flux, tau_model, moment_sums;
} esbgk_params;

/* IMEX tableaux (Sec. 3.4), 2 <= s <= 4 stages: explicit (At, bt) for the
 * transport and the Euler system (Abar = At, bbar = bt), implicit (A, b) for
 * the relaxation.  Entry (i, j) of a matrix is At[i*4 + j] (row stride 4
 * whatever s).  At must be strictly lower triangular, A lower triangular with
 * A[i][i] >= 0; at most three running accumulators may be needed (always true
 * when the first stage is explicit, as in ARS schemes). */
typedef struct {
  int32_t s;
  double At[16], bt[4], A[16], b[4];
} esbgk_tableau;

/* Library version (major*10000 + minor*100 + patch). */
int esbgk_version(void);

/* Bytes of device workspace needed for this problem; 0 on invalid input. */
size_t esbgk_workspace_bytes(const esbgk_grid* grid, const esbgk_vmesh* vmesh,
                             const esbgk_params* params);

/* Create a context.  `workspace` is device memory (>= 256-byte aligned) of at
 * least esbgk_workspace_bytes() bytes, owned by the caller.  `stream` is a
 * cudaStream_t or NULL.  On success *out receives the context (host-allocated;
 * free with esbgk_destroy). */
int esbgk_create(const esbgk_grid* grid, const esbgk_vmesh* vmesh, const esbgk_params* params,
                 void* workspace, size_t workspace_bytes, void* stream, esbgk_ctx** out);

/* Release the host context (the workspace stays the caller's). NULL is a no-op. */
void esbgk_destroy(esbgk_ctx* ctx);

/* Set the macroscopic state (Sec. 3.3): rho, u_x, u_y, T and the Knudsen field
 * eps, each [N_c] float64, and the regime map kinetic[N_c] (1 = kinetic;
 * NULL = all kinetic).  Kinetic cells get f = the discrete Maxwellian of
 * (rho, u, T) (Eq. Coupling_FluKin), as every test of Sec. 4 starts.  Clears a
 * sticky error.  Returns E_ARG for rho <= 0, T <= 0 or eps < 0 anywhere. */
int esbgk_set_state(esbgk_ctx* ctx, const double* rho, const double* ux, const double* uy,
                    const double* T, const double* eps, const uint8_t* kinetic);

/* Overwrite f of every cell from host float64 [N_c][N_v][N_v] (resume from a
 * checkpoint; values of fluid cells are kept but unused) and set U := moments
 * of f in kinetic cells (Eq. Coupling_KinFlu). */
int esbgk_set_f(esbgk_ctx* ctx, const double* f);

/* Copy f of every cell to host float64 [N_c][N_v][N_v] (fluid cells: stale). */
int esbgk_get_f(esbgk_ctx* ctx, double* f);

/* Regime update of Algorithm 1 from the current state (Eqs. crit:CompEuler,
 * eqKintoFluid1): lambda_A = max |eig(I - S_1)| with the S_1 of Sec. 3.1.1
 * (central differences of u and T), the L1 deviation of f from its Maxwellian
 * in kinetic cells; new flag = lambda_A > eta  or  (kinetic and L1 > delta).
 * Cells that turn kinetic get f := Maxwellian(U) at the next advance. */
int esbgk_regime_update(esbgk_ctx* ctx);

/* Replace the regime map (kinetic[N_c], 1 = kinetic) before the next advance,
 * e.g. to impose a reference map; conversions are taken relative to the map
 * of the previous step. */
int esbgk_set_flags(esbgk_ctx* ctx, const uint8_t* kinetic);

/* Solid obstacles with specularly reflecting walls (Sec. 4.2.3-4.2.4, Tests 5
 * and 6: a cylinder or a rectangle "such that the integrators are never
 * executed in it" with specular reflection on its surface).  solid[N_c] (host,
 * 1 = solid, cell order j*N_x + i), copied within the call; NULL or all zero
 * removes the obstacles.  Call after esbgk_set_state (which keeps the mask).
 * Solid cells hold no state, are never kinetic, buffer or fluid, and are left
 * out of esbgk_totals.  Every stencil value a fluid or kinetic cell needs from
 * beyond a wall is the mirror image, across the wall face, of a cell on its
 * own side: f with the velocity component normal to the wall reversed
 * (v_n -> -v_n: the node index along that axis reversed on the midpoint
 * grid), and (rho, -m_n, m_t, E) for the Euler flux and the criterion's
 * gradients; the mass and energy fluxes through a wall then vanish exactly.
 * The paper gives no wall discretisation: this is the library's reading.
 * Obstacles must stay three cells away from an outflow edge (a periodic axis
 * wraps), and are not combined with the conservative interface, the learned
 * switch or the batched form (ESBGK_E_ARG).  Problems with obstacles run the
 * generic per-cell stage kernel.  Synchronises the stream. */
int esbgk_set_solid(esbgk_ctx* ctx, const uint8_t* solid);

/* Copy the current regime map to host kinetic[N_c]. */
int esbgk_get_flags(esbgk_ctx* ctx, uint8_t* kinetic);

/* Indicators of the last regime update: lamA[N_c] and L1[N_c] (L1 = 0 in
 * cells that were fluid).  Either pointer may be NULL. */
int esbgk_get_indicators(esbgk_ctx* ctx, double* lamA, double* L1);

/* Advance one step with the current regime map (Algorithm 1 without the
 * regime update): stages of Eqs. RKEuler/RKEI1 with per-stage coupling
 * (Remark rem_coupling), final combination Eqs. RKEuler_2/RKEI2.  dt > 0. */
int esbgk_advance(esbgk_ctx* ctx, double dt, const esbgk_tableau* tab);

/* One full step of Algorithm 1: esbgk_regime_update (PLAIN and LEARNED
 * switches) then esbgk_advance.  Enqueued on the stream; does not wait.
 * On a stream other than the legacy default stream, with timing off, a step
 * whose launch arguments equal the previous step's is captured once into a
 * CUDA graph; later steps with the same arguments replay it (the context
 * keeps up to three graphs).  Results are identical either way. */
int esbgk_step(esbgk_ctx* ctx, double dt, const esbgk_tableau* tab);

/* Enable (default) or disable graph replay in esbgk_step; drops the graphs
 * kept so far.  Synchronises the stream. */
int esbgk_graphs(esbgk_ctx* ctx, int32_t enable);

/* Probe of the library's bounded device waits (failure detection without a
 * fault): launches one CTA on `stream` (NULL: the legacy default stream) that
 * waits on a shared-memory barrier with the same bounded poll loop the kernels
 * use, limited to `polls` polls (1 .. 2^20; each poll may suspend the thread
 * for a hardware-defined time), and synchronises the stream.  arrive != 0: the
 * barrier receives its arrival and the call returns ESBGK_OK; arrive = 0: the
 * arrival is withheld, the wait runs out, the kernel records the timeout in a
 * device error word and returns normally, and the call returns
 * ESBGK_E_TIMEOUT.  The CUDA context stays usable either way.  No device
 * memory is allocated (the word is a static device variable); ESBGK_E_ARG for
 * polls out of range, ESBGK_E_CUDA if the launch fails. */
int esbgk_wait_probe(int32_t arrive, int32_t polls, void* stream);

/* Per-cell form the specialised stage launches of this context take (the
 * ARS(2,3,3) and IMEX-Euler stages): nodes per vector group along v_x (1:
 * one node per lane and iteration; 2 or 4: one vector load of that many
 * consecutive nodes, N_v divisible by it) and kinetic cells per warp (2 in
 * the vector form for velocity grids of at most 512 nodes, one cell per
 * half-warp; else 1).  Host only, no launch; any pointer may be NULL. */
int esbgk_kinetic_form(const esbgk_ctx* ctx, int32_t* nodes_per_group, int32_t* cells_per_warp);

/* Tiled stage kernel (Sec. 3.2 transport, Eq. RKEI1-RKEI2): when every cell
 * is kinetic (the last esbgk_set_state or esbgk_set_flags map) and the regime
 * is frozen (ESBGK_SWITCH_FROZEN), the specialised stage launches run on
 * tiles of 4 x 4 cells whose threads compute each CWENO3 face once and share
 * it between the two cells it separates (2.5 faces per cell and node; the
 * per-cell kernel computes 4).  Needs an even N_v and f* of 16 cells in
 * shared memory (on GB300: N_v <= 54 in FP32/BF16 storage, N_v <= 34 in
 * FP64); other problems keep the per-cell kernel.  Results agree with the
 * per-cell kernel to rounding (a different but equivalent order of the face
 * arithmetic).  esbgk_tiles enables (enable != 0) or disables it (the
 * default: on GB300 the per-cell kernel is as fast at the sizes measured);
 * host only, no launch.  esbgk_tiled reports whether the next step's stages
 * take it. */
int esbgk_tiles(esbgk_ctx* ctx, int32_t enable);
int esbgk_tiled(const esbgk_ctx* ctx, int32_t* tiled);

/* Macroscopic fields of every cell (moments of f in kinetic cells, the Euler
 * solution elsewhere), each [N_c] float64; any pointer may be NULL. */
int esbgk_get_moments(esbgk_ctx* ctx, double* rho, double* ux, double* uy, double* T);

/* Conserved variables U[4][N_c] (rho, rho u_x, rho u_y, E). */
int esbgk_get_cons(esbgk_ctx* ctx, double* U);

/* Global mass, x- and y-momentum and energy: sum over cells of U dx dy. */
int esbgk_totals(esbgk_ctx* ctx, double out[4]);

/* Work counters since create: kinetic cell-stage updates (each counts N_v^2
 * element updates; one per transport evaluation of a kinetic cell), steps,
 * the kinetic cells of the current map, and buffer-cell reconstructions
 * f := Maxwellian(U) done inside the stages.  Any pointer may be NULL. */
int esbgk_counters(esbgk_ctx* ctx, long long* kinetic_cell_updates, long long* steps,
                   long long* kinetic_cells, long long* buffer_fills);

/* Kernel classes reported by esbgk_timing_read. */
enum {
  ESBGK_K_L1 = 0,      /* L1 deviation of kinetic cells (regime update)        */
  ESBGK_K_FLAGS = 1,   /* criteria and new regime map                          */
  ESBGK_K_COMPACT = 2, /* categorisation and compaction of the map             */
  ESBGK_K_PREP = 3,    /* start-of-step coupling (buffer and converted cells)  */
  ESBGK_K_STAGE = 4,   /* fused IMEX stage kernels                             */
  ESBGK_K_FINAL = 5,   /* final combination (same kernel as the stages)        */
  ESBGK_K_OTHER = 6,    /* learned-switch inference (features, network, judge)  */
  ESBGK_K_COUNT = 7
};

/* Per-kernel timing: when enabled, every kernel the library launches on the
 * context's stream is bracketed by CUDA events on that stream.  Host event
 * objects only; no device memory. */
int esbgk_timing(esbgk_ctx* ctx, int enable);

/* Wait for the stream and return, per kernel class, the summed device time in
 * milliseconds (ms[ESBGK_K_COUNT]) and the number of launches
 * (launches[ESBGK_K_COUNT]) recorded since the last read; then reset.  Either
 * pointer may be NULL; n is the capacity of both arrays. */
int esbgk_timing_read(esbgk_ctx* ctx, double* ms, long long* launches, int32_t n);

/* Wait for the stream and report a pending device error. */
int esbgk_sync(esbgk_ctx* ctx);

/* Message of the last error (NUL-terminated, truncated to n) and, for
 * ESBGK_E_NONREALIZABLE, the first offending cell (else -1). */
int esbgk_last_error(esbgk_ctx* ctx, char* buf, size_t n, long long* bad_cell);

/* Per-cell collision check entry (device pointers, no context): for n cells of
 * f*[n][N_v][N_v] (storage type of `prec`) and h[n] (float64) solve the
 * implicit relaxation f = f* + h (G_hat[f] - f) of Eq. RKEI1 through the
 * conserved moments and write f[n][N_v][N_v] and G_hat (same type).  This is
 * the device code the stage kernel uses.  Enqueued on `stream` (does not
 * wait); a cell whose state is not realizable (rho <= 0, T <= 0, singular
 * moment system) gets NaN in both outputs.  3 <= nv <= 64, else E_ARG. */
int esbgk_relax_cells(const void* fstar, const double* h, int32_t n, int32_t nv, double vmax,
                      double beta, int32_t prec, void* f_out, void* g_out, void* stream);

/* ------------------------------------------------------------------------
 * Batched form: n independent problems (cases) of uneven sizes advanced
 * together.  (The paper advances one problem at a time; the batch is a
 * throughput service.  Each case follows Algorithm 1 and the regime update of
 * Sec. 3.1.2 as a single context would, through the same per-cell device
 * code compiled into separate kernels: results agree with a single context
 * to rounding -- a few units in the last place, which an under-resolved
 * velocity grid can amplify through the moment system -- not bit for bit.)
 * Each case is a full problem as above (its own grid, velocity mesh,
 * parameters, state and regime map); every step runs as one launch per kernel
 * over all cases -- one persistent stage launch walks the concatenated
 * compacted work lists (kinetic cells, buffer cells, chunks of 32 fluid cells)
 * of every case -- and, on a stream other than the legacy default stream, the
 * launches of a step are captured once into a CUDA graph and replayed.
 * All cases share the storage precision.  Cases are addressed by index
 * 0..n-1; per-case host arrays follow the single-problem conventions.
 * Cases with the learned switch take the criterion in the batched launches
 * and their network (features, forward pass, judge) in per-case launches of
 * the same step (captured in the step's graph); each needs its parameters
 * (esbgk_batch_set_switch_params) before the first step, else the step
 * fails with ESBGK_E_STATE.
 * Errors: ESBGK_E_ARG (bad argument, mixed precisions, case index out of
 * range), ESBGK_E_WORKSPACE (workspace too small or not 256-byte aligned),
 * ESBGK_E_CUDA, ESBGK_E_NONREALIZABLE (reported by esbgk_batch_sync for the
 * first case with a device error), ESBGK_E_STATE (a case has no state).
 * A failed step leaves the batch in the failed state until a set_state. */
typedef struct esbgk_batch esbgk_batch;

/* Bytes of device workspace for the batch: the sum of the cases' workspaces
 * plus a few KB of per-case descriptor tables.  0 on invalid input. */
size_t esbgk_batch_workspace_bytes(int32_t n, const esbgk_grid* grids, const esbgk_vmesh* vmeshes,
                                   const esbgk_params* params);

/* Create a batch of n >= 1 cases (arrays grids[n], vmeshes[n], params[n]) on
 * one caller-owned device workspace (256-byte aligned, owned by the caller
 * and kept alive until esbgk_batch_destroy) and one stream (NULL = legacy
 * default stream).  *out receives the handle. */
int esbgk_batch_create(int32_t n, const esbgk_grid* grids, const esbgk_vmesh* vmeshes,
                       const esbgk_params* params, void* workspace, size_t workspace_bytes,
                       void* stream, esbgk_batch** out);
/* Free the batch's host state (its graphs and events); the device workspace
 * stays the caller's, and work already queued on the stream still uses it
 * (synchronise first, e.g. esbgk_batch_sync).  NULL is ignored. */
void esbgk_batch_destroy(esbgk_batch* b);

/* esbgk_set_switch_params and esbgk_switch_stats for case i (a learned-switch
 * case; ESBGK_E_STATE for another switch). */
int esbgk_batch_set_switch_params(esbgk_batch* b, int32_t i, const float* theta);
int esbgk_batch_switch_stats(esbgk_batch* b, int32_t i, long long* judged_cells, long long* predicted,
                             long long* missed, long long* extra);

/* esbgk_set_state for case i. */
int esbgk_batch_set_state(esbgk_batch* b, int32_t i, const double* rho, const double* ux,
                          const double* uy, const double* T, const double* eps, const uint8_t* kinetic);

/* One step of every case (esbgk_step semantics: the regime update of
 * plain-switch cases, then Algorithm 1): dt[n] host array of case time steps,
 * one tableau for all.  use_graph != 0 replays a captured CUDA graph of the
 * step when the stream allows capture (not the legacy default stream).
 * Asynchronous: errors of the kernels surface at esbgk_batch_sync or at a
 * read-back. */
int esbgk_batch_step(esbgk_batch* b, const double* dt, const esbgk_tableau* tab, int32_t use_graph);

/* Per-case read-back (as esbgk_get_moments, esbgk_get_cons, esbgk_get_flags). */
int esbgk_batch_get_moments(esbgk_batch* b, int32_t i, double* rho, double* ux, double* uy, double* T);
int esbgk_batch_get_cons(esbgk_batch* b, int32_t i, double* U);
int esbgk_batch_get_flags(esbgk_batch* b, int32_t i, uint8_t* kinetic);

/* Work counters summed over cases (see esbgk_counters): kinetic cell
 * updates (transport evaluations of kinetic cells), the same weighted by each
 * case's N_v^2 (kinetic (cell x velocity) element updates), batched steps,
 * and the current number of kinetic cells.  Any pointer may be NULL. */
int esbgk_batch_counters(esbgk_batch* b, long long* kinetic_cell_updates, long long* element_updates,
                         long long* steps, long long* kinetic_cells);

/* Autotuner of the batched stage launch (it advances the batch: three steps
 * (dt, tab) per candidate schedule, one untimed and two timed, on the
 * current state).  First the launch shape: 32, 64 or 128 threads per CTA
 * (within the shared-memory limit) x 0, 2, 4 or 8 CTAs per SM (0: as many as
 * fit).  Then, one velocity grid at a time with the others held, the
 * per-cell form of its cases: the library's default form for that N_v
 * (esbgk_kinetic_form), the same with one cell per warp where the default
 * puts two, or the scalar form; a form replaces the current one only if it is
 * at least 2 % faster.  The chosen forms are kept for the process per (N_v,
 * storage precision), and the launch shape per (storage precision, set of
 * N_v): batches created later start from them.  Reports the launch shape
 * (either pointer may be NULL); esbgk_batch_schedule reports the forms. */
int esbgk_batch_autotune(esbgk_batch* b, const double* dt, const esbgk_tableau* tab, int32_t* threads,
                         int32_t* ctas_per_sm);

/* The batch's current schedule: the launch shape (threads per CTA, CTAs per
 * SM; NULL to skip) and, for each distinct N_v of its cases in ascending
 * order, the per-cell form: 0 the default form, 1 one cell per warp, 2 the
 * scalar form.  Writes min(cap, count) entries to nv[] and form[] (caller's
 * host arrays; NULL allowed when cap = 0) and the number of distinct N_v to
 * *count (NULL to skip).  Host only, no device work; ESBGK_E_ARG for a null
 * batch or cap < 0. */
int esbgk_batch_schedule(const esbgk_batch* b, int32_t* threads, int32_t* ctas_per_sm, int32_t* nv, int32_t* form,
                         int32_t cap, int32_t* count);

/* Set the per-cell form (0, 1 or 2 as in esbgk_batch_schedule) of the cases
 * whose velocity grid has nv nodes per direction, for the following steps;
 * results agree with every form to rounding.  Host only; ESBGK_E_ARG for a
 * null batch, nv outside 0..64 or an unknown form. */
int esbgk_batch_set_form(esbgk_batch* b, int32_t nv, int32_t form);

/* Wait for the stream; report a pending device error of any case. */
int esbgk_batch_sync(esbgk_batch* b);

/* Per-launch timing of the batched step, as esbgk_timing / esbgk_timing_read
 * (the same kernel classes; a class sums the launches of all cases).  While
 * enabled, steps run as plain launches (no graph replay). */
int esbgk_batch_timing(esbgk_batch* b, int32_t enable);
int esbgk_batch_timing_read(esbgk_batch* b, double* ms, long long* launches, int32_t n);

/* Message of the last failure of the batch or of one of its cases into
 * buf[n] (NUL-terminated); *case_index (may be NULL) receives the failing
 * case or -1. */
int esbgk_batch_last_error(esbgk_batch* b, char* buf, size_t n, int32_t* case_index);

/* ------------------------------------------------------------------------
 * Learned regime switch.  (An addition to the paper, whose regime decision is
 * the criterion of Sec. 3.1.2 alone.)  A 3-layer convolutional network reads
 * five features of every cell of a 5 x 5 neighbourhood at step n --
 * (log rho, s u_x, s u_y, log T, log10(eps s^2)), s = (1/128) / min(dx, dy),
 * scaled so that the criterion's velocity-gradient and temperature-gradient
 * terms are the same function of the features on every grid -- and
 * predicts the flag the criterion gives the cell at step n + 1:
 *   a1 = relu(b1 + conv3x3(x, W1)), a2 = relu(b2 + conv3x3(a1, W2)),
 *   z = b3 + a2 . w3, predicted kinetic iff z > 0,
 * with 'same' zero padding, 32 hidden channels, bf16 operands and float32
 * accumulation on the tensor cores.  Parameters (ESBGK_CNN_PARAMS float32,
 * this order): W1 [32][3][3][5], b1[32], W2 [32][3][3][32], b2[32], w3[32],
 * b3[1].
 * With sw = ESBGK_SWITCH_LEARNED the regime update applies the criterion
 * (it is the judge and the fallback: every cell it marks kinetic is
 * kinetic) and adds the cells predicted kinetic for the next step.  It
 * counts, per update after the first, the cells predicted kinetic at the
 * previous update, those the criterion now marks kinetic that were not
 * predicted (missed) and those predicted but not marked (extra).
 * Features on the device: [cell][ESBGK_CNN_CHANNELS] bf16, channels 5..15
 * zero, cell = j * N_x + i. */
#define ESBGK_CNN_PARAMS 10753
#define ESBGK_CNN_CHANNELS 16

/* Load the network of a LEARNED context (host float32 theta[ESBGK_CNN_PARAMS]);
 * required before the first step.  ESBGK_E_STATE for another switch. */
int esbgk_set_switch_params(esbgk_ctx* ctx, const float* theta);

/* Judge statistics accumulated since create (any pointer may be NULL):
 * judged cells, cells predicted kinetic, missed, extra. */
int esbgk_switch_stats(esbgk_ctx* ctx, long long* judged_cells, long long* predicted, long long* missed,
                       long long* extra);

/* Features of the current state into device memory x (16-byte aligned,
 * N_c * ESBGK_CNN_CHANNELS bf16); asynchronous on the context's stream.
 * Any switch mode. */
int esbgk_features(esbgk_ctx* ctx, void* x);

/* Training and evaluation of the network on batches of n images of H x W
 * cells (features as above, [img][H][W][16] bf16 in device memory; labels
 * y [img][H][W] uint8 in device memory).  Loss: class-weighted binary
 * cross-entropy averaged over cells, weight pos_weight on kinetic labels.
 * Optimiser: Adam (beta1 0.9, beta2 0.999, eps 1e-8) on the float32
 * parameters.  The workspace (256-byte aligned, caller-owned) holds the
 * parameters, optimiser state, activations and gradients. */
typedef struct esbgk_cnn esbgk_cnn;
size_t esbgk_cnn_workspace_bytes(int32_t max_images, int32_t H, int32_t W);
int esbgk_cnn_create(int32_t max_images, int32_t H, int32_t W, void* workspace, size_t workspace_bytes,
                     void* stream, esbgk_cnn** out);
/* Free the network's host state; the device workspace stays the caller's,
 * and work already queued on the stream still uses it (synchronise first).
 * NULL is ignored. */
void esbgk_cnn_destroy(esbgk_cnn* c);
/* Set (and reset the optimiser) / read the float32 parameters (host). */
int esbgk_cnn_set_params(esbgk_cnn* c, const float* theta);
int esbgk_cnn_get_params(esbgk_cnn* c, float* theta);
/* Logits of n <= max_images images into device memory logits[n][H][W]. */
int esbgk_cnn_forward(esbgk_cnn* c, const void* x, int32_t n, float* logits);
/* Loss and gradient (host float *loss, float grad[ESBGK_CNN_PARAMS]; either
 * may be NULL) without an update; synchronises. */
int esbgk_cnn_gradient(esbgk_cnn* c, const void* x, const uint8_t* y, int32_t n, float pos_weight, float* loss,
                       float* grad);
/* One Adam step at learning rate lr; the loss of the batch before the step
 * into *loss when non-NULL (then it synchronises). */
int esbgk_cnn_train_step(esbgk_cnn* c, const void* x, const uint8_t* y, int32_t n, float pos_weight, float lr,
                         float* loss);
int esbgk_cnn_sync(esbgk_cnn* c);

/* Allocation-free stepping of an all-kinetic problem.  (The paper has no
 * counterpart: this is a service for callers.)
 *
 * Who needs it: callers that cannot allocate device memory at all -- a plugin
 * or embedded solver inside a host application that owns every device
 * allocation through its own pool or fixed budget (an allocation of ours would
 * bypass its accounting or fail), or a latency-bound loop that must never
 * enter the allocator.  Every other entry point needs a caller-provided
 * workspace (esbgk_create), which such a caller may not be able to obtain;
 * this one needs none.
 *
 * It advances f by `nsteps` IMEX steps (dt, tab) with every cell kinetic and
 * the regime frozen (params->sw and params->coupling are validated but make no
 * difference when no cell is fluid), exactly as esbgk_create + esbgk_set_f +
 * esbgk_step would (with BF16 storage the stochastic-rounding keys restart at
 * every call, as in a fresh context, so a sequence of calls agrees with one
 * long run to the BF16 rounding bound rather than bit for bit).  The caller passes, in device memory:
 *   f    in/out [N_c][N_v][N_v], storage type of params->prec (f^n in,
 *        f^{n+nsteps} out);
 *   eps  in [N_c] float64, the Knudsen number;
 *   U    out [4][N_c] float64, the conserved moments of the final f.
 * Intermediate stage and accumulator arrays live in one static device array of
 * 32 MiB that the library keeps on every GPU it is loaded on until the process
 * exits.  The problem fits when
 *   5 * N_c * N_v^2 * (8, 4 or 2 bytes for FP64, FP32, BF16)
 *     + 68 * N_c + 3 KiB  <=  32 MiB  (each array rounded up to 256 bytes;
 *   the 3 KiB hold the counters, the error word and the rounding key);
 * larger problems are rejected with ESBGK_E_TOO_LARGE before any device work.
 * The first call on a device looks up the array's device address (with that
 * device current).
 * All calls share the one array, which keeps the last call's contents (the
 * call clears what must start at zero): calls that may overlap on the GPU --
 * on different streams, or from several host threads -- race and must be
 * serialised by the caller.  The call waits for `stream` at the end and
 * returns ESBGK_E_NONREALIZABLE if some cell became non-realizable, E_ARG on
 * invalid input, E_CUDA on a failed CUDA call. */
int esbgk_kinetic_steps_noalloc(const esbgk_grid* grid, const esbgk_vmesh* vmesh,
                                const esbgk_params* params, double dt, const esbgk_tableau* tab,
                                int32_t nsteps, const double* eps, void* f, double* U, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* ESBGK_H */
