/*
 * swe_exprb.h -- C ABI of the GB300 exponential Rosenbrock shallow-water path.
 *
 * Method: Luan, Pudykiewicz, Reynolds, "Further development of efficient and
 * accurate time integration schemes for meteorological models"
 * (arXiv:1805.02144).  Equation names below are the paper's LaTeX labels
 * (eq3.17 etc.), because its printed numbering restarts in every section.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * State layout (Sec. 2, Eq. eq:dynu): u = (u_x, u_y, u_z, h), four planes of
 *   ncells doubles each, n = 4*ncells, cells in the grid's own order (a
 *   space-filling-curve order; swe_grid_cell_centres gives each cell's
 *   position so callers can build inputs in that order).
 * Pointers: every double* / const double* vector argument is a DEVICE pointer
 *   to n contiguous float64 values, owned by the caller; the library never
 *   frees or retains it beyond the call's stream work.  Arguments documented
 *   as "host" are plain host memory read during the call.
 * Streams: work is enqueued on `stream` (a cudaStream_t passed as void*,
 *   NULL = legacy default stream) and returns before it completes, except
 *   where a host result is requested (phi_stats), which waits for the stream.
 * Errors: every int-returning call returns SWE_OK (0) or a negative SWE_ERR_*
 *   code; swe_last_error() gives a message for the calling thread.  Errors
 *   found on the device (no convergence, non-finite values, a wait that ran
 *   out) are reported in phi_stats.status and by swe_device_status().
 * Grid handles are not thread-safe: one host thread per grid at a time.
 */
#ifndef SWE_EXPRB_H
#define SWE_EXPRB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SWE_OK = 0,
  SWE_ERR_INVALID_ARG = -1,
  SWE_ERR_NOMEM = -2,
  SWE_ERR_NOCONV = -3,     /* substep controller gave up (Algorithm 1)        */
  SWE_ERR_NONFINITE = -4,  /* NaN/Inf in a Krylov norm or coefficient          */
  SWE_ERR_TIMEOUT = -5,    /* a bounded device-side wait expired               */
  SWE_ERR_CUDA = -6
};

enum { SWE_EPI2 = 0, SWE_EXPRB42 = 1, SWE_PEXPRB43 = 2, SWE_EXPRB53 = 3, SWE_EPI3 = 4 };

typedef struct swe_grid swe_grid; /* opaque, library-owned */

/* Options of phipm_simul_iom2 (Sec. 4.3, Algorithm 1 and its initialisation).
 * Call swe_phi_opts_default() and change fields. */
typedef struct {
  double tol;        /* Tol of Algorithm 1 step 6                                  */
  int tol_mode;      /* 0: relative, Tol scaled by max_l ||v_l||_2; 1: absolute     */
  int m_init;        /* initial Krylov size (Algorithm 1: 1)                       */
  int m_max;         /* largest Krylov size, <= 64                                 */
  int iom;           /* orthogonalisation window: 2 (IOM2, the default) up to 64
                        (full Arnoldi when >= m_max); exprb_step_adjoint and
                        ensembles take 2 only                                      */
  double delta;      /* acceptance safety factor (Algorithm 1: 1.4)                */
  double gamma;      /* controller target for omega (0.8)                          */
  double kappa;      /* assumed error decrease per Krylov dimension (2)            */
  int max_reject;    /* SWE_ERR_NOCONV after this many rejections in one call      */
  int m_carry;       /* exprb_step: start each call slot at its last accepted m    */
  const double* replay;  /* host, optional: 3 doubles (tau, m, accepted) per attempt;
                            when non-NULL the step sizes, Krylov sizes and decisions
                            are taken from it instead of the controller (exprb_step:
                            the records of all the step's phi calls, in call order) */
  int n_replay;      /* number of attempts in replay                               */
  int precision;     /* 0: FP64 throughout.  1: mixed -- stencils, Krylov basis and
                        stage vectors of the phi evaluations in FP32 (FP32 operator
                        tables); reductions (partial sums per thread in FP32 over at
                        most a few dozen terms, then FP64), norms, controller and
                        exponential in FP64; F(u_n), D_ni and the state update in
                        FP64.  Public vectors stay FP64 either way.                 */
  int max_substeps;  /* SWE_ERR_NOCONV when one call needs more accepted substeps
                        (default 4096), or when an accepted substep would not move
                        t; bounds the run time of a launch whose step sizes the
                        controller has driven towards zero                      */
} phi_opts;

/* One controller attempt (trace record). */
typedef struct {
  double t, tau, omega;
  int m, accepted, call;  /* call: index of the phi evaluation within exprb_step */
  int pad;
} phi_attempt;

typedef struct {
  int n_jv;          /* Jacobian-vector products                 */
  int n_substeps;    /* accepted substeps                        */
  int n_reject;      /* rejected attempts                        */
  int m_last;        /* Krylov size of the last accepted substep */
  int m_max_used;
  int status;        /* SWE_OK or a negative SWE_ERR_* found on the device */
  phi_attempt* trace;  /* host buffer provided by the caller, or NULL */
  int trace_cap;       /* capacity of trace                          */
  int n_trace;         /* attempts written (<= trace_cap)            */
} phi_stats;

void swe_phi_opts_default(phi_opts* opts);

/* Build the level-`level` icosahedral geodesic Voronoi grid (Sec. 2: N_g =
 * 10*4^level + 2 cells, Voronoi control volumes, finite-volume operators
 * G, D, V, L of Eqs. eq:sweqsinv, eq:vort, eq:swdis) on the host, reorder it
 * along a space-filling curve when `reorder` != 0, and upload the operator
 * tables to the current CUDA device.  radius a [m], g [m s^-2], omega [s^-1],
 * gamma_h of Eq. eq:niu.  0 <= level <= 10.  The handle owns all device
 * memory it allocates (tables and the phi_action / exprb_step workspace). */
int swe_create_grid(int level, double radius, double g, double omega, double gamma_h,
                    int reorder, swe_grid** out);
void swe_destroy_grid(swe_grid* grid);

/* The same grid built on the host only (no CUDA call, no device memory):
 * queries and swe_grid_export work, compute entry points return
 * SWE_ERR_INVALID_ARG.  For preparing inputs or checking tables on a machine
 * without a GPU. */
int swe_create_grid_host(int level, double radius, double g, double omega, double gamma_h,
                         int reorder, swe_grid** out);

/* Host copy of one operator table, in the grid's cell order; `count` must be
 * the table's element count (error otherwise).  Names and layouts
 * (ncells = N_g, slot k = 0..5, component c = 0..2):
 *   "nbr"  int32  [6][N_g] neighbour of slot k (pentagons: slot 5 = the cell)
 *   "gen"  int32  [N_g]    generation index of each cell: the permutation from
 *                          the grid's order to the order refinement creates the
 *                          nodes in (the 12 icosahedron nodes: north pole,
 *                          northern ring at longitudes 2 pi k/5, southern ring
 *                          at 2 pi k/5 + pi/5, south pole; then, per
 *                          refinement, the new edge midpoints by ascending
 *                          (smaller, larger) generation index of the edge's
 *                          endpoints); cell i of the grid is node gen[i]
 *   "wl"   double [6][N_g] l_e/(d_e A_i);  "wld" double [N_g] -sum_k wl
 *   "nc"   double [3][6][N_g] edge-value weight x l_e nu_e/A_i of slot k
 *   "ndd"  double [3][N_g]    the same for the cell itself (D diagonal)
 *   "sdg"  double [3][N_g]    sum_e l_e nu_e / A_i (G diagonal = ndd - sdg)
 *   "vc", "vd" double: as nc, ndd with the edge tangent t_e
 * so that (L psi)_i = wld psi_i + sum_k wl psi_nbr, (D.q)_i = ndd.q_i +
 * sum_k nc.q_nbr, (V.u)_i = vd.u_i + sum_k vc.u_nbr and
 * (G psi)_i = P_i[(ndd - sdg) psi_i + sum_k nc psi_nbr].
 *   "wlT", "ncT", "vcT": the transposed slot tables, shaped as wl, nc, vc:
 * slot k of cell j holds the coefficient that row i = nbr[k][j] of wl, nc, vc
 * gives column j (0 in the pad slot of a pentagon), so that
 * (L^T psi)_j = wld psi_j + sum_k wlT psi_nbr (the diagonals are shared). */
int swe_grid_export(const swe_grid* grid, const char* table, void* host_out, int64_t count);

/* Sizes and constants: ncells, n = 4*ncells, n_A = structural nonzeros of J
 * (the n_A of the cost function Eq. eq:cost), nu of Eq. eq:niu.  Any output
 * pointer may be NULL. */
int swe_grid_query(const swe_grid* grid, int64_t* ncells, int64_t* n, int64_t* nA, double* nu);

/* Host output: unit cell centres, 3*ncells doubles laid out x[ncells],
 * y[ncells], z[ncells], in the grid's cell order. */
int swe_grid_cell_centres(const swe_grid* grid, double* xyz_host);

/* Host output: cell areas A_i [m^2] (ncells doubles), grid order. */
int swe_grid_cell_areas(const swe_grid* grid, double* area_host);

/* f = F(u), the semi-discrete shallow-water right-hand side of Eq. eq:sweqsinv
 * with the dissipation -nu L^2 of Eq. eq:swdis on every variable.  u, f:
 * device, n doubles, must not overlap. */
int swe_rhs(const swe_grid* grid, const double* u, double* f, void* stream);

/* jx = J(u) x, the Jacobian J = J_v + J_r + J_m of Eqs. eq:dynja-eq:dynjc
 * (second row of J_r taken as the derivative of F, see the oracle).  u, x, jx:
 * device, n doubles; jx must not overlap u or x. */
int swe_jv(const swe_grid* grid, const double* u, const double* x, double* jx, void* stream);

/* jx = J(u) x like swe_jv, but without allocating any device memory.  The
 * paper has no counterpart: this exists for callers that may not allocate at
 * the time of the call (code running under another framework's memory pool
 * or a fixed device budget reserved at start-up, real-time loops that cannot
 * take an allocation's latency or failure), since swe_jv allocates the grid's
 * workspace on first use.  Scratch is a static device array in the library
 * image sized for grids of at most 40962 cells (level 6; 3.9 MB held on every
 * GPU that loads the library until the process exits); larger grids return
 * SWE_ERR_INVALID_ARG.  The first call on each device looks the array up
 * (cudaGetSymbolAddress) with that device current and should come before any
 * stream capture.  All calls share the array, which keeps what the last call
 * wrote (every plane is written before it is read, so nothing is cleared):
 * calls that overlap on the GPU (e.g. on two streams) race and must be
 * serialised by the caller.  u, x, jx: device, n doubles; jx must not overlap
 * u or x (SWE_ERR_INVALID_ARG); the grid's device must be current
 * (SWE_ERR_INVALID_ARG otherwise). */
int swe_jv_noalloc(const swe_grid* grid, const double* u, const double* x, double* jx, void* stream);

/* Surface height h_s (Sec. 2: E = |u|^2/2 + g (h + h_s) in Eq. eq:sweqsinv):
 * hs_host is a host array of ncells doubles [m] in the grid's order, copied
 * to the device; NULL removes it (h_s = 0, the default).  Only F changes
 * (J does not depend on h_s).  Waits for the device.  Ensembles copy the
 * grid's tables when created, so set the topography first. */
int swe_grid_set_topography(swe_grid* grid, const double* hs_host);

/* Conservation diagnostics of the Rossby-Haurwitz section (total mass,
 * total energy and potential enstrophy of a state): out_host[0] =
 * sum_i A_i h_i, out_host[1] = sum_i A_i h_i (|u_i|^2/2 + g h_i/2),
 * out_host[2] = sum_i A_i (zeta_i + f_i)^2 / (2 h_i), zeta = V.u of Eq. eq:vort.
 * (Reading: the paper prints the energy density g h + |u|^2/2, the Bernoulli
 * function; the conserved total energy is the mass-weighted form with the
 * potential term halved.)  Summed per block and then over blocks in a fixed
 * order, so the result is reproducible.  u: device, n doubles; out_host:
 * host, 3 doubles.  Waits for the stream. */
int swe_diagnostics(const swe_grid* grid, const double* u, double* out_host, void* stream);

/* out = J(u)^T lam, the transpose of the Jacobian of Eqs. eq:dynja-eq:dynjc
 * (the operator the adjoint of a step applies; the paper defines J, its
 * transpose follows from it).  Each stencil row is transposed slot by slot
 * with tables built on the host.  u, lam, out: device, n doubles; out must not
 * overlap u or lam. */
int swe_jtv(const swe_grid* grid, const double* u, const double* lam, double* out, void* stream);

/* out = (J(x) - J(0))^T lam: the transpose of the derivative at x of the
 * quadratic part Q of F (F(u) = J(0) u + Q(u), Sec. 2; J(x) = J(0) + Q'(x)).
 * Because Q'(x) y is bilinear in (x, y), this is also the transpose, with
 * respect to u, of d/du [J(u) y] at y = x: the term the adjoint of a Krylov
 * projection with A = dt J(u_n) contributes to u_n.  x, lam, out: device,
 * n doubles; out must not overlap x or lam. */
int swe_dqtv(const swe_grid* grid, const double* x, const double* lam, double* out, void* stream);

/* phipm_simul_iom2 (Sec. 4.3, Algorithm 1): for A = dt*J(u_lin) and vectors
 * v_0..v_p, writes y_out[i] = sum_{l=0}^{p} rho_i^l phi_l(rho_i A) v_l
 * (Eq. eq:exp_multistage with the rho^l factor the drivers of Sec. 4.4 use),
 * i = 0..ns-1, by adaptive substepping (Eqs. eq3.17-eq3.18) with IOM2 Krylov
 * projections, all on the device in one persistent launch.
 *   v: host array of p+1 device pointers; a NULL entry is a zero vector.
 *   rho: host array, 0 < rho_0 < ... < rho_{ns-1} <= 1.  1 <= p <= 4, 1 <= ns <= 8.
 *   y_out: host array of ns device pointers (distinct from u_lin and v).
 *   opts: NULL = defaults.  stats: NULL, or filled after waiting for the stream.
 * The first call on a grid allocates its workspace (outside any stream capture). */
int phi_action(swe_grid* grid, const double* u_lin, double dt, int p,
               const double* const* v, int ns, const double* rho,
               double* const* y_out, const phi_opts* opts, phi_stats* stats, void* stream);

/* Per-scheme history (epi3's previous state, the m carried per call slot).
 * Create one per trajectory; reset before a new trajectory. */
typedef struct swe_scheme_state swe_scheme_state;
int swe_scheme_state_create(const swe_grid* grid, swe_scheme_state** out);
int swe_scheme_state_reset(swe_scheme_state* st);
void swe_scheme_state_destroy(swe_scheme_state* st);

/* One step u_{n+1} of EPI2 (Eq. eq3.5), exprb42 (eq3.11), pexprb43 (eq3.12),
 * exprb53 (eq3.13) or epi3 (eq_epi3, which starts with one EPI2 step), with
 * the phipm_simul_iom2 calls of Sec. 4.4.  u_n, u_np1: device, n doubles,
 * distinct.  state: required (epi3 history, m carry).  stats accumulate over
 * the step's phi calls. */
int exprb_step(swe_grid* grid, int scheme, double dt, const double* u_n, double* u_np1,
               swe_scheme_state* state, const phi_opts* opts, phi_stats* stats, void* stream);

/* Adjoint of one exprb_step: lam_n = (d u_{n+1} / d u_n)^T lam_np1 with the
 * substep decisions of the forward step frozen (the paper defines no
 * adjoint; the derivative is the one of the computed step, Algorithm 1 with
 * the step sizes, Krylov sizes and accept/reject choices of `trace`).
 *   scheme: SWE_EPI2, SWE_EXPRB42, SWE_PEXPRB43 or SWE_EXPRB53 (Eqs. eq3.5,
 *     eq3.11-eq3.13); epi3 (a two-step method) is not covered.
 *   u_n: the step's input state (device, n doubles), the checkpoint.
 *   trace: host array of the forward step's n_trace attempts, as exprb_step
 *     wrote them into phi_stats.trace (call indices 0..ncalls-1 in order).
 *   lam_np1: device, n doubles, adjoint of u_{n+1}; lam_n: device output,
 *     must not alias lam_np1 or u_n.
 *   opts: NULL or FP64 options (precision must be 0, iom must be 2); the
 *     replay fields are ignored (the trace is the replay).
 * The step is recomputed from u_n in replay mode with every accepted
 * substep's w_j, Krylov basis and small matrices kept on a device tape
 * (grown as needed and owned by the grid), then one persistent launch per
 * phipm_simul_iom2 call runs the reverse sweep, with J(u_n)^T and the
 * transposed derivative of J(u_n) x with respect to u_n applied by
 * transposed stencils.  stats (optional) reports the recomputation's counts
 * and status.  Waits for the stream.  A trace that does not match the
 * scheme, or a Krylov breakdown in a recorded substep, gives
 * SWE_ERR_INVALID_ARG. */
int exprb_step_adjoint(swe_grid* grid, int scheme, double dt, const double* u_n, const phi_attempt* trace,
                       int n_trace, const double* lam_np1, double* lam_n, const phi_opts* opts,
                       phi_stats* stats, void* stream);

/* Opt-in timing and operation counts (CUDA events recorded on the call's
 * stream around every persistent phi launch and every exprb_step / phi_action
 * call; counters of IOM2 iterations, w_j products and combination terms kept
 * on the device).  phi_flop is the operation count of the phi launches (per
 * cell: 346 per IOM2 iteration, 310 per w_j product, 8 per combination term;
 * FP64 or FP32 by the launch's precision); phi_bytes the algorithmic vector
 * bytes (per cell with FP64 vectors: 136 per IOM2 iteration, 104 per w_j
 * product, 32 per combination term; half with FP32 vectors), operator tables
 * excluded. */
typedef struct {
  double phi_ms;          /* summed duration of the persistent phi launches  */
  double call_ms;         /* summed duration of the whole calls              */
  double phi_flop;
  double phi_bytes;
  int64_t phi_launches;   /* persistent phi launches                         */
  int64_t kernel_launches;/* all kernels launched by the calls (phi included) */
  int64_t iom2_iterations, w_jv, comb_terms;
  /* time of the persistent launches by phase, as seen by block 0 (work plus
   * barrier wait): prologue, w_j pass 1, w_j pass 2, IOM2 pass 1, IOM2 pass 2
   * (+ its reduction: the window dots and the norm of the vector the previous
   * orthogonalisation made), orthogonalisation + next pass 1 (+ a barrier, or
   * the norm's own reduction after the last column), controller tail and
   * barrier, combination, Taylor exponential, controller head */
  double phase_ms[10];
  /* operator-table bytes the phi launches read (per cell, per IOM2 iteration
   * and per w_j product: 62 table reals and 12 int32 neighbour indices for a
   * pass 1 plus a pass 2), which a matrix-free stencil streams on top of the
   * vector bytes.  A launch that keeps its neighbour indices in shared memory
   * (the single-precision kernel when they fit) reads them once per launch
   * but is counted the same way, so its figure includes 48 B per cell per
   * iteration that it does not stream. */
  double phi_table_bytes;
} swe_profile;

/* on != 0: zero the counters and start recording; on == 0: stop. */
int swe_profile_enable(swe_grid* grid, int on);
/* Waits for `stream`, then fills *out with the totals since enabling. */
int swe_profile_read(swe_grid* grid, swe_profile* out, void* stream);

/* Ensembles (batching): nmem independent exprb42 trajectories, member m on
 * grids[m] (grids may repeat and may differ in level) with step dt[m] and
 * nsteps[m] steps per run, advanced together by ONE persistent cooperative
 * launch per run: the launch's blocks are split into one group per member,
 * each group runs its member's whole trajectory (F, both phipm_simul_iom2
 * calls of Sec. 4.4, D_n2, update) with its own grid barrier, control block
 * and Krylov workspace.  Member states are library-owned device buffers
 * (n_m doubles, grid order); set/get copy device to device.  A run enqueues
 * two memsets and one kernel and allocates nothing, so it can be captured in
 * a CUDA graph.  A group of blocks may hold several members, which then run
 * one after the other on those blocks (small members stacked, so that they
 * share blocks instead of idling on one each).  The launch starts with
 * 96-thread blocks (4 per SM), one member per group and a block split from a
 * work model (cells x 2^level x simulated time).  swe_ensemble_tune is the
 * autotuner: for each launch shape (96 x 4, 128 x 3, 192 x 2 and 384 x 1
 * threads x blocks per SM, which set how finely blocks, and so cells per
 * thread, can be divided between members) it runs the ensemble `rounds`
 * times, fits each member's time as serial + parallel / blocks from its last
 * two runs (carried to the next shape scaled by its block size), re-plans the
 * groups (stacking members that would take at most half the longest group's
 * time on one block) and the split that minimises the predicted longest
 * group, and finally keeps the shape, groups and split whose measured longest
 * group was shortest; it restores the states and carried Krylov sizes after
 * every run.  swe_ensemble_shape reports the launch in use.
 * Each member carries its last accepted Krylov size per call from step to
 * step and from run to run (m carry);
 * swe_ensemble_reset clears it, as for a new trajectory.
 * opts: FP64 only (precision 0), iom = 2, no replay (else
 * SWE_ERR_INVALID_ARG).  All grids must be device grids on the current
 * device. */
typedef struct swe_ensemble swe_ensemble;
int swe_ensemble_create(swe_grid* const* grids, int nmem, const double* dt, const int* nsteps,
                        const phi_opts* opts, swe_ensemble** out);
void swe_ensemble_destroy(swe_ensemble* ens);
int swe_ensemble_set_state(swe_ensemble* ens, int m, const double* u, void* stream);
int swe_ensemble_get_state(swe_ensemble* ens, int m, double* u, void* stream);
int swe_ensemble_run(swe_ensemble* ens, void* stream);
int swe_ensemble_reset(swe_ensemble* ens, void* stream);
int swe_ensemble_tune(swe_ensemble* ens, int rounds, void* stream);
/* Waits for `stream`; per-member statistics of the last run (array of nmem,
 * or NULL; trace not filled), each member's own time in ms (or NULL; from its
 * start to its end on its group's blocks) and its group's block count (or
 * NULL). */
int swe_ensemble_stats(swe_ensemble* ens, phi_stats* stats, double* member_ms, int* member_blocks,
                       void* stream);
/* The launch in use: threads per block, resident blocks per SM, blocks
 * launched, the number of member groups and, in member_group (nmem ints),
 * each member's group; groups run their members in ascending order (any
 * output may be NULL). */
int swe_ensemble_shape(const swe_ensemble* ens, int* threads, int* blocks_per_sm, int* nblocks, int* ngroups,
                       int* member_group);
/* Waits for `stream`; *flop = the algorithmic FP64 operation count of the
 * last run (per cell: 346 per IOM2 column, 310 per w_j product, 8 per
 * substep-combination term, the counts swe_profile reports for phi_action),
 * summed over members. */
int swe_ensemble_work(swe_ensemble* ens, double* flop, void* stream);

/* Self-test of the failure path of every device-side wait: one block whose
 * thread 0 polls, exactly as the grid barriers do, a flag that nothing sets.
 * The wait gives up after limit_ns of device time (1e3 <= limit_ns <= 1e9)
 * and the kernel returns normally; with preset_abort (a SWE_ERR_* code, or
 * 0) stored in the abort word first, it ends at the first check instead.
 * *status_out (host) receives the abort word: SWE_ERR_TIMEOUT when the wait
 * ran out, preset_abort when that was set.  The context stays usable.
 * Returns SWE_ERR_INVALID_ARG for a limit out of range, SWE_ERR_CUDA if the
 * launch or copies fail.  Synchronises `stream`. */
int swe_selftest_wait(int64_t limit_ns, int preset_abort, int* status_out, void* stream);

/* Waits for `stream` and returns the first device-side error of the grid's
 * last phi_action / exprb_step (SWE_OK if none), clearing it. */
int swe_device_status(swe_grid* grid, void* stream);

const char* swe_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SWE_EXPRB_H */
