/* lcp_gb300.h -- C ABI of the GB300 (sm_103a) collision-resolution library.
 *
 * The library solves, per time step, the linear complementarity problem
 *     0 <= x  perp  A x + b >= 0,     A = D^T M D,   b = (Phi + dt D^T U_nc) / dt
 * of the paper's Sec. 3, Eqs. (LCP) and (defAandb), for M rigid spheres in
 * Stokes flow.  x holds the normal contact-force magnitudes of the n contacts,
 * D maps them to per-body forces/torques, and M is the mobility of Sec. 2
 * (U = M F), applied as P M_stk P^T (Fig. 1): a second-kind boundary-integral
 * solve by GMRES whose every iteration is an O(N^2) stresslet sum over all
 * surface nodes.  The solvers are Mono-PQN (Algorithm 1, with Algorithm 2 and
 * the weighted prox of Proposition 1) and Bi-PQN (Algorithm 4) with a
 * Rotne-Prager-Yamakawa low-fidelity operator.
 *
 * Conventions (all entry points):
 *  - Plain C types only.  Host pointers are read/written synchronously;
 *    "_dev" variants take device pointers and run on the context's stream.
 *  - Per-body vectors are [M][6] = (Fx, Fy, Fz, Tx, Ty, Tz) for forces and
 *    (Ux, Uy, Uz, Wx, Wy, Wz) for velocities (Sec. 2, definition of U and F).
 *  - Node vectors are [N][3] with N = M * n_theta * n_phi, body-major; inside
 *    a body node q = j * n_phi + k (t_j = cos(theta_j) ascending Gauss-Legendre
 *    node, phi_k = 2 pi k / n_phi).
 *  - Contacts are in the caller's order, or in lexicographic (i, j) order
 *    when the library detects them.  x[l] is the force magnitude of contact l.
 *  - The library owns every device buffer of a context and frees it in
 *    lcp_destroy.  Caller buffers are never freed or retained.
 *  - Every entry point returns an lcp_status; nothing aborts or traps.  On
 *    error, lcp_last_error(ctx) returns a message (thread-local for NULL ctx).
 */
#ifndef LCP_GB300_H
#define LCP_GB300_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LCP_API __attribute__((visibility("default")))
#else
#define LCP_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  LCP_OK = 0,
  LCP_ERR_INVALID_ARG = -1,   /* bad size, pointer or option */
  LCP_ERR_OOM = -2,           /* device allocation failed */
  LCP_ERR_CUDA = -3,          /* a CUDA call failed; see lcp_last_error */
  LCP_ERR_NOT_CONVERGED = -4, /* iteration limit hit; outputs hold the best iterate */
  LCP_ERR_NUMERICAL = -5,     /* NaN/Inf or a breakdown (e.g. non-positive curvature) */
  LCP_ERR_TIMEOUT = -6,       /* a bounded device wait expired */
  LCP_ERR_REJECTED = -8       /* admission refused (memory budget) */
} lcp_status;

enum { LCP_FP64 = 0, LCP_MIXED = 1 };          /* precision of the stresslet sums */
enum { LCP_DF64 = 2 };                          /* double-FP32 sums (refinement residuals, ~1e-13) */
enum { LCP_MONO_PQN = 0, LCP_BI_PQN = 1 };     /* Algorithm 1 / Algorithm 4 */
enum { LCP_BB_PGD = 2 };                        /* baseline of Sec. 6: PGD with the Barzilai-Borwein step */
enum { LCP_HIGH = 0, LCP_LOW_RPY = 1 };        /* mobility fidelity */
enum { LCP_LOW_BIE = 2 };                       /* the boundary-integral mobility on the coarse low-fidelity grid */
enum { LCP_WARM_SLIP = 1, LCP_WARM_FORCES = 2, LCP_WARM_NO_INIT = 4 };  /* lcp_config.warm_start flags */

typedef struct {
  int n_theta, n_phi;       /* node grid per sphere; n_phi must be even */
  double radius;            /* hydrodynamic radius a of the boundary-integral surfaces */
  double contact_radius;    /* steric radius: gap_l = |c_j - c_i| - 2 contact_radius */
  double viscosity;         /* mu */
  double dt;                /* time step of Eq. (dvi) */
  double delta;             /* collisional threshold of Eq. (collisional-set) */
  int precision;            /* LCP_FP64 or LCP_MIXED */
  double gmres_tol;         /* relative residual of each mobility solve */
  int gmres_restart;        /* Krylov basis size m of GMRES(m) */
  int gmres_maxit;          /* total GMRES iterations per solve */
  double inner_tol;         /* LCP_MIXED: relative tolerance of each FP32-operator GMRES */
  int ir_maxit;             /* LCP_MIXED: maximum refinement sweeps */
  int kmax;                 /* PQN outer iteration limit */
  int kmax_inner;           /* Bi-PQN subproblem / low-fidelity init iteration limit */
  int memory;               /* quasi-Newton pairs kept, 1..48 (oldest quarter dropped when full) */
  int ssn_maxit;            /* semi-smooth Newton iterations per prox */
  double forcing;           /* Bi-PQN subproblem tolerance = max(0.1 tol, forcing * kkt) */
  int precondition;         /* 1: flexible GMRES with the isolated-sphere block-diagonal inverse */
  int residual_precision;   /* LCP_MIXED refinement residuals: LCP_FP64 or LCP_DF64 (default) */
  int autotune;             /* 1: time the FP32 pair-kernel variants at set-up, keep the fastest per size class */
  int own_stream;           /* 1: the context creates (and destroys) its own non-blocking stream */
  int h0_scaling;           /* 0: B_0 = H_0 = I as printed in Algorithm 1; 1: B_0 = delta I with
                               delta = y^T s / s^T s of the first step (H_0 = I / delta) */
  void* cuda_stream;        /* cudaStream_t to run on; NULL = the legacy default stream */
  /* Low-fidelity operator of Bi-PQN (Sec. 5.1: fidelity by coarseness of the
   * discretisation).  lowfi_n_theta = 0: the pairwise RPY mobility.  > 0: the
   * same boundary-integral mobility on a coarser lowfi_n_theta x lowfi_n_phi
   * grid, its GMRES solved with FP32 sums (no refinement) to relative residual
   * lowfi_tol (the paper's low-fidelity eps_gmres). */
  int lowfi_n_theta, lowfi_n_phi;
  double lowfi_tol;
  /* Bi-PQN's low-fidelity initialisation (Sec. 5.2, solved "approximately"):
   * stops at max(tol, init_forcing * its initial KKT error); 0 = to tol. */
  double init_forcing;
  /* Warm starts along a trajectory (lcp_step), a combination of flags:
   * LCP_WARM_SLIP: the slip solve for U_nc starts GMRES from the previous step's
   * density instead of zero; LCP_WARM_FORCES: the next LCP solve (when the caller
   * gives no x0) starts from the previous step's force on every contact whose
   * body pair persists (0 on new contacts).  Consecutive configurations differ by
   * one time step, so both starts are close.  LCP_WARM_NO_INIT (with
   * LCP_WARM_FORCES): Bi-PQN takes the carried forces as x(0) instead of running
   * its low-fidelity initialisation from them (Algorithm 4 runs it; off by
   * default).  Default LCP_WARM_FORCES: in mixed
   * precision a started slip solve needs one more double-float residual than it
   * saves in FP32 iterations; in FP64 mode LCP_WARM_SLIP saves outright.  The
   * paper names reuse across solves as future work ("Conclusions and Future
   * Work"); 0 = always start from zero. */
  int warm_start;
  /* Reuse across the mobility solves of one configuration (the MVPs of one LCP
   * share K + P and their right-hand sides differ little): the context keeps
   * up to `recycle` pairs (psi_k, w_k = (K + P) psi_k, w orthonormal) from its
   * earlier solves and starts each solve from the Galerkin projection
   * phi0 = Psi W^T rhs when that predicts at least a tenfold smaller residual
   * (Fischer's projection method for successive right-hand sides); when all
   * pairs are in use the set restarts from the newest solve.  Cleared when the
   * configuration changes and at the start of every LCP solve, so a solve's
   * result depends only on its configuration.  It pays where successive
   * right-hand sides are close (repeated or combined forces in mobility_apply);
   * the MVPs of a PQN solve multiply new search directions, which the kept
   * pairs do not predict.  The paper names reuse across solves as future work.
   * 0 = off (default); at most gmres_restart. */
  int recycle;
  /* 1: high-order quadrature of each sphere's self-interaction.  The pair sums
   * take a sphere's double layer on its own nodes by the product rule with the
   * global singularity subtraction (exact on rigid motions, algebraically
   * accurate otherwise); this adds one dense 3 ns x 3 ns correction, the same
   * for every body (all share the template), computed once per grid from a
   * polar quadrature about each node and the band-limited projection of the
   * density, and applied per body as a small GEMM in the sums' precision.  It
   * makes the two-sphere mobilities converge spectrally (the isolated-sphere
   * preconditioner includes it).  1 (default); 0: the product rule only. */
  int self_quadrature;
} lcp_config;

typedef struct {
  int i, j;                 /* bodies, i < j */
  double normal[3];         /* (c_j - c_i) / |c_j - c_i| */
  double gap;               /* |c_j - c_i| - 2 contact_radius */
} lcp_contact;

typedef struct {
  int converged;            /* 1 if ||min(x, A x + b)||_2 <= tol */
  int iterations;           /* outer PQN iterations */
  int hi_mvps, lo_mvps;     /* high-/low-fidelity matrix-vector products with A */
  int inner_iterations;     /* Bi-PQN: subproblem iterations, summed */
  int gmres_iterations;     /* GMRES iterations of all high-fidelity solves, summed */
  int fp64_applies;         /* FP64 stresslet applications */
  int fp32_applies;         /* FP32 stresslet applications */
  double kkt_abs;           /* ||min(x, g)||_2 with the final gradient g */
  double kkt_dot;           /* <x, g> (the test of Algorithms 1 and 4) */
  double e_mvps;            /* hi + lo * (mean lo time / mean hi time), Sec. 6 */
  double hi_mvp_seconds;    /* mean wall time of one high-fidelity MVP */
  double lo_mvp_seconds;    /* mean wall time of one low-fidelity MVP */
  double seconds;           /* wall time of the solve */
  int df64_applies;         /* double-FP32 stresslet applications (refinement residuals) */
  int resets;               /* quasi-Newton memory resets (non-descent direction) */
  int ssn_iterations;       /* semi-smooth Newton iterations of all prox evaluations */
  int ssn_fallbacks;        /* prox evaluations that needed the projected Gauss-Seidel fallback */
  double h0_delta;          /* scale delta of B_0 = delta I (1 when unscaled) */
  int unc_gmres_iterations; /* GMRES iterations of the slip solve that produced this LCP's b */
  int unc_warm_started;     /* 1 if that slip solve started from the previous step's density */
  int lo_gmres_iterations;  /* GMRES iterations of the coarse-grid low-fidelity solves, summed */
  int recycled_solves;      /* mobility solves (both grids) started from the projection (cfg.recycle) */
  int warm_x0;              /* 1 if the solve started from the previous time step's forces */
} lcp_stats;

typedef struct lcp_ctx lcp_ctx;   /* opaque, library-owned */

/* Fills cfg with defaults (grid 9 x 18, a = 1, contact radius 1.25, mu = 1,
 * dt = 0.01, delta = 0.05, FP64, GMRES tol 1e-12, restart 60, ...). */
LCP_API void lcp_default_config(lcp_config* cfg);

/* Builds a context for one configuration (Sec. 3, Eqs. collisional-set, LCP,
 * defAandb).  centers: host [M*3].  axes: host [M*3] unit Janus axes, or NULL
 * for no active slip.  contacts: n_contacts caller contacts (host), or NULL to
 * detect every pair with gap <= delta on the GPU (lexicographic order).
 * Computes the quadrature, the contact matrix D (CSR both ways), the
 * non-collisional velocity U_nc (one slip-driven mobility solve) and
 * b = gap / dt + D^T U_nc.  Allocates all device state; *out receives the
 * context (NULL on failure, message via lcp_last_error(NULL)). */
LCP_API int lcp_setup(const lcp_config* cfg, int n_bodies, const double* centers, const double* axes,
              int n_contacts, const lcp_contact* contacts, lcp_ctx** out);

/* Re-configures the context for new centres (same M and grid): uploads
 * centers [M*3] and axes [M*3] (NULL: no slip), detects the contacts (or takes
 * n_contacts caller contacts), rebuilds D, U_nc and b.  Reuses the device
 * buffers; the contact-sized ones grow when n exceeds their capacity.  This
 * is the per-time-step entry of a trajectory (Eq. dvi). */
LCP_API int lcp_update(lcp_ctx* ctx, const double* centers, const double* axes, int n_contacts,
               const lcp_contact* contacts);
/* Same with device pointers centers [M*3], axes [M*3] or NULL; contacts are
 * always detected. */
LCP_API int lcp_update_dev(lcp_ctx* ctx, const double* centers, const double* axes);

/* One forward Euler step of Eq. (dvi) after lcp_solve: body velocities
 * U = U_nc + M D x (M D x accumulated during the solve with the same MVP reuse
 * as the gradient, so no extra mobility solve), centres c += dt U, Janus axes
 * rotated by the angle |Omega| dt about Omega; then the context is
 * re-configured for the new positions (contacts, D, U_nc, b) as by lcp_update.
 * centers_out [M*3] / axes_out [M*3]: optional host copies of the new state. */
LCP_API int lcp_step(lcp_ctx* ctx, double dt, double* centers_out, double* axes_out);

/* Device bytes held by the context (its footprint for admission control). */
LCP_API int lcp_footprint(const lcp_ctx* ctx, size_t* bytes);

/* Upper estimate of lcp_footprint for a context of n_bodies bodies and about
 * n_contacts contacts with this config, computable before creating it. */
LCP_API int lcp_footprint_estimate(const lcp_config* cfg, int n_bodies, int n_contacts, size_t* bytes);

/* Name of the FP32 pair-kernel variant in use: "sym*" = the symmetric pair sum
 * (one evaluation per unordered node pair; the default is "sym_a4"), "t2c8" = the
 * plain sum with 2 targets per thread and 8 source bodies per shared-memory
 * tile, and so on; chosen by the autotuner when cfg.autotune is set.  The
 * symmetric variants (and the symmetric double-float residual sum that goes
 * with them) keep one reverse row per (512-node target block, later body),
 * about 1.4 KB per pair of bodies at 242 nodes each; where those rows would
 * exceed a quarter of the device's memory (above about 7 000 bodies at 242
 * nodes) they are not set up and the plain variants serve the context. */
LCP_API const char* lcp_kernel_variant(const lcp_ctx* ctx);

/* Forces the FP32 pair-kernel variant by name (one of the names
 * lcp_kernel_variant can return).  The operator is the same discrete K + P;
 * variants differ in summation order (FP32 rounding) and speed.  Errors:
 * LCP_ERR_INVALID_ARG for an unknown name or a variant that does not fit this
 * context's size. */
LCP_API int lcp_select_kernel_variant(lcp_ctx* ctx, const char* name);

/* Batched solves: solves count independent contexts with `workers` host
 * threads; contexts created with own_stream run concurrently on the GPU.
 * x_dev: optional array of device pointers [n_i] (NULL entries or NULL array:
 * results stay in the contexts).  stats: optional [count].  statuses [count]
 * receives each solve's status; returns the first non-OK status or LCP_OK.
 * Results are identical to solving the contexts one at a time. */
LCP_API int lcp_batch_solve(lcp_ctx** ctxs, int count, int method, double tol, double* const* x_dev, lcp_stats* stats,
                    int* statuses, int workers);

/* Continuous-batching solve server (the paper describes no serving layer; it
 * serves many simulations at once): `workers` host threads take requests as they arrive and
 * run them concurrently (each context on its own stream), while later
 * requests keep arriving.
 *
 * Simulations owned by the server (the request carries the problem):
 *   lcp_server_open registers a simulation (configuration, bodies, centres,
 *   optional Janus axes; copied) and allocates nothing on the device.
 *   lcp_server_request asks for a solve of its current LCP; with step_dt > 0
 *   the simulation then advances one time step (lcp_step), so the next
 *   request solves the next configuration.  The server creates the
 *   simulation's context on its first request, but only once the context's
 *   estimated device footprint (lcp_footprint_estimate with six contacts per
 *   body) fits hbm_budget_bytes next to everything resident; until then the
 *   request is held, first come first admitted.  The context then stays
 *   resident (geometry, Krylov and quasi-Newton state) for the simulation's
 *   later requests.  A simulation whose estimate alone exceeds the budget is
 *   rejected (LCP_ERR_REJECTED).  lcp_server_close (after its last request has
 *   been polled) destroys the context, returns its budget and admits held
 *   requests.  One request per simulation at a time (LCP_ERR_INVALID_ARG).
 *
 * Caller-owned contexts: lcp_server_admit counts lcp_footprint against the
 * budget (LCP_ERR_REJECTED when it would be exceeded), lcp_server_submit
 * queues a solve of an admitted context, lcp_server_release returns the budget
 * (and admits held simulation requests).
 *
 * lcp_server_poll waits at most timeout_us for the ticket (LCP_ERR_TIMEOUT
 * otherwise), copies x (host, at least n doubles) and the stats, and returns
 * the solve's (or, after a solve, the time step's) status.  lcp_server_stats:
 * bytes counted against the budget, requests waiting (held or queued), and
 * requests running. */
typedef struct lcp_server lcp_server;
LCP_API int lcp_server_create(int workers, size_t hbm_budget_bytes, lcp_server** out);
LCP_API void lcp_server_destroy(lcp_server* srv);
LCP_API int lcp_server_admit(lcp_server* srv, lcp_ctx* ctx);
LCP_API int lcp_server_release(lcp_server* srv, lcp_ctx* ctx);
LCP_API int lcp_server_submit(lcp_server* srv, lcp_ctx* ctx, int method, double tol, uint64_t* ticket);
LCP_API int lcp_server_poll(lcp_server* srv, uint64_t ticket, double* x, int x_len, lcp_stats* st, int timeout_us);
LCP_API int lcp_server_stats(lcp_server* srv, size_t* resident_bytes, int* queued, int* in_flight);
LCP_API int lcp_server_open(lcp_server* srv, const lcp_config* cfg, int n_bodies, const double* centers,
                            const double* axes, uint64_t* sim);
LCP_API int lcp_server_request(lcp_server* srv, uint64_t sim, int method, double tol, double step_dt,
                               uint64_t* ticket);
LCP_API int lcp_server_close(lcp_server* srv, uint64_t sim);

/* Kernel timing.  lcp_profile(ctx, 1) clears the record and starts timing
 * every stresslet-sum launch with CUDA events on the context's stream (inside
 * the captured GMRES steps too: those graphs then record their own events,
 * read after each replay, and replay as usual);
 * lcp_profile(ctx, 0) stops and clears.  lcp_profile_read returns the number
 * of launches of a kind (0 = FP32, 1 = FP64, 2 = double-FP32 pair sum; 3 = PQN direction,
 * 4 = PQN step, 5 = quasi-Newton rebuild, 6 = low-fidelity MVP) and their
 * summed duration in milliseconds (synchronises the stream). */
LCP_API int lcp_profile(lcp_ctx* ctx, int enable);
LCP_API int lcp_profile_read(lcp_ctx* ctx, int kind, int* count, double* total_ms);

/* The self-interaction correction of cfg.self_quadrature for one sphere
 * template (Gauss-Legendre n_theta x uniform n_phi nodes of radius `radius`,
 * node q = j n_phi + k with cos(theta_j) ascending): C, host [3 ns x 3 ns]
 * row-major (ns = n_theta n_phi), (C phi)_{3p+i} = sum_q C[3p+i][3q+j] phi_{3q+j}
 * is added to (K phi) on every body.  Computed on the host (cached per grid).
 * LCP_ERR_INVALID_ARG for a grid lcp_setup would refuse or a NULL C. */
LCP_API int lcp_self_correction(int n_theta, int n_phi, double radius, double* C);

/* Number of kernels this context has launched since lcp_setup. */
LCP_API int lcp_launch_count(const lcp_ctx* ctx, unsigned long long* count);

/* Mobility solves of one grid since lcp_setup (fidelity LCP_HIGH, or
 * LCP_LOW_BIE for the coarse low-fidelity grid): *solves solves (slip solves,
 * MVPs and direct mobility calls), *gmres_iterations their GMRES iterations,
 * *recycled those started from the projection on earlier solves
 * (cfg.recycle).  Host counters; no device work.  LCP_ERR_INVALID_ARG for
 * another fidelity or a missing coarse grid. */
LCP_API int lcp_solve_counters(const lcp_ctx* ctx, int fidelity, long long* solves, long long* gmres_iterations,
                               long long* recycled);

/* Frees every device buffer of the context.  NULL is ignored. */
LCP_API void lcp_destroy(lcp_ctx* ctx);

/* Message of the last failure on ctx (or of the calling thread's last failed
 * lcp_setup when ctx is NULL).  Valid until the next call on ctx. */
LCP_API const char* lcp_last_error(const lcp_ctx* ctx);

/* Sizes: bodies M, nodes N, contacts n. */
LCP_API int lcp_sizes(const lcp_ctx* ctx, int* n_bodies, int* n_nodes, int* n_contacts);

/* Copies the contacts (host [n]), b (host [n]) or U_nc (host [M*6]). */
LCP_API int lcp_get_contacts(lcp_ctx* ctx, lcp_contact* out);
LCP_API int lcp_get_b(lcp_ctx* ctx, double* b);
LCP_API int lcp_get_unc(lcp_ctx* ctx, double* U_nc);

/* U = M F (Sec. 2, Eq. mobility).  FT, UO: host [M*6].  include_slip adds the
 * Janus slip-driven part (U_nc for FT = 0).  fidelity: LCP_HIGH (boundary
 * integral, GMRES, precision of the context), LCP_LOW_RPY (pairwise RPY) or
 * LCP_LOW_BIE (boundary integral on the coarse grid; LCP_ERR_INVALID_ARG when
 * cfg.lowfi_n_theta = 0).  Only LCP_HIGH has the slip term. */
LCP_API int mobility_apply(lcp_ctx* ctx, const double* FT, double* UO, int include_slip, int fidelity);
/* Same on device pointers FT [M*6], UO [M*6], on the context's stream. */
LCP_API int mobility_apply_dev(lcp_ctx* ctx, const double* FT, double* UO, int include_slip, int fidelity);

/* One matrix-vector product A[x] = D^T M D x (Sec. 3, Eq. defAandb) of the
 * given fidelity (LCP_HIGH, LCP_LOW_RPY or LCP_LOW_BIE).  Host x [n], Ax [n].
 * Bi-PQN uses LCP_LOW_BIE when cfg.lowfi_n_theta > 0, else LCP_LOW_RPY. */
LCP_API int lcp_apply_A(lcp_ctx* ctx, const double* x, double* Ax, int fidelity);

/* Solves 0 <= x perp A x + b >= 0 by Mono-PQN (Algorithm 1), Bi-PQN
 * (Algorithm 4) or the BB-PGD baseline (Sec. 6, Eq. spectralStepSize, first
 * step tau_0 = 3 pi mu a) to ||min(x, A x + b)||_2 <= tol.  x0: host [n] initial guess
 * (projected onto x >= 0) or NULL for 0.  x: host [n] result.  st: optional.
 * Returns LCP_ERR_NOT_CONVERGED (x = last iterate) if kmax is reached. */
LCP_API int lcp_solve(lcp_ctx* ctx, int method, double tol, const double* x0, double* x, lcp_stats* st);
/* Same with device pointers x0 (or NULL) and x, both [n] FP64. */
LCP_API int lcp_solve_dev(lcp_ctx* ctx, int method, double tol, const double* x0, double* x, lcp_stats* st);

/* Building blocks of the mobility solve, on device pointers and the context's
 * stream (used by the parity tests):
 *   lcp_stokes_apply_dev: out = (K + P) phi, phi/out [N*3], precision
 *     LCP_FP64, LCP_MIXED (FP32 pair sums, compensated accumulation) or
 *     LCP_DF64 (double-FP32 pair sums);
 *   lcp_stokes_rhs_dev: rhs = s - S[F, T] at the nodes, FT [M*6], rhs [N*3];
 *   lcp_rigid_velocity_dev: UO = -(rigid coefficients of P phi), UO [M*6]. */
LCP_API int lcp_stokes_apply_dev(lcp_ctx* ctx, const double* phi, double* out, int precision);
LCP_API int lcp_stokes_rhs_dev(lcp_ctx* ctx, const double* FT, int include_slip, double* rhs);
LCP_API int lcp_rigid_velocity_dev(lcp_ctx* ctx, const double* phi, double* UO);

/* Allocation-free stresslet apply: out = (K + P) phi for n_bodies spheres of
 * radius `radius` on an n_theta x n_phi grid, with no context and no memory
 * allocation of any kind (no cudaMalloc, no cudaFree, no library routine that
 * allocates).  It is meant for callers that cannot allocate GPU memory:
 * code running inside an allocator or memory-pool callback, hosts that give
 * the whole device budget to another component, or real-time loops where an
 * allocation could block or fail.  The paper has no counterpart; it is the
 * same operator as lcp_stokes_apply_dev with self_quadrature = 0 (the product
 * rule for the self-interaction).
 *   centers [M*3], phi [N*3] and out [N*3] are device pointers (FP64), N =
 *   n_bodies * n_theta * n_phi; precision LCP_FP64 or LCP_MIXED; cuda_stream
 *   is a cudaStream_t (NULL = legacy default stream).  Returns after the
 *   result is complete (synchronises that stream).
 * Limits (the size of a fixed scratch area of about 1.8 MB compiled into the
 * library, held on every GPU that loads it until the process exits): at most
 * 128 bodies, 512 nodes per sphere and 16384 nodes in total, n_phi even.
 * Larger sizes return LCP_ERR_INVALID_ARG; the message is available from
 * lcp_last_error(NULL).
 * The first call on a device looks up the scratch area's device address;
 * make that first call before any stream capture.  The address (like the
 * raised shared-memory limits of the pair kernels) is kept for the life of
 * the process and does not survive cudaDeviceReset: do not call this entry
 * point after a reset of a device it has used.  All calls share the
 * scratch area: calls whose GPU work may overlap (other streams or threads
 * without ordering) race and must be serialised by the caller. */
LCP_API int lcp_stokes_apply_noalloc(int n_bodies, int n_theta, int n_phi, double radius, const double* centers,
                             const double* phi, double* out, int precision, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif
