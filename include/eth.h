/*
 * eth.h -- C ABI of the GB300 enriched Taylor--Hood (Q2--Q1*) Stokes/Oseen solver.
 *
 * Problem (Pestana & Silvester, Sec. 2 "Stokes problem" and Sec. 3 "Oseen
 * problem"): on a uniform n x n grid of rectangles of [x0,x1] x [y0,y1],
 * velocity in (Q2)^2 and pressure in the two-field frame Q1 + P0
 * (Sec. 2.1, Eq. eth_pressure_space / eth_spec), solve
 *
 *     [ F  B^T ] [u]   [f]        F = nu*A          (Stokes, Eq. saddle_point)
 *     [ B  0   ] [p] = [g]        F = nu*A + N(w)   (Oseen,  Eq. oseen-system)
 *
 * with b(u,p) = -int p div u, Dirichlet velocity on the whole boundary, and a
 * pressure defined only modulo span{e1, e0} (constant Q1 and constant P0
 * pressure, Sec. 2.1 Eq. pressure_null_vector and Sec. 3 Test problem 4).
 *
 * Layout (all vectors FP64, device-resident unless stated otherwise):
 *   Q2 lattice (2n+1)^2 nodes, node (i,j) at (x0 + i*hx/2, y0 + j*hy/2),
 *   flat index j*(2n+1) + i.  Velocity u = [u_x (N_v); u_y (N_v)], N_v = (2n+1)^2.
 *   Pressure p = [p1 ((n+1)^2 Q1 coefficients); p0 (n^2 element constants)],
 *   element (ex,ey) has index ey*n + ex (Eq. function_basis ordering).
 *   Full-system vectors are [u; p] of length N_t = 2 N_v + (n+1)^2 + n^2.
 *
 * Dirichlet treatment: the full lattice is kept; boundary velocity rows of K
 * are identity rows and boundary velocity columns are zero elsewhere.
 *
 * Ownership: the caller owns every pointer argument and never hands it to the
 * library; the handle owns its device workspace (multigrid hierarchy, Krylov
 * basis), allocated at eth_grid_create and freed by eth_grid_destroy.
 * Streams: device work of a handle is ordered on the stream given at creation:
 * eth_apply enqueues on it and returns; eth_solve* run on the handle's internal
 * streams (graphs need a capturable stream), which wait for the work already on
 * the user stream and are joined back to it, and synchronise once at the end to
 * fill eth_stats.
 * Devices: a handle belongs to the CUDA device that is current when it is
 * created (its workspace lives there, and its stream must belong to it); every
 * call on a handle makes that device current for its duration and restores the
 * caller's current device on return.
 * Errors: every call returns an eth_status; no exception crosses the ABI.
 * eth_last_error() returns a thread-local message for the last failure.
 */
#ifndef ETH_H
#define ETH_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct eth_grid eth_grid;
typedef struct eth_batch eth_batch;
typedef struct eth_mgrid eth_mgrid;

typedef enum {
  ETH_OK = 0,
  ETH_EINVAL = 1,         /* bad argument (size, pointer, option)            */
  ETH_ENOMEM = 2,         /* device allocation failed                        */
  ETH_ECUDA = 3,          /* CUDA runtime error                              */
  ETH_ENOTCONV = 4,       /* tolerance not reached within maxit              */
  ETH_EBREAKDOWN = 5,     /* Krylov breakdown (e.g. MINRES gamma^2 <= 0)     */
  ETH_EINCONSISTENT = 6,  /* right-hand side has a null-space component      */
  ETH_ETIMEOUT = 7,       /* bounded device wait gave up                     */
  ETH_ENAN = 8            /* NaN or Inf in a residual                        */
} eth_status;

typedef enum { ETH_STOKES = 0, ETH_OSEEN = 1 } eth_kind;

/* Operators of eth_apply.  K: full system (velocity Dirichlet rows identity);
 * KT: its transpose (element-transposed convection); A: nu*A (Dirichlet);
 * F: nu*A + N(w) (Dirichlet); B: [B1;B0] D_I u; BT: D_I B^T p;
 * MQ: M_Q = [Qk R^T; R Q0] (Sec. 2.3); MV: per-component Q2 mass (no BC);
 * K1: reduced system [F B1^T; B1 0] on [u; p1] (Sec. 3.1 Eq. reduced-system);
 * K1T: its transpose [F^T B1^T; B1 0]. */
typedef enum {
  ETH_OP_K = 0, ETH_OP_KT = 1, ETH_OP_A = 2, ETH_OP_F = 3, ETH_OP_B = 4,
  ETH_OP_BT = 5, ETH_OP_MQ = 6, ETH_OP_MV = 7, ETH_OP_K1 = 8, ETH_OP_K1T = 9
} eth_op;

/* Precision of the internal arithmetic. */
typedef enum { ETH_FP64 = 0, ETH_MIXED = 1 } eth_precision;

/* Approximation of the singular pressure mass solve M_Q^+ (Sec. 2.2-2.3):
 * VCYCLE the block elimination of Q0 with one Q1 V-cycle (default); EXACT inner
 * PCG to inner_tol (the P_1 form of Sec. 2.4); CHEB the Chebyshev semi-iteration
 * on multicolour symmetric Gauss-Seidel (the M_cheb block of P_2, Sec. 2.3-2.4). */
typedef enum { ETH_MQ_VCYCLE = 0, ETH_MQ_EXACT = 1, ETH_MQ_CHEB = 2 } eth_mq_mode;

typedef struct {
  double tol;              /* relative true residual ||b-Kx||/||b||          */
  int maxit;               /* total Krylov iterations (all stages/passes)    */
  int restart;             /* GMRES restart length (Oseen)                   */
  double c_stage;          /* two-stage factor c (Sec. 3.1), Step I to c*tol */
  int precision;           /* eth_precision                                  */
  int mg_pre, mg_post;     /* smoothing sweeps of the velocity V-cycle       */
  int mg_min_n;            /* coarsest grid size of the hierarchies (dense
                              solve there); 0: 4 for Stokes, 8 for Oseen     */
  int mq_mode;             /* eth_mq_mode                                    */
  int a_exact;             /* 1: exact velocity solves (inner PCG), P_1 form */
  double inner_tol;        /* inner exact-solve tolerance when exact         */
  double refine_inner_tol; /* mixed: relative tolerance of each inner solve  */
  int graph;               /* 0: stream launches; 1: CUDA graphs, the MINRES
                              loop run on the device by a conditional WHILE
                              node; 2: CUDA graphs of two MINRES iterations
                              replayed by the host (GMRES: 1 and 2 replay the
                              captured Arnoldi step)                        */
  int verbose;
  int autotune;            /* 1: before the first solve of a grid, time the
                              fused K apply with tiles of 32 x {4, 8, 16}
                              elements per CTA, the persistent 32 x 8 form
                              (mixed precision) and the warp-strip form with
                              {2, 4, 6, 8, 16} element rows per warp, and keep
                              the fastest (cached
                              per grid size, operator and precision for the
                              process), and for GMRES the basis vectors per
                              Gram-Schmidt pass in {4, 8, 16}; 0: warp strips
                              of 8 element rows, 16 vectors per pass         */
  int restart_max;         /* GMRES: when a restart cycle reduces the FP64
                              residual by less than a factor 2, the next
                              cycles use twice the restart length, up to
                              restart_max (<= 160); 0 or <= restart: fixed  */
  double mg_omega;         /* damping of the velocity multigrid's Jacobi
                              smoother (0 < omega < 2); 0: 0.9               */
  int oseen_prec;          /* Oseen grids: 0 the two-stage PCD method
                              (Sec. 3.1); 1 one GMRES run on the full system
                              with the LSC block-triangular preconditioner
                              M_3 (Sec. 3.2, Eq. nse-precon-lsc), plain LSC
                              (H = M)                                        */
  int lsc_cg;              /* LSC: conjugate-gradient steps of each solve with
                              the frame operator B M^{-1} B^T (block-diagonal
                              Q1 / cell-centred P0 V-cycle preconditioner);
                              0: 6                                           */
  int mq_cheb_steps;       /* ETH_MQ_CHEB: Chebyshev steps; 0: 20 (Sec. 2.4)  */
  double mq_cheb_a;        /* ETH_MQ_CHEB: lower end a of the Chebyshev
                              interval [a, 1] (smallest nonzero eigenvalue of
                              the SGS-preconditioned M_Q); 0: 0.655 / n^2     */
} eth_opts;

typedef struct {
  int iters_stage1, iters_stage2, refine_passes, iters_total;
  double relres_true;      /* FP64 ||b - K x|| / ||b|| at exit               */
  double relres0;          /* at entry                                       */
  double prop2_lhs, prop2_bound; /* Sec. 3.1 Prop. 2 at the stage switch   */
  double seconds;          /* wall time of the solve (device events)         */
  double alg_bytes;        /* algorithmic bytes moved (estimate)             */
  int status;              /* eth_status of the solve                        */
  int kernel_launches;     /* device kernels launched by the solve           */
  int escalations;         /* GMRES restart cycles that switched the Arnoldi
                              products of a mixed-precision solve to FP64
                              because the FP64 residual had grown (0 or 1 per
                              stage)                                         */
  int tile_rows;           /* element rows per tile of the fused K apply used */
  int tile_persistent;     /* 1: its persistent pipelined form was used;
                              2: the warp-strip form (tile_rows element rows
                              per warp)                                      */
} eth_stats;

/* Sizes of an n x n grid: N_v = (2n+1)^2, N_1 = (n+1)^2, N_0 = n^2.
 * Returns N_t = 2 N_v + N_1 + N_0, or -1 for n < 1. */
int eth_sizes(int n, int* nv, int* n1, int* n0);
const char* eth_status_string(eth_status s);
const char* eth_last_error(void);
void eth_default_opts(eth_opts* o);

/* Creates a handle for an n x n grid (n >= 2, n a multiple of 2) on
 * [x0,x1] x [y0,y1] and allocates its workspace.  cuda_stream is a
 * cudaStream_t (NULL = legacy default stream).  Sec. 2.1 / 3. */
eth_status eth_grid_create(int n, double x0, double x1, double y0, double y1,
                           eth_kind kind, void* cuda_stream, eth_grid** out);
void eth_grid_destroy(eth_grid* g);

/* Pins the tile of the fused K apply: 32 x rows elements per CTA, rows in
 * {4, 8, 16}, one tile per CTA; or, with persistent = 1 (rows = 8), a grid of
 * resident CTAs that walk over the tiles and copy the next tile's input
 * (cp.async) while computing the current one (FP32 element arithmetic only;
 * FP64 applies use 32 x 8 one tile per CTA); or, with persistent = 2, the
 * warp-strip form (the default): each warp walks `rows` element rows (2 to 32)
 * of a strip of 30 element columns, keeping the shared node row in
 * registers (FP32 or FP64 element arithmetic).  Turns the autotuner off for this
 * grid; rows = 0 restores the default and lets the next solve with
 * opts.autotune tune again.  Every apply gives bitwise the same K x whatever
 * the tile (each node sums its element contributions in one fixed order);
 * reductions group their partial sums by CTA.  ETH_EINVAL for other values or
 * when the shape needs more reduction partials than the grid holds.  The paper
 * has no counterpart. */
eth_status eth_grid_set_tile(eth_grid* g, int rows, int persistent);

/* Viscosity nu > 0 and, for ETH_OSEEN, the nodal Q2 wind w (device, 2*N_v
 * FP64, Sec. 3 "discrete wind w_h"); wind_dev must be NULL for ETH_STOKES.
 * Rebuilds the wind-dependent parts of the multigrid hierarchy. */
eth_status eth_set_coefficients(eth_grid* g, double nu, const double* wind_dev);

/* Right-hand side from the nodal Q2 body force f (device, 2*N_v FP64) and the
 * Dirichlet data (device, 2*N_v FP64, only boundary entries read):
 * b = [D_I (M_v f - F u_b) + D_B u_b ; -B u_b] (Sec. 2 Eq. saddle_point with
 * Dirichlet lifting).  Requires eth_set_coefficients first. */
eth_status eth_set_rhs(eth_grid* g, const double* f_nodal_dev, const double* ubc_dev);
/* Copies the assembled right-hand side b (N_t FP64) into b_dev. */
eth_status eth_get_rhs(eth_grid* g, double* b_dev);

/* Solves K x = b: Stokes by MINRES (Algorithm 1) with the block-diagonal
 * preconditioner (Eq. stokes_pre), Oseen by the two-stage PCD method
 * (Sec. 3.1).  The multigrid hierarchies halve n while it stays even, so the
 * solvers need n = c * 2^k with c <= 32 (ETH_EINVAL otherwise); the operator
 * applies take any even n.  u_dev (2*N_v) and p_dev (N_1 + N_0) hold the initial guess on
 * entry (boundary entries of u are overwritten by the Dirichlet data) and the
 * solution on exit, with sum(p1) = sum(p0) = 0.  stats may be NULL. */
eth_status eth_solve(eth_grid* g, const eth_opts* opts, double* u_dev,
                     double* p_dev, eth_stats* stats);

/* Same as eth_solve with HOST buffers: copies f_nodal and ubc (2*N_v each) in,
 * sets the right-hand side, solves from a zero initial guess and copies u and
 * p back.  All host<->device copies happen inside the call. */
eth_status eth_solve_host(eth_grid* g, const eth_opts* opts, const double* f_nodal_host,
                          const double* ubc_host, double* u_host, double* p_host,
                          eth_stats* stats);

/* Adjoint solve K^T [l_u; l_p] = [r_u; r_p].  Stokes: same solver (K
 * symmetric).  Oseen: the two-stage solver applied to K^T = [F^T B^T; B 0]
 * with PCD built on F1^T.  K^T is singular on the same pressure null space as K
 * (span{e1, e0}, Sec. 3 Test problem 4), so the solver removes the e1 and e0
 * components (the sums of the Q1 and P0 blocks) of r_p first, as eth_solve does
 * for its right-hand side; this is exactly the adjoint of the projection that
 * makes eth_solve's pressure canonical.  When the removed part exceeds
 * 1e-8 ||[r_u; r_p]|| the call returns ETH_EINCONSISTENT with the solution of
 * the projected system; l_p is canonical (zero block sums). */
eth_status eth_solve_adjoint(eth_grid* g, const eth_opts* opts, const double* ru_dev,
                             const double* rp_dev, double* lu_dev, double* lp_dev,
                             eth_stats* stats);

/* y = op(x) for one operator (see eth_op); fp32 != 0 selects FP32 element
 * arithmetic (inputs and outputs stay FP64).  Sizes: K, KT: N_t -> N_t;
 * A, F, MV: 2 N_v -> 2 N_v; B: 2 N_v -> N_1+N_0; BT: N_1+N_0 -> 2 N_v;
 * MQ: N_1+N_0 -> N_1+N_0; K1, K1T: 2 N_v+N_1 -> 2 N_v+N_1. */
eth_status eth_apply(eth_grid* g, eth_op op, int fp32, const double* x_dev, double* y_dev);

/* Gradients of J(u) = ||u - u_t||^2 from the adjoint velocity l_u (device,
 * 2 N_v; the solution of eth_solve_adjoint with r_u = 2(u - u_t), r_p = 0)
 * and the state velocity u (device, 2 N_v, boundary values included):
 *   grad_f  = M_v D_I l_u      (device, 2 N_v; d J / d f_nodal, f entering as M_v f)
 *   grad_nu = -(D_I l_u)^T A u (host scalar; d J / d nu, A the unscaled Laplacian)
 * D_I zeroes the Dirichlet nodes.  No counterpart in the paper: the
 * differentiation form wraps the solver (adjoint of K(nu) x = b(f, nu)). */
eth_status eth_adjoint_gradients(eth_grid* g, const double* lu_dev, const double* u_dev,
                                 double* grad_f_dev, double* grad_nu_host);

/* Allocation-free K apply with its dot product, for callers that cannot
 * allocate device memory (they run inside another framework's memory pool or
 * under a fixed memory budget, or must not call cudaMalloc after start-up) and
 * therefore cannot create an eth_grid.  Computes y = K x for the Stokes
 * operator (nu*A, Dirichlet velocity rows identity) of an n x n grid on
 * [x0,x1] x [y0,y1] and *dot_dev = <K x, x> (FP64), with FP32 element
 * arithmetic when fp32 != 0.  x_dev, y_dev: N_t FP64 device vectors; dot_dev:
 * one FP64 device value; all owned by the caller.  Nothing is allocated: the
 * reduction scratch is a fixed file-scope device array of 32768 block partials
 * (one per 32 x 8 element tile, ceil(n/31) * ceil(n/7) tiles, so every even n up
 * to 2666 fits; larger n returns ETH_EINVAL) that every GPU loading the library
 * holds until exit.  The first call on a device looks the array's address up
 * (cudaGetSymbolAddress) and should come before any stream capture.  All calls
 * share the array: calls whose kernels overlap on the GPU race.  The paper has
 * no counterpart of this entry point. */
eth_status eth_apply_k_dot_static(int n, double x0, double x1, double y0, double y1, double nu, int fp32,
                                  const double* x_dev, double* y_dev, double* dot_dev, void* cuda_stream);

/* Pressure convection-diffusion Schur approximation of Step I alone (Sec. 3.1,
 * Eq. discrete-commutator1x): zp = M_S^{-1} rp = Ap^+ F1 Q1^{-1} rp on the Q1
 * pressure, with Q1 the Q1 mass matrix, F1 = nu K1 + N1(w) the Q1
 * convection-diffusion matrix (adjoint != 0: its transpose, as the adjoint
 * Oseen solve uses), Ap = B1 Md^{-1} B1^T over interior velocity columns (Md
 * the diagonal of the velocity mass matrix) and Ap^+ its inverse on mean-free
 * vectors.  The Oseen solver applies -M_S^{-1} inside its block-triangular
 * preconditioner with 10 Chebyshev steps for Q1^{-1} and 2 PCG steps for Ap^+;
 * here cheb_steps (0..1000) and ap_its (1..1000) choose them, so large counts
 * give the exact block.  rp_dev, zp_dev: device, N_1 FP64 each (caller-owned);
 * zp has zero mean.  fp32 != 0 runs the inner steps in FP32.  g must be an
 * ETH_OSEEN grid with coefficients set; ETH_EINVAL otherwise.  Asynchronous on
 * g's stream. */
eth_status eth_apply_pcd(eth_grid* g, int adjoint, int fp32, int cheb_steps, int ap_its, const double* rp_dev,
                         double* zp_dev);

/* The cheap pressure-mass approximation of P_2 alone (Sec. 2.3-2.4): z = steps
 * steps of the Chebyshev semi-iteration on the interval [a, b] (a <= 0: 0.655 / n^2;
 * b <= 0: 1) preconditioned by symmetric Gauss-Seidel on M_Q in five colours (the
 * four parity classes of the Q1 nodes, then the P0 elements; forward, then back),
 * for M_Q z = r with r's component along k = [1; -1] removed first; z is returned
 * orthogonal to k (Euclidean).  r_dev, z_dev: device, N_1 + N_0 FP64 each
 * ([Q1; P0] layout, caller-owned).  fp32 != 0 runs the iteration in FP32.
 * ETH_EINVAL for steps outside 1..10000 or a >= b.  Asynchronous on g's stream. */
eth_status eth_apply_mqcheb(eth_grid* g, int fp32, int steps, double a, double b, const double* r_dev, double* z_dev);

/* Picard iteration for the steady Navier-Stokes problem (Sec. 3: the Oseen
 * systems are its linearisations).  g must be an ETH_OSEEN grid whose viscosity
 * was set with eth_set_coefficients (its wind is replaced).  Step 1 solves with
 * zero wind (the Stokes problem); step k+1 solves the Oseen problem with the
 * wind w = u_k.  f_nodal_dev, ubc_dev: device, 2*N_v FP64 (as eth_set_rhs).
 * u_dev, p_dev: device outputs (2*N_v, N_1+N_0), the last iterate.  nlres_host
 * (steps doubles, may be NULL): after step k the nonlinear residual
 * ||b(u_k) - K(u_k) [u_k; p_k]|| / ||b(u_k)|| of the system linearised at the
 * iterate itself (FP64 operator).  stats_host (steps entries, may be NULL): the
 * statistics of each Oseen solve.  Returns the first hard failure of a solve
 * (ETH_ENOTCONV of a step does not stop the iteration).  On return the grid's
 * coefficients and right-hand side are those linearised at the last iterate. */
eth_status eth_picard(eth_grid* g, const eth_opts* opts, const double* f_nodal_dev, const double* ubc_dev,
                      int steps, double* u_dev, double* p_dev, double* nlres_host, eth_stats* stats_host);

/* Capacity of the Lanczos record of a Stokes solve (iterations of its first MINRES run). */
#define ETH_LANCZOS_CAP 4096

/* Lanczos coefficients of the first MINRES run of the last Stokes solve on g
 * (Algorithm 1 runs a Lanczos process on P^{-1} K): delta_dev[j-1] = delta_j
 * (the diagonal of T_j) and gamma_dev[j-1] = gamma_{j+1} (the entry below it),
 * j = 1 .. min(k, cap), copied into device arrays of cap FP64 (either may be
 * NULL when cap is 0).  *k_host receives the number of recorded iterations (at
 * most ETH_LANCZOS_CAP; 0 before any Stokes solve).  With mixed precision and
 * iterative refinement only the first (longest) MINRES run is recorded.
 * Synchronises g's stream.  ETH_EINVAL for an Oseen grid or NULL pointers. */
eth_status eth_lanczos(eth_grid* g, int cap, double* delta_dev, double* gamma_dev, int* k_host);

/* EST-MINRES estimates of the discrete inf-sup constant gamma^2 (Sec. 2.4: the
 * smallest nonzero eigenvalue of B A^{-1} B^T v = lambda M_Q v, v orthogonal to
 * k).  From k Lanczos steps (device arrays in the layout of eth_lanczos) writes
 * est_dev[j-1] = theta^2 - theta for each j = 1 .. k, theta the negative
 * harmonic Ritz value of T_j closest to zero, or NaN while T_j has none (or is
 * singular).  With the exact block preconditioner P_1 (opts a_exact = 1, mq_mode
 * = ETH_MQ_EXACT) the estimates approach gamma^2 from above; with approximate
 * blocks they estimate the corresponding quantity of that preconditioner.
 * Asynchronous on g's stream; g only supplies the stream.  One warp per j:
 * each multisection round evaluates 32 Sturm counts of O(j) work. */
eth_status eth_est_infsup(eth_grid* g, const double* delta_dev, const double* gamma_dev, int k, double* est_dev);

/* ------------------------------------------------------------------------
 * Masked grids: inflow-outflow domains (Sec. 3, Test problem 3, the flow over
 * a step).  The domain is the union of the ACTIVE squares of an nx x ny grid of
 * square elements of side h on the box [x0, x0 + nx h] x [y0, y0 + ny h];
 * active_host[ey*nx + ex] != 0 marks element (ex, ey) active.  Unknowns live on
 * the full lattice of the box with the square-grid layout above (N_v =
 * (2nx+1)(2ny+1), N_1 = (nx+1)(ny+1), N_0 = nx ny); those of inactive nodes and
 * elements keep identity rows of K.  Node roles: a Q2 node is active when it
 * belongs to an active element, interior when every element around it is
 * active; the Dirichlet nodes are the active non-interior nodes except, with
 * outflow = 1, those strictly inside the right edge of the box (x = x0 + nx h),
 * where the weak form leaves the natural (do-nothing) outflow condition.
 * Velocity rows and columns of the Dirichlet and inactive nodes are treated as
 * on the square grid.  With an outflow boundary the pressure null space is
 * span{[0; k]}, k = 1 on the active Q1 nodes and -1 on the active elements.
 * Ownership, streams and errors as for eth_grid; all vectors FP64 device.
 * ------------------------------------------------------------------------ */

/* Creates a masked-grid handle (nx, ny >= 1, h > 0, outflow in {0, 1}, at
 * least one active element) on the current device; active_host holds nx*ny
 * bytes.  Builds the multigrid hierarchy of the velocity blocks: nx and ny are
 * halved while both are even and every 2 x 2 block of elements is wholly
 * active or inactive, and the coarsest level is solved exactly, so it may keep
 * at most 2048 free velocity nodes (ETH_EINVAL otherwise). */
eth_status eth_mgrid_create(int nx, int ny, double h, double x0, double y0, const unsigned char* active_host,
                            int outflow, void* cuda_stream, eth_mgrid** out);
void eth_mgrid_destroy(eth_mgrid* g);
/* The node roles of a masked grid computed on the host alone (no device work):
 * fixed_host and dirichlet_host receive N_v = (2nx+1)(2ny+1) bytes, q1_active_host
 * N_1 = (nx+1)(ny+1) bytes, with the definitions above (any output may be NULL).
 * The same routine sets the roles of every eth_mgrid level. */
eth_status eth_mask_roles(int nx, int ny, const unsigned char* active_host, int outflow, unsigned char* fixed_host,
                          unsigned char* dirichlet_host, unsigned char* q1_active_host);
/* N_v, N_1, N_0 and N_t = 2 N_v + N_1 + N_0 (any pointer may be NULL). */
eth_status eth_mgrid_sizes(const eth_mgrid* g, long long* nv, long long* n1, long long* n0, long long* nt);
/* Host copies of the node roles (N_v bytes: 1 on fixed = Dirichlet or inactive
 * velocity nodes; N_v bytes: 1 on Dirichlet nodes; N_1 bytes: 1 on active Q1
 * nodes), the number of multigrid levels and the free nodes of the coarsest
 * level; any pointer may be NULL. */
eth_status eth_mgrid_roles(const eth_mgrid* g, unsigned char* fixed_host, unsigned char* dirichlet_host,
                           unsigned char* q1_active_host, int* levels, int* coarse_free);
/* Viscosity nu > 0 and the nodal Q2 wind (device, 2 N_v; NULL: the Stokes
 * operator F = nu A). */
eth_status eth_mgrid_set_coefficients(eth_mgrid* g, double nu, const double* wind_dev);
/* y = op(x) on the masked grid: ETH_OP_K (N_t), ETH_OP_K1 (reduced system on
 * [u; p1], 2 N_v + N_1), ETH_OP_A, ETH_OP_F (2 N_v, Dirichlet and inactive rows
 * identity), ETH_OP_B (2 N_v -> N_1 + N_0, B D_I u over the active elements,
 * zero rows for inactive unknowns), ETH_OP_BT (N_1 + N_0 -> 2 N_v, D_I B^T p),
 * ETH_OP_MQ (the pressure mass over the active elements, zero rows for inactive
 * unknowns).  FP64 element arithmetic; other operators give ETH_EINVAL.
 * Asynchronous on the handle's stream. */
eth_status eth_mgrid_apply(eth_mgrid* g, eth_op op, const double* x_dev, double* y_dev);
/* Lifted right-hand side from the Dirichlet data u_b (device, 2 N_v; entries
 * off the Dirichlet nodes are ignored, no body force):
 * b = [D_I (-F u_b) + D_B u_b; -B u_b]. */
eth_status eth_mgrid_rhs(eth_mgrid* g, const double* ubc_dev, double* b_dev);
/* Solves K x = b (outflow = 1 only) by the two-stage PCD method of Sec. 3.1
 * from the lifted initial guess x0 = [D_B b_u; 0] (x's content on entry is
 * ignored): Step I restarted flexible GMRES(opts->restart) on the reduced
 * system with [F B1^T; 0 -M_S]^{-1}, M_S^{-1} = Ap^{-1} F1 Q1^{-1} (F1 = nu K1 +
 * N1(w) plus the inflow Robin term -int_{Gamma_in} (w.n) p q ds, Ap = B1 Md^{-1}
 * B1^T), to ||r|| <= c_stage tol ||b_red||; Step II GMRES on K with M_1 =
 * [F B^T; 0 -(1/nu) M_Q]^{-1} to tol ||b||.  F^{-1} is one V-cycle of the
 * masked multigrid (FP32 levels, damped Jacobi, streamline diffusion on the
 * levels of an Oseen operator); Ap^{-1} is three CG steps preconditioned by a
 * V-cycle of the Q1 Laplacian with a unit shift on the outflow column; M_Q^+
 * eliminates the P0 block and takes three CG steps on its Schur complement,
 * preconditioned by a natural-boundary Q1 V-cycle, with k projected out;
 * Q1^{-1} is ten Chebyshev steps.  Without a wind (the Stokes problem) Step I
 * uses the Stokes limit M_S^{-1} = nu Q1^{-1}.  With opts->graph != 0 the
 * preconditioner and operator of each Arnoldi step replay from a CUDA graph on
 * the handle's internal stream.  On exit k^T p = 0.  stats: stage iterations, the FP64 true
 * relative residual, the Prop. 2 quantities (||z*||^2 and its bound), status
 * ETH_ENOTCONV when tol was not reached within opts->maxit.  Synchronises. */
eth_status eth_mgrid_solve(eth_mgrid* g, const eth_opts* opts, const double* b_dev, double* x_dev, eth_stats* stats);
/* Picard iteration (Sec. 3, Test problem 3: the Oseen system after steps-1
 * fixed-point steps from the Stokes solution): step 1 solves the Stokes
 * problem, step k+1 the Oseen problem with the wind w = u_k, each by
 * eth_mgrid_solve with the right-hand side of u_b.  x_dev (N_t): the last
 * iterate; xs_dev (steps x N_t, may be NULL): every iterate; nlres_host (steps,
 * may be NULL): ||b(u_k) - K(u_k) x_k|| / ||b(u_k)||; stats_host (steps, may be
 * NULL).  The viscosity comes from eth_mgrid_set_coefficients; on return the
 * coefficients are those linearised at the last iterate. */
eth_status eth_mgrid_picard(eth_mgrid* g, const eth_opts* opts, const double* ubc_dev, int steps, double* x_dev,
                            double* xs_dev, double* nlres_host, eth_stats* stats_host);

/* Batched solves of independent instances (each created with its own handle,
 * all on the same stream). */
eth_status eth_batch_create(int count, eth_grid* const* grids, eth_batch** out);
eth_status eth_batch_solve(eth_batch* b, const eth_opts* opts, double* const* u_dev,
                           double* const* p_dev, eth_stats* stats_array);
void eth_batch_destroy(eth_batch* b);

#ifdef __cplusplus
}
#endif
#endif /* ETH_H */
