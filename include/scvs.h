/*
 * scvs.h - C ABI of a GB300 (sm_103a) solver for the spatio-spectral complex
 * Stokes method (SCVS) of Meng, Bhattacharjee & Esmaily, arXiv 2009.06725.
 *
 * A time-periodic creeping flow is expanded in Fourier modes
 * u = sum_k u_k e^{j omega_k t} (Eq. vaptransform); every mode k is the
 * independent complex boundary-value problem
 *     j omega_k rho u_k = -grad p_k + div(mu grad u_k),  div u_k = 0
 * (Eq. stokes_complex), discretised with unstabilised P2-P1 Taylor-Hood
 * Galerkin elements (Sec. 2.3) into
 *     A(omega_k) X_k = R_k,  A = [I_d (x) (mu K_s + j omega_k rho M_s), D; D^T, 0]
 * (Eqs. linear_sys, linear_sys_def, LS_construction).  This library builds the
 * sparsity pattern and the mode-independent real matrices once per mesh,
 * then solves all modes of a mesh together on one GPU and reconstructs the
 * time-domain field (Eq. sol_reconstruct).
 *
 * Conventions shared by every entry point
 *  - Return value: SCVS_OK (0) or a negative SCVS_ERR_* code; the message of
 *    the last failure is returned by scvs_last_error().
 *  - Host pointers are caller-owned; they are read or written during the call
 *    only and never retained.  Entry points named *_dev take device pointers
 *    (caller-owned, on the context's device) and work on the context's stream
 *    without host<->device copies.
 *  - Complex values are (re, im) pairs: scvs_c64 on the host, double2 / float2
 *    on the device.
 *  - Mesh arrays: xyz double [n_nodes][dim]; conn int32 [n_elem][6 or 10] in
 *    VTK quadratic-simplex order (vertices, then edge nodes (0,1),(1,2),(2,0)
 *    [, (0,3),(1,3),(2,3)]); vertex nodes are numbered first, so node ids
 *    0..n_vertices-1 are the P1 pressure dofs; tag uint8 [n_nodes] with bits
 *    SCVS_TAG_WALL / _INLET / _OUTLET / _NEUMANN.  A node tagged WALL or INLET
 *    is a Dirichlet node (all velocity components prescribed); the remaining
 *    boundary is traction-free (Eq. steady_stokes with h = 0) unless
 *    scvs_set_neumann gives a traction on faces tagged NEUMANN.
 *  - Dof ordering of one mode: velocity dof (node*dim + c), then the pressure
 *    dof of every vertex.  Device vectors hold every mode of a mesh
 *    interleaved: element (dof, k) at dof*ld + k with ld = scvs_mode_stride().
 *  - A context is not thread-safe; use one context per host thread/stream.
 */
#ifndef SCVS_H
#define SCVS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---------------------------------------------------- */
#define SCVS_OK 0
#define SCVS_ERR_ARG (-1)                /* bad argument / size / pointer */
#define SCVS_ERR_MESH (-2)               /* degenerate or inverted element, bad connectivity */
#define SCVS_ERR_PRESSURE_NULLSPACE (-3) /* no traction-free boundary: pressure undetermined */
#define SCVS_ERR_OOM (-4)                /* device allocation failed */
#define SCVS_ERR_CUDA (-5)               /* a CUDA call failed */
#define SCVS_ERR_STATE (-6)              /* call out of order (e.g. solve before set_modes) */
#define SCVS_ERR_TIMEOUT (-7)            /* a bounded device-side wait gave up */

/* ---- node tags --------------------------------------------------------- */
#define SCVS_TAG_WALL 1
#define SCVS_TAG_INLET 2
#define SCVS_TAG_OUTLET 4
#define SCVS_TAG_NEUMANN 8 /* traction boundary of scvs_set_neumann (not Dirichlet unless also WALL or INLET) */

/* ---- per-mode solve status (scvs_mode_report.status) -------------------- */
#define SCVS_CONVERGED 0  /* FP64 ||b - A x|| / ||b|| <= tol */
#define SCVS_MAX_ITER 1   /* cycle cap reached */
#define SCVS_STAGNATED 2  /* residual stopped decreasing */
#define SCVS_NON_FINITE 3 /* NaN/Inf met in this mode; other modes unaffected */

/* ---- options ----------------------------------------------------------- */
#define SCVS_PREC_MIXED 0 /* FP32 complex GMRES cycles inside FP64 refinement */
#define SCVS_PREC_FP64 1  /* all-FP64 GMRES */

#define SCVS_PC_BLOCK_CHEB 0   /* block-diagonal: Chebyshev-Jacobi polynomial of mu K + |omega| rho M for the
                                  velocity, Chebyshev Cahouet-Chabard mu M_p^-1 + j omega rho L_p^-1 for the pressure */
#define SCVS_PC_BLOCK_DIAG 1   /* block-diagonal, diagonal blocks only */
#define SCVS_PC_BLOCK_PMG 2    /* block-diagonal; velocity block by a two-level p-multigrid cycle: Chebyshev
                                  smoothing of mu K + |omega| rho M on P2 and a Chebyshev solve of the same
                                  operator on the nested P1 (vertex) space; pressure as BLOCK_CHEB */
#define SCVS_PC_TRI_PMG 3      /* block upper-triangular [A_u D; 0 S~] with the Schur complement approximation
                                  S~^-1 = -(mu M_p^-1 + j omega rho L_p^-1) (pressure first), then the velocity
                                  p-multigrid cycle of BLOCK_PMG on r_u - D z_p */
#define SCVS_PC_TRI_PMG_CS 4   /* TRI_PMG with an additive coarse correction of the Schur approximation:
                                  S~^-1 = -(mu M_p^-1 + j omega rho L_p^-1 + R_c (R_c^T D^T A~_u^-1 D R_c)^-1 R_c^T),
                                  R_c piecewise constant on graph aggregates of the vertices (opts.schur_agg per
                                  connected component), A~_u^-1 the velocity cycle of the preconditioner itself.
                                  The n_c x n_c matrices (real: the cycle is real-linear) are formed and inverted
                                  in FP64 on the first application after scvs_set_modes / scvs_set_physics /
                                  an option change (n_c/2 velocity cycles for all modes at once) */
#define SCVS_PC_AUTO 5         /* default: TRI_PMG_CS (with the default 16 aggregates per component the correction
                                  removes the iteration tails of long, thin, stenosed or branched domains, where the
                                  Cahouet-Chabard approximation alone degrades, and its set-up of 8 velocity cycles
                                  costs less than the iterations it saves even on the single 151k-node pipe) */

#define SCVS_GUESS_ZERO 0
#define SCVS_GUESS_MLP 1
#define SCVS_GUESS_CURRENT 2 /* start every mode from the solution the mesh holds (the last solve's, or the one
                                given by scvs_set_solution), its Dirichlet rows reset to g: warm start / resume */

#define SCVS_KRYLOV_FGMRES 0
#define SCVS_KRYLOV_COCR 1

typedef struct scvs_ctx scvs_ctx;
typedef struct { double re, im; } scvs_c64;

typedef struct {
  double tol;        /* relative residual target per mode (default 1e-8) */
  int32_t restart;   /* GMRES restart length m_r (default 30, max 64) */
  int32_t precision; /* SCVS_PREC_* (default MIXED) */
  int32_t precond;   /* SCVS_PC_* (default AUTO) */
  int32_t cheb_u;    /* Chebyshev degree of the velocity polynomial; with the p-multigrid kinds the degree of each
                        of the pre- and post-smoothers (default 2) */
  int32_t cheb_m;    /* Chebyshev degree, pressure mass (default 4) */
  int32_t cheb_l;    /* Chebyshev degree, pressure Laplacian, when lap_size = -1 (default 75) */
  int32_t max_cycles;/* cap on restart cycles; each cycle ends with an FP64 true residual (default 400) */
  int32_t guess;     /* SCVS_GUESS_* (default ZERO) */
  int32_t verbose;   /* 0 = silent */
  int32_t cheb_c;    /* Chebyshev degree of the coarse (P1) velocity solve of the p-multigrid kinds (default 16) */
  int32_t autotune;  /* 1 (default): time the launch shapes (modes per lane, row tile) of the FP32 SpMM and
                        Chebyshev kernels at scvs_set_modes and keep the fastest; the result is kept per
                        context for meshes of the same size (dim, nodes, vertices, nonzeros, mode
                        stride, components) and reused; 0: default shapes */
  void *stream;      /* cudaStream_t to run on; NULL = the legacy default stream */
  int32_t schur_agg; /* SCVS_PC_TRI_PMG_CS: aggregates per connected component of the vertex graph (1..512;
                        0 or default: 16); aggregates are grown to ceil(vertices / schur_agg) vertices, so a
                        component may end with somewhat more or fewer */
  int32_t stage;     /* staged gathers of the FP32 SpMM and fine Chebyshev kernels (row blocks of compact
                        footprint, the footprint copied into shared memory by TMA bulk copies or cp.async):
                        -1 (default): never (no row blocks are built; on the benchmark pipe the staged kernels
                        measured 3-5x slower than the L1-cached gathers); 0: the autotuner times them beside
                        the unstaged shapes and keeps the fastest; 4, 8, 16 or 32: always, with that many
                        modes per block (where the footprint fits shared memory) */
  int32_t krylov;    /* SCVS_KRYLOV_FGMRES (default): restarted flexible GMRES(restart); SCVS_KRYLOV_COCR:
                        preconditioned COCR, a short recurrence for complex symmetric systems (7 work vectors
                        per system), valid with the symmetric block-diagonal preconditioner kinds */
  int32_t inner_max; /* COCR iterations per FP64 refinement cycle (default 400) */
  int32_t graphs;    /* 1: replay every FGMRES Arnoldi step (preconditioner, SpMM, Arnoldi kernel) from a CUDA graph
                        captured on its first use after the first restart cycle of a solve; 0 (default): plain
                        launches.  Off while the kernel timers run.  A capture the runtime refuses falls back to
                        plain launches for the rest of the solve */
  int32_t lap_size;  /* pressure Laplacian L_p^-1 of the Schur approximation: 0 (default) or 1..4096: a symmetric
                        two-level cycle, S + coarse + S with S the lap_smooth-step Chebyshev-Jacobi polynomial on
                        [lambda/120, 1.1 lambda] and a Galerkin coarse level R (R^T L_p R)^-1 R^T on graph
                        aggregates of about this many vertices off the outlet (0: 32; at most 1024 aggregates
                        per connected component, larger components get larger aggregates); -1: one Chebyshev
                        polynomial of degree cheb_l on [lambda/3000, 1.1 lambda].  Meshes with a component
                        that no outlet vertex reaches keep the polynomial (scvs_lap_info) */
  int32_t lap_smooth;/* Chebyshev degree of each smoother of that cycle (1..64; 0 or default: 8) */
  int32_t reserved;
} scvs_opts;

/* Options of scvs_train_guess (learned initial guess). */
typedef struct {
  int32_t n_pod;             /* POD vectors per field block (velocity, pressure); default 32 */
  int32_t hidden;            /* width of the 3 hidden MLP layers; default 256 */
  int32_t steps;             /* Adam steps; default 3000 */
  int32_t batch;             /* minibatch size; default 256 */
  double lr;                 /* Adam learning rate; default 1e-3 (x0.3 after 1/2, x0.1 after 3/4 of the steps) */
  uint64_t seed;             /* weight initialisation and minibatch order; default 0 */
  int32_t max_pod_snapshots; /* snapshots entering the POD Gram matrix; default 512 */
  int32_t reserved;
} scvs_train_opts;

/* Result of one mode of one mesh after scvs_solve. */
typedef struct {
  int32_t status;     /* SCVS_CONVERGED / MAX_ITER / STAGNATED / NON_FINITE */
  int32_t iterations; /* Arnoldi steps spent on this mode */
  int32_t cycles;     /* restart cycles (= FP64 refinement steps) */
  int32_t guess_used; /* 1 if the learned initial guess was kept (its residual was below ||b||), or with
                         SCVS_GUESS_CURRENT */
  double rel_res;     /* final FP64 ||b_F - A_FF x_F - A_FD g|| / ||b_F|| (Eq. ls_error) */
  double res0;        /* the same relative residual at the start point: 1 for the zero start (x_F = 0),
                         below 1 where the learned guess was kept */
} scvs_mode_report;

/* Fill *opts with the defaults listed above. */
void scvs_default_opts(scvs_opts *opts);

/* Create a context on the current CUDA device.  opts may be NULL (defaults);
 * options outside the documented ranges return SCVS_ERR_ARG before any device
 * call (scvs_set_opts checks the same ranges).
 * Owns every device buffer it allocates.  Its device memory comes from a
 * memory pool of its own that keeps freed memory for reuse (re-creating a mesh
 * or a Krylov workspace of a size seen before maps nothing new), so the
 * context's footprint stays at its peak until scvs_destroy releases it. */
int scvs_create(scvs_ctx **out, const scvs_opts *opts);
void scvs_destroy(scvs_ctx *ctx);
const char *scvs_last_error(const scvs_ctx *ctx);
int scvs_set_opts(scvs_ctx *ctx, const scvs_opts *opts);

/* Add a P2 mesh (Sec. 2.3; conventions above) and build, on the GPU, its CSR
 * sparsity patterns (S: P2xP2, G: P2xP1, G^T) and the real mode-independent
 * matrices M_s, K_s, D_c of Eq. LS_construction plus the P1 pressure mass and
 * Laplacian used by the preconditioner.  Returns the mesh id (>= 0) or an
 * error (SCVS_ERR_MESH for a non-positive element Jacobian or a node id out
 * of range, SCVS_ERR_PRESSURE_NULLSPACE if no node is tagged OUTLET). */
int scvs_set_mesh(scvs_ctx *ctx, int32_t dim, int64_t n_nodes, int64_t n_vertices,
                  const double *xyz, int64_t n_elem, const int32_t *conn, const uint8_t *tag);
/* Same, with xyz/conn/tag already in device memory. */
int scvs_set_mesh_dev(scvs_ctx *ctx, int32_t dim, int64_t n_nodes, int64_t n_vertices,
                      const double *xyz_dev, int64_t n_elem, const int32_t *conn_dev,
                      const uint8_t *tag_dev);
/* Drop every mesh (and its modes) from the context. */
int scvs_clear_meshes(scvs_ctx *ctx);

/* Declare a mesh as the disjoint union of n_comp independent components
 * (node_comp[n_nodes] in [0, n_comp), host; no element may span two
 * components).  Every (component, mode) pair is then solved as its own
 * linear system (own Krylov space, convergence test and report entry) while
 * every kernel launch covers all components at once: this is how many meshes
 * of uneven size are batched.  Components share rho, mu and the mode list.
 * scvs_solve reports n_comp * n_modes entries for the mesh, component-major.
 * The learned guess is not applied to multi-component meshes.
 * Returns SCVS_ERR_MESH if an element couples two components. */
int scvs_set_components(scvs_ctx *ctx, int32_t mesh_id, int32_t n_comp, const int32_t *node_comp);

/* Physical constants rho, mu of a mesh (Eq. stokes_complex); defaults 1, 1. */
int scvs_set_physics(scvs_ctx *ctx, int32_t mesh_id, double rho, double mu);

/* Number of Dirichlet nodes of a mesh (nodes tagged WALL or INLET). */
int scvs_dirichlet_count(scvs_ctx *ctx, int32_t mesh_id, int64_t *n_dir);

/* Modes to solve on a mesh: omega[n_modes] and the prescribed velocity
 * g[n_modes][n_dir][dim] on the Dirichlet nodes in ascending node id
 * (Eq. dir_dis).  Builds the lifted right-hand sides (Eq. LS_construction:
 * B = -K G for the momentum rows and -D^T G for the continuity rows) and the
 * per-mode preconditioner.  Neumann data are zero (traction-free). */
int scvs_set_modes(scvs_ctx *ctx, int32_t mesh_id, int32_t n_modes, const double *omega,
                   const scvs_c64 *g);
int scvs_set_modes_dev(scvs_ctx *ctx, int32_t mesh_id, int32_t n_modes, const double *omega,
                       const void *g_dev /* double2 [n_modes][n_dir][dim] */);

/* Solve every mode of every mesh (mesh_id = -1) or of one mesh.  rep (host,
 * may be NULL) receives one entry per (mesh, component, mode) in mesh order,
 * rep_len entries at most.  Returns SCVS_OK even if some modes did not converge;
 * their status says so. */
int scvs_solve(scvs_ctx *ctx, int32_t mesh_id, scvs_mode_report *rep, int64_t rep_len);

/* Modal solution of a mesh: u[n_modes][n_nodes][dim], p[n_modes][n_vertices]
 * (host, either may be NULL). */
int scvs_get_modal(scvs_ctx *ctx, int32_t mesh_id, scvs_c64 *u, scvs_c64 *p);
/* Device view of the FP64 modal solution, interleaved [n_dof][ld] double2. */
int scvs_modal_dev(scvs_ctx *ctx, int32_t mesh_id, const void **x_dev, int64_t *n_dof, int32_t *ld);

/* Time reconstruction (Eq. sol_reconstruct, real fields):
 * u(x,t_s) = Re sum_k u_k(x) e^{j omega_k t_s}, t_s = s*period/n_t,
 * u_t[n_t][n_nodes][dim], p_t[n_t][n_vertices] (host; either may be NULL). */
int scvs_reconstruct(scvs_ctx *ctx, int32_t mesh_id, int32_t n_t, double period,
                     double *u_t, double *p_t);
int scvs_reconstruct_dev(scvs_ctx *ctx, int32_t mesh_id, int32_t n_t, double period,
                         double *u_t_dev, double *p_t_dev);

/* Allocation-free variant of scvs_reconstruct_dev (the paper has no
 * counterpart: this is a deployment convenience).  It is for callers that
 * must not allocate device memory during the call: code running while a
 * framework's caching allocator holds nearly all of the GPU's memory (a
 * cudaMalloc could fail or fragment it), and latency-critical pipelines that
 * cannot afford the device-wide synchronisation that cudaMalloc/cudaFree
 * imply.  The caller passes the modal solution (held by the context) and the
 * output buffers; the twiddle scratch e^{j omega_k t_s} lives in one
 * file-scope device table of SCVS_RECON_STATIC_MAX double2 entries (128 KiB),
 * which every GPU that loads the library holds until the process exits.
 * Limits and behaviour:
 *  - n_t * n_modes must not exceed SCVS_RECON_STATIC_MAX, else SCVS_ERR_ARG;
 *  - nothing is allocated: no cudaMalloc, cudaFree or allocating library call;
 *  - the first call on a device looks up the table's device address
 *    (cudaGetSymbolAddress) for that device; make that first call before any
 *    stream capture;
 *  - every call writes the table entries it reads, so nothing carries over
 *    between calls, but calls that overlap on the GPU (e.g. on two streams or
 *    from two contexts) race on the table: serialise them.
 * Output layout and accuracy are those of scvs_reconstruct_dev. */
#define SCVS_RECON_STATIC_MAX 8192
int scvs_reconstruct_dev_static(scvs_ctx *ctx, int32_t mesh_id, int32_t n_t, double period,
                                double *u_t_dev, double *p_t_dev);

/* Staged gathers of a mesh: info[10] = {row blocks built (1/0), blocks, nonzero
 * budget per block, largest footprint, largest vertex prefix of a footprint,
 * footprint entries in total, staged mode chunk of the SpMM and of the fine
 * Chebyshev kernels (0: unstaged), 1 if that SpMM / Chebyshev choice fits
 * shared memory (otherwise the unstaged kernel runs)}; us[8] (may be NULL) = autotuner times of
 * the staged SpMM and Chebyshev step with mode chunks 4, 8, 16, 32 (0: not
 * timed). */
int scvs_staged_info(scvs_ctx *ctx, int32_t mesh_id, int64_t *info, float *us);
/* The row blocks themselves (host copies; any pointer may be NULL): perm[N]
 * (rows in locality order), row0[n_blk+1] (block b = perm[row0[b]..row0[b+1])),
 * fp_ptr[n_blk+1] and fp_col[footprint total] (every block's ascending
 * distinct columns), fv_len[n_blk] (columns < n_vertices at the head of each
 * footprint), lcol[S nonzeros] (each nonzero's index in its row's block
 * footprint, S pattern order).  SCVS_ERR_STATE if none were built. */
int scvs_staged_blocks(scvs_ctx *ctx, int32_t mesh_id, int32_t *perm, int64_t *row0, int64_t *fp_ptr, int32_t *fp_col,
                       int32_t *fv_len, uint16_t *lcol);

/* ---- parity / inspection ------------------------------------------------ */
#define SCVS_CSR_S 0  /* P2 x P2 scalar pattern (values M_s, K_s) */
#define SCVS_CSR_G 1  /* P2 rows x P1 columns (values D_c) */
#define SCVS_CSR_GT 2 /* P1 rows x P2 columns (values D_c^T) */
#define SCVS_CSR_Q 3  /* P1 x P1 (values: P1 mass, P1 Laplacian) */

/* Rows and nonzeros of one pattern. */
int scvs_csr_size(scvs_ctx *ctx, int32_t mesh_id, int32_t which, int64_t *n_rows, int64_t *nnz);
/* Copy a pattern to the host: rowptr int64[n_rows+1], col int32[nnz]. */
int scvs_get_csr(scvs_ctx *ctx, int32_t mesh_id, int32_t which, int64_t *rowptr, int32_t *col);
/* Copy FP64 values to the host, in pattern order: S -> [2][nnz] (M_s, K_s);
 * G and GT -> [dim][nnz] (D_c resp. D_c^T); Q -> [2][nnz] (P1 mass, P1 Laplacian). */
int scvs_get_values(scvs_ctx *ctx, int32_t mesh_id, int32_t which, double *vals);

/* Row stride ld of the interleaved mode blocks of a mesh (>= n_modes). */
int scvs_mode_stride(scvs_ctx *ctx, int32_t mesh_id, int32_t *ld);
/* Degrees of freedom per mode, dim*n_nodes + n_vertices. */
int scvs_dof_count(scvs_ctx *ctx, int32_t mesh_id, int64_t *n_dof);

/* y_k = A_hat(omega_k) x_k for every mode k of a mesh, in one all-modes SpMM:
 * A_hat is A(omega_k) with Dirichlet velocity rows replaced by identity rows
 * and Dirichlet columns removed (the operator the Krylov solver iterates on).
 * precision SCVS_PREC_MIXED: x, y float2 [n_dof][ld]; SCVS_PREC_FP64: double2.
 * Device pointers, caller-owned, on the context's stream. */
int scvs_apply(scvs_ctx *ctx, int32_t mesh_id, int32_t precision, const void *x_dev, void *y_dev);
/* Same operator evaluated element by element (matrix-free): every element's
 * matrices (reference tables times its geometric factors; stored quadrature
 * matrices on curved elements) are applied once to its gathered nodal block
 * for all modes, colour by colour (no two elements of a colour share a node;
 * the colouring is built on the first call for a mesh), so no CSR values are
 * read and no atomics are used; same layouts and precisions as scvs_apply. */
int scvs_apply_matfree(scvs_ctx *ctx, int32_t mesh_id, int32_t precision, const void *x_dev, void *y_dev);
/* Lifted right-hand side of every mode, FP64 double2 [n_dof][ld] (device view):
 * b_F = -A_FD g on free rows, b_D = g on Dirichlet rows. */
int scvs_rhs_dev(scvs_ctx *ctx, int32_t mesh_id, const void **b_dev);
/* Apply the block preconditioner P^{-1}(omega_k) of every mode, of the kind
 * selected by opts.precond (default: block upper-triangular, SCVS_PC_TRI_PMG),
 * exactly as the FP32 Krylov cycles apply it: z = P^{-1} r, FP32 float2
 * [n_dof][ld] device arrays, r unchanged.  A linear operator in r (fixed
 * polynomials, no inner products).  Synchronises the context's stream (to
 * read the status of the bounded grid barriers of its persistent kernels:
 * SCVS_ERR_TIMEOUT, z void, if one gave up).  SCVS_ERR_STATE before
 * scvs_set_modes. */
int scvs_apply_precond(scvs_ctx *ctx, int32_t mesh_id, const void *r_dev, void *z_dev);

/* Failure detection of the persistent kernels' grid barrier (no paper
 * counterpart).  One cooperative launch of n_blocks blocks (1..SMs) in which
 * every block except absent_block (-1: none) passes two bounded grid barriers
 * with the given poll limit (1..2^24; the solver's kernels use 2^24, a few
 * seconds); absent_block returns without arriving, so the other blocks' wait
 * runs out: they record the time-out in the barrier's error word and return
 * instead of hanging.  Returns SCVS_OK if every barrier completed,
 * SCVS_ERR_TIMEOUT if a wait ran out (the barrier state is then reset, and the
 * context stays usable); *blocks_passed (may be NULL) = blocks that passed
 * both barriers.  Synchronises the context's stream. */
int scvs_barrier_selftest(scvs_ctx *ctx, int64_t spin_limit, int32_t n_blocks, int32_t absent_block,
                          int32_t *blocks_passed);

/* Number of kernel launches issued by this context since creation. */
int64_t scvs_launch_count(const scvs_ctx *ctx);
/* Device memory of the context's stream-ordered pool (every mesh, mode set and
 * Krylov workspace is taken from it), after synchronising the context's stream:
 * bytes in use, the high-water mark of bytes in use, and bytes reserved
 * (mapped; freed blocks stay reserved for reuse).  reset_high != 0 then
 * resets the high-water mark to the current use.  Any output may be NULL. */
int scvs_pool_usage(scvs_ctx *ctx, int32_t reset_high, int64_t *used, int64_t *used_high, int64_t *reserved);

/* ---- learned initial guess ----------------------------------------------
 * The modes of one geometry family share a node set; a converged mode x_k
 * divided by its boundary coefficient c_k (the problem is linear in c_k) is a
 * snapshot.  Training builds a POD basis of the snapshots per field block
 * (method of snapshots) and fits an MLP  f = (omega_k, Re c_k, Im c_k, R, s)
 * -> POD coefficients  (3 hidden GELU layers, BF16 weights, FP32 accumulate,
 * Adam, hand-written kernels).  With opts.guess = SCVS_GUESS_MLP and features
 * set for a mesh, scvs_solve starts every mode from x0 = c_k Phi a(f) (and g
 * on the Dirichlet rows); a mode whose x0 has a residual >= ||b|| starts from
 * zero instead.  The paper solves every mode from scratch; this is an
 * addition. features: host double [n_modes][5].
 *
 * POD: per field block (velocity rows, pressure rows) in the block's L2(Omega)
 * inner product <x, y> = x^H W y, W = M_s per velocity component and the P1
 * mass for the pressure, both of the mesh that gave the first snapshot (the
 * reference geometry; every snapshot shares its connectivity).  The Gram
 * matrix of the first max_pod_snapshots snapshots is formed on the GPU (FP32
 * data, FP64 accumulation), its eigenpairs on the host (FP64 Jacobi); every
 * eigenvector is scaled by a unit complex number that makes its
 * largest-magnitude entry real positive (this fixes each basis vector's
 * phase), Phi = X V Lambda^{-1/2} (Phi^H W Phi = I, stored FP32) with rank
 * r = min(n_pod, #eigenvalues > 1e-10 lambda_1), the same in both blocks;
 * the training targets are a_s = Phi^H W x_s.  Features and targets are
 * standardised by their means and population deviations (a deviation
 * below 1e-12 counts as 1). */
void scvs_default_train_opts(scvs_train_opts *opts);
/* Append the converged modes of a solved mesh to the training set. */
int scvs_guess_add_snapshots(scvs_ctx *ctx, int32_t mesh_id, const double *features);
/* POD + MLP training on the GPU; *final_loss (may be NULL) = last minibatch MSE (standardised units). */
int scvs_train_guess(scvs_ctx *ctx, const scvs_train_opts *opts, double *final_loss);
/* Features of the modes set on a mesh (used by the next scvs_solve). */
int scvs_guess_set_features(scvs_ctx *ctx, int32_t mesh_id, const double *features);
/* Training-set size, POD rank, 1 if a model is trained. */
int scvs_guess_info(scvs_ctx *ctx, int64_t *n_snapshots, int32_t *n_pod, int32_t *trained);
/* Drop snapshots and model. */
int scvs_guess_reset(scvs_ctx *ctx);
/* POD basis of a trained model: block 0 velocity (n_rows = dim N, row = node *
 * dim + component), 1 pressure (n_rows = P); phi host [n_rows][n_pod].
 * SCVS_ERR_STATE without a trained model, SCVS_ERR_ARG on a size mismatch. */
int scvs_guess_basis(scvs_ctx *ctx, int32_t block, int64_t n_rows, int32_t n_pod, scvs_c64 *phi);
/* POD coefficients a_s = Phi^H W x_s of every training snapshot (the training
 * targets before standardisation): a host [n_snapshots][n_pod]. */
int scvs_guess_coefficients(scvs_ctx *ctx, int32_t block, int64_t n_snapshots, int32_t n_pod, scvs_c64 *a);
/* The learned start of every mode of the mesh, without solving (features
 * set, model trained): x0 = c_k [Phi_u a_u; Phi_p a_p] with g on the
 * Dirichlet rows, its FP64 relative residual res0[k] = ||b - A x0|| / ||b||
 * (host [n_modes]) and kept[k] = 1 if scvs_solve with SCVS_GUESS_MLP would
 * start mode k from it (res0 < 1; otherwise that mode starts from zero).  x0,
 * kept or not, becomes the mesh's held solution (scvs_get_modal reads it).
 * SCVS_ERR_STATE if the model cannot serve the mesh (untrained, another node
 * set, no features, several components). */
int scvs_guess_initial(scvs_ctx *ctx, int32_t mesh_id, int64_t n_modes, double *res0, int32_t *kept);

/* Raw MLP (no feature/target scaling), for gradient checks and checkpoints.
 * Parameters are one flat FP32 array: for layer l = 0..3, W_l [in][out]
 * row-major then b_l [out], sizes n_in -> hidden -> hidden -> hidden -> n_out.
 * The kernels use the BF16 rounding of W and b and accumulate in FP32. */
int scvs_mlp_init(scvs_ctx *ctx, int32_t n_in, int32_t hidden, int32_t n_out, const float *params);
/* Overwrite the weights of the current MLP (same flat layout and size as
 * scvs_mlp_init) and keep everything else: a trained model keeps its POD
 * bases and standardisation.  SCVS_ERR_STATE without an MLP. */
int scvs_mlp_set_params(scvs_ctx *ctx, const float *params);
int scvs_mlp_num_params(scvs_ctx *ctx, int64_t *n);
int scvs_mlp_get_params(scvs_ctx *ctx, float *params);
/* y_dev[B][n_out] = MLP(x_dev[B][n_in]) (device pointers). */
int scvs_mlp_forward_dev(scvs_ctx *ctx, const float *x_dev, int64_t batch, float *y_dev);
/* Gradient of L = sum (y - t)^2 / (B n_out) into grad (host, flat layout); *loss = L. */
int scvs_mlp_gradient_dev(scvs_ctx *ctx, const float *x_dev, const float *t_dev, int64_t batch, float *grad,
                          double *loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8) with the last gradient. */
int scvs_mlp_adam_step(scvs_ctx *ctx, double lr);

/* ---- tracing ------------------------------------------------------------
 * Optional CUDA-event timers around every kernel launch, recorded on the
 * context's stream, grouped in classes:
 *   0 all-modes SpMM FP32, 1 all-modes SpMM FP64 (lift, true residual),
 *   2 block preconditioner: step 0, right-hand side of the triangular form,
 *   prolongation, 3 Arnoldi orthogonalisation + Hessenberg, 4 elementwise
 *   vector kernels, 5 pattern/assembly, 6 reconstruction, 7 matrix-free
 *   apply, 8 fine velocity Chebyshev sweeps and residual of the
 *   preconditioner, 9 pressure Schur solve (persistent), 10 coarse velocity
 *   solve (persistent).
 * Each class also sums the algorithmic bytes of its launches (the data the
 * kernel must read and write at minimum: matrix values and indices once,
 * every vector operand once).  scvs_kernel_timers(ctx, 1) clears and enables,
 * (ctx, 0) clears and disables.  scvs_kernel_times fills up to n_classes
 * entries of ms (summed device time), bytes and launches (any may be NULL)
 * and returns the number of classes. */
#define SCVS_KC_COUNT 11
int scvs_kernel_timers(scvs_ctx *ctx, int32_t enable);
int scvs_kernel_times(scvs_ctx *ctx, int32_t n_classes, double *ms, double *bytes, int64_t *launches);

/* Launch shapes chosen by the autotuner for a mesh (set by scvs_set_modes
 * when opts.autotune is on).  shape[4] = {modes per lane of the FP32 SpMM,
 * its row tile, modes per lane of the fine Chebyshev sweep, its row tile};
 * 0 = not tuned.  A row tile of t means a thread block walks
 * t x (row groups per block) consecutive rows before moving on, so that rows
 * sharing neighbours are gathered by the same SM.  us[2 * 3 * SCVS_TUNE_TILES]
 * holds the measured candidate times in microseconds, indexed
 * [kernel: SpMM, Chebyshev][modes per lane: 1, 2, 4][tile: 1, 2, 4, 8, 16];
 * 0 = candidate not valid for the mode stride.  Either pointer may be NULL. */
#define SCVS_TUNE_TILES 5
int scvs_tuned_shapes(scvs_ctx *ctx, int32_t mesh_id, int32_t *shape, float *us);

/* Neumann (traction) data of every mode (Eq. steady_stokes, boundary term of
 * Eq. LS_construction): the momentum right-hand side gains
 * b_u[A, c] = int_{Gamma_h} M_A h_c dGamma, with h interpolated from nodal values
 * by the P2 trace basis (b_u = M_Gamma h, M_Gamma the P2 boundary mass matrix of
 * straight-sided faces).  Gamma_h is the set of element faces whose nodes all
 * carry SCVS_TAG_NEUMANN and that belong to one element only.  Rows of
 * Dirichlet nodes keep their prescribed values.
 *   h        host, complex [n_modes][n_nodes][dim]: nodal traction of every mode
 *            (only nodes of Gamma_h are read; caller-owned, copied)
 *   n_faces  out (may be NULL): number of faces of Gamma_h
 * Call after scvs_set_modes (which clears the Neumann data); the data persist
 * across scvs_set_physics.  Returns SCVS_ERR_STATE before scvs_set_modes,
 * SCVS_ERR_ARG for a bad id or a null h. */
int scvs_set_neumann(scvs_ctx *ctx, int32_t mesh_id, const scvs_c64 *h, int64_t *n_faces);

/* Spectral preprocessing of sampled periodic boundary data (Sec. 3, steps 1
 * and 2 of the algorithm): the Fourier coefficients of Eq. SCVS_bc by the
 * rectangle rule on n_t uniform samples t_s = s T / n_t of one period, as the
 * solver's per-mode data, and the a priori truncation error of Eq. mode_error.
 *   n_t      samples (>= 2)
 *   n_pts    values per sample, e.g. n_dir * dim for Dirichlet data in the
 *            [node][component] layout of scvs_set_modes
 *   n_modes  modes 0..n_modes-1 (omega_i = 2 pi i / T), below the Nyquist
 *            frequency of the samples: 2 (n_modes - 1) < n_t
 *   g_t      device, FP64 [n_t][n_pts]: real samples (caller-owned)
 *   w        device, FP64 [n_pts]: weights of the L2(Gamma) inner product
 *            (e.g. nodal boundary areas), or NULL for unit weights
 *   c        device, out, complex128 [n_modes][n_pts]: c_0 = g~_0,
 *            c_i = 2 g~_i (i >= 1), so the field is Re sum_i c_i e^{j omega_i t};
 *            with n_pts = n_dir * dim this is the g argument of scvs_set_modes_dev
 *   e2       host, out, [n_modes]: e2[N] = ||g - g^_N||^2 / ||g||^2 in
 *            L2(Gamma x T) (time by the rectangle rule, space by w) for the
 *            series truncated after mode N, from the discrete Parseval identity
 *            (exact on the samples); all 0 if g is zero.  The Dirichlet and
 *            Neumann terms of Eq. mode_error are two calls whose e2 add.
 * FP64 throughout (twiddles cos/sin(2 pi j / n_t) in FP64; fixed-order
 * reductions, so the result is reproducible).  Runs on the context's stream
 * and synchronises it.  Returns SCVS_OK or SCVS_ERR_ARG (sizes, null pointers). */
int scvs_bc_spectrum(scvs_ctx *ctx, int32_t n_t, int64_t n_pts, int32_t n_modes, const double *g_t, const double *w,
                     void *c, double *e2);

/* A posteriori mode energies of a solved mesh (Sec. 3: the change of the
 * reconstruction of Eq. sol_reconstruct when mode N is added decides whether
 * more modes are needed).  For every component and mode (index comp * n_modes + k):
 *   E[.]      (host, out) time average over the period of
 *             ||Re(u~_k e^{j omega_k t})||^2_{L2(Omega)} of the velocity, with the P2
 *             mass matrix: ||Re u~_k||^2 for omega_k = 0, (1/2) u~_k^H M u~_k otherwise
 *   incr2[.]  (host, out, may be NULL) delta_N^2 = E_N / sum_{k <= N} E_k, the squared
 *             L2(Omega x T) change of the series truncated after mode N relative to
 *             its norm (modes in the order given to scvs_set_modes; exact for distinct
 *             harmonic frequencies omega_k = 2 pi k / T, which are orthogonal over the
 *             period); 0 where the series is zero
 * n_out must be at least n_components * n_modes.  FP64, fixed-order
 * reductions.  Runs on the context's stream and synchronises it.  Returns
 * SCVS_ERR_STATE before scvs_solve, SCVS_ERR_ARG for a bad id or size. */
int scvs_mode_energies(scvs_ctx *ctx, int32_t mesh_id, int64_t n_out, double *E, double *incr2);

/* A posteriori number of modes (Sec. 3, the remark after step 4: after each
 * mode, compare the reconstructions with N - 1 and N modes and go on while the
 * difference exceeds a tolerance).  incr2[0..n): the squared relative changes
 * of scvs_mode_energies for one system, modes in order.  *n_keep = the
 * smallest N >= 1 such that the changes of modes N, N+1, ..., N+patience-1 all
 * exist and are below eps (their square root); n if there is none.  patience
 * = 1 is the literal rule; a larger patience keeps going across a missing
 * harmonic (a zero change followed by energetic modes).  Host only.
 * SCVS_ERR_ARG if n < 1, patience < 1, eps <= 0 or a pointer is NULL. */
int scvs_modes_to_keep(const double *incr2, int64_t n, double eps, int32_t patience, int64_t *n_keep);

/* ---- checkpoint / resume --------------------------------------------------
 * Every mode is an independent problem, so the modal solution is the
 * checkpoint: a file holds the converged modes of one mesh with their omega_k,
 * status and residual, and a resumed run starts matching modes from it
 * (scvs_set_solution + opts.guess = SCVS_GUESS_CURRENT), so that they converge
 * at the first true-residual check.  No paper counterpart. */

/* Initial solution of every mode (layout of scvs_get_modal): u host complex
 * [n_modes][n_nodes][dim], p host complex [n_modes][n_vertices] (copied).  The
 * next scvs_solve with opts.guess = SCVS_GUESS_CURRENT starts from it.
 * SCVS_ERR_STATE before scvs_set_modes; SCVS_ERR_ARG for a bad id or null arrays. */
int scvs_set_solution(scvs_ctx *ctx, int32_t mesh_id, const scvs_c64 *u, const scvs_c64 *p);

typedef struct {
  int32_t dim, n_modes;
  int64_t n_nodes, n_vertices;
  uint64_t mesh_hash; /* scvs_mesh_hash of the mesh the modes belong to */
  double tol;         /* relative residual the modes were solved to */
  double rho, mu;     /* the physics the modes were solved with */
} scvs_ckpt_header;

/* FNV-1a 64 hash of one mode's boundary data: the Dirichlet values g (n_g
 * complex entries) and, when not NULL, the nodal tractions h (n_h entries).  A
 * stored mode is reused only for identical data.  Host only. */
int scvs_data_hash(const scvs_c64 *g, int64_t n_g, const scvs_c64 *h, int64_t n_h, uint64_t *hash);

/* FNV-1a 64 hash of a mesh's arrays (host pointers, the layout of
 * scvs_set_mesh): sizes, xyz, conn and tag bytes.  Host only. */
int scvs_mesh_hash(int32_t dim, int64_t n_nodes, int64_t n_vertices, const double *xyz, int64_t n_elem,
                   const int32_t *conn, const uint8_t *tag, uint64_t *hash);

/* Write / read a checkpoint file (host only; little-endian machine format):
 * magic "SCVSCKP2", the header, omega [n_modes], data_hash [n_modes]
 * (scvs_data_hash of every mode's boundary data), status [n_modes]
 * (SCVS_CONVERGED ...), rel_res [n_modes], u [n_modes][n_nodes][dim], p
 * [n_modes][n_vertices] (complex), then an FNV-1a 64 checksum of everything
 * before it.  Read checks magic, sizes and checksum and returns SCVS_ERR_ARG on
 * any mismatch (nothing written to the outputs).  With every output array NULL
 * it only reads the header (to size the arrays); with any array given, *header
 * is also an input: the file's dim, n_modes, n_nodes and n_vertices must equal
 * it (the arrays are sized for it), else SCVS_ERR_ARG before any copy. */
int scvs_checkpoint_write(const char *path, const scvs_ckpt_header *header, const double *omega,
                          const uint64_t *data_hash, const int32_t *status, const double *rel_res, const scvs_c64 *u,
                          const scvs_c64 *p);
int scvs_checkpoint_read(const char *path, scvs_ckpt_header *header, double *omega, uint64_t *data_hash,
                         int32_t *status, double *rel_res, scvs_c64 *u, scvs_c64 *p);

/* Graph aggregates of a vertex graph, the coarse space of SCVS_PC_TRI_PMG_CS
 * (no paper counterpart: part of the preconditioner).  Host only: no context,
 * no device work.
 *   n_vert         number of vertices (>= 0)
 *   row_ptr        [n_vert + 1] CSR row pointers (host, int64, non-decreasing, row_ptr[0] = 0)
 *   col            [row_ptr[n_vert]] neighbours of every vertex (host, int32; the vertex itself may be
 *                  listed; every entry must lie in [0, n_vert))
 *   target         aggregates per connected component (1..512)
 *   agg            [n_vert] out: aggregate of every vertex
 *   n_agg, n_blk   out (may be NULL): number of aggregates and of connected components
 * Connected components are numbered in the order of their lowest vertex; in
 * each, aggregates are grown breadth-first (neighbours in row order) from the
 * lowest unassigned vertex up to ceil(g * component size / target) vertices
 * (g = 1, raised 1.5x until no component has more than min(2 target, 1024)
 * aggregates); an aggregate below a third of that size joins the first
 * full-size aggregate adjacent to it.  Every aggregate is connected and lies
 * in one component; aggregates are numbered by component, then by seed.  The
 * result depends only on the arguments.  Returns SCVS_OK or SCVS_ERR_ARG
 * (null pointer, bad size, pointer or column out of range). */
int scvs_graph_aggregates(int64_t n_vert, const int64_t *row_ptr, const int32_t *col, int32_t target,
                          int32_t *agg, int32_t *n_agg, int32_t *n_blk);

/* State of the coarse Schur correction of a mesh after its last setup
 * (SCVS_PC_TRI_PMG_CS): info[4] = {aggregates, connected components, largest
 * component's aggregates, singular (component, mode) coarse matrices, whose
 * correction is off}; all 0 before the first application of that kind after
 * scvs_set_modes. */
int scvs_schur_coarse_info(scvs_ctx *ctx, int32_t mesh_id, int32_t *info);

/* Coarse level of the two-level pressure Laplacian of a mesh (opts.lap_size >= 0; built on the first
 * preconditioner application with that option and kept for the mesh's lifetime): info[6] = {1 if the
 * cycle is in use, else 0 (the plain polynomial), aggregates, connected components of the vertex graph
 * without the outlet vertices, largest component's aggregates, components whose coarse matrix was
 * singular (coarse correction off there), components no outlet vertex reaches (any: the plain
 * polynomial)}; all 0 before it is built.  agg (may be NULL, else [n_vertices]): every vertex's
 * aggregate, -1 on the outlet (all -1 while the cycle is not in use).  SCVS_ERR_ARG for a bad mesh id
 * or a null info. */
int scvs_lap_info(scvs_ctx *ctx, int32_t mesh_id, int32_t *info, int32_t *agg);

/* Spectral bounds behind the preconditioner's Chebyshev intervals (a 14-step power method on the
 * Jacobi-scaled operators, run by scvs_set_modes and scvs_set_physics): out[0] = lambda_max of
 * D^-1 M_p, out[1] of D^-1 L_p (outlet rows and columns removed), out[2 + k] of D^-1 A_r with the
 * velocity shift A_r = mu K + |omega_k| rho M of mode k (P2, Dirichlet rows removed) and
 * out[2 + n_modes + k] of its P1 (vertex) coarse operator; 2 + 2 n_modes doubles (host).
 * SCVS_ERR_ARG for a bad mesh id, a null out or n_modes other than the mesh's; SCVS_ERR_STATE before
 * scvs_set_modes. */
int scvs_pc_bounds(scvs_ctx *ctx, int32_t mesh_id, int32_t n_modes, double *out);

#ifdef __cplusplus
}
#endif
#endif /* SCVS_H */
