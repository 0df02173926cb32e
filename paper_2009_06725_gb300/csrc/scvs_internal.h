// Internal host-side structures of the SCVS library (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <complex>
#include <map>
#include <string>
#include <vector>
#include "../../include/scvs.h"
#include "common.cuh"
#include <cuda_bf16.h>

namespace scvs {

// Device allocations owned by one object, released together.
// Device allocations of one owner (a mesh, its mode set, the context), taken
// stream-ordered from the context's memory pool, which keeps freed memory
// cached: re-creating a mesh or a Krylov workspace of the same size costs no
// new mapping and no device-wide synchronisation.
struct DevArena {
  std::vector<void *> ptrs;
  cudaMemPool_t pool = nullptr;  // null: plain cudaMalloc / cudaFree
  cudaStream_t stream = nullptr;
  template <typename T> T *alloc(size_t count) {
    void *p = nullptr;
    if (count == 0) count = 1;
    cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, count * sizeof(T), pool, stream)
                         : cudaMalloc(&p, count * sizeof(T));
    if (e != cudaSuccess) { (void)cudaGetLastError(); throw std::bad_alloc(); }
    ptrs.push_back(p);
    return static_cast<T *>(p);
  }
  void release() {
    for (void *p : ptrs) {
      if (pool) cudaFreeAsync(p, stream); else cudaFree(p);
    }
    ptrs.clear();
  }
};

constexpr int CHUNK_ROWS = 2048;

// Counts every kernel launch of a context (reported by scvs_launch_count).
struct Launches { int64_t n = 0; };

// Kernel classes timed by the optional event timers (scvs_kernel_timers).
enum KClass : int {
  KC_SPMM32 = 0, KC_SPMM64, KC_PRECOND, KC_ARNOLDI, KC_VECTOR, KC_ASSEMBLY, KC_RECON, KC_MATFREE, KC_CHEB_FINE,
  KC_PRESSURE, KC_COARSE, KC_COUNT
};

// CUDA-event timing of kernel launches on the launching stream: a start and a
// stop event around each timed launch, resolved lazily; also sums the
// algorithmic bytes of each launch (what the kernel must move at minimum).
struct KTimers {
  bool on = false;
  struct Pend { cudaEvent_t a, b; int cls; double bytes; };
  std::vector<Pend> pend;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;
  double ms[KC_COUNT] = {0}, bytes[KC_COUNT] = {0};
  int64_t n[KC_COUNT] = {0};
  cudaEvent_t cur_a = nullptr;
  void begin(cudaStream_t s);
  void end(cudaStream_t s, int cls, double bytes);
  void resolve();
  void reset();
  void destroy();
};

// Per-mode Chebyshev coefficients of the block preconditioner of one mesh.
struct PcTables {
  double *inv_theta_u = nullptr, *alpha_u = nullptr, *beta_u = nullptr;  // device, [ld], [s_u][ld]
  double *inv_theta_c = nullptr, *alpha_c = nullptr, *beta_c = nullptr;  // coarse level, [ld], [s_c][ld]
  double *zeros = nullptr;                                                // [ld]
  int s_c = 0, kind = -1;
  std::vector<double> am, bm, al, bl;  // P1 mass / Laplacian recurrences
  double *am_d = nullptr, *bm_d = nullptr, *al_d = nullptr, *bl_d = nullptr;  // device copies
  double inv_theta_m = 0, inv_theta_l = 0;
  int s_u = 0, s_m = 0, s_l = 0;
  int lap_s = 0;  // > 0: two-level Laplacian with lap_s pre- and post-smoothing steps (al/bl, inv_theta_l)
  bool valid = false;
  // Coarse correction of the Schur approximation (SCVS_PC_TRI_PMG_CS): graph
  // aggregates of the vertices, grouped by connected component ("block"), and
  // the inverse coarse matrix of every (block, mode).
  int cs_target = 0;                 // aggregates per block asked for
  int n_agg = 0, n_blk = 0, na_max = 0;
  int32_t *agg = nullptr;            // [P] aggregate of every vertex
  int64_t *agg_ptr = nullptr;        // [n_agg+1] CSR of the aggregates' vertices (ascending ids)
  int32_t *agg_vert = nullptr;       // [P]
  int32_t *agg_blk = nullptr, *agg_loc = nullptr;  // [n_agg] block, index within the block
  int32_t *blk_na = nullptr, *blk_a0 = nullptr;    // [n_blk] aggregates of the block, its first aggregate
  int64_t *blk_so = nullptr;         // [n_blk] sum of n_a^2 over the blocks before it
  int64_t so_total = 0;
  void *sinv = nullptr;              // [so_total][ld] inverse coarse matrices (row-major per block), T
  int cs_bytes = 0;                  // sizeof(T) of sinv (0: not built)
  int cs_singular = 0;               // (block, mode) pairs whose coarse matrix was singular (correction off)
};

// Coarse level of the two-level pressure Laplacian solve (opts.lap_size >= 0):
// graph aggregates of the vertices off the outlet (where the Laplacian has
// p = 0) of about lap_size vertices each (a fixed aggregate diameter keeps the
// two-level convergence independent of the mesh size), grouped by connected
// component of that graph ("block"), and the inverse of every block's Galerkin
// matrix R^T L_p R (R the piecewise-constant indicator of the aggregates).
// Mode independent: built once per mesh and size.  Blocks not reached by an
// outlet vertex make L_p singular there; such a mesh keeps the plain
// Chebyshev polynomial (on = false).
constexpr int LAP_NA_MAX = 1024;  // aggregates of one block at most (larger blocks get larger aggregates)
constexpr int LAP_DEFAULT_SIZE = 32;
constexpr int LAP_DEFAULT_SMOOTH = 8;
struct LapCoarse {
  int target = 0;                    // aggregate size asked for (0: not built)
  bool on = false;
  int n_agg = 0, n_blk = 0, na_max = 0, singular = 0, unanchored = 0;
  int32_t *agg = nullptr;            // [P] aggregate of every vertex, -1 on the outlet
  int64_t *agg_ptr = nullptr;        // [n_agg+1] CSR of the aggregates' vertices (ascending ids)
  int32_t *agg_vert = nullptr;       // [P - outlet vertices]
  int32_t *agg_blk = nullptr, *agg_loc = nullptr;  // [n_agg]
  int32_t *blk_na = nullptr, *blk_a0 = nullptr;    // [n_blk]
  int64_t *blk_so = nullptr;         // [n_blk] sum of n_a^2 over the blocks before it
  int64_t so_total = 0;
  float *inv_f = nullptr;            // [so_total] inverse Galerkin matrices (row-major per block)
  double *inv_d = nullptr;           // the same values widened for the FP64 path
};

// Row blocks of a mesh for the staged gather kernels (blocks.cu): rows in a
// locality order cut into blocks of about `budget` nonzeros, the distinct
// columns ("footprint") of every block and every nonzero's index in it.
constexpr int RB_DEFAULT_BUDGET = 768;
constexpr size_t STAGE_SMEM_MAX = 200 * 1024;
struct RowBlocks {
  bool valid = false;
  int budget = 0, fp_max = 0, fv_max = 0;
  int64_t n_blk = 0, fp_total = 0;
  int32_t *perm = nullptr;     // [N]
  int64_t *row0 = nullptr;     // [n_blk + 1]
  int64_t *fp_ptr = nullptr;   // [n_blk + 1]
  int32_t *fp_col = nullptr;   // [fp_total]
  int32_t *fv_len = nullptr;   // [n_blk]
  uint16_t *lcol = nullptr;    // [s_nnz]
  // the arrays live in the mesh arena (released with the mesh)
  void release(cudaStream_t) { *this = RowBlocks{}; }
};

// One mesh and the state of its modes.
//
// Patterns: S (P2 x P2) is stored once; because vertex nodes carry the
// smallest ids, the columns < P of an S row are a prefix of it, and that
// prefix is the G row (P2 x P1); the S rows of the vertices (ids < P) are the
// G^T rows, and the G rows of the vertices are the Q rows (P1 x P1).
struct Mesh {
  int dim = 0, nl = 0, nv = 0;
  int64_t N = 0, P = 0, E = 0, n_dof = 0, n_dir = 0;
  DevArena arena;
  double *xyz = nullptr;
  int32_t *conn = nullptr;
  uint8_t *tag = nullptr;
  double *geom = nullptr;           // [E][GEOM_STRIDE]
  // curved (isoparametric) elements: slot of every element (-1: straight) and
  // their element matrices by quadrature, CM/CK [n_curved][nl][nl], CD [n_curved][dim][nl][nv]
  int64_t n_curved = 0;
  int32_t *cslot = nullptr;
  double *CM = nullptr, *CK = nullptr, *CD = nullptr;
  std::vector<int64_t> mf_col_ptr;  // matrix-free element colours: colour k = mf_el[ptr[k] .. ptr[k+1])
  int32_t *mf_el = nullptr;         // [E] elements by colour (built on the first matrix-free application)
  int64_t *n2e_ptr = nullptr;       // [N+1] node -> incident elements
  int32_t *n2e = nullptr;           // ascending element ids per node
  int64_t *s_ptr = nullptr;         // [N+1]
  int32_t *s_col = nullptr;         // [s_nnz]
  int32_t *s_len = nullptr;         // [N]
  int32_t *g_len = nullptr;         // [N] leading columns < P
  int64_t *g_ptr = nullptr;         // [N+1] G row pointers
  int64_t s_nnz = 0, g_nnz = 0, gt_nnz = 0, q_nnz = 0;
  int max_row = 0;
  // FP64 values, unmasked (pattern order)
  double *Ms = nullptr, *Ks = nullptr;   // [s_nnz]
  double *Dv = nullptr;                  // [dim][g_nnz]
  double *DTv = nullptr;                 // [dim][gt_nnz]
  double *Mp = nullptr, *Lp = nullptr;   // [q_nnz]
  // operator values with Dirichlet rows/columns removed
  double *Ms_m = nullptr, *Ks_m = nullptr, *Dv_m = nullptr, *DTv_m = nullptr, *Lp_m = nullptr;
  float *Ms_f = nullptr, *Ks_f = nullptr, *Dv_f = nullptr, *DTv_f = nullptr, *Mp_f = nullptr, *Lp_f = nullptr;
  double *ms_diag = nullptr, *ks_diag = nullptr;  // [N]
  // FP32 copies of the diagonals used by the FP32 preconditioner kernels
  float *ms_df = nullptr, *ks_df = nullptr;       // [N]
  float *mp_df = nullptr, *lp_df = nullptr, *k1_df = nullptr;  // [P]
  double *mp_diag = nullptr, *lp_diag = nullptr;  // [P] (lp: outlet rows -> 1)
  // two-level velocity preconditioner: P1 (vertex) coarse space nested in P2
  int32_t *edge_ends = nullptr;   // [N-P][2] end vertices of every edge node
  int64_t *v2e_ptr = nullptr;     // [P+1] vertex -> incident edge nodes
  int32_t *v2e = nullptr;         // ascending edge-node ids
  float *Kc_f = nullptr, *Mc_f = nullptr;  // [q_nnz] P1 stiffness / mass, Dirichlet vertices removed
  double *Kc_m = nullptr, *Mc_m = nullptr; // same in FP64
  double *k1_diag = nullptr;      // [P] unmasked P1 stiffness diagonal
  uint8_t *dirmask = nullptr;  // [N]
  uint8_t *outmask = nullptr;  // [P]
  int64_t *dir_nodes = nullptr;  // [n_dir] ascending
  // Independent components: the mesh may be the disjoint union of several
  // meshes; every (component, mode) pair is then its own linear system
  // ("system" s = comp * ld + k) with its own Krylov space and convergence.
  int n_comp = 1;
  int32_t *dof_comp = nullptr;   // [n_dof] component of every dof row (null: all 0)
  // Row chunks of at most CHUNK_ROWS rows that never straddle two
  // components, grouped by component: reductions are segmented by chunk.
  int64_t n_chunk = 0;
  int64_t *chunk_row0 = nullptr;
  int32_t *chunk_rows = nullptr, *chunk_comp = nullptr;
  int32_t *comp_chunk = nullptr;  // [n_comp+1] chunk range of every component
  uint8_t *comp_active = nullptr; // [n_comp] 0: every system of the component is done (kernels skip it)
  int n_sys() const { return n_comp * ld; }
  double rho = 1.0, mu = 1.0;
  // ---- modes
  int m = 0, ld = 0;
  DevArena mode_arena;
  std::vector<double> omega;     // host copy [ld] (padded with 0)
  double *omega_d = nullptr;     // [ld]
  double *wabs_d = nullptr, *wrho_d = nullptr;  // [ld] |omega_k| rho, omega_k rho
  float *wabs_f = nullptr, *wrho_f = nullptr;
  double2 *g = nullptr;          // [m][n_dir][dim]
  double2 *b = nullptr;          // [n_dof][ld] lifted RHS (b_D = g)
  double2 *x = nullptr;          // [n_dof][ld] FP64 solution
  double2 *neu = nullptr;        // [dim N][ld] Neumann load of the modes (null: traction-free)
  std::vector<double> bnorm;     // [n_comp * ld] ||b_F|| per system
  std::vector<double> lam_u;     // [ld] spectral radius estimate of D_r^-1 A_r per mode (velocity)
  std::vector<double> lam_c;     // [ld] same for the P1 coarse velocity operator
  double lam_m = 0, lam_l = 0;   // same for the P1 mass / Laplacian
  PcTables pc;
  LapCoarse lap;                         // two-level pressure Laplacian (mesh arena)
  RowBlocks rb;                          // staged-gather row blocks (FP32 path)
  int st_spmm = 0, st_cheb = 0;          // staged mode chunk of the SpMM / fine Chebyshev kernels (0: unstaged)
  int mpl_spmm = 0, mpl_cheb = 0;       // autotuned row-group shapes (0: default)
  int tile_spmm = 0, tile_cheb = 0;     // autotuned row tiles (0: default)
  std::vector<float> tune_us;            // measured candidates: [spmm mpl=1,2,4, cheb mpl=1,2,4] (us, 0 = n/a)
  std::vector<double> feat;      // [m][5] features of the modes (learned guess)
  bool solved = false;
  std::vector<scvs_mode_report> rep;
};

// Learned initial guess: snapshots, POD bases, MLP (see guess.cu).
struct GuessModel {
  int64_t n_dof = 0, n_u = 0, n_snap = 0, snap_cap = 0;
  float2 *snap = nullptr;           // [n_snap][n_dof] solutions divided by c_k
  std::vector<double> feat;         // [n_snap][5]
  // Mass matrices of the reference mesh (the one that gave the first
  // snapshot): the POD's inner products.  Device copies of the S pattern, the
  // G row offsets/lengths (the P1 mass lives on the vertex G rows), M_s and
  // the P1 mass.
  struct RefMass {
    int dim = 0;
    int64_t N = 0, P = 0;
    int64_t *s_ptr = nullptr, *g_ptr = nullptr;
    int32_t *s_col = nullptr, *g_len = nullptr;
    double *Ms = nullptr, *Mp = nullptr;
  } wref;
  int n_pod = 0;
  float2 *Phi_u = nullptr, *Phi_p = nullptr;  // [n_u][n_pod], [n_p][n_pod]
  std::vector<std::complex<double>> coef_u, coef_p;  // [n_snap][n_pod] POD coefficients of the snapshots
  std::vector<double> lam_u, lam_p;                   // Gram eigenvalues, descending
  std::vector<double> fmean, fstd, tmean, tstd;
  int hidden = 0, n_out = 0, dims[5] = {0, 0, 0, 0, 0};
  int64_t woff[4] = {0}, boff[4] = {0}, n_params = 0;
  float *Wf = nullptr, *grad = nullptr, *am = nullptr, *av = nullptr, *scal = nullptr;
  __nv_bfloat16 *Wb = nullptr, *Wt = nullptr;
  int64_t adam_t = 0;
  bool trained = false;
  float *acts = nullptr;
  int64_t act_cap = 0;
  int64_t per_sample() const { return 6 * (int64_t)hidden + 2 * (int64_t)n_out + 2 * (int64_t)std::max(hidden, n_out); }
  void ensure(int64_t B) {
    if (act_cap >= B && acts) return;
    if (acts) cudaFree(acts);
    act_cap = std::max<int64_t>(B, 64);
    if (cudaMalloc(&acts, (size_t)act_cap * per_sample() * sizeof(float)) != cudaSuccess) throw std::bad_alloc();
  }
  float *zbuf(int l) { return l < 3 ? acts + (int64_t)l * act_cap * hidden : acts + 6 * act_cap * hidden; }
  float *abuf(int l) { return acts + (int64_t)(3 + l) * act_cap * hidden; }
  float *ybuf() { return acts + 6 * act_cap * hidden + act_cap * n_out; }
  float *dbuf(int i) { return acts + 6 * act_cap * hidden + 2 * act_cap * n_out + (int64_t)i * act_cap * std::max(hidden, n_out); }
  void release_mlp() {
    for (void *p : {(void *)Wf, (void *)grad, (void *)am, (void *)av, (void *)scal, (void *)Wb, (void *)Wt, (void *)acts})
      if (p) cudaFree(p);
    Wf = grad = am = av = scal = acts = nullptr;
    Wb = Wt = nullptr;
    act_cap = 0;
    n_params = 0;
    trained = false;
  }
  void release() {
    release_mlp();
    for (void *p : {(void *)snap, (void *)Phi_u, (void *)Phi_p, (void *)wref.s_ptr, (void *)wref.g_ptr,
                    (void *)wref.s_col, (void *)wref.g_len, (void *)wref.Ms, (void *)wref.Mp})
      if (p) cudaFree(p);
    snap = nullptr; Phi_u = Phi_p = nullptr;
    wref = RefMass{};
    n_snap = snap_cap = n_dof = n_u = 0;
    n_pod = 0;
    feat.clear();
    coef_u.clear(); coef_p.clear(); lam_u.clear(); lam_p.clear();
  }
};

struct Ctx {
  scvs_opts opts;
  cudaStream_t stream = nullptr;
  int device = 0, num_sms = 0;
  std::string err;
  Launches launches;
  std::vector<Mesh *> meshes;
  DevArena work;            // Krylov workspace, grown on demand
  size_t work_bytes = 0;
  int *dev_err = nullptr;   // device error word (DevErr bits)
  GridSync *gsync = nullptr;
  RefTables ref2, ref3;
  QuadTables quad2, quad3;
  KTimers timers;
  GuessModel guess;
  // autotuned launch shapes by mesh size (dim, N, P, S nonzeros, G nonzeros,
  // mode stride, components): the timings depend on the pattern's size, not its values
  struct TuneRec { int mpl_spmm, tile_spmm, mpl_cheb, tile_cheb, st_spmm, st_cheb; std::vector<float> us; };
  std::map<std::vector<int64_t>, TuneRec> tune_cache;
  cudaMemPool_t pool = nullptr;  // every stream-ordered allocation of the context
};

// Stream-ordered allocation from the context's pool.
template <typename P> inline cudaError_t ctx_malloc(const Ctx &c, P **p, size_t bytes, cudaStream_t s) {
  return cudaMallocFromPoolAsync(reinterpret_cast<void **>(p), bytes, c.pool, s);
}

// Scoped timing of one launch: KT(c, class, algorithmic bytes) { launch; }
struct KScope {
  Ctx &c; int cls; double bytes;
  KScope(Ctx &c_, int cls_, double bytes_) : c(c_), cls(cls_), bytes(bytes_) { if (c.timers.on) c.timers.begin(c.stream); }
  ~KScope() { if (c.timers.on) c.timers.end(c.stream, cls, bytes); }
};

// ---- assembly.cu
void build_mesh(Ctx &c, Mesh &m, const double *xyz_dev, const int32_t *conn_dev, const uint8_t *tag_dev);
int64_t set_neumann(Ctx &c, Mesh &m, const double2 *h_host);  // returns the number of Neumann faces
void scan_exclusive(Ctx &c, const int32_t *in, int64_t *out, int64_t n);
void build_row_blocks(Ctx &c, Mesh &m, int budget);  // blocks.cu

// ---- operators.cu
template <typename T>
void apply_saddle(Ctx &c, const Mesh &m, const typename cpx<T>::t *x, typename cpx<T>::t *y);
void lift_rhs(Ctx &c, Mesh &m);
double saddle_bytes(const Mesh &m, int value_size);
int64_t precond_scratch_elems(const Mesh &m);
void autotune_shapes(Ctx &c, Mesh &m);
void residual_fp64(Ctx &c, Mesh &m, float2 *r32, double2 *r64, double *norm2_out_dev, bool zero_start = false);
void norms2_sys(Ctx &c, const Mesh &m, const double2 *v, double *out_dev);  // [n_sys] free-row squared norms
void set_chunks(Ctx &c, Mesh &m, const int32_t *node_comp_host, int n_comp);
void spectral_bounds(Ctx &c, Mesh &m);
int pc_kind(const Ctx &c, const Mesh &m);  // opts.precond with SCVS_PC_AUTO resolved for the mesh
template <typename T>
void apply_precond(Ctx &c, Mesh &m, const typename cpx<T>::t *r, typename cpx<T>::t *z,
                   typename cpx<T>::t *scratch, const double *rscale);
void apply_matfree(Ctx &c, Mesh &m, int precision, const void *x, void *y);
// Graph aggregates (host): agg [P] aggregate of every vertex, numbered by block
// (connected component, in order of its lowest vertex) then seed; per aggregate
// its block and index within it; per block its count and first aggregate.
struct AggResult {
  std::vector<int32_t> agg, blk, loc, na, a0;
  int n_blk = 0, na_max = 0;
};
AggResult graph_aggregates(int64_t P, const int64_t *ptr, const int32_t *col, int target, int na_cap = 0,
                           int size = 0);
void matfree_tables(Ctx &c);  // matfree.cu

// ---- krylov.cu
int solve_mesh(Ctx &c, Mesh &m);
bool guess_probe(Ctx &c, Mesh &m, double *res0, int *kept);
int barrier_selftest(Ctx &c, long long spin_limit, int n_blocks, int absent, int *passed);

// ---- guess.cu
void guess_add_snapshots(Ctx &c, Mesh &m, const double *features);
double guess_train(Ctx &c, const scvs_train_opts &o);
bool guess_initial(Ctx &c, Mesh &m);
void mlp_alloc(GuessModel &g, int n_in, int hidden, int n_out);
void mlp_refresh_bf16(Ctx &c, GuessModel &g);
void mlp_forward(Ctx &c, GuessModel &g, const float *x, int64_t B, float *y);
float mlp_gradient(Ctx &c, GuessModel &g, const float *x, const float *t, int64_t B, bool read_loss = true);
void mlp_adam(Ctx &c, GuessModel &g, float lr);

// ---- recon.cu
void reconstruct(Ctx &c, Mesh &m, int n_t, double period, double *u_t, double *p_t);
void reconstruct_static(Ctx &c, Mesh &m, int n_t, double period, double *u_t, double *p_t);
void modal_split(Ctx &c, Mesh &m, double2 *U, double2 *Pm);  // mode-major velocity / pressure copies
void bc_spectrum(Ctx &c, int n_t, int64_t n_pts, int n_modes, const double *g_t, const double *w, double2 *c_out,
                 double *e2);
void mode_energies(Ctx &c, Mesh &m, double *E, double *incr2);

int dev_error(Ctx &c);  // reads and clears the device error word
inline void count_launch(Ctx &c) { c.launches.n++; }

}  // namespace scvs
