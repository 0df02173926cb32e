// Argument blocks of the all-modes operator and preconditioner kernels,
// shared by operators.cu (gathers from global memory) and blocks.cu (gathers
// staged in shared memory).
#pragma once
#include "scvs_internal.h"

namespace scvs {

template <typename T> struct SaddleArgs {
  int64_t N, P;
  int ld;
  const int64_t *s_ptr;
  const int32_t *s_col;
  const int32_t *g_len;
  const int64_t *g_ptr;
  const T *Kv, *Mv, *Dv, *DTv;
  int64_t g_nnz, gt_nnz;
  const uint8_t *dirmask;  // null: no identity rows
  const double *omega;
  double rho, mu;
  const int32_t *dof_comp;      // null: one component
  const uint8_t *comp_active;   // rows of inactive components are skipped
  int tile;                     // row tile (SCVS_ROW_LOOP)
};

// true if the row's component has no active system (multi-component meshes)
__device__ __forceinline__ bool row_idle(const int32_t *dof_comp, const uint8_t *comp_active, int64_t dof) {
  return dof_comp && !comp_active[dof_comp[dof]];
}

struct PcArgs {
  int64_t N, P;
  int ld;
  const int64_t *s_ptr;
  const int32_t *s_col;
  const int32_t *g_len;
  const int64_t *g_ptr;
  const void *Kv, *Mv;         // masked velocity-block values (T)
  const void *Mpv, *Lpv;       // P1 mass, Laplacian (outlet rows identity) values (T), Q pattern
  const double *ms_diag, *ks_diag, *mp_diag, *lp_diag;
  const uint8_t *dirmask, *outmask;
  const double *omega;
  double rho, mu;
  // coarse (P1) velocity level
  const void *Kcv, *Mcv;       // masked P1 stiffness / mass (T), Q pattern
  const double *k1_diag;
  const int32_t *edge_ends;
  const int64_t *v2e_ptr;
  const int32_t *v2e;
  // diagonals and per-mode scalars in the kernel's precision T
  const void *ksd, *msd, *mpd, *lpd, *k1d;
  const void *wabs, *wrho;   // [ld] |omega_k| rho, omega_k rho
  const int32_t *dof_comp;   // null: one component
  const uint8_t *comp_active;
  int tile;                  // row tile of the gather kernels (SCVS_ROW_LOOP)
  const void *Dv;            // G block values (T), [dim][g_nnz] (block-triangular form)
  int64_t g_nnz;
};

// The velocity block of mode k, A_u = mu K_s + j omega rho M_s, is preconditioned
// through the real SPD shift A_r = mu K_s + |omega| rho M_s: the spectrum of
// A_r^-1 A_u lies on the arc from j to 1 (|z| >= 1/sqrt 2) for every omega, and
// A_r has a real positive Jacobi-scaled spectrum on which a Chebyshev
// polynomial on a real interval is effective.  vel_dinv is 1 / diag(A_r).
template <typename T>
__device__ __forceinline__ T vel_dinv(const PcArgs &a, int64_t A, int k) {
  return T(1) / ((T)a.mu * ((const T *)a.ksd)[A] + ((const T *)a.wabs)[k] * ((const T *)a.msd)[A]);
}

// Coefficients of one Chebyshev step i >= 1,
//   z_next = z + alpha (z - z_prev) + beta D^-1 (r - A z),
// of the velocity polynomial (k_pc_cheb: per-mode alpha_u, beta_u) or of the
// two pressure polynomials (P1 mass and P1 Laplacian, stepped together by
// k_pressure_solve).  z_prev is overwritten by z_next (each row reads its own
// z_prev first).
struct ChebCoef {
  const double *alpha_u, *beta_u;  // [ld] per mode (velocity)
  double alpha_m, beta_m, alpha_l, beta_l;
  int do_u, do_m, do_l;
  int prev_zero_u, prev_zero_m, prev_zero_l;
  int resid_l;  // pressure Laplacian: write the residual r - L_p z (0 on the outlet) instead of a step
};

// Row blocks of a mesh for the staged kernels (blocks.cu).
struct StagedArgs {
  const int32_t *perm;      // rows in locality order
  const int64_t *row0;      // [n_blk + 1] block b = perm[row0[b] .. row0[b+1])
  const int64_t *fp_ptr;    // [n_blk + 1] footprint offsets
  const int32_t *fp_col;    // ascending footprint columns of every block
  const int32_t *fv_len;    // [n_blk] vertex columns (ids < P) at the head of each footprint
  const uint16_t *lcol;     // [s_nnz] footprint index of every nonzero (original order)
  int fp_max;               // largest footprint (shared-memory layout)
  GridSync *gs;             // error word for a staging wait that gave up
};

template <typename T>
SaddleArgs<T> saddle_args(const Ctx &c, const Mesh &m, bool masked);

// blocks.cu
StagedArgs staged_args(const Ctx &c, const Mesh &m);
bool staged_ok(const Ctx &c, const Mesh &m, int mc, bool pres, const void *x);
void launch_cheb_staged(Ctx &c, const Mesh &m, const PcArgs &a, const ChebCoef &cc, const float2 *r, const float2 *zu,
                        float2 *zu_prev, int mc);
void launch_vel_residual_staged(Ctx &c, const Mesh &m, const PcArgs &a, const float2 *r, const float2 *z, float2 *rr,
                                int mc);
void launch_saddle_staged(Ctx &c, const Mesh &m, const SaddleArgs<float> &a, const float2 *x, float2 *y, int mc);

}  // namespace scvs
