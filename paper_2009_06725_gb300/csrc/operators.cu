// All-modes operators on mode-interleaved complex blocks.
//
// Block layout: element (dof, k) at dof*ld + k; velocity dof = node*dim + c,
// then the pressure dof of every vertex at dim*N + vertex (Eq. linear_sys_def).
//
//  * k_saddle   y_k = A(omega_k) x_k for all modes (Eq. linear_sys_def) with the
//               pattern of S (velocity rows: M_s, K_s over the whole row, D_c over
//               the leading P1 columns; pressure rows: D_c^T over the S row of the
//               vertex).  One row group of L lanes per row; each nonzero is
//               loaded once by one lane and broadcast by shuffle, so its column
//               index and values serve every mode of the row; every lane owns
//               MPL modes and gathers them with one 16-byte load per component.
//  * lift / residual / per-mode norms
//  * block preconditioner: Chebyshev-Jacobi polynomials of the velocity block
//    mu K_s + j omega rho M_s (per mode) and of the P1 pressure mass and
//    Laplacian (Cahouet-Chabard combination mu M_p^-1 + j omega rho L_p^-1),
//    or their diagonal versions.
#include <algorithm>
#include <cmath>
#include <type_traits>
#include "scvs_internal.h"
#include "vecops.cuh"
#include "opargs.cuh"

namespace scvs {



template <typename T, int MPL, int L, int DIM>
__global__ void __launch_bounds__(256)
k_saddle(const SaddleArgs<T> a, const typename cpx<T>::t *__restrict__ x, typename cpx<T>::t *__restrict__ y) {
  using C = typename cpx<T>::t;
  const int gpb = blockDim.x / L;
  const int lane = threadIdx.x % L, group = threadIdx.x / L;
  const unsigned gm = group_mask<L>();
  const int ld = a.ld;
  const int koff = lane * MPL;
  T wr[MPL];
#pragma unroll
  for (int i = 0; i < MPL; ++i) wr[i] = (T)(a.omega[koff + i] * a.rho);
  const T mu = (T)a.mu;
  const int64_t rows = a.N + a.P;
  const C *__restrict__ xp_base = x + (int64_t)DIM * a.N * ld + koff;
  SCVS_ROW_LOOP(row, 0, rows, gpb, group, a.tile) {
    if (row_idle(a.dof_comp, a.comp_active, row < a.N ? row * DIM : (int64_t)DIM * a.N + (row - a.N))) continue;
    if (row < a.N) {
      const int64_t A = row;
      if (a.dirmask && a.dirmask[A]) {
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          CV<T, MPL> v;
          ldv<T, MPL>(v, x + (A * DIM + c) * ld + koff);
          stv<T, MPL>(y + (A * DIM + c) * ld + koff, v);
        }
        continue;
      }
      // y = sum_B (mu K + j omega rho M)_AB x_B + sum_B D_AB x_p,B: one complex
      // coefficient per nonzero and mode, one accumulator per component
      CV<T, MPL> acc[DIM];
#pragma unroll
      for (int c = 0; c < DIM; ++c) acc[c].zero();
      const int64_t r0 = a.s_ptr[A], r1 = a.s_ptr[A + 1];
      const int64_t gend = r0 + a.g_len[A];
      const int64_t goff = a.g_ptr[A] - r0;
      for (int64_t base = r0; base < r1; base += L) {
        const int64_t t = base + lane;
        int32_t col = 0;
        T kv = 0, mv = 0, dv[DIM];
#pragma unroll
        for (int c = 0; c < DIM; ++c) dv[c] = 0;
        if (t < r1) {
          col = __ldg(a.s_col + t);
          kv = mu * __ldg(a.Kv + t);
          mv = __ldg(a.Mv + t);
          if (t < gend) {
#pragma unroll
            for (int c = 0; c < DIM; ++c) dv[c] = __ldg(a.Dv + c * a.g_nnz + t + goff);
          }
        }
        const int cnt = (int)min((int64_t)L, r1 - base);
        const int gcnt = (int)max((int64_t)0, min((int64_t)L, gend - base));
#pragma unroll 4
        for (int q = 0; q < cnt; ++q) {
          const int32_t B = gshfl<L>(gm, col, q);
          const T cr = gshfl<L>(gm, kv, q), mq = gshfl<L>(gm, mv, q);
          T ci[MPL];
#pragma unroll
          for (int i = 0; i < MPL; ++i) ci[i] = wr[i] * mq;
#pragma unroll
          for (int c = 0; c < DIM; ++c) {
            CV<T, MPL> xv;
            ldv<T, MPL>(xv, x + ((int64_t)B * DIM + c) * ld + koff);
#pragma unroll
            for (int i = 0; i < MPL; ++i) {
              acc[c].re[i] = fma(cr, xv.re[i], fma(-ci[i], xv.im[i], acc[c].re[i]));
              acc[c].im[i] = fma(cr, xv.im[i], fma(ci[i], xv.re[i], acc[c].im[i]));
            }
          }
          if (q < gcnt) {  // uniform across the row group
            CV<T, MPL> xq;
            ldv<T, MPL>(xq, xp_base + (int64_t)B * ld);
#pragma unroll
            for (int c = 0; c < DIM; ++c) axpy(acc[c], gshfl<L>(gm, dv[c], q), xq);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < DIM; ++c) stv<T, MPL>(y + (A * DIM + c) * ld + koff, acc[c]);
    } else {
      const int64_t B = row - a.N;
      CV<T, MPL> acc;
      acc.zero();
      const int64_t r0 = a.s_ptr[B], r1 = a.s_ptr[B + 1];
      for (int64_t base = r0; base < r1; base += L) {
        const int64_t t = base + lane;
        int32_t col = 0;
        T dt[DIM];
#pragma unroll
        for (int c = 0; c < DIM; ++c) dt[c] = 0;
        if (t < r1) {
          col = __ldg(a.s_col + t);
#pragma unroll
          for (int c = 0; c < DIM; ++c) dt[c] = __ldg(a.DTv + c * a.gt_nnz + t);
        }
        const int cnt = (int)min((int64_t)L, r1 - base);
#pragma unroll 4
        for (int q = 0; q < cnt; ++q) {
          const int32_t Acol = gshfl<L>(gm, col, q);
#pragma unroll
          for (int c = 0; c < DIM; ++c) {
            CV<T, MPL> xv;
            ldv<T, MPL>(xv, x + ((int64_t)Acol * DIM + c) * ld + koff);
            axpy(acc, gshfl<L>(gm, dt[c], q), xv);
          }
        }
      }
      stv<T, MPL>(y + ((int64_t)DIM * a.N + B) * ld + koff, acc);
    }
  }
}

template <typename T>
SaddleArgs<T> saddle_args(const Ctx &c, const Mesh &m, bool masked);

template <>
SaddleArgs<float> saddle_args<float>(const Ctx &, const Mesh &m, bool) {
  return SaddleArgs<float>{m.N, m.P, m.ld, m.s_ptr, m.s_col, m.g_len, m.g_ptr, m.Ks_f, m.Ms_f, m.Dv_f,
                           m.DTv_f, m.g_nnz, m.gt_nnz, m.dirmask, m.omega_d, m.rho, m.mu, m.dof_comp, m.comp_active,
                           m.tile_spmm ? m.tile_spmm : SCVS_DEFAULT_TILE};
}
template <>
SaddleArgs<double> saddle_args<double>(const Ctx &, const Mesh &m, bool masked) {
  return SaddleArgs<double>{m.N, m.P, m.ld, m.s_ptr, m.s_col, m.g_len, m.g_ptr,
                            masked ? m.Ks_m : m.Ks, masked ? m.Ms_m : m.Ms,
                            masked ? m.Dv_m : m.Dv, masked ? m.DTv_m : m.DTv,
                            m.g_nnz, m.gt_nnz, masked ? m.dirmask : nullptr, m.omega_d, m.rho, m.mu,
                            masked ? m.dof_comp : nullptr, m.comp_active, SCVS_DEFAULT_TILE};
}

// Algorithmic bytes of one all-modes SpMM: every index and value array once,
// x read once, y written once.
double saddle_bytes(const Mesh &m, int vs) {
  const double mat = (double)m.s_nnz * (4 + 2 * vs) + (double)m.dim * (m.g_nnz + m.gt_nnz) * vs +
                     (double)(m.N + 1) * 16 + (double)m.N * 5;
  return mat + 2.0 * m.n_dof * m.ld * 2 * vs;
}

static unsigned row_blocks(const Ctx &c, int64_t rows, int groups_per_block, int tile = 1) {
  const int64_t span = (int64_t)groups_per_block * tile;
  int64_t need = (rows + span - 1) / span;
  return (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)c.num_sms * 32));
}

template <typename T>
void launch_saddle(Ctx &c, const Mesh &m, const SaddleArgs<T> &a, const typename cpx<T>::t *x,
                   typename cpx<T>::t *y) {
  KScope ks(c, sizeof(T) == 4 ? KC_SPMM32 : KC_SPMM64, saddle_bytes(m, sizeof(T)));
  if constexpr (sizeof(T) == 4) {
    if (m.st_spmm && a.dirmask && staged_ok(c, m, m.st_spmm, true, x)) {
      launch_saddle_staged(c, m, a, x, y, m.st_spmm);
      return;
    }
    const int mpl = m.mpl_spmm ? m.mpl_spmm : default_mpl<T>(m.ld);
    SCVS_DISPATCH_SHAPE(m.ld, mpl, {
      const int gpb = 256 / L;
      const unsigned nb = row_blocks(c, m.N + m.P, gpb, a.tile);
      if (m.dim == 2)
        k_saddle<T, MPL, L, 2><<<nb, 256, 0, c.stream>>>(a, x, y);
      else
        k_saddle<T, MPL, L, 3><<<nb, 256, 0, c.stream>>>(a, x, y);
    });
  } else {
    SCVS_DISPATCH_LD(T, m.ld, {
      const int gpb = 256 / L;
      const unsigned nb = row_blocks(c, m.N + m.P, gpb, a.tile);
      if (m.dim == 2)
        k_saddle<T, MPL, L, 2><<<nb, 256, 0, c.stream>>>(a, x, y);
      else
        k_saddle<T, MPL, L, 3><<<nb, 256, 0, c.stream>>>(a, x, y);
    });
  }
  count_launch(c);
}

template <typename T>
void apply_saddle(Ctx &c, const Mesh &m, const typename cpx<T>::t *x, typename cpx<T>::t *y) {
  launch_saddle<T>(c, m, saddle_args<T>(c, m, true), x, y);
}
template void apply_saddle<float>(Ctx &, const Mesh &, const float2 *, float2 *);
template void apply_saddle<double>(Ctx &, const Mesh &, const double2 *, double2 *);

// ------------------------------------------------------------------- lift
__global__ void k_scatter_dirichlet(const double2 *__restrict__ g, const int64_t *__restrict__ dir_nodes,
                                    int64_t n_dir, int dim, int m, int ld, double2 *__restrict__ gfull) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int64_t total = (int64_t)m * n_dir * dim;
  if (t >= total) return;
  int k = (int)(t / (n_dir * dim));
  int64_t r = t % (n_dir * dim);
  int64_t i = r / dim;
  int c = (int)(r % dim);
  gfull[(dir_nodes[i] * dim + c) * ld + k] = g[t];
}

// b = -y (+ the Neumann load on velocity rows) on free rows, b = gfull on
// Dirichlet velocity rows
__global__ void k_lift_finish(const double2 *__restrict__ y, const double2 *__restrict__ gfull,
                              const uint8_t *__restrict__ dirm, int64_t N, int dim, int64_t n_dof, int ld,
                              const double2 *__restrict__ neu, double2 *__restrict__ b) {
  int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= n_dof * ld) return;
  int64_t dof = f / ld;
  bool dir = dof < N * dim && dirm[dof / dim];
  double2 v = y[f];
  if (dir) {
    b[f] = gfull[f];
  } else if (neu && dof < N * dim) {
    const double2 l = neu[f];
    b[f] = make_double2(l.x - v.x, l.y - v.y);
  } else {
    b[f] = make_double2(-v.x, -v.y);
  }
}

// Deterministic per-system squared norms over the free rows: one block per
// row chunk writes its partial per mode, then one thread per system sums the
// partials of its component's chunks in chunk order.
constexpr int NORM_T = 256;
__global__ void k_chunk_norm2(const double2 *__restrict__ v, const uint8_t *__restrict__ dirm, int64_t N, int dim,
                              int ld, int64_t n_chunk, const int64_t *__restrict__ row0,
                              const int32_t *__restrict__ rows, const int32_t *__restrict__ chunk_comp,
                              const uint8_t *__restrict__ comp_active, double *__restrict__ part) {
  __shared__ double s[NORM_T];
  for (int64_t ch = blockIdx.x; ch < n_chunk; ch += gridDim.x) {
    if (!comp_active[chunk_comp[ch]]) continue;  // block-uniform
    const int64_t f0 = row0[ch] * ld, f1 = (row0[ch] + rows[ch]) * ld;
    double acc = 0.0;
    for (int64_t f = f0 + threadIdx.x; f < f1; f += NORM_T) {  // stride is a multiple of ld
      const int64_t dof = f / ld;
      const bool dir = dof < N * dim && dirm[dof / dim];
      if (!dir) { const double2 z = v[f]; acc += z.x * z.x + z.y * z.y; }
    }
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = NORM_T / 2; w >= ld; w >>= 1) {
      if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
      __syncthreads();
    }
    // thread t < ld holds mode (f0 + t) % ld = t (f0 is a multiple of ld)
    if (threadIdx.x < ld) part[ch * ld + threadIdx.x] = s[threadIdx.x];
    __syncthreads();
  }
}

__global__ void k_comp_reduce(const double *__restrict__ part, const int32_t *__restrict__ comp_chunk, int n_comp,
                              int ld, double *__restrict__ out) {
  const int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= n_comp * ld) return;
  const int comp = sys / ld, k = sys % ld;
  double s = 0.0;
  for (int ch = comp_chunk[comp]; ch < comp_chunk[comp + 1]; ++ch) s += part[(int64_t)ch * ld + k];
  out[sys] = s;
}

void norms2_sys(Ctx &c, const Mesh &m, const double2 *v, double *out) {
  KScope ks(c, KC_VECTOR, (double)m.n_dof * m.ld * 16);
  double *part = nullptr;
  SCVS_CUDA(ctx_malloc(c, &part, (size_t)m.n_chunk * m.ld * sizeof(double), c.stream));
  const unsigned nb = (unsigned)std::min<int64_t>(m.n_chunk, 8 * c.num_sms);
  k_chunk_norm2<<<nb, NORM_T, 0, c.stream>>>(v, m.dirmask, m.N, m.dim, m.ld, m.n_chunk, m.chunk_row0, m.chunk_rows,
                                             m.chunk_comp, m.comp_active, part);
  k_comp_reduce<<<ceil_div(m.n_sys(), 128), 128, 0, c.stream>>>(part, m.comp_chunk, m.n_comp, m.ld, out);
  c.launches.n += 2;
  SCVS_CUDA(cudaFreeAsync(part, c.stream));
}

// Row chunks of a mesh: dof rows split where the component changes and every
// CHUNK_ROWS rows, then grouped by component (stable).  node_comp null: one
// component.
void set_chunks(Ctx &c, Mesh &m, const int32_t *node_comp, int n_comp) {
  std::vector<int32_t> dc(m.n_dof, 0);
  if (node_comp) {
    for (int64_t nd = 0; nd < m.N; ++nd)
      for (int q = 0; q < m.dim; ++q) dc[nd * m.dim + q] = node_comp[nd];
    for (int64_t v = 0; v < m.P; ++v) dc[(int64_t)m.dim * m.N + v] = node_comp[v];
  }
  std::vector<std::vector<std::pair<int64_t, int32_t>>> per(n_comp);
  int64_t r = 0;
  while (r < m.n_dof) {
    const int32_t cc = dc[r];
    int64_t e = r + 1;
    while (e < m.n_dof && e - r < CHUNK_ROWS && dc[e] == cc) ++e;
    per[cc].push_back({r, (int32_t)(e - r)});
    r = e;
  }
  std::vector<int64_t> r0;
  std::vector<int32_t> rows, comp, cptr(n_comp + 1, 0);
  for (int q = 0; q < n_comp; ++q) {
    cptr[q] = (int32_t)r0.size();
    for (auto &pr : per[q]) { r0.push_back(pr.first); rows.push_back(pr.second); comp.push_back(q); }
  }
  cptr[n_comp] = (int32_t)r0.size();
  m.n_comp = n_comp;
  m.n_chunk = (int64_t)r0.size();
  m.chunk_row0 = m.arena.alloc<int64_t>(m.n_chunk);
  m.chunk_rows = m.arena.alloc<int32_t>(m.n_chunk);
  m.chunk_comp = m.arena.alloc<int32_t>(m.n_chunk);
  m.comp_chunk = m.arena.alloc<int32_t>(n_comp + 1);
  SCVS_CUDA(cudaMemcpy(m.chunk_row0, r0.data(), r0.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
  SCVS_CUDA(cudaMemcpy(m.chunk_rows, rows.data(), rows.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  SCVS_CUDA(cudaMemcpy(m.chunk_comp, comp.data(), comp.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  SCVS_CUDA(cudaMemcpy(m.comp_chunk, cptr.data(), cptr.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  m.comp_active = m.arena.alloc<uint8_t>(n_comp);
  SCVS_CUDA(cudaMemset(m.comp_active, 1, n_comp));
  if (n_comp > 1) {
    m.dof_comp = m.arena.alloc<int32_t>(m.n_dof);
    SCVS_CUDA(cudaMemcpy(m.dof_comp, dc.data(), dc.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  } else {
    m.dof_comp = nullptr;
  }
}

void lift_rhs(Ctx &c, Mesh &m) {
  const int64_t total = m.n_dof * m.ld;
  double2 *gfull = nullptr, *y = nullptr;
  double *nrm = nullptr;
  SCVS_CUDA(ctx_malloc(c, &gfull, total * sizeof(double2), c.stream));
  SCVS_CUDA(ctx_malloc(c, &y, total * sizeof(double2), c.stream));
  SCVS_CUDA(ctx_malloc(c, &nrm, m.n_sys() * sizeof(double), c.stream));
  SCVS_CUDA(cudaMemsetAsync(gfull, 0, total * sizeof(double2), c.stream));
  if (m.n_dir > 0 && m.m > 0) {
    int64_t tt = (int64_t)m.m * m.n_dir * m.dim;
    k_scatter_dirichlet<<<ceil_div(tt, 256), 256, 0, c.stream>>>(m.g, m.dir_nodes, m.n_dir, m.dim, m.m, m.ld, gfull);
    count_launch(c);
  }
  launch_saddle<double>(c, m, saddle_args<double>(c, m, false), gfull, y);
  {
    KScope ks(c, KC_VECTOR, (double)total * 48);
    k_lift_finish<<<ceil_div(total, 256), 256, 0, c.stream>>>(y, gfull, m.dirmask, m.N, m.dim, m.n_dof, m.ld, m.neu,
                                                              m.b);
    count_launch(c);
  }
  norms2_sys(c, m, m.b, nrm);
  std::vector<double> h(m.n_sys());
  SCVS_CUDA(cudaMemcpyAsync(h.data(), nrm, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaFreeAsync(gfull, c.stream));
  SCVS_CUDA(cudaFreeAsync(y, c.stream));
  SCVS_CUDA(cudaFreeAsync(nrm, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  m.bnorm.assign(m.n_sys(), 0.0);
  for (int s = 0; s < m.n_sys(); ++s) m.bnorm[s] = std::sqrt(h[s]);
}

// --------------------------------------------------------------- residual
// r = b - A_hat x on every row (zero on Dirichlet rows when x_D = g); writes
// the FP32 copy (right-hand side of the next FP32 cycle) and, optionally, FP64.
__global__ void k_residual_finish(const double2 *__restrict__ b, const double2 *__restrict__ ax,
                                  const uint8_t *__restrict__ dirm, int64_t N, int dim, int64_t total, int ld,
                                  float2 *__restrict__ r32, double2 *__restrict__ r64,
                                  const int32_t *__restrict__ dof_comp, const uint8_t *__restrict__ comp_active) {
  int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= total) return;
  int64_t dof = f / ld;
  if (row_idle(dof_comp, comp_active, dof)) return;
  bool dir = dof < N * dim && dirm[dof / dim];
  double2 bb = b[f], a = ax ? ax[f] : make_double2(0.0, 0.0);
  double2 r = dir ? make_double2(0.0, 0.0) : make_double2(bb.x - a.x, bb.y - a.y);
  if (r32) r32[f] = make_float2((float)r.x, (float)r.y);
  if (r64) r64[f] = r;
}

// ----------------------------------------------------- preconditioner


// Step 0 of the velocity polynomial (elementwise over elements [0, f1) of the
// block), optionally rescaling r by rscale[k] first (written back: lazy
// normalisation of the Krylov vector): z_u = r / (diag A_r theta_u[k]),
// Dirichlet rows z_u = r.  The block-diagonal DIAG kind covers the whole block
// (f1 = n_dof ld) with the diagonal blocks only: z_u = r / diag A_r and
// z_p = (mu / diag M_p + j omega rho / diag L_p) r.  (The pressure polynomials
// of the other kinds start inside k_pressure_solve.)
template <typename T, int DIM, bool DIAG>
__global__ void k_pc_step0(const PcArgs a, typename cpx<T>::t *r, const double *__restrict__ rscale,
                           const double *__restrict__ inv_theta_u, typename cpx<T>::t *__restrict__ zu, int64_t f1) {
  using C = typename cpx<T>::t;
  int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= f1) return;
  const int64_t dof = f / a.ld;
  const int k = (int)(f % a.ld);
  if (row_idle(a.dof_comp, a.comp_active, dof)) return;
  C v = r[f];
  if (rscale) {
    T s = (T)rscale[(a.dof_comp ? a.dof_comp[dof] * a.ld : 0) + k];
    v.x *= s; v.y *= s;
    r[f] = v;
  }
  if (dof < (int64_t)DIM * a.N) {
    const int64_t A = dof / DIM;
    if (a.dirmask[A]) { zu[f] = v; return; }
    const T s = vel_dinv<T>(a, A, k) * (DIAG ? T(1) : (T)inv_theta_u[k]);
    zu[f] = mk<T>(s * v.x, s * v.y);
  } else if (DIAG) {
    const int64_t B = dof - (int64_t)DIM * a.N;
    const bool out = a.outmask[B];
    const double w = a.omega[k] * a.rho;
    const T cm = (T)(a.mu / a.mp_diag[B]);
    const T cl = out ? T(0) : (T)(w / a.lp_diag[B]);
    zu[f] = mk<T>(cm * v.x - cl * v.y, cm * v.y + cl * v.x);  // (cm + j cl) v
  }
}


// One Chebyshev step of both pressure polynomials (P1 mass, P1 Laplacian with
// p = 0 on the outlet) on pressure row B, for the lane's modes.
template <typename T, int MPL, int L, int DIM>
__device__ __forceinline__ void pressure_row_step(const PcArgs &a, const ChebCoef &cc, const int64_t B,
                                                  const typename cpx<T>::t *__restrict__ r,
                                                  const typename cpx<T>::t *__restrict__ zM,
                                                  typename cpx<T>::t *__restrict__ zM_prev,
                                                  const typename cpx<T>::t *__restrict__ zL,
                                                  typename cpx<T>::t *__restrict__ zL_prev, const int lane,
                                                  const unsigned gm) {
  using C = typename cpx<T>::t;
  const int ld = a.ld, koff = lane * MPL;
  const T *Mpv = (const T *)a.Mpv, *Lpv = (const T *)a.Lpv;
  const int64_t r0 = a.g_ptr[B], r1 = a.g_ptr[B + 1];  // Q row = leading part of the S row
  const int64_t s0 = a.s_ptr[B];
  CV<T, MPL> aMp, aLp;
  aMp.zero(); aLp.zero();
  for (int64_t base = r0; base < r1; base += L) {
    const int64_t t = base + lane;
    int32_t col = 0;
    T mv = 0, lv = 0;
    if (t < r1) { col = __ldg(a.s_col + s0 + (t - r0)); mv = __ldg(Mpv + t); lv = __ldg(Lpv + t); }
    const int cnt = (int)min((int64_t)L, r1 - base);
#pragma unroll 4
    for (int q = 0; q < cnt; ++q) {
      const int32_t Bc = gshfl<L>(gm, col, q);
      const T mq = gshfl<L>(gm, mv, q), lq = gshfl<L>(gm, lv, q);
      if (cc.do_m) { CV<T, MPL> v; ldv_co<T, MPL>(v, zM + (int64_t)Bc * ld + koff); axpy(aMp, mq, v); }
      if (cc.do_l) { CV<T, MPL> v; ldv_co<T, MPL>(v, zL + (int64_t)Bc * ld + koff); axpy(aLp, lq, v); }
    }
  }
  const int64_t rf = ((int64_t)DIM * a.N + B) * ld;
  const bool out = a.outmask[B];
  const T dm = T(1) / ((const T *)a.mpd)[B], dl = T(1) / ((const T *)a.lpd)[B];
#pragma unroll
  for (int i = 0; i < MPL; ++i) {
    const int k = koff + i;
    const int64_t pf = B * ld + k;
    const C rv = ld1co(r + rf + k);
    if (cc.do_m) {
      const C z = ld1co(zM + pf);
      const C zp = cc.prev_zero_m ? mk<T>(0, 0) : ld1co(zM_prev + pf);
      const T al = (T)cc.alpha_m, be = (T)cc.beta_m;
      zM_prev[pf] = mk<T>(z.x + al * (z.x - zp.x) + be * dm * (rv.x - aMp.re[i]),
                          z.y + al * (z.y - zp.y) + be * dm * (rv.y - aMp.im[i]));
    }
    if (cc.do_l) {
      const T rr = out ? T(0) : rv.x, ri = out ? T(0) : rv.y;
      if (cc.resid_l) {
        zL_prev[pf] = out ? mk<T>(0, 0) : mk<T>(rr - aLp.re[i], ri - aLp.im[i]);
      } else {
        const C z = ld1co(zL + pf);
        const C zp = cc.prev_zero_l ? mk<T>(0, 0) : ld1co(zL_prev + pf);
        const T al = (T)cc.alpha_l, be = (T)cc.beta_l;
        zL_prev[pf] = mk<T>(z.x + al * (z.x - zp.x) + be * dl * (rr - aLp.re[i]),
                            z.y + al * (z.y - zp.y) + be * dl * (ri - aLp.im[i]));
      }
    }
  }
}

template <typename T, int MPL, int L, int DIM>
__global__ void __launch_bounds__(256)
k_pc_cheb(const PcArgs a, const ChebCoef cc, const typename cpx<T>::t *__restrict__ r,
          const typename cpx<T>::t *__restrict__ zu, typename cpx<T>::t *__restrict__ zu_prev) {
  using C = typename cpx<T>::t;
  const int gpb = blockDim.x / L;
  const int lane = threadIdx.x % L, group = threadIdx.x / L;
  const unsigned gm = group_mask<L>();
  const int ld = a.ld, koff = lane * MPL;
  const T *Kv = (const T *)a.Kv, *Mv = (const T *)a.Mv;
  SCVS_ROW_LOOP(A, 0, a.N, gpb, group, a.tile) {
    if (row_idle(a.dof_comp, a.comp_active, A * DIM)) continue;
    {
      if (a.dirmask[A]) {
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          CV<T, MPL> v;
          ldv<T, MPL>(v, r + (A * DIM + c) * ld + koff);
          stv<T, MPL>(zu_prev + (A * DIM + c) * ld + koff, v);
        }
        continue;
      }
      CV<T, MPL> acc[DIM];  // A_r z with the real per-mode coefficient mu K + |omega| rho M
#pragma unroll
      for (int c = 0; c < DIM; ++c) acc[c].zero();
      T cw[MPL];
#pragma unroll
      for (int i = 0; i < MPL; ++i) cw[i] = ((const T *)a.wabs)[koff + i];
      const T muT = (T)a.mu;
      const int64_t r0 = a.s_ptr[A], r1 = a.s_ptr[A + 1];
      for (int64_t base = r0; base < r1; base += L) {
        const int64_t t = base + lane;
        int32_t col = 0;
        T kv = 0, mv = 0;
        if (t < r1) { col = __ldg(a.s_col + t); kv = muT * __ldg(Kv + t); mv = __ldg(Mv + t); }
        const int cnt = (int)min((int64_t)L, r1 - base);
#pragma unroll 4
        for (int q = 0; q < cnt; ++q) {
          const int32_t B = gshfl<L>(gm, col, q);
          const T kq = gshfl<L>(gm, kv, q), mq = gshfl<L>(gm, mv, q);
#pragma unroll
          for (int c = 0; c < DIM; ++c) {
            CV<T, MPL> xv;
            ldv<T, MPL>(xv, zu + ((int64_t)B * DIM + c) * ld + koff);
#pragma unroll
            for (int i = 0; i < MPL; ++i) {
              const T cf = fma(cw[i], mq, kq);
              acc[c].re[i] = fma(cf, xv.re[i], acc[c].re[i]);
              acc[c].im[i] = fma(cf, xv.im[i], acc[c].im[i]);
            }
          }
        }
      }
      T dr[MPL], al[MPL], be[MPL];
#pragma unroll
      for (int i = 0; i < MPL; ++i) {
        dr[i] = vel_dinv<T>(a, A, koff + i);
        al[i] = (T)cc.alpha_u[koff + i];
        be[i] = (T)cc.beta_u[koff + i];
      }
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        const int64_t f0 = (A * DIM + c) * ld + koff;
        CV<T, MPL> rv, z, zp, o;
        ldv<T, MPL>(rv, r + f0);
        ldv<T, MPL>(z, zu + f0);
        if (cc.prev_zero_u) zp.zero(); else ldv_cg<T, MPL>(zp, zu_prev + f0);
#pragma unroll
        for (int i = 0; i < MPL; ++i) {
          const T ur = dr[i] * (rv.re[i] - acc[c].re[i]), ui = dr[i] * (rv.im[i] - acc[c].im[i]);
          o.re[i] = z.re[i] + al[i] * (z.re[i] - zp.re[i]) + be[i] * ur;
          o.im[i] = z.im[i] + al[i] * (z.im[i] - zp.im[i]) + be[i] * ui;
        }
        stv<T, MPL>(zu_prev + f0, o);
      }
    }
  }
}


// ---------------------------------------------------- two-level velocity cycle
// rr = r - A_r z on the velocity rows (zero on Dirichlet rows).
template <typename T, int MPL, int L, int DIM>
__global__ void __launch_bounds__(256)
k_vel_residual(const PcArgs a, const typename cpx<T>::t *__restrict__ r, const typename cpx<T>::t *__restrict__ z,
               typename cpx<T>::t *__restrict__ rr) {
  using C = typename cpx<T>::t;
  const int gpb = blockDim.x / L;
  const int lane = threadIdx.x % L, group = threadIdx.x / L;
  const unsigned gm = group_mask<L>();
  const int ld = a.ld, koff = lane * MPL;
  const T *Kv = (const T *)a.Kv, *Mv = (const T *)a.Mv;
  SCVS_ROW_LOOP(A, 0, a.N, gpb, group, a.tile) {
    if (row_idle(a.dof_comp, a.comp_active, A * DIM)) continue;
    if (a.dirmask[A]) {
      CV<T, MPL> zz;
      zz.zero();
#pragma unroll
      for (int c = 0; c < DIM; ++c) stv<T, MPL>(rr + (A * DIM + c) * ld + koff, zz);
      continue;
    }
    CV<T, MPL> acc[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) acc[c].zero();
    T cr[MPL];
#pragma unroll
    for (int i = 0; i < MPL; ++i) cr[i] = ((const T *)a.wabs)[koff + i];
    const T mu = (T)a.mu;
    const int64_t r0 = a.s_ptr[A], r1 = a.s_ptr[A + 1];
    for (int64_t base = r0; base < r1; base += L) {
      const int64_t t = base + lane;
      int32_t col = 0;
      T kv = 0, mv = 0;
      if (t < r1) { col = __ldg(a.s_col + t); kv = __ldg(Kv + t); mv = __ldg(Mv + t); }
      const int cnt = (int)min((int64_t)L, r1 - base);
#pragma unroll 4
      for (int q = 0; q < cnt; ++q) {
        const int32_t B = gshfl<L>(gm, col, q);
        const T kq = mu * gshfl<L>(gm, kv, q), mq = gshfl<L>(gm, mv, q);
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          CV<T, MPL> xv;
          ldv<T, MPL>(xv, z + ((int64_t)B * DIM + c) * ld + koff);
#pragma unroll
          for (int i = 0; i < MPL; ++i) {
            const T cf = kq + cr[i] * mq;  // real coefficient of A_r
            acc[c].re[i] = fma(cf, xv.re[i], acc[c].re[i]);
            acc[c].im[i] = fma(cf, xv.im[i], acc[c].im[i]);
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      CV<T, MPL> rv, o;
      ldv<T, MPL>(rv, r + (A * DIM + c) * ld + koff);
#pragma unroll
      for (int i = 0; i < MPL; ++i) { o.re[i] = rv.re[i] - acc[c].re[i]; o.im[i] = rv.im[i] - acc[c].im[i]; }
      stv<T, MPL>(rr + (A * DIM + c) * ld + koff, o);
    }
  }
}

// z += P zc on the free velocity nodes (vertices copy, edge nodes average their ends).
template <typename T>
__global__ void k_prolong(const PcArgs a, int dim, const typename cpx<T>::t *__restrict__ zc,
                          typename cpx<T>::t *__restrict__ z) {
  // two consecutive elements (modes k, k+1 of one node and component) per
  // thread: dim * ld is even, so both belong to the same node
  const int64_t f = 2 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
  const int64_t per = (int64_t)dim * a.ld;
  if (f >= a.N * per) return;
  const int64_t n = f / per, rem = f % per;
  if (a.dirmask[n] || row_idle(a.dof_comp, a.comp_active, n * dim)) return;
  CV<T, 2> c0, o;
  if (n < a.P) {
    ldv<T, 2>(c0, zc + n * per + rem);
  } else {
    const int64_t i = n - a.P;
    CV<T, 2> c1;
    ldv<T, 2>(c0, zc + (int64_t)a.edge_ends[2 * i] * per + rem);
    ldv<T, 2>(c1, zc + (int64_t)a.edge_ends[2 * i + 1] * per + rem);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      c0.re[q] = T(0.5) * (c0.re[q] + c1.re[q]);
      c0.im[q] = T(0.5) * (c0.im[q] + c1.im[q]);
    }
  }
  ldv<T, 2>(o, z + f);
#pragma unroll
  for (int q = 0; q < 2; ++q) { o.re[q] += c0.re[q]; o.im[q] += c0.im[q]; }
  stv<T, 2>(z + f, o);
}

// Coarse operator A_c = mu K_1 + |omega| rho M_1 (P1, Dirichlet vertices removed);
// step 0: zc = rc / (diag A_c theta_c[k]).
template <typename T>
__device__ __forceinline__ T coarse_dinv(const PcArgs &a, int64_t v, int k) {
  return T(1) / ((T)a.mu * ((const T *)a.k1d)[v] + ((const T *)a.wabs)[k] * ((const T *)a.mpd)[v]);
}

// rc = P^T rr at element f of the coarse block [P][dim][ld]: own value plus
// half of every incident edge node (the transpose of P2 interpolation of a P1
// field); zero on Dirichlet vertices.
template <typename T>
__device__ __forceinline__ void restrict_elem(const PcArgs &a, int dim, const typename cpx<T>::t *__restrict__ rr,
                                              typename cpx<T>::t *__restrict__ rc, int64_t f) {
  const int64_t per = (int64_t)dim * a.ld;
  const int64_t v = f / per, rem = f % per;
  if (row_idle(a.dof_comp, a.comp_active, v * dim)) return;
  if (a.dirmask[v]) { rc[f] = mk<T>(0, 0); return; }
  auto s = rr[v * per + rem];
  T xr = s.x, xi = s.y;
  for (int64_t i = a.v2e_ptr[v]; i < a.v2e_ptr[v + 1]; ++i) {
    const auto e = rr[(int64_t)a.v2e[i] * per + rem];
    xr += T(0.5) * e.x;
    xi += T(0.5) * e.y;
  }
  rc[f] = mk<T>(xr, xi);
}

// One coarse Chebyshev step on vertex row v (all components, the lane's modes):
// zc_next = zc + alpha (zc - zc_prev) + beta D_c^-1 (rc - A_c zc), written over zc_prev.
template <typename T, int MPL, int L, int DIM>
__device__ __forceinline__ void coarse_row_step(const PcArgs &a, const double *__restrict__ alpha,
                                                const double *__restrict__ beta, bool prev_zero,
                                                const typename cpx<T>::t *__restrict__ rc,
                                                const typename cpx<T>::t *__restrict__ zc,
                                                typename cpx<T>::t *__restrict__ zc_prev, const int64_t v,
                                                const int lane, const unsigned gm) {
  using C = typename cpx<T>::t;
  const int ld = a.ld, koff = lane * MPL;
  if (a.dirmask[v]) {
    CV<T, MPL> zz;
    zz.zero();
#pragma unroll
    for (int c = 0; c < DIM; ++c) stv<T, MPL>(zc_prev + (v * DIM + c) * ld + koff, zz);
    return;
  }
  const T *Kc = (const T *)a.Kcv, *Mc = (const T *)a.Mcv;
  T cr[MPL];
#pragma unroll
  for (int i = 0; i < MPL; ++i) cr[i] = ((const T *)a.wabs)[koff + i];
  const T mu = (T)a.mu;
  CV<T, MPL> acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c].zero();
  const int64_t r0 = a.g_ptr[v], r1 = a.g_ptr[v + 1], s0 = a.s_ptr[v];
  for (int64_t base = r0; base < r1; base += L) {
    const int64_t t = base + lane;
    int32_t col = 0;
    T kv = 0, mv = 0;
    if (t < r1) { col = __ldg(a.s_col + s0 + (t - r0)); kv = __ldg(Kc + t); mv = __ldg(Mc + t); }
    const int cnt = (int)min((int64_t)L, r1 - base);
#pragma unroll 4
    for (int q = 0; q < cnt; ++q) {
      const int32_t B = gshfl<L>(gm, col, q);
      const T kq = mu * gshfl<L>(gm, kv, q), mq = gshfl<L>(gm, mv, q);
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        CV<T, MPL> xv;
        ldv_co<T, MPL>(xv, zc + ((int64_t)B * DIM + c) * ld + koff);
#pragma unroll
        for (int i = 0; i < MPL; ++i) {
          const T cf = kq + cr[i] * mq;
          acc[c].re[i] = fma(cf, xv.re[i], acc[c].re[i]);
          acc[c].im[i] = fma(cf, xv.im[i], acc[c].im[i]);
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < MPL; ++i) {
    const int k = koff + i;
    const T d = coarse_dinv<T>(a, v, k);
    const T al = (T)alpha[k], be = (T)beta[k];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const int64_t f = (v * DIM + c) * ld + k;
      const C rv = ld1co(rc + f), zv = ld1co(zc + f);
      const C zp = prev_zero ? mk<T>(0, 0) : ld1co(zc_prev + f);
      zc_prev[f] = mk<T>(zv.x + al * (zv.x - zp.x) + be * d * (rv.x - acc[c].re[i]),
                         zv.y + al * (zv.y - zp.y) + be * d * (rv.y - acc[c].im[i]));
    }
  }
}

// Row cache of the persistent P1 solves.  A row group owns the same rows in
// every Chebyshev step of a launch, so the first P1_KMAX of them keep their
// nonzeros in shared memory: entry (col, a, b, 0) with the row's two real
// matrices (M_p and L_p, or K_1 and M_1), plus one meta entry per row.  A
// cached step then reads no index or value from L2: it issues the own-row
// loads and the neighbour gathers back to back.  Rows longer than P1_CAP,
// beyond P1_KMAX, or of the FP64 path take the uncached step.
constexpr int P1_CAP = 32, P1_KMAX_P = 3, P1_KMAX_C = 3;
constexpr size_t P1_SMEM_MAX = 48 * 1024;  // dynamic shared memory without an opt-in
// rows cached per group so that the cache of gpb groups fits P1_SMEM_MAX
inline int p1_kmax(int gpb, int kmax) {
  return std::min<int>(kmax, (int)(P1_SMEM_MAX / ((size_t)gpb * (P1_CAP + 1) * sizeof(float4))));
}

template <typename T>
__device__ __forceinline__ void p1_cache_row(const PcArgs &a, const void *va, const void *vb, int64_t v, float4 *ent,
                                             float4 *meta, float m0, float m1, float m2, int lane, int L) {
  const int64_t r0 = a.g_ptr[v], r1 = a.g_ptr[v + 1], s0 = a.s_ptr[v];
  const int n = (int)(r1 - r0);
  const bool fits = n <= P1_CAP;
  if (fits)
    for (int t = lane; t < n; t += L)
      ent[t] = make_float4(__int_as_float(a.s_col[s0 + t]), ((const float *)va)[r0 + t], ((const float *)vb)[r0 + t], 0.f);
  if (lane == 0) *meta = make_float4(m0, m1, m2, __int_as_float(fits ? n : -1));
}

// Cached pressure step on row B (see pressure_row_step): meta = (1/diag M_p,
// 1/diag L_p, outlet flag, length).  DO_M / DO_L select the active
// polynomials (uniform per step), so the gathers of four nonzeros are issued
// together instead of one dependent round trip per nonzero.
template <typename T, int MPL, int DIM, bool DO_M, bool DO_L>
__device__ __forceinline__ void pressure_row_cached(const PcArgs &a, const ChebCoef &cc, const int64_t B,
                                                    const float4 *__restrict__ ent, const float4 mt,
                                                    const typename cpx<T>::t *__restrict__ r,
                                                    const typename cpx<T>::t *__restrict__ zM,
                                                    typename cpx<T>::t *__restrict__ zM_prev,
                                                    const typename cpx<T>::t *__restrict__ zL,
                                                    typename cpx<T>::t *__restrict__ zL_prev, const int lane) {
  const int ld = a.ld, koff = lane * MPL, len = __float_as_int(mt.w);
  const int64_t pf = B * ld + koff;
  CV<T, MPL> aM, aL;
  aM.zero();
  aL.zero();
  int q = 0;
  for (; q + 4 <= len; q += 4) {
    float4 e[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) e[u] = ent[q + u];
    if constexpr (DO_M) {
      CV<T, MPL> x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) ldv_co<T, MPL>(x[u], zM + (int64_t)__float_as_int(e[u].x) * ld + koff);
#pragma unroll
      for (int u = 0; u < 4; ++u) axpy(aM, (T)e[u].y, x[u]);
    }
    if constexpr (DO_L) {
      CV<T, MPL> x[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) ldv_co<T, MPL>(x[u], zL + (int64_t)__float_as_int(e[u].x) * ld + koff);
#pragma unroll
      for (int u = 0; u < 4; ++u) axpy(aL, (T)e[u].z, x[u]);
    }
  }
  for (; q < len; ++q) {
    const float4 e = ent[q];
    const int64_t Bc = __float_as_int(e.x);
    if constexpr (DO_M) { CV<T, MPL> x; ldv_co<T, MPL>(x, zM + Bc * ld + koff); axpy(aM, (T)e.y, x); }
    if constexpr (DO_L) { CV<T, MPL> x; ldv_co<T, MPL>(x, zL + Bc * ld + koff); axpy(aL, (T)e.z, x); }
  }
  CV<T, MPL> rv;
  ldv_co<T, MPL>(rv, r + ((int64_t)DIM * a.N + B) * ld + koff);
  if constexpr (DO_M) {
    CV<T, MPL> z, zp, o;
    ldv_co<T, MPL>(z, zM + pf);
    if (cc.prev_zero_m) zp.zero(); else ldv_co<T, MPL>(zp, zM_prev + pf);
    const T al = (T)cc.alpha_m, be = (T)cc.beta_m, dm = (T)mt.x;
#pragma unroll
    for (int i = 0; i < MPL; ++i) {
      o.re[i] = z.re[i] + al * (z.re[i] - zp.re[i]) + be * dm * (rv.re[i] - aM.re[i]);
      o.im[i] = z.im[i] + al * (z.im[i] - zp.im[i]) + be * dm * (rv.im[i] - aM.im[i]);
    }
    stv<T, MPL>(zM_prev + pf, o);
  }
  if constexpr (DO_L) {
    CV<T, MPL> o;
    const bool out = mt.z != 0.f;
    if (cc.resid_l) {
#pragma unroll
      for (int i = 0; i < MPL; ++i) {
        o.re[i] = out ? T(0) : rv.re[i] - aL.re[i];
        o.im[i] = out ? T(0) : rv.im[i] - aL.im[i];
      }
    } else {
      CV<T, MPL> z, zp;
      ldv_co<T, MPL>(z, zL + pf);
      if (cc.prev_zero_l) zp.zero(); else ldv_co<T, MPL>(zp, zL_prev + pf);
      const T al = (T)cc.alpha_l, be = (T)cc.beta_l, dl = (T)mt.y;
#pragma unroll
      for (int i = 0; i < MPL; ++i) {
        const T rr = out ? T(0) : rv.re[i], ri = out ? T(0) : rv.im[i];
        o.re[i] = z.re[i] + al * (z.re[i] - zp.re[i]) + be * dl * (rr - aL.re[i]);
        o.im[i] = z.im[i] + al * (z.im[i] - zp.im[i]) + be * dl * (ri - aL.im[i]);
      }
    }
    stv<T, MPL>(zL_prev + pf, o);
  }
}

// Cached coarse step on vertex row v (see coarse_row_step): meta = (diag K_1,
// diag M_1, Dirichlet flag, length).  The gathers of two nonzeros (all
// components) are issued together.
template <typename T, int MPL, int DIM>
__device__ __forceinline__ void coarse_row_cached(const PcArgs &a, const double *__restrict__ alpha,
                                                  const double *__restrict__ beta, bool prev_zero,
                                                  const float4 *__restrict__ ent, const float4 mt,
                                                  const typename cpx<T>::t *__restrict__ rc,
                                                  const typename cpx<T>::t *__restrict__ zc,
                                                  typename cpx<T>::t *__restrict__ zc_prev, const int64_t v,
                                                  const int lane) {
  const int ld = a.ld, koff = lane * MPL, len = __float_as_int(mt.w);
  if (mt.z != 0.f) {  // Dirichlet vertex
    CV<T, MPL> zz;
    zz.zero();
#pragma unroll
    for (int c = 0; c < DIM; ++c) stv<T, MPL>(zc_prev + (v * DIM + c) * ld + koff, zz);
    return;
  }
  T cr[MPL];
#pragma unroll
  for (int i = 0; i < MPL; ++i) cr[i] = ((const T *)a.wabs)[koff + i];
  const T mu = (T)a.mu;
  CV<T, MPL> acc[DIM];
#pragma unroll
  for (int c = 0; c < DIM; ++c) acc[c].zero();
  auto fma_row = [&](const float4 e, const CV<T, MPL> *x) {
    const T kq = mu * (T)e.y, mq = (T)e.z;
#pragma unroll
    for (int c = 0; c < DIM; ++c)
#pragma unroll
      for (int i = 0; i < MPL; ++i) {
        const T cf = kq + cr[i] * mq;
        acc[c].re[i] = fma(cf, x[c].re[i], acc[c].re[i]);
        acc[c].im[i] = fma(cf, x[c].im[i], acc[c].im[i]);
      }
  };
  int q = 0;
  for (; q + 2 <= len; q += 2) {
    const float4 e0 = ent[q], e1 = ent[q + 1];
    CV<T, MPL> x0[DIM], x1[DIM];
    const int64_t b0 = (int64_t)__float_as_int(e0.x) * DIM, b1 = (int64_t)__float_as_int(e1.x) * DIM;
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      ldv_co<T, MPL>(x0[c], zc + (b0 + c) * ld + koff);
      ldv_co<T, MPL>(x1[c], zc + (b1 + c) * ld + koff);
    }
    fma_row(e0, x0);
    fma_row(e1, x1);
  }
  if (q < len) {
    const float4 e0 = ent[q];
    CV<T, MPL> x0[DIM];
    const int64_t b0 = (int64_t)__float_as_int(e0.x) * DIM;
#pragma unroll
    for (int c = 0; c < DIM; ++c) ldv_co<T, MPL>(x0[c], zc + (b0 + c) * ld + koff);
    fma_row(e0, x0);
  }
#pragma unroll
  for (int c = 0; c < DIM; ++c) {
    const int64_t f = (v * DIM + c) * ld + koff;
    CV<T, MPL> rv, zv, zp, o;
    ldv_co<T, MPL>(rv, rc + f);
    ldv_co<T, MPL>(zv, zc + f);
    if (prev_zero) zp.zero(); else ldv_co<T, MPL>(zp, zc_prev + f);
#pragma unroll
    for (int i = 0; i < MPL; ++i) {
      const int k = koff + i;
      const T d = T(1) / (mu * (T)mt.x + cr[i] * (T)mt.y);
      const T al = (T)alpha[k], be = (T)beta[k];
      o.re[i] = zv.re[i] + al * (zv.re[i] - zp.re[i]) + be * d * (rv.re[i] - acc[c].re[i]);
      o.im[i] = zv.im[i] + al * (zv.im[i] - zp.im[i]) + be * d * (rv.im[i] - acc[c].im[i]);
    }
    stv<T, MPL>(zc_prev + f, o);
  }
}

// Coarse (P1) velocity solve of the two-level cycle as one cooperative launch:
// restriction rc = P^T rr, step 0 zc = rc / (diag A_c theta_c[k]) and s_c - 1
// Chebyshev steps, with a bounded grid barrier between the stages (a barrier
// that gives up sets the context's error word and every block returns).  The
// result is in zc[(s_c - 1) % 2].
template <typename T> struct CoarseArgs {
  const typename cpx<T>::t *rr;  // fine velocity residual [N][dim][ld]
  typename cpx<T>::t *rc;        // coarse right-hand side [P][dim][ld]
  typename cpx<T>::t *zc0, *zc1;
  const double *inv_theta, *alpha, *beta;  // [ld], [s_c][ld], [s_c][ld]
  int s_c;
  int kmax;  // rows cached per row group (the dynamic shared memory holds gpb * kmax rows)
  GridSync *gs;
};

template <typename T, int MPL, int L, int DIM>
__global__ void __launch_bounds__(256, 3) k_coarse_solve(const PcArgs a, const CoarseArgs<T> q) {
  const int64_t nc = a.P * DIM * a.ld;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t f = tid; f < nc; f += nth) restrict_elem<T>(a, DIM, q.rr, q.rc, f);
  if (!grid_sync(q.gs, gridDim.x)) return;
  for (int64_t f = tid; f < nc; f += nth) {
    const int64_t v = f / ((int64_t)DIM * a.ld);
    const int k = (int)(f % a.ld);
    if (row_idle(a.dof_comp, a.comp_active, v * DIM)) continue;
    const T sc = a.dirmask[v] ? T(0) : coarse_dinv<T>(a, v, k) * (T)q.inv_theta[k];
    const auto r = ld1co(q.rc + f);
    q.zc0[f] = mk<T>(sc * r.x, sc * r.y);
  }
  const int gpb = blockDim.x / L;
  const int lane = threadIdx.x % L, group = threadIdx.x / L;
  const unsigned gm = group_mask<L>();
  const int64_t G = (int64_t)gridDim.x * gpb, g = (int64_t)blockIdx.x * gpb + group;
  extern __shared__ float4 p1_smem[];
  const int kmax = sizeof(T) == 4 ? q.kmax : 0;
  float4 *ent = p1_smem + (size_t)group * kmax * P1_CAP;
  float4 *meta = p1_smem + (size_t)gpb * kmax * P1_CAP + group * kmax;
  if constexpr (sizeof(T) == 4) {
    for (int kk = 0; kk < kmax; ++kk) {
      const int64_t v = g + kk * G;
      if (v < a.P)
        p1_cache_row<T>(a, a.Kcv, a.Mcv, v, ent + kk * P1_CAP, meta + kk, ((const float *)a.k1d)[v],
                        ((const float *)a.mpd)[v], a.dirmask[v] ? 1.f : 0.f, lane, L);
    }
  }
  if (!grid_sync(q.gs, gridDim.x)) return;  // also orders the cache fill before its use
  typename cpx<T>::t *zcur = q.zc0, *znext = q.zc1;
  for (int i = 1; i < q.s_c; ++i) {
    int kk = 0;
    for (int64_t v = g; v < a.P; v += G, ++kk) {
      if (row_idle(a.dof_comp, a.comp_active, v * DIM)) continue;
      if (kk < kmax) {
        const float4 mt = meta[kk];
        if (__float_as_int(mt.w) >= 0) {
          coarse_row_cached<T, MPL, DIM>(a, q.alpha + (size_t)i * a.ld, q.beta + (size_t)i * a.ld, i == 1,
                                         ent + kk * P1_CAP, mt, q.rc, zcur, znext, v, lane);
          continue;
        }
      }
      coarse_row_step<T, MPL, L, DIM>(a, q.alpha + (size_t)i * a.ld, q.beta + (size_t)i * a.ld, i == 1, q.rc, zcur,
                                      znext, v, lane, gm);
    }
    typename cpx<T>::t *tmp = zcur;
    zcur = znext;
    znext = tmp;
    if (!grid_sync(q.gs, gridDim.x)) return;
  }
}

// Pressure block as one cooperative launch: step 0 of the P1 mass and P1
// Laplacian polynomials (r_p first scaled in place by rscale, if given), their
// Chebyshev steps with a bounded grid barrier between steps, and
// z_p = sign (mu zM + j omega rho zL) written to the pressure rows of z.
//
// With lap_s > 0 the Laplacian part is the symmetric two-level cycle
//   x1 = S r,  x2 = x1 + R A_c^-1 R^T (r - L_p x1),  x3 = x2 + S (r - L_p x2),
// S the lap_s-step Chebyshev-Jacobi polynomial (al, bl, inv_theta_l), R the
// indicator of the vertex aggregates (0 on the outlet) and A_c^-1 the inverse
// Galerkin matrix R^T L_p R of every block: the residual pass, the restriction
// (one thread block per aggregate, FP64 sums in a fixed order), the coarse
// product and the prolongation each end at a grid barrier; the post-smoother
// repeats the recurrence from x2 (its first step has alpha = 0).
template <typename T> struct PressureArgs {
  typename cpx<T>::t *r;   // the full block; only its pressure rows are read (and scaled)
  const double *rscale;    // [n_comp][ld] or null
  double inv_theta_m, inv_theta_l;
  const double *am, *bm, *al, *bl;  // recurrences, [s_m], [s_l]
  int s_m, s_l;
  typename cpx<T>::t *zM0, *zM1, *zL0, *zL1;
  typename cpx<T>::t *z;
  T sign;
  int kmax;  // rows cached per row group (the dynamic shared memory holds gpb * kmax rows)
  GridSync *gs;
  // two-level Laplacian (lap_s > 0; then s_l == lap_s)
  int lap_s, n_lagg;
  const int32_t *lagg, *lagg_vert, *lagg_blk, *lagg_loc, *lblk_na, *lblk_a0;
  const int64_t *lagg_ptr, *lblk_so;
  const T *linv;
  typename cpx<T>::t *q, *y;  // [n_lagg][ld] scratch
};

template <typename T, int MPL, int L, int DIM>
__global__ void __launch_bounds__(256, 3) k_pressure_solve(const PcArgs a, const PressureArgs<T> p) {
  using C = typename cpx<T>::t;
  const int ld = a.ld;
  const int64_t np = a.P * ld, fp = (int64_t)DIM * a.N * ld;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  for (int64_t e = tid; e < np; e += nth) {
    const int64_t B = e / ld, dof = (int64_t)DIM * a.N + B;
    const int k = (int)(e % ld);
    if (row_idle(a.dof_comp, a.comp_active, dof)) continue;
    C v = p.r[fp + e];
    if (p.rscale) {
      const T sc = (T)p.rscale[(a.dof_comp ? (int64_t)a.dof_comp[dof] * ld : 0) + k];
      v.x *= sc; v.y *= sc;
      p.r[fp + e] = v;
    }
    const T sm = (T)p.inv_theta_m / ((const T *)a.mpd)[B];
    p.zM0[e] = mk<T>(v.x * sm, v.y * sm);
    const T sl = a.outmask[B] ? T(0) : (T)p.inv_theta_l / ((const T *)a.lpd)[B];
    p.zL0[e] = mk<T>(v.x * sl, v.y * sl);
  }
  const int gpb = blockDim.x / L;
  const int lane = threadIdx.x % L, group = threadIdx.x / L;
  const unsigned gm = group_mask<L>();
  const int64_t G = (int64_t)gridDim.x * gpb, g = (int64_t)blockIdx.x * gpb + group;
  extern __shared__ float4 p1_smem[];
  const int kmax = sizeof(T) == 4 ? p.kmax : 0;
  float4 *ent = p1_smem + (size_t)group * kmax * P1_CAP;
  float4 *meta = p1_smem + (size_t)gpb * kmax * P1_CAP + group * kmax;
  if constexpr (sizeof(T) == 4) {
    for (int kk = 0; kk < kmax; ++kk) {
      const int64_t B = g + kk * G;
      if (B < a.P)
        p1_cache_row<T>(a, a.Mpv, a.Lpv, B, ent + kk * P1_CAP, meta + kk, 1.f / ((const float *)a.mpd)[B],
                        1.f / ((const float *)a.lpd)[B], a.outmask[B] ? 1.f : 0.f, lane, L);
    }
  }
  if (!grid_sync(p.gs, gridDim.x)) return;  // also orders the cache fill before its use
  C *mc = p.zM0, *mn = p.zM1, *lc = p.zL0, *ln = p.zL1;  // current / next iterates
  // one pass over the pressure rows of this group: the steps cc selects
  auto pass = [&](const ChebCoef &cc) {
    int kk = 0;
    for (int64_t B = g; B < a.P; B += G, ++kk) {
      if (row_idle(a.dof_comp, a.comp_active, (int64_t)DIM * a.N + B)) continue;
      if (kk < kmax) {
        const float4 mt = meta[kk];
        if (__float_as_int(mt.w) >= 0) {
          if (cc.do_m && cc.do_l)
            pressure_row_cached<T, MPL, DIM, true, true>(a, cc, B, ent + kk * P1_CAP, mt, p.r, mc, mn, lc, ln, lane);
          else if (cc.do_l)
            pressure_row_cached<T, MPL, DIM, false, true>(a, cc, B, ent + kk * P1_CAP, mt, p.r, mc, mn, lc, ln, lane);
          else
            pressure_row_cached<T, MPL, DIM, true, false>(a, cc, B, ent + kk * P1_CAP, mt, p.r, mc, mn, lc, ln, lane);
          continue;
        }
      }
      pressure_row_step<T, MPL, L, DIM>(a, cc, B, p.r, mc, mn, lc, ln, lane, gm);
    }
  };
  // steps 1 .. s_pre-1 of the polynomials; with the two-level Laplacian then the
  // residual pass (step s_pre), the coarse correction and lap_s post-smoothing steps
  const int s_pre = max(p.s_m, p.s_l), n_steps = s_pre + (p.lap_s > 0 ? p.lap_s + 1 : 0);
  for (int st = 1; st < n_steps; ++st) {
    ChebCoef cc{};
    if (st < s_pre) {
      cc.do_m = st < p.s_m;
      cc.do_l = st < p.s_l;
      cc.alpha_m = cc.do_m ? p.am[st] : 0.0; cc.beta_m = cc.do_m ? p.bm[st] : 0.0;
      cc.alpha_l = cc.do_l ? p.al[st] : 0.0; cc.beta_l = cc.do_l ? p.bl[st] : 0.0;
      cc.prev_zero_m = cc.prev_zero_l = (st == 1);
    } else if (st == s_pre) {
      cc.do_l = 1;
      cc.resid_l = 1;  // r - L_p x1 into ln
    } else {           // the same recurrence started from x2: its first step has alpha = 0
      const int ip = st - s_pre - 1;
      cc.do_l = 1;
      cc.alpha_l = ip ? p.al[ip] : 0.0;
      cc.beta_l = ip ? p.bl[ip] : p.inv_theta_l;
      cc.prev_zero_l = (ip == 0);
    }
    pass(cc);
    if (cc.do_m) { C *t = mc; mc = mn; mn = t; }
    if (cc.do_l && !cc.resid_l) { C *t = lc; lc = ln; ln = t; }
    if (!grid_sync(p.gs, gridDim.x)) return;
    if (st != s_pre || p.lap_s == 0) continue;
    // restriction q[a][k] = sum over the aggregate's vertices (ascending) of the residual
    __shared__ double2 part[256];
    {
      const int k = threadIdx.x % ld, ch = threadIdx.x / ld, nch = blockDim.x / ld;
      for (int ag = blockIdx.x; ag < p.n_lagg; ag += gridDim.x) {
        double sx = 0, sy = 0;
        for (int64_t i = p.lagg_ptr[ag] + ch; i < p.lagg_ptr[ag + 1]; i += nch) {
          const int64_t v = p.lagg_vert[i];
          if (row_idle(a.dof_comp, a.comp_active, (int64_t)DIM * a.N + v)) continue;
          const C rv = ld1co(ln + v * ld + k);
          sx += (double)rv.x;
          sy += (double)rv.y;
        }
        part[threadIdx.x] = make_double2(sx, sy);
        __syncthreads();
        for (int h = nch / 2; h > 0; h >>= 1) {
          if (ch < h) {
            const double2 o = part[threadIdx.x + h * ld];
            part[threadIdx.x].x += o.x;
            part[threadIdx.x].y += o.y;
          }
          __syncthreads();
        }
        if (ch == 0) p.q[(int64_t)ag * ld + k] = mk<T>((T)part[k].x, (T)part[k].y);
        __syncthreads();  // part is reused by the block's next aggregate
      }
    }
    if (!grid_sync(p.gs, gridDim.x)) return;
    // coarse solve y = A_c^-1 q of every block, one thread per (aggregate, mode)
    for (int64_t f = tid; f < (int64_t)p.n_lagg * ld; f += nth) {
      const int ag = (int)(f / ld), k = (int)(f % ld);
      const int b = p.lagg_blk[ag], n = p.lblk_na[b];
      const T *row = p.linv + p.lblk_so[b] + (int64_t)p.lagg_loc[ag] * n;
      const C *qb = p.q + (int64_t)p.lblk_a0[b] * ld + k;
      T sx = 0, sy = 0;
      for (int j = 0; j < n; ++j) {
        const T w = row[j];
        const C v = ld1co(qb + (int64_t)j * ld);
        sx = fma(w, v.x, sx);
        sy = fma(w, v.y, sy);
      }
      p.y[f] = mk<T>(sx, sy);
    }
    if (!grid_sync(p.gs, gridDim.x)) return;
    // prolongation x2 = x1 + R y
    for (int64_t e = tid; e < np; e += nth) {
      const int64_t B = e / ld;
      const int ag = p.lagg[B];
      if (ag < 0 || row_idle(a.dof_comp, a.comp_active, (int64_t)DIM * a.N + B)) continue;
      const C add = ld1co(p.y + (int64_t)ag * ld + e % ld);
      C o = ld1co(lc + e);
      o.x += add.x;
      o.y += add.y;
      lc[e] = o;
    }
    if (!grid_sync(p.gs, gridDim.x)) return;
  }
  const T mu = p.sign * (T)a.mu;
  for (int64_t e = tid; e < np; e += nth) {
    const int k = (int)(e % ld);
    if (row_idle(a.dof_comp, a.comp_active, (int64_t)DIM * a.N + e / ld)) continue;
    const T wr = p.sign * ((const T *)a.wrho)[k];
    const C m_ = ld1co(mc + e), l_ = ld1co(lc + e);
    p.z[fp + e] = mk<T>(mu * m_.x - wr * l_.y, mu * m_.y + wr * l_.x);
  }
}

// Block upper-triangular form, start of the velocity solve: normalise the
// Krylov vector's velocity rows in place (rscale, may be null), form the
// right-hand side of the velocity block rt = r_u - D z_p (D z_p gathered over
// the G row, whose columns are vertices; Dirichlet rows keep r_u) and write the
// first Chebyshev iterate z_u = rt / (diag A_r theta_u[k]).
template <typename T, int MPL, int L, int DIM>
__global__ void __launch_bounds__(256)
k_tri_vel0(const PcArgs a, typename cpx<T>::t *__restrict__ r, const double *__restrict__ rscale,
           const double *__restrict__ inv_theta_u, const typename cpx<T>::t *__restrict__ zp,
           typename cpx<T>::t *__restrict__ rt, typename cpx<T>::t *__restrict__ zu) {
  const int gpb = blockDim.x / L;
  const int lane = threadIdx.x % L, group = threadIdx.x / L;
  const unsigned gm = group_mask<L>();
  const int ld = a.ld, koff = lane * MPL;
  const T *Dv = (const T *)a.Dv;
  SCVS_ROW_LOOP(A, 0, a.N, gpb, group, a.tile) {
    if (row_idle(a.dof_comp, a.comp_active, A * DIM)) continue;
    CV<T, MPL> rv[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) ldv<T, MPL>(rv[c], r + (A * DIM + c) * ld + koff);
    if (rscale) {
      const double *rs = rscale + (a.dof_comp ? (int64_t)a.dof_comp[A * DIM] * ld : 0) + koff;
#pragma unroll
      for (int i = 0; i < MPL; ++i) {
        const T sc = (T)rs[i];
#pragma unroll
        for (int c = 0; c < DIM; ++c) { rv[c].re[i] *= sc; rv[c].im[i] *= sc; }
      }
#pragma unroll
      for (int c = 0; c < DIM; ++c) stv<T, MPL>(r + (A * DIM + c) * ld + koff, rv[c]);
    }
    if (a.dirmask[A]) {
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        stv<T, MPL>(rt + (A * DIM + c) * ld + koff, rv[c]);
        stv<T, MPL>(zu + (A * DIM + c) * ld + koff, rv[c]);
      }
      continue;
    }
    const int64_t s0 = a.s_ptr[A], g1 = s0 + a.g_len[A], goff = a.g_ptr[A] - s0;
    for (int64_t base = s0; base < g1; base += L) {
      const int64_t t = base + lane;
      int32_t col = 0;
      T dv[DIM];
#pragma unroll
      for (int c = 0; c < DIM; ++c) dv[c] = 0;
      if (t < g1) {
        col = __ldg(a.s_col + t);
#pragma unroll
        for (int c = 0; c < DIM; ++c) dv[c] = __ldg(Dv + c * a.g_nnz + t + goff);
      }
      const int cnt = (int)min((int64_t)L, g1 - base);
#pragma unroll 4
      for (int q = 0; q < cnt; ++q) {
        const int32_t B = gshfl<L>(gm, col, q);
        CV<T, MPL> xq;
        ldv<T, MPL>(xq, zp + (int64_t)B * ld + koff);
#pragma unroll
        for (int c = 0; c < DIM; ++c) axpy(rv[c], -gshfl<L>(gm, dv[c], q), xq);
      }
    }
    T sd[MPL];
#pragma unroll
    for (int i = 0; i < MPL; ++i) sd[i] = vel_dinv<T>(a, A, koff + i) * (T)inv_theta_u[koff + i];
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      CV<T, MPL> o;
#pragma unroll
      for (int i = 0; i < MPL; ++i) { o.re[i] = sd[i] * rv[c].re[i]; o.im[i] = sd[i] * rv[c].im[i]; }
      stv<T, MPL>(rt + (A * DIM + c) * ld + koff, rv[c]);
      stv<T, MPL>(zu + (A * DIM + c) * ld + koff, o);
    }
  }
}

// Chebyshev recurrence coefficients for the interval [lo, hi] (Saad, Iterative
// Methods for Sparse Linear Systems, Alg. 12.1): theta = (hi+lo)/2,
// delta = (hi-lo)/2, sigma = theta/delta, rho_0 = 1/sigma,
// rho_i = 1/(2 sigma - rho_{i-1}), alpha_i = rho_i rho_{i-1}, beta_i = 2 rho_i/delta.
struct ChebSeq {
  double inv_theta;
  std::vector<double> alpha, beta;
};
static ChebSeq cheb_seq(double lo, double hi, int s) {
  ChebSeq q;
  double th = 0.5 * (hi + lo), de = 0.5 * (hi - lo), sg = th / de;
  q.inv_theta = 1.0 / th;
  double rho_prev = 1.0 / sg;
  q.alpha.assign(std::max(s, 1), 0.0);
  q.beta.assign(std::max(s, 1), 0.0);
  for (int i = 1; i < s; ++i) {
    double rho = 1.0 / (2.0 * sg - rho_prev);
    q.alpha[i] = rho * rho_prev;
    q.beta[i] = 2.0 * rho / de;
    rho_prev = rho;
  }
  return q;
}

// Interval ratios lambda_max / lambda_low of the Chebyshev polynomials:
// velocity polynomial used alone (BLOCK_CHEB), velocity smoother of the
// two-level cycle (damps the upper part of the spectrum only), coarse
// velocity level (a degree-30 polynomial on [lambda/30, lambda] beat wider
// intervals for every mode on the benchmark pipe, the steady mode included),
// P1 mass and P1 Laplacian.
constexpr double CHEB_RATIO_U = 30.0, CHEB_RATIO_SMOOTH = 12.0, CHEB_RATIO_C = 30.0, CHEB_RATIO_M = 6.0,
                 CHEB_RATIO_L = 3000.0, CHEB_TOP = 1.10;
// Smoother of the two-level pressure Laplacian: damps [lambda/120, 1.1 lambda]
// and leaves the smooth end to the coarse level (on the benchmark pipe a wider
// interval than a plain smoother's beat [lambda/30] and [lambda/60]).
constexpr double CHEB_RATIO_LAP = 120.0;

static void lap_build(Ctx &c, Mesh &m, int size);
static int lap_size_of(const Ctx &c) { return c.opts.lap_size > 0 ? c.opts.lap_size : LAP_DEFAULT_SIZE; }
// Smoothing degree of the two-level pressure Laplacian of a mesh, 0 where the
// plain polynomial is used (option off, or no coarse level on this mesh).
static int lap_smooth_of(Ctx &c, Mesh &m) {
  if (c.opts.lap_size < 0) return 0;
  const int size = lap_size_of(c);
  if (m.lap.target != size) lap_build(c, m, size);
  return m.lap.on ? (c.opts.lap_smooth > 0 ? c.opts.lap_smooth : LAP_DEFAULT_SMOOTH) : 0;
}

template <typename T>
PcArgs pc_args(const Mesh &m) {
  const bool f = sizeof(T) == 4;
  return PcArgs{m.N, m.P, m.ld, m.s_ptr, m.s_col, m.g_len, m.g_ptr,
                f ? (const void *)m.Ks_f : (const void *)m.Ks_m, f ? (const void *)m.Ms_f : (const void *)m.Ms_m,
                f ? (const void *)m.Mp_f : (const void *)m.Mp, f ? (const void *)m.Lp_f : (const void *)m.Lp_m,
                m.ms_diag, m.ks_diag, m.mp_diag, m.lp_diag, m.dirmask, m.outmask, m.omega_d, m.rho, m.mu,
                f ? (const void *)m.Kc_f : (const void *)m.Kc_m, f ? (const void *)m.Mc_f : (const void *)m.Mc_m,
                m.k1_diag, m.edge_ends, m.v2e_ptr, m.v2e,
                f ? (const void *)m.ks_df : (const void *)m.ks_diag, f ? (const void *)m.ms_df : (const void *)m.ms_diag,
                f ? (const void *)m.mp_df : (const void *)m.mp_diag, f ? (const void *)m.lp_df : (const void *)m.lp_diag,
                f ? (const void *)m.k1_df : (const void *)m.k1_diag,
                f ? (const void *)m.wabs_f : (const void *)m.wabs_d, f ? (const void *)m.wrho_f : (const void *)m.wrho_d,
                m.dof_comp, m.comp_active, m.tile_cheb ? m.tile_cheb : SCVS_DEFAULT_TILE,
                f ? (const void *)m.Dv_f : (const void *)m.Dv_m, m.g_nnz};
}

// Per-mode Chebyshev sequences on [lam_k / ratio, 1.05 lam_k] uploaded as
// inv_theta[ld], alpha[s][ld], beta[s][ld].
static void per_mode_seq(Ctx &c, Mesh &m, const std::vector<double> &lam, double ratio, int s, double **inv_theta,
                         double **alpha, double **beta) {
  std::vector<double> th(m.ld), al((size_t)s * m.ld), be((size_t)s * m.ld);
  for (int k = 0; k < m.ld; ++k) {
    const double l = lam[k] > 0 ? lam[k] : 2.0;
    ChebSeq q = cheb_seq(l / ratio, CHEB_TOP * l, s);
    th[k] = q.inv_theta;
    for (int i = 0; i < s; ++i) { al[(size_t)i * m.ld + k] = q.alpha[i]; be[(size_t)i * m.ld + k] = q.beta[i]; }
  }
  *inv_theta = m.mode_arena.alloc<double>(m.ld);
  *alpha = m.mode_arena.alloc<double>(al.size());
  *beta = m.mode_arena.alloc<double>(be.size());
  SCVS_CUDA(cudaMemcpyAsync(*inv_theta, th.data(), th.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  SCVS_CUDA(cudaMemcpyAsync(*alpha, al.data(), al.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  SCVS_CUDA(cudaMemcpyAsync(*beta, be.data(), be.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
}

// The preconditioner kind of a mesh: SCVS_PC_AUTO resolves to the triangular
// form with the coarse Schur correction (with 16 aggregates per component it
// was the fastest kind on every workload measured, the single 151k-node pipe
// included).
int pc_kind(const Ctx &c, const Mesh &m) {
  (void)m;
  if (c.opts.precond != SCVS_PC_AUTO) return c.opts.precond;
  return SCVS_PC_TRI_PMG_CS;
}

static void pc_tables(Ctx &c, Mesh &m, PcTables &t) {
  const int su = std::max(1, c.opts.cheb_u), sm = std::max(1, c.opts.cheb_m), sl = std::max(1, c.opts.cheb_l);
  const int sc = std::max(1, c.opts.cheb_c), kind = pc_kind(c, m);
  const int lap = lap_smooth_of(c, m), sl_eff = lap ? lap : sl;
  if (t.valid && t.s_u == su && t.s_m == sm && t.s_l == sl_eff && t.lap_s == lap && t.s_c == sc && t.kind == kind)
    return;
  t.s_u = su; t.s_m = sm; t.s_l = sl_eff; t.lap_s = lap; t.s_c = sc; t.kind = kind;
  t.cs_bytes = 0;  // the coarse Schur matrices depend on the velocity cycle
  const bool pmg = kind == SCVS_PC_BLOCK_PMG || kind == SCVS_PC_TRI_PMG || kind == SCVS_PC_TRI_PMG_CS;
  per_mode_seq(c, m, m.lam_u, pmg ? CHEB_RATIO_SMOOTH : CHEB_RATIO_U, su, &t.inv_theta_u, &t.alpha_u, &t.beta_u);
  if (pmg) per_mode_seq(c, m, m.lam_c, CHEB_RATIO_C, sc, &t.inv_theta_c, &t.alpha_c, &t.beta_c);
  t.zeros = m.mode_arena.alloc<double>(m.ld);
  SCVS_CUDA(cudaMemsetAsync(t.zeros, 0, m.ld * sizeof(double), c.stream));
  ChebSeq qm = cheb_seq(m.lam_m / CHEB_RATIO_M, CHEB_TOP * m.lam_m, sm);
  ChebSeq ql = lap ? cheb_seq(m.lam_l / CHEB_RATIO_LAP, CHEB_TOP * m.lam_l, lap)
                  : cheb_seq(m.lam_l / CHEB_RATIO_L, CHEB_TOP * m.lam_l, sl);
  t.inv_theta_m = qm.inv_theta; t.am = qm.alpha; t.bm = qm.beta;
  t.inv_theta_l = ql.inv_theta; t.al = ql.alpha; t.bl = ql.beta;
  double **dst[4] = {&t.am_d, &t.bm_d, &t.al_d, &t.bl_d};
  const std::vector<double> *src[4] = {&t.am, &t.bm, &t.al, &t.bl};
  for (int i = 0; i < 4; ++i) {
    *dst[i] = m.mode_arena.alloc<double>(src[i]->size());
    SCVS_CUDA(cudaMemcpyAsync(*dst[i], src[i]->data(), src[i]->size() * sizeof(double), cudaMemcpyHostToDevice,
                              c.stream));
  }
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  t.valid = true;
}

// velocity iterate, pressure polynomials (2 x 2 P), coarse level (3 dim P), and
// the velocity right-hand side of the block-triangular form (dim N)
int64_t precond_scratch_elems(const Mesh &m) {
  return (m.n_dof + (4 + 3 * (int64_t)m.dim) * m.P + (int64_t)m.dim * m.N) * m.ld;
}

// One Chebyshev step launch over the velocity rows.
template <typename T>
static void cheb_launch(Ctx &c, const Mesh &m, const PcArgs &a, const ChebCoef &cc, const typename cpx<T>::t *r,
                        const typename cpx<T>::t *ucur, typename cpx<T>::t *uprev) {
  const double cs = 2.0 * sizeof(T), vb = (double)m.dim * m.N * m.ld * cs;
  KScope ksc(c, KC_CHEB_FINE,
             (double)m.s_nnz * (4 + 2 * sizeof(T)) + (double)(m.N + 1) * 8 + m.N + vb * (cc.prev_zero_u ? 3 : 4));
  if constexpr (sizeof(T) == 4) {
    if (m.st_cheb && staged_ok(c, m, m.st_cheb, false, ucur)) {
      launch_cheb_staged(c, m, a, cc, r, ucur, uprev, m.st_cheb);
      return;
    }
  }
  auto body = [&](auto mpl_c, auto l_c) {
    constexpr int MPL = decltype(mpl_c)::value, L = decltype(l_c)::value;
    const int gpb = 256 / L;
    const unsigned nb = row_blocks(c, m.N, gpb, a.tile);
    if (m.dim == 2)
      k_pc_cheb<T, MPL, L, 2><<<nb, 256, 0, c.stream>>>(a, cc, r, ucur, uprev);
    else
      k_pc_cheb<T, MPL, L, 3><<<nb, 256, 0, c.stream>>>(a, cc, r, ucur, uprev);
  };
  if constexpr (sizeof(T) == 4) {
    const int mpl = m.mpl_cheb ? m.mpl_cheb : default_mpl<T>(m.ld);
    SCVS_DISPATCH_SHAPE(m.ld, mpl, body(std::integral_constant<int, MPL>{}, std::integral_constant<int, L>{}));
  } else {
    SCVS_DISPATCH_LD(T, m.ld, body(std::integral_constant<int, MPL>{}, std::integral_constant<int, L>{}));
  }
  count_launch(c);
}

// Grid of a cooperative launch: every block resident at once (at most 4 per
// SM, which keeps the barrier's arrival counter short).
static int coop_grid(Ctx &c, const void *kfn, size_t smem) {
  int per_sm = 0;
  SCVS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, 256, smem));
  if (per_sm < 1) throw (int)SCVS_ERR_CUDA;
  return std::min(per_sm, 4) * c.num_sms;
}

template <typename T>
static void pressure_solve(Ctx &c, const Mesh &m, const PcArgs &a, const PcTables &t, typename cpx<T>::t *r,
                           const double *rscale, typename cpx<T>::t *const *pM, typename cpx<T>::t *const *pL,
                           typename cpx<T>::t *z, T sign, typename cpx<T>::t *lq, typename cpx<T>::t *ly) {
  const double cs = 2.0 * sizeof(T), pb = (double)m.P * m.ld * cs;
  double by = pb * (rscale ? 4 : 3) + (double)m.P * 2 * sizeof(T) + 3 * pb;  // step 0 and the combination
  const double lstep = (double)m.q_nnz * (4 + sizeof(T)) + (double)(m.P + 1) * 8;  // one pass over the L_p rows
  for (int ip = 1; ip < std::max(t.s_m, t.s_l); ++ip) {
    const int np = (ip < t.s_m) + (ip < t.s_l);
    by += (double)m.q_nnz * (4 + np * sizeof(T)) + (double)(m.P + 1) * 8 + pb + np * pb * (ip == 1 ? 2 : 3);
  }
  const LapCoarse &lap = m.lap;
  if (t.lap_s > 0) {
    const double qb = (double)lap.n_agg * m.ld * cs;
    by += lstep + 2 * pb;                                                   // residual
    by += pb + (double)m.P * 4 + (double)(lap.n_agg + 1) * 8 + qb;            // restriction
    by += (double)lap.so_total * sizeof(T) + (double)lap.n_agg * 12 + 2 * qb;  // coarse product (each row once)
    by += 2 * pb + (double)m.P * 4 + qb;                                    // prolongation
    by += t.lap_s * (lstep + 3 * pb) + pb;                                  // post-smoothing
  }
  KScope ks(c, KC_PRESSURE, by);
  PressureArgs<T> p{r, rscale, t.inv_theta_m, t.inv_theta_l, t.am_d, t.bm_d, t.al_d, t.bl_d, t.s_m, t.s_l,
                    pM[0], pM[1], pL[0], pL[1], z, sign, 0, c.gsync};
  if (t.lap_s > 0) {
    p.lap_s = t.lap_s;
    p.n_lagg = lap.n_agg;
    p.lagg = lap.agg; p.lagg_vert = lap.agg_vert; p.lagg_blk = lap.agg_blk; p.lagg_loc = lap.agg_loc;
    p.lblk_na = lap.blk_na; p.lblk_a0 = lap.blk_a0; p.lagg_ptr = lap.agg_ptr; p.lblk_so = lap.blk_so;
    p.linv = sizeof(T) == 4 ? (const T *)(const void *)lap.inv_f : (const T *)(const void *)lap.inv_d;
    p.q = lq;
    p.y = ly;
  }
  PcArgs aa = a;
  SCVS_DISPATCH_LD(T, m.ld, {
    const void *kfn = m.dim == 2 ? (const void *)k_pressure_solve<T, MPL, L, 2> : (const void *)k_pressure_solve<T, MPL, L, 3>;
    p.kmax = sizeof(T) == 4 ? p1_kmax(256 / L, P1_KMAX_P) : 0;
    const size_t smem = (size_t)(256 / L) * p.kmax * (P1_CAP + 1) * sizeof(float4);
    void *args[] = {(void *)&aa, (void *)&p};
    SCVS_CUDA(cudaLaunchCooperativeKernel(kfn, dim3(coop_grid(c, kfn, smem)), dim3(256), args, smem, c.stream));
  });
  count_launch(c);
}

// Returns the coarse buffer that holds the result.
template <typename T>
static typename cpx<T>::t *coarse_solve(Ctx &c, const Mesh &m, const PcArgs &a, const PcTables &t,
                                        const typename cpx<T>::t *rr, typename cpx<T>::t *rc,
                                        typename cpx<T>::t *const *zc) {
  const double cs = 2.0 * sizeof(T), cbk = (double)m.dim * m.P * m.ld * cs;
  double by = (double)m.dim * m.N * m.ld * cs + (double)(m.P + 1) * 8 + (double)(m.N - m.P) * 4 + cbk  // restriction
              + 2 * cbk + (double)m.P * 2 * sizeof(T);                                                  // step 0
  for (int i = 1; i < t.s_c; ++i)
    by += (double)m.q_nnz * (4 + 2 * sizeof(T)) + (double)(m.P + 1) * 8 + cbk * (i == 1 ? 3 : 4);
  KScope ks(c, KC_COARSE, by);
  CoarseArgs<T> q{rr, rc, zc[0], zc[1], t.inv_theta_c, t.alpha_c, t.beta_c, t.s_c, 0, c.gsync};
  PcArgs aa = a;
  SCVS_DISPATCH_LD(T, m.ld, {
    const void *kfn = m.dim == 2 ? (const void *)k_coarse_solve<T, MPL, L, 2> : (const void *)k_coarse_solve<T, MPL, L, 3>;
    q.kmax = sizeof(T) == 4 ? p1_kmax(256 / L, P1_KMAX_C) : 0;
    const size_t smem = (size_t)(256 / L) * q.kmax * (P1_CAP + 1) * sizeof(float4);
    void *args[] = {(void *)&aa, (void *)&q};
    SCVS_CUDA(cudaLaunchCooperativeKernel(kfn, dim3(coop_grid(c, kfn, smem)), dim3(256), args, smem, c.stream));
  });
  count_launch(c);
  return zc[(t.s_c - 1) % 2];
}

// ---------------------------------------- coarse Schur correction
// Additive two-level approximation of the inverse Schur complement (the
// triangular form's pressure block): on top of the Cahouet-Chabard term, a
// Galerkin coarse term R_c (R_c^T D^T A~_u^-1 D R_c)^-1 R_c^T with R_c the
// piecewise-constant functions of graph aggregates of the vertices and A~_u^-1
// the preconditioner's own velocity cycle.  The coarse space restores the
// smooth, domain-long pressure modes that the mass/Laplacian combination
// misses on elongated domains (the discrete inf-sup constant shrinks with the
// aspect ratio).  The velocity cycle applies the real shift
// mu K_s + |omega| rho M_s with real coefficients, so it is real-linear and
// the coarse matrices are real; a complex lane carries two coarse columns.

constexpr int CS_NA_MAX = 1024;  // aggregates of one block at most
constexpr int CS_DEFAULT_AGG = 16;

// q[a][k] = sum of r_p[v][k] over the vertices v of aggregate a.  One block of
// AGG_RT threads per aggregate (a few large aggregates: the whole block's width
// keeps loads in flight); thread (chunk, k) sums every (AGG_RT/ld)-th vertex
// in ascending order in FP64, and the chunk partials are added in a fixed
// tree order.
constexpr int AGG_RT = 1024;
template <typename T>
__global__ void __launch_bounds__(AGG_RT) k_agg_restrict(const int64_t *__restrict__ agg_ptr,
                                                         const int32_t *__restrict__ agg_vert, int ld,
                                                         const typename cpx<T>::t *__restrict__ rp,
                                                         typename cpx<T>::t *__restrict__ q) {
  __shared__ double2 part[AGG_RT];
  const int a = blockIdx.x;
  const int k = threadIdx.x % ld, ch = threadIdx.x / ld, nch = blockDim.x / ld;
  const int64_t v0 = agg_ptr[a], v1 = agg_ptr[a + 1];
  double sx = 0, sy = 0;
  for (int64_t i = v0 + ch; i < v1; i += nch) {
    const typename cpx<T>::t v = rp[(int64_t)agg_vert[i] * ld + k];
    sx += (double)v.x;
    sy += (double)v.y;
  }
  part[threadIdx.x] = make_double2(sx, sy);
  __syncthreads();
  for (int h = nch / 2; h > 0; h >>= 1) {
    if (ch < h) {
      const double2 o = part[threadIdx.x + h * ld];
      part[threadIdx.x].x += o.x;
      part[threadIdx.x].y += o.y;
    }
    __syncthreads();
  }
  if (ch == 0) q[(int64_t)a * ld + k] = mk<T>((T)part[k].x, (T)part[k].y);
}

// Setup: pressure block of the coarse columns j (real part) and j+1 (imaginary
// part) of every block: z_p[v][k] = [loc(v) == j] + i [loc(v) == j+1].
template <typename T>
__global__ void k_agg_indicator(const int32_t *__restrict__ agg, const int32_t *__restrict__ agg_loc, int64_t P,
                                int ld, int j, typename cpx<T>::t *__restrict__ zp) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= P * ld) return;
  const int l = agg_loc[agg[f / ld]];
  zp[f] = mk<T>(l == j ? T(1) : T(0), l == j + 1 ? T(1) : T(0));
}

// Setup: store the restricted images q = R_c^T D^T X of columns j, j+1 (X =
// -A~_u^-1 D R_c [e_j + i e_{j+1}]) as columns j, j+1 of the FP64 coarse matrix
// of every (block, mode), S = R_c^T D^T A~_u^-1 D R_c.  W holds per block and
// mode the augmented n x 2n matrix [S | I] (row-major) for the inversion.
template <typename T>
__global__ void k_cs_column(const int32_t *__restrict__ agg_blk, const int32_t *__restrict__ agg_loc,
                            const int32_t *__restrict__ blk_na, const int64_t *__restrict__ blk_so, int n_agg, int ld,
                            int j, const typename cpx<T>::t *__restrict__ q, double *__restrict__ W) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= (int64_t)n_agg * ld) return;
  const int a = (int)(f / ld), k = (int)(f % ld);
  const int b = agg_blk[a], n = blk_na[b];
  if (j >= n) return;
  const int i = agg_loc[a];
  double *A = W + 2 * blk_so[b] * ld + (int64_t)k * 2 * n * n;
  const typename cpx<T>::t v = q[f];
  A[(int64_t)i * 2 * n + j] = -(double)v.x;
  if (j + 1 < n) A[(int64_t)i * 2 * n + j + 1] = -(double)v.y;
}

// Setup: invert the coarse matrix of every (block, mode) by Gauss-Jordan
// elimination with partial pivoting in FP64 (one thread block per matrix; the
// pivot is the largest magnitude in the column, the lowest row on ties).  A
// pivot below 1e-13 of the largest entry (or a non-finite entry) marks the
// matrix singular: its inverse is written as zero, which switches the
// correction off for that system, and *n_singular is incremented.  The
// inverse is stored in T as sinv[(blk_so[b] + i n + j) ld + k].
template <typename T>
__global__ void __launch_bounds__(256) k_cs_invert(const int32_t *__restrict__ blk_na,
                                                   const int64_t *__restrict__ blk_so, int ld, double *__restrict__ W,
                                                   T *__restrict__ sinv, int *n_singular) {
  extern __shared__ double cs_sh[];
  const int b = blockIdx.x / ld, k = blockIdx.x % ld;
  const int n = blk_na[b], w = 2 * n, tid = threadIdx.x, bd = blockDim.x;
  double *A = W + 2 * blk_so[b] * ld + (int64_t)k * w * n;
  double *f = cs_sh, *prow = cs_sh + n, *rv = cs_sh + 3 * n;
  int *ri = reinterpret_cast<int *>(rv + bd);
  double amax = 0;
  for (int64_t e = tid; e < (int64_t)n * n; e += bd) {
    const int i = (int)(e / n), c = (int)(e % n);
    A[(int64_t)i * w + n + c] = (i == c) ? 1.0 : 0.0;
    const double v = fabs(A[(int64_t)i * w + c]);
    amax = (v > amax || v != v) ? v : amax;  // NaN propagates
  }
  rv[tid] = amax;
  __syncthreads();
  for (int h = bd / 2; h > 0; h >>= 1) {
    if (tid < h) {
      const double o = rv[tid + h];
      if (o > rv[tid] || o != o) rv[tid] = o;
    }
    __syncthreads();
  }
  amax = rv[0];
  __syncthreads();
  bool sing = !(amax > 0) || !isfinite(amax);
  for (int p = 0; p < n && !sing; ++p) {
    double best = -1;
    int bi = n;
    for (int i = p + tid; i < n; i += bd) {
      const double v = fabs(A[(int64_t)i * w + p]);
      if (v > best) { best = v; bi = i; }
    }
    rv[tid] = best;
    ri[tid] = bi;
    __syncthreads();
    for (int h = bd / 2; h > 0; h >>= 1) {
      if (tid < h) {
        const double o = rv[tid + h];
        const int oi = ri[tid + h];
        if (o > rv[tid] || (o == rv[tid] && oi < ri[tid])) { rv[tid] = o; ri[tid] = oi; }
      }
      __syncthreads();
    }
    const int piv = ri[0];
    const double pbest = rv[0];
    if (!(pbest > 1e-13 * amax) || piv >= n) { sing = true; break; }  // uniform: read from shared memory
    if (piv != p)
      for (int c = p + tid; c < w; c += bd) {
        const double x = A[(int64_t)p * w + c];
        A[(int64_t)p * w + c] = A[(int64_t)piv * w + c];
        A[(int64_t)piv * w + c] = x;
      }
    __syncthreads();
    const double inv = 1.0 / A[(int64_t)p * w + p];
    for (int c = p + tid; c < w; c += bd) prow[c] = A[(int64_t)p * w + c] * inv;
    for (int i = tid; i < n; i += bd) f[i] = A[(int64_t)i * w + p];
    __syncthreads();
    // columns < p of the left half are unit columns already and row p is zero there
    const int wc = w - p;
    for (int64_t e = tid; e < (int64_t)n * wc; e += bd) {
      const int i = (int)(e / wc), c = p + (int)(e % wc);
      A[(int64_t)i * w + c] = (i == p) ? prow[c] : A[(int64_t)i * w + c] - f[i] * prow[c];
    }
    __syncthreads();
  }
  for (int64_t e = tid; e < (int64_t)n * n; e += bd) {
    const int i = (int)(e / n), c = (int)(e % n);
    sinv[(blk_so[b] + e) * ld + k] = sing ? T(0) : (T)A[(int64_t)i * w + n + c];
  }
  if (sing && tid == 0) atomicAdd(n_singular, 1);
}

// y[a][k] = sum_j Sinv_{b,k}[loc(a)][j] q[a0(b) + j][k]: the coarse solve of every
// (block, mode), one thread per (aggregate, mode).
template <typename T>
__global__ void k_cs_product(const int32_t *__restrict__ agg_blk, const int32_t *__restrict__ agg_loc,
                             const int32_t *__restrict__ blk_na, const int32_t *__restrict__ blk_a0,
                             const int64_t *__restrict__ blk_so, int n_agg, int ld, const T *__restrict__ sinv,
                             const typename cpx<T>::t *__restrict__ q, typename cpx<T>::t *__restrict__ y) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= (int64_t)n_agg * ld) return;
  const int a = (int)(f / ld), k = (int)(f % ld);
  const int b = agg_blk[a], n = blk_na[b], i = agg_loc[a];
  const T *row = sinv + (blk_so[b] + (int64_t)i * n) * ld + k;
  const typename cpx<T>::t *qb = q + (int64_t)blk_a0[b] * ld + k;
  T sx = 0, sy = 0;
  for (int j = 0; j < n; ++j) {
    const T s = row[(int64_t)j * ld];
    const typename cpx<T>::t v = qb[(int64_t)j * ld];
    sx += s * v.x;
    sy += s * v.y;
  }
  y[f] = mk<T>(sx, sy);
}

// z_p[v][k] -= y[agg(v)][k] (the triangular form's pressure block is -S~^-1 r_p);
// rows of inactive components are left alone.
template <typename T>
__global__ void k_cs_broadcast(const PcArgs a, int dim, const int32_t *__restrict__ agg,
                               const typename cpx<T>::t *__restrict__ y, typename cpx<T>::t *__restrict__ zp) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= a.P * a.ld) return;
  const int64_t v = f / a.ld;
  if (row_idle(a.dof_comp, a.comp_active, (int64_t)dim * a.N + v)) return;
  const typename cpx<T>::t add = y[(int64_t)agg[v] * a.ld + f % a.ld];
  typename cpx<T>::t o = zp[f];
  o.x -= add.x;
  o.y -= add.y;
  zp[f] = o;
}

// Graph aggregates of the vertices (host, deterministic).  Connected
// components become blocks (numbered by their lowest vertex); in each,
// aggregates are grown breadth-first (neighbours in row order) from the lowest
// unassigned vertex up to ceil(grow * vertices / target) vertices; an
// aggregate left below a third of that size joins the first full-size
// aggregate next to it (if any).  Aggregates are numbered by block, then by
// seed.  grow starts at 1 and rises by 1.5x until no block has more than
// min(2 target, CS_NA_MAX) aggregates (na_cap instead, if positive).  With
// size > 0 every block's aggregates are grown to `size` vertices instead (times
// grow), whatever the block's size; target is then unused.  Columns outside
// [0, P) are ignored.
AggResult graph_aggregates(int64_t P, const int64_t *ptr, const int32_t *col, int target, int na_cap, int size) {
  AggResult r;
  std::vector<int32_t> comp(P, -1), queue;
  std::vector<int64_t> csize;
  queue.reserve(P);
  auto valid = [&](int32_t u) { return u >= 0 && (int64_t)u < P; };
  for (int64_t s0 = 0; s0 < P; ++s0) {
    if (comp[s0] >= 0) continue;
    const int32_t id = (int32_t)csize.size();
    queue.clear();
    queue.push_back((int32_t)s0);
    comp[s0] = id;
    for (size_t h = 0; h < queue.size(); ++h) {
      const int64_t v = queue[h];
      for (int64_t e = ptr[v]; e < ptr[v + 1]; ++e) {
        const int32_t u = col[e];
        if (valid(u) && comp[u] < 0) { comp[u] = id; queue.push_back(u); }
      }
    }
    csize.push_back((int64_t)queue.size());
  }
  const int nb = (int)csize.size();
  r.n_blk = nb;
  r.agg.assign(P, -1);
  r.na.assign(nb, 0);
  r.a0.assign(nb, 0);
  double grow = 1.0;
  for (;;) {
    std::vector<int64_t> size_b(nb);
    for (int b = 0; b < nb; ++b)
      size_b[b] = std::max<int64_t>(1, (int64_t)std::ceil(size > 0 ? grow * size : grow * (double)csize[b] / target));
    std::vector<int32_t> &agg = r.agg;
    std::fill(agg.begin(), agg.end(), -1);
    std::vector<int64_t> cnt;
    std::vector<int32_t> seed_blk, frontier, next;
    for (int64_t s0 = 0; s0 < P; ++s0) {
      if (agg[s0] >= 0) continue;
      const int32_t id = (int32_t)cnt.size();
      const int64_t cap = size_b[comp[s0]];
      int64_t n = 1;
      agg[s0] = id;
      frontier.assign(1, (int32_t)s0);
      while (!frontier.empty() && n < cap) {
        next.clear();
        for (int32_t v : frontier)
          for (int64_t e = ptr[v]; e < ptr[v + 1] && n < cap; ++e) {
            const int32_t u = col[e];
            if (valid(u) && agg[u] < 0) { agg[u] = id; ++n; next.push_back(u); }
          }
        frontier.swap(next);
      }
      cnt.push_back(n);
      seed_blk.push_back(comp[s0]);
    }
    const int na0 = (int)cnt.size();
    std::vector<int32_t> into(na0);
    std::vector<char> small(na0);
    for (int g = 0; g < na0; ++g) {
      into[g] = g;
      small[g] = 3 * cnt[g] < size_b[seed_blk[g]];
    }
    for (int64_t v = 0; v < P; ++v) {
      const int32_t g = agg[v];
      if (!small[g] || into[g] != g) continue;
      for (int64_t e = ptr[v]; e < ptr[v + 1]; ++e) {
        const int32_t u = col[e];
        if (valid(u) && !small[agg[u]]) { into[g] = agg[u]; break; }
      }
    }
    std::vector<int32_t> order;
    for (int g = 0; g < na0; ++g)
      if (into[g] == g) order.push_back(g);
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) { return seed_blk[x] < seed_blk[y]; });
    std::vector<int32_t> newid(na0, -1);
    for (size_t i = 0; i < order.size(); ++i) newid[order[i]] = (int32_t)i;
    for (int64_t v = 0; v < P; ++v) agg[v] = newid[into[agg[v]]];
    const int n_agg = (int)order.size();
    r.blk.assign(n_agg, 0);
    r.loc.assign(n_agg, 0);
    std::fill(r.na.begin(), r.na.end(), 0);
    for (int i = 0; i < n_agg; ++i) {
      const int b = seed_blk[order[i]];
      r.blk[i] = b;
      if (r.na[b] == 0) r.a0[b] = i;
      r.loc[i] = r.na[b]++;
    }
    r.na_max = 0;
    for (int b = 0; b < nb; ++b) r.na_max = std::max(r.na_max, r.na[b]);
    if (r.na_max <= (na_cap > 0 ? na_cap : std::min(CS_NA_MAX, 2 * target))) break;
    grow *= 1.5;
  }
  return r;
}

// Aggregates of the mesh's vertex graph (the Q pattern: the columns < P of a
// vertex's S row) uploaded with their block tables.
static void build_aggregates(Ctx &c, Mesh &m, PcTables &t, int target) {
  const int64_t P = m.P;
  std::vector<int64_t> sp(P + 1);
  std::vector<int32_t> gl(std::max<int64_t>(P, 1));
  SCVS_CUDA(cudaMemcpyAsync(sp.data(), m.s_ptr, (P + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaMemcpyAsync(gl.data(), m.g_len, P * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  std::vector<int32_t> scol(std::max<int64_t>(sp[P] - sp[0], 1));
  SCVS_CUDA(cudaMemcpyAsync(scol.data(), m.s_col + sp[0], (sp[P] - sp[0]) * sizeof(int32_t), cudaMemcpyDeviceToHost,
                            c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  std::vector<int64_t> qp(P + 1, 0);
  for (int64_t v = 0; v < P; ++v) qp[v + 1] = qp[v] + gl[v];
  std::vector<int32_t> qc(std::max<int64_t>(qp[P], 1));
  for (int64_t v = 0; v < P; ++v)
    std::copy(scol.begin() + (sp[v] - sp[0]), scol.begin() + (sp[v] - sp[0]) + gl[v], qc.begin() + qp[v]);
  const AggResult r = graph_aggregates(P, qp.data(), qc.data(), target);
  const int n_agg = (int)r.blk.size(), nb = r.n_blk;
  std::vector<int64_t> ptr(n_agg + 1, 0), so(nb);
  std::vector<int32_t> vert(std::max<int64_t>(P, 1));
  for (int64_t v = 0; v < P; ++v) ++ptr[r.agg[v] + 1];
  for (int i = 0; i < n_agg; ++i) ptr[i + 1] += ptr[i];
  {
    std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t v = 0; v < P; ++v) vert[fill[r.agg[v]]++] = (int32_t)v;
  }
  int64_t acc = 0;
  for (int b = 0; b < nb; ++b) { so[b] = acc; acc += (int64_t)r.na[b] * r.na[b]; }
  t.n_agg = n_agg;
  t.n_blk = nb;
  t.na_max = r.na_max;
  t.so_total = acc;
  t.cs_target = target;
  t.agg = m.mode_arena.alloc<int32_t>(P);
  t.agg_ptr = m.mode_arena.alloc<int64_t>(n_agg + 1);
  t.agg_vert = m.mode_arena.alloc<int32_t>(P);
  t.agg_blk = m.mode_arena.alloc<int32_t>(n_agg);
  t.agg_loc = m.mode_arena.alloc<int32_t>(n_agg);
  t.blk_na = m.mode_arena.alloc<int32_t>(nb);
  t.blk_a0 = m.mode_arena.alloc<int32_t>(nb);
  t.blk_so = m.mode_arena.alloc<int64_t>(nb);
  auto up = [&](void *d, const void *h, size_t bytes) {
    SCVS_CUDA(cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, c.stream));
  };
  up(t.agg, r.agg.data(), P * sizeof(int32_t));
  up(t.agg_ptr, ptr.data(), (n_agg + 1) * sizeof(int64_t));
  up(t.agg_vert, vert.data(), P * sizeof(int32_t));
  up(t.agg_blk, r.blk.data(), n_agg * sizeof(int32_t));
  up(t.agg_loc, r.loc.data(), n_agg * sizeof(int32_t));
  up(t.blk_na, r.na.data(), nb * sizeof(int32_t));
  up(t.blk_a0, r.a0.data(), nb * sizeof(int32_t));
  up(t.blk_so, so.data(), nb * sizeof(int64_t));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));  // the host vectors go out of scope
}

// ---------------------------------------- two-level pressure Laplacian: set-up
// Galerkin matrix of the Laplacian's coarse level, row a of its block b:
// W[so_b + loc(a) n_b + loc(agg(u))] = sum of L_p[v][u] over the vertices v of
// aggregate a and their neighbours u off the outlet.  One thread block per
// aggregate; thread t owns the columns t, t + 256, t + 512, t + 768 (n_b <=
// LAP_NA_MAX) and visits the nonzeros in storage order, so the sums are
// reproducible.
__global__ void __launch_bounds__(256) k_lap_galerkin(const int64_t *__restrict__ agg_ptr,
                                                      const int32_t *__restrict__ agg_vert,
                                                      const int32_t *__restrict__ agg, const int32_t *__restrict__ agg_blk,
                                                      const int32_t *__restrict__ agg_loc,
                                                      const int32_t *__restrict__ blk_na,
                                                      const int64_t *__restrict__ blk_so, const int64_t *__restrict__ g_ptr,
                                                      const int64_t *__restrict__ s_ptr, const int32_t *__restrict__ s_col,
                                                      const double *__restrict__ Lp, double *__restrict__ W) {
  constexpr int NC = LAP_NA_MAX / 256;
  const int a = blockIdx.x, b = agg_blk[a], n = blk_na[b], t = threadIdx.x;
  double acc[NC];
#pragma unroll
  for (int i = 0; i < NC; ++i) acc[i] = 0;
  for (int64_t i = agg_ptr[a]; i < agg_ptr[a + 1]; ++i) {
    const int64_t v = agg_vert[i];
    const int64_t r0 = g_ptr[v], r1 = g_ptr[v + 1], s0 = s_ptr[v];
    for (int64_t e = r0; e < r1; ++e) {
      const int32_t au = agg[s_col[s0 + (e - r0)]];
      if (au < 0) continue;
      const int c = agg_loc[au];
      if ((c & 255) == t) acc[c >> 8] += Lp[e];
    }
  }
#pragma unroll
  for (int i = 0; i < NC; ++i)
    if (t + 256 * i < n) W[blk_so[b] + (int64_t)agg_loc[a] * n + t + 256 * i] = acc[i];
}

// Inverse of every block's Galerkin matrix (symmetric positive definite when
// an outlet vertex anchors the block) by the blocked Gauss-Jordan sweep in
// FP32, all blocks at once in one cooperative launch.  For each group K of
// LAP_BS pivots (k0 .. k0+bs-1) of every block with n_b > k0, from the matrix
// A of the previous sweep into the other buffer A':
//   1. D = A[K,K]^-1 (one thread block per block, in shared memory),
//   2. A'[K,K] = D, A'[K,j] = D A[K,j] and A'[i,K] = -A[i,K] D (i, j outside K),
//   3. A'[i,j] = A[i,j] - A[i,K] A'[K,j] (i, j outside K; 32 x 32 tiles with both
//      factors staged in shared memory),
// each phase ending at a bounded grid barrier (three per pivot group instead
// of one per pivot).  A pivot at or below 1e-6 of the block's largest
// diagonal entry (or not finite) marks the block singular: its inverse is
// written as zero (coarse correction off there) and counted in *n_singular.
// tile0 / pan0 [n_blk+1] are the offsets of every block's 32 x 32 tiles and
// panel entries (2 LAP_BS n_b); dmax, bad and Dinv (n_blk LAP_BS^2) are
// scratch; A0 holds the matrices on entry, A1 the other buffer.
constexpr int LAP_BS = 32;
__device__ __forceinline__ int lap_find(const int64_t *__restrict__ off, int n, int64_t e) {
  int lo = 0, hi = n - 1;  // the last b with off[b] <= e
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= e) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void __launch_bounds__(256) k_lap_invert(const int32_t *__restrict__ blk_na,
                                                    const int64_t *__restrict__ blk_so,
                                                    const int64_t *__restrict__ tile0,
                                                    const int64_t *__restrict__ pan0, int n_blk, int na_max,
                                                    const double *__restrict__ W, float *A0, float *A1, float *dmax,
                                                    int *bad, float *Dinv, float *__restrict__ inv_f,
                                                    double *__restrict__ inv_d, int *n_singular, GridSync *gs) {
  __shared__ float sA[LAP_BS][LAP_BS + 1], sB[LAP_BS][LAP_BS + 1];
  __shared__ float s_piv;
  __shared__ int s_bad;
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, nth = (int64_t)gridDim.x * blockDim.x;
  const int64_t total = blk_so[n_blk - 1] + (int64_t)blk_na[n_blk - 1] * blk_na[n_blk - 1];
  for (int64_t e = tid; e < total; e += nth) A0[e] = (float)W[e];
  for (int64_t b = tid; b < n_blk; b += nth) {
    const int n = blk_na[b];
    float m = 0;
    for (int i = 0; i < n; ++i) m = fmaxf(m, fabsf((float)W[blk_so[b] + (int64_t)i * n + i]));
    dmax[b] = m;
    bad[b] = !(m > 0) || !isfinite(m);
  }
  if (!grid_sync(gs, gridDim.x)) return;
  float *cur = A0, *nxt = A1;
  const int t = threadIdx.x;
  for (int k0 = 0; k0 < na_max; k0 += LAP_BS) {
    // 1. D = A[K,K]^-1 per block (in-place Gauss-Jordan sweep in shared memory)
    for (int b = blockIdx.x; b < n_blk; b += gridDim.x) {
      const int n = blk_na[b];
      if (n <= k0 || ld1co(bad + b)) continue;  // block-uniform
      const int bs = min(LAP_BS, n - k0);
      const float *A = cur + blk_so[b];
      for (int e = t; e < bs * bs; e += blockDim.x)
        sA[e / bs][e % bs] = ld1co(A + (int64_t)(k0 + e / bs) * n + k0 + e % bs);
      if (t == 0) s_bad = 0;
      __syncthreads();
      const float dm = ld1co(dmax + b);
      for (int k = 0; k < bs; ++k) {
        if (t == 0) {
          const float pv = sA[k][k];
          if (!(pv > 1e-6f * dm) || !isfinite(pv)) s_bad = 1;
          s_piv = pv;
        }
        __syncthreads();
        if (s_bad) break;  // uniform: read from shared memory after the barrier
        const float ip = 1.f / s_piv;
        if (t < bs) sB[0][t] = sA[t][k];  // column k before the sweep
        __syncthreads();
        if (t < bs && t != k) sA[k][t] *= ip;
        __syncthreads();
        for (int e = t; e < bs * bs; e += blockDim.x) {
          const int i = e / bs, j = e % bs;
          if (i != k && j != k) sA[i][j] = fmaf(-sB[0][i], sA[k][j], sA[i][j]);
        }
        __syncthreads();
        if (t < bs) sA[t][k] = (t == k) ? ip : -sB[0][t] * ip;
        __syncthreads();
      }
      if (s_bad) {
        if (t == 0) bad[b] = 1;
      } else {
        for (int e = t; e < bs * bs; e += blockDim.x) Dinv[(int64_t)b * LAP_BS * LAP_BS + e] = sA[e / bs][e % bs];
      }
      __syncthreads();
    }
    if (!grid_sync(gs, gridDim.x)) return;
    // 2. the pivot rows and columns: A'[K,j] = D A[K,j] (with A'[K,K] = D), A'[i,K] = -A[i,K] D
    for (int64_t e = tid; e < pan0[n_blk]; e += nth) {
      const int b = lap_find(pan0, n_blk, e);
      const int n = blk_na[b];
      if (n <= k0 || ld1co(bad + b)) continue;
      const int bs = min(LAP_BS, n - k0);
      const int64_t q = e - pan0[b];
      const float *A = cur + blk_so[b];
      float *O = nxt + blk_so[b];
      const float *D = Dinv + (int64_t)b * LAP_BS * LAP_BS;
      if (q < (int64_t)LAP_BS * n) {  // row panel entry (k0 + r, j)
        const int r = (int)(q / n), j = (int)(q % n);
        if (r >= bs) continue;
        float o;
        if (j >= k0 && j < k0 + bs) {
          o = ld1co(D + r * bs + (j - k0));
        } else {
          o = 0.f;
          for (int u = 0; u < bs; ++u) o = fmaf(ld1co(D + r * bs + u), ld1co(A + (int64_t)(k0 + u) * n + j), o);
        }
        O[(int64_t)(k0 + r) * n + j] = o;
      } else {  // column panel entry (i, k0 + c), i outside K
        const int64_t q2 = q - (int64_t)LAP_BS * n;
        const int c = (int)(q2 / n), i = (int)(q2 % n);
        if (c >= bs || (i >= k0 && i < k0 + bs)) continue;
        float o = 0.f;
        for (int u = 0; u < bs; ++u) o = fmaf(ld1co(A + (int64_t)i * n + k0 + u), ld1co(D + u * bs + c), o);
        O[(int64_t)i * n + k0 + c] = -o;
      }
    }
    if (!grid_sync(gs, gridDim.x)) return;
    // 3. the rest: A'[i,j] = A[i,j] - A[i,K] A'[K,j], by 32 x 32 tiles (finished or
    //    singular blocks are carried over unchanged)
    for (int64_t tl = blockIdx.x; tl < tile0[n_blk]; tl += gridDim.x) {
      const int b = lap_find(tile0, n_blk, tl);
      const int n = blk_na[b], nt = (n + LAP_BS - 1) / LAP_BS;
      const int64_t q = tl - tile0[b];
      const int i0 = (int)(q / nt) * LAP_BS, j0 = (int)(q % nt) * LAP_BS;
      const float *A = cur + blk_so[b];
      float *O = nxt + blk_so[b];
      const bool active = n > k0 && !ld1co(bad + b);  // block-uniform
      const int bs = active ? min(LAP_BS, n - k0) : 0;
      if (active) {
        for (int e = t; e < LAP_BS * LAP_BS; e += blockDim.x) {
          const int r = e / LAP_BS, cc = e % LAP_BS;
          sA[r][cc] = (i0 + r < n && cc < bs) ? ld1co(A + (int64_t)(i0 + r) * n + k0 + cc) : 0.f;
          sB[r][cc] = (r < bs && j0 + cc < n) ? ld1co(O + (int64_t)(k0 + r) * n + j0 + cc) : 0.f;
        }
      }
      __syncthreads();
      for (int e = t; e < LAP_BS * LAP_BS; e += blockDim.x) {
        const int i = i0 + e / LAP_BS, j = j0 + e % LAP_BS;
        if (i >= n || j >= n) continue;
        const int64_t f = (int64_t)i * n + j;
        if (!active) { O[f] = ld1co(A + f); continue; }
        if ((i >= k0 && i < k0 + bs) || (j >= k0 && j < k0 + bs)) continue;  // written in phase 2
        float o = ld1co(A + f);
        for (int u = 0; u < bs; ++u) o = fmaf(-sA[e / LAP_BS][u], sB[u][e % LAP_BS], o);
        O[f] = o;
      }
      __syncthreads();
    }
    if (!grid_sync(gs, gridDim.x)) return;
    float *tmp = cur; cur = nxt; nxt = tmp;
  }
  for (int64_t e = tid; e < total; e += nth) {
    const int b = lap_find(blk_so, n_blk, e);
    const float v = ld1co(bad + b) ? 0.f : ld1co(cur + e);
    inv_f[e] = v;
    inv_d[e] = (double)v;
  }
  for (int64_t b = tid; b < n_blk; b += nth)
    if (ld1co(bad + b)) atomicAdd(n_singular, 1);
}

// Stream-ordered device temporaries of a set-up step, released when the
// owner goes out of scope (also when a CUDA error unwinds the step).
struct LapTemps {
  Ctx &c;
  std::vector<void *> p;
  ~LapTemps() {
    for (void *q : p) cudaFreeAsync(q, c.stream);
  }
  template <typename P> P *get(int64_t n) {
    P *q = nullptr;
    SCVS_CUDA(ctx_malloc(c, &q, (size_t)std::max<int64_t>(n, 1) * sizeof(P), c.stream));
    p.push_back(q);
    return q;
  }
};

// Coarse level of the pressure Laplacian (host aggregation, device Galerkin
// matrices and inverses), kept in the mesh arena for the mesh's lifetime.  The
// graph is the vertex graph with the outlet vertices (p = 0 there) removed;
// every connected component of it must touch the outlet, else the mesh keeps
// the plain polynomial.
static void lap_build(Ctx &c, Mesh &m, int size) {
  LapCoarse &L = m.lap;
  L = LapCoarse{};
  L.target = size;
  const int64_t P = m.P;
  std::vector<int64_t> sp(P + 1);
  std::vector<int32_t> gl(std::max<int64_t>(P, 1));
  std::vector<uint8_t> om(std::max<int64_t>(P, 1));
  SCVS_CUDA(cudaMemcpyAsync(sp.data(), m.s_ptr, (P + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaMemcpyAsync(gl.data(), m.g_len, P * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaMemcpyAsync(om.data(), m.outmask, P, cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  std::vector<int32_t> scol(std::max<int64_t>(sp[P] - sp[0], 1));
  SCVS_CUDA(cudaMemcpyAsync(scol.data(), m.s_col + sp[0], (sp[P] - sp[0]) * sizeof(int32_t), cudaMemcpyDeviceToHost,
                            c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  std::vector<int32_t> id(std::max<int64_t>(P, 1), -1);
  int64_t n = 0;
  for (int64_t v = 0; v < P; ++v)
    if (!om[v]) id[v] = (int32_t)n++;
  if (n == 0) { L.unanchored = 1; return; }
  std::vector<int64_t> cp(n + 1, 0);
  std::vector<int32_t> cc;
  std::vector<char> touch(n, 0);
  cc.reserve(sp[P] - sp[0]);
  for (int64_t v = 0; v < P; ++v) {
    if (om[v]) continue;
    const int64_t i = id[v];
    for (int64_t e = sp[v] - sp[0]; e < sp[v] - sp[0] + gl[v]; ++e) {
      const int32_t u = scol[e];
      if (om[u]) touch[i] = 1;
      else cc.push_back(id[u]);
    }
    cp[i + 1] = (int64_t)cc.size();
  }
  const AggResult r = graph_aggregates(n, cp.data(), cc.empty() ? nullptr : cc.data(), 1, LAP_NA_MAX, size);
  const int n_agg = (int)r.blk.size(), nb = r.n_blk;
  std::vector<char> anch(nb, 0);
  for (int64_t i = 0; i < n; ++i)
    if (touch[i]) anch[r.blk[r.agg[i]]] = 1;
  for (int b = 0; b < nb; ++b) L.unanchored += !anch[b];
  L.n_agg = n_agg;
  L.n_blk = nb;
  L.na_max = r.na_max;
  if (L.unanchored > 0 || r.na_max > LAP_NA_MAX) return;
  std::vector<int32_t> agg(P);
  std::vector<int64_t> ptr(n_agg + 1, 0), so(nb);
  std::vector<int32_t> vert(n);
  for (int64_t v = 0; v < P; ++v) {
    agg[v] = om[v] ? -1 : r.agg[id[v]];
    if (agg[v] >= 0) ++ptr[agg[v] + 1];
  }
  for (int i = 0; i < n_agg; ++i) ptr[i + 1] += ptr[i];
  {
    std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t v = 0; v < P; ++v)
      if (agg[v] >= 0) vert[fill[agg[v]]++] = (int32_t)v;
  }
  int64_t acc = 0;
  for (int b = 0; b < nb; ++b) { so[b] = acc; acc += (int64_t)r.na[b] * r.na[b]; }
  L.so_total = acc;
  L.agg = m.arena.alloc<int32_t>(P);
  L.agg_ptr = m.arena.alloc<int64_t>(n_agg + 1);
  L.agg_vert = m.arena.alloc<int32_t>(n);
  L.agg_blk = m.arena.alloc<int32_t>(n_agg);
  L.agg_loc = m.arena.alloc<int32_t>(n_agg);
  L.blk_na = m.arena.alloc<int32_t>(nb);
  L.blk_a0 = m.arena.alloc<int32_t>(nb);
  L.blk_so = m.arena.alloc<int64_t>(nb);
  L.inv_f = m.arena.alloc<float>(acc);
  L.inv_d = m.arena.alloc<double>(acc);
  auto up = [&](void *d, const void *h, size_t bytes) {
    SCVS_CUDA(cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, c.stream));
  };
  up(L.agg, agg.data(), P * sizeof(int32_t));
  up(L.agg_ptr, ptr.data(), (n_agg + 1) * sizeof(int64_t));
  up(L.agg_vert, vert.data(), n * sizeof(int32_t));
  up(L.agg_blk, r.blk.data(), n_agg * sizeof(int32_t));
  up(L.agg_loc, r.loc.data(), n_agg * sizeof(int32_t));
  up(L.blk_na, r.na.data(), nb * sizeof(int32_t));
  up(L.blk_a0, r.a0.data(), nb * sizeof(int32_t));
  up(L.blk_so, so.data(), nb * sizeof(int64_t));
  std::vector<int64_t> tile0(nb + 1, 0), pan0(nb + 1, 0);
  for (int b = 0; b < nb; ++b) {
    const int64_t nt = (r.na[b] + LAP_BS - 1) / LAP_BS;
    tile0[b + 1] = tile0[b] + nt * nt;
    pan0[b + 1] = pan0[b] + 2 * (int64_t)LAP_BS * r.na[b];
  }
  LapTemps tmp{c, {}};  // stream-ordered temporaries, released on every exit path
  double *W = tmp.get<double>(acc);
  float *A0 = tmp.get<float>(acc), *A1 = tmp.get<float>(acc), *dmax = tmp.get<float>(nb);
  float *Dinv = tmp.get<float>((int64_t)nb * LAP_BS * LAP_BS);
  int *bad = tmp.get<int>(nb), *nsing = tmp.get<int>(1);
  int64_t *tile0_d = tmp.get<int64_t>(nb + 1), *pan0_d = tmp.get<int64_t>(nb + 1);
  up(tile0_d, tile0.data(), (nb + 1) * sizeof(int64_t));
  up(pan0_d, pan0.data(), (nb + 1) * sizeof(int64_t));
  SCVS_CUDA(cudaMemsetAsync(W, 0, (size_t)acc * sizeof(double), c.stream));
  SCVS_CUDA(cudaMemsetAsync(nsing, 0, sizeof(int), c.stream));
  {
    KScope ks(c, KC_PRECOND, (double)n * 4 + (double)m.q_nnz * 28 + (double)acc * 8);
    k_lap_galerkin<<<n_agg, 256, 0, c.stream>>>(L.agg_ptr, L.agg_vert, L.agg, L.agg_blk, L.agg_loc, L.blk_na,
                                                L.blk_so, m.g_ptr, m.s_ptr, m.s_col, m.Lp, W);
    count_launch(c);
  }
  {
    KScope ks(c, KC_PRECOND, (double)acc * 20 + (double)((r.na_max + LAP_BS - 1) / LAP_BS) * acc * 12);
    const void *kfn = (const void *)k_lap_invert;
    int n_blk = nb, na_max = r.na_max;
    GridSync *gs = c.gsync;
    void *args[] = {(void *)&L.blk_na, (void *)&L.blk_so, (void *)&tile0_d, (void *)&pan0_d, (void *)&n_blk,
                    (void *)&na_max, (void *)&W, (void *)&A0, (void *)&A1, (void *)&dmax, (void *)&bad,
                    (void *)&Dinv, (void *)&L.inv_f, (void *)&L.inv_d, (void *)&nsing, (void *)&gs};
    SCVS_CUDA(cudaLaunchCooperativeKernel(kfn, dim3(coop_grid(c, kfn, 0)), dim3(256), args, 0, c.stream));
    count_launch(c);
  }
  int h_sing = 0, gerr = 0;
  SCVS_CUDA(cudaMemcpyAsync(&h_sing, nsing, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaMemcpyAsync(&gerr, &c.gsync->err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));  // the host vectors go out of scope
  if (gerr) {  // a barrier wait gave up: the inverses are incomplete
    SCVS_CUDA(cudaMemsetAsync(c.gsync, 0, sizeof(GridSync), c.stream));
    throw (int)SCVS_ERR_TIMEOUT;
  }
  L.singular = h_sing;
  L.on = true;
}

static int cs_target_of(const Ctx &c) { return c.opts.schur_agg > 0 ? c.opts.schur_agg : CS_DEFAULT_AGG; }

// Start of the velocity solve of the triangular form (k_tri_vel0): rt = r_u - D z_p
// and the first iterate of the velocity polynomial, written to uA.
template <typename T>
static void tri_vel0_launch(Ctx &c, const Mesh &m, const PcArgs &a, const PcTables &t, typename cpx<T>::t *r,
                            const double *rscale, const typename cpx<T>::t *zp, typename cpx<T>::t *rt,
                            typename cpx<T>::t *uA) {
  const double cs = 2.0 * sizeof(T), pb = (double)m.P * m.ld * cs, vb = (double)m.dim * m.N * m.ld * cs;
  KScope ks(c, KC_PRECOND, vb * (rscale ? 4 : 3) + (double)m.g_nnz * (4 + m.dim * sizeof(T)) + pb +
                               (double)(m.N + 1) * 8 + (double)m.N * 17);
  auto body = [&](auto mpl_c, auto l_c) {
    constexpr int MPL = decltype(mpl_c)::value, L = decltype(l_c)::value;
    const int gpb = 256 / L;
    const unsigned nb = row_blocks(c, m.N, gpb, a.tile);
    if (m.dim == 2)
      k_tri_vel0<T, MPL, L, 2><<<nb, 256, 0, c.stream>>>(a, r, rscale, t.inv_theta_u, zp, rt, uA);
    else
      k_tri_vel0<T, MPL, L, 3><<<nb, 256, 0, c.stream>>>(a, r, rscale, t.inv_theta_u, zp, rt, uA);
  };
  if constexpr (sizeof(T) == 4) {
    const int mpl = m.mpl_cheb ? m.mpl_cheb : default_mpl<T>(m.ld);
    SCVS_DISPATCH_SHAPE(m.ld, mpl, body(std::integral_constant<int, MPL>{}, std::integral_constant<int, L>{}));
  } else {
    SCVS_DISPATCH_LD(T, m.ld, body(std::integral_constant<int, MPL>{}, std::integral_constant<int, L>{}));
  }
  count_launch(c);
}

// Velocity iterate moves of one application: every Chebyshev step after step
// 0 moves the iterate between its two buffers once.
static int vel_moves(const PcTables &t, bool pmg) { return pmg ? (t.s_u - 1) + t.s_u : (t.s_u - 1); }

// Steps 1.. of the velocity solve from the first iterate in ucur (step 0 done):
// the velocity polynomial, or for the p-multigrid kinds pre-smoothing, fine
// residual, coarse solve, prolongation and post-smoothing.  ru is the velocity
// right-hand side; uprev, rc and zc are scratch.  Returns the buffer holding
// the result (ucur or uprev, after vel_moves(t, pmg) moves).
template <typename T>
static typename cpx<T>::t *vel_cycle(Ctx &c, const Mesh &m, const PcArgs &a, const PcTables &t, bool pmg,
                                     const typename cpx<T>::t *ru, typename cpx<T>::t *ucur,
                                     typename cpx<T>::t *uprev, typename cpx<T>::t *rc,
                                     typename cpx<T>::t *const *zc) {
  using C = typename cpx<T>::t;
  const double cs = 2.0 * sizeof(T), vb = (double)m.dim * m.N * m.ld * cs, cbk = (double)m.dim * m.P * m.ld * cs;
  auto step = [&](const double *al_u, const double *be_u, bool prev0_u) {
    ChebCoef cc{};
    cc.do_u = 1;
    cc.alpha_u = al_u;
    cc.beta_u = be_u;
    cc.prev_zero_u = prev0_u;
    cheb_launch<T>(c, m, a, cc, ru, ucur, uprev);
    std::swap(ucur, uprev);
  };
  // velocity polynomial / pre-smoothing
  for (int i = 1; i < t.s_u; ++i) step(t.alpha_u + (size_t)i * m.ld, t.beta_u + (size_t)i * m.ld, i == 1);
  if (pmg) {
    // fine residual, coarse solve (restriction + Chebyshev), prolongation
    {
      KScope ks(c, KC_CHEB_FINE, (double)m.s_nnz * (4 + 2 * sizeof(T)) + (double)(m.N + 1) * 8 + m.N + 3 * vb);
      bool staged = false;
      if constexpr (sizeof(T) == 4) {
        if (m.st_cheb && staged_ok(c, m, m.st_cheb, false, ucur)) {
          launch_vel_residual_staged(c, m, a, ru, ucur, uprev, m.st_cheb);
          staged = true;
        }
      }
      auto body = [&](auto mpl_c, auto l_c) {
        constexpr int MPL = decltype(mpl_c)::value, L = decltype(l_c)::value;
        const int gpb = 256 / L;
        const unsigned nb = row_blocks(c, m.N, gpb, a.tile);
        if (m.dim == 2)
          k_vel_residual<T, MPL, L, 2><<<nb, 256, 0, c.stream>>>(a, ru, ucur, uprev);
        else
          k_vel_residual<T, MPL, L, 3><<<nb, 256, 0, c.stream>>>(a, ru, ucur, uprev);
      };
      if (!staged) {
        if constexpr (sizeof(T) == 4) {
          const int mpl = m.mpl_cheb ? m.mpl_cheb : default_mpl<T>(m.ld);
          SCVS_DISPATCH_SHAPE(m.ld, mpl, body(std::integral_constant<int, MPL>{}, std::integral_constant<int, L>{}));
        } else {
          SCVS_DISPATCH_LD(T, m.ld, body(std::integral_constant<int, MPL>{}, std::integral_constant<int, L>{}));
        }
        count_launch(c);
      }
    }
    C *zres = coarse_solve<T>(c, m, a, t, uprev, rc, zc);
    {
      KScope ks(c, KC_PRECOND, 2 * vb + cbk + (double)(m.N - m.P) * 8 + m.N);
      k_prolong<T><<<ceil_div((int64_t)m.dim * m.N * m.ld, 512), 256, 0, c.stream>>>(a, m.dim, zres, ucur);
      count_launch(c);
    }
    // post-smoothing from the corrected iterate: first step z1 = z0 + D^-1 (r - A z0)/theta
    step(t.zeros, t.inv_theta_u, true);
    for (int i = 1; i < t.s_u; ++i) step(t.alpha_u + (size_t)i * m.ld, t.beta_u + (size_t)i * m.ld, false);
  }
  return ucur;
}

template <typename T>
static void schur_coarse_setup(Ctx &c, Mesh &m, PcTables &t);
template <typename T>
static void schur_coarse_apply(Ctx &c, const Mesh &m, const PcArgs &a, const PcTables &t,
                               const typename cpx<T>::t *r, typename cpx<T>::t *z, typename cpx<T>::t *q,
                               typename cpx<T>::t *y);

// z = P^-1 r for all modes (right block preconditioner).  scratch holds
// precond_scratch_elems(m) elements.  rscale (device, [ld], may be null): r is
// first scaled per mode and written back (lazy normalisation of v_j).
template <typename T>
void apply_precond(Ctx &c, Mesh &m, const typename cpx<T>::t *r_in, typename cpx<T>::t *z,
                   typename cpx<T>::t *scratch, const double *rscale) {
  using C = typename cpx<T>::t;
  C *r = const_cast<C *>(r_in);
  const int64_t total = m.n_dof * m.ld;
  const unsigned eb = ceil_div(total, 256);
  const double cs = 2.0 * sizeof(T), blk = (double)total * cs, vb = (double)m.dim * m.N * m.ld * cs;
  const int kind = pc_kind(c, m);
  if (kind == SCVS_PC_BLOCK_DIAG) {
    const PcArgs a = pc_args<T>(m);
    KScope ks(c, KC_PRECOND, blk * (rscale ? 3 : 2) + (double)m.N * 17 + (double)m.P * 17);
    if (m.dim == 2)
      k_pc_step0<T, 2, true><<<eb, 256, 0, c.stream>>>(a, r, rscale, nullptr, z, total);
    else
      k_pc_step0<T, 3, true><<<eb, 256, 0, c.stream>>>(a, r, rscale, nullptr, z, total);
    count_launch(c);
    return;
  }
  PcTables &t = m.pc;
  pc_tables(c, m, t);
  const bool cs_on = kind == SCVS_PC_TRI_PMG_CS;
  if (cs_on && (t.cs_bytes != (int)sizeof(T) || t.cs_target != cs_target_of(c))) schur_coarse_setup<T>(c, m, t);
  const PcArgs a = pc_args<T>(m);
  const bool tri = kind == SCVS_PC_TRI_PMG || cs_on;
  const bool pmg = kind == SCVS_PC_BLOCK_PMG || tri;
  const int64_t pblk = m.P * m.ld, cblk = (int64_t)m.dim * m.P * m.ld;
  C *other = scratch;  // velocity part lives in dofs [0, dim N)
  C *pM[2] = {scratch + total, scratch + total + pblk};
  C *pL[2] = {scratch + total + 2 * pblk, scratch + total + 3 * pblk};
  C *rc = scratch + total + 4 * pblk;
  C *zc[2] = {rc + cblk, rc + 2 * cblk};
  C *rt = rc + 3 * cblk;  // velocity right-hand side of the triangular form
  // the velocity iterate ping-pongs between z and `other`; the first iterate
  // goes where the last one lands on z
  C *uA = (vel_moves(t, pmg) % 2 == 0) ? z : other;
  C *uB = (uA == z) ? other : z;
  // 1. pressure block: z_p = -/+ (mu M_p^-1 + j omega rho L_p^-1) r_p (minus: Schur
  //    complement of the triangular form; plus: block-diagonal form)
  pressure_solve<T>(c, m, a, t, r, rscale, pM, pL, z, tri ? T(-1) : T(1), rc, zc[0]);
  // 1b. coarse Schur correction z_p -= R_c S_c^-1 R_c^T r_p (r_p already scaled
  //     by the pressure solve); the pressure polynomials' buffers are free again
  if (cs_on) schur_coarse_apply<T>(c, m, a, t, r, z, pM[0], pM[1]);
  // 2. velocity right-hand side and step 0 of the velocity polynomial
  const C *ru = r;
  if (tri) {
    tri_vel0_launch<T>(c, m, a, t, r, rscale, z + (int64_t)m.dim * m.N * m.ld, rt, uA);
    ru = rt;
  } else {
    const int64_t fu = (int64_t)m.dim * m.N * m.ld;
    KScope ks0(c, KC_PRECOND, vb * (rscale ? 3 : 2) + (double)m.N * 17);
    if (m.dim == 2)
      k_pc_step0<T, 2, false><<<ceil_div(fu, 256), 256, 0, c.stream>>>(a, r, rscale, t.inv_theta_u, uA, fu);
    else
      k_pc_step0<T, 3, false><<<ceil_div(fu, 256), 256, 0, c.stream>>>(a, r, rscale, t.inv_theta_u, uA, fu);
    count_launch(c);
  }
  // 3.-5. the rest of the velocity solve
  C *res = vel_cycle<T>(c, m, a, t, pmg, ru, uA, uB, rc, zc);
  if (res != z) throw (int)SCVS_ERR_STATE;  // buffer bookkeeping invariant
}
// Stream-ordered temporaries of the coarse Schur setup, released (and the
// components' activity flags restored) on every exit path.
struct CsTemps {
  Ctx &c;
  Mesh &m;
  std::vector<void *> p;
  uint8_t *saved = nullptr;
  CsTemps(Ctx &c_, Mesh &m_) : c(c_), m(m_) {}
  ~CsTemps() {
    if (saved) cudaMemcpyAsync(m.comp_active, saved, m.n_comp, cudaMemcpyDeviceToDevice, c.stream);
    for (void *q : p) cudaFreeAsync(q, c.stream);
  }
  template <typename P> P *get(int64_t n) {
    P *q = nullptr;
    SCVS_CUDA(ctx_malloc(c, &q, (size_t)std::max<int64_t>(n, 1) * sizeof(P), c.stream));
    p.push_back(q);
    return q;
  }
};

// Setup of the coarse Schur correction for the current modes, physics and
// polynomial degrees: the aggregates (host, once per target), then per pair of
// coarse columns (j, j+1) one velocity cycle for every block and mode at once,
// X = A~_u^-1 (-D R_c [e_j + i e_{j+1}]), its image D^T X (pressure rows of the
// saddle operator with zero pressure input), restricted to the aggregates, and
// finally the FP64 inverses.  Every component takes part whatever its current
// activity flag (restored afterwards).
template <typename T>
static void schur_coarse_setup(Ctx &c, Mesh &m, PcTables &t) {
  using C = typename cpx<T>::t;
  const int target = cs_target_of(c);
  if (t.cs_target != target || !t.agg) {
    build_aggregates(c, m, t, target);
    t.sinv = m.mode_arena.alloc<double>(std::max<int64_t>(1, t.so_total * m.ld));  // room for either precision
  }
  const int64_t total = m.n_dof * m.ld, fp = (int64_t)m.dim * m.N * m.ld, pl = m.P * m.ld;
  const int64_t pblk = pl, cblk = (int64_t)m.dim * m.P * m.ld;
  CsTemps tmp{c, m};
  if (m.comp_active) {
    uint8_t *sv = tmp.get<uint8_t>(m.n_comp);
    SCVS_CUDA(cudaMemcpyAsync(sv, m.comp_active, m.n_comp, cudaMemcpyDeviceToDevice, c.stream));
    tmp.saved = sv;
    SCVS_CUDA(cudaMemsetAsync(m.comp_active, 1, m.n_comp, c.stream));
  }
  C *Z = tmp.get<C>(total), *Y = tmp.get<C>(total), *R0 = tmp.get<C>(fp);
  C *scr = tmp.get<C>(precond_scratch_elems(m));
  C *q = tmp.get<C>((int64_t)t.n_agg * m.ld);
  double *W = tmp.get<double>(2 * t.so_total * m.ld);
  int *nsing = tmp.get<int>(1);
  SCVS_CUDA(cudaMemsetAsync(R0, 0, fp * sizeof(C), c.stream));
  SCVS_CUDA(cudaMemsetAsync(W, 0, 2 * t.so_total * m.ld * sizeof(double), c.stream));
  SCVS_CUDA(cudaMemsetAsync(nsing, 0, sizeof(int), c.stream));
  const PcArgs a = pc_args<T>(m);
  C *other = scr;
  C *rc = scr + total + 4 * pblk;
  C *zc[2] = {rc + cblk, rc + 2 * cblk};
  C *rt = rc + 3 * cblk;
  C *uA = (vel_moves(t, true) % 2 == 0) ? Z : other;
  C *uB = (uA == Z) ? other : Z;
  const double cs = 2.0 * sizeof(T);
  for (int j = 0; j < t.na_max; j += 2) {
    {
      KScope ks(c, KC_PRECOND, pl * cs + (double)m.P * 4 + (double)t.n_agg * 4);
      k_agg_indicator<T><<<ceil_div(pl, 256), 256, 0, c.stream>>>(t.agg, t.agg_loc, m.P, m.ld, j, Z + fp);
      count_launch(c);
    }
    tri_vel0_launch<T>(c, m, a, t, R0, nullptr, Z + fp, rt, uA);
    if (vel_cycle<T>(c, m, a, t, true, rt, uA, uB, rc, zc) != Z) throw (int)SCVS_ERR_STATE;
    SCVS_CUDA(cudaMemsetAsync(Z + fp, 0, pl * sizeof(C), c.stream));
    apply_saddle<T>(c, m, Z, Y);
    {
      KScope ks(c, KC_PRECOND, pl * cs + (double)m.P * 4 + (double)(t.n_agg + 1) * 8 + (double)t.n_agg * m.ld * cs);
      k_agg_restrict<T><<<t.n_agg, AGG_RT, 0, c.stream>>>(t.agg_ptr, t.agg_vert, m.ld, Y + fp, q);
      count_launch(c);
    }
    {
      KScope ks(c, KC_PRECOND, (double)t.n_agg * m.ld * (cs + 16) + (double)t.n_agg * 8);
      k_cs_column<T><<<ceil_div((int64_t)t.n_agg * m.ld, 256), 256, 0, c.stream>>>(
          t.agg_blk, t.agg_loc, t.blk_na, t.blk_so, t.n_agg, m.ld, j, q, W);
      count_launch(c);
    }
  }
  {
    KScope ks(c, KC_PRECOND, (double)t.so_total * m.ld * (16 + 8 + sizeof(T)));
    const size_t smem = (size_t)(3 * t.na_max + 256) * sizeof(double) + 256 * sizeof(int);
    k_cs_invert<T><<<t.n_blk * m.ld, 256, smem, c.stream>>>(t.blk_na, t.blk_so, m.ld, W, (T *)t.sinv, nsing);
    count_launch(c);
  }
  int h_sing = 0;
  SCVS_CUDA(cudaMemcpyAsync(&h_sing, nsing, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  t.cs_singular = h_sing;
  t.cs_bytes = (int)sizeof(T);
}

// z_p -= R_c S_c^-1 R_c^T r_p for every active (component, mode); q and y are
// scratch of n_agg * ld elements.
template <typename T>
static void schur_coarse_apply(Ctx &c, const Mesh &m, const PcArgs &a, const PcTables &t,
                               const typename cpx<T>::t *r, typename cpx<T>::t *z, typename cpx<T>::t *q,
                               typename cpx<T>::t *y) {
  const int64_t fp = (int64_t)m.dim * m.N * m.ld, pl = m.P * m.ld, ql = (int64_t)t.n_agg * m.ld;
  const double cs = 2.0 * sizeof(T);
  {
    KScope ks(c, KC_PRECOND, pl * cs + (double)m.P * 4 + (double)(t.n_agg + 1) * 8 + ql * cs);
    k_agg_restrict<T><<<t.n_agg, AGG_RT, 0, c.stream>>>(t.agg_ptr, t.agg_vert, m.ld, r + fp, q);
    count_launch(c);
  }
  {
    KScope ks(c, KC_PRECOND, (double)t.so_total * m.ld * sizeof(T) + 2 * ql * cs + (double)t.n_agg * 12);
    k_cs_product<T><<<ceil_div(ql, 256), 256, 0, c.stream>>>(t.agg_blk, t.agg_loc, t.blk_na, t.blk_a0, t.blk_so,
                                                            t.n_agg, m.ld, (const T *)t.sinv, q, y);
    count_launch(c);
  }
  {
    KScope ks(c, KC_PRECOND, 2 * pl * cs + (double)m.P * 4 + ql * cs);
    k_cs_broadcast<T><<<ceil_div(pl, 256), 256, 0, c.stream>>>(a, m.dim, t.agg, y, z + fp);
    count_launch(c);
  }
}

template void apply_precond<float>(Ctx &, Mesh &, const float2 *, float2 *, float2 *, const double *);
template void apply_precond<double>(Ctx &, Mesh &, const double2 *, double2 *, double2 *, const double *);

// ---------------------------------------------------------- power method
// y = D^-1 A v for the real-shifted velocity block A_r (per mode) and the two P1 matrices
// (mode-independent; evaluated on every mode column, read from column 0).
template <typename T, int MPL, int L, int DIM>
__global__ void __launch_bounds__(256)
k_jacobi_op(const PcArgs a, const typename cpx<T>::t *__restrict__ v, typename cpx<T>::t *__restrict__ y,
            const typename cpx<T>::t *__restrict__ vM, typename cpx<T>::t *__restrict__ yM,
            const typename cpx<T>::t *__restrict__ vL, typename cpx<T>::t *__restrict__ yL,
            const typename cpx<T>::t *__restrict__ vC, typename cpx<T>::t *__restrict__ yC,
            const double *__restrict__ vn2) {
  using C = typename cpx<T>::t;
  const int gpb = blockDim.x / L;
  const int lane = threadIdx.x % L, group = threadIdx.x / L;
  const unsigned gm = group_mask<L>();
  const int ld = a.ld, koff = lane * MPL;
  const T *Kv = (const T *)a.Kv, *Mv = (const T *)a.Mv, *Mpv = (const T *)a.Mpv, *Lpv = (const T *)a.Lpv;
  // vn2 (may be null): squared norms of the four input blocks per mode column,
  // [velocity | M_p | L_p | coarse][ld]; the outputs are divided by the norms,
  // which normalises the power iterate without a separate pass
  auto inv_norm = [&](int blk, int k) -> T {
    if (!vn2) return T(1);
    const double nn = vn2[blk * ld + k];
    return nn > 0 ? (T)(1.0 / sqrt(nn)) : T(0);
  };
  for (int64_t row = (int64_t)blockIdx.x * gpb + group; row < a.N + a.P; row += (int64_t)gridDim.x * gpb) {
    if (row < a.N) {
      const int64_t A = row;
      CV<T, MPL> aK[DIM], aM[DIM];
#pragma unroll
      for (int c = 0; c < DIM; ++c) { aK[c].zero(); aM[c].zero(); }
      const bool dir = a.dirmask[A];
      const int64_t r0 = a.s_ptr[A], r1 = dir ? r0 : a.s_ptr[A + 1];
      for (int64_t base = r0; base < r1; base += L) {
        const int64_t t = base + lane;
        int32_t col = 0;
        T kv = 0, mv = 0;
        if (t < r1) { col = a.s_col[t]; kv = Kv[t]; mv = Mv[t]; }
        const int cnt = (int)min((int64_t)L, r1 - base);
        for (int q = 0; q < cnt; ++q) {
          const int32_t B = gshfl<L>(gm, col, q);
          const T kq = gshfl<L>(gm, kv, q), mq = gshfl<L>(gm, mv, q);
#pragma unroll
          for (int c = 0; c < DIM; ++c) {
            CV<T, MPL> xv;
            ldv<T, MPL>(xv, v + ((int64_t)B * DIM + c) * ld + koff);
            axpy(aK[c], kq, xv);
            axpy(aM[c], mq, xv);
          }
        }
      }
#pragma unroll
      for (int i = 0; i < MPL; ++i) {
        const int k = koff + i;
        const T dr = vel_dinv<T>(a, A, k) * inv_norm(0, k);
        const T mu = (T)a.mu, wr = (T)(fabs(a.omega[k]) * a.rho);
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          const int64_t f = (A * DIM + c) * ld + k;
          T xr = mu * aK[c].re[i] + wr * aM[c].re[i], xi = mu * aK[c].im[i] + wr * aM[c].im[i];
          if (dir) { xr = 0; xi = 0; }
          y[f] = mk<T>(dr * xr, dr * xi);
        }
      }
    } else {
      const int64_t B = row - a.N;
      const int64_t r0 = a.g_ptr[B], r1 = a.g_ptr[B + 1], s0 = a.s_ptr[B];
      CV<T, MPL> aMp, aLp, aKc, aMc;
      aMp.zero(); aLp.zero(); aKc.zero(); aMc.zero();
      const T *Kc = (const T *)a.Kcv, *Mc = (const T *)a.Mcv;
      for (int64_t base = r0; base < r1; base += L) {
        const int64_t t = base + lane;
        int32_t col = 0;
        T mv = 0, lv = 0, kc = 0, mc = 0;
        if (t < r1) { col = a.s_col[s0 + (t - r0)]; mv = Mpv[t]; lv = Lpv[t]; kc = Kc[t]; mc = Mc[t]; }
        const int cnt = (int)min((int64_t)L, r1 - base);
        for (int q = 0; q < cnt; ++q) {
          const int32_t Bc = gshfl<L>(gm, col, q);
          const T mq = gshfl<L>(gm, mv, q), lq = gshfl<L>(gm, lv, q);
          const T kcq = gshfl<L>(gm, kc, q), mcq = gshfl<L>(gm, mc, q);
          CV<T, MPL> x1, x2, x3;
          ldv<T, MPL>(x1, vM + (int64_t)Bc * ld + koff);
          ldv<T, MPL>(x2, vL + (int64_t)Bc * ld + koff);
          ldv<T, MPL>(x3, vC + (int64_t)Bc * ld + koff);
          axpy(aMp, mq, x1);
          axpy(aLp, lq, x2);
          axpy(aKc, kcq, x3);
          axpy(aMc, mcq, x3);
        }
      }
      {
        CV<T, MPL> o3;
        const bool dir = a.dirmask[B];
#pragma unroll
        for (int i = 0; i < MPL; ++i) {
          const double w = a.omega[koff + i];
          const T d = dir ? T(0) : (T)(1.0 / (a.mu * a.k1_diag[B] + fabs(w) * a.rho * a.mp_diag[B])) * inv_norm(3, koff + i);
          const T cr = (T)(fabs(w) * a.rho), mu = (T)a.mu;
          o3.re[i] = d * (mu * aKc.re[i] + cr * aMc.re[i]);
          o3.im[i] = d * (mu * aKc.im[i] + cr * aMc.im[i]);
        }
        stv<T, MPL>(yC + B * ld + koff, o3);
      }
      const T dm = (T)(1.0 / a.mp_diag[B]), dl = (T)(1.0 / a.lp_diag[B]);
      CV<T, MPL> o1, o2;
#pragma unroll
      for (int i = 0; i < MPL; ++i) {
        const T sm = dm * inv_norm(1, koff + i), sl = dl * inv_norm(2, koff + i);
        o1.re[i] = sm * aMp.re[i]; o1.im[i] = sm * aMp.im[i];
        o2.re[i] = sl * aLp.re[i]; o2.im[i] = sl * aLp.im[i];
      }
      stv<T, MPL>(yM + B * ld + koff, o1);
      stv<T, MPL>(yL + B * ld + koff, o2);
    }
  }
}

// Per-mode 2-norms of a block of `rows` rows (free rows only where dirm != null,
// rows indexed as velocity dofs), accumulated in double into out2[ld] (atomic).
// Squared norm of every mode column of a block, deterministic: block b writes
// its partial sums to part[b][ld]; k_block_norm2_finish adds them in block
// order (the power-method bounds, and with them the Chebyshev intervals, are
// then bitwise reproducible).
template <typename T>
__global__ void k_block_norm2(const typename cpx<T>::t *__restrict__ v, int64_t rows, int ld, int dim,
                              const uint8_t *__restrict__ dirm, double *part) {
  __shared__ double s[256];
  double acc = 0.0;
  const int64_t total = rows * ld;
  for (int64_t f = blockIdx.x * 256ll + threadIdx.x; f < total; f += (int64_t)gridDim.x * 256) {
    if (dirm && dirm[(f / ld) / dim]) continue;
    auto z = v[f];
    acc += (double)z.x * z.x + (double)z.y * z.y;
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w >= ld; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x < ld) part[(int64_t)blockIdx.x * ld + threadIdx.x] = s[threadIdx.x];
}

// One block of 256 threads per mode column: strided partial sums, then a
// shared-memory tree, both in a fixed order.
__global__ void k_block_norm2_finish(const double *__restrict__ part, int nblocks, int ld, double *out2) {
  __shared__ double s[256];
  const int k = blockIdx.x;
  double acc = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += 256) acc += part[(int64_t)b * ld + k];
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) out2[k] = s[0];
}

__global__ void k_init_random(float2 *v, int64_t n) {
  int64_t i = blockIdx.x * 256ll + threadIdx.x;
  if (i >= n) return;
  // fixed hash of the index: deterministic start vector of the power method
  uint64_t h = (uint64_t)i * 0x9E3779B97F4A7C15ull;
  h ^= h >> 31; h *= 0xBF58476D1CE4E5B9ull; h ^= h >> 29;
  float a = (float)((h >> 40) & 0xFFFFFF) / 16777216.0f - 0.5f;
  float b = (float)((h >> 16) & 0xFFFFFF) / 16777216.0f - 0.5f;
  v[i] = make_float2(1.0f + a, b);
}

// Spectral radius estimates of D^-1 A for the real-shifted velocity block
// (per mode), the P1 mass and the P1 Laplacian (power method, 14 steps, FP32;
// it approaches lambda_max from below, and the Chebyshev intervals end at
// CHEB_TOP = 1.10 times the estimate.  On the benchmark pipe 40 steps with a 5%
// margin, 20 and 10 steps gave the same iteration counts and 7 steps let the
// smoothers diverge, so 14 keeps a margin above that edge).
void spectral_bounds(Ctx &c, Mesh &m) {
  const int ld = m.ld;
  const int64_t np = m.P * ld;
  const int64_t total = m.n_dof * ld;
  float2 *v = nullptr, *y = nullptr, *vM = nullptr, *yM = nullptr, *vL = nullptr, *yL = nullptr;
  float2 *vC = nullptr, *yC = nullptr;
  double *n2 = nullptr, *part = nullptr;
  SCVS_CUDA(ctx_malloc(c, &v, total * sizeof(float2), c.stream));
  SCVS_CUDA(ctx_malloc(c, &y, total * sizeof(float2), c.stream));
  SCVS_CUDA(ctx_malloc(c, &vM, np * sizeof(float2), c.stream));
  SCVS_CUDA(ctx_malloc(c, &yM, np * sizeof(float2), c.stream));
  SCVS_CUDA(ctx_malloc(c, &vL, np * sizeof(float2), c.stream));
  SCVS_CUDA(ctx_malloc(c, &yL, np * sizeof(float2), c.stream));
  SCVS_CUDA(ctx_malloc(c, &vC, np * sizeof(float2), c.stream));
  SCVS_CUDA(ctx_malloc(c, &yC, np * sizeof(float2), c.stream));
  SCVS_CUDA(ctx_malloc(c, &n2, 8 * ld * sizeof(double), c.stream));  // two alternating norm sets
  k_init_random<<<ceil_div(np, 256), 256, 0, c.stream>>>(vC, np);
  k_init_random<<<ceil_div(total, 256), 256, 0, c.stream>>>(v, total);
  k_init_random<<<ceil_div(np, 256), 256, 0, c.stream>>>(vM, np);
  k_init_random<<<ceil_div(np, 256), 256, 0, c.stream>>>(vL, np);
  c.launches.n += 4;
  const PcArgs a = pc_args<float>(m);
  const unsigned nbn = (unsigned)std::min<int64_t>(ceil_div(total, 256), 4 * c.num_sms);
  SCVS_CUDA(ctx_malloc(c, &part, (size_t)4 * nbn * ld * sizeof(double), c.stream));  // per-block partial norms
  std::vector<double> h(4 * ld, 0.0);
  const int iters = 14;
  for (int it = 0; it < iters; ++it) {
    // y = D^-1 A (v / ||v||) with ||v|| from the previous step (the start vector is used as is)
    const double *vn2 = it == 0 ? nullptr : n2 + ((it - 1) % 2) * 4 * ld;
    double *yn2 = n2 + (it % 2) * 4 * ld;
    SCVS_DISPATCH_LD(float, ld, {
      const int gpb = 256 / L;
      const unsigned nb = row_blocks(c, m.N + m.P, gpb);
      if (m.dim == 2)
        k_jacobi_op<float, MPL, L, 2><<<nb, 256, 0, c.stream>>>(a, v, y, vM, yM, vL, yL, vC, yC, vn2);
      else
        k_jacobi_op<float, MPL, L, 3><<<nb, 256, 0, c.stream>>>(a, v, y, vM, yM, vL, yL, vC, yC, vn2);
    });
    const float2 *blocks[4] = {y, yM, yL, yC};
    for (int q = 0; q < 4; ++q) {
      const int64_t rows = q == 0 ? (int64_t)m.dim * m.N : m.P;
      k_block_norm2<float><<<nbn, 256, 0, c.stream>>>(blocks[q], rows, ld, q == 0 ? m.dim : 1,
                                                      q == 0 ? m.dirmask : nullptr, part + (size_t)q * nbn * ld);
      k_block_norm2_finish<<<ld, 256, 0, c.stream>>>(part + (size_t)q * nbn * ld, (int)nbn, ld, yn2 + q * ld);
    }
    c.launches.n += 9;
    if (it == iters - 1) {
      // the input had unit norm: ||y|| is the Rayleigh-type estimate
      SCVS_CUDA(cudaMemcpyAsync(h.data(), yn2, 4 * ld * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
      break;
    }
    std::swap(v, y);
    std::swap(vM, yM);
    std::swap(vL, yL);
    std::swap(vC, yC);
  }
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  m.lam_u.assign(ld, 0.0);
  for (int k = 0; k < ld; ++k) m.lam_u[k] = std::sqrt(h[k]);
  // every mode column of the P1 blocks carries the same operator: use column 0
  m.lam_m = std::sqrt(h[ld + 0]);
  m.lam_l = std::sqrt(h[2 * ld + 0]);
  m.lam_c.assign(ld, 0.0);
  for (int k = 0; k < ld; ++k) m.lam_c[k] = std::sqrt(h[3 * ld + k]);
  for (float2 *p : {v, y, vM, yM, vL, yL, vC, yC}) SCVS_CUDA(cudaFreeAsync(p, c.stream));
  SCVS_CUDA(cudaFreeAsync(n2, c.stream));
  SCVS_CUDA(cudaFreeAsync(part, c.stream));
}

// Residual of the current FP64 iterate: r = b - A_hat x (FP64 SpMM) and the
// per-mode squared free-row norms into norm2_out_dev[ld].  zero_start: x is
// the zero start (g on the Dirichlet rows, 0 elsewhere), whose product with the
// masked operator A_hat is exactly zero (every Dirichlet column is masked), so
// r = b on the free rows bit for bit and the FP64 product is skipped.
void residual_fp64(Ctx &c, Mesh &m, float2 *r32, double2 *r64, double *norm2_out_dev, bool zero_start) {
  const int64_t total = m.n_dof * m.ld;
  if (zero_start) {
    if (r32 || r64) {
      KScope ks(c, KC_VECTOR, (double)total * (16 + (r64 ? 16 : 0) + (r32 ? 8 : 0)));
      k_residual_finish<<<ceil_div(total, 256), 256, 0, c.stream>>>(m.b, nullptr, m.dirmask, m.N, m.dim, total, m.ld,
                                                                    r32, r64, m.dof_comp, m.comp_active);
      count_launch(c);
    }
    norms2_sys(c, m, r64 ? r64 : m.b, norm2_out_dev);  // the free rows of r and b hold the same values
    return;
  }
  double2 *ax = nullptr;
  SCVS_CUDA(ctx_malloc(c, &ax, total * sizeof(double2), c.stream));
  launch_saddle<double>(c, m, saddle_args<double>(c, m, true), m.x, ax);
  double2 *r = r64 ? r64 : ax;
  {
    KScope ks(c, KC_VECTOR, (double)total * (32 + 16 + (r32 ? 8 : 0)));
    k_residual_finish<<<ceil_div(total, 256), 256, 0, c.stream>>>(m.b, ax, m.dirmask, m.N, m.dim, total, m.ld, r32,
                                                                  r64 ? r64 : ax, m.dof_comp, m.comp_active);
    count_launch(c);
  }
  norms2_sys(c, m, r, norm2_out_dev);
  SCVS_CUDA(cudaFreeAsync(ax, c.stream));
}

// ------------------------------------------------------------- autotuner
// Row-group shape (modes per lane) of the all-modes SpMM and of the fine
// Chebyshev step, chosen per mesh and mode stride by timing every valid
// candidate on this mesh with CUDA events (median of 3 launches after one
// warm-up) and kept in the mesh.
void autotune_shapes(Ctx &c, Mesh &m) {
  const int64_t total = m.n_dof * m.ld;
  float2 *x = nullptr, *y = nullptr;
  double *zeros = nullptr;
  SCVS_CUDA(ctx_malloc(c, &x, total * sizeof(float2), c.stream));
  SCVS_CUDA(ctx_malloc(c, &y, total * sizeof(float2), c.stream));
  SCVS_CUDA(ctx_malloc(c, &zeros, m.ld * sizeof(double), c.stream));
  SCVS_CUDA(cudaMemsetAsync(zeros, 0, m.ld * sizeof(double), c.stream));
  k_init_random<<<ceil_div(total, 256), 256, 0, c.stream>>>(x, total);
  count_launch(c);
  cudaEvent_t e0, e1;
  SCVS_CUDA(cudaEventCreate(&e0));
  SCVS_CUDA(cudaEventCreate(&e1));
  const bool timers_on = c.timers.on;
  c.timers.on = false;
  constexpr int NT = (int)(sizeof(SCVS_TILES) / sizeof(SCVS_TILES[0]));
  m.tune_us.assign(2 * 3 * NT, 0.0f);  // [SpMM | Chebyshev][MPL 1, 2, 4][tile]
  auto time_it = [&](auto &&launch) {
    launch();
    float best = 1e30f;
    for (int r = 0; r < 2; ++r) {
      SCVS_CUDA(cudaEventRecord(e0, c.stream));
      launch();
      SCVS_CUDA(cudaEventRecord(e1, c.stream));
      SCVS_CUDA(cudaEventSynchronize(e1));
      float t = 0;
      SCVS_CUDA(cudaEventElapsedTime(&t, e0, e1));
      best = std::min(best, t);
    }
    return best * 1e3f;
  };
  ChebCoef cc{};
  cc.do_u = 1;
  cc.alpha_u = zeros;
  cc.beta_u = zeros;
  cc.prev_zero_u = 1;
  int best_s[2] = {0, 0}, best_c[2] = {0, 0};
  float tb_s = 1e30f, tb_c = 1e30f;
  m.st_spmm = m.st_cheb = 0;
  for (int mi = 0; mi < 3; ++mi) {
    const int mpl = 1 << mi;
    if (!shape_valid(m.ld, mpl)) continue;
    for (int ti = 0; ti < NT; ++ti) {
      m.mpl_spmm = mpl;
      m.tile_spmm = SCVS_TILES[ti];
      const float ts = time_it([&]() { apply_saddle<float>(c, m, x, y); });
      m.mpl_cheb = mpl;
      m.tile_cheb = SCVS_TILES[ti];
      const PcArgs pa = pc_args<float>(m);
      const float tc = time_it([&]() { cheb_launch<float>(c, m, pa, cc, x, x, y); });
      m.tune_us[mi * NT + ti] = ts;
      m.tune_us[(3 + mi) * NT + ti] = tc;
      if (ts < tb_s) { tb_s = ts; best_s[0] = mpl; best_s[1] = SCVS_TILES[ti]; }
      if (tc < tb_c) { tb_c = tc; best_c[0] = mpl; best_c[1] = SCVS_TILES[ti]; }
    }
  }
  m.mpl_spmm = best_s[0];
  m.tile_spmm = best_s[1];
  m.mpl_cheb = best_c[0];
  m.tile_cheb = best_c[1];
  // staged (shared-memory) variants: mode chunks 4, 8, 16, 32 of the row blocks
  int st_s = 0, st_c = 0;
  m.tune_us.resize(m.tune_us.size() + 8, 0.0f);
  const size_t st0 = (size_t)2 * 3 * NT;
  if (c.opts.stage >= 0) {
    for (int qi = 0; qi < 4; ++qi) {
      const int mc = 4 << qi;
      if (mc > m.ld) break;
      if (staged_ok(c, m, mc, true, x)) {
        m.st_spmm = mc;
        const float ts = time_it([&]() { apply_saddle<float>(c, m, x, y); });
        m.tune_us[st0 + qi] = ts;
        if (ts < tb_s) { tb_s = ts; st_s = mc; }
      }
      if (staged_ok(c, m, mc, false, x)) {
        m.st_cheb = mc;
        const PcArgs pa = pc_args<float>(m);
        const float tc = time_it([&]() { cheb_launch<float>(c, m, pa, cc, x, x, y); });
        m.tune_us[st0 + 4 + qi] = tc;
        if (tc < tb_c) { tb_c = tc; st_c = mc; }
      }
    }
  }
  m.st_spmm = st_s;
  m.st_cheb = st_c;
  if (c.opts.stage > 0) m.st_spmm = m.st_cheb = c.opts.stage;  // forced mode chunk
  c.timers.on = timers_on;
  SCVS_CUDA(cudaEventDestroy(e0));
  SCVS_CUDA(cudaEventDestroy(e1));
  for (void *p : {(void *)x, (void *)y, (void *)zeros}) SCVS_CUDA(cudaFreeAsync(p, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
}

}  // namespace scvs
