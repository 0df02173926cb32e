// Matrix-free application of the all-modes saddle operator A_hat(omega_k)
// (Eqs. linear_sys_def, LS_construction) without the assembled CSR values.
//
// For affine P2 simplices every element matrix is a combination of fixed
// reference matrices: M_e = det J * Mref, K_e = sum_p gamma_p(e) Ksym_p,
// D_e[c] = -det J sum_i (J^-1)_ic Eref_i (curved elements: the stored
// matrices).  Element by element: each element's matrices are formed once and
// applied to its gathered nodal block (every node, component and mode), so
// every gathered value serves the element's whole local matrix; elements are
// processed colour by colour (no two elements of a colour share a node), so
// their contributions are added with plain stores, without atomics, in a
// fixed order (results reproducible bit for bit).  The contraction has K = 10
// (P2 tet) per element row, far too thin for tensor cores at FP32/FP64
// accuracy, so it runs on CUDA-core FMAs.
#include <algorithm>
#include "scvs_internal.h"
#include "vecops.cuh"

namespace scvs {

// reference tables of both dimensions ([0]: triangles, [1]: tets)
__constant__ RefTables c_mf[2];

void matfree_tables(Ctx &c) {
  SCVS_CUDA(cudaMemcpyToSymbol(c_mf, &c.ref2, sizeof(RefTables), 0));
  SCVS_CUDA(cudaMemcpyToSymbol(c_mf, &c.ref3, sizeof(RefTables), sizeof(RefTables)));
}

template <typename T> struct MfArgs {
  int64_t N, P;
  int ld, nl;
  const int32_t *conn;
  const double *geom;
  const int32_t *cslot;        // curved elements: stored matrices (null: none)
  const double *CM, *CK, *CD;
  const uint8_t *dirmask;
  const double *omega;
  double rho, mu;
  const int32_t *el;           // elements of the current colour (ascending ids)
  int64_t n_el;
};

// y = x on the Dirichlet velocity rows (identity rows), 0 elsewhere: the
// element passes then add every element's contribution to the other rows.
template <typename T>
__global__ void k_matfree_init(const uint8_t *__restrict__ dirmask, int64_t N, int dim, int64_t total, int ld,
                               const typename cpx<T>::t *__restrict__ x, typename cpx<T>::t *__restrict__ y) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= total) return;
  const int64_t dof = f / ld;
  const bool dir = dof < N * dim && dirmask[dof / dim];
  y[f] = dir ? x[f] : mk<T>(0, 0);
}

// One colour of elements: no two of them share a node, so every element adds
// its contribution y_e = A_e x_e to its nodes' rows with plain loads and
// stores (no atomics; the colours run in a fixed order, so the sum over a
// node's elements has a fixed order too).  A row group of L lanes (lanes over
// modes) takes one element: it forms the element's K_e, M_e and D_e in shared
// memory (reference tables times geometric factors, or the stored matrices of
// a curved element), gathers the element's nodal block component by
// component, and contracts: velocity rows a (not Dirichlet) get
// mu (K_e u)_a + j omega rho (M_e u)_a + (D_e p)_a, pressure rows beta get
// sum_b D_e[b][beta] . u_b, Dirichlet columns b left out.
template <typename T, int MPL, int L, int DIM>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1)
k_matfree(const MfArgs<T> a, const typename cpx<T>::t *__restrict__ x, typename cpx<T>::t *__restrict__ y) {
  constexpr int NL = DIM == 2 ? 6 : 10, NV = DIM + 1, NP = DIM * (DIM + 1) / 2;
  constexpr int NE = 2 * NL * NL + DIM * NL * NV;  // K, M, D entries of one element
  constexpr int NR = NP * NL * NL + NL * NL + DIM * NL * NV;  // reference tables
  extern __shared__ unsigned char mf_raw[];
  // the reference tables first (the lanes of a group read different entries:
  // from shared memory instead of the constant cache, which serialises them)
  T *rK = reinterpret_cast<T *>(mf_raw), *rM = rK + NP * NL * NL, *rE = rM + NL * NL;
  for (int t = threadIdx.x; t < NR; t += blockDim.x) {
    T v;
    if (t < NP * NL * NL) v = (T)c_mf[DIM - 2].ksym[t / (NL * NL)][(t / NL) % NL][t % NL];
    else if (t < NP * NL * NL + NL * NL) v = (T)c_mf[DIM - 2].mref[(t - NP * NL * NL) / NL][(t - NP * NL * NL) % NL];
    else {
      const int tt = t - NP * NL * NL - NL * NL;
      v = (T)c_mf[DIM - 2].eref[tt / (NL * NV)][(tt / NV) % NL][tt % NV];
    }
    rK[t] = v;  // rK, rM, rE are consecutive
  }
  __syncthreads();
  T *sh = rK + NR;
  const int gpb = blockDim.x / L;
  const int lane = threadIdx.x % L, group = threadIdx.x / L;
  const unsigned gm = group_mask<L>();
  const int ld = a.ld, koff = lane * MPL;
  T *sK = sh + (size_t)group * NE, *sM = sK + NL * NL, *sD = sM + NL * NL;  // sD[c][aa][beta]
  T wr[MPL];
#pragma unroll
  for (int i = 0; i < MPL; ++i) wr[i] = (T)(a.omega[koff + i] * a.rho);
  const T mu = (T)a.mu;
  const auto *xp_base = x + (int64_t)DIM * a.N * ld + koff;
  auto *yp_base = y + (int64_t)DIM * a.N * ld + koff;
  for (int64_t q = (int64_t)blockIdx.x * gpb + group; q < a.n_el; q += (int64_t)gridDim.x * gpb) {
    const int64_t e = __ldg(a.el + q);
    int32_t cn[NL];
    bool dir[NL];
#pragma unroll
    for (int b = 0; b < NL; ++b) cn[b] = __ldg(a.conn + e * NL + b);
#pragma unroll
    for (int b = 0; b < NL; ++b) dir[b] = a.dirmask[cn[b]] != 0;
    const double *g = a.geom + e * GEOM_STRIDE;
    const int cs = a.cslot ? __ldg(a.cslot + e) : -1;
    const T det = (T)__ldg(g);
    // element matrices into shared memory, entries split over the group's lanes
    for (int t = lane; t < NE; t += L) {
      T v;
      if (t < NL * NL) {  // K
        const int aa = t / NL, b = t % NL;
        if (cs >= 0) {
          v = (T)__ldg(a.CK + ((int64_t)cs * NL + aa) * NL + b);
        } else {
          v = 0;
#pragma unroll
          for (int p = 0; p < NP; ++p) v += (T)__ldg(g + 10 + p) * rK[(p * NL + aa) * NL + b];
        }
      } else if (t < 2 * NL * NL) {  // M
        const int tt = t - NL * NL, aa = tt / NL, b = tt % NL;
        v = cs >= 0 ? (T)__ldg(a.CM + ((int64_t)cs * NL + aa) * NL + b) : det * rM[aa * NL + b];
      } else {  // D[c][aa][beta]
        const int tt = t - 2 * NL * NL, c = tt / (NL * NV), aa = (tt / NV) % NL, be = tt % NV;
        if (cs >= 0) {
          v = (T)__ldg(a.CD + (((int64_t)cs * DIM + c) * NL + aa) * NV + be);
        } else {
          T sacc = 0;
#pragma unroll
          for (int i = 0; i < DIM; ++i) sacc += (T)__ldg(g + 1 + i * DIM + c) * rE[(i * NL + aa) * NV + be];
          v = -det * sacc;
        }
      }
      sh[(size_t)group * NE + t] = v;
    }
    __syncwarp(gm);
    CV<T, MPL> pv[NV], yp[NV];
#pragma unroll
    for (int be = 0; be < NV; ++be) {
      ldv<T, MPL>(pv[be], xp_base + (int64_t)cn[be] * ld);
      yp[be].zero();
    }
#pragma unroll 1
    for (int c = 0; c < DIM; ++c) {  // one component at a time keeps the nodal block in registers
      CV<T, MPL> u[NL];
#pragma unroll
      for (int b = 0; b < NL; ++b) {
        if (dir[b]) u[b].zero();  // Dirichlet columns are removed
        else ldv<T, MPL>(u[b], x + ((int64_t)cn[b] * DIM + c) * ld + koff);
      }
      // pressure rows: sum_b D[c][b][beta] u_b
#pragma unroll
      for (int b = 0; b < NL; ++b)
#pragma unroll
        for (int be = 0; be < NV; ++be) axpy(yp[be], sD[(c * NL + b) * NV + be], u[b]);
      // velocity rows: the rows' current sums are loaded together (one round trip), then updated
      CV<T, MPL> yv[NL];
#pragma unroll
      for (int aa = 0; aa < NL; ++aa)
        if (!dir[aa]) ldv<T, MPL>(yv[aa], y + ((int64_t)cn[aa] * DIM + c) * ld + koff);
#pragma unroll
      for (int aa = 0; aa < NL; ++aa) {
        if (dir[aa]) continue;
        CV<T, MPL> aK, aM, aD;
        aK.zero(); aM.zero(); aD.zero();
#pragma unroll
        for (int b = 0; b < NL; ++b) {
          axpy(aK, sK[aa * NL + b], u[b]);
          axpy(aM, sM[aa * NL + b], u[b]);
        }
#pragma unroll
        for (int be = 0; be < NV; ++be) axpy(aD, sD[(c * NL + aa) * NV + be], pv[be]);
#pragma unroll
        for (int i = 0; i < MPL; ++i) {
          yv[aa].re[i] += mu * aK.re[i] - wr[i] * aM.im[i] + aD.re[i];
          yv[aa].im[i] += mu * aK.im[i] + wr[i] * aM.re[i] + aD.im[i];
        }
        stv<T, MPL>(y + ((int64_t)cn[aa] * DIM + c) * ld + koff, yv[aa]);
      }
    }
    CV<T, MPL> po[NV];
#pragma unroll
    for (int be = 0; be < NV; ++be) ldv<T, MPL>(po[be], yp_base + (int64_t)cn[be] * ld);
#pragma unroll
    for (int be = 0; be < NV; ++be) {
#pragma unroll
      for (int i = 0; i < MPL; ++i) { po[be].re[i] += yp[be].re[i]; po[be].im[i] += yp[be].im[i]; }
      stv<T, MPL>(yp_base + (int64_t)cn[be] * ld, po[be]);
    }
    __syncwarp(gm);  // the group's shared matrices are rewritten for its next element
  }
}

// Colours of the elements for the element passes (host greedy, once per mesh):
// elements in ascending id take the lowest colour that no element sharing one
// of their nodes holds yet.  The elements are then listed colour by colour,
// ascending ids within a colour.
static void matfree_colours(Ctx &c, Mesh &m) {
  const int64_t E = m.E;
  const int nl = m.nl;
  std::vector<int32_t> conn((size_t)std::max<int64_t>(E, 1) * nl);
  SCVS_CUDA(cudaMemcpyAsync(conn.data(), m.conn, (size_t)E * nl * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  constexpr int W = 4;  // 256 colours at most
  std::vector<uint64_t> used((size_t)m.N * W, 0);
  std::vector<int16_t> col(std::max<int64_t>(E, 1), -1);
  int n_col = 0;
  for (int64_t e = 0; e < E; ++e) {
    uint64_t u[W] = {0, 0, 0, 0};
    for (int b = 0; b < nl; ++b)
      for (int w = 0; w < W; ++w) u[w] |= used[(size_t)conn[(size_t)e * nl + b] * W + w];
    int k = -1;
    for (int w = 0; w < W && k < 0; ++w)
      if (~u[w]) k = w * 64 + __builtin_ctzll(~u[w]);
    if (k < 0) throw (int)SCVS_ERR_STATE;  // more than 256 colours: not a simplex mesh of bounded degree
    col[e] = (int16_t)k;
    n_col = std::max(n_col, k + 1);
    for (int b = 0; b < nl; ++b) used[(size_t)conn[(size_t)e * nl + b] * W + k / 64] |= 1ull << (k % 64);
  }
  std::vector<int64_t> ptr(n_col + 1, 0);
  for (int64_t e = 0; e < E; ++e) ++ptr[col[e] + 1];
  for (int k = 0; k < n_col; ++k) ptr[k + 1] += ptr[k];
  std::vector<int32_t> list(std::max<int64_t>(E, 1));
  {
    std::vector<int64_t> fill(ptr.begin(), ptr.end() - 1);
    for (int64_t e = 0; e < E; ++e) list[fill[col[e]]++] = (int32_t)e;
  }
  m.mf_col_ptr = ptr;
  m.mf_el = m.arena.alloc<int32_t>(std::max<int64_t>(E, 1));
  SCVS_CUDA(cudaMemcpyAsync(m.mf_el, list.data(), (size_t)E * sizeof(int32_t), cudaMemcpyHostToDevice, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));  // the host list goes out of scope
}

#define SCVS_MF_DISPATCH(ld, ...)                                                        \
  do {                                                                                   \
    switch (ld) {                                                                        \
      SCVS_LD_CASE(2, 1, __VA_ARGS__) SCVS_LD_CASE(4, 1, __VA_ARGS__)                   \
      SCVS_LD_CASE(8, 1, __VA_ARGS__) SCVS_LD_CASE(16, 1, __VA_ARGS__)                  \
      SCVS_LD_CASE(32, 1, __VA_ARGS__) SCVS_LD_CASE(64, 2, __VA_ARGS__)                 \
      SCVS_LD_CASE(128, 4, __VA_ARGS__)                                                  \
      default: throw (int)SCVS_ERR_ARG;                                                  \
    }                                                                                    \
  } while (0)

template <typename T>
static void launch_matfree(Ctx &c, Mesh &m, const void *x, void *y) {
  using C = typename cpx<T>::t;
  if (m.mf_col_ptr.empty()) matfree_colours(c, m);
  const int64_t total = m.n_dof * m.ld;
  // algorithmic bytes: connectivity, geometry and the element list once, x read once, y written once
  KScope ks(c, KC_MATFREE, (double)m.E * (m.nl * 4 + GEOM_STRIDE * 8 + 4) + 2.0 * total * 2 * sizeof(T));
  k_matfree_init<T><<<ceil_div(total, 256), 256, 0, c.stream>>>(m.dirmask, m.N, m.dim, total, m.ld,
                                                                static_cast<const C *>(x), static_cast<C *>(y));
  count_launch(c);
  MfArgs<T> a{m.N, m.P, m.ld, m.nl, m.conn, m.geom, m.cslot, m.CM, m.CK, m.CD, m.dirmask, m.omega_d, m.rho, m.mu,
              nullptr, 0};
  const int n_col = (int)m.mf_col_ptr.size() - 1;
  for (int k = 0; k < n_col; ++k) {
    a.el = m.mf_el + m.mf_col_ptr[k];
    a.n_el = m.mf_col_ptr[k + 1] - m.mf_col_ptr[k];
    if (a.n_el == 0) continue;
    // one mode per lane up to 32 modes (the element's nodal block of one
    // component then takes 20 registers per lane), at most 16 groups per
    // block (their element matrices and the tables stay under 48 KB)
    SCVS_MF_DISPATCH(m.ld, {
      const int gpb = std::min(256 / L, 16), threads = gpb * L;
      const int nv = m.dim + 1, np = m.dim * (m.dim + 1) / 2;
      const int ne = 2 * m.nl * m.nl + m.dim * m.nl * nv, nr = np * m.nl * m.nl + m.nl * m.nl + m.dim * m.nl * nv;
      const size_t smem = (size_t)(gpb * ne + nr) * sizeof(T);
      const unsigned nb = (unsigned)std::max<int64_t>(1, (a.n_el + gpb - 1) / gpb);
      if (m.dim == 2)
        k_matfree<T, MPL, L, 2><<<nb, threads, smem, c.stream>>>(a, static_cast<const C *>(x), static_cast<C *>(y));
      else
        k_matfree<T, MPL, L, 3><<<nb, threads, smem, c.stream>>>(a, static_cast<const C *>(x), static_cast<C *>(y));
    });
    count_launch(c);
  }
}

void apply_matfree(Ctx &c, Mesh &m, int precision, const void *x, void *y) {
  if (precision == SCVS_PREC_FP64)
    launch_matfree<double>(c, m, x, y);
  else
    launch_matfree<float>(c, m, x, y);
}

}  // namespace scvs
