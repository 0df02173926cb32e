// Matrix-free application of the all-modes saddle operator A_hat(omega_k)
// (Eqs. linear_sys_def, LS_construction) without the assembled CSR values.
//
// For affine P2 simplices every element matrix is a combination of fixed
// reference matrices: M_e = det J * Mref, K_e = sum_p gamma_p(e) Ksym_p,
// D_e[c] = -det J sum_i (J^-1)_ic Eref_i.  A row group of L lanes (lanes over
// modes) owns one row; it walks the row's incident elements in ascending id
// order, forms the element-matrix row of its local node from the element's
// geometric factors and the reference tables, and contracts it with the
// gathered nodal block x_e (every node of the element, every component, every
// mode).  Owner-computes: no atomics, the summation order is fixed, results
// are reproducible bit for bit.  The contraction has K = 10 (P2 tet) per
// element and row, far too thin for tensor cores at FP32/FP64 accuracy, so it
// runs on CUDA-core FMAs.
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
  const int64_t *n2e_ptr;
  const int32_t *n2e;
  const int32_t *conn;
  const double *geom;
  const int32_t *cslot;        // curved elements: stored matrices (null: none)
  const double *CM, *CK, *CD;
  const uint8_t *dirmask;
  const double *omega;
  double rho, mu;
};

template <typename T, int MPL, int L, int DIM>
__global__ void __launch_bounds__(256)
k_matfree(const MfArgs<T> a, const typename cpx<T>::t *__restrict__ x, typename cpx<T>::t *__restrict__ y) {
  constexpr int NL = DIM == 2 ? 6 : 10, NV = DIM + 1, NP = DIM * (DIM + 1) / 2;
  const int gpb = blockDim.x / L;
  const int lane = threadIdx.x % L, group = threadIdx.x / L;
  const int ld = a.ld, koff = lane * MPL;
  T wr[MPL];
#pragma unroll
  for (int i = 0; i < MPL; ++i) wr[i] = (T)(a.omega[koff + i] * a.rho);
  const T mu = (T)a.mu;
  const auto *xp_base = x + (int64_t)DIM * a.N * ld + koff;
  for (int64_t row = (int64_t)blockIdx.x * gpb + group; row < a.N + a.P; row += (int64_t)gridDim.x * gpb) {
    const bool vel = row < a.N;
    const int64_t node = vel ? row : row - a.N;
    if (vel && a.dirmask[node]) {
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        CV<T, MPL> v;
        ldv<T, MPL>(v, x + (node * DIM + c) * ld + koff);
        stv<T, MPL>(y + (node * DIM + c) * ld + koff, v);
      }
      continue;
    }
    CV<T, MPL> aK[DIM], aM[DIM], aD[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) { aK[c].zero(); aM[c].zero(); aD[c].zero(); }
    for (int64_t ei = a.n2e_ptr[node]; ei < a.n2e_ptr[node + 1]; ++ei) {
      const int64_t e = __ldg(a.n2e + ei);
      int32_t cn[NL];
      int loc = 0;
#pragma unroll
      for (int b = 0; b < NL; ++b) {
        cn[b] = __ldg(a.conn + e * NL + b);
        if (cn[b] == (int32_t)node) loc = b;
      }
      const double *g = a.geom + e * GEOM_STRIDE;
      const int cs = a.cslot ? __ldg(a.cslot + e) : -1;
      const T det = (T)__ldg(g);
      T ji[DIM][DIM], ga[NP];
#pragma unroll
      for (int i = 0; i < DIM; ++i)
#pragma unroll
        for (int c = 0; c < DIM; ++c) ji[i][c] = (T)__ldg(g + 1 + i * DIM + c);
#pragma unroll
      for (int p = 0; p < NP; ++p) ga[p] = (T)__ldg(g + 10 + p);
      if (vel) {
        const int aa = loc;
#pragma unroll
        for (int b = 0; b < NL; ++b) {
          if (a.dirmask[cn[b]]) continue;  // Dirichlet columns are removed
          T kc = 0, mc;
          if (cs >= 0) {
            kc = (T)__ldg(a.CK + ((int64_t)cs * NL + aa) * NL + b);
            mc = (T)__ldg(a.CM + ((int64_t)cs * NL + aa) * NL + b);
          } else {
#pragma unroll
            for (int p = 0; p < NP; ++p) kc += ga[p] * (T)c_mf[DIM - 2].ksym[p][aa][b];
            mc = det * (T)c_mf[DIM - 2].mref[aa][b];
          }
#pragma unroll
          for (int c = 0; c < DIM; ++c) {
            CV<T, MPL> xv;
            ldv<T, MPL>(xv, x + ((int64_t)cn[b] * DIM + c) * ld + koff);
            axpy(aK[c], kc, xv);
            axpy(aM[c], mc, xv);
          }
        }
#pragma unroll
        for (int b = 0; b < NV; ++b) {
          CV<T, MPL> xq;
          ldv<T, MPL>(xq, xp_base + (int64_t)cn[b] * ld);
#pragma unroll
          for (int c = 0; c < DIM; ++c) {
            T dc;
            if (cs >= 0) {
              dc = (T)__ldg(a.CD + (((int64_t)cs * DIM + c) * NL + aa) * NV + b);
            } else {
              T s = 0;
#pragma unroll
              for (int i = 0; i < DIM; ++i) s += ji[i][c] * (T)c_mf[DIM - 2].eref[i][aa][b];
              dc = -det * s;
            }
            axpy(aD[c], dc, xq);
          }
        }
      } else {
        const int beta = loc;  // vertex: local index < NV
#pragma unroll
        for (int b = 0; b < NL; ++b) {
          if (a.dirmask[cn[b]]) continue;
#pragma unroll
          for (int c = 0; c < DIM; ++c) {
            T dc;
            if (cs >= 0) {
              dc = (T)__ldg(a.CD + (((int64_t)cs * DIM + c) * NL + b) * NV + beta);
            } else {
              T s = 0;
#pragma unroll
              for (int i = 0; i < DIM; ++i) s += ji[i][c] * (T)c_mf[DIM - 2].eref[i][b][beta];
              dc = -det * s;
            }
            CV<T, MPL> xv;
            ldv<T, MPL>(xv, x + ((int64_t)cn[b] * DIM + c) * ld + koff);
            axpy(aD[0], dc, xv);
          }
        }
      }
    }
    if (vel) {
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        CV<T, MPL> o;
#pragma unroll
        for (int i = 0; i < MPL; ++i) {
          o.re[i] = mu * aK[c].re[i] - wr[i] * aM[c].im[i] + aD[c].re[i];
          o.im[i] = mu * aK[c].im[i] + wr[i] * aM[c].re[i] + aD[c].im[i];
        }
        stv<T, MPL>(y + (node * DIM + c) * ld + koff, o);
      }
    } else {
      stv<T, MPL>(y + ((int64_t)DIM * a.N + node) * ld + koff, aD[0]);
    }
  }
}

template <typename T>
static void launch_matfree(Ctx &c, const Mesh &m, const void *x, void *y) {
  using C = typename cpx<T>::t;
  MfArgs<T> a{m.N, m.P, m.ld, m.nl, m.n2e_ptr, m.n2e, m.conn, m.geom, m.cslot, m.CM, m.CK, m.CD,
              m.dirmask, m.omega_d, m.rho, m.mu};
  // algorithmic bytes: connectivity, geometry and incidence once, x read once, y written once
  KScope ks(c, KC_MATFREE, (double)m.E * (m.nl * 4 + GEOM_STRIDE * 8) + (double)m.E * m.nl * 4 + (double)(m.N + 1) * 8 +
                               2.0 * m.n_dof * m.ld * 2 * sizeof(T));
  SCVS_DISPATCH_LD(T, m.ld, {
    const int gpb = 256 / L;
    int64_t need = (m.N + m.P + gpb - 1) / gpb;
    const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(need, (int64_t)c.num_sms * 32));
    if (m.dim == 2)
      k_matfree<T, MPL, L, 2><<<nb, 256, 0, c.stream>>>(a, static_cast<const C *>(x), static_cast<C *>(y));
    else
      k_matfree<T, MPL, L, 3><<<nb, 256, 0, c.stream>>>(a, static_cast<const C *>(x), static_cast<C *>(y));
  });
  count_launch(c);
}

void apply_matfree(Ctx &c, const Mesh &m, int precision, const void *x, void *y) {
  if (precision == SCVS_PREC_FP64)
    launch_matfree<double>(c, m, x, y);
  else
    launch_matfree<float>(c, m, x, y);
}

}  // namespace scvs
