// GPU construction of the sparsity patterns and of the mode-independent real
// matrices of the SCVS saddle-point system (Eqs. linear_sys_def, LS_construction).
//
//   1. per element: validation, affine map, det J, J^-1, gamma = det J^-1 J^-T
//   2. node -> element incidence (count, scan, fill, per-node sort)
//   3. S pattern, one warp per row: gather the nodes of every incident element,
//      bitonic sort in shared memory, drop duplicates -> ascending columns
//      (counted in a first pass, written in a second)
//   4. values, one warp per row: incident elements in ascending id order, the
//      lanes take the element's local columns (distinct positions), so every
//      entry is summed in the same order on every run (deterministic)
//   5. Dirichlet masking, FP32 copies and diagonals
#include <algorithm>
#include <array>
#include <climits>
#include <cmath>
#include <map>
#include "scvs_internal.h"

namespace scvs {

__constant__ RefTables c_ref;

// --------------------------------------------------------------- geometry
__global__ void k_geom(const double *__restrict__ xyz, const int32_t *__restrict__ conn, int64_t E,
                       int nl, int dim, int64_t N, int64_t P, double *__restrict__ geom, int *err) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int32_t *c = conn + e * nl;
  int bad = 0;
  for (int a = 0; a < nl; ++a) {
    int32_t v = c[a];
    if (v < 0 || v >= N) bad |= DEVERR_BAD_NODE;
    if (a <= dim && (v < 0 || v >= P)) bad |= DEVERR_BAD_VERTEX;
    if (a > dim && v < P) bad |= DEVERR_BAD_VERTEX;
    for (int b = 0; b < a; ++b)
      if (c[b] == v) bad |= DEVERR_DUP_NODE;
  }
  if (bad) { atomicOr(err, bad); return; }
  double *g = geom + e * GEOM_STRIDE;
  double J[3][3] = {{0}};
  for (int i = 0; i < dim; ++i)
    for (int r = 0; r < dim; ++r) J[r][i] = xyz[(int64_t)c[i + 1] * dim + r] - xyz[(int64_t)c[0] * dim + r];
  double det, Ji[3][3] = {{0}};
  if (dim == 2) {
    det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
    double id = 1.0 / det;
    Ji[0][0] = J[1][1] * id; Ji[0][1] = -J[0][1] * id;
    Ji[1][0] = -J[1][0] * id; Ji[1][1] = J[0][0] * id;
  } else {
    double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    double id = 1.0 / det;
    Ji[0][0] = c00 * id;
    Ji[1][0] = c01 * id;
    Ji[2][0] = c02 * id;
    Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id;
    Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id;
    Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id;
    Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
    Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
    Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
  }
  if (!(det > 0.0)) { atomicOr(err, DEVERR_JACOBIAN); return; }
  g[0] = det;
  for (int i = 0; i < dim; ++i)
    for (int k = 0; k < dim; ++k) g[1 + i * dim + k] = Ji[i][k];
  int p = 0;
  for (int i = 0; i < dim; ++i)
    for (int j = i; j < dim; ++j, ++p) {
      double s = 0;
      for (int k = 0; k < dim; ++k) s += Ji[i][k] * Ji[j][k];
      g[10 + p] = det * s;
    }
}

// ------------------------------------------------------ curved elements
// An element is curved (isoparametric) if one of its edge nodes is not at its
// edge's midpoint (relative tolerance 1e-12 of the edge length): the paper
// projects inserted boundary nodes onto curved walls (Sec. 3.1).
__global__ void k_curved_flag(const double *__restrict__ xyz, const int32_t *__restrict__ conn, int64_t E, int nl,
                              int dim, int32_t *__restrict__ flag) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int32_t *c = conn + e * nl;
  const int ne = dim == 2 ? 3 : 6;
  const int EA[6] = {0, 1, 2, 0, 1, 2}, EB[6] = {1, 2, 0, 3, 3, 3};
  int curved = 0;
  for (int j = 0; j < ne; ++j) {
    const double *xa = xyz + (int64_t)c[EA[j]] * dim, *xb = xyz + (int64_t)c[EB[j]] * dim;
    const double *xm = xyz + (int64_t)c[dim + 1 + j] * dim;
    double dev = 0.0, len = 0.0;
    for (int r = 0; r < dim; ++r) {
      const double d = xm[r] - 0.5 * (xa[r] + xb[r]), l = xb[r] - xa[r];
      dev += d * d;
      len += l * l;
    }
    if (dev > 1e-24 * len) curved = 1;
  }
  flag[e] = curved;
}

__global__ void k_curved_slot(const int32_t *__restrict__ flag, const int64_t *__restrict__ scan, int64_t E,
                              int32_t *__restrict__ slot) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e < E) slot[e] = flag[e] ? (int32_t)scan[e] : -1;
}

// Element matrices of the curved elements by quadrature of the isoparametric
// map x(xi) = sum_a x_a phi_a(xi): at every point J = sum_a x_a grad_xi phi_a^T,
// grad_x phi_a = J^-T grad_xi phi_a, and
//   CM[a][b] += w |J| phi_a phi_b,  CK[a][b] += w |J| grad_x phi_a . grad_x phi_b,
//   CD[c][a][b] += -w |J| d_c phi_a psi_b.
// One warp per element, lanes over the (a, b) pairs.
template <int DIM>
__global__ void __launch_bounds__(128) k_curved_mats(const double *__restrict__ xyz, const int32_t *__restrict__ conn,
                                                     const int32_t *__restrict__ slot, int64_t E,
                                                     const QuadTables *__restrict__ qt, double *__restrict__ CM,
                                                     double *__restrict__ CK, double *__restrict__ CD, int *err) {
  constexpr int NL = DIM == 2 ? 6 : 10, NV = DIM + 1, PPL = (NL * NL + 31) / 32;
  __shared__ double X[4][NL][DIM];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int64_t e = (int64_t)blockIdx.x * 4 + warp; e < E; e += (int64_t)gridDim.x * 4) {
    const int s = slot[e];
    if (s < 0) continue;  // warp-uniform
    if (lane < NL)
      for (int r = 0; r < DIM; ++r) X[warp][lane][r] = xyz[(int64_t)conn[e * NL + lane] * DIM + r];
    __syncwarp();
    double am[PPL], ak[PPL], ad[PPL][DIM];
#pragma unroll
    for (int u = 0; u < PPL; ++u) {
      am[u] = ak[u] = 0.0;
#pragma unroll
      for (int c = 0; c < DIM; ++c) ad[u][c] = 0.0;
    }
    bool bad = false;
    for (int q = 0; q < qt->nq; ++q) {
      double J[DIM][DIM];
#pragma unroll
      for (int r = 0; r < DIM; ++r)
#pragma unroll
        for (int i = 0; i < DIM; ++i) {
          double v = 0.0;
#pragma unroll
          for (int a = 0; a < NL; ++a) v += X[warp][a][r] * __ldg(&qt->dphi[q][a][i]);
          J[r][i] = v;
        }
      double det, Ji[DIM][DIM];  // Ji[i][r] = (J^-1)_{i r}
      if (DIM == 2) {
        det = J[0][0] * J[1][1] - J[0][1] * J[1][0];
        Ji[0][0] = J[1][1] / det; Ji[0][1] = -J[0][1] / det;
        Ji[1][0] = -J[1][0] / det; Ji[1][1] = J[0][0] / det;
      } else {
        const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
        const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
        const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
        det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
        Ji[0][0] = c00 / det;
        Ji[1][0] = c01 / det;
        Ji[2][0] = c02 / det;
        Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
        Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
        Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
        Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
        Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
        Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
      }
      if (!(det > 0.0)) bad = true;
      const double wd = __ldg(&qt->w[q]) * det;
#pragma unroll
      for (int u = 0; u < PPL; ++u) {
        const int pr = lane + 32 * u;
        if (pr >= NL * NL) break;
        const int a = pr / NL, b = pr % NL;
        double ga[DIM], gb[DIM];
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          double va = 0.0, vb = 0.0;
#pragma unroll
          for (int i = 0; i < DIM; ++i) {
            va += __ldg(&qt->dphi[q][a][i]) * Ji[i][c];
            vb += __ldg(&qt->dphi[q][b][i]) * Ji[i][c];
          }
          ga[c] = va;
          gb[c] = vb;
        }
        am[u] += wd * __ldg(&qt->phi[q][a]) * __ldg(&qt->phi[q][b]);
        double kd = 0.0;
#pragma unroll
        for (int c = 0; c < DIM; ++c) kd += ga[c] * gb[c];
        ak[u] += wd * kd;
        if (b < NV) {
          const double pb = __ldg(&qt->psi[q][b]);
#pragma unroll
          for (int c = 0; c < DIM; ++c) ad[u][c] -= wd * ga[c] * pb;
        }
      }
    }
    if (bad && lane == 0) atomicOr(err, DEVERR_JACOBIAN);
#pragma unroll
    for (int u = 0; u < PPL; ++u) {
      const int pr = lane + 32 * u;
      if (pr >= NL * NL) break;
      const int a = pr / NL, b = pr % NL;
      CM[(int64_t)s * NL * NL + pr] = am[u];
      CK[(int64_t)s * NL * NL + pr] = ak[u];
      if (b < NV)
#pragma unroll
        for (int c = 0; c < DIM; ++c) CD[((int64_t)s * DIM + c) * NL * NV + a * NV + b] = ad[u][c];
    }
    __syncwarp();
  }
}

// -------------------------------------------------------------- incidence
__global__ void k_count_incidence(const int32_t *__restrict__ conn, int64_t total, int32_t *cnt) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < total) atomicAdd(&cnt[conn[t]], 1);
}

__global__ void k_fill_incidence(const int32_t *__restrict__ conn, int64_t E, int nl,
                                 const int64_t *__restrict__ ptr, int32_t *fill, int32_t *n2e) {
  int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= E * nl) return;
  int32_t node = conn[t];
  int pos = atomicAdd(&fill[node], 1);
  n2e[ptr[node] + pos] = (int32_t)(t / nl);
}

// insertion sort of every node's (short) element list
__global__ void k_sort_incidence(const int64_t *__restrict__ ptr, int32_t *n2e, int64_t N, int *err) {
  int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (v >= N) return;
  int64_t b = ptr[v], e = ptr[v + 1];
  if (e == b) atomicOr(err, DEVERR_BAD_NODE);  // a node no element uses
  for (int64_t i = b + 1; i < e; ++i) {
    int32_t key = n2e[i];
    int64_t j = i - 1;
    while (j >= b && n2e[j] > key) { n2e[j + 1] = n2e[j]; --j; }
    n2e[j + 1] = key;
  }
}

// ---------------------------------------------------------------- pattern
constexpr int PAT_CAP = 2048;   // candidate slots per warp (incident elements x nl)
constexpr int PAT_WARPS = 4;

__device__ __forceinline__ int next_pow2(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

template <bool WRITE>
__global__ void __launch_bounds__(PAT_WARPS * 32)
k_row_pattern(const int64_t *__restrict__ n2e_ptr, const int32_t *__restrict__ n2e,
              const int32_t *__restrict__ conn, int nl, int64_t N, int64_t P,
              int32_t *__restrict__ s_len, int32_t *__restrict__ g_len,
              const int64_t *__restrict__ s_ptr, int32_t *__restrict__ s_col, int *err) {
  __shared__ int sbuf[PAT_WARPS][PAT_CAP];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int *buf = sbuf[warp];
  for (int64_t row = (int64_t)blockIdx.x * PAT_WARPS + warp; row < N; row += (int64_t)gridDim.x * PAT_WARPS) {
    const int64_t e0 = n2e_ptr[row], e1 = n2e_ptr[row + 1];
    const int count = (int)(e1 - e0) * nl;
    if (count > PAT_CAP) {
      if (lane == 0) atomicOr(err, DEVERR_VALENCE);
      continue;
    }
    const int n2 = next_pow2(count > 0 ? count : 1);
    for (int t = lane; t < n2; t += 32)
      buf[t] = t < count ? conn[(int64_t)n2e[e0 + t / nl] * nl + t % nl] : INT_MAX;
    __syncwarp();
    for (int k = 2; k <= n2; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int t = lane; t < n2; t += 32) {
          int u = t ^ j;
          if (u > t) {
            int a = buf[t], b = buf[u];
            bool up = (t & k) == 0;
            if ((a > b) == up) { buf[t] = b; buf[u] = a; }
          }
        }
        __syncwarp();
      }
    int running = 0, gcount = 0;
    const int64_t base_out = WRITE ? s_ptr[row] : 0;
    for (int base = 0; base < n2; base += 32) {
      int t = base + lane;
      int v = t < n2 ? buf[t] : INT_MAX;
      bool flag = (t < n2) && v != INT_MAX && (t == 0 || buf[t - 1] != v);
      unsigned bal = __ballot_sync(0xffffffffu, flag);
      unsigned gbal = __ballot_sync(0xffffffffu, flag && v < P);
      if (WRITE && flag) s_col[base_out + running + __popc(bal & ((1u << lane) - 1u))] = v;
      running += __popc(bal);
      gcount += __popc(gbal);
    }
    if (!WRITE && lane == 0) {
      s_len[row] = running;
      g_len[row] = gcount;
    }
    __syncwarp();
  }
}

__global__ void k_max_int(const int32_t *__restrict__ v, int64_t n, int *out) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int m = 0;
  for (; i < n; i += (int64_t)gridDim.x * blockDim.x) m = max(m, v[i]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// ------------------------------------------------------------------ values
// Shared-memory row accumulators of one warp: cols[cap] + acc[nacc][cap] doubles.
constexpr int ASM_WARPS = 2;

__global__ void __launch_bounds__(ASM_WARPS * 32)
k_assemble_rows(const int64_t *__restrict__ n2e_ptr, const int32_t *__restrict__ n2e,
                const int32_t *__restrict__ conn, const double *__restrict__ geom, int nl, int dim,
                int64_t N, int64_t P, const int64_t *__restrict__ s_ptr, const int32_t *__restrict__ s_col,
                const int32_t *__restrict__ g_len, const int64_t *__restrict__ g_ptr, int cap,
                int64_t g_nnz, int64_t gt_nnz, double *__restrict__ Ms, double *__restrict__ Ks,
                double *__restrict__ Dv, double *__restrict__ DTv, double *__restrict__ Mp,
                double *__restrict__ Lp, const int32_t *__restrict__ cslot, const double *__restrict__ CM,
                const double *__restrict__ CK, const double *__restrict__ CD, int *err) {
  extern __shared__ double smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // per warp: acc[10][cap] doubles, cols[cap] ints
  const int NACC = 10;  // M, K, D0..2, DT0..2, Mp, Lp
  double *acc = smem + (size_t)warp * (NACC * cap + cap / 2 + 1);
  int *cols = reinterpret_cast<int *>(acc + NACC * cap);
  const int nv = dim + 1;
  const int npair = dim * (dim + 1) / 2;
  for (int64_t row = (int64_t)blockIdx.x * ASM_WARPS + warp; row < N; row += (int64_t)gridDim.x * ASM_WARPS) {
    const int64_t r0 = s_ptr[row];
    const int len = (int)(s_ptr[row + 1] - r0);
    const int glen = g_len[row];
    for (int t = lane; t < len; t += 32) {
      cols[t] = s_col[r0 + t];
      for (int q = 0; q < NACC; ++q) acc[q * cap + t] = 0.0;
    }
    __syncwarp();
    const bool is_vertex = row < P;
    for (int64_t ei = n2e_ptr[row]; ei < n2e_ptr[row + 1]; ++ei) {
      const int64_t e = n2e[ei];
      const int32_t myc = lane < nl ? conn[e * nl + lane] : -1;
      const unsigned hit = __ballot_sync(0xffffffffu, myc == (int32_t)row);
      const int a = __ffs(hit) - 1;
      const double *g = geom + e * GEOM_STRIDE;
      if (a < 0 || (is_vertex && a >= nv)) {  // incidence list inconsistent with conn
        if (lane == 0) atomicOr(err, DEVERR_BAD_VERTEX);
        __syncwarp();
        continue;
      }
      if (lane < nl) {
        const int b = lane;
        // binary search of the column position
        int lo = 0, hi = len - 1, pos = -1;
        while (lo <= hi) {
          int mid = (lo + hi) >> 1;
          int cv = cols[mid];
          if (cv == myc) { pos = mid; break; }
          if (cv < myc) lo = mid + 1; else hi = mid - 1;
        }
        const int cs = cslot ? cslot[e] : -1;  // curved element: stored isoparametric matrices
        if (pos < 0) {
          atomicOr(err, DEVERR_BAD_NODE);
        } else if (cs >= 0) {
          acc[0 * cap + pos] += CM[((int64_t)cs * nl + a) * nl + b];
          acc[1 * cap + pos] += CK[((int64_t)cs * nl + a) * nl + b];
          if (b < nv)
            for (int cc = 0; cc < dim; ++cc) acc[(2 + cc) * cap + pos] += CD[(((int64_t)cs * dim + cc) * nl + a) * nv + b];
          if (is_vertex) {
            for (int cc = 0; cc < dim; ++cc) acc[(5 + cc) * cap + pos] += CD[(((int64_t)cs * dim + cc) * nl + b) * nv + a];
            if (b < nv) {  // the preconditioner's P1 operators keep the straight simplex of the vertices
              const double det = g[0];
              acc[8 * cap + pos] += det * c_ref.m1[a][b];
              double lv = 0.0;
              for (int p = 0; p < npair; ++p) lv += g[10 + p] * c_ref.k1sym[p][a][b];
              acc[9 * cap + pos] += lv;
            }
          }
        } else {
          const double det = g[0];
          acc[0 * cap + pos] += det * c_ref.mref[a][b];
          double kv = 0.0;
          for (int p = 0; p < npair; ++p) kv += g[10 + p] * c_ref.ksym[p][a][b];
          acc[1 * cap + pos] += kv;
          if (b < nv) {
            for (int cc = 0; cc < dim; ++cc) {
              double s = 0.0;
              for (int i = 0; i < dim; ++i) s += g[1 + i * dim + cc] * c_ref.eref[i][a][b];
              acc[(2 + cc) * cap + pos] += -det * s;
            }
          }
          if (is_vertex) {
            for (int cc = 0; cc < dim; ++cc) {
              double s = 0.0;
              for (int i = 0; i < dim; ++i) s += g[1 + i * dim + cc] * c_ref.eref[i][b][a];
              acc[(5 + cc) * cap + pos] += -det * s;
            }
            if (b < nv) {
              acc[8 * cap + pos] += det * c_ref.m1[a][b];
              double lv = 0.0;
              for (int p = 0; p < npair; ++p) lv += g[10 + p] * c_ref.k1sym[p][a][b];
              acc[9 * cap + pos] += lv;
            }
          }
        }
      }
      __syncwarp();
    }
    const int64_t gp = g_ptr[row];
    for (int t = lane; t < len; t += 32) {
      Ms[r0 + t] = acc[0 * cap + t];
      Ks[r0 + t] = acc[1 * cap + t];
      if (t < glen)
        for (int cc = 0; cc < dim; ++cc) Dv[cc * g_nnz + gp + t] = acc[(2 + cc) * cap + t];
      if (is_vertex) {
        for (int cc = 0; cc < dim; ++cc) DTv[cc * gt_nnz + r0 + t] = acc[(5 + cc) * cap + t];
        if (t < glen) {
          Mp[gp + t] = acc[8 * cap + t];
          Lp[gp + t] = acc[9 * cap + t];
        }
      }
    }
    __syncwarp();
  }
}

// ------------------------------------------------------- masks and copies
__global__ void k_masks(const uint8_t *__restrict__ tag, int64_t N, int64_t P, uint8_t *dirmask, uint8_t *outmask) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= N) return;
  dirmask[i] = (tag[i] & (SCVS_TAG_WALL | SCVS_TAG_INLET)) ? 1 : 0;
  if (i < P) outmask[i] = (tag[i] & SCVS_TAG_OUTLET) ? 1 : 0;
}

__global__ void k_mask_values(int64_t N, int64_t P, int dim, const int64_t *__restrict__ s_ptr,
                              const int32_t *__restrict__ s_col, const int32_t *__restrict__ g_len,
                              const int64_t *__restrict__ g_ptr, int64_t g_nnz, int64_t gt_nnz,
                              const uint8_t *__restrict__ dirm, const uint8_t *__restrict__ outm,
                              const double *Ms, const double *Ks, const double *Dv, const double *DTv,
                              const double *Mp, const double *Lp, double *Ms_m, double *Ks_m,
                              double *Dv_m, double *DTv_m, double *Lp_m, float *Ms_f, float *Ks_f,
                              float *Dv_f, float *DTv_f, float *Mp_f, float *Lp_f, double *ms_diag,
                              double *ks_diag, double *mp_diag, double *lp_diag, float *Kc_f, float *Mc_f,
                              double *k1_diag, double *Kc_m, double *Mc_m) {
  int64_t A = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (A >= N) return;
  const bool dA = dirm[A];
  const int64_t r0 = s_ptr[A], r1 = s_ptr[A + 1], gp = g_ptr[A];
  const int glen = g_len[A];
  for (int64_t t = r0; t < r1; ++t) {
    const int32_t B = s_col[t];
    const bool keep = !dA && !dirm[B];
    double ms = keep ? Ms[t] : 0.0, ks = keep ? Ks[t] : 0.0;
    Ms_m[t] = ms; Ks_m[t] = ks;
    Ms_f[t] = (float)ms; Ks_f[t] = (float)ks;
    if (B == A) { ms_diag[A] = Ms[t]; ks_diag[A] = Ks[t]; }
    if (A < P)
      for (int c = 0; c < dim; ++c) {
        double v = dirm[B] ? 0.0 : DTv[c * gt_nnz + t];
        DTv_m[c * gt_nnz + t] = v;
        DTv_f[c * gt_nnz + t] = (float)v;
      }
  }
  for (int t = 0; t < glen; ++t) {
    const int64_t q = gp + t;
    for (int c = 0; c < dim; ++c) {
      double v = dA ? 0.0 : Dv[c * g_nnz + q];
      Dv_m[c * g_nnz + q] = v;
      Dv_f[c * g_nnz + q] = (float)v;
    }
    if (A < P) {
      const int32_t B = s_col[r0 + t];
      const bool oA = outm[A], oB = outm[B];
      double l = (oA || oB) ? ((A == B) ? 1.0 : 0.0) : Lp[q];
      Lp_m[q] = l;
      Lp_f[q] = (float)l;
      Mp_f[q] = (float)Mp[q];
      const bool keep = !dA && !dirm[B];
      Kc_m[q] = keep ? Lp[q] : 0.0;
      Mc_m[q] = keep ? Mp[q] : 0.0;
      Kc_f[q] = (float)Kc_m[q];
      Mc_f[q] = (float)Mc_m[q];
      if (B == A) { mp_diag[A] = Mp[q]; lp_diag[A] = l; k1_diag[A] = Lp[q]; }
    }
  }
}

// ------------------------------------------- nested P1 space (coarse level)
__constant__ int c_edge_pairs[6][2] = {{0, 1}, {1, 2}, {2, 0}, {0, 3}, {1, 3}, {2, 3}};

// end vertices of every edge node (the same from every element sharing the edge)
__global__ void k_diag_f32(const double *__restrict__ a, float *__restrict__ b, int64_t n) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// End vertices of every edge node.  All elements sharing an edge write its
// entry; each writes the pair in ascending order, so the concurrent writes
// carry identical values whatever the orientation of the edge in an element.
__global__ void k_edge_ends(const int32_t *__restrict__ conn, int64_t E, int nl, int dim, int64_t P, int32_t *ends) {
  int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= E) return;
  const int nv = dim + 1;
  const int32_t *c = conn + e * nl;
  for (int k = 0; k < nl - nv; ++k) {
    const int64_t i = (int64_t)c[nv + k] - P;
    const int32_t a = c[c_edge_pairs[k][0]], b = c[c_edge_pairs[k][1]];
    ends[2 * i] = min(a, b);
    ends[2 * i + 1] = max(a, b);
  }
}

__global__ void k_count_v2e(const int32_t *__restrict__ ends, int64_t ne, int32_t *cnt) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= ne) return;
  atomicAdd(&cnt[ends[2 * i]], 1);
  atomicAdd(&cnt[ends[2 * i + 1]], 1);
}

__global__ void k_fill_v2e(const int32_t *__restrict__ ends, int64_t ne, int64_t P, const int64_t *__restrict__ ptr,
                           int32_t *fill, int32_t *v2e) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= ne) return;
  for (int s = 0; s < 2; ++s) {
    const int32_t v = ends[2 * i + s];
    const int pos = atomicAdd(&fill[v], 1);
    v2e[ptr[v] + pos] = (int32_t)(P + i);
  }
}

// ------------------------------------------------------------------- scan
// Exclusive scan of int32 counts into int64 offsets with out[n] = total.
constexpr int SCAN_T = 512, SCAN_ITEMS = 4, SCAN_TILE = SCAN_T * SCAN_ITEMS;

__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t *total) {
  __shared__ int64_t warp_sums[SCAN_T / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t inc = v;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t u = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += u;
  }
  if (lane == 31) warp_sums[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < SCAN_T / 32 ? warp_sums[lane] : 0;
    int64_t wi = w;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t u = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += u;
    }
    if (lane < SCAN_T / 32) warp_sums[lane] = wi - w;
    if (lane == SCAN_T / 32 - 1) *total = wi;
  }
  __syncthreads();
  int64_t r = inc - v + warp_sums[warp];
  __syncthreads();
  return r;
}

__global__ void k_scan_tiles(const int32_t *__restrict__ in, int64_t *out, int64_t n, int64_t *tile_sums) {
  __shared__ int64_t tot;
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
  int64_t v[SCAN_ITEMS], s = 0;
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0;
    s += v[i];
  }
  int64_t ex = block_exclusive_scan(s, &tot);
  for (int i = 0; i < SCAN_ITEMS; ++i) {
    if (base + i <= n) out[base + i] = ex;
    ex += v[i];
  }
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int64_t *sums, int64_t nt) {
  __shared__ int64_t tot;
  int64_t carry = 0;
  for (int64_t b = 0; b < nt; b += SCAN_T) {
    int64_t i = b + threadIdx.x;
    int64_t v = i < nt ? sums[i] : 0;
    int64_t ex = block_exclusive_scan(v, &tot);
    if (i < nt) sums[i] = ex + carry;
    carry += tot;
    __syncthreads();
  }
}

__global__ void k_scan_add(int64_t *out, int64_t n, const int64_t *__restrict__ sums) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i <= n) out[i] += sums[i / SCAN_TILE];
}

void scan_exclusive(Ctx &c, const int32_t *in, int64_t *out, int64_t n) {
  const int64_t nt = (n + 1 + SCAN_TILE - 1) / SCAN_TILE;
  int64_t *sums = nullptr;
  SCVS_CUDA(ctx_malloc(c, &sums, nt * sizeof(int64_t), c.stream));
  k_scan_tiles<<<(unsigned)nt, SCAN_T, 0, c.stream>>>(in, out, n, sums);
  k_scan_sums<<<1, SCAN_T, 0, c.stream>>>(sums, nt);
  k_scan_add<<<ceil_div(n + 1, 256), 256, 0, c.stream>>>(out, n, sums);
  c.launches.n += 3;
  SCVS_CUDA(cudaFreeAsync(sums, c.stream));
}

// ------------------------------------------------------------------ driver
void build_mesh(Ctx &c, Mesh &m, const double *xyz_in, const int32_t *conn_in, const uint8_t *tag_in) {
  cudaStream_t s = c.stream;
  KScope ks(c, KC_ASSEMBLY, 0.0);
  const int64_t N = m.N, P = m.P, E = m.E;
  const int nl = m.nl, dim = m.dim;
  m.xyz = m.arena.alloc<double>(N * dim);
  m.conn = m.arena.alloc<int32_t>(E * nl);
  m.tag = m.arena.alloc<uint8_t>(N);
  SCVS_CUDA(cudaMemcpyAsync(m.xyz, xyz_in, N * dim * sizeof(double), cudaMemcpyDefault, s));
  SCVS_CUDA(cudaMemcpyAsync(m.conn, conn_in, E * nl * sizeof(int32_t), cudaMemcpyDefault, s));
  SCVS_CUDA(cudaMemcpyAsync(m.tag, tag_in, N, cudaMemcpyDefault, s));
  SCVS_CUDA(cudaMemsetAsync(c.dev_err, 0, sizeof(int), s));

  m.geom = m.arena.alloc<double>(E * GEOM_STRIDE);
  k_geom<<<ceil_div(E, 256), 256, 0, s>>>(m.xyz, m.conn, E, nl, dim, N, P, m.geom, c.dev_err);
  count_launch(c);
  int derr = dev_error(c);
  if (derr) throw derr;

  // curved (isoparametric) elements: flags, slots, element matrices by quadrature
  {
    int32_t *flag = m.arena.alloc<int32_t>(E);
    int64_t *scan = m.arena.alloc<int64_t>(E + 1);
    k_curved_flag<<<ceil_div(E, 256), 256, 0, s>>>(m.xyz, m.conn, E, nl, dim, flag);
    count_launch(c);
    scan_exclusive(c, flag, scan, E);
    SCVS_CUDA(cudaMemcpyAsync(&m.n_curved, scan + E, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SCVS_CUDA(cudaStreamSynchronize(s));
    if (m.n_curved > 0) {
      m.cslot = m.arena.alloc<int32_t>(E);
      k_curved_slot<<<ceil_div(E, 256), 256, 0, s>>>(flag, scan, E, m.cslot);
      count_launch(c);
      m.CM = m.arena.alloc<double>(m.n_curved * nl * nl);
      m.CK = m.arena.alloc<double>(m.n_curved * nl * nl);
      m.CD = m.arena.alloc<double>(m.n_curved * dim * nl * m.nv);
      const QuadTables &qh = dim == 2 ? c.quad2 : c.quad3;
      QuadTables *qd = m.arena.alloc<QuadTables>(1);
      SCVS_CUDA(cudaMemcpyAsync(qd, &qh, sizeof(QuadTables), cudaMemcpyHostToDevice, s));
      const unsigned nb = (unsigned)std::min<int64_t>(ceil_div(E, 4), (int64_t)c.num_sms * 16);
      if (dim == 2)
        k_curved_mats<2><<<nb, 128, 0, s>>>(m.xyz, m.conn, m.cslot, E, qd, m.CM, m.CK, m.CD, c.dev_err);
      else
        k_curved_mats<3><<<nb, 128, 0, s>>>(m.xyz, m.conn, m.cslot, E, qd, m.CM, m.CK, m.CD, c.dev_err);
      count_launch(c);
      derr = dev_error(c);
      if (derr) throw derr;
    }
  }

  // node -> element incidence
  int32_t *cnt = m.arena.alloc<int32_t>(N);
  SCVS_CUDA(cudaMemsetAsync(cnt, 0, N * sizeof(int32_t), s));
  k_count_incidence<<<ceil_div(E * nl, 256), 256, 0, s>>>(m.conn, E * nl, cnt);
  count_launch(c);
  m.n2e_ptr = m.arena.alloc<int64_t>(N + 1);
  scan_exclusive(c, cnt, m.n2e_ptr, N);
  m.n2e = m.arena.alloc<int32_t>(E * nl);
  SCVS_CUDA(cudaMemsetAsync(cnt, 0, N * sizeof(int32_t), s));
  k_fill_incidence<<<ceil_div(E * nl, 256), 256, 0, s>>>(m.conn, E, nl, m.n2e_ptr, cnt, m.n2e);
  k_sort_incidence<<<ceil_div(N, 128), 128, 0, s>>>(m.n2e_ptr, m.n2e, N, c.dev_err);
  c.launches.n += 2;

  // S pattern: count, scan, write
  m.s_len = m.arena.alloc<int32_t>(N);
  m.g_len = m.arena.alloc<int32_t>(N);
  const unsigned pat_blocks = std::min<int64_t>(ceil_div(N, PAT_WARPS), (int64_t)c.num_sms * 16);
  k_row_pattern<false><<<pat_blocks, PAT_WARPS * 32, 0, s>>>(m.n2e_ptr, m.n2e, m.conn, nl, N, P, m.s_len,
                                                              m.g_len, nullptr, nullptr, c.dev_err);
  count_launch(c);
  derr = dev_error(c);
  if (derr) throw derr;
  m.s_ptr = m.arena.alloc<int64_t>(N + 1);
  m.g_ptr = m.arena.alloc<int64_t>(N + 1);
  scan_exclusive(c, m.s_len, m.s_ptr, N);
  scan_exclusive(c, m.g_len, m.g_ptr, N);
  SCVS_CUDA(cudaMemcpyAsync(&m.s_nnz, m.s_ptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SCVS_CUDA(cudaMemcpyAsync(&m.g_nnz, m.g_ptr + N, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SCVS_CUDA(cudaMemcpyAsync(&m.gt_nnz, m.s_ptr + P, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SCVS_CUDA(cudaMemcpyAsync(&m.q_nnz, m.g_ptr + P, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  int *dmax = m.arena.alloc<int>(1);
  SCVS_CUDA(cudaMemsetAsync(dmax, 0, sizeof(int), s));
  k_max_int<<<std::min<unsigned>(ceil_div(N, 256), 1024), 256, 0, s>>>(m.s_len, N, dmax);
  count_launch(c);
  SCVS_CUDA(cudaMemcpyAsync(&m.max_row, dmax, sizeof(int), cudaMemcpyDeviceToHost, s));
  SCVS_CUDA(cudaStreamSynchronize(s));
  m.s_col = m.arena.alloc<int32_t>(m.s_nnz);
  k_row_pattern<true><<<pat_blocks, PAT_WARPS * 32, 0, s>>>(m.n2e_ptr, m.n2e, m.conn, nl, N, P, m.s_len,
                                                             m.g_len, m.s_ptr, m.s_col, c.dev_err);
  count_launch(c);

  // values
  m.Ms = m.arena.alloc<double>(m.s_nnz);
  m.Ks = m.arena.alloc<double>(m.s_nnz);
  m.Dv = m.arena.alloc<double>(dim * m.g_nnz);
  m.DTv = m.arena.alloc<double>(dim * m.gt_nnz);
  m.Mp = m.arena.alloc<double>(m.q_nnz);
  m.Lp = m.arena.alloc<double>(m.q_nnz);
  const RefTables &rt = dim == 2 ? c.ref2 : c.ref3;
  SCVS_CUDA(cudaMemcpyToSymbolAsync(c_ref, &rt, sizeof(RefTables), 0, cudaMemcpyHostToDevice, s));
  int cap = std::max(32, (m.max_row + 31) / 32 * 32);
  size_t per_warp = (size_t)10 * cap * sizeof(double) + (cap / 2 + 1) * sizeof(double);
  size_t smem = per_warp * ASM_WARPS;
  if (smem > 200 * 1024) throw (int)DEVERR_VALENCE;
  SCVS_CUDA(cudaFuncSetAttribute(k_assemble_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned asm_blocks = std::min<int64_t>(ceil_div(N, ASM_WARPS), (int64_t)c.num_sms * 32);
  k_assemble_rows<<<asm_blocks, ASM_WARPS * 32, smem, s>>>(
      m.n2e_ptr, m.n2e, m.conn, m.geom, nl, dim, N, P, m.s_ptr, m.s_col, m.g_len, m.g_ptr, cap, m.g_nnz,
      m.gt_nnz, m.Ms, m.Ks, m.Dv, m.DTv, m.Mp, m.Lp, m.cslot, m.CM, m.CK, m.CD, c.dev_err);
  count_launch(c);
  derr = dev_error(c);
  if (derr) throw derr;

  // masks, masked values, FP32 copies, diagonals
  m.dirmask = m.arena.alloc<uint8_t>(N);
  m.outmask = m.arena.alloc<uint8_t>(P);
  k_masks<<<ceil_div(N, 256), 256, 0, s>>>(m.tag, N, P, m.dirmask, m.outmask);
  count_launch(c);
  m.Ms_m = m.arena.alloc<double>(m.s_nnz);
  m.Ks_m = m.arena.alloc<double>(m.s_nnz);
  m.Dv_m = m.arena.alloc<double>(dim * m.g_nnz);
  m.DTv_m = m.arena.alloc<double>(dim * m.gt_nnz);
  m.Lp_m = m.arena.alloc<double>(m.q_nnz);
  m.Ms_f = m.arena.alloc<float>(m.s_nnz);
  m.Ks_f = m.arena.alloc<float>(m.s_nnz);
  m.Dv_f = m.arena.alloc<float>(dim * m.g_nnz);
  m.DTv_f = m.arena.alloc<float>(dim * m.gt_nnz);
  m.Mp_f = m.arena.alloc<float>(m.q_nnz);
  m.Lp_f = m.arena.alloc<float>(m.q_nnz);
  m.ms_diag = m.arena.alloc<double>(N);
  m.ks_diag = m.arena.alloc<double>(N);
  m.mp_diag = m.arena.alloc<double>(P);
  m.lp_diag = m.arena.alloc<double>(P);
  m.Kc_f = m.arena.alloc<float>(m.q_nnz);
  m.Mc_f = m.arena.alloc<float>(m.q_nnz);
  m.Kc_m = m.arena.alloc<double>(m.q_nnz);
  m.Mc_m = m.arena.alloc<double>(m.q_nnz);
  m.k1_diag = m.arena.alloc<double>(P);
  k_mask_values<<<ceil_div(N, 128), 128, 0, s>>>(
      N, P, dim, m.s_ptr, m.s_col, m.g_len, m.g_ptr, m.g_nnz, m.gt_nnz, m.dirmask, m.outmask, m.Ms, m.Ks,
      m.Dv, m.DTv, m.Mp, m.Lp, m.Ms_m, m.Ks_m, m.Dv_m, m.DTv_m, m.Lp_m, m.Ms_f, m.Ks_f, m.Dv_f, m.DTv_f,
      m.Mp_f, m.Lp_f, m.ms_diag, m.ks_diag, m.mp_diag, m.lp_diag, m.Kc_f, m.Mc_f, m.k1_diag, m.Kc_m, m.Mc_m);
  count_launch(c);

  m.ms_df = m.arena.alloc<float>(N);
  m.ks_df = m.arena.alloc<float>(N);
  m.mp_df = m.arena.alloc<float>(P);
  m.lp_df = m.arena.alloc<float>(P);
  m.k1_df = m.arena.alloc<float>(P);
  k_diag_f32<<<ceil_div(N, 256), 256, 0, s>>>(m.ms_diag, m.ms_df, N);
  k_diag_f32<<<ceil_div(N, 256), 256, 0, s>>>(m.ks_diag, m.ks_df, N);
  k_diag_f32<<<ceil_div(P, 256), 256, 0, s>>>(m.mp_diag, m.mp_df, P);
  k_diag_f32<<<ceil_div(P, 256), 256, 0, s>>>(m.lp_diag, m.lp_df, P);
  k_diag_f32<<<ceil_div(P, 256), 256, 0, s>>>(m.k1_diag, m.k1_df, P);
  c.launches.n += 5;

  // nested P1 space: edge ends and vertex -> incident edge nodes (sorted)
  const int64_t ne = N - P;
  m.edge_ends = m.arena.alloc<int32_t>(2 * std::max<int64_t>(ne, 1));
  m.v2e_ptr = m.arena.alloc<int64_t>(P + 1);
  m.v2e = m.arena.alloc<int32_t>(2 * std::max<int64_t>(ne, 1));
  k_edge_ends<<<ceil_div(E, 256), 256, 0, s>>>(m.conn, E, nl, dim, P, m.edge_ends);
  int32_t *vc = m.arena.alloc<int32_t>(P);
  SCVS_CUDA(cudaMemsetAsync(vc, 0, P * sizeof(int32_t), s));
  if (ne > 0) k_count_v2e<<<ceil_div(ne, 256), 256, 0, s>>>(m.edge_ends, ne, vc);
  scan_exclusive(c, vc, m.v2e_ptr, P);
  SCVS_CUDA(cudaMemsetAsync(vc, 0, P * sizeof(int32_t), s));
  if (ne > 0) k_fill_v2e<<<ceil_div(ne, 256), 256, 0, s>>>(m.edge_ends, ne, P, m.v2e_ptr, vc, m.v2e);
  k_sort_incidence<<<ceil_div(P, 128), 128, 0, s>>>(m.v2e_ptr, m.v2e, P, c.dev_err);
  c.launches.n += 4;
  SCVS_CUDA(cudaStreamSynchronize(s));
  SCVS_CUDA(cudaGetLastError());
  // row blocks of the staged FP32 gather kernels (locality order, footprints)
  if (c.opts.stage >= 0) build_row_blocks(c, m, 0);
}

// ---- Neumann (traction) load ---------------------------------------------
// b_u[A, c] = int_{Gamma_h} M_A h_c dGamma (the boundary term of Eq.
// LS_construction) for a traction given by nodal values and interpolated with
// the P2 trace basis: b_u = M_Gamma h.  Gamma_h is the set of element faces
// whose nodes all carry SCVS_TAG_NEUMANN and that belong to one element only
// (found on the host; the count runs over the tagged faces, which include
// every face with the same nodes).  Straight-sided faces: M_F = |F| times the
// reference matrix of the P2 segment or triangle (closed forms, per unit
// measure).  The load is gathered per node over its incident faces in face
// order (no atomics: deterministic).

// local P2 faces of an element, each in the face's VTK order
static const int FACES2[3][3] = {{0, 1, 3}, {1, 2, 4}, {2, 0, 5}};
static const int FACES3[4][6] = {{0, 1, 2, 4, 5, 6}, {0, 1, 3, 4, 8, 7}, {1, 2, 3, 5, 9, 8}, {2, 0, 3, 6, 7, 9}};
// P2 face mass matrices per unit measure: segment (v0, v1, mid) and triangle
// (v0, v1, v2, e01, e12, e20)
static const double SEG_M[3][3] = {{4. / 30, -1. / 30, 2. / 30}, {-1. / 30, 4. / 30, 2. / 30}, {2. / 30, 2. / 30, 16. / 30}};
static const double TRI_M[6][6] = {{6. / 180, -1. / 180, -1. / 180, 0, -4. / 180, 0},
                                   {-1. / 180, 6. / 180, -1. / 180, 0, 0, -4. / 180},
                                   {-1. / 180, -1. / 180, 6. / 180, -4. / 180, 0, 0},
                                   {0, 0, -4. / 180, 32. / 180, 16. / 180, 16. / 180},
                                   {-4. / 180, 0, 0, 16. / 180, 32. / 180, 16. / 180},
                                   {0, -4. / 180, 0, 16. / 180, 16. / 180, 32. / 180}};

// neu[(A dim + c) ld + k] = sum over the faces of A (incidence order) of
// sum_b M_F[a][b] h[k][B_b][c]; one thread per (node, component, mode slot).
__global__ void k_neumann_load(const int64_t *__restrict__ inc_ptr, const int32_t *__restrict__ inc,
                               const int32_t *__restrict__ fnodes, const double *__restrict__ fmass, int nfl,
                               const double2 *__restrict__ h, int64_t N, int dim, int m, int ld,
                               double2 *__restrict__ neu) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= (int64_t)dim * N * ld) return;
  const int k = (int)(f % ld);
  const int64_t dof = f / ld, A = dof / dim;
  const int c = (int)(dof % dim);
  double sx = 0.0, sy = 0.0;
  if (k < m)
    for (int64_t t = inc_ptr[A]; t < inc_ptr[A + 1]; ++t) {
      const int fc = inc[2 * t], a = inc[2 * t + 1];
      const double *Mrow = fmass + ((int64_t)fc * nfl + a) * nfl;
      for (int b = 0; b < nfl; ++b) {
        const double2 v = h[((int64_t)k * N + fnodes[(int64_t)fc * nfl + b]) * dim + c];
        sx += Mrow[b] * v.x;
        sy += Mrow[b] * v.y;
      }
    }
  neu[f] = make_double2(sx, sy);
}

int64_t set_neumann(Ctx &c, Mesh &m, const double2 *h_host) {
  const int dim = m.dim, nl = m.nl, nfl = dim == 2 ? 3 : 6, nf_el = dim == 2 ? 3 : 4;
  const int64_t N = m.N, E = m.E;
  std::vector<int32_t> conn((size_t)E * nl);
  std::vector<uint8_t> tag(N);
  std::vector<double> xyz((size_t)N * dim);
  SCVS_CUDA(cudaMemcpyAsync(conn.data(), m.conn, conn.size() * sizeof(int32_t), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaMemcpyAsync(tag.data(), m.tag, N, cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaMemcpyAsync(xyz.data(), m.xyz, xyz.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  // tagged faces, keyed by their sorted vertices
  std::vector<std::array<int32_t, 6>> cand;
  std::map<std::array<int32_t, 3>, int> count;
  for (int64_t e = 0; e < E; ++e)
    for (int lf = 0; lf < nf_el; ++lf) {
      std::array<int32_t, 6> nodes{};
      bool all = true;
      for (int a = 0; a < nfl; ++a) {
        nodes[a] = conn[(size_t)e * nl + (dim == 2 ? FACES2[lf][a] : FACES3[lf][a])];
        all = all && (tag[nodes[a]] & SCVS_TAG_NEUMANN);
      }
      if (!all) continue;
      std::array<int32_t, 3> key{nodes[0], nodes[1], dim == 2 ? -1 : nodes[2]};
      std::sort(key.begin(), key.begin() + dim);
      ++count[key];
      cand.push_back(nodes);
    }
  std::vector<int32_t> fnodes;
  std::vector<double> fmass;
  for (const auto &nodes : cand) {
    std::array<int32_t, 3> key{nodes[0], nodes[1], dim == 2 ? -1 : nodes[2]};
    std::sort(key.begin(), key.begin() + dim);
    if (count[key] != 1) continue;  // shared by two elements: interior
    double meas;
    const double *p0 = &xyz[(size_t)nodes[0] * dim], *p1 = &xyz[(size_t)nodes[1] * dim];
    if (dim == 2) {
      meas = std::hypot(p1[0] - p0[0], p1[1] - p0[1]);
    } else {
      const double *p2 = &xyz[(size_t)nodes[2] * dim];
      const double u[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
      const double v[3] = {p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2]};
      const double cx = u[1] * v[2] - u[2] * v[1], cy = u[2] * v[0] - u[0] * v[2], cz = u[0] * v[1] - u[1] * v[0];
      meas = 0.5 * std::sqrt(cx * cx + cy * cy + cz * cz);
    }
    for (int a = 0; a < nfl; ++a) fnodes.push_back(nodes[a]);
    // a face with an edge node off its edge midpoint (meeting a projected,
    // curved wall) is integrated with its isoparametric map
    bool curved = false;
    const int nfe = dim == 2 ? 1 : 3;
    static const int FEA[3] = {0, 1, 2}, FEB[3] = {1, 2, 0};
    for (int j = 0; j < nfe; ++j) {
      const double *xa = &xyz[(size_t)nodes[FEA[j]] * dim], *xb = &xyz[(size_t)nodes[FEB[j]] * dim];
      const double *xm = &xyz[(size_t)nodes[dim + j] * dim];
      double dev = 0.0, len = 0.0;
      for (int r = 0; r < dim; ++r) {
        const double dd = xm[r] - 0.5 * (xa[r] + xb[r]), l = xb[r] - xa[r];
        dev += dd * dd;
        len += l * l;
      }
      if (dev > 1e-24 * len) curved = true;
    }
    if (curved) {
      double X[6 * 3], Mf[36];
      for (int a = 0; a < nfl; ++a)
        for (int r = 0; r < dim; ++r) X[a * dim + r] = xyz[(size_t)nodes[a] * dim + r];
      face_mass_iso(dim - 1, dim, ISO_QUAD, X, Mf);
      for (int q = 0; q < nfl * nfl; ++q) fmass.push_back(Mf[q]);
    } else {
      for (int a = 0; a < nfl; ++a)
        for (int b = 0; b < nfl; ++b) fmass.push_back(meas * (dim == 2 ? SEG_M[a][b] : TRI_M[a][b]));
    }
  }
  const int64_t nf = (int64_t)fnodes.size() / nfl;
  // node -> (face, local index) incidence, by node then face
  std::vector<int64_t> inc_ptr(N + 1, 0);
  for (int64_t f = 0; f < nf; ++f)
    for (int a = 0; a < nfl; ++a) ++inc_ptr[fnodes[(size_t)f * nfl + a] + 1];
  for (int64_t i = 0; i < N; ++i) inc_ptr[i + 1] += inc_ptr[i];
  std::vector<int32_t> inc(2 * std::max<int64_t>(inc_ptr[N], 1));
  {
    std::vector<int64_t> fill(inc_ptr.begin(), inc_ptr.end() - 1);
    for (int64_t f = 0; f < nf; ++f)
      for (int a = 0; a < nfl; ++a) {
        const int64_t t = fill[fnodes[(size_t)f * nfl + a]]++;
        inc[2 * t] = (int32_t)f;
        inc[2 * t + 1] = a;
      }
  }
  const int64_t nh = (int64_t)m.m * N * dim;
  int64_t *d_ptr = nullptr;
  int32_t *d_inc = nullptr, *d_fn = nullptr;
  double *d_fm = nullptr;
  double2 *d_h = nullptr;
  SCVS_CUDA(ctx_malloc(c, &d_ptr, (N + 1) * sizeof(int64_t), c.stream));
  SCVS_CUDA(ctx_malloc(c, &d_inc, inc.size() * sizeof(int32_t), c.stream));
  SCVS_CUDA(ctx_malloc(c, &d_fn, std::max<size_t>(fnodes.size(), 1) * sizeof(int32_t), c.stream));
  SCVS_CUDA(ctx_malloc(c, &d_fm, std::max<size_t>(fmass.size(), 1) * sizeof(double), c.stream));
  SCVS_CUDA(ctx_malloc(c, &d_h, nh * sizeof(double2), c.stream));
  SCVS_CUDA(cudaMemcpyAsync(d_ptr, inc_ptr.data(), (N + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, c.stream));
  SCVS_CUDA(cudaMemcpyAsync(d_inc, inc.data(), inc.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c.stream));
  if (nf) {
    SCVS_CUDA(cudaMemcpyAsync(d_fn, fnodes.data(), fnodes.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c.stream));
    SCVS_CUDA(cudaMemcpyAsync(d_fm, fmass.data(), fmass.size() * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  }
  SCVS_CUDA(cudaMemcpyAsync(d_h, h_host, nh * sizeof(double2), cudaMemcpyHostToDevice, c.stream));
  const int64_t nu = (int64_t)dim * N * m.ld;
  m.neu = m.mode_arena.alloc<double2>(nu);
  {
    KScope ks(c, KC_ASSEMBLY, (double)nu * 16 + (double)nf * nfl * (4 + 8 * nfl) + (double)nh * 16);
    k_neumann_load<<<ceil_div(nu, 256), 256, 0, c.stream>>>(d_ptr, d_inc, d_fn, d_fm, nfl, d_h, N, dim, m.m, m.ld,
                                                            m.neu);
    count_launch(c);
  }
  for (void *p : {(void *)d_ptr, (void *)d_inc, (void *)d_fn, (void *)d_fm, (void *)d_h})
    SCVS_CUDA(cudaFreeAsync(p, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  return nf;
}

}  // namespace scvs
