// Batched restarted flexible GMRES over all modes of a mesh (one independent
// Krylov space per mode), right-preconditioned, with an FP64
// iterative-refinement outer loop.
//
// The paper solves each mode's system with complex GMRES and a Jacobi
// preconditioner (Sec. 2.3); its convergence test is the relative residual
// ||R - A X|| / ||R|| (Eq. ls_error).  Here every restart cycle
//   1. evaluates the true residual r = b - A_hat x in FP64 and its free-row
//      norm per mode (modes at ||r||/||b|| <= tol are done),
//   2. runs up to m_r Arnoldi steps in FP32 (or FP64) on r for every active
//      mode at once: z = P^-1 v_j (block preconditioner), w = A_hat z (all-modes
//      SpMM), then one cooperative persistent kernel that computes the
//      Hermitian products <v_i, w> of all modes, reduces them across the grid,
//      subtracts the projections (classical Gram-Schmidt), writes v_{j+1},
//      reduces its norm and updates the Hessenberg column with complex Givens
//      rotations in FP64,
//   3. solves the small triangular systems (FP64), forms d = Z y from the kept
//      preconditioned vectors z_j (flexible GMRES, so the correction is exact
//      for whatever the preconditioner returned, and needs no extra
//      application of it) and adds it to x in FP64.
// The FP32 Krylov bulk therefore only ever computes corrections; the
// residual, the solution and the Hessenberg least-squares stay in FP64.
#include <algorithm>
#include <cmath>
#include <vector>
#include "scvs_internal.h"
#include "vecops.cuh"

namespace scvs {

template <typename T> struct ArnArgs {
  int64_t rows;
  int ld, m_r, n_comp;
  typename cpx<T>::t *V;        // [(m_r+1)][rows][ld]
  const typename cpx<T>::t *w;  // A_hat z
  int64_t vstride;              // rows * ld
  // row chunks (never straddling components), grouped by component
  int64_t n_chunk;
  const int64_t *chunk_row0;
  const int32_t *chunk_rows, *chunk_comp, *comp_chunk;
  const uint8_t *comp_active;   // chunks of inactive components are skipped
  double2 *part;                // [n_chunk][m_r+2][ld] chunk partials
  double2 *h;                   // [n_comp][m_r+2][ld] reduced products (slot j+1: ||w||^2)
  // per system s = comp * ld + k
  double2 *H;                   // [S][m_r+1][m_r]   rotated Hessenberg (R factor)
  double *cs;                   // [S][m_r]
  double2 *sn;                  // [S][m_r]
  double2 *gv;                  // [S][m_r+1]        rotated residual vector
  int *state;                   // [S] 1 = Arnoldi running for this system
  int *kdim;                    // [S] accepted steps in this cycle
  const double *target;         // [S] residual-estimate target
  double *rscale;               // [S] 1/||v_{j+1}|| for the next preconditioner step
  double *est;                  // [S] |g_{j+1}|
  int *n_active;                // [1] zeroed before the launch
  GridSync *gs;
  double breakdown;             // relative size of h_{j+1,j} treated as breakdown
};

constexpr int ARN_RPT = 4;  // rows per thread per tile

template <typename T, int TPR>
__device__ __forceinline__ T warp_rows_sum(T v) {
#pragma unroll
  for (int o = 16; o >= TPR; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// One Arnoldi step j for every system in one cooperative launch:
//   phase 1  chunk partials of <v_i, w> (i <= j) and ||w||^2
//   phase 2  per (component, slot, mode) sums over the component's chunks
//   phase 3  w' = w - sum_i h_i v_i -> v_{j+1}, chunk partials of ||w'||^2
//   phase 4  per system: sigma = ||w'||, Hessenberg column, complex Givens
//            rotations and residual estimate in FP64
// separated by bounded grid barriers.
template <typename T, int MPL, int TPR>
__global__ void __launch_bounds__(256, 3) k_arnoldi(const ArnArgs<T> a, const int j) {
  using C = typename cpx<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T *acc = reinterpret_cast<T *>(smem_raw);
  const int nwarps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane32 = threadIdx.x & 31;
  const int lane = threadIdx.x % TPR, roff = threadIdx.x / TPR;
  const int RPB = blockDim.x / TPR, TR = RPB * ARN_RPT;
  const int ld = a.ld, koff = lane * MPL;
  const int nvec = j + 1, nslots = j + 2;
  const int sstride = 2 * ld;                  // one slot: ld complex as (re, im)
  const int wstride = (a.m_r + 2) * sstride;   // one warp's slots
  const bool row_leader = lane32 < TPR;        // holds the warp's row-reduced sums
  const int64_t pstride = (int64_t)(a.m_r + 2) * ld;

  // ---------------- phase 1: chunk partials of <v_i, w> and ||w||^2
  T *myacc = acc + warp * wstride;
  for (int64_t ch = blockIdx.x; ch < a.n_chunk; ch += gridDim.x) {
    if (!a.comp_active[a.chunk_comp[ch]]) continue;  // block-uniform
    for (int t = lane32; t < nslots * sstride; t += 32) myacc[t] = T(0);
    __syncwarp();
    const int64_t r0 = a.chunk_row0[ch], r1 = r0 + a.chunk_rows[ch];
    for (int64_t tb = r0; tb < r1; tb += TR) {
      CV<T, MPL> wv[ARN_RPT];
      int64_t rr[ARN_RPT];
#pragma unroll
      for (int q = 0; q < ARN_RPT; ++q) {
        rr[q] = tb + roff + (int64_t)q * RPB;
        if (rr[q] < r1) ldv<T, MPL>(wv[q], a.w + rr[q] * ld + koff); else wv[q].zero();
      }
      {
        T s[MPL];
#pragma unroll
        for (int i = 0; i < MPL; ++i) {
          s[i] = 0;
#pragma unroll
          for (int q = 0; q < ARN_RPT; ++q) s[i] += wv[q].re[i] * wv[q].re[i] + wv[q].im[i] * wv[q].im[i];
          s[i] = warp_rows_sum<T, TPR>(s[i]);
        }
        if (row_leader)
#pragma unroll
          for (int i = 0; i < MPL; ++i) myacc[(j + 1) * sstride + 2 * (koff + i)] += s[i];
      }
      // Krylov vectors in pairs: 2 x ARN_RPT independent loads in flight per thread
      for (int vi = 0; vi < nvec; vi += 2) {
        const bool two = vi + 1 < nvec;
        const C *V0 = a.V + (int64_t)vi * a.vstride;
        const C *V1 = a.V + (int64_t)(two ? vi + 1 : vi) * a.vstride;
        CV<T, MPL> v0[ARN_RPT], v1[ARN_RPT];
#pragma unroll
        for (int q = 0; q < ARN_RPT; ++q) {
          if (rr[q] < r1) {
            ldv<T, MPL>(v0[q], V0 + rr[q] * ld + koff);
            if (two) ldv<T, MPL>(v1[q], V1 + rr[q] * ld + koff); else v1[q].zero();
          } else {
            v0[q].zero();
            v1[q].zero();
          }
        }
        T sr0[MPL], si0[MPL], sr1[MPL], si1[MPL];
#pragma unroll
        for (int i = 0; i < MPL; ++i) {
          sr0[i] = si0[i] = sr1[i] = si1[i] = 0;
#pragma unroll
          for (int q = 0; q < ARN_RPT; ++q) {  // conj(v) * w
            sr0[i] += v0[q].re[i] * wv[q].re[i] + v0[q].im[i] * wv[q].im[i];
            si0[i] += v0[q].re[i] * wv[q].im[i] - v0[q].im[i] * wv[q].re[i];
            sr1[i] += v1[q].re[i] * wv[q].re[i] + v1[q].im[i] * wv[q].im[i];
            si1[i] += v1[q].re[i] * wv[q].im[i] - v1[q].im[i] * wv[q].re[i];
          }
          sr0[i] = warp_rows_sum<T, TPR>(sr0[i]);
          si0[i] = warp_rows_sum<T, TPR>(si0[i]);
          sr1[i] = warp_rows_sum<T, TPR>(sr1[i]);
          si1[i] = warp_rows_sum<T, TPR>(si1[i]);
        }
        if (row_leader)
#pragma unroll
          for (int i = 0; i < MPL; ++i) {
            myacc[vi * sstride + 2 * (koff + i)] += sr0[i];
            myacc[vi * sstride + 2 * (koff + i) + 1] += si0[i];
            if (two) {
              myacc[(vi + 1) * sstride + 2 * (koff + i)] += sr1[i];
              myacc[(vi + 1) * sstride + 2 * (koff + i) + 1] += si1[i];
            }
          }
      }
    }
    __syncthreads();
    // chunk partial (warps summed in fixed order) -> global, FP64
    for (int e = threadIdx.x; e < nslots * ld; e += blockDim.x) {
      double re = 0, im = 0;
      for (int w = 0; w < nwarps; ++w) {
        re += (double)acc[w * wstride + 2 * e];
        im += (double)acc[w * wstride + 2 * e + 1];
      }
      a.part[ch * pstride + e] = make_double2(re, im);
    }
    __syncthreads();
  }
  if (!grid_sync(a.gs, gridDim.x)) return;

  // ---------------- phase 2: per (component, slot, mode) sums, one warp per item
  {
    const int items = a.n_comp * nslots * ld;
    for (int it = blockIdx.x * nwarps + warp; it < items; it += gridDim.x * nwarps) {
      const int comp = it / (nslots * ld), e = it % (nslots * ld);
      double re = 0, im = 0;
      for (int ch = a.comp_chunk[comp] + lane32; ch < a.comp_chunk[comp + 1]; ch += 32) {
        const double2 p = a.part[(int64_t)ch * pstride + e];
        re += p.x; im += p.y;
      }
      for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
      }
      if (lane32 == 0) a.h[(int64_t)comp * pstride + e] = make_double2(re, im);
    }
  }
  if (!grid_sync(a.gs, gridDim.x)) return;

  // ---------------- phase 3: w' = w - sum_i h_i v_i -> V_{j+1}; chunk partials of ||w'||^2
  T *hs = acc;                       // [nvec][ld] complex, for the current chunk's component
  T *nacc = acc + nvec * sstride;    // [nwarps][ld] (re only used)
  C *Vn = a.V + (int64_t)(j + 1) * a.vstride;
  for (int64_t ch = blockIdx.x; ch < a.n_chunk; ch += gridDim.x) {
    const int comp = a.chunk_comp[ch];
    if (!a.comp_active[comp]) continue;  // block-uniform
    for (int e = threadIdx.x; e < nvec * ld; e += blockDim.x) {
      const int k = e % ld;
      const double2 hv = a.state[comp * ld + k] ? a.h[(int64_t)comp * pstride + e] : make_double2(0.0, 0.0);
      hs[2 * e] = (T)hv.x;
      hs[2 * e + 1] = (T)hv.y;
    }
    for (int e = threadIdx.x; e < nwarps * ld; e += blockDim.x) nacc[2 * e] = T(0);
    __syncthreads();
    bool act[MPL];
#pragma unroll
    for (int i = 0; i < MPL; ++i) act[i] = a.state[comp * ld + koff + i] != 0;
    const int64_t r0 = a.chunk_row0[ch], r1 = r0 + a.chunk_rows[ch];
    for (int64_t tb = r0; tb < r1; tb += TR) {
      CV<T, MPL> wv[ARN_RPT];
      int64_t rr[ARN_RPT];
#pragma unroll
      for (int q = 0; q < ARN_RPT; ++q) {
        rr[q] = tb + roff + (int64_t)q * RPB;
        if (rr[q] < r1) ldv<T, MPL>(wv[q], a.w + rr[q] * ld + koff); else wv[q].zero();
      }
      for (int vi = 0; vi < nvec; vi += 2) {
        const bool two = vi + 1 < nvec;
        const C *V0 = a.V + (int64_t)vi * a.vstride;
        const C *V1 = a.V + (int64_t)(two ? vi + 1 : vi) * a.vstride;
        T hr0[MPL], hi0[MPL], hr1[MPL], hi1[MPL];
#pragma unroll
        for (int i = 0; i < MPL; ++i) {
          hr0[i] = hs[vi * sstride + 2 * (koff + i)];
          hi0[i] = hs[vi * sstride + 2 * (koff + i) + 1];
          hr1[i] = two ? hs[(vi + 1) * sstride + 2 * (koff + i)] : T(0);
          hi1[i] = two ? hs[(vi + 1) * sstride + 2 * (koff + i) + 1] : T(0);
        }
        CV<T, MPL> v0[ARN_RPT], v1[ARN_RPT];
#pragma unroll
        for (int q = 0; q < ARN_RPT; ++q) {
          if (rr[q] < r1) {
            ldv<T, MPL>(v0[q], V0 + rr[q] * ld + koff);
            if (two) ldv<T, MPL>(v1[q], V1 + rr[q] * ld + koff); else v1[q].zero();
          } else {
            v0[q].zero();
            v1[q].zero();
          }
        }
#pragma unroll
        for (int q = 0; q < ARN_RPT; ++q)
#pragma unroll
          for (int i = 0; i < MPL; ++i) {  // w -= h0 v0 + h1 v1
            wv[q].re[i] -= hr0[i] * v0[q].re[i] - hi0[i] * v0[q].im[i] + hr1[i] * v1[q].re[i] - hi1[i] * v1[q].im[i];
            wv[q].im[i] -= hr0[i] * v0[q].im[i] + hi0[i] * v0[q].re[i] + hr1[i] * v1[q].im[i] + hi1[i] * v1[q].re[i];
          }
      }
      T s[MPL];
#pragma unroll
      for (int i = 0; i < MPL; ++i) s[i] = 0;
#pragma unroll
      for (int q = 0; q < ARN_RPT; ++q) {
        if (rr[q] < r1) {
#pragma unroll
          for (int i = 0; i < MPL; ++i) {
            if (!act[i]) { wv[q].re[i] = 0; wv[q].im[i] = 0; }
            s[i] += wv[q].re[i] * wv[q].re[i] + wv[q].im[i] * wv[q].im[i];
          }
          stv<T, MPL>(Vn + rr[q] * ld + koff, wv[q]);
        }
      }
#pragma unroll
      for (int i = 0; i < MPL; ++i) s[i] = warp_rows_sum<T, TPR>(s[i]);
      if (row_leader)
#pragma unroll
        for (int i = 0; i < MPL; ++i) nacc[2 * (warp * ld + koff + i)] += s[i];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < ld; k += blockDim.x) {
      double sm = 0;
      for (int w = 0; w < nwarps; ++w) sm += (double)nacc[2 * (w * ld + k)];
      a.part[ch * pstride + k] = make_double2(sm, 0.0);
    }
    __syncthreads();
  }
  if (!grid_sync(a.gs, gridDim.x)) return;

  // ---------------- phase 4: one warp per system: norm, Hessenberg column, Givens, estimate
  const int S = a.n_comp * ld;
  for (int sys = blockIdx.x * nwarps + warp; sys < S; sys += gridDim.x * nwarps) {
    const int comp = sys / ld, k = sys % ld;
    double s2 = 0;
    for (int ch = a.comp_chunk[comp] + lane32; ch < a.comp_chunk[comp + 1]; ch += 32) s2 += a.part[(int64_t)ch * pstride + k].x;
    for (int o = 16; o > 0; o >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, o);
    if (lane32 != 0) continue;
    if (!a.state[sys]) { a.rscale[sys] = 0.0; continue; }
    const int m_r = a.m_r;
    const double2 *hc = a.h + (int64_t)comp * pstride;  // column: hc[i * ld + k]
    double2 *Hk = a.H + (int64_t)sys * (m_r + 1) * m_r;
    double *csk = a.cs + (int64_t)sys * m_r;
    double2 *snk = a.sn + (int64_t)sys * m_r;
    double2 *gk = a.gv + (int64_t)sys * (m_r + 1);
    const double sigma = sqrt(fmax(s2, 0.0));
    const double wn = sqrt(fmax(hc[(j + 1) * ld + k].x, 0.0));
    // apply the previous rotations to the new column, top-down
    double2 hprev = hc[0 * ld + k];
    for (int i = 0; i < j; ++i) {
      const double2 hnext = hc[(i + 1) * ld + k];
      const double c = csk[i];
      const double2 s = snk[i];
      // t = c h_i + s h_{i+1};  h_{i+1}' = -conj(s) h_i + c h_{i+1}
      double2 t = make_double2(c * hprev.x + s.x * hnext.x - s.y * hnext.y, c * hprev.y + s.x * hnext.y + s.y * hnext.x);
      double2 u = make_double2(-(s.x * hprev.x + s.y * hprev.y) + c * hnext.x, -(s.x * hprev.y - s.y * hprev.x) + c * hnext.y);
      Hk[(int64_t)i * m_r + j] = t;
      hprev = u;
    }
    // new rotation zeroing sigma below the diagonal
    const double aa = sqrt(hprev.x * hprev.x + hprev.y * hprev.y);
    const double r = sqrt(aa * aa + sigma * sigma);
    double c;
    double2 s;
    if (r == 0.0) {
      c = 1.0; s = make_double2(0.0, 0.0);
    } else if (aa == 0.0) {
      c = 0.0; s = make_double2(1.0, 0.0);  // conj(b)/|b| with b = sigma > 0
    } else {
      c = aa / r;
      const double2 ph = make_double2(hprev.x / aa, hprev.y / aa);  // a/|a|
      s = make_double2(ph.x * sigma / r, ph.y * sigma / r);         // (a/|a|) conj(b)/r, b real
    }
    csk[j] = c;
    snk[j] = s;
    Hk[(int64_t)j * m_r + j] = (aa == 0.0) ? make_double2(r, 0.0) : make_double2(hprev.x * r / aa, hprev.y * r / aa);
    const double2 gj = gk[j];
    gk[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
    gk[j] = make_double2(c * gj.x, c * gj.y);
    const double e = sqrt(gk[j + 1].x * gk[j + 1].x + gk[j + 1].y * gk[j + 1].y);
    a.est[sys] = e;
    a.kdim[sys] = j + 1;
    const bool broke = !(sigma > a.breakdown * wn);
    const bool nonfinite = !isfinite(e) || !isfinite(sigma);
    if (nonfinite) a.kdim[sys] = j;
    if (e <= a.target[sys] || broke || nonfinite || j + 1 >= m_r) {
      a.state[sys] = 0;
      a.rscale[sys] = 0.0;
    } else {
      a.rscale[sys] = 1.0 / sigma;
      atomicAdd(a.n_active, 1);
    }
  }
}

// Back substitution R y = g for every mode (FP64); y[i][k], zero past kdim.
__global__ void k_lsq(const double2 *__restrict__ H, const double2 *__restrict__ gv, const int *__restrict__ kdim,
                      int ld, int m_r, double2 *__restrict__ y) {
  // ld here is the number of systems S (y[i][s])
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= ld) return;
  const double2 *Hk = H + (int64_t)k * (m_r + 1) * m_r;
  const double2 *gk = gv + (int64_t)k * (m_r + 1);
  const int n = kdim[k];
  for (int i = m_r - 1; i >= n; --i) y[(int64_t)i * ld + k] = make_double2(0, 0);
  for (int i = n - 1; i >= 0; --i) {
    double2 s = gk[i];
    for (int l = i + 1; l < n; ++l) {
      const double2 h = Hk[(int64_t)i * m_r + l], yl = y[(int64_t)l * ld + k];
      s.x -= h.x * yl.x - h.y * yl.y;
      s.y -= h.x * yl.y + h.y * yl.x;
    }
    const double2 d = Hk[(int64_t)i * m_r + i];
    const double dd = d.x * d.x + d.y * d.y;
    double2 q = dd > 0 ? make_double2((s.x * d.x + s.y * d.y) / dd, (s.y * d.x - s.x * d.y) / dd) : make_double2(0, 0);
    if (!isfinite(q.x) || !isfinite(q.y)) q = make_double2(0, 0);
    y[(int64_t)i * ld + k] = q;
  }
}

// x += sum_{i<nv} y_i v_i (per mode), in one pass: per element four FP32
// partial sums (term i into sum i mod 4; a zero coefficient, a system past its
// Krylov dimension, contributes nothing, so stale vectors never propagate),
// combined as (s0 + s1) + (s2 + s3) and added to the FP64 iterate.  Two adjacent elements per thread, so every
// thread keeps eight basis loads in flight.
template <typename T>
__global__ void __launch_bounds__(256) k_combine_add(const typename cpx<T>::t *__restrict__ V, int64_t vstride,
                                                     const double2 *__restrict__ y, int nv, int ld, int S,
                                                     const int32_t *__restrict__ dof_comp,
                                                     const int *__restrict__ upd, int64_t total,
                                                     double2 *__restrict__ x) {
  const int64_t f0 = 2 * (blockIdx.x * (int64_t)blockDim.x + threadIdx.x);
  if (f0 >= total) return;
  int sys[2];
  bool on[2];
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    const int64_t f = f0 + e;
    sys[e] = f < total ? (dof_comp ? dof_comp[f / ld] * ld : 0) + (int)(f % ld) : 0;
    on[e] = f < total && upd[sys[e]];
  }
  if (!on[0] && !on[1]) return;
  T re[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}}, im[2][4] = {{0, 0, 0, 0}, {0, 0, 0, 0}};
  int i = 0;
  for (; i + 4 <= nv; i += 4) {
    typename cpx<T>::t v[4][2];
    double2 yy[4][2];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        yy[u][e] = y[(int64_t)(i + u) * S + sys[e]];
        v[u][e] = (f0 + e < total) ? V[(int64_t)(i + u) * vstride + f0 + e] : mk<T>(0, 0);
      }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        const bool z = yy[u][e].x == 0.0 && yy[u][e].y == 0.0;
        const T a = (T)yy[u][e].x, b = (T)yy[u][e].y;
        re[e][u] += z ? T(0) : a * v[u][e].x - b * v[u][e].y;
        im[e][u] += z ? T(0) : a * v[u][e].y + b * v[u][e].x;
      }
  }
  for (; i < nv; ++i)
#pragma unroll
    for (int e = 0; e < 2; ++e) {
      const double2 yy = y[(int64_t)i * S + sys[e]];
      const auto v = (f0 + e < total) ? V[(int64_t)i * vstride + f0 + e] : mk<T>(0, 0);
      const bool z = yy.x == 0.0 && yy.y == 0.0;
      re[e][0] += z ? T(0) : (T)yy.x * v.x - (T)yy.y * v.y;
      im[e][0] += z ? T(0) : (T)yy.x * v.y + (T)yy.y * v.x;
    }
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    if (!on[e]) continue;
    const T rs = (re[e][0] + re[e][1]) + (re[e][2] + re[e][3]), is = (im[e][0] + im[e][1]) + (im[e][2] + im[e][3]);
    double2 xv = x[f0 + e];
    xv.x += (double)rs;
    xv.y += (double)is;
    x[f0 + e] = xv;
  }
}

template <typename T>
__global__ void k_add_to_x(const typename cpx<T>::t *__restrict__ z, const int *__restrict__ upd, int ld,
                           const int32_t *__restrict__ dof_comp, int64_t total, double2 *__restrict__ x) {
  int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= total) return;
  if (!upd[(dof_comp ? dof_comp[f / ld] * ld : 0) + f % ld]) return;
  const auto d = z[f];
  double2 v = x[f];
  v.x += (double)d.x;
  v.y += (double)d.y;
  x[f] = v;
}

// x = b on Dirichlet rows (= g), 0 elsewhere (only the modes with reset[k] != 0
// when `reset` is given).
__global__ void k_init_x(const double2 *__restrict__ b, const uint8_t *__restrict__ dirm, int64_t N, int dim,
                         int64_t total, int ld, double2 *__restrict__ x, const int *__restrict__ reset,
                         const int32_t *__restrict__ dof_comp) {
  int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= total) return;
  if (reset && !reset[(dof_comp ? dof_comp[f / ld] * ld : 0) + f % ld]) return;
  const int64_t dof = f / ld;
  const bool dir = dof < N * dim && dirm[dof / dim];
  x[f] = dir ? b[f] : make_double2(0.0, 0.0);
}

// Warm start: keep x on free rows, x = b (= g) on Dirichlet velocity rows.
__global__ void k_warm_x(const double2 *__restrict__ b, const uint8_t *__restrict__ dirm, int64_t N, int dim,
                         int64_t total, int ld, double2 *__restrict__ x) {
  int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= total) return;
  const int64_t dof = f / ld;
  if (dof < N * dim && dirm[dof / dim]) x[f] = b[f];
}

// One CUDA graph per Arnoldi step j of a solve: the step's launches (block
// preconditioner, all-modes SpMM, the persistent Arnoldi kernel and the copy
// of the active-system count) are captured once, on an internal stream (the
// caller's stream may be the legacy default stream, which cannot capture),
// and replayed on the context's stream.  Launch counts advance as for plain
// launches.  A capture the runtime refuses switches graphs off for the solve.
struct StepGraphs {
  bool on;
  std::vector<cudaGraphExec_t> exec;
  std::vector<int64_t> launches;  // kernel launches per replay of step j
  cudaStream_t cap = nullptr;
  StepGraphs(int m_r, bool enable) : on(enable), exec(m_r, nullptr), launches(m_r, 0) {
    if (on && cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) { on = false; cap = nullptr; }
  }
  ~StepGraphs() {
    for (auto &e : exec) if (e) cudaGraphExecDestroy(e);
    if (cap) cudaStreamDestroy(cap);
  }
  template <typename F> bool capture(Ctx &c, int j, F &&body) {
    SCVS_CUDA(cudaStreamSynchronize(c.stream));
    cudaStream_t user = c.stream;
    const int64_t n0 = c.launches.n;
    c.stream = cap;
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      try {
        body();
      } catch (...) {
        cudaStreamEndCapture(cap, &g);
        if (g) cudaGraphDestroy(g);
        c.stream = user;
        (void)cudaGetLastError();
        on = false;
        c.launches.n = n0;
        return false;
      }
      ok = cudaStreamEndCapture(cap, &g) == cudaSuccess && g;
    }
    c.stream = user;
    launches[j] = c.launches.n - n0;
    c.launches.n = n0;
    if (ok) ok = cudaGraphInstantiate(&exec[j], g, 0) == cudaSuccess;
    if (g) cudaGraphDestroy(g);
    if (!ok) {
      (void)cudaGetLastError();
      exec[j] = nullptr;
      on = false;
    }
    return ok;
  }
  void launch(Ctx &c, int j) {
    SCVS_CUDA(cudaGraphLaunch(exec[j], c.stream));
    c.launches.n += launches[j];
  }
};

template <typename T>
struct Work {
  using C = typename cpx<T>::t;
  C *V = nullptr, *Z = nullptr, *W = nullptr, *S = nullptr;
  double2 *part = nullptr, *h = nullptr, *H = nullptr, *sn = nullptr, *gv = nullptr, *y = nullptr;
  double *cs = nullptr, *target = nullptr, *rscale = nullptr, *est = nullptr, *norm2 = nullptr;
  int *state = nullptr, *kdim = nullptr, *n_active = nullptr, *upd = nullptr;
  std::vector<void *> owned;
  cudaStream_t s = nullptr;
  cudaMemPool_t pool = nullptr;
  template <typename U> U *get(size_t n) {
    void *p = nullptr;
    SCVS_CUDA(cudaMallocFromPoolAsync(&p, std::max<size_t>(n, 1) * sizeof(U), pool, s));
    owned.push_back(p);
    return static_cast<U *>(p);
  }
  ~Work() { for (void *p : owned) cudaFreeAsync(p, s); }
};

// Algorithmic bytes of Arnoldi step j: v_0..v_j read twice (products, then
// update), w read twice, v_{j+1} written once.
static double arnoldi_bytes(int64_t total, int j, int cs) { return (double)(2 * (j + 1) + 3) * total * cs; }

template <typename T>
static void launch_arnoldi(Ctx &c, const ArnArgs<T> &a, int j, int grid, int block, size_t smem) {
  KScope ks(c, KC_ARNOLDI, arnoldi_bytes(a.vstride, j, 2 * sizeof(T)));
  SCVS_DISPATCH_LD(T, a.ld, {
    void *kfn = (void *)k_arnoldi<T, MPL, L>;
    ArnArgs<T> aa = a;
    int jj = j;
    void *args[] = {(void *)&aa, (void *)&jj};
    SCVS_CUDA(cudaLaunchCooperativeKernel(kfn, dim3(grid), dim3(block), args, smem, c.stream));
  });
  count_launch(c);
}

template <typename T>
static void arnoldi_config(Ctx &c, int ld, int m_r, int &grid, int &block, size_t &smem) {
  const int esz = 2 * sizeof(T);
  int nw = 8;
  while (nw > 1 && (size_t)nw * (m_r + 2) * ld * esz > 160 * 1024) nw >>= 1;
  block = nw * 32;
  smem = std::max<size_t>((size_t)nw * (m_r + 2) * ld * esz, ld * sizeof(double) + 64);
  int per_sm = 0;
  SCVS_DISPATCH_LD(T, ld, {
    void *kfn = (void *)k_arnoldi<T, MPL, L>;
    SCVS_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    SCVS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, block, smem));
  });
  if (per_sm < 1) throw (int)SCVS_ERR_CUDA;
  grid = per_sm * c.num_sms;
}

// ----------------------------------------------------------------- COCR
// Preconditioned COCR (conjugate orthogonal conjugate residual, Sogabe and
// Zhang 2007): the conjugate-residual recurrence with the bilinear form
// x^T y in place of the Hermitian product, valid for a complex symmetric
// operator (A_hat^T = A_hat, reading C1 of the continuity row) and a complex
// symmetric preconditioner M ~ A_hat^-1 (the block-diagonal kinds).  Paper
// Sec. 2.3 remarks that the left-hand side is symmetric; a short recurrence
// keeps 7 work vectors per system instead of a restart basis.  Per iteration,
// for every active system s:
//   q = M Ap,  mu = Ap^T q,  alpha = rho / mu
//   d += alpha p,  r -= alpha Ap,  z -= alpha q
//   Az = A_hat z,  rho' = z^T Az,  beta = rho' / rho
//   p = z + beta p,  Ap = Az + beta Ap
// with r the (FP32) residual of the correction equation A_hat d = r_0 of the
// refinement cycle, stopped when ||r|| reaches the cycle's target.
struct CocrState {
  double2 *part;      // [n_chunk][2][ld] chunk partials
  double2 *rho;       // [S] z^T Az
  double2 *alpha;     // [S]
  double2 *beta;      // [S]
  double *target2;    // [S] squared residual target of the cycle
  int *state;         // [S] 1 = iterating
  int *iters;         // [S] iterations of the cycle
  int *n_active;      // [1]
};

// Chunk partials of (a^T b) (bilinear) in slot 0 and, with NORM, ||c||^2 in
// slot 1 (.x), for every mode; one thread per (row group, mode).
template <typename T, bool NORM>
__global__ void __launch_bounds__(256) k_cocr_dot(const typename cpx<T>::t *__restrict__ a,
                                                  const typename cpx<T>::t *__restrict__ b,
                                                  const typename cpx<T>::t *__restrict__ cvec, int ld,
                                                  int64_t n_chunk, const int64_t *__restrict__ chunk_row0,
                                                  const int32_t *__restrict__ chunk_rows,
                                                  const int32_t *__restrict__ chunk_comp,
                                                  const uint8_t *__restrict__ comp_active, double2 *__restrict__ part) {
  __shared__ double sh[3][256];
  const int k = threadIdx.x % ld, rg = threadIdx.x / ld, RG = blockDim.x / ld;
  for (int64_t ch = blockIdx.x; ch < n_chunk; ch += gridDim.x) {
    if (!comp_active[chunk_comp[ch]]) continue;  // block-uniform
    const int64_t r0 = chunk_row0[ch], r1 = r0 + chunk_rows[ch];
    double sr = 0.0, si = 0.0, sn = 0.0;
    if (rg < RG)
      for (int64_t r = r0 + rg; r < r1; r += RG) {
        const auto x = a[r * ld + k], y = b[r * ld + k];
        sr = fma((double)x.x, (double)y.x, fma(-(double)x.y, (double)y.y, sr));
        si = fma((double)x.x, (double)y.y, fma((double)x.y, (double)y.x, si));
        if (NORM) {
          const auto z = cvec[r * ld + k];
          sn = fma((double)z.x, (double)z.x, fma((double)z.y, (double)z.y, sn));
        }
      }
    sh[0][threadIdx.x] = sr;
    sh[1][threadIdx.x] = si;
    sh[2][threadIdx.x] = sn;
    __syncthreads();
    if (rg == 0) {
      double tr = 0.0, ti = 0.0, tn = 0.0;
      for (int g = 0; g < RG; ++g) {  // fixed order
        tr += sh[0][g * ld + k];
        ti += sh[1][g * ld + k];
        tn += sh[2][g * ld + k];
      }
      part[(ch * 2 + 0) * ld + k] = make_double2(tr, ti);
      if (NORM) part[(ch * 2 + 1) * ld + k] = make_double2(tn, 0.0);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ double2 sum_chunks(const double2 *__restrict__ part, const int32_t *__restrict__ comp_chunk,
                                              int comp, int slot, int ld, int k) {
  double2 v = make_double2(0.0, 0.0);
  for (int ch = comp_chunk[comp]; ch < comp_chunk[comp + 1]; ++ch) {
    const double2 p = part[((int64_t)ch * 2 + slot) * ld + k];
    v.x += p.x;
    v.y += p.y;
  }
  return v;
}

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double d = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / d, (a.y * b.x - a.x * b.y) / d);
}

// rho = z^T Az of the cycle's start (one thread per system).
__global__ void k_cocr_init(CocrState st, const int32_t *__restrict__ comp_chunk, int S, int ld) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  st.iters[s] = 0;
  if (!st.state[s]) { st.rho[s] = make_double2(0.0, 0.0); return; }
  st.rho[s] = sum_chunks(st.part, comp_chunk, s / ld, 0, ld, s % ld);
}

// alpha = rho / (Ap^T q); a vanishing or non-finite denominator stops the system.
__global__ void k_cocr_alpha(CocrState st, const int32_t *__restrict__ comp_chunk, int S, int ld) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  double2 al = make_double2(0.0, 0.0);
  if (st.state[s]) {
    const double2 mu = sum_chunks(st.part, comp_chunk, s / ld, 0, ld, s % ld);
    al = cdiv(st.rho[s], mu);
    if (!(isfinite(al.x) && isfinite(al.y)) || (mu.x == 0.0 && mu.y == 0.0)) {
      st.state[s] = 0;
      al = make_double2(0.0, 0.0);
    } else {
      st.iters[s] += 1;
    }
  }
  st.alpha[s] = al;
}

// beta = rho' / rho and the convergence test ||r||^2 <= target^2.
__global__ void k_cocr_beta(CocrState st, const int32_t *__restrict__ comp_chunk, int S, int ld, int last) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  double2 be = make_double2(0.0, 0.0);
  if (st.state[s]) {
    const double2 rn = sum_chunks(st.part, comp_chunk, s / ld, 0, ld, s % ld);
    const double r2 = sum_chunks(st.part, comp_chunk, s / ld, 1, ld, s % ld).x;
    be = cdiv(rn, st.rho[s]);
    const bool ok = isfinite(be.x) && isfinite(be.y) && isfinite(r2);
    if (!ok || r2 <= st.target2[s] || last) {
      st.state[s] = 0;
      be = make_double2(0.0, 0.0);
    } else {
      st.rho[s] = rn;
      atomicAdd(st.n_active, 1);
    }
  }
  st.beta[s] = be;
}

// d += alpha p; r -= alpha Ap; z -= alpha q
template <typename T>
__global__ void k_cocr_update1(const double2 *__restrict__ alpha, const int32_t *__restrict__ dof_comp, int ld,
                               int64_t total, const typename cpx<T>::t *__restrict__ p,
                               const typename cpx<T>::t *__restrict__ Ap, const typename cpx<T>::t *__restrict__ q,
                               typename cpx<T>::t *__restrict__ d, typename cpx<T>::t *__restrict__ r,
                               typename cpx<T>::t *__restrict__ z) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= total) return;
  const double2 a = alpha[(dof_comp ? dof_comp[f / ld] * ld : 0) + f % ld];
  if (a.x == 0.0 && a.y == 0.0) return;
  const T ar = (T)a.x, ai = (T)a.y;
  const auto pv = p[f], av = Ap[f], qv = q[f];
  auto dv = d[f], rv = r[f], zv = z[f];
  dv.x += ar * pv.x - ai * pv.y;  dv.y += ar * pv.y + ai * pv.x;
  rv.x -= ar * av.x - ai * av.y;  rv.y -= ar * av.y + ai * av.x;
  zv.x -= ar * qv.x - ai * qv.y;  zv.y -= ar * qv.y + ai * qv.x;
  d[f] = dv;
  r[f] = rv;
  z[f] = zv;
}

// p = z + beta p; Ap = Az + beta Ap (systems still iterating)
template <typename T>
__global__ void k_cocr_update2(const double2 *__restrict__ beta, const int *__restrict__ state,
                               const int32_t *__restrict__ dof_comp, int ld, int64_t total,
                               const typename cpx<T>::t *__restrict__ z, const typename cpx<T>::t *__restrict__ Az,
                               typename cpx<T>::t *__restrict__ p, typename cpx<T>::t *__restrict__ Ap) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= total) return;
  const int sys = (dof_comp ? dof_comp[f / ld] * ld : 0) + (int)(f % ld);
  if (!state[sys]) return;
  const double2 b = beta[sys];
  const T br = (T)b.x, bi = (T)b.y;
  const auto zv = z[f], azv = Az[f];
  auto pv = p[f], av = Ap[f];
  p[f] = mk<T>(zv.x + br * pv.x - bi * pv.y, zv.y + br * pv.y + bi * pv.x);
  Ap[f] = mk<T>(azv.x + br * av.x - bi * av.y, azv.y + br * av.y + bi * av.x);
}

// One refinement cycle of COCR for every system with state[s] = 1: the
// correction equation A_hat d = r (r = the FP32/FP64 residual in V[0]) is
// iterated until ||r|| <= max(0.5 tol ||b||, tau_in ||r_0||) or inner_max
// iterations, then x += d in FP64.  Returns SCVS_OK or SCVS_ERR_TIMEOUT (a
// grid barrier of the preconditioner gave up).
template <typename T>
static int cocr_cycle(Ctx &c, Mesh &m, typename cpx<T>::t *V, typename cpx<T>::t *S_scratch, double2 *part,
                      int *upd, CocrState cs, const std::vector<int> &state, const std::vector<double> &n2, double tol,
                      int *h_active, std::vector<int> &iters) {
  using C = typename cpx<T>::t;
  const int ld = m.ld, S = m.n_sys();
  const int64_t total = m.n_dof * ld;
  const unsigned eb = ceil_div(total, 256), sb = ceil_div(S, 128);
  C *r = V, *d = r + total, *z = d + total, *Az = z + total, *p = Az + total, *Ap = p + total, *q = Ap + total;
  const double tau_in = sizeof(T) == 4 ? 1e-5 : 1e-12;
  std::vector<double> tg2(S, 0.0);
  for (int s = 0; s < S; ++s)
    if (state[s]) {
      const double t = std::max(0.5 * tol * m.bnorm[s], tau_in * std::sqrt(std::max(n2[s], 0.0)));
      tg2[s] = t * t;
    }
  SCVS_CUDA(cudaMemcpyAsync(cs.state, state.data(), S * sizeof(int), cudaMemcpyHostToDevice, c.stream));
  SCVS_CUDA(cudaMemcpyAsync(upd, state.data(), S * sizeof(int), cudaMemcpyHostToDevice, c.stream));
  SCVS_CUDA(cudaMemcpyAsync(cs.target2, tg2.data(), S * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  SCVS_CUDA(cudaMemsetAsync(d, 0, total * sizeof(C), c.stream));
  const unsigned db = (unsigned)std::min<int64_t>(m.n_chunk, (int64_t)c.num_sms * 8);
  const double vb = (double)total * sizeof(C);
  auto dot = [&](const C *a, const C *b, const C *nv) {
    KScope ks(c, KC_ARNOLDI, (nv ? 3 : 2) * vb);
    if (nv)
      k_cocr_dot<T, true><<<db, 256, 0, c.stream>>>(a, b, nv, ld, m.n_chunk, m.chunk_row0, m.chunk_rows, m.chunk_comp,
                                                    m.comp_active, part);
    else
      k_cocr_dot<T, false><<<db, 256, 0, c.stream>>>(a, b, nullptr, ld, m.n_chunk, m.chunk_row0, m.chunk_rows,
                                                     m.chunk_comp, m.comp_active, part);
    count_launch(c);
  };
  apply_precond<T>(c, m, r, z, S_scratch, nullptr);
  apply_saddle<T>(c, m, z, Az);
  SCVS_CUDA(cudaMemcpyAsync(p, z, total * sizeof(C), cudaMemcpyDeviceToDevice, c.stream));
  SCVS_CUDA(cudaMemcpyAsync(Ap, Az, total * sizeof(C), cudaMemcpyDeviceToDevice, c.stream));
  dot(z, Az, nullptr);
  k_cocr_init<<<sb, 128, 0, c.stream>>>(cs, m.comp_chunk, S, ld);
  count_launch(c);
  const int inner_max = std::max(1, c.opts.inner_max);
  for (int it = 0; it < inner_max; ++it) {
    apply_precond<T>(c, m, Ap, q, S_scratch, nullptr);
    dot(Ap, q, nullptr);
    k_cocr_alpha<<<sb, 128, 0, c.stream>>>(cs, m.comp_chunk, S, ld);
    {
      KScope ks(c, KC_ARNOLDI, 9 * vb);
      k_cocr_update1<T><<<eb, 256, 0, c.stream>>>(cs.alpha, m.dof_comp, ld, total, p, Ap, q, d, r, z);
    }
    c.launches.n += 2;
    apply_saddle<T>(c, m, z, Az);
    dot(z, Az, r);
    SCVS_CUDA(cudaMemsetAsync(cs.n_active, 0, sizeof(int), c.stream));
    k_cocr_beta<<<sb, 128, 0, c.stream>>>(cs, m.comp_chunk, S, ld, it + 1 == inner_max ? 1 : 0);
    {
      KScope ks(c, KC_ARNOLDI, 6 * vb);
      k_cocr_update2<T><<<eb, 256, 0, c.stream>>>(cs.beta, cs.state, m.dof_comp, ld, total, z, Az, p, Ap);
    }
    c.launches.n += 2;
    SCVS_CUDA(cudaMemcpyAsync(h_active, cs.n_active, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    SCVS_CUDA(cudaStreamSynchronize(c.stream));
    if (*h_active == 0) break;
  }
  int gerr = 0;
  SCVS_CUDA(cudaMemcpyAsync(&gerr, &c.gsync->err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaMemcpyAsync(iters.data(), cs.iters, S * sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  if (gerr) {
    SCVS_CUDA(cudaMemsetAsync(c.gsync, 0, sizeof(GridSync), c.stream));
    SCVS_CUDA(cudaStreamSynchronize(c.stream));
    return SCVS_ERR_TIMEOUT;
  }
  {
    KScope ks(c, KC_VECTOR, (double)total * (32 + sizeof(C)));
    k_add_to_x<T><<<eb, 256, 0, c.stream>>>(d, upd, ld, m.dof_comp, total, m.x);
    count_launch(c);
  }
  return SCVS_OK;
}

template <typename T>
static int solve_mesh_t(Ctx &c, Mesh &m) {
  using C = typename cpx<T>::t;
  const int ld = m.ld, m_r = std::max(1, std::min(64, c.opts.restart));
  const int S = m.n_sys(), nm = m.m;
  const int64_t total = m.n_dof * ld;
  const bool cocr = c.opts.krylov == SCVS_KRYLOV_COCR;
  Work<T> wk;
  wk.s = c.stream;
  wk.pool = c.pool;
  // COCR: 7 work vectors (r, d, z, Az, p, Ap, q); flexible GMRES: the basis V and z_j = P^-1 v_j
  wk.V = wk.template get<C>((size_t)(cocr ? 7 : m_r + 1) * total);
  wk.Z = cocr ? nullptr : wk.template get<C>((size_t)m_r * total);
  wk.W = wk.template get<C>(total);
  wk.S = wk.template get<C>(precond_scratch_elems(m));
  int grid, block;
  size_t smem;
  arnoldi_config<T>(c, ld, m_r, grid, block, smem);
  wk.part = wk.template get<double2>((size_t)m.n_chunk * (m_r + 2) * ld);
  wk.h = wk.template get<double2>((size_t)m.n_comp * (m_r + 2) * ld);
  wk.H = wk.template get<double2>((size_t)S * (m_r + 1) * m_r);
  wk.sn = wk.template get<double2>((size_t)S * m_r);
  wk.gv = wk.template get<double2>((size_t)S * (m_r + 1));
  wk.y = wk.template get<double2>((size_t)S * m_r);
  wk.cs = wk.template get<double>((size_t)S * m_r);
  wk.target = wk.template get<double>(S);
  wk.rscale = wk.template get<double>(S);
  wk.est = wk.template get<double>(S);
  wk.norm2 = wk.template get<double>(S);
  wk.state = wk.template get<int>(S);
  wk.kdim = wk.template get<int>(S);
  wk.upd = wk.template get<int>(S);
  wk.n_active = wk.template get<int>(1);
  CocrState cst{};
  if (cocr) {
    cst.part = wk.part;
    cst.rho = wk.template get<double2>(S);
    cst.alpha = wk.template get<double2>(S);
    cst.beta = wk.template get<double2>(S);
    cst.target2 = wk.template get<double>(S);
    cst.state = wk.state;
    cst.iters = wk.kdim;
    cst.n_active = wk.n_active;
  }

  ArnArgs<T> aa{};
  aa.rows = m.n_dof; aa.ld = ld; aa.m_r = m_r; aa.n_comp = m.n_comp; aa.V = wk.V; aa.w = wk.W; aa.vstride = total;
  aa.n_chunk = m.n_chunk; aa.chunk_row0 = m.chunk_row0; aa.chunk_rows = m.chunk_rows; aa.chunk_comp = m.chunk_comp;
  aa.comp_chunk = m.comp_chunk;
  aa.comp_active = m.comp_active;
  aa.part = wk.part; aa.h = wk.h; aa.H = wk.H; aa.cs = wk.cs; aa.sn = wk.sn; aa.gv = wk.gv;
  aa.state = wk.state; aa.kdim = wk.kdim; aa.target = wk.target; aa.rscale = wk.rscale; aa.est = wk.est;
  aa.n_active = wk.n_active; aa.gs = c.gsync;
  aa.breakdown = sizeof(T) == 4 ? 1e-6 : 1e-13;

  // systems s = comp * ld + k; reports are per (comp, mode): comp * m + k
  const double tol = c.opts.tol;
  m.rep.assign((size_t)m.n_comp * nm, scvs_mode_report{SCVS_MAX_ITER, 0, 0, 0, 0.0, 0.0});
  auto rep = [&](int s) -> scvs_mode_report & { return m.rep[(size_t)(s / ld) * nm + (s % ld)]; };
  std::vector<int> done(S, 0);
  std::vector<double> rel(S, 0.0), best(S, 1e300);
  std::vector<int> since_best(S, 0);
  for (int s = 0; s < S; ++s) {
    if (s % ld >= nm) { done[s] = 1; continue; }  // padding columns
    if (!std::isfinite(m.bnorm[s])) {  // non-finite boundary data: this system only
      done[s] = 1;
      rep(s).status = SCVS_NON_FINITE;
      rep(s).rel_res = m.bnorm[s];
    } else if (m.bnorm[s] == 0.0) {  // zero data: x = 0 (the Dirichlet lift is zero too) is exact
      done[s] = 1;
      rep(s).status = SCVS_CONVERGED;
    }
  }

  const int64_t eb = ceil_div(total, 256);
  const bool warm = c.opts.guess == SCVS_GUESS_CURRENT;
  const bool guess_on = !warm && c.opts.guess == SCVS_GUESS_MLP && m.n_comp == 1 && guess_initial(c, m);
  if (warm) {
    k_warm_x<<<(unsigned)eb, 256, 0, c.stream>>>(m.b, m.dirmask, m.N, m.dim, total, ld, m.x);
    count_launch(c);
  } else if (!guess_on) {
    k_init_x<<<(unsigned)eb, 256, 0, c.stream>>>(m.b, m.dirmask, m.N, m.dim, total, ld, m.x, nullptr, m.dof_comp);
    count_launch(c);
  }
  for (auto &r : m.rep) r.guess_used = (guess_on || warm) ? 1 : 0;
  bool check_guess = guess_on || warm;  // drop a start no better than zero, once

  // CUDA graphs of the Arnoldi steps (opts.graphs; off while the kernel
  // timers run, which record events around every launch)
  StepGraphs graphs(m_r, c.opts.graphs != 0 && !c.timers.on);
  // page-locked word for the per-step active-system count, freed on every exit path
  struct PinnedInt {
    int *p = nullptr;
    ~PinnedInt() { if (p) cudaFreeHost(p); }
  } pinned;
  SCVS_CUDA(cudaMallocHost(&pinned.p, sizeof(int)));
  int *h_active = pinned.p;
  std::vector<double> n2(S);
  std::vector<int> state(S), kd(S);
  const int max_cycles = std::max(1, c.opts.max_cycles);
  for (int cyc = 0; cyc <= max_cycles; ++cyc) {
    // 1. FP64 true residual; r goes to V_0 (unnormalized).  From the zero start
    //    it is the right-hand side itself (no product needed).
    const bool zero_start = cyc == 0 && !warm && !guess_on;
    if constexpr (sizeof(T) == 4)
      residual_fp64(c, m, wk.V, nullptr, wk.norm2, zero_start);
    else
      residual_fp64(c, m, nullptr, wk.V, wk.norm2, zero_start);
    SCVS_CUDA(cudaMemcpyAsync(n2.data(), wk.norm2, S * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    SCVS_CUDA(cudaStreamSynchronize(c.stream));
    if (cyc == 0 && check_guess) {
      // a guess no better than zero is dropped for that mode (zero-start fallback)
      std::vector<int> reset(S, 0);
      int n_reset = 0;
      for (int s = 0; s < S; ++s) {
        if (done[s]) continue;
        const double r = std::sqrt(std::max(n2[s], 0.0));
        if (!(r < m.bnorm[s])) { reset[s] = 1; ++n_reset; rep(s).guess_used = 0; }
      }
      check_guess = false;
      if (n_reset > 0) {
        SCVS_CUDA(cudaMemcpyAsync(wk.upd, reset.data(), S * sizeof(int), cudaMemcpyHostToDevice, c.stream));
        k_init_x<<<(unsigned)eb, 256, 0, c.stream>>>(m.b, m.dirmask, m.N, m.dim, total, ld, m.x, wk.upd, m.dof_comp);
        count_launch(c);
        --cyc;
        continue;
      }
    }
    int n_act = 0;
    for (int s = 0; s < S; ++s) {
      if (done[s]) continue;
      const double r = std::sqrt(std::max(n2[s], 0.0));
      rel[s] = r / m.bnorm[s];
      rep(s).rel_res = rel[s];
      if (cyc == 0) rep(s).res0 = rel[s];
      if (!std::isfinite(rel[s])) { done[s] = 1; rep(s).status = SCVS_NON_FINITE; continue; }
      if (rel[s] <= tol) { done[s] = 1; rep(s).status = SCVS_CONVERGED; continue; }
      // stagnation: 12 cycles without a 1% gain on the best residual so far
      if (rel[s] < 0.99 * best[s]) { best[s] = rel[s]; since_best[s] = 0; }
      else if (++since_best[s] >= 12) { done[s] = 1; rep(s).status = SCVS_STAGNATED; continue; }
      if (cyc == max_cycles) { done[s] = 1; rep(s).status = SCVS_MAX_ITER; continue; }
      ++n_act;
    }
    if (n_act == 0) break;
    if (m.n_comp > 1) {  // components whose systems are all done drop out of every kernel
      std::vector<uint8_t> ca(m.n_comp, 0);
      for (int s = 0; s < S; ++s)
        if (!done[s]) ca[s / ld] = 1;
      SCVS_CUDA(cudaMemcpyAsync(m.comp_active, ca.data(), m.n_comp, cudaMemcpyHostToDevice, c.stream));
    }
    if (cocr) {  // short-recurrence correction of every active system, then the next true residual
      for (int s = 0; s < S; ++s) state[s] = done[s] ? 0 : 1;
      std::vector<int> its(S, 0);
      const int rc = cocr_cycle<T>(c, m, wk.V, wk.S, wk.part, wk.upd, cst, state, n2, tol, h_active, its);
      if (rc != SCVS_OK) return rc;
      for (int s = 0; s < S; ++s)
        if (state[s]) { rep(s).iterations += its[s]; rep(s).cycles += 1; }
      continue;
    }
    // 2. cycle set-up: active systems, targets, first scale, Hessenberg reset
    std::vector<double> tgt(S, 0.0), rs(S, 0.0);
    std::vector<double2> g0((size_t)S * (m_r + 1), make_double2(0, 0));
    for (int s = 0; s < S; ++s) {
      state[s] = done[s] ? 0 : 1;
      if (!state[s]) continue;
      const double beta = std::sqrt(n2[s]);
      rs[s] = 1.0 / beta;
      tgt[s] = 0.5 * tol * m.bnorm[s];
      g0[(size_t)s * (m_r + 1)] = make_double2(beta, 0.0);
    }
    SCVS_CUDA(cudaMemcpyAsync(wk.state, state.data(), S * sizeof(int), cudaMemcpyHostToDevice, c.stream));
    SCVS_CUDA(cudaMemcpyAsync(wk.upd, state.data(), S * sizeof(int), cudaMemcpyHostToDevice, c.stream));
    SCVS_CUDA(cudaMemcpyAsync(wk.target, tgt.data(), S * sizeof(double), cudaMemcpyHostToDevice, c.stream));
    SCVS_CUDA(cudaMemcpyAsync(wk.rscale, rs.data(), S * sizeof(double), cudaMemcpyHostToDevice, c.stream));
    SCVS_CUDA(cudaMemcpyAsync(wk.gv, g0.data(), g0.size() * sizeof(double2), cudaMemcpyHostToDevice, c.stream));
    SCVS_CUDA(cudaMemsetAsync(wk.kdim, 0, S * sizeof(int), c.stream));
    // 3. Arnoldi steps (each step's launches replayed from a CUDA graph when
    //    graphs are on: captured on the step's first use after the first cycle)
    for (int j = 0; j < m_r; ++j) {
      C *Vj = wk.V + (int64_t)j * total, *Zj = wk.Z + (int64_t)j * total;
      auto body = [&]() {
        apply_precond<T>(c, m, Vj, Zj, wk.S, wk.rscale);  // normalizes v_j in place
        apply_saddle<T>(c, m, Zj, wk.W);
        SCVS_CUDA(cudaMemsetAsync(wk.n_active, 0, sizeof(int), c.stream));
        launch_arnoldi<T>(c, aa, j, grid, block, smem);
        SCVS_CUDA(cudaMemcpyAsync(h_active, wk.n_active, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
      };
      if (graphs.on && cyc > 0) {
        if (!graphs.exec[j] && !graphs.capture(c, j, body)) body();  // capture refused: plain launches from now
        if (graphs.exec[j]) graphs.launch(c, j);
      } else {
        body();
      }
      SCVS_CUDA(cudaStreamSynchronize(c.stream));
      if (*h_active == 0) break;
    }
    // a grid barrier that gave up makes every block leave the kernel: the
    // cycle's results are void, report the timeout
    {
      int gerr = 0;
      SCVS_CUDA(cudaMemcpyAsync(&gerr, &c.gsync->err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
      SCVS_CUDA(cudaStreamSynchronize(c.stream));
      if (gerr) {
        SCVS_CUDA(cudaMemsetAsync(c.gsync, 0, sizeof(GridSync), c.stream));
        SCVS_CUDA(cudaStreamSynchronize(c.stream));
        return SCVS_ERR_TIMEOUT;
      }
    }
    // 4. least squares, correction, update
    k_lsq<<<ceil_div(S, 64), 64, 0, c.stream>>>(wk.H, wk.gv, wk.kdim, S, m_r, wk.y);
    count_launch(c);
    SCVS_CUDA(cudaMemcpyAsync(kd.data(), wk.kdim, S * sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    SCVS_CUDA(cudaStreamSynchronize(c.stream));
    int nvmax = 0;
    for (int s = 0; s < S; ++s) {
      if (done[s]) continue;
      nvmax = std::max(nvmax, kd[s]);
      rep(s).iterations += kd[s];
      rep(s).cycles += 1;
    }
    if (nvmax > 0) {
      KScope ks(c, KC_VECTOR, (double)nvmax * total * 2 * sizeof(T) + (double)total * 32);
      k_combine_add<T><<<(unsigned)ceil_div(total, 512), 256, 0, c.stream>>>(wk.Z, total, wk.y, nvmax, ld, S,
                                                                             m.dof_comp, wk.upd, total, m.x);
      count_launch(c);
    }
  }
  if (m.n_comp > 1) SCVS_CUDA(cudaMemsetAsync(m.comp_active, 1, m.n_comp, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  return SCVS_OK;
}

int solve_mesh(Ctx &c, Mesh &m) {
  if (c.opts.precision == SCVS_PREC_FP64) return solve_mesh_t<double>(c, m);
  return solve_mesh_t<float>(c, m);
}

// Self-test of the bounded grid barrier: every block except `absent` (-1: none)
// passes two barriers with the given poll limit; `absent` returns at once, so
// the others' first wait runs out, they set the error word and return.
__global__ void k_barrier_selftest(GridSync *gs, long long spin_limit, int absent, int *passed) {
  if ((int)blockIdx.x == absent) return;
  for (int round = 0; round < 2; ++round)
    if (!grid_sync(gs, gridDim.x, spin_limit)) return;
  if (threadIdx.x == 0) atomicAdd(passed, 1);
}

int barrier_selftest(Ctx &c, long long spin_limit, int n_blocks, int absent, int *passed_out) {
  int *passed = nullptr;
  SCVS_CUDA(ctx_malloc(c, &passed, sizeof(int), c.stream));
  SCVS_CUDA(cudaMemsetAsync(passed, 0, sizeof(int), c.stream));
  void *args[] = {(void *)&c.gsync, (void *)&spin_limit, (void *)&absent, (void *)&passed};
  SCVS_CUDA(cudaLaunchCooperativeKernel((void *)k_barrier_selftest, dim3(n_blocks), dim3(64), args, 0, c.stream));
  count_launch(c);
  int gerr = 0, np = 0;
  SCVS_CUDA(cudaMemcpyAsync(&gerr, &c.gsync->err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaMemcpyAsync(&np, passed, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaFreeAsync(passed, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  *passed_out = np;
  if (gerr) {  // the barrier's count is left mid-round: reset it for the next cooperative kernel
    SCVS_CUDA(cudaMemsetAsync(c.gsync, 0, sizeof(GridSync), c.stream));
    SCVS_CUDA(cudaStreamSynchronize(c.stream));
    return SCVS_ERR_TIMEOUT;
  }
  return SCVS_OK;
}

// The learned start of every mode of a mesh, without solving: x0 from the MLP
// and the POD bases (Dirichlet rows = g), its FP64 relative residual
// ||b - A x0|| / ||b|| per mode, and whether solve_mesh_t would keep it
// (residual below ||b||; otherwise it starts that mode from zero).  x0 is left
// as the mesh's held solution as it is, kept or not.  Returns false if the
// model cannot serve the mesh.
bool guess_probe(Ctx &c, Mesh &m, double *res0, int *kept) {
  if (m.n_comp != 1 || !guess_initial(c, m)) return false;
  const int ld = m.ld;
  double *n2d = nullptr;
  SCVS_CUDA(ctx_malloc(c, &n2d, ld * sizeof(double), c.stream));
  residual_fp64(c, m, nullptr, nullptr, n2d);
  std::vector<double> n2(ld);
  SCVS_CUDA(cudaMemcpyAsync(n2.data(), n2d, ld * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaFreeAsync(n2d, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  for (int k = 0; k < m.m; ++k) {
    const double r = std::sqrt(std::max(n2[k], 0.0)), bn = m.bnorm[k];
    res0[k] = bn > 0.0 ? r / bn : r;
    kept[k] = (bn > 0.0 && r < bn) ? 1 : 0;
  }
  return true;
}

}  // namespace scvs
