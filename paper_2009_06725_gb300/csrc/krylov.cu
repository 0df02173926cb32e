// Batched restarted GMRES over all modes of a mesh (one independent Krylov
// space per mode), right-preconditioned, with an FP64 iterative-refinement
// outer loop.
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
//   3. solves the small triangular systems (FP64), forms d = P^-1 V y and adds
//      it to x in FP64.
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
  int ld, m_r;
  typename cpx<T>::t *V;        // [(m_r+1)][rows][ld]
  const typename cpx<T>::t *w;  // A_hat z
  int64_t vstride;              // rows * ld
  double2 *part;                // [gridDim][m_r+2][ld]
  double2 *h;                   // [m_r+2][ld]
  double2 *H;                   // [ld][m_r+1][m_r]   rotated Hessenberg (R factor)
  double *cs;                   // [ld][m_r]
  double2 *sn;                  // [ld][m_r]
  double2 *gv;                  // [ld][m_r+1]        rotated residual vector
  int *state;                   // [ld] 1 = Arnoldi running for this mode
  int *kdim;                    // [ld] accepted steps in this cycle
  const double *target;         // [ld] residual-estimate target
  double *rscale;               // [ld] 1/||v_{j+1}|| for the next preconditioner step
  double *est;                  // [ld] |g_{j+1}|
  int *n_active;                // [1]
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
  const int64_t ntiles = (a.rows + TR - 1) / TR;
  const bool row_leader = lane32 < TPR;        // holds the warp's row-reduced sums

  // ---------------- phase 1: partial Hermitian products <v_i, w> and ||w||^2
  T *myacc = acc + warp * wstride;
  for (int t = lane32; t < nslots * sstride; t += 32) myacc[t] = T(0);
  __syncwarp();
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    CV<T, MPL> wv[ARN_RPT];
    int64_t rr[ARN_RPT];
#pragma unroll
    for (int q = 0; q < ARN_RPT; ++q) {
      rr[q] = tile * TR + roff + (int64_t)q * RPB;
      if (rr[q] < a.rows) ldv<T, MPL>(wv[q], a.w + rr[q] * ld + koff); else wv[q].zero();
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
        if (rr[q] < a.rows) {
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
  // block partials (warps summed in fixed order) -> global, FP64
  for (int e = threadIdx.x; e < nslots * ld; e += blockDim.x) {
    double re = 0, im = 0;
    for (int w = 0; w < nwarps; ++w) {
      re += (double)acc[w * wstride + 2 * e];
      im += (double)acc[w * wstride + 2 * e + 1];
    }
    a.part[((int64_t)blockIdx.x * (a.m_r + 2)) * ld + e] = make_double2(re, im);
  }
  if (!grid_sync(a.gs, gridDim.x)) return;

  // ---------------- phase 2: grid reduction, one warp per (slot, mode)
  {
    const int items = nslots * ld;
    for (int it = blockIdx.x * nwarps + warp; it < items; it += gridDim.x * nwarps) {
      double re = 0, im = 0;
      for (int b = lane32; b < (int)gridDim.x; b += 32) {
        double2 p = a.part[((int64_t)b * (a.m_r + 2)) * ld + it];
        re += p.x; im += p.y;
      }
      for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
      }
      if (lane32 == 0) a.h[it] = make_double2(re, im);
    }
  }
  if (!grid_sync(a.gs, gridDim.x)) return;

  // ---------------- phase 3: w' = w - sum_i h_i v_i -> V_{j+1}; ||w'||^2 partials
  T *hs = acc;                       // [nvec][ld] complex
  T *nacc = acc + nvec * sstride;    // [nwarps][ld] (re only used)
  for (int e = threadIdx.x; e < nvec * ld; e += blockDim.x) {
    const int k = e % ld;
    double2 hv = a.state[k] ? a.h[e] : make_double2(0.0, 0.0);
    hs[2 * e] = (T)hv.x;
    hs[2 * e + 1] = (T)hv.y;
  }
  for (int e = threadIdx.x; e < nwarps * ld; e += blockDim.x) nacc[2 * e] = T(0);
  __syncthreads();
  bool act[MPL];
#pragma unroll
  for (int i = 0; i < MPL; ++i) act[i] = a.state[koff + i] != 0;
  C *Vn = a.V + (int64_t)(j + 1) * a.vstride;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    CV<T, MPL> wv[ARN_RPT];
    int64_t rr[ARN_RPT];
#pragma unroll
    for (int q = 0; q < ARN_RPT; ++q) {
      rr[q] = tile * TR + roff + (int64_t)q * RPB;
      if (rr[q] < a.rows) ldv<T, MPL>(wv[q], a.w + rr[q] * ld + koff); else wv[q].zero();
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
        if (rr[q] < a.rows) {
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
      if (rr[q] < a.rows) {
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
    double s = 0;
    for (int w = 0; w < nwarps; ++w) s += (double)nacc[2 * (w * ld + k)];
    a.part[((int64_t)blockIdx.x * (a.m_r + 2)) * ld + k] = make_double2(s, 0.0);
  }
  if (!grid_sync(a.gs, gridDim.x)) return;

  // ---------------- phase 4 (block 0): norms, Hessenberg column, Givens, estimate
  if (blockIdx.x != 0) return;
  double *sig2 = reinterpret_cast<double *>(smem_raw);  // [ld]
  __syncthreads();
  for (int k = warp; k < ld; k += nwarps) {
    double s = 0;
    for (int b = lane32; b < (int)gridDim.x; b += 32) s += a.part[((int64_t)b * (a.m_r + 2)) * ld + k].x;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane32 == 0) sig2[k] = s;
  }
  __syncthreads();
  __shared__ int s_active;
  if (threadIdx.x == 0) s_active = 0;
  __syncthreads();
  for (int k = threadIdx.x; k < ld; k += blockDim.x) {
    if (!a.state[k]) { a.rscale[k] = 0.0; continue; }
    const int m_r = a.m_r;
    double2 *Hk = a.H + (int64_t)k * (m_r + 1) * m_r;
    double *csk = a.cs + (int64_t)k * m_r;
    double2 *snk = a.sn + (int64_t)k * m_r;
    double2 *gk = a.gv + (int64_t)k * (m_r + 1);
    const double sigma = sqrt(fmax(sig2[k], 0.0));
    const double wn = sqrt(fmax(a.h[(j + 1) * ld + k].x, 0.0));
    double2 col[2];
    // apply the previous rotations to the new column, top-down
    double2 hprev = a.h[0 * ld + k];
    for (int i = 0; i < j; ++i) {
      const double2 hnext = a.h[(i + 1) * ld + k];
      const double c = csk[i];
      const double2 s = snk[i];
      // t = c h_i + s h_{i+1};  h_{i+1}' = -conj(s) h_i + c h_{i+1}
      double2 t = make_double2(c * hprev.x + s.x * hnext.x - s.y * hnext.y, c * hprev.y + s.x * hnext.y + s.y * hnext.x);
      double2 u = make_double2(-(s.x * hprev.x + s.y * hprev.y) + c * hnext.x, -(s.x * hprev.y - s.y * hprev.x) + c * hnext.y);
      Hk[(int64_t)i * m_r + j] = t;
      hprev = u;
    }
    col[0] = hprev;
    col[1] = make_double2(sigma, 0.0);
    // new rotation zeroing col[1]
    const double aa = sqrt(col[0].x * col[0].x + col[0].y * col[0].y);
    const double r = sqrt(aa * aa + sigma * sigma);
    double c;
    double2 s;
    if (r == 0.0) {
      c = 1.0; s = make_double2(0.0, 0.0);
    } else if (aa == 0.0) {
      c = 0.0; s = make_double2(1.0, 0.0);  // conj(b)/|b| with b = sigma > 0
    } else {
      c = aa / r;
      const double2 ph = make_double2(col[0].x / aa, col[0].y / aa);  // a/|a|
      s = make_double2(ph.x * sigma / r, ph.y * sigma / r);           // (a/|a|) conj(b)/r, b real
    }
    csk[j] = c;
    snk[j] = s;
    const double2 rr = (aa == 0.0) ? make_double2(r, 0.0) : make_double2(col[0].x * r / aa, col[0].y * r / aa);
    Hk[(int64_t)j * m_r + j] = rr;
    const double2 gj = gk[j];
    gk[j + 1] = make_double2(-(s.x * gj.x + s.y * gj.y), -(s.x * gj.y - s.y * gj.x));
    gk[j] = make_double2(c * gj.x, c * gj.y);
    const double e = sqrt(gk[j + 1].x * gk[j + 1].x + gk[j + 1].y * gk[j + 1].y);
    a.est[k] = e;
    a.kdim[k] = j + 1;
    const bool broke = !(sigma > a.breakdown * wn);
    const bool nonfinite = !isfinite(e) || !isfinite(sigma);
    if (nonfinite) { a.kdim[k] = j; }
    if (e <= a.target[k] || broke || nonfinite || j + 1 >= m_r) {
      a.state[k] = 0;
      a.rscale[k] = 0.0;
    } else {
      a.rscale[k] = 1.0 / sigma;
      atomicAdd(&s_active, 1);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) *a.n_active = s_active;
}

// Back substitution R y = g for every mode (FP64); y[i][k], zero past kdim.
__global__ void k_lsq(const double2 *__restrict__ H, const double2 *__restrict__ gv, const int *__restrict__ kdim,
                      int ld, int m_r, double2 *__restrict__ y) {
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

// u = sum_{i<nv} y_i v_i (per mode)
template <typename T>
__global__ void k_combine(const typename cpx<T>::t *__restrict__ V, int64_t vstride, const double2 *__restrict__ y,
                          int nv, int ld, int64_t total, typename cpx<T>::t *__restrict__ u) {
  int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= total) return;
  const int k = (int)(f % ld);
  T re = 0, im = 0;
  for (int i = 0; i < nv; ++i) {
    const double2 yy = y[(int64_t)i * ld + k];
    const auto v = V[(int64_t)i * vstride + f];
    re += (T)yy.x * v.x - (T)yy.y * v.y;
    im += (T)yy.x * v.y + (T)yy.y * v.x;
  }
  u[f] = mk<T>(re, im);
}

template <typename T>
__global__ void k_add_to_x(const typename cpx<T>::t *__restrict__ z, const int *__restrict__ upd, int ld, int64_t total,
                           double2 *__restrict__ x) {
  int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= total) return;
  if (!upd[f % ld]) return;
  const auto d = z[f];
  double2 v = x[f];
  v.x += (double)d.x;
  v.y += (double)d.y;
  x[f] = v;
}

// x = b on Dirichlet rows (= g), 0 elsewhere (only the modes with reset[k] != 0
// when `reset` is given).
__global__ void k_init_x(const double2 *__restrict__ b, const uint8_t *__restrict__ dirm, int64_t N, int dim,
                         int64_t total, int ld, double2 *__restrict__ x, const int *__restrict__ reset) {
  int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= total) return;
  if (reset && !reset[f % ld]) return;
  const int64_t dof = f / ld;
  const bool dir = dof < N * dim && dirm[dof / dim];
  x[f] = dir ? b[f] : make_double2(0.0, 0.0);
}

template <typename T>
struct Work {
  using C = typename cpx<T>::t;
  C *V = nullptr, *Z = nullptr, *W = nullptr, *S = nullptr;
  double2 *part = nullptr, *h = nullptr, *H = nullptr, *sn = nullptr, *gv = nullptr, *y = nullptr;
  double *cs = nullptr, *target = nullptr, *rscale = nullptr, *est = nullptr, *norm2 = nullptr;
  int *state = nullptr, *kdim = nullptr, *n_active = nullptr, *upd = nullptr;
  std::vector<void *> owned;
  cudaStream_t s = nullptr;
  template <typename U> U *get(size_t n) {
    void *p = nullptr;
    SCVS_CUDA(cudaMallocAsync(&p, std::max<size_t>(n, 1) * sizeof(U), s));
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

template <typename T>
static int solve_mesh_t(Ctx &c, Mesh &m) {
  using C = typename cpx<T>::t;
  const int ld = m.ld, m_r = std::max(1, std::min(64, c.opts.restart));
  const int64_t total = m.n_dof * ld;
  Work<T> wk;
  wk.s = c.stream;
  wk.V = wk.template get<C>((size_t)(m_r + 1) * total);
  wk.Z = wk.template get<C>(total);
  wk.W = wk.template get<C>(total);
  wk.S = wk.template get<C>(precond_scratch_elems(m));
  int grid, block;
  size_t smem;
  arnoldi_config<T>(c, ld, m_r, grid, block, smem);
  wk.part = wk.template get<double2>((size_t)grid * (m_r + 2) * ld);
  wk.h = wk.template get<double2>((size_t)(m_r + 2) * ld);
  wk.H = wk.template get<double2>((size_t)ld * (m_r + 1) * m_r);
  wk.sn = wk.template get<double2>((size_t)ld * m_r);
  wk.gv = wk.template get<double2>((size_t)ld * (m_r + 1));
  wk.y = wk.template get<double2>((size_t)ld * m_r);
  wk.cs = wk.template get<double>((size_t)ld * m_r);
  wk.target = wk.template get<double>(ld);
  wk.rscale = wk.template get<double>(ld);
  wk.est = wk.template get<double>(ld);
  wk.norm2 = wk.template get<double>(ld);
  wk.state = wk.template get<int>(ld);
  wk.kdim = wk.template get<int>(ld);
  wk.upd = wk.template get<int>(ld);
  wk.n_active = wk.template get<int>(1);

  ArnArgs<T> aa{};
  aa.rows = m.n_dof; aa.ld = ld; aa.m_r = m_r; aa.V = wk.V; aa.w = wk.W; aa.vstride = total;
  aa.part = wk.part; aa.h = wk.h; aa.H = wk.H; aa.cs = wk.cs; aa.sn = wk.sn; aa.gv = wk.gv;
  aa.state = wk.state; aa.kdim = wk.kdim; aa.target = wk.target; aa.rscale = wk.rscale; aa.est = wk.est;
  aa.n_active = wk.n_active; aa.gs = c.gsync;
  aa.breakdown = sizeof(T) == 4 ? 1e-6 : 1e-13;

  const double tol = c.opts.tol;
  m.rep.assign(m.m, scvs_mode_report{SCVS_MAX_ITER, 0, 0, 0, 0.0});
  std::vector<int> done(ld, 0);
  std::vector<double> rel(ld, 0.0), best(ld, 1e300);
  std::vector<int> since_best(ld, 0);
  for (int k = m.m; k < ld; ++k) done[k] = 1;  // padding columns
  for (int k = 0; k < m.m; ++k) {
    if (!std::isfinite(m.bnorm[k])) {  // non-finite boundary data: this mode only
      done[k] = 1;
      m.rep[k].status = SCVS_NON_FINITE;
      m.rep[k].rel_res = m.bnorm[k];
    } else if (m.bnorm[k] == 0.0) {  // zero data: x = 0 (the Dirichlet lift is zero too) is exact
      done[k] = 1;
      m.rep[k].status = SCVS_CONVERGED;
    }
  }

  const int64_t eb = ceil_div(total, 256);
  bool guess_on = c.opts.guess == SCVS_GUESS_MLP && guess_initial(c, m);
  if (!guess_on) {
    k_init_x<<<(unsigned)eb, 256, 0, c.stream>>>(m.b, m.dirmask, m.N, m.dim, total, ld, m.x, nullptr);
    count_launch(c);
  }
  for (int k = 0; k < m.m; ++k) m.rep[k].guess_used = guess_on ? 1 : 0;

  int *h_active = nullptr;
  SCVS_CUDA(cudaMallocHost(&h_active, sizeof(int)));
  std::vector<double> n2(ld), hbuf(ld);
  std::vector<int> state(ld), kd(ld);
  const int max_cycles = std::max(1, c.opts.max_cycles);
  for (int cyc = 0; cyc <= max_cycles; ++cyc) {
    // 1. FP64 true residual; r goes to V_0 (unnormalized)
    if constexpr (sizeof(T) == 4)
      residual_fp64(c, m, wk.V, nullptr, wk.norm2);
    else
      residual_fp64(c, m, nullptr, wk.V, wk.norm2);
    SCVS_CUDA(cudaMemcpyAsync(n2.data(), wk.norm2, ld * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    SCVS_CUDA(cudaStreamSynchronize(c.stream));
    if (cyc == 0 && guess_on) {
      // a guess no better than zero is dropped for that mode (zero-start fallback)
      std::vector<int> reset(ld, 0);
      int n_reset = 0;
      for (int k = 0; k < m.m; ++k) {
        if (done[k]) continue;
        const double r = std::sqrt(std::max(n2[k], 0.0));
        if (!(r < m.bnorm[k])) { reset[k] = 1; ++n_reset; m.rep[k].guess_used = 0; }
      }
      guess_on = false;
      if (n_reset > 0) {
        SCVS_CUDA(cudaMemcpyAsync(wk.upd, reset.data(), ld * sizeof(int), cudaMemcpyHostToDevice, c.stream));
        k_init_x<<<(unsigned)eb, 256, 0, c.stream>>>(m.b, m.dirmask, m.N, m.dim, total, ld, m.x, wk.upd);
        count_launch(c);
        --cyc;
        continue;
      }
    }
    int n_act = 0;
    for (int k = 0; k < m.m; ++k) {
      if (done[k]) continue;
      const double r = std::sqrt(std::max(n2[k], 0.0));
      rel[k] = r / m.bnorm[k];
      m.rep[k].rel_res = rel[k];
      if (!std::isfinite(rel[k])) { done[k] = 1; m.rep[k].status = SCVS_NON_FINITE; continue; }
      if (rel[k] <= tol) { done[k] = 1; m.rep[k].status = SCVS_CONVERGED; continue; }
      // stagnation: 12 cycles without a 1% gain on the best residual so far
      if (rel[k] < 0.99 * best[k]) { best[k] = rel[k]; since_best[k] = 0; }
      else if (++since_best[k] >= 12) { done[k] = 1; m.rep[k].status = SCVS_STAGNATED; continue; }
      if (cyc == max_cycles) { done[k] = 1; m.rep[k].status = SCVS_MAX_ITER; continue; }
      done[k] = 0;
      ++n_act;
    }
    if (n_act == 0) break;
    // 2. cycle set-up: active modes, targets, first scale, Hessenberg reset
    std::vector<double> tgt(ld, 0.0), rs(ld, 0.0);
    std::vector<double2> g0((size_t)ld * (m_r + 1), make_double2(0, 0));
    for (int k = 0; k < ld; ++k) {
      state[k] = done[k] ? 0 : 1;
      if (!state[k]) continue;
      const double beta = std::sqrt(n2[k]);
      rs[k] = 1.0 / beta;
      tgt[k] = 0.5 * tol * m.bnorm[k];
      g0[(size_t)k * (m_r + 1)] = make_double2(beta, 0.0);
    }
    SCVS_CUDA(cudaMemcpyAsync(wk.state, state.data(), ld * sizeof(int), cudaMemcpyHostToDevice, c.stream));
    SCVS_CUDA(cudaMemcpyAsync(wk.upd, state.data(), ld * sizeof(int), cudaMemcpyHostToDevice, c.stream));
    SCVS_CUDA(cudaMemcpyAsync(wk.target, tgt.data(), ld * sizeof(double), cudaMemcpyHostToDevice, c.stream));
    SCVS_CUDA(cudaMemcpyAsync(wk.rscale, rs.data(), ld * sizeof(double), cudaMemcpyHostToDevice, c.stream));
    SCVS_CUDA(cudaMemcpyAsync(wk.gv, g0.data(), g0.size() * sizeof(double2), cudaMemcpyHostToDevice, c.stream));
    SCVS_CUDA(cudaMemsetAsync(wk.kdim, 0, ld * sizeof(int), c.stream));
    // 3. Arnoldi steps
    int steps = 0;
    for (int j = 0; j < m_r; ++j) {
      C *Vj = wk.V + (int64_t)j * total;
      apply_precond<T>(c, m, Vj, wk.Z, wk.S, wk.rscale);  // normalizes v_j in place
      apply_saddle<T>(c, m, wk.Z, wk.W);
      launch_arnoldi<T>(c, aa, j, grid, block, smem);
      ++steps;
      SCVS_CUDA(cudaMemcpyAsync(h_active, wk.n_active, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
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
        cudaFreeHost(h_active);
        return SCVS_ERR_TIMEOUT;
      }
    }
    // 4. least squares, correction, update
    k_lsq<<<ceil_div(ld, 64), 64, 0, c.stream>>>(wk.H, wk.gv, wk.kdim, ld, m_r, wk.y);
    count_launch(c);
    SCVS_CUDA(cudaMemcpyAsync(kd.data(), wk.kdim, ld * sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    SCVS_CUDA(cudaStreamSynchronize(c.stream));
    int nvmax = 0;
    for (int k = 0; k < m.m; ++k) {
      if (done[k]) continue;
      nvmax = std::max(nvmax, kd[k]);
      m.rep[k].iterations += kd[k];
      m.rep[k].cycles += 1;
    }
    if (nvmax > 0) {
      {
        KScope ks(c, KC_VECTOR, (double)(nvmax + 1) * total * 2 * sizeof(T));
        k_combine<T><<<(unsigned)eb, 256, 0, c.stream>>>(wk.V, total, wk.y, nvmax, ld, total, wk.W);
        count_launch(c);
      }
      apply_precond<T>(c, m, wk.W, wk.Z, wk.S, nullptr);
      {
        KScope ks(c, KC_VECTOR, (double)total * (32 + 2 * sizeof(T)));
        k_add_to_x<T><<<(unsigned)eb, 256, 0, c.stream>>>(wk.Z, wk.upd, ld, total, m.x);
        count_launch(c);
      }
    }
    (void)steps;
  }
  cudaFreeHost(h_active);
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  return SCVS_OK;
}

int solve_mesh(Ctx &c, Mesh &m) {
  if (c.opts.precision == SCVS_PREC_FP64) return solve_mesh_t<double>(c, m);
  return solve_mesh_t<float>(c, m);
}

}  // namespace scvs
