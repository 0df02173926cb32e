// Learned initial guess for the per-mode solves (training and inference).
//
// Snapshots: converged modal solutions x_k of solved meshes, divided by the
// mode's boundary coefficient c_k (the problem is linear in c_k), stored as
// complex FP32 columns of length n_dof together with the mode features
// f = (omega_k, Re c_k, Im c_k, R, s).
// POD (method of snapshots, per field block u / p): Gram matrix X^H X by a
// complex GEMM, its leading eigenpairs on the host (cyclic Jacobi), basis
// Phi = X V Lambda^{-1/2}; training targets a = Phi^H x.
// MLP 5 -> H -> H -> H -> 4 n_pod with exact GELU on the hidden layers; the
// weights used by the forward/backward kernels are BF16 (FP32 master copies
// updated by Adam), every product is accumulated in FP32.
// Inference: x0 = c_k [Phi_u a_u; Phi_p a_p] on the free rows, g on the
// Dirichlet rows.
#include <cublas_v2.h>
#include <cuda_bf16.h>
#include <algorithm>
#include <cmath>
#include <complex>
#include <random>
#include <vector>
#include "scvs_internal.h"

namespace scvs {

#define SCVS_CUBLAS(call)                                                                \
  do {                                                                                  \
    cublasStatus_t _s = (call);                                                         \
    if (_s != CUBLAS_STATUS_SUCCESS) throw CudaError{cudaErrorUnknown, std::string(#call) + " (cuBLAS)"}; \
  } while (0)

// ------------------------------------------------------------ MLP kernels
constexpr int MLP_TB = 16;  // samples per block

__device__ __forceinline__ float gelu_f(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_grad_f(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// Z = A W + b (W BF16 [in][out], row = input neuron), A_out = gelu(Z) or Z.
// Block: 256 threads = output neurons j (grid.y tiles out), MLP_TB samples.
__global__ void __launch_bounds__(256) k_mlp_fwd(const float *__restrict__ A, int in, int out,
                                                 const __nv_bfloat16 *__restrict__ W,
                                                 const __nv_bfloat16 *__restrict__ bias, int64_t B,
                                                 float *__restrict__ Z, float *__restrict__ Aout, int act) {
  extern __shared__ float xs[];  // [MLP_TB][in]
  const int64_t s0 = (int64_t)blockIdx.x * MLP_TB;
  const int j = blockIdx.y * blockDim.x + threadIdx.x;
  for (int t = threadIdx.x; t < MLP_TB * in; t += blockDim.x) {
    const int s = t / in, i = t % in;
    xs[t] = (s0 + s < B) ? A[(s0 + s) * in + i] : 0.0f;
  }
  __syncthreads();
  if (j >= out) return;
  float acc[MLP_TB];
#pragma unroll
  for (int s = 0; s < MLP_TB; ++s) acc[s] = 0.0f;
  for (int i = 0; i < in; ++i) {
    const float w = __bfloat162float(W[(int64_t)i * out + j]);
#pragma unroll
    for (int s = 0; s < MLP_TB; ++s) acc[s] = fmaf(xs[s * in + i], w, acc[s]);
  }
  const float b = __bfloat162float(bias[j]);
#pragma unroll
  for (int s = 0; s < MLP_TB; ++s) {
    if (s0 + s >= B) break;
    const float z = acc[s] + b;
    if (Z) Z[(s0 + s) * out + j] = z;
    Aout[(s0 + s) * out + j] = act ? gelu_f(z) : z;
  }
}

// delta of the last layer for L = sum (y - t)^2 / (B n_out); loss partials.
__global__ void k_mse_delta(const float *__restrict__ y, const float *__restrict__ t, int64_t n, float scale,
                            float *__restrict__ d, float *__restrict__ loss) {
  __shared__ float s[256];
  float acc = 0.0f;
  for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) {
    const float e = y[i] - t[i];
    d[i] = 2.0f * e * scale;
    acc += e * e;
  }
  s[threadIdx.x] = acc;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, s[0] * scale);
}

// delta_l = (delta_{l+1} W^T) * gelu'(Z_l); Wt BF16 [out][in] (transposed copy).
__global__ void __launch_bounds__(256) k_mlp_bwd(const float *__restrict__ dnext, int in, int out,
                                                 const __nv_bfloat16 *__restrict__ Wt, const float *__restrict__ Z,
                                                 int64_t B, float *__restrict__ d) {
  extern __shared__ float ds[];  // [MLP_TB][out]
  const int64_t s0 = (int64_t)blockIdx.x * MLP_TB;
  const int i = blockIdx.y * blockDim.x + threadIdx.x;
  for (int t = threadIdx.x; t < MLP_TB * out; t += blockDim.x) {
    const int s = t / out, j = t % out;
    ds[t] = (s0 + s < B) ? dnext[(s0 + s) * out + j] : 0.0f;
  }
  __syncthreads();
  if (i >= in) return;
  float acc[MLP_TB];
#pragma unroll
  for (int s = 0; s < MLP_TB; ++s) acc[s] = 0.0f;
  for (int j = 0; j < out; ++j) {
    const float w = __bfloat162float(Wt[(int64_t)j * in + i]);
#pragma unroll
    for (int s = 0; s < MLP_TB; ++s) acc[s] = fmaf(ds[s * out + j], w, acc[s]);
  }
#pragma unroll
  for (int s = 0; s < MLP_TB; ++s) {
    if (s0 + s >= B) break;
    d[(s0 + s) * in + i] = acc[s] * gelu_grad_f(Z[(s0 + s) * in + i]);
  }
}

// dW[i][j] = sum_s A[s][i] delta[s][j]; db[j] = sum_s delta[s][j].
// Block: 256 threads over j, 8 input rows i per block (grid.x), grid.y tiles j.
__global__ void __launch_bounds__(256) k_mlp_wgrad(const float *__restrict__ A, const float *__restrict__ dl, int in,
                                                   int out, int64_t B, float *__restrict__ dW,
                                                   float *__restrict__ db) {
  const int j = blockIdx.y * blockDim.x + threadIdx.x;
  const int i0 = blockIdx.x * 8;
  if (j >= out) return;
  float acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  float bacc = 0.0f;
  for (int64_t s = 0; s < B; ++s) {
    const float dv = dl[s * out + j];
#pragma unroll
    for (int q = 0; q < 8; ++q)
      if (i0 + q < in) acc[q] = fmaf(A[s * in + i0 + q], dv, acc[q]);
    bacc += dv;
  }
#pragma unroll
  for (int q = 0; q < 8; ++q)
    if (i0 + q < in) dW[(int64_t)(i0 + q) * out + j] = acc[q];
  if (blockIdx.x == 0) db[j] = bacc;
}

// Adam on the FP32 master weights; refreshes the BF16 working copy.
__global__ void k_adam(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m, float *__restrict__ v,
                       int64_t n, float lr, float b1, float b2, float eps, float c1, float c2,
                       __nv_bfloat16 *__restrict__ wb) {
  const int64_t i = blockIdx.x * 256ll + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.0f - b1) * gi;
  const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  w[i] = wi;
  wb[i] = __float2bfloat16_rn(wi);
}

__global__ void k_to_bf16(const float *__restrict__ w, int64_t n, __nv_bfloat16 *__restrict__ wb) {
  const int64_t i = blockIdx.x * 256ll + threadIdx.x;
  if (i < n) wb[i] = __float2bfloat16_rn(w[i]);
}

// Wt[j][i] = W[i][j] (BF16)
__global__ void k_transpose_bf16(const __nv_bfloat16 *__restrict__ W, int in, int out, __nv_bfloat16 *__restrict__ Wt) {
  const int64_t t = blockIdx.x * 256ll + threadIdx.x;
  if (t >= (int64_t)in * out) return;
  const int i = (int)(t / out), j = (int)(t % out);
  Wt[(int64_t)j * in + i] = W[t];
}

// --------------------------------------------------------- guess kernels
// x[dof][k] = c_k sum_i Phi[dof][i] a[k][i] on free rows; b (= g) on Dirichlet rows.
__global__ void k_guess_expand(const float2 *__restrict__ Phi_u, const float2 *__restrict__ Phi_p, int n_pod,
                               const float2 *__restrict__ au, const float2 *__restrict__ ap,
                               const double2 *__restrict__ cmode, int m, int ld, int64_t n_u, int64_t n_dof,
                               const uint8_t *__restrict__ dirm, int dim, const double2 *__restrict__ b,
                               double2 *__restrict__ x) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= n_dof * ld) return;
  const int64_t dof = f / ld;
  const int k = (int)(f % ld);
  if (dof < n_u && dirm[dof / dim]) { x[f] = b[f]; return; }
  if (k >= m) { x[f] = make_double2(0.0, 0.0); return; }
  const bool isu = dof < n_u;
  const float2 *Phi = isu ? Phi_u + dof * n_pod : Phi_p + (dof - n_u) * n_pod;
  const float2 *a = (isu ? au : ap) + (int64_t)k * n_pod;
  float re = 0.0f, im = 0.0f;
  for (int i = 0; i < n_pod; ++i) {
    const float2 p = __ldg(Phi + i), c = __ldg(a + i);
    re = fmaf(p.x, c.x, fmaf(-p.y, c.y, re));
    im = fmaf(p.x, c.y, fmaf(p.y, c.x, im));
  }
  const double2 ck = cmode[k];
  x[f] = make_double2(ck.x * re - ck.y * im, ck.x * im + ck.y * re);
}

// snapshot column: x[dof][k] / c_k -> FP32 complex [n_dof]
__global__ void k_snapshot(const double2 *__restrict__ x, int64_t n_dof, int ld, int k, double2 c, float2 *__restrict__ out) {
  const int64_t d = blockIdx.x * 256ll + threadIdx.x;
  if (d >= n_dof) return;
  const double2 v = x[d * ld + k];
  const double den = c.x * c.x + c.y * c.y;
  out[d] = make_float2((float)((v.x * c.x + v.y * c.y) / den), (float)((v.y * c.x - v.x * c.y) / den));
}

// --------------------------------------------------------- host helpers
// Cyclic Jacobi eigen-decomposition of a Hermitian matrix (column-major,
// n x n); returns eigenvalues descending and the matching eigenvectors.
static void hermitian_eig(int n, std::vector<std::complex<double>> A, std::vector<double> &lam,
                          std::vector<std::complex<double>> &V) {
  using cd = std::complex<double>;
  V.assign((size_t)n * n, cd(0, 0));
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  auto at = [&](int r, int c) -> cd & { return A[(size_t)c * n + r]; };
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int c = 0; c < n; ++c)
      for (int r = 0; r < n; ++r) {
        const double a2 = std::norm(at(r, c));
        tot += a2;
        if (r != c) off += a2;
      }
    if (off <= 1e-26 * tot) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const cd apq = at(p, q);
        const double mag = std::abs(apq);
        if (mag < 1e-300) continue;
        const double app = at(p, p).real(), aqq = at(q, q).real();
        // A -> J^H A J with J acting on (p, q); phase e = apq/|apq| makes the
        // 2x2 block real symmetric [app mag; mag aqq]
        const cd e = apq / mag;
        const double tau = (aqq - app) / (2.0 * mag);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = t * cs;
        // columns: col_p' = cs col_p - sn conj(e) col_q ; col_q' = sn e col_p + cs col_q
        for (int r = 0; r < n; ++r) {
          const cd ap = at(r, p), aq = at(r, q);
          at(r, p) = cs * ap - sn * std::conj(e) * aq;
          at(r, q) = sn * e * ap + cs * aq;
        }
        for (int c = 0; c < n; ++c) {
          const cd ap = at(p, c), aq = at(q, c);
          at(p, c) = cs * ap - sn * e * aq;
          at(q, c) = sn * std::conj(e) * ap + cs * aq;
        }
        for (int r = 0; r < n; ++r) {
          const cd vp = V[(size_t)p * n + r], vq = V[(size_t)q * n + r];
          V[(size_t)p * n + r] = cs * vp - sn * std::conj(e) * vq;
          V[(size_t)q * n + r] = sn * e * vp + cs * vq;
        }
      }
  }
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return at(a, a).real() > at(b, b).real(); });
  lam.resize(n);
  std::vector<cd> Vs((size_t)n * n);
  for (int i = 0; i < n; ++i) {
    lam[i] = at(ord[i], ord[i]).real();
    for (int r = 0; r < n; ++r) Vs[(size_t)i * n + r] = V[(size_t)ord[i] * n + r];
  }
  V.swap(Vs);
}

static unsigned grid1(int64_t n) { return ceil_div(n, 256); }

// Run the raw MLP on [B][in] device inputs; saves pre-activations and
// activations of every layer in `w` (sized for B) when `keep`.
void mlp_forward(Ctx &c, GuessModel &g, const float *x, int64_t B, float *y) {
  g.ensure(B);
  const int H = g.hidden;
  const float *in = x;
  for (int l = 0; l < 4; ++l) {
    const int di = g.dims[l], dout = g.dims[l + 1];
    float *Z = g.zbuf(l), *A = (l == 3) ? y : g.abuf(l);
    dim3 grid(ceil_div(B, MLP_TB), ceil_div(dout, 256));
    k_mlp_fwd<<<grid, 256, MLP_TB * di * sizeof(float), c.stream>>>(in, di, dout, g.Wb + g.woff[l], g.Wb + g.boff[l],
                                                                     B, Z, A, l < 3);
    count_launch(c);
    in = A;
  }
  (void)H;
}

// Gradients of the MSE against targets t for a batch; returns into g.grad.
float mlp_gradient(Ctx &c, GuessModel &g, const float *x, const float *t, int64_t B) {
  g.ensure(B);
  float *y = g.ybuf();
  mlp_forward(c, g, x, B, y);
  float *loss = g.scal;
  SCVS_CUDA(cudaMemsetAsync(loss, 0, sizeof(float), c.stream));
  float *dcur = g.dbuf(0), *dprev = g.dbuf(1);
  const int64_t ny = B * g.n_out;
  k_mse_delta<<<std::min<unsigned>(grid1(ny), 1024), 256, 0, c.stream>>>(y, t, ny, 1.0f / (float)ny, dcur, loss);
  count_launch(c);
  for (int l = 3; l >= 0; --l) {
    const int di = g.dims[l], dout = g.dims[l + 1];
    const float *Ain = (l == 0) ? x : g.abuf(l - 1);
    dim3 gw(ceil_div(di, 8), ceil_div(dout, 256));
    k_mlp_wgrad<<<gw, 256, 0, c.stream>>>(Ain, dcur, di, dout, B, g.grad + g.woff[l], g.grad + g.boff[l]);
    count_launch(c);
    if (l > 0) {
      dim3 gb(ceil_div(B, MLP_TB), ceil_div(di, 256));
      k_mlp_bwd<<<gb, 256, MLP_TB * dout * sizeof(float), c.stream>>>(dcur, di, dout, g.Wt + g.woff[l], g.zbuf(l - 1),
                                                                      B, dprev);
      count_launch(c);
      std::swap(dcur, dprev);
    }
  }
  float h = 0;
  SCVS_CUDA(cudaMemcpyAsync(&h, loss, sizeof(float), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  return h;
}

void mlp_refresh_bf16(Ctx &c, GuessModel &g) {
  k_to_bf16<<<grid1(g.n_params), 256, 0, c.stream>>>(g.Wf, g.n_params, g.Wb);
  count_launch(c);
  for (int l = 0; l < 4; ++l) {
    k_transpose_bf16<<<grid1((int64_t)g.dims[l] * g.dims[l + 1]), 256, 0, c.stream>>>(g.Wb + g.woff[l], g.dims[l],
                                                                                      g.dims[l + 1], g.Wt + g.woff[l]);
    count_launch(c);
  }
}

void mlp_alloc(GuessModel &g, int n_in, int hidden, int n_out) {
  g.release_mlp();
  g.hidden = hidden;
  g.n_out = n_out;
  g.dims[0] = n_in; g.dims[1] = hidden; g.dims[2] = hidden; g.dims[3] = hidden; g.dims[4] = n_out;
  int64_t off = 0;
  for (int l = 0; l < 4; ++l) {
    g.woff[l] = off;
    off += (int64_t)g.dims[l] * g.dims[l + 1];
    g.boff[l] = off;
    off += g.dims[l + 1];
  }
  g.n_params = off;
  SCVS_CUDA(cudaMalloc(&g.Wf, off * sizeof(float)));
  SCVS_CUDA(cudaMalloc(&g.grad, off * sizeof(float)));
  SCVS_CUDA(cudaMalloc(&g.am, off * sizeof(float)));
  SCVS_CUDA(cudaMalloc(&g.av, off * sizeof(float)));
  SCVS_CUDA(cudaMalloc(&g.Wb, off * sizeof(__nv_bfloat16)));
  SCVS_CUDA(cudaMalloc(&g.Wt, off * sizeof(__nv_bfloat16)));
  SCVS_CUDA(cudaMalloc(&g.scal, 16 * sizeof(float)));
  SCVS_CUDA(cudaMemset(g.am, 0, off * sizeof(float)));
  SCVS_CUDA(cudaMemset(g.av, 0, off * sizeof(float)));
  g.adam_t = 0;
}

void mlp_adam(Ctx &c, GuessModel &g, float lr) {
  g.adam_t += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.0f - std::pow(b1, (float)g.adam_t), c2 = 1.0f - std::pow(b2, (float)g.adam_t);
  k_adam<<<grid1(g.n_params), 256, 0, c.stream>>>(g.Wf, g.grad, g.am, g.av, g.n_params, lr, b1, b2, 1e-8f, c1, c2, g.Wb);
  count_launch(c);
  for (int l = 0; l < 4; ++l) {
    k_transpose_bf16<<<grid1((int64_t)g.dims[l] * g.dims[l + 1]), 256, 0, c.stream>>>(g.Wb + g.woff[l], g.dims[l],
                                                                                      g.dims[l + 1], g.Wt + g.woff[l]);
    count_launch(c);
  }
}

// ------------------------------------------------------------- snapshots
void guess_add_snapshots(Ctx &c, Mesh &m, const double *features) {
  GuessModel &g = c.guess;
  if (g.n_dof == 0) {
    g.n_dof = m.n_dof;
    g.n_u = (int64_t)m.dim * m.N;
  } else if (g.n_dof != m.n_dof || g.n_u != (int64_t)m.dim * m.N) {
    throw (int)SCVS_ERR_ARG;  // snapshots must share the node set
  }
  for (int k = 0; k < m.m; ++k) {
    if (m.rep.empty() || m.rep[k].status != SCVS_CONVERGED) continue;
    const double cr = features[k * 5 + 1], ci = features[k * 5 + 2];
    if (cr * cr + ci * ci == 0.0) continue;
    if (g.n_snap == g.snap_cap) {
      const int64_t cap = std::max<int64_t>(64, g.snap_cap * 2);
      float2 *nx = nullptr;
      SCVS_CUDA(cudaMalloc(&nx, (size_t)cap * g.n_dof * sizeof(float2)));
      if (g.snap) {
        SCVS_CUDA(cudaMemcpyAsync(nx, g.snap, (size_t)g.n_snap * g.n_dof * sizeof(float2), cudaMemcpyDeviceToDevice,
                                  c.stream));
        SCVS_CUDA(cudaStreamSynchronize(c.stream));
        cudaFree(g.snap);
      }
      g.snap = nx;
      g.snap_cap = cap;
    }
    k_snapshot<<<grid1(m.n_dof), 256, 0, c.stream>>>(m.x, m.n_dof, m.ld, k, make_double2(cr, ci),
                                                     g.snap + (size_t)g.n_snap * g.n_dof);
    count_launch(c);
    for (int q = 0; q < 5; ++q) g.feat.push_back(features[k * 5 + q]);
    g.n_snap += 1;
  }
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
}

// POD of one block (rows [r0, r0 + nr) of the snapshots) -> Phi [nr][n_pod]
// row-major complex FP32; also the coefficients a [n_snap][n_pod].
static void pod_block(Ctx &c, GuessModel &g, cublasHandle_t h, int64_t r0, int64_t nr, int n_pod_req, int n_basis,
                      float2 **Phi_out, std::vector<std::complex<float>> &coef, int &n_pod_out) {
  const int S = (int)g.n_snap, Sb = std::min<int>(S, n_basis);
  const cuComplex one = make_cuComplex(1, 0), zero = make_cuComplex(0, 0);
  const cuComplex *X = reinterpret_cast<const cuComplex *>(g.snap + r0);  // column-major nr x S, lda = n_dof
  cuComplex *G = nullptr;
  SCVS_CUDA(cudaMalloc(&G, (size_t)Sb * Sb * sizeof(cuComplex)));
  SCVS_CUBLAS(cublasCgemm(h, CUBLAS_OP_C, CUBLAS_OP_N, Sb, Sb, (int)nr, &one, X, (int)g.n_dof, X, (int)g.n_dof, &zero,
                          G, Sb));
  std::vector<std::complex<float>> hg((size_t)Sb * Sb);
  SCVS_CUDA(cudaMemcpyAsync(hg.data(), G, hg.size() * sizeof(cuComplex), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  std::vector<std::complex<double>> A(hg.size());
  for (size_t i = 0; i < hg.size(); ++i) A[i] = std::complex<double>(hg[i].real(), hg[i].imag());
  for (int i = 0; i < Sb; ++i)  // exact Hermitian symmetry
    for (int j = i + 1; j < Sb; ++j) {
      const auto v = 0.5 * (A[(size_t)j * Sb + i] + std::conj(A[(size_t)i * Sb + j]));
      A[(size_t)j * Sb + i] = v;
      A[(size_t)i * Sb + j] = std::conj(v);
    }
  std::vector<double> lam;
  std::vector<std::complex<double>> V;
  hermitian_eig(Sb, A, lam, V);
  int r = 0;
  while (r < std::min(n_pod_req, Sb) && lam[r] > 1e-10 * lam[0]) ++r;
  n_pod_out = r;
  // W = V_r Lambda_r^{-1/2}  (Sb x r), Phi = X_b W  (nr x r, column-major)
  std::vector<cuComplex> Wh((size_t)Sb * r);
  for (int j = 0; j < r; ++j)
    for (int i = 0; i < Sb; ++i) {
      const auto v = V[(size_t)j * Sb + i] / std::sqrt(lam[j]);
      Wh[(size_t)j * Sb + i] = make_cuComplex((float)v.real(), (float)v.imag());
    }
  cuComplex *Wd = nullptr, *Pc = nullptr, *Cd = nullptr;
  SCVS_CUDA(cudaMalloc(&Wd, Wh.size() * sizeof(cuComplex)));
  SCVS_CUDA(cudaMalloc(&Pc, (size_t)nr * r * sizeof(cuComplex)));
  SCVS_CUDA(cudaMalloc(&Cd, (size_t)r * S * sizeof(cuComplex)));
  SCVS_CUDA(cudaMemcpyAsync(Wd, Wh.data(), Wh.size() * sizeof(cuComplex), cudaMemcpyHostToDevice, c.stream));
  SCVS_CUBLAS(cublasCgemm(h, CUBLAS_OP_N, CUBLAS_OP_N, (int)nr, r, Sb, &one, X, (int)g.n_dof, Wd, Sb, &zero, Pc, (int)nr));
  // coefficients of every snapshot: C = Phi^H X  (r x S)
  SCVS_CUBLAS(cublasCgemm(h, CUBLAS_OP_C, CUBLAS_OP_N, r, S, (int)nr, &one, Pc, (int)nr, X, (int)g.n_dof, &zero, Cd, r));
  coef.resize((size_t)r * S);
  SCVS_CUDA(cudaMemcpyAsync(coef.data(), Cd, coef.size() * sizeof(cuComplex), cudaMemcpyDeviceToHost, c.stream));
  // Phi stored row-major [nr][r] for the expansion kernel: transpose via GEMM-free copy on host
  std::vector<cuComplex> pc((size_t)nr * r), pr((size_t)nr * r);
  SCVS_CUDA(cudaMemcpyAsync(pc.data(), Pc, pc.size() * sizeof(cuComplex), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  for (int j = 0; j < r; ++j)
    for (int64_t i = 0; i < nr; ++i) pr[(size_t)i * r + j] = pc[(size_t)j * nr + i];
  float2 *Phi = nullptr;
  SCVS_CUDA(cudaMalloc(&Phi, pr.size() * sizeof(float2)));
  SCVS_CUDA(cudaMemcpyAsync(Phi, pr.data(), pr.size() * sizeof(float2), cudaMemcpyHostToDevice, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  cudaFree(G); cudaFree(Wd); cudaFree(Pc); cudaFree(Cd);
  *Phi_out = Phi;
}

// Train: POD of both blocks, targets, feature/target standardisation, Adam.
double guess_train(Ctx &c, const scvs_train_opts &o) {
  GuessModel &g = c.guess;
  if (g.n_snap < 4) throw (int)SCVS_ERR_STATE;
  cublasHandle_t h;
  SCVS_CUBLAS(cublasCreate(&h));
  SCVS_CUBLAS(cublasSetStream(h, c.stream));
  if (g.Phi_u) cudaFree(g.Phi_u);
  if (g.Phi_p) cudaFree(g.Phi_p);
  g.Phi_u = g.Phi_p = nullptr;
  std::vector<std::complex<float>> cu, cp;
  int ru = 0, rp = 0;
  try {
    pod_block(c, g, h, 0, g.n_u, o.n_pod, o.max_pod_snapshots, &g.Phi_u, cu, ru);
    pod_block(c, g, h, g.n_u, g.n_dof - g.n_u, o.n_pod, o.max_pod_snapshots, &g.Phi_p, cp, rp);
  } catch (...) {
    cublasDestroy(h);
    throw;
  }
  cublasDestroy(h);
  if (ru != rp) {  // keep both blocks at the same rank
    const int r = std::min(ru, rp);
    if (ru > r) {  // truncate u
      std::vector<float2> tmp((size_t)g.n_u * ru), nt((size_t)g.n_u * r);
      SCVS_CUDA(cudaMemcpy(tmp.data(), g.Phi_u, tmp.size() * sizeof(float2), cudaMemcpyDeviceToHost));
      for (int64_t i = 0; i < g.n_u; ++i)
        for (int j = 0; j < r; ++j) nt[(size_t)i * r + j] = tmp[(size_t)i * ru + j];
      SCVS_CUDA(cudaMemcpy(g.Phi_u, nt.data(), nt.size() * sizeof(float2), cudaMemcpyHostToDevice));
      std::vector<std::complex<float>> c2((size_t)r * g.n_snap);
      for (int64_t s = 0; s < g.n_snap; ++s)
        for (int j = 0; j < r; ++j) c2[(size_t)s * r + j] = cu[(size_t)s * ru + j];
      cu.swap(c2);
      ru = r;
    } else {
      std::vector<float2> tmp((size_t)(g.n_dof - g.n_u) * rp), nt((size_t)(g.n_dof - g.n_u) * r);
      SCVS_CUDA(cudaMemcpy(tmp.data(), g.Phi_p, tmp.size() * sizeof(float2), cudaMemcpyDeviceToHost));
      for (int64_t i = 0; i < g.n_dof - g.n_u; ++i)
        for (int j = 0; j < r; ++j) nt[(size_t)i * r + j] = tmp[(size_t)i * rp + j];
      SCVS_CUDA(cudaMemcpy(g.Phi_p, nt.data(), nt.size() * sizeof(float2), cudaMemcpyHostToDevice));
      std::vector<std::complex<float>> c2((size_t)r * g.n_snap);
      for (int64_t s = 0; s < g.n_snap; ++s)
        for (int j = 0; j < r; ++j) c2[(size_t)s * r + j] = cp[(size_t)s * rp + j];
      cp.swap(c2);
      rp = r;
    }
  }
  g.n_pod = ru;
  const int S = (int)g.n_snap, n_out = 4 * g.n_pod;
  // targets [S][n_out]: (Re a_u, Im a_u) then (Re a_p, Im a_p)
  std::vector<float> T((size_t)S * n_out), F((size_t)S * 5);
  for (int s = 0; s < S; ++s) {
    for (int j = 0; j < g.n_pod; ++j) {
      T[(size_t)s * n_out + 2 * j] = cu[(size_t)s * g.n_pod + j].real();
      T[(size_t)s * n_out + 2 * j + 1] = cu[(size_t)s * g.n_pod + j].imag();
      T[(size_t)s * n_out + 2 * g.n_pod + 2 * j] = cp[(size_t)s * g.n_pod + j].real();
      T[(size_t)s * n_out + 2 * g.n_pod + 2 * j + 1] = cp[(size_t)s * g.n_pod + j].imag();
    }
    for (int q = 0; q < 5; ++q) F[(size_t)s * 5 + q] = (float)g.feat[(size_t)s * 5 + q];
  }
  // standardise features and targets (statistics kept for inference)
  g.fmean.assign(5, 0.0); g.fstd.assign(5, 0.0);
  g.tmean.assign(n_out, 0.0); g.tstd.assign(n_out, 0.0);
  for (int q = 0; q < 5; ++q) {
    double mu = 0, s2 = 0;
    for (int s = 0; s < S; ++s) mu += F[(size_t)s * 5 + q];
    mu /= S;
    for (int s = 0; s < S; ++s) s2 += (F[(size_t)s * 5 + q] - mu) * (F[(size_t)s * 5 + q] - mu);
    g.fmean[q] = mu;
    g.fstd[q] = std::sqrt(s2 / S) > 1e-12 ? std::sqrt(s2 / S) : 1.0;
  }
  for (int j = 0; j < n_out; ++j) {
    double mu = 0, s2 = 0;
    for (int s = 0; s < S; ++s) mu += T[(size_t)s * n_out + j];
    mu /= S;
    for (int s = 0; s < S; ++s) s2 += (T[(size_t)s * n_out + j] - mu) * (T[(size_t)s * n_out + j] - mu);
    g.tmean[j] = mu;
    g.tstd[j] = std::sqrt(s2 / S) > 1e-30 ? std::sqrt(s2 / S) : 1.0;
  }
  for (int s = 0; s < S; ++s) {
    for (int q = 0; q < 5; ++q) F[(size_t)s * 5 + q] = (float)((F[(size_t)s * 5 + q] - g.fmean[q]) / g.fstd[q]);
    for (int j = 0; j < n_out; ++j)
      T[(size_t)s * n_out + j] = (float)((T[(size_t)s * n_out + j] - g.tmean[j]) / g.tstd[j]);
  }
  mlp_alloc(g, 5, o.hidden, n_out);
  // He-normal initialisation (seeded), zero biases
  std::mt19937_64 rng(o.seed);
  std::vector<float> w0(g.n_params, 0.0f);
  for (int l = 0; l < 4; ++l) {
    std::normal_distribution<float> nd(0.0f, std::sqrt(2.0f / g.dims[l]));
    for (int64_t i = 0; i < (int64_t)g.dims[l] * g.dims[l + 1]; ++i) w0[g.woff[l] + i] = nd(rng);
  }
  SCVS_CUDA(cudaMemcpy(g.Wf, w0.data(), w0.size() * sizeof(float), cudaMemcpyHostToDevice));
  mlp_refresh_bf16(c, g);
  // minibatch Adam
  const int B = std::min<int>(o.batch, S);
  float *Xd = nullptr, *Td = nullptr;
  SCVS_CUDA(cudaMalloc(&Xd, (size_t)B * 5 * sizeof(float)));
  SCVS_CUDA(cudaMalloc(&Td, (size_t)B * n_out * sizeof(float)));
  std::vector<int> perm(S);
  for (int i = 0; i < S; ++i) perm[i] = i;
  std::vector<float> xb((size_t)B * 5), tb((size_t)B * n_out);
  int pos = S;
  double last = 0;
  for (int step = 0; step < o.steps; ++step) {
    if (pos + B > S) { std::shuffle(perm.begin(), perm.end(), rng); pos = 0; }
    for (int b = 0; b < B; ++b) {
      const int s = perm[pos + b];
      std::copy(F.begin() + (size_t)s * 5, F.begin() + (size_t)s * 5 + 5, xb.begin() + (size_t)b * 5);
      std::copy(T.begin() + (size_t)s * n_out, T.begin() + (size_t)(s + 1) * n_out, tb.begin() + (size_t)b * n_out);
    }
    pos += B;
    SCVS_CUDA(cudaMemcpyAsync(Xd, xb.data(), xb.size() * sizeof(float), cudaMemcpyHostToDevice, c.stream));
    SCVS_CUDA(cudaMemcpyAsync(Td, tb.data(), tb.size() * sizeof(float), cudaMemcpyHostToDevice, c.stream));
    const float lr = (float)(o.lr * (step < o.steps / 2 ? 1.0 : (step < 3 * o.steps / 4 ? 0.3 : 0.1)));
    last = mlp_gradient(c, g, Xd, Td, B);
    mlp_adam(c, g, lr);
  }
  cudaFree(Xd);
  cudaFree(Td);
  g.trained = true;
  return last;
}

// x0 of every mode of a mesh from its features (guess enabled, model trained);
// returns false if the model cannot serve this mesh.
bool guess_initial(Ctx &c, Mesh &m) {
  GuessModel &g = c.guess;
  if (!g.trained || g.n_dof != m.n_dof || (int)m.feat.size() != 5 * m.m) return false;
  const int n_out = 4 * g.n_pod;
  std::vector<float> F((size_t)m.m * 5);
  for (int k = 0; k < m.m; ++k)
    for (int q = 0; q < 5; ++q) F[(size_t)k * 5 + q] = (float)((m.feat[(size_t)k * 5 + q] - g.fmean[q]) / g.fstd[q]);
  float *Xd = nullptr, *Yd = nullptr;
  SCVS_CUDA(ctx_malloc(c, &Xd, F.size() * sizeof(float), c.stream));
  SCVS_CUDA(ctx_malloc(c, &Yd, (size_t)m.m * n_out * sizeof(float), c.stream));
  SCVS_CUDA(cudaMemcpyAsync(Xd, F.data(), F.size() * sizeof(float), cudaMemcpyHostToDevice, c.stream));
  mlp_forward(c, g, Xd, m.m, Yd);
  std::vector<float> Y((size_t)m.m * n_out);
  SCVS_CUDA(cudaMemcpyAsync(Y.data(), Yd, Y.size() * sizeof(float), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  std::vector<float2> au((size_t)m.m * g.n_pod), ap((size_t)m.m * g.n_pod);
  std::vector<double2> ck(m.ld, make_double2(0, 0));
  for (int k = 0; k < m.m; ++k) {
    for (int j = 0; j < g.n_pod; ++j) {
      auto d = [&](int col) { return (float)(Y[(size_t)k * n_out + col] * g.tstd[col] + g.tmean[col]); };
      au[(size_t)k * g.n_pod + j] = make_float2(d(2 * j), d(2 * j + 1));
      ap[(size_t)k * g.n_pod + j] = make_float2(d(2 * g.n_pod + 2 * j), d(2 * g.n_pod + 2 * j + 1));
    }
    ck[k] = make_double2(m.feat[(size_t)k * 5 + 1], m.feat[(size_t)k * 5 + 2]);
  }
  float2 *aud = nullptr, *apd = nullptr;
  double2 *ckd = nullptr;
  SCVS_CUDA(ctx_malloc(c, &aud, au.size() * sizeof(float2), c.stream));
  SCVS_CUDA(ctx_malloc(c, &apd, ap.size() * sizeof(float2), c.stream));
  SCVS_CUDA(ctx_malloc(c, &ckd, ck.size() * sizeof(double2), c.stream));
  SCVS_CUDA(cudaMemcpyAsync(aud, au.data(), au.size() * sizeof(float2), cudaMemcpyHostToDevice, c.stream));
  SCVS_CUDA(cudaMemcpyAsync(apd, ap.data(), ap.size() * sizeof(float2), cudaMemcpyHostToDevice, c.stream));
  SCVS_CUDA(cudaMemcpyAsync(ckd, ck.data(), ck.size() * sizeof(double2), cudaMemcpyHostToDevice, c.stream));
  {
    KScope ks(c, KC_VECTOR, (double)m.n_dof * g.n_pod * 8 + (double)m.n_dof * m.ld * 32);
    k_guess_expand<<<ceil_div(m.n_dof * m.ld, 256), 256, 0, c.stream>>>(g.Phi_u, g.Phi_p, g.n_pod, aud, apd, ckd, m.m,
                                                                       m.ld, (int64_t)m.dim * m.N, m.n_dof, m.dirmask,
                                                                       m.dim, m.b, m.x);
    count_launch(c);
  }
  for (void *p : {(void *)Xd, (void *)Yd, (void *)aud, (void *)apd, (void *)ckd}) SCVS_CUDA(cudaFreeAsync(p, c.stream));
  return true;
}

}  // namespace scvs
