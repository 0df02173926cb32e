// Learned initial guess for the per-mode solves (training and inference).
//
// Snapshots: converged modal solutions x_k of solved meshes, divided by the
// mode's boundary coefficient c_k (the problem is linear in c_k), stored as
// complex FP32 columns of length n_dof together with the mode features
// f = (omega_k, Re c_k, Im c_k, R, s).
// POD (method of snapshots, per field block u / p) in the block's L2(Omega)
// inner product: Gram matrix X^H W X (W the reference mesh's mass matrix of the
// block) by the project's own FP64-accumulating Gram kernel, its leading
// eigenpairs on the host (Householder tridiagonalization + implicit QR), basis
// Phi = X V Lambda^{-1/2} with a fixed phase per vector; training targets
// a = Phi^H W x.
// MLP 5 -> H -> H -> H -> 4 n_pod with exact GELU on the hidden layers; the
// weights used by the forward/backward kernels are BF16 (FP32 master copies
// updated by Adam), every product is accumulated in FP32.
// Inference: x0 = c_k [Phi_u a_u; Phi_p a_p] on the free rows, g on the
// Dirichlet rows.
#include <cuda_bf16.h>
#include <algorithm>
#include <cmath>
#include <complex>
#include <random>
#include <type_traits>
#include <vector>
#include "scvs_internal.h"

namespace scvs {

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
// Eigen-decomposition of a Hermitian matrix (column-major, n x n); returns the
// eigenvalues descending and the matching eigenvectors (columns of V).
//  1. Householder reduction to a tridiagonal matrix, A = Q T Q^H: for column k
//     the reflector H = I - tau v v^H maps the part below the diagonal onto
//     alpha e_1 (alpha = -|x| x_0/|x_0|), and the trailing block becomes
//     B - v w^H - w v^H with p = tau B v, w = p - (tau/2)(v^H p) v.
//  2. The diagonal similarity D = diag(delta), delta_{k+1} = delta_k e_k/|e_k|,
//     makes T = D S D^H with S real symmetric tridiagonal (off-diagonal |e_k|).
//  3. Implicit symmetric QR steps with the Wilkinson shift on S (Givens
//     rotations chasing the bulge down each unreduced block), accumulating the
//     rotations into Z, until every off-diagonal entry is negligible.
//  4. Eigenvectors Q D Z (the reflectors applied in reverse order).
// Cost O(n^3) with unit-stride inner loops (the cyclic Jacobi method it
// replaced took ~40 s at n = 512 on one host core).
static void hermitian_eig(int n, std::vector<std::complex<double>> A, std::vector<double> &lam,
                          std::vector<std::complex<double>> &V) {
  using cd = std::complex<double>;
  // row-major copy: M[r * n + c] = A(r, c)
  std::vector<cd> M((size_t)n * n);
  for (int c = 0; c < n; ++c)
    for (int r = 0; r < n; ++r) M[(size_t)r * n + c] = A[(size_t)c * n + r];
  std::vector<double> d(n, 0.0), e(n, 0.0);
  std::vector<cd> sub(n, cd(0, 0));                 // T[k+1][k]
  std::vector<std::vector<cd>> vs(std::max(n - 2, 0));  // reflector vectors (length n - k - 1)
  std::vector<double> taus(std::max(n - 2, 0), 0.0);
  std::vector<cd> p(n), w(n);
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;
    std::vector<cd> &v = vs[k];
    v.resize(m);
    double sigma = 0;
    for (int i = 0; i < m; ++i) {
      v[i] = std::conj(M[(size_t)k * n + k + 1 + i]);  // column k below the diagonal (A Hermitian)
      if (i > 0) sigma += std::norm(v[i]);
    }
    const double ax0 = std::abs(v[0]);
    if (sigma == 0.0) {  // already tridiagonal in this column
      sub[k] = v[0];
      taus[k] = 0.0;
      continue;
    }
    const double nx = std::sqrt(ax0 * ax0 + sigma);
    const cd ph = ax0 > 0 ? v[0] / ax0 : cd(1, 0);
    const cd alpha = -ph * nx;
    v[0] -= alpha;
    const double vn2 = std::norm(v[0]) + sigma;
    const double tau = 2.0 / vn2;
    taus[k] = tau;
    sub[k] = alpha;
    // p = tau B v with B the trailing block rows/cols k+1 .. n-1
    cd vhp(0, 0);
    for (int i = 0; i < m; ++i) {
      const cd *row = &M[(size_t)(k + 1 + i) * n + k + 1];
      cd acc(0, 0);
      for (int j = 0; j < m; ++j) acc += row[j] * v[j];
      p[i] = tau * acc;
      vhp += std::conj(v[i]) * p[i];
    }
    const double K = 0.5 * tau * vhp.real();
    for (int i = 0; i < m; ++i) w[i] = p[i] - K * v[i];
    for (int i = 0; i < m; ++i) {
      cd *row = &M[(size_t)(k + 1 + i) * n + k + 1];
      const cd vi = v[i], wi = w[i];
      for (int j = 0; j < m; ++j) row[j] -= vi * std::conj(w[j]) + wi * std::conj(v[j]);
    }
  }
  for (int k = 0; k < n; ++k) d[k] = M[(size_t)k * n + k].real();
  if (n >= 2) sub[n - 2] = M[(size_t)(n - 1) * n + (n - 2)];
  // diagonal phases making the tridiagonal real
  std::vector<cd> delta(n, cd(1, 0));
  for (int k = 0; k + 1 < n; ++k) {
    const double a = std::abs(sub[k]);
    e[k] = a;
    delta[k + 1] = a > 0 ? delta[k] * (sub[k] / a) : delta[k];
  }
  // implicit symmetric QR with Wilkinson shifts; Z accumulates the rotations (row-major)
  std::vector<double> Z((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) Z[(size_t)i * n + i] = 1.0;
  const double eps = 2.220446049250313e-16;
  int hi = n - 1, guard = 0;
  while (hi > 0 && guard < 100 * n) {
    if (std::fabs(e[hi - 1]) <= eps * (std::fabs(d[hi - 1]) + std::fabs(d[hi]))) {
      e[hi - 1] = 0.0;
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && std::fabs(e[lo - 1]) > eps * (std::fabs(d[lo - 1]) + std::fabs(d[lo]))) --lo;
    ++guard;
    // Wilkinson shift from the trailing 2 x 2 block
    const double dl = 0.5 * (d[hi - 1] - d[hi]), eh = e[hi - 1];
    const double mu = d[hi] - eh * eh / (dl + (dl >= 0 ? 1.0 : -1.0) * std::hypot(dl, eh));
    double x = d[lo] - mu, z = e[lo];
    for (int k = lo; k < hi; ++k) {
      const double r = std::hypot(x, z);
      const double c = r > 0 ? x / r : 1.0, s = r > 0 ? z / r : 0.0;
      if (k > lo) e[k - 1] = r;
      const double dk = d[k], dk1 = d[k + 1], ek = e[k];
      d[k] = c * c * dk + 2 * c * s * ek + s * s * dk1;
      d[k + 1] = s * s * dk - 2 * c * s * ek + c * c * dk1;
      e[k] = c * s * (dk1 - dk) + (c * c - s * s) * ek;
      if (k + 1 < hi) {
        x = e[k];
        z = s * e[k + 1];  // the bulge at (k, k+2)
        e[k + 1] *= c;
      }
      for (int i = 0; i < n; ++i) {
        double *zr = &Z[(size_t)i * n];
        const double a = zr[k], b = zr[k + 1];
        zr[k] = c * a + s * b;
        zr[k + 1] = -s * a + c * b;
      }
    }
  }
  // eigenvectors of A: Q D z for every eigenvalue, in descending order
  std::vector<int> ord(n);
  for (int i = 0; i < n; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int a, int b) { return d[a] > d[b]; });
  lam.resize(n);
  V.assign((size_t)n * n, cd(0, 0));
  std::vector<cd> y(n);
  for (int q = 0; q < n; ++q) {
    const int col = ord[q];
    lam[q] = d[col];
    for (int i = 0; i < n; ++i) y[i] = delta[i] * Z[(size_t)i * n + col];
    for (int k = n - 3; k >= 0; --k) {  // y <- H_k y, last reflector first
      if (taus[k] == 0.0) continue;
      const std::vector<cd> &v = vs[k];
      cd dot(0, 0);
      for (int i = 0; i < (int)v.size(); ++i) dot += std::conj(v[i]) * y[k + 1 + i];
      dot *= taus[k];
      for (int i = 0; i < (int)v.size(); ++i) y[k + 1 + i] -= dot * v[i];
    }
    for (int i = 0; i < n; ++i) V[(size_t)q * n + i] = y[i];
  }
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
float mlp_gradient(Ctx &c, GuessModel &g, const float *x, const float *t, int64_t B, bool read_loss) {
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
  if (!read_loss) return 0.0f;  // the training loop reads only its last step's loss
  float h = 0;
  SCVS_CUDA(cudaMemcpyAsync(&h, loss, sizeof(float), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  return h;
}

// Minibatch of the training loop: rows idx[0..B) of the device-resident
// standardised features F [S][5] and targets T [S][n_out].
__global__ void k_gather_batch(const int32_t *__restrict__ idx, int64_t B, const float *__restrict__ F,
                               const float *__restrict__ T, int n_out, float *__restrict__ X, float *__restrict__ Y) {
  const int64_t i = blockIdx.x * 256ll + threadIdx.x;
  if (i < B * 5) X[i] = F[(int64_t)idx[i / 5] * 5 + i % 5];
  if (i < B * n_out) Y[i] = T[(int64_t)idx[i / n_out] * n_out + i % n_out];
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
    // the first mesh's mass matrices define the POD inner products
    GuessModel::RefMass &w = g.wref;
    w.dim = m.dim; w.N = m.N; w.P = m.P;
    auto dup = [&](auto *&dst, const auto *src, int64_t n) {
      using E = std::remove_cv_t<std::remove_pointer_t<std::remove_reference_t<decltype(dst)>>>;
      SCVS_CUDA(cudaMalloc(&dst, (size_t)std::max<int64_t>(n, 1) * sizeof(E)));
      SCVS_CUDA(cudaMemcpyAsync(dst, src, (size_t)n * sizeof(E), cudaMemcpyDeviceToDevice, c.stream));
    };
    dup(w.s_ptr, m.s_ptr, m.N + 1);
    dup(w.g_ptr, m.g_ptr, m.N + 1);
    dup(w.s_col, m.s_col, m.s_nnz);
    dup(w.g_len, m.g_len, m.N);
    dup(w.Ms, m.Ms, m.s_nnz);
    dup(w.Mp, m.Mp, m.q_nnz);
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

// ---------------------------------------------------------------- POD
// Mass weighting of snapshot-layout vectors of one field block: y_s = W x_s for
// s < ns, with W = M_s (x) I_d on the velocity block and the P1 mass on the
// pressure block, both of the reference mesh (the one that gave the first
// snapshot; morphs share its connectivity).  x_s at x + s * ldx, block row i
// at x_s[i]; FP64 accumulation of FP32 inputs, FP32 result.
__global__ void k_pod_weight_u(const GuessModel::RefMass w, const float2 *__restrict__ x, int64_t ldx, int ns,
                               float2 *__restrict__ y, int64_t ldy) {
  const int64_t n_u = (int64_t)w.dim * w.N;
  const int64_t t = blockIdx.x * 256ll + threadIdx.x;
  const int s = blockIdx.y;
  if (t >= n_u || s >= ns) return;
  const int64_t A = t / w.dim;
  const int c = (int)(t % w.dim);
  const float2 *xs = x + (int64_t)s * ldx;
  double re = 0.0, im = 0.0;
  for (int64_t q = w.s_ptr[A]; q < w.s_ptr[A + 1]; ++q) {
    const double mv = w.Ms[q];
    const float2 v = xs[(int64_t)w.s_col[q] * w.dim + c];
    re = fma(mv, (double)v.x, re);
    im = fma(mv, (double)v.y, im);
  }
  y[(int64_t)s * ldy + t] = make_float2((float)re, (float)im);
}

__global__ void k_pod_weight_p(const GuessModel::RefMass w, const float2 *__restrict__ x, int64_t ldx, int ns,
                               float2 *__restrict__ y, int64_t ldy) {
  const int64_t v = blockIdx.x * 256ll + threadIdx.x;
  const int s = blockIdx.y;
  if (v >= w.P || s >= ns) return;
  const float2 *xs = x + (int64_t)s * ldx;
  const int64_t q0 = w.g_ptr[v], c0 = w.s_ptr[v];
  double re = 0.0, im = 0.0;
  for (int t = 0; t < w.g_len[v]; ++t) {
    const double mv = w.Mp[q0 + t];
    const float2 e = xs[w.s_col[c0 + t]];
    re = fma(mv, (double)e.x, re);
    im = fma(mv, (double)e.y, im);
  }
  y[(int64_t)s * ldy + v] = make_float2((float)re, (float)im);
}

// Complex Gram products with FP64 accumulation of FP32 inputs:
// part[kc][i][j] = sum over rows r of chunk kc of conj(A_i[r]) B_j[r], with
// A_i at A + i * lda and B_j at B + j * ldb (i < na, j < nb, r < rows).  One
// 32 x 32 output tile per block of 256 threads (2 x 2 outputs per thread),
// rows staged 32 at a time in shared memory.
constexpr int GT = 32;
__global__ void __launch_bounds__(256) k_cgram(const float2 *__restrict__ A, int64_t lda, int na,
                                               const float2 *__restrict__ B, int64_t ldb, int nb, int64_t rows,
                                               int64_t chunk, double2 *__restrict__ part) {
  __shared__ float2 As[GT][GT + 1], Bs[GT][GT + 1];
  const int i0 = blockIdx.y * GT, j0 = blockIdx.x * GT;
  const int64_t r_begin = (int64_t)blockIdx.z * chunk, r_end = min(rows, r_begin + chunk);
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  double acc[2][2][2] = {};
  for (int64_t r0 = r_begin; r0 < r_end; r0 += GT) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = threadIdx.x + 256 * q;
      const int a = idx / GT, rr = idx % GT;
      const int64_t r = r0 + rr;
      const bool in_r = r < r_end;
      As[rr][a] = (in_r && i0 + a < na) ? A[(int64_t)(i0 + a) * lda + r] : make_float2(0.f, 0.f);
      Bs[rr][a] = (in_r && j0 + a < nb) ? B[(int64_t)(j0 + a) * ldb + r] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < GT; ++rr) {
      const float2 a0 = As[rr][2 * ty], a1 = As[rr][2 * ty + 1];
      const float2 b0 = Bs[rr][2 * tx], b1 = Bs[rr][2 * tx + 1];
      const float2 av[2] = {a0, a1}, bv[2] = {b0, b1};
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          const double ar = av[u].x, ai = av[u].y, br = bv[v].x, bi = bv[v].y;
          acc[u][v][0] = fma(ar, br, fma(ai, bi, acc[u][v][0]));
          acc[u][v][1] = fma(ar, bi, fma(-ai, br, acc[u][v][1]));
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int u = 0; u < 2; ++u)
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int i = i0 + 2 * ty + u, j = j0 + 2 * tx + v;
      if (i < na && j < nb)
        part[((int64_t)blockIdx.z * na + i) * nb + j] = make_double2(acc[u][v][0], acc[u][v][1]);
    }
}

// out[i][j] = sum_kc part[kc][i][j], chunks in order.
__global__ void k_cgram_sum(const double2 *__restrict__ part, int nkc, int64_t n, double2 *__restrict__ out) {
  const int64_t t = blockIdx.x * 256ll + threadIdx.x;
  if (t >= n) return;
  double re = 0.0, im = 0.0;
  for (int k = 0; k < nkc; ++k) {
    const double2 v = part[(int64_t)k * n + t];
    re += v.x;
    im += v.y;
  }
  out[t] = make_double2(re, im);
}

// Phi[i][j] = sum_{s < ns} X_s[i] Wm[s][j] (rows i < nr of the block, j < r),
// FP64 accumulation; writes Phi row-major [nr][r] and transposed Phit [r][nr].
// Block: 256 rows x 16 columns (grid.y tiles the columns); Wm staged 32
// snapshots at a time.
__global__ void __launch_bounds__(256) k_pod_basis(const float2 *__restrict__ X, int64_t ldx, int ns, int64_t nr,
                                                   const double2 *__restrict__ Wm, int r, float2 *__restrict__ Phi,
                                                   float2 *__restrict__ Phit) {
  __shared__ double2 ws[32][16];
  const int64_t i = blockIdx.x * 256ll + threadIdx.x;
  const int j0 = blockIdx.y * 16;
  double acc[16][2] = {};
  for (int s0 = 0; s0 < ns; s0 += 32) {
    for (int t = threadIdx.x; t < 32 * 16; t += 256) {
      const int ss = t / 16, jj = t % 16;
      ws[ss][jj] = (s0 + ss < ns && j0 + jj < r) ? Wm[(int64_t)(s0 + ss) * r + j0 + jj] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    if (i < nr) {
      const int sn = min(32, ns - s0);
      for (int ss = 0; ss < sn; ++ss) {
        const float2 xv = X[(int64_t)(s0 + ss) * ldx + i];
        const double xr = xv.x, xi = xv.y;
#pragma unroll
        for (int jj = 0; jj < 16; ++jj) {
          const double2 w = ws[ss][jj];
          acc[jj][0] = fma(xr, w.x, fma(-xi, w.y, acc[jj][0]));
          acc[jj][1] = fma(xr, w.y, fma(xi, w.x, acc[jj][1]));
        }
      }
    }
    __syncthreads();
  }
  if (i >= nr) return;
#pragma unroll
  for (int jj = 0; jj < 16; ++jj) {
    const int j = j0 + jj;
    if (j >= r) break;
    const float2 v = make_float2((float)acc[jj][0], (float)acc[jj][1]);
    Phi[i * r + j] = v;
    Phit[(int64_t)j * nr + i] = v;
  }
}

// Gram products conj(A)^T B of snapshot-layout operands over `rows` rows, on
// the device: returns out [na][nb] (device, FP64 complex, from the pool).
static double2 *cgram(Ctx &c, const float2 *A, int64_t lda, int na, const float2 *B, int64_t ldb, int nb,
                      int64_t rows) {
  const int ti = (int)ceil_div(na, GT), tj = (int)ceil_div(nb, GT);
  const int64_t want = std::max<int64_t>(1, (4 * (int64_t)c.num_sms + ti * tj - 1) / ((int64_t)ti * tj));
  const int64_t chunk = std::max<int64_t>(GT, ceil_div(ceil_div(rows, want), GT) * GT);
  const int nkc = (int)ceil_div(rows, chunk);
  const int64_t n = (int64_t)na * nb;
  double2 *part = nullptr, *out = nullptr;
  SCVS_CUDA(ctx_malloc(c, &part, (size_t)nkc * n * sizeof(double2), c.stream));
  SCVS_CUDA(ctx_malloc(c, &out, (size_t)n * sizeof(double2), c.stream));
  k_cgram<<<dim3(tj, ti, nkc), 256, 0, c.stream>>>(A, lda, na, B, ldb, nb, rows, chunk, part);
  count_launch(c);
  k_cgram_sum<<<(unsigned)ceil_div(n, 256), 256, 0, c.stream>>>(part, nkc, n, out);
  count_launch(c);
  SCVS_CUDA(cudaFreeAsync(part, c.stream));
  return out;
}

// y_s = W x_s (s < ns) for the field block `blk` (0: velocity, 1: pressure).
static void pod_weight(Ctx &c, const GuessModel &g, int blk, const float2 *x, int64_t ldx, int ns, float2 *y,
                       int64_t ldy) {
  const int64_t nr = blk == 0 ? g.n_u : g.n_dof - g.n_u;
  for (int s0 = 0; s0 < ns; s0 += 65535) {
    const int sn = std::min(65535, ns - s0);
    dim3 grid((unsigned)ceil_div(nr, 256), (unsigned)sn);
    if (blk == 0)
      k_pod_weight_u<<<grid, 256, 0, c.stream>>>(g.wref, x + (int64_t)s0 * ldx, ldx, sn, y + (int64_t)s0 * ldy, ldy);
    else
      k_pod_weight_p<<<grid, 256, 0, c.stream>>>(g.wref, x + (int64_t)s0 * ldx, ldx, sn, y + (int64_t)s0 * ldy, ldy);
    count_launch(c);
  }
}

// POD of one field block (rows [r0, r0 + nr) of the snapshots) in the block's
// L2(Omega) inner product: G = X_b^H W X_b over the first n_basis snapshots,
// its eigenpairs (host tridiagonal QR, FP64), every eigenvector's phase fixed
// so that its largest-magnitude entry is real positive, Phi = X_b V_r
// Lambda_r^{-1/2} (W-orthonormal), and the coefficients a_s = Phi^H W x_s of
// every snapshot.  Phi is row-major [nr][r] on the device; coef is [n_snap][r].
static void pod_block(Ctx &c, GuessModel &g, int blk, int n_pod_req, int n_basis, float2 **Phi_out,
                      std::vector<std::complex<double>> &coef, std::vector<double> &lam_out, int &n_pod_out) {
  const int64_t r0 = blk == 0 ? 0 : g.n_u, nr = blk == 0 ? g.n_u : g.n_dof - g.n_u;
  const int S = (int)g.n_snap, Sb = std::min<int>(S, n_basis);
  const float2 *X = g.snap + r0;  // snapshot s, block row i at X[s * n_dof + i]
  float2 *WX = nullptr;
  SCVS_CUDA(ctx_malloc(c, &WX, (size_t)Sb * nr * sizeof(float2), c.stream));
  pod_weight(c, g, blk, X, g.n_dof, Sb, WX, nr);
  double2 *Gd = cgram(c, X, g.n_dof, Sb, WX, nr, Sb, nr);  // G[i][j] = x_i^H W x_j
  std::vector<double2> hg((size_t)Sb * Sb);
  SCVS_CUDA(cudaMemcpyAsync(hg.data(), Gd, hg.size() * sizeof(double2), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaFreeAsync(Gd, c.stream));
  SCVS_CUDA(cudaFreeAsync(WX, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  // column-major Hermitian matrix for the eigensolver, made exactly Hermitian
  std::vector<std::complex<double>> A((size_t)Sb * Sb);
  for (int i = 0; i < Sb; ++i)
    for (int j = 0; j < Sb; ++j) {
      const double2 a = hg[(size_t)i * Sb + j], b = hg[(size_t)j * Sb + i];
      A[(size_t)j * Sb + i] = 0.5 * (std::complex<double>(a.x, a.y) + std::conj(std::complex<double>(b.x, b.y)));
    }
  std::vector<double> lam;
  std::vector<std::complex<double>> V;
  hermitian_eig(Sb, A, lam, V);
  int r = 0;
  while (r < std::min(n_pod_req, Sb) && lam[r] > 1e-10 * lam[0]) ++r;
  n_pod_out = r;
  lam_out = lam;
  // Wm = V_r Lambda_r^{-1/2} with each column's phase fixed, [Sb][r] row-major
  std::vector<double2> Wm((size_t)Sb * r);
  for (int j = 0; j < r; ++j) {
    const std::complex<double> *vj = V.data() + (size_t)j * Sb;
    int imax = 0;
    for (int i = 1; i < Sb; ++i)
      if (std::abs(vj[i]) > std::abs(vj[imax])) imax = i;
    const std::complex<double> ph = std::conj(vj[imax]) / std::abs(vj[imax]);
    const double sc = 1.0 / std::sqrt(lam[j]);
    for (int i = 0; i < Sb; ++i) {
      const std::complex<double> v = vj[i] * ph * sc;
      Wm[(size_t)i * r + j] = make_double2(v.real(), v.imag());
    }
  }
  double2 *Wmd = nullptr;
  float2 *Phi = nullptr, *Phit = nullptr, *WPhit = nullptr;
  SCVS_CUDA(ctx_malloc(c, &Wmd, Wm.size() * sizeof(double2), c.stream));
  SCVS_CUDA(cudaMemcpyAsync(Wmd, Wm.data(), Wm.size() * sizeof(double2), cudaMemcpyHostToDevice, c.stream));
  SCVS_CUDA(cudaMalloc(&Phi, (size_t)nr * r * sizeof(float2)));
  SCVS_CUDA(ctx_malloc(c, &Phit, (size_t)nr * r * sizeof(float2), c.stream));
  SCVS_CUDA(ctx_malloc(c, &WPhit, (size_t)nr * r * sizeof(float2), c.stream));
  k_pod_basis<<<dim3((unsigned)ceil_div(nr, 256), (unsigned)ceil_div(r, 16)), 256, 0, c.stream>>>(X, g.n_dof, Sb, nr,
                                                                                                 Wmd, r, Phi, Phit);
  count_launch(c);
  // coefficients: C[j][s] = (W phi_j)^H x_s = phi_j^H W x_s (W is real symmetric)
  pod_weight(c, g, blk, Phit, nr, r, WPhit, nr);
  double2 *Cd = cgram(c, WPhit, nr, r, X, g.n_dof, S, nr);
  std::vector<double2> hc((size_t)r * S);
  SCVS_CUDA(cudaMemcpyAsync(hc.data(), Cd, hc.size() * sizeof(double2), cudaMemcpyDeviceToHost, c.stream));
  for (void *p : {(void *)Wmd, (void *)Phit, (void *)WPhit, (void *)Cd}) SCVS_CUDA(cudaFreeAsync(p, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  coef.resize((size_t)S * r);
  for (int s = 0; s < S; ++s)
    for (int j = 0; j < r; ++j) coef[(size_t)s * r + j] = std::complex<double>(hc[(size_t)j * S + s].x, hc[(size_t)j * S + s].y);
  *Phi_out = Phi;
}

// Keep the first r columns of a row-major [n][r_old] device basis and of the
// [S][r_old] coefficients.
static void truncate_basis(Ctx &c, float2 *&Phi, int64_t n, int r_old, int r, std::vector<std::complex<double>> &coef,
                           int64_t S) {
  std::vector<float2> tmp((size_t)n * r_old), nt((size_t)n * r);
  SCVS_CUDA(cudaMemcpy(tmp.data(), Phi, tmp.size() * sizeof(float2), cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < n; ++i)
    for (int j = 0; j < r; ++j) nt[(size_t)i * r + j] = tmp[(size_t)i * r_old + j];
  SCVS_CUDA(cudaMemcpy(Phi, nt.data(), nt.size() * sizeof(float2), cudaMemcpyHostToDevice));
  std::vector<std::complex<double>> c2((size_t)S * r);
  for (int64_t s = 0; s < S; ++s)
    for (int j = 0; j < r; ++j) c2[(size_t)s * r + j] = coef[(size_t)s * r_old + j];
  coef.swap(c2);
  (void)c;
}

// Train: POD of both blocks, targets, feature/target standardisation, Adam.
double guess_train(Ctx &c, const scvs_train_opts &o) {
  GuessModel &g = c.guess;
  if (g.n_snap < 4) throw (int)SCVS_ERR_STATE;
  if (g.Phi_u) cudaFree(g.Phi_u);
  if (g.Phi_p) cudaFree(g.Phi_p);
  g.Phi_u = g.Phi_p = nullptr;
  std::vector<std::complex<double>> &cu = g.coef_u, &cp = g.coef_p;
  int ru = 0, rp = 0;
  pod_block(c, g, 0, o.n_pod, o.max_pod_snapshots, &g.Phi_u, cu, g.lam_u, ru);
  pod_block(c, g, 1, o.n_pod, o.max_pod_snapshots, &g.Phi_p, cp, g.lam_p, rp);
  if (ru > rp) { truncate_basis(c, g.Phi_u, g.n_u, ru, rp, cu, g.n_snap); ru = rp; }  // same rank in both blocks
  if (rp > ru) { truncate_basis(c, g.Phi_p, g.n_dof - g.n_u, rp, ru, cp, g.n_snap); rp = ru; }
  g.n_pod = ru;
  const int S = (int)g.n_snap, n_out = 4 * g.n_pod;
  // targets [S][n_out]: (Re a_u, Im a_u) then (Re a_p, Im a_p)
  std::vector<float> T((size_t)S * n_out), F((size_t)S * 5);
  for (int s = 0; s < S; ++s) {
    for (int j = 0; j < g.n_pod; ++j) {
      T[(size_t)s * n_out + 2 * j] = (float)cu[(size_t)s * g.n_pod + j].real();
      T[(size_t)s * n_out + 2 * j + 1] = (float)cu[(size_t)s * g.n_pod + j].imag();
      T[(size_t)s * n_out + 2 * g.n_pod + 2 * j] = (float)cp[(size_t)s * g.n_pod + j].real();
      T[(size_t)s * n_out + 2 * g.n_pod + 2 * j + 1] = (float)cp[(size_t)s * g.n_pod + j].imag();
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
    g.tstd[j] = std::sqrt(s2 / S) > 1e-12 ? std::sqrt(s2 / S) : 1.0;
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
  // minibatch Adam: the standardised data stay on the device, every step's
  // minibatch indices (seeded shuffles, drawn on the host up front) are
  // uploaded once, a kernel gathers each minibatch, and the host reads back
  // only the last step's loss, so the steps run back to back on the stream
  const int B = std::min<int>(o.batch, S);
  std::vector<int32_t> idx((size_t)std::max(o.steps, 0) * B);
  {
    std::vector<int> perm(S);
    for (int i = 0; i < S; ++i) perm[i] = i;
    int pos = S;
    for (int step = 0; step < o.steps; ++step) {
      if (pos + B > S) { std::shuffle(perm.begin(), perm.end(), rng); pos = 0; }
      for (int b = 0; b < B; ++b) idx[(size_t)step * B + b] = perm[pos + b];
      pos += B;
    }
  }
  float *Xd = nullptr, *Td = nullptr, *Fall = nullptr, *Tall = nullptr;
  int32_t *idx_d = nullptr;
  SCVS_CUDA(cudaMalloc(&Xd, (size_t)B * 5 * sizeof(float)));
  SCVS_CUDA(cudaMalloc(&Td, (size_t)B * n_out * sizeof(float)));
  SCVS_CUDA(cudaMalloc(&Fall, F.size() * sizeof(float)));
  SCVS_CUDA(cudaMalloc(&Tall, T.size() * sizeof(float)));
  SCVS_CUDA(cudaMalloc(&idx_d, std::max<size_t>(idx.size(), 1) * sizeof(int32_t)));
  SCVS_CUDA(cudaMemcpy(Fall, F.data(), F.size() * sizeof(float), cudaMemcpyHostToDevice));
  SCVS_CUDA(cudaMemcpy(Tall, T.data(), T.size() * sizeof(float), cudaMemcpyHostToDevice));
  SCVS_CUDA(cudaMemcpy(idx_d, idx.data(), idx.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
  double last = 0;
  for (int step = 0; step < o.steps; ++step) {
    k_gather_batch<<<grid1((int64_t)B * std::max(5, n_out)), 256, 0, c.stream>>>(idx_d + (size_t)step * B, B, Fall,
                                                                                Tall, n_out, Xd, Td);
    count_launch(c);
    const float lr = (float)(o.lr * (step < o.steps / 2 ? 1.0 : (step < 3 * o.steps / 4 ? 0.3 : 0.1)));
    const float l = mlp_gradient(c, g, Xd, Td, B, step == o.steps - 1);
    if (step == o.steps - 1) last = l;
    mlp_adam(c, g, lr);
  }
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  cudaFree(Xd);
  cudaFree(Td);
  cudaFree(Fall);
  cudaFree(Tall);
  cudaFree(idx_d);
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
