// Time reconstruction of the modal solution (Eq. sol_reconstruct):
//   u(x, t_s) = Re sum_k u_k(x) e^{j omega_k t_s},  t_s = s T / n_t,
// a direct inverse real DFT over the modes of every dof.  Each block stages a
// tile of dofs x modes in shared memory, each thread owns one dof and writes
// its n_t samples; consecutive threads write consecutive dofs of a sample
// (coalesced).  The twiddles e^{j omega_k t_s} are tabulated in FP64 on the
// host; accumulation is FP64.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>
#include "scvs_internal.h"

namespace scvs {

// ---- allocation-free variant ------------------------------------------
// Twiddle scratch of scvs_reconstruct_dev_static: a file-scope device table
// that every GPU loading the library holds until the process exits.  Host
// code must not pass the symbol itself to a kernel (on the host it only names
// a stand-in object); the device address is taken once per device with
// cudaGetSymbolAddress.
__device__ __align__(256) double2 g_recon_twiddles[SCVS_RECON_STATIC_MAX];

constexpr int MAX_DEVICES = 64;
static double2 *g_twiddle_addr[MAX_DEVICES] = {nullptr};
static std::mutex g_twiddle_mu;

// Device address of the twiddle table on the current device (set up on the
// first call per device).
static double2 *static_twiddles(int device) {
  if (device < 0 || device >= MAX_DEVICES) throw (int)SCVS_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_twiddle_mu);
  if (!g_twiddle_addr[device]) {
    void *p = nullptr;
    SCVS_CUDA(cudaGetSymbolAddress(&p, g_recon_twiddles));
    g_twiddle_addr[device] = static_cast<double2 *>(p);
  }
  return g_twiddle_addr[device];
}

// tw[s][k] = (cos, sin)(omega_k * s * period / n_t), computed on the device
__global__ void k_twiddles(const double *__restrict__ omega, int m, int n_t, double period, double2 *__restrict__ tw) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m * n_t) return;
  const int s = i / m, k = i % m;
  double sn, cs;
  sincos(omega[k] * (period * s / n_t), &sn, &cs);
  tw[i] = make_double2(cs, sn);
}

__global__ void k_reconstruct(const double2 *__restrict__ x, int64_t n_dof, int ld, int m, int n_t,
                              const double2 *__restrict__ tw, int64_t n_u, double *__restrict__ u_t,
                              double *__restrict__ p_t, int64_t n_p) {
  extern __shared__ double2 xs[];  // [blockDim][m]
  const int64_t d0 = (int64_t)blockIdx.x * blockDim.x;
  const int td = blockDim.x;
  for (int e = threadIdx.x; e < td * m; e += td) {
    const int r = e / m, k = e % m;
    const int64_t dof = d0 + r;
    xs[r * m + k] = dof < n_dof ? x[dof * ld + k] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  const int64_t dof = d0 + threadIdx.x;
  if (dof >= n_dof) return;
  const double2 *xr = xs + threadIdx.x * m;
  for (int s = 0; s < n_t; ++s) {
    const double2 *t = tw + (int64_t)s * m;
    double acc = 0.0;
    for (int k = 0; k < m; ++k) {
      const double2 a = xr[k], w = __ldg(t + k);
      acc = fma(a.x, w.x, acc);
      acc = fma(-a.y, w.y, acc);
    }
    if (dof < n_u) {
      if (u_t) u_t[(int64_t)s * n_u + dof] = acc;
    } else if (p_t) {
      p_t[(int64_t)s * n_p + (dof - n_u)] = acc;
    }
  }
}

static int recon_block(const Mesh &m, size_t &smem) {
  int td = 128;
  while (td > 32 && (size_t)td * m.m * sizeof(double2) > 96 * 1024) td >>= 1;
  smem = (size_t)td * m.m * sizeof(double2);
  return td;
}

void reconstruct_static(Ctx &c, Mesh &m, int n_t, double period, double *u_t, double *p_t) {
  if ((int64_t)n_t * m.m > SCVS_RECON_STATIC_MAX) throw (int)SCVS_ERR_ARG;
  int dev = 0;
  SCVS_CUDA(cudaGetDevice(&dev));
  double2 *tw = static_twiddles(dev);
  k_twiddles<<<ceil_div((int64_t)n_t * m.m, 256), 256, 0, c.stream>>>(m.omega_d, m.m, n_t, period, tw);
  count_launch(c);
  size_t smem;
  const int td = recon_block(m, smem);
  SCVS_CUDA(cudaFuncSetAttribute(k_reconstruct, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  k_reconstruct<<<ceil_div(m.n_dof, td), td, smem, c.stream>>>(m.x, m.n_dof, m.ld, m.m, n_t, tw,
                                                              (int64_t)m.dim * m.N, u_t, p_t, m.P);
  count_launch(c);
  SCVS_CUDA(cudaGetLastError());
}

// Mode-major copies of the modal solution: U[k][i] = x[i][k] for the velocity
// dofs i < n_u, Pm[k][v] = x[n_u + v][k] for the pressure dofs; 32 x 32 tiles
// of (dof, mode) transposed through shared memory (coalesced reads of the
// interleaved block and coalesced writes of the mode-major arrays).
__global__ void k_modal_split(const double2 *__restrict__ x, int64_t n_dof, int ld, int m, int64_t n_u,
                              double2 *__restrict__ U, double2 *__restrict__ Pm) {
  __shared__ double2 t[32][33];
  const int64_t d0 = (int64_t)blockIdx.x * 32;
  const int k0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t d = d0 + r;
    const int k = k0 + threadIdx.x;
    t[r][threadIdx.x] = (d < n_dof && k < m) ? x[d * ld + k] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int k = k0 + r;
    const int64_t d = d0 + threadIdx.x;
    if (k >= m || d >= n_dof) continue;
    const double2 v = t[threadIdx.x][r];
    if (d < n_u) U[(int64_t)k * n_u + d] = v;
    else Pm[(int64_t)k * (n_dof - n_u) + (d - n_u)] = v;
  }
}

void modal_split(Ctx &c, Mesh &m, double2 *U, double2 *Pm) {
  const int64_t n_u = (int64_t)m.dim * m.N;
  dim3 grid((unsigned)ceil_div(m.n_dof, 32), (unsigned)ceil_div(m.m, 32));
  KScope ks(c, KC_VECTOR, (double)m.n_dof * m.m * 32);
  k_modal_split<<<grid, dim3(32, 8), 0, c.stream>>>(m.x, m.n_dof, m.ld, m.m, n_u, U, Pm);
  count_launch(c);
}

void reconstruct(Ctx &c, Mesh &m, int n_t, double period, double *u_t, double *p_t) {
  std::vector<double2> tw((size_t)n_t * m.m);
  for (int s = 0; s < n_t; ++s) {
    const double t = period * s / n_t;
    for (int k = 0; k < m.m; ++k) {
      const double ph = m.omega[k] * t;
      tw[(size_t)s * m.m + k] = make_double2(std::cos(ph), std::sin(ph));
    }
  }
  double2 *twd = nullptr;
  SCVS_CUDA(ctx_malloc(c, &twd, tw.size() * sizeof(double2), c.stream));
  SCVS_CUDA(cudaMemcpyAsync(twd, tw.data(), tw.size() * sizeof(double2), cudaMemcpyHostToDevice, c.stream));
  int td = 128;
  while (td > 32 && (size_t)td * m.m * sizeof(double2) > 96 * 1024) td >>= 1;
  const size_t smem = (size_t)td * m.m * sizeof(double2);
  SCVS_CUDA(cudaFuncSetAttribute(k_reconstruct, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  KScope ks(c, KC_RECON, (double)m.n_dof * m.m * 16 + (double)n_t * m.n_dof * 8);
  k_reconstruct<<<ceil_div(m.n_dof, td), td, smem, c.stream>>>(m.x, m.n_dof, m.ld, m.m, n_t, twd,
                                                              (int64_t)m.dim * m.N, u_t, p_t, m.P);
  count_launch(c);
  SCVS_CUDA(cudaFreeAsync(twd, c.stream));
}

// ---- spectral preprocessing of sampled boundary data -------------------
// Fourier coefficients of a periodic boundary field from n_t uniform samples
// (Eq. SCVS_bc by the rectangle rule), returned as the solver's per-mode data
// c_0 = g~_0, c_i = 2 g~_i, and the a priori truncation error of Eq.
// mode_error through the discrete Parseval identity: with the samples' mean
// square E = (1/n_t) sum_s sum_p w_p g(t_s, p)^2 and mode energies
// e_0 = sum_p w_p |g~_0|^2, e_i = 2 sum_p w_p |g~_i|^2 (modes below the Nyquist
// frequency), the truncated series after mode N misses exactly
// E - sum_{i <= N} e_i.

// c[i][p] = (i ? 2 : 1) / n_t * sum_s g[s][p] e^{-j 2 pi i s / n_t}: one thread per
// (mode, point), samples in ascending order, twiddle index i s mod n_t stepped
// incrementally; consecutive threads read consecutive points of a sample.
__global__ void k_bc_dft(const double *__restrict__ g, int64_t n_pts, int n_t, int n_modes,
                         const double2 *__restrict__ tw, double2 *__restrict__ c) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= (int64_t)n_modes * n_pts) return;
  const int i = (int)(f / n_pts);
  const int64_t p = f % n_pts;
  double re = 0.0, im = 0.0;
  int idx = 0;
  for (int s = 0; s < n_t; ++s) {
    const double v = g[(int64_t)s * n_pts + p];
    const double2 t = tw[idx];
    re += v * t.x;
    im -= v * t.y;
    idx += i;
    if (idx >= n_t) idx -= n_t;
  }
  const double sc = (i ? 2.0 : 1.0) / n_t;
  c[f] = make_double2(re * sc, im * sc);
}

// out[i] = e_i for i < n_modes (from c: e_0 = w |c_0|^2, e_i = w |c_i|^2 / 2) and
// out[n_modes] = E; one block per entry, threads stride in order, fixed tree.
__global__ void __launch_bounds__(1024) k_bc_energy(const double *__restrict__ g, const double2 *__restrict__ c,
                                                    const double *__restrict__ w, int64_t n_pts, int n_t,
                                                    int n_modes, double *__restrict__ out) {
  __shared__ double red[1024];
  const int i = blockIdx.x, tid = threadIdx.x, bd = blockDim.x;
  double acc = 0.0;
  if (i < n_modes) {
    for (int64_t p = tid; p < n_pts; p += bd) {
      const double2 v = c[(int64_t)i * n_pts + p];
      acc += (w ? w[p] : 1.0) * (v.x * v.x + v.y * v.y);
    }
    if (i) acc *= 0.5;
  } else {
    const int64_t n = (int64_t)n_t * n_pts;
    for (int64_t e = tid; e < n; e += bd) {
      const double v = g[e];
      acc += (w ? w[e % n_pts] : 1.0) * v * v;
    }
    acc /= n_t;
  }
  red[tid] = acc;
  __syncthreads();
  for (int h = bd / 2; h > 0; h >>= 1) {
    if (tid < h) red[tid] += red[tid + h];
    __syncthreads();
  }
  if (tid == 0) out[i] = red[0];
}

void bc_spectrum(Ctx &c, int n_t, int64_t n_pts, int n_modes, const double *g_t, const double *w, double2 *c_out,
                 double *e2) {
  std::vector<double2> tw(n_t);
  for (int j = 0; j < n_t; ++j) {
    const double ph = 2.0 * M_PI * (double)j / (double)n_t;
    tw[j] = make_double2(std::cos(ph), std::sin(ph));
  }
  double2 *twd = nullptr;
  double *en = nullptr;
  SCVS_CUDA(ctx_malloc(c, &twd, (size_t)n_t * sizeof(double2), c.stream));
  SCVS_CUDA(ctx_malloc(c, &en, (size_t)(n_modes + 1) * sizeof(double), c.stream));
  SCVS_CUDA(cudaMemcpyAsync(twd, tw.data(), (size_t)n_t * sizeof(double2), cudaMemcpyHostToDevice, c.stream));
  const int64_t nc = (int64_t)n_modes * n_pts;
  {
    KScope ks(c, KC_RECON, (double)n_t * n_pts * 8 + (double)nc * 16);
    k_bc_dft<<<ceil_div(nc, 256), 256, 0, c.stream>>>(g_t, n_pts, n_t, n_modes, twd, c_out);
    count_launch(c);
  }
  {
    KScope ks(c, KC_RECON, (double)n_t * n_pts * 8 + (double)nc * 16 + (w ? (double)n_pts * 8 * (n_modes + 1) : 0.0));
    k_bc_energy<<<n_modes + 1, 1024, 0, c.stream>>>(g_t, c_out, w, n_pts, n_t, n_modes, en);
    count_launch(c);
  }
  std::vector<double> h(n_modes + 1);
  SCVS_CUDA(cudaMemcpyAsync(h.data(), en, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaFreeAsync(twd, c.stream));
  SCVS_CUDA(cudaFreeAsync(en, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  const double total = h[n_modes];
  double kept = 0.0;
  for (int i = 0; i < n_modes; ++i) {
    kept += h[i];
    e2[i] = total > 0.0 ? std::max(0.0, (total - kept) / total) : 0.0;
  }
}

// ---- a posteriori mode energies ------------------------------------------
// E_k = time average over the period of ||Re(u~_k e^{j omega_k t})||^2_{L2(Omega)}
// for the velocity of every solved (component, mode): ||Re u~_k||^2_{M_s} for
// omega_k = 0 and (1/2) u~_k^H (I_d (x) M_s) u~_k otherwise (harmonic frequencies,
// whose e^{2 j omega t} term averages out).  Distinct harmonics are orthogonal
// in L2(Omega x T), so the reconstruction truncated after mode N changes by
// delta_N^2 = E_N / sum_{k <= N} E_k relative to itself (Sec. 3, a posteriori
// choice of the number of modes).

// q[dof][k] = weight_k Re(conj(x_{A,c,k}) (M_s x_{.,c,k})_A) for the velocity dof
// A dim + c (one thread per (dof, mode), S row of A in pattern order; weight 1
// with the real part only for omega_k = 0, else 1/2 with the complex modulus).
__global__ void k_mass_quad(const double2 *__restrict__ x, const int64_t *__restrict__ s_ptr,
                            const int32_t *__restrict__ s_col, const double *__restrict__ Ms,
                            const double *__restrict__ omega, int64_t N, int dim, int ld, int m,
                            double *__restrict__ q) {
  const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (f >= (int64_t)dim * N * ld) return;
  const int k = (int)(f % ld);
  if (k >= m) { q[f] = 0.0; return; }
  const int64_t dof = f / ld, A = dof / dim;
  const int c = (int)(dof % dim);
  double sx = 0.0, sy = 0.0;
  for (int64_t t = s_ptr[A]; t < s_ptr[A + 1]; ++t) {
    const double2 v = x[((int64_t)s_col[t] * dim + c) * ld + k];
    const double mv = Ms[t];
    sx += mv * v.x;
    sy += mv * v.y;
  }
  const double2 u = x[f];
  q[f] = omega[k] == 0.0 ? u.x * sx : 0.5 * (u.x * sx + u.y * sy);
}

// Per row chunk and mode: sum of q over the chunk's rows (rows at or beyond
// n_q hold no value), strided in order and reduced by a fixed tree.
constexpr int ENERGY_T = 256;
__global__ void k_chunk_sum(const double *__restrict__ q, int64_t n_q, int ld, int64_t n_chunk,
                            const int64_t *__restrict__ row0, const int32_t *__restrict__ rows,
                            double *__restrict__ part) {
  __shared__ double s[ENERGY_T];
  for (int64_t ch = blockIdx.x; ch < n_chunk; ch += gridDim.x) {
    const int64_t f0 = row0[ch] * ld, f1 = min((row0[ch] + rows[ch]) * ld, n_q * ld);
    double acc = 0.0;
    for (int64_t f = f0 + threadIdx.x; f < f1; f += ENERGY_T) acc += q[f];  // stride is a multiple of ld
    s[threadIdx.x] = acc;
    __syncthreads();
    for (int w = ENERGY_T / 2; w >= ld; w >>= 1) {
      if (threadIdx.x < w) s[threadIdx.x] += s[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x < ld) part[ch * ld + threadIdx.x] = s[threadIdx.x];
    __syncthreads();
  }
}

// out[comp][k] = sum of the component's chunk partials in chunk order.
__global__ void k_sys_sum(const double *__restrict__ part, const int32_t *__restrict__ comp_chunk, int n_comp, int ld,
                          double *__restrict__ out) {
  const int sys = blockIdx.x * blockDim.x + threadIdx.x;
  if (sys >= n_comp * ld) return;
  const int comp = sys / ld, k = sys % ld;
  double acc = 0.0;
  for (int ch = comp_chunk[comp]; ch < comp_chunk[comp + 1]; ++ch) acc += part[(int64_t)ch * ld + k];
  out[sys] = acc;
}

void mode_energies(Ctx &c, Mesh &m, double *E, double *incr2) {
  const int64_t nq = (int64_t)m.dim * m.N;
  double *q = nullptr, *part = nullptr, *out = nullptr;
  SCVS_CUDA(ctx_malloc(c, &q, (size_t)nq * m.ld * sizeof(double), c.stream));
  SCVS_CUDA(ctx_malloc(c, &part, (size_t)m.n_chunk * m.ld * sizeof(double), c.stream));
  SCVS_CUDA(ctx_malloc(c, &out, (size_t)m.n_sys() * sizeof(double), c.stream));
  {
    KScope ks(c, KC_RECON, (double)m.s_nnz * 12 * m.dim * m.m + (double)nq * m.ld * 24);
    k_mass_quad<<<ceil_div(nq * m.ld, 256), 256, 0, c.stream>>>(m.x, m.s_ptr, m.s_col, m.Ms, m.omega_d, m.N, m.dim,
                                                                m.ld, m.m, q);
    count_launch(c);
  }
  {
    KScope ks(c, KC_RECON, (double)nq * m.ld * 8 + (double)m.n_chunk * m.ld * 8);
    const unsigned nb = (unsigned)std::max<int64_t>(1, std::min<int64_t>(m.n_chunk, 8 * c.num_sms));
    k_chunk_sum<<<nb, ENERGY_T, 0, c.stream>>>(q, nq, m.ld, m.n_chunk, m.chunk_row0, m.chunk_rows, part);
    count_launch(c);
  }
  {
    KScope ks(c, KC_RECON, (double)m.n_chunk * m.ld * 8 + (double)m.n_sys() * 8);
    k_sys_sum<<<ceil_div(m.n_sys(), 128), 128, 0, c.stream>>>(part, m.comp_chunk, m.n_comp, m.ld, out);
    count_launch(c);
  }
  std::vector<double> h(m.n_sys());
  SCVS_CUDA(cudaMemcpyAsync(h.data(), out, h.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  SCVS_CUDA(cudaFreeAsync(q, c.stream));
  SCVS_CUDA(cudaFreeAsync(part, c.stream));
  SCVS_CUDA(cudaFreeAsync(out, c.stream));
  SCVS_CUDA(cudaStreamSynchronize(c.stream));
  for (int comp = 0; comp < m.n_comp; ++comp) {
    double tot = 0.0;
    for (int k = 0; k < m.m; ++k) {
      const double e = h[(size_t)comp * m.ld + k];
      tot += e;
      E[(size_t)comp * m.m + k] = e;
      if (incr2) incr2[(size_t)comp * m.m + k] = tot > 0.0 ? e / tot : 0.0;
    }
  }
}

}  // namespace scvs
