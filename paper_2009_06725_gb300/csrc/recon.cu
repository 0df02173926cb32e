// Time reconstruction of the modal solution (Eq. sol_reconstruct):
//   u(x, t_s) = Re sum_k u_k(x) e^{j omega_k t_s},  t_s = s T / n_t,
// a direct inverse real DFT over the modes of every dof.  Each block stages a
// tile of dofs x modes in shared memory, each thread owns one dof and writes
// its n_t samples; consecutive threads write consecutive dofs of a sample
// (coalesced).  The twiddles e^{j omega_k t_s} are tabulated in FP64 on the
// host; accumulation is FP64.
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

}  // namespace scvs
