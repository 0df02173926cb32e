// Shared device/host helpers of the SCVS CUDA library (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

namespace scvs {

// ---------------------------------------------------------------- errors
struct CudaError {
  cudaError_t code;
  std::string where;
};

#define SCVS_CUDA(call)                                                          \
  do {                                                                           \
    cudaError_t _e = (call);                                                     \
    if (_e != cudaSuccess) throw ::scvs::CudaError{_e, std::string(#call) + " @ " \
                                                       + __FILE__ + ":" + std::to_string(__LINE__)}; \
  } while (0)

// Device-side error bits written by kernels into a flag word; the host turns
// them into return codes after the kernel.
enum DevErr : int {
  DEVERR_NONE = 0,
  DEVERR_BAD_NODE = 1,      // connectivity entry outside [0, n_nodes)
  DEVERR_BAD_VERTEX = 2,    // a simplex vertex id outside [0, n_vertices)
  DEVERR_JACOBIAN = 4,      // non-positive element Jacobian
  DEVERR_VALENCE = 8,       // too many elements around one node for the pattern kernel
  DEVERR_BARRIER = 16,      // a bounded grid barrier gave up
  DEVERR_DUP_NODE = 32,     // an element lists the same node twice
};

// --------------------------------------------------------- complex helpers
template <typename T> struct cpx;
template <> struct cpx<float> { using t = float2; };
template <> struct cpx<double> { using t = double2; };

template <typename T> __host__ __device__ __forceinline__ typename cpx<T>::t mk(T r, T i) {
  typename cpx<T>::t z; z.x = r; z.y = i; return z;
}

// ----------------------------------------------------------- grid barrier
// Bounded sense-counting barrier for cooperative launches: every block of the
// grid must be resident (the host launches with cudaLaunchCooperativeKernel).
// A block that waits more than spin_limit polls (default SPIN_LIMIT) sets the
// error word and returns false; every caller then exits the kernel.
struct GridSync {
  unsigned int count;
  unsigned int gen;
  int err;
  int pad;
};

constexpr long long SPIN_LIMIT = 1ll << 24;  // ~2-4 s with the back-off below

#ifdef __CUDACC__
__device__ __forceinline__ unsigned int ld_acquire_gpu(const unsigned int *p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned int atom_add_acq_rel_gpu(unsigned int *p, unsigned int v) {
  unsigned int old;
  asm volatile("atom.add.acq_rel.gpu.global.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}
__device__ __forceinline__ void st_relaxed_gpu(unsigned int *p, unsigned int v) {
  asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// The block's threads meet at a CTA barrier; thread 0 then arrives with an
// acquire-release add (its release covers the block's writes ordered before
// the CTA barrier), the last arriver resets the counter and publishes the new
// generation with a release add, and the others poll the generation with
// acquire loads.  (Measured on a GB300 with 456 blocks: 2.5 us per barrier
// against 3.2 us for full fences from every thread.)
__device__ __forceinline__ bool grid_sync(GridSync *gs, unsigned int nblocks, long long spin_limit = SPIN_LIMIT) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int g = ld_acquire_gpu(&gs->gen);
    int ok = 1;
    if (atom_add_acq_rel_gpu(&gs->count, 1u) == nblocks - 1) {
      st_relaxed_gpu(&gs->count, 0u);
      atom_add_acq_rel_gpu(&gs->gen, 1u);
    } else {
      volatile int *verr = &gs->err;
      long long spins = 0;
      while (ld_acquire_gpu(&gs->gen) == g) {
        if (*verr) { ok = 0; break; }
        if (++spins > spin_limit) { atomicExch(&gs->err, 1); ok = 0; break; }
        if (spins > 4096) __nanosleep(100);  // poll tightly first: most waits are a few microseconds
      }
    }
    s_ok = ok && (*(volatile int *)&gs->err == 0);
  }
  __syncthreads();
  return s_ok != 0;
}
#endif

// ------------------------------------------------------------- constants
constexpr int MAX_NL = 10;   // P2 tet
constexpr int MAX_NV = 4;    // P1 tet
constexpr int GEOM_STRIDE = 16;  // det, Jinv[3][3], gamma[6] (sym, ij i<=j)

// Exact integrals over the reference simplex (computed on the host, see refmats.cpp):
//   mref[a][b]        = int phi_a phi_b
//   ksym[p][a][b]     = int (d_i phi_a d_j phi_b + d_j phi_a d_i phi_b)/(1 + delta_ij),
//                       p enumerating (i,j), i <= j, in row order
//   eref[i][a][b]     = int d_i phi_a psi_b          (phi P2, psi P1)
//   m1[a][b]          = int psi_a psi_b
//   k1sym[p][a][b]    = as ksym for the P1 basis
struct RefTables {
  double mref[MAX_NL][MAX_NL];
  double ksym[6][MAX_NL][MAX_NL];
  double eref[3][MAX_NL][MAX_NV];
  double m1[MAX_NV][MAX_NV];
  double k1sym[6][MAX_NV][MAX_NV];
};

void reference_tables(int dim, RefTables *out);  // refmats.cpp

// Quadrature of curved (isoparametric) elements: points of the collapsed
// Gauss-Legendre rule with ISO_QUAD points per direction, weights, the P2
// basis, its reference gradients and the P1 basis at every point.
constexpr int ISO_QUAD = 6;
constexpr int ISO_QMAX = ISO_QUAD * ISO_QUAD * ISO_QUAD;
struct QuadTables {
  int dim, nq;
  double w[ISO_QMAX];
  double phi[ISO_QMAX][MAX_NL];
  double dphi[ISO_QMAX][MAX_NL][3];
  double psi[ISO_QMAX][MAX_NV];
};
void quad_tables(int dim, int n, QuadTables *out);  // refmats.cpp
void face_mass_iso(int fdim, int dim, int n, const double *X, double *M);  // refmats.cpp

inline unsigned int ceil_div(long long a, long long b) { return (unsigned int)((a + b - 1) / b); }

}  // namespace scvs
