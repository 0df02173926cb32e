// Row blocks with shared-memory staging of the gathered vector entries.
//
// The all-modes operators gather, for every nonzero of a row, the entries of
// the column node for every mode and component (768 bytes per nonzero with 32
// FP32 modes and 3 components).  Neighbouring rows share most of their
// columns, so a block of rows that is compact in the mesh needs far fewer
// distinct column nodes ("footprint") than it has nonzeros: on the benchmark
// pipe about a quarter.  This file builds such blocks once per mesh, on the
// GPU, and provides FP32 kernels that copy a block's footprint into shared
// memory with TMA bulk copies (cp.async.bulk, completion on an mbarrier) and
// then run the rows of the block against shared memory:
//   * locality order: nodes sorted by (slab along the longest bounding-box
//     axis, 2D Morton code of the other two coordinates, node id), slabs two
//     vertex spacings thick (bitonic sort of 64-bit keys);
//   * blocks: consecutive rows of that order holding about `budget` nonzeros;
//   * footprint: the ascending distinct columns of a block's rows; the
//     vertex columns (ids < P) are its prefix;
//   * lcol: every nonzero's index in its row's footprint (16 bits, stored in
//     the original nonzero order, so the matrix values keep their layout).
// Within a row the nonzeros are visited in the same order and with the same
// arithmetic as the unstaged kernels of operators.cu, so both give identical
// results.
#include <algorithm>
#include <climits>
#include <cmath>
#include "scvs_internal.h"
#include "vecops.cuh"
#include "opargs.cuh"

namespace scvs {

// ------------------------------------------------------------ ordering
__global__ void k_bbox(const double *__restrict__ xyz, int64_t N, int dim, double *out /* [2][3] */) {
  __shared__ double lo[3][256], hi[3][256];
  double l[3] = {1e300, 1e300, 1e300}, h[3] = {-1e300, -1e300, -1e300};
  for (int64_t i = threadIdx.x; i < N; i += blockDim.x)
    for (int c = 0; c < dim; ++c) {
      const double v = xyz[i * dim + c];
      l[c] = fmin(l[c], v);
      h[c] = fmax(h[c], v);
    }
  for (int c = 0; c < 3; ++c) { lo[c][threadIdx.x] = l[c]; hi[c][threadIdx.x] = h[c]; }
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int c = 0; c < 3; ++c) {
        lo[c][threadIdx.x] = fmin(lo[c][threadIdx.x], lo[c][threadIdx.x + w]);
        hi[c][threadIdx.x] = fmax(hi[c][threadIdx.x], hi[c][threadIdx.x + w]);
      }
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int c = 0; c < 3; ++c) { out[c] = lo[c][0]; out[3 + c] = hi[c][0]; }
}

__device__ __forceinline__ uint64_t spread14(uint64_t v) {  // 14 bits -> every other bit of 28
  v &= 0x3fff;
  v = (v | (v << 8)) & 0x00ff00ffull;
  v = (v | (v << 4)) & 0x0f0f0f0full;
  v = (v | (v << 2)) & 0x33333333ull;
  v = (v | (v << 1)) & 0x55555555ull;
  return v;
}

// key = slab (13 bits) | 2D Morton code (28 bits) | node id (23 bits); padding
// entries [N, n2) get the largest key.
__global__ void k_order_keys(const double *__restrict__ xyz, int64_t N, int dim, int axis, int a1, int a2,
                             double x0, double inv_slab, double y0, double z0, double inv_q, int64_t n2,
                             uint64_t *__restrict__ keys) {
  const int64_t i = blockIdx.x * 256ll + threadIdx.x;
  if (i >= n2) return;
  if (i >= N) { keys[i] = ~0ull; return; }
  const double *p = xyz + i * dim;
  const uint64_t slab = (uint64_t)min(8191.0, fmax(0.0, floor((p[axis] - x0) * inv_slab)));
  const uint64_t qa = (uint64_t)min(16383.0, fmax(0.0, (p[a1] - y0) * inv_q));
  const uint64_t qb = dim == 3 ? (uint64_t)min(16383.0, fmax(0.0, (p[a2] - z0) * inv_q)) : 0;
  const uint64_t morton = spread14(qa) | (spread14(qb) << 1);
  keys[i] = (slab << 51) | (morton << 23) | (uint64_t)i;
}

constexpr int BT = 2048;  // bitonic tile (shared memory) of 64-bit keys

// Sort every tile of BT keys for all k <= BT (the global direction rule:
// ascending where (i & k) == 0).
__global__ void __launch_bounds__(1024) k_bitonic_tile_sort(uint64_t *keys) {
  __shared__ uint64_t s[BT];
  const int64_t base = (int64_t)blockIdx.x * BT;
  for (int t = threadIdx.x; t < BT; t += 1024) s[t] = keys[base + t];
  __syncthreads();
  for (int k = 2; k <= BT; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < BT; t += 1024) {
        const int u = t ^ j;
        if (u > t) {
          const int64_t gi = base + t;
          const bool up = (gi & k) == 0;
          const uint64_t a = s[t], b = s[u];
          if ((a > b) == up) { s[t] = b; s[u] = a; }
        }
      }
      __syncthreads();
    }
  for (int t = threadIdx.x; t < BT; t += 1024) keys[base + t] = s[t];
}

// One global compare-exchange step (stride j >= BT) of merge stage k.
__global__ void k_bitonic_step(uint64_t *keys, int64_t n2, int64_t k, int64_t j) {
  const int64_t t = blockIdx.x * 256ll + threadIdx.x;
  if (t >= n2) return;
  const int64_t u = t ^ j;
  if (u > t) {
    const bool up = (t & k) == 0;
    const uint64_t a = keys[t], b = keys[u];
    if ((a > b) == up) { keys[t] = b; keys[u] = a; }
  }
}

// The strides j < BT of merge stage k inside each tile.
__global__ void __launch_bounds__(1024) k_bitonic_tile_merge(uint64_t *keys, int64_t k) {
  __shared__ uint64_t s[BT];
  const int64_t base = (int64_t)blockIdx.x * BT;
  for (int t = threadIdx.x; t < BT; t += 1024) s[t] = keys[base + t];
  __syncthreads();
  for (int j = BT >> 1; j > 0; j >>= 1) {
    for (int t = threadIdx.x; t < BT; t += 1024) {
      const int u = t ^ j;
      if (u > t) {
        const bool up = ((base + t) & k) == 0;
        const uint64_t a = s[t], b = s[u];
        if ((a > b) == up) { s[t] = b; s[u] = a; }
      }
    }
    __syncthreads();
  }
  for (int t = threadIdx.x; t < BT; t += 1024) keys[base + t] = s[t];
}

__global__ void k_perm_from_keys(const uint64_t *__restrict__ keys, int64_t N, const int32_t *__restrict__ s_len,
                                 int32_t *__restrict__ perm, int32_t *__restrict__ plen) {
  const int64_t i = blockIdx.x * 256ll + threadIdx.x;
  if (i >= N) return;
  const int32_t r = (int32_t)(keys[i] & ((1ull << 23) - 1));
  perm[i] = r;
  plen[i] = s_len[r];
}

// row0[b] = first position of block b; block of position i = cum[i] / budget
__global__ void k_block_starts(const int64_t *__restrict__ cum, int64_t N, int64_t budget, int64_t *__restrict__ row0) {
  const int64_t i = blockIdx.x * 256ll + threadIdx.x;
  if (i >= N) return;
  const int64_t b = cum[i] / budget;
  if (i == 0 || cum[i - 1] / budget != b) row0[b] = i;
  if (i == N - 1) row0[b + 1] = N;
}

constexpr int FP_CAP = 2048;  // nonzeros of one block, sorted in shared memory

// Footprint of every block: the block's columns sorted, duplicates dropped.
// Pass 1 (!WRITE): footprint size and its vertex prefix per block.  Pass 2:
// the columns themselves and every nonzero's local index.  One block of 1024
// threads per row block.
template <bool WRITE>
__global__ void __launch_bounds__(1024)
k_block_footprint(const int32_t *__restrict__ perm, const int64_t *__restrict__ row0, const int64_t *__restrict__ s_ptr,
                  const int32_t *__restrict__ s_col, int64_t P, int32_t *__restrict__ fp_len,
                  int32_t *__restrict__ fv_len, const int64_t *__restrict__ fp_ptr, int32_t *__restrict__ fp_col,
                  uint16_t *__restrict__ lcol, int *err) {
  __shared__ int buf[FP_CAP];
  __shared__ int uniq[FP_CAP];
  __shared__ int rof[FP_CAP + 1];
  __shared__ int wsum[32];
  const int64_t i0 = row0[blockIdx.x], i1 = row0[blockIdx.x + 1];
  const int nr = (int)(i1 - i0);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (nr > FP_CAP) {
    if (threadIdx.x == 0) atomicOr(err, DEVERR_VALENCE);
    return;
  }
  // offsets of the block's rows in its gathered column list
  if (threadIdx.x == 0) {
    int n = 0;
    for (int q = 0; q < nr; ++q) {
      rof[q] = n;
      const int A = perm[i0 + q];
      n += (int)(s_ptr[A + 1] - s_ptr[A]);
    }
    rof[nr] = n;
  }
  __syncthreads();
  const int nnz = rof[nr];
  if (nnz > FP_CAP) {
    if (threadIdx.x == 0) atomicOr(err, DEVERR_VALENCE);
    return;
  }
  int n2 = 1;
  while (n2 < nnz) n2 <<= 1;
  for (int t = threadIdx.x; t < n2; t += blockDim.x) buf[t] = INT_MAX;
  __syncthreads();
  for (int q = warp; q < nr; q += nw) {
    const int A = perm[i0 + q];
    const int64_t r0 = s_ptr[A];
    const int len = rof[q + 1] - rof[q];
    for (int t = lane; t < len; t += 32) buf[rof[q] + t] = s_col[r0 + t];
  }
  __syncthreads();
  for (int k = 2; k <= n2; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = threadIdx.x; t < n2; t += blockDim.x) {
        const int u = t ^ j;
        if (u > t) {
          const bool up = (t & k) == 0;
          const int a = buf[t], c = buf[u];
          if ((a > c) == up) { buf[t] = c; buf[u] = a; }
        }
      }
      __syncthreads();
    }
  // distinct values: every thread flags a contiguous run, then a block-wide scan
  const int nthr = blockDim.x;
  const int per = (n2 + nthr - 1) / nthr;
  auto flag = [&](int t) { const int v = buf[t]; return v != INT_MAX && (t == 0 || buf[t - 1] != v); };
  int local = 0;
  for (int q = 0; q < per; ++q) {
    const int t = threadIdx.x * per + q;
    if (t < n2 && flag(t)) ++local;
  }
  int incl = local;
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int v = lane < nw ? wsum[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      const int w = __shfl_up_sync(0xffffffffu, v, o);
      if (lane >= o) v += w;
    }
    wsum[lane] = v;  // inclusive over warps
  }
  __syncthreads();
  int run = (warp > 0 ? wsum[warp - 1] : 0) + incl - local;
  const int total = wsum[nw - 1];
  for (int q = 0; q < per; ++q) {
    const int t = threadIdx.x * per + q;
    if (t < n2 && flag(t)) uniq[run++] = buf[t];
  }
  __syncthreads();
  if (!WRITE) {
    if (threadIdx.x == 0) {
      int nv = 0;
      while (nv < total && uniq[nv] < P) ++nv;
      fp_len[blockIdx.x] = total;
      fv_len[blockIdx.x] = nv;
    }
    return;
  }
  const int64_t o = fp_ptr[blockIdx.x];
  for (int t = threadIdx.x; t < total; t += nthr) fp_col[o + t] = uniq[t];
  // local index of every nonzero (binary search in the sorted footprint)
  for (int q = warp; q < nr; q += nw) {
    const int A = perm[i0 + q];
    const int64_t r0 = s_ptr[A];
    const int len = rof[q + 1] - rof[q];
    for (int t = lane; t < len; t += 32) {
      const int v = s_col[r0 + t];
      int lo = 0, hi = total - 1;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (uniq[mid] < v) lo = mid + 1; else hi = mid;
      }
      lcol[r0 + t] = (uint16_t)lo;
    }
  }
}

__global__ void k_max_i32(const int32_t *__restrict__ v, int64_t n, int *out) {
  int m = 0;
  for (int64_t i = blockIdx.x * 256ll + threadIdx.x; i < n; i += (int64_t)gridDim.x * 256) m = max(m, v[i]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// Build the row blocks of a mesh (nonzero budget per block; 0 = default).
void build_row_blocks(Ctx &c, Mesh &m, int budget) {
  RowBlocks &rb = m.rb;
  rb.release(c.stream);
  if (m.N >= (1ll << 23) || m.nl == 0) return;  // ids must fit the sort key
  cudaStream_t s = c.stream;
  const int64_t N = m.N;
  budget = std::max(budget > 0 ? budget : RB_DEFAULT_BUDGET, m.max_row);
  if (budget + m.max_row > FP_CAP) return;
  // bounding box and key parameters
  double *bb = nullptr;
  SCVS_CUDA(ctx_malloc(c, &bb, 6 * sizeof(double), s));
  k_bbox<<<1, 256, 0, s>>>(m.xyz, N, m.dim, bb);
  count_launch(c);
  double h[6];
  SCVS_CUDA(cudaMemcpyAsync(h, bb, sizeof(h), cudaMemcpyDeviceToHost, s));
  SCVS_CUDA(cudaFreeAsync(bb, s));
  SCVS_CUDA(cudaStreamSynchronize(s));
  if (m.dim == 2) { h[2] = 0; h[5] = 0; }
  double ext[3] = {h[3] - h[0], h[4] - h[1], h[5] - h[2]};
  int axis = 0;
  for (int a = 1; a < m.dim; ++a)
    if (ext[a] > ext[axis]) axis = a;
  int o1 = (axis + 1) % 3, o2 = (axis + 2) % 3;
  if (m.dim == 2) { o1 = 1 - axis; o2 = 2; }
  double vol = 1.0;
  for (int a = 0; a < m.dim; ++a) vol *= std::max(ext[a], 1e-300);
  const double hv = std::pow(vol / (double)std::max<int64_t>(m.P, 1), 1.0 / m.dim);  // vertex spacing
  const double slab = 2.0 * hv;
  const double qext = std::max(std::max(ext[o1], m.dim == 3 ? ext[o2] : 0.0), 1e-300);
  int64_t n2 = BT;
  while (n2 < N) n2 <<= 1;
  uint64_t *keys = nullptr;
  SCVS_CUDA(ctx_malloc(c, &keys, n2 * sizeof(uint64_t), s));
  k_order_keys<<<ceil_div(n2, 256), 256, 0, s>>>(m.xyz, N, m.dim, axis, o1, o2, h[axis], 1.0 / slab, h[o1],
                                                 m.dim == 3 ? h[o2] : 0.0, 16383.0 / qext, n2, keys);
  k_bitonic_tile_sort<<<(unsigned)(n2 / BT), 1024, 0, s>>>(keys);
  c.launches.n += 2;
  for (int64_t k = 2 * BT; k <= n2; k <<= 1) {
    for (int64_t j = k >> 1; j >= BT; j >>= 1) {
      k_bitonic_step<<<ceil_div(n2, 256), 256, 0, s>>>(keys, n2, k, j);
      count_launch(c);
    }
    k_bitonic_tile_merge<<<(unsigned)(n2 / BT), 1024, 0, s>>>(keys, k);
    count_launch(c);
  }
  rb.perm = m.arena.alloc<int32_t>(N);
  int32_t *plen = nullptr;
  int64_t *cum = nullptr;
  SCVS_CUDA(ctx_malloc(c, &plen, N * sizeof(int32_t), s));
  SCVS_CUDA(ctx_malloc(c, &cum, (N + 1) * sizeof(int64_t), s));
  k_perm_from_keys<<<ceil_div(N, 256), 256, 0, s>>>(keys, N, m.s_len, rb.perm, plen);
  count_launch(c);
  scan_exclusive(c, plen, cum, N);
  int64_t last_start = 0;
  SCVS_CUDA(cudaMemcpyAsync(&last_start, cum + N - 1, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SCVS_CUDA(cudaStreamSynchronize(s));
  // block of position i = cum[i] / budget; consecutive rows start at most
  // max_row <= budget nonzeros apart, so every block up to the last row's is
  // non-empty and k_block_starts writes every entry of row0
  rb.n_blk = last_start / budget + 1;
  rb.row0 = m.arena.alloc<int64_t>(rb.n_blk + 1);
  k_block_starts<<<ceil_div(N, 256), 256, 0, s>>>(cum, N, budget, rb.row0);
  count_launch(c);
  int32_t *fpl = nullptr;
  SCVS_CUDA(ctx_malloc(c, &fpl, rb.n_blk * sizeof(int32_t), s));
  rb.fv_len = m.arena.alloc<int32_t>(rb.n_blk);
  rb.fp_ptr = m.arena.alloc<int64_t>(rb.n_blk + 1);
  SCVS_CUDA(cudaMemsetAsync(c.dev_err, 0, sizeof(int), s));
  k_block_footprint<false><<<(unsigned)rb.n_blk, 1024, 0, s>>>(rb.perm, rb.row0, m.s_ptr, m.s_col, m.P, fpl,
                                                              rb.fv_len, nullptr, nullptr, nullptr, c.dev_err);
  count_launch(c);
  scan_exclusive(c, fpl, rb.fp_ptr, rb.n_blk);
  int *mx = nullptr;
  SCVS_CUDA(ctx_malloc(c, &mx, 2 * sizeof(int), s));
  SCVS_CUDA(cudaMemsetAsync(mx, 0, 2 * sizeof(int), s));
  k_max_i32<<<std::min<int64_t>(ceil_div(rb.n_blk, 256), 256), 256, 0, s>>>(fpl, rb.n_blk, mx);
  k_max_i32<<<std::min<int64_t>(ceil_div(rb.n_blk, 256), 256), 256, 0, s>>>(rb.fv_len, rb.n_blk, mx + 1);
  c.launches.n += 2;
  int hm[2] = {0, 0};
  int64_t fp_total = 0;
  SCVS_CUDA(cudaMemcpyAsync(hm, mx, sizeof(hm), cudaMemcpyDeviceToHost, s));
  SCVS_CUDA(cudaMemcpyAsync(&fp_total, rb.fp_ptr + rb.n_blk, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  SCVS_CUDA(cudaStreamSynchronize(s));
  const int derr = dev_error(c);
  rb.fp_max = hm[0];
  rb.fv_max = hm[1];
  rb.fp_total = fp_total;
  bool ok = derr == 0 && rb.fp_max <= 65535;
  if (ok) {
    rb.fp_col = m.arena.alloc<int32_t>(std::max<int64_t>(fp_total, 1));
    rb.lcol = m.arena.alloc<uint16_t>(m.s_nnz);
    k_block_footprint<true><<<(unsigned)rb.n_blk, 1024, 0, s>>>(rb.perm, rb.row0, m.s_ptr, m.s_col, m.P, fpl,
                                                               rb.fv_len, rb.fp_ptr, rb.fp_col, rb.lcol, c.dev_err);
    count_launch(c);
  }
  for (void *p : {(void *)keys, (void *)plen, (void *)cum, (void *)fpl, (void *)mx}) SCVS_CUDA(cudaFreeAsync(p, s));
  SCVS_CUDA(cudaStreamSynchronize(s));
  if (!ok || dev_error(c)) { rb.n_blk = 0; return; }
  rb.budget = budget;
  rb.valid = true;
}

// ------------------------------------------------- staging (TMA bulk copies)
__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

constexpr long long MBAR_SPIN = 1ll << 20;

// Wait for phase 0 of the staging barrier, with a poll limit.  On a time-out
// the error word of the grid barrier is set (the host reports
// SCVS_ERR_TIMEOUT), the copies still in flight get a second bounded wait,
// and false is returned (the block then leaves without computing).
__device__ __forceinline__ bool stage_wait(uint64_t *bar, GridSync *gs) {
  long long n = 0;
  while (!mbar_try_wait(bar, 0)) {
    if (++n > MBAR_SPIN) {
      if (threadIdx.x == 0) atomicExch(&gs->err, 2);
      for (long long q = 0; q < MBAR_SPIN && !mbar_try_wait(bar, 0); ++q) __nanosleep(256);
      return false;
    }
    if (n > 64) __nanosleep(32);
  }
  return true;
}

// Copy the footprint of block b, mode chunk [k0, k0 + MC), into shared memory:
// xs[j][c][MC] for every footprint column j and component c, and (with
// PRES) ps[j][MC] = the pressure entries of the vertex columns j < fv.
// Chunks of at least 256 bytes (MC = 32) go by TMA bulk copies issued by warp
// 0 (each 16-byte aligned: k0 and ld are multiples of MC, the block base is
// 16-byte aligned; when MC = ld the DIM chunks of a column are one
// contiguous copy), completing on an mbarrier; smaller chunks by 16-byte
// cp.async copies spread over all threads (a TMA request per 32-128 bytes
// costs more than it moves).
template <int MC, int DIM, bool PRES>
__device__ __forceinline__ bool stage_footprint(const float2 *__restrict__ x, int ld, int64_t N, const int32_t *cols,
                                                int u, int fv, int k0, float2 *xs, float2 *ps, uint64_t *bar,
                                                GridSync *gs) {
  if constexpr (MC >= 32) {
    if (threadIdx.x == 0) mbar_init(bar, 1);
    __syncthreads();
    if (threadIdx.x < 32) {
      const unsigned chunk = MC * sizeof(float2);
      const bool whole = MC == ld;  // the DIM chunks of a column are contiguous
      if (threadIdx.x == 0) mbar_expect_tx(bar, chunk * (unsigned)(u * DIM + (PRES ? fv : 0)));
      __syncwarp();
      for (int j = threadIdx.x; j < u; j += 32) {
        const int64_t col = cols[j];
        if (whole) {
          bulk_g2s(xs + (int64_t)j * DIM * MC, x + col * DIM * ld + k0, chunk * DIM, bar);
        } else {
#pragma unroll
          for (int cc = 0; cc < DIM; ++cc)
            bulk_g2s(xs + ((int64_t)j * DIM + cc) * MC, x + (col * DIM + cc) * ld + k0, chunk, bar);
        }
        if (PRES && j < fv) bulk_g2s(ps + (int64_t)j * MC, x + ((int64_t)DIM * N + col) * ld + k0, chunk, bar);
      }
    }
    return stage_wait(bar, gs);
  } else {
    (void)bar;
    (void)gs;
    constexpr int PC = MC / 2;  // 16-byte pieces per chunk (two complex FP32)
    const int nx = u * DIM * PC;
    for (int idx = threadIdx.x; idx < nx; idx += blockDim.x) {
      const int j = idx / (DIM * PC), rem = idx % (DIM * PC), cc = rem / PC, pc = rem % PC;
      const float2 *src = x + ((int64_t)cols[j] * DIM + cc) * ld + k0 + 2 * pc;
      const uint32_t dst = smem_addr(xs + ((int64_t)j * DIM + cc) * MC + 2 * pc);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
    }
    if (PRES)
      for (int idx = threadIdx.x; idx < fv * PC; idx += blockDim.x) {
        const int j = idx / PC, pc = idx % PC;
        const float2 *src = x + ((int64_t)DIM * N + cols[j]) * ld + k0 + 2 * pc;
        const uint32_t dst = smem_addr(ps + (int64_t)j * MC + 2 * pc);
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
      }
    asm volatile("cp.async.commit_group;\n cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    return true;
  }
}

// Shared-memory layout of one block: the mbarrier, then xs, then ps.
template <int MC, int DIM, bool PRES>
__host__ __device__ constexpr size_t stage_bytes(int fp_max, int fv_max) {
  return 16 + ((size_t)fp_max * DIM + (PRES ? (size_t)fv_max : 0)) * MC * sizeof(float2);
}

// 16-byte loads of a lane's two modes from shared memory
__device__ __forceinline__ void lds2(CV<float, 2> &v, const float2 *p) {
  const float4 f = *reinterpret_cast<const float4 *>(p);
  v.re[0] = f.x; v.im[0] = f.y; v.re[1] = f.z; v.im[1] = f.w;
}

// ------------------------------------------------ staged Chebyshev step
// Same step as k_pc_cheb (operators.cu) on the rows of one block, gathering z
// from shared memory.  Block = (row block b, mode chunk mc); a lane owns 2
// modes, LG = MC / 2 lanes per row.
template <int MC, int DIM>
__global__ void __launch_bounds__(256)
k_pc_cheb_st(const PcArgs a, const ChebCoef cc, const StagedArgs st, const float2 *__restrict__ r,
             const float2 *__restrict__ zu, float2 *__restrict__ zu_prev) {
  constexpr int LG = MC / 2;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  float2 *xs = reinterpret_cast<float2 *>(smem + 16);
  const int n_mc = a.ld / MC;
  const int b = blockIdx.x / n_mc, mc = blockIdx.x % n_mc, k0 = mc * MC;
  const int64_t i0 = st.row0[b], i1 = st.row0[b + 1];
  const int64_t f0 = st.fp_ptr[b];
  const int u = (int)(st.fp_ptr[b + 1] - f0);
  if (!stage_footprint<MC, DIM, false>(zu, a.ld, a.N, st.fp_col + f0, u, 0, k0, xs, nullptr, bar, st.gs)) return;
  const int lane = threadIdx.x % LG, group = threadIdx.x / LG;
  const unsigned gm = group_mask<LG>();
  const int ld = a.ld, koff = k0 + lane * 2;
  const float *Kv = (const float *)a.Kv, *Mv = (const float *)a.Mv;
  float cw[2];
  cw[0] = ((const float *)a.wabs)[koff];
  cw[1] = ((const float *)a.wabs)[koff + 1];
  const float muT = (float)a.mu;
  for (int64_t i = i0 + group; i < i1; i += 256 / LG) {
    const int64_t A = st.perm[i];
    if (row_idle(a.dof_comp, a.comp_active, A * DIM)) continue;
    if (a.dirmask[A]) {
#pragma unroll
      for (int c = 0; c < DIM; ++c) {
        CV<float, 2> v;
        ldv<float, 2>(v, r + (A * DIM + c) * ld + koff);
        stv<float, 2>(zu_prev + (A * DIM + c) * ld + koff, v);
      }
      continue;
    }
    CV<float, 2> acc[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) acc[c].zero();
    const int64_t r0 = a.s_ptr[A], r1 = a.s_ptr[A + 1];
    for (int64_t base = r0; base < r1; base += LG) {
      const int64_t t = base + lane;
      int lc = 0;
      float kv = 0, mv = 0;
      if (t < r1) { lc = st.lcol[t]; kv = muT * __ldg(Kv + t); mv = __ldg(Mv + t); }
      const int cnt = (int)min((int64_t)LG, r1 - base);
#pragma unroll 4
      for (int q = 0; q < cnt; ++q) {
        const int B = gshfl<LG>(gm, lc, q);
        const float kq = gshfl<LG>(gm, kv, q), mq = gshfl<LG>(gm, mv, q);
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          CV<float, 2> xv;
          lds2(xv, xs + ((int64_t)B * DIM + c) * MC + lane * 2);
#pragma unroll
          for (int m2 = 0; m2 < 2; ++m2) {
            const float cf = fmaf(cw[m2], mq, kq);
            acc[c].re[m2] = fmaf(cf, xv.re[m2], acc[c].re[m2]);
            acc[c].im[m2] = fmaf(cf, xv.im[m2], acc[c].im[m2]);
          }
        }
      }
    }
    float dr[2], al[2], be[2];
#pragma unroll
    for (int m2 = 0; m2 < 2; ++m2) {
      dr[m2] = vel_dinv<float>(a, A, koff + m2);
      al[m2] = (float)cc.alpha_u[koff + m2];
      be[m2] = (float)cc.beta_u[koff + m2];
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      const int64_t f = (A * DIM + c) * ld + koff;
      CV<float, 2> rv, z, zp, o;
      ldv<float, 2>(rv, r + f);
      ldv<float, 2>(z, zu + f);
      if (cc.prev_zero_u) zp.zero(); else ldv_cg<float, 2>(zp, zu_prev + f);
#pragma unroll
      for (int m2 = 0; m2 < 2; ++m2) {
        const float ur = dr[m2] * (rv.re[m2] - acc[c].re[m2]), ui = dr[m2] * (rv.im[m2] - acc[c].im[m2]);
        o.re[m2] = z.re[m2] + al[m2] * (z.re[m2] - zp.re[m2]) + be[m2] * ur;
        o.im[m2] = z.im[m2] + al[m2] * (z.im[m2] - zp.im[m2]) + be[m2] * ui;
      }
      stv<float, 2>(zu_prev + f, o);
    }
  }
}

// rr = r - A_r z on the rows of one block (k_vel_residual, staged).
template <int MC, int DIM>
__global__ void __launch_bounds__(256)
k_vel_residual_st(const PcArgs a, const StagedArgs st, const float2 *__restrict__ r, const float2 *__restrict__ z,
                  float2 *__restrict__ rr) {
  constexpr int LG = MC / 2;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  float2 *xs = reinterpret_cast<float2 *>(smem + 16);
  const int n_mc = a.ld / MC;
  const int b = blockIdx.x / n_mc, mc = blockIdx.x % n_mc, k0 = mc * MC;
  const int64_t i0 = st.row0[b], i1 = st.row0[b + 1];
  const int64_t f0 = st.fp_ptr[b];
  const int u = (int)(st.fp_ptr[b + 1] - f0);
  if (!stage_footprint<MC, DIM, false>(z, a.ld, a.N, st.fp_col + f0, u, 0, k0, xs, nullptr, bar, st.gs)) return;
  const int lane = threadIdx.x % LG, group = threadIdx.x / LG;
  const unsigned gm = group_mask<LG>();
  const int ld = a.ld, koff = k0 + lane * 2;
  const float *Kv = (const float *)a.Kv, *Mv = (const float *)a.Mv;
  float cr[2];
  cr[0] = ((const float *)a.wabs)[koff];
  cr[1] = ((const float *)a.wabs)[koff + 1];
  const float mu = (float)a.mu;
  for (int64_t i = i0 + group; i < i1; i += 256 / LG) {
    const int64_t A = st.perm[i];
    if (row_idle(a.dof_comp, a.comp_active, A * DIM)) continue;
    if (a.dirmask[A]) {
      CV<float, 2> zz;
      zz.zero();
#pragma unroll
      for (int c = 0; c < DIM; ++c) stv<float, 2>(rr + (A * DIM + c) * ld + koff, zz);
      continue;
    }
    CV<float, 2> acc[DIM];
#pragma unroll
    for (int c = 0; c < DIM; ++c) acc[c].zero();
    const int64_t r0 = a.s_ptr[A], r1 = a.s_ptr[A + 1];
    for (int64_t base = r0; base < r1; base += LG) {
      const int64_t t = base + lane;
      int lc = 0;
      float kv = 0, mv = 0;
      if (t < r1) { lc = st.lcol[t]; kv = __ldg(Kv + t); mv = __ldg(Mv + t); }
      const int cnt = (int)min((int64_t)LG, r1 - base);
#pragma unroll 4
      for (int q = 0; q < cnt; ++q) {
        const int B = gshfl<LG>(gm, lc, q);
        const float kq = mu * gshfl<LG>(gm, kv, q), mq = gshfl<LG>(gm, mv, q);
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          CV<float, 2> xv;
          lds2(xv, xs + ((int64_t)B * DIM + c) * MC + lane * 2);
#pragma unroll
          for (int m2 = 0; m2 < 2; ++m2) {
            const float cf = kq + cr[m2] * mq;
            acc[c].re[m2] = fmaf(cf, xv.re[m2], acc[c].re[m2]);
            acc[c].im[m2] = fmaf(cf, xv.im[m2], acc[c].im[m2]);
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < DIM; ++c) {
      CV<float, 2> rv, o;
      ldv<float, 2>(rv, r + (A * DIM + c) * ld + koff);
#pragma unroll
      for (int m2 = 0; m2 < 2; ++m2) { o.re[m2] = rv.re[m2] - acc[c].re[m2]; o.im[m2] = rv.im[m2] - acc[c].im[m2]; }
      stv<float, 2>(rr + (A * DIM + c) * ld + koff, o);
    }
  }
}

// ------------------------------------------------ staged all-modes SpMM
// y_k = A_hat(omega_k) x_k on the rows of one block (k_saddle<float>,
// staged): the velocity rows of every node of the block and the pressure row
// of every vertex node of it, x_u of the footprint and x_p of its vertex
// prefix in shared memory.
template <int MC, int DIM>
__global__ void __launch_bounds__(256)
k_saddle_st(const SaddleArgs<float> a, const StagedArgs st, const float2 *__restrict__ x, float2 *__restrict__ y) {
  constexpr int LG = MC / 2;
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(smem);
  const int n_mc = a.ld / MC;
  const int b = blockIdx.x / n_mc, mc = blockIdx.x % n_mc, k0 = mc * MC;
  const int64_t i0 = st.row0[b], i1 = st.row0[b + 1];
  const int64_t f0 = st.fp_ptr[b];
  const int u = (int)(st.fp_ptr[b + 1] - f0), fv = st.fv_len[b];
  float2 *xs = reinterpret_cast<float2 *>(smem + 16);
  float2 *ps = xs + (int64_t)st.fp_max * DIM * MC;
  if (!stage_footprint<MC, DIM, true>(x, a.ld, a.N, st.fp_col + f0, u, fv, k0, xs, ps, bar, st.gs)) return;
  const int lane = threadIdx.x % LG, group = threadIdx.x / LG;
  const unsigned gm = group_mask<LG>();
  const int ld = a.ld, koff = k0 + lane * 2;
  float wr[2];
  wr[0] = (float)(a.omega[koff] * a.rho);
  wr[1] = (float)(a.omega[koff + 1] * a.rho);
  const float mu = (float)a.mu;
  // every node's velocity rows, then (second sweep) the vertex nodes' pressure rows
  for (int64_t w = group; w < 2 * (i1 - i0); w += 256 / LG) {
    const bool prow = w >= (i1 - i0);
    const int64_t A = st.perm[i0 + (prow ? w - (i1 - i0) : w)];
    if (!prow) {
      if (row_idle(a.dof_comp, a.comp_active, A * DIM)) continue;
      if (a.dirmask && a.dirmask[A]) {
#pragma unroll
        for (int c = 0; c < DIM; ++c) {
          CV<float, 2> v;
          ldv<float, 2>(v, x + (A * DIM + c) * ld + koff);
          stv<float, 2>(y + (A * DIM + c) * ld + koff, v);
        }
        continue;
      }
      CV<float, 2> acc[DIM];
#pragma unroll
      for (int c = 0; c < DIM; ++c) acc[c].zero();
      const int64_t r0 = a.s_ptr[A], r1 = a.s_ptr[A + 1];
      const int64_t gend = r0 + a.g_len[A];
      const int64_t goff = a.g_ptr[A] - r0;
      for (int64_t base = r0; base < r1; base += LG) {
        const int64_t t = base + lane;
        int lc = 0;
        float kv = 0, mv = 0, dv[DIM];
#pragma unroll
        for (int c = 0; c < DIM; ++c) dv[c] = 0;
        if (t < r1) {
          lc = st.lcol[t];
          kv = mu * __ldg(a.Kv + t);
          mv = __ldg(a.Mv + t);
          if (t < gend) {
#pragma unroll
            for (int c = 0; c < DIM; ++c) dv[c] = __ldg(a.Dv + c * a.g_nnz + t + goff);
          }
        }
        const int cnt = (int)min((int64_t)LG, r1 - base);
        const int gcnt = (int)max((int64_t)0, min((int64_t)LG, gend - base));
#pragma unroll 4
        for (int q = 0; q < cnt; ++q) {
          const int B = gshfl<LG>(gm, lc, q);
          const float cr = gshfl<LG>(gm, kv, q), mq = gshfl<LG>(gm, mv, q);
          float ci[2];
          ci[0] = wr[0] * mq;
          ci[1] = wr[1] * mq;
#pragma unroll
          for (int c = 0; c < DIM; ++c) {
            CV<float, 2> xv;
            lds2(xv, xs + ((int64_t)B * DIM + c) * MC + lane * 2);
#pragma unroll
            for (int m2 = 0; m2 < 2; ++m2) {
              acc[c].re[m2] = fmaf(cr, xv.re[m2], fmaf(-ci[m2], xv.im[m2], acc[c].re[m2]));
              acc[c].im[m2] = fmaf(cr, xv.im[m2], fmaf(ci[m2], xv.re[m2], acc[c].im[m2]));
            }
          }
          if (q < gcnt) {  // uniform across the row group; vertex columns are the footprint's prefix
            CV<float, 2> xq;
            lds2(xq, ps + (int64_t)B * MC + lane * 2);
#pragma unroll
            for (int c = 0; c < DIM; ++c) axpy(acc[c], gshfl<LG>(gm, dv[c], q), xq);
          }
        }
      }
#pragma unroll
      for (int c = 0; c < DIM; ++c) stv<float, 2>(y + (A * DIM + c) * ld + koff, acc[c]);
    } else {
      if (A >= a.P) continue;
      const int64_t Bv = A;
      if (row_idle(a.dof_comp, a.comp_active, (int64_t)DIM * a.N + Bv)) continue;
      CV<float, 2> acc;
      acc.zero();
      const int64_t r0 = a.s_ptr[Bv], r1 = a.s_ptr[Bv + 1];
      for (int64_t base = r0; base < r1; base += LG) {
        const int64_t t = base + lane;
        int lc = 0;
        float dt[DIM];
#pragma unroll
        for (int c = 0; c < DIM; ++c) dt[c] = 0;
        if (t < r1) {
          lc = st.lcol[t];
#pragma unroll
          for (int c = 0; c < DIM; ++c) dt[c] = __ldg(a.DTv + c * a.gt_nnz + t);
        }
        const int cnt = (int)min((int64_t)LG, r1 - base);
#pragma unroll 4
        for (int q = 0; q < cnt; ++q) {
          const int Bc = gshfl<LG>(gm, lc, q);
#pragma unroll
          for (int c = 0; c < DIM; ++c) {
            CV<float, 2> xv;
            lds2(xv, xs + ((int64_t)Bc * DIM + c) * MC + lane * 2);
            axpy(acc, gshfl<LG>(gm, dt[c], q), xv);
          }
        }
      }
      stv<float, 2>(y + ((int64_t)DIM * a.N + Bv) * ld + koff, acc);
    }
  }
}

// ------------------------------------------------------------- launchers
StagedArgs staged_args(const Ctx &c, const Mesh &m) {
  const RowBlocks &rb = m.rb;
  return StagedArgs{rb.perm, rb.row0, rb.fp_ptr, rb.fp_col, rb.fv_len, rb.lcol, rb.fp_max, c.gsync};
}

static int stage_mc(int ld, int mc) { return std::min(ld, mc); }

// true if the staged kernels can run on this mesh with mode chunk mc for the
// vector x (16-byte aligned base, footprint within shared memory)
bool staged_ok(const Ctx &c, const Mesh &m, int mc, bool pres, const void *x) {
  if (!m.rb.valid || mc <= 0 || (reinterpret_cast<uintptr_t>(x) & 15) != 0) return false;
  const int MC = stage_mc(m.ld, mc);
  if (MC < 2 || m.ld % MC != 0) return false;
  const size_t bytes = 16 + ((size_t)m.rb.fp_max * m.dim + (pres ? (size_t)m.rb.fv_max : 0)) * MC * sizeof(float2);
  (void)c;
  return bytes <= STAGE_SMEM_MAX;
}

#define SCVS_DISPATCH_MC(mcv, ...)                            \
  do {                                                        \
    switch (mcv) {                                            \
      case 2: { constexpr int MC = 2; __VA_ARGS__; } break;   \
      case 4: { constexpr int MC = 4; __VA_ARGS__; } break;   \
      case 8: { constexpr int MC = 8; __VA_ARGS__; } break;   \
      case 16: { constexpr int MC = 16; __VA_ARGS__; } break; \
      case 32: { constexpr int MC = 32; __VA_ARGS__; } break; \
      default: throw (int)SCVS_ERR_ARG;                       \
    }                                                         \
  } while (0)

void launch_cheb_staged(Ctx &c, const Mesh &m, const PcArgs &a, const ChebCoef &cc, const float2 *r, const float2 *zu,
                        float2 *zu_prev, int mc) {
  const StagedArgs st = staged_args(c, m);
  const int MCv = stage_mc(m.ld, mc);
  const unsigned grid = (unsigned)(m.rb.n_blk * (m.ld / MCv));
  SCVS_DISPATCH_MC(MCv, {
    const size_t smem = stage_bytes<MC, 3, false>(m.rb.fp_max, 0);
    if (m.dim == 2) {
      const size_t sm2 = stage_bytes<MC, 2, false>(m.rb.fp_max, 0);
      SCVS_CUDA(cudaFuncSetAttribute(k_pc_cheb_st<MC, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
      k_pc_cheb_st<MC, 2><<<grid, 256, sm2, c.stream>>>(a, cc, st, r, zu, zu_prev);
    } else {
      SCVS_CUDA(cudaFuncSetAttribute(k_pc_cheb_st<MC, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      k_pc_cheb_st<MC, 3><<<grid, 256, smem, c.stream>>>(a, cc, st, r, zu, zu_prev);
    }
  });
  count_launch(c);
}

void launch_vel_residual_staged(Ctx &c, const Mesh &m, const PcArgs &a, const float2 *r, const float2 *z, float2 *rr,
                                int mc) {
  const StagedArgs st = staged_args(c, m);
  const int MCv = stage_mc(m.ld, mc);
  const unsigned grid = (unsigned)(m.rb.n_blk * (m.ld / MCv));
  SCVS_DISPATCH_MC(MCv, {
    if (m.dim == 2) {
      const size_t sm2 = stage_bytes<MC, 2, false>(m.rb.fp_max, 0);
      SCVS_CUDA(cudaFuncSetAttribute(k_vel_residual_st<MC, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
      k_vel_residual_st<MC, 2><<<grid, 256, sm2, c.stream>>>(a, st, r, z, rr);
    } else {
      const size_t sm3 = stage_bytes<MC, 3, false>(m.rb.fp_max, 0);
      SCVS_CUDA(cudaFuncSetAttribute(k_vel_residual_st<MC, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
      k_vel_residual_st<MC, 3><<<grid, 256, sm3, c.stream>>>(a, st, r, z, rr);
    }
  });
  count_launch(c);
}

void launch_saddle_staged(Ctx &c, const Mesh &m, const SaddleArgs<float> &a, const float2 *x, float2 *y, int mc) {
  const StagedArgs st = staged_args(c, m);
  const int MCv = stage_mc(m.ld, mc);
  const unsigned grid = (unsigned)(m.rb.n_blk * (m.ld / MCv));
  SCVS_DISPATCH_MC(MCv, {
    if (m.dim == 2) {
      const size_t sm2 = stage_bytes<MC, 2, true>(m.rb.fp_max, m.rb.fv_max);
      SCVS_CUDA(cudaFuncSetAttribute(k_saddle_st<MC, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2));
      k_saddle_st<MC, 2><<<grid, 256, sm2, c.stream>>>(a, st, x, y);
    } else {
      const size_t sm3 = stage_bytes<MC, 3, true>(m.rb.fp_max, m.rb.fv_max);
      SCVS_CUDA(cudaFuncSetAttribute(k_saddle_st<MC, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm3));
      k_saddle_st<MC, 3><<<grid, 256, sm3, c.stream>>>(a, st, x, y);
    }
  });
  count_launch(c);
}

}  // namespace scvs
