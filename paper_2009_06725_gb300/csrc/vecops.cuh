// Small vector helpers for mode-interleaved complex blocks.
//
// A thread ("lane" of a row group of L threads) owns MPL consecutive modes of
// a row; a row of a block is ld = L * MPL complex numbers, so a group reads
// one contiguous row with vector loads.
#pragma once
#include "common.cuh"

namespace scvs {

template <typename T, int MPL> struct CV {
  T re[MPL], im[MPL];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < MPL; ++i) { re[i] = T(0); im[i] = T(0); }
  }
};

template <typename T, int MPL>
__device__ __forceinline__ void ldv(CV<T, MPL> &v, const typename cpx<T>::t *p) {
#pragma unroll
  for (int i = 0; i < MPL; ++i) { auto z = __ldg(p + i); v.re[i] = z.x; v.im[i] = z.y; }
}
template <>
__device__ __forceinline__ void ldv<float, 2>(CV<float, 2> &v, const float2 *p) {
  float4 f = __ldg(reinterpret_cast<const float4 *>(p));
  v.re[0] = f.x; v.im[0] = f.y; v.re[1] = f.z; v.im[1] = f.w;
}
template <>
__device__ __forceinline__ void ldv<float, 4>(CV<float, 4> &v, const float2 *p) {
  float4 f = __ldg(reinterpret_cast<const float4 *>(p));
  float4 g = __ldg(reinterpret_cast<const float4 *>(p) + 1);
  v.re[0] = f.x; v.im[0] = f.y; v.re[1] = f.z; v.im[1] = f.w;
  v.re[2] = g.x; v.im[2] = g.y; v.re[3] = g.z; v.im[3] = g.w;
}
// plain (coherent) load for buffers written earlier in the same kernel
template <typename T, int MPL>
__device__ __forceinline__ void ldv_cg(CV<T, MPL> &v, const typename cpx<T>::t *p) {
#pragma unroll
  for (int i = 0; i < MPL; ++i) { auto z = p[i]; v.re[i] = z.x; v.im[i] = z.y; }
}
template <>
__device__ __forceinline__ void ldv_cg<float, 2>(CV<float, 2> &v, const float2 *p) {
  float4 f = *reinterpret_cast<const float4 *>(p);
  v.re[0] = f.x; v.im[0] = f.y; v.re[1] = f.z; v.im[1] = f.w;
}

// Coherent loads (ld.global.ca, never the read-only path) for data a
// persistent kernel itself wrote before a grid barrier: the read-only path is
// only valid for data that stays unchanged for the whole launch.
__device__ __forceinline__ float ld1co(const float *p) { return __ldca(p); }
__device__ __forceinline__ int ld1co(const int *p) { return __ldca(p); }
__device__ __forceinline__ float2 ld1co(const float2 *p) { return __ldca(p); }
__device__ __forceinline__ double2 ld1co(const double2 *p) { return __ldca(p); }
template <typename T, int MPL>
__device__ __forceinline__ void ldv_co(CV<T, MPL> &v, const typename cpx<T>::t *p) {
#pragma unroll
  for (int i = 0; i < MPL; ++i) { auto z = ld1co(p + i); v.re[i] = z.x; v.im[i] = z.y; }
}
template <>
__device__ __forceinline__ void ldv_co<float, 2>(CV<float, 2> &v, const float2 *p) {
  float4 f = __ldca(reinterpret_cast<const float4 *>(p));
  v.re[0] = f.x; v.im[0] = f.y; v.re[1] = f.z; v.im[1] = f.w;
}
template <>
__device__ __forceinline__ void ldv_co<float, 4>(CV<float, 4> &v, const float2 *p) {
  float4 f = __ldca(reinterpret_cast<const float4 *>(p));
  float4 g = __ldca(reinterpret_cast<const float4 *>(p) + 1);
  v.re[0] = f.x; v.im[0] = f.y; v.re[1] = f.z; v.im[1] = f.w;
  v.re[2] = g.x; v.im[2] = g.y; v.re[3] = g.z; v.im[3] = g.w;
}

template <typename T, int MPL>
__device__ __forceinline__ void stv(typename cpx<T>::t *p, const CV<T, MPL> &v) {
#pragma unroll
  for (int i = 0; i < MPL; ++i) p[i] = mk<T>(v.re[i], v.im[i]);
}
template <>
__device__ __forceinline__ void stv<float, 2>(float2 *p, const CV<float, 2> &v) {
  *reinterpret_cast<float4 *>(p) = make_float4(v.re[0], v.im[0], v.re[1], v.im[1]);
}
template <>
__device__ __forceinline__ void stv<float, 4>(float2 *p, const CV<float, 4> &v) {
  reinterpret_cast<float4 *>(p)[0] = make_float4(v.re[0], v.im[0], v.re[1], v.im[1]);
  reinterpret_cast<float4 *>(p)[1] = make_float4(v.re[2], v.im[2], v.re[3], v.im[3]);
}

// acc += s * v (s real)
template <typename T, int MPL>
__device__ __forceinline__ void axpy(CV<T, MPL> &acc, T s, const CV<T, MPL> &v) {
#pragma unroll
  for (int i = 0; i < MPL; ++i) { acc.re[i] = fma(s, v.re[i], acc.re[i]); acc.im[i] = fma(s, v.im[i], acc.im[i]); }
}

// Row-group shuffle: broadcast from lane q of this group of L lanes.
template <int L, typename V>
__device__ __forceinline__ V gshfl(unsigned mask, V v, int q) {
  return __shfl_sync(mask, v, q, L);
}

template <int L>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (L >= 32) {
    return 0xffffffffu;
  } else {
    const unsigned base = (threadIdx.x & 31) / L * L;
    return ((1u << L) - 1u) << base;
  }
}

#define SCVS_SHAPE_KEY(LDV, MPLV) ((LDV) * 8 + (MPLV))
// Row-group shapes: a row of ld modes is split over L = ld / MPL lanes with
// MPL modes each.  SCVS_DISPATCH_SHAPE instantiates every valid (ld, MPL)
// pair (ld a power of two in [2, 128], MPL in {1, 2, 4}, L <= 32);
// SCVS_DISPATCH_LD picks the default shape (16-byte loads per lane).
#define SCVS_SHAPE_CASE(LDV, MPLV, ...)                  \
  case SCVS_SHAPE_KEY(LDV, MPLV): {                      \
    constexpr int MPL = MPLV, L = (LDV) / (MPLV);        \
    __VA_ARGS__;                                         \
  } break;

#define SCVS_DISPATCH_SHAPE(ld, mpl, ...)                                                       \
  do {                                                                                          \
    switch (SCVS_SHAPE_KEY(ld, mpl)) {                                                                 \
      SCVS_SHAPE_CASE(2, 1, __VA_ARGS__) SCVS_SHAPE_CASE(2, 2, __VA_ARGS__)                      \
      SCVS_SHAPE_CASE(4, 1, __VA_ARGS__) SCVS_SHAPE_CASE(4, 2, __VA_ARGS__)                      \
      SCVS_SHAPE_CASE(4, 4, __VA_ARGS__) SCVS_SHAPE_CASE(8, 1, __VA_ARGS__)                      \
      SCVS_SHAPE_CASE(8, 2, __VA_ARGS__) SCVS_SHAPE_CASE(8, 4, __VA_ARGS__)                      \
      SCVS_SHAPE_CASE(16, 1, __VA_ARGS__) SCVS_SHAPE_CASE(16, 2, __VA_ARGS__)                    \
      SCVS_SHAPE_CASE(16, 4, __VA_ARGS__) SCVS_SHAPE_CASE(32, 1, __VA_ARGS__)                    \
      SCVS_SHAPE_CASE(32, 2, __VA_ARGS__) SCVS_SHAPE_CASE(32, 4, __VA_ARGS__)                    \
      SCVS_SHAPE_CASE(64, 2, __VA_ARGS__) SCVS_SHAPE_CASE(64, 4, __VA_ARGS__)                    \
      SCVS_SHAPE_CASE(128, 4, __VA_ARGS__)                                                      \
      default: throw (int)SCVS_ERR_ARG;                                                         \
    }                                                                                           \
  } while (0)

template <typename T>
inline int default_mpl(int ld) {
  if (sizeof(T) == 4) return ld >= 128 ? 4 : 2;
  return ld >= 128 ? 4 : (ld >= 64 ? 2 : 1);
}
inline bool shape_valid(int ld, int mpl) { return mpl >= 1 && mpl <= 4 && ld % mpl == 0 && ld / mpl <= 32 && !(ld == 2 && mpl == 4); }

#define SCVS_LD_CASE(LDV, MPLV, ...)                     \
  case (LDV): {                                          \
    constexpr int MPL = MPLV, L = (LDV) / (MPLV);        \
    __VA_ARGS__;                                         \
  } break;

// default shape only (kernels that are not autotuned)
#define SCVS_DISPATCH_LD(T, ld, ...)                                           \
  do {                                                                         \
    if constexpr (sizeof(T) == 4) {                                            \
      switch (ld) {                                                            \
        SCVS_LD_CASE(2, 2, __VA_ARGS__) SCVS_LD_CASE(4, 2, __VA_ARGS__)   \
        SCVS_LD_CASE(8, 2, __VA_ARGS__) SCVS_LD_CASE(16, 2, __VA_ARGS__)  \
        SCVS_LD_CASE(32, 2, __VA_ARGS__) SCVS_LD_CASE(64, 2, __VA_ARGS__) \
        SCVS_LD_CASE(128, 4, __VA_ARGS__)                                   \
        default: throw (int)SCVS_ERR_ARG;                                      \
      }                                                                        \
    } else {                                                                   \
      switch (ld) {                                                            \
        SCVS_LD_CASE(2, 1, __VA_ARGS__) SCVS_LD_CASE(4, 1, __VA_ARGS__)   \
        SCVS_LD_CASE(8, 1, __VA_ARGS__) SCVS_LD_CASE(16, 1, __VA_ARGS__)  \
        SCVS_LD_CASE(32, 1, __VA_ARGS__) SCVS_LD_CASE(64, 2, __VA_ARGS__) \
        SCVS_LD_CASE(128, 4, __VA_ARGS__)                                   \
        default: throw (int)SCVS_ERR_ARG;                                      \
      }                                                                        \
    }                                                                          \
  } while (0)

// Row scheduling of the gather kernels.  Rows [lo, hi) are cut into tiles of
// gpb * tile consecutive rows; block b takes tiles b, b + gridDim.x, ... and
// its row groups walk a tile's rows in order.  Consecutive rows of a mesh
// share most of their neighbours, so a larger tile keeps the gathered vector
// entries in the SM's L1 across rows; tile 1 is a plain grid-stride loop.
#define SCVS_ROW_LOOP(row, lo, hi, gpb, group, tile)                                                  \
  for (int64_t row##_t0 = (int64_t)(lo) + (int64_t)blockIdx.x * (gpb) * (tile); row##_t0 < (int64_t)(hi); \
       row##_t0 += (int64_t)gridDim.x * (gpb) * (tile))                                                \
    for (int64_t row = row##_t0 + (group),                                                            \
                 row##_te = min(row##_t0 + (int64_t)(gpb) * (tile), (int64_t)(hi));                   \
         row < row##_te; row += (gpb))

// candidate row tiles of the autotuner (rows per tile = row groups per block x tile)
constexpr int SCVS_TILES[5] = {1, 2, 4, 8, 16};
constexpr int SCVS_DEFAULT_TILE = 4;

}  // namespace scvs
