// FP32 pass kernels and batch units for the lengths 3 x 2^k and 5 x 2^k with
// compile-time transform lengths (see fs_mixed.h).  FS_MX_ODD selects the
// family compiled into this object (3 or 5), so the two compile in parallel.
#include "fs_col_tma.cuh"
#include "fs_mixed.h"
#include "fs_row_async.cuh"
#include "fs_units.cuh"

#ifndef FS_MX_ODD
#error "FS_MX_ODD (3 or 5) must be defined"
#endif

namespace fs {

#if FS_MX_ODD == 3
#define FS_MX_COLS(X) X(192) X(384) X(768) X(1536) X(3072) X(6144)
#define FS_MX_ROWS(X) X(192) X(384) X(768) X(1536) X(3072)
#define FS_MX_SUFFIX 3
#else
#define FS_MX_COLS(X) X(160) X(320) X(640) X(1280) X(2560) X(5120)
#define FS_MX_ROWS(X) X(160) X(320) X(640) X(1280) X(2560)
#define FS_MX_SUFFIX 5
#endif

template <int M, int CC>
__device__ __noinline__ void mx_r2c_unit(const Desc &d, int unit, cx<float> *sm, const float *in, cx<float> *spec) {
  unit_row_r2c_t<float, mx_e(M), M, CC>(d, unit, CC, sm, in, spec);
}
template <int M, int CC>
__device__ __noinline__ void mx_c2r_unit(const Desc &d, int unit, cx<float> *sm, const cx<float> *spec, float *out,
                                         bool sh) {
  unit_row_c2r_t<float, mx_e(M), M, CC>(d, unit, CC, sm, spec, out, sh);
}
template <int L>
__device__ __noinline__ void mx_col1_unit(const Desc &d, int unit, int cnt, cx<float> *sm, cx<float> *wu,
                                          cx<float> *wv, bool sh) {
  unit_col_t<float, mx_e(L), false, L, 0>(d, unit, cnt, sm, wu, wv, sh);
}

// one family per object: the dispatchers below have a per-family name and
// the public ones (fs_mixed_dispatch) try both
#define FS_CAT2(a, b) a##b
#define FS_CAT(a, b) FS_CAT2(a, b)

__device__ bool FS_CAT(mx_unit_r2c_, FS_MX_SUFFIX)(const Desc &d, int unit, int cnt, cx<float> *sm,
                                                    const float *in, cx<float> *spec) {
  switch (d.M) {
#define C(m)                                                              \
  case m:                                                                 \
    if (d.rp_row.e != mx_e(m)) return false;                              \
    if (cnt == mx_row_cnt(m)) {                                           \
      mx_r2c_unit<m, mx_row_cnt(m)>(d, unit, sm, in, spec);               \
      return true;                                                        \
    }                                                                     \
    if (mx_row_cnt_256(m) != mx_row_cnt(m) && cnt == mx_row_cnt_256(m)) { \
      mx_r2c_unit<m, mx_row_cnt_256(m)>(d, unit, sm, in, spec);           \
      return true;                                                        \
    }                                                                     \
    return false;
    FS_MX_ROWS(C)
#undef C
    default:
      return false;
  }
}
__device__ bool FS_CAT(mx_unit_c2r_, FS_MX_SUFFIX)(const Desc &d, int unit, int cnt, cx<float> *sm,
                                                    const cx<float> *spec, float *out, bool sh) {
  switch (d.M) {
#define C(m)                                                              \
  case m:                                                                 \
    if (d.rp_row.e != mx_e(m)) return false;                              \
    if (cnt == mx_row_cnt(m)) {                                           \
      mx_c2r_unit<m, mx_row_cnt(m)>(d, unit, sm, spec, out, sh);          \
      return true;                                                        \
    }                                                                     \
    if (mx_row_cnt_256(m) != mx_row_cnt(m) && cnt == mx_row_cnt_256(m)) { \
      mx_c2r_unit<m, mx_row_cnt_256(m)>(d, unit, sm, spec, out, sh);      \
      return true;                                                        \
    }                                                                     \
    return false;
    FS_MX_ROWS(C)
#undef C
    default:
      return false;
  }
}
__device__ bool FS_CAT(mx_unit_col1_, FS_MX_SUFFIX)(const Desc &d, int unit, int cnt, cx<float> *sm,
                                                     cx<float> *wu, cx<float> *wv, bool sh) {
  switch (d.ny) {
#define C(l)                                    \
  case l:                                       \
    if (d.rp_col.e != mx_e(l)) return false;    \
    mx_col1_unit<l>(d, unit, cnt, sm, wu, wv, sh); \
    return true;
    FS_MX_COLS(C)
#undef C
    default:
      return false;
  }
}

// Staged batch units: column groups by bulk copies, C2R tiles by
// asynchronous copies, the next group / tile copied in while the current one
// computes (same arithmetic as the unstaged units above).  Called, not
// inlined, from the batch kernel so that its own code stays small.
template <int L>
__device__ __noinline__ MxColRet mx_col_tma_l(const Desc &d, int c0, int c1, int cnt, cx<float> *sm,
                                              uint64_t *bars, uint32_t ph, int *s_abort) {
  const int plen = (padded_len(cnt * L) + 1) & ~1;  // even: the second buffer stays 16-byte aligned
  const bool ok = col_tma_groups<L, 0, true>(d, c0, cnt, c1, cnt, sm, sm + plen, bars, ph, s_abort);
  return MxColRet{ok ? 1 : -1, ph};
}
template <int M, int CC>
__device__ __noinline__ void mx_r2c_staged_l(const Desc &d, int tile0, int tile1, cx<float> *sm, const float *in,
                                             cx<float> *spec) {
  r2c_staged_tiles<M, CC>(d, tile0, tile1, sm, in, spec);
}
template <int M, int CC>
__device__ __noinline__ void mx_c2r_staged_l(const Desc &d, int tile0, int tile1, cx<float> *sm,
                                             const cx<float> *spec, float *out) {
  c2r_staged_tiles<M, CC, true>(d, tile0, tile1, sm, spec, out);
}

__device__ MxColRet FS_CAT(mx_col_tma_unit_, FS_MX_SUFFIX)(const Desc &d, int c0, int c1, int cnt, cx<float> *sm,
                                                            uint64_t *bars, uint32_t ph, int *s_abort) {
  switch (d.ny) {
#define C(l)                                                  \
  case l:                                                     \
    if (d.rp_col.e != mx_e(l)) return MxColRet{0, ph};        \
    return mx_col_tma_l<l>(d, c0, c1, cnt, sm, bars, ph, s_abort);
    FS_MX_COLS(C)
#undef C
    default:
      return MxColRet{0, ph};
  }
}
__device__ bool FS_CAT(mx_r2c_staged_unit_, FS_MX_SUFFIX)(const Desc &d, int tile0, int tile1, int cnt,
                                                           cx<float> *sm, const float *in, cx<float> *spec) {
  switch (d.M) {
#define C(m)                                                                 \
  case m:                                                                    \
    if (d.rp_row.e != mx_e(m)) return false;                                 \
    if (cnt == mx_row_cnt(m)) {                                              \
      mx_r2c_staged_l<m, mx_row_cnt(m)>(d, tile0, tile1, sm, in, spec);      \
      return true;                                                           \
    }                                                                        \
    if constexpr (mx_row_cnt_256(m) != mx_row_cnt(m))                        \
      if (cnt == mx_row_cnt_256(m)) {                                        \
        mx_r2c_staged_l<m, mx_row_cnt_256(m)>(d, tile0, tile1, sm, in, spec); \
        return true;                                                         \
      }                                                                      \
    return false;
    FS_MX_ROWS(C)
#undef C
    default:
      return false;
  }
}
__device__ bool FS_CAT(mx_c2r_staged_unit_, FS_MX_SUFFIX)(const Desc &d, int tile0, int tile1, int cnt,
                                                           cx<float> *sm, const cx<float> *spec, float *out) {
  switch (d.M) {
#define C(m)                                                                                          \
  case m:                                                                                             \
    if (d.rp_row.e != mx_e(m)) return false;                                                          \
    if constexpr (mx_row_cnt(m) % 2 == 0)                                                             \
      if (cnt == mx_row_cnt(m)) {                                                                     \
        mx_c2r_staged_l<m, mx_row_cnt(m)>(d, tile0, tile1, sm, spec, out);                            \
        return true;                                                                                  \
      }                                                                                               \
    if constexpr (mx_row_cnt_256(m) != mx_row_cnt(m) && mx_row_cnt_256(m) % 2 == 0)                   \
      if (cnt == mx_row_cnt_256(m)) {                                                                 \
        mx_c2r_staged_l<m, mx_row_cnt_256(m)>(d, tile0, tile1, sm, spec, out);                        \
        return true;                                                                                  \
      }                                                                                               \
    return false;
    FS_MX_ROWS(C)
#undef C
    default:
      return false;
  }
}

// ---------------------------------------------------------------- standalone kernels
template <int M>
__global__ void __launch_bounds__(512) k_r2c_mx(const Desc d) {
  extern __shared__ __align__(16) unsigned char fs_smem[];
  int unit = blockIdx.x;
  const float *in = reinterpret_cast<const float *>(d.in_u);
  cx<float> *spec = reinterpret_cast<cx<float> *>(d.work_u);
  if (unit >= d.n_row_units) {
    unit -= d.n_row_units;
    in = reinterpret_cast<const float *>(d.in_v);
    spec = reinterpret_cast<cx<float> *>(d.work_v);
  }
  unit_row_r2c_t<float, mx_e(M), M, mx_row_cnt(M)>(d, unit, mx_row_cnt(M), reinterpret_cast<cx<float> *>(fs_smem),
                                                   in, spec);
}
template <int M>
__global__ void __launch_bounds__(512) k_c2r_mx(const Desc d) {
  extern __shared__ __align__(16) unsigned char fs_smem[];
  int unit = blockIdx.x;
  const cx<float> *spec = reinterpret_cast<const cx<float> *>(d.work_u);
  float *out = reinterpret_cast<float *>(d.out_u);
  if (unit >= d.n_row_units) {
    unit -= d.n_row_units;
    spec = reinterpret_cast<const cx<float> *>(d.work_v);
    out = reinterpret_cast<float *>(d.out_v);
  }
  unit_row_c2r_t<float, mx_e(M), M, mx_row_cnt(M)>(d, unit, mx_row_cnt(M), reinterpret_cast<cx<float> *>(fs_smem),
                                                   spec, out, false);
}
template <int L>
__global__ void __launch_bounds__(512) k_col_mx(const Desc d) {
  extern __shared__ __align__(16) unsigned char fs_smem[];
  unit_col_t<float, mx_e(L), false, L, 0>(d, blockIdx.x, d.cols_per_unit, reinterpret_cast<cx<float> *>(fs_smem),
                                          reinterpret_cast<cx<float> *>(d.work_u),
                                          reinterpret_cast<cx<float> *>(d.work_v), false);
}

PassKernel FS_CAT(mx_r2c_f32_, FS_MX_SUFFIX)(int M) {
  switch (M) {
#define C(m) \
  case m:    \
    return k_r2c_mx<m>;
    FS_MX_ROWS(C)
#undef C
    default:
      return nullptr;
  }
}
PassKernel FS_CAT(mx_c2r_f32_, FS_MX_SUFFIX)(int M) {
  switch (M) {
#define C(m) \
  case m:    \
    return k_c2r_mx<m>;
    FS_MX_ROWS(C)
#undef C
    default:
      return nullptr;
  }
}
PassKernel FS_CAT(mx_col1_f32_, FS_MX_SUFFIX)(int L) {
  switch (L) {
#define C(l) \
  case l:    \
    return k_col_mx<l>;
    FS_MX_COLS(C)
#undef C
    default:
      return nullptr;
  }
}

}  // namespace fs
