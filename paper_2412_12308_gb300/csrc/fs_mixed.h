// fs_mixed.h -- FP32 pass kernels and batch units specialised at compile time
// for the lengths 3 x 2^k and 5 x 2^k (the mixed-radix counterpart of
// fs_pow2.h).  The register tile is the plan's default for the family (24 for
// 3 x 2^k, 20 for 5 x 2^k), the radix plan power-of-two stages (largest
// dividing the tile first) followed by the odd stage, as in the runtime engine.
#pragma once
#include "fs_desc.h"
#include "fs_pow2.h"

namespace fs {

template <typename T>
struct cx;

constexpr int mx_odd(int x) { return x <= 0 ? 0 : (x % 2 == 0 ? mx_odd(x / 2) : x); }
// register tile of the family (0: not a compiled family)
constexpr int mx_e(int L) { return mx_odd(L) == 3 ? 24 : (mx_odd(L) == 5 ? 20 : 0); }
// compiled lengths: columns (ny) and rows (M = nx/2)
constexpr bool mx_col_ok(int L) {
  return L == 160 || L == 192 || L == 320 || L == 384 || L == 640 || L == 768 || L == 1280 || L == 1536 ||
         L == 2560 || L == 3072 || L == 5120 || L == 6144;
}
constexpr bool mx_row_ok(int M) { return M >= 160 && M <= 3072 && mx_col_ok(M); }
constexpr int mx_padded(int n) { return n + (n >> 4) + 1; }
// rows per tile of the plans' default tile shapes (at most 16 rows, 512
// threads and 96 KB of exchange scratch), and of a 256-thread batch CTA
constexpr int mx_row_cnt(int M) {
  int cr = 16;
  while (cr > 1 && (cr * (M / mx_e(M)) > 512 || 8 * mx_padded(cr * M) > 96 * 1024)) cr >>= 1;
  return cr;
}
constexpr int mx_row_cnt_256(int M) {
  return mx_row_cnt(M) * (M / mx_e(M)) <= 256 ? mx_row_cnt(M) : 256 / (M / mx_e(M));
}

// Device units for the batch and single-CTA paths; false when the length,
// tile or tile height is not compiled (the caller uses the runtime engine).
// One object per family (fs_mixed_f32.cu with FS_MX_ODD = 3 or 5).
// Result of a staged mixed-radix column unit: r as col_tma_unit (1 done, 0
// not compiled, -1 a copy timed out) and the CTA's barrier parities after it
// (returned, so that the caller's parity word stays in a register).
struct MxColRet {
  int r;
  uint32_t ph;
};

#define FS_MX_DECL(F)                                                                                         \
  __device__ bool mx_unit_r2c_##F(const Desc &d, int unit, int cnt, cx<float> *sm, const float *in,           \
                                  cx<float> *spec);                                                           \
  __device__ bool mx_unit_c2r_##F(const Desc &d, int unit, int cnt, cx<float> *sm, const cx<float> *spec,     \
                                  float *out, bool sh);                                                       \
  __device__ bool mx_unit_col1_##F(const Desc &d, int unit, int cnt, cx<float> *sm, cx<float> *wu,            \
                                   cx<float> *wv, bool sh);                                                   \
  __device__ MxColRet mx_col_tma_unit_##F(const Desc &d, int c0, int c1, int cnt, cx<float> *sm,              \
                                          uint64_t *bars, uint32_t ph, int *s_abort);                         \
  __device__ bool mx_r2c_staged_unit_##F(const Desc &d, int tile0, int tile1, int cnt, cx<float> *sm,         \
                                         const float *in, cx<float> *spec);                                   \
  __device__ bool mx_c2r_staged_unit_##F(const Desc &d, int tile0, int tile1, int cnt, cx<float> *sm,         \
                                         const cx<float> *spec, float *out);                                  \
  PassKernel mx_r2c_f32_##F(int M);                                                                          \
  PassKernel mx_c2r_f32_##F(int M);                                                                          \
  PassKernel mx_col1_f32_##F(int L);
FS_MX_DECL(3)
FS_MX_DECL(5)
#undef FS_MX_DECL

__device__ __forceinline__ bool mx_unit_r2c(const Desc &d, int unit, int cnt, cx<float> *sm, const float *in,
                                            cx<float> *spec) {
  const int o = mx_odd(d.M);
  return o == 3 ? mx_unit_r2c_3(d, unit, cnt, sm, in, spec) : (o == 5 && mx_unit_r2c_5(d, unit, cnt, sm, in, spec));
}
__device__ __forceinline__ bool mx_unit_c2r(const Desc &d, int unit, int cnt, cx<float> *sm, const cx<float> *spec,
                                            float *out, bool sh) {
  const int o = mx_odd(d.M);
  return o == 3 ? mx_unit_c2r_3(d, unit, cnt, sm, spec, out, sh)
                : (o == 5 && mx_unit_c2r_5(d, unit, cnt, sm, spec, out, sh));
}
__device__ __forceinline__ bool mx_unit_col1(const Desc &d, int unit, int cnt, cx<float> *sm, cx<float> *wu,
                                             cx<float> *wv, bool sh) {
  const int o = mx_odd(d.ny);
  return o == 3 ? mx_unit_col1_3(d, unit, cnt, sm, wu, wv, sh)
                : (o == 5 && mx_unit_col1_5(d, unit, cnt, sm, wu, wv, sh));
}

// Staged batch units (column groups by bulk copies, R2C and C2R tiles by
// asynchronous copies): 0 / false when the length, tile or tile height is not compiled;
// the column unit returns -1 when a copy timed out (as col_tma_groups).
__device__ __forceinline__ int mx_col_tma_unit(const Desc &d, int c0, int c1, int cnt, cx<float> *sm,
                                               uint64_t *bars, uint32_t &ph, int *s_abort) {
  const int o = mx_odd(d.ny);
  if (o != 3 && o != 5) return 0;
  const MxColRet r = o == 3 ? mx_col_tma_unit_3(d, c0, c1, cnt, sm, bars, ph, s_abort)
                            : mx_col_tma_unit_5(d, c0, c1, cnt, sm, bars, ph, s_abort);
  ph = r.ph;
  return r.r;
}
__device__ __forceinline__ bool mx_r2c_staged_unit(const Desc &d, int tile0, int tile1, int cnt, cx<float> *sm,
                                                   const float *in, cx<float> *spec) {
  const int o = mx_odd(d.M);
  return o == 3 ? mx_r2c_staged_unit_3(d, tile0, tile1, cnt, sm, in, spec)
                : (o == 5 && mx_r2c_staged_unit_5(d, tile0, tile1, cnt, sm, in, spec));
}
__device__ __forceinline__ bool mx_c2r_staged_unit(const Desc &d, int tile0, int tile1, int cnt, cx<float> *sm,
                                                   const cx<float> *spec, float *out) {
  const int o = mx_odd(d.M);
  return o == 3 ? mx_c2r_staged_unit_3(d, tile0, tile1, cnt, sm, spec, out)
                : (o == 5 && mx_c2r_staged_unit_5(d, tile0, tile1, cnt, sm, spec, out));
}

// Standalone pass kernels (nullptr when not compiled): rows with the plans'
// default tile height, single-field columns with any group width.
inline PassKernel mx_r2c_f32(int M) { return mx_odd(M) == 3 ? mx_r2c_f32_3(M) : (mx_odd(M) == 5 ? mx_r2c_f32_5(M) : nullptr); }
inline PassKernel mx_c2r_f32(int M) { return mx_odd(M) == 3 ? mx_c2r_f32_3(M) : (mx_odd(M) == 5 ? mx_c2r_f32_5(M) : nullptr); }
inline PassKernel mx_col1_f32(int L) {
  return mx_odd(L) == 3 ? mx_col1_f32_3(L) : (mx_odd(L) == 5 ? mx_col1_f32_5(L) : nullptr);
}

}  // namespace fs
