// fs_pow2.h -- pass kernels specialised at compile time for power-of-two
// lengths (FP32, 16-element register tiles).  Each kernel inlines one unit
// with the transform length and the rows/columns per CTA fixed, so the FFT
// engine's strides and stage structure are constants.
#pragma once
#include "fs_desc.h"

namespace fs {

typedef void (*PassKernel)(const Desc);

// Column pass: 256 threads per CTA (512 for length 8192).
constexpr int p2_col_cnt(int L) { return (L / 16) >= 256 ? 1 : 256 / (L / 16); }
constexpr bool p2_col_ok(int L) { return L >= 128 && L <= 8192 && (L & (L - 1)) == 0; }
// Row passes (length M = nx/2): up to 16 rows and 512 threads per CTA.
constexpr int p2_row_cnt(int M) {
  return (M / 16) >= 256 ? 2 : ((M / 16) * 16 <= 512 ? 16 : 512 / (M / 16));
}
// rows per tile of a 256-thread batch CTA (p2_row_cnt(M) where it fits)
constexpr int p2_row_cnt_256(int M) { return (M / 16) * p2_row_cnt(M) <= 256 ? p2_row_cnt(M) : 256 / (M / 16); }
// and of a 128-thread batch CTA (0 when a row needs more threads)
constexpr int p2_row_cnt_128(int M) {
  return (M / 16) > 128 ? 0 : ((M / 16) * p2_row_cnt_256(M) <= 128 ? p2_row_cnt_256(M) : 128 / (M / 16));
}
constexpr bool p2_row_ok(int M) { return M >= 128 && M <= 4096 && (M & (M - 1)) == 0; }
// Complex (C2C) rows of length N: up to 16 rows and 512 threads per CTA.
constexpr int p2_c2c_cnt(int N) { return (N / 16) * 16 <= 512 ? 16 : 512 / (N / 16); }
constexpr bool p2_c2c_ok(int N) { return N >= 128 && N <= 8192 && (N & (N - 1)) == 0; }

// Device-side unit functions for the persistent batch and single-CTA paths
// (row tiles must use p2_row_cnt(M) rows; columns take any count).  Return
// false when the length is not specialised.
template <typename T>
struct cx;
__device__ bool p2_unit_r2c(const Desc &d, int unit, int cnt, cx<float> *sm, const float *in, cx<float> *spec);
__device__ bool p2_unit_c2r(const Desc &d, int unit, int cnt, cx<float> *sm, const cx<float> *spec, float *out,
                            bool sh);
__device__ bool p2_unit_col1(const Desc &d, int unit, int cnt, cx<float> *sm, cx<float> *wu, cx<float> *wv,
                             bool sh);
// Staged R2C row tiles tile0 .. tile1-1 of a batch unit (FP32, rows of a
// compiled length and tile height; false otherwise): fs_row_async.cuh.
__device__ bool p2_r2c_staged_unit(const Desc &d, int tile0, int tile1, int cnt, cx<float> *sm, const float *in,
                                   cx<float> *spec);
// columns of an advance with a constant source, one or two fields
__device__ bool p2_unit_cols(const Desc &d, int unit, int cnt, cx<float> *sm, cx<float> *wu, cx<float> *wv,
                             bool sh);

// Shared memory of a batch column unit staged by bulk copies (F_COL_TMA,
// fs_col_tma.cuh): two padded buffers of cnt columns of length L.
size_t p2_col1_tma_unit_smem(int L, int cnt);

// Kernel lookup (nullptr when not specialised).
PassKernel p2_r2c_f32(int M);
PassKernel p2_c2r_f32(int M);
PassKernel p2_col1_f32(int L);
PassKernel p2_col2_f32(int L);
PassKernel p2_cols_f32(int L, bool two);  // advances with a constant source
PassKernel p2_c2c_f32(int N, bool inverse);  // complex rows, forward / inverse
// TMA-staged persistent column kernel (single field) and its shared memory.
PassKernel p2_col_tma_f32(int L);
// Split-BF16 tensor-core first stage (measured variant, FS_COLUMN_VARIANT=bf16x3).
bool tc_variant_requested();
PassKernel p2_col_tc_f32(int L, size_t *smem);
size_t p2_col_tma_smem(int L);

}  // namespace fs
