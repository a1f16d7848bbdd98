// fs_desc.h -- problem descriptor shared by host code and kernels.
//
// One Desc describes one solve or one advance on one grid: which operator,
// the radix plans of the two 1D transform lengths (nx/2 for the packed real
// row transform, ny for the column transform), the tile shapes, and every
// device pointer the units read or write.  The same descriptor drives the
// standalone pass kernels, the single-kernel small-grid path and the
// persistent batch kernel, so a problem computes bit-identically on all of
// them for a given tile shape.
#pragma once
#include <stdint.h>

namespace fs {

enum Op : int {
  OP_POISSON = 0,     // Eq. SolutionPoisson
  OP_DIFFUSION = 1,   // Eq. solCalorFourier, from a field
  OP_WAVE = 2,        // Eq. OmegaZero / OmegaNonZero, from fields
  OP_DIFF_ADV = 3,    // diffusion from a kept spectrum
  OP_WAVE_ADV = 4,    // wave from kept spectra
  OP_FORWARD = 5      // forward 2D DFT into kept spectra (state creation)
};

enum Flags : int {
  F_HAS_V0 = 1,   // wave: an initial velocity field / spectrum is present
  F_WANT_V = 2,   // wave advance: also produce v = u_t
  F_SOURCE = 4,   // advance: a kept constant-source spectrum st_s is added
  F_COL_TMA = 8,     // batch: column units stage each column group by a bulk copy
  F_ROW_STAGED = 16,  // batch: C2R row units stage each tile by asynchronous copies
  F_R2C_STAGED = 32   // batch: R2C row units stage each tile by asynchronous copies
};

// Unit kinds of the persistent batch kernel, in dependency order.
enum Kind : int { K_FACTOR = 0, K_ROW = 1, K_SMALL = 2, K_COL = 3, K_C2R = 4 };

struct RadixPlan {
  int32_t e;         // elements held per thread (the register tile)
  int32_t n;         // number of stages
  int32_t r[8];      // radix of each stage, product = transform length
};

// Column-independent operator constants of the FP32 path, split on the host
// from the double fields below into (hi, lo) float pairs, so the kernels do
// no FP64 arithmetic (GB300 runs FP64 at a small fraction of the FP32 rate).
struct OpConstF {
  float ct_hi, ct_lo;  // c * t
  float sc_hi, sc_lo;  // scale
  float dd_hi, dd_lo;  // D
  float cy_hi, cy_lo;  // wy_unit2
  float c, t, scale;
  int ready;           // 1 once filled (fill_op_consts)
};

struct Desc {
  int32_t op, flags;
  int32_t nx, ny, M;          // M = nx/2: length of the packed real row transform
  int32_t rows_per_unit;      // row tile height of the row passes
  int32_t cols_per_unit;      // columns per column-pass unit
  int32_t n_row_units;        // per field
  int32_t n_col_units;
  int32_t n_fac_units;
  int32_t row_g, col_g;       // batch: row tiles / column groups per work unit (>= 1)
  int32_t small;              // 1: whole problem in one CTA (shared-memory resident)
  int32_t small_rows;         // row group of the small path
  int32_t small_cols;         // column group of the small path
  RadixPlan rp_row;           // length M
  RadixPlan rp_col;           // length ny
  const void *in_u, *in_v;    // real fields [ny][nx]
  void *out_u, *out_v;        // real fields [ny][nx]
  void *work_u, *work_v;      // half-spectra [M+1][ny] (x-frequency major)
  const void *st_u, *st_v;    // kept spectra (advance ops)
  const void *st_s;           // kept source spectrum (advance ops with F_SOURCE)
  void *st_out_u, *st_out_v;  // where OP_FORWARD keeps the spectra
  const void *tw_x, *tw_y;    // omega_nx^m (m < nx), omega_ny^m (m < ny)
  const void *wx2, *wy2;      // |omega_x|^2 (a <= M), |omega_y|^2 (b < ny); two-float or double
  const double *wx2d, *wy2d;  // the same in float64 (factor tables)
  void *fac;                  // diffusion per-axis factors: x part [M+1], y part [ny]
  const float *pfac;          // FP32 Poisson: -1/(nx ny |omega|^2) per element [M+1][ny], FP64-evaluated (or null)
  double p_dt;                // D * t
  double p_d;                 // diffusivity D (source gain of the diffusion advance)
  double p_c;                 // wave speed c
  double p_t;                 // time t
  double scale;               // 1 / (nx * ny)
  double wy_unit2;            // (2 pi / Ly)^2: |omega_y(b)|^2 = wy_unit2 * b'^2 (FP32 operators)
  OpConstF fc;                // the above as float pairs (FP32 kernels)
};

}  // namespace fs
