// fs_host.h -- host-side plan/state objects shared by the C-ABI sources.
#pragma once
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <string>

#include "../../include/fsolve.h"
#include "fs_desc.h"

namespace fs {

extern std::atomic<unsigned long long> g_launches;

fs_status set_error(fs_status st, const std::string &msg);
fs_status cuda_error(cudaError_t e, const char *what);

// Radix factorisation and register-tile choice for a length-L transform.
int choose_e(int L, bool f64);
int radix_plan(int L, int e, int *out, int cap);
bool size_supported(int n);

struct TileConfig {
  int rows_per_unit;  // row passes
  int rows_per_unit_c;  // complex (C2C) row passes, length nx
  int cols_per_unit;  // column pass
  int small_rows, small_cols;
  size_t small_smem1, small_smem2;  // small-path smem with one / two resident spectra (0: too big)
};

}  // namespace fs

struct fs_plan_s {
  int nx, ny, M, dtype;
  double lx, ly;
  int device;
  fs::RadixPlan rp_row, rp_col;
  fs::RadixPlan rp_rowc;  // length nx: complex (C2C) row transforms
  fs::TileConfig tc;
  bool standalone_small;  // single-kernel path for one-off calls
  size_t csize;           // bytes per complex element
  // device tables (one allocation)
  void *tables;
  void *tw_x, *tw_y, *wx2, *wy2;
  double *wx2d, *wy2d;
  // device workspace
  void *work_u, *work_v, *fac;
  void *work_c, *work_cv;  // full spectra nx*ny for complex fields (allocated on first use)
  float *pfac;             // FP32 plans: Poisson factors [M+1][ny] (built on first use)
  size_t spec_bytes;  // (M+1)*ny complex
};

struct fs_state_s {
  fs_plan plan;
  void *su, *sv;
  void *ss;         // kept constant-source spectrum (nullptr: no source)
  bool has_v;
  bool has_s;       // the source is applied by advances
};

namespace fs {
// A tuned configuration of a grid's passes (0 = the default): register tile
// (hence radix split) of the row and column transforms, row-tile height and
// column-group width of the standalone pass kernels.
struct TuneCfg {
  int e_row, e_col, rows, cols;
};
// The tuning cache (fs_tune.cu): configurations by (GPU name, nx, ny, dtype,
// mode); mode 0 = standalone passes (plan creation), 1 = inside a batch (only
// the register tiles apply there).
bool tune_lookup(int device, int nx, int ny, int dtype, int mode, TuneCfg *out);
// Plan creation with a forced configuration (nullptr: the cache, else defaults).
fs_status plan_create_cfg(int nx, int ny, double lx, double ly, int dtype, const TuneCfg *force, fs_plan *out);
// Radix plan of a length-L transform with register tile e (false: not available).
bool make_rp_e(int L, int e, bool f64, RadixPlan *rp);
// Radix plans and tile shapes for an nx x ny grid (false: unsupported size).
bool plan_geometry(int nx, int ny, bool f64, RadixPlan *rr, RadixPlan *rc, TileConfig *tc);
// Descriptor with the plan's geometry, tables and tile shapes filled in.
Desc base_desc(const fs_plan_s *p);
// Forward 2D DFT of u0 (and v0 when not NULL) into the half spectra su (sv),
// stream-ordered; the plan's own path (single CTA or three passes).
fs_status forward_into(const fs_plan_s *p, const void *u0, const void *v0, void *su, void *sv,
                       fs_stream stream, const char *what);
size_t fac_bytes(const fs_plan_s *p);
// FP32 plans: the wave phase c |t| |omega|_max stays within 2^20 (the range
// in which the two-float phase reduction keeps its accuracy); FP64: always.
bool wave_phase_ok(const fs_plan_s *p, double c, double t);
}  // namespace fs
