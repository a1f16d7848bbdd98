// fs_api.cu -- plans, kept states and the one-shot / advance entry points of
// the C ABI (include/fsolve.h).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "fs_host.h"
#include "fs_kernels.cuh"
#include "fs_tma.cuh"

// The kernels are instantiated in fs_kernels_f32.cu / fs_kernels_f64.cu.
extern template struct fs::Launch<float>;
extern template struct fs::Launch<double>;

namespace fs {

std::atomic<unsigned long long> g_launches{0};

bool tma_enabled() {
  static const bool on = [] {
    const char *v = getenv("FS_NO_TMA");
    return !(v && *v && *v != '0');
  }();
  return on;
}

static thread_local std::string t_last_error;

fs_status set_error(fs_status st, const std::string &msg) {
  t_last_error = msg;
  return st;
}

fs_status cuda_error(cudaError_t e, const char *what) {
  char buf[256];
  snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
  if (e == cudaErrorMemoryAllocation) return set_error(FS_ERR_NOMEM, buf);
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return set_error(FS_ERR_NODEV, buf);
  return set_error(FS_ERR_CUDA, buf);
}

bool size_supported(int n) {
  if (n < 8 || n > 8192 || (n & 1)) return false;
  int m = n;
  while ((m & 1) == 0) m >>= 1;
  return m == 1 || m == 3 || m == 5;
}

// Elements per thread: the first register tile of the size's family (in
// preference order) that divides L with at most 512 threads per transform.
// FP64 prefers half-size tiles (twice the registers per element).
int choose_e(int L, bool f64) {
  int m = L;
  while ((m & 1) == 0) m >>= 1;
  static const int pow2[] = {16, 8, 4}, three[] = {24, 12, 6}, five[] = {20, 10, 5};
  static const int pow2d[] = {8, 4, 16}, threed[] = {12, 6, 24}, fived[] = {10, 5, 20};
  const int *cand = m == 1 ? (f64 ? pow2d : pow2)
                           : (m == 3 ? (f64 ? threed : three) : (m == 5 ? (f64 ? fived : five) : nullptr));
  if (!cand) return 0;
  for (int i = 0; i < 3; ++i) {
    const int e = cand[i];
    if (L >= e && L % e == 0 && L / e <= kMaxThreads) return e;
  }
  return 0;
}

// Radices dividing e, power-of-two stages largest first, then the odd stage.
int radix_plan(int L, int e, int *out, int cap) {
  if (L <= 0 || e <= 0) return 0;
  int odd = L, p2 = 1;
  while ((odd & 1) == 0) {
    odd >>= 1;
    p2 <<= 1;
  }
  if (odd != 1 && odd != 3 && odd != 5) return 0;
  if (odd > 1 && e % odd) return 0;
  int n = 0;
  static const int rs[] = {16, 8, 4, 2};
  while (p2 > 1) {
    int pick = 0;
    for (int r : rs)
      if (e % r == 0 && p2 % r == 0) {
        pick = r;
        break;
      }
    if (!pick || n >= cap) return 0;
    out[n++] = pick;
    p2 /= pick;
  }
  if (odd > 1) {
    if (n >= cap) return 0;
    out[n++] = odd;
  }
  return n;
}

static bool make_rp(int L, bool f64, RadixPlan *rp) {
  memset(rp, 0, sizeof *rp);
  rp->e = choose_e(L, f64);
  if (!rp->e) return false;
  rp->n = radix_plan(L, rp->e, rp->r, 8);
  return rp->n > 0;
}

static int env_int(const char *name, int dflt) {
  const char *v = getenv(name);
  return v && *v ? atoi(v) : dflt;
}

// Tile shapes: row tiles of up to 16 rows (longer contiguous runs in the
// x-frequency-major spectrum), column groups of up to 32 columns, at most 512
// threads and ~96 KB of exchange scratch per CTA.
static TileConfig make_tiles(int nx, int ny, const RadixPlan &rr, const RadixPlan &rc, size_t cs) {
  TileConfig t{};
  const int M = nx / 2;
  const int tr = M / rr.e, tcl = ny / rc.e;
  const size_t lim = 96 * 1024;
  int cr = 16;
  while (cr > 1 && (cr * tr > kMaxThreads || cs * padded_len(cr * M) > lim)) cr >>= 1;
  if (cr > ny) cr = ny;
  t.rows_per_unit = cr;
  int cc = 32;
  while (cc > 1 && (cc * tcl > kMaxThreads || cs * padded_len(cc * ny) > lim)) cc >>= 1;
  t.cols_per_unit = cc;
  // FP32 power-of-two lengths: the tile shapes of the compile-time kernels
  if (cs == 8 && rr.e == 16 && p2_row_ok(M)) t.rows_per_unit = p2_row_cnt(M) < ny ? p2_row_cnt(M) : ny;
  if (cs == 8 && rc.e == 16 && p2_col_ok(ny)) t.cols_per_unit = p2_col_cnt(ny);
  // small path: whole half spectrum resident in shared memory
  int sr = ny < kMaxThreads / tr ? ny : kMaxThreads / tr;
  int sc = (M + 1) < kMaxThreads / tcl ? (M + 1) : kMaxThreads / tcl;
  if (sr < 1) sr = 1;
  if (sc < 1) sc = 1;
  const size_t spec = (size_t)(M + 1) * ny;
  const size_t smem_lim = (size_t)env_int("FS_SMALL_SMEM_MAX", 200 * 1024);
  auto fit = [&](int nspec, int &r, int &c) -> size_t {
    for (;;) {
      const size_t x = (size_t)(padded_len(r * M) > padded_len(c * ny) ? padded_len(r * M)
                                                                       : padded_len(c * ny));
      const size_t b = cs * (spec * nspec + x);
      if (b <= smem_lim) return b;
      if (r > 1 && r * M >= c * ny) r = (r + 1) / 2;
      else if (c > 1) c = (c + 1) / 2;
      else return 0;
      if (cs * spec * nspec > smem_lim) return 0;
    }
  };
  int r1 = sr, c1 = sc;
  t.small_smem1 = fit(1, r1, c1);
  int r2 = r1, c2 = c1;
  t.small_smem2 = t.small_smem1 ? fit(2, r2, c2) : 0;
  // one row/column grouping for both variants (results must not depend on it)
  t.small_rows = t.small_smem2 ? r2 : r1;
  t.small_cols = t.small_smem2 ? c2 : c1;
  if (t.small_smem2) t.small_smem1 = cs * (spec + (size_t)(padded_len(r2 * M) > padded_len(c2 * ny)
                                                              ? padded_len(r2 * M)
                                                              : padded_len(c2 * ny)));
  return t;
}

bool plan_geometry(int nx, int ny, bool f64, RadixPlan *rr, RadixPlan *rc, TileConfig *tc) {
  if (!size_supported(nx) || !size_supported(ny)) return false;
  if (!make_rp(nx / 2, f64, rr) || !make_rp(ny, f64, rc)) return false;
  *tc = make_tiles(nx, ny, *rr, *rc, f64 ? 2 * sizeof(double) : 2 * sizeof(float));
  return true;
}

Desc base_desc(const fs_plan_s *p) {
  Desc d;
  memset(&d, 0, sizeof d);
  d.nx = p->nx;
  d.ny = p->ny;
  d.M = p->M;
  d.rows_per_unit = p->tc.rows_per_unit;
  d.cols_per_unit = p->tc.cols_per_unit;
  d.n_row_units = (p->ny + d.rows_per_unit - 1) / d.rows_per_unit;
  d.n_col_units = (p->M + 1 + d.cols_per_unit - 1) / d.cols_per_unit;
  d.n_fac_units = (p->M + 1 + p->ny + kFactorPerUnit - 1) / kFactorPerUnit;
  d.row_g = d.col_g = 1;
  d.small_rows = p->tc.small_rows;
  d.small_cols = p->tc.small_cols;
  d.rp_row = p->rp_row;
  d.rp_col = p->rp_col;
  d.tw_x = p->tw_x;
  d.tw_y = p->tw_y;
  d.wx2 = p->wx2;
  d.wy2 = p->wy2;
  d.wx2d = p->wx2d;
  d.wy2d = p->wy2d;
  d.fac = p->fac;
  d.work_u = p->work_u;
  d.work_v = p->work_v;
  d.scale = 1.0 / ((double)p->nx * (double)p->ny);
  d.wy_unit2 = (2.0 * M_PI / p->ly) * (2.0 * M_PI / p->ly);
  return d;
}

// x part for all nx frequencies (complex fields use a <= nx-1; real fields a <= nx/2)
size_t fac_bytes(const fs_plan_s *p) {
  return (size_t)(p->nx + p->ny) * (p->dtype == FS_F64 ? sizeof(double) : sizeof(float2));
}

// Signed-index angular wavenumber squared: (2 pi a'/L)^2, a' = a (a <= n/2) else a - n.
static double omega2_axis(int a, int n, double len) {
  const int ap = (2 * a <= n) ? a : a - n;
  const double w = 2.0 * M_PI * (double)ap / len;
  return w * w;
}

// The FP32 wave operators reduce the phase c |omega| t modulo 2 pi in
// two-float (~44 bits), so the phase keeps ~2^-44 |theta| absolute accuracy;
// beyond |theta| = 2^20 that would grow past the hardware sine/cosine's own
// error (2^-21.4), so FP32 plans reject larger phases.  FP64 plans evaluate
// the phase in double.
bool wave_phase_ok(const fs_plan_s *p, double c, double t) {
  if (p->dtype == FS_F64) return true;
  const double wx = M_PI * p->nx / p->lx, wy = M_PI * p->ny / p->ly;  // largest |omega_x|, |omega_y|
  return std::fabs(c * t) * std::sqrt(wx * wx + wy * wy) <= 1048576.0;
}

}  // namespace fs

using namespace fs;

static cudaError_t alloc_dev(void **p, size_t bytes) { return cudaMalloc(p, bytes); }

bool fs::make_rp_e(int L, int e, bool f64, RadixPlan *rp) {
  static const int es_f[] = {4, 5, 6, 8, 10, 12, 16, 20, 24}, es_d[] = {4, 5, 6, 8, 10, 12, 16};
  bool ok = false;
  for (int v : (f64 ? std::vector<int>(es_d, es_d + 7) : std::vector<int>(es_f, es_f + 9))) ok |= v == e;
  if (!ok || L < e || L % e || L / e > kMaxThreads) return false;
  memset(rp, 0, sizeof *rp);
  rp->e = e;
  rp->n = radix_plan(L, e, rp->r, 8);
  return rp->n > 0;
}

// Apply a tuned / forced configuration to a plan's geometry; false if it does
// not fit (the caller keeps the defaults or reports the error).
static bool apply_cfg(fs_plan_s *t, const TuneCfg &c) {
  const bool f64 = t->dtype == FS_F64;
  RadixPlan rr = t->rp_row, rc = t->rp_col;
  if (c.e_row && !make_rp_e(t->M, c.e_row, f64, &rr)) return false;
  if (c.e_col && !make_rp_e(t->ny, c.e_col, f64, &rc)) return false;
  TileConfig tc = make_tiles(t->nx, t->ny, rr, rc, t->csize);
  tc.rows_per_unit_c = t->tc.rows_per_unit_c;
  const int tr = t->M / rr.e, tcl = t->ny / rc.e;
  const size_t lim = 200 * 1024;
  if (c.rows) {
    const bool p2 = t->csize == 8 && rr.e == 16 && p2_row_ok(t->M) && c.rows == p2_row_cnt(t->M);
    if (c.rows > t->ny || c.rows * tr > (p2 ? 1024 : kMaxThreads) || t->csize * padded_len(c.rows * t->M) > lim)
      return false;
    tc.rows_per_unit = c.rows;
  }
  if (c.cols) {
    if (c.cols * tcl > kMaxThreads || t->csize * padded_len(c.cols * t->ny) > lim) return false;
    tc.cols_per_unit = c.cols;
  }
  t->rp_row = rr;
  t->rp_col = rc;
  t->tc = tc;
  return true;
}

// Poisson factors of an FP32 plan, -1/(nx ny |omega|^2) for every element
// (a, b) of the half spectrum, evaluated in FP64 from the FP64 axis tables
// and rounded once to float (Eq. SolutionPoisson with the normalisation of
// the inverse transform); the zero mode gets 0.
__global__ void k_poisson_table(float *out, const double *wx2d, const double *wy2d, int ncol, int ny,
                                double scale) {
  const size_t n = (size_t)ncol * ny;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(i / ny), b = (int)(i - (size_t)a * ny);
    const double w2 = wx2d[a] + wy2d[b];
    out[i] = w2 > 0.0 ? (float)(-scale / w2) : 0.0f;
  }
}

// The table is a measured variant, off by default (FS_POISSON_TABLE=1 turns
// it on): at 4096^2 its extra read of half a spectrum of floats made the
// column pass slower (88.0 us) than forming the factor per element in
// two-float (77.9 us), whose ~44-bit value rounds to the same float except in
// rare double-rounding cases.
static bool poisson_table_enabled() {
  static const bool on = [] {
    const char *v = getenv("FS_POISSON_TABLE");
    return v && *v && *v != '0';
  }();
  return on;
}

// Build the plan's Poisson table on first use (stream-ordered).
static fs_status ensure_pfac(fs_plan p, cudaStream_t s) {
  if (p->pfac) return FS_OK;
  const size_t n = (size_t)(p->M + 1) * p->ny;
  cudaError_t e = alloc_dev(reinterpret_cast<void **>(&p->pfac), n * sizeof(float));
  if (e != cudaSuccess) {
    p->pfac = nullptr;
    return cuda_error(e, "Poisson factor table allocation");
  }
  const int blocks = (int)std::min<size_t>((n + 255) / 256, 4096);
  k_poisson_table<<<blocks, 256, 0, s>>>(p->pfac, p->wx2d, p->wy2d, p->M + 1, p->ny,
                                           1.0 / ((double)p->nx * (double)p->ny));
  g_launches.fetch_add(1, std::memory_order_relaxed);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_error(e, "Poisson factor table");
  return FS_OK;
}

static fs_status ensure_work_v(fs_plan p) {
  if (p->work_v) return FS_OK;
  cudaError_t e = alloc_dev(&p->work_v, p->spec_bytes);
  if (e != cudaSuccess) return cuda_error(e, "workspace allocation");
  return FS_OK;
}

extern "C" {

const char *fs_last_error(void) { return t_last_error.c_str(); }

int fs_size_supported(int n) { return size_supported(n) ? 1 : 0; }

int fs_radix_plan(int L, int e, int *out, int cap) { return radix_plan(L, e, out, cap); }

uint64_t fs_kernel_launches(void) { return g_launches.load(); }

fs_status fs_device_status(int *code) {
  int v = 0;
  cudaError_t e = cudaMemcpyFromSymbol(&v, g_fs_dev_error, sizeof(int));
  if (e == cudaSuccess && v) {
    const int zero = 0;
    e = cudaMemcpyToSymbol(g_fs_dev_error, &zero, sizeof(int));
  }
  if (e != cudaSuccess) return cuda_error(e, "fs_device_status");
  if (code) *code = v;
  return v ? set_error(FS_ERR_TIMEOUT, "a bounded device wait expired") : FS_OK;
}

fs_status fs_plan_create(int nx, int ny, double lx, double ly, int dtype, fs_plan *out) {
  return plan_create_cfg(nx, ny, lx, ly, dtype, nullptr, out);
}

}  // extern "C"

fs_status fs::plan_create_cfg(int nx, int ny, double lx, double ly, int dtype, const TuneCfg *force,
                              fs_plan *out) {
  if (!out) return set_error(FS_ERR_ARG, "fs_plan_create: out is NULL");
  *out = nullptr;
  if (!(lx > 0.0) || !(ly > 0.0) || !std::isfinite(lx) || !std::isfinite(ly))
    return set_error(FS_ERR_ARG, "fs_plan_create: Lx and Ly must be finite and > 0");
  if (dtype != FS_F32 && dtype != FS_F64) return set_error(FS_ERR_ARG, "fs_plan_create: bad dtype");
  if (!size_supported(nx) || !size_supported(ny)) {
    char buf[160];
    snprintf(buf, sizeof buf,
             "fs_plan_create: unsupported size %d x %d (need even n = 2^a*{1,3,5}, 8 <= n <= 8192)",
             nx, ny);
    return set_error(FS_ERR_SIZE, buf);
  }
  fs_plan_s tmp;
  memset(&tmp, 0, sizeof tmp);
  tmp.nx = nx;
  tmp.ny = ny;
  tmp.M = nx / 2;
  tmp.lx = lx;
  tmp.ly = ly;
  tmp.dtype = dtype;
  if (!make_rp(tmp.M, dtype == FS_F64, &tmp.rp_row) || !make_rp(ny, dtype == FS_F64, &tmp.rp_col))
    return set_error(FS_ERR_SIZE, "fs_plan_create: no radix plan for this size");
  tmp.csize = dtype == FS_F64 ? 2 * sizeof(double) : 2 * sizeof(float);
  tmp.tc = make_tiles(nx, ny, tmp.rp_row, tmp.rp_col, tmp.csize);
  // complex (C2C) rows of length nx; some FP64 lengths (5 * 2^k, k >= 8) need
  // more radix-2 stages than a plan holds: complex solves then report FS_ERR_SIZE
  if (!make_rp(nx, dtype == FS_F64, &tmp.rp_rowc)) memset(&tmp.rp_rowc, 0, sizeof tmp.rp_rowc);
  if (tmp.rp_rowc.e) {  // complex row tiles: up to 16 rows, <= 512 threads, ~96 KB exchange
    const int tr = nx / tmp.rp_rowc.e;
    int cr = 16;
    while (cr > 1 && (cr * tr > kMaxThreads || tmp.csize * padded_len(cr * nx) > 96 * 1024)) cr >>= 1;
    tmp.tc.rows_per_unit_c = cr > ny ? ny : cr;
  }
  const int small_max = env_int("FS_SMALL_MAX", 128 * 128);
  tmp.standalone_small = (nx * ny <= small_max) && tmp.tc.small_smem2 > 0;
  tmp.spec_bytes = (size_t)(tmp.M + 1) * ny * tmp.csize;

  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    return set_error(FS_ERR_NODEV, "fs_plan_create: no CUDA device visible");
  }
  e = cudaGetDevice(&tmp.device);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  // tuned configuration: forced (tuner candidates) or from the cache
  {
    TuneCfg cfg{};
    if (force) {
      if (!apply_cfg(&tmp, *force)) return set_error(FS_ERR_ARG, "fs_plan_create: configuration does not fit");
    } else if (tune_lookup(tmp.device, nx, ny, dtype, 0, &cfg)) {
      fs_plan_s keep = tmp;
      if (!apply_cfg(&tmp, cfg)) tmp = keep;  // a stale entry: keep the defaults
    }
    tmp.standalone_small = (nx * ny <= small_max) && tmp.tc.small_smem2 > 0;
  }

  // ---- host tables in FP64
  const bool f64 = dtype == FS_F64;
  const int M = tmp.M;
  std::vector<double> wx2d(nx), wy2d(ny);  // x: all nx frequencies (complex fields)
  for (int a = 0; a < nx; ++a) wx2d[a] = omega2_axis(a, nx, lx);
  for (int b = 0; b < ny; ++b) wy2d[b] = omega2_axis(b, ny, ly);
  auto twiddles = [&](int n, std::vector<unsigned char> &buf) {
    buf.resize((size_t)n * tmp.csize);
    for (int m = 0; m < n; ++m) {
      const double ang = 2.0 * M_PI * (double)m / (double)n;  // exact integer m < n
      const double c = cos(ang), s = -sin(ang);                // e^{-2 pi i m / n}
      if (f64) {
        double *q = reinterpret_cast<double *>(buf.data()) + 2 * m;
        q[0] = c;
        q[1] = s;
      } else {
        float *q = reinterpret_cast<float *>(buf.data()) + 2 * m;
        q[0] = (float)c;
        q[1] = (float)s;
      }
    }
  };
  std::vector<unsigned char> twx, twy;
  twiddles(nx, twx);
  twiddles(ny, twy);
  auto axis_tab = [&](const std::vector<double> &w, std::vector<unsigned char> &buf) {
    if (f64) {
      buf.resize(w.size() * sizeof(double));
      memcpy(buf.data(), w.data(), buf.size());
    } else {
      buf.resize(w.size() * sizeof(float2));
      float *q = reinterpret_cast<float *>(buf.data());
      for (size_t i = 0; i < w.size(); ++i) split_double(w[i], q[2 * i], q[2 * i + 1]);
    }
  };
  std::vector<unsigned char> wxt, wyt;
  axis_tab(wx2d, wxt);
  axis_tab(wy2d, wyt);

  auto al = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t o_twx = 0, o_twy = o_twx + al(twx.size()), o_wx = o_twy + al(twy.size()),
               o_wy = o_wx + al(wxt.size()), o_wxd = o_wy + al(wyt.size()),
               o_wyd = o_wxd + al(wx2d.size() * 8), total = o_wyd + al(wy2d.size() * 8);

  fs_plan p = new (std::nothrow) fs_plan_s(tmp);
  if (!p) return set_error(FS_ERR_NOMEM, "fs_plan_create: host allocation");
  e = alloc_dev(&p->tables, total);
  if (e == cudaSuccess) e = alloc_dev(&p->work_u, p->spec_bytes);
  if (e == cudaSuccess) e = alloc_dev(&p->fac, fac_bytes(p));
  if (e != cudaSuccess) {
    cudaFree(p->tables);
    cudaFree(p->work_u);
    cudaFree(p->fac);
    delete p;
    return cuda_error(e, "fs_plan_create: device allocation");
  }
  char *base = reinterpret_cast<char *>(p->tables);
  p->tw_x = base + o_twx;
  p->tw_y = base + o_twy;
  p->wx2 = base + o_wx;
  p->wy2 = base + o_wy;
  p->wx2d = reinterpret_cast<double *>(base + o_wxd);
  p->wy2d = reinterpret_cast<double *>(base + o_wyd);
  e = cudaMemcpy(p->tw_x, twx.data(), twx.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->tw_y, twy.data(), twy.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->wx2, wxt.data(), wxt.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->wy2, wyt.data(), wyt.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->wx2d, wx2d.data(), wx2d.size() * 8, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->wy2d, wy2d.data(), wy2d.size() * 8, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    fs_plan_destroy(p);
    return cuda_error(e, "fs_plan_create: table upload");
  }
  *out = p;
  return FS_OK;
}

extern "C" {

fs_status fs_plan_tiles(fs_plan p, int *e_row, int *e_col, int *rows, int *cols) {
  if (!p) return set_error(FS_ERR_ARG, "fs_plan_tiles: plan is NULL");
  if (e_row) *e_row = p->rp_row.e;
  if (e_col) *e_col = p->rp_col.e;
  if (rows) *rows = p->tc.rows_per_unit;
  if (cols) *cols = p->tc.cols_per_unit;
  return FS_OK;
}

fs_status fs_plan_destroy(fs_plan p) {
  if (!p) return FS_OK;
  cudaDeviceSynchronize();
  cudaFree(p->tables);
  cudaFree(p->work_u);
  cudaFree(p->work_v);
  cudaFree(p->work_c);
  cudaFree(p->work_cv);
  cudaFree(p->fac);
  cudaFree(p->pfac);
  delete p;
  return FS_OK;
}

fs_status fs_plan_info(fs_plan p, int *nx, int *ny, int *dtype, int *path, size_t *ws) {
  if (!p) return set_error(FS_ERR_ARG, "fs_plan_info: plan is NULL");
  if (nx) *nx = p->nx;
  if (ny) *ny = p->ny;
  if (dtype) *dtype = p->dtype;
  if (path) *path = p->standalone_small ? 0 : 1;
  if (ws) *ws = p->spec_bytes * (p->work_v ? 2 : 1) + fac_bytes(p);
  return FS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- dispatch
template <typename T>
static cudaError_t run_desc(const fs_plan_s *p, const Desc &d, cudaStream_t s) {
  typedef Launch<T> L;
  const bool diff = d.op == OP_DIFFUSION || d.op == OP_DIFF_ADV;
  const bool adv = d.op == OP_DIFF_ADV || d.op == OP_WAVE_ADV;
  const bool has_v = (d.flags & F_HAS_V0) != 0;
  if (p->standalone_small) return L::small(d, s);
  cudaError_t e = cudaSuccess;
  if (diff) e = L::factor(d, s);
  if (e == cudaSuccess && !adv) {
    const int fields = ((d.op == OP_WAVE || d.op == OP_FORWARD) && has_v) ? 2 : 1;
    e = L::rows(d, fields, s);
  }
  if (e == cudaSuccess) e = L::cols(d, s);
  if (e == cudaSuccess && d.op != OP_FORWARD) {
    const int fields = (d.op == OP_WAVE_ADV && (d.flags & F_WANT_V)) ? 2 : 1;
    e = L::c2r(d, fields, s);
  }
  return e;
}

static fs_status run(const fs_plan_s *p, const Desc &d, fs_stream stream, const char *what) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = p->dtype == FS_F64 ? run_desc<double>(p, d, s) : run_desc<float>(p, d, s);
  if (e != cudaSuccess) return cuda_error(e, what);
  return FS_OK;
}

// ---------------------------------------------------------------- complex fields
// The full x spectrum: descriptor with M = nx - 1 (columns a = 0..nx-1 of the
// x-frequency-major spectrum; the column units, operators and factor tables
// cover them unchanged), complex row tiles and the length-nx radix plan.
static Desc complex_desc(const fs_plan_s *p) {
  Desc d = base_desc(p);
  d.M = p->nx - 1;
  d.rp_row = p->rp_rowc;
  d.rows_per_unit = p->tc.rows_per_unit_c;
  d.n_row_units = (p->ny + d.rows_per_unit - 1) / d.rows_per_unit;
  d.n_col_units = (p->nx + d.cols_per_unit - 1) / d.cols_per_unit;
  d.n_fac_units = (p->nx + p->ny + kFactorPerUnit - 1) / kFactorPerUnit;
  d.work_u = p->work_c;
  d.work_v = p->work_cv;
  d.small = 0;
  return d;
}

static fs_status ensure_work_c(fs_plan p, bool two) {
  const size_t bytes = (size_t)p->nx * p->ny * p->csize;
  cudaError_t e = cudaSuccess;
  if (!p->work_c) e = alloc_dev(&p->work_c, bytes);
  if (e == cudaSuccess && two && !p->work_cv) e = alloc_dev(&p->work_cv, bytes);
  if (e != cudaSuccess) return cuda_error(e, "complex workspace allocation");
  return FS_OK;
}

template <typename T>
static cudaError_t run_complex_desc(const Desc &d, cudaStream_t s) {
  typedef Launch<T> L;
  const PassKernels pk = pass_kernels<T>(d.rp_row.e);
  PassKernel kf = pk.c2cf, ki = pk.c2ci;
  // FP32 power-of-two rows: the compile-time kernels when the tile matches
  if (sizeof(T) == 4 && d.rp_row.e == 16 && p2_c2c_ok(d.nx) && d.rows_per_unit == p2_c2c_cnt(d.nx)) {
    kf = p2_c2c_f32(d.nx, false);
    ki = p2_c2c_f32(d.nx, true);
  }
  const int threads = round_up32(d.rows_per_unit * (d.nx / d.rp_row.e));
  const size_t smem = sizeof(cx<T>) * (size_t)padded_len(d.rows_per_unit * d.nx);
  const int fields = (d.op == OP_WAVE && (d.flags & F_HAS_V0)) ? 2 : 1;
  cudaError_t e = cudaSuccess;
  if (d.op == OP_DIFFUSION) e = L::factor(d, s);
  if (e == cudaSuccess) e = L::launch(kf, d.n_row_units * fields, threads, smem, d, s, PC_R2C);
  if (e == cudaSuccess) e = L::cols(d, s);
  if (e == cudaSuccess) e = L::launch(ki, d.n_row_units, threads, smem, d, s, PC_C2R);
  return e;
}

static fs_status run_complex(fs_plan p, Desc &d, fs_stream stream, const char *what) {
  if (!p->rp_rowc.e) return set_error(FS_ERR_SIZE, std::string(what) + ": no complex row plan for this nx and dtype");
  fs_status st = ensure_work_c(p, (d.flags & F_HAS_V0) != 0);
  if (st != FS_OK) return st;
  d.work_u = p->work_c;
  d.work_v = p->work_cv;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = p->dtype == FS_F64 ? run_complex_desc<double>(d, s) : run_complex_desc<float>(d, s);
  if (e != cudaSuccess) return cuda_error(e, what);
  return FS_OK;
}

namespace fs {
fs_status forward_into(const fs_plan_s *p, const void *u0, const void *v0, void *su, void *sv,
                       fs_stream stream, const char *what) {
  if (v0 && !p->standalone_small) {
    fs_status st = ensure_work_v(const_cast<fs_plan_s *>(p));
    if (st != FS_OK) return st;
  }
  Desc d = base_desc(p);
  d.op = OP_FORWARD;
  d.flags = v0 ? F_HAS_V0 : 0;
  d.in_u = u0;
  d.in_v = v0;
  d.st_out_u = su;
  d.st_out_v = sv;
  return run(p, d, stream, what);
}
}  // namespace fs

extern "C" {

fs_status fs_poisson_solve(fs_plan p, const void *f, void *u, fs_stream stream) {
  if (!p || !f || !u) return set_error(FS_ERR_ARG, "fs_poisson_solve: NULL argument");
  Desc d = base_desc(p);
  d.op = OP_POISSON;
  d.in_u = f;
  d.out_u = u;
  if (p->dtype == FS_F32 && !p->standalone_small && poisson_table_enabled()) {
    const fs_status st = ensure_pfac(p, reinterpret_cast<cudaStream_t>(stream));
    if (st != FS_OK) return st;
    d.pfac = p->pfac;
  }
  return run(p, d, stream, "fs_poisson_solve");
}

fs_status fs_diffusion_solve(fs_plan p, const void *u0, double D, double t, void *u,
                             fs_stream stream) {
  if (!p || !u0 || !u) return set_error(FS_ERR_ARG, "fs_diffusion_solve: NULL argument");
  if (!(D >= 0.0) || !(t >= 0.0) || !std::isfinite(D * t))
    return set_error(FS_ERR_ARG, "fs_diffusion_solve: need finite D >= 0 and t >= 0");
  Desc d = base_desc(p);
  d.op = OP_DIFFUSION;
  d.in_u = u0;
  d.out_u = u;
  d.p_dt = D * t;
  d.p_t = t;
  return run(p, d, stream, "fs_diffusion_solve");
}

fs_status fs_wave_solve(fs_plan p, const void *u0, const void *v0, double c, double t, void *u,
                        fs_stream stream) {
  if (!p || !u0 || !u) return set_error(FS_ERR_ARG, "fs_wave_solve: NULL argument");
  if (!(c > 0.0) || !std::isfinite(c) || !std::isfinite(t))
    return set_error(FS_ERR_ARG, "fs_wave_solve: need finite c > 0 and finite t");
  if (!wave_phase_ok(p, c, t))
    return set_error(FS_ERR_ARG, "fs_wave_solve: wave phase out of range (FP32 plans need c |t| |omega|_max <= 2^20)");
  if (v0 && !p->standalone_small) {
    fs_status st = ensure_work_v(p);
    if (st != FS_OK) return st;
  }
  Desc d = base_desc(p);
  d.op = OP_WAVE;
  d.flags = v0 ? F_HAS_V0 : 0;
  d.in_u = u0;
  d.in_v = v0;
  d.out_u = u;
  d.p_c = c;
  d.p_t = t;
  return run(p, d, stream, "fs_wave_solve");
}

}  // extern "C"

// ---------------------------------------------------------------- operator factors
// The real multiplier the FP32 column pass applies to each half-spectrum
// element (a, b) (for the wave: the factor of U0, cos(c|w|t) / (nx ny)),
// evaluated as the column pass does (two-float, fs_ops.cuh) or in FP64 and
// rounded once; a measurement of the FP32 path's factor precision and of
// the cost of FP64 evaluation on this GPU.
template <bool FP64>
__global__ void k_op_factors(const Desc d, float *out) {
  const size_t n = (size_t)(d.M + 1) * d.ny;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const int a = (int)(i / d.ny), b = (int)(i - (size_t)a * d.ny);
    if constexpr (FP64) {
      const int bp = (2 * b <= d.ny) ? b : b - d.ny;
      const double w2 = d.wx2d[a] + d.wy_unit2 * ((double)bp * (double)bp);
      double f;
      if (d.op == OP_POISSON) {
        f = w2 > 0.0 ? -d.scale / w2 : 0.0;
      } else if (d.op == OP_DIFFUSION) {
        f = d.scale * exp(-d.p_dt * w2);
      } else {
        f = d.scale * cos(d.p_c * d.p_t * sqrt(w2));
      }
      out[i] = (float)f;
    } else {
      const OpCtx<float> o = op_ctx<float>(d, a);
      float f;
      if (d.op == OP_POISSON) {
        f = poisson_mult(o, d, b);
      } else if (d.op == OP_DIFFUSION) {
        f = diff_mult(o, d, b);
      } else {
        f = wave_mult(o, d, b).cu;
      }
      out[i] = f;
    }
  }
}

extern "C" {

fs_status fs_operator_factors(fs_plan p, int op, double D, double c, double t, int fp64, void *out,
                              fs_stream stream) {
  if (!p || !out) return set_error(FS_ERR_ARG, "fs_operator_factors: NULL argument");
  if (p->dtype != FS_F32) return set_error(FS_ERR_ARG, "fs_operator_factors: FP32 plans only");
  Desc d = base_desc(p);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (op == FS_OP_POISSON) {
    d.op = OP_POISSON;
  } else if (op == FS_OP_DIFFUSION) {
    if (!(D >= 0.0) || !(t >= 0.0) || !std::isfinite(D * t))
      return set_error(FS_ERR_ARG, "fs_operator_factors: need finite D >= 0 and t >= 0");
    d.op = OP_DIFFUSION;
    d.p_dt = D * t;
    d.p_t = t;
  } else if (op == FS_OP_WAVE) {
    if (!(c > 0.0) || !std::isfinite(c) || !std::isfinite(t))
      return set_error(FS_ERR_ARG, "fs_operator_factors: need finite c > 0 and finite t");
    if (!wave_phase_ok(p, c, t))
      return set_error(FS_ERR_ARG,
                       "fs_operator_factors: wave phase out of range (FP32 plans need c |t| |omega|_max <= 2^20)");
    d.op = OP_WAVE;
    d.p_c = c;
    d.p_t = t;
  } else {
    return set_error(FS_ERR_ARG, "fs_operator_factors: op must be FS_OP_POISSON, FS_OP_DIFFUSION or FS_OP_WAVE");
  }
  fill_op_consts(d);
  cudaError_t e = cudaSuccess;
  if (d.op == OP_DIFFUSION && !fp64) e = Launch<float>::factor(d, s);
  if (e == cudaSuccess) {
    const size_t n = (size_t)(p->M + 1) * p->ny;
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 16);
    ProfScope ps(PC_FACTOR, s);
    if (fp64)
      k_op_factors<true><<<blocks, 256, 0, s>>>(d, reinterpret_cast<float *>(out));
    else
      k_op_factors<false><<<blocks, 256, 0, s>>>(d, reinterpret_cast<float *>(out));
    g_launches.fetch_add(1, std::memory_order_relaxed);
    e = cudaGetLastError();
  }
  return e == cudaSuccess ? FS_OK : cuda_error(e, "fs_operator_factors");
}

}  // extern "C"

// ---------------------------------------------------------------- slab passes
// The building blocks of a solve split across ranks by slabs (Sec. II.D: the
// 2D DFT is the x transforms of every row followed by the y transforms of
// every column, so a slab of rows and a slab of x frequencies are each
// transformed locally).  See include/fsolve.h.
template <typename T>
static cudaError_t slab_rows(const fs_plan_s *p, int nrows, const void *in, void *spec, void *out, bool inverse,
                             cudaStream_t s) {
  Desc d = base_desc(p);
  d.op = OP_FORWARD;
  d.ny = nrows;
  d.n_row_units = (nrows + d.rows_per_unit - 1) / d.rows_per_unit;
  d.in_u = in;
  d.work_u = spec;
  d.out_u = out;
  return inverse ? Launch<T>::c2r(d, 1, s) : Launch<T>::rows(d, 1, s);
}

template <typename T>
static cudaError_t slab_cols(const Desc &d, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (d.op == OP_DIFFUSION) e = Launch<T>::factor(d, s);
  if (e == cudaSuccess) e = Launch<T>::cols(d, s);
  return e;
}

extern "C" {

fs_status fs_rows_forward(fs_plan p, int nrows, const void *f, void *spec, fs_stream stream) {
  if (!p || !f || !spec) return set_error(FS_ERR_ARG, "fs_rows_forward: NULL argument");
  if (nrows < 1 || nrows > p->ny) return set_error(FS_ERR_ARG, "fs_rows_forward: need 1 <= nrows <= ny");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const cudaError_t e = p->dtype == FS_F64 ? slab_rows<double>(p, nrows, f, spec, nullptr, false, s)
                                           : slab_rows<float>(p, nrows, f, spec, nullptr, false, s);
  return e == cudaSuccess ? FS_OK : cuda_error(e, "fs_rows_forward");
}

fs_status fs_rows_inverse(fs_plan p, int nrows, const void *spec, void *u, fs_stream stream) {
  if (!p || !spec || !u) return set_error(FS_ERR_ARG, "fs_rows_inverse: NULL argument");
  if (nrows < 1 || nrows > p->ny) return set_error(FS_ERR_ARG, "fs_rows_inverse: need 1 <= nrows <= ny");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const cudaError_t e = p->dtype == FS_F64 ? slab_rows<double>(p, nrows, nullptr, const_cast<void *>(spec), u, true, s)
                                           : slab_rows<float>(p, nrows, nullptr, const_cast<void *>(spec), u, true, s);
  return e == cudaSuccess ? FS_OK : cuda_error(e, "fs_rows_inverse");
}

fs_status fs_columns_apply(fs_plan p, int a0, int ncols, int op, double D, double c, double t, void *spec_cols,
                           fs_stream stream) {
  if (!p || !spec_cols) return set_error(FS_ERR_ARG, "fs_columns_apply: NULL argument");
  if (a0 < 0 || ncols < 1 || a0 + ncols > p->M + 1)
    return set_error(FS_ERR_ARG, "fs_columns_apply: columns a0 .. a0+ncols-1 must lie in 0 .. nx/2");
  Desc d = base_desc(p);
  if (op == FS_OP_POISSON) {
    d.op = OP_POISSON;
  } else if (op == FS_OP_DIFFUSION) {
    if (!(D >= 0.0) || !(t >= 0.0) || !std::isfinite(D * t))
      return set_error(FS_ERR_ARG, "fs_columns_apply: need finite D >= 0 and t >= 0");
    d.op = OP_DIFFUSION;
    d.p_dt = D * t;
    d.p_t = t;
  } else if (op == FS_OP_WAVE) {
    if (!(c > 0.0) || !std::isfinite(c) || !std::isfinite(t))
      return set_error(FS_ERR_ARG, "fs_columns_apply: need finite c > 0 and finite t");
    if (!wave_phase_ok(p, c, t))
      return set_error(FS_ERR_ARG,
                       "fs_columns_apply: wave phase out of range (FP32 plans need c |t| |omega|_max <= 2^20)");
    d.op = OP_WAVE;
    d.p_c = c;
    d.p_t = t;
  } else {
    return set_error(FS_ERR_ARG, "fs_columns_apply: op must be FS_OP_POISSON, FS_OP_DIFFUSION or FS_OP_WAVE");
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // columns a0 .. a0+ncols-1 become 0 .. ncols-1 of the descriptor: the x
  // wavenumber tables (8 bytes per entry in both precisions) start at a0
  d.M = ncols - 1;
  d.n_col_units = (ncols + d.cols_per_unit - 1) / d.cols_per_unit;
  d.n_fac_units = (ncols + p->ny + kFactorPerUnit - 1) / kFactorPerUnit;
  d.wx2 = static_cast<const char *>(p->wx2) + (size_t)a0 * 8;
  d.wx2d = p->wx2d + a0;
  d.work_u = spec_cols;
  if (d.op == OP_POISSON && p->dtype == FS_F32 && poisson_table_enabled()) {
    const fs_status st = ensure_pfac(p, s);
    if (st != FS_OK) return st;
    d.pfac = p->pfac + (size_t)a0 * p->ny;
  }
  const cudaError_t e = p->dtype == FS_F64 ? slab_cols<double>(d, s) : slab_cols<float>(d, s);
  return e == cudaSuccess ? FS_OK : cuda_error(e, "fs_columns_apply");
}

fs_status fs_poisson_solve_c(fs_plan p, const void *f, void *u, fs_stream stream) {
  if (!p || !f || !u) return set_error(FS_ERR_ARG, "fs_poisson_solve_c: NULL argument");
  Desc d = complex_desc(p);
  d.op = OP_POISSON;
  d.in_u = f;
  d.out_u = u;
  return run_complex(p, d, stream, "fs_poisson_solve_c");
}

fs_status fs_diffusion_solve_c(fs_plan p, const void *u0, double D, double t, void *u, fs_stream stream) {
  if (!p || !u0 || !u) return set_error(FS_ERR_ARG, "fs_diffusion_solve_c: NULL argument");
  if (!(D >= 0.0) || !(t >= 0.0) || !std::isfinite(D * t))
    return set_error(FS_ERR_ARG, "fs_diffusion_solve_c: need finite D >= 0 and t >= 0");
  Desc d = complex_desc(p);
  d.op = OP_DIFFUSION;
  d.in_u = u0;
  d.out_u = u;
  d.p_dt = D * t;
  d.p_d = D;
  d.p_t = t;
  return run_complex(p, d, stream, "fs_diffusion_solve_c");
}

fs_status fs_wave_solve_c(fs_plan p, const void *u0, const void *v0, double c, double t, void *u,
                          fs_stream stream) {
  if (!p || !u0 || !u) return set_error(FS_ERR_ARG, "fs_wave_solve_c: NULL argument");
  if (!(c > 0.0) || !std::isfinite(c) || !std::isfinite(t))
    return set_error(FS_ERR_ARG, "fs_wave_solve_c: need finite c > 0 and finite t");
  if (!wave_phase_ok(p, c, t))
    return set_error(FS_ERR_ARG, "fs_wave_solve_c: wave phase out of range (FP32 plans need c |t| |omega|_max <= 2^20)");
  Desc d = complex_desc(p);
  d.op = OP_WAVE;
  d.flags = v0 ? F_HAS_V0 : 0;
  d.in_u = u0;
  d.in_v = v0;
  d.out_u = u;
  d.p_c = c;
  d.p_t = t;
  return run_complex(p, d, stream, "fs_wave_solve_c");
}

fs_status fs_state_create(fs_plan p, const void *u0, const void *v0, fs_stream stream,
                          fs_state *out) {
  if (!out) return set_error(FS_ERR_ARG, "fs_state_create: out is NULL");
  *out = nullptr;
  if (!p || !u0) return set_error(FS_ERR_ARG, "fs_state_create: NULL argument");
  if (v0 && !p->standalone_small) {
    fs_status st = ensure_work_v(p);
    if (st != FS_OK) return st;
  }
  fs_state s = new (std::nothrow) fs_state_s();
  if (!s) return set_error(FS_ERR_NOMEM, "fs_state_create: host allocation");
  s->plan = p;
  s->has_v = v0 != nullptr;
  cudaError_t e = alloc_dev(&s->su, p->spec_bytes);
  if (e == cudaSuccess && v0) e = alloc_dev(&s->sv, p->spec_bytes);
  if (e != cudaSuccess) {
    cudaFree(s->su);
    delete s;
    return cuda_error(e, "fs_state_create: device allocation");
  }
  Desc d = base_desc(p);
  d.op = OP_FORWARD;
  d.flags = v0 ? F_HAS_V0 : 0;
  d.in_u = u0;
  d.in_v = v0;
  d.st_out_u = s->su;
  d.st_out_v = s->sv;
  fs_status st = run(p, d, stream, "fs_state_create");
  if (st != FS_OK) {
    cudaFree(s->su);
    cudaFree(s->sv);
    delete s;
    return st;
  }
  *out = s;
  return FS_OK;
}

fs_status fs_state_reset(fs_state s, const void *u0, const void *v0, fs_stream stream) {
  if (!s || !u0) return set_error(FS_ERR_ARG, "fs_state_reset: NULL argument");
  if ((v0 != nullptr) != s->has_v)
    return set_error(FS_ERR_ARG, "fs_state_reset: v0 presence must match the state");
  fs_plan p = s->plan;
  Desc d = base_desc(p);
  d.op = OP_FORWARD;
  d.flags = v0 ? F_HAS_V0 : 0;
  d.in_u = u0;
  d.in_v = v0;
  d.st_out_u = s->su;
  d.st_out_v = s->sv;
  return run(p, d, stream, "fs_state_reset");
}

fs_status fs_state_set_source(fs_state s, const void *src, fs_stream stream) {
  if (!s) return set_error(FS_ERR_ARG, "fs_state_set_source: NULL state");
  if (!src) {
    s->has_s = false;
    return FS_OK;
  }
  fs_plan p = s->plan;
  if (!s->ss) {
    cudaError_t e = alloc_dev(&s->ss, p->spec_bytes);
    if (e != cudaSuccess) {
      s->ss = nullptr;
      return cuda_error(e, "fs_state_set_source: device allocation");
    }
  }
  Desc d = base_desc(p);
  d.op = OP_FORWARD;
  d.in_u = src;
  d.st_out_u = s->ss;
  fs_status st = run(p, d, stream, "fs_state_set_source");
  s->has_s = st == FS_OK;
  return st;
}

fs_status fs_state_destroy(fs_state s) {
  if (!s) return FS_OK;
  cudaDeviceSynchronize();
  cudaFree(s->su);
  cudaFree(s->sv);
  cudaFree(s->ss);
  delete s;
  return FS_OK;
}

// ---------------------------------------------------------------- checkpoints
// Header + the kept spectra (U0, then V0 when present, then the source
// spectrum when attached), each (nx/2+1) * ny complex of the plan dtype.
struct StateHeader {
  char magic[8];  // "FSSTATE1"
  int32_t nx, ny, dtype, has_v, has_s, pad;
  double lx, ly;
};

fs_status fs_state_bytes(fs_state s, size_t *bytes) {
  if (!s || !bytes) return set_error(FS_ERR_ARG, "fs_state_bytes: NULL argument");
  *bytes = sizeof(StateHeader) + s->plan->spec_bytes * (1 + (s->has_v ? 1 : 0) + (s->has_s ? 1 : 0));
  return FS_OK;
}

fs_status fs_state_save(fs_state s, void *dst, size_t cap, fs_stream stream) {
  size_t need = 0;
  fs_status st = fs_state_bytes(s, &need);
  if (st != FS_OK) return st;
  if (!dst || cap < need) return set_error(FS_ERR_ARG, "fs_state_save: destination missing or too small");
  const fs_plan_s *p = s->plan;
  StateHeader h;
  memset(&h, 0, sizeof h);
  memcpy(h.magic, "FSSTATE1", 8);
  h.nx = p->nx;
  h.ny = p->ny;
  h.dtype = p->dtype;
  h.has_v = s->has_v ? 1 : 0;
  h.has_s = s->has_s ? 1 : 0;
  h.lx = p->lx;
  h.ly = p->ly;
  memcpy(dst, &h, sizeof h);
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  char *q = static_cast<char *>(dst) + sizeof h;
  const void *parts[3] = {s->su, s->has_v ? s->sv : nullptr, s->has_s ? s->ss : nullptr};
  cudaError_t e = cudaSuccess;
  for (const void *src : parts) {
    if (!src || e != cudaSuccess) continue;
    e = cudaMemcpyAsync(q, src, p->spec_bytes, cudaMemcpyDeviceToHost, cs);
    q += p->spec_bytes;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);
  if (e != cudaSuccess) return cuda_error(e, "fs_state_save");
  return FS_OK;
}

fs_status fs_state_load(fs_state s, const void *src, size_t bytes, fs_stream stream) {
  if (!s || !src) return set_error(FS_ERR_ARG, "fs_state_load: NULL argument");
  if (bytes < sizeof(StateHeader)) return set_error(FS_ERR_ARG, "fs_state_load: checkpoint too short");
  StateHeader h;
  memcpy(&h, src, sizeof h);
  const fs_plan_s *p = s->plan;
  if (memcmp(h.magic, "FSSTATE1", 8) != 0) return set_error(FS_ERR_ARG, "fs_state_load: not a state checkpoint");
  if (h.nx != p->nx || h.ny != p->ny || h.dtype != p->dtype || h.lx != p->lx || h.ly != p->ly)
    return set_error(FS_ERR_ARG, "fs_state_load: checkpoint is for another grid, domain or dtype");
  if ((h.has_v != 0) != s->has_v)
    return set_error(FS_ERR_ARG, "fs_state_load: v0 presence must match the state");
  const size_t need = sizeof h + p->spec_bytes * (1 + (h.has_v ? 1 : 0) + (h.has_s ? 1 : 0));
  if (bytes < need) return set_error(FS_ERR_ARG, "fs_state_load: checkpoint truncated");
  if (h.has_s && !s->ss) {
    cudaError_t e = alloc_dev(&s->ss, p->spec_bytes);
    if (e != cudaSuccess) {
      s->ss = nullptr;
      return cuda_error(e, "fs_state_load: device allocation");
    }
  }
  cudaStream_t cs = reinterpret_cast<cudaStream_t>(stream);
  const char *q = static_cast<const char *>(src) + sizeof h;
  void *parts[3] = {s->su, h.has_v ? s->sv : nullptr, h.has_s ? s->ss : nullptr};
  cudaError_t e = cudaSuccess;
  for (void *dst : parts) {
    if (!dst || e != cudaSuccess) continue;
    e = cudaMemcpyAsync(dst, q, p->spec_bytes, cudaMemcpyHostToDevice, cs);
    q += p->spec_bytes;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(cs);  // the caller may reuse `src` on return
  if (e != cudaSuccess) return cuda_error(e, "fs_state_load");
  s->has_s = h.has_s != 0;
  return FS_OK;
}

fs_status fs_diffusion_advance(fs_state s, double D, double t, void *u_out, fs_stream stream) {
  if (!s || !u_out) return set_error(FS_ERR_ARG, "fs_diffusion_advance: NULL argument");
  if (!(D >= 0.0) || !(t >= 0.0) || !std::isfinite(D * t))
    return set_error(FS_ERR_ARG, "fs_diffusion_advance: need finite D >= 0 and t >= 0");
  fs_plan p = s->plan;
  Desc d = base_desc(p);
  d.op = OP_DIFF_ADV;
  d.st_u = s->su;
  d.out_u = u_out;
  d.p_dt = D * t;
  d.p_d = D;
  d.p_t = t;
  if (s->has_s) {
    d.flags |= F_SOURCE;
    d.st_s = s->ss;
  }
  return run(p, d, stream, "fs_diffusion_advance");
}

fs_status fs_wave_advance(fs_state s, double c, double t, void *u_out, void *v_out,
                          fs_stream stream) {
  if (!s || !u_out) return set_error(FS_ERR_ARG, "fs_wave_advance: NULL argument");
  if (!(c > 0.0) || !std::isfinite(c) || !std::isfinite(t))
    return set_error(FS_ERR_ARG, "fs_wave_advance: need finite c > 0 and finite t");
  if (!wave_phase_ok(s->plan, c, t))
    return set_error(FS_ERR_ARG, "fs_wave_advance: wave phase out of range (FP32 plans need c |t| |omega|_max <= 2^20)");
  fs_plan p = s->plan;
  if (v_out && !p->standalone_small) {
    fs_status st = ensure_work_v(p);
    if (st != FS_OK) return st;
  }
  Desc d = base_desc(p);
  d.op = OP_WAVE_ADV;
  d.flags = (s->has_v ? F_HAS_V0 : 0) | (v_out ? F_WANT_V : 0);
  d.st_u = s->su;
  d.st_v = s->sv;
  d.out_u = u_out;
  d.out_v = v_out;
  d.p_c = c;
  d.p_t = t;
  if (s->has_s) {
    d.flags |= F_SOURCE;
    d.st_s = s->ss;
  }
  return run(p, d, stream, "fs_wave_advance");
}

}  // extern "C"
