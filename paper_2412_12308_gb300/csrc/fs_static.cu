// fs_static.cu -- fs_poisson_solve_static: the FP32 Poisson solve with all of
// its scratch (work spectrum, twiddle and wavenumber tables) in one fixed,
// file-scope device array, so a call allocates nothing.
//
// Who needs it: callers that may not allocate device memory while they run
// -- code hosted inside an application that owns the device memory pool and
// forbids direct cudaMalloc, latency-critical loops where an allocation (which
// can synchronise the device) is not acceptable, and integrations that size
// all device memory once at start-up.  They pass inputs and outputs only.
//
// Costs and limits: every GPU that loads this library holds the array
// (kStaticMaxN = 1024: about 4.2 MB) until the process exits; grids above
// 1024 x 1024 are rejected.  All calls share the one array and it keeps the
// last call's contents, so calls whose GPU work overlaps (different streams,
// or different host threads, on one device) race and must be serialised by
// the caller.  Nothing in the array needs to start at zero: every call
// rewrites the tables and every spectrum element before reading it.
#include <cmath>
#include <cstring>
#include <mutex>

#include "fs_host.h"
#include "fs_kernels.cuh"

extern template struct fs::Launch<float>;

namespace fs {
namespace {
constexpr int kStaticMaxN = 1024;
constexpr size_t kSpec = (size_t)(kStaticMaxN / 2 + 1) * kStaticMaxN;  // work spectrum
constexpr size_t kOffTwX = kSpec;
constexpr size_t kOffTwY = kOffTwX + kStaticMaxN;
constexpr size_t kOffWx = kOffTwY + kStaticMaxN;
constexpr size_t kOffWy = kOffWx + (kStaticMaxN / 2 + 1);
constexpr size_t kWords = kOffWy + kStaticMaxN;  // float2 words
constexpr int kMaxDevices = 64;

std::mutex g_static_mu;
float2 *g_static_ptr[kMaxDevices];
}  // namespace

static __device__ __align__(256) float2 g_static_scratch[kWords];

// Twiddles omega_n^m (FP64 sincospi, rounded once) and two-float |omega|^2
// tables for the grid, written into the static array.
__global__ void k_static_tables(int nx, int ny, double lx, double ly, float2 *base) {
  const int M = nx / 2;
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  const double two_pi = 6.283185307179586476925286766559;
  float hi, lo;
  if (i < nx) {
    double s, c;
    sincospi(2.0 * (double)i / (double)nx, &s, &c);
    base[kOffTwX + i] = make_float2((float)c, (float)(-s));
    return;
  }
  i -= nx;
  if (i < ny) {
    double s, c;
    sincospi(2.0 * (double)i / (double)ny, &s, &c);
    base[kOffTwY + i] = make_float2((float)c, (float)(-s));
    return;
  }
  i -= ny;
  if (i <= M) {
    const double w = two_pi * (double)i / lx;
    split_double(w * w, hi, lo);
    base[kOffWx + i] = make_float2(hi, lo);
    return;
  }
  i -= M + 1;
  if (i < ny) {
    const int bp = (2 * i <= ny) ? i : i - ny;
    const double w = two_pi * (double)bp / ly;
    split_double(w * w, hi, lo);
    base[kOffWy + i] = make_float2(hi, lo);
  }
}

// Device address of the static array on the current device, looked up once
// per device (cudaGetSymbolAddress with that device current).
static fs_status static_scratch(float2 **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "fs_poisson_solve_static: cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices)
    return set_error(FS_ERR_NODEV, "fs_poisson_solve_static: device index out of range");
  std::lock_guard<std::mutex> g(g_static_mu);
  if (!g_static_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_error(e, "fs_poisson_solve_static: cudaGetSymbolAddress");
    g_static_ptr[dev] = static_cast<float2 *>(p);
  }
  *out = g_static_ptr[dev];
  return FS_OK;
}

}  // namespace fs

using namespace fs;

extern "C" fs_status fs_poisson_solve_static(int nx, int ny, double lx, double ly, const void *f,
                                             void *u, fs_stream stream) {
  if (!f || !u) return set_error(FS_ERR_ARG, "fs_poisson_solve_static: NULL field pointer");
  if (!(lx > 0.0) || !(ly > 0.0) || !std::isfinite(lx) || !std::isfinite(ly))
    return set_error(FS_ERR_ARG, "fs_poisson_solve_static: Lx and Ly must be finite and > 0");
  if (!size_supported(nx) || !size_supported(ny))
    return set_error(FS_ERR_SIZE, "fs_poisson_solve_static: unsupported size");
  if (nx > kStaticMaxN || ny > kStaticMaxN)
    return set_error(FS_ERR_SIZE,
                     "fs_poisson_solve_static: grid exceeds the fixed scratch limit of 1024 x 1024");
  RadixPlan rr, rc;
  TileConfig tc;
  if (!plan_geometry(nx, ny, false, &rr, &rc, &tc))
    return set_error(FS_ERR_SIZE, "fs_poisson_solve_static: no radix plan for this size");
  float2 *base = nullptr;
  fs_status st = static_scratch(&base);
  if (st != FS_OK) return st;

  Desc d;
  memset(&d, 0, sizeof d);
  d.op = OP_POISSON;
  d.nx = nx;
  d.ny = ny;
  d.M = nx / 2;
  d.rows_per_unit = tc.rows_per_unit;
  d.cols_per_unit = tc.cols_per_unit;
  d.n_row_units = (ny + d.rows_per_unit - 1) / d.rows_per_unit;
  d.n_col_units = (d.M + 1 + d.cols_per_unit - 1) / d.cols_per_unit;
  d.rp_row = rr;
  d.rp_col = rc;
  d.in_u = f;
  d.out_u = u;
  d.work_u = base;
  d.tw_x = base + kOffTwX;
  d.tw_y = base + kOffTwY;
  d.wx2 = base + kOffWx;
  d.wy2 = base + kOffWy;
  d.scale = 1.0 / ((double)nx * (double)ny);
  d.wy_unit2 = (2.0 * M_PI / ly) * (2.0 * M_PI / ly);

  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int n_tab = nx + ny + (d.M + 1) + ny;
  k_static_tables<<<(n_tab + 255) / 256, 256, 0, s>>>(nx, ny, lx, ly, base);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = Launch<float>::rows(d, 1, s);
  if (e == cudaSuccess) e = Launch<float>::cols(d, s);
  if (e == cudaSuccess) e = Launch<float>::c2r(d, 1, s);
  if (e != cudaSuccess) return cuda_error(e, "fs_poisson_solve_static");
  return FS_OK;
}
