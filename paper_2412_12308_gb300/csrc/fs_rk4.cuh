// fs_rk4.cuh -- RK4 time integration of the wave equation in Fourier space
// with a time-dependent source (Sec. III.C, example with an orbiting source).
//
// Per mode the wave equation is the first-order system of
// Eq. SystemOfODEsForWaveEquation, dU/dt = V, dV/dt = -c^2|w|^2 U + S(t),
// advanced with the classical fourth-order Runge-Kutta method.  The system is
// linear, so one step needs the source spectrum at three times only: t (kept
// from the previous step), t + dt/2 and t + dt.  One step is two launches:
//   rows    synthesise s(t + dt/2) and s(t + dt) on the grid (no input read)
//           and run the real row transforms of both      -> wa, wb
//   columns forward column transforms of wa and wb, then the whole RK4 step
//           for every mode in registers: read U, V, S(t); write U, V and
//           S(t + dt) (the next step's S(t)).
// The source is A exp(-|x - x0(tau)|^2/sigma^2) cos(gamma tau) with the
// minimum-image distance; the host gives, per stage time, the centre in grid
// index units and the amplitude A cos(gamma tau).
#pragma once
#include "fs_units.cuh"

namespace fs {

struct RkTime {
  double j0, i0;  // centre in index units: x0 = x_min + j0 hx, y0 = y_min + i0 hy, in [0, n)
  double amp;     // A cos(gamma tau)
};
struct RkStep {
  RkTime mid, end;  // source at t + dt/2 and t + dt
};

struct RkParams {
  const RkStep *steps;  // device table
  int step;             // this launch's entry
  int init;             // 1: S0 <- forward transform of the source at steps[step].mid
  double qx, qy;        // (hx/sigma)^2, (hy/sigma)^2: exponent per squared index distance
  double dt, c2;        // time step, c^2
  void *U, *V, *S0;     // half spectra [M+1][ny] (x-frequency major), updated in place
  void *wa, *wb;        // row-transformed source at t + dt/2 and t + dt
};

// Source samples at one stage time.  FP32: the index distance x - j0 is formed
// as (x - j0_hi) - j0_lo, where the first difference is exact, so the
// distance keeps its relative accuracy near the centre.
template <typename T>
struct OrbitGen;

template <>
struct OrbitGen<float> {
  float j0h, j0l, i0h, i0l, qx, qy, amp, nxf, nyf;
  __device__ OrbitGen(const RkTime &tm, const RkParams &r, int nx, int ny) {
    split_double(tm.j0, j0h, j0l);
    split_double(tm.i0, i0h, i0l);
    qx = (float)r.qx;
    qy = (float)r.qy;
    amp = (float)tm.amp;
    nxf = (float)nx;
    nyf = (float)ny;
  }
  __device__ static float wrap(float v, float n) {  // into [-n/2, n/2)
    return v >= 0.5f * n ? v - n : (v < -0.5f * n ? v + n : v);
  }
  __device__ cx<float> pair(int y, int x) const {
    const float dy = wrap(__fsub_rn(__fsub_rn((float)y, i0h), i0l), nyf);
    const float ey = dy * dy * qy;
    const float d0 = wrap(__fsub_rn(__fsub_rn((float)x, j0h), j0l), nxf);
    const float d1 = wrap(__fsub_rn(__fsub_rn((float)(x + 1), j0h), j0l), nxf);
    return mk<float>(amp * expf(-__fmaf_rn(d0 * d0, qx, ey)), amp * expf(-__fmaf_rn(d1 * d1, qx, ey)));
  }
};

template <>
struct OrbitGen<double> {
  double j0, i0, qx, qy, amp, nxd, nyd;
  __device__ OrbitGen(const RkTime &tm, const RkParams &r, int nx, int ny)
      : j0(tm.j0), i0(tm.i0), qx(r.qx), qy(r.qy), amp(tm.amp), nxd(nx), nyd(ny) {}
  __device__ static double wrap(double v, double n) {
    return v >= 0.5 * n ? v - n : (v < -0.5 * n ? v + n : v);
  }
  __device__ cx<double> pair(int y, int x) const {
    const double dy = wrap((double)y - i0, nyd);
    const double ey = dy * dy * qy;
    const double d0 = wrap((double)x - j0, nxd), d1 = wrap((double)(x + 1) - j0, nxd);
    return mk<double>(amp * exp(-(d0 * d0 * qx + ey)), amp * exp(-(d1 * d1 * qx + ey)));
  }
};

// Row pass: blocks [0, n_row_units) synthesise and transform the source at
// t + dt/2 into wa; with init == 0, blocks [n_row_units, 2 n_row_units) do
// t + dt into wb.
template <typename T, int E>
__device__ __forceinline__ void rk4_rows_body(const Desc &d, const RkParams &r, cx<T> *sm) {
  int unit = blockIdx.x;
  const RkStep &st = r.steps[r.step];
  const bool second = unit >= d.n_row_units;
  if (second) unit -= d.n_row_units;
  const OrbitGen<T> g(second ? st.end : st.mid, r, d.nx, d.ny);
  unit_row_r2c_t<T, E, 0, 0, OrbitGen<T>>(d, unit, d.rows_per_unit, sm, nullptr,
                                          reinterpret_cast<cx<T> *>(second ? r.wb : r.wa), &g);
}

__device__ __forceinline__ float rk_w2(const Desc &d, int a, int b, float c2) {
  const float2 wx = reinterpret_cast<const float2 *>(d.wx2)[a];
  const float2 wy = reinterpret_cast<const float2 *>(d.wy2)[b];
  return c2 * __fadd_rn(__fadd_rn(wx.x, wy.x), __fadd_rn(wx.y, wy.y));
}
__device__ __forceinline__ double rk_w2(const Desc &d, int a, int b, double c2) {
  return c2 * (reinterpret_cast<const double *>(d.wx2)[a] + reinterpret_cast<const double *>(d.wy2)[b]);
}

// Column pass: thread (rho, t) of column a = blockIdx.x * cols_per_unit + rho
// holds the frequencies b = t + Tseg*s after the forward transforms.
template <typename T, int E>
__device__ __forceinline__ void rk4_cols_body(const Desc &d, const RkParams &r, cx<T> *sm) {
  const int L = d.ny, M = d.M, Tseg = L / E, cnt = d.cols_per_unit;
  const int tid = threadIdx.x;
  const int rho = tid / Tseg, t = tid - rho * Tseg;
  const int a = blockIdx.x * cnt + rho;
  const bool active = (rho < cnt) && (a <= M);
  const XLayout lay{rho * L, 1};
  const cx<T> *tw = reinterpret_cast<const cx<T> *>(d.tw_y);
  const size_t cofs = (size_t)(active ? a : 0) * L;
  cx<T> *S0 = reinterpret_cast<cx<T> *>(r.S0) + cofs;
  cx<T> p[E];
  if (active) {
    const cx<T> *src = reinterpret_cast<const cx<T> *>(r.wa) + cofs;
#pragma unroll
    for (int s = 0; s < E; ++s) p[s] = ldg_cg(src + t + Tseg * s);
  } else {
#pragma unroll
    for (int s = 0; s < E; ++s) p[s] = zero_cx<T>();
  }
  fft_any<T, E, 0, 1, 1>(p, sm, lay, active, t, Tseg, L, d.rp_col, tw);
  if (r.init) {  // uniform over the launch
    if (active) {
#pragma unroll
      for (int s = 0; s < E; ++s) S0[t + Tseg * s] = p[s];
    }
    return;
  }
  cx<T> q[E];
  if (active) {
    const cx<T> *src = reinterpret_cast<const cx<T> *>(r.wb) + cofs;
#pragma unroll
    for (int s = 0; s < E; ++s) q[s] = ldg_cg(src + t + Tseg * s);
  } else {
#pragma unroll
    for (int s = 0; s < E; ++s) q[s] = zero_cx<T>();
  }
  __syncthreads();
  fft_any<T, E, 0, 1, 1>(q, sm, lay, active, t, Tseg, L, d.rp_col, tw);
  if (!active) return;
  cx<T> *U = reinterpret_cast<cx<T> *>(r.U) + cofs;
  cx<T> *V = reinterpret_cast<cx<T> *>(r.V) + cofs;
  const T h = (T)r.dt, hh = (T)(0.5 * r.dt), h6 = (T)(r.dt / 6.0), c2 = (T)r.c2;
#pragma unroll
  for (int s = 0; s < E; ++s) {
    const int b = t + Tseg * s;
    const T w2 = rk_w2(d, a, b, c2);
    const cx<T> u = ldg_cg(U + b), v = ldg_cg(V + b), s0 = ldg_cg(S0 + b);
    const cx<T> smid = p[s], s1 = q[s];
    // slopes of (U, V): k = (V, S - w2 U)
    const cx<T> k1u = v, k1v = s0 - w2 * u;
    const cx<T> k2u = v + hh * k1v, k2v = smid - w2 * (u + hh * k1u);
    const cx<T> k3u = v + hh * k2v, k3v = smid - w2 * (u + hh * k2u);
    const cx<T> k4u = v + h * k3v, k4v = s1 - w2 * (u + h * k3u);
    U[b] = u + h6 * (k1u + T(2) * (k2u + k3u) + k4u);
    V[b] = v + h6 * (k1v + T(2) * (k2v + k3v) + k4v);
    S0[b] = s1;
  }
}

typedef void (*Rk4Kernel)(const Desc, const RkParams);

#define FS_RK4_DECL(T, E)                                                  \
  __global__ void k_rk4r_##T##_##E(const Desc d, const RkParams r);        \
  __global__ void k_rk4c_##T##_##E(const Desc d, const RkParams r);

#define FS_RK4_DEF(T, E)                                                                    \
  __global__ void __launch_bounds__(512) k_rk4r_##T##_##E(const Desc d, const RkParams r) { \
    extern __shared__ __align__(16) unsigned char fs_smem[];                                \
    rk4_rows_body<T, E>(d, r, reinterpret_cast<cx<T> *>(fs_smem));                          \
  }                                                                                         \
  __global__ void __launch_bounds__(512) k_rk4c_##T##_##E(const Desc d, const RkParams r) { \
    extern __shared__ __align__(16) unsigned char fs_smem[];                                \
    rk4_cols_body<T, E>(d, r, reinterpret_cast<cx<T> *>(fs_smem));                          \
  }

FS_FOR_EACH_E_float(FS_RK4_DECL)
FS_FOR_EACH_E_double(FS_RK4_DECL)

#define FS_RK4_CASE(T, E) \
  case E:                 \
    return rows ? k_rk4r_##T##_##E : k_rk4c_##T##_##E;
template <typename T>
inline Rk4Kernel rk4_kernel(int e, bool rows);
template <>
inline Rk4Kernel rk4_kernel<float>(int e, bool rows) {
  switch (e) { FS_FOR_EACH_E_float(FS_RK4_CASE) default: return nullptr; }
}
template <>
inline Rk4Kernel rk4_kernel<double>(int e, bool rows) {
  switch (e) { FS_FOR_EACH_E_double(FS_RK4_CASE) default: return nullptr; }
}

}  // namespace fs
