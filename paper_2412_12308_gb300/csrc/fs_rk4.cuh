// fs_rk4.cuh -- RK4 time integration of the wave equation in Fourier space
// with a time-dependent source (Sec. III.C, example with an orbiting source).
//
// Per mode the wave equation is the first-order system of
// Eq. SystemOfODEsForWaveEquation, dU/dt = V, dV/dt = -c^2|w|^2 U + S(t),
// advanced with the classical fourth-order Runge-Kutta method.  The source
// A exp(-|x - x0(tau)|^2/sigma^2) cos(gamma tau) with the minimum-image
// distance factorises exactly into exp(-dx^2/sigma^2) exp(-dy^2/sigma^2), so
// the 2D DFT of its samples is the outer product of two 1D DFTs:
//   S(a, b, tau) = Gx_tau(a) Gy_tau(b),
// Gx the half spectrum (a <= nx/2) of A cos(gamma tau) exp(-dx^2/sigma^2)
// along x, Gy the spectrum of exp(-dy^2/sigma^2) along y.  For a chunk of
// steps the 1D spectra at every stage time t + j dt/2 are computed first
// (one CTA per time point and axis, on the same FFT engine as the solves);
// then every mode runs all steps of the chunk with U and V in registers.
#pragma once
#include "fs_units.cuh"

namespace fs {

struct RkTime {
  double j0, i0;  // centre in index units: x0 = x_min + j0 hx, y0 = y_min + i0 hy, in [0, n)
  double amp;     // A cos(gamma tau)
};

struct RkSrcParams {
  const RkTime *times;  // device table of time points
  int j_first;          // time point of block 0
  double qx, qy;        // (hx/sigma)^2, (hy/sigma)^2: exponent per squared index distance
  void *gx, *gy;        // tables [points][M+1] and [points][ny], point 0 = j_first
};

// x factor at one time point (amplitude folded in).  FP32: the index distance
// x - j0 is (x - j0_hi) - j0_lo, the first difference exact, so the distance
// keeps its relative accuracy near the centre.
template <typename T>
struct OrbitGenX;

template <>
struct OrbitGenX<float> {
  float j0h, j0l, qx, amp, nxf;
  __device__ OrbitGenX(const RkTime &tm, double q, int nx) {
    split_double(tm.j0, j0h, j0l);
    qx = (float)q;
    amp = (float)tm.amp;
    nxf = (float)nx;
  }
  __device__ float at(int x) const {
    float d = __fsub_rn(__fsub_rn((float)x, j0h), j0l);
    d = d >= 0.5f * nxf ? d - nxf : (d < -0.5f * nxf ? d + nxf : d);  // into [-n/2, n/2)
    return amp * expf(-(d * d) * qx);
  }
  __device__ cx<float> pair(int, int x) const { return mk<float>(at(x), at(x + 1)); }
};

template <>
struct OrbitGenX<double> {
  double j0, qx, amp, nxd;
  __device__ OrbitGenX(const RkTime &tm, double q, int nx) : j0(tm.j0), qx(q), amp(tm.amp), nxd(nx) {}
  __device__ double at(int x) const {
    double d = (double)x - j0;
    d = d >= 0.5 * nxd ? d - nxd : (d < -0.5 * nxd ? d + nxd : d);
    return amp * exp(-(d * d) * qx);
  }
  __device__ cx<double> pair(int, int x) const { return mk<double>(at(x), at(x + 1)); }
};

__device__ __forceinline__ float orbit_gy(const RkTime &tm, double q, int ny, int y, float) {
  float i0h, i0l;
  split_double(tm.i0, i0h, i0l);
  const float n = (float)ny;
  float d = __fsub_rn(__fsub_rn((float)y, i0h), i0l);
  d = d >= 0.5f * n ? d - n : (d < -0.5f * n ? d + n : d);
  return expf(-(d * d) * (float)q);
}
__device__ __forceinline__ double orbit_gy(const RkTime &tm, double q, int ny, int y, double) {
  double d = (double)y - tm.i0;
  d = d >= 0.5 * ny ? d - ny : (d < -0.5 * ny ? d + ny : d);
  return exp(-(d * d) * q);
}

// Gx of time point j_first + blockIdx.x: the real transform of one row of
// length nx (the row unit with a one-row spectrum), written to gx[blockIdx.x].
template <typename T, int E>
__device__ __forceinline__ void rk4_gx_body(const Desc &d, const RkSrcParams &p, cx<T> *sm) {
  const int j = blockIdx.x;
  const OrbitGenX<T> g(p.times[p.j_first + j], p.qx, d.nx);
  Desc d1 = d;
  d1.ny = 1;  // spectrum [M+1][1]
  unit_row_r2c_t<T, E, 0, 0, OrbitGenX<T>>(d1, 0, 1, sm, nullptr,
                                           reinterpret_cast<cx<T> *>(p.gx) + (size_t)j * (d.M + 1), &g);
}

// Gy of time point j_first + blockIdx.x: the complex transform of length ny of
// exp(-dy^2/sigma^2), written to gy[blockIdx.x] in natural order.
template <typename T, int E>
__device__ __forceinline__ void rk4_gy_body(const Desc &d, const RkSrcParams &p, cx<T> *sm) {
  const int j = blockIdx.x, L = d.ny, Tseg = L / E;
  const int t = threadIdx.x;
  const bool active = t < Tseg;
  const RkTime tm = p.times[p.j_first + j];
  cx<T> u[E];
#pragma unroll
  for (int s = 0; s < E; ++s) u[s] = active ? mk<T>(orbit_gy(tm, p.qy, L, t + Tseg * s, T(0)), T(0)) : zero_cx<T>();
  fft_any<T, E, 0, 1, 1>(u, sm, XLayout{0, 1}, active, t, Tseg, L, d.rp_col, reinterpret_cast<const cx<T> *>(d.tw_y));
  if (active) {
    cx<T> *dst = reinterpret_cast<cx<T> *>(p.gy) + (size_t)j * L;
#pragma unroll
    for (int s = 0; s < E; ++s) dst[t + Tseg * s] = u[s];
  }
}

typedef void (*Rk4Kernel)(const Desc, const RkSrcParams);

#define FS_RK4_DECL(T, E)                                                    \
  __global__ void k_rk4gx_##T##_##E(const Desc d, const RkSrcParams p);      \
  __global__ void k_rk4gy_##T##_##E(const Desc d, const RkSrcParams p);

#define FS_RK4_DEF(T, E)                                                                        \
  __global__ void __launch_bounds__(512) k_rk4gx_##T##_##E(const Desc d, const RkSrcParams p) { \
    extern __shared__ __align__(16) unsigned char fs_smem[];                                    \
    rk4_gx_body<T, E>(d, p, reinterpret_cast<cx<T> *>(fs_smem));                                \
  }                                                                                             \
  __global__ void __launch_bounds__(512) k_rk4gy_##T##_##E(const Desc d, const RkSrcParams p) { \
    extern __shared__ __align__(16) unsigned char fs_smem[];                                    \
    rk4_gy_body<T, E>(d, p, reinterpret_cast<cx<T> *>(fs_smem));                                \
  }

FS_FOR_EACH_E_float(FS_RK4_DECL)
FS_FOR_EACH_E_double(FS_RK4_DECL)

#define FS_RK4_CASE(T, E) \
  case E:                 \
    return x_axis ? k_rk4gx_##T##_##E : k_rk4gy_##T##_##E;
template <typename T>
inline Rk4Kernel rk4_kernel(int e, bool x_axis);
template <>
inline Rk4Kernel rk4_kernel<float>(int e, bool x_axis) {
  switch (e) { FS_FOR_EACH_E_float(FS_RK4_CASE) default: return nullptr; }
}
template <>
inline Rk4Kernel rk4_kernel<double>(int e, bool x_axis) {
  switch (e) { FS_FOR_EACH_E_double(FS_RK4_CASE) default: return nullptr; }
}

}  // namespace fs
