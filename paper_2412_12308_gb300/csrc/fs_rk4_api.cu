// fs_rk4_api.cu -- RK4 wave integration with an orbiting source (Sec. III.C,
// example with source): the mode-parallel RK4 kernel and the host API.
//
// The integrator owns the half spectra U, V (held in an fs_state_s so that
// outputs reuse the wave-advance path at t = 0, i.e. a plain inverse
// transform) and, per chunk of at most kChunk steps, tables of the 1D source
// spectra Gx, Gy at the chunk's 2 n + 1 stage times (fs_rk4.cuh).  A chunk is
// three launches: Gx (one CTA per time point), Gy (likewise), then
// k_rk4_modes, where every thread takes modes (a, b), loads U and V once, runs
// all steps of the chunk in registers with S = Gx(a) Gy(b) at each stage time
// and stores U and V once.  fs_rk4_step uploads the time-point table and
// replays a CUDA graph of the chunks, captured once per (step count, dt).
#include <cmath>
#include <map>
#include <new>
#include <utility>
#include <vector>

#include "fs_host.h"
#include "fs_kernels.cuh"
#include "fs_rk4.cuh"

using namespace fs;

namespace fs {

constexpr int kChunk = 128;  // steps per chunk (tables of 2 kChunk + 1 time points)

struct RkModes {
  void *U, *V;
  const void *gx, *gy;  // chunk tables; point 0 = the chunk's start time
  int nsteps;
  double dt, c2;
};

__device__ __forceinline__ float rk_w2(const Desc &d, int a, int b, float c2) {
  const float2 wx = reinterpret_cast<const float2 *>(d.wx2)[a];
  const float2 wy = reinterpret_cast<const float2 *>(d.wy2)[b];
  return c2 * __fadd_rn(__fadd_rn(wx.x, wy.x), __fadd_rn(wx.y, wy.y));
}
__device__ __forceinline__ double rk_w2(const Desc &d, int a, int b, double c2) {
  return c2 * (reinterpret_cast<const double *>(d.wx2)[a] + reinterpret_cast<const double *>(d.wy2)[b]);
}

// Mode (a, b) = (m / ny, m % ny) of the half spectrum; classical RK4 on
// dU/dt = V, dV/dt = S(t) - c^2 |w|^2 U with S at t_k, t_k + dt/2, t_k + dt.
template <typename T>
__global__ void __launch_bounds__(256) k_rk4_modes(const Desc d, const RkModes r) {
  const int M1 = d.M + 1, ny = d.ny;
  const long long total = (long long)M1 * ny;
  const cx<T> *gx = reinterpret_cast<const cx<T> *>(r.gx);
  const cx<T> *gy = reinterpret_cast<const cx<T> *>(r.gy);
  cx<T> *U = reinterpret_cast<cx<T> *>(r.U);
  cx<T> *V = reinterpret_cast<cx<T> *>(r.V);
  const T h = (T)r.dt, hh = (T)(0.5 * r.dt), h6 = (T)(r.dt / 6.0), c2 = (T)r.c2;
  for (long long m = (long long)blockIdx.x * blockDim.x + threadIdx.x; m < total;
       m += (long long)gridDim.x * blockDim.x) {
    const int a = (int)(m / ny), b = (int)(m - (long long)a * ny);
    const T w2 = rk_w2(d, a, b, c2);
    cx<T> u = U[m], v = V[m];
    cx<T> s0 = cmul(gx[a], gy[b]);
#pragma unroll 2
    for (int k = 0; k < r.nsteps; ++k) {
      const size_t jm = 2 * (size_t)k + 1, je = jm + 1;
      const cx<T> smid = cmul(gx[jm * M1 + a], gy[jm * ny + b]);
      const cx<T> s1 = cmul(gx[je * M1 + a], gy[je * ny + b]);
      const cx<T> k1u = v, k1v = s0 - w2 * u;
      const cx<T> k2u = v + hh * k1v, k2v = smid - w2 * (u + hh * k1u);
      const cx<T> k3u = v + hh * k2v, k3v = smid - w2 * (u + hh * k2u);
      const cx<T> k4u = v + h * k3v, k4v = s1 - w2 * (u + h * k3u);
      u = u + h6 * (k1u + T(2) * (k2u + k3u) + k4u);
      v = v + h6 * (k1v + T(2) * (k2v + k3v) + k4v);
      s0 = s1;
    }
    U[m] = u;
    V[m] = v;
  }
}

}  // namespace fs

struct fs_rk4_s {
  fs_plan plan;
  double c, t;
  fs_orbit_source src;
  fs_state_s st;  // su = U, sv = V
  void *gx, *gy;  // chunk tables
  RkTime *d_times;
  int cap;        // time points d_times holds
  std::vector<RkTime> h_times;
  cudaStream_t cap_stream;
  std::map<std::pair<int, double>, cudaGraphExec_t> graphs;  // by (step count, dt)
};

namespace {

double reduce_index(double v, int n) {
  double r = std::fmod(v, (double)n);
  if (r < 0.0) r += n;
  if (r >= n) r -= n;
  return r;
}

RkTime source_at(const fs_rk4_s *r, double tau) {
  const fs_plan_s *p = r->plan;
  const double hx = p->lx / p->nx, hy = p->ly / p->ny;
  const double x0 = r->src.radius * std::cos(r->src.Omega * tau);
  const double y0 = r->src.radius * std::sin(r->src.Omega * tau);
  RkTime tm;
  tm.j0 = reduce_index((x0 - r->src.x_min) / hx, p->nx);
  tm.i0 = reduce_index((y0 - r->src.y_min) / hy, p->ny);
  tm.amp = r->src.A * std::cos(r->src.gamma * tau);
  return tm;
}

template <typename T>
cudaError_t launch_chunk(const fs_rk4_s *r, int j_first, int nsteps, double dt, cudaStream_t s) {
  const Desc d = base_desc(r->plan);
  Rk4Kernel kx = rk4_kernel<T>(d.rp_row.e, true), ky = rk4_kernel<T>(d.rp_col.e, false);
  if (!kx || !ky) return cudaErrorInvalidConfiguration;
  const fs_plan_s *p = r->plan;
  const double hx = p->lx / p->nx, hy = p->ly / p->ny, sg = r->src.sigma;
  RkSrcParams q;
  q.times = r->d_times;
  q.j_first = j_first;
  q.qx = (hx / sg) * (hx / sg);
  q.qy = (hy / sg) * (hy / sg);
  q.gx = r->gx;
  q.gy = r->gy;
  const int points = 2 * nsteps + 1;
  const size_t sx = sizeof(cx<T>) * (size_t)padded_len(d.M), sy = sizeof(cx<T>) * (size_t)padded_len(d.ny);
  cudaError_t e = Launch<T>::set_smem((const void *)kx, sx);
  if (e == cudaSuccess) e = Launch<T>::set_smem((const void *)ky, sy);
  if (e != cudaSuccess) return e;
  kx<<<points, round_up32(d.M / d.rp_row.e), sx, s>>>(d, q);
  ky<<<points, round_up32(d.ny / d.rp_col.e), sy, s>>>(d, q);
  RkModes m;
  m.U = r->st.su;
  m.V = r->st.sv;
  m.gx = r->gx;
  m.gy = r->gy;
  m.nsteps = nsteps;
  m.dt = dt;
  m.c2 = r->c * r->c;
  const long long modes = (long long)(d.M + 1) * d.ny;
  int sms = 0, dev = 0, per_sm = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_rk4_modes<T>, 256, 0);
  if (e != cudaSuccess) return e;
  long long grid = (modes + 255) / 256;
  const long long cap = (long long)sms * (per_sm > 0 ? per_sm : 1);
  if (grid > cap) grid = cap;
  k_rk4_modes<T><<<(int)grid, 256, 0, s>>>(d, m);
  return cudaGetLastError();
}

cudaError_t launch_chunk(const fs_rk4_s *r, int j_first, int nsteps, double dt, cudaStream_t s) {
  return r->plan->dtype == FS_F64 ? launch_chunk<double>(r, j_first, nsteps, dt, s)
                                  : launch_chunk<float>(r, j_first, nsteps, dt, s);
}

void drop_graphs(fs_rk4_s *r) {
  for (auto &g : r->graphs) cudaGraphExecDestroy(g.second);
  r->graphs.clear();
}

fs_status ensure_times(fs_rk4_s *r, int points) {
  if (points <= r->cap) return FS_OK;
  drop_graphs(r);  // graphs hold the old table's address
  cudaFree(r->d_times);
  r->d_times = nullptr;
  r->cap = 0;
  cudaError_t e = cudaMalloc(&r->d_times, (size_t)points * sizeof(RkTime));
  if (e != cudaSuccess) return cuda_error(e, "fs_rk4: time table allocation");
  r->cap = points;
  return FS_OK;
}

void release(fs_rk4_s *r) {
  drop_graphs(r);
  cudaFree(r->st.su);
  cudaFree(r->st.sv);
  cudaFree(r->gx);
  cudaFree(r->gy);
  cudaFree(r->d_times);
  if (r->cap_stream) cudaStreamDestroy(r->cap_stream);
  delete r;
}

}  // namespace

extern "C" {

fs_status fs_rk4_create(fs_plan p, double c, const fs_orbit_source *src, const void *u0, const void *v0,
                        double t0, fs_stream stream, fs_rk4 *out) {
  if (!out) return set_error(FS_ERR_ARG, "fs_rk4_create: out is NULL");
  *out = nullptr;
  if (!p || !src) return set_error(FS_ERR_ARG, "fs_rk4_create: NULL argument");
  if (!(c > 0.0) || !std::isfinite(c) || !std::isfinite(t0))
    return set_error(FS_ERR_ARG, "fs_rk4_create: need finite c > 0 and finite t0");
  if (!(src->sigma > 0.0) || !std::isfinite(src->A) || !std::isfinite(src->radius) ||
      !std::isfinite(src->Omega) || !std::isfinite(src->gamma) || !std::isfinite(src->x_min) ||
      !std::isfinite(src->y_min) || !std::isfinite(src->sigma))
    return set_error(FS_ERR_ARG, "fs_rk4_create: source parameters must be finite, sigma > 0");
  fs_rk4_s *r = new (std::nothrow) fs_rk4_s();
  if (!r) return set_error(FS_ERR_NOMEM, "fs_rk4_create: host allocation");
  r->plan = p;
  r->c = c;
  r->t = t0;
  r->src = *src;
  r->st.plan = p;
  r->st.has_v = true;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t points = 2 * kChunk + 1;
  cudaError_t e = cudaMalloc(&r->st.su, p->spec_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&r->st.sv, p->spec_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&r->gx, points * (size_t)(p->M + 1) * p->csize);
  if (e == cudaSuccess) e = cudaMalloc(&r->gy, points * (size_t)p->ny * p->csize);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&r->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    release(r);
    return cuda_error(e, "fs_rk4_create: device allocation");
  }
  // initial data
  fs_status st = FS_OK;
  if (u0) {
    st = forward_into(p, u0, v0, r->st.su, v0 ? r->st.sv : nullptr, stream, "fs_rk4_create");
  } else {
    e = cudaMemsetAsync(r->st.su, 0, p->spec_bytes, s);
    if (e != cudaSuccess) st = cuda_error(e, "fs_rk4_create");
    if (st == FS_OK && v0) st = forward_into(p, v0, nullptr, r->st.sv, nullptr, stream, "fs_rk4_create");
  }
  if (st == FS_OK && !v0) {
    e = cudaMemsetAsync(r->st.sv, 0, p->spec_bytes, s);
    if (e != cudaSuccess) st = cuda_error(e, "fs_rk4_create");
  }
  if (st != FS_OK) {
    cudaStreamSynchronize(s);
    release(r);
    return st;
  }
  *out = r;
  return FS_OK;
}

fs_status fs_rk4_step(fs_rk4 r, double dt, int nsteps, fs_stream stream) {
  if (!r) return set_error(FS_ERR_ARG, "fs_rk4_step: NULL integrator");
  if (!(dt > 0.0) || !std::isfinite(dt) || nsteps < 0)
    return set_error(FS_ERR_ARG, "fs_rk4_step: need finite dt > 0 and nsteps >= 0");
  if (nsteps == 0) return FS_OK;
  fs_status st = ensure_times(r, 2 * nsteps + 1);
  if (st != FS_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // stage times of step k from t_k = t + k dt: t_k, t_k + dt/2, t_k + dt; the
  // start of step k > 0 is the end of step k - 1
  r->h_times.resize(2 * (size_t)nsteps + 1);
  r->h_times[0] = source_at(r, r->t);
  for (int k = 0; k < nsteps; ++k) {
    const double tk = r->t + k * dt;
    r->h_times[2 * k + 1] = source_at(r, tk + 0.5 * dt);
    r->h_times[2 * k + 2] = source_at(r, tk + dt);
  }
  // pageable source: ordered after earlier work on the stream, and staged
  // before the call returns (the host vector may be reused afterwards)
  cudaError_t e = cudaMemcpyAsync(r->d_times, r->h_times.data(), r->h_times.size() * sizeof(RkTime),
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_error(e, "fs_rk4_step: time table upload");
  // the graph bakes dt, the chunking and the table addresses into its launches
  const std::pair<int, double> key(nsteps, dt);
  auto it = r->graphs.find(key);
  cudaGraphExec_t gx = it != r->graphs.end() ? it->second : nullptr;
  int launches = 0;
  for (int k0 = 0; k0 < nsteps; k0 += kChunk) launches += 3;
  if (!gx) {
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(r->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t le = cudaSuccess;
      for (int k0 = 0; k0 < nsteps && le == cudaSuccess; k0 += kChunk) {
        const int n = nsteps - k0 < kChunk ? nsteps - k0 : kChunk;
        le = launch_chunk(r, 2 * k0, n, dt, r->cap_stream);
      }
      e = cudaStreamEndCapture(r->cap_stream, &g);
      if (e == cudaSuccess && le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&gx, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_error(e, "fs_rk4_step: graph capture");
    if (r->graphs.size() >= 8) drop_graphs(r);
    r->graphs[key] = gx;
  }
  e = cudaGraphLaunch(gx, s);
  if (e != cudaSuccess) return cuda_error(e, "fs_rk4_step: graph launch");
  g_launches.fetch_add((unsigned long long)launches, std::memory_order_relaxed);
  r->t += nsteps * dt;
  return FS_OK;
}

fs_status fs_rk4_output(fs_rk4 r, void *u_out, void *v_out, fs_stream stream) {
  if (!r || !u_out) return set_error(FS_ERR_ARG, "fs_rk4_output: NULL argument");
  return fs_wave_advance(&r->st, r->c, 0.0, u_out, v_out, stream);
}

fs_status fs_rk4_mean(fs_rk4 r, double *mean_u, fs_stream stream) {
  if (!r || !mean_u) return set_error(FS_ERR_ARG, "fs_rk4_mean: NULL argument");
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const fs_plan_s *p = r->plan;
  double re = 0.0;
  cudaError_t e;
  if (p->dtype == FS_F64) {
    double z[2];
    e = cudaMemcpyAsync(z, r->st.su, sizeof z, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    re = z[0];
  } else {
    float z[2];
    e = cudaMemcpyAsync(z, r->st.su, sizeof z, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    re = z[0];
  }
  if (e != cudaSuccess) return cuda_error(e, "fs_rk4_mean");
  *mean_u = re / ((double)p->nx * (double)p->ny);
  return FS_OK;
}

fs_status fs_rk4_time(fs_rk4 r, double *t) {
  if (!r || !t) return set_error(FS_ERR_ARG, "fs_rk4_time: NULL argument");
  *t = r->t;
  return FS_OK;
}

fs_status fs_rk4_destroy(fs_rk4 r) {
  if (!r) return FS_OK;
  cudaDeviceSynchronize();
  release(r);
  return FS_OK;
}

}  // extern "C"
