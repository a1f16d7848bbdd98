// fs_rk4_api.cu -- host side of the RK4 wave integration with an orbiting
// source (Sec. III.C, example with source; kernels in fs_rk4.cuh).
//
// The integrator owns the half spectra U, V (held in an fs_state_s so that
// outputs reuse the wave-advance path at t = 0, i.e. a plain inverse
// transform), the kept source spectrum S(t) and two row-transform buffers.
// fs_rk4_step writes the per-step source table (centre in index units and
// amplitude at t + dt/2 and t + dt) and replays a CUDA graph of the 2 x nsteps
// launches, captured once per (step count, dt).
#include <cmath>
#include <map>
#include <utility>
#include <new>
#include <vector>

#include "fs_host.h"
#include "fs_kernels.cuh"
#include "fs_rk4.cuh"

using namespace fs;

struct fs_rk4_s {
  fs_plan plan;
  double c, t;
  fs_orbit_source src;
  fs_state_s st;  // su = U, sv = V
  void *S0, *wa, *wb;
  RkStep *d_steps;
  int cap;
  std::vector<RkStep> h_steps;
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

RkParams params(const fs_rk4_s *r, int step, int init) {
  const fs_plan_s *p = r->plan;
  const double hx = p->lx / p->nx, hy = p->ly / p->ny, sg = r->src.sigma;
  RkParams q;
  q.steps = r->d_steps;
  q.step = step;
  q.init = init;
  q.qx = (hx / sg) * (hx / sg);
  q.qy = (hy / sg) * (hy / sg);
  q.dt = 0.0;
  q.c2 = r->c * r->c;
  q.U = r->st.su;
  q.V = r->st.sv;
  q.S0 = r->S0;
  q.wa = r->wa;
  q.wb = r->wb;
  return q;
}

template <typename T>
cudaError_t launch_step(const fs_rk4_s *r, const RkParams &q, cudaStream_t s) {
  const Desc d = base_desc(r->plan);
  Rk4Kernel kr = rk4_kernel<T>(d.rp_row.e, true), kc = rk4_kernel<T>(d.rp_col.e, false);
  if (!kr || !kc) return cudaErrorInvalidConfiguration;
  const size_t rs = Launch<T>::row_smem(d), cs = Launch<T>::col_smem(d);
  cudaError_t e = Launch<T>::set_smem((const void *)kr, rs);
  if (e == cudaSuccess) e = Launch<T>::set_smem((const void *)kc, cs);
  if (e != cudaSuccess) return e;
  kr<<<d.n_row_units * (q.init ? 1 : 2), Launch<T>::row_threads(d), rs, s>>>(d, q);
  kc<<<d.n_col_units, Launch<T>::col_threads(d), cs, s>>>(d, q);
  return cudaGetLastError();
}

cudaError_t launch(const fs_rk4_s *r, const RkParams &q, cudaStream_t s) {
  return r->plan->dtype == FS_F64 ? launch_step<double>(r, q, s) : launch_step<float>(r, q, s);
}

void drop_graphs(fs_rk4_s *r) {
  for (auto &g : r->graphs) cudaGraphExecDestroy(g.second);
  r->graphs.clear();
}

fs_status ensure_table(fs_rk4_s *r, int n) {
  if (n <= r->cap) return FS_OK;
  drop_graphs(r);  // graphs hold the old table's address
  cudaFree(r->d_steps);
  r->d_steps = nullptr;
  r->cap = 0;
  cudaError_t e = cudaMalloc(&r->d_steps, (size_t)n * sizeof(RkStep));
  if (e != cudaSuccess) return cuda_error(e, "fs_rk4: step table allocation");
  r->cap = n;
  return FS_OK;
}

void release(fs_rk4_s *r) {
  drop_graphs(r);
  cudaFree(r->st.su);
  cudaFree(r->st.sv);
  cudaFree(r->S0);
  cudaFree(r->wa);
  cudaFree(r->wb);
  cudaFree(r->d_steps);
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
  void **bufs[5] = {&r->st.su, &r->st.sv, &r->S0, &r->wa, &r->wb};
  cudaError_t e = cudaSuccess;
  for (void **b : bufs)
    if (e == cudaSuccess) e = cudaMalloc(b, p->spec_bytes);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&r->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    release(r);
    return cuda_error(e, "fs_rk4_create: device allocation");
  }
  fs_status st = ensure_table(r, 1);
  if (st != FS_OK) {
    release(r);
    return st;
  }
  // initial data
  if (u0) {
    st = forward_into(p, u0, v0, r->st.su, v0 ? r->st.sv : nullptr, stream, "fs_rk4_create");
  } else {
    e = cudaMemsetAsync(r->st.su, 0, p->spec_bytes, s);
    st = e == cudaSuccess ? FS_OK : cuda_error(e, "fs_rk4_create");
    if (st == FS_OK && v0) st = forward_into(p, v0, nullptr, r->st.sv, nullptr, stream, "fs_rk4_create");
  }
  if (st == FS_OK && !v0) {
    e = cudaMemsetAsync(r->st.sv, 0, p->spec_bytes, s);
    if (e != cudaSuccess) st = cuda_error(e, "fs_rk4_create");
  }
  // S(t0): the source at t0 through the RK4 row / column kernels (init mode)
  if (st == FS_OK) {
    RkStep first;
    first.mid = source_at(r, t0);
    first.end = first.mid;
    e = cudaMemcpyAsync(r->d_steps, &first, sizeof first, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = launch(r, params(r, 0, 1), s);
    if (e == cudaSuccess) g_launches.fetch_add(2, std::memory_order_relaxed);
    // `first` is pageable: the copy has been staged when cudaMemcpyAsync returns
    if (e != cudaSuccess) st = cuda_error(e, "fs_rk4_create: source transform");
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
  fs_status st = ensure_table(r, nsteps);
  if (st != FS_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // step k runs from t_k = t + k dt; stage times t_k + dt/2 and t_k + dt
  r->h_steps.resize(nsteps);
  for (int k = 0; k < nsteps; ++k) {
    const double tk = r->t + k * dt;
    r->h_steps[k].mid = source_at(r, tk + 0.5 * dt);
    r->h_steps[k].end = source_at(r, tk + dt);
  }
  // pageable source: ordered after earlier work on the stream, and staged
  // before the call returns (the host vector may be reused afterwards)
  cudaError_t e = cudaMemcpyAsync(r->d_steps, r->h_steps.data(), (size_t)nsteps * sizeof(RkStep),
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_error(e, "fs_rk4_step: step table upload");
  // the graph bakes dt and the table address into its launches
  const std::pair<int, double> key(nsteps, dt);
  auto it = r->graphs.find(key);
  cudaGraphExec_t gx = it != r->graphs.end() ? it->second : nullptr;
  if (!gx) {
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(r->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaError_t le = cudaSuccess;
      for (int k = 0; k < nsteps && le == cudaSuccess; ++k) {
        RkParams q = params(r, k, 0);
        q.dt = dt;
        le = launch(r, q, r->cap_stream);
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
  g_launches.fetch_add(2ULL * (unsigned long long)nsteps, std::memory_order_relaxed);
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
