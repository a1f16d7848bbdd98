// fs_tune.cu -- autotuner for the standalone passes of a grid, and its cache.
//
// For an (nx, ny, dtype) grid the tuner times candidate configurations of the
// three-pass Poisson solve on this GPU with CUDA events: the register tile of
// the row and column transforms (which fixes their radix split) and the row
// tile height / column group width.  Rows are tuned first (columns at their
// default), then columns with the best rows; the result replaces the default
// only if it is faster.  Results live in a process-wide cache keyed by (GPU
// name, nx, ny, dtype) that fs_plan_create consults; the cache can be saved to
// and loaded from a JSON-lines file (FS_TUNE_CACHE names one that is loaded
// on first use).  Grids that take the single-kernel small path are not tuned.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "fs_host.h"
#include "fs_kernels.cuh"

using namespace fs;

namespace {

typedef std::tuple<std::string, int, int, int, int> Key;  // GPU name, nx, ny, dtype, mode
struct Entry {
  TuneCfg cfg;
  double us;
};
std::mutex g_mu;
std::map<Key, Entry> g_cache;
bool g_env_loaded = false;

// device name, looked up once per device (cudaGetDeviceProperties is slow);
// called with g_mu held
std::string gpu_name(int device) {
  static std::map<int, std::string> names;
  auto it = names.find(device);
  if (it != names.end()) return it->second;
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return "unknown";
  return names[device] = prop.name;
}

// "key": number from a JSON line (false if absent)
bool field_num(const std::string &line, const char *key, double *v) {
  const std::string k = std::string("\"") + key + "\"";
  size_t p = line.find(k);
  if (p == std::string::npos) return false;
  p = line.find(':', p + k.size());
  if (p == std::string::npos) return false;
  char *end = nullptr;
  *v = strtod(line.c_str() + p + 1, &end);
  return end != line.c_str() + p + 1;
}
bool field_str(const std::string &line, const char *key, std::string *v) {
  const std::string k = std::string("\"") + key + "\"";
  size_t p = line.find(k);
  if (p == std::string::npos) return false;
  p = line.find(':', p + k.size());
  if (p == std::string::npos) return false;
  const size_t a = line.find('"', p + 1);
  if (a == std::string::npos) return false;
  const size_t b = line.find('"', a + 1);
  if (b == std::string::npos) return false;
  *v = line.substr(a + 1, b - a - 1);
  return true;
}

// load a JSON-lines cache; returns entries read, -1 if the file cannot be read
int load_locked(const char *path) {
  FILE *f = fopen(path, "r");
  if (!f) return -1;
  int n = 0;
  char buf[1024];
  while (fgets(buf, sizeof buf, f)) {
    const std::string line(buf);
    std::string gpu;
    double nx, ny, dt, er, ec, rows, cols, us = 0.0, mode = 0.0;
    if (!field_str(line, "gpu", &gpu) || !field_num(line, "nx", &nx) || !field_num(line, "ny", &ny) ||
        !field_num(line, "dtype", &dt) || !field_num(line, "e_row", &er) || !field_num(line, "e_col", &ec) ||
        !field_num(line, "rows", &rows) || !field_num(line, "cols", &cols))
      continue;  // not an entry
    field_num(line, "us", &us);
    field_num(line, "mode", &mode);  // absent: standalone
    Entry e{{(int)er, (int)ec, (int)rows, (int)cols}, us};
    g_cache[Key(gpu, (int)nx, (int)ny, (int)dt, (int)mode)] = e;
    ++n;
  }
  fclose(f);
  return n;
}

int save_locked(const char *path) {
  FILE *f = fopen(path, "w");
  if (!f) return -1;
  int n = 0;
  for (const auto &kv : g_cache) {
    const Key &k = kv.first;
    const Entry &e = kv.second;
    fprintf(f,
            "{\"gpu\": \"%s\", \"nx\": %d, \"ny\": %d, \"dtype\": %d, \"mode\": %d, \"e_row\": %d, "
            "\"e_col\": %d, \"rows\": %d, \"cols\": %d, \"us\": %.3f}\n",
            std::get<0>(k).c_str(), std::get<1>(k), std::get<2>(k), std::get<3>(k), std::get<4>(k), e.cfg.e_row,
            e.cfg.e_col, e.cfg.rows, e.cfg.cols, e.us);
    ++n;
  }
  fclose(f);
  return n;
}

void env_load_locked() {
  if (g_env_loaded) return;
  g_env_loaded = true;
  if (const char *p = getenv("FS_TUNE_CACHE")) load_locked(p);
}

// mean time of one Poisson solve (us) with a forced configuration; <0 if the
// configuration cannot be built or run
double time_cfg(int nx, int ny, double lx, double ly, int dtype, const TuneCfg &c, void *f, void *u,
                cudaStream_t s, int reps, bool *small) {
  fs_plan p = nullptr;
  if (plan_create_cfg(nx, ny, lx, ly, dtype, &c, &p) != FS_OK) return -1.0;
  if (small) *small = p->standalone_small;
  double us = -1.0;
  cudaEvent_t a = nullptr, b = nullptr;
  if (cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess) {
    bool ok = true;
    for (int i = 0; i < 2 && ok; ++i) ok = fs_poisson_solve(p, f, u, s) == FS_OK;
    if (ok) {
      cudaEventRecord(a, s);
      for (int i = 0; i < reps && ok; ++i) ok = fs_poisson_solve(p, f, u, s) == FS_OK;
      cudaEventRecord(b, s);
      float ms = 0.f;
      if (ok && cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess)
        us = 1e3 * ms / reps;
    }
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  cudaStreamSynchronize(s);
  fs_plan_destroy(p);
  return us;
}

}  // namespace

// candidate forced on the batch planner by fs_tune_batch (this thread only)
thread_local const TuneCfg *t_force_batch = nullptr;

bool fs::tune_lookup(int device, int nx, int ny, int dtype, int mode, TuneCfg *out) {
  if (mode == 1 && t_force_batch) {
    *out = *t_force_batch;
    return true;
  }
  std::lock_guard<std::mutex> g(g_mu);
  env_load_locked();
  if (g_cache.empty()) return false;
  auto it = g_cache.find(Key(gpu_name(device), nx, ny, dtype, mode));
  if (it == g_cache.end()) return false;
  *out = it->second.cfg;
  return true;
}

extern "C" {

fs_status fs_tune(int nx, int ny, double lx, double ly, int dtype, int reps, fs_tune_result *res) {
  if (!res) return set_error(FS_ERR_ARG, "fs_tune: result is NULL");
  memset(res, 0, sizeof *res);
  if (reps < 1) reps = 10;
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return cuda_error(e, "fs_tune");
  const size_t es = dtype == FS_F64 ? sizeof(double) : sizeof(float);
  void *f = nullptr, *u = nullptr;
  cudaStream_t s = nullptr;
  e = cudaMalloc(&f, (size_t)nx * ny * es);
  if (e == cudaSuccess) e = cudaMalloc(&u, (size_t)nx * ny * es);
  if (e == cudaSuccess) e = cudaMemset(f, 0x3c, (size_t)nx * ny * es);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaFree(f);
    cudaFree(u);
    return cuda_error(e, "fs_tune: buffers");
  }
  const TuneCfg none{0, 0, 0, 0};
  bool small = false;
  const double us_default = time_cfg(nx, ny, lx, ly, dtype, none, f, u, s, reps, &small);
  TuneCfg best = none;
  double us_best = us_default;
  int cand = 1;
  fs_status st = FS_OK;
  if (us_default < 0.0) {
    st = set_error(FS_ERR_SIZE, "fs_tune: the default configuration does not run");
  } else if (!small) {
    static const int es_f[] = {4, 5, 6, 8, 10, 12, 16, 20, 24}, es_d[] = {4, 5, 6, 8, 10, 12, 16};
    const int *elist = dtype == FS_F64 ? es_d : es_f;
    const int ne = dtype == FS_F64 ? 7 : 9;
    const bool f64 = dtype == FS_F64;
    // rows: register tile x tile height (columns at their default)
    TuneCfg best_r = none;
    double us_r = us_default;
    for (int i = 0; i < ne; ++i) {
      RadixPlan rp;
      if (!make_rp_e(nx / 2, elist[i], f64, &rp)) continue;
      for (int rows = 1; rows <= 16; rows *= 2) {
        const TuneCfg c{elist[i], 0, rows, 0};
        const double us = time_cfg(nx, ny, lx, ly, dtype, c, f, u, s, reps, nullptr);
        if (us < 0.0) continue;
        ++cand;
        if (us < us_r) {
          us_r = us;
          best_r = c;
        }
      }
    }
    // columns: register tile x group width, with the best rows
    TuneCfg best_c = best_r;
    double us_c = us_r;
    for (int i = 0; i < ne; ++i) {
      RadixPlan rp;
      if (!make_rp_e(ny, elist[i], f64, &rp)) continue;
      for (int cols = 1; cols <= 32; cols *= 2) {
        const TuneCfg c{best_r.e_row, elist[i], best_r.rows, cols};
        const double us = time_cfg(nx, ny, lx, ly, dtype, c, f, u, s, reps, nullptr);
        if (us < 0.0) continue;
        ++cand;
        if (us < us_c) {
          us_c = us;
          best_c = c;
        }
      }
    }
    best = best_c;
    us_best = us_c;
  }
  cudaStreamDestroy(s);
  cudaFree(f);
  cudaFree(u);
  if (st != FS_OK) return st;
  // an unset field keeps the default; store the full configuration
  fs_plan p = nullptr;
  if (plan_create_cfg(nx, ny, lx, ly, dtype, &best, &p) == FS_OK) {
    res->e_row = p->rp_row.e;
    res->e_col = p->rp_col.e;
    res->rows = p->tc.rows_per_unit;
    res->cols = p->tc.cols_per_unit;
    fs_plan_destroy(p);
  }
  res->us_default = us_default;
  res->us_tuned = us_best;
  res->candidates = cand;
  {
    std::lock_guard<std::mutex> g(g_mu);
    env_load_locked();
    g_cache[Key(gpu_name(device), nx, ny, dtype, 0)] =
        Entry{{res->e_row, res->e_col, res->rows, res->cols}, us_best};
    if (const char *path = getenv("FS_TUNE_CACHE")) save_locked(path);
  }
  return FS_OK;
}

fs_status fs_tune_batch(int nx, int ny, double lx, double ly, int dtype, int nprob, int reps, fs_tune_result *res) {
  if (!res) return set_error(FS_ERR_ARG, "fs_tune_batch: result is NULL");
  memset(res, 0, sizeof *res);
  if (reps < 1) reps = 5;
  if (nprob < 1) nprob = 8;
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e != cudaSuccess) return cuda_error(e, "fs_tune_batch");
  fs_plan p = nullptr;
  fs_status st = plan_create_cfg(nx, ny, lx, ly, dtype, nullptr, &p);
  if (st != FS_OK) return st;
  const size_t bytes = (size_t)nx * ny * (dtype == FS_F64 ? sizeof(double) : sizeof(float));
  void *f = nullptr, *u = nullptr;
  cudaStream_t s = nullptr;
  e = cudaMalloc(&f, bytes);
  if (e == cudaSuccess) e = cudaMalloc(&u, bytes * (size_t)nprob);
  if (e == cudaSuccess) e = cudaMemset(f, 0x3c, bytes);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    cudaFree(f);
    cudaFree(u);
    fs_plan_destroy(p);
    return cuda_error(e, "fs_tune_batch: buffers");
  }
  std::vector<fs_request> reqs(nprob);
  for (int i = 0; i < nprob; ++i) {
    memset(&reqs[i], 0, sizeof(fs_request));
    reqs[i].op = FS_OP_POISSON;
    reqs[i].plan = p;
    reqs[i].in_u = f;
    reqs[i].out_u = static_cast<char *>(u) + bytes * (size_t)i;
  }
  auto time_batch = [&](const TuneCfg *c) -> double {
    t_force_batch = c;
    double us = -1.0;
    cudaEvent_t a = nullptr, b = nullptr;
    bool ok = cudaEventCreate(&a) == cudaSuccess && cudaEventCreate(&b) == cudaSuccess;
    uint64_t tk = 0;
    for (int i = 0; i < 2 && ok; ++i)  // warm-up (graph capture)
      ok = fs_batch_submit(reqs.data(), nprob, &tk, s) == FS_OK && fs_batch_wait(tk, 60000000) == FS_OK;
    if (ok) {
      cudaEventRecord(a, s);
      for (int i = 0; i < reps && ok; ++i) ok = fs_batch_submit(reqs.data(), nprob, &tk, s) == FS_OK;
      cudaEventRecord(b, s);
      float ms = 0.f;
      if (ok && cudaEventSynchronize(b) == cudaSuccess && cudaEventElapsedTime(&ms, a, b) == cudaSuccess)
        us = 1e3 * ms / reps;
      if (ok) fs_batch_wait(tk, 60000000);
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaStreamSynchronize(s);
    t_force_batch = nullptr;
    return us;
  };
  const TuneCfg none{0, 0, 0, 0};
  const double us_default = time_batch(&none);
  TuneCfg best = none;
  double us_best = us_default;
  int cand = 1;
  if (us_default < 0.0) st = set_error(FS_ERR_SIZE, "fs_tune_batch: the default configuration does not run");
  static const int es_f[] = {4, 5, 6, 8, 10, 12, 16, 20, 24}, es_d[] = {4, 5, 6, 8, 10, 12, 16};
  const int *elist = dtype == FS_F64 ? es_d : es_f;
  const int ne = dtype == FS_F64 ? 7 : 9;
  for (int i = 0; i < ne && st == FS_OK; ++i) {
    RadixPlan rr;
    if (!make_rp_e(nx / 2, elist[i], dtype == FS_F64, &rr)) continue;
    for (int j = 0; j < ne; ++j) {
      RadixPlan rc;
      if (!make_rp_e(ny, elist[j], dtype == FS_F64, &rc)) continue;
      if (rr.e == p->rp_row.e && rc.e == p->rp_col.e) continue;  // the default, timed above
      const TuneCfg c{elist[i], elist[j], 0, 0};
      const double us = time_batch(&c);
      if (us < 0.0) continue;
      ++cand;
      if (us < us_best) {
        us_best = us;
        best = c;
      }
    }
  }
  cudaStreamDestroy(s);
  cudaFree(f);
  cudaFree(u);
  res->e_row = best.e_row ? best.e_row : p->rp_row.e;
  res->e_col = best.e_col ? best.e_col : p->rp_col.e;
  fs_plan_destroy(p);
  if (st != FS_OK) return st;
  res->us_default = us_default;
  res->us_tuned = us_best;
  res->candidates = cand;
  std::lock_guard<std::mutex> g(g_mu);
  env_load_locked();
  g_cache[Key(gpu_name(device), nx, ny, dtype, 1)] = Entry{{res->e_row, res->e_col, 0, 0}, us_best};
  if (const char *path = getenv("FS_TUNE_CACHE")) save_locked(path);
  return FS_OK;
}

int fs_tune_cache_load(const char *path) {
  if (!path) return -1;
  std::lock_guard<std::mutex> g(g_mu);
  return load_locked(path);
}

int fs_tune_cache_save(const char *path) {
  if (!path) return -1;
  std::lock_guard<std::mutex> g(g_mu);
  return save_locked(path);
}

int fs_tune_cache_clear(void) {
  std::lock_guard<std::mutex> g(g_mu);
  const int n = (int)g_cache.size();
  g_cache.clear();
  g_env_loaded = true;  // an explicit clear also drops the environment's file
  return n;
}

}  // extern "C"
