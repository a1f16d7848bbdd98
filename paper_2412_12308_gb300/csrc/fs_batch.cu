// fs_batch.cu -- the batch executor: many independent solves / advances in
// one persistent launch (k_batch), replayed from a CUDA graph when the batch
// shape repeats.
//
// Host side: build one Desc per request (geometry from its plan, workspace
// carved from the slot's arena), then a work table of units.  The order of
// the table is a three-stage software pipeline over chunks of problems
// (largest problems first): factor/row/small units of chunk i, column units
// of chunk i-1, C2R units of chunk i-2.  Every dependency (columns need the
// problem's rows and factors, C2R needs its columns) therefore points to an
// earlier table index, so the persistent CTAs that take indices in order
// never wait on work nobody has started, and each chunk's intermediate
// spectra are consumed while still resident in L2.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "fs_batch.h"
#include "fs_kernels.cuh"

extern template struct fs::Launch<float>;
extern template struct fs::Launch<double>;

namespace fs {

namespace {

constexpr size_t kChunkBytes = 24u << 20;     // intermediate bytes per pipeline chunk
constexpr size_t kMaxDynSmem = 227u * 1024u;  // per-CTA dynamic shared memory limit
constexpr int kMaxSlots = 3;                   // in-flight batches per device (serving keeps 3)

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

long long env_ll(const char *name, long long dflt) {
  const char *v = getenv(name);
  return v && *v ? atoll(v) : dflt;
}

struct Slot {
  int device = -1;
  cudaEvent_t ev = nullptr;
  cudaStream_t cap = nullptr;
  cudaStream_t cap2 = nullptr;                       // the small problems' branch of the graph
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;  // capture-time fork / join of that branch
  uint64_t ticket = 0;
  bool pending = false;
  Desc *d_descs = nullptr;
  int4 *d_units = nullptr;
  int *d_ctl = nullptr;
  int *d_done = nullptr;
  char *d_arena = nullptr;
  size_t cap_descs = 0, cap_units = 0, cap_arena = 0;
  Desc *h_descs = nullptr;
  int4 *h_units = nullptr;
  int *h_status = nullptr;  // ctl words of the two launches: [1] and [3] are their status
  cudaGraphExec_t gexec = nullptr;
  int key_descs = -1, key_units = -1, key_grid = -1, key_dtype = -1;
  size_t key_smem = 0;
  unsigned long long key_wait = 0;
  int key_threads = 0;
  int key_small_units = 0, key_small_grid = 0, key_small_threads = 0;
  size_t key_small_smem = 0;
};

// status of a slot's last batch: the first non-zero of its two launches
int slot_status(const Slot *s) { return s->h_status[1] != 0 ? s->h_status[1] : s->h_status[3]; }

std::mutex g_mu;
std::vector<Slot *> g_slots;
uint64_t g_next_ticket = 1;
std::deque<std::pair<uint64_t, int>> g_finished;  // recent (ticket, status)

void remember(uint64_t ticket, int status) {
  g_finished.emplace_back(ticket, status);
  while (g_finished.size() > 4096) g_finished.pop_front();
}

// Grow a device + pinned-host buffer pair (slot idle).
template <typename X>
cudaError_t grow(X **d, X **h, size_t &cap, size_t need) {
  if (need <= cap) return cudaSuccess;
  size_t n = std::max(need, cap * 2);
  cudaFree(*d);
  if (h) cudaFreeHost(*h);
  *d = nullptr;
  if (h) *h = nullptr;
  cap = 0;
  cudaError_t e = cudaMalloc((void **)d, n * sizeof(X));
  if (e == cudaSuccess && h) e = cudaMallocHost((void **)h, n * sizeof(X));
  if (e == cudaSuccess) cap = n;
  return e;
}

void drop_graph(Slot *s) {
  if (s->gexec) cudaGraphExecDestroy(s->gexec);
  s->gexec = nullptr;
  s->key_descs = -1;
}

}  // namespace

// ---------------------------------------------------------------- planning
fs_status plan_requests(const fs_request *reqs, int n, BatchPlan *bp, void *const *keep_out,
                        long long direct_min_points) {
  bp->descs.clear();
  bp->units.clear();
  bp->arena_bytes = 0;
  bp->smem = 0;
  bp->dtype = -1;
  struct Item {
    int idx;
    double cost;
    size_t ws;
  };
  std::vector<Item> items;
  std::vector<size_t> ws_off(n);
  std::vector<Desc> ds(n);
  for (int i = 0; i < n; ++i) {
    const fs_request &r = reqs[i];
    fs_plan p = r.plan;
    if ((r.op == FS_OP_DIFFUSION_ADVANCE || r.op == FS_OP_WAVE_ADVANCE)) {
      if (!r.state) return set_error(FS_ERR_ARG, "fs_batch_submit: advance request without a state");
      p = r.state->plan;
    }
    if (!p) return set_error(FS_ERR_ARG, "fs_batch_submit: request without a plan");
    if (!r.out_u) return set_error(FS_ERR_ARG, "fs_batch_submit: request without an output");
    if (bp->dtype < 0) bp->dtype = p->dtype;
    if (bp->dtype != p->dtype) return set_error(FS_ERR_SIZE, "fs_batch_submit: mixed dtypes in one batch");
    Desc d = base_desc(p);
    d.work_u = d.work_v = nullptr;
    d.fac = nullptr;
    d.out_u = r.out_u;
    switch (r.op) {
      case FS_OP_POISSON:
        if (!r.in_u) return set_error(FS_ERR_ARG, "fs_batch_submit: Poisson without input");
        d.op = OP_POISSON;
        d.in_u = r.in_u;
        break;
      case FS_OP_DIFFUSION:
      case FS_OP_DIFFUSION_ADVANCE:
        if (!(r.D >= 0.0) || !(r.t >= 0.0) || !std::isfinite(r.D * r.t))
          return set_error(FS_ERR_ARG, "fs_batch_submit: diffusion needs finite D >= 0, t >= 0");
        d.p_dt = r.D * r.t;
        d.p_d = r.D;
        d.p_t = r.t;
        if (r.op == FS_OP_DIFFUSION) {
          if (!r.in_u) return set_error(FS_ERR_ARG, "fs_batch_submit: diffusion without input");
          d.op = OP_DIFFUSION;
          d.in_u = r.in_u;
        } else {
          d.op = OP_DIFF_ADV;
          d.st_u = r.state->su;
          if (r.state->has_s) {
            d.flags |= F_SOURCE;
            d.st_s = r.state->ss;
          }
        }
        break;
      case FS_OP_WAVE:
      case FS_OP_WAVE_ADVANCE:
        if (!(r.c > 0.0) || !std::isfinite(r.c) || !std::isfinite(r.t))
          return set_error(FS_ERR_ARG, "fs_batch_submit: wave needs finite c > 0 and t");
        if (!wave_phase_ok(p, r.c, r.t))
          return set_error(FS_ERR_ARG, "fs_batch_submit: wave phase out of range (FP32: c |t| |omega|_max <= 2^20)");
        d.p_c = r.c;
        d.p_t = r.t;
        if (r.op == FS_OP_WAVE) {
          if (!r.in_u) return set_error(FS_ERR_ARG, "fs_batch_submit: wave without input");
          d.op = OP_WAVE;
          d.in_u = r.in_u;
          d.in_v = r.in_v;
          d.flags = r.in_v ? F_HAS_V0 : 0;
        } else {
          d.op = OP_WAVE_ADV;
          d.st_u = r.state->su;
          d.st_v = r.state->sv;
          d.flags = (r.state->has_v ? F_HAS_V0 : 0) | (r.out_v ? F_WANT_V : 0);
          d.out_v = r.out_v;
          if (r.state->has_s) {
            d.flags |= F_SOURCE;
            d.st_s = r.state->ss;
          }
        }
        break;
      default:
        return set_error(FS_ERR_ARG, "fs_batch_submit: unknown op");
    }
    if (keep_out && keep_out[i]) {
      if (d.op != OP_DIFFUSION && !(d.op == OP_WAVE && !(d.flags & F_HAS_V0)))
        return set_error(FS_ERR_ARG, "keep: only diffusion and zero-velocity wave solves keep spectra");
      d.st_out_u = keep_out[i];
    }
    const bool diff = d.op == OP_DIFFUSION || d.op == OP_DIFF_ADV;
    const int nspec = small_nspec(d);
    const size_t small_b = nspec == 2 ? p->tc.small_smem2 : p->tc.small_smem1;
    const long long small_max = env_ll("FS_BATCH_SMALL_MAX", 256LL * 256LL);
    d.small = (small_b > 0 && small_b <= kMaxDynSmem && (long long)p->nx * p->ny <= small_max) ? 1 : 0;
    // batch-mode tuned register tiles (fs_tune_batch) for problems run as units
    if (!d.small && !(direct_min_points > 0 && (long long)p->nx * p->ny >= direct_min_points)) {
      TuneCfg tc{};
      if (tune_lookup(p->device, p->nx, p->ny, p->dtype, 1, &tc)) {
        RadixPlan rr, rc;
        const bool f64 = p->dtype == FS_F64;
        if (tc.e_row && make_rp_e(d.M, tc.e_row, f64, &rr) && tc.e_col && make_rp_e(d.ny, tc.e_col, f64, &rc)) {
          d.rp_row = rr;
          d.rp_col = rc;
        }
      }
    }
    size_t ws = 0;
    if (diff) ws += align256(fac_bytes(p));
    if (!d.small) {
      ws += align256(p->spec_bytes);
      const bool need_v = (d.op == OP_WAVE && (d.flags & F_HAS_V0)) ||
                          (d.op == OP_WAVE_ADV && (d.flags & F_WANT_V));
      if (need_v) ws += align256(p->spec_bytes);
    }
    ws_off[i] = bp->arena_bytes;
    bp->arena_bytes += ws;
    ds[i] = d;
    // cost ~ bytes moved (3 passes) -> largest first
    items.push_back({i, (double)p->nx * p->ny * (d.small ? 1.0 : 3.0), ws});
  }
  // stable largest-first order
  std::stable_sort(items.begin(), items.end(), [](const Item &a, const Item &b) { return a.cost > b.cost; });
  bp->descs.resize(n);
  bp->direct.assign(n, 0);
  std::vector<int> slot_of(n);
  for (int k = 0; k < n; ++k) {
    slot_of[items[k].idx] = k;
    bp->descs[k] = ds[items[k].idx];
    bp->req_of_desc.push_back(items[k].idx);
    const Desc &d = bp->descs[k];
    if (direct_min_points > 0 && !d.small && (long long)d.nx * d.ny >= direct_min_points) bp->direct[k] = 1;
  }
  bp->ws_off.resize(n);
  for (int k = 0; k < n; ++k) bp->ws_off[k] = ws_off[items[k].idx];

  // CTA size: 256 threads (two CTAs per SM) when every problem run as units
  // has row and column transforms of at most 256 threads and none is a
  // single-CTA small problem (its whole solve would run on half the threads),
  // else 512; 128 threads (four CTAs per SM: a block barrier holds 4 warps,
  // not 8) when, in addition, every problem is an FP32 power-of-two grid of
  // at least 512^2 whose transforms fit 128 threads (the staged compile-time
  // units have tiles of that height; smaller grids lose to the per-unit
  // overhead).  Measured on GB300, 100 advances per batch: 256 vs 512 at
  // 1024^2 +9 %, a 512-problem mix with small problems -18 % at 256; 128 vs
  // 256: 1024^2 504 -> 477 us, 512^2 149 -> 140 us, 2048^2 2006 -> 1950 us,
  // 256^2 60 -> 63 us.  Tile shapes follow; a row's or column's arithmetic
  // does not depend on how many share a CTA.
  // Single-CTA small problems in a batch that also has work units run as a
  // second launch beside the persistent one (their half spectrum in shared
  // memory would otherwise set every CTA's shared memory and size, one CTA
  // of 512 threads per SM; measured on GB300, 512-problem mix: 6.82 ms with
  // them inside, 5.34 ms for the same batch without them).
  bool any_small = false, any_units = false;
  for (int k = 0; k < n; ++k) {
    if (bp->direct[k]) continue;
    (bp->descs[k].small ? any_small : any_units) = true;
  }
  const bool split_small = any_small && any_units;
  {
    int need = 1;
    bool p2_large = true;
    for (int k = 0; k < n; ++k) {
      if (bp->direct[k]) continue;
      const Desc &d = bp->descs[k];
      if (d.small && split_small) continue;
      need = std::max(need, std::max(d.M / d.rp_row.e, d.ny / d.rp_col.e));
      if (d.small) need = kMaxThreads;
      p2_large = p2_large && bp->dtype == FS_F32 && d.rp_row.e == 16 && d.rp_col.e == 16 && p2_row_ok(d.M) &&
                 p2_col_ok(d.ny) && (long long)d.nx * d.ny >= 512LL * 512LL;
    }
    const int bt = (need <= 128 && p2_large) ? 128 : (need <= 256 ? 256 : kMaxThreads);
    if (const char *v = getenv("FS_BATCH_THREADS")) {
      int maxe = 1;  // the override may force 256 when every transform fits
      for (int k = 0; k < n; ++k)
        if (!bp->direct[k] && !(bp->descs[k].small && split_small))
          maxe = std::max(maxe, std::max(bp->descs[k].M / bp->descs[k].rp_row.e, bp->descs[k].ny / bp->descs[k].rp_col.e));
      if (atoi(v) == 512 || (atoi(v) == 256 && maxe <= 256) || (atoi(v) == 128 && maxe <= 128))
        bp->threads = atoi(v);
      else bp->threads = bt;
    } else {
      bp->threads = bt;
    }
    for (int k = 0; k < n; ++k) {
      if (bp->direct[k]) continue;
      Desc &d = bp->descs[k];
      const int tseg = d.ny / d.rp_col.e, tr = d.M / d.rp_row.e;
      const size_t cs = bp->dtype == FS_F64 ? 16 : 8;
      int cc = bp->threads / tseg;
      if (cc > 32) cc = 32;
      if (cc < 1) cc = 1;
      while (cc > 1 && (size_t)padded_len(cc * d.ny) * cs > 100 * 1024) cc >>= 1;
      d.cols_per_unit = cc;
      // single-field FP32 columns of compiled lengths (powers of two with
      // tile 16, 3 x 2^k / 5 x 2^k with their family's tile): each column
      // group is staged into shared memory by one bulk copy while the
      // previous one computes
      const bool col_ct = (d.rp_col.e == 16 && p2_col_ok(d.ny)) || (mx_col_ok(d.ny) && d.rp_col.e == mx_e(d.ny));
      if (bp->dtype == FS_F32 && !d.small && col_ct && !col_two_fields(d) && !(d.flags & F_SOURCE) &&
          tma_enabled())
        d.flags |= F_COL_TMA;
      int rr = d.rows_per_unit;  // the plan's row tile
      if (rr * tr > bp->threads) rr = std::max(1, bp->threads / tr);
      d.rows_per_unit = rr;
      d.n_row_units = (d.ny + rr - 1) / rr;
      // C2R tiles of an even number of FP32 rows of compiled lengths and
      // tile heights: each tile is staged into shared memory by asynchronous
      // copies while the previous one computes
      const bool row_p2 = d.rp_row.e == 16 && p2_row_ok(d.M) &&
                          (rr == p2_row_cnt(d.M) || rr == p2_row_cnt_256(d.M) || rr == p2_row_cnt_128(d.M));
      const bool row_mx = mx_row_ok(d.M) && d.rp_row.e == mx_e(d.M) &&
                          (rr == mx_row_cnt(d.M) || rr == mx_row_cnt_256(d.M));
      if (bp->dtype == FS_F32 && !d.small && (row_p2 || row_mx) && rr % 2 == 0 && tma_enabled())
        d.flags |= F_ROW_STAGED;
      // R2C tiles of the same lengths and heights: a tile (whole rows, one
      // contiguous run of the real field) is staged by 16-byte asynchronous
      // copies while the previous one computes; the field must be 16-byte aligned
      const bool in_aligned = reinterpret_cast<uintptr_t>(d.in_u) % 16 == 0 &&
                              reinterpret_cast<uintptr_t>(d.in_v) % 16 == 0;
      if (bp->dtype == FS_F32 && !d.small && (row_p2 || row_mx) && in_aligned && tma_enabled())
        d.flags |= F_R2C_STAGED;
      d.n_col_units = (d.M + 1 + cc - 1) / cc;
      if (d.small) {
        const int st = split_small ? bp->small_threads : bp->threads;
        if (d.small_rows * tr > st) d.small_rows = std::max(1, st / tr);
        if (d.small_cols * tseg > st) d.small_cols = std::max(1, st / tseg);
      }
    }
  }

  // Work-unit granularity: each unit covers G row tiles / column groups, G
  // chosen so the batch still has several units per SM (grouping does not
  // change any problem's arithmetic).
  {
    long long tiles = 0;
    for (int k = 0; k < n; ++k) {
      const Desc &d = bp->descs[k];
      if (d.small || bp->direct[k]) continue;
      tiles += (d.ny + d.rows_per_unit - 1) / d.rows_per_unit;
      tiles += (d.M + 1 + d.cols_per_unit - 1) / d.cols_per_unit;
    }
    // measured on GB300 with staged units (the first tile of a unit is loaded
    // unhidden, the rest behind the previous tile's compute), 100 advances
    // per batch: 3 per unit beat 4 at 256^2..1536^2 (512^2: 153 vs 161 us,
    // 768^2: 898 vs 1005 us) and 1-2 (512^2: 0.207 ms at 1), 4 beat 3 from
    // 1024^2 up (2048^2: 2073 vs 2179 us), 6-8 lose (too few units to
    // balance); a batch with few tiles keeps one per unit so that they
    // spread over the CTAs
    int G = (int)(tiles / (4LL * 152LL));
    G = G < 1 ? 1 : (G > 3 ? 3 : G);
    const char *genv = getenv("FS_BATCH_GROUP");
    for (int k = 0; k < n; ++k) {
      Desc &d = bp->descs[k];
      int g = (G == 3 && (long long)d.nx * d.ny >= 1024LL * 1024LL) ? 4 : G;
      if (genv && atoi(genv) > 0) g = atoi(genv);
      d.row_g = d.col_g = g;
      const int rt = (d.ny + d.rows_per_unit - 1) / d.rows_per_unit;
      const int cg = (d.M + 1 + d.cols_per_unit - 1) / d.cols_per_unit;
      d.n_row_units = (rt + g - 1) / g;
      d.n_col_units = (cg + g - 1) / g;
    }
  }
  // chunks by intermediate bytes
  std::vector<int> chunk_start;
  size_t acc = 0;
  for (int k = 0; k < n; ++k) {
    if (k == 0 || acc >= kChunkBytes) {
      chunk_start.push_back(k);
      acc = 0;
    }
    acc += items[k].ws;
  }
  chunk_start.push_back(n);
  const int nch = (int)chunk_start.size() - 1;
  auto emit_front = [&](int c) {
    for (int k = chunk_start[c]; k < chunk_start[c + 1]; ++k) {
      const Desc &d = bp->descs[k];
      if (bp->direct[k]) continue;
      if (d.small) {
        if (!split_small) bp->units.push_back(make_int4(k, K_SMALL, 0, 0));
        continue;
      }
      if (d.op == OP_DIFFUSION || d.op == OP_DIFF_ADV)
        for (int u = 0; u < d.n_fac_units; ++u) bp->units.push_back(make_int4(k, K_FACTOR, u, 0));
      if (d.op != OP_DIFF_ADV && d.op != OP_WAVE_ADV) {
        const int fields = (d.op == OP_WAVE && (d.flags & F_HAS_V0)) ? 2 : 1;
        for (int f = 0; f < fields; ++f)
          for (int u = 0; u < d.n_row_units; ++u) bp->units.push_back(make_int4(k, K_ROW, u, f));
      }
    }
  };
  auto emit_col = [&](int c) {
    for (int k = chunk_start[c]; k < chunk_start[c + 1]; ++k) {
      const Desc &d = bp->descs[k];
      if (d.small || bp->direct[k]) continue;
      for (int u = 0; u < d.n_col_units; ++u) bp->units.push_back(make_int4(k, K_COL, u, 0));
    }
  };
  auto emit_c2r = [&](int c) {
    for (int k = chunk_start[c]; k < chunk_start[c + 1]; ++k) {
      const Desc &d = bp->descs[k];
      if (d.small || bp->direct[k]) continue;
      const int fields = (d.op == OP_WAVE_ADV && (d.flags & F_WANT_V)) ? 2 : 1;
      for (int f = 0; f < fields; ++f)
        for (int u = 0; u < d.n_row_units; ++u) bp->units.push_back(make_int4(k, K_C2R, u, f));
    }
  };
  for (int i = 0; i < nch + 2; ++i) {
    if (i < nch) emit_front(i);
    if (i - 1 >= 0 && i - 1 < nch) emit_col(i - 1);
    if (i - 2 >= 0 && i - 2 < nch) emit_c2r(i - 2);
  }
  // the second launch's table: small problems, largest first
  if (split_small)
    for (int k = 0; k < n; ++k)
      if (bp->descs[k].small && !bp->direct[k]) {
        bp->units.push_back(make_int4(k, K_SMALL, 0, 0));
        ++bp->n_small_units;
      }
  return FS_OK;
}

template <typename T>
static size_t unit_smem(const Desc &d) {
  if (d.small) return Launch<T>::small_smem(d);
  const size_t col = (d.flags & F_COL_TMA) ? p2_col1_tma_unit_smem(d.ny, d.cols_per_unit) : Launch<T>::col_smem(d);
  size_t row = (d.flags & F_ROW_STAGED) ? 2 * (size_t)c2r_stage_len(d.M, d.rows_per_unit) * sizeof(cx<T>)
                                         : Launch<T>::row_smem(d);
  if (d.flags & F_R2C_STAGED)
    row = std::max(row, 2 * (size_t)r2c_stage_len(d.M, d.rows_per_unit) * sizeof(cx<T>));
  return std::max(row, col);
}

// A problem run as standalone pass kernels (the per-call path) with the
// batch's workspace pointers.
template <typename T>
static cudaError_t run_direct(const Desc &d0, cudaStream_t s) {
  typedef Launch<T> L;
  Desc d = d0;
  d.row_g = d.col_g = 1;
  d.n_row_units = (d.ny + d.rows_per_unit - 1) / d.rows_per_unit;
  // the standalone column kernels use the plan's column grouping
  const int tseg = d.ny / d.rp_col.e;
  int cc = 32;
  while (cc > 1 && (cc * tseg > kMaxThreads || sizeof(cx<T>) * (size_t)padded_len(cc * d.ny) > 96 * 1024)) cc >>= 1;
  if (sizeof(T) == 4 && d.rp_col.e == 16 && p2_col_ok(d.ny)) cc = p2_col_cnt(d.ny);
  d.cols_per_unit = cc;
  d.n_col_units = (d.M + 1 + cc - 1) / cc;
  const bool diff = d.op == OP_DIFFUSION || d.op == OP_DIFF_ADV;
  const bool adv = d.op == OP_DIFF_ADV || d.op == OP_WAVE_ADV;
  cudaError_t e = cudaSuccess;
  if (diff) e = L::factor(d, s);
  if (e == cudaSuccess && !adv) e = L::rows(d, (d.op == OP_WAVE && (d.flags & F_HAS_V0)) ? 2 : 1, s);
  if (e == cudaSuccess) e = L::cols(d, s);
  if (e == cudaSuccess) e = L::c2r(d, (d.op == OP_WAVE_ADV && (d.flags & F_WANT_V)) ? 2 : 1, s);
  return e;
}

// Resolve arena offsets into pointers and compute the launch's shared memory.
template <typename T>
static size_t finish_descs(BatchPlan *bp, char *arena) {
  size_t smem = 0;
  bp->small_smem = 0;
  for (size_t k = 0; k < bp->descs.size(); ++k) {
    Desc &d = bp->descs[k];
    fill_op_consts(d);
    char *w = arena + bp->ws_off[k];
    const size_t fb = align256((size_t)(d.M + 1 + d.ny) * 8);  // float2 or double per entry
    const size_t sb = align256((size_t)(d.M + 1) * d.ny * 2 * sizeof(T));
    if (d.op == OP_DIFFUSION || d.op == OP_DIFF_ADV) {
      d.fac = w;
      w += fb;
    }
    if (!d.small) {
      d.work_u = w;
      w += sb;
      const bool need_v = (d.op == OP_WAVE && (d.flags & F_HAS_V0)) ||
                          (d.op == OP_WAVE_ADV && (d.flags & F_WANT_V));
      if (need_v) d.work_v = w;
    }
    if (bp->direct[k]) continue;
    if (d.small && bp->n_small_units > 0)
      bp->small_smem = std::max(bp->small_smem, unit_smem<T>(d));
    else
      smem = std::max(smem, unit_smem<T>(d));
  }
  return smem;
}

}  // namespace fs

namespace fs {

fs_status request_workspace(const fs_request &r, size_t *bytes) {
  BatchPlan bp;
  const fs_status st = plan_requests(&r, 1, &bp);
  *bytes = st == FS_OK ? bp.arena_bytes : 0;
  return st;
}

fs_status batch_submit_internal(const fs_request *reqs, int n, void *const *keep_out, uint64_t *ticket_out,
                                cudaStream_t stream, char *ext_arena, size_t ext_bytes, long long direct_min_points) {
  BatchPlan bp;
  fs_status st = plan_requests(reqs, n, &bp, keep_out, direct_min_points);
  if (st != FS_OK) return st;
  const unsigned long long wait_ns = (unsigned long long)env_ll("FS_BATCH_WAIT_NS", 2000000000LL);
  const bool inject = env_ll("FS_BATCH_INJECT_STALL", 0) != 0;

  std::lock_guard<std::mutex> lk(g_mu);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "fs_batch_submit: cudaGetDevice");
  // an idle slot of this device (its last batch finished); else a new one, up
  // to kMaxSlots per device; else wait for the oldest pending batch (a new
  // slot means device allocations and a graph capture on the host while the
  // GPU may be idle)
  Slot *s = nullptr, *oldest = nullptr;
  int on_dev = 0;
  for (Slot *c : g_slots) {
    if (c->device != dev) continue;
    ++on_dev;
    if (c->pending) {
      const cudaError_t q = cudaEventQuery(c->ev);
      if (q == cudaErrorNotReady) {
        if (!oldest || c->ticket < oldest->ticket) oldest = c;
        continue;
      }
      if (q != cudaSuccess) return cuda_error(q, "fs_batch_submit: event query");
      c->pending = false;
      remember(c->ticket, slot_status(c));
    }
    s = c;
    break;
  }
  if (!s && oldest && on_dev >= kMaxSlots) {
    e = cudaEventSynchronize(oldest->ev);
    if (e != cudaSuccess) return cuda_error(e, "fs_batch_submit: wait for a slot");
    oldest->pending = false;
    remember(oldest->ticket, slot_status(oldest));
    s = oldest;
  }
  if (!s) {
    s = new Slot();
    s->device = dev;
    e = cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->cap2, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&s->h_status, 4 * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&s->d_ctl, 4 * sizeof(int));
    if (e != cudaSuccess) return cuda_error(e, "fs_batch_submit: slot creation");
    g_slots.push_back(s);
  }
  const size_t nd = bp.descs.size(), nu = bp.units.size();
  const size_t cd = s->cap_descs;
  e = grow(&s->d_descs, &s->h_descs, s->cap_descs, nd);
  if (e == cudaSuccess && s->cap_descs != cd) {
    cudaFree(s->d_done);
    s->d_done = nullptr;
    e = cudaMalloc((void **)&s->d_done, 5 * s->cap_descs * sizeof(int));
    drop_graph(s);
  }
  const size_t cu = s->cap_units;
  if (e == cudaSuccess) e = grow(&s->d_units, &s->h_units, s->cap_units, nu);
  if (e == cudaSuccess && s->cap_units != cu) drop_graph(s);
  if (ext_arena && ext_bytes < bp.arena_bytes)
    return set_error(FS_ERR_ARG, "batch: external arena smaller than the batch workspace");
  if (e == cudaSuccess && !ext_arena && bp.arena_bytes > s->cap_arena) {
    cudaFree(s->d_arena);
    s->d_arena = nullptr;
    s->cap_arena = 0;
    e = cudaMalloc((void **)&s->d_arena, bp.arena_bytes);
    if (e == cudaSuccess) s->cap_arena = bp.arena_bytes;
  }
  if (e != cudaSuccess) return cuda_error(e, "fs_batch_submit: buffer allocation");

  const int dtype = bp.dtype;
  char *arena = ext_arena ? ext_arena : s->d_arena;
  const size_t smem = dtype == FS_F64 ? finish_descs<double>(&bp, arena) : finish_descs<float>(&bp, arena);
  if (smem > kMaxDynSmem || bp.small_smem > kMaxDynSmem)
    return set_error(FS_ERR_SIZE, "fs_batch_submit: unit shared memory too large");
  if (inject) {
    // test hook: make the first three-pass problem's column units wait for a
    // row tile that is never produced, so the bounded wait expires
    for (size_t k = 0; k < nd; ++k) {
      Desc &d = bp.descs[k];
      if (!d.small && !bp.direct[k] && d.op != OP_DIFF_ADV && d.op != OP_WAVE_ADV) {
        d.n_row_units += 1;
        break;
      }
    }
  }
  // problems above the direct threshold: standalone pass kernels, in order
  for (size_t k = 0; k < nd; ++k) {
    if (!bp.direct[k]) continue;
    e = dtype == FS_F64 ? run_direct<double>(bp.descs[k], stream) : run_direct<float>(bp.descs[k], stream);
    if (e != cudaSuccess) return cuda_error(e, "batch: standalone pass launch");
  }
  if (nu == 0) {
    s->h_status[0] = s->h_status[1] = s->h_status[2] = s->h_status[3] = 0;
    e = cudaEventRecord(s->ev, stream);
    if (e != cudaSuccess) return cuda_error(e, "batch: event record");
    s->pending = true;
    s->ticket = g_next_ticket++;
    if (ticket_out) *ticket_out = s->ticket;
    return FS_OK;
  }
  memcpy(s->h_descs, bp.descs.data(), nd * sizeof(Desc));
  memcpy(s->h_units, bp.units.data(), nu * sizeof(int4));

  // the persistent launch over the table's first nm units and, when the
  // batch has both kinds, the small problems' launch over the last ns
  const int ns = bp.n_small_units, nm = (int)nu - ns;
  int per_sm = 0, sms = 0;
  int threads = bp.threads;
  auto occupancy = [&](int th, size_t bytes, int *out) {
    return dtype == FS_F64 ? Launch<double>::batch_occupancy(th, bytes, out)
                           : Launch<float>::batch_occupancy(th, bytes, out);
  };
  e = occupancy(threads, smem, &per_sm);
  // 256-thread CTAs only pay when two fit on an SM (a resident small problem's
  // half spectrum can take most of the shared memory); the tiles also fit 512
  if (e == cudaSuccess && threads <= 256 && per_sm < 2) {
    threads = kMaxThreads;
    e = occupancy(threads, smem, &per_sm);
  }
  int per_sm2 = 0;
  const int threads2 = bp.small_threads;
  const size_t smem2 = bp.small_smem;
  if (e == cudaSuccess && ns > 0) e = occupancy(threads2, smem2, &per_sm2);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_error(e, "fs_batch_submit: occupancy");
  if (per_sm < 1 || (ns > 0 && per_sm2 < 1))
    return set_error(FS_ERR_SIZE, "fs_batch_submit: batch kernel does not fit on an SM");
  int grid = sms * per_sm;
  if (grid > nm) grid = nm;
  // The small problems' launch runs beside the persistent one from the start
  // on part of the GPU: its CTAs are dispatched first (high priority) and
  // loop over the small problems, the persistent CTAs fill the remaining room
  // and take the SMs it frees.  Its CTA count: enough that it ends well
  // within the persistent launch's time (estimated at 1.5 TB/s over the
  // units' bytes, ~150 us per single-CTA problem), at least a quarter of the
  // SMs, at most one per SM (measured on GB300, 512-problem mix: 4.39 ms
  // with one CTA per SM launched beside the persistent one).
  int grid2 = 0;
  if (ns > 0) {
    double unit_bytes = 0.0;
    for (size_t k = 0; k < nd; ++k)
      if (!bp.descs[k].small && !bp.direct[k]) unit_bytes += 24.0 * (double)bp.descs[k].nx * bp.descs[k].ny;
    const double t_main_us = unit_bytes / 1.5e6, t_small_us = 150.0;
    const int cap = std::min(ns, sms * per_sm2);
    grid2 = (int)std::ceil(ns * t_small_us / std::max(t_main_us, 1.0));
    grid2 = std::max(grid2, std::min(cap, std::max(1, sms / 4)));
    grid2 = std::min(grid2, cap);
  }

  const bool same = s->gexec && s->key_descs == (int)nd && s->key_units == (int)nu && s->key_grid == grid &&
                    s->key_dtype == dtype && s->key_smem == smem && s->key_wait == wait_ns &&
                    s->key_threads == threads && s->key_small_units == ns && s->key_small_grid == grid2 &&
                    s->key_small_threads == threads2 && s->key_small_smem == smem2;
  if (!same) {
    drop_graph(s);
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(s->cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      cudaMemcpyAsync(s->d_descs, s->h_descs, nd * sizeof(Desc), cudaMemcpyHostToDevice, s->cap);
      cudaMemcpyAsync(s->d_units, s->h_units, nu * sizeof(int4), cudaMemcpyHostToDevice, s->cap);
      cudaMemsetAsync(s->d_ctl, 0, 4 * sizeof(int), s->cap);
      cudaMemsetAsync(s->d_done, 0, 5 * nd * sizeof(int), s->cap);
      cudaError_t le = cudaSuccess;
      // the two launches are independent branches of the graph (no unit of
      // one waits on the other's)
      if (ns > 0) {
        le = cudaEventRecord(s->ev_fork, s->cap);
        if (le == cudaSuccess) le = cudaStreamWaitEvent(s->cap2, s->ev_fork, 0);
      }
      if (ns > 0 && le == cudaSuccess)
        le = dtype == FS_F64 ? Launch<double>::batch(s->d_descs, s->d_units + nm, ns, s->d_ctl + 2, s->d_done,
                                                     grid2, threads2, smem2, wait_ns, s->cap2, true)
                             : Launch<float>::batch(s->d_descs, s->d_units + nm, ns, s->d_ctl + 2, s->d_done,
                                                    grid2, threads2, smem2, wait_ns, s->cap2, true);
      if (le == cudaSuccess)
        le = dtype == FS_F64 ? Launch<double>::batch(s->d_descs, s->d_units, nm, s->d_ctl, s->d_done, grid,
                                                     threads, smem, wait_ns, s->cap)
                             : Launch<float>::batch(s->d_descs, s->d_units, nm, s->d_ctl, s->d_done, grid,
                                                    threads, smem, wait_ns, s->cap);
      if (ns > 0) {
        // join the branch whatever happened, so that the capture can end
        const cudaError_t je = cudaEventRecord(s->ev_join, s->cap2);
        const cudaError_t we = je == cudaSuccess ? cudaStreamWaitEvent(s->cap, s->ev_join, 0) : je;
        if (le == cudaSuccess) le = we;
      }
      cudaMemcpyAsync(s->h_status, s->d_ctl, 4 * sizeof(int), cudaMemcpyDeviceToHost, s->cap);
      e = cudaStreamEndCapture(s->cap, &g);
      if (e == cudaSuccess && le != cudaSuccess) e = le;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&s->gexec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess) {
      s->gexec = nullptr;
      return cuda_error(e, "fs_batch_submit: graph capture");
    }
    s->key_descs = (int)nd;
    s->key_units = (int)nu;
    s->key_grid = grid;
    s->key_dtype = dtype;
    s->key_smem = smem;
    s->key_wait = wait_ns;
    s->key_threads = threads;
    s->key_small_units = ns;
    s->key_small_grid = grid2;
    s->key_small_threads = threads2;
    s->key_small_smem = smem2;
  } else {
    g_launches.fetch_add(ns > 0 ? 2 : 1, std::memory_order_relaxed);  // the replayed k_batch launches
  }
  {
    ProfScope ps(PC_BATCH, stream);
    e = cudaGraphLaunch(s->gexec, stream);
  }
  if (e == cudaSuccess) e = cudaEventRecord(s->ev, stream);
  if (e != cudaSuccess) return cuda_error(e, "fs_batch_submit: graph launch");
  s->pending = true;
  s->ticket = g_next_ticket++;
  if (ticket_out) *ticket_out = s->ticket;
  return FS_OK;
}

}  // namespace fs

using namespace fs;

extern "C" fs_status fs_batch_submit(const fs_request *reqs, int n, uint64_t *ticket_out, fs_stream stream) {
  if (ticket_out) *ticket_out = 0;
  if (!reqs || n <= 0) return set_error(FS_ERR_ARG, "fs_batch_submit: empty batch");
  // grids of 4096^2 points and more fill the GPU on their own: they run as
  // the standalone pass kernels (persistent TMA row passes, staged column
  // pass), in order, before the persistent launch (measured on GB300, 50
  // wave advances of 4096^2: 11.5k/s as passes, 10.0k/s as batch units)
  const long long direct_min = env_ll("FS_BATCH_DIRECT_MIN", 4096LL * 4096LL);
  return batch_submit_internal(reqs, n, nullptr, ticket_out, reinterpret_cast<cudaStream_t>(stream), nullptr, 0,
                               direct_min);
}

extern "C" fs_status fs_batch_wait(uint64_t ticket, int timeout_us) {
  Slot *s = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &f : g_finished)
      if (f.first == ticket) return f.second == 0 ? FS_OK : set_error((fs_status)f.second, "batch failed");
    for (Slot *c : g_slots)
      if (c->ticket == ticket && c->pending) s = c;
    if (!s) {
      if (ticket == 0 || ticket >= g_next_ticket) return set_error(FS_ERR_ARG, "fs_batch_wait: unknown ticket");
      return FS_OK;  // finished long ago
    }
  }
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t q = cudaEventQuery(s->ev);
    if (q == cudaSuccess) break;
    if (q != cudaErrorNotReady) return cuda_error(q, "fs_batch_wait");
    if (timeout_us >= 0 && std::chrono::duration_cast<std::chrono::microseconds>(
                               std::chrono::steady_clock::now() - t0).count() > timeout_us)
      return set_error(FS_ERR_TIMEOUT, "fs_batch_wait: timed out");
    std::this_thread::yield();
  }
  std::lock_guard<std::mutex> lk(g_mu);
  int status = 0;
  if (s->pending && s->ticket == ticket) {
    s->pending = false;
    status = slot_status(s);
    remember(ticket, status);
  } else {
    for (auto &f : g_finished)
      if (f.first == ticket) status = f.second;
  }
  if (status != 0) return set_error((fs_status)status, "fs_batch_wait: a unit's bounded wait expired");
  return FS_OK;
}
