// fs_kernels.cuh -- __global__ entry points built from the units, and their
// host-side launchers.  Included once per element type (fs_kernels_f32.cu,
// fs_kernels_f64.cu) so the two precisions compile in parallel.
#pragma once
#include <atomic>

#include "fs_col_tma.cuh"
#include "fs_mixed.h"
#include "fs_pow2.h"
#include "fs_row_async.cuh"
#include "fs_tma.cuh"
#include "fs_units.cuh"

namespace fs {

extern std::atomic<unsigned long long> g_launches;

// TMA-staged kernels can be switched off (env FS_NO_TMA=1) for comparison.
bool tma_enabled();

// Optional per-launch event timing (fs_profile_enable); classes as in fsolve.h.
enum ProfClass { PC_R2C = 0, PC_COL = 1, PC_C2R = 2, PC_FACTOR = 3, PC_SMALL = 4, PC_BATCH = 5, PC_N = 6 };
bool prof_on();
void prof_begin(int cls, cudaStream_t s, void **tok);
void prof_end(void *tok, cudaStream_t s);
// NVTX ranges around each pass launch (env FS_NVTX=1; no-ops without a tool)
bool nvtx_on();
void nvtx_push(int cls);
void nvtx_pop();
struct ProfScope {
  void *tok = nullptr;
  cudaStream_t s;
  bool nv = false;
  ProfScope(int cls, cudaStream_t st) : s(st) {
    if (prof_on()) prof_begin(cls, st, &tok);
    if (nvtx_on()) {
      nvtx_push(cls);
      nv = true;
    }
  }
  ~ProfScope() {
    if (tok) prof_end(tok, s);
    if (nv) nvtx_pop();
  }
};

// Persistent TMA-staged row passes (fs_rows_tma.cu): FP32, power-of-two row
// transforms of length 512 .. 4096; false / not launched otherwise.
bool rows_tma_ok(const Desc &d, int nfields, bool c2r);
cudaError_t rows_tma_launch(const Desc &d, int nfields, bool c2r, cudaStream_t s);

constexpr int kMaxThreads = 512;
constexpr int kFactorPerUnit = 256;  // factor-table entries per factor unit

// ---------------------------------------------------------------- pass kernels
// The row R2C / column / row C2R pass kernels are defined per register tile in
// fs_units_inst.cu (k_r2c_<T>_<E>, k_col1/k_col2_<T>_<E>, k_c2r_<T>_<E>) so
// that each inlines its unit; the launchers below select them by tile size.

// Diffusion per-axis factor tables: grid = n_fac_units, 256 threads.
template <typename T>
__global__ void __launch_bounds__(256) k_factor(const Desc d) {
  unit_factor<T>(d, blockIdx.x * kFactorPerUnit, kFactorPerUnit, 256);
}

// Small grids: the whole solve in one CTA, grid = 1.
template <typename T>
__global__ void __launch_bounds__(kMaxThreads) k_small(const Desc d) {
  extern __shared__ __align__(16) unsigned char fs_smem[];
  unit_small<T>(d, reinterpret_cast<cx<T> *>(fs_smem));
}

// ---------------------------------------------------------------- persistent batch
// Work unit: x = problem, y = kind (K_*), z = unit index within its kind,
// w = field (0: u, 1: v).  Units are listed so that every dependency of a
// unit has a smaller index; CTAs take indices from ctl[0] in order, so a unit
// only ever waits on units already taken by running CTAs.
//   ctl[0] next unit, ctl[1] status (0 ok, else an fs_status),
//   done[5*p + kind] units of that kind finished for problem p.
__device__ __forceinline__ int ld_acquire(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// Batch column unit staged by bulk copies (F_COL_TMA): columns [c0, c1) in
// groups of cnt, the second group buffer after the first in `sm`.  Inlined
// (a call would keep the shared-memory descriptor's fields live across the
// ABI boundary and spill).  Returns 1 done, 0 length not specialised, -1 a
// copy timed out.
template <int L>
__device__ __forceinline__ int col_tma_unit_l(const Desc &d, int c0, int c1, int cnt, cx<float> *sm,
                                              uint64_t *bars, uint32_t &ph, int *s_abort) {
  const int plen = (padded_len(cnt * L) + 1) & ~1;  // even: the second buffer stays 16-byte aligned
  return col_tma_groups<L, 0>(d, c0, cnt, c1, cnt, sm, sm + plen, bars, ph, s_abort) ? 1 : -1;
}
__device__ __forceinline__ int col_tma_unit(const Desc &d, int c0, int c1, int cnt, cx<float> *sm, uint64_t *bars,
                                            uint32_t &ph, int *s_abort) {
  switch (d.ny) {
    case 128: return col_tma_unit_l<128>(d, c0, c1, cnt, sm, bars, ph, s_abort);
    case 256: return col_tma_unit_l<256>(d, c0, c1, cnt, sm, bars, ph, s_abort);
    case 512: return col_tma_unit_l<512>(d, c0, c1, cnt, sm, bars, ph, s_abort);
    case 1024: return col_tma_unit_l<1024>(d, c0, c1, cnt, sm, bars, ph, s_abort);
    case 2048: return col_tma_unit_l<2048>(d, c0, c1, cnt, sm, bars, ph, s_abort);
    case 4096: return col_tma_unit_l<4096>(d, c0, c1, cnt, sm, bars, ph, s_abort);
    case 8192: return col_tma_unit_l<8192>(d, c0, c1, cnt, sm, bars, ph, s_abort);
    default: return mx_col_tma_unit(d, c0, c1, cnt, sm, bars, ph, s_abort);  // 3 x 2^k, 5 x 2^k
  }
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// THREADS = 512 (one CTA per SM at 128 registers) or 256 (two CTAs per SM:
// one unit's barrier waits overlap the other's work); the batch plan picks 256
// when every problem's transforms fit and shapes its tiles accordingly.

template <typename T, int THREADS>
__global__ void __launch_bounds__(THREADS, THREADS == 128 ? 4 : (THREADS == 256 ? 2 : 1)) k_batch(const Desc *__restrict__ descs,
                                                       const int4 *__restrict__ units, int n_units,
                                                       int *ctl, int *done,
                                                       unsigned long long wait_ns) {
  extern __shared__ __align__(16) unsigned char fs_smem[];
  __shared__ Desc sd;
  __shared__ int s_unit, s_abort;
  cx<T> *sm = reinterpret_cast<cx<T> *>(fs_smem);
  __shared__ int s_next;
  // mbarriers of the bulk-copy column units (F_COL_TMA); ph = their next
  // completion parities, identical in every thread
  __shared__ uint64_t s_bars[2];
  uint32_t tma_ph = 0;
  if (threadIdx.x == 0) {
    s_next = atomicAdd(&ctl[0], 1);
    mbar_init(&s_bars[0], 1);
    mbar_init(&s_bars[1], 1);
    fence_mbar_init();
  }
  for (;;) {
    if (threadIdx.x == 0) {
      s_unit = s_next;
      s_abort = 0;
      // the next unit index is fetched while this one runs (indices are taken
      // and run in increasing order per CTA, so dependencies stay backward)
      if (s_unit < n_units) s_next = atomicAdd(&ctl[0], 1);
    }
    __syncthreads();
    const int k = s_unit;
    if (k >= n_units) break;
    const int4 u = units[k];
    // copy the descriptor into shared memory (word by word)
    {
      const int *src = reinterpret_cast<const int *>(descs + u.x);
      int *dst = reinterpret_cast<int *>(&sd);
      for (int i = threadIdx.x; i < (int)(sizeof(Desc) / sizeof(int)); i += blockDim.x)
        dst[i] = src[i];
    }
    if (threadIdx.x == 0) {
      // dependencies: columns need every row tile (and factor range) of the
      // problem, the C2R tiles need every column group.
      const Desc &dd = descs[u.x];
      int need0 = -1, cnt0 = 0, need1 = -1, cnt1 = 0;
      if (u.y == K_COL) {
        const bool adv = (dd.op == OP_DIFF_ADV || dd.op == OP_WAVE_ADV);
        const bool two = (dd.op == OP_WAVE || dd.op == OP_FORWARD) && (dd.flags & F_HAS_V0);
        if (!adv) {
          need0 = K_ROW;
          cnt0 = dd.n_row_units * (two ? 2 : 1);
        }
        if (dd.op == OP_DIFFUSION || dd.op == OP_DIFF_ADV) {
          need1 = K_FACTOR;
          cnt1 = dd.n_fac_units;
        }
      } else if (u.y == K_C2R) {
        need0 = K_COL;
        cnt0 = dd.n_col_units;
      }
      const unsigned long long t0 = global_ns();
      for (int pass = 0; pass < 2 && !s_abort; ++pass) {
        const int need = pass ? need1 : need0, cnt = pass ? cnt1 : cnt0;
        if (need < 0) continue;
        unsigned ns = 32;
        while (ld_acquire(&done[5 * u.x + need]) < cnt) {
          if (ld_acquire(&ctl[1]) != 0) {
            s_abort = 1;
            break;
          }
          if (global_ns() - t0 > wait_ns) {
            atomicCAS(&ctl[1], 0, -6 /* FS_ERR_TIMEOUT */);
            s_abort = 1;
            break;
          }
          __nanosleep(ns);
          if (ns < 1024) ns <<= 1;
        }
      }
    }
    __syncthreads();
    if (s_abort) break;
    const Desc &d = sd;
    bool tma_failed = false;
    switch (u.y) {
      case K_FACTOR:
        unit_factor<T>(d, u.z * kFactorPerUnit, kFactorPerUnit, blockDim.x);
        break;
      case K_ROW: {
        const int tiles = (d.ny + d.rows_per_unit - 1) / d.rows_per_unit;
        if constexpr (sizeof(T) == 4) {
          if (d.flags & F_R2C_STAGED) {
            const int t0 = u.z * d.row_g, t1 = min(tiles, t0 + d.row_g);
            const float *in = reinterpret_cast<const float *>(u.w ? d.in_v : d.in_u);
            cx<float> *spec = reinterpret_cast<cx<float> *>(u.w ? d.work_v : d.work_u);
            if (p2_r2c_staged_unit(d, t0, t1, d.rows_per_unit, sm, in, spec) ||
                mx_r2c_staged_unit(d, t0, t1, d.rows_per_unit, sm, in, spec))
              break;
          }
        }
        for (int g = 0; g < d.row_g; ++g) {
          const int tile = u.z * d.row_g + g;
          if (tile >= tiles) break;
          row_r2c_any<T>(d, tile, d.rows_per_unit, sm, reinterpret_cast<const T *>(u.w ? d.in_v : d.in_u),
                         reinterpret_cast<cx<T> *>(u.w ? d.work_v : d.work_u));
        }
        break;
      }
      case K_SMALL:
        unit_small<T>(d, sm);
        break;
      case K_COL: {
        if constexpr (sizeof(T) == 4) {
          if (d.flags & F_COL_TMA) {
            const int cnt = d.cols_per_unit;
            const int c0 = u.z * d.col_g * cnt;
            const int c1 = min(d.M + 1, c0 + d.col_g * cnt);
            const int r = col_tma_unit(d, c0, c1, cnt, sm, s_bars, tma_ph, &s_abort);
            if (r < 0) {
              if (threadIdx.x == 0) atomicCAS(&ctl[1], 0, -6 /* FS_ERR_TIMEOUT */);
              tma_failed = true;
            }
            if (r != 0) break;
          }
        }
        const int groups = (d.M + 1 + d.cols_per_unit - 1) / d.cols_per_unit;
        for (int g = 0; g < d.col_g; ++g) {
          const int grp = u.z * d.col_g + g;
          if (grp >= groups) break;
          col_any<T>(d, grp, d.cols_per_unit, sm, reinterpret_cast<cx<T> *>(d.work_u),
                     reinterpret_cast<cx<T> *>(d.work_v), false);
        }
        break;
      }
      case K_C2R: {
        const int tiles = (d.ny + d.rows_per_unit - 1) / d.rows_per_unit;
        if constexpr (sizeof(T) == 4) {
          if (d.flags & F_ROW_STAGED) {
            const int t0 = u.z * d.row_g, t1 = min(tiles, t0 + d.row_g);
            const cx<float> *spec = reinterpret_cast<const cx<float> *>(u.w ? d.work_v : d.work_u);
            float *out = reinterpret_cast<float *>(u.w ? d.out_v : d.out_u);
            if (c2r_staged_unit(d, t0, t1, d.rows_per_unit, sm, spec, out) ||
                mx_c2r_staged_unit(d, t0, t1, d.rows_per_unit, sm, spec, out))
              break;
          }
        }
        for (int g = 0; g < d.row_g; ++g) {
          const int tile = u.z * d.row_g + g;
          if (tile >= tiles) break;
          row_c2r_any<T>(d, tile, d.rows_per_unit, sm, reinterpret_cast<const cx<T> *>(u.w ? d.work_v : d.work_u),
                         reinterpret_cast<T *>(u.w ? d.out_v : d.out_u), false);
        }
        break;
      }
      default:
        break;
    }
    if (tma_failed) break;  // uniform: every thread read the same abort flag
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&done[5 * u.x + u.y], 1);
    }
  }
}

// ---------------------------------------------------------------- launchers
inline int round_up32(int n) { return (n + 31) / 32 * 32; }

template <typename T>
struct Launch {
  static size_t row_smem(const Desc &d) {
    return sizeof(cx<T>) * (size_t)padded_len(d.rows_per_unit * d.M);
  }
  static size_t col_smem(const Desc &d) {
    return sizeof(cx<T>) * (size_t)padded_len(d.cols_per_unit * d.ny);
  }
  static int row_threads(const Desc &d) { return round_up32(d.rows_per_unit * (d.M / d.rp_row.e)); }
  static int col_threads(const Desc &d) { return round_up32(d.cols_per_unit * (d.ny / d.rp_col.e)); }
  static size_t small_smem(const Desc &d) {
    const size_t spec = (size_t)(d.M + 1) * d.ny * small_nspec(d);
    const size_t x1 = padded_len(d.small_rows * d.M), x2 = padded_len(d.small_cols * d.ny);
    return sizeof(cx<T>) * (spec + (x1 > x2 ? x1 : x2));
  }
  static int small_threads(const Desc &d) {
    const int a = d.small_rows * (d.M / d.rp_row.e), b = d.small_cols * (d.ny / d.rp_col.e);
    return round_up32(a > b ? a : b);
  }
  static cudaError_t set_smem(const void *fn, size_t bytes) {
    // prefer the largest shared-memory carveout so several CTAs fit per SM
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout,
                                         (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess || bytes <= 48 * 1024) return e;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  }
  // power-of-two FP32 kernels with compile-time lengths, when the plan's tile
  // shapes are the ones they were compiled for
  static PassKernel p2_row(const Desc &d, bool c2r) {
    if (sizeof(T) != 4 || d.rp_row.e != 16 || !p2_row_ok(d.M) || d.rows_per_unit != p2_row_cnt(d.M))
      return nullptr;
    return c2r ? p2_c2r_f32(d.M) : p2_r2c_f32(d.M);
  }
  // FP32 3 x 2^k / 5 x 2^k kernels with compile-time lengths, same condition
  static PassKernel mx_row(const Desc &d, bool c2r) {
    if (sizeof(T) != 4 || !mx_row_ok(d.M) || d.rp_row.e != mx_e(d.M) || d.rows_per_unit != mx_row_cnt(d.M))
      return nullptr;
    return c2r ? mx_c2r_f32(d.M) : mx_r2c_f32(d.M);
  }
  static PassKernel p2_col(const Desc &d) {
    if (sizeof(T) != 4 || d.rp_col.e != 16 || !p2_col_ok(d.ny) || d.cols_per_unit != p2_col_cnt(d.ny))
      return nullptr;
    return col_two_fields(d) ? p2_col2_f32(d.ny) : p2_col1_f32(d.ny);
  }

  static cudaError_t launch(PassKernel k, int grid, int threads, size_t sm, const Desc &d,
                            cudaStream_t s, int cls) {
    if (!k) return cudaErrorInvalidConfiguration;
    cudaError_t e = set_smem((const void *)k, sm);
    if (e != cudaSuccess) return e;
    ProfScope ps(cls, s);
    k<<<grid, threads, sm, s>>>(d);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
  }
  // forward pass over the real field(s): fields = 1 or 2
  static cudaError_t rows(const Desc &d, int fields, cudaStream_t s) {
    if (sizeof(T) == 4 && rows_tma_ok(d, fields, false)) return rows_tma_launch(d, fields, false, s);
    PassKernel k = p2_row(d, false);
    if (!k) k = mx_row(d, false);
    if (!k) k = pass_kernels<T>(d.rp_row.e).r2c;
    return launch(k, d.n_row_units * fields, row_threads(d), row_smem(d), d, s, PC_R2C);
  }
  static cudaError_t cols(const Desc &d_in, cudaStream_t s) {
    Desc d = d_in;
    fill_op_consts(d);
    // advances with a constant source: their own instantiations
    if (d.flags & F_SOURCE) {
      PassKernel k = nullptr;
      if (sizeof(T) == 4 && d.rp_col.e == 16 && p2_col_ok(d.ny) && d.cols_per_unit == p2_col_cnt(d.ny))
        k = p2_cols_f32(d.ny, col_two_fields(d));
      if (!k) k = pass_kernels<T>(d.rp_col.e).cols;
      return launch(k, d.n_col_units, col_threads(d), col_smem(d), d, s, PC_COL);
    }
    // measured variant: split-BF16 tensor-core first stage (advances only)
    if (sizeof(T) == 4 && tc_variant_requested() && !col_two_fields(d) && d.rp_col.e == 16 &&
        (d.op == OP_DIFF_ADV || d.op == OP_WAVE_ADV)) {
      size_t sm = 0;
      PassKernel k = p2_col_tc_f32(d.ny, &sm);
      if (k) return launch(k, d.M + 1, d.ny / 16, sm, d, s, PC_COL);
    }
    // TMA-staged persistent kernel for single-field FP32 power-of-two columns
    if (sizeof(T) == 4 && !col_two_fields(d) && p2_col(d) && tma_enabled()) {
      PassKernel k = p2_col_tma_f32(d.ny);
      const size_t sm = p2_col_tma_smem(d.ny);
      cudaError_t e = set_smem((const void *)k, sm);
      if (e != cudaSuccess) return e;
      int per_sm = 0, sms = 0, dev = 0;
      const int threads = d.cols_per_unit * (d.ny / 16);
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, sm);
      if (e == cudaSuccess) e = cudaGetDevice(&dev);
      if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return e;
      int grid = sms * (per_sm > 0 ? per_sm : 1);
      if (grid > d.n_col_units) grid = d.n_col_units;
      ProfScope ps(PC_COL, s);
      k<<<grid, threads, sm, s>>>(d);
      g_launches.fetch_add(1, std::memory_order_relaxed);
      return cudaGetLastError();
    }
    PassKernel k = p2_col(d);
    if (!k && sizeof(T) == 4 && !col_two_fields(d) && mx_col_ok(d.ny) && d.rp_col.e == mx_e(d.ny))
      k = mx_col1_f32(d.ny);
    if (!k) {
      const PassKernels pk = pass_kernels<T>(d.rp_col.e);
      k = col_two_fields(d) ? pk.col2 : pk.col1;
    }
    return launch(k, d.n_col_units, col_threads(d), col_smem(d), d, s, PC_COL);
  }
  static cudaError_t c2r(const Desc &d, int fields, cudaStream_t s) {
    if (sizeof(T) == 4 && rows_tma_ok(d, fields, true)) return rows_tma_launch(d, fields, true, s);
    PassKernel k = p2_row(d, true);
    if (!k) k = mx_row(d, true);
    if (!k) k = pass_kernels<T>(d.rp_row.e).c2r;
    return launch(k, d.n_row_units * fields, row_threads(d), row_smem(d), d, s, PC_C2R);
  }
  static cudaError_t factor(const Desc &d, cudaStream_t s) {
    ProfScope ps(PC_FACTOR, s);
    k_factor<T><<<d.n_fac_units, 256, 0, s>>>(d);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
  }
  static cudaError_t small(const Desc &d_in, cudaStream_t s) {
    Desc d = d_in;
    fill_op_consts(d);
    const size_t sm = small_smem(d);
    cudaError_t e = set_smem((const void *)k_small<T>, sm);
    if (e != cudaSuccess) return e;
    ProfScope ps(PC_SMALL, s);
    k_small<T><<<1, small_threads(d), sm, s>>>(d);
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
  }
  typedef void (*BatchKernel)(const Desc *, const int4 *, int, int *, int *, unsigned long long);
  static BatchKernel batch_kernel(int threads) {
    return threads == 128 ? k_batch<T, 128> : (threads == 256 ? k_batch<T, 256> : k_batch<T, kMaxThreads>);
  }
  // high_priority: the launch's CTAs are dispatched before those of
  // concurrently pending default-priority work (a launch attribute, kept
  // when the launch is captured into a graph)
  static cudaError_t batch(const Desc *descs, const int4 *units, int n_units, int *ctl, int *done,
                           int grid, int threads, size_t smem, unsigned long long wait_ns, cudaStream_t s,
                           bool high_priority = false) {
    BatchKernel k = batch_kernel(threads);
    cudaError_t e = set_smem((const void *)k, smem);
    if (e != cudaSuccess) return e;
    if (!high_priority) {
      k<<<grid, threads, smem, s>>>(descs, units, n_units, ctl, done, wait_ns);
    } else {
      int least = 0, greatest = 0;
      e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
      if (e != cudaSuccess) return e;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(grid);
      cfg.blockDim = dim3(threads);
      cfg.dynamicSmemBytes = smem;
      cfg.stream = s;
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributePriority;
      attr[0].val.priority = greatest;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      e = cudaLaunchKernelEx(&cfg, k, descs, units, n_units, ctl, done, wait_ns);
      if (e != cudaSuccess) return e;
    }
    g_launches.fetch_add(1, std::memory_order_relaxed);
    return cudaGetLastError();
  }
  static cudaError_t batch_occupancy(int threads, size_t smem, int *per_sm) {
    BatchKernel k = batch_kernel(threads);
    cudaError_t e = set_smem((const void *)k, smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k, threads, smem);
  }
};

}  // namespace fs
