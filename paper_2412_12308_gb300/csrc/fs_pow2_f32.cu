// FP32 pass kernels specialised for power-of-two lengths (see fs_pow2.h).
#include "fs_col_tma.cuh"
#include "fs_pow2.h"
#include "fs_row_async.cuh"
#include "fs_tma.cuh"
#include "fs_units.cuh"

namespace fs {

namespace {
template <int THREADS>
constexpr int min_blocks() {
  return THREADS >= 512 ? 2 : (THREADS >= 256 ? 3 : 6);
}
}  // namespace

template <int M>
struct RowK {
  static constexpr int CC = p2_row_cnt(M);
  static constexpr int THREADS = CC * (M / 16);
};
template <int L>
struct ColK {
  static constexpr int CC = p2_col_cnt(L);
  static constexpr int THREADS = CC * (L / 16);
};

template <int M>
__global__ void __launch_bounds__(RowK<M>::THREADS, min_blocks<RowK<M>::THREADS>()) k_r2c_p2(const Desc d) {
  extern __shared__ __align__(16) unsigned char fs_smem[];
  int unit = blockIdx.x;
  const float *in = reinterpret_cast<const float *>(d.in_u);
  cx<float> *spec = reinterpret_cast<cx<float> *>(d.work_u);
  if (unit >= d.n_row_units) {
    unit -= d.n_row_units;
    in = reinterpret_cast<const float *>(d.in_v);
    spec = reinterpret_cast<cx<float> *>(d.work_v);
  }
  unit_row_r2c_t<float, 16, M, RowK<M>::CC>(d, unit, RowK<M>::CC, reinterpret_cast<cx<float> *>(fs_smem), in,
                                           spec);
}

template <int M>
__global__ void __launch_bounds__(RowK<M>::THREADS, min_blocks<RowK<M>::THREADS>()) k_c2r_p2(const Desc d) {
  extern __shared__ __align__(16) unsigned char fs_smem[];
  int unit = blockIdx.x;
  const cx<float> *spec = reinterpret_cast<const cx<float> *>(d.work_u);
  float *out = reinterpret_cast<float *>(d.out_u);
  if (unit >= d.n_row_units) {
    unit -= d.n_row_units;
    spec = reinterpret_cast<const cx<float> *>(d.work_v);
    out = reinterpret_cast<float *>(d.out_v);
  }
  unit_row_c2r_t<float, 16, M, RowK<M>::CC>(d, unit, RowK<M>::CC, reinterpret_cast<cx<float> *>(fs_smem), spec,
                                           out, false);
}

// 128 registers per thread where a tile would otherwise spill: two-field
// kernels (two 256-thread CTAs or one 512-thread CTA per SM) and the
// 512-thread length-8192 kernels (one CTA per SM; measured at 8192^2: column
// pass 436 -> 418 us, no spills)
template <int L, bool TWO>
__global__ void __launch_bounds__(ColK<L>::THREADS, TWO ? (ColK<L>::THREADS >= 512 ? 1 : 2)
                                                        : (ColK<L>::THREADS >= 512 ? 1 : min_blocks<ColK<L>::THREADS>())) k_col_p2(const Desc d) {
  extern __shared__ __align__(16) unsigned char fs_smem[];
  unit_col_t<float, 16, TWO, L, ColK<L>::CC>(d, blockIdx.x, ColK<L>::CC, reinterpret_cast<cx<float> *>(fs_smem),
                                             reinterpret_cast<cx<float> *>(d.work_u),
                                             reinterpret_cast<cx<float> *>(d.work_v), false);
}

// ---------------------------------------------------------------- complex rows
template <int N>
struct C2CK {
  static constexpr int CC = p2_c2c_cnt(N);
  static constexpr int THREADS = CC * (N / 16);
};
template <int N>
__global__ void __launch_bounds__(C2CK<N>::THREADS, min_blocks<C2CK<N>::THREADS>()) k_c2cf_p2(const Desc d) {
  extern __shared__ __align__(16) unsigned char fs_smem[];
  int unit = blockIdx.x;
  const bool second = unit >= d.n_row_units;
  if (second) unit -= d.n_row_units;
  unit_row_c2c_t<float, 16, N, C2CK<N>::CC>(d, unit, C2CK<N>::CC, reinterpret_cast<cx<float> *>(fs_smem),
                                            reinterpret_cast<const cx<float> *>(second ? d.in_v : d.in_u),
                                            reinterpret_cast<cx<float> *>(second ? d.work_v : d.work_u),
                                            nullptr, false);
}
template <int N>
__global__ void __launch_bounds__(C2CK<N>::THREADS, min_blocks<C2CK<N>::THREADS>()) k_c2ci_p2(const Desc d) {
  extern __shared__ __align__(16) unsigned char fs_smem[];
  unit_row_c2c_t<float, 16, N, C2CK<N>::CC>(d, blockIdx.x, C2CK<N>::CC, reinterpret_cast<cx<float> *>(fs_smem),
                                            nullptr, reinterpret_cast<cx<float> *>(d.work_u),
                                            reinterpret_cast<cx<float> *>(d.out_u), true);
}

template <int L>
struct ColT {
  static constexpr int CC = p2_col_cnt(L);
  static constexpr int THREADS = CC * (L / 16);
  static constexpr int PLEN = (padded_len(CC * L) + 1) & ~1;  // even: keeps buffer 1 16-byte aligned
};

template <int L>
__global__ void __launch_bounds__(ColT<L>::THREADS, ColT<L>::THREADS >= 512 ? 1 : min_blocks<ColT<L>::THREADS>()) k_col_tma(const Desc d) {
  extern __shared__ __align__(128) unsigned char fs_smem[];
  __shared__ uint64_t bars[2];
  __shared__ int s_abort;
  cx<float> *b0 = reinterpret_cast<cx<float> *>(fs_smem);
  if (threadIdx.x == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    fence_mbar_init();
  }
  uint32_t ph = 0;
  constexpr int CC = ColT<L>::CC;
  col_tma_groups<L, CC>(d, blockIdx.x * CC, gridDim.x * CC, d.M + 1, CC, b0, b0 + ColT<L>::PLEN, bars, ph,
                        &s_abort);
}

#define FS_P2_ROWS(X) X(128) X(256) X(512) X(1024) X(2048) X(4096)
#define FS_P2_COLS(X) X(128) X(256) X(512) X(1024) X(2048) X(4096) X(8192)

// ---------------------------------------------------------------- device dispatch for batch / small paths
// row tiles of the standalone kernels (CC = p2_row_cnt(M)) and of 256-thread
// batch CTAs (CC = 256 / (M/16) where that is smaller)
template <int M, int CC = RowK<M>::CC>
__device__ __noinline__ void p2_r2c_unit(const Desc &d, int unit, cx<float> *sm, const float *in, cx<float> *spec) {
  unit_row_r2c_t<float, 16, M, CC>(d, unit, CC, sm, in, spec);
}
template <int M, int CC = RowK<M>::CC>
__device__ __noinline__ void p2_c2r_unit(const Desc &d, int unit, cx<float> *sm, const cx<float> *spec, float *out,
                                         bool sh) {
  unit_row_c2r_t<float, 16, M, CC>(d, unit, CC, sm, spec, out, sh);
}
template <int L>
__device__ __noinline__ void p2_col1_unit(const Desc &d, int unit, int cnt, cx<float> *sm, cx<float> *wu,
                                          cx<float> *wv, bool sh) {
  unit_col_t<float, 16, false, L, 0>(d, unit, cnt, sm, wu, wv, sh);
}

// a row unit of tile height CC when the runtime count is CC (CC = 0: none)
template <int M, int CC>
__device__ __forceinline__ bool p2_r2c_try(const Desc &d, int unit, int cnt, cx<float> *sm, const float *in,
                                           cx<float> *spec) {
  if constexpr (CC > 0) {
    if (cnt == CC) {
      p2_r2c_unit<M, CC>(d, unit, sm, in, spec);
      return true;
    }
  }
  return false;
}
template <int M, int CC>
__device__ __forceinline__ bool p2_c2r_try(const Desc &d, int unit, int cnt, cx<float> *sm, const cx<float> *spec,
                                           float *out, bool sh) {
  if constexpr (CC > 0) {
    if (cnt == CC) {
      p2_c2r_unit<M, CC>(d, unit, sm, spec, out, sh);
      return true;
    }
  }
  return false;
}

// Staged R2C row tiles of a batch unit (F_R2C_STAGED): called, not inlined,
// so that the batch kernel's own code stays small.
template <int M, int CC>
__device__ __noinline__ void p2_r2c_staged_l(const Desc &d, int tile0, int tile1, cx<float> *sm, const float *in,
                                             cx<float> *spec) {
  r2c_staged_tiles<M, CC>(d, tile0, tile1, sm, in, spec);
}
template <int M, int CC>
__device__ __forceinline__ bool p2_r2c_staged_try(const Desc &d, int tile0, int tile1, int cnt, cx<float> *sm,
                                                  const float *in, cx<float> *spec) {
  if constexpr (CC > 0) {
    if (cnt == CC) {
      p2_r2c_staged_l<M, CC>(d, tile0, tile1, sm, in, spec);
      return true;
    }
  }
  return false;
}
__device__ bool p2_r2c_staged_unit(const Desc &d, int tile0, int tile1, int cnt, cx<float> *sm, const float *in,
                                   cx<float> *spec) {
  if (d.rp_row.e != 16) return false;
  switch (d.M) {
#define C(m)                                                                                                   \
  case m:                                                                                                      \
    return p2_r2c_staged_try<m, p2_row_cnt(m)>(d, tile0, tile1, cnt, sm, in, spec) ||                         \
           p2_r2c_staged_try<m, (p2_row_cnt_256(m) != p2_row_cnt(m) ? p2_row_cnt_256(m) : 0)>(d, tile0, tile1, \
                                                                                              cnt, sm, in, spec) || \
           p2_r2c_staged_try<m, (p2_row_cnt_128(m) != p2_row_cnt_256(m) ? p2_row_cnt_128(m) : 0)>(            \
               d, tile0, tile1, cnt, sm, in, spec);
    FS_P2_ROWS(C)
#undef C
    default:
      return false;
  }
}

// tile heights: standalone kernels, 256-thread and 128-thread batch CTAs
__device__ bool p2_unit_r2c(const Desc &d, int unit, int cnt, cx<float> *sm, const float *in, cx<float> *spec) {
  if (d.rp_row.e != 16) return false;
  switch (d.M) {
#define C(m)                                                                                           \
  case m:                                                                                              \
    return p2_r2c_try<m, p2_row_cnt(m)>(d, unit, cnt, sm, in, spec) ||                                 \
           p2_r2c_try<m, (p2_row_cnt_256(m) != p2_row_cnt(m) ? p2_row_cnt_256(m) : 0)>(d, unit, cnt, sm, in, \
                                                                                      spec) ||         \
           p2_r2c_try<m, (p2_row_cnt_128(m) != p2_row_cnt_256(m) ? p2_row_cnt_128(m) : 0)>(d, unit, cnt, sm,  \
                                                                                         in, spec);
    FS_P2_ROWS(C)
#undef C
    default:
      return false;
  }
}
__device__ bool p2_unit_c2r(const Desc &d, int unit, int cnt, cx<float> *sm, const cx<float> *spec, float *out,
                            bool sh) {
  if (d.rp_row.e != 16) return false;
  switch (d.M) {
#define C(m)                                                                                              \
  case m:                                                                                                 \
    return p2_c2r_try<m, p2_row_cnt(m)>(d, unit, cnt, sm, spec, out, sh) ||                               \
           p2_c2r_try<m, (p2_row_cnt_256(m) != p2_row_cnt(m) ? p2_row_cnt_256(m) : 0)>(d, unit, cnt, sm, spec, \
                                                                                      out, sh) ||         \
           p2_c2r_try<m, (p2_row_cnt_128(m) != p2_row_cnt_256(m) ? p2_row_cnt_128(m) : 0)>(d, unit, cnt, sm,   \
                                                                                         spec, out, sh);
    FS_P2_ROWS(C)
#undef C
    default:
      return false;
  }
}
__device__ bool p2_unit_col1(const Desc &d, int unit, int cnt, cx<float> *sm, cx<float> *wu, cx<float> *wv,
                             bool sh) {
  if (d.rp_col.e != 16) return false;
  switch (d.ny) {
#define C(l)                                           \
  case l:                                              \
    p2_col1_unit<l>(d, unit, cnt, sm, wu, wv, sh);     \
    return true;
    FS_P2_COLS(C)
#undef C
    default:
      return false;
  }
}

size_t p2_col1_tma_unit_smem(int L, int cnt) {
  return 2 * (size_t)((padded_len(cnt * L) + 1) & ~1) * sizeof(cx<float>);
}

PassKernel p2_r2c_f32(int M) {
  switch (M) {
#define C(m) \
  case m:    \
    return k_r2c_p2<m>;
    FS_P2_ROWS(C)
#undef C
    default:
      return nullptr;
  }
}
PassKernel p2_c2r_f32(int M) {
  switch (M) {
#define C(m) \
  case m:    \
    return k_c2r_p2<m>;
    FS_P2_ROWS(C)
#undef C
    default:
      return nullptr;
  }
}
PassKernel p2_col1_f32(int L) {
  switch (L) {
#define C(l) \
  case l:    \
    return k_col_p2<l, false>;
    FS_P2_COLS(C)
#undef C
    default:
      return nullptr;
  }
}
PassKernel p2_c2c_f32(int N, bool inverse) {
  switch (N) {
#define C(n) \
  case n:    \
    return inverse ? k_c2ci_p2<n> : k_c2cf_p2<n>;
    C(128) C(256) C(512) C(1024) C(2048) C(4096) C(8192)
#undef C
    default:
      return nullptr;
  }
}

PassKernel p2_col_tma_f32(int L) {
  switch (L) {
#define C(l) \
  case l:    \
    return k_col_tma<l>;
    FS_P2_COLS(C)
#undef C
    default:
      return nullptr;
  }
}
size_t p2_col_tma_smem(int L) {
  const int cc = p2_col_cnt(L);
  return 2 * (size_t)((padded_len(cc * L) + 1) & ~1) * 8;
}

PassKernel p2_col2_f32(int L) {
  switch (L) {
#define C(l) \
  case l:    \
    return k_col_p2<l, true>;
    FS_P2_COLS(C)
#undef C
    default:
      return nullptr;
  }
}

}  // namespace fs
