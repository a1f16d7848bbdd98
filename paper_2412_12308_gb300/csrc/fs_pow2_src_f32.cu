// FP32 column kernels for advances with a constant source (F_SOURCE),
// specialised for power-of-two lengths like fs_pow2_f32.cu: the column unit
// instantiated with the source term, the length and the columns per CTA fixed
// at compile time.  Kept in their own translation unit so that they compile in
// parallel with the source-free kernels and leave those unchanged.
#include "fs_pow2.h"
#include "fs_units.cuh"

namespace fs {

template <int L>
struct ColS {
  static constexpr int CC = p2_col_cnt(L);
  static constexpr int THREADS = CC * (L / 16);
  static constexpr int MINB = THREADS >= 512 ? 2 : (THREADS >= 256 ? 3 : 6);
};

template <int L, bool TWO>
__global__ void __launch_bounds__(ColS<L>::THREADS, TWO ? (ColS<L>::THREADS >= 512 ? 1 : 2) : ColS<L>::MINB)
    k_col_p2s(const Desc d) {
  extern __shared__ __align__(16) unsigned char fs_smem[];
  unit_col_t<float, 16, TWO, L, ColS<L>::CC, true>(d, blockIdx.x, ColS<L>::CC,
                                                   reinterpret_cast<cx<float> *>(fs_smem),
                                                   reinterpret_cast<cx<float> *>(d.work_u),
                                                   reinterpret_cast<cx<float> *>(d.work_v), false);
}

template <int L, bool TWO>
__device__ __noinline__ void p2_cols_unit(const Desc &d, int unit, int cnt, cx<float> *sm, cx<float> *wu,
                                          cx<float> *wv, bool sh) {
  unit_col_t<float, 16, TWO, L, 0, true>(d, unit, cnt, sm, wu, wv, sh);
}

#define FS_P2S_COLS(X) X(128) X(256) X(512) X(1024) X(2048) X(4096) X(8192)

__device__ bool p2_unit_cols(const Desc &d, int unit, int cnt, cx<float> *sm, cx<float> *wu, cx<float> *wv,
                             bool sh) {
  if (d.rp_col.e != 16) return false;
  const bool two = col_two_fields(d);
  switch (d.ny) {
#define C(l)                                                    \
  case l:                                                       \
    if (two)                                                    \
      p2_cols_unit<l, true>(d, unit, cnt, sm, wu, wv, sh);      \
    else                                                        \
      p2_cols_unit<l, false>(d, unit, cnt, sm, wu, wv, sh);     \
    return true;
    FS_P2S_COLS(C)
#undef C
    default:
      return false;
  }
}

PassKernel p2_cols_f32(int L, bool two) {
  switch (L) {
#define C(l) \
  case l:    \
    return two ? k_col_p2s<l, true> : k_col_p2s<l, false>;
    FS_P2S_COLS(C)
#undef C
    default:
      return nullptr;
  }
}

}  // namespace fs
