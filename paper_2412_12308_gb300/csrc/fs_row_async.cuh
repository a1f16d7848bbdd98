// fs_row_async.cuh -- C2R row tiles of the batch kernel staged into shared
// memory by asynchronous copies (FP32, an even number of rows per tile;
// power-of-two row lengths with register tile 16, 3 x 2^k / 5 x 2^k lengths
// with their family's tile, 24 / 20, instantiated in fs_mixed_f32.cu).
#pragma once
#include "fs_tma.cuh"
#include "fs_units.cuh"

namespace fs {

// 16-byte global -> shared copy that bypasses L1 (.cg), as every load of
// data produced inside a persistent launch does
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most N of this thread's committed copy groups are pending
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Elements of one staging buffer: the tile [a][r] (a = 0..M, r < cnt)
// unpadded, or the padded FFT exchange of the same rows, whichever is larger;
// even, so that the second buffer starts 16-byte aligned.
__host__ __device__ constexpr int c2r_stage_len(int M, int cnt) {
  return ((padded_len(M * cnt) > (M + 1) * cnt ? padded_len(M * cnt) : (M + 1) * cnt) + 1) & ~1;
}

// One staged C2R tile in `cur` ([a][row], unpadded), which then doubles as
// the FFT exchange area: rows tile*CC .. of the output.
// (t, rho): the thread's slot and row in the tile.
template <int M, int CC>
__device__ __forceinline__ void c2r_staged_tile(const Desc &d, int tile, cx<float> *cur, float *out, int t,
                                                int rho) {
  constexpr int E = mx_e(M) ? mx_e(M) : 16, Tseg = M / E;
  const int y = tile * CC + rho;
  const bool active = (t < Tseg) && (y < d.ny);
  cx<float> v[E];
  cx<float> xM = zero_cx<float>();
  if (active) {
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = cur[rho + (t + Tseg * s) * CC];
    if (t == 0) xM = cur[rho + M * CC];
  } else {
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = zero_cx<float>();
  }
  c2r_tile_finish<float, E, M, CC>(d, tile, CC, t, rho, active, v, xM,
                                   [&](int j) { return cur[rho + j * CC]; }, cur, out);
}
// the same out of line (a caller that keeps the copy loop's state in few registers)
template <int M, int CC>
__device__ __noinline__ void c2r_staged_tile_ool(const Desc &d, int tile, cx<float> *cur, float *out, int t,
                                                 int rho) {
  c2r_staged_tile<M, CC>(d, tile, cur, out, t, rho);
}

// Row tiles tile0 .. tile1-1 (CC rows each) of one field.  The tile after the
// current one is copied in while the current one is transformed (two
// buffers); a thread's copies complete without polling (cp.async.wait_group),
// and the barrier after the wait makes every thread's copies visible.  The
// current buffer then doubles as the FFT exchange area.  Rows past ny (a
// ragged last tile) are neither copied nor stored.
template <int M, int CC, bool OOL = false>
__device__ __forceinline__ void c2r_staged_tiles(const Desc &d, int tile0, int tile1, cx<float> *sm,
                                                 const cx<float> *spec, float *out) {
  static_assert(CC % 2 == 0, "a 16-byte copy moves two rows of one frequency");
  constexpr int LEN = c2r_stage_len(M, CC), HALF = CC / 2;
  const int ny = d.ny, tid = threadIdx.x, nthr = blockDim.x;
  const int t = tid / CC, rho = tid - t * CC;
  auto issue = [&](cx<float> *b, int tile) {
    const int y0 = tile * CC, rows = min(CC, ny - y0);  // even: ny and CC are even
#pragma unroll 1
    for (int idx = tid; idx < (M + 1) * HALF; idx += nthr) {
      const int a = idx / HALF, r = 2 * (idx - a * HALF);
      if (r < rows) cp_async16(b + a * CC + r, spec + (size_t)a * ny + y0 + r);
    }
    cp_async_commit();
  };
  issue(sm, tile0);
  for (int tile = tile0, i = 0; tile < tile1; ++tile, ++i) {
    cx<float> *cur = (i & 1) ? sm + LEN : sm;
    if (tile + 1 < tile1) {
      issue((i & 1) ? sm : sm + LEN, tile + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    if constexpr (OOL)
      c2r_staged_tile_ool<M, CC>(d, tile, cur, out, t, rho);
    else
      c2r_staged_tile<M, CC>(d, tile, cur, out, t, rho);
  }
}

// Elements of one R2C staging buffer: the tile's real rows as pairs, row r
// at r * r2c_row_stride (a pad after each row keeps the threads' reads of
// their row's slots on distinct banks), or the padded FFT exchange of the
// same rows, whichever is larger; even (16-byte aligned second buffer).
__host__ __device__ constexpr int r2c_row_stride(int M, int cnt) { return M + (cnt <= 8 ? 16 / cnt : 2); }
__host__ __device__ constexpr int r2c_stage_len(int M, int cnt) {
  return ((padded_len(M * cnt) > cnt * r2c_row_stride(M, cnt) ? padded_len(M * cnt) : cnt * r2c_row_stride(M, cnt)) +
          1) & ~1;
}

// One staged R2C tile: rows tile*CC .. of the tile copied into `cur` (row r
// at r * r2c_row_stride), which then doubles as the FFT exchange area.  Kept
// out of line so that the copy loop around it holds few registers.
template <int M, int CC>
__device__ __noinline__ void r2c_staged_tile(const Desc &d, int tile, cx<float> *cur, cx<float> *spec) {
  constexpr int E = mx_e(M) ? mx_e(M) : 16, Tseg = M / E, RS = r2c_row_stride(M, CC);
  const int tid = threadIdx.x;
  const int t = tid / CC, rho = tid - t * CC;
  const int y = tile * CC + rho;
  const bool active = (t < Tseg) && (y < d.ny);
  cx<float> v[E];
  if (active) {
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = cur[rho * RS + t + Tseg * s];
  } else {
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = zero_cx<float>();
  }
  // no barrier here: the transform's first exchange store into `cur` comes
  // after its own barrier, which every read above precedes
  r2c_tile_finish<float, E, M, CC>(d, CC, t, rho, y, active, v, cur, spec);
}

// Row R2C tiles tile0 .. tile1-1 (CC rows each) of one real field.  A
// tile's rows are one contiguous run of the field; it is copied into shared
// memory by 16-byte asynchronous copies (two pairs of one row each) while the
// previous tile is transformed (two buffers).  Needs `in` 16-byte aligned
// (the host checks); rows past ny (a ragged last tile) are neither copied
// nor stored.
template <int M, int CC>
__device__ __forceinline__ void r2c_staged_tiles(const Desc &d, int tile0, int tile1, cx<float> *sm,
                                                 const float *in, cx<float> *spec) {
  constexpr int LEN = r2c_stage_len(M, CC), RS = r2c_row_stride(M, CC), Q = M / 2;  // 16-byte chunks per row
  const int ny = d.ny, tid = threadIdx.x, nthr = blockDim.x;
  auto issue = [&](cx<float> *b, int tile) {
    const int y0 = tile * CC, rows = min(CC, ny - y0);
    const float *src = in + (size_t)y0 * (2 * M);
#pragma unroll 1
    for (int idx = tid; idx < rows * Q; idx += nthr) {
      const int r = idx / Q, q = idx - r * Q;
      cp_async16(b + r * RS + 2 * q, src + (size_t)r * (2 * M) + 4 * q);
    }
    cp_async_commit();
  };
  issue(sm, tile0);
#pragma unroll 1
  for (int tile = tile0, i = 0; tile < tile1; ++tile, ++i) {
    cx<float> *cur = (i & 1) ? sm + LEN : sm;
    if (tile + 1 < tile1) {
      issue((i & 1) ? sm : sm + LEN, tile + 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    r2c_staged_tile<M, CC>(d, tile, cur, spec);
  }
}

template <int M, int CC>
__device__ __forceinline__ bool c2r_staged_try(const Desc &d, int tile0, int tile1, int cnt, cx<float> *sm,
                                               const cx<float> *spec, float *out) {
  if constexpr (CC > 0 && CC % 2 == 0) {
    if (cnt == CC) {
      c2r_staged_tiles<M, CC>(d, tile0, tile1, sm, spec, out);
      return true;
    }
  }
  return false;
}

// Dispatch on the row length and the tile height (the standalone kernels'
// p2_row_cnt, the 256- or 128-thread batch's p2_row_cnt_256 / _128); false
// when none is compiled.
__device__ __forceinline__ bool c2r_staged_unit(const Desc &d, int tile0, int tile1, int cnt, cx<float> *sm,
                                                const cx<float> *spec, float *out) {
  switch (d.M) {
#define FS_C2R_STAGED(m)                                                                    \
  case m:                                                                                   \
    if (c2r_staged_try<m, p2_row_cnt(m)>(d, tile0, tile1, cnt, sm, spec, out)) return true; \
    if constexpr (p2_row_cnt_256(m) != p2_row_cnt(m))                                       \
      if (c2r_staged_try<m, p2_row_cnt_256(m)>(d, tile0, tile1, cnt, sm, spec, out)) return true; \
    if constexpr (p2_row_cnt_128(m) > 0 && p2_row_cnt_128(m) != p2_row_cnt_256(m))          \
      return c2r_staged_try<m, p2_row_cnt_128(m)>(d, tile0, tile1, cnt, sm, spec, out);     \
    return false;
    FS_C2R_STAGED(128)
    FS_C2R_STAGED(256)
    FS_C2R_STAGED(512)
    FS_C2R_STAGED(1024)
    FS_C2R_STAGED(2048)
    FS_C2R_STAGED(4096)
#undef FS_C2R_STAGED
    default:
      return false;
  }
}

}  // namespace fs
