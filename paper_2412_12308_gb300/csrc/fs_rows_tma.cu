// fs_rows_tma.cu -- persistent row passes staged by the tensor memory
// accelerator (FP32, power-of-two row transforms of length M = nx/2 in
// {512, 1024, 2048, 4096}, register tile 16).
//
// Same arithmetic as the row units of fs_units.cuh (Sec. II.D first step and
// its inverse: the packed real x transforms, R2C post-process and C2R
// pre-process), with the data movement moved off the SM's load/store path:
//
//   R2C  a tile of R consecutive real rows is one contiguous run of the input:
//        R one-dimensional bulk copies (one per row, padded row pitch) bring
//        the NEXT tile into shared memory while the current one is
//        transformed; the half-spectrum tile [a][y0..y0+R-1] (R values per
//        x frequency, a = 0..M) is written by 2D tensor-map stores, boxes of
//        R x 256 frequencies, straight from a shared staging buffer.
//   C2R  the spectrum tile is fetched by 2D tensor-map loads (zero fill past
//        a = M), double-buffered the same way; the real rows go out as R
//        one-dimensional bulk stores.
//
// Threads map rho-fastest (rho = tid % R): spectrum-side shared accesses
// ([a][rho]) are then contiguous, and the padded row pitch (32 bytes extra)
// keeps the row-side ones free of bank conflicts.  One CTA (or two for short
// rows) per SM walks the tiles blockIdx.x, += gridDim.x.  Every mbarrier wait
// is bounded (kTmaWaitNs); on expiry the device error word is set and the CTA
// leaves after waiting, bounded again, for the copies it issued.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "fs_host.h"
#include "fs_kernels.cuh"

namespace fs {

namespace {

constexpr int cmax(int a, int b) { return a > b ? a : b; }
constexpr int round16(int n) { return (n + 15) & ~15; }  // complex elements: 128 bytes

// Rows per tile: 4 (32-byte spectrum runs) up to M = 2048, 2 at M = 4096
// (shared memory).  Measured at 4096^2: tiles of 2 rows (two CTAs per SM,
// 16-byte runs) took the R2C pass from 42.1 to 58.3 us, C2R unchanged.
constexpr int rt_rows(int M) { return M >= 4096 ? 2 : 4; }

template <int M, int R_>
struct RT {
  static constexpr int R = R_;
  static constexpr int E = 16, TSEG = M / E, THREADS = R * TSEG;
  static constexpr int P = M + 4;  // row pitch of staged real rows (complex pairs)
  static constexpr int XL = padded_len(R * M);
  static constexpr int BA = 256;  // tensor box extent along the x frequency
  static constexpr int NBOX = (M + 1 + BA - 1) / BA;
  static constexpr int SPEC_TILE = NBOX * BA * R;  // spectrum tile incl. the clipped tail
  static constexpr int BUF_R2C = round16(cmax(R * P, XL));
  static constexpr int BUF_C2R = round16(cmax(SPEC_TILE, XL));
  // + 128 bytes: the buffers start at the first 128-byte boundary of the
  // dynamic shared memory (tensor copies need 128-byte aligned addresses)
  static constexpr size_t SMEM_R2C = (size_t)(2 * BUF_R2C + SPEC_TILE) * 8 + 128;
  static constexpr size_t SMEM_C2R = (size_t)(2 * BUF_C2R + round16(R * P)) * 8 + 128;
  static_assert(SMEM_R2C <= 227 * 1024 && SMEM_C2R <= 227 * 1024, "shared memory");
  // CTAs per SM the shared memory admits (the register budget follows it)
  static constexpr int MINB = (int)((227 * 1024) / (SMEM_R2C > SMEM_C2R ? SMEM_R2C : SMEM_C2R));
};

__device__ __forceinline__ void tma_load_2d(void *smem, const CUtensorMap *tm, int c0, int c1, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(smem)),
      "l"(reinterpret_cast<uint64_t>(tm)), "r"(c0), "r"(c1), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap *tm, int c0, int c1, const void *smem) {
  asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                   reinterpret_cast<uint64_t>(tm)),
               "r"(c0), "r"(c1), "r"(smem_u32(smem))
               : "memory");
}
__device__ __forceinline__ void bulk_s2g(void *gmem, const void *smem, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gmem), "r"(smem_u32(smem)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// the bulk stores issued so far have finished reading shared memory
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// ... and have completed
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

// First 128-byte boundary of the dynamic shared memory (its base is only
// guaranteed 16-byte aligned).
__device__ __forceinline__ cx<float> *smem_base128(unsigned char *dyn) {
  return reinterpret_cast<cx<float> *>(dyn + ((128u - (smem_u32(dyn) & 127u)) & 127u));
}

// Shared per-CTA pipeline state: two mbarriers (one per landing buffer), the
// parity of their next completion, an abort flag.
struct Pipe {
  uint64_t bar[2];
  int abort;
};

__device__ __forceinline__ void pipe_init(Pipe *p) {
  if (threadIdx.x == 0) {
    mbar_init(&p->bar[0], 1);
    mbar_init(&p->bar[1], 1);
    p->abort = 0;
    fence_mbar_init();
  }
  __syncthreads();
}

// Every thread waits (bounded) for buffer k's copy; on expiry the error word is
// set and the CTA agrees to leave: thread 0 waits, bounded, for the copies
// still in flight (this buffer's, and the other buffer's if one was issued).
// Returns false when the CTA must leave.
__device__ __forceinline__ bool pipe_wait(Pipe *p, int k, uint32_t &ph, bool other_in_flight) {
  if (!mbar_wait_bounded(&p->bar[k], (ph >> k) & 1u, kTmaWaitNs)) {
    atomicExch(&g_fs_dev_error, FS_DEV_ERR_TMA_TIMEOUT);
    p->abort = 1;
  }
  ph ^= 1u << k;
  __syncthreads();
  if (p->abort) {
    if (threadIdx.x == 0) {
      mbar_wait_bounded(&p->bar[k], ((ph >> k) & 1u) ^ 1u, kTmaWaitNs);
      if (other_in_flight) mbar_wait_bounded(&p->bar[k ^ 1], (ph >> (k ^ 1)) & 1u, kTmaWaitNs);
      bulk_wait0();
    }
    return false;
  }
  return true;
}

}  // namespace

// ---------------------------------------------------------------- R2C
// Tiles T = 0 .. nfields * ntiles - 1 (field = T / ntiles); tile rows
// y0 = (T mod ntiles) * R.  tm_u / tm_v: 2D maps of the work spectra
// (inner dimension y: ny 8-byte elements, outer a: M + 1), box {R, 256}.
template <int M, int R_>
__global__ void __launch_bounds__(RT<M, R_>::THREADS, RT<M, R_>::MINB)
    k_r2c_tma(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_v, const Desc d,
              int nfields) {
  using C = RT<M, R_>;
  constexpr int R = C::R, E = C::E, TSEG = C::TSEG, P = C::P;
  extern __shared__ __align__(16) unsigned char fs_smem[];
  __shared__ Pipe pipe;
  cx<float> *buf0 = smem_base128(fs_smem);
  cx<float> *stg = buf0 + 2 * C::BUF_R2C;
  const int tid = threadIdx.x, t = tid / R, rho = tid - t * R;
  const int nx = d.nx, ntiles = d.ny / R, ntot = nfields * ntiles;
  const cx<float> *tw = reinterpret_cast<const cx<float> *>(d.tw_x);
  pipe_init(&pipe);
  auto issue = [&](int T, int k) {
    const int f = T / ntiles, y0 = (T - f * ntiles) * R;
    const float *src = reinterpret_cast<const float *>(f ? d.in_v : d.in_u) + (size_t)y0 * nx;
    cx<float> *dst = buf0 + k * C::BUF_R2C;
    mbar_arrive_expect_tx(&pipe.bar[k], (uint32_t)(R * nx * 4));
#pragma unroll
    for (int r = 0; r < R; ++r) bulk_g2s(dst + r * P, src + (size_t)r * nx, (uint32_t)(nx * 4), &pipe.bar[k]);
  };
  uint32_t ph = 0;
  if (tid == 0 && (int)blockIdx.x < ntot) issue(blockIdx.x, 0);
  int i = 0;
  for (int T = blockIdx.x; T < ntot; T += gridDim.x, ++i) {
    const int k = i & 1;
    cx<float> *cur = buf0 + k * C::BUF_R2C;
    const bool more = T + (int)gridDim.x < ntot;
    if (tid == 0 && more) issue(T + gridDim.x, k ^ 1);
    if (!pipe_wait(&pipe, k, ph, more)) return;
    const int f = T / ntiles, y0 = (T - f * ntiles) * R;
    cx<float> v[E];
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = cur[rho * P + t + TSEG * s];
    __syncthreads();  // the landing tile is read: the buffer becomes the exchange area
    fft_ct_from<float, E, M, R, 2, 0>(v, cur, rho, true, t, tw);
    __syncthreads();
#pragma unroll
    for (int s = 0; s < E; ++s) cur[padi(rho + (t + TSEG * s) * R)] = v[s];
    if (tid == 0) bulk_wait_read0();  // the previous tile's stores have read the staging buffer
    __syncthreads();
    // X_a = (Z_a + conj Z_{M-a})/2 + w^a (Z_a - conj Z_{M-a})/(2i), X_0 and X_M real
#pragma unroll
    for (int s = 0; s < E; ++s) {
      const int kk = t + TSEG * s;
      const cx<float> zk = v[s];
      if (kk == 0) {
        stg[rho] = mk<float>(zk.x + zk.y, 0.f);
        stg[M * R + rho] = mk<float>(zk.x - zk.y, 0.f);
      } else {
        const cx<float> zm = conj(cur[padi(rho + (M - kk) * R)]);
        const cx<float> ev = 0.5f * (zk + zm);
        const cx<float> df_ = zk - zm;
        const cx<float> od = mk<float>(0.5f * df_.y, -0.5f * df_.x);
        stg[kk * R + rho] = ev + cmul(tw[kk], od);
      }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      const CUtensorMap *tm = f ? &tm_v : &tm_u;
#pragma unroll 1
      for (int b = 0; b < C::NBOX; ++b) tma_store_2d(tm, y0, b * C::BA, stg + b * C::BA * R);
      bulk_commit();
    }
  }
  if (tid == 0) bulk_wait0();
}

// ---------------------------------------------------------------- C2R
// Tiles as above; out_u / out_v real rows, tm_u / tm_v the work spectra.
template <int M, int R_>
__global__ void __launch_bounds__(RT<M, R_>::THREADS, RT<M, R_>::MINB)
    k_c2r_tma(const __grid_constant__ CUtensorMap tm_u, const __grid_constant__ CUtensorMap tm_v, const Desc d,
              int nfields) {
  using C = RT<M, R_>;
  constexpr int R = C::R, E = C::E, TSEG = C::TSEG, P = C::P;
  extern __shared__ __align__(16) unsigned char fs_smem[];
  __shared__ Pipe pipe;
  cx<float> *buf0 = smem_base128(fs_smem);
  cx<float> *stg = buf0 + 2 * C::BUF_C2R;
  const int tid = threadIdx.x, t = tid / R, rho = tid - t * R;
  const int nx = d.nx, ntiles = d.ny / R, ntot = nfields * ntiles;
  const cx<float> *tw = reinterpret_cast<const cx<float> *>(d.tw_x);
  pipe_init(&pipe);
  auto issue = [&](int T, int k) {
    const int f = T / ntiles, y0 = (T - f * ntiles) * R;
    const CUtensorMap *tm = f ? &tm_v : &tm_u;
    cx<float> *dst = buf0 + k * C::BUF_C2R;
    mbar_arrive_expect_tx(&pipe.bar[k], (uint32_t)(C::SPEC_TILE * 8));
#pragma unroll 1
    for (int b = 0; b < C::NBOX; ++b) tma_load_2d(dst + b * C::BA * R, tm, y0, b * C::BA, &pipe.bar[k]);
  };
  uint32_t ph = 0;
  if (tid == 0 && (int)blockIdx.x < ntot) issue(blockIdx.x, 0);
  int i = 0;
  for (int T = blockIdx.x; T < ntot; T += gridDim.x, ++i) {
    const int k = i & 1;
    cx<float> *cur = buf0 + k * C::BUF_C2R;
    const bool more = T + (int)gridDim.x < ntot;
    if (tid == 0 && more) issue(T + gridDim.x, k ^ 1);
    if (!pipe_wait(&pipe, k, ph, more)) return;
    const int f = T / ntiles, y0 = (T - f * ntiles) * R;
    cx<float> v[E];
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = cur[(t + TSEG * s) * R + rho];
    const cx<float> xM = t == 0 ? cur[M * R + rho] : zero_cx<float>();
    // F_a = X_a + conj X_{M-a}, G_a = (X_a - conj X_{M-a}) e^{+2 pi i a/nx};
    // the inverse transform of F + iG, by conjugation, gives x_{2m} + i x_{2m+1}
#pragma unroll
    for (int s = 0; s < E; ++s) {
      const int kk = t + TSEG * s;
      cx<float> xk = v[s], xm;
      if (kk == 0) {
        xk = mk<float>(xk.x, 0.f);
        xm = mk<float>(xM.x, 0.f);
      } else {
        xm = conj(cur[(M - kk) * R + rho]);
      }
      const cx<float> fa = xk + xm;
      const cx<float> g = cmul(xk - xm, conj(tw[kk]));
      v[s] = mk<float>(fa.x - g.y, -(fa.y + g.x));
    }
    // the engine's first exchange store follows its own barrier, which every
    // read of the landing tile above precedes
    fft_ct_from<float, E, M, R, 2, 0>(v, cur, rho, true, t, tw);
    if (tid == 0) bulk_wait_read0();  // the previous tile's row stores have read the staging rows
    __syncthreads();
#pragma unroll
    for (int s = 0; s < E; ++s) stg[rho * P + t + TSEG * s] = conj(v[s]);
    fence_proxy_async_smem();
    __syncthreads();
    if (tid == 0) {
      float *dst = reinterpret_cast<float *>(f ? d.out_v : d.out_u) + (size_t)y0 * nx;
#pragma unroll
      for (int r = 0; r < R; ++r) bulk_s2g(dst + (size_t)r * nx, stg + r * P, (uint32_t)(nx * 4));
      bulk_commit();
    }
  }
  if (tid == 0) bulk_wait0();
}

// ---------------------------------------------------------------- host side
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess)
      p = nullptr;
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }();
  return fn;
}

// The half spectrum [M+1][ny] of complex floats as a 2D tensor of 8-byte
// elements (inner y, outer a), box {R, 256}; reads past a = M fill zeros and
// stores there are dropped.
bool spec_map(CUtensorMap *tm, void *spec, int ny, int M, int R) {
  memset(tm, 0, sizeof *tm);
  if (!spec) return true;  // unused field: an all-zero map is never dereferenced
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)ny, (cuuint64_t)(M + 1)};
  const cuuint64_t strides[1] = {(cuuint64_t)ny * 8};
  const cuuint32_t box[2] = {(cuuint32_t)R, 256u};
  const cuuint32_t estr[2] = {1u, 1u};
  return enc(tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, spec, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }


template <int M, int R_>
cudaError_t launch_m(const Desc &d, int nfields, bool c2r, cudaStream_t s) {
  using C = RT<M, R_>;
  CUtensorMap tu, tv;
  if (!spec_map(&tu, d.work_u, d.ny, M, C::R) || !spec_map(&tv, nfields > 1 ? d.work_v : nullptr, d.ny, M, C::R))
    return cudaErrorInvalidValue;
  const void *fn = c2r ? (const void *)k_c2r_tma<M, R_> : (const void *)k_r2c_tma<M, R_>;
  const size_t smem = c2r ? C::SMEM_C2R : C::SMEM_R2C;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0, dev = 0, sms = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, C::THREADS, smem);
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int ntot = nfields * (d.ny / C::R);
  int grid = sms * (per_sm > 0 ? per_sm : 1);
  if (grid > ntot) grid = ntot;
  ProfScope ps(c2r ? PC_C2R : PC_R2C, s);
  if (c2r)
    k_c2r_tma<M, R_><<<grid, C::THREADS, smem, s>>>(tu, tv, d, nfields);
  else
    k_r2c_tma<M, R_><<<grid, C::THREADS, smem, s>>>(tu, tv, d, nfields);
  g_launches.fetch_add(1, std::memory_order_relaxed);
  return cudaGetLastError();
}

}  // namespace

// The TMA row kernels take FP32 plans with power-of-two row transforms of
// length 512 .. 4096 in 16-element register tiles, ny a multiple of the tile
// height, and 16-byte aligned fields and spectra.
bool rows_tma_ok(const Desc &d, int nfields, bool c2r) {
  if (!tma_enabled() || d.rp_row.e != 16) return false;
  if (d.M != 512 && d.M != 1024 && d.M != 2048 && d.M != 4096) return false;
  const int R = rt_rows(d.M);
  if (d.ny < R || d.ny % R) return false;
  if (!aligned16(d.work_u) || (nfields > 1 && !aligned16(d.work_v))) return false;
  const void *f0 = c2r ? d.out_u : d.in_u;
  const void *f1 = c2r ? d.out_v : d.in_v;
  if (!f0 || !aligned16(f0) || (nfields > 1 && (!f1 || !aligned16(f1)))) return false;
  return encode_fn() != nullptr;
}

cudaError_t rows_tma_launch(const Desc &d, int nfields, bool c2r, cudaStream_t s) {
  switch (d.M) {
    case 512: return launch_m<512, 4>(d, nfields, c2r, s);
    case 1024: return launch_m<1024, 4>(d, nfields, c2r, s);
    case 2048: return launch_m<2048, 4>(d, nfields, c2r, s);
    case 4096: return launch_m<4096, 2>(d, nfields, c2r, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace fs
