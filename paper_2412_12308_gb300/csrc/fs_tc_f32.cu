// fs_tc_f32.cu -- measured variant: the first radix-16 stage of the column
// pass as a DFT-as-matmul on the tensor cores with split-BF16 operands.
//
// In an advance (kept spectrum -> operator -> inverse y transform) the first
// Stockham stage of a length-L column transform is L/16 independent 16-point
// DFTs with no twiddles (the matrix form of Eq. DFT2 with N = 16).  In real
// arithmetic that is Y = A X with the 32 x 32 matrix
//   A = [[ Wr, -Wi ], [ Wi, Wr ]],  W = e^{-2 pi i m k / 16}
// applied to X = [Re x; Im x] (32 x L/16).  Both A and X are split into three
// bfloat16 terms (hi, mid, lo: 8 significant bits each, ~24 together) and the
// six products down to ~2^-24 (hh, hm, mh, hl, mm, lh) are accumulated in FP32
// by mma.sync m16n8k16.  The remaining stages run on the FP32 compile-time
// engine.  Selected with FS_COLUMN_VARIANT=bf16x3 (single-field advance ops,
// power-of-two column lengths 512..4096); otherwise the FP32 kernels run.
#include <cuda_bf16.h>

#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>

#include "fs_pow2.h"
#include "fs_units.cuh"

namespace fs {

// A split into three bf16 terms, [term][row m][col k], rows/cols 0..31.
__device__ __nv_bfloat16 g_tc_a[3][32][32];

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi) {
  uint16_t l, h;
  memcpy(&l, &lo, 2);
  memcpy(&h, &hi, 2);
  return (uint32_t)l | ((uint32_t)h << 16);
}

__device__ __forceinline__ void split3(float x, __nv_bfloat16 &h, __nv_bfloat16 &m, __nv_bfloat16 &l) {
  h = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(h);
  m = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(m);
  l = __float2bfloat16_rn(r2);
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

template <int L>
struct TcCfg {
  static constexpr int E = 16, Tseg = L / E;     // threads: one butterfly of stage 1 each
  static constexpr int XW = padded_len(L);       // exchange (complex)
  static constexpr int XB = 32 * Tseg;           // stage-1 operand staging (floats)
  static constexpr size_t SMEM = (size_t)XW * 8 + (size_t)XB * 4 + 3 * 32 * 32 * 2;
};

template <int L>
__global__ void __launch_bounds__(L / 16, 2) k_col_tc(const Desc d) {
  typedef TcCfg<L> C;
  constexpr int E = C::E, Tseg = C::Tseg;
  static_assert(Tseg % 32 == 0, "whole warps of butterflies");
  extern __shared__ __align__(16) unsigned char fs_smem[];
  cx<float> *sm = reinterpret_cast<cx<float> *>(fs_smem);
  float *xb = reinterpret_cast<float *>(fs_smem + (size_t)C::XW * 8);
  __nv_bfloat16 *as = reinterpret_cast<__nv_bfloat16 *>(fs_smem + (size_t)C::XW * 8 + (size_t)C::XB * 4);
  const int t = threadIdx.x;
  const int a = blockIdx.x;  // one column per CTA, grid = M + 1
  const cx<float> *tw = reinterpret_cast<const cx<float> *>(d.tw_y);

  // matrix terms into shared memory
  for (int i = t; i < 3 * 32 * 32; i += Tseg) as[i] = (&g_tc_a[0][0][0])[i];
  // kept spectrum column, operator (conjugated for the inverse by conjugation)
  cx<float> u[E];
  const cx<float> *src = reinterpret_cast<const cx<float> *>(d.st_u) + (size_t)a * L;
#pragma unroll
  for (int s = 0; s < E; ++s) u[s] = ldg_cg(src + t + Tseg * s);
  col_op_single<float, E>(d, op_ctx<float>(d, a), t, Tseg, u);
  // stage-1 operand: X[k][n] = inputs k (Re rows 0..15, Im rows 16..31) of butterfly n = t
#pragma unroll
  for (int s = 0; s < E; ++s) {
    xb[s * Tseg + t] = u[s].x;
    xb[(16 + s) * Tseg + t] = u[s].y;
  }
  __syncthreads();
  const int warp = t >> 5, lane = t & 31, g = lane >> 2, tig = lane & 3;
  // A fragments for (term, m-tile, k-tile), kept in registers
  uint32_t af[3][2][2][4];
#pragma unroll
  for (int tm = 0; tm < 3; ++tm)
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int kt = 0; kt < 2; ++kt) {
        const __nv_bfloat16 *A = as + tm * 1024;
        const int r0 = 16 * mt + g, c0 = 16 * kt + 2 * tig;
        af[tm][mt][kt][0] = pack2(A[r0 * 32 + c0], A[r0 * 32 + c0 + 1]);
        af[tm][mt][kt][1] = pack2(A[(r0 + 8) * 32 + c0], A[(r0 + 8) * 32 + c0 + 1]);
        af[tm][mt][kt][2] = pack2(A[r0 * 32 + c0 + 8], A[r0 * 32 + c0 + 9]);
        af[tm][mt][kt][3] = pack2(A[(r0 + 8) * 32 + c0 + 8], A[(r0 + 8) * 32 + c0 + 9]);
      }
  // each warp: its 32 butterflies as 4 n-tiles of 8
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int n0 = warp * 32 + i * 8;
    uint32_t bf[3][2][2];
#pragma unroll
    for (int kt = 0; kt < 2; ++kt) {
      const int k0 = 16 * kt + 2 * tig;
      const float x0 = xb[k0 * Tseg + n0 + g], x1 = xb[(k0 + 1) * Tseg + n0 + g];
      const float x2 = xb[(k0 + 8) * Tseg + n0 + g], x3 = xb[(k0 + 9) * Tseg + n0 + g];
      __nv_bfloat16 h0, m0, l0, h1, m1, l1, h2, m2, l2, h3, m3, l3;
      split3(x0, h0, m0, l0);
      split3(x1, h1, m1, l1);
      split3(x2, h2, m2, l2);
      split3(x3, h3, m3, l3);
      bf[0][kt][0] = pack2(h0, h1);
      bf[0][kt][1] = pack2(h2, h3);
      bf[1][kt][0] = pack2(m0, m1);
      bf[1][kt][1] = pack2(m2, m3);
      bf[2][kt][0] = pack2(l0, l1);
      bf[2][kt][1] = pack2(l2, l3);
    }
    float c[2][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
      for (int q = 0; q < 4; ++q) c[mt][q] = 0.f;
#pragma unroll
      for (int kt = 0; kt < 2; ++kt) {
        // smallest products first
        mma_bf16(c[mt], af[2][mt][kt], bf[0][kt]);  // lo * hi
        mma_bf16(c[mt], af[1][mt][kt], bf[1][kt]);  // mid * mid
        mma_bf16(c[mt], af[0][mt][kt], bf[2][kt]);  // hi * lo
        mma_bf16(c[mt], af[1][mt][kt], bf[0][kt]);  // mid * hi
        mma_bf16(c[mt], af[0][mt][kt], bf[1][kt]);  // hi * mid
        mma_bf16(c[mt], af[0][mt][kt], bf[0][kt]);  // hi * hi
      }
    }
    // outputs r = g and g + 8 of butterflies n = n0 + 2 tig + h -> element 16 n + r
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int n = n0 + 2 * tig + h;
      sm[padi(16 * n + g)] = mk<float>(c[0][h], c[1][h]);
      sm[padi(16 * n + g + 8)] = mk<float>(c[0][2 + h], c[1][2 + h]);
    }
  }
  __syncthreads();
  // remaining stages (2, 3, ...) on the compile-time engine
  fft_ct_from<float, E, L, 1, 1, 1>(u, sm, 0, true, t, tw);
  cx<float> *dst = reinterpret_cast<cx<float> *>(d.work_u) + (size_t)a * L;
#pragma unroll
  for (int s = 0; s < E; ++s) dst[t + Tseg * s] = conj(u[s]);
}

static std::once_flag g_tc_once;
static cudaError_t g_tc_init = cudaSuccess;

// bf16 round-to-nearest-even of a float, on the host
static uint16_t host_bf16(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  const uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  return (uint16_t)(u >> 16);
}
static float host_bf16_to_f(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  memcpy(&f, &u, 4);
  return f;
}

static cudaError_t tc_tables() {
  std::call_once(g_tc_once, [] {
    static uint16_t h[3][32][32];
    for (int m = 0; m < 16; ++m)
      for (int k = 0; k < 16; ++k) {
        const double ang = 2.0 * M_PI * (double)((m * k) % 16) / 16.0;
        const double wr = cos(ang), wi = -sin(ang);
        const double vals[4] = {wr, -wi, wi, wr};  // A[m][k], A[m][16+k], A[16+m][k], A[16+m][16+k]
        const int rows[4] = {m, m, 16 + m, 16 + m}, cols[4] = {k, 16 + k, k, 16 + k};
        for (int q = 0; q < 4; ++q) {
          double r = vals[q];
          for (int term = 0; term < 3; ++term) {
            const uint16_t b = host_bf16((float)r);
            h[term][rows[q]][cols[q]] = b;
            r -= (double)host_bf16_to_f(b);
          }
        }
      }
    g_tc_init = cudaMemcpyToSymbol(g_tc_a, h, sizeof h);
  });
  return g_tc_init;
}

bool tc_variant_requested() {
  const char *v = getenv("FS_COLUMN_VARIANT");
  return v && strcmp(v, "bf16x3") == 0;
}

PassKernel p2_col_tc_f32(int L, size_t *smem) {
  if (tc_tables() != cudaSuccess) return nullptr;
  switch (L) {
#define C(l)                   \
  case l:                      \
    *smem = TcCfg<l>::SMEM;    \
    return k_col_tc<l>;
    C(512) C(1024) C(2048) C(4096)
#undef C
    default:
      return nullptr;
  }
}

}  // namespace fs
