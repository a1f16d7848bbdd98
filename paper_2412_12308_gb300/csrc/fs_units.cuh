// fs_units.cuh -- the work units every kernel is built from.
//
//   row R2C tile   (Sec. II.D first step: the x-direction transforms of a tile
//                   of rows, real input packed two samples per complex value,
//                   half spectrum written x-frequency-major: spec[a][y])
//   column group   (Sec. II.D second step along y, fused with the spectral
//                   operator of Sec. III and the inverse y transform)
//   row C2R tile   (the inverse x transforms back to real rows)
//   factor range   (per-axis diffusion factors in FP64)
//   small problem  (all of the above for one grid inside one CTA, with the
//                   half spectrum resident in shared memory)
//
// Spectrum layout: [M+1][ny] complex, M = nx/2, element (a, b) at a*ny + b.
// Keeping the x frequency as the slow index makes every column a contiguous
// run (the column pass streams whole columns) and makes the row passes write
// and read runs of `rows_per_unit` consecutive y values per frequency.
#pragma once
#include <type_traits>
#include "fs_mixed.h"
#include "fs_ops.cuh"
#include "fs_pow2.h"

namespace fs {

template <typename T>
struct V2T;
template <>
struct V2T<float> {
  typedef float2 type;
};
template <>
struct V2T<double> {
  typedef double2 type;
};

// Global loads bypass L1 (.cg): data produced by other CTAs of a persistent
// launch must not be served from a stale L1 line.
template <typename T>
__device__ __forceinline__ cx<T> ldc(const cx<T> *p, bool sh) {
  if (sh) return *p;
  const auto v = __ldcg(reinterpret_cast<const typename V2T<T>::type *>(p));
  return mk<T>(v.x, v.y);
}
template <typename T>
__device__ __forceinline__ cx<T> ldg_cg(const cx<T> *p) {
  const auto v = __ldcg(reinterpret_cast<const typename V2T<T>::type *>(p));
  return mk<T>(v.x, v.y);
}
template <typename T>
__device__ __forceinline__ cx<T> zero_cx() {
  return mk<T>(T(0), T(0));
}

// ------------------------------------------------------------ row R2C
// The rest of a row R2C tile once thread (t, rho) holds its row's complex
// pairs z_m, m = t + Tseg*s, in v (row y; `active` as in unit_row_r2c_t):
// length-M FFT through the exchange buffer sm, then the R2C post-process into
// spec[a][y].  Shared by the loading units below and the staged batch tiles.
template <typename T, int E, int MC, int CC>
__device__ __forceinline__ void r2c_tile_finish(const Desc &d, int cnt, int t, int rho, int y, bool active,
                                                cx<T> (&v)[E], cx<T> *sm, cx<T> *spec) {
  const int M = MC ? MC : d.M, ny = d.ny, Tseg = M / E;
  const XLayout lay{rho, cnt};
  const cx<T> *tw = reinterpret_cast<const cx<T> *>(d.tw_x);
  fft_any<T, E, MC, CC, 2>(v, sm, lay, active, t, Tseg, M, d.rp_row, tw);
  __syncthreads();
  if (active) {
#pragma unroll
    for (int s = 0; s < E; ++s) sm[padi(rho + (t + Tseg * s) * cnt)] = v[s];
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int s = 0; s < E; ++s) {
      const int k = t + Tseg * s;
      const cx<T> zk = v[s];
      if (k == 0) {
        spec[y] = mk<T>(zk.x + zk.y, T(0));
        spec[(size_t)M * ny + y] = mk<T>(zk.x - zk.y, T(0));
      } else {
        const cx<T> zm = conj(sm[padi(rho + (M - k) * cnt)]);
        const cx<T> ev = T(0.5) * (zk + zm);
        const cx<T> df_ = zk - zm;
        const cx<T> od = mk<T>(T(0.5) * df_.y, T(-0.5) * df_.x);  // (zk - zm) / (2i)
        spec[(size_t)k * ny + y] = ev + cmul(tw[k], od);
      }
    }
  }
  __syncthreads();
}

// Rows y0..y0+cnt-1 of a real field -> spec[a][y] for a = 0..M.
// Thread (t, rho) = (tid / cnt, tid % cnt) transforms row y0+rho; it holds
// z_m = x_{2m} + i x_{2m+1} for m = t + Tseg*s.  After the length-M complex
// transform Z, X_a = (Z_a + conj Z_{M-a})/2 + w^a (Z_a - conj Z_{M-a})/(2i),
// w = e^{-2 pi i/nx}; X_0 and X_M are real.
// MC, CC: compile-time row length M and rows per tile (0 = read from d / cnt_rt).
// GEN: when not void, the real input is synthesised instead of loaded:
// gen->pair(y, x) returns (f(x, y), f(x + 1, y)) and `in` is unused.
template <typename T, int E, int MC = 0, int CC = 0, typename GEN = void>
__device__ __forceinline__ void unit_row_r2c_t(const Desc &d, int unit, int cnt_rt, cx<T> *sm,
                                               const T *__restrict__ in, cx<T> *spec,
                                               const GEN *gen = nullptr) {
  const int M = MC ? MC : d.M, ny = d.ny, Tseg = M / E;
  const int cnt = CC ? CC : cnt_rt;
  const int tid = threadIdx.x;
  const int t = tid / cnt, rho = tid - t * cnt;
  const int y = unit * cnt + rho;
  const bool active = (t < Tseg) && (y < ny);
  cx<T> v[E];
  if constexpr (std::is_void<GEN>::value) {
    // the tile's rows are contiguous runs of M pairs: load them with all the
    // CTA's threads along the rows (coalesced), stage them in the exchange
    // buffer ([m][row], the layout of the exchange below), then take the slots
    const int y0 = unit * cnt, rows = min(cnt, ny - y0), nthr = blockDim.x;
    const cx<T> *tile = reinterpret_cast<const cx<T> *>(in + (size_t)y0 * d.nx);
    for (int idx = tid; idx < rows * M; idx += nthr) {
      const int r = idx / M, m = idx - r * M;
      sm[padi(r + m * cnt)] = ldg_cg(tile + (size_t)r * M + m);
    }
    __syncthreads();
    if (active) {
#pragma unroll
      for (int s = 0; s < E; ++s) v[s] = sm[padi(rho + (t + Tseg * s) * cnt)];
    } else {
#pragma unroll
      for (int s = 0; s < E; ++s) v[s] = zero_cx<T>();
    }
    __syncthreads();
  } else {
    if (active) {
#pragma unroll
      for (int s = 0; s < E; ++s) v[s] = gen->pair(y, 2 * (t + Tseg * s));
    } else {
#pragma unroll
      for (int s = 0; s < E; ++s) v[s] = zero_cx<T>();
    }
  }
  r2c_tile_finish<T, E, MC, CC>(d, cnt, t, rho, y, active, v, sm, spec);
}

// ------------------------------------------------------------ row C2C (complex fields)
// Complex fields use the full x spectrum: rows y0..y0+cnt-1 of a complex field
// [ny][nx] <-> spec[a][y], a = 0..nx-1 (x-frequency major, like the half
// spectrum of real fields).  Same thread mapping as the real row units; the
// length-nx plan is d.rp_row of the complex descriptor.  The inverse runs by
// conjugation (conj of the forward DFT of conj); no scaling (1/(nx ny) is in
// the spectral multiplier).
// NC, CC: compile-time row length and rows per tile (0 = from d / cnt_rt).
template <typename T, int E, int NC = 0, int CC = 0>
__device__ __forceinline__ void unit_row_c2c_t(const Desc &d, int unit, int cnt_rt, cx<T> *sm, const cx<T> *in,
                                               cx<T> *spec, cx<T> *out, bool inverse) {
  const int N = NC ? NC : d.nx, ny = d.ny, Tseg = N / E;
  const int cnt = CC ? CC : cnt_rt;
  const int tid = threadIdx.x;
  const int t = tid / cnt, rho = tid - t * cnt;
  const int y = unit * cnt + rho;
  const bool active = (t < Tseg) && (y < ny);
  const XLayout lay{rho, cnt};
  const cx<T> *tw = reinterpret_cast<const cx<T> *>(d.tw_x);
  cx<T> v[E];
  if (active) {
    if (inverse) {
#pragma unroll
      for (int s = 0; s < E; ++s) v[s] = conj(ldg_cg(spec + (size_t)(t + Tseg * s) * ny + y));
    } else {
      const cx<T> *row = in + (size_t)y * N;
#pragma unroll
      for (int s = 0; s < E; ++s) v[s] = ldg_cg(row + t + Tseg * s);
    }
  } else {
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = zero_cx<T>();
  }
  fft_any<T, E, NC, CC, 1>(v, sm, lay, active, t, Tseg, N, d.rp_row, tw);
  if (active) {
    if (inverse) {
      cx<T> *row = out + (size_t)y * N;
#pragma unroll
      for (int s = 0; s < E; ++s) row[t + Tseg * s] = conj(v[s]);
    } else {
#pragma unroll
      for (int s = 0; s < E; ++s) spec[(size_t)(t + Tseg * s) * ny + y] = v[s];
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------ row C2R
// spec[a][y] (a = 0..M) for rows y0..y0+cnt-1 -> real rows.  With
// F_a = X_a + conj X_{M-a} and G_a = (X_a - conj X_{M-a}) e^{+2 pi i a/nx},
// the inverse length-M transform of F + iG gives x_{2m} + i x_{2m+1}.
// The imaginary parts of X_0 and X_M are ignored (they are zero for a real
// result).  No scaling here: 1/(nx ny) is folded into the spectral multiplier.
//
// c2r_tile_finish is the part after the loads: v[s] holds X_k, k = t + Tseg*s,
// of the thread's row, xM holds X_M (thread t == 0), and xs(j) returns X_j of
// the thread's row from shared memory (wherever the caller staged the tile).
template <typename T, int E, int MC, int CC, typename XS>
__device__ __forceinline__ void c2r_tile_finish(const Desc &d, int unit, int cnt, int t, int rho, bool active,
                                                cx<T> (&v)[E], cx<T> xM, XS xs, cx<T> *sm, T *out) {
  const int M = MC ? MC : d.M, ny = d.ny, Tseg = M / E;
  const int tid = threadIdx.x;
  const XLayout lay{rho, cnt};
  const cx<T> *tw = reinterpret_cast<const cx<T> *>(d.tw_x);
  if (active) {
#pragma unroll
    for (int s = 0; s < E; ++s) {
      const int k = t + Tseg * s;
      cx<T> xk = v[s], xm;
      if (k == 0) {
        xk = mk<T>(xk.x, T(0));
        xm = mk<T>(xM.x, T(0));
      } else {
        xm = conj(xs(M - k));
      }
      const cx<T> f = xk + xm;
      const cx<T> g = cmul(xk - xm, conj(tw[k]));
      // conjugated input of the inverse transform: conj(F + iG)
      v[s] = mk<T>(f.x - g.y, -(f.y + g.x));
    }
  }
  fft_any<T, E, MC, CC, 2>(v, sm, lay, active, t, Tseg, M, d.rp_row, tw);
  conj_tile(v);
  // stage the tile in the exchange buffer ([m][row]) and store whole rows with
  // all the CTA's threads along the rows (coalesced)
  __syncthreads();
  if (active) {
#pragma unroll
    for (int s = 0; s < E; ++s) sm[padi(rho + (t + Tseg * s) * cnt)] = v[s];
  }
  __syncthreads();
  {
    const int y0 = unit * cnt, rows = min(cnt, ny - y0), nthr = blockDim.x;
    cx<T> *tile = reinterpret_cast<cx<T> *>(out + (size_t)y0 * d.nx);
    for (int idx = tid; idx < rows * M; idx += nthr) {
      const int r = idx / M, m = idx - r * M;
      tile[(size_t)r * M + m] = sm[padi(r + m * cnt)];
    }
  }
  __syncthreads();
}

template <typename T, int E, int MC = 0, int CC = 0>
__device__ __forceinline__ void unit_row_c2r_t(const Desc &d, int unit, int cnt_rt, cx<T> *sm,
                                               const cx<T> *spec, T *out, bool sh) {
  const int M = MC ? MC : d.M, ny = d.ny, Tseg = M / E;
  const int cnt = CC ? CC : cnt_rt;
  const int tid = threadIdx.x;
  const int t = tid / cnt, rho = tid - t * cnt;
  const int y = unit * cnt + rho;
  const bool active = (t < Tseg) && (y < ny);
  cx<T> v[E];
  cx<T> xM = zero_cx<T>();
  if (active) {
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = ldc(spec + (size_t)(t + Tseg * s) * ny + y, sh);
    if (t == 0) xM = ldc(spec + (size_t)M * ny + y, sh);
  } else {
#pragma unroll
    for (int s = 0; s < E; ++s) v[s] = zero_cx<T>();
  }
  __syncthreads();
  if (active) {
#pragma unroll
    for (int s = 0; s < E; ++s) sm[padi(rho + (t + Tseg * s) * cnt)] = v[s];
  }
  __syncthreads();
  c2r_tile_finish<T, E, MC, CC>(d, unit, cnt, t, rho, active, v, xM,
                                [&](int j) { return sm[padi(rho + j * cnt)]; }, sm, out);
}

// ------------------------------------------------------------ column group
// Columns a0..a0+cnt-1 of the half spectrum.  Thread (rho, t) = (tid / Tseg,
// tid % Tseg) handles column a0+rho, frequencies b = t + Tseg*s.
//   solve ops    : load work, forward y-DFT, multiply, inverse y-DFT, store work
//   OP_FORWARD   : load work, forward y-DFT, store the kept spectrum
//   advance ops  : load kept spectra, multiply, inverse y-DFT, store work
// `wu`, `wv` are the work spectra (global, or shared in the small path).
// Single-field spectral operator on a column's register tile (frequency
// b = t + Tseg*s), results conjugated for the inverse-by-conjugation step.
template <typename T, int E>
__device__ __forceinline__ void col_op_single(const Desc &d, const OpCtx<T> &o, int t, int Tseg,
                                              cx<T> (&u)[E]) {
  const int op = d.op;
  if (op == OP_POISSON) {
#pragma unroll
    for (int s = 0; s < E; ++s) u[s] = conj(poisson_mult(o, d, t + Tseg * s) * u[s]);
  } else if (op == OP_DIFFUSION || op == OP_DIFF_ADV) {
#pragma unroll
    for (int s = 0; s < E; ++s) u[s] = conj(diff_mult(o, d, t + Tseg * s) * u[s]);
  } else {  // wave, zero initial velocity
#pragma unroll
    for (int s = 0; s < E; ++s) u[s] = conj(wave_mult(o, d, t + Tseg * s).cu * u[s]);
  }
}

// Single-field advance with a constant source; `sc` is the column of the kept
// source spectrum.  Diffusion, or the wave without initial velocity and
// without v output.
template <typename T, int E>
__device__ __forceinline__ void col_op_source(const Desc &d, const OpCtx<T> &o, int t, int Tseg,
                                              cx<T> (&u)[E], const cx<T> *sc) {
  if (d.op == OP_DIFF_ADV) {
#pragma unroll
    for (int s = 0; s < E; ++s) {
      const DiffS<T> f = diff_src_mult(o, d, t + Tseg * s);
      u[s] = conj(f.m * u[s] + f.g * ldg_cg(sc + t + Tseg * s));
    }
  } else {
#pragma unroll
    for (int s = 0; s < E; ++s) {
      const WaveS<T> f = wave_src_mult(o, d, t + Tseg * s);
      u[s] = conj(f.cu * u[s] + f.pu * ldg_cg(sc + t + Tseg * s));
    }
  }
}

// TWO: a second field (initial velocity in, or velocity out) is carried;
// the single-field variant holds one register tile only.
__host__ __device__ inline bool col_two_fields(const Desc &d) {
  const bool has_v = (d.flags & F_HAS_V0) != 0;
  const bool want_v = (d.flags & F_WANT_V) != 0;
  return ((d.op == OP_WAVE || d.op == OP_FORWARD || d.op == OP_WAVE_ADV) && has_v) ||
         (d.op == OP_WAVE_ADV && want_v);
}

// LC, CC: compile-time column length and columns per unit (0 = from d / cnt_rt).
// SRC: advance ops with a constant source (F_SOURCE); a separate instantiation
// so that the source-free kernels keep their register allocation.
template <typename T, int E, bool TWO, int LC = 0, int CC = 0, bool SRC = false>
__device__ __forceinline__ void unit_col_t(const Desc &d, int unit, int cnt_rt, cx<T> *sm, cx<T> *wu,
                                           cx<T> *wv, bool sh) {
  const int L = LC ? LC : d.ny, M = d.M, Tseg = L / E;
  const int cnt = CC ? CC : cnt_rt;
  const int tid = threadIdx.x;
  const int rho = tid / Tseg, t = tid - rho * Tseg;
  const int a = unit * cnt + rho;
  const bool active = (rho < cnt) && (a <= M);
  const XLayout lay{rho * L, 1};
  const cx<T> *tw = reinterpret_cast<const cx<T> *>(d.tw_y);
  const int op = d.op;
  const bool has_v = (d.flags & F_HAS_V0) != 0;
  const bool want_v = (d.flags & F_WANT_V) != 0;
  const size_t cofs = (size_t)(active ? a : 0) * L;
  const bool adv = (op == OP_DIFF_ADV || op == OP_WAVE_ADV);
  const bool two_in = TWO && (op == OP_WAVE || op == OP_FORWARD || op == OP_WAVE_ADV) && has_v;

  cx<T> u[E], w[TWO ? E : 1];
#pragma unroll
  for (int s = 0; s < E; ++s) u[s] = zero_cx<T>();
  if constexpr (TWO) {
#pragma unroll
    for (int s = 0; s < E; ++s) w[s] = zero_cx<T>();
  }
  if (active) {
    const cx<T> *src_u = adv ? reinterpret_cast<const cx<T> *>(d.st_u) : wu;
    const cx<T> *src_v = adv ? reinterpret_cast<const cx<T> *>(d.st_v) : wv;
    const bool s_sh = sh && !adv;
#pragma unroll
    for (int s = 0; s < E; ++s) u[s] = ldc(src_u + cofs + t + Tseg * s, s_sh);
    if constexpr (TWO) {
      if (two_in) {
#pragma unroll
        for (int s = 0; s < E; ++s) w[s] = ldc(src_v + cofs + t + Tseg * s, s_sh);
      }
    }
  }
  // ---- forward y transforms (one inlined engine, looped over the fields)
  if constexpr (TWO) {
    const int nfwd = adv ? 0 : (two_in ? 2 : 1);
#pragma unroll 1
    for (int f = 0; f < nfwd; ++f) {
      if (f) {
        __syncthreads();
        swap_tile(u, w);
      }
      fft_any<T, E, LC, 1, 1>(u, sm, lay, active, t, Tseg, L, d.rp_col, tw);
      if (f) swap_tile(u, w);
    }
  } else {
    if (!adv) fft_any<T, E, LC, 1, 1>(u, sm, lay, active, t, Tseg, L, d.rp_col, tw);
  }
  // keep the forward spectrum (state creation, or a solve that keeps its
  // spectrum for later advances)
  if (!adv && d.st_out_u) {
    if (active) {
      cx<T> *ou = reinterpret_cast<cx<T> *>(d.st_out_u) + cofs;
#pragma unroll
      for (int s = 0; s < E; ++s) ou[t + Tseg * s] = u[s];
      if constexpr (TWO) {
        if (has_v && d.st_out_v) {
          cx<T> *ov = reinterpret_cast<cx<T> *>(d.st_out_v) + cofs;
#pragma unroll
          for (int s = 0; s < E; ++s) ov[t + Tseg * s] = w[s];
        }
      }
    }
  }
  if (op == OP_FORWARD) {
    __syncthreads();
    return;
  }
  // ---- spectral operator (Sec. III), in registers; results conjugated for the
  // inverse transform by conjugation
  if (active) {
    const OpCtx<T> o = op_ctx<T>(d, a);
    if constexpr (SRC) {  // advance ops only (the host sets F_SOURCE on advances)
      const cx<T> *sc = reinterpret_cast<const cx<T> *>(d.st_s) + cofs;
      if (op == OP_DIFF_ADV || !TWO) {
        col_op_source<T, E>(d, o, t, Tseg, u, sc);
      } else if constexpr (TWO) {
#pragma unroll
        for (int s = 0; s < E; ++s) {
          const WaveS<T> f = wave_src_mult(o, d, t + Tseg * s);
          const cx<T> u0 = u[s], v0 = w[s], s0 = ldg_cg(sc + t + Tseg * s);
          u[s] = conj(f.cu * u0 + f.su * v0 + f.pu * s0);
          w[s] = conj(f.sv * u0 + f.cu * v0 + f.su * s0);
        }
      }
    } else if (op == OP_POISSON || op == OP_DIFFUSION || op == OP_DIFF_ADV || !TWO) {
      col_op_single<T, E>(d, o, t, Tseg, u);
    } else if constexpr (TWO) {  // wave carrying a velocity field
#pragma unroll
      for (int s = 0; s < E; ++s) {
        const WaveF<T> f = wave_mult(o, d, t + Tseg * s);
        const cx<T> u0 = u[s], v0 = w[s];
        u[s] = conj(f.cu * u0 + f.su * v0);
        w[s] = conj(f.sv * u0 + f.cu * v0);
      }
    }
  }
  // ---- inverse y transforms
  const int ninv = (TWO && op == OP_WAVE_ADV && want_v) ? 2 : 1;
#pragma unroll 1
  for (int f = 0; f < ninv; ++f) {
    __syncthreads();
    if constexpr (TWO) {
      if (f) swap_tile(u, w);
    }
    fft_any<T, E, LC, 1, 1>(u, sm, lay, active, t, Tseg, L, d.rp_col, tw);
    if (active) {
      cx<T> *dst = (f ? wv : wu) + cofs;
#pragma unroll
      for (int s = 0; s < E; ++s) dst[t + Tseg * s] = conj(u[s]);
    }
  }
  __syncthreads();
}

// ------------------------------------------------------------ diffusion factors
// fac[a] = scale * exp(-D t omega_x(a)^2)  (a <= M)
// fac[M+1+b] = exp(-D t omega_y(b)^2)      (b < ny)
// evaluated in FP64 (the per-axis split of exp(-D t |omega|^2)), stored as two
// floats (FP32 path) or a double (FP64 path).
template <typename T>
__device__ void unit_factor(const Desc &d, int first, int count, int stride) {
  const int n = d.M + 1 + d.ny;
  const int end = min(n, first + count);
  for (int i = first + (int)threadIdx.x; i < end; i += stride) {
    double w2, f;
    if (i <= d.M) {
      w2 = d.wx2d[i];
      f = d.scale * exp(-d.p_dt * w2);
    } else {
      w2 = d.wy2d[i - d.M - 1];
      f = exp(-d.p_dt * w2);
    }
    if constexpr (sizeof(T) == 4) {
      float hi, lo;
      split_double(f, hi, lo);
      reinterpret_cast<float2 *>(d.fac)[i] = make_float2(hi, lo);
    } else {
      reinterpret_cast<double *>(d.fac)[i] = f;
    }
  }
}

// ------------------------------------------------------------ pass kernel bodies
// Row R2C: grid = n_row_units per field; blockIdx >= n_row_units selects the v field.
template <typename T, int E>
__device__ __forceinline__ void kbody_r2c(const Desc &d, cx<T> *sm) {
  int unit = blockIdx.x;
  const T *in = reinterpret_cast<const T *>(d.in_u);
  cx<T> *spec = reinterpret_cast<cx<T> *>(d.work_u);
  if (unit >= d.n_row_units) {
    unit -= d.n_row_units;
    in = reinterpret_cast<const T *>(d.in_v);
    spec = reinterpret_cast<cx<T> *>(d.work_v);
  }
  unit_row_r2c_t<T, E>(d, unit, d.rows_per_unit, sm, in, spec);
}
// Row C2R: grid = n_row_units per field; blockIdx >= n_row_units selects the v field.
template <typename T, int E>
__device__ __forceinline__ void kbody_c2r(const Desc &d, cx<T> *sm) {
  int unit = blockIdx.x;
  const cx<T> *spec = reinterpret_cast<const cx<T> *>(d.work_u);
  T *out = reinterpret_cast<T *>(d.out_u);
  if (unit >= d.n_row_units) {
    unit -= d.n_row_units;
    spec = reinterpret_cast<const cx<T> *>(d.work_v);
    out = reinterpret_cast<T *>(d.out_v);
  }
  unit_row_c2r_t<T, E>(d, unit, d.rows_per_unit, sm, spec, out, false);
}

// ------------------------------------------------------------ per-tile wrappers
// One non-inlined function per (element type, register tile E) and unit kind,
// each compiled in its own translation unit (fs_units_<type>_e<E>.cu) and
// linked as relocatable device code, so the many instantiations compile in
// parallel.
#define FS_KERNEL_DECL(T, E)                                               \
  __global__ void k_r2c_##T##_##E(const Desc d);                           \
  __global__ void k_c2r_##T##_##E(const Desc d);                           \
  __global__ void k_col1_##T##_##E(const Desc d);                          \
  __global__ void k_col2_##T##_##E(const Desc d);                          \
  __global__ void k_cols_##T##_##E(const Desc d);                          \
  __global__ void k_c2cf_##T##_##E(const Desc d);                          \
  __global__ void k_c2ci_##T##_##E(const Desc d);

#define FS_UNIT_DECL(T, E)                                                                     \
  FS_KERNEL_DECL(T, E)                                                                         \
  __device__ __noinline__ void unit_row_r2c_##T##_##E(const Desc &d, int unit, int cnt,       \
                                                      cx<T> *sm, const T *in, cx<T> *spec);    \
  __device__ __noinline__ void unit_row_c2r_##T##_##E(const Desc &d, int unit, int cnt,       \
                                                      cx<T> *sm, const cx<T> *spec, T *out,    \
                                                      bool sh);                                \
  __device__ __noinline__ void unit_col_##T##_##E(const Desc &d, int unit, int cnt, cx<T> *sm, \
                                                  cx<T> *wu, cx<T> *wv, bool sh);              \
  __device__ __noinline__ void unit_col2_##T##_##E(const Desc &d, int unit, int cnt, cx<T> *sm,\
                                                   cx<T> *wu, cx<T> *wv, bool sh);             \
  __device__ __noinline__ void unit_cols_##T##_##E(const Desc &d, int unit, int cnt, cx<T> *sm,\
                                                   cx<T> *wu, cx<T> *wv, bool sh);

#define FS_UNIT_DEF(T, E)                                                                       \
  __device__ __noinline__ void unit_row_r2c_##T##_##E(const Desc &d, int unit, int cnt,        \
                                                      cx<T> *sm, const T *in, cx<T> *spec) {    \
    unit_row_r2c_t<T, E>(d, unit, cnt, sm, in, spec);                                           \
  }                                                                                             \
  __device__ __noinline__ void unit_row_c2r_##T##_##E(const Desc &d, int unit, int cnt,        \
                                                      cx<T> *sm, const cx<T> *spec, T *out,     \
                                                      bool sh) {                                \
    unit_row_c2r_t<T, E>(d, unit, cnt, sm, spec, out, sh);                                      \
  }                                                                                             \
  __device__ __noinline__ void unit_col_##T##_##E(const Desc &d, int unit, int cnt, cx<T> *sm,  \
                                                  cx<T> *wu, cx<T> *wv, bool sh) {              \
    unit_col_t<T, E, false>(d, unit, cnt, sm, wu, wv, sh);                                      \
  }                                                                                             \
  __device__ __noinline__ void unit_col2_##T##_##E(const Desc &d, int unit, int cnt, cx<T> *sm, \
                                                   cx<T> *wu, cx<T> *wv, bool sh) {             \
    unit_col_t<T, E, true>(d, unit, cnt, sm, wu, wv, sh);                                       \
  }                                                                                             \
  __device__ __noinline__ void unit_cols_##T##_##E(const Desc &d, int unit, int cnt, cx<T> *sm, \
                                                   cx<T> *wu, cx<T> *wv, bool sh) {             \
    unit_col_t<T, E, true, 0, 0, true>(d, unit, cnt, sm, wu, wv, sh);                           \
  }                                                                                             \
  __global__ void __launch_bounds__(512) k_r2c_##T##_##E(const Desc d) {                        \
    extern __shared__ __align__(16) unsigned char fs_smem[];                                    \
    kbody_r2c<T, E>(d, reinterpret_cast<cx<T> *>(fs_smem));                                     \
  }                                                                                             \
  __global__ void __launch_bounds__(512) k_c2r_##T##_##E(const Desc d) {                        \
    extern __shared__ __align__(16) unsigned char fs_smem[];                                    \
    kbody_c2r<T, E>(d, reinterpret_cast<cx<T> *>(fs_smem));                                     \
  }                                                                                             \
  __global__ void __launch_bounds__(512) k_col1_##T##_##E(const Desc d) {                       \
    extern __shared__ __align__(16) unsigned char fs_smem[];                                    \
    unit_col_t<T, E, false>(d, blockIdx.x, d.cols_per_unit, reinterpret_cast<cx<T> *>(fs_smem), \
                            reinterpret_cast<cx<T> *>(d.work_u),                                \
                            reinterpret_cast<cx<T> *>(d.work_v), false);                        \
  }                                                                                             \
  __global__ void __launch_bounds__(512) k_col2_##T##_##E(const Desc d) {                       \
    extern __shared__ __align__(16) unsigned char fs_smem[];                                    \
    unit_col_t<T, E, true>(d, blockIdx.x, d.cols_per_unit, reinterpret_cast<cx<T> *>(fs_smem),  \
                           reinterpret_cast<cx<T> *>(d.work_u),                                 \
                           reinterpret_cast<cx<T> *>(d.work_v), false);                         \
  }                                                                                             \
  __global__ void __launch_bounds__(512) k_c2cf_##T##_##E(const Desc d) {                       \
    extern __shared__ __align__(16) unsigned char fs_smem[];                                    \
    int unit = blockIdx.x;                                                                      \
    const bool second = unit >= d.n_row_units;                                                  \
    if (second) unit -= d.n_row_units;                                                          \
    unit_row_c2c_t<T, E>(d, unit, d.rows_per_unit, reinterpret_cast<cx<T> *>(fs_smem),          \
                         reinterpret_cast<const cx<T> *>(second ? d.in_v : d.in_u),             \
                         reinterpret_cast<cx<T> *>(second ? d.work_v : d.work_u), nullptr,      \
                         false);                                                                \
  }                                                                                             \
  __global__ void __launch_bounds__(512) k_c2ci_##T##_##E(const Desc d) {                       \
    extern __shared__ __align__(16) unsigned char fs_smem[];                                    \
    unit_row_c2c_t<T, E>(d, blockIdx.x, d.rows_per_unit, reinterpret_cast<cx<T> *>(fs_smem),    \
                         nullptr, reinterpret_cast<cx<T> *>(d.work_u),                          \
                         reinterpret_cast<cx<T> *>(d.out_u), true);                             \
  }                                                                                             \
  __global__ void __launch_bounds__(512) k_cols_##T##_##E(const Desc d) {                       \
    extern __shared__ __align__(16) unsigned char fs_smem[];                                    \
    unit_col_t<T, E, true, 0, 0, true>(d, blockIdx.x, d.cols_per_unit,                          \
                                       reinterpret_cast<cx<T> *>(fs_smem),                      \
                                       reinterpret_cast<cx<T> *>(d.work_u),                     \
                                       reinterpret_cast<cx<T> *>(d.work_v), false);             \
  }

// Register tiles: FP32 uses up to 16/24/20 elements per thread for the
// 2^k / 3*2^k / 5*2^k families; FP64 (twice the registers per element) up to
// 8/12/10, and 16 only for length 8192.
#define FS_FOR_EACH_E_float(X) X(float, 4) X(float, 5) X(float, 6) X(float, 8) X(float, 10) \
  X(float, 12) X(float, 16) X(float, 20) X(float, 24)
#define FS_FOR_EACH_E_double(X) X(double, 4) X(double, 5) X(double, 6) X(double, 8) \
  X(double, 10) X(double, 12) X(double, 16)
FS_FOR_EACH_E_float(FS_UNIT_DECL)
FS_FOR_EACH_E_double(FS_UNIT_DECL)

#define FS_E_CASE(T, E, FN, ...) \
  case E:                        \
    FN##_##T##_##E(__VA_ARGS__); \
    break;
#define FS_E_SWITCH_float(e, FN, ...)         \
  switch (e) {                                \
    FS_E_CASE(float, 4, FN, __VA_ARGS__)      \
    FS_E_CASE(float, 5, FN, __VA_ARGS__)      \
    FS_E_CASE(float, 6, FN, __VA_ARGS__)      \
    FS_E_CASE(float, 8, FN, __VA_ARGS__)      \
    FS_E_CASE(float, 10, FN, __VA_ARGS__)     \
    FS_E_CASE(float, 12, FN, __VA_ARGS__)     \
    FS_E_CASE(float, 16, FN, __VA_ARGS__)     \
    FS_E_CASE(float, 20, FN, __VA_ARGS__)     \
    FS_E_CASE(float, 24, FN, __VA_ARGS__)     \
    default:                                  \
      break;                                  \
  }
#define FS_E_SWITCH_double(e, FN, ...)        \
  switch (e) {                                \
    FS_E_CASE(double, 4, FN, __VA_ARGS__)     \
    FS_E_CASE(double, 5, FN, __VA_ARGS__)     \
    FS_E_CASE(double, 6, FN, __VA_ARGS__)     \
    FS_E_CASE(double, 8, FN, __VA_ARGS__)     \
    FS_E_CASE(double, 10, FN, __VA_ARGS__)    \
    FS_E_CASE(double, 12, FN, __VA_ARGS__)    \
    FS_E_CASE(double, 16, FN, __VA_ARGS__)    \
    default:                                  \
      break;                                  \
  }

// Host-side kernel lookup by register tile.
struct PassKernels {
  PassKernel r2c, c2r, col1, col2, cols, c2cf, c2ci;
};
#define FS_PK_CASE(T, E)                                                                      \
  case E:                                                                                     \
    return PassKernels{k_r2c_##T##_##E, k_c2r_##T##_##E, k_col1_##T##_##E, k_col2_##T##_##E, \
                       k_cols_##T##_##E, k_c2cf_##T##_##E, k_c2ci_##T##_##E};
template <typename T>
inline PassKernels pass_kernels(int e);
template <>
inline PassKernels pass_kernels<float>(int e) {
  switch (e) { FS_FOR_EACH_E_float(FS_PK_CASE) default: return PassKernels{}; }
}
template <>
inline PassKernels pass_kernels<double>(int e) {
  switch (e) { FS_FOR_EACH_E_double(FS_PK_CASE) default: return PassKernels{}; }
}

// Compile-time power-of-two units (FP32 only; defined in fs_pow2_f32.cu).
__device__ __forceinline__ bool pow2_r2c(const Desc &d, int unit, int cnt, cx<float> *sm, const float *in,
                                         cx<float> *spec) {
  return p2_unit_r2c(d, unit, cnt, sm, in, spec);
}
__device__ __forceinline__ bool pow2_r2c(const Desc &, int, int, cx<double> *, const double *, cx<double> *) {
  return false;
}
__device__ __forceinline__ bool pow2_c2r(const Desc &d, int unit, int cnt, cx<float> *sm, const cx<float> *spec,
                                         float *out, bool sh) {
  return p2_unit_c2r(d, unit, cnt, sm, spec, out, sh);
}
__device__ __forceinline__ bool pow2_c2r(const Desc &, int, int, cx<double> *, const cx<double> *, double *, bool) {
  return false;
}
__device__ __forceinline__ bool pow2_col1(const Desc &d, int unit, int cnt, cx<float> *sm, cx<float> *wu,
                                          cx<float> *wv, bool sh) {
  return p2_unit_col1(d, unit, cnt, sm, wu, wv, sh);
}
__device__ __forceinline__ bool pow2_col1(const Desc &, int, int, cx<double> *, cx<double> *, cx<double> *, bool) {
  return false;
}
__device__ __forceinline__ bool pow2_cols(const Desc &d, int unit, int cnt, cx<float> *sm, cx<float> *wu,
                                          cx<float> *wv, bool sh) {
  return p2_unit_cols(d, unit, cnt, sm, wu, wv, sh);
}
__device__ __forceinline__ bool pow2_cols(const Desc &, int, int, cx<double> *, cx<double> *, cx<double> *, bool) {
  return false;
}

// Compile-time 3 x 2^k / 5 x 2^k units (FP32 only; fs_mixed_f32.cu).
__device__ __forceinline__ bool mixed_r2c(const Desc &d, int unit, int cnt, cx<float> *sm, const float *in,
                                          cx<float> *spec) {
  return mx_unit_r2c(d, unit, cnt, sm, in, spec);
}
__device__ __forceinline__ bool mixed_r2c(const Desc &, int, int, cx<double> *, const double *, cx<double> *) {
  return false;
}
__device__ __forceinline__ bool mixed_c2r(const Desc &d, int unit, int cnt, cx<float> *sm, const cx<float> *spec,
                                          float *out, bool sh) {
  return mx_unit_c2r(d, unit, cnt, sm, spec, out, sh);
}
__device__ __forceinline__ bool mixed_c2r(const Desc &, int, int, cx<double> *, const cx<double> *, double *, bool) {
  return false;
}
__device__ __forceinline__ bool mixed_col1(const Desc &d, int unit, int cnt, cx<float> *sm, cx<float> *wu,
                                           cx<float> *wv, bool sh) {
  return mx_unit_col1(d, unit, cnt, sm, wu, wv, sh);
}
__device__ __forceinline__ bool mixed_col1(const Desc &, int, int, cx<double> *, cx<double> *, cx<double> *, bool) {
  return false;
}

template <typename T>
struct Units;
#define FS_UNITS_SPEC(T)                                                                        \
  template <>                                                                                   \
  struct Units<T> {                                                                             \
    static __device__ __forceinline__ void r2c(const Desc &d, int unit, int cnt, cx<T> *sm,     \
                                               const T *in, cx<T> *spec) {                      \
      if (pow2_r2c(d, unit, cnt, sm, in, spec)) return;                                         \
      if (mixed_r2c(d, unit, cnt, sm, in, spec)) return;                                        \
      FS_E_SWITCH_##T(d.rp_row.e, unit_row_r2c, d, unit, cnt, sm, in, spec)                      \
    }                                                                                           \
    static __device__ __forceinline__ void c2r(const Desc &d, int unit, int cnt, cx<T> *sm,     \
                                               const cx<T> *spec, T *out, bool sh) {            \
      if (pow2_c2r(d, unit, cnt, sm, spec, out, sh)) return;                                    \
      if (mixed_c2r(d, unit, cnt, sm, spec, out, sh)) return;                                   \
      FS_E_SWITCH_##T(d.rp_row.e, unit_row_c2r, d, unit, cnt, sm, spec, out, sh)                 \
    }                                                                                           \
    static __device__ __forceinline__ void col(const Desc &d, int unit, int cnt, cx<T> *sm,     \
                                               cx<T> *wu, cx<T> *wv, bool sh) {                 \
      if (d.flags & F_SOURCE) {                                                                 \
        if (pow2_cols(d, unit, cnt, sm, wu, wv, sh)) return;                                    \
        FS_E_SWITCH_##T(d.rp_col.e, unit_cols, d, unit, cnt, sm, wu, wv, sh)                    \
      } else if (col_two_fields(d)) {                                                           \
        FS_E_SWITCH_##T(d.rp_col.e, unit_col2, d, unit, cnt, sm, wu, wv, sh)                    \
      } else {                                                                                  \
        if (pow2_col1(d, unit, cnt, sm, wu, wv, sh)) return;                                    \
        if (mixed_col1(d, unit, cnt, sm, wu, wv, sh)) return;                                   \
        FS_E_SWITCH_##T(d.rp_col.e, unit_col, d, unit, cnt, sm, wu, wv, sh)                     \
      }                                                                                         \
    }                                                                                           \
  };
FS_UNITS_SPEC(float)
FS_UNITS_SPEC(double)

template <typename T>
__device__ __forceinline__ void row_r2c_any(const Desc &d, int unit, int cnt, cx<T> *sm,
                                            const T *in, cx<T> *spec) {
  Units<T>::r2c(d, unit, cnt, sm, in, spec);
}
template <typename T>
__device__ __forceinline__ void row_c2r_any(const Desc &d, int unit, int cnt, cx<T> *sm,
                                            const cx<T> *spec, T *out, bool sh) {
  Units<T>::c2r(d, unit, cnt, sm, spec, out, sh);
}
template <typename T>
__device__ __forceinline__ void col_any(const Desc &d, int unit, int cnt, cx<T> *sm, cx<T> *wu,
                                        cx<T> *wv, bool sh) {
  Units<T>::col(d, unit, cnt, sm, wu, wv, sh);
}

// ------------------------------------------------------------ small problem
// The whole solve in one CTA.  Shared memory: spec_u [(M+1)*ny], spec_v (when
// the op carries a second field), then the exchange scratch.
__host__ __device__ inline int small_nspec(const Desc &d) {
  const bool has_v = (d.flags & F_HAS_V0) != 0;
  if (d.op == OP_WAVE || d.op == OP_FORWARD) return has_v ? 2 : 1;
  if (d.op == OP_WAVE_ADV) return ((d.flags & F_WANT_V) != 0) ? 2 : 1;
  return 1;
}

template <typename T>
__device__ __forceinline__ void unit_small(const Desc &d, cx<T> *smem) {
  const int M = d.M, ny = d.ny;
  const size_t spec_n = (size_t)(M + 1) * ny;
  const int nspec = small_nspec(d);
  cx<T> *su = smem;
  cx<T> *sv = smem + spec_n;
  cx<T> *sx = smem + spec_n * nspec;
  const int cr = d.small_rows, cc = d.small_cols;
  const int op = d.op;
  const bool has_v = (d.flags & F_HAS_V0) != 0;
  const bool adv = (op == OP_DIFF_ADV || op == OP_WAVE_ADV);

  if (op == OP_DIFFUSION || op == OP_DIFF_ADV) {
    unit_factor<T>(d, 0, M + 1 + ny, blockDim.x);
    __syncthreads();
  }
  if (!adv) {
    const int nu = (ny + cr - 1) / cr;
    for (int g = 0; g < nu; ++g)
      row_r2c_any<T>(d, g, cr, sx, reinterpret_cast<const T *>(d.in_u), su);
    if ((op == OP_WAVE || op == OP_FORWARD) && has_v)
      for (int g = 0; g < nu; ++g)
        row_r2c_any<T>(d, g, cr, sx, reinterpret_cast<const T *>(d.in_v), sv);
  }
  const int ncu = (M + 1 + cc - 1) / cc;
  for (int g = 0; g < ncu; ++g) col_any<T>(d, g, cc, sx, su, sv, true);
  if (op == OP_FORWARD) return;
  const int nu = (ny + cr - 1) / cr;
  for (int g = 0; g < nu; ++g)
    row_c2r_any<T>(d, g, cr, sx, su, reinterpret_cast<T *>(d.out_u), true);
  if (op == OP_WAVE_ADV && (d.flags & F_WANT_V))
    for (int g = 0; g < nu; ++g)
      row_c2r_any<T>(d, g, cr, sx, sv, reinterpret_cast<T *>(d.out_v), true);
}

}  // namespace fs
