// fs_fft.cuh -- complex arithmetic, small DFT butterflies and the
// register-resident mixed-radix FFT engine used by every kernel.
//
// The engine computes the length-L DFT of Sec. II.B (Eq. DFT) with the
// even/odd splitting idea of Sec. II.C generalised to radix R in
// {2, 3, 4, 5, 8, 16} (the compile-time engine also composite last stages
// 6, 10, 12, 20, 24) (a Stockham auto-sort decimation-in-time ordering, so
// no bit reversal pass is needed).  Each thread holds E elements in registers;
// thread t of a segment owns indices t + Tseg*s (s < E, Tseg = L/E) both on
// entry and on exit, so global loads and stores are coalesced and a forward
// transform can hand its output straight to an inverse one in registers.
// Stages exchange data through shared memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "fs_desc.h"

namespace fs {

template <typename T>
struct alignas(2 * sizeof(T)) cx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ cx<T> mk(T x, T y) {
  cx<T> r;
  r.x = x;
  r.y = y;
  return r;
}
template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk<T>(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk<T>(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ cx<T> operator*(T s, cx<T> a) { return mk<T>(s * a.x, s * a.y); }
template <typename T>
__device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return mk<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__device__ __forceinline__ cx<T> conj(cx<T> a) { return mk<T>(a.x, -a.y); }
// multiply by -i (forward) or +i (inverse): the quarter-turn of omega_4
template <bool INV, typename T>
__device__ __forceinline__ cx<T> rot4(cx<T> a) {
  return INV ? mk<T>(-a.y, a.x) : mk<T>(a.y, -a.x);
}
// multiply by a constant root of unity given as (cos, sin) of the forward angle:
// forward uses cos - i sin, inverse cos + i sin.
template <bool INV, typename T>
__device__ __forceinline__ cx<T> crot(cx<T> a, T c, T s) {
  const T si = INV ? s : -s;
  return mk<T>(a.x * c - a.y * si, a.x * si + a.y * c);
}

// Mathematical constants (cos/sin of rational multiples of pi), 20 digits.
#define FS_SQRT1_2 0.70710678118654752440
#define FS_COS_PI8 0.92387953251128675613
#define FS_SIN_PI8 0.38268343236508977173
#define FS_SIN_PI3 0.86602540378443864676
#define FS_COS_2PI5 0.30901699437494742410
#define FS_SIN_2PI5 0.95105651629515357212
#define FS_COS_4PI5 (-0.80901699437494742410)
#define FS_SIN_4PI5 0.58778525229247312917

// ------------------------------------------------------------ butterflies
// In-place R-point DFT of b[0..R-1]: X_k = sum_n b_n w^{nk}, w = e^{-+2 pi i/R}.
template <bool INV, typename T>
__device__ __forceinline__ void dft2(cx<T> *b) {
  cx<T> a0 = b[0], a1 = b[1];
  b[0] = a0 + a1;
  b[1] = a0 - a1;
}

template <bool INV, typename T>
__device__ __forceinline__ void dft3(cx<T> *b) {
  const T h = T(FS_SIN_PI3);
  cx<T> t = b[1] + b[2];
  cx<T> d = b[1] - b[2];
  cx<T> m = b[0] - T(0.5) * t;
  // (-+ i sqrt(3)/2) d
  cx<T> r = INV ? mk<T>(-h * d.y, h * d.x) : mk<T>(h * d.y, -h * d.x);
  b[0] = b[0] + t;
  b[1] = m + r;
  b[2] = m - r;
}

template <bool INV, typename T>
__device__ __forceinline__ void dft4(cx<T> *b) {
  cx<T> t0 = b[0] + b[2], t1 = b[0] - b[2];
  cx<T> t2 = b[1] + b[3], t3 = rot4<INV>(b[1] - b[3]);
  b[0] = t0 + t2;
  b[2] = t0 - t2;
  b[1] = t1 + t3;
  b[3] = t1 - t3;
}

template <bool INV, typename T>
__device__ __forceinline__ void dft5(cx<T> *b) {
  const T c1 = T(FS_COS_2PI5), s1 = T(FS_SIN_2PI5);
  const T c2 = T(FS_COS_4PI5), s2 = T(FS_SIN_4PI5);
  cx<T> t1 = b[1] + b[4], d1 = b[1] - b[4];
  cx<T> t2 = b[2] + b[3], d2 = b[2] - b[3];
  cx<T> a0 = b[0];
  cx<T> r1 = a0 + c1 * t1 + c2 * t2;
  cx<T> r2 = a0 + c2 * t1 + c1 * t2;
  cx<T> q1 = s1 * d1 + s2 * d2;  // multiplies -+ i
  cx<T> q2 = s2 * d1 - s1 * d2;
  cx<T> i1 = rot4<INV>(q1);
  cx<T> i2 = rot4<INV>(q2);
  b[0] = a0 + t1 + t2;
  b[1] = r1 + i1;
  b[4] = r1 - i1;
  b[2] = r2 + i2;
  b[3] = r2 - i2;
}

template <bool INV, typename T>
__device__ __forceinline__ void dft8(cx<T> *b) {
  cx<T> e[4] = {b[0], b[2], b[4], b[6]};
  cx<T> o[4] = {b[1], b[3], b[5], b[7]};
  dft4<INV>(e);
  dft4<INV>(o);
  const T r = T(FS_SQRT1_2);
  cx<T> w1 = crot<INV>(o[1], r, r);
  cx<T> w2 = rot4<INV>(o[2]);
  cx<T> w3 = crot<INV>(o[3], -r, r);
  b[0] = e[0] + o[0];
  b[4] = e[0] - o[0];
  b[1] = e[1] + w1;
  b[5] = e[1] - w1;
  b[2] = e[2] + w2;
  b[6] = e[2] - w2;
  b[3] = e[3] + w3;
  b[7] = e[3] - w3;
}

template <bool INV, typename T>
__device__ __forceinline__ void dft16(cx<T> *b) {
  cx<T> e[8], o[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    e[i] = b[2 * i];
    o[i] = b[2 * i + 1];
  }
  dft8<INV>(e);
  dft8<INV>(o);
  const T c1 = T(FS_COS_PI8), s1 = T(FS_SIN_PI8), r = T(FS_SQRT1_2);
  cx<T> w[8];
  w[0] = o[0];
  w[1] = crot<INV>(o[1], c1, s1);
  w[2] = crot<INV>(o[2], r, r);
  w[3] = crot<INV>(o[3], s1, c1);
  w[4] = rot4<INV>(o[4]);
  w[5] = crot<INV>(o[5], -s1, c1);
  w[6] = crot<INV>(o[6], -r, r);
  w[7] = crot<INV>(o[7], -c1, s1);
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    b[i] = e[i] + w[i];
    b[i + 8] = e[i] - w[i];
  }
}

// cos / sin (2 pi m / R), m < R, for the composite last-stage radices (20
// digits; rational multiples of pi)
template <int R>
struct RootsR;
template <>
struct RootsR<6> {
  static constexpr double c[6] = {1.0000000000000000000, 0.50000000000000000000, -0.50000000000000000000, -1.0000000000000000000, -0.50000000000000000000, 0.50000000000000000000};
  static constexpr double s[6] = {0.0, 0.86602540378443864676, 0.86602540378443864676, 0.0, -0.86602540378443864676, -0.86602540378443864676};
};
template <>
struct RootsR<10> {
  static constexpr double c[10] = {1.0000000000000000000, 0.80901699437494742410, 0.30901699437494742410, -0.30901699437494742410, -0.80901699437494742410, -1.0000000000000000000, -0.80901699437494742410, -0.30901699437494742410, 0.30901699437494742410, 0.80901699437494742410};
  static constexpr double s[10] = {0.0, 0.58778525229247312917, 0.95105651629515357212, 0.95105651629515357212, 0.58778525229247312917, 0.0, -0.58778525229247312917, -0.95105651629515357212, -0.95105651629515357212, -0.58778525229247312917};
};
template <>
struct RootsR<12> {
  static constexpr double c[12] = {1.0000000000000000000, 0.86602540378443864676, 0.50000000000000000000, 0.0, -0.50000000000000000000, -0.86602540378443864676, -1.0000000000000000000, -0.86602540378443864676, -0.50000000000000000000, 0.0, 0.50000000000000000000, 0.86602540378443864676};
  static constexpr double s[12] = {0.0, 0.50000000000000000000, 0.86602540378443864676, 1.0000000000000000000, 0.86602540378443864676, 0.50000000000000000000, 0.0, -0.50000000000000000000, -0.86602540378443864676, -1.0000000000000000000, -0.86602540378443864676, -0.50000000000000000000};
};
template <>
struct RootsR<20> {
  static constexpr double c[20] = {1.0000000000000000000, 0.95105651629515357212, 0.80901699437494742410, 0.58778525229247312917, 0.30901699437494742410, 0.0, -0.30901699437494742410, -0.58778525229247312917, -0.80901699437494742410, -0.95105651629515357212, -1.0000000000000000000, -0.95105651629515357212, -0.80901699437494742410, -0.58778525229247312917, -0.30901699437494742410, 0.0, 0.30901699437494742410, 0.58778525229247312917, 0.80901699437494742410, 0.95105651629515357212};
  static constexpr double s[20] = {0.0, 0.30901699437494742410, 0.58778525229247312917, 0.80901699437494742410, 0.95105651629515357212, 1.0000000000000000000, 0.95105651629515357212, 0.80901699437494742410, 0.58778525229247312917, 0.30901699437494742410, 0.0, -0.30901699437494742410, -0.58778525229247312917, -0.80901699437494742410, -0.95105651629515357212, -1.0000000000000000000, -0.95105651629515357212, -0.80901699437494742410, -0.58778525229247312917, -0.30901699437494742410};
};
template <>
struct RootsR<24> {
  static constexpr double c[24] = {1.0000000000000000000, 0.96592582628906828675, 0.86602540378443864676, 0.70710678118654752440, 0.50000000000000000000, 0.25881904510252076235, 0.0, -0.25881904510252076235, -0.50000000000000000000, -0.70710678118654752440, -0.86602540378443864676, -0.96592582628906828675, -1.0000000000000000000, -0.96592582628906828675, -0.86602540378443864676, -0.70710678118654752440, -0.50000000000000000000, -0.25881904510252076235, 0.0, 0.25881904510252076235, 0.50000000000000000000, 0.70710678118654752440, 0.86602540378443864676, 0.96592582628906828675};
  static constexpr double s[24] = {0.0, 0.25881904510252076235, 0.50000000000000000000, 0.70710678118654752440, 0.86602540378443864676, 0.96592582628906828675, 1.0000000000000000000, 0.96592582628906828675, 0.86602540378443864676, 0.70710678118654752440, 0.50000000000000000000, 0.25881904510252076235, 0.0, -0.25881904510252076235, -0.50000000000000000000, -0.70710678118654752440, -0.86602540378443864676, -0.96592582628906828675, -1.0000000000000000000, -0.96592582628906828675, -0.86602540378443864676, -0.70710678118654752440, -0.50000000000000000000, -0.25881904510252076235};
};

template <int R, bool INV, typename T>
__device__ __forceinline__ void dftR(cx<T> *b);

// Twiddles w_R^{n2 k1} of the composite DFT below, n2 = N2.., k1 = K1..
// (compile-time indices, so every constant folds).
template <int A, int B, int N2, int K1, bool INV, typename T>
__device__ __forceinline__ void ab_twiddle(cx<T> (&y)[B][A]) {
  if constexpr (N2 < B) {
    if constexpr (K1 < A) {
      if constexpr (N2 > 0 && K1 > 0) {
        constexpr int m = (N2 * K1) % (A * B);
        constexpr double c = RootsR<A * B>::c[m], s = RootsR<A * B>::s[m];
        y[N2][K1] = crot<INV>(y[N2][K1], T(c), T(s));
      }
      ab_twiddle<A, B, N2, K1 + 1, INV>(y);
    } else {
      ab_twiddle<A, B, N2 + 1, 0, INV>(y);
    }
  }
}

// R = A B point DFT (A a power of two, B = 3 or 5) by one Cooley-Tukey split:
// with n = B n1 + n2 and k = k1 + A k2,
//   X_{k1 + A k2} = sum_{n2} w_B^{n2 k2} w_R^{n2 k1} sum_{n1} b_{B n1 + n2} w_A^{n1 k1},
// i.e. B DFTs of length A, the twiddles w_R^{n2 k1}, A DFTs of length B.
template <int A, int B, bool INV, typename T>
__device__ __forceinline__ void dft_ab(cx<T> *b) {
  cx<T> y[B][A];
#pragma unroll
  for (int n2 = 0; n2 < B; ++n2) {
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) y[n2][n1] = b[B * n1 + n2];
    dftR<A, INV>(y[n2]);
  }
  ab_twiddle<A, B, 1, 1, INV>(y);
#pragma unroll
  for (int k1 = 0; k1 < A; ++k1) {
    cx<T> z[B];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) z[n2] = y[n2][k1];
    dftR<B, INV>(z);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) b[k1 + A * k2] = z[k2];
  }
}

template <int R, bool INV, typename T>
__device__ __forceinline__ void dftR(cx<T> *b) {
  if constexpr (R == 2) dft2<INV>(b);
  else if constexpr (R == 3) dft3<INV>(b);
  else if constexpr (R == 4) dft4<INV>(b);
  else if constexpr (R == 5) dft5<INV>(b);
  else if constexpr (R == 8) dft8<INV>(b);
  else if constexpr (R == 16) dft16<INV>(b);
  else if constexpr (R == 6) dft_ab<2, 3, INV>(b);
  else if constexpr (R == 10) dft_ab<2, 5, INV>(b);
  else if constexpr (R == 12) dft_ab<4, 3, INV>(b);
  else if constexpr (R == 20) dft_ab<4, 5, INV>(b);
  else if constexpr (R == 24) dft_ab<8, 3, INV>(b);
}

// ------------------------------------------------------------ shared exchange
// Element idx of a segment lives at smem word pad(base + idx*sidx); one pad
// slot per 16 elements breaks the power-of-two strides of the early stages.
struct XLayout {
  int base;
  int sidx;
};
__device__ __forceinline__ int padi(int p) { return p + (p >> 4); }
__host__ __device__ constexpr int padded_len(int n) { return n + (n >> 4) + 1; }

// Twiddles w^r (r = 1..R-1) for one butterfly, w = tw[step]: the powers
// w, w^2, w^4, w^8 are read from the FP64-generated table (each rounded once)
// and the others formed by at most three complex products.
template <typename T, int R>
__device__ __forceinline__ void apply_twiddles(cx<T> *b, const cx<T> *__restrict__ tw, int step) {
  const cx<T> w1 = tw[step];
  if constexpr (R == 6 || R == 10 || R == 12 || R == 20 || R == 24) {
    // composite radices: w^r read from the table for powers of two r, the
    // others as the product of the highest power of two below r and the rest
    cx<T> w[R];
    w[1] = w1;
#pragma unroll
    for (int r = 2; r < R; ++r) {
      const int hb = r >= 16 ? 16 : (r >= 8 ? 8 : (r >= 4 ? 4 : 2));
      w[r] = r == hb ? tw[r * step] : cmul(w[hb], w[r - hb]);
    }
#pragma unroll
    for (int r = 1; r < R; ++r) b[r] = cmul(b[r], w[r]);
  } else if constexpr (R == 2) {
    b[1] = cmul(b[1], w1);
  } else {
    const cx<T> w2 = tw[2 * step];
    b[1] = cmul(b[1], w1);
    b[2] = cmul(b[2], w2);
    if constexpr (R >= 4) {
      const cx<T> w3 = cmul(w2, w1);
      b[3] = cmul(b[3], w3);
      if constexpr (R >= 5) {
        const cx<T> w4 = tw[4 * step];
        b[4] = cmul(b[4], w4);
        if constexpr (R >= 8) {
          const cx<T> w5 = cmul(w4, w1), w6 = cmul(w4, w2), w7 = cmul(w4, w3);
          b[5] = cmul(b[5], w5);
          b[6] = cmul(b[6], w6);
          b[7] = cmul(b[7], w7);
          if constexpr (R == 16) {
            const cx<T> w8 = tw[8 * step];
            b[8] = cmul(b[8], w8);
            b[9] = cmul(b[9], cmul(w8, w1));
            b[10] = cmul(b[10], cmul(w8, w2));
            b[11] = cmul(b[11], cmul(w8, w3));
            b[12] = cmul(b[12], cmul(w8, w4));
            b[13] = cmul(b[13], cmul(w8, w5));
            b[14] = cmul(b[14], cmul(w8, w6));
            b[15] = cmul(b[15], cmul(w8, w7));
          }
        }
      }
    }
  }
}

// One Stockham stage of radix R on the register tile.  Butterfly j = t + q*Tseg
// reads (already in registers, canonical slots q + r*E/R) elements j + r*L/R,
// applies the twiddles w_{Ns R}^{(j mod Ns) r}, and produces outputs that
// belong at indices expand(j) + r*Ns, expand(j) = (j/Ns)*Ns*R + j mod Ns.
template <typename T, int E, int R>
__device__ __forceinline__ void stage_compute(cx<T> (&v)[E], int t, int Tseg, int L, int Ns,
                                              const cx<T> *__restrict__ tw, int twmul) {
  if constexpr (E % R != 0) {
    return;
  } else {
    constexpr int Q = E / R;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int j = t + q * Tseg;
      cx<T> b[R];
#pragma unroll
      for (int r = 0; r < R; ++r) b[r] = v[q + r * Q];
      if (Ns > 1) {
        const int k = j % Ns;
        apply_twiddles<T, R>(b, tw, twmul * k * (L / (Ns * R)));
      }
      dftR<R, false>(b);
#pragma unroll
      for (int r = 0; r < R; ++r) v[q + r * Q] = b[r];
    }
  }
}

template <typename T, int E, int R>
__device__ __forceinline__ void stage_store(const cx<T> (&v)[E], cx<T> *sm, XLayout lay, int t,
                                            int Tseg, int Ns) {
  if constexpr (E % R != 0) {
    return;
  } else {
    constexpr int Q = E / R;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const int j = t + q * Tseg;
      const int k = j % Ns;
      const int base = (j / Ns) * Ns * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) sm[padi(lay.base + (base + r * Ns) * lay.sidx)] = v[q + r * Q];
    }
  }
}

// Full forward transform (e^{-2 pi i} kernel).  Every thread of the block must
// call it (it synchronises); inactive threads carry no data.  On return the
// register tile holds the result in canonical order; the caller must
// __syncthreads() before it next writes `sm` (other threads may still read the
// last exchange).  The inverse transform is obtained from the forward one by
// conjugating input and output (the iDFT identity stated after Eq. DFT2).
template <typename T, int E>
__device__ __forceinline__ void fft_run(cx<T> (&v)[E], cx<T> *sm, XLayout lay, bool active, int t, int Tseg,
                        int L, const RadixPlan &rp, const cx<T> *__restrict__ tw, int twmul) {
  int Ns = 1;
  const int n = rp.n;
  for (int st = 0; st < n; ++st) {
    const int R = rp.r[st];
    if (st > 0 && active) {
#pragma unroll
      for (int s = 0; s < E; ++s) v[s] = sm[padi(lay.base + (t + Tseg * s) * lay.sidx)];
    }
    if (active) {
      switch (R) {
        case 2: stage_compute<T, E, 2>(v, t, Tseg, L, Ns, tw, twmul); break;
        case 3: stage_compute<T, E, 3>(v, t, Tseg, L, Ns, tw, twmul); break;
        case 4: stage_compute<T, E, 4>(v, t, Tseg, L, Ns, tw, twmul); break;
        case 5: stage_compute<T, E, 5>(v, t, Tseg, L, Ns, tw, twmul); break;
        case 8: stage_compute<T, E, 8>(v, t, Tseg, L, Ns, tw, twmul); break;
        case 16: stage_compute<T, E, 16>(v, t, Tseg, L, Ns, tw, twmul); break;
        default: break;
      }
    }
    if (st < n - 1) {
      __syncthreads();
      if (active) {
        switch (R) {
          case 2: stage_store<T, E, 2>(v, sm, lay, t, Tseg, Ns); break;
          case 3: stage_store<T, E, 3>(v, sm, lay, t, Tseg, Ns); break;
          case 4: stage_store<T, E, 4>(v, sm, lay, t, Tseg, Ns); break;
          case 5: stage_store<T, E, 5>(v, sm, lay, t, Tseg, Ns); break;
          case 8: stage_store<T, E, 8>(v, sm, lay, t, Tseg, Ns); break;
          case 16: stage_store<T, E, 16>(v, sm, lay, t, Tseg, Ns); break;
          default: break;
        }
      }
      __syncthreads();
    }
    Ns *= R;
  }
}

// ------------------------------------------------------------ compile-time engine
// For lengths L = m 2^k (m in {1, 3, 5}) and tiles E = m 2^j the stage
// radices, the running product Ns and every index stride are compile-time
// constants, so the shared memory addresses reduce to a per-thread base plus
// immediate offsets.  Stages: power-of-two radices, largest dividing E
// first, as in fft_run with the plan of radix_plan (identical for m = 1); for
// m = 3, 5 the last stage takes the whole remaining factor m 2^j once it
// divides E (a composite radix 6, 10, 12, 20 or 24 in registers: one
// exchange fewer than the runtime plan's separate 2^j and m stages).
// Ns = product of the earlier radices and Tseg = L/E are therefore powers of
// two at every stage.
namespace ct {
constexpr int first_radix(int E) { return E % 16 == 0 ? 16 : (E % 8 == 0 ? 8 : (E % 4 == 0 ? 4 : 2)); }
constexpr int odd_of(int x) { return x % 2 == 0 ? odd_of(x / 2) : x; }
constexpr int pick(int rem, int E) {
  if (rem == 3 || rem == 5) return rem;  // the odd stage, last
  // the rest fits the tile and carries the odd factor: one composite stage
  // of radix rem = m 2^j (6, 10, 12, 20 or 24), last
  if (odd_of(rem) != 1 && E % rem == 0) return rem;
  int r = first_radix(E);
  while (rem % r) r >>= 1;
  return r;
}
constexpr int nstages(int L, int E) {
  int n = 0;
  for (int rem = L; rem > 1; rem /= pick(rem, E)) ++n;
  return n;
}
constexpr int radix(int L, int E, int st) {
  int rem = L;
  for (int i = 0; i < st; ++i) rem /= pick(rem, E);
  return pick(rem, E);
}
constexpr int ns(int L, int E, int st) {
  int rem = L, p = 1;
  for (int i = 0; i < st; ++i) {
    const int r = pick(rem, E);
    rem /= r;
    p *= r;
  }
  return p;
}
constexpr bool is_pow2(int x) { return x > 0 && (x & (x - 1)) == 0; }
// lengths and tiles the engine takes: odd part of L in {1, 3, 5}, E carrying
// the same odd part, L/E a power of two
constexpr int odd_part(int x) { return x % 2 == 0 ? odd_part(x / 2) : x; }
constexpr bool ok(int L, int E) {
  return L > 0 && E > 0 && L % E == 0 && (odd_part(L) == 1 || odd_part(L) == 3 || odd_part(L) == 5) &&
         odd_part(E) == odd_part(L) && is_pow2(L / E);
}
}  // namespace ct

template <typename T, int E, int L, int SIDX, int TWMUL, int ST>
__device__ __forceinline__ void fft_ct_from(cx<T> (&v)[E], cx<T> *sm, int base, bool active, int t,
                                            const cx<T> *__restrict__ tw) {
  constexpr int NST = ct::nstages(L, E);
  if constexpr (ST < NST) {
    constexpr int R = ct::radix(L, E, ST);
    constexpr int NS = ct::ns(L, E, ST);
    constexpr int Tseg = L / E;
    constexpr int Q = E / R;
    static_assert(E % R == 0, "radix must divide the tile");
    static_assert(ct::is_pow2(NS) && ct::is_pow2(Tseg), "odd stage last: Ns and Tseg are powers of two");
    if constexpr (ST > 0) {
      if (active) {
        const int pb = base + t * SIDX;
        const int ppb = padi(pb);
#pragma unroll
        for (int s = 0; s < E; ++s) {
          // canonical slot s <-> index t + Tseg*s
          const int off = Tseg * SIDX * s;
          v[s] = sm[(off % 16 == 0) ? ppb + off + off / 16 : padi(pb + off)];
        }
      }
    }
    if (active) {
#pragma unroll
      for (int q = 0; q < Q; ++q) {
        const int j = t + q * Tseg;
        cx<T> b[R];
#pragma unroll
        for (int r = 0; r < R; ++r) b[r] = v[q + r * Q];
        if constexpr (NS > 1) {
          const int k = j & (NS - 1);
          apply_twiddles<T, R>(b, tw, TWMUL * (L / (NS * R)) * k);
        }
        dftR<R, false>(b);
#pragma unroll
        for (int r = 0; r < R; ++r) v[q + r * Q] = b[r];
      }
    }
    if constexpr (ST < NST - 1) {
      __syncthreads();
      if (active) {
        if constexpr (NS <= Tseg) {
          // Ns divides Tseg: expand(j) = expand(t) + q*Tseg*R
          const int bt = (t / NS) * (NS * R) + (t & (NS - 1));
          const int pb = base + bt * SIDX;
          const int ppb = padi(pb);
#pragma unroll
          for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int r = 0; r < R; ++r) {
              const int off = (q * Tseg * R + r * NS) * SIDX;
              sm[(off % 16 == 0) ? ppb + off + off / 16 : padi(pb + off)] = v[q + r * Q];
            }
        } else {
          // Tseg divides Ns: j < Ns within each q block, expand(j) = const(q) + t
          const int pb = base + t * SIDX;
          const int ppb = padi(pb);
#pragma unroll
          for (int q = 0; q < Q; ++q)
#pragma unroll
            for (int r = 0; r < R; ++r) {
              const int jq = q * Tseg;
              const int off = ((jq / NS) * (NS * R) + (jq % NS) + r * NS) * SIDX;
              sm[(off % 16 == 0) ? ppb + off + off / 16 : padi(pb + off)] = v[q + r * Q];
            }
        }
      }
      __syncthreads();
    }
    fft_ct_from<T, E, L, SIDX, TWMUL, ST + 1>(v, sm, base, active, t, tw);
  }
}

// Engine selection: LC > 0 selects the compile-time engine for length LC
// with exchange stride SIDX; LC == 0 the runtime engine.
template <typename T, int E, int LC, int SIDX, int TWMUL>
__device__ __forceinline__ void fft_any(cx<T> (&v)[E], cx<T> *sm, XLayout lay, bool active, int t,
                                        int Tseg, int L, const RadixPlan &rp,
                                        const cx<T> *__restrict__ tw) {
  if constexpr (LC > 0) {
    static_assert(SIDX > 0 && ct::ok(LC, E), "compile-time engine: length m 2^k, tile m 2^j, fixed stride");
    fft_ct_from<T, E, LC, SIDX, TWMUL, 0>(v, sm, lay.base, active, t, tw);
  } else {
    fft_run<T, E>(v, sm, lay, active, t, Tseg, L, rp, tw, TWMUL);
  }
}

template <typename T, int E>
__device__ __forceinline__ void conj_tile(cx<T> (&v)[E]) {
#pragma unroll
  for (int s = 0; s < E; ++s) v[s].y = -v[s].y;
}
template <typename T, int E>
__device__ __forceinline__ void swap_tile(cx<T> (&a)[E], cx<T> (&b)[E]) {
#pragma unroll
  for (int s = 0; s < E; ++s) {
    const cx<T> t = a[s];
    a[s] = b[s];
    b[s] = t;
  }
}

}  // namespace fs
