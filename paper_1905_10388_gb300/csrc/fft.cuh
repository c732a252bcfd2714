// Shared-memory Stockham FFT for lengths N = 2^k or 3 * 2^k, batched over
// `nb` contiguous sequences, executed cooperatively by all threads of a CTA.
//
// Each pass is one radix-R step of the self-sorting Stockham formulation:
// with Ns the length of the sub-transforms already formed, element j of the
// N/R-long input stream has position k = j mod Ns inside its sub-transform,
// is twiddled by W_N^{t k N/(R Ns)} for input t, combined by a length-R DFT,
// and written to (j / Ns) R Ns + k + t Ns.  A radix-3 pass runs first when
// N has the factor 3, then at most one radix-2 pass, then radix-4 passes
// until Ns = N.  The result is in natural order; no bit reversal.
//
// `tw` holds W_N^t = exp(-2 pi i t / N), t < N, computed on the host in FP64
// (libm) and rounded to T.  sign = -1: forward DFT (exp(-i...)); sign = +1:
// unnormalized inverse (exp(+i...)).  On GB300 the FP64 pipe issues one warp
// instruction per 64 cycles per sub-partition and bounds the FP64 transforms,
// so passes count FP64 instructions: the first pass skips its twiddles (all
// 1), the radix-3 butterfly takes 4 per point (sums, differences and FMAs
// with the constants -1/2 and sqrt(3)/2, instead of products with the cube
// roots of unity), radix-8 about 10 and radix-4 7 per point.
#pragma once
#include "common.cuh"

namespace spectau {

template <typename T>
__device__ __forceinline__ C<T> tw_get(const C<T>* tw, int idx, int sign) {
  C<T> w = tw[idx];
  if (sign > 0) w.y = -w.y;
  return w;
}

// Copy the twiddle table to shared memory (every FFT pass reads it).
template <typename T>
__device__ __forceinline__ void load_twiddles(C<T>* dst, const C<T>* __restrict__ src, int N) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) dst[i] = src[i];
}

// z times i (sign > 0) or -i (sign < 0): multiplication by exp(sign i pi / 2)
template <typename T>
__device__ __forceinline__ C<T> times_i(C<T> z, int sign) {
  return (sign < 0) ? mk<T>(z.y, -z.x) : mk<T>(-z.y, z.x);
}

// 4-point DFT of (c0, c1, c2, c3) with root exp(sign 2 pi i / 4)
template <typename T>
__device__ __forceinline__ void dft4(C<T> c0, C<T> c1, C<T> c2, C<T> c3, int sign, C<T>* d) {
  const C<T> p0 = cadd<T>(c0, c2), p1 = csub<T>(c0, c2), p2 = cadd<T>(c1, c3);
  const C<T> p3 = times_i<T>(csub<T>(c1, c3), sign);
  d[0] = cadd<T>(p0, p2);
  d[1] = cadd<T>(p1, p3);
  d[2] = csub<T>(p0, p2);
  d[3] = csub<T>(p1, p3);
}

// One radix-R Stockham pass (R = 2, 3, 4 or 8) over nb sequences.  Ns is
// 2^ns_log2 or 3 * 2^ns_log2 (ns_has3); Q = N / R.  Index arithmetic avoids
// run-time integer division: j / Ns and j mod Ns use shifts and a division
// by the constant 3; the sequence index comes from one FP32 multiply.
template <typename T, int R>
__device__ __forceinline__ void stockham_pass(const C<T>* __restrict__ x, C<T>* __restrict__ y, int N, int Ns,
                                              int ns_log2, bool ns_has3, const C<T>* __restrict__ tw, int sign,
                                              int nb) {
  const int Q = N / R;
  const int step = N / (R * Ns);
  const bool twiddle = Ns > 1;                     // the first pass's twiddles are all 1
  // butterflies of all nb sequences share one thread loop; the sequence of
  // butterfly idx is floor((idx + 1/2) / Q), exact in FP32 for idx < 2^20
  const float invQ = 1.0f / (float)Q;
  const int total = nb * Q;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int b = (nb == 1) ? 0 : __float2int_rd(((float)idx + 0.5f) * invQ);
    const int j = idx - b * Q;
    const C<T>* xb = x + b * N;
    C<T>* yb = y + b * N;
    {
      int jq = j >> ns_log2;                       // j / Ns
      if (ns_has3) jq /= 3;
      const int k = j - jq * Ns;                   // j mod Ns
      C<T> a[R];
#pragma unroll
      for (int t = 0; t < R; ++t) {
        a[t] = xb[j + t * Q];
        if (t > 0 && twiddle) a[t] = cmul<T>(a[t], tw_get<T>(tw, t * k * step, sign));
      }
      const int o = jq * R * Ns + k;
      if (R == 2) {
        yb[o] = cadd<T>(a[0], a[1]);
        yb[o + Ns] = csub<T>(a[0], a[1]);
      } else if (R == 3) {
        // root w = exp(sign 2 pi i / 3) = -1/2 + sign i sqrt(3)/2:
        // X_0 = a0 + (a1 + a2), X_{1,2} = a0 - (a1 + a2)/2 +- sign i (sqrt(3)/2) (a1 - a2)
        const T c = (sign < 0 ? (T)-1 : (T)1) * (T)0.86602540378443864676;
        const C<T> s12 = cadd<T>(a[1], a[2]), d12 = csub<T>(a[1], a[2]);
        const C<T> m = mk<T>(fma((T)-0.5, s12.x, a[0].x), fma((T)-0.5, s12.y, a[0].y));
        yb[o] = cadd<T>(a[0], s12);
        yb[o + Ns] = mk<T>(fma(-c, d12.y, m.x), fma(c, d12.x, m.y));
        yb[o + 2 * Ns] = mk<T>(fma(c, d12.y, m.x), fma(-c, d12.x, m.y));
      } else if (R == 4) {
        C<T> d[4];
        dft4<T>(a[0], a[1], a[2], a[3], sign, d);
#pragma unroll
        for (int q = 0; q < 4; ++q) yb[o + q * Ns] = d[q];
      } else {
        // 8-point DFT: X_q = E_{q mod 4} + w^q O_{q mod 4}, X_{q+4} = E_q - w^q O_q,
        // E / O the 4-point DFTs of the even / odd inputs, w = exp(sign 2 pi i / 8)
        C<T> e[4], f[4];
        dft4<T>(a[0], a[2], a[4], a[6], sign, e);
        dft4<T>(a[1], a[3], a[5], a[7], sign, f);
        const T h = (T)0.70710678118654752440;
        const C<T> g1 = (sign < 0) ? mk<T>(h * (f[1].x + f[1].y), h * (f[1].y - f[1].x))
                                   : mk<T>(h * (f[1].x - f[1].y), h * (f[1].y + f[1].x));   // w f1
        const C<T> g2 = times_i<T>(f[2], sign);                                             // w^2 f2
        const C<T> g3 = (sign < 0) ? mk<T>(h * (f[3].y - f[3].x), -h * (f[3].x + f[3].y))
                                   : mk<T>(-h * (f[3].x + f[3].y), h * (f[3].x - f[3].y));  // w^3 f3
        yb[o] = cadd<T>(e[0], f[0]);
        yb[o + 4 * Ns] = csub<T>(e[0], f[0]);
        yb[o + Ns] = cadd<T>(e[1], g1);
        yb[o + 5 * Ns] = csub<T>(e[1], g1);
        yb[o + 2 * Ns] = cadd<T>(e[2], g2);
        yb[o + 6 * Ns] = csub<T>(e[2], g2);
        yb[o + 3 * Ns] = cadd<T>(e[3], g3);
        yb[o + 7 * Ns] = csub<T>(e[3], g3);
      }
    }
  }
  __syncthreads();
}

// Batched FFT of nb contiguous length-N sequences: a radix-3 pass when 3 | N,
// then, for the remaining 2^m, one radix-2 (m = 1 mod 3) or radix-4 pass
// (m = 2 mod 3) and radix-8 passes.  `tw` should point to shared memory.
// Returns the buffer holding the result (x or y).  Ends with __syncthreads.
template <typename T>
__device__ C<T>* fft_batched(C<T>* x, C<T>* y, int N, int radix3, const C<T>* __restrict__ tw,
                             int sign, int nb) {
  int Ns = 1, lg = 0;
  bool has3 = false;
  if (radix3) {
    stockham_pass<T, 3>(x, y, N, Ns, lg, has3, tw, sign, nb);
    C<T>* t = x; x = y; y = t;
    Ns = 3;
    has3 = true;
  }
  const int M = N / Ns;                 // a power of two
  const int m = 31 - __clz(M);
  if (m % 3 == 1) {
    stockham_pass<T, 2>(x, y, N, Ns, lg, has3, tw, sign, nb);
    C<T>* t = x; x = y; y = t;
    Ns *= 2;
    lg += 1;
  } else if (m % 3 == 2) {
    stockham_pass<T, 4>(x, y, N, Ns, lg, has3, tw, sign, nb);
    C<T>* t = x; x = y; y = t;
    Ns *= 4;
    lg += 2;
  }
  for (; Ns < N; Ns *= 8, lg += 3) {
    stockham_pass<T, 8>(x, y, N, Ns, lg, has3, tw, sign, nb);
    C<T>* t = x; x = y; y = t;
  }
  return x;
}

}  // namespace spectau
