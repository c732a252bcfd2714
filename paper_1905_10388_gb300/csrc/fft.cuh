// Shared-memory Stockham FFT for lengths N = 2^k or 3 * 2^k, batched over
// `nb` contiguous sequences, executed cooperatively by all threads of a CTA.
//
// Each pass is one radix-R step of the self-sorting Stockham formulation:
// with Ns the length of the sub-transforms already formed, element j of the
// N/R-long input stream has position k = j mod Ns inside its sub-transform,
// is twiddled by W_N^{t k N/(R Ns)} for input t, combined by a length-R DFT,
// and written to (j / Ns) R Ns + k + t Ns.  A radix-3 pass runs first when
// N has the factor 3, then radix-2 passes until Ns = N.  The result is in
// natural order; no bit reversal.
//
// `tw` holds W_N^t = exp(-2 pi i t / N), t < N, computed on the host in FP64
// (libm) and rounded to T.  sign = -1: forward DFT (exp(-i...)); sign = +1:
// unnormalized inverse (exp(+i...)).
#pragma once
#include "common.cuh"

namespace spectau {

template <typename T>
__device__ __forceinline__ C<T> tw_get(const C<T>* tw, int idx, int sign) {
  C<T> w = tw[idx];
  if (sign > 0) w.y = -w.y;
  return w;
}

// Returns the buffer holding the result (x or y).  Ends with __syncthreads.
template <typename T>
__device__ C<T>* fft_batched(C<T>* x, C<T>* y, int N, int radix3, const C<T>* __restrict__ tw,
                             int sign, int nb) {
  const int tid = threadIdx.x, nt = blockDim.x;
  int Ns = 1;
  if (radix3) {
    const int Q = N / 3;
    const C<T> w1 = tw_get<T>(tw, Q, sign), w2 = tw_get<T>(tw, 2 * Q, sign);
    for (int idx = tid; idx < nb * Q; idx += nt) {
      const int b = idx / Q, j = idx - b * Q;
      const C<T>* xb = x + b * N;
      C<T>* yb = y + b * N;
      const C<T> a0 = xb[j], a1 = xb[j + Q], a2 = xb[j + 2 * Q];
      // length-3 DFT, Ns = 1 (no twiddle)
      yb[3 * j] = cadd<T>(a0, cadd<T>(a1, a2));
      yb[3 * j + 1] = cadd<T>(a0, cadd<T>(cmul<T>(w1, a1), cmul<T>(w2, a2)));
      yb[3 * j + 2] = cadd<T>(a0, cadd<T>(cmul<T>(w2, a1), cmul<T>(w1, a2)));
    }
    __syncthreads();
    C<T>* t = x; x = y; y = t;
    Ns = 3;
  }
  const int H = N / 2;
  for (; Ns < N; Ns *= 2) {
    const int step = N / (2 * Ns);
    for (int idx = tid; idx < nb * H; idx += nt) {
      const int b = idx / H, j = idx - b * H;
      const int k = j % Ns;
      const C<T>* xb = x + b * N;
      C<T>* yb = y + b * N;
      const C<T> a0 = xb[j];
      const C<T> a1 = cmul<T>(xb[j + H], tw_get<T>(tw, k * step, sign));
      const int o = (j / Ns) * 2 * Ns + k;
      yb[o] = cadd<T>(a0, a1);
      yb[o + Ns] = csub<T>(a0, a1);
    }
    __syncthreads();
    C<T>* t = x; x = y; y = t;
  }
  return x;
}

}  // namespace spectau
