// Spectral transforms and dealiased products, sm_103a.
//
// Chebyshev axis (Sec. "Chebyshev basis"): with x_i = -cos(pi (i+1/2)/N),
// T_n(x_i) = (-1)^n cos(pi n (2i+1) / (2N)), so the forward transform
// c_n = (2 - delta_n0)/N sum_i g_i T_n(x_i) is a DCT-II and the backward
// g_i = sum_n c_n T_n(x_i) a DCT-III, both computed through one complex FFT
// of length N (Makhoul's even/odd reordering, v_j = g_{2j},
// v_{N-1-j} = g_{2j+1}, and a quarter-sample twiddle w_k = exp(-i pi k/2N)).
// The columns are complex (Fourier coefficients), and both maps are
// complex-linear, so one FFT serves the real and imaginary parts:
//   forward:  out_k = (w_k V_k + conj(w_k) V_{N-k}) / 2
//   backward: V_k = conj(w_k) (X_k - i X_{N-k}),  X_0 = d_0, X_k = d_k / 2,
//             d_n = (-1)^n c_n zero-padded to N (Sec. "Scaled transforms").
//
// Fourier axis (Sec. "Fourier basis"): real rows of length N_gx; two real
// fields a, b travel in one complex FFT z = a + i b.  Backward pads the
// N_x/2 stored modes (Nyquist dropped) and rebuilds the Hermitian spectrum;
// forward scales by 1/N_gx and keeps k < N_x/2.
//
// The x-row kernel fuses the backward x transforms of every grid field, the
// quadratic products F_e = sum coef * g_a * g_b on the dealiased grid, and
// the forward x transforms of the products, so grid-space data never leaves
// shared memory.  Data layouts: coefficient state [var][p][m] (double2),
// z-transformed rows gz[f][zg][p] and h[e][zg][p] (precision T), products'
// T coefficients fc[e][p][m] (double2).
#include <algorithm>

#include "fft.cuh"
#include "internal.h"

namespace spectau {


constexpr int Z_THREADS = 256;
constexpr int X_THREADS = 256;

// ---------------------------------------------------------------------------
// Chebyshev backward: coefficients (with optional i k_x) -> values on N_gz
// nodes, for the TP pencil columns [bx TP, bx TP + TP) of grid field by.
// ---------------------------------------------------------------------------
template <typename T, int TP>
__device__ __forceinline__ void cheb_backward_body(const ZDesc& d, int bx, int f, unsigned char* smem_raw) {
  const int Nc = d.Nc, Ng = d.Ng, P = d.P;
  const float invNg = 1.0f / (float)Ng, invNc = 1.0f / (float)Nc;
  C<T>* b0 = reinterpret_cast<C<T>*>(smem_raw);
  C<T>* b1 = b0 + TP * Ng;
  C<T>* tws = b1 + TP * Ng;
  const C<T>* wq = reinterpret_cast<const C<T>*>(d.wq);
  load_twiddles<T>(tws, reinterpret_cast<const C<T>*>(d.tw), Ng);
  const int p0 = bx * TP;
  const int var = d.f_var[f], op = d.f_op[f];
  // coefficients in the transform precision T: FP64 state, or its FP32 copy
  // in mixed mode, so that an FP32 transform executes no FP64 instruction
  const C<T>* src = reinterpret_cast<const C<T>*>(sizeof(T) == 8 ? (const void*)d.xc : (const void*)d.xc32) +
                    (size_t)var * d.xc_stride;
  const T* kxT = reinterpret_cast<const T*>(sizeof(T) == 8 ? (const void*)d.kx : (const void*)d.kx32);
  auto coef = [&](int c, int k) -> C<T> {  // X_k, zero beyond N_c
    const int p = p0 + c;
    if (p >= P || k >= Nc) return mk<T>(0, 0);
    C<T> x = src[(size_t)p * Nc + k];
    // kx holds k_x for every pencil followed by k_y (zero on 2D problems)
    if (op == SP_OP_DX) x = mk<T>(-kxT[p] * x.y, kxT[p] * x.x);
    else if (op == SP_OP_DY) x = mk<T>(-kxT[P + p] * x.y, kxT[P + p] * x.x);
    // weighted_in: transpose of the forward transform, c_k (2 - delta_k0) / N_g
    const T wgt = d.weighted_in ? (k == 0 ? (T)1 : (T)2) / (T)Ng : (T)1;
    const T s = ((k & 1) ? (T)-1 : (T)1) * (k == 0 ? (T)1 : (T)0.5) * wgt;
    return mk<T>(s * x.x, s * x.y);
  };
  for (int idx = threadIdx.x; idx < TP * Ng; idx += blockDim.x) {
    const int c = div_idx(idx, invNg), k = idx - c * Ng;
    const C<T> a = coef(c, k);
    const C<T> b = (k == 0) ? mk<T>(0, 0) : coef(c, Ng - k);
    // X_k - i X_{N-k}
    const C<T> dd = mk<T>(a.x + b.y, a.y - b.x);
    b0[idx] = cmulc<T>(dd, wq[k]);
  }
  __syncthreads();
  C<T>* res = fft_batched<T>(b0, b1, Ng, d.radix3, tws, +1, TP);
  C<T>* gz = reinterpret_cast<C<T>*>(d.gz);
  for (int idx = threadIdx.x; idx < TP * Ng; idx += blockDim.x) {
    const int zg = idx / TP, c = idx - zg * TP;
    const int p = p0 + c;
    if (p >= P) continue;
    const int j = (zg & 1) ? (Ng - 1 - (zg >> 1)) : (zg >> 1);
    gz[((size_t)f * Ng + zg) * P + p] = res[c * Ng + j];
  }
}

// ---------------------------------------------------------------------------
// Chebyshev forward: values on N_gz nodes -> first N_c coefficients (double2)
// ---------------------------------------------------------------------------
template <typename T, int TP>
__device__ __forceinline__ void cheb_forward_body(const ZDesc& d, int bx, int e, unsigned char* smem_raw) {
  const int Nc = d.Nc, Ng = d.Ng, P = d.P;
  const float invNg = 1.0f / (float)Ng, invNc = 1.0f / (float)Nc;
  C<T>* b0 = reinterpret_cast<C<T>*>(smem_raw);
  C<T>* b1 = b0 + TP * Ng;
  C<T>* tws = b1 + TP * Ng;
  const C<T>* wq = reinterpret_cast<const C<T>*>(d.wq);
  load_twiddles<T>(tws, reinterpret_cast<const C<T>*>(d.tw), Ng);
  const C<T>* h = reinterpret_cast<const C<T>*>(d.h);
  const int p0 = bx * TP;
  for (int idx = threadIdx.x; idx < TP * Ng; idx += blockDim.x) {
    const int zg = idx / TP, c = idx - zg * TP;
    const int p = p0 + c;
    const int j = (zg & 1) ? (Ng - 1 - (zg >> 1)) : (zg >> 1);
    b0[c * Ng + j] = (p < P) ? h[((size_t)e * Ng + zg) * P + p] : mk<T>(0, 0);
  }
  __syncthreads();
  C<T>* res = fft_batched<T>(b0, b1, Ng, d.radix3, tws, -1, TP);
  const T inv = (T)1 / (T)Ng;
  for (int idx = threadIdx.x; idx < TP * Nc; idx += blockDim.x) {
    const int c = div_idx(idx, invNc), k = idx - c * Nc;
    const int p = p0 + c;
    if (p >= P) continue;
    const C<T> Vk = res[c * Ng + k];
    const C<T> Vr = res[c * Ng + (k == 0 ? 0 : Ng - k)];
    const C<T> w = wq[k];
    const C<T> o = cadd<T>(cmul<T>(w, Vk), cmulc<T>(Vr, w));
    // out_k = 2 (-1)^k sum_i g_i T_k(x_i): coefficients (2 - delta_k0)/N_g
    // times that sum; transpose of the backward transform: the sum itself
    const T s = ((k & 1) ? (T)-1 : (T)1) * (d.unweighted ? (T)0.5 : (k == 0 ? inv * (T)0.5 : inv));
    // the k_x = 0 column is the transform of a real function: its
    // coefficients are real (rounding of the two half-spectrum terms would
    // leave an O(eps) imaginary part)
    d.fc[((size_t)e * P + p) * Nc + k] = make_double2((double)(o.x * s), p == 0 ? 0.0 : (double)(o.y * s));
  }
}

// ---------------------------------------------------------------------------
// Fourier rows: [backward x] -> [products] -> [forward x] for z-row `row`
//   mode & 1: input spectra from gz (else real rows from grid_in)
//   mode & 2: evaluate the bilinear terms (else pass the fields through)
//   mode & 4: output spectra to h (else real rows to grid_out)
// ---------------------------------------------------------------------------
// Field pairs transformed at once in the x-row kernel by default: the FFT
// buffers hold this many pairs, so many-field rows (3D: 15 fields) keep
// shared memory low enough for several CTAs per SM.  The one-problem FP64
// launch takes every pair in one round instead (XDesc::pairs): its FP64
// passes, not shared memory, bound it, and one round of five pairs gives the
// radix-8 passes 480 butterflies for 512 threads with three fewer barriers.
constexpr int X_PAIRS = 2;
constexpr int X_THREADS_FP64 = 512;

template <typename T>
__device__ __forceinline__ void fourier_rows_body(const XDesc& d, int row, unsigned char* smem_raw) {
  const int N = d.N, K = d.K, rows = d.rows, mode = d.mode, nf = d.nf, ne = d.ne;
  const float invN = 1.0f / (float)N, invK = 1.0f / (float)K;
  const int nout = (mode & 2) ? ne : nf;
  const int nbi = (nf + 1) / 2, nbo = (nout + 1) / 2;
  const int xp = d.pairs > 0 ? d.pairs : X_PAIRS;
  const int nbmax = max(min(nbi, xp), nbo);
  C<T>* b0 = reinterpret_cast<C<T>*>(smem_raw);
  C<T>* b1 = b0 + (size_t)nbmax * N;
  C<T>* tws = b1 + (size_t)nbmax * N;
  T* G = reinterpret_cast<T*>(tws + N);
  T* O = G + (size_t)nf * N;
  load_twiddles<T>(tws, reinterpret_cast<const C<T>*>(d.tw), N);
  const C<T>* gz = reinterpret_cast<const C<T>*>(d.gz);
  C<T>* h = reinterpret_cast<C<T>*>(d.h);
  const int tid = threadIdx.x, nt = blockDim.x;

  if (mode & 1) {
   for (int q0 = 0; q0 < nbi; q0 += xp) {
    const int nb = min(xp, nbi - q0);
    for (int idx = tid; idx < nb * N; idx += nt) {
      const int qq = div_idx(idx, invN);
      const int q = q0 + qq, k = idx - qq * N;
      const int fa = 2 * q, fb = 2 * q + 1;
      auto spec = [&](int f, int kk) -> C<T> {
        if (f >= nf) return mk<T>(0, 0);
        C<T> v = gz[((size_t)f * rows + row) * K + kk];
        if (d.xscale & 1) {            // transpose of forward x: (1/N) with k >= 1 halved
          const T sc = (kk == 0 ? (T)1 : (T)0.5) / (T)N;
          v = mk<T>(v.x * sc, v.y * sc);
        }
        return v;
      };
      C<T> z;
      if (k == 0) {
        z = mk<T>(spec(fa, 0).x, spec(fb, 0).x);
      } else if (k < K) {
        const C<T> A = spec(fa, k), B = spec(fb, k);
        z = mk<T>(A.x - B.y, A.y + B.x);               // A + i B
      } else if (k > N - K) {
        const C<T> A = spec(fa, N - k), B = spec(fb, N - k);
        z = mk<T>(A.x + B.y, B.x - A.y);               // conj(A) + i conj(B)
      } else {
        z = mk<T>(0, 0);
      }
      b0[idx] = z;
    }
    __syncthreads();
    C<T>* res = fft_batched<T>(b0, b1, N, d.radix3, tws, +1, nb);
    for (int idx = tid; idx < nb * N; idx += nt) {
      const int qq = div_idx(idx, invN);
      const int q = q0 + qq, i = idx - qq * N;
      G[(size_t)(2 * q) * N + i] = res[idx].x;
      if (2 * q + 1 < nf) G[(size_t)(2 * q + 1) * N + i] = res[idx].y;
    }
    __syncthreads();                             // b0 / b1 are reused by the next pairs
   }
  } else {
    for (int idx = tid; idx < nf * N; idx += nt) {
      const int f = idx / N, i = idx - f * N;
      G[idx] = (T)d.grid_in[((size_t)f * rows + row) * N + i];
    }
  }
  __syncthreads();

  const T* OUT = G;
  if (mode & 2) {
    // term tables in shared memory (at most MAX_TERMS terms)
    constexpr int MAX_TERMS = 16;
    __shared__ T tc[MAX_TERMS];
    __shared__ int ta[MAX_TERMS], tb[MAX_TERMS], te[MAX_TERMS];
    const int nterms = min(d.nterms, MAX_TERMS);
    const T* tcoef = reinterpret_cast<const T*>(sizeof(T) == 8 ? (const void*)d.t_coef : (const void*)d.t_coef32);
    if (tid < nterms) {
      tc[tid] = tcoef[tid]; ta[tid] = d.t_fa[tid] * N; tb[tid] = d.t_fb[tid] * N; te[tid] = d.t_eq[tid];
    }
    __syncthreads();
    // terms are grouped by equation (the host keeps them sorted by slot):
    // one pass over the terms, writing each equation's sum at its last term
    for (int i = tid; i < N; i += nt) {
      T acc = 0;
      for (int t = 0; t < nterms; ++t) {
        acc += tc[t] * G[ta[t] + i] * G[tb[t] + i];
        if (t + 1 == nterms || te[t + 1] != te[t]) {
          O[(size_t)te[t] * N + i] = acc;
          acc = 0;
        }
      }
    }
    __syncthreads();
    OUT = O;
  }

  if (mode & 4) {
    for (int idx = tid; idx < nbo * N; idx += nt) {
      const int q = div_idx(idx, invN), i = idx - q * N;
      const T a = OUT[(size_t)(2 * q) * N + i];
      const T b = (2 * q + 1 < nout) ? OUT[(size_t)(2 * q + 1) * N + i] : (T)0;
      b0[idx] = mk<T>(a, b);
    }
    __syncthreads();
    C<T>* res = fft_batched<T>(b0, b1, N, d.radix3, tws, -1, nbo);
    for (int idx = tid; idx < nbo * K; idx += nt) {
      const int q = div_idx(idx, invK), k = idx - q * K;
      // forward x: 1/N; transpose of backward x: (2 - delta_k0)
      const T s = (d.xscale & 2) ? ((k == 0) ? (T)0.5 : (T)1) : (T)1 / (T)(2 * N);
      const C<T> Z = res[(size_t)q * N + k];
      const C<T> Zr = res[(size_t)q * N + (k == 0 ? 0 : N - k)];
      h[((size_t)(2 * q) * rows + row) * K + k] = mk<T>((Z.x + Zr.x) * s, (Z.y - Zr.y) * s);
      if (2 * q + 1 < nout)
        h[((size_t)(2 * q + 1) * rows + row) * K + k] = mk<T>((Z.y + Zr.y) * s, (Zr.x - Z.x) * s);
    }
  } else {
    for (int idx = tid; idx < nout * N; idx += nt) {
      const int f = idx / N, i = idx - f * N;
      d.grid_out[((size_t)f * rows + row) * N + i] = (double)OUT[idx];
    }
  }
}

// ---------------------------------------------------------------------------
// Adjoint of the x-row stage for z-row `row`: given the forward fields'
// spectra gz[f] and the adjoint spectra of the products' forward transform
// hin[e] (already through the transpose of the z-forward transform), produce
// the adjoint spectra of the backward x transform of every grid field:
//   G_f = backward_x(gz_f)                      (forward grid fields)
//   R_e = (1/N) sum_{k<K} Re(hin_k e^{ikx})      (adjoint of forward x)
//   Abar_a += c G_b R_e, Abar_b += c G_a R_e     (adjoint of c g_a g_b)
//   out_k = (2 - delta_k0) sum_i Abar_i e^{-ikx_i}  (adjoint of backward x)
// ---------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void fourier_rows_adjoint_body(const XDesc& d, int row, unsigned char* smem_raw) {
  const int N = d.N, K = d.K, rows = d.rows, nf = d.nf, ne = d.ne;
  const float invN = 1.0f / (float)N;
  const int nbf = (nf + 1) / 2, nbe = (ne + 1) / 2;
  const int nbmax = max(nbf, nbe);
  C<T>* b0 = reinterpret_cast<C<T>*>(smem_raw);
  C<T>* b1 = b0 + (size_t)nbmax * N;
  C<T>* tws = b1 + (size_t)nbmax * N;
  T* G = reinterpret_cast<T*>(tws + N);
  T* R = G + (size_t)nf * N;
  load_twiddles<T>(tws, reinterpret_cast<const C<T>*>(d.tw), N);
  const C<T>* gz = reinterpret_cast<const C<T>*>(d.gz);
  const C<T>* hin = reinterpret_cast<const C<T>*>(d.hin);
  C<T>* out = reinterpret_cast<C<T>*>(d.gzadj);
  const int tid = threadIdx.x, nt = blockDim.x;
  // backward x of pairs of spectra from `src` (nfields) into `dst`, with
  // spectral scale sk(k)
  auto backward_pairs = [&](const C<T>* src, int nfields, T* dst, bool adjoint_scale) {
    const int nb = (nfields + 1) / 2;
    for (int idx = tid; idx < nb * N; idx += nt) {
      const int q = idx / N, k = idx - q * N;
      const int fa = 2 * q, fb = 2 * q + 1;
      auto spec = [&](int f, int kk) -> C<T> {
        if (f >= nfields) return mk<T>(0, 0);
        C<T> v = src[((size_t)f * rows + row) * K + kk];
        if (adjoint_scale) {
          const T sc = (kk == 0 ? (T)1 : (T)0.5) / (T)N;
          v = mk<T>(v.x * sc, v.y * sc);
        }
        return v;
      };
      C<T> z;
      if (k == 0) {
        z = mk<T>(spec(fa, 0).x, spec(fb, 0).x);
      } else if (k < K) {
        const C<T> A = spec(fa, k), B = spec(fb, k);
        z = mk<T>(A.x - B.y, A.y + B.x);
      } else if (k > N - K) {
        const C<T> A = spec(fa, N - k), B = spec(fb, N - k);
        z = mk<T>(A.x + B.y, B.x - A.y);
      } else {
        z = mk<T>(0, 0);
      }
      b0[idx] = z;
    }
    __syncthreads();
    C<T>* res = fft_batched<T>(b0, b1, N, d.radix3, tws, +1, nb);
    for (int idx = tid; idx < nb * N; idx += nt) {
      const int q = div_idx(idx, invN), i = idx - q * N;
      dst[(size_t)(2 * q) * N + i] = res[idx].x;
      if (2 * q + 1 < nfields) dst[(size_t)(2 * q + 1) * N + i] = res[idx].y;
    }
    __syncthreads();
  };
  backward_pairs(gz, nf, G, false);
  backward_pairs(hin, ne, R, true);
  // adjoint products, pointwise, written over G
  constexpr int MAX_TERMS = 16, MAX_F = 16;
  __shared__ T tc[MAX_TERMS];
  __shared__ int ta[MAX_TERMS], tb[MAX_TERMS], te[MAX_TERMS];
  const int nterms = min(d.nterms, MAX_TERMS);
  const T* tcoef = reinterpret_cast<const T*>(sizeof(T) == 8 ? (const void*)d.t_coef : (const void*)d.t_coef32);
  if (tid < nterms) { tc[tid] = tcoef[tid]; ta[tid] = d.t_fa[tid]; tb[tid] = d.t_fb[tid]; te[tid] = d.t_eq[tid]; }
  __syncthreads();
  for (int i = tid; i < N; i += nt) {
    T g[MAX_F], a[MAX_F];
#pragma unroll
    for (int f = 0; f < MAX_F; ++f) { g[f] = (f < nf) ? G[(size_t)f * N + i] : (T)0; a[f] = 0; }
    for (int t = 0; t < nterms; ++t) {
      const T r = tc[t] * R[(size_t)te[t] * N + i];
#pragma unroll
      for (int f = 0; f < MAX_F; ++f) {
        if (f == ta[t]) a[f] += r * g[tb[t]];
        if (f == tb[t]) a[f] += r * g[ta[t]];
      }
    }
#pragma unroll
    for (int f = 0; f < MAX_F; ++f)
      if (f < nf) G[(size_t)f * N + i] = a[f];
  }
  __syncthreads();
  // forward x of the adjoint fields, scaled by (2 - delta_k0) N
  for (int idx = tid; idx < nbf * N; idx += nt) {
    const int q = idx / N, i = idx - q * N;
    const T x = G[(size_t)(2 * q) * N + i];
    const T y = (2 * q + 1 < nf) ? G[(size_t)(2 * q + 1) * N + i] : (T)0;
    b0[idx] = mk<T>(x, y);
  }
  __syncthreads();
  C<T>* res = fft_batched<T>(b0, b1, N, d.radix3, tws, -1, nbf);
  for (int idx = tid; idx < nbf * K; idx += nt) {
    const int q = idx / K, k = idx - q * K;
    const C<T> Z = res[(size_t)q * N + k];
    const C<T> Zr = res[(size_t)q * N + (k == 0 ? 0 : N - k)];
    const T sc = (k == 0) ? (T)0.5 : (T)1;
    out[((size_t)(2 * q) * rows + row) * K + k] = mk<T>((Z.x + Zr.x) * sc, (Z.y - Zr.y) * sc);
    if (2 * q + 1 < nf)
      out[((size_t)(2 * q + 1) * rows + row) * K + k] = mk<T>((Z.y + Zr.y) * sc, (Zr.x - Z.x) * sc);
  }
}

// ---------------------------------------------------------------------------
// Fourier y axis (complex data, Sec. "Fourier basis"), for field f, z-row zg
// and the TX x-mode columns [bx TX, bx TX + TX): the N_y stored slots (FFT
// order, slot s = mode s for s < N_y/2 and s - N_y above, Nyquist slot
// dropped) and the N_gy grid points, one complex FFT of length N_gy per
// column.
//   backward (dir < 0): src[f][zg][s][ix] -> dst[f][zg][yg][ix],
//                       g_j = sum_n f_n exp(+2 pi i n j / N_gy)
//   forward  (dir > 0): src[f][zg][yg][ix] -> dst[f][zg][s][ix],
//                       f_n = (1/N_gy) sum_j g_j exp(-2 pi i n j / N_gy),
//                       Nyquist slot set to zero
// ---------------------------------------------------------------------------
template <typename T, int TX>
__device__ __forceinline__ void fourier_y_body(const YDesc& d, int bx, int zg, int f, unsigned char* smem_raw) {
  const int Ny = d.Ny, Ng = d.Ng, K = d.K;
  C<T>* b0 = reinterpret_cast<C<T>*>(smem_raw);
  C<T>* b1 = b0 + TX * Ng;
  C<T>* tws = b1 + TX * Ng;
  load_twiddles<T>(tws, reinterpret_cast<const C<T>*>(d.tw), Ng);
  const int ix0 = bx * TX;
  const C<T>* src = reinterpret_cast<const C<T>*>(d.src);
  C<T>* dst = reinterpret_cast<C<T>*>(d.dst);
  const int tid = threadIdx.x, nt = blockDim.x;
  const size_t plane = (size_t)f * d.nz + zg;
  const int half = Ny / 2;
  auto slot_index = [&](int sl) {       // position of slot sl in the length-N_gy spectrum
    const int n = sl < half ? sl : sl - Ny;
    return n < 0 ? n + Ng : n;
  };
  if (d.dir < 0) {
    for (int idx = tid; idx < TX * Ng; idx += nt) b0[idx] = mk<T>(0, 0);
    __syncthreads();
    const C<T>* in = src + plane * Ny * K;
    for (int idx = tid; idx < TX * Ny; idx += nt) {
      const int sl = idx / TX, c = idx - sl * TX;
      const int ix = ix0 + c;
      if (sl == half || ix >= K) continue;
      b0[c * Ng + slot_index(sl)] = in[(size_t)sl * K + ix];
    }
    __syncthreads();
    const C<T>* res = fft_batched<T>(b0, b1, Ng, d.radix3, tws, +1, TX);
    C<T>* out = dst + plane * Ng * K;
    for (int idx = tid; idx < TX * Ng; idx += nt) {
      const int yg = idx / TX, c = idx - yg * TX;
      const int ix = ix0 + c;
      if (ix < K) out[(size_t)yg * K + ix] = res[c * Ng + yg];
    }
  } else {
    const C<T>* in = src + plane * Ng * K;
    for (int idx = tid; idx < TX * Ng; idx += nt) {
      const int yg = idx / TX, c = idx - yg * TX;
      const int ix = ix0 + c;
      b0[c * Ng + yg] = (ix < K) ? in[(size_t)yg * K + ix] : mk<T>(0, 0);
    }
    __syncthreads();
    const C<T>* res = fft_batched<T>(b0, b1, Ng, d.radix3, tws, -1, TX);
    const T inv = (T)1 / (T)Ng;
    C<T>* out = dst + plane * Ny * K;
    for (int idx = tid; idx < TX * Ny; idx += nt) {
      const int sl = idx / TX, c = idx - sl * TX;
      const int ix = ix0 + c;
      if (ix >= K) continue;
      const C<T> v = (sl == half) ? mk<T>(0, 0) : res[c * Ng + slot_index(sl)];
      out[(size_t)sl * K + ix] = mk<T>(v.x * inv, v.y * inv);
    }
  }
}

// ---------------------------------------------------------------------------
// kernels: one problem (descriptor by value) or a batch (descriptor table +
// work list of (problem, x, y) items, one per CTA)
// ---------------------------------------------------------------------------
template <typename T, int TP>
__global__ void __launch_bounds__(Z_THREADS) k_cheb_backward(ZDesc d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cheb_backward_body<T, TP>(d, blockIdx.x, blockIdx.y, smem_raw);
}
template <typename T, int TP>
__global__ void __launch_bounds__(Z_THREADS) k_cheb_backward_batched(const ZDesc* __restrict__ ds,
                                                                   const int4* __restrict__ work, int nwork,
                                                                   int* queue) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for_each_item(nwork, queue, [&](int it) {
    const int4 w = work[it];
    cheb_backward_body<T, TP>(ds[w.x], w.y, w.z, smem_raw);
  });
}
template <typename T, int TP>
__global__ void __launch_bounds__(Z_THREADS) k_cheb_forward(ZDesc d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cheb_forward_body<T, TP>(d, blockIdx.x, blockIdx.y, smem_raw);
}
template <typename T, int TP>
__global__ void __launch_bounds__(Z_THREADS) k_cheb_forward_batched(const ZDesc* __restrict__ ds,
                                                                  const int4* __restrict__ work, int nwork,
                                                                  int* queue) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for_each_item(nwork, queue, [&](int it) {
    const int4 w = work[it];
    cheb_forward_body<T, TP>(ds[w.x], w.y, w.z, smem_raw);
  });
}
constexpr int Y_TILE = 4;
// FP32: 48 registers, five CTAs per SM (about 27 KB of shared memory each)
template <typename T>
__global__ void __launch_bounds__(Z_THREADS, sizeof(T) == 8 ? 3 : 5) k_fourier_y(YDesc d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  fourier_y_body<T, Y_TILE>(d, blockIdx.x, blockIdx.y, blockIdx.z, smem_raw);
}
// FP32: 48 registers, so that five 256-thread CTAs fit an SM (the 3D rows'
// ~45 KB of shared memory allows five); FP64: 512 threads, 64 registers
template <typename T>
__global__ void __launch_bounds__(sizeof(T) == 8 ? X_THREADS_FP64 : X_THREADS, sizeof(T) == 8 ? 2 : 5)
    k_fourier_rows(XDesc d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  fourier_rows_body<T>(d, blockIdx.x, smem_raw);
}
template <typename T>
__global__ void __launch_bounds__(X_THREADS) k_fourier_rows_adjoint(XDesc d) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  fourier_rows_adjoint_body<T>(d, blockIdx.x, smem_raw);
}
template <typename T>
__global__ void __launch_bounds__(X_THREADS) k_fourier_rows_batched(const XDesc* __restrict__ ds,
                                                                  const int4* __restrict__ work, int nwork,
                                                                  int* queue) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  for_each_item(nwork, queue, [&](int it) {
    const int4 w = work[it];
    fourier_rows_body<T>(ds[w.x], w.y, smem_raw);
  });
}

// ---------------------------------------------------------------------------
// shared-memory sizes and launchers
// ---------------------------------------------------------------------------
size_t z_smem_bytes(int prec, int Ng, int tile) {
  return (2ull * tile + 1) * Ng * (prec ? sizeof(float2) : sizeof(double2));
}
size_t x_smem_bytes(int prec, int N, int mode, int nf, int ne, int pairs) {
  const int nout = (mode & 2) ? ne : nf;
  const int nbmax = std::max(std::min((nf + 1) / 2, pairs > 0 ? pairs : X_PAIRS), (nout + 1) / 2);
  const size_t esz = prec ? sizeof(float) : sizeof(double);
  size_t smem = (2ull * nbmax + 1) * N * 2 * esz + (size_t)nf * N * esz;
  if (mode & 2) smem += (size_t)ne * N * esz;
  return smem;
}

template <typename K>
static cudaError_t set_smem(K kernel, size_t smem) {
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

// Pencil columns per CTA for a single-problem z launch: the widest tile that
// still gives at least two CTAs per SM (152 SMs).
static int z_tile_for(int P, int nfields) {
  // 8 columns: (2 * 8 + 1) N_gz complex of shared memory, up to eight
  // 256-thread CTAs per SM at N_gz = 192 in FP32
  if ((long long)((P + 7) / 8) * nfields >= 2 * 152) return 8;
  return 4;
}

#define SPECTAU_TILE_DISPATCH(TILE, CALL) \
  switch (TILE) {                         \
    case 4: CALL(4); break;               \
    case 16: CALL(16); break;             \
    default: CALL(8); break;              \
  }

cudaError_t launch_cheb_backward(cudaStream_t s, int prec, const TransformPlan& pz, int P, int nf,
                                 const int32_t* f_var, const int32_t* f_op, const double* kx,
                                 const double2* xc, int xc_field_stride, void* gz, const float* kx32,
                                 const float2* xc32, int weighted_in) {
  ZDesc d{};
  d.weighted_in = weighted_in;
  d.Nc = pz.Nc; d.Ng = pz.Ng; d.radix3 = pz.radix3; d.P = P;
  d.tw = prec ? pz.tw32 : pz.tw64; d.wq = prec ? pz.dct32 : pz.dct64;
  d.f_var = f_var; d.f_op = f_op; d.kx = kx; d.xc = xc; d.xc_stride = xc_field_stride; d.gz = gz;
  d.kx32 = kx32; d.xc32 = xc32;
  if (prec && !xc32) return cudaErrorInvalidValue;
  const int tile = z_tile_for(P, nf);
  const size_t smem = z_smem_bytes(prec, pz.Ng, tile);
  dim3 grid((P + tile - 1) / tile, nf);
  cudaError_t e = cudaSuccess;
#define CALL(TT)                                                                                   \
  if (prec) {                                                                                      \
    if ((e = set_smem(k_cheb_backward<float, TT>, smem)) == cudaSuccess)                           \
      k_cheb_backward<float, TT><<<grid, Z_THREADS, smem, s>>>(d);                                  \
  } else {                                                                                         \
    if ((e = set_smem(k_cheb_backward<double, TT>, smem)) == cudaSuccess)                          \
      k_cheb_backward<double, TT><<<grid, Z_THREADS, smem, s>>>(d);                                 \
  }
  SPECTAU_TILE_DISPATCH(tile, CALL)
#undef CALL
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_cheb_forward(cudaStream_t s, int prec, const TransformPlan& pz, int P, int ne,
                                const void* h, double2* fc, int unweighted) {
  ZDesc d{};
  d.unweighted = unweighted;
  d.Nc = pz.Nc; d.Ng = pz.Ng; d.radix3 = pz.radix3; d.P = P;
  d.tw = prec ? pz.tw32 : pz.tw64; d.wq = prec ? pz.dct32 : pz.dct64;
  d.h = h; d.fc = fc;
  const int tile = z_tile_for(P, ne);
  const size_t smem = z_smem_bytes(prec, pz.Ng, tile);
  dim3 grid((P + tile - 1) / tile, ne);
  cudaError_t e = cudaSuccess;
#define CALL(TT)                                                                                   \
  if (prec) {                                                                                      \
    if ((e = set_smem(k_cheb_forward<float, TT>, smem)) == cudaSuccess)                            \
      k_cheb_forward<float, TT><<<grid, Z_THREADS, smem, s>>>(d);                                   \
  } else {                                                                                         \
    if ((e = set_smem(k_cheb_forward<double, TT>, smem)) == cudaSuccess)                           \
      k_cheb_forward<double, TT><<<grid, Z_THREADS, smem, s>>>(d);                                  \
  }
  SPECTAU_TILE_DISPATCH(tile, CALL)
#undef CALL
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_fourier_rows(cudaStream_t s, int prec, const TransformPlan& px, int rows, int P, int mode,
                                int nf, const void* gz, double* grid_in, double* grid_out, int nterms,
                                const int32_t* t_eq, const double* t_coef, const int32_t* t_fa,
                                const int32_t* t_fb, int ne, void* h, const float* t_coef32, int xscale) {
  XDesc d{};
  d.xscale = xscale;
  d.N = px.Ng; d.radix3 = px.radix3; d.rows = rows; d.K = P; d.mode = mode; d.nf = nf;
  d.tw = prec ? px.tw32 : px.tw64;
  d.gz = gz; d.grid_in = grid_in; d.grid_out = grid_out;
  d.nterms = nterms; d.t_eq = t_eq; d.t_coef = t_coef; d.t_fa = t_fa; d.t_fb = t_fb; d.ne = ne; d.h = h;
  d.t_coef32 = t_coef32;
  if (prec && nterms > 0 && !t_coef32) return cudaErrorInvalidValue;
  if (!prec)   // FP64: as many pairs per round as shared memory holds
    for (int q = (nf + 1) / 2; q > X_PAIRS && !d.pairs; --q)
      if (x_smem_bytes(prec, px.Ng, mode, nf, ne, q) <= 227 * 1024) d.pairs = q;
  const size_t smem = x_smem_bytes(prec, px.Ng, mode, nf, ne, d.pairs);
  cudaError_t e;
  if (prec) {
    if ((e = set_smem(k_fourier_rows<float>, smem)) != cudaSuccess) return e;
    k_fourier_rows<float><<<rows, X_THREADS, smem, s>>>(d);
  } else {
    if ((e = set_smem(k_fourier_rows<double>, smem)) != cudaSuccess) return e;
    k_fourier_rows<double><<<rows, X_THREADS_FP64, smem, s>>>(d);
  }
  return cudaGetLastError();
}

cudaError_t launch_fourier_rows_adjoint(cudaStream_t s, int prec, const TransformPlan& px, int rows, int P,
                                        int nf, const void* gz, int ne, const void* hin, int nterms,
                                        const int32_t* t_eq, const double* t_coef, const float* t_coef32,
                                        const int32_t* t_fa, const int32_t* t_fb, void* gzadj) {
  XDesc d{};
  d.N = px.Ng; d.radix3 = px.radix3; d.rows = rows; d.K = P; d.mode = 0; d.nf = nf; d.ne = ne;
  d.tw = prec ? px.tw32 : px.tw64;
  d.gz = gz; d.hin = hin; d.gzadj = gzadj;
  d.nterms = nterms; d.t_eq = t_eq; d.t_coef = t_coef; d.t_coef32 = t_coef32; d.t_fa = t_fa; d.t_fb = t_fb;
  if (nf > 16 || ne > 16 || (prec && nterms > 0 && !t_coef32)) return cudaErrorInvalidValue;
  const int nbmax = std::max((nf + 1) / 2, (ne + 1) / 2);
  const size_t esz = prec ? sizeof(float) : sizeof(double);
  const size_t smem = (2ull * nbmax + 1) * px.Ng * 2 * esz + (size_t)(nf + ne) * px.Ng * esz;
  cudaError_t e;
  if (prec) {
    if ((e = set_smem(k_fourier_rows_adjoint<float>, smem)) != cudaSuccess) return e;
    k_fourier_rows_adjoint<float><<<rows, X_THREADS, smem, s>>>(d);
  } else {
    if ((e = set_smem(k_fourier_rows_adjoint<double>, smem)) != cudaSuccess) return e;
    k_fourier_rows_adjoint<double><<<rows, X_THREADS, smem, s>>>(d);
  }
  return cudaGetLastError();
}

// batched launches: one CTA per work item
// Grid of a batched launch: one CTA per item, or (queue set) a persistent
// grid of as many CTAs as fit on the GPU at once (at most one per item).
template <typename K>
static int batched_grid(K kernel, int threads, size_t smem, int nwork, const int* queue) {
  if (queue == nullptr) return nwork;
  int dev = 0, sms = 1, per_sm = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  return std::max(1, std::min(nwork, sms * per_sm));
}

cudaError_t launch_cheb_backward_batched(cudaStream_t s, int prec, int tile, const ZDesc* ds, const int4* work,
                                         int nwork, int max_ng, int* queue) {
  const size_t smem = z_smem_bytes(prec, max_ng, tile);
  cudaError_t e = cudaSuccess;
#define CALL(TT)                                                                                   \
  if (prec) {                                                                                      \
    if ((e = set_smem(k_cheb_backward_batched<float, TT>, smem)) == cudaSuccess)                   \
      k_cheb_backward_batched<float, TT><<<batched_grid(k_cheb_backward_batched<float, TT>, Z_THREADS, smem, \
                                                        nwork, queue), Z_THREADS, smem, s>>>(ds, work, nwork, queue); \
  } else {                                                                                         \
    if ((e = set_smem(k_cheb_backward_batched<double, TT>, smem)) == cudaSuccess)                  \
      k_cheb_backward_batched<double, TT><<<batched_grid(k_cheb_backward_batched<double, TT>, Z_THREADS, smem, \
                                                         nwork, queue), Z_THREADS, smem, s>>>(ds, work, nwork, queue); \
  }
  SPECTAU_TILE_DISPATCH(tile, CALL)
#undef CALL
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_cheb_forward_batched(cudaStream_t s, int prec, int tile, const ZDesc* ds, const int4* work,
                                        int nwork, int max_ng, int* queue) {
  const size_t smem = z_smem_bytes(prec, max_ng, tile);
  cudaError_t e = cudaSuccess;
#define CALL(TT)                                                                                   \
  if (prec) {                                                                                      \
    if ((e = set_smem(k_cheb_forward_batched<float, TT>, smem)) == cudaSuccess)                    \
      k_cheb_forward_batched<float, TT><<<batched_grid(k_cheb_forward_batched<float, TT>, Z_THREADS, smem, \
                                                       nwork, queue), Z_THREADS, smem, s>>>(ds, work, nwork, queue); \
  } else {                                                                                         \
    if ((e = set_smem(k_cheb_forward_batched<double, TT>, smem)) == cudaSuccess)                   \
      k_cheb_forward_batched<double, TT><<<batched_grid(k_cheb_forward_batched<double, TT>, Z_THREADS, smem, \
                                                        nwork, queue), Z_THREADS, smem, s>>>(ds, work, nwork, queue); \
  }
  SPECTAU_TILE_DISPATCH(tile, CALL)
#undef CALL
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

cudaError_t launch_fourier_rows_batched(cudaStream_t s, int prec, const XDesc* ds, const int4* work, int nwork,
                                        size_t smem, int* queue) {
  cudaError_t e;
  if (prec) {
    if ((e = set_smem(k_fourier_rows_batched<float>, smem)) != cudaSuccess) return e;
    k_fourier_rows_batched<float><<<batched_grid(k_fourier_rows_batched<float>, X_THREADS, smem, nwork, queue),
                                    X_THREADS, smem, s>>>(ds, work, nwork, queue);
  } else {
    if ((e = set_smem(k_fourier_rows_batched<double>, smem)) != cudaSuccess) return e;
    k_fourier_rows_batched<double><<<batched_grid(k_fourier_rows_batched<double>, X_THREADS, smem, nwork, queue),
                                     X_THREADS, smem, s>>>(ds, work, nwork, queue);
  }
  return cudaGetLastError();
}

cudaError_t launch_fourier_y(cudaStream_t s, int prec, const TransformPlan& py, int dir, int nf, int nz, int K,
                             const void* src, void* dst) {
  YDesc d{};
  d.Ny = py.Nc; d.Ng = py.Ng; d.K = K; d.nz = nz; d.radix3 = py.radix3; d.dir = dir;
  d.tw = prec ? py.tw32 : py.tw64;
  d.src = src; d.dst = dst;
  if (nz > 65535 || nf > 65535) return cudaErrorInvalidValue;
  const size_t smem = (2ull * Y_TILE + 1) * py.Ng * (prec ? sizeof(float2) : sizeof(double2));
  dim3 grid((K + Y_TILE - 1) / Y_TILE, nz, nf);
  cudaError_t e;
  if (prec) {
    if ((e = set_smem(k_fourier_y<float>, smem)) != cudaSuccess) return e;
    k_fourier_y<float><<<grid, Z_THREADS, smem, s>>>(d);
  } else {
    if ((e = set_smem(k_fourier_y<double>, smem)) != cudaSuccess) return e;
    k_fourier_y<double><<<grid, Z_THREADS, smem, s>>>(d);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// CFL frequency (Sec. "Timestep determination"): the largest over the grid
// points of sum_v |g_v| * inv_d(axis_v, point).  grid [v][iz][iy][ix] FP64;
// inv_dz[iz] the inverse spacing of the Chebyshev nodes; the maximum is
// accumulated into *out as the bit pattern of a non-negative double (whose
// integer order is its numeric order).
// ---------------------------------------------------------------------------
__global__ void k_cfl_max(const double* __restrict__ grid, int nvel, const int* __restrict__ axes, int Ngx, int Ngy,
                          int Ngz, double inv_dx, double inv_dy, const double* __restrict__ inv_dz,
                          unsigned long long* __restrict__ out) {
  const size_t npts = (size_t)Ngx * Ngy * Ngz;
  double m = 0.0;
  for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < npts; q += (size_t)gridDim.x * blockDim.x) {
    const int iz = (int)(q / ((size_t)Ngx * Ngy));
    double f = 0.0;
    for (int v = 0; v < nvel; ++v) {
      const int ax = axes[v];
      const double inv = ax == 0 ? inv_dx : (ax == 1 ? inv_dy : inv_dz[iz]);
      f += fabs(grid[(size_t)v * npts + q]) * inv;
    }
    m = fmax(m, f);
  }
  // warp, then block maximum, one atomic per block
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ double wm[32];
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) wm[w] = m;
  __syncthreads();
  if (w == 0) {
    m = l < (int)(blockDim.x >> 5) ? wm[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (l == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
  }
}

cudaError_t launch_cfl_max(cudaStream_t s, const double* grid, int nvel, const int* axes, int Ngx, int Ngy, int Ngz,
                           double inv_dx, double inv_dy, const double* inv_dz, unsigned long long* out) {
  const size_t npts = (size_t)Ngx * Ngy * Ngz;
  const int threads = 256;
  const int blocks = (int)std::min<size_t>((npts + threads - 1) / threads, (size_t)152 * 8);
  k_cfl_max<<<blocks, threads, 0, s>>>(grid, nvel, axes, Ngx, Ngy, Ngz, inv_dx, inv_dy, inv_dz, out);
  return cudaGetLastError();
}

}  // namespace spectau
