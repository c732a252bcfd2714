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

constexpr int Z_TILE = 8;       // pencils (columns) per CTA in the z kernels
constexpr int Z_THREADS = 256;
constexpr int X_THREADS = 256;

// ---------------------------------------------------------------------------
// Chebyshev backward: coefficients (with optional i k_x) -> values on N_gz nodes
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(Z_THREADS)
k_cheb_backward(int Nc, int Ng, int radix3, const C<T>* __restrict__ tw, const C<T>* __restrict__ wq, int P,
                const int32_t* __restrict__ f_var, const int32_t* __restrict__ f_op,
                const double* __restrict__ kx, const double2* __restrict__ xc, int xc_field_stride,
                C<T>* __restrict__ gz) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* b0 = reinterpret_cast<C<T>*>(smem_raw);
  C<T>* b1 = b0 + Z_TILE * Ng;
  C<T>* tws = b1 + Z_TILE * Ng;
  load_twiddles<T>(tws, tw, Ng);
  const int f = blockIdx.y;
  const int p0 = blockIdx.x * Z_TILE;
  const int var = f_var[f], op = f_op[f];
  const double2* src = xc + (size_t)var * xc_field_stride;
  auto coef = [&](int c, int k) -> double2 {  // X_k (double), zero beyond N_c
    const int p = p0 + c;
    if (p >= P || k >= Nc) return make_double2(0.0, 0.0);
    double2 x = src[(size_t)p * Nc + k];
    if (op == SP_OP_DX) x = make_double2(-kx[p] * x.y, kx[p] * x.x);
    const double s = ((k & 1) ? -1.0 : 1.0) * (k == 0 ? 1.0 : 0.5);
    return make_double2(s * x.x, s * x.y);
  };
  for (int idx = threadIdx.x; idx < Z_TILE * Ng; idx += blockDim.x) {
    const int c = idx / Ng, k = idx - c * Ng;
    const double2 a = coef(c, k);
    const double2 b = (k == 0) ? make_double2(0.0, 0.0) : coef(c, Ng - k);
    // X_k - i X_{N-k}
    const C<T> d = mk<T>((T)(a.x + b.y), (T)(a.y - b.x));
    b0[idx] = cmulc<T>(d, wq[k]);
  }
  __syncthreads();
  C<T>* res = fft_batched<T>(b0, b1, Ng, radix3, tws, +1, Z_TILE);
  for (int idx = threadIdx.x; idx < Z_TILE * Ng; idx += blockDim.x) {
    const int zg = idx / Z_TILE, c = idx - zg * Z_TILE;
    const int p = p0 + c;
    if (p >= P) continue;
    const int j = (zg & 1) ? (Ng - 1 - (zg >> 1)) : (zg >> 1);
    gz[((size_t)f * Ng + zg) * P + p] = res[c * Ng + j];
  }
}

// ---------------------------------------------------------------------------
// Chebyshev forward: values on N_gz nodes -> first N_c coefficients (double2)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(Z_THREADS)
k_cheb_forward(int Nc, int Ng, int radix3, const C<T>* __restrict__ tw, const C<T>* __restrict__ wq, int P,
               const C<T>* __restrict__ h, double2* __restrict__ fc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* b0 = reinterpret_cast<C<T>*>(smem_raw);
  C<T>* b1 = b0 + Z_TILE * Ng;
  C<T>* tws = b1 + Z_TILE * Ng;
  load_twiddles<T>(tws, tw, Ng);
  const int e = blockIdx.y;
  const int p0 = blockIdx.x * Z_TILE;
  for (int idx = threadIdx.x; idx < Z_TILE * Ng; idx += blockDim.x) {
    const int zg = idx / Z_TILE, c = idx - zg * Z_TILE;
    const int p = p0 + c;
    const int j = (zg & 1) ? (Ng - 1 - (zg >> 1)) : (zg >> 1);
    b0[c * Ng + j] = (p < P) ? h[((size_t)e * Ng + zg) * P + p] : mk<T>(0, 0);
  }
  __syncthreads();
  C<T>* res = fft_batched<T>(b0, b1, Ng, radix3, tws, -1, Z_TILE);
  const T inv = (T)1 / (T)Ng;
  for (int idx = threadIdx.x; idx < Z_TILE * Nc; idx += blockDim.x) {
    const int c = idx / Nc, k = idx - c * Nc;
    const int p = p0 + c;
    if (p >= P) continue;
    const C<T> Vk = res[c * Ng + k];
    const C<T> Vr = res[c * Ng + (k == 0 ? 0 : Ng - k)];
    const C<T> w = wq[k];
    const C<T> o = cadd<T>(cmul<T>(w, Vk), cmulc<T>(Vr, w));
    const T s = ((k & 1) ? (T)-1 : (T)1) * (k == 0 ? inv * (T)0.5 : inv);
    // the k_x = 0 column is the transform of a real function: its
    // coefficients are real (rounding of the two half-spectrum terms would
    // leave an O(eps) imaginary part)
    fc[((size_t)e * P + p) * Nc + k] = make_double2((double)(o.x * s), p == 0 ? 0.0 : (double)(o.y * s));
  }
}

// ---------------------------------------------------------------------------
// Fourier rows: [backward x] -> [products] -> [forward x]
//   mode & 1: input spectra from gz (else real rows from grid_in)
//   mode & 2: evaluate the bilinear terms (else pass the fields through)
//   mode & 4: output spectra to h (else real rows to grid_out)
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(X_THREADS)
k_fourier_rows(int N, int radix3, const C<T>* __restrict__ tw, int rows, int K, int mode, int nf,
               const C<T>* __restrict__ gz, const double* __restrict__ grid_in, double* __restrict__ grid_out,
               int nterms, const int32_t* __restrict__ t_eq, const double* __restrict__ t_coef,
               const int32_t* __restrict__ t_fa, const int32_t* __restrict__ t_fb, int ne,
               C<T>* __restrict__ h) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int nout = (mode & 2) ? ne : nf;
  const int nbi = (nf + 1) / 2, nbo = (nout + 1) / 2;
  const int nbmax = max(nbi, nbo);
  C<T>* b0 = reinterpret_cast<C<T>*>(smem_raw);
  C<T>* b1 = b0 + (size_t)nbmax * N;
  C<T>* tws = b1 + (size_t)nbmax * N;
  T* G = reinterpret_cast<T*>(tws + N);
  T* O = G + (size_t)nf * N;
  load_twiddles<T>(tws, tw, N);
  const int row = blockIdx.x;
  const int tid = threadIdx.x, nt = blockDim.x;

  if (mode & 1) {
    for (int idx = tid; idx < nbi * N; idx += nt) {
      const int q = idx / N, k = idx - q * N;
      const int fa = 2 * q, fb = 2 * q + 1;
      auto spec = [&](int f, int kk) -> C<T> {
        return (f < nf) ? gz[((size_t)f * rows + row) * K + kk] : mk<T>(0, 0);
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
    C<T>* res = fft_batched<T>(b0, b1, N, radix3, tws, +1, nbi);
    for (int idx = tid; idx < nbi * N; idx += nt) {
      const int q = idx / N, i = idx - q * N;
      G[(size_t)(2 * q) * N + i] = res[idx].x;
      if (2 * q + 1 < nf) G[(size_t)(2 * q + 1) * N + i] = res[idx].y;
    }
  } else {
    for (int idx = tid; idx < nf * N; idx += nt) {
      const int f = idx / N, i = idx - f * N;
      G[idx] = (T)grid_in[((size_t)f * rows + row) * N + i];
    }
  }
  __syncthreads();

  const T* OUT = G;
  if (mode & 2) {
    for (int idx = tid; idx < ne * N; idx += nt) {
      const int e = idx / N, i = idx - e * N;
      T acc = 0;
      for (int t = 0; t < nterms; ++t) {
        if (t_eq[t] != e) continue;
        acc += (T)t_coef[t] * G[(size_t)t_fa[t] * N + i] * G[(size_t)t_fb[t] * N + i];
      }
      O[idx] = acc;
    }
    __syncthreads();
    OUT = O;
  }

  if (mode & 4) {
    for (int idx = tid; idx < nbo * N; idx += nt) {
      const int q = idx / N, i = idx - q * N;
      const T a = OUT[(size_t)(2 * q) * N + i];
      const T b = (2 * q + 1 < nout) ? OUT[(size_t)(2 * q + 1) * N + i] : (T)0;
      b0[idx] = mk<T>(a, b);
    }
    __syncthreads();
    C<T>* res = fft_batched<T>(b0, b1, N, radix3, tws, -1, nbo);
    const T s = (T)1 / (T)(2 * N);
    for (int idx = tid; idx < nbo * K; idx += nt) {
      const int q = idx / K, k = idx - q * K;
      const C<T> Z = res[(size_t)q * N + k];
      const C<T> Zr = res[(size_t)q * N + (k == 0 ? 0 : N - k)];
      h[((size_t)(2 * q) * rows + row) * K + k] = mk<T>((Z.x + Zr.x) * s, (Z.y - Zr.y) * s);
      if (2 * q + 1 < nout)
        h[((size_t)(2 * q + 1) * rows + row) * K + k] = mk<T>((Z.y + Zr.y) * s, (Zr.x - Z.x) * s);
    }
  } else {
    for (int idx = tid; idx < nout * N; idx += nt) {
      const int f = idx / N, i = idx - f * N;
      grid_out[((size_t)f * rows + row) * N + i] = (double)OUT[idx];
    }
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename T>
static const C<T>* tw_of(const TransformPlan& pl) {
  return reinterpret_cast<const C<T>*>(sizeof(T) == 8 ? pl.tw64 : pl.tw32);
}
template <typename T>
static const C<T>* dct_of(const TransformPlan& pl) {
  return reinterpret_cast<const C<T>*>(sizeof(T) == 8 ? pl.dct64 : pl.dct32);
}

template <typename T>
static cudaError_t cheb_bwd_t(cudaStream_t s, const TransformPlan& pz, int P, int nf, const int32_t* f_var,
                              const int32_t* f_op, const double* kx, const double2* xc, int stride,
                              void* gz) {
  const size_t smem = (2ull * Z_TILE + 1) * pz.Ng * sizeof(C<T>);
  cudaFuncSetAttribute(k_cheb_backward<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid((P + Z_TILE - 1) / Z_TILE, nf);
  k_cheb_backward<T><<<grid, Z_THREADS, smem, s>>>(pz.Nc, pz.Ng, pz.radix3, tw_of<T>(pz), dct_of<T>(pz), P,
                                                    f_var, f_op, kx, xc, stride,
                                                    reinterpret_cast<C<T>*>(gz));
  return cudaGetLastError();
}

cudaError_t launch_cheb_backward(cudaStream_t s, int prec, const TransformPlan& pz, int P, int nf,
                                 const int32_t* f_var, const int32_t* f_op, const double* kx,
                                 const double2* xc, int xc_field_stride, void* gz) {
  return prec ? cheb_bwd_t<float>(s, pz, P, nf, f_var, f_op, kx, xc, xc_field_stride, gz)
              : cheb_bwd_t<double>(s, pz, P, nf, f_var, f_op, kx, xc, xc_field_stride, gz);
}

template <typename T>
static cudaError_t cheb_fwd_t(cudaStream_t s, const TransformPlan& pz, int P, int ne, const void* h,
                              double2* fc) {
  const size_t smem = (2ull * Z_TILE + 1) * pz.Ng * sizeof(C<T>);
  cudaFuncSetAttribute(k_cheb_forward<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  dim3 grid((P + Z_TILE - 1) / Z_TILE, ne);
  k_cheb_forward<T><<<grid, Z_THREADS, smem, s>>>(pz.Nc, pz.Ng, pz.radix3, tw_of<T>(pz), dct_of<T>(pz), P,
                                                   reinterpret_cast<const C<T>*>(h), fc);
  return cudaGetLastError();
}

cudaError_t launch_cheb_forward(cudaStream_t s, int prec, const TransformPlan& pz, int P, int ne,
                                const void* h, double2* fc) {
  return prec ? cheb_fwd_t<float>(s, pz, P, ne, h, fc) : cheb_fwd_t<double>(s, pz, P, ne, h, fc);
}

template <typename T>
static cudaError_t fourier_rows_t(cudaStream_t s, const TransformPlan& px, int rows, int P, int mode, int nf,
                                  const void* gz, double* grid_in, double* grid_out, int nterms,
                                  const int32_t* t_eq, const double* t_coef, const int32_t* t_fa,
                                  const int32_t* t_fb, int ne, void* h) {
  const int N = px.Ng;
  const int nout = (mode & 2) ? ne : nf;
  const int nbmax = std::max((nf + 1) / 2, (nout + 1) / 2);
  size_t smem = (2ull * nbmax + 1) * N * sizeof(C<T>) + (size_t)nf * N * sizeof(T);
  if (mode & 2) smem += (size_t)ne * N * sizeof(T);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  cudaFuncSetAttribute(k_fourier_rows<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  k_fourier_rows<T><<<rows, X_THREADS, smem, s>>>(N, px.radix3, tw_of<T>(px), rows, P, mode, nf,
                                                   reinterpret_cast<const C<T>*>(gz), grid_in, grid_out,
                                                   nterms, t_eq, t_coef, t_fa, t_fb, ne,
                                                   reinterpret_cast<C<T>*>(h));
  return cudaGetLastError();
}

cudaError_t launch_fourier_rows(cudaStream_t s, int prec, const TransformPlan& px, int rows, int P, int mode,
                                int nf, const void* gz, double* grid_in, double* grid_out, int nterms,
                                const int32_t* t_eq, const double* t_coef, const int32_t* t_fa,
                                const int32_t* t_fb, int ne, void* h) {
  return prec ? fourier_rows_t<float>(s, px, rows, P, mode, nf, gz, grid_in, grid_out, nterms, t_eq, t_coef,
                                      t_fa, t_fb, ne, h)
              : fourier_rows_t<double>(s, px, rows, P, mode, nf, gz, grid_in, grid_out, nterms, t_eq,
                                       t_coef, t_fa, t_fb, ne, h);
}

}  // namespace spectau
