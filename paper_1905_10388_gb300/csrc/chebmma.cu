// Chebyshev backward transform as a dense matrix product on the fifth-
// generation tensor cores (tcgen05), sm_103a.
//
// Sec. "Chebyshev basis": the values at the N_g Gauss nodes are
// g_i = sum_{n < N_z} c_n T_n(x_i), a matrix T (N_g x N_z) applied to every
// column of coefficients.  At small N_z (128 here) this is a dense
// contraction with intensity ~2 N_g N_z / ((N_z + N_g) 4 B) ~ 38 flop/B,
// above the FP32 CUDA-core ridge, so it runs on the tensor cores (the FFT-
// based DCT of transforms.cu is the other path).  The columns are the real
// and imaginary parts of every pencil of one variable, in the split FP32
// copy xs32[var][2p + c][m] that the solve epilogue writes, so the product
// is D[col][zg] = sum_m A[col][m] T[zg][m] with both operands K-major.
//
// Precision (mixed form, 1e-5 per field): kind::tf32 multiplies operands of
// 11 significant bits; each operand is split a = a_hi + a_lo with a_hi its
// TF32 truncation, and the product accumulates A_hi T_hi + A_hi T_lo +
// A_lo T_hi in FP32 (the dropped A_lo T_lo is ~2^-22 relative).  T_hi, T_lo
// are computed once on the host in FP64; A_hi and A_lo in shared memory.
//
// Per CTA: a tile of 128 columns (MMA M = 128), N = N_g, K in chunks of 32
// FP32 (one 128-byte swizzle row): TMA (cp.async.bulk.tensor) loads A and
// both halves of T into a two-stage ring, the threads split A, one thread
// issues the 12 MMAs of a chunk (tcgen05.mma, accumulator in TMEM) and
// commits them to the stage's empty barrier; the epilogue reads the
// accumulator with tcgen05.ld and writes every output field of the variable
// (the value, i k_x times it, i k_y times it) into the layout
// gz[f][zg][p] of the other transform kernels.  Every wait is bounded.
#include <cuda.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "internal.h"
#include "tma.cuh"

namespace spectau {

constexpr int CM_M = 128;          // columns per tile (MMA M)
constexpr int CM_KC = 32;          // K per chunk (FP32: 128 bytes)
constexpr int CM_STAGES = 2;
constexpr int CM_THREADS = 256;       // 8 warps: warps w and w + 4 share TMEM lane quadrant w
constexpr uint32_t CM_TMEM_COLS = 256;

__host__ __device__ inline size_t cm_stage_bytes(int Ng) {
  return (size_t)2 * CM_M * CM_KC * 4 + (size_t)2 * Ng * CM_KC * 4;   // A, A_lo, T_hi, T_lo
}
__host__ __device__ inline size_t cm_smem_bytes(int Ng) {
  return 1024 + CM_STAGES * cm_stage_bytes(Ng) + 256;                  // alignment pad, ring, barriers
}

bool cheb_mma_supported(int Nz, int Ng) {
  return Nz % CM_KC == 0 && Nz >= CM_KC && Ng % 16 == 0 && Ng >= 16 && Ng <= 256 &&
         cm_smem_bytes(Ng) <= 227 * 1024;
}

// K-major operand in the 128-byte swizzled layout (8-row atoms of 1024 B):
// start address, stride 1024 B between 8-row groups, descriptor version 1,
// swizzle mode 2 (128 B); the leading offset is unused for this layout.
__device__ __forceinline__ uint64_t cm_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// round to the nearest TF32 value (ties away from zero), in an FP32 container
__device__ __forceinline__ float cm_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

__device__ __forceinline__ void cm_mma(uint32_t tmem, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(
          tmem),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void cm_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ void cm_tma3(void* dst, const CUtensorMap* tm, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(
          smem_u32(dst)),
      "l"(tm), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void cm_tma2(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(tm), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

struct ChebMMAOut {
  int nv;                      // variables (grid.y)
  int var[16], nout[16];
  int f[16][3], op[16][3];     // output fields of each variable and their operators
};

__global__ void __launch_bounds__(CM_THREADS, 1)
    k_cheb_backward_mma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmThi,
                        const __grid_constant__ CUtensorMap tmTlo, ChebMMAOut o, int P, int Nz, int Ng,
                        const float* __restrict__ kx32, float* __restrict__ gz, DevStatus* st) {
  extern __shared__ unsigned char cm_raw[];
  unsigned char* base =
      reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(cm_raw) + 1023) & ~(uintptr_t)1023);
  const size_t sb = cm_stage_bytes(Ng);
  auto stA = [&](int s) { return reinterpret_cast<float*>(base + s * sb); };
  auto stAlo = [&](int s) { return reinterpret_cast<float*>(base + s * sb + CM_M * CM_KC * 4); };
  auto stThi = [&](int s) { return reinterpret_cast<float*>(base + s * sb + 2 * CM_M * CM_KC * 4); };
  auto stTlo = [&](int s) {
    return reinterpret_cast<float*>(base + s * sb + 2 * CM_M * CM_KC * 4 + (size_t)Ng * CM_KC * 4);
  };
  uint64_t* full = reinterpret_cast<uint64_t*>(base + CM_STAGES * sb);
  uint64_t* empty = full + CM_STAGES;
  uint64_t* done = empty + CM_STAGES;
  uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
  int* abort_flag = reinterpret_cast<int*>(tslot + 1);

  const int tile = blockIdx.x, vi = blockIdx.y;
  const int var = o.var[vi];
  const int nch = Nz / CM_KC;
  const uint32_t tx_bytes = (uint32_t)(CM_M * CM_KC * 4 + 2 * Ng * CM_KC * 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(CM_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    *abort_flag = 0;
    for (int s = 0; s < CM_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;

  auto issue = [&](int kc) {       // chunk kc into stage kc % CM_STAGES
    const int s = kc % CM_STAGES;
    mbar_expect_tx(&full[s], tx_bytes);
    cm_tma3(stA(s), &tmA, kc * CM_KC, tile * CM_M, var, &full[s]);
    cm_tma2(stThi(s), &tmThi, kc * CM_KC, 0, &full[s]);
    cm_tma2(stTlo(s), &tmTlo, kc * CM_KC, 0, &full[s]);
  };
  int issued = 0;
  if (threadIdx.x == 0)
    for (; issued < (nch < CM_STAGES ? nch : CM_STAGES); ++issued) issue(issued);

  // instruction descriptor: FP32 accumulator, TF32 A and B, both K-major,
  // N = Ng, M = 128
  const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(Ng >> 3) << 17) | ((uint32_t)(CM_M >> 4) << 24);
  int consumed = 0;
  for (int kc = 0; kc < nch; ++kc) {
    const int s = kc % CM_STAGES;
    if (!bounded_wait(&full[s], (kc / CM_STAGES) & 1)) atomicOr(abort_flag, 1);
    __syncthreads();
    if (*abort_flag) break;
    consumed = kc + 1;
    // A_hi = A rounded to TF32 (in place), A_lo = (A - A_hi) rounded to
    // TF32: both exactly representable, so the tensor core reads them as
    // they are; elementwise, so the swizzled placement does not matter
    float4* a4 = reinterpret_cast<float4*>(stA(s));
    float4* l4 = reinterpret_cast<float4*>(stAlo(s));
    for (int i = threadIdx.x; i < CM_M * CM_KC / 4; i += CM_THREADS) {
      float4 v = a4[i], h, l;
      h.x = cm_tf32(v.x); l.x = cm_tf32(v.x - h.x);
      h.y = cm_tf32(v.y); l.y = cm_tf32(v.y - h.y);
      h.z = cm_tf32(v.z); l.z = cm_tf32(v.z - h.z);
      h.w = cm_tf32(v.w); l.w = cm_tf32(v.w - h.w);
      a4[i] = h;
      l4[i] = l;
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic writes -> tensor-core reads
    __syncthreads();
    if (threadIdx.x == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint64_t dA = cm_desc(smem_u32(stA(s))), dL = cm_desc(smem_u32(stAlo(s)));
      const uint64_t dH = cm_desc(smem_u32(stThi(s))), dT = cm_desc(smem_u32(stTlo(s)));
#pragma unroll
      for (int ks = 0; ks < CM_KC / 8; ++ks) {       // K = 8 TF32 (32 bytes) per instruction
        const uint64_t k = (uint64_t)(ks * 32) >> 4;
        cm_mma(tmem, dA + k, dH + k, idesc, (kc | ks) ? 1u : 0u);
        cm_mma(tmem, dA + k, dT + k, idesc, 1u);
        cm_mma(tmem, dL + k, dH + k, idesc, 1u);
      }
      cm_commit(&empty[s]);                          // stage s is free once these MMAs are done
      if (issued < nch) {
        // the next chunk for this stage waits for the MMAs reading it
        if (bounded_wait(&empty[s], (kc / CM_STAGES) & 1)) {
          issue(issued);
          ++issued;
        } else {
          atomicOr(abort_flag, 1);
        }
      }
    }
  }
  if (threadIdx.x == 0) {
    cm_commit(done);                                  // every MMA issued so far
    if (!bounded_wait(done, 0)) atomicOr(abort_flag, 1);
    // copies issued but not consumed (after an abort) land before exit
    for (int q = consumed; q < issued; ++q) bounded_wait(&full[q % CM_STAGES], (q / CM_STAGES) & 1);
  }
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (*abort_flag) {
    if (threadIdx.x == 0) raise_status(st, SP_ERR_TIMEOUT, (long long)tile);
  } else {
    // epilogue: lane l of warp w reads accumulator row 32 (w & 3) + l, i.e.
    // column (pencil p, part c) of the tile, over every other 16-node chunk
    // (warps w and w + 4 split the nodes); its partner part is lane l ^ 1.
    // Output addresses and operator scales are fixed per thread.
    const int q4 = warp & 3, half = warp >> 2;
    const int col = tile * CM_M + 32 * q4 + lane;
    const bool valid = col < 2 * P;
    const int p = valid ? (col >> 1) : 0, c = col & 1;
    const int nout = o.nout[vi];
    const size_t zstride = (size_t)2 * P;
    float* outp[3];
    float sc[3];
    bool usew[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int qq = q < nout ? q : 0;
      const int op = o.op[vi][qq];
      const float kk = op == SP_OP_DX ? kx32[p] : kx32[P + p];
      // i k (x + i y) = -k y + i k x
      usew[q] = op != SP_OP_ID;
      sc[q] = c == 0 ? -kk : kk;
      outp[q] = gz + ((size_t)o.f[vi][qq] * Ng * P + p) * 2 + c;
    }
    for (int j0 = 16 * half; j0 < Ng; j0 += 32) {
      uint32_t r[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
            "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
          : "r"(tmem + ((uint32_t)(32 * q4) << 16) + (uint32_t)j0));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float v = __uint_as_float(r[i]);
        const float w = __shfl_xor_sync(0xffffffffu, v, 1);      // the other part of the same pencil
        const size_t off = (size_t)(j0 + i) * zstride;
#pragma unroll
        for (int q = 0; q < 3; ++q)
          if (q < nout && valid) outp[q][off] = usew[q] ? sc[q] * w : v;
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(CM_TMEM_COLS) : "memory");
}

// FP64 coefficients [S][P][Nz] complex -> split FP32 copy [S][2P][Nz]
__global__ void k_to_f32_split(const double2* __restrict__ src, float* __restrict__ dst, size_t ncols, int Nz) {
  const size_t total = ncols * Nz;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t col = i / Nz;
    const int m = (int)(i - col * Nz);
    const double2 v = src[i];
    dst[(2 * col) * Nz + m] = (float)v.x;
    dst[(2 * col + 1) * Nz + m] = (float)v.y;
  }
}

cudaError_t launch_to_f32_split(cudaStream_t s, const double2* src, float* dst, size_t ncols, int Nz) {
  const size_t total = ncols * Nz;
  if (total == 0) return cudaSuccess;
  k_to_f32_split<<<(int)std::min<size_t>((total + 255) / 256, 8192), 256, 0, s>>>(src, dst, ncols, Nz);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// host set-up: the transform matrix halves and the tensor maps
// ---------------------------------------------------------------------------
// nearest TF32 value of a finite float (ties away from zero, as cvt.rna):
// add half of the dropped 13-bit field to the magnitude, then clear it
static float tf32_round(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u = (u + 0x1000u) & 0xFFFFE000u;
  float r;
  std::memcpy(&r, &u, 4);
  return r;
}

typedef CUresult (*EncodeTiled)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encode_fn() {
  static EncodeTiled fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiled>(p);
  }
  return fn;
}

cudaError_t cheb_mma_setup(ChebMMA& c, int P, int Nz, int Ng, int S, cudaStream_t s) {
  static_assert(sizeof(CUtensorMap) == sizeof(c.tmA), "tensor map size");
  if (!cheb_mma_supported(Nz, Ng)) return cudaErrorInvalidValue;
  EncodeTiled enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  c.P = P; c.Nz = Nz; c.Ng = Ng; c.S = S;
  cudaError_t e;
  if (!c.xs32 && (e = cudaMalloc(&c.xs32, (size_t)S * 2 * P * Nz * sizeof(float))) != cudaSuccess) return e;
  if (!c.Thi && (e = cudaMalloc(&c.Thi, (size_t)Ng * Nz * sizeof(float))) != cudaSuccess) return e;
  if (!c.Tlo && (e = cudaMalloc(&c.Tlo, (size_t)Ng * Nz * sizeof(float))) != cudaSuccess) return e;
  // T[zg][m] = T_m(x_zg) = (-1)^m cos(pi m (zg + 1/2) / Ng) at the ascending
  // Gauss nodes x_zg = -cos(pi (zg + 1/2) / Ng), in FP64; hi = T rounded to
  // TF32, lo = (T - hi) rounded to TF32
  std::vector<float> hi((size_t)Ng * Nz), lo((size_t)Ng * Nz);
  const double pi = 3.14159265358979323846;
  for (int zg = 0; zg < Ng; ++zg)
    for (int m = 0; m < Nz; ++m) {
      const double t = ((m & 1) ? -1.0 : 1.0) * std::cos(pi * m * (zg + 0.5) / Ng);
      const float h = tf32_round((float)t);
      hi[(size_t)zg * Nz + m] = h;
      lo[(size_t)zg * Nz + m] = tf32_round((float)(t - (double)h));
    }
  if ((e = cudaMemcpyAsync(c.Thi, hi.data(), hi.size() * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(c.Tlo, lo.data(), lo.size() * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  // A: [S][2P][Nz] FP32, boxes of 32 (K) x 128 (columns) x 1 (variable),
  // out-of-range columns of the last tile read as zero
  {
    const cuuint64_t dims[3] = {(cuuint64_t)Nz, (cuuint64_t)2 * P, (cuuint64_t)S};
    const cuuint64_t strides[2] = {(cuuint64_t)Nz * 4, (cuuint64_t)2 * P * Nz * 4};
    const cuuint32_t box[3] = {CM_KC, CM_M, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    if (enc(reinterpret_cast<CUtensorMap*>(c.tmA), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, c.xs32, dims, strides, box,
            es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  for (int h = 0; h < 2; ++h) {
    const cuuint64_t dims[2] = {(cuuint64_t)Nz, (cuuint64_t)Ng};
    const cuuint64_t strides[1] = {(cuuint64_t)Nz * 4};
    const cuuint32_t box[2] = {CM_KC, (cuuint32_t)Ng};
    const cuuint32_t es[2] = {1, 1};
    if (enc(reinterpret_cast<CUtensorMap*>(h ? c.tmTlo : c.tmThi), CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
            h ? c.Tlo : c.Thi, dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return cudaErrorInvalidValue;
  }
  c.ready = true;
  return cudaSuccess;
}

void cheb_mma_free(ChebMMA& c) {
  if (c.xs32) cudaFree(c.xs32);
  if (c.Thi) cudaFree(c.Thi);
  if (c.Tlo) cudaFree(c.Tlo);
  c.xs32 = c.Thi = c.Tlo = nullptr;
  c.ready = false;
}

cudaError_t launch_cheb_backward_mma(cudaStream_t s, const ChebMMA& c, int nf, const int* f_var, const int* f_op,
                                     const float* kx32, void* gz, DevStatus* st) {
  if (!c.ready) return cudaErrorInvalidValue;
  ChebMMAOut o{};
  for (int f = 0; f < nf; ++f) {
    int vi = 0;
    while (vi < o.nv && o.var[vi] != f_var[f]) ++vi;
    if (vi == o.nv) {
      if (o.nv == 16) return cudaErrorInvalidValue;
      o.var[o.nv] = f_var[f];
      o.nout[o.nv++] = 0;
    }
    if (o.nout[vi] == 3) return cudaErrorInvalidValue;
    o.f[vi][o.nout[vi]] = f;
    o.op[vi][o.nout[vi]++] = f_op[f];
  }
  const size_t smem = cm_smem_bytes(c.Ng);
  cudaError_t e = cudaFuncSetAttribute(k_cheb_backward_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid((2 * c.P + CM_M - 1) / CM_M, o.nv);
  k_cheb_backward_mma<<<grid, CM_THREADS, smem, s>>>(*reinterpret_cast<const CUtensorMap*>(c.tmA),
                                                     *reinterpret_cast<const CUtensorMap*>(c.tmThi),
                                                     *reinterpret_cast<const CUtensorMap*>(c.tmTlo), o, c.P, c.Nz,
                                                     c.Ng, kx32, reinterpret_cast<float*>(gz), st);
  return cudaGetLastError();
}

}  // namespace spectau
