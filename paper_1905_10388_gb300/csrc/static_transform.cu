// Allocation-free backward transform (coefficients -> dealiased grid).
//
// The paper has no counterpart of this entry point; it exists for callers
// that cannot allocate device memory at the time they transform: code that
// runs while a stream is being captured into a CUDA graph (cudaMalloc and
// cudaFree are not capturable and may synchronize the device), programs whose
// device memory is owned entirely by another allocator or pool, and hosts
// that must not block on an implicit device synchronization.  Everything the
// transform needs beyond the caller's input and output -- the intermediate
// z-transformed fields and the twiddle tables -- lives in file-scope
// `static __device__` arrays of fixed size, reserved on every GPU that loads
// the library until the process exits.
//
// Set-up: the first call on a device (with that device current) resolves the
// device addresses of those arrays with cudaGetSymbolAddress; a host-side
// name of a __device__ array is not a device address.  Make that first call
// before any stream capture.  Later calls on the same device reuse the
// addresses; the set-up runs exactly once per device even when several host
// threads make their first calls at the same time (std::call_once).
//
// Sharing: every call uses the same arrays.  Calls that overlap on the GPU
// (different streams, or different threads, without ordering between them)
// race on them; order them on one stream or serialize them.  The twiddle
// tables are rewritten by each call before use, and the intermediate array is
// fully overwritten by each call before it is read, so no state carries over
// from the previous call.
#include <cstdio>
#include <cstring>
#include <mutex>

#include "internal.h"

namespace spectau {

// Capacity: nfields * N_gz * (N_x / 2) complex FP64 values of intermediate
// data (8 MiB), grid sizes up to 4096 (x) and 1536 (z).
constexpr size_t STATIC_SCRATCH_COMPLEX = 524288;
constexpr int STATIC_MAX_NGX = 4096;
constexpr int STATIC_MAX_NGZ = 1536;
constexpr int STATIC_MAX_FIELDS = 16;

static __device__ __align__(256) double2 s_scratch[STATIC_SCRATCH_COMPLEX];
static __device__ __align__(256) double2 s_tw_x[STATIC_MAX_NGX];
static __device__ __align__(256) double2 s_tw_z[STATIC_MAX_NGZ];
static __device__ __align__(256) double2 s_dct_z[STATIC_MAX_NGZ];
static __device__ __align__(256) int32_t s_field_index[STATIC_MAX_FIELDS] = {0, 1, 2,  3,  4,  5,  6,  7,
                                                                             8, 9, 10, 11, 12, 13, 14, 15};
static __device__ __align__(256) int32_t s_field_op[STATIC_MAX_FIELDS] = {0};

struct StaticAddrs {
  std::once_flag once;            // set-up runs once per device, whichever host thread gets there first
  cudaError_t setup = cudaSuccess;
  double2* scratch = nullptr;
  double2* tw_x = nullptr;
  double2* tw_z = nullptr;
  double2* dct_z = nullptr;
  int32_t* field_index = nullptr;
  int32_t* field_op = nullptr;
};
constexpr int STATIC_MAX_DEVICES = 64;
static StaticAddrs g_static[STATIC_MAX_DEVICES];

// exp(-2 pi i t / N) and exp(-i pi k / (2N)) with CUDA's sincospi
__global__ void k_static_twiddles(double2* tw, int N, double2* dct) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N; t += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * t / N, &s, &c);
    tw[t] = make_double2(c, -s);
    if (dct) {
      sincospi(0.5 * t / N, &s, &c);
      dct[t] = make_double2(c, -s);
    }
  }
}

static bool smooth(int N) {
  if (N <= 0) return false;
  if (N % 3 == 0) N /= 3;
  return (N & (N - 1)) == 0;
}

static sp_status report(char* errbuf, int errlen, sp_status code, const char* msg) {
  if (errbuf && errlen > 0) {
    std::strncpy(errbuf, msg, (size_t)errlen - 1);
    errbuf[errlen - 1] = '\0';
  }
  return code;
}

}  // namespace spectau

using namespace spectau;

extern "C" sp_status sp_transform_backward_static(const double* coef_dev, double* grid_dev, int nfields, int n_x,
                                                  int n_z, int scale_num, int scale_den, void* cuda_stream,
                                                  char* errbuf, int errlen) {
  char msg[256];
  if (!coef_dev || !grid_dev) return report(errbuf, errlen, SP_ERR_ARG, "null input or output pointer");
  if (nfields < 1 || nfields > STATIC_MAX_FIELDS) {
    std::snprintf(msg, sizeof msg, "nfields = %d outside [1, %d]", nfields, STATIC_MAX_FIELDS);
    return report(errbuf, errlen, SP_ERR_ARG, msg);
  }
  if (n_x < 4 || n_x % 2 || n_z < 4 || scale_num < scale_den || scale_den < 1 ||
      (n_x * scale_num) % scale_den || (n_z * scale_num) % scale_den)
    return report(errbuf, errlen, SP_ERR_ARG, "sizes must be even N_x >= 4, N_z >= 4, integer grids, scale >= 1");
  const int ngx = n_x * scale_num / scale_den, ngz = n_z * scale_num / scale_den;
  if (!smooth(ngx) || !smooth(ngz) || ngx < 8 || ngz < 8 || ngx > STATIC_MAX_NGX || ngz > STATIC_MAX_NGZ) {
    std::snprintf(msg, sizeof msg, "grid %d x %d: each side must be 2^k or 3*2^k, 8 <= N_gx <= %d, N_gz <= %d",
                  ngx, ngz, STATIC_MAX_NGX, STATIC_MAX_NGZ);
    return report(errbuf, errlen, SP_ERR_ARG, msg);
  }
  const int P = n_x / 2;
  const size_t need = (size_t)nfields * ngz * P;
  if (need > STATIC_SCRATCH_COMPLEX) {
    std::snprintf(msg, sizeof msg,
                  "needs %zu complex intermediate values (nfields * N_gz * N_x/2); the static buffer holds %zu",
                  need, STATIC_SCRATCH_COMPLEX);
    return report(errbuf, errlen, SP_ERR_ARG, msg);
  }
  // the x-row kernel keeps a whole grid row of every field in shared memory
  // (227 KiB per CTA), which bounds N_gx jointly with nfields
  const size_t xsm = x_smem_bytes(0, ngx, 1, nfields, 0);
  const size_t zsm = z_smem_bytes(0, ngz, 4);
  if (xsm > 227 * 1024 || zsm > 227 * 1024) {
    std::snprintf(msg, sizeof msg,
                  "%d fields at N_gx = %d, N_gz = %d need %zu B (x rows) / %zu B (z columns) of shared memory "
                  "per block; the limit is %d B",
                  nfields, ngx, ngz, xsm, zsm, 227 * 1024);
    return report(errbuf, errlen, SP_ERR_ARG, msg);
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= STATIC_MAX_DEVICES)
    return report(errbuf, errlen, SP_ERR_CUDA, "no current CUDA device");
  StaticAddrs& A = g_static[dev];
  // one-time set-up on this device: device addresses of the static arrays
  std::call_once(A.once, [&A]() {
    cudaError_t e = cudaGetSymbolAddress((void**)&A.scratch, s_scratch);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&A.tw_x, s_tw_x);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&A.tw_z, s_tw_z);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&A.dct_z, s_dct_z);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&A.field_index, s_field_index);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&A.field_op, s_field_op);
    A.setup = e;
  });
  if (A.setup != cudaSuccess) {
    std::snprintf(msg, sizeof msg, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(A.setup));
    return report(errbuf, errlen, SP_ERR_CUDA, msg);
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  TransformPlan pz, px;
  pz.Nc = n_z; pz.Ng = ngz; pz.radix3 = (ngz % 3 == 0); pz.tw64 = A.tw_z; pz.dct64 = A.dct_z;
  px.Nc = n_x; px.Ng = ngx; px.radix3 = (ngx % 3 == 0); px.tw64 = A.tw_x;
  k_static_twiddles<<<(ngz + 255) / 256, 256, 0, s>>>(A.tw_z, ngz, A.dct_z);
  k_static_twiddles<<<(ngx + 255) / 256, 256, 0, s>>>(A.tw_x, ngx, nullptr);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = launch_cheb_backward(s, 0, pz, P, nfields, A.field_index, A.field_op, nullptr,
                             reinterpret_cast<const double2*>(coef_dev), P * n_z, A.scratch);
  if (e == cudaSuccess)
    e = launch_fourier_rows(s, 0, px, ngz, P, 1, nfields, A.scratch, nullptr, grid_dev, 0, nullptr, nullptr,
                            nullptr, nullptr, 0, nullptr);
  if (e != cudaSuccess) {
    std::snprintf(msg, sizeof msg, "launch failed: %s", cudaGetErrorString(e));
    return report(errbuf, errlen, SP_ERR_CUDA, msg);
  }
  return report(errbuf, errlen, SP_OK, "");
}
