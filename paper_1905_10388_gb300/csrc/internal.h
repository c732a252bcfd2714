// Internal declarations shared by the spectau translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <vector>

#include "common.cuh"

namespace spectau {

// Column chunk streamed per bulk copy by the pencil-solve kernel, and the
// ring depth.  Factor arrays are padded to a multiple of SOLVE_CHUNK columns.
constexpr int SOLVE_CHUNK = 32;
constexpr int SOLVE_RING = 2;

// Banded LU factors of one matrix a*M~ + b*L~ for all pencils.
struct BandFactor {
  double alpha = 0, beta = 0;   // A = alpha M~ + beta L~
  double* L = nullptr;          // [P][npad][lpad]  multipliers of column j (rows j+1..j+kl)
  uint8_t* piv = nullptr;       // [P][npad]        pivot row offset (piv - j) in [0, kl]
  double* U = nullptr;          // [P][npad][upad]  t=0: 1/U_jj, t>=1: U_{j-t,j}/U_jj
  double* rd = nullptr;         // [P][npad]        1/U_jj (0 on padding columns)
  // lane-interleaved copies for k_pencil_lanes (groups of LANE_GROUP pencils):
  double* Lg = nullptr;         // [G][n][kl][16]
  double* Ug = nullptr;         // [G][n][cmax][16]  the listed U entries of column j (k = 0: 1/U_jj)
  int cmax = 0;                 // most entries listed for one column
  double u_listed = 0;          // mean listed entries per column, the diagonal excluded
  uint8_t* pg = nullptr;        // [G][n][16]
  unsigned long long* umask = nullptr;   // [n] bit t: U_{j-t,j} != 0 in some pencil (bit 0 set)
  // partitioned substitution (spike.cu): coupling matrices of the row blocks
  double* spD = nullptr;        // [P][nblk_f][7][8]   forward window after a block from the window before
  double* spE = nullptr;        // [P][nblk][kuu][32]  back-substitution outflow from the inflow
};

// Partitioned substitution of problems with few pencils (spike.cu).
struct SpikeArgs {
  int P, n, npad, kl, kuu, lpad, upad;
  int nblk, m;                  // back-substitution blocks per pencil and their rows
  int nblk_f, m_f;              // forward-substitution blocks and rows (multiples of 8)
  const double* L; const uint8_t* piv; const double* U; const double* rd;
  const double* D; const double* E;
  const double2* bg;            // B~ [p][n]
  double2* yg;                  // y = L^-1 P B~ [p][n]
  double2* xg;                  // x~ = y / U_jj [p][n] (the epilogue's input)
  double* s0; double* sst;      // forward outflows / inflows [p][nblk_f][2][8]
  double* o0; double* uin;      // backward outflows / inflows [p][nblk][2][32]
  DevStatus* status;
};
// Problems with fewer pencils than this (and kl <= 7, kl + ku <= 31, at
// least SPIKE_MIN_ROWS rows) use the partitioned substitution by default.
constexpr int SPIKE_MAX_PENCILS = 608;
constexpr int SPIKE_MIN_ROWS = 512;
bool spike_supported(int kl, int kuu, int npad, int nblk);
bool spike_bwd_supported(int kuu, int npad, int nblk);
cudaError_t launch_spike_coupling_bwd(cudaStream_t s, int P, int npad, int nblk, int kuu, int upad, const double* U,
                                      double* E);
cudaError_t launch_spike_backward(cudaStream_t st, const SpikeArgs& s);
cudaError_t launch_spike_coupling(cudaStream_t s, int P, int npad, int nblk_f, int nblk, int kl, int kuu, int lpad,
                                  int upad, const BandFactor& f);
// forward blocks of the partitioned substitution: 128 rows, or 64 or 32 when
// those divide the padded rows
inline int spike_forward_blocks(int npad) {
  for (int m = 128; m >= 32; m /= 2)
    if (npad % m == 0) return npad / m;
  return 1;
}
cudaError_t launch_spike_solve(cudaStream_t s, const SpikeArgs& a);

// Pencils per warp in the lane-per-pencil substitution (two lanes each:
// real and imaginary part).
constexpr int LANE_GROUP = 16;
// Problems with at least this many pencils use the lane-per-pencil
// substitution (2 P lanes = P / 16 warps: several per SM).
constexpr int LANE_MIN_PENCILS = 4096;

// Chebyshev backward transform on the tensor cores (chebmma.cu): the split
// FP32 copy of the coefficients it reads, the transform matrix halves, and
// the TMA tensor maps (opaque CUtensorMap storage, 64-byte aligned).
struct ChebMMA {
  bool ready = false;
  int P = 0, Nz = 0, Ng = 0, S = 0;
  float* xs32 = nullptr;        // [S][2P][Nz]: real part (column 2p) and imaginary part (2p + 1)
  float* Thi = nullptr;         // [Ng][Nz] T_m(x_zg) truncated to TF32
  float* Tlo = nullptr;         // [Ng][Nz] the FP32 remainder
  alignas(64) unsigned char tmA[128];
  alignas(64) unsigned char tmThi[128];
  alignas(64) unsigned char tmTlo[128];
};
bool cheb_mma_supported(int Nz, int Ng);
cudaError_t cheb_mma_setup(ChebMMA& c, int P, int Nz, int Ng, int S, cudaStream_t s);
void cheb_mma_free(ChebMMA& c);
// grid fields f (variable f_var[f], operator f_op[f]; host arrays) of the
// FP32 coefficients in c.xs32 to gz [f][Ng][P] complex FP32
cudaError_t launch_cheb_backward_mma(cudaStream_t s, const ChebMMA& c, int nf, const int* f_var, const int* f_op,
                                     const float* kx32, void* gz, DevStatus* st);
cudaError_t launch_to_f32_split(cudaStream_t s, const double2* src, float* dst, size_t ncols, int Nz);

// Up to four device vectors with coefficients, passed to kernels by value.
struct VecList4 {
  const double2* p[4];
  double c[4];
  int n;
};

// Adjoint-step helper kernels (band.cu).
cudaError_t launch_adj_gather(cudaStream_t s, int P, int Nz, int Ng, int n, int nslot, const int32_t* nl_eq,
                              const int32_t* row_map, const int32_t* eq_diff, const int32_t* eq_phase,
                              int nvec, const double2* const* vecs, const double* coefs, double2* fbar,
                              float2* fbar32);
cudaError_t launch_adj_combine(cudaStream_t s, int P, int Nz, int S, int n, int nf, const int32_t* f_var,
                               const int32_t* f_op, const double* kx, const double2* xbar,
                               const int32_t* col_map, const int32_t* var_rec, const int32_t* var_phase,
                               int nadd, const double2* const* adds, const double* add_coefs, double2* out);
cudaError_t launch_adj_tinvh(cudaStream_t s, int P, int Nz, int S, int n, const double2* xt_bar,
                             const int32_t* col_map, const int32_t* var_rec, const int32_t* var_phase,
                             double2* out);
cudaError_t launch_dz_adjoint(cudaStream_t s, int P, int Nz, double scale, const double2* dst_bar,
                              double2* src_bar);

// Stored vectors and right-hand sides one stage combines: RK443's fourth
// stage takes M~X~^0 and three L~X~^j, and four F~^j.
constexpr int SP_MAX_TERMS = 4;

// Arguments of the pencil right-hand-side assembly + solve + epilogue kernel.
struct SolveArgs {
  int P, n, Nz, S, nbc, nnz;
  int kl, kuu, npad, lpad, upad;
  const double* Lf; const uint8_t* piv; const double* Uf; const double* rd;
  // prologue: B = sum_k vec_coef[k] vec[k] + mv_coef (Mat x) + sum_k fc_coef[k] P^L Fc_k + bc_coef g
  int nvec; const double2* vec[SP_MAX_TERMS]; double vec_coef[SP_MAX_TERMS];
  const double2* mv_x; const double* mv_vals; double mv_coef; double2* mv_store;
  const int32_t* mv_indptr; const int32_t* mv_indices; int mv_nnz;   // pattern of mv_vals
  // + mv2_coef (Mat2 x) on the same x (null mv2_vals: none)
  const double* mv2_vals; double mv2_coef;
  const int32_t* mv2_indptr; const int32_t* mv2_indices; int mv2_nnz;
  int nfc; const double2* fc[SP_MAX_TERMS]; double fc_coef[SP_MAX_TERMS];
  // fc_coef / 2 and -fc_coef / 2 for the T-to-U rows, filled by the launcher
  double fc_half[SP_MAX_TERMS], fc_mhalf[SP_MAX_TERMS];
  double bc_coef;
  // epilogue
  double2* xt_out; double2* xc_out; float2* xc32_out;   // xc32_out: FP32 copy (mixed precision)
  float* xs32_out;                             // split FP32 copy [var][2p + c][m] (tensor-core z transform)
  const double* ep_mv_vals; double2* ep_mv_store;
  // epilogue (mode 2): store (B~ - ep_alpha M~X~) ep_from_b, i.e. L~X~ from the
  // stage's own right-hand side, when ep_from_b != 0 (mixed precision only)
  double ep_from_b, ep_alpha;
  const double2* ep_mv_addvec;                 // epilogue matvec acts on (X~ + addvec) if set
  const int32_t* ep_indptr; const int32_t* ep_indices; int ep_nnz;    // pattern of ep_mv_vals
  const int32_t* ep_rows; int ep_nrows;   // the pattern's non-empty rows (M~), or null: every row
  // tables (device)
  const int32_t* indptr; const int32_t* indices;
  const int32_t* row_map; const int32_t* col_map;
  const int32_t* var_recombine; const int32_t* var_phase;
  const int32_t* eq_differential; const int32_t* eq_phase;
  const int32_t* nl_eq; int n_nl;        // equation index of each nonlinear slot
  const int32_t* bc_rows; const double2* bc_values;
  DevStatus* status;
  // mode 0: assembly, substitution and epilogue in one kernel; 1: assembly
  // only, B~ to bg [p][n]; 2: epilogue only, from xg [p][n] (x~ = y / U_jj)
  // (the substitution then runs in k_pencil_lanes or the partitioned
  // kernels); 3: assembly and forward substitution, y = L^-1 P B~ to yg
  // [p][n] (the partitioned back substitution follows)
  int mode;
  double2* bg; const double2* xg; double2* yg;
  // 1: with kl <= 15, one warp runs both parts' forward substitution in two
  // 16-lane windows (half the FP64 issue; the batched solve, bound by the
  // FP64 pipe, sets it; a lone problem's whole-row chains are bound by their
  // latency and keep a 32-lane window per part)
  int fwd16;
  // factor in the lane-interleaved layout (null: not available)
  const double* Lg; const double* Ug; const uint8_t* pg; const unsigned long long* umask; int cmax;
  // coupling matrices of the partitioned substitution (null: not available)
  const double* spD; const double* spE;
};

// fc_half / fc_mhalf from fc_coef (exact scalings), before a launch
inline void fill_f_halves(SolveArgs& a) {
  for (int k = 0; k < SP_MAX_TERMS; ++k) {
    a.fc_half[k] = 0.5 * a.fc_coef[k];
    a.fc_mhalf[k] = -0.5 * a.fc_coef[k];
  }
}

// Transform arguments.
struct GridField { int var; int op; };

struct TransformPlan {
  int Nc, Ng;                   // coefficients and grid points along one axis
  int radix3;
  void* tw64 = nullptr;         // double2[Ng]  exp(-2 pi i t / Ng)
  void* tw32 = nullptr;         // float2[Ng]
  void* dct64 = nullptr;        // double2[Ng]  exp(-i pi k / (2 Ng))
  void* dct32 = nullptr;
};

// Per-problem descriptors of the transform kernels (tw / wq / gz / h are
// typed by the precision of the launch).
struct ZDesc {
  int Nc, Ng, radix3, P;
  const void* tw; const void* wq;
  // backward
  const int32_t* f_var; const int32_t* f_op; const double* kx; const double2* xc; int xc_stride; void* gz;
  const float* kx32; const float2* xc32;     // FP32 copies (mixed precision)
  // forward
  const void* h; double2* fc;
  int unweighted;                            // 1: transpose of the backward transform
  int weighted_in;                           // 1: transpose of the forward transform
};
struct XDesc {
  int N, radix3, rows, K, mode, nf;
  const void* tw;
  const void* gz; const double* grid_in; double* grid_out;
  int nterms; const int32_t* t_eq; const double* t_coef; const int32_t* t_fa; const int32_t* t_fb;
  int ne; void* h;
  const float* t_coef32;
  const void* hin; void* gzadj;             // adjoint rows: inputs / outputs
  int xscale;                                // bit 1: transpose of forward x on input; bit 2: of backward x on output
  int pairs;                                 // field pairs per backward FFT round (0: two)
};

// Complex Fourier y transform of nf x nz planes of N_y slots x K columns.
struct YDesc {
  int Ny, Ng, K, nz, radix3, dir;
  const void* tw;
  const void* src; void* dst;
};

// --- launchers (band.cu) ---------------------------------------------------
cudaError_t launch_band_factor(cudaStream_t s, int P, int n, int nnz, int kl, int ku,
                               const int32_t* indptr, const int32_t* indices,
                               const double* Mv, const double* Lv, double alpha, double beta,
                               double* work, const BandFactor& f, int npad, int lpad, int upad,
                               DevStatus* st);
cudaError_t launch_pencil_solve(cudaStream_t s, const SolveArgs& a);
cudaError_t launch_eig_update(cudaStream_t s, int P, int n, double2* x, const double2* y, double2* mu);
cudaError_t launch_eig_residual(cudaStream_t s, int P, int n, int nnz, const int32_t* indptr, const int32_t* indices,
                                const double* Mv, const double* Lv, const double2* x, const double2* sig,
                                double* res);
size_t pencil_solve_smem(int npad, int lpad, int upad);
// batched pencil solves: one CTA per (problem, pencil) work item
cudaError_t launch_pencil_solve_batched(cudaStream_t s, const SolveArgs* args, const int4* work, int nwork,
                                        int max_kuu, size_t smem);
// Lane-per-pencil substitution (many-pencil problems): forward and back
// substitution of P pencils, B~ [p][n] in, x~ = y / U_jj [p][n] out, y scratch
// [G][n][16] complex.  Returns cudaErrorInvalidValue when (kl, kl + ku) has
// no compiled instance (lanes_supported).
bool lanes_supported(int kl, int kuu);
cudaError_t launch_pencil_lanes(cudaStream_t s, int P, int n, int kl, int kuu, const double* Lg, const double* Uc,
                                int cmax, const uint8_t* pg, const unsigned long long* umask, const double2* b,
                                double2* y, double2* x);
// umask[j] |= bit t for every t <= kuu with U_{j-t,j} != 0 in some pencil
// (umask zeroed by the caller)
cudaError_t launch_u_mask(cudaStream_t s, int P, int n, int npad, int kuu, int upad, const double* U,
                          unsigned long long* umask);
cudaError_t launch_factor_relayout(cudaStream_t s, int P, int n, int npad, int kl, int kuu, int lpad, int upad,
                                   const BandFactor& f);
cudaError_t launch_coef_to_solve(cudaStream_t s, int P, int S, int Nz, const double2* xc,
                                 double2* xt, const int32_t* col_map, const int32_t* var_recombine,
                                 const int32_t* var_phase);
cudaError_t launch_dz(cudaStream_t s, int P, int Nz, double scale, const double2* src, double2* dst);
cudaError_t launch_to_f32(cudaStream_t s, const double2* src, float2* dst, size_t n);

// --- launchers (transforms.cu) ---------------------------------------------
// precision: 0 = double, 1 = float.  Buffers of the grid stages are typed by
// the precision; coefficient-space inputs/outputs are always double2.
cudaError_t launch_cheb_backward(cudaStream_t s, int prec, const TransformPlan& pz, int P,
                                 int nf, const int32_t* f_var, const int32_t* f_op,
                                 const double* kx, const double2* xc, int xc_field_stride,
                                 void* gz, const float* kx32 = nullptr, const float2* xc32 = nullptr,
                                 int weighted_in = 0);
cudaError_t launch_fourier_rows(cudaStream_t s, int prec, const TransformPlan& px, int rows,
                                int P, int mode, int nf, const void* gz, double* grid_in,
                                double* grid_out, int nterms, const int32_t* t_eq,
                                const double* t_coef, const int32_t* t_fa, const int32_t* t_fb,
                                int ne, void* h, const float* t_coef32 = nullptr, int xscale = 0);
cudaError_t launch_cheb_forward(cudaStream_t s, int prec, const TransformPlan& pz, int P, int ne,
                                const void* h, double2* fc, int unweighted = 0);
cudaError_t launch_fourier_rows_adjoint(cudaStream_t s, int prec, const TransformPlan& px, int rows, int P,
                                        int nf, const void* gz, int ne, const void* hin, int nterms,
                                        const int32_t* t_eq, const double* t_coef, const float* t_coef32,
                                        const int32_t* t_fa, const int32_t* t_fb, void* gzadj);
// dir < 0: slots -> grid, dir > 0: grid -> slots (1/N_gy, Nyquist slot zero);
// py = plan (N_y, N_gy); buffers [f][zg][slot or yg][K] in the precision.
cudaError_t launch_cfl_max(cudaStream_t s, const double* grid, int nvel, const int* axes, int Ngx, int Ngy, int Ngz,
                           double inv_dx, double inv_dy, const double* inv_dz, unsigned long long* out);
cudaError_t launch_fourier_y(cudaStream_t s, int prec, const TransformPlan& py, int dir, int nf, int nz, int K,
                             const void* src, void* dst);
size_t z_smem_bytes(int prec, int Ng, int tile);
size_t x_smem_bytes(int prec, int N, int mode, int nf, int ne, int pairs = 0);
// batched transforms: queue null: one CTA per work item; else a persistent
// grid pulling items from the device counter *queue (zero before the launch)
cudaError_t launch_cheb_backward_batched(cudaStream_t s, int prec, int tile, const ZDesc* ds, const int4* work,
                                         int nwork, int max_ng, int* queue = nullptr);
cudaError_t launch_cheb_forward_batched(cudaStream_t s, int prec, int tile, const ZDesc* ds, const int4* work,
                                        int nwork, int max_ng, int* queue = nullptr);
cudaError_t launch_fourier_rows_batched(cudaStream_t s, int prec, const XDesc* ds, const int4* work, int nwork,
                                        size_t smem, int* queue = nullptr);

}  // namespace spectau
