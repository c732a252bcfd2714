// Host runtime behind the C ABI (include/spectau.h): problem objects,
// validation, device tables, transform plans, factor/step orchestration,
// CUDA-graph replay and launch timing.  No computation of the step happens
// on the host; every stage is one of the kernels in band.cu / transforms.cu.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <string>
#include <tuple>
#include <vector>

#include "internal.h"

using namespace spectau;

namespace {

// ARS(2,2,2) of Ascher, Ruuth & Spiteri (1997), and RK111 (IMEX Euler):
// implicit H and explicit A tableaux with an explicit first stage.
struct Tableau {
  int s;
  double H[5][5];
  double A[5][5];
};

Tableau make_tableau(int scheme) {
  Tableau t{};
  if (scheme == SP_RK222) {
    const double g = 1.0 - 1.0 / std::sqrt(2.0), d = 1.0 - 1.0 / (2.0 * g);
    t.s = 2;
    t.H[1][1] = g;
    t.H[2][1] = 1.0 - g;
    t.H[2][2] = g;
    t.A[1][0] = g;
    t.A[2][0] = d;
    t.A[2][1] = 1.0 - d;
  } else if (scheme == SP_RK443) {
    // ARS(4,4,3): implicit diagonal 1/2, c = (0, 1/2, 2/3, 1/2, 1)
    t.s = 4;
    t.H[1][1] = 0.5;
    t.H[2][1] = 1.0 / 6.0; t.H[2][2] = 0.5;
    t.H[3][1] = -0.5; t.H[3][2] = 0.5; t.H[3][3] = 0.5;
    t.H[4][1] = 1.5; t.H[4][2] = -1.5; t.H[4][3] = 0.5; t.H[4][4] = 0.5;
    t.A[1][0] = 0.5;
    t.A[2][0] = 11.0 / 18.0; t.A[2][1] = 1.0 / 18.0;
    t.A[3][0] = 5.0 / 6.0; t.A[3][1] = -5.0 / 6.0; t.A[3][2] = 0.5;
    t.A[4][0] = 0.25; t.A[4][1] = 1.75; t.A[4][2] = 0.75; t.A[4][3] = -1.75;
  } else {  // RK111
    t.s = 1;
    t.H[1][1] = 1.0;
    t.A[1][0] = 1.0;
  }
  return t;
}

bool is_rk(int scheme) { return scheme == SP_RK222 || scheme == SP_RK111 || scheme == SP_RK443; }

// order of a multistep scheme, SBDF or CNAB (0 for the Runge-Kutta schemes)
int sbdf_order(int scheme) {
  switch (scheme) {
    case SP_SBDF1: return 1;
    case SP_SBDF2: return 2;
    case SP_SBDF3: return 3;
    case SP_SBDF4: return 4;
    case SP_CNAB1: return 1;
    case SP_CNAB2: return 2;
    default: return 0;
  }
}
bool is_cnab(int scheme) { return scheme == SP_CNAB1 || scheme == SP_CNAB2; }
// history slots of a multistep scheme (two at least: SBDF1 alternates too)
int sbdf_depth(int scheme) { return std::max(2, sbdf_order(scheme)); }

// Constant-step SBDF of order q (Wang & Ruuth 2008) multiplied through by dt:
//   (a_0 M + dt L) X^{n+1} = - sum_{j=1..q} a_j M X^{n+1-j} + dt sum_{j=1..q} c_j F^{n+1-j}
// (BDF weights a, extrapolation weights c; both rows of c sum to one).
const double SBDF_A[5][5] = {{0, 0, 0, 0, 0},
                             {1.0, -1.0, 0, 0, 0},
                             {1.5, -2.0, 0.5, 0, 0},
                             {11.0 / 6.0, -3.0, 1.5, -1.0 / 3.0, 0},
                             {25.0 / 12.0, -4.0, 3.0, -4.0 / 3.0, 0.25}};
const double SBDF_C[5][5] = {{0, 0, 0, 0, 0},
                             {0, 1.0, 0, 0, 0},
                             {0, 2.0, -1.0, 0, 0},
                             {0, 3.0, -3.0, 1.0, 0},
                             {0, 4.0, -6.0, 4.0, -1.0}};
// Constant-step CNAB1 / CNAB2 (Wang & Ruuth 2008) multiplied through by dt:
//   (M + dt/2 L) X^{n+1} = (M - dt/2 L) X^n + dt sum_{j=1..q} c_j F^{n+1-j}
// (trapezoidal implicit part, Adams-Bashforth weights c)
const double CNAB_C[3][3] = {{0, 0, 0}, {0, 1.0, 0}, {0, 1.5, -0.5}};

bool is_smooth_length(int N) {  // 2^k or 3 * 2^k
  if (N <= 0) return false;
  if (N % 3 == 0) N /= 3;
  return (N & (N - 1)) == 0;
}

template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
};

}  // namespace

struct Problem {
  int ndim = 2, S = 0, scheme = 0, prec = 0;
  sp_basis bx{}, by{}, bz{};
  int Nx = 0, Nz = 0, P = 0, Ngx = 0, Ngz = 0;
  int Ny = 1, Ngy = 1, K = 0;     // y axis (3D; 1 on 2D problems), K = N_x / 2 x modes per pencil row
  double Lx = 0, Ly = 0, za = 0, zb = 1;
  // layout
  bool has_layout = false;
  std::vector<int32_t> col_map, row_map, var_rec, var_ph, eq_diff, eq_ph, bc_rows;
  int nbc = 0;
  std::vector<double> bc_values;
  // pencils
  int n = 0;
  int64_t nnz = -1;
  std::vector<int32_t> indptr, indices;
  std::vector<double> Mv, Lv;
  std::vector<uint8_t> pset;
  int kl = 0, ku = 0;
  // bilinear rhs
  std::vector<int32_t> t_slot, t_fa, t_fb;
  std::vector<double> t_coef;
  std::vector<GridField> gfields;
  std::vector<int32_t> nl_eqs;
  // device
  bool uploaded = false;
  int32_t *d_indptr = nullptr, *d_indices = nullptr;
  double *d_Mv = nullptr, *d_Lv = nullptr;
  // M~ on its own compact pattern (entries nonzero in at least one pencil)
  int64_t nnzM = 0;
  int32_t *d_indptrM = nullptr, *d_indicesM = nullptr;
  int32_t* d_mrows = nullptr;   // rows of M~ with entries
  int nmrows = 0;
  double* d_MvC = nullptr;
  int32_t *d_col_map = nullptr, *d_row_map = nullptr, *d_var_rec = nullptr, *d_var_ph = nullptr;
  int32_t *d_eq_diff = nullptr, *d_eq_ph = nullptr, *d_bc_rows = nullptr, *d_nl_eq = nullptr;
  double2* d_bc_values = nullptr;
  double* d_kx = nullptr;
  int32_t *d_gvar = nullptr, *d_gop = nullptr, *d_tslot = nullptr, *d_tfa = nullptr, *d_tfb = nullptr;
  double* d_tcoef = nullptr;
  int32_t *d_ident = nullptr, *d_zero = nullptr;
  double2 *d_Xt = nullptr, *d_Xc = nullptr;
  float2* d_Xc32 = nullptr;        // FP32 copy of the T coefficients (mixed precision)
  float* d_kx32 = nullptr;
  float* d_tcoef32 = nullptr;
  bool xc32_valid = false;
  // Chebyshev backward transform on the tensor cores (mixed precision)
  int zkind = SP_ZT_AUTO;
  bool zmma = false;
  bool xs32_valid = false;
  ChebMMA cm;
  // linear boundary value solve: L~ factored in the first slot, its
  // right-hand-side slots [slot][P][Nz] and their equations
  bool lbvp_factored = false;
  // the last eigensolve's vectors (solve variables, [P][n]) and eigenvalues
  double2 *d_eigx = nullptr, *d_eigsig = nullptr;
  double2* d_lb_F = nullptr;
  int32_t* d_lb_eq = nullptr;
  int lb_cap = 0;
  // CFL frequency scratch (sp_cfl_frequency), allocated on first use
  double* d_cfl_grid = nullptr;
  void *d_cfl_mid1 = nullptr, *d_cfl_mid2 = nullptr;
  double* d_inv_dz = nullptr;
  int32_t* d_cfl_args = nullptr;             // vars[3], axes[3]
  unsigned long long* d_cfl_out = nullptr;
  int cfl_cap = 0;                           // fields the scratch holds
  double2* d_MX[4] = {nullptr, nullptr, nullptr, nullptr};   // M~X~ history (multistep: a ring)
  double2* d_LX[4] = {nullptr, nullptr, nullptr, nullptr};   // L~X~^j, j = 1 .. s - 1
  double2* d_Fc[4] = {nullptr, nullptr, nullptr, nullptr};   // F~ slots (RK: F^j, j < s)
  void* d_gz = nullptr;
  void* d_gy = nullptr;            // 3D: y-transformed fields [f][zg][yg][i_x]
  void* d_h = nullptr;
  BandFactor fac[4];                       // SBDFq: one per start-up order 1 .. q
  int nfac = 0;
  double fac_dt = 0;
  bool factored = false;
  int npad = 0, lpad = 0, upad = 0;
  // lane-per-pencil substitution (many pencils): its B~ / x~ / y buffers
  bool lanes = false;
  int solve_kind = SP_SOLVE_AUTO;
  double2 *d_bg = nullptr, *d_xg = nullptr, *d_yg = nullptr;
  // partitioned substitution (few pencils): blocks per pencil and the
  // inflow/outflow vectors of the blocks
  bool spike = false;
  int spike_blocks = 0;                      // requested (0: automatic)
  int nblk = 0, nblk_f = 0;
  double *d_sp_s0 = nullptr, *d_sp_s = nullptr, *d_sp_o0 = nullptr, *d_sp_u = nullptr;
  double* d_spT_u = nullptr;                 // inflow guesses of the transposed solves
  std::map<std::pair<int, int>, TransformPlan> plans;
  // stepping state
  int iteration = 0;
  bool xt_valid = false, mx_valid = false;
  // adjoint: factor of the transposed pencils and work buffers
  bool adj_ready = false;
  BandFactor facT;
  int klT = 0, kuT = 0, lpadT = 0;
  int32_t *d_indptrT = nullptr, *d_indicesT = nullptr;
  double *d_MvT = nullptr, *d_LvT = nullptr;
  double2 *d_mu[2] = {nullptr, nullptr}, *d_LTmu = nullptr, *d_MTmu = nullptr, *d_JF = nullptr, *d_lamx = nullptr;
  double2 *d_Xbar = nullptr, *d_Fbar = nullptr;
  float2* d_Fbar32 = nullptr;
  void* d_gzadj = nullptr;
  // graphs
  std::map<std::tuple<int, int, int, double>, cudaGraphExec_t> graphs;
  // timing
  bool timing = false;
  std::vector<cudaEvent_t> ev;
  size_t ev_used = 0;
};

struct Batch;
struct sp_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t capture = nullptr;
  std::string err;
  std::vector<std::unique_ptr<Problem>> probs;
  DevStatus* d_status = nullptr;
  // batches keyed by (problem ids, schedule phase); tile chosen per ids
  std::map<std::pair<std::vector<int>, int>, Batch*> batches;
  std::map<std::vector<int>, int> batch_tile;
  std::map<std::vector<int>, bool> batch_persist;
  std::map<std::vector<int>, bool> batch_persist_fixed;   // shapes set by sp_set_batch_persistent
};

namespace {

sp_status fail(sp_ctx* c, sp_status code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

#define CK(call)                                                                              \
  do {                                                                                        \
    cudaError_t e_ = (call);                                                                  \
    if (e_ != cudaSuccess)                                                                    \
      return fail(ctx, e_ == cudaErrorMemoryAllocation ? SP_ERR_OOM : SP_ERR_CUDA, "%s: %s (%s:%d)", \
                  #call, cudaGetErrorString(e_), __FILE__, __LINE__);                        \
  } while (0)

template <typename T>
cudaError_t dalloc(T** p, size_t count) {
  return cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T));
}

template <typename T>
cudaError_t upload(T** p, const std::vector<T>& v, cudaStream_t s) {
  cudaError_t e = dalloc(p, v.size());
  if (e != cudaSuccess) return e;
  if (v.empty()) return cudaSuccess;
  e = cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

Problem* get(sp_ctx* ctx, int id) {
  if (!ctx || id < 0 || id >= (int)ctx->probs.size()) return nullptr;
  return ctx->probs[id].get();
}

// exp(-2 pi i t / N) and exp(-i pi k / (2N)) from libm in FP64
sp_status make_plan(sp_ctx* ctx, Problem* pr, int Nc, int Ng, TransformPlan** out) {
  auto key = std::make_pair(Nc, Ng);
  auto it = pr->plans.find(key);
  if (it != pr->plans.end()) {
    *out = &it->second;
    return SP_OK;
  }
  if (!is_smooth_length(Ng) || Ng < 4 || Ng % 2) return fail(ctx, SP_ERR_ARG, "unsupported grid size %d", Ng);
  TransformPlan pl;
  pl.Nc = Nc;
  pl.Ng = Ng;
  pl.radix3 = (Ng % 3 == 0);
  std::vector<double2> tw(Ng), dq(Ng);
  std::vector<float2> tw32(Ng), dq32(Ng);
  const double pi = 3.14159265358979323846;
  for (int t = 0; t < Ng; ++t) {
    tw[t] = make_double2(std::cos(2.0 * pi * t / Ng), -std::sin(2.0 * pi * t / Ng));
    dq[t] = make_double2(std::cos(pi * t / (2.0 * Ng)), -std::sin(pi * t / (2.0 * Ng)));
    tw32[t] = make_float2((float)tw[t].x, (float)tw[t].y);
    dq32[t] = make_float2((float)dq[t].x, (float)dq[t].y);
  }
  double2 *a, *b;
  float2 *c, *d;
  CK(upload(&a, tw, ctx->stream));
  CK(upload(&b, dq, ctx->stream));
  CK(upload(&c, tw32, ctx->stream));
  CK(upload(&d, dq32, ctx->stream));
  pl.tw64 = a;
  pl.dct64 = b;
  pl.tw32 = c;
  pl.dct32 = d;
  pr->plans[key] = pl;
  *out = &pr->plans[key];
  return SP_OK;
}

// the partitioned back substitution starts its blocks from the previous
// solve's inflows (spike.cu); zero them, the transposed solves' too, so that
// a run (or a gradient) from a set state repeats bit for bit
cudaError_t reset_spike_guess(Problem* pr, cudaStream_t s) {
  if (!pr->spike) return cudaSuccess;
  const size_t bytes = (size_t)pr->P * pr->nblk * 2 * 32 * sizeof(double);
  cudaError_t e = cudaSuccess;
  if (pr->d_sp_u) e = cudaMemsetAsync(pr->d_sp_u, 0, bytes, s);
  if (e == cudaSuccess && pr->d_spT_u) e = cudaMemsetAsync(pr->d_spT_u, 0, bytes, s);
  return e;
}

// Blocks per pencil of the partitioned back substitution: about 1024 / P
// (two to four chains per GPU sub-partition with its two parts; measured at
// 256 pencils of 1792 rows: 4 blocks 0.224 ms per solve, 7 blocks 0.254, 14
// blocks 0.253, 28 blocks 0.274, whole pencils 0.289), each a whole number of
// 32-row chunks and at least 64 rows.
int default_spike_blocks(int npad, int P) {
  const int nch = npad / SOLVE_CHUNK;
  const int target = std::max(2, (1024 + std::max(P, 1) - 1) / std::max(P, 1));
  int best = 1;
  for (int nb = 2; nb <= nch / 2; ++nb)
    if (nch % nb == 0 && std::abs(nb - target) < std::abs(best - target)) best = nb;
  return best;
}

sp_status upload_problem(sp_ctx* ctx, Problem* pr) {
  if (pr->uploaded) return SP_OK;
  if (!pr->has_layout) return fail(ctx, SP_ERR_STATE, "sp_set_layout has not been called");
  if (pr->nnz < 0) return fail(ctx, SP_ERR_STATE, "sp_set_pencils has not been called");
  for (int p = 0; p < pr->P; ++p)
    if (!pr->pset[p]) return fail(ctx, SP_ERR_STATE, "pencil %d has no matrices", p);
  cudaStream_t s = ctx->stream;
  CK(upload(&pr->d_indptr, pr->indptr, s));
  CK(upload(&pr->d_indices, pr->indices, s));
  CK(upload(&pr->d_Mv, pr->Mv, s));
  CK(upload(&pr->d_Lv, pr->Lv, s));
  {
    std::vector<char> keep(pr->nnz, 0);
    for (int p = 0; p < pr->P; ++p)
      for (int64_t e = 0; e < pr->nnz; ++e)
        if (pr->Mv[(size_t)p * pr->nnz + e] != 0.0) keep[e] = 1;
    std::vector<int32_t> ip(pr->n + 1, 0), ix;
    std::vector<int64_t> src;
    for (int r = 0; r < pr->n; ++r) {
      for (int e = pr->indptr[r]; e < pr->indptr[r + 1]; ++e)
        if (keep[e]) { ix.push_back(pr->indices[e]); src.push_back(e); }
      ip[r + 1] = (int32_t)ix.size();
    }
    pr->nnzM = (int64_t)ix.size();
    std::vector<double> mv((size_t)pr->P * std::max<int64_t>(pr->nnzM, 1), 0.0);
    for (int p = 0; p < pr->P; ++p)
      for (int64_t k = 0; k < pr->nnzM; ++k) mv[(size_t)p * pr->nnzM + k] = pr->Mv[(size_t)p * pr->nnz + src[k]];
    CK(upload(&pr->d_indptrM, ip, s));
    CK(upload(&pr->d_indicesM, ix, s));
    std::vector<int32_t> mrows;
    for (int r = 0; r < pr->n; ++r)
      if (ip[r + 1] > ip[r]) mrows.push_back(r);
    pr->nmrows = (int)mrows.size();
    if (mrows.empty()) mrows.push_back(0);
    CK(upload(&pr->d_mrows, mrows, s));
    CK(upload(&pr->d_MvC, mv, s));
  }
  CK(upload(&pr->d_col_map, pr->col_map, s));
  CK(upload(&pr->d_row_map, pr->row_map, s));
  CK(upload(&pr->d_var_rec, pr->var_rec, s));
  CK(upload(&pr->d_var_ph, pr->var_ph, s));
  CK(upload(&pr->d_eq_diff, pr->eq_diff, s));
  CK(upload(&pr->d_eq_ph, pr->eq_ph, s));
  CK(upload(&pr->d_bc_rows, pr->bc_rows, s));
  std::vector<double2> bcv(pr->bc_values.size() / 2);
  for (size_t i = 0; i < bcv.size(); ++i) bcv[i] = make_double2(pr->bc_values[2 * i], pr->bc_values[2 * i + 1]);
  CK(upload(&pr->d_bc_values, bcv, s));
  // k_x of every pencil, then k_y (zero in 2D); y slots in FFT order
  std::vector<double> kx(2 * (size_t)pr->P, 0.0);
  const double twopi = 2.0 * 3.14159265358979323846;
  for (int p = 0; p < pr->P; ++p) {
    const int ix = p % pr->K, iy = p / pr->K;
    kx[p] = twopi * ix / pr->Lx;
    if (pr->ndim == 3) kx[pr->P + p] = twopi * (iy < pr->Ny / 2 ? iy : iy - pr->Ny) / pr->Ly;
  }
  CK(upload(&pr->d_kx, kx, s));
  std::vector<int32_t> gv, go;
  for (auto& g : pr->gfields) { gv.push_back(g.var); go.push_back(g.op); }
  CK(upload(&pr->d_gvar, gv, s));
  CK(upload(&pr->d_gop, go, s));
  CK(upload(&pr->d_tslot, pr->t_slot, s));
  CK(upload(&pr->d_tfa, pr->t_fa, s));
  CK(upload(&pr->d_tfb, pr->t_fb, s));
  CK(upload(&pr->d_tcoef, pr->t_coef, s));
  CK(upload(&pr->d_nl_eq, pr->nl_eqs, s));
  std::vector<int32_t> ident(64), zero(64, 0);
  for (int i = 0; i < 64; ++i) ident[i] = i;
  CK(upload(&pr->d_ident, ident, s));
  CK(upload(&pr->d_zero, zero, s));
  const size_t nvec = (size_t)pr->P * pr->n;
  CK(dalloc(&pr->d_Xt, nvec));
  CK(dalloc(&pr->d_Xc, nvec));
  if (pr->prec) {
    CK(dalloc(&pr->d_Xc32, nvec));
    std::vector<float> kx32(kx.begin(), kx.end()), tc32(pr->t_coef.begin(), pr->t_coef.end());
    CK(upload(&pr->d_kx32, kx32, s));
    CK(upload(&pr->d_tcoef32, tc32, s));
  }
  CK(cudaMemsetAsync(pr->d_Xc, 0, nvec * sizeof(double2), s));
  for (int j = 0; j < sbdf_depth(pr->scheme); ++j) CK(dalloc(&pr->d_MX[j], nvec));
  // RK443 keeps three L~X~^j and four F~^j; the other schemes two and three
  const int nlx = pr->scheme == SP_RK443 ? 4 : 3;
  const int nfc = (pr->scheme == SP_RK443 || pr->scheme == SP_SBDF4) ? 4 : 3;
  for (int j = 0; j < nlx; ++j) CK(dalloc(&pr->d_LX[j], nvec));
  const int nl = std::max<int>(1, (int)pr->nl_eqs.size());
  for (int j = 0; j < nfc; ++j) CK(dalloc(&pr->d_Fc[j], (size_t)nl * pr->P * pr->Nz));
  const size_t esz = pr->prec ? sizeof(float2) : sizeof(double2);
  const int nf = std::max<int>(1, (int)pr->gfields.size());
  const size_t rows = (size_t)pr->Ngz * pr->Ngy;   // x rows of the dealiased grid
  CK(cudaMalloc(&pr->d_gz, (size_t)std::max(nf, nl) * pr->Ngz * pr->P * esz));
  CK(cudaMalloc(&pr->d_h, (size_t)nl * rows * pr->K * esz));
  if (pr->ndim == 3) CK(cudaMalloc(&pr->d_gy, (size_t)nf * rows * pr->K * esz));
  TransformPlan* tp;
  sp_status st;
  if ((st = make_plan(ctx, pr, pr->Nz, pr->Ngz, &tp)) != SP_OK) return st;
  if ((st = make_plan(ctx, pr, pr->Nx, pr->Ngx, &tp)) != SP_OK) return st;
  if (pr->ndim == 3 && (st = make_plan(ctx, pr, pr->Ny, pr->Ngy, &tp)) != SP_OK) return st;
  // band storage
  const int kuu = pr->kl + pr->ku;
  pr->npad = (pr->n + SOLVE_CHUNK - 1) / SOLVE_CHUNK * SOLVE_CHUNK;
  pr->lpad = std::max(2, (pr->kl + 1) / 2 * 2);
  pr->upad = kuu <= 31 ? 32 : 64;
  // SBDFq keeps q factors (its start-up orders); the Runge-Kutta schemes one
  const int nfactors = is_cnab(pr->scheme) ? 1 : std::max(1, sbdf_order(pr->scheme));
  // thousands of pencils fill the GPU with one lane per right-hand side
  pr->lanes = pr->solve_kind == SP_SOLVE_LANES ||
              (pr->solve_kind == SP_SOLVE_AUTO && pr->P >= LANE_MIN_PENCILS && lanes_supported(pr->kl, kuu));
  const size_t ngroups = (pr->P + LANE_GROUP - 1) / LANE_GROUP;
  if (pr->lanes) {
    CK(dalloc(&pr->d_bg, (size_t)pr->P * pr->n));
    CK(dalloc(&pr->d_xg, (size_t)pr->P * pr->n));
    CK(dalloc(&pr->d_yg, ngroups * LANE_GROUP * pr->n));
  }
  // mixed precision: the Chebyshev backward transform on the tensor cores
  // (SP_ZT_MMA, or SP_ZT_AUTO on three-dimensional problems), when its sizes fit
  pr->zmma = pr->prec == SP_PREC_MIXED && cheb_mma_supported(pr->Nz, pr->Ngz) &&
             (pr->zkind == SP_ZT_MMA || (pr->zkind == SP_ZT_AUTO && pr->ndim == 3));
  if (pr->zmma) {
    cudaError_t e = cheb_mma_setup(pr->cm, pr->P, pr->Nz, pr->Ngz, pr->S, s);
    if (e != cudaSuccess) {
      cheb_mma_free(pr->cm);
      pr->zmma = false;
      if (pr->zkind == SP_ZT_MMA) CK(e);
    }
  }
  // a few hundred pencils are too few chains for the GPU: cut each pencil's
  // rows into blocks substituted in parallel (spike.cu)
  pr->nblk = pr->spike_blocks > 0 ? pr->spike_blocks : default_spike_blocks(pr->npad, pr->P);
  pr->spike = !pr->lanes && spike_supported(pr->kl, kuu, pr->npad, pr->nblk) &&
              (pr->solve_kind == SP_SOLVE_SPIKE ||
               (pr->solve_kind == SP_SOLVE_AUTO && pr->P < SPIKE_MAX_PENCILS && pr->npad >= SPIKE_MIN_ROWS));
  if (pr->spike) {
    CK(dalloc(&pr->d_bg, (size_t)pr->P * pr->n));
    CK(dalloc(&pr->d_xg, (size_t)pr->P * pr->n));
    CK(dalloc(&pr->d_yg, (size_t)pr->P * pr->n));
    pr->nblk_f = spike_forward_blocks(pr->npad);
    const size_t nv = (size_t)pr->P * pr->nblk * 2, nvf = (size_t)pr->P * pr->nblk_f * 2;
    CK(dalloc(&pr->d_sp_s0, nvf * 8));
    CK(dalloc(&pr->d_sp_s, nvf * 8));
    CK(dalloc(&pr->d_sp_o0, nv * 32));
    CK(dalloc(&pr->d_sp_u, nv * 32));
    CK(reset_spike_guess(pr, ctx->stream));
  }
  for (int fi = 0; fi < nfactors; ++fi) {
    BandFactor& f = pr->fac[fi];
    if (pr->lanes) {
      CK(dalloc(&f.Lg, ngroups * pr->n * pr->kl * LANE_GROUP));
      CK(dalloc(&f.pg, ngroups * pr->n * LANE_GROUP));
      CK(dalloc(&f.umask, (size_t)pr->n));
    }
    CK(dalloc(&f.L, (size_t)pr->P * pr->npad * pr->lpad));
    CK(dalloc(&f.piv, (size_t)pr->P * pr->npad));
    CK(dalloc(&f.U, (size_t)pr->P * pr->npad * pr->upad));
    CK(dalloc(&f.rd, (size_t)pr->P * pr->npad));
    if (pr->spike) {
      CK(dalloc(&f.spD, (size_t)pr->P * pr->nblk_f * 7 * 8));
      CK(dalloc(&f.spE, (size_t)pr->P * pr->nblk * kuu * 32));
    }
  }
  CK(cudaStreamSynchronize(s));
  pr->uploaded = true;
  return SP_OK;
}

void free_problem(Problem* pr) {
  auto F = [](void* p) { if (p) cudaFree(p); };
  F(pr->d_indptr); F(pr->d_indices); F(pr->d_Mv); F(pr->d_Lv); F(pr->d_indptrM); F(pr->d_indicesM); F(pr->d_mrows); F(pr->d_MvC); F(pr->d_col_map); F(pr->d_row_map);
  F(pr->d_var_rec); F(pr->d_var_ph); F(pr->d_eq_diff); F(pr->d_eq_ph); F(pr->d_bc_rows); F(pr->d_nl_eq);

  F(pr->d_cfl_grid); F(pr->d_cfl_mid1); F(pr->d_cfl_mid2); F(pr->d_inv_dz); F(pr->d_cfl_args); F(pr->d_cfl_out);
  F(pr->d_bc_values); F(pr->d_kx); F(pr->d_gvar); F(pr->d_gop); F(pr->d_tslot); F(pr->d_tfa); F(pr->d_tfb);
  F(pr->d_tcoef); F(pr->d_ident); F(pr->d_zero); F(pr->d_Xt); F(pr->d_Xc); F(pr->d_Xc32); F(pr->d_kx32);
  F(pr->d_tcoef32);
  for (auto b : pr->d_MX) F(b);
  for (auto b : pr->d_LX) F(b);
  for (auto b : pr->d_Fc) F(b);
  F(pr->d_gz); F(pr->d_gy); F(pr->d_h);
  for (auto& f : pr->fac) { F(f.L); F(f.piv); F(f.U); F(f.rd); F(f.Lg); F(f.Ug); F(f.pg); F(f.umask); F(f.spD); F(f.spE); }
  F(pr->d_bg); F(pr->d_xg); F(pr->d_yg);
  F(pr->d_sp_s0); F(pr->d_sp_s); F(pr->d_sp_o0); F(pr->d_sp_u);
  cheb_mma_free(pr->cm);
  F(pr->d_lb_F); F(pr->d_lb_eq); F(pr->d_eigx); F(pr->d_eigsig);
  F(pr->facT.L); F(pr->facT.piv); F(pr->facT.U); F(pr->facT.rd); F(pr->facT.spE); F(pr->d_spT_u);
  F(pr->d_indptrT); F(pr->d_indicesT); F(pr->d_MvT); F(pr->d_LvT);
  F(pr->d_mu[0]); F(pr->d_mu[1]); F(pr->d_LTmu); F(pr->d_MTmu); F(pr->d_JF); F(pr->d_lamx);
  F(pr->d_Xbar); F(pr->d_Fbar); F(pr->d_Fbar32); F(pr->d_gzadj);
  for (auto& kv : pr->plans) { F(kv.second.tw64); F(kv.second.tw32); F(kv.second.dct64); F(kv.second.dct32); }
  for (auto& kv : pr->graphs) cudaGraphExecDestroy(kv.second);
  for (auto e : pr->ev) cudaEventDestroy(e);
}

// Grid <-> coefficient transforms of nf fields at grid sizes (Ngx, Ngy, Ngz)
// (Ngy = 1 on 2D problems) in precision prec, device buffers:
//   grid [f][iz][iy][ix] real FP64, coefficients [f][p][m] complex FP64
//   (backward: fields f_var[0 .. nf) of xc with field stride xstride, or of
//   an FP32 copy xc32 in mixed precision).
// Scratch: mid1 and mid2, grid_scratch_elems complex values each in precision prec.
size_t grid_scratch_elems(Problem* pr, int nf, int Ngy, int Ngz) {
  return (size_t)nf * Ngz * std::max((size_t)Ngy * pr->K, (size_t)pr->P);
}
cudaError_t grid_to_coef(Problem* pr, cudaStream_t s, int prec, int nf, TransformPlan& px, TransformPlan* py,
                         TransformPlan& pz, int Ngy, int Ngz, double* grid, double2* coef, void* mid1, void* mid2) {
  cudaError_t e = launch_fourier_rows(s, prec, px, Ngz * Ngy, pr->K, 4, nf, nullptr, grid, nullptr, 0, nullptr,
                                      nullptr, nullptr, nullptr, 0, mid1);
  if (e != cudaSuccess) return e;
  if (pr->ndim == 3) {
    if ((e = launch_fourier_y(s, prec, *py, +1, nf, Ngz, pr->K, mid1, mid2)) != cudaSuccess) return e;
    return launch_cheb_forward(s, prec, pz, pr->P, nf, mid2, coef);
  }
  return launch_cheb_forward(s, prec, pz, pr->P, nf, mid1, coef);
}
cudaError_t coef_to_grid(Problem* pr, cudaStream_t s, int prec, int nf, TransformPlan& px, TransformPlan* py,
                         TransformPlan& pz, int Ngy, int Ngz, const int32_t* f_var, const double2* xc, int xstride,
                         const float2* xc32, double* grid, void* mid1, void* mid2) {
  void* zout = pr->ndim == 3 ? mid2 : mid1;
  cudaError_t e = launch_cheb_backward(s, prec, pz, pr->P, nf, f_var, pr->d_zero, pr->d_kx, xc, xstride, zout,
                                       pr->d_kx32, xc32);
  if (e != cudaSuccess) return e;
  if (pr->ndim == 3 && (e = launch_fourier_y(s, prec, *py, -1, nf, Ngz, pr->K, mid2, mid1)) != cudaSuccess)
    return e;
  return launch_fourier_rows(s, prec, px, Ngz * Ngy, pr->K, 1, nf, mid1, nullptr, grid, 0, nullptr, nullptr,
                             nullptr, nullptr, 0, nullptr);
}

// F(X) for the current coefficient state: z backward -> (y backward) -> x
// rows (products) -> (y forward) -> z forward
sp_status eval_rhs(sp_ctx* ctx, Problem* pr, cudaStream_t s, double2* fc_out) {
  if (pr->nl_eqs.empty()) {
    CK(cudaMemsetAsync(fc_out, 0, (size_t)pr->P * pr->Nz * sizeof(double2), s));
    return SP_OK;
  }
  TransformPlan& pz = pr->plans.at({pr->Nz, pr->Ngz});
  TransformPlan& px = pr->plans.at({pr->Nx, pr->Ngx});
  const int nf = (int)pr->gfields.size(), ne = (int)pr->nl_eqs.size();
  if (pr->prec && !pr->xc32_valid) {
    CK(launch_to_f32(s, pr->d_Xc, pr->d_Xc32, (size_t)pr->S * pr->P * pr->Nz));
    pr->xc32_valid = true;
  }
  if (pr->zmma) {
    // z backward on the tensor cores from the split FP32 copy
    if (!pr->xs32_valid) {
      CK(launch_to_f32_split(s, pr->d_Xc, pr->cm.xs32, (size_t)pr->S * pr->P, pr->Nz));
      pr->xs32_valid = true;
    }
    std::vector<int> fv(nf), fo(nf);
    for (int f = 0; f < nf; ++f) { fv[f] = pr->gfields[f].var; fo[f] = pr->gfields[f].op; }
    CK(launch_cheb_backward_mma(s, pr->cm, nf, fv.data(), fo.data(), pr->d_kx32, pr->d_gz, ctx->d_status));
  } else {
    CK(launch_cheb_backward(s, pr->prec, pz, pr->P, nf, pr->d_gvar, pr->d_gop, pr->d_kx, pr->d_Xc,
                            pr->P * pr->Nz, pr->d_gz, pr->d_kx32, pr->d_Xc32));
  }
  if (pr->ndim == 3) {
    TransformPlan& py = pr->plans.at({pr->Ny, pr->Ngy});
    CK(launch_fourier_y(s, pr->prec, py, -1, nf, pr->Ngz, pr->K, pr->d_gz, pr->d_gy));
    CK(launch_fourier_rows(s, pr->prec, px, pr->Ngz * pr->Ngy, pr->K, 7, nf, pr->d_gy, nullptr, nullptr,
                           (int)pr->t_slot.size(), pr->d_tslot, pr->d_tcoef, pr->d_tfa, pr->d_tfb, ne, pr->d_h,
                           pr->d_tcoef32));
    CK(launch_fourier_y(s, pr->prec, py, +1, ne, pr->Ngz, pr->K, pr->d_h, pr->d_gz));
    CK(launch_cheb_forward(s, pr->prec, pz, pr->P, ne, pr->d_gz, fc_out));
    return SP_OK;
  }
  CK(launch_fourier_rows(s, pr->prec, px, pr->Ngz, pr->K, 7, nf, pr->d_gz, nullptr, nullptr,
                         (int)pr->t_slot.size(), pr->d_tslot, pr->d_tcoef, pr->d_tfa, pr->d_tfb, ne, pr->d_h,
                         pr->d_tcoef32));
  CK(launch_cheb_forward(s, pr->prec, pz, pr->P, ne, pr->d_h, fc_out));
  return SP_OK;
}

SolveArgs base_args(Problem* pr, sp_ctx* ctx, int fac) {
  SolveArgs a{};
  a.P = pr->P; a.n = pr->n; a.Nz = pr->Nz; a.S = pr->S; a.nbc = pr->nbc; a.nnz = (int)pr->nnz;
  a.kl = pr->kl; a.kuu = pr->kl + pr->ku; a.npad = pr->npad; a.lpad = pr->lpad; a.upad = pr->upad;
  a.Lf = pr->fac[fac].L; a.piv = pr->fac[fac].piv; a.Uf = pr->fac[fac].U; a.rd = pr->fac[fac].rd;
  a.indptr = pr->d_indptr; a.indices = pr->d_indices;
  a.row_map = pr->d_row_map; a.col_map = pr->d_col_map;
  a.var_recombine = pr->d_var_rec; a.var_phase = pr->d_var_ph;
  a.eq_differential = pr->d_eq_diff; a.eq_phase = pr->d_eq_ph;
  a.nl_eq = pr->d_nl_eq; a.n_nl = (int)pr->nl_eqs.size();
  a.bc_rows = pr->d_bc_rows; a.bc_values = pr->d_bc_values;
  a.status = ctx->d_status;
  a.xc32_out = pr->d_Xc32;   // null unless mixed precision
  a.xs32_out = pr->zmma ? pr->cm.xs32 : nullptr;
  a.Lg = pr->fac[fac].Lg; a.Ug = pr->fac[fac].Ug; a.pg = pr->fac[fac].pg;   // null unless lane mode
  a.cmax = pr->fac[fac].cmax;
  a.umask = pr->fac[fac].umask;
  a.spD = pr->spike ? pr->fac[fac].spD : nullptr;   // null unless partitioned substitution
  a.spE = pr->spike ? pr->fac[fac].spE : nullptr;
  return a;
}

void set_mv_M(Problem* pr, SolveArgs& a) {
  a.mv_vals = pr->d_MvC; a.mv_indptr = pr->d_indptrM; a.mv_indices = pr->d_indicesM; a.mv_nnz = (int)pr->nnzM;
}
void set_ep_M(Problem* pr, SolveArgs& a) {
  a.ep_mv_vals = pr->d_MvC; a.ep_indptr = pr->d_indptrM; a.ep_indices = pr->d_indicesM; a.ep_nnz = (int)pr->nnzM;
  a.ep_rows = pr->d_mrows; a.ep_nrows = pr->nmrows;
}
void set_ep_L(Problem* pr, SolveArgs& a) {
  a.ep_mv_vals = pr->d_Lv; a.ep_indptr = pr->d_indptr; a.ep_indices = pr->d_indices; a.ep_nnz = (int)pr->nnz;
  a.ep_rows = nullptr; a.ep_nrows = 0;
}

sp_status solve(sp_ctx* ctx, Problem* pr, cudaStream_t s, const SolveArgs& a) {
  const bool t = pr->timing && pr->ev_used + 2 <= pr->ev.size();
  if (t) CK(cudaEventRecord(pr->ev[pr->ev_used], s));
  if (pr->spike && a.Lf && a.Lf == pr->facT.L && pr->facT.spE && pr->d_spT_u) {
    // transposed solve: assembly and whole-row forward substitution (mode 3),
    // partitioned back substitution from the last transposed solve's inflows,
    // epilogue
    SolveArgs a3 = a;
    a3.mode = 3; a3.yg = pr->d_yg;
    CK(launch_pencil_solve(s, a3));
    SpikeArgs sa{};
    sa.P = pr->P; sa.n = pr->n; sa.npad = pr->npad; sa.kl = a.kl; sa.kuu = a.kuu; sa.lpad = a.lpad;
    sa.upad = a.upad; sa.nblk = pr->nblk; sa.m = pr->npad / pr->nblk;
    sa.nblk_f = pr->nblk_f; sa.m_f = pr->npad / pr->nblk_f;
    sa.U = a.Uf; sa.rd = a.rd; sa.E = pr->facT.spE;
    sa.yg = pr->d_yg; sa.xg = pr->d_xg;
    sa.o0 = pr->d_sp_o0; sa.uin = pr->d_spT_u;
    sa.status = ctx->d_status;
    CK(launch_spike_backward(s, sa));
    SolveArgs a2 = a;
    a2.mode = 2; a2.xg = pr->d_xg; a2.bg = pr->d_bg;
    CK(launch_pencil_solve(s, a2));
    if (t) {
      CK(cudaEventRecord(pr->ev[pr->ev_used + 1], s));
      pr->ev_used += 2;
    }
    return SP_OK;
  }
  if ((a.Lg && pr->lanes) || (a.spD && pr->spike)) {
    // assembly -> lane-per-pencil or partitioned substitution -> epilogue
    SolveArgs a1 = a;
    a1.mode = 1; a1.bg = pr->d_bg;
    CK(launch_pencil_solve(s, a1));
    if (pr->lanes) {
      CK(launch_pencil_lanes(s, pr->P, pr->n, a.kl, a.kuu, a.Lg, a.Ug, a.cmax, a.pg, a.umask, pr->d_bg,
                             pr->d_yg, pr->d_xg));
    } else {
      SpikeArgs sa{};
      sa.P = pr->P; sa.n = pr->n; sa.npad = pr->npad; sa.kl = a.kl; sa.kuu = a.kuu; sa.lpad = a.lpad;
      sa.upad = a.upad; sa.nblk = pr->nblk; sa.m = pr->npad / pr->nblk;
      sa.nblk_f = pr->nblk_f; sa.m_f = pr->npad / pr->nblk_f;
      sa.L = a.Lf; sa.piv = a.piv; sa.U = a.Uf; sa.rd = a.rd; sa.D = a.spD; sa.E = a.spE;
      sa.bg = pr->d_bg; sa.yg = pr->d_yg; sa.xg = pr->d_xg;
      sa.s0 = pr->d_sp_s0; sa.sst = pr->d_sp_s; sa.o0 = pr->d_sp_o0; sa.uin = pr->d_sp_u;
      sa.status = ctx->d_status;
      CK(launch_spike_solve(s, sa));
    }
    SolveArgs a2 = a;
    a2.mode = 2; a2.xg = pr->d_xg; a2.bg = pr->d_bg;
    if (a2.ep_mv_vals == pr->d_Lv && pr->prec) {
      // L~ X~ of a stage.  FP64 form: the product with L~ itself.  Mixed
      // form: from the stage's own right-hand side, (B~ - alpha M~ X~) / beta
      // with the factored alpha M~ + beta L~, M~'s compact pattern instead of
      // L~'s (3D: 1508 against 6073 entries per pencil, ~0.5 ms of FP64 pipe
      // per stage at 256 x 256 x 128).  B~ is alpha M~ X~ up to O(beta), so
      // the difference cancels; the error it leaves in a later stage's
      // right-hand side, dt a_ij L~X~ = (a_ij / a_jj)(B~ - alpha M~ X~), is a
      // few FP64 roundings of M~X~, far below the FP32 transforms' 1e-7 but
      // above the FP64 form's own rounding (the 500-step RK222 adjoint
      // gradient drifts 15x past the oracle floor), hence FP64 keeps L~.
      int fi = 0;
      for (int q = 1; q < 4; ++q)
        if (a.Lf == pr->fac[q].L && pr->fac[q].L) fi = q;
      const BandFactor& f = pr->fac[fi];
      set_ep_M(pr, a2);
      a2.ep_alpha = f.alpha;
      a2.ep_from_b = 1.0 / f.beta;
    }
    CK(launch_pencil_solve(s, a2));
  } else {
    CK(launch_pencil_solve(s, a));
  }
  if (t) {
    CK(cudaEventRecord(pr->ev[pr->ev_used + 1], s));
    pr->ev_used += 2;
  }
  return SP_OK;
}

// One stage of a step: evaluate F of the current state into fc_out (if
// set), then one pencil solve with `args`.
struct StagePlan {
  double2* fc_out;
  SolveArgs args;
};

// The stages of one IMEX step (Sec. "Timesteppers") for the problem's
// current state, without touching that state.  Valid when xt_valid.
std::vector<StagePlan> plan_step(sp_ctx* ctx, Problem* pr, double dt) {
  std::vector<StagePlan> plan;
  if (is_rk(pr->scheme)) {
    const Tableau tb = make_tableau(pr->scheme);
    for (int i = 1; i <= tb.s; ++i) {
      SolveArgs a = base_args(pr, ctx, 0);
      // M~ X~^0 (stored, or computed on the first stage of a fresh state)
      if (i == 1 && !pr->mx_valid) {
        a.mv_x = pr->d_Xt; a.mv_coef = 1.0; a.mv_store = pr->d_MX[0];
        set_mv_M(pr, a);
      } else {
        a.vec[a.nvec] = pr->d_MX[0]; a.vec_coef[a.nvec++] = 1.0;
      }
      // - dt sum_{j<i} H_ij L~ X~^j (H_i0 = 0: the first stage is explicit)
      for (int j = 1; j < i; ++j)
        if (tb.H[i][j] != 0.0) { a.vec[a.nvec] = pr->d_LX[j]; a.vec_coef[a.nvec++] = -dt * tb.H[i][j]; }
      // dt sum_{j<i} A_ij F~^j, boundary rows get dt sum_j A_ij g
      double csum = 0.0;
      for (int j = 0; j < i; ++j)
        if (tb.A[i][j] != 0.0) { a.fc[a.nfc] = pr->d_Fc[j]; a.fc_coef[a.nfc++] = dt * tb.A[i][j]; csum += tb.A[i][j]; }
      a.bc_coef = dt * csum;
      a.xc_out = pr->d_Xc;
      if (i < tb.s) {
        set_ep_L(pr, a); a.ep_mv_store = pr->d_LX[i];             // L~ X~^i for later stages
      } else {
        a.xt_out = pr->d_Xt;
        set_ep_M(pr, a); a.ep_mv_store = pr->d_MX[0];             // M~ X~^{n+1} for the next step
      }
      plan.push_back(StagePlan{pr->d_Fc[i - 1], a});               // F(X^{i-1}) before stage i
    }
  } else if (is_cnab(pr->scheme)) {
    // CNAB1 / CNAB2: M~ X~^n and L~ X~^n evaluated in the prologue (two
    // matvecs on X~^n: B~ = M~X~^n - dt/2 L~X~^n + dt sum_j c_j F~), the F~
    // ring as in SBDF (slot it mod 2 holds step it's F~), one factor
    const int it = pr->iteration, D = sbdf_depth(pr->scheme);
    const int o = std::min(sbdf_order(pr->scheme), it + 1);
    const int cur = it % D;
    SolveArgs a = base_args(pr, ctx, 0);
    a.mv_x = pr->d_Xt; a.mv_coef = 1.0; a.mv_store = nullptr;
    set_mv_M(pr, a);
    a.mv2_vals = pr->d_Lv; a.mv2_coef = -0.5 * dt;
    a.mv2_indptr = pr->d_indptr; a.mv2_indices = pr->d_indices; a.mv2_nnz = (int)pr->nnz;
    for (int j = 1; j <= o; ++j) {
      const int slot = ((it + 1 - j) % D + D) % D;
      a.fc[a.nfc] = pr->d_Fc[slot]; a.fc_coef[a.nfc++] = dt * CNAB_C[o][j];
    }
    a.bc_coef = dt;
    a.xt_out = pr->d_Xt;
    a.xc_out = pr->d_Xc;
    plan.push_back(StagePlan{pr->d_Fc[cur], a});
  } else {
    // SBDF1 .. SBDF4 (Wang & Ruuth 2008), constant step, the first steps at
    // the orders the history allows (SBDF1, SBDF2, ...), with SBDF_A / SBDF_C.
    // Slot (it mod D) of the M~X~ and F~ rings holds step it's values.
    const int it = pr->iteration, D = sbdf_depth(pr->scheme);
    const int o = std::min(sbdf_order(pr->scheme), it + 1);
    const int cur = it % D;
    SolveArgs a = base_args(pr, ctx, o - 1);
    for (int j = 1; j <= o; ++j) {
      const int slot = ((it + 1 - j) % D + D) % D;
      const double cm = -SBDF_A[o][j];
      if (j == 1 && !pr->mx_valid) {
        a.mv_x = pr->d_Xt; a.mv_store = pr->d_MX[cur]; a.mv_coef = cm;
        set_mv_M(pr, a);
      } else {
        a.vec[a.nvec] = pr->d_MX[slot]; a.vec_coef[a.nvec++] = cm;
      }
      a.fc[a.nfc] = pr->d_Fc[slot]; a.fc_coef[a.nfc++] = dt * SBDF_C[o][j];
    }
    a.bc_coef = dt;
    a.xt_out = pr->d_Xt;
    a.xc_out = pr->d_Xc;
    set_ep_M(pr, a); a.ep_mv_store = pr->d_MX[(it + 1) % D];     // M~ X~^{n+1} for the next step
    plan.push_back(StagePlan{pr->d_Fc[cur], a});
  }
  return plan;
}

// state after a planned step has been queued
void commit_step(Problem* pr) {
  pr->mx_valid = true;
  if (sbdf_order(pr->scheme) > 0) pr->iteration += 1;
}

sp_status ensure_solve_vars(sp_ctx* ctx, Problem* pr, cudaStream_t s) {
  if (!pr->xt_valid) {
    CK(launch_coef_to_solve(s, pr->P, pr->S, pr->Nz, pr->d_Xc, pr->d_Xt, pr->d_col_map, pr->d_var_rec,
                            pr->d_var_ph));
    pr->xt_valid = true;
    pr->mx_valid = false;
  }
  return SP_OK;
}

// One IMEX step (Sec. "Timesteppers") queued on stream s.
sp_status one_step(sp_ctx* ctx, Problem* pr, cudaStream_t s, double dt) {
  sp_status st;
  if ((st = ensure_solve_vars(ctx, pr, s)) != SP_OK) return st;
  for (const StagePlan& sp : plan_step(ctx, pr, dt)) {
    if ((st = eval_rhs(ctx, pr, s, sp.fc_out)) != SP_OK) return st;
    if ((st = solve(ctx, pr, s, sp.args)) != SP_OK) return st;
  }
  commit_step(pr);
  return SP_OK;
}

// ---------------------------------------------------------------------------
// batches: every kernel type launched once per stage over all problems
// ---------------------------------------------------------------------------
ZDesc zdesc_backward(Problem* pr) {
  TransformPlan& pz = pr->plans.at({pr->Nz, pr->Ngz});
  ZDesc d{};
  d.Nc = pz.Nc; d.Ng = pz.Ng; d.radix3 = pz.radix3; d.P = pr->P;
  d.tw = pr->prec ? pz.tw32 : pz.tw64; d.wq = pr->prec ? pz.dct32 : pz.dct64;
  d.f_var = pr->d_gvar; d.f_op = pr->d_gop; d.kx = pr->d_kx; d.xc = pr->d_Xc; d.xc_stride = pr->P * pr->Nz;
  d.gz = pr->d_gz;
  d.kx32 = pr->d_kx32; d.xc32 = pr->d_Xc32;
  return d;
}
ZDesc zdesc_forward(Problem* pr, double2* fc) {
  ZDesc d = zdesc_backward(pr);
  d.h = pr->d_h; d.fc = fc;
  return d;
}
XDesc xdesc_rows(Problem* pr) {
  TransformPlan& px = pr->plans.at({pr->Nx, pr->Ngx});
  XDesc d{};
  d.N = px.Ng; d.radix3 = px.radix3; d.rows = pr->Ngz; d.K = pr->P; d.mode = 7; d.nf = (int)pr->gfields.size();
  d.tw = pr->prec ? px.tw32 : px.tw64;
  d.gz = pr->d_gz;
  d.nterms = (int)pr->t_slot.size(); d.t_eq = pr->d_tslot; d.t_coef = pr->d_tcoef; d.t_fa = pr->d_tfa;
  d.t_fb = pr->d_tfb; d.ne = (int)pr->nl_eqs.size(); d.h = pr->d_h;
  d.t_coef32 = pr->d_tcoef32;
  return d;
}

// --- adjoint ---------------------------------------------------------------
// Solve arguments for A~^T y = rhs with the transposed factor (no right-hand
// side assembly beyond stored vectors, no boundary values).
SolveArgs transposed_args(Problem* pr, sp_ctx* ctx) {
  SolveArgs a = base_args(pr, ctx, 0);
  a.kl = pr->klT; a.kuu = pr->klT + pr->kuT; a.lpad = pr->lpadT;
  a.Lf = pr->facT.L; a.piv = pr->facT.piv; a.Uf = pr->facT.U; a.rd = pr->facT.rd;
  a.n_nl = 0; a.nbc = 0; a.bc_coef = 0.0;
  a.xc32_out = nullptr;
  a.xs32_out = nullptr;
  a.Lg = nullptr; a.Ug = nullptr; a.pg = nullptr; a.umask = nullptr;
  a.spD = nullptr; a.spE = nullptr;      // no coupling matrices for the transposed factor
  a.ep_rows = nullptr; a.ep_nrows = 0;   // the transposed patterns carry no row list
  return a;
}

// out = J_F(X)^H (sum_k c_k vecs_k) + sum_a w_a adds_a in solve variables,
// X the T coefficients xc ([v][p][m], device) (Sec. "Runge-Kutta IMEX
// integrators": transpose of the right-hand side of a stage).  In mixed
// precision the FP32 copy of X is rebuilt in d_Xc32.
sp_status adjoint_rhs(sp_ctx* ctx, Problem* pr, cudaStream_t s, const double2* xc, int nv,
                      const double2* const* vecs, const double* coefs, int na, const double2* const* adds,
                      const double* wts, double2* out) {
  TransformPlan& pz = pr->plans.at({pr->Nz, pr->Ngz});
  TransformPlan& px = pr->plans.at({pr->Nx, pr->Ngx});
  const int nf = (int)pr->gfields.size(), ne = (int)pr->nl_eqs.size();
  if (pr->prec) {
    CK(launch_to_f32(s, xc, pr->d_Xc32, (size_t)pr->S * pr->P * pr->Nz));
    pr->xc32_valid = (xc == pr->d_Xc);
    pr->xs32_valid = false;
  }
  CK(launch_adj_gather(s, pr->P, pr->Nz, pr->Ngz, pr->n, ne, pr->d_nl_eq, pr->d_row_map, pr->d_eq_diff,
                       pr->d_eq_ph, nv, vecs, coefs, pr->d_Fbar, pr->prec ? pr->d_Fbar32 : nullptr));
  CK(launch_cheb_backward(s, pr->prec, pz, pr->P, nf, pr->d_gvar, pr->d_gop, pr->d_kx, xc, pr->P * pr->Nz,
                          pr->d_gz, pr->d_kx32, pr->d_Xc32));
  CK(launch_cheb_backward(s, pr->prec, pz, pr->P, ne, pr->d_ident, pr->d_zero, pr->d_kx, pr->d_Fbar,
                          pr->P * pr->Nz, pr->d_h, pr->d_kx32, pr->d_Fbar32));
  CK(launch_fourier_rows_adjoint(s, pr->prec, px, pr->Ngz, pr->P, nf, pr->d_gz, ne, pr->d_h,
                                 (int)pr->t_slot.size(), pr->d_tslot, pr->d_tcoef, pr->d_tcoef32, pr->d_tfa,
                                 pr->d_tfb, pr->d_gzadj));
  CK(launch_cheb_forward(s, pr->prec, pz, pr->P, nf, pr->d_gzadj, pr->d_Xbar, 1));
  CK(launch_adj_combine(s, pr->P, pr->Nz, pr->S, pr->n, nf, pr->d_gvar, pr->d_gop, pr->d_kx, pr->d_Xbar,
                        pr->d_col_map, pr->d_var_rec, pr->d_var_ph, na, adds, wts, out));
  return SP_OK;
}

}  // namespace

struct BatchStage {
  ZDesc* d_zb = nullptr; ZDesc* d_zf = nullptr; XDesc* d_x = nullptr; SolveArgs* d_args = nullptr;
};
struct Batch {
  std::vector<int> ids;
  int prec = 0, scheme = 0, nstage = 0, parity = 0;
  int tile = 8;
  int max_ngz = 0, max_kuu = 0;
  size_t x_smem = 0, s_smem = 0;
  int4 *d_wzb = nullptr, *d_wx = nullptr, *d_wzf = nullptr, *d_ws = nullptr;
  int nzb = 0, nx = 0, nzf = 0, ns = 0;
  std::vector<BatchStage> stages;
  std::map<int, cudaGraphExec_t> graphs;     // by block length
  // persistent launches: four work counters per stage, zeroed once per step
  bool persist = false;
  int* d_queue = nullptr;
};

namespace {

void free_batch(Batch* b) {
  auto F = [](void* p) { if (p) cudaFree(p); };
  F(b->d_wzb); F(b->d_wx); F(b->d_wzf); F(b->d_ws); F(b->d_queue);
  for (auto& st : b->stages) { F(st.d_zb); F(st.d_zf); F(st.d_x); F(st.d_args); }
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
}

template <typename T>
cudaError_t upload_vec(T** d, const std::vector<T>& v) {
  cudaError_t e = cudaMalloc((void**)d, std::max<size_t>(v.size(), 1) * sizeof(T));
  if (e != cudaSuccess || v.empty()) return e;
  return cudaMemcpy(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

// Work lists in descending cost order (largest items first).
sp_status build_batch(sp_ctx* ctx, const std::vector<Problem*>& ps, const std::vector<int>& ids, int tile,
                      int parity, bool persist, Batch* b) {
  b->ids = ids;
  b->persist = persist;
  b->prec = ps[0]->prec;
  b->scheme = ps[0]->scheme;
  b->tile = tile;
  b->parity = parity;
  std::vector<std::pair<long long, int4>> zb, xr, zf, sv;
  for (size_t q = 0; q < ps.size(); ++q) {
    Problem* pr = ps[q];
    const int nt = (pr->P + tile - 1) / tile;
    const long long zc = (long long)pr->Ngz * 100 + pr->Nz;
    for (int f = 0; f < (int)pr->gfields.size(); ++f)
      for (int t = 0; t < nt; ++t) zb.push_back({zc, make_int4((int)q, t, f, 0)});
    for (int e = 0; e < (int)pr->nl_eqs.size(); ++e)
      for (int t = 0; t < nt; ++t) zf.push_back({zc, make_int4((int)q, t, e, 0)});
    for (int r = 0; r < pr->Ngz; ++r) xr.push_back({(long long)pr->Ngx, make_int4((int)q, r, 0, 0)});
    for (int p = 0; p < pr->P; ++p) sv.push_back({(long long)pr->n, make_int4((int)q, p, 0, 0)});
    b->max_ngz = std::max(b->max_ngz, pr->Ngz);
    b->max_kuu = std::max(b->max_kuu, pr->kl + pr->ku);
    b->x_smem = std::max(b->x_smem, x_smem_bytes(pr->prec, pr->Ngx, 7, (int)pr->gfields.size(),
                                                 (int)pr->nl_eqs.size()));
    b->s_smem = std::max(b->s_smem, pencil_solve_smem(pr->npad, pr->lpad, pr->upad));
  }
  auto finish = [](std::vector<std::pair<long long, int4>>& v) {
    std::stable_sort(v.begin(), v.end(), [](const auto& a, const auto& c) { return a.first > c.first; });
    std::vector<int4> out;
    for (auto& x : v) out.push_back(x.second);
    return out;
  };
  auto wzb = finish(zb), wx = finish(xr), wzf = finish(zf), ws = finish(sv);
  b->nzb = (int)wzb.size(); b->nx = (int)wx.size(); b->nzf = (int)wzf.size(); b->ns = (int)ws.size();
  CK(upload_vec(&b->d_wzb, wzb));
  CK(upload_vec(&b->d_wx, wx));
  CK(upload_vec(&b->d_wzf, wzf));
  CK(upload_vec(&b->d_ws, ws));
  // per-stage descriptor tables from the single-problem plans, planned at
  // the requested schedule phase (multistep schemes rotate their buffers)
  std::vector<std::vector<StagePlan>> plans;
  for (Problem* pr : ps) {
    const int saved = pr->iteration;
    // a steady-state iteration of the requested phase (past the start-up orders)
    if (sbdf_order(b->scheme) > 0) pr->iteration = sbdf_depth(b->scheme) + parity;
    plans.push_back(plan_step(ctx, pr, pr->fac_dt));
    pr->iteration = saved;
  }
  b->nstage = (int)plans[0].size();
  for (int i = 0; i < b->nstage; ++i) {
    std::vector<ZDesc> zbv, zfv;
    std::vector<XDesc> xv;
    std::vector<SolveArgs> av;
    for (size_t q = 0; q < ps.size(); ++q) {
      zbv.push_back(zdesc_backward(ps[q]));
      xv.push_back(xdesc_rows(ps[q]));
      zfv.push_back(zdesc_forward(ps[q], plans[q][i].fc_out));
      av.push_back(plans[q][i].args);
      av.back().fwd16 = 1;            // throughput-bound: both parts' forward in one warp
      fill_f_halves(av.back());
    }
    BatchStage st;
    CK(upload_vec(&st.d_zb, zbv));
    CK(upload_vec(&st.d_x, xv));
    CK(upload_vec(&st.d_zf, zfv));
    CK(upload_vec(&st.d_args, av));
    b->stages.push_back(st);
  }
  CK(dalloc(&b->d_queue, (size_t)4 * std::max(1, b->nstage)));
  return SP_OK;
}

// A batch bakes each problem's factor pointers and step coefficients (dt H,
// dt A, the SBDF weights, the boundary-row coefficient) into its device
// argument tables and captured graphs; once a problem is re-factored, every
// cached batch that holds it is stale and is dropped.
void drop_batches(sp_ctx* ctx, int problem) {
  for (auto it = ctx->batches.begin(); it != ctx->batches.end();) {
    const std::vector<int>& ids = it->first.first;
    if (std::find(ids.begin(), ids.end(), problem) != ids.end()) {
      free_batch(it->second);
      delete it->second;
      it = ctx->batches.erase(it);
    } else {
      ++it;
    }
  }
}

sp_status batch_step(sp_ctx* ctx, Batch* b, cudaStream_t s) {
  if (b->persist) CK(cudaMemsetAsync(b->d_queue, 0, (size_t)4 * b->nstage * sizeof(int), s));
  for (int i = 0; i < b->nstage; ++i) {
    const BatchStage& st = b->stages[i];
    int* q = b->persist ? b->d_queue + 4 * i : nullptr;
    CK(launch_cheb_backward_batched(s, b->prec, b->tile, st.d_zb, b->d_wzb, b->nzb, b->max_ngz, q));
    CK(launch_fourier_rows_batched(s, b->prec, st.d_x, b->d_wx, b->nx, b->x_smem, q ? q + 1 : nullptr));
    CK(launch_cheb_forward_batched(s, b->prec, b->tile, st.d_zf, b->d_wzf, b->nzf, b->max_ngz, q ? q + 2 : nullptr));
    CK(launch_pencil_solve_batched(s, st.d_args, b->d_ws, b->ns, b->max_kuu, b->s_smem));
  }
  return SP_OK;
}

}  // namespace

// ===========================================================================
// ABI
// ===========================================================================
extern "C" {

sp_status sp_create(sp_ctx** out, int device, void* cuda_stream) {
  if (!out) return SP_ERR_ARG;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) return SP_ERR_CUDA;
  if (device < 0 || device >= count) return SP_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return SP_ERR_CUDA;
  auto* ctx = new sp_ctx();
  ctx->device = device;
  ctx->stream = (cudaStream_t)cuda_stream;
  if (cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking) != cudaSuccess ||
      cudaMalloc(&ctx->d_status, sizeof(DevStatus)) != cudaSuccess ||
      cudaMemset(ctx->d_status, 0, sizeof(DevStatus)) != cudaSuccess) {
    delete ctx;
    return SP_ERR_CUDA;
  }
  *out = ctx;
  return SP_OK;
}

sp_status sp_destroy(sp_ctx* ctx) {
  if (!ctx) return SP_ERR_ARG;
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  for (auto& kv : ctx->batches) { free_batch(kv.second); delete kv.second; }
  for (auto& p : ctx->probs) free_problem(p.get());
  if (ctx->d_status) cudaFree(ctx->d_status);
  if (ctx->capture) cudaStreamDestroy(ctx->capture);
  delete ctx;
  return SP_OK;
}

const char* sp_last_error(const sp_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

sp_status sp_add_problem(sp_ctx* ctx, int ndim, const sp_basis* bases, int nvars, int scheme, int precision,
                         int* problem_id) {
  if (!ctx) return SP_ERR_ARG;
  ctx->err.clear();
  if (ndim != 2 && ndim != 3)
    return fail(ctx, SP_ERR_ARG, "ndim must be 2 (Fourier x Chebyshev) or 3 (Fourier x Fourier x Chebyshev)");
  if (!bases || !problem_id) return fail(ctx, SP_ERR_ARG, "null argument");
  const sp_basis& bx = bases[0];
  const sp_basis& bz = bases[ndim - 1];
  if (bx.kind != SP_FOURIER || bz.kind != SP_CHEBYSHEV || (ndim == 3 && bases[1].kind != SP_FOURIER))
    return fail(ctx, SP_ERR_ARG, "bases must be Fourier axes followed by one Chebyshev axis (last)");
  if (nvars < 1 || nvars > 16) return fail(ctx, SP_ERR_ARG, "nvars must be in [1, 16]");
  if (scheme < SP_RK222 || scheme > SP_CNAB2) return fail(ctx, SP_ERR_ARG, "unknown scheme %d", scheme);
  if (precision != SP_PREC_FP64 && precision != SP_PREC_MIXED)
    return fail(ctx, SP_ERR_ARG, "unknown precision %d", precision);
  auto pr = std::make_unique<Problem>();
  pr->ndim = ndim;
  pr->S = nvars;
  pr->scheme = scheme;
  pr->prec = precision == SP_PREC_MIXED ? 1 : 0;
  pr->bx = bx;
  pr->bz = bz;
  pr->Nx = bx.n_coeff;
  pr->Nz = bz.n_coeff;
  if (pr->Nx < 4 || pr->Nx % 2) return fail(ctx, SP_ERR_ARG, "N_x must be even and >= 4");
  if (pr->Nz < 4) return fail(ctx, SP_ERR_ARG, "N_z must be >= 4");
  for (int i = 0; i < ndim; ++i) {
    const sp_basis* b = &bases[i];
    if (b->dealias_num <= 0 || b->dealias_den <= 0 || (b->n_coeff * b->dealias_num) % b->dealias_den)
      return fail(ctx, SP_ERR_ARG, "dealias scale must give an integer grid size");
    if (b->dealias_num < b->dealias_den) return fail(ctx, SP_ERR_ARG, "dealias scale must be >= 1");
    if (!(b->b > b->a)) return fail(ctx, SP_ERR_ARG, "interval must have b > a");
  }
  pr->Ngx = bx.n_coeff * bx.dealias_num / bx.dealias_den;
  pr->Ngz = bz.n_coeff * bz.dealias_num / bz.dealias_den;
  if (!is_smooth_length(pr->Ngx) || pr->Ngx < 16 || pr->Ngx > 4096)
    return fail(ctx, SP_ERR_ARG, "N_gx = %d must be 2^k or 3*2^k in [16, 4096]", pr->Ngx);
  if (!is_smooth_length(pr->Ngz) || pr->Ngz < 8 || pr->Ngz > 1536)
    return fail(ctx, SP_ERR_ARG, "N_gz = %d must be 2^k or 3*2^k in [8, 1536]", pr->Ngz);
  pr->K = pr->Nx / 2;
  if (ndim == 3) {
    const sp_basis& by = bases[1];
    pr->by = by;
    pr->Ny = by.n_coeff;
    if (pr->Ny < 2 || pr->Ny % 2) return fail(ctx, SP_ERR_ARG, "N_y must be even and >= 2");
    pr->Ngy = by.n_coeff * by.dealias_num / by.dealias_den;
    if (!is_smooth_length(pr->Ngy) || pr->Ngy < 4 || pr->Ngy > 4096)
      return fail(ctx, SP_ERR_ARG, "N_gy = %d must be 2^k or 3*2^k in [4, 4096]", pr->Ngy);
    pr->Ly = by.b - by.a;
  }
  pr->P = pr->Ny * pr->K;
  pr->Lx = bx.b - bx.a;
  pr->za = bz.a;
  pr->zb = bz.b;
  pr->n = pr->S * pr->Nz;
  pr->pset.assign(pr->P, 0);
  ctx->probs.push_back(std::move(pr));
  *problem_id = (int)ctx->probs.size() - 1;
  return SP_OK;
}

sp_status sp_set_layout(sp_ctx* ctx, int problem, const int32_t* col_map, const int32_t* row_map,
                        const int32_t* var_recombine, const int32_t* var_phase, const int32_t* eq_differential,
                        const int32_t* eq_phase, int nbc, const int32_t* bc_rows, const double* bc_values) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  if (pr->uploaded) return fail(ctx, SP_ERR_STATE, "layout is fixed once the problem is on the device");
  if (!col_map || !row_map || !var_recombine || !var_phase || !eq_differential || !eq_phase ||
      (nbc > 0 && (!bc_rows || !bc_values)))
    return fail(ctx, SP_ERR_ARG, "null argument");
  const int S = pr->S, Nz = pr->Nz, n = pr->n;
  if (nbc < 0 || nbc > n) return fail(ctx, SP_ERR_ARG, "bad nbc");
  std::vector<int> seen_c(n, 0), seen_r(n, 0);
  for (int i = 0; i < S * Nz; ++i) {
    if (col_map[i] < 0 || col_map[i] >= n || seen_c[col_map[i]]++)
      return fail(ctx, SP_ERR_ARG, "col_map is not a permutation of [0, n)");
    if (row_map[i] >= n || row_map[i] < -1) return fail(ctx, SP_ERR_ARG, "row_map entry out of range");
    if (row_map[i] >= 0 && seen_r[row_map[i]]++) return fail(ctx, SP_ERR_ARG, "row_map repeats a row");
  }
  for (int q = 0; q < nbc; ++q) {
    if (bc_rows[q] < 0 || bc_rows[q] >= n || seen_r[bc_rows[q]]++)
      return fail(ctx, SP_ERR_ARG, "bc_rows overlap the equation rows or repeat");
  }
  for (int r = 0; r < n; ++r)
    if (!seen_r[r]) return fail(ctx, SP_ERR_ARG, "row %d receives neither an equation nor a boundary row", r);
  for (int e = 0; e < S; ++e)
    if (eq_differential[e]) {
      // the last row of a differential equation is its tau row
      if (row_map[e * Nz + Nz - 1] != -1)
        return fail(ctx, SP_ERR_ARG, "differential equation %d keeps its last (tau) row", e);
    }
  pr->col_map.assign(col_map, col_map + S * Nz);
  pr->row_map.assign(row_map, row_map + S * Nz);
  pr->var_rec.assign(var_recombine, var_recombine + S);
  pr->var_ph.assign(var_phase, var_phase + S);
  pr->eq_diff.assign(eq_differential, eq_differential + S);
  pr->eq_ph.assign(eq_phase, eq_phase + S);
  pr->nbc = nbc;
  pr->bc_rows.assign(bc_rows, bc_rows + nbc);
  pr->bc_values.assign(bc_values, bc_values + (size_t)2 * nbc * pr->P);
  pr->has_layout = true;
  return SP_OK;
}

sp_status sp_set_pencils(sp_ctx* ctx, int problem, int64_t first_pencil, int64_t count, int n, int64_t nnz,
                         const int32_t* indptr, const int32_t* indices, const double* M_values,
                         const double* L_values) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  if (pr->uploaded) return fail(ctx, SP_ERR_STATE, "pencils are fixed once the problem is on the device");
  if (n != pr->n) return fail(ctx, SP_ERR_ARG, "n = %d but S * N_z = %d", n, pr->n);
  if (first_pencil < 0 || count < 1 || first_pencil + count > pr->P)
    return fail(ctx, SP_ERR_ARG, "pencil range out of [0, P)");
  if (!indptr || !indices || !M_values || !L_values) return fail(ctx, SP_ERR_ARG, "null argument");
  if (nnz < 1 || indptr[0] != 0 || indptr[n] != nnz) return fail(ctx, SP_ERR_ARG, "indptr inconsistent with nnz");
  int kl = 0, ku = 0;
  for (int r = 0; r < n; ++r) {
    if (indptr[r + 1] < indptr[r]) return fail(ctx, SP_ERR_ARG, "indptr not monotone");
    for (int e = indptr[r]; e < indptr[r + 1]; ++e) {
      const int c = indices[e];
      if (c < 0 || c >= n) return fail(ctx, SP_ERR_ARG, "column index out of range");
      if (e > indptr[r] && c <= indices[e - 1]) return fail(ctx, SP_ERR_ARG, "row %d indices not sorted/unique", r);
      kl = std::max(kl, r - c);
      ku = std::max(ku, c - r);
    }
  }
  if (kl > 31) return fail(ctx, SP_ERR_ARG, "lower band width %d > 31 is not supported", kl);
  if (kl + ku > 63) return fail(ctx, SP_ERR_ARG, "kl + ku = %d > 63 is not supported", kl + ku);
  if (pr->nnz < 0) {
    pr->nnz = nnz;
    pr->indptr.assign(indptr, indptr + n + 1);
    pr->indices.assign(indices, indices + nnz);
    pr->Mv.assign((size_t)pr->P * nnz, 0.0);
    pr->Lv.assign((size_t)pr->P * nnz, 0.0);
    pr->kl = kl;
    pr->ku = ku;
  } else {
    if (nnz != pr->nnz || std::memcmp(indptr, pr->indptr.data(), (n + 1) * sizeof(int32_t)) ||
        std::memcmp(indices, pr->indices.data(), nnz * sizeof(int32_t)))
      return fail(ctx, SP_ERR_ARG, "all pencils must share one CSR pattern");
  }
  std::memcpy(pr->Mv.data() + first_pencil * nnz, M_values, (size_t)count * nnz * sizeof(double));
  std::memcpy(pr->Lv.data() + first_pencil * nnz, L_values, (size_t)count * nnz * sizeof(double));
  for (int64_t p = first_pencil; p < first_pencil + count; ++p) pr->pset[p] = 1;
  return SP_OK;
}

sp_status sp_set_bilinear_rhs(sp_ctx* ctx, int problem, int nterms, const int32_t* eq, const double* coef,
                              const int32_t* op_a, const int32_t* var_a, const int32_t* op_b,
                              const int32_t* var_b) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  if (pr->uploaded) return fail(ctx, SP_ERR_STATE, "the right-hand side is fixed once the problem is on the device");
  if (nterms < 0 || (nterms > 0 && (!eq || !coef || !op_a || !var_a || !op_b || !var_b)))
    return fail(ctx, SP_ERR_ARG, "null argument");
  pr->t_slot.clear(); pr->t_fa.clear(); pr->t_fb.clear(); pr->t_coef.clear();
  pr->gfields.clear(); pr->nl_eqs.clear();
  auto field = [&](int op, int var) {
    for (size_t i = 0; i < pr->gfields.size(); ++i)
      if (pr->gfields[i].op == op && pr->gfields[i].var == var) return (int)i;
    pr->gfields.push_back(GridField{var, op});
    return (int)pr->gfields.size() - 1;
  };
  for (int t = 0; t < nterms; ++t) {
    if (eq[t] < 0 || eq[t] >= pr->S || var_a[t] < 0 || var_a[t] >= pr->S || var_b[t] < 0 || var_b[t] >= pr->S)
      return fail(ctx, SP_ERR_ARG, "term %d: index out of range", t);
    auto op_ok = [&](int op) { return op == SP_OP_ID || op == SP_OP_DX || (op == SP_OP_DY && pr->ndim == 3); };
    if (!op_ok(op_a[t]) || !op_ok(op_b[t]))
      return fail(ctx, SP_ERR_ARG, "term %d: unknown operator (DY needs a 3D problem)", t);
    int slot = -1;
    for (size_t i = 0; i < pr->nl_eqs.size(); ++i)
      if (pr->nl_eqs[i] == eq[t]) slot = (int)i;
    if (slot < 0) { pr->nl_eqs.push_back(eq[t]); slot = (int)pr->nl_eqs.size() - 1; }
    pr->t_slot.push_back(slot);
    pr->t_coef.push_back(coef[t]);
    pr->t_fa.push_back(field(op_a[t], var_a[t]));
    pr->t_fb.push_back(field(op_b[t], var_b[t]));
  }
  if (pr->gfields.size() > 16) return fail(ctx, SP_ERR_ARG, "at most 16 distinct grid fields");
  if (nterms > 16) return fail(ctx, SP_ERR_ARG, "at most 16 bilinear terms");
  // the product kernel sums each equation's terms in one run: order the
  // terms by slot (stable, so terms of one equation keep their order)
  {
    std::vector<int> order(pr->t_slot.size());
    for (size_t t = 0; t < order.size(); ++t) order[t] = (int)t;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return pr->t_slot[x] < pr->t_slot[y]; });
    std::vector<int32_t> sl, fa, fb;
    std::vector<double> cf;
    for (int t : order) {
      sl.push_back(pr->t_slot[t]); fa.push_back(pr->t_fa[t]); fb.push_back(pr->t_fb[t]); cf.push_back(pr->t_coef[t]);
    }
    pr->t_slot = sl; pr->t_fa = fa; pr->t_fb = fb; pr->t_coef = cf;
  }
  return SP_OK;
}

// Banded LU of alpha_f M~ + beta_f L~ into factor slots f < nf for every
// pencil (and, per solve kernel, the lane layout or the partitioned
// substitution's coupling matrices); synchronous.
static sp_status factor_matrices(sp_ctx* ctx, Problem* pr, int nf, const double (*ab)[2]) {
  CK(reset_spike_guess(pr, ctx->stream));
  const int ldab = 2 * pr->kl + pr->ku + 1;
  double* work = nullptr;
  CK(dalloc(&work, (size_t)pr->P * pr->n * ldab));
  for (int f = 0; f < nf; ++f) {
    pr->fac[f].alpha = ab[f][0];
    pr->fac[f].beta = ab[f][1];
    cudaError_t e = launch_band_factor(ctx->stream, pr->P, pr->n, (int)pr->nnz, pr->kl, pr->ku, pr->d_indptr,
                                       pr->d_indices, pr->d_Mv, pr->d_Lv, ab[f][0], ab[f][1], work, pr->fac[f],
                                       pr->npad, pr->lpad, pr->upad, ctx->d_status);
    if (e != cudaSuccess) { cudaFree(work); CK(e); }
    if (pr->spike) {
      e = launch_spike_coupling(ctx->stream, pr->P, pr->npad, pr->nblk_f, pr->nblk, pr->kl, pr->kl + pr->ku,
                                pr->lpad, pr->upad, pr->fac[f]);
      if (e != cudaSuccess) { cudaFree(work); CK(e); }
    }
    if (pr->lanes) {
      // lane layout: the union pattern of U over pencils, then the copy with
      // only the listed entries
      BandFactor& bf = pr->fac[f];
      e = cudaMemsetAsync(bf.umask, 0, (size_t)pr->n * sizeof(unsigned long long), ctx->stream);
      if (e == cudaSuccess)
        e = launch_u_mask(ctx->stream, pr->P, pr->n, pr->npad, pr->kl + pr->ku, pr->upad, bf.U, bf.umask);
      std::vector<unsigned long long> hm(pr->n);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(hm.data(), bf.umask, hm.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                            ctx->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
      if (e != cudaSuccess) { cudaFree(work); CK(e); }
      int cmax = 1;
      double listed = 0;
      for (unsigned long long m : hm) {
        cmax = std::max(cmax, __builtin_popcountll(m));
        listed += __builtin_popcountll(m) - 1;
      }
      bf.u_listed = listed / pr->n;
      if (cmax != bf.cmax || !bf.Ug) {
        if (bf.Ug) cudaFree(bf.Ug);
        bf.Ug = nullptr;
        const size_t ngroups = (pr->P + LANE_GROUP - 1) / LANE_GROUP;
        e = cudaMalloc((void**)&bf.Ug, ngroups * pr->n * cmax * LANE_GROUP * sizeof(double));
        if (e != cudaSuccess) { cudaFree(work); CK(e); }
        bf.cmax = cmax;
      }
      e = launch_factor_relayout(ctx->stream, pr->P, pr->n, pr->npad, pr->kl, pr->kl + pr->ku, pr->lpad, pr->upad,
                                 bf);
      if (e != cudaSuccess) { cudaFree(work); CK(e); }
    }
  }
  cudaError_t e = cudaStreamSynchronize(ctx->stream);
  cudaFree(work);
  CK(e);
  return SP_OK;
}

sp_status sp_factor(sp_ctx* ctx, int problem, double dt) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(ctx, SP_ERR_ARG, "dt must be positive and finite");
  CK(cudaSetDevice(ctx->device));
  sp_status st = upload_problem(ctx, pr);
  if (st != SP_OK) return st;
  double ab[4][2];
  int nf = 1;
  if (is_rk(pr->scheme)) {
    const Tableau tb = make_tableau(pr->scheme);
    ab[0][0] = 1.0; ab[0][1] = dt * tb.H[1][1];   // every stage: H_ii = H_11
  } else if (is_cnab(pr->scheme)) {
    ab[0][0] = 1.0; ab[0][1] = 0.5 * dt;         // both orders: M + dt/2 L
  } else {
    // SBDFq: the matrices a_0 M + dt L of the start-up orders 1 .. q
    nf = sbdf_order(pr->scheme);
    for (int f = 0; f < nf; ++f) { ab[f][0] = SBDF_A[f + 1][0]; ab[f][1] = dt; }
  }
  sp_status fst = factor_matrices(ctx, pr, nf, ab);
  if (fst != SP_OK) return fst;
  pr->lbvp_factored = false;
  pr->nfac = nf;
  pr->fac_dt = dt;
  pr->factored = true;
  for (auto& kv : pr->graphs) cudaGraphExecDestroy(kv.second);
  pr->graphs.clear();
  drop_batches(ctx, problem);
  return SP_OK;
}

sp_status sp_solve_lbvp(sp_ctx* ctx, int problem, int nslots, const int32_t* eqs, const void* F_host) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  if (nslots < 0 || nslots > pr->S || (nslots > 0 && (!eqs || !F_host)))
    return fail(ctx, SP_ERR_ARG, "bad right-hand-side slots");
  for (int q = 0; q < nslots; ++q)
    if (eqs[q] < 0 || eqs[q] >= pr->S) return fail(ctx, SP_ERR_ARG, "bad equation index %d", eqs[q]);
  CK(cudaSetDevice(ctx->device));
  sp_status st = upload_problem(ctx, pr);
  if (st != SP_OK) return st;
  cudaStream_t s = ctx->stream;
  if (!pr->lbvp_factored) {
    // L~ alone in the first factor slot: any stepping factorization is gone
    pr->factored = false;
    for (auto& kv : pr->graphs) cudaGraphExecDestroy(kv.second);
    pr->graphs.clear();
    drop_batches(ctx, problem);
    const double ab[1][2] = {{0.0, 1.0}};
    if ((st = factor_matrices(ctx, pr, 1, ab)) != SP_OK) return st;
    pr->lbvp_factored = true;
  }
  if (nslots > pr->lb_cap) {
    cudaFree(pr->d_lb_F);
    cudaFree(pr->d_lb_eq);
    pr->d_lb_F = nullptr;
    pr->d_lb_eq = nullptr;
    pr->lb_cap = 0;
    CK(dalloc(&pr->d_lb_F, (size_t)nslots * pr->P * pr->Nz));
    CK(dalloc(&pr->d_lb_eq, (size_t)nslots));
    pr->lb_cap = nslots;
  }
  if (nslots > 0) {
    CK(cudaMemcpyAsync(pr->d_lb_F, F_host, (size_t)nslots * pr->P * pr->Nz * sizeof(double2),
                       cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(pr->d_lb_eq, eqs, (size_t)nslots * sizeof(int32_t), cudaMemcpyHostToDevice, s));
  }
  // B~ = P^L F (tau rows dropped) + boundary values; X~ = L~^-1 B~; X = P^R X~
  SolveArgs a = base_args(pr, ctx, 0);
  a.nvec = 0;
  a.mv_x = nullptr;
  a.nfc = nslots > 0 ? 1 : 0;
  a.fc[0] = pr->d_lb_F; a.fc_coef[0] = 1.0;
  a.nl_eq = pr->d_lb_eq; a.n_nl = nslots;
  a.bc_coef = 1.0;
  a.xc_out = pr->d_Xc;
  a.xt_out = pr->d_Xt;
  a.ep_mv_vals = nullptr;
  if ((st = solve(ctx, pr, s, a)) != SP_OK) return st;
  CK(cudaStreamSynchronize(s));
  pr->xt_valid = true;
  pr->mx_valid = false;
  pr->iteration = 0;
  pr->xc32_valid = pr->prec != 0;     // the epilogue wrote the FP32 copies too
  pr->xs32_valid = pr->zmma;
  return SP_OK;
}

sp_status sp_set_field(sp_ctx* ctx, int problem, int var, const void* data, int on_device, char layout) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  if (var < 0 || var >= pr->S || !data) return fail(ctx, SP_ERR_ARG, "bad variable or null data");
  CK(cudaSetDevice(ctx->device));
  sp_status st = upload_problem(ctx, pr);
  if (st != SP_OK) return st;
  cudaStream_t s = ctx->stream;
  CK(reset_spike_guess(pr, s));                  // a run from a set state starts from zero inflows
  double2* dst = pr->d_Xc + (size_t)var * pr->P * pr->Nz;
  const size_t ncoef = (size_t)pr->P * pr->Nz;
  if (layout == 'c') {
    CK(cudaMemcpyAsync(dst, data, ncoef * sizeof(double2),
                       on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  } else if (layout == 'g') {
    // set-up transforms run in FP64 in every precision mode: an initial
    // state carries small perturbations on an O(1) background
    TransformPlan *px, *pz, *py = nullptr;
    if ((st = make_plan(ctx, pr, pr->Nx, pr->Nx, &px)) != SP_OK) return st;
    if ((st = make_plan(ctx, pr, pr->Nz, pr->Nz, &pz)) != SP_OK) return st;
    if (pr->ndim == 3 && (st = make_plan(ctx, pr, pr->Ny, pr->Ny, &py)) != SP_OK) return st;
    const size_t ng = (size_t)pr->Nz * pr->Ny * pr->Nx;
    double* grid = nullptr;
    double2 *m1 = nullptr, *m2 = nullptr;
    const size_t nm = grid_scratch_elems(pr, 1, pr->Ny, pr->Nz);
    CK(dalloc(&grid, ng));
    CK(dalloc(&m1, nm));
    CK(dalloc(&m2, nm));
    CK(cudaMemcpyAsync(grid, data, ng * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    CK(grid_to_coef(pr, s, 0, 1, *px, py, *pz, pr->Ny, pr->Nz, grid, dst, m1, m2));
    CK(cudaStreamSynchronize(s));
    cudaFree(grid);
    cudaFree(m1);
    cudaFree(m2);
  } else {
    return fail(ctx, SP_ERR_ARG, "layout must be 'c' or 'g'");
  }
  CK(cudaGetLastError());
  pr->xt_valid = false;
  pr->mx_valid = false;
  pr->xc32_valid = false;
  pr->xs32_valid = false;
  pr->iteration = 0;
  return SP_OK;
}

sp_status sp_get_field(sp_ctx* ctx, int problem, int var, void* data, int on_device, char layout) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  if (var < 0 || var >= pr->S || !data) return fail(ctx, SP_ERR_ARG, "bad variable or null data");
  if (!pr->uploaded) return fail(ctx, SP_ERR_STATE, "no state on the device yet");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  const double2* src = pr->d_Xc + (size_t)var * pr->P * pr->Nz;
  const size_t ncoef = (size_t)pr->P * pr->Nz;
  if (layout == 'c') {
    CK(cudaMemcpyAsync(data, src, ncoef * sizeof(double2), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
  } else if (layout == 'g') {
    TransformPlan *px, *pz, *py = nullptr;
    sp_status st;
    if ((st = make_plan(ctx, pr, pr->Nx, pr->Nx, &px)) != SP_OK) return st;
    if ((st = make_plan(ctx, pr, pr->Nz, pr->Nz, &pz)) != SP_OK) return st;
    if (pr->ndim == 3 && (st = make_plan(ctx, pr, pr->Ny, pr->Ny, &py)) != SP_OK) return st;
    const size_t ng = (size_t)pr->Nz * pr->Ny * pr->Nx;
    double* grid = nullptr;
    double2 *m1 = nullptr, *m2 = nullptr;
    const size_t nm = grid_scratch_elems(pr, 1, pr->Ny, pr->Nz);
    CK(dalloc(&grid, ng));
    CK(dalloc(&m1, nm));
    CK(dalloc(&m2, nm));
    CK(coef_to_grid(pr, s, 0, 1, *px, py, *pz, pr->Ny, pr->Nz, pr->d_ident + var, pr->d_Xc, pr->P * pr->Nz,
                    nullptr, grid, m1, m2));
    CK(cudaMemcpyAsync(data, grid, ng * sizeof(double), on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    cudaFree(grid);
    cudaFree(m1);
    cudaFree(m2);
  } else {
    return fail(ctx, SP_ERR_ARG, "layout must be 'c' or 'g'");
  }
  return SP_OK;
}

sp_status sp_dz(sp_ctx* ctx, int problem, int src_var, int dst_var) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  if (src_var < 0 || src_var >= pr->S || dst_var < 0 || dst_var >= pr->S || src_var == dst_var)
    return fail(ctx, SP_ERR_ARG, "bad variables");
  if (!pr->uploaded) return fail(ctx, SP_ERR_STATE, "no state on the device yet");
  CK(cudaSetDevice(ctx->device));
  const size_t f = (size_t)pr->P * pr->Nz;
  CK(launch_dz(ctx->stream, pr->P, pr->Nz, 2.0 / (pr->zb - pr->za), pr->d_Xc + src_var * f, pr->d_Xc + dst_var * f));
  pr->xt_valid = false;
  pr->xc32_valid = false;
  pr->xs32_valid = false;
  pr->mx_valid = false;
  pr->iteration = 0;
  return SP_OK;
}

sp_status sp_step(sp_ctx* ctx, int problem, double dt, int nsteps) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  if (nsteps < 0) return fail(ctx, SP_ERR_ARG, "nsteps < 0");
  if (!pr->factored || dt != pr->fac_dt)
    return fail(ctx, SP_ERR_NOT_FACTORED, "dt = %.17g is not the factored step size", dt);
  CK(cudaSetDevice(ctx->device));
  for (int k = 0; k < nsteps; ++k) {
    sp_status st = one_step(ctx, pr, ctx->stream, dt);
    if (st != SP_OK) return st;
  }
  return SP_OK;
}

sp_status sp_step_graph(sp_ctx* ctx, int problem, double dt, int nsteps) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  if (nsteps < 0) return fail(ctx, SP_ERR_ARG, "nsteps < 0");
  if (!pr->factored || dt != pr->fac_dt)
    return fail(ctx, SP_ERR_NOT_FACTORED, "dt = %.17g is not the factored step size", dt);
  CK(cudaSetDevice(ctx->device));
  int left = nsteps;
  // warm-up steps that change the buffer schedule run eagerly
  while (left > 0 && (!pr->xt_valid || !pr->mx_valid ||
                      (sbdf_order(pr->scheme) > 1 && pr->iteration < sbdf_order(pr->scheme) - 1))) {
    sp_status st = one_step(ctx, pr, ctx->stream, dt);
    if (st != SP_OK) return st;
    --left;
  }
  const bool timing = pr->timing;
  pr->timing = false;  // event nodes are not recorded inside graphs
  while (left > 0) {
    const int block = std::min(left, 16);
    const int parity = sbdf_order(pr->scheme) > 0 ? pr->iteration % sbdf_depth(pr->scheme) : 0;
    auto key = std::make_tuple(block, parity, pr->scheme, dt);
    cudaGraphExec_t exec = nullptr;
    auto it = pr->graphs.find(key);
    const int it0 = pr->iteration;
    if (it == pr->graphs.end()) {
      cudaGraph_t g;
      CK(cudaStreamBeginCapture(ctx->capture, cudaStreamCaptureModeThreadLocal));
      sp_status st = SP_OK;
      for (int k = 0; k < block && st == SP_OK; ++k) st = one_step(ctx, pr, ctx->capture, dt);
      cudaError_t e = cudaStreamEndCapture(ctx->capture, &g);
      if (st != SP_OK) { pr->timing = timing; return st; }
      CK(e);
      CK(cudaGraphInstantiate(&exec, g, 0));
      cudaGraphDestroy(g);
      pr->graphs[key] = exec;
    } else {
      exec = it->second;
      pr->iteration = it0 + block;
    }
    CK(cudaGraphLaunch(exec, ctx->stream));
    left -= block;
  }
  pr->timing = timing;
  return SP_OK;
}

sp_status sp_step_batched(sp_ctx* ctx, int nproblems, const int* problem_ids, const double* dts, int nsteps,
                          int use_graph) {
  if (!ctx) return SP_ERR_ARG;
  ctx->err.clear();
  if (nproblems < 1 || !problem_ids || !dts || nsteps < 0) return fail(ctx, SP_ERR_ARG, "bad arguments");
  std::vector<int> ids(problem_ids, problem_ids + nproblems);
  std::vector<Problem*> ps;
  for (int q = 0; q < nproblems; ++q) {
    Problem* pr = get(ctx, ids[q]);
    if (!pr) return fail(ctx, SP_ERR_ARG, "bad problem id %d", ids[q]);
    for (int r = 0; r < q; ++r)
      if (ids[r] == ids[q]) return fail(ctx, SP_ERR_ARG, "problem %d listed twice", ids[q]);
    if (!pr->factored || dts[q] != pr->fac_dt)
      return fail(ctx, SP_ERR_NOT_FACTORED, "problem %d: dt = %.17g is not its factored step size", ids[q], dts[q]);
    if (pr->nl_eqs.empty()) return fail(ctx, SP_ERR_ARG, "problem %d has no bilinear right-hand side", ids[q]);
    if (pr->ndim != 2) return fail(ctx, SP_ERR_ARG, "problem %d: batched stepping takes 2D problems", ids[q]);
    ps.push_back(pr);
  }
  for (Problem* pr : ps)
    if (pr->scheme != ps[0]->scheme || pr->prec != ps[0]->prec)
      return fail(ctx, SP_ERR_ARG, "all problems of a batch need the same scheme and precision");
  CK(cudaSetDevice(ctx->device));
  sp_status st;
  // eager steps until every problem is in its steady schedule (multistep
  // schemes: past their lower-order start-up steps)
  const int order = sbdf_order(ps[0]->scheme);
  auto steady = [&](Problem* pr) {
    return pr->xt_valid && pr->mx_valid && (order == 0 || pr->iteration >= order - 1);
  };
  while (nsteps > 0 && !std::all_of(ps.begin(), ps.end(), steady)) {
    for (Problem* pr : ps)
      if ((st = one_step(ctx, pr, ctx->stream, pr->fac_dt)) != SP_OK) return st;
    --nsteps;
  }
  if (nsteps == 0) return SP_OK;
  // multistep schemes rotate their history rings: the buffers a step uses
  // depend on its phase, iteration mod the ring depth D (one batch per phase)
  const bool multistep = order > 0;
  const int D = multistep ? sbdf_depth(ps[0]->scheme) : 1;
  for (Problem* pr : ps)
    if (multistep && pr->iteration % D != ps[0]->iteration % D)
      return fail(ctx, SP_ERR_STATE, "problems of a batch must be at the same step phase (iteration mod %d)", D);
  // tile autotuning of the z-transform kernels (first call for these ids)
  auto get_batch = [&](int parity, int tile, bool persist) -> Batch* {
    auto key = std::make_pair(ids, parity);
    auto it = ctx->batches.find(key);
    if (it != ctx->batches.end() && it->second->tile == tile && it->second->persist == persist) return it->second;
    if (it != ctx->batches.end()) { free_batch(it->second); delete it->second; ctx->batches.erase(it); }
    Batch* b = new Batch();
    if (build_batch(ctx, ps, ids, tile, parity, persist, b) != SP_OK) { free_batch(b); delete b; return nullptr; }
    ctx->batches[key] = b;
    return b;
  };
  if (!ctx->batch_tile.count(ids)) {
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    int best = 8;
    float best_ms = 1e30f;
    for (int tile : {4, 8, 16}) {
      Batch* b = get_batch(multistep ? ps[0]->iteration % D : 0, tile, false);
      if (!b) return fail(ctx, SP_ERR_CUDA, "building batch: %s", ctx->err.c_str());
      // the transform kernels write only scratch buffers that the next step overwrites
      const BatchStage& sg = b->stages[0];
      float tot = 0;
      for (int rep = 0; rep < 4; ++rep) {
        CK(cudaEventRecord(e0, ctx->stream));
        CK(launch_cheb_backward_batched(ctx->stream, b->prec, tile, sg.d_zb, b->d_wzb, b->nzb, b->max_ngz));
        CK(launch_cheb_forward_batched(ctx->stream, b->prec, tile, sg.d_zf, b->d_wzf, b->nzf, b->max_ngz));
        CK(cudaEventRecord(e1, ctx->stream));
        CK(cudaEventSynchronize(e1));
        float ms;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) tot += ms;
      }
      if (tot < best_ms) { best_ms = tot; best = tile; }
    }
    // launch shape: one CTA per work item, or persistent grids pulling the
    // items from device counters.  A batch step of each is timed; every
    // buffer a step writes (states, history rings, right-hand-side slots)
    // is copied aside first and restored afterwards, so the timing leaves
    // the problems exactly as they were.
    std::vector<std::pair<void*, size_t>> bufs;
    for (Problem* pr : ps) {
      const size_t nvec = (size_t)pr->P * pr->n * sizeof(double2);
      const size_t nfc = (size_t)std::max<int>(1, (int)pr->nl_eqs.size()) * pr->P * pr->Nz * sizeof(double2);
      bufs.push_back({pr->d_Xt, nvec});
      bufs.push_back({pr->d_Xc, nvec});
      if (pr->d_Xc32) bufs.push_back({pr->d_Xc32, (size_t)pr->P * pr->n * sizeof(float2)});
      for (double2* b : pr->d_MX) if (b) bufs.push_back({b, nvec});
      for (double2* b : pr->d_LX) if (b) bufs.push_back({b, nvec});
      for (double2* b : pr->d_Fc) if (b) bufs.push_back({b, nfc});
      if (pr->zmma) bufs.push_back({pr->cm.xs32, (size_t)pr->S * 2 * pr->P * pr->Nz * sizeof(float)});
    }
    size_t total = 0;
    for (auto& b : bufs) total += b.second;
    char* backup = nullptr;
    CK(cudaMalloc(&backup, total));
    size_t off = 0;
    for (auto& b : bufs) {
      CK(cudaMemcpyAsync(backup + off, b.first, b.second, cudaMemcpyDeviceToDevice, ctx->stream));
      off += b.second;
    }
    bool best_persist = false;
    float shape_ms[2] = {1e30f, 1e30f};
    for (int pm = 0; pm < 2; ++pm) {
      Batch* b = get_batch(multistep ? ps[0]->iteration % D : 0, best, pm == 1);
      if (!b) return fail(ctx, SP_ERR_CUDA, "building batch: %s", ctx->err.c_str());
      float tot = 0;
      for (int rep = 0; rep < 3; ++rep) {
        CK(cudaEventRecord(e0, ctx->stream));
        if ((st = batch_step(ctx, b, ctx->stream)) != SP_OK) return st;
        CK(cudaEventRecord(e1, ctx->stream));
        CK(cudaEventSynchronize(e1));
        float ms;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0) tot += ms;
      }
      shape_ms[pm] = tot;
    }
    best_persist = shape_ms[1] < shape_ms[0];
    auto fixed = ctx->batch_persist_fixed.find(ids);
    if (fixed != ctx->batch_persist_fixed.end()) best_persist = fixed->second;
    off = 0;
    for (auto& b : bufs) {
      CK(cudaMemcpyAsync(b.first, backup + off, b.second, cudaMemcpyDeviceToDevice, ctx->stream));
      off += b.second;
    }
    CK(cudaStreamSynchronize(ctx->stream));
    cudaFree(backup);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->batch_tile[ids] = best;
    ctx->batch_persist[ids] = best_persist;
  }
  const int tile = ctx->batch_tile[ids];
  const bool persist = ctx->batch_persist[ids];
  while (nsteps > 0) {
    const int parity = multistep ? ps[0]->iteration % D : 0;
    Batch* b = get_batch(parity, tile, persist);
    if (!b) return fail(ctx, SP_ERR_CUDA, "building batch: %s", ctx->err.c_str());
    if (!use_graph) {
      if ((st = batch_step(ctx, b, ctx->stream)) != SP_OK) return st;
      for (Problem* pr : ps) commit_step(pr);
      --nsteps;
      continue;
    }
    // a graph of `block` steps starting at this phase (phases cycle mod D)
    const int block = std::min(nsteps, 16);
    auto git = b->graphs.find(block);
    cudaGraphExec_t exec = nullptr;
    if (git == b->graphs.end()) {
      std::vector<Batch*> phase_batch(D, nullptr);
      for (int q = 0; q < D; ++q) {
        phase_batch[q] = q == parity ? b : get_batch(q, tile, persist);
        if (!phase_batch[q]) return fail(ctx, SP_ERR_CUDA, "building batch: %s", ctx->err.c_str());
      }
      cudaGraph_t g;
      CK(cudaStreamBeginCapture(ctx->capture, cudaStreamCaptureModeThreadLocal));
      st = SP_OK;
      for (int k = 0; k < block && st == SP_OK; ++k) st = batch_step(ctx, phase_batch[(parity + k) % D], ctx->capture);
      cudaError_t e = cudaStreamEndCapture(ctx->capture, &g);
      if (st != SP_OK) return st;
      CK(e);
      CK(cudaGraphInstantiate(&exec, g, 0));
      cudaGraphDestroy(g);
      b->graphs[block] = exec;
    } else {
      exec = git->second;
    }
    CK(cudaGraphLaunch(exec, ctx->stream));
    for (int k = 0; k < block; ++k)
      for (Problem* pr : ps) commit_step(pr);
    nsteps -= block;
  }
  return SP_OK;
}

sp_status sp_batch_tile(sp_ctx* ctx, int nproblems, const int* problem_ids, int* tile) {
  if (!ctx || nproblems < 1 || !problem_ids || !tile) return SP_ERR_ARG;
  std::vector<int> ids(problem_ids, problem_ids + nproblems);
  auto it = ctx->batch_tile.find(ids);
  if (it == ctx->batch_tile.end()) return fail(ctx, SP_ERR_STATE, "no batch step has run for these problems");
  *tile = it->second;
  return SP_OK;
}

sp_status sp_set_batch_persistent(sp_ctx* ctx, int nproblems, const int* problem_ids, int mode) {
  if (!ctx || nproblems < 1 || !problem_ids || mode < -1 || mode > 1) return SP_ERR_ARG;
  std::vector<int> ids(problem_ids, problem_ids + nproblems);
  if (mode < 0) ctx->batch_persist_fixed.erase(ids);
  else ctx->batch_persist_fixed[ids] = mode == 1;
  // the next batched step decides (or applies) the shape again
  ctx->batch_tile.erase(ids);
  ctx->batch_persist.erase(ids);
  return SP_OK;
}

sp_status sp_batch_persistent(sp_ctx* ctx, int nproblems, const int* problem_ids, int* persistent) {
  if (!ctx || nproblems < 1 || !problem_ids || !persistent) return SP_ERR_ARG;
  std::vector<int> ids(problem_ids, problem_ids + nproblems);
  auto it = ctx->batch_persist.find(ids);
  if (it == ctx->batch_persist.end()) return fail(ctx, SP_ERR_STATE, "no batch step has run for these problems");
  *persistent = it->second ? 1 : 0;
  return SP_OK;
}

sp_status sp_adjoint_init(sp_ctx* ctx, int problem) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  if (pr->scheme != SP_RK222 && pr->scheme != SP_RK111)
    return fail(ctx, SP_ERR_ARG, "the adjoint step is provided for the RK222 and RK111 schemes");
  if (pr->ndim != 2) return fail(ctx, SP_ERR_ARG, "the adjoint step is provided for 2D problems");
  if (!pr->factored) return fail(ctx, SP_ERR_STATE, "sp_factor must come before sp_adjoint_init");
  if (pr->nl_eqs.empty()) return fail(ctx, SP_ERR_ARG, "the problem has no bilinear right-hand side");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  const int n = pr->n;
  const int64_t nnz = pr->nnz;
  if (!pr->adj_ready) {
    // CSR of the transposed pencils (same pattern for every pencil)
    std::vector<int32_t> ipT(n + 1, 0), ixT(nnz);
    std::vector<int64_t> where(nnz);
    for (int64_t e = 0; e < nnz; ++e) ipT[pr->indices[e] + 1]++;
    for (int r = 0; r < n; ++r) ipT[r + 1] += ipT[r];
    std::vector<int32_t> fill(ipT.begin(), ipT.end() - 1);
    for (int r = 0; r < n; ++r)
      for (int e = pr->indptr[r]; e < pr->indptr[r + 1]; ++e) {
        const int c = pr->indices[e];
        ixT[fill[c]] = r;
        where[fill[c]] = e;
        fill[c]++;
      }
    std::vector<double> MT((size_t)pr->P * nnz), LT((size_t)pr->P * nnz);
    for (int p = 0; p < pr->P; ++p)
      for (int64_t k = 0; k < nnz; ++k) {
        MT[(size_t)p * nnz + k] = pr->Mv[(size_t)p * nnz + where[k]];
        LT[(size_t)p * nnz + k] = pr->Lv[(size_t)p * nnz + where[k]];
      }
    CK(upload(&pr->d_indptrT, ipT, s));
    CK(upload(&pr->d_indicesT, ixT, s));
    CK(upload(&pr->d_MvT, MT, s));
    CK(upload(&pr->d_LvT, LT, s));
    pr->klT = pr->ku;
    pr->kuT = pr->kl;
    if (pr->klT > 31) return fail(ctx, SP_ERR_ARG, "transposed lower band width %d > 31", pr->klT);
    pr->lpadT = std::max(2, (pr->klT + 1) / 2 * 2);
    CK(dalloc(&pr->facT.L, (size_t)pr->P * pr->npad * pr->lpadT));
    CK(dalloc(&pr->facT.piv, (size_t)pr->P * pr->npad));
    CK(dalloc(&pr->facT.U, (size_t)pr->P * pr->npad * pr->upad));
    CK(dalloc(&pr->facT.rd, (size_t)pr->P * pr->npad));
    const size_t nvec = (size_t)pr->P * n;
    for (auto& b : pr->d_mu) CK(dalloc(&b, nvec));
    CK(dalloc(&pr->d_LTmu, nvec));
    CK(dalloc(&pr->d_MTmu, nvec));
    CK(dalloc(&pr->d_JF, nvec));
    CK(dalloc(&pr->d_lamx, nvec));
    const int nf = (int)pr->gfields.size(), ne = (int)pr->nl_eqs.size();
    CK(dalloc(&pr->d_Xbar, (size_t)nf * pr->P * pr->Nz));
    CK(dalloc(&pr->d_Fbar, (size_t)ne * pr->P * pr->Nz));
    if (pr->prec) CK(dalloc(&pr->d_Fbar32, (size_t)ne * pr->P * pr->Nz));
    CK(cudaMalloc(&pr->d_gzadj, (size_t)nf * pr->Ngz * pr->P * (pr->prec ? 8 : 16)));
    pr->adj_ready = true;
  }
  // factor A~^T = alpha M~^T + beta L~^T with the forward step's coefficients
  const int ldab = pr->klT + pr->klT + pr->kuT + 1;
  double* work = nullptr;
  CK(dalloc(&work, (size_t)pr->P * n * ldab));
  cudaError_t e = launch_band_factor(s, pr->P, n, (int)nnz, pr->klT, pr->kuT, pr->d_indptrT, pr->d_indicesT,
                                     pr->d_MvT, pr->d_LvT, pr->fac[0].alpha, pr->fac[0].beta, work, pr->facT,
                                     pr->npad, pr->lpadT, pr->upad, ctx->d_status);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(work);
  CK(e);
  pr->facT.alpha = pr->fac[0].alpha;
  pr->facT.beta = pr->fac[0].beta;
  // the transposed solves' back substitution is partitioned like the forward
  // solves' (kl' + ku' = kl + ku); their forward substitution stays whole-row,
  // since kl' = ku is wider than the partitioned forward windows
  const int kuuT = pr->klT + pr->kuT;
  if (pr->spike && pr->upad == 32 && spike_bwd_supported(kuuT, pr->npad, pr->nblk)) {
    if (!pr->facT.spE) CK(dalloc(&pr->facT.spE, (size_t)pr->P * pr->nblk * kuuT * 32));
    if (!pr->d_spT_u) CK(dalloc(&pr->d_spT_u, (size_t)pr->P * pr->nblk * 2 * 32));
    CK(cudaMemsetAsync(pr->d_spT_u, 0, (size_t)pr->P * pr->nblk * 2 * 32 * sizeof(double), s));
    CK(launch_spike_coupling_bwd(s, pr->P, pr->npad, pr->nblk, kuuT, pr->upad, pr->facT.U, pr->facT.spE));
    CK(cudaStreamSynchronize(s));
  }
  return SP_OK;
}

sp_status sp_step_adjoint(sp_ctx* ctx, int problem, double dt, const void* states_dev, int nstates,
                          void* lambda_dev) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  if (!pr->adj_ready || pr->facT.beta != pr->fac[0].beta)
    return fail(ctx, SP_ERR_STATE, "sp_adjoint_init must follow the last sp_factor");
  if (!pr->factored || dt != pr->fac_dt)
    return fail(ctx, SP_ERR_NOT_FACTORED, "dt = %.17g is not the factored step size", dt);
  if (!states_dev || !lambda_dev) return fail(ctx, SP_ERR_ARG, "null pointer");
  const Tableau tb = make_tableau(pr->scheme);
  if (nstates != 1 && nstates != tb.s)
    return fail(ctx, SP_ERR_ARG, "nstates = %d: expected 1 or the number of stages %d", nstates, tb.s);
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  sp_status st;
  const size_t ncoef = (size_t)pr->S * pr->P * pr->Nz;
  const double2* X0 = reinterpret_cast<const double2*>(states_dev);
  const double2* X1 = nullptr;                        // stage-1 state (two-stage scheme)
  // the problem's state buffers are scratch from here on
  pr->xt_valid = false;
  pr->xc32_valid = false;
  pr->xs32_valid = false;
  pr->mx_valid = false;
  pr->iteration = 0;
  if (tb.s == 2 && nstates == 2) {
    X1 = X0 + ncoef;
  } else if (tb.s == 2) {
    // forward recomputation of the first stage from X^n
    CK(cudaMemcpyAsync(pr->d_Xc, X0, ncoef * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    if ((st = ensure_solve_vars(ctx, pr, s)) != SP_OK) return st;
    if ((st = eval_rhs(ctx, pr, s, pr->d_Fc[0])) != SP_OK) return st;
    SolveArgs a = base_args(pr, ctx, 0);
    a.mv_x = pr->d_Xt; a.mv_coef = 1.0; a.mv_store = nullptr;
    set_mv_M(pr, a);
    a.fc[0] = pr->d_Fc[0]; a.fc_coef[0] = dt * tb.A[1][0]; a.nfc = 1;
    a.bc_coef = dt * tb.A[1][0];
    a.xc_out = pr->d_Xc;
    a.xc32_out = nullptr;
    if ((st = solve(ctx, pr, s, a)) != SP_OK) return st;
    X1 = pr->d_Xc;
  }
  // lambda^s in solve variables: T^H lambda_X
  {
    const double2* none[1] = {nullptr};
    double w0[1] = {0.0};
    CK(launch_adj_combine(s, pr->P, pr->Nz, pr->S, pr->n, pr->S, pr->d_ident, pr->d_zero, nullptr,
                          reinterpret_cast<const double2*>(lambda_dev), pr->d_col_map, pr->d_var_rec, pr->d_var_ph,
                          0, none, w0, pr->d_lamx));
  }
  // stage s: mu_s = A~^-T lambda^s ; keep L~^T mu_s (two stages) or M~^T mu_s
  {
    SolveArgs t = transposed_args(pr, ctx);
    t.vec[0] = pr->d_lamx; t.vec_coef[0] = 1.0; t.nvec = 1;
    t.xt_out = pr->d_mu[tb.s - 1];
    t.ep_mv_vals = tb.s == 2 ? pr->d_LvT : pr->d_MvT;
    t.ep_indptr = pr->d_indptrT; t.ep_indices = pr->d_indicesT; t.ep_nnz = (int)pr->nnz;
    t.ep_mv_store = tb.s == 2 ? pr->d_LTmu : pr->d_MTmu;
    if ((st = solve(ctx, pr, s, t)) != SP_OK) return st;
  }
  if (tb.s == 2) {
    // lambda^1 = dt A21 J_F(X^1)^H mu_2 - dt H21 L~^T mu_2
    const double2* v[1] = {pr->d_mu[1]};
    const double c[1] = {dt * tb.A[2][1]};
    const double2* ad[1] = {pr->d_LTmu};
    const double w[1] = {-dt * tb.H[2][1]};
    if ((st = adjoint_rhs(ctx, pr, s, X1, 1, v, c, 1, ad, w, pr->d_JF)) != SP_OK) return st;
    // mu_1 = A~^-T lambda^1 ; M~^T (mu_1 + mu_2)
    SolveArgs t = transposed_args(pr, ctx);
    t.vec[0] = pr->d_JF; t.vec_coef[0] = 1.0; t.nvec = 1;
    t.xt_out = pr->d_mu[0];
    t.ep_mv_vals = pr->d_MvT; t.ep_indptr = pr->d_indptrT; t.ep_indices = pr->d_indicesT;
    t.ep_nnz = (int)pr->nnz; t.ep_mv_store = pr->d_MTmu; t.ep_mv_addvec = pr->d_mu[1];
    if ((st = solve(ctx, pr, s, t)) != SP_OK) return st;
  }
  // lambda^0 = M~^T sum_k mu_k + dt J_F(X^0)^H sum_k A_k0 mu_k
  {
    const double2* v[2];
    double c[2];
    int nv = 0;
    for (int k = 1; k <= tb.s; ++k) { v[nv] = pr->d_mu[k - 1]; c[nv++] = dt * tb.A[k][0]; }
    const double2* ad[1] = {pr->d_MTmu};
    const double w[1] = {1.0};
    if ((st = adjoint_rhs(ctx, pr, s, X0, nv, v, c, 1, ad, w, pr->d_lamx)) != SP_OK) return st;
  }
  CK(launch_adj_tinvh(s, pr->P, pr->Nz, pr->S, pr->n, pr->d_lamx, pr->d_col_map, pr->d_var_rec, pr->d_var_ph,
                      reinterpret_cast<double2*>(lambda_dev)));
  return SP_OK;
}

sp_status sp_step_record(sp_ctx* ctx, int problem, double dt, int nsteps, void* states_dev) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  if (pr->scheme != SP_RK222 && pr->scheme != SP_RK111)
    return fail(ctx, SP_ERR_ARG, "sp_step_record is provided for the RK222 and RK111 schemes");
  if (nsteps < 0) return fail(ctx, SP_ERR_ARG, "nsteps < 0");
  if (!states_dev && nsteps > 0) return fail(ctx, SP_ERR_ARG, "null pointer");
  if (!pr->factored || dt != pr->fac_dt)
    return fail(ctx, SP_ERR_NOT_FACTORED, "dt = %.17g is not the factored step size", dt);
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->stream;
  sp_status st;
  const size_t ncoef = (size_t)pr->S * pr->P * pr->Nz;
  double2* rec = reinterpret_cast<double2*>(states_dev);
  for (int k = 0; k < nsteps; ++k) {
    if ((st = ensure_solve_vars(ctx, pr, s)) != SP_OK) return st;
    const std::vector<StagePlan> plan = plan_step(ctx, pr, dt);
    const size_t ns = plan.size();
    for (size_t i = 0; i < ns; ++i) {
      // X^n before the first stage, X^i after stage i < s
      CK(cudaMemcpyAsync(rec + ((size_t)k * ns + i) * ncoef, pr->d_Xc, ncoef * sizeof(double2),
                         cudaMemcpyDeviceToDevice, s));
      if ((st = eval_rhs(ctx, pr, s, plan[i].fc_out)) != SP_OK) return st;
      if ((st = solve(ctx, pr, s, plan[i].args)) != SP_OK) return st;
    }
    commit_step(pr);
  }
  return SP_OK;
}

sp_status sp_transform_adjoint(sp_ctx* ctx, int problem, const void* in, void* out, int nfields, int direction,
                               int scale_num, int scale_den, int on_device) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  if (!in || !out || nfields < 1 || nfields > 16 || (direction != 1 && direction != -1))
    return fail(ctx, SP_ERR_ARG, "bad arguments");
  if (scale_num <= 0 || scale_den <= 0 || scale_num < scale_den ||
      (pr->Nx * scale_num) % scale_den || (pr->Nz * scale_num) % scale_den)
    return fail(ctx, SP_ERR_ARG, "scale must be >= 1 and give integer grid sizes");
  if (pr->ndim != 2) return fail(ctx, SP_ERR_ARG, "sp_transform_adjoint takes 2D problems");
  CK(cudaSetDevice(ctx->device));
  sp_status st = upload_problem(ctx, pr);
  if (st != SP_OK) return st;
  const int Ngx = pr->Nx * scale_num / scale_den, Ngz = pr->Nz * scale_num / scale_den;
  TransformPlan *px, *pz;
  if ((st = make_plan(ctx, pr, pr->Nx, Ngx, &px)) != SP_OK) return st;
  if ((st = make_plan(ctx, pr, pr->Nz, Ngz, &pz)) != SP_OK) return st;
  cudaStream_t s = ctx->stream;
  const size_t ncoef = (size_t)nfields * pr->P * pr->Nz, ngrid = (size_t)nfields * Ngz * Ngx;
  double2* coef = nullptr;
  double* grid = nullptr;
  void* mid = nullptr;
  CK(dalloc(&coef, ncoef));
  CK(dalloc(&grid, ngrid));
  CK(cudaMalloc(&mid, (size_t)nfields * Ngz * pr->P * 16));
  const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  cudaError_t e;
  if (direction < 0) {
    // transpose of coefficients -> grid: grid adjoint in, coefficient adjoint out
    e = cudaMemcpyAsync(grid, in, ngrid * sizeof(double), kin, s);
    if (e == cudaSuccess)
      e = launch_fourier_rows(s, 0, *px, Ngz, pr->P, 4, nfields, nullptr, grid, nullptr, 0, nullptr, nullptr,
                              nullptr, nullptr, 0, mid, nullptr, 2);
    if (e == cudaSuccess) e = launch_cheb_forward(s, 0, *pz, pr->P, nfields, mid, coef, 1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, coef, ncoef * sizeof(double2), kout, s);
  } else {
    // transpose of grid -> coefficients: coefficient adjoint in, grid adjoint out
    e = cudaMemcpyAsync(coef, in, ncoef * sizeof(double2), kin, s);
    if (e == cudaSuccess)
      e = launch_cheb_backward(s, 0, *pz, pr->P, nfields, pr->d_ident, pr->d_zero, pr->d_kx, coef, pr->P * pr->Nz,
                               mid, nullptr, nullptr, 1);
    if (e == cudaSuccess)
      e = launch_fourier_rows(s, 0, *px, Ngz, pr->P, 1, nfields, mid, nullptr, grid, 0, nullptr, nullptr, nullptr,
                              nullptr, 0, nullptr, nullptr, 1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, grid, ngrid * sizeof(double), kout, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(coef);
  cudaFree(grid);
  cudaFree(mid);
  CK(e);
  return SP_OK;
}

sp_status sp_dz_adjoint(sp_ctx* ctx, int problem, const void* dst_bar_dev, void* src_bar_dev) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  if (!dst_bar_dev || !src_bar_dev) return fail(ctx, SP_ERR_ARG, "null pointer");
  CK(cudaSetDevice(ctx->device));
  CK(launch_dz_adjoint(ctx->stream, pr->P, pr->Nz, 2.0 / (pr->zb - pr->za),
                       reinterpret_cast<const double2*>(dst_bar_dev), reinterpret_cast<double2*>(src_bar_dev)));
  return SP_OK;
}

sp_status sp_sync_status(sp_ctx* ctx, int64_t* pencil) {
  if (!ctx) return SP_ERR_ARG;
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  DevStatus h{};
  CK(cudaMemcpy(&h, ctx->d_status, sizeof h, cudaMemcpyDeviceToHost));
  CK(cudaMemset(ctx->d_status, 0, sizeof h));
  if (pencil) *pencil = h.code ? h.pencil : -1;
  if (h.code) {
    ctx->err = "device status " + std::to_string(h.code) + " at pencil " + std::to_string(h.pencil);
    return (sp_status)h.code;
  }
  return SP_OK;
}

sp_status sp_transform(sp_ctx* ctx, int problem, const void* in, void* out, int nfields, int direction,
                       int scale_num, int scale_den, int on_device) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  if (!in || !out || nfields < 1 || nfields > 16 || (direction != 1 && direction != -1))
    return fail(ctx, SP_ERR_ARG, "bad arguments");
  if (scale_num <= 0 || scale_den <= 0 || scale_num < scale_den || (pr->Nx * scale_num) % scale_den ||
      (pr->Nz * scale_num) % scale_den || (pr->ndim == 3 && (pr->Ny * scale_num) % scale_den))
    return fail(ctx, SP_ERR_ARG, "scale must be >= 1 and give integer grid sizes");
  CK(cudaSetDevice(ctx->device));
  sp_status st = upload_problem(ctx, pr);
  if (st != SP_OK) return st;
  const int Ngx = pr->Nx * scale_num / scale_den, Ngz = pr->Nz * scale_num / scale_den;
  const int Ngy = pr->ndim == 3 ? pr->Ny * scale_num / scale_den : 1;
  TransformPlan *px, *pz, *py = nullptr;
  if ((st = make_plan(ctx, pr, pr->Nx, Ngx, &px)) != SP_OK) return st;
  if ((st = make_plan(ctx, pr, pr->Nz, Ngz, &pz)) != SP_OK) return st;
  if (pr->ndim == 3 && (st = make_plan(ctx, pr, pr->Ny, Ngy, &py)) != SP_OK) return st;
  cudaStream_t s = ctx->stream;
  const size_t ncoef = (size_t)nfields * pr->P * pr->Nz, ngrid = (size_t)nfields * Ngz * Ngy * Ngx;
  const size_t esz = pr->prec ? 8 : 16;
  const size_t nm = grid_scratch_elems(pr, nfields, Ngy, Ngz);
  double2* coef = nullptr;
  double* grid = nullptr;
  void *m1 = nullptr, *m2 = nullptr;
  CK(dalloc(&coef, ncoef));
  CK(dalloc(&grid, ngrid));
  CK(cudaMalloc(&m1, nm * esz));
  CK(cudaMalloc(&m2, nm * esz));
  const cudaMemcpyKind kin = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  const cudaMemcpyKind kout = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  cudaError_t e;
  float2* coef32 = nullptr;
  if (direction < 0) {
    e = cudaMemcpyAsync(coef, in, ncoef * sizeof(double2), kin, s);
    if (e == cudaSuccess && pr->prec) {
      e = cudaMalloc(&coef32, ncoef * sizeof(float2));
      if (e == cudaSuccess) e = launch_to_f32(s, coef, coef32, ncoef);
    }
    if (e == cudaSuccess)
      e = coef_to_grid(pr, s, pr->prec, nfields, *px, py, *pz, Ngy, Ngz, pr->d_ident, coef, pr->P * pr->Nz, coef32,
                       grid, m1, m2);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, grid, ngrid * sizeof(double), kout, s);
  } else {
    e = cudaMemcpyAsync(grid, in, ngrid * sizeof(double), kin, s);
    if (e == cudaSuccess) e = grid_to_coef(pr, s, pr->prec, nfields, *px, py, *pz, Ngy, Ngz, grid, coef, m1, m2);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, coef, ncoef * sizeof(double2), kout, s);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(coef);
  cudaFree(grid);
  cudaFree(m1);
  cudaFree(m2);
  if (coef32) cudaFree(coef32);
  CK(e);
  return SP_OK;
}

sp_status sp_eval_rhs(sp_ctx* ctx, int problem, void* out_host, int* n_eq) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  if (!pr->uploaded) return fail(ctx, SP_ERR_STATE, "no state on the device yet");
  CK(cudaSetDevice(ctx->device));
  sp_status st = eval_rhs(ctx, pr, ctx->stream, pr->d_Fc[2]);
  if (st != SP_OK) return st;
  const size_t cnt = pr->nl_eqs.size() * (size_t)pr->P * pr->Nz;
  if (out_host && cnt) CK(cudaMemcpyAsync(out_host, pr->d_Fc[2], cnt * sizeof(double2), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaStreamSynchronize(ctx->stream));
  if (n_eq) *n_eq = (int)pr->nl_eqs.size();
  return SP_OK;
}

sp_status sp_get_band(sp_ctx* ctx, int problem, int* n, int* kl, int* ku) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  if (pr->nnz < 0) return fail(ctx, SP_ERR_STATE, "sp_set_pencils has not been called");
  if (n) *n = pr->n;
  if (kl) *kl = pr->kl;
  if (ku) *ku = pr->ku;
  return SP_OK;
}

sp_status sp_eig_target(sp_ctx* ctx, int problem, double sigma_t, int iters, const void* x0_host, double* sigma_re,
                        double* sigma_im) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  if (iters < 1 || !sigma_re || !sigma_im || !std::isfinite(sigma_t)) return fail(ctx, SP_ERR_ARG, "bad arguments");
  CK(cudaSetDevice(ctx->device));
  sp_status st = upload_problem(ctx, pr);
  if (st != SP_OK) return st;
  cudaStream_t s = ctx->stream;
  // L~ + sigma_T M~ into the first factor slot: the step's factorization is gone
  pr->factored = false;
  pr->lbvp_factored = false;
  for (auto& kv : pr->graphs) cudaGraphExecDestroy(kv.second);
  pr->graphs.clear();
  drop_batches(ctx, problem);
  const int ldab = 2 * pr->kl + pr->ku + 1;
  double* work = nullptr;
  CK(dalloc(&work, (size_t)pr->P * pr->n * ldab));
  cudaError_t e = launch_band_factor(s, pr->P, pr->n, (int)pr->nnz, pr->kl, pr->ku, pr->d_indptr, pr->d_indices,
                                     pr->d_Mv, pr->d_Lv, sigma_t, 1.0, work, pr->fac[0], pr->npad, pr->lpad,
                                     pr->upad, ctx->d_status);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaFree(work);
  CK(e);
  const size_t nv = (size_t)pr->P * pr->n;
  double2 *x = nullptr, *y = nullptr, *mu = nullptr;
  auto release = [&]() { cudaFree(x); cudaFree(y); cudaFree(mu); };
  if ((e = cudaMalloc(&x, nv * sizeof(double2))) == cudaSuccess && (e = cudaMalloc(&y, nv * sizeof(double2))) ==
      cudaSuccess)
    e = cudaMalloc(&mu, (size_t)pr->P * sizeof(double2));
  if (e != cudaSuccess) { release(); CK(e); }
  if (x0_host) {
    e = cudaMemcpyAsync(x, x0_host, nv * sizeof(double2), cudaMemcpyHostToDevice, s);
  } else {
    std::vector<double2> ones(nv, make_double2(1.0, 0.0));
    e = cudaMemcpyAsync(x, ones.data(), nv * sizeof(double2), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  }
  // y = (L~ + sigma_T M~)^{-1} M~ x: the solve kernel with the M~ matvec as
  // its whole right-hand side (no stored vectors, F~ or boundary values)
  SolveArgs a = base_args(pr, ctx, 0);
  a.mode = 0;
  a.nvec = 0; a.nfc = 0; a.n_nl = 0; a.nbc = 0; a.bc_coef = 0.0;
  a.mv_x = x; a.mv_coef = 1.0; a.mv_store = nullptr;
  set_mv_M(pr, a);
  a.xt_out = y; a.xc_out = nullptr; a.xc32_out = nullptr; a.ep_mv_vals = nullptr;
  a.Lg = nullptr; a.Ug = nullptr; a.pg = nullptr; a.umask = nullptr;
  for (int k = 0; e == cudaSuccess && k < iters; ++k) {
    e = launch_pencil_solve(s, a);
    if (e == cudaSuccess) e = launch_eig_update(s, pr->P, pr->n, x, y, mu);
  }
  std::vector<double2> hm(pr->P);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hm.data(), mu, hm.size() * sizeof(double2), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) { release(); CK(e); }
  std::vector<double2> hs(pr->P);
  for (int p = 0; p < pr->P; ++p) {
    // sigma = sigma_T - 1 / mu
    const double m2 = hm[p].x * hm[p].x + hm[p].y * hm[p].y;
    sigma_re[p] = m2 > 0 ? sigma_t - hm[p].x / m2 : NAN;
    sigma_im[p] = m2 > 0 ? hm[p].y / m2 : NAN;
    hs[p] = make_double2(sigma_re[p], sigma_im[p]);
  }
  // keep the eigenpairs for sp_eig_residual: x (normalized iterate) and sigma
  cudaFree(pr->d_eigx);
  cudaFree(pr->d_eigsig);
  pr->d_eigx = x;
  x = nullptr;
  pr->d_eigsig = nullptr;
  release();
  CK(dalloc(&pr->d_eigsig, (size_t)pr->P));
  CK(cudaMemcpy(pr->d_eigsig, hs.data(), hs.size() * sizeof(double2), cudaMemcpyHostToDevice));
  return SP_OK;
}

sp_status sp_eig_residual(sp_ctx* ctx, int problem, double* residual) {
  Problem* pr = get(ctx, problem);
  if (!pr || !residual) return fail(ctx, SP_ERR_ARG, "bad context, problem id or output");
  ctx->err.clear();
  if (!pr->d_eigx || !pr->d_eigsig) return fail(ctx, SP_ERR_STATE, "no eigensolve has run on this problem");
  CK(cudaSetDevice(ctx->device));
  double* d = nullptr;
  CK(dalloc(&d, (size_t)pr->P));
  cudaError_t e = launch_eig_residual(ctx->stream, pr->P, pr->n, (int)pr->nnz, pr->d_indptr, pr->d_indices, pr->d_Mv,
                                      pr->d_Lv, pr->d_eigx, pr->d_eigsig, d);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(residual, d, (size_t)pr->P * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(d);
  CK(e);
  return SP_OK;
}

sp_status sp_cfl_frequency(sp_ctx* ctx, int problem, int nvel, const int* vars, const int* axes, double* freq_out) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  if (nvel < 1 || nvel > 3 || !vars || !axes || !freq_out) return fail(ctx, SP_ERR_ARG, "bad arguments");
  for (int v = 0; v < nvel; ++v) {
    if (vars[v] < 0 || vars[v] >= pr->S) return fail(ctx, SP_ERR_ARG, "variable %d out of range", vars[v]);
    if (axes[v] != 0 && axes[v] != 2 && !(axes[v] == 1 && pr->ndim == 3))
      return fail(ctx, SP_ERR_ARG, "axis %d is not an axis of the problem", axes[v]);
  }
  CK(cudaSetDevice(ctx->device));
  sp_status st = upload_problem(ctx, pr);
  if (st != SP_OK) return st;
  TransformPlan *px, *pz, *py = nullptr;
  if ((st = make_plan(ctx, pr, pr->Nx, pr->Ngx, &px)) != SP_OK) return st;
  if ((st = make_plan(ctx, pr, pr->Nz, pr->Ngz, &pz)) != SP_OK) return st;
  if (pr->ndim == 3 && (st = make_plan(ctx, pr, pr->Ny, pr->Ngy, &py)) != SP_OK) return st;
  cudaStream_t s = ctx->stream;
  const int Ngy = pr->ndim == 3 ? pr->Ngy : 1;
  if (pr->cfl_cap < nvel) {
    // scratch for three fields, the inverse node spacings, the arguments
    cudaFree(pr->d_cfl_grid); cudaFree(pr->d_cfl_mid1); cudaFree(pr->d_cfl_mid2);
    pr->d_cfl_grid = nullptr; pr->d_cfl_mid1 = pr->d_cfl_mid2 = nullptr;
    const size_t nm = grid_scratch_elems(pr, 3, Ngy, pr->Ngz), esz = pr->prec ? 8 : 16;
    CK(dalloc(&pr->d_cfl_grid, (size_t)3 * pr->Ngz * Ngy * pr->Ngx));
    CK(cudaMalloc(&pr->d_cfl_mid1, nm * esz));
    CK(cudaMalloc(&pr->d_cfl_mid2, nm * esz));
    if (!pr->d_cfl_args) {
      CK(cudaMalloc((void**)&pr->d_cfl_args, 6 * sizeof(int32_t)));
      CK(cudaMalloc((void**)&pr->d_cfl_out, sizeof(unsigned long long)));
      // node spacing of the dealiased Chebyshev grid: centred differences,
      // one-sided at the two end nodes
      const int N = pr->Ngz;
      std::vector<double> z(N), inv(N);
      for (int i = 0; i < N; ++i)
        z[i] = pr->za + (pr->zb - pr->za) * 0.5 * (1.0 - std::cos(M_PI * (i + 0.5) / N));
      for (int i = 0; i < N; ++i) {
        const double d = (i == 0) ? z[1] - z[0] : (i == N - 1) ? z[N - 1] - z[N - 2] : 0.5 * (z[i + 1] - z[i - 1]);
        inv[i] = 1.0 / d;
      }
      CK(upload(&pr->d_inv_dz, inv, s));
    }
    pr->cfl_cap = 3;
  }
  int32_t args[6] = {0, 0, 0, 0, 0, 0};
  for (int v = 0; v < nvel; ++v) { args[v] = vars[v]; args[3 + v] = axes[v]; }
  CK(cudaMemcpyAsync(pr->d_cfl_args, args, sizeof(args), cudaMemcpyHostToDevice, s));
  if (pr->prec && !pr->xc32_valid) {
    CK(launch_to_f32(s, pr->d_Xc, pr->d_Xc32, (size_t)pr->S * pr->P * pr->Nz));
    pr->xc32_valid = true;
  }
  CK(coef_to_grid(pr, s, pr->prec, nvel, *px, py, *pz, Ngy, pr->Ngz, pr->d_cfl_args, pr->d_Xc,
                  pr->P * pr->Nz, pr->d_Xc32, pr->d_cfl_grid, pr->d_cfl_mid1, pr->d_cfl_mid2));
  CK(cudaMemsetAsync(pr->d_cfl_out, 0, sizeof(unsigned long long), s));
  const double inv_dx = pr->Ngx / pr->Lx, inv_dy = pr->ndim == 3 ? Ngy / pr->Ly : 0.0;
  CK(launch_cfl_max(s, pr->d_cfl_grid, nvel, pr->d_cfl_args + 3, pr->Ngx, Ngy, pr->Ngz, inv_dx, inv_dy,
                    pr->d_inv_dz, pr->d_cfl_out));
  unsigned long long bits = 0;
  CK(cudaMemcpyAsync(&bits, pr->d_cfl_out, sizeof(bits), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double f;
  std::memcpy(&f, &bits, sizeof f);
  *freq_out = f;
  return SP_OK;
}

sp_status sp_cfl_dt(double freq, double dt_prev, double safety, double min_dt, double max_dt, double min_change,
                    double max_change, double threshold, double* dt_out) {
  if (!dt_out || !(safety > 0.0) || !(freq >= 0.0) || !(min_dt >= 0.0) || !(max_dt >= min_dt) ||
      !(min_change > 0.0) || !(max_change >= min_change) || !(threshold >= 0.0))
    return SP_ERR_ARG;
  double dt = freq > 0.0 ? safety / freq : max_dt;
  dt = std::min(std::max(dt, min_dt), max_dt);
  if (dt_prev > 0.0) {
    dt = std::min(std::max(dt, min_change * dt_prev), max_change * dt_prev);
    if (std::fabs(dt - dt_prev) < threshold * dt_prev) dt = dt_prev;
  }
  *dt_out = dt;
  return SP_OK;
}

sp_status sp_get_solve_work(sp_ctx* ctx, int problem, double* fma_per_row, double* factor_bytes) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  if (!pr->factored) return fail(ctx, SP_ERR_NOT_FACTORED, "sp_factor has not been called");
  const BandFactor& f = pr->fac[pr->nfac - 1];
  const double n = pr->n, kl = pr->kl, kuu = pr->kl + pr->ku;
  double fma, bytes;
  if (pr->lanes) {
    fma = kl + f.u_listed;
    bytes = n * (kl + f.cmax) * 8.0 + n;
  } else {
    fma = kl + kuu;
    bytes = n * (kl + kuu + 1) * 8.0 + n;
  }
  if (fma_per_row) *fma_per_row = fma;
  if (factor_bytes) *factor_bytes = bytes;
  return SP_OK;
}

sp_status sp_set_solve_kernel(sp_ctx* ctx, int problem, int kind) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  if (kind != SP_SOLVE_AUTO && kind != SP_SOLVE_WINDOW && kind != SP_SOLVE_LANES && kind != SP_SOLVE_SPIKE)
    return fail(ctx, SP_ERR_ARG, "unknown solve kernel %d", kind);
  if (pr->uploaded) return fail(ctx, SP_ERR_STATE, "the solve kernel is fixed once the problem is on the device");
  if (kind == SP_SOLVE_LANES && (pr->nnz < 0 || !lanes_supported(pr->kl, pr->kl + pr->ku)))
    return fail(ctx, SP_ERR_ARG, "no lane-per-pencil substitution for kl = %d, kl + ku = %d (set the pencils first)",
                pr->kl, pr->kl + pr->ku);
  if (kind == SP_SOLVE_SPIKE) {
    const int npad = (pr->n + SOLVE_CHUNK - 1) / SOLVE_CHUNK * SOLVE_CHUNK;
    const int nblk = pr->spike_blocks > 0 ? pr->spike_blocks : default_spike_blocks(npad, pr->P);
    if (pr->nnz < 0 || !spike_supported(pr->kl, pr->kl + pr->ku, npad, nblk))
      return fail(ctx, SP_ERR_ARG, "no partitioned substitution for kl = %d, kl + ku = %d, %d rows in %d blocks "
                  "(needs kl <= 7, kl + ku <= 31, whole 32-row chunks per block; set the pencils first)",
                  pr->kl, pr->kl + pr->ku, npad, nblk);
  }
  pr->solve_kind = kind;
  return SP_OK;
}

sp_status sp_set_z_transform(sp_ctx* ctx, int problem, int kind) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  if (kind != SP_ZT_AUTO && kind != SP_ZT_FFT && kind != SP_ZT_MMA)
    return fail(ctx, SP_ERR_ARG, "unknown z transform %d", kind);
  if (pr->uploaded) return fail(ctx, SP_ERR_STATE, "the z transform is fixed once the problem is on the device");
  if (kind == SP_ZT_MMA) {
    const int ngz = pr->bz.n_coeff * pr->bz.dealias_num / std::max(1, pr->bz.dealias_den);
    if (pr->prec != SP_PREC_MIXED || !cheb_mma_supported(pr->bz.n_coeff, ngz))
      return fail(ctx, SP_ERR_ARG, "the tensor-core z transform needs mixed precision, N_z a multiple of 32 and "
                  "N_gz a multiple of 16 up to 256 (N_z = %d, N_gz = %d)", pr->bz.n_coeff, ngz);
  }
  pr->zkind = kind;
  return SP_OK;
}

sp_status sp_get_z_transform(sp_ctx* ctx, int problem, int* kind) {
  Problem* pr = get(ctx, problem);
  if (!pr || !kind) return fail(ctx, SP_ERR_ARG, "bad context, problem id or output");
  ctx->err.clear();
  *kind = !pr->uploaded ? pr->zkind : (pr->zmma ? SP_ZT_MMA : SP_ZT_FFT);
  return SP_OK;
}

sp_status sp_set_spike_blocks(sp_ctx* ctx, int problem, int nblk) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  if (pr->uploaded) return fail(ctx, SP_ERR_STATE, "the block count is fixed once the problem is on the device");
  if (nblk < 0) return fail(ctx, SP_ERR_ARG, "nblk must be >= 0");
  if (nblk > 0 && pr->nnz >= 0) {
    const int npad = (pr->n + SOLVE_CHUNK - 1) / SOLVE_CHUNK * SOLVE_CHUNK;
    if (npad % (nblk * SOLVE_CHUNK))
      return fail(ctx, SP_ERR_ARG, "%d rows do not split into %d blocks of whole 32-row chunks", npad, nblk);
  }
  pr->spike_blocks = nblk;
  return SP_OK;
}

sp_status sp_get_spike_blocks(sp_ctx* ctx, int problem, int* nblk) {
  Problem* pr = get(ctx, problem);
  if (!pr || !nblk) return fail(ctx, SP_ERR_ARG, "bad context, problem id or output");
  ctx->err.clear();
  *nblk = (pr->uploaded && pr->spike) ? pr->nblk : 0;
  return SP_OK;
}

sp_status sp_set_timing(sp_ctx* ctx, int problem, int max_launches) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  ctx->err.clear();
  CK(cudaSetDevice(ctx->device));
  while ((int)pr->ev.size() < 2 * max_launches) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    pr->ev.push_back(e);
  }
  pr->ev_used = 0;
  pr->timing = max_launches > 0;
  return SP_OK;
}

sp_status sp_last_solve_time(sp_ctx* ctx, int problem, double* ms_per_launch, int* launches) {
  Problem* pr = get(ctx, problem);
  if (!pr) return fail(ctx, SP_ERR_ARG, "bad context or problem id");
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->stream));
  double tot = 0;
  const int cnt = (int)(pr->ev_used / 2);
  for (int i = 0; i < cnt; ++i) {
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, pr->ev[2 * i], pr->ev[2 * i + 1]));
    tot += ms;
  }
  if (ms_per_launch) *ms_per_launch = cnt ? tot / cnt : 0.0;
  if (launches) *launches = cnt;
  return SP_OK;
}

}  // extern "C"
