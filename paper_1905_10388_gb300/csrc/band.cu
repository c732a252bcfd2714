// Banded pencil factorization and solve (FP64), sm_103a.
//
// Sec. "Matrix solvers": factor each pencil matrix once per step size and
// reuse it; Sec. "Multistep / Runge-Kutta IMEX integrators": B~ is a fixed
// linear combination of stored M~X~, L~X~ and F~ vectors.  The pencil
// matrices are banded after interleaving and Dirichlet recombination
// (Sec. "A general sparse tau method"), so the LU uses banded partial
// pivoting in the LAPACK gbtrf layout: L keeps kl multipliers per column and
// the row interchanges are applied interleaved with them; U holds
// kuu = kl + ku superdiagonals.
//
// GB300 FP64 runs at ~1 TFLOP/s with a 64-cycle dependent-FMA latency, so
// the substitution is a sequential chain per pencil.  One warp owns one
// pencil: its 32 lanes hold a rotating window of the right-hand side
// (lane = index mod 32 [mod 64 with two registers per lane]), one lane per
// band entry, the real and imaginary parts of the complex right-hand side
// sharing one real factor.  Each step broadcasts the settled entry with one
// shuffle and updates the window with one FMA per lane.  The factor is
// streamed through a shared-memory ring by bulk asynchronous copies (TMA,
// cp.async.bulk) issued by one lane and tracked with mbarriers; every wait
// is bounded and reports SP_ERR_TIMEOUT instead of hanging.
#include <algorithm>
#include <cstdio>

#include "internal.h"
#include "tma.cuh"

namespace spectau {

// ---------------------------------------------------------------------------
// factorization: one warp per pencil.  The band a*M~ + b*L~ is assembled in a
// global array AB[p][j][t] (t = i - j + kuu), then eliminated column by
// column (LAPACK gbtrf order: partial pivoting within the kl rows below the
// diagonal) in a shared-memory ring of the kuu + 1 columns a step touches;
// each column leaves the ring, in the solve layout, as soon as it is final,
// and the next column of AB enters.
// ---------------------------------------------------------------------------
__global__ void k_band_factor(int P, int n, int nnz, int kl, int ku, const int32_t* __restrict__ indptr,
                              const int32_t* __restrict__ indices, const double* __restrict__ Mv,
                              const double* __restrict__ Lv, double alpha, double beta,
                              double* __restrict__ work, double* __restrict__ Lf, uint8_t* __restrict__ piv,
                              double* __restrict__ Uf, double* __restrict__ Rd, int npad, int lpad, int upad,
                              DevStatus* st) {
  extern __shared__ __align__(16) double fring[];
  const int warps = blockDim.x / 32;
  const int wi = threadIdx.x / 32;
  const int p = blockIdx.x * warps + wi;
  const int lane = threadIdx.x & 31;
  if (p >= P) return;
  const int kuu = kl + ku;
  const int ldab = kl + kuu + 1;
  const int R = kuu + 1;                          // ring columns: j .. j + kuu
  double* ring = fring + (size_t)wi * R * ldab;
  const float invR = 1.0f / (float)R;
  auto slot = [&](int c) { return ring + (size_t)(c - R * div_idx(c, invR)) * ldab; };   // c mod R
  double* AB = work + (size_t)p * n * ldab;
  for (size_t e = lane; e < (size_t)n * ldab; e += 32) AB[e] = 0.0;
  __syncwarp();
  const double* M = Mv + (size_t)p * nnz;
  const double* L = Lv + (size_t)p * nnz;
  for (int r = lane; r < n; r += 32) {
    for (int e = indptr[r]; e < indptr[r + 1]; ++e) {
      const int c = indices[e];
      AB[(size_t)c * ldab + (r - c + kuu)] = alpha * M[e] + beta * L[e];
    }
  }
  __syncwarp();
  for (int c = 0; c < min(R, n); ++c)
    for (int t = lane; t < ldab; t += 32) slot(c)[t] = AB[(size_t)c * ldab + t];
  __syncwarp();
  uint8_t* pv = piv + (size_t)p * npad;
  double* Lp = Lf + (size_t)p * npad * lpad;
  double* Up = Uf + (size_t)p * npad * upad;
  double* Rp = Rd + (size_t)p * npad;
  // the column that enters the ring next, fetched into registers one step
  // ahead of its store (ldab <= 64: two entries per lane)
  double pre0 = 0.0, pre1 = 0.0;
  auto fetch = [&](int c) {
    pre0 = (c < n && lane < ldab) ? AB[(size_t)c * ldab + lane] : 0.0;
    pre1 = (c < n && lane + 32 < ldab) ? AB[(size_t)c * ldab + lane + 32] : 0.0;
  };
  fetch(R);
  bool singular = false;
  for (int j = 0; j < n; ++j) {
    const int m = min(kl, n - 1 - j);
    const int clast = min(n - 1, j + kuu);
    double* colj = slot(j);
    // pivot search: first maximum of |a| over rows j .. j+m, compared on the
    // bit patterns of |a| (their integer order is the numeric order of
    // non-negative doubles; no FP64 compare on the chain)
    unsigned long long a =
        (lane <= m) ? ((unsigned long long)__double_as_longlong(colj[kuu + lane]) & 0x7fffffffffffffffull) : 0ull;
    int ia = lane;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long b = __shfl_xor_sync(0xffffffffu, a, o);
      const int ib = __shfl_xor_sync(0xffffffffu, ia, o);
      if (b > a || (b == a && ib < ia)) { a = b; ia = ib; }
    }
    const int t = ia;
    if (lane == 0) pv[j] = (uint8_t)t;
    // a zero pivot, or an infinite or NaN one
    if (a == 0ull || a >= 0x7ff0000000000000ull) { singular = true; break; }
    // interchange rows j and j+t over columns j .. j+kuu
    if (t != 0) {
      for (int c = j + lane; c <= clast; c += 32) {
        double* col = slot(c);
        const int r0 = j - c + kuu, r1 = j + t - c + kuu;
        const double x0 = col[r0];
        col[r0] = col[r1];
        col[r1] = x0;
      }
    }
    __syncwarp();
    // multipliers by the reciprocal of the pivot (as LAPACK's gbtf2 scales)
    const double rd = 1.0 / colj[kuu];
    if (lane >= 1 && lane <= m) colj[kuu + lane] *= rd;
    __syncwarp();
    // rank-1 update of rows j+1..j+m, columns j+1..j+kuu: each lane loads
    // its column's m entries and the m multipliers, then updates them all
    // (independent FMAs in flight instead of one load-FMA-store at a time)
    constexpr int MREG = 16;
    for (int c = j + 1 + lane; c <= clast; c += 32) {
      double* col = slot(c);
      const double u = col[j - c + kuu];
      double* dst = col + (j - c + kuu);          // dst[tt]: row j + tt
      if (m <= MREG) {
        double lv[MREG], av[MREG];
#pragma unroll
        for (int tt = 0; tt < MREG; ++tt) {
          lv[tt] = tt < m ? colj[kuu + 1 + tt] : 0.0;
          av[tt] = tt < m ? dst[1 + tt] : 0.0;
        }
#pragma unroll
        for (int tt = 0; tt < MREG; ++tt)
          if (tt < m) dst[1 + tt] = fma(-lv[tt], u, av[tt]);
      } else {
        for (int tt = 1; tt <= m; ++tt) dst[tt] = fma(-colj[kuu + tt], u, dst[tt]);
      }
    }
    __syncwarp();
    // column j is final: L multipliers, 1/U_jj and the scaled U column
    for (int q = lane; q < lpad; q += 32)
      Lp[(size_t)j * lpad + q] = (q < kl && j + 1 + q < n) ? colj[kuu + 1 + q] : 0.0;
    for (int q = lane; q < upad; q += 32)
      Up[(size_t)j * upad + q] = q == 0 ? rd : ((q <= kuu && j - q >= 0) ? colj[kuu - q] * rd : 0.0);
    if (lane == 0) Rp[j] = rd;
    __syncwarp();
    // its slot takes column j + kuu + 1 (fetched during this step)
    if (j + R < n) {
      if (lane < ldab) colj[lane] = pre0;
      if (lane + 32 < ldab) colj[lane + 32] = pre1;
    }
    fetch(j + R + 1);
    __syncwarp();
  }
  if (singular) {
    if (lane == 0) raise_status(st, SP_ERR_SINGULAR, p);
    return;
  }
  for (int j = n + lane; j < npad; j += 32) {   // padding columns
    for (int q = 0; q < lpad; ++q) Lp[(size_t)j * lpad + q] = 0.0;
    for (int q = 0; q < upad; ++q) Up[(size_t)j * upad + q] = 0.0;
    pv[j] = 0;
    Rp[j] = 0.0;
  }
}

cudaError_t launch_band_factor(cudaStream_t s, int P, int n, int nnz, int kl, int ku,
                               const int32_t* indptr, const int32_t* indices, const double* Mv,
                               const double* Lv, double alpha, double beta, double* work,
                               const BandFactor& f, int npad, int lpad, int upad, DevStatus* st) {
  const int wpb = 4;
  const size_t smem = (size_t)wpb * (kl + ku + 1) * (2 * kl + ku + 1) * sizeof(double);
  if (smem > 227 * 1024 || 2 * kl + ku + 1 > 64) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_band_factor, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_band_factor<<<(P + wpb - 1) / wpb, 32 * wpb, smem, s>>>(P, n, nnz, kl, ku, indptr, indices, Mv, Lv,
                                                           alpha, beta, work, f.L, f.piv, f.U, f.rd, npad,
                                                           lpad, upad, st);
  return cudaGetLastError();
}

__device__ __forceinline__ double2 shfl2(double2 v, int src) {
  double2 r;
  r.x = __shfl_sync(0xffffffffu, v.x, src);
  r.y = __shfl_sync(0xffffffffu, v.y, src);
  return r;
}

// ---------------------------------------------------------------------------
// pencil solve: prologue (B~ assembly) -> L pass -> U pass -> epilogue
// ---------------------------------------------------------------------------
// acc + the left-preconditioned F~ entry of row (slot sl, mode m): the
// combination sum_k c_k F_k of the stored right-hand sides, through the
// T-to-U conversion P^L for differential equations (Appendix: row m holds
// (1 + delta_m0)/2 F_m - F_{m+2}/2) and the phase i^-q of the equation's
// real-ification.  One FMA per term and component: on GB300 every FP64
// instruction holds the sub-partition's FP64 pipe for 64 cycles, so the
// halves c/2 and -c/2 come precomputed with the arguments and the phase is
// applied to the loaded values (a sign and swap, no arithmetic).
__device__ __forceinline__ double2 add_f_row(const SolveArgs& a, int sl, int m, int p, double2 acc) {
  const int Nz = a.Nz;
  const int e = a.nl_eq[sl];
  const bool dif = a.eq_differential[e] != 0;
  const int ph = -a.eq_phase[e];
#pragma unroll
  for (int k = 0; k < SP_MAX_TERMS; ++k) {
    if (k >= a.nfc) break;
    const double2* F = a.fc[k] + ((size_t)sl * a.P + p) * Nz;
    const double2 v0 = cipow_d(F[m], ph);
    const double c = (dif && m > 0) ? a.fc_half[k] : a.fc_coef[k];
    acc.x = fma(c, v0.x, acc.x);
    acc.y = fma(c, v0.y, acc.y);
    if (dif && m + 2 < Nz) {
      const double2 v2 = cipow_d(F[m + 2], ph);
      acc.x = fma(a.fc_mhalf[k], v2.x, acc.x);
      acc.y = fma(a.fc_mhalf[k], v2.y, acc.y);
    }
  }
  return acc;
}

// c v, exactly v when c = 1 (tested on the bit pattern: no FP64 compare)
__device__ __forceinline__ double2 scale_first(double c, double2 v) {
  if (__double_as_longlong(c) == 0x3FF0000000000000LL) return v;
  return make_double2(c * v.x, c * v.y);
}

struct SolveSmem {
  double2* B;
  double* Lring;
  double* Uring;
  uint8_t* Pring;
  uint64_t* barL;
  uint64_t* barU;
  int* abort_flag;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// B holds npad + 64 entries: the padded columns plus the forward pass's
// one-window-ahead prefetch, zero beyond n.
__host__ __device__ inline size_t solve_smem_bytes(int npad, int lpad, int upad) {
  size_t off = align_up((size_t)(npad + 64) * 16, 128);
  off += align_up((size_t)SOLVE_RING * SOLVE_CHUNK * lpad * 8, 128);
  off += align_up((size_t)SOLVE_RING * SOLVE_CHUNK * upad * 8, 128);
  off += align_up((size_t)SOLVE_RING * SOLVE_CHUNK, 128);
  off += align_up((size_t)2 * SOLVE_RING * 8, 128);
  off += 128;
  return off;
}

// PPC pencils per CTA of NT threads (1 or 2); with PPC = 2 threads
// [0, NT/2) serve pencil 2b and [NT/2, NT) pencil 2b + 1, each half with its
// own shared-memory region.  Warps 0 and 1 of a pencil substitute; all NT/PPC
// threads share the assembly and the epilogue.
template <int RU, int PPC, int MODE = -1, int NT = 128>
__device__ __forceinline__ void pencil_solve_body(const SolveArgs& a, int block, unsigned char* smem_raw) {
  // MODE >= 0 fixes the stage at compile time (assembly-only and
  // epilogue-only kernels carry neither the factor ring nor the substitution)
  const int mode = MODE >= 0 ? MODE : a.mode;
  const int lp = (mode == 0 || mode == 3) ? a.lpad : 0, up = mode == 0 ? a.upad : 0;
  const int half = (PPC == 2) ? (int)(threadIdx.x / (NT / 2)) : 0;
  const int p = block * PPC + half;
  const bool active = p < a.P;
  const int tid = (PPC == 2) ? (int)(threadIdx.x % (NT / 2)) : (int)threadIdx.x;
  const int nt = NT / PPC;
  const int n = a.n;
  SolveSmem sm;
  {
    size_t off = (size_t)half * solve_smem_bytes(a.npad, lp, up);
    sm.B = reinterpret_cast<double2*>(smem_raw + off);
    off += align_up((size_t)(a.npad + 64) * 16, 128);
    sm.Lring = reinterpret_cast<double*>(smem_raw + off);
    off += align_up((size_t)SOLVE_RING * SOLVE_CHUNK * lp * 8, 128);
    sm.Uring = reinterpret_cast<double*>(smem_raw + off);
    off += align_up((size_t)SOLVE_RING * SOLVE_CHUNK * up * 8, 128);
    sm.Pring = reinterpret_cast<uint8_t*>(smem_raw + off);
    off += align_up((size_t)SOLVE_RING * SOLVE_CHUNK, 128);
    sm.barL = reinterpret_cast<uint64_t*>(smem_raw + off);
    sm.barU = sm.barL + SOLVE_RING;
    off += align_up((size_t)2 * SOLVE_RING * 8, 128);
    sm.abort_flag = reinterpret_cast<int*>(smem_raw + off);
  }
  const int nchunks = a.npad / SOLVE_CHUNK;
  const int pp = active ? p : 0;             // keeps addresses valid on an idle half
  const double* Lsrc = a.Lf + (size_t)pp * a.npad * a.lpad;
  const double* Usrc = a.Uf + (size_t)pp * a.npad * a.upad;
  const uint8_t* Psrc = a.piv + (size_t)pp * a.npad;
  const uint32_t lbytes = SOLVE_CHUNK * a.lpad * 8, ubytes = SOLVE_CHUNK * a.upad * 8;

  auto issue_L = [&](int c) {  // chunk c (forward order) into slot c % RING
    const int s = c % SOLVE_RING;
    mbar_expect_tx(&sm.barL[s], lbytes + SOLVE_CHUNK);
    bulk_g2s(sm.Lring + (size_t)s * SOLVE_CHUNK * a.lpad, Lsrc + (size_t)c * SOLVE_CHUNK * a.lpad, lbytes,
             &sm.barL[s]);
    bulk_g2s(sm.Pring + (size_t)s * SOLVE_CHUNK, Psrc + (size_t)c * SOLVE_CHUNK, SOLVE_CHUNK, &sm.barL[s]);
  };
  auto issue_U = [&](int k) {  // k-th chunk of the backward order (chunk nchunks-1-k)
    const int s = k % SOLVE_RING;
    const int c = nchunks - 1 - k;
    mbar_expect_tx(&sm.barU[s], ubytes);
    bulk_g2s(sm.Uring + (size_t)s * SOLVE_CHUNK * a.upad, Usrc + (size_t)c * SOLVE_CHUNK * a.upad, ubytes,
             &sm.barU[s]);
  };

  if (tid == 0 && active) {
    *sm.abort_flag = 0;
    if (mode == 0 || mode == 3) {
      for (int s = 0; s < SOLVE_RING; ++s) {
        mbar_init(&sm.barL[s], 1);
        mbar_init(&sm.barU[s], 1);
      }
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      // the factor does not depend on the prologue: start streaming now
      // (mode 3, forward substitution only: L alone)
      for (int c = 0; c < min(SOLVE_RING, nchunks); ++c) issue_L(c);
      if (mode == 0)
        for (int k = 0; k < min(SOLVE_RING, nchunks); ++k) issue_U(k);
    }
  }

  // ---- prologue: B~ = linear combination of stored vectors, one matvec,
  //      left-preconditioned F~ (T-to-U conversion, tau rows dropped) and
  //      boundary values
  const size_t prow = (size_t)pp * n;
  const int Nz = a.Nz;
  const float invNz = 1.0f / (float)Nz;
  if (mode == 2) {
    // epilogue only: X~ (already divided by U_jj) from the substitution kernel
    for (int r = tid; active && r < n; r += nt) sm.B[r] = a.xg[prow + r];
    __syncthreads();
  } else {
  // modes 0 and 1: two passes over the rows, each with every lane on the
  // same kind of row, since on GB300 an FP64 warp instruction holds the FP64
  // pipe for 64 cycles whatever its active mask: stored vectors and matvec
  // for every row, then the F~ entries by (slot, mode), then the boundary
  // rows.  Mode 1 (assembly only) then stores B~ for the substitution
  // kernel.
  for (int r = tid; active && r < n; r += nt) {
    double2 acc = make_double2(0.0, 0.0);
    if (a.nvec > 0) acc = scale_first(a.vec_coef[0], a.vec[0][prow + r]);
    for (int k = 1; k < a.nvec; ++k) {
      const double2 v = a.vec[k][prow + r];
      acc.x = fma(a.vec_coef[k], v.x, acc.x);
      acc.y = fma(a.vec_coef[k], v.y, acc.y);
    }
    if (a.mv_x != nullptr) {
      double2 s = make_double2(0.0, 0.0);
      const double* vals = a.mv_vals + (size_t)p * a.mv_nnz;
      for (int e = a.mv_indptr[r]; e < a.mv_indptr[r + 1]; ++e) {
        const double m = vals[e];
        const double2 x = a.mv_x[prow + a.mv_indices[e]];
        s.x = fma(m, x.x, s.x);
        s.y = fma(m, x.y, s.y);
      }
      if (a.mv_store != nullptr) a.mv_store[prow + r] = s;
      acc.x = fma(a.mv_coef, s.x, acc.x);
      acc.y = fma(a.mv_coef, s.y, acc.y);
    }
    if (a.mv2_vals != nullptr) {                 // a second matrix on the same vector (CNAB: L~ X~^n)
      double2 s = make_double2(0.0, 0.0);
      const double* vals = a.mv2_vals + (size_t)p * a.mv2_nnz;
      for (int e = a.mv2_indptr[r]; e < a.mv2_indptr[r + 1]; ++e) {
        const double m = vals[e];
        const double2 x = a.mv_x[prow + a.mv2_indices[e]];
        s.x = fma(m, x.x, s.x);
        s.y = fma(m, x.y, s.y);
      }
      acc.x = fma(a.mv2_coef, s.x, acc.x);
      acc.y = fma(a.mv2_coef, s.y, acc.y);
    }
    sm.B[r] = acc;
  }
  for (int r = n + tid; active && r < a.npad + 64; r += nt) sm.B[r] = make_double2(0.0, 0.0);
  __syncthreads();
  for (int idx = tid; active && idx < a.n_nl * Nz; idx += nt) {
    const int sl = div_idx(idx, invNz), m = idx - sl * Nz;
    const int e = a.nl_eq[sl];
    const int row = a.row_map[e * Nz + m];
    if (row < 0) continue;
    sm.B[row] = add_f_row(a, sl, m, p, sm.B[row]);
  }
  for (int q = tid; active && q < a.nbc; q += nt) {
    const int row = a.bc_rows[q];
    const double2 g = a.bc_values[(size_t)p * a.nbc + q];
    double2 b = sm.B[row];
    b.x = fma(a.bc_coef, g.x, b.x);
    b.y = fma(a.bc_coef, g.y, b.y);
    sm.B[row] = b;
  }
  __syncthreads();
  if (mode == 1) {
    for (int r = tid; active && r < n; r += nt) a.bg[prow + r] = sm.B[r];   // B~ for the substitution kernel
    return;
  }
  }


  // ---- substitution, over the padded columns [0, npad): padding columns
  //      carry zero factors, so they pass zeros through.  Warp 0 solves the
  //      real part and warp 1 the imaginary part of the right-hand side with
  //      the same real factor: on GB300 each SM sub-partition retires about
  //      one FP64 warp instruction per 64 cycles, so the two components run
  //      on two sub-partitions with one DFMA per step each.
  //      Chunks are SOLVE_CHUNK = 32 columns, aligned with the 32-lane window:
  //      within a chunk, step jj is owned by lane jj and lane l sits
  //      (l - jj) mod 32 rows below the pivot row (forward) or (jj - l) mod 32
  //      rows above the diagonal (backward).  The per-step dependency chain
  //      is one shuffle + one FMA; coefficients, pivots and the next window
  //      element are loaded ahead of use and merged with predicated selects.
  //      Both warps read each ring slot; named barrier 1 (64 threads) at the
  //      top of every chunk both agrees on a timed-out wait and frees the
  //      previous slot for refilling.
  if ((mode == 0 || mode == 3) && active && tid < 64) {
    const int lane = tid & 31;
    const int comp = tid >> 5;                 // 0: real part, 1: imaginary part
    double* Bd = reinterpret_cast<double*>(sm.B) + comp;   // element j at Bd[2 j]
    int doneL = 0, doneU = 0;                  // chunks consumed
    bool ok = true;
    auto chunk_sync = [&](uint64_t* bar, int k, int& done) -> bool {
      const bool got = bounded_wait(bar, (k / SOLVE_RING) & 1);
      if (!got) atomicOr(sm.abort_flag, 1);
      if (half == 0)
        asm volatile("bar.sync 1, 64;" ::: "memory");
      else
        asm volatile("bar.sync 2, 64;" ::: "memory");
      if (*sm.abort_flag) return false;
      done = k + 1;
      return true;
    };
    // forward: row interchanges and unit-lower multipliers.  With fwd16 and
    // kl <= 15 warp 0 carries both parts in two 16-lane windows (lanes 0-15
    // the real, 16-31 the imaginary part): one DFMA instruction per row for
    // both, half the FP64 issue of a 32-lane window per part, the same
    // arithmetic per element.  Warp 1 still joins every chunk's barrier
    // (ring slots).  Batched: 6.36 -> 5.72 ms per 64-instance step; a lone
    // 512 x 256 solve, bound by its chain latency, went 0.295 -> 0.309 ms.
    if (a.fwd16 && a.kl <= 15) {
      const int hl = lane & 15, hb = lane & 16;
      double* Bh = reinterpret_cast<double*>(sm.B) + (lane >> 4);   // this half's part
      double v = Bh[2 * hl];          // window element b[j + ((hl - j) & 15)]
      double nv = Bh[2 * (hl + 16)];  // the element this lane takes next
      double vs = v;
      for (int c = 0; c < nchunks; ++c) {
        const int s = c % SOLVE_RING;
        if (!chunk_sync(&sm.barL[s], c, doneL)) { ok = false; break; }
        if (tid == 0 && c >= 1 && c - 1 + SOLVE_RING < nchunks) {
          fence_proxy_async();
          issue_L(c - 1 + SOLVE_RING);   // both warps are past chunk c - 1
        }
        if (comp != 0) continue;
        const double* Lc = sm.Lring + (size_t)s * SOLVE_CHUNK * a.lpad;
        const uint32_t* Pw = reinterpret_cast<const uint32_t*>(sm.Pring + (size_t)s * SOLVE_CHUNK);
        const int j0 = c * SOLVE_CHUNK;
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
          const int off = (Pw[jj >> 2] >> (8 * (jj & 3))) & 0xff;
          const int q = jj & 15;
          const int pl = ((q + off) & 15) | hb;
          const int d = (hl - q) & 15;
          const double l = (d >= 1 && d <= a.kl) ? Lc[jj * a.lpad + d - 1] : 0.0;
          const double bj = __shfl_sync(0xffffffffu, vs, pl);        // pivot row value = y_j
          const double vo = __shfl_sync(0xffffffffu, vs, q | hb);    // old b_j moves to the pivot row
          const double nxt = Bh[2 * (j0 + jj + 32)];
          v = (lane == pl) ? vo : v;
          v = fma(-l, bj, v);
          vs = v;
          const bool own = (hl == q);
          if (own) Bh[2 * (j0 + jj)] = bj;
          v = own ? nv : v;
          nv = own ? nxt : nv;
        }
      }
    } else {
      double v = Bd[2 * lane];          // window element b[j + ((lane - j) & 31)]
      double nv = Bd[2 * (lane + 32)];  // the element this lane takes next
      // shuffle source: v before the owner lane swaps in its next element --
      // the shuffles of a step read the pivot lane and lane jj, never the
      // previous step's owner, so the swap stays off the dependency chain
      double vs = v;
      for (int c = 0; c < nchunks; ++c) {
        const int s = c % SOLVE_RING;
        if (!chunk_sync(&sm.barL[s], c, doneL)) { ok = false; break; }
        if (tid == 0 && c >= 1 && c - 1 + SOLVE_RING < nchunks) {
          fence_proxy_async();
          issue_L(c - 1 + SOLVE_RING);   // both warps are past chunk c - 1
        }
        const double* Lc = sm.Lring + (size_t)s * SOLVE_CHUNK * a.lpad;
        const uint32_t* Pw = reinterpret_cast<const uint32_t*>(sm.Pring + (size_t)s * SOLVE_CHUNK);
        const int j0 = c * SOLVE_CHUNK;
#pragma unroll
        for (int jj = 0; jj < 32; ++jj) {
          const int off = (Pw[jj >> 2] >> (8 * (jj & 3))) & 0xff;
          const int pl = (jj + off) & 31;
          const int d = (lane - jj) & 31;
          const double l = (d >= 1 && d <= a.kl) ? Lc[jj * a.lpad + d - 1] : 0.0;
          const double bj = __shfl_sync(0xffffffffu, vs, pl);  // pivot row value = y_j
          const double vo = __shfl_sync(0xffffffffu, vs, jj);  // old b_j moves to the pivot row
          const double nxt = Bd[2 * (j0 + jj + 64)];   // same address in every lane
          v = (lane == pl) ? vo : v;
          v = fma(-l, bj, v);
          vs = v;
          const bool own = (lane == jj);
          if (own) Bd[2 * (j0 + jj)] = bj;
          v = own ? nv : v;
          nv = own ? nxt : nv;
        }
      }
    }
    // both parts' y in B before either warp's back substitution
    if (half == 0)
      asm volatile("bar.sync 1, 64;" ::: "memory");
    else
      asm volatile("bar.sync 2, 64;" ::: "memory");
    // backward: scaled U columns (U_{j-t,j}/U_jj), window of 32*RU entries;
    // x_j = b_j / U_jj is applied once per chunk, lane l to row j0 + l
    // (mode 3 stops after the forward pass: y is in B)
    if (mode == 0) {
    constexpr int W = 32 * RU;
    const double* rdp = a.rd + (size_t)pp * a.npad;
    const int npad = a.npad;
    double w[RU], nw[RU];
#pragma unroll
    for (int r = 0; r < RU; ++r) {
      // the row of [npad - W, npad) congruent to lane + 32 r (mod W): slot
      // (lane, r) always holds rows of that residue (npad is a multiple of
      // 32 but not necessarily of W)
      const int base = npad - W;
      const int i = base + ((lane + 32 * r - base) & (W - 1));
      w[r] = (ok && i >= 0) ? Bd[2 * i] : 0.0;
      nw[r] = (ok && i - W >= 0) ? Bd[2 * (i - W)] : 0.0;
    }
    double ws = w[0];   // RU = 1: shuffle source before the owner's swap (as vs above)
    for (int k = 0; ok && k < nchunks; ++k) {
      const int s = k % SOLVE_RING;
      if (!chunk_sync(&sm.barU[s], k, doneU)) { ok = false; break; }
      if (tid == 0 && k >= 1 && k - 1 + SOLVE_RING < nchunks) {
        fence_proxy_async();
        issue_U(k - 1 + SOLVE_RING);
      }
      const double* Uc = sm.Uring + (size_t)s * SOLVE_CHUNK * a.upad;
      const int j0 = (nchunks - 1 - k) * SOLVE_CHUNK;
      const double rdl = rdp[j0 + lane];   // used after the chunk: off the chain
      double xo = 0.0;
#pragma unroll
      for (int jj = 31; jj >= 0; --jj) {
        const int j = j0 + jj;
        const double* Ucol = Uc + jj * a.upad;
        const int oreg = (RU == 1) ? 0 : ((j & (W - 1)) >> 5);
        double src = (RU == 1) ? ws : w[0];
#pragma unroll
        for (int r = 1; r < RU; ++r) src = (oreg == r) ? w[r] : src;
        const double bj = __shfl_sync(0xffffffffu, src, jj);
#pragma unroll
        for (int r = 0; r < RU; ++r) {
          const int t = (j - lane - 32 * r) & (W - 1);
          const double u = (t >= 1) ? Ucol[t] : 0.0;
          w[r] = fma(-u, bj, w[r]);
        }
        if (RU == 1) ws = w[0];
        const double nxt = (j - 2 * W >= 0) ? Bd[2 * (j - 2 * W)] : 0.0;   // same address in every lane
        const bool own = (lane == jj);
        xo = own ? bj : xo;
#pragma unroll
        for (int r = 0; r < RU; ++r) {
          const bool take = own && (oreg == r);
          w[r] = take ? nw[r] : w[r];
          nw[r] = take ? nxt : nw[r];
        }
      }
      Bd[2 * (j0 + lane)] = xo * rdl;
    }
    }
    if (!ok && tid == 0) {
      // report, then let every copy in flight land before the CTA exits
      raise_status(a.status, SP_ERR_TIMEOUT, p);
      // chunks issued: RING up front, then chunk q - 1 + RING at the top of chunk q
      const int issL = min(nchunks, doneL == 0 ? SOLVE_RING : doneL - 1 + SOLVE_RING);
      const int issU = mode == 0 ? min(nchunks, doneU == 0 ? SOLVE_RING : doneU - 1 + SOLVE_RING) : 0;
      for (int q = doneL; q < issL; ++q) bounded_wait(&sm.barL[q % SOLVE_RING], (q / SOLVE_RING) & 1);
      for (int q = doneU; q < issU; ++q) bounded_wait(&sm.barU[q % SOLVE_RING], (q / SOLVE_RING) & 1);
    }
  }
  __syncthreads();
  const bool work = active && !*sm.abort_flag;
  if (mode == 3) {
    // y = L^-1 P B~ for the partitioned back substitution
    for (int r = tid; work && r < n; r += nt) a.yg[prow + r] = sm.B[r];
    return;
  }

  // ---- epilogue: store X~, recombine to T coefficients, optional M~ X~
  bool finite = true;
  for (int r = tid; work && r < n; r += nt) {
    const double2 x = sm.B[r];
    finite = finite && dfinite(x.x) && dfinite(x.y);
    if (a.xt_out) a.xt_out[prow + r] = x;
  }
  if (a.xc_out) {
    for (int idx = tid; work && idx < a.S * Nz; idx += nt) {
      const int v = div_idx(idx, invNz), m = idx - v * Nz;
      double2 x = sm.B[a.col_map[idx]];
      if (a.var_recombine[v] && m + 2 < Nz) {
        const double2 x2 = sm.B[a.col_map[idx + 2]];
        x.x -= x2.x;
        x.y -= x2.y;
      }
      const double2 xv = cipow_d(x, a.var_phase[v]);
      a.xc_out[((size_t)v * a.P + p) * Nz + m] = xv;
      if (a.xc32_out) a.xc32_out[((size_t)v * a.P + p) * Nz + m] = make_float2((float)xv.x, (float)xv.y);
      if (a.xs32_out) {
        a.xs32_out[(((size_t)v * a.P + p) * 2) * Nz + m] = (float)xv.x;
        a.xs32_out[(((size_t)v * a.P + p) * 2 + 1) * Nz + m] = (float)xv.y;
      }
    }
  }
  if (a.ep_mv_vals) {
    const double* vals = a.ep_mv_vals + (size_t)p * a.ep_nnz;
    const bool listed = a.ep_rows != nullptr;
    if (listed) {
      // rows without entries first (zero, or B~/beta for L~X~ from the
      // stage right-hand side), then the listed rows with every lane on a
      // row that has entries; the barrier orders the two stores of a row
      for (int r = tid; work && r < n; r += nt) {
        double2 s = make_double2(0.0, 0.0);
        if (mode == 2 && a.ep_from_b != 0.0) {
          const double2 bb = a.bg[prow + r];
          s.x = bb.x * a.ep_from_b;
          s.y = bb.y * a.ep_from_b;
        }
        a.ep_mv_store[prow + r] = s;
      }
      __syncthreads();
    }
    const int nrows = listed ? a.ep_nrows : n;
    for (int i = tid; work && i < nrows; i += nt) {
      const int r = listed ? a.ep_rows[i] : i;
      double2 s = make_double2(0.0, 0.0);
      for (int e = a.ep_indptr[r]; e < a.ep_indptr[r + 1]; ++e) {
        const double m = vals[e];
        double2 x = sm.B[a.ep_indices[e]];
        if (a.ep_mv_addvec) {
          const double2 y = a.ep_mv_addvec[prow + a.ep_indices[e]];
          x.x += y.x;
          x.y += y.y;
        }
        s.x = fma(m, x.x, s.x);
        s.y = fma(m, x.y, s.y);
      }
      if (mode == 2 && a.ep_from_b != 0.0) {
        // L~ X~ = (B~ - alpha M~ X~) / beta for the stage matrix alpha M~ + beta L~
        const double2 bb = a.bg[prow + r];
        s.x = (bb.x - a.ep_alpha * s.x) * a.ep_from_b;
        s.y = (bb.y - a.ep_alpha * s.y) * a.ep_from_b;
      }
      a.ep_mv_store[prow + r] = s;
    }
  }
  if (!finite) raise_status(a.status, SP_ERR_NONFINITE, p);
}

// 256 threads: two pencils' CTAs fit on one SM (registers capped at 128 per
// thread), and the assembly and epilogue, bound by dependent global loads,
// run twice as wide as with the two substituting warps' 128
constexpr int SOLVE_THREADS = 256;
template <int RU, int PPC>
__global__ void __launch_bounds__(SOLVE_THREADS, 2) k_pencil_solve(SolveArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  pencil_solve_body<RU, PPC, -1, SOLVE_THREADS>(a, blockIdx.x, smem_raw);
}
// 128 threads, three CTAs per SM: for more pencils than two CTAs per SM
// hold, more concurrent chains outweigh the narrower assembly and epilogue
template <int RU>
__global__ void __launch_bounds__(128, 3) k_pencil_solve_narrow(SolveArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  pencil_solve_body<RU, 1, -1, 128>(a, blockIdx.x, smem_raw);
}

// right-hand-side assembly only (MODE 1) or epilogue only (MODE 2), around
// k_pencil_lanes: shared memory for B~ alone, several CTAs per SM
template <int MODE>
__global__ void __launch_bounds__(128, 6) k_pencil_stage(SolveArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  pencil_solve_body<1, 1, MODE>(a, blockIdx.x, smem_raw);
}

// the same with 512-thread CTAs, for problems with few pencils (one CTA
// per pencil would leave most of the GPU idle at 128 threads)
template <int MODE>
__global__ void __launch_bounds__(512, 2) k_pencil_stage_wide(SolveArgs a) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  pencil_solve_body<1, 1, MODE, 512>(a, blockIdx.x, smem_raw);
}

// a batch of problems: work item (problem, pencil) per CTA
template <int RU>
// (one CTA per pencil: its items are long dependent chains, so a
// persistent grid buys nothing here; 128 registers keep three CTAs per SM)
__global__ void __launch_bounds__(128, 4) k_pencil_solve_batched(const SolveArgs* __restrict__ args,
                                                                 const int4* __restrict__ work) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int4 w = work[blockIdx.x];
  pencil_solve_body<RU, 1>(args[w.x], w.y, smem_raw);
}

size_t pencil_solve_smem(int npad, int lpad, int upad) { return solve_smem_bytes(npad, lpad, upad); }

cudaError_t launch_pencil_solve_batched(cudaStream_t s, const SolveArgs* args, const int4* work, int nwork,
                                        int max_kuu, size_t smem) {
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  if (max_kuu <= 31) {
    cudaFuncSetAttribute(k_pencil_solve_batched<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_pencil_solve_batched<1><<<nwork, 128, smem, s>>>(args, work);
  } else {
    cudaFuncSetAttribute(k_pencil_solve_batched<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_pencil_solve_batched<2><<<nwork, 128, smem, s>>>(args, work);
  }
  return cudaGetLastError();
}

cudaError_t launch_pencil_solve(cudaStream_t s, const SolveArgs& args) {
  SolveArgs a = args;
  fill_f_halves(a);
  if (a.mode == 1 || a.mode == 2) {
    const size_t smem = solve_smem_bytes(a.npad, 0, 0);
    if (smem > 227 * 1024) return cudaErrorInvalidValue;
    if (a.P < 2 * 152) {
      if (a.mode == 1) {
        cudaFuncSetAttribute(k_pencil_stage_wide<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_pencil_stage_wide<1><<<a.P, 512, smem, s>>>(a);
      } else {
        cudaFuncSetAttribute(k_pencil_stage_wide<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        k_pencil_stage_wide<2><<<a.P, 512, smem, s>>>(a);
      }
      return cudaGetLastError();
    }
    if (a.mode == 1) {
      cudaFuncSetAttribute(k_pencil_stage<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_pencil_stage<1><<<a.P, 128, smem, s>>>(a);
    } else {
      cudaFuncSetAttribute(k_pencil_stage<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_pencil_stage<2><<<a.P, 128, smem, s>>>(a);
    }
    return cudaGetLastError();
  }
  constexpr int PPC = 1;
  const size_t smem = PPC * solve_smem_bytes(a.npad, a.lpad, a.upad);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  const int grid = (a.P + PPC - 1) / PPC;
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0) sms = 1;
  }
  // three CTAs of 128 threads per SM (228 KB of shared memory, 1 KB of it
  // reserved per CTA) when the pencils fill more than one wave of two
  if (a.P > 2 * sms && 3 * (smem + 1024) <= 228 * 1024) {
    if (a.kuu <= 31) {
      cudaFuncSetAttribute(k_pencil_solve_narrow<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_pencil_solve_narrow<1><<<grid, 128, smem, s>>>(a);
    } else {
      cudaFuncSetAttribute(k_pencil_solve_narrow<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_pencil_solve_narrow<2><<<grid, 128, smem, s>>>(a);
    }
    return cudaGetLastError();
  }
  if (a.kuu <= 31) {
    cudaFuncSetAttribute(k_pencil_solve<1, PPC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_pencil_solve<1, PPC><<<grid, SOLVE_THREADS, smem, s>>>(a);
  } else {
    cudaFuncSetAttribute(k_pencil_solve<2, PPC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_pencil_solve<2, PPC><<<grid, SOLVE_THREADS, smem, s>>>(a);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Lane-per-pencil substitution for problems with many pencils (3D): the
// window kernel above keeps one pencil's band across a warp's lanes, which
// leaves most lanes idle in the forward pass (kl of 32) and, with two window
// registers, in the back substitution (kl + ku of 64); it is the right shape
// when a few hundred dependent chains cannot fill the GPU anyway.  With tens
// of thousands of pencils the FP64 pipe is the limit instead, so here each
// lane carries one real right-hand side (lane 2i: real part, 2i + 1:
// imaginary part of pencil i of a group of LANE_GROUP) through the whole
// substitution with its window of pending rows in registers; every warp
// FMA does useful work on all 32 lanes.  The factor is stored interleaved
// by pencil within a group, so a warp's load of one factor entry reads 16
// consecutive doubles.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait2() { asm volatile("cp.async.wait_group 2;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Rows staged ahead in the lane substitution: LANE_BUFS buffers, the copy
// of row j + LANE_BUFS - 1 in flight while row j is used
constexpr int LANE_BUFS = 3;

// doubles of shared memory per warp: LANE_BUFS forward buffers (multipliers
// and pivots) or LANE_BUFS backward buffers (listed U entries), whichever is
// larger
__host__ __device__ inline int lane_stride(int kl, int cmax) {
  const int fw = LANE_BUFS * (kl * LANE_GROUP + 2), bw = LANE_BUFS * cmax * LANE_GROUP;
  return fw > bw ? fw : bw;
}

template <int KL, int KUU>
__global__ void __launch_bounds__(128) k_pencil_lanes(int P, int n, int cmax, const double* __restrict__ Lg,
                                                      const double* __restrict__ Uc,
                                                      const uint8_t* __restrict__ pg,
                                                      const unsigned long long* __restrict__ umask,
                                                      const double2* __restrict__ b, double2* __restrict__ y,
                                                      double2* __restrict__ x) {
  extern __shared__ __align__(16) double lane_stage[];   // [warp][2][cmax][LANE_GROUP]
  const int gl = blockIdx.x * blockDim.x + threadIdx.x;
  const int comp = gl & 1;
  const int pen = gl >> 1;                       // pencil; a warp holds the 16 pencils of one group
  const bool act = pen < P;                      // idle lanes of the last group keep the warp's rhythm
  const int g = pen / LANE_GROUP, i = pen - g * LANE_GROUP;
  if (g * LANE_GROUP >= P) return;               // a whole warp past the last group (no storage there)
  const int lane = threadIdx.x & 31;
  const double* bp = reinterpret_cast<const double*>(b + (size_t)(act ? pen : 0) * n) + comp;
  double* yp = reinterpret_cast<double*>(y + (size_t)g * n * LANE_GROUP + i) + comp;   // row j at yp[2 j LANE_GROUP]
  const size_t gn = (size_t)g * n;
  // per-warp staging area (lane_stride doubles): forward rows, then backward rows
  double* st = lane_stage + (size_t)(threadIdx.x >> 5) * lane_stride(KL, cmax);
  // forward: row interchanges and unit-lower multipliers; win[t] = row j + t.
  // Each row's multipliers and pivot offsets for the warp's 16 pencils are
  // copied into shared memory two rows ahead (cp.async, three buffers).
  constexpr int FW = KL * LANE_GROUP + 2;        // doubles per forward buffer (+16 bytes of pivots)
  auto fstage = [&](int jr) {
    const double* src = Lg + (gn + jr) * KL * LANE_GROUP;
    double* dst = st + (jr % LANE_BUFS) * FW;
    for (int c = lane; c < KL * (LANE_GROUP / 2); c += 32) cp_async16(dst + 2 * c, src + 2 * c);
    if (lane == 31) cp_async16(dst + KL * LANE_GROUP, pg + (gn + jr) * LANE_GROUP);
    cp_async_commit();
  };
  {
    double win[KL + 1];
#pragma unroll
    for (int t = 0; t <= KL; ++t) win[t] = (act && t < n) ? bp[2 * t] : 0.0;
    fstage(0);
    if (n > 1) fstage(1);
    else cp_async_commit();
    for (int j = 0; j < n; ++j) {
      if (j + 2 < n) fstage(j + 2);
      else cp_async_commit();                    // one group per row keeps wait_group 2 exact
      cp_async_wait2();
      __syncwarp();
      const double* Ls = st + (j % LANE_BUFS) * FW;
      const int off = reinterpret_cast<const uint8_t*>(Ls + KL * LANE_GROUP)[i];
      const double* Lrow = Ls + i;
      double piv_val = win[0];
#pragma unroll
      for (int t = 1; t <= KL; ++t) piv_val = (off == t) ? win[t] : piv_val;
#pragma unroll
      for (int t = 1; t <= KL; ++t) win[t] = (off == t) ? win[0] : win[t];
      const double yj = piv_val;
      yp[(size_t)2 * j * LANE_GROUP] = yj;
#pragma unroll
      for (int t = 1; t <= KL; ++t) win[t] = fma(-Lrow[(t - 1) * LANE_GROUP], yj, win[t]);
#pragma unroll
      for (int t = 0; t < KL; ++t) win[t] = win[t + 1];
      win[KL] = (act && j + KL + 1 < n) ? bp[2 * (j + KL + 1)] : 0.0;
      __syncwarp();                              // buffer j % 3 is refilled for row j + 3 next
    }
    cp_async_wait0();
    __syncwarp();
  }
  // back substitution with the scaled columns U_{j-t,j} / U_jj.  Only entries
  // nonzero in some pencil are stored: the k-th set bit t of umask[j] holds
  // U_{j-t,j} / U_jj at Uc[g][j][k] (k = 0: 1/U_jj).  Each row's entries
  // are copied into shared memory two rows ahead (cp.async, three buffers per
  // warp), and only the listed entries issue an FMA: the mask is the same for
  // the whole warp, so the loop branches (a predicated-off FP64 instruction
  // would still hold the FP64 pipe) and jumps to the FMA of its window
  // register.  The rows of y this lane wrote are read back by this lane only.
  auto stage = [&](int jr) {
    const int cnt = __popcll(umask[jr]);
    const double* src = Uc + (gn + jr) * (size_t)cmax * LANE_GROUP;
    double* dst = st + (jr % LANE_BUFS) * cmax * LANE_GROUP;
    for (int c = lane; c < cnt * (LANE_GROUP / 2); c += 32) cp_async16(dst + 2 * c, src + 2 * c);
    cp_async_commit();
  };
  double w[KUU + 1];                             // w[t] = pending row j - t
#pragma unroll
  for (int t = 0; t <= KUU; ++t) w[t] = (act && n - 1 - t >= 0) ? yp[(size_t)2 * (n - 1 - t) * LANE_GROUP] : 0.0;
  double* xp = reinterpret_cast<double*>(x + (size_t)(act ? pen : 0) * n) + comp;
  stage(n - 1);
  if (n > 1) stage(n - 2);
  else cp_async_commit();
  for (int j = n - 1; j >= 0; --j) {
    if (j >= 2) stage(j - 2);
    else cp_async_commit();                      // one group per row keeps wait_group 2 exact
    cp_async_wait2();
    __syncwarp();
    const double* vals = st + (j % LANE_BUFS) * cmax * LANE_GROUP + i;
    const unsigned long long m = umask[j];
    const double bj = w[0];
    if (act) xp[2 * j] = bj * vals[0];
    unsigned long long mm = m & ~1ull;
    int k = 1;
    while (mm) {
      const int t = __ffsll((long long)mm) - 1;
      mm &= mm - 1;
      const double ut = vals[(k++) * LANE_GROUP];
      switch (t) {
#define SP_LANE_CASE(T)                          \
  case T:                                        \
    if (T <= KUU) w[T] = fma(-ut, bj, w[T]);    \
    break;
        SP_LANE_CASE(1)
        SP_LANE_CASE(2)
        SP_LANE_CASE(3)
        SP_LANE_CASE(4)
        SP_LANE_CASE(5)
        SP_LANE_CASE(6)
        SP_LANE_CASE(7)
        SP_LANE_CASE(8)
        SP_LANE_CASE(9)
        SP_LANE_CASE(10)
        SP_LANE_CASE(11)
        SP_LANE_CASE(12)
        SP_LANE_CASE(13)
        SP_LANE_CASE(14)
        SP_LANE_CASE(15)
        SP_LANE_CASE(16)
        SP_LANE_CASE(17)
        SP_LANE_CASE(18)
        SP_LANE_CASE(19)
        SP_LANE_CASE(20)
        SP_LANE_CASE(21)
        SP_LANE_CASE(22)
        SP_LANE_CASE(23)
        SP_LANE_CASE(24)
        SP_LANE_CASE(25)
        SP_LANE_CASE(26)
        SP_LANE_CASE(27)
        SP_LANE_CASE(28)
        SP_LANE_CASE(29)
        SP_LANE_CASE(30)
        SP_LANE_CASE(31)
        SP_LANE_CASE(32)
        SP_LANE_CASE(33)
        SP_LANE_CASE(34)
        SP_LANE_CASE(35)
        SP_LANE_CASE(36)
        SP_LANE_CASE(37)
        SP_LANE_CASE(38)
        SP_LANE_CASE(39)
        SP_LANE_CASE(40)
        SP_LANE_CASE(41)
        SP_LANE_CASE(42)
        SP_LANE_CASE(43)
        SP_LANE_CASE(44)
        SP_LANE_CASE(45)
        SP_LANE_CASE(46)
        SP_LANE_CASE(47)
        SP_LANE_CASE(48)
        SP_LANE_CASE(49)
        SP_LANE_CASE(50)
        SP_LANE_CASE(51)
        SP_LANE_CASE(52)
        SP_LANE_CASE(53)
        SP_LANE_CASE(54)
        SP_LANE_CASE(55)
        SP_LANE_CASE(56)
        SP_LANE_CASE(57)
        SP_LANE_CASE(58)
        SP_LANE_CASE(59)
        SP_LANE_CASE(60)
        SP_LANE_CASE(61)
        SP_LANE_CASE(62)
        SP_LANE_CASE(63)
#undef SP_LANE_CASE
        default:
          break;
      }
    }
#pragma unroll
    for (int t = 0; t < KUU; ++t) w[t] = w[t + 1];
    const int row = j - KUU - 1;
    w[KUU] = (act && row >= 0) ? yp[(size_t)2 * row * LANE_GROUP] : 0.0;
    __syncwarp();                                // buffer j % 3 is refilled for row j - 3 next
  }
  cp_async_wait0();
}

bool lanes_supported(int kl, int kuu) { return (kl == 9 && kuu == 38) || (kl == 7 && kuu == 29); }

cudaError_t launch_pencil_lanes(cudaStream_t s, int P, int n, int kl, int kuu, const double* Lg, const double* Uc,
                                int cmax, const uint8_t* pg, const unsigned long long* umask, const double2* b,
                                double2* y, double2* x) {
  const int threads = 2 * P;
  const int grid = (threads + 127) / 128;
  const size_t smem = (size_t)4 * lane_stride(kl, cmax) * sizeof(double);
  cudaError_t e = cudaSuccess;
  if (kl == 9 && kuu == 38) {
    if ((e = cudaFuncSetAttribute(k_pencil_lanes<9, 38>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) ==
        cudaSuccess)
      k_pencil_lanes<9, 38><<<grid, 128, smem, s>>>(P, n, cmax, Lg, Uc, pg, umask, b, y, x);
  } else if (kl == 7 && kuu == 29) {
    if ((e = cudaFuncSetAttribute(k_pencil_lanes<7, 29>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) ==
        cudaSuccess)
      k_pencil_lanes<7, 29><<<grid, 128, smem, s>>>(P, n, cmax, Lg, Uc, pg, umask, b, y, x);
  } else {
    return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  return cudaGetLastError();
}

__global__ void k_u_mask(int P, int n, int npad, int kuu, int upad, const double* __restrict__ U,
                         unsigned long long* __restrict__ umask) {
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= (size_t)P * n) return;
  const int p = (int)(idx / n), j = (int)(idx - (size_t)p * n);
  const double* col = U + ((size_t)p * npad + j) * upad;
  unsigned long long m = 1ull;
  for (int t = 1; t <= kuu; ++t)
    if (col[t] != 0.0) m |= 1ull << t;
  if ((m & ~umask[j]) != 0ull) atomicOr(umask + j, m);
}

cudaError_t launch_u_mask(cudaStream_t s, int P, int n, int npad, int kuu, int upad, const double* U,
                          unsigned long long* umask) {
  if (kuu > 63) return cudaErrorInvalidValue;
  const size_t total = (size_t)P * n;
  k_u_mask<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(P, n, npad, kuu, upad, U, umask);
  return cudaGetLastError();
}

// Copy a factor into the lane layout (one thread per pencil row): dense
// multipliers and pivots, and the U entries listed in umask[j] in order of t.
__global__ void k_factor_relayout(int P, int n, int npad, int kl, int kuu, int lpad, int upad, int cmax,
                                  const double* __restrict__ L, const uint8_t* __restrict__ piv,
                                  const double* __restrict__ U, const unsigned long long* __restrict__ umask,
                                  double* __restrict__ Lg, double* __restrict__ Uc, uint8_t* __restrict__ pg) {
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= (size_t)P * n) return;
  const int p = (int)(idx / n), j = (int)(idx - (size_t)p * n);
  const int g = p / LANE_GROUP, i = p - g * LANE_GROUP;
  const size_t row = (size_t)g * n + j;
  for (int t = 0; t < kl; ++t) Lg[(row * kl + t) * LANE_GROUP + i] = L[((size_t)p * npad + j) * lpad + t];
  const double* col = U + ((size_t)p * npad + j) * upad;
  const unsigned long long m = umask[j];
  int k = 0;
  for (int t = 0; t <= kuu && k < cmax; ++t)
    if ((m >> t) & 1ull) Uc[(row * cmax + k++) * LANE_GROUP + i] = col[t];
  pg[row * LANE_GROUP + i] = piv[(size_t)p * npad + j];
}

cudaError_t launch_factor_relayout(cudaStream_t s, int P, int n, int npad, int kl, int kuu, int lpad, int upad,
                                   const BandFactor& f) {
  const size_t total = (size_t)P * n;
  k_factor_relayout<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(P, n, npad, kl, kuu, lpad, upad, f.cmax, f.L,
                                                                   f.piv, f.U, f.umask, f.Lg, f.Ug, f.pg);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// state conversion and Chebyshev derivative (set-up kernels)
// ---------------------------------------------------------------------------
// x~ = i^{-q_v} (P^R)^{-1} x : recombined variables invert x_m = x~_m - x~_{m+2}
__global__ void k_coef_to_solve(int P, int S, int Nz, const double2* __restrict__ xc, double2* __restrict__ xt,
                                const int32_t* __restrict__ col_map, const int32_t* __restrict__ rec,
                                const int32_t* __restrict__ ph) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= P * S) return;
  const int v = idx / P, p = idx - v * P;
  const double2* x = xc + ((size_t)v * P + p) * Nz;
  double2* out = xt + (size_t)p * S * Nz;
  double2 t1 = make_double2(0.0, 0.0), t2 = make_double2(0.0, 0.0);  // x~_{m+1}, x~_{m+2}
  for (int m = Nz - 1; m >= 0; --m) {
    double2 y = cipow<double>(x[m], -ph[v]);
    if (rec[v]) { y.x += t2.x; y.y += t2.y; }
    out[col_map[v * Nz + m]] = y;
    t2 = t1;
    t1 = y;
  }
}

cudaError_t launch_coef_to_solve(cudaStream_t s, int P, int S, int Nz, const double2* xc, double2* xt,
                                 const int32_t* col_map, const int32_t* var_recombine,
                                 const int32_t* var_phase) {
  const int total = P * S;
  k_coef_to_solve<<<(total + 127) / 128, 128, 0, s>>>(P, S, Nz, xc, xt, col_map, var_recombine, var_phase);
  return cudaGetLastError();
}

// c'_{m} = c'_{m+2} + 2 (m+1) c_{m+1}, c'_0 halved, times 2/(b-a)
__global__ void k_dz(int P, int Nz, double scale, const double2* __restrict__ src, double2* __restrict__ dst) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const double2* c = src + (size_t)p * Nz;
  double2* d = dst + (size_t)p * Nz;
  double2 d1 = make_double2(0.0, 0.0), d2 = make_double2(0.0, 0.0);  // d_{m+1}, d_{m+2}
  for (int m = Nz - 1; m >= 0; --m) {
    double2 dm = d2;
    if (m + 1 < Nz) {
      dm.x += 2.0 * (m + 1) * c[m + 1].x;
      dm.y += 2.0 * (m + 1) * c[m + 1].y;
    }
    const double h = (m == 0) ? 0.5 : 1.0;
    d[m] = make_double2(dm.x * h * scale, dm.y * h * scale);
    d2 = d1;
    d1 = dm;
  }
}

__global__ void k_to_f32(const double2* __restrict__ src, float2* __restrict__ dst, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    dst[i] = make_float2((float)src[i].x, (float)src[i].y);
}

cudaError_t launch_to_f32(cudaStream_t s, const double2* src, float2* dst, size_t n) {
  k_to_f32<<<(int)std::min<size_t>((n + 255) / 256, 4096), 256, 0, s>>>(src, dst, n);
  return cudaGetLastError();
}

cudaError_t launch_dz(cudaStream_t s, int P, int Nz, double scale, const double2* src, double2* dst) {
  k_dz<<<(P + 127) / 128, 128, 0, s>>>(P, Nz, scale, src, dst);
  return cudaGetLastError();
}


// ---------------------------------------------------------------------------
// adjoint-step helpers (discrete adjoint of the RK IMEX step)
// ---------------------------------------------------------------------------
// F-bar[slot][p][n] from row-space pencil vectors: the transpose of the
// right-hand-side placement (row_map), of the equation phase i^{-q_e}, of the
// T-to-U conversion with its dropped tau row, and of the forward Chebyshev
// weights (2 - delta_n0)/N_g (so that a plain backward transform follows):
//   u_m = i^{q_e} sum_k c_k v_k[row(e, m)]
//   differential: F_n = (u_n - u_{n-2}) / N_g;  algebraic: F_n = u_n (2 - delta_n0) / N_g
__global__ void k_adj_gather(int P, int Nz, int Ng, int n, int nslot, const int32_t* __restrict__ nl_eq,
                             const int32_t* __restrict__ row_map, const int32_t* __restrict__ eq_diff,
                             const int32_t* __restrict__ eq_phase, VecList4 vl, double2* __restrict__ fbar,
                             float2* __restrict__ fbar32) {
  const int p = blockIdx.x;
  const int nvec = vl.n;
  const double2* v[4];
  double c[4];
  for (int k = 0; k < nvec; ++k) { v[k] = vl.p[k] + (size_t)p * n; c[k] = vl.c[k]; }
  auto u_at = [&](int e, int m) -> double2 {
    const int row = row_map[e * Nz + m];
    if (row < 0) return make_double2(0.0, 0.0);
    double2 acc = make_double2(0.0, 0.0);
    for (int k = 0; k < nvec; ++k) {
      const double2 x = v[k][row];
      acc.x = fma(c[k], x.x, acc.x);
      acc.y = fma(c[k], x.y, acc.y);
    }
    return cipow_d(acc, eq_phase[e]);
  };
  const double inv = 1.0 / Ng;
  for (int idx = threadIdx.x; idx < nslot * Nz; idx += blockDim.x) {
    const int sl = idx / Nz, m = idx - sl * Nz;
    const int e = nl_eq[sl];
    double2 f;
    if (eq_diff[e]) {
      const double2 u0 = u_at(e, m);
      const double2 u2 = (m >= 2) ? u_at(e, m - 2) : make_double2(0.0, 0.0);
      f = make_double2((u0.x - u2.x) * inv, (u0.y - u2.y) * inv);
    } else {
      const double2 u0 = u_at(e, m);
      const double w = (m == 0 ? 1.0 : 2.0) * inv;
      f = make_double2(u0.x * w, u0.y * w);
    }
    const size_t o = ((size_t)sl * P + p) * Nz + m;
    fbar[o] = f;
    if (fbar32) fbar32[o] = make_float2((float)f.x, (float)f.y);
  }
}

cudaError_t launch_adj_gather(cudaStream_t s, int P, int Nz, int Ng, int n, int nslot, const int32_t* nl_eq,
                              const int32_t* row_map, const int32_t* eq_diff, const int32_t* eq_phase,
                              int nvec, const double2* const* vecs, const double* coefs, double2* fbar,
                              float2* fbar32) {
  if (nvec > 4) return cudaErrorInvalidValue;
  VecList4 vl{};
  vl.n = nvec;
  for (int k = 0; k < nvec; ++k) { vl.p[k] = vecs[k]; vl.c[k] = coefs[k]; }
  k_adj_gather<<<P, 256, 0, s>>>(P, Nz, Ng, n, nslot, nl_eq, row_map, eq_diff, eq_phase, vl, fbar, fbar32);
  return cudaGetLastError();
}

// out[p][col(v, m)] = i^{-q_v} (Xb_v[m] - rec_v Xb_v[m-2]) + sum_k a_k add_k[p][col(v, m)],
// Xb_v = sum over grid fields f of variable v of op_f^H xbar_f  (op DX: -i k_x)
__global__ void k_adj_combine(int P, int Nz, int S, int n, int nf, const int32_t* __restrict__ f_var,
                              const int32_t* __restrict__ f_op, const double* __restrict__ kx,
                              const double2* __restrict__ xbar, const int32_t* __restrict__ col_map,
                              const int32_t* __restrict__ var_rec, const int32_t* __restrict__ var_phase,
                              VecList4 al, double2* __restrict__ out) {
  const int p = blockIdx.x;
  const double k = kx ? kx[p] : 0.0;
  auto xb = [&](int v, int m) -> double2 {
    double2 acc = make_double2(0.0, 0.0);
    for (int f = 0; f < nf; ++f) {
      if (f_var[f] != v) continue;
      const double2 x = xbar[((size_t)f * P + p) * Nz + m];
      if (f_op[f] == SP_OP_DX) {       // times -i k
        acc.x = fma(k, x.y, acc.x);
        acc.y = fma(-k, x.x, acc.y);
      } else {
        acc.x += x.x;
        acc.y += x.y;
      }
    }
    return acc;
  };
  for (int idx = threadIdx.x; idx < S * Nz; idx += blockDim.x) {
    const int v = idx / Nz, m = idx - v * Nz;
    double2 y = xb(v, m);
    if (var_rec[v] && m >= 2) {
      const double2 y2 = xb(v, m - 2);
      y.x -= y2.x;
      y.y -= y2.y;
    }
    y = cipow_d(y, -var_phase[v]);
    const int c = col_map[idx];
    for (int a = 0; a < al.n; ++a) {
      const double2 z = al.p[a][(size_t)p * n + c];
      y.x = fma(al.c[a], z.x, y.x);
      y.y = fma(al.c[a], z.y, y.y);
    }
    out[(size_t)p * n + c] = y;
  }
}

cudaError_t launch_adj_combine(cudaStream_t s, int P, int Nz, int S, int n, int nf, const int32_t* f_var,
                               const int32_t* f_op, const double* kx, const double2* xbar,
                               const int32_t* col_map, const int32_t* var_rec, const int32_t* var_phase,
                               int nadd, const double2* const* adds, const double* add_coefs, double2* out) {
  if (nadd > 4) return cudaErrorInvalidValue;
  VecList4 al{};
  al.n = nadd;
  for (int k = 0; k < nadd; ++k) { al.p[k] = adds[k]; al.c[k] = add_coefs[k]; }
  k_adj_combine<<<P, 512, 0, s>>>(P, Nz, S, n, nf, f_var, f_op, kx, xbar, col_map, var_rec, var_phase, al, out);
  return cudaGetLastError();
}

// Inverse of the transposed change of variables: Xb_v[m] = i^{q_v} xt[col(v, m)] + rec_v Xb_v[m-2].
// With recombination Xb_v[m] is the sum of the y[j] = i^{q_v} xt[col(v, j)]
// with j <= m of the parity of m.  One warp per (variable, pencil): lane l
// takes modes 64c + 2l (even) and 64c + 2l + 1 (odd) of chunk c, one
// inclusive warp scan per parity adds them up, and the scans' last lane
// carries into the next chunk (a thread per row walking its modes in order
// left the launch waiting on one dependent load chain per row).
__global__ void __launch_bounds__(256) k_adj_tinvh(int P, int Nz, int S, int n, const double2* __restrict__ xt,
                                                   const int32_t* __restrict__ col_map,
                                                   const int32_t* __restrict__ var_rec,
                                                   const int32_t* __restrict__ var_phase, double2* __restrict__ out) {
  const int row = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= P * S) return;                      // whole warps leave together
  const int v = row / P, p = row - v * P;
  const bool rec = var_rec[v] != 0;
  const int q = var_phase[v];
  const double2* xp = xt + (size_t)p * n;
  double2* op = out + ((size_t)v * P + p) * Nz;
  double2 ce = make_double2(0.0, 0.0), co = make_double2(0.0, 0.0);   // carries of the two parities
  for (int c0 = 0; c0 < Nz; c0 += 64) {
    const int me = c0 + 2 * lane, mo = me + 1;
    double2 ye = me < Nz ? cipow_d(xp[col_map[v * Nz + me]], q) : make_double2(0.0, 0.0);
    double2 yo = mo < Nz ? cipow_d(xp[col_map[v * Nz + mo]], q) : make_double2(0.0, 0.0);
    if (rec) {
#pragma unroll
      for (int d = 1; d < 32; d <<= 1) {
        const double ex = __shfl_up_sync(0xffffffffu, ye.x, d), ey = __shfl_up_sync(0xffffffffu, ye.y, d);
        const double ox = __shfl_up_sync(0xffffffffu, yo.x, d), oy = __shfl_up_sync(0xffffffffu, yo.y, d);
        if (lane >= d) {
          ye.x += ex; ye.y += ey;
          yo.x += ox; yo.y += oy;
        }
      }
      ye.x += ce.x; ye.y += ce.y;
      yo.x += co.x; yo.y += co.y;
      ce = make_double2(__shfl_sync(0xffffffffu, ye.x, 31), __shfl_sync(0xffffffffu, ye.y, 31));
      co = make_double2(__shfl_sync(0xffffffffu, yo.x, 31), __shfl_sync(0xffffffffu, yo.y, 31));
    }
    if (me < Nz) op[me] = ye;
    if (mo < Nz) op[mo] = yo;
  }
}

cudaError_t launch_adj_tinvh(cudaStream_t s, int P, int Nz, int S, int n, const double2* xt_bar,
                             const int32_t* col_map, const int32_t* var_rec, const int32_t* var_phase,
                             double2* out) {
  const size_t threads = (size_t)P * S * 32;
  k_adj_tinvh<<<(unsigned)((threads + 255) / 256), 256, 0, s>>>(P, Nz, S, n, xt_bar, col_map, var_rec, var_phase,
                                                                out);
  return cudaGetLastError();
}

// Transpose of the Chebyshev derivative (k_dz): with d = D c,
// D_{ij} = scale 2 j / (1 + delta_i0) for i < j, j - i odd, the adjoint
// c_bar_j += scale 2 j sum_{i < j, j - i odd} d_bar_i / (1 + delta_i0).
__global__ void k_dz_adjoint(int P, int Nz, double scale, const double2* __restrict__ dbar,
                             double2* __restrict__ cbar) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P) return;
  const double2* d = dbar + (size_t)p * Nz;
  double2* c = cbar + (size_t)p * Nz;
  double2 run[2] = {make_double2(0.0, 0.0), make_double2(0.0, 0.0)};   // prefix sums by parity of i
  for (int j = 0; j < Nz; ++j) {
    // sum over i < j with i of parity opposite to j
    const double2 sacc = run[(j + 1) & 1];
    const double f = scale * 2.0 * j;
    c[j] = make_double2(c[j].x + f * sacc.x, c[j].y + f * sacc.y);
    const double w = (j == 0) ? 0.5 : 1.0;
    run[j & 1].x += w * d[j].x;
    run[j & 1].y += w * d[j].y;
  }
}

cudaError_t launch_dz_adjoint(cudaStream_t s, int P, int Nz, double scale, const double2* dst_bar,
                              double2* src_bar) {
  k_dz_adjoint<<<(P + 127) / 128, 128, 0, s>>>(P, Nz, scale, dst_bar, src_bar);
  return cudaGetLastError();
}
// ---------------------------------------------------------------------------
// Inverse iteration for the pencil eigenproblem (L~ + lambda M~) x = 0 with
// shift sigma (Sec. "Eigenvalue solver"): after y = (L~ + sigma M~)^{-1} M~ x
// (the solve kernel), per pencil mu = x^H y / x^H x, and x <- y / |y|;
// lambda = sigma - 1 / mu is the eigenvalue nearest sigma.  One CTA per pencil.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_eig_update(int P, int n, double2* __restrict__ x,
                                                    const double2* __restrict__ y, double2* __restrict__ mu) {
  const int p = blockIdx.x;
  if (p >= P) return;
  double2* xp = x + (size_t)p * n;
  const double2* yp = y + (size_t)p * n;
  double xr = 0, xi = 0, xx = 0, yy = 0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const double2 a = xp[r], b = yp[r];
    xr += a.x * b.x + a.y * b.y;            // conj(a) b
    xi += a.x * b.y - a.y * b.x;
    xx += a.x * a.x + a.y * a.y;
    yy += b.x * b.x + b.y * b.y;
  }
  __shared__ double red[4][8];
  for (int o = 16; o > 0; o >>= 1) {
    xr += __shfl_xor_sync(0xffffffffu, xr, o);
    xi += __shfl_xor_sync(0xffffffffu, xi, o);
    xx += __shfl_xor_sync(0xffffffffu, xx, o);
    yy += __shfl_xor_sync(0xffffffffu, yy, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { red[0][w] = xr; red[1][w] = xi; red[2][w] = xx; red[3][w] = yy; }
  __syncthreads();
  if (threadIdx.x == 0) {
    xr = xi = xx = yy = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
      xr += red[0][k]; xi += red[1][k]; xx += red[2][k]; yy += red[3][k];
    }
    mu[p] = make_double2(xx > 0 ? xr / xx : 0.0, xx > 0 ? xi / xx : 0.0);
    red[0][0] = yy > 0 ? 1.0 / sqrt(yy) : 0.0;
  }
  __syncthreads();
  const double sc = red[0][0];
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    const double2 b = yp[r];
    xp[r] = make_double2(b.x * sc, b.y * sc);
  }
}

// Relative residual of each pencil's eigenpair (sigma_p, x_p) of
// sigma M~ x + L~ x = 0: ||(L~ + sigma M~) x|| / (||L~ x|| + |sigma| ||M~ x||),
// one CTA per pencil, the pencils' CSR values on the shared pattern.
__global__ void __launch_bounds__(256) k_eig_residual(int P, int n, int nnz, const int32_t* __restrict__ indptr,
                                                      const int32_t* __restrict__ indices,
                                                      const double* __restrict__ Mv, const double* __restrict__ Lv,
                                                      const double2* __restrict__ x, const double2* __restrict__ sig,
                                                      double* __restrict__ res) {
  const int p = blockIdx.x;
  if (p >= P) return;
  const double* M = Mv + (size_t)p * nnz;
  const double* L = Lv + (size_t)p * nnz;
  const double2* xp = x + (size_t)p * n;
  const double2 sg = sig[p];
  double rr = 0, ll = 0, mm = 0;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    double2 lx = make_double2(0.0, 0.0), mx = make_double2(0.0, 0.0);
    for (int e = indptr[r]; e < indptr[r + 1]; ++e) {
      const double2 v = xp[indices[e]];
      lx.x = fma(L[e], v.x, lx.x); lx.y = fma(L[e], v.y, lx.y);
      mx.x = fma(M[e], v.x, mx.x); mx.y = fma(M[e], v.y, mx.y);
    }
    const double rx = lx.x + sg.x * mx.x - sg.y * mx.y, ry = lx.y + sg.x * mx.y + sg.y * mx.x;
    rr += rx * rx + ry * ry;
    ll += lx.x * lx.x + lx.y * lx.y;
    mm += mx.x * mx.x + mx.y * mx.y;
  }
  __shared__ double red[3][8];
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_xor_sync(0xffffffffu, rr, o);
    ll += __shfl_xor_sync(0xffffffffu, ll, o);
    mm += __shfl_xor_sync(0xffffffffu, mm, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { red[0][w] = rr; red[1][w] = ll; red[2][w] = mm; }
  __syncthreads();
  if (threadIdx.x == 0) {
    rr = ll = mm = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) { rr += red[0][k]; ll += red[1][k]; mm += red[2][k]; }
    const double den = sqrt(ll) + sqrt(sg.x * sg.x + sg.y * sg.y) * sqrt(mm);
    res[p] = den > 0 ? sqrt(rr) / den : 0.0;
  }
}

cudaError_t launch_eig_residual(cudaStream_t s, int P, int n, int nnz, const int32_t* indptr, const int32_t* indices,
                                const double* Mv, const double* Lv, const double2* x, const double2* sig,
                                double* res) {
  k_eig_residual<<<P, 256, 0, s>>>(P, n, nnz, indptr, indices, Mv, Lv, x, sig, res);
  return cudaGetLastError();
}

cudaError_t launch_eig_update(cudaStream_t s, int P, int n, double2* x, const double2* y, double2* mu) {
  k_eig_update<<<P, 256, 0, s>>>(P, n, x, y, mu);
  return cudaGetLastError();
}

}  // namespace spectau
