// Partitioned banded substitution for problems with few pencils (sm_103a).
//
// Sec. "Matrix solvers": each pencil's banded LU factor is reused for every
// solve while dt is fixed, and the solve is O(n) per pencil.  With a few
// hundred pencils the forward and back substitutions are a few hundred
// dependent chains of n rows each, fewer than GB300's 608 sub-partitions,
// and each row costs a shuffle and a dependent DFMA (~150 cycles): the chain
// latency, not the FP64 pipe, bounds the whole-row-order solve.  Here every
// pencil's rows are cut into nblk blocks of m rows and each block is
// substituted on its own, in the manner of the SPIKE family of partitioned
// banded solvers (Polizzi & Sameh): a block's substitution is an affine map
// of the values that flow into it from its neighbour (the forward window of
// 7 pending rows; the back substitution's kuu partial sums), so
//   1. every block runs with zero inflow, giving its outflow o0_k;
//   2. a short recurrence over blocks, inflow_{k+1} = o0_k + C_k inflow_k,
//      with C_k the block's coupling matrix (its response to unit inflows,
//      computed once per factorization), gives every block's true inflow;
//   3. every block runs again with its true inflow, giving its rows.
// The back substitution starts step 1 from a guess g_k instead of zero
// inflow, the true inflow of the problem's previous solve, and step 2
// becomes inflow_{k-1} = o_k + E_k (inflow_k - g_k): exact for any guess,
// but with zero inflow the velocity rows of a block's top (true values
// ~1e-3 of the buoyancy's early in a run) come out O(1) and the recurrence
// cancels them, so their rounding errors are O(1) too; consecutive solves of
// a time step differ by O(dt), the correction is small and nothing cancels.
// Factorization and setting a field reset the guesses to zero, and a guess
// that is not finite reads as zero.
// Forward substitution uses 8-lane windows (rows j .. j + 7, kl <= 7), four
// chains per warp, over its own (finer) blocks of about 128 rows: it is
// cheap in FP64 instructions and bound by its chain latency; back
// substitution a 32-lane window per chain (kl + ku <= 31), the U columns of
// the block streamed into shared memory by bulk asynchronous copies.  Steps 1 and 3 share one kernel per direction.  The
// block that needs no inflow (the first for the forward pass, the last for
// the back substitution) is exact after step 1.  Every row's arithmetic is
// the whole-row-order substitution's; only the inflows are summed in
// another order.
#include <algorithm>

#include "internal.h"
#include "tma.cuh"

namespace spectau {

constexpr int SPK_FW = 8;             // forward window rows (kl <= 7)
constexpr int SPK_FS = SPK_FW - 1;    // forward inflow: the window's first 7 rows
constexpr int SPK_BW = 32;            // backward window rows (kl + ku <= 31)
constexpr int SPK_RING = 2;           // U chunks in flight per block (16 KB: ~11 blocks per SM)
constexpr int SPK_CHUNK = 32;         // U columns per bulk copy

// ---------------------------------------------------------------------------
// factorization time: the coupling matrices, one thread per (pencil, block,
// unit inflow).  D_k[r][i]: forward window row r after block k for window
// row i = 1 before it (no fresh right-hand side); E_k[r][t]: backward
// outflow r (row j0 - kuu + r) for unit inflow t (row j1 - kuu + t).  The
// arithmetic is the substitution's own, written per row.
// ---------------------------------------------------------------------------
__global__ void k_spike_coupling(int P, int npad, int nblk_f, int nblk, int kl, int kuu, int lpad, int upad,
                                 const double* __restrict__ L, const uint8_t* __restrict__ piv,
                                 const double* __restrict__ U, double* __restrict__ D, double* __restrict__ E) {
  const long long nf = (long long)P * nblk_f * SPK_FS;
  const long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (idx >= nf + (long long)P * nblk * kuu) return;
  if (idx < nf) {
    const int i = (int)(idx % SPK_FS);
    const int k = (int)((idx / SPK_FS) % nblk_f);
    const int p = (int)(idx / ((long long)SPK_FS * nblk_f));
    const int m = npad / nblk_f, j0 = k * m, j1 = j0 + m;
    double win[SPK_FW];
    for (int t = 0; t < SPK_FW; ++t) win[t] = (t == i) ? 1.0 : 0.0;
    const double* Lp = L + (size_t)p * npad * lpad;
    const uint8_t* pv = piv + (size_t)p * npad;
    for (int j = j0; j < j1; ++j) {
      const int off = pv[j];
      const double y = win[off];        // the pivot row's value is y_j
      win[off] = win[0];                // row j's value moves to the pivot row
      for (int d = 1; d <= kl; ++d) win[d] = fma(-Lp[(size_t)j * lpad + d - 1], y, win[d]);
      for (int t = 0; t < SPK_FW - 1; ++t) win[t] = win[t + 1];
      win[SPK_FW - 1] = 0.0;
    }
    double* Dk = D + ((size_t)p * nblk_f + k) * SPK_FS * SPK_FW;
    for (int r = 0; r < SPK_FS; ++r) Dk[r * SPK_FW + i] = win[r];
  } else {
    const long long jdx = idx - nf;
    const int t0 = (int)(jdx % kuu);
    const int k = (int)((jdx / kuu) % nblk);
    const int p = (int)(jdx / ((long long)kuu * nblk));
    const int m = npad / nblk, j0 = k * m, j1 = j0 + m;
    double w[SPK_BW];                   // w[t]: pending row j - t
    for (int t = 0; t < SPK_BW; ++t) w[t] = 0.0;
    w[kuu - 1 - t0] = 1.0;
    const double* Up = U + (size_t)p * npad * upad;
    for (int j = j1 - 1; j >= j0; --j) {
      const double bj = w[0];
      for (int t = 1; t <= kuu; ++t) w[t] = fma(-Up[(size_t)j * upad + t], bj, w[t]);
      for (int t = 0; t < SPK_BW - 1; ++t) w[t] = w[t + 1];
      w[SPK_BW - 1] = 0.0;
    }
    double* Ek = E + ((size_t)p * nblk + k) * kuu * SPK_BW;
    for (int r = 0; r < kuu; ++r) Ek[r * SPK_BW + t0] = w[kuu - 1 - r];
  }
}

cudaError_t launch_spike_coupling(cudaStream_t s, int P, int npad, int nblk_f, int nblk, int kl, int kuu, int lpad,
                                  int upad, const BandFactor& f) {
  if (kl > SPK_FS || kuu >= SPK_BW || nblk < 1 || nblk_f < 1 || npad % (nblk * SPK_CHUNK) ||
      npad % (nblk_f * SPK_FW))
    return cudaErrorInvalidValue;
  const long long total = (long long)P * (nblk_f * SPK_FS + nblk * kuu);
  k_spike_coupling<<<(unsigned)((total + 127) / 128), 128, 0, s>>>(P, npad, nblk_f, nblk, kl, kuu, lpad, upad, f.L,
                                                                  f.piv, f.U, f.spD, f.spE);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// forward substitution of one block per 8-lane segment, four segments
// (chains: pencil, block, real or imaginary part) per warp.  Lane q of a
// segment holds row j + ((q - j) & 7) at step j.  PASS 1: zero inflow
// (the first block: its true rows 0..7), writes the outflow; PASS 2: the
// true inflow, writes y.
// ---------------------------------------------------------------------------
template <int PASS>
__global__ void __launch_bounds__(128) k_spike_fwd(SpikeArgs s) {
  const int gl = blockIdx.x * blockDim.x + threadIdx.x;
  const int q = threadIdx.x & 7;
  const int nk = PASS == 1 ? s.nblk_f - 1 : s.nblk_f;   // PASS 1 skips the last block (no next block)
  const int ch = gl >> 3;
  const bool act = ch < s.P * nk * 2;
  const int chv = act ? ch : 0;
  const int c = chv & 1, k = (chv >> 1) % nk, p = (chv >> 1) / nk;
  const int m = s.m_f, j0 = k * m, j1 = j0 + m, n = s.n;
  const double* Bp = reinterpret_cast<const double*>(s.bg + (size_t)p * n) + c;   // row r at Bp[2 r]
  auto fresh = [&](int r) -> double { return (act && r < n) ? Bp[2 * r] : 0.0; };
  const size_t sidx = (((size_t)p * s.nblk_f + k) * 2 + c) * SPK_FW;
  double v;
  if (PASS == 1)
    v = (k == 0 || q == SPK_FS) ? fresh(j0 + q) : 0.0;
  else
    v = (q < SPK_FS) ? (act ? s.sst[sidx + q] : 0.0) : fresh(j0 + q);
  const double* Lp = s.L + (size_t)p * s.npad * s.lpad;
  const uint8_t* pv = s.piv + (size_t)p * s.npad;
  double* Yp = reinterpret_cast<double*>(s.yg + (size_t)p * n) + c;
  const int kl = s.kl, lpad = s.lpad;
  // each 8-row chunk's pivots, multipliers and fresh right-hand side are
  // loaded one chunk ahead (warps issue in order: a load consumed in the
  // same chunk would stall the chain)
  unsigned long long pw;
  double lv[SPK_FW], nv;
  auto load = [&](int j8, unsigned long long& pw_, double* lv_, double& nv_) {
    const bool in = act && j8 < j1;
    pw_ = in ? *reinterpret_cast<const unsigned long long*>(pv + j8) : 0ull;
#pragma unroll
    for (int i = 0; i < SPK_FW; ++i) {
      const int d = (q - i) & 7;
      lv_[i] = (in && d >= 1 && d <= kl) ? Lp[(size_t)(j8 + i) * lpad + d - 1] : 0.0;
    }
    nv_ = in ? fresh(j8 + SPK_FW + q) : 0.0;
  };
  load(j0, pw, lv, nv);
  for (int j8 = j0; j8 < j1; j8 += SPK_FW) {
    unsigned long long pw2;
    double lv2[SPK_FW], nv2;
    load(j8 + SPK_FW, pw2, lv2, nv2);
#pragma unroll
    for (int i = 0; i < SPK_FW; ++i) {
      const int off = (int)((pw >> (8 * i)) & 0xff);
      const int pl = (i + off) & 7;
      const double bj = __shfl_sync(0xffffffffu, v, pl, 8);   // pivot row value = y_j
      const double vo = __shfl_sync(0xffffffffu, v, i, 8);    // old row j value moves to the pivot row
      v = (q == pl) ? vo : v;
      v = fma(-lv[i], bj, v);
      if (PASS == 2 && act && q == i && j8 + i < n) Yp[2 * (j8 + i)] = bj;
      v = (q == i) ? nv : v;                                   // row j + 8 enters in row j's slot
    }
    pw = pw2;
    nv = nv2;
#pragma unroll
    for (int i = 0; i < SPK_FW; ++i) lv[i] = lv2[i];
  }
  // lane q now holds row j1 + q: the outflow is rows j1 .. j1 + 6
  if (PASS == 1 && act && q < SPK_FS) s.s0[(((size_t)p * s.nblk_f + k + 1) * 2 + c) * SPK_FW + q] = v;
}

// forward inflows: s_0 = rows 0..6 of B~, s_1 from block 0 (exact), then
// s_{k+1} = s0_{k+1} + D_k s_k; one warp per (pencil, part), lanes 0..6.
// The next step's matrix row and outflow are loaded before this step's FMAs.
__global__ void __launch_bounds__(128) k_spike_fwd_rec(SpikeArgs s) {
  const int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= s.P * 2) return;
  const int p = w >> 1, c = w & 1;
  const int i = lane < SPK_FS ? lane : 0;
  const double* Bp = reinterpret_cast<const double*>(s.bg + (size_t)p * s.n) + c;
  auto at = [&](int k) { return (((size_t)p * s.nblk_f + k) * 2 + c) * SPK_FW; };
  double st = i < s.n ? Bp[2 * i] : 0.0;
  if (lane < SPK_FS) s.sst[at(0) + i] = st;
  if (s.nblk_f < 2) return;
  st = s.s0[at(1) + i];
  if (lane < SPK_FS) s.sst[at(1) + i] = st;
  double dn[SPK_FS], sn = 0.0;
  auto load = [&](int k) {
    const double* Dk = s.D + ((size_t)p * s.nblk_f + k) * SPK_FS * SPK_FW + i * SPK_FW;
#pragma unroll
    for (int t = 0; t < SPK_FS; ++t) dn[t] = Dk[t];
    sn = s.s0[at(k + 1) + i];
  };
  if (s.nblk_f > 2) load(1);
  for (int k = 1; k < s.nblk_f - 1; ++k) {
    double dc[SPK_FS];
#pragma unroll
    for (int t = 0; t < SPK_FS; ++t) dc[t] = dn[t];
    double acc = sn, acc2 = 0.0;      // two independent FMA chains per step
    if (k + 1 < s.nblk_f - 1) load(k + 1);
#pragma unroll
    for (int t = 0; t < SPK_FS; t += 2) acc = fma(dc[t], __shfl_sync(0xffffffffu, st, t), acc);
#pragma unroll
    for (int t = 1; t < SPK_FS; t += 2) acc2 = fma(dc[t], __shfl_sync(0xffffffffu, st, t), acc2);
    st = acc + acc2;
    if (lane < SPK_FS) s.sst[at(k + 1) + i] = st;
  }
}

// ---------------------------------------------------------------------------
// back substitution of one block, one CTA of two warps (real and imaginary
// part) per block, with the scaled U columns (U_{j-t,j} / U_jj, t = 0:
// 1/U_jj) streamed chunk by chunk into a shared-memory ring.  Lane l holds
// the row congruent to l mod 32 of rows j - 31 .. j.  PASS 1 (blocks 1 ..
// nblk - 1, or the one block): the guessed inflow, zero for the last
// block, writes the outflow (and x for the last block, which has no
// inflow); PASS 2 (blocks 0 .. nblk - 2): the true inflow, writes
// x = y / U_jj for the block's rows.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double spike_guess(double g) { return isfinite(g) ? g : 0.0; }

template <int PASS>
__global__ void __launch_bounds__(64, 10) k_spike_bwd(SpikeArgs s) {
  __shared__ __align__(128) double Uring[SPK_RING * SPK_CHUNK * SPK_BW];
  __shared__ __align__(8) uint64_t bar[SPK_RING];
  __shared__ int abort_flag;
  // PASS 1 skips block 0 (its outflow has no use); PASS 2 the last block,
  // final after PASS 1
  const int k0 = (PASS == 1 && s.nblk > 1) ? 1 : 0;
  const int nk = s.nblk > 1 ? s.nblk - 1 : 1;
  const int p = blockIdx.x / nk, k = k0 + (blockIdx.x - p * nk);
  const int lane = threadIdx.x & 31, c = threadIdx.x >> 5;
  const int m = s.m, j0 = k * m, j1 = j0 + m, n = s.n, kuu = s.kuu;
  const int nch = m / SPK_CHUNK, chi = j1 / SPK_CHUNK - 1;     // chunks chi, chi - 1, ..., chi - nch + 1
  const double* Usrc = s.U + (size_t)p * s.npad * s.upad;
  const uint32_t ubytes = SPK_CHUNK * SPK_BW * 8;
  auto issue = [&](int q) {                       // q-th chunk of the block in backward order
    const int sl = q % SPK_RING;
    mbar_expect_tx(&bar[sl], ubytes);
    bulk_g2s(Uring + (size_t)sl * SPK_CHUNK * SPK_BW, Usrc + (size_t)(chi - q) * SPK_CHUNK * s.upad, ubytes,
             &bar[sl]);
  };
  if (threadIdx.x == 0) {
    abort_flag = 0;
    for (int sl = 0; sl < SPK_RING; ++sl) mbar_init(&bar[sl], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int q = 0; q < (nch < SPK_RING ? nch : SPK_RING); ++q) issue(q);
  }
  __syncthreads();
  const double* Yp = reinterpret_cast<const double*>(s.yg + (size_t)p * n) + c;
  auto yv = [&](int r) -> double { return (r >= j0 && r < n) ? Yp[2 * r] : 0.0; };
  double w = yv(j1 - SPK_BW + lane);
  const int first_in = SPK_BW - kuu;              // lanes first_in .. 31 hold the inflow rows
  const size_t bidx = (((size_t)p * s.nblk + k) * 2 + c) * SPK_BW;
  if (lane >= first_in) {
    if (PASS == 2) w += s.uin[bidx + lane - first_in];
    else if (k < s.nblk - 1) w += spike_guess(s.uin[bidx + lane - first_in]);
  }
  // lane l takes row jc - 32 + l when it owns column jc + l of the chunk
  // at jc: nw holds that row, loaded one chunk ahead
  double nw = yv(j1 - 2 * SPK_BW + lane);
  double ws = w;   // shuffle source: w before the owner swaps in its next row (the
                   // next column's owner is another lane, so the swap stays off the chain)
  const bool store_x = PASS == 2 || k == s.nblk - 1;
  double* Xp = reinterpret_cast<double*>(s.xg + (size_t)p * n) + c;
  const double* rdp = s.rd + (size_t)p * s.npad;
  int done = 0;
  bool ok = true;
  for (int q = 0; q < nch; ++q) {
    const int sl = q % SPK_RING;
    const bool got = bounded_wait(&bar[sl], (q / SPK_RING) & 1);
    if (!got) atomicOr(&abort_flag, 1);
    __syncthreads();
    if (abort_flag) { ok = false; break; }
    done = q + 1;
    if (threadIdx.x == 0 && q >= 1 && q - 1 + SPK_RING < nch) {
      fence_proxy_async();
      issue(q - 1 + SPK_RING);                    // both warps are past chunk q - 1
    }
    const double* Uc = Uring + (size_t)sl * SPK_CHUNK * SPK_BW;
    const int jc = (chi - q) * SPK_CHUNK;
    const double rdl = store_x ? rdp[jc + lane] : 0.0;
    const double nxt = yv(jc - 2 * SPK_BW + lane);   // this lane's row of the next chunk
    double xo = 0.0;
#pragma unroll
    for (int jj = SPK_CHUNK - 1; jj >= 0; --jj) {
      const double bj = __shfl_sync(0xffffffffu, ws, jj);
      const int t = (jj - lane) & 31;
      const double u = (t >= 1) ? Uc[jj * SPK_BW + t] : 0.0;
      w = fma(-u, bj, w);
      ws = w;
      const bool own = lane == jj;
      xo = own ? bj : xo;
      w = own ? nw : w;
    }
    nw = nxt;
    if (store_x && jc + lane < n) Xp[2 * (jc + lane)] = xo * rdl;
  }
  if (!ok) {
    if (threadIdx.x == 0) {
      raise_status(s.status, SP_ERR_TIMEOUT, p);
      const int want = done == 0 ? SPK_RING : done - 1 + SPK_RING;
      const int issued = nch < want ? nch : want;
      for (int q = done; q < issued; ++q) bounded_wait(&bar[q % SPK_RING], (q / SPK_RING) & 1);
    }
    return;
  }
  // lane l holds row j0 - 32 + l: the outflow is rows j0 - kuu .. j0 - 1
  if (PASS == 1 && k > 0 && lane >= first_in) s.o0[bidx + lane - first_in] = w;
}

// backward inflows: u_{nblk-2} = o_{nblk-1} (exact), then
// u_{k-1} = o_k + E_k (u_k - g_k), g_k the guess PASS 1 started block k
// from, which u_k replaces in place; one CTA of four warps per (pencil,
// part): warp q multiplies columns 8q .. 8q + 7 of row r = lane (four
// sub-partitions share each step's FMAs), warp 0 adds the four partial
// sums.  The next step's matrix entries are loaded before this step's FMAs.
constexpr int SPK_REC_WARPS = 4;
constexpr int SPK_REC_COLS = SPK_BW / SPK_REC_WARPS;
__global__ void __launch_bounds__(SPK_REC_WARPS * 32) k_spike_bwd_rec(SpikeArgs s) {
  __shared__ double part[SPK_REC_WARPS][SPK_BW];
  __shared__ double ucur[SPK_BW];
  const int p = blockIdx.x >> 1, c = blockIdx.x & 1;
  const int r = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const int kuu = s.kuu;
  auto at = [&](int k) { return (((size_t)p * s.nblk + k) * 2 + c) * SPK_BW; };
  if (s.nblk < 2) return;
  if (wq == 0) {
    const double u = r < kuu ? s.o0[at(s.nblk - 1) + r] : 0.0;
    const double g = (r < kuu && s.nblk > 2) ? spike_guess(s.uin[at(s.nblk - 2) + r]) : 0.0;
    ucur[r] = u - g;                                 // u_k - g_k for the next step
    if (r < kuu) s.uin[at(s.nblk - 2) + r] = u;
  }
  double en[SPK_REC_COLS];
  auto load = [&](int k) {
    const double* Ek = s.E + ((size_t)p * s.nblk + k) * kuu * SPK_BW + (size_t)(r < kuu ? r : 0) * SPK_BW;
#pragma unroll
    for (int tt = 0; tt < SPK_REC_COLS; ++tt) {
      const int t = wq * SPK_REC_COLS + tt;
      en[tt] = (r < kuu && t < kuu) ? Ek[t] : 0.0;
    }
  };
  if (s.nblk > 2) load(s.nblk - 2);
  __syncthreads();
  for (int k = s.nblk - 2; k >= 1; --k) {
    double ec[SPK_REC_COLS];
#pragma unroll
    for (int tt = 0; tt < SPK_REC_COLS; ++tt) ec[tt] = en[tt];
    const double o = (wq == 0 && r < kuu) ? s.o0[at(k) + r] : 0.0;
    if (k > 1) load(k - 1);
    double acc = 0.0;
#pragma unroll
    for (int tt = 0; tt < SPK_REC_COLS; ++tt) acc = fma(ec[tt], ucur[wq * SPK_REC_COLS + tt], acc);
    part[wq][r] = acc;
    __syncthreads();
    if (wq == 0) {
      double u = o;
#pragma unroll
      for (int q = 0; q < SPK_REC_WARPS; ++q) u += part[q][r];
      const double g = (r < kuu && k > 1) ? spike_guess(s.uin[at(k - 1) + r]) : 0.0;
      ucur[r] = r < kuu ? u - g : 0.0;
      if (r < kuu) s.uin[at(k - 1) + r] = u;
    }
    __syncthreads();
  }
}

bool spike_supported(int kl, int kuu, int npad, int nblk) {
  return kl <= SPK_FS && spike_bwd_supported(kuu, npad, nblk);
}

bool spike_bwd_supported(int kuu, int npad, int nblk) {
  return kuu < SPK_BW && nblk >= 1 && npad % (nblk * SPK_CHUNK) == 0;
}

// the back substitution's coupling matrices alone, for factors whose lower
// band is wider than the forward windows (the transposed factor of the
// adjoint: kl' = ku)
cudaError_t launch_spike_coupling_bwd(cudaStream_t s, int P, int npad, int nblk, int kuu, int upad, const double* U,
                                      double* E) {
  if (!spike_bwd_supported(kuu, npad, nblk) || upad != SPK_BW) return cudaErrorInvalidValue;
  const long long total = (long long)P * nblk * kuu;
  k_spike_coupling<<<(unsigned)((total + 127) / 128), 128, 0, s>>>(P, npad, 0, nblk, 0, kuu, 0, upad, nullptr,
                                                                  nullptr, U, nullptr, E);
  return cudaGetLastError();
}

// y (yg) -> x~ = y / U_jj (xg): the back substitution's two passes and their
// recurrence (the forward substitution done elsewhere)
cudaError_t launch_spike_backward(cudaStream_t st, const SpikeArgs& s) {
  if (!spike_bwd_supported(s.kuu, s.npad, s.nblk) || s.m * s.nblk != s.npad || s.upad != SPK_BW)
    return cudaErrorInvalidValue;
  k_spike_bwd<1><<<s.P * (s.nblk > 1 ? s.nblk - 1 : 1), 64, 0, st>>>(s);
  if (s.nblk > 1) {
    k_spike_bwd_rec<<<s.P * 2, SPK_REC_WARPS * 32, 0, st>>>(s);
    k_spike_bwd<2><<<s.P * (s.nblk - 1), 64, 0, st>>>(s);
  }
  return cudaGetLastError();
}

// B~ (bg) -> x~ = y / U_jj (xg) through y (yg); five launches
cudaError_t launch_spike_solve(cudaStream_t st, const SpikeArgs& s) {
  if (!spike_supported(s.kl, s.kuu, s.npad, s.nblk) || s.m * s.nblk != s.npad || s.upad != SPK_BW ||
      s.nblk_f < 1 || s.m_f * s.nblk_f != s.npad || s.m_f % SPK_FW)
    return cudaErrorInvalidValue;
  const int T = 128;
  if (s.nblk_f > 1) {
    const long long lanes1 = (long long)s.P * (s.nblk_f - 1) * 2 * SPK_FW;
    k_spike_fwd<1><<<(unsigned)((lanes1 + T - 1) / T), T, 0, st>>>(s);
  }
  k_spike_fwd_rec<<<(unsigned)((s.P * 2 * 32 + T - 1) / T), T, 0, st>>>(s);
  const long long lanes2 = (long long)s.P * s.nblk_f * 2 * SPK_FW;
  k_spike_fwd<2><<<(unsigned)((lanes2 + T - 1) / T), T, 0, st>>>(s);
  k_spike_bwd<1><<<s.P * (s.nblk > 1 ? s.nblk - 1 : 1), 64, 0, st>>>(s);
  if (s.nblk > 1) {
    k_spike_bwd_rec<<<s.P * 2, SPK_REC_WARPS * 32, 0, st>>>(s);
    k_spike_bwd<2><<<s.P * (s.nblk - 1), 64, 0, st>>>(s);
  }
  return cudaGetLastError();
}

}  // namespace spectau
