// Blocked right-looking complex LU with partial pivoting and the solve
// (Kouya, Sec. IV-C, Fig. 3: for every block of K columns the rectangle
// A22 - L21 U12 is updated by a complex matrix product; "Normal LU" is K = 1).
//
// Every scalar result is formed exactly and rounded once to p bits
// (nearest-even); no floating point is used on the GPU.  Per panel column j:
//   1. pivot: the first row i >= j maximising RN_p(|Re a_ij| + |Im a_ij|)
//      (the |.|_1 pivot rule of LAPACK's complex LU);
//   2. swap rows j and the pivot row across the whole matrix;
//   3. l_ij = RN_p(a_ij / a_jj) for i > j, componentwise from the exact quotient;
//   4. a_ic = RN_p(a_ic - l_ij a_jc) (exact complex FMA per component) for the
//      rest of the panel (i > j, j < c < kend).
// After the panel (its interchanges all applied): U12 by the same update,
// j = kb..kend-1, for j < i < kend, c >= kend.
// After the panel: P = RN_p(L21 U12) by mpcgemm (Ozaki 3M/4M), A22 = RN_p(A22 - P).
// Solve: b permuted, forward substitution y_i = RN(y_i - l_ij y_j), backward
// x_j = RN(y_j / u_jj), y_i = RN(y_i - u_ij x_j), all column-oriented.
#include "common.cuh"
#include "kernels.h"
#include "mpscalar.cuh"
#include "mpscalar_fast.cuh"

namespace mpc {

namespace {

constexpr int kStSingular = 5;    // status word: 1 + first zero pivot column
constexpr int kStTruncated = 3;   // shares the "uncertified" word of the GEMM status

struct MatRW {
  uint8_t *sign[2];
  int32_t *exp[2];
  uint64_t *limb[2];
  int64_t ld, plane;
  __device__ __forceinline__ MPRef ref(int c, int64_t r, int64_t col) const {
    const int64_t idx = r * ld + col;
    return MPRef{sign[c][idx], exp[c][idx], limb[c] + idx, plane};
  }
  __device__ __forceinline__ MPOut out(int c, int64_t r, int64_t col) const {
    const int64_t idx = r * ld + col;
    return MPOut{sign[c] + idx, exp[c] + idx, limb[c] + idx, plane};
  }
};

// RN_p of the exact sum of the terms: the register-resident form for L = 4, 8 when the
// terms' window fits it, else the generic one (same result).  Not inlined: one copy serves
// every kernel.
__device__ __noinline__ bool sum_round(const Term *t, int nt, int p, int L, MPOut o, bool *truncated) {
  int r = -1;
  if (L == 8) r = fastmp::sum_round<8>(t, nt, p, o);
  else if (L == 4) r = fastmp::sum_round<4>(t, nt, p, o);
  if (r >= 0) {
    *truncated = false;
    return r == 1;
  }
  return mp_sum_round(t, nt, p, L, o, truncated);
}

// exact a - l * u per component (Eq. 4m_way_base), rounded once; into (r, col) of M
__device__ __noinline__ void cfma_store(const MatRW &M, int64_t r, int64_t col, const MPRef &are, const MPRef &aim,
                           const MPRef &lre, const MPRef &lim, const MPRef &ure, const MPRef &uim, int p, int L,
                           int32_t *status) {
  bool trunc = false, ok = true;
  MPOut ore = M.out(0, r, col), oim = M.out(1, r, col);
  {
    Term t[3] = {{are, are, false, false}, {lre, ure, true, true}, {lim, uim, true, false}};
    bool tr;
    ok &= sum_round(t, 3, p, L, ore, &tr);
    trunc |= tr;
  }
  {
    Term t[3] = {{aim, aim, false, false}, {lre, uim, true, true}, {lim, ure, true, true}};
    bool tr;
    ok &= sum_round(t, 3, p, L, oim, &tr);
    trunc |= tr;
  }
  if (trunc) atomicOr(reinterpret_cast<int *>(status) + kStTruncated, 1);
  if (!ok) atomicOr(reinterpret_cast<int *>(status) + kStErange, 1);
}

// complex quotient a / d, componentwise RN_p of the exact value, into (r, col).
// Both exact numerators are formed before anything is stored (the output may
// be a itself).
__device__ __noinline__ void cdiv_store(const MatRW &M, int64_t r, int64_t col, const MPRef &are, const MPRef &aim,
                                        const MPRef &dre, const MPRef &dim, int p, int L, int32_t *status) {
  {   // the register-resident form for L = 4, 8 when the windows fit it (same result)
    int rf = -1;
    if (L == 8) rf = fastmp::cdiv<8>(are, aim, dre, dim, p, M.out(0, r, col), M.out(1, r, col));
    else if (L == 4) rf = fastmp::cdiv<4>(are, aim, dre, dim, p, M.out(0, r, col), M.out(1, r, col));
    if (rf == 2) return;   // d == 0: refused earlier
    if (rf >= 0) {
      if (rf == 0) atomicOr(reinterpret_cast<int *>(status) + kStErange, 1);
      return;
    }
  }
  uint64_t den[kWinLimbs], num[2][kWinLimbs];
  int nwd, nwn[2];
  int64_t lsbd, lsbn[2];
  bool negd, negn[2], nz[2], tr, trunc = false, ok = true;
  Term td[2] = {{dre, dre, true, false}, {dim, dim, true, false}};
  if (!mp_sum_exact(td, 2, L, den, &nwd, &lsbd, &negd, &tr)) return;   // d == 0: refused earlier
  trunc |= tr;
  Term t0[2] = {{are, dre, true, false}, {aim, dim, true, false}};   // a_re d_re + a_im d_im
  Term t1[2] = {{aim, dre, true, false}, {are, dim, true, true}};    // a_im d_re - a_re d_im
  nz[0] = mp_sum_exact(t0, 2, L, num[0], &nwn[0], &lsbn[0], &negn[0], &tr);
  trunc |= tr;
  nz[1] = mp_sum_exact(t1, 2, L, num[1], &nwn[1], &lsbn[1], &negn[1], &tr);
  trunc |= tr;
  for (int c = 0; c < 2; ++c) {
    MPOut o = M.out(c, r, col);
    if (!nz[c]) store_zero(L, o.s, o.e, o.limb, o.stride);
    else ok &= mp_div_round(num[c], nwn[c], lsbn[c], negn[c], den, nwd, lsbd, p, L, o);
  }
  if (trunc) atomicOr(reinterpret_cast<int *>(status) + kStTruncated, 1);
  if (!ok) atomicOr(reinterpret_cast<int *>(status) + kStErange, 1);
}

// Component c of a - l u (Eq. 4m_way_base), rounded once, into (r, col) of M.  The two
// components read disjoint parts of (r, col), so two threads may form them independently.
__device__ __noinline__ void cfma_part(const MatRW &M, int64_t r, int64_t col, int c, const MPRef &a,
                                       const MPRef &lre, const MPRef &lim, const MPRef &ure, const MPRef &uim, int p,
                                       int L, int32_t *status) {
  // Re: a - l_re u_re + l_im u_im;  Im: a - l_re u_im - l_im u_re (operands selected, so
  // that the two lanes of a pair run the same instructions)
  bool trunc = false;
  Term t[3] = {{a, a, false, false}, {lre, c ? uim : ure, true, true}, {lim, c ? ure : uim, true, c != 0}};
  const bool ok = sum_round(t, 3, p, L, M.out(c, r, col), &trunc);
  if (trunc) atomicOr(reinterpret_cast<int *>(status) + kStTruncated, 1);
  if (!ok) atomicOr(reinterpret_cast<int *>(status) + kStErange, 1);
}

// Component c of the complex quotient a / d, RN_p of its exact value, into o (the
// register-resident form for L = 4, 8 when its windows fit, else the generic one).
// 1: done, 0: exponent overflow, 2: d == 0 (nothing written).
__device__ __noinline__ int cdiv_part(int c, const MPRef &are, const MPRef &aim, const MPRef &dre, const MPRef &dim,
                                      int p, int L, MPOut o, bool *trunc) {
  *trunc = false;
  int rf = -1;
  if (L == 8) rf = fastmp::cdiv_part<8>(are, aim, dre, dim, c, p, o);
  else if (L == 4) rf = fastmp::cdiv_part<4>(are, aim, dre, dim, c, p, o);
  if (rf >= 0) return rf;
  uint64_t den[kWinLimbs], num[kWinLimbs];
  int nwd, nwn;
  int64_t lsbd, lsbn;
  bool negd, negn, tr;
  Term td[2] = {{dre, dre, true, false}, {dim, dim, true, false}};
  if (!mp_sum_exact(td, 2, L, den, &nwd, &lsbd, &negd, &tr)) return 2;
  *trunc |= tr;
  Term t0[2] = {{are, dre, true, false}, {aim, dim, true, false}};   // a_re d_re + a_im d_im
  Term t1[2] = {{aim, dre, true, false}, {are, dim, true, true}};    // a_im d_re - a_re d_im
  const bool nz = mp_sum_exact(c == 0 ? t0 : t1, 2, L, num, &nwn, &lsbn, &negn, &tr);
  *trunc |= tr;
  if (!nz) {
    store_zero(L, o.s, o.e, o.limb, o.stride);
    return 1;
  }
  return mp_div_round(num, nwn, lsbn, negn, den, nwd, lsbd, p, L, o) ? 1 : 0;
}

// a / d into (r, col) of M by two adjacent lanes, lane parity = component; the result is
// held in registers until both lanes have read their operands (the output may be a
// itself).  Every lane of the warp must call it (`active`: this lane has an element).
__device__ __forceinline__ void cdiv_pair_store(const MatRW &M, int64_t r, int64_t col, bool active, const MPRef &are,
                                                const MPRef &aim, const MPRef &dre, const MPRef &dim, int p, int L,
                                                int32_t *status) {
  const int c = threadIdx.x & 1;
  uint8_t sg = 0;
  int32_t ex = 0;
  uint64_t lm[kMaxLimbs];
  MPOut tmp{&sg, &ex, lm, 1};
  int rf = 2;
  bool tr = false;
  if (active) rf = cdiv_part(c, are, aim, dre, dim, p, L, tmp, &tr);
  __syncwarp();
  if (!active || rf == 2) return;   // d == 0: refused earlier
  MPOut o = M.out(c, r, col);
  *o.s = sg;
  *o.e = ex;
  for (int j = 0; j < L; ++j) o.limb[(int64_t)j * o.stride] = lm[j];
  if (tr) atomicOr(reinterpret_cast<int *>(status) + kStTruncated, 1);
  if (rf == 0) atomicOr(reinterpret_cast<int *>(status) + kStErange, 1);
}

// the pivot key RN_p(|re| + |im|) as comparable words: (zero?, exponent, limbs)
struct Key {
  int32_t e;
  uint64_t m[kMaxLimbs];
  bool nz;
};

__device__ __forceinline__ bool key_greater(const Key &a, const Key &b, int L) {
  if (a.nz != b.nz) return a.nz;
  if (!a.nz) return false;
  if (a.e != b.e) return a.e > b.e;
  for (int j = L - 1; j >= 0; --j)
    if (a.m[j] != b.m[j]) return a.m[j] > b.m[j];
  return false;
}

}  // namespace

// (key, row) of the better candidate: the larger key, the first row among equal keys
__device__ __forceinline__ void pivot_take(Key &k, int64_t &row, const Key &ok, int64_t orow, int L) {
  if (orow < 0) return;
  if (row < 0 || key_greater(ok, k, L) || (!key_greater(k, ok, L) && orow < row)) {
    k = ok;
    row = orow;
  }
}

__device__ __forceinline__ void pivot_shfl(Key &k, int64_t &row, int off, int L) {
  Key o;
  o.e = __shfl_down_sync(0xffffffffu, k.e, off);
  o.nz = __shfl_down_sync(0xffffffffu, (int)k.nz, off) != 0;
  for (int x = 0; x < L; ++x) o.m[x] = __shfl_down_sync(0xffffffffu, k.m[x], off);
  const int64_t orow = __shfl_down_sync(0xffffffffu, row, off);
  pivot_take(k, row, o, orow, L);
}

constexpr int kPivotT = 512;
static_assert(kPivotT % 32 == 0 && kPivotT / 32 <= 32, "one warp reduces the per-warp candidates");

__global__ void __launch_bounds__(kPivotT) k_lu_pivot(MatRW A, int64_t n, int64_t j, int p, int L, int32_t *ipiv,
                                                      int32_t *status) {
  __shared__ Key keys[kPivotT / 32];
  __shared__ int64_t rows[kPivotT / 32];
  Key best;
  best.nz = false;
  best.e = 0;
  for (int x = 0; x < kMaxLimbs; ++x) best.m[x] = 0;
  int64_t brow = -1;
  for (int64_t i = j + threadIdx.x; i < n; i += blockDim.x) {
    MPRef re = A.ref(0, i, j), im = A.ref(1, i, j);
    re.s = 0;
    im.s = 0;   // absolute values
    Key k;
    uint8_t ks;
    MPOut o{&ks, &k.e, k.m, 1};
    Term t[2] = {{re, re, false, false}, {im, im, false, false}};
    bool tr;
    sum_round(t, 2, p, L, o, &tr);
    k.nz = k.m[L - 1] != 0;
    pivot_take(best, brow, k, i, L);
  }
  for (int off = 16; off > 0; off >>= 1) pivot_shfl(best, brow, off, L);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    keys[w] = best;
    rows[w] = brow;
  }
  __syncthreads();
  if (w == 0) {
    brow = -1;   // lanes beyond the block's warp count hold no candidate
    if (lane < kPivotT / 32) {
      best = keys[lane];
      brow = rows[lane];
    }
    for (int off = 16; off > 0; off >>= 1) pivot_shfl(best, brow, off, L);
    if (lane == 0) {
      ipiv[j] = (int32_t)brow;
      if (!best.nz && status[kStSingular] == 0) status[kStSingular] = (int32_t)(j + 1);
    }
  }
}

__global__ void k_lu_swap(MatRW A, int64_t ncols, int64_t j, const int32_t *ipiv, int L) {
  const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t r = ipiv[j];
  if (col >= ncols || r == j) return;
  for (int c = 0; c < 2; ++c) {
    const int64_t a = j * A.ld + col, b = r * A.ld + col;
    uint8_t s = A.sign[c][a];
    A.sign[c][a] = A.sign[c][b];
    A.sign[c][b] = s;
    int32_t e = A.exp[c][a];
    A.exp[c][a] = A.exp[c][b];
    A.exp[c][b] = e;
    for (int u = 0; u < L; ++u) {
      uint64_t v = A.limb[c][(int64_t)u * A.plane + a];
      A.limb[c][(int64_t)u * A.plane + a] = A.limb[c][(int64_t)u * A.plane + b];
      A.limb[c][(int64_t)u * A.plane + b] = v;
    }
  }
}

// two lanes per element, one per component
__global__ void k_lu_divide(MatRW A, int64_t n, int64_t j, int p, int L, int32_t *status) {
  const int64_t i = j + 1 + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 2;
  const bool active = i < n && !status[kStSingular];
  const int64_t r = active ? i : j;
  cdiv_pair_store(A, i, j, active, A.ref(0, r, j), A.ref(1, r, j), A.ref(0, j, j), A.ref(1, j, j), p, L, status);
}

// a_ic = RN(a_ic - a_ij a_jc) for i in [r0, r1), c in [c0, c1); two lanes per element
__global__ void k_lu_rank1(MatRW A, int64_t j, int64_t r0, int64_t r1, int64_t c0, int64_t c1, int p, int L,
                           int32_t *status) {
  const int64_t w = c1 - c0;
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 2;
  const int c = threadIdx.x & 1;
  if (t >= (r1 - r0) * w || status[kStSingular]) return;
  const int64_t i = r0 + t / w, col = c0 + t % w;
  cfma_part(A, i, col, c, A.ref(c, i, col), A.ref(0, i, j), A.ref(1, i, j), A.ref(0, j, col), A.ref(1, j, col), p, L,
            status);
}

// the GEMM's device-side failures count for the LU as well
__global__ void k_fold_status(int32_t *dst, const int32_t *gemm) {
  if (threadIdx.x == 0) {
    if (gemm[kStErange]) atomicOr(reinterpret_cast<int *>(dst) + kStErange, 1);
    if (gemm[kStUncertified]) atomicOr(reinterpret_cast<int *>(dst) + kStTruncated, 1);
    if (gemm[kStTimeout]) atomicOr(reinterpret_cast<int *>(dst) + kStTimeout, 1);
  }
}

// dst (contiguous rows x cols) = A[r0.., c0..]
__global__ void k_copy_block(MatRW A, int64_t r0, int64_t c0, int64_t rows, int64_t cols, MatRW D, int L) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= rows * cols) return;
  const int64_t r = t / cols, col = t % cols;
  const int64_t a = (r0 + r) * A.ld + c0 + col, d = r * D.ld + col;
  for (int c = 0; c < 2; ++c) {
    D.sign[c][d] = A.sign[c][a];
    D.exp[c][d] = A.exp[c][a];
    for (int u = 0; u < L; ++u) D.limb[c][(int64_t)u * D.plane + d] = A.limb[c][(int64_t)u * A.plane + a];
  }
}

// A[r0 + r][c0 + col] = RN(A - P[r][col]) componentwise
__global__ void k_sub_block(MatRW A, int64_t r0, int64_t c0, int64_t rows, int64_t cols, MatRW P, int p, int L,
                            int32_t *status) {
  const int64_t t = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 2;   // two lanes per element
  const int c = threadIdx.x & 1;
  if (t >= rows * cols || status[kStSingular]) return;
  const int64_t r = t / cols, col = t % cols;
  MPRef a = A.ref(c, r0 + r, c0 + col), q = P.ref(c, r, col);
  Term tt[2] = {{a, a, false, false}, {q, q, false, true}};
  bool tr;
  const bool ok = sum_round(tt, 2, p, L, A.out(c, r0 + r, c0 + col), &tr);
  if (tr) atomicOr(reinterpret_cast<int *>(status) + kStTruncated, 1);
  if (!ok) atomicOr(reinterpret_cast<int *>(status) + kStErange, 1);
}

// Solve with the factors for one right-hand side column per block (blockIdx.x), every
// step inside the block: for n up to the block size every row has a thread of its own,
// and a single launch costs less than 2n of them.
__global__ void __launch_bounds__(256) k_lu_solve(MatRW LU, int64_t n, const int32_t *ipiv, MatRW Bm, int p, int L,
                                                   int32_t *status) {
  const int64_t col = blockIdx.x;
  if (status[kStSingular]) return;
  if (threadIdx.x == 0) {   // apply the row interchanges in order
    for (int64_t j = 0; j < n; ++j) {
      const int64_t r = ipiv[j];
      if (r == j) continue;
      for (int c = 0; c < 2; ++c) {
        const int64_t a = j * Bm.ld + col, b = r * Bm.ld + col;
        uint8_t sg = Bm.sign[c][a];
        Bm.sign[c][a] = Bm.sign[c][b];
        Bm.sign[c][b] = sg;
        int32_t e = Bm.exp[c][a];
        Bm.exp[c][a] = Bm.exp[c][b];
        Bm.exp[c][b] = e;
        for (int u = 0; u < L; ++u) {
          uint64_t v = Bm.limb[c][(int64_t)u * Bm.plane + a];
          Bm.limb[c][(int64_t)u * Bm.plane + a] = Bm.limb[c][(int64_t)u * Bm.plane + b];
          Bm.limb[c][(int64_t)u * Bm.plane + b] = v;
        }
      }
    }
  }
  __syncthreads();
  for (int64_t j = 0; j < n; ++j) {   // forward: unit lower L
    for (int64_t i = j + 1 + threadIdx.x; i < n; i += blockDim.x)
      cfma_store(Bm, i, col, Bm.ref(0, i, col), Bm.ref(1, i, col), LU.ref(0, i, j), LU.ref(1, i, j),
                 Bm.ref(0, j, col), Bm.ref(1, j, col), p, L, status);
    __syncthreads();
  }
  for (int64_t j = n - 1; j >= 0; --j) {   // backward: upper U
    if (threadIdx.x == 0)
      cdiv_store(Bm, j, col, Bm.ref(0, j, col), Bm.ref(1, j, col), LU.ref(0, j, j), LU.ref(1, j, j), p, L, status);
    __syncthreads();
    for (int64_t i = threadIdx.x; i < j; i += blockDim.x)
      cfma_store(Bm, i, col, Bm.ref(0, i, col), Bm.ref(1, i, col), LU.ref(0, i, j), LU.ref(1, i, j),
                 Bm.ref(0, j, col), Bm.ref(1, j, col), p, L, status);
    __syncthreads();
  }
}

// Larger systems: one launch per step, so that every step spreads over the
// whole GPU (right-hand side column col0 + blockIdx.y).
// b := P b: the row interchanges in order, one thread per right-hand side column.
__global__ void k_solve_perm(MatRW Bm, int64_t n, int64_t nrhs, const int32_t *ipiv, int L, int32_t *status) {
  const int64_t col = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (col >= nrhs || status[kStSingular]) return;
  for (int64_t j = 0; j < n; ++j) {
    const int64_t r = ipiv[j];
    if (r == j) continue;
    for (int c = 0; c < 2; ++c) {
      const int64_t a = j * Bm.ld + col, b = r * Bm.ld + col;
      uint8_t sg = Bm.sign[c][a];
      Bm.sign[c][a] = Bm.sign[c][b];
      Bm.sign[c][b] = sg;
      int32_t e = Bm.exp[c][a];
      Bm.exp[c][a] = Bm.exp[c][b];
      Bm.exp[c][b] = e;
      for (int u = 0; u < L; ++u) {
        uint64_t v = Bm.limb[c][(int64_t)u * Bm.plane + a];
        Bm.limb[c][(int64_t)u * Bm.plane + a] = Bm.limb[c][(int64_t)u * Bm.plane + b];
        Bm.limb[c][(int64_t)u * Bm.plane + b] = v;
      }
    }
  }
}

// forward step j (unit lower L): y_i = RN(y_i - l_ij y_j) for j < i < n; two lanes per row
__global__ void k_solve_fwd(MatRW LU, int64_t n, int64_t j, MatRW Bm, int64_t col0, int p, int L, int32_t *status) {
  const int64_t col = col0 + blockIdx.y;
  const int64_t i = j + 1 + ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 2;
  const int c = threadIdx.x & 1;
  if (i >= n || status[kStSingular]) return;
  cfma_part(Bm, i, col, c, Bm.ref(c, i, col), LU.ref(0, i, j), LU.ref(1, i, j), Bm.ref(0, j, col), Bm.ref(1, j, col), p,
            L, status);
}

// x_j = RN(y_j / u_jj) for the last row (the first backward step); two lanes per column
__global__ void k_solve_last(MatRW LU, int64_t j, MatRW Bm, int64_t nrhs, int p, int L, int32_t *status) {
  const int64_t col = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 2;
  const bool active = col < nrhs && !status[kStSingular];
  const int64_t cc = active ? col : 0;
  cdiv_pair_store(Bm, j, col, active, Bm.ref(0, j, cc), Bm.ref(1, j, cc), LU.ref(0, j, j), LU.ref(1, j, j), p, L,
                  status);
}

// backward step j (upper U, x_j already in row j): y_i = RN(y_i - u_ij x_j) for i < j,
// two lanes per row; the lane pair of row j - 1 then forms x_{j-1} = RN(y_{j-1} / u_{j-1,j-1})
// for the next step (after a warp barrier: each lane needs the other's component of y_{j-1})
__global__ void k_solve_bwd(MatRW LU, int64_t j, MatRW Bm, int64_t col0, int p, int L, int32_t *status) {
  const int64_t col = col0 + blockIdx.y;
  const int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / 2;
  const int c = threadIdx.x & 1;
  const bool live = !status[kStSingular];
  if (i < j && live)
    cfma_part(Bm, i, col, c, Bm.ref(c, i, col), LU.ref(0, i, j), LU.ref(1, i, j), Bm.ref(0, j, col),
              Bm.ref(1, j, col), p, L, status);
  if ((int64_t)blockIdx.x * blockDim.x / 2 > j - 1 || (int64_t)(blockIdx.x + 1) * blockDim.x / 2 <= j - 1) return;
  __syncwarp();   // the warp holding row j - 1 (block-uniform test above: every lane of it is here)
  const bool act = i == j - 1 && live;
  const int64_t r = act ? i : j - 1;
  cdiv_pair_store(Bm, r, col, act, Bm.ref(0, r, col), Bm.ref(1, r, col), LU.ref(0, r, r), LU.ref(1, r, r), p, L,
                  status);
}

}  // namespace mpc

// ------------------------------------------------------------------ host driver

using namespace mpc;

namespace {

inline uint64_t al256(uint64_t x) { return (x + 255) & ~255ull; }

struct LuLayout {
  uint64_t off_status, off_l21, off_u12, off_p, off_gemm, gemm_bytes, total;
};

uint64_t mat_bytes(int64_t rows, int64_t cols, int L) { return (uint64_t)rows * cols * 2 * (1 + 4 + 8 * L); }

int lu_layout(int64_t n, int32_t p, int32_t K, int method, LuLayout *o) {
  if (n < 0 || p < 1 || p > MPC_MAX_P_BITS || K < 1 || (method != MPC_4M && method != MPC_3M)) return MPC_EINVAL;
  const int L = (p + 63) / 64;
  const int64_t kk = K < n ? K : (n > 0 ? n : 1);
  const int64_t rest = n > kk ? n - kk : 0;
  uint64_t off = 0;
  o->off_status = off;
  off = al256(off + 64);
  o->off_l21 = off;
  off = al256(off + mat_bytes(rest, kk, L) + 2048);
  o->off_u12 = off;
  off = al256(off + mat_bytes(kk, rest, L) + 2048);
  o->off_p = off;
  off = al256(off + mat_bytes(rest, rest, L) + 2048);
  o->gemm_bytes = rest > 0 ? mpcgemm_workspace_size(rest, rest, kk, p, method, MPC_OZAKI) : 0;
  o->off_gemm = off;
  off = al256(off + o->gemm_bytes);
  o->total = off;
  return MPC_OK;
}

// contiguous device matrix carved from the workspace
MatRW carve(char *base, int64_t rows, int64_t cols, int L, mpc_mat *pub) {
  MatRW m;
  const int64_t e = rows * cols;
  char *q = base;
  for (int c = 0; c < 2; ++c) {
    m.limb[c] = (uint64_t *)q;
    q += al256((uint64_t)e * 8 * L);
  }
  for (int c = 0; c < 2; ++c) {
    m.exp[c] = (int32_t *)q;
    q += al256((uint64_t)e * 4);
  }
  for (int c = 0; c < 2; ++c) {
    m.sign[c] = (uint8_t *)q;
    q += al256((uint64_t)e);
  }
  m.ld = cols;
  m.plane = e;
  if (pub) {
    pub->rows = rows;
    pub->cols = cols;
    pub->ld = cols;
    for (int c = 0; c < 2; ++c) {
      pub->sign[c] = m.sign[c];
      pub->exp[c] = m.exp[c];
      pub->limb[c] = m.limb[c];
    }
  }
  return m;
}

MatRW rw_of(mpc_mat *X) {
  MatRW m;
  for (int c = 0; c < 2; ++c) {
    m.sign[c] = X->sign[c];
    m.exp[c] = X->exp[c];
    m.limb[c] = X->limb[c];
  }
  m.ld = X->ld;
  m.plane = X->rows * X->ld;
  return m;
}

unsigned blocks_for(int64_t t, int th) { return (unsigned)((t + th - 1) / th); }

}  // namespace

extern "C" size_t mpcgesv_workspace_size(int64_t n, int32_t p_bits, int32_t block, int method) {
  LuLayout lay;
  if (lu_layout(n, p_bits, block, method, &lay) != MPC_OK) return 0;
  return (size_t)lay.total;
}

extern "C" int mpcgesv(int64_t n, int32_t p_bits, mpc_mat *A, int32_t *ipiv, mpc_mat *B, int32_t block, int method,
                       void *workspace, size_t ws_bytes, void *stream) {
  LuLayout lay;
  int rc = lu_layout(n, p_bits, block, method, &lay);
  if (rc != MPC_OK) return rc;
  if (!A || !B || A->rows != n || A->cols != n || B->rows != n || B->cols < 1 || A->ld < n || B->ld < B->cols)
    return MPC_EINVAL;
  if (n == 0) return MPC_OK;
  if (!ipiv || !workspace || ((uintptr_t)workspace & 255)) return MPC_EINVAL;
  if (ws_bytes < lay.total) return MPC_ENOSPC;
  cudaStream_t st = (cudaStream_t)stream;
  const int L = (p_bits + 63) / 64;
  char *ws = (char *)workspace;
  int32_t *status = (int32_t *)(ws + lay.off_status);
  cudaMemsetAsync(status, 0, 64, st);
  MatRW Am = rw_of(A), Bm = rw_of(B);
  const int64_t K = block;
  for (int64_t kb = 0; kb < n; kb += K) {
    const int64_t kend = kb + K < n ? kb + K : n;
    for (int64_t j = kb; j < kend; ++j) {
      k_lu_pivot<<<1, kPivotT, 0, st>>>(Am, n, j, p_bits, L, ipiv, status);
      k_lu_swap<<<blocks_for(n, 128), 128, 0, st>>>(Am, n, j, ipiv, L);
      if (j + 1 < n) k_lu_divide<<<blocks_for(2 * (n - j - 1), 64), 64, 0, st>>>(Am, n, j, p_bits, L, status);
      if (j + 1 < n && j + 1 < kend)   // rest of the panel
        k_lu_rank1<<<blocks_for(2 * (n - j - 1) * (kend - j - 1), 64), 64, 0, st>>>(Am, j, j + 1, n, j + 1, kend, p_bits,
                                                                                   L, status);
    }
    // U12 = L11^-1 A12, once every interchange of the panel has been applied
    if (kend < n)
      for (int64_t j = kb; j + 1 < kend; ++j)
        k_lu_rank1<<<blocks_for(2 * (kend - j - 1) * (n - kend), 64), 64, 0, st>>>(Am, j, j + 1, kend, kend, n, p_bits,
                                                                                   L, status);
    if (kend < n) {   // trailing update A22 -= L21 U12 through the Ozaki complex GEMM
      const int64_t rest = n - kend, w = kend - kb;
      mpc_mat l21, u12, pm;
      MatRW Lm = carve(ws + lay.off_l21, rest, w, L, &l21);
      MatRW Um = carve(ws + lay.off_u12, w, rest, L, &u12);
      MatRW Pm = carve(ws + lay.off_p, rest, rest, L, &pm);
      k_copy_block<<<blocks_for(rest * w, 128), 128, 0, st>>>(Am, kend, kb, rest, w, Lm, L);
      k_copy_block<<<blocks_for(rest * w, 128), 128, 0, st>>>(Am, kb, kend, w, rest, Um, L);
      rc = mpcgemm(rest, rest, w, p_bits, &l21, &u12, &pm, method, MPC_OZAKI, ws + lay.off_gemm, lay.gemm_bytes,
                   stream);
      if (rc != MPC_OK) return rc;
      k_fold_status<<<1, 32, 0, st>>>(status, (const int32_t *)(ws + lay.off_gemm));
      k_sub_block<<<blocks_for(2 * rest * rest, 64), 64, 0, st>>>(Am, kend, kend, rest, rest, Pm, p_bits, L, status);
    }
  }
  // solve: forward then backward substitution, every element's operations in the same
  // order as the column-oriented loops (bit-identical results), one launch per step
  const int64_t nrhs = B->cols;
  constexpr int64_t kSolveBlock = 256;   // one block per column up to n = 256, then a launch per step
  if (n > 0 && nrhs > 0 && n <= kSolveBlock) {
    k_lu_solve<<<(unsigned)nrhs, (unsigned)kSolveBlock, 0, st>>>(Am, n, ipiv, Bm, p_bits, L, status);
  } else if (n > 0 && nrhs > 0) {
    constexpr int64_t kMaxGridY = 65535;
    constexpr int kT = 64;
    k_solve_perm<<<blocks_for(nrhs, kT), kT, 0, st>>>(Bm, n, nrhs, ipiv, L, status);
    for (int64_t j = 0; j + 1 < n; ++j)
      for (int64_t c0 = 0; c0 < nrhs; c0 += kMaxGridY)
        k_solve_fwd<<<dim3(blocks_for(2 * (n - j - 1), kT), (unsigned)std::min(kMaxGridY, nrhs - c0)), kT, 0, st>>>(
            Am, n, j, Bm, c0, p_bits, L, status);
    k_solve_last<<<blocks_for(2 * nrhs, kT), kT, 0, st>>>(Am, n - 1, Bm, nrhs, p_bits, L, status);
    for (int64_t j = n - 1; j >= 1; --j)
      for (int64_t c0 = 0; c0 < nrhs; c0 += kMaxGridY)
        k_solve_bwd<<<dim3(blocks_for(2 * j, kT), (unsigned)std::min(kMaxGridY, nrhs - c0)), kT, 0, st>>>(
            Am, j, Bm, c0, p_bits, L, status);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? MPC_OK : MPC_ECUDA - (int)e;
}
