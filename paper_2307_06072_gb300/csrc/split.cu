// oz_split: the first half of Alg. 2 (Kouya, Sec. III-C) on the GPU.
//
//  * k_rowmax / k_colmax: mu_A / mu_B of Alg. 2 as exponents -- E_i, the
//    largest exponent of row i of A over the real AND imaginary planes (one
//    split for both parts, last paragraph of Sec. III-C), F_j likewise for
//    column j of B.  Every |a_il| < 2^E_i.
//  * k_oz_digits: the split itself.  Alg. 2 cuts A on a grid set by tau into
//    short floats whose products are exact.  Here the grid is fixed per row:
//    X = sign * floor(|a| 2^(ws-1-E)) and X is written in s balanced base-2^w
//    digits (w = 9 or 8: |d| <= 2^(w-1) <= 256, exact in bf16, products
//    exact), most significant first; digit t stands for slice A_{t+1}.  For
//    the 3M form (Eq. 3m_way)
//    the digits of X_re + X_im are produced as well (s+1 digits).  B is split
//    by columns and stored transposed (K-major), as the tensor cores read it.
//  * k_plain_digits: the plain path's fixed-point operands as signed
//    base-2^28 digits.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace mpc {

__device__ __forceinline__ bool comp_nonzero(const MatView &X, int c, int64_t idx, int L) {
  return X.limb[c][(int64_t)(L - 1) * X.plane + idx] != 0;
}

// E for each row of A (m x k): block per row, threads stride the row.
__global__ void k_rowmax(MatView A, int64_t m, int64_t k, int L, int32_t *E) {
  int64_t i = blockIdx.x;
  if (i >= m) return;
  int best = INT32_MIN;
  for (int64_t l = threadIdx.x; l < k; l += blockDim.x) {
    int64_t idx = i * A.ld + l;
#pragma unroll
    for (int c = 0; c < 2; ++c)
      if (comp_nonzero(A, c, idx, L)) best = max(best, A.exp[c][idx]);
  }
  for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
  __shared__ int red[32];
  int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) red[w] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    int r = INT32_MIN;
    for (int v = 0; v < (int)(blockDim.x >> 5); ++v) r = max(r, red[v]);
    E[i] = r;
  }
}

// F for each column of B (k x n): threads over columns, blocks over row chunks.
__global__ void k_colmax(MatView B, int64_t k, int64_t n, int L, int rows_per_block, int32_t *F) {
  int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  int64_t l0 = (int64_t)blockIdx.y * rows_per_block;
  int64_t l1 = min(k, l0 + rows_per_block);
  int best = INT32_MIN;
  for (int64_t l = l0; l < l1; ++l) {
    int64_t idx = l * B.ld + j;
#pragma unroll
    for (int c = 0; c < 2; ++c)
      if (comp_nonzero(B, c, idx, L)) best = max(best, B.exp[c][idx]);
  }
  if (best != INT32_MIN) atomicMax(F + j, best);
}

__global__ void k_init(int32_t *status, int32_t *E, int64_t m, int32_t *F, int64_t n, int32_t *lossyA,
                       int32_t *lossyB, int32_t *extra, int64_t n_extra) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < kStatusWords) status[t] = 0;
  if (t < n_extra) extra[t] = 0;
  if (t < m) { E[t] = INT32_MIN; lossyA[t] = 0; }
  if (t < n) { F[t] = INT32_MIN; lossyB[t] = 0; }
}

// 8 bits of the L-limb integer M starting at bit b (zero outside [0, 64L)).
__device__ __forceinline__ uint32_t byte_at(const uint64_t *M, int L, int64_t b) {
  if (b >= 64 * (int64_t)L || b <= -8) return 0;
  int64_t w = b >> 6;                 // floor division (b may be negative)
  int off = (int)(b & 63);
  uint64_t lo = (w >= 0 && w < L) ? M[w] : 0ull;
  uint64_t hi = (w + 1 >= 0 && w + 1 < L) ? M[w + 1] : 0ull;
  uint64_t v = off ? ((lo >> off) | (hi << (64 - off))) : lo;
  return (uint32_t)(v & 0xFFu);
}

// true iff every bit of M below bit `nb` is zero
__device__ __forceinline__ bool low_bits_zero(const uint64_t *M, int L, int64_t nb) {
  if (nb <= 0) return true;
  for (int j = 0; j < L; ++j) {
    int64_t lo = 64 * (int64_t)j;
    if (lo >= nb) break;
    int64_t take = nb - lo;
    uint64_t mask = take >= 64 ? ~0ull : ((1ull << take) - 1ull);
    if (M[j] & mask) return false;
  }
  return true;
}

// 64 bits of the L-limb integer M starting at bit b (zero outside [0, 64L)).
__device__ __forceinline__ uint64_t word_at_bit(const uint64_t *M, int L, int64_t b) {
  if (b >= 64 * (int64_t)L || b <= -64) return 0;
  const int64_t w = b >> 6;           // floor division (b may be negative)
  const int off = (int)(b & 63);
  const uint64_t lo = (w >= 0 && w < L) ? M[w] : 0ull;
  const uint64_t hi = (w + 1 >= 0 && w + 1 < L) ? M[w + 1] : 0ull;
  return off ? ((lo >> off) | (hi << (64 - off))) : lo;
}

// Per element and component: the shifted magnitude |X| = M >> sh (M the L-limb
// mantissa, sh may be negative), read 64 bits at a time, least significant first,
// straight from the input limbs: word w of |X| is bits [64 w + sh, 64 w + sh + 64)
// of M, i.e. limbs w + floor(sh / 64) and the next one; the next one is kept for
// the following word, so every limb is loaded once and nothing is held in memory
// indexed at run time.
struct LimbStream {
  const uint64_t *p;   // limb 0 of the element (limb j at p[j * stride])
  int64_t j;           // index of the limb in `cur`
  uint64_t cur;
  int off;             // sh mod 64
  bool live;
  __device__ __forceinline__ uint64_t limb(int64_t jj, int64_t stride, int L) const {
    return (live && jj >= 0 && jj < L) ? p[jj * stride] : 0ull;
  }
  __device__ __forceinline__ void start(const uint64_t *base, bool nz, int64_t sh, int64_t stride, int L) {
    p = base;
    live = nz;
    off = (int)(sh & 63);
    j = sh >> 6;   // floor
    cur = limb(j, stride, L);
  }
  __device__ __forceinline__ uint64_t next(int64_t stride, int L) {
    const uint64_t hi = limb(j + 1, stride, L);
    const uint64_t x = off ? ((cur >> off) | (hi << (64 - off))) : cur;
    cur = hi;
    ++j;
    return x;
  }
};

// One thread per (line, l, l+1): digits of two adjacent elements of a line.
// Side A: line = row i, element (i, l).  Side B: line = column j, element (l, j).
// Output planes: digits[(plane * lines + line) * kpad + l], plane = t (real),
// s + t (imaginary), 2s + 1 + t (sums, t = -1 .. s-1).
__device__ __forceinline__ void oz_digits_pair(const MatView &X, int side, int64_t lines, int64_t k, int64_t kpad,
                                               int L, int s, int wd, int want_sum, const int32_t *E, int32_t *lossy,
                                               __nv_bfloat16 *digits, int64_t l0, int64_t line, bool in_range,
                                               int *nz) {
  const bool leader = (threadIdx.x & 31) == 0;
  const int64_t pstride = lines * kpad;
  __nv_bfloat162 *out = reinterpret_cast<__nv_bfloat162 *>(digits + line * kpad + l0);
  const int64_t pstride2 = pstride / 2;
  const int nplanes = 2 * s + (want_sum ? s + 1 : 0);
  const int32_t e_line = in_range ? E[line] : INT32_MIN;
  const int64_t xbits = (int64_t)wd * s;                 // |X| < 2^(xbits - 1)
  LimbStream m[2][2];                                    // [element][re, im]
  bool neg[2][2];
  uint64_t cneg[2][2], csum[2];                          // two's-complement and X_re + X_im carries
  int cbal[2][2], cbal_s[2];                             // balanced-digit carries
  bool ok = true;
  bool nzv[2] = {false, false};   // a nonzero real / imaginary value among the two elements
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int64_t l = l0 + q;
    const bool live = in_range && (l < k) && (e_line != INT32_MIN);
    const int64_t idx = side == 0 ? line * X.ld + l : l * X.ld + line;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const bool nzc = live && comp_nonzero(X, c, idx, L);
      if (nzc) nzv[c] = true;
      // |X| bit b  <->  M bit b + sh:  X = |v| 2^(ws-1-E), |v| = M 2^(exp-64L)
      const int64_t sh = nzc ? (64 * (int64_t)L + (int64_t)e_line - (int64_t)X.exp[c][idx] - (xbits - 1)) : 0;
      m[q][c].start(X.limb[c] + idx, nzc, sh, X.plane, L);
      neg[q][c] = nzc && X.sign[c][idx];
      cneg[q][c] = 1;
      cbal[q][c] = 0;
      if (nzc && sh > 0) {   // the bits of M below sh are dropped: the line is lossy unless they are zero
        if (sh >= 64 * (int64_t)L) {
          ok = false;
        } else {
          for (int jj = 0; jj < L && 64 * (int64_t)jj < sh; ++jj) {
            const int64_t take = sh - 64 * (int64_t)jj;
            const uint64_t mask = take >= 64 ? ~0ull : ((1ull << take) - 1ull);
            if (X.limb[c][(int64_t)jj * X.plane + idx] & mask) ok = false;
          }
        }
      }
    }
    csum[q] = 0;
    cbal_s[q] = 0;
  }
  if (!ok) atomicOr(lossy + line, 1);
#pragma unroll
  for (int c = 0; c < 2; ++c)
    if (__ballot_sync(0xffffffffu, nzv[c]) && leader) nz[nplanes + c] = 1;
  // Digits, least significant first, from LSB-first bit streams of the two's-complement
  // words of X_re, X_im (wd*s bits) and X_re + X_im: every stream keeps a 128-bit buffer
  // (lo, hi) holding `nbuf` bits; all streams advance in step (wd bits per digit).
  const int ndig = want_sum ? s + 1 : s;
  const uint32_t fmask = (1u << wd) - 1u;
  const int half = 1 << (wd - 1), full = 1 << wd;
  uint64_t blo[2][3], bhi[2][3];                         // [element][re, im, sum]
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int c = 0; c < 3; ++c) blo[q][c] = bhi[q][c] = 0;
  int nbuf = 0, wnext = 0;
  for (int pos = 0; pos < ndig; ++pos) {
    if (nbuf < wd) {   // append word `wnext` of every stream above the bits still buffered
      uint64_t wc[2][3];
      const int64_t top = xbits - 64 * (int64_t)wnext;   // bits of |X| in this word
      const uint64_t tmask = top >= 64 ? ~0ull : (top <= 0 ? 0ull : ((1ull << top) - 1ull));
#pragma unroll
      for (int q = 0; q < 2; ++q) {
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          uint64_t x = m[q][c].next(X.plane, L) & tmask;
          if (neg[q][c]) {
            const uint64_t t = ~x + cneg[q][c];
            cneg[q][c] = (cneg[q][c] && t == 0) ? 1ull : 0ull;
            x = t;
          }
          wc[q][c] = x;
        }
        const uint64_t a0 = wc[q][0] + wc[q][1];
        const uint64_t c1 = a0 < wc[q][0];
        const uint64_t a1 = a0 + csum[q];
        const uint64_t c2 = a1 < a0;
        wc[q][2] = a1;
        csum[q] = c1 | c2;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          blo[q][c] |= wc[q][c] << nbuf;
          bhi[q][c] = nbuf ? (wc[q][c] >> (64 - nbuf)) : 0ull;
        }
      }
      nbuf += 64;
      ++wnext;
    }
    int fld[2][3];
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        fld[q][c] = (int)(blo[q][c] & fmask);
        blo[q][c] = (blo[q][c] >> wd) | (bhi[q][c] << (64 - wd));
        bhi[q][c] >>= wd;
      }
    nbuf -= wd;
    if (pos < s) {
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        float f[2];
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          int dg;
          if (pos == s - 1) {   // top digit: the signed field plus the carry
            dg = (fld[q][c] >= half ? fld[q][c] - full : fld[q][c]) + cbal[q][c];
          } else {
            dg = fld[q][c] + cbal[q][c];
            cbal[q][c] = dg >= half;
            if (dg >= half) dg -= full;
          }
          f[q] = (float)dg;
        }
        if (in_range) out[(int64_t)(c * s + (s - 1 - pos)) * pstride2] = __floats2bfloat162_rn(f[0], f[1]);
        if (__ballot_sync(0xffffffffu, f[0] != 0.f || f[1] != 0.f) && leader) nz[c * s + (s - 1 - pos)] = 1;
      }
    }
    if (want_sum) {
      float f[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        int dg;
        if (pos == s) {
          dg = (fld[q][2] >= half ? fld[q][2] - full : fld[q][2]) + cbal_s[q];
        } else {
          dg = fld[q][2] + cbal_s[q];
          cbal_s[q] = dg >= half;
          if (dg >= half) dg -= full;
        }
        f[q] = (float)dg;
      }
      if (in_range) out[(int64_t)(2 * s + (s - pos)) * pstride2] = __floats2bfloat162_rn(f[0], f[1]);
      if (__ballot_sync(0xffffffffu, f[0] != 0.f || f[1] != 0.f) && leader) nz[2 * s + (s - pos)] = 1;
    }
  }
}

// Digit planes of one operand; plane_nz[x] is set when plane x has a nonzero digit
// (the group table then skips the slice pairs of all-zero planes), and
// plane_nz[nplanes + c] when component c (re, im) has a nonzero value.
__global__ void k_oz_digits(MatView X, int side, int64_t lines, int64_t k, int64_t kpad, int L, int s,
                            int wd, int want_sum, const int32_t *E, int32_t *lossy, __nv_bfloat16 *digits,
                            int32_t *plane_nz) {
  __shared__ int nz[3 * kMaxSlices + 1 + 2];
  const int nflags = 2 * s + (want_sum ? s + 1 : 0) + 2;
  for (int x = threadIdx.x; x < nflags; x += blockDim.x) nz[x] = 0;
  __syncthreads();
  const int64_t l0 = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  const int64_t line = blockIdx.y;
  // kpad is even: l0 + 1 < kpad; out-of-range threads still take part in the warp votes
  oz_digits_pair(X, side, lines, k, kpad, L, s, wd, want_sum, E, lossy, digits, l0, line, l0 < kpad && line < lines,
                 nz);
  __syncthreads();
  for (int x = threadIdx.x; x < nflags; x += blockDim.x)
    if (nz[x]) atomicOr(plane_nz + x, 1);
}

// Plain path: X = floor(|a| 2^(64 Lp - E)) as Lp limbs (Lp = L + 1), sign kept apart.
// Layout: fix[(c * Lp + j) * lines * k + line * k + l], fsign[c * lines * k + line * k + l].
// Plain path operands.  Per row of A (column of B) the fixed point
//     X = sign * floor(|x| 2^(W - E_line)),   |X| < 2^W,  W = 28 D - 2,
// written in D balanced base-2^28 digits, least significant first:
// X = sum_t d_t 2^(28 t) with |d_t| <= 2^27, so that every digit product is
// below 2^54 in magnitude and a signed 64-bit column sum absorbs hundreds of
// them.  With want_sum (3M) a third plane holds the digits of X_re + X_im
// (|X_re + X_im| < 2^(W+1); its top digit is left unnormalised, still
// |d| <= 2^27).  Layout [plane][line][l][DP] (DP = D rounded up to 4).  A
// line is lossy when some element dropped nonzero bits (exponent more than
// W - p below E_line).  Threads run along the contiguous index of the matrix
// (l for A, the column for B); the second grid dimension strides.
__global__ void k_plain_digits(MatView X, int side, int64_t lines, int64_t k, int L, int D, int DP, int W,
                               int want_sum, const int32_t *E, int32_t *lossy, int32_t *digits) {
  const int64_t fast = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nslow = side == 0 ? lines : k;
  if (fast >= (side == 0 ? k : lines)) return;
  for (int64_t slow = blockIdx.y; slow < nslow; slow += gridDim.y) {
    const int64_t line = side == 0 ? slow : fast, l = side == 0 ? fast : slow;
    const int64_t idx = side == 0 ? line * X.ld + l : l * X.ld + line;
    const int32_t e_line = E[line];
    const int64_t plane = lines * k * DP;
    int32_t *out = digits + (line * k + l) * DP;
    int32_t dsum[kMaxPlainDigits];
    bool ok = true;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const bool nz = (e_line != INT32_MIN) && comp_nonzero(X, c, idx, L);
      uint64_t M[kMaxLimbs];
#pragma unroll
      for (int j = 0; j < kMaxLimbs; ++j) M[j] = (nz && j < L) ? X.limb[c][(int64_t)j * X.plane + idx] : 0ull;
      // |X| = M 2^sh (truncated); exp <= E_line, so sh <= W - 64 L
      const int64_t sh = nz ? (int64_t)W - 64 * (int64_t)L - ((int64_t)e_line - (int64_t)X.exp[c][idx]) : 0;
      if (nz && sh < 0 && (-sh >= 64 * (int64_t)L || !low_bits_zero(M, L, -sh))) ok = false;
      const bool neg = nz && X.sign[c][idx];
      int32_t carry = 0;
#pragma unroll
      for (int t = 0; t < kMaxPlainDigits; ++t) {
        if (t >= D) break;
        const uint32_t u = nz ? (uint32_t)(word_at_bit(M, L, 28 * (int64_t)t - sh) & 0xFFFFFFFull) : 0u;
        int32_t v = (int32_t)u + carry;              // [0, 2^28]
        carry = v >= (1 << 27) ? 1 : 0;
        v -= carry << 28;                            // [-2^27, 2^27)
        const int32_t d = neg ? -v : v;
        out[(int64_t)c * plane + t] = d;
        dsum[t] = c == 0 ? d : dsum[t] + d;
      }
      for (int t = D; t < DP; ++t) out[(int64_t)c * plane + t] = 0;
    }
    if (want_sum) {
      int32_t cy = 0;
#pragma unroll
      for (int t = 0; t < kMaxPlainDigits; ++t) {
        if (t >= D) break;
        int32_t v = dsum[t] + cy;                    // |v| <= 2^28 + 1
        if (t < D - 1) {
          cy = (v + (1 << 27)) >> 28;                // floor: v - cy 2^28 in [-2^27, 2^27)
          v -= cy * (1 << 28);
        }
        out[2 * plane + t] = v;
      }
      for (int t = D; t < DP; ++t) out[2 * plane + t] = 0;
    }
    if (!ok) atomicOr(lossy + line, 1);
  }
}

// ---------------------------------------------------------------- launchers

void launch_init(int32_t *status, int32_t *E, int64_t m, int32_t *F, int64_t n, int32_t *lossyA, int32_t *lossyB,
                 cudaStream_t st, int32_t *extra, int64_t n_extra) {
  int64_t tot = m > n ? m : n;
  if (tot < kStatusWords) tot = kStatusWords;
  if (tot < n_extra) tot = n_extra;
  k_init<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(status, E, m, F, n, lossyA, lossyB, extra, n_extra);
}

void launch_line_max(const MatView &A, const MatView &B, int64_t m, int64_t n, int64_t k, int L, int32_t *E,
                     int32_t *F, cudaStream_t st) {
  k_rowmax<<<(unsigned)m, 256, 0, st>>>(A, m, k, L, E);
  const int rpb = 64;
  dim3 g((unsigned)((n + 127) / 128), (unsigned)((k + rpb - 1) / rpb));
  k_colmax<<<g, 128, 0, st>>>(B, k, n, L, rpb, F);
}

void launch_oz_digits(const MatView &X, int side, int64_t lines, int64_t k, int64_t kpad, int L, int s, int wd,
                      int want_sum, const int32_t *E, int32_t *lossy, __nv_bfloat16 *digits, int32_t *plane_nz,
                      cudaStream_t st) {
  dim3 g((unsigned)((kpad / 2 + 127) / 128), (unsigned)lines);
  k_oz_digits<<<g, 128, 0, st>>>(X, side, lines, k, kpad, L, s, wd, want_sum, E, lossy, digits, plane_nz);
}

void launch_plain_digits(const MatView &X, int side, int64_t lines, int64_t k, int L, int D, int DP, int W,
                         int want_sum, const int32_t *E, int32_t *lossy, int32_t *digits, cudaStream_t st) {
  const int64_t fast = side == 0 ? k : lines, slow = side == 0 ? lines : k;
  dim3 g((unsigned)((fast + 127) / 128), (unsigned)(slow < 65535 ? slow : 65535));
  k_plain_digits<<<g, 128, 0, st>>>(X, side, lines, k, L, D, DP, W, want_sum, E, lossy, digits);
}

}  // namespace mpc
