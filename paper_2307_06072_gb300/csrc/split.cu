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

// Per-part split: z_P = min over lines of floor((E_line - E^P_line) / w), E^P_line the
// largest exponent of part P (re or im) in the line (rows of A, columns of B); parts
// without a nonzero element leave the word at 0 (offset kZCap).  Stored as kZCap - z
// through atomicMax (the status block starts zeroed).
__global__ void k_part_rows(MatView A, int64_t m, int64_t k, int L, int w, const int32_t *E, int32_t *zw) {
  const int64_t i = blockIdx.x;
  if (i >= m || E[i] == INT32_MIN) return;
  int best[2] = {INT32_MIN, INT32_MIN};
  for (int64_t l = threadIdx.x; l < k; l += blockDim.x) {
    const int64_t idx = i * A.ld + l;
#pragma unroll
    for (int c = 0; c < 2; ++c)
      if (comp_nonzero(A, c, idx, L)) best[c] = max(best[c], A.exp[c][idx]);
  }
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    for (int o = 16; o > 0; o >>= 1) best[c] = max(best[c], __shfl_xor_sync(0xffffffffu, best[c], o));
    if ((threadIdx.x & 31) == 0 && best[c] != INT32_MIN) {
      const int64_t z = ((int64_t)E[i] - best[c]) / w;   // E_i >= every exponent of the row
      atomicMax(zw + c, kZCap - (int)(z < kZCap ? z : kZCap));
    }
  }
}

__global__ void k_part_cols(MatView B, int64_t k, int64_t n, int L, int w, const int32_t *F, int32_t *zw) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n || F[j] == INT32_MIN) return;
  int best[2] = {INT32_MIN, INT32_MIN};
  for (int64_t l = 0; l < k; ++l) {
    const int64_t idx = l * B.ld + j;
#pragma unroll
    for (int c = 0; c < 2; ++c)
      if (comp_nonzero(B, c, idx, L)) best[c] = max(best[c], B.exp[c][idx]);
  }
#pragma unroll
  for (int c = 0; c < 2; ++c)
    if (best[c] != INT32_MIN) {
      const int64_t z = ((int64_t)F[j] - best[c]) / w;
      atomicMax(zw + c, kZCap - (int)(z < kZCap ? z : kZCap));
    }
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
// mantissa, sh may be negative), read 32 bits at a time, least significant first,
// straight from the input limbs (as 32-bit halves): word w of |X| is bits
// [32 w + sh, 32 w + sh + 32) of M; the upper half-limb is kept for the following
// word, so every half-limb is loaded once and nothing is held in memory indexed at
// run time.
struct LimbStream {
  const uint32_t *p;   // low half of limb 0 (half-limb j at p[(j / 2) * 2 * stride + (j & 1)])
  int64_t j;           // index of the half-limb in `cur`
  uint32_t cur;
  int off;             // sh mod 32
  bool live;
  __device__ __forceinline__ uint32_t half(int64_t jj, int64_t stride, int L) const {
    return (live && jj >= 0 && jj < 2 * (int64_t)L) ? p[(jj >> 1) * 2 * stride + (jj & 1)] : 0u;
  }
  __device__ __forceinline__ void start(const uint64_t *base, bool nz, int64_t sh, int64_t stride, int L) {
    p = reinterpret_cast<const uint32_t *>(base);
    live = nz;
    off = (int)(sh & 31);
    j = sh >> 5;   // floor
    cur = half(j, stride, L);
  }
  __device__ __forceinline__ uint32_t next(int64_t stride, int L) {
    const uint32_t hi = half(j + 1, stride, L);
    const uint32_t x = __funnelshift_r(cur, hi, off);   // off = 0: cur
    cur = hi;
    ++j;
    return x;
  }
};

// Balanced digits without a carry per digit.  With H = sum_{pos < T-1} 2^(w-1) 2^(w pos)
// and Y = X + H (two's complement), the digits of X in base 2^w with the lower digits in
// [-2^(w-1), 2^(w-1)) are  d_pos = field_pos(Y) - 2^(w-1)  (pos < T-1) and the top digit
// d_{T-1} = Y >> w (T-1) (arithmetic), the unique such representation of X.
//
// Digits are produced in blocks of 32 (32 w bits = w 32-bit words of Y), so that every
// field sits at a compile-time bit offset.  bf16 of a digit: the float 2^23 + field
// (an integer OR) minus 2^23 + 2^(w-1) (one exact subtraction), whose upper 16 bits are
// the bf16 (|d| <= 256 has at most 8 significant bits).
template <int W>
__host__ __device__ constexpr uint32_t hpattern(int j) {   // H's bits in word j of a block
  uint32_t v = 0;
  for (int b = 0; b < 32; ++b)
    if ((32 * j + b) % W == W - 1) v |= 1u << b;
  return v;
}

// The `width` bits at [off, off + width) of the W words y, in the low bits of the result;
// `next` is the word that follows y.  Called with `off` and `width` constant after loop
// unrolling, so the indexing and shifts fold away.
template <int W>
__device__ __forceinline__ uint32_t bits_at(const uint32_t *y, uint32_t next, int off, int width) {
  const int wd = off / 32, sh = off % 32;
  if (sh + width <= 32) return y[wd] >> sh;
  return __funnelshift_r(y[wd], wd + 1 == W ? next : y[wd + 1], sh);
}

// One block of 32 digit positions (global positions 32 blk + i) of one digit stream of
// two elements: y0 / y1 hold the 32 w bits of Y for each element.  T = digit count;
// TAIL: this block holds digit T-1 (the top digit) or positions >= T.
template <int W, bool TAIL>
__device__ __forceinline__ void emit_block(const uint32_t *y0, const uint32_t *y1, uint32_t next0, uint32_t next1,
                                           int blk, int T, __nv_bfloat162 *out, int64_t plane_step, bool store,
                                           uint32_t &nzmask) {
  constexpr uint32_t MASK = (1u << W) - 1u;
  const float bias = 8388608.0f + (float)(1 << (W - 1));   // 2^23 + 2^(w-1)
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const int pos = 32 * blk + i;
    float d0, d1;
    if (TAIL && pos == T - 1) {   // top digit: Y >> w (T-1) as a signed (w+1)-bit value
      const uint32_t f0 = bits_at<W>(y0, next0, W * i, W + 1), f1 = bits_at<W>(y1, next1, W * i, W + 1);
      const int t0 = ((int32_t)(f0 << (31 - W))) >> (31 - W), t1 = ((int32_t)(f1 << (31 - W))) >> (31 - W);
      d0 = __int_as_float(0x4B000000 | (uint32_t)(t0 + 2 * (1 << (W - 1)))) - (8388608.0f + (float)(2 << (W - 1)));
      d1 = __int_as_float(0x4B000000 | (uint32_t)(t1 + 2 * (1 << (W - 1)))) - (8388608.0f + (float)(2 << (W - 1)));
    } else {
      const uint32_t f0 = bits_at<W>(y0, next0, W * i, W), f1 = bits_at<W>(y1, next1, W * i, W);
      d0 = __int_as_float(0x4B000000 | (f0 & MASK)) - bias;
      d1 = __int_as_float(0x4B000000 | (f1 & MASK)) - bias;
    }
    const uint32_t packed = __byte_perm(__float_as_uint(d0), __float_as_uint(d1), 0x7632);
    if (!TAIL || pos < T) {
      if (store) out[-(int64_t)pos * plane_step] = *reinterpret_cast<const __nv_bfloat162 *>(&packed);
      if (packed) nzmask |= 1u << i;
    }
  }
}

// One thread per (line, l, l+1): digits of two adjacent elements of a line.
// Side A: line = row i, element (i, l).  Side B: line = column j, element (l, j).
// Output planes: digits[(plane * lines + line) * kpad + l], plane = t (real),
// s + t (imaginary), 2s + 1 + t (sums, t = -1 .. s-1); digit position pos (least
// significant first) of the real part is plane s - 1 - pos.
template <int W>
__global__ void __launch_bounds__(128, 4) k_oz_digits(MatView X, int side, int64_t lines, int64_t k, int64_t kpad, int L,
                                                   int s, int want_sum, const int32_t *E, int32_t *lossy,
                                                   __nv_bfloat16 *digits, int32_t *plane_nz,
                                                   const int32_t *zoff) {
  __shared__ uint32_t nzbits[3][8];   // [stream][32-digit block]: a nonzero digit there
  __shared__ int nzcomp[2];
  if (threadIdx.x < 24) nzbits[threadIdx.x / 8][threadIdx.x % 8] = 0;
  if (threadIdx.x < 2) nzcomp[threadIdx.x] = 0;
  __syncthreads();
  const int64_t l0 = 2 * ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
  const int64_t line = blockIdx.y;
  // kpad is even: l0 + 1 < kpad; out-of-range threads still take part in the warp reductions
  const bool in_range = l0 < kpad && line < lines;
  const int64_t pstride2 = lines * kpad / 2;
  __nv_bfloat162 *out = reinterpret_cast<__nv_bfloat162 *>(digits + line * kpad + l0);
  const int32_t e_line = in_range ? E[line] : INT32_MIN;
  const int64_t xbits = (int64_t)W * s;                  // |X| < 2^(xbits - 1)
  LimbStream m[2][2];                                    // [element][re, im]
  uint32_t neg[2][2];
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
      // per-part split: part c sits z_c digit positions lower on the line's grid (its s digits
      // are those of X scaled by 2^(w(s + z_c) - 1 - E)); |X| < 2^(ws-1) still holds
      const int64_t xb = zoff ? (int64_t)W * (s + (kZCap - zoff[c])) : xbits;
      const int64_t sh = nzc ? (64 * (int64_t)L + (int64_t)e_line - (int64_t)X.exp[c][idx] - (xb - 1)) : 0;
      m[q][c].start(X.limb[c] + idx, nzc, sh, X.plane, L);
      neg[q][c] = (nzc && X.sign[c][idx]) ? 1u : 0u;
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
  }
  if (!ok) atomicOr(lossy + line, 1);
#pragma unroll
  for (int c = 0; c < 2; ++c)
    if (__any_sync(0xffffffffu, nzv[c]) && (threadIdx.x & 31) == 0) nzcomp[c] = 1;
  // Y = X'' + H + neg for the real and imaginary parts (X'' = |X| or its one's complement,
  // so that X'' + neg is X in two's complement) and Y = X''_re + X''_im + H' + neg_re + neg_im
  // for the 3M sum, 32 digit positions (W words of 32 bits) per block.
  uint32_t cy[2][3];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    cy[q][0] = neg[q][0];
    cy[q][1] = neg[q][1];
    cy[q][2] = neg[q][0] + neg[q][1];
  }
  const int Ts = s + 1;                                   // digits of the 3M sums
  const int nblk = ((want_sum ? Ts : s) + 31) / 32;
  for (int blk = 0; blk < nblk; ++blk) {
    uint32_t xw[2][2][W];                                 // [element][re, im] one's-complement words of |X|
#pragma unroll
    for (int j = 0; j < W; ++j) {
      const int64_t top = xbits - 32 * ((int64_t)blk * W + j);   // bits of |X| in this word
      const uint32_t tmask = top >= 32 ? ~0u : (top <= 0 ? 0u : ((1u << top) - 1u));
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const uint32_t x = m[q][c].next(X.plane, L) & tmask;
          xw[q][c][j] = neg[q][c] ? ~x : x;
        }
    }
    // One stream at a time (not unrolled: a single copy of the block code keeps the
    // instruction cache warm); operands and carries are picked by selects so that
    // nothing is indexed at run time.  Stream st: 0 re (X_re + H), 1 im (X_im + H),
    // 2 the 3M sums (X_re + X_im + H').
#pragma unroll 1
    for (int st = 0; st < (want_sum ? 3 : 2); ++st) {
      const int T = st == 2 ? Ts : s;
      if (32 * blk >= T) continue;
      uint32_t y[2][W];
      uint32_t c[2];
#pragma unroll
      for (int q = 0; q < 2; ++q) c[q] = st == 0 ? cy[q][0] : st == 1 ? cy[q][1] : cy[q][2];
#pragma unroll
      for (int j = 0; j < W; ++j) {
        const int64_t lim = (int64_t)W * (T - 1) - 32 * ((int64_t)blk * W + j);   // H below digit T-1 only
        const uint32_t h = hpattern<W>(j) & (lim >= 32 ? ~0u : (lim <= 0 ? 0u : ((1u << lim) - 1u)));
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const uint32_t x = st == 1 ? xw[q][1][j] : xw[q][0][j];
          const uint32_t x2 = st == 2 ? xw[q][1][j] : 0u;
          const uint64_t t = (uint64_t)x + x2 + h + c[q];   // carry in and out <= 2
          c[q] = (uint32_t)(t >> 32);
          y[q][j] = (uint32_t)t;
        }
      }
#pragma unroll
      for (int q = 0; q < 2; ++q) {
        if (st == 0) cy[q][0] = c[q];
        else if (st == 1) cy[q][1] = c[q];
        else cy[q][2] = c[q];
      }
      // planes: re  s-1-pos,  im  2s-1-pos,  sums  3s-pos
      const int64_t plane0 = st == 0 ? s - 1 : st == 1 ? 2 * s - 1 : 3 * s;
      uint32_t nzmask = 0;
      if (32 * blk + 31 < T - 1) {
        emit_block<W, false>(y[0], y[1], 0u, 0u, blk, T, out + plane0 * pstride2, pstride2, in_range, nzmask);
      } else {
        // The block holds the top digit, so every bit of |X| lies in it (w T <= 32 w (blk + 1))
        // and the word after it is the sign extension of X'' (-1 per negative input) plus the
        // carry: it gives the top digit's sign bit when that digit ends the block.
        uint32_t nxt[2];
#pragma unroll
        for (int q = 0; q < 2; ++q)
          nxt[q] = c[q] - (st == 0 ? neg[q][0] : st == 1 ? neg[q][1] : neg[q][0] + neg[q][1]);
        emit_block<W, true>(y[0], y[1], nxt[0], nxt[1], blk, T, out + plane0 * pstride2, pstride2, in_range, nzmask);
      }
      const uint32_t any = __reduce_or_sync(0xffffffffu, nzmask);
      if ((threadIdx.x & 31) == 0 && any) atomicOr(&nzbits[st][blk], any);
    }
  }
  __syncthreads();
  // plane flags: digit position pos of stream st is plane plane0(st) - pos
  const int ndig[3] = {s, s, want_sum ? Ts : 0};
  for (int st = 0; st < 3; ++st)
    for (int pos = threadIdx.x; pos < ndig[st]; pos += blockDim.x)
      if ((nzbits[st][pos >> 5] >> (pos & 31)) & 1u) {   // block pos / 32, digit pos % 32
        const int plane = st == 0 ? s - 1 - pos : st == 1 ? 2 * s - 1 - pos : 3 * s - pos;
        atomicOr(plane_nz + plane, 1);
      }
  const int nplanes = 2 * s + (want_sum ? Ts : 0);
  if (threadIdx.x < 2 && nzcomp[threadIdx.x]) atomicOr(plane_nz + nplanes + threadIdx.x, 1);
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

void launch_part_offsets(const MatView &A, const MatView &B, int64_t m, int64_t n, int64_t k, int L, int w,
                         const int32_t *E, const int32_t *F, int32_t *status, cudaStream_t st) {
  k_part_rows<<<(unsigned)m, 256, 0, st>>>(A, m, k, L, w, E, status + kStPartZ);
  k_part_cols<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(B, k, n, L, w, F, status + kStPartZ + 2);
}

void launch_oz_digits(const MatView &X, int side, int64_t lines, int64_t k, int64_t kpad, int L, int s, int wd,
                      int want_sum, const int32_t *E, int32_t *lossy, __nv_bfloat16 *digits, int32_t *plane_nz,
                      const int32_t *zoff, cudaStream_t st) {
  dim3 g((unsigned)((kpad / 2 + 127) / 128), (unsigned)lines);
  if (wd == 9)
    k_oz_digits<9><<<g, 128, 0, st>>>(X, side, lines, k, kpad, L, s, want_sum, E, lossy, digits, plane_nz, zoff);
  else
    k_oz_digits<8><<<g, 128, 0, st>>>(X, side, lines, k, kpad, L, s, want_sum, E, lossy, digits, plane_nz, zoff);
}

void launch_plain_digits(const MatView &X, int side, int64_t lines, int64_t k, int L, int D, int DP, int W,
                         int want_sum, const int32_t *E, int32_t *lossy, int32_t *digits, cudaStream_t st) {
  const int64_t fast = side == 0 ? k : lines, slow = side == 0 ? lines : k;
  dim3 g((unsigned)((fast + 127) / 128), (unsigned)(slow < 65535 ? slow : 65535));
  k_plain_digits<<<g, 128, 0, st>>>(X, side, lines, k, L, D, DP, W, want_sum, E, lossy, digits);
}

}  // namespace mpc
