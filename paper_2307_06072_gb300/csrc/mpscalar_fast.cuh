// Register-resident forms of the exact scalar operations of mpscalar.cuh (the complex
// FMA of the LU's updates, the pivot key, the trailing subtraction, the complex
// quotient) for operands of L limbs with L fixed at compile time (used for L = 4, 8).
//
// Same results as the generic forms (every value exact, one rounding to p
// bits, nearest-even), but every array has a compile-time size and is indexed
// with compile-time subscripts, so it lives in registers: shifts by a run-time
// number of bits go through log-step barrel shifters (selects between
// compile-time permutations) followed by one funnel shift per word.  A result
// whose exact window is wider than W = 2L + 3 words (terms whose exponents lie
// far apart) is left to the generic form (return value -1).
#pragma once

#include "mpscalar.cuh"

namespace mpc {
namespace fastmp {

// a <<= s (0 <= s < 64 W): bits shifted past the top are lost
template <int W>
__device__ __forceinline__ void shl(uint64_t (&a)[W], int s) {
  const int q = s >> 6, r = s & 63;
#pragma unroll
  for (int k = 0; (1 << k) < W; ++k) {
    if (q & (1 << k)) {
#pragma unroll
      for (int w = W - 1; w >= 0; --w) a[w] = w >= (1 << k) ? a[w - (1 << k)] : 0ull;
    }
  }
  if (r) {
#pragma unroll
    for (int w = W - 1; w >= 0; --w) a[w] = (a[w] << r) | (w > 0 ? a[w - 1] >> (64 - r) : 0ull);
  }
}

// a >>= s (0 <= s < 64 W), logical
template <int W>
__device__ __forceinline__ void shr(uint64_t (&a)[W], int s) {
  const int q = s >> 6, r = s & 63;
#pragma unroll
  for (int k = 0; (1 << k) < W; ++k) {
    if (q & (1 << k)) {
#pragma unroll
      for (int w = 0; w < W; ++w) a[w] = w + (1 << k) < W ? a[w + (1 << k)] : 0ull;
    }
  }
  if (r) {
#pragma unroll
    for (int w = 0; w < W; ++w) a[w] = (a[w] >> r) | (w + 1 < W ? a[w + 1] << (64 - r) : 0ull);
  }
}

// acc += t (sub: acc -= t), W words, two's complement
template <int W>
__device__ __forceinline__ void add_words(uint64_t (&acc)[W], const uint64_t (&t)[W], bool sub) {
  uint64_t carry = sub ? 1ull : 0ull;   // acc - t = acc + ~t + 1
#pragma unroll
  for (int w = 0; w < W; ++w) {
    const uint64_t v = sub ? ~t[w] : t[w];
    const uint64_t s1 = acc[w] + v;
    const uint64_t c1 = s1 < v;
    const uint64_t s2 = s1 + carry;
    carry = c1 | (s2 < s1);
    acc[w] = s2;
  }
}

// P (low 2L words of a W-word array) = x * y, magnitudes of L limbs each
template <int L, int W>
__device__ __forceinline__ void mul_limbs(const MPRef &x, const MPRef &y, uint64_t (&P)[W]) {
  uint64_t xs[L], ys[L];
#pragma unroll
  for (int a = 0; a < L; ++a) {
    xs[a] = x.limb[(int64_t)a * x.stride];
    ys[a] = y.limb[(int64_t)a * y.stride];
  }
#pragma unroll
  for (int u = 0; u < W; ++u) P[u] = 0;
#pragma unroll
  for (int a = 0; a < L; ++a) {
    uint64_t carry = 0;
#pragma unroll
    for (int b = 0; b < L; ++b) {
      const uint64_t lo = xs[a] * ys[b];
      uint64_t hi = __umul64hi(xs[a], ys[b]);
      uint64_t s = P[a + b] + lo;
      hi += (s < lo);
      s += carry;
      hi += (s < carry);
      P[a + b] = s;
      carry = hi;
    }
    P[a + L] = carry;
  }
}

// Exact signed sum of the terms in a W-word window (bit 0 worth 2^bot): 1 on success
// (acc = |sum|, neg its sign), 0 if every term is zero, -1 if the window is too narrow.
template <int L, int W>
__device__ __forceinline__ int sum_exact(const Term *t, int nt, uint64_t (&acc)[W], int64_t &bot, bool &neg) {
  int64_t top = INT64_MIN;
  bot = INT64_MAX;
  for (int x = 0; x < nt; ++x) {
    if (t[x].x.zero(L) || (t[x].has_y && t[x].y.zero(L))) continue;
    const int64_t e = t[x].has_y ? (int64_t)t[x].x.e + t[x].y.e : (int64_t)t[x].x.e;
    const int64_t b = e - (t[x].has_y ? 128 : 64) * (int64_t)L;
    top = max(top, e);
    bot = min(bot, b);
  }
  if (top == INT64_MIN) return 0;
  if (top - bot + 8 > 64 * (int64_t)W - 2) return -1;   // + growth of the few terms and the sign
#pragma unroll
  for (int w = 0; w < W; ++w) acc[w] = 0;
  for (int x = 0; x < nt; ++x) {
    if (t[x].x.zero(L) || (t[x].has_y && t[x].y.zero(L))) continue;
    const bool ng = (t[x].has_y ? (t[x].x.s ^ t[x].y.s) : t[x].x.s) ^ (t[x].neg ? 1 : 0);
    uint64_t v[W];
    int64_t sh;
    if (t[x].has_y) {
      mul_limbs<L, W>(t[x].x, t[x].y, v);
      sh = (int64_t)t[x].x.e + t[x].y.e - 128 * (int64_t)L - bot;
    } else {
#pragma unroll
      for (int u = 0; u < W; ++u) v[u] = u < L ? t[x].x.limb[(int64_t)u * t[x].x.stride] : 0ull;
      sh = (int64_t)t[x].x.e - 64 * (int64_t)L - bot;
    }
    shl<W>(v, (int)sh);
    add_words<W>(acc, v, ng);
  }
  neg = (acc[W - 1] >> 63) != 0;
  if (neg) {
    uint64_t cc = 1;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const uint64_t v = ~acc[w] + cc;
      cc = (cc && v == 0) ? 1ull : 0ull;
      acc[w] = v;
    }
  }
  return 1;
}

// RN_p of |value| = mag 2^lsb (mag: W words) with sign neg, into L limbs; false on
// int32 exponent overflow.  Same steps as round_store: the p bits below the leading
// one, the round bit below them, the sticky bit below that, ties to even.
template <int L, int W>
__device__ __forceinline__ bool round_store_w(const uint64_t (&mag)[W], int64_t lsb, bool neg, int p, MPOut o) {
  int N = 0;
#pragma unroll
  for (int w = W - 1; w >= 0; --w)
    if (N == 0 && mag[w]) N = 64 * w + 64 - __clzll((long long)mag[w]);
  if (N == 0) {
    store_zero(L, o.s, o.e, o.limb, o.stride);
    return true;
  }
  bool rbit = false, sticky = false;
  const int rb = N - p - 1;   // the round bit's position
  if (rb >= 0) {
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const int lo = 64 * w;
      if (rb >= lo && rb < lo + 64) {
        rbit = (mag[w] >> (rb - lo)) & 1ull;
        if (rb > lo) sticky |= (mag[w] & ((1ull << (rb - lo)) - 1ull)) != 0;
      } else if (lo + 64 <= rb) {
        sticky |= mag[w] != 0;
      }
    }
  }
  uint64_t M[W];   // mag shifted so that its leading one is bit 64L - 1
#pragma unroll
  for (int w = 0; w < W; ++w) M[w] = mag[w];
  if (N >= 64 * L) shr<W>(M, N - 64 * L);
  else shl<W>(M, 64 * L - N);
  const int cut = 64 * L - p;   // 0 <= cut < 64 for 64 (L - 1) < p <= 64 L
  if (cut) M[0] &= ~((1ull << cut) - 1ull);
  int64_t e = lsb + N;
  if (rbit && (sticky || ((M[0] >> cut) & 1ull))) {
    uint64_t carry = 1ull << cut;
#pragma unroll
    for (int j = 0; j < L; ++j) {
      const uint64_t t = M[j] + carry;
      carry = t < carry ? 1ull : 0ull;
      M[j] = t;
    }
    if (carry) {   // 2^(64L): renormalise
      M[L - 1] = 1ull << 63;
      e += 1;
    }
  }
  if (e > INT32_MAX || e < (int64_t)INT32_MIN + 1) return false;
  *o.s = neg ? 1 : 0;
  *o.e = (int32_t)e;
#pragma unroll
  for (int j = 0; j < L; ++j) o.limb[(int64_t)j * o.stride] = M[j];
  return true;
}

// RN_p of the exact sum of the terms: 1 / 0 as mp_sum_round (0 on exponent overflow),
// -1 when the terms' window is too wide for W words (then nothing is written).
template <int L>
__device__ __forceinline__ int sum_round(const Term *t, int nt, int p, MPOut o) {
  constexpr int W = 2 * L + 3;
  uint64_t acc[W];
  int64_t bot;
  bool neg;
  const int r = sum_exact<L, W>(t, nt, acc, bot, neg);
  if (r < 0) return -1;
  if (r == 0) {
    store_zero(L, o.s, o.e, o.limb, o.stride);
    return 1;
  }
  return round_store_w<L, W>(acc, bot, neg, p, o) ? 1 : 0;
}

// RN_p of num / den for exact magnitudes num 2^lsb_n, den 2^lsb_d (W words each, both
// nonzero): Q = floor(num 2^sh / den) with p + 3 or p + 4 bits by long division on
// 64-bit digits (Knuth, TAOCP vol. 2, Sec. 4.3.1, Algorithm D; each trial digit from a
// 128-by-64-bit division of the top two words, corrected with the divisor's second word)
// with compile-time lengths: the divisor is shifted so that its leading one is bit
// 64 W - 1, the dividend so that it has 64 W + p + 3 bits.  The remainder gives a sticky
// bit below Q.
template <int L, int W>
__device__ __forceinline__ bool div_round(const uint64_t (&num)[W], int64_t lsb_n, bool neg,
                                          const uint64_t (&den)[W], int64_t lsb_d, int p, MPOut o) {
  constexpr int UW = W + L + 1;            // dividend words: 64 W + p + 3 < 64 UW
  constexpr int QN = UW - W + 1;           // quotient digits
  int nN = 0, nD = 0;
#pragma unroll
  for (int w = W - 1; w >= 0; --w) {
    if (nN == 0 && num[w]) nN = 64 * w + 64 - __clzll((long long)num[w]);
    if (nD == 0 && den[w]) nD = 64 * w + 64 - __clzll((long long)den[w]);
  }
  uint64_t v[W];
#pragma unroll
  for (int w = 0; w < W; ++w) v[w] = den[w];
  shl<W>(v, 64 * W - nD);
  const int shift_u = p + 3 + 64 * W - nN;   // > 0: no dividend bit is dropped
  uint64_t uv[UW];
#pragma unroll
  for (int w = 0; w < UW; ++w) uv[w] = w < W ? num[w] : 0ull;
  shl<UW>(uv, shift_u);
  uint64_t u[UW + 1];
#pragma unroll
  for (int w = 0; w < UW; ++w) u[w] = uv[w];
  u[UW] = 0;
  uint64_t q[QN];
#pragma unroll
  for (int j = QN - 1; j >= 0; --j) {
    uint64_t qhat, rhat;
    bool rbig = false;   // rhat >= 2^64: the correction test cannot fail
    if (u[j + W] >= v[W - 1]) {   // (only equality can occur) qhat = 2^64 - 1
      qhat = ~0ull;
      const unsigned __int128 r = (unsigned __int128)u[j + W - 1] + v[W - 1];
      rbig = (uint64_t)(r >> 64) != 0;
      rhat = (uint64_t)r;
    } else {
      const unsigned __int128 top = ((unsigned __int128)u[j + W] << 64) | u[j + W - 1];
      qhat = (uint64_t)(top / v[W - 1]);
      rhat = (uint64_t)(top - (unsigned __int128)qhat * v[W - 1]);
    }
    while (!rbig && (unsigned __int128)qhat * v[W - 2] > (((unsigned __int128)rhat << 64) | u[j + W - 2])) {
      --qhat;
      const unsigned __int128 r = (unsigned __int128)rhat + v[W - 1];
      rbig = (uint64_t)(r >> 64) != 0;
      rhat = (uint64_t)r;
    }
    uint64_t borrow = 0;   // u[j .. j + W] -= qhat v
#pragma unroll
    for (int i = 0; i < W; ++i) {
      const unsigned __int128 pr = (unsigned __int128)qhat * v[i] + borrow;
      const uint64_t lo = (uint64_t)pr;
      borrow = (uint64_t)(pr >> 64);
      const uint64_t t = u[i + j] - lo;
      borrow += u[i + j] < lo ? 1ull : 0ull;
      u[i + j] = t;
    }
    const bool below = u[j + W] < borrow;
    u[j + W] -= borrow;
    if (below) {   // qhat was one too large: add the divisor back
      --qhat;
      uint64_t carry = 0;
#pragma unroll
      for (int i = 0; i < W; ++i) {
        const unsigned __int128 s2 = (unsigned __int128)u[i + j] + v[i] + carry;
        u[i + j] = (uint64_t)s2;
        carry = (uint64_t)(s2 >> 64);
      }
      u[j + W] += carry;
    }
    q[j] = qhat;
  }
  bool sticky = false;
#pragma unroll
  for (int i = 0; i < W; ++i) sticky |= u[i] != 0;
  // Q' = 2 Q + sticky, value Q' 2^(lsb_n - lsb_d - (shift_u - 64 W + nD) - 1)
  constexpr int QW = QN + 1;
  uint64_t Qs[QW];
  uint64_t c = sticky ? 1ull : 0ull;
#pragma unroll
  for (int i = 0; i < QW; ++i) {
    const uint64_t w = i < QN ? q[i] : 0ull;
    Qs[i] = (w << 1) | c;
    c = w >> 63;
  }
  return round_store_w<L, QW>(Qs, lsb_n - lsb_d - (int64_t)(shift_u - 64 * W + nD) - 1, neg, p, o);
}

// Both components of the complex quotient a / d, each RN_p of its exact value:
// (a_re d_re + a_im d_im) / |d|^2 and (a_im d_re - a_re d_im) / |d|^2.  1 / 0 as
// cdiv_store's flags (0: exponent overflow), -1 when a window is too wide (nothing
// written), 2 when d == 0 (nothing written; the caller refused it earlier).  Both
// quotients are rounded into temporaries before anything is stored: the output may be
// a itself.
template <int L>
__device__ __forceinline__ int cdiv(const MPRef &are, const MPRef &aim, const MPRef &dre, const MPRef &dim, int p,
                                    MPOut ore, MPOut oim) {
  constexpr int W = 2 * L + 3;
  uint64_t den[W], num0[W], num1[W];
  int64_t bd, b0, b1;
  bool nd, n0, n1;
  Term td[2] = {{dre, dre, true, false}, {dim, dim, true, false}};
  Term t0[2] = {{are, dre, true, false}, {aim, dim, true, false}};
  Term t1[2] = {{aim, dre, true, false}, {are, dim, true, true}};
  const int rd = sum_exact<L, W>(td, 2, den, bd, nd);
  if (rd < 0) return -1;
  if (rd == 0) return 2;
  const int r0 = sum_exact<L, W>(t0, 2, num0, b0, n0);
  const int r1 = sum_exact<L, W>(t1, 2, num1, b1, n1);
  if (r0 < 0 || r1 < 0) return -1;
  bool nz0 = false, nz1 = false;
#pragma unroll
  for (int w = 0; w < W; ++w) {
    nz0 |= r0 > 0 && num0[w] != 0;
    nz1 |= r1 > 0 && num1[w] != 0;
  }
  uint8_t sg[2];
  int32_t ex[2];
  uint64_t lm[2][L];
  MPOut tmp[2] = {{&sg[0], &ex[0], lm[0], 1}, {&sg[1], &ex[1], lm[1], 1}};
  bool ok = true;
  if (!nz0) store_zero(L, tmp[0].s, tmp[0].e, tmp[0].limb, 1);
  else ok &= div_round<L, W>(num0, b0, n0, den, bd, p, tmp[0]);
  if (!nz1) store_zero(L, tmp[1].s, tmp[1].e, tmp[1].limb, 1);
  else ok &= div_round<L, W>(num1, b1, n1, den, bd, p, tmp[1]);
  if (!ok) return 0;
  const MPOut outs[2] = {ore, oim};
#pragma unroll
  for (int c = 0; c < 2; ++c) {
    *outs[c].s = sg[c];
    *outs[c].e = ex[c];
#pragma unroll
    for (int j = 0; j < L; ++j) outs[c].limb[(int64_t)j * outs[c].stride] = lm[c][j];
  }
  return 1;
}

// Component c (0: real, 1: imaginary) of the complex quotient a / d into o: RN_p of
// (a_re d_re + a_im d_im) / |d|^2 or (a_im d_re - a_re d_im) / |d|^2.  1 / 0 / -1 / 2 as cdiv.
template <int L>
__device__ __forceinline__ int cdiv_part(const MPRef &are, const MPRef &aim, const MPRef &dre, const MPRef &dim, int c,
                                         int p, MPOut o) {
  constexpr int W = 2 * L + 3;
  uint64_t den[W], num[W];
  int64_t bd, bn;
  bool nd, nn;
  Term td[2] = {{dre, dre, true, false}, {dim, dim, true, false}};
  const int rd = sum_exact<L, W>(td, 2, den, bd, nd);
  if (rd < 0) return -1;
  if (rd == 0) return 2;
  Term t0[2] = {{are, dre, true, false}, {aim, dim, true, false}};
  Term t1[2] = {{aim, dre, true, false}, {are, dim, true, true}};
  const int rn = sum_exact<L, W>(c == 0 ? t0 : t1, 2, num, bn, nn);
  if (rn < 0) return -1;
  bool nz = false;
#pragma unroll
  for (int w = 0; w < W; ++w) nz |= rn > 0 && num[w] != 0;
  if (!nz) {
    store_zero(L, o.s, o.e, o.limb, o.stride);
    return 1;
  }
  return div_round<L, W>(num, bn, nn, den, bd, p, o) ? 1 : 0;
}

}  // namespace fastmp
}  // namespace mpc
