// Exact multiple-precision scalar arithmetic on the GPU (one thread per result).
//
// A real component is (sign, exp, L limbs) in the library's format.  Results
// are formed exactly in a two's-complement fixed-point window and rounded
// once to p bits, nearest-even:
//   * mp_sum_round: sum of a few signed terms, each a component or a
//     product of two components (the complex FMA of the LU's updates, Eq.
//     4m_way_base per component);
//   * mp_cdiv_round: a component of the complex quotient a / d, i.e.
//     (a_re d_re + a_im d_im) / |d|^2 or (a_im d_re - a_re d_im) / |d|^2,
//     from exact numerator and denominator by long division on 32-bit
//     digits (Knuth's Algorithm D).
// If a term lies more than the window below the largest one, its low bits
// are dropped and `truncated` is reported (the caller records it).
#pragma once

#include "common.cuh"

namespace mpc {

constexpr int kWinLimbs = 64;   // 4096-bit window

struct MPRef {                  // one real component: value = (-1)^s M 2^(e - 64L)
  uint8_t s;
  int32_t e;
  const uint64_t *limb;         // limb j at limb[j * stride]
  int64_t stride;
  __device__ __forceinline__ bool zero(int L) const { return limb[(int64_t)(L - 1) * stride] == 0; }
};

__device__ __forceinline__ MPRef mp_ref(const uint8_t *sign, const int32_t *exp, const uint64_t *limb,
                                        int64_t plane, int64_t idx) {
  return MPRef{sign[idx], exp[idx], limb + idx, plane};
}

struct Term {                   // sign * x (* y)
  MPRef x, y;
  bool has_y, neg;
};

struct WinAcc {                 // 32-bit words of a little-endian uint64 array
  const uint64_t *base;
  __device__ __forceinline__ uint32_t operator()(int i) const { return (uint32_t)(base[i >> 1] >> (32 * (i & 1))); }
};

// win (nw limbs, two's complement) += / -= (P << shift), P = np limbs; shift may be < 0 (low bits dropped)
__device__ inline void win_add(uint64_t *win, int nw, const uint64_t *P, int np, int64_t shift, bool sub) {
  const int64_t w0 = shift >= 0 ? (shift >> 6) : 0;
  const int64_t wtop = (shift + 64 * (int64_t)np) / 64 + 1;
  uint64_t carry = 0;
  for (int64_t w = w0; w < nw; ++w) {
    uint64_t v = 0;
    if (w <= wtop) {
      const int64_t b = 64 * w - shift;
      if (b < 64 * (int64_t)np && b > -64) {
        const int64_t q = b >= 0 ? (b >> 6) : -1;
        const int off = (int)(b - 64 * q);
        const uint64_t lo = (q >= 0 && q < np) ? P[q] : 0ull;
        const uint64_t hi = (q + 1 >= 0 && q + 1 < np) ? P[q + 1] : 0ull;
        v = off ? ((lo >> off) | (hi << (64 - off))) : lo;
      }
    } else if (carry == 0) {
      break;
    }
    if (!sub) {
      uint64_t s = win[w] + v;
      uint64_t c1 = s < v;
      s += carry;
      c1 |= (s < carry);
      win[w] = s;
      carry = c1;
    } else {
      const uint64_t d = win[w] - v;
      uint64_t b1 = win[w] < v;
      const uint64_t d2 = d - carry;
      b1 |= (d < carry);
      win[w] = d2;
      carry = b1;
    }
  }
}

__device__ inline void limbs_mul(const MPRef &x, const MPRef &y, int L, uint64_t *P) {
  for (int u = 0; u < 2 * L; ++u) P[u] = 0;
  for (int a = 0; a < L; ++a) {
    const uint64_t xa = x.limb[(int64_t)a * x.stride];
    uint64_t carry = 0;
    for (int b = 0; b < L; ++b) {
      const uint64_t yb = y.limb[(int64_t)b * y.stride];
      const uint64_t lo = xa * yb;
      uint64_t hi = __umul64hi(xa, yb);
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

// Exact signed sum of the terms in a window; returns false if all terms are zero.
// On return: win holds |sum| (nw limbs), *neg its sign, *lsb the exponent of bit 0.
__device__ inline bool mp_sum_exact(const Term *t, int nt, int L, uint64_t *win, int *nw_out, int64_t *lsb,
                                    bool *neg, bool *truncated) {
  int64_t top = INT64_MIN, bot = INT64_MAX;
  for (int x = 0; x < nt; ++x) {
    if (t[x].x.zero(L) || (t[x].has_y && t[x].y.zero(L))) continue;
    const int64_t e = t[x].has_y ? (int64_t)t[x].x.e + t[x].y.e : (int64_t)t[x].x.e;
    const int64_t b = e - (t[x].has_y ? 128 : 64) * (int64_t)L;
    top = max(top, e);
    bot = min(bot, b);
  }
  if (top == INT64_MIN) return false;
  int64_t width = top - bot + 8;         // + growth of up to 2^8 terms and the sign
  int nw = (int)(width / 64 + 2);
  *truncated = false;
  if (nw > kWinLimbs) {
    nw = kWinLimbs;
    bot = top + 8 - 64 * (int64_t)(nw - 1);
    *truncated = true;
  }
  for (int w = 0; w < nw; ++w) win[w] = 0;
  uint64_t P[2 * kMaxLimbs];
  for (int x = 0; x < nt; ++x) {
    if (t[x].x.zero(L) || (t[x].has_y && t[x].y.zero(L))) continue;
    const bool ng = (t[x].has_y ? (t[x].x.s ^ t[x].y.s) : t[x].x.s) ^ (t[x].neg ? 1 : 0);
    if (t[x].has_y) {
      limbs_mul(t[x].x, t[x].y, L, P);
      win_add(win, nw, P, 2 * L, (int64_t)t[x].x.e + t[x].y.e - 128 * (int64_t)L - bot, ng);
    } else {
      for (int u = 0; u < L; ++u) P[u] = t[x].x.limb[(int64_t)u * t[x].x.stride];
      win_add(win, nw, P, L, (int64_t)t[x].x.e - 64 * (int64_t)L - bot, ng);
    }
  }
  *neg = (win[nw - 1] >> 63) != 0;
  if (*neg) {
    uint64_t cc = 1;
    for (int w = 0; w < nw; ++w) {
      const uint64_t v = ~win[w] + cc;
      cc = (cc && v == 0) ? 1ull : 0ull;
      win[w] = v;
    }
  }
  *nw_out = nw;
  *lsb = bot;
  return true;
}

struct MPOut {
  uint8_t *s;
  int32_t *e;
  uint64_t *limb;
  int64_t stride;
};

// RN_p of the exact sum of the terms; returns false on int32 exponent overflow.
__device__ inline bool mp_sum_round(const Term *t, int nt, int p, int L, MPOut o, bool *truncated) {
  uint64_t win[kWinLimbs];
  int nw;
  int64_t lsb;
  bool neg;
  if (!mp_sum_exact(t, nt, L, win, &nw, &lsb, &neg, truncated)) {
    store_zero(L, o.s, o.e, o.limb, o.stride);
    return true;
  }
  WinAcc mag{win};
  const int N = bitlen(mag, 2 * nw);
  if (N == 0) {
    store_zero(L, o.s, o.e, o.limb, o.stride);
    return true;
  }
  return round_store(mag, 2 * nw, N, neg, lsb, p, L, o.s, o.e, o.limb, o.stride);
}

// Quotient and remainder of unsigned 32-bit-digit integers (Knuth, TAOCP vol. 2,
// Sec. 4.3.1, Algorithm D): u[0..m) / v[0..n), v[n-1] != 0, m >= n.  q gets
// m - n + 1 digits; returns true iff the remainder is nonzero.  u is clobbered.
__device__ inline bool divmod_digits(uint32_t *u, int m, const uint32_t *v, int n, uint32_t *q) {
  if (n == 1) {
    uint64_t r = 0;
    for (int i = m - 1; i >= 0; --i) {
      const uint64_t cur = (r << 32) | u[i];
      q[i] = (uint32_t)(cur / v[0]);
      r = cur - (uint64_t)q[i] * v[0];
    }
    return r != 0;
  }
  constexpr int kMaxV = 80;
  uint32_t vn[kMaxV];
  const int s = __clz(v[n - 1]);     // normalise: top digit of the divisor gets its high bit set
  for (int i = n - 1; i > 0; --i) vn[i] = (v[i] << s) | (s ? (uint32_t)((uint64_t)v[i - 1] >> (32 - s)) : 0u);
  vn[0] = v[0] << s;
  // un = u << s, one digit longer
  uint32_t top = s ? (uint32_t)((uint64_t)u[m - 1] >> (32 - s)) : 0u;
  for (int i = m - 1; i > 0; --i) u[i] = (u[i] << s) | (s ? (uint32_t)((uint64_t)u[i - 1] >> (32 - s)) : 0u);
  u[0] = u[0] << s;
  u[m] = top;
  for (int j = m - n; j >= 0; --j) {
    const uint64_t num2 = ((uint64_t)u[j + n] << 32) | u[j + n - 1];
    uint64_t qhat = num2 / vn[n - 1];
    uint64_t rhat = num2 - qhat * vn[n - 1];
    while (qhat >= (1ull << 32) || qhat * vn[n - 2] > ((rhat << 32) | u[j + n - 2])) {
      --qhat;
      rhat += vn[n - 1];
      if (rhat >= (1ull << 32)) break;
    }
    int64_t borrow = 0;   // multiply and subtract
    for (int i = 0; i < n; ++i) {
      const uint64_t prod = qhat * vn[i];
      const int64_t t = (int64_t)u[i + j] - borrow - (int64_t)(prod & 0xFFFFFFFFull);
      u[i + j] = (uint32_t)t;
      borrow = (int64_t)(prod >> 32) - (t >> 32);
    }
    const int64_t t = (int64_t)u[j + n] - borrow;
    u[j + n] = (uint32_t)t;
    if (t < 0) {   // qhat was one too large: add the divisor back
      --qhat;
      uint64_t carry = 0;
      for (int i = 0; i < n; ++i) {
        const uint64_t s2 = (uint64_t)u[i + j] + vn[i] + carry;
        u[i + j] = (uint32_t)s2;
        carry = s2 >> 32;
      }
      u[j + n] += (uint32_t)carry;
    }
    q[j] = (uint32_t)qhat;
  }
  bool rem = false;
  for (int i = 0; i < n; ++i) rem |= u[i] != 0;
  return rem;
}

// RN_p of (num / den) where num, den are exact magnitudes (bit 0 worth 2^lsb_n, 2^lsb_d).
// Q = floor(num 2^sh / den) has p + 3 or p + 4 bits; the remainder (and any
// numerator bits shifted out) gives a sticky bit appended below Q, so one RNE
// rounding of 2Q + sticky is the correct rounding of the quotient.
__device__ inline bool mp_div_round(const uint64_t *num, int nwn, int64_t lsb_n, bool neg, const uint64_t *den,
                                    int nwd, int64_t lsb_d, int p, int L, MPOut o) {
  WinAcc an{num}, ad{den};
  const int nN = bitlen(an, 2 * nwn), nD = bitlen(ad, 2 * nwd);
  if (nN == 0 || nD == 0) {   // 0 / d = 0 ; division by zero is the caller's to refuse
    store_zero(L, o.s, o.e, o.limb, o.stride);
    return true;
  }
  constexpr int kMaxU = 160, kMaxQ = 48;
  const int sh = (p + 3) - (nN - nD);     // num 2^sh has nD + p + 3 bits
  const int ubits = nN + sh;
  const int m = (ubits + 31) / 32, n = (nD + 31) / 32;
  if (m + 1 > kMaxU || n > 80 || m - n + 1 > kMaxQ) return false;
  uint32_t u[kMaxU], v[80], q[kMaxQ];
  for (int i = 0; i < m; ++i) {            // digits of num 2^sh (low bits dropped if sh < 0)
    const uint64_t w = bits64_at(an, 2 * nwn, 32 * i - sh);
    u[i] = (uint32_t)w;
  }
  if (ubits % 32) u[m - 1] &= (1u << (ubits % 32)) - 1u;
  for (int i = 0; i < n; ++i) v[i] = word_at(ad, i, 2 * nwd);
  bool sticky = (m >= n) ? divmod_digits(u, m, v, n, q) : true;
  if (sh < 0) sticky |= any_below(an, 2 * nwn, -sh);   // numerator bits below the shifted window
  const int ql = m - n + 1;
  // Q' = 2 Q + sticky as 64-bit limbs, value = Q' 2^(lsb_n - lsb_d - sh - 1)
  uint64_t Qs[kMaxQ / 2 + 2];
  const int qw = (ql + 1) / 2 + 1;
  for (int i = 0; i < qw; ++i) Qs[i] = 0;
  for (int i = 0; i < ql; ++i) Qs[i >> 1] |= (uint64_t)q[i] << (32 * (i & 1));
  uint64_t c = sticky ? 1ull : 0ull;
  for (int i = 0; i < qw; ++i) {
    const uint64_t nc = Qs[i] >> 63;
    Qs[i] = (Qs[i] << 1) | c;
    c = nc;
  }
  WinAcc aq{Qs};
  const int NQ = bitlen(aq, 2 * qw);
  return round_store(aq, 2 * qw, NQ, neg, lsb_n - lsb_d - (int64_t)sh - 1, p, L, o.s, o.e, o.limb, o.stride);
}

}  // namespace mpc
