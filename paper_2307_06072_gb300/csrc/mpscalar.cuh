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
//     from exact numerator and denominator by binary long division.
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

// compare magnitudes a, b (n limbs each): -1, 0, 1
__device__ __forceinline__ int limbs_cmp(const uint64_t *a, const uint64_t *b, int n) {
  for (int i = n - 1; i >= 0; --i)
    if (a[i] != b[i]) return a[i] < b[i] ? -1 : 1;
  return 0;
}

// RN_p of (num / den) where num, den are exact magnitudes (bit 0 worth 2^lsb_n, 2^lsb_d).
// Restoring binary long division yields >= p + 2 quotient bits; the remainder
// gives the sticky bit, appended below them, so one RNE rounding is exact.
__device__ inline bool mp_div_round(const uint64_t *num, int nwn, int64_t lsb_n, bool neg, const uint64_t *den,
                                    int nwd, int64_t lsb_d, int p, int L, MPOut o) {
  WinAcc an{num}, ad{den};
  const int nN = bitlen(an, 2 * nwn), nD = bitlen(ad, 2 * nwd);
  if (nN == 0 || nD == 0) {   // 0 / d = 0 ; division by zero is the caller's to refuse
    store_zero(L, o.s, o.e, o.limb, o.stride);
    return true;
  }
  // quotient Q = floor(num * 2^sh / den) with bit length p + 2 or p + 3
  const int sh = (p + 3) - (nN - nD);     // num * 2^sh has nD + p + 3 bits
  const int qbits = nN + sh;              // bits of num * 2^sh
  const int dl = (nD + 63) / 64 + 1;      // remainder limbs
  uint64_t R[kWinLimbs / 2 + 2], D[kWinLimbs / 2 + 2], Q[kMaxLimbs + 2];
  if (dl > kWinLimbs / 2 + 2) return false;
  for (int i = 0; i < dl; ++i) {
    R[i] = 0;
    D[i] = i < nwd ? den[i] : 0;
  }
  const int ql = (p + 3 + 63) / 64 + 1;
  for (int i = 0; i < ql; ++i) Q[i] = 0;
  // bits of num * 2^sh from the top: bit b of the shifted value = bit (b - sh) of num
  for (int b = qbits - 1; b >= 0; --b) {
    uint64_t carry = (uint64_t)bit_at(an, 2 * nwn, b - sh);   // shift the remainder left, bring in a bit
    for (int i = 0; i < dl; ++i) {
      const uint64_t nc = R[i] >> 63;
      R[i] = (R[i] << 1) | carry;
      carry = nc;
    }
    if (limbs_cmp(R, D, dl) >= 0) {
      uint64_t br = 0;
      for (int i = 0; i < dl; ++i) {
        const uint64_t d = R[i] - D[i];
        const uint64_t b1 = R[i] < D[i];
        const uint64_t d2 = d - br;
        br = b1 | (d < br);
        R[i] = d2;
      }
      if (b < 64 * ql) Q[b >> 6] |= 1ull << (b & 63);
    }
  }
  bool sticky = false;
  for (int i = 0; i < dl; ++i) sticky |= R[i] != 0;
  if (sh < 0) sticky |= any_below(an, 2 * nwn, -sh);   // numerator bits below the shifted window
  // Q' = 2 Q + sticky, value = Q' 2^(lsb_n - lsb_d - sh - 1)
  uint64_t Qs[kMaxLimbs + 3];
  uint64_t c = sticky ? 1ull : 0ull;
  for (int i = 0; i < ql; ++i) {
    Qs[i] = (Q[i] << 1) | c;
    c = Q[i] >> 63;
  }
  Qs[ql] = c;
  WinAcc aq{Qs};
  const int NQ = bitlen(aq, 2 * (ql + 1));
  return round_store(aq, 2 * (ql + 1), NQ, neg, lsb_n - lsb_d - (int64_t)sh - 1, p, L, o.s, o.e, o.limb, o.stride);
}

}  // namespace mpc
