// Shared device/host helpers of the mpcgemm CUDA library (sm_103a).
//
// * Ozaki parameters and the slice-pair group table (Alg. 2's triangle of
//   products, cut into int32-exact groups).
// * Certified round-to-nearest-even of an exact signed multi-word integer.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/mpcgemm.h"

namespace mpc {

// Ozaki digits of w bits (9, or 8 for k >= 2^15): balanced base-2^w, |d| <= 2^(w-1),
// |d_a d_b| <= 2^(2w-2); the fp32 tensor-core sum of a chunk of inner products stays an
// exact integer below 2^24 (w = 8: 960 elements, 960 2^14 < 2^24; w = 9: 256, <= 2^24).
__host__ __device__ constexpr int prod_log2(int w) { return 2 * w - 2; }
__host__ __device__ constexpr int chunk_kblocks(int w) { return w == 9 ? 4 : 15; }   // 64-element k-blocks
constexpr int kKBlock = 64;            // digit-plane row padding (one 128-byte bf16 row)
constexpr int kMaxSlices = 160;
constexpr int kMaxLimbs = 16;          // p <= 1024
// plain path: base-2^28 digits, D <= 40 at p <= 1024 (28 D - 2 >= p + 32, D a multiple of 4)
constexpr int kPlainDigitBits = 28;
constexpr int kMaxPlainDigits = 40;
// group planes of one Ozaki call (the accumulate kernel keeps their table in shared memory)
constexpr int kMaxGroupsTotal = 6000;
// 64-bit limbs of an exact plain-path sum of k <= 2^17 digit products
// (|sum| < k 2^(56 D - 1), plus the sign and the 3M combination)
__host__ __device__ constexpr int plain_limbs(int D) { return (56 * D + 18 + 63) / 64; }
constexpr int kStatusWords = 16;
constexpr int kDefaultGuard = 40;

// status block (int32 words at the start of the workspace); words 10..13 hold the
// per-part split's offsets as kZCap - z (A re, A im, B re, B im; maxima, so 0 = zero part)
enum StatusWord { kStErange = 0, kStFallbackCount = 1, kStFallbackOverflow = 2, kStUncertified = 3, kStTimeout = 4,
                  kStUnitCounter = 8, kStPartZ = 10 };   // word 8: the tcgen05 slice GEMM's unit counter
// per-part split: the offset of an all-zero part, and the cap of every offset
constexpr int kZCap = 2048;

// Digit sets of one operand: planes [0, s) real part, [s, 2s) imaginary part,
// [2s, 3s+1) the 3M sums (positions -1 .. s-1).
struct ProductDesc {
  int32_t a_plane0;   // first digit plane of A used by this product
  int32_t a_pos0;     // digit position of that plane (0, or -1 for sums)
  int32_t a_npos;     // number of digit positions
  int32_t b_plane0, b_pos0, b_npos;
  int32_t group0;     // first entry of this product in the group table
  int32_t n_groups;
};

struct GroupEntry {   // one group: pairs (t, q - t), t = t0 .. t0 + count - 1
  int32_t prod, q, t0, count;
};

// Levels q = t + u, t in [a0, a0+na), u in [b0, b0+nb), q <= Q, each cut into
// runs of at most gmax pairs, levels ascending, t ascending inside a level.
// Writes up to `cap` entries into `out` (may be null) and returns the count.
__host__ __device__ inline int build_groups(int prod, int a0, int na, int b0, int nb, int Q, int gmax,
                                            GroupEntry *out, int cap) {
  int n = 0;
  int a1 = a0 + na - 1, b1 = b0 + nb - 1;
  int qhi = (a1 + b1 < Q) ? a1 + b1 : Q;
  for (int q = a0 + b0; q <= qhi; ++q) {
    int lo = (a0 > q - b1) ? a0 : q - b1;
    int hi = (a1 < q - b0) ? a1 : q - b0;
    for (int t = lo; t <= hi; t += gmax) {
      int c = hi - t + 1;
      if (c > gmax) c = gmax;
      if (out && n < cap) out[n] = GroupEntry{prod, q, t, c};
      ++n;
    }
  }
  return n;
}

// ceil(v / 2^beta)
__host__ __device__ inline uint64_t ceil_shift(uint64_t v, int beta) {
  if (beta == 0) return v;
  if (beta >= 64) return v ? 1 : 0;
  return (v >> beta) + ((v & ((1ull << beta) - 1)) ? 1 : 0);
}

// Number of pairs of level q (t in [a0,a0+na), u in [b0,b0+nb)).
__host__ __device__ inline int level_pairs(int a0, int na, int b0, int nb, int q) {
  int a1 = a0 + na - 1, b1 = b0 + nb - 1;
  int lo = (a0 > q - b1) ? a0 : q - b1;
  int hi = (a1 < q - b0) ? a1 : q - b0;
  return hi >= lo ? hi - lo + 1 : 0;
}

// Device views of the caller's matrices (component zero iff its top limb is 0).
struct MatView {
  const uint8_t *sign[2];
  const int32_t *exp[2];
  const uint64_t *limb[2];
  int64_t rows, cols, ld, plane;   // plane = rows * ld
};

struct OutView {
  uint8_t *sign[2];
  int32_t *exp[2];
  uint64_t *limb[2];
  int64_t rows, cols, ld, plane;
};


#ifdef __CUDACC__

__device__ __forceinline__ void status_set(int32_t *status, int word, int32_t v) {
  atomicOr(reinterpret_cast<int *>(status) + word, v);
}

// ---------------------------------------------------------------------------
// Bit access on a little-endian array of 32-bit words given by an accessor
// (Acc::operator()(i) -> uint32_t for 0 <= i < nd; words outside are 0).
template <class Acc>
__device__ __forceinline__ uint32_t word_at(const Acc &a, int i, int nd) {
  return (i >= 0 && i < nd) ? a(i) : 0u;
}

template <class Acc>
__device__ __forceinline__ uint64_t bits64_at(const Acc &a, int nd, int pos) {
  // 64 bits starting at bit `pos` (pos may be negative: zeros below bit 0)
  int w = pos >= 0 ? (pos >> 5) : -((-pos + 31) >> 5);
  int r = pos - 32 * w;
  uint64_t lo = (uint64_t)word_at(a, w, nd) | ((uint64_t)word_at(a, w + 1, nd) << 32);
  if (r == 0) return lo;
  uint64_t hi = word_at(a, w + 2, nd);
  return (lo >> r) | (hi << (64 - r));
}

template <class Acc>
__device__ __forceinline__ int bit_at(const Acc &a, int nd, int pos) {
  if (pos < 0) return 0;
  return (int)((word_at(a, pos >> 5, nd) >> (pos & 31)) & 1u);
}

template <class Acc>
__device__ __forceinline__ bool any_below(const Acc &a, int nd, int pos) {
  // any bit set in [0, pos)
  if (pos <= 0) return false;
  int w = pos >> 5;
  for (int i = 0; i < w && i < nd; ++i)
    if (a(i)) return true;
  int r = pos & 31;
  if (r && w < nd && (a(w) & ((1u << r) - 1u))) return true;
  return false;
}

template <class Acc>
__device__ __forceinline__ bool any_in(const Acc &a, int nd, int lo, int hi) {
  // any bit set in [lo, hi)
  for (int pos = lo; pos < hi;) {
    int w = pos >> 5, r = pos & 31;
    int take = 32 - r;
    if (take > hi - pos) take = hi - pos;
    uint32_t mask = (take == 32) ? 0xFFFFFFFFu : (((1u << take) - 1u) << r);
    if (word_at(a, w, nd) & mask) return true;
    pos += take;
  }
  return false;
}

template <class Acc>
__device__ __forceinline__ bool all_ones(const Acc &a, int nd, int lo, int hi) {
  // every bit in [lo, hi) set
  for (int pos = lo; pos < hi;) {
    int w = pos >> 5, r = pos & 31;
    int take = 32 - r;
    if (take > hi - pos) take = hi - pos;
    uint32_t mask = (take == 32) ? 0xFFFFFFFFu : (((1u << take) - 1u) << r);
    if ((word_at(a, w, nd) & mask) != mask) return false;
    pos += take;
  }
  return true;
}

template <class Acc>
__device__ __forceinline__ int bitlen(const Acc &a, int nd) {
  for (int i = nd - 1; i >= 0; --i) {
    uint32_t v = a(i);
    if (v) return 32 * i + (32 - __clz(v));
  }
  return 0;
}

__device__ __forceinline__ int bitlen64(uint64_t v) { return v ? 64 - __clzll((long long)v) : 0; }

// True iff no midpoint of the p-bit grid lies within b * 2^beta of the
// magnitude |Acc| (bit length N): then RN_p(Acc) == RN_p(T) for every T with
// |T - Acc| <= b 2^beta.  b == 0 means Acc is exact.
template <class Acc>
__device__ bool certified(const Acc &mag, int nd, int N, int p, uint64_t b, int beta) {
  if (b == 0) return true;
  if (N <= p) return false;
  int sh = N - p;
  if (bitlen64(b) + beta > sh - 3) return false;
  int wlen = sh - 1 - beta;                       // window bits [beta, sh-1)
  uint64_t lo = bits64_at(mag, nd, beta);
  if (wlen < 64) lo &= (wlen == 0) ? 0ull : ((~0ull) >> (64 - wlen));
  if (bit_at(mag, nd, sh - 1)) {                  // r >= h: D = r - h
    if (wlen > 64 && any_in(mag, nd, beta + 64, sh - 1)) return true;
    if (lo > b) return true;
    if (lo == b && any_below(mag, nd, beta)) return true;
    return false;
  } else {                                        // r < h: D = h - r; need ~W >= b
    if (wlen > 64) {
      if (!all_ones(mag, nd, beta + 64, sh - 1)) return true;
      return (~lo) >= b;
    }
    uint64_t full = (wlen == 64) ? ~0ull : ((1ull << wlen) - 1ull);
    return (full - lo) >= b;
  }
}

// Round |Acc| (bit length N >= 1) to p bits, nearest-even, and write the
// normalised L-limb mantissa, sign and exponent (value = |Acc| 2^scale_exp).
// Returns false (and writes nothing) if the exponent leaves int32.
template <class Acc>
__device__ bool round_store(const Acc &mag, int nd, int N, bool neg, int64_t scale_exp, int p, int L,
                            uint8_t *sign_out, int32_t *exp_out, uint64_t *limb_out, int64_t limb_stride) {
  const int top = 64 * L;
  // M = |Acc| shifted so that bit N-1 lands on bit 64L-1, truncated to p bits
  uint64_t M[kMaxLimbs];
#pragma unroll
  for (int j = 0; j < kMaxLimbs; ++j)
    if (j < L) M[j] = bits64_at(mag, nd, 64 * j + N - top);
  int cut = top - p;                               // bits of M below `cut` are dropped
  bool rbit = false, sticky = false;
  if (N > p) {
    rbit = bit_at(mag, nd, N - p - 1);
    sticky = any_below(mag, nd, N - p - 1);
  }
#pragma unroll
  for (int j = 0; j < kMaxLimbs; ++j) {
    if (j >= L) break;
    int lo = 64 * j, hi = lo + 64;
    if (hi <= cut) M[j] = 0;
    else if (lo < cut) M[j] &= ~((1ull << (cut - lo)) - 1ull);
  }
  int lsb_word = cut >> 6, lsb_bit = cut & 63;
  bool odd = (M[lsb_word] >> lsb_bit) & 1ull;
  int64_t e = scale_exp + N;
  if (rbit && (sticky || odd)) {
    uint64_t carry = 1ull << lsb_bit;
#pragma unroll
    for (int j = 0; j < kMaxLimbs; ++j) {
      if (j < lsb_word || j >= L) continue;
      uint64_t s = M[j] + carry;
      carry = (s < carry) ? 1ull : 0ull;
      M[j] = s;
    }
    if (carry) {                                   // 2^(64L): renormalise
      M[L - 1] = 1ull << 63;
      e += 1;
    }
  }
  if (e > INT32_MAX || e < (int64_t)INT32_MIN + 1) return false;
  *sign_out = neg ? 1 : 0;
  *exp_out = (int32_t)e;
#pragma unroll
  for (int j = 0; j < kMaxLimbs; ++j)
    if (j < L) limb_out[(int64_t)j * limb_stride] = M[j];
  return true;
}

__device__ __forceinline__ void store_zero(int L, uint8_t *sign_out, int32_t *exp_out, uint64_t *limb_out,
                                           int64_t limb_stride) {
  *sign_out = 0;
  *exp_out = INT32_MIN;
  for (int j = 0; j < L; ++j) limb_out[(int64_t)j * limb_stride] = 0;
}

#endif  // __CUDACC__

// sign with which product `prod` enters component c
__host__ __device__ inline int product_sign(int method, int c, int prod) {
  if (method == MPC_4M) {
    if (c == 0) return prod == 0 ? 1 : (prod == 1 ? -1 : 0);
    return (prod == 2 || prod == 3) ? 1 : 0;
  }
  if (c == 0) return prod == 0 ? 1 : (prod == 1 ? -1 : 0);
  return prod == 2 ? 1 : -1;
}

}  // namespace mpc
