// mp_gemm_plain: Eq. (simple_triple_loop) on the CUDA cores, in the 4M form
// of Eq. (4m_way_base) or the 3M form of Eq. (3m_way_base).
//
// Both operands were converted once to fixed point (k_plain_digits): row i
// of A as X_il = sign * floor(|a_il| 2^(W - E_i)), column j of B likewise,
// each in D signed base-2^28 digits.  No product needs an alignment shift:
//     T_ij 2^(2W - E_i - F_j) = sum_l X_il Y_lj        (exact integers)
// whenever the conversion dropped no bit (the usual case; otherwise the
// dropped part is bounded and the rounding is certified, or the entry falls
// back to the exact kernel).
//
// k_plain_gemm: four threads own one output element of one real product
// (4M: rr, ii, ri, ir; 3M: rr, ii and ss = (X_re + X_im)(Y_re + Y_im)); each
// takes one half of the x digits times one half of the y digits and forms its
// share of sum_l X_il Y_lj by schoolbook digit products, each one
// mad.wide.s32 into a signed 64-bit column sum (column t collects the
// products of digits a + b = t).  Carries are settled every 16 k-steps (at
// most 16 D/2 products of magnitude <= 2^54 reach a column in between), the
// last column keeps the sign.  The four shares are added in shared memory and
// the exact sum is written as plain_limbs(D) two's-complement limbs.
//
// k_plain_combine: one thread per output component adds the exact product
// sums (4M: Re = rr - ii, Im = ri + ir; 3M: Re = rr - ii, Im = ss - rr - ii),
// certifies and rounds once to p bits.
#include "common.cuh"
#include "kernels.h"

namespace mpc {

namespace {

// 8 x 8 outputs per 256-thread block; each output's product is split over four
// threads (x-digit half, y-digit half), one warp-uniform part per warp.
constexpr int kTI = 8, kTJ = 8, kKC = 16;

__device__ __forceinline__ void mad_wide(int64_t &acc, int32_t x, int32_t y) {
  asm("mad.wide.s32 %0, %1, %2, %0;" : "+l"(acc) : "r"(x), "r"(y));
}

// Little-endian 32-bit view of a limb array in registers.
template <int N>
struct LimbView {
  const uint64_t *v;
  __device__ __forceinline__ uint32_t operator()(int i) const { return (uint32_t)(v[i >> 1] >> (32 * (i & 1))); }
};

template <int D>
struct PlainSmem {
  static constexpr int DPS = D + 4;          // padded digit stride (conflict-free 8-byte loads)
  static constexpr int NCS = 2 * D + 1;      // padded column stride of the combination buffer
  static constexpr int kTile = 2 * kKC * kTI * DPS * 4;
  static constexpr int kComb = kTI * kTJ * NCS * 8;
  static constexpr int kBytes = kTile > kComb ? kTile : kComb;
};

}  // namespace

template <int D>
__global__ void __launch_bounds__(256, 2) k_plain_gemm(PlainGemmArgs a) {
  static_assert(D % 4 == 0, "digit halves must be even");
  constexpr int H = D / 2, NCT = 2 * H, NC = 2 * D, NLP = plain_limbs(D);
  constexpr int DPS = PlainSmem<D>::DPS, NCS = PlainSmem<D>::NCS, V = D / 4;
  __shared__ __align__(16) unsigned char smem[PlainSmem<D>::kBytes];
  int32_t(*sX)[kTI][DPS] = reinterpret_cast<int32_t(*)[kTI][DPS]>(smem);
  int32_t(*sY)[kTJ][DPS] = reinterpret_cast<int32_t(*)[kTJ][DPS]>(smem + kKC * kTI * DPS * 4);
  int64_t(*buf)[NCS] = reinterpret_cast<int64_t(*)[NCS]>(smem);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int part = warp & 3, hx = part & 1, hy = part >> 1;
  const int e = (warp >> 2) * 32 + lane, ti = e / kTJ, tj = e % kTJ;
  const int prod = blockIdx.z;
  const int64_t i0 = (int64_t)blockIdx.x * kTI;
  const int32_t *gA = a.dA + (int64_t)a.planeA[prod] * a.m * a.k * D;
  const int32_t *gB = a.dB + (int64_t)a.planeB[prod] * a.n * a.k * D;
  const int64_t tiles_j = (a.n + kTJ - 1) / kTJ;
  for (int64_t tjb = blockIdx.y; tjb < tiles_j; tjb += gridDim.y) {
    const int64_t j0 = tjb * kTJ;
    // this thread's share: x digits [hx H, hx H + H) times y digits [hy H, hy H + H),
    // column t here is column (hx + hy) H + t of the product
    int64_t col[NCT];
#pragma unroll
    for (int t = 0; t < NCT; ++t) col[t] = 0;
    for (int64_t l0 = 0; l0 < a.k; l0 += kKC) {
      for (int x = tid; x < kKC * kTI * V; x += 256) {
        const int q = x % V, kk = (x / V) % kKC, r = x / (V * kKC);
        const int64_t gi = i0 + r, gl = l0 + kk;
        int4 v = make_int4(0, 0, 0, 0);
        if (gi < a.m && gl < a.k) v = reinterpret_cast<const int4 *>(gA + (gi * a.k + gl) * D)[q];
        reinterpret_cast<int4 *>(&sX[kk][r][0])[q] = v;
      }
      for (int x = tid; x < kKC * kTJ * V; x += 256) {
        const int q = x % V, kk = (x / V) % kKC, r = x / (V * kKC);
        const int64_t gj = j0 + r, gl = l0 + kk;
        int4 v = make_int4(0, 0, 0, 0);
        if (gj < a.n && gl < a.k) v = reinterpret_cast<const int4 *>(gB + (gj * a.k + gl) * D)[q];
        reinterpret_cast<int4 *>(&sY[kk][r][0])[q] = v;
      }
      __syncthreads();
#pragma unroll 1
      for (int kk = 0; kk < kKC; ++kk) {
        int32_t y[H];
        const int2 *py = reinterpret_cast<const int2 *>(&sY[kk][tj][hy * H]);
        const int2 *px = reinterpret_cast<const int2 *>(&sX[kk][ti][hx * H]);
#pragma unroll
        for (int q = 0; q < H / 2; ++q) {
          const int2 v = py[q];
          y[2 * q] = v.x;
          y[2 * q + 1] = v.y;
        }
#pragma unroll
        for (int q = 0; q < H / 2; ++q) {
          const int2 v = px[q];
#pragma unroll
          for (int b = 0; b < H; ++b) mad_wide(col[2 * q + b], v.x, y[b]);
#pragma unroll
          for (int b = 0; b < H; ++b) mad_wide(col[2 * q + 1 + b], v.y, y[b]);
        }
      }
      __syncthreads();
      // settle carries (at most kKC H products of magnitude <= 2^54 reached a column)
#pragma unroll
      for (int t = 0; t < NCT - 1; ++t) {
        const int64_t c = col[t] >> kPlainDigitBits;
        col[t] &= (1ll << kPlainDigitBits) - 1;
        col[t + 1] += c;
      }
    }
    // add the four shares of each output in shared memory, one share per phase
    for (int x = tid; x < kTI * kTJ * NCS; x += 256) (&buf[0][0])[x] = 0;
    __syncthreads();
    const int off = (hx + hy) * H;
#pragma unroll 1
    for (int ph = 0; ph < 4; ++ph) {
      if (part == ph) {
#pragma unroll
        for (int t = 0; t < NCT; ++t) buf[e][off + t] += col[t];
      }
      __syncthreads();
    }
    const int64_t i = i0 + ti, j = j0 + tj;
    if (part == 0 && i < a.m && j < a.n) {
      uint64_t limb[NLP];
#pragma unroll
      for (int w = 0; w < NLP; ++w) limb[w] = 0;
      int64_t carry = 0;
#pragma unroll
      for (int t = 0; t < NC - 1; ++t) {
        const int64_t v = buf[e][t] + carry;
        carry = v >> kPlainDigitBits;
        const uint64_t ch = (uint64_t)(v & ((1ll << kPlainDigitBits) - 1));
        const int pos = kPlainDigitBits * t, w = pos >> 6, sh = pos & 63;
        limb[w] |= ch << sh;
        if (sh > 64 - kPlainDigitBits && w + 1 < NLP) limb[w + 1] |= ch >> (64 - sh);
      }
      {   // the signed last column, sign-extended over the remaining limbs
        const int64_t top = buf[e][NC - 1] + carry;
        constexpr int pos = kPlainDigitBits * (NC - 1), w0 = pos >> 6, sh = pos & 63;
        const uint64_t ext = top < 0 ? ~0ull : 0ull;
        uint64_t cy = 0;
#pragma unroll
        for (int w = w0; w < NLP; ++w) {
          uint64_t v;
          if (w == w0) v = (uint64_t)top << sh;
          else if (w == w0 + 1) v = sh ? (uint64_t)(top >> (64 - sh)) : ext;
          else v = ext;
          uint64_t s = limb[w] + v;
          uint64_t c1 = s < v ? 1ull : 0ull;
          s += cy;
          c1 |= s < cy ? 1ull : 0ull;
          limb[w] = s;
          cy = c1;
        }
      }
      const int64_t mn = a.m * a.n;
      uint64_t *o = a.sums + (int64_t)prod * NLP * mn + i * a.n + j;
#pragma unroll
      for (int w = 0; w < NLP; ++w) o[(int64_t)w * mn] = limb[w];
    }
    __syncthreads();   // buf is reused as the tile buffer of the next output tile
  }
}

template <int D>
__global__ void __launch_bounds__(256) k_plain_combine(PlainCombineArgs a, OutView C) {
  constexpr int NLP = plain_limbs(D);
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t mn = a.m * a.n;
  if (e >= 2 * mn) return;
  const int c = (int)(e & 1);
  const int64_t ij = e >> 1, i = ij / a.n, j = ij - i * a.n;
  const int64_t o = i * C.ld + j;
  const int32_t Ei = a.E[i], Fj = a.F[j];
  if (Ei == INT32_MIN || Fj == INT32_MIN) {
    store_zero(a.L, C.sign[c] + o, C.exp[c] + o, C.limb[c] + o, C.plane);
    return;
  }
  // terms (product, negated): Re = rr - ii; Im = ri + ir (4M) or ss - rr - ii (3M)
  int prods[3], negs[3], nt;
  if (c == 0) {
    prods[0] = 0; negs[0] = 0; prods[1] = 1; negs[1] = 1; nt = 2;
  } else if (a.method == MPC_4M) {
    prods[0] = 2; negs[0] = 0; prods[1] = 3; negs[1] = 0; nt = 2;
  } else {
    prods[0] = 2; negs[0] = 0; prods[1] = 0; negs[1] = 1; prods[2] = 1; negs[2] = 1; nt = 3;
  }
  uint64_t acc[NLP];
#pragma unroll
  for (int w = 0; w < NLP; ++w) acc[w] = 0;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    if (x >= nt) break;
    const uint64_t *s = a.sums + (int64_t)prods[x] * NLP * mn + ij;
    const uint64_t mask = negs[x] ? ~0ull : 0ull;   // acc + (v ^ mask) + negs: two's-complement subtract
    uint64_t carry = negs[x] ? 1ull : 0ull;
#pragma unroll
    for (int w = 0; w < NLP; ++w) {
      const uint64_t v = s[(int64_t)w * mn] ^ mask;
      uint64_t t = acc[w] + v;
      uint64_t c1 = t < v ? 1ull : 0ull;
      t += carry;
      c1 |= t < carry ? 1ull : 0ull;
      acc[w] = t;
      carry = c1;
    }
  }
  const bool neg = (acc[NLP - 1] >> 63) != 0;
  if (neg) {
    uint64_t cc = 1;
#pragma unroll
    for (int w = 0; w < NLP; ++w) {
      const uint64_t v = ~acc[w] + cc;
      cc = (cc && v == 0) ? 1ull : 0ull;
      acc[w] = v;
    }
  }
  LimbView<NLP> mag{acc};
  const int nd = 2 * NLP;
  const int N = bitlen(mag, nd);
  const uint64_t b = a.coef[c] * (uint64_t)a.k * (uint64_t)((a.lossyA[i] ? 1 : 0) + (a.lossyB[j] ? 1 : 0));
  const int beta = a.W;
  if (N == 0 && b == 0) {
    store_zero(a.L, C.sign[c] + o, C.exp[c] + o, C.limb[c] + o, C.plane);
  } else if (N > 0 && certified(mag, nd, N, a.p, b, beta)) {
    const int64_t scale = (int64_t)Ei + (int64_t)Fj - 2 * (int64_t)a.W;
    if (!round_store(mag, nd, N, neg, scale, a.p, a.L, C.sign[c] + o, C.exp[c] + o, C.limb[c] + o, C.plane)) {
      status_set(a.status, kStErange, 1);
      store_zero(a.L, C.sign[c] + o, C.exp[c] + o, C.limb[c] + o, C.plane);
    }
  } else {
    const int slot = atomicAdd(reinterpret_cast<int *>(a.status) + kStFallbackCount, 1);
    if (slot < a.fallback_cap) a.fallback[slot] = ij * 2 + c;
    else status_set(a.status, kStFallbackOverflow, 1);
  }
}

// Instantiated digit counts (multiples of 4, so that the four shares of a
// product are equal); a precision uses the smallest one that holds p + 32 bits
// (28 D - 2 >= p + 32), D <= kMaxPlainDigits.
#define MPC_PLAIN_DS(X) X(4) X(8) X(12) X(16) X(20) X(24) X(28) X(32) X(36) X(40)

int plain_digits_for(int p) {
  const int need = (p + 32 + 2 + kPlainDigitBits - 1) / kPlainDigitBits;
#define MPC_PICK(d) if (need <= d) return d;
  MPC_PLAIN_DS(MPC_PICK)
#undef MPC_PICK
  return -1;
}

template <int D>
static void launch_plain_d(const PlainGemmArgs &a, cudaStream_t st) {
  const int64_t ti = (a.m + kTI - 1) / kTI, tj = (a.n + kTJ - 1) / kTJ;
  dim3 g((unsigned)ti, (unsigned)(tj < 65535 ? tj : 65535), (unsigned)a.n_products);
  k_plain_gemm<D><<<g, 256, 0, st>>>(a);
}

template <int D>
static void launch_combine_d(const PlainCombineArgs &a, const OutView &C, cudaStream_t st) {
  const int64_t tot = 2 * a.m * a.n;
  k_plain_combine<D><<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(a, C);
}

void launch_plain_gemm(const PlainGemmArgs &a, cudaStream_t st) {
  switch (a.D) {
#define MPC_CASE(d) \
  case d:           \
    launch_plain_d<d>(a, st); break;
    MPC_PLAIN_DS(MPC_CASE)
#undef MPC_CASE
    default: break;
  }
}

void launch_plain_combine(const PlainCombineArgs &a, const OutView &C, cudaStream_t st) {
  switch (a.D) {
#define MPC_CASE(d) \
  case d:           \
    launch_combine_d<d>(a, C, st); break;
    MPC_PLAIN_DS(MPC_CASE)
#undef MPC_CASE
    default: break;
  }
}

}  // namespace mpc
