// mp_gemm_plain: Eq. (simple_triple_loop) with the 4M scalar product of
// Eq. (4m_way_base), on the CUDA cores.
//
// Both operands were converted once to fixed point (k_plain_fix): the row i
// of A as X_il = sign * floor(|a_il| 2^(64 Lp - E_i)), the column j of B
// likewise, Lp = L + 1 limbs, so that no product needs an alignment shift:
//     T_ij * 2^(128 Lp - E_i - F_j) = sum_l X_il Y_lj     (exact integers)
// when the conversion dropped no bit (the usual case; otherwise the dropped
// part is bounded and the rounding is certified or the entry falls back to
// the exact kernel).  One thread owns one component of one output element:
// a (2 Lp + 1)-limb two's-complement accumulator, schoolbook 64-bit limb
// products staged through shared memory, one rounding at the end.
#include "common.cuh"
#include "kernels.h"

namespace mpc {

namespace {

constexpr int kTI = 8, kTJ = 8, kKC = 4;   // 8 x 8 outputs x 2 components per 128-thread block

struct RegAcc {
  const uint64_t *base;
  __device__ __forceinline__ uint32_t operator()(int i) const {
    return (uint32_t)(base[i >> 1] >> (32 * (i & 1)));
  }
};

// acc +- x * y  (x, y: LP limbs in shared memory)
template <int LP>
__device__ __forceinline__ void mac(uint64_t (&acc)[2 * LP + 1], const uint64_t *x, const uint64_t *y, bool neg) {
  uint64_t P[2 * LP];
#pragma unroll
  for (int t = 0; t < 2 * LP; ++t) P[t] = 0;
#pragma unroll
  for (int i = 0; i < LP; ++i) {
    const uint64_t xi = x[i];
    uint64_t carry = 0;
#pragma unroll
    for (int j = 0; j < LP; ++j) {
      const uint64_t yj = y[j];
      const uint64_t lo = xi * yj;
      uint64_t hi = __umul64hi(xi, yj);
      uint64_t s = P[i + j] + lo;
      hi += (s < lo);
      s += carry;
      hi += (s < carry);
      P[i + j] = s;
      carry = hi;
    }
    P[i + LP] = carry;
  }
  // acc += neg ? (~P + 1) : P   over 2LP+1 limbs (branch-free)
  const uint64_t mask = neg ? ~0ull : 0ull;
  uint64_t c = neg ? 1ull : 0ull;
#pragma unroll
  for (int t = 0; t < 2 * LP; ++t) {
    const uint64_t v = P[t] ^ mask;
    uint64_t s = acc[t] + v;
    uint64_t c1 = s < v;
    s += c;
    c1 |= (s < c);
    acc[t] = s;
    c = c1;
  }
  acc[2 * LP] += mask + c;
}

}  // namespace

template <int LP>
__global__ void __launch_bounds__(128) k_plain_gemm(PlainArgs a, OutView C) {
  __shared__ uint64_t sA[kKC][kTI][2][LP];
  __shared__ uint64_t sB[kKC][kTJ][2][LP];
  __shared__ uint8_t sgA[kKC][kTI][2], sgB[kKC][kTJ][2];
  const int tid = threadIdx.x;
  const int c = tid >> 6, ti = (tid & 63) >> 3, tj = tid & 7;
  const int64_t i0 = (int64_t)blockIdx.y * kTI, j0 = (int64_t)blockIdx.x * kTJ;
  const int64_t i = i0 + ti, j = j0 + tj;
  const int64_t planeA = a.m * a.k, planeB = a.n * a.k;
  uint64_t acc[2 * LP + 1];
#pragma unroll
  for (int t = 0; t < 2 * LP + 1; ++t) acc[t] = 0;

  for (int64_t l0 = 0; l0 < a.k; l0 += kKC) {
    // cooperative load of the operand chunk (zeros beyond the edges)
    for (int x = tid; x < kKC * kTI * 2 * LP; x += 128) {
      const int limb = x % LP, cc = (x / LP) % 2, r = (x / (2 * LP)) % kTI, kk = x / (2 * LP * kTI);
      const int64_t gi = i0 + r, gl = l0 + kk;
      sA[kk][r][cc][limb] = (gi < a.m && gl < a.k) ? a.fixA[((int64_t)cc * a.Lp + limb) * planeA + gi * a.k + gl] : 0ull;
      const int64_t gj = j0 + r;
      sB[kk][r][cc][limb] = (gj < a.n && gl < a.k) ? a.fixB[((int64_t)cc * a.Lp + limb) * planeB + gj * a.k + gl] : 0ull;
    }
    for (int x = tid; x < kKC * kTI * 2; x += 128) {
      const int cc = x % 2, r = (x / 2) % kTI, kk = x / (2 * kTI);
      const int64_t gi = i0 + r, gj = j0 + r, gl = l0 + kk;
      sgA[kk][r][cc] = (gi < a.m && gl < a.k) ? a.sgnA[(int64_t)cc * planeA + gi * a.k + gl] : 0;
      sgB[kk][r][cc] = (gj < a.n && gl < a.k) ? a.sgnB[(int64_t)cc * planeB + gj * a.k + gl] : 0;
    }
    __syncthreads();
#pragma unroll 1
    for (int kk = 0; kk < kKC; ++kk) {
      // Re: +Xr Yr - Xi Yi ;  Im: +Xr Yi + Xi Yr
      const int b1 = c == 0 ? 0 : 1, b2 = c == 0 ? 1 : 0;
      mac<LP>(acc, sA[kk][ti][0], sB[kk][tj][b1], (sgA[kk][ti][0] ^ sgB[kk][tj][b1]) != 0);
      mac<LP>(acc, sA[kk][ti][1], sB[kk][tj][b2], ((sgA[kk][ti][1] ^ sgB[kk][tj][b2]) ^ (c == 0)) != 0);
    }
    __syncthreads();
  }
  if (i >= a.m || j >= a.n) return;
  const int64_t o = i * C.ld + j;
  const int32_t Ei = a.E[i], Fj = a.F[j];
  if (Ei == INT32_MIN || Fj == INT32_MIN) {
    store_zero(a.L, C.sign[c] + o, C.exp[c] + o, C.limb[c] + o, C.plane);
    return;
  }
  const bool neg = (acc[2 * LP] >> 63) != 0;
  if (neg) {
    uint64_t cc = 1;
#pragma unroll
    for (int t = 0; t < 2 * LP + 1; ++t) {
      const uint64_t v = ~acc[t] + cc;
      cc = (cc && v == 0) ? 1ull : 0ull;
      acc[t] = v;
    }
  }
  RegAcc mag{acc};
  const int nd = 2 * (2 * LP + 1);
  const int N = bitlen(mag, nd);
  // per component two products; each lossy operand contributes < 2^(64 Lp) per term
  const uint64_t b = 2ull * (uint64_t)a.k * (uint64_t)((a.lossyA[i] ? 1 : 0) + (a.lossyB[j] ? 1 : 0));
  const int beta = 64 * LP;
  if (N == 0 && b == 0) {
    store_zero(a.L, C.sign[c] + o, C.exp[c] + o, C.limb[c] + o, C.plane);
  } else if (N > 0 && certified(mag, nd, N, a.p, b, beta)) {
    const int64_t scale = (int64_t)Ei + (int64_t)Fj - 128 * (int64_t)LP;
    if (!round_store(mag, nd, N, neg, scale, a.p, a.L, C.sign[c] + o, C.exp[c] + o, C.limb[c] + o, C.plane)) {
      status_set(a.status, kStErange, 1);
      store_zero(a.L, C.sign[c] + o, C.exp[c] + o, C.limb[c] + o, C.plane);
    }
  } else {
    const int slot = atomicAdd(reinterpret_cast<int *>(a.status) + kStFallbackCount, 1);
    if (slot < a.fallback_cap) a.fallback[slot] = (i * a.n + j) * 2 + c;
    else status_set(a.status, kStFallbackOverflow, 1);
  }
}

template <int LP>
static void launch_plain_lp(const PlainArgs &a, const OutView &C, cudaStream_t st) {
  dim3 g((unsigned)((a.n + kTJ - 1) / kTJ), (unsigned)((a.m + kTI - 1) / kTI));
  k_plain_gemm<LP><<<g, 128, 0, st>>>(a, C);
}

void launch_plain_gemm(const PlainArgs &a, const OutView &C, cudaStream_t st) {
  switch (a.Lp) {
#define MPC_LP_CASE(v) \
  case v:              \
    launch_plain_lp<v>(a, C, st); break;
    MPC_LP_CASE(2) MPC_LP_CASE(3) MPC_LP_CASE(4) MPC_LP_CASE(5) MPC_LP_CASE(6) MPC_LP_CASE(7)
    MPC_LP_CASE(8) MPC_LP_CASE(9) MPC_LP_CASE(10) MPC_LP_CASE(11) MPC_LP_CASE(12) MPC_LP_CASE(13)
    MPC_LP_CASE(14) MPC_LP_CASE(15) MPC_LP_CASE(16) MPC_LP_CASE(17)
#undef MPC_LP_CASE
    default: break;
  }
}

}  // namespace mpc
