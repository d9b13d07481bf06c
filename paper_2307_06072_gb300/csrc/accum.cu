// oz_accum + cplx_assemble + rounding (Alg. 2's final L-bit accumulation and
// Eqs. (4m_way) / (3m_way)), and the exact fallback.
//
// k_oz_accum: one thread per output element (i, j).  The group sums of every
// real product are shifted by w (Q_c - q) and added, with the sign the complex
// formula gives them, into two exact accumulators (Re, Im; Q_c = Q unless the
// per-part split gives component c its own cut level):
//     4M: Re = rr - ii,        Im = ri + ir
//     3M: Re = rr - ii,        Im = ss - rr - ii
// Groups are visited in order of increasing shift; the groups of kAccLevels
// consecutive levels are summed in int64 (each scaled by its level's power of 2^w
// within the step), and each accumulator takes one such sum per step, keeping a
// running carry in registers and emitting finished 32-bit words.
// Value = Acc * 2^(E_i + F_j - (2w - 2) - w Q_c).
// The result is RN_p(Acc) when no rounding midpoint lies within the error
// bound b * 2^beta of Acc (then it equals RN_p of the exact product);
// otherwise the component is queued for k_exact_fallback.
//
// k_exact_fallback: one thread per queued component; the exact dot product
// of Eq. (simple_triple_loop) with Eq. (4m_way_base), in a fixed-point window
// wide enough for every product, then RN_p.
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace mpc {

namespace {

constexpr int kMaxWords = 88;   // 32-bit words of the exact accumulator (Q <= 2s, s <= 160)

// a block: kAccT consecutive elements of one row, one thread each
constexpr int kAccT = 256, kAccBatch = 16, kAccStages = 3;

// The exact accumulators' 32-bit words: a thread-local array (local memory, cached in
// L1; the kernel leaves most of L1 to it by staging only a batch of groups in shared
// memory).
struct AccWords {
  uint32_t *p;
  __device__ __forceinline__ uint32_t &operator[](int i) const { return p[i]; }
};

struct WordAcc {   // read access for the rounding helpers
  AccWords w;
  __device__ __forceinline__ uint32_t operator()(int i) const { return w[i]; }
};

struct LimbAcc {   // 32-bit words of a little-endian uint64 array
  const uint64_t *base;
  __device__ __forceinline__ uint32_t operator()(int i) const {
    return (uint32_t)(base[i >> 1] >> (32 * (i & 1)));
  }
};

// Exact signed integer built from one term per step, at shifts 0, W, 2W, ... with
// W = w kAccLevels <= 27 (a skipped step counts as a zero term): after each step the low
// W bits of the running signed carry are final, go to a bit buffer and leave the carry,
// so every shift is by a constant W.  A level has at most 3 x 160 int32 groups (< 2^40 in
// magnitude), a step three levels weighted 1, 2^w, 2^2w (< 2^59 for w <= 9), so
// |carry + h| < 2^60.
struct DigitAcc {
  int64_t c = 0;      // value not yet emitted, in units of 2^(bits emitted)
  uint64_t bb = 0;    // emitted bits not yet written to `out` (nb of them, nb < 32)
  int nb = 0, cur = 0, next = 0;   // next: shift of the next level
  __device__ __forceinline__ void step(const AccWords &out, int64_t h, int w) {
    c += h;
    bb |= (uint64_t)(c & ((1ll << w) - 1)) << nb;
    c >>= w;   // floor
    nb += w;
    next += w;
    if (nb >= 32) {
      out[cur++] = (uint32_t)bb;
      bb >>= 32;
      nb -= 32;
    }
  }
  __device__ __forceinline__ void add(const AccWords &out, int64_t h, int shift, int w) {
    while (next < shift) step(out, 0, w);
    step(out, h, w);
  }
  // emit the remaining words; returns the sign (magnitude left in out[0, nw))
  __device__ __forceinline__ bool finish(const AccWords &out, int nw) {
    if (cur < nw) {   // the buffered bits below the carry's bits (no carry between them)
      out[cur++] = (uint32_t)(bb | ((uint64_t)c << nb));
      c >>= (32 - nb);
    }
    while (cur < nw) {
      out[cur++] = (uint32_t)c;
      c >>= 32;
    }
    const bool neg = c < 0;
    if (neg) {
      uint64_t k = 1;
      for (int i = 0; i < nw; ++i) {
        const uint64_t t = (uint64_t)(uint32_t)~out[i] + k;
        out[i] = (uint32_t)t;
        k = t >> 32;
      }
    }
    return neg;
  }
};
}  // namespace

// acc + (int64) v * s in one instruction
__device__ __forceinline__ int64_t mad_wide(int32_t v, int32_t s, int64_t acc) {
  int64_t r;
  asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(r) : "r"(v), "r"(s), "l"(acc));
  return r;
}

// Round (or queue for the exact fallback) one component of one output element.
__device__ __forceinline__ void finish_component(const AccumArgs &a, const OutView &C, DigitAcc &acc,
                                                 const AccWords &words, int c, int64_t i, int64_t j, int32_t Ei,
                                                 int32_t Fj) {
  const int64_t o = i * C.ld + j;
  const bool neg = acc.finish(words, a.nslot);
  if (a.acc_dump) {   // the exact accumulator itself, for stage checks
    uint32_t *d = a.acc_dump + ((i * a.n + j) * 2 + c) * (int64_t)(a.nslot + 1);
    for (int x = 0; x < a.nslot; ++x) d[x] = words[x];
    d[a.nslot] = neg ? 1u : 0u;
  }
  WordAcc mag{words};
  const int N = bitlen(mag, a.nslot);
  const uint64_t b = a.bounds[c] + (uint64_t)a.k * ((a.lossyA[i] ? a.bounds[2 + c] : 0ull) +
                                                    (a.lossyB[j] ? a.bounds[4 + c] : 0ull));
  if (N == 0 && b == 0) {
    store_zero(a.L, C.sign[c] + o, C.exp[c] + o, C.limb[c] + o, C.plane);
  } else if (N > 0 && certified(mag, a.nslot, N, a.p, b, a.bound_shift)) {
    const int64_t Qc = (int64_t)a.bounds[8 + c];   // the component's cut level
    const int64_t scale = (int64_t)Ei + (int64_t)Fj - prod_log2(a.w) - (int64_t)a.w * Qc;
    if (!round_store(mag, a.nslot, N, neg, scale, a.p, a.L, C.sign[c] + o, C.exp[c] + o, C.limb[c] + o,
                     C.plane)) {
      status_set(a.status, kStErange, 1);
      store_zero(a.L, C.sign[c] + o, C.exp[c] + o, C.limb[c] + o, C.plane);
    }
  } else {
    const int slot = atomicAdd(reinterpret_cast<int *>(a.status) + kStFallbackCount, 1);
    if (slot < a.fallback_cap) a.fallback[slot] = (i * a.n + j) * 2 + c;
    else status_set(a.status, kStFallbackOverflow, 1);
  }
}

// One thread per output element (i, j); a block takes kAccT consecutive elements of
// one row.  The term table (plane, level shift, signs per group, in accumulation
// order, written by k_group_table; a multiplier is a sign times 2^(w (l % kAccLevels)))
// is copied into shared memory.  The group values are
// staged through shared memory kAccBatch groups at a time in a ring of kAccStages
// buffers filled by cp.async, so that the next batch is in flight while the block
// folds one.  Each warp copies contiguous runs of one group plane (16-byte copies when
// n is a multiple of 4).  The groups of one level are summed in plain int64
// (|sum| < 2^59) and folded into the exact accumulators once per kAccLevels levels.
constexpr size_t kAccStageBytes = (size_t)kAccStages * kAccBatch * kAccT * 4;

__device__ __forceinline__ void cp_async16(void *dst, const void *src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async4(void *dst, const void *src, int src_bytes) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

__global__ void __launch_bounds__(kAccT) k_oz_accum(AccumArgs a, OutView C) {
  extern __shared__ __align__(16) unsigned char acc_smem[];
  int32_t(*stage)[kAccBatch][kAccT] = reinterpret_cast<int32_t(*)[kAccBatch][kAccT]>(acc_smem);
  int4 *sterm = reinterpret_cast<int4 *>(acc_smem + kAccStageBytes);   // AccTerm as (plane, shift, s0, s1)
  const int tid = threadIdx.x;
  uint32_t wbuf[2][kMaxWords];
  const AccWords words[2] = {AccWords{wbuf[0]}, AccWords{wbuf[1]}};
  const int4 *terms = reinterpret_cast<const int4 *>(a.terms);
  for (int x = tid; x < a.n_entries; x += kAccT) sterm[x] = __ldg(&terms[x]);
  const int64_t i = blockIdx.y;
  const int64_t j0 = (int64_t)blockIdx.x * kAccT, j = j0 + tid;
  const int32_t Ei = a.E[i];
  if (Ei == INT32_MIN) {   // a zero row: the whole block's products are exactly 0 (block-uniform exit)
    if (j < a.n) {
      const int64_t o = i * C.ld + j;
      for (int c = 0; c < 2; ++c) store_zero(a.L, C.sign[c] + o, C.exp[c] + o, C.limb[c] + o, C.plane);
    }
    return;
  }
  const int32_t Fj = j < a.n ? a.F[j] : INT32_MIN;
  const bool active = j < a.n && Fj != INT32_MIN;
  const int64_t mn = a.m * a.n;
  const int32_t *row = a.planes + i * a.n + j0;
  const int nrun = (int)(a.n - j0 < kAccT ? a.n - j0 : kAccT);   // valid elements of this block's run
  const bool vec = (a.n & 3) == 0;
  const int nbatch = (a.n_entries + kAccBatch - 1) / kAccBatch;
  // 16-byte copies: this thread always copies the same 4 elements (c4) of the group rows
  // g0, g0 + 4, g0 + 8, ... of a batch, so their offset and valid count are fixed
  constexpr int kRowsPerPass = kAccT / (kAccT / 4);   // 4 group rows per pass of the block
  const int c4 = 4 * (tid % (kAccT / 4)), g0 = tid / (kAccT / 4);
  const int valid4 = nrun - c4 >= 4 ? 4 : (nrun > c4 ? nrun - c4 : 0);
  const int32_t *src4 = row + (valid4 ? c4 : 0);
  __syncthreads();   // the term table is in shared memory
  auto issue = [&](int bidx) {   // batch bidx into ring buffer bidx % kAccStages (an empty group if none)
    if (bidx < nbatch) {
      const int x0 = bidx * kAccBatch, buf = bidx % kAccStages;
      const int nb = a.n_entries - x0 < kAccBatch ? a.n_entries - x0 : kAccBatch;
      if (vec) {
#pragma unroll
        for (int g = g0; g < kAccBatch; g += kRowsPerPass) {
          if (g < nb) {
            const int plane = sterm[x0 + g].x;
            const bool take = plane >= 0;   // bytes beyond the copied ones are zero-filled
            cp_async16(&stage[buf][g][c4], src4 + (take ? (int64_t)plane * mn : 0), take ? 4 * valid4 : 0);
          }
        }
      } else {
        for (int q = tid; q < nb * kAccT; q += kAccT) {
          const int g = q / kAccT, c = q % kAccT;
          const int plane = sterm[x0 + g].x;
          const bool take = plane >= 0 && c < nrun;
          const int32_t *src = row + (take ? (int64_t)plane * mn + c : 0);
          cp_async4(&stage[buf][g][c], src, take ? 4 : 0);
        }
      }
    }
    cp_async_commit();   // always one group per batch slot: the wait counts stay uniform
  };
  DigitAcc acc[2];
  int64_t sum0 = 0, sum1 = 0;
#pragma unroll
  for (int b = 0; b < kAccStages - 1; ++b) issue(b);
  for (int bidx = 0; bidx < nbatch; ++bidx) {
    issue(bidx + kAccStages - 1);
    cp_async_wait<kAccStages - 1>();   // batch bidx has landed
    __syncthreads();
    if (active) {
      const int x0 = bidx * kAccBatch, buf = bidx % kAccStages;
      const int nb = a.n_entries - x0 < kAccBatch ? a.n_entries - x0 : kAccBatch;
#pragma unroll 4
      for (int u = 0; u < nb; ++u) {
        const int4 t = sterm[x0 + u];              // block-uniform (broadcast)
        const int32_t v = stage[buf][u][tid];
        sum0 = mad_wide(v, t.z, sum0);
        sum1 = mad_wide(v, t.w, sum1);
        if (t.y != -1) {   // a component's step ends here (most groups: neither, both shifts -1)
          const int sh0 = (int16_t)(t.y & 0xFFFF), sh1 = t.y >> 16;
          if (sh0 >= 0) {
            acc[0].add(words[0], sum0, sh0, a.w * kAccLevels);
            sum0 = 0;
          }
          if (sh1 >= 0) {
            acc[1].add(words[1], sum1, sh1, a.w * kAccLevels);
            sum1 = 0;
          }
        }
      }
    }
    __syncthreads();   // the buffer is free for the copy issued in the next iteration
  }
  if (j >= a.n) return;
  if (!active) {   // a zero column
    const int64_t o = i * C.ld + j;
    for (int c = 0; c < 2; ++c) store_zero(a.L, C.sign[c] + o, C.exp[c] + o, C.limb[c] + o, C.plane);
    return;
  }
  for (int c = 0; c < 2; ++c) finish_component(a, C, acc[c], words[c], c, i, j, Ei, Fj);
}

// ------------------------------------------------------------------ fallback

namespace {

// window (nw limbs, two's complement) += / -= (P << shift), P = 2L limbs; shift may be < 0
__device__ void window_add(uint64_t *win, int nw, const uint64_t *P, int np, int64_t shift, bool sub) {
  int64_t w0 = shift >= 0 ? (shift >> 6) : 0;
  int64_t wtop = (shift + 64 * (int64_t)np) / 64 + 1;   // last limb the operand can touch
  uint64_t carry = 0;
  for (int64_t w = w0; w < nw; ++w) {
    uint64_t v = 0;
    if (w <= wtop) {
      const int64_t b = 64 * w - shift;                  // operand bit at window bit 64w
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
      uint64_t d = win[w] - v;
      uint64_t b1 = win[w] < v;
      uint64_t d2 = d - carry;
      b1 |= (d < carry);
      win[w] = d2;
      carry = b1;
    }
  }
}

}  // namespace

__global__ void k_exact_fallback(FallbackArgs f, MatView A, MatView B, OutView C) {
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
  int64_t count = f.status[kStFallbackCount];
  if (count > f.cap) count = f.cap;
  uint64_t *win = f.scratch + tid * f.scratch_limbs;
  const int L = f.L;
  for (int64_t q = tid; q < count; q += nthreads) {
    const int64_t code = f.list[q];
    const int c = (int)(code & 1);
    const int64_t ij = code >> 1, i = ij / f.n, j = ij % f.n;
    // terms of Eq. (4m_way_base): (component of A, component of B, subtract)
    const int ta[2] = {0, 1}, tb[2] = {c == 0 ? 0 : 1, c == 0 ? 1 : 0};
    const bool tsub[2] = {false, c == 0};
    int64_t xmin = INT64_MAX, top = INT64_MIN;
    for (int64_t l = 0; l < f.k; ++l) {
      const int64_t ia = i * A.ld + l, ib = l * B.ld + j;
      for (int t = 0; t < 2; ++t) {
        if (!A.limb[ta[t]][(int64_t)(L - 1) * A.plane + ia] || !B.limb[tb[t]][(int64_t)(L - 1) * B.plane + ib])
          continue;
        const int64_t es = (int64_t)A.exp[ta[t]][ia] + (int64_t)B.exp[tb[t]][ib];
        xmin = min(xmin, es - 128 * (int64_t)L);
        top = max(top, es);
      }
    }
    const int64_t o = i * C.ld + j;
    if (top == INT64_MIN) {
      store_zero(L, C.sign[c] + o, C.exp[c] + o, C.limb[c] + o, C.plane);
      continue;
    }
    int growth = 2;
    while (((int64_t)1 << growth) < 4 * f.k) ++growth;
    int64_t width = top - xmin + growth + 2;
    int nw = (int)(width / 64 + 2);
    bool truncated = false;
    if (nw > f.scratch_limbs) {
      nw = f.scratch_limbs;
      xmin = top + growth + 2 - 64 * (int64_t)(nw - 1);
      truncated = true;
    }
    for (int w = 0; w < nw; ++w) win[w] = 0;
    uint64_t Ma[kMaxLimbs], Mb[kMaxLimbs], P[2 * kMaxLimbs];
    for (int64_t l = 0; l < f.k; ++l) {
      const int64_t ia = i * A.ld + l, ib = l * B.ld + j;
      for (int t = 0; t < 2; ++t) {
        if (!A.limb[ta[t]][(int64_t)(L - 1) * A.plane + ia] || !B.limb[tb[t]][(int64_t)(L - 1) * B.plane + ib])
          continue;
        for (int u = 0; u < L; ++u) {
          Ma[u] = A.limb[ta[t]][(int64_t)u * A.plane + ia];
          Mb[u] = B.limb[tb[t]][(int64_t)u * B.plane + ib];
        }
        for (int u = 0; u < 2 * L; ++u) P[u] = 0;
        for (int x = 0; x < L; ++x) {
          uint64_t carry = 0;
          for (int y = 0; y < L; ++y) {
            const uint64_t lo = Ma[x] * Mb[y];
            uint64_t hi = __umul64hi(Ma[x], Mb[y]);
            uint64_t s = P[x + y] + lo;
            hi += (s < lo);
            s += carry;
            hi += (s < carry);
            P[x + y] = s;
            carry = hi;
          }
          P[x + L] = carry;
        }
        const int64_t es = (int64_t)A.exp[ta[t]][ia] + (int64_t)B.exp[tb[t]][ib];
        const bool neg = (A.sign[ta[t]][ia] ^ B.sign[tb[t]][ib]) ^ (tsub[t] ? 1 : 0);
        window_add(win, nw, P, 2 * L, es - 128 * (int64_t)L - xmin, neg);
      }
    }
    const bool neg = (win[nw - 1] >> 63) != 0;
    if (neg) {
      uint64_t cc = 1;
      for (int w = 0; w < nw; ++w) {
        const uint64_t v = ~win[w] + cc;
        cc = (cc && v == 0) ? 1ull : 0ull;
        win[w] = v;
      }
    }
    LimbAcc mag{win};
    const int N = bitlen(mag, 2 * nw);
    // A truncated window dropped every term's bits below 2^xmin: |T - window| < (terms) 2^xmin
    // with at most 2k terms, so the rounding is still RN_p(T) when no midpoint lies that close.
    if (truncated && (N == 0 || !certified(mag, 2 * nw, N, f.p, (uint64_t)(2 * f.k), 0)))
      atomicAdd(reinterpret_cast<int *>(f.status) + kStUncertified, 1);
    if (N == 0) {
      store_zero(L, C.sign[c] + o, C.exp[c] + o, C.limb[c] + o, C.plane);
    } else if (!round_store(mag, 2 * nw, N, neg, xmin, f.p, L, C.sign[c] + o, C.exp[c] + o, C.limb[c] + o,
                            C.plane)) {
      status_set(f.status, kStErange, 1);
      store_zero(L, C.sign[c] + o, C.exp[c] + o, C.limb[c] + o, C.plane);
    }
  }
}

__global__ void k_zero_output(OutView C, int64_t m, int64_t n, int L) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m * n) return;
  const int64_t o = (t / n) * C.ld + (t % n);
  for (int c = 0; c < 2; ++c) store_zero(L, C.sign[c] + o, C.exp[c] + o, C.limb[c] + o, C.plane);
}

// ---------------------------------------------------------------- launchers

void launch_oz_accum(const AccumArgs &a, const OutView &C, cudaStream_t st) {
  const size_t smem = kAccStageBytes + (size_t)a.n_entries * sizeof(AccTerm);
  static std::once_flag once;   // allow the largest table any plan can have, once per process
  std::call_once(once, [] {
    cudaFuncSetAttribute(k_oz_accum, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)(kAccStageBytes + (size_t)kMaxGroupsTotal * sizeof(AccTerm)));
  });
  dim3 g((unsigned)((a.n + kAccT - 1) / kAccT), (unsigned)a.m);
  k_oz_accum<<<g, kAccT, smem, st>>>(a, C);
}

void launch_fallback(const FallbackArgs &f, const MatView &A, const MatView &B, const OutView &C, int blocks,
                     int threads, cudaStream_t st) {
  k_exact_fallback<<<blocks, threads, 0, st>>>(f, A, B, C);
}

void launch_zero_output(const OutView &C, int64_t m, int64_t n, int L, cudaStream_t st) {
  const int64_t tot = m * n;
  if (tot <= 0) return;
  k_zero_output<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(C, m, n, L);
}

}  // namespace mpc
