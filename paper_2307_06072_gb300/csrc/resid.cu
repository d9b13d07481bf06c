// The residual split of Alg. 2 (Kouya, Sec. III-C) on the GPU: MPC_SPLIT_RESIDUAL, 4M.
//
// Alg. 2 cuts every real matrix line by line and measures, before EVERY slice, the
// largest magnitude mu left in the line; the slice is the residual rounded to nearest
// at a unit set by ceil(log2 mu), and it is subtracted from the residual exactly.  Here
// a slice is a w-bit balanced digit d = RNE(R / 2^b), b = ceil(log2 max |R|) - (w - 1),
// so |d| <= 2^(w-1) and the digit is exact in bf16; after the slice |R| <= 2^(b-1), so
// units fall by at least w per slice, by more when the line's residual collapses.
//
//  * k_transpose_planes: B is cut by columns, so its format planes are first copied
//    K-major (one line per column), and both operands go through one line kernel.
//  * k_resid_split: one CTA per line, both parts, slice after slice.  Every residual
//    is a function of the input and the previous unit alone (R_t = bal(a, b_(t-1)), the
//    balanced remainder), so no residual is stored: the digit of unit b after unit b' is
//    F + t_b - 2^(b'-b) t_b', F the bits of |a| in [b, b') and t_x the round-up flag of
//    RNE(|a| / 2^x); the line's next ceil(log2 max |R|) comes from the bits of |a| below
//    b (a block-wide maximum).  Writes the digit planes, the unit of every (part, slice,
//    line), the plane and value flags, the lossy flags (a nonzero remainder) and, per
//    slice, whether some line's unit is not exactly w below its previous one.
//  * k_resid_table: one table entry per kept pair (t, u), t + u <= Q, levels in order;
//    pairs with an all-zero plane are emptied.  The slice products of a level can share
//    one tensor-core sum only where their units agree in every line, so consecutive
//    pairs of a level are merged into one exact group (at most the int32 limit) where
//    neither of the slices that changes steps by more than w in any line (the split
//    flags such slices); the run's first entry carries the count, the others are empty.
//    On lines that never skip (random full-precision data) this is the default split's
//    grouping.  Also the call's error bounds.
//  * k_resid_accum: one thread per output entry; for a batch of pair planes it adds
//    every product at its own offset o = b^A_(i,t) + b^B_(j,u) - lo_c into the exact
//    accumulator of its component, whose window is anchored at the largest anchor sum
//    of the component's products (lo_c = M - w Q).  Consecutive pairs of one (product,
//    level) with equal offset are summed first; a sum below the window is floored and
//    counted in the bound.  The accumulators stay in the workspace between batches; the
//    last batch certifies and rounds (or queues the exact fallback).
#include <cuda_bf16.h>
#include <climits>

#include "common.cuh"
#include "kernels.h"

namespace mpc {

namespace {

constexpr long long kNone = LLONG_MIN;   // no unit: a zero slice or a zero part
constexpr int kSplitT = 256;
constexpr int kAccT = 256;
constexpr int kAccWords = 88;            // as the default accumulation: Q <= 2s, s <= 160

// The L-limb magnitude of one element (limb j at limb[j * stride]).
struct Mag {
  const uint64_t *limb;
  int64_t stride;
  int L;
  __device__ __forceinline__ uint64_t at(int64_t q) const { return (q >= 0 && q < L) ? limb[q * stride] : 0ull; }
  // 64 bits starting at bit index r (any r; zeros outside [0, 64L))
  __device__ __forceinline__ uint64_t bits64(int64_t r) const {
    const int64_t q = r >> 6;   // floor division
    const int off = (int)(r & 63);
    const uint64_t lo = at(q), hi = at(q + 1);
    return off ? ((lo >> off) | (hi << (64 - off))) : lo;
  }
};

struct ElemInfo {
  bool nz;
  bool neg;
  int64_t x;     // absolute exponent of mantissa bit 0
  int64_t tz;    // index of the lowest set bit
  int64_t top;   // index of the highest set bit
};

__device__ __forceinline__ ElemInfo elem_info(const Mag &M, const uint8_t *sign, const int32_t *exp, int64_t idx) {
  ElemInfo e{};
  const uint64_t t = M.at(M.L - 1);
  e.nz = t != 0;
  if (!e.nz) return e;
  e.neg = sign[idx] != 0;
  e.x = (int64_t)exp[idx] - 64 * (int64_t)M.L;
  e.top = 64 * (int64_t)(M.L - 1) + 63 - __clzll((long long)t);
  for (int q = 0; q < M.L; ++q) {
    const uint64_t v = M.at(q);
    if (v) {
      e.tz = 64 * (int64_t)q + __ffsll((long long)v) - 1;
      break;
    }
  }
  return e;
}

// RNE(|a| / 2^b) - floor(|a| / 2^b) for the unit index rb = b - x
__device__ __forceinline__ int round_up_flag(const Mag &M, const ElemInfo &e, int64_t rb) {
  const uint64_t win = M.bits64(rb - 1);   // bit 0: index rb - 1, bit 1: index rb
  const int g = (int)(win & 1ull), par = (int)((win >> 1) & 1ull);
  const bool sticky = e.tz < rb - 1;
  return g && (sticky || par) ? 1 : 0;
}

// ceil(log2 |bal(a, b)|) as an absolute exponent, kNone if the balanced remainder is 0
__device__ __forceinline__ long long next_exponent(const Mag &M, const ElemInfo &e, int64_t rb, int tb) {
  if (!tb) {   // V = |a| mod 2^b: its highest set bit h (>= tz); a power of two iff h == tz
    int64_t r = rb - 1;
    if (r > e.top) r = e.top;
    while (r >= e.tz) {
      const uint64_t win = M.bits64(r - 63);   // bit 63: index r
      if (win) {
        const int64_t h = r - __clzll((long long)win);
        return (long long)(e.x + (h == e.tz ? h : h + 1));
      }
      r -= 64;
    }
    return kNone;
  }
  // V = 2^b - (|a| mod 2^b), |a| mod 2^b >= 2^(b-1): the highest zero bit above tz, + 1
  int64_t r = rb - 1;
  while (r > e.tz) {
    uint64_t m = ~M.bits64(r - 63);
    const int64_t jlim = e.tz - (r - 63);        // window bits j <= jlim are at or below tz
    if (jlim >= 63) m = 0;
    else if (jlim >= 0) m &= ~0ull << (jlim + 1);
    if (m) return (long long)(e.x + (r - __clzll((long long)m)) + 1);
    r -= 64;
  }
  return (long long)(e.x + e.tz);
}

__device__ __forceinline__ long long block_max(long long v, long long *red) {
  for (int o = 16; o > 0; o >>= 1) {
    const long long u = __shfl_xor_sync(0xffffffffu, v, o);
    v = u > v ? u : v;
  }
  const int w = threadIdx.x >> 5;
  __syncthreads();   // red is reused
  if ((threadIdx.x & 31) == 0) red[w] = v;
  __syncthreads();
  long long r = kNone;
  for (int x = 0; x < (int)(blockDim.x >> 5); ++x) r = red[x] > r ? red[x] : r;
  return r;
}

}  // namespace

template <int W>
__global__ void __launch_bounds__(kSplitT) k_resid_split(MatView X, int64_t lines, int64_t k, int64_t kpad, int L,
                                                         int s, __nv_bfloat16 *digits, int32_t *units, int32_t *lossy,
                                                         int32_t *flags, int32_t *irregular, int32_t *status) {
  __shared__ long long red[kSplitT / 32];
  const int64_t line = blockIdx.x;
  const int tid = threadIdx.x;
  constexpr int W2 = W + 2;
  bool lossy_line = false;
  for (int part = 0; part < 2; ++part) {
    const uint8_t *sg = X.sign[part];
    const int32_t *ex = X.exp[part];
    // c_0 = ceil(log2 max |a|) over the line
    long long c = kNone;
    for (int64_t l = tid; l < k; l += kSplitT) {
      const int64_t idx = line * X.ld + l;
      const Mag M{X.limb[part] + idx, X.plane, L};
      const ElemInfo e = elem_info(M, sg, ex, idx);
      if (!e.nz) continue;
      const long long ce = (long long)(e.x + (e.top == e.tz ? e.top : e.top + 1));
      c = ce > c ? ce : c;
    }
    c = block_max(c, red);
    if (c != kNone && tid == 0) flags[2 * s + part] = 1;   // the part has a nonzero value
    long long bp = kNone;
    for (int t = 0; t < s; ++t) {
      const int plane = part * s + t;
      __nv_bfloat16 *drow = digits + ((int64_t)plane * lines + line) * kpad;
      if (c == kNone) {   // the residual is zero: this and every later slice are zero
        for (int64_t l = tid; l < kpad; l += kSplitT) drow[l] = __float2bfloat16(0.0f);
        if (tid == 0) units[(int64_t)plane * lines + line] = INT32_MIN;
        continue;
      }
      const long long b = c - (W - 1);
      long long emax = kNone;
      bool nz = false;
      for (int64_t l = tid; l < kpad; l += kSplitT) {
        int d = 0;
        if (l < k) {
          const int64_t idx = line * X.ld + l;
          const Mag M{X.limb[part] + idx, X.plane, L};
          const ElemInfo e = elem_info(M, sg, ex, idx);
          if (e.nz) {
            const int64_t rb = b - e.x;
            const int tb = round_up_flag(M, e, rb);
            int64_t v = (int64_t)((M.bits64(rb) & ((1ull << W2) - 1ull))) + tb;
            if (bp != kNone) {
              const long long gap = bp - b;   // >= W
              if (gap < W2) {                   // F has only `gap` bits; subtract the carry of the unit above
                v = (int64_t)(M.bits64(rb) & ((1ull << gap) - 1ull)) + tb;
                v -= (int64_t)round_up_flag(M, e, bp - e.x) << gap;
              }
            }
            // |d| <= 2^(W-1): reduce modulo 2^(W+2) into [-2^(W+1), 2^(W+1))
            d = (int)(((v + (1ll << (W + 1))) & ((1ll << W2) - 1)) - (1ll << (W + 1)));
            if (e.neg) d = -d;
            const long long en = next_exponent(M, e, rb, tb);
            emax = en > emax ? en : emax;
          }
        }
        drow[l] = __int2bfloat16_rn(d);   // exact: |d| <= 256
        nz |= d != 0;
      }
      if (__syncthreads_or(nz) && tid == 0) flags[plane] = 1;
      emax = block_max(emax, red);
      if (tid == 0) {
        if (b < (long long)INT32_MIN + 1 || b > (long long)INT32_MAX) status_set(status, kStErange, 1);
        units[(int64_t)plane * lines + line] = (int32_t)b;
        if (bp != kNone && b != bp - W) irregular[plane] = 1;   // this line skipped grid positions here
      }
      bp = b;
      c = emax;
    }
    if (c != kNone) lossy_line = true;   // a nonzero remainder after the last slice
  }
  if (tid == 0 && lossy_line) lossy[line] = 1;
}

// Transpose planes of a k x n matrix (ld ldi) into n x k (ld k): out[z][j k + l] = in[z][l ldi + j].
template <typename T>
__global__ void k_transpose_planes(const T *in, int64_t in_plane, int64_t ldi, T *out, int64_t out_plane, int64_t k,
                                   int64_t n, int per_comp, const T *in2, T *out2) {
  __shared__ T tile[32][33];
  const int z = blockIdx.z;
  const T *src = (z < per_comp ? in : in2) + (int64_t)(z % per_comp) * in_plane;
  T *dst = (z < per_comp ? out : out2) + (int64_t)(z % per_comp) * out_plane;
  const int64_t j0 = (int64_t)blockIdx.x * 32, l0 = (int64_t)blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t l = l0 + r, j = j0 + threadIdx.x;
    if (l < k && j < n) tile[r][threadIdx.x] = src[l * ldi + j];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int64_t j = j0 + r, l = l0 + threadIdx.x;
    if (l < k && j < n) dst[j * k + l] = tile[threadIdx.x][r];
  }
}

namespace {

// 4M: product x = rr, ii, ri, ir; parts of its operands, its component and sign
__host__ __device__ __forceinline__ int part_a(int x) { return (x == 0 || x == 2) ? 0 : 1; }
__host__ __device__ __forceinline__ int part_b(int x) { return (x == 0 || x == 3) ? 0 : 1; }
__host__ __device__ __forceinline__ int comp_of(int x) { return x < 2 ? 0 : 1; }

__device__ __forceinline__ bool comp_vanishes(const int32_t *vA, const int32_t *vB, int c) {
  return c == 0 ? ((!vA[0] || !vB[0]) && (!vA[1] || !vB[1])) : ((!vA[0] || !vB[1]) && (!vA[1] || !vB[0]));
}

}  // namespace

__global__ void __launch_bounds__(128) k_resid_table(ResidTableArgs a) {
  __shared__ uint64_t s_bd[4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int32_t *vA = a.flagsA + a.planes_A, *vB = a.flagsB + a.planes_B;   // [re, im] values nonzero
  if (warp < 4) {
    const ProductDesc pd = a.prod[warp];
    if (lane == 0) build_groups(warp, 0, a.s, 0, a.s, a.Q, 1, a.table + pd.group0, pd.n_groups);
    __syncwarp();
    const bool needed = !comp_vanishes(vA, vB, comp_of(warp));
    auto live = [&](int t, int u) {
      return needed && a.flagsA[pd.a_plane0 + t] != 0 && a.flagsB[pd.b_plane0 + u] != 0;
    };
    for (int e = pd.group0 + lane; e < pd.group0 + pd.n_groups; e += 32) {
      GroupEntry g = a.table[e];
      if (!live(g.t0, g.q - g.t0)) g.count = 0;
      a.table[e] = g;
    }
    __syncwarp();
    // merge: within a level, pair (t + 1, u - 1) joins the run of (t, u) when both are live and
    // their offsets agree at every entry, i.e. slice t + 1 of A and slice u of B each sit exactly
    // w below the slice before it in every line (no irregular step); a run holds at most gmax
    // pairs (an exact int32 sum).  The run's first entry takes the count, the others become empty.
    const int32_t *irrA = a.irregularA + pd.a_plane0, *irrB = a.irregularB + pd.b_plane0;
    const int qhi = a.Q < 2 * a.s - 2 ? a.Q : 2 * a.s - 2;
    for (int q = lane; q <= qhi; q += 32) {
      int e0 = pd.group0;
      for (int x = 0; x < q; ++x) e0 += level_pairs(0, a.s, 0, a.s, x);
      const int cnt = level_pairs(0, a.s, 0, a.s, q);
      int head = -1;
      for (int e = e0; e < e0 + cnt; ++e) {
        GroupEntry g = a.table[e];
        if (g.count == 0) {
          head = -1;
          continue;
        }
        if (head >= 0) {
          GroupEntry h = a.table[head];
          const int u_prev = g.q - g.t0 + 1;   // the B slice of the pair before this one
          if (h.count < a.gmax && !irrA[g.t0] && !irrB[u_prev]) {
            ++h.count;
            a.table[head] = h;
            g.count = 0;
            a.table[e] = g;
            continue;
          }
        }
        head = e;
      }
    }
    // live dropped pairs per level above the cut
    uint64_t n1 = 0, nmax = 0;
    for (int q = a.Q + 1; q <= 2 * a.s - 2; ++q) {
      const int lo = q - (a.s - 1) > 0 ? q - (a.s - 1) : 0;
      const int hi = q < a.s - 1 ? q : a.s - 1;
      unsigned cnt = 0;
      for (int t = lo + lane; t <= hi; t += 32) cnt += live(t, q - t) ? 1u : 0u;
      cnt = __reduce_add_sync(0xffffffffu, cnt);
      if (q == a.Q + 1) n1 = cnt;
      else if (cnt > nmax) nmax = cnt;
    }
    if (lane == 0) s_bd[warp] = (uint64_t)a.k * (((uint64_t)1 << (a.w - 2)) * n1 + (nmax + 2) / 3);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int c = 0; c < 2; ++c) {
      uint64_t bd = 0, la = 0;
      for (int x = 0; x < 4; ++x) {
        if (comp_of(x) != c) continue;
        bd += ceil_shift(s_bd[x], a.beta);
        if (vA[part_a(x)] && vB[part_b(x)]) ++la;
      }
      const bool zero = comp_vanishes(vA, vB, c);
      a.bounds[c] = zero ? 0 : bd;
      a.bounds[2 + c] = zero ? 0 : la;
      a.bounds[4 + c] = zero ? 0 : la;
      a.bounds[6 + c] = zero ? 1 : 0;
      a.bounds[8 + c] = (uint64_t)(int64_t)a.Q;
    }
  }
}

namespace {

// words[0, nw) += v 2^off (two's complement, off >= 0; the sum fits nw words)
__device__ __forceinline__ void add_at(uint32_t *words, int nw, int64_t v, int64_t off) {
  const int q = (int)(off >> 5), r = (int)(off & 31);
  const uint64_t lo = (uint64_t)v << r;
  const uint32_t ext = v < 0 ? 0xFFFFFFFFu : 0u;
  const uint32_t part[3] = {(uint32_t)lo, (uint32_t)(lo >> 32), r ? (uint32_t)(v >> (64 - r)) : ext};
  uint64_t cy = 0;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    if (q + x >= nw) return;
    const uint64_t s = (uint64_t)words[q + x] + part[x] + cy;
    words[q + x] = (uint32_t)s;
    cy = s >> 32;
  }
  for (int x = q + 3; x < nw; ++x) {
    if ((cy == 0 && ext == 0) || (cy == 1 && ext == 0xFFFFFFFFu)) return;
    const uint64_t s = (uint64_t)words[x] + ext + cy;
    words[x] = (uint32_t)s;
    cy = s >> 32;
  }
}

struct AccWordsR {
  const uint32_t *p;
  __device__ __forceinline__ uint32_t operator()(int i) const { return p[i]; }
};

}  // namespace

__global__ void __launch_bounds__(kAccT) k_resid_accum(ResidAccumArgs a, OutView C) {
  __shared__ GroupEntry sg[64];
  const int tid = threadIdx.x;
  const int64_t i = blockIdx.y;
  const int64_t j = (int64_t)blockIdx.x * kAccT + tid;
  const bool in = j < a.n;
  const int64_t mn = a.m * a.n, e_ij = i * a.n + (in ? j : 0);
  // the windows: lo_c = max over the component's products of b^A_(i,0) + b^B_(j,0), minus w Q
  long long lo[2] = {kNone, kNone};
  if (in) {
    for (int x = 0; x < 4; ++x) {
      const int32_t ua = a.uA[(int64_t)part_a(x) * a.s * a.m + i];
      const int32_t ub = a.uB[(int64_t)part_b(x) * a.s * a.n + j];
      if (ua == INT32_MIN || ub == INT32_MIN) continue;
      const long long v = (long long)ua + ub;
      const int c = comp_of(x);
      lo[c] = (lo[c] == kNone || v > lo[c]) ? v : lo[c];
    }
    for (int c = 0; c < 2; ++c)
      if (lo[c] != kNone) lo[c] -= (long long)a.w * a.Q;
  }
  uint32_t wb[2][kAccWords];
  uint32_t trunc[2] = {0, 0};
  for (int c = 0; c < 2; ++c) {
    for (int x = 0; x < a.nslot; ++x) wb[c][x] = (!a.first && in) ? a.acc[((int64_t)c * a.nslot + x) * mn + e_ij] : 0u;
    if (!a.first && in) trunc[c] = a.trunc[(int64_t)c * mn + e_ij];
  }
  int64_t run_sum[2] = {0, 0};
  long long run_off[2] = {kNone, kNone};
  int run_key[2] = {-1, -1};
  auto flush = [&](int c) {
    if (run_off[c] == kNone) return;
    const int64_t v = run_sum[c];
    const long long off = run_off[c];
    if (v != 0) {
      if (off >= 0) {
        add_at(wb[c], a.nslot, v, off);
      } else {
        const long long sh = -off;
        const int64_t f = sh >= 63 ? (v < 0 ? -1 : 0) : (v >> sh);
        const bool dropped = sh >= 63 ? true : ((f << sh) != v);
        if (dropped) ++trunc[c];
        if (f) add_at(wb[c], a.nslot, f, 0);
      }
    }
    run_sum[c] = 0;
    run_off[c] = kNone;
  };
  for (int e0 = 0; e0 < a.n_entries; e0 += 64) {
    const int ne = a.n_entries - e0 < 64 ? a.n_entries - e0 : 64;
    __syncthreads();
    if (tid < ne) sg[tid] = a.table[e0 + tid];
    __syncthreads();
    if (!in) continue;
    for (int u0 = 0; u0 < ne; u0 += 8) {
      int32_t G[8];
#pragma unroll
      for (int x = 0; x < 8; ++x)   // the next 8 entries' values in flight together
        G[x] = (u0 + x < ne && sg[u0 + x].count) ? a.planes[(int64_t)(e0 + u0 + x) * mn + e_ij] : 0;
#pragma unroll
      for (int x = 0; x < 8; ++x) {
        if (u0 + x >= ne) break;
        const GroupEntry g = sg[u0 + x];
        if (!g.count) continue;
        const int pr = g.prod, c = comp_of(pr);
        if (lo[c] == kNone) continue;
        // the group's offset from its first A slice and its last (lowest) B slice: a line's
        // nonzero slices are a prefix, so if either is zero here every pair of the group is
        const int t = g.t0, ulast = g.q - g.t0 - (g.count - 1);
        const int32_t ua = a.uA[((int64_t)part_a(pr) * a.s + t) * a.m + i];
        const int32_t ub = a.uB[((int64_t)part_b(pr) * a.s + ulast) * a.n + j];
        if (ua == INT32_MIN || ub == INT32_MIN) continue;
        const long long off = (long long)ua + ub - (long long)a.w * (g.count - 1) - lo[c];
        const int key = pr * 1024 + g.q;
        if (key != run_key[c] || off != run_off[c]) {
          flush(c);
          run_key[c] = key;
          run_off[c] = off;
        }
        run_sum[c] += pr == 1 ? -(int64_t)G[x] : (int64_t)G[x];
      }
    }
  }
  if (!in) return;
  flush(0);
  flush(1);
  if (!a.last) {
    for (int c = 0; c < 2; ++c) {
      for (int x = 0; x < a.nslot; ++x) a.acc[((int64_t)c * a.nslot + x) * mn + e_ij] = wb[c][x];
      a.trunc[(int64_t)c * mn + e_ij] = trunc[c];
    }
    return;
  }
  const int64_t o = i * C.ld + j;
  for (int c = 0; c < 2; ++c) {
    uint32_t *w = wb[c];
    const bool neg = (w[a.nslot - 1] >> 31) != 0;
    if (neg) {   // magnitude
      uint64_t cy = 1;
      for (int x = 0; x < a.nslot; ++x) {
        const uint64_t v = (uint64_t)(uint32_t)~w[x] + cy;
        w[x] = (uint32_t)v;
        cy = v >> 32;
      }
    }
    if (a.acc_dump) {
      uint32_t *d = a.acc_dump + ((i * a.n + j) * 2 + c) * (int64_t)(a.nslot + 1);
      for (int x = 0; x < a.nslot; ++x) d[x] = w[x];
      d[a.nslot] = neg ? 1u : 0u;
    }
    if (lo[c] == kNone) {   // every product of this component vanishes here
      store_zero(a.L, C.sign[c] + o, C.exp[c] + o, C.limb[c] + o, C.plane);
      continue;
    }
    const AccWordsR mag{w};
    const int N = bitlen(mag, a.nslot);
    const uint64_t b = a.bounds[c] + (uint64_t)a.k * ((a.lossyA[i] ? a.bounds[2 + c] : 0ull) +
                                                      (a.lossyB[j] ? a.bounds[4 + c] : 0ull)) +
                       ceil_shift(trunc[c], a.beta);
    if (N == 0 && b == 0) {
      store_zero(a.L, C.sign[c] + o, C.exp[c] + o, C.limb[c] + o, C.plane);
    } else if (N > 0 && certified(mag, a.nslot, N, a.p, b, a.beta)) {
      if (!round_store(mag, a.nslot, N, neg, (int64_t)lo[c], a.p, a.L, C.sign[c] + o, C.exp[c] + o,
                       C.limb[c] + o, C.plane)) {
        status_set(a.status, kStErange, 1);
        store_zero(a.L, C.sign[c] + o, C.exp[c] + o, C.limb[c] + o, C.plane);
      }
    } else {
      const int slot = atomicAdd(reinterpret_cast<int *>(a.status) + kStFallbackCount, 1);
      if (slot < a.fallback_cap) a.fallback[slot] = (i * a.n + j) * 2 + c;
      else status_set(a.status, kStFallbackOverflow, 1);
    }
  }
}

// ---------------------------------------------------------------- launchers

void launch_transpose_operand(const MatView &B, int64_t k, int64_t n, int L, uint8_t *sign, int32_t *exp,
                              uint64_t *limb, cudaStream_t st) {
  const int64_t nk = n * k;
  const dim3 blk(32, 8);
  const unsigned gx = (unsigned)((n + 31) / 32), gy = (unsigned)((k + 31) / 32);
  k_transpose_planes<uint8_t><<<dim3(gx, gy, 2), blk, 0, st>>>(B.sign[0], 0, B.ld, sign, 0, k, n, 1, B.sign[1],
                                                                 sign + nk);
  k_transpose_planes<int32_t><<<dim3(gx, gy, 2), blk, 0, st>>>(B.exp[0], 0, B.ld, exp, 0, k, n, 1, B.exp[1],
                                                                 exp + nk);
  k_transpose_planes<uint64_t><<<dim3(gx, gy, 2 * L), blk, 0, st>>>(B.limb[0], B.plane, B.ld, limb, nk, k, n, L,
                                                                      B.limb[1], limb + (int64_t)L * nk);
}

void launch_resid_split(const MatView &X, int64_t lines, int64_t k, int64_t kpad, int L, int s, int w,
                        __nv_bfloat16 *digits, int32_t *units, int32_t *lossy, int32_t *flags, int32_t *irregular,
                        int32_t *status, cudaStream_t st) {
  if (lines <= 0) return;
  if (w == 9)
    k_resid_split<9><<<(unsigned)lines, kSplitT, 0, st>>>(X, lines, k, kpad, L, s, digits, units, lossy, flags,
                                                           irregular, status);
  else
    k_resid_split<8><<<(unsigned)lines, kSplitT, 0, st>>>(X, lines, k, kpad, L, s, digits, units, lossy, flags,
                                                           irregular, status);
}

void launch_resid_table(const ResidTableArgs &a, cudaStream_t st) { k_resid_table<<<1, 128, 0, st>>>(a); }

void launch_resid_accum(const ResidAccumArgs &a, const OutView &C, cudaStream_t st) {
  if (a.m <= 0 || a.n <= 0) return;
  const dim3 g((unsigned)((a.n + kAccT - 1) / kAccT), (unsigned)a.m);
  k_resid_accum<<<g, kAccT, 0, st>>>(a, C);
}

}  // namespace mpc
