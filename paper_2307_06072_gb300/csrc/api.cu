// C ABI of the mpcgemm library: argument checks, the plan (Alg. 2's
// parameters and the workspace layout) and the launch sequence on the
// caller's stream.  See include/mpcgemm.h for the contract.
#include <cstdio>
#include <cstring>
#include <mutex>
#include <vector>

#include "common.cuh"
#include "kernels.h"

namespace mpc {
namespace {

constexpr int kFallbackThreads = 128;
constexpr int kFallbackBlocks = 64;
constexpr int kFallbackLimbs = 192;     // exact window of the fallback: 12288 bits

inline uint64_t align256(uint64_t x) { return (x + 255) & ~255ull; }

inline int ceil_log2(int64_t k) {
  int r = 0;
  while (((int64_t)1 << r) < k) ++r;
  return r;
}

struct Plan {
  mpc_plan pub;
  ProductDesc prod[4];
  int kernel;
  long long wait_limit;   // cycles per barrier wait of the tcgen05 kernels (0: default)
};

constexpr uint64_t kPairBufferBytes = 32ull << 30;   // residual split: default pair-product buffer

// Residual split: the pair products are computed and accumulated batch by batch; a batch is
// a run of whole (product, level) groups of table entries holding at most pair_batch planes.
// Calls f(g0, g1, first, last) for every batch [g0, g1) in table order; returns the count.
template <class F>
int for_each_pair_batch(const Plan &pl, F f) {
  const mpc_plan &P = pl.pub;
  const int total = P.n_groups_total, cap = P.pair_batch;
  int g0 = 0, g = 0, nb = 0;
  for (int x = 0; x < 4; ++x) {
    const ProductDesc &d = pl.prod[x];
    const int qhi = P.Q < 2 * P.s - 2 ? P.Q : 2 * P.s - 2;
    for (int q = 0; q <= qhi; ++q) {
      const int cnt = level_pairs(d.a_pos0, d.a_npos, d.b_pos0, d.b_npos, q);
      if (g + cnt - g0 > cap && g > g0) {
        f(g0, g, nb == 0, false);
        ++nb;
        g0 = g;
      }
      g += cnt;
    }
  }
  if (g > g0 || total == 0) {
    f(g0, g, nb == 0, true);
    ++nb;
  }
  return nb;
}

// Integer bound on the pairs a product drops, in Acc units (dropped level Q + j
// contributes <= n_{Q+j} k 2^(2w-2) 2^(-w j)): k (2^(w-2) n_{Q+1} + ceil(max_{j>=2} n / 3)).
uint64_t drop_bound(const ProductDesc &pd, int Q, int64_t k, int w) {
  const int qmax = pd.a_pos0 + pd.a_npos - 1 + pd.b_pos0 + pd.b_npos - 1;
  if (Q + 1 > qmax) return 0;
  const uint64_t n1 = (uint64_t)level_pairs(pd.a_pos0, pd.a_npos, pd.b_pos0, pd.b_npos, Q + 1);
  uint64_t nmax = 0;
  for (int q = Q + 2; q <= qmax; ++q) {
    const uint64_t v = (uint64_t)level_pairs(pd.a_pos0, pd.a_npos, pd.b_pos0, pd.b_npos, q);
    if (v > nmax) nmax = v;
  }
  return (uint64_t)k * (((uint64_t)1 << (w - 2)) * n1 + (nmax + 2) / 3);
}

int make_plan(int64_t m, int64_t n, int64_t k, int32_t p, int method, int algo, const mpc_oz_params *prm,
              Plan *out) {
  std::memset(out, 0, sizeof(*out));
  mpc_plan &P = out->pub;
  if (m < 0 || n < 0 || k < 0 || p < 1 || p > MPC_MAX_P_BITS || k > MPC_MAX_K) return MPC_EINVAL;
  if (method != MPC_4M && method != MPC_3M) return MPC_EINVAL;
  if (algo != MPC_PLAIN && algo != MPC_OZAKI) return MPC_EINVAL;
  const int L = (p + 63) / 64;
  P.algo = algo;
  P.method = method;
  P.p_bits = p;
  P.limbs = L;
  out->kernel = prm ? prm->kernel : MPC_KERNEL_AUTO;
  if (out->kernel != MPC_KERNEL_AUTO && out->kernel != MPC_KERNEL_TCGEN05 && out->kernel != MPC_KERNEL_MMA_SYNC &&
      out->kernel != MPC_KERNEL_TCGEN05_2SM && out->kernel != MPC_KERNEL_TCGEN05_N128 &&
      out->kernel != MPC_KERNEL_TCGEN05_2SM_N128)
    return MPC_EINVAL;
  if (prm && prm->wait_limit_cycles < 0) return MPC_EINVAL;
  P.split = prm ? prm->split : MPC_SPLIT_COMMON;
  if (P.split != MPC_SPLIT_COMMON && P.split != MPC_SPLIT_PER_PART && P.split != MPC_SPLIT_RESIDUAL)
    return MPC_EINVAL;
  if (P.split != MPC_SPLIT_COMMON && algo == MPC_OZAKI && method != MPC_4M) return MPC_EINVAL;
  if (prm && prm->pair_planes < 0) return MPC_EINVAL;
  const bool resid = P.split == MPC_SPLIT_RESIDUAL && algo == MPC_OZAKI;
  out->wait_limit = prm ? prm->wait_limit_cycles : 0;
  uint64_t off = 0;
  P.off_status = off;
  off = align256(off + kStatusWords * 4);
  P.off_rowexp = off;
  off = align256(off + (uint64_t)m * 4);
  P.off_colexp = off;
  off = align256(off + (uint64_t)n * 4);
  P.off_rowlossy = off;
  off = align256(off + (uint64_t)m * 4);
  P.off_collossy = off;
  off = align256(off + (uint64_t)n * 4);
  P.fallback_capacity = (uint64_t)2 * m * n;
  P.off_fallback = off;
  off = align256(off + P.fallback_capacity * 8);
  P.fb_threads = (uint64_t)kFallbackThreads * kFallbackBlocks;
  P.fb_scratch_limbs = kFallbackLimbs;
  P.off_fb_scratch = off;
  off = align256(off + P.fb_threads * P.fb_scratch_limbs * 8);
  if (algo == MPC_PLAIN) {
    // signed base-2^28 digits of X = sign floor(|x| 2^(W - E)), W = 28 D - 2 >= p + 32
    const int D = plain_digits_for(p);
    if (D < 0) return MPC_EINVAL;
    const int DP = (D + 3) & ~3, NLP = plain_limbs(D);
    P.s = D;
    P.kpad = DP;
    P.digit_bits = kPlainDigitBits;
    P.bound_shift = kPlainDigitBits * D - 2;   // W: bounds are b 2^W in units of 2^(E+F-2W)
    P.n_products = method == MPC_4M ? 4 : 3;
    P.planes_A = P.planes_B = method == MPC_4M ? 2 : 3;
    P.acc_slots = 2 * NLP;
    for (int c = 0; c < 2; ++c) {
      // per unit of k and lossy operand: Re = rr - ii and 4M Im = ri + ir carry 2 terms;
      // 3M Im = ss - rr - ii: the sums' truncation is up to 2 + 2 (4), plus 1 + 1
      const uint64_t coef = (c == 1 && method == MPC_3M) ? 6 : 2;
      P.bound_lossy_a[c] = P.bound_lossy_b[c] = coef;
    }
    P.off_digits_a = off;
    off = align256(off + (uint64_t)P.planes_A * m * k * DP * 4);
    P.off_digits_b = off;
    off = align256(off + (uint64_t)P.planes_B * n * k * DP * 4);
    P.off_groups = off;   // exact product sums [product][limb][i][j]
    off = align256(off + (uint64_t)P.n_products * NLP * m * n * 8);
    P.ws_bytes = off;
    P.launches = 8;   // init, row max, column max, 2 x digits, plain GEMM, combine, fallback (+1 zero fill when k == 0)
    return MPC_OK;
  }
  // ---- Ozaki: the digit width, Alg. 2's number of slices and the kept triangle
  const int64_t kk = k > 0 ? k : 1;
  int w = prm ? prm->digit_bits : 0;
  if (w == 0) w = (kk << prod_log2(9)) <= (int64_t)INT32_MAX ? 9 : 8;   // a pair's sum must fit int32
  if (w != 8 && w != 9) return MPC_EINVAL;
  P.digit_bits = w;
  const int guard = (prm && prm->guard_bits > 0) ? prm->guard_bits : kDefaultGuard;
  int s = (prm && prm->slices > 0) ? prm->slices : (int)((p + ceil_log2(k) + guard + w - 1) / w);
  if (s < 1 || s > kMaxSlices) return MPC_EINVAL;
  const int Q = (prm && prm->cut_level > 0) ? prm->cut_level - 1 : s - 1;
  if (Q > 2 * s) return MPC_EINVAL;
  int gmax = (int)(((int64_t)INT32_MAX) / (kk << prod_log2(w)));
  if (gmax < 1) return MPC_EINVAL;
  if (prm && prm->max_group < 0) return MPC_EINVAL;
  if (prm && prm->max_group > 0 && prm->max_group < gmax) gmax = prm->max_group;
  // residual split: one table entry per pair (the device merges runs of up to gmax pairs
  // whose units agree in every line)
  const int gbuild = resid ? 1 : gmax;
  P.s = s;
  P.Q = Q;
  P.gmax = gmax;
  P.kpad = (int32_t)(((k + kKBlock - 1) / kKBlock) * kKBlock);
  P.n_products = method == MPC_4M ? 4 : 3;
  P.planes_A = P.planes_B = 2 * s + (method == MPC_3M ? s + 1 : 0);
  // digit sets: re planes [0, s), im [s, 2s), sums [2s, 3s+1) at positions -1 .. s-1
  const int re0 = 0, im0 = s, sum0 = 2 * s;
  int total = 0, qmin = 0;
  for (int pr = 0; pr < P.n_products; ++pr) {
    ProductDesc &d = out->prod[pr];
    int a0, b0;
    if (method == MPC_4M) {
      a0 = (pr == 0 || pr == 2) ? re0 : im0;       // rr, ii, ri, ir
      b0 = (pr == 0 || pr == 3) ? re0 : im0;
      d.a_pos0 = d.b_pos0 = 0;
      d.a_npos = d.b_npos = s;
    } else if (pr < 2) {
      a0 = b0 = pr == 0 ? re0 : im0;               // rr, ii
      d.a_pos0 = d.b_pos0 = 0;
      d.a_npos = d.b_npos = s;
    } else {
      a0 = b0 = sum0;                               // ss
      d.a_pos0 = d.b_pos0 = -1;
      d.a_npos = d.b_npos = s + 1;
    }
    d.a_plane0 = a0;
    d.b_plane0 = b0;
    d.group0 = total;
    d.n_groups = build_groups(pr, d.a_pos0, d.a_npos, d.b_pos0, d.b_npos, Q, gbuild, nullptr, 0);
    P.n_groups[pr] = d.n_groups;
    total += d.n_groups;
    if (d.a_pos0 + d.b_pos0 < qmin) qmin = d.a_pos0 + d.b_pos0;
  }
  P.n_groups_total = total;
  if (!resid && total > kMaxGroupsTotal) return MPC_EINVAL;   // the group-table kernel's per-group table in shared memory
  P.acc_slots = (w * (Q - qmin) + 64) / 32 + 3;
  if (P.acc_slots > 88) return MPC_EINVAL;   // the accumulate kernel's word budget
  // bounds: b = bound_drop[c] + k (lossyA * bound_lossy_a[c] + lossyB * bound_lossy_b[c]), times 2^beta
  const int beta = 2 * w - 1 + w * (Q - s) > 0 ? 2 * w - 1 + w * (Q - s) : 0;
  P.bound_shift = beta;
  for (int c = 0; c < 2; ++c) {
    int prods[3], np = 0;
    if (c == 0) { prods[np++] = 0; prods[np++] = 1; }
    else if (method == MPC_4M) { prods[np++] = 2; prods[np++] = 3; }
    else { prods[np++] = 2; prods[np++] = 0; prods[np++] = 1; }
    uint64_t bd = 0, la = 0, lb = 0;
    for (int x = 0; x < np; ++x) {
      const ProductDesc &d = out->prod[prods[x]];
      bd += ceil_shift(drop_bound(d, Q, k, w), beta);
      const uint64_t cf = (d.a_pos0 < 0) ? 2 : 1;   // sums: 2 ulps truncation, |.| < 2^(E+1)
      la += cf * cf;
      lb += cf * cf;
    }
    P.bound_drop[c] = bd;
    P.bound_lossy_a[c] = la;
    P.bound_lossy_b[c] = lb;
  }
  P.off_digits_a = off;
  off = align256(off + (uint64_t)P.planes_A * m * P.kpad * 2);
  P.off_digits_b = off;
  off = align256(off + (uint64_t)P.planes_B * n * P.kpad * 2);
  if (resid) {
    // planes per batch: the buffer budget, at least one whole level, at most every pair
    const uint64_t plane = (uint64_t)m * n * 4;
    uint64_t cap = (prm && prm->pair_planes > 0) ? (uint64_t)prm->pair_planes
                                                : (plane ? kPairBufferBytes / plane : (uint64_t)total);
    const uint64_t maxlev = (uint64_t)(Q + 1 < s ? Q + 1 : s);
    if (cap < maxlev) cap = maxlev;
    if (cap > (uint64_t)total) cap = (uint64_t)total;
    P.pair_batch = (int32_t)cap;
  }
  P.off_groups = off;
  off = align256(off + (uint64_t)(resid ? P.pair_batch : total) * m * n * 4);
  P.off_group_table = off;
  off = align256(off + (uint64_t)total * sizeof(GroupEntry));
  // accumulation order, the slice GEMM's schedule, the operands' flags, the data-dependent bounds
  // (residual split: the flags and the bounds only)
  P.off_group_order = off;
  off = align256(off + (resid ? order_region_bytes(0, P.planes_A + 2 * s, P.planes_B + 2 * s)
                              : order_region_bytes(total, P.planes_A, P.planes_B)));
  if (resid) {
    // slice units, the accumulators between batches, truncation counts, B copied K-major
    P.off_units = off;
    off = align256(off + (uint64_t)2 * s * (m + n) * 4);
    off = align256(off + (uint64_t)2 * P.acc_slots * m * n * 4);
    off = align256(off + (uint64_t)2 * m * n * 4);
    off = align256(off + (uint64_t)2 * n * k);
    off = align256(off + (uint64_t)2 * n * k * 4);
    off = align256(off + (uint64_t)2 * L * n * k * 8);
  }
  if (prm && prm->dump_accumulators) {
    P.off_acc_dump = off;
    off = align256(off + (uint64_t)2 * m * n * (P.acc_slots + 1) * 4);
  }
  P.ws_bytes = off;
  // init, row max, column max, group table, 2 x digits, slice GEMM, accumulate, fallback (+ 2 part offsets)
  P.launches = P.split == MPC_SPLIT_PER_PART ? 11 : 9;
  if (resid)   // init, 3 transposes, 2 splits, table, per batch slice GEMM + accumulate, fallback
    P.launches = 7 + 2 * for_each_pair_batch(*out, [](int, int, bool, bool) {}) + 1;
  return MPC_OK;
}

// the tcgen05 variant of a kernel choice (auto: single CTAs with 128 x 256 tiles)
int tile_of(int kernel) {
  return kernel == MPC_KERNEL_TCGEN05_2SM        ? kTile2Sm
         : kernel == MPC_KERNEL_TCGEN05_2SM_N128 ? kTile2SmNarrow
         : kernel == MPC_KERNEL_TCGEN05_N128     ? kTileNarrow
                                                 : kTileSingle;
}

int cuda_code(cudaError_t e) { return e == cudaSuccess ? MPC_OK : MPC_ECUDA - (int)e; }

bool mat_ok(const mpc_mat *X, int64_t rows, int64_t cols) {
  if (!X || X->rows != rows || X->cols != cols || X->ld < cols) return false;
  if (rows * cols == 0) return true;      // empty operand: nothing is read
  if (X->ld < 1) return false;
  for (int c = 0; c < 2; ++c)
    if (!X->sign[c] || !X->exp[c] || !X->limb[c]) return false;
  return true;
}

MatView view_of(const mpc_mat *X) {
  MatView v;
  for (int c = 0; c < 2; ++c) {
    v.sign[c] = X->sign[c];
    v.exp[c] = X->exp[c];
    v.limb[c] = X->limb[c];
  }
  v.rows = X->rows;
  v.cols = X->cols;
  v.ld = X->ld;
  v.plane = X->rows * X->ld;
  return v;
}

OutView out_of(mpc_mat *X) {
  OutView v;
  for (int c = 0; c < 2; ++c) {
    v.sign[c] = X->sign[c];
    v.exp[c] = X->exp[c];
    v.limb[c] = X->limb[c];
  }
  v.rows = X->rows;
  v.cols = X->cols;
  v.ld = X->ld;
  v.plane = X->rows * X->ld;
  return v;
}


// ---------------------------------------------------------------- one call, in stages

struct Call {
  Plan pl;
  int64_t m, n, k;
  int32_t p;
  bool empty;
  MatView A, B;
  OutView C;
  char *ws;
  int32_t *status, *E, *F, *lossyA, *lossyB;
  int64_t *fallback;
};

int call_setup(int64_t m, int64_t n, int64_t k, int32_t p_bits, const mpc_mat *A, const mpc_mat *B, mpc_mat *C,
               int method, int algo, const mpc_oz_params *params, void *workspace, size_t ws_bytes, Call *c) {
  int rc = make_plan(m, n, k, p_bits, method, algo, params, &c->pl);
  if (rc != MPC_OK) return rc;
  if (!mat_ok(A, m, k) || !mat_ok(B, k, n) || !mat_ok(C, m, n)) return MPC_EINVAL;
  c->m = m;
  c->n = n;
  c->k = k;
  c->p = p_bits;
  c->empty = (m == 0 || n == 0);
  if (c->empty) {   // nothing to compute; a batched call still clears the problem's status block
    const bool ws_ok = workspace && !((uintptr_t)workspace & 255) && ws_bytes >= kStatusWords * 4;
    c->status = ws_ok ? (int32_t *)((char *)workspace + c->pl.pub.off_status) : nullptr;
    return MPC_OK;
  }
  if (!workspace || ((uintptr_t)workspace & 255)) return MPC_EINVAL;
  if (ws_bytes < c->pl.pub.ws_bytes) return MPC_ENOSPC;
  const mpc_plan &P = c->pl.pub;
  c->ws = (char *)workspace;
  c->status = (int32_t *)(c->ws + P.off_status);
  c->E = (int32_t *)(c->ws + P.off_rowexp);
  c->F = (int32_t *)(c->ws + P.off_colexp);
  c->lossyA = (int32_t *)(c->ws + P.off_rowlossy);
  c->lossyB = (int32_t *)(c->ws + P.off_collossy);
  c->fallback = (int64_t *)(c->ws + P.off_fallback);
  c->A = view_of(A);
  c->B = view_of(B);
  c->C = out_of(C);
  return MPC_OK;
}

// exponents, then the split (digits + group tables) or the plain fixed-point operands
void call_pre(Call &c, cudaStream_t st) {
  const mpc_plan &P = c.pl.pub;
  const int L = P.limbs;
  // Ozaki: the operands' flags (digit planes, then the two components), after the order and schedule
  int32_t *plane_nz = P.algo == MPC_OZAKI ? (int32_t *)(c.ws + P.off_group_order) + 2 * (int64_t)P.n_groups_total
                                          : nullptr;
  const int flagsA = P.planes_A + 2;
  launch_init(c.status, c.E, c.m, c.F, c.n, c.lossyA, c.lossyB, st, plane_nz,
              plane_nz ? (int64_t)flagsA + P.planes_B + 2 : 0);
  if (c.k == 0) {
    launch_zero_output(c.C, c.m, c.n, L, st);
    return;
  }
  launch_line_max(c.A, c.B, c.m, c.n, c.k, L, c.E, c.F, st);
  if (P.algo == MPC_PLAIN) {
    const int W = P.bound_shift, want_sum = P.method == MPC_3M;
    launch_plain_digits(c.A, 0, c.m, c.k, L, P.s, P.kpad, W, want_sum, c.E, c.lossyA,
                        (int32_t *)(c.ws + P.off_digits_a), st);
    launch_plain_digits(c.B, 1, c.n, c.k, L, P.s, P.kpad, W, want_sum, c.F, c.lossyB,
                        (int32_t *)(c.ws + P.off_digits_b), st);
  } else {
    const int want_sum = P.method == MPC_3M;
    const bool per_part = P.split == MPC_SPLIT_PER_PART;
    if (per_part) launch_part_offsets(c.A, c.B, c.m, c.n, c.k, L, P.digit_bits, c.E, c.F, c.status, st);
    launch_oz_digits(c.A, 0, c.m, c.k, P.kpad, L, P.s, P.digit_bits, want_sum, c.E, c.lossyA,
                     (__nv_bfloat16 *)(c.ws + P.off_digits_a), plane_nz, per_part ? c.status + kStPartZ : nullptr, st);
    launch_oz_digits(c.B, 1, c.n, c.k, P.kpad, L, P.s, P.digit_bits, want_sum, c.F, c.lossyB,
                     (__nv_bfloat16 *)(c.ws + P.off_digits_b), plane_nz + flagsA,
                     per_part ? c.status + kStPartZ + 2 : nullptr, st);
    GroupTableArgs ga{};
    for (int x = 0; x < 4; ++x) ga.prod[x] = c.pl.prod[x];
    ga.n_products = P.n_products;
    ga.method = P.method;
    ga.Q = P.Q;
    ga.gmax = P.gmax;
    ga.beta = P.bound_shift;
    ga.w = P.digit_bits;
    ga.k = c.k;
    ga.planes_A = P.planes_A;
    ga.planes_B = P.planes_B;
    ga.flagsA = plane_nz;
    ga.flagsB = plane_nz + flagsA;
    ga.table = (GroupEntry *)(c.ws + P.off_group_table);
    ga.order = (int32_t *)(c.ws + P.off_group_order);
    ga.bounds = (uint64_t *)(c.ws + P.off_group_order + bounds_offset(P.n_groups_total, P.planes_A, P.planes_B));
    ga.terms = (AccTerm *)(c.ws + P.off_group_order + terms_offset(P.n_groups_total, P.planes_A, P.planes_B));
    ga.zwords = per_part ? c.status + kStPartZ : nullptr;
    launch_group_table(ga, st);
  }
}

SliceGemmArgs slice_args(const Call &c) {
  const mpc_plan &P = c.pl.pub;
  SliceGemmArgs sa{};
  sa.dA = (const __nv_bfloat16 *)(c.ws + P.off_digits_a);
  sa.dB = (const __nv_bfloat16 *)(c.ws + P.off_digits_b);
  sa.m = c.m;
  sa.n = c.n;
  sa.kpad = P.kpad;
  sa.chunk_kb = chunk_kblocks(P.digit_bits);
  sa.groups = (const GroupEntry *)(c.ws + P.off_group_table);
  sa.sched = (const int32_t *)(c.ws + P.off_group_order) + P.n_groups_total;
  sa.n_entries = P.n_groups_total;
  for (int x = 0; x < 4; ++x) sa.prod[x] = c.pl.prod[x];
  sa.out = (int32_t *)(c.ws + P.off_groups);
  sa.status = c.status;
  return sa;
}

void call_gemm_plain(Call &c, cudaStream_t st) {
  const mpc_plan &P = c.pl.pub;
  PlainGemmArgs ga{};
  ga.dA = (const int32_t *)(c.ws + P.off_digits_a);
  ga.dB = (const int32_t *)(c.ws + P.off_digits_b);
  ga.m = c.m;
  ga.n = c.n;
  ga.k = c.k;
  ga.D = P.s;
  ga.n_products = P.n_products;
  // operand planes: 4M rr, ii, ri, ir; 3M rr, ii, ss (plane 2 = X_re + X_im)
  static const int pa4[4] = {0, 1, 0, 1}, pb4[4] = {0, 1, 1, 0}, pa3[4] = {0, 1, 2, 0}, pb3[4] = {0, 1, 2, 0};
  for (int x = 0; x < 4; ++x) {
    ga.planeA[x] = P.method == MPC_4M ? pa4[x] : pa3[x];
    ga.planeB[x] = P.method == MPC_4M ? pb4[x] : pb3[x];
  }
  ga.sums = (uint64_t *)(c.ws + P.off_groups);
  launch_plain_gemm(ga, st);
}

// the plain path's accumulate-and-round stage: combine the exact product sums, certify, round
void call_plain_combine(Call &c, cudaStream_t st) {
  const mpc_plan &P = c.pl.pub;
  PlainCombineArgs ca{};
  ca.sums = (const uint64_t *)(c.ws + P.off_groups);
  ca.m = c.m;
  ca.n = c.n;
  ca.k = c.k;
  ca.p = c.p;
  ca.L = P.limbs;
  ca.D = P.s;
  ca.W = P.bound_shift;
  ca.method = P.method;
  ca.coef[0] = P.bound_lossy_a[0];
  ca.coef[1] = P.bound_lossy_a[1];
  ca.E = c.E;
  ca.F = c.F;
  ca.lossyA = c.lossyA;
  ca.lossyB = c.lossyB;
  ca.fallback = c.fallback;
  ca.fallback_cap = (int64_t)P.fallback_capacity;
  ca.status = c.status;
  launch_plain_combine(ca, c.C, st);
}

void call_accum(Call &c, cudaStream_t st) {
  const mpc_plan &P = c.pl.pub;
  if (P.algo != MPC_OZAKI) {
    call_plain_combine(c, st);
    return;
  }
  AccumArgs aa{};
  aa.planes = (const int32_t *)(c.ws + P.off_groups);
  aa.groups = (const GroupEntry *)(c.ws + P.off_group_table);
  aa.order = (const int32_t *)(c.ws + P.off_group_order);
  aa.n_entries = P.n_groups_total;
  aa.m = c.m;
  aa.n = c.n;
  aa.k = c.k;
  aa.p = c.p;
  aa.L = P.limbs;
  aa.Q = P.Q;
  aa.nslot = P.acc_slots;
  aa.method = P.method;
  aa.E = c.E;
  aa.F = c.F;
  aa.lossyA = c.lossyA;
  aa.lossyB = c.lossyB;
  aa.bound_shift = P.bound_shift;
  aa.w = P.digit_bits;
  aa.bounds = (const uint64_t *)(c.ws + P.off_group_order + bounds_offset(P.n_groups_total, P.planes_A, P.planes_B));
  aa.terms = (const AccTerm *)(c.ws + P.off_group_order + terms_offset(P.n_groups_total, P.planes_A, P.planes_B));
  for (int x = 0; x < 2; ++x) {
    aa.bound_drop[x] = P.bound_drop[x];
    aa.bound_lossy_a[x] = P.bound_lossy_a[x];
    aa.bound_lossy_b[x] = P.bound_lossy_b[x];
  }
  aa.fallback = c.fallback;
  aa.fallback_cap = (int64_t)P.fallback_capacity;
  aa.status = c.status;
  aa.acc_dump = P.off_acc_dump ? (uint32_t *)(c.ws + P.off_acc_dump) : nullptr;
  launch_oz_accum(aa, c.C, st);
}

void call_fallback(Call &c, cudaStream_t st) {
  const mpc_plan &P = c.pl.pub;
  FallbackArgs fa{};
  fa.m = c.m;
  fa.n = c.n;
  fa.k = c.k;
  fa.p = c.p;
  fa.L = P.limbs;
  fa.list = c.fallback;
  fa.cap = (int64_t)P.fallback_capacity;
  fa.scratch = (uint64_t *)(c.ws + P.off_fb_scratch);
  fa.scratch_limbs = (int)P.fb_scratch_limbs;
  fa.status = c.status;
  launch_fallback(fa, c.A, c.B, c.C, kFallbackBlocks, kFallbackThreads, st);
}

// The residual split (MPC_SPLIT_RESIDUAL, 4M): B copied K-major, both operands cut with a
// unit re-measured before every slice, the single-pair table and bounds, then the pair
// products and their accumulation batch by batch (whole levels), then the exact fallback.
int run_residual(Call &c, const mpc_stage_events *events, cudaStream_t st) {
  const mpc_plan &P = c.pl.pub;
  auto mark = [&](int x) {
    if (events && events->ev[x]) cudaEventRecord((cudaEvent_t)events->ev[x], st);
  };
  const int L = P.limbs, s = P.s;
  const int64_t m = c.m, n = c.n, k = c.k, mn = m * n, nk = n * k;
  // flags: A's planes, its two values, its slices' irregular steps; then the same for B
  int32_t *flags = (int32_t *)(c.ws + P.off_group_order);
  const int fA = P.planes_A + 2 + 2 * s, fB = P.planes_B + 2 + 2 * s;
  int32_t *flagsB = flags + fA, *irrA = flags + P.planes_A + 2, *irrB = flagsB + P.planes_B + 2;
  uint64_t *bounds = (uint64_t *)(c.ws + P.off_group_order + bounds_offset(0, fA - 2, fB - 2));
  mark(0);
  launch_init(c.status, c.E, m, c.F, n, c.lossyA, c.lossyB, st, flags, (int64_t)fA + fB);
  if (k == 0) {
    launch_zero_output(c.C, m, n, L, st);
    for (int x = 1; x <= 4; ++x) mark(x);
    return cuda_code(cudaGetLastError());
  }
  // the workspace regions of this variant (mpc_plan.off_units)
  uint64_t o = P.off_units;
  int32_t *uA = (int32_t *)(c.ws + o), *uB = uA + (int64_t)2 * s * m;
  o = align256(o + (uint64_t)2 * s * (m + n) * 4);
  uint32_t *acc = (uint32_t *)(c.ws + o);
  o = align256(o + (uint64_t)2 * P.acc_slots * mn * 4);
  uint32_t *trunc = (uint32_t *)(c.ws + o);
  o = align256(o + (uint64_t)2 * mn * 4);
  uint8_t *bt_sign = (uint8_t *)(c.ws + o);
  o = align256(o + (uint64_t)2 * nk);
  int32_t *bt_exp = (int32_t *)(c.ws + o);
  o = align256(o + (uint64_t)2 * nk * 4);
  uint64_t *bt_limb = (uint64_t *)(c.ws + o);
  launch_transpose_operand(c.B, k, n, L, bt_sign, bt_exp, bt_limb, st);
  MatView Bt;
  for (int x = 0; x < 2; ++x) {
    Bt.sign[x] = bt_sign + x * nk;
    Bt.exp[x] = bt_exp + x * nk;
    Bt.limb[x] = bt_limb + (int64_t)x * L * nk;
  }
  Bt.rows = n;
  Bt.cols = k;
  Bt.ld = k;
  Bt.plane = nk;
  __nv_bfloat16 *dA = (__nv_bfloat16 *)(c.ws + P.off_digits_a), *dB = (__nv_bfloat16 *)(c.ws + P.off_digits_b);
  launch_resid_split(c.A, m, k, P.kpad, L, s, P.digit_bits, dA, uA, c.lossyA, flags, irrA, c.status, st);
  launch_resid_split(Bt, n, k, P.kpad, L, s, P.digit_bits, dB, uB, c.lossyB, flagsB, irrB, c.status, st);
  GroupEntry *table = (GroupEntry *)(c.ws + P.off_group_table);
  ResidTableArgs ta{};
  for (int x = 0; x < 4; ++x) ta.prod[x] = c.pl.prod[x];
  ta.s = s;
  ta.Q = P.Q;
  ta.w = P.digit_bits;
  ta.beta = P.bound_shift;
  ta.k = k;
  ta.planes_A = P.planes_A;
  ta.planes_B = P.planes_B;
  ta.gmax = P.gmax;
  ta.flagsA = flags;
  ta.flagsB = flagsB;
  ta.irregularA = irrA;
  ta.irregularB = irrB;
  ta.table = table;
  ta.bounds = bounds;
  launch_resid_table(ta, st);
  mark(1);
  SliceGemmArgs sa = slice_args(c);
  sa.sched = nullptr;   // table order
  ResidAccumArgs aa{};
  aa.planes = (const int32_t *)(c.ws + P.off_groups);
  aa.m = m;
  aa.n = n;
  aa.k = k;
  aa.p = c.p;
  aa.L = L;
  aa.Q = P.Q;
  aa.s = s;
  aa.w = P.digit_bits;
  aa.nslot = P.acc_slots;
  aa.beta = P.bound_shift;
  aa.uA = uA;
  aa.uB = uB;
  aa.acc = acc;
  aa.trunc = trunc;
  aa.bounds = bounds;
  aa.lossyA = c.lossyA;
  aa.lossyB = c.lossyB;
  aa.fallback = c.fallback;
  aa.fallback_cap = (int64_t)P.fallback_capacity;
  aa.status = c.status;
  aa.acc_dump = P.off_acc_dump ? (uint32_t *)(c.ws + P.off_acc_dump) : nullptr;
  int rc = MPC_OK;
  for_each_pair_batch(c.pl, [&](int g0, int g1, bool first, bool last) {
    if (rc != MPC_OK) return;
    sa.groups = table + g0;
    sa.n_entries = g1 - g0;
    if (sa.n_entries > 0) {
      if (c.pl.kernel == MPC_KERNEL_MMA_SYNC) {
        launch_slicegemm_mma(sa, st);
      } else {
        cudaMemsetAsync(c.status + kStUnitCounter, 0, 4, st);   // the persistent kernel's unit counter
        const cudaError_t e = launch_slicegemm_tc(sa, st, tile_of(c.pl.kernel), c.pl.wait_limit);
        if (e == cudaErrorNotSupported && c.pl.kernel == MPC_KERNEL_AUTO) launch_slicegemm_mma(sa, st);
        else if (e != cudaSuccess) rc = e == cudaErrorNotSupported ? MPC_ENOTSUP : cuda_code(e);
      }
    }
    if (rc != MPC_OK) return;
    if (last) mark(2);
    aa.table = table + g0;
    aa.n_entries = g1 - g0;
    aa.first = first;
    aa.last = last;
    launch_resid_accum(aa, c.C, st);
  });
  if (rc != MPC_OK) return rc;
  mark(3);
  call_fallback(c, st);
  mark(4);
  return cuda_code(cudaGetLastError());
}

}  // namespace
}  // namespace mpc

using namespace mpc;

extern "C" {

int mpcgemm_plan(int64_t m, int64_t n, int64_t k, int32_t p_bits, int method, int algo,
                 const mpc_oz_params *params, mpc_plan *out) {
  if (!out) return MPC_EINVAL;
  Plan pl;
  const int rc = make_plan(m, n, k, p_bits, method, algo, params, &pl);
  if (rc == MPC_OK) *out = pl.pub;
  return rc;
}

size_t mpcgemm_workspace_size(int64_t m, int64_t n, int64_t k, int32_t p_bits, int method, int algo) {
  Plan pl;
  if (make_plan(m, n, k, p_bits, method, algo, nullptr, &pl) != MPC_OK) return 0;
  return (size_t)pl.pub.ws_bytes;
}

int mpcgemm_profiled(int64_t m, int64_t n, int64_t k, int32_t p_bits, const mpc_mat *A, const mpc_mat *B,
                     mpc_mat *C, int method, int algo, const mpc_oz_params *params, const mpc_stage_events *events,
                     void *workspace, size_t ws_bytes, void *stream) {
  Call c;
  int rc = call_setup(m, n, k, p_bits, A, B, C, method, algo, params, workspace, ws_bytes, &c);
  if (rc != MPC_OK || c.empty) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  cudaGetLastError();   // clear a stale error of an earlier, unrelated call
  if (c.pl.pub.algo == MPC_OZAKI && c.pl.pub.split == MPC_SPLIT_RESIDUAL) return run_residual(c, events, st);
  auto mark = [&](int x) {
    if (events && events->ev[x]) cudaEventRecord((cudaEvent_t)events->ev[x], st);
  };
  mark(0);
  call_pre(c, st);
  mark(1);
  if (c.k > 0) {
    if (c.pl.pub.algo == MPC_PLAIN) {
      call_gemm_plain(c, st);
    } else {
      SliceGemmArgs sa = slice_args(c);
      if (c.pl.kernel == MPC_KERNEL_MMA_SYNC) {
        launch_slicegemm_mma(sa, st);
      } else {   // auto: the single-CTA tcgen05 kernel with 128 x 256 tiles
        const cudaError_t e = launch_slicegemm_tc(sa, st, tile_of(c.pl.kernel), c.pl.wait_limit);
        if (e == cudaErrorNotSupported && c.pl.kernel == MPC_KERNEL_AUTO) launch_slicegemm_mma(sa, st);
        else if (e != cudaSuccess) return e == cudaErrorNotSupported ? MPC_ENOTSUP : cuda_code(e);
      }
    }
  }
  mark(2);
  if (c.k > 0) call_accum(c, st);
  mark(3);
  if (c.k > 0) call_fallback(c, st);
  mark(4);
  return cuda_code(cudaGetLastError());
}

int mpcgemm_batched_workspace(int count, const mpc_problem *probs, const mpc_oz_params *params, uint64_t *offsets,
                              size_t *total) {
  if (count < 0 || (count > 0 && !probs) || !total) return MPC_EINVAL;
  if (params && params->split == MPC_SPLIT_RESIDUAL) return MPC_EINVAL;   // single calls only
  uint64_t off = 0;
  for (int x = 0; x < count; ++x) {
    Plan pl;
    const mpc_problem &q = probs[x];
    const int rc = make_plan(q.m, q.n, q.k, q.p_bits, q.method, q.algo, params, &pl);
    if (rc != MPC_OK) return rc;
    if (offsets) offsets[x] = off;
    off = align256(off + pl.pub.ws_bytes);
  }
  *total = (size_t)off;
  return MPC_OK;
}

namespace {

// Side streams of a batched call: the small per-problem kernels (split, group table,
// accumulation) of different problems are independent, so they are spread over a pool
// of streams forked from and joined back into the caller's stream (under stream capture
// this becomes parallel branches of the graph).  Every caller stream gets a pool of its
// own, so that batched calls on independent streams stay independent; a pool is created
// the first time its stream makes a batched call outside capture, and its mutex keeps
// the fork / join events of concurrent calls on that stream apart while they are
// enqueued.  Past kMaxPools caller streams, calls run on the caller's stream alone.
// Only batches of at least kSideMinBatch problems use side streams: the GPU has few
// hardware work queues (8 by default), and the streams of many small concurrent calls
// (a serving loop's slots) would share them with each other's long slice-GEMM launches.
constexpr int kSideStreams = 8;
constexpr int kSideMinBatch = 16;
constexpr int kMaxPools = 64;
struct SidePool {
  int dev = -1;
  cudaStream_t caller = nullptr;
  bool ok = false;
  cudaStream_t s[kSideStreams];
  cudaEvent_t fork, join[kSideStreams];
  std::mutex mu;
};
SidePool g_pools[kMaxPools];
int g_npools = 0;
std::mutex g_pools_mu;

// nullptr: run on the caller's stream (no pool is created while `st` is being captured,
// since creating streams and events there could invalidate the capture)
SidePool *side_pool(cudaStream_t st) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> lk(g_pools_mu);
  for (int x = 0; x < g_npools; ++x)
    if (g_pools[x].dev == dev && g_pools[x].caller == st) return g_pools[x].ok ? &g_pools[x] : nullptr;
  if (cs != cudaStreamCaptureStatusNone || g_npools == kMaxPools) return nullptr;
  SidePool &sp = g_pools[g_npools++];
  sp.dev = dev;
  sp.caller = st;
  bool ok = cudaEventCreateWithFlags(&sp.fork, cudaEventDisableTiming) == cudaSuccess;
  for (int x = 0; x < kSideStreams && ok; ++x)
    ok = cudaStreamCreateWithFlags(&sp.s[x], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&sp.join[x], cudaEventDisableTiming) == cudaSuccess;
  sp.ok = ok;
  return ok ? &sp : nullptr;
}

void side_fork(SidePool *sp, cudaStream_t st) {
  cudaEventRecord(sp->fork, st);
  for (int x = 0; x < kSideStreams; ++x) cudaStreamWaitEvent(sp->s[x], sp->fork, 0);
}

void side_join(SidePool *sp, cudaStream_t st) {
  for (int x = 0; x < kSideStreams; ++x) {
    cudaEventRecord(sp->join[x], sp->s[x]);
    cudaStreamWaitEvent(st, sp->join[x], 0);
  }
}

}  // namespace

int mpcgemm_batched(int count, const mpc_problem *probs, const mpc_oz_params *params, void *workspace,
                    size_t ws_bytes, void *stream) {
  if (count < 0 || (count > 0 && !probs)) return MPC_EINVAL;
  if (params && params->split == MPC_SPLIT_RESIDUAL) return MPC_EINVAL;   // single calls only
  if (count == 0) return MPC_OK;
  thread_local std::vector<Call> calls;   // reused: no host allocation once it has grown
  if (calls.size() < (size_t)count) calls.resize((size_t)count);
  uint64_t off = 0;
  for (int x = 0; x < count; ++x) {   // plan and check everything before any launch
    const mpc_problem &q = probs[x];
    if (!workspace || ws_bytes < off) return MPC_ENOSPC;
    const int rc = call_setup(q.m, q.n, q.k, q.p_bits, q.A, q.B, q.C, q.method, q.algo, params,
                              (char *)workspace + off, ws_bytes - (size_t)off, &calls[x]);
    if (rc != MPC_OK) return rc;
    off = align256(off + calls[x].pl.pub.ws_bytes);
  }
  cudaStream_t st = (cudaStream_t)stream;
  cudaGetLastError();
  SidePool *sp = count >= kSideMinBatch ? side_pool(st) : nullptr;
  std::unique_lock<std::mutex> lock;
  if (sp) {
    lock = std::unique_lock<std::mutex>(sp->mu);
    side_fork(sp, st);
  }
  auto lane = [&](int x) { return sp ? sp->s[x % kSideStreams] : st; };
  for (int x = 0; x < count; ++x) {
    if (!calls[x].empty) call_pre(calls[x], lane(x));
    else if (calls[x].status) cudaMemsetAsync(calls[x].status, 0, kStatusWords * 4, lane(x));
  }
  if (sp) side_join(sp, st);
  thread_local std::vector<SliceGemmArgs> slices;
  slices.clear();
  const int kernel = params ? params->kernel : MPC_KERNEL_AUTO;
  for (int x = 0; x < count; ++x) {
    Call &c = calls[x];
    if (c.empty || c.k == 0) continue;
    if (c.pl.pub.algo == MPC_PLAIN) {
      call_gemm_plain(c, st);
    } else if (kernel == MPC_KERNEL_MMA_SYNC) {
      launch_slicegemm_mma(slice_args(c), st);
    } else {
      slices.push_back(slice_args(c));
    }
  }
  if (!slices.empty()) {   // one persistent launch for every Ozaki problem (64 per launch)
    const cudaError_t e = launch_slicegemm_tc_batch(slices.data(), (int)slices.size(), st, tile_of(kernel),
                                                    params ? params->wait_limit_cycles : 0);
    if (e == cudaErrorNotSupported && kernel == MPC_KERNEL_AUTO) {
      for (const SliceGemmArgs &sa : slices) launch_slicegemm_mma(sa, st);
    } else if (e != cudaSuccess) {
      return e == cudaErrorNotSupported ? MPC_ENOTSUP : cuda_code(e);
    }
  }
  if (sp) side_fork(sp, st);
  for (int x = 0; x < count; ++x)
    if (!calls[x].empty && calls[x].k > 0) {
      call_accum(calls[x], lane(x));
      call_fallback(calls[x], lane(x));
    }
  if (sp) side_join(sp, st);
  return cuda_code(cudaGetLastError());
}

int mpcgemm_ex(int64_t m, int64_t n, int64_t k, int32_t p_bits, const mpc_mat *A, const mpc_mat *B, mpc_mat *C,
               int method, int algo, const mpc_oz_params *params, void *workspace, size_t ws_bytes,
               void *stream) {
  return mpcgemm_profiled(m, n, k, p_bits, A, B, C, method, algo, params, nullptr, workspace, ws_bytes, stream);
}

int mpcgemm(int64_t m, int64_t n, int64_t k, int32_t p_bits, const mpc_mat *A, const mpc_mat *B, mpc_mat *C,
            int method, int algo, void *workspace, size_t ws_bytes, void *stream) {
  return mpcgemm_ex(m, n, k, p_bits, A, B, C, method, algo, nullptr, workspace, ws_bytes, stream);
}

int mpcgemm_read_status(const void *workspace, size_t ws_bytes, mpc_status *status, void *stream) {
  if (!workspace || !status || ws_bytes < kStatusWords * 4) return MPC_EINVAL;
  int32_t words[kStatusWords];
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess) e = cudaMemcpy(words, workspace, sizeof(words), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_code(e);
  status->erange = words[kStErange];
  status->fallback_entries = words[kStFallbackCount];
  status->fallback_overflow = words[kStFallbackOverflow];
  status->uncertified = words[kStUncertified];
  status->device_timeout = words[kStTimeout];
  return status->erange ? MPC_ERANGE : MPC_OK;
}

const char *mpcgemm_strerror(int code) {
  switch (code) {
    case MPC_OK: return "success";
    case MPC_EINVAL: return "invalid argument (size, precision, pointer, method or parameter)";
    case MPC_ENOSPC: return "workspace too small";
    case MPC_ERANGE: return "result exponent outside int32";
    case MPC_ENOTSUP: return "not supported on this device";
    default: break;
  }
  if (code <= MPC_ECUDA) return cudaGetErrorString((cudaError_t)(MPC_ECUDA - code));
  return "unknown error";
}

int mpcgemm_version(void) { return 100; }

}  // extern "C"
