// The group table of one Ozaki call (Alg. 2's product loop, as grouped here):
// which slice pairs (t, q - t) of which real product are summed together into one
// int32 plane, in what order the accumulation visits them, in what order the slice
// GEMM hands out its units, and the call's error bounds.  It runs once per call,
// after the digit kernels, because it trims the pairs of all-zero digit planes.
#include "common.cuh"
#include "kernels.h"

namespace mpc {

// Component c of A B vanishes for every entry, given which components (re, im) of A
// and B have a nonzero value somewhere.
__device__ __forceinline__ bool component_zero(const int32_t *vA, const int32_t *vB, int c) {
  return c == 0 ? ((!vA[0] || !vB[0]) && (!vA[1] || !vB[1])) : ((!vA[0] || !vB[1]) && (!vA[1] || !vB[0]));
}

// digit-set kinds of the two operands of real product `prod`: 0 re, 1 im, 2 sums
__device__ __forceinline__ void product_kinds(int method, int prod, int &ka, int &kb) {
  if (method == MPC_4M) {
    ka = (prod == 0 || prod == 2) ? 0 : 1;   // rr, ii, ri, ir
    kb = (prod == 0 || prod == 3) ? 0 : 1;
  } else {
    ka = kb = prod;                           // rr, ii, ss
  }
}

constexpr int kMaxFlagPlanes = 512;   // digit planes of an operand (3 s + 1 <= 481) and its two value flags
constexpr int kCountBuckets = kMaxSlices + 2;   // group pair counts 0 .. kMaxSlices + 1

__device__ void accumulation_order(const GroupTableArgs &a, const int32_t *s_qc, int16_t *s_order);
__device__ void unit_schedule(const GroupTableArgs &a, const int32_t *s_qc, int *s_hist);
__device__ void call_bounds(const GroupTableArgs &a, const uint64_t *s_bd);

// product whose groups contain table entry e (the products' groups are consecutive)
__device__ __forceinline__ int product_of(const GroupTableArgs &a, int e) {
  int x = 0;
  while (x + 1 < a.n_products && e >= a.prod[x + 1].group0) ++x;
  return x;
}

// Per product (one warp each): the group table, levels ascending; then every
// group loses the pairs at its two ends whose A or B digit plane is all zero
// (their products are exactly zero), so it never splits and the table keeps its
// size; a group of zero pairs only keeps its place (count 0: no unit, no term).
// The warp also counts the dropped pairs (levels above the product's cut level)
// whose planes are both nonzero.  Then the block forms the accumulation order
// (descending level, i.e. ascending shift: every group finds its own place by binary
// searches in the other products' level-sorted lists), a warp per product sorts the
// slice GEMM's unit schedule, and thread 0 writes the call's error bounds:
//   drop[c]    = sum over the products of component c of ceil(B_prod / 2^beta),
//                B_prod = k (2^(w-2) n_{Q+1} + ceil(max_{j>=2} n_{Q+j} / 3)) over live pairs;
//   lossy_a[c] = sum of the products' truncation factors (4 for the 3M sums, else 1),
//                counted only when both operand components of the product have a
//                nonzero value somewhere (otherwise the product is exactly zero);
//   lossy_b[c] likewise;
// all three are zero for a component of A B that vanishes identically, and
// zero[c] (bounds[6 + c]) tells the accumulation to add nothing into it: a product
// needed only there (the 3M sums for real inputs) was emptied.  Finally all threads
// write the accumulation's term table (one entry per group, in accumulation order).
//
// Per-part split (zwords set, 4M): the digit positions of product x's operands start
// at the parts' offsets z (read from the status words), component c is cut at
// Q_c = Q + z_c, z_c = min over its products of z_a + z_b, and the product's pairs are
// t + u <= Q_c.  Levels are true positions while the order, the bounds and the terms
// are formed; the table entries are then rewritten relative to the operands' first
// digit plane (t0 - z_a, q - z_a - z_b), which is what the slice-GEMM kernels index.
__global__ void __launch_bounds__(128) k_group_table(GroupTableArgs a) {
  __shared__ uint64_t s_bd[4];
  __shared__ int32_t s_qc[kMaxGroupsTotal];   // per group: (q + 8) << 16 | count
  __shared__ int16_t s_order[kMaxGroupsTotal];   // the accumulation order (a copy of a.order)
  __shared__ int s_hist[4][kCountBuckets];    // per product: unit-schedule buckets
  __shared__ uint8_t s_fa[kMaxFlagPlanes], s_fb[kMaxFlagPlanes];   // plane / value flags of A and B
  __shared__ int s_pos[4][2];                 // per product: true first digit positions of A and B
  __shared__ int s_qp[4];                     // per product: its cut level
  __shared__ int s_qcomp[2];                  // per component: its cut level Q_c
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int x = threadIdx.x; x < a.planes_A + 2; x += blockDim.x) s_fa[x] = a.flagsA[x] != 0;
  for (int x = threadIdx.x; x < a.planes_B + 2; x += blockDim.x) s_fb[x] = a.flagsB[x] != 0;
  if (threadIdx.x == 0) {
    int zc[2] = {1 << 30, 1 << 30};
    for (int x = 0; x < a.n_products; ++x) {
      int pa = a.prod[x].a_pos0, pb = a.prod[x].b_pos0;
      if (a.zwords) {   // 4M: operands re (kind 0) or im (kind 1) of A and B
        int ka, kb;
        product_kinds(a.method, x, ka, kb);
        pa = kZCap - a.zwords[ka];
        pb = kZCap - a.zwords[2 + kb];
        for (int c = 0; c < 2; ++c)
          if (product_sign(a.method, c, x) != 0 && pa + pb < zc[c]) zc[c] = pa + pb;
      }
      s_pos[x][0] = pa;
      s_pos[x][1] = pb;
    }
    for (int c = 0; c < 2; ++c) s_qcomp[c] = a.Q + (a.zwords ? zc[c] : 0);
    for (int x = 0; x < a.n_products; ++x)   // 4M: every product enters one component
      s_qp[x] = a.zwords ? s_qcomp[product_sign(a.method, 0, x) != 0 ? 0 : 1] : a.Q;
  }
  __syncthreads();
  if (warp < a.n_products) {
    ProductDesc pd = a.prod[warp];
    pd.a_pos0 = s_pos[warp][0];
    pd.b_pos0 = s_pos[warp][1];
    const int Qp = s_qp[warp];
    if (lane == 0)
      build_groups(warp, pd.a_pos0, pd.a_npos, pd.b_pos0, pd.b_npos, Qp, a.gmax, a.table + pd.group0,
                   pd.n_groups);
    __syncwarp();
    // a product that enters only components of A B that vanish identically is not needed
    // (the 3M sums for real or purely imaginary inputs): all its groups are emptied
    const int32_t *vA = a.flagsA + a.planes_A, *vB = a.flagsB + a.planes_B;
    bool needed = false;
    for (int c = 0; c < 2; ++c)
      if (product_sign(a.method, c, warp) != 0 && !component_zero(vA, vB, c)) needed = true;
    auto live = [&](int t, int u) {
      return needed && s_fa[pd.a_plane0 + t - pd.a_pos0] && s_fb[pd.b_plane0 + u - pd.b_pos0];
    };
    const int ng = build_groups(warp, pd.a_pos0, pd.a_npos, pd.b_pos0, pd.b_npos, Qp, a.gmax, nullptr, 0);
    for (int e = pd.group0 + lane; e < pd.group0 + pd.n_groups; e += 32) {
      GroupEntry g = a.table[e];
      if (e >= pd.group0 + ng) {   // beyond the product's cut: an empty group at its top level (lists stay ascending)
        const int qtop = min(Qp, pd.a_pos0 + pd.a_npos - 1 + pd.b_pos0 + pd.b_npos - 1);
        g = GroupEntry{warp, qtop, pd.a_pos0, 0};
      }
      while (g.count > 0 && !live(g.t0, g.q - g.t0)) {
        ++g.t0;
        --g.count;
      }
      while (g.count > 0 && !live(g.t0 + g.count - 1, g.q - (g.t0 + g.count - 1))) --g.count;
      a.table[e] = g;
    }
    // live dropped pairs per level above the cut
    const int qmax = pd.a_pos0 + pd.a_npos - 1 + pd.b_pos0 + pd.b_npos - 1;
    uint64_t n1 = 0, nmax = 0;
    for (int q = Qp + 1; q <= qmax; ++q) {
      const int lo = max(pd.a_pos0, q - (pd.b_pos0 + pd.b_npos - 1));
      const int hi = min(pd.a_pos0 + pd.a_npos - 1, q - pd.b_pos0);
      unsigned cnt = 0;
      for (int t = lo + lane; t <= hi; t += 32) cnt += live(t, q - t) ? 1u : 0u;
      cnt = __reduce_add_sync(0xffffffffu, cnt);
      if (q == Qp + 1) n1 = cnt;
      else if (cnt > nmax) nmax = cnt;
    }
    if (lane == 0) s_bd[warp] = (uint64_t)a.k * (((uint64_t)1 << (a.w - 2)) * n1 + (nmax + 2) / 3);
  }
  __syncthreads();   // the trimmed table is complete
  int n_groups = 0;
  for (int x = 0; x < a.n_products; ++x) n_groups = max(n_groups, a.prod[x].group0 + a.prod[x].n_groups);
  for (int e = threadIdx.x; e < n_groups; e += blockDim.x) {
    const GroupEntry g = a.table[e];
    s_qc[e] = ((g.q + 8) << 16) | g.count;   // q >= -2, count <= kMaxSlices + 1
  }
  __syncthreads();
  accumulation_order(a, s_qc, s_order);
  if (warp < a.n_products) unit_schedule(a, s_qc, s_hist[warp]);
  if (threadIdx.x == 0) {
    call_bounds(a, s_bd);
    for (int c = 0; c < 2; ++c) a.bounds[8 + c] = (uint64_t)(int64_t)s_qcomp[c];
  }
  __syncthreads();   // order (and its shared copy) and bounds written
  // The accumulation's term table, one entry per group in the accumulation order.  For
  // component c the groups of the products entering it form levels l = Q_c - q, taken
  // kAccLevels at a time: a group's multiplier is its sign times 2^(w (l % kAccLevels)),
  // and the last group of each step carries the step's shift w kAccLevels (l / kAccLevels).
  const int G = n_groups;
  const bool z0 = a.bounds[6] != 0, z1 = a.bounds[7] != 0;   // components that vanish identically
  for (int x = threadIdx.x; x < G; x += blockDim.x) {
    const int e = s_order[x];
    const int q = (s_qc[e] >> 16) - 8, count = s_qc[e] & 0xFFFF;
    const bool empty = count == 0;   // all its pairs were zero: its plane is never written
    const int prod = product_of(a, e);
    int shift[2], mult[2];
    for (int c = 0; c < 2; ++c) {
      shift[c] = -1;
      mult[c] = 0;
      if (product_sign(a.method, c, prod) == 0) continue;
      const int l = s_qcomp[c] - q;   // >= 0: no kept group lies above its component's cut
      mult[c] = product_sign(a.method, c, prod) << (a.w * (l % kAccLevels));
      bool last = true;
      for (int y = x + 1; y < G; ++y) {
        const int f = s_order[y];
        if (product_sign(a.method, c, product_of(a, f)) == 0) continue;
        last = (s_qcomp[c] - ((s_qc[f] >> 16) - 8)) / kAccLevels != l / kAccLevels;
        break;
      }
      if (last) shift[c] = a.w * kAccLevels * (l / kAccLevels);
    }
    a.terms[x] = AccTerm{empty ? -1 : e, (int32_t)(((uint32_t)shift[1] << 16) | ((uint32_t)shift[0] & 0xFFFFu)),
                         empty || z0 ? 0 : mult[0], empty || z1 ? 0 : mult[1]};
  }
  __syncthreads();   // every reader of the true levels is done
  if (a.zwords) {    // the slice GEMMs index digit planes from each operand's first position
    for (int e = threadIdx.x; e < G; e += blockDim.x) {
      GroupEntry g = a.table[e];
      const int pa = s_pos[g.prod][0], pb = s_pos[g.prod][1];
      g.q -= pa + pb;
      g.t0 -= pa;
      a.table[e] = g;
    }
  }
}

// Entries of [g0, g0 + n) (levels ascending) whose level key (s_qc >> 16) is <= key.
__device__ __forceinline__ int count_level_le(const int32_t *s_qc, int g0, int n, int key) {
  int lo = 0, hi = n;   // the first entry with a larger key lies in [lo, hi]
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if ((s_qc[g0 + mid] >> 16) <= key) lo = mid + 1;
    else hi = mid;
  }
  return lo;
}

// The accumulation order: the products' groups (each product's list ascending in level)
// by descending level; within a level product by product, and within a product's level
// by descending table position.  Group e of product x at level q lands at rank
//   (its product's groups after it) + sum over x' < x of |{level >= q}| + sum over x' > x of |{level > q}|,
// each count a binary search in x''s list.  Written to a.order and to s_order.
__device__ void accumulation_order(const GroupTableArgs &a, const int32_t *s_qc, int16_t *s_order) {
  const ProductDesc *pds = a.prod;
  int G = 0;
  for (int x = 0; x < a.n_products; ++x) G = max(G, pds[x].group0 + pds[x].n_groups);
  for (int e = threadIdx.x; e < G; e += blockDim.x) {
    const int x = product_of(a, e);
    const int key = s_qc[e] >> 16;
    int r = pds[x].group0 + pds[x].n_groups - 1 - e;
    for (int y = 0; y < a.n_products; ++y) {
      if (y == x) continue;
      const int n = pds[y].n_groups;
      r += n - count_level_le(s_qc, pds[y].group0, n, y < x ? key - 1 : key);
    }
    a.order[r] = e;
    s_order[r] = (int16_t)e;
  }
}

// The slice GEMM's schedule (after the accumulation order in a.order): product by
// product, groups by descending pair count, stable, so that consecutive units take nearly
// equally long and the groups of adjacent levels, which share digit planes, stay next to
// each other.  One warp per product: a counting sort whose scatter takes 32 groups at a
// time, lanes with equal counts ranked by lane (table order).
__device__ void unit_schedule(const GroupTableArgs &a, const int32_t *s_qc, int *hist) {
  const ProductDesc *pds = a.prod;
  const int x = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int G = 0, out = 0;
  for (int y = 0; y < a.n_products; ++y) {
    G = max(G, pds[y].group0 + pds[y].n_groups);
    if (y < x) out += pds[y].n_groups;
  }
  int32_t *sched = a.order + G;
  const int g0 = pds[x].group0, g1 = g0 + pds[x].n_groups;
  for (int b = lane; b < kCountBuckets; b += 32) hist[b] = 0;
  __syncwarp();
  for (int e = g0 + lane; e < g1; e += 32) atomicAdd(&hist[kMaxSlices + 1 - (s_qc[e] & 0xFFFF)], 1);
  __syncwarp();
  if (lane == 0)   // bucket starts (descending count = ascending bucket)
    for (int b = 0; b < kCountBuckets; ++b) {
      const int c = hist[b];
      hist[b] = out;
      out += c;
    }
  __syncwarp();
  for (int base = g0; base < g1; base += 32) {
    const int e = base + lane;
    const bool v = e < g1;
    const int b = v ? kMaxSlices + 1 - (s_qc[e] & 0xFFFF) : -1 - lane;   // idle lanes: keys of their own
    const unsigned same = __match_any_sync(0xffffffffu, b);
    const int rank = __popc(same & ((1u << lane) - 1u));
    const int pos = v ? hist[b] + rank : 0;
    __syncwarp();
    if (v && rank == 0) hist[b] += __popc(same);
    __syncwarp();
    if (v) sched[pos] = e;
  }
}

// Thread 0: the call's error bounds.
__device__ void call_bounds(const GroupTableArgs &a, const uint64_t *s_bd) {
  const int n_products = a.n_products;
  const int32_t *valA = a.flagsA + a.planes_A, *valB = a.flagsB + a.planes_B;   // [re, im] values nonzero
  for (int c = 0; c < 2; ++c) {
    uint64_t bd = 0, la = 0, lb = 0;
    for (int x = 0; x < n_products; ++x) {
      if (product_sign(a.method, c, x) == 0) continue;
      int ka, kb;
      product_kinds(a.method, x, ka, kb);
      const bool va = ka == 2 ? (valA[0] || valA[1]) : valA[ka] != 0;
      const bool vb = kb == 2 ? (valB[0] || valB[1]) : valB[kb] != 0;
      bd += ceil_shift(s_bd[x], a.beta);
      const uint64_t cf = ka == 2 ? 2 : 1;   // sums: 2 ulps truncation, |.| < 2^(E+1)
      if (va && vb) {
        la += cf * cf;
        lb += cf * cf;
      }
    }
    // component c of A B vanishes identically (given which components are nonzero): every
    // product entering it, and the 3M sums, which equal one part digit for digit, cancel
    // exactly, so its accumulator is exactly zero
    const bool zero = component_zero(valA, valB, c);
    a.bounds[c] = zero ? 0 : bd;
    a.bounds[2 + c] = zero ? 0 : la;
    a.bounds[4 + c] = zero ? 0 : lb;
    a.bounds[6 + c] = zero ? 1 : 0;   // the accumulation adds nothing into this component
  }
}

// ---------------------------------------------------------------- launcher

void launch_group_table(const GroupTableArgs &a, cudaStream_t st) {
  k_group_table<<<1, 128, 0, st>>>(a);
}

}  // namespace mpc
