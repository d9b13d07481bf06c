// Internal launchers of the mpcgemm CUDA kernels (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "common.cuh"

namespace mpc {

struct SliceGemmArgs {
  const __nv_bfloat16 *dA;      // digit planes of A: [plane][m][kpad]
  const __nv_bfloat16 *dB;      // digit planes of B: [plane][n][kpad]
  int64_t m, n, kpad;
  int chunk_kb;                 // k-blocks of 64 per exact fp32 chunk (digit width)
  const GroupEntry *groups;     // group table (n_entries)
  const int32_t *sched;         // order in which the groups' units are handed out (null: table order)
  int32_t n_entries;
  ProductDesc prod[4];
  int32_t *out;                 // group sums: [entry][m][n] int32
  int32_t *status;
};

// Levels folded into the exact accumulators per step: the level l = Q_c - q (l >= 0) of
// component c belongs to step l / kAccLevels and enters it with weight 2^(w (l % kAccLevels)).
constexpr int kAccLevels = 3;

// One accumulation term per group, in the accumulation order (descending level):
// group plane index (-1: an emptied group), the two multipliers, and per component -- on
// the last group of a step among the groups of the products entering that component --
// the step's shift w kAccLevels (l / kAccLevels), else -1.  Written by k_group_table, read
// by k_oz_accum.
struct __align__(16) AccTerm {
  int32_t plane;
  int32_t shifts;   // low 16 bits: real part's shift, high 16 bits: imaginary part's (int16, -1: none)
  int32_t s0, s1;   // the group's multiplier in the real / imaginary part: its sign (-1, 0, 1)
                    // times 2^(w (l % kAccLevels))
};
static_assert(sizeof(AccTerm) == 16, "AccTerm is read as one int4");

// Group table, accumulation order, unit schedule and the data-dependent error
// bounds of one Ozaki call (k_group_table, after the digits).
struct GroupTableArgs {
  ProductDesc prod[4];
  int n_products, method, Q, gmax, beta, w;
  int64_t k;
  int planes_A, planes_B;
  const int32_t *flagsA, *flagsB;   // per digit plane: any nonzero digit; then per component: any nonzero value
  GroupEntry *table;
  int32_t *order;                   // accumulation order [G], then the unit schedule [G]
  uint64_t *bounds;                 // out: drop[2], lossy_a[2], lossy_b[2], zero[2], then Q_c[2] (int64)
  AccTerm *terms;                      // out: the accumulation's term table [G]
  const int32_t *zwords;               // per-part split: kZCap - z of A re, A im, B re, B im (else null)
};

// byte offset of the bounds inside the group-order region
__host__ __device__ inline uint64_t bounds_offset(int64_t groups, int planes_A, int planes_B) {
  const uint64_t b = (uint64_t)groups * 8 + (uint64_t)(planes_A + 2 + planes_B + 2) * 4;
  return (b + 7) & ~7ull;
}

// byte offset of the term table inside the group-order region (after the 8 bounds and
// the two components' cut levels Q_c), and the region's size
__host__ __device__ inline uint64_t terms_offset(int64_t groups, int planes_A, int planes_B) {
  return (bounds_offset(groups, planes_A, planes_B) + 10 * 8 + 15) & ~15ull;
}
__host__ __device__ inline uint64_t order_region_bytes(int64_t groups, int planes_A, int planes_B) {
  return terms_offset(groups, planes_A, planes_B) + (uint64_t)groups * sizeof(AccTerm);
}

struct AccumArgs {
  const int32_t *planes;        // group sums [entry][m][n]
  const GroupEntry *groups;
  const int32_t *order;         // groups by descending level
  int32_t n_entries;
  int64_t m, n, k;
  int p, L, Q, nslot, method;
  const int32_t *E, *F, *lossyA, *lossyB;
  int bound_shift, w;          // bounds are b 2^beta; w bits per digit
  uint64_t bound_drop[2], bound_lossy_a[2], bound_lossy_b[2];   // data-independent (plan)
  const uint64_t *bounds;       // the call's bounds (drop[2], lossy_a[2], lossy_b[2], zero[2]) and cut
                                // levels Q_c[2] (int64), from k_group_table
  const AccTerm *terms;            // the term table, from k_group_table
  int64_t *fallback;            // list of (i*n + j)*2 + c
  int64_t fallback_cap;
  int32_t *status;
  uint32_t *acc_dump;           // null, or per component: nslot words of |Acc| and its sign
};

struct FallbackArgs {
  int64_t m, n, k;
  int p, L;
  const int64_t *list;
  int64_t cap;
  uint64_t *scratch;            // per thread: scratch_limbs words
  int scratch_limbs;
  int32_t *status;
};

// Plain path (k_plain_gemm / k_plain_combine).  Operand digits [plane][line][l][DP]
// (int32, base 2^28, least significant first); exact product sums
// [product][limb][i][j] (two's complement, plain_limbs(D) 64-bit limbs).
struct PlainGemmArgs {
  const int32_t *dA, *dB;
  int64_t m, n, k;
  int D;
  int n_products;
  int planeA[4], planeB[4];   // operand planes of each real product
  uint64_t *sums;
};

struct PlainCombineArgs {
  const uint64_t *sums;
  int64_t m, n, k;
  int p, L, D, W, method;
  uint64_t coef[2];           // lossy bound per unit of k and lossy operand, Re / Im
  const int32_t *E, *F, *lossyA, *lossyB;
  int64_t *fallback;
  int64_t fallback_cap;
  int32_t *status;
};

// Residual split (MPC_SPLIT_RESIDUAL, 4M): the single-pair group table and the call's bounds.
struct ResidTableArgs {
  ProductDesc prod[4];
  int s, Q, w, beta, gmax;
  int64_t k;
  int planes_A, planes_B;
  const int32_t *flagsA, *flagsB;   // per digit plane: any nonzero digit; then per part: any nonzero value
  const int32_t *irregularA, *irregularB;   // per digit plane: some line's unit is not w below the last one
  GroupEntry *table;
  uint64_t *bounds;                 // out: drop[2], lossy_a[2], lossy_b[2], zero[2], Q_c[2]
};

// Residual split: one batch of pair planes folded into the exact accumulators.
struct ResidAccumArgs {
  const int32_t *planes;        // the batch's pair products [entry][m][n]
  const GroupEntry *table;      // the batch's table entries
  int32_t n_entries;
  int64_t m, n, k;
  int p, L, Q, s, w, nslot, beta;
  const int32_t *uA, *uB;       // slice units [part][slice][line] (INT32_MIN: a zero slice)
  uint32_t *acc;                // accumulator words between batches [comp][word][m n]
  uint32_t *trunc;              // truncation counts [comp][m n]
  int first, last;
  const uint64_t *bounds;       // from k_resid_table
  const int32_t *lossyA, *lossyB;
  int64_t *fallback;
  int64_t fallback_cap;
  int32_t *status;
  uint32_t *acc_dump;           // null, or per component: nslot words of |Acc| and its sign
};

// digits per operand of the plain path at precision p (an instantiated size)
int plain_digits_for(int p);

void launch_init(int32_t *status, int32_t *E, int64_t m, int32_t *F, int64_t n, int32_t *lossyA, int32_t *lossyB,
                 cudaStream_t st, int32_t *extra = nullptr, int64_t n_extra = 0);
void launch_line_max(const MatView &A, const MatView &B, int64_t m, int64_t n, int64_t k, int L, int32_t *E,
                     int32_t *F, cudaStream_t st);
// per-part split: the part offsets z of A (re, im) and B (re, im) into status words kStPartZ..
void launch_part_offsets(const MatView &A, const MatView &B, int64_t m, int64_t n, int64_t k, int L, int w,
                         const int32_t *E, const int32_t *F, int32_t *status, cudaStream_t st);
// zoff: null (one grid per line) or this operand's two offset words (kZCap - z of re, im)
void launch_oz_digits(const MatView &X, int side, int64_t lines, int64_t k, int64_t kpad, int L, int s, int wd,
                      int want_sum, const int32_t *E, int32_t *lossy, __nv_bfloat16 *digits, int32_t *plane_nz,
                      const int32_t *zoff, cudaStream_t st);
void launch_plain_digits(const MatView &X, int side, int64_t lines, int64_t k, int L, int D, int DP, int W,
                         int want_sum, const int32_t *E, int32_t *lossy, int32_t *digits, cudaStream_t st);
void launch_group_table(const GroupTableArgs &a, cudaStream_t st);
void launch_slicegemm_mma(const SliceGemmArgs &a, cudaStream_t st);
// tile: kTileSingle (one CTA per 128 x 256 tile, two TMEM accumulators), kTile2Sm (CTA
// pairs running one cta_group::2 MMA of M = 256, N = 256), kTile2SmNarrow (the same with
// N = 128, four TMEM accumulators per CTA) or kTileNarrow (one CTA per 128 x 128 tile,
// four TMEM accumulators); wait_limit: cycles a barrier wait may take (0: the
// default of about 2 s), a positive limit makes the waits poll so that it is exact
enum { kTileSingle = 0, kTile2Sm = 1, kTileNarrow = 2, kTile2SmNarrow = 3 };
cudaError_t launch_slicegemm_tc(const SliceGemmArgs &a, cudaStream_t st, int tile, long long wait_limit = 0);
cudaError_t launch_slicegemm_tc_batch(const SliceGemmArgs *list, int count, cudaStream_t st, int tile,
                                      long long wait_limit = 0);
void launch_oz_accum(const AccumArgs &a, const OutView &C, cudaStream_t st);
void launch_fallback(const FallbackArgs &f, const MatView &A, const MatView &B, const OutView &C, int blocks,
                     int threads, cudaStream_t st);
void launch_plain_gemm(const PlainGemmArgs &a, cudaStream_t st);
void launch_plain_combine(const PlainCombineArgs &a, const OutView &C, cudaStream_t st);
void launch_zero_output(const OutView &C, int64_t m, int64_t n, int L, cudaStream_t st);
// residual split: B's format planes copied K-major (n lines of k), the split of one operand's
// lines, the table and bounds, and one batch of the accumulation
void launch_transpose_operand(const MatView &B, int64_t k, int64_t n, int L, uint8_t *sign, int32_t *exp,
                              uint64_t *limb, cudaStream_t st);
void launch_resid_split(const MatView &X, int64_t lines, int64_t k, int64_t kpad, int L, int s, int w,
                        __nv_bfloat16 *digits, int32_t *units, int32_t *lossy, int32_t *flags, int32_t *irregular,
                        int32_t *status, cudaStream_t st);
void launch_resid_table(const ResidTableArgs &a, cudaStream_t st);
void launch_resid_accum(const ResidAccumArgs &a, const OutView &C, cudaStream_t st);

}  // namespace mpc
