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
  const GroupEntry *groups;     // group table (n_entries)
  int32_t n_entries;
  ProductDesc prod[4];
  int32_t *out;                 // group sums: [entry][m][n] int32
  int32_t *status;
};

struct AccumArgs {
  const int32_t *planes;        // group sums [entry][m][n]
  const GroupEntry *groups;
  const int32_t *order;         // groups by descending level
  int32_t n_entries;
  int64_t m, n, k;
  int p, L, Q, nslot, method;
  const int32_t *E, *F, *lossyA, *lossyB;
  int bound_shift;
  uint64_t bound_drop[2], bound_lossy_a[2], bound_lossy_b[2];
  int64_t *fallback;            // list of (i*n + j)*2 + c
  int64_t fallback_cap;
  int32_t *status;
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

struct PlainArgs {
  const uint64_t *fixA, *fixB;  // [c][limb][line][k]
  const uint8_t *sgnA, *sgnB;   // [c][line][k]
  int64_t m, n, k;
  int p, L, Lp;
  const int32_t *E, *F, *lossyA, *lossyB;
  int64_t *fallback;
  int64_t fallback_cap;
  int32_t *status;
};

void launch_init(int32_t *status, int32_t *E, int64_t m, int32_t *F, int64_t n, int32_t *lossyA, int32_t *lossyB,
                 cudaStream_t st);
void launch_line_max(const MatView &A, const MatView &B, int64_t m, int64_t n, int64_t k, int L, int32_t *E,
                     int32_t *F, cudaStream_t st);
void launch_oz_digits(const MatView &X, int side, int64_t lines, int64_t k, int64_t kpad, int L, int s,
                      int want_sum, const int32_t *E, int32_t *lossy, __nv_bfloat16 *digits, cudaStream_t st);
void launch_plain_fix(const MatView &X, int side, int64_t lines, int64_t k, int L, int Lp, const int32_t *E,
                      int32_t *lossy, uint64_t *fix, uint8_t *fsign, cudaStream_t st);
void launch_group_table(const ProductDesc *prods, int n_products, int Q, int gmax, GroupEntry *table,
                        int32_t *order, cudaStream_t st);
void launch_slicegemm_mma(const SliceGemmArgs &a, cudaStream_t st);
cudaError_t launch_slicegemm_tc(const SliceGemmArgs &a, cudaStream_t st, int cluster);
cudaError_t launch_slicegemm_tc_batch(const SliceGemmArgs *list, int count, cudaStream_t st, int cluster);
void launch_oz_accum(const AccumArgs &a, const OutView &C, cudaStream_t st);
void launch_fallback(const FallbackArgs &f, const MatView &A, const MatView &B, const OutView &C, int blocks,
                     int threads, cudaStream_t st);
void launch_plain_gemm(const PlainArgs &a, const OutView &C, cudaStream_t st);
void launch_zero_output(const OutView &C, int64_t m, int64_t n, int L, cudaStream_t st);

}  // namespace mpc
