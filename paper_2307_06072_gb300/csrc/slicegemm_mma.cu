// oz_slicegemm, warp-level mma.sync form (the second half of Alg. 2:
// C_ab := A_a B_b over the kept pair triangle).
//
// One CTA computes one 128 x 128 tile of one group sum
//     G_g = sum_{(t,u) in g} D^A_t (D^B_u)^T,
// i.e. one GEMM over the concatenated inner dimension K' = count * kpad.
// Operands are integer digits |d| <= 2^(w-1) (w = 9 or 8) carried in bf16;
// products (<= 2^(2w-2)) are exact and the fp32 accumulators stay exact over a
// chunk of inner elements (256 for w = 9, 960 for w = 8), after which the fp32
// tile is converted to int32 and added to int32 registers (the group bound
// keeps every partial sum below 2^31).  This kernel is kept as an independent
// second implementation of the tcgen05 kernel's contract.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.h"

namespace mpc {

namespace {
constexpr int MT = 128, NT = 128, KT = 32, LDS = 40;   // LDS: smem row stride (bf16), 80 B
static_assert((64 % KT) == 0, "a k-block must be whole k steps");

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
  uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }

__device__ __forceinline__ void ldmatrix_x4(uint32_t &r0, uint32_t &r1, uint32_t &r2, uint32_t &r3,
                                            const void *p) {
  uint32_t s = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(s));
}

__device__ __forceinline__ void mma_bf16_16816(float *d, const uint32_t *a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
}  // namespace

__global__ void __launch_bounds__(256) k_slicegemm_mma(SliceGemmArgs a, int tiles_m, int tiles_n) {
  __shared__ __align__(128) __nv_bfloat16 sA[2][MT * LDS];
  __shared__ __align__(128) __nv_bfloat16 sB[2][NT * LDS];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 2, wn = warp & 3;   // 2 (M) x 4 (N) warps, warp tile 64 x 32
  const int tiles = tiles_m * tiles_n;
  const int e = (int)(blockIdx.x / tiles);
  const int tile = (int)(blockIdx.x % tiles);
  const int64_t m0 = (int64_t)(tile / tiles_n) * MT, n0 = (int64_t)(tile % tiles_n) * NT;
  const GroupEntry g = a.groups[e];
  if (g.count == 0) return;   // every pair of the group has an all-zero digit plane: nothing to store
  const ProductDesc pd = a.prod[g.prod];
  const int64_t planeA = a.m * a.kpad, planeB = a.n * a.kpad;
  const int steps_per_pair = (int)(a.kpad / KT);
  const int steps_per_chunk = a.chunk_kb * (64 / KT);   // exact fp32 chunk (digit width)
  const int total_steps = g.count * steps_per_pair;

  auto load_stage = [&](int stage, int step) {
    const int pi = step / steps_per_pair;
    const int64_t kk = (int64_t)(step % steps_per_pair) * KT;
    const int t = g.t0 + pi, u = g.q - t;
    const __nv_bfloat16 *pA = a.dA + (int64_t)(pd.a_plane0 + t - pd.a_pos0) * planeA;
    const __nv_bfloat16 *pB = a.dB + (int64_t)(pd.b_plane0 + u - pd.b_pos0) * planeB;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int c = tid + 256 * r, row = c >> 2, c8 = (c & 3) * 8;
      const int64_t gr = m0 + row, gc = n0 + row;
      cp_async16(&sA[stage][row * LDS + c8], pA + (gr < a.m ? gr : 0) * a.kpad + kk + c8, gr < a.m ? 16 : 0);
      cp_async16(&sB[stage][row * LDS + c8], pB + (gc < a.n ? gc : 0) * a.kpad + kk + c8, gc < a.n ? 16 : 0);
    }
  };

  float accf[4][4][4];
  int32_t acci[4][4][4];
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y)
#pragma unroll
      for (int z = 0; z < 4; ++z) {
        accf[x][y][z] = 0.f;
        acci[x][y][z] = 0;
      }

  load_stage(0, 0);
  cp_async_commit();
  for (int step = 0; step < total_steps; ++step) {
    const int stage = step & 1;
    if (step + 1 < total_steps) load_stage(stage ^ 1, step + 1);
    cp_async_commit();
    cp_async_wait1();
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      uint32_t af[4][4], bfr[4][2];
#pragma unroll
      for (int mt = 0; mt < 4; ++mt) {
        const int row = wm * 64 + mt * 16 + (lane & 15);
        const int col = ks * 16 + (lane >> 4) * 8;
        ldmatrix_x4(af[mt][0], af[mt][1], af[mt][2], af[mt][3], &sA[stage][row * LDS + col]);
      }
#pragma unroll
      for (int nt2 = 0; nt2 < 2; ++nt2) {
        const int row = wn * 32 + nt2 * 16 + (lane >> 4) * 8 + (lane & 7);
        const int col = ks * 16 + ((lane >> 3) & 1) * 8;
        ldmatrix_x4(bfr[2 * nt2][0], bfr[2 * nt2][1], bfr[2 * nt2 + 1][0], bfr[2 * nt2 + 1][1],
                    &sB[stage][row * LDS + col]);
      }
#pragma unroll
      for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_bf16_16816(accf[mt][nt], af[mt], bfr[nt][0], bfr[nt][1]);
    }
    __syncthreads();
    if ((step + 1) % steps_per_chunk == 0 || step + 1 == total_steps) {
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y)
#pragma unroll
          for (int z = 0; z < 4; ++z) {
            acci[x][y][z] += __float2int_rn(accf[x][y][z]);
            accf[x][y][z] = 0.f;
          }
    }
  }

  int32_t *out = a.out + (int64_t)e * a.m * a.n;
#pragma unroll
  for (int mt = 0; mt < 4; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int64_t row = m0 + wm * 64 + mt * 16 + (lane >> 2) + 8 * h;
        const int64_t col = n0 + wn * 32 + nt * 8 + (lane & 3) * 2;
        if (row < a.m) {
          if (col < a.n) out[row * a.n + col] = acci[mt][nt][2 * h];
          if (col + 1 < a.n) out[row * a.n + col + 1] = acci[mt][nt][2 * h + 1];
        }
      }
}

void launch_slicegemm_mma(const SliceGemmArgs &a, cudaStream_t st) {
  const int tm = (int)((a.m + MT - 1) / MT), tn = (int)((a.n + NT - 1) / NT);
  const long long blocks = (long long)a.n_entries * tm * tn;
  if (blocks <= 0) return;
  k_slicegemm_mma<<<(unsigned)blocks, 256, 0, st>>>(a, tm, tn);
}

}  // namespace mpc
