// oz_slicegemm on the 5th-generation tensor cores (tcgen05, sm_103a):
// the slice products C_ab := A_a B_b of Alg. 2 (Kouya, Sec. III-C), summed
// over the pairs of one group, exactly.
//
// Work unit = (group g, output tile).  Its GEMM runs over the concatenated
// inner dimension K' = count * kpad: for pair (t, q - t) the digit planes
// D^A_t (rows of A) and D^B_{q-t} (columns of B, K-major).
//
// Two variants, both persistent (one CTA, or one CTA pair, per SM or SM
// pair), warp-specialised, 320 threads per CTA:
//   * single CTA: a unit is one 128 x 256 tile;
//   * 2-SM: a cluster of two CTAs runs a unit of two vertically adjacent
//     128 x 256 tiles as one tcgen05.mma.cta_group::2 of M = 256.  Each CTA
//     loads its own 128 rows of A and its half of the 256-row B tile (plain
//     TMA loads, no multicast: the tensor cores read the peer's half from the
//     peer's shared memory), so an SM fetches 32 KB per k-block instead of
//     48 KB and a 7-stage ring fits.
// Units are handed out dynamically (a global counter): the producer (of the
// leader CTA) takes the next unit index and publishes it to the MMA and
// epilogue warps (of both CTAs) through a 4-slot shared ring, so the units in
// flight on all SMs stay a contiguous window of the unit order (group-major,
// groups of equal pair count next to each other, so that the units in flight
// take equally long and stay in step) and share the same digit planes in L2.
//   warp 0      TMA producer: 64-element k-blocks of A and B into the
//               shared-memory ring (128-byte swizzle).
//   warp 1      TMEM owner (512 columns) and, on one lane (of the leader),
//               the MMA issuer: bf16 x bf16 -> fp32 into one of two 256-column
//               TMEM accumulators.
//   warps 2..9  epilogue: every chunk of inner elements (4 k-blocks for 9-bit
//               digits: 256 2^16 <= 2^24; 15 for 8-bit: 960 2^14 < 2^24) the
//               accumulator holds an exact integer; it is read with
//               tcgen05.ld, converted exactly to int32 and added to int32
//               registers (the group bound keeps every sum below 2^31).
//               The two TMEM buffers let the MMA fill one while the other
//               drains.  At the end of a unit the int32 tile is stored.
// Every mbarrier wait is bounded (a per-call cycle limit): on a timeout the
// kernel records it in the status block, lets in-flight copies and MMAs land,
// frees TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>
#include <mutex>

#include "common.cuh"
#include "kernels.h"

namespace mpc {

namespace {

constexpr int BM = 128, BK = 64;

// A variant: one CTA or a CTA pair (TWO) per unit, unit tiles of BM x BNT per CTA.
// The TMEM's 512 columns hold NBUF = 512 / BNT fp32 accumulators; the stage ring fills
// the shared memory (227 KB).
template <bool TWO, int BNT>
struct TcCfg {
  static constexpr int kPair = TWO ? 2 : 1;                  // CTAs per unit
  static constexpr int BN = BNT;
  static constexpr int B_ROWS = TWO ? BNT / 2 : BNT;        // B rows in this CTA's shared memory
  static constexpr int A_BYTES = BM * BK * 2, B_BYTES = B_ROWS * BK * 2, STAGE_BYTES = A_BYTES + B_BYTES;
  static constexpr int STAGES = (227 * 1024 - 1024 - 512) / STAGE_BYTES;   // 4 (48 KB stages) or 7 (32 KB)
  static constexpr int NBUF = 512 / BNT;
  static constexpr size_t SMEM = 1024 + (size_t)STAGES * STAGE_BYTES + 512;
};
constexpr int EPI_WARPS = 8;   // 16 warps of 64 columns measured slower (more spills, no faster drain)
constexpr uint32_t TMEM_COLS = 512;
constexpr long long kDefaultWaitCycles = 4000000000ll;   // ~2 s at 2 GHz
constexpr int URING = 4;                                   // unit-index ring slots
constexpr int kMaxBatch = 64;                              // problems per launch (kernel parameter space)

// One launch serves a set of up to kMaxBatch independent problems (a single
// GEMM is a set of one): their units are numbered consecutively and each
// problem brings its own tensor maps, group table and output planes.
struct TcProblem {
  int64_t m, n;        // the GEMM the units tile (a transposed problem: n and m of C)
  int64_t unit0;       // first unit of this problem
  int tr;              // nonzero: C^T = B^T A^T is computed (A-side operand: B's digits) and
                       // stored transposed, so the output planes keep C's layout
  int kbpp;            // k-blocks per pair (kpad / 64)
  int tiles_m, tiles_n;
  int chunk_kb;        // k-blocks per exact fp32 chunk (4 for 9-bit digits, 15 for 8-bit)
  const GroupEntry *groups;
  const int32_t *sched;   // unit order over the groups (null: table order)
  int32_t *out;
  ProductDesc prod[4];
};

struct TcMaps {
  CUtensorMap a[kMaxBatch];
  CUtensorMap b[kMaxBatch];
};

struct TcParams {
  int count;
  int poll;               // nonzero: waits poll (mbarrier.test_wait) so that wait_limit is exact
  int64_t units;
  long long wait_limit;   // cycles a barrier wait may take before the kernel gives up
  int32_t *status;
  TcProblem prob[kMaxBatch];
};

static_assert(sizeof(TcMaps) + sizeof(TcParams) <= 32764, "kernel parameters must fit the 32 KB parameter space");

// the problem whose units include unit u (binary search over the problems' first units)
__device__ __forceinline__ int problem_of(const TcParams &P, int64_t u) {
  int lo = 0, hi = P.count - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (P.prob[mid].unit0 <= u) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// What a bounded wait needs: the CTA's abort flag, the status block and the limit.
struct Waits {
  volatile int *abort;
  int32_t *status;
  long long limit;
  bool poll;
};

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// one probe of phase `parity`: try_wait may suspend for a while, test_wait returns at once
template <bool CLUSTER>
__device__ __forceinline__ bool mbar_probe(uint64_t *bar, uint32_t parity, bool poll) {
  uint32_t ok;
  if (poll) {
    if (CLUSTER)
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.test_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
          " selp.u32 %0, 1, 0, p;\n}"
          : "=r"(ok)
          : "r"(smem_u32(bar)), "r"(parity)
          : "memory");
    else
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
          : "=r"(ok)
          : "r"(smem_u32(bar)), "r"(parity)
          : "memory");
  } else {
    if (CLUSTER)
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
          " selp.u32 %0, 1, 0, p;\n}"
          : "=r"(ok)
          : "r"(smem_u32(bar)), "r"(parity)
          : "memory");
    else
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
          : "=r"(ok)
          : "r"(smem_u32(bar)), "r"(parity)
          : "memory");
  }
  return ok != 0;
}

// Bounded wait; false on abort (another role gave up) or timeout (sets abort + status).
// CLUSTER: acquire at cluster scope (the phase may have been completed by the peer CTA).
template <bool CLUSTER = false>
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, const Waits &w) {
  const long long t0 = clock64();
  while (!mbar_probe<CLUSTER>(bar, parity, w.poll)) {
    if (*w.abort) return false;
    if (clock64() - t0 > w.limit) {
      *w.abort = 1;
      atomicOr(reinterpret_cast<int *>(w.status) + kStTimeout, 1);
      return false;
    }
  }
  return true;
}

// short bounded wait used only while shutting down after an abort
__device__ __forceinline__ void mbar_drain(uint64_t *bar, uint32_t parity) {
  const long long t0 = clock64();
  while (!mbar_probe<false>(bar, parity, false) && clock64() - t0 < 2000000ll) {
  }
}

__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

// TMA load into this CTA's shared memory whose completion is signalled on a barrier that
// may sit in the peer CTA of the pair (shared::cluster address); no multicast.
__device__ __forceinline__ void tma_load_3d_pair(void *dst, const CUtensorMap *map, int c0, int c1, int c2,
                                                 uint32_t bar_cluster) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
      "[%0], [%1, {%3, %4, %5}], [%2];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(bar_cluster), "r"(c0), "r"(c1), "r"(c2)
      : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;\n barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// shared::cluster address of the same shared-memory location in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t mapa(uint32_t addr, uint32_t rank) {
  uint32_t r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
  return r;
}

__device__ __forceinline__ void st_cluster_u32(uint32_t addr, uint32_t v) {
  asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// Arrive without release semantics: only for a signal that publishes no memory writes
// (the peer's epilogue handing back a TMEM buffer whose reads tcgen05.wait::ld has
// already completed).  The release form waits on the order of a thousand cycles per
// call, longer than the epilogue spends draining a chunk.
__device__ __forceinline__ void mbar_arrive_cluster_relaxed(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.relaxed.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128-byte swizzle, 8-row atoms 1024 B apart.
__device__ __forceinline__ uint64_t smem_desc(const void *p) {
  const uint64_t addr = smem_u32(p);
  uint64_t d = 0;
  d |= (addr >> 4) & 0x3FFFull;            // start address
  d |= (uint64_t)1 << 16;                  // leading byte offset (unused with 128B swizzle), 16 B
  d |= (uint64_t)(1024 >> 4) << 32;        // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1 << 46;                  // descriptor version for tcgen05
  d |= (uint64_t)2 << 61;                  // swizzle mode: 128 B
  return d;
}

// Instruction descriptor, kind::f16: D fp32, A = B = bf16, both K-major, N = BNT, M = 128 (one
// CTA) or 256 (a CTA pair: the leader's 128 rows in its TMEM, the peer's in the peer's TMEM).
template <bool TWO, int BNT>
__host__ __device__ constexpr uint32_t idesc() {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BNT >> 3) << 17) | ((uint32_t)((TWO ? 2 : 1) * BM >> 4) << 24);
}

template <bool TWO, int BNT>
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate) {
  if (TWO)
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc<true, BNT>()), "r"(accumulate));
  else
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc<false, BNT>()), "r"(accumulate));
}

// Arrive on `bar` once the MMAs issued so far complete.  The CTA pair's commit arrives on
// the barrier at this offset in both CTAs (an arrive signal, not a data copy).
template <bool TWO>
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  if (TWO)
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"((uint16_t)0x3)
        : "memory");
  else
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

struct Unit {
  GroupEntry g;
  ProductDesc pd;
  int tm, tn, nkb;
  int e;
  int prob;
};

// unit u -> (group, tile); for CTA pairs a unit is a pair of row tiles, CTA `rank` takes one
template <bool TWO>
__device__ __forceinline__ Unit decode(const TcParams &P, int64_t u, uint32_t rank) {
  constexpr int CP = TWO ? 2 : 1;
  Unit x;
  const int pi = problem_of(P, u);
  const TcProblem &q = P.prob[pi];
  const int64_t r = u - q.unit0;
  const int tiles_mu = (q.tiles_m + CP - 1) / CP;
  const int tiles = tiles_mu * q.tiles_n;
  x.prob = pi;
  x.e = q.sched ? q.sched[r / tiles] : (int)(r / tiles);
  const int t = (int)(r % tiles);
  x.tm = (t / q.tiles_n) * CP + (int)rank;
  x.tn = t % q.tiles_n;
  x.g = q.groups[x.e];
  x.pd = q.prod[x.g.prod];
  x.nkb = x.g.count * q.kbpp;
  return x;
}

// the group of unit u has no pairs left (all its digit planes were zero)
template <bool TWO>
__device__ __forceinline__ bool unit_empty(const TcParams &P, int64_t u) {
  const TcProblem &q = P.prob[problem_of(P, u)];
  const int64_t r = u - q.unit0;
  const int tiles = ((q.tiles_m + (TWO ? 1 : 0)) / (TWO ? 2 : 1)) * q.tiles_n;
  const int e = q.sched ? q.sched[r / tiles] : (int)(r / tiles);
  return q.groups[e].count == 0;
}

}  // namespace

// TWO = false: one CTA per 128 x 256 unit tile.  TWO = true: a cluster of two
// CTAs computes the two vertically adjacent tiles of one unit with one
// cta_group::2 MMA of M = 256 issued by the leader (rank 0); each CTA's TMA
// loads (its 128 A rows and its half of B) complete on the leader's stage
// barrier, TMEM is allocated and freed by both CTAs together, the leader's MMA
// commits arrive on both CTAs' barriers, and both CTAs' epilogues hand each
// drained TMEM buffer back on the leader's barrier.  The leader hands out the
// unit indices to both CTAs through distributed shared memory.
template <bool TWO, int BNT>
__global__ void __launch_bounds__(64 + 32 * EPI_WARPS, 1)
    k_slicegemm_tc(const __grid_constant__ TcMaps maps, const __grid_constant__ TcParams P) {
  using C = TcCfg<TWO, BNT>;
  constexpr int BN = BNT, NBUF = C::NBUF;
  constexpr int COLS = 4 * BN / EPI_WARPS;    // accumulator columns per epilogue thread (one TMEM lane)
  constexpr int STAGES = C::STAGES, A_BYTES = C::A_BYTES, B_BYTES = C::B_BYTES, STAGE_BYTES = C::STAGE_BYTES;
  extern __shared__ uint8_t smem_raw[];
  uint8_t *smem = smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023);
  uint8_t *sA = smem;
  uint8_t *sB = smem + STAGES * A_BYTES;
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + STAGES * STAGE_BYTES);
  uint64_t *empty = full + STAGES;
  uint64_t *tfull = empty + STAGES;
  uint64_t *tempty = tfull + NBUF;
  uint64_t *ufull = tempty + NBUF;
  uint64_t *uempty = ufull + URING;
  uint64_t *mdone = uempty + URING;   // the MMA issuer's last commit: every MMA has completed
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(mdone + 1);
  volatile int *abort = reinterpret_cast<volatile int *>(tmem_slot + 1);
  volatile int *uring = reinterpret_cast<volatile int *>(tmem_slot + 2);
  const Waits W{abort, P.status, P.wait_limit, P.poll != 0};

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = TWO ? cluster_rank() : 0u;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);   // one (for the pair: multicast) MMA commit
    }
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], TWO ? 2 * EPI_WARPS : EPI_WARPS);   // pair: both CTAs drain the leader's MMA
    }
    for (int r = 0; r < URING; ++r) {
      mbar_init(&ufull[r], 1);
      mbar_init(&uempty[r], TWO ? 2 * (1 + EPI_WARPS) + 1 : 1 + EPI_WARPS);
    }
    mbar_init(mdone, 1);
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (int q = 0; q < P.count; ++q) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.a[q])) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.b[q])) : "memory");
    }
  }
  if (warp == 1) {
    if (TWO) {   // one warp of each CTA of the pair allocates, collectively
      asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
    } else {
      asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                   "r"(TMEM_COLS)
                   : "memory");
      asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
  }
  tc_fence_before();
  if (TWO) cluster_sync();   // every barrier of both CTAs initialised before any remote use
  else __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;
  // the unit ring is filled by the leader (rank 0); everyone releases slots on the leader's barrier
  const uint32_t uempty_leader = TWO ? mapa(smem_u32(uempty), 0) : smem_u32(uempty);
  auto release_slot = [&](int slot) {
    if (TWO) mbar_arrive_cluster(uempty_leader + 8u * (uint32_t)slot);
    else mbar_arrive(&uempty[slot]);
  };

  if (warp == 0) {
    if (lane == 0) {
      // ---------------- TMA producer
      int stage = 0, slot = 0;
      uint32_t phase = 0, uphase = 0;
      bool ok = true;
      int *counter = reinterpret_cast<int *>(P.status) + kStUnitCounter;
      while (ok) {
        int u;
        if (rank == 0) {
          if (!mbar_wait(&uempty[slot], uphase ^ 1, W)) { ok = false; break; }
          int64_t v = atomicAdd(counter, 1);
          while (v < P.units && unit_empty<TWO>(P, v)) v = atomicAdd(counter, 1);   // groups of zero pairs
          u = v >= P.units ? -1 : (int)v;
          uring[slot] = u;
          mbar_arrive(&ufull[slot]);
          if (TWO) {
            st_cluster_u32(mapa(smem_u32((const void *)&uring[slot]), 1), (uint32_t)u);
            mbar_arrive_cluster(mapa(smem_u32(&ufull[slot]), 1));
          }
        } else {
          if (!mbar_wait<true>(&ufull[slot], uphase, W)) { ok = false; break; }
          u = uring[slot];
          release_slot(slot);
        }
        if (++slot == URING) { slot = 0; uphase ^= 1; }
        if (u < 0) break;
        const Unit x = decode<TWO>(P, u, rank);
        const int kbpp = P.prob[x.prob].kbpp;
        const CUtensorMap *tmA = &maps.a[x.prob], *tmB = &maps.b[x.prob];
        for (int kb = 0; kb < x.nkb; ++kb) {
          const int pi = kb / kbpp;
          const int k0 = (kb - pi * kbpp) * BK;
          int t = x.g.t0 + pi, uu = x.g.q - t;   // digit positions of A and of B
          if (P.prob[x.prob].tr) {                // the A side carries B's digits
            const int sw = t;
            t = uu;
            uu = sw;
          }
          const int planeA = x.pd.a_plane0 + t - x.pd.a_pos0;
          const int planeB = x.pd.b_plane0 + uu - x.pd.b_pos0;
          if (!mbar_wait(&empty[stage], phase ^ 1, W)) { ok = false; break; }
          if (TWO) {   // both CTAs' copies complete on the leader's stage barrier
            const uint32_t fb = mapa(smem_u32(&full[stage]), 0);
            if (rank == 0) mbar_expect_tx(&full[stage], 2 * STAGE_BYTES);
            tma_load_3d_pair(sA + stage * A_BYTES, tmA, k0, x.tm * BM, planeA, fb);
            tma_load_3d_pair(sB + stage * B_BYTES, tmB, k0, x.tn * BN + (int)rank * (BN / 2), planeB, fb);
          } else {
            mbar_expect_tx(&full[stage], STAGE_BYTES);
            tma_load_3d(sA + stage * A_BYTES, tmA, k0, x.tm * BM, planeA, &full[stage]);
            tma_load_3d(sB + stage * B_BYTES, tmB, k0, x.tn * BN, planeB, &full[stage]);
          }
          if (++stage == STAGES) { stage = 0; phase ^= 1; }
        }
      }
      if (!ok) {   // let copies still in flight land before the CTA exits
        for (int s = 0; s < STAGES; ++s) {
          mbar_drain(&full[s], 0);
          mbar_drain(&full[s], 1);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0 && rank == 0) {
      // ---------------- MMA issuer (for the pair: the leader's, M = 256 across both CTAs)
      int stage = 0, buf = 0, slot = 0;
      uint32_t phase = 0, tphase = 0, uphase = 0;
      bool ok = true;
      while (ok) {
        if (!mbar_wait<TWO>(&ufull[slot], uphase, W)) { ok = false; break; }
        const int u = uring[slot];
        release_slot(slot);
        if (++slot == URING) { slot = 0; uphase ^= 1; }
        if (u < 0) break;
        const Unit x = decode<TWO>(P, u, rank);
        const int ck = P.prob[x.prob].chunk_kb;
        for (int c0 = 0; c0 < x.nkb && ok; c0 += ck) {
          const int cend = min(x.nkb, c0 + ck);
          // the epilogue (both CTAs' epilogues) has drained this accumulator
          if (!mbar_wait<TWO>(&tempty[buf], tphase ^ 1, W)) { ok = false; break; }
          tc_fence_after();
          const uint32_t d_tmem = tmem_base + (uint32_t)(buf * BN);
          for (int kb = c0; kb < cend; ++kb) {
            // the stage has landed (for the pair: both CTAs' halves; the peer's copies signal here too)
            if (!mbar_wait<TWO>(&full[stage], phase, W)) { ok = false; break; }
            tc_fence_after();
            const uint64_t ad = smem_desc(sA + stage * A_BYTES);
            const uint64_t bd = smem_desc(sB + stage * B_BYTES);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)   // K = 16 per instruction: +32 B in the swizzled row
              mma_f16<TWO, BNT>(d_tmem, ad + (uint64_t)(2 * kk), bd + (uint64_t)(2 * kk), (kb > c0 || kk > 0) ? 1u : 0u);
            mma_commit<TWO>(&empty[stage]);   // the producer(s) may refill the stage
            if (++stage == STAGES) { stage = 0; phase ^= 1; }
          }
          if (!ok) break;
          mma_commit<TWO>(&tfull[buf]);       // the epilogue(s) may drain
          if (++buf == NBUF) { buf = 0; tphase ^= 1; }
        }
      }
      // Whether it finished or gave up: every MMA issued must complete before TMEM is freed
      // (after an abort the epilogue may no longer be waiting for the last chunk).
      mma_commit<TWO>(mdone);
      mbar_drain(mdone, 0);
    } else if (TWO && lane == 0) {
      // ---------------- the peer's warp 1: no MMA to issue; only takes its turn on the unit ring
      int slot = 0;
      uint32_t uphase = 0;
      while (true) {
        if (!mbar_wait<true>(&ufull[slot], uphase, W)) break;
        const int u = uring[slot];
        release_slot(slot);
        if (++slot == URING) { slot = 0; uphase ^= 1; }
        if (u < 0) break;
      }
    }
  } else {
    // ---------------- epilogue: warps 2..9
    const int quad = warp & 3;                 // TMEM lanes 32*quad .. +31 (hardware rule: warp id % 4)
    const int part = (warp - 2) >> 2;          // columns part*COLS .. +COLS-1
    const int row_in_tile = quad * 32 + lane;
    int buf = 0, slot = 0;
    uint32_t tphase = 0, uphase = 0;
    bool ok = true;
    int32_t acc[COLS];
#pragma unroll
    for (int x = 0; x < COLS; ++x) acc[x] = 0;
    while (ok) {
      if (!mbar_wait<TWO>(&ufull[slot], uphase, W)) { ok = false; break; }
      const int u = uring[slot];
      __syncwarp();
      if (lane == 0) release_slot(slot);
      if (++slot == URING) { slot = 0; uphase ^= 1; }
      if (u < 0) break;
      const Unit x = decode<TWO>(P, u, rank);
      const int ck = P.prob[x.prob].chunk_kb;
      for (int c0 = 0; c0 < x.nkb; c0 += ck) {
        if (!mbar_wait(&tfull[buf], tphase, W)) { ok = false; break; }
        tc_fence_after();
        const uint32_t taddr = tmem_base + ((uint32_t)(quad * 32) << 16) + (uint32_t)(buf * BN + part * COLS);
#pragma unroll
        for (int j = 0; j < COLS / 32; ++j) {
          uint32_t r[32];
          tmem_ld32(taddr + (uint32_t)(j * 32), r);
#pragma unroll
          for (int y = 0; y < 32; ++y) acc[j * 32 + y] += __float2int_rn(__uint_as_float(r[y]));
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {   // pair: the peer's warps release the buffer on the leader's barrier
          if (TWO && rank == 1) mbar_arrive_cluster_relaxed(mapa(smem_u32(&tempty[buf]), 0));
          else mbar_arrive(&tempty[buf]);
        }
        if (++buf == NBUF) { buf = 0; tphase ^= 1; }
      }
      if (!ok) break;
      // store the int32 tile rows of this thread
      const int64_t pm = P.prob[x.prob].m, pn = P.prob[x.prob].n;
      const int64_t row = (int64_t)x.tm * BM + row_in_tile;
      const int64_t col0 = (int64_t)x.tn * BN + part * COLS;
      if (P.prob[x.prob].tr) {   // tile row = column `row` of C, tile columns = rows of C
        if (row < pm) {
          int32_t *dst = P.prob[x.prob].out + (int64_t)x.e * pm * pn + row;
#pragma unroll
          for (int v = 0; v < COLS; ++v)   // a warp writes 32 consecutive columns of one row
            if (col0 + v < pn) dst[(col0 + v) * pm] = acc[v];
        }
      } else if (row < pm) {
        int32_t *dst = P.prob[x.prob].out + (int64_t)x.e * pm * pn + row * pn + col0;
        if (col0 + COLS <= pn && ((pn & 3) == 0)) {
#pragma unroll
          for (int v = 0; v < COLS / 4; ++v)
            reinterpret_cast<int4 *>(dst)[v] = make_int4(acc[4 * v], acc[4 * v + 1], acc[4 * v + 2], acc[4 * v + 3]);
        } else {
#pragma unroll
          for (int v = 0; v < COLS; ++v)
            if (col0 + v < pn) dst[v] = acc[v];
        }
      }
#pragma unroll
      for (int v = 0; v < COLS; ++v) acc[v] = 0;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (TWO) cluster_sync();   // the leader's MMAs into the peer's TMEM are all drained
  if (warp == 1) {
    tc_fence_after();
    __syncwarp();
    if (TWO)
      asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                   : "memory");
    else
      asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(TMEM_COLS)
                   : "memory");
  }
  if (TWO) cluster_sync();   // neither CTA leaves while its peer may still signal it
}

// ------------------------------------------------------------------ host side

namespace {

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

bool make_map(CUtensorMap *map, const void *base, int64_t rows, int64_t kpad, int64_t planes, int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[3] = {(cuuint64_t)kpad, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)kpad * 2, (cuuint64_t)rows * kpad * 2};
  cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
  }
  return sms;
}

}  // namespace

// One persistent launch over the units of up to kMaxBatch problems (the unit
// counter lives in the first problem's status block, zeroed by its init).
template <bool TWO, int BNT>
static cudaError_t launch_set(const SliceGemmArgs *list, int count, cudaStream_t st, long long wait_limit) {
  using C = TcCfg<TWO, BNT>;
  static TcMaps maps;    // host staging of the kernel parameters (copied at launch)
  static TcParams P;
  std::memset(&P, 0, sizeof(P));
  constexpr int pair = C::kPair;   // CTAs per unit
  int64_t units = 0;
  for (int q = 0; q < count; ++q) {
    const SliceGemmArgs &a = list[q];
    int planes_a = 0, planes_b = 0;
    for (int x = 0; x < 4; ++x) {
      if (a.prod[x].a_plane0 + a.prod[x].a_npos > planes_a) planes_a = a.prod[x].a_plane0 + a.prod[x].a_npos;
      if (a.prod[x].b_plane0 + a.prod[x].b_npos > planes_b) planes_b = a.prod[x].b_plane0 + a.prod[x].b_npos;
    }
    // Orientation: the side that pads less under the 128-row tiles becomes the row side
    // (C^T = B^T A^T computed and stored transposed).  CTA pairs keep C's orientation.
    auto padded = [](int64_t r, int64_t c) {
      return ((r + BM - 1) / BM) * BM * (((c + BNT - 1) / BNT) * BNT);
    };
    const bool tr = !TWO && padded(a.n, a.m) < padded(a.m, a.n);
    if (tr ? (!make_map(&maps.a[q], a.dB, a.n, a.kpad, planes_b, BM) ||
              !make_map(&maps.b[q], a.dA, a.m, a.kpad, planes_a, C::B_ROWS))
           : (!make_map(&maps.a[q], a.dA, a.m, a.kpad, planes_a, BM) ||
              !make_map(&maps.b[q], a.dB, a.n, a.kpad, planes_b, C::B_ROWS)))
      return cudaErrorNotSupported;
    TcProblem &t = P.prob[q];
    t.tr = tr ? 1 : 0;
    t.m = tr ? a.n : a.m;
    t.n = tr ? a.m : a.n;
    t.kbpp = (int)(a.kpad / BK);
    t.tiles_m = (int)((t.m + BM - 1) / BM);
    t.tiles_n = (int)((t.n + BNT - 1) / BNT);
    t.chunk_kb = a.chunk_kb;
    t.unit0 = units;
    t.groups = a.groups;
    t.sched = a.sched;
    t.out = a.out;
    for (int x = 0; x < 4; ++x) {
      t.prod[x] = a.prod[x];
      if (tr) {   // the operands' roles swap
        t.prod[x].a_plane0 = a.prod[x].b_plane0;
        t.prod[x].a_pos0 = a.prod[x].b_pos0;
        t.prod[x].a_npos = a.prod[x].b_npos;
        t.prod[x].b_plane0 = a.prod[x].a_plane0;
        t.prod[x].b_pos0 = a.prod[x].a_pos0;
        t.prod[x].b_npos = a.prod[x].a_npos;
      }
    }
    units += (int64_t)a.n_entries * ((t.tiles_m + pair - 1) / pair) * t.tiles_n;
  }
  P.count = count;
  P.units = units;
  P.status = list[0].status;
  P.poll = wait_limit > 0;
  P.wait_limit = wait_limit > 0 ? wait_limit : kDefaultWaitCycles;
  if (units == 0) return cudaSuccess;
  static bool attr = false;   // one per instantiation
  auto kfn = k_slicegemm_tc<TWO, BNT>;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  cudaLaunchConfig_t cfg = {};
  cudaLaunchAttribute la[1];
  cfg.blockDim = dim3(64 + 32 * EPI_WARPS, 1, 1);
  cfg.dynamicSmemBytes = C::SMEM;
  cfg.stream = st;
  int ctas = num_sms();
  if (TWO) {
    la[0].id = cudaLaunchAttributeClusterDimension;
    la[0].val.clusterDim.x = 2;
    la[0].val.clusterDim.y = 1;
    la[0].val.clusterDim.z = 1;
    cfg.attrs = la;
    cfg.numAttrs = 1;
    cfg.gridDim = dim3((unsigned)ctas, 1, 1);
    static int clusters = 0;   // queried once (also keeps graph capture query-free)
    if (clusters == 0 && (cudaOccupancyMaxActiveClusters(&clusters, kfn, &cfg) != cudaSuccess || clusters < 1))
      clusters = ctas / 2;
    ctas = 2 * clusters;
  }
  const int64_t need = units * pair;
  if (need < ctas) ctas = (int)need;
  cfg.gridDim = dim3((unsigned)ctas, 1, 1);
  return cudaLaunchKernelEx(&cfg, kfn, maps, P);
}

cudaError_t launch_slicegemm_tc_batch(const SliceGemmArgs *list, int count, cudaStream_t st, int tile,
                                      long long wait_limit) {
  int dev = 0, major = 0, minor = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
  cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
  if (major != 10 || minor != 3) return cudaErrorNotSupported;   // built for sm_103a only
  static std::mutex mu;            // the parameter staging below is shared
  std::lock_guard<std::mutex> lock(mu);
  for (int q0 = 0; q0 < count; q0 += kMaxBatch) {
    const int c = count - q0 < kMaxBatch ? count - q0 : kMaxBatch;
    const cudaError_t e = tile == kTile2Sm         ? launch_set<true, 256>(list + q0, c, st, wait_limit)
                          : tile == kTile2SmNarrow ? launch_set<true, 128>(list + q0, c, st, wait_limit)
                          : tile == kTileNarrow    ? launch_set<false, 128>(list + q0, c, st, wait_limit)
                                                : launch_set<false, 256>(list + q0, c, st, wait_limit);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_slicegemm_tc(const SliceGemmArgs &a, cudaStream_t st, int tile, long long wait_limit) {
  return launch_slicegemm_tc_batch(&a, 1, st, tile, wait_limit);
}

}  // namespace mpc
