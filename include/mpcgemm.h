/*
 * mpcgemm.h -- arbitrary-precision complex matrix multiplication on one
 * NVIDIA GB300 (sm_103a), by the Ozaki scheme under the 4M and 3M complex
 * formulations, or by a plain multi-limb GEMM.
 *
 * The operation (Kouya, "Acceleration of complex matrix multiplication
 * using arbitrary precision floating-point arithmetic", Sec. III-A,
 * Eq. (cmatmul)):  C := A B,  A in C^{m x k}, B in C^{k x n}, every real and
 * imaginary part a p-bit binary floating-point number.  C is the product
 * rounded once, to nearest with ties to even, to p bits per component:
 * the result is the correctly rounded exact product, whatever the algorithm.
 *
 * ------------------------------------------------------------------------
 * Number format (one real component; Sec. II's F_bM, one fixed width):
 *
 *     value = (-1)^sign * M * 2^(exp - 64 L),   L = ceil(p / 64),
 *     M = sum_{j < L} limb_j 2^(64 j)          (limb 0 least significant).
 *
 * A component is ZERO iff its top limb (limb L-1) is 0; sign and exp are then
 * ignored.  A nonzero input is used as given (normalised inputs have bit 63 of
 * limb L-1 set; the kernels only need |value| < 2^exp, which every M with a
 * nonzero top limb satisfies).  Outputs are normalised, have at most p
 * significant bits (the 64L-p low bits of M are 0), and zero is written as
 * sign 0, exp INT32_MIN, M 0.  Exponents are int32; a result whose exponent
 * does not fit makes the call report MPC_ERANGE.
 *
 * Matrix layout (struct mpc_mat): separate real and imaginary planes, each a
 * row-major rows x cols array with leading dimension ld >= cols, element
 * (r, c) at index idx = r*ld + c:
 *     sign[ri][idx]                  uint8   (0 = +, 1 = -)
 *     exp[ri][idx]                   int32
 *     limb[ri][j * rows * ld + idx]  uint64  limb j
 * with ri = 0 for the real and 1 for the imaginary plane.  All pointers
 * are DEVICE pointers owned by the caller; the library never frees or
 * retains them past the call's stream work.
 *
 * ------------------------------------------------------------------------
 * Conventions for every entry point:
 *   * Asynchronous on `stream` (a cudaStream_t passed as void*; NULL = the
 *     legacy default stream).  Returns MPC_OK once the work is enqueued.
 *   * Argument errors are detected on the host before any launch and return
 *     a negative code with nothing enqueued.
 *   * Errors that only the device can see (exponent overflow, a fallback
 *     list overflow) are written to a status block inside the workspace;
 *     read it with mpcgemm_read_status() (which synchronises the stream).
 *   * The library allocates no device memory and no pinned host memory:
 *     all scratch space lives in the caller's `workspace` of `ws_bytes`
 *     bytes (device memory, 256-byte aligned), sized by
 *     mpcgemm_workspace_size().  C must not alias A, B or the workspace.
 *     The one exception is mpcgemm_noalloc(), whose scratch is a static
 *     device array of the library (see there).
 *   * k == 0 gives C = 0; m == 0 or n == 0 is a no-op (the workspace may be
 *     NULL); inside a batched call such a problem's status block is cleared.
 */
#ifndef MPCGEMM_H
#define MPCGEMM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define MPC_OK 0
#define MPC_EINVAL (-22)    /* bad size, precision, pointer, method or parameter */
#define MPC_ENOSPC (-28)    /* workspace too small */
#define MPC_ERANGE (-34)    /* a result exponent does not fit int32 (device-detected) */
#define MPC_ENOTSUP (-95)   /* unsupported on this device (needs sm_103a) */
#define MPC_ECUDA (-1000)   /* a CUDA runtime error e occurred: returns MPC_ECUDA - e */

/* ---- algorithm selection --------------------------------------------- */
enum { MPC_4M = 0, MPC_3M = 1 };          /* Eq. (4m_way) / Eq. (3m_way) */
enum { MPC_PLAIN = 0, MPC_OZAKI = 1 };    /* Eq. (simple_triple_loop) / Alg. 2 */
/* Split of the Ozaki path: one exponent per row / column for both parts (default), or
 * the per-part split of Alg. 2 (4M only; see mpc_oz_params.split). */
enum { MPC_SPLIT_COMMON = 0, MPC_SPLIT_PER_PART = 1, MPC_SPLIT_RESIDUAL = 2 };
/* Slice-GEMM kernels (value 3 is not used and is rejected). */
enum { MPC_KERNEL_AUTO = 0, MPC_KERNEL_TCGEN05 = 1, MPC_KERNEL_MMA_SYNC = 2, MPC_KERNEL_TCGEN05_2SM = 4,
       MPC_KERNEL_TCGEN05_N128 = 5, MPC_KERNEL_TCGEN05_2SM_N128 = 6 };

/* Largest supported precision and inner size. */
#define MPC_MAX_P_BITS 1024
#define MPC_MAX_K 131071

typedef struct mpc_mat {
    int64_t rows, cols, ld;
    uint8_t *sign[2];
    int32_t *exp[2];
    uint64_t *limb[2];
} mpc_mat;

/*
 * Optional tuning of the Ozaki path (Alg. 2's number of divisions d and pair
 * triangle).  Zero-initialise and set what you need; a zeroed struct (or a
 * NULL pointer) means the defaults.
 *   guard_bits  extra fixed-point bits: s = ceil((p + ceil(log2 k) + guard)/w)
 *               slices (0 -> 40).  More guard bits make exact fallbacks rarer.
 *   digit_bits  w, the bits per slice digit: 9 (balanced base-512 digits,
 *               |d| <= 256, exact in bf16, fp32-exact for 256 inner elements)
 *               or 8 (base 256, 960 inner elements); 0 -> 9 when k < 2^15,
 *               else 8 (a group of one pair must fit int32: k 2^(2w-2) < 2^31).
 *   slices      s itself (0 -> the rule above); 1 <= s <= 160.
 *   cut_level   Q + 1, where pairs (t, u) with t + u <= Q are multiplied
 *               (0 -> Q = s - 1, the paper's triangle alpha + beta <= d + 1).
 *   max_group   cap on the slice pairs summed in one group (0 -> the int32 limit
 *               G_max); smaller groups make more, shorter work units.
 *   kernel      MPC_KERNEL_*: which slice-GEMM kernel (auto = TCGEN05, single
 *               CTAs with 128 x 256 tiles and two TMEM accumulators; TCGEN05_N128
 *               single CTAs with 128 x 128 tiles and four; TCGEN05_2SM CTA pairs
 *               that run one 256-row MMA across both SMs, each loading its own
 *               rows of A and half of B, 256 columns (two accumulators per CTA);
 *               TCGEN05_2SM_N128 the same with 128 columns (four accumulators
 *               per CTA); the mma.sync kernel is a second, independent
 *               implementation of the same sums).
 *   wait_limit_cycles
 *               SM clock cycles that one barrier wait of the tcgen05 kernels may
 *               last before the kernel gives up (0 -> about 4e9, some 2 s).  A
 *               positive value makes the waits poll, so that the limit holds to
 *               within a few cycles.  A wait that runs out sets
 *               mpc_status.device_timeout, the kernel lets its copies and MMAs in
 *               flight complete, frees its tensor memory and returns; the results
 *               of that call are then invalid, the device and the library stay
 *               usable.  For tests of that path; leave it 0 otherwise.
 *   dump_accumulators
 *               nonzero: the plan adds a workspace region (mpc_plan.off_acc_dump)
 *               where the accumulation stage writes, for every output component,
 *               its exact accumulator Acc (Alg. 2's L-bit sum of the slice
 *               products, before rounding): acc_slots 32-bit words of |Acc|,
 *               least significant first, then one word holding 1 if Acc < 0,
 *               at index ((i n + j) 2 + c) (acc_slots + 1), c = 0 real, 1
 *               imaginary; its value is Acc 2^(E_i + F_j - (2w - 2) - w Q).
 *               Rows of A or columns of B that are all zero are not written.
 *               For stage checks; leave it 0 otherwise.
 *   split       MPC_SPLIT_COMMON (0): one exponent per row of A / column of B for
 *               both parts, s digits each.  MPC_SPLIT_PER_PART (1, 4M only, else
 *               MPC_EINVAL): Alg. 2 cuts every real part (Re A, Im A, Re B, Im B)
 *               on its own; here part P gets a digit offset z_P, the number of
 *               leading digit positions that are zero in every row (column) of P,
 *               measured on the device, and its s digits sit at positions
 *               z_P .. z_P + s - 1 of the row's grid; each output component c is
 *               cut at level Q_c = Q + z_c (z_c = min over its products of
 *               z_a + z_b, Sec. V item 3: divisions that follow the magnitudes of
 *               the real and imaginary parts).  When one part is smaller than the
 *               other by 2^-D everywhere it keeps all its s digits (the default
 *               loses about D/w of them to leading zeros, and its rounding then
 *               needs the exact fallback); when no part is smaller it is the
 *               default split.  The result is the same correctly rounded product.
 *               MPC_SPLIT_RESIDUAL (2, 4M only, else MPC_EINVAL; not in batched calls):
 *               Alg. 2 as printed (Sec. III-C): every real part of every row of A
 *               (column of B) is cut slice after slice, and before each slice the
 *               largest magnitude mu left in the line is measured again; the slice is
 *               the residual rounded to nearest (ties to even) at the unit
 *               2^(ceil(log2 mu) - (w - 1)), so a line whose residual collapses skips
 *               grid positions.  (The paper's tau is a power of two, which rounds
 *               negative residuals at half that unit; the extraction is read as
 *               symmetric, i.e. tau = 3 2^(k-1).)  The slices of one level then sit at
 *               different units in different lines, so every kept pair (t, u),
 *               t + u <= Q, has its own table entry and the accumulation adds each
 *               product at its own per-entry offset; consecutive pairs of a level whose
 *               slices step by exactly w in every line are merged into one exact
 *               tensor-core group of at most max_group (else the int32 limit) pairs,
 *               so lines that never skip are grouped as in the default split.  The pair
 *               products are streamed through a buffer of mpc_plan.pair_batch planes
 *               (whole levels at a time), so the workspace stays bounded; the exact
 *               accumulators live in the workspace between batches.  Same correctly
 *               rounded product.
 *   pair_planes residual split: planes in the pair-product buffer (0 -> about 32 GiB
 *               worth, at least one level, at most all pairs); other splits ignore it.
 */
typedef struct mpc_oz_params {
    int32_t guard_bits;
    int32_t slices;
    int32_t cut_level;
    int32_t kernel;
    int32_t max_group;
    int32_t digit_bits;
    int32_t wait_limit_cycles;
    int32_t dump_accumulators;
    int32_t split;
    int32_t pair_planes;
    int32_t reserved[2];
} mpc_oz_params;

/*
 * The plan of one call: chosen parameters and the workspace layout (byte
 * offsets into the workspace).  Filled by mpcgemm_plan(); useful to inspect
 * intermediate stages (digit planes, group sums) after a call.
 */
typedef struct mpc_plan {
    int32_t algo, method, p_bits, limbs;
    int32_t s, Q;                 /* slices per operand, highest kept level */
    int32_t kpad;                 /* k rounded up to 64 (digit-plane row length) */
    int32_t gmax;                 /* max pairs per group (int32-exact group sums) */
    int32_t n_products;           /* 4 (4M) or 3 (3M) real products */
    int32_t n_groups_total;       /* group planes over all products */
    int32_t n_groups[4];          /* per product: rr, ii, ri|ss, ir */
    int32_t planes_A, planes_B;   /* digit planes per operand */
    int32_t acc_slots;            /* 32-bit slots of the exact accumulator */
    int32_t bound_shift;          /* beta: bounds are b * 2^beta */
    uint64_t bound_drop[2];       /* ceil(dropped-pair bound / 2^beta), Re / Im */
    uint64_t bound_lossy_a[2];    /* per unit of k: added when the row of A is lossy */
    uint64_t bound_lossy_b[2];    /* per unit of k: added when the column of B is lossy */
    uint64_t off_status, off_rowexp, off_colexp, off_rowlossy, off_collossy;
    uint64_t off_digits_a, off_digits_b, off_groups, off_group_table;
    uint64_t off_fallback, fallback_capacity, off_fb_scratch, fb_scratch_limbs, fb_threads;
    uint64_t off_acc_dump;        /* accumulator dump (dump_accumulators), else 0 */
    uint64_t off_units;           /* residual split (else 0): slice units int32 [part][slice][row of A],
                                     then [part][slice][column of B] (INT32_MIN: a zero slice); then,
                                     256-byte aligned, the accumulator words between batches
                                     [comp][acc_slots][m n] u32, the truncation counts [comp][m n] u32,
                                     and B copied K-major (sign, exp, limb planes of n x k) */
    uint64_t ws_bytes;
    int32_t launches;             /* kernel launches one call makes */
    int32_t digit_bits;           /* Ozaki: bits per digit w (8 or 9); plain: 28 */
    uint64_t off_group_order;     /* groups ordered by descending level */
    int32_t split;                /* MPC_SPLIT_* */
    int32_t pair_batch;           /* residual split: planes per pair-product batch (off_groups), else 0 */
} mpc_plan;

/*
 * Optional stage timing: cudaEvent_t handles (passed as void*) created by the
 * caller with timing enabled.  When a handle is non-NULL the library records it
 * on `stream` at that stage boundary:
 *   ev[0] call start, ev[1] after the split (row/column exponents, digits or
 *   fixed-point operands), ev[2] after the slice products (Ozaki) or the plain
 *   GEMM, ev[3] after the accumulation (plain: combination) and rounding,
 *   ev[4] after the exact fallback.  ev[5..7] unused.  With the residual split the
 *   products and the accumulation alternate batch by batch: ev[2] is recorded
 *   before the last batch's accumulation, so earlier batches' accumulations count
 *   in the slice-product stage.
 */
typedef struct mpc_stage_events {
    void *ev[8];
} mpc_stage_events;

/* Device-side outcome of a call (read back by mpcgemm_read_status). */
typedef struct mpc_status {
    int32_t erange;           /* nonzero: some result exponent did not fit int32 */
    int32_t fallback_entries; /* components recomputed exactly (certification failed) */
    int32_t fallback_overflow;/* nonzero: more failures than the list holds */
    int32_t uncertified;      /* components whose exact fallback window was too wide
                                 (their terms span more than 12 288 bits) AND whose
                                 rounding the truncated window could not certify: only
                                 these may differ from RN_p of the exact value */
    int32_t device_timeout;   /* nonzero: a kernel's bounded wait gave up (results invalid) */
} mpc_status;

/*
 * C := RN_p(A B) for m x k A and k x n B, 1 <= p_bits <= MPC_MAX_P_BITS,
 * k <= MPC_MAX_K.  method: MPC_4M or MPC_3M (Eqs. 4m_way / 3m_way; with
 * exact arithmetic both give the same C).  algo: MPC_OZAKI (Alg. 2 on the
 * tensor cores: balanced 9-bit integer slices (8-bit when k >= 2^15) carried
 * exactly in bf16, exact slice products, exact accumulation, certified
 * rounding with exact fallback) or MPC_PLAIN (the
 * triple loop of Eq. simple_triple_loop as an exact fixed-point GEMM on the
 * CUDA cores: base-2^28 digit products summed exactly, 4 real products for
 * MPC_4M, 3 for MPC_3M (Eq. 3m_way_base), certified rounding with exact
 * fallback).  Sizes use A->rows == m,
 * A->cols == k, B->rows == k, B->cols == n, C->rows == m, C->cols == n.
 * Returns MPC_OK, MPC_EINVAL, MPC_ENOSPC, MPC_ENOTSUP or MPC_ECUDA - e.
 */
int mpcgemm(int64_t m, int64_t n, int64_t k, int32_t p_bits,
            const mpc_mat *A, const mpc_mat *B, mpc_mat *C,
            int method, int algo, void *workspace, size_t ws_bytes, void *stream);

/* As mpcgemm(), with Ozaki tuning (params may be NULL). */
int mpcgemm_ex(int64_t m, int64_t n, int64_t k, int32_t p_bits,
               const mpc_mat *A, const mpc_mat *B, mpc_mat *C,
               int method, int algo, const mpc_oz_params *params,
               void *workspace, size_t ws_bytes, void *stream);

/* As mpcgemm_ex(), recording the caller's events at stage boundaries
 * (events may be NULL: then identical to mpcgemm_ex). */
int mpcgemm_profiled(int64_t m, int64_t n, int64_t k, int32_t p_bits,
                     const mpc_mat *A, const mpc_mat *B, mpc_mat *C,
                     int method, int algo, const mpc_oz_params *params,
                     const mpc_stage_events *events,
                     void *workspace, size_t ws_bytes, void *stream);

/*
 * Batched form: `count` independent complex GEMMs, possibly of different sizes,
 * precisions and methods, in one call.  The Ozaki problems share ONE persistent
 * tcgen05 slice-GEMM launch (64 problems per launch), so small problems fill
 * the GPU together; the split, accumulation and fallback kernels run per
 * problem; in batches of 16 problems or more they are spread over 8
 * library-owned side streams that are forked from and
 * joined back into `stream` (under capture: parallel branches of the graph),
 * so the call stays ordered on `stream` like any other.  Each caller stream
 * (up to 64 per process) has side streams of its own, created by its first
 * batched call made outside stream capture; until then, and beyond 64 caller
 * streams, everything runs on `stream`.  Concurrent batched calls on the same
 * stream from several host threads enqueue one after the other.  The
 * call is asynchronous and allocates no memory, so it can be captured in a
 * CUDA graph and replayed.  Each problem uses its own region of
 * the workspace, at offsets[i] from mpcgemm_batched_workspace(); its device
 * status is read with mpcgemm_read_status(workspace + offsets[i], ...).
 * This extends the paper's CGEMM (Sec. III) to a batch; the paper has no batch.
 */
typedef struct mpc_problem {
    int64_t m, n, k;
    int32_t p_bits, method, algo, reserved;
    const mpc_mat *A, *B;
    mpc_mat *C;
} mpc_problem;

/* Per-problem workspace offsets (offsets may be NULL) and the total bytes. */
int mpcgemm_batched_workspace(int count, const mpc_problem *probs, const mpc_oz_params *params,
                              uint64_t *offsets, size_t *total);

int mpcgemm_batched(int count, const mpc_problem *probs, const mpc_oz_params *params,
                    void *workspace, size_t ws_bytes, void *stream);

/*
 * Complex linear solve A X = B by blocked right-looking LU with partial
 * pivoting (Kouya, Sec. IV-C, Fig. 3: each block of `block` columns is
 * factored, then A22 - L21 U12 is updated by the Ozaki complex GEMM with
 * `method`; block = 1 is the paper's "Normal LU"), then forward and backward
 * substitution (Sec. IV-C).  A (n x n) is overwritten by its factors (unit L
 * below the diagonal, U on and above), ipiv[j] (device int32, n entries) gets
 * the row swapped with row j, B (n x nrhs) is overwritten by X.  Every scalar
 * result is computed exactly and rounded once to p bits (nearest-even); the
 * pivot of column j is the first row maximising RN_p(|Re| + |Im|).
 * Device status (mpcgemm_read_status on the workspace): erange as for the
 * GEMM; `uncertified` = some exact window was truncated; word 5 (read it as
 * an int32 at workspace + 20) = 1 + the first column whose pivot is zero.
 */
size_t mpcgesv_workspace_size(int64_t n, int32_t p_bits, int32_t block, int method);
int mpcgesv(int64_t n, int32_t p_bits, mpc_mat *A, int32_t *ipiv, mpc_mat *B, int32_t block, int method,
            void *workspace, size_t ws_bytes, void *stream);

/* Bytes of workspace a call with these arguments needs (0 on bad arguments). */
size_t mpcgemm_workspace_size(int64_t m, int64_t n, int64_t k, int32_t p_bits,
                              int method, int algo);

/* The plan (parameters + workspace layout) of a call; params may be NULL. */
int mpcgemm_plan(int64_t m, int64_t n, int64_t k, int32_t p_bits, int method, int algo,
                 const mpc_oz_params *params, mpc_plan *out);

/* Synchronise `stream` and read the device status of the last call that used
 * this workspace.  Returns MPC_OK, or MPC_ERANGE if status->erange is set. */
int mpcgemm_read_status(const void *workspace, size_t ws_bytes, mpc_status *status, void *stream);

/*
 * Allocation-free variant of mpcgemm(), for callers that cannot allocate device
 * memory themselves -- for example a plug-in or callback that its host
 * application hands only the input and output buffers, or a latency-bound loop
 * that must not allocate once it is running.  The paper has no counterpart: this
 * is an interface convenience of the library.
 *
 * Instead of a caller workspace it uses one static device array of
 * MPC_NOALLOC_SCRATCH_BYTES (64 MiB) inside the library.  The array is
 * reserved on a device when its device code is loaded there: with CUDA's
 * default lazy module loading, when this entry point (or its status reader)
 * first runs on that device; with CUDA_MODULE_LOADING=EAGER, on every device
 * the process initialises, whether or not it calls this entry point.  It stays
 * reserved until the process exits.  A problem whose
 * mpcgemm_workspace_size() exceeds it is rejected with MPC_ENOSPC before
 * anything is enqueued (for example m = n = k = 192 fits at p = 256 and 128 at
 * p = 1024 for Ozaki 4M/3M and for plain; 256 at p = 256 for Ozaki
 * does not).  The first call on a device looks
 * up the array's device address (it allocates nothing); make that first call
 * outside any stream capture.  Every call uses the same array and finds the
 * previous call's contents there (each call re-initialises what it reads), so
 * calls whose GPU work overlaps -- on different streams or from different host
 * threads -- race and produce wrong results: serialise them.  Arguments, results
 * and errors are those of mpcgemm(), with no workspace arguments; the device
 * status of the last call on the current device is read with
 * mpcgemm_noalloc_read_status().
 */
#define MPC_NOALLOC_SCRATCH_BYTES (64u << 20)
int mpcgemm_noalloc(int64_t m, int64_t n, int64_t k, int32_t p_bits,
                    const mpc_mat *A, const mpc_mat *B, mpc_mat *C,
                    int method, int algo, void *stream);

/* mpcgemm_read_status() for mpcgemm_noalloc(): synchronises `stream` and reads
 * the status block of the static array on the current device (the last call
 * there).  Allocates nothing.  Returns MPC_OK, MPC_ERANGE (status->erange set)
 * or an error code. */
int mpcgemm_noalloc_read_status(mpc_status *status, void *stream);

/* Human-readable text of a status code (static storage). */
const char *mpcgemm_strerror(int code);

/* Library version: major*10000 + minor*100 + patch. */
int mpcgemm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* MPCGEMM_H */
