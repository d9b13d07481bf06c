/*
 * O1 in C -- exact complex matrix product rounded once to p bits.
 * TEST INFRASTRUCTURE: only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference leg load this library.  It shares no code with
 * the CUDA path (own limb arithmetic, own rounding).
 *
 * Definition followed (Kouya, Sec. III-A):
 *   Eq. (simple_triple_loop): (C)_ij = sum_l (A)_il (B)_lj
 *   Eq. (4m_way_base):        Re = ReA ReB - ImA ImB, Im = ReA ImB + ImA ReB
 * The sum is formed exactly in a two's-complement fixed-point window wide
 * enough for every product of the dot product, then rounded to nearest,
 * ties to even, on a p-bit significand.
 *
 * Number format (per real component): value = (-1)^sign * M * 2^(exp-64L),
 * M = sum_j limb[j] 2^(64j), zero iff the top limb limb[L-1] == 0.  Arrays are dense planes:
 *   sign[c*R*C + idx], exp[c*R*C + idx], limb[(c*L + j)*R*C + idx],
 *   idx = r*C + col, c = 0 real, 1 imaginary.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;

#define ORACLE_OK 0
#define ORACLE_ERANGE (-34)
#define ORACLE_ENOMEM (-12)

typedef struct {
    const uint8_t *sign;
    const int32_t *exp;
    const uint64_t *limb;
    int64_t R, C;
    int L;
} omat;

/* zero iff the top limb is 0 (format definition) */
static int is_zero(const omat *a, int c, int64_t idx) {
    int64_t plane = a->R * a->C;
    return a->limb[((int64_t)c * a->L + a->L - 1) * plane + idx] == 0;
}

static void load_mant(const omat *a, int c, int64_t idx, uint64_t *out) {
    int64_t plane = a->R * a->C;
    for (int j = 0; j < a->L; j++) out[j] = a->limb[((int64_t)c * a->L + j) * plane + idx];
}

/* out[0..2L) = x[0..L) * y[0..L), schoolbook */
static void mul_limbs(const uint64_t *x, const uint64_t *y, int L, uint64_t *out) {
    memset(out, 0, sizeof(uint64_t) * 2 * L);
    for (int i = 0; i < L; i++) {
        uint64_t carry = 0;
        for (int j = 0; j < L; j++) {
            u128 t = (u128)x[i] * y[j] + out[i + j] + carry;
            out[i + j] = (uint64_t)t;
            carry = (uint64_t)(t >> 64);
        }
        out[i + L] = carry;
    }
}

/* acc (nw limbs, two's complement) += (negate ? -1 : 1) * (p[0..np) << shift) */
static void add_shifted(uint64_t *acc, int nw, const uint64_t *p, int np, int64_t shift, int negate) {
    int64_t w = shift >> 6;
    int b = (int)(shift & 63);
    /* the shifted operand occupies limbs w .. w+np (np+1 limbs) */
    uint64_t borrow_or_carry = 0;
    int64_t top = w + np;
    for (int64_t i = w; i < nw; i++) {
        uint64_t v;
        int64_t j = i - w;
        if (j <= np) {
            uint64_t lo = (j < np) ? p[j] : 0;
            uint64_t hi = (j >= 1 && j - 1 < np) ? p[j - 1] : 0;
            v = b ? ((lo << b) | (hi >> (64 - b))) : lo;
        } else {
            v = 0;
        }
        if (!negate) {
            u128 t = (u128)acc[i] + v + borrow_or_carry;
            acc[i] = (uint64_t)t;
            borrow_or_carry = (uint64_t)(t >> 64);
        } else {
            u128 t = (u128)acc[i] - v - borrow_or_carry;
            acc[i] = (uint64_t)t;
            borrow_or_carry = (uint64_t)(t >> 64) ? 1 : 0;
        }
        if (i > top && borrow_or_carry == 0) break;
    }
}

static int bitlen_limbs(const uint64_t *a, int n) {
    for (int i = n - 1; i >= 0; i--)
        if (a[i]) return 64 * i + (64 - __builtin_clzll(a[i]));
    return 0;
}

static int get_bit(const uint64_t *a, int64_t pos) {
    if (pos < 0) return 0;
    return (int)((a[pos >> 6] >> (pos & 63)) & 1);
}

/* any bit set strictly below position pos */
static int any_below(const uint64_t *a, int64_t pos) {
    if (pos <= 0) return 0;
    int64_t w = pos >> 6;
    for (int64_t i = 0; i < w; i++)
        if (a[i]) return 1;
    int b = (int)(pos & 63);
    if (b && (a[w] & ((1ull << b) - 1))) return 1;
    return 0;
}

/*
 * Round mag (nw limbs, value mag * 2^x) to p bits, nearest-even, and encode
 * into sign/exp/limbs (L limbs, normalised).  Returns ORACLE_ERANGE if the
 * exponent does not fit int32.
 */
static int round_encode(uint64_t *mag, int nw, int64_t x, int neg, int p, int L,
                        uint8_t *sign_out, int32_t *exp_out, uint64_t *limb_out, int64_t ostride) {
    int n = bitlen_limbs(mag, nw);
    if (n == 0) {
        *sign_out = 0;
        *exp_out = INT32_MIN;
        for (int j = 0; j < L; j++) limb_out[j * ostride] = 0;
        return ORACLE_OK;
    }
    int64_t e;
    /* q = top min(n,p) bits */
    uint64_t q[64];
    int qn = (p + 64) / 64 + 1;
    memset(q, 0, sizeof(q));
    int64_t sh = n > p ? n - p : 0;
    for (int64_t i = 0; i < p + 1 && sh + i < n; i++)
        if (get_bit(mag, sh + i)) q[i >> 6] |= 1ull << (i & 63);
    if (sh > 0) {
        int rbit = get_bit(mag, sh - 1);
        int sticky = any_below(mag, sh - 1);
        int odd = (int)(q[0] & 1);
        if (rbit && (sticky || odd)) {
            for (int i = 0; i < qn; i++) {
                q[i] += 1;
                if (q[i] != 0) break;
            }
        }
    }
    int qb = bitlen_limbs(q, qn);
    e = x + sh + qb;
    if (e > INT32_MAX || e < (int64_t)INT32_MIN + 1) return ORACLE_ERANGE;
    /* M = q << (64L - qb) */
    uint64_t M[64];
    memset(M, 0, sizeof(M));
    int64_t s = 64 * (int64_t)L - qb;
    for (int64_t i = 0; i < qb; i++)
        if (get_bit(q, i)) M[(i + s) >> 6] |= 1ull << ((i + s) & 63);
    *sign_out = (uint8_t)neg;
    *exp_out = (int32_t)e;
    for (int j = 0; j < L; j++) limb_out[j * ostride] = M[j];
    return ORACLE_OK;
}

typedef struct {
    int ca, cb;     /* component of A and of B */
    int negate;
} term_t;

/*
 * Exact sum over l of the listed real products, then rounded.
 * Window: LSB at xmin = min over nonzero products of (ea+eb-128L); width
 * covers the largest product (< 2^(ea+eb)) plus log2(2k)+2 bits of growth.
 */
static int exact_component(const omat *A, const omat *B, int64_t i, int64_t j, int64_t k,
                           const term_t *terms, int nterms, int p,
                           uint64_t **accbuf, int *acccap,
                           uint8_t *sign_out, int32_t *exp_out, uint64_t *limb_out, int64_t ostride) {
    int L = A->L;
    int64_t xmin = INT64_MAX, top = INT64_MIN;
    for (int64_t l = 0; l < k; l++) {
        int64_t ia = i * A->C + l, ib = l * B->C + j;
        for (int t = 0; t < nterms; t++) {
            if (is_zero(A, terms[t].ca, ia) || is_zero(B, terms[t].cb, ib)) continue;
            int64_t es = (int64_t)A->exp[(int64_t)terms[t].ca * A->R * A->C + ia] +
                         (int64_t)B->exp[(int64_t)terms[t].cb * B->R * B->C + ib];
            if (es - 128 * (int64_t)L < xmin) xmin = es - 128 * (int64_t)L;
            if (es > top) top = es;
        }
    }
    if (top == INT64_MIN) {
        uint64_t z = 0;
        return round_encode(&z, 1, 0, 0, p, L, sign_out, exp_out, limb_out, ostride);
    }
    int64_t growth = 2;
    while (((int64_t)1 << growth) < 2 * k * nterms) growth++;
    int64_t width = top - xmin + growth + 2;
    int nw = (int)(width / 64 + 2);
    if (nw > *acccap) {
        free(*accbuf);
        *accbuf = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)nw);
        if (!*accbuf) { *acccap = 0; return ORACLE_ENOMEM; }
        *acccap = nw;
    }
    uint64_t *acc = *accbuf;
    memset(acc, 0, sizeof(uint64_t) * (size_t)nw);
    uint64_t ma[32], mb[32], pr[64];
    for (int64_t l = 0; l < k; l++) {
        int64_t ia = i * A->C + l, ib = l * B->C + j;
        for (int t = 0; t < nterms; t++) {
            int ca = terms[t].ca, cb = terms[t].cb;
            if (is_zero(A, ca, ia) || is_zero(B, cb, ib)) continue;
            load_mant(A, ca, ia, ma);
            load_mant(B, cb, ib, mb);
            mul_limbs(ma, mb, L, pr);
            int64_t planeA = A->R * A->C, planeB = B->R * B->C;
            int sa = A->sign[ca * planeA + ia], sb = B->sign[cb * planeB + ib];
            int64_t es = (int64_t)A->exp[ca * planeA + ia] + (int64_t)B->exp[cb * planeB + ib];
            int neg = (sa ^ sb) ^ terms[t].negate;
            add_shifted(acc, nw, pr, 2 * L, es - 128 * (int64_t)L - xmin, neg);
        }
    }
    int neg = (int)(acc[nw - 1] >> 63);
    if (neg) { /* two's complement negate */
        uint64_t c = 1;
        for (int w = 0; w < nw; w++) {
            u128 t = (u128)(~acc[w]) + c;
            acc[w] = (uint64_t)t;
            c = (uint64_t)(t >> 64);
        }
    }
    return round_encode(acc, nw, xmin, neg, p, L, sign_out, exp_out, limb_out, ostride);
}

/*
 * C = RN_p(A B).  If entries != NULL, only the listed (i, j) pairs are
 * computed and outputs are dense over the list (plane = n_entries);
 * otherwise all m*n entries (plane = m*n, idx = i*n + j).
 */
int oracle_cgemm(int64_t m, int64_t n, int64_t k, int p,
                 const uint8_t *Asign, const int32_t *Aexp, const uint64_t *Alimb,
                 const uint8_t *Bsign, const int32_t *Bexp, const uint64_t *Blimb,
                 const int64_t *entries, int64_t n_entries,
                 uint8_t *Csign, int32_t *Cexp, uint64_t *Climb, int nthreads) {
    int L = (p + 63) / 64;
    if (L > 31 || p < 1) return -22;
    omat A = {Asign, Aexp, Alimb, m, k, L};
    omat B = {Bsign, Bexp, Blimb, k, n, L};
    int64_t total = entries ? n_entries : m * n;
    term_t re_terms[2] = {{0, 0, 0}, {1, 1, 1}};
    term_t im_terms[2] = {{0, 1, 0}, {1, 0, 0}};
    int status = ORACLE_OK;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        uint64_t *accbuf = NULL;
        int acccap = 0;
#pragma omp for schedule(dynamic, 4)
        for (int64_t e = 0; e < total; e++) {
            int64_t i = entries ? entries[2 * e] : e / n;
            int64_t j = entries ? entries[2 * e + 1] : e % n;
            for (int c = 0; c < 2; c++) {
                int rc = exact_component(&A, &B, i, j, k, c == 0 ? re_terms : im_terms, 2, p,
                                         &accbuf, &acccap,
                                         Csign + c * total + e, Cexp + c * total + e,
                                         Climb + (int64_t)c * L * total + e, total);
                if (rc != ORACLE_OK) {
#pragma omp critical
                    status = rc;
                }
            }
        }
        free(accbuf);
    }
    return status;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
