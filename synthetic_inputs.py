"""Seeded synthetic multiple-precision complex matrices.

This module only *draws* inputs.  It holds none of the method's arithmetic:
no splitting, no products, no rounding.  Both the CPU oracle (``oracle/``)
and the CUDA path (through its tests and ``bench.py``) take their inputs from
here, so that the two never share anything else.

Number format (the on-device format of the C ABI, see ``include/mpcgemm.h``):
each real component of an element is

    value = (-1)**sign * M * 2**(exp - 64*L),      L = ceil(p / 64)

with M an L-limb unsigned integer (limb 0 least significant).  A nonzero
value drawn here is normalised (bit 64L-1 of M set) and has at most p
significant bits (the 64L-p low bits of M are zero).  Zero is M == 0,
sign 0, exp = INT32_MIN.

Array layout of an ``MPCMatrix`` (dense, row-major, ld == cols):

    sign[c, r, col]      uint8    c = 0 real part, c = 1 imaginary part
    exp[c, r, col]       int32
    limb[c, j, r, col]   uint64   j = limb index, 0 = least significant

Distributions (the paper's benchmark matrices have real and imaginary parts
drawn at random in [-1, 1], Sec. IV-A; BASELINE configs restate this):

* ``uniform``      each component uniform on the p-bit grid of [-1, 1):
                   u * 2**-p with u uniform in [0, 2**p), random sign.
* ``uniform_exp``  the same times 2**e, e uniform integer in [emin, emax],
                   independently per element and component (widens the
                   exponent spread inside rows and columns).
"""
from __future__ import annotations

import dataclasses

import numpy as np

INT32_MIN = -(2 ** 31)

# seeds used by the configurations (20230712 = the paper's arXiv month, + index)
SEED_BASE = 20230712


def limbs_for(p_bits: int) -> int:
    """Number of 64-bit limbs that hold a p-bit mantissa."""
    if p_bits < 1:
        raise ValueError("p_bits must be >= 1")
    return (p_bits + 63) // 64


@dataclasses.dataclass
class MPCMatrix:
    """A dense complex matrix in the C-ABI number format (host numpy arrays)."""

    rows: int
    cols: int
    p: int
    sign: np.ndarray  # (2, rows, cols) uint8
    exp: np.ndarray   # (2, rows, cols) int32
    limb: np.ndarray  # (2, L, rows, cols) uint64

    @property
    def L(self) -> int:
        return self.limb.shape[1]

    def copy(self) -> "MPCMatrix":
        return MPCMatrix(self.rows, self.cols, self.p, self.sign.copy(),
                         self.exp.copy(), self.limb.copy())

    @staticmethod
    def zeros(rows: int, cols: int, p: int) -> "MPCMatrix":
        L = limbs_for(p)
        return MPCMatrix(rows, cols, p,
                         np.zeros((2, rows, cols), np.uint8),
                         np.full((2, rows, cols), INT32_MIN, np.int32),
                         np.zeros((2, L, rows, cols), np.uint64))

    def submatrix(self, r0: int, r1: int, c0: int, c1: int) -> "MPCMatrix":
        return MPCMatrix(r1 - r0, c1 - c0, self.p,
                         np.ascontiguousarray(self.sign[:, r0:r1, c0:c1]),
                         np.ascontiguousarray(self.exp[:, r0:r1, c0:c1]),
                         np.ascontiguousarray(self.limb[:, :, r0:r1, c0:c1]))

    def transpose(self) -> "MPCMatrix":
        return MPCMatrix(self.cols, self.rows, self.p,
                         np.ascontiguousarray(self.sign.transpose(0, 2, 1)),
                         np.ascontiguousarray(self.exp.transpose(0, 2, 1)),
                         np.ascontiguousarray(self.limb.transpose(0, 1, 3, 2)))

    def nbytes(self) -> int:
        return self.sign.nbytes + self.exp.nbytes + self.limb.nbytes


def _keep_top_bits_mask(L: int, cut: np.ndarray) -> list:
    """Per-limb masks that clear every bit of an L-limb word below bit `cut`."""
    masks = []
    full = np.uint64(0xFFFFFFFFFFFFFFFF)
    for j in range(L):
        lo = 64 * j
        rel = cut - lo  # bits of this limb to clear (may be <=0 or >=64)
        m = np.where(rel <= 0, full, np.uint64(0))
        part = (rel > 0) & (rel < 64)
        relc = np.clip(rel, 0, 63).astype(np.uint64)
        m = np.where(part, full ^ ((np.uint64(1) << relc) - np.uint64(1)), m)
        masks.append(m.astype(np.uint64))
    return masks


def random_matrix(rows: int, cols: int, p: int, seed: int,
                  dist: str = "uniform", emin: int = -20, emax: int = 20,
                  zero_frac: float = 0.0) -> MPCMatrix:
    """Draw a seeded complex matrix (see module docstring for distributions).

    A p-bit uniform integer u in [0, 2**p) has bit length p - z with
    P(z = j) = 2**-(j+1) and uniform bits below its leading one; drawing z
    and the remaining bits directly gives exactly that distribution without
    big-integer work.  z >= p means u == 0.
    """
    rng = np.random.default_rng(seed)
    L = limbs_for(p)
    shape = (2, rows, cols)
    limb = rng.integers(0, 2 ** 64, size=(2, L, rows, cols), dtype=np.uint64,
                        endpoint=False)
    z = rng.geometric(0.5, size=shape).astype(np.int64) - 1
    sign = rng.integers(0, 2, size=shape, dtype=np.uint8)
    # top bit set, bits below (64L - p + z) cleared
    cut = (64 * L - p) + z
    masks = _keep_top_bits_mask(L, cut)
    for j in range(L):
        limb[:, j] &= masks[j]
    limb[:, L - 1] |= np.uint64(1) << np.uint64(63)
    exp = (-z).astype(np.int64)
    if dist == "uniform":
        pass
    elif dist == "uniform_exp":
        exp = exp + rng.integers(emin, emax + 1, size=shape, dtype=np.int64)
    else:
        raise ValueError(f"unknown distribution {dist!r}")
    zero = z >= p
    if zero_frac > 0.0:
        zero |= rng.random(shape) < zero_frac
    sign = np.where(zero, 0, sign).astype(np.uint8)
    exp = np.where(zero, INT32_MIN, exp).astype(np.int32)
    limb = np.where(zero[:, None], np.uint64(0), limb)
    return MPCMatrix(rows, cols, p, sign, exp, np.ascontiguousarray(limb))


def small_integer_matrix(rows: int, cols: int, p: int, seed: int,
                         lo: int = -3, hi: int = 3) -> MPCMatrix:
    """Complex matrix whose components are small integers in [lo, hi].

    Used for cases that a library routine (numpy integer matmul) can check.
    Integer v != 0 is encoded as M = |v| << (64L - bitlen|v|), exp = bitlen|v|.
    """
    rng = np.random.default_rng(seed)
    vals = rng.integers(lo, hi + 1, size=(2, rows, cols), dtype=np.int64)
    return from_integers(vals, p)


def from_integers(vals: np.ndarray, p: int) -> MPCMatrix:
    """Encode an int64 array of shape (2, rows, cols) (|v| < 2**62) exactly."""
    L = limbs_for(p)
    _, rows, cols = vals.shape
    mag = np.abs(vals).astype(np.uint64)
    sign = (vals < 0).astype(np.uint8)
    bl = np.zeros(vals.shape, np.int64)
    t = mag.copy()
    while np.any(t):
        nz = t != 0
        bl += nz
        t >>= np.uint64(1)
    if np.any(bl > p):
        raise ValueError("integer needs more than p bits")
    limb = np.zeros((2, L, rows, cols), np.uint64)
    sh = (64 - bl).astype(np.uint64)
    top = np.where(bl > 0, mag << np.where(bl > 0, sh, 0).astype(np.uint64), 0)
    limb[:, L - 1] = top.astype(np.uint64)
    exp = np.where(bl > 0, bl, INT32_MIN).astype(np.int32)
    sign = np.where(bl > 0, sign, 0).astype(np.uint8)
    return MPCMatrix(rows, cols, p, sign, exp, limb)


def identity_matrix(n: int, p: int) -> MPCMatrix:
    v = np.zeros((2, n, n), np.int64)
    v[0] = np.eye(n, dtype=np.int64)
    return from_integers(v, p)


def shifted_diagonal_matrix(n: int, p: int, seed: int) -> MPCMatrix:
    """A = U + n I with U uniform on [-1, 1) per component (the LU workload).

    Off-diagonal entries are drawn as in ``random_matrix``; the real diagonal
    is n + u with u uniform on the grid of spacing 2**-(p - 1 - bitlen(n)),
    so that n + u is exactly a p-bit number and no rounding is needed.
    """
    import random as _random
    A = random_matrix(n, n, p, seed, "uniform")
    rng = _random.Random(seed + 1)
    L = limbs_for(p)
    nb = int(n).bit_length()
    frac_bits = p - 1 - nb
    for i in range(n):
        u = rng.getrandbits(frac_bits + 1) - (1 << frac_bits)      # u * 2^-frac_bits in [-1, 1)
        v = (n << frac_bits) + u                                     # value * 2^frac_bits, > 0
        bl = v.bit_length()
        M = v << (64 * L - bl)
        A.sign[0, i, i] = 0
        A.exp[0, i, i] = bl - frac_bits
        for j in range(L):
            A.limb[0, j, i, i] = (M >> (64 * j)) & 0xFFFFFFFFFFFFFFFF
    return A


def config_inputs(name: str):
    """The seeded workloads of the benchmark configurations.

    Returns (m, n, k, p, dist) for a named configuration.  The matrices are
    drawn with ``random_matrix(m, k, p, SEED_BASE + idx, dist)`` for A and
    seed + 1000 for B.
    """
    table = {
        # plain 4M, 32^3, p = 128, uniform [-1, 1)
        "c0_plain_32_p128": (32, 32, 32, 128, "uniform", 0),
        # Ozaki 4M, 256^3, p = 256, uniform [-1, 1)
        "c1_ozaki_256_p256": (256, 256, 256, 256, "uniform", 1),
        # Ozaki 3M / 4M / plain, n in {1024, 2048}, p in {256, 512, 1024}, u * 2^e
        "c2_1024_p256": (1024, 1024, 1024, 256, "uniform_exp", 2),
        "c2_2048_p256": (2048, 2048, 2048, 256, "uniform_exp", 2),
        "c2_1024_p512": (1024, 1024, 1024, 512, "uniform_exp", 2),
        "c2_1024_p1024": (1024, 1024, 1024, 1024, "uniform_exp", 2),
        "c2_2048_p512": (2048, 2048, 2048, 512, "uniform_exp", 2),
        "c2_2048_p1024": (2048, 2048, 2048, 1024, "uniform_exp", 2),
    }
    return table[name]


def make_config(name: str):
    m, n, k, p, dist, idx = config_inputs(name)
    A = random_matrix(m, k, p, SEED_BASE + idx, dist)
    B = random_matrix(k, n, p, SEED_BASE + idx + 1000, dist)
    return A, B, p


def batch_specs(count: int = 64, seed: int = SEED_BASE + 3):
    """The batched workload: (m, k, n, p) of `count` problems, m, n, k log-uniform in
    [64, 1024], p drawn from {256, 512, 1024}."""
    rng = np.random.default_rng(seed)
    mnk = np.exp(rng.uniform(np.log(64), np.log(1024), size=(count, 3))).astype(int)
    ps = rng.choice([256, 512, 1024], size=count)
    return [(int(m), int(k), int(n), int(p)) for (m, n, k), p in zip(mnk, ps)]


def batch_problems(specs):
    """The seeded operands (host side) of the batched workload: [(A, B, p)]."""
    out = []
    for x, (m, k, n, p) in enumerate(specs):
        A = random_matrix(m, k, p, SEED_BASE + 3000 + 2 * x, "uniform")
        B = random_matrix(k, n, p, SEED_BASE + 3001 + 2 * x, "uniform")
        out.append((A, B, p))
    return out

