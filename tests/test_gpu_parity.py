"""CUDA path vs the oracle, through the C ABI.

Integer stages (digits, group sums) must equal O2 bit for bit; every output
must equal O1 = RN_p(exact product) bit for bit (certified rounding plus exact
fallback make the result the correctly rounded product).  Each case also
reports the error in units of 2^-p, which is 0 or <= 1/2 ulp by construction.
"""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import c_oracle, exact, ozaki
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


def _check_group_sums(ws, pl, r, m, n):
    """Every written group sum equals O2's; a group that the all-zero digit planes emptied
    (count 0 on the device) is not written, and O2's sum for it is zero; a product that
    enters only components vanishing identically has every group emptied."""
    G = gu.ws_groups(ws, pl, m, n)
    table, _, _ = gu.ws_group_tables(ws, pl)
    e = 0
    for pr in r.params.products:
        needed = ozaki.product_needed(r.splitA, r.splitB, pr, r.params.method)
        for Gr in r.group_sums[pr]:
            if not needed:
                assert table[e, 3] == 0, (pr, e)
            elif table[e, 3] > 0:
                assert np.array_equal(G[e], Gr), (pr, e)
            else:
                assert not np.any(Gr), (pr, e)
            e += 1
    assert e == G.shape[0]


def _check_against_o1(C, A, B, p):
    ref = c_oracle.rounded_cgemm_matrix(A, B, p)
    bad = gu.mismatches(C, ref)
    assert len(bad) == 0, f"{len(bad)} mismatching components, first {bad[:5].tolist()}"


@pytest.mark.parametrize("method", ["4m", "3m"])
def test_plain_config0_bit_exact(method):
    A, B, p = si.make_config("c0_plain_32_p128")
    C, ws, st = gu.run(A, B, p, method, "plain")
    assert gu.same(C, exact.rounded_cgemm(A, B, p))
    assert st["erange"] == 0


@pytest.mark.parametrize("method", ["4m", "3m"])
@pytest.mark.parametrize("dist,zf", [("uniform", 0.0), ("uniform_exp", 0.1)])
def test_ozaki_ragged_tiles_bit_exact(method, dist, zf):
    """Several 128 x 128 tiles with ragged edges and a k tail (k = 150 -> kpad 192)."""
    p = 128
    A = si.random_matrix(200, 150, p, 301, dist, zero_frac=zf)
    B = si.random_matrix(150, 300, p, 302, dist, zero_frac=zf)
    C, ws, st = gu.run(A, B, p, method, "ozaki")
    _check_against_o1(C, A, B, p)
    assert st["fallback_overflow"] == 0 and st["uncertified"] == 0


@pytest.mark.parametrize("method", ["4m", "3m"])
@pytest.mark.parametrize("p", [192, 1000])
def test_plain_ragged_bit_exact(method, p):
    """5 x 2 output tiles of 8 x 16 with ragged edges, a k tail (70 = 8 * 8 + 6); p = 1000
    takes the largest digit count (38 digits of 28 bits)."""
    A = si.random_matrix(37, 70, p, 311, "uniform_exp", zero_frac=0.1)
    B = si.random_matrix(70, 29, p, 312, "uniform_exp")
    C, ws, st = gu.run(A, B, p, method, "plain")
    _check_against_o1(C, A, B, p)
    assert st["uncertified"] == 0


def _largest_digit_mantissa(pl, L):
    """Mantissa whose plain-path digits are all -2^27 (the largest magnitude) above the
    bits that the fixed-point shift leaves zero, for an element at the row's exponent."""
    D, W = pl["s"], pl["bound_shift"]
    sh = W - 64 * L                              # X = M 2^sh
    t0 = -(-sh // 28) + 1
    X = (1 << 27) << (28 * t0)
    for t in range(t0 + 1, D - 1):
        X += ((1 << 27) - 1) << (28 * t)
    X += ((1 << 26) - 1) << (28 * (D - 1))       # top group: bit W-1 set (normalised)
    assert X >> (W - 1) == 1 and X % (1 << sh) == 0
    M = X >> sh
    return [(M >> (64 * j)) & 0xFFFFFFFFFFFFFFFF for j in range(L)]


@pytest.mark.parametrize("method", ["4m", "3m"])
def test_plain_long_k_largest_sums(method):
    """k = 20000 products of digits at their largest magnitude, all of one sign: every
    column sum of the plain kernel and its signed top column reach their largest values."""
    p, k = 256, 20000
    A = si.random_matrix(3, k, p, 315)
    B = si.random_matrix(k, 4, p, 316)
    L = si.limbs_for(p)
    limbs = _largest_digit_mantissa(gu.plan(A, B, p, method, "plain"), L)
    for X in (A, B):
        for j in range(L):
            X.limb[:, j] = np.uint64(limbs[j])
        X.sign[:] = 0
        X.exp[:] = 0
    B.sign[1] = 1                      # Im(B) < 0: Re(AB) = rr - ii adds up, Im(AB) cancels to 0
    C, ws, st = gu.run(A, B, p, method, "plain")
    _check_against_o1(C, A, B, p)


@pytest.mark.parametrize("method", ["4m", "3m"])
@pytest.mark.parametrize("w", [9, 8])
def test_config1_stage_parity(method, w):
    """256^3, p = 256: digits and every group sum equal O2; output equals O1 (9- and
    8-bit digits)."""
    A, B, p = si.make_config("c1_ozaki_256_p256")
    params = dict(digit_bits=w)
    C, ws, st = gu.run(A, B, p, method, "ozaki", params=params)
    pl = gu.plan(A, B, p, method, params=params)
    assert pl["digit_bits"] == w
    r = ozaki.ozaki_cgemm(A, B, p, method, fallback=lambda i, j: ((0, 0), (0, 0)), w=w)
    s, kp, k = r.params.s, pl["kpad"], A.cols
    dA = gu.ws_digits(ws, pl, "A", A.rows)
    dB = gu.ws_digits(ws, pl, "B", B.cols)
    assert np.array_equal(dA[:s, :, :k], r.splitA.digits["re"])
    assert np.array_equal(dA[s:2 * s, :, :k], r.splitA.digits["im"])
    assert np.array_equal(dB[:s, :, :k], r.splitB.digits["re"])
    assert np.array_equal(dB[s:2 * s, :, :k], r.splitB.digits["im"])
    if method == "3m":
        assert np.array_equal(dA[2 * s:, :, :k], r.splitA.digits["sum"])
        assert np.array_equal(dB[2 * s:, :, :k], r.splitB.digits["sum"])
    assert not np.any(dA[:, :, k:]) and not np.any(dB[:, :, k:])
    _check_group_sums(ws, pl, r, A.rows, B.cols)
    assert st["fallback_entries"] == int((~r.certified).sum())
    _check_against_o1(C, A, B, p)


@pytest.mark.parametrize("method", ["4m", "3m"])
def test_group_table_order_and_unit_schedule(method):
    """The device-built group table equals O2's groups; the accumulation order visits levels
    in descending order; the slice GEMM's unit schedule is a permutation that keeps each
    product's groups together, by descending pair count, stable."""
    p = 256
    A = si.random_matrix(130, 300, p, 345, "uniform_exp")
    B = si.random_matrix(300, 140, p, 346, "uniform_exp")
    params = dict(max_group=5)
    C, ws, st = gu.run(A, B, p, method, "ozaki", params=params)
    pl = gu.plan(A, B, p, method, params=params)
    table, order, sched = gu.ws_group_tables(ws, pl)
    r = ozaki.ozaki_cgemm(A, B, p, method, max_group=5, fallback=lambda i, j: ((0, 0), (0, 0)))
    ref = [(x, h.q, h.t0, h.count) for x, pr in enumerate(r.params.products)
           for h in ozaki.trim_groups(r.splitA, r.splitB, pr, r.groups[pr], method)]
    got = [tuple(int(v) for v in row) for row in table]
    assert [(g[0], g[1], g[3]) for g in got] == [(g[0], g[1], g[3]) for g in ref]
    assert all(a[2] == b[2] for a, b in zip(got, ref) if b[3] > 0)
    G = len(ref)
    assert sorted(order.tolist()) == list(range(G)) and sorted(sched.tolist()) == list(range(G))
    levels = table[order, 1]
    assert np.all(levels[:-1] >= levels[1:])
    prods = table[sched, 0]
    assert np.all(prods[:-1] <= prods[1:])                       # product by product
    for x in range(int(table[:, 0].max()) + 1):
        part = sched[prods == x]
        key = [(-int(table[e, 3]), int(e)) for e in part]       # descending count, then table order
        assert key == sorted(key)
    _check_against_o1(C, A, B, p)


def _drop_part(mat, c):
    out = mat.copy()
    out.limb[c] = 0
    out.sign[c] = 0
    out.exp[c] = si.INT32_MIN
    return out


def _shift_part(mat, c, by):
    out = mat.copy()
    nz = out.limb[c, -1] != 0
    out.exp[c] = np.where(nz, out.exp[c] + by, out.exp[c]).astype(np.int32)
    return out


@pytest.mark.parametrize("method", ["4m", "3m"])
@pytest.mark.parametrize("case", ["real", "small_imaginary", "imaginary_A"])
@pytest.mark.parametrize("kernel", ["auto", "mma_sync"])
def test_zero_digit_planes_are_skipped(method, case, kernel):
    """Groups lose the pairs of all-zero digit planes at their ends exactly as O2 trims them
    (real inputs, an imaginary part 2^-100 smaller, a purely imaginary A); the result is
    still the correctly rounded product."""
    p = 256
    A = si.random_matrix(200, 150, p, 351, "uniform_exp")
    B = si.random_matrix(150, 300, p, 352, "uniform_exp")
    if case == "real":
        A, B = _drop_part(A, 1), _drop_part(B, 1)
    elif case == "small_imaginary":
        A, B = _shift_part(A, 1, -100), _shift_part(B, 1, -100)
    else:
        A = _drop_part(A, 0)
    params = dict(kernel=kernel)
    C, ws, st = gu.run(A, B, p, method, "ozaki", params=params)
    pl = gu.plan(A, B, p, method, params=params)
    table, order, sched = gu.ws_group_tables(ws, pl)
    r = ozaki.ozaki_cgemm(A, B, p, method, fallback=lambda i, j: ((0, 0), (0, 0)))
    ref = []
    for x, pr in enumerate(r.params.products):
        for h in ozaki.trim_groups(r.splitA, r.splitB, pr, r.groups[pr], method):
            ref.append((x, h.q, h.t0, h.count))
    got = [tuple(int(v) for v in row) for row in table]
    assert [g[:2] + (g[3],) for g in got] == [g[:2] + (g[3],) for g in ref]
    assert all(a[2] == b[2] for a, b in zip(got, ref) if b[3] > 0)
    empty = sum(1 for g in ref if g[3] == 0)
    assert empty > 0
    _check_group_sums(ws, pl, r, A.rows, B.cols)
    _check_against_o1(C, A, B, p)
    assert st["fallback_entries"] == int((~r.certified).sum())     # the same data-dependent bound
    if case == "real":
        assert r.certified[1].all() and st["fallback_entries"] == int((~r.certified[0]).sum())
    assert st["fallback_overflow"] == 0 and st["uncertified"] == 0


def _digit_pattern_mantissa(top, low, s, w, L):
    """Mantissa (exponent 0) whose w-bit balanced digits are top, then low repeated."""
    R = 1 << w
    X = top * R ** (s - 1) + sum(low * R ** (s - 1 - t) for t in range(1, s))
    assert (1 << (w * s - 2)) <= X < (1 << (w * s - 1))    # the row maximum has exponent 0
    assert ozaki.balanced_digits(X, s, w) == [top] + [low] * (s - 1)
    sh = 64 * L + 1 - w * s                                  # a = X 2^(1 - ws) = M 2^(-64L)
    M = X << sh if sh >= 0 else X >> (-sh)
    assert (M << (-sh) if sh < 0 else M >> sh) == X and M >> (64 * L - 1) == 1
    return [(M >> (64 * j)) & 0xFFFFFFFFFFFFFFFF for j in range(L)]


@pytest.mark.parametrize("kernel", ["auto", "mma_sync"])
@pytest.mark.parametrize("method", ["4m", "3m"])
def test_largest_digits_fill_the_fp32_chunk_exactly(kernel, method):
    """9-bit digits all -256 (top digit 200), equal signs, k = 512: every 256-element fp32
    chunk of the tensor cores sums to exactly 2^24; group sums equal O2, output equals O1."""
    p, k, s_ = 256, 512, 29
    L = si.limbs_for(p)
    limbs = _digit_pattern_mantissa(200, -256, s_, 9, L)
    A = si.random_matrix(6, k, p, 361)
    B = si.random_matrix(k, 5, p, 362)
    for X in (A, B):
        for j in range(L):
            X.limb[:, j] = np.uint64(limbs[j])
        X.sign[:] = 0
        X.exp[:] = 0
    B.sign[1] = 1
    params = dict(kernel=kernel, slices=s_, digit_bits=9)
    C, ws, st = gu.run(A, B, p, method, "ozaki", params=params)
    pl = gu.plan(A, B, p, method, params=params)
    r = ozaki.ozaki_cgemm(A, B, p, method, s=s_, w=9, fallback=lambda i, j: ((0, 0), (0, 0)))
    _check_group_sums(ws, pl, r, A.rows, B.cols)
    _check_against_o1(C, A, B, p)


@pytest.mark.parametrize("kernel", ["auto", "tcgen05", "mma_sync"])
def test_group_cap_stage_parity(kernel):
    """Groups capped at 5 pairs: every group sum still equals O2's (same cap)."""
    p = 256
    A = si.random_matrix(130, 300, p, 341, "uniform_exp")
    B = si.random_matrix(300, 140, p, 342, "uniform_exp")
    params = dict(max_group=5, kernel=kernel)
    C, ws, st = gu.run(A, B, p, "3m", "ozaki", params=params)
    pl = gu.plan(A, B, p, "3m", params=params)
    r = ozaki.ozaki_cgemm(A, B, p, "3m", max_group=5, fallback=lambda i, j: ((0, 0), (0, 0)))
    assert all(g.count <= 5 for pr in r.params.products for g in r.groups[pr])
    _check_group_sums(ws, pl, r, A.rows, B.cols)
    _check_against_o1(C, A, B, p)


@pytest.mark.parametrize("method", ["4m", "3m"])
def test_forced_fallbacks_stay_exact(method):
    """Two guard bits: many components fail certification and are recomputed exactly."""
    p = 128
    A = si.random_matrix(40, 33, p, 321, "uniform_exp")
    B = si.random_matrix(33, 50, p, 322, "uniform_exp")
    C, ws, st = gu.run(A, B, p, method, "ozaki", params=dict(guard_bits=1))
    r = ozaki.ozaki_cgemm(A, B, p, method, guard=1, fallback=lambda i, j: ((0, 0), (0, 0)))
    assert st["fallback_entries"] == int((~r.certified).sum()) > 0
    _check_against_o1(C, A, B, p)


def test_full_pair_set_lossless_is_exact_without_fallback():
    p = 128
    A = si.random_matrix(64, 40, p, 331)
    B = si.random_matrix(40, 64, p, 332)
    prm = ozaki.make_params(p, 40, "4m", guard=70)
    C, ws, st = gu.run(A, B, p, "4m", "ozaki", params=dict(guard_bits=70, cut_level=2 * prm.s))
    assert st["fallback_entries"] == 0
    _check_against_o1(C, A, B, p)


def test_methods_and_algorithms_agree_bitwise():
    p = 320
    A = si.random_matrix(150, 140, p, 341, "uniform_exp")
    B = si.random_matrix(140, 130, p, 342, "uniform_exp")
    outs = [gu.run(A, B, p, m_, a_)[0] for m_, a_ in (("4m", "ozaki"), ("3m", "ozaki"), ("4m", "plain"),
                                                       ("3m", "plain"))]
    assert all(gu.same(outs[0], o) for o in outs[1:])
    _check_against_o1(outs[0], A, B, p)


# ------------------------------------------------------------------ edge cases

@pytest.mark.parametrize("algo", ["ozaki", "plain"])
def test_k_zero_gives_zero(algo):
    p = 128
    A = si.random_matrix(5, 0, p, 1)
    B = si.random_matrix(0, 7, p, 2)
    C, ws, st = gu.run(A, B, p, "4m", algo)
    assert not C.limb.any() and not C.sign.any() and np.all(C.exp == si.INT32_MIN)


@pytest.mark.parametrize("algo,method", [("ozaki", "4m"), ("ozaki", "3m"), ("plain", "4m"), ("plain", "3m")])
def test_zero_rows_columns_identity_and_padded_ld(algo, method):
    p = 256
    A = si.random_matrix(20, 20, p, 351, "uniform_exp")
    A.limb[:, :, 3, :] = 0          # zero row
    A.limb[0, :, 7, :] = 0          # row with a zero real part
    B = si.identity_matrix(20, p)
    C, ws, st = gu.run(A, B, p, method, algo, ld_pad=5)
    Aref = exact.rounded_cgemm(A, si.identity_matrix(20, p), p)
    assert gu.same(C, Aref)
    B2 = si.random_matrix(20, 9, p, 352)
    B2.limb[:, :, :, 4] = 0          # zero column
    C2, _, _ = gu.run(A, B2, p, method, algo)
    _check_against_o1(C2, A, B2, p)


@pytest.mark.parametrize("algo,method", [("ozaki", "4m"), ("ozaki", "3m"), ("plain", "4m"), ("plain", "3m")])
def test_tiny_and_one_by_one(algo, method):
    for (m, k, n, p) in ((1, 1, 1, 64), (1, 3, 2, 1), (3, 1, 2, 1000), (2, 2, 2, 65)):
        A = si.random_matrix(m, k, p, 360 + m, "uniform_exp")
        B = si.random_matrix(k, n, p, 370 + n, "uniform_exp")
        C, _, _ = gu.run(A, B, p, method, algo)
        assert gu.same(C, exact.rounded_cgemm(A, B, p)), (m, k, n, p)


@pytest.mark.parametrize("algo,method", [("ozaki", "4m"), ("ozaki", "3m"), ("plain", "4m"), ("plain", "3m")])
def test_huge_exponent_spread(algo, method):
    """Exponents over +-3000: lossy splits, uncertified entries, exact fallbacks."""
    p = 128
    A = si.random_matrix(24, 16, p, 381, "uniform_exp", emin=-3000, emax=3000)
    B = si.random_matrix(16, 20, p, 382, "uniform_exp", emin=-3000, emax=3000)
    C, ws, st = gu.run(A, B, p, method, algo)
    _check_against_o1(C, A, B, p)


@pytest.mark.parametrize("algo", ["ozaki", "plain"])
def test_spread_beyond_the_fallback_window(algo):
    """Exponents over +-8000: a dot product's terms span more than the exact fallback's
    12 288-bit window, which keeps the top of the sum and drops each term's bits below it
    (less than one unit of the window per term); the rounding is certified against that
    bound, so every component is RN_p of the exact value and none is uncertified."""
    p = 128
    A = si.random_matrix(20, 16, p, 383, "uniform_exp", emin=-8000, emax=8000)
    B = si.random_matrix(16, 18, p, 384, "uniform_exp", emin=-8000, emax=8000)
    C, ws, st = gu.run(A, B, p, "4m", algo)
    assert st["fallback_entries"] > 0 and st["uncertified"] == 0
    _check_against_o1(C, A, B, p)


@pytest.mark.parametrize("algo", ["ozaki", "plain"])
def test_exponent_overflow_sets_status(algo):
    p = 128
    A = si.random_matrix(3, 4, p, 391)
    B = si.random_matrix(4, 3, p, 392)
    A.exp[:] = 2 ** 30 + 7
    B.exp[:] = 2 ** 30 + 7
    C, ws, st = gu.run(A, B, p, "4m", algo)
    assert st["erange"] == 1


# ------------------------------------------------------------------ full sizes, sampled

def _sampled(C, A, B, p, n_samples, seed):
    ent = gu.sampled_entries(A.rows, B.cols, n_samples, seed)
    sg, ex, li = c_oracle.rounded_cgemm(A, B, p, ent)
    gs, ge, gl = gu.take_entries(C, ent)
    bad = np.argwhere(np.any(gl != li, axis=1) | (gs != sg) | (ge != ex))
    assert len(bad) == 0, f"{len(bad)} sampled components differ, first {bad[:4].tolist()}"


_INPUTS = {}


def _config(name):
    if name not in _INPUTS:
        _INPUTS.clear()   # one full-size input set at a time
        _INPUTS[name] = si.make_config(name)
    return _INPUTS[name]


# every (n, p) the benchmark times, with both methods and both algorithms, at the
# size and in the launch configuration it times them (default kernel choice)
BENCH_CONFIGS = [f"c2_{n}_p{p}" for n in (1024, 2048) for p in (256, 512, 1024)]


@pytest.mark.parametrize("algo,method", [("ozaki", "3m"), ("ozaki", "4m"), ("plain", "3m"), ("plain", "4m")])
@pytest.mark.parametrize("name", BENCH_CONFIGS)
def test_bench_configs_sampled(name, algo, method):
    """Sampled entries (both components, the corner entries always among them) equal the
    exact C oracle bit for bit; the device status shows no uncertified rounding."""
    A, B, p = _config(name)
    C, ws, st = gu.run(A, B, p, method, algo)
    assert st["uncertified"] == 0 and st["fallback_overflow"] == 0 and st["device_timeout"] == 0
    _sampled(C, A, B, p, 48 if A.rows == 2048 else 96, 7 + len(name) + 3 * (algo == "plain") + (method == "4m"))


@pytest.mark.parametrize("method", ["4m", "3m"])
def test_long_k_switches_to_8bit_digits(method):
    """k >= 2^15: one 9-bit slice pair could reach k 2^16 > 2^31, so the plan takes
    8-bit digits (groups of 3 pairs at k = 40000, 15-k-block chunks); every entry is
    checked against the exact C oracle."""
    k, p = 40000, 128
    A = si.random_matrix(8, k, p, 371, "uniform_exp")
    B = si.random_matrix(k, 6, p, 372, "uniform_exp")
    pl = gu.plan(A, B, p, method)
    assert pl["digit_bits"] == 8 and pl["gmax"] == 3
    C, ws, st = gu.run(A, B, p, method, "ozaki")
    assert st["uncertified"] == 0 and st["fallback_overflow"] == 0 and st["device_timeout"] == 0
    ent = np.array([(i, j) for i in range(A.rows) for j in range(B.cols)])
    sg, ex, li = c_oracle.rounded_cgemm(A, B, p, ent)
    gs, ge, gl = gu.take_entries(C, ent)
    assert np.array_equal(gs, sg) and np.array_equal(ge, ex) and np.array_equal(gl, li)


@pytest.mark.parametrize("method", ["4m", "3m"])
def test_accumulators_equal_o2(method):
    """The exact accumulators of the accumulation stage (before rounding) equal O2's
    accumulators Acc = sum over groups of +-G 2^(w (Q - q)), element by element, for both
    components: this pins the fold separately from the certified rounding."""
    p = 192
    A = si.random_matrix(96, 200, p, 331, "uniform_exp")
    B = si.random_matrix(200, 72, p, 332, "uniform_exp")
    params = dict(dump_accumulators=1)
    C, ws, st = gu.run(A, B, p, method, "ozaki", params=params)
    pl = gu.plan(A, B, p, method, params=params)
    assert pl["off_acc_dump"] > 0
    r = ozaki.ozaki_cgemm(A, B, p, method)
    acc = gu.ws_accumulators(ws, pl, A.rows, B.cols)
    for c, comp in enumerate(("re", "im")):
        bad = np.argwhere(acc[c] != r.acc[comp])
        assert len(bad) == 0, f"{comp}: {len(bad)} accumulators differ, first {bad[:4].tolist()}"
    _check_against_o1(C, A, B, p)
