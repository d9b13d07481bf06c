"""The per-part split (mpc_oz_params.split = MPC_SPLIT_PER_PART, 4M) against O2's variant.

Every integer stage must equal the emulation bit for bit: the part offsets z
(through the digit planes they place), the digit planes, the group table (the
device stores it relative to each operand's first digit position), every group
sum, the exact accumulators and the number of components sent to the exact
fallback; every output must equal O1.  Inputs: imaginary parts shifted against
the real parts by -100, -37, +45 and 0 bits (0: the split is the default one).
"""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import c_oracle, ozaki
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


def _shift_part(mat, c, by):
    out = mat.copy()
    nz = out.limb[c, -1] != 0
    out.exp[c] = np.where(nz, out.exp[c] + by, out.exp[c]).astype(np.int32)
    return out


def _inputs(shift, p, seed, m=150, k=130, n=170):
    A = _shift_part(si.random_matrix(m, k, p, seed, "uniform_exp", zero_frac=0.03), 1, shift)
    B = _shift_part(si.random_matrix(k, n, p, seed + 1, "uniform_exp"), 1, shift)
    return A, B


@pytest.mark.parametrize("kernel", ["auto", "mma_sync"])
@pytest.mark.parametrize("shift", [-100, -37, 45, 0])
def test_per_part_stage_parity(shift, kernel):
    p = 256
    A, B = _inputs(shift, p, 611 + abs(shift))
    params = dict(split="per_part", dump_accumulators=1, kernel=kernel)
    C, ws, st = gu.run(A, B, p, "4m", "ozaki", params=params)
    pl = gu.plan(A, B, p, "4m", params=params)
    r = ozaki.ozaki_cgemm(A, B, p, "4m", split="per_part", fallback=lambda i, j: ((0, 0), (0, 0)))
    s, k = r.params.s, A.cols
    za, zb = r.splitA.first_pos, r.splitB.first_pos
    if shift == 0:
        assert za == zb == {"re": 0, "im": 0}
    elif shift < 0:
        assert za["im"] > 0 and za["re"] == 0
    else:
        assert za["re"] > 0 and za["im"] == 0
    dA, dB = gu.ws_digits(ws, pl, "A", A.rows), gu.ws_digits(ws, pl, "B", B.cols)
    assert np.array_equal(dA[:s, :, :k], r.splitA.digits["re"]) and np.array_equal(dA[s:2 * s, :, :k], r.splitA.digits["im"])
    assert np.array_equal(dB[:s, :, :k], r.splitB.digits["re"]) and np.array_equal(dB[s:2 * s, :, :k], r.splitB.digits["im"])
    # group table (relative coordinates on the device) and group sums
    table, _, _ = gu.ws_group_tables(ws, pl)
    G = gu.ws_groups(ws, pl, A.rows, B.cols)
    operands = {"rr": ("re", "re"), "ii": ("im", "im"), "ri": ("re", "im"), "ir": ("im", "re")}
    e = 0
    for x, pr in enumerate(r.params.products):
        wa, wb = operands[pr]
        trimmed = ozaki.trim_groups(r.splitA, r.splitB, pr, r.groups[pr], "4m")
        for h, Gr in zip(trimmed, r.group_sums[pr]):
            got = tuple(int(v) for v in table[e])
            assert got[0] == x and got[1] == h.q - za[wa] - zb[wb] and got[3] == h.count, (pr, e, got, h)
            if h.count > 0:
                assert got[2] == h.t0 - za[wa] and np.array_equal(G[e], Gr), (pr, e)
            else:
                assert not np.any(Gr)
            e += 1
        while e < len(table) and int(table[e, 0]) == x:   # beyond the product's cut: empty entries
            assert int(table[e, 3]) == 0
            e += 1
    assert e == len(table)
    acc = gu.ws_accumulators(ws, pl, A.rows, B.cols)
    for c, comp in enumerate(("re", "im")):
        assert np.array_equal(acc[c], r.acc[comp]), comp
    assert st["fallback_entries"] == int((~r.certified).sum())
    assert st["uncertified"] == 0 and st["fallback_overflow"] == 0 and st["device_timeout"] == 0
    assert gu.same(C, c_oracle.rounded_cgemm_matrix(A, B, p))
    if shift == 0:   # no part is smaller: the default split, bit for bit
        C0, ws0, _ = gu.run(A, B, p, "4m", "ozaki", params=dict(kernel=kernel))
        assert gu.same(C, C0)
        assert np.array_equal(gu.ws_groups(ws0, gu.plan(A, B, p, "4m"), A.rows, B.cols), G)


def test_per_part_avoids_the_fallback_cliff():
    """Im = 2^-100 Re in scale: the default split certifies no imaginary component (every one
    goes to the exact fallback); the per-part split certifies them all.  Same bits."""
    p = 256
    A, B = _inputs(-100, p, 631, m=96, k=200, n=80)
    Cc, _, stc = gu.run(A, B, p, "4m", "ozaki")
    Cp, _, stp = gu.run(A, B, p, "4m", "ozaki", params=dict(split="per_part"))
    assert stc["fallback_entries"] >= A.rows * B.cols
    assert stp["fallback_entries"] == 0
    assert gu.same(Cc, Cp) and gu.same(Cp, c_oracle.rounded_cgemm_matrix(A, B, p))
