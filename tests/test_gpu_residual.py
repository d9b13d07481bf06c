"""The residual split (mpc_oz_params.split = MPC_SPLIT_RESIDUAL, 4M) against O2r.

Alg. 2 as printed: every real part of every line is cut slice after slice with the unit
re-measured from the largest residual left in the line.  Every integer stage must equal
the emulation bit for bit: the unit of every (part, slice, line), the digit planes, the
lossy flags, the pair table with its merged runs and emptied pairs, the exact accumulators and
the number of components sent to the exact fallback; every output equals O1.  The pair
products are streamed through a bounded buffer: a run with a small buffer (many
batches, the accumulators kept in the workspace between them) gives the same bits.
Inputs: regular lines, imaginary parts 2^-100 below the real parts, lines whose elements
share a run of zero bits (their units skip it), zero rows and columns; sizes that span
several tiles with ragged edges.
"""
import numpy as np
import pytest

import synthetic_inputs as si
from oracle import c_oracle, exact, ozaki, residual
from tests import gpu_util as gu

pytestmark = pytest.mark.gpu


def _shift_im(mat, by):
    out = mat.copy()
    nz = out.limb[1, -1] != 0
    out.exp[1] = np.where(nz, out.exp[1] + by, out.exp[1]).astype(np.int32)
    return out


def _gap_matrix(rows, cols, p, seed, gap_len=70, hi_bits=24):
    """Row i: every element (H 2^gap_len + Lo) 2^x with H of hi_bits bits and Lo of a
    row-dependent width: all elements of a row share a run of gap_len zero bits."""
    rng = np.random.default_rng(seed)
    re = [[None] * cols for _ in range(rows)]
    im = [[None] * cols for _ in range(rows)]
    for i in range(rows):
        lo_bits = 4 + (7 * i) % 40
        for j in range(cols):
            for out in (re, im):
                H = int(rng.integers(1 << (hi_bits - 1), 1 << hi_bits))
                Lo = int.from_bytes(rng.bytes((lo_bits + 7) // 8), "little") & ((1 << lo_bits) - 1)
                N = (H << (gap_len + lo_bits)) + Lo
                N = -N if rng.integers(0, 2) else N
                out[i][j] = exact.round_nearest_even((N, -(hi_bits + gap_len + lo_bits)), p)
    return exact.pack(re, im, p)


def _inputs(case, p, m, k, n, seed):
    if case == "gap":
        A = _gap_matrix(m, k, p, seed)
        B = _gap_matrix(n, k, p, seed + 1).transpose()
    else:
        A = si.random_matrix(m, k, p, seed, "uniform_exp", zero_frac=0.03 if case == "zeros" else 0.0)
        B = si.random_matrix(k, n, p, seed + 1, "uniform_exp")
        if case == "im_small":
            A, B = _shift_im(A, -100), _shift_im(B, -100)
        if case == "zeros":
            A.limb[:, :, 3, :] = 0       # a zero row of A
            B.limb[:, :, :, 5] = 0       # a zero column of B
            B.limb[1, :, :, 7] = 0       # a column of B with a zero imaginary part
    return A, B


def _ws_units(ws, pl, m, n):
    import torch
    s = pl["s"]
    off = pl["off_units"]
    raw = ws.tensor[off: off + 4 * 2 * s * (m + n)].view(torch.int32).cpu().numpy()
    return raw[: 2 * s * m].reshape(2, s, m), raw[2 * s * m:].reshape(2, s, n)


def _ref_units(sp, s, lines):
    out = np.full((2, s, lines), np.iinfo(np.int32).min, np.int64)
    for c, part in enumerate(("re", "im")):
        for t in range(s):
            for i in range(lines):
                u = sp.units[part][t][i]
                if u is not None:
                    out[c, t, i] = u
    return out


@pytest.mark.parametrize("kernel", ["auto", "mma_sync"])
@pytest.mark.parametrize("case", ["regular", "im_small", "gap", "zeros"])
def test_residual_stage_parity(case, kernel):
    p = 256
    m, k, n = 150, 130, 170
    A, B = _inputs(case, p, m, k, n, 700 + len(case))
    params = dict(split="residual", dump_accumulators=1, kernel=kernel)
    C, ws, st = gu.run(A, B, p, "4m", "ozaki", params=params)
    pl = gu.plan(A, B, p, "4m", params=params)
    r = residual.ozaki_cgemm_residual(A, B, p, fallback=lambda i, j: ((0, 0), (0, 0)))
    s = r.params.s
    assert pl["s"] == s and pl["Q"] == r.params.Q
    uA, uB = _ws_units(ws, pl, m, n)
    assert np.array_equal(uA, _ref_units(r.splitA, s, m))
    assert np.array_equal(uB, _ref_units(r.splitB, s, n))
    dA, dB = gu.ws_digits(ws, pl, "A", m), gu.ws_digits(ws, pl, "B", n)
    assert np.array_equal(dA[:s, :, :k], r.splitA.digits["re"]) and np.array_equal(dA[s:, :, :k], r.splitA.digits["im"])
    assert np.array_equal(dB[:s, :, :k], r.splitB.digits["re"]) and np.array_equal(dB[s:, :, :k], r.splitB.digits["im"])
    assert not np.any(dA[:, :, k:]) and not np.any(dB[:, :, k:])
    la, lb = gu.ws_lossy(ws, pl, m, n)
    assert np.array_equal(la != 0, ~np.array(r.splitA.lossless)) and np.array_equal(lb != 0, ~np.array(r.splitB.lossless))
    table, _, _ = gu.ws_group_tables(ws, pl)
    assert len(table) == len(r.groups)
    for e, ((pr, q, t, cnt), got) in enumerate(zip(r.groups, table)):
        assert tuple(int(v) for v in got) == (residual.PRODUCTS.index(pr), q, t, cnt), e
    acc = gu.ws_accumulators(ws, pl, m, n)
    for c, comp in enumerate(("re", "im")):
        assert np.array_equal(acc[c], r.acc[comp]), comp
    assert st["fallback_entries"] == int((~r.certified).sum())
    assert st["uncertified"] == 0 and st["fallback_overflow"] == 0 and st["device_timeout"] == 0
    assert st["erange"] == 0
    assert gu.same(C, c_oracle.rounded_cgemm_matrix(A, B, p))


@pytest.mark.parametrize("case", ["regular", "im_small"])
def test_batches_of_pair_planes_give_the_same_bits(case):
    """A buffer of 3 levels' worth of planes: many batches, the exact accumulators kept in the
    workspace between them; accumulators and outputs equal the one-batch run."""
    p = 192
    A, B = _inputs(case, p, 140, 100, 300, 731)
    one = dict(split="residual", dump_accumulators=1)
    many = dict(split="residual", dump_accumulators=1, pair_planes=3 * 30)
    C1, ws1, st1 = gu.run(A, B, p, "4m", "ozaki", params=one)
    Cm, wsm, stm = gu.run(A, B, p, "4m", "ozaki", params=many)
    pl1, plm = gu.plan(A, B, p, "4m", params=one), gu.plan(A, B, p, "4m", params=many)
    assert plm["launches"] > pl1["launches"] + 10
    a1, am = gu.ws_accumulators(ws1, pl1, 140, 300), gu.ws_accumulators(wsm, plm, 140, 300)
    assert np.array_equal(a1, am)
    assert st1 == stm
    assert gu.same(C1, Cm) and gu.same(C1, c_oracle.rounded_cgemm_matrix(A, B, p))


def test_small_imaginary_parts_need_no_fallback():
    """Im = 2^-100 Re in scale: the default split certifies no imaginary component (each goes to
    the exact fallback); the residual split certifies every component.  Same bits."""
    p = 256
    A, B = _inputs("im_small", p, 96, 200, 80, 741)
    Cc, _, stc = gu.run(A, B, p, "4m", "ozaki")
    Cr, _, str_ = gu.run(A, B, p, "4m", "ozaki", params=dict(split="residual"))
    assert stc["fallback_entries"] >= A.rows * B.cols
    assert str_["fallback_entries"] == 0
    assert gu.same(Cc, Cr) and gu.same(Cr, c_oracle.rounded_cgemm_matrix(A, B, p))


@pytest.mark.parametrize("kernel", ["auto", "tcgen05_2sm"])
def test_bench_size_sampled(kernel):
    """1024^3, p = 512, imaginary parts 2^-100 below the real parts (the bench's residual leg):
    sampled entries equal the exact oracle; no component needs the fallback."""
    import torch
    M = gu.mp()
    p, nn = 512, 1024
    A = _shift_im(si.random_matrix(nn, nn, p, 751, "uniform_exp"), -100)
    B = _shift_im(si.random_matrix(nn, nn, p, 752, "uniform_exp"), -100)
    dA, dB = M.DeviceMatrix.from_mpc(A), M.DeviceMatrix.from_mpc(B)
    dC = M.DeviceMatrix.empty(nn, nn, p)
    ws = M.mpcgemm(dA, dB, dC, p, "4m", "ozaki", params=dict(split="residual", kernel=kernel))
    st = M.read_status(ws)
    torch.cuda.synchronize()
    assert st["fallback_entries"] == 0 and st["erange"] == 0 and st["device_timeout"] == 0
    s, e, l = dC.to_host()
    C = si.MPCMatrix(nn, nn, p, s, e, l)
    ent = gu.sampled_entries(nn, nn, 48, 753)
    sg, ex, li = c_oracle.rounded_cgemm(A, B, p, ent)
    gs, ge, gl = gu.take_entries(C, ent)
    assert np.array_equal(gs, sg) and np.array_equal(ge, ex) and np.array_equal(gl, li)
