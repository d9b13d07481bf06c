"""C-ABI library: builds, loads without a GPU, exports every declared symbol,
rejects bad arguments on the host, and plans like the oracle (no GPU compute)."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle import ozaki

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "mpcgemm.h")


@pytest.fixture(scope="module")
def mp():
    from paper_2307_06072_gb300 import build
    build.build()
    import paper_2307_06072_gb300 as mp
    return mp


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mpcge(?:mm|sv)\w*)\s*\(", src)))


def test_every_declared_symbol_is_exported(mp):
    names = declared_functions()
    assert "mpcgemm" in names and "mpcgemm_plan" in names and len(names) >= 8
    lib = ctypes.CDLL(mp._native.LIB_PATH)
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(mp._native.EXPORTED)


def test_version_and_strerror(mp):
    assert mp.version() >= 100
    assert "workspace" in mp.strerror(-28)
    assert "exponent" in mp.strerror(-34)


def _dummy_mat(rows, cols, ld=None):
    m = mp_native().MpcMat()
    m.rows, m.cols, m.ld = rows, cols, cols if ld is None else ld
    for c in range(2):
        m.sign[c] = m.exp[c] = m.limb[c] = 0x1000 * (c + 1)   # never dereferenced
    return m


def mp_native():
    import paper_2307_06072_gb300._native as n
    return n


@pytest.mark.parametrize("m,n,k,p,method,algo,code", [
    (4, 4, 4, 0, 0, 1, -22), (4, 4, 4, 1025, 0, 1, -22), (4, 4, 131072, 128, 0, 1, -22),
    (4, 4, 4, 128, 2, 1, -22), (4, 4, 4, 128, 0, 2, -22), (-1, 4, 4, 128, 0, 1, -22)])
def test_bad_arguments_rejected_on_host(mp, m, n, k, p, method, algo, code):
    A, B, C = _dummy_mat(max(m, 0), max(k, 0)), _dummy_mat(max(k, 0), n), _dummy_mat(max(m, 0), n)
    rc = mp.lib().mpcgemm(m, n, k, p, ctypes.byref(A), ctypes.byref(B), ctypes.byref(C), method, algo,
                          ctypes.c_void_p(0x100000), 1 << 40, None)
    assert rc == code


def test_shape_mismatch_and_workspace_checks(mp):
    A, B, C = _dummy_mat(8, 5), _dummy_mat(6, 7), _dummy_mat(8, 7)
    lib = mp.lib()
    assert lib.mpcgemm(8, 7, 5, 128, ctypes.byref(A), ctypes.byref(B), ctypes.byref(C), 0, 1,
                       ctypes.c_void_p(0x100000), 1 << 40, None) == -22
    B = _dummy_mat(5, 7)
    Cbad = _dummy_mat(8, 7, ld=3)
    assert lib.mpcgemm(8, 7, 5, 128, ctypes.byref(A), ctypes.byref(B), ctypes.byref(Cbad), 0, 1,
                       ctypes.c_void_p(0x100000), 1 << 40, None) == -22
    need = lib.mpcgemm_workspace_size(8, 7, 5, 128, 0, 1)
    assert need > 0
    assert lib.mpcgemm(8, 7, 5, 128, ctypes.byref(A), ctypes.byref(B), ctypes.byref(C), 0, 1,
                       ctypes.c_void_p(0x100000), need - 1, None) == -28
    assert lib.mpcgemm(8, 7, 5, 128, ctypes.byref(A), ctypes.byref(B), ctypes.byref(C), 0, 1,
                       ctypes.c_void_p(0x100001), need, None) == -22   # misaligned workspace
    # m == 0: a no-op that succeeds without touching anything
    Z = _dummy_mat(0, 5)
    Cz = _dummy_mat(0, 7)
    assert lib.mpcgemm(0, 7, 5, 128, ctypes.byref(Z), ctypes.byref(B), ctypes.byref(Cz), 0, 1,
                       ctypes.c_void_p(0x100000), need, None) == 0


@pytest.mark.parametrize("p,k,method,guard,s,Q,w", [
    (128, 32, "4m", None, None, None, None), (256, 256, "4m", None, None, None, None),
    (256, 256, "3m", None, None, None, None), (1024, 2048, "3m", None, None, None, None),
    (1024, 2048, "3m", None, None, None, 8), (512, 1024, "4m", 8, None, None, None),
    (128, 9, "3m", 0, None, 3, None), (128, 8, "4m", None, 10, 18, None), (192, 2048, "3m", None, 30, 33, 8),
    (256, 40000, "4m", None, None, None, None),
    (128, 131071, "3m", None, None, None, None)])   # the largest k: 8-bit digits, one pair per group
def test_plan_matches_the_oracle_parameters(mp, p, k, method, guard, s, Q, w):
    """Digit width, s, Q, group counts and bound constants of the C plan equal O2's
    (w = 9 by default, 8 when k >= 2^15 or when asked for)."""
    prm = ozaki.make_params(p, k, method, guard if guard is not None else ozaki.DEFAULT_GUARD, s, Q, w=w)
    params = dict(guard_bits=guard or 0, slices=s or 0, cut_level=(Q + 1) if Q is not None else 0,
                  digit_bits=w or 0)
    if guard == 0:
        params["guard_bits"] = 0
        prm = ozaki.make_params(p, k, method, ozaki.DEFAULT_GUARD, s, Q, w=w)   # 0 means default in the ABI
    pl = mp.plan(64, 48, k, p, method, "ozaki", params)
    assert pl["digit_bits"] == prm.w == (w or (9 if k < 32768 else 8))
    assert (pl["s"], pl["Q"], pl["gmax"]) == (prm.s, prm.Q, prm.gmax)
    first = {"re": 0, "im": 0, "sum": -1}
    npos = {"re": prm.s, "im": prm.s, "sum": prm.s + 1}
    for idx, pr in enumerate(prm.products):
        wa, wb = ozaki.PRODUCT_OPERANDS[pr]
        gs = ozaki.groups_for((first[wa], first[wa] + npos[wa] - 1), (first[wb], first[wb] + npos[wb] - 1),
                              prm.Q, prm.gmax)
        assert pl["n_groups"][idx] == len(gs)
    # the bound constants: compare with entry_bound on synthetic split summaries
    class FakeSplit:
        def __init__(self, lossless):
            self.E = [0]
            self.lossless = [lossless]
            self.first_pos = first
            self.digits = {w: np.zeros((npos[w], 1, 1)) for w in ("re", "im", "sum")}
            # the plan's constants are the data-independent upper bound: every plane and component live
            self.live = {w: [True] * npos[w] for w in ("re", "im", "sum")}
            self.values = (True, True)
    for la in (True, False):
        for lb in (True, False):
            for c, comp in enumerate(("re", "im")):
                b, beta = ozaki.entry_bound(prm, FakeSplit(la), FakeSplit(lb), 0, 0, comp)
                want = pl["bound_drop"][c] + k * ((0 if la else pl["bound_lossy_a"][c]) +
                                                  (0 if lb else pl["bound_lossy_b"][c]))
                assert (b, beta) == (want, pl["bound_shift"])


def test_lu_arguments_checked_on_host(mp):
    """mpcgesv rejects bad arguments before any launch (no GPU needed to see it)."""
    n = mp_native()
    lib = n.lib()
    lib.mpcgesv_workspace_size.restype = ctypes.c_size_t
    lib.mpcgesv_workspace_size.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_int32, ctypes.c_int]
    M3 = n.METHODS["3m"]
    for args in [(-1, 128, 16, M3), (8, 0, 16, M3), (8, 1025, 16, M3), (8, 128, 0, M3), (8, 128, 16, 7)]:
        assert lib.mpcgesv_workspace_size(*args) == 0, args
    need = lib.mpcgesv_workspace_size(64, 256, 16, M3)
    assert need > 0 and lib.mpcgesv_workspace_size(128, 256, 16, M3) > need
    lib.mpcgesv.restype = ctypes.c_int
    lib.mpcgesv.argtypes = [ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                            ctypes.c_int32, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p]
    A, B = _dummy_mat(64, 64), _dummy_mat(64, 2)
    ipiv, ws = ctypes.c_void_p(0x2000), ctypes.c_void_p(0x100000)
    call = lambda nn, a, b, piv, w, wb, p=256: lib.mpcgesv(nn, p, a, piv, b, 16, M3, w, wb, None)
    assert call(64, None, ctypes.byref(B), ipiv, ws, need) == n.MPC_EINVAL                  # no A
    assert call(64, ctypes.byref(_dummy_mat(64, 63)), ctypes.byref(B), ipiv, ws, need) == n.MPC_EINVAL
    assert call(64, ctypes.byref(A), ctypes.byref(_dummy_mat(63, 2)), ipiv, ws, need) == n.MPC_EINVAL
    assert call(64, ctypes.byref(A), ctypes.byref(B), None, ws, need) == n.MPC_EINVAL        # no ipiv
    assert call(64, ctypes.byref(A), ctypes.byref(B), ipiv, ctypes.c_void_p(0x100010), need) == n.MPC_EINVAL
    assert call(64, ctypes.byref(A), ctypes.byref(B), ipiv, ws, need - 1) == n.MPC_ENOSPC
    assert call(64, ctypes.byref(A), ctypes.byref(B), ipiv, ws, need, p=2000) == n.MPC_EINVAL
    Z = _dummy_mat(0, 0)
    assert call(0, ctypes.byref(Z), ctypes.byref(_dummy_mat(0, 1)), None, None, 0) == n.MPC_OK   # empty: no-op


def test_batched_arguments_checked_on_host(mp):
    """mpcgemm_batched plans and checks every problem before its first launch."""
    n = mp_native()
    lib = n.lib()
    keep = []

    def problem(m, nn, k, p=256, method="3m", algo="ozaki"):
        A, B, C = _dummy_mat(m, k), _dummy_mat(k, nn), _dummy_mat(m, nn)
        keep.extend([A, B, C])
        return n.MpcProblem(m, nn, k, p, n.METHODS[method], n.ALGOS[algo], 0,
                            ctypes.addressof(A), ctypes.addressof(B), ctypes.addressof(C))

    good = [problem(32, 40, 24), problem(16, 8, 64, 512, "4m")]
    arr = (n.MpcProblem * 2)(*good)
    total = ctypes.c_size_t(0)
    assert lib.mpcgemm_batched_workspace(2, arr, None, None, ctypes.byref(total)) == n.MPC_OK and total.value > 0
    ws = ctypes.c_void_p(0x100000)
    assert lib.mpcgemm_batched(-1, arr, None, ws, total.value, None) == n.MPC_EINVAL
    assert lib.mpcgemm_batched(2, None, None, ws, total.value, None) == n.MPC_EINVAL
    assert lib.mpcgemm_batched(0, None, None, None, 0, None) == n.MPC_OK                  # empty batch
    assert lib.mpcgemm_batched(2, arr, None, ws, total.value - 256, None) == n.MPC_ENOSPC
    bad = (n.MpcProblem * 2)(good[0], problem(16, 8, 64, 2000))                          # p out of range
    assert lib.mpcgemm_batched(2, bad, None, ws, total.value, None) == n.MPC_EINVAL


def test_per_part_split_plan(mp):
    """The per-part split is a 4M option: 3M is rejected on the host; a 4M plan keeps the
    default sizes (the device cuts fewer pairs, never more) and makes two more launches
    (the part offsets of A and B)."""
    import ctypes
    out = mp._native.Plan()
    prm = mp._native.oz_params(split="per_part")
    rc = mp.lib().mpcgemm_plan(64, 64, 64, 256, 1, 1, ctypes.byref(prm), ctypes.byref(out))
    assert rc == mp._native.MPC_EINVAL
    d = mp.plan(300, 200, 100, 256, "4m", "ozaki", dict(split="per_part"))
    base = mp.plan(300, 200, 100, 256, "4m", "ozaki")
    assert d["split"] == 1 and base["split"] == 0
    assert d["ws_bytes"] == base["ws_bytes"] and d["n_groups_total"] == base["n_groups_total"]
    assert d["launches"] == base["launches"] + 2
    prm.split = 3
    rc = mp.lib().mpcgemm_plan(64, 64, 64, 256, 0, 1, ctypes.byref(prm), ctypes.byref(out))
    assert rc == mp._native.MPC_EINVAL


def test_residual_split_plan(mp):
    """The residual split is a 4M option of single calls: 3M and batched calls are rejected on
    the host.  The table has one entry per kept pair (s(s+1)/2 per product at Q = s - 1; the
    device merges runs of up to gmax pairs into their first entry); the
    pair products go through a buffer of pair_batch planes, whole levels at a time, so the
    launches are init, three transposes, two splits, the table, a slice GEMM and an
    accumulation per batch, and the fallback."""
    import ctypes
    from oracle import ozaki
    out = mp._native.Plan()
    prm = mp._native.oz_params(split="residual")
    rc = mp.lib().mpcgemm_plan(64, 64, 64, 256, 1, 1, ctypes.byref(prm), ctypes.byref(out))
    assert rc == mp._native.MPC_EINVAL
    m, n, k, p = 300, 200, 100, 256
    d = mp.plan(m, n, k, p, "4m", "ozaki", dict(split="residual"))
    s, Q = d["s"], d["Q"]
    assert d["split"] == 2 and d["gmax"] == ozaki.make_params(p, k, "4m").gmax and Q == s - 1
    assert d["n_groups"] == [s * (s + 1) // 2] * 4 and d["n_groups_total"] == 2 * s * (s + 1)
    assert d["pair_batch"] == d["n_groups_total"]          # everything fits the default buffer
    assert d["launches"] == 7 + 2 + 1 and d["off_units"] > 0
    prm0 = ozaki.make_params(p, k, "4m")
    assert (s, Q) == (prm0.s, prm0.Q)
    # a buffer of 50 planes: whole levels (at most s = 33 pairs), packed greedily
    d2 = mp.plan(m, n, k, p, "4m", "ozaki", dict(split="residual", pair_planes=50))
    batches, cur = 0, 0
    for _ in range(4):
        for q, lo, cnt in ozaki.level_pairs((0, s - 1), (0, s - 1), Q):
            if cur + cnt > 50 and cur > 0:
                batches, cur = batches + 1, 0
            cur += cnt
    batches += 1
    assert d2["pair_batch"] == 50 and d2["launches"] == 7 + 2 * batches + 1
    assert d2["ws_bytes"] < d["ws_bytes"]
    d3 = mp.plan(m, n, k, p, "4m", "ozaki", dict(split="residual", pair_planes=5))
    assert d3["pair_batch"] == s                             # at least one whole level
    base = mp.plan(m, n, k, p, "4m", "ozaki")
    assert base["off_units"] == 0 and base["pair_batch"] == 0
    prm.pair_planes = -1
    rc = mp.lib().mpcgemm_plan(m, n, k, p, 0, 1, ctypes.byref(prm), ctypes.byref(out))
    assert rc == mp._native.MPC_EINVAL
    total = ctypes.c_size_t()
    prm.pair_planes = 0
    rc = mp.lib().mpcgemm_batched_workspace(0, None, ctypes.byref(prm), None, ctypes.byref(total))
    assert rc == mp._native.MPC_EINVAL
