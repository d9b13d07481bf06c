"""Helpers for the GPU tests: run the C ABI on MPCMatrix inputs, read stages back."""
import numpy as np

from synthetic_inputs import MPCMatrix


def mp():
    from paper_2307_06072_gb300 import build
    build.build()
    import paper_2307_06072_gb300 as m
    return m


def run(A, B, p, method="4m", algo="ozaki", params=None, ld_pad=0):
    import torch
    M = mp()
    m, k, n = A.rows, A.cols, B.cols
    dA = M.DeviceMatrix.from_mpc(A)
    dB = M.DeviceMatrix.from_mpc(B)
    dC = M.DeviceMatrix.empty(m, n, p, ld=n + ld_pad)
    ws = M.mpcgemm(dA, dB, dC, p, method, algo, params=params)
    status = M.read_status(ws)
    torch.cuda.synchronize()
    s, e, l = dC.to_host()
    return MPCMatrix(m, n, p, s, e, l), ws, status


def plan(A, B, p, method, algo="ozaki", params=None):
    return mp().plan(A.rows, B.cols, A.cols, p, method, algo, params)


def ws_digits(ws, pl, side, lines):
    import torch
    off = pl["off_digits_a"] if side == "A" else pl["off_digits_b"]
    planes = pl["planes_A"] if side == "A" else pl["planes_B"]
    cnt = planes * lines * pl["kpad"]
    raw = ws.tensor[off: off + 2 * cnt].view(torch.bfloat16).float().cpu().numpy()
    return raw.reshape(planes, lines, pl["kpad"]).astype(np.int64)


def ws_groups(ws, pl, m, n):
    import torch
    off = pl["off_groups"]
    cnt = pl["n_groups_total"] * m * n
    return ws.tensor[off: off + 4 * cnt].view(torch.int32).cpu().numpy().reshape(-1, m, n)


def ws_group_tables(ws, pl):
    """(table [G, 4] = (product, level, first t, count), accumulation order [G], unit schedule [G])."""
    import torch
    G = pl["n_groups_total"]
    t = ws.tensor[pl["off_group_table"]: pl["off_group_table"] + 16 * G].view(torch.int32).cpu().numpy()
    o = ws.tensor[pl["off_group_order"]: pl["off_group_order"] + 8 * G].view(torch.int32).cpu().numpy()
    return t.reshape(G, 4), o[:G], o[G:]


def ws_lossy(ws, pl, m, n):
    import torch
    a = ws.tensor[pl["off_rowlossy"]: pl["off_rowlossy"] + 4 * m].view(torch.int32).cpu().numpy()
    b = ws.tensor[pl["off_collossy"]: pl["off_collossy"] + 4 * n].view(torch.int32).cpu().numpy()
    return a, b


def same(X, Y):
    return (np.array_equal(X.sign, Y.sign) and np.array_equal(X.exp, Y.exp)
            and np.array_equal(X.limb, Y.limb))


def mismatches(X, Y):
    bad = np.any(X.limb != Y.limb, axis=1) | (X.sign != Y.sign) | (X.exp != Y.exp)
    return np.argwhere(bad)


def take_entries(C, entries):
    """(sign[2, N], exp[2, N], limb[2, L, N]) of listed (i, j) entries."""
    ii, jj = entries[:, 0], entries[:, 1]
    return C.sign[:, ii, jj], C.exp[:, ii, jj], C.limb[:, :, ii, jj]


def ws_accumulators(ws, pl, m, n):
    """Exact accumulators dumped by the accumulation stage: object array [2, m, n] of Python ints."""
    import torch
    ns = pl["acc_slots"] + 1
    off = pl["off_acc_dump"]
    raw = ws.tensor[off: off + 4 * 2 * m * n * ns].view(torch.int32).cpu().numpy().view(np.uint32)
    raw = raw.reshape(m, n, 2, ns)
    out = np.zeros((2, m, n), dtype=object)
    for i in range(m):
        for j in range(n):
            for c in range(2):
                w = raw[i, j, c]
                v = int.from_bytes(w[:-1].astype("<u4").tobytes(), "little")
                out[c, i, j] = -v if w[-1] else v
    return out


def sampled_entries(m, n, count, seed):
    """`count` random output entries, the first and last one always included."""
    rng = np.random.default_rng(seed)
    ent = np.stack([rng.integers(0, m, count), rng.integers(0, n, count)], axis=1)
    ent[0] = (0, 0)
    ent[1] = (m - 1, n - 1)
    return ent
