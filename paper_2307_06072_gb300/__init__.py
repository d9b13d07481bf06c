"""Arbitrary-precision complex GEMM on GB300 (sm_103a): Ozaki scheme (4M / 3M) and plain.

C := RN_p(A B) for complex matrices whose real and imaginary parts are p-bit
binary floating-point numbers (Kouya, Sec. III).  The computation runs in the
CUDA library ``libmpcgemm.so`` behind a C ABI (``include/mpcgemm.h``); this
package only marshals arguments.  PyTorch provides device memory and streams.

    import paper_2307_06072_gb300 as mp
    A = mp.DeviceMatrix.from_host(sign, exp, limb)        # numpy arrays
    C = mp.DeviceMatrix.empty(m, n, p)
    mp.mpcgemm(A, B, C, p, method="3m", algo="ozaki")
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass

import numpy as np

from . import _native
from ._native import MPCError, check, lib, oz_params, strerror  # noqa: F401

__all__ = ["DeviceMatrix", "mpcgemm", "mpcgemm_batched", "batched_workspace", "mpcgesv", "workspace_size", "plan",
           "read_status", "strerror", "version", "MPCError", "Workspace"]


def _torch():
    import torch
    return torch


def limbs_for(p: int) -> int:
    return (p + 63) // 64


@dataclass
class DeviceMatrix:
    """A complex matrix in the library's number format, in device memory.

    sign: (2, rows, ld) uint8, exp: (2, rows, ld) int32, limb: (2, L, rows, ld)
    int64 (bit pattern of the uint64 limbs); element (r, c) at r * ld + c.
    """
    rows: int
    cols: int
    p: int
    sign: object
    exp: object
    limb: object

    @property
    def ld(self) -> int:
        return int(self.sign.shape[2])

    @property
    def L(self) -> int:
        return int(self.limb.shape[1])

    @staticmethod
    def empty(rows: int, cols: int, p: int, device="cuda", ld: int | None = None) -> "DeviceMatrix":
        torch = _torch()
        ld = cols if ld is None else ld
        L = limbs_for(p)
        return DeviceMatrix(rows, cols, p,
                            torch.zeros((2, rows, ld), dtype=torch.uint8, device=device),
                            torch.zeros((2, rows, ld), dtype=torch.int32, device=device),
                            torch.zeros((2, L, rows, ld), dtype=torch.int64, device=device))

    @staticmethod
    def from_host(sign: np.ndarray, exp: np.ndarray, limb: np.ndarray, p: int | None = None,
                  device="cuda", non_blocking: bool = False) -> "DeviceMatrix":
        torch = _torch()
        _, rows, cols = sign.shape
        L = limb.shape[1]
        p = 64 * L if p is None else p
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(device, non_blocking=non_blocking)
        return DeviceMatrix(rows, cols, p, t(sign.astype(np.uint8)), t(exp.astype(np.int32)),
                            t(limb.view(np.int64)))

    @staticmethod
    def from_mpc(mat, device="cuda") -> "DeviceMatrix":
        """From any object with numpy ``sign``, ``exp``, ``limb`` arrays and ``p``."""
        return DeviceMatrix.from_host(mat.sign, mat.exp, mat.limb, mat.p, device)

    def to_host(self):
        """(sign uint8, exp int32, limb uint64) numpy arrays over the rows x cols part."""
        s = self.sign[:, :, : self.cols].cpu().numpy()
        e = self.exp[:, :, : self.cols].cpu().numpy()
        l = self.limb[:, :, :, : self.cols].cpu().numpy().view(np.uint64)
        return np.ascontiguousarray(s), np.ascontiguousarray(e), np.ascontiguousarray(l)

    def struct(self) -> _native.MpcMat:
        m = _native.MpcMat()
        m.rows, m.cols, m.ld = self.rows, self.cols, self.ld
        for c in range(2):
            m.sign[c] = self.sign[c].data_ptr()
            m.exp[c] = self.exp[c].data_ptr()
            m.limb[c] = self.limb[c].data_ptr()
        return m


class Workspace:
    """Caller-owned scratch memory for mpcgemm (a device byte tensor, grown on demand)."""

    def __init__(self, device="cuda"):
        self.device = device
        self.tensor = None

    def get(self, nbytes: int):
        torch = _torch()
        if self.tensor is None or self.tensor.numel() < nbytes:
            self.tensor = None
            self.tensor = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=self.device)
        return self.tensor

    @property
    def ptr(self) -> int:
        return self.tensor.data_ptr()

    @property
    def nbytes(self) -> int:
        return self.tensor.numel()


def _stream_handle(stream) -> int | None:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else (int(stream) if stream else None)


def workspace_size(m, n, k, p, method="4m", algo="ozaki", params=None) -> int:
    return int(plan(m, n, k, p, method, algo, params)["ws_bytes"])


def plan(m, n, k, p, method="4m", algo="ozaki", params=None) -> dict:
    out = _native.Plan()
    prm = params if params is None or isinstance(params, _native.OzParams) else oz_params(**params)
    check(lib().mpcgemm_plan(m, n, k, p, _native.METHODS[method], _native.ALGOS[algo],
                             ctypes.byref(prm) if prm is not None else None, ctypes.byref(out)))
    return out.as_dict()


def mpcgemm(A: DeviceMatrix, B: DeviceMatrix, C: DeviceMatrix, p: int, method: str = "4m",
            algo: str = "ozaki", workspace: Workspace | None = None, stream=None, params=None,
            check_status: bool = False, events=None) -> Workspace:
    """C := RN_p(A B) on the device (asynchronous on ``stream``).  Returns the workspace used.

    ``events``: optional list of up to 8 ``torch.cuda.Event(enable_timing=True)``
    (or None entries) recorded at the stage boundaries (see mpc_stage_events).
    """
    m, k, n = A.rows, A.cols, B.cols
    prm = params if params is None or isinstance(params, _native.OzParams) else oz_params(**params)
    need = workspace_size(m, n, k, p, method, algo, prm)
    ws = workspace if workspace is not None else Workspace(A.sign.device)
    t = ws.get(need)
    sa, sb, sc = A.struct(), B.struct(), C.struct()
    ev = None
    if events is not None:
        ev = _native.StageEvents()
        torch = _torch()
        for x, e in enumerate(events[:8]):
            if e is not None and not int(e.cuda_event):
                e.record(stream if stream is not None else torch.cuda.current_stream())  # creates the event
            ev.ev[x] = int(e.cuda_event) if e is not None else None
    code = lib().mpcgemm_profiled(m, n, k, p, ctypes.byref(sa), ctypes.byref(sb), ctypes.byref(sc),
                                  _native.METHODS[method], _native.ALGOS[algo],
                                  ctypes.byref(prm) if prm is not None else None,
                                  ctypes.byref(ev) if ev is not None else None, t.data_ptr(), t.numel(),
                                  _stream_handle(stream))
    check(code)
    if check_status:
        st = read_status(ws, stream)
        if st["erange"]:
            raise MPCError(_native.MPC_ERANGE)
    return ws


def _problems(problems):
    """ctypes array of mpc_problem (and the structs it points to, kept alive)."""
    arr = (_native.MpcProblem * len(problems))()
    keep = []
    for x, (A, B, C, p, method, algo) in enumerate(problems):
        sa, sb, sc = A.struct(), B.struct(), C.struct()
        keep += [sa, sb, sc]
        arr[x] = _native.MpcProblem(A.rows, B.cols, A.cols, p, _native.METHODS[method], _native.ALGOS[algo], 0,
                                    ctypes.addressof(sa), ctypes.addressof(sb), ctypes.addressof(sc))
    return arr, keep


def batched_workspace(problems, params=None):
    """(total bytes, per-problem offsets) for ``mpcgemm_batched``."""
    arr, keep = _problems(problems)
    prm = params if params is None or isinstance(params, _native.OzParams) else oz_params(**params)
    offs = (ctypes.c_uint64 * max(1, len(problems)))()
    total = ctypes.c_size_t()
    check(lib().mpcgemm_batched_workspace(len(problems), arr, ctypes.byref(prm) if prm is not None else None,
                                          offs, ctypes.byref(total)))
    return int(total.value), [int(offs[x]) for x in range(len(problems))]


def mpcgemm_batched(problems, params=None, workspace: Workspace | None = None, stream=None) -> Workspace:
    """Many complex GEMMs in one call; ``problems``: list of (A, B, C, p, method, algo).

    The Ozaki problems share one persistent tcgen05 launch.  Asynchronous and
    allocation-free inside the library, so it can be captured in a CUDA graph.
    """
    arr, keep = _problems(problems)
    prm = params if params is None or isinstance(params, _native.OzParams) else oz_params(**params)
    total, _ = batched_workspace(problems, prm)
    ws = workspace if workspace is not None else Workspace(problems[0][0].sign.device)
    t = ws.get(total)
    check(lib().mpcgemm_batched(len(problems), arr, ctypes.byref(prm) if prm is not None else None, t.data_ptr(),
                                t.numel(), _stream_handle(stream)))
    return ws


def read_status(workspace: Workspace, stream=None, offset: int = 0) -> dict:
    """Device status of the last call on this workspace (``offset``: a batched problem's region)."""
    st = _native.Status()
    code = lib().mpcgemm_read_status(workspace.ptr + offset, workspace.nbytes - offset, ctypes.byref(st),
                                     _stream_handle(stream))
    if code not in (_native.MPC_OK, _native.MPC_ERANGE):
        check(code)
    return {"erange": st.erange, "fallback_entries": st.fallback_entries,
            "fallback_overflow": st.fallback_overflow, "uncertified": st.uncertified,
            "device_timeout": st.device_timeout}


def mpcgesv(A: DeviceMatrix, B: DeviceMatrix, p: int, block: int = 128, method: str = "3m",
            workspace: Workspace | None = None, stream=None):
    """Solve A X = B in place (A <- LU factors, B <- X); returns (ipiv tensor, workspace)."""
    torch = _torch()
    n = A.rows
    need = int(lib().mpcgesv_workspace_size(n, p, block, _native.METHODS[method]))
    if need == 0 and n > 0:
        raise MPCError(_native.MPC_EINVAL)
    ws = workspace if workspace is not None else Workspace(A.sign.device)
    t = ws.get(max(need, 256))
    ipiv = torch.zeros(max(n, 1), dtype=torch.int32, device=A.sign.device)
    sa, sb = A.struct(), B.struct()
    check(lib().mpcgesv(n, p, ctypes.byref(sa), ipiv.data_ptr(), ctypes.byref(sb), block, _native.METHODS[method],
                        t.data_ptr(), t.numel(), _stream_handle(stream)))
    return ipiv[:n], ws


def lu_singular_column(workspace: Workspace) -> int:
    """1 + the first column whose pivot was zero (0 if none); synchronises."""
    torch = _torch()
    torch.cuda.synchronize()
    return int(workspace.tensor[20:24].view(torch.int32).item())


def version() -> int:
    return int(lib().mpcgemm_version())
