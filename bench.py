"""Benchmark: complex multiple-precision GEMM rate (8 m n k per second) on GB300.

One step = one C := RN_p(A B) through the library's C ABI, the whole hot
path: split (row/column exponents + digits), slice products on the tensor
cores, exact accumulation + certified rounding, exact fallback.

Default workload: m = n = k = 2048, p = 1024 bits, Ozaki 3M, entries
u * 2^e (u uniform on the p-bit grid of [-1, 1), e uniform in [-20, 20]),
seeded.  Ozaki 4M and the plain GEMM (3M and 4M) are timed beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs an independent replica of the
workload on its own GPU (the product shards by independent problems: no
collective on the data path); rank 0 prints one JSON line with the
whole-job rate (all ranks' units over the max-over-ranks time).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic_inputs as si  # noqa: E402

METRIC = "complex MP GEMM 8mnk/s at p=256/512/1024 bits: Ozaki-INT8 vs plain, 1 GB300"
UNIT = "8mnk/s"
# name -> (m, n, k, p, dist, seed index): the seeded workloads of synthetic_inputs
SWEEP = [f"c2_{n}_p{p}" for n in (1024, 2048) for p in (256, 512, 1024)]
WORKLOADS = {name: si.config_inputs(name) for name in SWEEP}
WORKLOADS["c1_256_p256"] = si.config_inputs("c1_ozaki_256_p256")
BATCH_WORKLOAD = "c3_batch64"
PROFILE = os.path.join(ROOT, "profiles", "oz_slicegemm_c2_1024_p1024.md")
# the slice GEMM kernel and the group table / unit schedule it runs over
SLICEGEMM_SRC = [os.path.join(ROOT, "paper_2307_06072_gb300", "csrc", f) for f in ("slicegemm_tc.cu", "grouptable.cu")]


def sources_hash(paths) -> str:
    h = hashlib.sha256()
    for f in paths:
        if not os.path.exists(f):
            return ""
        h.update(open(f, "rb").read())
    return h.hexdigest()[:16]


def log(*a):
    print(*a, file=sys.stderr, flush=True)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def reduce_max(v: float, ws: int, device) -> float:
    """The largest of every rank's v (the job's time is its slowest rank's)."""
    if ws == 1:
        return v
    import torch
    import torch.distributed as tdist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def make_inputs(workload: str, rank: int):
    m, n, k, p, dist, idx = WORKLOADS[workload]
    A = si.random_matrix(m, k, p, si.SEED_BASE + idx + 7919 * rank, dist)
    B = si.random_matrix(k, n, p, si.SEED_BASE + idx + 1000 + 7919 * rank, dist)
    return A, B, p


batch_specs = si.batch_specs
batch_host_problems = si.batch_problems


def run_batched(mp, torch, dev, stream, steps: int, warmup: int):
    """One step = one batched call over the 64 problems, replayed from a CUDA graph."""
    from paper_2307_06072_gb300.autotune import Autotuner
    stream = torch.cuda.Stream(dev)          # graphs are captured on a side stream
    specs = batch_specs()
    probs = []
    for x, (A, B, p) in enumerate(batch_host_problems(specs)):
        m, k, n = A.rows, A.cols, B.cols
        probs.append((mp.DeviceMatrix.from_mpc(A, dev), mp.DeviceMatrix.from_mpc(B, dev),
                      mp.DeviceMatrix.empty(m, n, p, dev), p, "3m", "ozaki"))
    tuner = Autotuner()
    best = tuner.choose(probs, stream=stream)
    total, _ = mp.batched_workspace(probs, best)
    ws = mp.Workspace(dev)
    ws.get(total)
    mp.mpcgemm_batched(probs, best, ws, stream)
    torch.cuda.synchronize(dev)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        mp.mpcgemm_batched(probs, best, ws, stream)
    with torch.cuda.stream(stream):          # replay on the stream the events are recorded on
        for _ in range(warmup):
            g.replay()
        torch.cuda.synchronize(dev)
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for _ in range(steps):
            g.replay()
        end.record(stream)
    torch.cuda.synchronize(dev)
    ms = start.elapsed_time(end) / steps
    work = sum(8.0 * m * n * k for (m, k, n, p) in specs)
    flops = 0.0
    for (m, k, n, p) in specs:
        pl = mp.plan(m, n, k, p, "3m", "ozaki", best)
        flops += pair_count(pl["s"], pl["Q"], "3m") * 2.0 * m * n * k
    return {"value": work / (ms / 1e3), "unit": UNIT, "ms_per_step": ms, "problems": len(specs),
            "sum_8mnk": work, "tuned": best, "tuning_ms": {str(c): round(t, 3) for c, t in tuner.last_timings},
            "workspace_gb": round(total / 1e9, 2),
            "tensor_tflops_whole_call": round(flops / (ms / 1e3) / 1e12, 1),
            "slice_gemm_launches": -(-len(specs) // 64) if best.get("kernel") != "mma_sync" else len(specs),
            "launch": "one CUDA graph replay per step (split/accumulate per problem, one persistent tcgen05 "
                      "slice-GEMM launch for all 64 problems)"}


def shifted_part(mat, c: int, by: int):
    """The matrix with component c scaled by 2^by (exponents of its nonzero entries)."""
    out = mat.copy()
    nz = out.limb[c, -1] != 0
    out.exp[c] = np.where(nz, out.exp[c] + by, out.exp[c]).astype(np.int32)
    return out


def run_split_variants(mp, torch, dev, stream, n: int = 512, p: int = 512, shift: int = -100, steps: int = 3):
    """The per-part and the residual split (Alg. 2 with the unit re-measured before every
    slice) against the default one when every imaginary part is 2^shift times the size of
    the real parts: times, stage times (the default split sends every imaginary component
    to the exact fallback), part offsets, kept pairs, oracle check."""
    A = shifted_part(si.random_matrix(n, n, p, si.SEED_BASE + 6, "uniform_exp"), 1, shift)
    B = shifted_part(si.random_matrix(n, n, p, si.SEED_BASE + 1006, "uniform_exp"), 1, shift)
    dA, dB = mp.DeviceMatrix.from_mpc(A, dev), mp.DeviceMatrix.from_mpc(B, dev)
    out = {"m": n, "n": n, "k": n, "p_bits": p, "method": "4m", "imaginary_scale": f"2^{shift}"}
    for split in ("common", "per_part", "residual"):
        dC = mp.DeviceMatrix.empty(n, n, p, dev)
        prm = {"split": split}
        ws = mp.Workspace(dev)
        mp.mpcgemm(dA, dB, dC, p, "4m", "ozaki", workspace=ws, stream=stream, params=prm)
        torch.cuda.synchronize(dev)
        evs = []
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for _ in range(steps):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
            mp.mpcgemm(dA, dB, dC, p, "4m", "ozaki", workspace=ws, stream=stream, params=prm, events=ev)
            evs.append(ev)
        end.record(stream)
        torch.cuda.synchronize(dev)
        st = mp.read_status(ws, stream)
        pl = mp.plan(n, n, n, p, "4m", "ozaki", prm)
        G = pl["n_groups_total"]
        table = ws.tensor[pl["off_group_table"]: pl["off_group_table"] + 16 * G].view(torch.int32).cpu().numpy()
        zw = ws.tensor[40:56].view(torch.int32).cpu().numpy()
        ms = start.elapsed_time(end) / steps
        out[split] = {"ms_per_step": round(ms, 3), "value": 8.0 * n ** 3 / (ms / 1e3), "unit": UNIT,
                      "stage_ms": {k_: round(float(np.mean([e[x].elapsed_time(e[x + 1]) for e in evs])), 3)
                                   for x, k_ in enumerate(("split", "slice_gemm", "accumulate_round", "fallback"))},
                      "slices_per_part": pl["s"], "kept_pairs": int(table.reshape(G, 4)[:, 3].sum()),
                      "fallback_components": st["fallback_entries"], "device_status": st,
                      "oracle_check": sampled_check(mp, A, B, p, dC, 16, 77)}
        if split == "per_part":
            out[split]["part_offsets_z"] = {"A_re": 2048 - int(zw[0]), "A_im": 2048 - int(zw[1]),
                                            "B_re": 2048 - int(zw[2]), "B_im": 2048 - int(zw[3])}
        if split == "residual":
            out[split]["pair_batch"] = pl["pair_batch"]
            out[split]["launches"] = pl["launches"]
        del ws, dC
    for split in ("per_part", "residual"):
        out[f"speedup_{split}_vs_common"] = round(out["common"]["ms_per_step"] / out[split]["ms_per_step"], 1)
    return out


def run_lu(mp, torch, dev, n: int = 2048, p: int = 512, block: int = 128, method: str = "3m"):
    """Config 4: A = U + n I, x = 1 + i, b = RN(A x) (by this library's GEMM), solve, error of x."""
    from fractions import Fraction
    A = si.shifted_diagonal_matrix(n, p, si.SEED_BASE + 4)
    ones = np.zeros((2, n, 1), np.int64)
    ones[:] = 1
    X1 = si.from_integers(ones, p)
    dA, dx = mp.DeviceMatrix.from_mpc(A, dev), mp.DeviceMatrix.from_mpc(X1, dev)
    db = mp.DeviceMatrix.empty(n, 1, p, dev)
    mp.mpcgemm(dA, dx, db, p, "4m", "ozaki")
    torch.cuda.synchronize(dev)
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    stream = torch.cuda.current_stream(dev)
    start.record(stream)
    ipiv, ws = mp.mpcgesv(dA, db, p, block, method, stream=stream)
    end.record(stream)
    torch.cuda.synchronize(dev)
    st = mp.read_status(ws)
    s, e, l = db.to_host()
    worst = Fraction(0)
    for i in range(n):
        for c in range(2):
            Mv = 0
            for j in range(l.shape[1] - 1, -1, -1):
                Mv = (Mv << 64) | int(l[c, j, i, 0])
            v = Fraction(-Mv if s[c, i, 0] else Mv) * Fraction(2) ** (int(e[c, i, 0]) - 64 * l.shape[1]) if Mv else 0
            worst = max(worst, abs(v - 1))
    rel = float(worst)   # |x_i - (1 + i)| per component relative to 1
    return {"n": n, "p_bits": p, "block": block, "method": method, "seconds": start.elapsed_time(end) / 1e3,
            "max_rel_err_component": rel, "rel_err_in_ulps_of_2^-p": rel * 2.0 ** p,
            "singular": mp.lu_singular_column(ws), "status": st,
            "note": "A = U + nI (U uniform [-1,1)), x = 1+i, b = RN(Ax) by this library's GEMM"}


def run_serving(mp, torch, dev, seed: int = si.SEED_BASE + 5, count: int = 1200,
                gaps_ms=(8.0, 4.0, 2.0), pool: int = 32):
    """Mixed GEMM (batched-workload shapes) and LU (n 64..256) requests, Poisson arrivals,
    at several offered loads.

    GEMM operands come from a pool of ``pool`` (shape, p) entries generated once; every
    request has its own output.  An LU solve overwrites its operands, so each LU request
    gets fresh device copies of a pooled system before every load."""
    from paper_2307_06072_gb300.serve import Request, Server
    rng = np.random.default_rng(seed)
    gem, lus = [], []
    for x in range(pool):
        m, k, n = (int(v) for v in np.exp(rng.uniform(np.log(64), np.log(1024), 3)))
        p = int(rng.choice([256, 512, 1024]))
        gem.append((m, k, n, p, mp.DeviceMatrix.from_mpc(si.random_matrix(m, k, p, seed + 10 * x), dev),
                    mp.DeviceMatrix.from_mpc(si.random_matrix(k, n, p, seed + 10 * x + 1), dev)))
    for x in range(8):
        n, p = (64, 128, 256)[x % 3], (256, 512)[x % 2]
        lus.append((n, p, si.shifted_diagonal_matrix(n, p, seed + 500 + x), si.random_matrix(n, 1, p, seed + 600 + x)))
    kinds = ["lu" if x % 10 == 9 else "gemm" for x in range(count)]
    picks = [int(rng.integers(len(lus) if kd == "lu" else len(gem))) for kd in kinds]
    outs = {x: mp.DeviceMatrix.empty(gem[q][0], gem[q][2], gem[q][3], dev)
            for x, (kd, q) in enumerate(zip(kinds, picks)) if kd == "gemm"}
    budget = 48 << 30
    srv = Server(slots=4, hbm_budget=budget, device=dev)
    loads = []
    for gap in gaps_ms:
        t, reqs = 0.0, []
        for x, (kd, q) in enumerate(zip(kinds, picks)):
            t += float(rng.exponential(gap / 1e3))
            if kd == "lu":
                n, p, A, B = lus[q]
                reqs.append(Request(x, "lu", t, mp.DeviceMatrix.from_mpc(A, dev), mp.DeviceMatrix.from_mpc(B, dev),
                                    p, block=64, work=8.0 * n ** 3 / 3))
            else:
                m, k, n, p, A, B = gem[q]
                reqs.append(Request(x, "gemm", t, A, B, p, C=outs[x], work=8.0 * m * n * k))
        torch.cuda.synchronize()
        srv.batches, srv.max_inflight, srv.peak_in_use = [], 0, 0
        out = srv.run(reqs)
        lat_g = np.array([r.latency for r in reqs if r.kind == "gemm" and r.t_done is not None])
        lat_l = np.array([r.latency for r in reqs if r.kind == "lu" and r.t_done is not None])
        out.update({"offered_req_s": round(count / t, 1), "mean_gap_ms": gap,
                    "gemm_p50_ms": float(np.percentile(lat_g, 50) * 1e3),
                    "gemm_p99_ms": float(np.percentile(lat_g, 99) * 1e3),
                    "lu_p50_ms": float(np.percentile(lat_l, 50) * 1e3) if lat_l.size else None,
                    "lu_p99_ms": float(np.percentile(lat_l, 99) * 1e3) if lat_l.size else None})
        loads.append({k_: (round(v, 3) if isinstance(v, float) else v) for k_, v in out.items()})
    return {"loads": loads,
            "note": (f"{count} requests per load (every 10th an LU solve, n in {{64, 128, 256}}, p in {{256, 512}}; "
                     f"GEMMs m, n, k log-uniform in [64, 1024], p in {{256, 512, 1024}}, operands from a pool of "
                     f"{pool}), Poisson arrivals at mean gaps {list(gaps_ms)} ms, 4 stream slots each with a "
                     f"{budget / 4 / 2**30:.0f} GiB workspace reserved at start, at most 64 GEMMs per batched call; "
                     "latency = completion on the GPU - arrival")}


def hbm_stage_rooflines(pl, m, n, k, stages, hbm_gbs, src):
    """Split and accumulate stages: algorithmic bytes / stage event time.

    split: read every element's limbs, sign and exponent (2 components, 8L + 5 B each) of
    A and B; write every digit plane (bf16) of both operands.  accumulate: read every
    group sum (int32) once; write C (2 components, 8L + 5 B each)."""
    L = pl["limbs"]
    elem = 2 * (8 * L + 5)
    split_bytes = (m * k + k * n) * elem + (pl["planes_A"] * m + pl["planes_B"] * n) * pl["kpad"] * 2
    acc_bytes = pl["n_groups_total"] * m * n * 4 + m * n * elem
    out = {}
    for name, nbytes, ms in (("split", split_bytes, stages[0]), ("accumulate_round", acc_bytes, stages[2])):
        gbs = nbytes / (ms / 1e3) / 1e9
        out[name] = {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm_gbs, "unit": "GB/s",
                     "frac": round(gbs / hbm_gbs, 4), "algorithmic_bytes": nbytes, "stage_ms": round(ms, 3),
                     "peak_source": f"hbm_gbs ({src})"}
    return out


# Plain path roof: one mad.wide.s32 (a 32 x 32 -> 64-bit digit product added into a 64-bit
# sum) per IMAD lane per clock, 64 lanes per SM (a register-only loop of independent
# mad.wide.s32 ran at 60 per clock per SM on a GB300), 152 SMs at the 2070 MHz maximum clock.
PLAIN_PRODUCTS_PER_CLK_SM = 64
SMS, MAX_SM_GHZ = 152, 2.07


def plain_roofline(mp, m, n, k, p, method, gemm_ms):
    """ALU roofline of the plain GEMM kernel: schoolbook digit products / its event time."""
    pl = mp.plan(m, n, k, p, method, "plain")
    products = pl["n_products"] * pl["s"] ** 2 * m * n * k
    peak = PLAIN_PRODUCTS_PER_CLK_SM * SMS * MAX_SM_GHZ * 1e9
    achieved = products / (gemm_ms / 1e3)
    return {"bound": "alu", "kernel": "k_plain_gemm", "achieved": round(achieved / 1e12, 3),
            "peak": round(peak / 1e12, 3), "unit": "T digit-products/s (32x32->64 bit)",
            "frac": round(achieved / peak, 4), "traffic": None, "digits": pl["s"],
            "algorithmic_products_per_launch": products, "kernel_ms": round(gemm_ms, 3),
            "peak_source": "64 mad.wide.s32/clk/SM (60 measured) x 152 SMs x 2.07 GHz"}


def pair_count(s: int, Q: int, method: str) -> int:
    """Kept slice pairs over all real products (Alg. 2's triangle t + u <= Q)."""
    def tri(a0, na, b0, nb):
        return sum(1 for t in range(a0, a0 + na) for u in range(b0, b0 + nb) if t + u <= Q)
    if method == "4m":
        return 4 * tri(0, s, 0, s)
    return 2 * tri(0, s, 0, s) + tri(-1, s + 1, -1, s + 1)


class ClockSampler:
    """nvidia-smi samples during the timed region (read only; never sets clocks)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = [l.split(",") for l in open(self.path) if l.strip()]
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        busy = [v for v in sm if mx and v > 0.3 * mx] or sm
        return {"sm_mhz": statistics.median(busy) if busy else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def committed_traffic(kernel_hash: str):
    """DRAM bytes per launch of the slice-GEMM kernel from the committed ncu summary,
    or None if the summary is missing or was taken on a different kernel source."""
    if not os.path.exists(PROFILE):
        return None
    txt = open(PROFILE).read()
    h = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", txt)
    t = re.search(r"dram_bytes_per_full_launch:\s*([0-9.eE+]+)", txt)
    if not h or not t or h.group(1) != kernel_hash:
        return None
    return float(t.group(1))


def sampled_check(mp, A, B, p, dC, count: int, seed: int) -> dict:
    """Compare `count` sampled output entries (both components) with the exact C oracle."""
    from oracle import c_oracle
    rng = np.random.default_rng(seed)
    ent = np.stack([rng.integers(0, A.rows, count), rng.integers(0, B.cols, count)], axis=1)
    sg, ex, li = c_oracle.rounded_cgemm(A, B, p, ent)
    s_, e_, l_ = dC.to_host()
    ii, jj = ent[:, 0], ent[:, 1]
    bad = (s_[:, ii, jj] != sg) | (e_[:, ii, jj] != ex) | np.any(l_[:, :, ii, jj] != li, axis=1)
    return {"entries": int(count), "components": int(2 * count), "mismatches": int(bad.sum())}


def slice_roofline(pl, method, m, n, k, gemm_ms, peak, peak_src):
    flops = pair_count(pl["s"], pl["Q"], method) * 2.0 * m * n * k
    achieved = flops / (gemm_ms / 1e3) / 1e12
    return {"bound": "tensor", "kernel": "oz_slicegemm", "achieved": round(achieved, 2), "peak": peak,
            "unit": "TFLOP/s", "frac": round(achieved / peak, 4), "traffic": None,
            "algorithmic_flops_per_launch": flops, "kernel_ms": round(gemm_ms, 3),
            "peak_source": f"bf16_tflops_sustained ({peak_src})"}


def run_sweep(mp, torch, dev, stream, ws, names, skip=None, known=None):
    """Every precision of the metric at n = 1024 and 2048: Ozaki 3M / 4M and plain 3M / 4M,
    each with its roofline, the speedup of Ozaki over plain, and a sampled oracle check.
    ``known``: results already measured for the workload ``skip`` (the timed headline)."""
    peaks, peak_src = measured_peaks()
    peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
    out = {}
    for name in names:
        m, n, k, p, _, _ = WORKLOADS[name]
        units = 8.0 * m * n * k
        if name == skip and known is not None:
            out[name] = known
            continue
        t0 = time.time()
        A, B, p = si.make_config(name)
        dA, dB = mp.DeviceMatrix.from_mpc(A, dev), mp.DeviceMatrix.from_mpc(B, dev)
        dC = mp.DeviceMatrix.empty(m, n, p, dev)
        res = {"m": m, "n": n, "k": k, "p_bits": p}
        for algo in ("ozaki", "plain"):
            for method in ("3m", "4m"):
                steps, warm = (3, 2) if algo == "ozaki" else (1, 1)
                for _ in range(warm):
                    mp.mpcgemm(dA, dB, dC, p, method, algo, workspace=ws, stream=stream)
                torch.cuda.synchronize(dev)
                evs = []
                start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                start.record(stream)
                for _ in range(steps):
                    ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
                    mp.mpcgemm(dA, dB, dC, p, method, algo, workspace=ws, stream=stream, events=ev)
                    evs.append(ev)
                end.record(stream)
                torch.cuda.synchronize(dev)
                ms = start.elapsed_time(end) / steps
                stages = [float(np.mean([e[x].elapsed_time(e[x + 1]) for e in evs])) for x in range(4)]
                pl = mp.plan(m, n, k, p, method, algo)
                roof = (slice_roofline(pl, method, m, n, k, stages[1], peak, peak_src) if algo == "ozaki"
                        else plain_roofline(mp, m, n, k, p, method, stages[1]))
                st = mp.read_status(ws, stream)
                res[f"{algo}_{method}"] = {"value": units / (ms / 1e3), "unit": UNIT, "ms_per_step": round(ms, 3),
                                           "steps": steps, "stage_ms": [round(x, 3) for x in stages],
                                           "roofline": roof, "device_status": st,
                                           "oracle_check": sampled_check(mp, A, B, p, dC, 16, 4242 + len(name))}
        for method in ("3m", "4m"):
            res[f"ozaki_speedup_vs_plain_{method}"] = round(res[f"ozaki_{method}"]["value"] /
                                                            res[f"plain_{method}"]["value"], 2)
        res["wall_s"] = round(time.time() - t0, 1)
        out[name] = res
        log(f"sweep {name}: ozaki 3m {res['ozaki_3m']['ms_per_step']:.2f} ms, plain 3m "
            f"{res['plain_3m']['ms_per_step']:.1f} ms")
        del dA, dB, dC
    return out


def run_ours(args):
    import torch
    import torch.distributed as tdist
    ws_, rank, local = dist_env()
    if ws_ > 1:
        torch.cuda.set_device(local)
        tdist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws_ > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_2307_06072_gb300 import build
    if rank == 0 or ws_ == 1:
        build.build()
    if ws_ > 1:
        tdist.barrier()
    import paper_2307_06072_gb300 as mp

    if args.workload == BATCH_WORKLOAD:
        stream = torch.cuda.current_stream(dev)
        with ClockSampler(dev.index or 0) as clocks:
            r = run_batched(mp, torch, dev, stream, args.steps, args.warmup)
        if rank == 0:
            peaks, peak_src = measured_peaks()
            peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
            line = {"metric": METRIC, "value": r["value"] * ws_, "unit": UNIT, "n_gpus": ws_, "steps": args.steps,
                    "warmup": args.warmup, "ms_per_step": r["ms_per_step"], "higher_is_better": True,
                    "scaling": "weak", "vs_baseline": None, "dtype": "bf16 slices (exact int), u64 limbs",
                    "data": "synthetic (seeded)",
                    "config": {"workload": "c3_batch64: 64 Ozaki 3M GEMMs, m,n,k log-uniform in [64,1024], "
                                           "p in {256,512,1024}, uniform [-1,1) entries, CUDA-graph replay",
                               "parallelism": f"replicas x{ws_}"},
                    "roofline": {"bound": "tensor", "achieved": r["tensor_tflops_whole_call"], "peak": peak,
                                 "unit": "TFLOP/s", "frac": round(r["tensor_tflops_whole_call"] / peak, 4),
                                 "traffic": None, "kernel": "whole batched call (slice pairs x 2mnk / call time)",
                                 "peak_source": f"bf16_tflops_sustained ({peak_src})"},
                    "cpu_baseline": None, "e2e": None, "gpu_launches": None, "clocks": clocks.summary(),
                    "batched": r}
            print(json.dumps(line), flush=True)
        return
    m, n, k, p, dist, _ = WORKLOADS[args.workload]
    t0 = time.time()
    A, B, p = make_inputs(args.workload, rank)
    log(f"[rank {rank}] inputs {m}x{k}x{n} p={p} generated in {time.time() - t0:.1f}s")
    dA, dB = mp.DeviceMatrix.from_mpc(A, dev), mp.DeviceMatrix.from_mpc(B, dev)
    dC = mp.DeviceMatrix.empty(m, n, p, dev)
    stream = torch.cuda.current_stream(dev)
    method = args.method
    algo = args.algo
    if args.split != "common" and (method != "4m" or algo != "ozaki"):
        raise SystemExit("--split per_part / residual is a 4M Ozaki option")
    params = {"kernel": args.kernel, "split": args.split, "pair_planes": args.pair_planes} if algo == "ozaki" else None
    pl = mp.plan(m, n, k, p, method, algo, params)
    ws = mp.Workspace(dev)
    ws.get(pl["ws_bytes"])

    def timed(method_, algo_, steps, warmup, with_events=False):
        evs = []
        prm = dict(params, split=args.split if method_ == "4m" else "common") if algo_ == "ozaki" else None
        for _ in range(warmup):
            mp.mpcgemm(dA, dB, dC, p, method_, algo_, workspace=ws, stream=stream, params=prm)
        torch.cuda.synchronize(dev)
        if ws_ > 1:
            tdist.barrier()
        torch.cuda.synchronize(dev)
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        start.record(stream)
        for _ in range(steps):
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(5)] if with_events else None
            mp.mpcgemm(dA, dB, dC, p, method_, algo_, workspace=ws, stream=stream, events=ev, params=prm)
            if ev:
                evs.append(ev)
        end.record(stream)
        torch.cuda.synchronize(dev)
        if ws_ > 1:
            tdist.barrier()
        ms = start.elapsed_time(end)
        stages = None
        if evs:
            stages = [float(np.mean([e[x].elapsed_time(e[x + 1]) for e in evs])) for x in range(4)]
        return ms, stages

    def max_over_ranks(v: float) -> float:
        return reduce_max(v, ws_, dev)

    units = 8.0 * m * n * k
    with ClockSampler(dev.index or 0) as clocks:
        ms_main, stages = timed(method, algo, args.steps, args.warmup, with_events=True)
    ms_main = max_over_ranks(ms_main)
    st = mp.read_status(ws, stream)
    value = units * args.steps * ws_ / (ms_main / 1e3)
    gpu_out = dC.to_host() if rank == 0 and ws_ == 1 and not args.no_cpu else None   # checked by the oracle below
    extras = {}
    if not args.quick and algo == "ozaki":
        other = "4m" if method == "3m" else "3m"
        ms_o, st_o = timed(other, "ozaki", max(1, args.steps // 2), 1, with_events=True)
        extras[f"ozaki_{other}"] = {"value": units * max(1, args.steps // 2) * ws_ / (max_over_ranks(ms_o) / 1e3),
                                    "ms_per_step": ms_o / max(1, args.steps // 2),
                                    "stage_ms": st_o}
        for pm in (method, other):
            ms_pl, st_pl = timed(pm, "plain", 1, 1, with_events=True)
            extras[f"plain_{pm}"] = {"value": units * ws_ / (max_over_ranks(ms_pl) / 1e3), "ms_per_step": ms_pl,
                                     "stage_ms": st_pl, "roofline": plain_roofline(mp, m, n, k, p, pm, st_pl[1])}
        extras["ozaki_speedup_vs_plain"] = value / extras[f"plain_{method}"]["value"]
        if not args.no_sweep and ws_ == 1:
            peaks0, src0 = measured_peaks()
            pk = float(peaks0.get("bf16_tflops_sustained", peaks0.get("bf16_tflops")))
            known = {"m": m, "n": n, "k": k, "p_bits": p, "reused": "the timed headline measurement"}
            for mt, ms_, stg in ((method, ms_main / args.steps, stages),
                                 (other, extras[f"ozaki_{other}"]["ms_per_step"], extras[f"ozaki_{other}"]["stage_ms"])):
                known[f"ozaki_{mt}"] = {"value": units / (ms_ / 1e3), "unit": UNIT, "ms_per_step": round(ms_, 3),
                                        "stage_ms": [round(x, 3) for x in stg],
                                        "roofline": slice_roofline(mp.plan(m, n, k, p, mt, "ozaki"), mt, m, n, k,
                                                                   stg[1], pk, src0)}
            for mt in (method, other):
                known[f"plain_{mt}"] = extras[f"plain_{mt}"]
            for mt in ("3m", "4m"):
                known[f"ozaki_speedup_vs_plain_{mt}"] = round(known[f"ozaki_{mt}"]["value"] /
                                                              known[f"plain_{mt}"]["value"], 2)
            extras["precision_sweep"] = run_sweep(mp, torch, dev, stream, ws, SWEEP, skip=args.workload, known=known)
        if not args.no_sweep and ws_ == 1:
            extras["split_variants"] = run_split_variants(mp, torch, dev, stream)
        if not args.no_batched:
            extras["batched_c3"] = run_batched(mp, torch, dev, stream, 3, 3)
        if not args.no_lu:
            extras["lu_c4"] = run_lu(mp, torch, dev)
            extras["serving"] = run_serving(mp, torch, dev)

    # roofline of the dominant kernel (the slice GEMM): algorithmic MMA flops / its event time
    pairs = pair_count(pl["s"], pl["Q"], method) if algo == "ozaki" else 0
    flops = pairs * 2.0 * m * n * k
    gemm_ms = stages[1]
    peaks, peak_src = measured_peaks()
    peak = float(peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops")))
    achieved = flops / (gemm_ms / 1e3) / 1e12
    khash = sources_hash(SLICEGEMM_SRC)
    roofline = {"bound": "tensor", "achieved": round(achieved, 2), "peak": peak, "unit": "TFLOP/s",
                "frac": round(achieved / peak, 4), "traffic": committed_traffic(khash),
                "kernel": "oz_slicegemm", "peak_source": f"bf16_tflops_sustained ({peak_src})",
                "algorithmic_flops_per_launch": flops, "kernel_ms": round(gemm_ms, 3)}
    if algo == "plain":
        roofline = plain_roofline(mp, m, n, k, p, method, gemm_ms)
    else:   # the HBM-bound stages around the slice GEMM, against the measured copy bandwidth
        if args.split != "residual":   # (the residual split interleaves its accumulation with the products)
            extras["hbm_stages"] = hbm_stage_rooflines(pl, m, n, k, stages, float(peaks["hbm_gbs"]), peak_src)

    # e2e through the public API with host buffers: every step copies its inputs from
    # pinned host memory and its result back, inside the timed region.  Two device
    # buffer sets let step i+1's input copy and step i's output copy (copy stream)
    # overlap step i's compute (compute stream), as a user of the async API would.
    e2e = None
    if not args.no_e2e:
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
        hA = [pin(A.sign), pin(A.exp), pin(A.limb.view(np.int64))]
        hB = [pin(B.sign), pin(B.exp), pin(B.limb.view(np.int64))]
        hC = [[torch.empty_like(t, device="cpu").pin_memory() for t in (dC.sign, dC.exp, dC.limb)] for _ in range(2)]
        h2d = sum(t.numel() * t.element_size() for t in hA + hB)
        d2h = sum(t.numel() * t.element_size() for t in hC[0])
        sets = [(dA, dB, dC), (mp.DeviceMatrix.empty(m, k, p, dev), mp.DeviceMatrix.empty(k, n, p, dev),
                             mp.DeviceMatrix.empty(m, n, p, dev))]
        cstream = torch.cuda.Stream(dev)
        ev = lambda: torch.cuda.Event()

        def run_e2e(steps):
            h2d_done, comp_done, d2h_done = [ev(), ev()], [ev(), ev()], [ev(), ev()]
            comp_started = [False, False]

            def copy_in(bset, ready):
                with torch.cuda.stream(cstream):
                    if ready is not None:
                        cstream.wait_event(ready)
                    X, Y, _ = sets[bset]
                    for dst, src in zip((X.sign, X.exp, X.limb, Y.sign, Y.exp, Y.limb), hA + hB):
                        dst.copy_(src, non_blocking=True)
                    h2d_done[bset].record(cstream)
            copy_in(0, None)
            for i in range(steps):
                b_ = i % 2
                X, Y, Z = sets[b_]
                stream.wait_event(h2d_done[b_])
                if i >= 2:
                    stream.wait_event(d2h_done[b_])
                mp.mpcgemm(X, Y, Z, p, method, algo, workspace=ws, stream=stream, params=params)
                comp_done[b_].record(stream)
                comp_started[b_] = True
                if i + 1 < steps:
                    nb = (i + 1) % 2
                    copy_in(nb, comp_done[nb] if comp_started[nb] else None)
                with torch.cuda.stream(cstream):
                    cstream.wait_event(comp_done[b_])
                    for dst, src in zip(hC[b_], (Z.sign, Z.exp, Z.limb)):
                        dst.copy_(src, non_blocking=True)
                    d2h_done[b_].record(cstream)
            torch.cuda.synchronize(dev)

        run_e2e(2)
        t1 = time.perf_counter()
        es = max(2, args.steps)
        run_e2e(es)
        e2e_s = max_over_ranks(time.perf_counter() - t1)
        # raw copy bandwidths, for the record
        t2 = time.perf_counter()
        for dst, src in zip((dA.sign, dA.exp, dA.limb, dB.sign, dB.exp, dB.limb), hA + hB):
            dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize(dev)
        t3 = time.perf_counter()
        for dst, src in zip(hC[0], (dC.sign, dC.exp, dC.limb)):
            dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize(dev)
        t4 = time.perf_counter()
        e2e = {"value": units * es * ws_ / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "steps": es,
               "pipeline": "double-buffered: copies of step i+1 / i on a second stream overlap step i",
               "h2d_gbs": round(h2d / (t3 - t2) / 1e9, 1), "d2h_gbs": round(d2h / (t4 - t3) / 1e9, 1)}

    cpu = None
    if rank == 0 and ws_ == 1 and not args.no_cpu:
        cpu = cpu_baseline(A, B, p, args.cpu_seconds, gpu_out=gpu_out)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws_, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_main / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16 slices (exact int), u64 limbs",
            "data": "synthetic (seeded)",
            "config": {"workload": f"{args.workload}: {algo} {method}, m=n=k={m}, p={p} bits, entries u*2^e, "
                                   "e in [-20,20]", "method": method, "algo": algo, "m": m, "n": n, "k": k,
                       "p_bits": p, "kernel": args.kernel, "split": args.split, "slices": pl["s"], "cut_level_Q": pl["Q"], "pairs": pairs,
                       "l2": "inputs (A, B: %.2f GB) larger than L2 (126 MB)" % ((A.nbytes() + B.nbytes()) / 1e9),
                       "parallelism": f"replicas x{ws_}"},
            "stage_ms": {"split": stages[0], "slice_gemm": stages[1], "accumulate_round": stages[2],
                         "fallback": stages[3]},
            "device_status": st,
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": pl["launches"] * args.steps,
            "oracle_mismatches": cpu.get("oracle_mismatches") if cpu else None,
            "clocks": clocks.summary(), "extras": extras,
        }
        print(json.dumps(line), flush=True)
    if ws_ > 1:
        tdist.barrier()
        tdist.destroy_process_group()


def cpu_baseline(A, B, p, seconds: float, entries_hint: int = 0, gpu_out=None):
    """Time the oracle (C, exact, all host threads) on a bounded sample of output entries.

    ``gpu_out``: (sign, exp, limb) of the GPU's product of the same A, B; the sampled
    oracle entries are compared with it (both components, bit for bit)."""
    from oracle import c_oracle
    m, k, n = A.rows, A.cols, B.cols
    threads = c_oracle.max_threads()
    rng = np.random.default_rng(12345)

    def sample(cnt):
        return np.stack([rng.integers(0, m, cnt), rng.integers(0, n, cnt)], axis=1)
    probe = max(threads, 16)
    t0 = time.perf_counter()
    c_oracle.rounded_cgemm(A, B, p, sample(probe))
    dt = time.perf_counter() - t0
    cnt = entries_hint or int(max(probe, min(200000, probe * seconds / max(dt, 1e-6))))
    ent = sample(cnt)
    t0 = time.perf_counter()
    sg, ex, li = c_oracle.rounded_cgemm(A, B, p, ent)
    dt = time.perf_counter() - t0
    out = {"value": 8.0 * k * cnt / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": f"{cnt} random output entries (both components) of the same {m}x{k}x{n} p={p} product, "
                     f"exact C oracle, {dt:.1f} s"}
    if gpu_out is not None:
        s_, e_, l_ = gpu_out
        ii, jj = ent[:, 0], ent[:, 1]
        bad = (s_[:, ii, jj] != sg) | (e_[:, ii, jj] != ex) | np.any(l_[:, :, ii, jj] != li, axis=1)
        out["oracle_checked_components"] = int(2 * cnt)
        out["oracle_mismatches"] = int(bad.sum())
    return out


def cpu_baseline_batch(problems, seconds: float):
    """The oracle on the same number of random output entries of every problem of the batch."""
    from oracle import c_oracle
    rng = np.random.default_rng(12346)

    def once(cnt):
        units, t0 = 0.0, time.perf_counter()
        for (A, B, p) in problems:
            ent = np.stack([rng.integers(0, A.rows, cnt), rng.integers(0, B.cols, cnt)], axis=1)
            c_oracle.rounded_cgemm(A, B, p, ent)
            units += 8.0 * A.cols * cnt
        return units, time.perf_counter() - t0
    _, dt1 = once(1)
    cnt = max(1, int(seconds / max(dt1, 1e-6)))
    units, dt = once(cnt)
    return {"value": units / dt, "unit": UNIT, "cores": c_oracle.max_threads(), "kind": "oracle",
            "sample": f"{cnt} random output entries of each of the {len(problems)} problems, exact C oracle, "
                      f"{dt:.1f} s"}


def run_reference_batch(args, ws_):
    specs = batch_specs()
    problems = batch_host_problems(specs)
    per_step = min(max(2.0, 60.0 / max(1, args.steps + args.warmup)), args.cpu_seconds)
    for _ in range(args.warmup):
        cpu_baseline_batch(problems, min(per_step, 5.0))
    vals, cb = [], None
    for _ in range(args.steps):
        cb = cpu_baseline_batch(problems, per_step)
        vals.append(cb["value"])
    value = float(np.mean(vals))
    cb["value"] = value
    work = sum(8.0 * m * n * k for (m, k, n, p) in specs)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws_,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": work / value * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "exact integer (u64 limbs)", "data": "synthetic (seeded)",
            "config": {"workload": "c3_batch64: 64 complex GEMMs, m,n,k log-uniform in [64,1024], "
                                   "p in {256,512,1024}, uniform [-1,1) entries, exact oracle"},
            "cpu_baseline": cb, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_reference(args):
    ws_, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle import c_oracle
    c_oracle.build()
    if args.workload == BATCH_WORKLOAD:
        run_reference_batch(args, ws_)
        return
    m, n, k, p, dist, _ = WORKLOADS[args.workload]
    A, B, p = make_inputs(args.workload, 0)
    per_step = min(max(2.0, 60.0 / max(1, args.steps + args.warmup)), args.cpu_seconds)
    for _ in range(args.warmup):
        cpu_baseline(A, B, p, min(per_step, 5.0))
    vals = []
    cb = None
    for _ in range(args.steps):
        cb = cpu_baseline(A, B, p, per_step)
        vals.append(cb["value"])
    value = float(np.mean(vals))
    cb["value"] = value
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws_,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 8.0 * m * n * k / value * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "exact integer (u64 limbs)", "data": "synthetic (seeded)",
            "config": {"workload": f"{args.workload}: exact oracle, m=n=k={m}, p={p} bits, entries u*2^e",
                       "m": m, "n": n, "k": k, "p_bits": p},
            "cpu_baseline": cb, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS) + [BATCH_WORKLOAD], default="c2_2048_p1024")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched side measurement")
    ap.add_argument("--no-lu", action="store_true", help="skip the LU and serving side measurements")
    ap.add_argument("--method", choices=["3m", "4m"], default="3m")
    ap.add_argument("--split", choices=["common", "per_part", "residual"], default="common",
                    help="how the operands are cut (4M Ozaki only; default: one grid per line)")
    ap.add_argument("--pair-planes", type=int, default=0,
                    help="residual split: planes in the pair-product buffer (0: the library's default)")
    ap.add_argument("--algo", choices=["ozaki", "plain"], default="ozaki",
                    help="the timed step's algorithm (plain: the CUDA-core GEMM, no side measurements)")
    ap.add_argument("--kernel", choices=["auto", "tcgen05", "tcgen05_n128", "tcgen05_2sm", "tcgen05_2sm_n128", "mma_sync"], default="auto",
                    help="slice-GEMM kernel")
    ap.add_argument("--quick", action="store_true", help="skip the 4M / plain side measurements")
    ap.add_argument("--no-sweep", action="store_true", help="skip the precision sweep (n 1024/2048, p 256/512/1024)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="CPU oracle sample per measurement: the cpu_baseline leg, and the cap of each step of --impl reference")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        log("note: warm-up raised to the minimum of 3 steps")
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
