#!/usr/bin/env python
"""Benchmark of the bf16xN split GEMM (Henry, Tang & Heinecke, Sec. IV-A / V).

Workload (N = 1): FP32 A, B of 8192 x 8192 x 8192 with entries u * 2^e,
u ~ U[-1, 1], e ~ U{-8..8} (seeded); one step = the whole GEMM path: split of
A, transposed split of B, and the tcgen05 bf16x6 product with FP32 output.
value = effective FP32 TFLOP/s = 2 m n k / step time, summed over ranks.
Inputs (256 MiB each) and pieces (768 MiB) exceed the 126 MB L2, so no L2
flush is needed between steps.

Extra keys on the single JSON line: the other variants (bf16x3/x9, the
16384 x 16384 x 256 tall-skinny shape, the FP32 SIMT baseline), the error on
sampled rows against the FP64 product (numpy; the oracle runs only in the
CPU-baseline legs) and the stated bound, the roofline of the
dominant kernel, the CPU baseline (the oracle itself on a bounded row sample),
clocks sampled during the timed region and the end-to-end number through the
public API with host buffers.

--impl reference times the CPU oracle (the only reference this paper has) on
a bounded sample of the same workload.
Multi-GPU (torchrun): every rank runs its own independent GEMM of the same
shape (weak scaling, no collective in the data path; a barrier brackets the
timed region and the max time over ranks is used).
"""
from __future__ import annotations

import argparse
import atexit
import datetime
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "bf16xN GEMM eff. FP32 TFLOP/s at stated error; IR solves/s, p50/p99 latency"
WORKLOAD = "split-BF16 GEMM at scale, 8192x8192x8192, u*2^e entries (e in [-8,8]), bf16x6"
EPS = 2.0 ** -24


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["bfx", "reference"], default="bfx")
    p.add_argument("--mode", type=int, default=6, choices=[1, 3, 6, 9])
    p.add_argument("--m", type=int, default=8192)
    p.add_argument("--n", type=int, default=8192)
    p.add_argument("--k", type=int, default=8192)
    p.add_argument("--quick", action="store_true",
                   help="main measurement only (no variants, CPU baseline or e2e); for profiling")
    p.add_argument("--cpu-rows", type=int, default=16, help="rows of the CPU-baseline sample")
    p.add_argument("--no-solves", action="store_true",
                   help="skip the solve workloads (single IR, batched, serving)")
    p.add_argument("--serve-requests", type=int, default=200)
    return p.parse_args()


# ----------------------------------------------------------------- helpers
def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d["hbm_gbs"], d["bf16_tflops"], d["bf16_tflops_sustained"], "measured"
    except Exception:
        return 6400.0, 1800.0, 1400.0, "fallback"


class Clocks:
    """nvidia-smi sampled every 100 ms for the whole run (started early, so it
    is sampling when the timed region begins); only the samples whose
    timestamps fall inside the timed region are kept."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev: int):
        self.dev = dev
        self.proc = None
        self.path = None
        self.window = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.dev), "-f", self.path], stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
            atexit.register(self._end)  # never leave the sampler running
        except Exception:
            self.proc = None

    def _end(self):
        if self.proc and self.proc.poll() is None:
            self.proc.terminate()

    def mark(self, t0: float, t1: float):
        """The timed region in host wall-clock seconds (time.time())."""
        self.window = (t0, t1)

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.15)  # let the sample after the window arrive
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 10:
                    continue
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(f[2]), float(f[3]),
                             [nm for nm, v in zip(names, f[6:10]) if v.lower().startswith("active")]))
            os.unlink(self.path)
        except Exception:
            return None
        if not rows:
            return None
        inside = rows
        if self.window:
            t0, t1 = self.window
            inside = [r for r in rows if t0 <= r[0] <= t1]
            if not inside:  # a region shorter than the sampling period: the next sample
                later = [r for r in rows if r[0] >= t0]
                inside = later[:1] or rows[-1:]
        reasons = sorted({nm for r in inside for nm in r[3]})
        return {"sm_mhz": statistics.median(r[1] for r in inside),
                "sm_max_mhz": max(r[2] for r in inside), "samples": len(inside),
                "reasons": reasons}


def fp64_rows(A, B, rows=None):
    """The plain definition the errors are measured against: C64 = A B and
    |A||B| in FP64 (numpy), for the selected rows of A (all rows if None)."""
    A = np.asarray(A, np.float32)
    Ar = A if rows is None else A[np.asarray(rows)]
    A64, B64 = Ar.astype(np.float64), np.asarray(B, np.float32).astype(np.float64)
    return A64 @ B64, np.abs(A64) @ np.abs(B64)


def kernel_hash():
    h = hashlib.sha256()
    for f in ("gemm_tc.cu", "bfx_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1904_06376_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(mode, m, n, k):
    """DRAM bytes per launch of the GEMM kernel from the committed ncu summary,
    if it was taken on the current kernel source for this shape and mode."""
    path = os.path.join(ROOT, "profiles", "gemm_tc_traffic.json")
    try:
        d = json.load(open(path))
        e = d["entries"][f"x{mode}_{m}x{n}x{k}"]
        if e["kernel_hash"] != kernel_hash():
            return None
        return e["dram_bytes_per_launch"]
    except Exception:
        return None


# ----------------------------------------------------------------- reference arm
def run_reference(args, rank, world):
    """The CPU oracle on the same workload: each step computes one 16 x 256
    block of C (a bounded sample) with the oracle's FP32-FMA bf16xN model."""
    if rank != 0:
        return
    import oracle
    import bfx_inputs as bi

    m, n, k, mode = args.m, args.n, args.k, args.mode
    br, bc = 16, 256
    A = bi.wide_range((m, k), 60)
    B = bi.wide_range((k, n), 61)
    oracle.lib()
    rng = np.random.default_rng(5)

    def one():
        r0 = int(rng.integers(0, m - br + 1))
        c0 = int(rng.integers(0, n - bc + 1))
        oracle.gemm(mode, A[r0:r0 + br], np.ascontiguousarray(B[:, c0:c0 + bc]))

    for _ in range(max(args.warmup, 0)):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    t = (time.perf_counter() - t0) / max(args.steps, 1)
    v = 2.0 * br * bc * k / t / 1e12
    cores = min(br, oracle.num_threads())
    sample = (f"one {br}x{bc} block of C per step from the {m}x{n}x{k} product, by the oracle's "
              f"sequential FP32-FMA bf16x{mode} model")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "TFLOP/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": {"workload": WORKLOAD.replace("bf16x6", f"bf16x{mode}"),
                                        "m": m, "n": n, "k": k, "mode": f"x{mode}"},
        "cpu_baseline": {"value": v, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- solve workloads
def _fe(x, x_true):
    return float(np.max(np.abs(x - x_true)) / np.max(np.abs(x_true)))


def _ratio_to_dgesv(pairs, sample):
    """Forward error of each solve divided by that of LAPACK's FP64 dgesv
    (numpy) on the same system: pairs = [(x, P)]; returns the distribution."""
    r = []
    for x, P in pairs:
        xd = np.linalg.solve(P.A32.astype(np.float64), P.b)
        r.append(_fe(x, P.x_true) / max(_fe(xd, P.x_true), 1e-300))
    r = np.array(r)
    if r.size == 0:
        return {"sample": sample, "count": 0}
    return {"reference": "LAPACK dgesv (numpy), FP64, same A32 and b", "sample": sample,
            "count": int(r.size), "median_ratio": float(np.median(r)),
            "p90_ratio": float(np.percentile(r, 90)), "max_ratio": float(r.max()),
            "frac_within_10x": float(np.mean(r <= 10.0))}


def bench_ir_single(bfx, oracle, bi, dev):
    """Config 3: one n = 4096 system per condition number, bf16x3 trailing
    updates with escalation to x6, then GMRES-IR if plain refinement stalls;
    FP64 residual; forward error against x_true beside that of the FP64
    oracle LU solve (timed on the host)."""
    import torch

    n, out = 4096, {"n": 4096, "mode": "x3 (escalate to x6, then GMRES-IR)", "solves": []}
    times = []
    for kappa in (1e1, 1e4, 1e8, 1e12):
        P = bi.svd_system(n, kappa, 11)
        A = torch.from_numpy(P.A32).to(dev)
        b = torch.from_numpy(P.b).to(dev)
        bfx.solve_ir(3, A, b)  # warm-up
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        x, res, code = bfx.solve_ir(3, A, b)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        times.append(dt)
        t1 = time.perf_counter()
        xd, _ = oracle.dgesv(P.A32, P.b)
        tcpu = time.perf_counter() - t1
        fe, fe64 = _fe(x.cpu().numpy(), P.x_true), _fe(xd, P.x_true)
        out["solves"].append({"kappa": kappa, "ms": dt * 1e3, "status": code, "converged": res["converged"],
                              "iters": res["iters"], "refactorizations": res["refactorizations"],
                              "gmres_steps": res["gmres_steps"], "arnoldi_steps": res["arnoldi"],
                              "mode_used": res["mode_used"], "berr": res["berr"],
                              "forward_error": fe, "forward_error_fp64_lu": fe64,
                              "ratio_to_fp64": fe / fe64 if fe64 > 0 else None,
                              "oracle_dgesv_s": tcpu})
    out["solves_per_s"] = len(times) / sum(times)
    out["cpu_baseline"] = {"value": len(times) / sum(s["oracle_dgesv_s"] for s in out["solves"]),
                           "unit": "solves/s", "kind": "oracle", "cores": oracle.num_threads(),
                           "sample": "the oracle's FP64 LU + solve of the same 4 systems"}
    return out


def bench_batched(bfx, oracle, bi, dev, count=2000):
    """Config 4: 2000 systems, n ~ U{32..512}, log10 kappa ~ U[2,8], nrhs 1,
    bf16x6, one CUDA-graph launch; solves/s, convergence and forward error."""
    import torch

    probs = bi.batched_systems(count, 0)
    ns = [p.n for p in probs]
    B0 = bfx.Batch(6, ns, max_iter=12)
    A, b = B0.pack([p.A32 for p in probs], [p.b for p in probs])
    del B0
    # the project's autotuner picks the tile shapes for this batch
    best, best_ms, table = bfx.batch_autotune(6, ns, A, b, reps=2, max_iter=12)
    B = bfx.Batch(6, ns, max_iter=12, config=best)
    x, st = B.solve(A, b)
    torch.cuda.synchronize()
    reps = 5
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(reps):
        B.solve(A, b, x=x, status=st)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / reps
    conv, iters, info, berr = B.decode_status(st)
    xs = B.unpack(x)
    fe = np.array([_fe(xx, p.x_true) for xx, p in zip(xs, probs)])
    lk = np.log10([p.kappa_nominal for p in probs])
    by = {}
    for lo in range(2, 8):
        msk = (lk >= lo) & (lk < lo + 1)
        by[f"1e{lo}-1e{lo + 1}"] = {"systems": int(msk.sum()), "converged": float(conv[msk].mean()),
                                    "median_forward_error": float(np.median(fe[msk])),
                                    "max_forward_error": float(fe[msk].max())}
    ratio = _ratio_to_dgesv(list(zip(xs, probs)), f"all {count} systems")
    sample = list(range(0, count, count // 16))[:16]
    t0 = time.perf_counter()
    for i in sample:
        oracle.lu_solve_ir(6, probs[i].A32, probs[i].b)
    tcpu = time.perf_counter() - t0
    flops = sum(2.0 / 3.0 * p.n ** 3 for p in probs)
    return {"systems": count, "mode": "x6", "ms_per_batch": ms, "solves_per_s": count / (ms * 1e-3),
            "lu_eff_tflops": flops / (ms * 1e-3) / 1e12, "converged": float(conv.mean()),
            "mean_iters": float(iters.mean()), "by_condition": by,
            "forward_error_vs_fp64_dgesv": ratio,
            "graph": "whole batch captured once, replayed per solve",
            "tile_shape": {"nb": best[0], "gemm_bn": best[1]},
            "autotune": [{"nb": r[0], "gemm_bn": r[1], "ms": r[2], "status": r[3]} for r in table],
            "cpu_baseline": {"value": len(sample) / tcpu, "unit": "solves/s", "kind": "oracle",
                             "cores": 1, "sample": f"{len(sample)} of the systems by the oracle's "
                                                   "bf16x6-update LU + FP64 refinement"}}


def bench_accuracy(bfx, bi, dev, size=2048, rows=256):
    """Sec. IV-A's GEMM accuracy study on the device: relative Frobenius error
    against the FP64 product (numpy, on a sample of rows) of each mode and of the FP32
    SIMT GEMM, for the narrow, maximal-exponent and Gaussian-exponent ranges."""
    import torch

    gens = {"uniform [-1,1]": bi.uniform_pm1,
            "random exponent [-60,60]": bi.random_exponent,
            "gaussian exponent (sigma 10)": bi.gaussian_exponent}
    sel = np.sort(np.random.default_rng(5).choice(size, rows, replace=False)).astype(np.int64)
    out = {}
    for name, g in gens.items():
        A = g((size, size), 80)
        B = g((size, size), 81)
        Ad, Bd = torch.from_numpy(A).to(dev), torch.from_numpy(B).to(dev)
        C64, _ = fp64_rows(A, B, sel)
        res = {}
        for label, fn in (("x3", lambda: bfx.gemm_bf16xN(3, Ad, Bd)), ("x6", lambda: bfx.gemm_bf16xN(6, Ad, Bd)),
                          ("x8", lambda: bfx.gemm_bf16xN(8, Ad, Bd)), ("x9", lambda: bfx.gemm_bf16xN(9, Ad, Bd)),
                          ("fp32_simt", lambda: bfx.sgemm_simt(Ad, Bd))):
            C = fn()[torch.from_numpy(sel).to(dev)].cpu().numpy().astype(np.float64)
            res[label] = float(np.linalg.norm(C - C64) / np.linalg.norm(C64))
        out[name] = res
    return {"size": size, "rows_sampled": rows, "relative_frobenius_error": out}


def bench_single_type_lu(bfx, oracle, bi, dev, n=50, per_kappa=100):
    """Sec. IV-B's plain IR table on the device: 100 systems of order 50 per
    condition number, LU computed entirely in FP32, bfloat16 or binary16 (every
    operation rounded to the type), then FP64 residual-form refinement with the
    tolerance cond(A) 2^-53, at most 50 corrections.  One launch (one warp per
    system) per type and condition number."""
    import torch

    names = {bfx.LOWP_FP32: "FP32", bfx.LOWP_BF16: "BF16", bfx.LOWP_FP16: "FP16"}
    rows = []
    t_oracle = None
    for kappa in (10.0, 100.0, 1000.0, 10000.0):
        probs = [bi.svd_system(n, kappa, 9000 + int(np.log10(kappa)) * 1000 + s) for s in range(per_kappa)]
        A = torch.from_numpy(np.stack([p.A32 for p in probs])).to(dev)
        b = torch.from_numpy(np.stack([p.b[:, 0] for p in probs])).to(dev)
        tol = torch.full((per_kappa,), kappa * 2.0 ** -53, dtype=torch.float64, device=dev)
        for typ in (bfx.LOWP_FP32, bfx.LOWP_BF16, bfx.LOWP_FP16):
            bfx.lowp_lu_ir_batched(typ, A, b, tol)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            x, iters, conv, info = bfx.lowp_lu_ir_batched(typ, A, b, tol)
            e1.record()
            torch.cuda.synchronize()
            it, cv = iters.cpu().numpy(), conv.cpu().numpy().astype(bool)
            rows.append({"precision": names[typ], "cond": kappa, "converged_pct": float(100 * cv.mean()),
                         "mean_iterations_converged": float(it[cv].mean()) if cv.any() else None,
                         "mean_iterations_all": float(it.mean()), "ms": e0.elapsed_time(e1)})
        if kappa == 1000.0:  # the oracle on the same 100 systems, one type, for scale
            t0 = time.perf_counter()
            for p in probs:
                oracle.lowp_lu_solve_ir(2, p.A32, p.b, tol=kappa * 2.0 ** -53)
            t_oracle = (time.perf_counter() - t0) * 1e3
    return {"n": n, "systems_per_cond": per_kappa, "tolerance": "cond(A) 2^-53 on |d|/|x|",
            "max_iter": 50, "rows": rows, "oracle_ms_fp16_cond1e3_1core": t_oracle}


def bench_lu_accuracy(bfx, bi, dev):
    """Sec. IV-A's LU figure on the device: mean element error of the bf16x6
    LU over that of the FP32 LU, both against the FP64 LU of the same FP32
    matrix, for [-1, 1] and [-1e10, 1e10] (runs whose pivots differ from the
    FP64 LU's are left out, as their factors are not comparable).  The block
    width leaves several trailing updates at every size (n / nb >= 8): the
    two LUs share the FP32 panel and differ in the updates only, so at
    n = 128 a width of 64 would compare one 64 x 64 update and the panel's
    noise."""
    import scipy.linalg
    import torch

    out = {}
    for scale in (1.0, 1e10):
        for n, runs, nb in ((128, 20, 16), (512, 10, 64), (1024, 4, 64)):
            ratios = []
            for s in range(runs):
                A = (bi.uniform_pm1((n, n), 300 + s) * scale).astype(np.float32)
                LU64, p64 = scipy.linalg.lu_factor(A.astype(np.float64), check_finite=False)
                res = []
                for mode in (0, 6):
                    Ad = torch.from_numpy(A.copy()).to(dev)
                    _, ip, _ = bfx.lu_bf16xN(mode, Ad, nb=nb)
                    res.append((Ad.cpu().numpy(), ip.cpu().numpy()[:n]))
                if not all(np.array_equal(p, p64) for _, p in res):
                    continue
                den = np.maximum(np.abs(LU64), np.finfo(np.float64).tiny)
                e0, e6 = (float(np.mean(np.abs(L - LU64) / den)) for L, _ in res)
                ratios.append(e6 / e0)
            out[f"[-{scale:g},{scale:g}] n={n}"] = {
                "nb": nb, "runs_compared": len(ratios),
                "mean_ratio_x6_over_fp32": float(np.mean(ratios)) if ratios else None}
    return out


def _serve_stream(bfx, arrivals, systems, max_inflight, mode, batch_max_n):
    """Submit the systems at their arrival times; returns (results, seconds, stats)."""
    srv = bfx.Server(budget_bytes=60 * 10 ** 9, max_inflight=max_inflight, mode=mode, escalate=True,
                     batch_max_n=batch_max_n)
    t_start = time.perf_counter()
    tickets = []
    for ta, P in zip(arrivals, systems):
        while time.perf_counter() - t_start < ta:
            pass
        tickets.append(srv.submit(P.A32, P.b))
    results = [srv.wait(t) for t in tickets]
    t_end = time.perf_counter()
    stats = srv.stats()
    srv.close()
    return results, t_end - t_start, stats


def bench_serving(bfx, bi, count, max_inflight=32, mode=6, batch_max_n=0, batched_n=256):
    """Config 5: Poisson arrivals at 5000 req/s, n log-uniform [64, 4096],
    nrhs U{1..16}, log10 kappa U[1,10], 60 GB pool; latency measured from
    submission to completion inside the server.  bf16x6 factors with
    escalation to GMRES-IR.  At 5000 req/s the arrivals outpace the device,
    so the stream is also run at a sweep of lower Poisson rates (a few
    seconds of arrivals each) to find the highest rate the server sustains
    with p99 latency under 1 s.  The same burst is also served with
    continuous batching of the requests with n <= batched_n that wait
    together (one grouped batched solve): in this mix a batch waits for its
    slowest member, a hard system whose GMRES-IR runs on one CTA, so it is
    reported beside the main line rather than used for it."""
    reqs = bi.serving_stream(count, 3)
    systems = [bi.fast_system(r.n, 10.0 ** r.log10_kappa, r.seed, nrhs=r.nrhs) for r in reqs]
    results, secs, stats = _serve_stream(bfx, [r.t_arrival for r in reqs], systems, max_inflight,
                                         mode, batch_max_n)
    lat = np.array([r[1]["latency_s"] for r in results])
    conv = np.array([r[1]["converged"] for r in results])
    fe = np.array([_fe(x, P.x_true) for (x, _), P in zip(results, systems)])
    lk = np.array([r.log10_kappa for r in reqs])
    big = [i for i, P in enumerate(systems) if P.n > 1024][:8]
    pick = [i for i, P in enumerate(systems) if P.n <= 1024] + big
    ratio = _ratio_to_dgesv([(results[i][0], systems[i]) for i in pick],
                            f"every request with n <= 1024 and {len(big)} larger ones")
    out = {"requests": count, "arrival_rate_per_s": 5000,
           "mode": (f"x{mode}, escalation to GMRES-IR (row-sliced preconditioner)"
                    + (f"; n <= {batch_max_n} batched" if batch_max_n else "")),
           "solves_per_s": count / secs,
           "p50_latency_ms": float(np.percentile(lat, 50) * 1e3),
           "p99_latency_ms": float(np.percentile(lat, 99) * 1e3),
           "mean_queue_ms": float(np.mean([r[1]["queue_s"] for r in results]) * 1e3),
           "converged": float(conv.mean()),
           "converged_log10k_le_7": float(conv[lk <= 7].mean()),
           "median_forward_error": float(np.median(fe)),
           "forward_error_vs_fp64_dgesv": ratio,
           "batches": stats["batches"],
           "peak_running": stats["peak_running"], "peak_pool_bytes": stats["peak_used_bytes"],
           "budget_bytes": stats["pool_bytes"], "max_inflight": max_inflight,
           "generator": "O(n^2) Householder/permutation construction with exact kappa"}
    # steady state: the same requests with Poisson arrivals at lower rates
    sweep = []
    for rate in (40, 80, 120, 160, 200, 240, 280):
        arr = np.cumsum(np.random.default_rng(70 + rate).exponential(1.0 / rate, size=count))
        res, sec, st = _serve_stream(bfx, arr, systems, max_inflight, mode, batch_max_n)
        la = np.array([r[1]["latency_s"] for r in res])
        sweep.append({"rate_per_s": rate, "requests": count, "completed_per_s": count / sec,
                      "p50_latency_ms": float(np.percentile(la, 50) * 1e3),
                      "p99_latency_ms": float(np.percentile(la, 99) * 1e3),
                      "converged": float(np.mean([r[1]["converged"] for r in res])),
                      "batches": st["batches"]})
    held = [s_["rate_per_s"] for s_ in sweep
            if s_["p99_latency_ms"] <= 1000.0 and s_["completed_per_s"] >= 0.9 * s_["rate_per_s"]]
    out["steady_state"] = {"sweep": sweep, "p99_target_ms": 1000.0,
                           "highest_rate_held_per_s": max(held) if held else None,
                           "held_means": "p99 latency <= 1 s and completions >= 90 % of the rate",
                           "arrivals": f"the same {count} requests, Poisson arrivals at each rate"}
    if batched_n:
        res, sec, st = _serve_stream(bfx, [r.t_arrival for r in reqs], systems, max_inflight, mode,
                                     batched_n)
        la = np.array([r[1]["latency_s"] for r in res])
        out["continuous_batching"] = {
            "batch_max_n": batched_n, "solves_per_s": count / sec,
            "p50_latency_ms": float(np.percentile(la, 50) * 1e3),
            "p99_latency_ms": float(np.percentile(la, 99) * 1e3),
            "converged": float(np.mean([r[1]["converged"] for r in res])), "batches": st["batches"]}
    return out


# ----------------------------------------------------------------- bfx arm
def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch

    import bfx_inputs as bi
    import paper_1904_06376_b300 as bfx

    torch.cuda.set_device(local)
    clocks = Clocks(local)  # sampling from here on; the timed region's samples are kept
    clocks.start()
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist:
            dist.barrier()

    dev = torch.device("cuda", local)
    m, n, k, mode = args.m, args.n, args.k, args.mode
    npc = {1: 1, 3: 2, 6: 3, 9: 3}[mode]
    Ah = torch.from_numpy(bi.wide_range((m, k), 60 + 2 * rank))
    Bh = torch.from_numpy(bi.wide_range((k, n), 61 + 2 * rank))
    A = Ah.to(dev)
    B = Bh.to(dev)
    C = torch.empty((m, n), dtype=torch.float32, device=dev)
    kp = (k + 7) // 8 * 8
    Ap = torch.empty((npc, m, kp), dtype=torch.int16, device=dev)
    Bp = torch.empty((npc, n, kp), dtype=torch.int16, device=dev)
    stream = torch.cuda.current_stream()

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        # both operands' pieces in one launch (split of A, transposed split of B)
        bfx.split_pair(A, B, npc, npc, out_a=[Ap[i][:, :k] for i in range(npc)],
                       out_b=[Bp[i][:, :k] for i in range(npc)])
        if ev is not None:
            ev[1].record(stream)
        bfx.gemm_presplit(mode, Ap, Bp, k, C)
        if ev is not None:
            ev[2].record(stream)

    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    wall0 = time.time()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for i in range(args.steps):
        step(evs[i])
    t1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clocks.mark(wall0, time.time())
    clk = clocks.stop()
    ms = t0.elapsed_time(t1) / args.steps
    split_ms = statistics.mean(e[0].elapsed_time(e[1]) for e in evs)
    gemm_ms = statistics.mean(e[1].elapsed_time(e[2]) for e in evs)
    if dist:  # the slowest rank's time
        from paper_1904_06376_b300.replicas import max_over_ranks

        ms = max_over_ranks(ms, dist, dev)
    flops = 2.0 * m * n * k
    value = world * flops / (ms * 1e-3) / 1e12
    hbm, bf16_peak, bf16_sus, peak_src = peaks()
    # the burst peak for a short timed region at full clocks; the sustained one
    # (seconds of back-to-back GEMMs under the power cap) once the clocks
    # sampled during the timed region show the power cap holding them down
    capped = bool(clk) and clk["sm_mhz"] < 0.9 * clk["sm_max_mhz"]
    peak = bf16_sus if capped else bf16_peak
    peak_name = ("dense bf16 sustained (MEASURED_PEAKS.json bf16_tflops_sustained; SM clock "
                 "power-capped during the timed region)" if capped else
                 "dense bf16 burst (MEASURED_PEAKS.json bf16_tflops)")
    achieved = mode * flops / (gemm_ms * 1e-3) / 1e12
    traffic = profiled_traffic(mode, m, n, k)
    split_bytes = (m * k + k * n) * (4 + 2 * npc)
    roof = {"kernel": f"gemm_tc_kernel<x{mode}>", "bound": "tensor", "achieved": achieved,
            "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_source": f"{peak_src} {peak_name}",
            "frac_of_burst_peak": achieved / bf16_peak,
            "algorithmic": f"{mode} bf16 products x 2mnk = {mode * flops:.4g} flop per launch",
            "kernel_ms": gemm_ms, "traffic": traffic,
            "split_pass": {"ms": split_ms, "bytes": split_bytes,
                           "GB/s": split_bytes / (split_ms * 1e-3) / 1e9, "peak_GB/s": hbm,
                           "frac": split_bytes / (split_ms * 1e-3) / 1e9 / hbm}}
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x6->f32" if mode == 6 else f"bf16x{mode}->f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD if mode == 6 else WORKLOAD.replace("bf16x6", f"bf16x{mode}"),
                   "m": m, "n": n, "k": k, "mode": f"x{mode}", "global_batch": world,
                   "l2": "inputs and pieces larger than L2 (no flush)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": roof,
        "gpu_launches": 3 * args.steps,
        "clocks": clk,
    }
    if args.quick or rank != 0:
        if rank == 0:
            print(json.dumps(line), flush=True)
        if dist:
            dist.destroy_process_group()
        return

    # ---------------------------------------------------------- variants (rank 0)
    def time_call(fn, reps=5, warm=2):
        for _ in range(warm):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    variants = {}
    ws = torch.empty(bfx.gemm_workspace_size(9, m, n, k), dtype=torch.uint8, device=dev)
    for md in (1, 3, 6, 9):
        t = time_call(lambda: bfx.gemm_bf16xN(md, A, B, C, workspace=ws))
        variants[f"x{md}_{m}x{n}x{k}"] = {"ms": t, "TFLOP/s": flops / (t * 1e-3) / 1e12}
    for md in (3, 6):  # split fused into the tensor-core kernel (no piece workspace)
        t = time_call(lambda: bfx.gemm_bf16xN_fused(md, A, B, C))
        variants[f"x{md}_fused_split_{m}x{n}x{k}"] = {
            "ms": t, "TFLOP/s": flops / (t * 1e-3) / 1e12,
            "bf16_TFLOP/s": md * flops / (t * 1e-3) / 1e12,
            "vs_separate_split": variants[f"x{md}_{m}x{n}x{k}"]["ms"] / t}
    # Sec. II-G's asymmetric split (A two pieces, B three; five products) and
    # Sec. IV-A's FP64 collection ("d", one accumulator per product, C in FP64)
    t = time_call(lambda: bfx.gemm_bf16xN(bfx.BFX_X5, A, B, C, workspace=ws))
    variants[f"x5_asym_2x3_{m}x{n}x{k}"] = {"ms": t, "TFLOP/s": flops / (t * 1e-3) / 1e12}
    C64o = torch.empty((m, n), dtype=torch.float64, device=dev)
    for md in (3, 6):
        t = time_call(lambda: bfx.gemm_bf16xN_f64(md, A, B, C64o, workspace=ws))
        variants[f"x{md}d_f64_collect_{m}x{n}x{k}"] = {
            "ms": t, "TFLOP/s": flops / (t * 1e-3) / 1e12,
            "bf16_TFLOP/s": md * flops / (t * 1e-3) / 1e12}
    del C64o
    t = time_call(lambda: bfx.sgemm_simt(A, B, C), reps=2, warm=1)
    simt_peak = bfx.measure_fma_peak(False)  # FFMA rate of the CUDA cores, measured here
    variants[f"fp32_simt_{m}x{n}x{k}"] = {
        "ms": t, "TFLOP/s": flops / (t * 1e-3) / 1e12,
        "roofline": {"bound": "alu (FP32 FFMA)", "peak": simt_peak, "unit": "TFLOP/s",
                     "frac": flops / (t * 1e-3) / 1e12 / simt_peak,
                     "peak_source": "measured: bfx_measure_fma_peak (independent FFMA chains, "
                                    "every SM, CUDA events), same run"}}
    line["fp64_fma_peak_tflops"] = bfx.measure_fma_peak(True)
    ts = (16384, 16384, 256)
    At = torch.from_numpy(bi.wide_range((ts[0], ts[2]), 70)).to(dev)
    Bt = torch.from_numpy(bi.wide_range((ts[2], ts[1]), 71)).to(dev)
    Ct = torch.empty((ts[0], ts[1]), device=dev)
    wst = torch.empty(bfx.gemm_workspace_size(9, *ts), dtype=torch.uint8, device=dev)
    fl_t = 2.0 * ts[0] * ts[1] * ts[2]
    for md in (3, 6):
        t = time_call(lambda: bfx.gemm_bf16xN(md, At, Bt, Ct, workspace=wst))
        variants[f"x{md}_16384x16384x256"] = {"ms": t, "TFLOP/s": fl_t / (t * 1e-3) / 1e12}
        t = time_call(lambda: bfx.gemm_bf16xN_fused(md, At, Bt, Ct))
        variants[f"x{md}_fused_split_16384x16384x256"] = {"ms": t, "TFLOP/s": fl_t / (t * 1e-3) / 1e12}
    t = time_call(lambda: bfx.sgemm_simt(At, Bt, Ct), reps=3, warm=1)
    variants["fp32_simt_16384x16384x256"] = {"ms": t, "TFLOP/s": fl_t / (t * 1e-3) / 1e12}
    del At, Bt, Ct, wst
    line["variants"] = variants
    line["speedup_vs_fp32_simt"] = variants[f"fp32_simt_{m}x{n}x{k}"]["ms"] / (gemm_ms + split_ms)

    # ---------------------------------------------------------- end to end (host buffers)
    # Every step copies its inputs from pinned host memory, runs the GEMM and
    # reads C back.  Sequential: one stream.  Pipelined: two streams with
    # their own device buffers and workspaces, so one step's copies (PCIe is
    # full duplex) overlap the other's GEMM; each step still moves all of its
    # bytes inside the timed region.
    Ahp = Ah.pin_memory()
    Bhp = Bh.pin_memory()
    Chp = torch.empty((m, n), dtype=torch.float32).pin_memory()

    def e2e_step():
        A.copy_(Ahp, non_blocking=True)
        B.copy_(Bhp, non_blocking=True)
        bfx.gemm_bf16xN(mode, A, B, C, workspace=ws)
        Chp.copy_(C, non_blocking=True)

    te_seq = time_call(e2e_step, reps=5, warm=1)
    lanes = []
    for _ in range(2):
        lanes.append({"s": torch.cuda.Stream(), "A": torch.empty_like(A), "B": torch.empty_like(B),
                      "C": torch.empty_like(C), "ws": torch.empty_like(ws),
                      "Ch": torch.empty((m, n), dtype=torch.float32).pin_memory()})

    def e2e_steps(count):
        for kk in range(count):
            ln = lanes[kk % 2]
            with torch.cuda.stream(ln["s"]):
                ln["A"].copy_(Ahp, non_blocking=True)
                ln["B"].copy_(Bhp, non_blocking=True)
                bfx.gemm_bf16xN(mode, ln["A"], ln["B"], ln["C"], workspace=ln["ws"])
                ln["Ch"].copy_(ln["C"], non_blocking=True)

    e2e_steps(2)
    torch.cuda.synchronize()
    ke = 6
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for ln in lanes:
        ln["s"].wait_event(ev0)
    e2e_steps(ke)
    for ln in lanes:
        ev = torch.cuda.Event()
        ev.record(ln["s"])
        stream.wait_event(ev)
    ev1.record(stream)
    torch.cuda.synchronize()
    te = ev0.elapsed_time(ev1) / ke
    del lanes
    line["e2e"] = {"value": flops / (te * 1e-3) / 1e12, "unit": "TFLOP/s", "ms_per_step": te,
                   "h2d_bytes_per_step": 4 * (m * k + k * n), "d2h_bytes_per_step": 4 * m * n,
                   "pipeline": "two streams, two steps in flight",
                   "sequential_ms_per_step": te_seq,
                   "sequential_value": flops / (te_seq * 1e-3) / 1e12,
                   "api": "paper_1904_06376_b300.gemm_bf16xN (C-ABI bfx_gemm_bf16xN) with pinned host buffers"}

    # ---------------------------------------------------------- error + CPU baseline
    import oracle

    step()
    torch.cuda.synchronize()
    rows = np.sort(np.random.default_rng(7).choice(m, args.cpu_rows, replace=False)).astype(np.int64)
    Cs = C[torch.from_numpy(rows).to(dev)].cpu().numpy().astype(np.float64)
    An, Bn = Ah.numpy(), Bh.numpy()
    C64, Cabs = fp64_rows(An, Bn, rows)
    bound = 2 * max(k, 2) * EPS
    ratio = float(np.max(np.abs(Cs - C64) / (bound * Cabs + 1e-38)))
    relF = float(np.linalg.norm(Cs - C64) / np.linalg.norm(C64))
    line["error"] = {"rows_checked": int(rows.size), "bound": "|C-C64| <= 2k 2^-24 (|A||B|) elementwise",
                     "max_ratio_to_bound": ratio, "rel_frobenius_vs_fp64": relF,
                     "within_bound": ratio <= 1.0}
    t0c = time.perf_counter()
    oracle.gemm(mode, An[rows], Bn)
    tc = time.perf_counter() - t0c
    cores = min(int(rows.size), oracle.num_threads())
    line["cpu_baseline"] = {"value": 2.0 * rows.size * n * k / tc / 1e12, "unit": "TFLOP/s",
                            "cores": cores, "kind": "oracle", "seconds": tc,
                            "sample": f"{rows.size} rows of the {m}x{n}x{k} product, the oracle's "
                                      f"sequential FP32-FMA bf16x{mode} model (split of B included)"}
    del A, B, C, Ap, Bp, ws, Ahp, Bhp, Chp
    torch.cuda.empty_cache()
    if not args.no_solves:
        line["accuracy"] = bench_accuracy(bfx, bi, dev)
        line["single_type_lu_ir"] = bench_single_type_lu(bfx, oracle, bi, dev)
        line["lu_accuracy"] = bench_lu_accuracy(bfx, bi, dev)
        line["ir_single"] = bench_ir_single(bfx, oracle, bi, dev)
        line["batched"] = bench_batched(bfx, oracle, bi, dev)
        line["serving"] = bench_serving(bfx, bi, args.serve_requests)
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
