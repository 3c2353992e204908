"""Benchmark: FP64 SPC5 SpMV on one GB300 (or N independent replicas).

Workload (FP64 plain SpMV over synthetic matrices, every beta(r,c) in
{1x8, 2x4, 2x8, 4x4, 4x8, 8x4}):
  - 3D 27-point stencil on 100^3 (n = 1e6, nnz = 26,463,592), values N(0,1)
  - FEM-like 3x3 dense node blocks on a random-geometric mesh of 1e6 nodes
    (n = 3e6, about 80 entries per row), Morton-ordered, values N(0,1)
  - power-law row lengths (Zipf s = 2, mean 20, n = 2e6), columns near the
    diagonal (sigma = 1000), values N(0,1)
  - uniform-random columns, 16 per row (n = 1e6), values N(0,1)
  x ~ U[-1, 1).  The matrices are converted once (timed separately); one
  step = one y = A x for each of the 24 (matrix, beta) pairs.

Reported: GFlop/s = 2 * nnz / time over the whole step (device-resident
inputs, CUDA events on the launching stream), the HBM roofline of the
dominant SpMV launch (algorithmic bytes = values + block column indices +
masks + panel pointers + x + y, per launch, over the launch's own
event-timed duration) with its fraction of the measured FP64 FMA rate
beside it, every case's error against the CPU oracle, an end-to-end figure
through the C-ABI with host vectors (pinned x and y copied every step), and
the oracle's CSR product timed on the host cores (one thread and all
cores, whole matrices).  Extra sections (outside the step): FP32/BF16
storage, the batched kernel, mixed-precision CG, the autograd backward,
the hybrid form, and the paper's dense 2048 x 2048 matrix.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SPC5 SpMV GFlop/s & HBM GB/s vs peak; FP64 vs FP32/BF16 at stated error"
UNIT = "GFlop/s"
BETAS = [(1, 8), (2, 4), (2, 8), (4, 4), (4, 8), (8, 4)]
MATRICES = ["stencil27", "fem3d", "powerlaw", "uniform"]
DESCR = {
    "stencil27": "3D 27-point stencil 100^3 (n=1e6)",
    "fem3d": "FEM 3x3 node blocks, random-geometric mesh, 1e6 nodes (n=3e6)",
    "powerlaw": "power-law rows Zipf(2) mean 20, n=2e6, column sigma 1000",
    "uniform": "uniform random columns, 16 per row, n=1e6",
}
L2_BYTES = 129 * 1024 * 1024
FP64_TOL = 1e-13  # |y - y_ref| <= 1e-13 * sum_j |a_ij x_j| per row (FP64 storage)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--matrices", default=",".join(MATRICES))
    ap.add_argument("--scale", default="full", choices=["full", "profile"],
                    help="profile: smaller instances (still larger than L2) for ncu captures")
    ap.add_argument("--no-check", action="store_true",
                    help="skip the comparison of every case with the CPU oracle")
    ap.add_argument("--betas", default=",".join(f"{r}x{c}" for r, c in BETAS),
                    help="subset of block shapes (e.g. 4x8), for profiling one kernel")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-cg", action="store_true")
    ap.add_argument("--no-grad", action="store_true")
    ap.add_argument("--no-hybrid", action="store_true")
    ap.add_argument("--no-dense", action="store_true")
    ap.add_argument("--no-tune", action="store_true",
                    help="keep the planner's default mapping instead of autotuning it")
    ap.add_argument("--cases-out", default=None, help="write the per-case table here")
    ap.add_argument("--clocks-out", default=None,
                    help="directory for the raw nvidia-smi clock samples (default: a temp dir)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device="cuda") -> float:
    """The largest x over all ranks (timings are the slowest rank's)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(world: int, flops_per_step: float, seconds_per_step: float) -> float:
    """GFlop/s of the whole job: every rank runs the full workload (replicas,
    weak scaling), so N ranks do N times the work in the slowest rank's time."""
    return world * flops_per_step / seconds_per_step / 1e9


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


VALUE_BYTES = {0: 8, 1: 4, 2: 2}  # FP64, FP32, BF16 storage
# Nominal FP64 FMA rate of the GB300 (2 per cycle per SM: ncu's
# sm__sass_thread_inst_executed_op_dfma peak_sustained is 304 per cycle over
# 152 SMs, at the 2070 MHz maximum SM clock); used only if the measurement
# by spc5_measure_fma_peak fails.
FP64_NOMINAL_TFLOPS = 152 * 2 * 2 * 2.070e9 / 1e12


def fma_peaks(spc5, log):
    """FP64 and FP32 FMA throughput measured on this device (TFLOP/s)."""
    out = {}
    for name, code in (("f64", spc5.SPC5_F64), ("f32", spc5.SPC5_F32)):
        try:
            out[name] = spc5.spc5_measure_fma_peak(code)
        except Exception as e:  # noqa: BLE001 - report and fall back
            log(f"FMA peak measurement ({name}) failed: {e}")
    log(f"measured FMA peaks (TFLOP/s): {out}")
    return out


def plan_label(info):
    """The SpMV's work mapping: blocks (block-balanced), values (value-balanced
    block rounds), expanded, or rows/G<lanes per row>/b<body> (row groups,
    with "/dyn" when tiles come from the counter)."""
    flat = {1: "blocks", 2: "expanded", 3: "values"}.get(info["flat"])
    if flat:
        return flat
    label = f"rows/G{info['lanes_per_row']}"
    if "body" in info:
        label += (f"/b{info['body']}" + ("/dyn" if info.get("dynamic") else "") +
                  ("/half" if info.get("halves") else ""))
    return label


def algorithmic_bytes(info: dict) -> int:
    """Bytes an SpMV must move: values + block column indices + masks + panel
    pointers (block_rowptr and panel value offsets) + x + y.  FP64 matrices
    use FP64 vectors, FP32/BF16 matrices FP32 vectors."""
    nb, npan = info["nblocks"], info["npanels"]
    sv = VALUE_BYTES[info["value_dtype"]]
    sx = 8 if info["value_dtype"] == 0 else 4
    return (sv * info["nnz"] + 4 * nb + info["mask_bytes"] * nb + 8 * (npan + 1)
            + sx * info["ncols"] + sx * info["nrows"])


def kernel_source_hash() -> str:
    """Hash of the SpMV kernels' code with comments and blank lines removed,
    so that editing a comment keeps the committed ncu figures valid."""
    import re
    h = hashlib.sha256()
    for name in ("spc5_spmv.cu", "spc5_flat.cuh"):
        with open(os.path.join(ROOT, "paper_2307_14774_gb300", "csrc", name)) as f:
            text = re.sub(r"/\*.*?\*/", "", f.read(), flags=re.S)
        code = [re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines()]
        h.update("\n".join(ln for ln in code if ln).encode())
    return h.hexdigest()[:16]


def ncu_traffic_ratios():
    """DRAM bytes over algorithmic bytes per SpMV launch, per (matrix, beta),
    from the committed ncu summary (captured on the profile-scale instances of
    the same generators, where DRAM traffic grows with the units processed),
    if it was taken on the current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "spc5_spmv_dram.txt")
    if not os.path.exists(path):
        return None
    src, per_case = None, {}
    for line in open(path):
        line = line.strip()
        if line.startswith("source_sha256:"):
            src = line.split(":", 1)[1].strip()
        elif line and not line.startswith("#"):
            parts = line.split()
            if len(parts) >= 5 and parts[0] in MATRICES:
                try:
                    per_case[(parts[0], parts[1])] = float(parts[4])
                except ValueError:
                    pass
    if src != kernel_source_hash() or not per_case:
        return None
    return per_case


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, out_dir=None):
        import tempfile
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(out_dir or tempfile.gettempdir(),
                                 f"spc5_clocks_rank{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return None
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def roofline_object(case_rows, hbm, peak_kind, fp64_peak, fp64_kind, ratios, step):
    """HBM roofline of the dominant SpMV launch (the case with the longest
    event-timed duration): algorithmic bytes per launch over its duration,
    against the measured HBM copy bandwidth, with the launch's fraction of
    the measured FP64 FMA rate beside it (FP64 FMAs can bind before HBM on
    GB300) and the step's aggregate over all launches."""
    dom = max(case_rows, key=lambda r: r["us"])
    gbs = dom["bytes"] / (dom["us"] * 1e-6) / 1e9
    tflops = 2.0 * dom["nnz"] / (dom["us"] * 1e-6) / 1e12
    traffic = None
    if ratios and (dom["matrix"], dom["beta"]) in ratios:
        traffic = int(round(ratios[(dom["matrix"], dom["beta"])] * dom["bytes"]))
    return {"bound": "hbm", "achieved": round(gbs, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(gbs / hbm, 4), "traffic": traffic,
            "peak_kind": peak_kind,
            "kernel": f"FP64 SpMV {dom['matrix']} beta({dom['beta']}), plan {dom['plan']}",
            "bytes_per_launch": dom["bytes"], "launch_us": dom["us"],
            "traffic_note": "ncu dram__bytes_read.sum + dram__bytes_write.sum over the "
                            "algorithmic bytes, measured on the profile-scale instance and "
                            "applied to this launch's algorithmic bytes",
            "fp64_pipe": {"achieved": round(tflops, 4), "peak": round(fp64_peak, 4),
                          "unit": "TFLOP/s", "frac": round(tflops / fp64_peak, 4),
                          "peak_kind": fp64_kind},
            "step": step}


# ------------------------------------------------------------------ native --

def build_cases(names, torch, spc5, synth, log, betas, tune=True, scale="full"):
    """Generate, upload and convert every (matrix, beta); return cases and
    the host matrices (kept for the CPU baseline sample)."""
    cases, hosts = [], {}
    for name in names:
        t0 = time.time()
        A = synth.workload(name, scale)
        x = synth.vector_uniform(A.ncols, seed=1)
        hosts[name] = (A, x)
        log(f"generated {name}: n={A.nrows} nnz={A.nnz} in {time.time() - t0:.1f}s")
        dev = [torch.from_numpy(a).cuda() for a in (A.rowptr, A.colidx, A.vals)]
        dx = torch.from_numpy(x).cuda()
        dy = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
        for r, c in BETAS:
            if f"{r}x{c}" not in betas:
                continue
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            M = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, *dev, r=r, c=c)
            t_conv = time.perf_counter() - t1
            if tune:
                spc5.spc5_tune(M, dx, dy, iters=3)
            info = M.info()
            cases.append({"matrix": name, "r": r, "c": c, "M": M, "x": dx, "y": dy,
                          "info": info, "bytes": algorithmic_bytes(info), "nnz": A.nnz,
                          "convert_s": t_conv})
        del dev
        torch.cuda.synchronize()
    return cases, hosts


PRECISION_TOL = {"f32": 2e-6, "bf16": 1e-2}  # |y - y_ref| <= tol * sum_j |a_ij x_j|


def err_over_tol(y, y_ref, scale, tol):
    """Largest |y - y_ref| / (tol * S_i) over the rows (inf for an error on a
    row whose S_i is 0)."""
    import numpy as np
    err = np.abs(np.asarray(y, dtype=np.float64) - y_ref)
    bound = tol * scale
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(bound > 0, err / np.where(bound > 0, bound, 1.0),
                     np.where(err > 0, np.inf, 0.0))
    return float(r.max()) if r.size else 0.0


def precision_section(hosts, refs, torch, spc5, stream, hbm, case_rows, log, reps=10, tune=True):
    """FP32 and BF16 value storage (FP32 x, y, accumulation) on the 27-point
    and FEM matrices, every beta: time per SpMV, HBM fraction, speed-up over
    the FP64 case of the main step, and the largest error relative to the
    stated tolerance against the CPU oracle (FP64 product of the original
    FP64 values and x, S_i = sum_j |a_ij x_j|)."""
    fp64_us = {(r["matrix"], r["beta"]): r["us"] for r in case_rows}
    rows = []
    for name in ("stencil27", "fem3d"):
        if name not in hosts:
            continue
        A, x = hosts[name]
        y_ref, scale = refs[name]
        dev = [torch.from_numpy(a).cuda() for a in (A.rowptr, A.colidx, A.vals)]
        x32 = torch.from_numpy(x).cuda().float()
        y32 = torch.empty(A.nrows, dtype=torch.float32, device="cuda")
        flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda")
        for r, c in BETAS:
            for dt, code in (("f32", spc5.SPC5_F32), ("bf16", spc5.SPC5_BF16)):
                M = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, *dev, store_dtype=code, r=r,
                                          c=c)
                if tune:
                    spc5.spc5_tune(M, x32, y32, iters=3)
                info = M.info()
                for _ in range(3):
                    spc5.spc5_spmv(M, x32, y32, 1.0, 0.0, stream)
                evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                       for _ in range(reps)]
                for e0, e1 in evs:
                    flush.zero_()  # the reduced-precision matrices can fit in L2
                    e0.record(stream)
                    spc5.spc5_spmv(M, x32, y32, 1.0, 0.0, stream)
                    e1.record(stream)
                torch.cuda.synchronize()
                us = statistics.median(e0.elapsed_time(e1) for e0, e1 in evs) * 1e3
                ratio = err_over_tol(y32.double().cpu().numpy(), y_ref, scale, PRECISION_TOL[dt])
                b = algorithmic_bytes(info)
                ref = fp64_us.get((name, f"{r}x{c}"))
                rows.append({"matrix": name, "beta": f"{r}x{c}", "dtype": dt,
                             "us": round(us, 2),
                             "gflops": round(2.0 * A.nnz / (us * 1e-6) / 1e9, 1),
                             "gbs": round(b / (us * 1e-6) / 1e9, 1),
                             "frac": round(b / (us * 1e-6) / 1e9 / hbm, 3),
                             "speedup_vs_fp64": round(ref / us, 2) if ref else None,
                             "tol": PRECISION_TOL[dt], "max_err_over_tol": round(ratio, 4),
                             "plan": plan_label(info)})
                del M
        del dev, flush
        torch.cuda.synchronize()
        log(f"precision rows for {name} done")
    return rows


def hybrid_section(hosts, torch, spc5, stream, hbm, case_rows, log, reps=10, tune=True):
    """Hybrid form (single-value blocks as scalar CSR entries) of the
    power-law and uniform matrices, every beta, FP64: time per SpMV (tuned
    like the main step), the share of entries stored as scalars, and the
    speed-up over the plain beta(r,c) case of the main step."""
    base_us = {(r["matrix"], r["beta"]): r["us"] for r in case_rows}
    rows = []
    for name in ("powerlaw", "uniform"):
        if name not in hosts:
            continue
        A, x = hosts[name]
        dev = [torch.from_numpy(a).cuda() for a in (A.rowptr, A.colidx, A.vals)]
        dx = torch.from_numpy(x).cuda()
        dy = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
        for r, c in BETAS:
            M = spc5.spc5_convert_hybrid(A.nrows, A.ncols, A.nnz, *dev, r=r, c=c)
            if tune:
                spc5.spc5_tune(M, dx, dy, iters=3)
            info = M.info()
            for _ in range(3):
                spc5.spc5_spmv(M, dx, dy, 1.0, 0.0, stream)
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(reps)]
            for e0, e1 in evs:
                e0.record(stream)
                spc5.spc5_spmv(M, dx, dy, 1.0, 0.0, stream)
                e1.record(stream)
            torch.cuda.synchronize()
            us = statistics.median(e0.elapsed_time(e1) for e0, e1 in evs) * 1e3
            ns = info["nscalars"]
            nb, npan = info["nblocks"], info["npanels"]
            b = (8 * A.nnz + 4 * nb + info["mask_bytes"] * nb + 8 * (npan + 1) + 4 * ns
                 + 4 * (A.nrows + 1) + 8 * A.ncols + 8 * A.nrows)
            ref = base_us.get((name, f"{r}x{c}"))
            rows.append({"matrix": name, "beta": f"{r}x{c}", "us": round(us, 2),
                         "gflops": round(2.0 * A.nnz / (us * 1e-6) / 1e9, 1),
                         "gbs": round(b / (us * 1e-6) / 1e9, 1),
                         "frac": round(b / (us * 1e-6) / 1e9 / hbm, 3),
                         "scalar_share": round(ns / A.nnz, 3),
                         "speedup_vs_blocks": round(ref / us, 2) if ref else None,
                         "plan": plan_label(info)})
            del M
        del dev
        torch.cuda.synchronize()
        log(f"hybrid rows for {name} done")
    return rows


def dense_section(torch, spc5, synth, stream, hbm, log, n=2048, reps=20, tune=True):
    """The paper's dense n x n matrix (filling 100%: every block full), every
    beta, FP64: time per SpMV against the HBM roofline and the FP64 FMA
    floor.  Its 33.6 MB of values fit in the 129 MB L2, so a buffer larger
    than L2 is written before every timed launch (each launch starts cold)."""
    A = synth.dense(n, n, values="normal")
    x = synth.vector_uniform(n, seed=0)
    dev = [torch.from_numpy(a).cuda() for a in (A.rowptr, A.colidx, A.vals)]
    dx = torch.from_numpy(x).cuda()
    dy = torch.empty(n, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 2**20, dtype=torch.uint8, device="cuda")
    rows = []
    for r, c in BETAS:
        M = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, *dev, r=r, c=c)
        if tune:
            spc5.spc5_tune(M, dx, dy, iters=3)
        info = M.info()
        for _ in range(3):
            spc5.spc5_spmv(M, dx, dy, 1.0, 0.0, stream)
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            spc5.spc5_spmv(M, dx, dy, 1.0, 0.0, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1) * 1e3)
        us = statistics.median(ts)
        b = algorithmic_bytes(info)
        rows.append({"beta": f"{r}x{c}", "us": round(us, 2), "nblocks": info["nblocks"],
                     "filling": round(info["filling"], 4),
                     "gflops": round(2.0 * A.nnz / (us * 1e-6) / 1e9, 1),
                     "gbs": round(b / (us * 1e-6) / 1e9, 1),
                     "frac": round(b / (us * 1e-6) / 1e9 / hbm, 3),
                     "plan": plan_label(info)})
        del M
    del dev, flush
    torch.cuda.synchronize()
    log("dense rows done")
    return {"n": n, "nnz": A.nnz, "note": "the paper's dense matrix, FP64, L2 flushed (a 256 MB "
            "write) before every timed launch; median of " + str(reps), "rows": rows}


def cg_section(torch, spc5, synth, stream, hbm, log, tune=True):
    """Mixed-precision iterative-refinement CG on the SPD 27-point Poisson
    matrix on 128^3 (26 on the diagonal, -1 off it), b ~ U[-1,1), to
    ||b - A x|| / ||b|| <= 1e-10, with the inner solve in FP32, BF16 and (as
    the all-FP64 reference) FP64 storage; the outer residual is FP64.  Both
    matrices are tuned first, as every benchmarked matrix is."""
    A = synth.workload("poisson27_128")
    b = synth.vector_uniform(A.nrows, seed=8)
    dev = [torch.from_numpy(a).cuda() for a in (A.rowptr, A.colidx, A.vals)]
    db = torch.from_numpy(b).cuda()
    A64 = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, *dev, r=4, c=8, stream=stream)
    x64 = torch.empty(A.ncols, dtype=torch.float64, device="cuda")
    y64 = torch.empty(A.nrows, dtype=torch.float64, device="cuda")
    x32 = torch.empty(A.ncols, dtype=torch.float32, device="cuda")
    y32 = torch.empty(A.nrows, dtype=torch.float32, device="cuda")
    if tune:
        spc5.spc5_tune(A64, x64, y64, iters=3)
    out = {"matrix": "27-point Poisson 128^3", "n": A.nrows, "nnz": A.nnz, "tol": 1e-10,
           "outer_plan": plan_label(A64.info()), "rows": []}
    for name, code in (("f32", spc5.SPC5_F32), ("bf16", spc5.SPC5_BF16), ("f64", spc5.SPC5_F64)):
        Alo = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, *dev, store_dtype=code, r=4, c=8,
                                    stream=stream)
        if tune:
            if code == spc5.SPC5_F64:
                spc5.spc5_tune(Alo, x64, y64, iters=3)
            else:
                spc5.spc5_tune(Alo, x32, y32, iters=3)
        for _ in range(2):  # first run warms up; second is timed
            dx = torch.zeros(A.nrows, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rep = spc5.spc5_ircg(A64, Alo, db, dx, tol=1e-10, max_outer=40, inner_tol=1e-3,
                                 max_inner=2000, stream=stream)
            torch.cuda.synchronize()
            secs = time.perf_counter() - t0
        # independent FP64 check of the final residual with the FP64 SpMV
        r = db.clone()
        spc5.spc5_spmv(A64, dx, r, -1.0, 1.0, stream)
        torch.cuda.synchronize()
        relres = float(r.norm() / db.norm())
        # one inner iteration: q = A p (the SpMV), p.q (reads p, q), d += a p
        # and r -= a q with r.r (reads p, q, d, r; writes d, r), p = r + b p
        # (reads r, p; writes p): 11 vector passes besides the SpMV
        ilo = Alo.info()
        vbytes = 11 * A.nrows * (8 if code == spc5.SPC5_F64 else 4)
        it_bytes = algorithmic_bytes(ilo) + vbytes
        us_it = secs / max(1, rep["inner_iters"]) * 1e6
        out["rows"].append({"inner": name, "plan": plan_label(ilo), "seconds": round(secs, 4), **rep,
                            "relres_check": relres,
                            "us_per_inner_iter": round(us_it, 2),
                            "bytes_per_inner_iter": int(it_bytes),
                            "frac": round(it_bytes / (us_it * 1e-6) / 1e9 / hbm, 3),
                            "frac_note": "algorithmic bytes of one inner iteration (SpMV + 11 "
                                         "vector passes) over the solve's wall time per inner "
                                         "iteration (outer FP64 steps included)"})
        log(f"ircg inner={name}: {secs:.3f}s {rep}")
        del Alo
    return out


def grad_section(torch, spc5, synth, hbm, log, reps=10):
    """torch.autograd.Function y = A(vals) x on the 27-point stencil on 100^3
    with FP32 value storage, x ~ U[-1,1) FP32: forward (values stored into the
    matrix, then the SpMV) and backward (dx = A^T g and dvals = g[row] x[col]
    over the stored entries), timed with CUDA events; each of the four
    kernels (value update, SpMV, transposed SpMV, value gradient) is also
    timed alone, with its algorithmic bytes and HBM fraction.  Then again
    with the transposed copy (spc5_build_transpose): the transposed product
    as a plain SpMV over A^T, and the value update refreshing both copies."""
    from paper_2307_14774_gb300.autograd import SpMVFunction
    A = synth.workload("stencil27")
    dev = [torch.from_numpy(a).cuda() for a in (A.rowptr, A.colidx, A.vals)]
    M = spc5.spc5_convert_csr(A.nrows, A.ncols, A.nnz, *dev, store_dtype=spc5.SPC5_F32,
                              r=4, c=8)
    vals = dev[2].clone().requires_grad_(True)
    x = torch.from_numpy(synth.vector_uniform(A.ncols, seed=1).astype("float32")).cuda()
    x.requires_grad_(True)
    g = torch.from_numpy(synth.vector_normal(A.nrows, seed=2).astype("float32")).cuda()
    flush = torch.empty(256 * 2 ** 20, dtype=torch.uint8, device="cuda")

    def step(backward):
        vals.grad = None
        x.grad = None
        y = SpMVFunction.apply(M, vals, x)
        if backward:
            y.backward(g)

    def timed(fn):
        for _ in range(3):
            fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return sorted(ts)[len(ts) // 2]

    out = {"matrix": "27-point stencil 100^3, FP32 values", "nnz": A.nnz}
    for name, bwd in (("forward", False), ("forward_backward", True)):
        ms = timed(lambda: step(bwd))
        # forward: 2 nnz flops; backward: 2 nnz (A^T g) + nnz (g[row] x[col])
        flops = 2 * A.nnz + (3 * A.nnz if bwd else 0)
        out[name] = {"ms": round(ms, 4), "gflops": round(flops / (ms * 1e-3) / 1e9, 1)}
    info = M.info()
    nb, npan, mb = info["nblocks"], info["npanels"], info["mask_bytes"]
    meta = 4 * nb + mb * nb + 8 * (npan + 1)
    y = torch.empty(A.nrows, dtype=torch.float32, device="cuda")
    dx = torch.empty(A.ncols, dtype=torch.float32, device="cuda")
    dvals = torch.empty(A.nnz, dtype=torch.float32, device="cuda")
    vals64 = dev[2]
    x32 = x.detach()
    kernels = {
        # CSR-ordered FP64 values gathered through value_src, stored as FP32
        "set_values": (lambda: spc5.spc5_set_values(M, vals64), (8 + 4 + 4) * A.nnz),
        "spmv": (lambda: spc5.spc5_spmv(M, x32, y), algorithmic_bytes(info)),
        # stored values + blocks + g + dx (written once)
        "spmv_t": (lambda: spc5.spc5_spmv_t(M, g, dx),
                   4 * A.nnz + meta + 4 * A.nrows + 4 * A.ncols),
        # blocks + g + x + the CSR row pointer + dvals (written from each
        # row's CSR start; value_src is not read)
        "values_grad": (lambda: spc5.spc5_values_grad(M, g, x32, dvals),
                        meta + 4 * A.nrows + 4 * A.ncols + 4 * (A.nrows + 1) + 4 * A.nnz),
    }
    out["kernels"] = {}

    def run_kernels(ks):
        for name, (fn, b) in ks.items():
            ms = timed(fn)
            out["kernels"][name] = {"us": round(ms * 1e3, 2), "bytes": int(b),
                                    "gbs": round(b / (ms * 1e-3) / 1e9, 1),
                                    "frac": round(b / (ms * 1e-3) / 1e9 / hbm, 3)}
    run_kernels(kernels)
    # the transposed copy: spc5_spmv_t becomes a product over A^T (the
    # 27-point pattern is symmetric, so A^T has A's blocks and bytes), and
    # spc5_set_values refreshes it too
    t0 = time.perf_counter()
    spc5.spc5_build_transpose(M)
    torch.cuda.synchronize()
    out["build_transpose_ms"] = round((time.perf_counter() - t0) * 1e3, 2)
    ms = timed(lambda: step(True))
    out["forward_backward_transposed"] = {"ms": round(ms, 4),
                                          "gflops": round(5 * A.nnz / (ms * 1e-3) / 1e9, 1)}
    run_kernels({"spmv_t_transposed": (lambda: spc5.spc5_spmv_t(M, g, dx),
                                       algorithmic_bytes(info)),
                 "set_values_with_transposed": (lambda: spc5.spc5_set_values(M, vals64),
                                                2 * (8 + 4 + 4) * A.nnz)})
    log(f"autograd: {out}")
    del M, dev, flush
    return out


def batched_section(torch, spc5, synth, stream, hbm, log, nmat=256, reps=10):
    """256 matrices of uneven size (n log-uniform in [1e3, 2e5]; 5-point,
    27-point and power-law generators in turn), FP32 values, each converted
    into the block shape and mapping whose row-group plan (the plan the
    batched kernel runs) the autotuner finds fastest; for every k in
    {1, 4, 8, 16}: one persistent batched launch captured in a CUDA graph,
    timed by replaying the graph."""
    import math
    import numpy as np
    rng = np.random.default_rng(4)
    sizes = np.exp(rng.uniform(math.log(1e3), math.log(2e5), nmat))
    mats, shapes = [], {}
    t0 = time.perf_counter()
    nnz_total = 0
    mat_bytes, vec_elems = 0, 0
    for i, n in enumerate(sizes):
        kind = i % 3
        if kind == 0:
            side = max(4, int(round(math.sqrt(n))))
            A = synth.laplace2d(side, side)
        elif kind == 1:
            side = max(3, int(round(n ** (1 / 3))))
            A = synth.stencil27(side, side, side, values="normal", seed=i)
        else:
            A = synth.powerlaw(int(n), seed=100 + i)
        dev = [torch.from_numpy(a).cuda() for a in (A.rowptr, A.colidx, A.vals)]
        M = spc5.spc5_convert_tuned_ex(A.nrows, A.ncols, A.nnz, *dev, store_dtype=spc5.SPC5_F32,
                                       iters=3, rows_plan=True, stream=stream)
        info = M.info()
        key = f"{info['r']}x{info['c']}/G{info['lanes_per_row']}"
        shapes[key] = shapes.get(key, 0) + 1
        mats.append((M, A.nrows, A.ncols))
        nnz_total += A.nnz
        mat_bytes += algorithmic_bytes(info) - 4 * (A.nrows + A.ncols)  # matrix part
        vec_elems += A.nrows + A.ncols
    setup_s = time.perf_counter() - t0
    log(f"batched: {nmat} matrices, nnz {nnz_total}, converted+tuned in {setup_s:.1f}s")
    rows = []
    for k in (1, 4, 8, 16):
        X = [torch.rand(nc, k, device="cuda", dtype=torch.float32) * 2 - 1 for _, _, nc in mats]
        Y = [torch.empty(nr, k, device="cuda", dtype=torch.float32) for _, nr, _ in mats]
        B = spc5.Batch([m for m, _, _ in mats], X, Y, k, stream=stream)
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            B.run(stream=side)
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            B.run(stream=torch.cuda.current_stream())
        for _ in range(3):
            graph.replay()
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(reps)]
        for e0, e1 in evs:
            e0.record()
            graph.replay()
            e1.record()
        torch.cuda.synchronize()
        us = statistics.median(e0.elapsed_time(e1) for e0, e1 in evs) * 1e3
        b = mat_bytes + 4 * k * vec_elems  # FP32 X [n][k] read, Y [n][k] written
        rows.append({"k": k, "us": round(us, 2),
                     "gflops": round(2.0 * nnz_total * k / (us * 1e-6) / 1e9, 1),
                     "bytes": int(b), "gbs": round(b / (us * 1e-6) / 1e9, 1),
                     "frac": round(b / (us * 1e-6) / 1e9 / hbm, 3)})
        del B, graph, X, Y
    return {"matrices": nmat, "nnz_total": int(nnz_total), "dtype": "f32 values, f32 x/y",
            "bytes_note": "algorithmic bytes: every matrix's values, block columns, masks and "
                          "panel pointers once, plus k FP32 x and y values per row and column",
            "n_range": [int(sizes.min()), int(sizes.max())], "setup_s": round(setup_s, 1),
            "tuned_shapes": shapes, "rows": rows,
            "launch": "one CUDA graph replay = one persistent kernel over all matrices' tiles "
                      "(+ one fixup kernel for split panels)"}


def cpu_model() -> str:
    """Host CPU model (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine()


def host_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_baseline(hosts, log, reps=5):
    """The oracle's CSR product (Section 2.3) on the host cores over the
    whole matrices: the parity oracle as it stands (compensated FP64 sum,
    with S_i) and the textbook loop, each on one thread and on every core the
    process may use (OpenMP over rows; each row summed by one thread, so the
    results do not depend on the thread count).  Returns the timing record
    and the oracle's (y, S) per matrix, which the parity check of every
    benchmark case uses."""
    import oracle
    O = oracle.timing_oracle()
    if O is None:
        O = oracle.Oracle()
        log("oracle OpenMP build unavailable: CPU baseline on one thread")
    nthreads = host_threads()
    flops = sum(2.0 * A.nnz for A, _ in hosts.values())
    rec = {"cpu_model": cpu_model(), "host_threads": nthreads}
    refs = {}

    def passes(fn, n, warm):
        for _ in range(warm):
            for name, (A, x) in hosts.items():
                fn(name, A, x)
        ts = []
        for _ in range(n):
            t0 = time.perf_counter()
            for name, (A, x) in hosts.items():
                fn(name, A, x)
            ts.append(time.perf_counter() - t0)
        return statistics.median(ts)

    def comp(name, A, x):
        refs[name] = O.csr_spmv(A, x)

    def plain(name, A, x):
        O.csr_spmv_plain(A, x)

    for label, nthr, n in (("all", nthreads, reps), ("one", 1, 1)):
        used = O.set_threads(nthr)
        for kind, fn in (("oracle", comp), ("plain", plain)):
            secs = passes(fn, n, 1 if label == "all" else 0)
            rec[f"{kind}_{label}"] = {"gflops": round(flops / secs / 1e9, 4), "threads": used,
                                      "s_per_pass": round(secs, 4)}
    O.set_threads(nthreads)
    log(f"cpu baseline: {rec}")
    return rec, refs


def run_native(args):
    import numpy as np
    import torch

    import paper_2307_14774_gb300 as spc5
    import synth

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    log = (lambda m: print(f"[bench] {m}", file=sys.stderr, flush=True)) if rank == 0 else (
        lambda m: None)
    spc5.load()
    peaks = fma_peaks(spc5, log)
    names = [n for n in args.matrices.split(",") if n]
    cases, hosts = build_cases(names, torch, spc5, synth, log, args.betas.split(","),
                               tune=not args.no_tune, scale=args.scale)
    stream = torch.cuda.current_stream()
    nlaunch = len(cases)

    def step(events=None):
        for i, cs in enumerate(cases):
            if events is not None:
                events[i][0].record(stream)
            spc5.spc5_spmv(cs["M"], cs["x"], cs["y"], 1.0, 0.0, stream)
            if events is not None:
                events[i][1].record(stream)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    ev = [[[torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)]
           for _ in cases] for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local, args.clocks_out) as clk:
        time.sleep(0.3)
        torch.cuda.nvtx.range_push("spc5_timed")
        t_start.record(stream)
        for k in range(args.steps):
            step(ev[k])
        t_end.record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        time.sleep(0.3)
    if world > 1:
        torch.distributed.barrier()
    total_ms = max_over_ranks(t_start.elapsed_time(t_end), world)
    ms_per_step = total_ms / args.steps
    flops_per_step = sum(2.0 * cs["nnz"] for cs in cases)
    value = whole_job_value(world, flops_per_step, ms_per_step * 1e-3)

    # per-launch durations (CUDA events on the launching stream)
    per_case_ms = [statistics.median(ev[k][i][0].elapsed_time(ev[k][i][1])
                                     for k in range(args.steps)) for i in range(nlaunch)]
    sum_launch_ms = sum(sum(ev[k][i][0].elapsed_time(ev[k][i][1]) for i in range(nlaunch))
                        for k in range(args.steps))
    bytes_per_step = sum(cs["bytes"] for cs in cases)
    hbm, peak_kind = measured_peaks()
    peak_kind = (f"{peak_kind}: MEASURED_PEAKS.json hbm_gbs (copy bandwidth)"
                 if peak_kind == "measured" else "fallback: 6.8 TB/s")
    if "f64" in peaks:
        fp64_peak, fp64_kind = peaks["f64"], "measured: spc5_measure_fma_peak (FP64 FMA chains)"
    else:
        fp64_peak, fp64_kind = FP64_NOMINAL_TFLOPS, "nominal: 152 SMs x 2 FMA/cycle x 2070 MHz"
    achieved = bytes_per_step * args.steps / (sum_launch_ms * 1e-3) / 1e9
    achieved_tflops = flops_per_step * args.steps / (sum_launch_ms * 1e-3) / 1e12
    case_rows = []
    for cs, ms in zip(cases, per_case_ms):
        gbs = cs["bytes"] / (ms * 1e-3) / 1e9
        gf = 2.0 * cs["nnz"] / (ms * 1e-3) / 1e9
        t_hbm = cs["bytes"] / (hbm * 1e9) * 1e6
        t_fp64 = 2.0 * cs["nnz"] / (fp64_peak * 1e12) * 1e6
        info = cs["info"]
        conv_bytes = (4 * (info["nrows"] + 1) + 12 * cs["nnz"]  # CSR read
                      + (VALUE_BYTES[info["value_dtype"]] + 4) * cs["nnz"]  # values, value_src
                      + (4 + info["mask_bytes"]) * info["nblocks"] + 8 * (info["npanels"] + 1))
        case_rows.append({"matrix": cs["matrix"], "beta": f"{cs['r']}x{cs['c']}",
                          "nnz": cs["nnz"], "nblocks": info["nblocks"],
                          "filling": round(info["filling"], 4), "bytes": cs["bytes"],
                          "us": round(ms * 1e3, 2), "gflops": round(gf, 1),
                          "gbs": round(gbs, 1), "frac": round(gbs / hbm, 3),
                          "fp64_frac": round(gf / (fp64_peak * 1e3), 3),
                          "bound": "fp64" if t_fp64 > t_hbm else "hbm",
                          "floor_us": round(max(t_hbm, t_fp64), 2),
                          "plan": plan_label(info),
                          "convert_ms": round(cs["convert_s"] * 1e3, 2),
                          "convert_gbs": round(conv_bytes / cs["convert_s"] / 1e9, 1)})
    step_roof = {"achieved_gbs": round(achieved, 1), "frac": round(achieved / hbm, 4),
                 "fp64_tflops": round(achieved_tflops, 4),
                 "fp64_frac": round(achieved_tflops / fp64_peak, 4),
                 "bytes_per_step": bytes_per_step, "flops_per_step": flops_per_step,
                 "note": "all launches of a step: algorithmic bytes and FLOPs over the sum of "
                         "their event-timed durations"}
    ratios = ncu_traffic_ratios()

    # the oracle on the host cores (rank 0 at N=1): timed, and its products
    # are the reference every case is checked against
    cpu_rec, refs = None, {}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_rec, refs = cpu_baseline(hosts, log)
        for cs, row in zip(cases, case_rows):
            spc5.spc5_spmv(cs["M"], cs["x"], cs["y"], 1.0, 0.0, stream)
            torch.cuda.synchronize()
            y_ref, scale = refs[cs["matrix"]]
            row["max_err_over_tol"] = round(
                err_over_tol(cs["y"].cpu().numpy(), y_ref, scale, FP64_TOL), 4)

    result = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": round(ms_per_step, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "FP64 SpMV, every beta(r,c) in {1x8,2x4,2x8,4x4,4x8,8x4}, over: "
                   + "; ".join(DESCR[n] for n in names),
                   "matrices": names, "betas": [f"{r}x{c}" for r, c in BETAS],
                   "spmv_per_step": nlaunch, "nnz_per_step": int(flops_per_step / 2),
                   "scale": args.scale,
                   "l2": "inputs larger than L2: every SpMV streams >= "
                         f"{min(cs['bytes'] for cs in cases) / 1e6:.0f} MB (L2 129 MB)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                   "mapping": "autotuned per matrix during setup (spc5_tune): lanes per row, "
                              "row-stream bodies, block-balanced or expanded plan"
                              if not args.no_tune else "planner default"},
        "roofline": roofline_object(case_rows, hbm, peak_kind, fp64_peak, fp64_kind, ratios,
                                    step_roof),
        "fma_peaks_tflops": {k: round(v, 4) for k, v in peaks.items()},
        "gpu_launches": sum(cs["info"].get("launches_per_spmv", 1) for cs in cases) * args.steps,
        "cases": case_rows,
        "convert": {"ms_total": round(sum(cs["convert_s"] for cs in cases) * 1e3, 1),
                    "note": "CSR (device) -> beta(r,c), all 24 conversions, wall clock; "
                            "per case convert_gbs = minimal bytes (CSR read; values, value "
                            "sources, block columns, masks, panel pointers written) over the "
                            "conversion's wall time"},
    }
    clocks = clk.summary()
    if clocks:
        result["clocks"] = clocks

    if case_rows and all("max_err_over_tol" in r for r in case_rows):
        result["parity"] = {"tol": FP64_TOL,
                            "max_err_over_tol": max(r["max_err_over_tol"] for r in case_rows),
                            "note": "every case's y (the tuned plan timed above) against the "
                                    "CPU oracle's compensated FP64 CSR product, "
                                    "|y - y_ref| / (1e-13 * sum_j |a_ij x_j|), worst row"}

    if not args.no_precision and rank == 0 and refs:
        prec = precision_section(hosts, refs, torch, spc5, stream, hbm, case_rows, log,
                                 tune=not args.no_tune)
        result["precision"] = {
            "note": "FP32/BF16 value storage, FP32 x/y/accumulation; error vs the CPU oracle "
                    "(FP64 values and x), relative to tol * sum_j |a_ij x_j|",
            "rows": prec,
            "summary": {dt: {"gflops_total": round(
                sum(2.0 * cs_nnz for cs_nnz in [hosts[rw["matrix"]][0].nnz for rw in prec
                                                if rw["dtype"] == dt])
                / (sum(rw["us"] for rw in prec if rw["dtype"] == dt) * 1e-6) / 1e9, 1),
                "max_err_over_tol": max(rw["max_err_over_tol"] for rw in prec if rw["dtype"] == dt)}
                for dt in ("f32", "bf16")} if prec else {}}

    if not args.no_batched and rank == 0:
        result["batched"] = batched_section(torch, spc5, synth, stream, hbm, log)
    if not args.no_cg and rank == 0:
        result["ircg"] = cg_section(torch, spc5, synth, stream, hbm, log, tune=not args.no_tune)
    if not args.no_grad and rank == 0:
        result["autograd"] = grad_section(torch, spc5, synth, hbm, log)
    if not args.no_dense and rank == 0:
        result["dense"] = dense_section(torch, spc5, synth, stream, hbm, log,
                                        tune=not args.no_tune)
    if not args.no_hybrid and rank == 0:
        result["hybrid"] = {
            "note": "single-value blocks stored as scalar CSR entries (FP64); algorithmic bytes "
                    "add 4 bytes per scalar column and the scalar row pointer",
            "rows": hybrid_section(hosts, torch, spc5, stream, hbm, case_rows, log,
                                   tune=not args.no_tune)}

    # end to end through the C-ABI with host vectors: every step copies x from
    # pinned host memory and reads y back
    if not args.no_e2e:
        hx, hy = {}, {}
        for name in names:
            A, x = hosts[name]
            hx[name] = torch.from_numpy(x).pin_memory()
            hy[name] = torch.empty(A.nrows, dtype=torch.float64).pin_memory()
        h2d = sum(8 * cs["info"]["ncols"] for cs in cases)
        d2h = sum(8 * cs["info"]["nrows"] for cs in cases)

        def e2e_step():
            for cs in cases:
                spc5.spc5_spmv(cs["M"], hx[cs["matrix"]], hy[cs["matrix"]], 1.0, 0.0, stream)

        for _ in range(3):
            e2e_step()
        if world > 1:
            torch.distributed.barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            e2e_step()
        torch.cuda.synchronize()
        dt = max_over_ranks((time.perf_counter() - t0) / args.steps, world)
        result["e2e"] = {"value": round(whole_job_value(world, flops_per_step, dt), 2),
                         "unit": UNIT,
                         "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                         "ms_per_step": round(dt * 1e3, 3),
                         "api": "spc5_spmv with pinned host x and y"}

    if cpu_rec is not None:
        best = cpu_rec["oracle_all"]
        result["cpu_baseline"] = {
            "value": best["gflops"], "unit": UNIT, "cores": best["threads"], "kind": "oracle",
            "cpu_model": cpu_rec["cpu_model"],
            "one_thread": cpu_rec["oracle_one"]["gflops"],
            "textbook_csr": {"all_cores": cpu_rec["plain_all"]["gflops"],
                             "one_thread": cpu_rec["plain_one"]["gflops"]},
            "sample": "whole matrices: the oracle's CSR product y = A x (compensated FP64 sum "
                      "with S_i, the parity reference) over the 4 matrices, OpenMP over rows on "
                      f"{best['threads']} host threads (median of 5 passes) and on one thread; "
                      "textbook_csr: the uncompensated CSR loop, same passes"}
    if args.cases_out and rank == 0:
        with open(args.cases_out, "w") as f:
            json.dump(case_rows, f, indent=1)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# --------------------------------------------------------------- reference --

def run_reference(args):
    """The oracle timed on the host cores: each step is the workload's 24
    FP64 products (every matrix once per beta) computed by the oracle's CSR
    product (compensated FP64 sum, the parity reference) over the whole
    matrices, OpenMP over rows on every host thread the process may use."""
    rank, world, local = dist_env()
    if rank != 0:
        return
    import oracle
    import synth
    names = [n for n in args.matrices.split(",") if n]
    O = oracle.timing_oracle() or oracle.Oracle()
    threads = O.set_threads(host_threads())
    mats = []
    for name in names:
        A = synth.workload(name, args.scale)
        mats.append((A, synth.vector_uniform(A.ncols, seed=1)))
    betas = [b for b in args.betas.split(",") if b]

    def step():
        for _ in betas:
            for A, x in mats:
                O.csr_spmv(A, x)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = (time.perf_counter() - t0) / args.steps
    flops = len(betas) * sum(2.0 * A.nnz for A, _ in mats)
    value = flops / dt / 1e9
    sample = ("whole matrices: the CPU oracle's CSR product (compensated FP64 sum), each "
              f"matrix once per beta, OpenMP over rows on {threads} host threads")
    result = {
        "metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(dt * 1e3, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference",
        "config": {"workload": "FP64 SpMV, every beta(r,c) in {1x8,2x4,2x8,4x4,4x8,8x4}, over: "
                   + "; ".join(DESCR[n] for n in names), "matrices": names,
                   "spmv_per_step": len(betas) * len(mats)},
        "cpu_baseline": {"value": round(value, 4), "unit": UNIT, "cores": threads,
                         "kind": "oracle", "cpu_model": cpu_model(), "sample": sample},
        "e2e": {"value": round(value, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(result), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_native(args)


if __name__ == "__main__":
    main()
