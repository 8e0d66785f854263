#!/usr/bin/env python
"""Benchmark: FP64 sparse matrix-vector multiplication y = A x on GB300.

Workload (one step = one SpMVM over the whole matrix, the hot path of the
paper's Sect. 2 CRS kernel): the synthetic Holstein-Hubbard-like matrix,
N = 6,000,000 rows, symmetric, banded plus 20% scattered entries, about 13
entries per row (see paper_0910_4836_gb300/synth.py, hh_like).  The matrix
(about 1 GB) is resident in HBM like an operator inside an eigen-solver; x
and y are the step's input and output.

Prints ONE JSON line.  --impl reference times the CPU oracle instead (the
paper's best CPU setting: CRS with an OpenMP static schedule).
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

# The CPU oracle's OpenMP threads sit one per core, packed (the paper's
# pinned runs).  Set before any OpenMP runtime in this process starts.
os.environ.setdefault("OMP_PROC_BIND", "close")
os.environ.setdefault("OMP_PLACES", "cores")
# host cores this process may use, read before any OpenMP binding narrows
# the main thread's own mask to one core
AFFINITY_CORES = len(os.sched_getaffinity(0))

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SpMVM GFlop/s & HBM GB/s vs roofline; batched & fwd+bwd speedup vs plain"
WORKLOAD = ("hh_like N=6,000,000 FP64 SpMVM, fastest of CRS and the JDS family "
            "(symmetric banded + 20% scattered, ~13 nnz/row)")
WORKLOADS = {
    0: "laplace2d 64x64 FP64 SpMVM (5-point, Dirichlet; latency-bound)",
    1: WORKLOAD,
    2: "zipf_rows N=4,000,000 FP64 SpMVM (Zipf(2) row lengths up to 5000, random columns)",
    4: "stencil27 100^3 FP64 SpMVM (27-point, N=1,000,000)",
}
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3000)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--config", type=int, default=1, choices=[1, 2, 4])
    p.add_argument("--kernel", default="auto", help="auto, or a name prefix (CRS, JDS, NUJDS, ...)")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the FP32, batched and forward+backward measurements")
    p.add_argument("--cpu-seconds", type=float, default=15.0)
    p.add_argument("--ncu-case", action="store_true",
                   help="no timing: run 3 launches of the --kernel candidate on a 2,000,000-row "
                        "HH-like matrix (larger than L2, small enough for an ncu capture)")
    p.add_argument("--micro", action="store_true",
                   help="instead of the SpMVM step: the basic gather operations of Sect. 3.1 "
                        "(ADD/SCP over PD, CS, IS, IR; stride sweep; Gaussian stride plane), one JSON line")
    p.add_argument("--analysis", action="store_true",
                   help="instead of the SpMVM step: stride distribution and sectors per warp gather of "
                        "every storage scheme, and block / lanes / window sweeps (Sect. 4), one JSON line")
    return p.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def make_workload(cfg):
    from paper_0910_4836_gb300 import synth as S
    A = S.config(cfg)
    x = S.vector(A.n_cols, cfg)
    return A, x


def algorithmic_bytes(n_rows, n_cols, nnz, vbytes=8):
    # val + col streamed once, row_ptr once, x read at least once, y written once
    return vbytes * nnz + 4 * nnz + 4 * (n_rows + 1) + vbytes * n_cols + vbytes * n_rows


# ------------------------------------------------------------- clocks ------

class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index
        self.path = os.path.join("/tmp", f"gbspmv_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(rows), "reasons": reasons,
                "power_w_max": max((float(r[3]) for r in rows if r[3].replace(".", "").isdigit()),
                                   default=None)}


# ---------------------------------------------------------- distributed ----

def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, device=None) -> float:
    """Largest `value` over all ranks (the job's time is the slowest
    replica's); the identity without a process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, max_ms: float) -> float:
    """Whole-job rate: the units all ranks processed over the slowest time."""
    return world * units_per_rank / (max_ms * 1e-3)


# the functions a step kernel is made of (kernel, its launchers), by scheme
STEP_FUNCTIONS = {"SELL": ("jds.cu", ("sell_walk(const JdsArgs &a)", "sell_kernel(JdsArgs a)", "sell_kernel_f64(JdsArgs a)",
                                     "launch_sell_U(JdsArgs a", "launch_sell(const Mat"))}


def _function_text(src: str, signature: str) -> str:
    """The text of the definition that contains `signature`, from the start
    of its line (attributes such as launch bounds included) and its
    template header, through its closing brace."""
    j = src.index(signature)
    i = src.rfind("\n", 0, j) + 1
    prev = src.rfind("\n", 0, max(i - 1, 0)) + 1
    if src[prev:i].lstrip().startswith("template"):
        i = prev
    j = src.index("{", j)
    depth = 0
    for k in range(j, len(src)):
        depth += {"{": 1, "}": -1}.get(src[k], 0)
        if depth == 0:
            return src[i:k + 1]
    raise ValueError(signature)


def kernel_source_hash(kname: str = "SELL") -> str:
    """Hash of the step kernel's own source (its functions and the
    accumulator header), so that edits elsewhere in the library do not
    invalidate a measurement of it."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_0910_4836_gb300", "csrc")
    with open(os.path.join(csrc, "accum.cuh"), "rb") as fh:
        h.update(fh.read())
    fam = STEP_FUNCTIONS.get(kname.split()[0])
    if fam is None:
        with open(os.path.join(csrc, "jds.cu"), "rb") as fh:
            h.update(fh.read())
    else:
        with open(os.path.join(csrc, fam[0])) as fh:
            src = fh.read()
        for sig in fam[1]:
            h.update(_function_text(src, sig).encode())
    return h.hexdigest()[:12]


# DRAM bytes (read + write) per launch of the step kernel on the full
# workload, from one ncu capture (dram__bytes_read.sum + dram__bytes_write.sum,
# a one-pass metric set), keyed by (config, kernel, source hash); a different
# hash means the kernel changed since and traffic is reported null.
NCU_TRAFFIC = {(1, "SELL row_only w=128 u=4", "6ca13edede86"): 1142551552 + 40393984}


# --------------------------------------------------------------- ours ------

def _timer(dev):
    import torch
    stream = torch.cuda.current_stream(dev)

    def time_launches(fn, reps):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
        torch.cuda.synchronize(dev)
        ev[0].record(stream)
        for i in range(reps):
            fn()
            ev[i + 1].record(stream)
        torch.cuda.synchronize(dev)
        return [ev[i].elapsed_time(ev[i + 1]) for i in range(reps)]

    return time_launches


def candidates(M, A, x, only=None):
    """(name, handle, input vector, algorithmic bytes, setting) of every
    storage scheme and kernel option on this matrix (the paper's serial
    comparison of Sect. 3.2, on GB300).  JDS-family inputs are in their
    permuted basis.  `only`: a name prefix; other schemes are not built."""
    crs_b = algorithmic_bytes(A.n_rows, A.n_cols, A.nnz)
    out = []
    want = lambda name: only is None or name.startswith(only)
    for l, r in ((4, 4), (8, 2), (16, 2)):
        out.append((f"CRS vector l{l} r{r}", M, x, crs_b, ("vector", l, r)))
    for t in (1024, 2048):
        out.append((f"CRS tiled {t}", M, x, crs_b, ("tiled", t)))
    for perm, w, u in (("row_only", 128, 2), ("row_only", 128, 4), ("row_only", 512, 4),
                       ("row_only", 4096, 4)):
        name = f"SELL {perm} w={w} u={u}"
        if want(name):
            G = M.to_jds("SELL", perm, window=w, unroll=u)
            xs = G.permute(x) if perm == "symmetric" else x
            gb = 12 * A.nnz + 4 * (G.n_blocks + 1) + 4 * A.n_rows + 8 * A.n_cols + 8 * A.n_rows
            out.append((name, G, xs, gb, ("fixed",)))
    for perm, w, u in (("row_only", 64, 2), ("row_only", 64, 4), ("row_only", 128, 4)):
        name = f"PSELL {perm} w={w} u={u}"
        if want(name):
            G = M.to_jds("PSELL", perm, window=w, unroll=u)
            xs = G.permute(x) if perm == "symmetric" else x
            gb = 12 * A.nnz + 4 * (G.n_blocks + 1) + 4 * A.n_rows + 8 * A.n_cols + 8 * A.n_rows
            out.append((name, G, xs, gb, ("fixed",)))
    for perm in ("symmetric", "row_only"):
        if only is not None and not any(f"{f} {perm}".startswith(only) or only.startswith(f"{f} {perm}")
                                        for f in ("JDS", "NUJDS", "NBJDS", "JDS_LITERAL", "RBJDS", "SOJDS")):
            continue
        J = M.to_jds("JDS", perm)
        xp = J.permute(x) if perm == "symmetric" else x
        jb = 12 * A.nnz + 4 * (J.n_diag + 1) + 8 * A.n_cols + 8 * A.n_rows
        for fmt, b, u, r in (("JDS", 0, 0, 1), ("NUJDS", 0, 2, 1), ("NUJDS", 0, 4, 1), ("NUJDS", 0, 8, 1),
                             ("NUJDS", 0, 2, 2), ("NUJDS", 0, 4, 2), ("NUJDS", 0, 2, 4), ("NUJDS", 0, 4, 4),
                             ("NBJDS", 1024, 0, 1), ("NBJDS", 2048, 0, 1), ("JDS_LITERAL", 0, 0, 1)):
            name = (f"{fmt} {perm}" + (f" b={b}" if b else "") + (f" u={u}" if u else "")
                    + (f" r={r}" if r > 1 else ""))
            out.append((name, J, xp, jb, ("jds", fmt, b, u, r)))
        for fmt in ("RBJDS", "SOJDS"):
            if not want(f"{fmt} {perm} b=1024"):
                continue
            R = M.to_jds(fmt, perm, block=1024)
            rb = jb + 4 * (R.n_blocks + 1)
            out.append((f"{fmt} {perm} b=1024", R, xp, rb, ("fixed",)))
    return out


def configure(H, how):
    if how[0] == "vector":
        H.set_kernel("vector", lanes=how[1], rows_per_warp=how[2])
    elif how[0] == "tiled":
        H.prepare_tiled(how[1])
    elif how[0] == "jds":
        H.set_format(how[1], block=how[2], unroll=how[3])
        H.set_kernel("vector", rows_per_warp=how[4])


def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)

    import paper_0910_4836_gb300 as g
    from paper_0910_4836_gb300 import CRSMatrix
    g.build()
    time_launches = _timer(dev)

    A, x_host = make_workload(args.config)
    M = CRSMatrix.from_host(A, device=dev, dtype=torch.float64)
    x = torch.as_tensor(x_host).to(dev)
    y = torch.empty(A.n_rows, dtype=torch.float64, device=dev)
    peak, peak_kind = peaks()

    # every scheme timed (median of 10 launches); the fastest is the step
    table, best = {}, None
    for name, H, xin, nbytes, how in candidates(M, A, x, None if args.kernel == "auto" else args.kernel):
        if args.kernel != "auto" and not name.startswith(args.kernel):
            continue
        configure(H, how)
        t = statistics.median(time_launches(lambda: H.spmv(xin, out=y), 10))
        table[name] = {"gflops": round(2.0 * A.nnz / (t * 1e-3) / 1e9, 1),
                       "gbs": round(nbytes / (t * 1e-3) / 1e9, 1), "ms": round(t, 4),
                       "frac": round(nbytes / (t * 1e-3) / 1e9 / peak, 3)}
        # a later scheme replaces the choice only when more than 1% faster,
        # so near-ties keep the earlier (listed first) scheme from run to run
        if best is None or t < 0.99 * best[0]:
            best = (t, name, H, xin, nbytes, how)
    _, kname, H, xin, alg, how = best
    configure(H, how)

    def step():
        H.spmv(xin, out=y)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    with ClockSampler(torch.cuda.current_device() if world == 1 else local) as clk:
        times = time_launches(step, args.steps)
        torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    total_ms = max_over_ranks(sum(times), dev)
    ms = total_ms / args.steps
    flops = 2.0 * A.nnz
    gflops = job_throughput(flops, world, ms) / 1e9
    gbs = alg / (ms * 1e-3) / 1e9
    h = kernel_source_hash(kname)
    traffic = NCU_TRAFFIC.get((args.config, kname, h))

    # end to end through the public API: every step is one C-ABI call with
    # host vectors (gbsp_spmv_host), which copies x in from pinned host
    # memory, runs the product and copies y back to pinned host memory, in
    # order on its stream.  Steps go round-robin over four streams, each
    # with its own device stages and host output: a stream's copy in,
    # product and copy out run in order, so four of them keep the copies in
    # both directions and the products overlapping.
    nstr = 4
    xh = xin.detach().cpu().pin_memory()
    yh = [torch.empty(A.n_rows, dtype=torch.float64).pin_memory() for _ in range(nstr)]
    stages = [H.host_stage() for _ in range(nstr)]
    streams = [torch.cuda.Stream(dev) for _ in range(nstr)]
    main = torch.cuda.current_stream(dev)

    def e2e_steps(n):
        for i in range(n):
            b = i % nstr
            H.spmv_host(xh, out=yh[b], stage=stages[b], stream=streams[b])

    def fenced(n):
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(main)
        for st in streams:
            st.wait_event(t0)
        e2e_steps(n)
        for st in streams:
            main.wait_stream(st)
        t1.record(main)
        return t0, t1

    fenced(4)
    torch.cuda.synchronize(dev)
    e2e_n = 50
    t_start, t_end = fenced(e2e_n)
    torch.cuda.synchronize(dev)
    e2e_ms = t_start.elapsed_time(t_end) / e2e_n

    result = None
    if rank == 0:
        basis = "original basis" if kname.startswith("CRS") else "permuted basis (Sect. 2)"
        result = {
            "metric": METRIC, "value": round(gflops, 2), "unit": "GFlop/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 5),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded SplitMix64; stand-in for the paper's Holstein-Hubbard matrix)",
            "hbm_gbs": round(gbs, 1),
            "config": {"workload": WORKLOADS.get(args.config, WORKLOAD), "config_index": args.config, "n_rows": A.n_rows,
                       "nnz": A.nnz, "kernel": kname, "vectors": basis,
                       "l2": "inputs larger than L2 (matrix ~1 GB), no flush",
                       "parallelism": f"replicas x{world}"},
            "roofline": {"bound": "hbm", "achieved": round(gbs, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(gbs / peak, 4), "traffic": traffic,
                         "frac_of_8tbs_spec": round(gbs / 8000.0, 4),
                         "algorithmic_bytes": alg, "peak_source": f"{peak_kind} hbm_gbs (burst)",
                         "kernel_source_hash": h},
            "e2e": {"value": round(world * flops / (e2e_ms * 1e-3) / 1e9, 2), "unit": "GFlop/s",
                    "h2d_bytes_per_step": 8 * A.n_cols, "d2h_bytes_per_step": 8 * A.n_rows,
                    "ms_per_step": round(e2e_ms, 4),
                    "how": "one gbsp_spmv_host call per step (pinned host x in, product, pinned host y out, "
                           "in order on its stream); steps round-robin over four streams and stage sets"},
            "gpu_launches": args.steps * launches_per_step(kname, H),
            "clocks": clk.summary(),
            "formats": table,
        }
        if not args.no_extras:
            result["fp32"] = fp32_numbers(M, A, x, y, dev, time_launches, table[kname]["ms"])
            torch.cuda.empty_cache()
            result["symmetric"] = symmetric_numbers(M, A, x, dev, time_launches, table[kname]["ms"])
            del table
            torch.cuda.empty_cache()
            result["spmm_adjoint"] = spmm_adjoint_numbers(M, A, x, dev, time_launches, peak)
            torch.cuda.empty_cache()
            result["batched"] = batched_speedups(dev, time_launches)
            torch.cuda.empty_cache()
            result["fwd_bwd"] = fwd_bwd_speedup(dev, time_launches)
            torch.cuda.empty_cache()
            result["zipf_rows"] = zipf_numbers(dev, time_launches, peak)
            torch.cuda.empty_cache()
            result["hybrid_dia"] = hybrid_numbers(dev, time_launches, peak)
            torch.cuda.empty_cache()
            result["laplace_64x64"] = small_numbers(dev, time_launches)
        result["cpu_baseline"] = cpu_baseline(A, x_host, args.cpu_seconds)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return result


def launches_per_step(kname, H):
    if kname.startswith("JDS_LITERAL"):
        return int(H.n_diag) + 1  # one zeroing launch and one launch per diagonal
    return 1



# ------------------------------------------------------------- extras ------

def fp32_numbers(M, A, x, y64, dev, time_launches, ms64):
    """FP32 values with compensated (Dot2) row sums on the same matrix: speed
    and the error against the FP64 GPU result, relative to sum |a||x|."""
    import torch
    from paper_0910_4836_gb300 import CRSMatrix
    M32 = CRSMatrix(M.row_ptr, M.col, M.val.float(), A.n_cols)
    M32.set_kernel("vector", compensated=True)
    x32 = x.float()
    y32 = torch.empty(A.n_rows, dtype=torch.float32, device=dev)
    J32 = M32.to_jds("NUJDS", "symmetric", unroll=4)
    xp32 = J32.permute(x32)
    G32 = M32.to_jds("SELL", "row_only", window=128, unroll=4)
    G32w = M32.to_jds("SELL", "row_only", window=1024, unroll=4)
    res = {}
    opts = [("CRS vector l4 r4", M32, x32, lambda: M32.set_kernel("vector", lanes=4, rows_per_warp=4)),
            ("CRS tiled 1024", M32, x32, lambda: M32.prepare_tiled(1024)),
            ("NUJDS symmetric u=4", J32, xp32, lambda: None),
            ("SELL row_only w=128 u=4", G32, x32, lambda: None),
            ("SELL row_only w=1024 u=4", G32w, x32, lambda: None)]
    best = None
    for name, H, xin, conf in opts:
        conf()
        t = statistics.median(time_launches(lambda: H.spmv(xin, out=y32), 10))
        res[name] = {"gflops": round(2.0 * A.nnz / (t * 1e-3) / 1e9, 1), "ms": round(t, 4),
                     "gbs": round((8 * A.nnz + 4 * (A.n_rows + 1) + 4 * (A.n_rows + A.n_cols))
                                  / (t * 1e-3) / 1e9, 1)}
        if best is None or t < best[0]:
            best = (t, name)
    # accuracy against the FP64 product on the GPU (itself within 1e-14 of the oracle)
    M.set_kernel("vector", lanes=4, rows_per_warp=4)
    ref = M.spmv(x)
    Mabs = CRSMatrix(M.row_ptr, M.col, M.val.abs(), A.n_cols)
    sabs = Mabs.spmv(x.abs())
    M32.set_kernel("vector", lanes=4, rows_per_warp=4, compensated=True)
    yc = M32.spmv(x32).double()
    M32.set_kernel("vector", lanes=4, rows_per_warp=4, compensated=False)
    yp = M32.spmv(x32).double()
    den = sabs.clamp_min(1e-300)
    return {"best": best[1], "speedup_vs_fp64": round(ms64 / best[0], 3), "kernels": res,
            "max_err_over_sum_abs_compensated": float(((yc - ref).abs() / den).max()),
            "max_err_over_sum_abs_plain": float(((yp - ref).abs() / den).max()),
            "per_config": fp32_errors(dev),
            "note": "error of FP32 data and FP32 vector against the FP64 product of the FP64 data"}


def fp32_errors(dev):
    """Max |y32 - y64| / sum|a||x| per workload (FP32 values and vector,
    compensated and plain row sums, against the FP64 GPU product of the
    FP64 data): the Laplacian, the HH-like matrix, the Zipf rows and the
    27-point stencil."""
    import torch
    from paper_0910_4836_gb300 import CRSMatrix, synth as S
    out = {}
    for i, name in ((0, "laplace_64x64"), (1, "hh_like_6M"), (2, "zipf_rows_4M"), (4, "stencil27_100^3")):
        A = S.config(i)
        M = CRSMatrix.from_host(A, device=dev)
        x = torch.as_tensor(S.vector(A.n_cols, i)).to(dev)
        ref = M.spmv(x)
        sabs = CRSMatrix(M.row_ptr, M.col, M.val.abs(), A.n_cols).spmv(x.abs()).clamp_min(1e-300)
        M32 = CRSMatrix(M.row_ptr, M.col, M.val.float(), A.n_cols)
        row = {}
        for comp in (True, False):
            M32.set_kernel("vector", lanes=4, rows_per_warp=4, compensated=comp)
            y = M32.spmv(x.float()).double()
            row["compensated" if comp else "plain"] = float(((y - ref).abs() / sabs).max())
        out[name] = row
        del M, M32, ref, sabs
        torch.cuda.empty_cache()
    return out


def spmm_adjoint_numbers(M, A, x, dev, time_launches, peak):
    """The SpMM, adjoint and dval rows on the HH-like matrix, each against
    its own algorithmic bytes and the HBM peak: Y = A X for k = 4 and 16
    (CRS and SELL), A^T g through the transposed CRS and through a NUJDS of
    A^T, and dval_k = g[row_k] x[col_k]."""
    import torch
    N, Nc, nnz = A.n_rows, A.n_cols, A.nnz
    out = {}

    def row(t_ms, nbytes, flops):
        return {"ms": round(t_ms, 4), "gflops": round(flops / (t_ms * 1e-3) / 1e9, 1),
                "gbs": round(nbytes / (t_ms * 1e-3) / 1e9, 1),
                "frac": round(nbytes / (t_ms * 1e-3) / 1e9 / peak, 3)}

    M.set_kernel("vector", lanes=4, rows_per_warp=4)
    G = M.to_jds("SELL", "row_only", window=128, unroll=4)
    for k in (4, 16):
        X = torch.rand(Nc, k, dtype=torch.float64, device=dev)
        Y = torch.empty(N, k, dtype=torch.float64, device=dev)
        nb = 12 * nnz + 4 * (N + 1) + 8 * k * (Nc + N)
        for name, fn in (("CRS", lambda: M.spmm(X, out=Y)), ("SELL row_only w=128", lambda: G.spmm(X, out=Y))):
            t = statistics.median(time_launches(fn, 10))
            out[f"spmm k={k} {name}"] = row(t, nb, 2.0 * nnz * k)
        del X, Y
    del G
    torch.cuda.empty_cache()
    T = M.transpose()
    g = torch.rand(N, dtype=torch.float64, device=dev)
    z = torch.empty(Nc, dtype=torch.float64, device=dev)
    ab = 12 * nnz + 4 * (Nc + 1) + 8 * N + 8 * Nc
    t = statistics.median(time_launches(lambda: M.spmv(g, out=z, transpose=True), 10))
    out["adjoint A^T g, transposed CRS"] = row(t, ab, 2.0 * nnz)
    JT = T.to_jds("NUJDS", "row_only", unroll=2)
    t = statistics.median(time_launches(lambda: JT.spmv(g, out=z), 10))
    out["adjoint A^T g, NUJDS of A^T"] = row(t, 12 * nnz + 4 * (JT.n_diag + 1) + 16 * Nc, 2.0 * nnz)
    del JT
    d = torch.empty(nnz, dtype=torch.float64, device=dev)
    db = 8 * nnz + 4 * nnz + 4 * (N + 1) + 8 * N + 8 * Nc
    t = statistics.median(time_launches(lambda: M.dval(g, x, out=d), 10))
    out["dval"] = row(t, db, 1.0 * nnz)
    out["bytes"] = {"spmm": "12 nnz + 4(N+1) + 8k(N_c+N)", "adjoint": "12 nnz + 4(N_c+1) + 8N + 8N_c",
                    "dval": "8 nnz written + 4 nnz col + 4(N+1) + 8N + 8N_c"}
    return out


def symmetric_numbers(M, A, x, dev, time_launches, ms_full):
    """The product from the upper triangle only (FP64 atomic scatter of the
    transposed half) on the same matrix: its time against the full-storage
    step, and the entries it reads."""
    import torch
    U = M.upper()
    y = torch.zeros(A.n_rows, dtype=torch.float64, device=dev)
    out = {"nnz_upper": U.nnz, "nnz_full": A.nnz, "full_step_ms": ms_full}
    for name, H in (("CRS upper", U), ("SELL upper row_only w=128 u=4", U.to_jds("SELL", "row_only", window=128,
                                                                                 unroll=4))):
        t = statistics.median(time_launches(lambda: H.spmv_symmetric(x, out=y), 10))
        out[name] = {"ms": round(t, 4), "gflops": round(2.0 * A.nnz / (t * 1e-3) / 1e9, 1),
                     "speedup_vs_full": round(ms_full / t, 3)}
    return out


def hybrid_numbers(dev, time_launches, peak):
    """The DIA + remainder hybrid on the second HH stand-in (60% of the
    entries on twelve dense outer diagonals, as Sect. 3.2 describes the real
    matrix), against SELL and CRS on the same matrix."""
    import torch
    from paper_0910_4836_gb300 import CRSMatrix, HybridMatrix, synth as S
    A = S.hh_diagonals(6_000_000, 5)
    M = CRSMatrix.from_host(A, device=dev)
    x = torch.as_tensor(S.vector(A.n_cols, 5)).to(dev)
    y = torch.empty(A.n_rows, dtype=torch.float64, device=dev)
    crs_b = algorithmic_bytes(A.n_rows, A.n_cols, A.nnz)
    out = {"workload": "hh_diagonals N=6,000,000 (12 dense outer diagonals + band of 400)", "nnz": A.nnz,
           "kernels": {}}

    def rec(name, fn, nbytes):
        t = statistics.median(time_launches(fn, 10))
        out["kernels"][name] = {"ms": round(t, 4), "gflops": round(2.0 * A.nnz / (t * 1e-3) / 1e9, 1),
                                "gbs": round(nbytes / (t * 1e-3) / 1e9, 1),
                                "frac": round(nbytes / (t * 1e-3) / 1e9 / peak, 3)}

    M.set_kernel("vector", lanes=4, rows_per_warp=4)
    rec("CRS vector l4 r4", lambda: M.spmv(x, out=y), crs_b)
    G = M.to_jds("SELL", "row_only", window=128, unroll=4)
    rec("SELL row_only w=128 u=4", lambda: G.spmv(x, out=y),
        12 * A.nnz + 4 * (G.n_blocks + 1) + 20 * A.n_rows)
    del G
    for rem in ("SELL", "CRS"):
        H = HybridMatrix(M, 16, 2.0 / 3.0, remainder=rem, window=128, unroll=4)
        nd = len(H.offsets_host)
        hb = 8 * nd * A.n_rows + 12 * H.nnz_rem + 4 * (A.n_rows + 1) + 16 * A.n_rows
        rec(f"hybrid DIA({nd}) + {rem}", lambda: H.spmv(x, out=y), hb)
        out["dia_diagonals"], out["nnz_dia"] = nd, H.nnz_dia
        del H
    return out


def small_numbers(dev, time_launches):
    """The 64x64 Laplacian (N=4096, fits in L2): latency-bound, so the figures
    are microseconds per SpMVM, eager (one launch each) and as one replay of
    a CUDA graph holding 100 SpMVMs."""
    import torch
    from paper_0910_4836_gb300 import CRSMatrix, synth as S
    A = S.config(0)
    M = CRSMatrix.from_host(A, device=dev)
    x = torch.as_tensor(S.vector(A.n_cols, 0)).to(dev)
    out = {"n_rows": A.n_rows, "nnz": A.nnz}
    for name, H, xin in (("CRS vector", M, x), ("SELL row_only w=128 u=4", M.to_jds("SELL", "row_only", window=128, unroll=4), x),
                         ("NUJDS row_only u=2", M.to_jds("NUJDS", "row_only", unroll=2), x)):
        if name.startswith("CRS"):
            H.autotune()
        y = torch.empty(A.n_rows, dtype=torch.float64, device=dev)
        eager = statistics.median(time_launches(lambda: H.spmv(xin, out=y), 200))
        s = torch.cuda.Stream(dev)
        s.wait_stream(torch.cuda.current_stream(dev))
        with torch.cuda.stream(s):
            H.spmv(xin, out=y)
        torch.cuda.current_stream(dev).wait_stream(s)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(100):
                H.spmv(xin, out=y)
        replay = statistics.median(time_launches(g.replay, 20)) / 100
        out[name] = {"eager_us": round(eager * 1e3, 2), "graph_us": round(replay * 1e3, 2)}
    return out


def zipf_numbers(dev, time_launches, peak):
    """The irregular workload (N = 4e6, Zipf(2) row lengths up to 5000,
    random columns): FP64 SpMVM in the candidate schemes; JDS needs the
    deep-diagonal split, since a few rows have thousands of entries."""
    import torch
    from paper_0910_4836_gb300 import CRSMatrix, synth as S
    A = S.config(2)
    M = CRSMatrix.from_host(A, device=dev)
    x = torch.as_tensor(S.vector(A.n_cols, 2)).to(dev)
    y = torch.empty(A.n_rows, dtype=torch.float64, device=dev)
    crs_b = algorithmic_bytes(A.n_rows, A.n_cols, A.nnz)
    out = {"n_rows": A.n_rows, "nnz": A.nnz, "max_row": int(A.row_lengths().max())}
    runs = []
    M.set_kernel("vector", lanes=4, rows_per_warp=4)
    runs.append(("CRS vector l4 r4", lambda: M.spmv(x, out=y), crs_b))
    M2 = CRSMatrix(M.row_ptr, M.col, M.val, A.n_cols)
    M2.prepare_tiled(1024)
    runs.append(("CRS tiled 1024", lambda: M2.spmv(x, out=y), crs_b))
    J = M.to_jds("NUJDS", "row_only", unroll=2)
    jb = 12 * A.nnz + 4 * (J.n_diag + 1) + 16 * A.n_rows
    J.split(16, 64)
    runs.append(("NUJDS row_only u=2 split 16/64", lambda: J.spmv(x, out=y), jb))
    table, best = {}, None
    for name, fn, nbytes in runs:
        t = statistics.median(time_launches(fn, 10))
        table[name] = {"gflops": round(2.0 * A.nnz / (t * 1e-3) / 1e9, 1), "ms": round(t, 4),
                       "gbs": round(nbytes / (t * 1e-3) / 1e9, 1),
                       "frac": round(nbytes / (t * 1e-3) / 1e9 / peak, 3)}
        if best is None or t < best[0]:
            best = (t, name)
    out["kernels"] = table
    out["best"] = best[1]
    return out


def batched_speedups(dev, time_launches):
    """256 uneven matrices (half 7-point stencils, half random rows) in one
    persistent launch replayed from a CUDA graph, against the plain path:
    one CRS launch per matrix and right-hand side, no graph."""
    import torch
    from paper_0910_4836_gb300 import Batch, CRSMatrix, synth as S
    mats = S.batch_set(256, 3)
    out = {"matrices": len(mats), "rows": int(sum(m.n_rows for m in mats)),
           "nnz": int(sum(m.nnz for m in mats))}
    for dtype, kmode in ((torch.float64, "1"), (torch.float64, "16"), (torch.float64, "mixed"),
                         (torch.float32, "mixed")):
        ks = S.batch_k(len(mats), kmode)
        bt, handles, Xs, Ys = Batch.autotuned(mats, ks, dtype, device=dev, chunk=16384)
        for X in Xs:
            X.uniform_(-1, 1)
        g = bt.graph()
        t_batch = statistics.median(time_launches(g.replay, 20))
        plain = [CRSMatrix(h.row_ptr, h.col, h.val, h.n_cols) if isinstance(h, CRSMatrix)
                 else CRSMatrix.from_host(m, device=dev, dtype=dtype) for h, m in zip(handles, mats)]
        for P in plain:
            if dtype == torch.float32:
                P.set_kernel("vector", compensated=True)
        cols = [[torch.empty(m.n_cols, dtype=dtype, device=dev).uniform_(-1, 1) for _ in range(k)]
                for m, k in zip(mats, ks)]
        outs = [torch.empty(m.n_rows, dtype=dtype, device=dev) for m in mats]

        def plain_run():
            for P, cs, o in zip(plain, cols, outs):
                for c in cs:
                    P.spmv(c, out=o)

        t_plain = statistics.median(time_launches(plain_run, 5))
        flops = sum(2.0 * m.nnz * k for m, k in zip(mats, ks))
        nw, grid = bt.info()
        out[f"{'f64' if dtype == torch.float64 else 'f32'}_k{kmode}"] = {
            "batched_ms": round(t_batch, 4), "plain_ms": round(t_plain, 4),
            "speedup": round(t_plain / t_batch, 2), "batched_gflops": round(flops / (t_batch * 1e-3) / 1e9, 1),
            "launches_plain": int(sum(ks)), "work_items": nw, "ctas": grid,
            "jds_items": sum(1 for h in handles if not isinstance(h, CRSMatrix))}
        del bt, handles, Xs, Ys, plain, cols, outs, g
        torch.cuda.empty_cache()
    return out


def fwd_bwd_speedup(dev, time_launches):
    """loss = ||A^20 x||^2 on the 27-point stencil, 100^3: forward and
    backward, plain (all 20 activations stored, one dval launch per step)
    against tuned (checkpoint every 5 steps, fused multi-step dval)."""
    import torch
    from paper_0910_4836_gb300 import synth as S
    from paper_0910_4836_gb300.autograd import Pattern, power_apply
    A = S.stencil27(100, 4)
    m = 20
    res = {"n_rows": A.n_rows, "nnz": A.nnz, "m": m}
    for dtype in (torch.float64, torch.float32):
        # plain: default CRS kernels, explicit transposed CRS
        p = Pattern.from_host(A, device=dev, dtype=dtype)
        # tuned: autotuned forward and adjoint kernels (CRS or JDS, either side)
        pt = Pattern.from_host(A, device=dev, dtype=dtype, forward="auto", adjoint="auto")
        val = torch.as_tensor(A.val).to(device=dev, dtype=dtype)
        x0 = torch.as_tensor(S.vector(A.n_cols, 4)).to(device=dev, dtype=dtype)
        M = p.bind(val)
        p.adjoint_op(val)  # build the transposed structure once
        AT = p.AT
        pt.forward_op(val)
        pt.adjoint_op(val)

        def plain():
            xs = [x0]
            for _ in range(m):
                xs.append(M.spmv(xs[-1]))
            g = 2 * xs[-1]
            dval = torch.zeros(A.nnz, dtype=dtype, device=dev)
            for t in range(m, 0, -1):
                M.dval(g, xs[t - 1], out=dval, accumulate=True)
                g = AT.spmv(g)
            return dval, g

        def tuned(c=5):
            v = val.clone().requires_grad_(True)
            xx = x0.clone().requires_grad_(True)
            y = power_apply(pt, v, xx, m, checkpoint=c)
            (y * y).sum().backward()
            return v.grad, xx.grad

        for _ in range(2):
            plain(), tuned()
        tp = statistics.median(time_launches(plain, 5))
        tt = statistics.median(time_launches(tuned, 5))
        key = "f64" if dtype == torch.float64 else "f32"
        res[key] = {"plain_ms": round(tp, 3), "tuned_ms": round(tt, 3), "speedup": round(tp / tt, 3),
                    "vectors_stored_plain": m + 1, "vectors_stored_tuned": m // 5 + 5,
                    "tuned_forward": getattr(pt.F, "fmt", "CRS"), "tuned_adjoint": getattr(pt._adj, "fmt", "CRS")}
    return res


# ------------------------------------------------------------ CPU side -----

def host_copy_gbs(nbytes=1 << 30, reps=5):
    """STREAM-style copy bandwidth of the host (torch CPU copy, all its
    threads), read + write bytes per second: the CPU side's own roofline."""
    import torch
    src = torch.ones(nbytes // 8, dtype=torch.float64)
    dst = torch.empty_like(src)
    dst.copy_(src)
    best = None
    for _ in range(reps):
        t0 = time.perf_counter()
        dst.copy_(src)
        el = time.perf_counter() - t0
        best = el if best is None else min(best, el)
    return round(2 * nbytes / best / 1e9, 1)


def cpu_baseline(A, x, seconds):
    """The oracle on the host cores: its OpenMP static-schedule CRS loop (the
    paper's best parallel setting) on the full matrix, repeated for about
    `seconds`; the serial literal CRS and JDS loops on one core, once each;
    and the host copy bandwidth."""
    import oracle as O
    y = np.zeros(A.n_rows)
    O.crs_spmv_omp(A, x, y)  # first touch
    times = []
    t_all = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        O.crs_spmv_omp(A, x, y)
        times.append(time.perf_counter() - t0)
        el = time.perf_counter() - t_all
        if (el >= seconds and len(times) >= 5) or len(times) >= 200:
            break
    per = statistics.median(times)
    out = {"value": round(2.0 * A.nnz / per / 1e9, 3), "unit": "GFlop/s",
           "cores": O.num_threads(), "kind": "oracle",
           "cores_in_affinity_mask": AFFINITY_CORES,
           "omp": {k: os.environ.get(k) for k in ("OMP_PROC_BIND", "OMP_PLACES")},
           "sample": f"full matrix, median of {len(times)} SpMVMs with the OpenMP static CRS loop ({el:.1f} s)"}
    t0 = time.perf_counter()
    O.crs_spmv(A, x)
    out["serial_crs_gflops"] = round(2.0 * A.nnz / (time.perf_counter() - t0) / 1e9, 3)
    J = O.jds_build(A, symmetric=True)
    xp = O.permute(J.perm, x)
    t0 = time.perf_counter()
    O.jds_spmv(J, xp)
    out["serial_jds_gflops"] = round(2.0 * A.nnz / (time.perf_counter() - t0) / 1e9, 3)
    out["serial_cores"] = 1
    out["host_copy_gbs"] = host_copy_gbs()
    return out


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return None
    A, x = make_workload(args.config)
    import oracle as O
    y = np.zeros(A.n_rows)
    O.crs_spmv_omp(A, x, y)
    for _ in range(max(args.warmup, 3)):
        O.crs_spmv_omp(A, x, y)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        O.crs_spmv_omp(A, x, y)
    el = time.perf_counter() - t0
    per = el / args.steps
    val = round(2.0 * A.nnz / per / 1e9, 3)
    return {"metric": METRIC, "value": val, "unit": "GFlop/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": round(per * 1e3, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOADS.get(args.config, WORKLOAD), "config_index": args.config, "n_rows": A.n_rows,
                       "nnz": A.nnz, "kernel": "oracle CRS loop, OpenMP static schedule"},
            "cpu_baseline": {"value": val, "unit": "GFlop/s", "cores": O.num_threads(),
                             "kind": "oracle", "sample": f"full matrix, {args.steps} timed SpMVMs"},
            "e2e": {"value": val, "unit": "GFlop/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_micro(args):
    """The basic sparse vector operations of Sect. 3.1 on the device: the
    table of ADD / SCP over packed dense (PD), constant stride (CS) and
    indirect (IS: ind(i) = k i; IR: random strides of mean k, as the paper
    draws them) access at the paper's strides 1, 8 and 530; the IS / IR
    stride sweep; and IR with Gaussian strides over a mean/variance plane.
    Each point: median of 7 launches, L2 flushed (a 512 MB write) before
    each, CUDA events around the launch only."""
    import torch
    from paper_0910_4836_gb300 import build, synth as S
    from paper_0910_4836_gb300.gather import GatherSum
    build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(64 * 2 ** 20, dtype=torch.float64, device=dev)
    i32max = 2 ** 31 - 1
    gen = torch.Generator(device=dev)
    gen.manual_seed(11)
    B = torch.rand(i32max + 1, dtype=torch.float64, device=dev, generator=gen)
    A = torch.rand(2 ** 26, dtype=torch.float64, device=dev, generator=gen)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(g):
        t = []
        for _ in range(7):
            flush.fill_(1.0)
            e0.record(stream)
            g()
            e1.record(stream)
            e1.synchronize()
            t.append(e0.elapsed_time(e1))
        return statistics.median(t)

    def point(op, access, n, k=1, ind=None):
        ind_d = None if ind is None else torch.as_tensor(ind).to(dev)
        g = GatherSum(op, access, n, B, a=A[:n] if op == "SCP" else None, k=k, ind=ind_d)
        ms = timed(g)
        useful = n * (8 + (8 if op == "SCP" else 0) + (4 if access == "IND" else 0))
        res = {"n": n, "us": round(ms * 1e3, 2), "gups": round(n / (ms * 1e-3) / 1e9, 2),
               "useful_gbs": round(useful / (ms * 1e-3) / 1e9, 1)}
        return res

    def n_for(k, cap=2 ** 26):
        return int(min(cap, 0.9 * i32max / k))

    table = {}
    for op in ("ADD", "SCP"):
        table[f"PD{op}"] = point(op, "PD", 2 ** 26)
        for k in (8, 530):
            n = n_for(k)
            table[f"CS{op} k={k}"] = point(op, "CS", n, k=k)
            table[f"IS{op} k={k}"] = point(op, "IND", n, ind=S.stride_indices(n, k))
        for k in (1, 8, 530):
            n = n_for(k)
            table[f"IR{op} k={k}"] = point(op, "IND", n, ind=S.geometric_indices(n, 1.0 / k, 100 + k))
    sweep = {}
    for k in (1, 2, 3, 4, 6, 8, 12, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512, 530, 1024):
        n = n_for(k, 2 ** 25)
        sweep[str(k)] = {"ISSCP": point("SCP", "IND", n, ind=S.stride_indices(n, k)),
                         "IRSCP": point("SCP", "IND", n, ind=S.geometric_indices(n, 1.0 / k, 200 + k))}
    plane = {}
    n = 2 ** 23
    for mean in (1, 4, 16, 64, 256):
        length = min(n * mean, i32max)
        for var in (0, 1, 16, 256, 4096, 65536):
            ind = S.gaussian_indices(n, float(mean), float(var), length, 300 + mean)
            plane[f"mean={mean} var={var}"] = point("SCP", "IND", n, ind=ind)
    return {"metric": "basic gather operations (Sect. 3.1): G element updates/s", "unit": "G updates/s",
            "dtype": "f64", "data": "synthetic (torch.rand values; SplitMix64 index arrays)",
            "l2": "flushed before every launch", "table": table, "stride_sweep": sweep,
            "gaussian_plane": plane}


def run_analysis(args):
    """Sect. 4's analysis of the storage schemes on the bench workload: the
    stride distribution of the x accesses in storage order (Fig. 4a: CRS,
    JDS, RBJDS with block 1 and 1024, SOJDS 1024, plus SELL-32-sigma), the
    sectors per warp-wide gather of the GPU kernels, and the block-size
    sweep of NBJDS / RBJDS / SOJDS (Fig. 5) with the GPU's own knobs (CRS
    lanes x rows per warp, NUJDS unroll x rows, SELL window x unroll)."""
    import torch
    from paper_0910_4836_gb300 import CRSMatrix, build
    from paper_0910_4836_gb300.analysis import mean_sectors, stride_hist, summary, warp_sectors
    build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    time_launches = _timer(dev)
    A, x_host = make_workload(args.config)
    M = CRSMatrix.from_host(A, device=dev)
    x = torch.as_tensor(x_host).to(dev)
    y = torch.empty(A.n_rows, dtype=torch.float64, device=dev)
    out = {"workload": WORKLOAD, "n_rows": A.n_rows, "nnz": A.nnz, "stride_dist": {}, "warp_sectors": {},
           "sweep": {}}

    def strides(name, col):
        f, b = stride_hist(col)
        out["stride_dist"][name] = {"forward": f.tolist(), "backward": b.tolist(), **summary(f, b)}

    def sectors(name, H, lanes=32):
        h = warp_sectors(H, lanes)
        out["warp_sectors"][name] = {"mean": round(mean_sectors(h), 3), "hist": h.tolist()}

    def timed(name, H, xin, configure_fn=None):
        if configure_fn:
            configure_fn()
        t = statistics.median(time_launches(lambda: H.spmv(xin, out=y), 10))
        out["sweep"][name] = {"us": round(t * 1e3, 1), "gflops": round(2.0 * A.nnz / (t * 1e-3) / 1e9, 1)}

    # throughput against the number of CTAs in use (the GPU counterpart of
    # the paper's performance against threads per socket, Sect. 5)
    out["cta_scaling"] = {}
    alg = 12 * A.nnz + 20 * A.n_rows

    def scaling(name, H, xin, limits):
        row = {}
        for lim in limits:
            H.set_grid_limit(lim)
            t = statistics.median(time_launches(lambda: H.spmv(xin, out=y), 10))
            row[str(lim or "all")] = {"us": round(t * 1e3, 1), "gbs": round(alg / (t * 1e-3) / 1e9, 1)}
        H.set_grid_limit(0)
        out["cta_scaling"][name] = row

    G = M.to_jds("SELL", "row_only", window=128, unroll=4)
    scaling("SELL w=128 u=4 (1024-thread CTAs, at most 2 per SM)", G, x,
            (8, 16, 32, 48, 64, 76, 96, 128, 152, 228, 304, 0))
    del G
    J = M.to_jds("NUJDS", "row_only", unroll=2)
    scaling("NUJDS u=2 (256-thread CTAs)", J, x, (38, 76, 152, 304, 608, 1216, 2432, 0))
    del J
    M.set_kernel("vector", lanes=4, rows_per_warp=4)
    scaling("CRS vector l4 r4 (256-thread CTAs)", M, x, (38, 76, 152, 304, 608, 1216, 2432, 0))
    torch.cuda.empty_cache()

    strides("CRS", M.col)
    for l, r in ((1, 1), (2, 2), (4, 4), (8, 2), (16, 2), (32, 1)):
        if r == 1 or l in (2, 4):
            sectors(f"CRS lanes={l}", M, l)
        timed(f"CRS vector l{l} r{r}", M, x, lambda l=l, r=r: M.set_kernel("vector", lanes=l, rows_per_warp=r))
    for perm in ("symmetric", "row_only"):
        J = M.to_jds("JDS", perm)
        xp = J.permute(x) if perm == "symmetric" else x
        strides(f"JDS {perm}", J.col)
        sectors(f"JDS {perm}", J)
        for u, r in ((1, 1), (2, 1), (4, 1), (8, 1), (2, 2), (4, 2), (2, 4)):
            timed(f"NUJDS {perm} u={u} r={r}", J, xp,
                  lambda u=u, r=r: (J.set_format("NUJDS" if u > 1 else "JDS", unroll=u),
                                    J.set_kernel("vector", rows_per_warp=r)))
        for b in (64, 128, 256, 512, 1024, 2048, 4096):
            timed(f"NBJDS {perm} b={b}", J, xp, lambda b=b: (J.set_format("NBJDS", block=b),
                                                            J.set_kernel("vector", rows_per_warp=1)))
        del J
        torch.cuda.empty_cache()
        for fmt in ("RBJDS", "SOJDS"):
            for b in ((1, 1024) if perm == "symmetric" else ()):
                R = M.to_jds(fmt, perm, block=b)
                strides(f"{fmt} {perm} b={b}", R.col)
                del R
            for b in (64, 256, 1024, 4096):
                R = M.to_jds(fmt, perm, block=b)
                timed(f"{fmt} {perm} b={b}", R, xp)
                del R
            torch.cuda.empty_cache()
        for w in (32, 128, 1024, 8192):
            G = M.to_jds("SELL", perm, window=w)
            strides(f"SELL {perm} w={w}", G.col)
            sectors(f"SELL {perm} w={w}", G)
            xs = G.permute(x) if perm == "symmetric" else x
            for u in (1, 2, 4):
                timed(f"SELL {perm} w={w} u={u}", G, xs, lambda u=u, G=G: G.set_format("SELL", unroll=u))
            del G
            torch.cuda.empty_cache()
    return out


def run_ncu_case(args):
    """A few launches of one kernel on a 2e6-row HH-like matrix (~350 MB,
    above the 129 MB L2) for an ncu capture; prints nothing to time.  With
    --config 2: the Zipf-rows matrix (345 MB) and its NUJDS walk split at
    depth 16 in chunks of 64."""
    import torch
    from paper_0910_4836_gb300 import CRSMatrix, build, synth as S
    build()
    if args.config == 2:
        A = S.config(2)
        M = CRSMatrix.from_host(A)
        x = torch.as_tensor(S.vector(A.n_cols, 2)).cuda()
        y = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
        J = M.to_jds("NUJDS", "row_only", unroll=2)
        J.split(16, 64)
        for _ in range(3):
            J.spmv(x, out=y)
        torch.cuda.synchronize()
        print("ran NUJDS row_only u=2 split 16/64 on the Zipf rows")
        return
    A = S.hh_like(2_000_000, 1)
    M = CRSMatrix.from_host(A)
    x = torch.as_tensor(S.vector(A.n_cols, 1)).cuda()
    y = torch.empty(A.n_rows, dtype=torch.float64, device="cuda")
    only = None if args.kernel == "auto" else args.kernel
    for name, H, xin, _, how in candidates(M, A, x, only):
        if only is not None and name != only:
            continue
        configure(H, how)
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        for _ in range(3):
            H.spmv(xin, out=y)
        torch.cuda.synchronize()
        print("ran", name)


def main():
    args = parse()
    if args.ncu_case:
        run_ncu_case(args)
        return
    if args.micro:
        print(json.dumps(run_micro(args)), flush=True)
        return
    if args.analysis:
        print(json.dumps(run_analysis(args)), flush=True)
        return
    res = run_reference(args) if args.impl == "reference" else run_ours(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
