"""Benchmark: exp(-iHt)v solves/s on the XXZ chain with Dzyaloshinskii-Moriya phases.

Workload: L = 22 periodic XXZ-DM chain (d = 4,194,304, nnz = 50,331,648,
complex128 CSR), Neel initial state, t = 50, Krylov dimension m = 40,
err_max = 1e-8.  One step = one complete solve (every restart of Algorithm 1:
Lanczos with the fused SpMV, eigen-decomposition, error-integral step search,
recombination).  Inputs (H: 1.0 GB, the Krylov basis: 2.8 GB) are far larger
than the 129 MB L2, so no flush is needed between steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
N > 1 runs under torch.distributed.run: one independent solve stream per GPU
(replicas; the method has no exchange step), time = max over ranks.
"""
from __future__ import annotations

import os

# the oracle's BLAS-1 calls stay on one thread (the paper's setting, Sec. 5)
os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
os.environ.setdefault("OMP_NUM_THREADS", "1")
os.environ.setdefault("MKL_NUM_THREADS", "1")

import argparse
import hashlib
import json
import re
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "exp(-iHt)v solves/s and p50/p99 latency at bound 1e-8; SpMV HBM GB/s vs peak"
WORKLOAD = "xxzdm_L22"
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "k_spmv_sellv_xxzdm_L22.md")
# committed ncu summaries of the dominant kernel (K1) per single-solve workload
K1_SUMMARIES = {"xxzdm_L22": PROFILE_SUMMARY,
                "memory_K10": os.path.join(ROOT, "profiles", "k_spmv_sellr_memory_K10.md"),
                "random_L20": os.path.join(ROOT, "profiles", "k_spmv_sell_random_L20.md")}
K1_SOURCES = [os.path.join(ROOT, "paper_2205_15346_gb300", "csrc", f)
              for f in ("te_sell.cu", "te_slices.cuh")]
# FP64 issue rate of GB300: 2 DFMA lanes per SM per cycle (ncu reports a sustained
# peak of 304 DFMA thread-instructions per cycle over the 152 SMs)
SMS = 152
DFMA_LANES_PER_SM = 2


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float) -> float:
    """Largest value of x over the ranks of the default process group (x itself
    without one).  Used for the timed region: the slowest replica sets the time."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(steps: int, world: int, elapsed_s: float) -> float:
    """Whole-job solves/s: every rank runs `steps` independent solves."""
    return steps * world / elapsed_s


def attainable_fp64(ctx, achieved_tf):
    """The FP64 FMA rate this GPU sustains on independent chains (te_measure_fp64),
    and the kernel's fraction of it, beside the derived pipe peak."""
    from paper_2205_15346_gb300 import te
    rate = te.te_measure_fp64(ctx)
    mma = te.te_measure_fp64_mma(ctx)
    return {"tflops": rate, "frac": achieved_tf / rate,
            "how": "te_measure_fp64: independent DFMA chains, no memory traffic, after the timed region",
            "fp64_mma_tflops": mma,
            "fp64_mma_how": "te_measure_fp64_mma: mma.sync m8n8k4 .f64 on independent tiles, after the timed region"}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def k1_source_hash(sources=None) -> str:
    """First 16 hex digits of the SHA-256 of a kernel's sources (default: K1's,
    te_sell.cu + te_slices.cuh)."""
    h = hashlib.sha256()
    for f in sources or K1_SOURCES:
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _csrc(*names):
    return [os.path.join(ROOT, "paper_2205_15346_gb300", "csrc", n) for n in names]


def recorded_traffic(summary=PROFILE_SUMMARY, sources=None):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the
    current kernel source (else None)."""
    if not os.path.exists(summary):
        return None
    txt = open(summary).read()
    h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    b = re.search(r"dram_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    if not h or not b or h.group(1) != k1_source_hash(sources):
        return None
    return float(b.group(1))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- oracle (CPU) timing

_ORACLE_H = {}


def oracle_matrix(wl):
    """The oracle's H (the array-form builders for the bosons and the paper's system,
    bitwise equal to the row-by-row ones)."""
    from oracle import models
    if wl["name"] not in _ORACLE_H:
        p = wl["params"]
        if p["model"] == "coo":
            A = models.coo_to_csr(wl["d"], *W.random_hermitian_coo(p["L"], p["seed"]))
        elif p["model"] == "bose":
            A = models.bose_csr_vec(p)
        elif p["model"] == "memory":
            A = models.memory_csr_vec(p)
        else:
            A = models.build(p)
        _ORACLE_H[wl["name"]] = A.to_scipy()
    return _ORACLE_H[wl["name"]]


def single_view(wl):
    """The one-vector workload behind a batched one (its first vector), or the
    K = K' = 10 size of the runtime study."""
    if "sizes" in wl:
        q = wl["sizes"][3]
        return {"name": "memory_K10", "params": q["params"], "d": q["d"], "v0": q["v0"],
                "t": wl["t"], "m": wl["m"], "tol": wl["tol"]}
    if "nvec" not in wl:
        return wl
    v = dict(wl)
    v["v0"] = ("random", wl["v0_seeds"][0])
    return v


def oracle_sample(wl, max_restarts: int = 1, threads=None):
    """Time the oracle on a bounded sample: its first `max_restarts` restarts of
    the workload's solve (matrix assembly excluded).  threads None: scipy's
    product on one thread (the oracle as it stands, the paper's setting); a
    count: the oracle's C product on that many threads.  Returns (solves/s
    estimate, wall seconds, time covered, result)."""
    from oracle import krylov
    A = oracle_matrix(wl)
    v0 = W.initial_vector(wl["v0"], wl["d"])
    t0 = time.perf_counter()
    res = krylov.evolve(A, v0, wl["t"], wl["tol"], wl["m"], max_restarts=max_restarts, threads=threads)
    wall = time.perf_counter() - t0
    covered = abs(res.t_reached)
    return (covered / wl["t"]) / wall, wall, covered, res


def sm_mhz_now(gpu: int) -> float:
    """Current SM clock (MHz) from nvidia-smi; the maximum, 2070, if unavailable."""
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(gpu), "--query-gpu=clocks.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True,
                             timeout=10).stdout
        return float(out.strip().splitlines()[0])
    except (OSError, subprocess.SubprocessError, ValueError, IndexError):
        return 2070.0


def host_cpu():
    """Core count and CPU model of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            for ln in open("/proc/cpuinfo"):
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": os.uname().machine}


def cpu_baseline_entry(wl, restarts: int = 5):
    """The oracle's first `restarts` restarts on one thread and on all host cores;
    solves/s = (fraction of t covered) / wall time (a per-restart rate)."""
    from oracle import native
    info = host_cpu()
    n = info["nproc"] or 1
    r1, w1, c1, res1 = oracle_sample(wl, restarts)
    entry = {"unit": "solves/s", "kind": "oracle", "cpu_model": info["cpu_model"],
             "nproc": n, "machine": info["machine"],
             "one_thread": {"value": r1, "cores": 1, "wall_s": w1, "restarts": res1.restarts,
                            "t_covered": c1}}
    if native.available():
        rn, wn, cn, resn = oracle_sample(wl, restarts, threads=n)
        entry.update({"value": rn, "cores": n, "threads": n,
                      "all_cores": {"value": rn, "cores": n, "wall_s": wn, "restarts": resn.restarts,
                                    "t_covered": cn}})
    else:
        entry.update({"value": r1, "cores": 1, "threads": 1})
    entry["sample"] = (f"per-restart rate: the oracle's first {res1.restarts} restarts of the "
                       f"{wl['name']} solve ({res1.matvecs} matvecs, t advanced {c1:.4g} of {wl['t']}), "
                       f"on 1 thread (numpy/scipy, {w1:.1f} s) and on all {n} cores (the oracle's "
                       f"C product on {n} threads, vector work numpy on one); "
                       f"solves/s = (fraction of t covered) / wall time")
    return entry


def oracle_multi_sample(wl):
    """The oracle's first restart of every problem of a grouped workload; the
    group's time is estimated as the sum over problems of wall / fraction of t."""
    from oracle import krylov, models
    est, wall_total, matvecs = 0.0, 0.0, 0
    for q in wl["problems"]:
        A = models.build(q["params"]).to_scipy()
        v0 = W.random_state(q["v0_seed"], q["d"])
        t0 = time.perf_counter()
        res = krylov.evolve(A, v0, q["t"], wl["tol"], wl["m"], max_restarts=1)
        wall = time.perf_counter() - t0
        wall_total += wall
        matvecs += res.matvecs
        est += wall / (abs(res.t_reached) / q["t"])
    return len(wl["problems"]) / est, wall_total, matvecs


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    if "problems" in W.workload(args.workload):
        return run_reference_multi(args)
    wl = single_view(W.workload(args.workload))
    from oracle import native
    info = host_cpu()
    threads = info["nproc"] if native.available() else None
    rates, walls = [], []
    for i in range(args.warmup + args.steps):
        rate, wall, covered, res = oracle_sample(wl, 1, threads=threads)
        if i >= args.warmup:
            rates.append(rate)
            walls.append(wall)
    value = float(np.mean(rates))
    cores = threads or 1
    line = {
        "metric": METRIC, "impl": "reference", "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * float(np.mean(walls)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "complex128", "data": "synthetic",
        "config": config_block(wl, args),
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                         "cpu_model": info["cpu_model"], "nproc": info["nproc"],
                         "sample": (f"each step: the oracle's first restart of the workload solve "
                                    f"(its C product on {cores} threads); solves/s = fraction of t "
                                    f"covered / wall time")},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference_multi(args):
    wl = W.workload(args.workload)
    rates, walls = [], []
    for i in range(args.warmup + args.steps):
        rate, wall, mv = oracle_multi_sample(wl)
        if i >= args.warmup:
            rates.append(rate)
            walls.append(wall)
    value = float(np.mean(rates))
    sample = ("each step: the oracle's first restart of each of the 32 problems (1 thread); "
              "solves/s = 32 / sum over problems of (wall / fraction of t covered)")
    line = {
        "metric": METRIC, "impl": "reference", "value": value, "unit": "solves/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * float(np.mean(walls)), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "complex128", "data": "synthetic",
        "config": config_block(wl, args),
        "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


DESCRIBE = {
    "random_L20": ("general complex Hermitian matrix from COO (random value per coupled pair, "
                   "spin-chain pattern) d=1048576, nnz=11534336, full-value sliced copy, random v0"),
    "xxzdm_L22": "XXZ-DM chain L=22 periodic, d=4194304, nnz=50331648, Neel v0",
    "xxzdm_L20": "XXZ-DM chain L=20 periodic, d=1048576, nnz=11534336, random v0",
    "tfim_L12": "TFIM chain L=12 open, d=4096, nnz=53248, random v0",
    "bose_K14_N10": ("bosons K=14 modes N=10 (hash-indexed basis), d=1144066, nnz=91674506, "
                     "rows 14..131, v0 = |1^10 0^4>"),
    "memory_K10": ("the paper's example system (Sec. 5) at its benchmark size: K=K'=10, Nm=5, "
                   "N0=Nc=100, d=1565904, v0 = |N0,0,1^5,0^15>"),
    "batch_xxzdm_L20_x64": ("64 random normalised initial vectors (seeds 301..364) under one "
                            "XXZ-DM chain L=20 periodic, d=1048576, nnz=11534336"),
    "memory_K10_sampled": ("the paper's example system at its benchmark size (d=1565904) with "
                           "all 22 mode occupations sampled at 100 times (Sec. 2.4, Sec. 5)"),
    "memory_scaling": ("the paper's runtime-vs-dimension study (Sec. 5): its example system at "
                       "K=K'=4,6,8,10 (Nm=K/2, N0=Nc=100) and K=K'=10, N0=Nc=139, t=10"),
    "tfim_multi_x32": ("32 independent open TFIM chains, L uniform on 10..20 (total d=9182208), "
                       "t ~ U[1,20], random v0"),
}
# The paper's single-thread CPU wall time for memory_K10 (353 s, i9-9900K, Sec. 5):
# the only workload here with a published number for the same metric.
PAPER_SOLVES_PER_S = {"memory_K10": 1.0 / 353.0}


def config_block(wl, args):
    if "problems" in wl:
        return {"workload": f"{wl['name']}: {DESCRIBE[wl['name']]}, m={wl['m']}, tol={wl['tol']}",
                "global_batch": len(wl["problems"]) * args.gpus, "parallelism": f"replicas{args.gpus}",
                "l2": "inputs larger than L2 (Krylov blocks 4.6 GB); no flush"}
    if "nvec" in wl:
        return {"workload": f"{wl['name']}: {DESCRIBE[wl['name']]}, "
                            f"t={wl['t']}, m={wl['m']}, tol={wl['tol']}",
                "global_batch": wl["nvec"] * args.gpus, "parallelism": f"replicas{args.gpus}",
                "l2": "inputs larger than L2 (vector block 1.07 GB, Krylov blocks 44 GB); no flush"}
    return {"workload": f"{wl['name']}: {DESCRIBE[wl['name']]}, "
                        f"t={wl['t']}, m={wl['m']}, tol={wl['tol']}",
            "global_batch": args.gpus, "parallelism": f"replicas{args.gpus}",
            "l2": "inputs larger than L2 (H 1.0 GB, Krylov basis 2.8 GB); no flush"}


# ---------------------------------------------------------------- GPU arm

# The other configurations, each run in a child process of its own after the headline
# workload (a failure there is recorded, not raised): configs 1, 3a, 3b and 4 with a few
# timed steps, the general complex CSR, and a short request stream at 0.8 x capacity.
OTHER_CONFIGS = [
    ("tfim_L12", ["--steps", "20", "--warmup", "3"]),
    ("bose_K14_N10", ["--steps", "3", "--warmup", "3"]),
    ("batch_xxzdm_L20_x64", ["--steps", "3", "--warmup", "3"]),
    ("tfim_multi_x32", ["--steps", "5", "--warmup", "3"]),
    ("random_L20", ["--steps", "5", "--warmup", "3"]),
    ("serve_mix", ["--requests", "80", "--loads", "0.8"]),
]


def other_configs():
    out = {}
    for name, extra in OTHER_CONFIGS:
        cmd = [sys.executable, os.path.abspath(__file__), "--workload", name, "--no-cpu-baseline", *extra]
        t0 = time.perf_counter()
        try:
            res = subprocess.run(cmd, capture_output=True, text=True, timeout=600)
            lines = [ln for ln in res.stdout.splitlines() if ln.startswith("{")]
            if res.returncode != 0 or not lines:
                out[name] = {"error": f"exit {res.returncode}: {res.stderr.strip()[-300:]}"}
                continue
            d = json.loads(lines[-1])
        except (subprocess.SubprocessError, OSError, ValueError) as e:
            out[name] = {"error": str(e)[:300]}
            continue
        keep = {k: d[k] for k in ("value", "unit", "ms_per_step", "steps", "latency_ms", "e2e",
                                  "one_at_a_time", "runs", "max_diff_over_tol_vs_alone",
                                  "mode", "clocks") if k in d}
        if "roofline" in d:
            r = d["roofline"]
            keep["roofline"] = {k: r.get(k) for k in ("bound", "kernel", "achieved", "peak", "unit",
                                                        "frac", "traffic", "avg_launch_ms")}
            if isinstance(r.get("hbm"), dict):
                keep["roofline"]["hbm_frac"] = r["hbm"].get("frac")
        keep["config"] = d.get("config", {}).get("workload")
        keep["wall_s"] = time.perf_counter() - t0
        out[name] = keep
    return out


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2205_15346_gb300 import te

    wl = W.workload(args.workload)
    p, d, t, tol, m = wl["params"], wl["d"], wl["t"], wl["tol"], wl["m"]
    ctx = te.te_create(local)
    if p["model"] == "coo":                   # a general matrix handed over as COO triplets
        rows, cols, vals = W.random_hermitian_coo(p["L"], p["seed"])
        H = te.te_build_csr(ctx, d, rows, cols, vals)
        del rows, cols, vals
    else:
        H = te.te_build_model(ctx, p)
    te.te_matrix_tune(ctx, H)                 # SpMV work-item size, timed on this GPU
    info = te.te_matrix_info_get(H)
    v0 = W.initial_vector(wl["v0"], d, index_of=lambda occ: te.te_model_basis_index(p, occ))
    vin = torch.from_numpy(v0).cuda()
    vout = torch.empty_like(vin)
    opt = te.make_options(profile=True)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        te.te_evolve(ctx, H, vin, t, tol, m, opt, v_out=vout)
    barrier()
    lat, stats = [], []
    with ClockSampler(local) as clk:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            e_a = torch.cuda.Event(enable_timing=True)
            e_b = torch.cuda.Event(enable_timing=True)
            e_a.record(stream)
            _, st, _ = te.te_evolve(ctx, H, vin, t, tol, m, opt, v_out=vout)
            e_b.record(stream)
            e_b.synchronize()
            lat.append(e_a.elapsed_time(e_b))
            stats.append(st)
        ev1.record(stream)
        barrier()
    elapsed = max_over_ranks(ev0.elapsed_time(ev1) / 1000.0)
    value = job_throughput(args.steps, world, elapsed)

    # end to end through the C ABI with pinned host buffers (copies inside the timed region)
    hin = torch.from_numpy(v0).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    opt_e2e = te.make_options()
    te.te_evolve(ctx, H, hin.numpy(), t, tol, m, opt_e2e, v_out=hout.numpy())
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        te.te_evolve(ctx, H, hin.numpy(), t, tol, m, opt_e2e, v_out=hout.numpy())
    barrier()
    e2e_elapsed = max_over_ranks(time.perf_counter() - t0)
    e2e_value = job_throughput(args.steps, world, e2e_elapsed)

    # roofline of the dominant kernel (K1, fused SpMV + alpha partials), live CUDA-event times.
    # K1 is bound by the FP64 pipe.  It executes 3 DFMA (6 FLOP) per stored complex
    # entry (the three-multiplication complex product) plus 12 FLOP per row (combine,
    # scale, three-term subtraction, alpha partial); the plain complex product would
    # take 8 FLOP per entry.  Bytes: a, (b-a, a+b) and the column per entry; x, x+y,
    # u_{j-1} read and y written per row; slice offsets.  HBM is reported beside it.
    nnz = info["nnz"]
    nslices = (d + 31) // 32
    if info["sell_dict"] > 0 and info["sell_real"]:
        # real value table: 2 DFMA (4 FLOP) per off-diagonal entry, no x+y gather and
        # no combination of three sums per row
        off = nnz - d
        k1_bytes = 6 * off + 8 * d + 4 * (nslices + 1) + 48 * d + 8 * info["sell_dict"]
        k1_flops = 4 * off + 14 * d
        k1_flops_complex = 8 * off + 16 * d
    elif info["sell_dict"] > 0:
        # value-indexed copy: column + 16-bit table index per off-diagonal entry, the
        # real diagonal per row (the model builders store every diagonal entry, so
        # there are nnz - d off-diagonal entries); diagonal term 2 DFMA per row
        off = nnz - d
        k1_bytes = 6 * off + 8 * d + 4 * (nslices + 1) + 56 * d + 24 * info["sell_dict"]
        k1_flops = 6 * off + 16 * d
        k1_flops_complex = 8 * off + 16 * d
    else:
        k1_bytes = 28 * nnz + 4 * (nslices + 1) + 56 * d
        k1_flops = 6 * nnz + 12 * d
        k1_flops_complex = 8 * nnz + 12 * d
    spmv_ms = sum(s["spmv_ms"] for s in stats)
    spmv_n = sum(s["spmv_launches"] for s in stats)
    fused = stats[0]["fused_restarts"] > 0
    if fused:
        # small d: the m Lanczos steps of a restart run as one cooperative kernel, timed
        # whole (every restart); one launch carries matvecs/restarts steps of K1 + K2
        # (K2: 10 FLOP per row; the fused loop keeps y in registers and writes w, x+y)
        steps = sum(s["matvecs"] for s in stats) / sum(s["restarts"] for s in stats)
        k1_flops = steps * (k1_flops + 10 * d)
        k1_flops_complex = steps * (k1_flops_complex + 10 * d)
        k1_bytes = steps * (k1_bytes - 16 * d + 24 * d)
    k1_avg_s = spmv_ms / spmv_n / 1000.0
    peaks, kind = measured_peaks()
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp64_peak = SMS * DFMA_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12      # TFLOP/s
    achieved_tf = k1_flops / k1_avg_s / 1e12
    fp64_att = attainable_fp64(ctx, achieved_tf)
    achieved = k1_bytes / k1_avg_s / 1e9
    restarts = [s["restarts"] for s in stats]
    if fused:   # per restart: memset + fused loop, step kernel, recombination, state copy
        launches = sum(3 + s["restarts"] * 3 for s in stats)
    else:
        launches = sum(3 + s["restarts"] * (2 * m + 2) for s in stats)
    if fused:
        k1_name = "k_lanczos_fused (K1 + K2 of all Lanczos steps of a restart, one cooperative kernel)"
        k1_timing = "CUDA events around the fused Lanczos kernel of every restart inside the timed solves"
    else:
        k1_name = (("k_spmv_sellr" if info["sell_dict"] > 0 and info["sell_real"]
                    else ("k_spmv_sellv_pair" if info.get("sell_async") == 1
                          else f"k_spmv_sellv_async<{info['sell_async']}>" if info.get("sell_async")
                          else "k_spmv_sellv") if info["sell_dict"] > 0 else "k_spmv_sell") +
                   " (K1: y = s H u_j - b u_{j-1}, Re<u_j,y> partials)")
        k1_timing = ("CUDA events around the Lanczos step m/2 product of every "
                     "restart inside the timed solves")

    # HBM fraction on the algorithmic bytes of one Lanczos step of the plain CSR method
    # (complex128 value + int32 column per entry, the row pointer, v_j and v_{j-1} read,
    # v_{j+1} written: 20 nnz + 4 (d + 1) + 48 d), over the K1 launch and over the whole
    # solve time per Lanczos step (K1, K2, and the step's share of K3 and K4)
    b_step = 20 * nnz + 4 * (d + 1) + 48 * d
    step_s = (elapsed / args.steps) / max(1, stats[0]["matvecs"])
    csr_step = {"bytes_per_step": b_step, "unit": "GB/s", "peak": peaks["hbm_gbs"],
                "k1_achieved": b_step / k1_avg_s / 1e9, "k1_frac": b_step / k1_avg_s / 1e9 / peaks["hbm_gbs"],
                "solve_ms_per_step": 1e3 * step_s,
                "solve_achieved": b_step / step_s / 1e9,
                "solve_frac": b_step / step_s / 1e9 / peaks["hbm_gbs"]} if not fused else None
    traffic = (recorded_traffic(K1_SUMMARIES[args.workload]) if args.workload in K1_SUMMARIES else None)
    te.te_matrix_free(H)
    te.te_destroy(ctx)
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": (value / PAPER_SOLVES_PER_S[args.workload]
                            if args.workload in PAPER_SOLVES_PER_S else None),
            "dtype": "complex128", "data": ("synthetic (seeded model parameters, "
                                            f"{DESCRIBE[args.workload].split(',')[0]})"),
            "config": config_block(wl, argparse.Namespace(gpus=world, workload=args.workload)),
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": fp64_peak,
                         "unit": "TFLOP/s", "frac": achieved_tf / fp64_peak,
                         "traffic": traffic,
                         "kernel": k1_name,
                         "timing": k1_timing,
                         "value_table": info["sell_dict"],
                         "slices_per_task": info["sell_tpt"],
                         "flops_per_launch": k1_flops, "bytes_per_launch": k1_bytes,
                         "complex_equivalent_tflops": k1_flops_complex / k1_avg_s / 1e12,
                         "avg_launch_ms": 1000.0 * k1_avg_s,
                         "peak_kind": ("derived FP64 pipe peak: 152 SMs x 2 DFMA lanes x 2 FLOP x "
                                       f"{sm_max_mhz:.0f} MHz"),
                         "attainable": fp64_att,
                         "hbm": {"achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                 "frac": achieved / peaks["hbm_gbs"],
                                 "peak_kind": f"{kind} (MEASURED_PEAKS.json hbm_gbs)"},
                         "hbm_csr_step": csr_step,
                         "dram_overfetch": (traffic / k1_bytes if traffic else None)},
            "spmv_gbs": achieved,
            "solve": {"restarts": restarts[0], "matvecs": stats[0]["matvecs"],
                      "err_bound": stats[0]["err_bound"], "roundoff_est": stats[0]["roundoff_est"],
                      "quad_integrals": stats[0]["quad_integrals"], "quad_nodes": stats[0]["quad_nodes"],
                      "step_kernel_mcycles": {"eig": stats[0]["eig_mcycles"],
                                              "search": stats[0]["search_mcycles"]}},
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": 16 * d,
                    "d2h_bytes_per_step": 16 * d},
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        if world == 1 and not args.no_cpu_baseline and wl["params"]["model"] in ("tfim", "xxzdm", "coo"):
            line["cpu_baseline"] = cpu_baseline_entry(wl)
        if world == 1 and args.workload == WORKLOAD and not args.no_other_configs:
            line["other_configs"] = other_configs()
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_batch(args):
    """Many vectors under one H through te_evolve_batch (one block product per
    Lanczos step), against the same vectors solved one at a time (te_evolve)."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2205_15346_gb300 import te

    wl = W.workload(args.workload)
    p, d, t, tol, m, nvec = wl["params"], wl["d"], wl["t"], wl["tol"], wl["m"], wl["nvec"]
    ctx = te.te_create(local)
    H = te.te_build_model(ctx, p)
    te.te_matrix_tune(ctx, H)                 # the one-at-a-time comparison uses the sliced SpMV
    info = te.te_matrix_info_get(H)
    V0 = W.initial_block(wl["v0_seeds"], d)
    vin = torch.from_numpy(V0).cuda()
    vout = torch.empty_like(vin)
    opt = te.make_options(profile=True)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        te.te_evolve_batch(ctx, H, vin, t, tol, m, opt, v_out=vout)
    barrier()
    stats = []
    with ClockSampler(local) as clk:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            _, sts, _, _ = te.te_evolve_batch(ctx, H, vin, t, tol, m, opt, v_out=vout)
            stats.append(sts)
        ev1.record(stream)
        barrier()
    elapsed = max_over_ranks(ev0.elapsed_time(ev1) / 1000.0)
    value = nvec * job_throughput(args.steps, world, elapsed)

    # the same vectors one at a time through te_evolve (the plain GPU method)
    single = torch.empty((nvec, d), dtype=torch.complex128, device="cuda")
    te.te_evolve(ctx, H, vin[0], t, tol, m, v_out=single[0])
    torch.cuda.synchronize()
    a = time.perf_counter()
    for b in range(nvec):
        te.te_evolve(ctx, H, vin[b], t, tol, m, v_out=single[b])
    torch.cuda.synchronize()
    solo_s = time.perf_counter() - a
    worst = max(torch.linalg.vector_norm(single[b] - vout[b]).item() / tol for b in range(nvec))
    del single

    # end to end through the C ABI with pinned host blocks (copies inside the timed region)
    hin = torch.from_numpy(V0).pin_memory()
    hout = torch.empty_like(hin).pin_memory()
    opt_e2e = te.make_options()
    te.te_evolve_batch(ctx, H, hin.numpy(), t, tol, m, opt_e2e, v_out=hout.numpy())
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        te.te_evolve_batch(ctx, H, hin.numpy(), t, tol, m, opt_e2e, v_out=hout.numpy())
    barrier()
    e2e_value = nvec * job_throughput(args.steps, world, max_over_ranks(time.perf_counter() - t0))

    # roofline of the block product (KB1), live CUDA-event times.  It executes
    # 3 DFMA per stored entry per vector (the three-multiplication complex product)
    # plus 8 FP64 instructions per row per vector (12 FLOP: combine, scale,
    # three-term subtraction, alpha partial); the plain complex product would
    # need 8 FLOP per entry per vector.
    nnz = info["nnz"]
    B = 1 << (nvec - 1).bit_length()
    kb1_flops = (6 * nnz + 12 * d) * B
    kb1_flops_complex = (8 * nnz + 12 * d) * B
    kb1_bytes = 28 * nnz + 4 * (d + 1) + 56 * d * B
    s0 = stats[0][0]
    spmv_ms = sum(st[0]["spmv_ms"] for st in stats)
    spmv_n = sum(st[0]["spmv_launches"] for st in stats)
    kb1_avg_s = spmv_ms / spmv_n / 1000.0
    peaks, kind = measured_peaks()
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp64_peak = SMS * DFMA_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
    achieved_tf = kb1_flops / kb1_avg_s / 1e12
    fp64_att = attainable_fp64(ctx, achieved_tf)
    achieved_gbs = kb1_bytes / kb1_avg_s / 1e9
    rounds = [max(x["restarts"] for x in st) for st in stats]
    launches = sum(4 + r * (4 * m + 3) for r in rounds)
    te.te_matrix_free(H)
    te.te_destroy(ctx)
    if rank == 0:
        line = {
            "metric": METRIC, "mode": "batch", "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "complex128",
            "data": "synthetic (seeded XXZ-DM parameters and 64 seeded random initial vectors)",
            "config": config_block(wl, argparse.Namespace(gpus=world, workload=args.workload)),
            "one_at_a_time": {"solves_per_s": nvec / solo_s,
                              "how": "te_evolve on the same vectors, one after another"},
            "batched_over_one_at_a_time": value / (nvec / solo_s),
            "max_diff_over_tol_vs_alone": worst,
            "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": fp64_peak,
                         "unit": "TFLOP/s", "frac": achieved_tf / fp64_peak,
                         "traffic": recorded_traffic(
                             os.path.join(ROOT, "profiles", "k_spmm_block_batch_xxzdm_L20_x64.md"),
                             _csrc("te_block.cu")),
                         "kernel": "k_spmm_block (KB1: Y = s H X - b X_prev per vector, alpha partials)",
                         "flops_per_launch": kb1_flops,
                         "complex_equivalent_tflops": kb1_flops_complex / kb1_avg_s / 1e12,
                         "bytes_per_launch": kb1_bytes, "avg_launch_ms": 1000.0 * kb1_avg_s,
                         "peak_kind": ("derived FP64 pipe peak: 152 SMs x 2 DFMA lanes x 2 FLOP x "
                                       f"{sm_max_mhz:.0f} MHz"),
                         "attainable": fp64_att,
                         "hbm": {"achieved": achieved_gbs, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                                 "frac": achieved_gbs / peaks["hbm_gbs"],
                                 "peak_kind": f"{kind} (MEASURED_PEAKS.json hbm_gbs)"}},
            "solve": {"restart_rounds": rounds[0], "restarts_vec0": s0["restarts"],
                      "matvecs_vec0": s0["matvecs"], "err_bound_vec0": s0["err_bound"]},
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": 16 * d * nvec,
                    "d2h_bytes_per_step": 16 * d * nvec},
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline_entry(single_view(wl))
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_multi(args):
    """Independent problems through te_evolve_multi (one grouped launch per
    Lanczos step), against the same problems one at a time (te_evolve) and all
    submitted at once to the request scheduler (te_submit)."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2205_15346_gb300 import te

    wl = W.workload(args.workload)
    probs, tol, m = wl["problems"], wl["tol"], wl["m"]
    n = len(probs)
    ctx = te.te_create(local)
    Hs = [te.te_build_model(ctx, q["params"]) for q in probs]
    for H in Hs:
        te.te_matrix_tune(ctx, H)
    infos = [te.te_matrix_info_get(H) for H in Hs]
    v0 = [W.random_state(q["v0_seed"], q["d"]) for q in probs]
    vin = [torch.from_numpy(v).cuda() for v in v0]
    vout = [torch.empty_like(v) for v in vin]
    ts = [q["t"] for q in probs]
    opt = te.make_options(profile=True)
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        te.te_evolve_multi(ctx, Hs, vin, ts, tol, m, opt, v_outs=vout)
    barrier()
    stats = []
    with ClockSampler(local) as clk:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            _, sts, _, _ = te.te_evolve_multi(ctx, Hs, vin, ts, tol, m, opt, v_outs=vout)
            stats.append(sts)
        ev1.record(stream)
        barrier()
    elapsed = max_over_ranks(ev0.elapsed_time(ev1) / 1000.0)
    value = n * job_throughput(args.steps, world, elapsed)

    # one at a time (te_evolve), and all at once through the request scheduler
    single = [torch.empty_like(v) for v in vin]
    for i in range(n):
        te.te_evolve(ctx, Hs[i], vin[i], ts[i], tol, m, v_out=single[i])
    torch.cuda.synchronize()
    a = time.perf_counter()
    worst = 0.0
    for i in range(n):
        te.te_evolve(ctx, Hs[i], vin[i], ts[i], tol, m, v_out=single[i])
    torch.cuda.synchronize()
    solo_s = time.perf_counter() - a
    for i in range(n):
        worst = max(worst, torch.linalg.vector_norm(single[i] - vout[i]).item() / tol)
    a = time.perf_counter()
    reqs = [te.te_submit(ctx, Hs[i], vin[i], ts[i], tol, m) for i in range(n)]
    for i, r in enumerate(reqs):
        s_, _ = te.te_wait(r, -1.0, single[i])
        te.te_request_free(r)
    sched_s = time.perf_counter() - a

    # end to end with pinned host vectors (copies inside the timed region)
    hin = [torch.from_numpy(v).pin_memory() for v in v0]
    hout = [torch.empty_like(h).pin_memory() for h in hin]
    opt_e2e = te.make_options()
    te.te_evolve_multi(ctx, Hs, [h.numpy() for h in hin], ts, tol, m, opt_e2e,
                       v_outs=[h.numpy() for h in hout])
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        te.te_evolve_multi(ctx, Hs, [h.numpy() for h in hin], ts, tol, m, opt_e2e,
                           v_outs=[h.numpy() for h in hout])
    barrier()
    e2e_value = n * job_throughput(args.steps, world, max_over_ranks(time.perf_counter() - t0))

    # roofline of the grouped SpMV (KM1): executed FP64 work over all its launches
    def flops_per_matvec(info):
        d, nnz = info["d"], info["nnz"]
        if info["sell_dict"] > 0 and info["sell_real"]:
            return 4 * (nnz - d) + 14 * d
        if info["sell_dict"] > 0:
            return 6 * (nnz - d) + 16 * d
        return 6 * nnz + 12 * d
    fl = [flops_per_matvec(x) for x in infos]
    # one grouped product per round is timed (Lanczos step m/2); problem i takes part
    # in rounds 1..restarts_i, so the timed products carry sum_i restarts_i fl_i
    total_flops = sum(sum(st[i]["restarts"] * fl[i] for i in range(n)) for st in stats)
    spmv_ms = sum(st[0]["spmv_ms"] for st in stats)
    spmv_n = sum(st[0]["spmv_launches"] for st in stats)
    peaks, kind = measured_peaks()
    sm_max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp64_peak = SMS * DFMA_LANES_PER_SM * 2 * sm_max_mhz * 1e6 / 1e12
    achieved_tf = total_flops / (spmv_ms / 1000.0) / 1e12
    fp64_att = attainable_fp64(ctx, achieved_tf)
    rounds = [max(x["restarts"] for x in st) for st in stats]
    launches = sum(2 * n + 2 + r * (4 * m + 3) for r in rounds)
    for H in Hs:
        te.te_matrix_free(H)
    te.te_destroy(ctx)
    if rank == 0:
        line = {
            "metric": METRIC, "mode": "multi", "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "complex128",
            "data": "synthetic (32 seeded TFIM parameter sets, seeded random initial vectors)",
            "config": config_block(wl, argparse.Namespace(gpus=world, workload=args.workload)),
            "one_at_a_time": {"solves_per_s": n / solo_s,
                              "how": "te_evolve on each problem, one after another"},
            "scheduler_all_at_once": {"solves_per_s": n / sched_s,
                                      "how": "te_submit of all problems, then te_wait"},
            "grouped_over_one_at_a_time": value / (n / solo_s),
            "max_diff_over_tol_vs_alone": worst,
            "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": fp64_peak,
                         "unit": "TFLOP/s", "frac": achieved_tf / fp64_peak,
                         "traffic": recorded_traffic(
                             os.path.join(ROOT, "profiles", "k_spmv_multi_tfim_multi_x32.md"),
                             _csrc("te_multi.cu", "te_slices.cuh")),
                         "kernel": "k_spmv_multi (KM1: grouped SpMV of all running problems)",
                         "avg_launch_ms": spmv_ms / spmv_n,
                         "flops": ("executed FP64 work of the timed grouped SpMV launches (step m/2 "
                                   "of every round) / their CUDA-event time"),
                         "peak_kind": ("derived FP64 pipe peak: 152 SMs x 2 DFMA lanes x 2 FLOP x "
                                       f"{sm_max_mhz:.0f} MHz"),
                         "attainable": fp64_att},
            "solve": {"restart_rounds": rounds[0],
                      "restarts": [x["restarts"] for x in stats[0]]},
            "e2e": {"value": e2e_value, "unit": "solves/s",
                    "h2d_bytes_per_step": 16 * sum(q["d"] for q in probs),
                    "d2h_bytes_per_step": 16 * sum(q["d"] for q in probs)},
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        if world == 1 and not args.no_cpu_baseline:
            rate, wall, mv = oracle_multi_sample(wl)
            line["cpu_baseline"] = {"value": rate, "unit": "solves/s", "cores": 1, "kind": "oracle",
                                    "sample": (f"oracle (1 thread) first restart of each of the "
                                               f"{n} problems ({mv} matvecs, {wall:.1f} s); solves/s = "
                                               f"{n} / sum of (wall / fraction of t covered)")}
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def run_sampled(args):
    """A solve with intermediate samples and observables (te_evolve_sampled),
    against the same solve without them (te_evolve)."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    from paper_2205_15346_gb300 import te

    wl = W.workload(args.workload)
    p, d, t, tol, m = wl["params"], wl["d"], wl["t"], wl["tol"], wl["m"]
    ts = wl["samples"]
    ctx = te.te_create(local)
    H = te.te_build_model(ctx, p)
    te.te_matrix_tune(ctx, H)
    L = 2 + p["K"] + p["Kp"]
    occ = torch.stack([te.te_model_occupation(ctx, p, l, out=torch.empty(d, dtype=torch.float64,
                                                                         device="cuda"))
                       for l in range(L)])
    v0 = W.initial_vector(wl["v0"], d, index_of=lambda o: te.te_model_basis_index(p, o))
    vin = torch.from_numpy(v0).cuda()
    opt = te.make_options()
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        te.te_evolve_sampled(ctx, H, vin, t, ts, tol, m, opt, observables=occ, want_vectors=False)
    barrier()
    with ClockSampler(local) as clk:
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            _, _, n, bounds, st, _ = te.te_evolve_sampled(ctx, H, vin, t, ts, tol, m, opt,
                                                          observables=occ, want_vectors=False)
        ev1.record(stream)
        barrier()
    elapsed = max_over_ranks(ev0.elapsed_time(ev1) / 1000.0)
    value = job_throughput(args.steps, world, elapsed)
    # the same solve without samples
    vout = torch.empty_like(vin)
    te.te_evolve(ctx, H, vin, t, tol, m, opt, v_out=vout)
    torch.cuda.synchronize()
    a = time.perf_counter()
    for _ in range(args.steps):
        te.te_evolve(ctx, H, vin, t, tol, m, opt, v_out=vout)
    torch.cuda.synchronize()
    plain = args.steps / (time.perf_counter() - a)
    # end to end with host buffers: v_in, v_out and the observables cross the link
    hin = v0.copy()
    occ_h = occ.cpu().numpy()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        te.te_evolve_sampled(ctx, H, hin, t, ts, tol, m, opt, observables=occ_h, want_vectors=False)
    barrier()
    e2e_value = job_throughput(args.steps, world, max_over_ranks(time.perf_counter() - t0))
    conserved = max(float(np.max(np.abs(n[:, 0] + n[:, 1] - p["N0"]))),
                    float(np.max(np.abs(n[:, 2:].sum(1) - p["Nm"]))))
    launches = 4 + st["restarts"] * (2 * m + 5) + 2
    te.te_matrix_free(H)
    te.te_destroy(ctx)
    if rank == 0:
        line = {
            "metric": METRIC, "mode": "sampled", "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak",
            "vs_baseline": (value / PAPER_SOLVES_PER_S["memory_K10"]),
            "dtype": "complex128", "data": "the paper's example system (deterministic parameters, Sec. 5)",
            "config": config_block(wl, argparse.Namespace(gpus=world, workload=args.workload)),
            "samples": len(ts), "observables": L,
            "without_samples": {"solves_per_s": plain, "how": "te_evolve, same solve"},
            "sampling_overhead": plain / value - 1.0,
            "max_conservation_violation": conserved,
            "max_sample_bound": float(np.max(bounds)),
            "solve": {"restarts": st["restarts"], "matvecs": st["matvecs"], "err_bound": st["err_bound"]},
            "e2e": {"value": e2e_value, "unit": "solves/s",
                    "h2d_bytes_per_step": 16 * d + 8 * d * L,
                    "d2h_bytes_per_step": 16 * d + 8 * len(ts) * L},
            "gpu_launches": launches,
            "clocks": clk.summary(),
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# The paper's fit of its single-thread CPU runtime, t = a d^b (Sec. 5).
PAPER_FIT_A, PAPER_FIT_B = 8.1e-6, 1.23


def run_scaling(args):
    """Solve time against the dimension for the sizes of the paper's runtime study,
    beside the paper's fitted CPU times (context: other hardware)."""
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    from paper_2205_15346_gb300 import te
    wl = W.workload(args.workload)
    t, tol, m = wl["t"], wl["tol"], wl["m"]
    ctx = te.te_create(local)
    rows = []
    with ClockSampler(local) as clk:
        for q in wl["sizes"]:
            p, d = q["params"], q["d"]
            H = te.te_build_model(ctx, p)
            te.te_matrix_tune(ctx, H)
            v0 = W.initial_vector(q["v0"], d, index_of=lambda o: te.te_model_basis_index(p, o))
            vin = torch.from_numpy(v0).cuda()
            vout = torch.empty_like(vin)

            def timed(opt):
                for _ in range(args.warmup):
                    te.te_evolve(ctx, H, vin, t, tol, m, opt, v_out=vout)
                torch.cuda.synchronize()
                ev0 = torch.cuda.Event(enable_timing=True)
                ev1 = torch.cuda.Event(enable_timing=True)
                ev0.record()
                for _ in range(args.steps):
                    _, st, _ = te.te_evolve(ctx, H, vin, t, tol, m, opt, v_out=vout)
                ev1.record()
                torch.cuda.synchronize()
                return ev0.elapsed_time(ev1) / 1000.0 / args.steps, st

            sec, st = timed(te.make_options())
            fit = PAPER_FIT_A * d ** PAPER_FIT_B
            row = {"K": p["K"], "N0": p["N0"], "d": d, "nnz": te.te_matrix_info_get(H)["nnz"],
                   "gpu_s_per_solve": sec, "paper_fit_cpu_s": fit, "ratio_to_fit": fit / sec,
                   "restarts": st["restarts"], "err_bound": st["err_bound"]}
            if args.quad_study:
                # Sec. 4: Gauss-Legendre against tanh-sinh for the error integral.  The step
                # kernel's SM cycles over the solve give its share of the solve time.
                quad = {}
                outs = {}
                for name in ("tanh-sinh", "gauss"):
                    qs, qst = timed(te.make_options(quad=name))
                    k3_ms = (qst["eig_mcycles"] + qst["search_mcycles"]) * 1e3 / sm_mhz_now(local)
                    quad[name] = {"s_per_solve": qs, "solves_per_s": 1.0 / qs,
                                  "restarts": qst["restarts"], "quad_integrals": qst["quad_integrals"],
                                  "quad_nodes": qst["quad_nodes"], "step_kernel_ms": k3_ms,
                                  "step_kernel_share": k3_ms / (1e3 * qs), "err_bound": qst["err_bound"]}
                    outs[name] = vout.clone()
                quad["norm_diff"] = torch.linalg.vector_norm(outs["gauss"] - outs["tanh-sinh"]).item()
                quad["norm_diff_over_tol"] = quad["norm_diff"] / tol
                row["quadrature"] = quad
            rows.append(row)
            te.te_matrix_free(H)
    te.te_destroy(ctx)
    # the GPU's own power law over the four fitted sizes
    xs = np.log([r["d"] for r in rows[:4]])
    ys = np.log([r["gpu_s_per_solve"] for r in rows[:4]])
    b, loga = np.polyfit(xs, ys, 1)
    k10 = rows[3]
    line = {
        "metric": METRIC, "mode": "scaling", "value": 1.0 / k10["gpu_s_per_solve"], "unit": "solves/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * k10["gpu_s_per_solve"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": (1.0 / k10["gpu_s_per_solve"]) / PAPER_SOLVES_PER_S["memory_K10"],
        "dtype": "complex128", "data": "the paper's example system (deterministic parameters, Sec. 5)",
        "config": {"workload": f"{wl['name']}: {DESCRIBE[wl['name']]}, m={m}, tol={tol}",
                   "value_is": "solves/s at K=K'=10, N0=Nc=100 (d=1565904)"},
        "sizes": rows,
        "gpu_fit": {"a": float(np.exp(loga)), "b": float(b)},
        "paper_fit": {"a": PAPER_FIT_A, "b": PAPER_FIT_B, "hardware": "i9-9900K, 1 thread"},
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def run_serve(args):
    """Serving (the request-stream configuration): Poisson arrivals of mixed
    requests through te_submit (continuous batching), against the one-at-a-time
    GPU method (te_evolve, one request after the other, first come first served)
    on the same arrivals.

    The one-at-a-time service time s_i of every request is measured by solving
    the requests one after another; its latencies at an arrival process a_i are
    then those of a single FIFO server: f_i = max(a_i, f_{i-1}) + s_i,
    latency_i = f_i - a_i (exact for a server that runs one solve at a time).
    Capacity = 1 / mean(s_i); each load sets the arrival rate to load x capacity.
    Both sides take host vectors and return host vectors."""
    import torch
    from paper_2205_15346_gb300 import te
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    ctx = te.te_create(local)
    te.te_serve_config(ctx, te.TE_SERVE_BATCH, 40, args.arena, args.large_nnz, args.small_nnz)
    m = 40
    pool = []
    for fam, p in W.serve_pool():
        H = te.te_build_model(ctx, p)
        te.te_matrix_tune(ctx, H)
        d = te.te_matrix_info_get(H)["d"]
        # four seeded initial states per Hamiltonian; request i takes variant i mod 4
        pool.append((H, d, [W.random_state(600 + 4 * len(pool) + j, d) for j in range(4)]))
    nnz_of = [te.te_matrix_info_get(H)["nnz"] for H, _, _ in pool]

    def lane_of(k):
        n = nnz_of[k]
        if args.large_nnz > 0 and n >= args.large_nnz:
            return "large"
        return "small" if n < args.small_nnz else "medium"
    loads = [float(x) for x in args.loads.split(",")]
    counts = ([int(x) for x in args.requests_per_load.split(",")] if args.requests_per_load
              else [args.requests] * len(loads))
    if len(counts) != len(loads):
        raise SystemExit("--requests-per-load needs one count per load")
    n_max = max(counts)
    reqs = W.serve_requests(n_max)
    vin = lambda i: pool[reqs[i][0]][2][i % 4]
    outbuf = {d: np.empty(d, dtype=np.complex128) for _, d, _ in pool}
    check = set(range(0, n_max, max(1, n_max // 48)))      # results compared alone vs mixed
    clk = ClockSampler(local).__enter__()          # sampled over warm-up, solo and served runs
    # warm-up: a solve per Hamiltonian (plans, graphs) and a few served requests (arena, graphs)
    for H, d, vs in pool:
        te.te_evolve(ctx, H, vs[0], 1.0, 1e-8, m)
    warm = [te.te_submit(ctx, pool[k][0], pool[k][2][0], 1.0, 1e-8, m) for k in range(0, len(pool), 5)]
    for r in warm:
        te.te_wait(r, -1.0, None)
        te.te_request_free(r)
    # one at a time: service time of every request
    solo_s, solo_out = [], {}
    t_solo = time.perf_counter()
    for i, (k, t, tol, sd, gap) in enumerate(reqs):
        a = time.perf_counter()
        out, st, _ = te.te_evolve(ctx, pool[k][0], vin(i), t, tol, m, v_out=outbuf[pool[k][1]])
        solo_s.append(time.perf_counter() - a)
        if i in check:
            solo_out[i] = out.copy()
    solo_wall = time.perf_counter() - t_solo
    solo_s = np.array(solo_s)
    cap_per_s = 1.0 / float(np.mean(solo_s))
    runs, worst = [], 0.0
    for load, n in zip(loads, counts):
        rate = load * cap_per_s
        arrivals = np.cumsum([reqs[i][4] / rate for i in range(n)])
        arrivals -= arrivals[0]
        # the one-at-a-time server on these arrivals
        f, lat_solo = 0.0, []
        for i in range(n):
            f = max(arrivals[i], f) + solo_s[i]
            lat_solo.append(f - arrivals[i])
        solo_span = f - arrivals[0]
        # served: submit at the arrival times, poll, copy each result out
        pending, lat = {}, np.zeros(n)
        nxt = 0
        t0 = time.perf_counter()
        while nxt < n or pending:
            now = time.perf_counter() - t0
            while nxt < n and arrivals[nxt] <= now:
                k, t, tol, sd, gap = reqs[nxt]
                pending[nxt] = te.te_submit(ctx, pool[k][0], vin(nxt), t, tol, m)
                nxt += 1
            for i in list(pending):
                if te.te_poll(pending[i], None)[0] == te.TE_PENDING:
                    continue
                k = reqs[i][0]
                out = outbuf[pool[k][1]]
                s, st = te.te_poll(pending[i], out)
                if s != te.TE_OK:
                    raise RuntimeError(f"request {i} failed: {te.te_status_string(s)} "
                                       f"({te.te_last_error(ctx)})")
                lat[i] = time.perf_counter() - t0 - arrivals[i]
                if i in solo_out:
                    worst = max(worst, float(np.linalg.norm(out - solo_out[i])) / reqs[i][2])
                te.te_request_free(pending.pop(i))
            time.sleep(0.0002)
        span = time.perf_counter() - t0
        by_lane = {}
        for lane in ("small", "medium", "large"):
            idx = [i for i in range(n) if lane_of(reqs[i][0]) == lane]
            if idx:
                by_lane[lane] = {"requests": len(idx),
                                 "served_ms_p50": 1e3 * float(np.percentile(lat[idx], 50)),
                                 "served_ms_p99": 1e3 * float(np.percentile(lat[idx], 99)),
                                 "one_at_a_time_ms_p50": 1e3 * float(np.percentile(np.array(lat_solo)[idx], 50)),
                                 "one_at_a_time_ms_p99": 1e3 * float(np.percentile(np.array(lat_solo)[idx], 99)),
                                 "service_ms_p50": 1e3 * float(np.percentile(solo_s[idx], 50))}
        runs.append({
            "by_lane": by_lane,
            "load": load, "requests": n, "arrival_rate_per_s": rate,
            "served": {"solves_per_s": n / span, "latency_ms_p50": 1e3 * float(np.percentile(lat, 50)),
                       "latency_ms_p99": 1e3 * float(np.percentile(lat, 99)),
                       "latency_ms_mean": 1e3 * float(np.mean(lat))},
            "one_at_a_time": {"solves_per_s": n / solo_span,
                              "latency_ms_p50": 1e3 * float(np.percentile(lat_solo, 50)),
                              "latency_ms_p99": 1e3 * float(np.percentile(lat_solo, 99)),
                              "latency_ms_mean": 1e3 * float(np.mean(lat_solo))},
        })
    clk.__exit__(None, None, None)
    head = runs[loads.index(0.8)] if 0.8 in loads else runs[0]
    lane = ((f"large lane (one at a time, solo solve) for nnz >= {args.large_nnz}" if args.large_nnz > 0
             else "no large lane") + "; " +
            (f"small batch for nnz < {args.small_nnz}, medium batch above" if args.small_nnz > 0
             else "one batch"))
    line = {
        "metric": METRIC, "mode": "serve", "value": head["served"]["solves_per_s"], "unit": "solves/s",
        "n_gpus": 1, "steps": head["requests"], "warmup": len(pool) + len(warm),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "ms_per_step": 1e3 / head["served"]["solves_per_s"], "dtype": "complex128",
        "data": ("synthetic Poisson request mix (workloads.serve_requests, seed 5; four seeded "
                 "initial states per Hamiltonian)"),
        "config": {"workload": ("serving: Poisson requests over 2 x 16 Hamiltonians (spin: TFIM/XXZ-DM "
                                "L 10..22; bosons: K=12 N=6 and K=14 N=6..10), half of each, "
                                "t log-U[1,100], tol in {1e-6,1e-8,1e-10}, m=40; continuous batching "
                                f"(arena {args.arena} elements per Krylov column); " + lane),
                   "loads": loads, "requests_per_load": counts,
                   "l2": "inputs larger than L2 for the large requests; no flush"},
        "latency_ms": {"p50": head["served"]["latency_ms_p50"], "p99": head["served"]["latency_ms_p99"]},
        "one_at_a_time": {"capacity_solves_per_s": cap_per_s, "requests_timed": n_max,
                          "wall_s": solo_wall,
                          "service_ms_p50": 1e3 * float(np.percentile(solo_s, 50)),
                          "service_ms_p99": 1e3 * float(np.percentile(solo_s, 99))},
        "runs": runs,
        "max_diff_over_tol_vs_alone": worst,
        "compared_alone_vs_mixed": len(check),
        "clocks": clk.summary(),
    }
    for H, d, vs in pool:
        te.te_matrix_free(H)
    te.te_destroy(ctx)
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-other-configs", action="store_true",
                    help="default workload: skip the short runs of the other configurations")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(DESCRIBE) + ["serve_mix"])
    ap.add_argument("--requests", type=int, default=200, help="serve_mix: requests per load")
    ap.add_argument("--requests-per-load", default="",
                    help="serve_mix: comma-separated request counts, one per load")
    ap.add_argument("--loads", default="0.5,0.8,1.0,1.2",
                    help="serve_mix: arrival rates as fractions of one-at-a-time capacity")
    ap.add_argument("--quad-study", action="store_true",
                    help="memory_scaling: also time every size with Gauss-Legendre and tanh-sinh")
    ap.add_argument("--large-nnz", type=int, default=1 << 24,
                    help="serve_mix: large-lane threshold on nnz (negative: batch everything)")
    ap.add_argument("--small-nnz", type=int, default=1 << 21,
                    help="serve_mix: small-batch threshold on nnz (negative: one batch)")
    ap.add_argument("--arena", type=int, default=1 << 25,
                    help="serve_mix: elements per Krylov column of the serving arena")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)     # at least three untimed warm-up steps
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serve_mix":
        return run_serve(args)
    if "nvec" in W.workload(args.workload):
        return run_batch(args)
    if "problems" in W.workload(args.workload):
        return run_multi(args)
    if "samples" in W.workload(args.workload):
        return run_sampled(args)
    if "sizes" in W.workload(args.workload):
        return run_scaling(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
