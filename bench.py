#!/usr/bin/env python
"""Benchmark: factor + solve DOF/s at relative residual 1e-12 (HIF-DE, GB300).

One step = one pass of the whole hot path on the 2D high-contrast workload
(511 x 511 interior grid, quantized field of contrast 1e6, b = 1e-3,
eps = 1e-6, 8 standard-normal right-hand sides): ``hif_factor`` (Algorithm 4.1)
then ``hif_solve`` (PCG with F^-1 to ||b - A x|| <= 1e-12 ||b|| for every
column), inputs resident in HBM.  The L2 cache is flushed (256 MB write)
between timed steps, outside the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on a bounded sample of the same workload instead.  With N > 1 (torchrun) every
rank runs an independent replica of the workload (the method has no exchange
step for one problem on one GPU): value = DOF of all ranks / max rank time.

Other workloads, one JSON line each:

    python bench.py --workload3d laplace3d_n64|contrast3d_n128 [--eps E] [--variant hifde|hifde3x]
                    [--precision fp64|mixed|fp32_apply] [--tensor-cores 0|1|2|3|-1]
    python bench.py --batched          # 64 independent 2D problems, 32 RHS each
                                       # (under torchrun: problems sharded over the ranks)
    python bench.py --tc-roofline      # the tensor-core Schur update alone

and the profiling helpers ``--ncu-apply K`` / ``--ncu-solve K`` (fixed launch
shapes, for ncu captures).
"""
import os

# the CPU oracle legs measure single-threaded numpy; set before numpy loads
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "factor+solve DOF/s at rel. residual 1e-12: learned/mixed vs plain FP64 GPU"
WORKLOAD = "2D high-contrast 511x511 (contrast 1e6, b=1e-3), eps=1e-6, 8 RHS, PCG to 1e-12"
TOL = 1e-12
ORACLE_SAMPLE_N = 128      # the CPU oracle's bounded sample: same recipe on a 127 x 127 grid
ORACLE_SAMPLE_TOL = 1e-9   # FP64 CG floor of that sample is ~5e-11 (no double-double in the oracle)


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.samples = []
        self._stop = threading.Event()
        self._proc = None
        self._thr = None

    def start(self):
        try:
            self._proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self._proc = None
            return

        def reader():
            for line in self._proc.stdout:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    self.samples.append(parts)
                if self._stop.is_set():
                    break

        self._thr = threading.Thread(target=reader, daemon=True)
        self._thr.start()

    def stop(self):
        self._stop.set()
        if self._proc is not None:
            self._proc.terminate()
            try:
                self._proc.wait(timeout=5)
            except Exception:
                self._proc.kill()
        if self._thr is not None:
            self._thr.join(timeout=2)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for s in self.samples:
            for name, val in zip(names, s[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(self.samples)}


def _workload_arrays(name: str = "contrast2d_n512"):
    from paper_1307_2895_gb300 import inputs
    w = inputs.workload(name)
    f = inputs.rhs(w["dim"], w["n"], w["nrhs"], seed=0)
    return w, f


# ---------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# ---------------------------------------------------------------------------
def oracle_sample_step():
    """One bounded oracle step: factor + PCG (1 RHS) on the same recipe at n = 128."""
    from oracle import hifde, stencil
    from paper_1307_2895_gb300 import inputs
    n = ORACLE_SAMPLE_N
    a, _ = inputs.high_contrast_coefficients(2, n, seed=2, low=1e-3, high=1e3)
    b = np.full((n - 1) ** 2, 1e-3)
    f = inputs.rhs(2, n, 1, seed=0)
    A = stencil.assemble(2, n, a, b)
    t0 = time.perf_counter()
    F = hifde.factor(A, 2, n, 1e-6)
    x, iters, rel = hifde.pcg(A, F, f, tol=ORACLE_SAMPLE_TOL, maxit=400)
    dt = time.perf_counter() - t0
    return (n - 1) ** 2 * 1, dt, iters[0], rel[0]


ORACLE_PCG_PROBE = 2   # PCG iterations timed per oracle run (one column)


def oracle_bench_grid(want_finv: bool = False):
    """The oracle on the bench workload itself (511^2, contrast 1e6): the
    factorization in full, then ``ORACLE_PCG_PROBE`` iterations of its PCG on
    one column (each iteration one F^-1 apply and one product with A; the
    run applies F^-1 once more to start and A once more to finish, so the
    time is split over probe + 1 iterations).  Returns the times, and with
    want_finv the oracle's F^-1 f on the 8 right-hand sides."""
    from oracle import hifde, stencil
    w, f = _workload_arrays()
    A = stencil.assemble(w["dim"], w["n"], w["a_stag"], w["b"])
    t0 = time.perf_counter()
    F = hifde.factor(A, w["dim"], w["n"], w["eps"])
    t_factor = time.perf_counter() - t0
    t0 = time.perf_counter()
    hifde.pcg(A, F, f[:, :1], tol=1e-9, maxit=ORACLE_PCG_PROBE)
    t_iter = (time.perf_counter() - t0) / (ORACLE_PCG_PROBE + 1)
    out = {"t_factor": t_factor, "t_iter": t_iter, "N": (w["n"] - 1) ** w["dim"], "nrhs": w["nrhs"]}
    if want_finv:
        out["finv"] = F.apply_inverse(f)
    return out


def _oracle_replica(_):
    return oracle_bench_grid(False)


def cpu_baseline(gpu_iters: int):
    """The oracle on the GPU machine's host cores, on the bench workload: one
    process (one core; numpy single-threaded), then one replica per core at
    once (spawned processes).  The oracle's FP64 PCG cannot reach 1e-12 on
    this field (its residual floor is ~2.5e-10), so its solve is costed at
    the GPU's iteration count: time = t_factor + gpu_iters x nrhs x t_iter."""
    import multiprocessing as mp
    one = oracle_bench_grid(True)
    N, nrhs = one["N"], one["nrhs"]

    def secs(r):
        return r["t_factor"] + gpu_iters * nrhs * r["t_iter"]

    cores = os.cpu_count() or 1
    allc = None
    try:
        with mp.get_context("spawn").Pool(cores) as pool:
            t0 = time.perf_counter()
            reps = pool.map(_oracle_replica, range(cores))
            wall = time.perf_counter() - t0
        allc = {"value": cores * N * nrhs / max(secs(r) for r in reps), "unit": "DOF/s", "cores": cores,
                "sample": f"{cores} concurrent single-threaded replicas of the same measurement "
                          f"({wall:.1f} s wall); value = replicas x N x nrhs / the slowest replica's time"}
    except Exception as exc:   # the all-core leg must not hide the rest
        allc = {"error": repr(exc)}
    base = {"value": N * nrhs / secs(one), "unit": "DOF/s", "cores": 1, "kind": "oracle",
            "sample": f"FP64 numpy oracle on the bench workload (511^2, contrast 1e6, eps 1e-6, 8 RHS): "
                      f"factor {one['t_factor']:.1f} s measured; PCG costed as {gpu_iters} iterations (the "
                      f"GPU's count to 1e-12) x {nrhs} RHS x {one['t_iter']:.3f} s per one-column iteration, "
                      f"measured over {ORACLE_PCG_PROBE} iterations",
            "all_core": allc}
    return base, one["finv"]


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        oracle_sample_step()
    dofs, secs = 0, 0.0
    for _ in range(args.steps):
        d, s, _, _ = oracle_sample_step()
        dofs += d
        secs += s
    value = dofs / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD + " (bounded CPU sample)",
                                            "sample_grid": f"{ORACLE_SAMPLE_N - 1}^2", "nrhs": 1,
                                            "tol": ORACLE_SAMPLE_TOL},
            "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": 1, "kind": "oracle",
                             "sample": f"same recipe on a {ORACLE_SAMPLE_N - 1}^2 grid, 1 RHS, "
                                       f"factor + PCG to {ORACLE_SAMPLE_TOL:g}"},
            "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# replicas over N ranks (weak scaling, no data-path collective)
# ---------------------------------------------------------------------------
def max_over_ranks(secs: float, world: int, device=None) -> float:
    """The slowest rank's time: an all-reduce MAX of one number over the
    default process group (the local time when world == 1)."""
    if world <= 1:
        return secs
    import torch
    import torch.distributed as dist
    t = torch.tensor([secs], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_step: int, steps: int, world: int, tmax_s: float) -> float:
    """Whole-job throughput of `world` independent replicas: the units every
    rank processed in `steps` steps over the slowest rank's time."""
    return world * steps * units_per_step / tmax_s


def shard_problems(sizes, world: int):
    """Independent problems onto `world` ranks by largest-first bin packing:
    in descending size (ties: lower index first), each problem goes to the
    rank with the least work so far (ties: lower rank).  Returns, per rank,
    its problem indices in ascending order; every problem lands on exactly
    one rank and no data moves between ranks afterwards."""
    load = [0] * world
    parts = [[] for _ in range(world)]
    for p in sorted(range(len(sizes)), key=lambda i: (-sizes[i], i)):
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(p)
        load[r] += sizes[p]
    return [sorted(x) for x in parts]


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_gpu(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist
    from paper_1307_2895_gb300 import hif

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    hif.load()
    w, f_np = _workload_arrays()
    dim, n, eps, nrhs = w["dim"], w["n"], w["eps"], w["nrhs"]
    N = (n - 1) ** dim
    st = torch.cuda.Stream(device=dev)
    a = torch.from_numpy(w["a_stag"]).to(dev)
    b = torch.from_numpy(w["b"]).to(dev)
    f = torch.from_numpy(f_np).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            dist.barrier()

    def one_step(precision, profile=False):
        G = hif.factor(dim, n, a, b, eps, precision=precision, stream=st)
        try:
            if profile:
                G.profile(True)
            x, info = G.solve(f, tol=TOL, maxit=1000)
            prof = G.profile(False) if profile else None
            stats = G.stats()
        finally:
            G.free()
        return info, stats, prof

    def timed(precision, steps, warmup, profile=False):
        for _ in range(warmup):
            one_step(precision)
        torch.cuda.synchronize()
        ms, infos, profs, stats = [], [], [], None
        l0 = hif.kernel_launches()
        for _ in range(steps):
            with torch.cuda.stream(st):
                flush.fill_(1.0)
            torch.cuda.synchronize()
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st)
            info, stats, prof = one_step(precision, profile)
            e1.record(st)
            torch.cuda.synchronize()
            barrier()
            ms.append(e0.elapsed_time(e1))
            infos.append(info)
            profs.append(prof)
        launches = hif.kernel_launches() - l0
        return ms, infos, profs, stats, launches

    prec = args.precision
    clocks = ClockSampler(local_rank)
    clocks.start()
    ms, infos, profs, stats, launches = timed(prec, args.steps, args.warmup, profile=True)
    clocks.stop()
    tmax = max_over_ranks(sum(ms) / 1e3, world, dev)
    dofs_per_step = N * nrhs
    value = replica_throughput(dofs_per_step, args.steps, world, tmax)
    conv = all(i["converged"] and i["relres_max"] <= TOL for i in infos)

    # roofline of the dominant kernels (apply sweeps of F^-1), live events
    sweep_ms = sum(p["sweep_ms"] for p in profs)
    sweep_launches = sum(p["sweep_launches"] for p in profs)
    sweep_bytes = sum(p["sweep_bytes"] for p in profs)
    peak, peak_kind = _peaks()
    achieved = (sweep_bytes / sweep_launches) / (sweep_ms / sweep_launches / 1e3) / 1e9 if sweep_ms > 0 else None
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": (achieved / peak) if achieved else None, "traffic": _sweep_traffic(),
            "kernel": "k_apply_up/k_apply_down/k_apply_root (F^-1 sweeps)", "peak_kind": peak_kind,
            "avg_launch_us": 1e3 * sweep_ms / max(sweep_launches, 1),
            "bytes_per_launch": sweep_bytes / max(sweep_launches, 1),
            "share_of_step": sweep_ms / sum(ms) if sum(ms) > 0 else None}

    # plain FP64 GPU path on the same workload (the comparison the metric names)
    plain = None
    if not args.skip_plain:
        pms, pinfos, _, _, _ = timed("fp64", max(1, args.steps // 2), 1)
        ptot = sum(pms) / 1e3
        plain = {"value": len(pms) * dofs_per_step / ptot, "ms_per_step": 1e3 * ptot / len(pms),
                 "iters": pinfos[-1]["iters"], "converged": all(i["converged"] for i in pinfos)}

    # end-to-end through the C ABI with host buffers (pinned), copies inside the step
    e2e = None
    if not args.skip_e2e:
        a_h = torch.from_numpy(w["a_stag"]).pin_memory()
        b_h = torch.from_numpy(w["b"]).pin_memory()
        f_h = torch.from_numpy(f_np).pin_memory()
        x_h = torch.empty_like(f_h).pin_memory()
        e_ms = []
        for i in range(args.steps + 1):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            G = hif.factor(dim, n, a_h, b_h, eps, precision=prec, stream=st)
            try:
                G.solve(f_h, tol=TOL, maxit=1000, out=x_h)
            finally:
                G.free()
            torch.cuda.synchronize()
            if i > 0:
                e_ms.append(1e3 * (time.perf_counter() - t0))
        e_max = max_over_ranks(sum(e_ms) / 1e3, world, dev)
        e2e = {"value": replica_throughput(dofs_per_step, len(e_ms), world, e_max), "unit": "DOF/s",
               "h2d_bytes_per_step": int(a_h.numel() * 8 + b_h.numel() * 8 + f_h.numel() * 8),
               "d2h_bytes_per_step": int(x_h.numel() * 8)}

    cpu = None
    err = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        try:
            cpu, finv_oracle = cpu_baseline(infos[-1]["iters"])
            # error of the timed mode's F^-1 against the FP64 oracle's, same
            # workload and right-hand sides, outside the timed region
            G = hif.factor(dim, n, a, b, eps, precision=prec, stream=st)
            try:
                y = G.apply(f).cpu().numpy()
            finally:
                G.free()
            err = {"what": f"F^-1 f ({prec}) against the FP64 oracle's F^-1 f, bench workload (511^2, 8 RHS)",
                   "rel_2norm": float(np.linalg.norm(y - finv_oracle) / np.linalg.norm(finv_oracle)),
                   "rel_elementwise": float(np.abs(y - finv_oracle).max() / np.abs(finv_oracle).max())}
        except Exception as exc:  # the oracle leg must not hide the GPU result
            cpu = {"error": repr(exc)}

    others = None
    if rank == 0 and world == 1 and not args.skip_others:
        others = other_workloads()

    if rank != 0:
        return 0
    last = infos[-1]
    line = {
        "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum(ms) / len(ms), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "N": N, "nrhs": nrhs, "eps": eps, "tol": TOL,
                   "precision": prec, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "flushed between steps (256 MB write, outside the timed region)",
                   "arith": "factorization f64; factor stored and applied in f32; CG f64 with a "
                            "double-double iterate and residual"},
        "converged": conv, "relres_max": max(i["relres_max"] for i in infos),
        "cg_iters": last["iters"], "refinement_steps": last["outer"],
        "t_factor_ms": stats["t_factor_ms"] if stats else None,
        "root_size": stats["root_size"] if stats else None,
        "plain_fp64": plain,
        "speedup_vs_plain_fp64": (value / world / plain["value"]) if plain else None,
        "e2e": e2e, "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu, "err_vs_oracle": err,
        "other_workloads": others,
        "clocks": clocks.summary(),
    }
    print(json.dumps(line), flush=True)
    return 0


def _sweep_traffic():
    """Measured DRAM bytes per F^-1 sweep launch (dram__bytes_read + write,
    one ncu capture of the same workload), from the committed profile summary;
    None once the sweep kernel source differs from the one captured."""
    import hashlib
    prof = os.path.join(ROOT, "profiles", "dram_sweeps_contrast2d_n512.md")
    src = os.path.join(ROOT, "paper_1307_2895_gb300", "csrc", "kernels_apply.cu")
    try:
        text = open(prof).read()
        sha = hashlib.sha256(open(src, "rb").read()).hexdigest()
    except OSError:
        return None
    val = cap_sha = None
    for line in text.splitlines():
        if line.startswith("traffic_per_launch_bytes:"):
            val = float(line.split(":", 1)[1])
        if line.startswith("kernels_apply.cu sha256:"):
            cap_sha = line.split(":", 1)[1].strip()
    return val if (val is not None and cap_sha == sha) else None


def measure_batched(precision: str, steps: int, warmup: int, rank: int = 0, world: int = 1, local_rank: int = 0):
    """The batched workload (64 independent 2D problems, 32 RHS each) through
    hif_factor_batch / hif_solve_batch: DOF x RHS per second.  With N ranks
    the problems are sharded (shard_problems, weighted by DOF x RHS) and each
    rank factors and solves its own; value = all problems' units over the
    slowest rank's time."""
    import torch
    from paper_1307_2895_gb300 import hif, inputs
    torch.cuda.set_device(local_rank)
    hif.load()
    allp = inputs.batched_problems(64, seed=0)
    units_all = [(p["n"] - 1) ** 2 * p["nrhs"] for p in allp]
    mine = shard_problems(units_all, world)[rank]
    probs = [allp[i] for i in mine]
    rhs = [inputs.rhs(2, p["n"], p["nrhs"], seed=p["seed"]) for p in probs]
    spec = [(p["dim"], p["n"], p["a_stag"], p["b"]) for p in probs]
    units = sum(units_all)
    ms = []
    conv = True
    for step in range(warmup + steps):
        torch.cuda.synchronize()
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        t0 = time.perf_counter()
        facts = hif.factor_batch(spec, 1e-6, precision=precision, nthreads=8)
        try:
            res = hif.solve_batch(facts, rhs, tol=TOL, maxit=2000, nthreads=8)
        finally:
            for F in facts:
                F.free()
        torch.cuda.synchronize()
        if step >= warmup:
            ms.append(1e3 * (time.perf_counter() - t0))
            conv = conv and all(r[1]["converged"] and r[1]["relres_max"] <= TOL for r in res)
    dev = torch.device("cuda", local_rank)
    t = max_over_ranks(sum(ms) / 1e3, world, dev)
    conv = max_over_ranks(0.0 if conv else 1.0, world, dev) == 0.0   # every rank converged
    return {"metric": "factor+solve DOF x RHS/s at rel. residual 1e-12, 64 independent problems",
            "value": units * steps / t, "unit": "DOF*RHS/s", "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": t * 1e3 / steps, "higher_is_better": True,
            "dtype": "f64+f32", "data": "synthetic", "converged": conv,
            "config": {"workload": "64 x 2D contrast 1e2/1e4/1e6, interior edges log-uniform 127..1023 "
                                   "(sum N = %d), 32 RHS each, eps=1e-6" % sum((p["n"] - 1) ** 2 for p in allp),
                       "precision": precision,
                       "parallelism": "8 host threads, one stream per problem" + (
                           "; problems sharded over %d ranks (largest first)" % world if world > 1 else "")},
            "scaling": "strong"}


def run_batched(args, rank: int = 0, world: int = 1, local_rank: int = 0):
    """One JSON line of measure_batched (rank 0)."""
    line = measure_batched(args.precision, args.steps, args.warmup, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def _tf32_peak():
    """Dense TF32 tensor peak: the measured bf16 burst GEMM rate times the
    nominal TF32 / BF16 ratio (1.1 / 2.25 PFLOP/s dense)."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["bf16_tflops"]) * 1.1 / 2.25, "measured bf16 x nominal tf32/bf16"
    except (OSError, KeyError, ValueError):
        return 1900.0 * 1.1 / 2.25, "fallback bf16 x nominal tf32/bf16"


def tc_roofline(split: int = 3, nb: int = 16, m: int = 1024, k: int = 2048, reps: int = 5):
    """The tensor-core Schur update (hif_schur_update_f32) timed alone with CUDA
    events on its stream: nb blocks U -= G G^T, G m x k (inputs 192 MB, beyond
    L2).  Useful work m (m + 1) k flops per block (the lower triangle and the
    diagonal; the mirror is a copy); the tensor pipe issues 1, 3 or 6 TF32
    products for each (split = 1, 2, 3 parts per operand value), over the
    128 x 64 output blocks on and below the diagonal."""
    import torch
    from paper_1307_2895_gb300 import hif
    dev = torch.device("cuda", 0)
    st = torch.cuda.Stream(device=dev)
    gen = torch.Generator(device=dev).manual_seed(0)
    G = torch.randn((nb, m, k), device=dev, generator=gen, dtype=torch.float32)
    U0 = torch.randn((nb, m, m), device=dev, generator=gen, dtype=torch.float32)
    U = U0.clone()
    with torch.cuda.stream(st):
        hif.schur_update(G, U, split=split, stream=st)        # warm-up
        ms = []
        for _ in range(reps):
            U.copy_(U0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            hif.schur_update(G, U, split=split, stream=st)
            e1.record(st)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
    t = sorted(ms)[len(ms) // 2] / 1e3
    rb = (m + 63) // 64
    issued_blocks = sum(min(2 * a + 2, rb) for a in range((rb + 1) // 2))   # (128-row, 64-col) blocks run
    useful = nb * m * (m + 1) * k
    issued = nb * issued_blocks * 128 * 64 * 2 * k * {1: 1, 2: 3, 3: 6}[split]
    peak, how = _tf32_peak()
    achieved = issued / t / 1e12
    return {"kernel": "k_tc_syrk_flat", "shape": f"{nb} x (U {m}x{m} -= G G^T, G {m}x{k})", "split": split,
            "ms": t * 1e3, "useful_fp32_tflops": useful / t / 1e12,
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "peak_source": how, "traffic": None}}


def measure_3d(workload: str, eps: float, variant: str, precision: str, steps: int, warmup: int,
               tensor_cores: int = 0):
    """A 3D workload: factor + 4-RHS PCG to 1e-12 per step, wall clock with a
    device synchronize on both sides (the factorization's host work
    included).  Returns the figures of one JSON object."""
    import torch
    from paper_1307_2895_gb300 import hif, inputs
    hif.load()
    w = inputs.workload(workload)
    n, nrhs = w["n"], w["nrhs"]
    eps = eps if eps > 0 else w["eps"]
    dev = torch.device("cuda", 0)
    st = torch.cuda.Stream(device=dev)
    a = torch.from_numpy(w["a_stag"]).to(dev)
    b = torch.from_numpy(w["b"]).to(dev)
    f = torch.from_numpy(inputs.rhs(3, n, nrhs, seed=0)).to(dev)
    fac, sol, infos, stats = [], [], [], []
    for step in range(warmup + steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        G = hif.factor(3, n, a, b, eps, variant=variant, precision=precision, stream=st,
                       tensor_cores=tensor_cores)
        try:
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            x, info = G.solve(f, tol=TOL, maxit=500)
            torch.cuda.synchronize()
            t2 = time.perf_counter()
            s = G.stats()
        finally:
            G.free()
        if step >= warmup:
            fac.append(t1 - t0)
            sol.append(t2 - t1)
            infos.append(info)
            stats.append(s)
    t = sum(fac) + sum(sol)
    N = (n - 1) ** 3
    return {"metric": "factor+solve DOF x RHS/s at rel. residual 1e-12 (3D)",
            "value": N * nrhs * steps / t, "unit": "DOF*RHS/s", "n_gpus": 1, "steps": steps,
            "warmup": warmup, "ms_per_step": 1e3 * t / steps, "higher_is_better": True,
            "dtype": {"fp64": "f64", "mixed": "f32+f64", "fp32_apply": "f64+f32"}[precision],
            "data": "synthetic",
            "config": {"workload": f"{workload}: {n - 1}^3, eps={eps:g}, {nrhs} RHS",
                       "variant": {"hifde": "hifde3", "hifde3x": "hifde3x"}[variant], "precision": precision,
                       "tensor_cores": tensor_cores},
            "factor_ms": 1e3 * sum(fac) / len(fac), "solve_ms": 1e3 * sum(sol) / len(sol),
            "t_fronts_ms": stats[-1]["t_fronts_ms"], "root_size": stats[-1]["root_size"],
            "cg_iters": infos[-1]["iters"], "relres_max": max(i["relres_max"] for i in infos),
            "converged": all(i["converged"] for i in infos)}


def run_3d(args):
    """One JSON line of measure_3d; in the mixed mode also the tensor-core
    Schur update timed alone."""
    line = measure_3d(args.workload3d, args.eps, args.variant, args.precision, args.steps, args.warmup,
                      args.tensor_cores)
    if args.precision == "mixed" and args.tensor_cores >= 0:
        line["tensor_core_kernel"] = tc_roofline(split=args.tensor_cores or 3)
    print(json.dumps(line), flush=True)
    return 0


def other_workloads():
    """The other configurations of the method, one step each after one
    warm-up (outside the headline's timed region): the 3D Laplacian 63^3 with
    hifde3x at eps 1e-3 and 1e-6 (Example 4; Table 7 gives |s_L| 578 / 2466
    and 11 / 3 iterations), the 3D high-contrast 127^3 (Example 5 recipe)
    with hifde3, and the 64 independent 2D problems."""
    out = {}
    for eps in (1e-3, 1e-6):
        try:
            r = measure_3d("laplace3d_n64", eps, "hifde3x", "fp32_apply", 1, 1)
            out[f"laplace3d_n64_hifde3x_eps{eps:g}"] = r
        except Exception as exc:
            out[f"laplace3d_n64_hifde3x_eps{eps:g}"] = {"error": repr(exc)}
    try:
        out["contrast3d_n128_hifde3"] = measure_3d("contrast3d_n128", 0.0, "hifde", "fp32_apply", 1, 1)
    except Exception as exc:
        out["contrast3d_n128_hifde3"] = {"error": repr(exc)}
    try:
        out["batched_64x2d"] = measure_batched("fp32_apply", 1, 1)
    except Exception as exc:
        out["batched_64x2d"] = {"error": repr(exc)}
    return out


def run_solve_only(args):
    """Factor the workload and run one 8-RHS solve, this many times: the
    command ncu captures the CG vector kernels and the factor kernels of."""
    import torch
    from paper_1307_2895_gb300 import hif
    hif.load()
    w, f_np = _workload_arrays()
    dev = torch.device("cuda", 0)
    st = torch.cuda.Stream(device=dev)
    a = torch.from_numpy(w["a_stag"]).to(dev)
    b = torch.from_numpy(w["b"]).to(dev)
    f = torch.from_numpy(f_np).to(dev)
    for _ in range(args.ncu_solve):
        G = hif.factor(w["dim"], w["n"], a, b, w["eps"], precision=args.precision, stream=st, autotune=False)
        try:
            x, info = G.solve(f, tol=TOL, maxit=1000)
        finally:
            G.free()
    torch.cuda.synchronize()
    print(json.dumps({"solves": args.ncu_solve, "info": info}))
    return 0


def run_apply_only(args):
    """Factor the workload once and run a number of F^-1 applies (its RHS
    count: 8 for the 2D headline, 4 for the 3D ones): the command ncu captures
    the sweep kernels of.  The built-in launch shapes (no autotuning), so that
    the n-th sweep launch is the same every run; the bytes a launch moves do
    not depend on its shape.  With --workload3d the 3D workload (and
    --variant, --eps) instead of the headline one."""
    import torch
    from paper_1307_2895_gb300 import hif
    hif.load()
    w, f_np = _workload_arrays(args.workload3d or "contrast2d_n512")
    eps = args.eps if (args.workload3d and args.eps > 0) else w["eps"]
    variant = args.variant if args.workload3d else "hifde"
    dev = torch.device("cuda", 0)
    st = torch.cuda.Stream(device=dev)
    a = torch.from_numpy(w["a_stag"]).to(dev)
    b = torch.from_numpy(w["b"]).to(dev)
    f = torch.from_numpy(f_np).to(dev)
    G = hif.factor(w["dim"], w["n"], a, b, eps, precision=args.precision, stream=st, autotune=False,
                   variant=variant)
    try:
        for _ in range(args.ncu_apply):
            G.apply(f)
        torch.cuda.synchronize()
        print(json.dumps({"applies": args.ncu_apply, "stats": G.stats()}))
    finally:
        G.free()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--precision", default="fp32_apply", choices=["fp64", "mixed", "fp32_apply"])
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-others", action="store_true",
                    help="leave out the other configurations (3D 63^3 hifde3x, 127^3, the batched problems)")
    ap.add_argument("--batched", action="store_true",
                    help="time the batched workload (64 independent problems) instead of the headline one")
    ap.add_argument("--workload3d", default="", choices=["", "laplace3d_n64", "contrast3d_n128"],
                    help="time a 3D workload (factor + PCG) instead of the headline one")
    ap.add_argument("--eps", type=float, default=0.0, help="3D workloads: eps (default: the workload's)")
    ap.add_argument("--variant", default="hifde", choices=["hifde", "hifde3x"],
                    help="3D workloads: hifde3 (faces) or hifde3x (faces and edges, Section 4.5)")
    ap.add_argument("--tensor-cores", type=int, default=0, choices=[0, 1, 2, 3, -1],
                    help="mixed precision: 0 or 3 three-part TF32 split, 2 two-part, 1 plain TF32, -1 SIMT FP32")
    ap.add_argument("--tc-roofline", action="store_true",
                    help="time the tensor-core Schur update alone (one JSON line) and exit")
    ap.add_argument("--ncu-solve", type=int, default=0,
                    help="profiling helper: this many factor + 8-RHS solves of the workload, then exit")
    ap.add_argument("--ncu-apply", type=int, default=0,
                    help="profiling helper: factor the workload, then run this many F^-1 applies and exit")
    args = ap.parse_args()
    if args.ncu_apply:
        return run_apply_only(args)
    if args.ncu_solve:
        return run_solve_only(args)
    if args.workload3d:
        return run_3d(args)
    if args.tc_roofline:
        from paper_1307_2895_gb300 import hif
        hif.load()
        print(json.dumps(tc_roofline(split=args.tensor_cores if args.tensor_cores > 0 else 3)), flush=True)
        return 0
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        if args.batched:
            return run_batched(args, rank, world, local_rank)
        return run_gpu(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
