#!/usr/bin/env python3
"""Throughput of the free-BC Poisson solve at 256^3 (FP32) on GB300.

One step = one solve (the five passes: forward x, forward y, z forward +
K^F multiply + inverse, inverse y, inverse x, plus the Hartree energy) of a
256^3 Gaussian-mixture density with free boundary conditions on all axes
(padded FFT 512^3). Inputs are resident in HBM; a 512 MiB buffer is written
between steps so no step starts with its data in L2. The metric is physical
grid points per second (n1 n2 n3 / time per solve) and the fraction of the
HBM roofline of the dominant kernel and of the whole solve.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Other workloads (one JSON line each, same keys):
    --workload free512      512^3 free FP32 (padded FFT 1024^3)
    --workload bc128 --bc B 128^3, B in fff / pff (wire) / ppf (surface) / ppp
                            (--n NX,NY,NZ: another grid with the same recipe)
    --workload hartree192   192^3 free: forward solve + adjoint backward
                            (torch.autograd through ps_solve_vjp) per step
    --workload localpot256  the 256^3 solve with a caller's even kernel
    --workload batched64    64 uneven mixed-BC problems per step
    --dtype f64             FP64 plans (reported against the FP64 ALU roof)

Multi-GPU (torchrun): every rank solves its own density (replicas, weak
scaling, no collective on the data path); rank 0 prints the JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid points/s per Poisson solve (free BCs, 256³) and % of HBM roofline at stated error"
UNIT = "grid points/s"
WORKLOAD = "free256_f32"
FALLBACK_HBM_GBS = 6800.0
NOMINAL_HBM_GBS = 7900.0  # GB300 HBM3e data-sheet bandwidth (context beside the measured peak)
# FP64 arithmetic roof of the GB300: 1.25 TFLOP/s dense FP64 (nominal; the
# FP64 pipe is a small fraction of the FP32 one on this part)
FP64_PEAK_TFLOPS = 1.25
BC_NAMES = {"fff": "free", "pff": "wire", "ppf": "surface", "ppp": "periodic"}
PASS_NAMES = ["p1_fwd_x_r2c", "p2_fwd_y", "p3_z_fwd_mul_inv", "p4_inv_y", "p5_inv_x_c2r"]

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one
# ncu capture of the named kernel on this workload, with the hash of the
# source files that kernel is built from; reported as null once they change.
Z_KERNEL_FILES = ("fast_zsoa.cu", "fft_soa.cuh", "fft_regs.cuh", "fft_fast.cuh", "reduce.cuh", "common.cuh",
                  "../../include/psolver.h")
TRAFFIC = {
    ("p3_z_fwd_mul_inv", "free256_f32"): {"bytes": 367789568 + 221741824, "files": Z_KERNEL_FILES,
                                          "src": "3a25e6ce393611ad"},
}

def _src_hash(files=None):
    """Hash of the CUDA sources (all of them, or the named files)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1211_5244_gb300", "csrc")
    names = files if files is not None else sorted(n for n in os.listdir(csrc) if n.endswith((".cu", ".cuh")))
    for name in names:
        h.update(open(os.path.normpath(os.path.join(csrc, name)), "rb").read())
    return h.hexdigest()[:16]


def _peak_hbm():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return float(json.load(f)["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback (6.8 TB/s, no MEASURED_PEAKS.json)"


def _workload_desc(w, bc="fff", dtype="f32", L=None):
    n = w["n"]
    L = L or [2 * v if b == "f" else v for v, b in zip(n, bc)]
    neutral = ", mean subtracted" if "p" in bc else ""
    return (f"{BC_NAMES.get(bc, bc)}-BC ({bc}) Poisson solve {n[0]}x{n[1]}x{n[2]} {'FP32' if dtype == 'f32' else 'FP64'} "
            f"(padded FFT {L[0]}x{L[1]}x{L[2]}), {w['n_gauss']}-Gaussian density + {w['noise']:g} noise"
            f"{neutral}, h={w['h']}, seed {w['seed']}")


def _paper_unfused_bytes(info, esz):
    """HBM bytes of the paper's separate GPU kernels (§3 step list), each reading
    its input and writing its output once: spread_X, R2C 1DFFT_X, transpose
    (+spread) and 1DFFT_Y, transpose(+spread) and 1DFFT_Z, the kernel
    multiplication (K^F at the full half-spectrum size), and the mirror steps
    of the inverse with compactions. Context for the five fused passes."""
    n, S = list(info.n), list(info.L)
    a, b, c3 = list(info.order)         # the steps in processing order
    free = [bc == 1 for bc in info.bc]
    c = info.c
    N = n[0] * n[1] * n[2]
    r, cx = esz, 2 * esz
    xrows = S[a] * n[b] * n[c3] * r     # padded real rows of the first axis
    A = c * n[b] * n[c3] * cx           # after the first transform
    B = c * S[b] * n[c3] * cx           # after the second
    Z = c * S[b] * S[c3] * cx           # full half spectrum
    one_way = ((N * r + xrows) if free[a] else 0) + (xrows + A) + (A + B) + 2 * B + (B + Z) + 2 * Z
    multiply = 2 * Z + c * S[b] * S[c3] * r
    return 2 * one_way + multiply


def _pass_flops(info):
    """Nominal FLOPs of each pass by the usual FFT benchmark count: 5 L log2 L
    per complex line transform, 2.5 L log2 L per real one, no credit for the
    pruned zero inputs and discarded outputs; the z pass adds its inverse
    transforms and 2 FLOPs per point for the multiply by the real K^F."""
    import math
    out = []
    for k in range(5):
        lines, L = info.lines[k], info.line_len[k]
        per = 5.0 * L * math.log2(max(L, 2))
        if k in (0, 4):
            per *= 0.5
        if k == 2:
            per = 2 * per + 2 * L
        out.append(lines * per)
    return out


def _pass_bytes(info, esz):
    """Algorithmic HBM bytes of each pass (one launch each). Where the x and y
    passes are fused (info.fused), the forward kernel moves rho in and B out
    and the inverse B in and V out; the fused-away passes move nothing."""
    n, L = list(info.n), list(info.L)
    a, b, cx = list(info.order)        # processing order (x, y, z unless the axis rule permutes it)
    c = info.c
    N = n[0] * n[1] * n[2]
    A = c * n[b] * n[cx] * 2 * esz     # complex spectrum after the first pass
    B = c * L[b] * n[cx] * 2 * esz     # after the second pass
    Koct = (L[0] // 2 + 1) * (L[1] // 2 + 1) * (L[2] // 2 + 1) * esz
    if getattr(info, "fused", 0):
        return [N * esz + B, 0, 2 * B + Koct, B + N * esz, 0]
    if getattr(info, "chunks", 1) > 1:  # x and y passes interleaved chunk by chunk: timed together
        return [N * esz + 2 * A + B, 0, 2 * B + Koct, B + 2 * A + N * esz, 0]
    return [N * esz + A, A + B, 2 * B + Koct, B + A, A + N * esz]


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples taken during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
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
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _density(w, rank=0, bc="fff", dtype="f32"):
    import numpy as np
    from paper_1211_5244_gb300 import replicas, synth
    rho = synth.gaussian_mixture(w["n"], w["h"], w["n_gauss"], replicas.replica_seed(w["seed"], rank),
                                 noise=w["noise"], subtract_mean="p" in bc)
    return rho.astype(np.float32 if dtype == "f32" else np.float64)


def _localpot_octant(w):
    """Even kernel of the local-potential workload: a Gaussian of width 2 grid
    steps over the offsets (a stand-in for the convolution kernel of a local
    potential applied to wave functions, §5), on its octant (L/2 + 1)^3."""
    import numpy as np
    d = np.arange(w["n"][0] + 1, dtype=np.float64)
    r2 = d[:, None, None] ** 2 + d[None, :, None] ** 2 + d[None, None, :] ** 2
    return np.exp(-r2 / 8.0)


def _errors(V_gpu, Vo, E_gpu=None, Eo=None, vs="FP64 oracle, full grid"):
    import numpy as np
    err = {"rel_l2": float(np.linalg.norm(V_gpu - Vo) / np.linalg.norm(Vo)),
           "rel_max": float(np.abs(V_gpu - Vo).max() / np.abs(Vo).max()), "vs": vs}
    if E_gpu is not None:
        err["energy_rel"] = float(abs(E_gpu - Eo) / abs(Eo))
    return err


def _host_cpu():
    """(nproc, CPU model) of the host the oracle runs on."""
    import platform
    nproc = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return nproc, model or platform.processor() or platform.machine()


def _oracle_workers(n, bc, cap=64):
    """Concurrent oracle processes the host holds: one per core, at most as
    many as fit in 60% of the available memory (a solve keeps about four
    copies of the padded complex grid and the padded K^F)."""
    L = [2 * v if b == "f" else v for v, b in zip(n, bc)]
    per_gb = 16.0 * L[0] * L[1] * L[2] * 4 / 1e9 + 1.0
    k = min(os.cpu_count() or 1, cap)
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                k = min(k, max(1, int(0.6 * int(line.split()[1]) / 1e6 / per_gb)))
                break
    except Exception:
        pass
    return max(1, k)


def _oracle_worker(task, barrier, out_q):
    """One spawned oracle process: builds K^F and its densities (untimed), runs
    its untimed warm-up solves, waits for the other processes, then times its
    solves; puts (start, end, solves) on out_q (wall clock)."""
    import numpy as np
    from oracle import poisson as op
    from paper_1211_5244_gb300 import synth
    n, bc, h, n_gauss, noise, seeds, warm = task
    KF = op.kernel_fourier(n, bc, h)
    rhos = [synth.gaussian_mixture(n, h, n_gauss, sd, noise=noise, subtract_mean="p" in bc)
            .astype(np.float32).astype(np.float64) for sd in seeds]
    for i in range(warm):
        op.solve(rhos[i % len(rhos)], bc, h, KF=KF)
    barrier.wait()
    t0 = time.time()
    for r in rhos:
        op.solve(r, bc, h, KF=KF)
    out_q.put((t0, time.time(), len(rhos)))


def _oracle_concurrent(w, bc, nsolves, workers, warmup=0):
    """`nsolves` oracle solves of independently seeded densities of the
    workload, spread over `workers` spawned processes (one per core) that
    start together; returns (points/s over the whole run, wall seconds,
    processes used)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    workers = max(1, min(workers, nsolves))
    barrier = ctx.Barrier(workers)
    q = ctx.Queue()
    procs = []
    for k in range(workers):
        seeds = [w["seed"] + 1000 + i for i in range(k, nsolves, workers)]
        warm = len(range(k, warmup, workers))
        task = (tuple(w["n"]), bc, w["h"], w["n_gauss"], w["noise"], seeds, warm)
        pr = ctx.Process(target=_oracle_worker, args=(task, barrier, q))
        pr.start()
        procs.append(pr)
    res = [q.get() for _ in procs]
    for pr in procs:
        pr.join()
    wall = max(r[1] for r in res) - min(r[0] for r in res)
    done = sum(r[2] for r in res)
    npts = int(w["n"][0]) * int(w["n"][1]) * int(w["n"][2])
    return done * npts / wall, wall, workers


def _oracle_item(args):
    """One oracle solve (a pool task): (V, E) of a density in FP64."""
    from oracle import poisson as op
    rho, bc, h = args
    return op.solve(rho, bc, h)


def _oracle_baseline(w, bc, rho_in, V_gpu, E_gpu, kernel=None, max_full=256):
    """The FP64 oracle as it stands, timed on the host on one full solve of the
    workload (K^F built before the timed region, like the GPU's kernel build),
    and the GPU result's error against it. Grids above ``max_full`` per axis
    are too large for a full oracle solve within the bench: the oracle is then
    timed on the same recipe at max_full^3 and the error is taken on sampled
    points of Eq. 2 evaluated directly (free BCs)."""
    import numpy as np
    from oracle import poisson as op
    from paper_1211_5244_gb300 import synth
    rho = rho_in.astype(np.float64)
    full = max(w["n"]) <= max_full
    if full:
        rs, ns = rho, w["n"]
    else:
        ns = (max_full,) * 3
        rs = synth.gaussian_mixture(ns, w["h"], w["n_gauss"], w["seed"], noise=w["noise"],
                                    subtract_mean="p" in bc).astype(rho_in.dtype).astype(np.float64)
    KF = (op.kernel_fourier(ns, bc, w["h"]) if kernel is None
          else op.kernel_fourier_from_real(kernel, ns, bc))
    t0 = time.perf_counter()
    Vo, Eo = op.solve(rs, bc, w["h"], KF=KF)
    dt = time.perf_counter() - t0
    Ls = "x".join(str(2 * v if b == "f" else v) for v, b in zip(ns, bc))
    nproc, model = _host_cpu()
    one = {"value": rs.size / dt, "cores": 1,
           "sample": f"one full {ns[0]}x{ns[1]}x{ns[2]} {bc} oracle solve (numpy FFT of the padded "
                     f"{Ls} grid, FP64, single thread), {dt:.1f} s; K^F built untimed"
                     + ("" if full else f"; a bounded sample of the {w['n'][0]}^3 workload (same recipe)")}
    base = {"value": one["value"], "unit": UNIT, "cores": 1, "kind": "oracle", "sample": one["sample"],
            "nproc": nproc, "cpu_model": model, "single_core": one}
    if kernel is None:
        # all cores: one oracle process per core (as many as the memory holds),
        # each solving its own seeded density of the same recipe and size
        try:
            wk = _oracle_workers(ns, bc)
            v_all, wall, wk = _oracle_concurrent(dict(w, n=ns), bc, wk, wk)
            base["all_cores"] = {"value": v_all, "cores": wk,
                                 "sample": f"{wk} concurrent oracle processes (spawned, one per core, as many "
                                           f"as 60% of the host memory holds), one full {ns[0]}x{ns[1]}x{ns[2]} "
                                           f"solve each, {wall:.1f} s wall; K^F built untimed"}
        except Exception as exc:  # the single-core figure stands on its own
            base["all_cores"] = {"value": None, "error": f"{type(exc).__name__}: {exc}"}
    if full:
        return base, _errors(V_gpu, Vo, E_gpu, Eo), (Vo, Eo)
    assert bc == "fff" and kernel is None
    n1, n2, n3 = w["n"]
    rng = np.random.default_rng(7)
    pts = [(n3 // 2, n2 // 2, n1 // 2), (0, 0, 0), (n3 - 1, n2 - 1, n1 - 1)]
    pts += [tuple(int(v) for v in rng.integers(0, [n3, n2, n1])) for _ in range(3)]
    ref = op.direct_at(rho, w["h"], pts)
    got = np.array([V_gpu[p] for p in pts])
    scale = np.abs(V_gpu).max()
    err = {"rel_max_sampled": float(np.abs(got - ref).max() / scale),
           "points": len(pts), "vs": "Eq. 2 summed directly in FP64 at sampled points (relative to max|V|)"}
    return base, err, None


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, on this arm's own
    workload (256^3 free BCs, the same recipe). Each step is one full oracle
    solve of an independently seeded density; the W warm-up and K timed solves
    are spread over one spawned process per core (as many as the host memory
    holds), which start together. When the timed solves would take more than
    about three minutes at that concurrency, fewer are timed and the line says
    how many."""
    from paper_1211_5244_gb300 import synth
    from paper_1211_5244_gb300 import replicas
    rank, world, _ = replicas.dist_env()
    if rank != 0:
        return
    w = dict(synth.WORKLOADS[WORKLOAD])
    workers = _oracle_workers(w["n"], "fff")
    # about 8 s per 256^3 solve and core on the GPU hosts measured so far
    est_s = 8.0 * -(-(args.steps + args.warmup) // workers)
    steps = args.steps if est_s <= 180 else max(1, int(180 / 8.0) * workers - args.warmup)
    value, wall, workers = _oracle_concurrent(w, "fff", steps, workers, warmup=min(args.warmup, workers))
    nproc, model = _host_cpu()
    sample = (f"each step one full FP64 oracle solve of a 256^3 free-BC density of the workload's recipe "
              f"(numpy FFT of the padded 512^3 grid, K^F built untimed), {steps} timed solves over {workers} "
              f"concurrent spawned processes (one per core), {wall:.1f} s wall")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": _workload_desc(w), "bc": "fff", "n": list(w["n"])},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": workers, "kind": "oracle", "sample": sample,
                             "nproc": nproc, "cpu_model": model},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    if steps != args.steps:
        line["note"] = f"{steps} of the {args.steps} requested steps timed (each is a full 256^3 oracle solve)"
    print(json.dumps(line), flush=True)


def _batched_measure(K, W, rank=0, dist=None, with_oracle=False):
    """The uneven batch: 64 problems (n ~ U{24..160} per axis, BC uniform over
    free, wire, surface, periodic; FP32), autotuned plans, one
    ps_solve_batched per step, an L2 flush before every step. Returns the
    measured object (and each item's error against the FP64 oracle when asked:
    the oracle solves run on spawned processes, one per core)."""
    import numpy as np
    import torch
    from paper_1211_5244_gb300 import psolver, replicas, synth
    w = synth.WORKLOADS["batched64"]
    shapes = synth.batched_shapes(w["count"], w["nmin"], w["nmax"], w["seed"])
    tune = not os.environ.get("PS_BENCH_NO_TUNE")
    t_tune = time.perf_counter()
    plans, rhos, rnp = [], [], []
    for i, (n, bc) in enumerate(shapes):
        plans.append(psolver.Plan(n, bc, w["h"], "f32", autotune=tune))
        r = synth.gaussian_mixture(n, w["h"], w["n_gauss"], replicas.replica_seed(w["seed"] + 1000 * (rank + 1), i),
                                   noise=w["noise"], subtract_mean="p" in bc).astype(np.float32)
        rnp.append(r)
        rhos.append(torch.from_numpy(r).cuda())
    t_tune = time.perf_counter() - t_tune
    Vs = [torch.empty_like(r) for r in rhos]
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(W):
        flush.zero_()
        psolver.solve_batched(plans, rhos, Vs, stream=stream)
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    replicas.barrier(dist)
    torch.cuda.synchronize()
    E = None
    for i in range(K):
        flush.zero_()
        starts[i].record(stream)
        _, E = psolver.solve_batched(plans, rhos, Vs, stream=stream)
        ends[i].record(stream)
    torch.cuda.synchronize()
    replicas.barrier(dist)
    npts = sum(int(np.prod(n)) for n, _ in shapes)
    value, total_s = replicas.aggregate(sum(s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)) / 1e3,
                                        npts * K, dist, device="cuda")
    ms = total_s * 1e3 / K
    alg = sum(p.info().alg_bytes for p in plans)
    peak, peak_src = _peak_hbm()
    out = {"ms_per_batch": ms, "value": value, "unit": UNIT, "points": npts,
           "workload": f"64 problems, n ~ U{{24..160}} per axis, BC uniform over fff/pff/ppf/ppp, FP32, "
                       f"seed {w['seed']}, autotuned={tune}",
           "lengths": [list(p.info().L) for p in plans], "autotune_s": t_tune,
           "solve_roofline": {"alg_bytes": alg, "achieved": alg / (ms / 1e3) / 1e9, "peak": peak,
                              "unit": "GB/s", "frac": alg / (ms / 1e3) / 1e9 / peak, "peak_source": peak_src},
           "gpu_launches": sum(p.info().launches for p in plans) * K}
    if with_oracle:
        import multiprocessing as mp
        jobs = [(r.astype(np.float64), bc, w["h"]) for r, (_, bc) in zip(rnp, shapes)]
        with mp.get_context("spawn").Pool(min(os.cpu_count() or 1, 16)) as pool:
            ref = pool.map(_oracle_item, jobs, chunksize=1)
        Eh = E.double().cpu().numpy()
        worst = {"rel_l2": 0.0, "rel_max": 0.0, "energy_rel": 0.0}
        for (Vo, Eo), V, e in zip(ref, Vs, Eh):
            err = _errors(V.double().cpu().numpy(), Vo, float(e), Eo)
            for k in worst:
                worst[k] = max(worst[k], err[k])
        worst["vs"] = "FP64 oracle, every item, full grids (worst over the 64 items)"
        out["error_vs_oracle"] = worst
    return out


def run_batched(args):
    """--workload batched64: the uneven batch as its own JSON line. The metric
    is total physical points per second of the batch."""
    import torch
    from paper_1211_5244_gb300 import build as _build
    from paper_1211_5244_gb300 import replicas
    rank, world, local = replicas.dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    sampler = ClockSampler(local)
    sampler.start()
    b = _batched_measure(args.steps, args.warmup, rank, dist,
                         with_oracle=(rank == 0 and world == 1 and not args.no_cpu_baseline))
    clocks = sampler.stop()
    line = {"metric": "grid points/s of a batch of 64 uneven mixed-BC Poisson solves", "value": b["value"],
            "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": b["ms_per_batch"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": b["workload"], "points": b["points"], "lengths": b["lengths"]},
            "solve_roofline": b["solve_roofline"], "gpu_launches": b["gpu_launches"], "clocks": clocks}
    if "error_vs_oracle" in b:
        line["error_vs_oracle"] = b["error_vs_oracle"]
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _spec(args):
    """(workload parameters, bc, description suffix, caller's kernel) of a solve workload."""
    from paper_1211_5244_gb300 import synth
    if args.workload in (WORKLOAD, "localpot256"):
        w, bc = dict(synth.WORKLOADS[WORKLOAD]), "fff"
    elif args.workload == "free512":
        w, bc = dict(synth.WORKLOADS["free512_f32"]), "fff"
    elif args.workload == "hartree192":
        w, bc = dict(synth.WORKLOADS["hartree192_f32"]), "fff"
    else:
        w0 = synth.WORKLOADS["bc128"]
        if len(args.bc) != 3 or any(b not in "pf" for b in args.bc):
            raise SystemExit("--bc must name the x, y, z axes with p / f, e.g. pff")
        w, bc = {k: w0[k] for k in ("n", "h", "n_gauss", "noise", "seed")}, args.bc
        if args.n:
            n = tuple(int(v) for v in args.n.split(","))
            if len(n) != 3 or min(n) < 2:
                raise SystemExit("--n must give three sizes >= 2, e.g. 128,128,512")
            w["n"] = n
    kernel = _localpot_octant(w) if args.workload == "localpot256" else None
    return w, bc, kernel


def _timed_steps(step, K, flush, stream, sampler, dist):
    """K steps, each after an L2 flush, with CUDA events around the step on the
    solve stream; returns per-step ms and the clock record."""
    import torch
    from paper_1211_5244_gb300 import replicas
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    replicas.barrier(dist)
    torch.cuda.synchronize()
    if sampler is not None:
        sampler.start()
        time.sleep(0.2)
    for i in range(K):
        flush.zero_()
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    replicas.barrier(dist)
    clocks = sampler.stop() if sampler is not None else None
    return [s_.elapsed_time(e_) for s_, e_ in zip(starts, ends)], clocks


def _rooflines(info, pass_ms, dtype, workload, math_mode):
    """The dominant kernel's roofline (HBM bytes for FP32, FP64 ALU for FP64 plans)
    and the per-pass table."""
    peak, peak_src = _peak_hbm()
    esz = 4 if dtype == "f32" else 8
    pbytes = _pass_bytes(info, esz)
    pflops = _pass_flops(info)
    if getattr(info, "fused", 0) or getattr(info, "chunks", 1) > 1:  # two passes per timed entry
        pflops = [pflops[0] + pflops[1], 0.0, pflops[2], pflops[3] + pflops[4], 0.0]
    dom = max(range(5), key=lambda k: pass_ms[k])
    fused = getattr(info, "fused", 0)
    if getattr(info, "chunks", 1) > 1:
        fused = (1 << 1) | (1 << 4)  # interleaved in chunks: x and y of one direction timed together
    passes = {}
    for k in range(5):
        if fused & (1 << k):
            key = "fused_into" if getattr(info, "fused", 0) else "timed_with"
            passes[PASS_NAMES[k]] = {key: PASS_NAMES[k - 1 if k == 1 else 3], "ms": pass_ms[k]}
            continue
        passes[PASS_NAMES[k]] = {"ms": pass_ms[k], "alg_bytes": pbytes[k],
                                 "GB/s": pbytes[k] / (pass_ms[k] / 1e3) / 1e9,
                                 "frac_hbm": pbytes[k] / (pass_ms[k] / 1e3) / 1e9 / peak,
                                 "nominal_flops": pflops[k],
                                 "TFLOP/s": pflops[k] / (pass_ms[k] / 1e3) / 1e12}
    if dtype == "f32":
        achieved = pbytes[dom] / (pass_ms[dom] / 1e3) / 1e9
        tr = TRAFFIC.get((PASS_NAMES[dom], workload))
        traffic = tr["bytes"] if (tr and math_mode == "cudacore" and tr["src"] == _src_hash(tr["files"])) else None
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": PASS_NAMES[dom], "alg_bytes_per_launch": pbytes[dom],
                "peak_source": peak_src}
    else:
        achieved = pflops[dom] / (pass_ms[dom] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None, "kernel": PASS_NAMES[dom],
                "nominal_flops_per_launch": pflops[dom],
                "peak_source": "nominal dense FP64 of the GB300 (1.25 TFLOP/s); FLOPs by the 5 L log2 L count",
                "hbm_frac": pbytes[dom] / (pass_ms[dom] / 1e3) / 1e9 / peak}
    return roof, passes


def run_hartree(args):
    """Differentiable Hartree energy at 192^3 free (padded 384^3 = 2^7 3 per
    axis): each step is the forward solve (V, E) through the autograd
    function and the backward pass with incoming gradients (Vbar, 1) on (V, E),
    i.e. rhobar = K Vbar + h^3 V through ps_solve_vjp (an adjoint solve and the
    energy term's axpy). Metric: grid points per second of forward + backward
    steps."""
    import numpy as np
    import torch
    from paper_1211_5244_gb300 import build as _build
    from paper_1211_5244_gb300 import psolver, replicas, synth
    from paper_1211_5244_gb300.autograd import hartree
    rank, world, local = replicas.dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()
    w, bc, _ = _spec(args)
    dt = args.dtype
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    K = args.steps
    h = _hartree_setup(w, bc, dt, not args.no_autotune, rank)
    plan, info, step, out, rho_np, vbar_np = h["plan"], h["info"], h["step"], h["out"], h["rho_np"], h["vbar_np"]
    gE = h["gE"]
    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    step_ms, clocks = _timed_steps(step, K, flush, stream, ClockSampler(local), dist)
    npts = int(np.prod(w["n"]))
    value, total_s = replicas.aggregate(sum(step_ms) / 1e3, K * npts, dist, device="cuda")
    ms_per_step = total_s * 1e3 / K

    plan.set_profiling(True)
    plan.pass_times()
    for _ in range(K):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    plan.set_profiling(False)
    pass_ms, nrec = plan.pass_times()
    pass_ms = [t / max(nrec, 1) for t in pass_ms]   # per solve (forward and adjoint alike)
    roof, passes = _rooflines(info, pass_ms, dt, args.workload, "cudacore")
    peak, _ = _peak_hbm()
    esz = 4 if dt == "f32" else 8
    step_bytes = 2 * info.alg_bytes + 3 * npts * esz      # two solves + the axpy (read 2, write 1)
    gbs = step_bytes / (ms_per_step / 1e3) / 1e9

    # end to end through the public API from pinned host memory: upload rho and
    # Vbar, forward + backward, download V, E and the gradient
    rho_h = torch.from_numpy(rho_np).pin_memory()
    vbar_h = torch.from_numpy(vbar_np).pin_memory()
    V_h = torch.empty_like(rho_h).pin_memory()
    g_h = torch.empty_like(rho_h).pin_memory()
    E_h = torch.empty((), dtype=torch.float64).pin_memory()

    def e2e_step():
        r = rho_h.to("cuda", non_blocking=True).requires_grad_(True)
        vb = vbar_h.to("cuda", non_blocking=True)
        V, E = hartree(r, plan)
        torch.autograd.backward([E, V], [gE, vb])
        V_h.copy_(V, non_blocking=True)
        g_h.copy_(r.grad, non_blocking=True)
        E_h.copy_(E, non_blocking=True)
    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    replicas.barrier(dist)
    t0 = time.perf_counter()
    for _ in range(K):
        e2e_step()
    torch.cuda.synchronize()
    e2e_value, _ = replicas.aggregate(time.perf_counter() - t0, K * npts, dist, device="cuda")
    e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 2 * npts * esz,
           "d2h_bytes_per_step": 2 * npts * esz + 8,
           "api": "torch.autograd through hartree() (ps_solve + ps_solve_vjp), pinned host buffers, host wall clock"}

    line = {
        "metric": "grid points/s of a differentiable Hartree step (forward solve + adjoint backward)",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": dt, "data": "synthetic",
        "config": {"workload": _workload_desc(w, bc, dt, list(info.L)) +
                   "; step = forward (V, E) + backward with (Vbar, 1) through ps_solve_vjp",
                   "n": list(w["n"]), "bc": bc, "h": w["h"], "L": list(info.L), "autotuned": not args.no_autotune,
                   "blocks": list(info.blocks),
                   "l2": "flushed (512 MiB write) before every step; per-step CUDA events",
                   "pass_times": "separate profiled loop, per solve (forward and adjoint solves averaged)",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": roof,
        "solve_roofline": {"alg_bytes": step_bytes, "achieved": gbs, "peak": peak, "unit": "GB/s",
                           "frac": gbs / peak, "per": "step (two solves + the energy term's axpy)"},
        "passes": passes, "e2e": e2e, "gpu_launches": (2 * info.launches + 1) * K, "clocks": clocks,
        "kernel_src": _src_hash(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"], line["error_vs_oracle"] = _hartree_oracle(w, bc, rho_np, vbar_np, out)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _hartree_setup(w, bc, dt, autotune, rank):
    """The plan, densities and step function of the differentiable Hartree
    workload: one step is the forward solve (V, E) through the autograd
    function and the backward pass with incoming gradients (Vbar, 1)."""
    import torch
    from paper_1211_5244_gb300 import psolver
    from paper_1211_5244_gb300.autograd import hartree
    rho_np = _density(w, rank, bc, dt)
    vbar_np = _density(dict(w, seed=w["seed"] + 77), rank, bc, dt)
    rho = torch.from_numpy(rho_np).cuda()
    vbar = torch.from_numpy(vbar_np).cuda()
    gE = torch.ones((), dtype=torch.float64, device="cuda")
    # the free-axis lengths are the autotuner's choice among 2n, the smallest
    # 2-, 2*3- and 2*3*5*7-smooth lengths >= 2n - 1 and the smallest one with
    # register kernels (all give the same result); without it L = 2n (384 =
    # 2^7 * 3 at n = 192)
    plan = psolver.Plan(w["n"], bc, w["h"], dt, autotune=autotune)
    out = {}

    def step():
        r = rho.detach().requires_grad_(True)
        V, E = hartree(r, plan)
        torch.autograd.backward([E, V], [gE, vbar])
        out["V"], out["E"], out["g"] = V, E, r.grad

    return {"plan": plan, "info": plan.info(), "step": step, "out": out, "rho_np": rho_np, "vbar_np": vbar_np,
            "gE": gE}


def _hartree_oracle(w, bc, rho_np, vbar_np, out):
    """The FP64 oracle's forward + backward step on the same densities, timed
    on one host core, and the GPU step's errors against it (V, E, gradient)."""
    import numpy as _np
    from oracle import poisson as op
    r64 = rho_np.astype(_np.float64)
    vb64 = vbar_np.astype(_np.float64)
    KF = op.kernel_fourier(w["n"], bc, w["h"])
    t0 = time.perf_counter()
    Vo, Eo = op.solve(r64, bc, w["h"], KF=KF)
    KVb, _ = op.solve(vb64, bc, w["h"], KF=KF)
    go = KVb + w["h"] ** 3 * Vo
    tcpu = time.perf_counter() - t0
    npts = int(_np.prod(w["n"]))
    base = {"value": npts / tcpu, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one full forward + backward step in the FP64 oracle (two numpy FFT "
                      f"solves of the padded grid and the energy term), single thread, "
                      f"{tcpu:.1f} s; K^F built untimed"}
    err = _errors(out["V"].detach().double().cpu().numpy(), Vo, float(out["E"].item()), Eo)
    gerr = _errors(out["g"].detach().double().cpu().numpy(), go)
    err["grad_rel_l2"], err["grad_rel_max"] = gerr["rel_l2"], gerr["rel_max"]
    return base, err


def _hartree_measure(K, W, flush, stream, rank, dist, with_oracle):
    """The 192^3 differentiable Hartree workload (forward + adjoint backward,
    autotuned lengths) for the headline line: ms per step with the same timing
    rules, and the errors of V, E and the gradient against the FP64 oracle."""
    import numpy as np
    import torch
    from paper_1211_5244_gb300 import replicas, synth
    w, bc, dt = dict(synth.WORKLOADS["hartree192_f32"]), "fff", "f32"
    h = _hartree_setup(w, bc, dt, True, rank)
    for _ in range(W):
        flush.zero_()
        h["step"]()
    torch.cuda.synchronize()
    step_ms, _ = _timed_steps(h["step"], K, flush, stream, None, dist)
    npts = int(np.prod(w["n"]))
    value, total_s = replicas.aggregate(sum(step_ms) / 1e3, K * npts, dist, device="cuda")
    ms = total_s * 1e3 / K
    info = h["info"]
    peak, _ = _peak_hbm()
    step_bytes = 2 * info.alg_bytes + 3 * npts * 4
    res = {"ms_per_step": ms, "value": value, "unit": UNIT, "L": list(info.L),
           "workload": _workload_desc(w, bc, dt, list(info.L)) + "; step = forward (V, E) + backward with "
                       "(Vbar, 1) through ps_solve_vjp, autotuned lengths",
           "step_roofline": {"alg_bytes": step_bytes, "frac": step_bytes / (ms / 1e3) / 1e9 / peak,
                             "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}}
    if with_oracle:
        _, res["error_vs_oracle"] = _hartree_oracle(w, bc, h["rho_np"], h["vbar_np"], h["out"])
    return res


def _tf32x3_measure(w, bc, rho, K, W, flush, stream, dist, ref):
    """One solve per step of the same density with PS_MATH_TF32X3 (the z pass's
    32-point stages as tcgen05 TF32 MMAs on split operands): per-step CUDA
    events after an L2 flush, the per-pass times of a second loop, and the
    error against the FP64 oracle's solve of the same density."""
    import torch
    from paper_1211_5244_gb300 import psolver, replicas
    plan = psolver.Plan(w["n"], bc, w["h"], "f32", math="tf32x3")
    info = plan.info()
    V = torch.empty_like(rho)
    E = torch.empty((), dtype=torch.float64, device="cuda")

    def step():
        plan.solve(rho, V, stream=stream, E=E)

    for _ in range(W):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    replicas.barrier(dist)
    for i in range(K):
        flush.zero_()
        starts[i].record(stream)
        step()
        ends[i].record(stream)
    torch.cuda.synchronize()
    npts = int(w["n"][0]) * int(w["n"][1]) * int(w["n"][2])
    value, total_s = replicas.aggregate(sum(a.elapsed_time(b) for a, b in zip(starts, ends)) / 1e3, K * npts, dist,
                                        device="cuda")
    ms = total_s * 1e3 / K
    plan.set_profiling(True)
    plan.pass_times()
    for _ in range(K):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    plan.set_profiling(False)
    pass_ms, nrec = plan.pass_times()
    pass_ms = [t / max(nrec, 1) for t in pass_ms]
    plan.device_status()
    peak, _ = _peak_hbm()
    zb = _pass_bytes(info, 4)[2]
    out = {"ms_per_step": ms, "value": value, "unit": UNIT, "tensor_passes": info.tensor_passes,
           "z_pass_ms": pass_ms[2], "z_frac_hbm": zb / (pass_ms[2] / 1e3) / 1e9 / peak,
           "solve_frac_hbm": info.alg_bytes / (ms / 1e3) / 1e9 / peak, "pass_ms": pass_ms,
           "note": "z pass as tcgen05 TF32 MMAs with hi/lo operand splits (FP32 accumulation)"}
    if ref is not None:
        out["error_vs_oracle"] = _errors(V.double().cpu().numpy(), ref[0], float(E.item()), ref[1])
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline line without its tf32x3, batched64 and hartree192 objects")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "free512", "bc128", "hartree192", "localpot256", "batched64"],
                    help="localpot256: the 256^3 free solve with a caller's even kernel (ps_kernel_set_real)")
    ap.add_argument("--bc", default="fff",
                    help="boundary conditions of --workload bc128, x y z: any of the 8 assignments (fff, pff, fpf, "
                         "ffp, ppf, pfp, fpp, ppp)")
    ap.add_argument("--xy", type=int, default=0, choices=[0, 1],
                    help="1: the fused x/y kernels (thread-block clusters) where the shapes have them")
    ap.add_argument("--chunks", type=int, default=0,
                    help="chunks of z planes for the x and y passes (0: the plan's default)")
    ap.add_argument("--order", default="rule", choices=["rule", "xfirst"],
                    help="axis processing order: the paper's rule (periodic axes first) or x, y, z")
    ap.add_argument("--n", default="",
                    help="grid of --workload bc128 as NX,NY,NZ (default 128,128,128)")
    ap.add_argument("--dtype", default="f32", choices=["f32", "f64"])
    ap.add_argument("--no-autotune", action="store_true",
                    help="hartree192: padded lengths 2n instead of the autotuner's choice")
    ap.add_argument("--math", default="cudacore", choices=["cudacore", "tf32x3"],
                    help="arithmetic of the transforms (tf32x3: z pass on the tensor cores)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batched64":
        run_batched(args)
        return
    if args.workload == "hartree192":
        run_hartree(args)
        return

    import numpy as np
    import torch

    from paper_1211_5244_gb300 import build as _build
    from paper_1211_5244_gb300 import psolver, replicas

    rank, world, local = replicas.dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    _build.build()

    w, bc, kernel = _spec(args)
    dt = args.dtype
    esz = 4 if dt == "f32" else 8
    rho_np = _density(w, rank, bc, dt)
    rho = torch.from_numpy(rho_np).cuda()
    plan = psolver.Plan(w["n"], bc, w["h"], dt, math=args.math,
                        order=(0, 1, 2) if args.order == "xfirst" else None,
                        schedule=({"chunks": args.chunks, "xy": args.xy} if (args.chunks or args.xy) else None))
    if kernel is not None:
        plan.set_kernel_real(kernel)
    info = plan.info()
    V = torch.empty_like(rho)
    E = torch.empty((), dtype=torch.float64, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        plan.solve(rho, V, stream=stream, E=E)

    for _ in range(args.warmup):
        flush.zero_()
        step()
    torch.cuda.synchronize()

    # ---- timed region (device-resident inputs) ----
    K = args.steps
    step_ms, clocks = _timed_steps(step, K, flush, stream, ClockSampler(local), dist)
    npts = int(np.prod(w["n"]))
    value, total_s = replicas.aggregate(sum(step_ms) / 1e3, K * npts, dist, device="cuda")
    ms_per_step = total_s * 1e3 / K

    # ---- per-pass times: the same steps again with an event between passes
    # (passes serialised on the solve stream), for the per-kernel roofline
    plan.set_profiling(True)
    plan.pass_times()  # forget anything recorded earlier
    for i in range(K):
        flush.zero_()
        step()
    torch.cuda.synchronize()
    plan.set_profiling(False)
    pass_ms, nrec = plan.pass_times()
    pass_ms = [t / max(nrec, 1) for t in pass_ms]

    # ---- the same steps without the L2 flush (context: at 128^3 and below the
    # working set of a solve fits in the 129 MB L2)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for i in range(K):
        step()
    ev1.record(stream)
    torch.cuda.synchronize()
    unflushed_ms = ev0.elapsed_time(ev1) / K

    # ---- end-to-end through the host-buffer entry point (pinned memory): K
    # densities, each uploaded, solved and downloaded (with its energy), the
    # transfers of one density overlapped with the solves of its neighbours
    rho_host = torch.from_numpy(rho_np).pin_memory()
    V_hosts = [torch.empty_like(rho_host).pin_memory() for _ in range(2)]
    plan.solve_host_stream([rho_host] * 4, [V_hosts[i % 2] for i in range(4)])
    replicas.barrier(dist)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan.solve_host_stream([rho_host] * K, [V_hosts[i % 2] for i in range(K)])
    torch.cuda.synchronize()
    e2e_value, _ = replicas.aggregate(time.perf_counter() - t0, K * npts, dist, device="cuda")
    e2e = {"value": e2e_value, "unit": UNIT,
           "h2d_bytes_per_step": npts * esz, "d2h_bytes_per_step": npts * esz + 8,
           "api": "ps_solve_host_stream (pinned host buffers, host wall clock)"}

    # ---- roofline ----
    wl_key = WORKLOAD if (args.workload == WORKLOAD and dt == "f32") else args.workload
    roof, passes = _rooflines(info, pass_ms, dt, wl_key, args.math)
    peak, _ = _peak_hbm()
    solve_gbs = info.alg_bytes / (ms_per_step / 1e3) / 1e9
    n = w["n"]
    compulsory = 2 * npts * esz + info.c * (info.L[1] // 2 + 1) * (info.L[2] // 2 + 1) * esz

    desc = _workload_desc(w, bc, dt, list(info.L))
    if kernel is not None:
        desc += "; caller's kernel: Gaussian of width 2 steps (ps_kernel_set_real)"
    line = {
        "metric": METRIC if (args.workload in (WORKLOAD, "localpot256") and dt == "f32")
        else f"grid points/s per Poisson solve ({BC_NAMES.get(bc, bc)} BCs, {n[0]}x{n[1]}x{n[2]}, {dt.upper()})",
        "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "ms_median": statistics.median(step_ms),
        "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dt, "data": "synthetic",
        "config": {"workload": desc, "n": list(n), "bc": bc, "h": w["h"], "L": list(info.L),
                   "order": "".join("xyz"[a] for a in info.order), "chunks": info.chunks,
                   "math": args.math, "tensor_passes": info.tensor_passes, "blocks": list(info.blocks),
                   "l2": "flushed (512 MiB write) before every step; per-step CUDA events",
                   "pass_times": "separate profiled loop of the same K steps, one event between passes",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": roof,
        "solve_roofline": {"alg_bytes": info.alg_bytes, "achieved": solve_gbs, "peak": peak,
                           "unit": "GB/s", "frac": solve_gbs / peak,
                           "compulsory_bytes": compulsory,
                           "compulsory_frac": compulsory / (ms_per_step / 1e3) / 1e9 / peak,
                           "frac_of_nominal": solve_gbs / NOMINAL_HBM_GBS,
                           "paper_unfused_bytes": _paper_unfused_bytes(info, esz)},
        "l2_unflushed": {"ms_per_step": unflushed_ms, "value": npts / (unflushed_ms / 1e3),
                         "note": "the same K steps back to back without the L2 flush (not the headline)"},
        "passes": passes,
        "e2e": e2e,
        "gpu_launches": info.launches * K,
        "clocks": clocks,
        "kernel_src": _src_hash(),
    }
    ref = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base, err, ref = _oracle_baseline(w, bc, rho_np, V.double().cpu().numpy(), float(E.item()), kernel)
        line["cpu_baseline"] = base
        line["error_vs_oracle"] = err
    headline = args.workload == WORKLOAD and dt == "f32" and args.math == "cudacore"
    if headline and not args.no_extras:
        # the same workload with the z pass on the tensor cores (TF32 split
        # products), timed the same way, and its error against the same oracle;
        # then the uneven batched workload, every item against the oracle. A
        # failure in either is reported in its object; the headline stands.
        try:
            line["tf32x3"] = _tf32x3_measure(w, bc, rho, K, args.warmup, flush, stream, dist, ref)
        except Exception as exc:
            line["tf32x3"] = {"error": f"{type(exc).__name__}: {exc}"}
        try:
            line["batched64"] = _batched_measure(K, args.warmup, rank, dist,
                                                 with_oracle=(rank == 0 and world == 1 and not args.no_cpu_baseline))
        except Exception as exc:
            line["batched64"] = {"error": f"{type(exc).__name__}: {exc}"}
        try:
            line["hartree192"] = _hartree_measure(min(K, 50), args.warmup, flush, stream, rank, dist,
                                                  with_oracle=(rank == 0 and world == 1
                                                               and not args.no_cpu_baseline))
        except Exception as exc:
            line["hartree192"] = {"error": f"{type(exc).__name__}: {exc}"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
