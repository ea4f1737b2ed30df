#!/usr/bin/env python
"""Benchmark of the joint p0 / speed-of-sound reconstruction hot path on GB300.

Headline: gradient evaluations per second (one step = one call of
pat_adjoint_grad: forward solve with checkpoints every s = 32 steps, residual
and objective, segment recompute and time-reversed adjoint accumulating
dJ/dp0_k and dJ/dc over the K data sets) on the 256 x 256 domain (300 x 300
FFT grid with a 22-cell PML), K = 8 vessel-like p0 sets, 512 sensors on a
circle, Nt = 1800, FP32.  Inputs are seeded synthetic stand-ins for the
paper's phantoms (pat_synth).

Also reported: forward-only Gcell-steps/s (Ng^2 K (Nt-1) / s), an
end-to-end number through host buffers (H2D of c, p0, data, weights and D2H
of both gradients and J inside the timed region), the roofline of the
dominant kernel (algorithmic bytes per launch / average launch time from
CUDA events on the launching stream), SM clocks sampled during the timed
region and the FP64 oracle timed on the host cores on a bounded sample.

``--impl reference`` times the FP64 oracle (the only reference: the paper
ships no code) on the same workload, on bounded samples scaled to the metric.

Multi-GPU (torchrun): every rank solves its own independent problem (weak
scaling, replicas: the path needs no collective on one box); rank 0 prints.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "grad evals/s & Gcell-steps/s at 256²×K=8; time-to-rel.err vs plain GPU"
UNIT = "grad evals/s"
WL = dict(workload="vessels256", n=256, K=8, M=512, nt=1800, ckpt_every=32, dx=1e-4, c_lo=1350.0, c_hi=1750.0,
          cfl=0.3, pml_alpha=2.0, c_bg=1500.0)

# Algorithmic bytes per grid cell (Ng^2 cells per data set) and launch, FP32.
# A spectrum row holds Ng/2+1 complex values: 8 (Ng/2+1)/Ng bytes per cell.
def bytes_per_cell(cls: int, ng: int, n: int, ckpt_hist: bool = True) -> float:
    spec = 8.0 * (ng // 2 + 1) / ng
    dom = (n * n) / float(ng * ng)
    table = {
        1: 2 * spec + 8 + 4 + 8 + spec + (4 if ckpt_hist else 0),   # row_rho: 2 spectra, rho r+w, c, p spectrum, hist
        2: 2 * spec + 8 + 8 + 2 * spec,                              # row_u: 2 spectra in, u r+w, 2 spectra out
        3: spec + 2 * spec,                                          # col grad: 1 in, 2 out
        4: 2 * spec + 2 * spec,                                      # col pair: 2 in, 2 out
        5: 2 * spec + spec,                                          # col sum: 2 in, 1 out
        6: spec + 8 + 4 + 4 + 8 * dom + 8 + 2 * spec,                # adj rho: spectrum, rb r+w, c, hist, cbar r+w, 2 out
        7: 2 * spec + 8 + 8 + 2 * spec,                              # adj u
    }
    return table[cls]


# Algorithmic bytes per cell-step of a whole forward solve and of a gradient evaluation
# (forward + segment recompute + adjoint), FP32: the state read and written once per step,
# c, checkpoint amortisation, the stored history and the dJ/dc accumulation.
FWD_BYTES = 36.5
GRAD_BYTES = 125.0

KERNEL_FILES = ("fft.cuh", "fft2l.cuh", "geo.cuh", "sync.cuh", "dcheck.cuh", "kfixed.cuh", "kfixed_300.cu", "kernels.cu", "api.cu")


def kernel_source_hash() -> str:
    """Hash of the sources of the solver kernels (the profiles are valid while it is unchanged)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2505_08482_gb300", "csrc")
    for f in KERNEL_FILES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ckpt", type=int, default=WL["ckpt_every"])
    ap.add_argument("--nt", type=int, default=WL["nt"], help="time samples (fewer only for profiling captures)")
    ap.add_argument("--no-graphs", action="store_true", help="launch every kernel from the host (no CUDA graphs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ttr", action="store_true", help="skip the time-to-relative-error comparison")
    ap.add_argument("--no-table2-sample", action="store_true",
                    help="skip the simple-phantom K=4 vs K=1 reconstructions of the default line")
    ap.add_argument("--no-ws-sample", action="store_true",
                    help="skip the reduced warm-start comparison of the default line")
    ap.add_argument("--ws-sample-train", type=int, default=2048, help="training pairs of the reduced warm start")
    ap.add_argument("--ws-sample-test", type=int, default=64, help="held-out seeds of the reduced warm start")
    ap.add_argument("--ws-sample-epochs", type=int, default=6)
    ap.add_argument("--ttr-instances", type=int, default=8)
    ap.add_argument("--ttr-ec", type=float, default=2.0, help="E_c target (%%) of the time-to-target comparison")
    ap.add_argument("--ttr-ep0", type=float, default=50.0, help="E_p0 target (%%) of the time-to-target comparison")
    ap.add_argument("--ttr-iters", type=int, default=20)
    ap.add_argument("--variant", type=int, default=None,
                    help="use this kernel variant instead of the autotuner's choice (profiling runs)")
    ap.add_argument("--cpu-sample-steps", type=int, default=0, help="oracle sample length (0 = auto)")
    ap.add_argument("--batch", action="store_true",
                    help="batched sweep: 64 reconstructions of uneven size and K, grouped by grid side")
    ap.add_argument("--batch-instances", type=int, default=64)
    ap.add_argument("--batch-iters", type=int, default=2)
    ap.add_argument("--batch-plain", type=int, default=64, help="instances also solved one by one")
    ap.add_argument("--batch-sample", type=int, default=16,
                    help="instances of the reduced batched sweep in the default line (0: none)")
    ap.add_argument("--persistent", action="store_true",
                    help="--batch: forward sweeps of the batched arm as persistent launches")
    ap.add_argument("--roofline-k", type=int, default=0,
                    help="per-pass bandwidth of forward steps with this many data sets on the headline grid "
                         "(working set beyond L2 for K >= 64); uses --nt and --variant")
    ap.add_argument("--many-waves-k", type=int, default=64,
                    help="data sets of the default line's many-waves pass measurement (0: none)")
    ap.add_argument("--cluster", action="store_true",
                    help="with --roofline-k: forward sweeps in the cluster-resident form (pat_plan_set_cluster)")
    ap.add_argument("--recon256", action="store_true",
                    help="time to the E_c / E_p0 targets of one plain reconstruction at the headline workload "
                         "(256^2, K=8, Nt=1800, levels 64->128->256)")
    ap.add_argument("--prior-cost", action="store_true",
                    help="cost of the Ornstein-Uhlenbeck prior terms on the headline grid (9 fields)")
    ap.add_argument("--table2", action="store_true",
                    help="simple-phantom experiment of Sec. 4.1: data on a fine grid (no inverse crime), joint "
                         "reconstruction with K=4 data sets against K=1 over four multigrid levels")
    ap.add_argument("--t2-iters", type=int, default=30, help="L-BFGS iterations per level in --table2")
    ap.add_argument("--profile-eval", type=int, default=0,
                    help="profiling runs: this many gradient evaluations of the workload (variant from --variant, "
                         "default 0; no autotuning, no timing) after one warm-up evaluation, then exit")
    ap.add_argument("--gemm", action="store_true",
                    help="BF16 GEMM of the warm-start network: tcgen05 against the warp-level path (TFLOP/s)")
    ap.add_argument("--warmstart", action="store_true",
                    help="learned warm start: train the U-Net on solver-generated pairs, compare with the plain start")
    ap.add_argument("--ws-train", type=int, default=20000)
    ap.add_argument("--ws-test", type=int, default=512)
    ap.add_argument("--ws-epochs", type=int, default=12)
    ap.add_argument("--ws-iters", type=int, default=20)
    ap.add_argument("--ws-ep0", type=float, default=50.0, help="E_p0 target (%%) of the joint comparison")
    return ap.parse_args()


def inputs(seed: int):
    import numpy as np
    import pat_synth as ps
    w = ps.workload(WL["workload"], seed)
    c_init = 0.5 * (w.c_true.min() + w.c_true.max())
    return w, c_init


def pml_auto(n, min_pml=20):
    from paper_2505_08482_gb300.solver import pml_auto as pa
    return pa(n, min_pml)


class ClockSampler:
    """nvidia-smi clock / throttle-reason sampling during the timed region."""

    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def mark(self, begin: bool):
        """Host time of the start or the end of the timed region (samples outside are dropped)."""
        import datetime
        if begin:
            self.t0 = datetime.datetime.now()
        else:
            self.t1 = datetime.datetime.now()

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        import datetime
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f")
                if (self.t0 and ts < self.t0) or (self.t1 and ts > self.t1):
                    continue
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), util=float(parts[4]),
                                 hw=parts[6], hwt=parts[7], swt=parts[8], pcap=parts[9]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        load = [r for r in rows if r["util"] >= 50] or rows
        reasons = set()
        for r in load:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
                if r[key].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in load), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": sorted(reasons), "samples": len(load)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def stored_traffic(cls: int, src_hash: str, key: str = "dram_bytes_per_launch_full"):
    """Per-launch DRAM bytes (or another per-launch ncu figure) of kernel class cls from the
    committed ncu summary, if current."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    e = d.get(str(cls))
    if not e or d.get("kernel_source_hash") != src_hash:
        return None
    return e.get(key)


# ---------------------------------------------------------------------------
def oracle_plain64():
    """The oracle on the 64 x 64 plain workload (K = 1, M = 64, Nt = 400), timed whole on one core:
    one forward, one gradient and one projected L-BFGS iteration from the plain start (seconds)."""
    import numpy as np
    import pat_synth as ps
    from oracle.adjoint import adjoint_grad, objective
    from oracle.forward import forward
    from oracle.grid import make_grid
    from oracle.lbfgs import projected_lbfgs
    from oracle.sensors import sensor_matrix
    w = ps.workload("plain64", 0)
    g = make_grid(64, w.dx, 400, c_ref=WL["c_hi"], cfl=WL["cfl"])
    S = sensor_matrix(g, w.sensors)
    t0 = time.perf_counter()
    y = forward(g, w.c_true, w.p0_true, S)
    t1 = time.perf_counter()
    ym = ps.add_noise(y, ps.rng_for(100))
    wt = ps.noise_weights(ym)
    c0 = np.full((64, 64), 0.5 * (w.c_true.min() + w.c_true.max()))
    t2 = time.perf_counter()
    adjoint_grad(g, c0, 0.5 * w.p0_true, S, ym, wt)
    t3 = time.perf_counter()
    npx = 64 * 64
    unpack = lambda x: (x[:npx].reshape(1, 64, 64), x[npx:].reshape(64, 64))
    fun = lambda x: objective(g, unpack(x)[1], unpack(x)[0], S, ym, wt)[0]

    def fun_grad(x):
        J, gp, gc = adjoint_grad(g, unpack(x)[1], unpack(x)[0], S, ym, wt)
        return J, np.concatenate([gp.ravel(), gc.ravel()])

    x0 = np.concatenate([np.zeros(npx), c0.ravel()])
    lo = np.concatenate([np.zeros(npx), np.full(npx, WL["c_lo"])])
    hi = np.concatenate([np.full(npx, np.inf), np.full(npx, WL["c_hi"])])
    sc = np.concatenate([np.full(npx, 0.25), np.full(npx, (WL["c_hi"] - WL["c_lo"]) / 4.0)])
    t4 = time.perf_counter()
    projected_lbfgs(fun, fun_grad, x0, lo, hi, sc, mem=20, max_iter=1, rtol=0.0)
    t5 = time.perf_counter()
    return {"forward_s": t1 - t0, "gradient_s": t3 - t2, "lbfgs_iteration_s": t5 - t4, "cores": 1}


def _oracle_pool_init():
    import numpy  # noqa: F401
    import oracle.adjoint  # noqa: F401


def _oracle_grad_one(task):
    """One oracle gradient of data set k of the headline workload over nt_s samples (seconds)."""
    seed, k, nt_s = task
    import numpy as np
    import pat_synth as ps
    from oracle.adjoint import adjoint_grad
    from oracle.grid import make_grid
    from oracle.sensors import sensor_matrix
    w, c_init = inputs(seed)
    g = make_grid(w.n, w.dx, nt_s, c_ref=WL["c_hi"], cfl=WL["cfl"])
    S = sensor_matrix(g, w.sensors)
    ym = ps.rng_for(1000 + 16 * seed + k).standard_normal((1, nt_s, w.m)) * 0.01
    t = time.perf_counter()
    adjoint_grad(g, np.full((w.n, w.n), c_init), 0.5 * w.p0_true[k:k + 1], S, ym, np.ones(1))
    return time.perf_counter() - t


class OraclePool:
    """Spawned worker processes that run the oracle's gradient, one data set per task.

    The K data sets of an evaluation are independent until their dJ/dc are summed, so the
    oracle (single-threaded NumPy) runs them side by side, one process per host core.
    """

    def __init__(self, workers: int):
        import multiprocessing as mp
        from concurrent.futures import ProcessPoolExecutor
        self.workers = workers
        self.ex = ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn"), initializer=_oracle_pool_init)
        list(self.ex.map(time.sleep, [0.5] * workers))   # start every worker before timing

    def sample(self, nt_s: int, K_s: int, seed: int = 0):
        """Wall seconds of K_s one-data-set gradients run in parallel, and their summed CPU seconds."""
        t = time.perf_counter()
        per = list(self.ex.map(_oracle_grad_one, [(seed, k, nt_s) for k in range(K_s)]))
        return time.perf_counter() - t, sum(per)

    def close(self):
        self.ex.shutdown()


def cpu_workers() -> int:
    return max(1, min(WL["K"], os.cpu_count() or 1))


def cpu_value(seconds: float, nt_s: int, K_s: int) -> float:
    """Oracle grad evals/s scaled from a sample (cost is linear in K and in Nt)."""
    scale = (WL["K"] * (WL["nt"] - 1)) / float(K_s * (nt_s - 1))
    return 1.0 / (seconds * scale)


def solo_class_times(plan, gs, sensors, c0, p0, stream, dev):
    """Average launch time (us) of each kernel class with its launches timed alone.

    Forward classes: every launch of the class bracketed by events in an eager forward sweep
    (pat_forward on a forward workspace, nothing else on the GPU).  Adjoint classes: the same
    in pat_vjp of a second plan that keeps the whole pressure history, whose reverse sweep
    runs no recompute stream beside the adjoint.  Returns {(class, "forward"|"adjoint"):
    (us per launch, launches timed)}.
    """
    import torch
    from paper_2505_08482_gb300 import _binding as B
    from paper_2505_08482_gb300.solver import Plan
    L = B.lib()
    K, nt, M = plan.K, plan.nt, plan.m
    out = {}
    y = torch.empty((K, nt, M), dtype=torch.float32, device=dev)
    plan.forward(c0, p0, y=y, stream=stream)
    for cls in (B.PAT_K_ROW_RHO, B.PAT_K_ROW_U, B.PAT_K_COL_GRAD, B.PAT_K_COL_PAIR):
        B.check(L.pat_timing_enable(cls, 2 * nt, 1), "pat_timing_enable")
        plan.forward(c0, p0, y=y, stream=stream)
        tot, cnt = ctypes_read(L)
        out[(cls, "forward")] = (1e3 * tot / max(cnt, 1), cnt)
    B.check(L.pat_timing_enable(0, 0, 1), "pat_timing_enable")
    hplan = Plan(gs, sensors, K, ckpt_every=nt, device=dev)
    hplan.variant = plan.variant
    ybar = torch.full((K, nt, M), 1e-3, dtype=torch.float32, device=dev)
    for cls in (0, B.PAT_K_COL_PAIR, B.PAT_K_COL_SUM, B.PAT_K_ROW_ADJ_RHO, B.PAT_K_ROW_ADJ_U):
        hplan.forward(c0, p0, y=y, keep_checkpoints=True, stream=stream)
        if cls:
            B.check(L.pat_timing_enable(cls, 2 * nt, 1), "pat_timing_enable")
        hplan.vjp(c0, p0, ybar, stream=stream)
        tot, cnt = ctypes_read(L)
        if cls:
            out[(cls, "adjoint")] = (1e3 * tot / max(cnt, 1), cnt)
    B.check(L.pat_timing_enable(0, 0, 1), "pat_timing_enable")
    torch.cuda.synchronize()
    del hplan
    torch.cuda.empty_cache()
    return out


def max_over_ranks(t_ms: float, device) -> float:
    """Slowest rank's time: every rank of the process group gets the maximum of t_ms."""
    import torch
    import torch.distributed as tdist
    tt = torch.tensor([t_ms], dtype=torch.float64, device=device)
    tdist.all_reduce(tt, op=tdist.ReduceOp.MAX)
    return float(tt.item())


def whole_job_rate(world: int, steps: int, t_ms: float) -> float:
    """Units per second of the whole job: every rank ran `steps` units in at most t_ms."""
    return world * steps / (t_ms / 1000.0)


def run_reference(args, rank):
    if rank != 0:
        return
    nt_s = args.cpu_sample_steps or 200
    pool = OraclePool(cpu_workers())
    K = WL["K"]
    for _ in range(args.warmup):
        pool.sample(nt_s, K)
    walls, cpus = [], []
    for _ in range(args.steps):
        wall, cpu = pool.sample(nt_s, K)
        walls.append(wall)
        cpus.append(cpu)
    pool.close()
    t = sum(walls) / len(walls)
    v = cpu_value(t, nt_s, K)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * t,
            "ms_per_eval_scaled": 1000.0 / v, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": cfg_dict(args),
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": pool.workers, "kind": "oracle",
                             "sample": f"per step: the FP64 oracle gradient of all K={K} data sets on the same "
                                       f"300^2 grid over Nt={nt_s} samples, one data set per process on "
                                       f"{pool.workers} host cores ({t:.2f} s wall), scaled by (Nt-1) to "
                                       f"Nt={WL['nt']}; ms_per_step is the sample's wall time per step, "
                                       f"ms_per_eval_scaled the scaled time of one whole evaluation (1 / value)",
                             "single_core_value": cpu_value(sum(cpus) / len(cpus), nt_s, K),
                             "sample_wall_ms_per_step": 1000.0 * t, "nproc": os.cpu_count()},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cfg_dict(args):
    return {"workload": f"{WL['workload']}: 256x256 domain (Ng 300, PML 22), K=8 vessel p0 sets, "
                        f"M=512 circle sensors, Nt={args.nt}, s={args.ckpt}, 6 c inclusions",
            "global_batch": WL["K"] * args.gpus, "n": WL["n"], "K": WL["K"], "M": WL["M"], "nt": args.nt,
            "ckpt_every": args.ckpt, "parallelism": f"replicas x{args.gpus}",
            "l2": "256 MiB buffer written between timed steps (working set of one step is L2-resident)"}


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch

    import pat_synth as ps
    import paper_2505_08482_gb300 as pkg
    from paper_2505_08482_gb300 import _binding as B
    from paper_2505_08482_gb300.solver import GridSpec, Plan

    pkg.build()
    # the oracle's worker processes start (spawn) before the first GPU call
    pool = OraclePool(cpu_workers()) if (rank == 0 and world == 1 and not args.no_cpu_baseline) else None
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    L = B.lib()
    w, c_init = inputs(rank)
    n, K, M, nt = WL["n"], WL["K"], WL["M"], args.nt
    P = pml_auto(n)
    dt = WL["cfl"] * WL["dx"] / WL["c_hi"]
    gs = GridSpec(n=n, pml=P, dx=WL["dx"], dt=dt, nt=nt, c_ref=WL["c_hi"], pml_alpha=WL["pml_alpha"],
                  c_bg=WL["c_bg"])
    ng = gs.ng
    plan = Plan(gs, w.sensors, K, ckpt_every=args.ckpt, device=dev)
    if args.variant is None:
        tuned = plan.autotune()       # the library's autotuner picks the variant on this GPU
    else:
        plan.variant = args.variant
        tuned = {}
    f32 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    c_true, p0_true = f32(w.c_true), f32(w.p0_true)
    y_clean = plan.forward(c_true, p0_true).cpu().numpy()
    ym_np = ps.add_noise(y_clean, ps.rng_for(500 + rank))
    w_np = ps.noise_weights(ym_np)
    ym, wt = f32(ym_np), f32(w_np)
    c0 = f32(np.full((n, n), c_init))
    p0 = f32(0.5 * w.p0_true)
    gp0 = torch.empty((K, n, n), dtype=torch.float32, device=dev)
    gc = torch.empty((n, n), dtype=torch.float32, device=dev)
    J = torch.empty((), dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    # a dedicated stream: whole calls are captured into CUDA graphs and replayed (pat_plan_set_graphs)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)

    def grad_eval():
        plan.adjoint_grad(c0, p0, ym, wt, grad_p0=gp0, grad_c=gc, J=J, stream=stream)

    for _ in range(args.warmup):
        grad_eval()
    torch.cuda.synchronize()
    # launches of every kernel class in one evaluation (counted outside the timed region)
    launches_per_eval = {}
    for cls in B.KERNEL_CLASSES:
        B.check(L.pat_timing_enable(cls, 8000, 1), "pat_timing_enable")
        grad_eval()
        launches_per_eval[cls] = ctypes_read(L)[1]
    B.check(L.pat_timing_enable(0, 0, 1), "pat_timing_enable")
    torch.cuda.synchronize()
    solo = solo_class_times(plan, gs, w.sensors, c0, p0, stream, dev)
    # the clock sampler starts here, so that its own start-up (NVML initialisation on a fresh
    # machine) falls before the timed region; it keeps only the samples inside the region
    sampler = ClockSampler(local_rank)
    sampler.start()
    if not args.no_graphs:
        plan.set_graphs(True)
    # the timed loop's own body (flush, evaluation): 3 iterations, and with graphs until 2 s
    # have passed (a fresh machine's first process otherwise sees slower first seconds of
    # replays); eager runs keep a fixed count so that profiler runs launch the same kernels
    t_w, n_w = time.perf_counter(), 0
    floor_s = 0.0 if args.no_graphs else 2.0
    while n_w < 3 or (time.perf_counter() - t_w < floor_s and n_w < 64):
        flush.zero_()
        grad_eval()
        torch.cuda.synchronize()
        n_w += 1

    dist = world > 1
    if dist:
        import torch.distributed as tdist
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches0 = L.pat_kernel_launches()
    # kernel launches before the timed region (the skip count of an ncu launch list of it)
    print(f"launches_before_timed={launches0}", file=sys.stderr, flush=True)
    if dist:
        tdist.barrier()
    torch.cuda.synchronize()
    sampler.mark(True)
    e0.record(stream)
    for _ in range(args.steps):
        flush.zero_()
        grad_eval()
    e1.record(stream)
    torch.cuda.synchronize()
    sampler.mark(False)
    if dist:
        tdist.barrier()
    clocks = sampler.stop()
    launches = int(L.pat_kernel_launches() - launches0)
    t_ms = e0.elapsed_time(e1)
    if dist:
        t_ms = max_over_ranks(t_ms, dev)
    value = whole_job_rate(world, args.steps, t_ms)

    # forward-only throughput (Gcell-steps/s) on the same workload
    yb = torch.empty((K, nt, M), dtype=torch.float32, device=dev)
    for _ in range(2):
        plan.forward(c0, p0, y=yb, stream=stream)
    torch.cuda.synchronize()
    nf = max(2, args.steps)
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(nf):
        flush.zero_()
        plan.forward(c0, p0, y=yb, stream=stream)
    f1.record(stream)
    torch.cuda.synchronize()
    fwd_s = f0.elapsed_time(f1) / 1000.0 / nf
    gcell = ng * ng * K * (nt - 1) / fwd_s / 1e9

    # end to end through host buffers (pinned), the call a user makes
    pin = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32).pin_memory()
    h_c, h_p0, h_ym, h_w = pin(np.full((n, n), c_init)), pin(0.5 * w.p0_true), pin(ym_np), pin(w_np)
    h_gp0 = torch.empty((K, n, n), dtype=torch.float32).pin_memory()
    h_gc = torch.empty((n, n), dtype=torch.float32).pin_memory()
    h_J = torch.empty((), dtype=torch.float64).pin_memory()
    d_c, d_p0, d_ym, d_w = (torch.empty_like(t, device=dev) for t in (h_c, h_p0, h_ym, h_w))
    h2d = sum(t.numel() * t.element_size() for t in (h_c, h_p0, h_ym, h_w))
    d2h = sum(t.numel() * t.element_size() for t in (h_gp0, h_gc, h_J))

    def e2e_step():
        for d, h in ((d_c, h_c), (d_p0, h_p0), (d_ym, h_ym), (d_w, h_w)):
            d.copy_(h, non_blocking=True)
        plan.adjoint_grad(d_c, d_p0, d_ym, d_w, grad_p0=gp0, grad_c=gc, J=J, stream=stream)
        h_gp0.copy_(gp0, non_blocking=True)
        h_gc.copy_(gc, non_blocking=True)
        h_J.copy_(J, non_blocking=True)

    e2e_step()
    torch.cuda.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if dist:
        tdist.barrier()
    g0.record(stream)
    for _ in range(args.steps):
        flush.zero_()
        e2e_step()
    g1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = g0.elapsed_time(g1)
    if dist:
        e2e_ms = max_over_ranks(e2e_ms, dev)
    e2e_val = whole_job_rate(world, args.steps, e2e_ms)

    # roofline of the dominant kernel: the class with the largest solo time per evaluation
    # (solo launch time x launches per evaluation); its own launches timed alone
    peak, peak_kind = measured_peaks()
    src_hash = kernel_source_hash()
    # launches of each measured entry per evaluation: the forward classes run in the forward
    # sweep and again in the segment recompute, the adjoint classes once
    phase_launches = {k: (2 if k[1] == "forward" else 1) * (nt - 1) for k in solo}
    dom_key = max(solo, key=lambda k: solo[k][0] * phase_launches[k])
    serial_us = sum(solo[k][0] * phase_launches[k] for k in solo)
    dom, dom_phase = dom_key
    dom_us, dom_cnt = solo[dom_key]
    bpl = bytes_per_cell(dom, ng, n) * ng * ng * K
    achieved = bpl / (dom_us * 1e-6) / 1e9
    per_eval_ms = t_ms / args.steps
    cells = ng * ng * K * (nt - 1)
    # the same launches against the instruction-issue peak (4 schedulers per SM, one warp
    # instruction per cycle each, at the maximum SM clock), from the warp instructions per launch
    # of the committed ncu capture
    insts = stored_traffic(dom, src_hash, "warp_instructions_per_launch")
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_max = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("sm_max_mhz", 2070.0)) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 2070.0
    issue_peak = 4.0 * sms * sm_max * 1e6
    issue = None if insts is None else {
        "bound": "alu", "unit": "warp instructions/s", "instructions_per_launch": insts,
        "achieved": insts / (dom_us * 1e-6), "peak": issue_peak, "frac": insts / (dom_us * 1e-6) / issue_peak,
        "peak_kind": f"4 schedulers x {sms} SMs x {sm_max:.0f} MHz (one warp instruction per cycle each)",
        "source": "smsp__inst_executed.sum of the dominant pass (ncu, profiles/traffic.json)"}
    roof = {"bound": "hbm", "kernel": f"{B.KERNEL_CLASSES[dom]} ({dom_phase} sweep)", "achieved": achieved,
            "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": stored_traffic(dom, src_hash),
            "peak_kind": f"{peak_kind} hbm_gbs (burst copy)", "algorithmic_bytes_per_launch": bpl,
            "avg_launch_us": dom_us, "launches_timed": dom_cnt,
            "timing": "every launch of the class bracketed by CUDA events on its stream in an eager sweep that "
                      "runs alone on the GPU (forward classes: pat_forward; adjoint classes: pat_vjp of a plan "
                      "that keeps the whole pressure history, so no recompute stream runs beside it); the events "
                      "also end the programmatic launch overlap with the neighbouring kernels",
            "solo_us_per_launch": {f"{B.KERNEL_CLASSES[c]} ({ph})": round(v[0], 3) for (c, ph), v in solo.items()},
            "launches_per_eval": {B.KERNEL_CLASSES[c]: v for c, v in launches_per_eval.items()},
            "issue": issue,
            "share_of_serialised_sum": round(dom_us * phase_launches[dom_key] / serial_us, 3),
            "share_note": "the dominant class's serialised time over the sum of every class's (solo launch time x "
                          "launches per evaluation): the quantity an ncu launch list of one evaluation gives",
            "note": "solo launch times are serialised times: inside an evaluation the passes overlap with their "
                    "neighbours (programmatic dependent launch) and the recompute stream runs beside the "
                    "adjoint, so solo time x launches summed over classes exceeds the evaluation time",
            "step_level": {
                "gradient": {"bytes_per_cell_step": GRAD_BYTES, "cell_steps": cells,
                             "achieved_GBs": GRAD_BYTES * cells / (per_eval_ms * 1e-3) / 1e9,
                             "frac": GRAD_BYTES * cells / (per_eval_ms * 1e-3) / 1e9 / peak},
                "forward": {"bytes_per_cell_step": FWD_BYTES, "cell_steps": cells,
                            "achieved_GBs": FWD_BYTES * cells / fwd_s / 1e9,
                            "frac": FWD_BYTES * cells / fwd_s / 1e9 / peak}}}

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": cfg_dict(args),
            "forward_gcell_steps_per_s": gcell * world, "forward_ms": fwd_s * 1000.0,
            "grad_gcell_steps_per_s": value * ng * ng * K * (nt - 1) / 1e9,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches, "roofline": roof, "clocks": clocks, "kernel_source_hash": src_hash,
            "autotune_ms_per_grad_eval": {str(v): round(t, 2) for v, t in tuned.items()}, "variant": plan.variant,
            "cuda_graphs": not args.no_graphs}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        nt_s = args.cpu_sample_steps or 200
        wall, cpu = pool.sample(nt_s, K)
        pool.close()
        v = cpu_value(wall, nt_s, K)
        line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": pool.workers, "kind": "oracle",
                                "sample": f"the FP64 oracle gradient of all K={K} data sets on the same 300^2 grid "
                                          f"over Nt={nt_s} samples, one data set per process on {pool.workers} "
                                          f"host cores ({wall:.1f} s wall), scaled by (Nt-1) to Nt={WL['nt']}",
                                "single_core_value": cpu_value(cpu, nt_s, K), "nproc": os.cpu_count(),
                                "plain64_unscaled_s": oracle_plain64()}
    if rank == 0 and world == 1 and args.many_waves_k > 0:
        # the same passes with many waves of CTAs (working set beyond L2): the HBM-bound regime
        mw = roofline_k(args.many_waves_k, 400, None, WL["ckpt_every"], 2, 3)
        line["roofline"]["many_waves"] = {"workload": mw["config"]["workload"], "variant": mw["variant"],
                                          "forward_gcell_steps_per_s": mw["forward_gcell_steps_per_s"],
                                          "passes": mw["passes"], "peak": mw["peak"],
                                          "timing": "CUDA events around every launch of a class in an eager "
                                                    "forward sweep that runs alone; variant from the autotuner"}
    if rank == 0 and world == 1 and not args.no_ttr:
        line["time_to_rel_err"] = time_to_rel_err(args, dev)
        # the plain solve at the headline workload itself (256^2, K = 8, three levels)
        line["time_to_rel_err"]["headline_plain"] = recon256(args, dev)
        if not args.no_ws_sample:
            line["time_to_rel_err"]["warm_start"] = warm_start_sample(args)
        if not args.no_table2_sample:
            # the simple phantoms of Sec. 4.1 (K = 4 against K = 1, Table 2 trend)
            line["table2_trend"] = table2(args.t2_iters)
        if args.batch_sample > 0:
            # the batched serving-style sweep on a reduced sample (all of it also solved one by one)
            b = batch_sweep(args.batch_sample, args.batch_sample, args.batch_iters, False)
            b["config"]["workload"] = "reduced sample (bench.py --batch runs 64): " + b["config"]["workload"]
            line["batched_sweep"] = b
    if rank == 0:
        print(json.dumps(line), flush=True)


def time_to_rel_err(args, dev):
    """Time to equal relative errors in c and p0 (Eq. RelativeError), plain GPU solve against the
    batched solve, on the 128 x 128 vessel workload (K = 4, M = 256, Nt = 900, 6 inclusions,
    levels 64 -> 128, 1 % noise).

    Plain: the instances one after another, each a pat_reconstruct-equivalent call (one
    instance).  Batched: all instances in one pat_reconstruct_batched call.  Every instance
    stops once E_c <= ttr_ec and E_p0 <= ttr_ep0 on the finest level (at most ttr_iters L-BFGS
    iterations per level).  All instances arrive at once: an instance's latency is the time
    from the common start until its call returns.
    """
    import numpy as np
    import torch

    import pat_synth as ps
    from paper_2505_08482_gb300.solver import GridSpec, Plan, ReconConfig, reconstruct_batched
    f32 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    n, K, M, nt = 128, 4, 256, 900
    dx = WL["dx"]
    gs = GridSpec(n=n, pml=pml_auto(n), dx=dx, dt=WL["cfl"] * dx / WL["c_hi"], nt=nt, c_ref=WL["c_hi"])
    insts = []
    for i in range(args.ttr_instances):
        wl = ps.workload("vessels128", 7000 + i)
        gen = Plan(gs, wl.sensors, K, device=dev)
        y = ps.add_noise(gen.forward(f32(wl.c_true), f32(wl.p0_true)).cpu().numpy(), ps.rng_for(7500 + i))
        del gen
        insts.append(dict(y_meas=f32(y), w=f32(ps.noise_weights(y)),
                          c_init=f32(np.full((n, n), 0.5 * (wl.c_true.min() + wl.c_true.max()))),
                          c_true=f32(wl.c_true), p0_true=f32(wl.p0_true), ec_target=args.ttr_ec,
                          ep0_target=args.ttr_ep0))
    sensors = ps.workload("vessels128", 7000).sensors
    cfg = ReconConfig(levels=(64, 128), L=n * dx, dt_data=gs.dt, nt_data=nt, sensors_xy=sensors, K=K,
                      iters=args.ttr_iters, mem=20, ckpt_every=32, rtol=0.0)
    reconstruct_batched(cfg, insts[:1])        # first use of the kernels of both levels
    torch.cuda.synchronize()

    def reached(rows):
        fin = [r for r in rows if r["level"] == 1]
        return bool(fin) and fin[-1]["Ec"] <= args.ttr_ec and fin[-1]["Ep0"] <= args.ttr_ep0

    # plain: one instance per call, in arrival order
    done, ok_plain, it_plain = [], [], []
    t0 = time.perf_counter()
    for ins in insts:
        (res, _) = reconstruct_batched(cfg, [ins])
        torch.cuda.synchronize()
        done.append(time.perf_counter() - t0)
        ok_plain.append(reached(res[0][2]))
        it_plain.append(len(res[0][2]))
    wall_plain = time.perf_counter() - t0
    t0 = time.perf_counter()
    res, _ = reconstruct_batched(cfg, insts)
    torch.cuda.synchronize()
    wall_b = time.perf_counter() - t0
    ok_b = [reached(r[2]) for r in res]
    q = lambda v, f: float(np.percentile(v, f))
    return {"workload": f"vessels128: 128x128, K={K}, M={M}, Nt={nt}, levels 64->128, "
                        f"{args.ttr_instances} seeded instances arriving together",
            "targets": {"E_c_pct": args.ttr_ec, "E_p0_pct": args.ttr_ep0,
                        "max_iterations_per_level": args.ttr_iters},
            "plain": {"wall_s": wall_plain, "latency_s_p50": q(done, 50), "latency_s_p99": q(done, 99),
                      "reached": sum(ok_plain) / len(ok_plain),
                      "iterations_median": float(np.median(it_plain))},
            "batched": {"wall_s": wall_b, "latency_s_p50": wall_b, "latency_s_p99": wall_b,
                        "reached": sum(ok_b) / len(ok_b),
                        "iterations_median": float(np.median([len(r[2]) for r in res]))},
            "speedup_batched_vs_plain": wall_plain / wall_b}


def run_recon256(args):
    import paper_2505_08482_gb300 as pkg
    pkg.build()
    import torch
    print(json.dumps(recon256(args, torch.device("cuda", 0))), flush=True)


def recon256(args, dev):
    """One plain reconstruction (pat_reconstruct through the batched call with one instance) of
    the headline workload: 256 x 256 domain, K = 8 vessel p0 sets, M = 512 sensors, Nt = 1800,
    s = 32, 1 % noise, levels 64 -> 128 -> 256 with at most ttr_iters L-BFGS iterations each,
    c starting at the midpoint of the true range, p0 at zero.  E_c and E_p0 (Eq. RelativeError)
    are tracked after every iteration against the true c and p0 resampled to the level; the run
    leaves a level (the finest: stops) once both targets are met.  Returns the line: wall time,
    iterations per level and the iteration time until the targets were first met on the finest
    level."""
    import numpy as np
    import torch

    import pat_synth as ps
    from paper_2505_08482_gb300.solver import GridSpec, Plan, ReconConfig, reconstruct_batched
    f32 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    w, c_init = inputs(0)
    n, K, M, nt = WL["n"], WL["K"], WL["M"], WL["nt"]
    dx = WL["dx"]
    gs = GridSpec(n=n, pml=pml_auto(n), dx=dx, dt=WL["cfl"] * dx / WL["c_hi"], nt=nt, c_ref=WL["c_hi"])
    gen = Plan(gs, w.sensors, K, device=dev)
    y = ps.add_noise(gen.forward(f32(w.c_true), f32(w.p0_true)).cpu().numpy(), ps.rng_for(500))
    del gen
    ins = dict(y_meas=f32(y), w=f32(ps.noise_weights(y)), c_init=f32(np.full((n, n), c_init)),
               c_true=f32(w.c_true), p0_true=f32(w.p0_true), ec_target=args.ttr_ec, ep0_target=args.ttr_ep0)
    cfg = ReconConfig(levels=(64, 128, 256), L=n * dx, dt_data=gs.dt, nt_data=nt, sensors_xy=w.sensors, K=K,
                      iters=args.ttr_iters, mem=20, ckpt_every=WL["ckpt_every"], rtol=0.0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res, total_ms = reconstruct_batched(cfg, [ins])
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    rows = res[0][2]
    fin = [r for r in rows if r["level"] == 2]
    hit = next((i for i, r in enumerate(rows) if r["level"] == 2 and r["Ec"] <= args.ttr_ec
                and r["Ep0"] <= args.ttr_ep0), None)
    per_level = {str(cfg.levels[lv]): {"iterations": sum(1 for r in rows if r["level"] == lv),
                                       "ms": sum(r["ms"] for r in rows if r["level"] == lv)} for lv in range(3)}
    line = {"metric": "time to E_c / E_p0 targets, plain GPU reconstruction", "value": wall, "unit": "s",
            "n_gpus": 1, "higher_is_better": False, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{WL['workload']}: 256x256 (Ng 300), K={K}, M={M}, Nt={nt}, s={WL['ckpt_every']}, "
                                   "levels 64->128->256, 1 % noise, c from the midpoint of the true range",
                       "targets": {"E_c_pct": args.ttr_ec, "E_p0_pct": args.ttr_ep0,
                                   "max_iterations_per_level": args.ttr_iters}},
            "reached": hit is not None, "iterations": len(rows), "per_level": per_level,
            "iteration_time_to_targets_s": None if hit is None else sum(r["ms"] for r in rows[:hit + 1]) / 1e3,
            "E_c_initial_pct": float(100.0 * np.linalg.norm(c_init - w.c_true) / np.linalg.norm(w.c_true)),
            "E_c_final_pct": fin[-1]["Ec"] if fin else None, "E_p0_final_pct": fin[-1]["Ep0"] if fin else None,
            "status": res[0][3], "library_total_ms": total_ms}
    return line


def warm_start_sample(args):
    """The learned warm start against the plain start on a reduced sample of its workload:
    the U-Net (4 levels x 32 channels, BF16 on the tcgen05 tensor cores) trained on
    ws_sample_train solver-generated pairs (128 x 128, K = 4, M = 256, Nt = 600, 2-8 inclusions)
    for ws_sample_epochs epochs, then ws_sample_test held-out seeds reconstructed from each start
    (levels 64 -> 128, at most ttr_iters L-BFGS iterations per level, every instance in one batched
    call per arm, each instance stopping once E_c <= ttr_ec and E_p0 <= ttr_ep0, Eq. RelativeError).
    The full-size run (20,000 pairs, 512 seeds) is bench.py --warmstart.
    """
    import numpy as np
    import torch

    from paper_2505_08482_gb300.solver import ReconConfig, reconstruct_batched
    from paper_2505_08482_gb300.warmstart import (PairGenerator, UNet, init_params, iterations_to, predict_c,
                                                  relative_error, train)
    n, K = 128, 4
    gen = PairGenerator(n=n, K=K, M=256, nt=600, batch=64)
    t0 = time.perf_counter()
    X, T, _ = gen.make(list(range(args.ws_sample_train)))
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    net = UNet(4, 32, K, n, n, max_batch=32)
    net.set_params(init_params(4, 32, K, seed=1))
    t0 = time.perf_counter()
    hist = train(net, X, T, epochs=args.ws_sample_epochs, batch=32, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del X, T
    Xh, _, raw = gen.make(list(range(10 ** 6, 10 ** 6 + args.ws_sample_test)), keep_data=True)
    c_true = torch.stack([r["c_true"] for r in raw])
    t0 = time.perf_counter()
    c_warm = predict_c(net, Xh)
    torch.cuda.synchronize()
    t_pred = time.perf_counter() - t0
    c_plain = torch.stack([torch.full_like(ct, 0.5 * float(ct.min() + ct.max())) for ct in c_true])
    cfg = ReconConfig(levels=(64, n), L=n * 1e-4, dt_data=gen.gs.dt, nt_data=gen.nt, sensors_xy=gen.sensors, K=K,
                      iters=args.ttr_iters, mem=20, ckpt_every=32, rtol=0.0)
    out = {}
    for name, cinit in (("plain", c_plain), ("warm", c_warm)):
        insts = [dict(y_meas=r["y_meas"].contiguous(), w=r["w"].contiguous(), c_init=cinit[j].contiguous(),
                      c_true=r["c_true"].contiguous(), p0_true=r["p0_true"].contiguous(), ec_target=args.ttr_ec,
                      ep0_target=args.ttr_ep0) for j, r in enumerate(raw)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res, _ = reconstruct_batched(cfg, insts)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        its = [iterations_to(rows, args.ttr_ec, 2, args.ttr_ep0) for _, _, rows, _ in res]
        reached = [i for i, _ in its if i is not None]
        out[name] = {"initial_Ec_median": float(np.median(relative_error(cinit, c_true).cpu().numpy())),
                     "reached": len(reached) / len(its),
                     "iterations_median": float(np.median(reached)) if reached else None,
                     "ms_median": float(np.median([m for i, m in its if i is not None])) if reached else None,
                     "wall_s_batched": wall}
    out["warm"]["prediction_s"] = t_pred
    return {"workload": f"reduced sample of the warm-start workload: U-Net 4 levels x 32 trained on "
                        f"{args.ws_sample_train} solver-generated pairs (128x128, K=4, M=256, Nt=600, 2-8 "
                        f"inclusions) for {args.ws_sample_epochs} epochs, {args.ws_sample_test} held-out seeds, "
                        f"levels 64->128; the full run is bench.py --warmstart",
            "targets": {"E_c_pct": args.ttr_ec, "E_p0_pct": args.ttr_ep0, "max_iterations_per_level": args.ttr_iters},
            "pair_generation_s": t_gen, "training_s": t_train, "train_loss_first_last": [hist[0], hist[-1]],
            "plain": out["plain"], "warm": out["warm"],
            "speedup_warm_vs_plain_median_ms": (out["plain"]["ms_median"] / out["warm"]["ms_median"])
            if out["plain"]["ms_median"] and out["warm"]["ms_median"] else None}


def run_batch(args):
    """Batched serving-style sweep (two-level multigrid N/2 -> N per instance)."""
    print(json.dumps(batch_sweep(args.batch_instances, args.batch_plain, args.batch_iters, args.persistent)),
          flush=True)


def batch_sweep(n_inst, n_plain, iters, persistent):
    """n_inst reconstructions with N ~ U{96,128,160,192,256}, K ~ U{1,2,4,8}, M = 2N, Nt = 7N (two
    multigrid levels N/2 -> N, iters L-BFGS iterations per level), solved batched (one
    pat_reconstruct_batched call per grid side, the sides concurrently) and about n_plain of them
    one by one; returns the measurement line."""
    import threading

    import numpy as np
    import torch

    import pat_synth as ps
    import paper_2505_08482_gb300 as pkg
    from paper_2505_08482_gb300 import _binding as B
    from paper_2505_08482_gb300.solver import GridSpec, Plan, ReconConfig, reconstruct, reconstruct_batched
    pkg.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    rng = ps.rng_for(2024)
    sides = [96, 128, 160, 192, 256]
    specs = [(int(rng.choice(sides)), int(rng.choice([1, 2, 4, 8]))) for _ in range(n_inst)]
    dx, c_hi = 1e-4, 1750.0
    f32 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    groups = {}
    for i, (n, K) in enumerate(specs):
        groups.setdefault(n, []).append((i, K))
    data = {}
    cell_steps = 0.0
    for n, members in groups.items():
        M, nt = 2 * n, 7 * n
        P = pml_auto(n)
        gs = GridSpec(n=n, pml=P, dx=dx, dt=0.3 * dx / c_hi, nt=nt, c_ref=c_hi)
        xy = ps.circle_sensors(n, M, dx)
        Ks = [K for _, K in members]
        gen = Plan(gs, xy, Ks, ckpt_every=32, device=dev)
        cs, p0s = [], []
        for i, K in members:
            r = ps.rng_for(3000 + i)
            cs.append(ps.ellipse_phantom(n, int(r.integers(2, 9)), r))
            p0s.append(np.stack([ps.vessel_p0(n, r) for _ in range(K)]))
        y = gen.forward(f32(np.stack(cs)), f32(np.concatenate(p0s))).cpu().numpy()
        del gen
        k0 = 0
        for (i, K), c in zip(members, cs):
            yk = ps.add_noise(y[k0:k0 + K], ps.rng_for(4000 + i))
            data[i] = dict(y_meas=f32(yk), w=f32(ps.noise_weights(yk)),
                           c_init=f32(np.full((n, n), 0.5 * (c.min() + c.max()))))
            k0 += K
        data[("cfg", n)] = ReconConfig(levels=(n // 2, n), L=n * dx, dt_data=gs.dt, nt_data=nt, sensors_xy=xy, K=1,
                                       iters=iters, mem=20, ckpt_every=32, autotune=True,
                                       persistent=persistent)
    torch.cuda.synchronize()
    # batched: one call per grid side, the sides concurrently on their own streams
    lat = {}
    launches0 = B.lib().pat_kernel_launches()
    errors = []

    def group_run(n, members):
        try:
            stream = torch.cuda.Stream(device=dev)
            with torch.cuda.stream(stream):
                res, ms = reconstruct_batched(data[("cfg", n)], [data[i] for i, _ in members], stream=stream)
            for (i, _), r in zip(members, res):
                lat[i] = ms
                data[i]["rows"] = r[2]
        except Exception as e:  # reported below
            errors.append(repr(e))

    t0 = time.perf_counter()
    th = [threading.Thread(target=group_run, args=(n, m)) for n, m in groups.items()]
    for t in th:
        t.start()
    for t in th:
        t.join()
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    if errors:
        raise RuntimeError(errors[0])
    batched_launches = int(B.lib().pat_kernel_launches() - launches0)
    # forward-equivalent cell-steps: every trial = 1 forward, every gradient = 3
    for n, members in groups.items():
        for i, K in members:
            for r in data[i]["rows"]:
                lvl_n = n // 2 if r["level"] == 0 else n
                ng = lvl_n + 2 * pml_auto(lvl_n)
                nt_l = int(round((7 * n - 1) * (lvl_n / n))) + 1
                cell_steps += ng * ng * K * (nt_l - 1) * (r["trials"] + 3)
    # plain GPU: the same instances one at a time, no batching, no graphs, default variant
    plain, plain_arrival = {}, {}
    tp0 = time.perf_counter()
    for n, members in groups.items():
        for i, K in members[: max(1, n_plain * len(members) // len(specs))]:
            cfg = data[("cfg", n)]
            cfg.K = K
            cfg.autotune = False
            cfg.persistent = False
            t1 = time.perf_counter()
            reconstruct(cfg, data[i]["y_meas"], data[i]["w"], data[i]["c_init"])
            torch.cuda.synchronize()
            plain[i] = (time.perf_counter() - t1) * 1e3
            plain_arrival[i] = (time.perf_counter() - tp0) * 1e3
    plain_wall = time.perf_counter() - tp0
    lats = sorted(lat.values())
    pl = sorted(plain.values())
    q = lambda v, f: float(np.percentile(v, f)) if v else None
    frac = len(plain) / len(specs)
    line = {"metric": "batched sweep aggregate Gcell-steps/s", "value": cell_steps / wall / 1e9,
            "unit": "Gcell-steps/s", "n_gpus": 1, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"{len(specs)} reconstructions, N~U{{96..256}}, K~U{{1,2,4,8}}, M=2N, Nt=7N, "
                                   f"levels N/2->N, {iters} L-BFGS iterations per level",
                       "groups": {str(n): len(m) for n, m in groups.items()}},
            "wall_s": wall, "latency_ms_p50": q(lats, 50), "latency_ms_p99": q(lats, 99),
            "plain_wall_s_scaled": plain_wall / frac if frac > 0 else None,
            "plain_latency_ms_p50": q(pl, 50), "plain_latency_ms_p99": q(pl, 99),
            "latency_note": "all instances arrive together: the batched latency is the time until the batched "
                            "call of the instance's grid side returns; plain_latency_* is each reconstruction's "
                            "own duration and plain_arrival_latency_* the time from the common arrival until it "
                            "is done when they are served one after another",
            "plain_arrival_latency_ms_p50": q(sorted(plain_arrival.values()), 50),
            "plain_arrival_latency_ms_p99": q(sorted(plain_arrival.values()), 99),
            "persistent_sweeps": bool(persistent),
            "plain_instances_timed": len(plain), "gpu_launches": batched_launches,
            "speedup_vs_plain": (plain_wall / frac) / wall if frac > 0 else None}
    return line


def run_roofline_k(args):
    print(json.dumps(roofline_k(args.roofline_k, args.nt, args.variant, args.ckpt, args.warmup, args.steps,
                                args.cluster)), flush=True)


def roofline_k(K, nt, variant, ckpt, warmup, steps, cluster=False):
    """Per-pass achieved bandwidth of forward sweeps on the 300^2 grid with K data sets.

    At K = 8 the state and spectra of a step (about 30 MB) stay in L2 and the passes are
    latency-bound; with K = 64 they take about 140 MB, more than L2, so each pass streams its
    fields through HBM.  The K data sets are the headline's eight vessel sets repeated.
    """
    import numpy as np
    import torch

    import paper_2505_08482_gb300 as pkg
    from paper_2505_08482_gb300 import _binding as B
    from paper_2505_08482_gb300.solver import GridSpec, Plan

    pkg.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    L = B.lib()
    w, _ = inputs(0)
    n = WL["n"]
    P = pml_auto(n)
    dt = WL["cfl"] * WL["dx"] / WL["c_hi"]
    gs = GridSpec(n=n, pml=P, dx=WL["dx"], dt=dt, nt=nt, c_ref=WL["c_hi"], pml_alpha=WL["pml_alpha"],
                  c_bg=WL["c_bg"])
    ng = gs.ng
    plan = Plan(gs, w.sensors, K, ckpt_every=ckpt, device=dev)
    if variant is None:
        plan.autotune(gradient=False)
    else:
        plan.variant = variant
    if cluster:
        plan.cluster = True
    f32 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    reps = -(-K // w.p0_true.shape[0])
    c, p0 = f32(w.c_true), f32(np.concatenate([w.p0_true] * reps)[:K])
    y = torch.empty((K, nt, WL["M"]), dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)
    prev_stream = torch.cuda.current_stream(dev)
    torch.cuda.set_stream(stream)
    for _ in range(max(warmup, 1)):
        plan.forward(c, p0, y=y, stream=stream)
    torch.cuda.synchronize()
    peak, peak_kind = measured_peaks()
    passes = {}
    for cls in (() if cluster else (3, 2, 4, 1)):     # the four passes of a forward step
        B.check(L.pat_timing_enable(cls, nt + 8, 1), "pat_timing_enable")
        plan.forward(c, p0, y=y, stream=stream)
        tot, cnt = ctypes_read(L)
        B.check(L.pat_timing_enable(0, 0, 1), "pat_timing_enable")
        bpl = bytes_per_cell(cls, ng, n, ckpt_hist=False) * ng * ng * K
        us = tot * 1000.0 / max(cnt, 1)
        passes[B.KERNEL_CLASSES[cls]] = {"launches": cnt, "avg_launch_us": round(us, 2),
                                         "algorithmic_bytes_per_launch": bpl,
                                         "achieved_gbs": round(bpl / (us * 1e-6) / 1e9, 1),
                                         "frac": round(bpl / (us * 1e-6) / 1e9 / peak, 3)}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        plan.forward(c, p0, y=y, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    fwd_s = e0.elapsed_time(e1) / 1000.0 / steps
    torch.cuda.set_stream(prev_stream)
    return {"metric": f"per-pass achieved algorithmic HBM GB/s, forward sweep at K={K}",
                      "unit": "GB/s", "n_gpus": 1, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": f"vessels256 grid (Ng {ng}) with K={K} data sets, M={WL['M']}, "
                                             f"Nt={nt}", "K": K, "nt": nt},
                      "variant": plan.variant, "cluster_resident": bool(cluster),
                      "peak": peak, "peak_kind": f"{peak_kind} hbm_gbs",
                      "passes": passes, "forward_ms": fwd_s * 1000.0,
                      "forward_gcell_steps_per_s": ng * ng * K * (nt - 1) / fwd_s / 1e9,
                      "kernel_source_hash": kernel_source_hash()}


def run_prior_cost(args):
    """Time one evaluation of the prior terms (value and gradient) for c and the 8 p0 fields
    of the headline workload on its 256 x 256 grid (dx 0.1 mm, tau 1.5 mm): cold start, then
    started from that solution after adding white noise of 0.1 % of each field's peak (a rough
    change: it excites the high spatial frequencies, where Xi's eigenvalues are smallest)."""
    import numpy as np
    import torch

    import pat_synth as ps
    import paper_2505_08482_gb300 as pkg
    from paper_2505_08482_gb300.solver import Prior

    pkg.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    w, _ = inputs(0)
    n, K = WL["n"], WL["K"]
    f32 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    x = f32(np.concatenate([w.p0_true, w.c_true[None]]))
    lo, hi = float(w.c_true.min()), float(w.c_true.max())
    eta = [0.5] * K + [0.5 * (lo + hi)]
    sig = [0.25] * K + [0.25 * (hi - lo)]
    pr = Prior(n, WL["dx"], 1.5e-3, K + 1, device=dev)
    out = {}
    for _ in range(2):                       # first launches of the kernels
        pr.eval(x, eta, sig, tol=1e-5, maxit=500)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    v, g, z, it = pr.eval(x, eta, sig, tol=1e-5, maxit=500)
    out["cold"] = {"ms": 1000 * (time.perf_counter() - t0), "iterations": it}
    torch.manual_seed(0)
    x2 = x + 1e-3 * torch.randn_like(x) * x.abs().amax(dim=(1, 2), keepdim=True)
    t0 = time.perf_counter()
    v2, g2, z2, it2 = pr.eval(x2, eta, sig, z=z, tol=1e-5, maxit=500)
    out["warm_after_white_noise"] = {"ms": 1000 * (time.perf_counter() - t0), "iterations": it2}
    print(json.dumps({"metric": "Ornstein-Uhlenbeck prior terms: ms per evaluation (value and gradient)",
                      "unit": "ms", "n_gpus": 1, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": f"{n}x{n} grid, dx 0.1 mm, tau 1.5 mm, {K + 1} fields (8 p0 + c), "
                                             "PCG to a relative residual of 1e-5"},
                      "results": out}), flush=True)


def run_table2(args):
    print(json.dumps(table2(args.t2_iters)), flush=True)


def table2(t2_iters):
    """Simple-phantom experiment (Sec. 4.1, Table 2 trend) on the paper's geometry.

    Data: 334 x 334 grid of 63.7 um over the 20 mm target plus its sensor layer, 236 sensors
    0.2 mm outside the target, dt = 12.1 ns (smaller if the CFL number would exceed 0.3),
    1747 samples over the same duration, 1 % noise.  Reconstruction on four coarser levels
    (sides 40, 58, 94, 136: the even sides nearest to the Table 1 pixel sizes) with the
    Ornstein-Uhlenbeck prior (tau = 1.5 mm, means and deviations as in Sec. 4.1.2), once with
    all four data sets and once with p0_1 alone; E_c and E_p0^1 on the finest level.
    """
    import numpy as np
    import torch

    import pat_synth as ps
    import paper_2505_08482_gb300 as pkg
    from paper_2505_08482_gb300.solver import GridSpec, Plan, ReconConfig, reconstruct

    pkg.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(0)
    L, n_d = ps.SIMPLE_L, 334
    dx_d = L / n_d
    T = 1746 * 12.1e-9
    levels = (40, 58, 94, 136)
    nf = levels[-1]
    xy = ps.square_sensors()
    f32 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    err = lambda a, b: float(100.0 * np.linalg.norm(a - b) / np.linalg.norm(a))
    paper = {"circles": (2.0, 3.2, 17.0, 24.9), "water": (2.1, 3.5, None, None), "bone": (12.0, 14.5, None, None)}
    out = {}
    t_all = time.perf_counter()
    for kind in ("circles", "water", "bone"):
        U = 3000.0 if kind == "bone" else 1800.0
        dt_d = min(12.1e-9, 0.3 * dx_d / U)
        nt_d = int(round(T / dt_d)) + 1
        c_d, p0_d = ps.simple_phantom_c(kind, n_d), ps.simple_phantom_p0(n_d, 4)
        gs = GridSpec(n=n_d, pml=pml_auto(n_d), dx=dx_d, dt=dt_d, nt=nt_d, c_ref=U, c_bg=1430.0)
        plan = Plan(gs, xy, 4, device=dev)
        y = ps.add_noise(plan.forward(f32(c_d), f32(p0_d)).cpu().numpy(), ps.rng_for(300))
        wts = ps.noise_weights(y)
        del plan
        c_t, p0_t = ps.simple_phantom_c(kind, nf), ps.simple_phantom_p0(nf, 4)
        eta_c = 1482.0 if kind == "bone" else 0.5 * (1430.0 + 1580.0)
        sig_c = 0.25 * (c_t.max() - c_t.min())
        row = {"U_c": U, "data_grid": f"{n_d}^2, dx {dx_d * 1e6:.1f} um, dt {dt_d * 1e9:.2f} ns, Nt {nt_d}"}
        for K in (4, 1):
            cfg = ReconConfig(levels=levels, L=L, dt_data=dt_d, nt_data=nt_d, sensors_xy=xy, K=K, cfl=0.3,
                              c_lo=1300.0, c_hi=U, p0_lo=0.0, c_bg=1430.0, mem=20, iters=t2_iters, rtol=1e-5,
                              sigma_p0=2.5, prior_tau=1.5e-3, prior_eta_c=eta_c, prior_sigma_c=sig_c,
                              prior_eta_p0=5.0, prior_sigma_p0=2.5)
            t0 = time.perf_counter()
            c_r, p0_r, rows, status, ms = reconstruct(cfg, f32(y[:K]), f32(wts[:K]), f32(np.full((nf, nf), eta_c)))
            wall = time.perf_counter() - t0
            c_r, p0_r = c_r.cpu().numpy(), p0_r.cpu().numpy()
            row[f"K{K}"] = {"E_c": err(c_t, c_r), "E_p0_1": err(p0_t[0], p0_r[0]), "iterations": len(rows),
                            "wall_s": wall, "status": status,
                            "E_c_initial": err(c_t, np.full_like(c_t, eta_c))}
        pe = paper[kind]
        row["paper_table2"] = {"E_c_K4": pe[0], "E_c_K1": pe[1], "E_p0_1_K4": pe[2], "E_p0_1_K1": pe[3]}
        out[kind] = row
    return {"metric": "E_c and E_p0^1 (%) of the joint reconstruction, K=4 data sets vs K=1",
                      "unit": "%", "n_gpus": 1, "dtype": "f32", "data": "synthetic",
                      "config": {"workload": "simple phantoms of Sec. 4.1 on the paper's 236-sensor square, data "
                                             "on a finer grid than every reconstruction level, levels "
                                             f"{levels}, {t2_iters} iterations per level, OU prior"},
                      "results": out, "total_s": time.perf_counter() - t_all}


def run_warmstart(args):
    """Learned warm start (128x128, K=4): iterations and time to E_c <= 2 % with and without it."""
    import numpy as np
    import torch

    import paper_2505_08482_gb300 as pkg
    from paper_2505_08482_gb300 import _binding as B
    from paper_2505_08482_gb300.solver import ReconConfig, reconstruct_batched
    from paper_2505_08482_gb300.warmstart import (PairGenerator, UNet, init_params, iterations_to, predict_c,
                                                  relative_error, train)
    pkg.build()
    torch.cuda.set_device(0)
    n, K = 128, 4
    gen = PairGenerator(n=n, K=K, M=256, nt=600, batch=64)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    X, T, _ = gen.make(list(range(args.ws_train)))
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    net = UNet(4, 32, K, n, n, max_batch=32)
    net.set_params(init_params(4, 32, K, seed=1))
    t0 = time.perf_counter()
    launches0 = B.lib().pat_kernel_launches()
    hist = train(net, X, T, epochs=args.ws_epochs, batch=32, lr=1e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    train_launches = int(B.lib().pat_kernel_launches() - launches0)
    del X, T
    Xh, Th, raw = gen.make(list(range(10 ** 6, 10 ** 6 + args.ws_test)), keep_data=True)
    c_true = torch.stack([r["c_true"] for r in raw])
    c_warm = predict_c(net, Xh)
    c_plain = torch.stack([torch.full_like(ct, 0.5 * float(ct.min() + ct.max())) for ct in c_true])
    e_warm0 = relative_error(c_warm, c_true).cpu().numpy()
    e_plain0 = relative_error(c_plain, c_true).cpu().numpy()
    cfg = ReconConfig(levels=(64, 128), L=n * 1e-4, dt_data=gen.gs.dt, nt_data=gen.nt, sensors_xy=gen.sensors, K=K,
                      iters=args.ws_iters, mem=20, ckpt_every=32, rtol=0.0)
    arms = {}
    ep0_t = args.ws_ep0
    for name, cinit in (("plain", c_plain), ("warm", c_warm)):
        its, mss, fin, its2, mss2, finp = [], [], [], [], [], []
        t0 = time.perf_counter()
        for b0 in range(0, len(raw), 64):
            # E_c target alone (the instance leaves a level once E_c <= 2 %)
            insts = [dict(y_meas=r["y_meas"].contiguous(), w=r["w"].contiguous(), c_init=cinit[b0 + j].contiguous(),
                          c_true=r["c_true"].contiguous(), ec_target=2.0) for j, r in enumerate(raw[b0:b0 + 64])]
            res, _ = reconstruct_batched(cfg, insts)
            for c_rec, _, rows, _ in res:
                i_, m_ = iterations_to(rows, 2.0, 2)
                its.append(i_)
                mss.append(m_)
                fin.append([r["Ec"] for r in rows if r["level"] == 1][-1] if rows else None)
            # equal relative errors in c and p0: E_c <= 2 % and E_p0 <= ws_ep0 (Eq. RelativeError)
            insts = [dict(d, p0_true=r["p0_true"].contiguous(), ep0_target=ep0_t)
                     for d, r in zip(insts, raw[b0:b0 + 64])]
            res, _ = reconstruct_batched(cfg, insts)
            for c_rec, _, rows, _ in res:
                i_, m_ = iterations_to(rows, 2.0, 2, ep0_t)
                its2.append(i_)
                mss2.append(m_)
                finp.append([r["Ep0"] for r in rows if r["level"] == 1][-1] if rows else None)
        wall = time.perf_counter() - t0
        reached = [i for i in its if i is not None]
        reached2 = [i for i in its2 if i is not None]
        arms[name] = {"reached_2pct": len(reached) / len(its),
                      "iterations_median": float(np.median(reached)) if reached else None,
                      "ms_median": float(np.median([m for m in mss if m is not None])) if reached else None,
                      "final_Ec_median": float(np.median([f for f in fin if f is not None])),
                      "joint": {"E_c_pct": 2.0, "E_p0_pct": ep0_t, "reached": len(reached2) / len(its2),
                                "iterations_median": float(np.median(reached2)) if reached2 else None,
                                "ms_median": float(np.median([m for m in mss2 if m is not None]))
                                if reached2 else None,
                                "final_Ep0_median": float(np.median([f for f in finp if f is not None]))},
                      "wall_s": wall}
    line = {"metric": "learned warm start: iterations / time to E_c <= 2 %", "unit": "iterations",
            "value": arms["warm"]["iterations_median"], "higher_is_better": False, "n_gpus": 1, "dtype": "bf16+f32",
            "data": "synthetic",
            "config": {"workload": f"U-Net 4 levels x 32, {args.ws_train} solver-generated pairs (128x128, K=4, "
                                   f"M=256, Nt=600), {args.ws_test} held-out seeds, levels 64->128, "
                                   f"<= {args.ws_iters} L-BFGS iterations per level"},
            "pair_generation_s": t_gen, "training_s": t_train, "train_loss": hist, "training_launches": train_launches,
            "initial_Ec_median": {"plain": float(np.median(e_plain0)), "warm": float(np.median(e_warm0))},
            "arms": arms}
    print(json.dumps(line), flush=True)


def run_gemm(args):
    """TFLOP/s of the network's BF16 GEMM on both tensor-core paths (pat_gemm_bf16), on a large
    square product and on the shapes of the U-Net's convolutions at 128 x 128, batch 32."""
    import ctypes

    import torch

    import paper_2505_08482_gb300 as pkg
    from paper_2505_08482_gb300 import _binding as B
    pkg.build()
    torch.cuda.set_device(0)
    L = B.lib()
    peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    bf16_peak = float(peak.get("bf16_tflops", 1900.0))
    P = 32 * 128 * 128
    shapes = [("square 8192", 8192, 8192, 8192), ("square 4096", 4096, 4096, 4096),
              ("conv 3x3 32->32 fwd", P, 32, 288), ("conv 3x3 64->64 fwd (64^2)", P // 4, 64, 576),
              ("conv 3x3 256->256 fwd (16^2)", P // 64, 256, 2304), ("weight grad 32x288 over pixels", 32, 288, P)]
    rows = []
    st = torch.cuda.current_stream()
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    for name, M, N, K in shapes:
        A = torch.randn((M, K), device="cuda").to(torch.bfloat16)
        Bm = torch.randn((N, K), device="cuda").to(torch.bfloat16)
        C = torch.empty((M, N), dtype=torch.float32, device="cuda")
        status = torch.zeros((1,), dtype=torch.int32, device="cuda")
        row = {"shape": name, "M": M, "N": N, "K": K}
        for path in (0, 1):
            def call():
                rc = L.pat_gemm_bf16(ctypes.c_void_p(A.data_ptr()), K, ctypes.c_void_p(Bm.data_ptr()), K, M, N, K,
                                     ctypes.c_void_p(C.data_ptr()), N, path, ctypes.c_void_p(status.data_ptr()),
                                     ctypes.c_void_p(st.cuda_stream))
                assert rc == 0, L.pat_last_error()
            for _ in range(3):
                call()
            torch.cuda.synchronize()
            reps = 10
            ts = []
            for _ in range(reps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                call()
                e1.record(st)
                torch.cuda.synchronize()
                ts.append(e0.elapsed_time(e1))
            ms = statistics.median(ts)
            tf = 2.0 * M * N * K / (ms * 1e-3) / 1e12
            row[f"path{path}"] = {"ms": ms, "tflops": tf, "frac_of_bf16_peak": tf / bf16_peak}
        row["status"] = int(status.item())
        row["tcgen05_speedup"] = row["path0"]["ms"] / row["path1"]["ms"]
        rows.append(row)
        del A, Bm, C
    print(json.dumps({"metric": "BF16 GEMM TFLOP/s (C = A B^T, FP32 accumulation)", "unit": "TFLOP/s",
                      "bf16_peak_tflops": bf16_peak, "peak_kind": "measured bf16_tflops (burst)",
                      "paths": {"0": "mma.sync m16n8k16 (warp level)", "1": "tcgen05.mma + TMEM + TMA"},
                      "l2": "256 MiB written between timed calls", "rows": rows}), flush=True)


def run_profile_eval(args):
    """Gradient evaluations of the headline workload for ncu captures: one warm-up evaluation,
    then --profile-eval evaluations inside the NVTX range "profiled"; eager launches, no
    autotuning, no timing."""
    import numpy as np
    import torch

    import paper_2505_08482_gb300 as pkg
    from paper_2505_08482_gb300 import _binding as B
    from paper_2505_08482_gb300.solver import GridSpec, Plan
    pkg.build()
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    L = B.lib()
    w, c_init = inputs(0)
    n, K, M, nt = WL["n"], WL["K"], WL["M"], args.nt
    gs = GridSpec(n=n, pml=pml_auto(n), dx=WL["dx"], dt=WL["cfl"] * WL["dx"] / WL["c_hi"], nt=nt, c_ref=WL["c_hi"])
    plan = Plan(gs, w.sensors, K, ckpt_every=args.ckpt, device=dev)
    plan.variant = 0 if args.variant is None else args.variant
    f32 = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float32, device=dev)
    c0, p0 = f32(np.full((n, n), c_init)), f32(0.5 * w.p0_true)
    ym = f32(np.random.default_rng(0).standard_normal((K, nt, M)) * 0.01)
    wt = f32(np.ones(K))
    l0 = L.pat_kernel_launches()
    plan.adjoint_grad(c0, p0, ym, wt)
    torch.cuda.synchronize()
    print(f"launches_per_eval={L.pat_kernel_launches() - l0} (the library's kernels; memsets and copies are not "
          f"kernels)", file=sys.stderr, flush=True)
    torch.cuda.nvtx.range_push("profiled")   # ncu --nvtx --nvtx-include "profiled/" captures these
    for _ in range(args.profile_eval):
        plan.adjoint_grad(c0, p0, ym, wt)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()


def ctypes_read(L):
    import ctypes
    tot = ctypes.c_double(0.0)
    cnt = ctypes.c_longlong(0)
    rc = L.pat_timing_read(ctypes.byref(tot), ctypes.byref(cnt))
    if rc != 0:
        raise RuntimeError("pat_timing_read failed")
    return tot.value, cnt.value


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return
    if args.batch:
        run_batch(args)
        return
    if args.warmstart:
        run_warmstart(args)
        return
    if args.gemm:
        run_gemm(args)
        return
    if args.profile_eval:
        run_profile_eval(args)
        return
    if args.roofline_k:
        run_roofline_k(args)
        return
    if args.table2:
        run_table2(args)
        return
    if args.prior_cost:
        run_prior_cost(args)
        return
    if args.recon256:
        run_recon256(args)
        return
    if world > 1:
        import torch
        import torch.distributed as tdist
        torch.cuda.set_device(local_rank)
        tdist.init_process_group("nccl")
    run_ours(args, rank, world, local_rank)
    if world > 1:
        import torch.distributed as tdist
        tdist.destroy_process_group()


if __name__ == "__main__":
    main()
