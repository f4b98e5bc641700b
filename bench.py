#!/usr/bin/env python3
"""Benchmark of the 3DGS Levenberg-Marquardt hot path on one GB300.

Metric: LM-step ms and J p + J^T u HBM GB/s at 1.5M Gaussians, chosen form vs
plain FP32. One step = one LM iteration of the paper-scale synthetic workload
(1.5M Gaussians in 20 clusters, 200 cameras at 1264x832, four subsets of 25
views): per subset the gradient cache, the diagonal and the PCG solve
(Algorithm 1, 8 iterations, break test 0.01), then the weighted mean of the
subset directions, rho with the trial render at gamma = 1 and the damping
update (--line-search n adds Eq. line-search over n step scales).

Forms: "chosen" = BF16 cache, learned diagonal preconditioner (trained on the
GPU on step 0's subset systems before timing), the subsets' solves batched and
replayed from one CUDA graph; "plain" = FP32 cache, Jacobi, one subset after
another. Besides the paper's fixed 8 iterations, one LM step of each form is
also timed with PCG run to a relative residual of 1e-3 (equal_residual).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0). With N > 1 (launched by torch.distributed.run)
every rank runs an independent replica of the step; the line reports the max
over ranks. ``--impl reference`` times the FP64 CPU oracle on a bounded sample
of the same workload on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LM-step ms and J*p+J^T*u HBM GB/s at 1.5M Gaussians, chosen vs plain FP32"
CHOSEN_FORM = "chosen: 16-bit cache, batched subsets in CUDA graphs, preconditioner judged at 1e-3"
FALLBACK_HBM_GBS = 6800.0


def parse_args(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="paper")
    ap.add_argument("--cache-fmt", default="bf16", help="cache payload of the chosen form")
    ap.add_argument("--skip-plain", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--group", type=int, default=32)
    ap.add_argument("--subsets", type=int, default=0,
                    help="override: number of image subsets per LM step (profiling-sized cases)")
    ap.add_argument("--views", type=int, default=0, help="override: views per subset (profiling-sized cases)")
    ap.add_argument("--precond", choices=["learned", "jacobi"], default="learned",
                    help="preconditioner of the chosen form")
    ap.add_argument("--train-steps", type=int, default=12, help="Adam steps of the learned preconditioner")
    ap.add_argument("--train-K", type=int, default=8, help="unrolled PCG iterations of the training loss")
    ap.add_argument("--train-lr", type=float, default=3e-3)
    ap.add_argument("--train-systems", type=int, default=5,
                    help="train on the first subset system of each of LM steps 1..n")
    ap.add_argument("--skip-equal", action="store_true", help="skip the equal-residual comparison")
    ap.add_argument("--equal-cap", type=int, default=1000, help="PCG iteration cap of the equal-residual step")
    ap.add_argument("--equal-lambdas", default="1e-3,1,1e4",
                    help="LM dampings of the equal-residual steps (both forms), comma-separated")
    ap.add_argument("--cpu-views", type=int, default=1, help="views per subset of the CPU oracle sample")
    ap.add_argument("--detail", default="", help="also write the full record of the run to this JSON file")
    ap.add_argument("--cpu-suite", default="",
                    help="only time the oracle on the host (comma list of tiny, crop, medium_subset) and print it")
    ap.add_argument("--objective", choices=["l2", "l1ssim"], default="l2",
                    help="energy of the LM step: sum of squares (the timed configuration) or Eq. gn-loss")
    ap.add_argument("--line-search", type=int, default=0,
                    help="line-search candidates of the timed LM steps (0: gamma = 1, the workload's setting)")
    ap.add_argument("--equal-line-search", type=int, default=8,
                    help="line-search candidates of the equal-residual step")
    ap.add_argument("--apply-pass", action="store_true",
                    help="kernel mode: one cache of the first --apply-views cameras, then one J^T u and one J p "
                         "(for ncu captures); with --sweep, every kernel variant timed")
    ap.add_argument("--apply-views", type=int, default=8)
    ap.add_argument("--apply-variant", type=int, default=3, help="1..10: forced apply kernel variant 0..9")
    ap.add_argument("--sweep", action="store_true")
    ap.add_argument("--formats", default="",
                    help="with --apply-pass: cache formats to compare (e.g. fp32,bf16,thin): bytes and the times "
                         "of J p, J^T u and diag(J^T J) on the same views")
    return ap.parse_args(argv)


# ----------------------------------------------------------------------------- distributed
def dist_init(backend: str):
    import torch
    import torch.distributed as dist
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, None
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    dist.init_process_group(backend=backend)
    return dist.get_rank(), ws, dist


def max_over_ranks(x: float, dist, device=None) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(dist):
    if dist is not None:
        dist.barrier()


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while it runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int = 0):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=2)
        return self.summarize(self.lines)

    @staticmethod
    def summarize(lines) -> dict:
        """Median SM clock, maximum SM clock, the throttle reasons seen active and
        the largest power draw, from nvidia-smi CSV lines of FIELDS."""
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def load_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": FALLBACK_HBM_GBS, "source": "fallback"}


# A timed region that saw one of these is not a valid measurement; sw_power_cap
# is kept and reported.
BAD_CLOCK_REASONS = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown")


def clocks_rejected(clk) -> str:
    """Why a timed region's clock record voids its number ('' if it does not): a
    hardware or thermal slowdown seen, or a median SM clock under 85% of the
    maximum with no reason active (a clock lock left by another process)."""
    if not clk or clk.get("sm_mhz") is None:
        return ""
    bad = [r for r in clk.get("reasons", []) if r in BAD_CLOCK_REASONS]
    if bad:
        return "slowdown: " + ", ".join(bad)
    if clk.get("sm_max_mhz") and clk["sm_mhz"] < 0.85 * clk["sm_max_mhz"] and not clk.get("reasons"):
        return f"SM clock {clk['sm_mhz']:.0f} of {clk['sm_max_mhz']:.0f} MHz with no reason active"
    return ""


def agree_remeasure(why: str, dist, device=None) -> bool:
    """Whether any rank's timed region was void: every rank takes the same
    decision, so all of them time the steps again (or none does)."""
    return max_over_ranks(1.0 if why else 0.0, dist, device) > 0.0


# ----------------------------------------------------------------------------- workload
def workload(args):
    """The named workload, with the subset shape optionally overridden."""
    import dataclasses
    import synth
    wl = synth.WORKLOADS[args.workload]
    if args.subsets or args.views:
        ns = args.subsets or len(wl.subset_sizes)
        nv = args.views or wl.subset_sizes[0]
        wl = dataclasses.replace(wl, subset_sizes=[nv] * ns)
    return wl


def build_workload(wl, device):
    """Scene, cameras and GPU-rendered targets (perturbed copy + pixel noise), resident in HBM."""
    import numpy as np
    import torch
    import synth
    import paper_2409_12892_gb300 as g
    P = synth.make_gaussians(wl)
    cams = synth.make_cameras(wl)
    pert = g.to_soa(synth.perturbed_copy(wl, P), device=device)
    n_pix = g.n_pixels(cams)
    targets = torch.empty((n_pix, 3), dtype=torch.float32, device=device)
    ctx = g.Context()
    off = 0
    chunk = 25
    for i in range(0, len(cams), chunk):
        cc = cams[i:i + chunk]
        npx = g.n_pixels(cc)
        ctx.render(pert, P.shape[0], cc, img=targets[off:off + npx])
        off += npx
    del pert
    noise = torch.from_numpy(synth.pixel_noise(wl, n_pix * 3)).view(-1, 3).to(device)
    targets += noise
    del noise
    torch.cuda.synchronize()
    ctx.close()
    torch.cuda.empty_cache()      # hand torch's cached blocks back: the LM step's caches need the room
    return wl, P, cams, targets


def run_steps(g, ctx, params, N, cams, targets, wl, steps: int, warmup: int, dist, clocks=None):
    """W untimed then K timed LM steps; returns (ms_per_step, per-step stats, kernel launches)."""
    import torch
    import synth
    st = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lam, stats, launches0 = wl.lambda0, [], 0
    for s in range(warmup + steps):
        if s == warmup:
            barrier(dist)
            torch.cuda.synchronize()
            if clocks is not None:
                clocks.start()
            launches0 = g.kernel_launches()
            ev0.record(st)
        subsets = synth.subset_views(wl, s)
        ctx.memory_usage(reset_peak=True)         # host-side read of the pool's counters
        state, lm = ctx.lm_step(params, N, cams, targets, subsets, lam, s)
        lm.mem_peak = ctx.memory_usage()["peak"]
        lm.lam_in = lam
        lm.n_pix = sum(cams[v].width * cams[v].height for sub in subsets for v in sub)
        lam = state.lambda_
        if s >= warmup:
            stats.append(lm)
    ev1.record(st)
    torch.cuda.synchronize()
    barrier(dist)
    launches = g.kernel_launches() - launches0
    clk = clocks.stop() if clocks is not None else None
    ms = ev0.elapsed_time(ev1) / max(steps, 1)
    return ms, stats, launches, clk


def run_e2e(g, ctx, P_host, N, ld, cams, targets, wl, steps: int, warmup: int, dist):
    """The same step through the C ABI from pinned host buffers: each step copies
    the parameters and the targets of its views (one copy per view) to the
    device, runs the LM step and copies the parameters back. The targets of step
    s + 1 are copied on a second stream while step s runs (two device buffers,
    ordered by events); the parameters go up before and come back after each
    step on the step's own stream."""
    import numpy as np
    import torch
    import synth
    dev = targets.device
    h_params = g.to_soa(P_host, device="cpu", ld=ld).pin_memory()
    h_targets = targets.cpu().pin_memory()
    offs = np.cumsum([0] + [c.width * c.height for c in cams])
    d_params = torch.empty_like(h_params, device=dev)
    st = torch.cuda.current_stream()
    cp = torch.cuda.Stream(device=dev)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lam, h2d, d2h = wl.lambda0, 0, 0

    def plan(s):
        subsets = synth.subset_views(wl, s)
        views = [v for sub in subsets for v in sub]
        remap = {v: i for i, v in enumerate(views)}
        return views, [cams[v] for v in views], [[remap[v] for v in sub] for sub in subsets], \
            int(sum(offs[v + 1] - offs[v] for v in views))

    plans = [plan(s) for s in range(warmup + steps)]
    npx_max = max(p[3] for p in plans)
    bufs = [torch.empty((npx_max, 3), dtype=torch.float32, device=dev) for _ in range(2)]
    free = [torch.cuda.Event(), torch.cuda.Event()]     # the step that read the buffer has finished
    ready = [torch.cuda.Event(), torch.cuda.Event()]    # the buffer holds its step's targets

    def upload(s):
        views, _, _, _ = plans[s]
        k = s % 2
        with torch.cuda.stream(cp):
            cp.wait_event(free[k])
            o = 0
            for v in views:
                n = int(offs[v + 1] - offs[v])
                bufs[k][o:o + n].copy_(h_targets[offs[v]:offs[v + 1]], non_blocking=True)
                o += n
            ready[k].record(cp)

    for k in range(2):
        free[k].record(st)
    for s in range(warmup + steps):
        if s == warmup:
            barrier(dist)
            torch.cuda.synchronize()
            ev0.record(st)
        if s == 0 or s == warmup:     # the timed region copies its own first targets
            upload(s)
        views, cc, subs, npx = plans[s]
        k = s % 2
        d_params.copy_(h_params, non_blocking=True)
        st.wait_event(ready[k])
        if s + 1 < warmup + steps and s + 1 != warmup:
            upload(s + 1)
        state, _ = ctx.lm_step(d_params, N, cc, bufs[k][:npx], subs, lam, s)
        free[k].record(st)
        lam = state.lambda_
        h_params.copy_(d_params, non_blocking=True)
        if s >= warmup:
            h2d += npx * 12 + h_params.numel() * 4
            d2h += h_params.numel() * 4
    ev1.record(st)
    torch.cuda.synchronize()
    barrier(dist)
    return ev0.elapsed_time(ev1) / max(steps, 1), h2d // max(steps, 1), d2h // max(steps, 1)


# ----------------------------------------------------------------------------- CPU oracle sample
# Gaussians of the CPU sample: the trial render of the step at lambda0 draws
# splats whose log-scales grew by tens, each over the whole view, and sets the
# oracle's time; this many keep a sample step to a few seconds on 4 cores.
ORACLE_SAMPLE_GAUSSIANS = 200
ORACLE_SAMPLE = "oracle LM step: {ng} Gaussians nearest cluster 0's mean, 4 subsets x {vps} view"


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith(("model name", "cpu model")):
                    return ln.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_sample_inputs(workload: str = "paper", views_per_subset: int = 1, n_keep: int = ORACLE_SAMPLE_GAUSSIANS):
    """The crop's parameters, its subsets' cameras and targets (oracle renders of the perturbed crop)."""
    import warnings
    import numpy as np
    import synth
    from oracle import jacobian as J
    warnings.filterwarnings("ignore")
    wl = synth.WORKLOADS[workload]
    P = synth.make_gaussians(wl)
    cams = synth.make_cameras(wl)
    idx = synth.crop_2k(wl, P, n_keep)
    subsets = [[cams[v] for v in vs[:views_per_subset]] for vs in synth.subset_views(wl, 0)]
    Pc = P[idx].astype(np.float64)
    Pt = synth.perturbed_copy(wl, P)[idx].astype(np.float64)
    return wl, Pc, subsets, [J.render(Pt, cc) for cc in subsets]


def _oracle_subset_worker(conn):
    """One image subset of an oracle LM step in its own process: build and solve
    the subset's system, return (Delta_i, M_i, cost_i); then, given the combined
    Delta, return the subset's predicted and trial costs."""
    import os as _os
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        _os.environ[k] = "1"
    import warnings
    import numpy as np
    from oracle import jacobian as J, solver
    warnings.filterwarnings("ignore")
    while True:
        msg = conn.recv()
        if msg is None:
            return
        params, cams, tgt, lam, n_iters, brk = msg
        sys_ = solver.build_subset(params, cams, tgt)
        d, st = solver.solve_subset(sys_, lam, n_iters, brk)
        conn.send((d, sys_.M, sys_.cost, sum(vl.a.shape[0] for vl in sys_.lin)))
        delta = conn.recv()
        u = J.apply_J(sys_.lin, delta, sys_.F.shape[0]) + sys_.F
        cost1 = float(np.sum((J.render(params + delta, cams) - tgt) ** 2))
        conn.send((float(np.dot(u, u)), cost1))


def oracle_lm_step_timed(Pc, subsets, targets, lam, n_iters=8, brk=0.01, workers=1) -> dict:
    """Wall time of one oracle LM step (gamma = 1). workers = 1: oracle.solver.lm_step in
    this process; workers > 1: the subsets' independent parts (Eq. combine-pcg) run in
    one process each, the combine and rho here."""
    import multiprocessing as mp
    import numpy as np
    from oracle import solver
    if workers <= 1:
        t0 = time.perf_counter()
        r = solver.lm_step(Pc, subsets, targets, lam, n_iters=n_iters, break_rel2=brk)
        return {"ms": (time.perf_counter() - t0) * 1e3, "accepted": bool(r.accepted), "rho": r.rho,
                "cost": r.cost, "cost_new": r.cost_new}
    ctx = mp.get_context("spawn")
    procs, conns = [], []
    for _ in range(len(subsets)):
        a, b = ctx.Pipe()
        pr = ctx.Process(target=_oracle_subset_worker, args=(b,), daemon=True)
        pr.start()
        procs.append(pr)
        conns.append(a)
    try:
        for c in conns:             # workers up (imports done) before the clock starts
            c.send((Pc[:1], subsets[0][:1], targets[0][:subsets[0][0].width * subsets[0][0].height * 3],
                    lam, 0, 0.0))
            c.recv()
            c.send(np.zeros_like(Pc[:1]))
            c.recv()
        t0 = time.perf_counter()
        for c, cams, tgt in zip(conns, subsets, targets):
            c.send((Pc, cams, tgt, lam, n_iters, brk))
        out = [c.recv() for c in conns]
        delta = solver.combine([o[0] for o in out], [o[1] for o in out])
        cost0 = sum(o[2] for o in out)
        for c in conns:
            c.send(delta)
        pc_ = [c.recv() for c in conns]
        pred = sum(p_ for p_, _ in pc_)
        cost1 = sum(c_ for _, c_ in pc_)
        ms = (time.perf_counter() - t0) * 1e3
        den = cost0 - pred
        rho = (cost0 - cost1) / den if den > 0 else -math.inf
        return {"ms": ms, "accepted": bool(den > 0 and rho > 1e-5), "rho": rho, "cost": cost0, "cost_new": cost1,
                "entries": sum(o[3] for o in out)}
    finally:
        for c in conns:
            try:
                c.send(None)
            except (OSError, BrokenPipeError):
                pass
        for pr in procs:
            pr.join(timeout=10)


def cpu_baseline(workload: str = "paper", views_per_subset: int = 1) -> dict:
    """The oracle LM step on the crop sample, measured at 1 thread and at one process
    per subset (bounded by the host's cores), with the host CPU recorded."""
    wl, Pc, subsets, targets = oracle_sample_inputs(workload, views_per_subset)
    nproc = os.cpu_count() or 1
    one = oracle_lm_step_timed(Pc, subsets, targets, wl.lambda0, wl.pcg_iters, 0.01, workers=1)
    par = oracle_lm_step_timed(Pc, subsets, targets, wl.lambda0, wl.pcg_iters, 0.01, workers=len(subsets))
    w = min(nproc, len(subsets))
    return {"value": one["ms"], "unit": "ms per sample LM step", "cores": 1, "kind": "oracle",
            "sample": ORACLE_SAMPLE.format(ng=ORACLE_SAMPLE_GAUSSIANS, vps=views_per_subset),
            "cpu_model": cpu_model(), "host_cores": nproc,
            "threads_1_ms": one["ms"], "threads_nproc_ms": par["ms"], "threads_nproc_cores": w}


def cpu_suite(items=("tiny", "crop", "medium_subset")) -> dict:
    """The oracle timed outright on the host cores, for the record (not run by the
    default bench): the tiny workload's 5 LM steps (one subset, so one thread);
    the paper crop's LM step (2,000 Gaussians, step 0's 4 subsets x 1 view) at one
    thread and one process per subset; one 8-view subset of the medium workload
    (cache, diag and 8-iteration PCG) at one thread."""
    import warnings
    import numpy as np
    import synth
    from oracle import jacobian as J, solver
    warnings.filterwarnings("ignore")
    out = {"cpu_model": cpu_model(), "host_cores": os.cpu_count()}
    if "tiny" in items:
        wl = synth.WORKLOADS["tiny"]
        P = synth.make_gaussians(wl).astype(np.float64)
        cams = synth.make_cameras(wl)
        tgt = J.render(synth.perturbed_copy(wl, P).astype(np.float64), cams) + synth.pixel_noise(wl, sum(
            c.width * c.height * 3 for c in cams))
        lam, steps, t0 = wl.lambda0, [], time.perf_counter()
        for s in range(5):
            t1 = time.perf_counter()
            r = solver.lm_step(P, [cams], [tgt], lam, n_iters=wl.pcg_iters, break_rel2=0.01)
            steps.append({"ms": (time.perf_counter() - t1) * 1e3, "accepted": int(r.accepted), "lambda": lam})
            P, lam = r.params, r.lam
        out["tiny_5_lm_steps"] = {"ms": (time.perf_counter() - t0) * 1e3, "cores": 1, "steps": steps}
    if "crop" in items:
        wl, Pc, subsets, targets = oracle_sample_inputs("paper", 1, 2000)
        one = oracle_lm_step_timed(Pc, subsets, targets, wl.lambda0, wl.pcg_iters, 0.01, workers=1)
        par = oracle_lm_step_timed(Pc, subsets, targets, wl.lambda0, wl.pcg_iters, 0.01, workers=len(subsets))
        out["paper_crop_2k_lm_step"] = {"threads_1_ms": one["ms"], "procs_4_ms": par["ms"],
                                        "sample": "2,000 Gaussians nearest cluster 0's mean, 4 subsets x 1 view"}
    if "medium_subset" in items:
        wl = synth.WORKLOADS["medium"]
        P = synth.make_gaussians(wl).astype(np.float64)
        cams = synth.make_cameras(wl)
        vs = synth.subset_views(wl, 0)[0]
        cc = [cams[v] for v in vs]
        tgt = J.render(synth.perturbed_copy(wl, P).astype(np.float64), cc)
        t0 = time.perf_counter()
        sys_ = solver.build_subset(P, cc, tgt)
        t1 = time.perf_counter()
        solver.solve_subset(sys_, wl.lambda0, wl.pcg_iters, 0.01)
        t2 = time.perf_counter()
        out["medium_one_subset"] = {"build_ms": (t1 - t0) * 1e3, "pcg_ms": (t2 - t1) * 1e3, "cores": 1,
                                    "entries": int(sum(vl.a.shape[0] for vl in sys_.lin)),
                                    "views": len(cc)}
    return out


def cpu_baseline_subprocess(workload: str = "paper", views_per_subset: int = 1) -> dict:
    """cpu_baseline in a fresh process with one BLAS / OpenMP thread (no GPU state inherited)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    code = ("import json, bench; print(json.dumps(bench.cpu_baseline(%r, %d)))" % (workload, views_per_subset))
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_step_entries_estimate(workload: str = "paper", n_views: int = 2, tile_frac: float = 0.05) -> float:
    """Cache entries of one full LM step estimated with the oracle alone: blend a
    deterministic 5% sample of the tiles of two of step 0's views and scale to all
    tiles and to every view of the step."""
    import warnings
    import numpy as np
    import synth
    from oracle import projection, raster, conventions as cv
    warnings.filterwarnings("ignore")
    wl = synth.WORKLOADS[workload]
    P = synth.make_gaussians(wl).astype(np.float64)
    cams = synth.make_cameras(wl)
    subsets = synth.subset_views(wl, 0)
    views = [v for s in subsets for v in s]
    rng = np.random.default_rng(7)
    per_view = []
    for v in views[:n_views]:
        cam = cams[v]
        pr = projection.project(P, cam, want_jac=False)
        tx, ty = (cam.width + 15) // 16, (cam.height + 15) // 16
        tiles = rng.choice(tx * ty, max(1, int(tile_frac * tx * ty)), replace=False)
        order = raster.blend_order(pr)
        r = pr.rect[order]
        cnt = 0
        for t in tiles:
            x, y = t % tx, t // tx
            sel = order[(r[:, 0] <= x) & (x < r[:, 2]) & (r[:, 1] <= y) & (y < r[:, 3])]
            if sel.size == 0:
                continue
            gy, gx = np.meshgrid(np.arange(y * 16, min(cam.height, y * 16 + 16)),
                                 np.arange(x * 16, min(cam.width, x * 16 + 16)), indexing="ij")
            px, py = gx.ravel() + 0.5, gy.ravel() + 0.5
            yv = pr.y[sel]
            dx, dy = px[:, None] - yv[None, :, 0], py[:, None] - yv[None, :, 1]
            a = np.minimum(cv.ALPHA_MAX, yv[:, 5] * np.exp(-0.5 * (yv[:, 2] * dx * dx + yv[:, 4] * dy * dy)
                                                           - yv[:, 3] * dx * dy))
            valid = a >= cv.ALPHA_MIN
            om = np.where(valid, 1 - a, 1.0)
            Tb = np.concatenate([np.ones((om.shape[0], 1)), np.cumprod(om, 1)[:, :-1]], 1)
            stop = valid & (Tb * (1 - a) < cv.T_MIN)
            sa = np.where(stop.any(1), stop.argmax(1), sel.size)
            cnt += int((valid & (np.arange(sel.size)[None, :] < sa[:, None])).sum())
        per_view.append(cnt * (tx * ty) / len(tiles))
    return float(np.mean(per_view) * len(views))


# ----------------------------------------------------------------------------- arms
def run_reference(args):
    """The oracle on the host cores, on a bounded sample of the workload: each step is
    one oracle LM step on the crop sample (one process per image subset), and the
    value is that measured step's time, so that the steps fit the run's own clock.
    The same time scaled to one step of the whole workload by cache entries is
    reported beside it as an extrapolation, labelled so."""
    rank, ws, dist = dist_init("gloo")
    if rank != 0:
        return 0
    t_est0 = time.perf_counter()
    E_step = oracle_step_entries_estimate(args.workload)
    t_est = time.perf_counter() - t_est0
    wl, Pc, subsets, targets = oracle_sample_inputs(args.workload, args.cpu_views)
    runs = [oracle_lm_step_timed(Pc, subsets, targets, wl.lambda0, wl.pcg_iters, 0.01, workers=len(subsets))
            for _ in range(args.warmup + args.steps)][args.warmup:]
    value = statistics.mean(r["ms"] for r in runs)
    entries = runs[0]["entries"]
    nproc = os.cpu_count() or 1
    cb = {"value": value, "unit": "ms per sample LM step", "cores": min(nproc, len(subsets)), "kind": "oracle",
          "sample": ORACLE_SAMPLE.format(ng=ORACLE_SAMPLE_GAUSSIANS, vps=args.cpu_views), "cpu_model": cpu_model(),
          "host_cores": nproc, "value_kind": "measured: one oracle LM step of the sample, mean over the timed steps",
          "extrapolated_full_step_ms": value * E_step / max(entries, 1),
          "extrapolation": "the sample's ms x (cache entries of one workload step, estimated by the oracle on a "
                           "5% tile sample of two views) / (cache entries of the sample)",
          "sample_entries": entries, "step_entries_estimate": E_step, "estimate_seconds": t_est}
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "ms", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": value, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(args, CHOSEN_FORM), cache_fmt=args.cache_fmt),
        "cpu_baseline": cb,
        "e2e": {"value": value, "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(sig(line)), flush=True)
    return 0


def workload_config(args, form: str) -> dict:
    wl = workload(args)
    return {
        "workload": (f"{wl.name}: {wl.n_gaussians / 1e6:g}M Gaussians ({wl.n_clusters} clusters), "
                     f"{wl.n_cameras} cameras {'/'.join(f'{w}x{h}' for w, h in wl.resolutions)}, "
                     + (f"{len(wl.subset_sizes)}x{wl.subset_sizes[0]}" if len(set(wl.subset_sizes)) == 1
                        else "+".join(str(v) for v in wl.subset_sizes))
                     + " views per LM step"),
        "form": form, "pcg_iters": wl.pcg_iters, "break_rel2": 0.01, "lambda0": wl.lambda0,
        "line_search": args.line_search, "objective": args.objective,
        "l2_flush": "inputs larger than L2",
        "parallelism": f"{args.gpus} independent replicas" if args.gpus > 1 else "single GPU",
    }


def summarize_phases(stats) -> dict:
    names = ["build_cache", "jacobi_diag", "tangent", "apply_J", "apply_JT", "adjoint", "pcg_vector", "rho"]
    out = {}
    for i, n in enumerate(names):
        out[n] = statistics.mean(s.ms_phase[i] for s in stats)
    return out


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum, one-pass ncu
# captures) per algorithmic byte of the J p + J^T u pair (tangent, tile kernels,
# per-splat sums, adjoint), tile-kernel variant 9: BF16 from every pair kernel of
# one LM step of the 1.5M-Gaussian workload (4 subsets x 9 pairs: 1343.6 GB for
# 36 pairs of 29.38 GB); FP32 from one pair of a 25-view subset of the same
# workload (63.18 GB for 55.21 GB). The pair's traffic grows with its entries,
# pixels and splats, so a launch's traffic is this ratio times its algorithmic
# bytes.
PAIR_DRAM_PER_ALG_BYTE = {0: 1.144, 1: 1.270}   # FP32, BF16


def pair_roofline(stats, peak: dict, fmt: int = None) -> dict:
    t = sum(s.ms_phase[2] + s.ms_phase[3] + s.ms_phase[4] + s.ms_phase[5] for s in stats) / 1e3
    b = sum(s.pair_bytes for s in stats)
    n = sum(s.n_pairs for s in stats)
    gbs = b / t / 1e9 if t > 0 else 0.0
    ratio = PAIR_DRAM_PER_ALG_BYTE.get(fmt)
    return {"bound": "hbm", "achieved": gbs, "peak": peak["hbm_gbs"], "unit": "GB/s",
            "frac": gbs / peak["hbm_gbs"],
            "traffic": ratio * b / max(n, 1) if ratio is not None else None,
            "bytes_per_pair": b / max(n, 1), "ms_per_pair": t * 1e3 / max(n, 1),
            "peak_source": "measured" if peak["source"] == "measured" else "fallback 6.8 TB/s"}


def subset_targets(targets, cams, views):
    """The rows of `targets` that belong to `views`, concatenated (device copy)."""
    import numpy as np
    import torch
    offs = np.cumsum([0] + [c.width * c.height for c in cams])
    return torch.cat([targets[int(offs[v]):int(offs[v + 1])] for v in views])


def train_precond(g, ctx, params, N, cams, targets, wl, args):
    """The learned preconditioner, trained on the GPU (Adam on the unrolled-PCG
    residual) on the first subset system of each of LM steps 1..train_systems, at
    the damping each of those steps runs at when the steps before it are rejected
    (lambda0 2^s). Returns (network, report)."""
    import torch
    import synth
    t0 = time.perf_counter()
    steps = list(range(1, max(1, args.train_systems) + 1))
    systems = []
    for s in steps:
        vs = synth.subset_views(wl, s)[0]
        cc = [cams[v] for v in vs]
        cache = ctx.build_cache(params, N, cc, subset_targets(targets, cams, vs), want_F=False)
        diag = ctx.jacobi_diag(cache)
        lam = min(max(wl.lambda0 * 2.0 ** s, wl.lambda_min), wl.lambda_max)
        systems.append((cache, diag, ctx.precond_features(cache, diag), lam))
    pc = g.Precond(ctx, seed=0)
    pc.fit_standardizer(torch.cat([phi for _, _, phi, _ in systems]))
    losses = []
    for _ in range(args.train_steps):
        L = 0.0
        for cache, diag, phi, lam in systems:
            L += pc.accumulate(cache, phi, cache.b, diag, lam, args.train_K, 1.0 / len(systems))
        losses.append(L / len(systems))
        pc.adam(args.train_lr)
    # cost of using the network on one subset: features and inference
    cache, diag, _, _ = systems[0]
    st = torch.cuda.current_stream()
    e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    e0.record(st)
    phi = ctx.precond_features(cache, diag)
    e1.record(st)
    pc.apply(phi, diag)
    e2.record(st)
    torch.cuda.synchronize()
    for cache, _, _, _ in systems:
        cache.free()
    del systems, phi
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    rep = {"systems": [f"step {s}, first subset, lambda {min(max(wl.lambda0 * 2.0 ** s, wl.lambda_min), wl.lambda_max):g}"
                       for s in steps],
           "adam_steps": args.train_steps, "K": args.train_K, "lr": args.train_lr,
           "loss_first": losses[0] if losses else None, "loss_last": losses[-1] if losses else None,
           "seconds": time.perf_counter() - t0, "features_ms": e0.elapsed_time(e1), "inference_ms": e1.elapsed_time(e2),
           "weights": "bfloat16 weight matrices, float32 biases, float32 activations and sums",
           "loss": "1/2 log(||r_K||^2/||b||^2) after K iterations of Algorithm 1 with D"}
    return pc, rep


def judge_precond(g, ctx, pc, params, N, cams, targets, wl, lambdas, cap: int = 200, rel: float = 1e-3) -> dict:
    """The rule for keeping the learned preconditioner: on LM step 0's first subset
    system, PCG iterations to ||r|| <= rel ||b|| with the network against Jacobi at
    every damping in `lambdas` (the values the timed steps run at, from lambda0 up);
    the network is kept only if it needs fewer iterations than Jacobi at each of them."""
    import synth
    vs = synth.subset_views(wl, 0)[0]
    cache = ctx.build_cache(params, N, [cams[v] for v in vs], subset_targets(targets, cams, vs), want_F=False)
    diag = ctx.jacobi_diag(cache)
    D = pc.apply(ctx.precond_features(cache, diag), diag)
    rows = []
    ctx.set_options(n_iters=cap, break_rel2=rel * rel)
    for lam in lambdas:
        row = {"lambda": lam}
        for name, pre in (("jacobi", None), ("learned", D)):
            _, st, _ = ctx.pcg_solve(cache, cache.b, diag, lam, precond=pre)
            row[name] = st.iters if st.rr <= rel * rel * st.bb else None
        rows.append(row)
    ctx.set_options(n_iters=wl.pcg_iters, break_rel2=0.01)
    cache.free()
    keep = all(r["learned"] is not None and (r["jacobi"] is None or r["learned"] < r["jacobi"]) for r in rows)
    return {"iters_to_1e-3": rows, "cap": cap, "keep_learned": keep,
            "rule": "keep the network only if it reaches ||r|| <= 1e-3 ||b|| in fewer PCG iterations than Jacobi "
                    "at every damping the timed steps use"}


def psnr_from_cost(cost: float, n_pix: int) -> float:
    mse = cost / (3.0 * n_pix)
    return 10.0 * math.log10(1.0 / mse) if mse > 0 else float("inf")


def equal_residual_step(g, ctx, P, N, ld, cams, targets, wl, dev, cap: int, pc=None, lam: float = 1e-3,
                        ls: int = 8, ls_timed: int = 0) -> dict:
    """One LM step from the initial parameters with every subset's PCG run to
    ||r|| <= 1e-3 ||b|| (at most `cap` iterations), with the network `pc` as
    preconditioner or Jacobi; device time by CUDA events."""
    import torch
    import synth
    ctx.set_precond(pc)
    ctx.set_options(n_iters=cap, break_rel2=1e-6, line_search=ls)
    params = g.to_soa(P, device=dev, ld=ld)
    subsets = synth.subset_views(wl, 0)
    st = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(st)
    state, lm = ctx.lm_step(params, N, cams, targets, subsets, lam, 0)
    ev1.record(st)
    torch.cuda.synchronize()
    n_pix = sum(cams[v].width * cams[v].height for s in subsets for v in s)
    ctx.set_options(n_iters=wl.pcg_iters, break_rel2=0.01, line_search=ls_timed)
    ctx.set_precond(None)
    del params
    after = lm.cost_new if lm.accepted else lm.cost
    return {"ms": ev0.elapsed_time(ev1), "precond": "learned" if pc is not None else "jacobi", "lambda": lam,
            "gamma": lm.gamma,
            "reached": lm.pcg_iters < cap * len(subsets), "pcg_iters_total": lm.pcg_iters,
            "pcg_iters_per_subset": lm.pcg_iters / len(subsets), "accepted": int(lm.accepted), "rho": lm.rho,
            "cost": lm.cost, "cost_new": lm.cost_new, "predicted": lm.predicted,
            "psnr_before_db": psnr_from_cost(lm.cost, n_pix), "psnr_after_db": psnr_from_cost(after, n_pix)}


def profiled_step(g, ctx, params, N, cams, targets, wl, step: int):
    """One extra LM step with per-phase CUDA events (the timed steps run without them)."""
    import synth
    ctx.set_options(profile=1)
    state, lm = ctx.lm_step(params, N, cams, targets, synth.subset_views(wl, step), wl.lambda0, step)
    ctx.set_options(profile=0)
    return lm


def sig(x, n: int = 4):
    """x rounded to n significant digits (recursively through lists and dicts), so
    that the JSON line stays short; a non-finite float becomes null (strict JSON:
    e.g. rho of a step whose trial render overflowed or whose model predicts no
    decrease), and a float that rounds to a whole number prints without its ".0"."""
    if isinstance(x, float):
        if not math.isfinite(x):
            return None
        if x == 0.0:
            return 0
        r = float(f"{x:.{n}g}")
        return int(r) if r.is_integer() and abs(r) < 1e15 else r
    if isinstance(x, dict):
        return {k: sig(v, n) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [sig(v, n) for v in x]
    return x


def timed_lambdas(wl, steps: int, warmup: int) -> list:
    """Dampings the judge checks: lambda0 and the first and last damping of the timed
    steps when every step is rejected (lambda doubles per rejection), clamped."""
    cl = lambda v: min(max(v, wl.lambda_min), wl.lambda_max)
    return sorted({cl(wl.lambda0), cl(wl.lambda0 * 2.0 ** warmup), cl(wl.lambda0 * 2.0 ** (warmup + steps - 1))})


def equal_forms(g, ctx, pc, P, N, ld, cams, targets, wl, dev, lambdas, cap, args, with_learned) -> dict:
    """equal_residual_step at each damping: Jacobi, and the network capped at Jacobi's iterations."""
    out = {}
    for lam in lambdas:
        ej = equal_residual_step(g, ctx, P, N, ld, cams, targets, wl, dev, cap, lam=lam,
                                 ls=args.equal_line_search, ls_timed=args.line_search)
        row = {"jacobi": ej}
        if with_learned and pc is not None:
            cap_l = max(1, int(math.ceil(ej["pcg_iters_per_subset"])))
            row["learned"] = equal_residual_step(g, ctx, P, N, ld, cams, targets, wl, dev, cap_l, pc, lam=lam,
                                                 ls=args.equal_line_search, ls_timed=args.line_search)
        out[lam] = row
    return out


def run_ours(args):
    import torch
    import paper_2409_12892_gb300 as g
    from paper_2409_12892_gb300 import build as b
    rank, ws, dist = dist_init("nccl")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    b.build() if rank == 0 else None
    barrier(dist)
    g.load_library()
    peak = load_peaks()
    wl = workload(args)
    wl, P, cams, targets = build_workload(wl, dev)
    N = P.shape[0]
    ld = g.padded_ld(N)
    eq_lams = [float(v) for v in args.equal_lambdas.split(",") if v.strip()]
    result = {}
    forms = [("chosen", args.cache_fmt)]
    if not args.skip_plain:
        forms.append(("plain", "fp32"))
    for form, fmt in forms:
        chosen = form == "chosen"
        ctx = g.Context(cache_fmt=fmt, n_iters=wl.pcg_iters, break_rel2=0.01, lambda_min=wl.lambda_min,
                        lambda_max=wl.lambda_max, profile=not chosen, group=args.group, batch=chosen, graph=chosen,
                        line_search=args.line_search, objective=args.objective)
        params = g.to_soa(P, device=dev, ld=ld)
        pc, train, judge = None, None, None
        if chosen and args.precond == "learned":
            pc, train = train_precond(g, ctx, params, N, cams, targets, wl, args)
            judge = judge_precond(g, ctx, pc, params, N, cams, targets, wl,
                                  timed_lambdas(wl, args.steps, args.warmup))
            if judge["keep_learned"]:
                ctx.set_precond(pc)
        clocks = ClockSampler(local) if chosen else None
        ms, stats, launches, clk = run_steps(g, ctx, params, N, cams, targets, wl, args.steps, args.warmup, dist,
                                             clocks)
        remeasured = None
        if chosen:
            why = clocks_rejected(clk)
            if agree_remeasure(why, dist, dev):   # measured again, once
                remeasured = {"first_ms": ms, "first_clocks": clk, "why": why or "another rank's clock record"}
                ms, stats, launches, clk = run_steps(g, ctx, params, N, cams, targets, wl, args.steps, args.warmup,
                                                     dist, ClockSampler(local))
        ms = max_over_ranks(ms, dist, dev)
        prof = [profiled_step(g, ctx, params, N, cams, targets, wl, args.warmup + args.steps)] if chosen else stats
        result[form] = {"ms": ms, "stats": stats, "prof": prof, "launches": launches, "clocks": clk, "fmt": fmt,
                        "remeasured": remeasured,
                        "autotune": ctx.autotune_info(), "train": train, "judge": judge,
                        "precond": "learned" if (judge or {}).get("keep_learned") else "jacobi"}
        if chosen and not args.skip_e2e:
            e2e_ms, h2d, d2h = run_e2e(g, ctx, P, N, ld, cams, targets, wl, args.steps, args.warmup, dist)
            result["e2e"] = {"value": max_over_ranks(e2e_ms, dist, dev), "unit": "ms", "h2d_bytes_per_step": h2d,
                             "d2h_bytes_per_step": d2h}
        del params
        torch.cuda.empty_cache()
        if not args.skip_equal:
            ctx.set_precond(None)
            result[form]["equal"] = equal_forms(g, ctx, pc, P, N, ld, cams, targets, wl, dev, eq_lams,
                                                args.equal_cap, args, chosen)
        ctx.set_precond(None)
        if pc is not None:
            pc.free()
        ctx.close()
        torch.cuda.empty_cache()
    if rank != 0:
        return 0
    ch = result["chosen"]
    stats = ch["stats"]
    E_step = statistics.mean(s.cache_entries for s in stats)
    pre = "learned preconditioner" if ch["precond"] == "learned" else "Jacobi"
    fmt_name = {"fp32": "f32", "bf16": "bf16-cache/f32-accumulate", "fp16s": "f16-scaled-cache/f32-accumulate"}
    detail = {}
    line = {
        "metric": METRIC, "value": ch["ms"], "unit": "ms", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ch["ms"], "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": fmt_name.get(ch["fmt"], ch["fmt"]), "data": "synthetic",
        "gpu_launches": ch["launches"] // max(args.steps, 1),
        "config": dict(workload_config(args, CHOSEN_FORM), cache_fmt=ch["fmt"]),
        "precond": ch["precond"],
        "roofline": pair_roofline(ch["prof"], peak, {"fp32": 0, "bf16": 1, "fp16s": 2}.get(ch["fmt"])),
        "e2e": result.get("e2e"),
        "clocks": {k: v for k, v in (ch["clocks"] or {}).items() if k in ("sm_mhz", "sm_max_mhz", "reasons")},
        "phase_ms": sig(summarize_phases(ch["prof"]), 3),
        "lm": {"lambda": sig([s.lam_in for s in stats], 2),
               "accepted": "".join(str(int(s.accepted)) for s in stats),
               "rho": sig([s.rho for s in stats], 2), "pcg_iters": [s.pcg_iters for s in stats],
               "trial_overflows": sum(s.trial_overflows for s in stats),
               "psnr_first_last": [psnr_from_cost(stats[0].cost, stats[0].n_pix),
                                   psnr_from_cost(stats[-1].cost_new if stats[-1].accepted else stats[-1].cost,
                                                  stats[-1].n_pix)],
               "cache_entries": E_step, "cache_gb": statistics.mean(s.cache_bytes for s in stats) / 1e9,
               "device_peak_gb": max(s.mem_peak for s in stats) / 1e9},
    }
    detail["lm_ms"] = [s.ms_total for s in stats]
    detail["clocks"] = ch["clocks"]
    if ch["remeasured"] is not None:
        line["clocks_remeasured"] = ch["remeasured"]
    if ch["judge"] is not None:
        line["precond_judge"] = {"keep": ch["judge"]["keep_learned"],
                                 "iters_to_1e-3": [[r["lambda"], r["jacobi"], r["learned"]]
                                                   for r in ch["judge"]["iters_to_1e-3"]]}
        detail["precond_judge"] = ch["judge"]
        detail["precond_training"] = ch["train"]
    if "plain" in result:
        pl = result["plain"]
        rf = pair_roofline(pl["stats"], peak, 0)
        line["plain_fp32"] = {"ms": pl["ms"], "pair_frac": rf["frac"]}
        line["speedup_vs_plain"] = pl["ms"] / ch["ms"]
        detail["plain_fp32"] = {"roofline": rf, "autotune": pl["autotune"], "phase_ms": summarize_phases(pl["stats"]),
                                "cache_gb": statistics.mean(s.cache_bytes for s in pl["stats"]) / 1e9}
    if "equal" in ch:
        eqs, short = {}, []
        for lam, row in ch["equal"].items():
            cands = [e for e in (row.get("learned"), row["jacobi"]) if e is not None and e["reached"]]
            best = min(cands, key=lambda e: e["ms"]) if cands else row["jacobi"]
            ent = {"chosen": best, "chosen_jacobi": row["jacobi"], "chosen_learned": row.get("learned")}
            # per damping: ms [chosen, plain], iterations per subset, reached / accepted
            # [chosen, plain], speedup
            # PSNR gains of the two forms (dB); the PSNR before the step once, beside the steps
            srow = {"lambda": lam, "ms": [best["ms"]], "its": best["pcg_iters_per_subset"],
                    "reached": [int(best["reached"])], "accepted": [best["accepted"]],
                    "psnr_gain": [best["psnr_after_db"] - best["psnr_before_db"]]}
            psnr_before = best["psnr_before_db"]   # the same initial parameters at every damping
            if best["precond"] != "jacobi":
                srow["precond"] = best["precond"]
            pe = result.get("plain", {}).get("equal", {}).get(lam)
            if pe is not None:
                pj = pe["jacobi"]
                ent["plain_fp32_jacobi"] = pj
                srow["ms"].append(pj["ms"])
                srow["reached"].append(int(pj["reached"]))
                srow["accepted"].append(pj["accepted"])
                srow["psnr_gain"].append(pj["psnr_after_db"] - pj["psnr_before_db"])
                srow["psnr_after_diff_db"] = best["psnr_after_db"] - pj["psnr_after_db"]
                srow["speedup"] = pj["ms"] / best["ms"]
            eqs[lam] = ent
            short.append(srow)
        line["equal_residual"] = {"cap": args.equal_cap, "psnr_before": psnr_before, "steps": short}
        detail["equal_residual"] = {str(k): v for k, v in eqs.items()}
    if not args.skip_cpu:
        cb = cpu_baseline_subprocess(args.workload, args.cpu_views)
        line["cpu_baseline"] = cb
    detail["autotune"] = ch["autotune"]
    line = sig(line)
    if args.detail:
        with open(args.detail, "w") as f:
            json.dump(sig(dict(detail, line=line), 6), f, indent=1)
    print(json.dumps(line), flush=True)
    return 0


def run_apply_pass(args):
    """One subset cache (FP32, or --cache-fmt) of the first --apply-views cameras of the
    workload, then one J^T u and one J p with a forced kernel variant; with --sweep the
    median of 5 timed calls of each variant (CUDA events), as one JSON line."""
    import numpy as np
    import torch
    import synth
    import paper_2409_12892_gb300 as g
    from paper_2409_12892_gb300 import build as b
    b.build()
    wl = workload(args)
    P = synth.make_gaussians(wl)
    cams = synth.make_cameras(wl)[:args.apply_views]
    N = P.shape[0]
    params = g.to_soa(P)
    ctx = g.Context(cache_fmt=args.cache_fmt, autotune=False, apply_variant=args.apply_variant)
    tg = torch.empty((g.n_pixels(cams), 3), device="cuda")
    ctx.render(g.to_soa(synth.perturbed_copy(wl, P)), N, cams, img=tg)
    cache = ctx.build_cache(params, N, cams, tg)
    info = cache.info()
    u = torch.from_numpy(synth.random_vector(5, (g.n_pixels(cams), 3)).astype(np.float32)).cuda()
    p = torch.from_numpy(synth.random_vector(3, (59, cache.ld)).astype(np.float32)).cuda()
    gout = ctx.apply_JT(cache, u)
    uo = ctx.apply_J(cache, p)
    torch.cuda.synchronize()
    free_b, total_b = torch.cuda.mem_get_info()
    out = {"mode": "apply-pass", "workload": wl.name, "views": len(cams), "cache_fmt": args.cache_fmt,
           "entries": info.entries, "segments": info.segments, "pixels": info.pixels, "splats": info.splats,
           "active_splats": info.active_splats, "cache_bytes": info.bytes,
           "device_free_gb": free_b / 1e9, "device_total_gb": total_b / 1e9}
    if args.sweep:
        pay = 16 if args.cache_fmt == "fp32" else 8
        for v in range(1, 11):
            ctx.set_options(apply_variant=v)
            for name, call in (("J", lambda: ctx.apply_J(cache, p, uo)), ("JT", lambda: ctx.apply_JT(cache, u, gout))):
                ts = []
                for r in range(6):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    call()
                    e1.record()
                    torch.cuda.synchronize()
                    if r:
                        ts.append(e0.elapsed_time(e1))
                ms = float(np.median(ts))
                out[f"{name}_variant{v - 1}_ms"] = ms
                out[f"{name}_variant{v - 1}_entry_GBps"] = info.entries * (pay + 1) / ms / 1e6
    print(json.dumps(out), flush=True)
    cache.free()
    ctx.close()
    return 0


def run_format_pass(args):
    """Per cache format, one cache of the first --apply-views cameras: device bytes,
    build time and the median of 5 timed J p (with the tangent), J^T u (with the
    per-splat sums and the adjoint) and diag(J^T J) calls (CUDA events), one JSON line."""
    import numpy as np
    import torch
    import synth
    import paper_2409_12892_gb300 as g
    from paper_2409_12892_gb300 import build as b
    b.build()
    wl = workload(args)
    P = synth.make_gaussians(wl)
    cams = synth.make_cameras(wl)[:args.apply_views]
    N = P.shape[0]
    params = g.to_soa(P)
    tg = torch.empty((g.n_pixels(cams), 3), device="cuda")
    g.Context().render(g.to_soa(synth.perturbed_copy(wl, P)), N, cams, img=tg)
    u = torch.from_numpy(synth.random_vector(5, (g.n_pixels(cams), 3)).astype(np.float32)).cuda()
    out = {"mode": "format-pass", "workload": wl.name, "views": len(cams)}

    def timed(call, reps=6):
        ts = []
        for r in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            call()
            e1.record()
            torch.cuda.synchronize()
            if r:
                ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))

    for fmt in args.formats.split(","):
        ctx = g.Context(cache_fmt=fmt)
        torch.cuda.synchronize()
        cache = ctx.build_cache(params, N, cams, tg)
        cache.free()
        t_build = timed(lambda: ctx.build_cache(params, N, cams, tg).free(), reps=3)
        cache = ctx.build_cache(params, N, cams, tg)
        info = cache.info()
        p = torch.from_numpy(synth.random_vector(3, (59, cache.ld)).astype(np.float32)).cuda()
        uo = ctx.apply_J(cache, p)
        go = ctx.apply_JT(cache, u)
        dg = ctx.jacobi_diag(cache)
        out[fmt] = {"entries": info.entries, "segments": info.segments, "bytes": info.bytes,
                    "build_ms": t_build, "J_ms": timed(lambda: ctx.apply_J(cache, p, uo)),
                    "JT_ms": timed(lambda: ctx.apply_JT(cache, u, go)),
                    "diag_ms": timed(lambda: ctx.jacobi_diag(cache, dg))}
        cache.free()
        ctx.close()
        torch.cuda.empty_cache()
    print(json.dumps(sig(out)), flush=True)
    return 0


def main(argv=None):
    args = parse_args(argv)
    if args.cpu_suite:
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            os.environ.setdefault(k, "1")
        print(json.dumps(sig(cpu_suite(tuple(args.cpu_suite.split(","))))), flush=True)
        return 0
    if args.apply_pass and args.formats:
        return run_format_pass(args)
    if args.apply_pass:
        return run_apply_pass(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
