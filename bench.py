"""Benchmark of the CoNCPD-APG hot path on GB300.

A step is one APG iteration (Algorithm 1: every mode of every block, the
objective and, when F rises, the w = 0 re-update) over the resident tensors
of the workload.  Default workload: K = 5 coupled tensors of 256^3 in FP32,
R = 10, L = [3, 3, 0], 10 dB noise (the simulation workload at scale).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload NAME] [--storage f32|bf16|bf16x2] [--lra]
    python bench.py --time-to-fit [--workload NAME]

Prints one JSON line (rank 0).  The default line also carries a
"time_to_fit" record on the precision workload (4 x 512 x 512 x 256, R = 20):
seconds from cncpd_create on device-resident FP32 tensors until the global
Fit, evaluated on the original FP32 tensors, is within 1e-4 of the FP64
oracle's converged Fit, for FP32, BF16 and BF16 hi+lo storage, and a
"workloads" record: iterations/s and the dominant pass's roofline on that
workload in BF16 and BF16 hi+lo storage and on the 16 uneven fourth-order
EEG-shaped blocks (FP32), and "time_to_fit_lra": the same measurement on the
face shape (8 x 400x400x160, sparse first mode) for FP32, BF16 and BF16 with
the LRA step of lraCoNCPD-APG (R~ = 30).  The tensors (5 x 67 MB) exceed the 129 MB
L2, so no flush is needed between iterations.  --lra runs the low-rank
approximation step of lraCoNCPD-APG (rank R~ of the workload) before the
timed iterations, which then use the collapsed products.  --time-to-fit
prints that record alone for --workload (with a BF16 + LRA arm when the
workload has an R~).  The roofline's pass times are CUDA
events around each tensor pass of every 8th iteration of the timed region.
"""

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

UNIT = "iterations/s"


def _metric(w, storage):
    dims = "x".join(str(d) for d in w.dims[0]) if len(set(map(tuple, w.dims))) == 1 else "uneven"
    return (f"APG iterations/s (coupled NCP sweep, X in {storage.upper()}, FP32 factors, "
            f"{w.K} blocks of {dims}, R={w.R})")


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return ws, rank


def _max_over_ranks(ms, ws, device):
    """Largest per-rank time of the timed region (every rank must call it)."""
    if ws <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_value(steps, ws, ms):
    """Whole-job iterations/s: every rank runs `steps` iterations of its own
    replica (weak scaling), timed by the slowest rank."""
    return steps * ws / (ms / 1e3)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def _traffic(kernel, workload, storage):
    """DRAM bytes per launch of ``kernel`` from the committed ncu summary
    (profiles/<kernel>_<workload>[_bf16].md), if the kernel's source file is
    unchanged since it was captured."""
    name = f"{kernel}_{workload}" + ("" if storage in (None, "f32") else f"_{storage}")
    path = os.path.join(ROOT, "profiles", name + ".md")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    h = re.search(r"source_sha256:\s*([0-9a-f]+)", txt)
    f = re.search(r"source_file:\s*(\S+)", txt)
    if not m or not h:
        return None
    src_name = f.group(1) if f else "mttkrp_tma.cu"
    src = open(os.path.join(ROOT, "paper_2302_05119_gb300", "csrc", src_name), "rb").read()
    if hashlib.sha256(src).hexdigest() != h.group(1):
        return None
    return float(m.group(1))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _workload(name):
    import synth
    return synth.workload(name)


def _fit_target(w):
    """The FP64 oracle's converged global Fit for workload ``w`` (written by
    tests/golden/make_fit_targets.py, which calls only the oracle), or None."""
    p = os.path.join(ROOT, "tests", "golden", "fit_targets.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        rec = json.load(f).get(w.name)
    if not rec or rec.get("seed") != w.seed or rec.get("R") != w.R or rec.get("L") != w.L:
        return None
    return rec


def _pass_roofline(w, storage, s):
    """(dominant pass, its algorithmic GB/s, fraction of the measured HBM peak)
    from the CUDA-event pass times of a profiled step call."""
    es = {"f32": 4, "bf16": 2, "bf16x2": 4}[storage]
    h = (w.N + 1) // 2
    R = w.ranks()
    x_bytes = sum(w.elements()) * es
    trail = x_bytes + sum((int(np.prod(d[:h])) + sum(d[h:])) * r * 4 for d, r in zip(w.dims, R))
    lead = x_bytes + sum((int(np.prod(d[h:])) + sum(d[:h])) * r * 4 for d, r in zip(w.dims, R))
    nl = max(1, s["stream_launches"] // 2)
    t_trail, t_lead = s["trail_ms"] / nl, s["lead_ms"] / nl
    kern, t, b = ("lead_contract", t_lead, lead) if t_lead >= t_trail else ("trailing_contract", t_trail, trail)
    if s["stream_launches"] == 0 or t <= 0:
        return None
    peak, _ = _peaks()
    gbs = b / (t / 1e3) / 1e9
    return {"kernel": kern, "achieved_gbs": gbs, "frac": gbs / peak, "pass_ms": t, "algorithmic_bytes": b}


def measure_workload(name, storage, Xd=None, steps=200, warmup=5):
    """iterations/s (CUDA events around `steps` graph-replayed iterations) and
    the dominant pass's roofline on one workload, inputs resident on the GPU."""
    import torch
    import paper_2302_05119_gb300 as P
    import synth
    w = _workload(name)
    if Xd is None:
        Xs, _ = synth.make_tensors(w, dtype=np.float32)
        Xd = [torch.from_numpy(X).cuda() for X in Xs]
        del Xs
    m = P.CoupledNCP(Xd, w.R, w.L, profile=True, storage=storage)
    m.set_factors(synth.init_factors(w.dims, w.R, w.seed))
    m.step(warmup)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    s = m.step(steps)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    m.close()
    return {"workload": w.name, "storage": storage, "K": w.K, "R": w.R, "L": w.L,
            "value": steps / (ms / 1e3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
            "roofline": _pass_roofline(w, storage, s), "lead_plan": s["lead_plan"],
            "trail_ranges": s["trail_ranges"]}


def time_to_fit(name, arms, check_every=10, cap=2000, lra_check_every=100, Xd=None):
    """Wall time from cncpd_create on device-resident FP32 tensors to the
    first check at which the global Fit of the arm's factors, evaluated on
    the original FP32 tensors, is within 1e-4 of the target: the FP64
    oracle's converged Fit (Section III-C termination, eps = 1e-8) when it is
    cached for this workload and seed, else the library's own FP64 path run
    to convergence (labelled as such).  ``arms`` lists (storage, lra) pairs.
    Every arm pays the same check: its factors are copied (on the device)
    into an FP32-storage handle of the original tensors, whose global Fit
    decides."""
    import torch
    import paper_2302_05119_gb300 as P
    import synth
    w = _workload(name)
    U0 = synth.init_factors(w.dims, w.R, w.seed)
    if Xd is None:
        Xs, _ = synth.make_tensors(w, dtype=np.float32)
        Xd = [torch.from_numpy(X).cuda() for X in Xs]
        del Xs
    rec = _fit_target(w)
    if rec is not None:
        target = {"fit": rec["fit"], "source": "FP64 oracle (tests/golden/fit_targets.json)",
                  "oracle_iterations": rec["iterations"]}
    else:
        t0 = time.perf_counter()
        ref = P.CoupledNCP([X.double() for X in Xd], w.R, w.L, eps=1e-8, max_it=1000)
        ref.set_factors(U0)
        sf = ref.fit()
        target = {"fit": ref.global_fit(), "source": "library FP64 path to convergence (no oracle target cached)",
                  "iterations": sf["total_iters"], "seconds": time.perf_counter() - t0}
        ref.close()
    bar = target["fit"] - 1e-4
    ref32 = P.CoupledNCP(Xd, w.R, w.L, storage="f32")
    Ub = [[torch.empty((w.dims[k][n], w.ranks()[k]), dtype=torch.float32, device="cuda") for n in range(w.N)]
          for k in range(w.K)]

    def fit_on_data(m):
        for k in range(w.K):
            for n in range(w.N):
                m.factor(k, n, out=Ub[k][n])
        ref32.set_factors(Ub)
        return ref32.global_fit()

    out = {"workload": w.name, "metric": "seconds to a global Fit within 1e-4 of the target, on the FP32 data",
           "unit": "s", "target": target, "arms": {}}
    for storage, lra in arms:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m = P.CoupledNCP(Xd, w.R, w.L, storage=storage)
        m.set_factors(U0)
        lra_s = None
        if lra:
            m.lra(w.R_lra, synth.init_lra_factors(w.dims, w.R_lra, w.seed))
            lra_s = time.perf_counter() - t0
        every = lra_check_every if lra else check_every
        it, f = 0, 0.0
        while it < cap:
            m.step(every)
            it += every
            f = fit_on_data(m)
            if f >= bar:
                break
        dt = time.perf_counter() - t0
        f_stored = m.global_fit()
        m.close()
        key = storage + ("+lra" if lra else "")
        out["arms"][key] = {"seconds": dt, "iterations": it, "fit_fp32_data": f, "fit_stored": f_stored,
                            "reached": bool(f >= bar), "lra_seconds": lra_s, "check_every": every}
    ref32.close()
    torch.cuda.empty_cache()
    base = out["arms"].get("f32")
    if base and base["reached"]:
        for key, a in out["arms"].items():
            if key != "f32":
                a["speedup_vs_f32"] = base["seconds"] / a["seconds"] if a["reached"] else None
    return out


def _oracle_rate(w, Xs, U0, n_iters, blocks):
    """Oracle iterations/s on a bounded sample: ``n_iters`` APG iterations of
    the oracle restricted to ``blocks`` (its cost is linear in the blocks),
    scaled to whole-workload iterations."""
    from oracle import cncpd_oracle as O
    sub = [Xs[k].astype(np.float64) for k in blocks]
    prob = O.Problem(sub, [w.R] * len(blocks), w.L)
    t0 = time.perf_counter()
    O.apg(prob, [U0[k] for k in blocks], max_it=n_iters, eps=0.0)
    dt = time.perf_counter() - t0
    return n_iters * len(blocks) / w.K / dt, dt


def _threads():
    try:
        from threadpoolctl import threadpool_info
        n = [i.get("num_threads") for i in threadpool_info() if i.get("internal_api") in ("openblas", "mkl", "blis")]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count()


def run_reference(args):
    ws, rank = _dist()
    if rank != 0:
        return
    w = _workload(args.workload)
    import synth
    blocks = [0]
    Xs, _ = synth.make_tensors(w, dtype=np.float32, blocks=blocks)
    Xfull = {0: Xs[0]}
    U0 = synth.init_factors(w.dims, w.R, w.seed)
    from oracle import cncpd_oracle as O
    prob = O.Problem([Xfull[0].astype(np.float64)], [w.R], w.L)
    # a step = one oracle APG iteration on one block (1/K of the workload)
    res_w = O.apg(prob, [U0[0]], max_it=max(1, min(args.warmup, 1)), eps=0.0)
    t0 = time.perf_counter()
    O.apg(prob, [U0[0]], max_it=args.steps, eps=0.0)
    dt = time.perf_counter() - t0
    value = args.steps / w.K / dt
    line = {
        "impl": "reference", "metric": _metric(w, "f32"), "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded Uniform[0,1] factors, 10 dB Gaussian noise, clipped)",
        "config": {"workload": w.name, "K": w.K, "dims": list(w.dims[0]), "R": w.R, "L": w.L},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": _threads(), "kind": "oracle",
                         "sample": f"FP64 numpy oracle, {args.steps} APG iterations on 1 of {w.K} "
                                   f"blocks (each step = 1/{w.K} of a workload iteration)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    ws, rank = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import paper_2302_05119_gb300 as P
    import synth

    w = _workload(args.workload)
    Xs, _ = synth.make_tensors(w, dtype=np.float32)
    U0 = synth.init_factors(w.dims, w.R, w.seed)
    # streamed X reads the tensors from page-locked host memory block by block
    # (device copies would defeat the point)
    Xd = ([torch.from_numpy(X).pin_memory() for X in Xs] if args.stream_x
          else [torch.from_numpy(X).cuda() for X in Xs])
    torch.cuda.synchronize()

    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    m = P.CoupledNCP(Xd, w.R, w.L, profile=True, storage=args.storage, tf32=args.tf32,
                     autotune=not args.no_autotune, stream_x=args.stream_x)
    handle_bytes = free0 - torch.cuda.mem_get_info()[0]
    m.set_factors(U0)
    lra = None
    if args.lra:
        Rt = w.R_lra or w.R
        t0 = time.perf_counter()
        sl = m.lra(Rt, synth.init_lra_factors(w.dims, Rt, w.seed))
        lra = {"R_tilde": Rt, "seconds": time.perf_counter() - t0, "als_sweeps": sl["lra_sweeps"],
               "als_relerr": sl["lra_relerr"], "stream_x": args.stream_x,
               "handle_device_bytes": handle_bytes}
    m.step(args.warmup)
    t0 = time.perf_counter()
    m.step(10)
    t_iter = (time.perf_counter() - t0) / 10

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # clocks are sampled over an untimed load phase (--clock-load-s, 0.4 s by
    # default) just before the timed region and over the timed region itself (a timed
    # region of a few milliseconds is shorter than one nvidia-smi sample)
    clocks = ClockSampler(local)
    clocks.start()
    if args.clock_load_s > 0:
        m.step(max(1, min(20000, int(args.clock_load_s / max(t_iter, 1e-5)))))
    barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    s = m.step(args.steps)
    e1.record()
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    ms = _max_over_ranks(ms, ws, "cuda")
    value = _job_value(args.steps, ws, ms)

    # roofline of the dominant tensor-streaming kernel
    es = {"f32": 4, "bf16": 2, "bf16x2": 4}[args.storage]  # bytes of X per element
    h = (w.N + 1) // 2
    # algorithmic bytes of one launch: X read once, the factors of the modes
    # contracted away read once, the level-1 product written once
    lead_rows = [int(np.prod(d[:h])) for d in w.dims]
    trail_cols = [int(np.prod(d[h:])) for d in w.dims]
    x_bytes = sum(w.elements()) * es
    trail_alg = x_bytes + sum((lr + sum(d[h:])) * w.R * 4 for lr, d in zip(lead_rows, w.dims))
    lead_alg = x_bytes + sum((tc + sum(d[:h])) * w.R * 4 for tc, d in zip(trail_cols, w.dims))
    nl = max(1, s["stream_launches"] // 2)
    t_trail = s["trail_ms"] / nl
    t_lead = s["lead_ms"] / nl
    kern, tk = ("lead_contract", t_lead) if t_lead >= t_trail else ("trailing_contract", t_trail)
    peak, peak_kind = _peaks()
    pass_bytes = lead_alg if kern == "lead_contract" else trail_alg
    if s["stream_launches"] > 0:
        achieved = pass_bytes / (tk / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": kern, "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": _traffic("trailing_tf32" if (kern == "trailing_contract" and s["trail_tensor_cores"]
                                                        and args.storage == "f32") else kern, w.name, args.storage),
                "other_kernel_ms": t_trail if kern == "lead_contract" else t_lead,
                "algorithmic_bytes_per_launch": pass_bytes,
                "timed_launches": nl,
                "timing": "CUDA events on the launching stream around each pass of the first iteration of the timed region and every 8th one after it"}
    else:  # after the LRA step no iteration reads X
        roof = {"bound": "latency", "kernel": None, "achieved": None, "peak": peak, "unit": "GB/s", "frac": None,
                "peak_source": peak_kind, "traffic": None,
                "note": "collapsed products: the iterations read only the low-rank factors (launch/latency bound)"}
    m.close()
    del Xd

    # end to end through the public API with host buffers (pinned)
    Xh = [torch.from_numpy(X).pin_memory() for X in Xs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    m2 = P.CoupledNCP(Xh, w.R, w.L, storage=args.storage, tf32=args.tf32, autotune=not args.no_autotune,
                      stream_x=args.stream_x)
    m2.set_factors(U0)
    if args.lra:
        m2.lra(lra["R_tilde"], synth.init_lra_factors(w.dims, lra["R_tilde"], w.seed))
    s2 = m2.step(args.steps)
    out = m2.factors(np.float32)
    t_e2e = time.perf_counter() - t0
    m2.close()
    h2d = (sum(X.nbytes for X in Xs) + sum(A.nbytes for Uk in U0 for A in Uk)) / args.steps
    d2h = sum(A.nbytes for Uk in out for A in Uk) / args.steps
    t_e2e = _max_over_ranks(t_e2e * 1e3, ws, "cuda") / 1e3
    e2e = {"value": _job_value(args.steps, ws, t_e2e * 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "scope": "cncpd_create from pinned host tensors + set_factors + steps + factor copy-out, per job"}

    ttf = None
    ttf_lra = None
    others = None
    if rank == 0 and ws == 1 and not args.no_time_to_fit:
        # the metric's second part: mixed precision against plain FP32 on the
        # precision workload (512 x 512 x 256 x 4, R = 20), evaluated on the FP32
        # data; then the same data in BF16 and BF16 hi+lo storage, and the
        # uneven fourth-order EEG-shaped blocks, for iterations/s and roofline
        wp = _workload("bf16_512x512x256")
        Xp, _ = synth.make_tensors(wp, dtype=np.float32)
        Xpd = [torch.from_numpy(X).cuda() for X in Xp]
        del Xp
        ttf = time_to_fit(wp.name, [("f32", False), ("bf16", False), ("bf16x2", False)], Xd=Xpd)
        others = [measure_workload(wp.name, st, Xd=Xpd) for st in ("bf16", "bf16x2")]
        del Xpd
        torch.cuda.empty_cache()
        others.append(measure_workload("eeg_uneven_4th", "f32"))
        torch.cuda.empty_cache()
        # lraCoNCPD-APG against the plain method on the face shape (scaled so
        # that the FP64 oracle's converged fit could be computed for it)
        ttf_lra = time_to_fit("face_lra_400x400x160", [("f32", False), ("bf16", False), ("bf16", True)])
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, dt = _oracle_rate(w, Xs, U0, 2, list(range(w.K)))
        cpu = {"value": rate, "unit": UNIT, "cores": _threads(), "kind": "oracle",
               "sample": f"FP64 numpy oracle, 2 APG iterations of the full workload ({dt:.1f} s)"}

    if rank == 0:
        line = {
            "metric": _metric(w, args.storage), "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded Uniform[0,1] factors, 10 dB Gaussian noise, clipped)",
            "config": {"workload": w.name, "K": w.K, "dims": list(w.dims[0]), "R": w.R, "L": w.L,
                       "storage": args.storage, **({"tf32_trailing": True} if args.tf32 else {}),
                       "l2": f"inputs larger than L2 ({x_bytes / 1e6:.0f} MB of stored tensors)",
                       "parallelism": "replicas" if ws > 1 else "single GPU"},
            "reupdates": s["reupdates"], "fit": s["fit"], "lra": lra,
            "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": s["launches"], "clocks": clk, "time_to_fit": ttf, "time_to_fit_lra": ttf_lra,
            "workloads": others,
            "lead_plan": {"units_per_sm": s["lead_plan"], "measured": bool(s["lead_plan_tuned"])},
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


def run_time_to_fit(args):
    """--time-to-fit: the time-to-fit record alone for --workload: FP32,
    BF16 and BF16 hi+lo storage, plus BF16 storage with the LRA step when the
    workload has an LRA rank."""
    import torch
    torch.cuda.set_device(0)
    w = _workload(args.workload)
    arms = [("f32", False), ("bf16", False), ("bf16x2", False)]
    if w.R_lra:
        arms.append(("bf16", True))
    print(json.dumps(time_to_fit(w.name, arms)), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="sim_256cube")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "bf16x2"],
                    help="element type of X on the device (factors and accumulation stay FP32)")
    ap.add_argument("--lra", action="store_true", help="run the LRA step (lraCoNCPD-APG) before the timed steps")
    ap.add_argument("--time-to-fit", action="store_true",
                    help="time to reach the converged FP64 fit within 1e-4, FP32 vs mixed precision")
    ap.add_argument("--clock-load-s", type=float, default=0.4,
                    help="seconds of untimed iterations run just before the timed region while the "
                         "clocks are sampled (0 under a profiler)")
    ap.add_argument("--no-time-to-fit", action="store_true",
                    help="leave the time-to-fit record out of the default line")
    ap.add_argument("--no-autotune", action="store_true",
                    help="lead-pass plan from the cost model instead of the measuring tuner (for profiler "
                         "runs, whose serialised launches would bias the tuner's choice)")
    ap.add_argument("--stream-x", action="store_true",
                    help="with --lra: keep one block of X on the device at a time (cncpd_opts.stream_x)")
    ap.add_argument("--tf32", action="store_true",
                    help="FP32 third-order data: trailing pass on the TF32 tensor cores (opt-in, slower)")
    args = ap.parse_args()
    if args.stream_x and not args.lra:
        ap.error("--stream-x needs --lra: only the lraCoNCPD-APG iterations run without X on the device")
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.time_to_fit:
        run_time_to_fit(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
