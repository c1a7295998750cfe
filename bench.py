"""Throughput of per-point rank-one convexification on GB300.

Workload (one GPU): a 128 x 128 Q1 mesh x 4 Gauss points = 65,536 quadrature
points, F from a seeded synthetic displacement (affine stretch 1.3 + 8 Fourier
modes + a 45 degree shear band), history from the previous load step; NH with
exponential damage (mu=1, lambda=5, D_inf=0.99, D_0=0.5); 64 x 64 angle grid
(4096 rank-one directions), 1025 samples per line on t in [-0.5, 0.5],
lamination depth 3.  A step is the whole path: history update (Eq. 2.5) and
the convexification with W^R and P (Secs. 4-5).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank convexifies
its own mesh (weak scaling, no collective in the data path).
"""
from __future__ import annotations

import argparse
import hashlib
import glob
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "quadrature points convexified/s (W^R+P) at 1e-6 rel. error, surrogate vs full-scan"
MAT = dict(mu=1.0, lambda_L=5.0, D_inf=0.99, D0=0.5)
NX, STRETCH, ANGLES, LINE, DEPTH, T_HALF = 128, 1.3, 64, 1025, 3, 0.5
FLOP_PER_SAMPLE = 30  # algorithmic FP32 work per valid line sample (energy 22 + hull 8)
FP32_LANES_PER_SM = 128


def workload_desc(n):
    return (f"mesh {NX}x{NX} Q1 x 4 Gauss points = {n} points, stretch {STRETCH}, "
            f"{ANGLES}x{ANGLES} angles, L={LINE}, t in [-{T_HALF},{T_HALF}], depth {DEPTH}, full scan")


def args_parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=NX, help="mesh size (default 128 -> 65,536 points)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-points", type=int, default=0, help="oracle sample size (0 = auto)")
    ap.add_argument("--form", default="full-scan", choices=["full-scan", "surrogate", "train"],
                    help="surrogate: the learned-proposal form over a load path; train: "
                         "training and inference of the proposal network (own lines)")
    ap.add_argument("--train-epochs", type=int, default=10)
    ap.add_argument("--gap-tol", type=float, default=1e-6, help="surrogate fallback tolerance")
    ap.add_argument("--window", type=int, default=4, help="surrogate window half-width (cells)")
    ap.add_argument("--gap-one-sided", action="store_true",
                    help="surrogate: fall back only when the proposed laminate beats the window")
    ap.add_argument("--load-steps", type=int, default=20)
    ap.add_argument("--check-points", type=int, default=4096,
                    help="surrogate: subsample checked against the full scan")
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, dist=None, device=None):
    """Max of a per-rank float over all ranks (x itself without a process group)."""
    if dist is None:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(n_per_rank, ws, steps, t_max_ms):
    """Points all ranks convexified / the slowest rank's time (weak scaling)."""
    return ws * n_per_rank * steps / (t_max_ms / 1e3)


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def make_inputs(nx, rank):
    from paper_2211_14318_gb300 import inputs

    F, F_prev = inputs.mesh_points(nx, stretch=STRETCH, seed=rank)
    return F, F_prev


# --------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        # raw samples: CVX_CLOCKS_DIR if set, else the system's temporary directory
        d = os.environ.get("CVX_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"clocks_{os.getpid()}.csv")

    def start(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-i", str(self.dev), "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in open(self.path):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                power.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm),
                "power_w_max": max(power) if power else None,
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------- roofline
def fp32_peak_tflops(torch, dev):
    props = torch.cuda.get_device_properties(dev)
    mhz = 2070.0
    src = "sm_max_mhz 2070 (nominal)"
    try:
        mp = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        if mp.get("sm_max_mhz"):
            mhz = float(mp["sm_max_mhz"])
            src = "MEASURED_PEAKS.json sm_max_mhz"
    except (OSError, ValueError):
        pass
    sms = props.multi_processor_count
    return sms * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12, sms, mhz, src


SCAN_SOURCES = ("cvx_pipeline.cu", "cvx_bridge.cuh", "cvx_device.cuh", "cvx_line.cuh",
                "cvx_internal.h")


def scan_source_hash():
    """Hash of the sources the line-scan kernel is compiled from."""
    h = hashlib.sha256()
    c = os.path.join(ROOT, "paper_2211_14318_gb300", "csrc")
    for f in SCAN_SOURCES:
        h.update(open(os.path.join(c, f), "rb").read())
    h.update(open(os.path.join(ROOT, "include", "convexify.h"), "rb").read())
    return h.hexdigest()[:16]


def traffic_per_launch(valid_per_launch):
    """DRAM bytes per scan launch from the committed ncu summary, scaled to
    this launch's work; None if the kernel changed since the capture."""
    path = os.path.join(ROOT, "profiles", "k_scan_traffic.json")
    try:
        t = json.load(open(path))
    except (OSError, ValueError):
        return None
    if t.get("source_sha") != scan_source_hash():
        return None
    per_sample = t["dram_bytes"] / max(1, t["valid_samples"])
    return per_sample * valid_per_launch


# ----------------------------------------------------------------- oracle arm
def oracle_rate(F, F_prev, npts, cores):
    """The CPU oracle (as it stands) on npts points of the same workload."""
    import oracle

    mat = oracle.Material(MAT["mu"], MAT["lambda_L"], MAT["D_inf"], MAT["D0"])
    sc = oracle.Scan(oracle.angle_directions(ANGLES, ANGLES), LINE, T_HALF, DEPTH)
    idx = [int(i) for i in __import__("numpy").linspace(0, F.shape[0] - 1, npts)]
    Fs, Fps = F[idx], F_prev[idx]
    t0 = time.perf_counter()
    beta = oracle.history_update(mat, Fps)
    oracle.convexify(mat, sc, Fs, beta, nthreads=cores)
    dt = time.perf_counter() - t0
    return npts / dt, dt


def run_reference(a):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import oracle

    oracle.build()
    cores = host_cores()
    F, F_prev = make_inputs(a.nx, 0)
    npts = a.cpu_points or max(cores, 2 * cores)
    for _ in range(a.warmup):
        oracle_rate(F, F_prev, max(1, cores // 4), cores)
    rates, times = [], []
    for _ in range(a.steps):
        r, dt = oracle_rate(F, F_prev, npts, cores)
        rates.append(r)
        times.append(dt)
    value = npts * a.steps / sum(times)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "points/s",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * sum(times) / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(F.shape[0]), "form": "full-scan"},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle",
                         "sample": f"{npts} evenly spaced points of the workload per step"},
        "e2e": {"value": value, "unit": "points/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- our arm
def run_ours(a):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")

    import __graft_entry__

    __graft_entry__.build()
    from paper_2211_14318_gb300 import api

    F, F_prev = make_inputs(a.nx, rank)
    n = F.shape[0]
    p = api.Params(n_theta_a=ANGLES, n_theta_b=ANGLES, line_points=LINE, t_half=T_HALF,
                   depth=DEPTH, **MAT)
    cv = api.Convexifier(local)
    Fd = torch.from_numpy(F).to(dev)
    Fpd = torch.from_numpy(F_prev).to(dev)
    out = dict(W_R=torch.empty(n, dtype=torch.float64, device=dev),
               P=torch.empty(n, 4, dtype=torch.float64, device=dev),
               status=torch.empty(n, dtype=torch.int32, device=dev))
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2

    def step(Fx, Fpx):
        beta = cv.history_update(p, Fpx)
        return cv.convexify_points(p, Fx, beta, out=out)

    for _ in range(a.warmup):
        step(Fd, Fpd)
    torch.cuda.synchronize()

    # ---- device-resident timed region
    cv.stats(reset=True)
    cv.set_profiling(True)
    cv.scan_timing(reset=True)
    uuid = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    clocks = ClockSampler(f"GPU-{uuid}" if uuid is not None else str(local))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(a.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    wall0 = time.perf_counter()
    for k in range(a.steps):
        flush.zero_()
        ev[k][0].record()
        step(Fd, Fpd)
        ev[k][1].record()
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    ck = clocks.stop()
    if ws > 1:
        dist.barrier()
    dev_ms = sum(e0.elapsed_time(e1) for e0, e1 in ev)
    scan_ms, scan_launches = cv.scan_timing(reset=True)
    cv.set_profiling(False)
    st = cv.stats(reset=True)
    t_max = max_over_ranks(dev_ms, dist if ws > 1 else None, dev)
    value = whole_job_rate(n, ws, a.steps, t_max)

    # ---- end to end through the public API from pinned host buffers
    Fh = torch.from_numpy(F).pin_memory()
    Fph = torch.from_numpy(F_prev).pin_memory()
    Wh = torch.empty(n, dtype=torch.float64).pin_memory()
    Ph = torch.empty(n, 4, dtype=torch.float64).pin_memory()
    e2e_ev = []
    for k in range(a.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        Fx = Fh.to(dev, non_blocking=True)
        Fpx = Fph.to(dev, non_blocking=True)
        o = step(Fx, Fpx)
        Wh.copy_(o["W_R"], non_blocking=True)
        Ph.copy_(o["P"], non_blocking=True)
        e1.record()
        e2e_ev.append((e0, e1))
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(sum(e0.elapsed_time(e1) for e0, e1 in e2e_ev),
                            dist if ws > 1 else None, dev)
    e2e_value = whole_job_rate(n, ws, a.steps, e2e_ms)

    peak, sms, mhz, peak_src = fp32_peak_tflops(torch, dev)
    flop = FLOP_PER_SAMPLE * st["valid_samples"]
    achieved = flop / (scan_ms / 1e3) / 1e12 if scan_ms > 0 else None
    valid_per_launch = st["valid_samples"] / max(1, scan_launches)
    traffic = traffic_per_launch(valid_per_launch)

    if rank == 0:
        cpu = None
        if ws == 1 and not a.no_cpu_baseline:
            import oracle

            oracle.build()
            cores = host_cores()
            npts = a.cpu_points or 2 * cores
            rate, dt = oracle_rate(F, F_prev, npts, cores)
            cpu = {"value": rate, "unit": "points/s", "cores": cores, "kind": "oracle",
                   "sample": f"{npts} evenly spaced points of the workload ({dt:.1f} s of CPU time)"}
        line = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws,
            "steps": a.steps, "warmup": a.warmup, "ms_per_step": t_max / a.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32/f64", "data": "synthetic",
            "config": {"workload": workload_desc(n), "form": "full-scan",
                       "points_per_gpu": n, "angles": [ANGLES, ANGLES], "line_points": LINE,
                       "depth": DEPTH, "l2": "flushed between steps (512 MiB write)",
                       "wall_s_timed_region": wall},
            "roofline": {"bound": "alu", "kernel": "k_scan", "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s",
                         "frac": (achieved / peak) if achieved else None,
                         "traffic": traffic,
                         "peak_source": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {mhz:.0f} MHz ({peak_src})",
                         "flop_per_valid_sample": FLOP_PER_SAMPLE,
                         "kernel_share_of_step": scan_ms / dev_ms if dev_ms else None,
                         "launches": scan_launches},
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "points/s",
                    "h2d_bytes_per_step": 2 * n * 4 * 8, "d2h_bytes_per_step": n * 8 + n * 4 * 8},
            "gpu_launches": a.steps * (3 + 4 * DEPTH),  # history, init, 4 per level, leaf
            "clocks": ck,
            "stats": st,
        }
        print(json.dumps(line), flush=True)
    cv.close()
    if ws > 1:
        dist.destroy_process_group()


# ------------------------------------------------------- surrogate form
S_ANGLES, S_LINE, S_DEPTH = 128, 2049, 3


def run_surrogate(a):
    """The learned-proposal form over a load path (stretch 1.0 -> 1.8, history
    updated every step): 128 x 128 angles, window +-w cells, L = 2049, depth 3,
    fallback per gap_tol.  The network is first trained on labels from the
    GPU's own full scans (material points with lambda in [1, 2] and points of
    the load path; labels on the 128^2 grid, L = 513, depth 2).  Reported: the
    proposed form's points/s over the whole path, its fallback rate, its W^R
    error against the full scan on a subsample at three steps, and the plain
    full scan's points/s on the same mesh and on coarser angle grids with their
    own errors (the plain form's curve of points/s against error)."""
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2211_14318_gb300 import api, inputs

    dev = torch.device("cuda:0")
    torch.cuda.set_device(0)
    cv = api.Convexifier(0)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    def timed(f):
        e0, e1 = ev(), ev()
        e0.record()
        r = f()
        e1.record()
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1) / 1e3

    # ---- training data and training
    pl = api.Params(n_theta_a=S_ANGLES, n_theta_b=S_ANGLES, line_points=513, depth=2, **MAT)
    path = inputs.load_path(a.nx, n_steps=a.load_steps, stretch_end=1.8, seed=7)
    F1, Fp1 = inputs.surrogate_inputs(131072, seed=100)
    b1 = cv.history_update(pl, Fp1)
    Xs, Ys, t_label = [], [], 0.0
    out, dt = timed(lambda: cv.convexify_points(pl, F1, b1, want_tree=True))
    t_label += dt
    X, Y = cv.surrogate_labels(pl, b1, out["tree"], F1.shape[0])
    Xs.append(X)
    Ys.append(Y)
    for k in (3, 7, 11, 15, 19):
        k = min(k, a.load_steps - 1)
        Fk = path[k]
        bk = cv.history_update(pl, path[k - 1]).cpu().numpy()
        idx = np.random.default_rng(k).choice(Fk.shape[0], min(16384, Fk.shape[0]), replace=False)
        out, dt = timed(lambda: cv.convexify_points(pl, Fk[idx], bk[idx], want_tree=True))
        t_label += dt
        X, Y = cv.surrogate_labels(pl, bk[idx], out["tree"], len(idx))
        Xs.append(X)
        Ys.append(Y)
    X, Y = torch.cat(Xs), torch.cat(Ys)
    t0 = time.perf_counter()
    log = cv.surrogate_train(X, Y, epochs=30, batch=8192, lr=1e-3, init=True, seed=0)
    t_train = time.perf_counter() - t0

    # ---- load path
    p = api.Params(n_theta_a=S_ANGLES, n_theta_b=S_ANGLES, line_points=S_LINE, depth=S_DEPTH,
                   gap_one_sided=a.gap_one_sided, **MAT)
    n = path[0].shape[0]
    sub = np.linspace(0, n - 1, min(a.check_points, n)).astype(int)
    sub_t = torch.from_numpy(sub).to(dev)
    beta = torch.zeros(n, dtype=torch.float64, device=dev)
    out = dict(W_R=torch.empty(n, dtype=torch.float64, device=dev),
               P=torch.empty(n, 4, dtype=torch.float64, device=dev),
               status=torch.empty(n, dtype=torch.int32, device=dev),
               fell_back=torch.empty(n, dtype=torch.uint8, device=dev))
    checks = {max(1, a.load_steps // 4), max(1, a.load_steps // 2), a.load_steps}
    t_sur, fell, rows = 0.0, 0.0, []
    cv.stats(reset=True)
    uuid = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    clocks = ClockSampler(f"GPU-{uuid}" if uuid is not None else "0")
    clocks.start()
    for k in range(1, a.load_steps + 1):
        Fk = torch.from_numpy(path[k - 1]).to(dev)

        def step():
            return cv.surrogate_propose(p, Fk, beta, window=a.window, gap_tol=a.gap_tol, out=out)

        r, dt = timed(step)
        t_sur += dt
        fell += float(r["fell_back"].float().mean())
        if k in checks:
            # reference: the plain full scan on the same 128^2 grid (itself
            # parity-tested against the FP64 oracle), on the subsample
            Fs, bs = Fk[sub_t], beta[sub_t]
            ref = cv.convexify_points(p, Fs, bs)
            W = r["W_R"].cpu().numpy()[sub]
            refW = ref["W_R"].cpu().numpy()
            e = np.abs(W - refW) / (1e-8 + np.abs(refW))
            # throughput of the plain form on (up to) 65,536 points of the mesh
            nt = min(n, 65536)
            _, dt_ref = timed(lambda: cv.convexify_points(p, Fk[:nt], beta[:nt]))
            row = {"step": k, "surrogate_pts_per_s": n / dt, "full_scan_pts_per_s": nt / dt_ref,
                   "err_p50": float(np.quantile(e, 0.5)), "err_p99": float(np.quantile(e, 0.99)),
                   "err_max": float(e.max()), "fell_back": float(r["fell_back"].float().mean())}
            for na in (16, 32, 64):
                q = api.Params(n_theta_a=na, n_theta_b=na, line_points=S_LINE, depth=S_DEPTH, **MAT)
                rq = cv.convexify_points(q, Fs, bs)
                _, dtq = timed(lambda: cv.convexify_points(q, Fk[:nt], beta[:nt]))
                eq = np.abs(rq["W_R"].cpu().numpy() - refW) / (1e-8 + np.abs(refW))
                row[f"plain_{na}x{na}"] = {"pts_per_s": nt / dtq, "err_p50": float(np.quantile(eq, 0.5)),
                                           "err_p99": float(np.quantile(eq, 0.99))}
            rows.append(row)
        beta = cv.history_update(p, Fk, beta)
    ck = clocks.stop()
    st = cv.stats(reset=True)
    line = {
        "metric": METRIC, "value": n * a.load_steps / t_sur, "unit": "points/s", "n_gpus": 1,
        "steps": a.load_steps, "warmup": 0, "ms_per_step": 1e3 * t_sur / a.load_steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16/f32/f64",
        "data": "synthetic",
        "config": {"workload": f"load path, mesh {a.nx}x{a.nx} Q1 x 4 Gauss points = {n} points, "
                               f"stretch 1.0 -> 1.8 in {a.load_steps} steps, {S_ANGLES}x{S_ANGLES} "
                               f"angles, window +-{a.window}, L={S_LINE}, depth {S_DEPTH}",
                   "form": "surrogate", "gap_tol": a.gap_tol, "window": a.window,
                   "gap_test": "one-sided" if a.gap_one_sided else "two-sided",
                   "timed": "surrogate_propose per step (CUDA events); history update excluded"},
        "surrogate": {"fell_back_points_mean": fell / a.load_steps,
                      "window_nodes": st["window_nodes"], "fallback_nodes": st["fallbacks"],
                      "train": {"samples": int(X.shape[0]), "label_s": t_label, "train_s": t_train,
                                "loss_first": float(log[0]), "loss_last": float(log[-1])},
                      "checks": rows},
        "clocks": ck,
    }
    print(json.dumps(line), flush=True)
    cv.close()


def run_train(a):
    """The proposal network's training and inference on the tensor cores:
    labels from the full scan of material points (16 x 16 angles, L = 201,
    t in [-0.5, 0.5], depth 2, lambda in [1, 2]), 2 M training samples, Adam
    with batch 8,192; then inference on 1 M held-out points.  Throughput in
    samples/s and algorithmic TFLOP/s of the GEMMs (forward 2 x 200,192 FLOP
    per sample, training 3 x that less the unused input gradient) against the
    measured BF16 peak; held-out quality: the proposed cell of the 16 x 16
    grid against the full scan's direction on laminated points."""
    import math

    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2211_14318_gb300 import api, inputs

    dev = torch.device("cuda:0")
    torch.cuda.set_device(0)
    cv = api.Convexifier(0)

    def timed(f):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        r = f()
        e1.record()
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1) / 1e3

    p = api.Params(n_theta_a=16, n_theta_b=16, line_points=201, depth=2, **MAT)
    F, Fp = inputs.surrogate_inputs(1_000_000, seed=200)
    beta = cv.history_update(p, Fp)
    Fd = torch.from_numpy(F).to(dev)
    out, t_label = timed(lambda: cv.convexify_points(p, Fd, beta, want_tree=True))
    X, Y = cv.surrogate_labels(p, beta, out["tree"], F.shape[0])
    n_train = min(2_000_000, X.shape[0])
    X, Y = X[:n_train].contiguous(), Y[:n_train].contiguous()
    log, t_train = timed(lambda: cv.surrogate_train(X, Y, epochs=a.train_epochs, batch=8192,
                                                    lr=1e-3, init=True, seed=0))
    fwd_flop = 2.0 * (256 * 6 + 3 * 256 * 256 + 7 * 256)
    train_flop = 3.0 * fwd_flop - 2.0 * 256 * 6
    steps = a.train_epochs * (n_train // 8192)
    train_rate = steps * 8192 / t_train

    Fh, Fph = inputs.surrogate_inputs(1_000_000, seed=201)
    bh = cv.history_update(p, Fph)
    Fhd = torch.from_numpy(Fh).to(dev)
    J = Fhd[:, 0] * Fhd[:, 3] - Fhd[:, 1] * Fhd[:, 2]
    Xh = torch.cat([Fhd, bh[:, None], torch.log(J)[:, None]], dim=1).float().contiguous()
    cv.surrogate_forward(Xh[:8192])  # warm
    o, t_inf = timed(lambda: cv.surrogate_forward(Xh))
    inf_rate = Xh.shape[0] / t_inf
    # held-out quality: root decisions of the full scan (depth 1)
    p1 = api.Params(n_theta_a=16, n_theta_b=16, line_points=201, depth=1, **MAT)
    r1 = cv.convexify_points(p1, Fhd, bh, want_root=True)
    root = api.root_numpy(r1["root"], Fh.shape[0])
    lam = root["laminated"] == 1
    oh = o.cpu().numpy()
    ia = np.mod(np.floor(np.mod(oh[:, 0], math.pi) * 16 / math.pi + 0.5), 16).astype(int)
    ib = np.mod(np.floor(np.mod(oh[:, 1], math.pi) * 16 / math.pi + 0.5), 16).astype(int)
    la, lb = root["dir"] // 16, root["dir"] % 16

    def cdist(x, y):
        d = np.abs(x - y) % 16
        return np.minimum(d, 16 - d)

    da, db = cdist(ia, la)[lam], cdist(ib, lb)[lam]
    peak = None
    try:
        peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops"]
    except (OSError, ValueError, KeyError):
        pass
    ach_inf = fwd_flop * inf_rate / 1e12
    line = {
        "metric": "proposal-network samples/s (training, BF16 tensor cores)",
        "value": train_rate, "unit": "samples/s", "n_gpus": 1, "steps": steps, "warmup": 0,
        "ms_per_step": 1e3 * t_train / max(1, steps), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16/f32", "data": "synthetic",
        "config": {"workload": "network 6 -> 256 x 4 -> 7 GELU; labels from the full scan of 1 M "
                               "material points (16x16 angles, L=201, depth 2, lambda in [1,2])",
                   "form": "train", "train_samples": int(n_train), "batch": 8192,
                   "epochs": a.train_epochs, "held_out": int(Xh.shape[0])},
        "roofline": {"bound": "tensor", "kernel": "k_gemm (forward, inference)",
                     "achieved": ach_inf, "peak": peak, "unit": "TFLOP/s",
                     "frac": ach_inf / peak if peak else None,
                     "training_tflops": train_flop * train_rate / 1e12,
                     "peak_source": "MEASURED_PEAKS.json bf16_tflops (cuBLAS burst), of measured"},
        "inference": {"value": inf_rate, "unit": "points/s", "points": int(Xh.shape[0])},
        "labels": {"points": int(F.shape[0]), "samples": int(X.shape[0]), "seconds": t_label,
                   "points_per_s": F.shape[0] / t_label},
        "loss": {"first": float(log[0]), "last": float(log[-1])},
        "held_out_quality": {"laminated_points": int(lam.sum()),
                             "cell_exact": float(np.mean((da == 0) & (db == 0))),
                             "within_one_cell": float(np.mean((da <= 1) & (db <= 1)))},
    }
    print(json.dumps(line), flush=True)
    cv.close()


def main():
    a = args_parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.form == "surrogate":
        run_surrogate(a)
    elif a.form == "train":
        run_train(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
