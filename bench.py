"""Throughput of per-point rank-one convexification on GB300.

Default workload (the metric's): a load path on a 512 x 512 Q1 mesh x 4
Gauss points = 1,048,576 quadrature points, 20 load steps (stretch 1.0 ->
1.8, seeded smooth field and shear band), history updated after every step
(Eq. 2.5); NH with exponential damage (mu=1, lambda=5, D_inf=0.99, D_0=0.5);
128 x 128 angle grid (16,384 rank-one directions), 2049 samples per line on
t in [-0.5, 0.5], lamination depth 3.  A step is one load step of the
surrogate-proposed form: the network proposes a direction per tree node, a
+-4-cell angular window around it is scanned (re-centred on its border
minimum up to 4 times), nodes whose window minimum stays on its border fall
back to the full scan of all 16,384 directions; then W^R and P (Secs. 4-5).
Beside it, in the same JSON line: the plain full scan on the same steps, its
accuracy and the coarser plain grids (points/s against W^R error), the
accuracy of the proposed form against the FP64 oracle on 4,096 points at
steps 1, 10 and 20 (stored oracle results under tests/golden), the 1 M-point
full scan at 16 x 16 angles, L = 201, depth 2 with its own roofline, and the
65,536-point mesh at 64 x 64 angles, L = 1025, depth 3.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
                  [--form loadpath|full-scan|train]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank runs its own
load path (weak scaling, no collective in the data path).
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
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nx", type=int, default=NX, help="mesh size (default 128 -> 65,536 points)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-points", type=int, default=0, help="oracle sample size (0 = auto)")
    ap.add_argument("--form", default="loadpath",
                    choices=["loadpath", "full-scan", "points1m", "batch", "surrogate", "train",
                             "grid"],
                    help="loadpath: the metric's workload (default); full-scan: the 65,536-point "
                         "mesh alone; surrogate: the load path with the older report; train: "
                         "training and inference of the proposal network (own lines)")
    ap.add_argument("--train-epochs", type=int, default=10)
    ap.add_argument("--gap-tol", type=float, default=1e30,
                    help="surrogate energy-gap fallback tolerance (1e30: border test only)")
    ap.add_argument("--window", type=int, default=4, help="surrogate window half-width (cells)")
    ap.add_argument("--recentre", type=int, default=4, help="surrogate window re-centrings")
    ap.add_argument("--no-mirror", action="store_true",
                    help="surrogate form without the mirror window (twin basins of an isotropic W)")
    ap.add_argument("--lp-nx", type=int, default=512, help="load-path mesh size (512: 1,048,576 points)")
    ap.add_argument("--scaling", default="weak", choices=["weak", "strong"],
                    help="loadpath with N > 1: weak = one load path per rank; strong = one "
                         "load path split into contiguous point ranges weighted by expected "
                         "tree size")
    ap.add_argument("--mp-points", type=int, default=1 << 20,
                    help="points1m: material points (default 1,048,576)")
    ap.add_argument("--profile-step", type=int, default=0,
                    help="loadpath: bracket this timed load step with cudaProfilerStart/Stop "
                         "(for ncu --profile-from-start off)")
    ap.add_argument("--no-extras", action="store_true",
                    help="loadpath: skip the 1M-point L = 201 and the 65,536-point mesh lines")
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


def rank_ranges(weights, ws):
    """Contiguous point ranges [lo, hi) of one problem, one per rank, whose
    total weights (expected tree size per point) are as equal as contiguous
    cuts allow: rank r's range ends where the weight prefix sum first reaches
    (r + 1) / ws of the total."""
    import numpy as np

    w = np.asarray(weights, dtype=np.float64)
    c = np.cumsum(w)
    total = c[-1] if c.size else 0.0
    cuts = [0]
    for r in range(1, ws):
        cuts.append(int(np.searchsorted(c, total * r / ws, side="left")) + 1 if total > 0 else
                    (w.size * r) // ws)
    cuts.append(w.size)
    cuts = [min(max(x, 0), w.size) for x in cuts]
    for i in range(1, len(cuts)):
        cuts[i] = max(cuts[i], cuts[i - 1])
    return [(cuts[r], cuts[r + 1]) for r in range(ws)]


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


# the translation unit of k_scan_lanes (the kernel and its launch) and the
# headers it includes
SCAN_SOURCES = ("cvx_scan_lanes.cu", "cvx_line.cuh", "cvx_bridge.cuh", "cvx_device.cuh",
                "cvx_internal.h")


GRID_SOURCES = ("cvx_grid.cu", "cvx_device.cuh", "cvx_internal.h", "cvx_handle.h")


def _header_defs():
    """The parts of include/convexify.h a kernel compiles against: the header
    without its comments and function prototypes (types, enums, macros)."""
    import re

    txt = open(os.path.join(ROOT, "include", "convexify.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    txt = re.sub(r"^int\s+\w+\s*\([^;]*\);", "", txt, flags=re.S | re.M)
    return "\n".join(ln.rstrip() for ln in txt.splitlines() if ln.strip()).encode()


def scan_source_hash(sources=SCAN_SOURCES):
    """Hash of the sources a kernel is compiled from (the line scan's by
    default)."""
    h = hashlib.sha256()
    c = os.path.join(ROOT, "paper_2211_14318_gb300", "csrc")
    for f in sources:
        h.update(open(os.path.join(c, f), "rb").read())
    h.update(_header_defs())
    return h.hexdigest()[:16]


def traffic_per_launch(valid_per_launch, name="k_scan_traffic.json", sources=SCAN_SOURCES):
    """DRAM bytes per launch from the committed ncu summary, scaled to this
    launch's work; None if the kernel changed since the capture."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        t = json.load(open(path))
    except (OSError, ValueError):
        return None
    if t.get("source_sha") != scan_source_hash(sources):
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
    """The FP64 CPU oracle on the default workload (the load path), each step
    a bounded sample: `cpu_points` (default 8) evenly spaced points of load
    step k (k = 1, 2, ... cycling over the path), with their history."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_2211_14318_gb300 import inputs

    oracle.build()
    cores = host_cores()
    path = inputs.load_path(a.lp_nx, n_steps=LP_STEPS, stretch_end=LP_STRETCH, seed=LP_SEED)
    npts = a.cpu_points or 8
    for i in range(a.warmup):
        loadpath_oracle_rate(path, 1 + i % LP_STEPS, cores, 1)
    times = []
    for i in range(a.steps):
        r = loadpath_oracle_rate(path, 1 + i % LP_STEPS, cores, npts)
        times.append(npts / r["value"])
    value = npts * a.steps / sum(times)
    n = path[0].shape[0]
    sample = (f"{npts} evenly spaced points of load step k per step (k = 1, 2, ... cycling over "
              f"the {LP_STEPS} steps), with their history")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "points/s",
        "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * sum(times) / a.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": (f"load path, {a.lp_nx}x{a.lp_nx} Q1 mesh x 4 Gauss points = {n} "
                                f"points, {LP_STEPS} load steps (stretch 1.0 -> {LP_STRETCH}), "
                                f"history updated, {LP_ANGLES}x{LP_ANGLES} angles, L={LP_LINE}, "
                                f"t in [-0.5,0.5], depth {LP_DEPTH}"),
                   "form": "full scan (the oracle has no proposal network)"},
        "cpu_baseline": {"value": value, "unit": "points/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
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


# ----------------------------------------------------- load path (the metric)
LP_STEPS, LP_ANGLES, LP_LINE, LP_DEPTH, LP_SEED, LP_STRETCH = 20, 128, 2049, 3, 7, 1.8
MP_ANGLES, MP_LINE, MP_DEPTH, MP_POINTS, MP_SEED = 16, 201, 2, 1 << 20, 201
GOLDEN = os.path.join(ROOT, "tests", "golden")
CHECK_STEPS = (1, 10, 20)


def load_golden(name):
    """Stored FP64 oracle results of 4,096 points of a workload (or None)."""
    import numpy as np

    path = os.path.join(GOLDEN, f"{name}.npz")
    if not os.path.exists(path):
        return None
    g = dict(np.load(path))
    g["meta"] = json.loads(str(g["meta"]))
    return g


def err_stats(W, Wo, P=None, Po=None):
    """Relative W^R and P errors (gamma = 1e-8, Sec. 6.2): p50 / p99 / max."""
    import numpy as np

    e = np.abs(W - Wo) / (1e-8 + np.abs(Wo))
    out = {"points": int(e.size), "W_R_p50": float(np.quantile(e, 0.5)),
           "W_R_p99": float(np.quantile(e, 0.99)), "W_R_max": float(e.max())}
    if P is not None:
        ep = np.linalg.norm(P - Po, axis=1) / (1e-8 + np.linalg.norm(Po, axis=1))
        out.update(P_p50=float(np.quantile(ep, 0.5)), P_p99=float(np.quantile(ep, 0.99)),
                   P_max=float(ep.max()))
    return out


def train_proposal(cv, api, inputs, path, dev):
    """The proposal network, trained on the GPU: labels from the GPU's own full
    scans (131,072 material points with lambda in [1, 2], and 16,384 points
    of the load path at five steps; 128^2 grid, L = 513, depth 2), then 30
    epochs of Adam (batch 8,192) on the tensor cores."""
    import numpy as np
    import torch

    pl = api.Params(n_theta_a=LP_ANGLES, n_theta_b=LP_ANGLES, line_points=513, depth=2, **MAT)
    F1, Fp1 = inputs.surrogate_inputs(131072, seed=100)
    b1 = cv.history_update(pl, Fp1)
    t0 = time.perf_counter()
    out = cv.convexify_points(pl, F1, b1, want_tree=True)
    X, Y = cv.surrogate_labels(pl, b1, out["tree"], F1.shape[0])
    Xs, Ys = [X], [Y]
    steps = len(path)
    for k in (3, 7, 11, 15, 19):
        k = min(k, steps - 1)
        Fk = path[k]
        bk = cv.history_update(pl, path[k - 1]).cpu().numpy()
        idx = np.random.default_rng(k).choice(Fk.shape[0], min(16384, Fk.shape[0]), replace=False)
        out = cv.convexify_points(pl, Fk[idx], bk[idx], want_tree=True)
        X, Y = cv.surrogate_labels(pl, bk[idx], out["tree"], len(idx))
        Xs.append(X)
        Ys.append(Y)
    X, Y = torch.cat(Xs), torch.cat(Ys)
    torch.cuda.synchronize()
    t_label = time.perf_counter() - t0
    t0 = time.perf_counter()
    log = cv.surrogate_train(X, Y, epochs=30, batch=8192, lr=1e-3, init=True, seed=0)
    return {"samples": int(X.shape[0]), "label_s": t_label, "train_s": time.perf_counter() - t0,
            "loss_first": float(log[0]), "loss_last": float(log[-1])}


def propose_launches(n, K, R, mirror=False):
    """Kernels of this library one surrogate_propose call and its history
    update launch: k_init; per level and 65,536-node chunk the features, five
    tensor-core GEMMs and the decoding; per level R + 1 window passes, R + 1
    mirror-window passes (with the mirror window) and the fallback pass (line
    scan, select, refine, commit each); k_leaf, k_fell_back; k_history."""
    chunks = sum(-(-(n << l) // 65536) for l in range(K))
    passes = (R + 1) * (2 if mirror else 1) + 1
    return 1 + 7 * chunks + 4 * passes * K + 3


def timed_full_scan(cv, p, F, beta, steps, torch):
    """CUDA-event time of `steps` plain convexify_points calls (after two
    warm calls), the line-scan launches' own time and the counters."""
    import numpy as np

    for _ in range(2):
        cv.convexify_points(p, F, beta)
    torch.cuda.synchronize()
    cv.stats(reset=True)
    cv.set_profiling(True)
    cv.scan_timing(reset=True)
    ms = 0.0
    for _ in range(steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = cv.convexify_points(p, F, beta)
        e1.record()
        torch.cuda.synchronize()
        ms += e0.elapsed_time(e1)
    scan_ms, launches = cv.scan_timing(reset=True)
    cv.set_profiling(False)
    st = cv.stats(reset=True)
    return ms, scan_ms, launches, st, out


def roofline_obj(st, scan_ms, launches, step_ms, peak, sms, mhz, peak_src, traffic_name=None):
    flop = FLOP_PER_SAMPLE * st["valid_samples"]
    achieved = flop / (scan_ms / 1e3) / 1e12 if scan_ms > 0 else None
    traffic = (traffic_per_launch(st["valid_samples"] / max(1, launches), traffic_name)
               if traffic_name else None)
    return {"bound": "alu", "kernel": "k_scan_lanes", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": (achieved / peak) if achieved else None,
            "traffic": traffic,
            "peak_source": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {mhz:.0f} MHz ({peak_src})",
            "flop_per_valid_sample": FLOP_PER_SAMPLE,
            "kernel_share_of_step": scan_ms / step_ms if step_ms else None,
            "launches": launches}


def run_loadpath(a):
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
    from paper_2211_14318_gb300 import api, inputs

    cv = api.Convexifier(local)
    strong = ws > 1 and a.scaling == "strong"
    path = inputs.load_path(a.lp_nx, n_steps=LP_STEPS, stretch_end=LP_STRETCH,
                            seed=LP_SEED + (0 if strong else rank))
    K = max(1, min(a.steps, LP_STEPS))
    train = train_proposal(cv, api, inputs, path, dev)
    p = api.Params(n_theta_a=LP_ANGLES, n_theta_b=LP_ANGLES, line_points=LP_LINE, depth=LP_DEPTH,
                   recentre=a.recentre, gap_one_sided=a.gap_one_sided, mirror=not a.no_mirror,
                   **MAT)
    pf = api.Params(n_theta_a=LP_ANGLES, n_theta_b=LP_ANGLES, line_points=LP_LINE,
                    depth=LP_DEPTH, **MAT)
    n_all = path[0].shape[0]
    lo, hi = 0, n_all
    if strong:
        # one problem split into contiguous ranges weighted by expected tree
        # size: a point past its history at the last timed step (psi0 > beta)
        # is expected to split (about 3 more scanned nodes at depth 3)
        bK = torch.zeros(n_all, dtype=torch.float64, device=dev)
        for j in range(K - 1):
            bK = cv.history_update(pf, path[j], bK)
        ps = cv.history_update(pf, path[K - 1])
        wts = (1.0 + 3.0 * (ps > bK).double()).cpu().numpy()
        lo, hi = rank_ranges(wts, ws)[rank]
        path = [x[lo:hi].copy() for x in path]
    n = path[0].shape[0]
    kw = dict(window=a.window, gap_tol=a.gap_tol)

    # ---- warm-up: load steps of the proposed form on the first 65,536 points
    nw = min(n, 65536)
    bw = torch.zeros(nw, dtype=torch.float64, device=dev)
    for k in range(a.warmup):
        Fk = torch.from_numpy(path[k % LP_STEPS][:nw]).to(dev)
        cv.surrogate_propose(p, Fk, bw, **kw)
        bw = cv.history_update(p, Fk, bw)
    torch.cuda.synchronize()

    # ---- timed: K load steps of 1,048,576 points, history carried over
    Fh = torch.empty((n, 4), dtype=torch.float64).pin_memory()
    Wh = torch.empty(n, dtype=torch.float64).pin_memory()
    Ph = torch.empty((n, 4), dtype=torch.float64).pin_memory()
    Fd = torch.empty((n, 4), dtype=torch.float64, device=dev)
    beta = torch.zeros(n, dtype=torch.float64, device=dev)
    out = dict(W_R=torch.empty(n, dtype=torch.float64, device=dev),
               P=torch.empty(n, 4, dtype=torch.float64, device=dev),
               status=torch.empty(n, dtype=torch.int32, device=dev),
               fell_back=torch.empty(n, dtype=torch.uint8, device=dev))
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > 129 MB L2
    gold = {}
    if rank == 0 and a.lp_nx == 512 and not strong:
        for k in CHECK_STEPS:
            g = load_golden(f"loadpath512_s{k:02d}")
            if g is not None and k <= K:
                gold[k] = g
    uuid = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    clocks = ClockSampler(f"GPU-{uuid}" if uuid is not None else str(local))
    cv.stats(reset=True)
    cv.set_profiling(True)
    cv.scan_timing(reset=True)
    comp_ms, e2e_ms, per_step, fell, checks = 0.0, 0.0, [], [], {}
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    wall0 = time.perf_counter()
    for k in range(1, K + 1):
        Fh.copy_(torch.from_numpy(path[k - 1]))
        flush.zero_()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record()
        Fd.copy_(Fh, non_blocking=True)
        ev[1].record()
        if k == a.profile_step:
            torch.cuda.profiler.start()
        cv.surrogate_propose(p, Fd, beta, out=out, **kw)
        beta = cv.history_update(p, Fd, beta)  # Eq. (2.5) for the next load step
        if k == a.profile_step:
            torch.cuda.profiler.stop()
        ev[2].record()
        Wh.copy_(out["W_R"], non_blocking=True)
        Ph.copy_(out["P"], non_blocking=True)
        ev[3].record()
        torch.cuda.synchronize()
        t = ev[1].elapsed_time(ev[2])
        comp_ms += t
        e2e_ms += ev[0].elapsed_time(ev[3])
        per_step.append(t)
        fell.append(float(out["fell_back"].float().mean()))
        if k in gold:
            idx = gold[k]["idx"]
            checks[k] = (Wh.numpy()[idx].copy(), Ph.numpy()[idx].copy(),
                         float(np.abs(path[k - 1][idx] - gold[k]["F"]).max()))
    wall = time.perf_counter() - wall0
    ck = clocks.stop()
    if ws > 1:
        dist.barrier()
    scan_ms, scan_launches = cv.scan_timing(reset=True)
    cv.set_profiling(False)
    st = cv.stats(reset=True)
    t_max = max_over_ranks(comp_ms, dist if ws > 1 else None, dev)
    e2e_max = max_over_ranks(e2e_ms, dist if ws > 1 else None, dev)
    if strong:  # all ranks together convexified the one problem
        value = n_all * K / (t_max / 1e3)
        e2e_value = n_all * K / (e2e_max / 1e3)
    else:
        value = whole_job_rate(n, ws, K, t_max)
        e2e_value = whole_job_rate(n, ws, K, e2e_max)
    peak, sms, mhz, peak_src = fp32_peak_tflops(torch, dev)

    if rank == 0:
        # accuracy of the proposed form against the oracle (stored results)
        acc = {}
        for k, (W, P, dF) in checks.items():
            g = gold[k]
            acc[f"step_{k}"] = dict(err_stats(W, g["W_R"], P, g["P"]), max_abs_dF=dF,
                                    fell_back_points=fell[k - 1])
        # the plain full scan on the same steps: points/s on 65,536 points of
        # the step, and its own accuracy on the 4,096 stored points
        full, pareto = {}, {}
        nt = min(n, 65536)
        for k in CHECK_STEPS:
            if k > K:
                continue
            bk = torch.zeros(nt, dtype=torch.float64, device=dev)
            for j in range(k - 1):
                bk = cv.history_update(pf, path[j][:nt], bk)
            Fk = torch.from_numpy(path[k - 1][:nt]).to(dev)
            ms, _, _, _, _ = timed_full_scan(cv, pf, Fk, bk, 1, torch)
            row = {"pts_per_s": nt / (ms / 1e3), "proposed_pts_per_s": n / (per_step[k - 1] / 1e3)}
            if k in gold:
                g = gold[k]
                r = cv.convexify_points(pf, g["F"], g["beta"])
                row.update(err_stats(r["W_R"].cpu().numpy(), g["W_R"], r["P"].cpu().numpy(), g["P"]))
                for na in (16, 32, 64):
                    q = api.Params(n_theta_a=na, n_theta_b=na, line_points=LP_LINE, depth=LP_DEPTH,
                                   **MAT)
                    rq = cv.convexify_points(q, g["F"], g["beta"])
                    msq, _, _, _, _ = timed_full_scan(cv, q, Fk, bk, 1, torch)
                    pareto.setdefault(f"{na}x{na}", {})[f"step_{k}"] = dict(
                        err_stats(rq["W_R"].cpu().numpy(), g["W_R"]), pts_per_s=nt / (msq / 1e3))
            full[f"step_{k}"] = row
        extras = {}
        if not a.no_extras:
            extras["material_points_l201"] = material_points_line(
                a, cv, api, inputs, torch, dev, peak, sms, mhz, peak_src, K)
            extras["material_points_l201_adaptive_window"] = material_points_line(
                a, cv, api, inputs, torch, dev, peak, sms, mhz, peak_src, 3, doublings=5)
            extras["mesh128"] = mesh128_line(cv, api, torch, dev, peak, sms, mhz, peak_src,
                                             min(K, 5))
            extras["global_grid"] = global_grid_line(a, cv, api, inputs, torch, dev, sms, mhz,
                                                     peak_src, cpu=ws == 1 and not a.no_cpu_baseline)
        cpu = None
        if ws == 1 and not a.no_cpu_baseline:
            cpu = loadpath_oracle_rate(path, K, host_cores(), 8)
            cpu1 = loadpath_oracle_rate(path, K, 1, 1)
            cpu["one_core"] = {"value": cpu1["value"], "sample": cpu1["sample"]}
        wn, fb, rc = st["window_nodes"], st["fallbacks"], st["recentred"]
        first_pass = max(1, wn - rc - st["mirror_windows"])
        line = {
            "metric": METRIC, "value": value, "unit": "points/s", "n_gpus": ws, "steps": K,
            "warmup": a.warmup, "ms_per_step": t_max / K, "higher_is_better": True,
            "scaling": "strong" if strong else "weak", "vs_baseline": None,
            "dtype": "bf16/f32/f64", "data": "synthetic",
            "config": {
                "workload": (f"load path, {a.lp_nx}x{a.lp_nx} Q1 mesh x 4 Gauss points = {n_all} points, "
                             f"load steps 1..{K} of {LP_STEPS} (stretch 1.0 -> {LP_STRETCH}), history "
                             f"updated, {LP_ANGLES}x{LP_ANGLES} angles, window +-{a.window} "
                             f"re-centred up to {a.recentre} times"
                             + ("" if a.no_mirror else f", mirror window +-{(a.window + 1) // 2}")
                             + f", L={LP_LINE}, t in [-0.5,0.5], "
                             f"depth {LP_DEPTH}; surrogate-proposed with full-scan fallback"),
                "form": "surrogate", "points_per_gpu": n, "window": a.window,
                "mirror_window": None if a.no_mirror else (a.window + 1) // 2,
                "rank_range": [lo, hi] if strong else None,
                "recentre": a.recentre, "gap_tol": a.gap_tol,
                "fallback_rule": ("border: the window minimum still on the window border after "
                                  "the re-centrings" + ("" if a.gap_tol >= 1e29 else
                                                        f"; or energy gap > {a.gap_tol}")),
                "l2": "flushed between steps (512 MiB write)",
                "timed": "H2D of F excluded from value (included in e2e); proposal + history update",
                "wall_s_timed_region": wall},
            "roofline": roofline_obj(st, scan_ms, scan_launches, comp_ms, peak, sms, mhz, peak_src,
                                     "k_scan_lanes_traffic.json"),
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "points/s", "h2d_bytes_per_step": n * 4 * 8,
                    "d2h_bytes_per_step": n * 8 + n * 4 * 8},
            "gpu_launches": K * propose_launches(n, LP_DEPTH, a.recentre, not a.no_mirror),
            "clocks": ck,
            "accuracy_vs_oracle": acc,
            "fallback": {"window_nodes_first_pass": first_pass, "recentred": rc, "fallback_nodes": fb,
                         "fallback_rate": fb / first_pass,
                         "mirror_windows": st["mirror_windows"], "mirror_won": st["mirror_won"],
                         "points_with_a_fallback_mean": sum(fell) / len(fell)},
            "full_scan": full, "pareto": pareto, "train": train,
            "per_step_ms": per_step,
            **extras,
            "stats": st,
        }
        print(json.dumps(line), flush=True)
    cv.close()
    if ws > 1:
        dist.destroy_process_group()


def material_points_line(a, cv, api, inputs, torch, dev, peak, sms, mhz, peak_src, steps, doublings=0):
    """1,048,576 material points at 16 x 16 angles, L = 201, depth 2 (the
    full scan): throughput, the line scan's roofline and the error against the
    stored oracle results of 4,096 points (placed at their rows).  With
    doublings > 0 the adaptive line window (t_half up to 0.5 2^doublings): the
    same workload with laminates no longer cut at t = +-0.5 (no stored oracle
    results: its W^R is compared with the fixed window's instead)."""
    import numpy as np

    npts = getattr(a, "mp_points", MP_POINTS)
    F, Fp = inputs.surrogate_inputs(npts, seed=MP_SEED)
    p = api.Params(n_theta_a=MP_ANGLES, n_theta_b=MP_ANGLES, line_points=MP_LINE, depth=MP_DEPTH,
                   window_doublings=doublings, **MAT)
    beta = cv.history_update(p, Fp).cpu().numpy()
    g = load_golden("material1m_l201") if npts == MP_POINTS else None
    if g is not None:
        F[g["idx"]] = g["F"]
        beta[g["idx"]] = g["beta"]
    Fd = torch.from_numpy(F).to(dev)
    bd = torch.from_numpy(beta).to(dev)
    ms, scan_ms, launches, st, out = timed_full_scan(cv, p, Fd, bd, steps, torch)
    res = {"workload": (f"{npts} material points (F = Q diag(lam, lam^-0.3) Q^T + noise, "
                        f"lam ~ U[1, 2]), {MP_ANGLES}x{MP_ANGLES} angles, L={MP_LINE}, "
                        f"t in [-0.5,0.5]" + (f" doubled up to {doublings} times per node"
                                              if doublings else "") +
                        f", depth {MP_DEPTH}, full scan"),
           "value": npts * steps / (ms / 1e3), "unit": "points/s", "steps": steps,
           "ms_per_step": ms / steps,
           "roofline": roofline_obj(st, scan_ms, launches, ms, peak, sms, mhz, peak_src,
                                    "k_scan_lanes_l201_traffic.json"),
           "stats": st}
    if g is not None and not doublings:
        it = torch.from_numpy(g["idx"]).to(dev)
        res["accuracy_vs_oracle"] = err_stats(out["W_R"][it].cpu().numpy(), g["W_R"],
                                              out["P"][it].cpu().numpy(), g["P"])
    if doublings:
        q = api.Params(n_theta_a=MP_ANGLES, n_theta_b=MP_ANGLES, line_points=MP_LINE,
                       depth=MP_DEPTH, **MAT)
        fixed = cv.convexify_points(q, Fd, bd)["W_R"]
        d = fixed - out["W_R"]  # W units: how much lower the wider windows relax
        res["W_R_drop_vs_fixed_window"] = {
            "mean": float(d.mean()), "max": float(d.max()), "min": float(d.min()),
            "points_lower": float((d > 0).double().mean()),
            "mean_fixed_W_R": float(fixed.mean())}
    return res


def mesh128_line(cv, api, torch, dev, peak, sms, mhz, peak_src, steps):
    """The 65,536-point mesh (128 x 128 Q1 x 4 Gauss points, stretch 1.3),
    64 x 64 angles, L = 1025, depth 3, full scan."""
    from paper_2211_14318_gb300 import inputs

    F, Fp = inputs.mesh_points(NX, stretch=STRETCH, seed=0)
    p = api.Params(n_theta_a=ANGLES, n_theta_b=ANGLES, line_points=LINE, t_half=T_HALF,
                   depth=DEPTH, **MAT)
    beta = cv.history_update(p, Fp).cpu().numpy()
    g = load_golden("mesh128")
    if g is not None:
        F[g["idx"]] = g["F"]
        beta[g["idx"]] = g["beta"]
    Fd = torch.from_numpy(F).to(dev)
    bd = torch.from_numpy(beta).to(dev)
    ms, scan_ms, launches, st, out = timed_full_scan(cv, p, Fd, bd, steps, torch)
    res = {"workload": workload_desc(F.shape[0]), "value": F.shape[0] * steps / (ms / 1e3),
           "unit": "points/s", "steps": steps, "ms_per_step": ms / steps,
           "roofline": roofline_obj(st, scan_ms, launches, ms, peak, sms, mhz, peak_src),
           "stats": st}
    if g is not None:
        it = torch.from_numpy(g["idx"]).to(dev)
        res["accuracy_vs_oracle"] = err_stats(out["W_R"][it].cpu().numpy(), g["W_R"],
                                              out["P"][it].cpu().numpy(), g["P"])
    return res


# The global-grid study of Sec. 6.1 (Table tab:2Dconvexification, NH row)
GRID61 = dict(diag=(0.1, 3.4), off=(-2.55, 2.55), delta=(0.15, 0.15), beta=0.06, kmax=20,
              tol=1e-4, mat=dict(mu=1.0, lambda_L=0.5, D_inf=0.9, D0=0.3))
# the strong-scaling study of Sec. 6.4 times a 43,681-point grid (11 x 19 x 19 x 11
# points) whose bounds are not printed; this one has that shape at delta 0.15
GRID_SCALING = dict(diag=(0.4, 1.9), off=(-1.35, 1.35), delta=(0.15, 0.15))
FP64_FMA_PER_SM = 2       # FP64 FMA per SM per clock on GB300 (1.25 TFLOP/s nominal)
GRID_FLOP_PER_POINT_DIR = 12  # Algorithm 1 (2 predicates x 4) + the chord at the point (4)


def global_grid_line(a, cv, api, inputs, torch, dev, sms, mhz, peak_src, runs=10,
                     cpu=True):
    """The paper's own algorithm on the grid of its Sec. 6.1 study: 648,025
    grid points, R^1_1, W^0 then Eq. (4.3) until the largest decrease is at
    most 1e-4 (15 steps), timed whole on the device (L2 flushed before each
    run); the line kernel's roofline against the FP64 pipe; Algorithms 2/3 at
    1,048,576 query points; accuracy against the stored oracle results."""
    import numpy as np

    c = GRID61
    g = api.GridSpec.from_bounds(c["diag"], c["off"], c["delta"])
    off = api.grid_r11()
    p = api.Params(**c["mat"])
    N, nd = g.count, off.shape[0]
    out = dict(W=torch.empty(N, dtype=torch.float64, device=dev),
               forest=torch.empty(c["kmax"], N, 3, dtype=torch.int32, device=dev),
               decs=torch.empty(c["kmax"], dtype=torch.float64, device=dev),
               iters=torch.empty(1, dtype=torch.int32, device=dev))
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def run(kmax=c["kmax"]):
        return cv.grid_convexify(p, g, c["beta"], off, kmax=kmax, tol=c["tol"], det_rule=1,
                                 out=out)

    for _ in range(2):
        run()
    torch.cuda.synchronize()
    K = int(out["iters"].cpu()[0])
    ms = []
    for _ in range(runs):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    t = statistics.median(ms)
    # the line kernel alone: a run with kmax = K (no skipped launches), events
    # on the launching stream around each line-kernel launch
    flush.zero_()
    cv.set_profiling(True)
    cv.scan_timing(reset=True)
    run(K)
    torch.cuda.synchronize()
    lines_ms, launches = cv.scan_timing(reset=True)
    cv.set_profiling(False)
    flop = GRID_FLOP_PER_POINT_DIR * N * nd * launches
    peak = sms * FP64_FMA_PER_SM * 2 * mhz * 1e6 / 1e12
    achieved = flop / (lines_ms / 1e3) / 1e12 if lines_ms > 0 else None
    traffic = traffic_per_launch(N * nd, "k_grid_lines_traffic.json", GRID_SOURCES)
    res = {"workload": (f"global grid of the Sec. 6.1 NH study: {g.n[0]}x{g.n[1]}x{g.n[2]}x{g.n[3]} "
                        f"= {N} grid points (delta 0.15, diagonal {list(c['diag'])}, off-diagonal "
                        f"{list(c['off'])}), R^1_1 ({nd} directions), beta_k {c['beta']}, "
                        f"W^0 then Eq. (4.3) to tol {c['tol']} (kmax {c['kmax']}), ln|det F|"),
           "value": N * K / (t / 1e3), "unit": "grid-point updates/s (points x steps)",
           "steps_to_tol": K, "ms_to_tol": t, "ms_runs": ms,
           "l2": "flushed before each run (256 MiB write); the grid (5.2 MB) fits in L2 within a run",
           "roofline": {"bound": "alu", "kernel": "k_grid_lines", "achieved": achieved,
                        "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak if achieved else None,
                        "traffic": traffic,
                        "peak_source": (f"{sms} SMs x {FP64_FMA_PER_SM} FP64 FMA x 2 x {mhz:.0f} MHz "
                                        f"(nominal FP64 rate; {peak_src})"),
                        "flop_per_point_direction": GRID_FLOP_PER_POINT_DIR,
                        "kernel_ms_per_launch": lines_ms / max(1, launches),
                        "kernel_share": lines_ms / t, "launches": launches},
           "gpu_launches_per_run": 1 + 1 + c["kmax"] * 3 + 1}
    # Algorithms 2 and 3 at 1,048,576 points of the grid's box
    lo = np.array(g.lo)
    hi = lo + (np.array(g.n) - 1) * np.array(g.delta)
    Fq = torch.from_numpy(inputs.cuboid_points(lo, hi, 1 << 20, seed=62)).to(dev)
    fo = out["forest"][:K]
    for _ in range(2):
        cv.grid_query(p, g, c["beta"], off, out["W"], fo, Fq, det_rule=1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    wi, wt, Pq, nl = cv.grid_query(p, g, c["beta"], off, out["W"], fo, Fq, det_rule=1)
    e1.record()
    torch.cuda.synchronize()
    qms = e0.elapsed_time(e1)
    cv.grid_query(p, g, c["beta"], off, out["W"], fo, Fq, det_rule=1, want_A=True)
    torch.cuda.synchronize()
    e0.record()
    cv.grid_query(p, g, c["beta"], off, out["W"], fo, Fq, det_rule=1, want_A=True)
    e1.record()
    torch.cuda.synchronize()
    ams = e0.elapsed_time(e1)
    res["query"] = {"points": int(Fq.shape[0]), "pts_per_s": Fq.shape[0] / (qms / 1e3),
                    "ms_with_tangent": ams,
                    "ms": qms, "leaves_mean": float(nl.double().mean()),
                    "leaves_max": int(nl.max()),
                    "tree_minus_interp_max": float((wt - wi).abs().max())}
    gold = load_golden("grid61")
    if gold is not None:
        Wg = out["W"].cpu().numpy()[gold["idx"]]
        d = np.asarray(gold["decs"])
        dg = out["decs"].cpu().numpy()[:K]
        wi2, wt2, P2, nl2 = cv.grid_query(p, g, c["beta"], off, out["W"], fo, gold["F_query"],
                                          det_rule=1)
        res["accuracy_vs_oracle"] = {
            "steps_equal": bool(K == d.size),
            "decrease_max_abs_diff": float(np.max(np.abs(dg - d))) if K == d.size else None,
            "W_K": err_stats(Wg, gold["W_K"]),
            "query": err_stats(wt2.cpu().numpy(), gold["W_tree"], P2.cpu().numpy(), gold["P"]),
            "query_P_note": ("P follows the laminates, which differ from the oracle's at "
                             "zero-decrease splits decided by the last bit of W^0 (each side's "
                             "libm); from the same forest P agrees within 1e-12"),
            "query_leaves_equal": float(np.mean(nl2.cpu().numpy() == gold["leaves"]))}
    # the shape of the Sec. 6.4 strong-scaling grid (context for the paper's timings)
    gs = api.GridSpec.from_bounds(GRID_SCALING["diag"], GRID_SCALING["off"], GRID_SCALING["delta"])
    for _ in range(2):
        o2 = cv.grid_convexify(p, gs, c["beta"], off, kmax=c["kmax"], tol=c["tol"], det_rule=1,
                               want_forest=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    o2 = cv.grid_convexify(p, gs, c["beta"], off, kmax=c["kmax"], tol=c["tol"], det_rule=1,
                           want_forest=False)
    e1.record()
    torch.cuda.synchronize()
    res["grid_43681"] = {"grid": list(gs.n), "points": gs.count,
                         "steps_to_tol": int(o2["iters"].cpu()[0]), "ms_to_tol": e0.elapsed_time(e1),
                         "paper_context": ("Sec. 6.4: 1960.7 s on 1 thread, 49.06 s on 64 threads of a "
                                           "Xeon Phi 7210 for a 43,681-point grid with R^1_1, no tree "
                                           "(bounds not printed)")}
    res["stvk61"] = grid_study_line(cv, api, torch, dev, flush, "stvk61", sms, mhz)
    res["grid3d"] = grid_study_line(cv, api, torch, dev, flush, "grid3d", sms, mhz)
    if cpu:
        res["cpu_baseline"] = grid_oracle_rate(out["W"], K)
    return res


def grid_study_line(cv, api, torch, dev, flush, name, sms, mhz, runs=5):
    """The STVK study of Sec. 6.1 (672,400 points, Eq. 2.2 kept where
    det F <= 0) or the nine-dimensional NH study of Sec. 6.8 (3,581,577
    points, 169 directions): time to tol, the line kernel's FP64 rate and the
    accuracy against the stored oracle run (and the printed curves)."""
    import numpy as np

    gold = load_golden(name)
    c = GRID61["mat"]
    if name == "stvk61":
        g = api.GridSpec.from_bounds((0.1, 2.0), (-2.0, 2.0), (0.1, 0.1))
        p = api.Params(energy=api.ENERGY_STVK_DAMAGE, **c)
        beta, rule, off = 0.07, 1, api.grid_r11(2)
    else:
        g = api.GridSpec.from_bounds((1.0, 3.4), (-0.15, 0.15), (0.15, 0.15), dim=3)
        p = api.Params(**c)
        beta = gold["meta"]["beta"] if gold is not None else 0.0625
        rule, off = 0, api.grid_r11(3)
    N, nd = g.count, off.shape[0]
    out = dict(W=torch.empty(N, dtype=torch.float64, device=dev),
               forest=torch.empty(20, N, 3, dtype=torch.int32, device=dev),
               decs=torch.empty(20, dtype=torch.float64, device=dev),
               iters=torch.empty(1, dtype=torch.int32, device=dev))

    def run(kmax=20):
        return cv.grid_convexify(p, g, beta, off, kmax=kmax, tol=1e-4, det_rule=rule, out=out)

    run()
    torch.cuda.synchronize()
    K = int(out["iters"].cpu()[0])
    ms = []
    for _ in range(runs):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    t = statistics.median(ms)
    flush.zero_()
    cv.set_profiling(True)
    cv.scan_timing(reset=True)
    run(K)
    torch.cuda.synchronize()
    lines_ms, launches = cv.scan_timing(reset=True)
    cv.set_profiling(False)
    chunks = max(1, launches // K)
    flop = GRID_FLOP_PER_POINT_DIR * N * nd * K
    peak = sms * FP64_FMA_PER_SM * 2 * mhz * 1e6 / 1e12
    achieved = flop / (lines_ms / 1e3) / 1e12 if lines_ms > 0 else None
    res = {"workload": (f"{'STVK study of Sec. 6.1' if name == 'stvk61' else 'nine-dimensional NH study of Sec. 6.8'}: "
                        f"{N} grid points, {nd} directions, tol 1e-4"),
           "value": N * K / (t / 1e3), "unit": "grid-point updates/s (points x steps)",
           "steps_to_tol": K, "ms_to_tol": t,
           "line_kernel": {"achieved_tflops": achieved, "frac_of_fp64_peak": achieved / peak if achieved else None,
                           "ms_per_step": lines_ms / K, "launches_per_step": chunks,
                           "share": lines_ms / t}}
    if gold is not None:
        WK = out["W"].cpu().numpy()
        acc = {"steps_equal": bool(K == gold["decs"].size),
               "decrease_max_abs_diff": float(np.max(np.abs(out["decs"].cpu().numpy()[:K] - gold["decs"])))
               if K == gold["decs"].size else None,
               "W_K": err_stats(WK[gold["idx"]], gold["W_K"])}
        if name == "grid3d":
            rows = np.array([[float(v) for v in ln.split()] for ln in
                             open(os.path.join(GOLDEN, "nh3d_paths.txt"))
                             if ln.strip() and not ln.startswith("#")])
            acc["paths_vs_oracle_max_abs"] = float(np.max(np.abs(WK[gold["paths"]] - gold["W_paths"])))
            acc["biaxial_vs_printed_max_abs"] = float(np.max(np.abs(WK[gold["paths"][1]] - rows[:, 4])))
            acc["triaxial_vs_printed_max_abs"] = float(np.max(np.abs(WK[gold["paths"][2]] - rows[:, 6])))
        res["accuracy_vs_oracle"] = acc
    return res


def grid_oracle_rate(WK, K):
    """The FP64 CPU oracle (as it stands) taking one step of Eq. (4.3) on the
    whole 648,025-point grid from the device's W^K (all host cores)."""
    import oracle

    oracle.build()
    c = GRID61
    go = oracle.Grid.from_bounds(c["diag"], c["off"], c["delta"])
    off = oracle.r11_directions()
    W = WK.cpu().numpy()
    t0 = time.perf_counter()
    oracle.grid_step(go, off, W)
    dt = time.perf_counter() - t0
    return {"value": go.count / dt, "unit": "grid-point updates/s (points x steps)",
            "cores": host_cores(), "kind": "oracle",
            "sample": f"one step of Eq. (4.3) on the whole {go.count}-point grid ({dt:.2f} s)"}


def run_grid(a):
    """The global-grid form alone: one JSON line."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2211_14318_gb300 import api, inputs

    dev = torch.device("cuda:0")
    torch.cuda.set_device(0)
    cv = api.Convexifier(0)
    _, sms, mhz, peak_src = fp32_peak_tflops(torch, dev)
    uuid = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    clocks = ClockSampler(f"GPU-{uuid}" if uuid is not None else "0")
    clocks.start()
    res = global_grid_line(a, cv, api, inputs, torch, dev, sms, mhz, peak_src,
                           runs=max(3, a.steps), cpu=not a.no_cpu_baseline)
    ck = clocks.stop()
    res.update(metric="grid-point updates/s of the global-grid rank-one convexification (Eq. 4.3)",
               n_gpus=1, warmup=2, higher_is_better=True, dtype="f64", data="synthetic",
               clocks=ck)
    print(json.dumps(res), flush=True)
    cv.close()


def loadpath_oracle_rate(path, step, cores, npts):
    """The FP64 CPU oracle (as it stands) on npts evenly spaced points of load
    step `step` of the path, with the history of the earlier steps."""
    import numpy as np

    import oracle

    oracle.build()
    mat = oracle.Material(MAT["mu"], MAT["lambda_L"], MAT["D_inf"], MAT["D0"])
    sc = oracle.Scan(oracle.angle_directions(LP_ANGLES, LP_ANGLES), LP_LINE, 0.5, LP_DEPTH)
    n = path[0].shape[0]
    idx = np.linspace(0, n - 1, npts).astype(np.int64)
    beta = np.zeros(npts)
    for j in range(step - 1):
        beta = oracle.history_update(mat, path[j][idx], beta)
    t0 = time.perf_counter()
    oracle.convexify(mat, sc, path[step - 1][idx], beta, nthreads=cores)
    dt = time.perf_counter() - t0
    return {"value": npts / dt, "unit": "points/s", "cores": cores, "kind": "oracle",
            "sample": f"{npts} evenly spaced points of load step {step} ({dt:.1f} s)"}


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
                   gap_one_sided=a.gap_one_sided, recentre=a.recentre, mirror=not a.no_mirror,
                   **MAT)
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


# ------------------------------------------------------------- batched form
def run_batch(a):
    """The batched form: 256 meshes with log-uniform point counts in
    [1e3, 1e5] (about 5.5 M points), per-problem stretch, angle grid (32^2 or
    64^2), line (513 or 1025) and depth (2 or 3), in one autotuned,
    graph-captured run; a step is one graph replay over all problems.  Also
    the same batch with the launch shape fixed to the warp-per-line scan's
    default (8 warps, no item cap), for the autotuner's gain."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2211_14318_gb300 import api, inputs

    dev = torch.device("cuda:0")
    torch.cuda.set_device(0)
    probs = inputs.batch_problems(256, seed=0)
    cache = os.path.join(tempfile.gettempdir(), f"cvx_tune_{os.getpid()}.json")
    if os.path.exists(cache):
        os.remove(cache)
    os.environ["CVX_AUTOTUNE_CACHE"] = cache

    def make(cv):
        items, total = [], 0
        for pr in probs:
            p = api.Params(n_theta_a=pr.n_angle, n_theta_b=pr.n_angle, line_points=pr.L,
                           depth=pr.depth, **MAT)
            beta = cv.history_update(p, pr.F_prev)
            items.append((p, torch.as_tensor(pr.F, device=dev), beta))
            total += pr.F.shape[0]
        return items, total

    def timed(cv, items):
        t0 = time.perf_counter()
        outs = cv.convexify_batch(items)  # autotune + capture (+ launch)
        torch.cuda.synchronize()
        setup = time.perf_counter() - t0
        for _ in range(a.warmup):
            cv.convexify_batch(items, outs=outs)
        torch.cuda.synchronize()
        cv.stats(reset=True)
        ms = 0.0
        for _ in range(a.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            cv.convexify_batch(items, outs=outs)
            e1.record()
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
        return ms, setup, cv.stats(reset=True), cv.batch_tuning()

    cv = api.Convexifier(0)
    items, total = make(cv)
    ms, setup, st, tune = timed(cv, items)
    cv.close()
    # the default launch shape, through the cache file (the library's key:
    # energy and the set of (L, directions, depth))
    keys = sorted({f"{pr.L}.{pr.n_angle * pr.n_angle}.{pr.depth}" for pr in probs})
    with open(cache, "w") as f:
        f.write("{\n  \"e0_" + "_".join(keys) + "\": [8, 0]\n}\n")
    cv2 = api.Convexifier(0)
    items2, _ = make(cv2)
    ms_def, _, _, tune_def = timed(cv2, items2)
    cv2.close()
    os.remove(cache)
    flop = FLOP_PER_SAMPLE * st["valid_samples"]
    peak = fp32_peak_tflops(torch, dev)[0]
    line = {
        "metric": "quadrature points convexified/s (W^R+P), batched form",
        "value": total * a.steps / (ms / 1e3), "unit": "points/s", "n_gpus": 1,
        "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms / a.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32/f64",
        "data": "synthetic",
        "config": {"workload": (f"256 meshes, {total} points (log-uniform 1e3..1e5 per mesh), "
                                "stretch U[1.1, 1.8], 32^2 or 64^2 angles, L 513 or 1025, "
                                "depth 2 or 3, one captured CUDA graph per replay"),
                   "form": "batch"},
        "autotune": {"warps_per_cta": tune[0], "dirs_per_item_cap": tune[1],
                     "meaning": "warps 0 = lane-per-line scan", "setup_s": setup,
                     "default_shape_pts_per_s": total * a.steps / (ms_def / 1e3),
                     "default_shape": list(tune_def[:2]), "from_cache": tune_def[2],
                     "gain": ms_def / ms},
        "step_flop_rate": {"achieved": flop / (ms / 1e3) / 1e12, "peak": peak, "unit": "TFLOP/s",
                           "frac": flop / (ms / 1e3) / 1e12 / peak,
                           "note": "30 FLOP per valid sample over the whole replay (all kernels): "
                                   "a lower bound of the line scan's own rate"},
        "stats": st,
    }
    print(json.dumps(line), flush=True)


def run_material_points(a):
    """The full scan of material points at 16 x 16 angles, L = 201, depth 2
    (1,048,576 points by default) on its own: one JSON line."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    from paper_2211_14318_gb300 import api, inputs

    dev = torch.device("cuda:0")
    torch.cuda.set_device(0)
    cv = api.Convexifier(0)
    peak, sms, mhz, peak_src = fp32_peak_tflops(torch, dev)
    res = material_points_line(a, cv, api, inputs, torch, dev, peak, sms, mhz, peak_src, a.steps)
    res.update(metric="quadrature points convexified/s (W^R+P), full scan", n_gpus=1,
               warmup=2, higher_is_better=True, dtype="f32/f64", data="synthetic")
    print(json.dumps(res), flush=True)
    cv.close()


def main():
    a = args_parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.form == "loadpath":
        run_loadpath(a)
    elif a.form == "batch":
        run_batch(a)
    elif a.form == "points1m":
        run_material_points(a)
    elif a.form == "grid":
        run_grid(a)
    elif a.form == "surrogate":
        run_surrogate(a)
    elif a.form == "train":
        run_train(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
