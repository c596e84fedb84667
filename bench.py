"""Benchmark of one D2V16-FFT-TLB Runge-Kutta step (all four passes of both stages).

Workload: a static circular droplet (R = 128, tanh interface of width 2, Maxwell
coexistence densities at T = 0.85) on a 1024 x 1024 periodic grid, with the
phase-separation parameter set (tau = dt = 1e-4, dx = dy = 1/256, K = 5e-6, q = -0.004).
Synthetic, seeded inputs; the metric is MLUPS (lattice-node updates per second, one
update = one full two-stage step), headline = the FP32-spectral path (LBM_MIXED), with
the plain FP64 path measured beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Timing: W untimed steps, then K steps each between CUDA events on the library's stream,
with a 256 MiB buffer written between steps (outside the events) to flush the 126 MB L2;
then K more steps with per-launch events around every kernel, which give the per-kernel
durations of the roofline object. Under torchrun every rank runs its own replica (no
data-path collective: a single grid does not shard without an all-to-all); value = all
ranks' node updates / the slowest rank's time. One JSON line is printed by rank 0.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_GRID = 1024
WORKLOAD = "droplet R=128 on 1024x1024 periodic grid, T=0.85, phase-separation parameter set"
PARAMS = dict(tau=1e-4, dt=1e-4, dx=1.0 / 256, dy=1.0 / 256, K=5e-6, q=-0.004)
T0, RADIUS = 0.85, 128
# algorithmic bytes per node and launch, in units of the path's element size
# (col 34, macro 17, flux 8; update 61 in stage 1 and 77 in stage 2: mean 69)
ELEMS_PER_NODE = {"col": 34, "macro": 17, "flux": 8, "update": 69}
ELEMS_PER_NODE_STEP = 2 * (34 + 17 + 8) + 61 + 77  # 256
KERNEL_NAMES = {"col": "col_deriv_kernel", "macro": "macro_row_kernel", "flux": "col_deriv_kernel",
                "update": "update_row_kernel"}
FP64_PEAK_TFLOPS = 1.25  # GB300 nominal dense FP64 (no tensor path for this work)
# FP64 flops of one step of the FP64 path per node (DADD + DMUL + 2 DFMA thread instructions
# of its four kernels, counted by ncu at 1024^2: 5.35 GFLOP per step; the count does not
# depend on the launch shapes)
FP64_FLOP_PER_NODE_STEP = 5.353e9 / (1024 * 1024)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# the device code of the passes (kernels, FFT engine, shared layouts and launch limits); the
# host orchestration (lbm_api.cu, lbm_noalloc.cu) is not part of it, and the launch shapes a
# profile was taken with are checked separately
DEVICE_SOURCES = ("fft_reg.cuh", "kernels_batch.cu", "kernels_col.cu", "kernels_misc.cu", "kernels_row.cu",
                  "kernels_sf.cu", "lbm_internal.cuh", "pass_bodies.cuh", "tma.cuh")


def source_digest():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1403_3746_gb300", "csrc")
    for f in DEVICE_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


# launch shapes (column width, macro rows, update rows, flux width, column form, flux form,
# update CTAs per row) that each kernel's traffic depends on
SHAPES_OF = {"col": (0, 4), "macro": (1,), "flux": (3, 5), "update": (2, 6)}


def ncu_traffic(kernel_key, precision, shapes):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    device sources with the same launch shapes of that kernel."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            d = json.load(fh)
        e = d[f"{precision}:{kernel_key}"]
        cap = list(e.get("launch_shapes", []))
        if e.get("source_digest") != source_digest() or any(cap[i] != list(shapes)[i] for i in SHAPES_OF[kernel_key]):
            return None
        return e["dram_bytes_per_launch_full_size"]
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 50 ms while running; entering waits
    (up to 5 s) for the first sample, so the timed region that follows is covered."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None
        self.lines = []

    def _read(self):
        for line in self.p.stdout:
            self.lines.append(line)
            self.first.set()
        self.first.set()

    def __enter__(self):
        import threading
        self.first = threading.Event()
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None
            return self
        self.reader = threading.Thread(target=self._read, daemon=True)
        self.reader.start()
        self.first.wait(timeout=5)
        return self

    def __exit__(self, *exc):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()
            self.reader.join(timeout=5)
        self.out = "".join(self.lines)

    def summary(self):
        rows = []
        for line in (getattr(self, "out", "") or "").strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 9:
                try:
                    rows.append(f)
                except Exception:
                    pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def make_fields(lbm, synthetic, n=N_GRID, radius=RADIUS):
    rl, rv = lbm.maxwell(T0)
    return synthetic.droplet(n, n, radius, rl, rv, T0, width=2.0)


def time_path(lbm, torch, precision, steps, warmup, fields, stream, autotune=True):
    """Two timed loops of `steps` steps each on the same state, an L2 flush between steps.
    Loop A (the headline): lbm_step as the library runs it (one CUDA graph per step), one event
    pair around each step. Loop B: per-launch timing on (direct launches, an event pair around
    every kernel), which gives each kernel's mean duration for the roofline."""
    p = lbm.default_params(precision=precision, **PARAMS)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def loop(sim):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for a, b in ev:
            a.record(stream)
            sim.step(1)
            b.record(stream)
            flush.fill_(float(len(ev)))
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev], time.perf_counter() - t0

    with lbm.Simulation(N_GRID, N_GRID, p, stream=stream.cuda_stream) as sim:
        sim.init(*fields)
        geometry = sim.autotune()[0] if autotune else sim.geometry()  # launch shapes, before any timed step
        geometry = list(geometry) + list(sim.pass_kinds())  # + column, flux column kinds, update CTAs per row
        with torch.cuda.stream(stream):
            for _ in range(warmup):
                sim.step(1)
                flush.fill_(1.0)
            stream.synchronize()
            step_ms, wall = loop(sim)
            sim.timing(True)
            step_ms_b, _ = loop(sim)
        keys = list(ELEMS_PER_NODE) + (["rho64"] if precision == lbm.LBM_MIXED_RHO64 else [])
        kern = {k: sim.timing_read(k) for k in keys}
        sim.timing(False)
        diag = sim.diagnostics()
    return step_ms, kern, wall, diag, step_ms_b, geometry


def e2e_path(lbm, torch, precision, steps, fields):
    """Through the C ABI with host buffers: init from pinned host memory, every step lbm_step and
    a diagnostics request whose per-block partial sums come back to pinned host memory
    (lbm_diagnostics_begin: the request rides on the next step's first macro pass; the previous
    step's request is reduced with lbm_diagnostics_end while this step runs), and the final
    moments read back to pinned host memory."""
    p = lbm.default_params(precision=precision, **PARAMS)
    pinned = [torch.empty((N_GRID, N_GRID), dtype=torch.float64, pin_memory=True).numpy() for _ in range(8)]
    for dst, src in zip(pinned[:4], fields):
        dst[...] = src
    with lbm.Simulation(N_GRID, N_GRID, p) as sim:
        sim.init(*pinned[:4])
        sim.step(2)
        sim.synchronize()
        t0 = time.perf_counter()
        sim.init(*pinned[:4])
        diags = []
        for k in range(steps):
            sim.step(1)
            sim.diagnostics_begin()
            if k > 0:
                diags.append(sim.diagnostics_end())
        diags.append(sim.diagnostics_end())
        sim.moments(out=pinned[4:])
        wall = time.perf_counter() - t0
    n = N_GRID * N_GRID
    blocks = N_GRID  # the fused requests' partial sums: 5 per macro-pass CTA (one row each), and the error word
    assert len(diags) == steps and diags[-1]["steps"] == steps
    return {"value": n * steps / wall / 1e6, "unit": "MLUPS",
            "h2d_bytes_per_step": 4 * n * 8 / steps, "d2h_bytes_per_step": blocks * 5 * 8 + 4 + 4 * n * 8 / steps,
            "note": "init from pinned host + per step lbm_step and a diagnostics read (lbm_diagnostics_begin "
                    "/ _end; each request fused into the next step's macro pass) + final moments"}


BATCH_SIZES = [128] * 32 + [256] * 32 + [512] * 32
BATCH_WORKLOAD = ("96 independent spinodal quenches (32 each at 128^2, 256^2, 512^2), rho = 1 +/- 1% noise, "
                  "T_k uniform in [0.80, 0.95]")


def batch_path(lbm, torch, synthetic, precision, steps, warmup, stream, form=None):
    """The batched form: all instances advanced by one graph launch per step (form None: the
    graph of per-pass kernels; LBM_BATCH_PERSISTENT: one persistent kernel per step). The state
    (about 2.9 GB in LBM_MIXED) is far larger than L2, so no flush is needed between steps."""
    p = lbm.default_params(precision=precision, **PARAMS)
    temps = synthetic.quench_temperatures(4, len(BATCH_SIZES))
    nodes = sum(n * n for n in BATCH_SIZES)
    with lbm.Batch([(n, n) for n in BATCH_SIZES], p, stream=stream.cuda_stream) as b:
        for k, n in enumerate(BATCH_SIZES):
            b.init(k, *synthetic.spinodal(n, n, 1.0, 0.01, float(temps[k]), seed=4000 + k))
        if form is not None:
            b.set_form(form)
        b.autotune()  # launch shapes per size group (and the persistent kernel's CTA size), by measurement
        shapes = {f"{n}x{n}": list(b.geometry(BATCH_SIZES.index(n))) for n in sorted(set(BATCH_SIZES))}
        with torch.cuda.stream(stream):
            b.step(warmup)
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.step(steps)
            e1.record(stream)
            stream.synchronize()
        b.synchronize()
        ms = e0.elapsed_time(e1)
        ok = all(abs(b.diagnostics(k)["mass"]) > 0 for k in (0, len(BATCH_SIZES) - 1))
    out = {"value": nodes * steps / (ms * 1e-3) / 1e6, "unit": "MLUPS", "steps": steps,
           "ms_per_step": ms / steps, "nodes": nodes, "finite": ok}
    if form is None:
        out["launch_shapes"] = shapes
    return out


def batch_full_run(lbm, synthetic, steps=2000):
    """The batched workload over its whole quench (2000 steps, graph form, LBM_MIXED): every
    instance's mass drift and max |u| at the end, and whether every state stayed finite."""
    p = lbm.default_params(precision=lbm.LBM_MIXED, **PARAMS)
    temps = synthetic.quench_temperatures(4, len(BATCH_SIZES))
    t0 = time.perf_counter()
    with lbm.Batch([(n, n) for n in BATCH_SIZES], p) as b:
        for k, n in enumerate(BATCH_SIZES):
            b.init(k, *synthetic.spinodal(n, n, 1.0, 0.01, float(temps[k]), seed=4000 + k))
        d0 = [b.diagnostics(k) for k in range(len(BATCH_SIZES))]
        b.step(steps)
        b.synchronize()
        wall = time.perf_counter() - t0
        try:
            d1 = [b.diagnostics(k) for k in range(len(BATCH_SIZES))]
            finite = True
        except lbm.LbmError:  # a non-finite diagnostic
            d1, finite = d0, False
    drift = max(abs(a["mass"] / c["mass"] - 1) for a, c in zip(d1, d0))
    return {"steps": steps, "wall_s": wall, "finite": finite, "mass_drift_max": drift,
            "umax_max": max(a["umax"] for a in d1)}


LARGE_N = 4096
TALL_NX = 256  # width of the tall grid of `--profile tall`


def large_run(lbm, torch, synthetic, steps, stream):
    """The large single run: a 4096^2 spinodal quench (rho = 1 +/- 1%, T = 0.9, seed 5) in
    LBM_MIXED, timed over `steps` graph-launched steps (inputs far larger than L2), then the
    circularly averaged structure factor after those steps against the FP64 path from the
    same seed."""
    fields = synthetic.spinodal(LARGE_N, LARGE_N, 1.0, 0.01, 0.9, seed=5)
    n = LARGE_N * LARGE_N
    nbins = int(np.ceil(np.sqrt(2) * LARGE_N / 2)) + 2  # every shell of the box
    out = {"workload": f"spinodal quench {LARGE_N}x{LARGE_N}, rho = 1 +/- 1% (seed 5), T = 0.9", "steps": steps}
    S = {}
    for prec, name in ((lbm.LBM_MIXED, "mixed"), (lbm.LBM_FP64, "fp64")):
        p = lbm.default_params(precision=prec, **PARAMS)
        with lbm.Simulation(LARGE_N, LARGE_N, p, stream=stream.cuda_stream) as sim:
            sim.init(*fields)
            sim.autotune()
            with torch.cuda.stream(stream):
                sim.step(2)
                stream.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sim.step(steps)
                e1.record(stream)
                stream.synchronize()
            ms = e0.elapsed_time(e1) / steps
            S[name] = sim.structure_factor(nbins)[0]
            out[name] = {"value": n / (ms * 1e-3) / 1e6, "unit": "MLUPS", "ms_per_step": ms,
                         "launch_shapes": list(sim.geometry()) + list(sim.pass_kinds())}
    out["mixed"]["step_frac_of_hbm_roofline"] = (ELEMS_PER_NODE_STEP * 4 * n / (out["mixed"]["ms_per_step"] * 1e-3)
                                                 / 1e9 / peaks()[0])
    k = int(np.argmax(S["fp64"][1:])) + 1
    out["structure_factor"] = {"shells": nbins, "peak_shell_fp64": k,
                               "rel_l2_mixed_vs_fp64": float(np.linalg.norm(S["mixed"] - S["fp64"])
                                                             / np.linalg.norm(S["fp64"]))}
    return out


ORACLE_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, {root!r})
import numpy as np
import oracle, synthetic
from oracle.dvm import D2V16
from oracle.model import init_feq, rk2_step
n, steps, warm = {n}, {steps}, {warm}
rl, rv = oracle.coexistence({T0})
fields = synthetic.droplet(n, n, {radius}, rl, rv, {T0}, width=2.0)
p = oracle.Params(deriv={deriv!r}, **{params!r})
d = D2V16(p.eta0)
f = init_feq(d, *fields, p)
for _ in range(warm):
    f = rk2_step(d, f, p)
ts = []
for _ in range(steps):
    t = time.perf_counter(); f = rk2_step(d, f, p); ts.append(time.perf_counter() - t)
print(json.dumps({{"step_s": ts}}))
"""


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_oracle(n, steps, warm, radius, procs=1, deriv="fft", blas_threads=1):
    """The oracle as it stands, timed on the host: `procs` independent copies of the run, each
    its own interpreter (started by exec, no inherited CUDA state), run at the same time, each
    taking `steps` timed Runge-Kutta steps (or steps[j] in process j) after `warm` untimed ones. Returns (per-process
    lists of step times, wall time of the whole set)."""
    env = dict(os.environ, OMP_NUM_THREADS=str(blas_threads), OPENBLAS_NUM_THREADS=str(blas_threads),
               MKL_NUM_THREADS=str(blas_threads), CUDA_VISIBLE_DEVICES="")
    counts = list(steps) if isinstance(steps, (list, tuple)) else [steps] * procs
    codes = [ORACLE_SNIPPET.format(root=ROOT, n=n, steps=k, warm=warm, T0=T0, radius=radius, params=PARAMS,
                                   deriv=deriv) for k in counts]
    t0 = time.perf_counter()
    ps = [subprocess.Popen([sys.executable, "-c", code], stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True,
                           env=env) for code in codes]
    out = []
    for pr in ps:
        so, se = pr.communicate(timeout=1800)
        if pr.returncode != 0:
            raise RuntimeError("oracle run failed: " + se[-2000:])
        out.append(json.loads(so.strip().splitlines()[-1])["step_s"])
    return out, time.perf_counter() - t0


def oracle_mlups(n, per_proc):
    """Whole-set throughput: all processes' node updates over the longest process's timed span."""
    return n * n * sum(len(t) for t in per_proc) / max(sum(t) for t in per_proc) / 1e6


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(x, device):
    """The largest of every rank's x (the job time of replicas is the slowest rank's); x itself
    outside an initialised process group."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_mlups(nodes_per_rank, steps, world, job_ms):
    """All ranks' node updates over the job time, in millions per second."""
    return world * nodes_per_rank * steps / (job_ms * 1e-3) / 1e6


def reference_main(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    # the oracle on every host core: one copy of the 1024^2 droplet run per core, the K timed
    # Runge-Kutta steps shared out among them, each after one untimed step
    cores = host_cores()
    procs = max(1, min(cores, args.steps))
    share = [args.steps // procs + (1 if j < args.steps % procs else 0) for j in range(procs)]
    per, _ = run_oracle(N_GRID, share, min(args.warmup, 1), RADIUS, procs=procs)
    v = oracle_mlups(N_GRID, per)
    sample = (f"{args.steps} RK2 steps of the 1024x1024 droplet (R={RADIUS}) shared out over {procs} concurrent "
              f"oracle processes (numpy FP64, FFT derivatives, 1 thread each)")
    line = {"metric": "MLUPS of D2V16 RK2 step at 1024^2", "value": v, "unit": "MLUPS",
            "impl": "reference", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * max(sum(t) for t in per) / max(len(t) for t in per),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": "full 1024x1024 workload", "l2": "n/a (CPU)"},
            "cpu_baseline": {"value": v, "unit": "MLUPS", "cores": procs, "kind": "oracle", "sample": sample},
            "e2e": {"value": v, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def profile_main(args):
    """Launch sequences for ncu launch lists (the kernels and their order are fixed; nothing is
    timed here and no number printed by a run under ncu is a bench value)."""
    import torch
    import paper_1403_3746_gb300 as lbm
    from paper_1403_3746_gb300 import build as lbm_build
    import synthetic

    torch.cuda.set_device(0)
    if not os.path.exists(lbm_build.LIB):
        lbm_build.build()
    p = lbm.default_params(precision=lbm.LBM_MIXED, **PARAMS)
    if args.profile == "large":
        fields = synthetic.spinodal(LARGE_N, LARGE_N, 1.0, 0.01, 0.9, seed=5)
        with lbm.Simulation(LARGE_N, LARGE_N, p) as sim:
            sim.init(*fields)
            sim.step(1)
            sim.step(2)
            sim.synchronize()
            out = {"profile": "large", "n": LARGE_N, "steps": 3, "launch_shapes": list(sim.geometry()) + list(sim.pass_kinds())}
    elif args.profile in ("tall", "tall-tma1"):
        # 4096-point columns on a small grid (256 x 4096, about 0.3 GB): the column pass's
        # 4-column tiles at a size one ncu capture of a single launch covers quickly; "tall" in
        # the direct form, "tall-tma1" in the default one there (TMA, one staging buffer)
        fields = synthetic.spinodal(TALL_NX, LARGE_N, 1.0, 0.01, 0.9, seed=5)
        with lbm.Simulation(TALL_NX, LARGE_N, p) as sim:
            sim.init(*fields)
            if args.profile == "tall":
                sim.set_pass_kinds((lbm.LBM_COL_DIRECT, lbm.LBM_COL_DIRECT, 1))
            sim.step(1)
            sim.step(2)
            sim.synchronize()
            out = {"profile": args.profile, "nx": TALL_NX, "ny": LARGE_N, "steps": 3,
                   "launch_shapes": list(sim.geometry()) + list(sim.pass_kinds())}
    elif args.profile == "tma":
        fields = make_fields(lbm, synthetic)
        with lbm.Simulation(N_GRID, N_GRID, p) as sim:
            sim.init(*fields)
            sim.set_pass_kinds((lbm.LBM_COL_TMA, lbm.LBM_COL_TMA, 1))
            sim.step(1)
            sim.step(2)
            sim.synchronize()
            out = {"profile": "tma", "n": N_GRID, "steps": 3, "launch_shapes": list(sim.geometry()) + list(sim.pass_kinds())}
    else:
        fields = make_fields(lbm, synthetic)
        with lbm.Simulation(N_GRID, N_GRID, p) as sim:
            sim.init(*fields)
            sim.step(1)
            d = [sim.diagnostics() for _ in range(3)]
            out = {"profile": "diag", "n": N_GRID, "steps": 1, "diagnostics": 3, "mass": d[-1]["mass"]}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--fp64-steps", type=int, default=None)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the batched form and the error table")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes (for profiler runs, whose timing would mislead the tuner)")
    ap.add_argument("--profile", choices=["large", "diag", "tma", "tall", "tall-tma1"], default=None,
                    help="a fixed short launch sequence for ncu launch lists (default shapes, no timing): "
                         "large = 4096^2 mixed spinodal, init + 1 + 2 steps; diag = 1024^2 mixed droplet, "
                         "init + 1 step + 3 diagnostics requests; tma = the 1024^2 droplet with both column "
                         "passes in the TMA form (16-column tiles), init + 1 + 2 steps; tall = a 256 x 4096 "
                         "mixed spinodal (4096-point columns), direct column passes, init + 1 + 2 steps; "
                         "tall-tma1 = the same in the default column form there (TMA, one staging buffer)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_main(args)
    if args.profile:
        return profile_main(args)

    import torch
    import paper_1403_3746_gb300 as lbm
    from paper_1403_3746_gb300 import build as lbm_build
    import synthetic

    world, rank, local = dist_setup(args)
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if not os.path.exists(lbm_build.LIB):
        lbm_build.build()
    lbm.lib()
    dev = torch.cuda.current_device()
    stream = torch.cuda.Stream()
    fields = make_fields(lbm, synthetic)
    hbm, peak_kind = peaks()

    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(dev) as clk:
        step_ms, kern, wall, diag, step_ms_b, geom = time_path(lbm, torch, lbm.LBM_MIXED, args.steps, args.warmup,
                                                                fields, stream, not args.no_autotune)
    clocks = clk.summary()
    total_ms = max_over_ranks(sum(step_ms), "cuda")
    n = N_GRID * N_GRID
    value = whole_job_mlups(n, args.steps, world, total_ms)

    # FP64 path on the same workload (plain method)
    k64 = args.fp64_steps or max(3, args.steps // 10)
    step64, kern64, _, _, _, geom64 = time_path(lbm, torch, lbm.LBM_FP64, k64, min(args.warmup, 3), fields, stream,
                                                not args.no_autotune)
    fp64_mlups = n * k64 / (sum(step64) * 1e-3) / 1e6

    dom = max(kern, key=lambda k: kern[k][0])
    ms, cnt = kern[dom]
    per_launch_s = ms * 1e-3 / max(cnt, 1)
    alg_bytes = ELEMS_PER_NODE[dom] * 4 * n
    achieved = alg_bytes / per_launch_s / 1e9
    roofline = {"bound": "hbm", "kernel": KERNEL_NAMES[dom] + "<float>", "achieved": achieved, "peak": hbm,
                "unit": "GB/s", "frac": achieved / hbm, "traffic": ncu_traffic(dom, "mixed", geom),
                "peak_source": peak_kind, "alg_bytes_per_launch": alg_bytes,
                "duration_source": "mean CUDA-event time per launch in a second timed loop of the same steps "
                                   "with an event pair around every kernel",
                "step_frac": ELEMS_PER_NODE_STEP * 4 * n / (total_ms * 1e-3 / args.steps) / 1e9 / hbm}
    launches = sum(c for _, c in kern.values())  # loop B; loop A's graphs hold the same kernels per step
    e2e = e2e_path(lbm, torch, lbm.LBM_MIXED, max(200, args.steps), fields) if rank == 0 else None

    extras = {}
    if not args.no_extras:
        kb = max(5, args.steps // 10)
        extras["batched_form"] = {
            "workload": BATCH_WORKLOAD,
            "launch": "mixed / fp64: one CUDA graph per step, size groups as parallel branches; mixed_persistent: "
                      "one persistent kernel launch per step over a queue of (stage, pass, group, instance, tile)",
            "mixed": batch_path(lbm, torch, synthetic, lbm.LBM_MIXED, kb, 3, stream),
            "mixed_persistent": batch_path(lbm, torch, synthetic, lbm.LBM_MIXED, kb, 3, stream,
                                           lbm.LBM_BATCH_PERSISTENT),
            "fp64": batch_path(lbm, torch, synthetic, lbm.LBM_FP64, max(3, kb // 4), 3, stream),
            "whole_quench_mixed": batch_full_run(lbm, synthetic)}
        if rank == 0:
            from paper_1403_3746_gb300 import accuracy
            tab = accuracy.error_table(rho64=True)
            sl, dr = tab["slab"]["rows"], tab["droplet"]["rows"]
            extras["large_run"] = large_run(lbm, torch, synthetic, max(20, args.steps // 2), stream)
            lp = accuracy.laplace_check()
            extras["laplace_law"] = {
                "runs": f"mixed droplets R={[r['R'] for r in lp['rows']]} on 128^2 at T={lp['T']}, "
                        f"{lp['steps']} steps; sigma from a 256x2 slab",
                "sigma": lp["sigma"], "dp_R_over_sigma": {r["R"]: r["dp_R_over_sigma"] for r in lp["rows"]}}
            extras["accuracy_mixed_vs_fp64"] = {
                "coexistence_rel_err_max": max(max(r["rel_err_rho_l"], r["rel_err_rho_v"]) for r in sl),
                "mass_drift_mixed_max": max(abs(r["mass_drift_mixed"]) for r in sl + dr),
                "mass_drift_fp64_max": max(abs(r["mass_drift_fp64"]) for r in sl + dr),
                "spurious_velocity_rel_err_max": max(r["rel_err_umax"] for r in dr),
                "pressure_jump_rel_err_max": max(r["rel_err_dp"] for r in dr),
                "runs": f"slabs 256x2 at T={[r['T'] for r in sl]}, {tab['slab']['steps']} steps; droplets "
                        f"R={[r['R'] for r in dr]} on 128^2 at T=0.9, {tab['droplet']['steps']} steps",
                "rho64": {  # LBM_MIXED_RHO64 against float64, same runs
                    "coexistence_rel_err_max": max(max(r["rel_err_rho_l_rho64"], r["rel_err_rho_v_rho64"]) for r in sl),
                    "mass_drift_max": max(abs(r["mass_drift_rho64"]) for r in sl + dr),
                    "spurious_velocity_rel_err_max": max(r["rel_err_umax_rho64"] for r in dr),
                    "pressure_jump_rel_err_max": max(r["rel_err_dp_rho64"] for r in dr)}}
            # the same workload with the density chain in float64 (LBM_MIXED_RHO64)
            kr = max(5, args.steps // 4)
            step_r, kern_r, _, _, _, geom_r = time_path(lbm, torch, lbm.LBM_MIXED_RHO64, kr, 3, fields, stream,
                                                        not args.no_autotune)
            extras["rho64_path"] = {
                "value": n * kr / (sum(step_r) * 1e-3) / 1e6, "unit": "MLUPS", "steps": kr,
                "ms_per_step": sum(step_r) / kr, "launch_shapes": list(geom_r),
                "kernels_ms_per_step": {k: v[0] / kr for k, v in kern_r.items()},
                "note": "LBM_MIXED with rho as a float64 sum, its derivatives by float64 transforms and the "
                        "pressure and Lambda terms in float64; kernels_ms_per_step.rho64 is the float64 chain"}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cores = host_cores()
        per, _ = run_oracle(N_GRID, 1, 0, RADIUS, procs=cores)
        cpu = {"value": oracle_mlups(N_GRID, per), "unit": "MLUPS", "cores": cores, "kind": "oracle",
               "sample": f"1 RK2 step of the 1024x1024 droplet in each of {cores} concurrent oracle processes "
                         "(numpy FP64, FFT derivatives, 1 thread each)"}
        dft, _ = run_oracle(N_GRID, 1, 0, RADIUS, procs=1, deriv="dft", blas_threads=cores)
        cpu["direct_dft"] = {"value": oracle_mlups(N_GRID, dft), "unit": "MLUPS", "cores": cores,
                             "sample": "sampled: 1 RK2 step of the 1024x1024 droplet with the oracle's explicit-DFT "
                                       f"derivatives (dense N x N operators, BLAS on {cores} threads)"}
    if world > 1:
        dist.barrier()
    if rank == 0:
        line = {
            "metric": "MLUPS of D2V16 RK2 step at 1024^2", "value": value, "unit": "MLUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD,
                       "precision": "LBM_MIXED (f32 storage and arithmetic, f64 tables, exact fixed-quantum moment sums)",
                       "l2": "flushed between steps (256 MiB write)",
                       "launch": "lbm_step: one CUDA graph per step (8 kernels)",
                       "launch_shapes": {"col_tile_width": geom[0], "macro_rows_per_cta": geom[1],
                                         "update_rows_per_cta": geom[2], "flux_tile_width": geom[3],
                                         "col_kind": geom[4], "flux_kind": geom[5], "update_ctas_per_row": geom[6],
                                         "chosen_by": "defaults" if args.no_autotune else "lbm_autotune"},
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "fp64_path": {"value": fp64_mlups, "unit": "MLUPS", "steps": k64, "launch_shapes": list(geom64),
                          "ms_per_step": sum(step64) / k64,
                          "kernels_ms_per_step": {k: v[0] / k64 for k, v in kern64.items()},
                          "bound": "alu (fp64)", "fp64_peak_tflops_nominal": FP64_PEAK_TFLOPS,
                          "roofline": {"bound": "alu", "unit": "TFLOP/s", "peak": FP64_PEAK_TFLOPS,
                                       "peak_source": "nominal (GB300 FP64)",
                                       "achieved": FP64_FLOP_PER_NODE_STEP * n / (sum(step64) / k64 * 1e-3) / 1e12,
                                       "frac": FP64_FLOP_PER_NODE_STEP * n / (sum(step64) / k64 * 1e-3) / 1e12
                                               / FP64_PEAK_TFLOPS,
                                       "flop_source": "ncu FP64 thread-instruction counts per step (DFMA = 2)"}},
            "kernels_ms_per_step": {k: v[0] / args.steps for k, v in kern.items()},
            "roofline": roofline, "gpu_launches": launches, "e2e": e2e, "cpu_baseline": cpu,
            "ms_per_step_kernel_timed_loop": sum(step_ms_b) / args.steps,
            "clocks": clocks, "wall_s_timed_loop": wall,
            "check": {"mass": diag["mass"], "umax": diag["umax"]},
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
