#!/usr/bin/env python3
"""Benchmark of the PWL-VIE hot path on GB300.

Workload (one step = the whole hot path over one batch): the 64^3 head-size
ellipsoid phantom (4 nested shells + smoothed seeded noise, 3 mm voxels,
298 MHz), 16 right-hand sides from z-directed Hertzian dipoles on a 15 cm ring;
one step is a batched mixed-precision solve (FP32 FFT matvec and FP32 GMRES
inside FP64 iterative refinement) to a preconditioned relative residual of
1e-6 for all 16 right-hand sides, followed by the post-processing of the
solution (tested fields / PWL field coefficients and absorbed-power density).
`value` is right-hand sides solved per second over all ranks.

Also reported: the plain FP64 GPU solve of the same batch (solves/s and the
ratio), step latency p50/p99, the batched FP32 matvec's algorithmic HBM
throughput, the roofline of the dominant kernel (device time from CUDA events
recorded around every library launch on the launch stream), the end-to-end
figure through the C ABI with host buffers, and the FP64 CPU oracle on a
bounded sample.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 launch with torch.distributed.run; each rank solves its own batch
(independent replicas, weak scaling).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PWL-VIE matvec HBM GB/s & solves/s vs plain FP64 at 1e-6 residual; p99 latency"
WORKLOAD = ("head64: 64x64x64 head ellipsoid phantom (4 shells + smoothed noise, seed 1234), 3 mm voxels, "
            "298 MHz, 16 z-dipole RHS on a 15 cm ring; batched FP32 GMRES + FP64 refinement to 1e-6 "
            "preconditioned residual, then fields + SAR post-processing")
NRHS = 16
TOL = 1e-6
RESTART = 50
MAXIT = 30


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 comparison solve")
    ap.add_argument("--fp64-reps", type=int, default=3, help="plain FP64 solves timed (the median is reported)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the incl64 three-arm precision comparison attached to the default line")
    ap.add_argument("--serving", type=int, default=0, metavar="N",
                    help="serving stream: N requests (grids from --serving-sizes, 1-32 dipoles, 64/128/298 MHz), "
                         "first all at once (capacity), then as Poisson arrivals at 0.8x that capacity "
                         "(p50/p99 latency); prints one JSON line")
    ap.add_argument("--serving-sizes", default="32,48,64",
                    help="grid sizes n of the n^3 serving requests (the stream's full set is 32,48,64,96)")
    ap.add_argument("--serving-slots", type=int, default=4, help="requests in flight at once")
    ap.add_argument("--config-run", default="", metavar="NAME",
                    help="one mixed-precision and one plain FP64 solve of a named workload (body128: the "
                         "body-scale stack; incl64: the high-contrast inclusions), with iteration counts, "
                         "times and the mixed-vs-FP64 difference; prints one JSON line")
    ap.add_argument("--no-ref", action="store_true",
                    help="config-run: skip the FP64 reference solve at 1e-10 (the arms' errors are then not reported)")
    ap.add_argument("--tucker", default="", metavar="NAME",
                    help="Tucker compression of the Green tensors of a workload (head64, body128): time, ranks, "
                         "bytes, and the FP64 matvec / mixed solve with the compressed tensors")
    ap.add_argument("--jm", action="store_true",
                    help="full JM-VIE: a magnetodielectric sphere at 16^3-32^3 against the Mie series, FP64 solve time")
    ap.add_argument("--cufft-compare", action="store_true",
                    help="time a matvec built from torch.fft (cuFFT) and torch.einsum on the head64 sizes beside "
                         "vie_matvec (timing comparison only; its Green tensor is random data of the right shape)")
    ap.add_argument("--matvec-only", type=int, default=0, metavar="N",
                    help="profiling mode: set up the head64 workload and run N batched FP32 matvecs and one FP64 "
                         "matvec (16 RHS), print their timings; the solve benchmark is not run")
    ap.add_argument("--line-matvec", action="store_true",
                    help="profiling mode for the line-transform path: one warm-up and one timed FP32 matvec of 4 "
                         "random RHS on a 128 x 96 x 64 tissue grid (FFT 256 x 256 x 128, about 3 GB on the "
                         "device), per-kernel device times printed")
    return ap.parse_args()


def dist_init(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample (subprocess: fresh interpreter, no CUDA)
# ---------------------------------------------------------------------------
# Mean GMRES(50) iterations per right-hand side of the head64 batch to a 1e-6 preconditioned
# residual, measured once with the plain FP64 GPU solve of the same workload (the oracle runs the
# same GMRES(50) with the same preconditioner and stopping rule; its modified Gram-Schmidt differs
# from the GPU's classical one only in rounding).
HEAD64_ITERS_PER_RHS = 227.6

ORACLE_SAMPLE = r"""
import os, sys, time, json
sys.path.insert(0, {root!r})
import numpy as np
from synth import workload
from oracle import operator as O
w = workload("head64")
g = w["grid"]
prob = O.Problem(g, w["freq"], w["eps_real"], w["sigma"])
# Green setup excluded: the apply's arithmetic and memory traffic do not depend on the tensor
# values, so a seeded random table of the oracle's Toeplitz shape stands in for the 4.7 GB one
rng = np.random.Generator(np.random.PCG64(3))
shape = (12, 12, 2 * g.nz - 1, 2 * g.ny - 1, 2 * g.nx - 1)
T = rng.standard_normal(shape) + 1j * rng.standard_normal(shape)
t0 = time.perf_counter(); Nop = O.NOperator(g, prob.k0, T); t_setup = time.perf_counter() - t0
del T
x = rng.standard_normal((1, 12) + g.shape) + 1j * rng.standard_normal((1, 12) + g.shape)
times = []
for s in range({reps}):
    t0 = time.perf_counter()
    y = O.apply_PA(prob, Nop, x)
    times.append(time.perf_counter() - t0)
print(json.dumps(dict(times=times, setup_s=t_setup, workers=O.FFT_WORKERS, nv=g.nv)))
"""


def oracle_sample(reps):
    """The oracle's preconditioned FFT-Toeplitz matvec (P^-1 A x, NumPy + scipy.fft) of one right-hand
    side on the full 64^3 head64 grid, `reps` times; returns dict(times, setup_s, workers, nv)."""
    env = dict(os.environ)
    env["CUDA_VISIBLE_DEVICES"] = ""
    code = ORACLE_SAMPLE.format(root=ROOT, reps=reps)
    p = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if p.returncode != 0:
        raise RuntimeError("oracle sample failed: " + p.stderr[-2000:])
    return json.loads(p.stdout.strip().splitlines()[-1])


def oracle_solves_per_s(t_matvec_1rhs):
    """Oracle solves/s derived from its measured full-size matvec: one matvec per GMRES iteration,
    HEAD64_ITERS_PER_RHS iterations per right-hand side.  Its Gram-Schmidt, restarts and
    post-processing are left out, so this overstates the oracle's rate."""
    return 1.0 / (HEAD64_ITERS_PER_RHS * t_matvec_1rhs)


def oracle_sample_text(t, s, n):
    return (f"oracle P^-1 A x matvec (NumPy, scipy.fft with {s['workers']} workers) of one right-hand side on "
            f"the full 64^3 head64 grid: median {t:.2f} s over {n} timed runs; solves/s = 1 / "
            f"({HEAD64_ITERS_PER_RHS:.0f} GMRES iterations per right-hand side x that time), Gram-Schmidt left "
            f"out; Green setup excluded (seeded random table of the Toeplitz shape, {s['setup_s']:.1f} s)")


def cpu_baseline_block(reps=5):
    s = oracle_sample(reps=reps + 1)
    t = statistics.median(s["times"][1:])
    return dict(value=oracle_solves_per_s(t), unit="solves/s", cores=s["workers"], kind="oracle",
                sample=oracle_sample_text(t, s, reps), sample_seconds=sum(s["times"]))


# ---------------------------------------------------------------------------
# Reference arm: the oracle, as it stands
# ---------------------------------------------------------------------------
def run_reference(args, ws, rank):
    if rank != 0:
        return
    s = oracle_sample(reps=args.warmup + args.steps)
    times = s["times"][args.warmup:]
    t = statistics.median(times)
    value = oracle_solves_per_s(t)
    line = dict(
        impl="reference", metric=METRIC, value=value, unit="solves/s", n_gpus=args.gpus, steps=args.steps,
        warmup=args.warmup, ms_per_step=1000.0 * sum(times) / len(times), higher_is_better=True, scaling="weak",
        vs_baseline=None, dtype="f64", data="synthetic",
        config=dict(workload=WORKLOAD, nrhs=NRHS, tol=TOL, restart=RESTART,
                    step="one oracle matvec of one right-hand side at 64^3 (bounded sample)"),
        cpu_baseline=dict(value=value, unit="solves/s", cores=s["workers"], kind="oracle",
                          sample=oracle_sample_text(t, s, len(times))),
        e2e=dict(value=value, unit="solves/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0),
    )
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# Clock sampling during the timed region
# ---------------------------------------------------------------------------
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return dict(sm_mhz=None, sm_max_mhz=None, reasons=["nvidia-smi unavailable"])
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return dict(sm_mhz=statistics.median(sm) if sm else None, sm_max_mhz=smax, reasons=sorted(reasons),
                    samples=len(sm))


# ---------------------------------------------------------------------------
# Algorithmic bytes / flops per launch of the matvec kernels (FP32: c = 8 bytes, FP64: c = 16)
# ---------------------------------------------------------------------------
def kernel_model(name, grid, L, R):
    nx, ny, nz = grid
    Lx, Ly, Lz = L
    Ox, Oy, Oz = Lx // 2 + 1, Ly // 2 + 1, Lz // 2 + 1
    c = 16 if name.endswith("f64") else 8
    C = 12 * R
    nv = nx * ny * nz
    lg = math.log2
    if name.startswith("fft_x"):
        return C * nv * c + C * nz * ny * Lx * c, 5.0 * Lx * lg(Lx) * C * nz * ny
    if name.startswith("fft_y"):
        return C * nz * ny * Lx * c + C * nz * Ly * Lx * c, 5.0 * Ly * lg(Ly) * C * nz * Lx
    if name.startswith("zpass_block"):
        b = 2 * C * nz * Ly * Lx * c + 60 * Ox * Oy * Oz * c
        f = 2 * 5.0 * Lz * lg(Lz) * C * Lx * Ly + 144 * 8.0 * R * Lx * Ly * Lz
        return b, f
    if name.startswith("ifft_y"):
        return C * nz * Ly * Lx * c + C * nz * ny * Lx * c, 5.0 * Ly * lg(Ly) * C * nz * Lx
    if name.startswith("ifft_x_epilogue"):
        return C * nz * ny * Lx * c + 2 * C * nv * c + 2 * nv * c, 5.0 * Lx * lg(Lx) * C * nz * ny
    return None, None


def matvec_alg_bytes(grid, L, R, c):
    """Three-sweep lower bound of one batched matvec: x read, the half-padded spectrum (Nz planes of
    Ly x Lx per component) written after the forward xy transforms, read and written by the z pass,
    read by the inverse xy pass, x re-read and y written by the epilogue, and the Green octant read
    once: 3 C N_V c + 4 C Nz Ly Lx c + 60 Ox Oy Oz c."""
    nx, ny, nz = grid
    Lx, Ly, Lz = L
    C = 12 * R
    spec = C * nz * Ly * Lx * c
    return C * nx * ny * nz * c * 3 + 4 * spec + 60 * (Lx // 2 + 1) * (Ly // 2 + 1) * (Lz // 2 + 1) * c


def source_hash(files):
    """Hash of the kernel sources a recorded ncu measurement was taken on (paths relative to csrc/)."""
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1902_02196_gb300", "csrc")
    for f in sorted(files):
        p = os.path.join(d, f)
        if not os.path.exists(p):
            return None
        h.update(f.encode())
        h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary (profiles/traffic.json), when it was taken
    on the current sources of that kernel; else None."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
    except ValueError:
        return None
    e = d.get(kernel)
    if not e or e.get("source_hash") != source_hash(e.get("sources", [])):
        return None
    return e.get("dram_bytes_per_launch")


def max_over_ranks(x, device=None):
    """Largest value of x over the ranks of the default process group (x itself without one)."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world_size, max_seconds):
    """Whole-job throughput: the units all ranks processed over the slowest rank's time."""
    return units_per_rank * world_size / max_seconds


def fp32_clock_mhz():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)).get("sm_max_mhz", 2070.0)
    return 2070.0


def scaled_traffic(kernel, grid, L, bytes_per_launch):
    """The recorded ncu traffic (taken on launches of all NRHS right-hand sides) scaled to a launch
    with the given algorithmic bytes, i.e. to the right-hand sides the timed launches transformed."""
    t = measured_traffic(kernel)
    full, _ = kernel_model(kernel, grid, L, NRHS)
    if t is None or not full:
        return t
    return t * bytes_per_launch / full


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# Our arm
# ---------------------------------------------------------------------------
def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    import paper_1902_02196_gb300 as vie
    from synth import workload

    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    vie.build()
    w = workload("head64")
    g = w["grid"]
    grid = (g.nx, g.ny, g.nz)
    t0 = time.perf_counter()
    h = vie.vie_setup((g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), w["freq"], w["eps_real"], w["sigma"])
    setup_s = time.perf_counter() - t0
    L, _ = vie.vie_info(h)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    shape = (NRHS, 12) + g.shape
    e_inc = torch.empty(shape, dtype=torch.complex128, device=dev)
    b = torch.empty_like(e_inc)
    vie.vie_rhs_dipoles(h, w["dip_pos"], w["dip_mom"], e_inc, b, stream=stream)
    x = torch.empty_like(b)
    e_coeff = torch.empty_like(b)
    p_abs = torch.empty((NRHS,) + g.shape, dtype=torch.float64, device=dev)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    def step(mode=vie.VIE_SOLVE_FP32_REFINE):
        rc, info = vie.vie_solve(h, b, x, tol=TOL, restart=RESTART, maxit=MAXIT, mode=mode, stream=stream)
        P = vie.vie_fields(h, x, e_inc, e_coeff, p_abs, stream=stream)
        return rc, info, P

    def run_e2e():
        """The same step through the C ABI with the inputs (b, e_inc) in pinned host memory and the
        results (field map, SAR map, P_abs) read back into pinned host memory, copies inside the
        timed region; the current coefficients x stay on the device between the two calls, as the
        intermediate they are."""
        bh = b.cpu().pin_memory()
        eh = e_inc.cpu().pin_memory()
        xd = torch.empty_like(b)
        ph = torch.empty((NRHS,) + g.shape, dtype=torch.float64).pin_memory()
        ech = torch.empty(shape, dtype=torch.complex128).pin_memory()
        split = [0.0, 0.0]

        def step_host():
            # vie_solve returns with x on the device; vie_fields returns after its device-to-host
            # copies (host buffers synchronize the stream)
            t0 = time.perf_counter()
            vie.vie_solve(h, bh, xd, tol=TOL, restart=RESTART, maxit=MAXIT, mode=vie.VIE_SOLVE_FP32_REFINE,
                          stream=stream)
            t1 = time.perf_counter()
            P = vie.vie_fields(h, xd, eh, ech, ph, stream=stream)
            split[0] += t1 - t0
            split[1] += time.perf_counter() - t1
            return P

        step_host()
        ke = max(1, min(3, args.steps))
        barrier()
        torch.cuda.synchronize()
        split[:] = [0.0, 0.0]
        t0 = time.perf_counter()
        for _ in range(ke):
            step_host()
        torch.cuda.synchronize()
        te = max_over_ranks((time.perf_counter() - t0) / ke, dev)
        vb = NRHS * 12 * g.nv * 16
        return dict(value=job_throughput(NRHS, ws, te), unit="solves/s", h2d_bytes_per_step=2 * vb,
                    d2h_bytes_per_step=vb + NRHS * g.nv * 8 + NRHS * 8,
                    solve_ms=1e3 * split[0] / ke, fields_ms=1e3 * split[1] / ke,
                    note="C ABI with pinned host buffers: b and e_inc in, field map, p_abs and P_abs out "
                         "(x stays on the device between vie_solve and vie_fields); slowest rank")

    for _ in range(max(3, args.warmup)):
        rc, info, P = step()
    barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    launches_before, _ = vie.vie_stats_read()  # setup and warm-up launches (the ncu window's offset)
    vie.vie_stats_reset(True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    infos = []
    barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    for i in range(args.steps):
        evs[i][0].record(stream)
        rc, info, P = step()
        evs[i][1].record(stream)
        infos.append((rc, info, P))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    barrier()
    clk = clocks.stop()
    total_launches, kstats = vie.vie_stats_read()
    vie.vie_stats_reset(False)
    step_ms = [a.elapsed_time(bb) for a, bb in evs]
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, dev)
    value = job_throughput(NRHS * args.steps, ws, total_ms / 1000.0)
    rcs = [r for r, _, _ in infos]
    last_info = infos[-1][1]
    e2e = None if args.no_e2e else run_e2e()  # every rank, like the timed steps
    if rank != 0:
        if ws > 1:
            torch.distributed.barrier()
        return

    # dominant kernel over the timed region (device time from events around every library launch)
    dname, (dl, dms, dbytes) = max(kstats.items(), key=lambda kv: kv[1][1])
    hbm_peak, peak_kind = peaks()
    avg_s = dms / dl / 1000.0
    if dname.endswith("f64"):
        b0, _ = kernel_model(dname, grid, L, 0)
        b1, f1 = kernel_model(dname, grid, L, 1)
        flops_pl = f1 * (dbytes / dl - b0) / (b1 - b0) if f1 else None
        fp64_peak = 1250.0  # GFLOP/s, nominal GB300 FP64 rate
        achieved = flops_pl / avg_s / 1e9 if flops_pl else None
        roofline = dict(bound="alu", kernel=dname, achieved=achieved, peak=fp64_peak, unit="GFLOP/s",
                        frac=achieved / fp64_peak if achieved else None, traffic=scaled_traffic(dname, grid, L, dbytes / dl),
                        peak_kind="nominal FP64", launches=dl, avg_ms=1000 * avg_s)
    else:
        achieved = dbytes / (dms / 1000.0) / 1e9
        roofline = dict(bound="hbm", kernel=dname, achieved=achieved, peak=hbm_peak, unit="GB/s",
                        frac=achieved / hbm_peak, traffic=scaled_traffic(dname, grid, L, dbytes / dl), peak_kind=peak_kind,
                        launches=dl, avg_ms=1000 * avg_s, alg_bytes_per_launch=dbytes / dl)
        # right-hand sides a launch actually transformed (the solver skips converged ones), from the
        # library's per-launch algorithmic bytes, which are affine in that count; flops are linear in it
        b0, _ = kernel_model(dname, grid, L, 0)
        b1, f1 = kernel_model(dname, grid, L, 1)
        flops_pl = f1 * (dbytes / dl - b0) / (b1 - b0) if f1 else None
        if flops_pl:
            # FP32 CUDA-core peak from unit counts and clock: SMs x 128 FP32 lanes x 2 flops x max SM clock
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            alu_peak = sms * 128 * 2 * fp32_clock_mhz() * 1e6 / 1e9
            if flops_pl / alu_peak > (dbytes / dl) / hbm_peak:  # the ALU time floor is the larger one
                alu = flops_pl / avg_s / 1e9
                roofline = dict(bound="alu", kernel=dname, achieved=alu, peak=alu_peak, unit="GFLOP/s",
                                frac=alu / alu_peak, traffic=scaled_traffic(dname, grid, L, dbytes / dl),
                                peak_kind=f"FP32 FMA: {sms} SMs x 128 lanes x 2 x max SM clock",
                                launches=dl, avg_ms=1000 * avg_s, alg_flops_per_launch=flops_pl,
                                rhs_per_launch=(dbytes / dl - b0) / (b1 - b0),
                                alg_bytes_per_launch=dbytes / dl, hbm_achieved=achieved,
                                hbm_frac=achieved / hbm_peak, hbm_peak=hbm_peak, hbm_peak_kind=peak_kind)
    tot_ms = sum(v[1] for v in kstats.values())
    share = {k: dict(share=round(v[1] / max(1e-9, tot_ms), 4), launches=v[0], ms=round(v[1], 3),
                     gbs=round(v[2] / (v[1] / 1000.0) / 1e9, 1) if v[1] > 0 and v[2] > 0 else None)
             for k, v in sorted(kstats.items(), key=lambda kv: -kv[1][1])[:10]}

    # batched FP32 matvec throughput (events on the launch stream)
    g32 = torch.Generator(device=dev)
    g32.manual_seed(5)
    x32 = torch.randn(shape, dtype=torch.complex64, device=dev, generator=g32)
    y32 = torch.empty_like(x32)
    for _ in range(3):
        vie.vie_matvec(h, x32, y32, vie.VIE_FP32, vie.VIE_OP_PA, stream=stream)
    nmv = 20
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(nmv):
        vie.vie_matvec(h, x32, y32, vie.VIE_FP32, vie.VIE_OP_PA, stream=stream)
    a1.record(stream)
    torch.cuda.synchronize()
    mv_ms = a0.elapsed_time(a1) / nmv
    mv_bytes = matvec_alg_bytes(grid, L, NRHS, 8)
    a0.record(stream)
    for _ in range(nmv):
        vie.vie_matvec(h, x32, y32, vie.VIE_BF16X3, vie.VIE_OP_PA, stream=stream)
    a1.record(stream)
    torch.cuda.synchronize()
    mv16_ms = a0.elapsed_time(a1) / nmv
    x64 = x32.to(torch.complex128)
    y64 = torch.empty_like(x64)
    vie.vie_matvec(h, x64, y64, vie.VIE_FP64, vie.VIE_OP_PA, stream=stream)
    a0.record(stream)
    vie.vie_matvec(h, x64, y64, vie.VIE_FP64, vie.VIE_OP_PA, stream=stream)
    a1.record(stream)
    torch.cuda.synchronize()
    mv64_ms = a0.elapsed_time(a1)
    del x32, y32, x64, y64

    out = dict(
        metric=METRIC, value=value, unit="solves/s", n_gpus=ws, steps=args.steps, warmup=args.warmup,
        ms_per_step=total_ms / args.steps, higher_is_better=True, scaling="weak", vs_baseline=None,
        dtype="f32/f64", data="synthetic",
        config=dict(workload=WORKLOAD, nrhs=NRHS, grid=list(grid), fft=list(L), tol=TOL, restart=RESTART,
                    l2="inputs larger than L2 (16-RHS batch: 805 MB per vector)", parallelism=f"replicas x{ws}"),
        latency_ms=dict(p50=statistics.median(step_ms), p99=float(np.percentile(step_ms, 99)),
                        max=max(step_ms)),
        solve=dict(rc=rcs[-1], iterations=[i["iterations"] for i in last_info][:4],
                   refinements=last_info[0]["refinements"], fp64_matvecs=last_info[0]["fp64_matvecs"],
                   max_resid=max(i["resid"] for i in last_info), converged=all(i["converged"] for i in last_info),
                   max_err_est=max(i["err_est"] for i in last_info)),
        matvec=dict(fp32_ms=mv_ms, fp32_alg_gbs=mv_bytes / (mv_ms / 1000) / 1e9,
                    fp32_frac_of_hbm=mv_bytes / (mv_ms / 1000) / 1e9 / hbm_peak, fp64_ms=mv64_ms,
                    bf16x3_ms=mv16_ms,
                    alg_bytes=mv_bytes),
        roofline=roofline, kernels=share, gpu_launches=total_launches, launches_before_timed=launches_before,
        autotune=vie.vie_tuning(), cycle_graphs=True,
        setup_s=setup_s, clocks=clk,
        wall_s=wall,
    )

    if not args.no_fp64:
        t64s = []
        for _ in range(max(1, args.fp64_reps)):
            torch.cuda.synchronize()
            f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            f0.record(stream)
            rc64, info64, _ = step(vie.VIE_SOLVE_FP64)
            f1.record(stream)
            torch.cuda.synchronize()
            t64s.append(f0.elapsed_time(f1) / 1000.0)
        t64 = statistics.median(t64s)
        it64 = [i["iterations"] for i in info64]
        out["fp64"] = dict(value=NRHS / t64, unit="solves/s", seconds=t64, seconds_all=t64s, rc=rc64,
                           iterations=it64, mean_iterations=sum(it64) / len(it64),
                           max_resid=max(i["resid"] for i in info64))
        out["speedup_vs_fp64"] = value / (NRHS * ws / t64)

    if e2e is not None:
        out["e2e"] = e2e
    if not args.no_configs and ws == 1:
        # the high-contrast precision stress (64^3 inclusions, 32 RHS, 447 MHz): BF16x3 vs FP32 vs
        # FP64 arms, iterations and the solvers' forward-error estimates (errors against an FP64
        # solve to 1e-10: --config-run incl64)
        torch.cuda.synchronize()
        out["configs"] = {"incl64": config_measure("incl64", local, no_fp64=args.no_fp64, no_ref=True)}
        torch.cuda.set_stream(stream)
    if not args.no_cpu and ws == 1:
        try:
            out["cpu_baseline"] = cpu_baseline_block()
        except Exception as ex:  # the CPU leg is informative only
            out["cpu_baseline"] = dict(value=None, unit="solves/s", cores=1, kind="oracle", sample=str(ex)[:200])
    print(json.dumps(out), flush=True)
    h.close()
    if ws > 1:
        torch.distributed.barrier()


def run_matvec_only(args, local):
    """Small, bounded command for kernel profiling: N FP32 matvecs + 1 FP64 matvec on head64, 16 RHS."""
    import torch

    import paper_1902_02196_gb300 as vie
    from synth import workload

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    vie.build()
    w = workload("head64")
    g = w["grid"]
    h = vie.vie_setup((g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), w["freq"], w["eps_real"], w["sigma"])
    L, _ = vie.vie_info(h)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    shape = (NRHS, 12) + g.shape
    gen = torch.Generator(device=dev)
    gen.manual_seed(5)
    x = torch.randn(shape, dtype=torch.complex64, device=dev, generator=gen)
    y = torch.empty_like(x)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    vie.vie_stats_reset(1)
    for _ in range(args.matvec_only):
        a0.record(stream)
        vie.vie_matvec(h, x, y, vie.VIE_FP32, vie.VIE_OP_PA, stream=stream)
        a1.record(stream)
        torch.cuda.synchronize()
        times.append(a0.elapsed_time(a1))
    times16 = []
    for _ in range(args.matvec_only):
        a0.record(stream)
        vie.vie_matvec(h, x, y, vie.VIE_BF16X3, vie.VIE_OP_PA, stream=stream)
        a1.record(stream)
        torch.cuda.synchronize()
        times16.append(a0.elapsed_time(a1))
    kernels = {k: [v[0], round(v[1] / max(v[0], 1), 4), round(v[2] / max(v[1], 1e-9) / 1e6, 1)]
               for k, v in vie.vie_stats_read()[1].items()}
    vie.vie_stats_reset(0)
    x64 = x.to(torch.complex128)
    y64 = torch.empty_like(x64)
    a0.record(stream)
    vie.vie_matvec(h, x64, y64, vie.VIE_FP64, vie.VIE_OP_PA, stream=stream)
    a1.record(stream)
    torch.cuda.synchronize()
    b = matvec_alg_bytes((g.nx, g.ny, g.nz), L, NRHS, 8)
    print(json.dumps(dict(mode="matvec-only", workload="head64, 16 RHS", fp32_ms=times, bf16x3_ms=times16,
                          fp32_alg_gbs=b / (min(times) / 1000) / 1e9, fp64_ms=a0.elapsed_time(a1),
                          kernels_launches_ms_gbs=kernels)), flush=True)
    h.close()


def run_serving(args, local):
    """Request loop (vie_submit / vie_poll) on a stream of head-phantom solves."""
    import numpy as np
    import torch

    import paper_1902_02196_gb300 as vie
    from synth import serving_stream

    torch.cuda.set_device(local)
    vie.build()
    sizes = tuple(int(v) for v in args.serving_sizes.split(","))
    reqs = serving_stream(args.serving, seed=77, sizes=sizes)

    def submit(srv, r):
        g = r["grid"]
        return srv.submit((g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), r["freq"], r["eps_real"], r["sigma"], r["dip_pos"],
                          r["dip_mom"], tol=TOL, restart=RESTART, maxit=MAXIT, mode=vie.VIE_SOLVE_FP32_REFINE)

    def collect(srv, pending, t0, done):
        while pending:
            for t in list(pending):
                res = srv.poll(t, timeout_us=2000)
                if res is not None:
                    done.append((pending.pop(t), res, time.perf_counter() - t0))

    # warm-up: one small request (library load, kernel attributes)
    srv = vie.Server(max_concurrent=args.serving_slots)
    w = serving_stream(1, seed=5, sizes=(32,))[0]
    w["dip_pos"], w["dip_mom"] = w["dip_pos"][:1], w["dip_mom"][:1]
    collect(srv, {submit(srv, w): -1}, time.perf_counter(), [])
    srv.close()
    # closed loop: everything submitted at once, on a fresh loop (cold Green cache)
    srv = vie.Server(max_concurrent=args.serving_slots)
    t0 = time.perf_counter()
    pending = {submit(srv, r): i for i, r in enumerate(reqs)}
    closed = []
    collect(srv, pending, t0, closed)
    span = max(c[2] for c in closed)
    srv.close()
    cap = len(reqs) / span
    # open loop: Poisson arrivals at 0.8 x the measured capacity, fresh loop
    lam = 0.8 * cap
    srv = vie.Server(max_concurrent=args.serving_slots)
    t0 = time.perf_counter()
    pending, opened, sub_t, tnext = {}, [], {}, 0.0
    for i, r in enumerate(reqs):
        tnext += r["gap"] / lam
        while time.perf_counter() - t0 < tnext:
            for t in list(pending):
                res = srv.poll(t, timeout_us=0)
                if res is not None:
                    opened.append((pending.pop(t), res, time.perf_counter() - t0))
            time.sleep(0.001)
        t = submit(srv, r)
        pending[t] = i
        sub_t[i] = time.perf_counter() - t0
    collect(srv, pending, t0, opened)
    span_o = max(c[2] for c in opened)
    srv.close()
    lat = np.array([c[1]["queued_s"] + c[1]["run_s"] for c in opened]) * 1000.0

    def concurrency(done):
        """Requests on the device at once, from their device spans: time average over the busy
        span and maximum."""
        ev = sorted([(c[1]["dev_start_s"], 1) for c in done] + [(c[1]["dev_end_s"], -1) for c in done])
        busy, area, cur, peak, last = 0.0, 0.0, 0, 0, None
        for t, d in ev:
            if last is not None and cur > 0:
                busy += t - last
                area += cur * (t - last)
            cur += d
            peak = max(peak, cur)
            last = t
        return dict(mean=area / busy if busy > 0 else 0.0, max=peak)
    rhs = sum(int(r["dip_pos"].shape[0]) for r in reqs)
    status = [c[1]["status"] for c in closed + opened]
    line = dict(mode="serving", metric="serving stream: solves/s and p50/p99 request latency", unit="solves/s",
                requests=len(reqs), right_hand_sides=rhs, slots=args.serving_slots,
                sizes=list(sizes), freqs_mhz=[64, 128, 298], tol=TOL, data="synthetic",
                closed_loop=dict(seconds=span, requests_per_s=cap, solves_per_s=rhs / span,
                                 green_cache_hits=sum(c[1]["green_cached"] for c in closed),
                                 device_concurrency=concurrency(closed)),
                open_loop=dict(arrival_rate_per_s=lam, seconds=span_o, solves_per_s=rhs / span_o,
                               latency_ms=dict(p50=float(np.percentile(lat, 50)), p99=float(np.percentile(lat, 99)),
                                               max=float(lat.max())),
                               green_cache_hits=sum(c[1]["green_cached"] for c in opened),
                               device_concurrency=concurrency(opened)),
                all_ok=all(s in (vie.VIE_OK,) for s in status),
                max_iterations=max(c[1]["iterations"] for c in closed + opened))
    print(json.dumps(line), flush=True)


def run_config(args, local):
    """Mixed vs plain FP64 on one named workload (precision stress / body scale)."""
    import torch

    torch.cuda.set_device(local)
    print(json.dumps(config_measure(args.config_run, local, args.no_fp64, args.no_ref)), flush=True)


def config_measure(name, local, no_fp64=False, no_ref=False):
    """The arms BF16x3, FP32 (+ FP64 refinement) and plain FP64 on one named workload, with
    iterations, times, the solvers' error estimates and, unless no_ref, the error against an FP64
    solve to 1e-10; returns the result as a dict."""
    import numpy as np
    import torch

    import paper_1902_02196_gb300 as vie
    from synth import workload

    dev = torch.device("cuda", local)
    vie.build()
    w = workload(name)
    g = w["grid"]
    R = int(w["dip_pos"].shape[0])
    t0 = time.perf_counter()
    h = vie.vie_setup((g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), w["freq"], w["eps_real"], w["sigma"])
    setup_s = time.perf_counter() - t0
    L, _ = vie.vie_info(h)
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    shape = (R, 12) + g.shape
    e_inc = torch.empty(shape, dtype=torch.complex128, device=dev)
    b = torch.empty_like(e_inc)
    vie.vie_rhs_dipoles(h, w["dip_pos"], w["dip_mom"], e_inc, b, stream=stream)
    out = dict(mode="config-run", workload=name, grid=[g.nx, g.ny, g.nz], fft=list(L), nrhs=R,
               freq_mhz=w["freq"] / 1e6, tol=TOL, restart=RESTART, setup_s=setup_s, data="synthetic")
    sol = {}
    arms = [("bf16x3", vie.VIE_SOLVE_BF16X3_REFINE, TOL), ("mixed", vie.VIE_SOLVE_FP32_REFINE, TOL)]
    if not no_fp64:
        # the plain FP64 arm, and the same method to 1e-10 as the reference the arms' errors are taken
        # against (the FP64 path is parity-pinned to the oracle; the oracle itself cannot solve this size)
        arms += [("fp64", vie.VIE_SOLVE_FP64, TOL)]
        if not no_ref:
            arms += [("fp64_ref", vie.VIE_SOLVE_FP64, 1e-10)]
    for name, mode, tol in arms:
        x = torch.empty_like(b)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        rc, info = vie.vie_solve(h, b, x, tol=tol, restart=RESTART, maxit=400, mode=mode, stream=stream)
        a1.record(stream)
        torch.cuda.synchronize()
        pa = torch.empty((R,) + g.shape, dtype=torch.float64, device=dev)
        P = vie.vie_fields(h, x, e_inc, None, pa, stream=stream)
        sec = a0.elapsed_time(a1) / 1000.0
        sol[name] = (x, np.asarray(P))
        its = [i["iterations"] for i in info]
        out[name] = dict(rc=rc, tol=tol, seconds=sec, solves_per_s=R / sec, iterations_max=max(its),
                         iterations_mean=sum(its) / len(its), refinements=info[0]["refinements"],
                         fp64_matvecs=info[0]["fp64_matvecs"], inner_matvecs=info[0]["fp32_matvecs"],
                         max_resid=max(i["resid"] for i in info), max_err_est=max(i["err_est"] for i in info))
    if "fp64" in sol:
        out["speedup_vs_fp64"] = {k: out["fp64"]["seconds"] / out[k]["seconds"] for k in ("bf16x3", "mixed")}
    if "fp64_ref" in sol:
        xr, Pr = sol["fp64_ref"]
        for name in ("bf16x3", "mixed", "fp64"):
            xm, Pm = sol[name]
            out[name]["x_rel_vs_ref"] = float(torch.linalg.vector_norm(xm - xr) / torch.linalg.vector_norm(xr))
            out[name]["P_abs_rel_max_vs_ref"] = float(np.max(np.abs(Pm - Pr) / np.abs(Pr)))
    x32 = torch.randn(shape, dtype=torch.complex64, device=dev)
    y32 = torch.empty_like(x32)
    for _ in range(2):
        vie.vie_matvec(h, x32, y32, vie.VIE_FP32, vie.VIE_OP_PA, stream=stream)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    for _ in range(5):
        vie.vie_matvec(h, x32, y32, vie.VIE_FP32, vie.VIE_OP_PA, stream=stream)
    a1.record(stream)
    torch.cuda.synchronize()
    mv = a0.elapsed_time(a1) / 5
    mvb = matvec_alg_bytes((g.nx, g.ny, g.nz), L, R, 8)
    out["matvec_fp32"] = dict(ms=mv, alg_gbs=mvb / (mv / 1000) / 1e9)
    if L[2] <= 512:
        for _ in range(2):
            vie.vie_matvec(h, x32, y32, vie.VIE_BF16X3, vie.VIE_OP_PA, stream=stream)
        a0.record(stream)
        for _ in range(5):
            vie.vie_matvec(h, x32, y32, vie.VIE_BF16X3, vie.VIE_OP_PA, stream=stream)
        a1.record(stream)
        torch.cuda.synchronize()
        mvb16 = a0.elapsed_time(a1) / 5
        out["matvec_bf16x3"] = dict(ms=mvb16, alg_gbs=mvb / (mvb16 / 1000) / 1e9)
    h.close()
    return out


def run_tucker(args, local):
    """Tucker compression (vie_green_tucker) of a workload's Green tensors at tol 1e-6 and 1e-7: device
    time, ranks, bytes against the full table, and the FP64 matvec and mixed solve before / after."""
    import numpy as np
    import torch

    import paper_1902_02196_gb300 as vie
    from synth import workload

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    vie.build()
    w = workload(args.tucker)
    g = w["grid"]
    R = int(w["dip_pos"].shape[0])
    out = dict(mode="tucker", workload=args.tucker, grid=[g.nx, g.ny, g.nz], nrhs=R, data="synthetic",
               table_bytes=60 * g.nv * 16)
    gen = torch.Generator(device=dev)
    gen.manual_seed(3)
    v = torch.randn((2, 12) + g.shape, dtype=torch.complex128, device=dev, generator=gen)
    for tol in (1e-6, 1e-7):
        t0 = time.perf_counter()
        h = vie.vie_setup((g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), w["freq"], w["eps_real"], w["sigma"])
        setup_s = time.perf_counter() - t0
        y0 = torch.empty_like(v)
        vie.vie_matvec(h, v, y0, vie.VIE_FP64, vie.VIE_OP_NSCAT)
        shape = (R, 12) + g.shape
        e_inc = torch.empty(shape, dtype=torch.complex128, device=dev)
        b = torch.empty_like(e_inc)
        vie.vie_rhs_dipoles(h, w["dip_pos"], w["dip_mom"], e_inc, b)
        x0 = torch.empty_like(b)
        torch.cuda.synchronize()
        vie.vie_solve(h, b, x0, tol=TOL, restart=RESTART, maxit=400)
        torch.cuda.synchronize()
        _, bytes0 = vie.vie_info(h)  # (after the solve's workspaces)
        t0 = time.perf_counter()
        ranks, err, nbytes = vie.vie_green_tucker(h, tol, apply=True)
        tucker_s = time.perf_counter() - t0
        _, bytes1 = vie.vie_info(h)
        y1 = torch.empty_like(v)
        vie.vie_matvec(h, v, y1, vie.VIE_FP64, vie.VIE_OP_NSCAT)
        x1 = torch.empty_like(b)
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record()
        rc, info = vie.vie_solve(h, b, x1, tol=TOL, restart=RESTART, maxit=400)
        a1.record()
        torch.cuda.synchronize()
        h.close()
        rs = np.asarray(ranks)
        out[f"tol_{tol:g}"] = dict(
            setup_s=setup_s, tucker_s=tucker_s, compressed_bytes=int(nbytes),
            ratio=out["table_bytes"] / nbytes, max_rel_err=float(np.max(err)),
            ranks_min=rs.min(0).tolist(), ranks_median=np.median(rs, 0).tolist(), ranks_max=rs.max(0).tolist(),
            handle_bytes_before=int(bytes0), handle_bytes_after=int(bytes1),
            matvec_fp64_rel_diff=float(torch.linalg.vector_norm(y1 - y0) / torch.linalg.vector_norm(y0)),
            solve_rc=rc, solve_s=a0.elapsed_time(a1) / 1000,
            iterations_max=max(i["iterations"] for i in info),
            x_rel_diff=float(torch.linalg.vector_norm(x1 - x0) / torch.linalg.vector_norm(x0)))
    print(json.dumps(out), flush=True)


def run_jm(args, local):
    """Full JM-VIE (vie_jm_*): a magnetodielectric sphere (eps_r 50, sigma 0.5 S/m, mu_r 2 - 0.5 i,
    radius 0.1 m) in an x-polarised plane wave along z at 298 MHz on 16^3 .. 64^3: GMRES to 1e-8 in
    FP64 and in FP32 with FP64 refinement, the absorbed power (electric + magnetic loss) under
    refinement, and the solve times (the K spectra built by one product before the timed solves).
    (The comparison with the Mie series is a GPU test.)"""
    import numpy as np
    import torch

    import paper_1902_02196_gb300 as vie
    from synth import Grid, sphere_phantom

    torch.cuda.set_device(local)
    vie.build()
    f, eta0 = 298e6, 1.0 / (8.8541878128e-12 * 299792458.0)
    mu_s = 2.0 - 0.5j
    rows = []
    for n in (16, 24, 32, 64):
        hgt = 0.2 / n
        g = Grid(n, n, n, hgt, hgt, hgt)
        eps, sig = sphere_phantom(g, 0.1, 50.0, 0.5)
        inside = eps != 1.0
        h = vie.vie_setup((n, n, n, hgt, hgt, hgt), f, eps, sig)
        vie.vie_set_permeability(h, np.where(inside, mu_s.real, 1.0), np.where(inside, -mu_s.imag, 0.0))
        e_t = np.empty((1, 12) + g.shape, dtype=np.complex128)
        h_t = np.empty_like(e_t)
        vie.vie_rhs_planewave(h, [1.0, 0.0, 0.0], [0.0, 0.0, 1.0], e_t[0], None)
        vie.vie_rhs_planewave(h, [0.0, 1.0 / eta0, 0.0], [0.0, 0.0, 1.0], h_t[0], None)
        b = np.empty((1, 2, 12) + g.shape, dtype=np.complex128)
        vie.vie_jm_rhs(h, e_t, h_t, b)
        x = np.empty_like(b)
        vie.vie_jm_matvec(h, b, x, vie.VIE_OP_PA)  # builds the K spectra
        row = dict(n=n)
        # one JM product P^-1 A x of the right-hand side, device buffers, FP64 and FP32
        for tag, prec, dt in (("jm_matvec_fp64_ms", vie.VIE_FP64, torch.complex128),
                              ("jm_matvec_fp32_ms", vie.VIE_FP32, torch.complex64)):
            xd = torch.from_numpy(b).to(device=f"cuda:{local}", dtype=dt)
            yd = torch.empty_like(xd)
            ts = []
            for _ in range(4):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                vie.vie_jm_matvec(h, xd, yd, vie.VIE_OP_PA, precision=prec)
                torch.cuda.synchronize()
                ts.append(time.perf_counter() - t0)
            row[tag] = 1e3 * min(ts[1:])
        for tag, mode in (("fp64", vie.VIE_SOLVE_FP64), ("fp32_refine", vie.VIE_SOLVE_FP32_REFINE)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rc, info = vie.vie_jm_solve(h, b, x, tol=1e-8, restart=60, maxit=40, mode=mode)
            sec = time.perf_counter() - t0
            P = vie.vie_jm_fields(h, x, e_t, h_t)[0]
            row[tag] = dict(rc=rc, seconds=sec, iterations=info[0]["iterations"], fp64_matvecs=info[0]["fp64_matvecs"],
                            fp32_matvecs=info[0]["fp32_matvecs"], P_abs=P)
        h.close()
        rows.append(row)
    # the K operator (row f1) on the head64 batch: FP64 K matvec of 16 right-hand sides (the K
    # spectrum built on first use, timed apart) and the magnetic post-processing (h, b1+, W_m)
    from synth import workload

    wl = workload("head64")
    g = wl["grid"]
    h = vie.vie_setup((g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), wl["freq"], wl["eps_real"], wl["sigma"])
    dev = torch.device("cuda", local)
    shape = (NRHS, 12) + g.shape
    x = torch.randn(shape, dtype=torch.complex128, device=dev)
    y = torch.empty_like(x)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    vie.vie_matvec(h, x[:1], y[:1], vie.VIE_FP64, vie.VIE_OP_K)
    torch.cuda.synchronize()
    kspec_s = time.perf_counter() - t0
    times, times32 = [], []
    x32, y32 = x.to(torch.complex64), torch.empty(shape, dtype=torch.complex64, device=dev)
    torch.cuda.synchronize()
    for _ in range(3):
        t0 = time.perf_counter()
        vie.vie_matvec(h, x, y, vie.VIE_FP64, vie.VIE_OP_K)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
        t0 = time.perf_counter()
        vie.vie_matvec(h, x32, y32, vie.VIE_FP32, vie.VIE_OP_K)
        torch.cuda.synchronize()
        times32.append(time.perf_counter() - t0)
    hinc = torch.empty_like(x)
    vie.vie_rhs_dipoles_h(h, wl["dip_pos"], wl["dip_mom"], hinc)
    b1 = torch.empty((NRHS,) + g.shape, dtype=torch.complex128, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    vie.vie_hfields(h, x, hinc, None, b1)
    torch.cuda.synchronize()
    hf_s = time.perf_counter() - t0
    h.close()
    kmv = dict(workload="head64, 16 RHS", k_spectrum_setup_s=kspec_s, k_matvec_fp64_ms=1e3 * min(times),
               k_matvec_fp32_ms=1e3 * min(times32), hfields_fp64_ms=1e3 * hf_s,
               note="the N operator's transforms with the K block in the z pass (octant K spectra)")
    print(json.dumps(dict(mode="jm", workload="magnetodielectric sphere, plane wave", runs=rows, k_operator=kmv,
                          data="synthetic")), flush=True)


def run_cufft_compare(args, local):
    """cuFFT (torch.fft) + einsum matvec of the head64 batch, timed beside the library's FP32 matvec."""
    import torch

    import paper_1902_02196_gb300 as vie
    from synth import workload

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    vie.build()
    w = workload("head64")
    g = w["grid"]
    h = vie.vie_setup((g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), w["freq"], w["eps_real"], w["sigma"])
    L, _ = vie.vie_info(h)
    Lx, Ly, Lz = L
    stream = torch.cuda.Stream(device=dev)
    torch.cuda.set_stream(stream)
    gen = torch.Generator(device=dev)
    gen.manual_seed(5)
    shape = (NRHS, 12) + g.shape
    x = torch.randn(shape, dtype=torch.complex64, device=dev, generator=gen)
    y = torch.empty_like(x)
    B = torch.randn((12, 12, Lz, Ly, Lx), dtype=torch.complex64, device=dev, generator=gen)
    c1 = torch.randn(g.shape, dtype=torch.complex64, device=dev, generator=gen)
    c2 = torch.randn(g.shape, dtype=torch.complex64, device=dev, generator=gen)

    def ours():
        vie.vie_matvec(h, x, y, vie.VIE_FP32, vie.VIE_OP_PA, stream=stream)

    xp = torch.zeros((NRHS, 12, Lz, Ly, Lx), dtype=torch.complex64, device=dev)

    def cufft():
        xp[:, :, :g.nz, :g.ny, :g.nx] = x
        X = torch.fft.fftn(xp, dim=(-3, -2, -1))
        Y = torch.einsum("abzyx,rbzyx->razyx", B, X)
        yy = torch.fft.ifftn(Y, dim=(-3, -2, -1))[:, :, :g.nz, :g.ny, :g.nx]
        return c1 * x - c2 * yy

    def timeit(fn, n=5):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        for _ in range(n):
            fn()
        a1.record(stream)
        torch.cuda.synchronize()
        return a0.elapsed_time(a1) / n

    t_ours = timeit(ours)
    t_cufft = timeit(cufft)
    # the transforms alone (pad + forward + inverse 3-D FFT of the batch)
    t_fft = timeit(lambda: torch.fft.ifftn(torch.fft.fftn(xp, dim=(-3, -2, -1)), dim=(-3, -2, -1)))
    h.close()
    print(json.dumps(dict(mode="cufft-compare", workload="head64, 16 RHS", fft=list(L),
                          ours_fp32_matvec_ms=t_ours, cufft_einsum_matvec_ms=t_cufft,
                          cufft_fft_pair_only_ms=t_fft, ratio=t_cufft / t_ours)), flush=True)


def run_line_matvec(args, local):
    """One warm-up and one timed FP32 matvec (op PA) of 4 random right-hand sides on a 128 x 96 x 64
    grid of random tissue (3 mm voxels, 298 MHz): Lx = Ly = 256, so the xy transforms take the
    line path, on inputs larger than L2; per-kernel device times from the library's counters."""
    import torch

    import paper_1902_02196_gb300 as vie
    from synth import Grid, random_tissue

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    vie.build()
    g = Grid(128, 96, 64, 0.003, 0.003, 0.003)
    eps, sig = random_tissue(g, seed=3)
    h = vie.vie_setup((g.nx, g.ny, g.nz, g.dx, g.dy, g.dz), 298e6, eps, sig)
    x = torch.randn((4, 12) + g.shape, dtype=torch.complex64, device=dev,
                    generator=torch.Generator(device=dev).manual_seed(5))
    y = torch.empty_like(x)
    torch.cuda.synchronize()
    vie.vie_matvec(h, x, y, vie.VIE_FP32, vie.VIE_OP_PA)
    torch.cuda.synchronize()
    vie.vie_stats_reset(True)
    vie.vie_matvec(h, x, y, vie.VIE_FP32, vie.VIE_OP_PA)
    torch.cuda.synchronize()
    _, st = vie.vie_stats_read()
    vie.vie_stats_reset(False)
    h.close()
    kernels = {k: dict(launches=v[0], ms=v[1], gbs=v[2] / max(v[1], 1e-9) / 1e6) for k, v in st.items()}
    print(json.dumps(dict(mode="line-matvec", workload="128x96x64 random tissue, 4 RHS, FP32 op PA",
                          fft=[256, 256, 128], kernels=kernels)), flush=True)


def main():
    args = parse()
    ws, rank, local = dist_init(args)
    if args.cufft_compare:
        if rank == 0:
            run_cufft_compare(args, local)
        return
    if args.config_run:
        if rank == 0:
            run_config(args, local)
        return
    if args.tucker:
        if rank == 0:
            run_tucker(args, local)
        return
    if args.jm:
        if rank == 0:
            run_jm(args, local)
        return
    if args.serving:
        if rank == 0:
            run_serving(args, local)
        return
    if args.matvec_only:
        run_matvec_only(args, local)
        return
    if args.line_matvec:
        if rank == 0:
            run_line_matvec(args, local)
        return
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
