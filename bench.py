"""Throughput of the arrested-Newton-flow hot path on GB300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl native|reference]

Workload: chiral magnet (J = D = 1, h = 0.6, K = 0.1, interfacial DMI) on a
4096 x 4096 grid (dx = 0.2, halo included), compensated FP32 fields (value +
remainder planes; the flow's sums in float-float pairs, E and dE kept in FP64), 400 compact
skyrmions at seeded positions
(minimum separation 8). Its arrays (8 x 201 MB) are far larger than the 129 MB L2,
so every timed step streams HBM.

One bench step = one call ss_step(ctx, 32): 32 flow steps, each two fused kernels
(pass 1: RK stages 1-2 with the energy / residual / energy-change reductions and
the arrest decision; pass 2: RK stages 3-4 and the RK4 combination), enqueued as
one CUDA graph. value = interior site-updates per second.
e2e: the same calls with the field copied in from pinned host memory and out
again every bench step (ss_set_fields / ss_step / ss_get_fields on host buffers),
from two host threads that each drive one solver context on its own stream, so one
context's copies overlap the other's flow; "serial" in the e2e object is one context
driven from one thread, its copies between its flows.
--impl reference: the FP64 CPU oracle on the host cores, same metric, each step one
oracle flow step on a 512 x 512 crop of the same workload.

--workload configs: time to dx dy max|G| < 1e-6 of the single-problem configurations
(Abelian Higgs 128^2 FP64, chiral magnet 1024^2, chiral magnet 4096^2) on the GPU and
with the FP64 oracle on the host cores.

--workload methods: arrested Newton flow against gradient descent (the first-order
method Sec. 3.2 compares it with; explicit Euler at 0.8 x its stability limit) on
the same configurations and precisions, each to dx dy max|G| < 1e-6 or a step cap:
steps, force evaluations (4 per flow step, 1 per descent step) and seconds.

--workload baby-skyrme: the Baby Skyrme model (Table 1; kappa = 1, mu = 0.7, standard
potential) through the same kernels: flow throughput on 2048^2 with 100 skyrmions
(compensated FP32), and time to dx dy max|G| < 1e-6 of a 256^2 box with 4 skyrmions
on the GPU (FP64, compensated FP32) against the FP64 oracle on the host cores.

--workload bec: the rotating trapped BEC (Table 1; grand canonical, g = 1): flow
throughput on 2048^2 (mu = 40, Omega = 0.9, box 24 x 24) in compensated FP32, and
the vortex-lattice relaxation of the tests (96^2, mu = 10, Omega = 0.85, to
dx dy max|G| < 1e-4) on the GPU against the FP64 oracle on the host cores.

--workload sid: the s+id two-band superconductor (Table 1; a1 = -1, a2 = -0.6, b1 = 0.5,
b2 = 0.4, b3 = 0.3, b4 = 0.15, nu = 0.35): flow throughput on 2048^2 (dx 0.3, 64
vortices) in compensated FP32, and a 256^2 box with 4 vortices relaxed to
dx dy max|G| < 1e-4 on the GPU against the FP64 oracle on the host cores.

--workload demag: the chiral magnet with demagnetisation (Eq. 6, mu_d = 0.8): per-step
cost on the 4096^2 workload (passes and the sine-transform Poisson solve) against the
same workload without it, and time to dx dy max|G| < 1e-6 of the 1024^2 configuration
(8 skyrmions) with and without it.

--workload unet: the learned initialiser's training step (ss_net_train_step) and forward
pass at 256^2, batch 16, Abelian Higgs channels, on seeded synthetic fields: ms per call
after warm-up (CUDA-synchronised wall clock over --steps calls).

--workload ah-batch: time per solve to dx dy max|G| < 1e-6 on the batched Abelian
Higgs set (256 problems, sides 64..512, dx = 0.1, lambda ~ U[0.5, 2], N in 1..4):
one bench step = the whole set relaxed in one batch (compensated FP32), against
the all-FP64 flow run one problem at a time on a seeded subsample of every side.
The line also carries the set's flow throughput while every problem runs.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2603_24370_gb300 import dist as D  # noqa: E402  (no CUDA import)

INNER = 32          # flow steps per bench step (one captured graph)
N = 4096
DX = 0.2
COUNT = 400
SEED = 20264
CROP = 512          # oracle sample (CPU baseline / reference arm)
C = 3
# planes per component of the method's minimum traffic in compensated FP32: phi
# (value, remainder) and v read and written; descent: phi read and written
MIN_PLANES = {False: 6, True: 4}
WORKLOAD = ("chiral magnet 4096x4096 (halo incl.), dx=0.2, J=D=1, h=0.6, K=0.1, interfacial DMI, "
            "400 skyrmions min-sep 8, compensated FP32 fields (value + remainder planes), float-float flow sums "
            "(E and dE kept in FP64), ANF-RK4 (2 fused kernels/step)")


def interior(n: int) -> int:
    return (n - 4) * (n - 4)


# algorithmic bytes per interior site of each kernel of a step (compensated FP32,
# C components; phi is two FP32 planes, value and remainder): pass 1 reads phi,
# v, phi^{n-1} and writes k_v1, k_v2 (7C values); pass 2 reads phi, v, k_v1, k_v2
# and writes phi', v' (8C values).
PASS_BYTES = {1: 4 * 7 * C, 2: 4 * 8 * C}
# the gradient-descent kernel (--method gradient) reads phi (value, remainder) and
# writes phi' (value, remainder) and -G: 5C values
GD_BYTES = 4 * 5 * C


def measured_peaks() -> tuple[dict, str]:
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for fn in ("ss_flow_kernel.cuh", "ss_flow.cu", "ss_device.cuh", "ss_flow_cm.cu", "ss_pack.cuh"):
        with open(os.path.join(ROOT, "paper_2603_24370_gb300", "csrc", fn), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, tile_shape: int):
    """DRAM bytes per launch of `kernel` at tile shape `tile_shape` from the committed
    ncu summary, if it was taken on the current kernel source (else None)."""
    p = os.path.join(ROOT, "profiles", "stage_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as fh:
        d = json.load(fh)
    if d.get("source_hash") != kernel_source_hash():
        return None
    return d.get("bytes_per_launch", {}).get(f"ts{tile_shape}", {}).get(kernel)


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: str):
        self.index = index
        self.proc = None
        self.lines: list[str] = []
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.index, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        self.t0 = time.time()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self) -> dict:
        self.t1 = time.time()
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ts, line in self.lines:
            if ts < self.t0 or ts > self.t1 + 0.1:
                continue
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_sample(steps_budget_s: float = 12.0, max_steps: int = 2000, min_steps: int = 3):
    """Oracle (FP64, as it stands) flow steps on a 512^2 crop of the workload."""
    import numpy as np
    import oracle as O
    from paper_2603_24370_gb300 import inputs as I
    p = I.cm_skyrmions(n=N, count=COUNT, seed=SEED)
    # crop: the workload's skyrmions that fall in the central 512^2 window
    sol = [s for s in p.solitons if abs(s[0]) < 0.5 * CROP * DX - 4 and abs(s[1]) < 0.5 * CROP * DX - 4]
    f = O.ansatz(O.CHIRAL_MAGNET, sol if sol else [(0.0, 0.0, 1.0, 2.0, 0.0)], CROP, CROP, DX, DX)
    v = np.zeros_like(f)
    E = O.energy(O.CHIRAL_MAGNET, p.params, f, DX, DX)
    dt = O.time_step(DX, DX)
    t0 = time.perf_counter()
    n = 0
    while n < min_steps or (time.perf_counter() - t0 < steps_budget_s and n < max_steps):
        f, v, E, _ = O.anf_step(O.CHIRAL_MAGNET, p.params, f, v, DX, DX, dt, E)
        n += 1
    dt_s = time.perf_counter() - t0
    return {"value": interior(CROP) * n / dt_s, "unit": "site-updates/s", "cores": O.num_threads(), "kind": "oracle",
            "sample": f"{n} oracle FP64 flow steps on a {CROP}x{CROP} crop of the workload ({len(sol)} skyrmions), "
                      f"{dt_s:.1f} s"}


def run_reference(args) -> int:
    rank, _, world = D.env_rank()
    if rank != 0:
        return 0
    import numpy as np
    import oracle as O
    from paper_2603_24370_gb300 import inputs as I
    O.build()
    p = I.cm_skyrmions(n=N, count=COUNT, seed=SEED)
    sol = [s for s in p.solitons if abs(s[0]) < 0.5 * CROP * DX - 4 and abs(s[1]) < 0.5 * CROP * DX - 4]
    f = O.ansatz(O.CHIRAL_MAGNET, sol if sol else [(0.0, 0.0, 1.0, 2.0, 0.0)], CROP, CROP, DX, DX)
    v = np.zeros_like(f)
    E = O.energy(O.CHIRAL_MAGNET, p.params, f, DX, DX)
    dt = O.time_step(DX, DX)
    for _ in range(args.warmup):
        f, v, E, _ = O.anf_step(O.CHIRAL_MAGNET, p.params, f, v, DX, DX, dt, E)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f, v, E, _ = O.anf_step(O.CHIRAL_MAGNET, p.params, f, v, DX, DX, dt, E)
    sec = time.perf_counter() - t0
    value = interior(CROP) * args.steps / sec
    line = {
        "impl": "reference", "metric": "site-updates/s", "value": value, "unit": "site-updates/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "reference_sample": f"one oracle flow step per bench step on a {CROP}x{CROP} crop"},
        "cpu_baseline": {"value": value, "unit": "site-updates/s", "cores": O.num_threads(), "kind": "oracle",
                         "sample": f"{args.steps} oracle FP64 flow steps on a {CROP}x{CROP} crop"},
        "e2e": {"value": value, "unit": "site-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_native(args) -> int:
    rank, local_rank, world = D.env_rank()
    D.pin_visible_device(local_rank, world)
    import numpy as np
    import torch
    import torch.distributed as tdist

    if world > 1:
        torch.cuda.set_device(0)
        tdist.init_process_group("nccl")
    from paper_2603_24370_gb300 import build as B
    from paper_2603_24370_gb300 import inputs as I
    from paper_2603_24370_gb300 import soliton as S
    B.build()
    S.load_library()

    n = args.grid
    p = I.cm_skyrmions(n=n, count=COUNT if n >= 2048 else max(1, COUNT * n * n // (N * N)), seed=SEED)
    stream = torch.cuda.Stream()
    s = S.Solver(S.SS_CHIRAL_MAGNET, p.params, n, n, DX, DX, S.SS_FP32, stream=stream)
    s.init_ansatz(p.soliton_array())
    gd = args.method == "gradient"
    if gd:
        s.set_method(S.SS_METHOD_GRADIENT)
    if args.tile_shape == "auto":
        tuned = s.autotune(4)  # tile shape and pass grids for this grid (the flow restarts from rest)
    else:
        s.set_launch(int(args.tile_shape))
        tuned = {"tile_shape": int(args.tile_shape), "blocks": None, "set_by_hand": True}
    f_init = s.fields()
    launches_per_call = 2 + ((INNER + 31) // 32) * 32 * 2  # set_run + head + graph chunk(s)
    if gd:  # set_run + INNER + 1 descent launches (the last evaluates the final field)
        launches_per_call = 1 + INNER + 1

    for _ in range(args.warmup):
        s.step(INNER)

    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_index = vis.split(",")[0].strip() if vis and vis.split(",")[0].strip().isdigit() else str(local_rank)
    clocks = ClockSampler(smi_index)
    clocks.start()
    D.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        st = s.step(INNER)
    ev1.record(stream)
    torch.cuda.synchronize()
    D.barrier()
    clk = clocks.stop()
    sec = ev0.elapsed_time(ev1) / 1e3
    units, job_sec = D.aggregate(interior(n) * INNER * args.steps, sec)
    value = units / job_sec

    # per-kernel durations (CUDA events around each launch on the context stream)
    stage_ms = S.ss_profile_stages(s.ctx, 24)  # mean launch durations over 24 flow steps
    dominant = max(range(2), key=lambda i: stage_ms[i]) + 1
    peaks, src = measured_peaks()
    kname = f"k_pass<CM, float, {dominant}>"
    alg = PASS_BYTES[dominant] * interior(n)
    if gd:
        dominant, kname, alg = 3, "k_pass<CM, float, 3> (gradient descent)", GD_BYTES * interior(n)
    kernel_ms = stage_ms[0] if gd else stage_ms[dominant - 1]
    achieved = alg / (kernel_ms * 1e-3) / 1e9
    traffic = ncu_traffic(f"pass{dominant}", tuned["tile_shape"])
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic, "kernel": kname,
                "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else "fallback 6.8 TB/s",
                "algorithmic_bytes_per_launch": alg,
                "pass_ms": stage_ms,
                "step_bytes_per_site_update": GD_BYTES if gd else sum(PASS_BYTES.values()),
                "step_frac": ((GD_BYTES if gd else sum(PASS_BYTES.values())) * interior(n)
                              / (sum(stage_ms) * 1e-3) / 1e9) / peaks["hbm_gbs"],
                # the method's own minimum per site-update at the run's storage precision,
                # reachable only by a single-pass (temporally blocked) step: phi (value and
                # remainder planes) and v in and out; descent: phi in and out
                "min_bytes_per_site_update": MIN_PLANES[gd] * 4 * C,
                "min_bytes_basis": ("compensated FP32: phi value + remainder in and out" if gd else
                                    "compensated FP32: phi value + remainder and v, in and out"),
                "effective_frac": (MIN_PLANES[gd] * 4 * C * interior(n)
                                   / (sum(stage_ms) * 1e-3) / 1e9) / peaks["hbm_gbs"]}

    # end to end through the C-ABI with host buffers: field in from pinned memory,
    # 32 flow steps, field out to pinned memory, every bench step
    host_in = torch.from_numpy(np.ascontiguousarray(f_init)).pin_memory()
    host_out = [torch.empty(host_in.shape, dtype=torch.float32).pin_memory() for _ in range(2)]
    e2e_steps = 2 * max(2, (args.steps + 7) // 8)  # bench steps, split over the two threads

    def drive(sv, out, k, err):
        try:
            for _ in range(k):
                sv.set_fields(host_in)
                sv.step(INNER)
                S.ss_get_fields(sv.ctx, out)
        except Exception as exc:  # re-raised by the timing thread
            err.append(exc)

    # one context, one host thread: each step's copies sit between its flows
    s.set_fields(host_in)
    s.step(INNER)
    D.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    err = []
    drive(s, host_out[0], e2e_steps, err)
    torch.cuda.synchronize()
    if err:
        raise err[0]
    serial_units, serial_sec = D.aggregate(interior(n) * INNER * e2e_steps, time.perf_counter() - t0)
    # two contexts, two host threads: one context's copies overlap the other's flow
    s2 = S.Solver(S.SS_CHIRAL_MAGNET, p.params, n, n, DX, DX, S.SS_FP32, stream=torch.cuda.Stream())
    s2.set_fields(host_in)
    if gd:
        s2.set_method(S.SS_METHOD_GRADIENT)
    s2.set_launch(tuned["tile_shape"], tuned.get("blocks"))  # the first context's launch shape
    s2.step(INNER)  # its graphs are captured here, before the threads start
    D.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    err = []
    th = [threading.Thread(target=drive, args=(sv, host_out[i], e2e_steps // 2, err)) for i, sv in enumerate((s, s2))]
    for t in th:
        t.start()
    for t in th:
        t.join()
    torch.cuda.synchronize()
    if err:
        raise err[0]
    e_units, e_sec = D.aggregate(interior(n) * INNER * e2e_steps, time.perf_counter() - t0)
    s2.close()
    nbytes = C * n * n * 4

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_sample()
    solve = None
    if world == 1 and args.grid == N and not args.no_solve and not gd:
        try:
            solve = solve_summary(S, I, np)
        except Exception as exc:  # recorded, never fatal for the throughput line
            solve = {"error": str(exc)[:200]}

    s.close()
    if rank == 0:
        line = {
            "metric": "site-updates/s", "value": value, "unit": "site-updates/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * job_sec / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": (WORKLOAD if n == N else WORKLOAD.replace("4096x4096", f"{n}x{n}")).replace(
                           "ANF-RK4 (2 fused kernels/step)",
                           "gradient descent (1 fused kernel/step)" if gd else "ANF-RK4 (2 fused kernels/step)"),
                       "flow_steps_per_bench_step": INNER, "grid": [n, n],
                       "interior_sites": interior(n), "parallelism": "replicas" if world > 1 else "single",
                       "autotuned": tuned,
                       "l2": f"working set {8 * C * n * n * 4 / 1e9:.2f} GB vs 129 MB L2"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e_units / e_sec, "unit": "site-updates/s", "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes, "steps": e2e_steps,
                    "overlap": "two solver contexts on two streams, driven from two host threads",
                    "serial": {"value": serial_units / serial_sec, "steps": e2e_steps,
                               "overlap": "none: one context, one host thread"}},
            "gpu_launches": launches_per_call * args.steps,
            "clocks": clk,
            "final_energy": st["energy"], "final_grad_max": st["grad_max"],
            "time_per_solve": solve,
        }
        print(json.dumps(line))
    if world > 1:
        tdist.destroy_process_group()
    return 0


BATCH_COUNT = 256
BATCH_SEED = 20262
BATCH_TOL = 1e-6
BATCH_CAP = 40000
BATCH_WORKLOAD = ("256 Abelian Higgs relaxations in one batch, sides U{64,128,256,512} (halo incl.), dx=0.1, "
                  "lambda U[0.5,2], N U{1..4} unit vortices uniform in the central half, compensated FP32 "
                  "fields (float-float flow sums, E and dE kept in FP64), to dx dy max|G| < 1e-6")


def solve_summary(S, I, np, count: int = 64, fp64_per_side: int = 4) -> dict:
    """Time per solve of a 64-problem slice of the batched Abelian Higgs set (the
    ah-batch recipe) relaxed as one compensated-FP32 batch (its autotuning timed apart),
    against the all-FP64 flow one problem at a time on `fp64_per_side` seeded problems
    of each side (size-weighted). Both arms count a solve as converged only when the
    FP64 residual of the field is below the tolerance. Also the same comparison
    restricted to the sampled problems that converged in both arms: those alone as
    one batch against their FP64 times."""
    import torch
    probs = I.ah_batch(count, BATCH_SEED)

    def batched(ps):
        b = S.ss_batch_create(S.SS_ABELIAN_HIGGS, S.SS_FP32, ps)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.ss_batch_autotune(b, 4)  # restores every field at rest
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        _, st = S.ss_batch_minimise(b, BATCH_TOL, BATCH_CAP)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        S.ss_batch_destroy(b)
        return t2 - t1, t1 - t0, st

    t_batch, t_tune, st = batched(probs)
    rng = I.SplitMix64(4242)
    by_side = {}
    for i, p in enumerate(probs):
        by_side.setdefault(p.nx, []).append(i)
    t64, c64, per_side = {}, {}, {}
    for side, idx in sorted(by_side.items()):
        pick = sorted({idx[rng.next_u64() % len(idx)] for _ in range(fp64_per_side)})
        for i in pick:
            p = probs[i]
            with S.Solver(S.SS_ABELIAN_HIGGS, p.params, p.nx, p.ny, p.dx, p.dy, S.SS_FP64) as sv:
                sv.init_ansatz(p.soliton_array())
                torch.cuda.synchronize()
                t1 = time.perf_counter()
                r = sv.minimise(BATCH_TOL, BATCH_CAP)
                torch.cuda.synchronize()
                t64[i] = time.perf_counter() - t1
                c64[i] = bool(r["converged"])
        per_side[side] = {"problems": len(idx), "batched_converged": sum(1 for i in idx if st[i]["converged"]),
                          "fp64_sampled": len(pick), "fp64_converged": sum(1 for i in pick if c64[i]),
                          "fp64_mean_s": float(np.mean([t64[i] for i in pick]))}
    plain = sum(v["fp64_mean_s"] * v["problems"] for v in per_side.values()) / count
    both = [i for i in sorted(t64) if c64[i] and st[i]["converged"]]
    conv_both = None
    if both:
        tb, _, stb = batched([probs[i] for i in both])
        conv_both = {"problems": len(both), "batched_fp32_s_per_solve": tb / len(both),
                     "plain_fp64_s_per_solve": float(np.mean([t64[i] for i in both])),
                     "batched_converged": sum(1 for x in stb if x["converged"])}
        conv_both["speedup"] = conv_both["plain_fp64_s_per_solve"] / conv_both["batched_fp32_s_per_solve"]
    return {"problems": count, "batched_fp32_s_per_solve": t_batch / count, "autotune_s": t_tune,
            "plain_fp64_s_per_solve": plain, "speedup": plain / (t_batch / count),
            "batched_converged": sum(1 for x in st if x["converged"]),
            "fp64_converged": sum(c64.values()), "fp64_sampled": len(t64),
            "fp64_sample": f"{fp64_per_side} seeded problems per side, one at a time", "per_side": per_side,
            "converged_in_both": conv_both, "tol": BATCH_TOL, "step_cap": BATCH_CAP,
            "verdict": "FP64 residual of the stored field (FP32 batch: value + remainder)"}


def run_solve(args) -> int:
    """Time per solve: the batched set against the all-FP64 flow one problem at a time."""
    rank, local_rank, world = D.env_rank()
    D.pin_visible_device(local_rank, world)
    import numpy as np
    import torch
    import torch.distributed as tdist

    if world > 1:
        torch.cuda.set_device(0)
        tdist.init_process_group("nccl")
    from paper_2603_24370_gb300 import build as B
    from paper_2603_24370_gb300 import inputs as I
    from paper_2603_24370_gb300 import soliton as S
    B.build()
    S.load_library()
    # the one set of the recipe, its work list sharded across ranks by interior sites
    # (strong scaling: the job's work is fixed); each rank relaxes its share as one
    # batch, and the per-problem results are gathered in problem order
    allp = I.ah_batch(BATCH_COUNT, BATCH_SEED)
    parts = D.shard([p.interior_sites for p in allp], world)
    mine = parts[rank]
    probs = [allp[i] for i in mine]
    warm = I.ah_batch(8, BATCH_SEED + 999, sides=(64, 128))
    for _ in range(args.warmup):
        b = S.ss_batch_create(S.SS_ABELIAN_HIGGS, S.SS_FP32, warm)
        S.ss_batch_minimise(b, BATCH_TOL, 2000)
        S.ss_batch_destroy(b)
    D.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    steps_all, conv = [], 0
    tuned = None
    tune_s = 0.0
    st = []
    for _ in range(args.steps):
        b = S.ss_batch_create(S.SS_ABELIAN_HIGGS, S.SS_FP32, probs)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        tuned = S.ss_batch_autotune(b, 4)  # autotuning, timed apart (restores the fields at rest)
        torch.cuda.synchronize()
        tune_s += time.perf_counter() - t1
        _, st = S.ss_batch_minimise(b, BATCH_TOL, BATCH_CAP)
        S.ss_batch_destroy(b)
    torch.cuda.synchronize()
    sec = time.perf_counter() - t0 - tune_s
    D.barrier()
    units, job_sec = D.aggregate(len(probs) * args.steps, sec)
    per_solve = job_sec / units
    recs = D.gather_records([{"index": i, "converged": x["converged"], "steps": x["steps"], "arrests": x["arrests"],
                              "energy": x["energy"], "grad_max": x["grad_max"], "charge": 0.0, "flux": 0.0}
                             for i, x in zip(mine, st)], len(allp))
    steps_all = [r["steps"] for r in recs]
    conv = sum(1 for r in recs if r["converged"])
    probs = allp

    # flow throughput of the whole set while every problem runs (the first steps from the
    # ansatz), against the measured HBM bandwidth for the passes' algorithmic bytes
    thr = None
    if rank == 0:
        peaks, _ = measured_peaks()
        b = S.ss_batch_create(S.SS_ABELIAN_HIGGS, S.SS_FP32, allp)
        try:
            S.ss_batch_autotune(b, 4)
            for _ in range(3):
                S.ss_batch_step(b, INNER)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            nthr = 4
            for _ in range(nthr):
                _, sts = S.ss_batch_step(b, INNER)
            torch.cuda.synchronize()
            ms_step = 1e3 * (time.perf_counter() - t1) / (nthr * INNER)
        finally:
            S.ss_batch_destroy(b)
        sites = sum(p.interior_sites for p in allp)
        bps = 60 * 4  # compensated FP32, C = 4: pass 1 28 C, pass 2 32 C bytes per site
        thr = {"site_updates_per_s": sites / (ms_step * 1e-3), "ms_per_flow_step": ms_step,
               "interior_sites": sites, "bytes_per_site_update": bps,
               "step_hbm_frac_of_measured": sites * bps / (ms_step * 1e-3) / 1e9 / peaks["hbm_gbs"],
               "running_after": sum(1 for x in sts if not x["converged"]),
               "timed": f"{nthr} x {INNER} flow steps after 3 x {INNER}, from the ansatz"}

    # all-FP64 flow, one problem at a time, on a seeded subsample of every side;
    # the set's mean is the size-weighted mean of the per-side means
    plain = None
    if rank == 0:
        rng = I.SplitMix64(4242)
        by_side = {}
        for p in probs:
            by_side.setdefault(p.nx, []).append(p)
        per_side, sample = {}, 0
        for side, ps in sorted(by_side.items()):
            pick = [ps[rng.next_u64() % len(ps)] for _ in range(args.fp64_per_side)]
            times, conv64 = [], 0
            for p in pick:
                with S.Solver(S.SS_ABELIAN_HIGGS, p.params, p.nx, p.ny, p.dx, p.dy, S.SS_FP64) as sv:
                    sv.init_ansatz(p.soliton_array())
                    torch.cuda.synchronize()
                    t1 = time.perf_counter()
                    r = sv.minimise(BATCH_TOL, BATCH_CAP)
                    torch.cuda.synchronize()
                    times.append(time.perf_counter() - t1)
                    conv64 += 1 if r["converged"] else 0
            per_side[side] = {"mean_s": float(np.mean(times)), "sampled": len(pick), "converged": conv64,
                              "problems_in_set": len(ps)}
            sample += len(pick)
        mean64 = sum(v["mean_s"] * v["problems_in_set"] for v in per_side.values()) / len(probs)
        plain = {"s_per_solve": mean64, "per_side": per_side,
                 "sample": f"{sample} problems ({args.fp64_per_side} per side), one at a time, FP64"}
    if rank == 0:
        line = {
            "metric": "time per solve to dx dy max|G| < 1e-6", "value": per_solve, "unit": "s/solve",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * job_sec / args.steps,
            "higher_is_better": False, "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": BATCH_WORKLOAD, "problems": BATCH_COUNT, "step_cap": BATCH_CAP,
                       "autotuned_rank0": tuned, "autotune_s_rank0": tune_s,
                       "parallelism": (f"work list sharded over {world} ranks by interior sites, "
                                       f"{[len(p) for p in parts]} problems") if world > 1 else "single"},
            "converged": conv, "verdict": "FP64 residual of the stored field (value + remainder)",
            "throughput_all_running": thr,
            "mean_flow_steps": float(np.mean(steps_all)), "max_flow_steps": int(max(steps_all)),
            "converged_by_side": {str(side): sum(1 for p, r in zip(allp, recs) if p.nx == side and r["converged"])
                                  for side in sorted({p.nx for p in allp})},
            "plain_fp64": plain,
            "speedup_vs_plain_fp64": (plain["s_per_solve"] / per_solve) if plain else None,
        }
        print(json.dumps(line))
    if world > 1:
        tdist.destroy_process_group()
    return 0


def run_configs(args) -> int:
    """Time to dx dy max|G| < 1e-6 for each single-problem workload configuration, on
    the GPU (all-FP64 flow and compensated FP32) and with the FP64 oracle on the host
    cores (in full where that takes seconds, else its per-step time on a bounded
    sample times the GPU FP64 step count, stated as such)."""
    rank, local_rank, world = D.env_rank()
    if rank != 0:
        return 0
    D.pin_visible_device(local_rank, 1)
    import numpy as np
    import torch
    import oracle as O
    from paper_2603_24370_gb300 import build as B
    from paper_2603_24370_gb300 import inputs as I
    from paper_2603_24370_gb300 import soliton as S
    B.build()
    O.build()
    S.load_library()

    def gpu_solve(p, prec, tune=True):
        with S.Solver(p.theory, p.params, p.nx, p.ny, p.dx, p.dy, prec) as sv:
            sv.init_ansatz(p.soliton_array())
            if tune:
                sv.autotune(4)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = sv.minimise(1e-6, 100000)
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
            o = sv.observables()
        return {"seconds": sec, "steps": r["steps"], "converged": bool(r["converged"]), "energy": o["energy"],
                "charge": o["charge"]}

    def oracle_step_rate(p, n_crop=None, steps=3):
        nx = n_crop or p.nx
        sol = p.soliton_array()
        if n_crop:
            half = 0.5 * n_crop * p.dx - 4
            sol = np.array([s for s in sol if abs(s[0]) < half and abs(s[1]) < half]) if len(sol) else sol
            if len(sol) == 0:
                sol = p.soliton_array()[:1] * np.array([0, 0, 1, 1, 1])
        f = O.ansatz(p.theory, sol, nx, nx, p.dx, p.dy)
        v = np.zeros_like(f)
        E = O.energy(p.theory, p.params, f, p.dx, p.dy)
        dt = O.time_step(p.dx, p.dy)
        t0 = time.perf_counter()
        for _ in range(steps):
            f, v, E, _ = O.anf_step(p.theory, p.params, f, v, p.dx, p.dy, dt, E)
        return (time.perf_counter() - t0) / steps, (nx - 4) ** 2

    out = {}
    # configuration 0: Abelian Higgs 128^2, one vortex, lambda = 1
    p0 = I.ah_single_vortex()
    g64 = gpu_solve(p0, S.SS_FP64)
    f0 = O.ansatz(p0.theory, p0.soliton_array(), p0.nx, p0.ny, p0.dx, p0.dy)
    t0 = time.perf_counter()
    r0 = O.minimise(p0.theory, p0.params, f0, p0.dx, p0.dy, 1e-6, 100000)
    out["ah128_fp64"] = {"gpu_fp64": g64, "gpu_fp32c": gpu_solve(p0, S.SS_FP32),
                         "oracle": {"seconds": time.perf_counter() - t0, "steps": r0["steps"],
                                    "converged": r0["converged"], "energy": r0["energy"], "timed": "in full"}}
    # configuration 1: chiral magnet 1024^2, 8 skyrmions
    p1 = I.cm_skyrmions()
    g64 = gpu_solve(p1, S.SS_FP64)
    sec_step, sites = oracle_step_rate(p1)
    out["cm1024"] = {"gpu_fp64": g64, "gpu_fp32c": gpu_solve(p1, S.SS_FP32),
                     "oracle": {"seconds": sec_step * g64["steps"], "steps": g64["steps"],
                                "timed": f"3 oracle steps on the full grid x the GPU FP64 step count"}}
    # large: chiral magnet 4096^2, 400 skyrmions (oracle on the 512^2 crop, scaled by sites)
    p4 = I.cm_skyrmions(n=N, count=COUNT, seed=SEED)
    g32 = gpu_solve(p4, S.SS_FP32)
    sec_step, sites = oracle_step_rate(p4, n_crop=CROP)
    out["cm4096"] = {"gpu_fp32c": g32,
                     "oracle": {"seconds": sec_step * interior(N) / sites * g32["steps"], "steps": g32["steps"],
                                "timed": "3 oracle steps on the 512^2 crop, scaled by interior sites and the GPU "
                                         "FP32 step count"}}
    line = {"metric": "time to dx dy max|G| < 1e-6 per configuration", "unit": "s", "higher_is_better": False,
            "n_gpus": 1, "data": "synthetic", "oracle_cores": O.num_threads(), "configs": out}
    print(json.dumps(line))
    return 0


def launch_shape(sv, args) -> dict:
    """Autotune a context's tile shape and pass grids, or fix the tile shape with its
    default grids (--tile-shape, for profiling one launch configuration)."""
    if args.tile_shape == "auto":
        return sv.autotune(4)
    sv.set_launch(int(args.tile_shape))
    return {"tile_shape": int(args.tile_shape), "blocks": None, "set_by_hand": True}


def throughput_only(metric: str, thr: dict) -> int:
    """--no-solve: the workload's throughput record alone (for profiling captures)."""
    print(json.dumps({"metric": metric, "unit": "site-updates/s", "n_gpus": 1, "data": "synthetic",
                      "throughput": thr}))
    return 0


def run_methods(args) -> int:
    """Arrested Newton flow vs gradient descent, to dx dy max|G| < 1e-6 or a cap."""
    rank, local_rank, world = D.env_rank()
    if rank != 0:
        return 0
    D.pin_visible_device(local_rank, 1)
    import torch
    from paper_2603_24370_gb300 import build as B
    from paper_2603_24370_gb300 import inputs as I
    from paper_2603_24370_gb300 import soliton as S
    B.build()
    S.load_library()

    def solve(p, prec, method, cap):
        with S.Solver(p.theory, p.params, p.nx, p.ny, p.dx, p.dy, prec) as sv:
            sv.init_ansatz(p.soliton_array())
            sv.set_method(method)
            sv.autotune(4)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = sv.minimise(1e-6, cap)
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
            o = sv.observables()
        per = 4 if method == S.SS_METHOD_ANF else 1
        return {"seconds": round(sec, 4), "steps": r["steps"], "force_evals": per * r["steps"],
                "converged": bool(r["converged"]), "grad_max": r["grad_max"], "energy": o["energy"],
                "charge": o["charge"], "arrests_or_rises": r["arrests"], "step_cap": cap}

    cases = [("ah128", I.ah_single_vortex(), S.SS_FP64, 2_000_000),
             ("cm1024", I.cm_skyrmions(), S.SS_FP32, 2_000_000),
             ("cm4096", I.cm_skyrmions(n=N, count=COUNT, seed=SEED), S.SS_FP32, 200_000)]
    out = {}
    for name, p, prec, gd_cap in cases:
        anf = solve(p, prec, S.SS_METHOD_ANF, 100_000)
        gd = solve(p, prec, S.SS_METHOD_GRADIENT, gd_cap)
        out[name] = {"precision": {1: "fp32c", 2: "fp64", 3: "fp32"}[prec], "anf": anf, "gradient": gd,
                     "gd_over_anf": {"steps": round(gd["steps"] / max(anf["steps"], 1), 2),
                                     "force_evals": round(gd["force_evals"] / max(anf["force_evals"], 1), 2),
                                     "seconds": round(gd["seconds"] / max(anf["seconds"], 1e-9), 2)}}
        print(json.dumps({name: out[name]}), file=sys.stderr, flush=True)
    line = {"metric": "minimiser comparison to dx dy max|G| < 1e-6", "unit": "s", "higher_is_better": False,
            "n_gpus": 1, "data": "synthetic", "gd_step": "0.8 x (3/8) / (1/dx^2 + 1/dy^2)", "configs": out}
    print(json.dumps(line))
    return 0


def run_baby_skyrme(args) -> int:
    """Baby Skyrme: flow throughput and time to solution (see the module docstring)."""
    rank, local_rank, world = D.env_rank()
    if rank != 0:
        return 0
    D.pin_visible_device(local_rank, 1)
    import numpy as np
    import torch
    import oracle as O
    from paper_2603_24370_gb300 import build as B
    from paper_2603_24370_gb300 import inputs as I
    from paper_2603_24370_gb300 import soliton as S
    B.build()
    O.build()
    S.load_library()
    peaks, src = measured_peaks()
    n = 2048
    p = I.bs_skyrmions(n=n)
    with S.Solver(S.SS_BABY_SKYRME, p.params, n, n, p.dx, p.dy, S.SS_FP32) as sv:
        sv.init_ansatz(p.soliton_array())
        tuned = launch_shape(sv, args)
        for _ in range(args.warmup):
            sv.step(INNER)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sv.step(INNER)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        ms = S.ss_profile_stages(sv.ctx, 8)
        o = sv.observables()
    thr = {"site_updates_per_s": interior(n) * INNER * args.steps / sec, "pass_ms": ms, "autotuned": tuned,
           "hbm_frac_of_measured": [PASS_BYTES[k + 1] * interior(n) / (ms[k] * 1e-3) / 1e9 / peaks["hbm_gbs"]
                                    for k in range(2)],
           "charge_after": o["charge"], "skyrmions": len(p.solitons)}
    if args.no_solve:
        return throughput_only("Baby Skyrme: site-updates/s at 2048^2", thr)

    q = I.bs_skyrmions(n=256, count=4, seed=20266)
    sol = q.soliton_array()
    gpu = {}
    for name, prec in (("fp64", S.SS_FP64), ("fp32c", S.SS_FP32)):
        with S.Solver(S.SS_BABY_SKYRME, q.params, q.nx, q.ny, q.dx, q.dy, prec) as sv:
            sv.init_ansatz(sol)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = sv.minimise(1e-6, 100000)
            torch.cuda.synchronize()
            o = sv.observables()
            gpu[name] = {"seconds": time.perf_counter() - t0, "steps": r["steps"], "converged": bool(r["converged"]),
                         "energy": o["energy"], "charge": o["charge"]}
    f = O.ansatz(q.theory, sol, q.nx, q.ny, q.dx, q.dy)
    v = np.zeros_like(f)
    E = O.energy(q.theory, q.params, f, q.dx, q.dy)
    t0 = time.perf_counter()
    k = 0
    while time.perf_counter() - t0 < 10.0 and k < 2000:
        f, v, E, _ = O.anf_step(q.theory, q.params, f, v, q.dx, q.dy, O.time_step(q.dx, q.dy), E)
        k += 1
    oracle_step = (time.perf_counter() - t0) / k
    line = {"metric": "Baby Skyrme: site-updates/s at 2048^2; time to dx dy max|G| < 1e-6 at 256^2", "unit": "s",
            "n_gpus": 1, "data": "synthetic", "dtype": "f32 (throughput); f64 and f32c (time to solution)",
            "config": {"workload": "Baby Skyrme kappa=1, mu=0.7, nu=0, dx=0.2; 2048^2 with 100 compact skyrmions "
                                   "(R 2.5, min-sep 10); 256^2 with 4", "flow_steps_per_bench_step": INNER},
            "throughput": thr, "time_to_solution": {"gpu": gpu, "oracle": {
                "seconds": oracle_step * gpu["fp64"]["steps"], "per_step_s": oracle_step, "sampled_steps": k,
                "cores": O.num_threads(), "timed": "oracle steps for ~10 s x the GPU FP64 step count"}}}
    print(json.dumps(line))
    return 0


def run_bec(args) -> int:
    """Rotating BEC: flow throughput and vortex-lattice time to solution."""
    rank, local_rank, world = D.env_rank()
    if rank != 0:
        return 0
    D.pin_visible_device(local_rank, 1)
    import math
    import numpy as np
    import torch
    import oracle as O
    from paper_2603_24370_gb300 import build as B
    from paper_2603_24370_gb300 import soliton as S
    B.build()
    O.build()
    S.load_library()
    peaks, src = measured_peaks()
    n, L = 2048, 24.0
    dx = L / (n - 1)
    prm = (1.0, 0.9, 40.0)
    ring = [[3.0 * math.cos(a), 3.0 * math.sin(a), 1, 0.3, 0.0] for a in np.linspace(0, 2 * math.pi, 9)[:-1]]
    with S.Solver(S.SS_BEC, prm, n, n, dx, dx, S.SS_FP32) as sv:
        sv.init_ansatz(ring)
        tuned = launch_shape(sv, args)
        for _ in range(args.warmup):
            sv.step(INNER)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sv.step(INNER)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        ms = S.ss_profile_stages(sv.ctx, 8)
        o = sv.observables()
    # the same box at the fixed atom number of that state: the refresh's cost per step
    fixed = {}
    with S.Solver(S.SS_BEC, (prm[0], prm[1], 0.0, o["atoms"]), n, n, dx, dx, S.SS_FP32) as sv:
        sv.init_ansatz(ring)
        sv.set_launch(tuned["tile_shape"], tuned["blocks"])  # the grand-canonical run's launch shape
        for _ in range(args.warmup):
            sv.step(INNER)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sv.step(INNER)
        torch.cuda.synchronize()
        fsec = time.perf_counter() - t0
        of = sv.observables()
        fixed = {"ms_per_flow_step": fsec / (INNER * args.steps) * 1e3,
                 "grand_canonical_ms_per_flow_step": sec / (INNER * args.steps) * 1e3,
                 "atoms": of["atoms"], "chemical_potential": of["chemical_potential"]}
    bytes2 = {1: 4 * 7 * 2, 2: 4 * 8 * 2}  # compensated FP32, C = 2
    thr = {"site_updates_per_s": interior(n) * INNER * args.steps / sec, "pass_ms": ms, "autotuned": tuned,
           "hbm_frac_of_measured": [bytes2[k + 1] * interior(n) / (ms[k] * 1e-3) / 1e9 / peaks["hbm_gbs"]
                                    for k in range(2)],
           "atoms": o["atoms"], "angular_momentum_per_atom": o["angular_momentum"] / o["atoms"],
           "fixed_atom_number": fixed}
    if args.no_solve:
        return throughput_only("BEC: site-updates/s at 2048^2", thr)
    n2, dx2 = 96, 0.15
    prm2 = (1.0, 0.85, 10.0)
    vort = [[1.2 * math.cos(a), 1.2 * math.sin(a), 1, 0.4, 0.0] for a in np.linspace(0, 2 * math.pi, 6)[:-1]]
    gpu = {}
    for name, prec in (("fp64", S.SS_FP64), ("fp32c", S.SS_FP32)):
        with S.Solver(S.SS_BEC, prm2, n2, n2, dx2, dx2, prec) as sv:
            sv.init_ansatz(vort)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = sv.minimise(1e-4, 30000)
            torch.cuda.synchronize()
            o = sv.observables()
            gpu[name] = {"seconds": time.perf_counter() - t0, "steps": r["steps"], "converged": bool(r["converged"]),
                         "energy": o["energy"], "atoms": o["atoms"],
                         "angular_momentum_per_atom": o["angular_momentum"] / o["atoms"]}
    # the same lattice at a fixed atom number (that of the grand-canonical solution)
    n_atoms = gpu["fp64"]["atoms"]
    gpu_fixed = {}
    for name, prec in (("fp64", S.SS_FP64), ("fp32c", S.SS_FP32)):
        with S.Solver(S.SS_BEC, (prm2[0], prm2[1], 0.0, n_atoms), n2, n2, dx2, dx2, prec) as sv:
            sv.init_ansatz(vort)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = sv.minimise(1e-4, 30000)
            torch.cuda.synchronize()
            o = sv.observables()
            gpu_fixed[name] = {"seconds": time.perf_counter() - t0, "steps": r["steps"],
                               "converged": bool(r["converged"]), "energy": o["energy"], "atoms": o["atoms"],
                               "chemical_potential": o["chemical_potential"],
                               "angular_momentum_per_atom": o["angular_momentum"] / o["atoms"]}
    f = O.ansatz_bec(prm2, vort, n2, n2, dx2, dx2)
    t0 = time.perf_counter()
    ref = O.minimise(4, prm2, f, dx2, dx2, 1e-4, 30000)
    osec = time.perf_counter() - t0
    f = O.ansatz_bec((prm2[0], prm2[1], math.sqrt(prm2[0] * n_atoms / math.pi)), vort, n2, n2, dx2, dx2)
    t0 = time.perf_counter()
    ref_f = O.minimise_fixed_n(prm2[:2], n_atoms, f, dx2, dx2, 1e-4, 30000)
    osec_f = time.perf_counter() - t0
    line = {"metric": "BEC: site-updates/s at 2048^2; time to dx dy max|G| < 1e-4 of a vortex lattice at 96^2",
            "unit": "s", "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "rotating BEC, grand canonical, g=1; throughput 2048^2 box 24, mu=40, Omega=0.9, "
                                   "8-vortex ring ansatz, compensated FP32; lattice 96^2 dx=0.15, mu=10, "
                                   "Omega=0.85, 5-vortex ring ansatz", "flow_steps_per_bench_step": INNER},
            "throughput": thr,
            "time_to_solution": {"gpu": gpu, "oracle": {"seconds": osec, "steps": ref["steps"],
                                                         "energy": ref["energy"], "cores": O.num_threads(),
                                                         "timed": "in full"}},
            "time_to_solution_fixed_atom_number": {
                "atoms": n_atoms, "gpu": gpu_fixed,
                "oracle": {"seconds": osec_f, "steps": ref_f["steps"], "energy": ref_f["energy"], "mu": ref_f["mu"],
                           "cores": O.num_threads(), "timed": "in full"}}}
    print(json.dumps(line))
    return 0


def run_sid(args) -> int:
    """s+id: flow throughput and time to solution (see the module docstring)."""
    rank, local_rank, world = D.env_rank()
    if rank != 0:
        return 0
    D.pin_visible_device(local_rank, 1)
    import numpy as np
    import torch
    import oracle as O
    from paper_2603_24370_gb300 import build as B
    from paper_2603_24370_gb300 import inputs as I
    from paper_2603_24370_gb300 import soliton as S
    B.build()
    O.build()
    S.load_library()
    peaks, src = measured_peaks()
    prm = (-1.0, -0.6, 0.5, 0.4, 0.3, 0.15, 0.35)

    def vortices(n, dx, count, seed):
        rng = I.SplitMix64(seed)
        half = 0.5 * (n - 1) * dx
        pts = I._separated_positions(rng, count, half, half, 6.0, 5.0)
        return [(x, y, 1.0, 1.0, 0.0) for x, y in pts]

    n, dx = 2048, 0.3
    with S.Solver(S.SS_SID, prm, n, n, dx, dx, S.SS_FP32) as sv:
        sv.init_ansatz(vortices(n, dx, 64, 20267))
        tuned = launch_shape(sv, args)
        for _ in range(args.warmup):
            sv.step(INNER)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            sv.step(INNER)
        torch.cuda.synchronize()
        sec = time.perf_counter() - t0
        ms = S.ss_profile_stages(sv.ctx, 8)
        o = sv.observables()
    bytes6 = {1: 4 * 7 * 6, 2: 4 * 8 * 6}  # compensated FP32, C = 6
    thr = {"site_updates_per_s": interior(n) * INNER * args.steps / sec, "pass_ms": ms, "autotuned": tuned,
           "hbm_frac_of_measured": [bytes6[k + 1] * interior(n) / (ms[k] * 1e-3) / 1e9 / peaks["hbm_gbs"]
                                    for k in range(2)],
           "winding_after": o["charge"], "flux_over_2pi": o["flux"] / (2 * np.pi)}
    if args.no_solve:
        return throughput_only("s+id: site-updates/s at 2048^2", thr)
    m, dxm = 256, 0.3
    vort = vortices(m, dxm, 4, 20268)
    gpu = {}
    for name, prec in (("fp64", S.SS_FP64), ("fp32c", S.SS_FP32)):
        with S.Solver(S.SS_SID, prm, m, m, dxm, dxm, prec) as sv:
            sv.init_ansatz(vort)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = sv.minimise(1e-4, 100000)
            torch.cuda.synchronize()
            o = sv.observables()
            gpu[name] = {"seconds": time.perf_counter() - t0, "steps": r["steps"], "converged": bool(r["converged"]),
                         "energy": o["energy"], "winding": o["charge"], "flux_over_2pi": o["flux"] / (2 * np.pi)}
    f, _ = O.ansatz_sid(prm, vort, m, m, dxm, dxm)
    t0 = time.perf_counter()
    ref = O.minimise(5, prm, f, dxm, dxm, 1e-4, 100000)
    osec = time.perf_counter() - t0
    line = {"metric": "s+id: site-updates/s at 2048^2; time to dx dy max|G| < 1e-4 at 256^2", "unit": "s",
            "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "s+id a1=-1 a2=-0.6 b1=0.5 b2=0.4 b3=0.3 b4=0.15 nu=0.35, dx=0.3; 2048^2 with 64 "
                                   "unit vortices (min-sep 5), 256^2 with 4", "flow_steps_per_bench_step": INNER},
            "throughput": thr,
            "time_to_solution": {"gpu": gpu, "oracle": {"seconds": osec, "steps": ref["steps"],
                                                         "energy": ref["energy"], "converged": ref["converged"],
                                                         "cores": O.num_threads(), "timed": "in full"}}}
    print(json.dumps(line))
    return 0


def run_demag(args) -> int:
    """Chiral magnet with demagnetisation: step cost and time to solution."""
    rank, local_rank, world = D.env_rank()
    if rank != 0:
        return 0
    D.pin_visible_device(local_rank, 1)
    import torch
    from paper_2603_24370_gb300 import build as B
    from paper_2603_24370_gb300 import inputs as I
    from paper_2603_24370_gb300 import soliton as S
    B.build()
    S.load_library()
    mu_d = 0.8
    out = {}
    p = I.cm_skyrmions(n=N, count=COUNT, seed=SEED)
    for name, prm in (("demag", tuple(p.params) + (mu_d,)), ("plain", tuple(p.params))):
        with S.Solver(S.SS_CHIRAL_MAGNET, prm, N, N, DX, DX, S.SS_FP32) as sv:
            sv.init_ansatz(p.soliton_array())
            tuned = sv.autotune(4)
            for _ in range(args.warmup):
                sv.step(INNER)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                sv.step(INNER)
            torch.cuda.synchronize()
            ms_step = 1e3 * (time.perf_counter() - t0) / (args.steps * INNER)
            ms = S.ss_profile_stages(sv.ctx, 8)
        out[name] = {"site_updates_per_s": interior(N) / (ms_step * 1e-3), "ms_per_flow_step": ms_step,
                     "pass_ms": ms, "autotuned": tuned}
    out["demag"]["poisson_solve_ms_per_step"] = out["demag"]["ms_per_flow_step"] - sum(out["demag"]["pass_ms"])
    q = I.cm_skyrmions()
    tts = {}
    arms = () if args.no_solve else (("demag_fp32c", S.SS_FP32, tuple(q.params) + (mu_d,)),
                                     ("demag_fp64", S.SS_FP64, tuple(q.params) + (mu_d,)),
                                     ("plain_fp32c", S.SS_FP32, tuple(q.params)))
    for name, prec, prm in arms:
        with S.Solver(S.SS_CHIRAL_MAGNET, prm, q.nx, q.ny, q.dx, q.dy, prec) as sv:
            sv.init_ansatz(q.soliton_array())
            sv.autotune(4)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = sv.minimise(1e-6, 100000)
            torch.cuda.synchronize()
            o = sv.observables()
            tts[name] = {"seconds": time.perf_counter() - t0, "steps": r["steps"], "converged": bool(r["converged"]),
                         "energy": o["energy"], "charge": o["charge"]}
    line = {"metric": "chiral magnet with demagnetisation: ms per flow step at 4096^2; time to 1e-6 at 1024^2",
            "unit": "ms", "n_gpus": 1, "data": "synthetic",
            "config": {"workload": f"chiral magnet (J=D=1, K=0.1, h=0.6, interfacial), mu_d={mu_d}, dx=0.2; "
                                   "4096^2 with 400 skyrmions, 1024^2 with 8; compensated FP32 unless stated",
                       "flow_steps_per_bench_step": INNER},
            "step_cost_4096": out, "time_to_solution_1024": tts}
    print(json.dumps(line))
    return 0


def run_unet(args) -> int:
    """U-Net training step and forward pass at 256^2, batch 16 (see the module docstring)."""
    rank, local_rank, world = D.env_rank()
    if rank != 0:
        return 0
    D.pin_visible_device(local_rank, 1)
    import numpy as np
    import torch
    from paper_2603_24370_gb300 import build as B
    from paper_2603_24370_gb300 import soliton as S
    B.build()
    S.load_library()
    nb, side, C = 16, 256, 4
    g = torch.Generator(device="cuda").manual_seed(1)
    ansatz = torch.randn((nb, C, side, side), generator=g, device="cuda") * 0.5
    relaxed = ansatz + 0.05 * torch.randn((nb, C, side, side), generator=g, device="cuda")
    cp = np.linspace(0.5, 1.5, nb)
    out = torch.empty((nb, side, side, 16), device="cuda")
    net = S.ss_net_create(S.SS_ABELIAN_HIGGS, side, nb, seed=3)
    try:
        for _ in range(max(args.warmup, 3)):
            S.ss_net_train_step(net, ansatz, cp, relaxed, nb, 1e-4)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            loss = S.ss_net_train_step(net, ansatz, cp, relaxed, nb, 1e-4)
        torch.cuda.synchronize()
        train_ms = 1e3 * (time.perf_counter() - t0) / args.steps
        t0 = time.perf_counter()
        for _ in range(args.steps):
            S.ss_net_forward(net, ansatz, cp, nb, out)
        torch.cuda.synchronize()
        fwd_ms = 1e3 * (time.perf_counter() - t0) / args.steps
    finally:
        S.ss_net_destroy(net)
    print(json.dumps({"metric": "U-Net training step and forward pass, 256^2, batch 16", "unit": "ms",
                      "higher_is_better": False, "n_gpus": 1, "data": "synthetic", "dtype": "bf16 (fp32 accumulate)",
                      "steps": args.steps, "warmup": max(args.warmup, 3),
                      "config": {"workload": "4-level U-Net (16/32/48/96 channels), Abelian Higgs input, 256^2 x 16"},
                      "train_step_ms": train_ms, "forward_ms": fwd_ms, "loss": loss}))
    return 0


def main() -> int:
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("native", "reference"), default="native")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--grid", type=int, default=N, help="grid side (default: the 4096 workload; smaller for ncu)")
    ap.add_argument("--workload",
                    choices=("cm4096", "ah-batch", "configs", "methods", "baby-skyrme", "bec", "sid", "demag", "unet"),
                    default="cm4096")
    ap.add_argument("--tile-shape", choices=("auto", "0", "1"), default="auto",
                    help="flow tile shape: autotuned (default) or fixed with default grids (for profiling "
                         "one shape; the default run and the baby-skyrme, bec and sid workloads)")
    ap.add_argument("--fp64-per-side", type=int, default=2, help="ah-batch: FP64 problems timed per side")
    ap.add_argument("--no-solve", action="store_true",
                    help="skip the time-per-solve record of the default run, and the time-to-solution runs of "
                         "the baby-skyrme, bec and sid workloads")
    ap.add_argument("--method", choices=("anf", "gradient"), default="anf",
                    help="minimiser timed by the default workload (gradient: one descent kernel per step)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ah-batch":
        return run_solve(args)
    if args.workload == "configs":
        return run_configs(args)
    if args.workload == "methods":
        return run_methods(args)
    if args.workload == "baby-skyrme":
        return run_baby_skyrme(args)
    if args.workload == "bec":
        return run_bec(args)
    if args.workload == "sid":
        return run_sid(args)
    if args.workload == "demag":
        return run_demag(args)
    if args.workload == "unet":
        return run_unet(args)
    return run_native(args)


if __name__ == "__main__":
    sys.exit(main())
