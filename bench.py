"""Benchmark: forward + adjoint of the 8x8 loop metasurface (64 ports, 4096 capacitance
configurations, 65,536 grid points + 64 loss points, 63.6 MHz) through the C ABI.

One step = mts_solve (port solves, objective, adjoint gradient at the loss points) +
mts_superpose (the full field B = H I, complex64) + mts_backward (grad_C from the loss
cotangent) over one batch of 4096 configurations. Inputs are resident in HBM; L2 is flushed
(256 MB write) between timed steps. Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision mixed|bf16|fp64] [--no-cpu-baseline] [--no-fp64-path]

--impl reference times the CPU oracle (the reference implementation of the method for this
build) on the host cores, on a bounded sample of the same workload per step.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "8×8 array forward+adjoint configs/s at rel err ≤1e-6 vs FP64; % of roofline"
UNIT = "configs/s"
N_CFG = 4096
WORKLOAD = ("array_8x8: 8x8 square loops (side 50 mm, pitch 55 mm, 16 segments/side, 64 ports), "
            "4096 configs C~U[20,200] pF, 1 freq 63.6 MHz, Bz on 4x128x128 points at z=10..40 mm "
            "+ 64 loss points at z=40 mm, loss |Bz| MSE to N(0,1)e-6 T targets")
# ncu DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch at the full
# workload, with the hash of the kernel source it was taken from; reported as null once the
# source changes. Captured on 1024 configurations and scaled by 4 (both kernels' traffic is
# proportional to the configurations); see profiles/.
TRAFFIC = {"superpose_tc.cu": {"sha256_12": "53a4d1e63df5", "bytes": 4 * (33.5488e6 + 477.061376e6)},
           "solve_mixed.cu": {"sha256_12": "7e2cb62e4f4b", "bytes": 4 * (0.706048e6 + 0.027648e6)},
           "field_adjoint_tc.cu": {"sha256_12": "d542b2ab4e30", "bytes": 4 * (585.531648e6 + 12.9728e6)}}


def fp32_peak():
    """FP32 FMA throughput of this GPU for the ALU rooflines: measured by the probe program
    built beside libmts.so (packed fma.rn.f32x2 chains, best of five launches), else derived
    from the device's SM count and clock (128 FP32 lanes x 2 flops per SM and cycle)."""
    import torch
    from paper_2503_18479_gb300.build_lib import PEAK_PROBE
    try:
        r = subprocess.run([PEAK_PROBE], capture_output=True, text=True, timeout=120)
        d = json.loads(r.stdout.strip().splitlines()[-1])
        return {"tflops": float(d["ffma2_tflops"]), "ffma_tflops": float(d["ffma_tflops"]),
                "fp64_tflops": float(d["dfma_tflops"]),
                "source": "measured: fp32_peak probe (packed fma.rn.f32x2 chains, 8 x 256-thread "
                          f"CTAs per SM, best of 5), {d['sms']} SMs at {d['clock_mhz']:.0f} MHz"}
    except Exception as e:  # derived from the device properties
        props = torch.cuda.get_device_properties(torch.cuda.current_device())
        sms = props.multi_processor_count
        mhz = float(subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"],
                                   capture_output=True, text=True).stdout.split()[0])
        return {"tflops": sms * 128 * 2 * mhz * 1e6 / 1e12, "fp64_tflops": sms * 2 * 2 * mhz * 1e6 / 1e12,
                "source": f"derived: {sms} SMs x 128 FP32 lanes x 2 flops x {mhz:.0f} MHz "
                          f"(probe unavailable: {type(e).__name__})"}


def lu_flops(N: int) -> int:
    """Real flops of one complex LU factorisation, 8N^3/3."""
    return (8 * N ** 3) // 3


def solve_flops_per_system(N: int, L: int) -> int:
    """Algorithmic flops of one system's solve + objective + adjoint (real flops; a complex
    multiply-add is 8): LU 8N^3/3, two triangular-solve pairs (currents and adjoint) 8N^2
    each, one FP64-accurate residual per solve 8N^2 each, B at the L loss points and
    u = H^T conj(G) 4LN each. Refinement corrections beyond one residual are not counted."""
    return (8 * N ** 3) // 3 + 2 * 8 * N * N + 2 * 8 * N * N + 2 * 4 * L * N


def sha12(path):
    with open(path, "rb") as f:
        return hashlib.sha256(f.read()).hexdigest()[:12]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "bf16", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64-path", action="store_true")
    ap.add_argument("--e2e-steps", type=int, default=200)
    ap.add_argument("--n-cfg", type=int, default=N_CFG, help="configurations per GPU (profiling runs)")
    ap.add_argument("--other-workloads", default="loop,line,ragged,32x32,fit,fit8x8,sroute",
                    help="comma list of extra workloads timed after the headline (loop, line, "
                         "ragged, 32x32, fit, fit8x8, sroute; empty for none); reported under "
                         "other_workloads")
    ap.add_argument("--x32-configs", type=int, default=256,
                    help="configurations of the 32x32 entry (256 = the benchmark's; fewer for a "
                         "profiler capture)")
    ap.add_argument("--x32-grid", type=int, default=512,
                    help="grid points per side of each field plane of the 32x32 entry")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(x: float, world: int, device) -> float:
    """The largest x over all ranks (all_reduce MAX; no-op for one rank)."""
    import torch
    import torch.distributed as tdist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    if world > 1:
        tdist.all_reduce(t, op=tdist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(n_cfg_per_rank: int, steps: int, world: int, max_ms: float) -> float:
    """Configurations per second of the whole job: every rank's batches over the slowest
    rank's time (weak scaling: each rank owns n_cfg_per_rank configurations)."""
    return world * n_cfg_per_rank * steps / (max_ms / 1e3)


# ---------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id = gpu_id
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.gpu_id, f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                pw.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(pw) if pw else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_uuid(dev):
    import torch
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return str(dev.index if dev.index is not None else 0)


# ---------------------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------------------
def run_ours(args, rank, world, local):
    import torch
    import torch.distributed as tdist

    from paper_2503_18479_gb300 import native as nv
    from paper_2503_18479_gb300 import workloads as W
    from paper_2503_18479_gb300.build_lib import build
    from paper_2503_18479_gb300.simulator import Simulator

    build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    peak32 = fp32_peak()
    if world > 1:
        tdist.init_process_group("nccl", device_id=dev)
    wl = W.array_8x8(seed=rank, n_cfg=args.n_cfg)
    prec = args.precision
    sim = Simulator(wl, prec, device=dev)
    st = torch.cuda.current_stream()
    n_cfg = wl.n_cfg
    C = torch.from_numpy(wl.C).to(dev)
    ev = sim.make_eval(C, True)
    tape = sim.alloc_tape(n_cfg)
    B = torch.empty((n_cfg, sim.sumFP), dtype=sim.b_dtype, device=dev)
    loss = torch.empty((n_cfg, 1), dtype=torch.float64, device=dev)
    grad_C = torch.empty((n_cfg, sim.n_ports), dtype=torch.float64, device=dev)
    gl = torch.ones((n_cfg, 1), dtype=torch.float64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step(e_mid1=None, e_mid2=None):
        nv.mts_solve(sim.pb, sim.prec, sim.basis, ev, None, loss, tape)
        if e_mid1 is not None:
            e_mid1.record(st)
        nv.mts_superpose(sim.pb, sim.prec, sim.basis, ev, tape, B)
        if e_mid2 is not None:
            e_mid2.record(st)
        nv.mts_backward(sim.pb, sim.prec, sim.basis, ev, tape, None, gl, grad_C)

    for _ in range(max(args.warmup, 3)):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    code, n_bad = sim.status(tape, n_cfg)

    K = args.steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
    sampler = ClockSampler(gpu_uuid(dev))
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        tdist.barrier()
    torch.cuda.synchronize()
    n0 = nv.mts_launch_count()
    t_wall = time.perf_counter()
    for i in range(K):
        flush.fill_(1)
        e0, e1, e2, e3 = evs[i]
        e0.record(st)
        step(e1, e2)
        e3.record(st)
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall
    if world > 1:
        tdist.barrier()
    launches = nv.mts_launch_count() - n0
    clocks = sampler.stop()
    total_ms = sum(e[0].elapsed_time(e[3]) for e in evs)
    gemm_ms = sum(e[1].elapsed_time(e[2]) for e in evs) / K
    solve_ms = sum(e[0].elapsed_time(e[1]) for e in evs) / K
    bwd_ms = sum(e[2].elapsed_time(e[3]) for e in evs) / K
    max_ms = max_over_ranks(total_ms, world, dev)
    value = whole_job_value(n_cfg, K, world, max_ms)

    # ---- end to end through the public API, host buffers, copies inside the timed region.
    # Every step uploads its C from pinned host memory and downloads its loss and dloss/dC;
    # the copies run on a second stream, double-buffered, so that step i+1's upload and
    # step i's download overlap step i's kernels (the host waits for each download).
    Ch = [torch.from_numpy(wl.C).pin_memory(), torch.from_numpy(wl.C).pin_memory()]
    loss_h = [torch.empty((n_cfg, 1), dtype=torch.float64).pin_memory() for _ in range(2)]
    grad_h = [torch.empty((n_cfg, sim.n_ports), dtype=torch.float64).pin_memory() for _ in range(2)]
    Cd = [torch.empty_like(C), torch.empty_like(C)]
    loss_d = [loss, torch.empty_like(loss)]
    grad_d = [grad_C, torch.empty_like(grad_C)]
    ev2 = [sim.make_eval(Cd[0], True), sim.make_eval(Cd[1], True)]
    cs = torch.cuda.Stream(device=dev)
    KE = max(1, min(args.e2e_steps, K))

    def e2e_run(nsteps):
        """nsteps pipelined steps; returns the CUDA-event time from the first upload to the
        last download (ms)."""
        e_in = [torch.cuda.Event() for _ in range(2)]
        e_done = [torch.cuda.Event() for _ in range(2)]
        e_out = [torch.cuda.Event() for _ in range(2)]
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(cs)
        with torch.cuda.stream(cs):
            Cd[0].copy_(Ch[0], non_blocking=True)
        e_in[0].record(cs)
        for i in range(nsteps):
            j = i % 2
            st.wait_event(e_in[j])
            nv.mts_forward(sim.pb, sim.prec, sim.basis, ev2[j], B, None, loss_d[j], tape, st)
            nv.mts_backward(sim.pb, sim.prec, sim.basis, ev2[j], tape, None, gl, grad_d[j], st)
            e_done[j].record(st)
            if i + 1 < nsteps:  # next upload, once step i-1 no longer reads that buffer
                if i >= 1:
                    cs.wait_event(e_done[1 - j])
                with torch.cuda.stream(cs):
                    Cd[1 - j].copy_(Ch[1 - j], non_blocking=True)
                e_in[1 - j].record(cs)
            cs.wait_event(e_done[j])
            with torch.cuda.stream(cs):
                loss_h[j].copy_(loss_d[j], non_blocking=True)
                grad_h[j].copy_(grad_d[j], non_blocking=True)
            e_out[j].record(cs)
            if i >= 1:
                e_out[1 - j].synchronize()  # the host reads step i-1's results
        t1.record(cs)
        t1.synchronize()
        return t0.elapsed_time(t1)

    e2e_run(3)
    torch.cuda.synchronize()
    flush.fill_(1)
    torch.cuda.synchronize()
    e2e_ms = e2e_run(KE)
    e2e_value = whole_job_value(n_cfg, KE, world, max_over_ranks(e2e_ms, world, dev))

    # ---- rooflines: the solve (ALU-bound) and the superposition (HBM-bound); the line's
    # `roofline` is whichever took longer in the timed region (the dominant kernel)
    P = wl.n_points
    npc = {"mixed": 3, "bf16": 1, "fp64": 0}[prec]
    if prec == "fp64":
        alg_bytes = n_cfg * P * 16 + P * 64 * 8 + n_cfg * 64 * 16
    else:
        alg_bytes = n_cfg * P * 8 + npc * 2 * ((P + 127) // 128 * 128) * 64 + npc * 2 * 2 * n_cfg * 64
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        hbm_peak, peak_src = float(peaks["hbm_gbs"]), "measured"
    except Exception:
        hbm_peak, peak_src = 6800.0, "fallback"
    csrc = os.path.join(ROOT, "paper_2503_18479_gb300", "csrc")

    def traffic_of(src):
        tr = TRAFFIC.get(src, {})
        return tr.get("bytes") if (tr.get("sha256_12") == sha12(os.path.join(csrc, src)) and prec != "fp64") else None

    achieved = alg_bytes / (gemm_ms / 1e3) / 1e9
    roof_gemm = {"kernel": "superpose_tc_kernel<3>" if prec == "mixed" else
                 ("superpose_tc_kernel<1>" if prec == "bf16" else "superpose_simt_kernel<double>"),
                 "bound": "hbm", "achieved": achieved, "peak": hbm_peak,
                 "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)", "unit": "GB/s",
                 "frac": achieved / hbm_peak, "traffic": traffic_of("superpose_tc.cu"),
                 "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": gemm_ms}
    st0 = wl.structures[0]
    flops = n_cfg * solve_flops_per_system(st0.n_ports, st0.n_loss)
    tf = flops / (solve_ms / 1e3) / 1e12
    alu_peak = peak32["tflops"] if prec != "fp64" else peak32["fp64_tflops"]
    roof_solve = {"kernel": "solve_mixed_v4<64>" if prec != "fp64" else "solve_fp64_kernel<64>",
                  "bound": "alu", "achieved": tf, "peak": alu_peak,
                  "peak_source": peak32["source"] + (" (FP64 chains)" if prec == "fp64" else ""),
                  "unit": "TFLOP/s", "frac": tf / alu_peak, "traffic": traffic_of("solve_mixed.cu"),
                  "algorithmic_flops_per_launch": flops, "avg_launch_ms": solve_ms,
                  "note": "duration includes the plan and reduce launches of mts_solve (~2 %)"}
    dominant, secondary = (roof_solve, roof_gemm) if solve_ms >= gemm_ms else (roof_gemm, roof_solve)

    # ---- backward with a full-field cotangent grad_B (dL/dRe B + j dL/dIm B for every
    # configuration and point): u = H^T conj(grad_B), mu = A^-1 u, dloss/dC
    backward_field = None
    if rank == 0:
        gB = torch.randn((n_cfg, sim.sumFP), dtype=sim.b_dtype, device=dev)
        gb_bytes = gB.numel() * gB.element_size()

        def time_backward(s_, ev_, tape_, gC_):
            nv.mts_backward(s_.pb, s_.prec, s_.basis, ev_, tape_, gB, gl, gC_)
            torch.cuda.synchronize()
            tot = 0.0
            for _ in range(5):
                flush.fill_(1)
                b0 = torch.cuda.Event(enable_timing=True)
                b1 = torch.cuda.Event(enable_timing=True)
                b0.record(st)
                nv.mts_backward(s_.pb, s_.prec, s_.basis, ev_, tape_, gB, gl, gC_, st)
                b1.record(st)
                b1.synchronize()
                tot += b0.elapsed_time(b1)
            return tot / 5

        gC2 = torch.empty_like(grad_C)
        ms_refactor = time_backward(sim, ev, tape, gC2)
        ms_keep = None
        if prec != "fp64":
            # the same problem built with keep_factors: the forward stores the register
            # solve's factors, the backward solves with them instead of factoring again
            simk = Simulator(wl, prec, device=dev, keep_factors=True)
            evk = simk.make_eval(C, True)
            tapek = simk.alloc_tape(n_cfg)
            lossk = torch.empty_like(loss)
            nv.mts_forward(simk.pb, simk.prec, simk.basis, evk, None, None, lossk, tapek, st)
            gC3 = torch.empty_like(grad_C)
            ms_keep = time_backward(simk, evk, tapek, gC3)
            same = bool(torch.equal(gC2, gC3))
            del simk, evk, tapek, lossk, gC3
        msb = ms_keep if ms_keep is not None else ms_refactor
        backward_field = {"ms": msb, "ms_factoring_again": ms_refactor,
                          "u_kernel_traffic": traffic_of("field_adjoint_tc.cu"),
                          "ms_kept_factors": ms_keep,
                          "kept_equals_refactored": same if ms_keep is not None else None,
                          "grad_B_bytes": gb_bytes,
                          "grad_B_read_GBs": gb_bytes / (msb / 1e3) / 1e9,
                          "hbm_frac_of_call": gb_bytes / (msb / 1e3) / 1e9 / hbm_peak,
                          "steps": 5,
                          "note": "one mts_backward call with a full-field cotangent (random, "
                                  "complex64) and the loss cotangent: u = H^T conj(grad_B) over all "
                                  "points on the tensor cores, the adjoint solve of every system "
                                  "(with the forward's factors when the problem keeps them), "
                                  "dloss/dC; 256 MB L2 flush before each call"}
        del gB, gC2
        torch.cuda.empty_cache()

    # ---- FP64 GPU path on the same workload (context for the mixed-precision speed-up)
    fp64_path = None
    if not args.no_fp64_path and prec != "fp64":
        sim64 = Simulator(wl, "fp64", device=dev)
        ev64 = sim64.make_eval(C, True)
        tape64 = sim64.alloc_tape(n_cfg)
        B64 = torch.empty((n_cfg, sim64.sumFP), dtype=torch.complex128, device=dev)
        loss64 = torch.empty((n_cfg, 1), dtype=torch.float64, device=dev)
        g64 = torch.empty_like(grad_C)

        def step64():
            nv.mts_forward(sim64.pb, sim64.prec, sim64.basis, ev64, B64, None, loss64, tape64)
            nv.mts_backward(sim64.pb, sim64.prec, sim64.basis, ev64, tape64, None, gl, g64)

        step64()
        torch.cuda.synchronize()
        k64 = 3
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(st)
        for _ in range(k64):
            step64()
        a1.record(st)
        a1.synchronize()
        ms64 = a0.elapsed_time(a1) / k64
        fp64_path = {"value": n_cfg / (ms64 / 1e3), "unit": UNIT, "ms_per_step": ms64, "steps": k64,
                     "speedup_of_this_line": (n_cfg * K / (total_ms / 1e3)) / (n_cfg / (ms64 / 1e3))}
        del B64, sim64
        torch.cuda.empty_cache()

    stash = {}
    setup = basis_setup(sim, wl, dev, peak32) if rank == 0 else None
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
        "warmup": args.warmup, "ms_per_step": max_ms / K, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"mixed": "f32", "bf16": "f32", "fp64": "f64"}[prec],
        "dtype_detail": {"mixed": "f32 LU + double-float (f32 pair) residuals + bf16x3 pieces on "
                                  "the tensor cores with f32 accumulation",
                         "bf16": "f32 LU + double-float (f32 pair) residuals + bf16 operands on "
                                 "the tensor cores with f32 accumulation",
                         "fp64": "f64 throughout"}[prec],
        "data": "synthetic (seeded PCG64 per rank); shapes of the paper's 8x8 metasurface",
        "config": {"workload": WORKLOAD, "n_cfg_per_gpu": n_cfg, "points": P, "ports": 64,
                   "precision": prec, "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"replicas x{world} (independent batches, no collective)"},
        "field_points_per_s": value * P,
        "breakdown_ms": {"solve_loss_adjoint": solve_ms, "superpose": gemm_ms, "backward": bwd_ms},
        "e2e": {"value": e2e_value, "unit": UNIT, "steps": KE,
                "h2d_bytes_per_step": int(Ch[0].numel() * 8),
                "d2h_bytes_per_step": int(loss_h[0].numel() * 8 + grad_h[0].numel() * 8),
                "note": "every step copies its C in and its loss and grad_C out (pinned host "
                        "memory; the host waits for each step's results); copies double-"
                        "buffered on a second stream, overlapping the neighbouring steps' "
                        "kernels; the field B stays on the device; no L2 flush between "
                        "these steps (each writes 2.15 GB of B, more than the 129 MB L2), so "
                        "the basis operand stays L2-resident as in steady-state serving"},
        "gpu_launches": int(launches),
        "gpu_launches_per_step": launches / K,
        "roofline": dominant,
        "roofline_other": secondary,
        "clocks": clocks,
        "wall_s_timed_loop": t_wall,
        "status": {"code": code, "systems_flagged": n_bad},
        "fp64_path": fp64_path,
        "fp32_peak": peak32,
        "backward_field": backward_field,
        "basis_setup": setup,
        "other_workloads": other_workloads(args, dev, prec, peak32, stash) if rank == 0 else None,
    }
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"], out["accuracy"] = cpu_baseline_and_accuracy(wl, sim, C, B, loss, grad_C, gl, tape, ev)
        if "32x32" in stash and out.get("other_workloads"):
            out["other_workloads"]["32x32"]["accuracy_per_path"] = path_errors_32x32(stash["32x32"])
    if world > 1:
        tdist.destroy_process_group()
    if rank == 0:
        print(json.dumps(out))


# Algorithmic flops of one segment-point pair of the Biot-Savart basis (closed form of the
# segment's Bz: R2 = R1 + d 3, (R1 x d)_z 3, |R1|^2 and |R2|^2 10, R1.R2 5, two square roots
# 2, n1 n2 (n1 n2 + R1.R2) 3, (n1 + n2) / den 2, times the cross product 1, accumulate 1;
# a square root or a division counts as one flop)
BASIS_FLOPS_PER_PAIR = 30


def basis_setup(sim, wl, dev, peak):
    """Time mts_build_basis for the workload (CUDA events; the basis is rebuilt in place)
    and split it into the Biot-Savart basis H and the partial inductances M by rebuilding a
    copy of the problem with one field point per structure (M only)."""
    import dataclasses

    import torch

    from paper_2503_18479_gb300 import native as nv

    def timed_build(s):
        nv.mts_build_basis(s.pb, s.prec, s.basis)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record()
        nv.mts_build_basis(s.pb, s.prec, s.basis)
        a1.record()
        a1.synchronize()
        return a0.elapsed_time(a1)

    from paper_2503_18479_gb300.simulator import Simulator
    t_all = timed_build(sim)
    one = [dataclasses.replace(st, px=st.px[:1], py=st.py[:1], pz=st.pz[:1], loss_idx=st.loss_idx[:0],
                               pcomp=None if getattr(st, "pcomp", None) is None else st.pcomp[:1])
           for st in wl.structures]
    wl1 = dataclasses.replace(wl, structures=one, target=None, target_rule=None)
    sim1 = Simulator(wl1, "mixed", device=dev)
    t_m = timed_build(sim1)
    del sim1
    torch.cuda.empty_cache()
    seg = [len(st.vx) for st in wl.structures]
    pairs_h = sum(st.n_points * S for st, S in zip(wl.structures, seg))
    pairs_m = sum(S * (S + 1) // 2 for S in seg)  # loop pairs k <= l, every segment pair
    t_h = max(t_all - t_m, 1e-6)
    tf = pairs_h * BASIS_FLOPS_PER_PAIR / (t_h / 1e3) / 1e12
    return {"ms": t_all, "ms_field_basis_H": t_h, "ms_inductances_M": t_m,
            "segment_point_pairs": pairs_h, "segment_pairs": pairs_m,
            "H_pairs_per_s": pairs_h / (t_h / 1e3), "M_pairs_per_s": pairs_m / (t_m / 1e3),
            "H_roofline": {"bound": "alu", "achieved": tf, "peak": peak["tflops"], "unit": "TFLOP/s",
                           "frac": tf / peak["tflops"],
                           "flops_per_pair": BASIS_FLOPS_PER_PAIR,
                           "note": "FP32 closed form per segment-point pair; FP64 near-field terms and "
                                   "the near-field test are not counted"},
            "note": "M time from a rebuild with one field point per structure; H = total - M"}


def other_workloads(args, dev, prec, peak, stash):
    """The same step (solve + objective + adjoint, superposition, gradient) on the other
    synthetic workloads: configs/s, systems/s and field points/s at one GPU, CUDA events
    over a few steps with the L2 flushed between them, the split between the solve call and
    the superposition call, the LU's share of the FP32 peak, and the basis setup time."""
    import torch

    from paper_2503_18479_gb300 import native as nv
    from paper_2503_18479_gb300 import workloads as W
    from paper_2503_18479_gb300.simulator import Simulator
    makers = {
        "loop": ("single_loop: circular 64-gon, 1 config, 101 freqs, 32x32 grid", lambda: W.single_loop(seed=0)),
        "line": ("line_8x1: 8x1 square loops, 1024 configs, 201 freqs, 64x64 grid", lambda: W.line_8x1(seed=0)),
        "ragged": ("ragged: 10,000 structures of 1..128 ports, 1-16 freqs, 64x64 grid each", lambda: W.ragged(seed=0)),
        "32x32": (f"array_32x32: 1024 ports, {args.x32_configs} configs, 4x{args.x32_grid}x{args.x32_grid} grid",
                  lambda: W.array_32x32(seed=0, n_cfg=args.x32_configs, grid=args.x32_grid)),
        "fit": ("loop_sweep: Adam fits (lr 1e-13) of 100 initial C x 100 target fields on the "
                "single loop at 63.6 MHz, 200 epochs replayed from one CUDA graph", None),
        "fit8x8": ("array_8x8: 4096 independent Adam fits (lr 1e-13) of the 64 capacitances to "
                   "the 64-point target, 200 epochs (solve + objective + adjoint + Adam, no field) "
                   "replayed from one CUDA graph", None),
        "sroute": ("sroute_8x8: scattering-parameter route, 65 structure ports (64 RC-loaded cells "
                   "+ a drive port fed through S_C12), 4096 configs, 63.6 MHz, 4x128x128 + 64 "
                   "points; step = Eq. 2-3 loads, W = (1 - S11 S0)^-1 S12, Bcomb = field W, "
                   "objective, Eq. 10 adjoint, dL/dC", None),
    }
    res = {}
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    st = torch.cuda.current_stream()
    for name in [x for x in args.other_workloads.split(",") if x]:
        desc, make = makers[name]
        if name == "fit":
            res[name] = fit_sweep(desc, dev, prec)
            continue
        if name == "fit8x8":
            res[name] = fit_array(desc, dev, prec)
            continue
        if name == "sroute":
            res[name] = sroute_bench(desc, dev, prec, flush)
            continue
        wl = make()
        if wl.target is None:  # timing only: a zero target costs the same work
            wl.target = np.zeros(sum(s.n_freq * s.n_loss for s in wl.structures))
        sim = Simulator(wl, prec, device=dev)
        setup = basis_setup(sim, wl, dev, peak) if name in ("32x32",) else None
        n = wl.n_cfg
        C = torch.from_numpy(wl.C).to(dev)
        ev = sim.make_eval(C, True)
        tape = sim.alloc_tape(n)
        B = torch.empty((n, sim.sumFP), dtype=sim.b_dtype, device=dev)
        loss = torch.empty((n, sim.n_struct), dtype=torch.float64, device=dev)
        g = torch.empty((n, sim.n_ports), dtype=torch.float64, device=dev)
        gl = torch.ones((n, sim.n_struct), dtype=torch.float64, device=dev)
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(4)]

        def step(m=None):
            if m:
                m[0].record(st)
            nv.mts_solve(sim.pb, sim.prec, sim.basis, ev, None, loss, tape)
            if m:
                m[1].record(st)
            nv.mts_superpose(sim.pb, sim.prec, sim.basis, ev, tape, B)
            if m:
                m[2].record(st)
            nv.mts_backward(sim.pb, sim.prec, sim.basis, ev, tape, None, gl, g)
            if m:
                m[3].record(st)

        for _ in range(3):
            flush.fill_(1)
            step()
        torch.cuda.synchronize()
        code, bad = sim.status(tape, n)
        K = 10
        ms = ms_solve = ms_sup = 0.0
        for _ in range(K):
            flush.fill_(1)
            step(marks)
            marks[3].synchronize()
            ms += marks[0].elapsed_time(marks[3])
            ms_solve += marks[0].elapsed_time(marks[1])
            ms_sup += marks[1].elapsed_time(marks[2])
        ms, ms_solve, ms_sup = ms / K, ms_solve / K, ms_sup / K
        n_sys = n * sum(s.n_freq for s in wl.structures)
        lu = n * sum(s.n_freq * lu_flops(s.n_ports) for s in wl.structures)
        lu_tf = lu / (ms_solve / 1e3) / 1e12
        bytes_b = n * sim.sumFP * (16 if prec == "fp64" else 8)
        mac = 8 * n * sum(s.n_freq * s.n_points * s.n_ports for s in wl.structures)  # complex B = H I
        r = {"workload": desc, "precision": prec, "ms_per_step": ms,
             "configs_per_s": n / (ms / 1e3), "systems_per_s": n_sys / (ms / 1e3),
             "field_points_per_s": n * sim.sumFP / (ms / 1e3), "steps": K,
             "breakdown_ms": {"solve_loss_adjoint": ms_solve, "superpose": ms_sup,
                              "backward": ms - ms_solve - ms_sup},
             "solve_roofline": {"bound": "alu", "achieved": lu_tf, "peak": peak["tflops"], "unit": "TFLOP/s",
                                "frac": lu_tf / peak["tflops"], "algorithmic_flops": lu,
                                "note": "LU flops 8N^3/3 only, over the whole mts_solve call (refinement, "
                                        "objective and adjoint not counted)"},
             "superpose": {"B_bytes": bytes_b, "achieved_GBs": bytes_b / (ms_sup / 1e3) / 1e9,
                           "achieved_TFLOPs_real": 2 * mac / 8 / (ms_sup / 1e3) / 1e12},
             "status": {"code": code, "systems_flagged": bad}}
        if setup:
            r["basis_setup"] = setup
        res[name] = r
        if name == "32x32":
            stash["32x32"] = path_samples(wl, sim, C, B, dev, prec)
        del sim, B, tape
        torch.cuda.empty_cache()
    return res


def path_samples(wl, sim, C, B, dev, prec, n_cfg=2, n_pts=4096, seed=11):
    """B of the first n_cfg configurations at n_pts sampled field points from every
    precision path (MTS_MIXED and MTS_BF16 on the tensor cores, MTS_FP64) for the per-path
    error against the oracle; the timed step's own precision comes from its output."""
    import torch

    from paper_2503_18479_gb300.simulator import Simulator
    st = wl.structures[0]
    rng = np.random.Generator(np.random.PCG64(seed))
    idx = np.sort(rng.choice(st.n_points, size=min(n_pts, st.n_points), replace=False))
    it = torch.from_numpy(idx).to(dev)
    out = {"idx": idx, "C": wl.C[:n_cfg], prec: B[:n_cfg][:, it].cpu().numpy()}
    for p in ("mixed", "bf16", "fp64"):
        if p in out:
            continue
        s = Simulator(wl, p, device=dev)
        if p != "fp64":  # a few configurations: force the tensor-core superposition path
            s.tuning["simt_max_sys"] = -1
        o = s.forward(C[:n_cfg], want_B=True, want_loss=False)
        out[p] = o["B"][:, it].cpu().numpy()
        del s, o
        torch.cuda.empty_cache()
    return out


def sroute_bench(desc, dev, prec, flush, K=10):
    """The scattering-parameter route on the synthetic 8x8-plus-drive workload: configs/s of
    the whole step and the time of its parts (CUDA events, L2 flushed between steps)."""
    import torch

    from paper_2503_18479_gb300 import native as nv
    from paper_2503_18479_gb300 import workloads as W
    from paper_2503_18479_gb300.sroute import SRoute
    wl = W.sroute_array(seed=0, n_cfg=N_CFG)
    sr = SRoute(wl.S0, wl.field, wl.rows, wl.cols, wl.n1, sc_const=wl.sc_const,
                loss_idx=wl.loss_idx, target=wl.target, precision=prec, device=dev)
    n, F, nS = wl.n_cfg, sr.F, sr.nS
    R = torch.from_numpy(wl.R).to(dev)
    C = torch.from_numpy(wl.C).to(dev)
    om = torch.from_numpy(wl.omega).to(dev)
    svar = torch.empty((n, F, nS, 2), dtype=torch.float64, device=dev)
    ev = nv.SrouteEval(svar, sr.target, sr.loss_mode)
    tape = sr.alloc_tape(n)
    B = torch.empty((n, sr.n1, F, sr.P), dtype=sr.b_dtype, device=dev)
    loss = torch.empty(n, dtype=torch.float64, device=dev)
    gl = torch.ones(n, dtype=torch.float64, device=dev)
    gs = torch.empty((n, F, nS, 2), dtype=torch.float64, device=dev)
    gC = torch.empty((n, nS), dtype=torch.float64, device=dev)
    st = torch.cuda.current_stream()
    ev_ = [torch.cuda.Event(enable_timing=True) for _ in range(5)]

    def step(marks=False):
        if marks:
            ev_[0].record(st)
        nv.mts_rc_reflection(n, F, nS, om, R, C, wl.Z0, nS, 0, svar)
        nv.mts_sroute_forward(sr.sp, sr.prec, sr.sbasis, ev, B_out=None, loss_out=loss, tape=tape)
        if marks:
            ev_[1].record(st)
        nv.mts_sroute_backward(sr.sp, sr.prec, sr.sbasis, ev, tape, grad_loss=gl, grad_svar=gs)
        nv.mts_rc_reflection_vjp(n, F, nS, om, R, C, wl.Z0, nS, 0, gs, grad_C=gC)
        if marks:
            ev_[2].record(st)

    def full_step():
        nv.mts_rc_reflection(n, F, nS, om, R, C, wl.Z0, nS, 0, svar)
        nv.mts_sroute_forward(sr.sp, sr.prec, sr.sbasis, ev, B_out=B, loss_out=loss, tape=tape)
        nv.mts_sroute_backward(sr.sp, sr.prec, sr.sbasis, ev, tape, grad_loss=gl, grad_svar=gs)
        nv.mts_rc_reflection_vjp(n, F, nS, om, R, C, wl.Z0, nS, 0, gs, grad_C=gC)

    for _ in range(3):
        flush.fill_(1)
        full_step()
    torch.cuda.synchronize()
    code, bad = sr.status(tape, n)
    ms = ms_nob = ms_fwd = 0.0
    for _ in range(K):
        flush.fill_(1)
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(st)
        full_step()
        a1.record(st)
        a1.synchronize()
        ms += a0.elapsed_time(a1)
        flush.fill_(1)
        step(marks=True)
        ev_[2].synchronize()
        ms_fwd += ev_[0].elapsed_time(ev_[1])
        ms_nob += ev_[0].elapsed_time(ev_[2])
    ms, ms_nob, ms_fwd = ms / K, ms_nob / K, ms_fwd / K
    out = {"workload": desc, "precision": prec, "ms_per_step": ms,
           "configs_per_s": n / (ms / 1e3), "field_points_per_s": n * sr.n1 * F * sr.P / (ms / 1e3),
           "ms_loads_solve_objective": ms_fwd, "ms_adjoint_and_vjp": ms_nob - ms_fwd,
           "ms_superposition": ms - ms_nob, "steps": K,
           "status": {"code": code, "systems_flagged": bad}}
    del sr, B, tape
    torch.cuda.empty_cache()
    return out


def fit_sweep(desc, dev, prec, epochs=200):
    """The optimisation loop on the initialisation sweep: fit-epochs per second."""
    import torch

    from paper_2503_18479_gb300 import workloads as W
    from paper_2503_18479_gb300.optimize import AdamFit
    from paper_2503_18479_gb300.simulator import Simulator
    wl = W.loop_sweep()
    st = wl.structures[0]
    # targets: |Bz| at the loss points for the target capacitances (forward map on the GPU)
    sim0 = Simulator(wl, prec, device=dev)
    Ct = torch.from_numpy(wl.target_rule[1]).to(dev)
    B = sim0.forward(Ct, want_B=True, want_loss=False)["B"]
    t = B.reshape(wl.n_cfg, st.n_freq, st.n_points)[:, :, torch.as_tensor(st.loss_idx, device=dev)].abs()
    sim = Simulator(wl, prec, device=dev, target=t.reshape(-1).double().cpu().numpy(), target_per_cfg=True)
    fit = AdamFit(sim, torch.from_numpy(wl.C), lr=1e-13, max_epochs=epochs + 2)
    fit.run(2)  # warm-up: one eager epoch, the graph capture and one replay
    torch.cuda.synchronize()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record()
    fit.run(epochs)
    a1.record()
    a1.synchronize()
    ms = a0.elapsed_time(a1)
    h = fit.history[: epochs + 2].cpu().numpy()[:, :, 0]
    improved = float(((h[-1] < 1e-2 * h[0]) | (h[0] == 0)).mean())
    return {"workload": desc, "precision": prec, "fits": wl.n_cfg, "epochs": epochs,
            "ms": ms, "fit_epochs_per_s": wl.n_cfg * epochs / (ms / 1e3),
            "share_of_fits_loss_down_100x": improved}


def fit_array(desc, dev, prec, epochs=200):
    """The optimisation loop on the 8x8 array: 4096 fits, fit-epochs per second."""
    import torch

    from paper_2503_18479_gb300 import workloads as W
    from paper_2503_18479_gb300.optimize import AdamFit
    from paper_2503_18479_gb300.simulator import Simulator
    wl = W.array_8x8(seed=0, n_cfg=N_CFG, grid=8, planes=(0.02,))  # the field grid is unused
    sim = Simulator(wl, prec, device=dev)
    fit = AdamFit(sim, torch.from_numpy(wl.C), lr=1e-13, max_epochs=epochs + 2)
    fit.run(2)
    torch.cuda.synchronize()
    a0 = torch.cuda.Event(enable_timing=True)
    a1 = torch.cuda.Event(enable_timing=True)
    a0.record()
    fit.run(epochs)
    a1.record()
    a1.synchronize()
    ms = a0.elapsed_time(a1)
    h = fit.history[: epochs + 2].cpu().numpy()[:, :, 0]
    return {"workload": desc, "precision": prec, "fits": wl.n_cfg, "epochs": epochs, "ms": ms,
            "fit_epochs_per_s": wl.n_cfg * epochs / (ms / 1e3),
            "ms_per_epoch_all_fits": ms / epochs,
            "median_loss_ratio_last_over_first": float(np.median(h[-1] / h[0]))}


def cpu_baseline_and_accuracy(wl, sim, C, B, loss, grad_C, gl, tape, ev):
    """Time the FP64 oracle (as it stands) on a bounded sample of the same workload on the
    host cores, and compare the GPU outputs of the same configurations with it."""
    import torch

    import oracle
    from paper_2503_18479_gb300 import native as nv
    st = wl.structures[0]
    H = oracle.basis(st.loop_vtx_off, st.vx, st.vy, st.vz, st.px, st.py, st.pz, wl.wire_radius)
    _, M = oracle.inductance(st.loop_vtx_off, st.vx, st.vy, st.vz, wl.wire_radius)
    t = wl.structure_target(0)
    # calibrate, then size the sample for ~10 s of CPU work
    t0 = time.perf_counter()
    oracle.forward(H, M, st.R, wl.C[:8], st.omega, st.V, st.loss_idx, t)
    oracle.gradient(H, M, st.R, wl.C[:8], st.omega, st.V, st.loss_idx, t)
    per = (time.perf_counter() - t0) / 8
    n = int(max(8, min(wl.n_cfg, 10.0 / max(per, 1e-6))))
    idx = np.arange(n)
    t0 = time.perf_counter()
    ref = oracle.forward(H, M, st.R, wl.C[idx], st.omega, st.V, st.loss_idx, t)
    g = oracle.gradient(H, M, st.R, wl.C[idx], st.omega, st.V, st.loss_idx, t)
    dt = time.perf_counter() - t0
    cores = oracle.num_threads()
    base = {"value": n / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{n} of the 4096 configurations, forward (full field at all {wl.n_points} points) "
                      f"+ loss + adjoint gradient, FP64, {cores} OpenMP threads; basis setup untimed",
            "single_thread": oracle_single_thread()}
    # accuracy of the GPU path (last timed step) on the same configurations
    torch.cuda.synchronize()
    Bg = B[:n].cpu().numpy().reshape(n, 1, -1)
    lg = loss[:n, 0].cpu().numpy()
    gg = grad_C[:n].cpu().numpy()
    rel = lambda a, b: float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))
    ga, gb = gg.ravel(), g.ravel()
    acc = {"sample_configs": n, "B_rel_l2": rel(Bg, ref["B"]), "loss_rel_l2": rel(lg, ref["loss"]),
           "grad_rel_l2": rel(gg, g), "grad_cosine": float(ga @ gb / (np.linalg.norm(ga) * np.linalg.norm(gb)))}
    return base, acc


def path_errors_32x32(smp):
    """Relative L2 error of B from each precision path against the FP64 oracle on the
    sampled configurations and field points of the 32x32 array (the oracle's own basis and
    inductances of the full geometry)."""
    import oracle
    from paper_2503_18479_gb300 import workloads as W
    wl = W.array_32x32(seed=0)
    st = wl.structures[0]
    idx = smp["idx"]
    t0 = time.perf_counter()
    H = oracle.basis(st.loop_vtx_off, st.vx, st.vy, st.vz, st.px[idx], st.py[idx], st.pz[idx], wl.wire_radius)
    _, M = oracle.inductance(st.loop_vtx_off, st.vx, st.vy, st.vz, wl.wire_radius)
    ref = oracle.forward(H, M, st.R, smp["C"], st.omega, st.V)["B"].reshape(len(smp["C"]), -1)
    rel = lambda a, b: float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))
    out = {p: rel(smp[p].reshape(ref.shape), ref) for p in ("fp64", "mixed", "bf16")}
    out.update({"sample": f"{len(smp['C'])} configurations x {len(idx)} random field points of "
                          f"{st.n_points}; oracle basis and inductances of the full geometry",
                "oracle_s": time.perf_counter() - t0,
                "bounds": {"fp64": 1e-10, "mixed": 1e-6, "bf16": 1e-2}})
    return out


def oracle_single_thread(n=16):
    """configs/s of the oracle restricted to one thread (OMP_NUM_THREADS=1, a child
    process) on the first n configurations of the 8x8 workload: forward (full field) + loss
    + adjoint gradient, basis setup untimed."""
    code = (
        "import json, sys, time, numpy as np\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "import oracle\n"
        "from paper_2503_18479_gb300 import workloads as W\n"
        "wl = W.array_8x8(seed=0, n_cfg=%d)\n"
        "st = wl.structures[0]\n"
        "H = oracle.basis(st.loop_vtx_off, st.vx, st.vy, st.vz, st.px, st.py, st.pz, wl.wire_radius)\n"
        "_, M = oracle.inductance(st.loop_vtx_off, st.vx, st.vy, st.vz, wl.wire_radius)\n"
        "t = wl.structure_target(0)\n"
        "t0 = time.perf_counter()\n"
        "oracle.forward(H, M, st.R, wl.C, st.omega, st.V, st.loss_idx, t)\n"
        "oracle.gradient(H, M, st.R, wl.C, st.omega, st.V, st.loss_idx, t)\n"
        "dt = time.perf_counter() - t0\n"
        "print(json.dumps({'value': wl.n_cfg / dt, 'threads': oracle.num_threads()}))\n") % n
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    try:
        d = json.loads(r.stdout.strip().splitlines()[-1])
    except Exception:
        return {"value": None, "error": r.stderr[-300:]}
    return {"value": d["value"], "unit": UNIT, "cores": d["threads"],
            "sample": f"{n} configurations, forward (full field) + loss + adjoint gradient, FP64, "
                      "one thread"}


# ---------------------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on the host cores
# ---------------------------------------------------------------------------------------
def run_reference(args, rank, world, local):
    if rank != 0:
        return
    import oracle
    from paper_2503_18479_gb300 import workloads as W
    oracle.build()
    wl = W.array_8x8(seed=0, n_cfg=N_CFG)
    st = wl.structures[0]
    H = oracle.basis(st.loop_vtx_off, st.vx, st.vy, st.vz, st.px, st.py, st.pz, wl.wire_radius)
    _, M = oracle.inductance(st.loop_vtx_off, st.vx, st.vy, st.vz, wl.wire_radius)
    t = wl.structure_target(0)

    def step(idx):
        oracle.forward(H, M, st.R, wl.C[idx], st.omega, st.V, st.loss_idx, t)
        oracle.gradient(H, M, st.R, wl.C[idx], st.omega, st.V, st.loss_idx, t)

    t0 = time.perf_counter()
    step(np.arange(8))
    per = (time.perf_counter() - t0) / 8
    K, Wm = args.steps, max(args.warmup, 3)
    budget = 150.0 / (K + Wm)  # whole run within a few minutes
    n = int(max(1, min(N_CFG, budget / max(per, 1e-6))))
    for i in range(Wm):
        step(np.arange(i * n, i * n + n) % N_CFG)
    t0 = time.perf_counter()
    for i in range(K):
        step(np.arange(i * n, i * n + n) % N_CFG)
    dt = time.perf_counter() - t0
    value = n * K / dt
    cores = oracle.num_threads()
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
           "steps": K, "warmup": args.warmup, "ms_per_step": dt / K * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded PCG64)",
           "config": {"workload": WORKLOAD, "sample_configs_per_step": n},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": f"{n} configurations per step, forward + loss + adjoint, FP64"},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
           "gpu_launches": 0}
    print(json.dumps(out))


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world, local)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
