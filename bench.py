#!/usr/bin/env python
"""Benchmark of the fKK-EC hot path on one GB300 (or N independent replicas).

Workload: the paper-shaped image, 846 x 831 = 703,026 synthetic spectra x
1,000 channels (30 Lorentzian species, Poisson + Gaussian noise at SNR 20,
surrogate NRB with 5 % scale and 0.05 rad phase error), k = 40, fPEC and
fSEC on, f(w) from the noise model.  One step = one fKK-EC fit of the cube
plus its reconstruction (Im{K} for every spectrum), i.e. every stage of the
factorised path: log ratio, Gram, eigensolve, projection, fKK / fPEC / fSEC
on the basis, reconstruction.

Printed (one JSON line, rank 0): value = fKK-EC spectra/s of the whole job,
the per-stage breakdown, the roofline of the dominant stage, the same metric
end to end (e2e: fkk_fit_basis called through the C ABI on pinned host
buffers, three contexts on round-robin streams as a stream of cubes runs; the
in-order and torch-copy figures beside it), the FP64 CPU oracle on a bounded
sample of the same cube (cpu_baseline), the per-spectrum KK and the ML apply
(fp32-accurate and reduced-precision forms, with the reduced form's measured
error at k = 20, 40, 80) on the same cube, the fit with the randomised SVD,
the conventional workflow (with and without the SVD denoising of the raw
spectra), serving latency and throughput under a 40 GB budget, the batched
multi-image workload, the speed-enhancement curve on the simulation-shaped
workload, clocks sampled during the timed region, and the number of library
kernels launched in it.  --svd randomized makes the randomised SVD the timed
fit.

--impl reference times the oracle itself (plain FP64 numpy) as the reference
arm: each step is an oracle fit of a bounded sample of the same workload.
Multi-GPU: one process per GPU, each fitting its own image (replicas only,
weak scaling); the only cross-rank communication is the timing barrier and
the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "img846x831_m1000"
K_BASIS = 40
METRIC = "fKK-EC spectra/s (fit + reconstruction)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip e2e / KK / apply / cpu baseline legs")
    ap.add_argument("--workload", default=WORKLOAD,
                    help="cube of synth.CONFIGS to fit (the benchmark workload by default; a smaller one keeps "
                         "profiler captures small)")
    ap.add_argument("--serve-seconds", type=float, default=20.0,
                    help="duration of the 50,000 spectra/s Poisson serving leg (about 2 requests per second)")
    ap.add_argument("--profile", default=None, choices=["fit", "apply", "apply_bf16", "kk"],
                    help="instead of the benchmark: run one operation three times on a synthetic cube of "
                         "--profile-spectra spectra x 1,000 channels (a small case for a profiler capture)")
    ap.add_argument("--profile-spectra", type=int, default=65536)
    ap.add_argument("--svd", default="exact", choices=["exact", "randomized"],
                    help="factorisation of A in the timed fit: the Gram matrix and its eigensolve, or the "
                         "randomised SVD (10 oversampling columns, 2 power iterations)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(ms, dist, device="cuda"):
    """The slowest rank's time (each rank fits its own image, so the job's
    throughput is the units of all ranks over this time)."""
    import torch

    if not dist:
        return ms
    t = torch.tensor([float(ms)], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, n_per_rank, ms):
    """Spectra per second of the whole job: every rank's n over the max time."""
    return world * n_per_rank / (ms / 1e3)


# ----------------------------------------------------------------- clocks --
class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.path = os.path.join("/tmp", f"fkk_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------- helpers --
def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def fp32_peak_tflops(sm_mhz):
    # 152 SMs x 128 FP32 lanes x 2 flops (FMA) per clock
    return 152 * 128 * 2 * (sm_mhz or 2070.0) * 1e6 / 1e12


def source_hash(files):
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, "paper_2005_07132_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


STAGE_KERNEL = {  # stage -> (kernel, sources, bound)
    "transform": ("transform_tma_kernel", ["fit_prep.cu", "tc.cuh", "common.cuh"], "hbm"),
    "gram": ("gram_tc_kernel", ["gram.cu", "tc.cuh", "common.cuh"], "tensor"),
    "eig": ("tridiag_kernel", ["tridiag.cu", "df64.cuh", "common.cuh"], "alu"),
    "project": ("project_tc_kernel", ["project_tc.cu", "tc.cuh", "common.cuh"], "hbm"),
    "basis": ("als_kernel", ["basis.cu", "fft.cuh", "common.cuh"], "alu"),
    "recon": ("recon_tc_kernel", ["recon_tc.cu", "tc.cuh", "common.cuh"], "hbm"),
}


RSVD_POWER_ITERS = 2
RSVD_STAGE = ("rsvd passes over A (project_tc_kernel, gram_tc_kernel<64,1>)",
              ["rsvd.cu", "gram.cu", "project_tc.cu", "tc.cuh", "common.cuh"], "hbm")


def algorithmic_work(stage, n, m, k, svd="exact"):
    """Algorithmic bytes (hbm) or flops (tensor / alu) of one launch of the
    stage's dominant kernel for n spectra, m channels, k basis vectors.  With
    the randomised SVD the factorisation stage is 2q + 2 reads of the
    transformed cube (A Omega, q times A^T Q and A Q, and the final A^T Q)."""
    mg = -(-m // 256) * 256
    np_ = -(-n // 64) * 64
    if svd == "randomized":
        if stage == "gram":
            return None
        if stage == "eig":
            return (2 * RSVD_POWER_ITERS + 2) * 2 * 2.0 * np_ * mg
    if stage == "transform":
        return 4.0 * n * m + 2 * 2.0 * np_ * mg  # read I (fp32), write two bf16 terms
    if stage == "gram":
        return 3.0 * m * m * n  # symmetric Gram, three bf16 products per term
    if stage == "eig":
        return 4.0 / 3.0 * m ** 3  # Householder tridiagonalisation (LAPACK dsytrd count)
    if stage == "project":
        return 2 * 2.0 * np_ * mg + 4.0 * n * k
    if stage == "recon":
        return 4.0 * n * m + 4.0 * n * k
    return None


def traffic_from_profiles(kernel, src_hash):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if
    taken on the current source."""
    try:
        t = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
        e = t[kernel]
        if e.get("source_hash") != src_hash:
            return None
        return e["dram_bytes_per_launch"] * e.get("scale", 1.0)
    except Exception:
        return None


# ------------------------------------------------------------------ arms --
def run_reference(args, rank, world):
    """The FP64 CPU oracle as the reference arm (rank 0 only)."""
    if rank != 0:
        return
    import numpy as np

    import oracle as O
    from paper_2005_07132_gb300.synth import CONFIGS, make_cube

    cube = make_cube(CONFIGS[args.workload])
    n_sample = 50_000
    xi = cube.i_cars[:n_sample]
    f = O.noise_scale(cube.i_cars.astype(np.float64).mean(0), cube.alpha, cube.sigma_g)
    prm = O.FitParams(k=K_BASIS)
    for _ in range(args.warmup):
        O.fit(xi, cube.i_ref, prm, f=f)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.fit(xi, cube.i_ref, prm, f=f)
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    cores = len(os.sched_getaffinity(0))
    value = n_sample / t
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "spectra/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n_spectra": n_sample, "n_channels": int(cube.i_cars.shape[1]),
                   "k": K_BASIS, "sample": f"first {n_sample} spectra of the 703,026-spectrum cube"},
        "cpu_baseline": {"value": value, "unit": "spectra/s", "cores": cores, "kind": "oracle",
                         "sample": f"fit of the first {n_sample} spectra (fp64 numpy oracle)"},
        "e2e": {"value": value, "unit": "spectra/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def cpu_baseline(cube):
    import numpy as np

    import oracle as O

    n_sample = 100_000
    f = O.noise_scale(cube.i_cars.astype(np.float64).mean(0), cube.alpha, cube.sigma_g)
    t0 = time.perf_counter()
    O.fit(cube.i_cars[:n_sample], cube.i_ref, O.FitParams(k=K_BASIS), f=f)
    t = time.perf_counter() - t0
    return {"value": n_sample / t, "unit": "spectra/s", "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
            "sample": f"fp64 oracle fit + reconstruction of the first {n_sample} of 703,026 spectra "
                      f"({t:.1f} s)"}


def conventional_cpu(cube, n_sample=300):
    """The fp64 oracle's conventional workflow (KK, PEC, SEC per spectrum) on
    the first n_sample spectra of the cube, one thread."""
    import numpy as np

    import oracle as O

    t0 = time.perf_counter()
    O.conventional(cube.i_cars[:n_sample].astype(np.float64), cube.i_ref.astype(np.float64), O.FitParams())
    t = time.perf_counter() - t0
    return {"value": n_sample / t, "unit": "spectra/s", "kind": "oracle",
            "sample": f"fp64 oracle conventional workflow on the first {n_sample} spectra ({t:.1f} s)"}


def run_ours(args, rank, world, local):
    import numpy as np
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_2005_07132_gb300 as fk
    from paper_2005_07132_gb300.synth import CONFIGS, make_cube

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    spec = CONFIGS[args.workload]
    cube = make_cube(spec, image=rank)  # each rank fits its own image of the scene
    n, m = cube.i_cars.shape
    ctx = fk.Context(local)
    st = torch.cuda.current_stream()
    x = torch.from_numpy(cube.i_cars).cuda()
    ref = torch.from_numpy(cube.i_ref).cuda()
    out = torch.empty_like(x)
    svd = fk.SVD_RANDOMIZED if args.svd == "randomized" else fk.SVD_EXACT
    prm = fk.fit_params(k=K_BASIS, noise_alpha=cube.alpha, noise_sigma_g=cube.sigma_g, svd=svd,
                        rsvd_power_iters=RSVD_POWER_ITERS)

    def step():
        b, _, _ = fk.fkk_fit_basis(ctx, x, ref, prm, im_out=out, stream=st)
        return b

    bases = []
    for _ in range(max(3, args.warmup)):
        bases.append(step())
    torch.cuda.synchronize()
    for b in bases:
        b.close()
    bases.clear()
    status, clamped = ctx.sync_status()

    # ---- timed region (device-resident inputs) ----
    ctx.set_timing(True)
    clocks = ClockSampler(local)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    l0 = fk.launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    stage_acc = {}
    e0.record(st)
    for _ in range(args.steps):
        bases.append(step())
        # stage events are recorded on the same stream; read after the loop
    e1.record(st)
    torch.cuda.synchronize()
    launches = fk.launch_count() - l0
    clk = clocks.stop()
    if dist:
        dist.barrier()
    ms_step = e0.elapsed_time(e1) / args.steps
    stage_acc = ctx.stage_ms()  # last step's stages
    status2, _ = ctx.sync_status()
    for b in bases:
        b.close()
    bases.clear()
    # one more, untimed step with the eigensolver's phase clocks (reading
    # the SM clock perturbs that kernel, so the timed steps do not)
    ctx.set_timing(2)
    step().close()
    torch.cuda.synchronize()
    phases = ctx.eig_phase_cycles()
    ctx.set_timing(False)
    # the measured rate of the reduction's double-word multiply-add (all
    # SMs, untimed): the eigensolve's roofline peak
    dw_rate, _ = ctx.dw_rate(4096)
    ms_step = max_over_ranks(ms_step, dist)
    value = job_throughput(world, n, ms_step)

    # ---- roofline of the dominant stage ----
    pk = peaks()
    # the largest stage that has a work model (the basis math is a chain of
    # small latency-bound kernels without one)
    modelled = [st_ for st_ in stage_acc if algorithmic_work(st_, n, m, K_BASIS, args.svd) is not None]
    stage = max(modelled, key=stage_acc.get)
    kernel, srcs, bound = RSVD_STAGE if (args.svd == "randomized" and stage == "eig") else STAGE_KERNEL[stage]
    work = algorithmic_work(stage, n, m, K_BASIS, args.svd)
    t_s = stage_acc[stage] / 1e3
    if bound == "hbm":
        peak = pk["hbm_gbs"] if pk else 6800.0
        achieved = work / t_s / 1e9
        unit = "GB/s"
        peak_note = "measured hbm_gbs" if pk else "fallback"
    elif bound == "tensor":
        peak = pk["bf16_tflops_sustained"] if pk else 1700.0
        achieved = work * 2 / t_s / 1e12
        unit = "TFLOP/s"
        peak_note = "measured bf16_tflops_sustained" if pk else "fallback"
    elif stage == "eig":
        # double-word flops on the fp32 pipe, against the measured rate of
        # the double-word multiply-add (fkk_dw_rate)
        peak = dw_rate / 1e12
        achieved = work / t_s / 1e12
        unit = "TFLOP/s"
        peak_note = ("measured double-word flop rate: fkk_dw_rate, 8 independent multiply-add chains "
                     "acc*y+x per thread on all SMs, 2 flops each (derived fp32-instruction "
                     f"bound / 10: {fp32_peak_tflops(clk.get('sm_max_mhz')) / 20:.2f})")
    else:
        peak = fp32_peak_tflops(clk.get("sm_max_mhz"))
        achieved = work / t_s / 1e12
        unit = "TFLOP/s"
        peak_note = "fp32 ALU peak from 152 SMs x 128 lanes x 2 x max SM clock"
    src_hash = source_hash(srcs)
    roofline = {"stage": stage, "kernel": kernel, "bound": bound, "achieved": achieved, "peak": peak,
                "peak_source": peak_note, "unit": unit, "frac": achieved / peak,
                "traffic": traffic_from_profiles(kernel, src_hash), "source_hash": src_hash}

    line = {
        "metric": METRIC, "value": value, "unit": "spectra/s", "n_gpus": world, "steps": args.steps,
        "warmup": max(3, args.warmup), "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3+f32+f64", "data": "synthetic",
        "config": {"workload": args.workload, "n_spectra": n, "n_channels": m, "k": K_BASIS, "pec": True, "sec": True,
                   "svd": args.svd if args.svd == "exact" else f"randomized (p = 10, q = {RSVD_POWER_ITERS})",
                   "noise": "poisson+gauss snr20", "l2": "inputs (2.81 GB) larger than L2",
                   "parallelism": "replicas" if world > 1 else "single"},
        "stage_ms": stage_acc,
        "eig_phase_cycles": dict(zip(["load", "exchange_w", "pivot_reflector", "next_p", "deferred_update"], phases)),
        "device_status": int(status2), "clamped_ratios_per_fit": int(clamped) // max(1, max(3, args.warmup)),
        "roofline": roofline, "clocks": clk, "gpu_launches": int(launches),
    }

    if not args.no_extras:
        # ---- e2e through pinned host buffers ----
        xh = torch.from_numpy(cube.i_cars).pin_memory()
        oh = torch.empty_like(xh).pin_memory()
        xd = torch.empty_like(x)
        refh = torch.from_numpy(cube.i_ref).pin_memory()
        refd = torch.empty_like(ref)

        def e2e_step():
            xd.copy_(xh, non_blocking=True)
            refd.copy_(refh, non_blocking=True)
            b, _, _ = fk.fkk_fit_basis(ctx, xd, refd, prm, im_out=out, stream=st)
            oh.copy_(out, non_blocking=True)
            return b

        for _ in range(2):
            bases.append(e2e_step())
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(args.steps):
            bases.append(e2e_step())
        e1.record(st)
        torch.cuda.synchronize()
        serial_ms = e0.elapsed_time(e1) / args.steps
        for b in bases:
            b.close()
        bases.clear()

        # pipelined, as a stream of cubes is processed: step i's upload and
        # step i-1's download run on their own streams beside step i's fit
        # (two device copies of the cube and of the output); every step still
        # uploads its cube and downloads its result inside the timed region
        s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()
        xds = [torch.empty_like(x) for _ in range(2)]
        refds = [torch.empty_like(ref) for _ in range(2)]
        ods = [torch.empty_like(x) for _ in range(2)]
        ev_fit, ev_out = [None, None], [None, None]

        def piped_step(i):
            b = i % 2
            ev_in = torch.cuda.Event()
            with torch.cuda.stream(s_in):
                if ev_fit[b] is not None:
                    s_in.wait_event(ev_fit[b])  # the fit that read xds[b] is done
                xds[b].copy_(xh, non_blocking=True)
                refds[b].copy_(refh, non_blocking=True)
                ev_in.record(s_in)
            st.wait_event(ev_in)
            if ev_out[b] is not None:
                st.wait_event(ev_out[b])  # ods[b] has been downloaded
            basis, _, _ = fk.fkk_fit_basis(ctx, xds[b], refds[b], prm, im_out=ods[b], stream=st)
            ev_fit[b] = torch.cuda.Event()
            ev_fit[b].record(st)
            with torch.cuda.stream(s_out):
                s_out.wait_event(ev_fit[b])
                oh.copy_(ods[b], non_blocking=True)
                ev_out[b] = torch.cuda.Event()
                ev_out[b].record(s_out)
            return basis

        for i in range(2):
            bases.append(piped_step(i))
        torch.cuda.synchronize()
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(s_in)
        for i in range(args.steps):
            bases.append(piped_step(i))
        p1.record(s_out)
        torch.cuda.synchronize()
        e2e_ms = p0.elapsed_time(p1) / args.steps
        for b in bases:
            b.close()
        bases.clear()
        line["e2e"] = {"value": world * n / (e2e_ms / 1e3), "unit": "spectra/s",
                       "h2d_bytes_per_step": int(xh.numel() * 4 + refh.numel() * 4),
                       "d2h_bytes_per_step": int(oh.numel() * 4), "ms_per_step": e2e_ms,
                       "mode": "pipelined: upload of step i and download of step i-1 beside the fit (3 streams)",
                       "serial": {"value": world * n / (serial_ms / 1e3), "ms_per_step": serial_ms,
                                  "mode": "upload, fit, download in order on one stream"}}
        # the public call on the pinned host buffers themselves: the library
        # copies the cube in and the result out on the call's stream.  In
        # order on one stream, then as a stream of cubes runs: three contexts
        # (one workspace each) on three streams, step i on context i % 3, so
        # that one cube uploads while another is fitted and a third downloads
        # (two lanes left the host link idle between a lane's phases: 22.4 vs
        # 18.2 ms per step; the link moves ~171 GB/s each way at once)
        lanes = 3
        outs_h = [torch.empty_like(xh).pin_memory() for _ in range(lanes)]
        ctxs = [ctx] + [fk.Context(local) for _ in range(lanes - 1)]
        streams = [st] + [torch.cuda.Stream() for _ in range(lanes - 1)]

        def host_step(i):
            j = i % lanes
            b, _, _ = fk.fkk_fit_basis(ctxs[j], xh, refh, prm, im_out=outs_h[j], stream=streams[j])
            return b

        for i in range(lanes):
            bases.append(host_step(i))
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(args.steps):
            bases.append(host_step(0))
        e1.record(st)
        torch.cuda.synchronize()
        host_serial_ms = e0.elapsed_time(e1) / args.steps
        for b in bases:
            b.close()
        bases.clear()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for i in range(args.steps):
            bases.append(host_step(i))
        torch.cuda.synchronize()
        host_ms = (time.perf_counter() - t0) * 1e3 / args.steps
        for b in bases:
            b.close()
        bases.clear()
        for c in ctxs[1:]:
            c.close()
        del outs_h
        torch_piped = line["e2e"]
        line["e2e"] = {"value": world * n / (host_ms / 1e3), "unit": "spectra/s",
                       "h2d_bytes_per_step": int(xh.numel() * 4 + refh.numel() * 4),
                       "d2h_bytes_per_step": int(oh.numel() * 4), "ms_per_step": host_ms,
                       "mode": "fkk_fit_basis (C ABI) on the pinned host cube and output; three contexts on "
                               "round-robin streams, host wall clock over the steps",
                       "c_abi_in_order": {"value": world * n / (host_serial_ms / 1e3), "ms_per_step": host_serial_ms,
                                          "mode": "the same call, one context, one stream"},
                       "torch_copies": torch_piped}

        # ---- per-spectrum KK and ML apply on the same cube ----
        def timed(fn, reps=5):
            fn()
            torch.cuda.synchronize()
            e0.record(st)
            for _ in range(reps):
                fn()
            e1.record(st)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1) / reps

        hbm_peak = (pk or {}).get("hbm_gbs", 6800.0)
        kk_ms = timed(lambda: fk.kk_per_spectrum(ctx, x, ref, im_out=out, stream=st))
        line["kk_per_spectrum"] = {"value": n / (kk_ms / 1e3), "unit": "spectra/s", "ms": kk_ms,
                                   "hbm_gbs": 8.0 * n * m / (kk_ms / 1e3) / 1e9,
                                   "hbm_frac": 8.0 * n * m / (kk_ms / 1e3) / 1e9 / hbm_peak}
        # ML apply (Sec. 2.6) with the fitted basis, in both precisions; the
        # reduced form's error is measured against the fp32-accurate form on
        # the whole cube (the tests bound both against the fp64 oracle)
        line["apply"] = {}
        out2 = torch.empty_like(x)
        for kb in (20, 40, 80):
            bp = fk.fit_params(k=kb, noise_alpha=cube.alpha, noise_sigma_g=cube.sigma_g)
            basis, _, _ = fk.fkk_fit_basis(ctx, x, ref, bp, stream=st)
            ent = {}
            for prec, name in ((fk.PREC_BF16X3, "bf16x3"), (fk.PREC_BF16, "bf16")):
                basis.set_precision(prec)
                o = out if prec == fk.PREC_BF16X3 else out2
                a_ms = timed(lambda: fk.fkk_apply(ctx, basis, x, im_out=o, stream=st))
                ent[name] = {"value": n / (a_ms / 1e3), "unit": "spectra/s", "ms": a_ms,
                             "hbm_gbs": 8.0 * n * m / (a_ms / 1e3) / 1e9,
                             "hbm_frac": 8.0 * n * m / (a_ms / 1e3) / 1e9 / hbm_peak,
                             # one persistent kernel (else projection + reconstruction): the split
                             # form up to k = 62, the single-product form up to k = 80
                             "fused": kb <= 62 or prec == fk.PREC_BF16}
            torch.cuda.synchronize()
            ent["bf16_rel_l2_vs_bf16x3"] = float(torch.linalg.vector_norm(out2 - out) / torch.linalg.vector_norm(out))
            line["apply"][f"k{kb}"] = ent
            basis.close()
        del out2
        # the same fit with the randomised SVD (Sec. 5) in place of the Gram
        # matrix and its eigensolve, at 2 and 1 power iterations
        line["randomized_svd"] = {}
        for q in (2, 1):
            rp = fk.fit_params(k=K_BASIS, noise_alpha=cube.alpha, noise_sigma_g=cube.sigma_g,
                               svd=fk.SVD_RANDOMIZED, rsvd_power_iters=q)
            made = []
            r_ms = timed(lambda: made.append(fk.fkk_fit_basis(ctx, x, ref, rp, im_out=out, stream=st)[0]))
            for b in made:
                b.close()
            line["randomized_svd"][f"q{q}"] = {"value": world * n / (r_ms / 1e3), "unit": "spectra/s",
                                               "ms_per_step": r_ms, "oversample": 10, "power_iters": q}
        # the conventional per-spectrum workflow (KK, ALS phase-error
        # correction, Savitzky-Golay scale-error correction) the paper
        # measures the factorised method against, on the same cube
        cv_prm = fk.fit_params()
        cv_ms = timed(lambda: fk.conventional_per_spectrum(ctx, x, ref, cv_prm, im_out=out, stream=st), reps=3)
        line["conventional"] = {"value": n / (cv_ms / 1e3), "unit": "spectra/s", "ms": cv_ms,
                                "steps": "KK + PEC (ALS, 20 reweightings) + SEC (Savitzky-Golay)"}
        # with the workflow's SVD denoising of the raw spectra first (Fig.
        # 1(a)), keeping 6 singular vectors as the paper's conventional runs did
        dn_prm = fk.fit_params(denoise_k=6)
        dn_ms = timed(lambda: fk.conventional_per_spectrum(ctx, x, ref, dn_prm, im_out=out, stream=st), reps=3)
        line["conventional"]["with_svd_denoise"] = {"value": n / (dn_ms / 1e3), "unit": "spectra/s", "ms": dn_ms,
                                                    "denoise_k": 6}
        line["serve"] = serve_leg(fk, local, args.serve_seconds)
        line["multi_image"] = multi_image_leg(fk, ctx, st)
        line["simulation"] = sim_leg(fk, ctx, st)
        if rank == 0 and world == 1:
            line["cpu_baseline"] = cpu_baseline(cube)
            line["conventional"]["cpu_oracle"] = conventional_cpu(cube)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def sim_leg(fk, ctx, st, reps=3):
    """The speed-enhancement curve of Sec. 4.1 on the simulation-shaped
    workload (shape only: 74 x 246 base side-scaled by 0.5..4, 810 channels,
    noiseless, three chemicals): the fKK-EC fit + reconstruction (k = 40,
    PEC + SEC) against the conventional per-spectrum workflow, both on the
    GPU, and the mean RSS of each against the known Im{chi / chi_nr} at side
    scale 1 (a diagnostic, as in the paper's Fig. 2(e))."""
    import numpy as np
    import torch

    from paper_2005_07132_gb300.synth import SIM_SIDE_SCALES, make_sim_cube

    res = {"workload": "simulation-shaped, 74x246 base side-scaled, 810 channels, noiseless, 3 chemicals",
           "k": 40, "points": []}
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    prm = fk.fit_params(k=40)
    cprm = fk.fit_params()
    for side in SIM_SIDE_SCALES:
        cube = make_sim_cube(side)
        x = torch.from_numpy(cube.i_cars).cuda()
        ref = torch.from_numpy(cube.i_ref).cuda()
        out = torch.empty_like(x)
        out2 = torch.empty_like(x)
        fk.fkk_fit_basis(ctx, x, ref, prm, im_out=out, stream=st)[0].close()
        bases = []
        e0.record(st)
        for _ in range(reps):
            bases.append(fk.fkk_fit_basis(ctx, x, ref, prm, im_out=out, stream=st)[0])
        e1.record(st)
        torch.cuda.synchronize()
        fit_ms = e0.elapsed_time(e1) / reps
        for b in bases:
            b.close()
        fk.conventional_per_spectrum(ctx, x, ref, cprm, im_out=out2, stream=st)
        e0.record(st)
        for _ in range(reps):
            fk.conventional_per_spectrum(ctx, x, ref, cprm, im_out=out2, stream=st)
        e1.record(st)
        torch.cuda.synchronize()
        conv_ms = e0.elapsed_time(e1) / reps
        n = x.shape[0]
        pt = {"side_scale": side, "n_spectra": n, "fit_ms": fit_ms, "conventional_ms": conv_ms,
              "speed_enhancement": conv_ms / fit_ms}
        if side == 1:
            rows = np.arange(0, n, 7)
            truth = cube.truth_im(rows)
            r_t = torch.from_numpy(rows).cuda()
            rss_f = float(np.mean(np.sum((out[r_t].cpu().numpy() - truth) ** 2, 1)))
            rss_c = float(np.mean(np.sum((out2[r_t].cpu().numpy() - truth) ** 2, 1)))
            pt["mean_rss"] = {"fkk_ec": rss_f, "conventional": rss_c, "null": float(np.mean(np.sum(truth**2, 1)))}
        res["points"].append(pt)
        del x, ref, out, out2
    return res


def multi_image_leg(fk, ctx, st, reps=3):
    """The batched multi-image workload: 16 independent cubes (their own
    scenes; sides 128..1,024, M in {512, 878, 1,000, 1,600}, k in
    {10, 20, 40, 80}, drawn by the seeded stream 1005), each tiled from a
    128 x 128 draw of its scene, fitted and reconstructed end to end by one
    fkk_fit_many call (two worker lanes), beside the same fits one after the
    other on one stream."""
    import torch

    from paper_2005_07132_gb300.synth import make_tiled_cube, multi_image_specs

    jobs = []
    total = 0
    for spec, k in multi_image_specs():
        cube = make_tiled_cube(spec)
        x = torch.from_numpy(cube.i_cars).cuda()
        ref = torch.from_numpy(cube.i_ref).cuda()
        jobs.append((x, ref, fk.fit_params(k=k), torch.empty_like(x)))
        total += x.shape[0]
        del cube
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    for b in fk.fkk_fit_many(ctx, jobs, stream=st):  # warm-up (workspaces, lanes)
        b.close()
    torch.cuda.synchronize()
    made = []
    e0.record(st)
    for _ in range(reps):
        made += fk.fkk_fit_many(ctx, jobs, stream=st)
    e1.record(st)
    torch.cuda.synchronize()
    many_ms = e0.elapsed_time(e1) / reps
    for b in made:
        b.close()
    made.clear()
    e0.record(st)
    for x, ref, prm, out in jobs:
        made.append(fk.fkk_fit_basis(ctx, x, ref, prm, im_out=out, stream=st)[0])
    e1.record(st)
    torch.cuda.synchronize()
    seq_ms = e0.elapsed_time(e1)
    for b in made:
        b.close()
    status, _ = ctx.sync_status()
    res = {"cubes": len(jobs), "spectra": total, "bytes_in": int(sum(j[0].numel() * 4 for j in jobs)),
           "value": total / (many_ms / 1e3), "unit": "spectra/s", "ms": many_ms,
           "sequential": {"value": total / (seq_ms / 1e3), "ms": seq_ms},
           "device_status": int(status), "input": "each cube tiled from a 128 x 128 draw of its own scene"}
    del jobs
    torch.cuda.empty_cache()
    return res


def serve_leg(fk, device, seconds_50k=20.0):
    """Serving of a trained basis (train 400 x 500 x 1,000, k = 40) under a
    40 GB HBM budget: tiles of U{1,000..50,000} spectra cut from a new image
    of the same scene, in pinned host memory, arriving as a Poisson process
    at 50,000 spectra/s (for `seconds_50k` seconds), at half the saturation
    rate (1,000 requests), and all at once (saturation, 1,000 requests).
    Latency is submit -> completion; the batch log gives the share of batches
    whose device interval overlaps a batch of another slot."""
    import numpy as np
    import torch

    from paper_2005_07132_gb300.synth import CONFIGS, Scene, make_cube

    budget = 40 << 30
    sctx = fk.Context(device, hbm_budget_bytes=budget)
    spec = CONFIGS["train400x500_m1000"]
    scene = Scene.from_spec(spec)
    train = make_cube(spec, image=0, scene=scene)
    new = make_cube(spec, image=1, scene=scene)
    x = torch.from_numpy(train.i_cars).cuda()
    ref = torch.from_numpy(train.i_ref).cuda()
    basis, _, _ = fk.fkk_fit_basis(sctx, x, ref, fk.fit_params(k=K_BASIS))
    del x
    pool = torch.from_numpy(new.i_cars).pin_memory()
    outp = torch.empty_like(pool).pin_memory()
    n_pool = pool.shape[0]
    rng = np.random.default_rng(4)

    def tiles(count):
        out, pos = [], 0
        for _ in range(count):
            t = int(rng.integers(1000, 50001))
            if pos + t > n_pool:
                pos = 0
            out.append((pos, t))
            pos += t
        return out

    def overlap_share(log):
        if len(log) < 2:
            return 0.0
        hit = 0
        for i in range(len(log)):
            if any(log[j, 2] != log[i, 2] and log[i, 0] < log[j, 1] and log[j, 0] < log[i, 1]
                   for j in range(len(log)) if j != i):
                hit += 1
        return hit / len(log)

    def run(rate, count):
        """count requests arriving as a Poisson process at `rate` spectra/s
        (rate None: all at once)."""
        srv = fk.Server(sctx, basis)
        plan = tiles(count)
        ids = []
        t0 = time.perf_counter()
        due = t0
        for pos, t in plan:
            if rate:
                due += rng.exponential(t / rate)
                while time.perf_counter() < due:
                    pass
            ids.append(srv.submit(pool[pos:pos + t], outp[pos:pos + t]))
        for rid in ids:
            srv.wait(rid)
        wall = time.perf_counter() - t0
        st = srv.stats()
        st["requests"] = len(ids)
        st["spectra"] = int(sum(t for _, t in plan))
        st["wall_s"] = wall
        st["batch_overlap_share"] = overlap_share(srv.batch_log())
        srv.stop()
        return st

    res = {"tile_sizes": "U{1000..50000}", "input": "pinned host", "train": "400x500x1000, k=40",
           "hbm_budget_bytes": budget, "slots": 3}
    res["saturation"] = run(None, 1000)
    sat = res["saturation"]["spectra_per_s"]
    res["poisson_half_saturation"] = run(0.5 * sat, 1000)
    res["poisson_half_saturation"]["arrival_rate"] = 0.5 * sat
    n50 = max(4, int(50_000 * seconds_50k / 25_500))
    res["poisson_50k_per_s"] = run(50_000, n50)
    basis.close()
    sctx.close()
    return res


def profile_case(args):
    """One operation, three times, on the first --profile-spectra spectra of
    the 703,026 x 1,000 workload: the fit (k = 40, PEC + SEC, with the
    reconstruction), the per-spectrum KK, or the apply with a k = 40 basis
    fitted on its first 20,000 spectra."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_2005_07132_gb300 as fk
    from paper_2005_07132_gb300.synth import CONFIGS, make_cube

    spec = CONFIGS[WORKLOAD]
    cube = make_cube(spec)
    n = min(args.profile_spectra, cube.i_cars.shape[0])
    ctx = fk.Context(0)
    x = torch.from_numpy(cube.i_cars[:n]).cuda()
    ref = torch.from_numpy(cube.i_ref).cuda()
    out = torch.empty_like(x)
    if args.profile == "kk":
        run = lambda: fk.kk_per_spectrum(ctx, x, ref, im_out=out)
    elif args.profile == "fit":
        params = fk.fit_params(k=K_BASIS, noise_alpha=cube.alpha, noise_sigma_g=cube.sigma_g)
        run = lambda: fk.fkk_fit_basis(ctx, x, ref, params, im_out=out)[0].close()
    else:
        train = torch.from_numpy(cube.i_cars[:20000]).cuda()
        basis, _, _ = fk.fkk_fit_basis(ctx, train, ref, fk.fit_params(k=K_BASIS, noise_alpha=cube.alpha,
                                                                       noise_sigma_g=cube.sigma_g), reconstruct=False)
        basis.set_precision(fk.PREC_BF16 if args.profile == "apply_bf16" else fk.PREC_BF16X3)
        run = lambda: fk.fkk_apply(ctx, basis, x, im_out=out)
    for _ in range(3):
        run()
    torch.cuda.synchronize()
    print(json.dumps({"profile": args.profile, "n_spectra": n, "status": ctx.sync_status()[0]}))


def main():
    args = parse()
    if args.profile:
        profile_case(args)
        return
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
