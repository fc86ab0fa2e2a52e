#!/usr/bin/env python
"""Benchmark of the Elfpie gradient step on GB300.

One step = one outer iteration of Algorithm 1 over all K LEDs (every kernel of
the iteration: tile kernel, Hessian branch, Eq. 9 gather + Eq. 19 update, Eq. 18
pupil gradient and update, FP64 costs).  Metric: LED sub-image updates/s
(K x iterations / s).  Default workload: 15x15 LEDs, 256x256 images, 1024x1024
spectrum, mixed corruptions (seeded synthetic data).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun each rank runs an independent
replica of the workload (the per-problem path does not shard); value = the units
of all ranks / the max over ranks of the timed region.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import threading
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from paper_2209_14671_gb300 import inputs as IN  # noqa: E402

METRIC = "LED sub-image updates/s (K×iters/s) at fixed error vs FP64 oracle; p99 latency"
UNIT = "LED sub-image updates/s"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_PATH = os.path.join(ROOT, "profiles", "tile_stage_traffic.json")
TILE_SOURCES = ["paper_2209_14671_gb300/csrc/tile_split.cu", "paper_2209_14671_gb300/csrc/fft.cuh",
                "paper_2209_14671_gb300/csrc/reduce.cuh"]
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU work of the one-core oracle sample")
    ap.add_argument("--check-iters", type=int, default=100,
                    help="iterations of the error check against the FP64 oracle (also the all-cores oracle timing)")
    ap.add_argument("--no-precision", action="store_true", help="skip the tensor-core precision leg")
    ap.add_argument("--no-fidelity", action="store_true", help="skip the fidelity-variant leg")
    ap.add_argument("--no-mux", action="store_true", help="skip the multiplexed-illumination leg")
    ap.add_argument("--no-eval", action="store_true", help="skip the evaluation leg (Eqs. 20-22)")
    ap.add_argument("--no-workloads", action="store_true", help="skip the other-workload throughput leg")
    ap.add_argument("--serving-requests", type=int, default=2000,
                    help="requests of the mixed serving stream (0 disables the serving leg)")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))


def max_over_ranks(value: float, world: int, device) -> float:
    """The slowest rank's time (the job's time when every rank runs its own replica)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def tile_sources_hash() -> str:
    h = hashlib.sha256()
    for p in TILE_SOURCES:
        h.update(open(os.path.join(ROOT, p), "rb").read())
    return h.hexdigest()[:16]


def tile_flops_per_led(n: int) -> float:
    """Algorithmic FLOPs of one LED's tile work: the inverse and forward n x n 2D FFTs at the
    conventional 5 B log2 B each (B = n^2, unpruned) plus ~40 FLOP per pixel of pointwise work
    (crop x pupil, residual, gradient, normaliser, divergence, W)."""
    B = n * n
    return 2 * 5.0 * B * math.log2(B) + 40.0 * B


def fp32_nominal_tflops(sms: int, sm_mhz):
    """FP32 CUDA-core nominal peak: SMs x 128 FP32 lanes x 2 FLOP per FMA x the maximum SM clock
    (context for the measured figure)."""
    mhz = float(sm_mhz) if sm_mhz else 2070.0
    return sms * 128 * 2 * mhz * 1e6 / 1e12


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo) and its logical core count."""
    name = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                name = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not name and os.path.exists("/proc/cpuinfo"):
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                name = line.split(":", 1)[1].strip()
                break
    return f"{name or 'unknown'} ({os.cpu_count()} logical cores)"


def peaks():
    if os.path.exists(PEAKS_PATH):
        d = json.load(open(PEAKS_PATH))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms.  Reported: the samples read from one
    period before start() to one period after stop(), i.e. the timed region and the warm-up steps
    just before it (a short region can fall between two samples)."""

    PERIOD_S = 0.2
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        self.lines = []  # (host time when read, line)
        self.t_start = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.reader = threading.Thread(target=self._read, daemon=True)
        self.reader.start()
        t0 = time.perf_counter()  # the sampler is live (first line read) before the timed region
        while not self.lines and time.perf_counter() - t0 < 10.0 and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line))

    def start(self):
        self.t_start = time.perf_counter()

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        t_end = time.perf_counter()
        time.sleep(self.PERIOD_S)  # the sample after the region
        self.proc.terminate()
        try:
            self.proc.wait(timeout=10)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.reader.join(timeout=10)
        t0 = self.t_start if self.t_start is not None else -float("inf")
        window = [ln for t, ln in self.lines if t0 - self.PERIOD_S <= t <= t_end + self.PERIOD_S]
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in window:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "timed_region_s": round(t_end - t0, 4) if self.t_start is not None else None,
                "reasons": sorted(reasons)}


def oracle_error_check(I_host: np.ndarray, w: dict, elf_factory, iters: int):
    """The metric's fixed-error condition, measured in the benchmark run itself, and the
    all-cores oracle rate: the FP64 oracle (LED blocks over a process pool, oracle/parallel.py)
    runs `iters` iterations of the workload from its own state after 3 iterations (rounded to
    FP32), timed; the CUDA path runs the same iterations from the same state through the C ABI
    in the benchmarked launch configuration (elf_step, 8-iteration graphs); relative L2 of the
    final Psi, P and object and the largest relative difference of the per-iteration costs."""
    import oracle as O  # the CPU baseline legs are the only product-side users of the oracle
    from oracle.parallel import ParallelOracle
    geo = O.make_geometry(w["n"], w["u"], w["k_xy"], w["na"], w["wavelength_um"], w["pixel_um"])
    opt = O.Options()
    I = I_host.astype(np.float64)

    def rel(a, b):
        return float(np.linalg.norm((np.asarray(a) - np.asarray(b)).ravel()) / np.linalg.norm(np.asarray(b).ravel()))
    with ParallelOracle(geo, I) as po:
        st = O.init_state(I, geo, w["k_xy"], opt)
        st, _ = po.run(st, opt, 3)
        for k in ("psi", "mu_psi", "pupil", "mu_p"):
            setattr(st, k, getattr(st, k).astype(np.complex64).astype(np.complex128))
        for k in ("v_psi", "delta_psi", "v_p", "delta_p"):
            setattr(st, k, getattr(st, k).astype(np.float32).astype(np.float64))
        t0 = time.perf_counter()
        ref, costs_ref = po.run(st, opt, iters)
        el = time.perf_counter() - t0
        cores = po.cores
    with elf_factory() as elf:
        elf.set_measurements(I_host)
        elf.set_state(st.psi, st.mu_psi, st.v_psi, st.delta_psi, st.pupil, st.mu_p, st.v_p, st.delta_p, st.t,
                      st.alpha, st.beta)
        elf.step(iters)
        out = elf.get_state()
        obj = elf.get_object()
        costs = elf.get_costs()[-iters:]
    ce = np.abs(costs - costs_ref) / np.abs(costs_ref)
    err = {"run": f"{iters} iterations from the FP64 oracle's state after 3 iterations (rounded to FP32), "
                  "elf_step in 8-iteration graphs",
           "psi": rel(out["psi"], ref.psi), "pupil": rel(out["pupil"], ref.pupil),
           "object": rel(obj, O.object_from_spectrum(ref.psi)),
           "costs_max_rel": {"L_fid": float(ce[:, 0].max()), "L_A": float(ce[:, 1].max()),
                             "L_Phi": float(ce[:, 2].max())},
           "bound": 1e-4}
    rate = geo.K * iters / el
    return err, rate, cores, el


def oracle_sample_rate(I_host: np.ndarray, w: dict, seconds: float):
    """FP64 oracle iterations of the same workload on the host cores, bounded to ~`seconds`."""
    import oracle as O  # the CPU baseline legs are the only product-side users of the oracle
    geo = O.make_geometry(w["n"], w["u"], w["k_xy"], w["na"], w["wavelength_um"], w["pixel_um"])
    opt = O.Options()
    I = I_host.astype(np.float64)
    st = O.init_state(I, geo, w["k_xy"], opt)
    t0 = time.perf_counter()
    its = 0
    while True:
        st, _, _ = O.iteration(st, I, geo, opt)
        its += 1
        el = time.perf_counter() - t0
        if el >= seconds or its >= 50:
            break
    return geo.K * its / el, its, el


def make_inputs(w: dict, wid: int, torch, dev):
    """Measurements of the workload: the GPU forward model (elf_simulate) at the true LED
    positions, then the seeded degradations of the workload's recipe."""
    from paper_2209_14671_gb300 import elfpie as E
    obj = torch.from_numpy(IN.object_field(wid, w).astype(np.complex64)).to(dev)
    with E.Elf(w["n"], w["u"], w["k_xy_true"], w["na"], w["wavelength_um"], w["pixel_um"]) as sim:
        I_clean = torch.empty((w["K"], w["n"], w["n"]), dtype=torch.float32, device=dev)
        sim.simulate(obj, I_clean)
    return IN.corrupt(I_clean.cpu().numpy(), wid, w)


def serving_leg(args, torch, dev):
    """Continuous-batching server on a Poisson stream of mixed reconstructions.

    Requests: low-res side n in {64, 128, 256} x LED grid {7, 11, 15} (K = 49, 121, 225),
    uniform mix, 50 iterations each, workload-0 optics, FP32, 150 GB device budget.
    Arrivals: Poisson at 0.8 x the one-at-a-time capacity measured on the same mix.
    Also a saturated run (all requests at t = 0) for throughput against the serial path."""
    from paper_2209_14671_gb300 import elfpie as E
    from paper_2209_14671_gb300 import serve as SV
    R = args.serving_requests
    classes = [(n, g) for n in (64, 128, 256) for g in (7, 11, 15)]
    pool = {}
    for ci, (n, g) in enumerate(classes):
        w = IN.problem(0, grid=g, n=n)
        sets = []
        for v in range(2):
            obj = torch.from_numpy(IN.object_field(100 + 10 * ci + v, w).astype(np.complex64)).to(dev)
            with E.Elf(n, w["u"], w["k_xy_true"], w["na"], w["wavelength_um"], w["pixel_um"]) as sim:
                Ic = torch.empty((w["K"], n, n), dtype=torch.float32, device=dev)
                sim.simulate(obj, Ic)
            I = IN.corrupt(Ic.cpu().numpy(), 0, w)
            sets.append(torch.from_numpy(I).pin_memory().numpy())
        pool[(n, g)] = (w, sets)
    rng = IN.rng(4, IN.STREAM_ARRIVALS)
    picks = rng.integers(0, len(classes), size=R)
    reqs = []
    for i, ci in enumerate(picks):
        w, sets = pool[classes[ci]]
        reqs.append(dict(n=w["n"], u=w["u"], k_xy=w["k_xy"].astype(np.float32), na=w["na"], wl=w["wavelength_um"],
                         dx=w["pixel_um"], I=sets[i % 2], n_iter=50))
    # warm-up: every shape once through both paths (handle creation, graph capture)
    first = [reqs[list(picks).index(c)] for c in sorted(set(picks.tolist()))]
    SV.run_serial(first)
    budget = 150 << 30
    with SV.Server(budget, max_active=32) as srv:
        SV.run_stream(srv, first, np.zeros(len(first)))
        serial_t, serial_total, _ = SV.run_serial(reqs)
        cap = R / serial_total
        gaps = rng.exponential(1.0 / (0.8 * cap), size=R)
        arrivals = np.cumsum(gaps) - gaps[0]
        lat, makespan, _ = SV.run_stream(srv, reqs, arrivals)
        _, sat_makespan, _ = SV.run_stream(srv, reqs, np.zeros(R))
        st = srv.stats()
    return {"requests": R, "mix": "n in {64,128,256} x K in {49,121,225}, 50 iterations each",
            "arrival_rate_per_s": 0.8 * cap, "p50_ms": float(np.percentile(lat, 50) * 1e3),
            "p99_ms": float(np.percentile(lat, 99) * 1e3), "tiles_per_s_at_load": R / makespan,
            "saturated_tiles_per_s": R / sat_makespan, "serial_tiles_per_s": cap,
            "saturated_speedup_vs_serial": (R / sat_makespan) / cap,
            "serial_p50_ms": float(np.percentile(serial_t, 50) * 1e3),
            "handles_created": st["handles_created"], "device_bytes": st["used_bytes"],
            "budget_bytes": budget}


def precision_leg(torch, dev):
    """Tensor-core tile transforms (BF16 3-term split, FP32 accumulation) against the FP32
    FFT path on the 128 x 128 / 225-LED / 512 x 512 workload: time per iteration, tile
    stage time, achieved tensor FLOP/s of the tile GEMMs, and the relative L2 difference
    of the two paths' spectra after 20 iterations from the same initial state."""
    from paper_2209_14671_gb300 import elfpie as E
    w = IN.problem(3)
    I_dev = torch.from_numpy(make_inputs(w, 3, torch, dev)).to(dev)
    stream = torch.cuda.current_stream(dev)
    res = {}
    psi = {}
    for td in (0, 1):
        elf = E.Elf(w["n"], w["u"], w["k_xy"], w["na"], w["wavelength_um"], w["pixel_um"],
                    options=dict(tile_dft=td), stream=stream)
        elf.set_measurements(I_dev)
        elf.step(20)
        psi[td] = elf.get_spectrum()
        elf.set_tracing(True)
        for _ in range(3):
            elf.step(1)
        t_it, t_tile = [], []
        for _ in range(10):
            elf.step(1)
            st = elf.stage_times()
            t_it.append(st["iteration"])
            t_tile.append(st["tile"])
        res[td] = (float(np.median(t_it)), float(np.median(t_tile)))
        elf.close()
    # tile GEMM work per LED as executed (M = 128, three BF16 products per real product):
    # 2 M N K over gemm 1 (two A, N = 64, K = 3 x 128), gemm 2 (N = 256, K = 3 x 128),
    # gemm 3 (two A, N = 128, K = 3 x 256) and gemm 4 (N = 128, K = 3 x 256)
    flop = w["K"] * 2 * 128 * (2 * 64 * 384 + 256 * 384 + 2 * 128 * 768 + 128 * 768)
    diff = float(np.linalg.norm(psi[1] - psi[0]) / np.linalg.norm(psi[0]))
    return {"workload": w["name"], "fp32_fft_ms_per_iter": res[0][0], "tensor_core_ms_per_iter": res[1][0],
            "fp32_fft_tile_ms": res[0][1], "tensor_core_tile_ms": res[1][1],
            "speedup_iteration": res[0][0] / res[1][0], "speedup_tile": res[0][1] / res[1][1],
            "tile_gemm_tflops": flop / (res[1][1] * 1e-3) / 1e12,
            "rel_l2_psi_tc_vs_fp32_after_20_iterations": diff,
            "note": "error vs the FP64 oracle: tests/test_gpu_precision.py"}


def fidelity_leg(w, I_dev, torch, dev):
    """The four fidelities on the benchmark workload (same measurements, same initial state):
    intensity (Eq. 5), amplitude (Eq. 4) and the Sec. 6.3 maps g(x) = x^0.375 and ln(x + 1).
    Median tile-kernel and iteration times over 10 traced steps after 3 warm-up steps."""
    from paper_2209_14671_gb300 import elfpie as E
    stream = torch.cuda.current_stream(dev)
    variants = [("intensity (Eq. 5)", dict(fidelity=0)), ("amplitude (Eq. 4)", dict(fidelity=1)),
                ("power x^0.375 (Sec. 6.3)", dict(fidelity=2, g_exponent=0.375)),
                ("log ln(x+1) (Sec. 6.3)", dict(fidelity=3))]
    out = {}
    for name, opts in variants:
        elf = E.Elf(w["n"], w["u"], w["k_xy"], w["na"], w["wavelength_um"], w["pixel_um"], options=opts,
                    stream=stream)
        elf.set_measurements(I_dev)
        elf.set_tracing(True)
        for _ in range(3):
            elf.step(1)
        t_it, t_tile = [], []
        for _ in range(10):
            elf.step(1)
            st = elf.stage_times()
            t_it.append(st["iteration"])
            t_tile.append(st["tile"])
        elf.close()
        out[name] = {"tile_ms": float(np.median(t_tile)), "iteration_ms": float(np.median(t_it)),
                     "led_updates_per_s": w["K"] / (float(np.median(t_it)) * 1e-3)}
    return {"workload": w["name"], "variants": out,
            "note": "traced steps (CUDA events inside the graph); parity: tests/test_gpu_parity.py"}


def mux_leg(wid, w, obj_dev, torch, dev):
    """Multiplexed illumination (Eq. 1): the benchmark workload's 225 LEDs lit 5 at a time
    (45 images, LEDs 5j .. 5j+4 per image), measurements from the GPU's multiplexed forward
    model plus the workload's seeded Gaussian noise level of 1e-3.  Median iteration and tile
    stage (|o|^2 pass, per-image residual and normaliser, W = o f pass) over 10 traced steps."""
    from paper_2209_14671_gb300 import elfpie as E
    M = 5
    stream = torch.cuda.current_stream(dev)
    elf = E.Elf(w["n"], w["u"], w["k_xy"], w["na"], w["wavelength_um"], w["pixel_um"], stream=stream, mux=M)
    I = torch.empty((w["K"] // M, w["n"], w["n"]), dtype=torch.float32, device=dev)
    elf.simulate(obj_dev, I)
    g = torch.Generator(device=dev)
    g.manual_seed(5)
    I += 1e-3 * torch.randn(I.shape, generator=g, device=dev)
    elf.set_measurements(I)
    elf.set_tracing(True)
    for _ in range(3):
        elf.step(1)
    t_it, t_tile = [], []
    for _ in range(10):
        elf.step(1)
        st = elf.stage_times()
        t_it.append(st["iteration"])
        t_tile.append(st["tile"])
    elf.close()
    it = float(np.median(t_it))
    return {"workload": f"{w['name']}_mux{M}", "leds_per_image": M, "images": w["K"] // M,
            "iteration_ms": it, "tile_stage_ms": float(np.median(t_tile)),
            "led_updates_per_s": w["K"] / (it * 1e-3),
            "note": "traced steps; parity: tests/test_gpu_mux.py"}


def eval_leg(wid, w, I_dev, obj_dev, torch, dev):
    """Sec. 4.1 evaluation on the GPU for the benchmark workload: NL (Eq. 21) of its measurements
    against the clean forward model at the true LED positions, and the amplitude / phase LSNR
    (Eq. 22, global phase removed) of a 100-iteration reconstruction against the true object.
    Also the time of one elf_degrade call (Eq. 20 uneven illumination c = 0.2 with w = 15 px,
    Gaussian a = 1e-3, salt & pepper 0.05, background) over all 225 images, random fields given."""
    from paper_2209_14671_gb300 import elfpie as E
    stream = torch.cuda.current_stream(dev)
    with E.Elf(w["n"], w["u"], w["k_xy_true"], w["na"], w["wavelength_um"], w["pixel_um"], stream=stream) as sim:
        I_clean = torch.empty((w["K"], w["n"], w["n"]), dtype=torch.float32, device=dev)
        sim.simulate(obj_dev, I_clean)
        nl = sim.noise_level(I_clean, I_dev)
        g = torch.Generator(device=dev)
        g.manual_seed(20)
        zeta = torch.randn(I_clean.shape, generator=g, device=dev)
        xi = torch.randn(I_clean.shape, generator=g, device=dev)
        u = torch.rand(I_clean.shape, generator=g, device=dev)
        bg = 0.1 * torch.rand((w["K"],), generator=g, device=dev)
        out = torch.empty_like(I_clean)
        kw = dict(c=0.2, waist_px=15.0, zeta=zeta, background=bg, gauss_a=1e-3, xi=xi, snp_density=0.05, u_snp=u)
        sim.degrade(I_clean, out, **kw)
        t = []
        for _ in range(5):
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            sim.degrade(I_clean, out, **kw)  # synchronises
            s1.record(stream)
            torch.cuda.synchronize(dev)
            t.append(s0.elapsed_time(s1))
    with E.Elf(w["n"], w["u"], w["k_xy"], w["na"], w["wavelength_um"], w["pixel_um"], stream=stream) as elf:
        elf.set_measurements(I_dev)
        elf.step(100)
        la, lp = elf.object_quality(obj_dev)
    return {"workload": w["name"], "nl_percent_darkfield": nl, "lsnr_amplitude_db_100_iters": la,
            "lsnr_phase_db_100_iters": lp, "degrade_ms_225_images": float(np.median(t)),
            "note": "parity: tests/test_gpu_eval.py; quality values have no counterpart in the paper "
                    "(its images are not available)"}


def workloads_leg(torch, dev, steps=50, warmup=5):
    """Throughput of the other two workloads (not the headline): the 64 x 64 / 49-LED / 256 x 256
    problem and the 128 x 128 / 225-LED / 512 x 512 problem, each timed over `steps` iterations with
    CUDA events on its stream after `warmup` iterations (inputs resident, L2 not flushed: these
    problems fit in L2)."""
    from paper_2209_14671_gb300 import elfpie as E
    out = {}
    stream = torch.cuda.current_stream(dev)
    for wid in (0, 3):
        w = IN.problem(wid)
        I = torch.from_numpy(make_inputs(w, wid, torch, dev)).to(dev)
        with E.Elf(w["n"], w["u"], w["k_xy"], w["na"], w["wavelength_um"], w["pixel_um"], stream=stream) as elf:
            elf.set_measurements(I)
            elf.step(warmup)
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            s0.record(stream)
            elf.step(steps)
            s1.record(stream)
            torch.cuda.synchronize(dev)
            ms = s0.elapsed_time(s1) / steps
        out[w["name"]] = {"ms_per_iteration": ms, "led_updates_per_s": w["K"] / (ms * 1e-3)}
    return out


def run_reference(args):
    """The oracle as the reference arm: each step is one full FP64 oracle iteration of the
    workload (all K LEDs, Hessian branch, updates), with the LED blocks spread over the host's
    cores (oracle/parallel.py); on rank 0 only."""
    rank, _, world = dist_env()
    if rank != 0:
        return
    w = IN.problem(args.workload)
    import oracle as O
    from oracle.parallel import ParallelOracle
    geo_t = O.make_geometry(w["n"], w["u"], w["k_xy_true"], w["na"], w["wavelength_um"], w["pixel_um"])
    obj = IN.object_field(args.workload, w)
    I = IN.corrupt(O.forward_intensity(O.spectrum_from_object(obj), geo_t.support.astype(complex), geo_t),
                   args.workload, w).astype(np.float64)
    geo = O.make_geometry(w["n"], w["u"], w["k_xy"], w["na"], w["wavelength_um"], w["pixel_um"])
    opt = O.Options()
    st = O.init_state(I, geo, w["k_xy"], opt)
    with ParallelOracle(geo, I) as po:
        st, _ = po.run(st, opt, args.warmup)
        t0 = time.perf_counter()
        st, _ = po.run(st, opt, args.steps)
        el = time.perf_counter() - t0
        cores = po.cores
    val = geo.K * args.steps / el
    sample = (f"{args.steps} full FP64 oracle iterations of this workload ({geo.K} LEDs each) after {args.warmup} "
              f"warm-up iterations; LED blocks on {cores - 1} worker processes, the Hessian branch on the main "
              f"process; {el:.1f} s; host CPU {cpu_model()}")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded generator, FP64 oracle forward model + workload degradations)",
            "config": {"workload": w["name"], "n": w["n"], "N": w["N"], "K": w["K"]},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    from paper_2209_14671_gb300 import build as B
    from paper_2209_14671_gb300 import elfpie as E

    rank, local, world = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    B.build()
    E.load()
    wid = args.workload
    w = IN.problem(wid)
    I_host = make_inputs(w, wid, torch, dev)
    I_dev = torch.from_numpy(I_host).to(dev)
    stream = torch.cuda.current_stream(dev)
    elf = E.Elf(w["n"], w["u"], w["k_xy"], w["na"], w["wavelength_um"], w["pixel_um"], stream=stream)
    elf.set_measurements(I_dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    # stage breakdown (not timed for the metric): the same steps with CUDA events recorded
    # inside the graph around each stage, on the stream each stage runs on
    elf.set_tracing(True)
    stage_ms, stage_spans = [], []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        elf.step(1)
        if i >= args.warmup:
            stage_ms.append(elf.stage_times())  # synchronises after the step
            stage_spans.append(elf.stage_spans())
    elf.set_tracing(False)
    kernels_per_step = elf.kernels_per_step()

    clocks = ClockSampler(local)  # live before the warm-up steps, so they and the timed steps are sampled
    for _ in range(args.warmup):
        flush.zero_()
        elf.step(1)
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    torch.cuda.synchronize(dev)
    clocks.start()
    for i in range(args.steps):
        flush.zero_()                     # L2 flush between timed iterations (outside the events)
        starts[i].record(stream)
        elf.step(1)
        ends[i].record(stream)
    torch.cuda.synchronize(dev)
    clk = clocks.stop()
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    total_ms = max_over_ranks(float(sum(step_ms)), world, dev)
    if world > 1:
        torch.distributed.barrier()
    units = w["K"] * args.steps * world
    value = units / (total_ms / 1e3)

    # dominant kernel: the per-LED tile kernel
    tile_ms = float(np.mean([s["tile"] for s in stage_ms]))
    S = elf.S
    tile_bytes = w["K"] * (4 * w["n"] ** 2 + 16 * S) + 8 * S
    tile_flops = w["K"] * tile_flops_per_led(w["n"])
    hbm, peak_kind = peaks()
    achieved = tile_bytes / (tile_ms / 1e3) / 1e9
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    # FP32 peak measured on this GPU (the library's FMA-throughput kernel), right after the timed steps
    alu_peak, fma_ms = E.measure_fp32_peak(stream=stream)
    alu_src = (f"measured: FMA-throughput kernel of the library (elf_measure_fp32_peak: {sms} SMs x 8 blocks x 256 "
               f"threads x 8 independent FMA chains, best of 5 launches of {fma_ms:.2f} ms), run right after the "
               f"timed steps; nominal {fp32_nominal_tflops(sms, clk.get('sm_max_mhz') if clk else None):.1f} TFLOP/s "
               f"at the maximum SM clock")
    achieved_tf = tile_flops / (tile_ms / 1e3) / 1e12
    traffic = None
    if os.path.exists(TRAFFIC_PATH):
        tr = json.load(open(TRAFFIC_PATH))
        if tr.get("sources_sha256_16") == tile_sources_hash() and tr.get("workload") == w["name"]:
            traffic = tr.get("dram_bytes_per_launch")
    stage_mean = {k: float(np.mean([s[k] for s in stage_ms])) for k in stage_ms[0]}
    span_median = {k: [round(float(np.median([s[k][e] for s in stage_spans])), 4) for e in (0, 1)]
                   for k in stage_spans[0]}
    it_bytes = w["K"] * (4 * w["n"] ** 2 + 32 * S) + 72 * w["N"] ** 2

    # end to end through the public API with host buffers: one full reconstruction per step
    e2e = None
    if not args.no_e2e:
        I_pin = torch.from_numpy(I_host).pin_memory()
        O_pin = torch.empty((w["N"], w["N"]), dtype=torch.complex64).pin_memory()
        elf.set_tracing(False)
        jobs, warm = max(3, args.steps // 4), max(1, args.warmup // 2)
        iters = w["iters"]
        for _ in range(warm):
            elf.set_measurements(I_pin.numpy())
            elf.step(iters)
            elf.get_object(O_pin.numpy())
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(jobs):
            elf.set_measurements(I_pin.numpy())   # H2D of the job's measurements + initial state
            elf.step(iters)
            elf.get_object(O_pin.numpy())         # D2H of the reconstructed object (synchronises)
        el = max_over_ranks(time.perf_counter() - t0, world, dev)
        e2e = {"value": w["K"] * iters * jobs * world / el, "unit": UNIT,
               "h2d_bytes_per_step": int(I_host.nbytes), "d2h_bytes_per_step": int(O_pin.numel() * 8),
               "step": f"one reconstruction: elf_set_measurements(pinned host) + elf_step({iters}) + "
                       f"elf_get_object(pinned host); {jobs} jobs timed by wall clock"}

    precision = None
    if not args.no_precision and world == 1:
        precision = precision_leg(torch, dev)

    fidelity = None
    if not args.no_fidelity and world == 1:
        fidelity = fidelity_leg(w, I_dev, torch, dev)

    workloads = None
    if not args.no_workloads and world == 1:
        workloads = workloads_leg(torch, dev)

    evaluation = None
    if not args.no_eval and world == 1:
        obj = torch.from_numpy(IN.object_field(wid, w).astype(np.complex64)).to(dev)
        evaluation = eval_leg(wid, w, I_dev, obj, torch, dev)

    mux = None
    if not args.no_mux and world == 1:
        obj = torch.from_numpy(IN.object_field(wid, w).astype(np.complex64)).to(dev)
        mux = mux_leg(wid, w, obj, torch, dev)

    serving = None
    if args.serving_requests > 0:
        serving = serving_leg(args, torch, dev)

    cpu = None
    error_vs_oracle = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate1, its, el1 = oracle_sample_rate(I_host, w, args.cpu_seconds)
        error_vs_oracle, rate_all, cores, el_all = oracle_error_check(
            I_host, w, lambda: E.Elf(w["n"], w["u"], w["k_xy"], w["na"], w["wavelength_um"], w["pixel_um"],
                                     stream=stream), args.check_iters)
        cpu = {"value": rate_all, "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"{args.check_iters} full FP64 oracle iterations of this workload ({w['K']} LEDs each) from "
                         f"its state after 3 iterations, {el_all:.1f} s: LED blocks on {cores - 1} worker processes, "
                         f"the Hessian branch on the main process (the run the error check compares with)",
               "cpu_model": cpu_model(),
               "single_core": {"value": rate1, "unit": UNIT, "cores": 1,
                               "sample": f"{its} full FP64 oracle iterations of this workload from its initial state, "
                                         f"{el1:.1f} s on one host core (NumPy pocketfft, single-threaded)"}}
    elf.close()
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic: seeded smooth random object, GPU forward model at jittered LED positions, "
                    "workload degradations (Gaussian, Poisson, salt & pepper, background, vignetting)",
            "config": {"workload": w["name"], "n": w["n"], "N": w["N"], "K": w["K"], "iters_per_step": 1,
                       "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{world}",
                       "learn_pupil": 1, "fidelity": "intensity (Eq. 5)"},
            "roofline": {"bound": "alu", "achieved": achieved_tf, "peak": alu_peak, "unit": "TFLOP/s",
                         "frac": achieved_tf / alu_peak, "traffic": traffic,
                         "kernel": "tile stage (the per-LED work of Eqs. 1, 5, 12, 11, F_B^H): rows_inv_kernel<256> + "
                                   "cols_kernel<256,0,1> + rows_fwd_kernel<256>, one launch each per iteration",
                         "algorithmic_flops": tile_flops, "launch_ms": tile_ms, "peak_source": alu_src,
                         "flop_model": "per LED: two n x n 2D FFTs at 5 B log2 B each + 40 FLOP per pixel",
                         "hbm": {"achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                                 "algorithmic_bytes": tile_bytes, "peak_source": peak_kind}},
            "iteration_roofline": {"algorithmic_bytes": it_bytes, "achieved_gbs": it_bytes / (total_ms / args.steps / 1e3) / 1e9,
                                   "frac": it_bytes / (total_ms / args.steps / 1e3) / 1e9 / hbm},
            "stage_ms": stage_mean,
            "stage_spans_ms": span_median,
            "clocks": clk,
            "gpu_launches": kernels_per_step * args.steps,
            "e2e": e2e,
            "serving": serving,
            "precision": precision,
            "fidelity_variants": fidelity,
            "multiplexed": mux,
            "evaluation": evaluation,
            "other_workloads": workloads,
            "cpu_baseline": cpu,
            "error_vs_oracle": error_vs_oracle,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
