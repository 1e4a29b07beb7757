"""Benchmark: D3Q19 TRT FP32 stream-collide sweep on a 256^3 periodic box.

One bench step is one lattice Boltzmann time step (one fused stream-collide
sweep over all 16.8 M cells, AA in-place pattern).  Synthetic input: 3-D
Taylor-Green vortex, u0 = 0.02 plus U(-1e-4, 1e-4) noise (SplitMix64 seed 42),
rho = 1; omega_e = 1.8, Lambda = 3/16.  The population array (1.27 GB) is far
larger than the 129 MB L2, so no flush is needed between timed steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

The line also carries "variants" (the other workloads of the metric: two-grid
pull, esoteric twist, FP16-shifted storage, Smagorinsky, KBC, the MRT channel,
the D3Q27 cumulant, D2Q9 FP64 and the adjoint step against the forward step)
and "accuracy" (FP32 and FP16-shifted storage against FP64 runs of the same
kernels on the TGV, the channel and the cumulant TGV, with kinetic-energy
decay).

--impl reference times the FP64 numpy oracle on the host cores on a bounded
sample of the same workload (a 32^3 periodic box per step).  Under torchrun
(N > 1) every rank runs its own replica (weak scaling, no collective on the
data path); the elapsed time is the maximum over ranks.
"""
import argparse
import hashlib
import glob
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SIDE = 256
OMEGA_E, MAGIC = 1.8, 3.0 / 16.0
U0, NOISE, SEED = 0.02, 1e-4, 42
Q, ELEM = 19, 4
METRIC = "MLUPS and % of HBM roofline per stencil/collision; FP16/FP32 vs FP64 error"
WORKLOAD = "D3Q19 TRT FP32 256^3 periodic Taylor-Green vortex, AA in-place pattern"
REF_SIDE = 32


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def algorithmic_bytes(q, value_bytes, fluid_cells, mask_cells=0):
    """Bytes one stream-collide step must move (Sec. V: read and write every
    population once, 2 q values per fluid cell), plus the 4-byte link mask of
    every cell of a masked domain."""
    return 2 * q * value_bytes * fluid_cells + 4 * mask_cells


def roofline_mlups(bandwidth_gbs, q, value_bytes):
    """Memory-bound MLUPS limit: bandwidth / bytes per cell update."""
    return bandwidth_gbs * 1e9 / algorithmic_bytes(q, value_bytes, 1) / 1e6


def kernel_source_hash():
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(ROOT, "paper_2001_11806_gb300", "csrc", "*"))):
        with open(p, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(cells):
    """DRAM bytes per launch from the committed ncu summary, or None if the
    kernel sources changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as fh:
            rec = json.load(fh)
    except Exception:
        return None
    if rec.get("source_hash") != kernel_source_hash():
        return None
    return rec["dram_bytes_per_cell"] * cells


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v, device=None):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def smi_device_id(local):
    """nvidia-smi -i id of this rank's GPU: the local-th entry of
    CUDA_VISIBLE_DEVICES (an index or a UUID, both accepted by -i), else the
    local rank itself."""
    vis = [v.strip() for v in os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",") if v.strip()]
    return vis[local] if local < len(vis) else str(local)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region.

    start() returns only after the first sample has arrived, so that the
    sampler's own start-up never overlaps the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def _reader(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line))

    def start(self):
        import threading
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._reader, daemon=True)
        self.thread.start()
        t0 = time.time()
        while not self.lines and time.time() - t0 < 20.0:
            time.sleep(0.05)
        self.skip = len(self.lines)

    @staticmethod
    def _text(entry):
        return entry[1] if isinstance(entry, tuple) else entry

    def window_mhz(self, t0, t1):
        """Median SM clock of the samples that arrived between host times t0
        and t1 (None when the window held no sample)."""
        sm = []
        for entry in self.lines:
            if not isinstance(entry, tuple) or not (t0 <= entry[0] <= t1):
                continue
            parts = [p.strip() for p in entry[1].split(",")]
            try:
                sm.append(float(parts[1]))
            except (IndexError, ValueError):
                continue
        return float(np.median(sm)) if sm else None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=10)
        except Exception:
            self.proc.kill()
        if self.thread is not None:
            self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for entry in self.lines[self.skip:]:
            line = self._text(entry)
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)]
        return {"sm_mhz": float(np.median(loaded)), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample_run(steps, warmup, budget_s=None, side=REF_SIDE, barrier=None):
    """The FP64 oracle on a side^3 periodic box of the same workload: (MLUPS,
    steps timed, seconds)."""
    from oracle import collision as oco
    from oracle import lattice as olat
    from oracle import lbm as olbm
    from paper_2001_11806_gb300 import inputs
    lat = olat.d3q19()
    sim = olbm.Sim(oco.Method(lat, "trt", [OMEGA_E, oco.trt_odd_rate(OMEGA_E, MAGIC)]), (side,) * 3)
    rho, u = inputs.tgv3d(side, U0, NOISE, SEED)
    sim.init_equilibrium(rho, u)
    sim.step(warmup)
    if barrier is not None:
        barrier.wait()
    t0 = time.perf_counter()
    done = 0
    while done < steps:
        sim.step(1)
        done += 1
        if budget_s is not None and time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return side ** 3 * done / dt / 1e6, done, dt


def _oracle_worker(args):
    steps, warmup, budget_s, side, barrier = args
    return oracle_sample_run(steps, warmup, budget_s, side, barrier)


def host_cpu():
    """CPU model name and logical core count of this host (lscpu, else
    /proc/cpuinfo)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except Exception:
        pass
    return model, os.cpu_count() or 1


def oracle_parallel_run(procs, steps, warmup, budget_s, side):
    """The oracle timed on `procs` host cores at once: one spawned process
    per core, each stepping its own side^3 box of the workload (the oracle
    itself is unchanged and single-threaded; BLAS threads are pinned to 1).
    Returns (aggregate MLUPS, steps of the slowest process, seconds)."""
    import multiprocessing as mpl
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[var] = "1"
    if procs <= 1:
        return oracle_sample_run(steps, warmup, budget_s, side)
    ctx = mpl.get_context("spawn")
    with ctx.Manager() as mgr:
        barrier = mgr.Barrier(procs)
        with ctx.Pool(procs) as pool:
            res = pool.map(_oracle_worker, [(steps, warmup, budget_s, side, barrier)] * procs)
    cells_steps = sum(side ** 3 * done for _, done, _ in res)
    wall = max(dt for _, _, dt in res)
    return cells_steps / wall / 1e6, min(done for _, done, _ in res), wall


REF_BUDGET_S = 120.0  # the reference arm stops timing after this many seconds
REPEATS = 5  # the timed steps are split into this many repeats (median reported)
CPU_SIDE = 64  # box edge of each oracle process


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    model, cores = host_cpu()
    mlups, done, dt = oracle_parallel_run(cores, args.steps, args.warmup, REF_BUDGET_S, CPU_SIDE)
    sample = (f"FP64 numpy oracle, one {CPU_SIDE}^3 periodic box of the same TGV workload per process on "
              f"{cores} processes ({model}), {done} steps each")
    if done < args.steps:
        sample += f" (of {args.steps} requested; timing stops after {REF_BUDGET_S:.0f} s)"
    line = {"impl": "reference", "metric": METRIC, "value": round(mlups, 4), "unit": "MLUPS",
            "n_gpus": args.gpus, "steps": done, "warmup": args.warmup,
            "ms_per_step": round(1e3 * dt / done, 3), "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"{cores} x {CPU_SIDE}^3 boxes", "cpu_model": model},
            "cpu_baseline": {"value": round(mlups, 4), "unit": "MLUPS", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": round(mlups, 4), "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _time_steps(sim, steps, torch):
    stream = torch.cuda.current_stream(sim.device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)
    e1.record(stream)
    torch.cuda.synchronize(sim.device)
    return e0.elapsed_time(e1) / steps


def run_variants(device, peak, only=None, steps_override=None, warmup=10):
    """The other workloads of the metric, one line each: MLUPS over all cells,
    algorithmic GB/s (2 q sizeof per fluid cell, plus the 4 B link mask per
    cell when boundaries are present) and its fraction of the measured peak.
    only: run just the workloads whose name contains this string (and not the
    adjoint line), with steps_override timed steps after `warmup` steps."""
    import torch

    from paper_2001_11806_gb300 import inputs
    from paper_2001_11806_gb300.sim import Sim
    elem = {"f64": 8, "f32": 4, "f32s": 4, "f16s": 2}
    out = []
    specs = [
        ("D3Q19 TRT FP32 256^3 two-grid pull", dict(stencil="D3Q19", collision="trt", storage="f32", pattern="pull",
                                                  shape=(256,) * 3, omega=[OMEGA_E], trt_magic=MAGIC), "tgv", 300),
        ("D3Q19 TRT FP16-shifted 256^3 AA", dict(stencil="D3Q19", collision="trt", storage="f16s", pattern="aa",
                                                 shape=(256,) * 3, omega=[OMEGA_E], trt_magic=MAGIC), "tgv", 300),
        ("D3Q19 TRT FP16-shifted 256^3 two-grid pull", dict(stencil="D3Q19", collision="trt", storage="f16s",
                                                            pattern="pull", shape=(256,) * 3, omega=[OMEGA_E],
                                                            trt_magic=MAGIC), "tgv", 300),
        ("D3Q19 TRT FP16-shifted 256^3 esoteric twist", dict(stencil="D3Q19", collision="trt", storage="f16s",
                                                             pattern="eso", shape=(256,) * 3, omega=[OMEGA_E],
                                                             trt_magic=MAGIC), "tgv", 300),
        ("D3Q19 TRT FP32 256^3 esoteric twist", dict(stencil="D3Q19", collision="trt", storage="f32", pattern="eso",
                                                     shape=(256,) * 3, omega=[OMEGA_E], trt_magic=MAGIC), "tgv", 300),
        ("D3Q19 MRT FP32 256^3 AA, one higher-order rate", dict(stencil="D3Q19", collision="mrt", storage="f32",
                                                                pattern="aa", shape=(256,) * 3,
                                                                omega=[1.7, 1.0, 1.0, 1.0]), "tgv", 200),
        ("D3Q19 MRT FP32 256^3 AA, four rates (moment matrix)", dict(stencil="D3Q19", collision="mrt",
                                                                     storage="f32", pattern="aa", shape=(256,) * 3,
                                                                     omega=[1.7, 1.1, 0.9, 1.3]), "tgv", 200),
        ("D3Q27 TRT FP32 256^3 AA", dict(stencil="D3Q27", collision="trt", storage="f32", pattern="aa",
                                         shape=(256,) * 3, omega=[OMEGA_E], trt_magic=MAGIC), "tgv", 200),
        ("D3Q19 TRT FP64 256^3 AA", dict(stencil="D3Q19", collision="trt", storage="f64", pattern="aa",
                                         shape=(256,) * 3, omega=[OMEGA_E], trt_magic=MAGIC), "tgv", 50),
        ("D3Q19 SRT + Smagorinsky (C_S 0.17) FP32 256^3 AA",
         dict(stencil="D3Q19", collision="srt", storage="f32", pattern="aa", shape=(256,) * 3, omega=[1.95],
              smagorinsky_cs=0.17), "tgv", 300),
        ("D3Q19 KBC FP32 256^3 AA", dict(stencil="D3Q19", collision="kbc", storage="f32", pattern="aa",
                                         shape=(256,) * 3, omega=[1.95, 1.95]), "tgv", 300),
        ("D3Q27 KBC FP32 256^3 AA", dict(stencil="D3Q27", collision="kbc", storage="f32", pattern="aa",
                                         shape=(256,) * 3, omega=[1.95, 1.95]), "tgv", 200),
        ("D3Q19 MRT FP32 channel 512x128x128 AA", dict(stencil="D3Q19", collision="mrt", storage="f32", pattern="aa",
                                                       shape=(512, 128, 128), omega=[1.7, 1.0, 1.0, 1.0],
                                                       periodic=(False, False, False), u_wall=(0.05, 0, 0)),
         "channel", 300),
        ("D3Q19 MRT FP32 channel 512x128x128 two-grid pull", dict(stencil="D3Q19", collision="mrt", storage="f32",
                                                                  pattern="pull", shape=(512, 128, 128),
                                                                  omega=[1.7, 1.0, 1.0, 1.0],
                                                                  periodic=(False, False, False),
                                                                  u_wall=(0.05, 0, 0)),
         "channel", 300),
        ("D3Q19 MRT FP32 channel 512x128x128 two-grid pull, separate boundary kernel",
         dict(stencil="D3Q19", collision="mrt", storage="f32", pattern="pull", shape=(512, 128, 128),
              omega=[1.7, 1.0, 1.0, 1.0], periodic=(False, False, False), u_wall=(0.05, 0, 0),
              boundary="separate"), "channel", 300),
        ("D3Q19 MRT FP16-shifted channel 512x128x128 AA", dict(stencil="D3Q19", collision="mrt", storage="f16s",
                                                                 pattern="aa", shape=(512, 128, 128),
                                                                 omega=[1.7, 1.0, 1.0, 1.0],
                                                                 periodic=(False, False, False), u_wall=(0.05, 0, 0)),
         "channel", 300),
        ("D3Q27 cumulant FP32 384^3 AA", dict(stencil="D3Q27", collision="cumulant", storage="f32", pattern="aa",
                                              shape=(384,) * 3, omega=[1.95, 1.0, 1.0]), "tgv", 100),
        ("D3Q27 cumulant FP32-shifted 384^3 AA", dict(stencil="D3Q27", collision="cumulant", storage="f32s",
                                                      pattern="aa", shape=(384,) * 3, omega=[1.95, 1.0, 1.0]),
         "tgv", 100),
        ("D2Q9 SRT FP64 64^2 pull", dict(stencil="D2Q9", collision="srt", storage="f64", pattern="pull",
                                         shape=(64, 64, 1), omega=[1.6]), "tgv2d", 2000),
    ]
    if only is not None:
        specs = [sp for sp in specs if only in sp[0]]
        if not specs:
            raise SystemExit(f"no variant matches {only!r}")
    flags_channel = None
    for name, kw, init, steps in specs:
        if steps_override is not None:
            steps = steps_override
        flags = None
        if init == "channel":
            if flags_channel is None:
                flags_channel = inputs.channel_flags(512, 128, 128)
            flags = flags_channel
        sim = Sim(device=device, flags=flags, **kw)
        N, q = sim.N, sim.q
        if init == "tgv":
            rho, u = inputs.tgv3d(kw["shape"][0], U0, NOISE, SEED)
        elif init == "tgv2d":
            rho, u = inputs.tgv2d(64, 0.01)
        else:
            rho, u = np.ones(N), np.zeros((3, N))
        sim.init_equilibrium(rho.reshape(-1), u.reshape(sim.d, -1))
        sim.step(warmup)
        ms = _time_steps(sim, steps, torch)
        fluid = N if flags is None else int((flags == 0).sum())
        nbytes = algorithmic_bytes(q, elem[kw["storage"]], fluid, N if flags is not None else 0)
        gbs = nbytes / (ms * 1e-3) / 1e9
        out.append({"workload": name, "mlups": round(N / ms / 1e3, 1),
                    "fluid_mlups": round(fluid / ms / 1e3, 1), "ms_per_step": round(ms, 4),
                    "gbs": round(gbs, 1), "frac": round(gbs / peak, 4)})
        sim.close()
        del sim
        torch.cuda.empty_cache()
    if only is not None:
        return out
    out += run_adjoint(device, peak)
    return out


def run_adjoint(device, peak, T=1000):
    """Config 5 (D3Q19 TRT FP32 128^3 TGV, uniform force 1e-6): one adjoint
    step against one forward step, and the whole gradient (forward with
    sqrt(T) checkpoints, seed, recomputation and reverse sweep) against T
    forward steps."""
    import torch

    from paper_2001_11806_gb300 import _lib, inputs
    from paper_2001_11806_gb300.adjoint import Rollout
    from paper_2001_11806_gb300.sim import Sim
    out = []
    sim = Sim("D3Q19", "trt", "f32", "pull", (128,) * 3, omega=[OMEGA_E], trt_magic=MAGIC, force=[1e-6, 0, 0],
              device=device)
    rho, u = inputs.tgv3d(128, U0, NOISE, SEED)
    sim.init_equilibrium(rho.reshape(-1), u.reshape(3, -1))
    sim.step(10)
    fwd = _time_steps(sim, 200, torch)
    raw, _ = sim.get_pdfs()
    # a dense adjoint field (every force row non-zero), as in a real reverse sweep
    gen = torch.Generator(device=device).manual_seed(5)
    lam = [torch.randn((19, sim.N), dtype=torch.float32, device=device, generator=gen) for _ in range(2)]
    dF = torch.zeros(3, dtype=torch.float64, device=device)
    stream = torch.cuda.current_stream(sim.device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for i in range(5):
        _lib.lib().lbm_adjoint_step(sim.ctx, raw.data_ptr(), lam[i % 2].data_ptr(), lam[1 - i % 2].data_ptr(),
                                    dF.data_ptr())
    e0.record(stream)
    for i in range(200):
        _lib.lib().lbm_adjoint_step(sim.ctx, raw.data_ptr(), lam[i % 2].data_ptr(), lam[1 - i % 2].data_ptr(),
                                    dF.data_ptr())
    e1.record(stream)
    torch.cuda.synchronize(device)
    adj = e0.elapsed_time(e1) / 200
    gbs = 3 * 19 * 4 * sim.N / (adj * 1e-3) / 1e9
    out.append({"workload": "D3Q19 TRT FP32 128^3 adjoint step", "ms_per_step": round(adj, 4),
                "forward_ms_per_step": round(fwd, 4), "adjoint_over_forward": round(adj / fwd, 3),
                "gbs": round(gbs, 1), "frac": round(gbs / peak, 4)})
    sim.close()
    del sim, lam, raw
    torch.cuda.empty_cache()
    box = (48, 80, 48, 80, 48, 80)
    rho0, u0 = rho.reshape(-1), u.reshape(3, -1)
    ro = Rollout("D3Q19", "trt", "f32", (128,) * 3, [OMEGA_E], T, box, trt_magic=MAGIC, device=device)
    ro.gradient(rho0, u0, [1e-6, 0.0, 0.0])
    stream = torch.cuda.current_stream(device)
    reps = []
    for _ in range(3):
        e0.record(stream)
        ro.gradient(rho0, u0, [1e-6, 0.0, 0.0])
        e1.record(stream)
        torch.cuda.synchronize(device)
        grad_ms = e0.elapsed_time(e1)
        e0.record(stream)
        ro.loss(rho0, u0, [1e-6, 0.0, 0.0])
        e1.record(stream)
        torch.cuda.synchronize(device)
        reps.append((grad_ms, e0.elapsed_time(e1)))
    grad_ms, loss_ms = sorted(reps)[1]
    out.append({"workload": f"D3Q19 TRT FP32 128^3 gradient of the box kinetic energy, T = {T}, sqrt(T) checkpoints",
                "gradient_ms": round(grad_ms, 2), "forward_ms": round(loss_ms, 2),
                "gradient_over_forward": round(grad_ms / loss_ms, 3),
                "checkpoint_buffers": len(ro._ckpt) + len(ro._seg)})
    del ro
    torch.cuda.empty_cache()
    return out


def _rel_errors(fields, ref, mask=None):
    """Relative L2 of rho - 1 and (worst component) of u against ref."""
    r, v = fields
    r64, u64 = ref
    if mask is not None:
        r, v, r64, u64 = r[mask], v[:, mask], r64[mask], u64[:, mask]
    return {"rho_minus_1": float(np.linalg.norm(r - r64) / np.linalg.norm(r64 - 1.0)),
            "u": float(max(np.linalg.norm(v[a] - u64[a]) / np.linalg.norm(u64[a]) for a in range(v.shape[0])))}


def run_accuracy(device, cumulant_steps=100):
    """FP32 and FP16-shifted storage against an FP64 run of the same kernels
    (the secondary reference; the FP64 oracle is too slow at these sizes).
    Relative L2 of rho - 1 and of u (fluid cells), kinetic energy ratios.
    - D3Q19 TRT 256^3 TGV, 1000 steps, AA;
    - D3Q19 MRT channel 512x128x128 (walls, inlet 0.05, outlet, obstacles),
      2000 steps from rest, AA;
    - D3Q27 cumulant 384^3 TGV u0 = 0.05: FP32 kinetic-energy decay over 5000
      steps, and FP32 against FP64 after `cumulant_steps` steps (100 by
      default: FP64 cumulant arithmetic runs at about 0.5 GLUPS on this part,
      so the 5000 steps of the workload take about ten minutes, which
      --accuracy-only --cumulant-steps 5000 runs on its own)."""
    import torch

    from paper_2001_11806_gb300 import inputs
    from paper_2001_11806_gb300.sim import Sim

    def run(kw, rho, u, T, storages, mask=None):
        fields, ke = {}, {}
        for st in storages:
            sim = Sim(storage=st, device=device, **kw)
            sim.init_equilibrium(rho.reshape(-1), u.reshape(sim.d, -1))
            e0 = sim.reduce()[4]
            sim.step(T)
            ke[st] = sim.reduce()[4] / e0 if e0 > 0 else None
            r, v = sim.macroscopic(True)
            fields[st] = (r.cpu().numpy(), v.cpu().numpy())
            sim.close()
            del sim
            torch.cuda.empty_cache()
        return fields, ke

    out = []
    # D3Q19 TRT TGV
    n, T = N_SIDE, 1000
    rho, u = inputs.tgv3d(n, U0, NOISE, SEED)
    kw = dict(stencil="D3Q19", collision="trt", pattern="aa", shape=(n,) * 3, omega=[OMEGA_E], trt_magic=MAGIC)
    fields, ke = run(kw, rho, u, T, ["f64", "f32", "f16s"])
    entry = {"workload": "D3Q19 TRT 256^3 TGV u0 = 0.02, 1000 steps, AA; reference: FP64 GPU run",
             "ke_ratio_f64": round(float(ke["f64"]), 8)}
    for st in ["f32", "f16s"]:
        entry[st] = dict(_rel_errors(fields[st], fields["f64"]), ke_ratio=round(float(ke[st]), 8))
    out.append(entry)
    # D3Q19 MRT channel
    shape = (512, 128, 128)
    flags = inputs.channel_flags(*shape)
    fluid = flags.reshape(-1) == 0
    N = flags.size
    kw = dict(stencil="D3Q19", collision="mrt", pattern="aa", shape=shape, omega=[1.7, 1.0, 1.0, 1.0],
              periodic=(False, False, False), u_wall=(0.05, 0.0, 0.0), flags=flags)
    fields, _ = run(kw, np.ones(N), np.zeros((3, N)), 2000, ["f64", "f32", "f16s"])
    entry = {"workload": "D3Q19 MRT channel 512x128x128, inlet 0.05, 2000 steps from rest, AA; fluid cells; "
                         "reference: FP64 GPU run",
             "mean_ux_f64": round(float(fields["f64"][1][0][fluid].mean()), 8)}
    for st in ["f32", "f16s"]:
        entry[st] = _rel_errors(fields[st], fields["f64"], fluid)
    out.append(entry)
    # D3Q27 cumulant TGV
    n = 384
    rho, u = inputs.tgv3d(n, 0.05, 0.0, SEED)
    kw = dict(stencil="D3Q27", collision="cumulant", pattern="aa", shape=(n,) * 3, omega=[1.95, 1.0, 1.0])
    sim = Sim(storage="f32", device=device, **kw)
    sim.init_equilibrium(rho.reshape(-1), u.reshape(3, -1))
    e0 = sim.reduce()[4]
    decay = {}
    for t in range(1000, 5001, 1000):
        sim.step(1000)
        decay[str(t)] = round(float(sim.reduce()[4] / e0), 6)
    sim.close()
    del sim
    torch.cuda.empty_cache()
    fields, ke = run(kw, rho, u, cumulant_steps, ["f64", "f32"])
    out.append({"workload": "D3Q27 cumulant 384^3 TGV u0 = 0.05, omega 1.95, AA",
                "ke_ratio_f32": decay,
                f"f32_vs_f64_after_{cumulant_steps}_steps": dict(_rel_errors(fields["f32"], fields["f64"]),
                                                                 ke_ratio_f64=round(float(ke["f64"]), 8),
                                                                 ke_ratio_f32=round(float(ke["f32"]), 8))})
    return out


def run_gpu(args, world, rank, local):
    import torch

    from paper_2001_11806_gb300 import inputs
    from paper_2001_11806_gb300.sim import Sim

    device = torch.device(f"cuda:{local}")
    torch.cuda.set_device(device)
    n = args.size
    cells = n ** 3
    rho, u = inputs.tgv3d(n, U0, NOISE, SEED)
    rho_h = torch.from_numpy(rho.reshape(-1)).pin_memory()
    u_h = torch.from_numpy(u.reshape(3, -1)).pin_memory()
    stream = torch.cuda.current_stream(device)

    sim = Sim("D3Q19", "trt", "f32", "aa", (n, n, n), omega=[OMEGA_E], trt_magic=MAGIC, device=device)
    sim.init_equilibrium(rho_h.to(device), u_h.to(device))
    sim.step(args.warmup)
    torch.cuda.synchronize(device)

    # ---- device-resident timed region: the K steps run as R repeats of
    # about K / R steps, each bracketed by CUDA events on the launching
    # stream and a synchronize (host times give each repeat's clock window);
    # the headline is the median repeat, min and max are reported beside it
    R = min(REPEATS, args.steps)
    sizes = [args.steps // R] * R
    sizes[-1] += args.steps - sum(sizes)
    clocks = ClockSampler(smi_device_id(local))
    clocks.start()
    barrier(world)
    torch.cuda.synchronize(device)
    rep_ms, rep_win = [], []
    total_ms = 0.0
    for n_rep in sizes:
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t_host0 = time.time()
        ev0.record(stream)
        sim.step(n_rep)
        ev1.record(stream)
        torch.cuda.synchronize(device)
        rep_win.append((t_host0, time.time()))
        t = ev0.elapsed_time(ev1)
        total_ms += t
        rep_ms.append(t / n_rep)
    barrier(world)
    clk = clocks.stop()
    per_rep = [max_over_ranks(world, v, device) for v in rep_ms]
    ms_step = float(np.median(per_rep))
    total_ms = max_over_ranks(world, total_ms, device)
    mlups = cells * world / (ms_step * 1e-3) / 1e6
    repeats = {"n": R, "steps": sizes, "ms_per_step": [round(v, 5) for v in per_rep],
               "median_ms_per_step": round(ms_step, 5), "min_ms_per_step": round(min(per_rep), 5),
               "max_ms_per_step": round(max(per_rep), 5), "total_ms": round(total_ms, 3),
               "sm_mhz": [clocks.window_mhz(t0 - 0.15, t1 + 0.15) for t0, t1 in rep_win]}

    # ---- end to end through the public API with host buffers: every pass
    # copies rho/u from pinned host memory, initialises, steps, computes the
    # macroscopic fields and copies them back to pinned host memory.  One
    # untimed pass with the warm-up step count comes first: the first GPU
    # access to freshly pinned host pages costs 10-20 ms once (measured on
    # GB300), which a caller that reuses its buffers pays only once
    out_rho = torch.empty(cells, dtype=torch.float32).pin_memory()
    out_u = torch.empty((3, cells), dtype=torch.float32).pin_memory()

    def e2e_pass(n_steps):
        rd = rho_h.to(device, non_blocking=True)
        ud = u_h.to(device, non_blocking=True)
        sim.init_equilibrium(rd, ud)
        sim.step(n_steps)
        r_dev, u_dev = sim.macroscopic(f64=False)
        out_rho.copy_(r_dev, non_blocking=True)
        out_u.copy_(u_dev, non_blocking=True)

    e2e_pass(args.warmup)
    barrier(world)
    torch.cuda.synchronize(device)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_pass(args.steps)
    e1.record(stream)
    torch.cuda.synchronize(device)
    barrier(world)
    e2e_ms = max_over_ranks(world, e0.elapsed_time(e1), device)
    e2e = {"value": round(cells * args.steps * world / (e2e_ms * 1e-3) / 1e6, 2), "unit": "MLUPS",
           "h2d_bytes_per_step": int((rho_h.numel() + u_h.numel()) * 8 / args.steps),
           "d2h_bytes_per_step": int((out_rho.numel() + out_u.numel()) * 4 / args.steps)}
    assert np.isfinite(out_rho.numpy()).all()

    if rank != 0:
        return 0
    peak, peak_kind = measured_peak()
    bytes_per_launch = algorithmic_bytes(Q, ELEM, cells)
    if n != N_SIDE:
        line_workload = WORKLOAD.replace("256^3", f"{n}^3")
    else:
        line_workload = WORKLOAD
    achieved = bytes_per_launch / (ms_step * 1e-3) / 1e9
    traffic = recorded_traffic(cells)
    cpu_model, cpu_cores = host_cpu()
    if args.no_cpu_baseline:
        cpu_mlups, cpu_steps, cpu_dt = float("nan"), 0, 0.0
    else:
        # spawned processes only: this process has used the GPU already
        cpu_mlups, cpu_steps, cpu_dt = oracle_parallel_run(cpu_cores, 10 ** 9, 1, 12.0, CPU_SIDE)
    variants = None if args.no_variants else run_variants(device, peak)
    accuracy = None if args.no_variants else run_accuracy(device, args.cumulant_steps)
    line = {
        "metric": METRIC, "value": round(mlups, 2), "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_step, 5), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "repeats": repeats,
        "config": {"workload": line_workload, "stencil": "D3Q19", "collision": "TRT", "omega_e": OMEGA_E,
                   "magic": MAGIC, "storage": "f32", "pattern": "aa", "cells": cells,
                   "l2": "inputs larger than L2 (1.27 GB population array vs 129 MB L2)",
                   "parallelism": f"{world} independent replicas"},
        "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "traffic": traffic,
                     "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": bytes_per_launch},
        "cpu_baseline": {"value": round(cpu_mlups, 4), "unit": "MLUPS", "cores": cpu_cores, "kind": "oracle",
                         "sample": f"FP64 numpy oracle, one {CPU_SIDE}^3 periodic box of the same workload per "
                                   f"process on {cpu_cores} processes ({cpu_model}), {cpu_steps} steps each in "
                                   f"{cpu_dt:.1f} s"},
        "e2e": e2e,
        "gpu_launches": args.steps,
        "host_cpu": cpu_model,
        "clocks": clk,
        "variants": variants,
        "accuracy": accuracy,
    }
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    # profiling aids: a smaller box of the same kernel, and skipping the CPU leg
    ap.add_argument("--size", type=int, default=N_SIDE)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-variants", action="store_true")
    # the FP32/FP16 accuracy runs alone; the cumulant's FP32-vs-FP64 length
    ap.add_argument("--accuracy-only", action="store_true")
    ap.add_argument("--cumulant-steps", type=int, default=100)
    # run one variant workload alone (name substring), e.g. to profile it;
    # "adjoint" runs the adjoint step and the whole gradient with T = --steps
    ap.add_argument("--variant", default=None)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.accuracy_only:
        import torch
        torch.cuda.set_device(0)
        print(json.dumps({"accuracy": run_accuracy(torch.device("cuda:0"), args.cumulant_steps)}))
        return 0
    if args.variant is not None:
        import torch
        torch.cuda.set_device(0)
        peak = measured_peak()[0]
        if args.variant == "adjoint":
            # the adjoint step and the whole gradient, with T = --steps
            for v in run_adjoint(torch.device("cuda:0"), peak, T=args.steps):
                print(json.dumps(v))
            return 0
        for v in run_variants(torch.device("cuda:0"), peak, only=args.variant, steps_override=args.steps,
                              warmup=args.warmup):
            print(json.dumps(v))
        return 0
    world, rank, local = dist_setup()
    if args.impl == "reference":
        rc = run_reference(args, world, rank)
    else:
        rc = run_gpu(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
