"""Benchmark of the binary-fluid D3Q19 lattice-Boltzmann step on GB300.

Workload: spinodal decomposition on a periodic 384^3 lattice (56.6M sites),
phi seeded noise in [-0.05, 0.05], rho = 1, u = 0, A = -0.0625, B = 0.0625,
kappa = 0.04, Gamma = 0.5, tau_f = tau_g = 1. A step is one full timestep
(moments, phi stencil and mu, force, collisions of f and g, propagation, in
the storage codec of the precision), run by the library's CUDA kernels
through the C ABI; the timed region ends with the FP64 conservation totals.

Metric: MLUPS (million lattice-site updates per second), with the fraction
of the HBM roofline: algorithmic bytes per site = 76 x (bytes per stored
value): 19 f and 19 g values read and written. The primary line is the FP32
storage form; FP64 and the FP16/BF16 deviation forms are reported in
"per_precision". The state (>= 8.6 GB) is far larger than L2 (129 MB), so no
flush is needed between steps.

--impl reference times the FP64 CPU oracle (test infrastructure) on a
bounded sample of the same workload on the host cores.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

BYTES_PER_VALUE = {"fp64": 8, "fp32": 4, "fp16dev": 2, "bf16dev": 2}
VALUES_PER_SITE = 76  # 2 x 19 distributions, read + write
FALLBACK_HBM_GBS = 6800.0
METRIC = "MLUPS & % of HBM roofline per precision on 1 GB300; adjoint/forward cost ratio"
SEED = 5
# the CUDA kernel behind each step-kernel choice of the library
KERNEL_NAMES = {"fused": "k_step_fused", "fused_staged": "k_step_staged", "generic": "k_phi+k_mu+k_collide"}


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--size", type=int, default=384, help="lattice edge (cubic, periodic)")
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--precisions", default="fp32,fp64,fp16dev,bf16dev",
                    help="comma list; the first one is the primary line")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-lc", action="store_true", help="skip the liquid-crystal step line")
    ap.add_argument("--lc-size", type=int, default=256, help="lattice edge of the liquid-crystal step line")
    ap.add_argument("--no-per-size", action="store_true",
                    help="skip the FP32 line at 256^3 (the size of the FP32 roofline target)")
    ap.add_argument("--stencil", type=int, default=7, choices=[7, 19],
                    help="order-parameter stencils: 7-point (default) or 19-point isotropic")
    return ap.parse_args()


def config_of(args):
    n = args.size
    return {"workload": f"spinodal-{n}^3-periodic", "lattice": [n, n, n], "sites": n ** 3,
            "init": "phi uniform seeded noise in [-0.05,0.05] (SplitMix64 seed 5), rho=1, u=0, f,g at equilibrium",
            "params": {"A": -0.0625, "B": 0.0625, "kappa": 0.04, "Gamma": 0.5, "tau_f": 1.0, "tau_g": 1.0,
                       "stencil": args.stencil},
            "bytes_per_site_algorithmic": None, "l2": "no flush: state is larger than L2 (129 MB)",
            "parallelism": "replicas (one independent lattice per GPU)"}


# --------------------------------------------------------------------------
def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


_TOKENS = re.compile(r'//[^\n]*|/\*.*?\*/|"(?:\\.|[^"\\\n])*"|\'(?:\\.|[^\'\\\n])*\'', re.S)


def _code_hash(rels):
    """Hash of the code in the given sources with comments removed and
    whitespace runs collapsed, so that a record taken on a kernel stays
    valid through edits of its comments but not of its code."""
    h = hashlib.sha256()
    for rel in rels:
        with open(os.path.join(ROOT, rel), encoding="utf-8") as fh:
            text = fh.read()
        code = _TOKENS.sub(lambda mt: " " if mt.group(0)[0] == "/" else mt.group(0), text)
        h.update(" ".join(code.split()).encode())
        h.update(b"\0")
    return h.hexdigest()[:16]


def kernel_source_hash():
    return _code_hash(("paper_1609_01479_gb300/csrc/ld_fused.cuh", "paper_1609_01479_gb300/csrc/ld_common.cuh",
                       "paper_1609_01479_gb300/csrc/ld_async.cuh"))


def fp64_source_hash():
    return _code_hash(("paper_1609_01479_gb300/csrc/ld_generic.cuh", "paper_1609_01479_gb300/csrc/ld_common.cuh",
                       "paper_1609_01479_gb300/csrc/ld_prec_f64.cu"))


def recorded_fp64_ops():
    """FP64-pipe thread instructions per site of the FP64 step (the generic
    launches, which the library picks for FP64), from the committed ncu
    counter summary, if taken on the current source."""
    path = os.path.join(ROOT, "profiles", "fp64_pipe.txt")
    if not os.path.exists(path):
        return None
    want = fp64_source_hash()
    with open(path) as fh:
        for line in fh:
            parts = line.split("#")[0].split()
            if len(parts) >= 4 and parts[0] == "generic" and parts[1] == "fp64" and parts[3] == want:
                return float(parts[2])
    return None


def fp64_pipe_probe(torch, ld, reps=5):
    """Measured FP64 instruction rate of this GPU (the library's throughput
    probe: 8 independent chains of one FP64 operation per thread, full
    occupancy), best of `reps` timed launches per operation, in G
    instructions/s; the roof of the FP64 step, which the FP64 pipe bounds."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    blocks, iters = 8 * sms, 4096
    sink = torch.zeros(blocks, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream()
    rates = {}
    for op, name in ((0, "dfma"), (1, "dadd"), (2, "dmul")):
        for _ in range(2):
            ld.ld_probe_fp64_rate(op, blocks, iters, sink, stream.cuda_stream)
        best = None
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ld.ld_probe_fp64_rate(op, blocks, iters, sink, stream.cuda_stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            best = ms if best is None else min(best, ms)
        rates[name] = blocks * 256 * 8 * iters / (best * 1e-3) / 1e9
    return rates


def copy_probe_gbs(torch, nbytes=2 << 30, reps=10):
    """Device-to-device copy bandwidth (read + write bytes / time) of a buffer
    far larger than L2, timed with CUDA events: the achievable-bandwidth probe
    beside the measured peak."""
    src = torch.empty(nbytes // 4, dtype=torch.float32, device="cuda")
    dst = torch.empty_like(src)
    src.fill_(1.0)
    for _ in range(3):
        dst.copy_(src)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        dst.copy_(src)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    del src, dst
    torch.cuda.empty_cache()
    return 2.0 * nbytes / (ms * 1e-3) / 1e9


def recorded_traffic(precision, size):
    """DRAM bytes per launch of the fused step from the committed ncu summary,
    if it was taken on the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    want = kernel_source_hash()
    with open(path) as fh:
        for line in fh:
            parts = line.split("#")[0].split()
            if len(parts) < 5:
                continue
            kernel, prec, sz, bytes_per_launch, src_hash = parts[:5]
            if prec == precision and int(sz) == size and src_hash == want:
                return float(bytes_per_launch)
    return None


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.proc = None
        self.lines = []
        target = None
        try:
            import torch

            uuid = str(torch.cuda.get_device_properties(device_index).uuid)
            target = uuid if uuid.startswith("GPU-") else f"GPU-{uuid}"
        except Exception:
            target = str(device_index)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", target, f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            cols = [c.strip() for c in line.split(",")]
            if len(cols) < 8:
                continue
            try:
                sm.append(float(cols[0]))
                smax.append(float(cols[1]))
                power.append(float(cols[2]))
            except ValueError:
                continue
            for name, val in zip(names, cols[4:8]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


# --------------------------------------------------------------------------
def dist_setup(args):
    import torch

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(world, value):
    """Largest value over all ranks (NCCL on the GPU, gloo on the host)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist

    device = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def time_precision(args, ld, phi_dev, precision, world, sample_clocks=False, n=None):
    """Warm up, then time exactly args.steps steps (plus the final totals) on
    an n^3 lattice (the bench lattice unless given)."""
    import torch

    n = args.size if n is None else n
    stream = torch.cuda.current_stream()
    sim = ld.LdSim(n, n, n, precision=precision, stream=stream.cuda_stream, stencil=args.stencil)
    sim.init(phi_dev)
    sim.step(args.warmup)
    totals = torch.empty(5, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    region0 = torch.cuda.Event(enable_timing=True)
    region1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device()) if sample_clocks else None
    if sampler is not None:
        time.sleep(0.3)  # let the sampler start before the region
    region0.record(stream)
    for k in range(args.steps):
        starts[k].record(stream)
        ld.ld_step(sim.ctx, 1)
        ends[k].record(stream)
    ld.ld_moments(sim.ctx, totals=totals)
    region1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler is not None else None
    barrier(world)
    region_ms = region0.elapsed_time(region1)
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    tot = totals.cpu().numpy()
    kernel = ld.ld_step_kernel(sim.ctx)
    sim.close()
    del sim
    torch.cuda.empty_cache()
    return {"region_ms": region_ms, "kernel_ms_mean": float(np.mean(step_ms)),
            "kernel_ms_median": float(np.median(step_ms)), "totals": tot.tolist(), "clocks": clocks,
            "kernel": kernel}


def time_e2e(args, ld, phi_host_pinned, precision):
    """Whole run through the public API with host buffers: H2D of phi0 from
    pinned memory, init, args.steps steps, D2H of phi; MLUPS of that run."""
    import torch

    n = args.size
    stream = torch.cuda.current_stream()
    sim = ld.LdSim(n, n, n, precision=precision, stream=stream.cuda_stream, stencil=args.stencil)
    phi_dev = torch.empty(phi_host_pinned.shape, dtype=torch.float64, device="cuda")
    phi_out_dev = torch.empty_like(phi_dev)
    phi_out_host = torch.empty(phi_host_pinned.shape, dtype=torch.float64, pin_memory=True)
    # one untimed pass for warm-up
    for timed in (False, True):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        phi_dev.copy_(phi_host_pinned, non_blocking=True)
        sim.init(phi_dev)
        sim.step(args.steps if timed else args.warmup)
        ld.ld_moments(sim.ctx, phi=phi_out_dev)
        phi_out_host.copy_(phi_out_dev, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    sim.close()
    del sim
    torch.cuda.empty_cache()
    nbytes = phi_host_pinned.numel() * 8
    return ms, nbytes


def time_adjoint(args, ld, phi_dev, precision, steps=40, every=10):
    """Backward pass of a differentiable run on the bench lattice: seed, then
    per segment (last first) recompute into a tape with ld_step_between and
    run ld_adjoint_step over it in reverse, then ld_adjoint_init. Returns the
    backward time per step, split into recompute and adjoint kernels, and the
    forward time per step of the same run (plain ld_step)."""
    import torch

    n = args.size
    stream = torch.cuda.current_stream()
    sim = ld.LdSim(n, n, n, precision=precision, stream=stream.cuda_stream, stencil=args.stencil)
    sim.init(phi_dev)
    nbytes = ld.ld_state_bytes(sim.ctx)
    ckpts = [torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(steps // every)]
    tape = [torch.empty(nbytes, dtype=torch.uint8, device="cuda") for _ in range(every - 1)]
    fbytes = ld.ld_fields_bytes(sim.ctx)
    fields = [torch.empty(fbytes, dtype=torch.uint8, device="cuda") for _ in range(every - 1)]
    adj_ws = torch.empty(ld.ld_adjoint_workspace_bytes(sim.ctx), dtype=torch.uint8, device="cuda")
    ld.ld_adjoint_attach(sim.ctx, adj_ws)
    grad = torch.zeros(2, dtype=torch.float64, device="cuda")
    phibar = torch.empty_like(phi_dev).normal_()
    gphi0 = torch.empty_like(phi_dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    # forward with checkpoints
    f0, f1 = ev(), ev()
    torch.cuda.synchronize()
    f0.record(stream)
    for c in ckpts:
        ld.ld_save_state(sim.ctx, c)
        ld.ld_step(sim.ctx, every)
    f1.record(stream)
    # backward
    marks = []
    b0 = ev()
    b0.record(stream)
    ld.ld_adjoint_seed(sim.ctx, phibar)
    for c in reversed(ckpts):
        r0, r1, a1 = ev(), ev(), ev()
        r0.record(stream)
        states = [c] + tape
        for j in range(1, every):
            ld.ld_step_between(sim.ctx, states[j - 1], states[j], fields[j - 1])
        r1.record(stream)
        for j in reversed(range(every)):
            ld.ld_adjoint_step(sim.ctx, states[j], grad, fields[j] if j < every - 1 else None)
        a1.record(stream)
        marks.append((r0, r1, a1))
    ld.ld_adjoint_init(sim.ctx, phi_dev, gphi0, None, grad)
    b1 = ev()
    b1.record(stream)
    torch.cuda.synchronize()
    rec_ms = sum(r0.elapsed_time(r1) for r0, r1, _ in marks)
    adj_ms = sum(r1.elapsed_time(a1) for _, r1, a1 in marks)
    out = {"steps": steps, "checkpoint_every": every, "forward_ms_per_step": f0.elapsed_time(f1) / steps,
           "backward_ms_per_step": b0.elapsed_time(b1) / steps, "recompute_ms_per_step": rec_ms / steps,
           "adjoint_kernels_ms_per_step": adj_ms / steps, "precision": precision}
    sim.close()
    del sim, ckpts, tape, fields, adj_ws
    torch.cuda.empty_cache()
    return out


def time_lc(args, ld, n, precision):
    """The liquid-crystal step (Q-tensor + D3Q19 fluid, the context's own
    step kernel) on an n^3 lattice from a disordered seeded Q, at rest:
    args.warmup untimed steps, then args.steps timed with CUDA events on the
    launching stream. Returns (ms per step, step kernel)."""
    import torch

    from paper_1609_01479_gb300 import inputs

    stream = torch.cuda.current_stream()
    sim = ld.LcSim(n, n, n, precision=precision, stream=stream.cuda_stream)
    sim.init(torch.from_numpy(inputs.random_q(n, n, n, seed=SEED)).to("cuda"))
    sim.step(args.warmup)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sim.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    kernel = sim.kernel
    sim.close()
    del sim
    torch.cuda.empty_cache()
    return ms, kernel


def cpu_baseline(sample_edge=96, sample_steps=20):
    """The FP64 oracle, as it stands, on the host cores: MLUPS on a bounded
    sample (a sample_edge^3 lattice of the same workload, sample_steps steps)."""
    import oracle
    from paper_1609_01479_gb300 import inputs

    oracle.build()
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    prm = oracle.param_vector()
    phi = inputs.spinodal_phi(sample_edge, sample_edge, sample_edge, seed=SEED)
    f, g = oracle.init(phi, prm)
    f, g = oracle.step(f, g, prm, 1)  # warm-up
    t0 = time.perf_counter()
    oracle.step(f, g, prm, sample_steps)
    dt = time.perf_counter() - t0
    return {"value": sample_edge ** 3 * sample_steps / dt / 1e6, "unit": "MLUPS", "cores": oracle.get_threads(),
            "kind": "oracle",
            "sample": f"{sample_edge}^3 lattice of the same spinodal workload, {sample_steps} steps, FP64 oracle "
                      f"(C++ -O2, OpenMP over z-planes), {dt:.2f} s"}


def lc_cpu_baseline(sample_edge=96, sample_steps=5):
    """The liquid-crystal FP64 oracle, as it stands, on the host cores (OpenMP
    over z-planes), on a bounded sample of the bench's liquid-crystal
    workload: a sample_edge^3 lattice from the same disordered Q,
    sample_steps steps."""
    import oracle
    from paper_1609_01479_gb300 import inputs

    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    n = sample_edge
    prm = oracle.lc_param_vector()
    q = inputs.random_q(n, n, n, seed=SEED)
    f = oracle.lc_init((n, n, n), prm, rho=np.ones((n, n, n)), u=np.zeros((3, n, n, n)))
    f, q = oracle.lc_step(f, q, prm, 1)  # warm-up
    t0 = time.perf_counter()
    oracle.lc_step(f, q, prm, sample_steps)
    dt = time.perf_counter() - t0
    return {"value": n ** 3 * sample_steps / dt / 1e6, "unit": "MLUPS", "cores": oracle.get_threads(),
            "kind": "oracle",
            "sample": f"{n}^3 lattice of the liquid-crystal workload, {sample_steps} steps, FP64 oracle "
                      f"(C++ -O2, OpenMP over z-planes), {dt:.2f} s"}


# --------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle
    from paper_1609_01479_gb300 import inputs

    oracle.build()
    threads = os.cpu_count() or 1
    oracle.set_threads(threads)
    prm = oracle.param_vector()
    edge = 64  # bounded sample of the 384^3 workload per step
    phi = inputs.spinodal_phi(edge, edge, edge, seed=SEED)
    f, g = oracle.init(phi, prm)
    for _ in range(args.warmup):
        f, g = oracle.step(f, g, prm, 1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        f, g = oracle.step(f, g, prm, 1)
    dt = time.perf_counter() - t0
    mlups = edge ** 3 * args.steps / dt / 1e6
    cfg = config_of(args)
    cfg["bytes_per_site_algorithmic"] = VALUES_PER_SITE * 8
    sample = f"{edge}^3 sample of the {args.size}^3 workload per step, FP64 oracle on {oracle.get_threads()} threads"
    line = {"impl": "reference", "metric": METRIC, "value": mlups, "unit": "MLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": oracle.get_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch

    from paper_1609_01479_gb300 import inputs, ld

    world, rank, local = dist_setup(args)
    ld.lib()
    n = args.size
    precisions = [p.strip() for p in args.precisions.split(",") if p.strip()]
    phi_np = inputs.spinodal_phi(n, n, n, seed=SEED)
    phi_dev = torch.from_numpy(phi_np).to("cuda")
    peak, peak_kind = measured_hbm_peak()

    results = {}
    for i, prec in enumerate(precisions):
        r = time_precision(args, ld, phi_dev, prec, world, sample_clocks=(i == 0))
        region_ms = max_over_ranks(world, r["region_ms"])
        kernel_ms = max_over_ranks(world, r["kernel_ms_mean"])
        sites = n ** 3
        bps = VALUES_PER_SITE * BYTES_PER_VALUE[prec]
        results[prec] = {
            "kernel": r["kernel"],
            "mlups": world * sites * args.steps / (region_ms * 1e-3) / 1e6,
            "ms_per_step": region_ms / args.steps,
            "kernel_ms": kernel_ms,
            "algorithmic_gbs": sites * bps / (kernel_ms * 1e-3) / 1e9,
            "bytes_per_site": bps,
            "totals": r["totals"],
            "clocks": r["clocks"],
        }
        results[prec]["roofline_frac"] = results[prec]["algorithmic_gbs"] / peak

    primary = precisions[0]
    P = results[primary]
    # The FP32 fused step's roofline target is stated at 256^3: time that
    # lattice too (same seed, same steps), beside the bench lattice.
    per_size = {}
    if not args.no_per_size and n != 256 and "fp32" in results:
        n2 = 256
        phi2 = torch.from_numpy(inputs.spinodal_phi(n2, n2, n2, seed=SEED)).to("cuda")
        r2 = time_precision(args, ld, phi2, "fp32", world, n=n2)
        del phi2
        reg2 = max_over_ranks(world, r2["region_ms"])
        k2 = max_over_ranks(world, r2["kernel_ms_mean"])
        bps = VALUES_PER_SITE * BYTES_PER_VALUE["fp32"]
        gbs = n2 ** 3 * bps / (k2 * 1e-3) / 1e9
        per_size[str(n2)] = {"precision": "fp32", "sites": n2 ** 3, "steps": args.steps,
                             "mlups": world * n2 ** 3 * args.steps / (reg2 * 1e-3) / 1e6,
                             "ms_per_step": reg2 / args.steps, "kernel_ms": k2, "algorithmic_gbs": gbs,
                             "roofline_frac": gbs / peak, "kernel": r2["kernel"]}
    if "fp64" in results:
        # FP64 is bounded by the FP64 pipe. Its roof is the FP64 instruction
        # rate measured on this GPU by the library's probe (the best of DFMA,
        # DADD and DMUL); the nominal figure (2 FP64 instructions per clock
        # per SM: 1.25 TFLOP/s with an FMA counted as 2 flops at 152 SMs x
        # 2.07 GHz) is reported beside it.
        ops = recorded_fp64_ops() if args.stencil == 7 else None  # the record is for the default stencils
        sms = torch.cuda.get_device_properties(0).multi_processor_count
        mhz = (P["clocks"] or {}).get("sm_max_mhz") or 2070.0
        nominal = 2.0 * sms * mhz * 1e6 / 1e9
        rates = fp64_pipe_probe(torch, ld)
        peak_ops = max(rates.values())
        R64 = results["fp64"]
        achieved = None if ops is None else R64["mlups"] * 1e6 * ops / 1e9
        R64["alu"] = {"bound": "alu", "achieved": achieved, "peak": peak_ops, "unit": "G FP64 inst/s",
                      "frac": None if achieved is None else achieved / peak_ops, "fp64_inst_per_site": ops,
                      "peak_source": "measured: ld_probe_fp64_rate, best of DFMA/DADD/DMUL chains",
                      "probe_rates": rates, "nominal_peak": nominal,
                      "nominal_source": f"2 FP64 inst/clk/SM x {sms} SMs x {mhz:.0f} MHz"}
    probe = copy_probe_gbs(torch) if rank == 0 else None
    e2e = None
    if not args.no_e2e:
        phi_pinned = torch.from_numpy(phi_np).pin_memory()
        ms, nbytes = time_e2e(args, ld, phi_pinned, primary)
        ms = max_over_ranks(world, ms)
        e2e = {"value": world * n ** 3 * args.steps / (ms * 1e-3) / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": nbytes / args.steps, "d2h_bytes_per_step": nbytes / args.steps,
               "what": f"pinned phi0 H2D + ld_init + {args.steps} ld_step + ld_moments(phi) + D2H, one run"}
    adj = None if args.no_adjoint else time_adjoint(args, ld, phi_dev, primary)
    # The liquid-crystal step (the paper's Ludwig test case), 256^3 by default: its
    # state is f (19 values) and Q (5 values) per site, read and written once
    # a step at the least: 48 values. What the launches move on top:
    #   fused (z-marching field + collision, then the Q update): Q read once
    #     more (5), u written and read (6): 59 values;
    #   generic (three per-site launches): Q read once more (5), H (10),
    #     sigma (18) and u (6) written and read: 87 values.
    lc = {}
    if not args.no_lc:
        n_lc = args.lc_size
        launch_values = {"fused": 59, "generic": 87}
        for prec in ("fp32", "fp64"):
            ms, kernel = time_lc(args, ld, n_lc, prec)
            ms = max_over_ranks(world, ms)
            bps = 48 * BYTES_PER_VALUE[prec]
            lbps = launch_values[kernel] * BYTES_PER_VALUE[prec]
            gbs = n_lc ** 3 * bps / (ms * 1e-3) / 1e9
            lgbs = n_lc ** 3 * lbps / (ms * 1e-3) / 1e9
            lc[prec] = {"lattice": [n_lc] * 3, "kernel": kernel,
                        "mlups": world * n_lc ** 3 / (ms * 1e-3) / 1e6, "ms_per_step": ms,
                        "state_bytes_per_site": bps, "launch_bytes_per_site": lbps,
                        "state_gbs": gbs, "roofline_frac_of_state": gbs / peak,
                        "launch_gbs": lgbs, "roofline_frac_of_launch_bytes": lgbs / peak}
    if rank != 0:
        return
    cpu = None if args.no_cpu_baseline or world > 1 else cpu_baseline()
    if lc and not args.no_cpu_baseline and world == 1:
        lc["cpu_baseline"] = lc_cpu_baseline()
    cfg = config_of(args)
    cfg["bytes_per_site_algorithmic"] = P["bytes_per_site"]
    cfg["precision"] = primary
    traffic = recorded_traffic(primary, n) if args.stencil == 7 else None  # recorded for the default stencils
    line = {
        "metric": METRIC,
        "value": P["mlups"],
        "unit": "MLUPS",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": P["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if primary == "fp32" else ("f64" if primary == "fp64" else "f32-compute/16-bit-storage"),
        "data": "synthetic",
        "config": cfg,
        "roofline": {"bound": "hbm", "achieved": P["algorithmic_gbs"], "peak": peak, "unit": "GB/s",
                     "frac": P["roofline_frac"], "traffic": traffic,
                     "kernel": KERNEL_NAMES.get(P["kernel"], P["kernel"]), "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)"
                     if peak_kind == "measured" else "fallback 6.8 TB/s",
                     "per_site_bytes": P["bytes_per_site"], "kernel_ms": P["kernel_ms"],
                     "copy_probe_gbs": probe, "frac_of_copy_probe": None if not probe else P["algorithmic_gbs"] / probe},
        "clocks": P["clocks"],
        "e2e": e2e,
        "gpu_launches": args.steps + 2,
        "cpu_baseline": cpu,
        "per_precision": {p: {k: v for k, v in r.items() if k not in ("clocks",)} for p, r in results.items()},
        "per_size": per_size,
        "lc": lc,
        "adjoint_forward_ratio": None if adj is None else adj["backward_ms_per_step"] / P["ms_per_step"],
        "adjoint": adj,
    }
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
