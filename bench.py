"""Benchmark: composed split-operator propagation of a 3-D three-surface
vibronic-coupling wavepacket (64^3 grid per surface, complex128) on GB300.

Metric: grid-points x substeps per second (a substep is one kinetic action of
the pruned composition; grid points = prod n_d).  A "step" here is one
composed time step of the Suzuki-fractal order-6 scheme (25 substeps).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun, one process per GPU)
every rank propagates its own independently seeded wavepacket (weak scaling,
no data exchange); ``value`` is the sum of all ranks' work over the slowest
rank's time.  ``--impl reference`` times the FP64 CPU oracle on the host
cores on a bounded sample of the same workload (one substep per step).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "grid-pts x substeps/s"
UNIT = "grid-pts*substeps/s"
T_FINAL = 2000.0
SEED = 1904
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2

# Workloads.  The default is the 64^3 three-surface FP64 propagation the
# metric is quoted on; "precision128" is the FP32 storage-and-FFT mode on a
# 128^3 three-surface grid (orders 4 or 8), reported with its error against
# the FP64 path.
WORKLOADS = {
    "pyrazine64": dict(grid=(64, 64, 64), S=3, order=6, scheme="suzuki", dt=T_FINAL / 128, fp32=False),
    "precision128": dict(grid=(128, 128, 128), S=3, order=4, scheme="triple_jump", dt=T_FINAL / 128, fp32=True),
}
W = dict(WORKLOADS["pyrazine64"])
N_GRID, S, ORDER, SCHEME_NAME, DT = W["grid"], W["S"], W["order"], W["scheme"], W["dt"]


def select_workload(name, order=None):
    global W, N_GRID, S, ORDER, SCHEME_NAME, DT
    W = dict(WORKLOADS[name])
    if order:
        W["order"] = order
    W["name"] = name
    N_GRID, S, ORDER, SCHEME_NAME, DT = W["grid"], W["S"], W["order"], W["scheme"], W["dt"]


def workload(seed=SEED):
    import synth
    return synth.pyrazine_like(seed=seed, n=N_GRID, S=S)


def scheme_code():
    from paper_1903_04946_gb300 import DSO_SUZUKI, DSO_TRIPLE_JUMP
    return DSO_SUZUKI if SCHEME_NAME == "suzuki" else DSO_TRIPLE_JUMP


def substeps_per_step():
    from paper_1903_04946_gb300 import dso_scheme_coefficients
    a, b, *_ = dso_scheme_coefficients(ORDER, scheme_code())
    return len(b)


def config_dict(extra=None):
    sname = "Suzuki" if SCHEME_NAME == "suzuki" else "triple-jump"
    d = {"workload": f"pyrazine-like 3-D vibronic model, {S} surfaces, "
                     f"{'x'.join(map(str, N_GRID))} grid per surface, "
                     f"{'complex64 storage and FFT' if W['fp32'] else 'complex128'}, "
                     f"{sname} order {ORDER}, dt = {DT} a.u.",
         "grid": list(N_GRID), "surfaces": S, "order": ORDER, "scheme": SCHEME_NAME, "dt": DT,
         "seed": SEED, "parallelism": "independent wavepacket per GPU"}
    if extra:
        d.update(extra)
    return d


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_seed(rank: int) -> int:
    """Each rank propagates its own independently seeded wavepacket."""
    return SEED + rank


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Slowest rank's time (control-path reduction only; no wavefunction data
    crosses ranks)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world: int, points: int, substeps: int, steps: int, seconds: float) -> float:
    """Whole-job grid-points x substeps per second: every rank does the same
    amount of work, timed by the slowest rank."""
    return world * points * substeps * steps / seconds


# --------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        # the raw samples go to DSO_BENCH_OUT (default: the system temporary directory)
        import tempfile
        out = os.environ.get("DSO_BENCH_OUT") or tempfile.gettempdir()
        self.path = os.path.join(out, f"clocks_rank{device_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------
# roofline of the dominant kernel
# --------------------------------------------------------------------------

def fp64_peak_tflops():
    """FP64 peak of GB300 from unit counts and clock: 152 SMs x 2 FP64 FMA
    lanes per SM per clock x 2 flops x 2070 MHz = 1.259 TFLOP/s."""
    return 152 * 2 * 2 * 2070e6 / 1e12


def pass_flops_bytes(kind, n, S, esz=16):
    """Nominal algorithmic FLOPs and bytes of one launch of a pass kind:
    5 L log2 L flops per complex FFT of a length-L line, 8 S^2 - 2 S flops per
    grid point per S x S complex matvec, 6 flops per amplitude for the kinetic
    phase; bytes = psi read + write (16 B per amplitude each) plus the
    operator tables read (16 B per packed complex entry)."""
    import math
    P = 1
    for x in n:
        P *= x
    L = n[kind["axis"]]
    f = kind["flags"]
    nfft = (1 if f & 1 else 0) + (1 if f & 2 else 0) + (1 if f & 4 else 0)
    amps = S * P
    flops = nfft * (amps // L) * 5 * L * math.log2(L)
    nU = (1 if f & 256 else 0) + (1 if f & 512 else 0)
    flops += nU * (8 * S * S - 2 * S) * P
    bytes_ = 2 * esz * amps + nU * esz * (S * (S + 1) // 2) * P
    if f & 4:
        flops += 6 * amps
        bytes_ += esz * P
    return flops, bytes_


def kind_name(k):
    f = k["flags"]
    parts = []
    if f & 1:
        parts.append(f"I{k['axis']}")
    if f & 256:
        parts.append("V" + ("V" if f & 512 else ""))
    if f & 2:
        parts.append(f"F{k['axis']}")
    if f & 4:
        parts.append(f"T I{k['axis']}")
    name = {1: "axis_pass_pq_kernel", 2: "axis_pass_tma_kernel", 3: "axis_pass_tmap_kernel"}.get(
        k.get("variant"), "axis_pass_kernel")
    return "%s<L=%d,SV=%d%s> [%s]" % (name, N_GRID[k["axis"]], k["surfaces"], ",float2" if W["fp32"] else "",
                                      " ".join(parts))


# --------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------

def kernel_sources_hash() -> str:
    """First 16 hex digits of the SHA-256 over the device code of the axis
    passes (csrc/*.cuh and their argument struct csrc/pass_args.h, in name
    order, each prefixed by its base name)."""
    import glob
    import hashlib
    csrc = os.path.join(ROOT, "paper_1903_04946_gb300", "csrc")
    h = hashlib.sha256()
    for f in sorted(glob.glob(os.path.join(csrc, "*.cuh")) + [os.path.join(csrc, "pass_args.h")],
                    key=os.path.basename):
        h.update(os.path.basename(f).encode())
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel: str):
    """DRAM bytes per launch (read + write) of `kernel` from the committed ncu
    summaries, or None when no summary covers it or the kernel sources have
    changed since the counters were taken."""
    import glob
    import re
    want = kernel_sources_hash()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as fh:
            text = fh.read()
        m = re.search(r"kernel_sources_sha256_16 = ([0-9a-f]{16})", text)
        if not m or m.group(1) != want:
            continue
        for k, v in re.findall(r"traffic_bytes_per_launch: `(.+?)` = (\d+)", text):
            if k == kernel:
                return int(v), os.path.relpath(path, ROOT)
    return None


def run_gpu(args):
    import numpy as np
    import torch

    import paper_1903_04946_gb300 as dso

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    device = local if world > 1 else 0
    torch.cuda.set_device(device)
    dso.build()
    dso.load()
    pr = workload(rank_seed(rank))
    nsub = substeps_per_step()
    pts = int(np.prod(N_GRID))
    fp32 = W["fp32"]
    esz = 8 if fp32 else 16
    stream = torch.cuda.Stream(device=device)
    ctx = dso.Context(device=device, stream=stream, precision=dso.DSO_FP32 if fp32 else dso.DSO_FP64)
    ctx.load_problem(pr)
    dso.dso_set_scheme(ctx.ctx, ORDER, scheme_code())
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=f"cuda:{device}")

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    # warm-up (tables, graph capture, clocks)
    for _ in range(args.warmup):
        ctx.propagate(DT, DT)
    torch.cuda.synchronize()
    if args.profile_steps:
        # capture range for `ncu --profile-from-start off`: exactly these steps
        l0 = dso.dso_launch_count(ctx.ctx)
        torch.cuda.profiler.start()
        with torch.cuda.stream(stream):
            for _ in range(args.profile_steps):
                ctx.propagate(DT, DT)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        launches = dso.dso_launch_count(ctx.ctx) - l0
        ctx.close()
        if rank == 0:
            print(json.dumps({"profiled_steps": args.profile_steps, "workload": W.get("name", "pyrazine64"),
                              "kernel_launches": int(launches)}))
        return

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    clocks = ClockSampler(device)
    clocks.start()
    time.sleep(0.3)
    launches0 = dso.dso_launch_count(ctx.ctx)
    barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(float(k))                 # evict L2 between timed steps
            starts[k].record(stream)
            ctx.propagate(DT, DT)                 # one composed time step
            ends[k].record(stream)
    torch.cuda.synchronize()
    barrier()
    launches = dso.dso_launch_count(ctx.ctx) - launches0
    ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
    clk = clocks.stop()
    ms = max_over_ranks(ms, world, f"cuda:{device}")
    value = job_throughput(world, pts, nsub, args.steps, ms * 1e-3)

    # end to end through the public API with host buffers: each step copies
    # psi in from pinned host memory, propagates one step and reads psi back
    host_in = torch.from_numpy(pr.psi0.astype(np.complex64 if fp32 else np.complex128)).pin_memory()
    host_out = torch.empty_like(host_in).pin_memory()
    e2e_steps = max(3, min(args.steps, 20))
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        dso.dso_set_psi(ctx.ctx, host_in)
        ctx.propagate(DT, DT)
        dso.dso_get_psi(ctx.ctx, host_out)
    torch.cuda.synchronize()
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e_s = max_over_ranks(e2e_s, world, f"cuda:{device}")
    bytes_psi = S * pts * esz
    e2e = {"value": job_throughput(world, pts, nsub, e2e_steps, e2e_s), "unit": UNIT,
           "h2d_bytes_per_step": bytes_psi, "d2h_bytes_per_step": bytes_psi}

    # per-kernel durations with CUDA events around every launch (same sizes,
    # same pass list as the timed steps)
    kinds = dso.dso_profile_steps(ctx.ctx, DT, max(2, min(args.steps, 10)))
    for k in kinds:
        k["flops"], k["bytes"] = pass_flops_bytes(k, N_GRID, S, esz)
        k["ms_per_step"] = k["avg_ms"] * k["launches_per_step"]
    dom = max(kinds, key=lambda k: k["ms_per_step"])
    prof_step_ms = sum(k["ms_per_step"] for k in kinds)
    try:
        hbm_peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]
        hbm_src = "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, ValueError, KeyError):
        hbm_peak, hbm_src = 6800.0, "fallback"
    if fp32:
        achieved = dom["bytes"] / (dom["avg_ms"] * 1e-3) / 1e9
        roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm_peak, "unit": "GB/s",
                    "frac": round(achieved / hbm_peak, 4), "traffic": None, "peak_source": hbm_src}
    else:
        peak = fp64_peak_tflops()
        achieved = dom["flops"] / (dom["avg_ms"] * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
                    "frac": round(achieved / peak, 4), "traffic": None,
                    "peak_source": "FP64 unit count x max SM clock (152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz)"}
    roofline.update({
                "kernel": kind_name(dom), "kernel_avg_us": round(dom["avg_ms"] * 1e3, 2),
                "kernel_share_of_step": round(dom["ms_per_step"] / prof_step_ms, 4),
                "hbm_gbs_achieved": round(dom["bytes"] / (dom["avg_ms"] * 1e-3) / 1e9, 1),
                "kinds": [{"kernel": kind_name(k), "avg_us": round(k["avg_ms"] * 1e3, 2),
                           "launches_per_step": k["launches_per_step"], "tile_lines": k["tile_lines"],
                           "variant": ["tile", "persistent", "tma", "tma_persistent"][k["variant"]],
                           "tflops": round(k["flops"] / (k["avg_ms"] * 1e-3) / 1e12, 4),
                           "gbs": round(k["bytes"] / (k["avg_ms"] * 1e-3) / 1e9, 1)} for k in kinds]})
    roofline["hbm_peak_gbs_measured"] = hbm_peak
    tr = profiled_traffic(roofline["kernel"])
    if tr is not None:
        roofline["traffic"] = tr[0]
        roofline["traffic_source"] = f"ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, {tr[1]}"
    # the autotuned kernel configuration; DSO_PLAN=<this> reproduces it (profiling)
    roofline["plan"] = dso.dso_tuned_plan(ctx.ctx)

    precision = None
    if fp32:
        # error of the FP32 state against the FP64 path on the same input and
        # the same number of steps (the FP64 GPU path stands in for the CPU
        # oracle at this size; the tests pin it to the oracle)
        nchk = max(2, min(args.steps, 8))
        c32 = dso.Context(pr, device=device, order=ORDER, scheme=scheme_code(), precision=dso.DSO_FP32)
        c64 = dso.Context(pr, device=device, order=ORDER, scheme=scheme_code(), precision=dso.DSO_FP64)
        c32.propagate(nchk * DT, DT)
        c64.propagate(nchk * DT, DT)
        a32 = c32.psi().astype(np.complex128)
        a64 = c64.psi()
        n32, _, _ = c32.observables()
        c32.close()
        c64.close()
        precision = {"steps": nchk, "rel_l2_vs_fp64": float(np.sqrt(np.sum(np.abs(a32 - a64) ** 2) /
                                                                       np.sum(np.abs(a64) ** 2))),
                     "norm_drift": float(abs(n32 - 1.0)), "reference": "FP64 GPU path, same input and steps"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(sample_substeps=args.cpu_substeps)
    ctx.close()

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32" if fp32 else "f64",
                "data": "synthetic (seeded)",
                "config": config_dict({"l2": "flushed before every timed step (256 MiB write outside the "
                                             "per-step CUDA events)",
                                       "substeps_per_step": nsub, "grid_points": pts}),
                "e2e": e2e, "gpu_launches": int(launches), "roofline": roofline, "clocks": clk}
        if cpu is not None:
            line["cpu_baseline"] = cpu
        if precision is not None:
            line["precision"] = precision
        print(json.dumps(line))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# --------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# --------------------------------------------------------------------------

def _oracle_substep_runner():
    import numpy as np
    from oracle import propagate as P
    pr = workload(SEED)
    prop = P.Propagator(pr)
    seq = P.action_sequence(P.VTV, ORDER, SCHEME_NAME)
    # one substep = the potential action before a kinetic action plus that
    # kinetic action (forward FFT, phase, inverse FFT), cycling through the
    # step's pruned sequence
    pairs = [(seq[i], seq[i + 1]) for i in range(0, len(seq) - 1, 2)]
    state = {"psi": pr.psi0.copy(), "i": 0}

    def one():
        (opv, a), (opt, b) = pairs[state["i"] % len(pairs)]
        psi = prop.apply_V(state["psi"], a * DT)
        state["psi"] = prop.apply_T(psi, b * DT)
        state["i"] += 1
    return one, int(np.prod(N_GRID))


def cpu_baseline(sample_substeps=20):
    one, pts = _oracle_substep_runner()
    one()  # builds the cached operators
    t0 = time.perf_counter()
    for _ in range(sample_substeps):
        one()
    dt = time.perf_counter() - t0
    return {"value": pts * sample_substeps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{sample_substeps} substeps (potential action + FFT/phase/inverse FFT) of the same "
                      f"{'x'.join(map(str, N_GRID))} x {S} workload, numpy FP64 oracle, single thread"}


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    one, pts = _oracle_substep_runner()
    for _ in range(args.warmup):
        one()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        one()
    dt = time.perf_counter() - t0
    value = pts * args.steps / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)",
            "config": config_dict({"reference_step": "one substep of the composed sequence (bounded sample)"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} substeps of the 64^3 x 3 workload"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-substeps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default="pyrazine64", choices=sorted(WORKLOADS))
    ap.add_argument("--order", type=int, default=0, help="override the workload's composition order")
    ap.add_argument("--profile-steps", type=int, default=0,
                    help="after the warm-up, run this many steps inside cudaProfilerStart/Stop and exit "
                         "(for ncu --profile-from-start off)")
    args = ap.parse_args()
    select_workload(args.workload, args.order or None)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
