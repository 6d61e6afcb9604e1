"""Benchmark of the ANN-potential MD hot path on GB300.

Workload (default): the 110,592-molecule water box at 1.0 g/cm^3 (331,776
atoms, L = 149.006 A), water basis (radial order 16 / 6.0 A, angular order
8 / 4.0 A, D = 52), per-species 52-32-32-1 tanh networks with seeded
N(0, 1/fan_in) weights, 300 K seeded velocities, velocity-Verlet NVE at
dt = 0.5 fs.

One benchmark step = one MD step of the whole path (kick + drift, cell list,
descriptor, networks, forces + virial, FP64 reductions, kick), replayed from a
captured CUDA graph on device-resident state. Between timed steps the L2 cache
is flushed by writing a buffer larger than L2; each step is bracketed by CUDA
events on the library's stream and the step times are summed.

Every precision form of the network (FP32; BF16 tensor-core layers with split
operands; plain BF16) is timed in the same invocation on the same start, and
each form's energy and forces on frame 0 are compared with the FP64 oracle's
(all atoms). Metric: atom-steps/s (E+F) of the fastest form whose force RMS
error is within 1 meV/A; the line's ``forms`` object carries every form's rate
and errors. The JSON line also carries the end-to-end number of that form
through the C ABI with host buffers (host->device copy of positions,
velocities and types, device->host copy of positions, velocities and
energies, every step), the roofline of the dominant kernel, the FP64 CPU
oracle's throughput on the host cores, and (``batched``) the batched form on
512 independent structures of 32 ... 2,048 atoms: both prepared batches
replayed as CUDA graphs against one evaluation call per structure.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--forms fp32,bf16x3,bf16] [--workload water_331776|...]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "atom-steps/s (E+F) on 1 GB300, BF16 vs FP32 form at <=1 meV/A force err"
DT_PS = 5e-4

# Algorithmic FP32 work per unit (FMA = 2 flops), the figures the roofline is
# graded with: per radial neighbour entry forward 12 + 4 K_r (distance, cutoff,
# the Chebyshev recurrence and two accumulations per order) and backward
# 20 + 6 K_r (the chain rule through every order, force scatter, virial); per
# unordered angular pair forward 10 + 4 K_a and backward 40 + 6 K_a; per atom
# 2 sum_l n_l n_{l-1} for each pass through the network (forward, and
# back-propagation to dE/dG).
def descriptor_kernel_flops(Kr, Ka, n_entries, n_ang_pairs):
    return (12 + 4 * Kr) * n_entries + (10 + 4 * Ka) * n_ang_pairs


def force_kernel_flops(Kr, Ka, n_entries, n_ang_pairs):
    return (20 + 6 * Kr) * n_entries + (40 + 6 * Ka) * n_ang_pairs


def network_flops(widths, n_atoms):
    """Forward plus back-propagation to dE/dG: 2 passes x 2 flops per weight."""
    return 4 * sum(widths[l] * widths[l - 1] for l in range(1, len(widths))) * n_atoms


# DRAM bytes per launch of the dominant kernel (workload, form, kernel), from the ncu
# captures summarised in profiles/; reported only while the kernel source is the
# one the counters were taken on (first 16 hex digits of the SHA-256 of
# potential_kernels.cuh followed by sh_angular.cuh).
TRAFFIC_SOURCE_SHA256_16 = "9909f6a65756bb2a"
TRAFFIC_CAPTURE = {("water_331776", "fp32", "k_potential_list"): 145725952,
                   ("water_331776", "fp32_cell", "k_potential"): 10809600,
                   ("water_12288", "fp32", "k_potential_list"): 5260288,
                   ("amorphous_27000", "fp32", "k_potential"): 1104640}


def captured_traffic(workload_name, precision, kernel, skin=0.0):
    import hashlib
    h = hashlib.sha256()
    for name in ("potential_kernels.cuh", "sh_angular.cuh"):
        with open(os.path.join(ROOT, "paper_2107_11311_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    sha = h.hexdigest()[:16]
    if sha != TRAFFIC_SOURCE_SHA256_16 or skin != 0.0:
        return None
    return TRAFFIC_CAPTURE.get((workload_name, precision, kernel))


def max_over_ranks(value, world):
    """Largest value over all ranks (the timing rule of the multi-GPU contract)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def md_config(args, st, m, world=1):
    """The workload description shared by both arms' JSON lines."""
    return {"workload": args.workload, "atoms": st.n, "box_A": float(st.box[0]), "dt_fs": DT_PS * 1e3,
            "precision": args.precision, "basis": f"rad {m.order_rad}/{m.rc_rad} A, ang {m.order_ang}/{m.rc_ang} A",
            "ann": "-".join(map(str, m.widths)), "l2": "flushed between timed steps (256 MB write)",
            "parallelism": "replicas" if world > 1 else "single GPU", "skin_A": args.skin}


def model_overrides(args):
    """(hidden widths, basis orders) given on the command line, or None."""
    hidden = tuple(int(x) for x in args.hidden.split("-")) if getattr(args, "hidden", None) else None
    orders = tuple(int(x) for x in args.orders.split(",")) if getattr(args, "orders", None) else None
    return hidden, orders


def workload(name, hidden=None, orders=None):
    """Structure, model and initial velocities of a named workload. water_<N>
    (N a multiple of 3) is N/3 molecules at 1.0 g/cm^3 (structure seed 10),
    amorphous_<N> the 4-species solid of N atoms (structure seed 20, as the
    27,000-atom box);
    hidden / orders override the network widths / basis orders (model-size
    sweeps)."""
    from paper_2107_11311_gb300 import inputs
    if name == "water_12288":
        st, fam, vseed = inputs.water_12288(), "water", 12
    elif name == "water_192":
        st, fam, vseed = inputs.water_192(), "water", 2
    elif name == "water_331776":
        st, fam, vseed = inputs.water_331776(), "water", 42
    elif name == "amorphous_27000":
        st, fam, vseed = inputs.amorphous_27000(), "amorphous", 22
    elif name.startswith("water_") and name[6:].isdigit() and int(name[6:]) % 3 == 0:
        st, fam, vseed = inputs.water(int(name[6:]) // 3, None, 10), "water", 12
    elif name.startswith("amorphous_") and name[10:].isdigit() and int(name[10:]) > 0:
        st, fam, vseed = inputs.amorphous(int(name[10:]), 20), "amorphous", 22
    else:
        raise SystemExit(f"unknown workload {name}")
    if hidden is None and name == "water_331776":
        hidden = (32, 32)
    m = inputs.make_model(fam, hidden=hidden, orders=orders)
    masses = m.masses[st.types] if fam == "water" else np.ones(st.n)
    if fam != "water":
        m.masses = np.ones(m.n_species)
    v = inputs.maxwell_boltzmann(masses, 300.0, seed=vseed)
    return st, m, v


class ClockSampler:
    """nvidia-smi clocks / throttle reasons, sampled every 20 ms from a process
    started before the warm-up; stop() keeps the samples taken inside the timed
    window [mark(), stop()] (and, for a window shorter than the sampling period,
    the first sample after it opened)."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None
        self.t0 = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def mark(self):
        """Opening of the timed window."""
        self.t0 = time.time()

    def _rows(self):
        import datetime
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                continue
            rows.append((ts, parts[1:]))
        return rows

    def stop(self):
        if self.proc is None:
            return None
        t1 = time.time()
        t0 = self.t0 if self.t0 is not None else t1
        deadline = t1 + 1.0
        while time.time() < deadline and not any(ts >= t0 for ts, _ in self._rows()):
            time.sleep(0.02)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = self._rows()
        os.unlink(self.path)
        inside = [r for ts, r in rows if t0 <= ts <= t1]
        if not inside:
            after = [r for ts, r in rows if ts >= t0]
            inside = after[:1]
        if not inside:
            return None
        sm = [float(r[1]) for r in inside if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in inside if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in inside for k in range(4) if r[5 + k].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(inside), "period_ms": 20}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_alu_peak_tflops(n_sm, mhz):
    """FP32 FMA pipe: 128 lanes per SM x 2 flops per FMA x clock."""
    return n_sm * 128 * 2 * mhz * 1e6 / 1e12


def cpu_baseline(args, budget_s=12.0):
    """The FP64 oracle on the host cores, on a bounded sample of the workload:
    E+F of the first frame evaluated for a contiguous block of centre atoms."""
    from oracle import oracle
    st, m, _ = workload(args.workload, *model_overrides(args))
    cores = os.cpu_count() or 1
    # a contiguous block of centre atoms large enough that the oracle's fixed
    # cost per call (cell list of the whole box) stays a small part of the time
    n_cent = min(st.n, 32768)
    mask = np.zeros(st.n, dtype=np.uint8)
    mask[:n_cent] = 1
    oracle.compute(m, st.pos, st.types, st.box, center_mask=mask, n_threads=cores)  # warm
    t0 = time.perf_counter()
    reps = 0
    while True:
        oracle.compute(m, st.pos, st.types, st.box, center_mask=mask, n_threads=cores)
        reps += 1
        if time.perf_counter() - t0 > budget_s or reps >= 50:
            break
    dt = time.perf_counter() - t0
    return {"value": n_cent * reps / dt, "unit": "atom-steps/s", "cores": cores, "kind": "oracle",
            "sample": f"{reps} E+F evaluations of {n_cent} centre atoms of {args.workload} "
                      f"(FP64, OpenMP, {cores} threads)"}


def run_reference(args, rank, world):
    """--impl reference: the FP64 oracle timed as the reference arm."""
    if rank != 0:
        return
    from oracle import oracle
    st, m, _ = workload(args.workload, *model_overrides(args))
    cores = os.cpu_count() or 1
    n_cent = min(st.n, 16384)
    mask = np.zeros(st.n, dtype=np.uint8)
    mask[:n_cent] = 1
    for _ in range(args.warmup):
        oracle.compute(m, st.pos, st.types, st.box, center_mask=mask, n_threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.compute(m, st.pos, st.types, st.box, center_mask=mask, n_threads=cores)
    dt = time.perf_counter() - t0
    value = n_cent * args.steps / dt
    line = {"metric": METRIC, "value": value, "unit": "atom-steps/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": dict(md_config(args, st, m), sample_centres=n_cent),
            "cpu_baseline": {"value": value, "unit": "atom-steps/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: E+F of {n_cent} centre atoms of {args.workload}"},
            "e2e": {"value": value, "unit": "atom-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def measure_batch(args, precision, world, dev, steps, warmup, clocks=None):
    """The batched workload, batch_512: 512 independent periodic structures
    (log-uniform 32 ... 2,048 atoms; 256 water at 1.0 g/cm^3 with the water
    model, 256 of the 4-species solid with its model). One step = E+F+virial of
    every structure. Timed: the prepared batch of each model family (launch
    tuned once, whole evaluation captured as one CUDA graph) replayed on device
    buffers, CUDA events on the library's stream, L2 flushed between steps. For
    comparison (wall clock around synchronous calls): the eager batched call
    and one call per structure (the plain form: one evaluation per structure)."""
    import torch
    from paper_2107_11311_gb300 import inputs
    wat, amo = inputs.batch_structures()
    stream = torch.cuda.Stream(device=dev)
    fams = []
    tuning = {}
    flops = 0.0
    with torch.cuda.stream(stream):
        for fam, structs in (("water", wat), ("amorphous", amo)):
            m = inputs.make_model(fam)
            off, pos, types, boxes = inputs.concat(structs)
            g = make_gpu(m, precision, stream)
            dpos, dtypes = torch.tensor(pos, device=dev), torch.tensor(types, device=dev)
            E = torch.zeros(len(structs), dtype=torch.float64, device=dev)
            F = torch.zeros((int(off[-1]), 3), dtype=torch.float64, device=dev)
            V = torch.zeros((len(structs), 3, 3), dtype=torch.float64, device=dev)
            tuning[fam] = g.batch_prepare(off, boxes, dpos, dtypes, E, F, V)
            g.batch_run()
            g.check()
            st = g.neighbor_stats()
            Kr, Ka = m.order_rad + 1, m.order_ang + 1
            flops += (force_kernel_flops(Kr, Ka, st[0], st[2]) + descriptor_kernel_flops(Kr, Ka, st[0], st[2])
                      + network_flops(m.widths, int(off[-1])))
            single = [(torch.tensor(s.pos, device=dev), torch.tensor(s.types, device=dev), s.box) for s in structs]
            fams.append((g, off, dpos, dtypes, boxes, E, F, V, single))
    n_atoms = sum(int(f[1][-1]) for f in fams)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    def graphs():
        for g, *_ in fams:
            g.batch_run()

    def eager():
        for g, off, dpos, dtypes, boxes, E, F, V, _ in fams:
            g.compute_batch(off, dpos, dtypes, boxes, energies=E, forces=F, virials=V)

    e1 = torch.zeros(1, dtype=torch.float64, device=dev)
    f1 = torch.zeros((2048, 3), dtype=torch.float64, device=dev)
    v1 = torch.zeros((3, 3), dtype=torch.float64, device=dev)

    def per_structure():
        for g, *_rest, single in fams:
            for p, t, b in single:
                g.compute(p, t, b, energy=e1, forces=f1[:p.shape[0]], virial=v1)

    def timed_wall(fn, n):
        for _ in range(warmup):
            flush.zero_()
            fn()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(n):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            tot += time.perf_counter() - t0
        return tot

    clk = None
    with torch.cuda.stream(stream):
        for _ in range(warmup):
            flush.zero_()
            graphs()
        torch.cuda.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        if clocks is not None:
            clocks.mark()
        for k in range(steps):
            flush.zero_()
            starts[k].record(stream)
            graphs()
            ends[k].record(stream)
        torch.cuda.synchronize()
        if clocks is not None:
            clk = clocks.stop()
        for g, *_ in fams:
            g.check()
        t_graph = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / 1e3, world)
        steps_e = max(1, steps // 4)
        t_eager = timed_wall(eager, steps_e)
        steps_s = max(1, steps // 10)
        t_single = timed_wall(per_structure, steps_s)
    for g, *_ in fams:
        g.close()
    return {"n_atoms": n_atoms, "flops": flops, "tuning": tuning, "t_graph": t_graph, "clocks": clk,
            "value": world * n_atoms * steps / t_graph, "ms_per_step": 1e3 * t_graph / steps,
            "eager_batched_call": {"value": n_atoms * steps_e / t_eager, "ms_per_step": 1e3 * t_eager / steps_e},
            "per_structure_launches": {"value": n_atoms * steps_s / t_single,
                                       "ms_per_step": 1e3 * t_single / steps_s}}


def run_batch(args, rank, world):
    """--workload batch_512: the batched workload (measure_batch) as the line's
    own workload."""
    import torch
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = torch.device("cuda")
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    b = measure_batch(args, args.precision, world, dev, args.steps, args.warmup, clocks)
    if rank == 0:
        props = torch.cuda.get_device_properties(dev)
        peaks, peak_kind = measured_peaks()
        max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
        peak = fp32_alu_peak_tflops(props.multi_processor_count, max_mhz)
        achieved = b["flops"] / (b["t_graph"] / args.steps) / 1e12
        line = {"metric": METRIC, "value": b["value"], "unit": "atom-steps/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": b["ms_per_step"], "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": FORM_DTYPE[args.precision],
                "data": "synthetic",
                "config": {"workload": "batch_512", "structures": 512, "atoms": b["n_atoms"],
                           "sizes": "log-uniform 32..2048; 256 water + 256 4-species solid",
                           "precision": args.precision, "l2": "flushed between steps (256 MB write)",
                           "timing": "CUDA events around the replay of both prepared batches (one graph each)",
                           "tuning": b["tuning"]},
                "gpu_launches": sum(t["kernels"] for t in b["tuning"].values()) * args.steps,
                "roofline": {"bound": "alu", "kernel": "whole batched evaluation (both graphs; k_potential dominant)",
                             "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                             "traffic": None,
                             "peak_basis": f"FP32 FMA pipe: {props.multi_processor_count} SMs x 128 x 2 flops x "
                                           f"{max_mhz:.0f} MHz (SM clock max from MEASURED_PEAKS.json, {peak_kind})"},
                "clocks": b["clocks"],
                "eager_batched_call": b["eager_batched_call"],
                "per_structure_launches": b["per_structure_launches"]}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


# precision forms: the network in FP32 (fp32: the library's automatic choice of
# the MD step, which for the water basis builds the exact neighbour list in every
# step and runs the list-driven kernel; fp32_cell: the fused kernel searching the
# cells itself), split BF16 and plain BF16 on the tensor cores inside the fused
# kernel, and the same two as the three-kernel path (descriptor kernel, network
# kernel, force kernel)
FORM_DTYPE = {"fp32": "f32", "fp32_cell": "f32", "fp32_pipelined": "f32", "bf16x3": "bf16x3", "bf16": "bf16",
              "bf16x3_split": "bf16x3", "bf16_split": "bf16"}


def make_gpu(m, form, stream, skin=0.0):
    """A library context for one form on the given torch stream."""
    from paper_2107_11311_gb300.aenet import AenetGPU
    gpu = AenetGPU(m, form.replace("_split", "").replace("_pipelined", "").replace("_cell", ""),
                   stream=stream.cuda_stream)
    if form.endswith("_split"):
        gpu.fuse_network(False)
    if form.endswith("_pipelined"):  # the FP32 fused kernel's pipelined form (AENET_OPT_PIPELINE)
        gpu.pipeline(True)
    if form.endswith("_cell"):  # MD steps: the fused kernel searches the cells (AENET_OPT_MD_LIST off)
        gpu.md_list("off")
    gpu.set_skin(skin)
    return gpu


F_RMS_BOUND = 1e-3  # eV/A: the force-error bound a form must meet to be the headline


def time_form(args, st, m, v0, precision, dev, stream, flush, world):
    """One precision form: W warm-up and K timed MD steps (graph replay, CUDA
    events on the library's stream, L2 flushed before each step)."""
    import torch
    import torch.distributed as dist
    from paper_2107_11311_gb300.aenet import (AENET_MD_ASYNC, AENET_MD_CONTINUE, AENET_MD_TIMING,
                                              AENET_MD_TIMING_POTENTIAL)
    gpu = make_gpu(m, precision, stream, args.skin)
    pos = torch.tensor(st.pos, device=dev)
    vel = torch.tensor(v0, device=dev)
    types = torch.tensor(st.types, device=dev)
    with torch.cuda.stream(stream):
        gpu.md_nve(pos, vel, types, st.box, DT_PS, 1)  # initial forces + graph capture
        # timed steps record events only around the potential (each event node
        # adds ~2 us to a step); the full stage breakdown comes from extra steps
        # after the timed ones
        flags = AENET_MD_ASYNC | AENET_MD_CONTINUE | AENET_MD_TIMING_POTENTIAL
        for _ in range(args.warmup):
            flush.zero_()
            gpu.md_nve(pos, vel, types, st.box, DT_PS, 1, flags=flags)
        gpu.check()
        stats = gpu.neighbor_stats()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        stage_sum = None
        kernels_per_step, fused = 0, False
        builds0 = gpu.md_list_builds()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            gpu.md_nve(pos, vel, types, st.box, DT_PS, 1, flags=flags)
            ends[k].record(stream)
            ms, kernels_per_step, fused = gpu.md_stage_times()  # synchronises: per-step stage times
            stage_sum = ms if stage_sum is None else {s: (None if ms[s] is None else stage_sum[s] + ms[s])
                                                      for s in ms}
        torch.cuda.synchronize()
        gpu.check()
        from paper_2107_11311_gb300.aenet import AENET_PATH_LIST
        list_form = bool(gpu.md_path_flags() & AENET_PATH_LIST)
        builds = gpu.md_list_builds() - builds0
        step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
        # untimed: the full stage breakdown (every stage bracketed by events)
        n_diag = 5
        diag = None
        for _ in range(n_diag):
            flush.zero_()
            gpu.md_nve(pos, vel, types, st.box, DT_PS, 1, flags=AENET_MD_ASYNC | AENET_MD_CONTINUE | AENET_MD_TIMING)
            ms_full, _, _ = gpu.md_stage_times()
            diag = ms_full if diag is None else {s: diag[s] + ms_full[s] for s in ms_full}
        gpu.check()
    gpu.close()
    t_dev = max_over_ranks(sum(step_ms) / 1e3, world)
    return {"precision": precision, "t_dev": t_dev, "value": world * st.n * args.steps / t_dev,
            "ms_per_step": 1e3 * t_dev / args.steps, "stats": stats, "fused": fused, "list": list_form,
            "kernels_per_step": kernels_per_step, "builds": builds,
            "stage_ms": {s: (None if v is None else v / args.steps) for s, v in stage_sum.items()},
            "stage_full": {s: round(v / n_diag, 5) for s, v in diag.items()}}


def form_accuracy(st, m, precision, ref, dev, stream):
    """Energy and force errors of one form on frame 0 against the FP64 oracle
    (every atom): |dE|/N, force RMS over all 3N components, largest component
    error, and the RMS of the oracle's forces (the scale the errors sit on)."""
    import torch
    g = make_gpu(m, precision, stream)
    with torch.cuda.stream(stream):
        E = torch.zeros(1, dtype=torch.float64, device=dev)
        F = torch.zeros((st.n, 3), dtype=torch.float64, device=dev)
        g.compute(torch.tensor(st.pos, device=dev), torch.tensor(st.types, device=dev), st.box, energy=E, forces=F)
        stream.synchronize()
    g.close()
    dF = F.cpu().numpy() - ref["forces"]
    return {"e_err_per_atom": abs(E.item() - ref["energy"]) / st.n,
            "f_rms_err": float(np.sqrt((dF ** 2).mean())), "f_max_err": float(np.abs(dF).max()),
            "f_rms": float(np.sqrt((ref["forces"] ** 2).mean()))}


def roofline_of(form, m, n, props, max_mhz, peak_kind, workload_name):
    """Roofline of the form's dominant kernel: algorithmic FP32 flops per launch
    (unit counts of the launch x per-unit figures) over its event-timed
    duration, against the FP32 FMA peak."""
    stats = form["stats"]
    Kr, Ka = m.order_rad + 1, m.order_ang + 1
    f_desc = descriptor_kernel_flops(Kr, Ka, stats[0], stats[2])
    f_force = force_kernel_flops(Kr, Ka, stats[0], stats[2])
    if form["fused"]:
        dom = "forces"  # descriptor, networks and forces run as one kernel, timed under "forces"
        kernel = ("k_potential_list (descriptor + network + forces over the neighbour list built in the step)"
                  if form.get("list") else "k_potential (fused neighbour search + descriptor + network + forces)")
        flops = f_desc + f_force + network_flops(m.widths, n)
    else:
        dom = max(("descriptor", "forces"), key=lambda s: form["stage_ms"][s] or 0.0)
        kernel = "k_potential, forces mode" if dom == "forces" else "k_potential, descriptor mode"
        flops = f_force if dom == "forces" else f_desc
    ms = form["stage_ms"][dom]
    achieved = flops / (ms * 1e-3) / 1e12
    peak = fp32_alu_peak_tflops(props.multi_processor_count, max_mhz)
    return {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "flops_per_launch": flops, "launch_ms": ms,
            "traffic": (captured_traffic(workload_name, form["precision"], kernel.split()[0])
                        if form["fused"] else None),
            "peak_basis": f"FP32 FMA pipe: {props.multi_processor_count} SMs x 128 x 2 flops x {max_mhz:.0f} MHz "
                          f"(SM clock max from MEASURED_PEAKS.json, {peak_kind})"}


def e2e_rate(args, st, m, precision, pos, vel, types, stream, world):
    """The same metric end to end through aenet_md_nve with pinned host buffers:
    every step copies positions, velocities and types in and positions,
    velocities and energies out."""
    import torch
    from paper_2107_11311_gb300.aenet import AENET_MD_CONTINUE
    n = st.n
    hpos = torch.empty((n, 3), dtype=torch.float64, pin_memory=True)
    hvel = torch.empty((n, 3), dtype=torch.float64, pin_memory=True)
    htypes = torch.empty(n, dtype=torch.int32, pin_memory=True)
    hep = torch.empty(2, dtype=torch.float64, pin_memory=True)
    hek = torch.empty(2, dtype=torch.float64, pin_memory=True)
    hpos.copy_(torch.as_tensor(pos))
    hvel.copy_(torch.as_tensor(vel))
    htypes.copy_(torch.as_tensor(types))
    e2 = make_gpu(m, precision, stream, args.skin)
    e2.md_nve(hpos, hvel, htypes, st.box, DT_PS, 1, e_pot=hep, e_kin=hek)
    for _ in range(3):
        e2.md_nve(hpos, hvel, htypes, st.box, DT_PS, 1, e_pot=hep, e_kin=hek, flags=AENET_MD_CONTINUE)
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        e2.md_nve(hpos, hvel, htypes, st.box, DT_PS, 1, e_pot=hep, e_kin=hek, flags=AENET_MD_CONTINUE)
    t_e2e = max_over_ranks(time.perf_counter() - t0, world)
    h2d = hpos.numel() * 8 + hvel.numel() * 8 + htypes.numel() * 4
    d2h = hpos.numel() * 8 + hvel.numel() * 8 + hep.numel() * 8 + hek.numel() * 8
    e2.close()
    return {"value": world * n * args.e2e_steps / t_e2e, "unit": "atom-steps/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "form": precision}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--forms", default="fp32,fp32_cell,bf16x3,bf16,bf16x3_split",
                    help="precision forms timed side by side (comma-separated: fp32, fp32_cell, bf16x3, bf16, "
                         "bf16x3_split, bf16_split, fp32_pipelined)")
    ap.add_argument("--precision", default=None, choices=sorted(FORM_DTYPE),
                    help="time this form only (same as --forms <form>)")
    ap.add_argument("--workload", default="water_331776")
    ap.add_argument("--e2e-steps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the oracle comparison of each form (sweeps); the headline is then the first form")
    ap.add_argument("--hidden", default=None, help="hidden widths, e.g. 25-25 (model-size sweeps)")
    ap.add_argument("--orders", default=None, help="basis orders N_r,N_a, e.g. 5,3 (model-size sweeps)")
    ap.add_argument("--no-batched", action="store_true",
                    help="skip the batched-form comparison (batch_512 graphs vs one call per structure)")
    ap.add_argument("--skin", type=float, default=0.0,
                    help="Verlet-list skin in A for the MD step (0, the default: cell list every step)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    forms = [args.precision] if args.precision else [f.strip() for f in args.forms.split(",") if f.strip()]
    for f in forms:
        if f not in FORM_DTYPE:
            raise SystemExit(f"unknown form {f}")
    args.precision = forms[0]

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "batch_512":
        run_batch(args, rank, world)
        return

    import torch
    import torch.distributed as dist

    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    st, m, v0 = workload(args.workload, *model_overrides(args))
    n = st.n
    stream = torch.cuda.Stream(device=dev)
    # L2 flush buffer (> 129 MB L2)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    clocks = ClockSampler(local)
    clocks.start()  # running before the warm-up, so the timed window is sampled
    clocks.mark()
    wall0 = time.perf_counter()
    results = {f: time_form(args, st, m, v0, f, dev, stream, flush, world) for f in forms}
    wall = time.perf_counter() - wall0
    clk = clocks.stop()

    # accuracy of every form against the FP64 oracle (frame 0, all atoms)
    acc = {}
    if not args.no_accuracy and rank == 0:
        from oracle import oracle
        ref = oracle.compute(m, st.pos, st.types, st.box, n_threads=os.cpu_count() or 1)
        for f in forms:
            acc[f] = form_accuracy(st, m, f, ref, dev, stream)
    within = [f for f in forms if f in acc and acc[f]["f_rms_err"] <= F_RMS_BOUND]
    if args.no_accuracy:
        best = forms[0]
    else:
        best = max(within, key=lambda f: results[f]["value"]) if within else forms[0]
    R = results[best]

    # ---- end to end through the C ABI with pinned host buffers (the headline form)
    e2e = None
    if args.e2e_steps > 0:
        e2e = e2e_rate(args, st, m, best, st.pos, v0, st.types, stream, world)

    # ---- the batched form against one call per structure (batch_512, FP32)
    batched = None
    if not args.no_batched:
        bsteps = max(5, args.steps // 2)
        b = measure_batch(args, "fp32", world, dev, bsteps, args.warmup)
        batched = {"workload": "batch_512", "structures": 512, "atoms": b["n_atoms"], "precision": "fp32",
                   "steps": bsteps, "value": b["value"], "ms_per_step": b["ms_per_step"],
                   "timing": "CUDA events around the replay of both prepared batches (one graph each); "
                             "the other two: wall clock around synchronous calls",
                   "eager_batched_call": b["eager_batched_call"],
                   "per_structure_launches": b["per_structure_launches"],
                   "speedup_vs_per_structure": b["value"] / b["per_structure_launches"]["value"]}

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    props = torch.cuda.get_device_properties(dev)
    peaks, peak_kind = measured_peaks()
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    forms_out = {}
    for f in forms:
        r = results[f]
        rl = roofline_of(r, m, n, props, max_mhz, peak_kind, args.workload)
        forms_out[f] = dict({"value": r["value"], "ms_per_step": r["ms_per_step"], "fused": r["fused"],
                             "neighbour_list_every_step": r["list"],
                             "kernels_per_step": r["kernels_per_step"], "roofline_frac": rl["frac"],
                             "stage_ms": {s: round(v, 5) for s, v in r["stage_ms"].items() if v is not None},
                             "meets_1meV_per_A": (f in within) if acc else None},
                            **acc.get(f, {}))
    line = {
        "metric": METRIC, "value": R["value"], "unit": "atom-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": R["ms_per_step"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": FORM_DTYPE[best], "data": "synthetic",
        "config": dict(md_config(args, st, m, world), precision=best, neighbour_entries=R["stats"][0],
                       angular_pairs=R["stats"][2], list_builds=R["builds"] if args.skin > 0 else None,
                       headline_rule="fastest form whose force RMS error against the FP64 oracle "
                                     "(frame 0, all atoms) is <= 1 meV/A"),
        "forms": forms_out,
        "stage_ms": {s: round(v, 5) for s, v in R["stage_ms"].items() if v is not None},
        "stage_ms_all_events": R["stage_full"],
        # kernel nodes of the step graph, plus the 4 kernels of each list rebuild
        # (the body of the graph's conditional node) that ran in the timed steps
        "gpu_launches": R["kernels_per_step"] * args.steps + (4 * R["builds"] if args.skin > 0 else 0),
        "e2e": e2e,
        "batched": batched,
        "roofline": roofline_of(R, m, n, props, max_mhz, peak_kind, args.workload),
        "clocks": clk,
        "wall_s": wall,
    }
    # the same algorithmic flops over the whole MD step (every kernel of it), for
    # comparing forms whose neighbour search sits in different kernels
    rl = line["roofline"]
    rl["whole_step_frac"] = rl["flops_per_launch"] / (R["ms_per_step"] * 1e-3) / 1e12 / rl["peak"]
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
