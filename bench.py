"""Benchmark of the ANN-potential MD hot path on GB300.

Workload (default): the 4,096-molecule water box at 1.0 g/cm^3 (12,288 atoms,
L = 49.669 A), water basis (radial order 16 / 6.0 A, angular order 8 / 4.0 A,
D = 52), per-species 52-15-15-1 tanh networks with seeded N(0, 1/fan_in)
weights, 300 K seeded velocities, velocity-Verlet NVE at dt = 0.5 fs.

One benchmark step = one MD step of the whole path (kick + drift, cell list,
descriptor, networks, forces + virial, FP64 reductions, kick), replayed from a
captured CUDA graph on device-resident state. Between timed steps the L2 cache
is flushed by writing a buffer larger than L2; each step is bracketed by CUDA
events on the library's stream and the step times are summed.

Metric: atom-steps/s (E+F). The JSON line also carries the end-to-end number
through the C ABI with host buffers (host->device copy of positions, velocities
and types, device->host copy of positions, velocities and energies, every
step), the roofline of the dominant kernel, and the FP64 CPU oracle's
throughput on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision fp32|bf16|bf16x3] [--workload water_12288|...]
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

# FP32 operations per unit of the two fingerprint kernels (FMA = 2 flops):
# per radial neighbour entry and per unordered angular pair, counted from the
# arithmetic each unit needs. Forward: the Chebyshev recurrence T_a and two
# accumulations (plain and species-weighted) per order, plus the distance,
# cutoff and weight. Backward: per order the coefficient and the Clenshaw
# steps for S = sum a_q T_q and S' = sum a_q T_q', plus the cutoff derivative,
# the radial or angle chain rule to the displacement vectors, the force
# scatter and the virial outer product.
def force_kernel_flops(Kr, Ka, n_entries, n_ang_pairs):
    """Chain rule with Clenshaw's recurrence for S and S' (9 flops per order)."""
    return (9 * (Kr - 1) + 42) * n_entries + (9 * (Ka - 1) + 57) * n_ang_pairs


def descriptor_kernel_flops(Kr, Ka, n_entries, n_ang_pairs):
    return (6 * (Kr - 1) + 10) * n_entries + (6 * (Ka - 1) + 10) * n_ang_pairs


def network_flops(widths, n_atoms):
    """Forward plus back-propagation to dE/dG: 2 x 2 flops per weight."""
    return 4 * sum(widths[l] * widths[l - 1] for l in range(1, len(widths))) * n_atoms


# DRAM bytes per launch of the dominant kernel, from the ncu captures summarised in
# profiles/k_potential_<workload>.md; reported only while the kernel source is the
# one the counters were taken on (first 16 hex digits of its SHA-256).
TRAFFIC_SOURCE_SHA256_16 = "a502f65dbc8664b2"
TRAFFIC_CAPTURE = {("water_12288", "fp32"): 521984, ("amorphous_27000", "fp32"): 1075200}


def captured_traffic(workload_name, precision, skin=0.0):
    import hashlib
    src = os.path.join(ROOT, "paper_2107_11311_gb300", "csrc", "potential_kernels.cuh")
    with open(src, "rb") as f:
        sha = hashlib.sha256(f.read()).hexdigest()[:16]
    if sha != TRAFFIC_SOURCE_SHA256_16 or skin != 0.0:
        return None
    return TRAFFIC_CAPTURE.get((workload_name, precision))


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
    (N a multiple of 3) is N/3 molecules at 1.0 g/cm^3 (structure seed 10);
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
    n_cent = min(st.n, 2048)
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
    n_cent = min(st.n, 1024)
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


def run_batch(args, rank, world):
    """--workload batch_512: 512 independent periodic structures (log-uniform 32 ...
    2,048 atoms; 256 water at 1.0 g/cm^3 with the water model, 256 of the
    4-species solid with its model). One step = E+F+virial of every structure.
    Timed: the prepared batch of each model family (launch tuned once, whole
    evaluation captured as one CUDA graph) replayed on device buffers, CUDA events
    on the library's stream, L2 flushed between steps. For comparison (wall clock
    around synchronous calls): the eager batched call and one call per structure."""
    import torch
    from paper_2107_11311_gb300 import inputs
    from paper_2107_11311_gb300.aenet import AenetGPU
    torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
    dev = torch.device("cuda")
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    wat, amo = inputs.batch_structures()
    stream = torch.cuda.Stream(device=dev)
    fams = []
    tuning = {}
    flops = 0.0
    with torch.cuda.stream(stream):
        for fam, structs in (("water", wat), ("amorphous", amo)):
            m = inputs.make_model(fam)
            off, pos, types, boxes = inputs.concat(structs)
            g = AenetGPU(m, args.precision, stream=stream.cuda_stream)
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

    def timed_wall(fn, steps):
        for _ in range(args.warmup):
            flush.zero_()
            fn()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(steps):
            flush.zero_()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn()
            torch.cuda.synchronize()
            tot += time.perf_counter() - t0
        return tot

    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            graphs()
        torch.cuda.synchronize()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        clocks.mark()
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            graphs()
            ends[k].record(stream)
        torch.cuda.synchronize()
        clk = clocks.stop()
        for g, *_ in fams:
            g.check()
        t_graph = max_over_ranks(sum(s.elapsed_time(e) for s, e in zip(starts, ends)) / 1e3, world)
        t_eager = timed_wall(eager, max(1, args.steps // 4))
        steps_s = max(1, args.steps // 10)
        t_single = timed_wall(per_structure, steps_s)
    steps_e = max(1, args.steps // 4)
    if rank == 0:
        props = torch.cuda.get_device_properties(dev)
        peaks, peak_kind = measured_peaks()
        max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
        peak = fp32_alu_peak_tflops(props.multi_processor_count, max_mhz)
        achieved = flops / (t_graph / args.steps) / 1e12
        line = {"metric": METRIC, "value": world * n_atoms * args.steps / t_graph, "unit": "atom-steps/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * t_graph / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else args.precision,
                "data": "synthetic",
                "config": {"workload": "batch_512", "structures": 512, "atoms": n_atoms,
                           "sizes": "log-uniform 32..2048; 256 water + 256 4-species solid",
                           "precision": args.precision, "l2": "flushed between steps (256 MB write)",
                           "timing": "CUDA events around the replay of both prepared batches (one graph each)",
                           "tuning": tuning},
                "gpu_launches": sum(t["kernels"] for t in tuning.values()) * args.steps,
                "roofline": {"bound": "alu", "kernel": "whole batched evaluation (both graphs; k_potential dominant)",
                             "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                             "traffic": None,
                             "peak_basis": f"FP32 FMA pipe: {props.multi_processor_count} SMs x 128 x 2 flops x "
                                           f"{max_mhz:.0f} MHz (SM clock max from MEASURED_PEAKS.json, {peak_kind})"},
                "clocks": clk,
                "eager_batched_call": {"value": n_atoms * steps_e / t_eager, "ms_per_step": 1e3 * t_eager / steps_e},
                "per_structure_launches": {"value": n_atoms * steps_s / t_single,
                                           "ms_per_step": 1e3 * t_single / steps_s}}
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "bf16", "bf16x3"])
    ap.add_argument("--workload", default="water_12288")
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--hidden", default=None, help="hidden widths, e.g. 25-25 (model-size sweeps)")
    ap.add_argument("--orders", default=None, help="basis orders N_r,N_a, e.g. 5,3 (model-size sweeps)")
    ap.add_argument("--skin", type=float, default=0.0,
                    help="Verlet-list skin in A for the MD step (0, the default: cell list every step)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

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
    from paper_2107_11311_gb300.aenet import (AENET_MD_ASYNC, AENET_MD_CONTINUE, AENET_MD_TIMING,
                                              AENET_MD_TIMING_POTENTIAL, AenetGPU)

    if world > 1:
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    st, m, v0 = workload(args.workload, *model_overrides(args))
    n = st.n

    stream = torch.cuda.Stream(device=dev)
    gpu = AenetGPU(m, args.precision, stream=stream.cuda_stream)
    gpu.set_skin(args.skin)
    pos = torch.tensor(st.pos, device=dev)
    vel = torch.tensor(v0, device=dev)
    types = torch.tensor(st.types, device=dev)
    # L2 flush buffer (> 129 MB L2)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)

    clocks = ClockSampler(local)
    clocks.start()  # running before the warm-up, so the timed window is sampled
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
        kernels_per_step = 0
        fused = False
        builds0 = gpu.md_list_builds()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        clocks.mark()
        wall0 = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            starts[k].record(stream)
            gpu.md_nve(pos, vel, types, st.box, DT_PS, 1, flags=flags)
            ends[k].record(stream)
            ms, kernels_per_step, fused = gpu.md_stage_times()  # synchronises: per-step stage times
            stage_sum = ms if stage_sum is None else {s: (None if ms[s] is None else stage_sum[s] + ms[s])
                                                      for s in ms}
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
        clk = clocks.stop()
        gpu.check()
        builds = gpu.md_list_builds() - builds0
        step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        # untimed: the full stage breakdown (every stage bracketed by events)
        n_diag = 10
        diag = None
        for _ in range(n_diag):
            flush.zero_()
            gpu.md_nve(pos, vel, types, st.box, DT_PS, 1,
                       flags=AENET_MD_ASYNC | AENET_MD_CONTINUE | AENET_MD_TIMING)
            ms_full, _, _ = gpu.md_stage_times()
            diag = ms_full if diag is None else {s: diag[s] + ms_full[s] for s in ms_full}
        gpu.check()
    t_dev = max_over_ranks(sum(step_ms) / 1e3, world)
    value = world * n * args.steps / t_dev
    stage_avg = {s: (None if v is None else v / args.steps) for s, v in stage_sum.items()}
    stage_full = {s: round(v / n_diag, 5) for s, v in diag.items()}

    # ---- end to end through the C ABI with pinned host buffers
    e2e = None
    if args.e2e_steps > 0:
        hpos = torch.empty((n, 3), dtype=torch.float64, pin_memory=True)
        hvel = torch.empty((n, 3), dtype=torch.float64, pin_memory=True)
        htypes = torch.empty(n, dtype=torch.int32, pin_memory=True)
        hep = torch.empty(2, dtype=torch.float64, pin_memory=True)
        hek = torch.empty(2, dtype=torch.float64, pin_memory=True)
        hpos.copy_(pos.cpu())
        hvel.copy_(vel.cpu())
        htypes.copy_(types.cpu())
        e2 = AenetGPU(m, args.precision, stream=stream.cuda_stream)
        e2.set_skin(args.skin)
        e2.md_nve(hpos, hvel, htypes, st.box, DT_PS, 1, e_pot=hep, e_kin=hek)
        for _ in range(3):
            e2.md_nve(hpos, hvel, htypes, st.box, DT_PS, 1, e_pot=hep, e_kin=hek, flags=AENET_MD_CONTINUE)
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            e2.md_nve(hpos, hvel, htypes, st.box, DT_PS, 1, e_pot=hep, e_kin=hek, flags=AENET_MD_CONTINUE)
        t_e2e = max_over_ranks(time.perf_counter() - t0, world)
        h2d = hpos.numel() * 8 + hvel.numel() * 8 + htypes.numel() * 4
        d2h = hpos.numel() * 8 + hvel.numel() * 8 + hep.numel() * 8 + hek.numel() * 8
        e2e = {"value": world * n * args.e2e_steps / t_e2e, "unit": "atom-steps/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}
        e2.close()

    if rank != 0:
        gpu.close()
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel (FP32 ALU bound)
    props = torch.cuda.get_device_properties(dev)
    peaks, peak_kind = measured_peaks()
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    Kr, Ka = m.order_rad + 1, m.order_ang + 1
    flops_force = force_kernel_flops(Kr, Ka, stats[0], stats[2])
    flops_desc = descriptor_kernel_flops(Kr, Ka, stats[0], stats[2])
    if fused:
        # descriptor, networks and forces run as one kernel, timed under "forces"
        dom = "forces"
        kernel_name = ("k_potential_list (fused descriptor + network + forces over the Verlet list)"
                       if args.skin > 0 else "k_potential (fused descriptor + network + forces)")
        flops = flops_force + flops_desc + network_flops(m.widths, n)
    else:
        dom = max(("descriptor", "forces"), key=lambda s: stage_avg[s])
        kernel_name = "k_fingerprint backward (forces)" if dom == "forces" else "k_fingerprint forward (descriptor)"
        flops = flops_force if dom == "forces" else flops_desc
    achieved = flops / (stage_avg[dom] * 1e-3) / 1e12
    peak = fp32_alu_peak_tflops(props.multi_processor_count, max_mhz)
    line = {
        "metric": METRIC, "value": value, "unit": "atom-steps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else args.precision,
        "data": "synthetic",
        "config": dict(md_config(args, st, m, world), neighbour_entries=stats[0], angular_pairs=stats[2],
                       list_builds=builds if args.skin > 0 else None),
        "stage_ms": {s: round(v, 5) for s, v in stage_avg.items() if v is not None},
        "stage_ms_all_events": stage_full,
        # kernel nodes of the step graph, plus the 4 kernels of each list rebuild
        # (the body of the graph's conditional node) that ran in the timed steps
        "gpu_launches": kernels_per_step * args.steps + (4 * builds if args.skin > 0 else 0),
        "e2e": e2e,
        "roofline": {"bound": "alu", "kernel": kernel_name, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak,
                     "traffic": captured_traffic(args.workload, args.precision, args.skin) if fused else None,
                     "peak_basis": f"FP32 FMA pipe: {props.multi_processor_count} SMs x 128 x 2 flops x {max_mhz:.0f} MHz "
                                   f"(SM clock max from MEASURED_PEAKS.json, {peak_kind})"},
        "clocks": clk,
        "wall_s": wall,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args)
    print(json.dumps(line), flush=True)
    gpu.close()
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
