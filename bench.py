#!/usr/bin/env python
"""Throughput of the damage-diffusion hot path on GB300: E1 pair-terms/s.

A step is one pass of the hot path over the 64x64-raster workload: the cumulative field
(Eq. 5) at 128x128 supersampled points (pitch/2) at the end of each of the 64 scan rows,
plus the dwell-start dose of all 4096 visits, FP32-mixed precision, through the C-ABI
(dd_field_at_times + dd_per_probe_dose).  One pair-term is one E1 difference phi_i(r, t)
with t_i < t.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (oracle/, plain C FP64) on a bounded sample of the
same workload on the host cores.  Under torchrun every rank runs its own copy of the
workload on its own GPU (weak scaling; no collective on the data path) and rank 0 prints
one JSON line with the whole-job throughput.
"""
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

import numpy as np  # noqa: E402

METRIC = "E1 pair-terms/s"
UNIT = "pair-terms/s"
# FP32 FLOPs of one pair term on the kernel's dominant path (moment regime, see the
# design notes): rho^2 (5 flops shared by 4 snapshots) + a, h (2) + exponent argument (1)
# + degree-8 Horner (16) + scale (1) + accumulate (1).
FLOPS_PER_PAIR = 22.25
# FP32 peak from the unit counts and the maximum clock: 152 SMs x 128 lanes x 2 x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64/e2e/CPU legs")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


class ClockSampler:
    """nvidia-smi clock / throttle samples every 100 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        sm = []
        mx = None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
            except (ValueError, IndexError):
                continue
            for name, v in zip(names, r[3:7]):
                if v.strip().lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_sha():
    h = hashlib.sha256()
    for name in ("dd_field_impl.cuh", "dd_e1.cuh", "dd_coef.cuh", "dd_field.cu"):
        with open(os.path.join(ROOT, "paper_2507_00294_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if taken on this source."""
    path = os.path.join(ROOT, "profiles", "field_mixed_raster64.md")
    if not os.path.exists(path):
        return None
    vals = {}
    for line in open(path):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel") != kernel or vals.get("source_sha") != kernel_source_sha():
        return None
    try:
        return int(vals["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def workload():
    from paper_2507_00294_gb300 import workloads as w
    job = w.raster_64_supersampled()
    n = w.n_visits(job.scan)
    ts = np.arange(n, dtype=np.float64) * job.scan.dwell_s
    field_pairs = w.causal_pairs(ts, job.times, len(job.pts_xy))
    dose_pairs = n * (n - 1) // 2
    return job, n, field_pairs, dose_pairs


def cpu_oracle_sample(job, seconds, seed=11):
    """Time the oracle on seeded (point, time) samples of the workload for ~`seconds`."""
    import oracle
    from oracle import scan as oscan
    from paper_2507_00294_gb300 import workloads as w
    s = job.scan
    xs, ys, ts, taus, _ = oscan.sources(s.nx, s.ny, s.pitch_m, s.dwell_s, order=s.order)
    src = oracle.Sources(xs, ys, ts, taus)
    cores = oracle.max_threads()

    def run(count, sd):
        ip, it = w.sample_pairs(len(job.pts_xy), len(job.times), count, seed=sd)
        pairs = int(np.searchsorted(ts, job.times[it], side="left").sum())
        t0 = time.perf_counter()
        oracle.field_pairs(src, s.sigma_m ** 2, s.D_m2s, s.Q0, job.pts_xy[ip, 0], job.pts_xy[ip, 1],
                           job.times[it])
        return pairs, time.perf_counter() - t0
    p0, t0 = run(64, seed)
    rate = p0 / max(t0, 1e-6)
    count = int(max(64, min(len(job.pts_xy) * len(job.times), rate * seconds / (p0 / 64))))
    return run, rate, count, cores


def run_reference(args):
    rank, _, world = dist_env()
    if rank != 0:
        return 0
    job, n, field_pairs, dose_pairs = workload()
    per_step_seconds = max(1.0, 150.0 / max(1, args.steps + args.warmup))
    run, rate, count, cores = cpu_oracle_sample(job, per_step_seconds)
    for k in range(args.warmup):
        run(count, 100 + k)
    pairs = 0
    secs = 0.0
    for k in range(args.steps):
        p, t = run(count, 1000 + k)
        pairs += p
        secs += t
    value = pairs / secs
    sample = ("%d seeded (point, snapshot) pairs of the workload per step (%d pair-terms per "
              "step on average), field only" % (count, pairs // max(1, args.steps)))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": job.name, "points": len(job.pts_xy), "snapshots": len(job.times),
                   "visits": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    from paper_2507_00294_gb300 import binding as b

    rank, local_rank, world = dist_env()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    b.load()
    job, n, field_pairs, dose_pairs = workload()
    pairs_step = field_pairs + dose_pairs
    scan = b.Scan(job.scan)
    pts = torch.from_numpy(job.pts_xy).to(dev)
    times = np.ascontiguousarray(job.times)
    out = torch.empty((len(times), len(job.pts_xy)), dtype=torch.float64, device=dev)
    dose = torch.empty(n, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def step(prec):
        b.dd_field_at_times(scan, pts, times, prec, out=out, stream=stream)
        b.dd_per_probe_dose(scan, prec, out=dose, stream=stream)

    for _ in range(args.warmup):
        step("mixed")
    torch.cuda.synchronize(dev)
    if dist is not None:
        dist.barrier()
    b.dd_profile_reset()
    b.dd_profile_enable(True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    with ClockSampler(local_rank) as clocks:
        for k in range(args.steps):
            flush.fill_(float(k))                    # evict L2 between steps (untimed)
            ev[k][0].record(stream)
            step("mixed")
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
    b.dd_profile_enable(False)
    prof = b.dd_profile_read()
    step_ms = [a.elapsed_time(z) for a, z in ev]
    total_ms = sum(step_ms)
    if dist is not None:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        dist.barrier()
    value = pairs_step * args.steps * world / (total_ms / 1e3)

    # roofline of the dominant kernel (field_mixed), from its own events in the timed region
    fl, fms = prof.get("field_mixed", (0, 0.0))
    avg_ms = fms / max(1, fl)
    achieved = FLOPS_PER_PAIR * field_pairs / (avg_ms / 1e3) / 1e12 if fl else None
    traffic = recorded_traffic("field_mixed")
    roofline = {"bound": "alu", "kernel": "field_mixed", "achieved": achieved,
                "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": (achieved / FP32_PEAK_TFLOPS) if achieved else None,
                "traffic": traffic, "avg_launch_ms": avg_ms,
                "flops_per_pair": FLOPS_PER_PAIR, "pairs_per_launch": field_pairs,
                "peak_note": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz (nominal max clock)"}
    launches = int(sum(v[0] for v in prof.values()))
    shares = {k: round(v[1] / max(1e-9, sum(x[1] for x in prof.values())), 4) for k, v in prof.items()}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32-mixed", "data": "synthetic",
        "config": {"workload": job.name, "scan": "64x64 raster, pitch 0.5 nm, sigma 0.1 nm, "
                   "D 6e-14 m^2/s, Q0 1 u/s, dwell 1 us", "points": len(job.pts_xy),
                   "snapshots": len(times), "visits": n, "pairs_per_step": pairs_step,
                   "field_pairs": field_pairs, "dose_pairs": dose_pairs, "precision": "mixed",
                   "l2": "flushed between steps (256 MB write, outside the timed events)",
                   "parallelism": "replica per GPU" if world > 1 else "single GPU"},
        "roofline": roofline, "gpu_launches": launches, "kernel_time_share": shares,
        "clocks": clocks.summary(),
    }

    if not args.no_extras:
        # FP64 path on the same workload (device-resident inputs)
        b.dd_profile_enable(False)
        step("fp64")
        torch.cuda.synchronize(dev)
        e64 = []
        for k in range(args.fp64_steps):
            flush.fill_(float(k))
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step("fp64")
            z.record(stream)
            e64.append((a, z))
        torch.cuda.synchronize(dev)
        ms64 = sum(a.elapsed_time(z) for a, z in e64) / len(e64)
        v64 = pairs_step / (ms64 / 1e3)
        line["fp64"] = {"value": v64, "unit": UNIT, "ms_per_step": ms64, "steps": len(e64)}
        line["mixed_over_fp64"] = (value / world) / v64

        # end to end through the public API with host buffers: scan build, H2D of the
        # points and the visit list, both kernels chains, D2H of the field and the dose
        pts_h = np.ascontiguousarray(job.pts_xy)
        out_h = np.empty((len(times), len(job.pts_xy)))
        dose_h = np.empty(n)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for k in range(args.steps):
            s2 = b.Scan(job.scan)
            b.dd_field_at_times(s2, pts_h, times, "mixed", out=out_h)
            b.dd_per_probe_dose(s2, "mixed", out=dose_h)
            s2.close()
        e2e_s = time.perf_counter() - t0
        line["e2e"] = {"value": pairs_step * args.steps / e2e_s * world, "unit": UNIT,
                       "h2d_bytes_per_step": int(pts_h.nbytes + 4 * n * 8),
                       "d2h_bytes_per_step": int(out_h.nbytes + dose_h.nbytes),
                       "ms_per_step": e2e_s / args.steps * 1e3}

        if rank == 0 and world == 1:
            run, rate, count, cores = cpu_oracle_sample(job, args.cpu_seconds)
            p, t = run(count, 7)
            line["cpu_baseline"] = {
                "value": p / t, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": "%d seeded (point, snapshot) pairs of the workload, %d pair-terms, "
                          "%.1f s, field only" % (count, p, t)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
