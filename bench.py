#!/usr/bin/env python
"""Throughput of the damage-diffusion hot path on GB300: E1 pair-terms/s.

A step is one pass of the hot path over the 64x64-raster workload: the cumulative field
(Eq. 5) at 128x128 supersampled points (pitch/2) at the end of each of the 64 scan rows,
plus the dwell-start dose of all 4096 visits, FP32-mixed precision, through the C-ABI
(dd_field_at_times + dd_per_probe_dose).  One pair-term is one E1 difference phi_i(r, t)
with t_i < t.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (oracle/, plain C FP64) on a bounded sample of the
same workload on the host cores.  Under torchrun the step is split across the ranks
(strong scaling): each GPU evaluates a range of point tiles at every snapshot and a
cost-balanced range of dose targets, the outputs are all-gathered once per step, and
rank 0 prints one JSON line with the whole-job throughput (MAX of the ranks' times).
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
# Algorithmic cost of one pair term on each path of the field kernel's FP32 exponent
# series (FMA = 2 flops): rho^2 costs 5 flops per (point, visit), shared by the 4
# snapshots of a chunk (1.25 per pair); a series path of degree d adds its exponent (2d
# flops for d = 2, 4 in rho^2; 2d + 1 for d = 8, 12 in h) and the accumulating add, plus
# one ex2 (degree 2 up to h = 0.04, 4 up to 0.33, 8 up to 1.25, 12 up to 2.0); the
# general path (two E1 values) about 55 flops and 4 MUFU operations (2 ex2, 2 rcp); a
# pair with a >= 87 only its rho^2.
FLOPS_SERIES = {2: 6.25, 4: 10.25, 8: 19.25, 12: 27.25}
FLOPS_GENERAL = 56.25
FLOPS_ZERO = 1.25
MUFU_SERIES, MUFU_GENERAL = 1.0, 4.0
# The same on a grid tile (128 columns x 4 rows x 4 snapshots, dd_field_on_grid): dx and
# dx^2 cost 2 flops per (column, visit), shared by 16 pairs (0.125); rho^2 = dx^2 + dy^2 one
# FMA per (point, visit), shared by 4 snapshots (0.5).  A degree-2 pair is X Y (+ A B):
# the column factor X = 2^(g_0 + g_1x dx^2 + g_2x dx^4) costs 2 FMAs and one ex2 per
# (column, visit, snapshot), shared by the 4 rows (1 flop, 0.25 ex2 per pair); the row
# factor Y is shared by 128 columns (~0.02 flops, 0.008 ex2); the pair itself one FMA (2
# flops); where the cross term is needed, A = X (2 ln2 g_2x) dx^2 (3 multiplies per
# column, visit and snapshot: 0.75) and one more FMA (2).  Higher degrees as above with
# the grid's rho^2 (0.625 instead of 1.25).
GRID_FLOPS_SEP1, GRID_FLOPS_SEP2, GRID_MUFU_SEP = 3.17, 5.92, 0.258
GRID_FLOPS_RHO, GRID_FLOPS_ZERO = 0.625, 0.125
# FP32 peak from the unit counts and the maximum clock: 152 SMs x 128 lanes x 2 x 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# FP64 FMA peak: 1.6 per clock per SM (a microbenchmark on this GPU: 0.50 T DFMA/s at
# 1.995 GHz) x 152 x 2.07 GHz.
FP64_PEAK_TDFMA = 152 * 1.6 * 2.07e9 / 1e12
# MUFU ex2 peak: 32 per clock per SM (GB300 doubles the SFU exponential rate of B200; a
# microbenchmark on this GPU measured 30.6 per clock per SM at 1.995 GHz) x 152 x 2.07 GHz.
MUFU_PEAK_TOPS = 152 * 32 * 2.07e9 / 1e12
L2_FLUSH_BYTES = 256 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64/e2e/CPU/batch/surrogate legs")
    ap.add_argument("--surrogate-maps", type=int, default=20000)
    ap.add_argument("--surrogate-epochs", type=int, default=60)
    ap.add_argument("--no-surrogate", action="store_true")
    ap.add_argument("--leg", choices=["all", "batched", "surrogate-infer", "surrogate", "dose"], default="all",
                    help="run one leg alone (for profiling): the 512-scan batch, or the surrogate "
                         "network's inference at batch 256 (random weights)")
    return ap.parse_args()


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("LOCAL_RANK", 0)),
            int(os.environ.get("WORLD_SIZE", 1)))


class ClockSampler:
    """nvidia-smi clock / throttle samples every PERIOD_MS (10 ms), each stamped with the host clock.

    The timed region of a short run lasts tens of milliseconds, so the sampler is started
    first and the region opens only once a sample has arrived; `mark()` brackets the region
    (after the closing synchronise, so it covers the device work) and `summary()` keeps the
    samples inside it."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 10

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None
        self.window = None
        self.first = threading.Event()

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            self.first.wait(timeout=10.0)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.monotonic(), [c.strip() for c in line.split(",")]))
            self.first.set()

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(2.0 * self.PERIOD_MS / 1e3)   # the sample that closes the window
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.thread.join(timeout=2)

    def summary(self):
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = self.rows
        where = "inside the timed region"
        if self.window is not None:
            t0, t1 = self.window
            inside = [r for r in rows if t0 <= r[0] <= t1]
            if inside:
                rows = inside
            else:
                # no sample fell inside: keep the ones nearest either edge of the region
                near = sorted(rows, key=lambda r: min(abs(r[0] - t0), abs(r[0] - t1)))[:2]
                rows, where = near, "nearest the timed region (none fell inside it)"
        sm = []
        mx = None
        reasons = set()
        for _, r in rows:
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
                "samples": len(sm), "period_ms": self.PERIOD_MS, "window": where}


def whole_job(job_pairs_per_step, steps, rank_total_ms, dist=None, device=None):
    """Whole-job throughput: the job's work is the whole workload (split across the ranks
    when there are several: strong scaling), its time the slowest rank's (MAX over ranks).
    Only this timing reduction and the output gather run as collectives."""
    world = 1
    total_ms = float(rank_total_ms)
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        t = torch.tensor([total_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    return job_pairs_per_step * steps / (total_ms / 1e3), total_ms, world


# Per kernel: the ncu summary under profiles/ that records its DRAM traffic, and the
# sources whose text fixes its code (the summary's source_sha is their hash).
PROFILED = {
    "field_mixed": ("field_mixed_raster64.md", ("dd_field_impl.cuh", "dd_e1.cuh", "dd_coef.cuh")),
    "field_grid_mixed": ("field_grid_mixed_raster64.md",
                         ("dd_field_grid.cuh", "dd_field_impl.cuh", "dd_e1.cuh", "dd_coef.cuh")),
}


def kernel_source_sha(kernel):
    h = hashlib.sha256()
    for name in PROFILED[kernel][1]:
        with open(os.path.join(ROOT, "paper_2507_00294_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_profile(kernel):
    """The "- key: value" lines of the committed ncu summary, if taken on this source."""
    path = os.path.join(ROOT, "profiles", PROFILED[kernel][0])
    if not os.path.exists(path):
        return {}
    vals = {}
    for line in open(path):
        if ":" in line and line.strip().startswith("- "):
            k, v = line.strip()[2:].split(":", 1)
            vals[k.strip()] = v.strip()
    if vals.get("kernel") != kernel or vals.get("source_sha") != kernel_source_sha(kernel):
        return {}
    return vals


def recorded_traffic(kernel):
    """DRAM bytes per launch from the committed ncu summary, if taken on this source."""
    try:
        return int(recorded_profile(kernel)["dram_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def recorded_pipes(kernel):
    """Pipe and issue utilisation of the committed ncu capture (fractions), if taken on this
    source: what the kernel keeps busy, beside the algorithmic fraction of the roofline."""
    vals = recorded_profile(kernel)
    keys = {"fma_pipe_pct": "fma_pipe", "xu_pipe_pct": "xu_pipe", "issue_active_pct": "issue_active"}
    try:
        out = {name: float(vals[k]) / 100.0 for k, name in keys.items()}
        out["thread_instructions_per_pair"] = float(vals["thread_instructions_per_pair"])
    except (KeyError, ValueError):
        return None
    out["note"] = ("ncu --set full capture of one launch on this source (profiles/%s): pipe busy "
                   "fractions and issue-slot use per SM sub-partition" % PROFILED[kernel][0])
    return out


# BF16 tensor-core peak: the measured cuBLAS burst figure, else the recipe's fallback
def bf16_peak_tflops():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured (cuBLAS bf16 burst, MEASURED_PEAKS.json)"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback (1.9 PFLOP/s bf16)"


def tensor_core_line(prof, kernel, tc_pairs, flops_per_pair):
    """A tensor-core contraction of the grid field: field_grid_tc (degree 2: 7 BF16 MMAs of 2
    flops per (row, column, visit) triple, 14 tensor flops per pair-term) or field_grid_tc4
    (degree 4: 12 MMAs, 24 flops).  Its event time runs from its launch on the side stream to
    its end, overlapping the CUDA-core tile kernel (whose CTAs are placed first), so the rate
    below is a lower bound of what it does alone."""
    n, ms = prof.get(kernel, (0, 0.0))
    if not n or not tc_pairs:
        return None
    avg = ms / n
    peak, note = bf16_peak_tflops()
    achieved = flops_per_pair * tc_pairs / (avg / 1e3) / 1e12
    return {"kernel": kernel, "bound": "tensor", "pairs_per_launch": tc_pairs, "flops_per_pair": flops_per_pair,
            "avg_launch_ms": avg, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "peak_note": note, "note": "event time overlaps the CUDA-core tile kernel (side stream)"}


def cumulant_l2(r):
    """l_2 of the FP32 record's exponent series (half the variance of s under the weight
    r / (1 + r s) on [0, 1]), by a 2000-node midpoint rule: enough to place a pair in the
    degree-2 class with or without the cross term."""
    sg = (np.arange(2000) + 0.5) / 2000
    out = np.empty(len(r))
    for k0 in range(0, len(r), 4096):
        rr = r[k0:k0 + 4096, None]
        wgt = rr / (1 + rr * sg[None, :])
        m0 = wgt.mean(1)
        m1 = (wgt * sg).mean(1) / m0
        m2 = (wgt * sg ** 2).mean(1) / m0
        out[k0:k0 + 4096] = 0.5 * (m2 - m1 ** 2)
    return out


def ops_per_pair(job, samples=400_000, seed=5, grid=False, prefix=None):
    """Algorithmic FP32 FLOPs and MUFU operations per pair-term of the field kernel on this
    workload: the cost of the cheapest path that meets the FP32 accuracy target for each
    pair (series degree from that pair's own h, zero when a >= 87; on a grid, the degree-2
    pairs in their separable form, with the cross term where its size 2 g_2x dx^2 dy^2
    exceeds the 2.5e-7 budget), averaged over seeded pairs.  prefix[j]: visits of snapshot
    j that the tensor-core contraction takes (the CUDA-core tile kernel sums the rest; the
    pairs sampled here are its pairs)."""
    from paper_2507_00294_gb300 import workloads as w
    s = job.scan
    rng = np.random.default_rng(seed)
    n = w.n_visits(s)
    ts = np.arange(n) * s.dwell_s
    it = rng.integers(0, len(job.times), samples)
    t = job.times[it]
    nact = np.searchsorted(ts, t, side="left")
    k0 = np.zeros(samples, np.int64) if prefix is None else np.asarray(prefix, np.int64)[it]
    i = k0 + (rng.random(samples) * (nact - k0)).astype(np.int64)
    ip = rng.integers(0, len(job.pts_xy), samples)
    g = i                                        # raster: visit k is grid index k
    dx = job.pts_xy[ip, 0] - (g % s.nx) * s.pitch_m
    dy = job.pts_xy[ip, 1] - (g // s.nx) * s.pitch_m
    rho2 = dx * dx + dy * dy
    dt = t - ts[i]
    Ds, D, tau = s.sigma_m ** 2, s.D_m2s, s.dwell_s
    w1 = 2 * Ds + 4 * D * dt
    w0 = np.where(dt <= tau, 2 * Ds, 2 * Ds + 4 * D * (dt - tau))
    a, h = rho2 / w1, rho2 / w0 - rho2 / w1
    zero = a >= 87
    f = np.where(zero, FLOPS_ZERO,
                 np.where(h <= 0.04, FLOPS_SERIES[2],
                          np.where(h <= 0.33, FLOPS_SERIES[4],
                                   np.where(h <= 1.25, FLOPS_SERIES[8],
                                            np.where(h <= 2.0, FLOPS_SERIES[12], FLOPS_GENERAL)))))
    m = np.where(zero, 0.0, np.where(h <= 2.0, MUFU_SERIES, MUFU_GENERAL))
    if grid:
        # grid tile: rho^2 shared more widely, degree 2 in the separable form
        dqp = (1.0 / w0 - 1.0 / w1) * s.pitch_m ** 2                     # dq in pitch units
        rr = np.where(dt <= tau, 4 * D * dt, 4 * D * tau) / w0             # r = w1 / w0 - 1
        d2 = h <= 0.04
        cross = np.zeros(samples)
        cross[d2] = (2 * 1.4426950408889634 * cumulant_l2(rr[d2]) * dqp[d2] ** 2
                     * (dx[d2] / s.pitch_m) ** 2 * (dy[d2] / s.pitch_m) ** 2)
        sep = np.where(cross <= 2.5e-7, GRID_FLOPS_SEP1, GRID_FLOPS_SEP2)
        f = np.where(zero, GRID_FLOPS_ZERO, np.where(d2, sep, f - FLOPS_ZERO + GRID_FLOPS_RHO))
        m = np.where(zero, 0.0, np.where(d2, GRID_MUFU_SEP, m))
    wgt = (nact - k0).astype(np.float64)         # pairs are sampled per snapshot: weight by their count
    return (float(np.sum(f * wgt) / np.sum(wgt)), float(np.sum(m * wgt) / np.sum(wgt)),
            float(np.sum(zero * wgt) / np.sum(wgt)))


def dfma_per_pair_fp64(job, samples=200_000, seed=6):
    """Algorithmic FP64 operations (DFMA-equivalents) per pair of the FP64 field kernel on
    this workload: rho^2 shared by the 4 snapshots of a chunk (1), the moment polynomial of
    the cheapest degree whose range holds the pair's h (4, 8, 11, 15 up to h = 1e-3, 0.052,
    0.19, 0.5: D + 1 with the final product), exp(-a) as 15, the two-E1 path as 60, a pair
    with a >= 745 its rho^2 only."""
    from paper_2507_00294_gb300 import workloads as w
    s = job.scan
    rng = np.random.default_rng(seed)
    n = w.n_visits(s)
    ts = np.arange(n) * s.dwell_s
    it = rng.integers(0, len(job.times), samples)
    t = job.times[it]
    nact = np.searchsorted(ts, t, side="left")
    i = (rng.random(samples) * nact).astype(np.int64)
    ip = rng.integers(0, len(job.pts_xy), samples)
    dx = job.pts_xy[ip, 0] - (i % s.nx) * s.pitch_m
    dy = job.pts_xy[ip, 1] - (i // s.nx) * s.pitch_m
    rho2 = dx * dx + dy * dy
    dt = t - ts[i]
    Ds, D, tau = s.sigma_m ** 2, s.D_m2s, s.dwell_s
    w1 = 2 * Ds + 4 * D * dt
    w0 = np.where(dt <= tau, 2 * Ds, 2 * Ds + 4 * D * (dt - tau))
    a, h = rho2 / w1, rho2 / w0 - rho2 / w1
    c = np.where(a >= 745, 1.0, np.where(h <= 1e-3, 1 + 5 + 15, np.where(h <= 0.052, 1 + 9 + 15,
                 np.where(h <= 0.19, 1 + 12 + 15, np.where(h <= 0.5, 1 + 16 + 15, 1 + 60)))))
    return float(np.sum(c * nact) / np.sum(nact))


# Batch grid tile (32 x 32 points, one snapshot, 8 rows per thread): a degree-2 pair is one
# FMA (2 flops) plus its share of the column factor X (2 FMAs and one ex2 per column and
# visit, shared by 8 rows: 0.5 flops, 0.125 ex2) and of dx, dx^2 (0.25); with the cross term
# A = X (2 ln2 g_2x) dx^2 (3 multiplies / 8 = 0.375) and one more FMA (2); degree 4 and above
# per point with rho^2 = dx^2 + dy^2 (one FMA, 2 flops).
# per class: zero (a >= 87), degree 2 without / with the cross term, degree 4, 8, 12, two E1
BATCH_FLOPS = np.array([0.25, 2.75, 5.125, 2.0 + 8.0 + 1.0, 2.0 + 17.0 + 1.0, 2.0 + 25.0 + 1.0, 2.0 + 55.0])
BATCH_MUFU = np.array([0.0, 0.125, 0.125, 1.0, 1.0, 1.0, 4.0])


def batch_ops_per_pair(jobs, samples=200_000, seed=7, prefix=None):
    """Algorithmic FP32 flops and ex2 per pair-term of the batch grid kernel on the 512-scan
    workload (each pair at the cheapest class its own h allows, degree 2 with the cross term
    where 2 g_2x dx^2 dy^2 exceeds 2.5e-7), pairs sampled in proportion to each scan's.
    prefix[k]: visits of scan k that the tensor-core contraction takes (the pairs sampled
    are then the CUDA-core tile kernel's own)."""
    from paper_2507_00294_gb300 import binding as b
    from paper_2507_00294_gb300 import workloads as w
    rng = np.random.default_rng(seed)
    k0 = np.zeros(len(jobs), np.int64) if prefix is None else np.asarray(prefix, np.int64)
    pairs = np.array([(w.n_visits(j.scan) - k0[k]) * len(j.pts_xy) for k, j in enumerate(jobs)], dtype=np.float64)
    ks = rng.choice(len(jobs), samples, p=pairs / pairs.sum())
    code = np.empty(samples, dtype=np.int64)
    for k in np.unique(ks):
        sel = np.nonzero(ks == k)[0]
        j = jobs[k]
        s = j.scan
        sc = b.Scan(s)
        g = sc.visits()[0].astype(np.int64)
        sc.close()
        nv = len(g)
        i = rng.integers(k0[k], nv, len(sel))
        ip = rng.integers(0, len(j.pts_xy), len(sel))
        dx = j.pts_xy[ip, 0] / s.pitch_m - g[i] % s.nx
        dy = j.pts_xy[ip, 1] / s.pitch_m - g[i] // s.nx
        rho2 = dx * dx + dy * dy
        kap, ss = s.D_m2s * s.dwell_s / s.pitch_m ** 2, (s.sigma_m / s.pitch_m) ** 2
        L = (nv - i).astype(np.float64)                  # lag of visit i at the scan's end
        w1 = 2 * ss + 4 * kap * L
        w0 = 2 * ss + 4 * kap * (L - 1)
        dq = 1 / w0 - 1 / w1
        a, h = rho2 / w1, rho2 * dq
        cross = 2 * 1.4426950408889634 * cumulant_l2(4 * kap / w0) * dq ** 2 * dx ** 2 * dy ** 2
        code[sel] = np.where(a >= 87, 0, np.where(h <= 0.04, np.where(cross <= 2.5e-7, 1, 2),
                             np.where(h <= 0.33, 3, np.where(h <= 1.25, 4, np.where(h <= 2.0, 5, 6)))))
    return float(BATCH_FLOPS[code].mean()), float(BATCH_MUFU[code].mean())


def dose_ops_per_pair(spec, samples=200_000, seed=9):
    """Algorithmic FP32 flops and MUFU operations per pair of the dwell-start dose on a
    uniform scan: target j, source i = j - k seen k dwells later at distance rho_jk, each
    pair at the cheapest class its own h allows; rho^2 is per pair here (about 4 flops: two
    differences and one multiply-add)."""
    from paper_2507_00294_gb300 import binding as b
    rng = np.random.default_rng(seed)
    sc = b.Scan(spec)
    g = sc.visits()[0].astype(np.int64)
    sc.close()
    n = len(g)
    # pairs (j, k) uniform over the triangle k < j: j with weight j, then k uniform
    j = np.floor(np.sqrt(rng.random(samples)) * (n - 1)).astype(np.int64) + 1
    k = np.floor(rng.random(samples) * j).astype(np.int64) + 1
    i = j - k
    dx = (g[j] % spec.nx - g[i] % spec.nx).astype(np.float64)
    dy = (g[j] // spec.nx - g[i] // spec.nx).astype(np.float64)
    rho2 = dx * dx + dy * dy
    kap, ss = spec.D_m2s * spec.dwell_s / spec.pitch_m ** 2, (spec.sigma_m / spec.pitch_m) ** 2
    w1 = 2 * ss + 4 * kap * k
    w0 = 2 * ss + 4 * kap * (k - 1)
    a, h = rho2 / w1, rho2 * (1 / w0 - 1 / w1)
    rho = 4.0 - FLOPS_ZERO                               # the per-pair rho^2 in place of the shared one
    f = np.where(a >= 87, 4.0, np.where(h <= 0.04, FLOPS_SERIES[2] + rho, np.where(h <= 0.33, FLOPS_SERIES[4] + rho,
                 np.where(h <= 1.25, FLOPS_SERIES[8] + rho, np.where(h <= 2.0, FLOPS_SERIES[12] + rho,
                                                                     FLOPS_GENERAL + rho)))))
    m = np.where(a >= 87, 0.0, np.where(h <= 2.0, MUFU_SERIES, MUFU_GENERAL))
    return float(f.mean()), float(m.mean())


def bench_dose(b, dev, stream, job, n, reps=10):
    """The dwell-start dose alone: the bench workload's 4096 visits and the 256 x 256
    precision study's 65,536 (2.1e9 pairs), FP32-mixed, kernels on the device."""
    import torch
    from paper_2507_00294_gb300 import workloads as w
    out = {}
    for name, spec in (("raster64", job.scan), ("grid256_raster", w.precision_study(w.RASTER, 0).scan)):
        scan = b.Scan(spec)
        nv = len(scan)
        dose = torch.empty(nv, dtype=torch.float64, device=dev)
        for _ in range(2):
            b.dd_per_probe_dose(scan, "mixed", out=dose, stream=stream)
        torch.cuda.synchronize(dev)
        b.dd_profile_reset()
        b.dd_profile_enable(True)
        for _ in range(reps):
            b.dd_per_probe_dose(scan, "mixed", out=dose, stream=stream)
        torch.cuda.synchronize(dev)
        b.dd_profile_enable(False)
        prof = b.dd_profile_read()
        ms = sum(v[1] for v in prof.values()) / reps
        kl, kms = prof.get("dose_mixed", (0, 0.0))
        pairs = nv * (nv - 1) // 2
        fpp, mpp = dose_ops_per_pair(spec)
        krate = pairs / (kms / max(1, kl) / 1e3) if kl else None
        out[name] = {"visits": nv, "pairs": pairs, "ms": ms, "value": pairs / (ms / 1e3), "unit": UNIT,
                     "roofline": {"bound": "alu", "kernel": "dose_mixed", "pipe": "fp32",
                                  "achieved": fpp * krate / 1e12 if krate else None, "peak": FP32_PEAK_TFLOPS,
                                  "unit": "TFLOP/s", "frac": fpp * krate / 1e12 / FP32_PEAK_TFLOPS if krate else None,
                                  "mufu_frac": mpp * krate / 1e12 / MUFU_PEAK_TOPS if krate else None,
                                  "ops_per_pair": round(fpp, 2), "mufu_per_pair": round(mpp, 3),
                                  "avg_launch_ms": kms / max(1, kl)}}
        scan.close()
    return out


def workload():
    """The 64x64 raster job, its evaluation grid (x0, y0, dx, dy, columns, rows) -- the
    job's 128 x 128 points at pitch / 2 are that grid in row-major order -- and the pair
    counts of the field and the dose."""
    from paper_2507_00294_gb300 import workloads as w
    job = w.raster_64_supersampled()
    n = w.n_visits(job.scan)
    half = job.scan.pitch_m / 2
    job.extra["grid"] = (0.0, 0.0, half, half, 128, 128)
    assert np.array_equal(w.grid_points(128, half), job.pts_xy)
    ts = np.arange(n, dtype=np.float64) * job.scan.dwell_s
    field_pairs = w.causal_pairs(ts, job.times, len(job.pts_xy))
    dose_pairs = n * (n - 1) // 2
    return job, n, field_pairs, dose_pairs


def cpu_oracle_sample(job, seconds, seed=11, threads=0):
    """Time the oracle on seeded (point, time) samples of the workload for ~`seconds`, on
    `threads` host threads (0: all the cores the process may use)."""
    import oracle
    from oracle import scan as oscan
    from paper_2507_00294_gb300 import workloads as w
    s = job.scan
    xs, ys, ts, taus, _ = oscan.sources(s.nx, s.ny, s.pitch_m, s.dwell_s, order=s.order)
    src = oracle.Sources(xs, ys, ts, taus)
    cores = threads if threads > 0 else oracle.max_threads()

    def run(count, sd):
        ip, it = w.sample_pairs(len(job.pts_xy), len(job.times), count, seed=sd)
        pairs = int(np.searchsorted(ts, job.times[it], side="left").sum())
        t0 = time.perf_counter()
        oracle.field_pairs(src, s.sigma_m ** 2, s.D_m2s, s.Q0, job.pts_xy[ip, 0], job.pts_xy[ip, 1],
                           job.times[it], threads=threads)
        return pairs, time.perf_counter() - t0
    p0, t0 = run(64, seed)
    rate = p0 / max(t0, 1e-6)
    count = int(max(64, min(len(job.pts_xy) * len(job.times), rate * seconds / (p0 / 64))))
    return run, rate, count, cores


def bench_batched(dev, stream, runs=10, rank=0, world=1, dist=None, grid=True):
    """The 512-scan batched workload through one tuned, graph-replayed plan (FP32-mixed),
    each scan on its probe grid (dd_batch_create_grid; grid=False: the same points as
    lists).  With several ranks the scans are dealt out longest-first by pair count (LPT),
    each rank runs a plan of its own scans, and the fields are gathered once per run."""
    import torch
    from paper_2507_00294_gb300 import binding as b
    from paper_2507_00294_gb300 import shard
    from paper_2507_00294_gb300 import workloads as w
    jobs_all = w.batched_scans()
    costs = [w.n_visits(j.scan) * len(j.pts_xy) for j in jobs_all]     # one snapshot at the end
    total_pairs = int(sum(costs))
    mine = shard.lpt_assign(costs, world)[rank]
    jobs = [jobs_all[k] for k in mine]
    offs = np.concatenate([[0], np.cumsum([len(j.pts_xy) for j in jobs])]).astype(np.int64)
    times = np.array([j.times[0] for j in jobs])
    scans = [b.Scan(j.scan) for j in jobs]
    if grid:
        pts = None
        plan = b.Batch(scans, None, times, "mixed",
                       grids=[(0.0, 0.0, j.scan.pitch_m, j.scan.pitch_m, j.scan.nx, j.scan.ny) for j in jobs])
    else:
        pts = torch.from_numpy(np.ascontiguousarray(np.concatenate([j.pts_xy for j in jobs]))).to(dev)
        plan = b.Batch(scans, offs, times, "mixed")
    variant = plan.tune(pts)
    out = torch.empty(int(offs[-1]), dtype=torch.float64, device=dev)
    sizes = None
    if world > 1:
        n_out = torch.tensor([int(offs[-1])], device=dev)
        allsz = [torch.zeros_like(n_out) for _ in range(world)]
        dist.all_gather(allsz, n_out)
        sizes = [int(x.item()) for x in allsz]
        ranges = [(0, sz) for sz in sizes]

    def run():
        plan.run(pts, out=out, stream=stream)
        if world > 1:
            shard.gather_vector(out, ranges, rank, dist)

    for _ in range(2):
        run()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    ev = []
    for k in range(runs):
        flush.fill_(float(k))
        a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run()
        z.record(stream)
        ev.append((a, z))
    torch.cuda.synchronize(dev)
    value, ms_total, _ = whole_job(total_pairs, runs, sum(a.elapsed_time(z) for a, z in ev), dist, dev)
    info = plan.info()
    plan.close()
    roof = None
    if grid and world == 1:
        # the plan's split: the tensor-core contraction takes each scan's prefix on the
        # degree-2 (and then degree-4) series at every point of its grid (grids of at least
        # 64 x 64 points), the CUDA-core tile kernel the rest
        k2, k4 = [], []
        for j in jobs_all:
            sc = b.Scan(j.scan)
            K, K2 = b.dd_field_grid_split(sc, 0.0, 0.0, j.scan.pitch_m, j.scan.pitch_m, j.scan.nx, j.scan.ny,
                                          j.times[:1], degree2=True)
            sc.close()
            k2.append(int(K2[0]))
            k4.append(int(K[0]))
        npts = np.array([len(j.pts_xy) for j in jobs_all], dtype=np.float64)
        tc2 = float(np.sum(np.array(k2) * npts))
        tc4 = float(np.sum((np.array(k4) - np.array(k2)) * npts))
        core = total_pairs - tc2 - tc4
        fpp, mpp = batch_ops_per_pair(jobs_all, prefix=k4)
        t_run = ms_total / runs / 1e3
        rate = core / t_run
        bf16, bf16_note = bf16_peak_tflops()
        roof = {"bound": "alu", "kernel": "batch_grid_mixed_32x32", "pipe": "fp32", "achieved": fpp * rate / 1e12,
                "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": fpp * rate / 1e12 / FP32_PEAK_TFLOPS,
                "pairs_per_run": core, "ops_per_pair": round(fpp, 3), "mufu_per_pair": round(mpp, 4),
                "mufu_frac": mpp * rate / 1e12 / MUFU_PEAK_TOPS,
                "note": "the CUDA-core tile kernel's own pairs over the event time of the whole graph "
                        "(coefficients, contraction, tile kernel, reduce, one after another): a lower bound "
                        "of that kernel's rate",
                "tensor_core": {"pairs_per_run": tc2 + tc4, "degree2_pairs": tc2, "degree4_pairs": tc4,
                                "flops_per_run": 14 * tc2 + 24 * tc4,
                                "achieved": (14 * tc2 + 24 * tc4) / t_run / 1e12, "peak": bf16, "unit": "TFLOP/s",
                                "frac": (14 * tc2 + 24 * tc4) / t_run / 1e12 / bf16, "peak_note": bf16_note,
                                "note": "over the whole graph's event time: a lower bound"}}
    return {"value": value, "unit": UNIT, "ms_per_run": ms_total / runs, "runs": runs, "roofline": roof,
            "pairs_per_run": total_pairs, "rank_pairs_per_run": info["pairs"], "scans": len(jobs_all),
            "rank_scans": len(jobs), "work_items": info["items"], "tuned_variant": variant,
            "workload": "512 scans, n ~ U{32..128}, D log-U[1e-15,1e-12], "
            "dwell log-U[1e-7,1e-5] s, sigma U[0.05,0.2] nm, keep U[0.1,1], random order, final field on the n x n grid",
            "points": "each scan's probe grid, dd_batch_create_grid (older visits of grids >= 64 x 64 on "
                      "the tensor cores, the rest in 32 x 32 grid tiles)" if grid
                      else "each scan's probe grid as a point list (512-point tiles)",
            "launch": "persistent kernel, atomic work claim, CUDA graph replay" +
                      (", scans split over %d GPUs longest-first, one gather per run" % world if world > 1 else "")}


def bench_runtime_curve(dev, stream, sizes=(8, 16, 20, 32, 64), frames=(1e-6, 10e-6), reps=5):
    """Runtime vs number of probe positions for two frame times (the setting of Fig. 2):
    n x n raster, 1 us dwell, field on the probe grid at every frame time, FP32-mixed."""
    import torch
    from paper_2507_00294_gb300 import binding as b
    from paper_2507_00294_gb300 import workloads as w
    rows = []
    for frame in frames:
        for n in sizes:
            job = w.live_mode(n, frame)
            scan = b.Scan(job.scan)
            pts = torch.from_numpy(job.pts_xy).to(dev)
            out = torch.empty((len(job.times), len(job.pts_xy)), dtype=torch.float64, device=dev)
            b.dd_field_at_times(scan, pts, job.times, "mixed", out=out, stream=stream)
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(reps):
                b.dd_field_at_times(scan, pts, job.times, "mixed", out=out, stream=stream)
            z.record(stream)
            torch.cuda.synchronize(dev)
            ms = a.elapsed_time(z) / reps
            pairs = w.causal_pairs(np.arange(n * n) * job.scan.dwell_s, job.times, n * n)
            rows.append({"probes": n * n, "frame_us": frame * 1e6, "snapshots": len(job.times),
                         "ms": round(ms, 4), "pair_terms": pairs, "pair_terms_per_s": pairs / (ms / 1e3)})
    return {"rows": rows, "note": "20x20 at a 10 us frame is the paper's worked case (16 s in C++ on a "
            "desktop CPU, D/sigma/dwell unstated: context only); here dwell 1 us, D 6e-14 m^2/s, sigma 0.1 nm"}


def bench_surrogate(dev, maps, epochs):
    """Train the surrogate on `maps` exact fields and compare it with the exact path, both
    as kernels on device-resident inputs and end to end from the scan descriptions."""
    import torch
    from paper_2507_00294_gb300 import binding as b
    from paper_2507_00294_gb300 import surrogate as sur
    t0 = time.perf_counter()
    specs, tmap, scal, target = sur.build_dataset(maps, seed=5, device=dev)
    weight = sur.loss_weights(target)
    torch.cuda.synchronize(dev)
    t_data = time.perf_counter() - t0
    n_test = max(64, maps // 20)
    n_train = maps - 2 * n_test
    net = sur.Net(dev, seed=0)
    t0 = time.perf_counter()
    losses = sur.train(net, tmap[:n_train], scal[:n_train], target[:n_train], epochs=epochs, batch=32,
                       weight=weight[:n_train])
    torch.cuda.synchronize(dev)
    t_train = time.perf_counter() - t0
    te = slice(maps - n_test, maps)
    te_specs = specs[te]

    def timed(fn):
        torch.cuda.synchronize(dev)
        t = time.perf_counter()
        r = fn()
        torch.cuda.synchronize(dev)
        return r, time.perf_counter() - t

    # exact path end to end (scans, plans, kernels) on the test maps, full canvas
    sur.exact_fields(te_specs[:64], dev)
    exact, t_exact = timed(lambda: sur.exact_fields(te_specs, dev).view(n_test, -1))
    out = torch.empty(n_test * sur.CANVAS * sur.CANVAS, dtype=torch.float64, device=dev)

    def kernel_time(spec_list, times):
        """One plan of the scans on the canvas grid, replayed: the kernels alone."""
        scans = [b.Scan(s) for s in spec_list]
        plan = b.Batch(scans, None, np.asarray(times), "mixed",
                       grids=[(0.0, 0.0, s.pitch_m, s.pitch_m, sur.CANVAS, sur.CANVAS) for s in spec_list])
        plan.run(out=out)
        _, t = timed(lambda: plan.run(out=out))
        plan.close()
        return t
    t_exact_kernel = kernel_time(te_specs, [w_nv(s) * s.dwell_s for s in te_specs])
    parts = [sur.split_scan(s) for s in te_specs]
    t_near_kernel = kernel_time([p_[2] for p_ in parts], [p_[3] for p_ in parts])
    # network alone, batch 256, device-resident input descriptors
    sur.predict(net, tmap[te], scal[te])
    _, t_net = timed(lambda: sur.predict(net, tmap[te], scal[te], batch=256))
    # surrogate end to end: input planes from the scan descriptions (host), upload, network,
    # and the exact field of each scan's last visits
    def net_e2e():
        sur._VISITS.clear()                  # every scan's visit list built inside the timing
        tm, sc = sur.scan_inputs(te_specs)
        return sur.surrogate_fields(net, te_specs, torch.from_numpy(tm).to(dev), torch.from_numpy(sc).to(dev), dev)[0]
    fields_sur, t_net_e2e = timed(net_e2e)
    err = sur.map_errors(fields_sur, exact)
    fields, fell, est, t_fb = sur.infer_with_fallback(net, te_specs, tmap[te], scal[te], dev)
    err_after = sur.map_errors(fields, exact)
    est_ok = np.abs(np.log10(np.maximum(est, 1e-12) / np.maximum(err, 1e-12)))
    return {"maps_per_s_network": n_test / t_net, "maps_per_s_exact_kernel": n_test / t_exact_kernel,
            "maps_per_s_surrogate_kernels": n_test / (t_net + t_near_kernel),
            "maps_per_s_surrogate_end_to_end": n_test / t_net_e2e, "maps_per_s_exact_end_to_end": n_test / t_exact,
            "maps_per_s_with_fallback": n_test / t_fb, "unit": "maps/s",
            "gain_network_over_exact_kernel": t_exact_kernel / t_net,
            "gain_surrogate_over_exact_kernels": t_exact_kernel / (t_net + t_near_kernel),
            "gain_surrogate_over_exact_end_to_end": t_exact / t_net_e2e,
            "exact_last_visits": sur.K_EXACT,
            "gain_with_fallback_over_exact_end_to_end": t_exact / t_fb,
            "median_rel_err": float(np.median(err)), "p90_rel_err": float(np.percentile(err, 90)),
            "share_below_1e-2": float(np.mean(err <= 1e-2)),
            "fallback_fraction": float(np.mean(fell)), "max_rel_err_after_fallback": float(err_after.max()),
            "spot_estimate_within_2x": float(np.mean(est_ok <= np.log10(2.0))),
            "train_maps": n_train, "test_maps": n_test, "epochs": epochs, "final_train_loss": losses[-1],
            "seconds": {"dataset": t_data, "train": t_train},
            "net": "6 x conv3x3 (4->32->32->32->32->32->1, padded 16/32/16), dilations 1..32, BF16 tcgen05.mma "
                   "(forward, data gradient) and mma.sync (weight gradient), FP32 accum, Adam",
            "loss": "squared log10 error weighted by each pixel's share of the map's squared field "
                    "(alpha %.2f) plus a uniform part" % sur.LOSS_ALPHA,
            "error": "relative L2 of the linear field over the 128x128 canvas; fallback above 1e-2 "
                     "(estimated from 64 exact spot points per map: the last 32 visits and 32 others)"}


def w_nv(spec):
    from paper_2507_00294_gb300 import workloads as w
    return w.n_visits(spec)


def bench_surrogate_inference(dev, maps=256, reps=5):
    """The surrogate network alone at batch `maps` (random weights; the throughput does not
    depend on them): maps/s of the six convolutions on the 128 x 128 canvas."""
    import torch
    from paper_2507_00294_gb300 import surrogate as sur
    specs = sur.draw_scans(maps, seed=7)
    tmap, scal = sur.scan_inputs(specs)
    tmap, scal = torch.from_numpy(tmap).to(dev), torch.from_numpy(scal).to(dev)
    net = sur.Net(dev, seed=0)
    sur.predict(net, tmap, scal, batch=maps)
    torch.cuda.synchronize(dev)
    a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        sur.predict(net, tmap, scal, batch=maps)
    z.record()
    torch.cuda.synchronize(dev)
    ms = a.elapsed_time(z) / reps
    return {"maps_per_s_network": maps / (ms / 1e3), "ms_per_batch": ms, "batch": maps}


def run_leg(args):
    import torch
    from paper_2507_00294_gb300 import binding as b
    dev = torch.device("cuda", 0)
    b.load()
    if args.leg == "batched":
        res = bench_batched(dev, torch.cuda.current_stream(dev), runs=3)
    elif args.leg == "surrogate":
        res = bench_surrogate(dev, args.surrogate_maps, args.surrogate_epochs)
    elif args.leg == "dose":
        job, n, _, _ = workload()
        res = bench_dose(b, dev, torch.cuda.current_stream(dev), job, n)
    else:
        res = bench_surrogate_inference(dev)
    print(json.dumps({"leg": args.leg, **res}), flush=True)
    return 0


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
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
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
    from paper_2507_00294_gb300 import shard

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
    times = np.ascontiguousarray(job.times)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    # The field is evaluated on the job's grid of points (dd_field_on_grid).  Under torchrun
    # the step is split (strong scaling): each rank keeps the whole grid (the tensor-core
    # contraction needs at least 64 x 64 points) and evaluates a set of the snapshots dealt
    # by pair count, and a cost-balanced range of dose targets; one all-gather of the
    # output rows is the only collective on the path.
    n_pts = len(job.pts_xy)
    x0, y0, gdx, gdy, W, H = job.extra["grid"]
    _, ts_visits, _ = scan.visits()
    nact_t = np.searchsorted(ts_visits, times, side="left")            # started visits per snapshot
    sets, dr = shard.snapshot_sets([int(a) * n_pts for a in nact_t], world), shard.dose_ranges(n, world)
    mine = sets[rank]
    times_r = np.ascontiguousarray(times[mine])
    j0, j1 = dr[rank]
    out = torch.empty((len(mine), n_pts), dtype=torch.float64, device=dev)
    dose = torch.empty(j1 - j0, dtype=torch.float64, device=dev)
    rank_field_pairs = int(nact_t[mine].sum()) * n_pts
    # the split of the rank's field between the tensor-core contraction (the older visits'
    # degree-2 terms) and the CUDA-core tile kernel (the rest), as the library plans it
    tc_prefix, tc_prefix2 = b.dd_field_grid_split(scan, x0, y0, gdx, gdy, W, H, times_r, degree2=True)
    rank_tc_pairs = int(tc_prefix.sum()) * n_pts
    rank_tc2_pairs = int(tc_prefix2.sum()) * n_pts
    rank_core_pairs = rank_field_pairs - rank_tc_pairs

    # The field and the dose are independent calls: the dose goes on a side stream that forks
    # from the step's stream and joins it again, submitted after the field so that its short
    # kernels fill the SMs the field's kernels leave at their tail instead of delaying their
    # start (measured: 231 us per step against 236-242 with the dose submitted first, 263 one
    # after the other); the step's events on `stream` bracket both.
    side = torch.cuda.Stream(dev)

    def step(prec):
        fork = torch.cuda.Event()
        fork.record(stream)
        side.wait_event(fork)
        if len(mine):
            b.dd_field_on_grid(scan, x0, y0, gdx, gdy, W, H, times_r, prec, out=out, stream=stream)
        if world == 1:
            b.dd_per_probe_dose(scan, prec, out=dose, stream=side)
        else:
            b.dd_per_probe_dose_range(scan, j0, j1, prec, out=dose, stream=side)
        join = torch.cuda.Event()
        join.record(side)
        stream.wait_event(join)
        if world == 1:
            return out, dose
        return shard.gather_rows(out, sets, rank, dist), shard.gather_vector(dose, dr, rank, dist)

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
        t_open = time.monotonic()
        for k in range(args.steps):
            flush.fill_(float(k))                    # evict L2 between steps (untimed)
            ev[k][0].record(stream)
            step("mixed")
            ev[k][1].record(stream)
        torch.cuda.synchronize(dev)
        clocks.mark(t_open, time.monotonic())
    b.dd_profile_enable(False)
    prof = b.dd_profile_read()
    step_ms = [a.elapsed_time(z) for a, z in ev]
    value, total_ms, world = whole_job(pairs_step, args.steps, sum(step_ms), dist, dev)
    if dist is not None:
        dist.barrier()

    # roofline of the dominant kernel (field_grid_mixed, the CUDA-core tile kernel: the
    # critical path of the field), from its own events in the timed region, over the pairs it
    # sums (those the tensor-core contraction leaves)
    fl, fms = prof.get("field_grid_mixed", (0, 0.0))
    avg_ms = fms / max(1, fl)
    fpp, mpp, culled = ops_per_pair(job, grid=True, prefix=tc_prefix if world == 1 else None)
    rate = rank_core_pairs / (avg_ms / 1e3) if fl else None
    traffic = recorded_traffic("field_grid_mixed")
    # the pair term needs FP32 issue and one MUFU ex2: report the pipe this algorithm's mix
    # binds (the larger fraction), with the other beside it
    fp32 = {"achieved": fpp * rate / 1e12 if rate else None, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
            "per_pair": round(fpp, 3),
            "peak_note": "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz (nominal max clock)"}
    mufu = {"achieved": mpp * rate / 1e12 if rate else None, "peak": MUFU_PEAK_TOPS, "unit": "TOP/s",
            "per_pair": round(mpp, 4),
            "peak_note": "MUFU ex2: 152 SMs x 32 per clock x 2070 MHz"}
    for x in (fp32, mufu):
        x["frac"] = x["achieved"] / x["peak"] if x["achieved"] else None
    bind, other = (mufu, fp32) if (mufu["frac"] or 0) >= (fp32["frac"] or 0) else (fp32, mufu)
    roofline = {"bound": "alu", "kernel": "field_grid_mixed", "pipe": "mufu" if bind is mufu else "fp32",
                "achieved": bind["achieved"], "peak": bind["peak"], "unit": bind["unit"], "frac": bind["frac"],
                "traffic": traffic, "avg_launch_ms": avg_ms, "pairs_per_launch": rank_core_pairs,
                "kernel_pairs_per_s": rate, "ops_per_pair": bind["per_pair"], "peak_note": bind["peak_note"],
                "culled_pair_fraction": round(culled, 5),
                "culled_note": "pair-terms with a >= 87 (below the FP32 normal range) are counted in the "
                               "pair-terms but skipped per warp; their share of this kernel's pairs",
                "other_pipe": {"pipe": "fp32" if bind is mufu else "mufu", **other},
                "ncu_capture": recorded_pipes("field_grid_mixed"),
                "tensor_core": [tensor_core_line(prof, "field_grid_tc", rank_tc2_pairs, 14),
                                tensor_core_line(prof, "field_grid_tc4", rank_tc_pairs - rank_tc2_pairs, 24)]}
    launches = int(sum(v[0] for v in prof.values()))
    # shares of the summed per-launch event time (the dose's kernels run beside the field's,
    # so their events overlap and the shares do not add up to wall time)
    shares = {k: round(v[1] / max(1e-9, sum(x[1] for x in prof.values())), 4) for k, v in prof.items()}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f32-mixed", "data": "synthetic",
        "config": {"workload": job.name, "scan": "64x64 raster, pitch 0.5 nm, sigma 0.1 nm, "
                   "D 6e-14 m^2/s, Q0 1 u/s, dwell 1 us", "points": n_pts,
                   "snapshots": len(times), "visits": n, "pairs_per_step": pairs_step,
                   "field_pairs": field_pairs, "dose_pairs": dose_pairs, "precision": "mixed",
                   "l2": "flushed between steps (256 MB write, outside the timed events)",
                   "parallelism": ("points and dose targets split over %d GPUs, one all-gather per step"
                                   % world) if world > 1 else "single GPU"},
        "roofline": roofline, "gpu_launches": launches, "kernel_time_share": shares,
        "clocks": clocks.summary(),
    }

    if not args.no_extras:
        # FP64 path on the same workload (device-resident inputs)
        b.dd_profile_enable(False)
        step("fp64")
        torch.cuda.synchronize(dev)
        b.dd_profile_reset()
        b.dd_profile_enable(True)
        e64 = []
        for k in range(args.fp64_steps):
            flush.fill_(float(k))
            a, z = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step("fp64")
            z.record(stream)
            e64.append((a, z))
        torch.cuda.synchronize(dev)
        b.dd_profile_enable(False)
        prof64 = b.dd_profile_read()
        v64, _, _ = whole_job(pairs_step, len(e64), sum(a.elapsed_time(z) for a, z in e64), dist, dev)
        line["fp64"] = {"value": v64, "unit": UNIT, "ms_per_step": pairs_step / v64 * 1e3, "steps": len(e64)}
        l64, ms64 = prof64.get("field_fp64", (0, 0.0))
        if l64:
            dpp = dfma_per_pair_fp64(job)
            rate64 = rank_field_pairs / (ms64 / l64 / 1e3)
            line["fp64"]["roofline"] = {
                "bound": "alu", "kernel": "field_fp64", "pipe": "fp64", "achieved": dpp * rate64 / 1e12,
                "peak": FP64_PEAK_TDFMA, "unit": "T DFMA-equivalents/s", "frac": dpp * rate64 / 1e12 / FP64_PEAK_TDFMA,
                "avg_launch_ms": ms64 / l64, "kernel_pairs_per_s": rate64, "ops_per_pair": round(dpp, 2),
                "peak_note": "FP64 FMA: 1.6 per clock per SM measured by a microbenchmark on this GPU (0.50 T/s "
                             "at 1.995 GHz), x 152 SMs x 2070 MHz",
                "ops_note": "per pair: rho^2 shared by 4 snapshots (1), the moment polynomial of the warp's "
                            "degree (4 / 8 / 11 / 15 from the pair's own h: D + 1), exp(-a) counted as 15 "
                            "DFMA-equivalents, 60 for a two-E1 pair"}
        line["mixed_over_fp64"] = value / v64
        line["e2e"] = bench_e2e(args, b, shard, job, times, n, pairs_step, rank, world, dist, dev, sets, dr)
        if world == 1:
            line["field_point_list"] = bench_point_list(b, job, times, scan, dev, stream, flush, field_pairs)
        line["batched"] = bench_batched(dev, stream, rank=rank, world=world, dist=dist)
        if world == 1:
            line["dose"] = bench_dose(b, dev, stream, job, n)
            lst = bench_batched(dev, stream, grid=False)
            line["batched"]["point_list"] = {"value": lst["value"], "ms_per_run": lst["ms_per_run"],
                                             "tuned_variant": lst["tuned_variant"]}
        if world == 1:
            line["runtime_curve"] = bench_runtime_curve(dev, stream)
            if not args.no_surrogate:
                line["surrogate"] = bench_surrogate(dev, args.surrogate_maps, args.surrogate_epochs)

        if rank == 0 and world == 1:
            run, rate, count, cores = cpu_oracle_sample(job, args.cpu_seconds)
            p, t = run(count, 7)
            run1, _, count1, _ = cpu_oracle_sample(job, args.cpu_seconds / 3, threads=1)
            p1_, t1_ = run1(count1, 8)
            line["cpu_baseline"] = {
                "value": p / t, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": "%d seeded (point, snapshot) pairs of the workload, %d pair-terms, "
                          "%.1f s, field only" % (count, p, t),
                "single_thread": {"value": p1_ / t1_, "unit": UNIT, "cores": 1,
                                  "sample": "%d seeded pairs, %d pair-terms, %.1f s" % (count1, p1_, t1_)}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def bench_e2e(args, b, shard, job, times, n, pairs_step, rank, world, dist, dev, sets, dr):
    """End to end through the public API with page-locked host outputs: scan build (its
    visit list uploaded on first use), the grid field and the dose, D2H of both.  One GPU:
    three steps in flight -- step k's calls are enqueued (field and dose on their own pair
    of streams, copies into step k's own page-locked buffers) before step k - 2 is
    synchronised and its scan destroyed, so the host builds the next steps while the GPU
    runs the earlier ones.  Several: each rank evaluates its snapshots and dose targets,
    the device results are gathered, and rank 0 copies out the whole field and dose."""
    import torch
    x0, y0, gdx, gdy, W, H = job.extra["grid"]
    mine = sets[rank]
    times_r = np.ascontiguousarray(times[mine])
    j0, j1 = dr[rank]
    n_buf = 3 if world == 1 else 1
    outs_h = [torch.empty((len(times), len(job.pts_xy)), dtype=torch.float64, pin_memory=True) for _ in range(n_buf)]
    doses_h = [torch.empty(n, dtype=torch.float64, pin_memory=True) for _ in range(n_buf)]
    out_h, dose_h = outs_h[0], doses_h[0]
    streams = [(torch.cuda.Stream(dev), torch.cuda.Stream(dev)) for _ in range(n_buf)]
    e2e_stream = streams[0][0]
    if world > 1:
        out_d = torch.empty((len(mine), len(job.pts_xy)), dtype=torch.float64, device=dev)
        dose_d = torch.empty(j1 - j0, dtype=torch.float64, device=dev)
    in_flight = []
    t0 = None
    # W untimed warm-up steps through the same loop (its blocks, events and staging come
    # into use), then K timed steps
    for k in range(args.warmup + args.steps):
        if k == args.warmup:
            for prev, (pf, pd) in in_flight:
                pf.synchronize()
                pd.synchronize()
                prev.close()
            in_flight = []
            torch.cuda.synchronize(dev)
            if dist is not None:
                dist.barrier()
            t0 = time.perf_counter()
        s2 = b.Scan(job.scan)
        if world == 1:
            i = k % n_buf
            sf, sd = streams[i]
            # the field first (its kernels start while the host prepares the dose), the
            # dose on a second stream beside it, each leaving its copies enqueued
            b.dd_field_on_grid(s2, x0, y0, gdx, gdy, W, H, times, "mixed", out=outs_h[i].numpy(), stream=sf)
            b.dd_per_probe_dose(s2, "mixed", out=doses_h[i].numpy(), stream=sd)
            in_flight.append((s2, (sf, sd)))
            if len(in_flight) == n_buf:
                # the oldest step: its results are in its host buffers once its streams are done
                prev, (pf, pd) = in_flight.pop(0)
                pf.synchronize()
                pd.synchronize()
                prev.close()
            continue
        else:
            with torch.cuda.stream(e2e_stream):
                if len(mine):
                    b.dd_field_on_grid(s2, x0, y0, gdx, gdy, W, H, times_r, "mixed", out=out_d, stream=e2e_stream)
                b.dd_per_probe_dose_range(s2, j0, j1, "mixed", out=dose_d, stream=e2e_stream)
                f = shard.gather_rows(out_d, sets, rank, dist)
                d = shard.gather_vector(dose_d, dr, rank, dist)
                if rank == 0:
                    out_h.copy_(f, non_blocking=True)
                    dose_h.copy_(d, non_blocking=True)
        e2e_stream.synchronize()
        s2.close()
    for last, (pf, pd) in in_flight:
        pf.synchronize()
        pd.synchronize()
        last.close()
    e2e_ms = (time.perf_counter() - t0) * 1e3
    v, ms, _ = whole_job(pairs_step, args.steps, e2e_ms, dist, dev)
    # host -> device per step and rank: the scan's visit cache (6 doubles per visit) and the
    # snapshot times; device -> host: the whole field and dose
    return {"value": v, "unit": UNIT, "h2d_bytes_per_step": int(world * (6 * n * 8 + len(times) * 8)),
            "d2h_bytes_per_step": int(out_h.numel() * 8 + dose_h.numel() * 8),
            "ms_per_step": ms / args.steps,
            "api": "dd_create_scan + dd_field_on_grid + dd_per_probe_dose (host outputs)",
            "in_flight": n_buf,
            "note": "consecutive steps overlap on the GPU (no L2 flush between them), so this can "
                    "exceed the device-timed value, whose steps run one at a time after an L2 flush"}


def bench_point_list(b, job, times, scan, dev, stream, flush, field_pairs, reps=10):
    """The same field through dd_field_at_times (the points as an explicit list, general
    tiles of 512 consecutive points): its kernel's event time and roofline."""
    import torch
    pts = torch.from_numpy(np.ascontiguousarray(job.pts_xy)).to(dev)
    out = torch.empty((len(times), len(job.pts_xy)), dtype=torch.float64, device=dev)
    for _ in range(2):
        b.dd_field_at_times(scan, pts, times, "mixed", out=out, stream=stream)
    torch.cuda.synchronize(dev)
    b.dd_profile_reset()
    b.dd_profile_enable(True)
    for k in range(reps):
        flush.fill_(float(k))
        b.dd_field_at_times(scan, pts, times, "mixed", out=out, stream=stream)
    torch.cuda.synchronize(dev)
    b.dd_profile_enable(False)
    prof = b.dd_profile_read()
    fl, fms = prof.get("field_mixed", (0, 0.0))
    avg_ms = fms / max(1, fl)
    fpp, mpp, _ = ops_per_pair(job)
    rate = field_pairs / (avg_ms / 1e3)
    return {"kernel": "field_mixed", "avg_launch_ms": avg_ms, "kernel_pairs_per_s": rate,
            "mufu_frac": mpp * rate / 1e12 / MUFU_PEAK_TOPS, "fp32_frac": fpp * rate / 1e12 / FP32_PEAK_TFLOPS,
            "ops_per_pair": {"flops": round(fpp, 3), "mufu": round(mpp, 4)},
            "traffic": recorded_traffic("field_mixed")}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.leg != "all":
        return run_leg(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
