"""Work split of the field and the dose across ranks (one process per GPU).

The paper runs the cumulative sum of Eq. 5 as independent tasks, each over a subset of
the probe positions, with the load balanced across threads (Sec. 3).  Every (point,
snapshot) output and every dwell-start dose is an independent sum, so the same split
carries over to several GPUs with no exchange inside the computation:

  * the field: each rank takes a contiguous range of the evaluation points (whole point
    tiles of the field kernel, 512 points) for every snapshot -- or, on a grid of points,
    a set of the snapshots for every point (each rank keeps the whole grid, which the
    tensor-core contraction needs: at least 64 x 64 points), dealt by pair count;
  * the dose: each rank takes a contiguous range of target visits; visit j costs about j
    pair terms, so the ranges are cut where the triangle's area is split evenly;
  * a batch of scans: scans are dealt to ranks longest-first (LPT) by pair count.

The probe list is replicated (each rank builds the same scan from its description).  One
gather of the output rows at the end is the only collective.  This module holds the
partition and gather logic only; the computation on each rank is the library's.
"""
import math

POINT_TILE = 512          # points per CTA tile of the field kernel (128 threads x 4 points)
DOSE_TILE = 256           # targets per CTA tile of the dose kernel


def point_ranges(n_pts, world, align=POINT_TILE):
    """Contiguous [p0, p1) per rank, whole tiles of `align` points, as even as tiles allow."""
    tiles = (int(n_pts) + align - 1) // align
    out = []
    for r in range(world):
        t0 = (tiles * r) // world
        t1 = (tiles * (r + 1)) // world
        out.append((min(n_pts, t0 * align), min(n_pts, t1 * align)))
    return out


def snapshot_sets(costs, world):
    """The snapshots of each rank (ascending indices) with about equal total cost
    (costs[j]: the pair count of snapshot j, its started visits times the points): the
    longest-processing-time-first deal of lpt_assign, within 4/3 of the best split (a
    contiguous cut leaves up to half the costliest snapshot's cost of imbalance)."""
    return lpt_assign(list(costs), world)


def dose_ranges(n_visits, world, align=DOSE_TILE):
    """Contiguous [j0, j1) per rank with about equal pair counts: the dose of visit j sums
    j earlier visits, so the work below j grows as j^2 / 2 and rank r's range ends at
    n sqrt((r + 1) / world), rounded to whole target tiles."""
    n = int(n_visits)
    cuts = [0]
    for r in range(1, world):
        c = int(round(n * math.sqrt(r / world) / align)) * align
        cuts.append(min(n, max(cuts[-1], c)))
    cuts.append(n)
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def lpt_assign(costs, world):
    """Longest-processing-time-first: scans in falling cost order, each to the rank with the
    least work so far (ties to the lower rank).  Returns the scan indices of each rank, in
    ascending order."""
    order = sorted(range(len(costs)), key=lambda k: (-costs[k], k))
    load = [0] * world
    parts = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(k)
        load[r] += costs[k]
    return [sorted(p) for p in parts]


def gather_columns(local, ranges, rank, dist):
    """All-gather of per-rank column blocks: local [rows, p1 - p0] of this rank's range
    -> [rows, total] on every rank.  Blocks are padded to the widest range for the
    collective (all_gather needs equal shapes) and cut back afterwards."""
    import torch
    world = len(ranges)
    rows = local.shape[0]
    width = max(p1 - p0 for p0, p1 in ranges)
    buf = torch.zeros((rows, width), dtype=local.dtype, device=local.device)
    buf[:, :local.shape[1]] = local
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf.contiguous())
    return torch.cat([parts[r][:, :ranges[r][1] - ranges[r][0]] for r in range(world)], dim=1)


def gather_rows(local, sets, rank, dist):
    """All-gather of per-rank rows: local [len(sets[rank]), cols], the rows (snapshots)
    sets[rank] of the output -> [total, cols] on every rank, each rank's rows put back at
    their indices (blocks padded to the largest set for the collective)."""
    import torch
    world = len(sets)
    cols = local.shape[1]
    total = sum(len(x) for x in sets)
    height = max(1, max(len(x) for x in sets))
    buf = torch.zeros((height, cols), dtype=local.dtype, device=local.device)
    buf[:local.shape[0]] = local
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf.contiguous())
    out = torch.empty((total, cols), dtype=local.dtype, device=local.device)
    for r in range(world):
        if sets[r]:
            idx = torch.as_tensor(sets[r], dtype=torch.long, device=local.device)
            out[idx] = parts[r][:len(sets[r])]
    return out


def gather_vector(local, ranges, rank, dist):
    """All-gather of per-rank pieces of a vector: local [j1 - j0] -> [total] on every rank."""
    return gather_columns(local.reshape(1, -1), ranges, rank, dist)[0]


def grid_field_and_dose(rank, world, snapshot_costs, n_visits, field_fn, dose_fn, dist=None):
    """The same with the field split by snapshots (a grid of points kept whole on every
    rank): field_fn(snaps) -> [len(snaps), n_pts] tensor of the snapshots `snaps`."""
    sets = snapshot_sets(snapshot_costs, world)
    dr = dose_ranges(n_visits, world)
    j0, j1 = dr[rank]
    field = field_fn(sets[rank])
    dose = dose_fn(j0, j1)
    if dist is None or world == 1:
        return field, dose
    return gather_rows(field, sets, rank, dist), gather_vector(dose, dr, rank, dist)


def field_and_dose(rank, world, n_pts, n_visits, field_fn, dose_fn, dist=None):
    """One rank's share of the field at every snapshot and of the dwell-start dose, then
    the gather: field_fn(p0, p1) -> [n_t, p1 - p0] tensor, dose_fn(j0, j1) -> [j1 - j0]
    tensor.  Returns (field [n_t, n_pts], dose [n_visits]) on every rank (the local pieces
    when world == 1 or dist is None)."""
    pr = point_ranges(n_pts, world)
    dr = dose_ranges(n_visits, world)
    p0, p1 = pr[rank]
    j0, j1 = dr[rank]
    field = field_fn(p0, p1)
    dose = dose_fn(j0, j1)
    if dist is None or world == 1:
        return field, dose
    return gather_columns(field, pr, rank, dist), gather_vector(dose, dr, rank, dist)
